/* Test instrumentation: an NVTX 3 injection library that writes every range push and pop of the process to the
 * file named by HBUGKS_NVTX_LOG, one line each ("push <name>", "pop").  A process loads it when the variable
 * NVTX_INJECTION64_PATH names it before its first NVTX call; the tests build it with the host C compiler.
 * Only the core module's RangePushA and RangePop slots are filled; every other NVTX call stays a no-op. */
#include <stdio.h>
#include <stdlib.h>

#include <nvtx3/nvToolsExt.h>

static FILE* out;

static int record_push(const char* name)
{
    if (out) {
        fprintf(out, "push %s\n", name ? name : "");
        fflush(out);
    }
    return 0;
}

static int record_pop(void)
{
    if (out) {
        fputs("pop\n", out);
        fflush(out);
    }
    return 0;
}

/* Entry point the NVTX loader looks up in the injection library: fill the core callback slots. */
int InitializeInjectionNvtx2(NvtxGetExportTableFunc_t get_table)
{
    const NvtxExportTableCallbacks* cb = (const NvtxExportTableCallbacks*)get_table(NVTX_ETID_CALLBACKS);
    NvtxFunctionTable table = 0;
    unsigned int size = 0;
    if (!cb || !cb->GetModuleFunctionTable || !cb->GetModuleFunctionTable(NVTX_CB_MODULE_CORE, &table, &size))
        return 0;
    if (size <= NVTX_CBID_CORE_RangePop) return 0;
    const char* path = getenv("HBUGKS_NVTX_LOG");
    out = path ? fopen(path, "w") : NULL;
    *table[NVTX_CBID_CORE_RangePushA] = (NvtxFunctionPointer)record_push;
    *table[NVTX_CBID_CORE_RangePop] = (NvtxFunctionPointer)record_pop;
    return 1;
}
