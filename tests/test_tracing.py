"""Tracing: every C-ABI call, and every kernel stage an iteration enqueues, is an NVTX range.

An NVTX injection library of the tests (tests/nvtx_recorder.c) records the ranges of a child process; the CPU
test checks a host-only call, the GPU test a handle's whole life."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


def cuda_include():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")


@pytest.fixture(scope="module")
def recorder(tmp_path_factory):
    from paper_2605_03479_gb300 import build
    build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lib = str(tmp_path_factory.mktemp("nvtx") / "libnvtx_recorder.so")
    subprocess.check_call([cc, "-shared", "-fPIC", "-O1", "-I", cuda_include(), "-o", lib,
                           os.path.join(HERE, "nvtx_recorder.c")])
    return lib


def run_traced(recorder, tmp_path, code):
    log = tmp_path / "nvtx.log"
    env = dict(os.environ, NVTX_INJECTION64_PATH=recorder, HBUGKS_NVTX_LOG=str(log), PYTHONPATH=ROOT)
    subprocess.run([sys.executable, "-c", code], check=True, env=env, cwd=ROOT, timeout=600)
    return log.read_text().splitlines()


def balanced(lines):
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        assert depth >= 0, "pop without push"
    return depth == 0


def test_host_call_is_a_range(recorder, tmp_path):
    code = ("from paper_2605_03479_gb300 import hbugks, inputs as I\n"
            "c = I.make_case('t', 4, 8, kn=0.1, st=1.0, nh=1)\n"
            "assert hbugks.workspace_bytes([c]) > 0\n")
    lines = run_traced(recorder, tmp_path, code)
    assert lines == ["push hbugks_workspace_bytes", "pop"]


@pytest.mark.gpu
def test_handle_calls_and_kernel_stages_are_ranges(recorder, tmp_path):
    code = ("from paper_2605_03479_gb300 import hbugks as hb, inputs as I\n"
            "c = I.make_case('t', 8, 8, kn=0.1, st=1.0, nh=1, drive='shear')\n"
            "s = hb.Solver(c)\n"
            "s.iterate(3)\n"
            "s.profile_kernels(1)\n"
            "s.harmonic(0, 1)\n"
            "s.destroy()\n")
    lines = run_traced(recorder, tmp_path, code)
    pushed = [ln[5:] for ln in lines if ln.startswith("push ")]
    for name in ("hbugks_workspace_bytes", "hbugks_create", "hbugks_iterate", "hbugks_profile_kernels",
                 "hbugks_get_harmonic", "hbugks_destroy", "k1_cells", "k2_face_params", "k3_macro", "k_tables",
                 "k4_cells", "k5_finish"):
        assert name in pushed, name
    assert balanced(lines)
    # the kernel stages of the profiled iteration nest inside the profiling call
    i = lines.index("push hbugks_profile_kernels")
    inner = lines[i + 1:i + 1 + 12]
    assert inner[0] == "push k1_cells" and "push k4_cells" in inner
