/*
 * hbugks.h — C ABI of the GB300 HB-UGKS library.
 *
 * The library advances the time-domain harmonic balance unified gas-kinetic scheme (HB-UGKS) of
 * Zhu, Wu, Wei, Xu, "A Time-Domain Harmonic Balance Unified Gas-Kinetic Scheme for Temporally Periodic
 * Flows Across all Knudsen Regimes" (arXiv 2605.03479), on one GPU: one pseudo-time iteration updates
 * every cell, discrete velocity and sub-time level of a 2-D cavity (Sec 2.2 - 2.4).
 *
 * Units used throughout (Sec 3.1.1): lengths in cavity heights (the Knudsen number of Eq. def_Kn is
 * taken with H = 1), velocities in sqrt(2 R T0), densities in rho0, temperatures in T0.  So R T0 = 1/2,
 * lambda = 1/(2RT) = 1/T, and the Strouhal number of Eq. def_St equals the angular frequency omega.
 *
 * Memory ownership:
 *   - All device memory is owned by the caller: hbugks_workspace_bytes() says how much one handle needs,
 *     the caller allocates it (for example with PyTorch) and passes it to hbugks_create().  The library
 *     never allocates or frees device memory.  The workspace must stay allocated until hbugks_destroy().
 *   - Host arrays passed in (meshes, velocity grids) are copied during hbugks_create(); the caller may free
 *     them afterwards.  Host output buffers are owned by the caller.
 * Streams: all work is enqueued on the CUDA stream given to hbugks_create() (NULL = legacy default stream).
 *   Calls that return host data synchronise that stream before returning.
 * Errors: every call returns an hbugks_status; no C++ exception or abort crosses the ABI.  A handle is not
 *   thread safe; distinct handles are independent.
 * Layouts of host state arrays (the "canonical" layout, FP64):
 *   W[level][cell][4]            conservative variables (rho, rho U, rho V, rho E), Eq. moment
 *   h[level][cell][velocity]     reduced distribution h of Eq. reduced_h;  b likewise (Eq. reduced_b)
 *   cell = j * nx + i (i along x), velocity = jv * nu + iu (tensor grid, u index fastest).
 */
#ifndef HBUGKS_H
#define HBUGKS_H

#include <stddef.h>

#if defined(__GNUC__)
#define HBUGKS_API __attribute__((visibility("default")))
#else
#define HBUGKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hbugks_solver* hbugks_t;

typedef enum {
    HBUGKS_OK = 0,
    HBUGKS_NOT_CONVERGED = 1,   /* warning: the iteration budget ran out before the residual target */
    HBUGKS_EINVAL = -1,         /* invalid argument (sizes, pointers, unsupported combination) */
    HBUGKS_ECUDA = -2,          /* a CUDA runtime call failed */
    HBUGKS_ENOMEM = -3,         /* workspace smaller than hbugks_workspace_bytes(), or host memory exhausted */
    HBUGKS_DIVERGED = -4,       /* a residual became NaN/Inf or exceeded 1e10 */
    HBUGKS_TIMEOUT = -5         /* a bounded device-side wait ran out (500 ms for a bulk copy); the iteration
                                   in which it happened left the state unchanged */
} hbugks_status;

/* Non-uniform Cartesian mesh of the cavity: node coordinates, nx + 1 and ny + 1 increasing values
 * (finite-volume cells of Eq. fv_W; cell volume = dx dy, face lengths dy (x-normal) and dx (y-normal)). */
typedef struct {
    int nx, ny;
    const double* xnodes;
    const double* ynodes;
} hbugks_mesh;

/* Tensor-product discrete velocity grid {u_alpha, w_alpha} (Sec 2.1): nodes u[nu] with weights wu[nu] and
 * v[nv] with weights wv[nv]; the weight of (u_iu, v_jv) is wu[iu] * wv[jv].  umax, vmax: the truncation
 * bounds of velocity space used in the convective spectral radius (Eq. nu_conv). */
typedef struct {
    int nu, nv;
    const double* u;
    const double* wu;
    const double* v;
    const double* wv;
    double umax, vmax;
} hbugks_vgrid;

/* Physical and numerical parameters of one case. */
typedef struct {
    double kn;           /* Knudsen number (Eq. def_Kn, VSS with w_vss, alpha_vss) */
    double st;           /* Strouhal number (Eq. def_St) */
    double pr;           /* Prandtl number of the Shakhov model (Eq. shakhov); 1 gives BGK */
    double cfl;          /* CFL number of the local pseudo-time step (Eq. dt_hb) */
    double w_vss;        /* viscosity index: mu = mu(T0) (T/T0)^w_vss */
    double alpha_vss;    /* VSS angular scattering parameter */
    double gamma;        /* ratio of specific heats in the sound speed of Eq. nu_conv */
    int n_harmonics;     /* N_H >= 0; N_T = 2 N_H + 1 sub-time levels (Eq. collocation_points) */
    int face_step;       /* 0: min(dG_L, dG_R); 1: harmonic mean (Eq. dt_face) */
    int precision;       /* 0: FP64 everywhere; 1: FP32-split (distribution stored as FP32 deviation from
                            the T0 Maxwellian, FP64 moments, interface parameters, macro update, residual) */
    int td_steps;        /* 0: harmonic balance (the pseudo-time iteration of Sec 2.4).  > 0: explicit
                            time-domain UGKS on the same fluxes and walls, the scheme the paper compares
                            HB-UGKS against (Sec 3.1, Eq. benchmark_residuals): requires n_harmonics = 0 and
                            st > 0; every iteration is one physical step dt = 2 pi / (st td_steps) (td_steps
                            steps per forcing period) with that global step in place of the local ones, and
                            the walls at the phase of the step's midpoint, 2 pi (s + 1/2) / td_steps for the
                            s-th step of a period counted from the iteration count. */
    int spectral_implicit; /* 0: the spectral source at the old pseudo-time iterate, as printed in Eqs. fv_W and
                            fv_h (forward Euler; it amplifies the modes the source rotates by about
                            (dG omega k)^2 / 2 per iteration).  1: at the new iterate, solved across the levels
                            of each cell (and velocity): the same fixed point, those modes damped.  The paper
                            names an implicit HB scheme as future work (Sec 4); this is that choice for the
                            spectral source only. */
} hbugks_physics;

/* Wall waveform (Eqs. bc_vel, bc_temp): state at level n = mean + Re(amp exp(i 2 pi n / N_T)),
 * amp = re + i im, for the wall velocity (U, V) and temperature T (in T0). */
typedef struct {
    double u_mean, v_mean, T_mean;
    double u_re, u_im, v_re, v_im, T_re, T_im;
} hbugks_wall;

/* One cavity case.  walls[0] bottom (y = y0), [1] right (x = x_nx), [2] top (y = y_ny), [3] left (x = x0). */
typedef struct {
    hbugks_mesh mesh;
    hbugks_vgrid vgrid;
    hbugks_physics phys;
    hbugks_wall walls[4];
} hbugks_case;

/* Device workspace (bytes) a handle for these cases needs; 0 if the cases are invalid.
 * All cases of one handle must have the same precision.  Invalid: a non-finite or non-positive size, weight,
 * Kn, CFL, gamma, Pr, VSS alpha or speed bound; non-finite nodes or wall parameters; nodes not increasing; a
 * wall temperature <= 0 on some level; N_T > 15; or a case so large that its per-face or per-cell expm1
 * tables ((nf or 2 nc) x N_T x (nu + nv) elements) exceed 2^31 - 1 elements, the kernels' 32-bit offsets. */
HBUGKS_API size_t hbugks_workspace_bytes(int ncases, const hbugks_case* cases);

/* Create a handle for `ncases` cases (a batch of one or more uneven cases iterated together).
 * d_workspace: caller-owned device memory, 256-byte aligned, at least hbugks_workspace_bytes() bytes.
 * cuda_stream: a cudaStream_t (or NULL).  The state is set to the uniform rest Maxwellian
 * (rho = 1, U = V = 0, T = 1) on every level.  On success *out receives the handle. */
HBUGKS_API hbugks_status hbugks_create(int ncases, const hbugks_case* cases, void* d_workspace, size_t bytes,
                            void* cuda_stream, hbugks_t* out);

/* Release the handle's host resources (captured graphs, host copies).  Does not free the workspace. */
HBUGKS_API void hbugks_destroy(hbugks_t h);

/* Replace the wall waveform of one wall of one case (takes effect at the next iteration). */
HBUGKS_API hbugks_status hbugks_set_wall(hbugks_t h, int case_index, int wall, const hbugks_wall* w);

/* Uniform Maxwellian state (reduced h, b of Eq. maxwellian with K = 1) with density rho, velocity (u, v)
 * and temperature T on every level of one case (case_index = -1: all cases); W = its continuous moments. */
HBUGKS_API hbugks_status hbugks_init_uniform(hbugks_t h, int case_index, double rho, double u, double v, double T);

/* Copy a state in (set) or out (get), canonical FP64 layout, host pointers (see top of file).
 * Sizes in doubles: W nt*nc*4, h and b nt*nc*nu*nv each.  get: hh and bb may both be NULL to read W only. */
HBUGKS_API hbugks_status hbugks_set_state(hbugks_t h, int case_index, const double* W, const double* hh, const double* bb);
HBUGKS_API hbugks_status hbugks_get_state(hbugks_t h, int case_index, double* W, double* hh, double* bb);

/* Run pseudo-time iterations (Sec 2.4) on every active case until each case's level-0 density residual
 * (Eq. benchmark_residuals) is <= tol_rho or max_iters iterations have run.  tol_rho <= 0 runs exactly
 * max_iters iterations.  Cases that reached the target stop iterating.  iters_done (may be NULL) receives
 * ncases values: the iterations each case ran in this call; resid_out (may be NULL) receives ncases * 4
 * values: the last residual of (rho, rho U, rho V, rho E) per case.
 * Returns HBUGKS_OK if every case reached tol_rho (or tol_rho <= 0), HBUGKS_NOT_CONVERGED otherwise,
 * HBUGKS_DIVERGED if a residual became non-finite or > 1e10. */
HBUGKS_API hbugks_status hbugks_iterate(hbugks_t h, int max_iters, double tol_rho, int* iters_done, double* resid_out);

/* Mark cases active (1) or frozen (0) for later hbugks_iterate calls; flags has ncases entries. */
HBUGKS_API hbugks_status hbugks_set_active(hbugks_t h, const int* flags);

/* Residual history of one case: the last `n` iterations' (rho, rho U, rho V, rho E) residuals, oldest
 * first, into out[n][4]; n <= 4096. */
HBUGKS_API hbugks_status hbugks_residual_history(hbugks_t h, int case_index, int n, double* out);

/* Macroscopic fields of one level from the moments of h and b (Sec 3.1.1), host out[8][nc]:
 * rho, U, V, T/T0, tau_xy (Eq. shear_stress_eval), q_x, q_y, p. */
HBUGKS_API hbugks_status hbugks_get_level_fields(hbugks_t h, int case_index, int level, double* out);

/* k-th Fourier coefficient (Eq. dft_general, 0 <= k <= N_H) of the same 8 fields: re[8][nc], im[8][nc].
 * Negative k follow from conjugate symmetry (Sec 2.2). */
HBUGKS_API hbugks_status hbugks_get_harmonic(hbugks_t h, int case_index, int k, double* re, double* im);

/* Number of iterations run on a case since its state was last set. */
HBUGKS_API long long hbugks_iteration_count(hbugks_t h, int case_index);

/* Human-readable name of a status. */
HBUGKS_API const char* hbugks_status_string(hbugks_status s);

/* Description of the CUDA error behind the last HBUGKS_ECUDA returned on the calling thread. */
HBUGKS_API const char* hbugks_cuda_error_string(void);

/* Kernel-level timing support: enqueue `n` iterations on the handle's stream without any host
 * synchronisation or residual check (for timing with CUDA events around the call).  A device-side wait that
 * runs out in these iterations is reported by the next hbugks_iterate call (HBUGKS_TIMEOUT). */
HBUGKS_API hbugks_status hbugks_enqueue_iterations(hbugks_t h, int n);

/* Kernel timing: run `n` iterations kernel by kernel (not graph-captured) with a CUDA event pair around each
 * launch on the stream the kernels run on, synchronise, and write the average milliseconds per iteration of
 * each kernel kind into ms[5]: face moments, face parameters, macro update, micro update, residual. */
HBUGKS_API hbugks_status hbugks_profile_kernels(hbugks_t h, int n, double* ms);

/* Harmonic of the macroscopic fields for callers that cannot allocate device memory.
 * Some callers cannot call cudaMalloc at all (code that runs inside an allocator-controlled runtime, or a
 * host that has already handed out every byte of device memory) and have no workspace to give a handle.
 * This entry point needs neither a handle nor a workspace: it takes a state that already lives in device
 * memory and writes the k-th Fourier coefficient (0 <= k <= (nt - 1) / 2) of the 8 fields of
 * hbugks_get_level_fields() into the caller's device buffers re[8][nx*ny] and im[8][nx*ny].
 * Inputs (device pointers, FP64, canonical layout of this header): u[nu], wu[nu], v[nv], wv[nv], and
 * h, b[nt][nx*ny][nu*nv].  Its intermediate per-level fields live in a fixed array inside the library
 * (HBUGKS_NOALLOC_MAX_DOUBLES doubles, 4 MiB, held on every device that loads the library until the
 * process exits), so it requires 8 * nt * nx * ny <= HBUGKS_NOALLOC_MAX_DOUBLES and returns HBUGKS_EINVAL
 * otherwise.  It calls no allocating CUDA or library routine.  The first call on a device (and the first after
 * the device's context has been rebuilt, for example by cudaDeviceReset) looks up that device's address of the
 * array; make that first call before any stream capture.  The array is reserved when the library's device
 * code is loaded into a context, which under CUDA's default lazy loading happens at the first call into the
 * library on that device (this entry point, or hbugks_create): that first call must find about 4 MiB of
 * device memory still free, and fails with HBUGKS_ECUDA otherwise.  All calls share the
 * one array, so calls whose work overlaps on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller.  The paper has no counterpart of this entry point. */
#define HBUGKS_NOALLOC_MAX_DOUBLES (1 << 19)
HBUGKS_API hbugks_status hbugks_harmonic_noalloc(int nx, int ny, int nu, int nv, const double* u, const double* wu,
                                                 const double* v, const double* wv, int nt, const double* h,
                                                 const double* b, int k, double* re, double* im, void* cuda_stream);

/* Variant of the micro-update kernel of a case: its tile (tx x ty cells per CTA, all levels) and vpl, the
 * blocks of 32 velocities per CTA (1, or 2: each lane then updates one velocity of each of two blocks of the
 * same sign class, sharing the per-cell and per-face indices and parameters between them).  The variants are
 * 4x4, 4x2, 2x2 and 8x4 with vpl 1, and 4x2 with vpl 2, which needs single precision and sign classes that
 * each hold an even number of velocity blocks.  hbugks_create() picks one per case by timing every variant the
 * case can run on the case itself (autotuning, cached per process by mesh size, velocity grid, level count,
 * precision and SM count).  get: the variant of case `case_index`.  set: pin one, for example to reproduce a
 * run exactly; HBUGKS_EINVAL if it is not one of these, needs more shared memory than a CTA may have, or needs
 * what the case lacks.  Every variant gives bitwise the same iterate; the state is unchanged and the iteration
 * graphs are rebuilt.  The tile-shape pair is the same with vpl = 1 (set) or any vpl (get).  The paper has no
 * counterpart (a GPU tuning choice). */
HBUGKS_API hbugks_status hbugks_get_micro_variant(hbugks_t h, int case_index, int* tx, int* ty, int* vpl);
HBUGKS_API hbugks_status hbugks_set_micro_variant(hbugks_t h, int case_index, int tx, int ty, int vpl);
HBUGKS_API hbugks_status hbugks_get_tile_shape(hbugks_t h, int case_index, int* tx, int* ty);
HBUGKS_API hbugks_status hbugks_set_tile_shape(hbugks_t h, int case_index, int tx, int ty);

/* Copy the state of case src_case of handle src into case dst_case of handle dst, converting between the two
 * handles' precisions.  The use it serves is mixed-precision refinement: iterate an FP32-split handle close to
 * convergence, copy its state into an FP64 handle of the same case, and let a few FP64 iterations remove the
 * rounding floor of the FP32 storage (the fixed point is the FP64 one).  Both cases must have the same mesh,
 * velocity grid and N_T (HBUGKS_EINVAL otherwise); walls and physics are those of dst.  Runs after all work
 * enqueued on src's stream, on dst's stream, and resets dst's iteration count for that case.  Both handles must
 * live on the current device.  The paper has no counterpart (a precision choice of this library). */
HBUGKS_API hbugks_status hbugks_copy_state(hbugks_t dst, int dst_case, hbugks_t src, int src_case);

/* Failure-path test hook.  Every device-side wait of the iteration kernels (a bulk copy into shared memory
 * completing on an mbarrier) is bounded by elapsed time: on expiry the kernel sets the handle's error word, its
 * CTA waits (bounded) for the copies it has issued and exits, every later kernel of the iteration returns
 * without work, and hbugks_iterate returns HBUGKS_TIMEOUT after the chunk of iterations in which it happened,
 * with the state of the last completed iteration.  This call makes the micro-update kernel of the next
 * iteration report its first wait as expired right after that wait has completed, so the whole failure path
 * runs without any copy actually failing.  hbugks_iterate clears the hook together with the error word when it
 * returns HBUGKS_TIMEOUT; the next call iterates normally.  The paper has no counterpart (failure handling). */
HBUGKS_API hbugks_status hbugks_test_expire_wait(hbugks_t h);

/* Number of kernel launches one iteration enqueues for this handle. */
HBUGKS_API int hbugks_launches_per_iteration(hbugks_t h);

/* How hbugks_iterate and hbugks_enqueue_iterations run their iterations.  mode 0 (default): one launch of a
 * CUDA graph whose conditional while node repeats one iteration and a one-thread loop test until the count is
 * spent, every case has converged or diverged, or a device wait has failed; the host reads the statuses once, at
 * the end.  mode 1: graphs of 16 iterations launched from the host, which reads the statuses after each (the
 * earlier design, kept for comparison).  Both run the same kernels and give bitwise the same state.  The paper
 * has no counterpart. */
HBUGKS_API hbugks_status hbugks_set_loop_mode(hbugks_t h, int mode);

#ifdef __cplusplus
}
#endif

#endif /* HBUGKS_H */
