/*
 * pmeft.h -- C ABI of the GB300 (sm_103a) library for the screened EFTofDE
 * particle-mesh path of arXiv 2604.15434 (PySCo-EFT / ECOSMOG-EFT).
 *
 * Conventions for every entry point
 *   - Grids are n^3 arrays of double in device memory, index (k*n + j)*n + i with
 *     x (i) fastest; cell i is centred at (i + 1/2)/n in box units (box = 1,
 *     supercomoving code units of Sec. 3.1).  n must be a power of two >= 8.
 *   - Particle arrays are [3][np] doubles in device memory (rows x, y, z), positions
 *     in [0, 1).
 *   - The caller allocates and owns every input and output buffer.  The context
 *     owns its scratch (multigrid levels, FFT plans, accumulators); it allocates it
 *     on first use for a given n and keeps it until pm_destroy.
 *   - All work is enqueued on the context's stream.  Only scalar_mg_solve*, pm_step
 *     and the calls that return host scalars synchronise that stream.
 *   - Errors are reported only through the return code; pm_last_error(ctx) gives a
 *     one-line message.  Nothing is thrown across the ABI.  A context is used by one
 *     host thread at a time.
 */
#ifndef PMEFT_H
#define PMEFT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pm_ctx pm_ctx;

typedef enum {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1, /* bad pointer, size, parameter or alignment */
    PM_ERR_CUDA = 2,        /* a CUDA runtime or cuFFT call failed */
    PM_ERR_OOM = 3,         /* device allocation failed */
    PM_ERR_NONFINITE = 4,   /* a NaN or Inf appeared in the input or the iteration */
    PM_ERR_NOCONV = 5,      /* max_cycles reached before the tolerance */
    PM_ERR_TIMEOUT = 6,     /* a device-side wait gave up (bounded spin) */
    PM_ERR_OVERFLOW = 7,    /* fixed-point deposit capacity exceeded */
    PM_ERR_TOO_LARGE = 8    /* the request exceeds a fixed-size buffer of the library */
} pm_status;

/* Solver parameters.  pm_default_params fills the defaults noted here. */
typedef struct {
    double omega_m0;       /* Omega_m0 of the LCDM background (0.3; Sec. 3.6.1) */
    double eta;            /* discriminant floor sqrt(D_floor) = eta * 6|nu|/h^2 (0.35; Sec. 3.3) */
    int npre, npost;       /* smoothing sweeps before / after the coarse correction (2, 2) */
    int max_cycles;        /* cap on V-cycles (FP64) or outer iterations (mixed) (100) */
    int coarsest_n;        /* coarsest grid of the V-cycle (4) */
    int coarse_sweeps;     /* sweeps of the coarsest-level solve (8) */
    int precision;         /* 0: FP64 FAS cycle; 1: FP32 inner cycle inside a defect-correction loop whose
                              outer residual is evaluated in float-float arithmetic (two FP32 words per value,
                              about 48 significant bits) and whose stop is confirmed by an FP64 residual;
                              2: the same FP32 inner cycle inside an FP64 defect-correction loop (FP64 outer
                              residual and FP64 iterate) */
    int include_dot_alphaB;/* 1: keep alpha_B-dot/H = d alpha_B/d ln a in C2 (Sec. 2.2) */
    int inner_cycles;      /* precision 1: FP32 V-cycles on the correction per FP64 outer residual (1) */
    int autotune;          /* 1: time the tile variants of the FP32 sweep on first use of each size (1) */
    int linear_eft;        /* 1: pm_step / pm_run use the linearised equations (Sec. 2.5, Eq. linearised):
                              chi = (xi/nu) Psi_N from the one FFT Poisson solve, no screening and no
                              chi multigrid solve (0) */
    int smoother;          /* local solve of the FP64 sweeps (pm_mg_sweep and the precision-0 cycle):
                              0 Method I, the quadratic in the cell value (Sec. 3.2.1); 1 Method II,
                              operator splitting, the quadratic in the cell's Laplacian with the
                              traceless Hessian from the neighbours (Sec. 3.2.2, Eq. opsplit).  The two
                              give the same update in exact arithmetic; FP32 levels use Method I (0) */
    int coarse_exact;      /* 1: the coarsest grid (at most 4^3 cells; coarsest_n <= 4) is solved exactly in FP64
                              by Newton's method with a dense Jacobian and LU with partial pivoting, the gauge
                              multiplier as an extra unknown and the mean constraint as an extra row (Sec. 3.4
                              leaves the coarse solve open), in the FP64 cycle and in the FP32 inner cycle alike;
                              0: coarse_sweeps red-black sweeps with gauge updates (0) */
    int grad_order;        /* force_interp / pm_step gradient: 4 the five-point fourth-order difference of
                              Sec. 3.5.2, 2 the two-point central difference (4) */
    int batch_persistent;  /* scalar_mg_solve_batched: 1 runs the inner V-cycle's levels 32^3 .. 4^3 of every box of
                              at least 64^3 in one persistent cooperative launch per outer iteration, with grid
                              barriers whose waits are bounded (PM_ERR_TIMEOUT when one gives up); 0 launches
                              them per box (1; applies with coarse_exact = 0, coarsest_n = 4, inner_cycles = 1) */
    int zero_start;        /* precision 1: the first sweep of each inner cycle on the finest inner level of grids
                              >= 256^3 (the level that receives the background's coefficients) runs the
                              zero-start kernel, which exploits that the correction starts at zero (same
                              result as clearing it and sweeping; npre >= 1); 0 clears it and sweeps (1) */
} pm_params;

/* Report of one solve.  rel_res = |r|_2 / |f - <f>|_2 of the FP64 residual. */
typedef struct {
    int cycles;                /* V-cycles (FP64) or outer iterations (mixed) performed */
    int vcycles;               /* V-cycles performed in total (FP64 or FP32 inner) */
    int status;                /* the pm_status the solve returned */
    double rel_res;            /* final relative residual */
    double lambda;             /* gauge multiplier: N(chi) = f + lambda on a periodic box */
    long long floored_cells;   /* cells on the floored discriminant at the end (Sec. 3.3) */
    int unstable_nu;           /* 1 when nu <= 0 (non-viable model, Sec. 2.5) */
    double rel_res_hist[64];   /* rel_res before each cycle, [0..min(cycles, 63)] */
    double ms_total;           /* wall time of the solve on the stream, milliseconds */
    double guess_rel_res;      /* rel_res of the caller's initial guess */
    int guess_rejected;        /* 1 when that guess was replaced by chi = 0 (see scalar_mg_solve) */
} pm_solve_info;

/* EFT coefficients at scale factor a (Sec. 2.2, Eq. alpha-a, G_eff/G, Eq. linearised,
 * Eq. chi_scm).  kappa = C4/(4 E^2 a^4); src = xi (3/2)(G_eff/G) a Omega_m0 is the
 * factor of the chi source f = src * delta. */
typedef struct {
    double omega_m_a, alpha_B, alpha_M, geff, E2, C2, C4, nu, xi, kappa, mu_chi, mu_psi, src, poisson_fac;
} pm_coeffs;

void pm_default_params(pm_params* p);

/* Host-only; no context needed.  Returns PM_ERR_INVALID_ARG for a <= 0, omega_m0 outside (0,1). */
pm_status pm_coefficients(double alpha_B0, double alpha_M0, double a, double omega_m0, int include_dot_alphaB,
                          pm_coeffs* out);

/* Create a context on CUDA device `device` that enqueues on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  p may be NULL for defaults. */
pm_status pm_create(pm_ctx** ctx, int device, void* cuda_stream, const pm_params* p);
void pm_destroy(pm_ctx* ctx);
const char* pm_last_error(const pm_ctx* ctx);
pm_status pm_set_params(pm_ctx* ctx, const pm_params* p);

/*
 * CIC density assignment (Sec. 3.6.2; cell-centred CIC).  Each particle adds
 * round((w_x w_y) w_z * 2^40) to 8 cells of an int64 accumulator with integer
 * atomics, so the grid is bit-exact and independent of particle order; then
 * delta = acc * 2^-40 * n^3/np - 1.  pos: device [3][np] in [0,1); delta: device n^3.
 * PM_ERR_INVALID_ARG for np < 1, a bad n or NULL pointers.
 */
pm_status pm_deposit_cic(pm_ctx* ctx, const double* pos, long long np, int n, double* delta);
/* The same deposit, returning the raw int64 fixed-point grid (device n^3 long long). */
pm_status pm_deposit_cic_fixed(pm_ctx* ctx, const double* pos, long long np, int n, long long* acc);

/*
 * Standard Poisson equation in code units with the G_eff factor (Eq. phipsi_mod,
 * Sec. 3.5.1):  L_7pt psi_N = (3/2)(G_eff/G) a Omega_m0 delta on the periodic box,
 * solved by FFT with the discrete 7-point eigenvalues; psi_N has zero mean.
 * delta, psi_N: device n^3 (may not alias).
 */
pm_status poisson_solve(pm_ctx* ctx, const double* delta, int n, double a, double alpha_M0, double* psi_N);

/*
 * Scalar-field solve (Eq. chi_scm; Method I discretisation Sec. 3.2.1; void floor
 * Sec. 3.3; FAS multigrid Sec. 3.4):
 *     nu L(chi) - kappa q2(chi) = xi (3/2)(G_eff/G) a Omega_m0 delta + lambda,  <chi> = 0,
 * with red-black Newton-Gauss-Seidel smoothing, to relative residual <= tol.
 * phi_inout: device n^3, initial guess on entry (zeros for a cold start), chi on
 * exit.  info (host, nullable) receives the report.  Returns PM_ERR_NOCONV when
 * max_cycles is reached (phi_inout then holds the last iterate), PM_ERR_NONFINITE
 * if the iteration produced NaN/Inf.  An initial guess whose relative residual is not
 * finite or exceeds 2 (twice the residual of chi = 0 without floored cells, which is f
 * itself) is replaced by chi = 0 before the first cycle; info.guess_rejected reports it and rel_res_hist then
 * starts from chi = 0.  params.precision selects the FP64 cycle or the
 * FP32-inner / FP64-outer defect correction.  xi = 0 returns chi = 0 at once.
 */
pm_status scalar_mg_solve(pm_ctx* ctx, const double* delta, int n, double alpha_B0, double alpha_M0, double a,
                          double tol, double* phi_inout, pm_solve_info* info);

/*
 * Batched scalar-field solve: nbox independent periodic boxes, each with its own mesh size
 * n[b] (power of two >= 8), density delta[b], parameters (alpha_B0[b], alpha_M0[b], a[b])
 * and initial guess / result phi_inout[b] (device n[b]^3 doubles).  The arrays of sizes,
 * pointers and parameters are host arrays of length nbox.  Every box runs the FP32-inner /
 * FP64-outer defect correction of scalar_mg_solve (precision 1 semantics, whatever
 * params.precision says) to relative residual <= tol; after one eager iteration, one outer
 * iteration of all unconverged boxes is a single CUDA graph launch with one branch per box.
 * infos (host, nullable) receives nbox reports; ms_total is the time of the whole batch.
 * Returns PM_OK when every box converged, else the first failing box's status.
 */
pm_status scalar_mg_solve_batched(pm_ctx* ctx, int nbox, const int* n, const double* const* delta,
                                  const double* alpha_B0, const double* alpha_M0, const double* a, double tol,
                                  double* const* phi_inout, pm_solve_info* infos);

/*
 * Test hook of the batched solve's bounded grid barrier (pm_params.batch_persistent).  With
 * block >= 0, block `block` of the persistent coarse-level kernel leaves the kernel just
 * before its `barrier`-th grid barrier (counted from 0) in every launch, so that the other
 * blocks' bounded waits run out: the batched solve then returns PM_ERR_TIMEOUT with its
 * results undefined, and the context stays usable.  Nothing faults: the blocks only stop
 * early.  block < 0 restores normal operation.  wait_s (> 0) sets how long one barrier wait
 * may take before it gives up (default 2 s); <= 0 keeps the current bound.
 */
pm_status pm_batch_barrier_test(pm_ctx* ctx, int block, int barrier, double wait_s);

/*
 * Force interpolation (Eq. force, Eq. phipsi_mod, Sec. 3.5.2): acc = -grad Psi at the
 * particles, Psi = psi_N + (alpha_B - alpha_M) chi, the five-point fourth-order
 * gradient on the mesh and the CIC weights of the deposit.  phi may be NULL (psi_N
 * alone).  acc: device [3][np].
 */
pm_status force_interp(pm_ctx* ctx, const double* psi_N, const double* phi, int n, double alpha_B0,
                       double alpha_M0, double a, const double* pos, long long np, double* acc);

/*
 * Lensing potential (Eq. phipsi_mod, second line): Phi = Psi_N + alpha_B(a) chi, i.e.
 * L Phi = (3/2)(G_eff/G) a Omega_m0 delta + alpha_B L chi.  psi_N, chi, Phi: device n^3.
 * In the linear regime Phi = mu_Phi Psi_N with mu_Phi = 1 + xi alpha_B / nu (Eq. linearised).
 */
pm_status lensing_potential(pm_ctx* ctx, const double* psi_N, const double* chi, int n, double alpha_B0,
                            double alpha_M0, double a, double* Phi);

/*
 * One particle-mesh step (Sec. 3.5.1 order): deposit, Poisson, chi solve (warm
 * started from phi_state, which receives chi; with params.linear_eft the linearised
 * chi = (xi/nu) Psi_N instead), force interpolation, then one kick and one drift:
 * v += g dt; x = frac(x + v dt).  pos, vel: device [3][np], updated
 * in place.  phi_state: device n^3.  info as for scalar_mg_solve.
 */
pm_status pm_step(pm_ctx* ctx, double* pos, double* vel, long long np, int n, double alpha_B0, double alpha_M0,
                  double a, double dt, double tol, double* phi_state, pm_solve_info* info);

/*
 * nsteps particle-mesh steps (pm_step) at equal steps of supercomoving time t~
 * (dt~ = H0 dt / a^2, so dt~/da = 1/(a^3 E(a)) on the flat background of Sec. 3.1) from
 * a_start to a_end, each step's coefficients taken at the scale factor where it starts,
 * and each chi solve warm-started from the previous step's chi (Sec. 3.5.1): a multi-step
 * run of the method.  The time integrator is the kick-drift of pm_step (reading: the paper
 * does not give one).  info (nullable) receives the last step's report; on a solve that
 * fails, the run stops with that step's status.
 */
pm_status pm_run(pm_ctx* ctx, double* pos, double* vel, long long np, int n, double alpha_B0, double alpha_M0,
                 double a_start, double a_end, int nsteps, double tol, double* phi_state, pm_solve_info* info);

/*
 * Allocation-free CIC deposit.  The paper has no counterpart: this entry point exists
 * for callers that cannot allocate device memory themselves, such as a host
 * application that hands the library a fixed, pre-reserved memory budget, or a
 * plug-in environment that forbids allocations once it is running.  It computes the
 * same delta as pm_deposit_cic (bit for bit) without a context and without calling
 * cudaMalloc, cudaFree or any allocating routine: the int64 accumulator is a
 * file-scope device array of 128^3 entries (16 MiB), which every GPU that loads the
 * library holds until the process exits.
 *   pos: device [3][np] in [0,1); delta: device n^3 (caller-owned, written);
 *   cuda_stream: the cudaStream_t to enqueue on (NULL = legacy default stream).
 *   n must be a power of two with 8 <= n <= 128: n > 128 returns PM_ERR_TOO_LARGE,
 *   other bad arguments PM_ERR_INVALID_ARG; PM_ERR_OVERFLOW as for pm_deposit_cic.
 * The current device must be the one that holds pos and delta.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress) with that
 * device current and keeps it for later calls; make that first call before any stream
 * capture is begun on the device.  Every call uses
 * the same array and clears the part it needs, so calls whose work overlaps on the
 * GPU (other streams, other threads) race with each other.  The call synchronises
 * the stream to read the overflow flag.
 */
pm_status pm_deposit_cic_static(const double* pos, long long np, int n, double* delta, void* cuda_stream);

/* ---- learned warm start (not in the paper) ----
 * A periodic 3D U-Net (3 levels, 16/32/64 channels, 3x3x3 convolutions, ReLU) maps
 * (asinh delta, alpha_B0, alpha_M0, a) to the screened source T = nu L(chi) / src, which is
 * delta where screening is off.  The warm start is chi_0 = (src/nu) L^-1 T_hat (one FFT
 * Poisson solve).  Convolutions run on BF16 tensor cores with FP32 accumulation; weights
 * are kept in FP32 (flat: per conv W[tap][ci][co] then b[co], taps t = (dz+1)*9 + (dy+1)*3
 * + (dx+1); then the 1x1x1 head w[16], b) and repacked to BF16 after every update.
 * Grids: n a power of two >= 16.  All buffers device memory unless stated. */
typedef struct pm_unet pm_unet;
long long pm_unet_num_params(void);
pm_status pm_unet_create(pm_ctx* ctx, pm_unet** net);   /* parameters start at zero */
void pm_unet_destroy(pm_unet* net);
/* The convolution kernels of the network's forward and backward-data passes: 0 the
 * mma.sync (m16n8k16) implicit GEMM, 1 the tcgen05 implicit GEMM with its accumulator in
 * tensor memory (grids of at least 16^3; smaller ones keep path 0).  Default 1.  With path
 * 1 a pass returns PM_ERR_TIMEOUT if a bounded accumulator wait of a convolution gave up. */
pm_status pm_unet_set_conv_path(pm_unet* net, int path);
/* host <-> device copies of the FP32 parameters (which = 0) or accumulated gradients (which = 1) */
pm_status pm_unet_set_params(pm_unet* net, const float* host, long long count);
pm_status pm_unet_get_params(pm_unet* net, float* host, long long count, int which);
/* T_out (n^3 doubles) = network output for delta */
pm_status pm_unet_forward(pm_unet* net, const double* delta, int n, double alpha_B0, double alpha_M0, double a,
                          double* T_out);
/* forward + backward of the loss mean((T_hat - target)^2); gradients are added to the
 * accumulator; *loss (host) receives the loss.  target: n^3 float. */
pm_status pm_unet_loss_grad(pm_unet* net, const double* delta, const float* target, int n, double alpha_B0,
                            double alpha_M0, double a, double* loss);
/* one Adam step on the accumulated gradients (which it then zeroes) */
pm_status pm_unet_adam_step(pm_unet* net, float lr, float beta1, float beta2, float eps);
pm_status pm_unet_zero_grad(pm_unet* net);
/* training target T = nu L(chi) / src of a solved chi (7-point Laplacian); T_out n^3 float */
pm_status pm_unet_target(pm_ctx* ctx, const double* chi, int n, double alpha_B0, double alpha_M0, double a,
                         float* T_out);
/* initial guesses for scalar_mg_solve: the learned one, and the linear solution
 * L chi_0 = (xi / nu)(3/2)(G_eff/G) a Omega_m0 delta that the paper's PySCo-EFT starts from (Sec. 3.5.1).
 * Being guesses, both come from an FP32 FFT Poisson solve (relative accuracy ~1e-6); phi_out is FP64. */
pm_status pm_unet_warm_start(pm_unet* net, const double* delta, int n, double alpha_B0, double alpha_M0, double a,
                             double* phi_out);
pm_status pm_linear_start(pm_ctx* ctx, const double* delta, int n, double alpha_B0, double alpha_M0, double a,
                          double* phi_out);

/* ---- tracing: per-kernel-class device time and launch counts ----
 * With tracing on, the library records a CUDA event pair around each of its kernel
 * launches on the context stream (a small overhead) and sums the elapsed times per
 * class.  Launch counts are kept whether tracing is on or not. */
typedef enum {
    PM_K_SWEEP64 = 0,   /* FP64 red-black half-sweeps, all levels */
    PM_K_SWEEP32 = 1,   /* FP32 half-sweeps of the inner cycle, all levels */
    PM_K_RESID64 = 2,   /* FP64 residual kernels (fine level of either path) */
    PM_K_RESID32 = 3,   /* FP32 residual kernels */
    PM_K_TRANSFER = 4,  /* restriction, FAS right-hand side, prolongation */
    PM_K_COARSEST = 5,  /* coarsest-level solve */
    PM_K_REDUCE = 6,    /* reductions, re-centring, corrections, copies */
    PM_K_PM = 7,        /* deposit, density, Poisson (own kernels + cuFFT), force, kick-drift */
    PM_K_COUNT = 8
} pm_kernel_class;

typedef struct {
    long long launches[PM_K_COUNT];  /* own kernel launches per class (cuFFT counted as 1 each) */
    double ms[PM_K_COUNT];           /* summed event time per class (0 unless tracing was on) */
    long long cells[PM_K_COUNT];     /* cells processed by the finest-level launches per class */
    long long fine_launches[PM_K_COUNT]; /* launches that ran on the finest level of their call */
    double fine_ms[PM_K_COUNT];      /* event time of those finest-level launches */
} pm_profile;

/* Turn per-launch event tracing on (1) or off (0); resets the counters. */
pm_status pm_trace_enable(pm_ctx* ctx, int on);
/* Turn tracing on for a subset of launches only: classes whose bit (1 << PM_K_*) is set in
 * class_mask, and with fine_only != 0 only the launches on the finest level of their call.
 * The other launches are still counted in `launches` but get no events, so timing a few
 * kernels costs the stream almost nothing.  class_mask 0 turns tracing off.  Resets the
 * counters.  PM_ERR_INVALID_ARG if ctx is null. */
pm_status pm_trace_select(pm_ctx* ctx, unsigned class_mask, int fine_only);
/* Synchronise the stream and return the counters accumulated since the last reset. */
pm_status pm_trace_get(pm_ctx* ctx, pm_profile* out);
pm_status pm_trace_reset(pm_ctx* ctx);

/* FMA throughput probe: GFLOP/s of independent FP64 and FP32 FMA chains on this device
 * (the denominator of the ALU roofline of the FP64 stencil kernels).  Allocates and frees
 * a small device buffer; synchronises the stream. */
pm_status pm_probe_fma(pm_ctx* ctx, double* fp64_gflops, double* fp32_gflops);

/* Text report of the autotuner's choices so far (one line per tuned key); NUL-terminated,
 * truncated to len bytes.  Returns the full length. */
int pm_tune_log(const pm_ctx* ctx, char* buf, int len);

/* ---- single multigrid operations on a periodic n^3 grid (for testing the kernels
 * one at a time against a reference; same semantics as inside scalar_mg_solve) ---- */

/* One red-black sweep (red = (i+j+k) even first; a half-sweep reads same-colour
 * neighbours from the values at its start).  u updated in place; f the right-hand
 * side; lambda added to it.  kmask (device n^3 bytes, nullable): per cell, the eighths
 * of the screening term switched off: 0 keeps kappa, k in 1..7 keeps (8-k)/8 of it, 8 or
 * more removes it (the coarse levels of the FAS cycle store there the mean unscreened
 * fraction of a cell's children).  h = 1/n.  The local solve is the one the context's
 * pm_params.smoother selects (Method I or Method II). */
pm_status pm_mg_sweep(pm_ctx* ctx, double* u, const double* f, double lambda, int n, double nu, double kappa,
                      double eta, const unsigned char* kmask);
/* The same sweep on an FP32 grid: mode 0 runs the two half-sweep kernels, mode k >= 1
 * the single-pass fused kernel with tile variant k-1 (pm_tune_log lists the variants the
 * autotuner chose; on FP32 levels of 64^3 and up the inner cycle takes whichever of these
 * kernels and the two half-sweep launches the autotuner timed fastest), and
 * mode 100 + k variant k-1 with the background entering through its six bilinear
 * coefficients rounded to BF16 (the form in which the finest inner level of grids >= 256^3
 * receives it; needs bg and gap and no kmask), and mode 200 the zero-start kernel on those
 * coefficients: the sweep of u = 0 (the values passed in are ignored; n >= 64), which is the
 * first sweep of each inner cycle when pm_params.zero_start is on (200 + k: its variant k - 1,
 * k = 1..6: tiles 64 x 8 and 64 x 16 with fields loaded one or two planes ahead, 128 x 4,
 * 128 x 8; a variant whose tile does not divide n returns PM_ERR_INVALID_ARG).  A variant that
 * does not tile n or cannot
 * take these inputs falls back to mode 0.  u, f: device n^3 float.
 * bg (nullable): the correction form of the mixed-precision inner cycle, where u is the
 * correction to the background bg and the operator is N(bg + u) - N(bg); gap (nullable,
 * needs bg): L_sat - L(bg) per cell, as the finest inner level receives it from the outer
 * residual. */
pm_status pm_mg_sweep_f32(pm_ctx* ctx, float* u, const float* f, float lambda, int n, double nu, double kappa,
                          double eta, const unsigned char* kmask, const float* bg, const float* gap, int mode);
/* Residual: r = f + lambda - N(u) in cells with a real root, nu (L_sat - L(u)) in floored
 * cells; floored (device n^3 bytes, nullable) receives the floored-cell flags. */
pm_status pm_mg_residual(pm_ctx* ctx, const double* u, const double* f, double lambda, int n, double nu,
                         double kappa, double eta, const unsigned char* kmask, double* r, unsigned char* floored);
/* The exact coarsest-level solve of pm_params.coarse_exact alone, on a periodic n^3 grid with
 * n = 2 or 4 (h = 1/n): u (device n^3, in: start, out: solution) of N(u) = f + lambda in
 * cells with a real root and L(u) = L_sat where the discriminant is floored, the mean of u
 * kept; kmask as for pm_mg_sweep (nullable); *lambda_out (host, nullable) receives lambda.
 * PM_ERR_INVALID_ARG for other n or NULL u / f. */
pm_status pm_mg_coarse_exact(pm_ctx* ctx, double* u, const double* f, int n, double nu, double kappa, double eta,
                             const unsigned char* kmask, double* lambda_out);
/* Restriction (average of 8 children) fine n^3 -> coarse (n/2)^3. */
pm_status pm_mg_restrict(pm_ctx* ctx, const double* fine, int n, double* coarse);
/* fine (n^3) += trilinear cell-centred prolongation of coarse ((n/2)^3), periodic. */
pm_status pm_mg_prolong_add(pm_ctx* ctx, const double* coarse, int n, double* fine);

#ifdef __cplusplus
}
#endif
#endif /* PMEFT_H */
