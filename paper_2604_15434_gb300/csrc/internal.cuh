// internal.cuh -- shared declarations of the pmeft CUDA library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cufft.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <string>
#include <vector>

#include "pmeft.h"

#define PM_CUDA(call)                                                                    \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess) {                                                         \
            ctx->set_error(std::string(#call) + ": " + cudaGetErrorString(e_));          \
            return e_ == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;           \
        }                                                                                \
    } while (0)

#define PM_TRY(expr)                          \
    do {                                      \
        pm_status s_ = (expr);                \
        if (s_ != PM_OK) return s_;           \
    } while (0)

namespace pmeft {

constexpr int kThreads = 256;
constexpr int kMaxPartials = 4096;  // blocks of a reduction launch (fixed => deterministic)
// An initial guess whose relative residual exceeds this (the residual of chi = 0 without
// floored cells is exactly 1) is replaced by chi = 0 before the first cycle.
constexpr double kGuessLimit = 2.0;

// ------------------------------------------------------------------ block reductions

// 8 running sums per block: [0] sum r, [1] sum r over unfloored, [2] sum r^2,
// [3] count unfloored, [4] count non-finite, [5] sum x, [6] sum x^2, [7] spare.
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// The launch counter of a partials buffer: one unsigned after its kMaxPartials * 8 doubles
// (allocated with them, zero between launches).
__device__ __forceinline__ unsigned* partials_counter(double* partials)
{
    return reinterpret_cast<unsigned*>(partials + (size_t)kMaxPartials * 8);
}

// The block's NV sums into partials[block * 8 + q].  fin_out (nullable): the block that
// finishes last (ticket from the partials counter, after a fence on every block's writes)
// also sums all blocks' partials, in a fixed order, into fin_out[0..7] and the gauge shift
// fin_out[8] = sum r / count unfloored, and resets the counter, with no second launch.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* partials, unsigned block,
                                           double* fin_out = nullptr)
{
    __shared__ double sh[NV][32];
    __shared__ bool last;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = warp_sum(v[q]);
        if (lane == 0) sh[q][wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = lane < nw ? sh[q][lane] : 0.0;
            s = warp_sum(s);
            if (lane == 0) partials[(size_t)block * 8 + q] = s;
        }
    }
    if (!fin_out) return;
    const unsigned nblocks = gridDim.x * gridDim.y * gridDim.z;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(partials_counter(partials), 1u) == nblocks - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    __shared__ double fs[8][32];
    double acc[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) acc[q] = 0.0;
    for (unsigned b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int q = 0; q < 8; ++q) acc[q] += __ldcg(partials + (size_t)b * 8 + q);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const double s = warp_sum(acc[q]);
        if (lane == 0) fs[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot[8];
        for (int q = 0; q < 8; ++q) {
            tot[q] = 0.0;
            for (int w = 0; w < nw; ++w) tot[q] += fs[q][w];
            fin_out[q] = tot[q];
        }
        fin_out[8] = tot[3] > 0.0 ? tot[0] / tot[3] : 0.0;
        *partials_counter(partials) = 0u;
    }
}

template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* partials, double* fin_out = nullptr)
{
    block_sums<NV>(v, partials, blockIdx.x, fin_out);
}

// Screening weight of a cell from its mask byte k: the cell keeps (8 - k)/8 of kappa,
// none for k >= 8.  Coarse FAS levels store in k the mean unscreened fraction of a cell's
// 8 children in eighths (a floored child counts as unscreened: its equation is linear).
template <typename T>
__device__ __forceinline__ T screen_w(const uint8_t* __restrict__ kmask, size_t c)
{
    if (!kmask) return T(1);
    const int k = kmask[c];
    return k >= 8 ? T(0) : T(8 - k) * T(0.125);
}

// One multigrid level of one precision.  u[0]/u[1] ping-pong under the red-black sweep.
template <typename T>
struct Level {
    int n = 0;
    size_t cells = 0;
    T* u[2] = {nullptr, nullptr};
    int cur = 0;            // index of the buffer holding the current iterate
    T* f = nullptr;         // right-hand side (coarse levels; level 0 reads the source directly)
    T* r = nullptr;         // residual, then the restricted residual of the finer level
    T* ur = nullptr;        // restriction of the finer iterate (for the FAS correction)
    T* bg = nullptr;        // background field of the correction form (mixed precision), or null
    T* gap = nullptr;       // L_sat - L(background) from the FP64 iterate (finest inner level), or null
    uint32_t* coef = nullptr;  // the background's bilinear coefficients, 3 planes of BF16 pairs (finest
                               // inner level of grids >= kCoefMinN), or null
    const T* lamp = nullptr;   // device scalar added to the right-hand side (graph-captured solves), or null
    uint8_t* kmask = nullptr;  // 1: screening term off (coarse levels)
    uint8_t* sat = nullptr;    // 1: floored piece used by the last residual
    bool fine = false;         // finest level of its hierarchy (for tracing)
    bool zero = false;         // the iterate is zero and not stored: the next sweep is the zero-start kernel
};

struct Workspace {
    int n = 0;
    int nlev = 0;
    std::vector<Level<double>> d;  // FP64 hierarchy
    std::vector<Level<float>> s;   // FP32 hierarchy (mixed precision inner cycle)
    float* rplain = nullptr;       // FP32 inner right-hand side f + lambda - N(chi) at level 0
    float2* ff_alt = nullptr;      // second float-float iterate buffer (the residual writes the corrected
                                   // iterate out of place)
    uint32_t* coef_test = nullptr; // coefficients of a caller's background (pm_mg_sweep_f32, mode > 100)
    double* psi = nullptr;         // scratch n^3 (Poisson output / total potential)
    double* grad = nullptr;        // scratch 4 n^3: total potential and its gradient (force kernels)
    double* delta = nullptr;       // scratch n^3 (pm_step)
    long long* acc = nullptr;      // int64 fixed-point deposit grid
    cufftHandle plan_r2c = 0, plan_c2r = 0;
    double2* spec = nullptr;       // n*n*(n/2+1) complex
    bool fft_ready = false;
    cufftHandle plan_r2c32 = 0, plan_c2r32 = 0;  // FP32 transforms of the start fields (guesses)
    float2* spec32 = nullptr;
    float* buf32 = nullptr;
    bool fft32_ready = false;
    // own stream, reductions and device scalars of one box of a batched solve
    cudaStream_t stream = nullptr;
    double* partials = nullptr;    // kMaxPartials * 8
    double* out = nullptr;         // 64 device results
    double* host = nullptr;        // 64 pinned host mirror
    double* lam = nullptr;         // gauge multiplier (device)
    float* shift = nullptr;        // rhs shift of the inner cycle, -gm (device)
    cudaGraphExec_t graph = nullptr;
};

}  // namespace pmeft

struct pm_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    pm_params prm{};
    std::string err;
    std::map<int, pmeft::Workspace*> ws;
    std::vector<pmeft::Workspace*> batch;  // one workspace per box of a batched solve
    cudaStream_t batch_stream = nullptr;    // capture / launch stream of the batched graph
    double* red_partials = nullptr;  // kMaxPartials * 8 doubles
    double* red_out = nullptr;       // device results (64 doubles: [0..8] residual, [16..] mean, [32..] norms)
    double* host_out = nullptr;      // pinned host mirror (64 doubles)
    int* flag = nullptr;             // device error flag
    int num_sms = 152;
    // the batched solve's persistent coarse-level kernel: box table, active flags, sums,
    // barrier words (counter, generation, error) and its test knob
    void* coop_boxes = nullptr;
    int* coop_active = nullptr;
    int* coop_active_host = nullptr;  // pinned
    double* coop_partials = nullptr;
    float* coop_gm = nullptr;
    unsigned* coop_bar = nullptr;
    int* coop_err_host = nullptr;     // pinned
    int coop_cap = 0;
    int coop_fail_block = -1, coop_fail_barrier = -1;
    double coop_wait_s = 2.0;
    int conv_path = 0;  // convolution kernels of the U-Net call in progress (its pm_unet::conv_path)
    std::map<int, int> tuned;  // autotuned tile variant per (level size, inputs)
    std::string tune_log;
    // tracing (pm_trace_*): event pairs per launch, summed per class on read-out
    bool tracing = false;
    unsigned trace_mask = ~0u;  // classes traced while tracing is on
    bool trace_fine_only = false;
    bool traced(int cls, bool fine) const
    {
        return tracing && ((trace_mask >> cls) & 1u) && (fine || !trace_fine_only);
    }
    pm_profile prof{};
    struct Rec {
        int cls;
        bool fine;
        cudaEvent_t a, b;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    int open_cls = -1;
    bool open_fine = false;
    cudaEvent_t open_a = nullptr;
    void set_error(const std::string& m) { err = m; }
    cudaEvent_t ev()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e;
        cudaEventCreate(&e);
        return e;
    }
    // bracket one launch: begin(cls) ... launch ... end()
    void begin(int cls, bool fine = false, long long cells = 0)
    {
        prof.launches[cls] += 1;
        if (fine) {
            prof.fine_launches[cls] += 1;
            prof.cells[cls] += cells;
        }
        if (!traced(cls, fine)) return;
        open_cls = cls;
        open_fine = fine;
        open_a = ev();
        cudaEventRecord(open_a, stream);
    }
    void end()
    {
        if (!tracing || open_cls < 0) return;
        cudaEvent_t b = ev();
        cudaEventRecord(b, stream);
        recs.push_back({open_cls, open_fine, open_a, b});
        open_cls = -1;
    }
};

namespace pmeft {

// Where one solve enqueues its work: the stream, its reduction buffers, and whether
// per-launch event tracing is allowed (not while a stream is being captured into a graph).
// The single-box solve uses the context's own; each box of a batched solve has its own.
struct Exec {
    pm_ctx* c;
    cudaStream_t stream;
    double* red_partials;
    double* red_out;
    double* host_out;
    bool trace_ok;
    const pm_params& prm;
    int num_sms;
    std::map<int, int>& tuned;
    std::string& tune_log;
    Exec(pm_ctx* ctx, cudaStream_t s, double* part, double* out, double* host, bool trace)
        : c(ctx), stream(s), red_partials(part), red_out(out), host_out(host), trace_ok(trace), prm(ctx->prm),
          num_sms(ctx->num_sms), tuned(ctx->tuned), tune_log(ctx->tune_log)
    {
    }
    explicit Exec(pm_ctx* ctx)
        : Exec(ctx, ctx->stream, ctx->red_partials, ctx->red_out, ctx->host_out, true)
    {
    }
    void set_error(const std::string& m) { c->set_error(m); }
    bool tracing() const { return trace_ok && c->tracing; }
    int open_cls = -1;
    bool open_fine = false;
    cudaEvent_t open_a = nullptr;
    void begin(int cls, bool fine = false, long long cells = 0)
    {
        c->prof.launches[cls] += 1;
        if (fine) {
            c->prof.fine_launches[cls] += 1;
            c->prof.cells[cls] += cells;
        }
        if (!trace_ok || !c->traced(cls, fine)) return;
        open_cls = cls;
        open_fine = fine;
        open_a = c->ev();
        cudaEventRecord(open_a, stream);
    }
    void end()
    {
        if (!tracing() || open_cls < 0) return;
        cudaEvent_t b = c->ev();
        cudaEventRecord(b, stream);
        c->recs.push_back({open_cls, open_fine, open_a, b});
        open_cls = -1;
    }
};

inline int grid_for(Exec* x, size_t work, int threads = 256)
{
    size_t blocks = (work + threads - 1) / threads;
    size_t cap = (size_t)x->num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

pm_status get_workspace(pm_ctx* ctx, int n, Workspace** out);
void delete_workspace(Workspace* w);
pm_status ensure_mg(pm_ctx* ctx, Workspace* w, bool want_fp32);
pm_status mg_solve_batched(pm_ctx* ctx, int nbox, const int* n, const double* const* delta, const double* aB0,
                           const double* aM0, const double* a, double tol, double* const* phi, pm_solve_info* infos);
pm_status ensure_fft(pm_ctx* ctx, Workspace* w);
bool valid_n(int n);
int grid_for(pm_ctx* ctx, size_t work, int threads = kThreads);
void coefficients(double aB0, double aM0, double a, double om0, int include_dot, pm_coeffs* c);

// Multigrid entry used by scalar_mg_solve and pm_step.
pm_status mg_solve(pm_ctx* ctx, const double* delta, int n, const pm_coeffs& c, double tol, double* phi,
                   pm_solve_info* info);
// Poisson (psi_N) and the particle kernels.
pm_status poisson(pm_ctx* ctx, const double* delta, int n, double fac, double* psi);
// the same solve through FP32 transforms (for initial guesses); delta and psi FP64
pm_status poisson32(pm_ctx* ctx, const double* delta, int n, double fac, double* psi);
pm_status ensure_fft32(pm_ctx* ctx, Workspace* w);
pm_status deposit(pm_ctx* ctx, const double* pos, long long np, int n, long long* acc);
pm_status density(pm_ctx* ctx, const long long* acc, int n, long long np, double* delta);
pm_status interp_force(pm_ctx* ctx, const double* psiN, const double* chi, double xi, int n, const double* pos,
                       long long np, double* acc);
pm_status kick_drift(pm_ctx* ctx, double* pos, double* vel, const double* acc, long long np, double dt);

// ---------------------------------------------------------------------------------------
// Device side: the local quadratic of Eq. chi_discrete at one cell (Sec. 3.2.1).
// Values: c0 centre; ax/ay/az sums of the two face neighbours per axis; exy/exz/eyz the
// four-corner cross sums (x+y+ - x+y- - x-y+ + x-y-) of the 4h^2 cross differences.
// ---------------------------------------------------------------------------------------
template <typename T>
struct Local {
    T G, Ep, P, D, L, g;  // g = L_sat - L, the floored gap (valid when kappa != 0)
};

template <typename T>
struct Stencil {
    T c0, ax, ay, az, exy, exz, eyz;
};

// Load the 19-point stencil around (i, j, k) of a periodic n^3 grid; the centre and the
// 12 edge neighbours (same red/black colour) come from `own`, the 6 faces from `oth`.
template <typename T>
__device__ __forceinline__ Stencil<T> load_stencil(const T* __restrict__ own, const T* __restrict__ oth, int i,
                                                   int j, int k, int n)
{
    const int m = n - 1;
    const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m, kp = (k + 1) & m,
              km = (k - 1) & m;
    const size_t sn = (size_t)n, row = (size_t)k * sn + j;
    const size_t rk = row * sn;
    auto at = [&](const T* p, int ii, int jj, int kk) { return p[((size_t)kk * sn + jj) * sn + ii]; };
    Stencil<T> s;
    s.c0 = own[rk + i];
    s.ax = oth[rk + ip] + oth[rk + im];
    s.ay = at(oth, i, jp, k) + at(oth, i, jm, k);
    s.az = at(oth, i, j, kp) + at(oth, i, j, km);
    s.exy = at(own, ip, jp, k) - at(own, ip, jm, k) - at(own, im, jp, k) + at(own, im, jm, k);
    s.exz = at(own, ip, j, kp) - at(own, ip, j, km) - at(own, im, j, kp) + at(own, im, j, km);
    s.eyz = at(own, i, jp, kp) - at(own, i, jp, km) - at(own, i, jm, kp) + at(own, i, jm, km);
    return s;
}

// N and the local quadratic about the current centre value.  ih2 = 1/h^2 (exact for
// power-of-two n).  rhs = f + lambda.  lsat = L_sat = 3 nu (1 - eta)/(4 kappa), the
// Laplacian of the floored root (unused when kappa = 0).
//
// With a background b (correction form of the mixed-precision inner cycle) the operator
// is N(b + u) - N(b), evaluated without cancellation, and L is L(b + u).  On the finest
// inner level the caller passes gapx = L_sat - L(b) computed in FP64 from the FP64
// iterate: near convergence it is small in floored cells, so its FP32 rounding is
// relative, whereas L(b) itself (or the FP32 copy's second differences) would leave an
// absolute error ~eps |L_sat| under the outer residual.
template <typename T, bool BG>
__device__ __forceinline__ Local<T> local_eval(const Stencil<T>& s, const Stencil<T>& b, T ih2, T nu, T kap, T rhs,
                                               T lsat, bool use_gap = false, T gapx = T(0))
{
    // Work in h = 1 units: X = h^2 chi_xx, cross terms h^2 chi_xy = exy/4, and fold 1/h^2
    // and 1/h^4 into nu and kappa.  n is a power of two, so h^2 is a power of two and
    // every rescaled product rounds exactly as the unscaled one would.
    const T X = s.ax - T(2) * s.c0;
    const T Y = s.ay - T(2) * s.c0;
    const T Z = s.az - T(2) * s.c0;
    Local<T> o;
    const T L1 = X + Y + Z;  // h^2 L
    // h^4 q2 = 2 (XY + YZ + ZX) - 2 (exy^2 + exz^2 + eyz^2)/16
    T q2 = T(2) * (X * Y + Y * Z + Z * X) - T(0.125) * (s.exy * s.exy + s.exz * s.exz + s.eyz * s.eyz);
    T L1tot = L1;
    if (BG) {
        const T Xb = b.ax - T(2) * b.c0;
        const T Yb = b.ay - T(2) * b.c0;
        const T Zb = b.az - T(2) * b.c0;
        // q2(b + u) - q2(b) = q2(u) + 2[Xb(Y+Z) + Yb(X+Z) + Zb(X+Y)] - 4[bxy cxy + bxz cxz + byz cyz]
        q2 += T(2) * (Xb * (Y + Z) + Yb * (X + Z) + Zb * (X + Y)) -
              T(0.25) * (b.exy * s.exy + b.exz * s.exz + b.eyz * s.eyz);
        L1tot = L1 + (Xb + Yb + Zb);
    }
    T Ltot = L1tot * ih2;
    if (kap != T(0)) {
        if (use_gap) {
            o.g = gapx - L1 * ih2;
            Ltot = lsat - o.g;
        } else {
            o.g = lsat - Ltot;
        }
    } else {
        o.g = T(0);
    }
    o.L = Ltot;
    const T nu1 = nu * ih2, kap1 = kap * ih2 * ih2;
    const T N = nu1 * L1 - kap1 * q2;
    o.G = N - rhs;
    o.Ep = (T(-6) * nu + T(8) * kap * o.L) * ih2;
    o.P = T(-24) * kap1;
    o.D = o.Ep * o.Ep - T(4) * o.P * o.G;
    return o;
}

// ---------------------------------------------------------------- background coefficients
//
// In the correction form the background b enters the operator only through the bilinear
// part of q2(b + u) - q2(b) - q2(u) = cX X + cY Y + cZ Z + cxy exy + cxz exz + cyz eyz
// (h = 1 units, X = u_xx h^2 ..., exy the raw 4-point cross difference of u), with
// cX = 2(Yb + Zb), cY = 2(Xb + Zb), cZ = 2(Xb + Yb), cxy = -bxy/4, cxz = -bxz/4, cyz = -byz/4
// from b's second and cross differences.  The finest inner level of large grids keeps these
// six numbers per cell in BF16 (three planes of packed pairs, 12 bytes per cell), written
// by the outer residual once per outer iteration from the differences of the float-float
// iterate it has just formed (whose high parts b is), instead of re-reading b's 19-point
// stencil in every sweep.  BF16 perturbs only this bilinear part of the inner
// (preconditioning) operator, by 2^-9 relative; the outer float-float residual, which
// decides convergence, is unaffected.
constexpr int kCoefMinN = 256;

struct BgCoef {
    float cX, cY, cZ, cxy, cxz, cyz;
};

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ BgCoef unpack_bg_coef(uint32_t k0, uint32_t k1, uint32_t k2)
{
    return BgCoef{__uint_as_float(k0 << 16), __uint_as_float(k0 & 0xffff0000u), __uint_as_float(k1 << 16),
                  __uint_as_float(k1 & 0xffff0000u), __uint_as_float(k2 << 16), __uint_as_float(k2 & 0xffff0000u)};
}

// local_eval<float, BG = true> with the gap of the finest inner level, the background given
// by its coefficients
__device__ __forceinline__ Local<float> local_eval_cf(const Stencil<float>& s, const BgCoef& cf, float ih2, float nu,
                                                      float kap, float rhs, float lsat, float gapx)
{
    const float X = s.ax - 2.f * s.c0;
    const float Y = s.ay - 2.f * s.c0;
    const float Z = s.az - 2.f * s.c0;
    Local<float> o;
    const float L1 = X + Y + Z;
    float q2 = 2.f * (X * Y + Y * Z + Z * X) - 0.125f * (s.exy * s.exy + s.exz * s.exz + s.eyz * s.eyz);
    q2 += cf.cX * X + cf.cY * Y + cf.cZ * Z + cf.cxy * s.exy + cf.cxz * s.exz + cf.cyz * s.eyz;
    float Ltot;
    if (kap != 0.f) {
        o.g = gapx - L1 * ih2;
        Ltot = lsat - o.g;
    } else {
        o.g = 0.f;
        Ltot = L1 * ih2;  // unused: the screening term is off
    }
    o.L = Ltot;
    const float nu1 = nu * ih2, kap1 = kap * ih2 * ih2;
    const float N = nu1 * L1 - kap1 * q2;
    o.G = N - rhs;
    o.Ep = (-6.f * nu + 8.f * kap * o.L) * ih2;
    o.P = -24.f * kap1;
    o.D = o.Ep * o.Ep - 4.f * o.P * o.G;
    return o;
}

// Correction e = c_new - c0: the root continuing the linear solution (Eq. quadratic),
// with the discriminant floored at Df (Sec. 3.3).  sp = -sgn(nu).  The floored root is
// (sp sqrt(Df) - Ep)/(2P), which equals -g h^2/6 exactly (the centre value that puts L on
// L_sat); the latter form is used because it carries no cancellation.
template <typename T>
__device__ __forceinline__ T local_update(const Local<T>& o, T sp, T Df, T ih2)
{
    if (o.P == T(0)) return -o.G / o.Ep;
    if (o.D < Df) return -o.g / (T(6) * ih2);
    const T sq = sqrt(o.D);
    if (o.Ep * sp > T(0)) return T(-2) * o.G / (o.Ep + sp * sq);
    return (sp * sq - o.Ep) / (T(2) * o.P);
}

// FP32 variant for the inner cycle of the defect-correction loop: the same branches with
// the approximate hardware reciprocal and square root (relative error ~1e-7), and the
// constant divisions folded into multiplications.  The outer residual decides the accuracy
// of the result, so the inner update only has to be a good correction.
__device__ __forceinline__ float local_update_fast(const Local<float>& o, float sp, float Df, float h2over6,
                                                   float inv2P)
{
    if (o.P == 0.f) return __fdividef(-o.G, o.Ep);
    if (o.D < Df) return -o.g * h2over6;
    const float sq = __fsqrt_rn(o.D);
    if (o.Ep * sp > 0.f) return __fdividef(-2.f * o.G, o.Ep + sp * sq);
    return (sp * sq - o.Ep) * inv2P;
}

}  // namespace pmeft
