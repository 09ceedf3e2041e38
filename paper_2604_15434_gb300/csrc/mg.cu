// mg.cu -- FAS multigrid for the screened chi equation (Sec. 3.2.1, 3.3, 3.4 of arXiv 2604.15434).
//
// Discrete problem (identical to the CPU reference):
//   N(chi) = nu L(chi) - kappa q2(chi) = f + lambda on the periodic n^3 mesh, <chi> = 0,
//   with the root of Eq. quadratic that continues the linear solution and the
//   discriminant floored at D_floor = (eta 6|nu|/h^2)^2 (Sec. 3.3).  Red-black
//   Newton-Gauss-Seidel: a half-sweep reads the 12 same-colour edge neighbours from the
//   values at its start (out-of-place ping-pong of two buffers).
// Residual: f + lambda - N in cells with a real root, nu (L_sat - L) in floored cells; the
// floored piece belongs to the finest level, coarse levels fix their pieces by the
// restricted mask (screening off where at least half the children were floored).
// Two drivers: an FP64 FAS V-cycle, and an FP64 defect-correction loop whose inner
// FAS V-cycle runs in FP32 on the correction e with the FP64 iterate as background.
#include <cmath>

#include "internal.cuh"
#include "sweep_fused.cuh"
#include "sweep_pair.cuh"
#include "sweep_col.cuh"
#include "sweep_zero.cuh"
#include "outer_ff.cuh"
#include "resid_fused.cuh"

namespace pmeft {

// ------------------------------------------------------------------ reductions

// ------------------------------------------------------------------ smoother

// Method II, operator splitting (Sec. 3.2.2, Eq. opsplit): the cell's equation
// nu L - kap [(2/3) L^2 - T2] = rhs as a quadratic in its Laplacian L, T2 the squared
// traceless Hessian, which holds no centre value (X - L/3 = (2 a_x - a_y - a_z)/(3 h^2));
// the root continuing the linear solution, the discriminant floored at (eta nu)^2 (the
// floor of Method I carried to this variable, whose floored root is L_sat), then the
// Newton update that gives the centre that Laplacian.  In exact arithmetic this is
// Method I's update; it is a second, independent form of the same local solve.
template <typename T>
__device__ __forceinline__ T opsplit_update(const Stencil<T>& s, T ih2, T nu, T kap, T rhs, T etanu)
{
    const T Lnow = (s.ax + s.ay + s.az - T(6) * s.c0) * ih2;
    T Lroot;
    if (kap == T(0)) {
        Lroot = rhs / nu;
    } else {
        const T third = T(1) / T(3);
        const T tx = (T(2) * s.ax - s.ay - s.az) * ih2 * third;
        const T ty = (T(2) * s.ay - s.ax - s.az) * ih2 * third;
        const T tz = (T(2) * s.az - s.ax - s.ay) * ih2 * third;
        const T q = T(0.25) * ih2;
        const T cxy = s.exy * q, cxz = s.exz * q, cyz = s.eyz * q;
        const T T2 = tx * tx + ty * ty + tz * tz + T(2) * (cxy * cxy + cxz * cxz + cyz * cyz);
        const T a = T(-2) * kap * third, cc = kap * T2 - rhs;
        const T D = nu * nu - T(4) * a * cc;
        const T sb = nu >= T(0) ? T(1) : T(-1);
        if (D < etanu * etanu)
            Lroot = (-nu + sb * etanu) / (T(2) * a);
        else
            Lroot = T(-2) * cc / (nu + sb * sqrt(D));
    }
    return s.c0 + (Lnow - Lroot) / (T(6) * ih2);
}

// One cell of a colour half-sweep: element t of the n^3/2 cells of `colour`
// ((i+j+k) & 1 == colour), lg = log2 n.  own: array holding this colour's current values;
// oth: the other colour's; out: receives the new values of this colour.  rhs = fscale * F +
// lam.  OPS: the local solve of Method II (opsplit_update; etanu = eta |nu|) instead of
// Method I's.
template <typename T, bool BG, bool OPS>
__device__ __forceinline__ void half_sweep_cell(const T* own, const T* oth,
                                                T* out, const T* F, T fscale, T lam,
                                                const uint8_t* kmask, const T* bg,
                                                const T* gap, int n, int lg, int colour, T ih2, T nu,
                                                T kap, T sp, T Df, T lsat_c, T etanu, size_t t)
{
    const int hn = n >> 1;
    const int m = (int)(t & (size_t)(hn - 1));  // n (hence hn) is a power of two
    const size_t row = t >> (lg - 1);
    const int j = (int)(row & (size_t)(n - 1)), k = (int)(row >> lg);
    const int i = 2 * m + ((j + k + colour) & 1);
    const size_t c = row * n + i;
    Stencil<T> s = load_stencil(own, oth, i, j, k, n);
    Stencil<T> b;
    if (BG) b = load_stencil(bg, bg, i, j, k, n);
    const T w = screen_w<T>(kmask, c);
    const T kc = kap * w;
    if (OPS) {
        out[c] = opsplit_update<T>(s, ih2, nu, kc, fscale * F[c] + lam, etanu);
        return;
    }
    const T lsat = kc != T(0) ? (kmask ? lsat_c / w : lsat_c) : T(0);  // w = 1 without a mask
    Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, fscale * F[c] + lam, lsat, gap != nullptr, gap ? gap[c] : T(0));
    out[c] = s.c0 + local_update(o, sp, Df, ih2);
}

// One colour half-sweep over the n^3/2 cells of `colour` (half_sweep_cell).
template <typename T, bool BG, bool OPS = false>
__global__ void __launch_bounds__(256) k_half_sweep(const T* __restrict__ own, const T* __restrict__ oth,
                                                    T* __restrict__ out, const T* __restrict__ F, T fscale, T lam,
                                                    const uint8_t* __restrict__ kmask, const T* __restrict__ bg,
                                                    const T* __restrict__ gap, int n, int colour, T ih2, T nu, T kap,
                                                    T sp, T Df, T lsat_c, const T* __restrict__ lamp, T etanu)
{
    if (lamp) lam += *lamp;
    const size_t total = (size_t)n * n * (n >> 1);
    const int lg = __ffs(n) - 1;
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x)
        half_sweep_cell<T, BG, OPS>(own, oth, out, F, fscale, lam, kmask, bg, gap, n, lg, colour, ih2, nu, kap, sp, Df,
                                    lsat_c, etanu, t);
}

// ------------------------------------------------------------------ residual

// One cell of the residual: r = f + lam - N (real root) or nu (L_sat - L) (floored), its
// floored flag, and the cell's share of the sums fa: [0] sum r, [1] sum r over unfloored,
// [2] sum r^2, [3] count unfloored, [4] count non-finite.  MIXED (FP64 level 0 of the
// defect-correction loop) also writes the FP32 copies: the plain residual -G for the inner
// right-hand side, the iterate as the inner background, and the floored gap.
template <typename T, bool BG, bool WRITE_R, bool MIXED>
__device__ __forceinline__ void residual_cell_s(const Stencil<T>& s, const Stencil<T>& b, const T* F, T fscale,
                                                T lam, const uint8_t* kmask, const T* gap, T ih2, T nu, T kap, T Df,
                                                T lsat_c, bool floor_piece, T* r, uint8_t* sat, float* rplain,
                                                float* chi32, float* gap32, size_t c, float (&fa)[5]);

template <typename T, bool BG, bool WRITE_R, bool MIXED>
__device__ __forceinline__ void residual_cell(const T* u, const T* F, T fscale, T lam,
                                              const uint8_t* kmask, const T* bg,
                                              const T* gap, int n, int lg, T ih2, T nu, T kap, T Df,
                                              T lsat_c, bool floor_piece, T* r,
                                              uint8_t* sat, float* rplain,
                                              float* chi32, float* gap32, size_t c,
                                              float (&fa)[5])
{
    const int i = (int)(c & (size_t)(n - 1));  // n is a power of two
    const size_t row = c >> lg;
    const int j = (int)(row & (size_t)(n - 1)), k = (int)(row >> lg);
    Stencil<T> s = load_stencil(u, u, i, j, k, n);
    Stencil<T> b;
    if (BG) b = load_stencil(bg, bg, i, j, k, n);
    residual_cell_s<T, BG, WRITE_R, MIXED>(s, b, F, fscale, lam, kmask, gap, ih2, nu, kap, Df, lsat_c, floor_piece, r,
                                           sat, rplain, chi32, gap32, c, fa);
}

// The residual of one cell from its stencil (residual_cell, or a tiled kernel's shared copy).
template <typename T, bool BG, bool WRITE_R, bool MIXED>
__device__ __forceinline__ void residual_cell_s(const Stencil<T>& s, const Stencil<T>& b, const T* F, T fscale,
                                                T lam, const uint8_t* kmask, const T* gap, T ih2, T nu, T kap, T Df,
                                                T lsat_c, bool floor_piece, T* r, uint8_t* sat, float* rplain,
                                                float* chi32, float* gap32, size_t c, float (&fa)[5])
{
    const T w = screen_w<T>(kmask, c);
    const T kc = kap * w;
    const T lsat = kc != T(0) ? (kmask ? lsat_c / w : lsat_c) : T(0);  // w = 1 without a mask
    Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, fscale * F[c] + lam, lsat, gap != nullptr, gap ? gap[c] : T(0));
    // the floored piece exists on the finest level; coarse levels take their pieces from
    // the restricted mask (linear where masked, quadratic elsewhere), so their right-hand
    // side and their smoother solve the same equation (FAS consistency), except where a
    // coarse cell's quadratic has no real root (D < 0): the smoother's safeguard puts such a
    // cell at the floored update, and its residual is the floored piece as well
    const bool fl = (o.P != T(0)) && (o.D < (floor_piece ? Df : T(0)));
    // floored piece nu (L_sat - L) = nu g
    const T rv = fl ? nu * o.g : -o.G;
    if (WRITE_R) r[c] = rv;
    if (sat) sat[c] = fl ? 1 : 0;
    if (MIXED) {
        rplain[c] = (float)(-o.G);
        chi32[c] = (float)s.c0;
        gap32[c] = (float)o.g;
    }
    // per-thread partial sums in FP32 (a few hundred terms each); the block and grid
    // reductions are FP64.  The sums only set the gauge shift and the stopping norm.
    const float d = (float)rv;
    if (!isfinite(d)) {
        fa[4] += 1.f;
    } else {
        fa[0] += d;
        fa[2] += d * d;
        if (!fl) {
            fa[1] += d;
            fa[3] += 1.f;
        }
    }
}

// The residual of a level (residual_cell) and its block sums for the gauge update and the
// norm.
template <typename T, bool BG, bool WRITE_R, bool MIXED>
__global__ void __launch_bounds__(256) k_residual(const T* __restrict__ u, const T* __restrict__ F, T fscale, T lam,
                                                  const uint8_t* __restrict__ kmask, const T* __restrict__ bg,
                                                  const T* __restrict__ gap, int n, T ih2, T nu, T kap, T Df,
                                                  T lsat_c, bool floor_piece, T* __restrict__ r,
                                                  uint8_t* __restrict__ sat,
                                                  double* __restrict__ partials, float* __restrict__ rplain,
                                                  float* __restrict__ chi32, float* __restrict__ gap32,
                                                  const T* __restrict__ lamp, double* __restrict__ fin_out = nullptr)
{
    if (lamp) lam += *lamp;
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const size_t total = (size_t)n * n * n;
    const int lg = __ffs(n) - 1;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        residual_cell<T, BG, WRITE_R, MIXED>(u, F, fscale, lam, kmask, bg, gap, n, lg, ih2, nu, kap, Df, lsat_c,
                                             floor_piece, r, sat, rplain, chi32, gap32, c, fa);
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, fin_out);
}

// The FP64 residual of a level without a background (the FP64 cycle's levels, the mixed
// loops' confirming residual and the FP64 outer loop), marching up z: a block of 32 x 8
// threads keeps three planes of its 32 x 8 tile and their one-cell halo in a shared ring, so
// each iterate value is read from global memory once per block instead of once per stencil
// point.  Arithmetic and sums as k_residual (residual_cell_s); grid (n/32, n/8, n/nz).
constexpr int kR64TX = 32, kR64TY = 8;
template <bool WRITE_R, bool MIXED>
__global__ void __launch_bounds__(256) k_residual64_zm(const double* __restrict__ u, const double* __restrict__ F,
                                                       double fscale, double lam, const uint8_t* __restrict__ kmask,
                                                       int n, int nz, double ih2, double nu, double kap, double Df,
                                                       double lsat_c, bool floor_piece, double* __restrict__ r,
                                                       uint8_t* __restrict__ sat, double* __restrict__ partials,
                                                       float* __restrict__ rplain, float* __restrict__ chi32,
                                                       float* __restrict__ gap32, const double* __restrict__ lamp,
                                                       double* __restrict__ fin_out)
{
    constexpr int WX = kR64TX + 2, WY = kR64TY + 2, PL = WX * WY;
    __shared__ double ring[3][PL];
    if (lamp) lam += *lamp;
    const int m = n - 1;
    const int x0 = blockIdx.x * kR64TX, y0 = blockIdx.y * kR64TY, z0 = blockIdx.z * nz;
    const int t = threadIdx.x, tx = t & (kR64TX - 1), ty = t / kR64TX;
    const size_t plane = (size_t)n * n;
    auto load = [&](int z, int slot) {
        const size_t zo = (size_t)(z & m) * plane;
        for (int e = t; e < PL; e += 256) {
            const int xx = e % WX, yy = e / WX;
            ring[slot][e] = u[zo + (size_t)((y0 - 1 + yy) & m) * n + ((x0 - 1 + xx) & m)];
        }
    };
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    load(z0 - 1, 0);
    load(z0, 1);
    const int cl = (ty + 1) * WX + tx + 1;
    for (int s = 0; s < nz; ++s) {
        const int z = z0 + s;
        load(z + 1, (s + 2) % 3);
        __syncthreads();
        const double* pm = ring[s % 3];        // plane z - 1
        const double* pc = ring[(s + 1) % 3];  // plane z
        const double* pp = ring[(s + 2) % 3];  // plane z + 1
        Stencil<double> st, b;
        st.c0 = pc[cl];
        st.ax = pc[cl + 1] + pc[cl - 1];
        st.ay = pc[cl + WX] + pc[cl - WX];
        st.az = pp[cl] + pm[cl];
        st.exy = pc[cl + 1 + WX] - pc[cl + 1 - WX] - pc[cl - 1 + WX] + pc[cl - 1 - WX];
        st.exz = pp[cl + 1] - pm[cl + 1] - pp[cl - 1] + pm[cl - 1];
        st.eyz = pp[cl + WX] - pm[cl + WX] - pp[cl - WX] + pm[cl - WX];
        const size_t c = (size_t)z * plane + (size_t)(y0 + ty) * n + (x0 + tx);
        residual_cell_s<double, false, WRITE_R, MIXED>(st, b, F, fscale, lam, kmask, nullptr, ih2, nu, kap, Df, lsat_c,
                                                       floor_piece, r, sat, rplain, chi32, gap32, c, fa);
        __syncthreads();  // the slot of plane z - 1 is refilled next step
    }
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z), fin_out);
}

// ------------------------------------------------------------------ transfers

// Coarse cell c = average of its 8 children, for the iterate (-> ur and the coarse start
// value) and the gauge-projected residual r - gm * [unfloored]; the coarse screening mask
// holds the children's mean unscreened fraction in eighths (floored children count 8).
template <typename T>
__device__ __forceinline__ void restrict_fas_cell(const T* uf, const T* rf,
                                                  const uint8_t* satf, const uint8_t* kmf,
                                                  T gm, int nc, int lgc, T* ur, T* uc,
                                                  T* rc, uint8_t* kmc, size_t c)
{
    const int nf = 2 * nc;
    const int I = (int)(c & (size_t)(nc - 1));  // nc is a power of two
    const size_t row = c >> lgc;
    const int J = (int)(row & (size_t)(nc - 1)), K = (int)(row >> lgc);
    T su = T(0), sr = T(0);
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const int di = q & 1, dj = (q >> 1) & 1, dk = (q >> 2) & 1;
        const size_t f = ((size_t)(2 * K + dk) * nf + (2 * J + dj)) * nf + (2 * I + di);
        su += uf[f];
        const bool fl = satf[f] != 0;
        sr += fl ? rf[f] : rf[f] - gm;
        const int kf = kmf ? (kmf[f] < 8 ? kmf[f] : 8) : 0;
        cnt += fl ? 8 : kf;  // unscreened eighths of the child
    }
    su *= T(0.125);
    ur[c] = su;
    uc[c] = su;
    rc[c] = sr * T(0.125);
    kmc[c] = (uint8_t)((cnt + 4) >> 3);  // mean of the children, rounded to eighths
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_fas(const T* __restrict__ uf, const T* __restrict__ rf,
                                                      const uint8_t* __restrict__ satf,
                                                      const uint8_t* __restrict__ kmf, const double* __restrict__ gm_ptr,
                                                      int nc, T* __restrict__ ur, T* __restrict__ uc,
                                                      T* __restrict__ rc, uint8_t* __restrict__ kmc)
{
    const size_t total = (size_t)nc * nc * nc;
    const T gm = gm_ptr ? (T)(*gm_ptr) : T(0);
    const int lgc = __ffs(nc) - 1;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        restrict_fas_cell<T>(uf, rf, satf, kmf, gm, nc, lgc, ur, uc, rc, kmc, c);
}

// Plain 8-child average (background field of the correction form).
template <typename T>
__global__ void k_restrict(const T* __restrict__ uf, int nc, T* __restrict__ uc)
{
    const int nf = 2 * nc;
    const size_t total = (size_t)nc * nc * nc;
    const int lgc = __ffs(nc) - 1;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const int I = (int)(c & (size_t)(nc - 1));  // nc is a power of two
        const size_t row = c >> lgc;
        const int J = (int)(row & (size_t)(nc - 1)), K = (int)(row >> lgc);
        T su = T(0);
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int di = q & 1, dj = (q >> 1) & 1, dk = (q >> 2) & 1;
            su += uf[((size_t)(2 * K + dk) * nf + (2 * J + dj)) * nf + (2 * I + di)];
        }
        uc[c] = su * T(0.125);
    }
}

// FAS right-hand side f_H = N_H(R u) + R r (no gauge term on coarse levels).
// coefo / gapo (BG, FP32 levels of at least kCoefMinN): also the level's background
// coefficients (the layout the finest level's float-float residual writes) and its floored
// gap L_sat/w - L(background), w the cell's screening weight, for the coefficient sweep.
// gm_ptr (non-null after the restricting residual k_residual_zm<.., RESTRICT>): rc holds the
// children's raw mean residual and the mask byte carries the unfloored children in its high
// nibble; the gauge term -gm * (unfloored children)/8 is applied here and the nibble cleared.
template <typename T, bool BG>
__device__ __forceinline__ void fas_rhs_cell(const T* uc, const T* rc,
                                             uint8_t* kmask, const T* bg, int n, int lg,
                                             T ih2, T nu, T kap, T* fc, uint32_t* coefo,
                                             float* gapo, float lsat, bool apply_gm, T gm, size_t total,
                                             size_t c)
{
    const int i = (int)(c & (size_t)(n - 1));  // n is a power of two
    const size_t row = c >> lg;
    const int j = (int)(row & (size_t)(n - 1)), k = (int)(row >> lg);
    Stencil<T> s = load_stencil(uc, uc, i, j, k, n);
    Stencil<T> b;
    if (BG) b = load_stencil(bg, bg, i, j, k, n);
    T rcv = rc[c];
    if (apply_gm) {
        const uint8_t kb = kmask[c];
        rcv -= gm * (T)(kb >> 4) * T(0.125);
        kmask[c] = kb & 15;
    }
    const T w = screen_w<T>(kmask, c);
    const T kc = kap * w;
    Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, T(0), T(0));
    fc[c] = o.G + rcv;
    if (BG && coefo) {
        const float Xb = (float)(b.ax - T(2) * b.c0), Yb = (float)(b.ay - T(2) * b.c0),
                    Zb = (float)(b.az - T(2) * b.c0);
        coefo[c] = pack_bf16x2(2.f * (Yb + Zb), 2.f * (Xb + Zb));
        coefo[total + c] = pack_bf16x2(2.f * (Xb + Yb), -0.25f * (float)b.exy);
        coefo[2 * total + c] = pack_bf16x2(-0.25f * (float)b.exz, -0.25f * (float)b.eyz);
        gapo[c] = kc != T(0) ? lsat / (float)w - (float)ih2 * (Xb + Yb + Zb) : 0.f;
    }
}

template <typename T, bool BG>
__global__ void __launch_bounds__(256) k_fas_rhs(const T* __restrict__ uc, const T* __restrict__ rc,
                                                 uint8_t* __restrict__ kmask, const T* __restrict__ bg, int n,
                                                 T ih2, T nu, T kap, T* __restrict__ fc, uint32_t* __restrict__ coefo,
                                                 float* __restrict__ gapo, float lsat, const double* __restrict__ gm_ptr)
{
    const T gm = gm_ptr ? (T)(*gm_ptr) : T(0);
    const size_t total = (size_t)n * n * n;
    const int lg = __ffs(n) - 1;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        fas_rhs_cell<T, BG>(uc, rc, kmask, bg, n, lg, ih2, nu, kap, fc, coefo, gapo, lsat, gm_ptr != nullptr, gm, total,
                            c);
}

// k_fas_rhs for levels of at least 32^3, tiled: a block stages the iterate (and the
// background) of a 32 x 4 x 4 brick with its one-cell halo in shared memory, and each
// thread evaluates two cells' stencils from there, with the arithmetic of load_stencil and
// k_fas_rhs.  Grid (n/32, n/4, n/4), 256 threads.
template <typename T, bool BG>
__global__ void __launch_bounds__(256) k_fas_rhs_tile(const T* __restrict__ uc, const T* __restrict__ rc,
                                                      uint8_t* __restrict__ kmask, const T* __restrict__ bg, int n,
                                                      T ih2, T nu, T kap, T* __restrict__ fc,
                                                      uint32_t* __restrict__ coefo, float* __restrict__ gapo,
                                                      float lsat, const double* __restrict__ gm_ptr)
{
    constexpr int BX = 32, BY = 4, BZ = 4, WX = BX + 2, WY = BY + 2, WZ = BZ + 2, WXY = WX * WY, P = WXY * WZ;
    __shared__ T su[P];
    __shared__ T sb[BG ? P : 1];
    const int m = n - 1;
    const int X0 = blockIdx.x * BX, Y0 = blockIdx.y * BY, Z0 = blockIdx.z * BZ;
    for (int e = threadIdx.x; e < P; e += 256) {
        const int xx = e % WX, yy = (e / WX) % WY, zz = e / WXY;
        const size_t g = ((size_t)((Z0 - 1 + zz) & m) * n + ((Y0 - 1 + yy) & m)) * n + ((X0 - 1 + xx) & m);
        su[e] = uc[g];
        if (BG) sb[e] = bg[g];
    }
    __syncthreads();
    auto stencil = [&](const T* p, int c) {
        Stencil<T> s;
        s.c0 = p[c];
        s.ax = p[c + 1] + p[c - 1];
        s.ay = p[c + WX] + p[c - WX];
        s.az = p[c + WXY] + p[c - WXY];
        s.exy = p[c + 1 + WX] - p[c + 1 - WX] - p[c - 1 + WX] + p[c - 1 - WX];
        s.exz = p[c + 1 + WXY] - p[c + 1 - WXY] - p[c - 1 + WXY] + p[c - 1 - WXY];
        s.eyz = p[c + WX + WXY] - p[c + WX - WXY] - p[c - WX + WXY] + p[c - WX - WXY];
        return s;
    };
    const T gm = gm_ptr ? (T)(*gm_ptr) : T(0);
    const size_t total = (size_t)n * n * n;
    const int x = threadIdx.x & 31, y = (threadIdx.x >> 5) & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int z = (threadIdx.x >> 7) + 2 * h;
        const int cl = ((z + 1) * WY + (y + 1)) * WX + x + 1;
        const size_t c = ((size_t)(Z0 + z) * n + (Y0 + y)) * n + (X0 + x);
        Stencil<T> s = stencil(su, cl);
        Stencil<T> b;
        if (BG) b = stencil(sb, cl);
        T rcv = rc[c];
        if (gm_ptr) {
            const uint8_t kb = kmask[c];
            rcv -= gm * (T)(kb >> 4) * T(0.125);
            kmask[c] = kb & 15;
        }
        const T w = screen_w<T>(kmask, c);
        const T kc = kap * w;
        Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, T(0), T(0));
        fc[c] = o.G + rcv;
        if (BG && coefo) {
            const float Xb = (float)(b.ax - T(2) * b.c0), Yb = (float)(b.ay - T(2) * b.c0),
                        Zb = (float)(b.az - T(2) * b.c0);
            coefo[c] = pack_bf16x2(2.f * (Yb + Zb), 2.f * (Xb + Zb));
            coefo[total + c] = pack_bf16x2(2.f * (Xb + Yb), -0.25f * (float)b.exy);
            coefo[2 * total + c] = pack_bf16x2(-0.25f * (float)b.exz, -0.25f * (float)b.eyz);
            gapo[c] = kc != T(0) ? lsat / (float)w - (float)ih2 * (Xb + Yb + Zb) : 0.f;
        }
    }
}

// fine += trilinear cell-centred prolongation of (uc - ur), periodic.  One thread per
// coarse cell writes its 8 children: the 3x3x3 coarse neighbourhood is interpolated
// separably (weights 3/4 and 1/4 per axis, i.e. 27/64, 9/64, 3/64, 1/64 in 3D), and the
// children are updated as pairs along x (8-byte / 16-byte accesses).
template <typename T>
__device__ __forceinline__ void prolong_add_cell(const T* uc, const T* ur, int nc, int lgc,
                                                 T* uf, size_t c)
{
    const int nf = 2 * nc, mc = nc - 1;
    const T a = T(0.75), b = T(0.25);
    const int I = (int)(c & (size_t)mc);  // nc is a power of two
    const size_t row = c >> lgc;
    const int J = (int)(row & (size_t)mc), K = (int)(row >> lgc);
    const int xs[3] = {(I - 1) & mc, I, (I + 1) & mc};
    const int ys[3] = {(J - 1) & mc, J, (J + 1) & mc};
    const int zs[3] = {(K - 1) & mc, K, (K + 1) & mc};
    // along x: px[z][y][child]
    T px[3][3][2];
#pragma unroll
    for (int kz = 0; kz < 3; ++kz)
#pragma unroll
        for (int jy = 0; jy < 3; ++jy) {
            const size_t base = ((size_t)zs[kz] * nc + ys[jy]) * nc;
            T v[3];
#pragma unroll
            for (int ix = 0; ix < 3; ++ix) v[ix] = ur ? uc[base + xs[ix]] - ur[base + xs[ix]] : uc[base + xs[ix]];
            px[kz][jy][0] = a * v[1] + b * v[0];
            px[kz][jy][1] = a * v[1] + b * v[2];
        }
    // along y, then z, then add to the children
#pragma unroll
    for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy) {
            T out[2];
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) {
                T py[3];
#pragma unroll
                for (int kz = 0; kz < 3; ++kz) py[kz] = a * px[kz][1][dx] + b * px[kz][dy ? 2 : 0][dx];
                out[dx] = a * py[1] + b * py[dz ? 2 : 0];
            }
            T* f = uf + ((size_t)(2 * K + dz) * nf + (2 * J + dy)) * nf + 2 * I;
            f[0] += out[0];
            f[1] += out[1];
        }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add(const T* __restrict__ uc, const T* __restrict__ ur, int nc,
                                                     T* __restrict__ uf)
{
    const int lgc = __ffs(nc) - 1;
    const size_t total = (size_t)nc * nc * nc;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        prolong_add_cell<T>(uc, ur, nc, lgc, uf, c);
}

// The same prolongation for coarse grids of at least 32^3, tiled: a block stages the
// differences uc - ur of a 32 x 4 x 4 coarse brick and its one-cell halo (34 x 6 x 6) in
// shared memory once, then each thread interpolates the children of two coarse cells from
// there (the interpolation and its order as in k_prolong_add) and updates them as x pairs.
// Grid (nc/32, nc/4, nc/4), 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_prolong_add_tile(const T* __restrict__ uc, const T* __restrict__ ur,
                                                          int nc, T* __restrict__ uf)
{
    constexpr int BX = 32, BY = 4, BZ = 4, WX = BX + 2, WY = BY + 2, WZ = BZ + 2, P = WX * WY * WZ;
    __shared__ T sd[P];
    const int mc = nc - 1, nf = 2 * nc;
    const int X0 = blockIdx.x * BX, Y0 = blockIdx.y * BY, Z0 = blockIdx.z * BZ;
    for (int e = threadIdx.x; e < P; e += 256) {
        const int xx = e % WX, yy = (e / WX) % WY, zz = e / (WX * WY);
        const size_t g = ((size_t)((Z0 - 1 + zz) & mc) * nc + ((Y0 - 1 + yy) & mc)) * nc + ((X0 - 1 + xx) & mc);
        sd[e] = ur ? uc[g] - ur[g] : uc[g];
    }
    __syncthreads();
    const T a = T(0.75), b = T(0.25);
    const int x = threadIdx.x & 31, y = (threadIdx.x >> 5) & 3;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int z = (threadIdx.x >> 7) + 2 * h;
        T px[3][3][2];
#pragma unroll
        for (int kz = 0; kz < 3; ++kz)
#pragma unroll
            for (int jy = 0; jy < 3; ++jy) {
                const T* v = sd + ((z + kz) * WY + (y + jy)) * WX + x;
                px[kz][jy][0] = a * v[1] + b * v[0];
                px[kz][jy][1] = a * v[1] + b * v[2];
            }
        const int I = X0 + x, J = Y0 + y, K = Z0 + z;
#pragma unroll
        for (int dz = 0; dz < 2; ++dz)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy) {
                T out[2];
#pragma unroll
                for (int dx = 0; dx < 2; ++dx) {
                    T py[3];
#pragma unroll
                    for (int kz = 0; kz < 3; ++kz) py[kz] = a * px[kz][1][dx] + b * px[kz][dy ? 2 : 0][dx];
                    out[dx] = a * py[1] + b * py[dz ? 2 : 0];
                }
                T* f = uf + ((size_t)(2 * K + dz) * nf + (2 * J + dy)) * nf + 2 * I;
                f[0] += out[0];
                f[1] += out[1];
            }
    }
}

// ------------------------------------------------------------------ coarsest level

// Exact-enough solve of the coarsest level (at most 8^3 cells) in one thread block, in the
// storage type's arithmetic (FP64 for the FP64 cycle, FP32 inside the FP32 inner cycle):
// `sweeps` red-black sweeps, each followed by the gauge update lambda -= sum r / #unfloored.
// The block sums go through warp shuffles and one exchange between the warps.
template <typename T>
struct CoarsestSmem {
    T su[512], ss[512], sf[512], sb[512];
    uint8_t sk[512];
    T red[2][8];
};

// The coarsest solve of one level (at most 8^3 cells) by the calling block, its arrays in sm.
template <typename T, bool BG>
__device__ void coarsest_block(T* u, const T* F, T fscale, const uint8_t* kmask,
                               const T* bg, int n, double ih2_d, double nu_d, double kap_d, double eta,
                               int sweeps, bool floor_piece, CoarsestSmem<T>& sm)
{
    T* su = sm.su;
    T* ss = sm.ss;
    T* sf = sm.sf;
    T* sb = sm.sb;
    uint8_t* sk = sm.sk;
    const int cells = n * n * n, t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const T ih2 = (T)ih2_d, nu = (T)nu_d, kap = (T)kap_d;
    for (int c = t; c < cells; c += blockDim.x) {
        su[c] = u[c];
        sf[c] = fscale * F[c];
        sk[c] = kmask ? kmask[c] : 0;
        sb[c] = BG ? bg[c] : T(0);
    }
    __syncthreads();
    const T sp = nu >= T(0) ? T(-1) : T(1);
    const double sqDf = eta * 6.0 * fabs(nu_d) * ih2_d;
    const T Df = (T)(sqDf * sqDf);
    const T lsat_c = kap != T(0) ? (T)(0.75 * nu_d * (1.0 - eta) / kap_d) : T(0);  // L_sat
    T lam = T(0);
    for (int it = 0; it < sweeps; ++it) {
        for (int colour = 0; colour < 2; ++colour) {
            for (int c = t; c < cells; c += blockDim.x) ss[c] = su[c];
            __syncthreads();
            for (int c = t; c < cells; c += blockDim.x) {
                const int i = c % n, j = (c / n) % n, k = c / (n * n);
                if (((i + j + k) & 1) != colour) continue;
                Stencil<T> s = load_stencil<T>(ss, ss, i, j, k, n);
                Stencil<T> b;
                if (BG) b = load_stencil<T>(sb, sb, i, j, k, n);
                const T w = sk[c] >= 8 ? T(0) : (T)(8 - sk[c]) * T(0.125);
                const T kc = kap * w;
                Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, sf[c] + lam, kc != T(0) ? (kmask ? lsat_c / w : lsat_c) : T(0));
                su[c] = s.c0 + local_update(o, sp, Df, ih2);
            }
            __syncthreads();
        }
        // gauge update from the residual
        T a0 = T(0), a1 = T(0);
        for (int c = t; c < cells; c += blockDim.x) {
            const int i = c % n, j = (c / n) % n, k = c / (n * n);
            Stencil<T> s = load_stencil<T>(su, su, i, j, k, n);
            Stencil<T> b;
            if (BG) b = load_stencil<T>(sb, sb, i, j, k, n);
            const T w = sk[c] >= 8 ? T(0) : (T)(8 - sk[c]) * T(0.125);
            const T kc = kap * w;
            Local<T> o = local_eval<T, BG>(s, b, ih2, nu, kc, sf[c] + lam, kc != T(0) ? (kmask ? lsat_c / w : lsat_c) : T(0));
            const bool fl = (o.P != T(0)) && (o.D < (floor_piece ? Df : T(0)));
            a0 += fl ? nu * o.g : -o.G;
            a1 += fl ? T(0) : T(1);
        }
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_down_sync(0xffffffffu, a0, o);
            a1 += __shfl_down_sync(0xffffffffu, a1, o);
        }
        if (lane == 0) {
            sm.red[0][wid] = a0;
            sm.red[1][wid] = a1;
        }
        __syncthreads();
        T s0 = T(0), s1 = T(0);
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {  // every thread, the same order
            s0 += sm.red[0][q];
            s1 += sm.red[1][q];
        }
        if (s1 > T(0)) lam -= s0 / s1;
        __syncthreads();
    }
    for (int c = t; c < cells; c += blockDim.x) u[c] = su[c];
}

template <typename T, bool BG>
__global__ void __launch_bounds__(256) k_coarsest(T* __restrict__ u, const T* __restrict__ F, T fscale,
                                                  const uint8_t* __restrict__ kmask, const T* __restrict__ bg, int n,
                                                  double ih2_d, double nu_d, double kap_d, double eta, int sweeps,
                                                  bool floor_piece)
{
    __shared__ CoarsestSmem<T> sm;
    coarsest_block<T, BG>(u, F, fscale, kmask, bg, n, ih2_d, nu_d, kap_d, eta, sweeps, floor_piece, sm);
}

// ------------------------------------------------------------------ exact coarsest solve

// Exact solve of a coarsest level of at most kExactMaxCells cells, in FP64 whatever the
// storage type, in one block: Newton's method on the level's whole discrete system (the
// paper's FAS leaves the coarse solve open; Sec. 3.4), its Jacobian written out as a dense
// matrix and solved by LU with partial pivoting.  Unknowns: the m cell values and the gauge
// multiplier lambda.  Equations: each cell's residual piece with its sign flipped (N - f -
// lambda where the discriminant has a real root, nu (L - L_sat) where it is floored; Sec. 3.3)
// and the mean constraint sum(chi) = its value on entry, scaled by 6|nu|/h^2.  The floored set
// is taken afresh at every iterate, and a backtracking line search on |F| keeps each step from
// increasing it.  Stops at |F| <= 1e-14 |f - <f>| or after kExactMaxIter iterations.  With a
// background (the FP32 inner cycle's correction form) the unknown is the total field bg + u
// and the right-hand side f + N(bg), i.e. N(bg + u) - N(bg) = f + lambda; u is written back
// in the storage type.  lam_out (nullable) receives lambda.
constexpr int kExactMaxCells = 64;
constexpr int kExactThreads = 128;
constexpr int kExactMaxIter = 30;

template <bool JAC>
__device__ double exact_eval(const double* __restrict__ x, double lam, const double* __restrict__ rhs,
                             const double* __restrict__ wk, int n, double ih2, double nu, double kap, double eta,
                             double* __restrict__ Fv, double* __restrict__ J, int ld, double* red, double scale,
                             double msum)
{
    const int m = n * n * n, t = threadIdx.x, M = m + 1;
    const double sqDf = eta * 6.0 * fabs(nu) * ih2, Df = sqDf * sqDf;
    double f2 = 0.0;
    for (int c = t; c < m; c += blockDim.x) {
        const int mm = n - 1, i = c & mm, j = (c / n) & mm, k = c / (n * n);
        const Stencil<double> s = load_stencil<double>(x, x, i, j, k, n);
        const double kc = kap * wk[c];
        const double lsat = kc != 0.0 ? 0.75 * nu * (1.0 - eta) / kc : 0.0;
        const Local<double> o = local_eval<double, false>(s, s, ih2, nu, kc, rhs[c] + lam, lsat);
        const bool fl = (o.P != 0.0) && (o.D < Df);
        const double Fc = fl ? -nu * o.g : o.G;  // nu (L - L_sat) = -nu g
        Fv[c] = Fc;
        f2 += Fc * Fc;
        if (!JAC) continue;
        double* row = J + (size_t)c * ld;
        for (int q = 0; q < M; ++q) row[q] = 0.0;
        auto at = [&](int di, int dj, int dk) { return (((k + dk) & mm) * n + ((j + dj) & mm)) * n + ((i + di) & mm); };
        row[c] += -6.0 * nu * ih2;
        const int fo[6][3] = {{1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1}};
        for (int q = 0; q < 6; ++q) row[at(fo[q][0], fo[q][1], fo[q][2])] += nu * ih2;
        if (fl) continue;
        row[m] = -1.0;
        if (kc == 0.0) continue;
        // -kappa dq2, q2 = 2(XY + YZ + ZX) - 2(cxy^2 + cxz^2 + cyz^2), physical units
        const double X = (s.ax - 2.0 * s.c0) * ih2, Y = (s.ay - 2.0 * s.c0) * ih2, Z = (s.az - 2.0 * s.c0) * ih2;
        const double dq[3] = {2.0 * (Y + Z), 2.0 * (X + Z), 2.0 * (X + Y)};
        row[c] -= kc * (-2.0 * ih2) * (dq[0] + dq[1] + dq[2]);
        for (int q = 0; q < 6; ++q) row[at(fo[q][0], fo[q][1], fo[q][2])] -= kc * dq[q / 2] * ih2;
        const double cc[3] = {s.exy * 0.25 * ih2, s.exz * 0.25 * ih2, s.eyz * 0.25 * ih2};
        const int ax[3][2] = {{0, 1}, {0, 2}, {1, 2}};
        for (int q = 0; q < 3; ++q)
            for (int s1 = -1; s1 <= 1; s1 += 2)
                for (int s2 = -1; s2 <= 1; s2 += 2) {
                    int o3[3] = {0, 0, 0};
                    o3[ax[q][0]] = s1;
                    o3[ax[q][1]] = s2;
                    // d(-2 c^2)/dc = -4c and dc/d(corner) = s1 s2 / (4 h^2)
                    row[at(o3[0], o3[1], o3[2])] += kc * cc[q] * (double)(s1 * s2) * ih2;
                }
    }
    // the mean row
    double sx = 0.0;
    for (int c = t; c < m; c += blockDim.x) sx += x[c];
    for (int o = 16; o > 0; o >>= 1) {
        f2 += __shfl_down_sync(0xffffffffu, f2, o);
        sx += __shfl_down_sync(0xffffffffu, sx, o);
    }
    const int lane = t & 31, wid = t >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        red[wid] = f2;
        red[8 + wid] = sx;
    }
    __syncthreads();
    double a = 0.0, b = 0.0;
    for (int q = 0; q < nw; ++q) {  // every thread, the same order
        a += red[q];
        b += red[8 + q];
    }
    const double Fm = scale * (b - msum);
    if (t == 0) Fv[m] = Fm;
    if (JAC)
        for (int q = t; q < m; q += blockDim.x) J[(size_t)m * ld + q] = scale;
    if (JAC && t == 0) J[(size_t)m * ld + m] = 0.0;
    __syncthreads();
    return sqrt(a + Fm * Fm);
}

template <typename T, bool BG>
__global__ void __launch_bounds__(kExactThreads) k_coarsest_exact(T* __restrict__ u, const T* __restrict__ F,
                                                                  T fscale, const uint8_t* __restrict__ kmask,
                                                                  const T* __restrict__ bg, int n, double ih2,
                                                                  double nu, double kap, double eta,
                                                                  double* __restrict__ lam_out)
{
    constexpr int MX = kExactMaxCells + 1, LD = MX + 1;
    __shared__ double J[MX * LD];
    __shared__ double b[MX], Fv[MX];
    __shared__ double x[kExactMaxCells], xt[kExactMaxCells], rhs[kExactMaxCells], wk[kExactMaxCells];
    __shared__ double red[16];
    __shared__ int piv;
    __shared__ bool singular;
    const int m = n * n * n, M = m + 1, t = threadIdx.x;
    const double scale = 6.0 * fabs(nu) * ih2;
    for (int c = t; c < m; c += blockDim.x) {
        x[c] = (double)u[c] + (BG ? (double)bg[c] : 0.0);
        wk[c] = kmask ? (kmask[c] >= 8 ? 0.0 : (double)(8 - kmask[c]) * 0.125) : 1.0;
        xt[c] = BG ? (double)bg[c] : 0.0;
    }
    __syncthreads();
    // right-hand side f (+ N(bg) in the correction form) and its centred norm
    double fs = 0.0, fq = 0.0;
    for (int c = t; c < m; c += blockDim.x) {
        double r = (double)fscale * (double)F[c];
        if (BG) {
            const int mm = n - 1, i = c & mm, j = (c / n) & mm, k = c / (n * n);
            const Stencil<double> s = load_stencil<double>(xt, xt, i, j, k, n);
            const double kc = kap * wk[c];
            r += local_eval<double, false>(s, s, ih2, nu, kc, 0.0, 0.0).G;  // N(bg)
        }
        rhs[c] = r;
        fs += r;
        fq += r * r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        fs += __shfl_down_sync(0xffffffffu, fs, o);
        fq += __shfl_down_sync(0xffffffffu, fq, o);
    }
    if ((t & 31) == 0) {
        red[t >> 5] = fs;
        red[8 + (t >> 5)] = fq;
    }
    __syncthreads();
    double sfs = 0.0, sfq = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
        sfs += red[q];
        sfq += red[8 + q];
    }
    const double fnorm = sqrt(fmax(sfq - sfs * sfs / (double)m, 0.0));
    double msum = 0.0;
    for (int c = 0; c < m; ++c) msum += x[c];  // every thread, the same order
    __syncthreads();
    double lam = 0.0;
    double nrm = exact_eval<true>(x, lam, rhs, wk, n, ih2, nu, kap, eta, Fv, J, LD, red, scale, msum);
    for (int it = 0; it < kExactMaxIter; ++it) {
        if (!(nrm > 1e-14 * fnorm) || nrm == 0.0) break;
        // J d = -F by LU with partial pivoting (the multipliers stored below the diagonal)
        for (int q = t; q < M; q += blockDim.x) b[q] = -Fv[q];
        if (t == 0) singular = false;
        __syncthreads();
        for (int k = 0; k < M; ++k) {
            if (t < 32) {
                double best = -1.0;
                int bi = k;
                for (int i = k + t; i < M; i += 32) {
                    const double v = fabs(J[(size_t)i * LD + k]);
                    if (v > best) {
                        best = v;
                        bi = i;
                    }
                }
                for (int o = 16; o > 0; o >>= 1) {
                    const double ov = __shfl_down_sync(0xffffffffu, best, o);
                    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
                    if (ov > best || (ov == best && oi < bi)) {
                        best = ov;
                        bi = oi;
                    }
                }
                if (t == 0) {
                    piv = bi;
                    if (best == 0.0) singular = true;
                }
            }
            __syncthreads();
            if (singular) break;
            const int p = piv;
            if (p != k) {
                for (int q = k + t; q < M; q += blockDim.x) {
                    const double a = J[(size_t)k * LD + q];
                    J[(size_t)k * LD + q] = J[(size_t)p * LD + q];
                    J[(size_t)p * LD + q] = a;
                }
                if (t == 0) {
                    const double a = b[k];
                    b[k] = b[p];
                    b[p] = a;
                }
                __syncthreads();
            }
            const double dinv = 1.0 / J[(size_t)k * LD + k];
            for (int i = k + 1 + t; i < M; i += blockDim.x) J[(size_t)i * LD + k] *= dinv;
            __syncthreads();
            const int w = M - k;  // columns k..M-1; column k carries the right-hand side update
            for (int q = t; q < (M - k - 1) * w; q += blockDim.x) {
                const int i = k + 1 + q / w, j = k + q % w;
                const double l = J[(size_t)i * LD + k];
                if (j == k) b[i] -= l * b[k];
                else J[(size_t)i * LD + j] -= l * J[(size_t)k * LD + j];
            }
            __syncthreads();
        }
        if (singular) break;
        for (int k = M - 1; k >= 0; --k) {
            if (t == 0) b[k] /= J[(size_t)k * LD + k];
            __syncthreads();
            for (int i = t; i < k; i += blockDim.x) b[i] -= J[(size_t)i * LD + k] * b[k];
            __syncthreads();
        }
        // backtracking line search on |F|
        double step = 1.0, nt = nrm, lt = lam;
        for (;;) {
            for (int c = t; c < m; c += blockDim.x) xt[c] = x[c] + step * b[c];
            lt = lam + step * b[m];
            __syncthreads();
            nt = exact_eval<false>(xt, lt, rhs, wk, n, ih2, nu, kap, eta, Fv, J, LD, red, scale, msum);
            if (nt < (1.0 - 1e-4 * step) * nrm || step < 1e-4) break;
            step *= 0.5;
        }
        if (!(nt < nrm)) break;  // no decrease along the Newton direction: keep the iterate
        for (int c = t; c < m; c += blockDim.x) x[c] = xt[c];
        lam = lt;
        __syncthreads();
        nrm = exact_eval<true>(x, lam, rhs, wk, n, ih2, nu, kap, eta, Fv, J, LD, red, scale, msum);
    }
    for (int c = t; c < m; c += blockDim.x) u[c] = (T)(x[c] - (BG ? (double)bg[c] : 0.0));
    if (lam_out && t == 0) *lam_out = lam;
}

// ------------------------------------------------------------------ misc

template <typename T>
__global__ void k_sum(const T* __restrict__ x, size_t total, double* __restrict__ partials,
                      double* __restrict__ fin_out = nullptr)
{
    double v[2] = {0.0, 0.0};
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    if constexpr (sizeof(T) == 4) {
        // FP32 data: 16-byte loads and FP32 per-thread sums (a few hundred terms each; the
        // FP64 pipe would otherwise bound the pass), FP64 across threads
        float a = 0.f, b = 0.f;
        const size_t n4 = total / 4;
        const float4* x4 = reinterpret_cast<const float4*>(x);
        for (size_t c = tid; c < n4; c += stride) {
            const float4 q = x4[c];
            a += (q.x + q.y) + (q.z + q.w);
            b += (q.x * q.x + q.y * q.y) + (q.z * q.z + q.w * q.w);
        }
        for (size_t c = 4 * n4 + tid; c < total; c += stride) {
            a += (float)x[c];
            b += (float)x[c] * (float)x[c];
        }
        v[0] = a;
        v[1] = b;
    } else {
        for (size_t c = tid; c < total; c += stride) {
            const double d = (double)x[c];
            v[0] += d;
            v[1] += d * d;
        }
    }
    block_sums<2>(v, partials, fin_out);
}

// sum of (x - mean)^2 with the mean read from the device
__global__ void k_sum_centred(const double* __restrict__ x, size_t total, const double* __restrict__ sums,
                              double* __restrict__ partials, double* __restrict__ fin_out = nullptr)
{
    const double mean = sums[0] / (double)total;
    double v[1] = {0.0};
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const double d = x[c] - mean;
        v[0] += d * d;
    }
    block_sums<1>(v, partials, fin_out);
}

template <typename T>
__global__ void k_sub_mean(T* __restrict__ x, size_t total, const double* __restrict__ sums)
{
    const T mean = (T)(sums[0] / (double)total);
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        x[c] -= mean;
}

__global__ void k_add_correction(double* __restrict__ x, const float* __restrict__ e, size_t total)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        x[c] += (double)e[c];
}

// The bilinear coefficients of a background field b (BgCoef in internal.cuh) packed to BF16
// pairs, as the finest inner level of a large solve receives them from the outer residual:
// (2(Yb+Zb), 2(Xb+Zb)), (2(Xb+Yb), -bxy/4), (-bxz/4, -byz/4), h = 1 units.
__global__ void k_bg_coef(const float* __restrict__ bg, int n, uint32_t* __restrict__ coef)
{
    const size_t total = (size_t)n * n * n;
    const int lg = __ffs(n) - 1;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c & (size_t)(n - 1));
        const size_t row = c >> lg;
        const int j = (int)(row & (size_t)(n - 1)), k = (int)(row >> lg);
        const Stencil<float> b = load_stencil<float>(bg, bg, i, j, k, n);
        const float Xb = b.ax - 2.f * b.c0, Yb = b.ay - 2.f * b.c0, Zb = b.az - 2.f * b.c0;
        coef[c] = pack_bf16x2(2.f * (Yb + Zb), 2.f * (Xb + Zb));
        coef[total + c] = pack_bf16x2(2.f * (Xb + Yb), -0.25f * b.exy);
        coef[2 * total + c] = pack_bf16x2(-0.25f * b.exz, -0.25f * b.eyz);
    }
}

// x += e - <e> in FP64, the mean of e read from the device (sums[0] = sum e)
__global__ void k_add_correction_centred(double* __restrict__ x, const float* __restrict__ e, size_t total,
                                         const double* __restrict__ sums)
{
    const double mean = sums[0] / (double)total;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        x[c] += (double)e[c] - mean;
}

// ------------------------------------------------------------------ host drivers

struct Coef {
    double nu, kap, eta, src;
};

constexpr int kFusedMinN = 64;  // single-pass candidates from this size up (the autotuner chooses)
constexpr int kResidZmMinN = 128;  // FP32 residual: z-marching kernel from this size up

// Tile variants of the single-pass FP32 sweep: (TX, TY) x-y tile, NZ planes per block.
struct FusedCfg {
    int tx, ty, nz;
    bool pair;  // k_sweep_pair (two cells per thread) instead of k_sweep_fused
    bool bal;   // k_sweep_pair with one warp per red unit (coefficient levels)
    bool col;   // k_sweep_col (column-resident stencils; coefficient levels without a mask)
};
static const FusedCfg kFusedCfgs[] = {
    {64, 16, 32, false, false, false}, {64, 8, 32, false, false, false}, {64, 8, 64, false, false, false},
    {32, 8, 32, false, false, false},  {32, 8, 64, false, false, false}, {64, 4, 64, false, false, false},
    {64, 16, 16, false, false, false}, {64, 8, 16, false, false, false}, {64, 8, 32, true, false, false},
    {64, 8, 64, true, false, false},   {64, 16, 32, true, false, false}, {64, 16, 64, true, false, false},
    {64, 4, 64, true, false, false},   {64, 8, 16, true, false, false},  {64, 16, 32, true, true, false},
    {64, 8, 32, true, true, false},    {64, 8, 32, false, false, true},  {64, 8, 64, false, false, true},
    {64, 16, 32, false, false, true},  {64, 16, 64, false, false, true},  {64, 16, 16, true, true, false},
    {64, 8, 16, true, true, false}};
constexpr int kNumFusedCfgs = sizeof(kFusedCfgs) / sizeof(kFusedCfgs[0]);

template <int TX, int TY, bool BG, bool GAP>
static void launch_fused(Exec* ctx, const float* A, float* B, const float* F, float fscale, float lam,
                         const Level<float>& L, int nz, float h2inv, const Coef& c, float sp, float Df, float lsn)
{
    const int n = L.n;
    constexpr size_t sm = fused_smem_bytes<float, TX, TY, BG, GAP>();
    auto k = k_sweep_fused<float, TX, TY, BG, GAP>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const dim3 grid(n / TX, n / TY, n / nz);
    k<<<grid, 256, sm, ctx->stream>>>(A, B, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz, h2inv, (float)c.nu,
                                      (float)c.kap, sp, Df, lsn, L.lamp);
}

template <int TY, bool BG, bool GAP, bool COEF = false, bool BAL = false>
static void launch_pair(Exec* ctx, const float* A, float* B, const float* F, float fscale, float lam,
                        const Level<float>& L, int nz, float h2inv, const Coef& c, float sp, float Df, float lsn)
{
    const int n = L.n;
    constexpr size_t sm = pair_smem_bytes<TY, BG, COEF>();
    auto k = k_sweep_pair<TY, BG, GAP, COEF, BAL>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const dim3 grid(n / 64, n / TY, n / nz);
    k<<<grid, PairGeom<TY, BAL>::NT, sm, ctx->stream>>>(A, B, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz, h2inv,
                                                   (float)c.nu, (float)c.kap, sp, Df, lsn, L.lamp,
                                                   COEF ? L.coef : nullptr);
}

template <int TY>
static void launch_col(Exec* ctx, const float* A, float* B, const float* F, float fscale, float lam,
                       const Level<float>& L, int nz, float h2inv, const Coef& c, float sp, float Df, float lsn)
{
    const int n = L.n;
    constexpr size_t sm = col_smem_bytes<TY>();
    auto k = k_sweep_col<TY>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    const dim3 grid(n / 64, n / TY, n / nz);
    k<<<grid, ColGeom<TY>::NT, sm, ctx->stream>>>(A, B, F, fscale, lam, L.gap, n, nz, h2inv, (float)c.nu,
                                                  (float)c.kap, sp, Df, lsn, L.lamp, L.coef);
}

// the column kernel's inputs: background coefficients and gap, no screening mask
static bool col_level(const Level<float>& L) { return L.bg && L.gap && L.coef && !L.kmask; }

template <bool BG, bool GAP>
static void launch_fused_cfg(Exec* ctx, int cfg, const float* A, float* B, const float* F, float fscale, float lam,
                             const Level<float>& L, float h2inv, const Coef& c, float sp, float Df, float lsn)
{
    const FusedCfg& g = kFusedCfgs[cfg];
    if (g.col) {
        if (g.ty == 8) launch_col<8>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn);
        else launch_col<16>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn);
        return;
    }
#define PM_FUSED_CASE(TX_, TY_)                                                                        \
    if (!g.pair && g.tx == TX_ && g.ty == TY_) {                                                       \
        launch_fused<TX_, TY_, BG, GAP>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn);    \
        return;                                                                                        \
    }
#define PM_PAIR_CASE(TY_)                                                                              \
    if (g.pair && g.ty == TY_) {                                                                       \
        if (BG && GAP && L.coef && g.bal)                                                              \
            launch_pair<TY_, true, true, true, true>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn); \
        else if (BG && GAP && L.coef)                                                                  \
            launch_pair<TY_, true, true, true>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn); \
        else                                                                                           \
            launch_pair<TY_, BG, GAP>(ctx, A, B, F, fscale, lam, L, g.nz, h2inv, c, sp, Df, lsn);      \
        return;                                                                                        \
    }
    PM_FUSED_CASE(64, 16)
    PM_FUSED_CASE(64, 8)
    PM_FUSED_CASE(32, 8)
    PM_FUSED_CASE(64, 4)
    PM_PAIR_CASE(16)
    PM_PAIR_CASE(8)
    PM_PAIR_CASE(4)
#undef PM_FUSED_CASE
#undef PM_PAIR_CASE
}

static bool fused_cfg_fits(int cfg, int n)
{
    const FusedCfg& g = kFusedCfgs[cfg];
    return n >= g.tx && n >= g.ty && n >= g.nz && n % g.tx == 0 && n % g.ty == 0 && n % g.nz == 0;
}

// a variant that can sweep level L: the column kernel only on coefficient levels without a
// mask, the balanced pair kernel only on coefficient levels
static bool fused_cfg_usable(int cfg, const Level<float>& L)
{
    const FusedCfg& g = kFusedCfgs[cfg];
    if (!fused_cfg_fits(cfg, L.n)) return false;
    if (g.col) return col_level(L);
    if (g.bal) return L.coef && L.gap;
    if (L.coef && L.gap) return g.pair;  // only the pair kernels read coefficients
    return true;
}

// One red-black sweep of an FP32 level in a single pass (k_sweep_fused) with tile variant cfg.
static void sweep_fused_f32(Exec* ctx, Level<float>& L, const float* F, float fscale, float lam, const Coef& c,
                            int cfg)
{
    const int n = L.n;
    const float h2inv = (float)((double)n * (double)n);
    const float sp = c.nu >= 0.0 ? -1.f : 1.f;
    const double sqDf = c.eta * 6.0 * std::fabs(c.nu) * (double)n * (double)n;
    const float Df = (float)(sqDf * sqDf);
    const float lsn = c.kap != 0.0 ? (float)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : 0.f;  // L_sat
    float* A = L.u[L.cur];
    float* B = L.u[1 - L.cur];
    ctx->begin(PM_K_SWEEP32, L.fine, (long long)L.cells);
    if (L.bg && L.gap) launch_fused_cfg<true, true>(ctx, cfg, A, B, F, fscale, lam, L, h2inv, c, sp, Df, lsn);
    else if (L.bg) launch_fused_cfg<true, false>(ctx, cfg, A, B, F, fscale, lam, L, h2inv, c, sp, Df, lsn);
    else launch_fused_cfg<false, false>(ctx, cfg, A, B, F, fscale, lam, L, h2inv, c, sp, Df, lsn);
    ctx->end();
    L.cur = 1 - L.cur;
}

template <typename T>
static void sweep_halves(Exec* ctx, Level<T>& L, const T* F, T fscale, T lam, const Coef& c);

// Autotuner: the first time a level of size n (with a given input set) is swept, every
// fitting tile variant runs once on the real data (out of place, A -> B, so the state is
// unchanged whichever runs last) and the fastest is kept for that key.
static int tuned_cfg(Exec* ctx, Level<float>& L, const float* F, float fscale, float lam, const Coef& c)
{
    const bool cf = L.coef && L.gap;
    const int key = L.n * 16 + (L.kmask ? 8 : 0) + (cf ? 4 : 0) + (L.bg ? 2 : 0) + (L.gap ? 1 : 0);
    auto it = ctx->tuned.find(key);
    if (it != ctx->tuned.end()) return it->second;
    int best = 0;
    if (cf)  // only the pair kernel reads coefficients: start from its first variant
        while (best + 1 < kNumFusedCfgs && !kFusedCfgs[best].pair) ++best;
    if (ctx->prm.autotune) {
        float best_ms = 1e30f;
        std::string trials;  // "variant:ms" of every candidate
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        const bool was = ctx->c->tracing;
        ctx->c->tracing = false;
        for (int cfg = -1; cfg < kNumFusedCfgs; ++cfg) {  // -1: the two half-sweep launches
            if (cfg >= 0 && !fused_cfg_usable(cfg, L)) continue;
            // one untimed launch, then three timed back to back
            for (int rep = 0; rep < 2; ++rep) {
                const int launches = rep == 0 ? 1 : 3;
                cudaEventRecord(e0, ctx->stream);
                for (int q = 0; q < launches; ++q) {
                    if (cfg < 0) sweep_halves(ctx, L, F, fscale, lam, c);
                    else sweep_fused_f32(ctx, L, F, fscale, lam, c, cfg);
                    L.cur = 1 - L.cur;  // keep A as the input of every trial
                }
                cudaEventRecord(e1, ctx->stream);
                cudaEventSynchronize(e1);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                ms /= (float)launches;
                if (rep == 1) {
                    trials += " " + std::to_string(cfg) + ":" + std::to_string(ms).substr(0, 6);
                    if (ms < best_ms) {
                        best_ms = ms;
                        best = cfg;
                    }
                }
            }
        }
        ctx->c->tracing = was;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        std::string choice = "two half-sweep launches";
        if (best >= 0) {
            const FusedCfg& g = kFusedCfgs[best];
            choice = "tile " + std::to_string(g.tx) + "x" + std::to_string(g.ty) + " nz " + std::to_string(g.nz) +
                     (g.col ? " col" : g.pair ? (g.bal ? " pair bal" : " pair") : " single");
        }
        ctx->tune_log += "sweep32 n=" + std::to_string(L.n) + (L.bg ? " bg" : "") + (L.gap ? " gap" : "") +
                         (L.kmask ? " mask" : "") + (cf ? " coef" : "") + ": " + choice + " " +
                         std::to_string(best_ms) + " ms (variants tried, ms:" + trials + ")\n";
    } else if (L.n < kCoefMinN) {
        best = -1;  // without timing, the levels below the coefficient levels keep the half-sweeps
    }
    ctx->tuned[key] = best;
    return best;
}

// One red-black sweep as two half-sweep launches (one per colour), out of place: A = u[cur]
// is read, B = u[1 - cur] receives the new values, then cur flips.
template <typename T>
static void sweep_halves(Exec* ctx, Level<T>& L, const T* F, T fscale, T lam, const Coef& c)
{
    const int n = L.n;
    const T h2inv = (T)((double)n * (double)n);
    const T sp = c.nu >= 0.0 ? T(-1) : T(1);
    const double sqDf = c.eta * 6.0 * std::fabs(c.nu) * (double)n * (double)n;
    const T lsn = c.kap != 0.0 ? (T)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : T(0);  // L_sat
    const int grid = grid_for(ctx, L.cells / 2);
    T* A = L.u[L.cur];
    T* B = L.u[1 - L.cur];
    const bool bg = L.bg != nullptr;
    for (int colour = 0; colour < 2; ++colour) {
        const T* own = A;
        const T* oth = colour == 0 ? A : B;
        if (bg) {
            ctx->begin(sizeof(T) == 8 ? PM_K_SWEEP64 : PM_K_SWEEP32, L.fine, (long long)(L.cells / 2));
            k_half_sweep<T, true><<<grid, kThreads, 0, ctx->stream>>>(own, oth, B, F, fscale, lam, L.kmask, L.bg,
                                                                      L.gap, n, colour, h2inv, (T)c.nu, (T)c.kap, sp,
                                                                      (T)(sqDf * sqDf), lsn, L.lamp, T(0));
            ctx->end();
        } else {
            ctx->begin(sizeof(T) == 8 ? PM_K_SWEEP64 : PM_K_SWEEP32, L.fine, (long long)(L.cells / 2));
            // Method II where the parameters ask for it (the FP64 cycle; FP32 levels keep Method I)
            const bool ops = sizeof(T) == 8 && ctx->prm.smoother == 1;
            const T etanu = (T)(c.eta * std::fabs(c.nu));
            if (ops)
                k_half_sweep<T, false, true><<<grid, kThreads, 0, ctx->stream>>>(
                    own, oth, B, F, fscale, lam, L.kmask, nullptr, nullptr, n, colour, h2inv, (T)c.nu, (T)c.kap, sp,
                    (T)(sqDf * sqDf), lsn, L.lamp, etanu);
            else
                k_half_sweep<T, false><<<grid, kThreads, 0, ctx->stream>>>(
                    own, oth, B, F, fscale, lam, L.kmask, nullptr, nullptr, n, colour, h2inv, (T)c.nu, (T)c.kap, sp,
                    (T)(sqDf * sqDf), lsn, L.lamp, etanu);
            ctx->end();
        }
    }
    L.cur = 1 - L.cur;
}

// The first sweep of a coefficient level whose iterate is zero (L.zero): the zero-start kernel
// writes the swept field into the other buffer; the zero iterate itself was never stored.
// Variants (rows per block, planes of fields loaded ahead); the autotuner times them on the
// first use of each size, as it does the general sweep's tiles.
struct ZeroCfg {
    int tx, ty, pf;
};
static const ZeroCfg kZeroCfgs[] = {{64, 8, 1}, {64, 8, 2}, {64, 16, 1}, {64, 16, 2}, {128, 4, 1}, {128, 8, 1}};
constexpr int kNumZeroCfgs = sizeof(kZeroCfgs) / sizeof(kZeroCfgs[0]);
static bool zero_start_level(const Level<float>& L) { return col_level(L) && L.n >= 64; }

template <int TX, int TY, int PF>
static void launch_zero(Exec* ctx, float* V, const float* F, float fscale, float lam, const Level<float>& L,
                        float h2inv, const Coef& c, float sp, float Df, float lsn)
{
    const int n = L.n;
    const int nz = n < 32 ? n : 32;
    const dim3 grid(n / TX, n / TY, n / nz);
    k_sweep_zero<TX, TY, PF><<<grid, ZeroGeom<TX, TY>::NT, 0, ctx->stream>>>(V, F, fscale, lam, L.gap, n, nz, h2inv,
                                                                     (float)c.nu, (float)c.kap, sp, Df, lsn, L.lamp,
                                                                     L.coef);
}

static void launch_zero_cfg(Exec* ctx, int cfg, const float* F, float fscale, float lam, Level<float>& L,
                            const Coef& c)
{
    const int n = L.n;
    const float h2inv = (float)((double)n * (double)n);
    const float sp = c.nu >= 0.0 ? -1.f : 1.f;
    const double sqDf = c.eta * 6.0 * std::fabs(c.nu) * (double)n * (double)n;
    const float Df = (float)(sqDf * sqDf);
    const float lsn = c.kap != 0.0 ? (float)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : 0.f;  // L_sat
    float* V = L.u[1 - L.cur];
    switch (cfg) {
    case 0: launch_zero<64, 8, 1>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    case 1: launch_zero<64, 8, 2>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    case 2: launch_zero<64, 16, 1>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    case 3: launch_zero<64, 16, 2>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    case 4: launch_zero<128, 4, 1>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    default: launch_zero<128, 8, 1>(ctx, V, F, fscale, lam, L, h2inv, c, sp, Df, lsn); break;
    }
}

static bool zero_cfg_fits(int cfg, int n) { return n % kZeroCfgs[cfg].tx == 0 && n % kZeroCfgs[cfg].ty == 0; }

// force_cfg >= 0: that variant instead of the autotuner's choice
static void sweep_zero_f32(Exec* ctx, Level<float>& L, const float* F, float fscale, float lam, const Coef& c,
                           int force_cfg = -1)
{
    const int key = -L.n;  // the general sweep's keys are positive
    auto it = ctx->tuned.find(key);
    int best = 0;
    if (force_cfg >= 0) {
        best = force_cfg;
    } else if (it != ctx->tuned.end()) {
        best = it->second;
    } else {
        if (ctx->prm.autotune) {
            float best_ms = 1e30f;
            std::string trials;
            cudaEvent_t e0, e1;
            cudaEventCreate(&e0);
            cudaEventCreate(&e1);
            for (int cfg = 0; cfg < kNumZeroCfgs; ++cfg) {
                if (!zero_cfg_fits(cfg, L.n)) continue;
                for (int rep = 0; rep < 2; ++rep) {  // one untimed launch, then three timed
                    const int launches = rep == 0 ? 1 : 3;
                    cudaEventRecord(e0, ctx->stream);
                    for (int q = 0; q < launches; ++q) launch_zero_cfg(ctx, cfg, F, fscale, lam, L, c);
                    cudaEventRecord(e1, ctx->stream);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= (float)launches;
                    if (rep == 1) {
                        trials += " " + std::to_string(cfg) + ":" + std::to_string(ms).substr(0, 6);
                        if (ms < best_ms) {
                            best_ms = ms;
                            best = cfg;
                        }
                    }
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            ctx->tune_log += "sweep32 zero-start n=" + std::to_string(L.n) + ": tile " +
                             std::to_string(kZeroCfgs[best].tx) + "x" + std::to_string(kZeroCfgs[best].ty) + " ahead " + std::to_string(kZeroCfgs[best].pf) +
                             " " + std::to_string(best_ms) + " ms (variants tried, ms:" + trials + ")\n";
        }
        ctx->tuned[key] = best;
    }
    // traced as an FP32 sweep but not as a finest-level launch: the finest-level class times
    // the general sweep kernel
    ctx->begin(PM_K_SWEEP32, false, 0);
    launch_zero_cfg(ctx, best, F, fscale, lam, L, c);
    ctx->end();
    L.cur = 1 - L.cur;
    L.zero = false;
}

// Start level L's iterate at zero: either mark it for the zero-start sweep (FP32 coefficient
// levels, when the first thing to touch the iterate is a sweep) or clear it.
template <typename T>
static void start_at_zero(Exec* ctx, Level<T>& L)
{
    L.cur = 0;
    L.zero = false;
    if constexpr (sizeof(T) == 4) {
        if (ctx->prm.zero_start && ctx->prm.npre >= 1 && zero_start_level(L)) {
            L.zero = true;
            return;
        }
    }
    cudaMemsetAsync(L.u[0], 0, L.cells * sizeof(T), ctx->stream);
}

template <typename T>
static void sweep(Exec* ctx, Level<T>& L, const T* F, T fscale, T lam, const Coef& c, int force_mode = -1)
{
    if constexpr (sizeof(T) == 4) {
        if (L.zero) {
            sweep_zero_f32(ctx, L, F, fscale, lam, c);
            return;
        }
    }
    // FP32 levels of at least kFusedMinN^3: the autotuner's choice among the single-pass
    // kernels and the two half-sweep launches (force_mode 0: the half-sweeps, k >= 1: tile
    // variant k - 1, -1: the autotuner's choice)
    if constexpr (sizeof(T) == 4) {
        if (force_mode >= 1 && force_mode <= kNumFusedCfgs && fused_cfg_usable(force_mode - 1, L)) {
            sweep_fused_f32(ctx, L, F, fscale, lam, c, force_mode - 1);
            return;
        }
        if (force_mode < 0 && L.n >= kFusedMinN && fused_cfg_fits(0, L.n)) {
            const int cfg = tuned_cfg(ctx, L, F, fscale, lam, c);
            if (cfg >= 0) {
                sweep_fused_f32(ctx, L, F, fscale, lam, c, cfg);
                return;
            }
        }
    }
    sweep_halves(ctx, L, F, fscale, lam, c);
}

template <typename T, bool WRITE_R, bool MIXED>
static int residual(Exec* ctx, Level<T>& L, const T* u, const T* F, T fscale, T lam, const Coef& c, float* rplain,
                    float* chi32, float* gap32 = nullptr)
{
    const int n = L.n;
    const T h2inv = (T)((double)n * (double)n);
    const double sqDf = c.eta * 6.0 * std::fabs(c.nu) * (double)n * (double)n;
    int grid = grid_for(ctx, L.cells);
    if (grid > kMaxPartials) grid = kMaxPartials;
    const T lsn = c.kap != 0.0 ? (T)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : T(0);  // L_sat
    if constexpr (sizeof(T) == 4 && WRITE_R && !MIXED) {
        // large FP32 levels: the z-marching kernel, one block per 64 x 8 x NZ brick
        if (n >= kResidZmMinN) {
            int nz = 8;
            while ((size_t)(n / kRzTX) * (n / kRzTY) * (n / nz) > (size_t)kMaxPartials) nz *= 2;
            const dim3 g3(n / kRzTX, n / kRzTY, n / nz);
            const int nb = (int)(g3.x * g3.y * g3.z);
            ctx->begin(PM_K_RESID32, L.fine, (long long)L.cells);
            if (L.coef && L.gap) {
                constexpr size_t sm = resid_zm_smem_bytes<true, true>();
                k_residual_zm<true, true><<<g3, 256, sm, ctx->stream>>>(
                    u, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz, h2inv, (T)c.nu, (T)c.kap, (T)(sqDf * sqDf), lsn,
                    L.fine, L.r, L.sat, ctx->red_partials, L.lamp, L.coef, nullptr, nullptr, nullptr, nullptr,
                    ctx->red_out);
            } else if (L.bg) {
                constexpr size_t sm = resid_zm_smem_bytes<true>();
                k_residual_zm<true><<<g3, 256, sm, ctx->stream>>>(u, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz,
                                                                  h2inv, (T)c.nu, (T)c.kap, (T)(sqDf * sqDf), lsn,
                                                                  L.fine, L.r, L.sat, ctx->red_partials, L.lamp,
                                                                  nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                  ctx->red_out);
            } else {
                constexpr size_t sm = resid_zm_smem_bytes<false>();
                k_residual_zm<false><<<g3, 256, sm, ctx->stream>>>(u, F, fscale, lam, L.kmask, nullptr, nullptr, n, nz,
                                                                   h2inv, (T)c.nu, (T)c.kap, (T)(sqDf * sqDf), lsn,
                                                                   L.fine, L.r, L.sat, ctx->red_partials, L.lamp,
                                                                   nullptr, nullptr, nullptr, nullptr, nullptr,
                                                                   ctx->red_out);
            }
            ctx->end();
            return nb;
        }
    }
    if constexpr (sizeof(T) == 8) {
        // FP64 levels from 64^3 up without a background: the z-marching kernel
        if (!L.bg && !L.gap && n >= 64) {
            int nz = 8;
            while ((size_t)(n / kR64TX) * (n / kR64TY) * (n / nz) > (size_t)kMaxPartials) nz *= 2;
            const dim3 g3(n / kR64TX, n / kR64TY, n / nz);
            ctx->begin(PM_K_RESID64, L.fine, (long long)L.cells);
            k_residual64_zm<WRITE_R, MIXED><<<g3, 256, 0, ctx->stream>>>(
                u, F, fscale, lam, L.kmask, n, nz, h2inv, c.nu, c.kap, sqDf * sqDf, (double)lsn, L.fine, L.r, L.sat,
                ctx->red_partials, rplain, chi32, gap32, L.lamp, ctx->red_out);
            ctx->end();
            return (int)(g3.x * g3.y * g3.z);
        }
    }
    if (L.bg) {
        ctx->begin(sizeof(T) == 8 ? PM_K_RESID64 : PM_K_RESID32, L.fine, (long long)L.cells);
        k_residual<T, true, WRITE_R, MIXED><<<grid, kThreads, 0, ctx->stream>>>(
            u, F, fscale, lam, L.kmask, L.bg, L.gap, n, h2inv, (T)c.nu, (T)c.kap, (T)(sqDf * sqDf), lsn, L.fine, L.r,
            L.sat, ctx->red_partials, rplain, chi32, gap32, L.lamp, ctx->red_out);
        ctx->end();
    } else {
        ctx->begin(sizeof(T) == 8 ? PM_K_RESID64 : PM_K_RESID32, L.fine, (long long)L.cells);
        k_residual<T, false, WRITE_R, MIXED><<<grid, kThreads, 0, ctx->stream>>>(
            u, F, fscale, lam, L.kmask, nullptr, nullptr, n, h2inv, (T)c.nu, (T)c.kap, (T)(sqDf * sqDf), lsn, L.fine,
            L.r, L.sat, ctx->red_partials, rplain, chi32, gap32, L.lamp, ctx->red_out);
        ctx->end();
    }
    return grid;
}

// The residual of a large FP32 level with the FAS restriction to C folded in
// (k_residual_zm<.., RESTRICT>): C.ur, C.u[0], C.r (raw) and C.kmask (packed) are written,
// L.r and L.sat are not.  Returns false (nothing launched) where the z-marching kernel does
// not apply.
static bool residual_restrict_f32(Exec* ctx, Level<float>& L, Level<float>& C, const float* u, const float* F,
                                  float fscale, float lam, const Coef& c)
{
    const int n = L.n;
    if (n < kResidZmMinN || !C.kmask) return false;
    int nz = 8;
    while ((size_t)(n / kRzTX) * (n / kRzTY) * (n / nz) > (size_t)kMaxPartials) nz *= 2;
    const dim3 g3(n / kRzTX, n / kRzTY, n / nz);  // at most kMaxPartials blocks
    const float h2inv = (float)((double)n * (double)n);
    const double sqDf = c.eta * 6.0 * std::fabs(c.nu) * (double)n * (double)n;
    const float lsn = c.kap != 0.0 ? (float)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : 0.f;  // L_sat
    ctx->begin(PM_K_RESID32, L.fine, (long long)L.cells);
    if (L.coef && L.gap) {
        constexpr size_t sm = resid_zm_smem_bytes<true, true>();
        k_residual_zm<true, true, true><<<g3, 256, sm, ctx->stream>>>(
            u, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz, h2inv, (float)c.nu, (float)c.kap, (float)(sqDf * sqDf),
            lsn, L.fine, nullptr, nullptr, ctx->red_partials, L.lamp, L.coef, C.ur, C.u[0], C.r, C.kmask, ctx->red_out);
    } else if (L.bg) {
        constexpr size_t sm = resid_zm_smem_bytes<true>();
        k_residual_zm<true, false, true><<<g3, 256, sm, ctx->stream>>>(
            u, F, fscale, lam, L.kmask, L.bg, L.gap, n, nz, h2inv, (float)c.nu, (float)c.kap, (float)(sqDf * sqDf),
            lsn, L.fine, nullptr, nullptr, ctx->red_partials, L.lamp, nullptr, C.ur, C.u[0], C.r, C.kmask, ctx->red_out);
    } else {
        constexpr size_t sm = resid_zm_smem_bytes<false>();
        k_residual_zm<false, false, true><<<g3, 256, sm, ctx->stream>>>(
            u, F, fscale, lam, L.kmask, nullptr, nullptr, n, nz, h2inv, (float)c.nu, (float)c.kap,
            (float)(sqDf * sqDf), lsn, L.fine, nullptr, nullptr, ctx->red_partials, L.lamp, nullptr, C.ur, C.u[0],
            C.r, C.kmask, ctx->red_out);
    }
    ctx->end();
    return true;
}

// The first half of one level of the FAS V-cycle: pre-smoothing, residual, restriction
// to level l+1 and its right-hand side.
template <typename T>
static void level_down(Exec* ctx, std::vector<Level<T>>& lv, int l, const T* F0, T fs0, T lam0, const Coef& c)
{
    Level<T>& L = lv[l];
    const T* F = l == 0 ? F0 : L.f;
    const T fs = l == 0 ? fs0 : T(1);
    const T lam = l == 0 ? lam0 : T(0);
    for (int s = 0; s < ctx->prm.npre; ++s) sweep(ctx, L, F, fs, lam, c);
    Level<T>& C = lv[l + 1];
    C.cur = 0;
    const int gc = grid_for(ctx, C.cells);
    // large FP32 levels: the residual kernel restricts as well (gauge term left to k_fas_rhs)
    bool fused = false;
    if constexpr (sizeof(T) == 4) fused = residual_restrict_f32(ctx, L, C, L.u[L.cur], F, fs, lam, c);
    if (!fused) {
        residual<T, true, false>(ctx, L, L.u[L.cur], F, fs, lam, c, nullptr, nullptr);
        ctx->begin(PM_K_TRANSFER, false, 0);
        k_restrict_fas<T><<<gc, kThreads, 0, ctx->stream>>>(L.u[L.cur], L.r, L.sat, L.kmask, ctx->red_out + 8, C.n,
                                                            C.ur, C.u[0], C.r, C.kmask);
        ctx->end();
    }
    const double* gmp = fused ? ctx->red_out + 8 : nullptr;
    const T ih2c = (T)((double)C.n * (double)C.n);
    if (C.bg) {
        ctx->begin(PM_K_TRANSFER, false, 0);
        // FP32 coarse levels with coefficients: the level's coefficients and gap as well
        uint32_t* co = sizeof(T) == 4 ? C.coef : nullptr;
        float* go = (sizeof(T) == 4 && co) ? reinterpret_cast<float*>(C.gap) : nullptr;
        const float lsn = c.kap != 0.0 ? (float)(0.75 * c.nu * (1.0 - c.eta) / c.kap) : 0.f;  // L_sat
        if (C.n >= 32)
            k_fas_rhs_tile<T, true><<<dim3(C.n / 32, C.n / 4, C.n / 4), 256, 0, ctx->stream>>>(
                C.u[0], C.r, C.kmask, C.bg, C.n, ih2c, (T)c.nu, (T)c.kap, C.f, co, go, lsn, gmp);
        else
            k_fas_rhs<T, true><<<gc, kThreads, 0, ctx->stream>>>(C.u[0], C.r, C.kmask, C.bg, C.n, ih2c, (T)c.nu,
                                                                 (T)c.kap, C.f, co, go, lsn, gmp);
        ctx->end();
    } else {
        ctx->begin(PM_K_TRANSFER, false, 0);
        if (C.n >= 32)
            k_fas_rhs_tile<T, false><<<dim3(C.n / 32, C.n / 4, C.n / 4), 256, 0, ctx->stream>>>(
                C.u[0], C.r, C.kmask, nullptr, C.n, ih2c, (T)c.nu, (T)c.kap, C.f, nullptr, nullptr, 0.f, gmp);
        else
            k_fas_rhs<T, false><<<gc, kThreads, 0, ctx->stream>>>(C.u[0], C.r, C.kmask, nullptr, C.n, ih2c, (T)c.nu,
                                                                  (T)c.kap, C.f, nullptr, nullptr, 0.f, gmp);
        ctx->end();
    }
}

// The second half: prolongation of level l+1's correction and post-smoothing.
template <typename T>
static void level_up(Exec* ctx, std::vector<Level<T>>& lv, int l, const T* F0, T fs0, T lam0, const Coef& c)
{
    Level<T>& L = lv[l];
    const T* F = l == 0 ? F0 : L.f;
    const T fs = l == 0 ? fs0 : T(1);
    const T lam = l == 0 ? lam0 : T(0);
    Level<T>& C = lv[l + 1];
    ctx->begin(PM_K_TRANSFER, false, 0);
    if (C.n >= 32)
        k_prolong_add_tile<T><<<dim3(C.n / 32, C.n / 4, C.n / 4), 256, 0, ctx->stream>>>(C.u[C.cur], C.ur, C.n,
                                                                                          L.u[L.cur]);
    else
        k_prolong_add<T><<<grid_for(ctx, C.cells), kThreads, 0, ctx->stream>>>(C.u[C.cur], C.ur, C.n, L.u[L.cur]);
    ctx->end();
    for (int s = 0; s < ctx->prm.npost; ++s) sweep(ctx, L, F, fs, lam, c);
}

template <typename T>
static void vcycle(Exec* ctx, std::vector<Level<T>>& lv, int l, const T* F0, T fs0, T lam0, const Coef& c)
{
    Level<T>& L = lv[l];
    const T* F = l == 0 ? F0 : L.f;
    const T fs = l == 0 ? fs0 : T(1);
    const T lam = l == 0 ? lam0 : T(0);
    const int nlev = (int)lv.size();
    if (l == nlev - 1) {
        const double ih2 = (double)L.n * (double)L.n;
        if (ctx->prm.coarse_exact && L.cells <= (size_t)kExactMaxCells) {
            ctx->begin(PM_K_COARSEST, false, 0);
            if (L.bg)
                k_coarsest_exact<T, true><<<1, kExactThreads, 0, ctx->stream>>>(
                    L.u[L.cur], F, fs, L.kmask, L.bg, L.n, ih2, c.nu, c.kap, c.eta, nullptr);
            else
                k_coarsest_exact<T, false><<<1, kExactThreads, 0, ctx->stream>>>(
                    L.u[L.cur], F, fs, L.kmask, nullptr, L.n, ih2, c.nu, c.kap, c.eta, nullptr);
            ctx->end();
            return;
        }
        if (L.bg) {
            ctx->begin(PM_K_COARSEST, false, 0);
            k_coarsest<T, true><<<1, 256, 0, ctx->stream>>>(L.u[L.cur], F, fs, L.kmask, L.bg, L.n, ih2, c.nu, c.kap,
                                                            c.eta, ctx->prm.coarse_sweeps, L.fine);
            ctx->end();
        } else {
            ctx->begin(PM_K_COARSEST, false, 0);
            k_coarsest<T, false><<<1, 256, 0, ctx->stream>>>(L.u[L.cur], F, fs, L.kmask, nullptr, L.n, ih2, c.nu,
                                                             c.kap, c.eta, ctx->prm.coarse_sweeps, L.fine);
            ctx->end();
        }
        return;
    }
    level_down(ctx, lv, l, F0, fs0, lam0, c);
    vcycle(ctx, lv, l + 1, F0, fs0, lam0, c);
    level_up(ctx, lv, l, F0, fs0, lam0, c);
}

// The levels above `stop` of a V-cycle, down and up; level `stop` and below are solved in
// between by the caller (the batched solve's cooperative coarse kernel).
template <typename T>
static void vcycle_down(Exec* ctx, std::vector<Level<T>>& lv, int stop, const T* F0, T fs0, T lam0, const Coef& c)
{
    for (int l = 0; l < stop; ++l) level_down(ctx, lv, l, F0, fs0, lam0, c);
}
template <typename T>
static void vcycle_up(Exec* ctx, std::vector<Level<T>>& lv, int stop, const T* F0, T fs0, T lam0, const Coef& c)
{
    for (int l = stop - 1; l >= 0; --l) level_up(ctx, lv, l, F0, fs0, lam0, c);
}

template <typename T>
static void recentre(Exec* ctx, T* x, size_t cells)
{
    int grid = grid_for(ctx, cells);
    if (grid > kMaxPartials) grid = kMaxPartials;
    ctx->begin(PM_K_REDUCE, false, 0);
    k_sum<T><<<grid, kThreads, 0, ctx->stream>>>(x, cells, ctx->red_partials, ctx->red_out + 16);
    ctx->end();
    ctx->begin(PM_K_REDUCE, false, 0);
    k_sub_mean<T><<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(x, cells, ctx->red_out + 16);
    ctx->end();
}

static pm_status read_sums(Exec* ctx, int count)
{
    PM_CUDA(cudaMemcpyAsync(ctx->host_out, ctx->red_out, sizeof(double) * count, cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

// |f - <f>|_2 for f = src * delta
static pm_status source_norm(Exec* ctx, const double* delta, size_t cells, double src, double* out)
{
    int grid = grid_for(ctx, cells);
    if (grid > kMaxPartials) grid = kMaxPartials;
    ctx->begin(PM_K_REDUCE, false, 0);
    k_sum<double><<<grid, kThreads, 0, ctx->stream>>>(delta, cells, ctx->red_partials, ctx->red_out + 32);
    ctx->end();
    ctx->begin(PM_K_REDUCE, false, 0);
    k_sum_centred<<<grid, kThreads, 0, ctx->stream>>>(delta, cells, ctx->red_out + 32, ctx->red_partials,
                                                       ctx->red_out + 48);
    ctx->end();
    PM_CUDA(cudaMemcpyAsync(ctx->host_out, ctx->red_out + 48, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    *out = std::fabs(src) * std::sqrt(ctx->host_out[0]);
    return PM_OK;
}

// float-float outer residual of the mixed path (outer_ff.cuh); sums into red_out[0..8].
// With a pending correction e (n >= kFzTX only; <e> already summed into red_out[16]) the
// residual is that of xff + e - <e>, and that corrected iterate is written to xout.
static void residual_ff(Exec* ctx, Workspace* w, const float2* xff, const float2* fff, double lam,
                        const double* lamp, const FFCoef& fk, const float* e = nullptr, float2* xout = nullptr)
{
    const int n = w->n;
    const size_t cells = (size_t)n * n * n;
    int grid = grid_for(ctx, cells);
    if (grid > kMaxPartials) grid = kMaxPartials;
    ctx->begin(PM_K_RESID64, true, (long long)cells);
    if (n >= kFzTX) {
        int nz = 8 < n ? 8 : n;
        while ((size_t)(n / kFzTX) * (n / kFzTY) * (n / nz) > (size_t)kMaxPartials) nz *= 2;
        const dim3 g3(n / kFzTX, n / kFzTY, n / nz);
        grid = (int)(g3.x * g3.y * g3.z);
        if (e)
            k_residual_ff_zm<true><<<g3, 256, kFzSmemCorr, ctx->stream>>>(
                xff, fff, lam, lamp, n, nz, fk, w->rplain, w->s[0].bg, w->s[0].gap, w->s[0].coef,
                ctx->red_partials, e, ctx->red_out + 16, xout, ctx->red_out);
        else
            k_residual_ff_zm<false><<<g3, 256, kFzSmem, ctx->stream>>>(
                xff, fff, lam, lamp, n, nz, fk, w->rplain, w->s[0].bg, w->s[0].gap, w->s[0].coef,
                ctx->red_partials, nullptr, nullptr, nullptr, ctx->red_out);
    } else {
        k_residual_ff<<<grid, kThreads, 0, ctx->stream>>>(xff, fff, lam, lamp, n, fk, w->rplain, w->s[0].bg,
                                                          w->s[0].gap, ctx->red_partials, ctx->red_out);
    }
    ctx->end();
}

// sum of the correction e into red_out[16]
static void correction_sum(Exec* ctx, const float* e, size_t cells)
{
    int grid = grid_for(ctx, cells);
    if (grid > kMaxPartials) grid = kMaxPartials;
    ctx->begin(PM_K_REDUCE, false, 0);
    k_sum<float><<<grid, kThreads, 0, ctx->stream>>>(e, cells, ctx->red_partials, ctx->red_out + 16);
    ctx->end();
}

// chi += e - <e> on the float-float iterate
static void add_correction_ff(Exec* ctx, float2* xff, const float* e, size_t cells)
{
    correction_sum(ctx, e, cells);
    ctx->begin(PM_K_REDUCE, false, 0);
    k_add_correction_ff<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(xff, e, cells, ctx->red_out + 16);
    ctx->end();
}

// the float-float iterate and right-hand side of the mixed path live in the FP64 level-0
// buffers that path does not otherwise use (8 bytes per cell each)
static float2* ff_chi(Workspace* w) { return reinterpret_cast<float2*>(w->d[0].u[1]); }
static float2* ff_rhs(Workspace* w) { return reinterpret_cast<float2*>(w->d[0].r); }

// relative residual from the sums of a residual launch (red_out[0..8] as read back)
static double rel_from_sums(const double* h, double fnorm, double* gm_out)
{
    const double gm = h[3] > 0.0 ? h[0] / h[3] : 0.0;
    const double r2 = h[2] - 2.0 * gm * h[1] + gm * gm * h[3];
    if (gm_out) *gm_out = gm;
    const double r = std::sqrt(r2 > 0.0 ? r2 : 0.0);
    return fnorm > 0.0 ? r / fnorm : r;
}

pm_status mg_solve(pm_ctx* pctx, const double* delta, int n, const pm_coeffs& cf, double tol, double* phi,
                   pm_solve_info* info)
{
    Exec ex(pctx);
    Exec* ctx = &ex;
    const pm_params& P = ctx->prm;
    pm_solve_info local{};
    pm_solve_info* inf = info ? info : &local;
    *inf = pm_solve_info{};
    inf->unstable_nu = cf.nu <= 0.0 ? 1 : 0;
    const size_t cells = (size_t)n * n * n;
    if (cf.xi == 0.0) {  // no coupling: chi = 0 solves the equation exactly
        PM_CUDA(cudaMemsetAsync(phi, 0, cells * sizeof(double), ctx->stream));
        inf->status = PM_OK;
        return PM_OK;
    }
    if (cf.nu == 0.0 || !std::isfinite(cf.nu) || !std::isfinite(cf.kappa)) {
        ctx->set_error("nu = 0: the chi operator is degenerate");
        return PM_ERR_INVALID_ARG;
    }
    Workspace* w = nullptr;
    PM_TRY(get_workspace(pctx, n, &w));
    // mixed: an FP32 inner cycle on the correction; ffo: its outer loop in float-float
    // (precision 1), else in FP64 (precision 2)
    const bool mixed = P.precision >= 1;
    const bool ffo = P.precision == 1;
    PM_TRY(ensure_mg(pctx, w, mixed));
    // The BF16 background coefficients of the finest inner level are written by the
    // float-float residual only: with the FP64 outer residual that level sweeps through the
    // background's own planes (the coefficient pointer is hidden for this solve).
    struct CoefHide {
        Level<float>* L = nullptr;
        uint32_t* saved = nullptr;
        ~CoefHide()
        {
            if (L) L->coef = saved;
        }
    } hide;
    if (mixed && !ffo) {
        hide.L = &w->s[0];
        hide.saved = w->s[0].coef;
        w->s[0].coef = nullptr;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, ctx->stream);
    Coef c{cf.nu, cf.kappa, P.eta, cf.src};
    double fnorm = 0.0;
    PM_TRY(source_norm(ctx, delta, cells, cf.src, &fnorm));
    Level<double>& L0 = w->d[0];
    L0.cur = 0;
    PM_CUDA(cudaMemcpyAsync(L0.u[0], phi, cells * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    float2* xff = ffo ? ff_chi(w) : nullptr;
    float2* fff = ffo ? ff_rhs(w) : nullptr;
    const FFCoef fk = make_ffcoef(cf.nu, cf.kappa, P.eta, n);
    if (mixed && !ffo) recentre<double>(ctx, L0.u[0], cells);
    if (ffo) {
        recentre<double>(ctx, L0.u[0], cells);
        ctx->begin(PM_K_REDUCE, false, 0);
        k_to_ff<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(delta, cf.src, cells, fff);
        ctx->end();
        ctx->begin(PM_K_REDUCE, false, 0);
        k_to_ff<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(L0.u[0], 1.0, cells, xff);
        ctx->end();
    }
    double lam = 0.0, rr = 0.0;
    int cyc = 0, vcyc = 0;
    pm_status st = PM_ERR_NOCONV;
    // mixed: the iterate lives in xff or w->ff_alt; the correction of an outer iteration is
    // applied by the next residual launch (pend), which writes the corrected iterate to the
    // other buffer
    const float* pend = nullptr;
    for (;;) {
        if (ffo) {
            float2* xo = xff == ff_chi(w) ? w->ff_alt : ff_chi(w);
            residual_ff(ctx, w, xff, fff, lam, nullptr, fk, pend, pend ? xo : nullptr);
            if (pend) xff = xo;
            pend = nullptr;
        } else if (mixed) {
            // FP64 outer residual; it also writes the inner right-hand side, background and gap
            residual<double, false, true>(ctx, L0, L0.u[L0.cur], delta, cf.src, lam, c, w->rplain, w->s[0].bg,
                                          w->s[0].gap);
        } else
            residual<double, false, false>(ctx, L0, L0.u[L0.cur], delta, cf.src, lam, c, nullptr, nullptr);
        PM_TRY(read_sums(ctx, 9));
        const double* h = ctx->host_out;
        double gm = 0.0;
        rr = rel_from_sums(h, fnorm, &gm);
        lam -= gm;
        inf->floored_cells = (long long)((double)cells - h[3]);
        if (cyc == 0 && !inf->guess_rejected) {
            inf->guess_rel_res = (h[4] > 0.0 || !std::isfinite(rr)) ? INFINITY : rr;
            if (!(inf->guess_rel_res <= kGuessLimit)) {
                // the guess is far worse than chi = 0: start from zero instead
                inf->guess_rejected = 1;
                lam = 0.0;
                if (ffo)
                    PM_CUDA(cudaMemsetAsync(xff, 0, cells * sizeof(float2), ctx->stream));
                else
                    PM_CUDA(cudaMemsetAsync(L0.u[L0.cur], 0, cells * sizeof(double), ctx->stream));
                continue;
            }
        }
        if (cyc < 64) inf->rel_res_hist[cyc] = rr;
        if (h[4] > 0.0 || !std::isfinite(rr)) {
            st = PM_ERR_NONFINITE;
            ctx->set_error("non-finite residual");
            break;
        }
        if (rr <= tol || fnorm == 0.0) {
            if (!ffo) {
                st = PM_OK;
                break;
            }
            // confirm the float-float stop test with the FP64 residual of the FP64 result
            ctx->begin(PM_K_REDUCE, false, 0);
            k_from_ff<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(xff, cells, L0.u[0]);
            ctx->end();
            residual<double, false, false>(ctx, L0, L0.u[0], delta, cf.src, lam, c, nullptr, nullptr);
            PM_TRY(read_sums(ctx, 9));
            double gm64 = 0.0;
            const double rr64 = rel_from_sums(ctx->host_out, fnorm, &gm64);
            if (rr64 <= tol || fnorm == 0.0) {
                lam -= gm64;
                rr = rr64;
                st = PM_OK;
                break;
            }
        }
        if (cyc >= P.max_cycles) {
            ctx->set_error("max_cycles reached before the tolerance");
            break;
        }
        if (mixed) {
            // inner FP32 FAS V-cycle on the correction e, background chi32, rhs rplain - gm
            std::vector<Level<float>>& s = w->s;
            for (size_t l = 0; l + 1 < s.size(); ++l) {
                ctx->begin(PM_K_TRANSFER, false, 0);
                k_restrict<float><<<grid_for(ctx, s[l + 1].cells), kThreads, 0, ctx->stream>>>(s[l].bg, s[l + 1].n,
                                                                                               s[l + 1].bg);
                ctx->end();
            }
            start_at_zero(ctx, s[0]);
            PM_CUDA(cudaGetLastError());
            for (int k = 0; k < P.inner_cycles; ++k) {
                vcycle<float>(ctx, s, 0, w->rplain, 1.0f, (float)(-gm), c);
                ++vcyc;
            }
            if (!ffo) {
                // FP64 iterate: chi += e - <e>
                correction_sum(ctx, s[0].u[s[0].cur], cells);
                ctx->begin(PM_K_REDUCE, false, 0);
                k_add_correction_centred<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(
                    L0.u[L0.cur], s[0].u[s[0].cur], cells, ctx->red_out + 16);
                ctx->end();
            } else if (n >= kFzTX) {
                correction_sum(ctx, s[0].u[s[0].cur], cells);
                pend = s[0].u[s[0].cur];
            } else {
                add_correction_ff(ctx, xff, s[0].u[s[0].cur], cells);
            }
        } else {
            vcycle<double>(ctx, w->d, 0, delta, cf.src, lam, c);
            ++vcyc;
            recentre<double>(ctx, L0.u[L0.cur], cells);
        }
        ++cyc;
    }
    if (ffo) {
        if (st != PM_OK) {
            ctx->begin(PM_K_REDUCE, false, 0);
            k_from_ff<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(xff, cells, L0.u[0]);
            ctx->end();
        }
        recentre<double>(ctx, L0.u[0], cells);  // <chi> = 0 to FP64 rounding
    } else if (mixed) {
        recentre<double>(ctx, L0.u[L0.cur], cells);
    }
    PM_CUDA(cudaMemcpyAsync(phi, L0.u[L0.cur], cells * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    cudaEventRecord(e1, ctx->stream);
    PM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    inf->cycles = cyc;
    inf->vcycles = vcyc;
    inf->rel_res = rr;
    inf->lambda = lam;
    inf->ms_total = ms;
    inf->status = st;
    return st;
}

}  // namespace pmeft

#include "batch_coop.cuh"
#include "batch.cuh"

using namespace pmeft;

// ------------------------------------------------------------------ single-operation ABI

static pm_status check_mg_args(pm_ctx* ctx, int n)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (!valid_n(n)) {
        ctx->set_error("n must be a power of two >= 8");
        return PM_ERR_INVALID_ARG;
    }
    return PM_OK;
}

extern "C" pm_status pm_mg_sweep(pm_ctx* ctx, double* u, const double* f, double lambda, int n, double nu,
                                 double kappa, double eta, const unsigned char* kmask)
{
    PM_TRY(check_mg_args(ctx, n));
    if (!u || !f) return PM_ERR_INVALID_ARG;
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    PM_TRY(ensure_mg(ctx, w, false));
    Level<double> L = w->d[0];  // borrow the buffers, with the caller's mask
    L.kmask = (uint8_t*)kmask;
    L.bg = nullptr;
    L.cur = 0;
    const size_t cells = L.cells;
    PM_CUDA(cudaMemcpyAsync(L.u[0], u, cells * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    Coef c{nu, kappa, eta, 1.0};
    Exec ex(ctx);
    sweep<double>(&ex, L, f, 1.0, lambda, c);
    PM_CUDA(cudaMemcpyAsync(u, L.u[L.cur], cells * sizeof(double), cudaMemcpyDeviceToDevice, ctx->stream));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_mg_sweep_f32(pm_ctx* ctx, float* u, const float* f, float lambda, int n, double nu,
                                     double kappa, double eta, const unsigned char* kmask, const float* bg,
                                     const float* gap, int mode)
{
    PM_TRY(check_mg_args(ctx, n));
    // mode 100 + k: variant k - 1 with the background entering through its BF16 coefficients;
    // mode 200: the zero-start kernel (u taken as zero), 200 + k its variant k - 1
    const bool from_zero = mode >= 200 && mode <= 200 + kNumZeroCfgs;
    const int zero_cfg = from_zero ? mode - 201 : -1;
    if (from_zero) mode = 101;
    const bool via_coef = mode > 100;
    if (via_coef) mode -= 100;
    if (!u || !f || mode < 0 || mode > kNumFusedCfgs || (gap && !bg) || (via_coef && (!bg || !gap || kmask)) ||
        (from_zero && (n < 64 || (zero_cfg >= 0 && !zero_cfg_fits(zero_cfg, n)))))
        return PM_ERR_INVALID_ARG;
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    PM_TRY(ensure_mg(ctx, w, true));
    Level<float> L = w->s[0];  // borrow the buffers, with the caller's mask, background and gap
    L.kmask = (uint8_t*)kmask;
    L.bg = (float*)bg;
    L.gap = (float*)gap;
    L.coef = nullptr;  // the background is the caller's field, not the solve's coefficients
    L.cur = 0;
    const size_t cells = L.cells;
    if (via_coef) {
        if (!w->coef_test) PM_CUDA(cudaMalloc(&w->coef_test, 3 * cells * sizeof(uint32_t)));
        L.coef = w->coef_test;
        k_bg_coef<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(bg, n, L.coef);
        PM_CUDA(cudaGetLastError());
    }
    PM_CUDA(cudaMemcpyAsync(L.u[0], u, cells * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    Coef c{nu, kappa, eta, 1.0};
    Exec ex(ctx);
    if (from_zero) sweep_zero_f32(&ex, L, f, 1.0f, lambda, c, zero_cfg);
    else sweep<float>(&ex, L, f, 1.0f, lambda, c, mode);
    PM_CUDA(cudaMemcpyAsync(u, L.u[L.cur], cells * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_mg_residual(pm_ctx* ctx, const double* u, const double* f, double lambda, int n, double nu,
                                    double kappa, double eta, const unsigned char* kmask, double* r,
                                    unsigned char* floored)
{
    PM_TRY(check_mg_args(ctx, n));
    if (!u || !f || !r) return PM_ERR_INVALID_ARG;
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    PM_TRY(ensure_mg(ctx, w, false));
    Level<double> L = w->d[0];
    L.kmask = (uint8_t*)kmask;
    L.bg = nullptr;
    L.r = r;
    L.sat = floored ? floored : w->d[0].sat;
    Coef c{nu, kappa, eta, 1.0};
    Exec ex(ctx);
    residual<double, true, false>(&ex, L, u, f, 1.0, lambda, c, nullptr, nullptr);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_mg_restrict(pm_ctx* ctx, const double* fine, int n, double* coarse)
{
    PM_TRY(check_mg_args(ctx, n));
    if (!fine || !coarse) return PM_ERR_INVALID_ARG;
    const int nc = n / 2;
    ctx->begin(PM_K_TRANSFER, false, 0);
    k_restrict<double><<<grid_for(ctx, (size_t)nc * nc * nc), kThreads, 0, ctx->stream>>>(fine, nc, coarse);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_mg_prolong_add(pm_ctx* ctx, const double* coarse, int n, double* fine)
{
    PM_TRY(check_mg_args(ctx, n));
    if (!fine || !coarse) return PM_ERR_INVALID_ARG;
    const int nc = n / 2;
    ctx->begin(PM_K_TRANSFER, false, 0);
    if (nc >= 32)  // the tiled kernel of the V-cycle from 32^3 coarse cells up
        k_prolong_add_tile<double><<<dim3(nc / 32, nc / 4, nc / 4), 256, 0, ctx->stream>>>(coarse, nullptr, nc, fine);
    else
        k_prolong_add<double><<<grid_for(ctx, (size_t)nc * nc * nc), kThreads, 0, ctx->stream>>>(coarse, nullptr, nc,
                                                                                                fine);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_mg_coarse_exact(pm_ctx* ctx, double* u, const double* f, int n, double nu, double kappa,
                                        double eta, const unsigned char* kmask, double* lambda_out)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (!(n == 2 || n == 4) || !u || !f || nu == 0.0 || !std::isfinite(nu) || !std::isfinite(kappa) ||
        !(eta >= 0.0 && eta < 1.0)) {
        ctx->set_error("pm_mg_coarse_exact: n must be 2 or 4, u and f non-null, nu finite and nonzero");
        return PM_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PM_ERR_CUDA;
    double* d_lam = ctx->red_out + 60;  // a slot no solve uses between calls
    k_coarsest_exact<double, false><<<1, kExactThreads, 0, ctx->stream>>>(
        u, f, 1.0, kmask, nullptr, n, (double)n * (double)n, nu, kappa, eta, d_lam);
    PM_CUDA(cudaGetLastError());
    PM_CUDA(cudaMemcpyAsync(ctx->host_out + 60, d_lam, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (lambda_out) *lambda_out = ctx->host_out[60];
    return PM_OK;
}

extern "C" pm_status scalar_mg_solve(pm_ctx* ctx, const double* delta, int n, double alpha_B0, double alpha_M0,
                                     double a, double tol, double* phi_inout, pm_solve_info* info)
{
    PM_TRY(check_mg_args(ctx, n));
    if (!delta || !phi_inout || !(tol > 0.0) || !(a > 0.0)) {
        ctx->set_error("scalar_mg_solve: null buffer, tol <= 0 or a <= 0");
        return PM_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PM_ERR_CUDA;
    pm_coeffs cf;
    coefficients(alpha_B0, alpha_M0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    return mg_solve(ctx, delta, n, cf, tol, phi_inout, info);
}

extern "C" pm_status scalar_mg_solve_batched(pm_ctx* ctx, int nbox, const int* n, const double* const* delta,
                                             const double* alpha_B0, const double* alpha_M0, const double* a,
                                             double tol, double* const* phi_inout, pm_solve_info* infos)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (nbox < 1 || !n || !delta || !alpha_B0 || !alpha_M0 || !a || !phi_inout || !(tol > 0.0)) {
        ctx->set_error("scalar_mg_solve_batched: bad arguments");
        return PM_ERR_INVALID_ARG;
    }
    for (int b = 0; b < nbox; ++b) {
        if (!valid_n(n[b]) || !delta[b] || !phi_inout[b] || !(a[b] > 0.0)) {
            ctx->set_error("scalar_mg_solve_batched: bad box " + std::to_string(b));
            return PM_ERR_INVALID_ARG;
        }
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PM_ERR_CUDA;
    return mg_solve_batched(ctx, nbox, n, delta, alpha_B0, alpha_M0, a, tol, phi_inout, infos);
}
