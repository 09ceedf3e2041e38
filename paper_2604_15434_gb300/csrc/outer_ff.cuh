// outer_ff.cuh -- the outer loop of the mixed-precision solve in float-float arithmetic.
//
// GB300 runs FP64 at about 1/58 of its FP32 rate (measured), and the outer residual of the defect
// correction (19-point stencil, the quadratic q2, the floor test) costs ~60 FP64
// instructions per cell: on the FP64 pipe it took longer than the whole FP32 inner cycle.
// The outer iterate chi is therefore kept as an unevaluated sum hi + lo of two floats
// (about 48 significant bits, against the 24 of FP32 and the 53 of FP64), and the
// residual is evaluated with error-free transformations on the FP32 pipe:
//   * TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s + e == a + b exactly;
//   * Fast2Sum (Dekker 1971): the same in three operations when |a| >= |b|;
//   * TwoProd with a fused multiply-add: p + e == a * b exactly.
// Sums use the "sloppy" pairing (TwoSum of the high parts, low parts added, Fast2Sum),
// whose error is ~2^-47 of the operands' magnitude: the same kind of bound as FP64's
// 2^-53, a factor 64 looser, far below the 1e-8 relative residual the loop stops at.  The
// z-marching kernel keeps chains of such sums unnormalised (high parts by TwoSum, every
// tail summed in FP32) and normalises once per quantity, with the same kind of bound.
// The right-hand side src*delta is converted to float-float once per solve; the caller's
// FP64 guess once on entry and the result once on exit, where one FP64 residual of the
// returned chi confirms the stop test.
#pragma once

#include "internal.cuh"
#include "sweep_fused.cuh"

namespace pmeft {

struct ff {
    float hi, lo;
};

__device__ __forceinline__ float ff_two_sum(float a, float b, float& e)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

__device__ __forceinline__ ff ff_norm(float s, float e)
{
    ff r;
    r.hi = __fadd_rn(s, e);
    r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ ff ff_add(ff a, ff b)
{
    float e;
    const float s = ff_two_sum(a.hi, b.hi, e);
    return ff_norm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff{-a.hi, -a.lo}; }
__device__ __forceinline__ ff ff_sub(ff a, ff b) { return ff_add(a, ff_neg(b)); }

__device__ __forceinline__ ff ff_mul(ff a, ff b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_norm(p, e);
}

// multiplication by a power of two is exact
__device__ __forceinline__ ff ff_scale2(ff a, float p2) { return ff{a.hi * p2, a.lo * p2}; }

__device__ __forceinline__ ff ff_from_double(double x)
{
    const float hi = __double2float_rn(x);
    return ff{hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ ff ff_load(const float2* __restrict__ p, size_t i)
{
    const float2 v = p[i];
    return ff{v.x, v.y};
}

// float-float constants of one solve, split on the host
struct FFCoef {
    float nu1_hi, nu1_lo;    // nu / h^2
    float kap1_hi, kap1_lo;  // kappa / h^4
    float lsat_hi, lsat_lo;  // L_sat = 3 nu (1 - eta) / (4 kappa)
    float nu_hi, nu_lo;      // nu
    float ih2;               // 1/h^2 (a power of two)
    float nu_f, kap_f, Df;   // FP32 copies for the floor test only
};

inline FFCoef make_ffcoef(double nu, double kap, double eta, int n)
{
    auto split = [](double x, float& hi, float& lo) {
        hi = (float)x;
        lo = (float)(x - (double)hi);
    };
    FFCoef c{};
    const double ih2 = (double)n * (double)n;
    split(nu * ih2, c.nu1_hi, c.nu1_lo);
    split(kap * ih2 * ih2, c.kap1_hi, c.kap1_lo);
    split(kap != 0.0 ? 3.0 * nu * (1.0 - eta) / (4.0 * kap) : 0.0, c.lsat_hi, c.lsat_lo);
    split(nu, c.nu_hi, c.nu_lo);
    c.ih2 = (float)ih2;
    c.nu_f = (float)nu;
    c.kap_f = (float)kap;
    const double sqDf = eta * 6.0 * std::fabs(nu) * ih2;
    c.Df = (float)(sqDf * sqDf);
    return c;
}

// y = ff(scale * x)
__global__ void k_to_ff(const double* __restrict__ x, double scale, size_t total, float2* __restrict__ y)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const ff v = ff_from_double(scale * x[c]);
        y[c] = make_float2(v.hi, v.lo);
    }
}

__global__ void k_from_ff(const float2* __restrict__ x, size_t total, double* __restrict__ y)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const float2 v = x[c];
        y[c] = (double)v.x + (double)v.y;
    }
}

// chi += e - <e>, the correction of one outer iteration; subtracting the correction's
// mean keeps <chi> = 0 (the gauge) without a second pass over chi.
__global__ void k_add_correction_ff(float2* __restrict__ x, const float* __restrict__ e, size_t total,
                                    const double* __restrict__ sums)
{
    const double mean = sums[0] / (double)total;
    const float mhi = (float)mean, mlo = (float)(mean - (double)mhi);
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const float2 v = x[c];
        float err;
        const float s = ff_two_sum(e[c], -mhi, err);
        const ff d = ff_norm(s, __fsub_rn(err, mlo));
        const ff r = ff_add(ff{v.x, v.y}, d);
        x[c] = make_float2(r.hi, r.lo);
    }
}

// Outer residual of the defect correction in float-float, with the same outputs as the
// FP64 residual of the mixed path: rplain = f + lambda - N(chi) (FP32), chi32 = the FP32
// background (the high part of chi), gap32 = L_sat - L(chi) (FP32), and per-block sums
// [r, r over unfloored cells, r^2, unfloored count, non-finite count] of the NCP residual
// r = f + lambda - N (unfloored) or nu (L_sat - L) (floored).
__global__ void __launch_bounds__(256) k_residual_ff(const float2* __restrict__ U, const float2* __restrict__ F,
                                                     double lam_host, const double* __restrict__ lamp, int n,
                                                     FFCoef k, float* __restrict__ rplain, float* __restrict__ chi32,
                                                     float* __restrict__ gap32, double* __restrict__ partials,
                                                     double* __restrict__ fin_out = nullptr)
{
    const double lam_d = lam_host + (lamp ? *lamp : 0.0);
    const ff lam = ff_from_double(lam_d);
    const ff nu1{k.nu1_hi, k.nu1_lo}, kap1{k.kap1_hi, k.kap1_lo}, lsat{k.lsat_hi, k.lsat_lo}, nu{k.nu_hi, k.nu_lo};
    const bool screened = k.kap_f != 0.f;
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    const size_t total = (size_t)n * n * n;
    const int m = n - 1;
    const size_t sn = (size_t)n;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c & (size_t)m);
        const int lg = __ffs(n) - 1;  // n = 2^lg
        const size_t row = c >> lg;
        const int j = (int)(row & (size_t)m), kz = (int)(row >> lg);
        const int ip = (i + 1) & m, im = (i - 1) & m, jp = (j + 1) & m, jm = (j - 1) & m, kp = (kz + 1) & m,
                  km = (kz - 1) & m;
        auto at = [&](int ii, int jj, int kk) { return ff_load(U, ((size_t)kk * sn + jj) * sn + ii); };
        const ff c0 = ff_load(U, c);
        const ff m2c = ff_scale2(c0, -2.f);
        // second differences (h = 1 units) and the cross differences exy = 4 h^2 chi_xy
        const ff X = ff_add(ff_add(at(ip, j, kz), at(im, j, kz)), m2c);
        const ff Y = ff_add(ff_add(at(i, jp, kz), at(i, jm, kz)), m2c);
        const ff Z = ff_add(ff_add(at(i, j, kp), at(i, j, km)), m2c);
        const ff exy = ff_sub(ff_sub(at(ip, jp, kz), at(ip, jm, kz)), ff_sub(at(im, jp, kz), at(im, jm, kz)));
        const ff exz = ff_sub(ff_sub(at(ip, j, kp), at(ip, j, km)), ff_sub(at(im, j, kp), at(im, j, km)));
        const ff eyz = ff_sub(ff_sub(at(i, jp, kp), at(i, jp, km)), ff_sub(at(i, jm, kp), at(i, jm, km)));
        const ff L1 = ff_add(ff_add(X, Y), Z);  // h^2 L
        // h^4 q2 = 2 (XY + YZ + ZX) - (exy^2 + exz^2 + eyz^2) / 8
        const ff sq = ff_add(ff_add(ff_mul(exy, exy), ff_mul(exz, exz)), ff_mul(eyz, eyz));
        const ff pr = ff_add(ff_add(ff_mul(X, Y), ff_mul(Y, Z)), ff_mul(Z, X));
        const ff q2 = ff_sub(ff_scale2(pr, 2.f), ff_scale2(sq, 0.125f));
        const ff N = ff_sub(ff_mul(nu1, L1), ff_mul(kap1, q2));
        const ff rhs = ff_add(ff_load(F, c), lam);
        const ff G = ff_sub(N, rhs);  // N - f - lambda
        const ff L = ff_scale2(L1, k.ih2);
        const ff g = screened ? ff_sub(lsat, L) : ff{0.f, 0.f};
        // floor test in FP32: Ep = (-6 nu + 8 kappa L)/h^2, P = -24 kappa/h^4, D = Ep^2 - 4 P G
        const float Lf = L.hi + L.lo, Gf = G.hi + G.lo;
        const float Ep = (-6.f * k.nu_f + 8.f * k.kap_f * Lf) * k.ih2;
        const float P = -24.f * k.kap_f * k.ih2 * k.ih2;
        const float D = Ep * Ep - 4.f * P * Gf;
        const bool fl = screened && D < k.Df;
        const ff rv = fl ? ff_mul(nu, g) : ff_neg(G);
        rplain[c] = -Gf;
        chi32[c] = c0.hi;
        gap32[c] = g.hi + g.lo;
        const float d = rv.hi + rv.lo;
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
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, fin_out);
}


// ------------------------------------------------------------------ two cells per thread
//
// Blackwell issues FADD2 / FMUL2 / FFMA2: one instruction for a float2 of operations, each
// component rounded exactly as its scalar form.  The z-marching residual below keeps two
// cells per thread in the two components (hi parts in one float2, lo parts in another), so
// every error-free transformation costs the instructions of one cell.

struct ff2 {
    float2 hi, lo;  // components: cell A, cell B
};

__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 p_splat(float a) { return make_float2(a, a); }

__device__ __forceinline__ ff2 ff2_norm(float2 s, float2 e)
{
    ff2 r;
    r.hi = p_add(s, e);
    r.lo = p_sub(e, p_sub(r.hi, s));
    return r;
}

__device__ __forceinline__ ff2 ff2_add(ff2 a, ff2 b)
{
    const float2 s = p_add(a.hi, b.hi);
    const float2 bb = p_sub(s, a.hi);
    const float2 e = p_add(p_sub(a.hi, p_sub(s, bb)), p_sub(b.hi, bb));
    return ff2_norm(s, p_add(e, p_add(a.lo, b.lo)));
}

__device__ __forceinline__ ff2 ff2_neg(ff2 a) { return ff2{make_float2(-a.hi.x, -a.hi.y), make_float2(-a.lo.x, -a.lo.y)}; }
__device__ __forceinline__ ff2 ff2_sub(ff2 a, ff2 b) { return ff2_add(a, ff2_neg(b)); }

__device__ __forceinline__ ff2 ff2_mul(ff2 a, ff2 b)
{
    const float2 p = p_mul(a.hi, b.hi);
    float2 e = p_fma(a.hi, b.hi, make_float2(-p.x, -p.y));
    e = p_fma(a.hi, b.lo, e);
    e = p_fma(a.lo, b.hi, e);
    return ff2_norm(p, e);
}

__device__ __forceinline__ ff2 ff2_scale2(ff2 a, float p2) { return ff2{p_mul(a.hi, p_splat(p2)), p_mul(a.lo, p_splat(p2))}; }
__device__ __forceinline__ float2 p_neg(float2 a) { return make_float2(-a.x, -a.y); }

// TwoSum on pairs: s + e == a + b exactly (6 instructions)
__device__ __forceinline__ float2 two_sum2(float2 a, float2 b, float2& e)
{
    const float2 s = p_add(a, b);
    const float2 bb = p_sub(s, a);
    e = p_add(p_sub(a, p_sub(s, bb)), p_sub(b, bb));
    return s;
}

// a * b = p + e for float-float a, b, unnormalised: TwoProd of the high parts plus the two
// cross terms (4 instructions; error ~2^-47 of |a b|)
__device__ __forceinline__ float2 uprod2(const ff2& a, const ff2& b, float2& e)
{
    const float2 p = p_mul(a.hi, b.hi);
    e = p_fma(a.hi, b.hi, p_neg(p));
    e = p_fma(a.hi, b.lo, e);
    e = p_fma(a.lo, b.hi, e);
    return p;
}

// (a + b) + m2h + m2l for float-float a, b and the pair (m2h, m2l) = -2 c: the second
// difference, normalised once (19 instructions against 24 for two float-float additions)
__device__ __forceinline__ ff2 second_diff2(const ff2& a, const ff2& b, float2 m2h, float2 m2l)
{
    float2 e1, e2;
    const float2 s1 = two_sum2(a.hi, b.hi, e1);
    const float2 t1 = p_add(p_add(a.lo, b.lo), e1);
    const float2 s2 = two_sum2(s1, m2h, e2);
    return ff2_norm(s2, p_add(p_add(t1, m2l), e2));
}

// (a - b) - (c - d), normalised once (27 instructions against 33)
__device__ __forceinline__ ff2 cross_diff2(const ff2& a, const ff2& b, const ff2& c, const ff2& d)
{
    float2 e1, e2, e3;
    const float2 s1 = two_sum2(a.hi, p_neg(b.hi), e1);
    const float2 t1 = p_add(p_sub(a.lo, b.lo), e1);
    const float2 s2 = two_sum2(c.hi, p_neg(d.hi), e2);
    const float2 t2 = p_add(p_sub(c.lo, d.lo), e2);
    const float2 s3 = two_sum2(s1, p_neg(s2), e3);
    return ff2_norm(s3, p_add(p_sub(t1, t2), e3));
}

// p1 + p2 + p3 with tails e1..e3, unnormalised: the high parts by TwoSum, all tails in t
__device__ __forceinline__ float2 sum3_2(float2 p1, float2 e1, float2 p2, float2 e2, float2 p3, float2 e3, float2& t)
{
    float2 f1, f2;
    const float2 s1 = two_sum2(p1, p2, f1);
    const float2 s2 = two_sum2(s1, p3, f2);
    t = p_add(p_add(p_add(e1, e2), e3), p_add(f1, f2));
    return s2;
}
__device__ __forceinline__ ff2 ff2_splat(ff a) { return ff2{p_splat(a.hi), p_splat(a.lo)}; }

constexpr int kFzTX = 64, kFzTY = 8;
constexpr int kFzW = kFzTX + 2, kFzP = kFzW * (kFzTY + 2);  // plane region with a 1-cell halo
constexpr size_t kFzSmem = sizeof(float) * 2 * 4 * kFzP;       // hi and lo, 4 ring slots
constexpr size_t kFzSmemCorr = sizeof(float) * 3 * 5 * kFzP;   // + the pending correction e, 5 slots

// The float-float residual of k_residual_ff, z-marching: a block owns a 64 x 8 (x, y) tile
// and NZ planes; the hi and lo parts of the iterate's planes (tile + 1 halo) arrive in
// shared memory by asynchronous copies one plane ahead; each thread evaluates cells
// (x, y) and (x, y + 4) of its plane together.  Grid (n/64, n/8, n/NZ), at most
// kMaxPartials blocks.
//
// CORR: the iterate is U + (E - <E>), the pending correction of the previous outer iteration
// (esum[0] = sum of E), applied to every plane as it arrives in shared memory; the corrected
// iterate is written to Uout (never U: other blocks still read U as their halo), which
// replaces a separate pass chi += e - <e> over the float-float iterate.
template <bool CORR>
__global__ void __launch_bounds__(256, 3) k_residual_ff_zm(const float2* __restrict__ U, const float2* __restrict__ F,
                                                        double lam_host, const double* __restrict__ lamp, int n,
                                                        int NZ, FFCoef k, float* __restrict__ rplain,
                                                        float* __restrict__ chi32, float* __restrict__ gap32,
                                                        uint32_t* __restrict__ coef, double* __restrict__ partials,
                                                        const float* __restrict__ E, const double* __restrict__ esum,
                                                        float2* __restrict__ Uout, double* __restrict__ fin_out = nullptr)
{
    const ff lam1 = ff_from_double(lam_host + (lamp ? *lamp : 0.0));
    const ff2 lam = ff2_splat(lam1);
    const ff2 nu1 = ff2_splat(ff{k.nu1_hi, k.nu1_lo}), kap1 = ff2_splat(ff{k.kap1_hi, k.kap1_lo});
    const ff2 lsat = ff2_splat(ff{k.lsat_hi, k.lsat_lo}), nu = ff2_splat(ff{k.nu_hi, k.nu_lo});
    const bool screened = k.kap_f != 0.f;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // ring slots: 4 (planes s-1 .. s+1 read, s+2 arriving); CORR 5 (s+2 being corrected,
    // s+3 arriving), so that a plane is corrected one step before it is read and the next
    // step's barrier publishes it
    constexpr int NSL = CORR ? 5 : 4;
    float* sh = reinterpret_cast<float*>(smem_raw);  // [NSL][H][W] hi parts
    float* sl = sh + NSL * kFzP;                      // [NSL][H][W] lo parts
    float* se = sl + NSL * kFzP;                      // [NSL][H][W] correction (CORR)
    const unsigned sh_s = (unsigned)__cvta_generic_to_shared(sh);
    const unsigned sl_s = (unsigned)__cvta_generic_to_shared(sl);
    const unsigned se_s = (unsigned)__cvta_generic_to_shared(se);
    float mhi = 0.f, mlo = 0.f;  // <E> as a float-float pair
    if (CORR) {
        const double mean = esum[0] / ((double)n * n * n);
        mhi = (float)mean;
        mlo = (float)(mean - (double)mhi);
    }
    const int m = n - 1;
    const int x0 = blockIdx.x * kFzTX, y0 = blockIdx.y * kFzTY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x;
    const size_t plane = (size_t)n * n;
    auto slot = [&](int p) { return ((p - z0 + 1) % NSL) * kFzP; };  // p >= z0 - 1
    constexpr int K = (kFzP + 255) / 256;
    int off[K];
#pragma unroll
    for (int q = 0; q < K; ++q) {
        const int e = t + 256 * q;
        const int yy = e / kFzW, xx = e - yy * kFzW;
        off[q] = e < kFzP ? (((y0 - 1 + yy) & m) * n + ((x0 - 1 + xx) & m)) : -1;
    }
    auto issue = [&](int p) {
        const float* Up = reinterpret_cast<const float*>(U + (size_t)(p & m) * plane);
        const int so = slot(p);
#pragma unroll
        for (int q = 0; q < K; ++q) {
            if (off[q] < 0) continue;
            const unsigned d = 4u * (unsigned)(so + t + 256 * q);
            cp_async4(sh_s + d, Up + 2 * off[q]);
            cp_async4(sl_s + d, Up + 2 * off[q] + 1);
            if (CORR) cp_async4(se_s + d, E + (size_t)(p & m) * plane + off[q]);
        }
        cp_async_commit_group();
    };
    // CORR: hi + lo += e - <e> on the ring slot of plane p (every element of the region).
    // (hi + e) - <e>_hi by two TwoSums, the tails in one sum, one normalisation; elements
    // t and t + 256 of the region go through the paired instructions together.
    static_assert(K == 3 && kFzP > 512 && kFzP <= 768, "three region elements per thread");
    auto correct = [&](int p) {
        const int so = slot(p);
        {
            const int i0 = so + t, i1 = i0 + 256;
            float2 t1, t2;
            const float2 s1 = two_sum2(make_float2(sh[i0], sh[i1]), make_float2(se[i0], se[i1]), t1);
            const float2 s2 = two_sum2(s1, p_splat(-mhi), t2);
            const ff2 r = ff2_norm(s2, p_add(p_add(make_float2(sl[i0], sl[i1]), t1), p_sub(t2, p_splat(mlo))));
            sh[i0] = r.hi.x;
            sh[i1] = r.hi.y;
            sl[i0] = r.lo.x;
            sl[i1] = r.lo.y;
        }
        if (off[2] >= 0) {
            const int i = so + t + 512;
            float t1, t2;
            const float s1 = ff_two_sum(sh[i], se[i], t1);
            const float s2 = ff_two_sum(s1, -mhi, t2);
            const ff r = ff_norm(s2, __fadd_rn(__fadd_rn(sl[i], t1), __fsub_rn(t2, mlo)));
            sh[i] = r.hi;
            sl[i] = r.lo;
        }
    };
    const int x = t & 63, yA = t >> 6;
    const int cA = (yA + 1) * kFzW + x + 1, cB = cA + 4 * kFzW;
    const int gA = (y0 + yA) * n + x0 + x, gB = gA + 4 * n;
    // value of plane slot `b` at offset d from the two centres, as a pair
    auto ld = [&](int b, int d) {
        return ff2{make_float2(sh[b + cA + d], sh[b + cB + d]), make_float2(sl[b + cA + d], sl[b + cB + d])};
    };
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    if (CORR) {
        // each thread corrects the elements it copied itself (no barrier needed for that)
        issue(z0 + 2);  // NZ >= 2
        cp_async_wait_all();
        correct(z0 - 1);
        correct(z0);
        correct(z0 + 1);
        correct(z0 + 2);
    }
    for (int s = z0; s < z0 + NZ; ++s) {
        const size_t os = (size_t)s * plane;  // s is inside [0, n)
        const float2 fA = F[os + gA], fB = F[os + gB];
        if (CORR) {
            if (s > z0) {
                cp_async_wait_all();  // plane s+2, issued during the previous step
                if (s + 2 <= z0 + NZ) correct(s + 2);
            }
            __syncthreads();  // planes up to s+2 corrected and visible; step s-1 done
            if (s + 3 <= z0 + NZ) issue(s + 3);  // its slot held plane s-2, no longer read
        } else {
            cp_async_wait_all();  // planes up to s+1
            __syncthreads();
            if (s + 2 <= z0 + NZ) issue(s + 2);  // its slot held plane s-2, no longer read
        }
        const int bp = slot(s - 1), bc = slot(s), bn = slot(s + 1);
        constexpr int W = kFzW;
        // Error-free transformations with the tails summed in FP32 and one normalisation per
        // quantity; every step's error is ~2^-47 of the largest operand, as in ff2_add.
        const ff2 c0 = ld(bc, 0);
        const float2 m2h = p_mul(p_splat(-2.f), c0.hi), m2l = p_mul(p_splat(-2.f), c0.lo);
        const ff2 X = second_diff2(ld(bc, 1), ld(bc, -1), m2h, m2l);
        const ff2 Y = second_diff2(ld(bc, W), ld(bc, -W), m2h, m2l);
        const ff2 Z = second_diff2(ld(bn, 0), ld(bp, 0), m2h, m2l);
        const ff2 exy = cross_diff2(ld(bc, 1 + W), ld(bc, 1 - W), ld(bc, -1 + W), ld(bc, -1 - W));
        const ff2 exz = cross_diff2(ld(bn, 1), ld(bp, 1), ld(bn, -1), ld(bp, -1));
        const ff2 eyz = cross_diff2(ld(bn, W), ld(bp, W), ld(bn, -W), ld(bp, -W));
        ff2 L1;
        {
            float2 e1, e2;
            const float2 s1 = two_sum2(X.hi, Y.hi, e1);
            const float2 s2 = two_sum2(s1, Z.hi, e2);
            L1 = ff2_norm(s2, p_add(p_add(p_add(X.lo, Y.lo), Z.lo), p_add(e1, e2)));
        }
        // q2 = 2 (XY + YZ + ZX) - (exy^2 + exz^2 + eyz^2) / 8
        ff2 q2;
        {
            float2 e1, e2, e3, e4, e5, e6, prt, sqt, f;
            const float2 p1 = uprod2(X, Y, e1), p2 = uprod2(Y, Z, e2), p3 = uprod2(Z, X, e3);
            const float2 p4 = uprod2(exy, exy, e4), p5 = uprod2(exz, exz, e5), p6 = uprod2(eyz, eyz, e6);
            const float2 prs = sum3_2(p1, e1, p2, e2, p3, e3, prt);
            const float2 sqs = sum3_2(p4, e4, p5, e5, p6, e6, sqt);
            const float2 qs = two_sum2(p_mul(p_splat(2.f), prs), p_mul(p_splat(-0.125f), sqs), f);
            q2 = ff2_norm(qs, p_add(p_fma(p_splat(2.f), prt, p_mul(p_splat(-0.125f), sqt)), f));
        }
        // G = nu1 L1 - kap1 q2 - (f + lambda), one TwoSum chain; only its rounded value is used
        float2 Gf;
        {
            float2 e1, e2, f1, f2, f3;
            const float2 a1 = uprod2(nu1, L1, e1), a2 = uprod2(kap1, q2, e2);
            const float2 fh = make_float2(fA.x, fB.x), fl = make_float2(fA.y, fB.y);
            const float2 s1 = two_sum2(a1, p_neg(a2), f1);
            const float2 s2 = two_sum2(s1, p_neg(fh), f2);
            const float2 s3 = two_sum2(s2, p_neg(lam.hi), f3);
            const float2 t = p_add(p_add(p_sub(p_sub(e1, e2), p_add(fl, lam.lo)), p_add(f1, f2)), f3);
            Gf = p_add(s3, t);
        }
        // g = L_sat - L1/h^2 (1/h^2 a power of two) and nu g, the floored cells' residual
        float2 gf, ngf;
        {
            float2 f;
            const float2 ih2 = p_splat(k.ih2);
            const float2 gs = two_sum2(lsat.hi, p_neg(p_mul(ih2, L1.hi)), f);
            const float2 gt = p_add(p_sub(lsat.lo, p_mul(ih2, L1.lo)), f);
            gf = p_add(gs, gt);
            const float2 p = p_mul(nu.hi, gs);
            float2 e = p_fma(nu.hi, gs, p_neg(p));
            e = p_fma(nu.hi, gt, e);
            e = p_fma(nu.lo, gs, e);
            ngf = p_add(p, e);
        }
        const float2 Lf = p_mul(p_add(L1.hi, L1.lo), p_splat(k.ih2));
        const float2 Ep = p_mul(p_fma(p_splat(8.f * k.kap_f), Lf, p_splat(-6.f * k.nu_f)), p_splat(k.ih2));
        const float P4 = -96.f * k.kap_f * k.ih2 * k.ih2;  // 4 P
        const float2 D = p_fma(p_splat(-P4), Gf, p_mul(Ep, Ep));
        const bool flA = screened && D.x < k.Df, flB = screened && D.y < k.Df;
        const float rvA = flA ? ngf.x : -Gf.x;
        const float rvB = flB ? ngf.y : -Gf.y;
        if (coef) {
            // the background's bilinear coefficients for the inner sweeps, from the second and
            // cross differences just formed (their high parts: BF16 needs no more)
            const size_t cells = plane * (size_t)n;
            const float2 cX = p_mul(p_splat(2.f), p_add(Y.hi, Z.hi)), cY = p_mul(p_splat(2.f), p_add(X.hi, Z.hi));
            const float2 cZ = p_mul(p_splat(2.f), p_add(X.hi, Y.hi));
            const float2 cxy = p_mul(p_splat(-0.25f), exy.hi), cxz = p_mul(p_splat(-0.25f), exz.hi),
                         cyz = p_mul(p_splat(-0.25f), eyz.hi);
            coef[os + gA] = pack_bf16x2(cX.x, cY.x);
            coef[os + gB] = pack_bf16x2(cX.y, cY.y);
            coef[cells + os + gA] = pack_bf16x2(cZ.x, cxy.x);
            coef[cells + os + gB] = pack_bf16x2(cZ.y, cxy.y);
            coef[2 * cells + os + gA] = pack_bf16x2(cxz.x, cyz.x);
            coef[2 * cells + os + gB] = pack_bf16x2(cxz.y, cyz.y);
        }
        if (CORR) {
            Uout[os + gA] = make_float2(c0.hi.x, c0.lo.x);
            Uout[os + gB] = make_float2(c0.hi.y, c0.lo.y);
        }
        rplain[os + gA] = -Gf.x;
        rplain[os + gB] = -Gf.y;
        chi32[os + gA] = c0.hi.x;
        chi32[os + gB] = c0.hi.y;
        gap32[os + gA] = screened ? gf.x : 0.f;
        gap32[os + gB] = screened ? gf.y : 0.f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float d = h ? rvB : rvA;
            const bool fl = h ? flB : flA;
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
    }
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x, fin_out);
}

}  // namespace pmeft
