// outer_ff.cuh -- the outer loop of the mixed-precision solve in float-float arithmetic.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, and the outer residual of the defect
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
// 2^-53, a factor 64 looser, far below the 1e-8 relative residual the loop stops at.
// The right-hand side src*delta is converted to float-float once per solve; the caller's
// FP64 guess once on entry and the result once on exit, where one FP64 residual of the
// returned chi confirms the stop test.
#pragma once

#include "internal.cuh"

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
                                                     float* __restrict__ gap32, double* __restrict__ partials)
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
    block_sums<5>(acc, partials);
}

}  // namespace pmeft
