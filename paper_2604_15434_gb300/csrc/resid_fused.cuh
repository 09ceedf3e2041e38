// resid_fused.cuh -- the FP32 residual of the inner cycle on large levels, z-marching.
//
// The same per-cell arithmetic as k_residual (FP32, background, floored piece, the five
// block sums), but each block owns a 64 x 8 (x, y) tile and walks NZ planes in z, with the
// planes of the iterate and of the background (tile + 1-cell halo) arriving in shared
// memory through asynchronous copies issued one plane ahead.  The 19-point stencil is then
// read from shared memory instead of 38 scattered global loads per cell; every input is
// read from DRAM once, the halos from L2.
#pragma once

#include "sweep_fused.cuh"

namespace pmeft {

constexpr int kRzTX = 64, kRzTY = 8;
constexpr int kRzW = kRzTX + 2, kRzH = kRzTY + 2, kRzP = kRzW * kRzH;  // plane region with halo
constexpr int kRzSlots = 4;  // planes s-1 .. s+1 in use, s+2 arriving

template <bool BG, bool COEF = false>
constexpr size_t resid_zm_smem_bytes()
{
    return sizeof(float) * (size_t)kRzSlots * kRzP * ((BG && !COEF) ? 2 : 1);
}

// Grid (n/64, n/8, n/NZ), 256 threads; the block count must not exceed kMaxPartials.
// COEF: the background enters through its per-cell coefficients (BgCoef), not its planes.
template <bool BG, bool COEF = false>
__global__ void __launch_bounds__(256) k_residual_zm(const float* __restrict__ u, const float* __restrict__ F,
                                                     float fscale, float lam, const uint8_t* __restrict__ kmask,
                                                     const float* __restrict__ bg, const float* __restrict__ gap, int n,
                                                     int NZ, float ih2, float nu, float kap, float Df, float lsat_c,
                                                     bool floor_piece, float* __restrict__ r,
                                                     uint8_t* __restrict__ sat, double* __restrict__ partials,
                                                     const float* __restrict__ lamp, const uint32_t* __restrict__ coef)
{
    constexpr bool BGRING = BG && !COEF;
    if (lamp) lam += *lamp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* su = reinterpret_cast<float*>(smem_raw);  // [slots][H][W]
    float* sb = su + kRzSlots * kRzP;                 // [slots][H][W] (BG)
    const unsigned su_s = (unsigned)__cvta_generic_to_shared(su);
    const unsigned sb_s = (unsigned)__cvta_generic_to_shared(sb);
    const int m = n - 1;
    const int x0 = blockIdx.x * kRzTX, y0 = blockIdx.y * kRzTY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x;
    const size_t plane = (size_t)n * n;
    auto slot = [&](int p) { return ((p - z0 + 4) & 3) * kRzP; };  // p >= z0 - 1
    constexpr int K = (kRzP + 255) / 256;
    int off[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int q = t + 256 * k;
        const int yy = q / kRzW, xx = q - yy * kRzW;
        off[k] = q < kRzP ? (((y0 - 1 + yy) & m) * n + ((x0 - 1 + xx) & m)) : -1;
    }
    auto issue = [&](int p) {
        const float* Up = u + (size_t)(p & m) * plane;
        const float* Bp = bg + (size_t)(p & m) * plane;
        const int so = slot(p);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            if (off[k] < 0) continue;
            const unsigned d = 4u * (unsigned)(so + t + 256 * k);
            cp_async4(su_s + d, Up + off[k]);
            if (BGRING) cp_async4(sb_s + d, Bp + off[k]);
        }
        cp_async_commit_group();
    };
    // two cells per thread and plane: (x, y) and (x, y + 4)
    const int x = t & 63, yA = t >> 6;
    const int cs[2] = {(yA + 1) * kRzW + x + 1, (yA + 5) * kRzW + x + 1};
    const int gxy[2] = {(y0 + yA) * n + x0 + x, (y0 + yA + 4) * n + x0 + x};
    auto stencil = [&](const float* rp, const float* rc, const float* rn, int c) {
        Stencil<float> s;
        s.c0 = rc[c];
        s.ax = rc[c + 1] + rc[c - 1];
        s.ay = rc[c + kRzW] + rc[c - kRzW];
        s.az = rn[c] + rp[c];
        s.exy = rc[c + 1 + kRzW] - rc[c + 1 - kRzW] - rc[c - 1 + kRzW] + rc[c - 1 - kRzW];
        s.exz = rn[c + 1] - rp[c + 1] - rn[c - 1] + rp[c - 1];
        s.eyz = rn[c + kRzW] - rp[c + kRzW] - rn[c - kRzW] + rp[c - kRzW];
        return s;
    };
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    for (int s = z0; s < z0 + NZ; ++s) {
        const size_t os = (size_t)s * plane;  // s is inside [0, n)
        float fv[2], gv[2];
        uint32_t cw[2][3];
        float wk[2];  // screening weights
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            fv[h] = F[os + gxy[h]];
            gv[h] = gap ? gap[os + gxy[h]] : 0.f;
            wk[h] = screen_w<float>(kmask, os + gxy[h]);
            if (COEF) {
                const size_t cells = plane * (size_t)n;
                cw[h][0] = coef[os + gxy[h]];
                cw[h][1] = coef[cells + os + gxy[h]];
                cw[h][2] = coef[2 * cells + os + gxy[h]];
            }
        }
        cp_async_wait_all();  // planes up to s+1
        __syncthreads();
        if (s + 2 <= z0 + NZ) issue(s + 2);  // its slot held plane s-2, no longer read
        const float* up = su + slot(s - 1);
        const float* uc = su + slot(s);
        const float* un = su + slot(s + 1);
        const float* bp = sb + slot(s - 1);
        const float* bc = sb + slot(s);
        const float* bn = sb + slot(s + 1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            Stencil<float> a = stencil(up, uc, un, cs[h]);
            const float kc = kap * wk[h];
            const float lsat = kc != 0.f ? lsat_c / wk[h] : 0.f;
            Local<float> o;
            if (COEF) {
                o = local_eval_cf(a, unpack_bg_coef(cw[h][0], cw[h][1], cw[h][2]), ih2, nu, kc, fscale * fv[h] + lam,
                                  lsat, gv[h]);
            } else {
                Stencil<float> b;
                if (BG) b = stencil(bp, bc, bn, cs[h]);
                o = local_eval<float, BG>(a, b, ih2, nu, kc, fscale * fv[h] + lam, lsat, gap != nullptr, gv[h]);
            }
            // the floored piece exists on the finest level only (see k_residual)
            const bool fl = floor_piece && (o.P != 0.f) && (o.D < Df);
            const float rv = fl ? nu * o.g : -o.G;
            r[os + gxy[h]] = rv;
            if (sat) sat[os + gxy[h]] = fl ? 1 : 0;
            if (!isfinite(rv)) {
                fa[4] += 1.f;
            } else {
                fa[0] += rv;
                fa[2] += rv * rv;
                if (!fl) {
                    fa[1] += rv;
                    fa[3] += 1.f;
                }
            }
        }
    }
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x);
}

}  // namespace pmeft
