// resid_fused.cuh -- the FP32 residual of the inner cycle on large levels, z-marching.
//
// The same per-cell arithmetic as k_residual (FP32, background, floored piece, the five
// block sums), but each block owns a 64 x 8 (x, y) tile and walks NZ planes in z, with the
// planes of the iterate and of the background (tile + 1-cell halo) arriving in shared
// memory through asynchronous copies issued one plane ahead.  The 19-point stencil is then
// read from shared memory instead of 38 scattered global loads per cell; every input is
// read from DRAM once, the halos from L2.
#pragma once

#include "sweep_pair.cuh"

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
// RESTRICT: the FAS restriction is done here instead of writing r and sat for k_restrict_fas:
// for every coarse cell (2x2x2 children; NZ even) it writes the children's mean iterate to
// ur and uc, the children's mean raw residual to rc, and the byte kmc = (mean unscreened
// eighths, as k_restrict_fas) | (unfloored children << 4).  The gauge term -gm * [unfloored]
// needs the finished residual sums, so k_fas_rhs applies it from the high nibble and clears
// it.  Children pair up across lanes x, x^1 (shuffle), rows y, y+1 (threads t, t+64: shared
// memory) and planes s, s+1 (registers).
template <bool BG, bool COEF = false, bool RESTRICT = false>
__global__ void __launch_bounds__(256) k_residual_zm(const float* __restrict__ u, const float* __restrict__ F,
                                                     float fscale, float lam, const uint8_t* __restrict__ kmask,
                                                     const float* __restrict__ bg, const float* __restrict__ gap, int n,
                                                     int NZ, float ih2, float nu, float kap, float Df, float lsat_c,
                                                     bool floor_piece, float* __restrict__ r,
                                                     uint8_t* __restrict__ sat, double* __restrict__ partials,
                                                     const float* __restrict__ lamp, const uint32_t* __restrict__ coef,
                                                     float* __restrict__ urc = nullptr, float* __restrict__ ucc = nullptr,
                                                     float* __restrict__ rcc = nullptr, uint8_t* __restrict__ kmc = nullptr,
                                                     double* __restrict__ fin_out = nullptr)
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
    float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // RESTRICT: per cell h the running sums over the plane pair of iterate, residual,
    // unscreened eighths and unfloored children; xch carries rows y+1 to rows y
    float au[2] = {0.f, 0.f}, ar[2] = {0.f, 0.f}, ac[2] = {0.f, 0.f}, an[2] = {0.f, 0.f};
    __shared__ float xch[RESTRICT ? 8 : 1][64];
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
        // both cells of the thread evaluated together on the paired FP32 instructions
        // (local_eval2 / local_eval2_cf of the pair sweep)
        auto st2 = [&](const float* rp, const float* rc, const float* rn) {
            auto at = [&](const float* p, int d) { return make_float2(p[cs[0] + d], p[cs[1] + d]); };
            constexpr int W = kRzW;
            Stencil2 q;
            q.c0 = at(rc, 0);
            q.ax = f2add(at(rc, 1), at(rc, -1));
            q.ay = f2add(at(rc, W), at(rc, -W));
            q.az = f2add(at(rn, 0), at(rp, 0));
            q.exy = f2add(f2sub(f2sub(at(rc, 1 + W), at(rc, 1 - W)), at(rc, -1 + W)), at(rc, -1 - W));
            q.exz = f2add(f2sub(f2sub(at(rn, 1), at(rp, 1)), at(rn, -1)), at(rp, -1));
            q.eyz = f2add(f2sub(f2sub(at(rn, W), at(rp, W)), at(rn, -W)), at(rp, -W));
            return q;
        };
        const Stencil2 a2 = st2(up, uc, un);
        const float2 kc2 = make_float2(kap * wk[0], kap * wk[1]);
        // L_sat / w (w = 1 without a mask: no division)
        const float2 lsat2 = kmask ? make_float2(kc2.x != 0.f ? lsat_c / wk[0] : 0.f, kc2.y != 0.f ? lsat_c / wk[1] : 0.f)
                                   : make_float2(kc2.x != 0.f ? lsat_c : 0.f, kc2.y != 0.f ? lsat_c : 0.f);
        const float2 rhs2 = make_float2(fscale * fv[0] + lam, fscale * fv[1] + lam);
        const float2 gap2 = make_float2(gv[0], gv[1]);
        Local2 o2;
        if (COEF) {
            o2 = local_eval2_cf(a2, unpack_bg_coef(cw[0][0], cw[0][1], cw[0][2]),
                                unpack_bg_coef(cw[1][0], cw[1][1], cw[1][2]), ih2, nu, kc2, rhs2, lsat2, gap2);
        } else {
            Stencil2 b2;
            if (BG) b2 = st2(bp, bc, bn);
            o2 = gap ? local_eval2<BG, true>(a2, b2, ih2, nu, kc2, rhs2, lsat2, gap2)
                     : local_eval2<BG, false>(a2, b2, ih2, nu, kc2, rhs2, lsat2, gap2);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float oG = h ? o2.G.y : o2.G.x, oP = h ? o2.P.y : o2.P.x, oD = h ? o2.D.y : o2.D.x,
                        og = h ? o2.g.y : o2.g.x;
            // the floored piece exists on the finest level only (see k_residual)
            const bool fl = (oP != 0.f) && (oD < (floor_piece ? Df : 0.f));
            const float rv = fl ? nu * og : -oG;
            if (RESTRICT) {
                const int kf = kmask ? (kmask[os + gxy[h]] < 8 ? kmask[os + gxy[h]] : 8) : 0;
                au[h] += h ? a2.c0.y : a2.c0.x;
                ar[h] += rv;
                ac[h] += fl ? 8.f : (float)kf;
                an[h] += fl ? 0.f : 1.f;
            } else {
                r[os + gxy[h]] = rv;
                if (sat) sat[os + gxy[h]] = fl ? 1 : 0;
            }
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
        if (RESTRICT && ((s - z0) & 1)) {
            // the plane pair (s - 1, s) is complete: combine x pairs, then row pairs
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                au[h] += __shfl_xor_sync(0xffffffffu, au[h], 1);
                ar[h] += __shfl_xor_sync(0xffffffffu, ar[h], 1);
                ac[h] += __shfl_xor_sync(0xffffffffu, ac[h], 1);
                an[h] += __shfl_xor_sync(0xffffffffu, an[h], 1);
            }
            const int q = (yA >> 1) * 32 + (x >> 1);
            if ((yA & 1) && !(x & 1)) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    xch[4 * h + 0][q] = au[h];
                    xch[4 * h + 1][q] = ar[h];
                    xch[4 * h + 2][q] = ac[h];
                    xch[4 * h + 3][q] = an[h];
                }
            }
            __syncthreads();
            if (!(yA & 1) && !(x & 1)) {
                const int nc = n >> 1;
                const size_t K = (size_t)(s >> 1), I = (size_t)((x0 + x) >> 1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float su = au[h] + xch[4 * h + 0][q], sr = ar[h] + xch[4 * h + 1][q];
                    const int cnt = (int)(ac[h] + xch[4 * h + 2][q]), nun = (int)(an[h] + xch[4 * h + 3][q]);
                    const size_t J = (size_t)((y0 + yA + 4 * h) >> 1);
                    const size_t c = (K * nc + J) * nc + I;
                    urc[c] = 0.125f * su;
                    ucc[c] = 0.125f * su;
                    rcc[c] = 0.125f * sr;
                    kmc[c] = (uint8_t)(((cnt + 4) >> 3) | (nun << 4));
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h) au[h] = ar[h] = ac[h] = an[h] = 0.f;
        }
    }
    double acc[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) acc[q] = (double)fa[q];
    block_sums<5>(acc, partials, (blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x, fin_out);
}

}  // namespace pmeft
