// sweep_zero.cuh -- the first red-black sweep of the finest inner level, from a zero start.
//
// Every outer iteration of the mixed-precision loop starts the FP32 inner V-cycle on the
// correction e = 0 (Sec. 3.4 FAS, in the correction form of the defect-correction loop).  The
// first pre-smoothing sweep then needs almost nothing of the general kernels' 19-point
// stencils:
//   - red cells see only zeros: X = Y = Z = 0, no cross differences, so q2 = 0 and the local
//     quadratic of Sec. 3.2.1 has E = -(f + lambda), E' = (8 kappa (L_sat - gap) - 6 nu)/h^2;
//     the update depends on the cell's own right-hand side and gap alone;
//   - black cells see the six new red faces and zeros elsewhere (their centre and the 12
//     same-colour edge neighbours are still zero at the half-sweep's start), so only the
//     background coefficients of X, Y and Z enter (the first two coefficient words).
// The arithmetic is that of the general kernels (local_eval2_cf and pick_update of
// sweep_pair.cuh) with those zeros put in, so the result is the general sweep's on e = 0.
// The kernel replaces the clearing of e and the first general sweep: it reads the right-hand
// side, the gap and two of the three coefficient words and writes e, 20 bytes per cell
// instead of 4 + 29.
//
// Layout: a block owns a TX x TY tile of x-y rows and marches NZ planes up z.  A thread owns
// the column pair (x, x + 1), x even, of one row; on every plane one of the two is red and the
// other black.  Step s computes the red cell of plane s (rows -1 .. TY of the tile, so the
// black cells on the tile's y edges have their faces) and the black cell of plane s - 2, each
// by a scalar formula with the zeros taken out.  The black cell's z-faces are the red values
// of planes s - 1 and s - 3 in its column, which this thread computed itself; its in-plane
// faces are the red values of plane s - 2 of the pair and of the neighbouring pairs and rows,
// from a three-slot shared ring (one value per pair: the red one).  One more warp computes the
// red cells just outside the tile in x (x = -1 and x = TX).  Fields are loaded PF planes
// ahead into registers (8-byte loads of the pair, coalesced per row).
#pragma once

#include "sweep_pair.cuh"

namespace pmeft {

template <int TX, int TY>
struct ZeroGeom {
    static constexpr int WPR = TX / 64;             // warps per row (32 column pairs each)
    static constexpr int RW = TX / 2 + 2;           // ring row: x = -1, the pairs, x = TX
    static constexpr int RH = TY + 2;               // ring rows: y = -1 .. TY
    static constexpr int NXH = 2 * RH;              // x-halo lanes
    static constexpr int NXW = (NXH + 31) / 32;     // x-halo warps
    static constexpr int NRW = RH * WPR;            // row warps
    static constexpr int NW = NRW + NXW;            // row warps + x-halo warps
    static constexpr int NT = 32 * NW;
};

// The general kernels' local evaluation (local_eval2_cf, per lane) and pick_update with the
// zeros of the first sweep put in, operation for operation, so that each result is the
// general sweep's; the terms the zeros remove are left out.  The round-to-nearest intrinsics
// keep the compiler from contracting a product into a neighbouring sum (the general kernels'
// paired instructions are never contracted either).
struct ZeroConst {
    float ih2, nuih2, nu6, kap, kap1, m4P, sp, Df, lsat, h2over6, inv2P;
};

__device__ __forceinline__ float zero_pick(const ZeroConst& k, float G, float Ltot, float g)
{
    const float Ep = __fmul_rn(__fmaf_rn(8.f, __fmul_rn(k.kap, Ltot), k.nu6), k.ih2);
    if (k.kap == 0.f) return div_ftz(-G, Ep);
    const float D = __fmaf_rn(k.m4P, G, __fmul_rn(Ep, Ep));
    return pick_update(G, Ep, 0.f, D, g, k.sp, k.Df, k.h2over6, k.inv2P);
}

// Red cell: every stencil value zero, so L = 0 and q2 = 0: E = -(rhs), the gap unchanged.
__device__ __forceinline__ float zero_red(const ZeroConst& k, float rhs, float gapx)
{
    const float lsat = k.kap != 0.f ? k.lsat : 0.f;
    const float Ltot = __fsub_rn(lsat, gapx);
    const float g = k.kap != 0.f ? gapx : 0.f;
    return __fadd_rn(0.f, zero_pick(k, __fsub_rn(0.f, rhs), Ltot, g));
}

// Black cell: the six faces (sums ax, ay, az of the new red values), centre and edges zero, so
// X = ax, Y = ay, Z = az and no cross differences; the background enters through cX, cY, cZ.
__device__ __forceinline__ float zero_black(const ZeroConst& k, float ax, float ay, float az, const BgCoef& cf,
                                            float rhs, float gapx)
{
    const float L1 = __fadd_rn(__fadd_rn(ax, ay), az);
    float pr = __fmul_rn(ax, ay);
    pr = __fmaf_rn(ay, az, pr);
    pr = __fmaf_rn(az, ax, pr);
    float q2 = __fmul_rn(2.f, pr);
    q2 = __fmaf_rn(cf.cX, ax, q2);
    q2 = __fmaf_rn(cf.cY, ay, q2);
    q2 = __fmaf_rn(cf.cZ, az, q2);
    const float lsat = k.kap != 0.f ? k.lsat : 0.f;
    float g = __fmaf_rn(-k.ih2, L1, gapx);
    const float Ltot = __fsub_rn(lsat, g);
    g = k.kap != 0.f ? g : 0.f;
    const float N = __fmaf_rn(-1.f, __fmul_rn(k.kap1, q2), __fmul_rn(k.nuih2, L1));
    return __fadd_rn(0.f, zero_pick(k, __fsub_rn(N, rhs), Ltot, g));
}

// One sweep from e = 0 into V (n^3).  F: right-hand side (fscale F + lam [+ *lamp]); gap:
// L_sat - L(background); coef: the three BF16-pair planes of the background coefficients
// (only the first two are read).  Tile TX x TY (TX = 64 or 128), PF: planes of fields loaded
// ahead.  Grid (n / TX, n / TY, n / NZ), n >= TX.
template <int TX, int TY, int PF>
__global__ void __launch_bounds__(ZeroGeom<TX, TY>::NT, ZeroGeom<TX, TY>::NT <= 512 ? 2 : 1) k_sweep_zero(float* __restrict__ V, const float* __restrict__ F,
                                                                 float fscale, float lam, const float* __restrict__ gap,
                                                                 int n, int NZ, float ih2, float nu, float kap, float sp,
                                                                 float Df, float lsat, const float* __restrict__ lamp,
                                                                 const uint32_t* __restrict__ coef)
{
    using G = ZeroGeom<TX, TY>;
    constexpr int RW = G::RW, RH = G::RH;
    __shared__ float ring[3][RH][RW];  // red values of three planes, slot (p - z0 + 1) mod 3
    if (lamp) lam += *lamp;
    const int m = n - 1;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const size_t plane = (size_t)n * n, cells = plane * (size_t)n;
    ZeroConst K;
    K.ih2 = ih2;
    K.nuih2 = nu * ih2;
    K.nu6 = -6.f * nu;
    K.kap = kap;
    K.kap1 = kap * (ih2 * ih2);
    K.m4P = -4.f * (-24.f * K.kap1);
    K.sp = sp;
    K.Df = Df;
    K.lsat = lsat;
    K.h2over6 = 1.f / (6.f * ih2);
    K.inv2P = kap != 0.f ? 1.f / (-48.f * kap * ih2 * ih2) : 0.f;
    auto slot = [&](int p) { return (p - z0 + 1) % 3; };  // p >= z0 - 1
    const int zred = z0 + NZ;                            // red planes z0 - 1 .. zred

    if (warp < G::NRW) {
        // ---------------------------------------------------------------- row warps
        const int y = warp / G::WPR - 1;  // -1 .. TY
        const bool interior = y >= 0 && y < TY;
        const int q = (warp % G::WPR) * 32 + lane;  // column pair
        const size_t rowoff = (size_t)((y0 + y) & m) * n + x0 + 2 * q;  // x0 + 2q + 1 < n: no wrap in x
        // fields of the next PF planes: k = 0 the next, PF - 1 the last loaded
        float2 fN[PF], gN[PF];
        uint2 c0N[PF], c1N[PF];
#pragma unroll
        for (int k = 0; k < PF; ++k) {
            fN[k] = gN[k] = make_float2(0.f, 0.f);
            c0N[k] = c1N[k] = make_uint2(0u, 0u);
        }
        auto load = [&](int p, int k) {
            const size_t o = (size_t)(p & m) * plane + rowoff;
            fN[k] = *reinterpret_cast<const float2*>(F + o);
            gN[k] = *reinterpret_cast<const float2*>(gap + o);
            if (interior) {
                c0N[k] = *reinterpret_cast<const uint2*>(coef + o);
                c1N[k] = *reinterpret_cast<const uint2*>(coef + cells + o);
            }
        };
        // fields of the black cells of planes s - 1 (b1) and s - 2 (b2)
        float b1F = 0.f, b1G = 0.f, b2F = 0.f, b2G = 0.f;
        uint32_t b1C0 = 0u, b1C1 = 0u, b2C0 = 0u, b2C1 = 0u;
        // red values of planes s - 1 (column 1 - C), s - 2 (column C), s - 3 (column 1 - C)
        float r1 = 0.f, r2 = 0.f, r3 = 0.f;
#pragma unroll
        for (int k = 0; k < PF; ++k)
            if (z0 - 1 + k <= zred) load(z0 - 1 + k, k);
        for (int s = z0 - 1; s <= zred + 1; ++s) {
            const float2 fc = fN[0], gc = gN[0];
            const uint2 c0c = c0N[0], c1c = c1N[0];
#pragma unroll
            for (int k = 0; k + 1 < PF; ++k) {
                fN[k] = fN[k + 1];
                gN[k] = gN[k + 1];
                c0N[k] = c0N[k + 1];
                c1N[k] = c1N[k + 1];
            }
            if (s + PF <= zred) load(s + PF, PF - 1);
            const int C = (y0 + y + s) & 1;  // the column of the pair that is red on planes s, s - 2
            const bool blk = interior && s - 2 >= z0;
            // black cell of plane s - 2 (column 1 - C): in-plane faces from the ring
            float bax = 0.f, bay = 0.f;
            if (blk) {
                const float(*r)[RW] = ring[slot(s - 2)];
                // its x-neighbour outside the pair: the red cell of pair q + 1 (black column 1) or of
                // pair q - 1 (black column 0)
                const float rout = C ? r[y + 1][q] : r[y + 1][q + 2];
                bax = __fadd_rn(r2, rout);
                bay = __fadd_rn(r[y + 2][q + 1], r[y][q + 1]);
            }
            // the red cell of plane s
            const float vr = zero_red(K, __fmaf_rn(fscale, C ? fc.y : fc.x, lam), C ? gc.y : gc.x);
            if (s <= zred) ring[slot(s)][y + 1][q + 1] = vr;
            if (blk) {
                // the black cell of plane s - 2
                const float vb = zero_black(K, bax, bay, __fadd_rn(r1, r3), unpack_bg_coef(b2C0, b2C1, 0u),
                                            __fmaf_rn(fscale, b2F, lam), b2G);
                const float2 out = C ? make_float2(vb, r2) : make_float2(r2, vb);
                *reinterpret_cast<float2*>(V + (size_t)(s - 2) * plane + rowoff) = out;
            }
            // the black cell of plane s is column 1 - C
            b2F = b1F;
            b2G = b1G;
            b2C0 = b1C0;
            b2C1 = b1C1;
            b1F = C ? fc.x : fc.y;
            b1G = C ? gc.x : gc.y;
            b1C0 = C ? c0c.x : c0c.y;
            b1C1 = C ? c1c.x : c1c.y;
            r3 = r2;
            r2 = r1;
            r1 = vr;
            __syncthreads();
        }
    } else {
        // ---------------------------------------------------------------- x-halo lanes
        const int idx = (warp - G::NRW) * 32 + lane;
        const bool active = idx < G::NXH;
        const int side = idx < RH ? 0 : 1;  // 0: x = -1, 1: x = TX
        const int y = (active ? idx % RH : 0) - 1;
        const int xg = side ? ((x0 + TX) & m) : ((x0 - 1) & m);
        const int col = side ? RW - 1 : 0;
        const size_t rowoff = (size_t)((y0 + y) & m) * n + xg;
        for (int s = z0 - 1; s <= zred + 1; ++s) {
            // red on plane s when x + y + s is even (x = x0 - 1 or x0 + TX, x0 even)
            const bool red = active && s <= zred && ((1 - side + y0 + y + s) & 1) == 0;
            if (red) {
                const size_t o = (size_t)(s & m) * plane + rowoff;
                ring[slot(s)][y + 1][col] = zero_red(K, __fmaf_rn(fscale, F[o], lam), gap[o]);
            }
            __syncthreads();
        }
    }
}

}  // namespace pmeft
