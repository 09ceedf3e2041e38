// sweep_pair.cuh -- the single-pass FP32 red-black sweep, two cells per thread.
//
// The plane ring, the snapshot semantics and the arithmetic are those of k_sweep_fused
// (sweep_fused.cuh); what changes is the work split.  Each thread updates two cells of the
// same colour at once, held in the two components of float2 values, so that every
// arithmetic step is one paired Blackwell instruction (FADD2 / FMUL2 / FFMA2) for both
// cells, and the index and address work of a unit is shared by its two cells.  The update
// is branch-free: every candidate root is computed and the right one selected per cell.
//
// Tile 64 x TY, 16*TY threads.  Red cells of the tile + 1 halo: per row 33, taken as
// pairs (k, k + 16), k < 16, by half-warps on two adjacent rows (the two rows have
// opposite colour parity, so the half-warps fall on the even and the odd banks); the 33rd
// cell of every row forms pairs of rows (r, r + HR/2) in one extra unit.  Black cells of
// the tile: pairs (k, k + 16) of the 32 per row, half-warps on adjacent rows.
#pragma once

#include "sweep_fused.cuh"

namespace pmeft {

// BAL: one warp per red unit (TY/2 + 2 warps), so that the red update takes one round; the
// black update then leaves two warps idle.  Otherwise TY/2 warps (16 TY threads).
template <int TY, bool BAL = false>
struct PairGeom {
    static constexpr int TX = 64;
    static constexpr int WU = TX + 4, HU = TY + 4;  // old-value / background region
    static constexpr int WR = TX + 2, HR = TY + 2;  // red-update region
    static constexpr int PU = WU * HU, PR = WR * HR;
    static constexpr int NS = 5;                    // ring slots of old planes: s-2 .. s+2
    static constexpr int NT = BAL ? 32 * (TY / 2 + 2) : 16 * TY;  // threads
    static constexpr int NW = NT / 32;
    static constexpr int RED_MAIN = HR / 2;         // row-pair units of red pairs (k, k+16)
    static constexpr int RED_UNITS = RED_MAIN + 1;  // + the unit of the 33rd cells
    static constexpr int BLK_UNITS = TY / 2;
    static constexpr int NRU = (RED_UNITS + NW - 1) / NW;
    static constexpr int NBU = (BLK_UNITS + NW - 1) / NW;
};

template <int TY, bool BG, bool COEF = false>
constexpr size_t pair_smem_bytes()
{
    using G = PairGeom<TY>;
    return sizeof(float) * ((size_t)G::NS * G::PU * ((BG && !COEF) ? 2 : 1) + (size_t)3 * G::PR);
}

__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

struct Stencil2 {
    float2 c0, ax, ay, az, exy, exz, eyz;
};

struct Local2 {
    float2 G, Ep, P, D, g;
};

// local_eval<float, BG> for two cells (h = 1 units; see internal.cuh)
template <bool BG, bool GAP>
__device__ __forceinline__ Local2 local_eval2(const Stencil2& s, const Stencil2& b, float ih2, float nu, float2 kap,
                                              float2 rhs, float2 lsat_c, float2 gapx)
{
    const float2 m2 = f2(-2.f);
    const float2 X = f2fma(m2, s.c0, s.ax);
    const float2 Y = f2fma(m2, s.c0, s.ay);
    const float2 Z = f2fma(m2, s.c0, s.az);
    const float2 L1 = f2add(f2add(X, Y), Z);
    float2 pr = f2mul(X, Y);
    pr = f2fma(Y, Z, pr);
    pr = f2fma(Z, X, pr);
    float2 sq = f2mul(s.exy, s.exy);
    sq = f2fma(s.exz, s.exz, sq);
    sq = f2fma(s.eyz, s.eyz, sq);
    float2 q2 = f2fma(f2(-0.125f), sq, f2mul(f2(2.f), pr));
    float2 L1tot = L1;
    if (BG) {
        const float2 Xb = f2fma(m2, b.c0, b.ax);
        const float2 Yb = f2fma(m2, b.c0, b.ay);
        const float2 Zb = f2fma(m2, b.c0, b.az);
        float2 A = f2mul(Xb, f2add(Y, Z));
        A = f2fma(Yb, f2add(X, Z), A);
        A = f2fma(Zb, f2add(X, Y), A);
        float2 B = f2mul(b.exy, s.exy);
        B = f2fma(b.exz, s.exz, B);
        B = f2fma(b.eyz, s.eyz, B);
        q2 = f2fma(f2(2.f), A, q2);
        q2 = f2fma(f2(-0.25f), B, q2);
        if (!GAP) L1tot = f2add(L1, f2add(f2add(Xb, Yb), Zb));
    }
    Local2 o;
    const float2 lsat = make_float2(kap.x != 0.f ? lsat_c.x : 0.f, kap.y != 0.f ? lsat_c.y : 0.f);
    float2 Ltot;
    if (GAP) {
        o.g = f2fma(f2(-ih2), L1, gapx);  // gap - L1/h^2
        Ltot = f2sub(lsat, o.g);
    } else {
        Ltot = f2mul(L1tot, f2(ih2));
        o.g = f2sub(lsat, Ltot);
    }
    o.g = make_float2(kap.x != 0.f ? o.g.x : 0.f, kap.y != 0.f ? o.g.y : 0.f);
    const float2 kap1 = f2mul(kap, f2(ih2 * ih2));
    const float2 N = f2fma(f2(-1.f), f2mul(kap1, q2), f2mul(f2(nu * ih2), L1));
    o.G = f2sub(N, rhs);
    o.Ep = f2mul(f2fma(f2(8.f), f2mul(kap, Ltot), f2(-6.f * nu)), f2(ih2));
    o.P = f2mul(f2(-24.f), kap1);
    o.D = f2fma(f2mul(f2(-4.f), o.P), o.G, f2mul(o.Ep, o.Ep));
    return o;
}

// local_eval2<BG = true, GAP = true> with the background given by its coefficients (BgCoef
// of both cells, internal.cuh)
__device__ __forceinline__ Local2 local_eval2_cf(const Stencil2& s, const BgCoef& ca, const BgCoef& cb, float ih2,
                                                 float nu, float2 kap, float2 rhs, float2 lsat_c, float2 gapx)
{
    const float2 m2 = f2(-2.f);
    const float2 X = f2fma(m2, s.c0, s.ax);
    const float2 Y = f2fma(m2, s.c0, s.ay);
    const float2 Z = f2fma(m2, s.c0, s.az);
    const float2 L1 = f2add(f2add(X, Y), Z);
    float2 pr = f2mul(X, Y);
    pr = f2fma(Y, Z, pr);
    pr = f2fma(Z, X, pr);
    float2 sq = f2mul(s.exy, s.exy);
    sq = f2fma(s.exz, s.exz, sq);
    sq = f2fma(s.eyz, s.eyz, sq);
    float2 q2 = f2fma(f2(-0.125f), sq, f2mul(f2(2.f), pr));
    q2 = f2fma(make_float2(ca.cX, cb.cX), X, q2);
    q2 = f2fma(make_float2(ca.cY, cb.cY), Y, q2);
    q2 = f2fma(make_float2(ca.cZ, cb.cZ), Z, q2);
    q2 = f2fma(make_float2(ca.cxy, cb.cxy), s.exy, q2);
    q2 = f2fma(make_float2(ca.cxz, cb.cxz), s.exz, q2);
    q2 = f2fma(make_float2(ca.cyz, cb.cyz), s.eyz, q2);
    Local2 o;
    const float2 lsat = make_float2(kap.x != 0.f ? lsat_c.x : 0.f, kap.y != 0.f ? lsat_c.y : 0.f);
    o.g = f2fma(f2(-ih2), L1, gapx);  // gap - L1/h^2
    const float2 Ltot = f2sub(lsat, o.g);
    o.g = make_float2(kap.x != 0.f ? o.g.x : 0.f, kap.y != 0.f ? o.g.y : 0.f);
    const float2 kap1 = f2mul(kap, f2(ih2 * ih2));
    const float2 N = f2fma(f2(-1.f), f2mul(kap1, q2), f2mul(f2(nu * ih2), L1));
    o.G = f2sub(N, rhs);
    o.Ep = f2mul(f2fma(f2(8.f), f2mul(kap, Ltot), f2(-6.f * nu)), f2(ih2));
    o.P = f2mul(f2(-24.f), kap1);
    o.D = f2fma(f2mul(f2(-4.f), o.P), o.G, f2mul(o.Ep, o.Ep));
    return o;
}

// Approximate reciprocal square root and quotient of the special-function unit with subnormal
// inputs and results flushed to zero: for the normal operands of the sweeps they return what
// rsqrtf and __fdividef return, without the instructions that rescale subnormal operands.
__device__ __forceinline__ float rsqrt_ftz(float x)
{
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ float div_ftz(float a, float b)
{
    float r;
    asm("div.approx.ftz.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// local_update_fast for one cell, without branches
__device__ __forceinline__ float pick_update(float G, float Ep, float P, float D, float g, float sp, float Df,
                                             float h2over6, float inv2P)
{
    const float Dc = fmaxf(D, Df);
    const float sq = Dc * rsqrt_ftz(Dc);
    const float r1 = div_ftz(-2.f * G, Ep + sp * sq);
    const float r2 = (sp * sq - Ep) * inv2P;
    float e = (Ep * sp > 0.f) ? r1 : r2;
    e = (D < Df) ? -g * h2over6 : e;
    return e;
}

// COEF (with BG and GAP): the finest inner level, the background entering through its
// per-cell coefficients (three packed BF16 planes) instead of a ring of its planes.
template <int TY, bool BG, bool GAP, bool COEF = false, bool BAL = false>
__global__ void __launch_bounds__(PairGeom<TY, BAL>::NT, TY >= 16 ? (BAL ? 2 : 3) : 1) k_sweep_pair(const float* __restrict__ U, float* __restrict__ V,
                                                       const float* __restrict__ F, float fscale, float lam,
                                                       const uint8_t* __restrict__ kmask, const float* __restrict__ bg,
                                                       const float* __restrict__ gap, int n, int NZ, float ih2,
                                                       float nu, float kap, float sp, float Df, float lsat,
                                                       const float* __restrict__ lamp,
                                                       const uint32_t* __restrict__ coef)
{
    using G = PairGeom<TY, BAL>;
    constexpr bool BGRING = BG && !COEF;
    constexpr int NS = G::NS, NT = G::NT, NW = G::NW, WU = G::WU, WR = G::WR;
    if (lamp) lam += *lamp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* su = reinterpret_cast<float*>(smem_raw);  // [NS][HU][WU] old values
    float* sb = su + NS * G::PU;                      // [NS][HU][WU] background (BG)
    float* sr = sb + (BGRING ? NS * G::PU : 0);       // [3][HR][WR] new red values
    const unsigned su_s = (unsigned)__cvta_generic_to_shared(su);
    const unsigned sb_s = (unsigned)__cvta_generic_to_shared(sb);
    const int m = n - 1;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x;
    const size_t plane = (size_t)n * n;
    auto uslot = [&](int p) { return ((p - z0 + 10) % NS) * G::PU; };
    auto rslot = [&](int p) { return ((p - z0 + 9) % 3) * G::PR; };

    constexpr int KU = (G::PU + NT - 1) / NT;
    int offu[KU];
#pragma unroll
    for (int k = 0; k < KU; ++k) {
        const int q = t + k * NT;
        const int yy = q / WU, xx = q - yy * WU;
        offu[k] = q < G::PU ? (((y0 - 2 + yy) & m) * n + ((x0 - 2 + xx) & m)) : -1;
    }
    auto issue = [&](int p) {
        const float* Up = U + (size_t)(p & m) * plane;
        const float* Bp = bg + (size_t)(p & m) * plane;
        const int so = uslot(p);
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            if (offu[k] < 0) continue;
            const unsigned d = 4u * (unsigned)(so + t + k * NT);
            cp_async4(su_s + d, Up + offu[k]);
            if (BGRING) cp_async4(sb_s + d, Bp + offu[k]);
        }
        cp_async_commit_group();
    };

    const int lane = t & 31, warp = t >> 5;
    const int half = lane >> 4, hl = lane & 15;
    // red pair units: rows (rowA, rowB), smem offsets of the parity-0 cells, global (x, y)
    // offsets of both parities
    int r_rowA[G::NRU], r_rowB[G::NRU], r_cuA[G::NRU], r_cuB[G::NRU], r_crA[G::NRU], r_crB[G::NRU];
    int r_gA0[G::NRU], r_gA1[G::NRU], r_gB0[G::NRU], r_gB1[G::NRU];
#pragma unroll
    for (int it = 0; it < G::NRU; ++it) {
        const int u = warp + NW * it;
        int ra = -1, rb = -1, xa = 0, xb = 0;  // rows and red-region x of parity 0
        if (u < G::RED_MAIN) {
            ra = rb = 2 * u + half;
            xa = 2 * hl;
            xb = xa + 32;
        } else if (u == G::RED_MAIN && lane < G::HR / 2) {
            ra = lane;
            rb = lane + G::HR / 2;
            xa = xb = 64;
        }
        r_rowA[it] = ra;
        r_rowB[it] = rb;
        const int raa = ra < 0 ? 0 : ra, rbb = rb < 0 ? 0 : rb;
        r_cuA[it] = (raa + 1) * WU + xa + 1;
        r_cuB[it] = (rbb + 1) * WU + xb + 1;
        r_crA[it] = raa * WR + xa;
        r_crB[it] = rbb * WR + xb;
        const int oa = ((y0 - 1 + raa) & m) * n, ob = ((y0 - 1 + rbb) & m) * n;
        r_gA0[it] = oa + ((x0 - 1 + xa) & m);
        r_gA1[it] = oa + ((x0 + xa) & m);
        r_gB0[it] = ob + ((x0 - 1 + xb) & m);
        r_gB1[it] = ob + ((x0 + xb) & m);
    }
    // black pair units: row, first pair index
    int b_row[G::NBU];
#pragma unroll
    for (int it = 0; it < G::NBU; ++it) {
        const int u = warp + NW * it;
        b_row[it] = u < G::BLK_UNITS ? 2 * u + half : -1;
    }
    const int bkq = hl;  // black pairs (x2, x2 + 32) with x2 = 2 * bkq

    const float h2over6 = 1.f / (6.f * ih2), inv2P = kap != 0.f ? 1.f / (-48.f * kap * ih2 * ih2) : 0.f;
    auto stencil2 = [&](const float* rp, const float* rc, const float* rn, int ca, int cb) {
        Stencil2 s;
        s.c0 = make_float2(rc[ca], rc[cb]);
        s.ax = f2add(make_float2(rc[ca + 1], rc[cb + 1]), make_float2(rc[ca - 1], rc[cb - 1]));
        s.ay = f2add(make_float2(rc[ca + WU], rc[cb + WU]), make_float2(rc[ca - WU], rc[cb - WU]));
        s.az = f2add(make_float2(rn[ca], rn[cb]), make_float2(rp[ca], rp[cb]));
        s.exy = f2sub(f2sub(make_float2(rc[ca + 1 + WU], rc[cb + 1 + WU]), make_float2(rc[ca + 1 - WU], rc[cb + 1 - WU])),
                      f2sub(make_float2(rc[ca - 1 + WU], rc[cb - 1 + WU]), make_float2(rc[ca - 1 - WU], rc[cb - 1 - WU])));
        s.exz = f2sub(f2sub(make_float2(rn[ca + 1], rn[cb + 1]), make_float2(rp[ca + 1], rp[cb + 1])),
                      f2sub(make_float2(rn[ca - 1], rn[cb - 1]), make_float2(rp[ca - 1], rp[cb - 1])));
        s.eyz = f2sub(f2sub(make_float2(rn[ca + WU], rn[cb + WU]), make_float2(rp[ca + WU], rp[cb + WU])),
                      f2sub(make_float2(rn[ca - WU], rn[cb - WU]), make_float2(rp[ca - WU], rp[cb - WU])));
        return s;
    };
    // iw: 1/weight of a partly screened cell (L_sat and 1/(2P) scale as 1/kappa)
    auto update2 = [&](const Local2& o, float2 kc, float2 iw) {
        float2 e;
        e.x = pick_update(o.G.x, o.Ep.x, o.P.x, o.D.x, o.g.x, sp, Df, h2over6, inv2P * iw.x);
        e.y = pick_update(o.G.y, o.Ep.y, o.P.y, o.D.y, o.g.y, sp, Df, h2over6, inv2P * iw.y);
        if (kc.x == 0.f || kc.y == 0.f) {  // unscreened cells: the linear (Newton) step
            if (kc.x == 0.f) e.x = div_ftz(-o.G.x, o.Ep.x);
            if (kc.y == 0.f) e.y = div_ftz(-o.G.y, o.Ep.y);
        }
        return e;
    };

    issue(z0 - 2);
    issue(z0 - 1);
    issue(z0);
    for (int s = z0 - 1; s <= z0 + NZ; ++s) {
        const int pb = s - 1;
        const bool black = pb >= z0;
        // this step's right-hand side, gap and mask values, before the barrier
        float2 rF[G::NRU], rG[G::NRU], bF[G::NBU], bG[G::NBU];
        float2 rW[G::NRU], bW[G::NBU];  // screening weights (1 without a mask)
        uint2 rC[G::NRU][3], bC[G::NBU][3];  // background coefficients (COEF): .x cell A, .y cell B
        {
            const size_t cells = plane * (size_t)n;
            const size_t os = (size_t)(s & m) * plane, ob = (size_t)(pb & m) * plane;
#pragma unroll
            for (int it = 0; it < G::NRU; ++it) {
                rF[it] = rG[it] = f2(0.f);
                rW[it] = f2(1.f);
                if (r_rowA[it] >= 0) {
                    const size_t ga = os + (size_t)(((r_rowA[it] + s) & 1) ? r_gA1[it] : r_gA0[it]);
                    const size_t gb = os + (size_t)(((r_rowB[it] + s) & 1) ? r_gB1[it] : r_gB0[it]);
                    rF[it] = make_float2(F[ga], F[gb]);
                    if (GAP) rG[it] = make_float2(gap[ga], gap[gb]);
                    if (kmask) {
                        rW[it] = make_float2(screen_w<float>(kmask, ga), screen_w<float>(kmask, gb));
                    }
                    if (COEF) {
#pragma unroll
                        for (int q = 0; q < 3; ++q) rC[it][q] = make_uint2(coef[q * cells + ga], coef[q * cells + gb]);
                    }
                }
            }
#pragma unroll
            for (int it = 0; it < G::NBU; ++it) {
                const int y = b_row[it];
                bF[it] = bG[it] = f2(0.f);
                bW[it] = f2(1.f);
                if (black && y >= 0) {
                    const size_t ga = ob + (size_t)((y0 + y) * n + x0 + 2 * bkq + (((y + pb) & 1) ? 0 : 1));
                    bF[it] = make_float2(F[ga], F[ga + 32]);
                    if (GAP) bG[it] = make_float2(gap[ga], gap[ga + 32]);
                    if (kmask) {
                        bW[it] = make_float2(screen_w<float>(kmask, ga), screen_w<float>(kmask, ga + 32));
                    }
                    if (COEF) {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            bC[it][q] = make_uint2(coef[q * cells + ga], coef[q * cells + ga + 32]);
                    }
                }
            }
        }
        cp_async_wait_all();  // plane s+1, copied during the previous step
        __syncthreads();
        if (s + 2 <= z0 + NZ + 1) issue(s + 2);  // its slot held plane s-3, no longer read
        // ---- red update of plane s on the tile + 1 halo (all inputs old) ----
        {
            const float* up = su + uslot(s - 1);
            const float* uc = su + uslot(s);
            const float* un = su + uslot(s + 1);
            const float* bp = sb + uslot(s - 1);
            const float* bc = sb + uslot(s);
            const float* bn = sb + uslot(s + 1);
            float* rc = sr + rslot(s);
#pragma unroll
            for (int it = 0; it < G::NRU; ++it) {
                if (r_rowA[it] < 0) continue;
                const int pa = (r_rowA[it] + s) & 1, pbb = (r_rowB[it] + s) & 1;
                const int ca = r_cuA[it] + pa, cb = r_cuB[it] + pbb;
                const Stencil2 a = stencil2(up, uc, un, ca, cb);
                const float2 kc = f2mul(f2(kap), rW[it]);
                const float2 iw = kmask ? make_float2(rW[it].x > 0.f ? __frcp_rn(rW[it].x) : 1.f,
                                                      rW[it].y > 0.f ? __frcp_rn(rW[it].y) : 1.f)
                                        : f2(1.f);
                Local2 o;
                if (COEF) {
                    o = local_eval2_cf(a, unpack_bg_coef(rC[it][0].x, rC[it][1].x, rC[it][2].x),
                                       unpack_bg_coef(rC[it][0].y, rC[it][1].y, rC[it][2].y), ih2, nu, kc,
                                       f2fma(f2(fscale), rF[it], f2(lam)), f2mul(f2(lsat), iw), rG[it]);
                } else {
                    Stencil2 b;
                    if (BG) b = stencil2(bp, bc, bn, ca, cb);
                    o = local_eval2<BG, GAP>(a, b, ih2, nu, kc, f2fma(f2(fscale), rF[it], f2(lam)),
                                             f2mul(f2(lsat), iw), rG[it]);
                }
                const float2 e = update2(o, kc, iw);
                rc[r_crA[it] + pa] = a.c0.x + e.x;
                rc[r_crB[it] + pbb] = a.c0.y + e.y;
            }
        }
        __syncthreads();
        // ---- black update of plane pb = s - 1 on the tile, then store the plane ----
        if (black) {
            const float* up = su + uslot(pb - 1);
            const float* uc = su + uslot(pb);
            const float* un = su + uslot(pb + 1);
            const float* bp = sb + uslot(pb - 1);
            const float* bc = sb + uslot(pb);
            const float* bn = sb + uslot(pb + 1);
            const float* rp = sr + rslot(pb - 1);
            const float* rc = sr + rslot(pb);
            const float* rn = sr + rslot(pb + 1);
            float* Vp = V + (size_t)pb * plane;  // pb is inside [0, n): no wrap
#pragma unroll
            for (int it = 0; it < G::NBU; ++it) {
                const int y = b_row[it];
                if (y < 0) continue;
                const int par = (y + pb) & 1;  // 1: the first cell of each x pair is black
                const int xbk = 2 * bkq + (par ? 0 : 1), xrd = 2 * bkq + par;
                // black cells: centre and edges from the old values, faces from the new red values
                const int ca = (y + 2) * WU + xbk + 2, cb = ca + 32;
                const int ra = (y + 1) * WR + xbk + 1, rb = ra + 32;
                Stencil2 a;
                a.c0 = make_float2(uc[ca], uc[cb]);
                a.ax = f2add(make_float2(rc[ra + 1], rc[rb + 1]), make_float2(rc[ra - 1], rc[rb - 1]));
                a.ay = f2add(make_float2(rc[ra + WR], rc[rb + WR]), make_float2(rc[ra - WR], rc[rb - WR]));
                a.az = f2add(make_float2(rn[ra], rn[rb]), make_float2(rp[ra], rp[rb]));
                a.exy = f2sub(f2sub(make_float2(uc[ca + 1 + WU], uc[cb + 1 + WU]), make_float2(uc[ca + 1 - WU], uc[cb + 1 - WU])),
                              f2sub(make_float2(uc[ca - 1 + WU], uc[cb - 1 + WU]), make_float2(uc[ca - 1 - WU], uc[cb - 1 - WU])));
                a.exz = f2sub(f2sub(make_float2(un[ca + 1], un[cb + 1]), make_float2(up[ca + 1], up[cb + 1])),
                              f2sub(make_float2(un[ca - 1], un[cb - 1]), make_float2(up[ca - 1], up[cb - 1])));
                a.eyz = f2sub(f2sub(make_float2(un[ca + WU], un[cb + WU]), make_float2(up[ca + WU], up[cb + WU])),
                              f2sub(make_float2(un[ca - WU], un[cb - WU]), make_float2(up[ca - WU], up[cb - WU])));
                const float2 kc = f2mul(f2(kap), bW[it]);
                const float2 iw = kmask ? make_float2(bW[it].x > 0.f ? __frcp_rn(bW[it].x) : 1.f,
                                                      bW[it].y > 0.f ? __frcp_rn(bW[it].y) : 1.f)
                                        : f2(1.f);
                Local2 o;
                if (COEF) {
                    o = local_eval2_cf(a, unpack_bg_coef(bC[it][0].x, bC[it][1].x, bC[it][2].x),
                                       unpack_bg_coef(bC[it][0].y, bC[it][1].y, bC[it][2].y), ih2, nu, kc,
                                       f2fma(f2(fscale), bF[it], f2(lam)), f2mul(f2(lsat), iw), bG[it]);
                } else {
                    Stencil2 b;
                    if (BG) b = stencil2(bp, bc, bn, ca, cb);
                    o = local_eval2<BG, GAP>(a, b, ih2, nu, kc, f2fma(f2(fscale), bF[it], f2(lam)),
                                             f2mul(f2(lsat), iw), bG[it]);
                }
                const float2 e = update2(o, kc, iw);
                const float vba = a.c0.x + e.x, vbb = a.c0.y + e.y;
                const int rr = (y + 1) * WR + xrd + 1;
                const float vra = rc[rr], vrb = rc[rr + 32];
                float* row = Vp + (y0 + y) * n + x0 + 2 * bkq;
                *reinterpret_cast<float2*>(row) = par ? make_float2(vba, vra) : make_float2(vra, vba);
                *reinterpret_cast<float2*>(row + 32) = par ? make_float2(vbb, vrb) : make_float2(vrb, vbb);
            }
        }
    }
}

}  // namespace pmeft
