// sweep_fused.cuh -- one full red-black sweep in a single pass over memory (FP32 levels).
//
// Same arithmetic and the same snapshot semantics as two k_half_sweep launches: red cells
// are updated from the old field; black cells from the old black values (centre and the 12
// same-colour edge neighbours) and the new red values (the 6 faces).  A thread block owns
// a TX x TY tile of (x, y) and marches along z through a chunk of NZ planes.  Shared
// memory holds a ring of old planes and of the background (tile + 2-cell halo) and a ring
// of 3 planes of new red values (tile + 1-cell halo).  At step s it computes the red update
// of plane s on the tile + 1 halo, then the black update of plane s-1 on the tile, and
// writes the whole of plane s-1 (red and black) with coalesced paired stores, while plane
// s+2 is being copied in.  Each input is read from DRAM once per sweep; the halo re-reads
// come from L2.
#pragma once

#include "internal.cuh"

namespace pmeft {

template <int TX, int TY>
struct FusedGeom {
    static constexpr int WU = TX + 4, HU = TY + 4;  // old-value / background region
    static constexpr int WR = TX + 2, HR = TY + 2;  // red-update region
    static constexpr int PU = WU * HU, PR = WR * HR;
    static constexpr int NS = 5;                    // ring slots of old planes: s-2 .. s+2
};

template <typename T, int TX, int TY, bool BG, bool GAP>
constexpr size_t fused_smem_bytes()
{
    using G = FusedGeom<TX, TY>;
    return sizeof(T) * ((size_t)G::NS * G::PU * (BG ? 2 : 1) + (size_t)3 * G::PR);
}

__device__ __forceinline__ void cp_async4(unsigned smem_addr, const void* gmem)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Data movement: the old planes (and the background) arrive through a 5-slot ring filled
// by asynchronous copies one plane ahead, so the copy of plane s+2 overlaps the updates of
// step s; the right-hand side, gap and mask values of a step's cells are loaded into
// registers before the step's barrier.  Every per-cell index is an int32 offset computed
// once per thread (n^3 <= 2^30); a step adds only the plane bases and the colour parity.
template <typename T, int TX, int TY, bool BG, bool GAP>
__global__ void __launch_bounds__(256) k_sweep_fused(const T* __restrict__ U, T* __restrict__ V,
                                                     const T* __restrict__ F, T fscale, T lam,
                                                     const uint8_t* __restrict__ kmask, const T* __restrict__ bg,
                                                     const T* __restrict__ gap, int n, int NZ, T ih2, T nu, T kap,
                                                     T sp, T Df, T lsat, const T* __restrict__ lamp)
{
    static_assert(sizeof(T) == 4, "the single-pass sweep is the FP32 smoother");
    static_assert(TX % 32 == 0 && TY % 2 == 0, "tile");
    if (lamp) lam += *lamp;
    using G = FusedGeom<TX, TY>;
    constexpr int NS = G::NS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);            // [NS][HU][WU] old values
    T* sb = su + NS * G::PU;                           // [NS][HU][WU] background (BG)
    T* sr = sb + (BG ? NS * G::PU : 0);                // [3][HR][WR] new red values
    const unsigned su_s = (unsigned)__cvta_generic_to_shared(su);
    const unsigned sb_s = (unsigned)__cvta_generic_to_shared(sb);
    const int m = n - 1;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x;
    const size_t plane = (size_t)n * n;
    // ring slots from (plane - z0 + 10) and (plane - z0 + 9), never negative here
    auto uslot = [&](int p) { return ((p - z0 + 10) % NS) * G::PU; };
    auto rslot = [&](int p) { return ((p - z0 + 9) % 3) * G::PR; };

    // this thread's share of a plane copy: the same (x, y) offsets (with the periodic
    // wrap) on every plane
    constexpr int KU = (G::PU + 255) / 256;
    int offu[KU];
#pragma unroll
    for (int k = 0; k < KU; ++k) {
        const int q = t + k * 256;
        const int yy = q / G::WU, xx = q - yy * G::WU;
        offu[k] = q < G::PU ? (((y0 - 2 + yy) & m) * n + ((x0 - 2 + xx) & m)) : -1;
    }
    auto issue = [&](int p) {
        const T* Up = U + (size_t)(p & m) * plane;
        const T* Bp = bg + (size_t)(p & m) * plane;
        const int so = uslot(p);
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            if (offu[k] < 0) continue;
            const unsigned d = 4u * (unsigned)(so + t + k * 256);
            cp_async4(su_s + d, Up + offu[k]);
            if (BG) cp_async4(sb_s + d, Bp + offu[k]);
        }
        cp_async_commit_group();
    };

    // Work units.  Same-colour cells of one row sit two words apart, so a warp reading 32
    // of them from one row would hit every bank twice; each warp instead takes 16 cells
    // from each of two adjacent rows (opposite colour parity, even widths), which fall on
    // the even and the odd banks.
    const int lane = t & 31, warp = t >> 5;
    const int half = lane >> 4, hl = lane & 15;
    // red cells of the tile + 1 halo: per_row per row, 16-cell chunks, then the ragged rest
    constexpr int per_row = G::WR / 2;
    constexpr int chunks = per_row / 16;
    constexpr int rest = per_row - 16 * chunks;
    constexpr int units = ((G::HR + 1) / 2) * chunks;
    constexpr int rest_units = (rest * G::HR + 31) / 32;
    constexpr int NRU = (units + rest_units + 7) / 8;
    int r_row[NRU], r_cu[NRU], r_cr[NRU], r_g0[NRU], r_g1[NRU];
#pragma unroll
    for (int it = 0; it < NRU; ++it) {
        const int wu = warp + 8 * it;
        int yr = G::HR, k = per_row;
        if (wu < units) {
            const int rp2 = wu / chunks, ch = wu - rp2 * chunks;
            yr = 2 * rp2 + half;
            k = ch * 16 + hl;
        } else if (rest > 0 && wu < units + rest_units) {
            const int q = (wu - units) * 32 + lane;
            yr = q / (rest > 0 ? rest : 1);
            k = 16 * chunks + q - yr * rest;
        }
        const bool ok = yr < G::HR && k < per_row;
        r_row[it] = ok ? yr : -1;
        r_cu[it] = (yr + 1) * G::WU + 2 * k + 1;   // + colour parity
        r_cr[it] = yr * G::WR + 2 * k;             // + colour parity
        const int gy = ((y0 - 1 + yr) & m) * n;
        r_g0[it] = gy + ((x0 - 1 + 2 * k) & m);
        r_g1[it] = gy + ((x0 + 2 * k) & m);
    }
    // black cells of the tile, one per (x, x+1) pair
    constexpr int pairs = TX / 2;
    constexpr int bchunks = (pairs + 15) / 16;
    constexpr int bunits = ((TY + 1) / 2) * bchunks;
    constexpr int NBU = (bunits + 7) / 8;
    int b_row[NBU], b_x2[NBU];
#pragma unroll
    for (int it = 0; it < NBU; ++it) {
        const int wu = warp + 8 * it;
        const int rp2 = wu / bchunks, ch = wu - rp2 * bchunks;
        const int y = 2 * rp2 + half, kq = ch * 16 + hl;
        const bool ok = wu < bunits && y < TY && kq < pairs;
        b_row[it] = ok ? y : -1;
        b_x2[it] = 2 * kq;
    }

    const T h2over6 = T(1) / (T(6) * ih2), inv2P = kap != T(0) ? T(1) / (T(-48) * kap * ih2 * ih2) : T(0);
    auto stencil_u = [&](const T* rp, const T* rc, const T* rn, int c) {
        Stencil<T> s;
        s.c0 = rc[c];
        s.ax = rc[c + 1] + rc[c - 1];
        s.ay = rc[c + G::WU] + rc[c - G::WU];
        s.az = rn[c] + rp[c];
        s.exy = rc[c + 1 + G::WU] - rc[c + 1 - G::WU] - rc[c - 1 + G::WU] + rc[c - 1 - G::WU];
        s.exz = rn[c + 1] - rp[c + 1] - rn[c - 1] + rp[c - 1];
        s.eyz = rn[c + G::WU] - rp[c + G::WU] - rn[c - G::WU] + rp[c - G::WU];
        return s;
    };

    issue(z0 - 2);
    issue(z0 - 1);
    issue(z0);
    for (int s = z0 - 1; s <= z0 + NZ; ++s) {
        const int pb = s - 1;
        const bool black = pb >= z0;
        // this step's right-hand side, gap and mask values, before the barrier
        T rF[NRU], rG[NRU], bF[NBU], bG[NBU];
        T rW[NRU], bW[NBU];  // screening weights (1 without a mask)
        {
            const size_t os = (size_t)(s & m) * plane, ob = (size_t)(pb & m) * plane;
#pragma unroll
            for (int it = 0; it < NRU; ++it) {
                rF[it] = T(0);
                rG[it] = T(0);
                rW[it] = T(1);
                if (r_row[it] >= 0) {
                    const size_t g = os + (size_t)(((r_row[it] + s) & 1) ? r_g1[it] : r_g0[it]);
                    rF[it] = F[g];
                    if (GAP) rG[it] = gap[g];
                    if (kmask) rW[it] = screen_w<T>(kmask, g);
                }
            }
#pragma unroll
            for (int it = 0; it < NBU; ++it) {
                const int y = b_row[it];
                bF[it] = T(0);
                bG[it] = T(0);
                bW[it] = T(1);
                if (black && y >= 0) {
                    const size_t gb = ob + (size_t)((y0 + y) * n + x0 + b_x2[it] + (((y + pb) & 1) ? 0 : 1));
                    bF[it] = F[gb];
                    if (GAP) bG[it] = gap[gb];
                    if (kmask) bW[it] = screen_w<T>(kmask, gb);
                }
            }
        }
        cp_async_wait_all();  // plane s+1, copied during the previous step
        __syncthreads();
        if (s + 2 <= z0 + NZ + 1) issue(s + 2);  // its slot held plane s-3, no longer read
        // ---- red update of plane s on the tile + 1 halo (all inputs old) ----
        {
            const T* up = su + uslot(s - 1);
            const T* uc = su + uslot(s);
            const T* un = su + uslot(s + 1);
            const T* bp = sb + uslot(s - 1);
            const T* bc = sb + uslot(s);
            const T* bn = sb + uslot(s + 1);
            T* rc = sr + rslot(s);
#pragma unroll
            for (int it = 0; it < NRU; ++it) {
                if (r_row[it] < 0) continue;
                const int par = (r_row[it] + s) & 1;
                const int cu = r_cu[it] + par;
                Stencil<T> a = stencil_u(up, uc, un, cu);
                Stencil<T> b;
                if (BG) b = stencil_u(bp, bc, bn, cu);
                const T kc = kap * rW[it];
                const T iw = (kmask && kc != T(0)) ? T(1) / rW[it] : T(1);  // L_sat and 1/(2P) scale as 1/kappa
                Local<T> o = local_eval<T, BG>(a, b, ih2, nu, kc, fscale * rF[it] + lam, lsat * iw, GAP, rG[it]);
                rc[r_cr[it] + par] = a.c0 + local_update_fast(o, sp, Df, h2over6, kc != T(0) ? inv2P * iw : T(0));
            }
        }
        __syncthreads();
        // ---- black update of plane pb = s - 1 on the tile, then store the plane ----
        if (black) {
            const T* up = su + uslot(pb - 1);
            const T* uc = su + uslot(pb);
            const T* un = su + uslot(pb + 1);
            const T* bp = sb + uslot(pb - 1);
            const T* bc = sb + uslot(pb);
            const T* bn = sb + uslot(pb + 1);
            const T* rp = sr + rslot(pb - 1);
            const T* rc = sr + rslot(pb);
            const T* rn = sr + rslot(pb + 1);
            T* Vp = V + (size_t)pb * plane;  // pb is inside [0, n): no wrap
#pragma unroll
            for (int it = 0; it < NBU; ++it) {
                const int y = b_row[it];
                if (y < 0) continue;
                const int x2 = b_x2[it];
                const int par = (y + pb) & 1;  // 1: the first cell of the pair is black
                const int xbk = x2 + (par ? 0 : 1), xrd = x2 + par;
                // black cell: centre and edges from the old values, faces from the new red values
                const int cu = (y + 2) * G::WU + xbk + 2, cr = (y + 1) * G::WR + xbk + 1;
                Stencil<T> a;
                a.c0 = uc[cu];
                a.ax = rc[cr + 1] + rc[cr - 1];
                a.ay = rc[cr + G::WR] + rc[cr - G::WR];
                a.az = rn[cr] + rp[cr];
                a.exy = uc[cu + 1 + G::WU] - uc[cu + 1 - G::WU] - uc[cu - 1 + G::WU] + uc[cu - 1 - G::WU];
                a.exz = un[cu + 1] - up[cu + 1] - un[cu - 1] + up[cu - 1];
                a.eyz = un[cu + G::WU] - up[cu + G::WU] - un[cu - G::WU] + up[cu - G::WU];
                Stencil<T> b;
                if (BG) b = stencil_u(bp, bc, bn, cu);
                const T kc = kap * bW[it];
                const T iw = (kmask && kc != T(0)) ? T(1) / bW[it] : T(1);
                Local<T> o = local_eval<T, BG>(a, b, ih2, nu, kc, fscale * bF[it] + lam, lsat * iw, GAP, bG[it]);
                const T vb = a.c0 + local_update_fast(o, sp, Df, h2over6, kc != T(0) ? inv2P * iw : T(0));
                const T vr = rc[(y + 1) * G::WR + xrd + 1];
                *reinterpret_cast<float2*>(Vp + (y0 + y) * n + x0 + x2) =
                    par ? make_float2(vb, vr) : make_float2(vr, vb);
            }
        }
    }
}

}  // namespace pmeft
