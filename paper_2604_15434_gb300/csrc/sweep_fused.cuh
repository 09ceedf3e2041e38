// sweep_fused.cuh -- one full red-black sweep in a single pass over memory (FP32 levels).
//
// Same arithmetic and the same snapshot semantics as two k_half_sweep launches: red cells
// are updated from the old field; black cells from the old black values (centre and the 12
// same-colour edge neighbours) and the new red values (the 6 faces).  A thread block owns
// a TX x TY tile of (x, y) and marches along z through a chunk of NZ planes, keeping in
// shared memory a ring of 4 old planes and of the background (tile + 2-cell halo) and a
// ring of 3 planes of new red values (tile + 1-cell halo); the right-hand side and the gap
// are read at the cell from global memory.  At step s it loads plane s+1, computes the
// red update of plane s on the
// tile + 1 halo, then the black update of plane s-1 on the tile, and writes the whole of
// plane s-1 (red and black) with coalesced paired stores.  Each input is read from DRAM
// once per sweep; the halo re-reads come from L2.
#pragma once

#include "internal.cuh"

namespace pmeft {

template <int TX, int TY>
struct FusedGeom {
    static constexpr int WU = TX + 4, HU = TY + 4;  // old-value / background region
    static constexpr int WR = TX + 2, HR = TY + 2;  // red-update region
    static constexpr int PU = WU * HU, PR = WR * HR;
};

template <typename T, int TX, int TY, bool BG, bool GAP>
constexpr size_t fused_smem_bytes()
{
    using G = FusedGeom<TX, TY>;
    return sizeof(T) * ((size_t)4 * G::PU * (BG ? 2 : 1) + (size_t)3 * G::PR);
}

template <typename T, int TX, int TY, bool BG, bool GAP>
__global__ void __launch_bounds__(256) k_sweep_fused(const T* __restrict__ U, T* __restrict__ V,
                                                     const T* __restrict__ F, T fscale, T lam,
                                                     const uint8_t* __restrict__ kmask, const T* __restrict__ bg,
                                                     const T* __restrict__ gap, int n, int NZ, T ih2, T nu, T kap,
                                                     T sp, T Df, T lsat, const T* __restrict__ lamp)
{
    if (lamp) lam += *lamp;
    using G = FusedGeom<TX, TY>;
    extern __shared__ unsigned char smem_raw[];
    T* su = reinterpret_cast<T*>(smem_raw);            // [4][HU][WU] old values
    T* sb = su + 4 * G::PU;                            // [4][HU][WU] background (BG)
    T* sr = sb + (BG ? 4 * G::PU : 0);                 // [3][HR][WR] new red values
    const int m = n - 1;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x, nt = blockDim.x;
    const size_t sn = (size_t)n;
    auto gidx = [&](int x, int y, int z) { return ((size_t)(z & m) * sn + (y & m)) * sn + (x & m); };
    // ring slots are taken from (plane - z0 + 8), which is never negative here
    auto uslot = [&](int p) { return ((p - z0 + 8) & 3) * G::PU; };
    auto rslot = [&](int p) { return ((p - z0 + 9) % 3) * G::PR; };

    // the (x, y) offsets of this thread's share of a plane load are the same on every
    // plane: compute them once (with the periodic wrap) and add the plane offset later
    constexpr int KU = (G::PU + 255) / 256;
    int offu[KU];
#pragma unroll
    for (int k = 0; k < KU; ++k) {
        const int q = t + k * 256;
        const int yy = q / G::WU, xx = q - yy * G::WU;
        offu[k] = q < G::PU ? (((y0 - 2 + yy) & m) * n + ((x0 - 2 + xx) & m)) : -1;
    }
    const size_t plane = (size_t)n * n;
    auto load_u = [&](int p) {
        T* du = su + uslot(p);
        T* db = sb + uslot(p);
        const T* Up = U + (size_t)(p & m) * plane;
        const T* Bp = bg + (size_t)(p & m) * plane;
#pragma unroll
        for (int k = 0; k < KU; ++k) {
            if (offu[k] < 0) continue;
            du[t + k * 256] = Up[offu[k]];
            if (BG) db[t + k * 256] = Bp[offu[k]];
        }
    };
    const T h2over6 = T(1) / (T(6) * ih2), inv2P = kap != T(0) ? T(1) / (T(-48) * kap * ih2 * ih2) : T(0);
    auto update = [&](const Local<T>& o, T kc) -> T {
        if constexpr (sizeof(T) == 4)
            return local_update_fast(o, sp, Df, h2over6, kc != T(0) ? inv2P : T(0));
        else
            return local_update(o, sp, Df, ih2);
    };
    // 19-point stencil of the U region around (xu, yu) of plane p, faces from `face`
    auto stencil_u = [&](const T* rp, const T* rc, const T* rn, int xu, int yu) {
        Stencil<T> s;
        const int c = yu * G::WU + xu;
        s.c0 = rc[c];
        s.ax = rc[c + 1] + rc[c - 1];
        s.ay = rc[c + G::WU] + rc[c - G::WU];
        s.az = rn[c] + rp[c];
        s.exy = rc[c + 1 + G::WU] - rc[c + 1 - G::WU] - rc[c - 1 + G::WU] + rc[c - 1 - G::WU];
        s.exz = rn[c + 1] - rp[c + 1] - rn[c - 1] + rp[c - 1];
        s.eyz = rn[c + G::WU] - rp[c + G::WU] - rn[c - G::WU] + rp[c - G::WU];
        return s;
    };

    // Same-colour cells of one row sit two words apart, so a warp reading 32 of them from
    // one row would hit every bank twice.  Each warp instead takes 16 cells from each of two
    // adjacent rows: the rows alternate colour parity and have even widths, so the two
    // halves fall on the even and the odd banks.
    const int lane = t & 31, warp = t >> 5, nwarps = nt >> 5;
    const int half = lane >> 4, hl = lane & 15;
    const T* F_ = F;
    auto rhs_at = [&](int gx, int gy, int p) { return fscale * F_[gidx(gx, gy, p)] + lam; };

    load_u(z0 - 2);
    load_u(z0 - 1);
    for (int s = z0 - 1; s <= z0 + NZ; ++s) {
        load_u(s + 1);
        __syncthreads();
        // ---- red update of plane s on the tile + 1 halo (all inputs old) ----
        {
            const T* up = su + uslot(s - 1);
            const T* uc = su + uslot(s);
            const T* un = su + uslot(s + 1);
            const T* bp = sb + uslot(s - 1);
            const T* bc = sb + uslot(s);
            const T* bn = sb + uslot(s + 1);
            T* rc = sr + rslot(s);
            constexpr int per_row = G::WR / 2;            // red cells per row of the region
            constexpr int chunks = per_row / 16;          // full 16-cell chunks per row
            constexpr int rest = per_row - 16 * chunks;   // cells left at the end of each row
            constexpr int units = ((G::HR + 1) / 2) * chunks;  // (row pair, chunk) work units
            constexpr int rest_units = (rest * G::HR + 31) / 32;  // leftover cells, 32 per unit
            for (int wu = warp; wu < units + rest_units; wu += nwarps) {
                int yr, k;
                if (wu < units) {
                    const int rp2 = wu / chunks, ch = wu - rp2 * chunks;
                    yr = 2 * rp2 + half;
                    k = ch * 16 + hl;
                } else {
                    const int q = (wu - units) * 32 + lane;  // q-th leftover cell
                    yr = rest > 0 ? q / rest : G::HR;
                    k = 16 * chunks + (rest > 0 ? q - yr * rest : 0);
                }
                if (yr >= G::HR || k >= per_row) continue;
                const int xr = 2 * k + ((x0 - 1 + y0 - 1 + yr + s) & 1);
                const int xu = xr + 1, yu = yr + 1;
                Stencil<T> a = stencil_u(up, uc, un, xu, yu);
                Stencil<T> b;
                if (BG) b = stencil_u(bp, bc, bn, xu, yu);
                const size_t g = gidx(x0 - 1 + xr, y0 - 1 + yr, s);
                const T kc = (kmask && kmask[g]) ? T(0) : kap;
                Local<T> o = local_eval<T, BG>(a, b, ih2, nu, kc, fscale * F_[g] + lam, lsat, GAP, GAP ? gap[g] : T(0));
                rc[yr * G::WR + xr] = a.c0 + update(o, kc);
            }
        }
        __syncthreads();
        // ---- black update of plane b = s - 1 on the tile, then store the plane ----
        const int pb = s - 1;
        if (pb >= z0) {
            const T* up = su + uslot(pb - 1);
            const T* uc = su + uslot(pb);
            const T* un = su + uslot(pb + 1);
            const T* bp = sb + uslot(pb - 1);
            const T* bc = sb + uslot(pb);
            const T* bn = sb + uslot(pb + 1);
            const T* rp = sr + rslot(pb - 1);
            const T* rc = sr + rslot(pb);
            const T* rn = sr + rslot(pb + 1);
            constexpr int pairs = TX / 2;                 // black cells (and pairs) per tile row
            constexpr int chunks = (pairs + 15) / 16;
            constexpr int units = ((TY + 1) / 2) * chunks;
            for (int wu = warp; wu < units; wu += nwarps) {
                const int rp2 = wu / chunks, ch = wu - rp2 * chunks;
                const int y = 2 * rp2 + half;
                const int kq = ch * 16 + hl;
                if (y >= TY || kq >= pairs) continue;
                const int x2 = 2 * kq;
                const int par = (x0 + x2 + y0 + y + pb) & 1;  // 1: the first cell of the pair is black
                const int xbk = x2 + (par ? 0 : 1), xrd = x2 + (par ? 1 : 0);
                // black cell: centre and edges from the old values, faces from the new red values
                const int xu = xbk + 2, yu = y + 2, xr = xbk + 1, yr = y + 1;
                const int cu = yu * G::WU + xu, cr = yr * G::WR + xr;
                Stencil<T> a;
                a.c0 = uc[cu];
                a.ax = rc[cr + 1] + rc[cr - 1];
                a.ay = rc[cr + G::WR] + rc[cr - G::WR];
                a.az = rn[cr] + rp[cr];
                a.exy = uc[cu + 1 + G::WU] - uc[cu + 1 - G::WU] - uc[cu - 1 + G::WU] + uc[cu - 1 - G::WU];
                a.exz = un[cu + 1] - up[cu + 1] - un[cu - 1] + up[cu - 1];
                a.eyz = un[cu + G::WU] - up[cu + G::WU] - un[cu - G::WU] + up[cu - G::WU];
                Stencil<T> b;
                if (BG) b = stencil_u(bp, bc, bn, xu, yu);
                const size_t gb = gidx(x0 + xbk, y0 + y, pb);
                const T kc = (kmask && kmask[gb]) ? T(0) : kap;
                Local<T> o = local_eval<T, BG>(a, b, ih2, nu, kc, fscale * F_[gb] + lam, lsat, GAP, GAP ? gap[gb] : T(0));
                const T vb = a.c0 + update(o, kc);
                const T vr = rc[yr * G::WR + xrd + 1];
                const size_t g0 = gidx(x0 + x2, y0 + y, pb);
                if (sizeof(T) == 4) {
                    float2 v2 = par ? make_float2((float)vb, (float)vr) : make_float2((float)vr, (float)vb);
                    *reinterpret_cast<float2*>(V + g0) = v2;
                } else {
                    V[g0] = par ? vb : vr;
                    V[g0 + 1] = par ? vr : vb;
                }
            }
        }
        __syncthreads();
    }
}

}  // namespace pmeft
