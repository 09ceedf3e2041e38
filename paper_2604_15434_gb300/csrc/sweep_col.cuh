// sweep_col.cuh -- the finest-level FP32 red-black sweep with column-resident stencils.
//
// Same update and the same snapshot semantics as k_sweep_pair with background coefficients
// (COEF): red cells from the old field, black cells from the old black values (centre and
// the 12 same-colour edge neighbours) and the new red values (the 6 faces).  What changes is
// where the stencil comes from.  A thread owns the two columns (x, x+1), x even, of one row y
// of a 64 x TY tile and marches in z.  Once per plane it reads that plane's old values around
// its columns (three rows, 9 shared-memory loads) and keeps, per column, the pieces every later
// stencil needs in registers: the value, the x- and y-differences Dx = u(x+1) - u(x-1) and
// Dy = u(y+1) - u(y-1), the in-plane cross difference exy = Dx(y+1) - Dx(y-1) and, for the
// column that is red on that plane, the old face sums.  The z-faces and the xz / yz cross
// differences of a cell at plane z are then register arithmetic on the pieces of planes z - 1
// and z + 1 (exz = Dx(z+1) - Dx(z-1)), so a cell costs a handful of shared-memory accesses
// instead of 19.
//
// At step s a thread updates the red cell of plane s of one column (c, the column with
// x + y + s even) and the black cell of plane s - 2 of the other (c'), the two as the lanes of
// paired FP32 instructions (FADD2 / FMUL2 / FFMA2).  The black cell two planes back depends
// only on red values of planes s - 1 and s - 3 (its z-faces) and s - 2 (its in-plane faces),
// all final by then, so the two lanes are independent.  Its in-plane faces come from the red
// values of the neighbouring threads, written to a three-slot ring of new-red planes.
//
// Halo: black cells on the tile edge need red values just outside it, so the red update also
// covers the rows y = -1 and y = TY (two warps running the column code, red only) and the
// columns x = -1 and x = 64 (one lane per row on the x-halo warps, which read their 19-point
// stencils from the ring of old planes).
//
// Data movement: every input plane (old correction, right-hand side, floored gap, three
// coefficient words) arrives by 16-byte asynchronous copies, issued three planes ahead into
// shared-memory rings, so each value is read from DRAM once per sweep (halos from L2).
// Output: after the black update of plane s - 2, both columns of that plane are final and are
// stored with one 8-byte store per thread.
#pragma once

#include <type_traits>

#include "sweep_pair.cuh"

namespace pmeft {

__device__ __forceinline__ void cp_async16(unsigned smem_addr, const void* gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_2() { asm volatile("cp.async.wait_group 2;\n" ::: "memory"); }

template <int TY>
struct ColGeom {
    static constexpr int TX = 64;
    static constexpr int WS = 72;            // shared row stride (floats): x in [-4, 68)
    static constexpr int XO = 4;             // shared column of x = 0
    static constexpr int HE = TY + 4;        // old-value rows: y in [-2, TY + 2)
    static constexpr int HF = TY + 2;        // field and new-red rows: y in [-1, TY + 1)
    static constexpr int PE = WS * HE, PF = WS * HF;
    static constexpr int NSE = 5;            // old-value slots: planes s-1 .. s+3
    static constexpr int NSF = 4;            // field slots: planes s .. s+3
    static constexpr int NSR = 3;            // new-red slots: planes s-2 .. s
    static constexpr int NFLD = 5;           // right-hand side, gap, three coefficient words
    static constexpr int NXH = 2 * HF;       // x-halo lanes: x = -1 and x = 64 on every field row
    static constexpr int WXH = (NXH + 31) / 32;
    static constexpr int NW = TY + 2 + WXH;  // row warps, the two halo rows, x-halo warps
    static constexpr int NT = 32 * NW;
    static constexpr int CH_E = 18 * HE;     // 16-byte chunks of an old-value plane region
    static constexpr int CH_F = 18 * HF;     // ... of one field plane region
    static_assert(CH_E <= NT && CH_F <= NT, "one chunk of each array per thread");
};

template <int TY>
constexpr size_t col_smem_bytes()
{
    using G = ColGeom<TY>;
    return sizeof(float) * ((size_t)G::NSE * G::PE + (size_t)G::NSF * G::NFLD * G::PF + (size_t)G::NSR * G::PF);
}

template <int C>
__device__ __forceinline__ float cmp(float2 v)
{
    return C ? v.y : v.x;
}

// The per-column pieces a thread keeps for its two columns (.x column x, .y column x + 1).
// Index 0 is the oldest plane kept.
struct ColState {
    float2 U[4];       // old values, planes s-2 .. s+1
    float2 DX[5], DY[5];  // x- and y-differences, planes s-3 .. s+1
    float2 EXY[4];     // in-plane cross differences, planes s-2 .. s+1
    float AXR[2], AYR[2];  // old face sums of the column red on the plane, planes s, s+1
    float2 RL, RP;     // per column: its latest new red value and the one before
    float BF[2][5];    // fields of the black cells of planes s-2, s-1 (the column black there)
};

// The 8-term update of one cell (both colours), without a screening mask: pick_update of
// sweep_pair.cuh, or the linear step where the screening term is off.
__device__ __forceinline__ float col_update1(const Local<float>& o, float kap, float sp, float Df, float h2over6,
                                             float inv2P)
{
    if (kap == 0.f) return __fdividef(-o.G, o.Ep);
    return pick_update(o.G, o.Ep, o.P, o.D, o.g, sp, Df, h2over6, inv2P);
}

template <int TY>
__global__ void __launch_bounds__(ColGeom<TY>::NT, TY <= 8 ? 2 : 1)
    k_sweep_col(const float* __restrict__ U, float* __restrict__ V, const float* __restrict__ F, float fscale,
                float lam, const float* __restrict__ gap, int n, int NZ, float ih2, float nu, float kap, float sp,
                float Df, float lsat, const float* __restrict__ lamp, const uint32_t* __restrict__ coef)
{
    using G = ColGeom<TY>;
    constexpr int WS = G::WS, XO = G::XO;
    if (lamp) lam += *lamp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* se = reinterpret_cast<float*>(smem_raw);          // [NSE][HE][WS] old values
    float* sf = se + G::NSE * G::PE;                          // [NFLD][NSF][HF][WS] fields
    float* sr = sf + G::NFLD * G::NSF * G::PF;                // [NSR][HF][WS] new red values
    const unsigned se_s = (unsigned)__cvta_generic_to_shared(se);
    const unsigned sf_s = (unsigned)__cvta_generic_to_shared(sf);
    const int m = n - 1;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const size_t plane = (size_t)n * n, cells = plane * (size_t)n;
    auto eslot = [&](int p) { return ((p - z0 + 20) % G::NSE) * G::PE; };
    auto fslot = [&](int p) { return ((p - z0 + 20) % G::NSF) * G::PF; };
    auto rslot = [&](int p) { return ((p - z0 + 21) % G::NSR) * G::PF; };

    // this thread's 16-byte chunk of each plane region (the same in-plane offsets on every plane)
    int goE = -1, soE = 0, goF = -1, soF = 0;
    if (t < G::CH_E) {
        const int row = t / 18, cx = t - row * 18;
        goE = ((y0 - 2 + row) & m) * n + ((x0 - 4 + 4 * cx) & m);
        soE = row * WS + 4 * cx;
    }
    if (t < G::CH_F) {
        const int row = t / 18, cx = t - row * 18;
        goF = ((y0 - 1 + row) & m) * n + ((x0 - 4 + 4 * cx) & m);
        soF = row * WS + 4 * cx;
    }
    auto issue = [&](int p) {
        const size_t po = (size_t)(p & m) * plane;
        if (goE >= 0) cp_async16(se_s + 4u * (unsigned)(eslot(p) + soE), U + po + goE);
        if (goF >= 0) {
            const unsigned d = sf_s + 4u * (unsigned)(fslot(p) + soF);
            constexpr unsigned fstride = 4u * G::NSF * G::PF;
            cp_async16(d, F + po + goF);
            cp_async16(d + fstride, gap + po + goF);
            cp_async16(d + 2 * fstride, coef + po + goF);
            cp_async16(d + 3 * fstride, coef + cells + po + goF);
            cp_async16(d + 4 * fstride, coef + 2 * cells + po + goF);
        }
        cp_async_commit_group();
    };
    auto fld = [&](int f, int p) { return sf + f * (G::NSF * G::PF) + fslot(p); };

    const float h2over6 = 1.f / (6.f * ih2), inv2P = kap != 0.f ? 1.f / (-48.f * kap * ih2 * ih2) : 0.f;

    const bool xhalo = warp >= TY + 2;
    const int zlast = z0 + NZ;  // red planes z0-1 .. z0+NZ, black planes z0 .. z0+NZ-1

    // planes z0-2 .. z0+1 before the first step; step s waits for s+1 and issues s+3
    issue(z0 - 2);
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);

    if (!xhalo) {
        // ---------------------------------------------------------------- column warps
        const int y = warp < TY ? warp : (warp == TY ? -1 : TY);
        const bool interior = warp < TY;
        const int q = lane;              // columns 2q, 2q + 1
        const int yg = y0 + y;
        const int cE = (y + 2) * WS + XO + 2 * q;   // old-value region, row y, column 2q
        const int cF = (y + 1) * WS + XO + 2 * q;   // field / red region, row y, column 2q
        ColState S;
        // the pieces of one old plane p, for both columns
        auto derive = [&](int p, float2& u, float2& dx, float2& dy, float2& exy, float2& ax, float2& ay) {
            const float* e = se + eslot(p) + cE;
            const float2 um = *reinterpret_cast<const float2*>(e - WS);
            const float2 uc = *reinterpret_cast<const float2*>(e);
            const float2 up = *reinterpret_cast<const float2*>(e + WS);
            const float lmm = e[-WS - 1], lmc = e[-1], lmp = e[WS - 1];
            const float rpm = e[-WS + 2], rpc = e[2], rpp = e[WS + 2];
            u = uc;
            dx = f2sub(make_float2(uc.y, rpc), make_float2(lmc, uc.x));
            dy = f2sub(up, um);
            const float2 dxp = f2sub(make_float2(up.y, rpp), make_float2(lmp, up.x));
            const float2 dxm = f2sub(make_float2(um.y, rpm), make_float2(lmm, um.x));
            exy = f2sub(dxp, dxm);
            ax = f2add(make_float2(uc.y, rpc), make_float2(lmc, uc.x));
            ay = f2add(up, um);
        };
        // prologue: the pieces of planes z0-2 and z0-1, placed as a step before s = z0-1 leaves
        // them (U[2..3], DX/DY[3..4], EXY[2..3], AXR/AYR[1] for the red column of z0-1)
        cp_async_wait_2();
        __syncthreads();
        {
            float2 ax, ay;
            derive(z0 - 2, S.U[2], S.DX[3], S.DY[3], S.EXY[2], ax, ay);
            derive(z0 - 1, S.U[3], S.DX[4], S.DY[4], S.EXY[3], ax, ay);
            S.AXR[1] = ((yg + z0 - 1) & 1) ? ax.y : ax.x;
            S.AYR[1] = ((yg + z0 - 1) & 1) ? ay.y : ay.x;
            S.U[0] = S.U[1] = S.U[2];
            S.DX[0] = S.DX[1] = S.DX[2] = S.DX[3];
            S.DY[0] = S.DY[1] = S.DY[2] = S.DY[3];
            S.EXY[0] = S.EXY[1] = S.EXY[2];
            S.AXR[0] = S.AXR[1];
            S.AYR[0] = S.AYR[1];
            S.RL = S.RP = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int f = 0; f < 5; ++f) S.BF[a][f] = 0.f;
        }
        // The step body for the red column C of plane s (C = 0: column x, 1: x + 1).
        auto step = [&](auto Ct, int s) {
            constexpr int C = decltype(Ct)::value, Cb = 1 - C;
            // wait for plane s+1 (s+2 may still be in flight), then start plane s+3
            cp_async_wait_1();
            __syncthreads();
            if (s + 3 <= zlast + 1) issue(s + 3);
            else cp_async_commit_group();  // keep the group count in step
            // shift: index of plane s+1 becomes free
            S.U[0] = S.U[1]; S.U[1] = S.U[2]; S.U[2] = S.U[3];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                S.DX[k] = S.DX[k + 1];
                S.DY[k] = S.DY[k + 1];
            }
            S.EXY[0] = S.EXY[1]; S.EXY[1] = S.EXY[2]; S.EXY[2] = S.EXY[3];
            S.AXR[0] = S.AXR[1];
            S.AYR[0] = S.AYR[1];
            // now U[0..2] = s-2 .. s, DX[0..3] = s-3 .. s, EXY[0..2] = s-2 .. s; derive s+1
            {
                float2 ax, ay;
                derive(s + 1, S.U[3], S.DX[4], S.DY[4], S.EXY[3], ax, ay);
                S.AXR[1] = cmp<Cb>(ax);  // the column red on plane s+1 is the other one
                S.AYR[1] = cmp<Cb>(ay);
            }
            const bool red_ok = s <= zlast;
            const bool blk_ok = interior && s - 2 >= z0 && s - 2 < zlast;
            // fields of plane s: the red cell's now, the black cell's kept for step s+2
            // (BF[0] holds plane s-2's black cell, BF[1] plane s-1's)
            float fr[5], bf[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const float2 v = *reinterpret_cast<const float2*>(fld(f, s) + cF);
                fr[f] = cmp<C>(v);
                bf[f] = S.BF[0][f];
                S.BF[0][f] = S.BF[1][f];
                S.BF[1][f] = cmp<Cb>(v);
            }
            // black cell (Cb, s-2): its in-plane faces from the new red values of plane s-2
            float bax = 0.f, bay = 0.f;
            if (blk_ok) {
                const float* r = sr + rslot(s - 2) + cF;
                const float rout = Cb ? r[2] : r[-1];  // the neighbour outside the pair
                bax = cmp<C>(S.RL) + rout;               // the pair's own red column, plane s-2
                bay = r[Cb + WS] + r[Cb - WS];
            }
            Stencil2 st;
            st.c0 = make_float2(cmp<C>(S.U[2]), cmp<Cb>(S.U[0]));
            st.ax = make_float2(S.AXR[0], bax);
            st.ay = make_float2(S.AYR[0], bay);
            st.az = make_float2(cmp<C>(S.U[3]) + cmp<C>(S.U[1]), cmp<Cb>(S.RL) + cmp<Cb>(S.RP));
            st.exy = make_float2(cmp<C>(S.EXY[2]), cmp<Cb>(S.EXY[0]));
            st.exz = make_float2(cmp<C>(S.DX[4]) - cmp<C>(S.DX[2]), cmp<Cb>(S.DX[2]) - cmp<Cb>(S.DX[0]));
            st.eyz = make_float2(cmp<C>(S.DY[4]) - cmp<C>(S.DY[2]), cmp<Cb>(S.DY[2]) - cmp<Cb>(S.DY[0]));
            const BgCoef ca = unpack_bg_coef(__float_as_uint(fr[2]), __float_as_uint(fr[3]), __float_as_uint(fr[4]));
            const BgCoef cb = unpack_bg_coef(__float_as_uint(bf[2]), __float_as_uint(bf[3]), __float_as_uint(bf[4]));
            const float2 kc = f2(kap);
            const Local2 o = local_eval2_cf(st, ca, cb, ih2, nu, kc, f2fma(f2(fscale), make_float2(fr[0], bf[0]), f2(lam)),
                                            f2(lsat), make_float2(fr[1], bf[1]));
            float er, eb;
            if (kap == 0.f) {
                er = __fdividef(-o.G.x, o.Ep.x);
                eb = __fdividef(-o.G.y, o.Ep.y);
            } else {
                er = pick_update(o.G.x, o.Ep.x, o.P.x, o.D.x, o.g.x, sp, Df, h2over6, inv2P);
                eb = pick_update(o.G.y, o.Ep.y, o.P.y, o.D.y, o.g.y, sp, Df, h2over6, inv2P);
            }
            const float rnew = st.c0.x + er;
            const float bnew = st.c0.y + eb;
            // plane s-2 is final for both columns: its red cell (column C) and the black one
            if (blk_ok) {
                const float2 out = C ? make_float2(bnew, S.RL.y) : make_float2(S.RL.x, bnew);
                *reinterpret_cast<float2*>(V + (size_t)(s - 2) * plane + (size_t)yg * n + x0 + 2 * q) = out;
            }
            if (red_ok) {
                sr[rslot(s) + cF + C] = rnew;
                if (C) {
                    S.RP.y = S.RL.y;
                    S.RL.y = rnew;
                } else {
                    S.RP.x = S.RL.x;
                    S.RL.x = rnew;
                }
            }
        };
        for (int s = z0 - 1; s <= zlast + 1; ++s) {
            if ((yg + s) & 1) step(std::integral_constant<int, 1>{}, s);
            else step(std::integral_constant<int, 0>{}, s);
        }
    } else {
        // ---------------------------------------------------------------- x-halo lanes
        const int idx = (warp - TY - 2) * 32 + lane;
        const bool active = idx < G::NXH;
        const int xh = idx < G::HF ? -1 : 64;
        const int y = (active ? idx % G::HF : 0) - 1;
        const int par = (x0 + xh + y0 + y) & 1;
        const int cE = (y + 2) * WS + XO + xh;
        const int cF = (y + 1) * WS + XO + xh;
        cp_async_wait_2();
        __syncthreads();
        for (int s = z0 - 1; s <= zlast + 1; ++s) {
            cp_async_wait_1();
            __syncthreads();
            if (s + 3 <= zlast + 1) issue(s + 3);
            else cp_async_commit_group();
            if (!active || s > zlast || ((par + s) & 1)) continue;
            const float* up = se + eslot(s - 1) + cE;
            const float* uc = se + eslot(s) + cE;
            const float* un = se + eslot(s + 1) + cE;
            Stencil<float> st;
            st.c0 = uc[0];
            st.ax = uc[1] + uc[-1];
            st.ay = uc[WS] + uc[-WS];
            st.az = un[0] + up[0];
            st.exy = (uc[1 + WS] - uc[1 - WS]) - (uc[-1 + WS] - uc[-1 - WS]);
            st.exz = (un[1] - up[1]) - (un[-1] - up[-1]);
            st.eyz = (un[WS] - up[WS]) - (un[-WS] - up[-WS]);
            const float rhs = fscale * fld(0, s)[cF] + lam;
            const BgCoef cf = unpack_bg_coef(__float_as_uint(fld(2, s)[cF]), __float_as_uint(fld(3, s)[cF]),
                                             __float_as_uint(fld(4, s)[cF]));
            const Local<float> o = local_eval_cf(st, cf, ih2, nu, kap, rhs, lsat, fld(1, s)[cF]);
            sr[rslot(s) + cF] = st.c0 + col_update1(o, kap, sp, Df, h2over6, inv2P);
        }
    }
}

}  // namespace pmeft
