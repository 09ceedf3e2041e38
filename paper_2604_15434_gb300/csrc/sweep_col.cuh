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
//
// Bookkeeping: every ring (shared-memory slots and the per-column register history) has four
// entries indexed by the plane number mod 4, and the z loop is unrolled by four steps, so all
// ring positions are compile-time constants: no modulo arithmetic and no register shifting.
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
    static constexpr int NS = 4;             // slots of every ring (plane mod 4)
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
    return sizeof(float) * ((size_t)G::NS * G::PE + (size_t)G::NS * G::NFLD * G::PF + (size_t)G::NS * G::PF);
}

template <int C>
__device__ __forceinline__ float cmp(float2 v)
{
    return C ? v.y : v.x;
}

// The update of one cell without a screening mask: pick_update of sweep_pair.cuh, or the
// linear step where the screening term is off.
__device__ __forceinline__ float col_update1(const Local<float>& o, float kap, float sp, float Df, float h2over6,
                                             float inv2P)
{
    if (kap == 0.f) return div_ftz(-o.G, o.Ep);
    return pick_update(o.G, o.Ep, o.P, o.D, o.g, sp, Df, h2over6, inv2P);
}

// The kept pieces of one column pair (.x column x, .y column x + 1); the arrays are rings
// indexed by plane mod 4 (AXR / AYR / BF by plane mod 2).
struct ColState {
    float2 U[4], DX[4], DY[4], EXY[4];
    float AXR[2], AYR[2];  // old face sums of the column red on the plane
    float2 RL, RP;         // per column: its latest new red value and the one before
    float BF[2][5];        // fields of the black cell of the plane
};

// The pieces of one x-halo column (one cell per plane).
struct HaloState {
    float U[4], DX[4], DY[4];
    float AX[4], AY[4], EXY[4];
};

template <int TY>
__global__ void __launch_bounds__(ColGeom<TY>::NT, TY <= 8 ? 2 : 1)
    k_sweep_col(const float* __restrict__ U, float* __restrict__ V, const float* __restrict__ F, float fscale,
                float lam, const float* __restrict__ gap, int n, int NZ, float ih2, float nu, float kap, float sp,
                float Df, float lsat, const float* __restrict__ lamp, const uint32_t* __restrict__ coef)
{
    using G = ColGeom<TY>;
    constexpr int WS = G::WS, XO = G::XO, PE = G::PE, PF = G::PF;
    if (lamp) lam += *lamp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* se = reinterpret_cast<float*>(smem_raw);  // [4][HE][WS] old values
    float* sf = se + G::NS * PE;                      // [NFLD][4][HF][WS] fields
    float* sr = sf + G::NFLD * G::NS * PF;            // [4][HF][WS] new red values
    const unsigned se_s = (unsigned)__cvta_generic_to_shared(se);
    const unsigned sf_s = (unsigned)__cvta_generic_to_shared(sf);
    const int m = n - 1;
    const int x0 = blockIdx.x * G::TX, y0 = blockIdx.y * TY, z0 = blockIdx.z * NZ;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const size_t plane = (size_t)n * n, cells = plane * (size_t)n;
    const int zlast = z0 + NZ;  // red planes z0-1 .. z0+NZ, black planes z0 .. z0+NZ-1

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
    // copies of plane p into ring slot k = (p - z0 + 1) mod 4 (k given, compile-time at the call)
    auto issue = [&](int p, int k) {
        if (p <= zlast + 1) {
            const size_t po = (size_t)(p & m) * plane;
            if (goE >= 0) cp_async16(se_s + 4u * (unsigned)(k * PE + soE), U + po + goE);
            if (goF >= 0) {
                const unsigned d = sf_s + 4u * (unsigned)(k * PF + soF);
                constexpr unsigned fstride = 4u * G::NS * PF;
                const size_t o = po + (size_t)goF;
                cp_async16(d, F + o);
                cp_async16(d + fstride, gap + o);
                cp_async16(d + 2 * fstride, coef + o);
                cp_async16(d + 3 * fstride, coef + cells + o);
                cp_async16(d + 4 * fstride, coef + 2 * cells + o);
            }
        }
        cp_async_commit_group();  // an empty group past the last plane keeps the count in step
    };
    auto fld = [&](int f, int k) { return sf + (f * G::NS + k) * PF; };

    const float h2over6 = 1.f / (6.f * ih2), inv2P = kap != 0.f ? 1.f / (-48.f * kap * ih2 * ih2) : 0.f;
    const bool xhalo = warp >= TY + 2;

    // planes z0-2 .. z0+1 before the first step (slots 3, 0, 1, 2)
    issue(z0 - 2, 3);
    issue(z0 - 1, 0);
    issue(z0, 1);
    issue(z0 + 1, 2);
    const int nsteps = (NZ + 3 + 3) & ~3;  // steps s = z0-1 .. z0+NZ+1, rounded up to whole 4-step rounds

    if (!xhalo) {
        // ---------------------------------------------------------------- column warps
        const int y = warp < TY ? warp : (warp == TY ? -1 : TY);
        const bool interior = warp < TY;
        const int q = lane;  // columns 2q, 2q + 1
        const int yg = y0 + y;
        const int cE = (y + 2) * WS + XO + 2 * q;  // old-value region, row y, column 2q
        const int cF = (y + 1) * WS + XO + 2 * q;  // field / red region, row y, column 2q
        float* const Vrow = V + (size_t)(yg & m) * n + x0 + 2 * q;  // used by the interior rows only
        ColState S;
        // the pieces of old plane slot k, for both columns
        auto derive = [&](int k, float2& u, float2& dx, float2& dy, float2& exy, float2& ax, float2& ay) {
            const float* e = se + k * PE + cE;
            const float2 um = *reinterpret_cast<const float2*>(e - WS);
            const float2 uc = *reinterpret_cast<const float2*>(e);
            const float2 up = *reinterpret_cast<const float2*>(e + WS);
            const float lmm = e[-WS - 1], lmc = e[-1], lmp = e[WS - 1];
            const float rpm = e[-WS + 2], rpc = e[2], rpp = e[WS + 2];
            u = uc;
            dx = f2sub(make_float2(uc.y, rpc), make_float2(lmc, uc.x));
            dy = f2sub(up, um);
            exy = f2sub(f2sub(make_float2(up.y, rpp), make_float2(lmp, up.x)),
                        f2sub(make_float2(um.y, rpm), make_float2(lmm, um.x)));
            ax = f2add(make_float2(uc.y, rpc), make_float2(lmc, uc.x));
            ay = f2add(up, um);
        };
        cp_async_wait_2();
        __syncthreads();
        {
            float2 ax, ay;
            derive(3, S.U[3], S.DX[3], S.DY[3], S.EXY[3], ax, ay);  // plane z0-2
            derive(0, S.U[0], S.DX[0], S.DY[0], S.EXY[0], ax, ay);  // plane z0-1
            const bool c1 = ((yg + z0 - 1) & 1) != 0;                 // red column of plane z0-1
            S.AXR[0] = c1 ? ax.y : ax.x;                              // slot (z0-1 - z0 + 1) & 1 = 0
            S.AYR[0] = c1 ? ay.y : ay.x;
            S.U[2] = S.U[1] = S.U[3];
            S.DX[2] = S.DX[1] = S.DX[3];
            S.DY[2] = S.DY[1] = S.DY[3];
            S.EXY[2] = S.EXY[1] = S.EXY[3];
            S.AXR[1] = S.AXR[0];
            S.AYR[1] = S.AYR[0];
            S.RL = S.RP = make_float2(0.f, 0.f);
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int f = 0; f < 5; ++f) S.BF[a][f] = 0.f;
        }
        // step s, J = (s - z0 + 1) mod 4, C = the column red on plane s
        auto step = [&](auto Jt, auto Ct, int s) {
            constexpr int J = decltype(Jt)::value, C = decltype(Ct)::value, Cb = 1 - C;
            constexpr int K0 = J, K1 = (J + 1) & 3, Km1 = (J + 3) & 3, Km2 = (J + 2) & 3, Km3 = (J + 1) & 3;
            constexpr int A0 = J & 1, A1 = (J + 1) & 1;  // plane s and s+1 in the rings of two
            cp_async_wait_1();  // plane s+1 (s+2 may still be in flight)
            __syncthreads();
            issue(s + 3, Km1);  // into the slot of plane s-1, no longer read
            // the black cell's pieces of plane s-3 before its ring entry takes plane s+1
            const float dxm3 = cmp<Cb>(S.DX[Km3]), dym3 = cmp<Cb>(S.DY[Km3]);
            {
                float2 ax, ay;
                derive(K1, S.U[K1], S.DX[K1], S.DY[K1], S.EXY[K1], ax, ay);
                S.AXR[A1] = cmp<Cb>(ax);  // the column red on plane s+1 is the other one
                S.AYR[A1] = cmp<Cb>(ay);
            }
            const bool red_ok = s <= zlast;
            const bool blk_ok = interior && s - 2 >= z0 && s - 2 < zlast;
            // fields of plane s: the red cell's now, the black cell's kept for step s+2
            float fr[5], bf[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const float2 v = *reinterpret_cast<const float2*>(fld(f, K0) + cF);
                fr[f] = cmp<C>(v);
                bf[f] = S.BF[A0][f];  // plane s-2's black cell
                S.BF[A0][f] = cmp<Cb>(v);
            }
            // black cell (Cb, s-2): its in-plane faces from the new red values of plane s-2
            float bax = 0.f, bay = 0.f;
            if (interior) {
                const float* r = sr + Km2 * PF + cF;
                const float rout = Cb ? r[2] : r[-1];  // the neighbour outside the pair
                bax = cmp<C>(S.RL) + rout;              // the pair's own red column, plane s-2
                bay = r[Cb + WS] + r[Cb - WS];
            }
            Stencil2 st;
            st.c0 = make_float2(cmp<C>(S.U[K0]), cmp<Cb>(S.U[Km2]));
            st.ax = make_float2(S.AXR[A0], bax);
            st.ay = make_float2(S.AYR[A0], bay);
            st.az = make_float2(cmp<C>(S.U[K1]) + cmp<C>(S.U[Km1]), cmp<Cb>(S.RL) + cmp<Cb>(S.RP));
            st.exy = make_float2(cmp<C>(S.EXY[K0]), cmp<Cb>(S.EXY[Km2]));
            st.exz = make_float2(cmp<C>(S.DX[K1]) - cmp<C>(S.DX[Km1]), cmp<Cb>(S.DX[Km1]) - dxm3);
            st.eyz = make_float2(cmp<C>(S.DY[K1]) - cmp<C>(S.DY[Km1]), cmp<Cb>(S.DY[Km1]) - dym3);
            const BgCoef ca = unpack_bg_coef(__float_as_uint(fr[2]), __float_as_uint(fr[3]), __float_as_uint(fr[4]));
            const BgCoef cb = unpack_bg_coef(__float_as_uint(bf[2]), __float_as_uint(bf[3]), __float_as_uint(bf[4]));
            const Local2 o = local_eval2_cf(st, ca, cb, ih2, nu, f2(kap),
                                            f2fma(f2(fscale), make_float2(fr[0], bf[0]), f2(lam)), f2(lsat),
                                            make_float2(fr[1], bf[1]));
            float er, eb;
            if (kap == 0.f) {
                er = div_ftz(-o.G.x, o.Ep.x);
                eb = div_ftz(-o.G.y, o.Ep.y);
            } else {
                er = pick_update(o.G.x, o.Ep.x, o.P.x, o.D.x, o.g.x, sp, Df, h2over6, inv2P);
                eb = pick_update(o.G.y, o.Ep.y, o.P.y, o.D.y, o.g.y, sp, Df, h2over6, inv2P);
            }
            const float rnew = st.c0.x + er;
            const float bnew = st.c0.y + eb;
            // plane s-2 is final for both columns: its red cell (column C) and the black one
            if (blk_ok) {
                const float2 out = C ? make_float2(bnew, S.RL.y) : make_float2(S.RL.x, bnew);
                *reinterpret_cast<float2*>(Vrow + (size_t)(s - 2) * plane) = out;
            }
            if (red_ok) sr[K0 * PF + cF + C] = rnew;
            if (C) {
                S.RP.y = S.RL.y;
                S.RL.y = rnew;
            } else {
                S.RP.x = S.RL.x;
                S.RL.x = rnew;
            }
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        using I3 = std::integral_constant<int, 3>;
        if (((yg + z0 - 1) & 1) == 0) {  // column x red on planes z0-1, z0+1, ...
            for (int it = 0; it < nsteps; it += 4) {
                const int s = z0 - 1 + it;
                step(I0{}, I0{}, s);
                step(I1{}, I1{}, s + 1);
                step(I2{}, I0{}, s + 2);
                step(I3{}, I1{}, s + 3);
            }
        } else {
            for (int it = 0; it < nsteps; it += 4) {
                const int s = z0 - 1 + it;
                step(I0{}, I1{}, s);
                step(I1{}, I0{}, s + 1);
                step(I2{}, I1{}, s + 2);
                step(I3{}, I0{}, s + 3);
            }
        }
    } else {
        // ---------------------------------------------------------------- x-halo lanes
        const int idx = (warp - TY - 2) * 32 + lane;
        const bool active = idx < G::NXH;
        const int xh = idx < G::HF ? -1 : 64;
        const int y = (active ? idx % G::HF : 0) - 1;
        const int par = (x0 + xh + y0 + y) & 1;  // the cell is red on planes p with p + par even
        const int cE = (y + 2) * WS + XO + xh;
        const int cF = (y + 1) * WS + XO + xh;
        HaloState H;
        auto derive1 = [&](int k) {
            const float* e = se + k * PE + cE;
            const float um = e[-WS], uc = e[0], up = e[WS];
            const float lm = e[-1], rp = e[1];
            H.U[k] = uc;
            H.DX[k] = rp - lm;
            H.DY[k] = up - um;
            H.AX[k] = rp + lm;
            H.AY[k] = up + um;
            H.EXY[k] = (e[WS + 1] - e[WS - 1]) - (e[-WS + 1] - e[-WS - 1]);
        };
        cp_async_wait_2();
        __syncthreads();
        derive1(3);
        derive1(0);
        auto hstep = [&](auto Jt, int s) {
            constexpr int J = decltype(Jt)::value;
            constexpr int K0 = J, K1 = (J + 1) & 3, Km1 = (J + 3) & 3;
            cp_async_wait_1();
            __syncthreads();
            issue(s + 3, Km1);
            derive1(K1);
            if (!active || s > zlast || ((par + s) & 1)) return;
            Stencil<float> st;
            st.c0 = H.U[K0];
            st.ax = H.AX[K0];
            st.ay = H.AY[K0];
            st.az = H.U[K1] + H.U[Km1];
            st.exy = H.EXY[K0];
            st.exz = H.DX[K1] - H.DX[Km1];
            st.eyz = H.DY[K1] - H.DY[Km1];
            const float rhs = fscale * fld(0, K0)[cF] + lam;
            const BgCoef cf = unpack_bg_coef(__float_as_uint(fld(2, K0)[cF]), __float_as_uint(fld(3, K0)[cF]),
                                             __float_as_uint(fld(4, K0)[cF]));
            const Local<float> o = local_eval_cf(st, cf, ih2, nu, kap, rhs, lsat, fld(1, K0)[cF]);
            sr[K0 * PF + cF] = st.c0 + col_update1(o, kap, sp, Df, h2over6, inv2P);
        };
        using I0 = std::integral_constant<int, 0>;
        using I1 = std::integral_constant<int, 1>;
        using I2 = std::integral_constant<int, 2>;
        using I3 = std::integral_constant<int, 3>;
        for (int it = 0; it < nsteps; it += 4) {
            const int s = z0 - 1 + it;
            hstep(I0{}, s);
            hstep(I1{}, s + 1);
            hstep(I2{}, s + 2);
            hstep(I3{}, s + 3);
        }
    }
}

}  // namespace pmeft
