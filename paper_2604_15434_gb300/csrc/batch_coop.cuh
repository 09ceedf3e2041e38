// batch_coop.cuh -- the coarse part of every box's inner V-cycle in one persistent,
// cooperative launch (included by mg.cu; uses its per-cell device functions).
//
// In a batched solve every box whose mesh is at least 2 kCoopTop runs the levels above
// kCoopTop^3 as ordinary kernels on its own graph branch; the levels kCoopTop^3 .. 4^3 of all
// boxes then run in a single cooperative launch that walks a list of phases (the half-sweeps,
// residual, gauge reduction, restriction and FAS right-hand side of each level on the way
// down, the coarsest solve, and the prolongation and half-sweeps on the way up).  In a phase
// the work items are (box, chunk of kCoopItem cells) pairs, spread over the blocks; a grid
// barrier separates dependent phases.  This replaces some forty small launches per box and
// outer iteration (each a few microseconds of launch latency on a 32^3-or-smaller grid) by
// one launch for all boxes.
//
// The grid barrier counts arrivals in global memory and spins on a generation word with a
// bounded wait: a block that waits longer than spin_limit clock cycles records
// PM_ERR_TIMEOUT in the error word and leaves, and every block that then reaches a barrier
// (or is spinning in one) sees the error and leaves too, so a lost block cannot hang the GPU.
// The host reads the error word after the launch.  For testing that path, fail_block /
// fail_barrier make one block leave the kernel just before a given barrier, so that the
// others' waits run out (nothing faults: the blocks only stop early).
#pragma once

namespace pmeft {

constexpr int kCoopTop = 32;       // finest level size the cooperative kernel takes
constexpr int kCoopLevels = 4;     // 32^3, 16^3, 8^3, 4^3
constexpr int kCoopItem = 2048;    // cells per work item
constexpr int kCoopThreads = 256;
constexpr int kCoopMaxItems = (kCoopTop * kCoopTop * kCoopTop + kCoopItem - 1) / kCoopItem;  // per box and level

struct CoopLevel {
    float* u[2];
    float* f;
    float* r;
    float* ur;
    const float* bg;
    uint8_t* kmask;
    uint8_t* sat;
    int n;
};

struct CoopBox {
    CoopLevel lv[kCoopLevels];
    float nu, kap;      // the level coefficients in the inner cycle's precision
    double nu_d, kap_d;
};

struct CoopParams {
    const CoopBox* boxes;
    const int* active;  // per box: 0 once it has converged (its items are skipped)
    int nbox;
    int npre, npost, coarse_sweeps;
    double eta;
    double* partials;   // [nbox][kCoopMaxItems][2]: residual sum and unfloored count per item
    float* gm;          // [nbox]: gauge shift of the level being restricted
    unsigned* bar;      // [2]: arrival counter, generation
    int* err;           // PM_OK, or PM_ERR_TIMEOUT after a wait that gave up
    long long spin_limit;
    int fail_block, fail_barrier;  // test knob: that block leaves before that barrier (-1: off)
};

// Grid-wide barrier with a bounded wait; returns false once the error word is set.
__device__ __forceinline__ bool coop_sync(const CoopParams& P, int& nbar)
{
    const int id = nbar++;
    if ((int)blockIdx.x == P.fail_block && id == P.fail_barrier) return false;  // test knob: this block leaves
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        volatile unsigned* gen = P.bar + 1;
        volatile int* err = P.err;
        const unsigned g = *gen;
        __threadfence();
        const unsigned nb = gridDim.x;
        if (atomicAdd(P.bar, 1u) == nb - 1) {
            atomicExch(P.bar, 0u);
            __threadfence();
            atomicAdd(P.bar + 1, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (*err != PM_OK) break;
                if (clock64() - t0 > P.spin_limit) {
                    atomicCAS(P.err, PM_OK, (int)PM_ERR_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        ok = *err == PM_OK;
    }
    __syncthreads();
    return ok != 0;
}

__global__ void __launch_bounds__(kCoopThreads) k_batch_coarse(CoopParams P)
{
    __shared__ CoarsestSmem<float> csm;
    __shared__ double bred[2][kCoopThreads / 32];
    int nbar = 0;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    const int nl = kCoopLevels;
    // every block checks the box table first (the same checks everywhere, so all leave
    // together): a null buffer or an unexpected level size is recorded and nothing is accessed
    {
        __shared__ int bad;
        if (t == 0) {
            bad = 0;
            for (int b = 0; b < P.nbox && !bad; ++b)
                for (int k = 0; k < nl; ++k) {
                    const CoopLevel& L = P.boxes[b].lv[k];
                    if (!L.u[0] || !L.u[1] || !L.f || !L.r || !L.ur || !L.bg || !L.kmask || !L.sat ||
                        L.n != (kCoopTop >> k))
                        bad = 1;
                }
        }
        __syncthreads();
        if (bad) {
            if (t == 0) atomicCAS(P.err, PM_OK, (int)PM_ERR_INVALID_ARG);
            return;
        }
    }
    // every box has the same level sizes here: 32, 16, 8, 4
    int cur[kCoopLevels] = {0, 0, 0, 0};

    // run fn(box, cell) over `cells` cells of every active box, items spread over the blocks
    auto for_cells = [&](size_t cells, auto&& fn) {
        const int ipb = (int)((cells + kCoopItem - 1) / kCoopItem);
        const int items = P.nbox * ipb;
        for (int it = blockIdx.x; it < items; it += gridDim.x) {
            const int b = it / ipb, ch = it - b * ipb;
            if (!P.active[b]) continue;
            const size_t c0 = (size_t)ch * kCoopItem;
            const size_t c1 = c0 + kCoopItem < cells ? c0 + kCoopItem : cells;
            for (size_t c = c0 + t; c < c1; c += blockDim.x) fn(b, c, it);
        }
    };
    auto sweep = [&](int l) -> bool {
        for (int colour = 0; colour < 2; ++colour) {
            const int n = P.boxes[0].lv[l].n;
            const int lg = __ffs(n) - 1;
            const size_t half = (size_t)n * n * (n >> 1);
            for_cells(half, [&](int b, size_t c, int) {
                const CoopBox& B = P.boxes[b];
                const CoopLevel& L = B.lv[l];
                const float* A = L.u[cur[l]];
                float* Bv = L.u[1 - cur[l]];
                const double nn = (double)n * (double)n;
                const float sp = B.nu >= 0.f ? -1.f : 1.f;
                const double sqDf = P.eta * 6.0 * fabs(B.nu_d) * nn;
                const float lsn = B.kap != 0.f ? (float)(0.75 * B.nu_d * (1.0 - P.eta) / B.kap_d) : 0.f;
                half_sweep_cell<float, true, false>(A, colour == 0 ? A : Bv, Bv, L.f, 1.f, 0.f, L.kmask, L.bg, nullptr, n,
                                                    lg, colour, (float)nn, B.nu, B.kap, sp, (float)(sqDf * sqDf), lsn,
                                                    0.f, c);
            });
            if (!coop_sync(P, nbar)) return false;
        }
        cur[l] = 1 - cur[l];
        return true;
    };

    // ---- down: levels 0 .. nl-2 (32^3 .. 8^3)
    for (int l = 0; l + 1 < nl; ++l) {
        for (int s = 0; s < P.npre; ++s)
            if (!sweep(l)) return;
        // residual (no floored piece on coarse levels) and its per-item sums
        {
            const int n = P.boxes[0].lv[l].n;
            const int lg = __ffs(n) - 1;
            const size_t cells = (size_t)n * n * n;
            const int ipb = (int)((cells + kCoopItem - 1) / kCoopItem);
            const int items = P.nbox * ipb;
            for (int it = blockIdx.x; it < items; it += gridDim.x) {
                const int b = it / ipb, ch = it - b * ipb;
                if (!P.active[b]) continue;  // uniform across the block
                const CoopBox& B = P.boxes[b];
                const CoopLevel& L = B.lv[l];
                const double nn = (double)n * (double)n;
                const double sqDf = P.eta * 6.0 * fabs(B.nu_d) * nn;
                const float lsn = B.kap != 0.f ? (float)(0.75 * B.nu_d * (1.0 - P.eta) / B.kap_d) : 0.f;
                float fa[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
                const size_t c0 = (size_t)ch * kCoopItem;
                const size_t c1 = c0 + kCoopItem < cells ? c0 + kCoopItem : cells;
                for (size_t c = c0 + t; c < c1; c += blockDim.x)
                    residual_cell<float, true, true, false>(L.u[cur[l]], L.f, 1.f, 0.f, L.kmask, L.bg, nullptr, n, lg,
                                                            (float)nn, B.nu, B.kap, (float)(sqDf * sqDf), lsn, false,
                                                            L.r, L.sat, nullptr, nullptr, nullptr, c, fa);
                double s0 = fa[0], s1 = fa[3];
                for (int o = 16; o > 0; o >>= 1) {
                    s0 += __shfl_down_sync(0xffffffffu, s0, o);
                    s1 += __shfl_down_sync(0xffffffffu, s1, o);
                }
                if (lane == 0) {
                    bred[0][wid] = s0;
                    bred[1][wid] = s1;
                }
                __syncthreads();
                if (t == 0) {
                    double a = 0.0, w = 0.0;
                    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                        a += bred[0][q];
                        w += bred[1][q];
                    }
                    P.partials[((size_t)b * kCoopMaxItems + ch) * 2] = a;
                    P.partials[((size_t)b * kCoopMaxItems + ch) * 2 + 1] = w;
                }
                __syncthreads();
            }
            if (!coop_sync(P, nbar)) return;
            // the gauge shift of every box: sum r / count unfloored, in a fixed order
            if (blockIdx.x == 0)
                for (int b = t; b < P.nbox; b += blockDim.x) {
                    double a = 0.0, w = 0.0;
                    for (int ch = 0; ch < ipb; ++ch) {
                        a += P.partials[((size_t)b * kCoopMaxItems + ch) * 2];
                        w += P.partials[((size_t)b * kCoopMaxItems + ch) * 2 + 1];
                    }
                    P.gm[b] = w > 0.0 ? (float)(a / w) : 0.f;
                }
            if (!coop_sync(P, nbar)) return;
        }
        // restriction to level l+1 and its FAS right-hand side
        {
            const int nc = P.boxes[0].lv[l + 1].n;
            const int lgc = __ffs(nc) - 1;
            const size_t cc = (size_t)nc * nc * nc;
            for_cells(cc, [&](int b, size_t c, int) {
                const CoopLevel& L = P.boxes[b].lv[l];
                const CoopLevel& C = P.boxes[b].lv[l + 1];
                restrict_fas_cell<float>(L.u[cur[l]], L.r, L.sat, L.kmask, P.gm[b], nc, lgc, C.ur, C.u[0], C.r, C.kmask,
                                         c);
            });
            if (!coop_sync(P, nbar)) return;
            cur[l + 1] = 0;
            for_cells(cc, [&](int b, size_t c, int) {
                const CoopBox& B = P.boxes[b];
                const CoopLevel& C = B.lv[l + 1];
                fas_rhs_cell<float, true>(C.u[0], C.r, C.kmask, C.bg, nc, lgc, (float)((double)nc * (double)nc), B.nu,
                                          B.kap, C.f, nullptr, nullptr, 0.f, false, 0.f, cc, c);
            });
            if (!coop_sync(P, nbar)) return;
        }
    }
    // ---- coarsest level: one block per box
    {
        const int l = nl - 1;
        for (int b = blockIdx.x; b < P.nbox; b += gridDim.x) {
            if (!P.active[b]) continue;
            const CoopBox& B = P.boxes[b];
            const CoopLevel& L = B.lv[l];
            coarsest_block<float, true>(L.u[0], L.f, 1.f, L.kmask, L.bg, L.n, (double)L.n * (double)L.n, B.nu_d,
                                        B.kap_d, P.eta, P.coarse_sweeps, false, csm);
            __syncthreads();
        }
        cur[l] = 0;
        if (!coop_sync(P, nbar)) return;
    }
    // ---- up: levels nl-2 .. 0
    for (int l = nl - 2; l >= 0; --l) {
        const int nc = P.boxes[0].lv[l + 1].n;
        const int lgc = __ffs(nc) - 1;
        const size_t cc = (size_t)nc * nc * nc;
        for_cells(cc, [&](int b, size_t c, int) {
            const CoopLevel& L = P.boxes[b].lv[l];
            const CoopLevel& C = P.boxes[b].lv[l + 1];
            prolong_add_cell<float>(C.u[cur[l + 1]], C.ur, nc, lgc, L.u[cur[l]], c);
        });
        if (!coop_sync(P, nbar)) return;
        for (int s = 0; s < P.npost; ++s)
            if (!sweep(l)) return;
    }
}

}  // namespace pmeft
