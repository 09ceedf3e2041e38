// conv_umma.cuh -- the U-Net's 3x3x3 periodic convolution on the fifth-generation tensor cores:
// tcgen05.mma (BF16 x BF16 -> FP32) with the accumulator in tensor memory.
//
// Implicit GEMM per output tile of M = 128 voxels (8 in x, 16 in y, one z plane): D[128 x NT]
// = sum over taps and 16-channel input chunks of A[128 x 16] B[16 x NT], where the A rows are
// the tile's voxels shifted by the tap and B is the tap's weight block.  Both operands sit in
// shared memory in the K-major, unswizzled layout of the tensor core's descriptors: 8 rows of
// 16 bytes (8 BF16 k-values) form a 128-byte core matrix; the leading byte offset steps to the
// next 8 k, the stride byte offset to the next 8 rows.
//   A: a block marches an 8 x 16 column of tiles up z.  It keeps four patch planes (10 x 18
//      voxels, periodic) in a ring, each as [chunk][k-half][y][x] x 16 bytes: eight consecutive
//      x of one patch row are a core matrix, the next y row is the next one (stride 160 bytes),
//      so the A operand of a tap is the plane z + dz with its start moved by (dy, dx); no data is
//      copied per tap, and each input plane is loaded once per column (plus two halo planes
//      per work item) instead of three times.
//   B: the layer's weights for NT output channels, resident for the block's lifetime, as
//      [tap][chunk][k-half][co] x 16 bytes (stride 128 bytes per 8 outputs).
// Pipeline per plane z: the block waits (bounded) for plane z - 1's MMAs, starts the copy of
// plane z + 2 into the slot plane z - 2 left, waits for plane z + 1, then one thread issues the
// 27 x chunks MMAs of plane z into one of two tensor-memory accumulators (128 lanes x NT FP32
// columns each) and commits them to that accumulator's mbarrier, while every warp reads plane
// z - 1's 32 rows from the other accumulator with tcgen05.ld, adds the bias, applies ReLU / the
// mask and stores BF16.  So the tensor core, the copies and the epilogue overlap.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace pmeft {

constexpr int kUmTX = 8, kUmTY = 16;                       // output tile (x, y), one z plane
constexpr int kUmPX = kUmTX + 2, kUmPY = kUmTY + 2;
constexpr int kUmPP = kUmPX * kUmPY;                       // 180 voxels per patch plane
constexpr int kUmSlots = 4;                                // patch planes held: three read, one loading
constexpr int kUmThreads = 128;
constexpr long long kUmSpin = 1ll << 26;                   // bound on an mbarrier wait (polls)

__device__ __forceinline__ uint32_t um_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// the descriptor version 1 (bits 46-47), no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t um_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16 (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t um_idesc(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void um_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t accum)
{
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
        "l"(a), "l"(b), "r"(idesc), "r"(accum));
}

__device__ __forceinline__ void um_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(um_smem(mbar))
                 : "memory");
}

__device__ __forceinline__ bool um_try_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(um_smem(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void um_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

__device__ __forceinline__ void um_cp16(uint32_t dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src));
}

// dynamic shared memory of k_conv3d_umma for Cin input channels and NT outputs: the resident
// weights, kUmSlots patch planes, two mbarriers and the tensor-memory address
template <int NT>
constexpr size_t umma_smem(int cin)
{
    return (size_t)27 * (cin / 16) * NT * 32 + (size_t)kUmSlots * (cin / 16) * kUmPP * 32 + 64;
}

// tensor-memory columns of the block: two accumulators of NT columns, each at a power-of-two
// column offset, the allocation a power of two of at least 32
template <int NT>
constexpr uint32_t um_acc_stride()
{
    return NT <= 16 ? 16 : (NT <= 32 ? 32 : (NT <= 64 ? 64 : 128));
}

// out[v][out_off + co0 + c] = act(sum_tap sum_ci in[v + tap][ci] W[tap][ci][co0 + c] + bias[co0 + c]),
// c < NT, optionally times (mask[v][mask_off + co0 + c] > 0); bias may be null (no bias term).
// wt: the packed weights [tap][Cin/16][Cout][16] of the whole layer (Cout outputs).  Work item:
// an 8 x 16 column of outputs over zl planes (zl divides n).  err (nullable): set to 1 if an
// mbarrier wait gave up (the block then stops; what it has not written stays unwritten).
template <int NT>
__global__ void __launch_bounds__(kUmThreads) k_conv3d_umma(const __nv_bfloat16* __restrict__ in, int in_ld, int in_off,
                                                            int Cin, const __nv_bfloat16* __restrict__ wt, int Cout,
                                                            int co0, const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ out, int out_ld, int out_off,
                                                            int n, int zl, int relu,
                                                            const __nv_bfloat16* __restrict__ mask, int mask_ld,
                                                            int mask_off, int* __restrict__ err)
{
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 128, "N of a kind::f16 MMA with M = 128");
    constexpr uint32_t kStride = um_acc_stride<NT>();
    constexpr uint32_t kCols = 2 * kStride < 32 ? 32 : 2 * kStride;
    extern __shared__ __align__(128) unsigned char um_raw[];
    const int kch = Cin / 16;
    const uint32_t slot_bytes = (uint32_t)kch * 2 * kUmPP * 16;
    unsigned char* sW = um_raw;                                   // [27][kch][2][NT] x 16 B
    unsigned char* sP = sW + (size_t)27 * kch * NT * 32;          // [slot][kch][2][PY][PX] x 16 B
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sP + (size_t)kUmSlots * slot_bytes);  // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t sW_s = um_smem(sW), sP_s = um_smem(sP);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem(tslot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(um_smem(mbar)), "r"(1));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(um_smem(mbar + 1)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");  // visible to the tensor core's arrive
    }
    // resident weights: 16-byte piece (tap, chunk, half, c) of output co0 + c
    const int wpieces = 27 * kch * 2 * NT;
    for (int q = t; q < wpieces; q += kUmThreads) {
        const int c = q % NT, r = q / NT;  // r = (tap * kch + ch) * 2 + half
        const int half = r & 1, tc = r >> 1;
        const __nv_bfloat16* src = wt + ((size_t)tc * Cout + co0 + c) * 16 + half * 8;
        um_cp16(sW_s + (uint32_t)q * 16u, src);
    }
    asm volatile("cp.async.commit_group;\n" ::);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;

    const int m = n - 1;
    const int tx = n / kUmTX, ty = n / kUmTY, nzs = n / zl;
    const long long items = (long long)tx * ty * nzs;
    constexpr uint32_t idesc = um_idesc(128, NT);
    // descriptors of the first A and B core matrices; the others differ only in the start
    // address field (addresses below 256 KB, so adding (offset >> 4) never carries out of it)
    const uint64_t dA0 = um_desc(sP_s, kUmPP * 16, kUmPX * 16);
    const uint64_t dB0 = um_desc(sW_s, NT * 16, 128);
    const int ppieces = kch * 2 * kUmPP;
    uint32_t ph[2] = {0u, 0u};  // parity of each mbarrier's next completion
    int inflight = -1;          // the accumulator whose MMAs are committed but not yet waited for
    bool failed = false;

    // all threads poll (bounded) for the completion of accumulator b's MMAs
    auto wait_mma = [&](int b) -> bool {
        bool done = false;
        for (long long it = 0; it < kUmSpin && !done; ++it) done = um_try_wait(mbar + b, ph[b]);
        if (done) {
            ph[b] ^= 1u;
            inflight = -1;
        }
        return done;
    };

    for (long long item = blockIdx.x; item < items && !failed; item += gridDim.x) {
        const int bx = (int)(item % tx), by = (int)((item / tx) % ty), bz = (int)(item / ((long long)tx * ty));
        const int x0 = bx * kUmTX, y0 = by * kUmTY, zs = bz * zl;
        // patch plane z (periodic) into slot sl: 16-byte piece (chunk, half, y, x)
        auto load_plane = [&](int z, int sl) {
            const uint32_t base = sP_s + (uint32_t)sl * slot_bytes;
            const size_t zo = (size_t)(z & m) * n;
            for (int q = t; q < ppieces; q += kUmThreads) {
                const int p = q % kUmPP, r = q / kUmPP;  // r = chunk * 2 + half
                const int px = p % kUmPX, py = p / kUmPX;
                const size_t v = (zo + ((y0 - 1 + py) & m)) * n + ((x0 - 1 + px) & m);
                um_cp16(base + (uint32_t)q * 16u, in + v * in_ld + in_off + r * 8);
            }
            asm volatile("cp.async.commit_group;\n" ::);
        };
        // the outputs of plane z from accumulator b: row warp * 32 + lane is voxel (x0 + row % 8,
        // y0 + row / 8)
        auto epilogue = [&](int z, int b) {
            const int row = warp * 32 + lane;
            const int xv = x0 + (row & 7), yv = y0 + (row >> 3);
            const size_t v = ((size_t)z * n + yv) * n + xv;
#pragma unroll
            for (int c0 = 0; c0 < NT; c0 += 16) {
                float d[16];
                um_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)b * kStride + (uint32_t)c0, d);
                __align__(16) __nv_bfloat16 o[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    float y = bias ? d[q] + bias[co0 + c0 + q] : d[q];  // no bias in the backward-data convolution
                    if (relu) y = fmaxf(y, 0.f);
                    if (mask && !(__bfloat162float(mask[v * mask_ld + mask_off + co0 + c0 + q]) > 0.f)) y = 0.f;
                    o[q] = __float2bfloat16(y);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + v * out_ld + out_off + co0 + c0);
                dst[0] = reinterpret_cast<const uint4*>(o)[0];
                dst[1] = reinterpret_cast<const uint4*>(o)[1];
            }
        };
        // planes zs - 1 .. zs + zl are read; plane z sits in slot (z - zs + 1) % kUmSlots
        load_plane(zs - 1, 0);
        load_plane(zs, 1);
        load_plane(zs + 1, 2);
        for (int s = 0; s < zl; ++s) {
            const int z = zs + s;
            // plane z - 1's MMAs done: its accumulator is ready and plane z - 2's slot is free
            bool ok = s == 0 || wait_mma((s - 1) & 1);
            const bool more = s + 2 <= zl;
            if (more) load_plane(z + 2, (s + 3) % kUmSlots);
            // plane z + 1 has landed (the newest group, plane z + 2, may still be in flight)
            if (more) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
            else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor core
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            ok = __syncthreads_and(ok) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) {  // block-uniform
                failed = true;
                break;
            }
            // plane z: 27 taps x kch chunks into accumulator s % 2
            if (t == 0) {
                uint32_t acc = 0;
                for (int ch = 0; ch < kch; ++ch)
                    for (int tap = 0; tap < 27; ++tap) {
                        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                        const uint32_t aoff = (uint32_t)((s + dz) % kUmSlots) * slot_bytes +
                                              (uint32_t)(ch * 2 * kUmPP + dy * kUmPX + dx) * 16u;
                        const uint32_t boff = (uint32_t)((tap * kch + ch) * 2 * NT) * 16u;
                        um_mma(tmem + (uint32_t)(s & 1) * kStride, dA0 + (aoff >> 4), dB0 + (boff >> 4), idesc, acc);
                        acc = 1;
                    }
                um_commit(mbar + (s & 1));
            }
            inflight = s & 1;
            if (s >= 1) epilogue(z - 1, (s - 1) & 1);
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        if (failed) break;
        // the last plane
        bool ok = wait_mma((zl - 1) & 1);
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        ok = __syncthreads_and(ok) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) {
            failed = true;
            break;
        }
        epilogue(zs + zl - 1, (zl - 1) & 1);
        // every thread is done with the accumulators and the slots before the next item
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (failed) {
        if (t == 0) {
            if (err) atomicExch(err, 1);
            // give the MMAs still in flight one more bounded wait before their memory is released
            if (inflight >= 0)
                for (long long it = 0; it < kUmSpin; ++it)
                    if (um_try_wait(mbar + inflight, ph[inflight])) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

}  // namespace pmeft
