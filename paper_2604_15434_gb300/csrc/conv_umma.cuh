// conv_umma.cuh -- the U-Net's 3x3x3 periodic convolution on the fifth-generation tensor cores:
// tcgen05.mma (BF16 x BF16 -> FP32) with the accumulator in tensor memory.
//
// Implicit GEMM per output tile of M = 128 voxels (8 in x, 16 in y, one z plane): D[128 x NT]
// = sum over taps and 16-channel input chunks of A[128 x 16] B[16 x NT], where the A rows are
// the tile's voxels shifted by the tap and B is the tap's weight block.  Both operands sit in
// shared memory in the K-major, unswizzled layout of the tensor core's descriptors: 8 rows of
// 16 bytes (8 BF16 k-values) form a 128-byte core matrix; the leading byte offset steps to the
// next 8 k, the stride byte offset to the next 8 rows.
//   A: the block stages the tile's input patch (10 x 18 x 3 voxels, periodic) as
//      [chunk][k-half][z][y][x] x 16 bytes.  Eight consecutive x of one patch row are a core
//      matrix, the next y row is the next one (stride 160 bytes), so the A operand of a tap is
//      the same patch with its start moved by the tap's offset: no data is copied per tap.
//   B: the layer's weights for NT output channels, resident for the block's lifetime, as
//      [tap][chunk][k-half][co] x 16 bytes (stride 128 bytes per 8 outputs).
// One thread issues the 27 x chunks MMAs of a tile into the tensor-memory accumulator (128 lanes
// x NT FP32 columns) and commits them to an mbarrier; after its (bounded) wait, each warp reads
// its 32 rows back with tcgen05.ld, adds the bias, applies ReLU / the mask, and stores BF16.
// Blocks are persistent over tiles; the next tile's patch is staged while no MMA reads the
// buffer, and several blocks per SM keep the tensor core busy while one of them loads.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace pmeft {

constexpr int kUmTX = 8, kUmTY = 16;                       // output tile (x, y), one z plane
constexpr int kUmPX = kUmTX + 2, kUmPY = kUmTY + 2, kUmPZ = 3;
constexpr int kUmPV = kUmPX * kUmPY * kUmPZ;               // 540 patch voxels
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

// dynamic shared memory of k_conv3d_umma for Cin input channels and NT outputs
template <int NT>
constexpr size_t umma_smem(int cin)
{
    return (size_t)27 * (cin / 16) * NT * 32 + (size_t)(cin / 16) * kUmPV * 32 + 64;
}

// out[v][out_off + co0 + c] = act(sum_tap sum_ci in[v + tap][ci] W[tap][ci][co0 + c] + bias[co0 + c]),
// c < NT, optionally times (mask[v][mask_off + co0 + c] > 0); bias may be null (no bias term).  wt: the packed weights
// [tap][Cin/16][Cout][16] of the whole layer (Cout outputs).  err (nullable): set to 1 if an
// mbarrier wait gave up (the tile's output is then not written).
template <int NT>
__global__ void __launch_bounds__(kUmThreads) k_conv3d_umma(const __nv_bfloat16* __restrict__ in, int in_ld, int in_off,
                                                            int Cin, const __nv_bfloat16* __restrict__ wt, int Cout,
                                                            int co0, const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ out, int out_ld, int out_off,
                                                            int n, int relu, const __nv_bfloat16* __restrict__ mask,
                                                            int mask_ld, int mask_off, int* __restrict__ err)
{
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 256, "N of a kind::f16 MMA with M = 128");
    constexpr uint32_t kCols = NT <= 32 ? 32 : (NT <= 64 ? 64 : (NT <= 128 ? 128 : 256));
    extern __shared__ __align__(128) unsigned char um_raw[];
    const int kch = Cin / 16;
    unsigned char* sW = um_raw;                                   // [27][kch][2][NT] x 16 B
    unsigned char* sP = sW + (size_t)27 * kch * NT * 32;          // [kch][2][PZ][PY][PX] x 16 B
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sP + (size_t)kch * kUmPV * 32);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t sW_s = um_smem(sW), sP_s = um_smem(sP);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(um_smem(tslot)),
                     "r"(kCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(um_smem(mbar)), "r"(1));
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
    const int tx = n / kUmTX, ty = n / kUmTY;
    const long long ntiles = (long long)tx * ty * n;
    constexpr uint32_t idesc = um_idesc(128, NT);
    const uint32_t lboA = kUmPV * 16, sboA = kUmPX * 16;
    const uint32_t lboB = NT * 16, sboB = 128;
    uint32_t phase = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int bx = (int)(tile % tx), by = (int)((tile / tx) % ty), bz = (int)(tile / ((long long)tx * ty));
        const int x0 = bx * kUmTX, y0 = by * kUmTY, z0 = bz;
        // the input patch of the tile: 16-byte piece (chunk, half, voxel)
        const int ppieces = kch * 2 * kUmPV;
        for (int q = t; q < ppieces; q += kUmThreads) {
            const int p = q % kUmPV, r = q / kUmPV;  // r = chunk * 2 + half
            const int half = r & 1, ch = r >> 1;
            const int px = p % kUmPX, py = (p / kUmPX) % kUmPY, pz = p / (kUmPX * kUmPY);
            const size_t v = ((size_t)((z0 - 1 + pz) & m) * n + ((y0 - 1 + py) & m)) * n + ((x0 - 1 + px) & m);
            um_cp16(sP_s + (uint32_t)q * 16u, in + v * in_ld + in_off + ch * 16 + half * 8);
        }
        asm volatile("cp.async.commit_group;\n" ::);
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        // make the copies visible to the tensor core's (async-proxy) reads
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (t == 0) {
            uint32_t acc = 0;
            for (int ch = 0; ch < kch; ++ch)
                for (int tap = 0; tap < 27; ++tap) {
                    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
                    const uint32_t a = sP_s + (uint32_t)(ch * 2 * kUmPV + (dz * kUmPY + dy) * kUmPX + dx) * 16u;
                    const uint32_t b = sW_s + (uint32_t)((tap * kch + ch) * 2 * NT) * 16u;
                    um_mma(tmem, um_desc(a, lboA, sboA), um_desc(b, lboB, sboB), idesc, acc);
                    acc = 1;
                }
            um_commit(mbar);
        }
        // one thread waits for the accumulator (bounded) and tells the block
        __shared__ int ok;
        if (t == 0) {
            int done = 0;
            for (long long it = 0; it < kUmSpin && !done; ++it) done = um_try_wait(mbar, phase) ? 1 : 0;
            ok = done;
            if (!done && err) atomicExch(err, 1);
        }
        __syncthreads();
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        if (!ok) {  // block-uniform
            failed = true;
            break;
        }
        // epilogue: row 32 warp + lane of the accumulator
        const int row = warp * 32 + lane;
        const int xv = x0 + (row & 7), yv = y0 + (row >> 3);
        const size_t v = ((size_t)z0 * n + yv) * n + xv;
#pragma unroll
        for (int c0 = 0; c0 < NT; c0 += 16) {
            float d[16];
            um_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, d);
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
        // every thread is done with the accumulator and the patch before the next tile
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
    }
    if (failed && t == 0) {
        // give the MMAs still in flight one more bounded wait before their memory is released
        for (long long it = 0; it < kUmSpin; ++it)
            if (um_try_wait(mbar, phase ^ 1u)) break;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

}  // namespace pmeft
