// conv_umma.cuh -- the U-Net's 3x3x3 periodic convolution on the fifth-generation tensor cores:
// tcgen05.mma (BF16 x BF16 -> FP32) with the accumulator in tensor memory.
//
// Implicit GEMM per output tile of M = 128 voxels (8 in x, 16 in y, one z plane): D[128 x NT]
// = sum over taps and 16-channel input chunks of A[128 x 16] B[16 x NT], where the A rows are
// the tile's voxels shifted by the tap and B is the tap's weight block.  Both operands sit in
// shared memory in the K-major, unswizzled layout of the tensor core's descriptors: 8 rows of
// 16 bytes (8 BF16 k-values) form a 128-byte core matrix; the leading byte offset steps to the
// next 8 k, the stride byte offset to the next 8 rows.
//   A: a block marches an 8 x 16 column of tiles up z.  It keeps SLOTS patch planes (10 x 18
//      voxels, periodic) in a ring, each as [chunk][k-half][y][x] x 16 bytes: eight consecutive
//      x of one patch row are a core matrix, the next y row is the next one (stride 160 bytes),
//      so the A operand of a tap is the plane z + dz with its start moved by (dy, dx); no data is
//      copied per tap, and each input plane is loaded once per column (plus two halo planes
//      per work item) instead of three times.
//   B: the layer's weights for NT output channels, resident for the block's lifetime, as
//      [tap][chunk][k-half][co] x 16 bytes (stride 128 bytes per 8 outputs).
// Pipeline per plane z: the block waits (bounded) for plane z - 1's MMAs, starts the copy of
// plane z + SLOTS - 2 into the slot plane z - 2 left (SLOTS - 3 planes are in flight), waits for
// plane z + 1, then one thread issues the
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

// zero 16 FP32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void um_st16_zero(uint32_t taddr)
{
    const uint32_t z = 0u;
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1,%1};\n" ::"r"(taddr),
        "r"(z)
        : "memory");
}

// weights held per (in-plane tap, chunk, k-half): the NT-row blocks of the z taps in the order
// dz = 2, 1, 0, 2, 1, so that every rotation of (2, 1, 0) is a window of three blocks
constexpr int kUmWGroups = 5;

// dynamic shared memory of k_conv3d_umma for Cin input channels, NT outputs and SLOTS patch
// planes: the resident weights, the planes, one mbarrier, the tensor-memory address and the NT
// biases
template <int NT, int SLOTS>
constexpr size_t umma_smem(int cin)
{
    return (size_t)9 * (cin / 16) * 2 * kUmWGroups * NT * 16 + (size_t)SLOTS * (cin / 16) * kUmPP * 32 + 32 + NT * 4;
}

// tensor-memory columns of the block: three output planes of NT FP32 columns each, the
// allocation a power of two of at least 32
template <int NT>
constexpr uint32_t um_cols()
{
    return 3 * NT <= 32 ? 32 : (3 * NT <= 64 ? 64 : (3 * NT <= 128 ? 128 : 256));
}

// out[v][out_off + co0 + c] = act(sum_tap sum_ci in[v + tap][ci] W[tap][ci][co0 + c] + bias[co0 + c]),
// c < NT (NT <= 64), optionally times (mask[v][mask_off + co0 + c] > 0); bias may be null (no bias
// term).  wt: the packed weights [tap][Cin/16][Cout][16] of the whole layer (Cout outputs).
// Work item: an 8 x 16 column of outputs over zl planes (zl divides n).
//
// The block walks the input planes p = zs - 1 .. zs + zl of its column.  Input plane p feeds
// output planes p + 1, p, p - 1 through the z taps dz = 0, 1, 2, so for each in-plane tap
// (dy, dx) and chunk one MMA of N = 3 NT (B = the three z taps' weight blocks side by side)
// adds its A operand, read once from shared memory, into all three outputs.  Each output plane
// z keeps NT tensor-memory columns at slot (z - zs) mod 3; the B window is chosen so that the
// three column groups of an MMA land in the slots of the right planes, and every MMA
// accumulates (a slot is zeroed when its plane starts).  Output plane p - 2 is complete after
// input plane p - 1's MMAs: the block waits (bounded) for them, reads that slot back with
// tcgen05.ld (bias, ReLU / mask, BF16 stores), zeroes it for plane p + 1, starts the copy of
// input plane p + SLOTS - 1, waits for plane p, and one thread issues plane p's 9 x chunks
// MMAs.  Several blocks per SM overlap one block's epilogue with another's MMAs.
// err (nullable): set to 1 if an mbarrier wait gave up (the block then stops; what it has not
// written stays unwritten).
template <int NT, int SLOTS>
__global__ void __launch_bounds__(kUmThreads) k_conv3d_umma(const __nv_bfloat16* __restrict__ in, int in_ld, int in_off,
                                                            int Cin, const __nv_bfloat16* __restrict__ wt, int Cout,
                                                            int co0, const float* __restrict__ bias,
                                                            __nv_bfloat16* __restrict__ out, int out_ld, int out_off,
                                                            int n, int zl, int relu,
                                                            const __nv_bfloat16* __restrict__ mask, int mask_ld,
                                                            int mask_off, int* __restrict__ err)
{
    static_assert(NT % 16 == 0 && NT >= 16 && NT <= 64, "N = 3 NT of a kind::f16 MMA with M = 128");
    static_assert(SLOTS >= 2, "the plane the MMAs read and at least one loading");
    constexpr int P = SLOTS - 1;  // planes loaded ahead of the one the MMAs read
    constexpr uint32_t kCols = um_cols<NT>();
    extern __shared__ __align__(128) unsigned char um_raw[];
    const int kch = Cin / 16;
    const uint32_t slot_bytes = (uint32_t)kch * 2 * kUmPP * 16;
    const uint32_t slot16 = slot_bytes >> 4;  // one patch-plane slot in 16-byte units
    unsigned char* sW = um_raw;                                               // [9][kch][2][5 NT] x 16 B
    unsigned char* sP = sW + (size_t)9 * kch * 2 * kUmWGroups * NT * 16;      // [slot][kch][2][PY][PX] x 16 B
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sP + (size_t)SLOTS * slot_bytes);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 2);
    float* sBias = reinterpret_cast<float*>(mbar + 4);  // [NT]
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
    if (bias)
        for (int c = t; c < NT; c += kUmThreads) sBias[c] = bias[co0 + c];
    // resident weights: 16-byte piece (tap9, chunk, half, group, c) = output co0 + c of the z tap
    // dz = (2 - group) mod 3 at in-plane tap tap9 = dy * 3 + dx
    const int wpieces = 9 * kch * 2 * kUmWGroups * NT;
    for (int q = t; q < wpieces; q += kUmThreads) {
        const int c = q % NT, r = q / NT;  // r = ((tap9 * kch + ch) * 2 + half) * 5 + group
        const int g = r % kUmWGroups, r2 = r / kUmWGroups;
        const int half = r2 & 1, tc = r2 >> 1;  // tc = tap9 * kch + ch
        const int tap9 = tc / kch, ch = tc - tap9 * kch;
        const int dz = (2 - g + 3) % 3;
        const int tap27 = dz * 9 + tap9;
        const __nv_bfloat16* src = wt + (((size_t)tap27 * kch + ch) * Cout + co0 + c) * 16 + half * 8;
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
    constexpr uint32_t idesc = um_idesc(128, 3 * NT);
    // descriptors of the first A and B core matrices; the others differ only in the start
    // address field (addresses below 256 KB, so adding (offset >> 4) never carries out of it)
    const uint64_t dA0 = um_desc(sP_s, kUmPP * 16, kUmPX * 16);
    const uint64_t dB0 = um_desc(sW_s, kUmWGroups * NT * 16, 128);
    const int ppieces = kch * 2 * kUmPP;
    uint32_t phase = 0;     // parity of the mbarrier's next completion
    bool inflight = false;  // MMAs committed but not yet waited for
    bool failed = false;

    // all threads poll (bounded) for the completion of the committed MMAs
    auto wait_mma = [&]() -> bool {
        bool done = false;
        for (long long it = 0; it < kUmSpin && !done; ++it) done = um_try_wait(mbar, phase);
        if (done) {
            phase ^= 1u;
            inflight = false;
        }
        return done;
    };

    for (long long item = blockIdx.x; item < items && !failed; item += gridDim.x) {
        const int bx = (int)(item % tx), by = (int)((item / tx) % ty), bz = (int)(item / ((long long)tx * ty));
        const int x0 = bx * kUmTX, y0 = by * kUmTY, zs = bz * zl;
        // input plane z (periodic) into slot sl: 16-byte piece (chunk, half, y, x); one copy group
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
        // tensor-memory column of output plane z's slot, for this warp's lanes
        auto slot_addr = [&](int z) {
            return tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(((z - zs + 3) % 3) * NT);
        };
        // the outputs of plane z from its slot: row warp * 32 + lane is voxel (x0 + row % 8,
        // y0 + row / 8)
        auto epilogue = [&](int z) {
            const int row = warp * 32 + lane;
            const int xv = x0 + (row & 7), yv = y0 + (row >> 3);
            const size_t v = ((size_t)z * n + yv) * n + xv;
#pragma unroll
            for (int c0 = 0; c0 < NT; c0 += 16) {
                float d[16];
                um_ld16(slot_addr(z) + (uint32_t)c0, d);
                __align__(16) __nv_bfloat16 o[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    float y = bias ? d[q] + sBias[c0 + q] : d[q];  // no bias in the backward-data convolution
                    if (relu) y = fmaxf(y, 0.f);
                    if (mask && !(__bfloat162float(mask[v * mask_ld + mask_off + co0 + c0 + q]) > 0.f)) y = 0.f;
                    o[q] = __float2bfloat16(y);
                }
                uint4* dst = reinterpret_cast<uint4*>(out + v * out_ld + out_off + co0 + c0);
                dst[0] = reinterpret_cast<const uint4*>(o)[0];
                dst[1] = reinterpret_cast<const uint4*>(o)[1];
            }
        };
        // input plane p sits in slot (p - zs + 1) % SLOTS; planes zs - 1 .. zs - 1 + P first
        for (int k = 0; k < P; ++k) load_plane(zs - 1 + k, k);
        for (int p = zs - 1; p <= zs + zl; ++p) {
            const int pr = p - zs + 1;  // 0 .. zl + 1
            bool ok = true;
            if (pr >= 1) {
                // input plane p - 1's MMAs done: output plane p - 2 is complete, and plane p - 1's
                // slot is free
                ok = wait_mma();
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                if (ok && p - 2 >= zs) epilogue(p - 2);
            }
            // output plane p + 1 starts in the slot plane p - 2 leaves
#pragma unroll
            for (int c0 = 0; c0 < NT; c0 += 16) um_st16_zero(slot_addr(p + 1) + (uint32_t)c0);
            asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            if (p + P <= zs + zl) load_plane(p + P, (pr + P) % SLOTS);
            else asm volatile("cp.async.commit_group;\n" ::);
            // plane p has landed (the P newest groups may still be in flight)
            asm volatile("cp.async.wait_group %0;\n" ::"n"(P) : "memory");
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // visible to the tensor core
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            ok = __syncthreads_and(ok) != 0;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) {  // block-uniform
                failed = true;
                break;
            }
            // plane p: 9 in-plane taps x kch chunks, N = 3 NT into the slots of planes p + 1, p, p - 1
            if (t == 0) {
                const int q3 = (p - zs + 3) % 3;
                const int j = (4 - q3) % 3;  // B window: column group k gets dz = (2 - j - k) mod 3
                const uint64_t ab = dA0 + (uint64_t)((uint32_t)(pr % SLOTS) * slot16);
                const uint64_t bb = dB0 + (uint64_t)(j * NT);
                const uint64_t bstep = (uint64_t)(kch * 2 * kUmWGroups * NT);  // one in-plane tap of B, 16-byte units
                for (int ch = 0; ch < kch; ++ch) {
                    const uint64_t ac = ab + (uint64_t)(ch * 2 * kUmPP);
                    const uint64_t bc = bb + (uint64_t)(ch * 2 * kUmWGroups * NT);
#pragma unroll
                    for (int tap9 = 0; tap9 < 9; ++tap9) {
                        const int dy = tap9 / 3, dx = tap9 % 3;
                        um_mma(tmem, ac + (uint64_t)(dy * kUmPX + dx), bc + (uint64_t)tap9 * bstep, idesc, 1u);
                    }
                }
                um_commit(mbar);
            }
            inflight = true;
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        }
        if (failed) break;
        // the last output plane
        bool ok = wait_mma();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        ok = __syncthreads_and(ok) != 0;
        if (!ok) {
            failed = true;
            break;
        }
        epilogue(zs + zl - 1);
        // every thread is done with the slots before the next item
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    if (failed && t == 0) {
        if (err) atomicExch(err, 1);
        // give the MMAs still in flight one more bounded wait before their memory is released
        if (inflight)
            for (long long it = 0; it < kUmSpin; ++it)
                if (um_try_wait(mbar, phase)) break;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
}

}  // namespace pmeft
