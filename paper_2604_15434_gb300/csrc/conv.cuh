// conv.cuh -- 3x3x3 periodic convolutions on BF16 tensor cores (mma.sync m16n8k16, FP32
// accumulation) for the learned warm start, plus their backward passes.
//
// Activations are NDHWC (channels fastest) BF16 on an n^3 periodic grid; a tensor may be a
// channel slice of a wider buffer (row stride `ld`, channel offset `off`, both multiples
// of 16 so every 16-channel chunk is 32-byte aligned).  Forward weights are packed as
// [tap][Cin/16][Cout][16] so one (tap, 16-channel chunk) step is a contiguous 16 x Cout
// block.  Taps are ordered t = (dz+1)*9 + (dy+1)*3 + (dx+1).
//
// Forward (implicit GEMM): M = voxels (128 per block), N = Cout, K = 27 x Cin, streamed in
// steps of one tap x 16 channels with a two-stage cp.async pipeline.  The backward data
// pass is the same kernel with the weights flipped in space and transposed in channels,
// followed by the ReLU mask of the layer input.  The weight gradient is a GEMM over voxels
// per tap: each block owns one tap and a chunk of voxels, stages both operands transposed
// in shared memory (channels x voxels) and writes an FP32 partial reduced in fixed order.
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

namespace pmeft {

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// D += A(16x16, row) * B(16x8, col), BF16 inputs, FP32 accumulators
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int kConvM = 128;    // voxels per block
constexpr int kRowA = 24;      // shared row stride of a 16-channel A row (bf16), conflict-free
constexpr int kWgTile = 128;   // voxels per staged block of the weight gradient
constexpr int kRowT = kWgTile + 8;  // shared row stride of a transposed row (bf16)

__device__ __forceinline__ int tap_voxel(int v, int n, int tap)
{
    const int m = n - 1;
    const int x = v & m, y = (v / n) & m, z = v / (n * n);
    const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
    return (((z + dz) & m) * n + ((y + dy) & m)) * n + ((x + dx) & m);
}

// out[v][off + c] = act(sum_tap sum_ci in[v + tap][ci] W[tap][ci][c] + bias[c]), optionally
// times (mask[v][moff + c] > 0).  N = Cout (multiple of 16, <= 96).  128 threads.
template <int N>
__global__ void __launch_bounds__(128) k_conv3d_fwd(const __nv_bfloat16* __restrict__ in, int in_ld, int in_off,
                                                   int Cin, const __nv_bfloat16* __restrict__ wt,
                                                   const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                   int out_ld, int out_off, int n, int relu,
                                                   const __nv_bfloat16* __restrict__ mask, int mask_ld, int mask_off)
{
    __shared__ __align__(16) __nv_bfloat16 sA[2][kConvM * kRowA];
    __shared__ __align__(16) __nv_bfloat16 sB[2][N * kRowA];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const long long vbase = (long long)blockIdx.x * kConvM;
    const int nvox = n * n * n;
    const int kchunks = Cin / 16, steps = 27 * kchunks;
    constexpr int NT = N / 8;
    float acc[2][NT][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    auto stage = [&](int s, int buf) {
        const int tap = s / kchunks, ch = s - tap * kchunks;
        // A: row t = voxel vbase + t shifted by the tap, 16 channels = 2 x 16 B
        const int v = (int)(vbase + t);
        const int vs = tap_voxel(v < nvox ? v : 0, n, tap);
        const __nv_bfloat16* src = in + (size_t)vs * in_ld + in_off + ch * 16;
        cp_async16(&sA[buf][t * kRowA], src);
        cp_async16(&sA[buf][t * kRowA + 8], src + 8);
        // B: the 16 x N weight block of this step, rows of 16 k per output channel
        const __nv_bfloat16* wsrc = wt + (size_t)s * N * 16;
        for (int q = t; q < N * 2; q += 128) cp_async16(&sB[buf][(q >> 1) * kRowA + (q & 1) * 8], wsrc + q * 8);
        cp_async_commit();
    };

    stage(0, 0);
    for (int s = 0; s < steps; ++s) {
        const int buf = s & 1;
        if (s + 1 < steps) {
            stage(s + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const unsigned* A32 = reinterpret_cast<const unsigned*>(sA[buf]);
        const unsigned* B32 = reinterpret_cast<const unsigned*>(sB[buf]);
        unsigned a[2][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const int r0 = warp * 32 + mt * 16 + g;
            a[mt][0] = A32[(r0 * kRowA) / 2 + t4];
            a[mt][1] = A32[((r0 + 8) * kRowA) / 2 + t4];
            a[mt][2] = A32[(r0 * kRowA) / 2 + t4 + 4];
            a[mt][3] = A32[((r0 + 8) * kRowA) / 2 + t4 + 4];
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            unsigned b[2];
            const int c = nt * 8 + g;
            b[0] = B32[(c * kRowA) / 2 + t4];
            b[1] = B32[(c * kRowA) / 2 + t4 + 4];
            mma_bf16(acc[0][nt], a[0], b);
            mma_bf16(acc[1][nt], a[1], b);
        }
        __syncthreads();
    }
    // epilogue: bias, activation, optional mask, BF16 pairs
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
        for (int hr = 0; hr < 2; ++hr) {
            const long long v = vbase + warp * 32 + mt * 16 + g + hr * 8;
            if (v >= nvox) continue;
#pragma unroll
            for (int nt = 0; nt < NT; ++nt) {
                const int c = nt * 8 + 2 * t4;
                float y0 = acc[mt][nt][2 * hr], y1 = acc[mt][nt][2 * hr + 1];
                if (bias) {
                    y0 += bias[c];
                    y1 += bias[c + 1];
                }
                if (relu) {
                    y0 = fmaxf(y0, 0.f);
                    y1 = fmaxf(y1, 0.f);
                }
                if (mask) {
                    const __nv_bfloat162 mk =
                        *reinterpret_cast<const __nv_bfloat162*>(mask + (size_t)v * mask_ld + mask_off + c);
                    if (!(__bfloat162float(mk.x) > 0.f)) y0 = 0.f;
                    if (!(__bfloat162float(mk.y) > 0.f)) y1 = 0.f;
                }
                *reinterpret_cast<__nv_bfloat162*>(out + (size_t)v * out_ld + out_off + c) = __floats2bfloat162_rn(y0, y1);
            }
        }
    }
}

// Partial weight gradient of one tap over one chunk of voxels:
// part[chunk][tap][ci][co] = sum_{v in chunk} x[v + tap][ci] dy[v][co].
// CI, CO multiples of 16 (CI <= 96, CO <= 96).  128 threads; a warp owns a set of 16x8
// output tiles.
template <int CI, int CO>
__global__ void __launch_bounds__(128) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ x, int x_ld, int x_off,
                                                     const __nv_bfloat16* __restrict__ dy, int dy_ld, int dy_off,
                                                     int n, int chunk_vox, float* __restrict__ part)
{
    __shared__ __align__(16) __nv_bfloat16 sX[CI * kRowT];
    __shared__ __align__(16) __nv_bfloat16 sD[CO * kRowT];
    const int tap = blockIdx.x, chunk = blockIdx.y;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int nvox = n * n * n;
    constexpr int MT = CI / 16, NT = CO / 8, TILES = MT * NT, PER = (TILES + 3) / 4;
    float acc[PER][4];
#pragma unroll
    for (int i = 0; i < PER; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[i][q] = 0.f;
    const int v0 = chunk * chunk_vox;
    for (int vb = v0; vb < v0 + chunk_vox && vb < nvox; vb += kWgTile) {
        // stage x (shifted by the tap) and dy transposed: channel-major rows of kWgTile voxels
        for (int q = t; q < kWgTile * (CI / 8); q += 128) {
            const int vv = q / (CI / 8), c8 = (q - vv * (CI / 8)) * 8;
            const int v = vb + vv;
            uint4 raw = make_uint4(0, 0, 0, 0);
            if (v < nvox) raw = *reinterpret_cast<const uint4*>(x + (size_t)tap_voxel(v, n, tap) * x_ld + x_off + c8);
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) sX[(c8 + k) * kRowT + vv] = e[k];
        }
        for (int q = t; q < kWgTile * (CO / 8); q += 128) {
            const int vv = q / (CO / 8), c8 = (q - vv * (CO / 8)) * 8;
            const int v = vb + vv;
            uint4 raw = make_uint4(0, 0, 0, 0);
            if (v < nvox) raw = *reinterpret_cast<const uint4*>(dy + (size_t)v * dy_ld + dy_off + c8);
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
            for (int k = 0; k < 8; ++k) sD[(c8 + k) * kRowT + vv] = e[k];
        }
        __syncthreads();
        const unsigned* X32 = reinterpret_cast<const unsigned*>(sX);
        const unsigned* D32 = reinterpret_cast<const unsigned*>(sD);
#pragma unroll
        for (int kk = 0; kk < kWgTile / 16; ++kk) {
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const int tile = warp + 4 * i;
                if (tile >= TILES) continue;
                const int mt = tile / NT, nt = tile - mt * NT;
                const int r0 = mt * 16 + g, c = nt * 8 + g;
                unsigned a[4], b[2];
                a[0] = X32[(r0 * kRowT) / 2 + kk * 8 + t4];
                a[1] = X32[((r0 + 8) * kRowT) / 2 + kk * 8 + t4];
                a[2] = X32[(r0 * kRowT) / 2 + kk * 8 + t4 + 4];
                a[3] = X32[((r0 + 8) * kRowT) / 2 + kk * 8 + t4 + 4];
                b[0] = D32[(c * kRowT) / 2 + kk * 8 + t4];
                b[1] = D32[(c * kRowT) / 2 + kk * 8 + t4 + 4];
                mma_bf16(acc[i], a, b);
            }
        }
        __syncthreads();
    }
    float* dst = part + ((size_t)chunk * 27 + tap) * CI * CO;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
        const int tile = warp + 4 * i;
        if (tile >= TILES) continue;
        const int mt = tile / NT, nt = tile - mt * NT;
        const int r = mt * 16 + g, c = nt * 8 + 2 * t4;
        dst[r * CO + c] = acc[i][0];
        dst[r * CO + c + 1] = acc[i][1];
        dst[(r + 8) * CO + c] = acc[i][2];
        dst[(r + 8) * CO + c + 1] = acc[i][3];
    }
}


// ------------------------------------------------------------------ tiled forward conv
//
// Persistent implicit-GEMM 3x3x3 convolution for grids of at least 16^3.  A block keeps
// the layer's BF16 weights resident in shared memory ([tap][ci/16][N][16], each 32-byte
// row of 16 k with its two 16-byte halves swapped on every other group of four rows, so
// that ldmatrix rows fall on distinct banks) and walks output tiles of 16 x 8 x 2 voxels.
// Per tile and 16-channel chunk it stages the 18 x 10 x 4 input patch (the same half
// swizzle per voxel) by cp.async, then runs all 27 taps without a barrier: each warp owns
// two 16-voxel rows of the tile (M = 16 each) and all N outputs, its A fragments come from
// ldmatrix with per-lane patch addresses (the tap shift is an address offset), B from the
// resident weights.  mma.sync m16n8k16, BF16 inputs, FP32 accumulators.  (A second patch
// buffer, to copy the next tile during the multiplications, was measured slower: it halves
// the resident blocks, which already overlap one another's copies.)

constexpr int kTX = 16, kTY = 8, kTZ = 2;                        // output tile
constexpr int kPX = kTX + 2, kPY = kTY + 2, kPZ = kTZ + 2;       // input patch
constexpr int kPV = kPX * kPY * kPZ;                             // 720 patch voxels

__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], unsigned addr)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}

// byte offset of half h (0: k 0-7, 1: k 8-15) of 32-byte row r
__device__ __forceinline__ unsigned swz_row(int r, int h) { return (unsigned)(r * 32 + ((h ^ ((r >> 2) & 1)) << 4)); }

template <int N>
constexpr size_t conv_tile_smem(int cin)
{
    return (size_t)27 * cin * N * 2 + (size_t)kPV * 32;
}

template <int N>
__global__ void __launch_bounds__(256) k_conv3d_tile(const __nv_bfloat16* __restrict__ in, int in_ld, int in_off,
                                                    int Cin, const __nv_bfloat16* __restrict__ wt,
                                                    const float* __restrict__ bias, __nv_bfloat16* __restrict__ out,
                                                    int out_ld, int out_off, int n, int relu,
                                                    const __nv_bfloat16* __restrict__ mask, int mask_ld, int mask_off)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const int kchunks = Cin / 16;
    unsigned char* sW = sm;                                   // [27 * kchunks * N] rows of 32 B
    unsigned char* sP = sm + (size_t)27 * kchunks * N * 32;   // [kPV] rows of 32 B
    const unsigned sW_s = (unsigned)__cvta_generic_to_shared(sW);
    const unsigned sP_s = (unsigned)__cvta_generic_to_shared(sP);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int g = lane >> 2, t4 = lane & 3;
    const int m = n - 1;
    constexpr int NT = N / 8;

    // resident weights: row q = (tap * kchunks + ch) * N + co, 16 k each
    const int wrows = 27 * kchunks * N;
    for (int q = t; q < wrows * 2; q += 256) {
        const int r = q >> 1, h = q & 1;
        const unsigned d = sW_s + swz_row(r, h);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(wt + (size_t)r * 16 + h * 8));
    }
    cp_async_commit();

    // lane roles in ldmatrix: A rows (voxels) and k halves; B rows (outputs) and k halves
    const int mi = lane >> 3, rr = lane & 7;
    const int a_row = rr + 8 * (mi & 1), a_h = mi >> 1;
    const int b_row = rr + 8 * (mi >> 1), b_h = mi & 1;
    // this warp's two M rows of the tile: (y, z) = (mt & 7, mt >> 3), x = 0..15
    const int mt0 = 2 * warp, mt1 = 2 * warp + 1;
    const int prow0 = ((mt0 >> 3) * kPY + (mt0 & 7)) * kPX;
    const int prow1 = ((mt1 >> 3) * kPY + (mt1 & 7)) * kPX;

    const int tx = n / kTX, ty = n / kTY, tz = n / kTZ;
    const long long tiles = (long long)tx * ty * tz;
    for (long long tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int bx = (int)(tile % tx), by = (int)((tile / tx) % ty), bz = (int)(tile / ((long long)tx * ty));
        const int x0 = bx * kTX, y0 = by * kTY, z0 = bz * kTZ;
        float acc[2][NT][4];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int j = 0; j < NT; ++j)
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;
        for (int ch = 0; ch < kchunks; ++ch) {
            // the patch of this chunk: voxel p = (pz * kPY + py) * kPX + px, two 16-byte halves
            for (int q = t; q < kPV * 2; q += 256) {
                const int p = q >> 1, h = q & 1;
                const int px = p % kPX, py = (p / kPX) % kPY, pz = p / (kPX * kPY);
                const int gx = (x0 - 1 + px) & m, gy = (y0 - 1 + py) & m, gz = (z0 - 1 + pz) & m;
                const __nv_bfloat16* src = in + ((size_t)(gz * n + gy) * n + gx) * in_ld + in_off + ch * 16 + h * 8;
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sP_s + swz_row(p, h)), "l"(src));
            }
            cp_async_commit();
            cp_async_wait<0>();
            __syncthreads();
#pragma unroll 1
            for (int tap = 0; tap < 27; ++tap) {
                const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;  // patch offsets 0..2
                const int sh = (dz * kPY + dy) * kPX + dx;
                unsigned a0[4], a1[4];
                ldsm_x4(a0, sP_s + swz_row(prow0 + sh + a_row, a_h));
                ldsm_x4(a1, sP_s + swz_row(prow1 + sh + a_row, a_h));
                const int wbase = (tap * kchunks + ch) * N;
#pragma unroll
                for (int j = 0; j < NT; j += 2) {
                    unsigned b[4];
                    ldsm_x4(b, sW_s + swz_row(wbase + 8 * j + b_row, b_h));
                    const unsigned b0[2] = {b[0], b[1]}, b1[2] = {b[2], b[3]};
                    mma_bf16(acc[0][j], a0, b0);
                    mma_bf16(acc[1][j], a1, b0);
                    mma_bf16(acc[0][j + 1], a0, b1);
                    mma_bf16(acc[1][j + 1], a1, b1);
                }
            }
            __syncthreads();  // the patch is refilled next
        }
        // epilogue: bias, activation, optional mask, BF16 pairs
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int mt = 2 * warp + i;
            const int y = y0 + (mt & 7), z = z0 + (mt >> 3);
#pragma unroll
            for (int hr = 0; hr < 2; ++hr) {
                const int x = x0 + g + 8 * hr;
                const size_t v = ((size_t)z * n + y) * n + x;
#pragma unroll
                for (int j = 0; j < NT; ++j) {
                    const int c = j * 8 + 2 * t4;
                    float y0v = acc[i][j][2 * hr], y1v = acc[i][j][2 * hr + 1];
                    if (bias) {
                        y0v += bias[c];
                        y1v += bias[c + 1];
                    }
                    if (relu) {
                        y0v = fmaxf(y0v, 0.f);
                        y1v = fmaxf(y1v, 0.f);
                    }
                    if (mask) {
                        const __nv_bfloat162 mk =
                            *reinterpret_cast<const __nv_bfloat162*>(mask + v * mask_ld + mask_off + c);
                        if (!(__bfloat162float(mk.x) > 0.f)) y0v = 0.f;
                        if (!(__bfloat162float(mk.y) > 0.f)) y1v = 0.f;
                    }
                    *reinterpret_cast<__nv_bfloat162*>(out + v * out_ld + out_off + c) = __floats2bfloat162_rn(y0v, y1v);
                }
            }
        }
    }
    cp_async_wait<0>();
}

}  // namespace pmeft
