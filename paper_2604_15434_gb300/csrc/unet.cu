// unet.cu -- learned warm start for the chi solve: a small periodic 3D U-Net on BF16 tensor
// cores, its training step, and the warm-start initial guess.
//
// The network maps (asinh delta, alpha_B0, alpha_M0, a) to the "screened source"
// T = nu L(chi) / src, which equals delta where screening is off (linear limit).  The
// warm start is chi_0 = (src / nu) L^-1 T_hat, one FFT Poisson solve: the network only has
// to learn the local effect of screening, the potential's long range comes from the FFT.
//
// Architecture (3 levels, 3x3x3 periodic convolutions, ReLU, channels 16/32/64):
//   c0 16->16, c1 16->16 -> [cat1 32:48]          (level n; input padded to 16 channels)
//   pool -> c2 16->32, c3 32->32 -> [cat2 64:96]   (n/2)
//   pool -> c4 32->64, c5 64->64                   (n/4)
//   up -> [cat2 0:64], c6 96->32, c7 32->32        (n/2)
//   up -> [cat1 0:32], c8 48->16, c9 16->16        (n)
//   head 1x1x1 16->1 (linear) -> T_hat
// Parameters (FP32 master copy, flat): per conv W[tap][ci][co] then b[co]; head w[16], b.
#include <algorithm>
#include <cmath>
#include <vector>

#include "conv.cuh"
#include "conv_umma.cuh"
#include "internal.cuh"

struct pm_unet;

namespace pmeft {

struct ConvSpec {
    int ci, co, level;
};
static const ConvSpec kConvs[10] = {{16, 16, 0}, {16, 16, 0}, {16, 32, 1}, {32, 32, 1}, {32, 64, 2},
                                    {64, 64, 2}, {96, 32, 1}, {32, 32, 1}, {48, 16, 0}, {16, 16, 0}};

static long long conv_params(int i) { return 27LL * kConvs[i].ci * kConvs[i].co + kConvs[i].co; }
static long long total_params()
{
    long long s = 17;  // head
    for (int i = 0; i < 10; ++i) s += conv_params(i);
    return s;
}

// ---------------------------------------------------------------- small kernels

__global__ void k_pack_input(const double* __restrict__ delta, int nvox, float p1, float p2, float p3,
                             __nv_bfloat16* __restrict__ out)
{
    // the network sees asinh(delta) in BF16: FP32 asinh is far below that rounding
    const __nv_bfloat16 b1 = __float2bfloat16(p1), b2 = __float2bfloat16(p2), b3 = __float2bfloat16(p3);
    const __nv_bfloat16 z = __float2bfloat16(0.f);
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += gridDim.x * blockDim.x) {
        __align__(16) __nv_bfloat16 o[8] = {__float2bfloat16(asinhf((float)delta[v])), b1, b2, b3, z, z, z, z};
        uint4* dst = reinterpret_cast<uint4*>(out + (size_t)v * 16);
        dst[0] = *reinterpret_cast<const uint4*>(o);
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// out (n/2 grid, C channels) = average of the 8 children of in (slice ld/off)
__global__ void k_pool2(const __nv_bfloat16* __restrict__ in, int ld, int off, int C, int n, __nv_bfloat16* __restrict__ out)
{
    // one thread per (coarse voxel, group of 8 channels); n is a power of two, C, ld and
    // off multiples of 8 (16-byte accesses)
    const int nc = n / 2, lgc = __ffs(nc) - 1, G = C / 8, total = nc * nc * nc * G;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int cg = q % G, v = q / G;
        const int X = v & (nc - 1), Y = (v >> lgc) & (nc - 1), Z = v >> (2 * lgc);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int f = ((2 * Z + (k >> 2)) * n + (2 * Y + ((k >> 1) & 1))) * n + (2 * X + (k & 1));
            const uint4 raw = *reinterpret_cast<const uint4*>(in + (size_t)f * ld + off + cg * 8);
            const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
            for (int c = 0; c < 8; ++c) s[c] += __bfloat162float(e[c]);
        }
        __align__(16) __nv_bfloat16 o[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) o[c] = __float2bfloat16(0.125f * s[c]);
        *reinterpret_cast<uint4*>(out + (size_t)v * C + cg * 8) = *reinterpret_cast<const uint4*>(o);
    }
}

// d_in[child][off + c] += mask(child) * d_out[parent][c] / 8  (backward of k_pool2)
__global__ void k_pool2_bwd_add(const __nv_bfloat16* __restrict__ dout, int C, int n, __nv_bfloat16* __restrict__ din,
                                int ld, int off, const __nv_bfloat16* __restrict__ mask)
{
    const long long total = (long long)n * n * n * C;  // 2^31 at 512^3 x 16 channels
    const int nc = n / 2;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(q % C), v = (int)(q / C);
        const int x = v % n, y = (v / n) % n, z = v / (n * n);
        const int p = ((z >> 1) * nc + (y >> 1)) * nc + (x >> 1);
        const size_t idx = (size_t)v * ld + off + c;
        float g = 0.125f * __bfloat162float(dout[(size_t)p * C + c]);
        if (!(__bfloat162float(mask[idx]) > 0.f)) g = 0.f;
        din[idx] = __float2bfloat16(__bfloat162float(din[idx]) + g);
    }
}

// out[child][off + c] = in[parent][c]  (nearest upsampling into a channel slice)
__global__ void k_up2(const __nv_bfloat16* __restrict__ in, int C, int nc, __nv_bfloat16* __restrict__ out, int ld, int off)
{
    // one thread per (fine voxel, group of 8 channels), 16-byte copies; the count stays
    // below 2^31 up to 512^3 x 64 channels
    const int n = 2 * nc, lg = __ffs(n) - 1, G = C / 8, total = n * n * n * G;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int cg = q % G, v = q / G;
        const int x = v & (n - 1), y = (v >> lg) & (n - 1), z = v >> (2 * lg);
        const size_t pv = (size_t)(((z >> 1) * nc + (y >> 1)) * nc + (x >> 1));
        *reinterpret_cast<uint4*>(out + (size_t)v * ld + off + cg * 8) =
            *reinterpret_cast<const uint4*>(in + pv * C + cg * 8);
    }
}

// d_in[parent][c] = sum of d_out over the 8 children (backward of k_up2)
__global__ void k_up2_bwd(const __nv_bfloat16* __restrict__ dout, int ld, int off, int C, int nc,
                          __nv_bfloat16* __restrict__ din)
{
    const int n = 2 * nc, total = nc * nc * nc * C;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int c = q % C, v = q / C;
        const int X = v % nc, Y = (v / nc) % nc, Z = v / (nc * nc);
        float s = 0.f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int f = ((2 * Z + (k >> 2)) * n + (2 * Y + ((k >> 1) & 1))) * n + (2 * X + (k & 1));
            s += __bfloat162float(dout[(size_t)f * ld + off + c]);
        }
        din[(size_t)v * C + c] = __float2bfloat16(s);
    }
}

// T_hat[v] = sum_c w[c] y[v][c] + b
__global__ void k_head(const __nv_bfloat16* __restrict__ y, const float* __restrict__ w, int nvox, double* __restrict__ out)
{
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += gridDim.x * blockDim.x) {
        const uint4* src = reinterpret_cast<const uint4*>(y + (size_t)v * 16);
        const uint4 r0 = src[0], r1 = src[1];
        const __nv_bfloat16* e0 = reinterpret_cast<const __nv_bfloat16*>(&r0);
        const __nv_bfloat16* e1 = reinterpret_cast<const __nv_bfloat16*>(&r1);
        float s = w[16];
#pragma unroll
        for (int c = 0; c < 8; ++c) s += w[c] * __bfloat162float(e0[c]);
#pragma unroll
        for (int c = 0; c < 8; ++c) s += w[8 + c] * __bfloat162float(e1[c]);
        out[v] = (double)s;
    }
}

// loss partials and the head's backward: g = 2 (T_hat - T) / V; dy[v][c] = g w[c] (masked by
// relu'(y)); per-block partials of sum g^2-style loss, sum_v g y[v][c] and sum_v g
__global__ void k_head_bwd(const double* __restrict__ that, const float* __restrict__ target,
                           const __nv_bfloat16* __restrict__ y, const float* __restrict__ w, int nvox,
                           __nv_bfloat16* __restrict__ dy, double* __restrict__ partials)
{
    double acc[19];
#pragma unroll
    for (int q = 0; q < 19; ++q) acc[q] = 0.0;
    const double inv = 1.0 / (double)nvox;
    for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += gridDim.x * blockDim.x) {
        const double d = that[v] - (double)target[v];
        const float g = (float)(2.0 * d * inv);
        acc[0] += d * d * inv;
#pragma unroll
        for (int c = 0; c < 16; ++c) {
            const float yc = __bfloat162float(y[(size_t)v * 16 + c]);
            acc[1 + c] += (double)(g * yc);
            dy[(size_t)v * 16 + c] = __float2bfloat16(yc > 0.f ? g * w[c] : 0.f);
        }
        acc[17] += (double)g;
    }
    __shared__ double sh[19][256];
#pragma unroll
    for (int q = 0; q < 19; ++q) sh[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s)
            for (int q = 0; q < 19; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int q = 0; q < 19; ++q) partials[(size_t)blockIdx.x * 19 + q] = sh[q][0];
}

// bias gradient partials: per block, sum over its voxels of dy[v][c] for every channel
__global__ void k_bias_grad(const __nv_bfloat16* __restrict__ dy, int ld, int off, int C, int nvox,
                            float* __restrict__ partials)
{
    __shared__ float sh[256];
    for (int c = 0; c < C; ++c) {
        float s = 0.f;
        for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < nvox; v += gridDim.x * blockDim.x)
            s += __bfloat162float(dy[(size_t)v * ld + off + c]);
        sh[threadIdx.x] = s;
        __syncthreads();
        for (int w = blockDim.x / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) partials[(size_t)blockIdx.x * C + c] = sh[0];
        __syncthreads();
    }
}

// grad[i] += sum over blocks of partials[b][i] (fixed order)
__global__ void k_reduce_add(const float* __restrict__ partials, int nblocks, int count, float* __restrict__ grad)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        float s = 0.f;
        for (int b = 0; b < nblocks; ++b) s += partials[(size_t)b * count + i];
        grad[i] += s;
    }
}

// Adam on the flat FP32 parameters, then zero the gradient accumulator
__global__ void k_adam(float* __restrict__ p, float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long count, float lr, float b1, float b2, float eps, float c1, float c2)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
        g[i] = 0.f;
    }
}

// pack W[tap][ci][co] into the forward layout [tap][ci/16][co][16] and the backward-data
// layout (taps flipped, channels swapped) [tap'][co/16][ci][16], both BF16
__global__ void k_pack_weights(const float* __restrict__ W, int ci, int co, __nv_bfloat16* __restrict__ fwd,
                               __nv_bfloat16* __restrict__ bwd)
{
    const int total = 27 * ci * co;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const int o = q % co, i = (q / co) % ci, t = q / (ci * co);
        const __nv_bfloat16 w = __float2bfloat16(W[q]);
        fwd[(((size_t)t * (ci / 16) + i / 16) * co + o) * 16 + (i & 15)] = w;
        const int tp = 26 - t;
        bwd[(((size_t)tp * (co / 16) + o / 16) * ci + i) * 16 + (o & 15)] = w;
    }
}

// T = nu L(chi) / src with the 7-point Laplacian (training target from a solved chi)
__global__ void k_target(const double* __restrict__ chi, int n, double scale, float* __restrict__ T)
{
    const int m = n - 1;
    const size_t total = (size_t)n * n * n;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((size_t)n * n));
        auto at = [&](int i, int j, int k) { return chi[((size_t)(k & m) * n + (j & m)) * n + (i & m)]; };
        const double L = at(x + 1, y, z) + at(x - 1, y, z) + at(x, y + 1, z) + at(x, y - 1, z) + at(x, y, z + 1) +
                         at(x, y, z - 1) - 6.0 * chi[c];
        T[c] = (float)(L * scale);
    }
}

// ---------------------------------------------------------------- network state

struct Acts {
    int n = 0;
    __nv_bfloat16 *in = nullptr, *y0 = nullptr, *cat1 = nullptr, *p1 = nullptr, *y2 = nullptr, *cat2 = nullptr,
                  *p2 = nullptr, *y4 = nullptr, *y5 = nullptr, *y6 = nullptr, *y7 = nullptr, *y8 = nullptr,
                  *y9 = nullptr;
    // gradients (training)
    __nv_bfloat16 *d9 = nullptr, *d8 = nullptr, *dcat1 = nullptr, *d7 = nullptr, *d6 = nullptr, *dcat2 = nullptr,
                  *d5 = nullptr, *d4 = nullptr, *dp2 = nullptr, *d2 = nullptr, *dp1 = nullptr, *d0 = nullptr;
    double* that = nullptr;
    float* part = nullptr;  // weight-gradient partials
    size_t part_count = 0;
    double* lpart = nullptr;
    bool train = false;
};

}  // namespace pmeft

struct pm_unet {
    pm_ctx* ctx = nullptr;
    long long np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // flat FP32
    __nv_bfloat16* wf[10] = {};
    __nv_bfloat16* wb[10] = {};
    long long off[11] = {};  // parameter offsets of each conv and of the head
    pmeft::Acts acts;
    int adam_t = 0;
    int conv_path = 1;  // 0 mma.sync, 1 tcgen05 convolutions (pm_unet_set_conv_path)
};

namespace pmeft {

template <typename T>
static pm_status dalloc(pm_ctx* ctx, T** p, size_t count)
{
    PM_CUDA(cudaMalloc(p, count * sizeof(T)));
    return PM_OK;
}

static void free_acts(Acts& a)
{
    __nv_bfloat16** bufs[] = {&a.in, &a.y0, &a.cat1, &a.p1, &a.y2, &a.cat2, &a.p2, &a.y4, &a.y5, &a.y6, &a.y7, &a.y8,
                              &a.y9, &a.d9, &a.d8, &a.dcat1, &a.d7, &a.d6, &a.dcat2, &a.d5, &a.d4, &a.dp2, &a.d2,
                              &a.dp1, &a.d0};
    for (auto b : bufs) {
        cudaFree(*b);
        *b = nullptr;
    }
    cudaFree(a.that);
    cudaFree(a.part);
    cudaFree(a.lpart);
    a = Acts();
}

static pm_status ensure_acts(pm_unet* u, int n, bool train)
{
    pm_ctx* ctx = u->ctx;
    Acts& a = u->acts;
    if (a.n == n && (a.train || !train)) return PM_OK;
    free_acts(a);
    const size_t v0 = (size_t)n * n * n, v1 = v0 / 8, v2 = v0 / 64;
    PM_TRY(dalloc(ctx, &a.in, v0 * 16));
    PM_TRY(dalloc(ctx, &a.y0, v0 * 16));
    PM_TRY(dalloc(ctx, &a.cat1, v0 * 48));
    PM_TRY(dalloc(ctx, &a.p1, v1 * 16));
    PM_TRY(dalloc(ctx, &a.y2, v1 * 32));
    PM_TRY(dalloc(ctx, &a.cat2, v1 * 96));
    PM_TRY(dalloc(ctx, &a.p2, v2 * 32));
    PM_TRY(dalloc(ctx, &a.y4, v2 * 64));
    PM_TRY(dalloc(ctx, &a.y5, v2 * 64));
    PM_TRY(dalloc(ctx, &a.y6, v1 * 32));
    PM_TRY(dalloc(ctx, &a.y7, v1 * 32));
    PM_TRY(dalloc(ctx, &a.y8, v0 * 16));
    PM_TRY(dalloc(ctx, &a.y9, v0 * 16));
    PM_TRY(dalloc(ctx, &a.that, v0));
    PM_TRY(dalloc(ctx, &a.lpart, (size_t)kMaxPartials * 19));
    if (train) {
        PM_TRY(dalloc(ctx, &a.d9, v0 * 16));
        PM_TRY(dalloc(ctx, &a.d8, v0 * 16));
        PM_TRY(dalloc(ctx, &a.dcat1, v0 * 48));
        PM_TRY(dalloc(ctx, &a.d7, v1 * 32));
        PM_TRY(dalloc(ctx, &a.d6, v1 * 32));
        PM_TRY(dalloc(ctx, &a.dcat2, v1 * 96));
        PM_TRY(dalloc(ctx, &a.d5, v2 * 64));
        PM_TRY(dalloc(ctx, &a.d4, v2 * 64));
        PM_TRY(dalloc(ctx, &a.dp2, v2 * 32));
        PM_TRY(dalloc(ctx, &a.d2, v1 * 32));
        PM_TRY(dalloc(ctx, &a.dp1, v1 * 16));
        PM_TRY(dalloc(ctx, &a.d0, v0 * 16));
        // largest partial buffer: chunks * 27 * ci * co over the convs
        size_t mx = 0;
        for (int i = 0; i < 10; ++i) {
            const size_t nv = (size_t)(n >> kConvs[i].level) * (n >> kConvs[i].level) * (n >> kConvs[i].level);
            const size_t chunks = (nv + 8191) / 8192;
            mx = std::max(mx, chunks * 27 * kConvs[i].ci * kConvs[i].co);
        }
        mx = std::max(mx, (size_t)kMaxPartials * 96);
        a.part_count = mx;
        PM_TRY(dalloc(ctx, &a.part, mx));
    }
    a.n = n;
    a.train = train;
    return PM_OK;
}

static int blocks_for(pm_ctx* ctx, size_t work) { return grid_for(ctx, work); }

// The convolution on the tcgen05 tensor cores (conv_umma.cuh), in slices of NT output channels
// whose resident weights fit next to the patch planes in shared memory.  Returns false (nothing
// launched) where it does not apply.
template <int NT, int SLOTS>
static void launch_umma(pm_ctx* ctx, const __nv_bfloat16* in, int in_ld, int in_off, int ci, const __nv_bfloat16* w,
                        int co, int co0, const float* bias, __nv_bfloat16* out, int out_ld, int out_off, int n, bool relu,
                        const __nv_bfloat16* mask, int mask_ld, int mask_off)
{
    const size_t smem = umma_smem<NT, SLOTS>(ci);
    auto k = k_conv3d_umma<NT, SLOTS>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // blocks per SM from the kernel's own limits: shared memory (plus the 1 KB the system
    // reserves per block), registers, threads, and the SM's 512 tensor-memory columns
    int smem_sm = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, ctx->device);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, ctx->device);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k);
    constexpr int cols = (int)um_cols<NT>();
    int per_sm = std::min(smem_sm / (int)(smem + 1024), 2048 / kUmThreads);
    if (fa.numRegs > 0) per_sm = std::min(per_sm, regs_sm / (fa.numRegs * kUmThreads));
    per_sm = std::max(1, std::min(per_sm, 512 / cols));
    // z planes per work item: n / 8 within [4, 64] (a divisor of n), enough items for every SM
    const int zl = std::max(4, std::min(64, n / 8));
    const long long items = (long long)(n / kUmTX) * (n / kUmTY) * (n / zl);
    const long long g = std::min<long long>(items, (long long)ctx->num_sms * per_sm);
    k<<<(int)g, kUmThreads, smem, ctx->stream>>>(in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, zl,
                                                  relu ? 1 : 0, mask, mask_ld, mask_off, ctx->flag + 2);
}

// three plane slots (two planes loading ahead) where the block still fits twice per SM, else two
template <int NT>
static void launch_umma_slots(pm_ctx* ctx, const __nv_bfloat16* in, int in_ld, int in_off, int ci,
                              const __nv_bfloat16* w, int co, int co0, const float* bias, __nv_bfloat16* out,
                              int out_ld, int out_off, int n, bool relu, const __nv_bfloat16* mask, int mask_ld,
                              int mask_off)
{
    if (umma_smem<NT, 3>(ci) <= (size_t)112 * 1024)
        launch_umma<NT, 3>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld,
                           mask_off);
    else
        launch_umma<NT, 2>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld,
                           mask_off);
}

static bool conv_umma(pm_ctx* ctx, const __nv_bfloat16* in, int in_ld, int in_off, int ci, const __nv_bfloat16* w,
                      int co, const float* bias, __nv_bfloat16* out, int out_ld, int out_off, int n, bool relu,
                      const __nv_bfloat16* mask, int mask_ld, int mask_off)
{
    if (ctx->conv_path != 1 || n < kUmTY || n % kUmTY != 0 || ci % 16 != 0 || co % 16 != 0) return false;
    auto bytes = [&](int nt) {  // umma_smem<nt, 2>(ci)
        return (size_t)9 * (ci / 16) * 2 * kUmWGroups * nt * 16 + (size_t)2 * (ci / 16) * kUmPP * 32 + 32 + (size_t)nt * 4;
    };
    int nt = co;  // the widest slice (at most 64 outputs) whose weights fit
    while ((nt > 64 || bytes(nt) > (size_t)227 * 1024) && nt % 32 == 0) nt /= 2;
    if (nt > 64 || bytes(nt) > (size_t)227 * 1024) return false;
    for (int co0 = 0; co0 < co; co0 += nt) {
        switch (nt) {
            case 16: launch_umma_slots<16>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld, mask_off); break;
            case 32: launch_umma_slots<32>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld, mask_off); break;
            case 48: launch_umma_slots<48>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld, mask_off); break;
            case 64: launch_umma_slots<64>(ctx, in, in_ld, in_off, ci, w, co, co0, bias, out, out_ld, out_off, n, relu, mask, mask_ld, mask_off); break;
            default: return false;
        }
    }
    return true;
}

// forward conv launcher (also the backward-data conv with a mask)
static void conv_fwd(pm_ctx* ctx, const __nv_bfloat16* in, int in_ld, int in_off, int ci, const __nv_bfloat16* w,
                     int co, const float* bias, __nv_bfloat16* out, int out_ld, int out_off, int n, bool relu,
                     const __nv_bfloat16* mask = nullptr, int mask_ld = 0, int mask_off = 0)
{
    const int nvox = n * n * n, grid = (nvox + kConvM - 1) / kConvM;
    ctx->begin(PM_K_PM);
    if (conv_umma(ctx, in, in_ld, in_off, ci, w, co, bias, out, out_ld, out_off, n, relu, mask, mask_ld, mask_off)) {
        ctx->end();
        return;
    }
    // grids of 16^3 and up whose weights fit next to the patch in shared memory take the
    // persistent tiled kernel, the rest the per-128-voxel kernel
    bool tiled = false;
    if (n >= kTX && n % kTX == 0) {
        int dev = 0, sms = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        const long long tiles = (long long)(n / kTX) * (n / kTY) * (n / kTZ);
#define PM_TILE_CASE(N_)                                                                                          \
    case N_: {                                                                                                    \
        const size_t smem = conv_tile_smem<N_>(ci);                                                               \
        if (smem <= 227 * 1024) {                                                                                 \
            auto k = k_conv3d_tile<N_>;                                                                           \
            cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);                      \
            int per_sm = 0;                                                                                       \
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);                                 \
            const long long g = std::min<long long>(tiles, (long long)sms * std::max(per_sm, 1));                 \
            k<<<(int)g, 256, smem, ctx->stream>>>(in, in_ld, in_off, ci, w, bias, out, out_ld, out_off, n,        \
                                                 relu ? 1 : 0, mask, mask_ld, mask_off);                          \
            tiled = true;                                                                                         \
        }                                                                                                         \
        break;                                                                                                    \
    }
        switch (co) {
            PM_TILE_CASE(16)
            PM_TILE_CASE(32)
            PM_TILE_CASE(48)
            PM_TILE_CASE(64)
            PM_TILE_CASE(96)
        }
#undef PM_TILE_CASE
    }
    if (!tiled) {
#define PM_CONV_CASE(N_)                                                                                           \
    case N_:                                                                                                       \
        k_conv3d_fwd<N_><<<grid, 128, 0, ctx->stream>>>(in, in_ld, in_off, ci, w, bias, out, out_ld, out_off, n,    \
                                                        relu ? 1 : 0, mask, mask_ld, mask_off);                    \
        break;
        switch (co) {
            PM_CONV_CASE(16)
            PM_CONV_CASE(32)
            PM_CONV_CASE(48)
            PM_CONV_CASE(64)
            PM_CONV_CASE(96)
        }
#undef PM_CONV_CASE
    }
    ctx->end();
}

// weight gradient of conv i: grad[off .. off + 27 ci co) += sum over voxels; then the bias
static void conv_wgrad(pm_unet* u, int i, const __nv_bfloat16* x, int x_ld, int x_off, const __nv_bfloat16* dy,
                       int dy_ld, int dy_off, int n)
{
    pm_ctx* ctx = u->ctx;
    const int ci = kConvs[i].ci, co = kConvs[i].co;
    const int nvox = n * n * n;
    const int chunk = 8192, chunks = (nvox + chunk - 1) / chunk;
    const dim3 grid(27, chunks);
    ctx->begin(PM_K_PM);
#define PM_WG_CASE(CI_, CO_)                                                                                        \
    if (ci == CI_ && co == CO_)                                                                                     \
        k_conv3d_wgrad<CI_, CO_><<<grid, 128, 0, ctx->stream>>>(x, x_ld, x_off, dy, dy_ld, dy_off, n, chunk, u->acts.part);
    PM_WG_CASE(16, 16)
    PM_WG_CASE(16, 32)
    PM_WG_CASE(32, 32)
    PM_WG_CASE(32, 64)
    PM_WG_CASE(64, 64)
    PM_WG_CASE(96, 32)
    PM_WG_CASE(48, 16)
#undef PM_WG_CASE
    ctx->end();
    const int count = 27 * ci * co;
    ctx->begin(PM_K_PM);
    k_reduce_add<<<blocks_for(ctx, count), 256, 0, ctx->stream>>>(u->acts.part, chunks, count, u->g + u->off[i]);
    ctx->end();
    const int bb = std::min(blocks_for(ctx, nvox), kMaxPartials);
    ctx->begin(PM_K_PM);
    k_bias_grad<<<bb, 256, 0, ctx->stream>>>(dy, dy_ld, dy_off, co, nvox, u->acts.part);
    ctx->end();
    ctx->begin(PM_K_PM);
    k_reduce_add<<<1, 256, 0, ctx->stream>>>(u->acts.part, bb, co, u->g + u->off[i] + 27LL * ci * co);
    ctx->end();
}

static const float* bias_of(pm_unet* u, int i)
{
    return u->p + u->off[i] + 27LL * kConvs[i].ci * kConvs[i].co;
}

// After a pass with the tcgen05 convolutions: PM_ERR_TIMEOUT if an accumulator wait of
// k_conv3d_umma gave up (its error word is cleared for the next pass), else PM_OK.
static pm_status umma_status(pm_ctx* ctx)
{
    if (ctx->conv_path != 1) return PM_OK;
    PM_CUDA(cudaMemcpyAsync(ctx->host_out + 62, ctx->flag + 2, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (*reinterpret_cast<int*>(ctx->host_out + 62) != 0) {
        cudaMemsetAsync(ctx->flag + 2, 0, sizeof(int), ctx->stream);
        ctx->set_error("tensor-core convolution: an accumulator wait gave up");
        return PM_ERR_TIMEOUT;
    }
    return PM_OK;
}

static pm_status unet_forward(pm_unet* u, const double* delta, int n, double aB0, double aM0, double a)
{
    pm_ctx* ctx = u->ctx;
    ctx->conv_path = u->conv_path;  // the convolution launcher reads it from the context
    Acts& A = u->acts;
    const int n1 = n / 2, n2 = n / 4;
    const size_t v0 = (size_t)n * n * n;
    ctx->begin(PM_K_PM);
    k_pack_input<<<blocks_for(ctx, v0), 256, 0, ctx->stream>>>(delta, (int)v0, (float)aB0, (float)aM0, (float)a, A.in);
    ctx->end();
    conv_fwd(ctx, A.in, 16, 0, 16, u->wf[0], 16, bias_of(u, 0), A.y0, 16, 0, n, true);
    conv_fwd(ctx, A.y0, 16, 0, 16, u->wf[1], 16, bias_of(u, 1), A.cat1, 48, 32, n, true);
    ctx->begin(PM_K_PM);
    k_pool2<<<blocks_for(ctx, v0 / 8 * 16), 256, 0, ctx->stream>>>(A.cat1, 48, 32, 16, n, A.p1);
    ctx->end();
    conv_fwd(ctx, A.p1, 16, 0, 16, u->wf[2], 32, bias_of(u, 2), A.y2, 32, 0, n1, true);
    conv_fwd(ctx, A.y2, 32, 0, 32, u->wf[3], 32, bias_of(u, 3), A.cat2, 96, 64, n1, true);
    ctx->begin(PM_K_PM);
    k_pool2<<<blocks_for(ctx, v0 / 64 * 32), 256, 0, ctx->stream>>>(A.cat2, 96, 64, 32, n1, A.p2);
    ctx->end();
    conv_fwd(ctx, A.p2, 32, 0, 32, u->wf[4], 64, bias_of(u, 4), A.y4, 64, 0, n2, true);
    conv_fwd(ctx, A.y4, 64, 0, 64, u->wf[5], 64, bias_of(u, 5), A.y5, 64, 0, n2, true);
    ctx->begin(PM_K_PM);
    k_up2<<<blocks_for(ctx, v0 / 8 * 64), 256, 0, ctx->stream>>>(A.y5, 64, n2, A.cat2, 96, 0);
    ctx->end();
    conv_fwd(ctx, A.cat2, 96, 0, 96, u->wf[6], 32, bias_of(u, 6), A.y6, 32, 0, n1, true);
    conv_fwd(ctx, A.y6, 32, 0, 32, u->wf[7], 32, bias_of(u, 7), A.y7, 32, 0, n1, true);
    ctx->begin(PM_K_PM);
    k_up2<<<blocks_for(ctx, v0 * 32), 256, 0, ctx->stream>>>(A.y7, 32, n1, A.cat1, 48, 0);
    ctx->end();
    conv_fwd(ctx, A.cat1, 48, 0, 48, u->wf[8], 16, bias_of(u, 8), A.y8, 16, 0, n, true);
    conv_fwd(ctx, A.y8, 16, 0, 16, u->wf[9], 16, bias_of(u, 9), A.y9, 16, 0, n, true);
    ctx->begin(PM_K_PM);
    k_head<<<blocks_for(ctx, v0), 256, 0, ctx->stream>>>(A.y9, u->p + u->off[10], (int)v0, A.that);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return umma_status(ctx);
}

// backward of the loss 1/V sum (T_hat - T)^2 into u->g (accumulated); returns the loss
static pm_status unet_backward(pm_unet* u, const float* target, int n, double* loss)
{
    pm_ctx* ctx = u->ctx;
    Acts& A = u->acts;
    const int n1 = n / 2, n2 = n / 4;
    const size_t v0 = (size_t)n * n * n, v1 = v0 / 8, v2 = v0 / 64;
    const int bb = std::min(blocks_for(ctx, v0), kMaxPartials);
    ctx->begin(PM_K_PM);
    k_head_bwd<<<bb, 256, 0, ctx->stream>>>(A.that, target, A.y9, u->p + u->off[10], (int)v0, A.d9, A.lpart);
    ctx->end();
    // head gradients and the loss: sum the block partials on the host (19 x bb doubles)
    std::vector<double> hp((size_t)bb * 19);
    PM_CUDA(cudaMemcpyAsync(hp.data(), A.lpart, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    double s[19] = {};
    for (int b = 0; b < bb; ++b)
        for (int q = 0; q < 19; ++q) s[q] += hp[(size_t)b * 19 + q];
    *loss = s[0];
    float hg[17];
    for (int c = 0; c < 16; ++c) hg[c] = (float)s[1 + c];
    hg[16] = (float)s[17];
    std::vector<float> cur(17);
    PM_CUDA(cudaMemcpy(cur.data(), u->g + u->off[10], 17 * sizeof(float), cudaMemcpyDeviceToHost));
    for (int c = 0; c < 17; ++c) cur[c] += hg[c];
    PM_CUDA(cudaMemcpyAsync(u->g + u->off[10], cur.data(), 17 * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    // c9: x = y8, dy = d9
    conv_wgrad(u, 9, A.y8, 16, 0, A.d9, 16, 0, n);
    conv_fwd(ctx, A.d9, 16, 0, 16, u->wb[9], 16, nullptr, A.d8, 16, 0, n, false, A.y8, 16, 0);
    // c8: x = cat1, dy = d8 -> dcat1 (masked by cat1 > 0)
    conv_wgrad(u, 8, A.cat1, 48, 0, A.d8, 16, 0, n);
    conv_fwd(ctx, A.d8, 16, 0, 16, u->wb[8], 48, nullptr, A.dcat1, 48, 0, n, false, A.cat1, 48, 0);
    // up1 backward: d7 = sum of children of dcat1[0:32]
    ctx->begin(PM_K_PM);
    k_up2_bwd<<<blocks_for(ctx, v1 * 32), 256, 0, ctx->stream>>>(A.dcat1, 48, 0, 32, n1, A.d7);
    ctx->end();
    // c7: x = y6, dy = d7
    conv_wgrad(u, 7, A.y6, 32, 0, A.d7, 32, 0, n1);
    conv_fwd(ctx, A.d7, 32, 0, 32, u->wb[7], 32, nullptr, A.d6, 32, 0, n1, false, A.y6, 32, 0);
    // c6: x = cat2, dy = d6 -> dcat2 (masked by cat2 > 0)
    conv_wgrad(u, 6, A.cat2, 96, 0, A.d6, 32, 0, n1);
    conv_fwd(ctx, A.d6, 32, 0, 32, u->wb[6], 96, nullptr, A.dcat2, 96, 0, n1, false, A.cat2, 96, 0);
    // up2 backward: d5 = sum of children of dcat2[0:64]
    ctx->begin(PM_K_PM);
    k_up2_bwd<<<blocks_for(ctx, v2 * 64), 256, 0, ctx->stream>>>(A.dcat2, 96, 0, 64, n2, A.d5);
    ctx->end();
    // c5: x = y4, dy = d5
    conv_wgrad(u, 5, A.y4, 64, 0, A.d5, 64, 0, n2);
    conv_fwd(ctx, A.d5, 64, 0, 64, u->wb[5], 64, nullptr, A.d4, 64, 0, n2, false, A.y4, 64, 0);
    // c4: x = p2, dy = d4 -> dp2 (pooling is linear: no mask)
    conv_wgrad(u, 4, A.p2, 32, 0, A.d4, 64, 0, n2);
    conv_fwd(ctx, A.d4, 64, 0, 64, u->wb[4], 32, nullptr, A.dp2, 32, 0, n2, false);
    // pool2 backward into dcat2[64:96], masked by c3's activation
    ctx->begin(PM_K_PM);
    k_pool2_bwd_add<<<blocks_for(ctx, v1 * 32), 256, 0, ctx->stream>>>(A.dp2, 32, n1, A.dcat2, 96, 64, A.cat2);
    ctx->end();
    // c3: x = y2, dy = dcat2[64:96]
    conv_wgrad(u, 3, A.y2, 32, 0, A.dcat2, 96, 64, n1);
    conv_fwd(ctx, A.dcat2, 96, 64, 32, u->wb[3], 32, nullptr, A.d2, 32, 0, n1, false, A.y2, 32, 0);
    // c2: x = p1, dy = d2 -> dp1
    conv_wgrad(u, 2, A.p1, 16, 0, A.d2, 32, 0, n1);
    conv_fwd(ctx, A.d2, 32, 0, 32, u->wb[2], 16, nullptr, A.dp1, 16, 0, n1, false);
    // pool1 backward into dcat1[32:48], masked by c1's activation
    ctx->begin(PM_K_PM);
    k_pool2_bwd_add<<<blocks_for(ctx, v0 * 16), 256, 0, ctx->stream>>>(A.dp1, 16, n, A.dcat1, 48, 32, A.cat1);
    ctx->end();
    // c1: x = y0, dy = dcat1[32:48]
    conv_wgrad(u, 1, A.y0, 16, 0, A.dcat1, 48, 32, n);
    conv_fwd(ctx, A.dcat1, 48, 32, 16, u->wb[1], 16, nullptr, A.d0, 16, 0, n, false, A.y0, 16, 0);
    // c0: x = input, dy = d0 (no input gradient)
    conv_wgrad(u, 0, A.in, 16, 0, A.d0, 16, 0, n);
    PM_CUDA(cudaGetLastError());
    return umma_status(ctx);
}

static pm_status repack(pm_unet* u)
{
    pm_ctx* ctx = u->ctx;
    for (int i = 0; i < 10; ++i) {
        const int cnt = 27 * kConvs[i].ci * kConvs[i].co;
        ctx->begin(PM_K_PM);
        k_pack_weights<<<blocks_for(ctx, cnt), 256, 0, ctx->stream>>>(u->p + u->off[i], kConvs[i].ci, kConvs[i].co,
                                                                      u->wf[i], u->wb[i]);
        ctx->end();
    }
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

}  // namespace pmeft

using namespace pmeft;

static bool unet_n_ok(int n) { return n >= 16 && (n & (n - 1)) == 0 && n <= 1024; }

extern "C" long long pm_unet_num_params(void) { return total_params(); }

extern "C" pm_status pm_unet_create(pm_ctx* ctx, pm_unet** out)
{
    if (!ctx || !out) return PM_ERR_INVALID_ARG;
    pm_unet* u = new pm_unet();
    u->ctx = ctx;
    u->np = total_params();
    long long o = 0;
    for (int i = 0; i < 10; ++i) {
        u->off[i] = o;
        o += conv_params(i);
    }
    u->off[10] = o;
    pm_status st = PM_OK;
    if ((st = dalloc(ctx, &u->p, u->np)) != PM_OK || (st = dalloc(ctx, &u->g, u->np)) != PM_OK ||
        (st = dalloc(ctx, &u->m, u->np)) != PM_OK || (st = dalloc(ctx, &u->v, u->np)) != PM_OK) {
        delete u;
        return st;
    }
    for (int i = 0; i < 10; ++i) {
        const size_t cnt = 27 * (size_t)kConvs[i].ci * kConvs[i].co;
        if ((st = dalloc(ctx, &u->wf[i], cnt)) != PM_OK || (st = dalloc(ctx, &u->wb[i], cnt)) != PM_OK) {
            delete u;
            return st;
        }
    }
    cudaMemset(u->p, 0, u->np * sizeof(float));
    cudaMemset(u->g, 0, u->np * sizeof(float));
    cudaMemset(u->m, 0, u->np * sizeof(float));
    cudaMemset(u->v, 0, u->np * sizeof(float));
    *out = u;
    return PM_OK;
}

extern "C" void pm_unet_destroy(pm_unet* u)
{
    if (!u) return;
    // cudaFree synchronises the device; the context may already be gone (its handle is not
    // touched here, so the two can be destroyed in either order)
    free_acts(u->acts);
    cudaFree(u->p);
    cudaFree(u->g);
    cudaFree(u->m);
    cudaFree(u->v);
    for (int i = 0; i < 10; ++i) {
        cudaFree(u->wf[i]);
        cudaFree(u->wb[i]);
    }
    delete u;
}

extern "C" pm_status pm_unet_set_params(pm_unet* u, const float* host, long long count)
{
    if (!u || !host || count != u->np) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    PM_CUDA(cudaMemcpyAsync(u->p, host, count * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    PM_TRY(repack(u));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

extern "C" pm_status pm_unet_get_params(pm_unet* u, float* host, long long count, int which)
{
    if (!u || !host || count != u->np || which < 0 || which > 1) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    PM_CUDA(cudaMemcpyAsync(host, which == 0 ? u->p : u->g, count * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

extern "C" pm_status pm_unet_set_conv_path(pm_unet* u, int path)
{
    if (!u || path < 0 || path > 1) return PM_ERR_INVALID_ARG;
    u->conv_path = path;
    return PM_OK;
}

extern "C" pm_status pm_unet_forward(pm_unet* u, const double* delta, int n, double aB0, double aM0, double a,
                                     double* T_out)
{
    if (!u || !delta || !T_out || !unet_n_ok(n)) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    PM_TRY(ensure_acts(u, n, false));
    PM_TRY(unet_forward(u, delta, n, aB0, aM0, a));
    PM_CUDA(cudaMemcpyAsync(T_out, u->acts.that, (size_t)n * n * n * sizeof(double), cudaMemcpyDeviceToDevice,
                            ctx->stream));
    return PM_OK;
}

extern "C" pm_status pm_unet_loss_grad(pm_unet* u, const double* delta, const float* target, int n, double aB0,
                                       double aM0, double a, double* loss)
{
    if (!u || !delta || !target || !loss || !unet_n_ok(n)) return PM_ERR_INVALID_ARG;
    PM_TRY(ensure_acts(u, n, true));
    PM_TRY(unet_forward(u, delta, n, aB0, aM0, a));
    return unet_backward(u, target, n, loss);
}

extern "C" pm_status pm_unet_adam_step(pm_unet* u, float lr, float beta1, float beta2, float eps)
{
    if (!u || !(lr >= 0.f)) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    u->adam_t += 1;
    const float c1 = 1.f / (1.f - powf(beta1, (float)u->adam_t)), c2 = 1.f / (1.f - powf(beta2, (float)u->adam_t));
    ctx->begin(PM_K_PM);
    k_adam<<<blocks_for(ctx, (size_t)u->np), 256, 0, ctx->stream>>>(u->p, u->g, u->m, u->v, u->np, lr, beta1, beta2,
                                                                     eps, c1, c2);
    ctx->end();
    return repack(u);
}

extern "C" pm_status pm_unet_zero_grad(pm_unet* u)
{
    if (!u) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    PM_CUDA(cudaMemsetAsync(u->g, 0, u->np * sizeof(float), ctx->stream));
    return PM_OK;
}

extern "C" pm_status pm_unet_target(pm_ctx* ctx, const double* chi, int n, double aB0, double aM0, double a,
                                    float* T_out)
{
    if (!ctx || !chi || !T_out || !valid_n(n)) return PM_ERR_INVALID_ARG;
    pm_coeffs cf;
    coefficients(aB0, aM0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    if (cf.src == 0.0) return PM_ERR_INVALID_ARG;
    const double scale = cf.nu * (double)n * (double)n / cf.src;  // nu L(chi) / src
    ctx->begin(PM_K_PM);
    k_target<<<grid_for(ctx, (size_t)n * n * n), 256, 0, ctx->stream>>>(chi, n, scale, T_out);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_unet_warm_start(pm_unet* u, const double* delta, int n, double aB0, double aM0, double a,
                                        double* phi_out)
{
    if (!u || !delta || !phi_out || !unet_n_ok(n)) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = u->ctx;
    pm_coeffs cf;
    coefficients(aB0, aM0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    if (cf.xi == 0.0 || cf.nu == 0.0) {
        PM_CUDA(cudaMemsetAsync(phi_out, 0, (size_t)n * n * n * sizeof(double), ctx->stream));
        return PM_OK;
    }
    PM_TRY(ensure_acts(u, n, false));
    PM_TRY(unet_forward(u, delta, n, aB0, aM0, a));
    // L chi_0 = (src / nu) T_hat, zero mean
    return poisson32(ctx, u->acts.that, n, cf.src / cf.nu, phi_out);
}

extern "C" pm_status pm_linear_start(pm_ctx* ctx, const double* delta, int n, double aB0, double aM0, double a,
                                     double* phi_out)
{
    if (!ctx || !delta || !phi_out || !valid_n(n)) return PM_ERR_INVALID_ARG;
    pm_coeffs cf;
    coefficients(aB0, aM0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    if (cf.xi == 0.0 || cf.nu == 0.0) {
        PM_CUDA(cudaMemsetAsync(phi_out, 0, (size_t)n * n * n * sizeof(double), ctx->stream));
        return PM_OK;
    }
    return poisson32(ctx, delta, n, cf.src / cf.nu, phi_out);
}
