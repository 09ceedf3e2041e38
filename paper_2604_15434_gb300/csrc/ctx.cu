// ctx.cu -- context, parameters, workspaces and the EFT coefficients of the pmeft C ABI.
#include <cmath>
#include <cstring>

#include "internal.cuh"

namespace pmeft {

bool valid_n(int n) { return n >= 8 && n <= 4096 && (n & (n - 1)) == 0; }

int grid_for(pm_ctx* ctx, size_t work, int threads)
{
    // a multiple of the SM count, capped so every block still has work
    size_t blocks = (work + threads - 1) / threads;
    size_t cap = (size_t)ctx->num_sms * 16;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

// Sec. 2.2 (C2, C4 with alpha_T = 0), Eq. alpha-a, G_eff/G of Sec. 2.4, nu and xi of
// Eq. linearised, kappa = C4/(4 E^2 a^4) of Eq. chi_scm.
void coefficients(double aB0, double aM0, double a, double om0, int include_dot, pm_coeffs* c)
{
    const double a3 = a * a * a;
    const double oma = om0 / (om0 + (1.0 - om0) * a3);
    const double aB = aB0 * (1.0 - oma) / (1.0 - om0);
    const double aM = aM0 * (1.0 - oma) / (1.0 - om0);
    const double geff = std::pow(oma, aM0 / (3.0 * (1.0 - om0)));
    const double E2 = om0 / a3 + (1.0 - om0);
    const double hdot = -1.5 * oma;                          // H-dot / H^2 of the LCDM background
    const double aBdot = include_dot ? 3.0 * aB * oma : 0.0;  // d alpha_B / d ln a
    const double rho = 1.5 * oma * geff;                     // rho_m / (2 H^2 M^2)
    c->omega_m_a = oma;
    c->alpha_B = aB;
    c->alpha_M = aM;
    c->geff = geff;
    c->E2 = E2;
    c->C2 = -aM + aB * (1.0 + aM) + (1.0 + aB) * hdot + aBdot + rho;
    c->C4 = -4.0 * aB + 2.0 * aM;
    c->nu = -c->C2 + aB * (2.0 * aM - aB);
    c->xi = aB - aM;
    c->kappa = c->C4 / (4.0 * E2 * a3 * a);
    c->mu_chi = c->xi / c->nu;
    c->mu_psi = 1.0 + c->xi * c->xi / c->nu;
    c->src = c->xi * 1.5 * geff * a * om0;
    c->poisson_fac = 1.5 * geff * a * om0;
}

template <typename T>
static pm_status alloc_level(pm_ctx* ctx, Level<T>& L, int n, bool coarse, bool bg)
{
    L.n = n;
    L.fine = !coarse;
    L.cells = (size_t)n * n * n;
    const size_t b = L.cells * sizeof(T);
    PM_CUDA(cudaMalloc(&L.u[0], b));
    PM_CUDA(cudaMalloc(&L.u[1], b));
    PM_CUDA(cudaMalloc(&L.r, b));
    PM_CUDA(cudaMalloc(&L.sat, L.cells));
    if (coarse) {
        PM_CUDA(cudaMalloc(&L.f, b));
        PM_CUDA(cudaMalloc(&L.ur, b));
        PM_CUDA(cudaMalloc(&L.kmask, L.cells));
    }
    if (bg) PM_CUDA(cudaMalloc(&L.bg, b));
    return PM_OK;
}

template <typename T>
static void free_level(Level<T>& L)
{
    cudaFree(L.u[0]);
    cudaFree(L.u[1]);
    cudaFree(L.r);
    cudaFree(L.sat);
    cudaFree(L.f);
    cudaFree(L.ur);
    cudaFree(L.kmask);
    cudaFree(L.bg);
    cudaFree(L.gap);
    cudaFree(L.coef);
    L = Level<T>();
}

pm_status get_workspace(pm_ctx* ctx, int n, Workspace** out)
{
    auto it = ctx->ws.find(n);
    if (it != ctx->ws.end()) {
        *out = it->second;
        return PM_OK;
    }
    Workspace* w = new Workspace();
    w->n = n;
    ctx->ws[n] = w;
    *out = w;
    return PM_OK;
}

pm_status ensure_mg(pm_ctx* ctx, Workspace* w, bool want_fp32)
{
    const int n = w->n;
    int nlev = 1;
    while ((n >> (nlev - 1)) > ctx->prm.coarsest_n) ++nlev;
    if (w->d.empty() || w->nlev != nlev) {
        for (auto& L : w->d) free_level(L);
        for (auto& L : w->s) free_level(L);
        w->d.assign(nlev, Level<double>());
        w->s.clear();
        w->nlev = nlev;
        for (int l = 0; l < nlev; ++l) PM_TRY(alloc_level(ctx, w->d[l], n >> l, l > 0, false));
    }
    if (want_fp32 && w->s.empty()) {
        w->s.assign(nlev, Level<float>());
        for (int l = 0; l < nlev; ++l) PM_TRY(alloc_level(ctx, w->s[l], n >> l, l > 0, true));
        // the inner level 0 keeps its right-hand side in rplain; give it the f slot too
        PM_CUDA(cudaMalloc(&w->rplain, w->s[0].cells * sizeof(float)));
        PM_CUDA(cudaMalloc(&w->ff_alt, w->s[0].cells * sizeof(float2)));
        PM_CUDA(cudaMalloc(&w->s[0].gap, w->s[0].cells * sizeof(float)));
        if (n >= kCoefMinN) PM_CUDA(cudaMalloc(&w->s[0].coef, 3 * w->s[0].cells * sizeof(uint32_t)));
        // the first coarse inner level, when large enough, also sweeps through coefficients
        // (written by the FAS right-hand side kernel, with its floored gap)
        if (nlev > 1 && (n >> 1) >= kCoefMinN) {
            PM_CUDA(cudaMalloc(&w->s[1].coef, 3 * w->s[1].cells * sizeof(uint32_t)));
            PM_CUDA(cudaMalloc(&w->s[1].gap, w->s[1].cells * sizeof(float)));
        }
    }
    return PM_OK;
}

pm_status ensure_fft(pm_ctx* ctx, Workspace* w)
{
    if (w->fft_ready) return PM_OK;
    const int n = w->n;
    if (cufftPlan3d(&w->plan_r2c, n, n, n, CUFFT_D2Z) != CUFFT_SUCCESS ||
        cufftPlan3d(&w->plan_c2r, n, n, n, CUFFT_Z2D) != CUFFT_SUCCESS) {
        ctx->set_error("cufftPlan3d failed");
        return PM_ERR_CUDA;
    }
    cufftSetStream(w->plan_r2c, ctx->stream);
    cufftSetStream(w->plan_c2r, ctx->stream);
    PM_CUDA(cudaMalloc(&w->spec, (size_t)n * n * (n / 2 + 1) * sizeof(double2)));
    w->fft_ready = true;
    return PM_OK;
}

pm_status ensure_fft32(pm_ctx* ctx, Workspace* w)
{
    if (w->fft32_ready) return PM_OK;
    const int n = w->n;
    if (cufftPlan3d(&w->plan_r2c32, n, n, n, CUFFT_R2C) != CUFFT_SUCCESS ||
        cufftPlan3d(&w->plan_c2r32, n, n, n, CUFFT_C2R) != CUFFT_SUCCESS) {
        ctx->set_error("cufftPlan3d (FP32) failed");
        return PM_ERR_CUDA;
    }
    cufftSetStream(w->plan_r2c32, ctx->stream);
    cufftSetStream(w->plan_c2r32, ctx->stream);
    PM_CUDA(cudaMalloc(&w->spec32, (size_t)n * n * (n / 2 + 1) * sizeof(float2)));
    PM_CUDA(cudaMalloc(&w->buf32, (size_t)n * n * n * sizeof(float)));
    w->fft32_ready = true;
    return PM_OK;
}

void delete_workspace(Workspace* w)
{
    if (!w) return;
    if (w->stream) cudaStreamSynchronize(w->stream);
    for (auto& L : w->d) free_level(L);
    for (auto& L : w->s) free_level(L);
    cudaFree(w->rplain);
    cudaFree(w->ff_alt);
    cudaFree(w->coef_test);
    cudaFree(w->grad);
    cudaFree(w->psi);
    cudaFree(w->delta);
    cudaFree(w->acc);
    cudaFree(w->spec);
    if (w->plan_r2c) cufftDestroy(w->plan_r2c);
    if (w->plan_r2c32) cufftDestroy(w->plan_r2c32);
    if (w->plan_c2r32) cufftDestroy(w->plan_c2r32);
    cudaFree(w->spec32);
    cudaFree(w->buf32);
    if (w->plan_c2r) cufftDestroy(w->plan_c2r);
    cudaFree(w->partials);
    cudaFree(w->out);
    cudaFreeHost(w->host);
    cudaFree(w->lam);
    cudaFree(w->shift);
    if (w->graph) cudaGraphExecDestroy(w->graph);
    if (w->stream) cudaStreamDestroy(w->stream);
    delete w;
}

}  // namespace pmeft

using namespace pmeft;

extern "C" void pm_default_params(pm_params* p)
{
    if (!p) return;
    p->omega_m0 = 0.3;
    p->eta = 0.35;
    p->npre = 2;
    p->npost = 2;
    p->max_cycles = 100;
    p->coarsest_n = 4;
    p->coarse_sweeps = 8;
    p->precision = 0;
    p->include_dot_alphaB = 1;
    p->inner_cycles = 1;
    p->autotune = 1;
    p->linear_eft = 0;
    p->smoother = 0;
    p->coarse_exact = 0;
    p->grad_order = 4;
    p->batch_persistent = 1;
    p->zero_start = 1;
}

static bool params_ok(const pm_params* p)
{
    return p->omega_m0 > 0.0 && p->omega_m0 < 1.0 && p->eta >= 0.0 && p->eta < 1.0 && p->npre >= 0 &&
           p->npost >= 0 && p->npre + p->npost > 0 && p->max_cycles >= 0 && p->coarsest_n >= 2 &&
           p->coarsest_n <= 8 && (p->coarsest_n & (p->coarsest_n - 1)) == 0 && p->coarse_sweeps >= 1 &&
           (p->precision >= 0 && p->precision <= 2) && p->inner_cycles >= 1 && p->inner_cycles <= 16 &&
           (p->autotune == 0 || p->autotune == 1) && (p->linear_eft == 0 || p->linear_eft == 1) &&
           (p->smoother == 0 || p->smoother == 1) && (p->coarse_exact == 0 || (p->coarse_exact == 1 &&
           p->coarsest_n <= 4)) && (p->grad_order == 2 || p->grad_order == 4) &&
           (p->batch_persistent == 0 || p->batch_persistent == 1) && (p->zero_start == 0 || p->zero_start == 1);
}

extern "C" pm_status pm_coefficients(double aB0, double aM0, double a, double om0, int include_dot, pm_coeffs* out)
{
    if (!out || !(a > 0.0) || !(om0 > 0.0) || !(om0 < 1.0) || !std::isfinite(aB0) || !std::isfinite(aM0))
        return PM_ERR_INVALID_ARG;
    coefficients(aB0, aM0, a, om0, include_dot, out);
    return PM_OK;
}

extern "C" pm_status pm_create(pm_ctx** out, int device, void* stream, const pm_params* p)
{
    if (!out) return PM_ERR_INVALID_ARG;
    *out = nullptr;
    pm_params prm;
    pm_default_params(&prm);
    if (p) {
        if (!params_ok(p)) return PM_ERR_INVALID_ARG;
        prm = *p;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return PM_ERR_INVALID_ARG;
    pm_ctx* ctx = new pm_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)stream;
    ctx->prm = prm;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete ctx;
        return PM_ERR_CUDA;
    }
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaMalloc(&ctx->red_partials, sizeof(double) * (kMaxPartials * 8 + 8)) != cudaSuccess ||
        cudaMalloc(&ctx->red_out, sizeof(double) * 64) != cudaSuccess ||
        cudaMalloc(&ctx->flag, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost(&ctx->host_out, sizeof(double) * 64) != cudaSuccess) {
        pm_destroy(ctx);
        return PM_ERR_OOM;
    }
    cudaMemset(ctx->flag, 0, sizeof(int) * 4);
    cudaMemset(ctx->red_partials, 0, sizeof(double) * (kMaxPartials * 8 + 8));  // partials and their counter
    cudaMemset(ctx->red_out, 0, sizeof(double) * 64);
    *out = ctx;
    return PM_OK;
}

extern "C" void pm_destroy(pm_ctx* ctx)
{
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto& kv : ctx->ws) delete_workspace(kv.second);
    for (auto* w : ctx->batch) delete_workspace(w);
    if (ctx->batch_stream) cudaStreamDestroy(ctx->batch_stream);
    for (auto& r : ctx->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->pool) cudaEventDestroy(e);
    cudaFree(ctx->red_partials);
    cudaFree(ctx->red_out);
    cudaFree(ctx->flag);
    cudaFreeHost(ctx->host_out);
    cudaFree(ctx->coop_boxes);
    cudaFree(ctx->coop_active);
    cudaFreeHost(ctx->coop_active_host);
    cudaFree(ctx->coop_partials);
    cudaFree(ctx->coop_gm);
    cudaFree(ctx->coop_bar);
    cudaFreeHost(ctx->coop_err_host);
    delete ctx;
}

extern "C" pm_status pm_batch_barrier_test(pm_ctx* ctx, int block, int barrier, double wait_s)
{
    if (!ctx || barrier < 0) return PM_ERR_INVALID_ARG;
    ctx->coop_fail_block = block < 0 ? -1 : block;
    ctx->coop_fail_barrier = block < 0 ? -1 : barrier;
    if (wait_s > 0.0) ctx->coop_wait_s = wait_s;
    return PM_OK;
}

extern "C" const char* pm_last_error(const pm_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

extern "C" pm_status pm_set_params(pm_ctx* ctx, const pm_params* p)
{
    if (!ctx || !p || !params_ok(p)) return PM_ERR_INVALID_ARG;
    ctx->prm = *p;
    return PM_OK;
}

extern "C" pm_status pm_trace_reset(pm_ctx* ctx)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    else cudaDeviceSynchronize();
    for (auto& r : ctx->recs) {
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    ctx->prof = pm_profile{};
    return PM_OK;
}

extern "C" pm_status pm_trace_enable(pm_ctx* ctx, int on)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    pm_trace_reset(ctx);
    ctx->tracing = on != 0;
    ctx->trace_mask = ~0u;
    ctx->trace_fine_only = false;
    return PM_OK;
}

extern "C" pm_status pm_trace_select(pm_ctx* ctx, unsigned class_mask, int fine_only)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    pm_trace_reset(ctx);
    ctx->tracing = class_mask != 0;
    ctx->trace_mask = class_mask;
    ctx->trace_fine_only = fine_only != 0;
    return PM_OK;
}

extern "C" pm_status pm_trace_get(pm_ctx* ctx, pm_profile* out)
{
    if (!ctx || !out) return PM_ERR_INVALID_ARG;
    cudaError_t e = ctx->stream ? cudaStreamSynchronize(ctx->stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ctx->set_error(std::string("pm_trace_get: ") + cudaGetErrorString(e));
        return PM_ERR_CUDA;
    }
    for (auto& r : ctx->recs) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, r.a, r.b);
        ctx->prof.ms[r.cls] += ms;
        if (r.fine) ctx->prof.fine_ms[r.cls] += ms;
        ctx->pool.push_back(r.a);
        ctx->pool.push_back(r.b);
    }
    ctx->recs.clear();
    *out = ctx->prof;
    return PM_OK;
}

extern "C" int pm_tune_log(const pm_ctx* ctx, char* buf, int len)
{
    if (!ctx) return 0;
    const int full = (int)ctx->tune_log.size();
    if (buf && len > 0) {
        const int k = full < len - 1 ? full : len - 1;
        memcpy(buf, ctx->tune_log.data(), (size_t)k);
        buf[k] = 0;
    }
    return full;
}
