// pm.cu -- particle-mesh steps around the chi solve (arXiv 2604.15434, Sec. 3.1, 3.5, 3.6):
// CIC deposit in 2^40 fixed point, the FFT Poisson solve of Eq. phipsi_mod, the five-point
// gradient of Psi = Psi_N + (alpha_B - alpha_M) chi interpolated to particles (Eq. force),
// and one kick-drift.
#include <cmath>

#include "internal.cuh"

namespace pmeft {

// Cell-centred CIC weights of one coordinate; every operation rounded as written
// (no contraction) so that the weights are identical on every machine.
__device__ __forceinline__ void cic_1d(double x, int n, int& i0, int& i1, double& w0, double& w1)
{
    const double u = __dmul_rn(x, (double)n);
    const double s = __dsub_rn(u, 0.5);
    const double fl = floor(s);
    const double d = __dsub_rn(s, fl);
    const int i = (int)fl;
    i0 = i & (n - 1);
    i1 = (i + 1) & (n - 1);
    w0 = __dsub_rn(1.0, d);
    w1 = d;
}

__global__ void __launch_bounds__(256) k_deposit(const double* __restrict__ pos, long long np, int n,
                                                 unsigned long long* __restrict__ acc)
{
    const double scale = 1099511627776.0;  // 2^40
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        cic_1d(pos[p], n, ix[0], ix[1], wx[0], wx[1]);
        cic_1d(pos[np + p], n, iy[0], iy[1], wy[0], wy[1]);
        cic_1d(pos[2 * np + p], n, iz[0], iz[1], wz[0], wz[1]);
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            const double w = __dmul_rn(__dmul_rn(wx[a], wy[b]), wz[e]);
            const long long q = __double2ll_rn(__dmul_rn(w, scale));
            atomicAdd(&acc[((size_t)iz[e] * n + iy[b]) * n + ix[a]], (unsigned long long)q);
        }
    }
}

// delta = acc 2^-40 (n^3/np) - 1; a negative accumulator means the int64 capacity
// (2^23 particles at full weight in one cell) was exceeded.
__global__ void k_density(const long long* __restrict__ acc, size_t cells, double fac, double* __restrict__ delta,
                          int* __restrict__ flag)
{
    const double inv = 1.0 / 1099511627776.0;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < cells; c += (size_t)gridDim.x * blockDim.x) {
        const long long a = acc[c];
        if (a < 0) flag[0] = 1;
        delta[c] = __dsub_rn(__dmul_rn(__dmul_rn((double)a, inv), fac), 1.0);
    }
}

// Multiply the spectrum by fac / lambda_k with lambda_k = -(4/h^2) sum sin^2(pi m/n), the
// 7-point Laplacian's eigenvalues; the zero mode is set to 0.  Also folds in 1/n^3.  Each
// block first tabulates sin^2(pi m/n), m < n, in shared memory (n doubles), so the FP64 sines
// are evaluated n times per block instead of three times per mode.
__global__ void k_green(double2* __restrict__ spec, int n, double fac)
{
    extern __shared__ double s2[];  // [n]
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        const double sm = sinpi((double)m / n);
        s2[m] = sm * sm;
    }
    __syncthreads();
    const int nh = n / 2 + 1;
    const size_t total = (size_t)n * n * nh;
    const double h2inv = (double)n * (double)n;
    const double norm = 1.0 / ((double)n * (double)n * (double)n);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int mx = (int)(t % nh);
        const size_t row = t / nh;
        const int my = (int)(row % n), mz = (int)(row / n);
        const double lam = -4.0 * h2inv * (s2[mx] + s2[my] + s2[mz]);
        double2 v = spec[t];
        if (t == 0) {
            v.x = 0.0;
            v.y = 0.0;
        } else {
            const double g = fac * norm / lam;
            v.x *= g;
            v.y *= g;
        }
        spec[t] = v;
    }
}

// k_green in FP32 (the start fields' solve): the same eigenvalues, zero mode and 1/n^3
__global__ void k_green32(float2* __restrict__ spec, int n, float fac)
{
    const int nh = n / 2 + 1;
    const size_t total = (size_t)n * n * nh;
    const float h2inv = (float)n * (float)n;
    const float scale = fac / ((float)n * (float)n * (float)n);
    for (size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (size_t)gridDim.x * blockDim.x) {
        const int mx = (int)(t % nh);
        const size_t row = t / nh;
        const int my = (int)(row % n), mz = (int)(row / n);
        const float sx = sinpif((float)mx / n), sy = sinpif((float)my / n), sz = sinpif((float)mz / n);
        const float lam = -4.f * h2inv * (sx * sx + sy * sy + sz * sz);
        float2 v = spec[t];
        if (t == 0) {
            v = make_float2(0.f, 0.f);
        } else {
            const float g = scale / lam;
            v.x *= g;
            v.y *= g;
        }
        spec[t] = v;
    }
}

__global__ void k_d2f(const double* __restrict__ x, size_t total, float* __restrict__ y)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        y[c] = (float)x[c];
}

__global__ void k_f2d(const float* __restrict__ x, size_t total, double* __restrict__ y)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        y[c] = (double)x[c];
}

// Psi = psiN + xi chi on the grid (psiN alone when chi is null), rounded as written.
__global__ void k_psi_total(const double* __restrict__ psiN, const double* __restrict__ chi, double xi,
                            size_t total, double* __restrict__ psi)
{
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x)
        psi[c] = chi ? __dadd_rn(psiN[c], __dmul_rn(xi, chi[c])) : psiN[c];
}

// g = -grad Psi on the grid, one cell per thread: the five-point difference
// (-f+2 + 8 f+1 - 8 f-1 + f-2)/(12 h) per axis (FOUR; else the two-point (f+1 - f-1)/(2 h)),
// periodic.  g holds the three components one after the other ([3][n^3]).
template <bool FOUR>
__global__ void __launch_bounds__(256) k_grad(const double* __restrict__ psi, int n, double* __restrict__ g)
{
    const int m = n - 1;
    const size_t total = (size_t)n * n * n;
    const double inv12h = (double)n / 12.0, inv2h = (double)n * 0.5;
    for (size_t c = (size_t)blockIdx.x * blockDim.x + threadIdx.x; c < total; c += (size_t)gridDim.x * blockDim.x) {
        const int i = (int)(c & (size_t)m);  // n is a power of two
        const int j = (int)((c / n) & (size_t)m), k = (int)(c / ((size_t)n * n));
        auto at = [&](int x, int y, int z) { return psi[((size_t)(z & m) * n + (y & m)) * n + (x & m)]; };
        double gx, gy, gz;
        if (FOUR) {
            gx = (-at(i + 2, j, k) + 8.0 * at(i + 1, j, k) - 8.0 * at(i - 1, j, k) + at(i - 2, j, k)) * inv12h;
            gy = (-at(i, j + 2, k) + 8.0 * at(i, j + 1, k) - 8.0 * at(i, j - 1, k) + at(i, j - 2, k)) * inv12h;
            gz = (-at(i, j, k + 2) + 8.0 * at(i, j, k + 1) - 8.0 * at(i, j, k - 1) + at(i, j, k - 2)) * inv12h;
        } else {
            gx = (at(i + 1, j, k) - at(i - 1, j, k)) * inv2h;
            gy = (at(i, j + 1, k) - at(i, j - 1, k)) * inv2h;
            gz = (at(i, j, k + 1) - at(i, j, k - 1)) * inv2h;
        }
        g[c] = -gx;
        g[total + c] = -gy;
        g[2 * total + c] = -gz;
    }
}

// the force at each particle: the grid force g ([3][n^3]) at the 8 CIC corners (in the
// deposit's corner order), weighted by the corner's CIC weight (the deposit's adjoint)
__global__ void __launch_bounds__(256) k_interp_force(const double* __restrict__ g, int n,
                                                      const double* __restrict__ pos, long long np,
                                                      double* __restrict__ acc)
{
    const int m = n - 1;
    const size_t total = (size_t)n * n * n;
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (long long)gridDim.x * blockDim.x) {
        int ix[2], iy[2], iz[2];
        double wx[2], wy[2], wz[2];
        cic_1d(pos[p], n, ix[0], ix[1], wx[0], wx[1]);
        cic_1d(pos[np + p], n, iy[0], iy[1], wy[0], wy[1]);
        cic_1d(pos[2 * np + p], n, iz[0], iz[1], wz[0], wz[1]);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int a = c & 1, b = (c >> 1) & 1, e = (c >> 2) & 1;
            const size_t cell = ((size_t)(iz[e] & m) * n + (iy[b] & m)) * n + (ix[a] & m);
            const double w = __dmul_rn(__dmul_rn(wx[a], wy[b]), wz[e]);
            s0 += w * g[cell];
            s1 += w * g[total + cell];
            s2 += w * g[2 * total + cell];
        }
        acc[p] = s0;
        acc[np + p] = s1;
        acc[2 * np + p] = s2;
    }
}

// v += g dt; x = frac(x + v dt), each product and sum rounded as written.
__global__ void k_kick_drift(double* __restrict__ pos, double* __restrict__ vel, const double* __restrict__ acc,
                             long long total, double dt)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const double v = __dadd_rn(vel[i], __dmul_rn(acc[i], dt));
        vel[i] = v;
        double x = __dadd_rn(pos[i], __dmul_rn(v, dt));
        x = __dsub_rn(x, floor(x));
        if (x >= 1.0) x = 0.0;
        pos[i] = x;
    }
}

// out = s * x (+ y), each product and sum rounded as written
__global__ void k_scale_add(const double* __restrict__ x, double s, const double* __restrict__ y, size_t total,
                            double* __restrict__ out)
{
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const double v = __dmul_rn(s, x[i]);
        out[i] = y ? __dadd_rn(y[i], v) : v;
    }
}

static void scale_add(pm_ctx* ctx, const double* x, double s, const double* y, size_t total, double* out)
{
    ctx->begin(PM_K_PM, false, 0);
    k_scale_add<<<grid_for(ctx, total), kThreads, 0, ctx->stream>>>(x, s, y, total, out);
    ctx->end();
}

pm_status deposit(pm_ctx* ctx, const double* pos, long long np, int n, long long* acc)
{
    const size_t cells = (size_t)n * n * n;
    PM_CUDA(cudaMemsetAsync(acc, 0, cells * sizeof(long long), ctx->stream));
    ctx->begin(PM_K_PM, false, 0);
    k_deposit<<<grid_for(ctx, (size_t)np), kThreads, 0, ctx->stream>>>(pos, np, n, (unsigned long long*)acc);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status density(pm_ctx* ctx, const long long* acc, int n, long long np, double* delta)
{
    const size_t cells = (size_t)n * n * n;
    PM_CUDA(cudaMemsetAsync(ctx->flag, 0, sizeof(int), ctx->stream));
    ctx->begin(PM_K_PM, false, 0);
    k_density<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(acc, cells, (double)cells / (double)np, delta,
                                                                   ctx->flag);
    ctx->end();
    int hflag = 0;
    PM_CUDA(cudaMemcpyAsync(&hflag, ctx->flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    if (hflag) {
        ctx->set_error("fixed-point deposit overflow (more than 2^23 particles in one cell)");
        return PM_ERR_OVERFLOW;
    }
    return PM_OK;
}

pm_status poisson(pm_ctx* ctx, const double* delta, int n, double fac, double* psi)
{
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    PM_TRY(ensure_fft(ctx, w));
    ctx->prof.launches[PM_K_PM] += 2;  // the two cuFFT executions (library kernels)
    if (cufftExecD2Z(w->plan_r2c, (cufftDoubleReal*)delta, (cufftDoubleComplex*)w->spec) != CUFFT_SUCCESS) {
        ctx->set_error("cufftExecD2Z failed");
        return PM_ERR_CUDA;
    }
    ctx->begin(PM_K_PM, false, 0);
    k_green<<<grid_for(ctx, (size_t)n * n * (n / 2 + 1)), kThreads, (size_t)n * sizeof(double), ctx->stream>>>(w->spec, n,
                                                                                                         fac);
    ctx->end();
    if (cufftExecZ2D(w->plan_c2r, (cufftDoubleComplex*)w->spec, (cufftDoubleReal*)psi) != CUFFT_SUCCESS) {
        ctx->set_error("cufftExecZ2D failed");
        return PM_ERR_CUDA;
    }
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status poisson32(pm_ctx* ctx, const double* delta, int n, double fac, double* psi)
{
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    PM_TRY(ensure_fft32(ctx, w));
    const size_t cells = (size_t)n * n * n;
    ctx->begin(PM_K_PM, false, 0);
    k_d2f<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(delta, cells, w->buf32);
    ctx->end();
    ctx->prof.launches[PM_K_PM] += 2;  // the two cuFFT executions (library kernels)
    if (cufftExecR2C(w->plan_r2c32, (cufftReal*)w->buf32, (cufftComplex*)w->spec32) != CUFFT_SUCCESS) {
        ctx->set_error("cufftExecR2C failed");
        return PM_ERR_CUDA;
    }
    ctx->begin(PM_K_PM, false, 0);
    k_green32<<<grid_for(ctx, (size_t)n * n * (n / 2 + 1)), kThreads, 0, ctx->stream>>>(w->spec32, n, (float)fac);
    ctx->end();
    if (cufftExecC2R(w->plan_c2r32, (cufftComplex*)w->spec32, (cufftReal*)w->buf32) != CUFFT_SUCCESS) {
        ctx->set_error("cufftExecC2R failed");
        return PM_ERR_CUDA;
    }
    ctx->begin(PM_K_PM, false, 0);
    k_f2d<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(w->buf32, cells, psi);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

// g = -grad(psiN + xi chi) at each particle (Eq. force, Sec. 3.5.2): the total potential and
// its gradient on the grid (workspace [4][n^3]: Psi, then the three components), then the
// CIC interpolation of the grid force.
pm_status interp_force(pm_ctx* ctx, const double* psiN, const double* chi, double xi, int n, const double* pos,
                       long long np, double* acc)
{
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    const size_t cells = (size_t)n * n * n;
    if (!w->grad) PM_CUDA(cudaMalloc(&w->grad, 4 * cells * sizeof(double)));
    double* psi = w->grad;
    double* g = w->grad + cells;
    ctx->begin(PM_K_PM, false, 0);
    k_psi_total<<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(psiN, chi, xi, cells, psi);
    ctx->end();
    ctx->begin(PM_K_PM, false, 0);
    if (ctx->prm.grad_order == 2)
        k_grad<false><<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(psi, n, g);
    else
        k_grad<true><<<grid_for(ctx, cells), kThreads, 0, ctx->stream>>>(psi, n, g);
    ctx->end();
    ctx->begin(PM_K_PM, false, 0);
    k_interp_force<<<grid_for(ctx, (size_t)np), kThreads, 0, ctx->stream>>>(g, n, pos, np, acc);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

pm_status kick_drift(pm_ctx* ctx, double* pos, double* vel, const double* acc, long long np, double dt)
{
    ctx->begin(PM_K_PM, false, 0);
    k_kick_drift<<<grid_for(ctx, (size_t)(3 * np)), kThreads, 0, ctx->stream>>>(pos, vel, acc, 3 * np, dt);
    ctx->end();
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}

// Launchers on a bare stream (no context), used by the allocation-free deposit.
static int grid_on(int sms, size_t work)
{
    size_t blocks = (work + kThreads - 1) / kThreads, cap = (size_t)(sms > 0 ? sms : 152) * 16;
    return (int)(blocks < 1 ? 1 : (blocks > cap ? cap : blocks));
}

void launch_deposit_on(cudaStream_t s, int sms, const double* pos, long long np, int n, unsigned long long* acc)
{
    k_deposit<<<grid_on(sms, (size_t)np), kThreads, 0, s>>>(pos, np, n, acc);
}

void launch_density_on(cudaStream_t s, int sms, const long long* acc, int n, long long np, double* delta, int* flag)
{
    const size_t cells = (size_t)n * n * n;
    k_density<<<grid_on(sms, cells), kThreads, 0, s>>>(acc, cells, (double)cells / (double)np, delta, flag);
}

}  // namespace pmeft

using namespace pmeft;

static pm_status check_common(pm_ctx* ctx, int n)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (!valid_n(n)) {
        ctx->set_error("n must be a power of two >= 8");
        return PM_ERR_INVALID_ARG;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) return PM_ERR_CUDA;
    return PM_OK;
}

extern "C" pm_status pm_deposit_cic_fixed(pm_ctx* ctx, const double* pos, long long np, int n, long long* acc)
{
    PM_TRY(check_common(ctx, n));
    if (!pos || !acc || np < 1) {
        ctx->set_error("pm_deposit_cic: null buffer or np < 1");
        return PM_ERR_INVALID_ARG;
    }
    return deposit(ctx, pos, np, n, acc);
}

extern "C" pm_status pm_deposit_cic(pm_ctx* ctx, const double* pos, long long np, int n, double* delta)
{
    PM_TRY(check_common(ctx, n));
    if (!pos || !delta || np < 1) {
        ctx->set_error("pm_deposit_cic: null buffer or np < 1");
        return PM_ERR_INVALID_ARG;
    }
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    if (!w->acc) PM_CUDA(cudaMalloc(&w->acc, (size_t)n * n * n * sizeof(long long)));
    PM_TRY(deposit(ctx, pos, np, n, w->acc));
    return density(ctx, w->acc, n, np, delta);
}

extern "C" pm_status poisson_solve(pm_ctx* ctx, const double* delta, int n, double a, double alpha_M0, double* psi_N)
{
    PM_TRY(check_common(ctx, n));
    if (!delta || !psi_N || delta == psi_N || !(a > 0.0)) {
        ctx->set_error("poisson_solve: null or aliased buffer, or a <= 0");
        return PM_ERR_INVALID_ARG;
    }
    pm_coeffs cf;
    coefficients(0.0, alpha_M0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    return poisson(ctx, delta, n, cf.poisson_fac, psi_N);
}

extern "C" pm_status force_interp(pm_ctx* ctx, const double* psi_N, const double* phi, int n, double alpha_B0,
                                  double alpha_M0, double a, const double* pos, long long np, double* acc)
{
    PM_TRY(check_common(ctx, n));
    if (!psi_N || !pos || !acc || np < 1 || !(a > 0.0)) {
        ctx->set_error("force_interp: null buffer, np < 1 or a <= 0");
        return PM_ERR_INVALID_ARG;
    }
    pm_coeffs cf;
    coefficients(alpha_B0, alpha_M0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    return interp_force(ctx, psi_N, phi, cf.xi, n, pos, np, acc);
}

extern "C" pm_status pm_step(pm_ctx* ctx, double* pos, double* vel, long long np, int n, double alpha_B0,
                             double alpha_M0, double a, double dt, double tol, double* phi_state, pm_solve_info* info)
{
    PM_TRY(check_common(ctx, n));
    if (!pos || !vel || !phi_state || np < 1 || !(a > 0.0) || !(tol > 0.0)) {
        ctx->set_error("pm_step: null buffer, np < 1, a <= 0 or tol <= 0");
        return PM_ERR_INVALID_ARG;
    }
    Workspace* w = nullptr;
    PM_TRY(get_workspace(ctx, n, &w));
    const size_t cells = (size_t)n * n * n;
    if (!w->acc) PM_CUDA(cudaMalloc(&w->acc, cells * sizeof(long long)));
    if (!w->delta) PM_CUDA(cudaMalloc(&w->delta, cells * sizeof(double)));
    if (!w->psi) PM_CUDA(cudaMalloc(&w->psi, cells * sizeof(double)));
    pm_coeffs cf;
    coefficients(alpha_B0, alpha_M0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    PM_TRY(deposit(ctx, pos, np, n, w->acc));
    PM_TRY(density(ctx, w->acc, n, np, w->delta));
    PM_TRY(poisson(ctx, w->delta, n, cf.poisson_fac, w->psi));
    if (ctx->prm.linear_eft) {
        // linearised equations: nu L chi = xi S and L Psi_N = S, so chi = (xi / nu) Psi_N
        if (cf.nu == 0.0 && cf.xi != 0.0) {
            ctx->set_error("pm_step: nu = 0, the linearised chi equation is degenerate");
            return PM_ERR_INVALID_ARG;
        }
        scale_add(ctx, w->psi, cf.xi != 0.0 ? cf.xi / cf.nu : 0.0, nullptr, cells, phi_state);
        if (info) *info = pm_solve_info{};
    } else {
        pm_status st = mg_solve(ctx, w->delta, n, cf, tol, phi_state, info);
        if (st != PM_OK) return st;
    }
    // the acceleration goes into the (now free) fixed-point grid's storage when it fits
    double* acc = nullptr;
    const size_t need = (size_t)3 * np * sizeof(double);
    if (need <= cells * sizeof(long long)) {
        acc = (double*)w->acc;
    } else {
        PM_CUDA(cudaMallocAsync(&acc, need, ctx->stream));
    }
    PM_TRY(interp_force(ctx, w->psi, phi_state, cf.xi, n, pos, np, acc));
    PM_TRY(kick_drift(ctx, pos, vel, acc, np, dt));
    if ((void*)acc != (void*)w->acc) PM_CUDA(cudaFreeAsync(acc, ctx->stream));
    PM_CUDA(cudaStreamSynchronize(ctx->stream));
    return PM_OK;
}

// ------------------------------------------------------------------ several steps

// supercomoving time per unit scale factor: dt~/da = 1 / (a^3 E(a)), E^2 = Om a^-3 + 1 - Om
static double dtda(double a, double om) { return 1.0 / (a * a * a * std::sqrt(om / (a * a * a) + 1.0 - om)); }
static double dadt(double a, double om) { return a * a * a * std::sqrt(om / (a * a * a) + 1.0 - om); }

extern "C" pm_status pm_run(pm_ctx* ctx, double* pos, double* vel, long long np, int n, double alpha_B0,
                            double alpha_M0, double a_start, double a_end, int nsteps, double tol,
                            double* phi_state, pm_solve_info* info)
{
    PM_TRY(check_common(ctx, n));
    if (!(a_start > 0.0) || !(a_end >= a_start) || nsteps < 1) {
        ctx->set_error("pm_run: need 0 < a_start <= a_end and nsteps >= 1");
        return PM_ERR_INVALID_ARG;
    }
    const double om = ctx->prm.omega_m0;
    // total supercomoving time by composite Simpson in a (4096 intervals), equal steps in it
    const int K = 4096;
    const double ha = (a_end - a_start) / K;
    double T = dtda(a_start, om) + dtda(a_end, om);
    for (int k = 1; k < K; ++k) T += (k & 1 ? 4.0 : 2.0) * dtda(a_start + k * ha, om);
    T *= ha / 3.0;
    const double dt = T / nsteps;
    double a = a_start;
    pm_solve_info local{};
    for (int s = 0; s < nsteps; ++s) {
        PM_TRY(pm_step(ctx, pos, vel, np, n, alpha_B0, alpha_M0, a, dt, tol, phi_state, info ? info : &local));
        // advance a over the step: classical Runge-Kutta on da/dt~ = a^3 E(a), 8 substeps
        const double hs = dt / 8.0;
        for (int q = 0; q < 8; ++q) {
            const double k1 = dadt(a, om), k2 = dadt(a + 0.5 * hs * k1, om), k3 = dadt(a + 0.5 * hs * k2, om),
                         k4 = dadt(a + hs * k3, om);
            a += hs * (k1 + 2.0 * k2 + 2.0 * k3 + k4) / 6.0;
        }
    }
    return PM_OK;
}

extern "C" pm_status lensing_potential(pm_ctx* ctx, const double* psi_N, const double* chi, int n, double alpha_B0,
                                       double alpha_M0, double a, double* Phi)
{
    PM_TRY(check_common(ctx, n));
    if (!psi_N || !chi || !Phi || !(a > 0.0)) {
        ctx->set_error("lensing_potential: null buffer or a <= 0");
        return PM_ERR_INVALID_ARG;
    }
    pm_coeffs cf;
    coefficients(alpha_B0, alpha_M0, a, ctx->prm.omega_m0, ctx->prm.include_dot_alphaB, &cf);
    scale_add(ctx, chi, cf.alpha_B, psi_N, (size_t)n * n * n, Phi);
    PM_CUDA(cudaGetLastError());
    return PM_OK;
}
