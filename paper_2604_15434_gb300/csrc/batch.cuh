// batch.cuh -- many boxes with their own sizes and EFT parameters in one graph launch per
// outer iteration (included by mg.cu; uses its kernels and host helpers).
//
// Each box runs the mixed-precision defect-correction loop of the single-box solve: a
// float-float residual (its gauge multiplier kept on the device), then `inner_cycles` FP32
// FAS V-cycles on the correction and the float-float update; a converged box's result is
// confirmed by one FP64 residual, as in the single-box solve.  One outer iteration of
// every unconverged box is captured into a single CUDA graph with one branch per box, so
// the small boxes' kernels run side by side and the host issues one launch per iteration.
// The host reads all boxes' residual norms after each launch (one synchronisation); a box
// that has converged has its nodes disabled in the executable graph, so the graph is captured
// and instantiated once per call.  The first iteration runs eagerly so the autotuner has
// chosen every tile before capture.
#pragma once

#include <set>

namespace pmeft {

__global__ void k_update_shift(const double* __restrict__ sums, double* __restrict__ lam, float* __restrict__ shift)
{
    const double gm = sums[3] > 0.0 ? sums[0] / sums[3] : 0.0;
    *lam -= gm;
    *shift = (float)(-gm);
}

struct BoxRun {
    Workspace* w = nullptr;
    pm_coeffs cf{};
    Coef c{};
    const double* delta = nullptr;
    double* phi = nullptr;
    double fnorm = 0.0, rr = 0.0;
    int cyc = 0, vcyc = 0;
    pm_status st = PM_ERR_NOCONV;
    bool active = false, trivial = false;
    size_t cells = 0;
    double hist[64] = {};
    double guess_rr = 0.0;
    bool guess_rejected = false;
    FFCoef fk{};
    double lam_fix = 0.0;  // gauge shift found by the confirming FP64 residual
};

static pm_status box_prepare(pm_ctx* ctx, Workspace* w)
{
    if (!w->stream) PM_CUDA(cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking));
    if (!w->partials) {
        PM_CUDA(cudaMalloc(&w->partials, sizeof(double) * (kMaxPartials * 8 + 8)));
        PM_CUDA(cudaMemset(w->partials, 0, sizeof(double) * (kMaxPartials * 8 + 8)));  // with the launch counter
    }
    if (!w->out) PM_CUDA(cudaMalloc(&w->out, sizeof(double) * 64));
    if (!w->host) PM_CUDA(cudaMallocHost(&w->host, sizeof(double) * 64));
    if (!w->lam) PM_CUDA(cudaMalloc(&w->lam, sizeof(double)));
    if (!w->shift) PM_CUDA(cudaMalloc(&w->shift, sizeof(float)));
    return PM_OK;
}

// Float-float residual of the box's iterate with the device-side gauge multiplier;
// updates the multiplier and the inner shift on the device and copies the sums to pinned
// host memory.
static void box_residual(Exec* x, BoxRun& B)
{
    Workspace* w = B.w;
    residual_ff(x, w, ff_chi(w), ff_rhs(w), 0.0, w->lam, B.fk);
    x->begin(PM_K_REDUCE);
    k_update_shift<<<1, 1, 0, x->stream>>>(x->red_out, w->lam, w->shift);
    x->end();
    cudaMemcpyAsync(w->host, x->red_out, sizeof(double) * 9, cudaMemcpyDeviceToHost, x->stream);
}

// One outer iteration after a residual: inner V-cycles, the correction, residual.
static void box_iteration(Exec* x, BoxRun& B)
{
    Workspace* w = B.w;
    auto& s = w->s;
    for (size_t l = 0; l + 1 < s.size(); ++l) {
        x->begin(PM_K_TRANSFER);
        k_restrict<float><<<grid_for(x, s[l + 1].cells), kThreads, 0, x->stream>>>(s[l].bg, s[l + 1].n, s[l + 1].bg);
        x->end();
    }
    s[0].lamp = w->shift;
    start_at_zero(x, s[0]);
    for (int k = 0; k < x->prm.inner_cycles; ++k) vcycle<float>(x, s, 0, w->rplain, 1.0f, 0.0f, B.c);
    add_correction_ff(x, ff_chi(w), s[0].u[s[0].cur], B.cells);
    box_residual(x, B);
}

// The same iteration split around the cooperative coarse kernel: box_down runs the levels
// above level l32 (the 32^3 level) down, box_up the prolongations and post-smoothing back
// up, the correction and the next residual; level l32's iterate is in u[cur32] after the
// cooperative kernel.
static void box_down(Exec* x, BoxRun& B, int l32)
{
    Workspace* w = B.w;
    auto& s = w->s;
    for (size_t l = 0; l + 1 < s.size(); ++l) {
        x->begin(PM_K_TRANSFER);
        k_restrict<float><<<grid_for(x, s[l + 1].cells), kThreads, 0, x->stream>>>(s[l].bg, s[l + 1].n, s[l + 1].bg);
        x->end();
    }
    s[0].lamp = w->shift;
    start_at_zero(x, s[0]);
    vcycle_down<float>(x, s, l32, w->rplain, 1.0f, 0.0f, B.c);
}

static void box_up(Exec* x, BoxRun& B, int l32, int cur32)
{
    Workspace* w = B.w;
    auto& s = w->s;
    s[l32].cur = cur32;
    vcycle_up<float>(x, s, l32, w->rplain, 1.0f, 0.0f, B.c);
    add_correction_ff(x, ff_chi(w), s[0].u[s[0].cur], B.cells);
    box_residual(x, B);
}

// level index of the 32^3 level of a box of size n
static int coop_level(int n)
{
    int l = 0;
    while ((n >> l) > kCoopTop) ++l;
    return l;
}

static pm_status coop_alloc(pm_ctx* ctx, int nbox)
{
    if (ctx->coop_cap >= nbox) return PM_OK;
    cudaFree(ctx->coop_boxes);
    cudaFree(ctx->coop_active);
    cudaFreeHost(ctx->coop_active_host);
    cudaFree(ctx->coop_partials);
    cudaFree(ctx->coop_gm);
    ctx->coop_boxes = nullptr;
    ctx->coop_active = nullptr;
    ctx->coop_active_host = nullptr;
    ctx->coop_partials = nullptr;
    ctx->coop_gm = nullptr;
    ctx->coop_cap = 0;
    PM_CUDA(cudaMalloc(&ctx->coop_boxes, sizeof(CoopBox) * nbox));
    PM_CUDA(cudaMalloc(&ctx->coop_active, sizeof(int) * nbox));
    PM_CUDA(cudaMallocHost(&ctx->coop_active_host, sizeof(int) * nbox));
    PM_CUDA(cudaMalloc(&ctx->coop_partials, sizeof(double) * 2 * kCoopMaxItems * nbox));
    PM_CUDA(cudaMalloc(&ctx->coop_gm, sizeof(float) * nbox));
    if (!ctx->coop_bar) PM_CUDA(cudaMalloc(&ctx->coop_bar, sizeof(unsigned) * 4));
    if (!ctx->coop_err_host) PM_CUDA(cudaMallocHost(&ctx->coop_err_host, sizeof(int)));
    ctx->coop_cap = nbox;
    return PM_OK;
}

// FP64 result of a box and its FP64 residual (sums to pinned host memory), eager.
static void box_confirm(Exec* x, BoxRun& B)
{
    Workspace* w = B.w;
    Level<double>& L0 = w->d[0];
    x->begin(PM_K_REDUCE);
    k_from_ff<<<grid_for(x, B.cells), kThreads, 0, x->stream>>>(ff_chi(w), B.cells, L0.u[0]);
    x->end();
    recentre<double>(x, L0.u[0], B.cells);
    L0.lamp = w->lam;
    residual<double, false, false>(x, L0, L0.u[0], B.delta, B.cf.src, 0.0, B.c, nullptr, nullptr);
    L0.lamp = nullptr;
    cudaMemcpyAsync(w->host, x->red_out, sizeof(double) * 9, cudaMemcpyDeviceToHost, x->stream);
}

// Host side of the stopping test from the sums of the last residual.
static void box_check(const pm_params& P, BoxRun& B, double tol)
{
    const double* h = B.w->host;
    const double gm = h[3] > 0.0 ? h[0] / h[3] : 0.0;
    const double r2 = h[2] - 2.0 * gm * h[1] + gm * gm * h[3];
    B.rr = B.fnorm > 0.0 ? std::sqrt(r2 > 0.0 ? r2 : 0.0) / B.fnorm : std::sqrt(r2 > 0.0 ? r2 : 0.0);
    if (B.cyc < 64) B.hist[B.cyc] = B.rr;
    if (h[4] > 0.0 || !std::isfinite(B.rr)) {
        B.st = PM_ERR_NONFINITE;
        B.active = false;
    } else if (B.rr <= tol || B.fnorm == 0.0) {
        B.st = PM_OK;
        B.active = false;
    } else if (B.cyc >= P.max_cycles) {
        B.st = PM_ERR_NOCONV;
        B.active = false;
    }
}

pm_status mg_solve_batched(pm_ctx* ctx, int nbox, const int* nn, const double* const* delta, const double* aB0,
                           const double* aM0, const double* aa, double tol, double* const* phi, pm_solve_info* infos)
{
    const pm_params& P = ctx->prm;
    if ((int)ctx->batch.size() < nbox) ctx->batch.resize(nbox, nullptr);
    std::vector<BoxRun> B(nbox);
    cudaEvent_t start, stop, ready;
    cudaEventCreate(&start);
    cudaEventCreate(&stop);
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventRecord(start, ctx->stream);
    cudaEventRecord(ready, ctx->stream);
    if (!ctx->batch_stream) PM_CUDA(cudaStreamCreateWithFlags(&ctx->batch_stream, cudaStreamNonBlocking));
    // per-box set-up, eager: workspaces, norms, first residual
    for (int b = 0; b < nbox; ++b) {
        BoxRun& R = B[b];
        coefficients(aB0[b], aM0[b], aa[b], P.omega_m0, P.include_dot_alphaB, &R.cf);
        R.cells = (size_t)nn[b] * nn[b] * nn[b];
        R.delta = delta[b];
        R.phi = phi[b];
        R.c = Coef{R.cf.nu, R.cf.kappa, P.eta, R.cf.src};
        if (R.cf.xi == 0.0) {
            R.trivial = true;
            R.st = PM_OK;
            PM_CUDA(cudaMemsetAsync(R.phi, 0, R.cells * sizeof(double), ctx->stream));
            continue;
        }
        if (R.cf.nu == 0.0 || !std::isfinite(R.cf.nu) || !std::isfinite(R.cf.kappa)) {
            ctx->set_error("box " + std::to_string(b) + ": nu = 0");
            return PM_ERR_INVALID_ARG;
        }
        Workspace*& w = ctx->batch[b];
        if (w && w->n != nn[b]) {
            delete_workspace(w);
            w = nullptr;
        }
        if (!w) {
            w = new Workspace();
            w->n = nn[b];
        }
        R.w = w;
        PM_TRY(ensure_mg(ctx, w, true));
        PM_TRY(box_prepare(ctx, w));
        PM_CUDA(cudaStreamWaitEvent(w->stream, ready, 0));
        Exec x(ctx, w->stream, w->partials, w->out, w->host, false);
        PM_TRY(source_norm(&x, R.delta, R.cells, R.cf.src, &R.fnorm));
        w->d[0].cur = 0;
        R.fk = make_ffcoef(R.cf.nu, R.cf.kappa, P.eta, nn[b]);
        PM_CUDA(cudaMemcpyAsync(w->d[0].u[0], R.phi, R.cells * sizeof(double), cudaMemcpyDeviceToDevice, w->stream));
        recentre<double>(&x, w->d[0].u[0], R.cells);
        x.begin(PM_K_REDUCE);
        k_to_ff<<<grid_for(&x, R.cells), kThreads, 0, w->stream>>>(R.delta, R.cf.src, R.cells, ff_rhs(w));
        x.end();
        x.begin(PM_K_REDUCE);
        k_to_ff<<<grid_for(&x, R.cells), kThreads, 0, w->stream>>>(w->d[0].u[0], 1.0, R.cells, ff_chi(w));
        x.end();
        PM_CUDA(cudaMemsetAsync(w->lam, 0, sizeof(double), w->stream));
        box_residual(&x, R);
        R.active = true;
    }
    for (int b = 0; b < nbox; ++b)
        if (B[b].active) PM_CUDA(cudaStreamSynchronize(B[b].w->stream));
    // a guess worse than chi = 0 (or non-finite) is replaced by zero, as in the single solve
    bool redo = false;
    for (int b = 0; b < nbox; ++b) {
        if (!B[b].active) continue;
        box_check(P, B[b], tol);
        B[b].guess_rr = B[b].st == PM_ERR_NONFINITE ? INFINITY : B[b].rr;
        if (!(B[b].guess_rr <= kGuessLimit)) {
            BoxRun& R = B[b];
            R.guess_rejected = true;
            R.st = PM_ERR_NOCONV;
            R.active = true;
            Exec x(ctx, R.w->stream, R.w->partials, R.w->out, R.w->host, false);
            PM_CUDA(cudaMemsetAsync(ff_chi(R.w), 0, R.cells * sizeof(float2), R.w->stream));
            PM_CUDA(cudaMemsetAsync(R.w->lam, 0, sizeof(double), R.w->stream));
            box_residual(&x, R);
            redo = true;
        }
    }
    if (redo)
        for (int b = 0; b < nbox; ++b)
            if (B[b].guess_rejected) {
                PM_CUDA(cudaStreamSynchronize(B[b].w->stream));
                box_check(P, B[b], tol);
            }
    // first iteration eagerly on the boxes' own streams (the autotuner runs here)
    for (int b = 0; b < nbox; ++b) {
        if (!B[b].active) continue;
        Exec x(ctx, B[b].w->stream, B[b].w->partials, B[b].w->out, B[b].w->host, false);
        box_iteration(&x, B[b]);
    }
    for (int b = 0; b < nbox; ++b)
        if (B[b].active) {
            PM_CUDA(cudaStreamSynchronize(B[b].w->stream));
            ++B[b].cyc;
            B[b].vcyc += P.inner_cycles;
            box_check(P, B[b], tol);
        }
    // graph-captured iterations.  The boxes still active after the eager iteration are captured
    // once, each box's kernel, memset and memcpy nodes recorded; a box that converges later has
    // its nodes disabled in the executable graph (cudaGraphNodeSetEnabled) instead of a new
    // capture and instantiation of the remaining boxes.
    // the executable graph and the captured graph (kept until the end: its nodes name the
    // executable graph's nodes), released on every return path
    struct GraphHold {
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t graph = nullptr;
        ~GraphHold()
        {
            if (exec) cudaGraphExecDestroy(exec);
            if (graph) cudaGraphDestroy(graph);
        }
    } hold;
    cudaGraphExec_t& exec = hold.exec;
    cudaGraph_t& graph = hold.graph;
    std::vector<std::vector<cudaGraphNode_t>> box_nodes(nbox);
    std::vector<pm_profile> box_prof(nbox);
    std::vector<char> enabled(nbox, 0);
    // the boxes whose levels 32^3 .. 4^3 run in the cooperative kernel, and their table
    std::vector<int> coop_idx(nbox, -1);
    int ncoop = 0;
    long long coop_launches = 0;
    if (P.batch_persistent && !P.coarse_exact && P.coarsest_n == 4 && P.inner_cycles == 1) {
        std::vector<CoopBox> tab;
        for (int b = 0; b < nbox; ++b) {
            if (!B[b].active || nn[b] < 2 * kCoopTop) continue;
            Workspace* w = B[b].w;
            const int l32 = coop_level(nn[b]);
            if ((int)w->s.size() != l32 + kCoopLevels) continue;
            CoopBox cb{};
            bool ok = true;
            for (int k = 0; k < kCoopLevels; ++k) {
                Level<float>& L = w->s[l32 + k];
                cb.lv[k] = CoopLevel{{L.u[0], L.u[1]}, L.f, L.r, L.ur, L.bg, L.kmask, L.sat, L.n};
                ok = ok && L.u[0] && L.u[1] && L.f && L.r && L.ur && L.bg && L.kmask && L.sat && L.n == (kCoopTop >> k);
            }
            if (!ok) continue;  // not the level set the kernel expects: this box keeps per-box launches
            cb.nu = (float)B[b].c.nu;
            cb.kap = (float)B[b].c.kap;
            cb.nu_d = B[b].c.nu;
            cb.kap_d = B[b].c.kap;
            coop_idx[b] = ncoop++;
            tab.push_back(cb);
        }
        if (ncoop > 0) {
            PM_TRY(coop_alloc(ctx, ncoop));
            PM_CUDA(cudaMemcpy(ctx->coop_boxes, tab.data(), sizeof(CoopBox) * ncoop, cudaMemcpyHostToDevice));
        }
    }
    {
        std::vector<int> act;
        for (int b = 0; b < nbox; ++b)
            if (B[b].active) act.push_back(b);
        // if the cooperative launch cannot be captured, capture again without it
        for (int attempt = 0; attempt < 2 && !act.empty() && !exec; ++attempt) {
            if (attempt == 1) {
                if (ncoop == 0) break;
                ncoop = 0;
                for (int b = 0; b < nbox; ++b) {
                    coop_idx[b] = -1;
                    box_nodes[b].clear();
                    box_prof[b] = pm_profile{};
                }
                coop_launches = 0;
            }
            const pm_profile before = ctx->prof;
            cudaStream_t ms = ctx->batch_stream;
            cudaEvent_t fork;
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
            PM_CUDA(cudaStreamBeginCapture(ms, cudaStreamCaptureModeThreadLocal));
            cudaEventRecord(fork, ms);
            cudaGraph_t cg = nullptr;
            cudaStreamCaptureStatus cs;
            cudaStreamGetCaptureInfo(ms, &cs, nullptr, &cg, nullptr, nullptr, nullptr);
            std::set<cudaGraphNode_t> seen;
            auto new_nodes = [&](std::vector<cudaGraphNode_t>& out) {
                size_t nn = 0;
                cudaGraphGetNodes(cg, nullptr, &nn);
                std::vector<cudaGraphNode_t> all(nn);
                cudaGraphGetNodes(cg, all.data(), &nn);
                for (auto nd : all) {
                    if (!seen.insert(nd).second) continue;
                    cudaGraphNodeType ty;
                    cudaGraphNodeGetType(nd, &ty);
                    if (ty == cudaGraphNodeTypeKernel || ty == cudaGraphNodeTypeMemset || ty == cudaGraphNodeTypeMemcpy)
                        out.push_back(nd);
                }
            };
            std::vector<cudaGraphNode_t> dummy;
            new_nodes(dummy);  // the fork
            std::vector<cudaEvent_t> joins;
            auto join_into_ms = [&](cudaStream_t st) {
                cudaEvent_t join;
                cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
                cudaEventRecord(join, st);
                cudaStreamWaitEvent(ms, join, 0);
                joins.push_back(join);
            };
            auto add_prof = [&](int b, const pm_profile& pb) {
                for (int k = 0; k < PM_K_COUNT; ++k) {
                    box_prof[b].launches[k] += ctx->prof.launches[k] - pb.launches[k];
                    box_prof[b].fine_launches[k] += ctx->prof.fine_launches[k] - pb.fine_launches[k];
                    box_prof[b].cells[k] += ctx->prof.cells[k] - pb.cells[k];
                }
            };
            // down: the coarse-kernel boxes to their 32^3 level, every other box a whole iteration
            for (int b : act) {
                Workspace* w = B[b].w;
                const pm_profile pb = ctx->prof;
                cudaStreamWaitEvent(w->stream, fork, 0);
                Exec x(ctx, w->stream, w->partials, w->out, w->host, false);
                if (coop_idx[b] >= 0) box_down(&x, B[b], coop_level(nn[b]));
                else box_iteration(&x, B[b]);
                join_into_ms(w->stream);
                new_nodes(box_nodes[b]);
                add_prof(b, pb);
                enabled[b] = 1;
            }
            if (ncoop > 0) {
                // the coarse levels of every box in one cooperative launch
                cudaMemsetAsync(ctx->coop_bar, 0, sizeof(unsigned) * 4, ms);  // errors surface at the end of capture
                CoopParams cp{};
                cp.boxes = reinterpret_cast<const CoopBox*>(ctx->coop_boxes);
                cp.active = ctx->coop_active;
                cp.nbox = ncoop;
                cp.npre = P.npre;
                cp.npost = P.npost;
                cp.coarse_sweeps = P.coarse_sweeps;
                cp.eta = P.eta;
                cp.partials = ctx->coop_partials;
                cp.gm = ctx->coop_gm;
                cp.bar = ctx->coop_bar;
                cp.err = reinterpret_cast<int*>(ctx->coop_bar + 2);
                int khz = 0;
                cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, ctx->device);
                cp.spin_limit = (long long)(ctx->coop_wait_s * (double)(khz > 0 ? khz : 2000000) * 1e3);
                cp.fail_block = ctx->coop_fail_block;
                cp.fail_barrier = ctx->coop_fail_barrier;
                int per_sm = 0;
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_coarse, kCoopThreads, 0);
                int grid = ctx->num_sms * (per_sm < 2 ? per_sm : 2);
                if (grid < 1) grid = 1;
                cudaLaunchConfig_t lc{};
                lc.gridDim = dim3(grid);
                lc.blockDim = dim3(kCoopThreads);
                lc.dynamicSmemBytes = 0;
                lc.stream = ms;
                cudaLaunchAttribute at[1];
                at[0].id = cudaLaunchAttributeCooperative;
                at[0].val.cooperative = 1;
                lc.attrs = at;
                lc.numAttrs = 1;
                ctx->prof.launches[PM_K_TRANSFER] += 1;
                coop_launches += 1;
                if (cudaLaunchKernelEx(&lc, k_batch_coarse, cp) != cudaSuccess) cudaGetLastError();
                cudaMemcpyAsync(ctx->coop_err_host, ctx->coop_bar + 2, sizeof(int), cudaMemcpyDeviceToHost, ms);
                {
                    std::vector<cudaGraphNode_t> shared;  // the memset, kernel and copy belong to no box
                    new_nodes(shared);
                }
                cudaEvent_t fork2;
                cudaEventCreateWithFlags(&fork2, cudaEventDisableTiming);
                cudaEventRecord(fork2, ms);
                joins.push_back(fork2);
                const int cur32 = (P.npre + P.npost) & 1;
                for (int b : act) {
                    if (coop_idx[b] < 0) continue;
                    Workspace* w = B[b].w;
                    const pm_profile pb = ctx->prof;
                    cudaStreamWaitEvent(w->stream, fork2, 0);
                    Exec x(ctx, w->stream, w->partials, w->out, w->host, false);
                    box_up(&x, B[b], coop_level(nn[b]), cur32);
                    join_into_ms(w->stream);
                    new_nodes(box_nodes[b]);
                    add_prof(b, pb);
                }
            }
            cudaGraph_t g = nullptr;
            cudaError_t ce = cudaStreamEndCapture(ms, &g);
            for (auto e : joins) cudaEventDestroy(e);
            cudaEventDestroy(fork);
            ctx->prof = before;  // capture launched nothing; replays are counted below
            if (ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                if (attempt == 0 && ncoop > 0) continue;
                ctx->set_error(std::string("graph capture failed: ") + cudaGetErrorString(ce));
                return PM_ERR_CUDA;
            }
            graph = g;
            PM_CUDA(cudaGraphInstantiate(&exec, g, 0));
        }
    }
    for (;;) {
        std::vector<int> act;
        for (int b = 0; b < nbox; ++b)
            if (B[b].active) act.push_back(b);
        if (act.empty() || !exec) break;
        for (int b = 0; b < nbox; ++b)
            if (enabled[b] && !B[b].active) {
                for (auto nd : box_nodes[b]) PM_CUDA(cudaGraphNodeSetEnabled(exec, nd, 0));
                enabled[b] = 0;
            }
        if (ncoop > 0) {
            for (int b = 0; b < nbox; ++b)
                if (coop_idx[b] >= 0) ctx->coop_active_host[coop_idx[b]] = B[b].active ? 1 : 0;
            PM_CUDA(cudaMemcpyAsync(ctx->coop_active, ctx->coop_active_host, sizeof(int) * ncoop,
                                    cudaMemcpyHostToDevice, ctx->batch_stream));
        }
        PM_CUDA(cudaGraphLaunch(exec, ctx->batch_stream));
        PM_CUDA(cudaStreamSynchronize(ctx->batch_stream));
        if (ncoop > 0) {
            ctx->prof.launches[PM_K_TRANSFER] += coop_launches;
            const int e = *ctx->coop_err_host;
            if (e == PM_ERR_TIMEOUT) {
                ctx->set_error("batched solve: a grid barrier wait of the persistent coarse-level kernel gave up");
                return PM_ERR_TIMEOUT;
            }
            if (e != PM_OK) {
                ctx->set_error("batched solve: the persistent coarse-level kernel rejected its box table");
                return PM_ERR_CUDA;
            }
        }
        for (int b : act) {
            for (int k = 0; k < PM_K_COUNT; ++k) {
                ctx->prof.launches[k] += box_prof[b].launches[k];
                ctx->prof.fine_launches[k] += box_prof[b].fine_launches[k];
                ctx->prof.cells[k] += box_prof[b].cells[k];
            }
            ++B[b].cyc;
            B[b].vcyc += P.inner_cycles;
            box_check(P, B[b], tol);
        }
    }
    // FP64 result of every box; a converged box's stop test is confirmed by its FP64
    // residual (a box that misses it by rounding gets further outer iterations, eagerly)
    for (int b = 0; b < nbox; ++b) {
        if (B[b].trivial || !B[b].w) continue;
        BoxRun& R = B[b];
        Exec x(ctx, R.w->stream, R.w->partials, R.w->out, R.w->host, false);
        for (;;) {
            box_confirm(&x, R);
            PM_CUDA(cudaStreamSynchronize(R.w->stream));
            if (R.st != PM_OK) break;
            double gm64 = 0.0;
            const double rr64 = rel_from_sums(R.w->host, R.fnorm, &gm64);
            if (rr64 <= tol || R.fnorm == 0.0) {
                R.rr = rr64;
                R.lam_fix = gm64;
                break;
            }
            if (R.cyc >= P.max_cycles) {
                R.st = PM_ERR_NOCONV;
                break;
            }
            R.active = true;
            box_iteration(&x, R);
            PM_CUDA(cudaStreamSynchronize(R.w->stream));
            ++R.cyc;
            R.vcyc += P.inner_cycles;
            R.st = PM_ERR_NOCONV;
            box_check(P, R, tol);
        }
    }
    // results back to the callers' buffers, ordered after everything on the context stream
    for (int b = 0; b < nbox; ++b) {
        if (B[b].trivial) continue;
        Workspace* w = B[b].w;
        PM_CUDA(cudaMemcpyAsync(B[b].phi, w->d[0].u[0], B[b].cells * sizeof(double), cudaMemcpyDeviceToDevice,
                                w->stream));
        double lam = 0.0;
        PM_CUDA(cudaMemcpyAsync(&lam, w->lam, sizeof(double), cudaMemcpyDeviceToHost, w->stream));
        PM_CUDA(cudaStreamSynchronize(w->stream));
        if (infos) {
            pm_solve_info& I = infos[b];
            I = pm_solve_info{};
            I.cycles = B[b].cyc;
            I.vcycles = B[b].vcyc;
            I.status = B[b].st;
            I.rel_res = B[b].rr;
            I.lambda = lam - B[b].lam_fix;
            I.floored_cells = (long long)((double)B[b].cells - w->host[3]);
            I.unstable_nu = B[b].cf.nu <= 0.0;
            for (int k = 0; k < 64; ++k) I.rel_res_hist[k] = B[b].hist[k];
            I.guess_rel_res = B[b].guess_rr;
            I.guess_rejected = B[b].guess_rejected ? 1 : 0;
        }
    }
    cudaEventRecord(stop, ctx->stream);
    cudaEventSynchronize(stop);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, start, stop);
    cudaEventDestroy(start);
    cudaEventDestroy(stop);
    cudaEventDestroy(ready);
    pm_status worst = PM_OK;
    for (int b = 0; b < nbox; ++b) {
        if (infos) infos[b].ms_total = ms;
        if (B[b].st != PM_OK && worst == PM_OK) worst = B[b].st;
    }
    if (worst == PM_ERR_NOCONV) ctx->set_error("a box reached max_cycles before the tolerance");
    if (worst == PM_ERR_NONFINITE) ctx->set_error("non-finite residual in a box");
    return worst;
}

}  // namespace pmeft
