// solve.cu -- pr_solve: the fused sweep driven to convergence on the device.
//
// The loop runs inside a CUDA graph whose WHILE node repeats the sweep kernel
// until the sweep's last block clears the condition (error <= threshold or
// max_iter sweeps); the host synchronises once per solve.  A host-driven loop
// (use_graph = 0) launches the same kernel in batches and polls the state.
// Defect-correction precisions are driven from dc.cu.
#include <string.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "solve_impl.cuh"
#include "sweep.cuh"

namespace fpr {

pr_status validate_options(const pr_options *o)
{
    if (!o) {
        set_error("options are NULL");
        return PR_ERR_INVALID_ARG;
    }
    if (!(o->d >= 0.0 && o->d < 1.0)) {
        set_error("d must lie in [0, 1)");
        return PR_ERR_INVALID_ARG;
    }
    if (o->max_iter < 1 || !(o->threshold >= 0.0) || std::isnan(o->threshold)) {
        set_error("need max_iter >= 1 and threshold >= 0");
        return PR_ERR_INVALID_ARG;
    }
    if (o->variant != PR_JACOBI && o->variant != PR_FUSED_GS) {
        set_error("unknown variant");
        return PR_ERR_INVALID_ARG;
    }
    if (o->precision < PR_FP64 || o->precision > PR_FP16_DC) {
        set_error("unknown precision");
        return PR_ERR_INVALID_ARG;
    }
    if (o->norm != PR_NORM_L1 && o->norm != PR_NORM_LINF) {
        set_error("unknown norm");
        return PR_ERR_INVALID_ARG;
    }
    if (!(o->perforate_eps >= 0.0) || std::isinf(o->perforate_eps) || o->perforate_period < 0) {
        set_error("need perforate_eps >= 0 (finite) and perforate_period >= 0");
        return PR_ERR_INVALID_ARG;
    }
    return PR_OK;
}

pr_status check_device(pr_graph *g)
{
    int dev = -1;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev != g->device) {
        set_error("graph lives on device %d, current device is %d", g->device, dev);
        return PR_ERR_INVALID_ARG;
    }
    return PR_OK;
}

pr_status ensure_workspace(pr_graph *g, cudaStream_t s)
{
    const size_t n = (size_t)g->n;
    PR_TRY(buf_alloc(g, g->ybuf, 2 * n * sizeof(double) + 512, s));
    return PR_OK;
}

// static shared memory of a sweep block (partial sums) plus slack
constexpr int SWEEP_STATIC_SMEM = 2048;

void fill_params(pr_graph *g, SweepParams &p, bool fp64, size_t elem, bool perf)
{
    Items &it = g->items;
    memset(&p, 0, sizeof(p));
    p.n = g->n;
    p.col_ptr = g->r_col_ptr.as<int32_t>();
    p.row_idx = g->r_row_idx.as<int32_t>();
    p.outdeg = g->r_outdeg.as<int32_t>();
    p.inv = fp64 ? g->r_inv64.p : g->r_inv32.p;
    p.ew = g->weighted ? (fp64 ? g->p64_csc.p : g->p32_csc.p) : nullptr;
    p.nhub = it.nhub;
    p.desc = it.desc.as<int4>();
    p.nhubseg = it.nhubseg;
    p.hubseg_start = it.hubseg_start.as<int32_t>();
    p.seg_acc = it.seg_acc.as<double>();
    p.hub_cnt = it.hub_cnt.as<int32_t>();
    for (int k = 0; k < 5; ++k) p.mi[k] = it.mi[k];
    p.nlt = it.nlt;
    p.lcap = it.lcap;
    // staged copy of stage_kb KB, at most the room left beside the warp
    // slices (shared memory is taken from the L1 cache, which also keeps hot
    // contributions, so a modest copy serves best)
    const Layout L0 = make_layout(p.lcap, fp64 ? 8 : 4, (int)elem, perf, 0);
    int64_t stage = ((int64_t)g->max_smem - L0.total - SWEEP_STATIC_SMEM) / (int64_t)elem;
    stage = it.stage_kb > 0 ? std::min<int64_t>(stage, (int64_t)it.stage_kb * 1024 / elem) : 0;
    p.stage = (int32_t)std::max<int64_t>(0, std::min<int64_t>(g->n, stage));
    p.item_lo = 0;
    p.item_hi = it.nhubseg + it.mi[4] + it.nlt;
    p.close = 1;
    p.wait_limit = (uint32_t)it.wait_limit;
    p.test_stall = it.test_stall;
    p.y0 = g->ybuf.p;
    p.y1 = static_cast<char *>(g->ybuf.p) + ((g->n * elem + 255) & ~(size_t)255);
    p.st = g->state.as<SolveState>();
}

// SWEEP_MINB persistent blocks of SWEEP_BS threads per SM (fewer if there are
// fewer items than warps); 0 with the error set if the shared memory does
// not fit.
unsigned sweep_grid(const pr_graph *g, int nitems, const void *func, size_t smem)
{
    if (smem + SWEEP_STATIC_SMEM > (size_t)g->max_smem) {
        set_error("a sweep block needs %zu bytes of shared memory (limit %d): use a smaller "
                  "tile or t_lo",
                  smem + SWEEP_STATIC_SMEM, g->max_smem);
        return 0;
    }
    cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    const int grid = std::min((nitems + SWEEP_WARPS - 1) / SWEEP_WARPS, g->num_sms * SWEEP_MINB);
    return (unsigned)std::max(grid, 1);
}

template <typename T, typename A>
static const void *pick_sweep(bool gs, bool weighted)
{
    if (gs)
        return weighted ? reinterpret_cast<const void *>(&k_sweep<T, A, true, true>)
                        : reinterpret_cast<const void *>(&k_sweep<T, A, true, false>);
    return weighted ? reinterpret_cast<const void *>(&k_sweep<T, A, false, true>)
                    : reinterpret_cast<const void *>(&k_sweep<T, A, false, false>);
}

template <typename T, typename A>
pr_status make_plan(pr_graph *g, const SweepParams &p, bool gs, SweepPlan &plan)
{
    plan.func = pick_sweep<T, A>(gs, p.ew != nullptr);
    plan.smem = layout_of<T, A, false>(p).total;
    // fused sweep: the hottest items (hub segments and the widest mid
    // groups) first, so the rest reads their new values; one launch only
    // where pr_tune.fused_split asks for it
    const int total = p.nhubseg + p.mi[4] + p.nlt;
    const int split = p.nhubseg + p.mi[1];
    const bool one = g->items.fused_split == 2;
    if (gs && !one && split > 0 && split < total) {
        plan.nlaunch = 2;
        plan.p[0] = p;
        plan.p[0].item_lo = 0;
        plan.p[0].item_hi = split;
        plan.p[0].close = 0;
        // 4- and 2-byte stored vectors: the first launch's vertices,
        // [0, mb[1]), write their new values to y1 (so that launch gathers
        // from an array nobody writes) and a copy puts them into y0 before
        // the second launch; FP64 sweeps update in place (the copy bought
        // them no time and cost two sweeps)
        if (sizeof(T) < 8) {
            plan.p[0].write_alt = 1;
            plan.copy_func = reinterpret_cast<const void *>(&k_copy_front<T>);
            plan.copy_n = g->items.mb[1];
            plan.copy_grid =
                (unsigned)std::max(1, std::min((plan.copy_n + 255) / 256, g->num_sms * 4));
            plan.copy_st = p.st;
            plan.copy_src = p.y1;
            plan.copy_dst = p.y0;
        }
        plan.p[1] = p;
        plan.p[1].item_lo = split;
        plan.p[1].item_hi = total;
        plan.p[1].close = 1;
        plan.grid[0] = sweep_grid(g, split, plan.func, plan.smem);
        plan.grid[1] = sweep_grid(g, total - split, plan.func, plan.smem);
    } else {
        plan.nlaunch = 1;
        plan.p[0] = p;
        plan.p[0].item_lo = 0;
        plan.p[0].item_hi = total;
        plan.p[0].close = 1;
        plan.grid[0] = sweep_grid(g, total, plan.func, plan.smem);
        plan.grid[1] = 1;
    }
    if (plan.grid[0] == 0 || plan.grid[1] == 0) return PR_ERR_INVALID_ARG;
    return PR_OK;
}
template pr_status make_plan<double, double>(pr_graph *, const SweepParams &, bool, SweepPlan &);
template pr_status make_plan<float, float>(pr_graph *, const SweepParams &, bool, SweepPlan &);
template pr_status make_plan<__nv_bfloat16, float>(pr_graph *, const SweepParams &, bool,
                                                   SweepPlan &);
template pr_status make_plan<__half, float>(pr_graph *, const SweepParams &, bool, SweepPlan &);

pr_status add_plan_nodes(cudaGraph_t body, SweepPlan &plan, cudaGraphConditionalHandle h,
                         cudaGraphNode_t *last)
{
    cudaGraphNode_t prev = nullptr;
    for (int k = 0; k < plan.nlaunch; ++k) {
        plan.p[k].cond = h;
        plan.p[k].use_cond = 1;
        void *args[] = {&plan.p[k]};
        cudaKernelNodeParams kp = {};
        kp.func = const_cast<void *>(plan.func);
        kp.gridDim = dim3(plan.grid[k]);
        kp.blockDim = dim3(plan.block);
        kp.sharedMemBytes = (unsigned)plan.smem;
        kp.kernelParams = args;
        cudaGraphNode_t node;
        PR_CUDA(cudaGraphAddKernelNode(&node, body, prev ? &prev : nullptr, prev ? 1 : 0, &kp));
        prev = node;
        if (k == 0 && plan.nlaunch > 1 && plan.copy_func) {
            void *cargs[] = {&plan.copy_st, &plan.copy_src, &plan.copy_dst, &plan.copy_n};
            cudaKernelNodeParams cp = {};
            cp.func = const_cast<void *>(plan.copy_func);
            cp.gridDim = dim3(plan.copy_grid);
            cp.blockDim = dim3(256);
            cp.kernelParams = cargs;
            PR_CUDA(cudaGraphAddKernelNode(&node, body, &prev, 1, &cp));
            prev = node;
        }
    }
    if (last) *last = prev;
    return PR_OK;
}

pr_status launch_plan(SweepPlan &plan, cudaStream_t s)
{
    for (int k = 0; k < plan.nlaunch; ++k) {
        plan.p[k].use_cond = 0;
        void *args[] = {&plan.p[k]};
        PR_CUDA(cudaLaunchKernel(plan.func, dim3(plan.grid[k]), dim3(plan.block), args,
                                 plan.smem, s));
        note_launch();
        if (k == 0 && plan.nlaunch > 1 && plan.copy_func) {
            void *cargs[] = {&plan.copy_st, &plan.copy_src, &plan.copy_dst, &plan.copy_n};
            PR_CUDA(cudaLaunchKernel(plan.copy_func, dim3(plan.copy_grid), dim3(256), cargs, 0, s));
            note_launch();
        }
    }
    return PR_OK;
}

void release_graphs(pr_graph *g)
{
    for (auto &c : g->graphs) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        if (c.graph) cudaGraphDestroy(c.graph);
    }
    g->graphs.clear();
}

pr_status loop_graph(pr_graph *g, int key, SweepPlan &plan, cudaGraphExec_t *exec_out)
{
    for (auto &c : g->graphs)
        if (c.key == key) {
            *exec_out = c.exec;
            return PR_OK;
        }
    cudaGraph_t graph = nullptr;
    PR_CUDA(cudaGraphCreate(&graph, 0));
    cudaGraphConditionalHandle h;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_status(e, "cudaGraphConditionalHandleCreate", __FILE__, __LINE__);
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cnode;
    e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_status(e, "cudaGraphAddNode(while)", __FILE__, __LINE__);
    }
    pr_status st = add_plan_nodes(cp.conditional.phGraph_out[0], plan, h, nullptr);
    if (st != PR_OK) {
        cudaGraphDestroy(graph);
        return st;
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_status(e, "loop graph", __FILE__, __LINE__);
    }
    pr_graph::Cached c;
    c.key = key;
    c.exec = exec;
    c.graph = graph;
    g->graphs.push_back(c);
    *exec_out = exec;
    return PR_OK;
}

void init_state(pr_graph *g, const pr_options *o, SolveState &h)
{
    memset(&h, 0, sizeof(h));
    h.norm = o->norm;
    h.max_iter = o->max_iter;
    h.tau = o->threshold;
    h.d = o->d;
    h.base = (1.0 - o->d) / (double)g->n;
    h.inv_n = 1.0 / (double)g->n;
    h.sigma = 1.0;
    h.history = o->history;
    h.record = o->history != nullptr;
    h.status = PR_NOT_CONVERGED;
}

pr_status finish_result(pr_graph *g, pr_result *res, cudaStream_t s, int outer)
{
    PR_CUDA(cudaMemcpyAsync(g->host_state, g->state.p, sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    const SolveState &h = *g->host_state;
    pr_status st = (pr_status)h.status;
    if (res) {
        res->iters = h.iter;
        res->outer_iters = outer ? h.outer_iter : 0;
        res->residual = h.norm ? h.resmax : h.res;
        res->sum_before_norm = h.sigma * h.sum;
        res->status = st;
    }
    return st;
}

// Runs the sweep loop for precision T (plain forms).
template <typename T, typename A>
static pr_status solve_plain(pr_graph *g, const pr_options *o, const pr_tune &tn, double *x_out,
                             pr_result *res, cudaStream_t s)
{
    constexpr bool fp64 = sizeof(A) == 8;
    const bool gs = o->variant == PR_FUSED_GS;
    const bool serial = gs && tn.deterministic_gs;
    const bool weighted = g->weighted;
    if (serial && (g->n > 65536 || !fp64 || weighted)) {
        set_error("the deterministic fused sweep needs FP64, an unweighted graph and n <= 65536");
        return PR_ERR_UNSUPPORTED;
    }
    const bool perf = o->perforate_eps > 0.0;
    if (perf && (gs || weighted)) {
        set_error("loop perforation needs the Jacobi sweep and an unweighted graph");
        return PR_ERR_UNSUPPORTED;
    }
    SweepParams p;
    fill_params(g, p, fp64, sizeof(T), perf);
    const int32_t *n2o = g->n2o.as<int32_t>();
    const int32_t *o2n = g->o2n.as<int32_t>();
    if (serial) {  // strict Eq. 9 order on the input ids
        p.col_ptr = g->col_ptr.as<int32_t>();
        p.row_idx = g->row_idx.as<int32_t>();
        p.outdeg = g->outdeg.as<int32_t>();
        p.inv = g->inv64.p;
        n2o = o2n = nullptr;
    }
    p.renorm = (gs && !o->no_rescale) ? 1 : 0;
    SweepPlan plan;
    if (serial) {
        plan.func = reinterpret_cast<const void *>(&k_sweep_serial<T, A>);
        plan.nlaunch = 1;
        plan.p[0] = p;
        plan.grid[0] = 1;
        plan.block = 32;
    } else if (perf) {
        PR_TRY(buf_alloc(g, g->lastbuf, (size_t)g->n * sizeof(A) + 256, s));
        p.last = g->lastbuf.p;
        plan.func = reinterpret_cast<const void *>(&k_sweep_perf<T, A>);
        plan.smem = layout_of<T, A, true>(p).total;
        plan.nlaunch = 1;
        plan.p[0] = p;
        plan.grid[0] = sweep_grid(g, p.item_hi, plan.func, plan.smem);
        if (plan.grid[0] == 0) return PR_ERR_INVALID_ARG;
    } else {
        PR_TRY((make_plan<T, A>(g, p, gs, plan)));
    }
    SolveState *hs = g->host_state;
    init_state(g, o, *hs);
    hs->perf = perf ? 1 : 0;
    hs->perf_period = o->perforate_period;
    hs->perf_eps = o->perforate_eps;
    PR_CUDA(cudaMemcpyAsync(g->state.p, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int ib = std::max(1, std::min<int>((g->n + 255) / 256, g->num_sms * 8));
    k_init<T, A><<<ib, 256, 0, s>>>(g->n, o->x0, n2o, p.outdeg, static_cast<const A *>(p.inv),
                                   static_cast<T *>(p.y0), p.st, p.renorm, weighted ? 1 : 0);
    note_launch();
    PR_LAUNCH_CHECK();

    bool graph_loop = false;
    if (o->use_graph) {
        const int key = (fp64 ? 1 : 0) | (gs ? 2 : 0) | (serial ? 4 : 0) | (weighted ? 8 : 0) |
                        (g->items.test_stall ? 32 : 0) | (p.renorm ? 128 : 0) |
                        (perf ? 256 : 0);
        cudaGraphExec_t exec;
        PR_TRY(loop_graph(g, key, plan, &exec));
        PR_CUDA(cudaGraphLaunch(exec, s));
        graph_loop = true;
    } else {
        int launched = 0;
        while (launched < o->max_iter) {
            const int batch = std::min(16, o->max_iter - launched);
            for (int k = 0; k < batch; ++k) PR_TRY(launch_plan(plan, s));
            launched += batch;
            PR_CUDA(cudaMemcpyAsync(g->host_state, g->state.p, sizeof(SolveState),
                                    cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (g->host_state->done) break;
        }
    }
    k_output<T><<<ib, 256, 0, s>>>(g->n, o2n, p.outdeg, static_cast<const T *>(p.y0),
                                   static_cast<const T *>(p.y1), gs ? 0 : 1, p.st, x_out,
                                   weighted ? 1 : 0);
    note_launch();
    PR_LAUNCH_CHECK();
    pr_status st = finish_result(g, res, s, 0);
    if (res) res->gathered = perf ? (int64_t)g->host_state->gathered : (int64_t)res->iters * g->m;
    // loop sweeps + the launch that sees the stop flag
    if (graph_loop) note_launch((uint64_t)plan_launches(plan) * (g->host_state->iter + 1));
    return st;
}

pr_status prepare_solve(pr_graph *g, const pr_options *o, pr_tune &tn, cudaStream_t s)
{
    PR_TRY(validate_options(o));
    PR_TRY(check_device(g));
    tn = effective_tune(g, o->tune);
    const Items &it = g->items;
    if (it.t_lo != tn.t_lo || it.t_hub != tn.t_hub || it.hub_seg != tn.hub_seg ||
        it.tile_c != tn.tile || it.stage_kb != tn.stage_kb || it.wait_limit != tn.wait_limit ||
        it.test_stall != test_stall_requested() || it.fused_split != tn.fused_split ||
        it.mid_wide != tn.mid_wide)
        release_graphs(g);  // cached loops hold the old launch parameters
    PR_TRY(ensure_items(g, tn, s));
    PR_TRY(ensure_workspace(g, s));
    return PR_OK;
}

}  // namespace fpr

using namespace fpr;

extern "C" pr_status pr_options_default(pr_options *o)
{
    if (!o) {
        set_error("pr_options_default: NULL");
        return PR_ERR_INVALID_ARG;
    }
    memset(o, 0, sizeof(*o));
    o->d = 0.85;
    o->threshold = 1e-10;
    o->max_iter = 1000;
    o->variant = PR_JACOBI;
    o->precision = PR_FP64;
    o->norm = PR_NORM_L1;
    o->use_graph = 1;
    return PR_OK;
}

extern "C" pr_status pr_solve(pr_graph *g, const pr_options *o, double *x_out, pr_result *res,
                              void *stream)
{
    if (res) memset(res, 0, sizeof(*res));
    if (!g || !x_out) {
        set_error("pr_solve: graph and x_out are required");
        return PR_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pr_tune tn;
    PR_TRY(prepare_solve(g, o, tn, s));
    if (tn.blocking) return solve_blocked(g, o, x_out, res, s);
    if (o->perforate_eps > 0.0 && o->precision != PR_FP64 && o->precision != PR_FP32) {
        set_error("loop perforation needs PR_FP64 or PR_FP32");
        return PR_ERR_UNSUPPORTED;
    }
    switch (o->precision) {
    case PR_FP64: return solve_plain<double, double>(g, o, tn, x_out, res, s);
    case PR_FP32: return solve_plain<float, float>(g, o, tn, x_out, res, s);
    default: return solve_dc(g, o, tn, x_out, res, s);
    }
}

extern "C" const char *pr_status_string(pr_status s)
{
    switch (s) {
    case PR_OK: return "ok";
    case PR_ERR_INVALID_ARG: return "invalid argument";
    case PR_ERR_OOM: return "out of device memory";
    case PR_ERR_CUDA: return "CUDA error";
    case PR_NOT_CONVERGED: return "not converged (max_iter reached)";
    case PR_ERR_TIMEOUT: return "device wait timed out";
    case PR_ERR_UNSUPPORTED: return "unsupported option combination";
    case PR_ERR_NUMERIC: return "non-finite value in the iterate";
    }
    return "unknown status";
}
