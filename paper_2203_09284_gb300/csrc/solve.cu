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

// ------------------------------------------------------------- helpers
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
    PR_TRY(buf_alloc(g, g->ybuf, 2 * n * sizeof(double) + 256, s));
    return PR_OK;
}

void fill_params(pr_graph *g, SweepParams &p, bool fp64, cudaStream_t)
{
    Items &it = g->items;
    memset(&p, 0, sizeof(p));
    p.n = g->n;
    p.col_ptr = g->col_ptr.as<int32_t>();
    p.row_idx = g->row_idx.as<int32_t>();
    p.outdeg = g->outdeg.as<int32_t>();
    p.inv = fp64 ? g->inv64.p : g->inv32.p;
    p.bins = it.bins.as<int32_t>();
    p.nlow = it.nlow;
    p.nmid = it.nmid;
    p.nhub = it.nhub;
    p.hubseg_start = it.hubseg_start.as<int32_t>();
    p.nhubseg = it.nhubseg;
    p.hub_seg = it.hub_seg;
    p.seg_acc = it.seg_acc.as<double>();
    p.hub_cnt = it.hub_cnt.as<int32_t>();
    p.low_rounds = it.low_rounds;
    p.mid_per_warp = it.mid_per_warp;
    p.mid_blocks = it.mid_blocks(SWEEP_BS);
    p.low_blocks = it.low_blocks(SWEEP_BS);
    p.y0 = g->ybuf.p;
    p.y1 = static_cast<char *>(g->ybuf.p) + ((g->n * (size_t)(fp64 ? 8 : 4) + 255) & ~(size_t)255);
    p.st = g->state.as<SolveState>();
}

// Persistent grid: as many resident blocks as the kernel allows on every SM,
// capped by the number of work items.
unsigned sweep_grid(const pr_graph *g, const SweepParams &p, const void *func)
{
    const int nitems = p.nhubseg + p.mid_blocks + p.low_blocks;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, func, SWEEP_BS, 0) != cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        per_sm = 1;
    }
    const int grid = std::min(nitems, per_sm * g->num_sms);
    return (unsigned)std::max(grid, 1);
}

void release_graphs(pr_graph *g)
{
    for (auto &c : g->graphs) {
        if (c.exec) cudaGraphExecDestroy(c.exec);
        if (c.graph) cudaGraphDestroy(c.graph);
    }
    g->graphs.clear();
}

// Instantiates (or reuses) a graph: WHILE(cond) { kernel<<<grid, block>>>(p) }.
pr_status loop_graph(pr_graph *g, int key, const void *func, unsigned grid, unsigned block,
                     SweepParams &p, cudaGraphExec_t *exec_out)
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
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    p.cond = h;
    p.use_cond = 1;
    void *args[] = {&p};
    cudaKernelNodeParams kp = {};
    kp.func = const_cast<void *>(func);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(block);
    kp.kernelParams = args;
    cudaGraphNode_t knode;
    e = cudaGraphAddKernelNode(&knode, body, nullptr, 0, &kp);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
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
    SweepParams p;
    fill_params(g, p, fp64, s);
    const bool gs = o->variant == PR_FUSED_GS;
    const bool serial = gs && tn.deterministic_gs;
    if (serial && g->n > 65536) {
        set_error("deterministic fused sweep is limited to n <= 65536");
        return PR_ERR_UNSUPPORTED;
    }
    p.renorm = gs ? 1 : 0;
    SolveState *hs = g->host_state;
    init_state(g, o, *hs);
    PR_CUDA(cudaMemcpyAsync(g->state.p, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int ib = std::min<int>((g->n + 255) / 256, g->num_sms * 8);
    k_init<T, A><<<std::max(ib, 1), 256, 0, s>>>(g->n, o->x0, p.outdeg,
                                                static_cast<const A *>(p.inv),
                                                static_cast<T *>(p.y0), p.st, p.renorm); note_launch();
    PR_LAUNCH_CHECK();

    const void *func;
    unsigned grid, block;
    bool graph_loop = false;
    if (serial) {
        func = reinterpret_cast<const void *>(&k_sweep_serial<T, A>);
        grid = 1;
        block = 32;
    } else {
        func = gs ? reinterpret_cast<const void *>(&k_sweep<T, A, true>)
                  : reinterpret_cast<const void *>(&k_sweep<T, A, false>);
        grid = sweep_grid(g, p, func);
        block = SWEEP_BS;
    }
    if (o->use_graph) {
        const int key = (fp64 ? 1 : 0) | (gs ? 2 : 0) | (serial ? 4 : 0);
        cudaGraphExec_t exec;
        PR_TRY(loop_graph(g, key, func, grid, block, p, &exec));
        PR_CUDA(cudaGraphLaunch(exec, s));
        graph_loop = true;
    } else {
        p.use_cond = 0;
        void *args[] = {&p};
        int launched = 0;
        while (launched < o->max_iter) {
            const int batch = std::min(16, o->max_iter - launched);
            for (int k = 0; k < batch; ++k) {
                PR_CUDA(cudaLaunchKernel(func, dim3(grid), dim3(block), args, 0, s));
                note_launch();
            }
            launched += batch;
            PR_CUDA(cudaMemcpyAsync(g->host_state, g->state.p, sizeof(SolveState),
                                    cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (g->host_state->done) break;
        }
    }
    k_output<T><<<std::max(ib, 1), 256, 0, s>>>(g->n, p.outdeg, static_cast<const T *>(p.y0),
                                               static_cast<const T *>(p.y1), gs ? 0 : 1, p.st,
                                               x_out); note_launch();
    PR_LAUNCH_CHECK();
    pr_status st = finish_result(g, res, s, 0);
    if (graph_loop) note_launch((uint64_t)g->host_state->iter + 1);  // loop sweeps + final check
    return st;
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
    o->max_outer = 8;
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
    PR_TRY(validate_options(o));
    PR_TRY(check_device(g));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pr_tune tn = effective_tune(g, o->tune);
    bool rebin = g->items.t_lo != tn.t_lo || g->items.t_hub != tn.t_hub ||
                 g->items.hub_seg != tn.hub_seg || g->items.low_rounds != tn.low_rounds ||
                 g->items.mid_per_warp != tn.mid_per_warp;
    if (rebin) release_graphs(g);
    PR_TRY(ensure_items(g, tn, s));
    PR_TRY(ensure_workspace(g, s));
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
    }
    return "unknown status";
}
