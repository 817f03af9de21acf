// multi.cu -- many independent graphs solved together: every sweep is one
// launch over the work items of all graphs that have not stopped yet.
//
// Each graph keeps its own degree-ordered in-lists, work items, stored
// vectors and solve state.  The items of graph k occupy [off[k], off[k+1]) of
// one global item range, taken by warps in the sweep's serpentine order, so
// small graphs share the machine with large ones instead of each leaving
// most SMs idle.  After an item the warp adds its partial sums to the item's
// graph and counts the item; the warp that counts a graph's last item closes
// that graph's sweep (stop test, next scalars).  The block that finishes the
// launch last keeps the device loop running while any graph is active.
// Jacobi (Algorithm 1: the result does not depend on which warp runs which
// item) or the fused sweep (Algorithm 2 / Eq. 9: each graph's stored vector
// is updated in place, as the single-graph fused sweep in one launch, and
// rescaled to sum 1 after each sweep).
#include <string.h>

#include <algorithm>
#include <vector>

#include "solve_impl.cuh"

namespace fpr {

struct MultiState {
    unsigned int ticket;
    int done;
};

struct MultiParams {
    int32_t G;
    const SweepParams *params;  // [G], device
    const int32_t *off;         // [G + 1] first item of each graph
    int32_t lcap;               // low-tile slots per warp (largest over the graphs)
    MultiState *ms;
    cudaGraphConditionalHandle cond;
    int32_t use_cond;
};

template <typename T, typename A, bool GS, bool W>
__device__ __forceinline__ void multi_item(const SweepParams &p, int j, int lane,
                                           unsigned char *slice, const Layout &L)
{
    SolveState *st = p.st;
    const int iter = st->iter;
    const T *yin;
    T *yout;
    if constexpr (GS) {
        yin = static_cast<const T *>(p.y0);
        yout = static_cast<T *>(p.y0);
    } else {
        yin = static_cast<const T *>((iter & 1) ? p.y1 : p.y0);
        yout = static_cast<T *>((iter & 1) ? p.y0 : p.y1);
    }
    SweepFin<T, A, GS, W> fin(p, load_ctx<A>(st), yout);
    const Src<T, GS> src{yin, nullptr, 0};
    const int nh = p.nhubseg, nm = p.mi[4];
    const int4 d = __ldg(p.desc + j);
    if (j < nh) hub_item<T, A, GS, W>(p, j, d, src, fin, lane);
    else if (j < nh + nm) mid_item<T, A, GS, W>(p, j - nh, d, src, fin, lane);
    else low_item<T, A, GS, W>(p, d, src, fin, lane, slice, L);
    // this item's sums, then the item count; the last item closes the sweep
    const double l1 = warp_sum(static_cast<double>(fin.pt.l1));
    const double lm = warp_max(static_cast<double>(fin.pt.lmax));
    const double dm = warp_sum(static_cast<double>(fin.pt.dm));
    const double sm = warp_sum(static_cast<double>(fin.pt.sm));
    int last = 0;
    if (lane == 0) {
        AccSlot &s = st->acc[j % ACC_SLOTS];
        if (l1 != 0) fx_add(&s.res_hi, &s.res_lo, l1);
        if (lm != 0) atomicMax(&s.res_max, static_cast<unsigned long long>(__double_as_longlong(lm)));
        if (dm != 0) fx_add(&s.dang_hi, &s.dang_lo, dm);
        if (sm != 0) fx_add(&s.sum_hi, &s.sum_lo, sm);
        __threadfence();
        const unsigned nitems = (unsigned)(nh + nm + p.nlt);
        last = atomicAdd(&st->ticket, 1u) == nitems - 1;
    }
    if (__shfl_sync(FULL, last, 0)) close_sweep(p);  // resets the ticket
    __syncwarp();
}

template <typename T, typename A, bool GS>
__global__ void __launch_bounds__(SWEEP_BS, SWEEP_MINB) k_multi_sweep(MultiParams mp)
{
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    __shared__ bool is_last;
    if (mp.ms->done) {
        if (mp.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(mp.cond, 0u);
        return;
    }
    const Layout L = make_layout(mp.lcap, sizeof(A), sizeof(T), false, 0);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned char *slice = dyn_smem + L.warps + warp * L.wbytes;
    const int gw = warp * gridDim.x + blockIdx.x;  // blocks interleaved, as in run_items
    const int nw = gridDim.x * SWEEP_WARPS;
    const int total = __ldg(mp.off + mp.G);
    for (int r = 0;; ++r) {
        const int i = r * nw + ((r & 1) ? nw - 1 - gw : gw);
        if (i >= total) break;
        int lo = 0, hi = mp.G - 1;  // graph owning item i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(mp.off + mid) <= i) lo = mid;
            else hi = mid - 1;
        }
        const SweepParams &p = mp.params[lo];
        if (*reinterpret_cast<volatile int *>(&p.st->done)) continue;
        const int j = i - __ldg(mp.off + lo);
        if (p.ew) multi_item<T, A, GS, true>(p, j, lane, slice, L);
        else multi_item<T, A, GS, false>(p, j, lane, slice, L);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&mp.ms->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    int active = 0;
    for (int k = threadIdx.x; k < mp.G; k += blockDim.x)
        active |= *reinterpret_cast<volatile int *>(&mp.params[k].st->done) == 0;
    const int n_active = __syncthreads_count(active);
    if (threadIdx.x == 0) {
        mp.ms->ticket = 0;
        mp.ms->done = n_active == 0 ? 1 : 0;
        __threadfence();
        if (mp.use_cond) cudaGraphSetConditional(mp.cond, n_active ? 1u : 0u);
    }
}

template <typename T, typename A>
static pr_status solve_multi(pr_graph *const *graphs, int32_t G, const pr_options *o,
                             double *const *x_out, pr_result *res, cudaStream_t s)
{
    constexpr bool fp64 = sizeof(A) == 8;
    const bool gs = o->variant == PR_FUSED_GS;
    pr_graph *g0 = graphs[0];
    std::vector<SweepParams> hp((size_t)G);
    std::vector<int32_t> off((size_t)G + 1, 0);
    int32_t lcap = 0;
    for (int k = 0; k < G; ++k) {
        pr_graph *g = graphs[k];
        SweepParams &p = hp[(size_t)k];
        fill_params(g, p, fp64, sizeof(T), false);
        p.stage = 0;
        p.close = 1;
        p.use_cond = 0;
        p.renorm = (gs && !o->no_rescale) ? 1 : 0;
        lcap = std::max(lcap, p.lcap);
        off[(size_t)k + 1] = off[(size_t)k] + p.nhubseg + p.mi[4] + p.nlt;
        SolveState *hs = g->host_state;
        init_state(g, o, *hs);
        PR_CUDA(cudaMemcpyAsync(g->state.p, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
        const int ib = std::max(1, std::min<int>((g->n + 255) / 256, g->num_sms * 8));
        k_init<T, A><<<ib, 256, 0, s>>>(g->n, nullptr, g->n2o.as<int32_t>(),
                                       p.outdeg, static_cast<const A *>(p.inv),
                                       static_cast<T *>(p.y0), p.st, p.renorm,
                                       g->weighted ? 1 : 0);
        note_launch();
    }
    PR_LAUNCH_CHECK();
    // device copies of the parameters, item offsets and loop state
    const size_t pbytes = sizeof(SweepParams) * (size_t)G;
    const size_t obytes = sizeof(int32_t) * ((size_t)G + 1);
    PR_TRY(buf_alloc(g0, g0->aux, pbytes + obytes + sizeof(MultiState) + 64, s));
    char *base = static_cast<char *>(g0->aux.p);
    SweepParams *dparams = reinterpret_cast<SweepParams *>(base);
    int32_t *doff = reinterpret_cast<int32_t *>(base + pbytes);
    MultiState *ms = reinterpret_cast<MultiState *>(base + ((pbytes + obytes + 15) & ~(size_t)15));
    PR_CUDA(cudaMemcpyAsync(dparams, hp.data(), pbytes, cudaMemcpyHostToDevice, s));
    PR_CUDA(cudaMemcpyAsync(doff, off.data(), obytes, cudaMemcpyHostToDevice, s));
    PR_CUDA(cudaMemsetAsync(ms, 0, sizeof(MultiState), s));

    MultiParams mp;
    memset(&mp, 0, sizeof(mp));
    mp.G = G;
    mp.params = dparams;
    mp.off = doff;
    mp.lcap = lcap;
    mp.ms = ms;
    const void *func = gs ? reinterpret_cast<const void *>(&k_multi_sweep<T, A, true>)
                          : reinterpret_cast<const void *>(&k_multi_sweep<T, A, false>);
    const size_t smem = make_layout(lcap, sizeof(A), sizeof(T), false, 0).total;
    const unsigned grid = sweep_grid(g0, off[(size_t)G], func, smem);
    if (grid == 0) return PR_ERR_INVALID_ARG;
    int sweeps = 0;
    if (o->use_graph) {
        cudaGraph_t graph = nullptr;
        PR_CUDA(cudaGraphCreate(&graph, 0));
        cudaGraphConditionalHandle h;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = h;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode, knode;
        if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
        if (e == cudaSuccess) {
            mp.cond = h;
            mp.use_cond = 1;
            void *args[] = {&mp};
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void *>(func);
            kp.gridDim = dim3(grid);
            kp.blockDim = dim3(SWEEP_BS);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&knode, cp.conditional.phGraph_out[0], nullptr, 0, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e, "multi-graph loop", __FILE__, __LINE__);
    } else {
        mp.use_cond = 0;
        void *args[] = {&mp};
        MultiState hms = {0, 0};
        while (sweeps < o->max_iter && !hms.done) {
            const int batch = std::min(16, o->max_iter - sweeps);
            for (int k = 0; k < batch; ++k) {
                PR_CUDA(cudaLaunchKernel(func, dim3(grid), dim3(SWEEP_BS), args, smem, s));
                note_launch();
            }
            sweeps += batch;
            PR_CUDA(cudaMemcpyAsync(&hms, ms, sizeof(hms), cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
        }
    }
    pr_status all = PR_OK;
    int max_iters = 0;
    for (int k = 0; k < G; ++k) {
        pr_graph *g = graphs[k];
        const SweepParams &p = hp[(size_t)k];
        const int ib = std::max(1, std::min<int>((g->n + 255) / 256, g->num_sms * 8));
        k_output<T><<<ib, 256, 0, s>>>(g->n, g->o2n.as<int32_t>(), p.outdeg,
                                       static_cast<const T *>(p.y0), static_cast<const T *>(p.y1),
                                       gs ? 0 : 1, p.st, x_out[k], g->weighted ? 1 : 0);
        note_launch();
        PR_LAUNCH_CHECK();
        pr_status st = finish_result(g, res ? &res[k] : nullptr, s, 0);
        max_iters = std::max(max_iters, g->host_state->iter);
        if (st != PR_OK && st != PR_NOT_CONVERGED) return st;
        if (st == PR_NOT_CONVERGED) all = st;
    }
    if (o->use_graph) note_launch((uint64_t)max_iters + 1);
    return all;
}

}  // namespace fpr

using namespace fpr;

extern "C" pr_status pr_solve_multi(pr_graph *const *graphs, int32_t G, const pr_options *o,
                                    double *const *x_out, pr_result *res, void *stream)
{
    if (res && G > 0) memset(res, 0, sizeof(pr_result) * (size_t)G);
    if (!graphs || G < 1 || !o || !x_out) {
        set_error("pr_solve_multi: need G >= 1 graphs, options and outputs");
        return PR_ERR_INVALID_ARG;
    }
    PR_TRY(validate_options(o));
    if ((o->precision != PR_FP64 && o->precision != PR_FP32) || o->x0 ||
        o->perforate_eps > 0.0) {
        set_error("pr_solve_multi: supports the Jacobi and fused sweeps in FP64 or FP32 from "
                  "x0 = 1/n");
        return PR_ERR_UNSUPPORTED;
    }
    for (int k = 0; k < G; ++k) {
        if (!graphs[k] || !x_out[k]) {
            set_error("pr_solve_multi: graph %d or its output is NULL", k);
            return PR_ERR_INVALID_ARG;
        }
        for (int j = 0; j < k; ++j)
            if (graphs[j] == graphs[k]) {
                set_error("pr_solve_multi: graph %d appears twice", k);
                return PR_ERR_INVALID_ARG;
            }
        if (graphs[k]->device != graphs[0]->device) {
            set_error("pr_solve_multi: all graphs must live on one device");
            return PR_ERR_INVALID_ARG;
        }
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    for (int k = 0; k < G; ++k) {
        pr_tune tn;
        PR_TRY(prepare_solve(graphs[k], o, tn, s));
    }
    return o->precision == PR_FP64 ? solve_multi<double, double>(graphs, G, o, x_out, res, s)
                                   : solve_multi<float, float>(graphs, G, o, x_out, res, s);
}
