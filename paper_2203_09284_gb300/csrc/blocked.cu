// blocked.cu -- propagation-blocked Jacobi sweep (binning by destination
// range), the locality technique the paper's related work cites (Beamer et
// al.) for gathers whose vector does not fit in cache.
//
// The in-list slots are regrouped once into bins of 2^PB_BITS consecutive
// destinations (degree-ordered ids), ordered by source inside each bin.  A
// sweep is three launches:
//   scatter     in source order, each out-edge copies its source's stored
//               contribution y_v into the edge's slot of its destination's
//               bin (the sources and the contribution vector are read in
//               order; the writes land in each bin's slot range in order)
//   accumulate  a block per chunk of at most PB_CHUNK slots of one bin adds
//               the chunk's values into a shared-memory copy of the bin's
//               2^PB_BITS sums (shared atomics), then adds the nonzero sums
//               into the global sums (global atomics)
//   epilogue    per vertex: the Jacobi update of Algorithm 1 / Eq. 2 from the
//               global sum (the sweep's epilogue functor), which clears it for
//               the next sweep; block partials and the stop test as the
//               persistent sweep.
// The atomic additions make the order of a vertex's sum vary from run to
// run (results agree to rounding); Jacobi only, unweighted, FP64 or FP32.
#include <string.h>

#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "solve_impl.cuh"

namespace fpr {

constexpr int PB_BITS = 14;        // destinations per bin: 16384
constexpr int PB_BIN = 1 << PB_BITS;
constexpr int PB_CHUNK = 1 << 16;  // bin slots per accumulation block
constexpr int PB_BS = 1024;

// Device arrays of the blocked layout (built on the first blocked solve).
struct PbLayout {
    int64_t m = 0;
    int32_t nbins = 0, nunits = 0;
    Buf csrc;   // [m] source of each out-edge, sources ascending (scatter order)
    Buf pos;    // [m] bin slot of that out-edge
    Buf dl;     // [m] destination of each bin slot, minus its bin's first id
    Buf units;  // [nunits] int4 {bin, first slot, end slot, 0}
    Buf val;    // [m] stored contributions in bin order (8 bytes each)
    Buf gacc;   // [nbins * PB_BIN] sums (8 bytes each), zero between sweeps
};

// key = (bin of the destination) << 32 | source, value = destination within
// the bin, for every relabelled in-list slot (a warp per vertex)
__global__ void k_pb_keys(int32_t n, const int32_t *__restrict__ r_col_ptr,
                          const int32_t *__restrict__ r_row_idx, uint64_t *keys, int32_t *vals)
{
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int a = r_col_ptr[u], e = r_col_ptr[u + 1];
        const uint64_t hi = static_cast<uint64_t>(u >> PB_BITS) << 32;
        for (int s = a + lane; s < e; s += 32) {
            keys[s] = hi | static_cast<uint32_t>(r_row_idx[s]);
            vals[s] = u & (PB_BIN - 1);
        }
    }
}

// after the sort by (bin, source): the sources as the keys of a second sort
// (by source), carrying each slot's bin position
__global__ void k_pb_second(int64_t m, const uint64_t *__restrict__ k1, uint64_t *k2,
                            int32_t *v2)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        k2[j] = static_cast<uint32_t>(k1[j]);
        v2[j] = static_cast<int32_t>(j);
    }
}

__global__ void k_pb_low32(int64_t m, const uint64_t *__restrict__ k, int32_t *out)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride)
        out[j] = static_cast<int32_t>(static_cast<uint32_t>(k[j]));
}

// ---------------------------------------------------------------- sweep
template <typename T>
__global__ void k_pb_scatter(const SolveState *st, int64_t m, const int32_t *__restrict__ csrc,
                             const int32_t *__restrict__ pos, const T *y0, const T *y1, T *val)
{
    if (st->done) return;
    const T *yin = (st->iter & 1) ? y1 : y0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += stride)
        val[pos[q]] = yin[csrc[q]];
}

template <typename T, typename A>
__global__ void __launch_bounds__(PB_BS) k_pb_accumulate(const SolveState *st, int32_t nunits,
                                                         const int4 *__restrict__ units,
                                                         const T *__restrict__ val,
                                                         const int32_t *__restrict__ dl, A *gacc)
{
    extern __shared__ __align__(16) unsigned char pb_smem[];
    A *acc = reinterpret_cast<A *>(pb_smem);
    if (st->done) return;
    for (int k = blockIdx.x; k < nunits; k += gridDim.x) {
        const int4 d = units[k];
        for (int i = threadIdx.x; i < PB_BIN; i += blockDim.x) acc[i] = A(0);
        __syncthreads();
        for (int j = d.y + threadIdx.x; j < d.z; j += blockDim.x)
            atomicAdd(&acc[dl[j]], static_cast<A>(val[j]));
        __syncthreads();
        A *g = gacc + (size_t)d.x * PB_BIN;
        for (int i = threadIdx.x; i < PB_BIN; i += blockDim.x)
            if (acc[i] != A(0)) atomicAdd(&g[i], acc[i]);
        __syncthreads();
    }
}

template <typename T, typename A>
__global__ void __launch_bounds__(PB_BS) k_pb_epilogue(SweepParams p, A *gacc)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    const int iter = st->iter;
    T *yout = static_cast<T *>((iter & 1) ? p.y0 : p.y1);
    const T *yin = static_cast<const T *>((iter & 1) ? p.y1 : p.y0);
    SweepFin<T, A, false, false> fin(p, load_ctx<A>(st), yout);
    const A *inv = static_cast<const A *>(p.inv);
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < p.n; u += gridDim.x * blockDim.x) {
        const A acc = gacc[u];
        gacc[u] = A(0);
        fin(u, acc, p.outdeg[u], inv[u], yin[u], fin.rterm(p, u));
    }
    block_partials<A>(st, fin.pt);
    if (last_block(st) && threadIdx.x < 32) close_sweep(p);
}

// ---------------------------------------------------------------- build
// Each graph's layout, built on its first blocked solve (its buffers are
// owned by the graph and freed with it; the record goes at destroy).
static std::mutex pb_mu;
static std::unordered_map<const pr_graph *, PbLayout *> pb_layouts;

static PbLayout &layout_of_graph(pr_graph *g)
{
    std::lock_guard<std::mutex> lk(pb_mu);
    PbLayout *&L = pb_layouts[g];
    if (!L) L = new PbLayout();
    return *L;
}

// device scratch of the layout build, freed on every return path
struct TempDev {
    pr_graph *g;
    cudaStream_t s;
    size_t bytes;
    void *p;
    TempDev(pr_graph *g_, size_t b, cudaStream_t s_) : g(g_), s(s_), bytes(b ? b : 16)
    {
        p = g->mem.alloc(bytes, s);
    }
    ~TempDev()
    {
        if (p) g->mem.free(p, bytes, s);
    }
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

static pr_status ensure_blocked(pr_graph *g, cudaStream_t s)
{
    PbLayout &L = layout_of_graph(g);
    if (L.val.p && L.m == g->m) return PR_OK;
    const int32_t n = g->n;
    const int64_t m = g->m;
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    L.m = -1;  // set once the layout is complete
    L.nbins = (n + PB_BIN - 1) / PB_BIN;
    PR_TRY(buf_alloc(g, L.csrc, sizeof(int32_t) * mm, s));
    PR_TRY(buf_alloc(g, L.pos, sizeof(int32_t) * mm, s));
    PR_TRY(buf_alloc(g, L.dl, sizeof(int32_t) * mm, s));
    PR_TRY(buf_alloc(g, L.val, sizeof(double) * mm, s));
    PR_TRY(buf_alloc(g, L.gacc, sizeof(double) * (size_t)L.nbins * PB_BIN, s));
    PR_CUDA(cudaMemsetAsync(L.gacc.p, 0, sizeof(double) * (size_t)L.nbins * PB_BIN, s));
    std::vector<int4> units;
    if (m > 0) {
        TempDev tka(g, sizeof(uint64_t) * mm, s), tkb(g, sizeof(uint64_t) * mm, s);
        TempDev tvb(g, sizeof(int32_t) * mm, s), tbins(g, sizeof(int32_t) * (L.nbins + 1), s);
        uint64_t *ka = tka.as<uint64_t>(), *kb = tkb.as<uint64_t>();
        int32_t *vb = tvb.as<int32_t>(), *bins = tbins.as<int32_t>();
        pr_status st = (ka && kb && vb && bins) ? PR_OK : PR_ERR_OOM;
        if (st != PR_OK) set_error("device allocation for the blocked layout failed");
        uint64_t *kr = nullptr;
        int32_t *vr = nullptr;
        if (st == PR_OK) {
            const unsigned wb = (unsigned)std::min<int64_t>(((int64_t)n * 32 + 255) / 256,
                                                            (int64_t)g->num_sms * 16);
            k_pb_keys<<<wb, 256, 0, s>>>(n, g->r_col_ptr.as<int32_t>(), g->r_row_idx.as<int32_t>(),
                                         ka, L.dl.as<int32_t>());
            note_launch();
            // by (bin, source): stable, so equal keys keep the in-list order
            std::vector<int> shifts = digit_shifts(n, 0);
            for (int sh : digit_shifts(L.nbins, 32)) shifts.push_back(sh);
            st = radix_sort(g, ka, L.dl.as<int32_t>(), kb, vb, m, shifts, s, &kr, &vr);
        }
        if (st == PR_OK) {
            if (vr != L.dl.as<int32_t>())
                PR_CUDA(cudaMemcpyAsync(L.dl.p, vr, sizeof(int32_t) * (size_t)m,
                                        cudaMemcpyDeviceToDevice, s));
            // bin sizes: runs of equal high words
            PR_CUDA(cudaMemsetAsync(bins, 0, sizeof(int32_t) * (L.nbins + 1), s));
            const unsigned rb = (unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 32);
            k_run_degrees<<<rb, 256, 0, s>>>(m, kr, 1, bins, nullptr);
            note_launch();
            // second sort: by source, carrying each slot's bin position
            uint64_t *k2 = kr == ka ? kb : ka;
            k_pb_second<<<rb, 256, 0, s>>>(m, kr, k2, L.pos.as<int32_t>());
            note_launch();
            uint64_t *k2r = nullptr;
            int32_t *v2r = nullptr;
            st = radix_sort(g, k2, L.pos.as<int32_t>(), kr, vb, m, digit_shifts(n, 0), s, &k2r,
                            &v2r);
            if (st == PR_OK) {
                k_pb_low32<<<rb, 256, 0, s>>>(m, k2r, L.csrc.as<int32_t>());
                note_launch();
                if (v2r != L.pos.as<int32_t>())
                    PR_CUDA(cudaMemcpyAsync(L.pos.p, v2r, sizeof(int32_t) * (size_t)m,
                                            cudaMemcpyDeviceToDevice, s));
            }
        }
        std::vector<int32_t> hb((size_t)L.nbins + 1, 0);
        if (st == PR_OK) {
            PR_CUDA(cudaMemcpyAsync(hb.data(), bins, sizeof(int32_t) * L.nbins,
                                    cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
        }
        PR_TRY(st);
        int64_t start = 0;
        for (int b = 0; b < L.nbins; ++b) {
            const int64_t end = start + hb[(size_t)b];
            for (int64_t a = start; a < end; a += PB_CHUNK)
                units.push_back(make_int4(b, (int)a, (int)std::min<int64_t>(end, a + PB_CHUNK), 0));
            start = end;
        }
    }
    L.nunits = (int32_t)units.size();
    PR_TRY(buf_alloc(g, L.units, sizeof(int4) * std::max<size_t>(units.size(), 1), s));
    if (!units.empty())
        PR_CUDA(cudaMemcpyAsync(L.units.p, units.data(), sizeof(int4) * units.size(),
                                cudaMemcpyHostToDevice, s));
    PR_CUDA(cudaStreamSynchronize(s));
    PR_LAUNCH_CHECK();
    L.m = m;
    return PR_OK;
}

void release_blocked(pr_graph *g)
{
    std::lock_guard<std::mutex> lk(pb_mu);
    auto it = pb_layouts.find(g);
    if (it == pb_layouts.end()) return;
    delete it->second;
    pb_layouts.erase(it);
}

// ---------------------------------------------------------------- solve
template <typename T, typename A>
static pr_status solve_blocked_t(pr_graph *g, const pr_options *o, double *x_out, pr_result *res,
                                 cudaStream_t s)
{
    constexpr bool fp64 = sizeof(A) == 8;
    PR_TRY(ensure_blocked(g, s));
    PbLayout &L = layout_of_graph(g);
    SweepParams p;
    fill_params(g, p, fp64, sizeof(T), false);
    p.renorm = 0;
    SolveState *hs = g->host_state;
    init_state(g, o, *hs);
    PR_CUDA(cudaMemcpyAsync(g->state.p, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int32_t n = g->n;
    const int ib = std::max(1, std::min<int>((n + 255) / 256, g->num_sms * 8));
    k_init<T, A><<<ib, 256, 0, s>>>(n, o->x0, g->n2o.as<int32_t>(), p.outdeg,
                                   static_cast<const A *>(p.inv), static_cast<T *>(p.y0), p.st, 0,
                                   0);
    note_launch();
    PR_LAUNCH_CHECK();

    const void *f_sc = reinterpret_cast<const void *>(&k_pb_scatter<T>);
    const void *f_ac = reinterpret_cast<const void *>(&k_pb_accumulate<T, A>);
    const void *f_ep = reinterpret_cast<const void *>(&k_pb_epilogue<T, A>);
    const size_t smem_ac = sizeof(A) * PB_BIN;
    PR_CUDA(cudaFuncSetAttribute(f_ac, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_ac));
    const unsigned g_sc = (unsigned)std::max<int64_t>(1, std::min<int64_t>((L.m + 255) / 256,
                                                                         (int64_t)g->num_sms * 16));
    const unsigned g_ac = (unsigned)std::max(1, std::min(L.nunits, g->num_sms * 2));
    // one block per SM: the per-block partial sums and the closing ticket
    // are a few hundred atomics, not thousands
    const unsigned g_ep = (unsigned)std::max(1, std::min((n + PB_BS - 1) / PB_BS, g->num_sms));
    const SolveState *cst = p.st;
    int64_t mloc = L.m;
    const int32_t *csrc = L.csrc.as<int32_t>(), *pos = L.pos.as<int32_t>();
    const int32_t *dl = L.dl.as<int32_t>();
    const int4 *units = L.units.as<int4>();
    const void *y0 = p.y0, *y1 = p.y1;
    void *val = L.val.p;
    void *gacc = L.gacc.p;
    int32_t nunits = L.nunits;
    void *a_sc[] = {&cst, &mloc, &csrc, &pos, &y0, &y1, &val};
    void *a_ac[] = {&cst, &nunits, &units, &val, &dl, &gacc};
    bool graph_loop = false;
    if (o->use_graph) {
        const int key = 512 | (fp64 ? 1 : 0);
        cudaGraphExec_t exec = nullptr;
        for (auto &c : g->graphs)
            if (c.key == key) exec = c.exec;
        if (!exec) {
            cudaGraph_t graph = nullptr;
            PR_CUDA(cudaGraphCreate(&graph, 0));
            cudaGraphConditionalHandle h;
            cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1,
                                                             cudaGraphCondAssignDefault);
            cudaGraphNodeParams cp = {};
            cp.type = cudaGraphNodeTypeConditional;
            cp.conditional.handle = h;
            cp.conditional.type = cudaGraphCondTypeWhile;
            cp.conditional.size = 1;
            cudaGraphNode_t cnode, n1, n2, n3;
            if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, graph, nullptr, nullptr, 0, &cp);
            SweepParams pe = p;
            pe.cond = h;
            pe.use_cond = 1;
            void *a_ep[] = {&pe, &gacc};
            cudaKernelNodeParams k1 = {}, k2 = {}, k3 = {};
            k1.func = const_cast<void *>(f_sc);
            k1.gridDim = dim3(g_sc);
            k1.blockDim = dim3(256);
            k1.kernelParams = a_sc;
            k2.func = const_cast<void *>(f_ac);
            k2.gridDim = dim3(g_ac);
            k2.blockDim = dim3(PB_BS);
            k2.sharedMemBytes = (unsigned)smem_ac;
            k2.kernelParams = a_ac;
            k3.func = const_cast<void *>(f_ep);
            k3.gridDim = dim3(g_ep);
            k3.blockDim = dim3(PB_BS);
            k3.kernelParams = a_ep;
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n1, body, nullptr, 0, &k1);
            if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n2, body, &n1, 1, &k2);
            if (e == cudaSuccess) e = cudaGraphAddKernelNode(&n3, body, &n2, 1, &k3);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                return cuda_status(e, "blocked loop graph", __FILE__, __LINE__);
            }
            pr_graph::Cached c;
            c.key = key;
            c.exec = exec;
            c.graph = graph;
            g->graphs.push_back(c);
        }
        PR_CUDA(cudaGraphLaunch(exec, s));
        graph_loop = true;
    } else {
        SweepParams pe = p;
        pe.use_cond = 0;
        void *a_ep[] = {&pe, &gacc};
        int launched = 0;
        while (launched < o->max_iter) {
            const int batch = std::min(16, o->max_iter - launched);
            for (int k = 0; k < batch; ++k) {
                PR_CUDA(cudaLaunchKernel(f_sc, dim3(g_sc), dim3(256), a_sc, 0, s));
                PR_CUDA(cudaLaunchKernel(f_ac, dim3(g_ac), dim3(PB_BS), a_ac, smem_ac, s));
                PR_CUDA(cudaLaunchKernel(f_ep, dim3(g_ep), dim3(PB_BS), a_ep, 0, s));
                note_launch(3);
            }
            launched += batch;
            PR_CUDA(cudaMemcpyAsync(g->host_state, g->state.p, sizeof(SolveState),
                                    cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (g->host_state->done) break;
        }
    }
    k_output<T><<<ib, 256, 0, s>>>(n, g->o2n.as<int32_t>(), p.outdeg, static_cast<const T *>(p.y0),
                                   static_cast<const T *>(p.y1), 1, p.st, x_out, 0);
    note_launch();
    PR_LAUNCH_CHECK();
    pr_status st = finish_result(g, res, s, 0);
    if (res) res->gathered = (int64_t)res->iters * g->m;
    if (graph_loop) note_launch((uint64_t)3 * (g->host_state->iter + 1));
    return st;
}

pr_status solve_blocked(pr_graph *g, const pr_options *o, double *x_out, pr_result *res,
                        cudaStream_t s)
{
    if (o->variant != PR_JACOBI || g->weighted || o->perforate_eps > 0.0 ||
        (o->precision != PR_FP64 && o->precision != PR_FP32)) {
        set_error("the blocked sweep needs Jacobi, FP64 or FP32, an unweighted graph and no "
                  "perforation");
        return PR_ERR_UNSUPPORTED;
    }
    return o->precision == PR_FP64 ? solve_blocked_t<double, double>(g, o, x_out, res, s)
                                   : solve_blocked_t<float, float>(g, o, x_out, res, s);
}

}  // namespace fpr
