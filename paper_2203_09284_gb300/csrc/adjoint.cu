// adjoint.cu -- reverse mode of the PageRank fixed point (pr_backward).
//
// At the fixed point x = (1-d)/n + d M x, with M = P^T + (1/n) 1 a^T (a the
// dangling indicator, P_uv = w_uv / s_u the row-normalised weights), a loss
// L(x) has the gradient lambda^T (dF/dtheta) where
//   (I - d M)^T lambda = dL/dx.
// lambda is iterated (Jacobi) as
//   lambda'_u = g_u + d (sum_{v in out(u)} P_uv lambda_v + a_u S / n),
//   S = sum_v lambda_v,
// a pull over the out-lists.  It runs on the graph with every edge reversed
// (whose in-lists are the out-lists), built once per graph, through the
// sweep's work items with the per-slot coefficient P_uv.  Then, for every
// edge e = u -> v (chain rule through the row normalisation),
//   dL/dw_e = (d x_u / s_u) (lambda_v - (P lambda)_u),
//   dL/dd   = lambda^T (M x - 1/n) = sum_u x_u (P lambda)_u + (D_x - 1) S / n,
// with D_x the dangling mass of x.
#include <string.h>

#include <algorithm>

#include "solve_impl.cuh"

namespace fpr {

// owner[q] = the vertex whose in-list holds slot q (warp per vertex)
__global__ void k_slot_owner(int32_t n, const int32_t *__restrict__ col_ptr, int32_t *owner)
{
    const int lane = threadIdx.x & 31;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n;
         u += (gridDim.x * blockDim.x) >> 5)
        for (int q = col_ptr[u] + lane; q < col_ptr[u + 1]; q += 32) owner[q] = u;
}

// Per slot of the reversed graph's degree-ordered in-lists (vertex u's
// out-edges): P_uv = w_e / s_u in FP64 and FP32, and s_u (warp per vertex;
// raw weights w in input edge order, or null for w = 1).
__global__ void k_adj_coef(int32_t n, const int32_t *__restrict__ rcol_ptr,
                           const int32_t *__restrict__ rcsc_eid,
                           const int32_t *__restrict__ fwd_csc_eid, const float *__restrict__ w,
                           double *p64, float *p32, double *srow)
{
    const int lane = threadIdx.x & 31;
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n;
         u += (gridDim.x * blockDim.x) >> 5) {
        const int a = rcol_ptr[u], e = rcol_ptr[u + 1];
        double s = 0.0;
        for (int q = a + lane; q < e; q += 32)
            s += w ? static_cast<double>(w[fwd_csc_eid[rcsc_eid[q]]]) : 1.0;
        s = warp_sum(s);
        for (int q = a + lane; q < e; q += 32) {
            const double pw = (w ? static_cast<double>(w[fwd_csc_eid[rcsc_eid[q]]]) : 1.0) / s;
            p64[q] = pw;
            p32[q] = static_cast<float>(pw);
        }
        if (lane == 0) srow[u] = s;
    }
}

// lambda^0 = g (the right-hand side too), in the reversed graph's ids; its sum.
template <typename T, typename A>
__global__ void k_adj_init(int32_t n, const int32_t *__restrict__ n2o, const double *grad_x,
                           T *y, A *rhs, SolveState *st)
{
    Part<A> pt;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const A gv = static_cast<A>(grad_x[n2o[u]]);
        y[u] = from_a<T>(gv);
        rhs[u] = gv;
        pt.sm += gv;
    }
    block_partials<A>(st, pt);
    if (last_block(st) && threadIdx.x < 32) {
        double res, resmax, dang, sum;
        take_sums(st, res, resmax, dang, sum);
        if (threadIdx.x == 0) st->sum = sum;
    }
}

// Epilogue of the adjoint sweep: lambda'_u from the gathered sum of P_uv
// lambda_v (u's out-edges); the dangling term S/n only for vertices without
// out-edges (no slots in the reversed in-list).
template <typename T, typename A>
struct AdjFin {
    const SweepParams &p;
    A d, sdn;
    T *yout;
    Part<A> pt;
    __device__ AdjFin(const SweepParams &p_, A d_, A sdn_, T *yo) : p(p_), d(d_), sdn(sdn_), yout(yo) {}
    __device__ __forceinline__ A rterm(const SweepParams &q, int u) const
    {
        return q.rhs ? static_cast<const A *>(q.rhs)[u] : A(0);
    }
    __device__ __forceinline__ T operator()(int u, A acc, int, A, T yold, A r)
    {
        const bool dangling = __ldg(p.col_ptr + u + 1) == __ldg(p.col_ptr + u);
        const A ln = r + d * (acc + (dangling ? sdn : A(0)));
        const T yn = from_a<T>(ln);
        st_y<T, false>(yout, u, yn);
        const A diff = aabs(ln - to_a<A>(yold));
        pt.l1 += diff;
        pt.lmax = diff > pt.lmax ? diff : pt.lmax;
        pt.sm += ln;
        return yn;
    }
};

template <typename T, typename A>
__global__ void __launch_bounds__(SWEEP_BS, SWEEP_MINB) k_adj_sweep(SweepParams p)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.close && p.use_cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    const int iter = st->iter;
    const T *yin = static_cast<const T *>((iter & 1) ? p.y1 : p.y0);
    T *yout = static_cast<T *>((iter & 1) ? p.y0 : p.y1);
    AdjFin<T, A> fin(p, static_cast<A>(st->d), static_cast<A>(st->sum * st->inv_n), yout);
    run_items<T, A, false, true>(p, yin, fin);
    block_partials<A>(st, fin.pt);
    if (p.close && last_block(st) && threadIdx.x < 32) close_sweep(p);
}

struct GradParams {
    int32_t n;
    const int32_t *col_ptr, *row_idx;  // reversed graph, degree-ordered ids
    const int32_t *rcsc_eid;           // reversed slot -> forward in-list slot
    const int32_t *fwd_csc_eid;        // forward in-list slot -> input edge id
    const int32_t *n2o;                // reversed ids -> input ids
    const double *p64, *srow;
    const double *x;                   // forward result, input ids
    double d;
    double *grad_w;                    // input edge order, or null
    double *grad_d;                    // or null
    SolveState *st;                    // sums: x.(P lambda), D_x, S
};

// Gradients from lambda (warp per vertex u of the reversed graph).
template <typename T>
__global__ void k_adj_grad(GradParams q, const T *__restrict__ lam)
{
    const int lane = threadIdx.x & 31;
    Part<double> pt;  // l1: sum x_u (P lambda)_u, dm: D_x, sm: S
    for (int u = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < q.n;
         u += (gridDim.x * blockDim.x) >> 5) {
        const int a = q.col_ptr[u], e = q.col_ptr[u + 1];
        double pl = 0.0;
        for (int k = a + lane; k < e; k += 32) pl += q.p64[k] * to_d(lam[q.row_idx[k]]);
        pl = warp_sum(pl);
        const double xu = q.x[q.n2o[u]];
        if (q.grad_w && e > a) {
            const double c = q.d * xu / q.srow[u];
            for (int k = a + lane; k < e; k += 32)
                q.grad_w[q.fwd_csc_eid[q.rcsc_eid[k]]] = c * (to_d(lam[q.row_idx[k]]) - pl);
        }
        if (lane == 0) {
            pt.l1 += xu * pl;
            if (e == a) pt.dm += xu;
            pt.sm += to_d(lam[u]);
        }
    }
    block_partials<double>(q.st, pt);
    if (last_block(q.st) && threadIdx.x < 32) {
        double xpl, unused, dx, S;
        take_sums(q.st, xpl, unused, dx, S);
        if (threadIdx.x == 0 && q.grad_d) *q.grad_d = xpl + (dx - 1.0) * S / static_cast<double>(q.n);
    }
}

// The reversed graph and the coefficients of its slots (built once).
static pr_status ensure_reverse(pr_graph *g, cudaStream_t s)
{
    if (g->rev) return PR_OK;
    const int32_t n = g->n;
    const int64_t m = g->m;
    Buf owner;
    PR_TRY(buf_alloc(g, owner, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), s));
    pr_status st = PR_OK;
    if (m > 0) {
        k_slot_owner<<<g->num_sms * 8, 256, 0, s>>>(n, g->col_ptr.as<int32_t>(), owner.as<int32_t>());
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "slot owners", __FILE__, __LINE__);
    }
    // reversed edge q: owner[q] -> row_idx[q] (forward edge row_idx[q] -> owner[q])
    pr_graph *rev = nullptr;
    if (st == PR_OK)
        st = pr_graph_create(n, m, owner.as<int32_t>(), g->row_idx.as<int32_t>(), nullptr, 0,
                             g->mem.has_hooks ? &g->mem.hooks : nullptr, s, &rev);
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &owner), g->owned.end());
    buf_free(g, owner, s);
    if (st != PR_OK) return st;
    g->rev = rev;
    const size_t mm = (size_t)std::max<int64_t>(m, 1) + 16;
    PR_TRY(buf_alloc(g, g->adj_p64, sizeof(double) * mm, s));
    PR_TRY(buf_alloc(g, g->adj_p32, sizeof(float) * mm, s));
    PR_TRY(buf_alloc(g, g->adj_s, sizeof(double) * (size_t)n, s));  // s_u per reversed id
    PR_CUDA(cudaMemsetAsync(g->adj_p64.p, 0, sizeof(double) * mm, s));
    PR_CUDA(cudaMemsetAsync(g->adj_p32.p, 0, sizeof(float) * mm, s));
    k_adj_coef<<<g->num_sms * 8, 256, 0, s>>>(n, rev->r_col_ptr.as<int32_t>(),
                                             rev->r_csc_eid.as<int32_t>(),
                                             g->csc_eid.as<int32_t>(),
                                             g->weighted ? g->w.as<float>() : nullptr,
                                             g->adj_p64.as<double>(), g->adj_p32.as<float>(),
                                             g->adj_s.as<double>());
    note_launch();
    PR_LAUNCH_CHECK();
    PR_CUDA(cudaStreamSynchronize(s));
    return PR_OK;
}

template <typename T, typename A>
static pr_status backward(pr_graph *g, const pr_options *o, const double *x,
                          const double *grad_x, double *grad_w, double *grad_d, pr_result *res,
                          cudaStream_t s)
{
    constexpr bool fp64 = sizeof(A) == 8;
    PR_TRY(ensure_reverse(g, s));
    pr_graph *rev = g->rev;
    pr_tune tn;
    PR_TRY(prepare_solve(rev, o, tn, s));
    const int32_t n = g->n;
    PR_TRY(buf_alloc(rev, rev->rbuf, sizeof(A) * (size_t)n + 64, s));
    SweepParams p;
    fill_params(rev, p, fp64, sizeof(T), false);
    p.ew = fp64 ? static_cast<const void *>(g->adj_p64.p) : static_cast<const void *>(g->adj_p32.p);
    p.rhs = rev->rbuf.p;
    p.renorm = 0;
    SweepPlan plan;
    PR_TRY((make_plan<T, A>(rev, p, false, plan)));
    plan.func = reinterpret_cast<const void *>(&k_adj_sweep<T, A>);
    PR_CUDA(cudaFuncSetAttribute(plan.func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)plan.smem));

    SolveState *hs = rev->host_state;
    init_state(rev, o, *hs);
    PR_CUDA(cudaMemcpyAsync(rev->state.p, hs, sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int ib = std::max(1, std::min<int>((n + 255) / 256, g->num_sms * 8));
    k_adj_init<T, A><<<ib, 256, 0, s>>>(n, rev->n2o.as<int32_t>(), grad_x, static_cast<T *>(p.y0),
                                       static_cast<A *>(rev->rbuf.p), p.st);
    note_launch();
    PR_LAUNCH_CHECK();
    if (o->use_graph) {
        cudaGraphExec_t exec;
        PR_TRY(loop_graph(rev, 64 | (fp64 ? 1 : 0) | (rev->items.test_stall ? 32 : 0), plan,
                          &exec));
        PR_CUDA(cudaGraphLaunch(exec, s));
    } else {
        int launched = 0;
        while (launched < o->max_iter) {
            const int batch = std::min(16, o->max_iter - launched);
            for (int k = 0; k < batch; ++k) PR_TRY(launch_plan(plan, s));
            launched += batch;
            PR_CUDA(cudaMemcpyAsync(hs, rev->state.p, sizeof(SolveState), cudaMemcpyDeviceToHost,
                                    s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (hs->done) break;
        }
    }
    pr_status st = finish_result(rev, res, s, 0);
    if (o->use_graph) note_launch((uint64_t)hs->iter + 1);
    if (st != PR_OK && st != PR_NOT_CONVERGED) return st;

    GradParams q;
    memset(&q, 0, sizeof(q));
    q.n = n;
    q.col_ptr = rev->r_col_ptr.as<int32_t>();
    q.row_idx = rev->r_row_idx.as<int32_t>();
    q.rcsc_eid = rev->r_csc_eid.as<int32_t>();
    q.fwd_csc_eid = g->csc_eid.as<int32_t>();
    q.n2o = rev->n2o.as<int32_t>();
    q.p64 = g->adj_p64.as<double>();
    q.srow = g->adj_s.as<double>();
    q.x = x;
    q.d = o->d;
    q.grad_w = grad_w;
    q.grad_d = grad_d;
    // repeated edges dropped by PR_DEDUP take no part: their gradient is 0
    if (grad_w && g->m_in != g->m)
        PR_CUDA(cudaMemsetAsync(grad_w, 0, sizeof(double) * (size_t)g->m_in, s));
    q.st = rev->state.as<SolveState>();
    const T *lam = static_cast<const T *>((hs->iter & 1) ? p.y1 : p.y0);
    k_adj_grad<T><<<g->num_sms * 4, 256, 0, s>>>(q, lam);
    note_launch();
    PR_LAUNCH_CHECK();
    PR_CUDA(cudaStreamSynchronize(s));
    return st;
}

}  // namespace fpr

using namespace fpr;

extern "C" pr_status pr_backward(pr_graph *g, const pr_options *o, const double *x,
                                 const double *grad_x, double *grad_w, double *grad_d,
                                 pr_result *res, void *stream)
{
    if (res) memset(res, 0, sizeof(*res));
    if (!g || !o || !x || !grad_x) {
        set_error("pr_backward: graph, options, x and grad_x are required");
        return PR_ERR_INVALID_ARG;
    }
    PR_TRY(validate_options(o));
    PR_TRY(check_device(g));
    if (o->precision != PR_FP64 && o->precision != PR_FP32) {
        set_error("pr_backward: the adjoint iterates in FP64 or FP32");
        return PR_ERR_UNSUPPORTED;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return o->precision == PR_FP64
               ? backward<double, double>(g, o, x, grad_x, grad_w, grad_d, res, s)
               : backward<float, float>(g, o, x, grad_x, grad_w, grad_d, res, s);
}
