// dc.cu -- mixed precision with FP64 defect correction.
//
// The FP64 iterate x (stored in the contribution form Y64 with scale sigma_x)
// is improved by corrections e that solve (I - d M) e = r, r = F(x) - x:
//   outer step:  r = (1-d)/n + d M x - x    FP64 gather and arithmetic (the
//                                           only FP64 sweep); stop if
//                                           ||r||_1 <= threshold
//   inner loop:  e <- r + d M e              the cheap sweep, e stored as
//                                           FP32 / BF16 / FP16 times 2^k,
//                                           FP32 accumulation; Jacobi or fused
//   update:      x <- (x + e) / sum(x + e)   FP64
// The three steps are nested WHILE loops of one CUDA graph: the residual
// kernel decides whether another inner solve is needed, the last inner sweep
// ends the inner loop, the update kernel ends the outer loop once the
// residual kernel has declared convergence.
#include <string.h>

#include <algorithm>
#include <cmath>

#include "solve_impl.cuh"
#include "sweep.cuh"

namespace fpr {

struct DCParams {
    SweepParams p;           // traversal of the FP64 residual sweep (y0 = Y64)
    float *r32;              // right-hand side of the correction solve
    void *e0, *e1;           // correction buffers (stored form)
    const float *inv32;      // degree-ordered 1/outdeg
    const double *inv64;
    double *y64;
    SolveState *sx, *se;     // outer and inner states
    cudaGraphConditionalHandle h_inner, h_outer;
    int use_cond;
    int gs;                  // inner sweeps are fused (in place)
    int fp16;                // scale the correction into the FP16 range
    int weighted;
};

// Epilogue of the residual sweep: r_u in FP64, stored as FP32; unless the
// correction needs a scale (FP16), also the first correction iterate e = r
// in the correction's stored form.  A non-finite r_u ends the solve with
// PR_ERR_NUMERIC.
template <typename Te>
struct ResidFin {
    const DCParams &q;
    Ctx<double> c;
    Part<double> pt;
    __device__ ResidFin(const DCParams &q_, const Ctx<double> &c_) : q(q_), c(c_) {}
    __device__ __forceinline__ double rterm(const SweepParams &, int) const { return 0.0; }
    __device__ __forceinline__ double operator()(int u, double acc, int od, double, double yo,
                                                 double)
    {
        const bool plain = q.weighted || od == 0;  // stored value is x itself
        const double xold = plain ? yo : yo * static_cast<double>(od);
        const double xnew = fma(c.ds, acc, c.bc);
        const double r = xnew - c.sig * xold;
        if (!isfinite(r)) atomicCAS(&q.sx->error, 0, (int)PR_ERR_NUMERIC);
        const float rf = static_cast<float>(r);
        q.r32[u] = rf;
        if (!q.fp16) static_cast<Te *>(q.e0)[u] = from_a<Te>(plain ? rf : rf * q.inv32[u]);
        const double ar = fabs(r);
        pt.l1 += ar;
        if (c.linf) pt.lmax = ar > pt.lmax ? ar : pt.lmax;
        pt.sm += rf;
        if (od == 0) pt.dm += rf;
        return xnew;
    }
};

// Fused correction sweeps drift in the sum of e (the dangling mass is taken
// at sweep start while values change in place), which slows them far below
// the Jacobi rate.  The solution's sum is known, so after each sweep
//   e <- e + beta x,   beta = (sum(r)/(1-d) - sum(e)) / sum(x)
// restores it along the current PageRank estimate: in stored units
// e~ += shift * Y64.  The last block clears the pending shift.
template <typename Te>
__global__ void k_dc_shift(DCParams q)
{
    SolveState *se = q.se;
    const double gam = se->shift;
    Te *e = static_cast<Te *>(q.e0);
    const int n = q.p.n;
    if (gam != 0.0) {
        const float g32 = static_cast<float>(gam);
        for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x)
            e[u] = from_a<Te>(to_a<float>(e[u]) + g32 * static_cast<float>(q.y64[u]));
    }
    __shared__ bool is_last;
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&se->shift_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (is_last && threadIdx.x == 0) {
        se->shift = 0.0;
        se->shift_ticket = 0;
    }
}

// FP16 correction scale sigma_e = 2^-k: the stored entries are bounded by
// ||e||_1 / sigma_e <= ||r||_1 / ((1-d) sigma_e) (M does not increase the
// 1-norm, so neither the iterates nor the solution of e = r + d M e exceed
// it), which k keeps below 2^14, far from FP16's largest value 65504.
__device__ __forceinline__ double fp16_scale(double rnorm, double d)
{
    if (!(rnorm > 0.0)) return 1.0;
    int k = (int)floor(log2(16384.0 * (1.0 - d) / rnorm));
    k = max(-120, min(120, k));
    return ldexp(1.0, -k);
}

template <typename Te, bool W>
__global__ void __launch_bounds__(SWEEP_BS, SWEEP_MINB) k_dc_resid(DCParams q)
{
    SolveState *sx = q.sx, *se = q.se;
    if (sx->done) {
        if (q.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(q.h_inner, 0u);
        return;
    }
    ResidFin<Te> fin(q, load_ctx<double>(sx));
    run_items<double, double, false, W>(q.p, q.y64, fin);
    block_partials<double>(sx, fin.pt);
    if (!(last_block(sx) && threadIdx.x < 32)) return;
    double res, resmax, dang_r, sum_r;
    take_sums(sx, res, resmax, dang_r, sum_r);
    if (threadIdx.x != 0) return;
    sx->outer_iter += 1;
    const int total = sx->iter + 1;
    sx->iter = total;
    sx->rnorm = res;
    sx->res = res;
    sx->resmax = resmax;
    const double err = sx->norm ? resmax : res;
    if (sx->history) sx->history[total - 1] = err;
    const bool conv = err <= sx->tau;
    const int error = *reinterpret_cast<volatile int *>(&sx->error);
    const bool go_on =
        !(conv || error || sx->outer_iter >= sx->max_outer || total >= sx->max_iter);
    if (!go_on) {
        sx->done = 1;
        sx->status = error ? error : (conv ? PR_OK : PR_NOT_CONVERGED);
        se->done = 1;
    } else {
        const double scale = q.fp16 ? fp16_scale(res, sx->d) : 1.0;
        sx->scale = scale;
        se->iter = 0;
        se->done = 0;
        se->best = INFINITY;
        se->since = 0;
        se->dang = dang_r / scale;
        se->sum = sum_r / scale;
        se->sigma = scale;
        // 1^T (I - d M) = (1-d) 1^T: the correction sums to sum(r) / (1-d)
        se->mass_target = sum_r / (1.0 - sx->d);
        se->shift = 0.0;
        // inner stop on the L1 change of e (true units); the last outer step
        // need not over-solve below the outer threshold
        se->tau = fmax(sx->inner_rel * res, sx->inner_floor * sx->tau);
        se->norm = 0;
    }
    __threadfence();
    if (q.use_cond) cudaGraphSetConditional(q.h_inner, go_on ? 1u : 0u);
}

// x <- x + e, renormalised through sigma_x; ends the outer loop when done.
template <typename Te>
__global__ void k_dc_update(DCParams q)
{
    SolveState *sx = q.sx, *se = q.se;
    if (sx->done) {
        if (q.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(q.h_outer, 0u);
        return;
    }
    const Te *eb = static_cast<const Te *>((!q.gs && (se->iter & 1)) ? q.e1 : q.e0);
    const double sgx = sx->sigma, sge = se->sigma;
    Part<double> pt;
    const int n = q.p.n;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int od = q.p.outdeg[u];
        const bool plain = q.weighted || od == 0;
        const double yx = q.y64[u];
        const double xs = plain ? yx : yx * static_cast<double>(od);
        const float ev = to_a<float>(eb[u]);
        const float es = plain ? ev : ev * static_cast<float>(od);
        const double xn = sgx * xs + sge * static_cast<double>(es);
        q.y64[u] = plain ? xn : xn * q.inv64[u];
        pt.sm += xn;
        if (od == 0) pt.dm += xn;
    }
    block_partials<double>(sx, pt);
    if (!(last_block(sx) && threadIdx.x < 32)) return;
    double res, resmax, dang, sum;
    take_sums(sx, res, resmax, dang, sum);
    if (threadIdx.x != 0) return;
    sx->sum = sum;
    sx->dang = dang;
    sx->sigma = sum > 0 ? 1.0 / sum : 1.0;
    __threadfence();
    if (q.use_cond) cudaGraphSetConditional(q.h_outer, 1u);
}

// FP16 correction: e = r / sigma_e in the stored form, once the residual
// kernel has chosen sigma_e from ||r||_1.
template <typename Te>
__global__ void k_dc_first_e(DCParams q)
{
    const SolveState *se = q.se;
    if (q.sx->done || se->done) return;
    const float rs = static_cast<float>(1.0 / se->sigma);
    Te *e = static_cast<Te *>(q.e0);
    const int n = q.p.n;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const bool plain = q.weighted || q.p.outdeg[u] == 0;
        const float es = q.r32[u] * rs;
        e[u] = from_a<Te>(plain ? es : es * q.inv32[u]);
    }
}

// Inner stop, relative to ||r||_1 (measured at R-MAT scales 22 and 25: the
// FP32 forms reach the FP64 threshold in the fewest sweeps with these).  The
// 16-bit forms stop at 1e-2, above their storage floor: an FP16 correction
// scaled by its L1 bound stalls near 4e-3 of ||r||_1 at scale 25 (its small
// entries fall into FP16's subnormal range), so a 4e-3 target ran every
// inner solve into the stall rule (65 inner sweeps, slower than FP64); BF16's
// 8-bit significand floors at a few 1e-3.
static double default_eta(pr_precision pr, bool gs)
{
    switch (pr) {
    case PR_FP32_DC: return gs ? 3e-5 : 1e-5;
    case PR_FP16_DC: return 1e-2;
    case PR_BF16_DC: return 1e-2;
    default: return 1e-5;
    }
}

static int default_max_outer(pr_precision pr)
{
    switch (pr) {
    case PR_FP32_DC: return 8;
    case PR_FP16_DC: return 16;
    case PR_BF16_DC: return 24;
    default: return 8;
    }
}

struct DCLaunch {
    const void *f_r, *f_u;
    const void *f_shift;  // fused inner sweeps only
    const void *f_e;      // FP16 only
    unsigned grid_r, grid_u;
    size_t smem_r;
    SweepPlan inner;
};

static pr_status dc_graph(pr_graph *g, int key, DCParams &q, DCLaunch &L,
                          cudaGraphExec_t *exec_out)
{
    for (auto &c : g->graphs)
        if (c.key == key) {
            *exec_out = c.exec;
            return PR_OK;
        }
    cudaGraph_t top = nullptr;
    PR_CUDA(cudaGraphCreate(&top, 0));
    auto fail = [&](cudaError_t e, const char *what) {
        cudaGraphDestroy(top);
        return cuda_status(e, what, __FILE__, __LINE__);
    };
    cudaGraphConditionalHandle h_outer, h_inner;
    cudaError_t e = cudaGraphConditionalHandleCreate(&h_outer, top, 1, cudaGraphCondAssignDefault);
    if (e != cudaSuccess) return fail(e, "outer handle");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h_outer;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t n_outer;
    e = cudaGraphAddNode(&n_outer, top, nullptr, nullptr, 0, &cp);
    if (e != cudaSuccess) return fail(e, "outer while");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    e = cudaGraphConditionalHandleCreate(&h_inner, body, 0, 0);
    if (e != cudaSuccess) return fail(e, "inner handle");
    q.h_inner = h_inner;
    q.h_outer = h_outer;
    q.use_cond = 1;

    // body: residual -> WHILE(inner) { correction sweep } -> update
    cudaKernelNodeParams kp = {};
    void *args_q[] = {&q};
    kp.func = const_cast<void *>(L.f_r);
    kp.gridDim = dim3(L.grid_r);
    kp.blockDim = dim3(SWEEP_BS);
    kp.sharedMemBytes = (unsigned)L.smem_r;
    kp.kernelParams = args_q;
    cudaGraphNode_t n_r;
    e = cudaGraphAddKernelNode(&n_r, body, nullptr, 0, &kp);
    if (e != cudaSuccess) return fail(e, "residual node");
    if (L.f_e) {  // FP16: the first correction iterate, after the scale is known
        kp.func = const_cast<void *>(L.f_e);
        kp.gridDim = dim3(L.grid_u);
        kp.blockDim = dim3(256);
        kp.sharedMemBytes = 0;
        cudaGraphNode_t n_e;
        e = cudaGraphAddKernelNode(&n_e, body, &n_r, 1, &kp);
        if (e != cudaSuccess) return fail(e, "first correction node");
        n_r = n_e;
    }

    cudaGraphNodeParams ci = {};
    ci.type = cudaGraphNodeTypeConditional;
    ci.conditional.handle = h_inner;
    ci.conditional.type = cudaGraphCondTypeWhile;
    ci.conditional.size = 1;
    cudaGraphNode_t n_inner;
    e = cudaGraphAddNode(&n_inner, body, &n_r, nullptr, 1, &ci);
    if (e != cudaSuccess) return fail(e, "inner while");
    cudaGraphNode_t n_last = nullptr;
    pr_status st = add_plan_nodes(ci.conditional.phGraph_out[0], L.inner, h_inner, &n_last);
    if (st != PR_OK) {
        cudaGraphDestroy(top);
        return st;
    }
    if (L.f_shift) {
        kp.func = const_cast<void *>(L.f_shift);
        kp.gridDim = dim3(L.grid_u);
        kp.blockDim = dim3(256);
        kp.sharedMemBytes = 0;
        kp.kernelParams = args_q;
        cudaGraphNode_t n_sh;
        e = cudaGraphAddKernelNode(&n_sh, ci.conditional.phGraph_out[0], &n_last, 1, &kp);
        if (e != cudaSuccess) return fail(e, "shift node");
    }

    kp.func = const_cast<void *>(L.f_u);
    kp.gridDim = dim3(L.grid_u);
    kp.blockDim = dim3(256);
    kp.sharedMemBytes = 0;
    kp.kernelParams = args_q;
    cudaGraphNode_t n_u;
    e = cudaGraphAddKernelNode(&n_u, body, &n_inner, 1, &kp);  // after the inner loop
    if (e != cudaSuccess) return fail(e, "update node");

    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, top, 0);
    if (e != cudaSuccess) return fail(e, "instantiate");
    pr_graph::Cached c;
    c.key = key;
    c.exec = exec;
    c.graph = top;
    g->graphs.push_back(c);
    *exec_out = exec;
    return PR_OK;
}

template <typename Te>
static pr_status run_dc(pr_graph *g, const pr_options *o, const pr_tune &, double *x_out,
                        pr_result *res, cudaStream_t s)
{
    const int32_t n = g->n;
    PR_TRY(buf_alloc(g, g->xbuf, sizeof(double) * (size_t)n + 64, s));  // 16-byte staged reads
    PR_TRY(buf_alloc(g, g->rbuf, sizeof(float) * (size_t)n + 64, s));  // 16-byte widened copies
    const bool gs = o->variant == PR_FUSED_GS;
    const bool fp16 = o->precision == PR_FP16_DC;
    const bool weighted = g->weighted;

    SolveState *sx = g->state.as<SolveState>();
    SolveState *se = sx + 1;
    DCParams q;
    memset(&q, 0, sizeof(q));
    fill_params(g, q.p, true, sizeof(double), false);
    q.p.y0 = g->xbuf.p;
    q.p.y1 = g->xbuf.p;
    q.p.st = sx;
    q.r32 = g->rbuf.as<float>();
    SweepParams inner;
    fill_params(g, inner, false, sizeof(Te), false);  // correction buffers in ybuf, FP32 1/outdeg
    q.e0 = inner.y0;
    q.e1 = inner.y1;
    q.inv32 = g->r_inv32.as<float>();
    q.inv64 = g->r_inv64.as<double>();
    q.y64 = g->xbuf.as<double>();
    q.sx = sx;
    q.se = se;
    q.gs = gs ? 1 : 0;
    q.fp16 = fp16 ? 1 : 0;
    q.weighted = weighted ? 1 : 0;
    inner.rhs = q.r32;
    inner.st = se;
    inner.st_outer = sx;
    inner.dc = 1;
    inner.renorm = 0;
    inner.shift = gs ? 1 : 0;

    SolveState *hs = g->host_state;
    init_state(g, o, hs[0]);
    hs[0].max_outer = o->max_outer > 0 ? o->max_outer : default_max_outer(o->precision);
    hs[0].inner_rel = o->inner_rel > 0 ? o->inner_rel : default_eta(o->precision, gs);
    // the last inner solve stops at 0.5 tau (Jacobi: the residual after the
    // update is at most d times the inner solve's last change, 0.425 tau);
    // fused inner sweeps keep the wider margin 0.05 tau, which the 16-bit
    // forms need (one more outer step otherwise).  Measured at R-MAT scale 22:
    // Jacobi FP32-stored correction 60 -> 54 sweeps, BF16/FP16 66 -> 51.
    hs[0].inner_floor = gs ? 0.05 : 0.5;
    hs[0].scale = 1.0;
    memset(&hs[1], 0, sizeof(SolveState));
    hs[1].d = o->d;
    hs[1].base = hs[0].base;
    hs[1].inv_n = hs[0].inv_n;
    hs[1].sigma = 1.0;
    hs[1].max_iter = 256;  // per inner solve
    hs[1].done = 1;
    PR_CUDA(cudaMemcpyAsync(sx, hs, 2 * sizeof(SolveState), cudaMemcpyHostToDevice, s));
    const int ib = std::max(1, std::min<int>((n + 255) / 256, g->num_sms * 8));
    k_init<double, double><<<ib, 256, 0, s>>>(n, o->x0, g->n2o.as<int32_t>(), q.p.outdeg, q.inv64,
                                             q.y64, sx, 1, weighted ? 1 : 0);
    note_launch();
    PR_LAUNCH_CHECK();

    DCLaunch L;
    L.f_r = weighted ? reinterpret_cast<const void *>(&k_dc_resid<Te, true>)
                     : reinterpret_cast<const void *>(&k_dc_resid<Te, false>);
    L.f_u = reinterpret_cast<const void *>(&k_dc_update<Te>);
    L.f_shift = gs ? reinterpret_cast<const void *>(&k_dc_shift<Te>) : nullptr;
    L.f_e = fp16 ? reinterpret_cast<const void *>(&k_dc_first_e<Te>) : nullptr;
    L.smem_r = layout_of<double, double, false>(q.p).total;
    L.grid_r = sweep_grid(g, q.p.nhubseg + q.p.mi[4] + q.p.nlt, L.f_r, L.smem_r);
    if (L.grid_r == 0) return PR_ERR_INVALID_ARG;
    PR_TRY((make_plan<Te, float>(g, inner, gs, L.inner)));
    L.grid_u = (unsigned)ib;
    bool graph_loop = false;
    if (o->use_graph) {
        const int key = 16 | (gs ? 2 : 0) | (weighted ? 8 : 0) | (g->items.test_stall ? 32 : 0) |
                        ((int)o->precision << 8);
        cudaGraphExec_t exec;
        PR_TRY(dc_graph(g, key, q, L, &exec));
        PR_CUDA(cudaGraphLaunch(exec, s));
        graph_loop = true;
    } else {
        q.use_cond = 0;
        void *aq[] = {&q};
        for (int outer = 0; outer < 1000; ++outer) {
            PR_CUDA(cudaLaunchKernel(L.f_r, dim3(L.grid_r), dim3(SWEEP_BS), aq, L.smem_r, s));
            note_launch();
            if (L.f_e) {
                PR_CUDA(cudaLaunchKernel(L.f_e, dim3(L.grid_u), dim3(256), aq, 0, s));
                note_launch();
            }
            PR_CUDA(cudaMemcpyAsync(hs, sx, 2 * sizeof(SolveState), cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (hs[0].done) break;
            while (true) {
                for (int k = 0; k < 8; ++k) {
                    PR_TRY(launch_plan(L.inner, s));
                    if (L.f_shift) {
                        PR_CUDA(cudaLaunchKernel(L.f_shift, dim3(L.grid_u), dim3(256), aq, 0, s));
                        note_launch();
                    }
                }
                PR_CUDA(cudaMemcpyAsync(hs, sx, 2 * sizeof(SolveState), cudaMemcpyDeviceToHost, s));
                PR_CUDA(cudaStreamSynchronize(s));
                if (hs[1].done) break;
            }
            PR_CUDA(cudaLaunchKernel(L.f_u, dim3(L.grid_u), dim3(256), aq, 0, s));
            note_launch();
        }
    }
    k_output<double><<<ib, 256, 0, s>>>(n, g->o2n.as<int32_t>(), q.p.outdeg, q.y64, q.y64, 0, sx,
                                       x_out, weighted ? 1 : 0);
    note_launch();
    PR_LAUNCH_CHECK();
    PR_CUDA(cudaMemcpyAsync(hs, sx, 2 * sizeof(SolveState), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    if (graph_loop)  // residual and update kernels per outer step, the inner sweeps
        note_launch((uint64_t)2 * hs[0].outer_iter +
                    (uint64_t)(plan_launches(L.inner) + (L.f_shift ? 1 : 0)) *
                        (hs[0].iter - hs[0].outer_iter));
    pr_status st = (pr_status)hs[0].status;
    if (res) {
        res->outer_iters = hs[0].outer_iter;
        res->iters = hs[0].iter - hs[0].outer_iter;
        res->residual = hs[0].norm ? hs[0].resmax : hs[0].res;
        res->sum_before_norm = hs[0].sigma * hs[0].sum;
        res->status = st;
        res->gathered = (int64_t)hs[0].iter * g->m;
    }
    return st;
}

pr_status solve_dc(pr_graph *g, const pr_options *o, const pr_tune &tn, double *x_out,
                   pr_result *res, cudaStream_t s)
{
    switch (o->precision) {
    case PR_FP32_DC: return run_dc<float>(g, o, tn, x_out, res, s);
    case PR_BF16_DC: return run_dc<__nv_bfloat16>(g, o, tn, x_out, res, s);
    case PR_FP16_DC: return run_dc<__half>(g, o, tn, x_out, res, s);
    default:
        set_error("not a defect-correction precision");
        return PR_ERR_INVALID_ARG;
    }
}

}  // namespace fpr
