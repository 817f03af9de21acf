// sweep.cuh -- the fused PageRank sweep (one kernel per sweep).
//
// One launch gathers the stored contribution vector through the in-lists,
// applies teleport and dangling mass, writes the new stored value, and
// accumulates the sweep's L1/max error, dangling mass and total; the block
// that finishes last turns those sums into the next sweep's scalars and the
// stop decision (Algorithm 1/2 `while error > threshold`).
//
// Stored vector y (one entry per vertex):
//   y_u = x~_u * inv_outdeg[u]   if u has out-edges (its contribution, the
//                                 paper's contributionList entry)
//   y_u = x~_u                    if u is dangling (never gathered)
// where the true rank is x_u = sigma * x~_u.  Reading a vertex's own old rank
// and gathering its in-neighbours touch the same array.
//
// Work items, in launch order (heavy first):
//   hub segments  in-degree > t_hub: a block sums hub_seg in-edges; the
//                 block finishing a hub's last segment adds the segment sums
//                 in order and updates the hub
//   mid chunks    t_lo < in-degree <= t_hub: warp per vertex
//   low chunks    in-degree <= t_lo: thread per vertex
// The per-vertex epilogue is a functor, so the same traversal serves the
// PageRank sweep, the correction sweep and the FP64 residual sweep of the
// defect-correction forms.
//
// Jacobi (Algorithm 1, Eq. 2): reads y[iter & 1], writes the other buffer.
// Fused (Algorithm 2, Eq. 9): one buffer updated in place with L2-coherent
// loads and stores, so a vertex sees whichever contribution is there (new if
// its in-neighbour was already updated in this sweep).  Inside a low chunk,
// values updated in earlier rounds are read from shared memory.  After each
// fused sweep the iterate is rescaled to sum 1 by folding 1/sum into sigma.
#pragma once

#include "common.cuh"

namespace fpr {

constexpr int SWEEP_BS = 256;
constexpr int LOW_MAX_ROUNDS = 8;

struct SweepParams {
    int32_t n;
    const int32_t *__restrict__ col_ptr;
    const int32_t *__restrict__ row_idx;
    const int32_t *__restrict__ outdeg;
    const void *inv;              // A[n]: 1/outdeg in the arithmetic type
    const int32_t *bins;          // low | mid | hub vertex ids
    int32_t nlow, nmid, nhub;
    const int32_t *hubseg_start;  // [nhub + 1]
    int32_t nhubseg, hub_seg;
    double *seg_acc;              // [nhubseg]
    int32_t *hub_cnt;             // [nhub]
    int32_t mid_blocks, low_blocks;
    int32_t low_rounds, mid_per_warp;
    void *y0, *y1;                // stored vectors
    const void *rhs;              // A[n] right-hand side, or null: (1-d)/n
    SolveState *st;
    SolveState *st_outer;         // correction sweeps: the outer (FP64) state
    cudaGraphConditionalHandle cond;
    int32_t use_cond;
    int32_t renorm;               // fused sweep: rescale to sum 1
    int32_t dc;                   // correction sweep of a defect-correction solve
};

template <typename T, bool GS>
__device__ __forceinline__ T ld_y(const T *p, int i)
{
    if constexpr (GS) return __ldcg(p + i);
    else return __ldg(p + i);
}

template <typename T, bool GS>
__device__ __forceinline__ void st_y(T *p, int i, T v)
{
    if constexpr (GS) __stcg(p + i, v);
    else p[i] = v;
}

// 16-bit storage: loads/stores through the raw 16-bit pattern
template <>
__device__ __forceinline__ __nv_bfloat16 ld_y<__nv_bfloat16, true>(const __nv_bfloat16 *p, int i)
{
    unsigned short r = __ldcg(reinterpret_cast<const unsigned short *>(p) + i);
    return __ushort_as_bfloat16(r);
}
template <>
__device__ __forceinline__ __nv_bfloat16 ld_y<__nv_bfloat16, false>(const __nv_bfloat16 *p, int i)
{
    unsigned short r = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __ushort_as_bfloat16(r);
}
template <>
__device__ __forceinline__ __half ld_y<__half, true>(const __half *p, int i)
{
    unsigned short r = __ldcg(reinterpret_cast<const unsigned short *>(p) + i);
    return __ushort_as_half(r);
}
template <>
__device__ __forceinline__ __half ld_y<__half, false>(const __half *p, int i)
{
    unsigned short r = __ldg(reinterpret_cast<const unsigned short *>(p) + i);
    return __ushort_as_half(r);
}
template <>
__device__ __forceinline__ void st_y<__nv_bfloat16, true>(__nv_bfloat16 *p, int i, __nv_bfloat16 v)
{
    __stcg(reinterpret_cast<unsigned short *>(p) + i, __bfloat16_as_ushort(v));
}
template <>
__device__ __forceinline__ void st_y<__half, true>(__half *p, int i, __half v)
{
    __stcg(reinterpret_cast<unsigned short *>(p) + i, __half_as_ushort(v));
}

template <typename A, typename T>
__device__ __forceinline__ A to_a(T v) { return static_cast<A>(v); }
template <>
__device__ __forceinline__ float to_a<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_a<float, __half>(__half v) { return __half2float(v); }
template <typename T, typename A>
__device__ __forceinline__ T from_a(A v) { return static_cast<T>(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 from_a<__nv_bfloat16, float>(float v) { return __float2bfloat16_rn(v); }
template <>
__device__ __forceinline__ __half from_a<__half, float>(float v) { return __float2half_rn(v); }

__device__ __forceinline__ double aabs(double v) { return fabs(v); }
__device__ __forceinline__ float aabs(float v) { return fabsf(v); }

template <typename A>
struct Ctx {
    A d, base, sig, rsig, dt;
};

template <typename A>
struct Part {
    A l1 = 0, lmax = 0, dm = 0, sm = 0;
};

template <typename A>
__device__ __forceinline__ Ctx<A> load_ctx(const SolveState *st)
{
    Ctx<A> c;
    c.d = static_cast<A>(st->d);
    c.base = static_cast<A>(st->base);
    c.sig = static_cast<A>(st->sigma);
    c.rsig = static_cast<A>(1.0 / st->sigma);
    c.dt = static_cast<A>(st->dang * st->inv_n);
    return c;
}

// Epilogue of the PageRank (or correction) sweep: new value of vertex u from
// its gathered sum `acc` (stored units); returns the stored value written.
template <typename T, typename A, bool GS>
struct SweepFin {
    const SweepParams &p;
    Ctx<A> c;
    const T *yin;
    T *yout;
    Part<A> pt;
    __device__ SweepFin(const SweepParams &p_, const Ctx<A> &c_, const T *yi, T *yo)
        : p(p_), c(c_), yin(yi), yout(yo) {}
    __device__ __forceinline__ T operator()(int u, A acc)
    {
        const int od = p.outdeg[u];
        const A inv = static_cast<const A *>(p.inv)[u];
        const A yo = to_a<A>(ld_y<T, GS>(yin, u));
        const A xold = od > 0 ? yo * static_cast<A>(od) : yo;  // stored units
        const A r = p.rhs ? static_cast<const A *>(p.rhs)[u] : c.base;
        const A xnew = r + c.d * (c.sig * (acc + c.dt));       // true units
        const A diff = aabs(xnew - c.sig * xold);
        const A xs = xnew * c.rsig;                             // stored units
        const T yn = from_a<T>(od > 0 ? xs * inv : xs);
        st_y<T, GS>(yout, u, yn);
        pt.l1 += diff;
        pt.lmax = diff > pt.lmax ? diff : pt.lmax;
        pt.sm += xs;
        if (od == 0) pt.dm += xs;
        return yn;
    }
};

// Sum of y over in-list slots [a, b) by one warp, int4 index loads in the body.
template <typename T, typename A, bool GS>
__device__ __forceinline__ A warp_gather(const int32_t *__restrict__ row_idx, const T *y, int a,
                                         int b, int lane)
{
    A acc = 0;
    if (b - a < 64) {
        for (int i = a + lane; i < b; i += 32) acc += to_a<A>(ld_y<T, GS>(y, row_idx[i]));
        return acc;
    }
    const int a4 = (a + 3) & ~3;
    const int b4 = b & ~3;
    if (lane < a4 - a) acc += to_a<A>(ld_y<T, GS>(y, row_idx[a + lane]));
    for (int i = a4 + 4 * lane; i < b4; i += 128) {
        const int4 q = __ldg(reinterpret_cast<const int4 *>(row_idx + i));
        A s0 = to_a<A>(ld_y<T, GS>(y, q.x));
        A s1 = to_a<A>(ld_y<T, GS>(y, q.y));
        A s2 = to_a<A>(ld_y<T, GS>(y, q.z));
        A s3 = to_a<A>(ld_y<T, GS>(y, q.w));
        acc += (s0 + s1) + (s2 + s3);
    }
    if (lane < b - b4) acc += to_a<A>(ld_y<T, GS>(y, row_idx[b4 + lane]));
    return acc;
}

// Reduces the block's partial sums and adds them to the sweep accumulators.
template <typename A>
__device__ __forceinline__ void block_partials(SolveState *st, const Part<A> &pt)
{
    __shared__ double red[4][SWEEP_BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double l1 = warp_sum(static_cast<double>(pt.l1));
    double lm = warp_max(static_cast<double>(pt.lmax));
    double dm = warp_sum(static_cast<double>(pt.dm));
    double sm = warp_sum(static_cast<double>(pt.sm));
    if (lane == 0) {
        red[0][warp] = l1;
        red[1][warp] = lm;
        red[2][warp] = dm;
        red[3][warp] = sm;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = blockDim.x >> 5;
        double a = 0, b = 0, c = 0, e = 0;
        for (int w = 0; w < nw; ++w) {
            a += red[0][w];
            b = fmax(b, red[1][w]);
            c += red[2][w];
            e += red[3][w];
        }
        AccSlot &s = st->acc[blockIdx.x % ACC_SLOTS];
        if (a != 0) fx_add(&s.res_hi, &s.res_lo, a);
        if (b != 0) atomicMax(&s.res_max, static_cast<unsigned long long>(__double_as_longlong(b)));
        if (c != 0) fx_add(&s.dang_hi, &s.dang_lo, c);
        if (e != 0) fx_add(&s.sum_hi, &s.sum_lo, e);
    }
}

// Called by every block at its end; true in the block that arrives last.
__device__ __forceinline__ bool last_block(SolveState *st)
{
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    return is_last;
}

__device__ __forceinline__ void take_sums(SolveState *st, double &res, double &resmax,
                                          double &dang, double &sum)
{
    __threadfence();
    long long rh = 0, rl = 0, dh = 0, dl = 0, sh = 0, sl = 0;
    unsigned long long mx = 0;
    for (int k = 0; k < ACC_SLOTS; ++k) {
        volatile AccSlot *v = &st->acc[k];
        rh += v->res_hi;
        rl += v->res_lo;
        dh += v->dang_hi;
        dl += v->dang_lo;
        sh += v->sum_hi;
        sl += v->sum_lo;
        mx = v->res_max > mx ? v->res_max : mx;
        v->res_hi = v->res_lo = v->dang_hi = v->dang_lo = v->sum_hi = v->sum_lo = 0;
        v->res_max = 0;
    }
    res = fx_value(rh, rl);
    resmax = __longlong_as_double(static_cast<long long>(mx));
    dang = fx_value(dh, dl);
    sum = fx_value(sh, sl);
    st->ticket = 0;
}

// Closes a PageRank sweep (dc == 0) or a correction sweep (dc != 0): next
// scalars, history, stop test, loop condition.
__device__ __forceinline__ void close_sweep(const SweepParams &p)
{
    SolveState *st = p.st;
    double res, resmax, dang, sum;
    take_sums(st, res, resmax, dang, sum);
    const int it = st->iter + 1;
    st->iter = it;
    st->res = res;
    st->resmax = resmax;
    st->dang = dang;
    st->sum = sum;
    if (p.renorm && sum > 0) st->sigma = 1.0 / sum;
    const double err = st->norm ? resmax : res;
    bool stop, conv;
    if (!p.dc) {
        if (st->history) st->history[it - 1] = err;
        conv = err <= st->tau;
        stop = conv || it >= st->max_iter;
        st->status = conv ? PR_OK : PR_NOT_CONVERGED;
    } else {
        SolveState *so = p.st_outer;
        const int total = so->iter + 1;
        so->iter = total;
        st->inner_iter += 1;
        if (so->history) so->history[total - 1] = err;
        conv = err <= st->tau;
        stop = conv || it >= st->max_iter || total >= so->max_iter;
    }
    st->done = stop ? 1 : 0;
    __threadfence();
    if (p.use_cond) cudaGraphSetConditional(p.cond, stop ? 0u : 1u);
}

// Hub segment b: a block sums hub_seg in-edges of one hub; the block that
// completes the hub's last segment adds the segment sums in order and calls
// the epilogue (thread 0).
template <typename T, typename A, bool GS, typename Fin>
__device__ __forceinline__ void hub_segment(const SweepParams &p, int b, const T *yin, Fin &fin)
{
    __shared__ double red[SWEEP_BS / 32];
    __shared__ int sh_h;
    if (threadIdx.x == 0) {
        int lo = 0, hi = p.nhub - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (p.hubseg_start[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        sh_h = lo;
    }
    __syncthreads();
    const int h = sh_h;
    const int u = p.bins[p.nlow + p.nmid + h];
    const int s0 = p.hubseg_start[h];
    const int nseg = p.hubseg_start[h + 1] - s0;
    const int k = b - s0;
    const int a = p.col_ptr[u] + k * p.hub_seg;
    const int e = min(a + p.hub_seg, p.col_ptr[u + 1]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int per = (((e - a) + nw - 1) / nw + 3) & ~3;  // keep warp starts 4-aligned
    const int wa = min(e, a + warp * per), wb = min(e, wa + per);
    A acc = warp_gather<T, A, GS>(p.row_idx, yin, wa, wb, lane);
    double s = warp_sum(static_cast<double>(acc));
    if (lane == 0) red[warp] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double tot = 0;
        for (int w = 0; w < nw; ++w) tot += red[w];
        p.seg_acc[b] = tot;
        __threadfence();
        const int done = atomicAdd(&p.hub_cnt[h], 1);
        if (done == nseg - 1) {
            __threadfence();
            const volatile double *sa = p.seg_acc;
            double all = 0;
            for (int j = 0; j < nseg; ++j) all += sa[s0 + j];
            p.hub_cnt[h] = 0;
            fin(u, static_cast<A>(all));
        }
    }
}

template <typename T, typename A, bool GS, typename Fin>
__device__ __forceinline__ void mid_chunk(const SweepParams &p, int b, const T *yin, Fin &fin)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int base = b * nw * p.mid_per_warp + warp * p.mid_per_warp;
    for (int k = 0; k < p.mid_per_warp; ++k) {
        const int idx = base + k;
        if (idx >= p.nmid) break;
        const int u = p.bins[p.nlow + idx];
        const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
        A acc = warp_gather<T, A, GS>(p.row_idx, yin, a, e, lane);
        acc = warp_sum(acc);
        if (lane == 0) fin(u, acc);
    }
}

template <typename T, typename A, bool GS, typename Fin>
__device__ __forceinline__ void low_chunk(const SweepParams &p, int b, const T *yin, Fin &fin)
{
    const int per = blockDim.x * p.low_rounds;
    const int base = b * per;
    if constexpr (!GS) {
        for (int r = 0; r < p.low_rounds; ++r) {
            const int idx = base + r * blockDim.x + threadIdx.x;
            if (idx >= p.nlow) break;
            const int u = p.bins[idx];
            const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
            A acc = 0;
            int i = a;
            for (; i + 4 <= e; i += 4) {  // four independent gathers in flight
                const int v0 = p.row_idx[i], v1 = p.row_idx[i + 1];
                const int v2 = p.row_idx[i + 2], v3 = p.row_idx[i + 3];
                const A s0 = to_a<A>(ld_y<T, GS>(yin, v0)), s1 = to_a<A>(ld_y<T, GS>(yin, v1));
                const A s2 = to_a<A>(ld_y<T, GS>(yin, v2)), s3 = to_a<A>(ld_y<T, GS>(yin, v3));
                acc += s0;  // same association as a sequential sum
                acc += s1;
                acc += s2;
                acc += s3;
            }
            for (; i < e; ++i) acc += to_a<A>(ld_y<T, GS>(yin, p.row_idx[i]));
            fin(u, acc);
        }
    } else {
        // Tile of this chunk: ids (ascending) and the values updated in
        // earlier rounds, kept in shared memory for in-tile reads.
        __shared__ int ids[SWEEP_BS * LOW_MAX_ROUNDS];
        __shared__ T fresh[SWEEP_BS * LOW_MAX_ROUNDS];
        const int cnt = min(per, p.nlow - base);
        for (int i = threadIdx.x; i < cnt; i += blockDim.x) ids[i] = p.bins[base + i];
        __syncthreads();
        const int first = ids[0];
        for (int r = 0; r < p.low_rounds; ++r) {
            const int done = min(r * (int)blockDim.x, cnt);  // entries of earlier rounds
            const int last = done > 0 ? ids[done - 1] : -1;
            const int idx = r * blockDim.x + threadIdx.x;
            if (idx < cnt) {
                const int u = ids[idx];
                const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
                A acc = 0;
                for (int i = a; i < e; ++i) {
                    const int v = p.row_idx[i];
                    int pos = -1;
                    if (v >= first && v <= last) {
                        int lo = 0, hi = done - 1;
                        while (lo < hi) {
                            int mid = (lo + hi) >> 1;
                            if (ids[mid] < v) lo = mid + 1;
                            else hi = mid;
                        }
                        if (ids[lo] == v) pos = lo;
                    }
                    acc += pos >= 0 ? to_a<A>(fresh[pos]) : to_a<A>(ld_y<T, GS>(yin, v));
                }
                fresh[idx] = fin(u, acc);
            }
            __syncthreads();
        }
    }
}

// Persistent loop: block b takes items b, b + G, b + 2G, ... (G = grid size)
// in that fixed order, so every block's partial sums are reproducible.
template <typename T, typename A, bool GS, typename Fin>
__device__ __forceinline__ void run_items(const SweepParams &p, const T *yin, Fin &fin)
{
    const int nitems = p.nhubseg + p.mid_blocks + p.low_blocks;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        int b = item;
        if (b < p.nhubseg) {
            hub_segment<T, A, GS>(p, b, yin, fin);
        } else if ((b -= p.nhubseg) < p.mid_blocks) {
            mid_chunk<T, A, GS>(p, b, yin, fin);
        } else {
            b -= p.mid_blocks;
            low_chunk<T, A, GS>(p, b, yin, fin);
        }
        __syncthreads();  // shared memory of this item is reused by the next
    }
}

template <typename T, typename A, bool GS>
__global__ void __launch_bounds__(SWEEP_BS, 4) k_sweep(SweepParams p)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
        return;
    }
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
    SweepFin<T, A, GS> fin(p, load_ctx<A>(st), yin, yout);
    run_items<T, A, GS>(p, yin, fin);
    block_partials<A>(st, fin.pt);
    if (last_block(st) && threadIdx.x == 0) close_sweep(p);
}

// Fused sweep in strict increasing id order (Eq. 9 exactly): one warp, one
// vertex at a time.  For small graphs and checks only.
template <typename T, typename A>
__global__ void k_sweep_serial(SweepParams p)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.use_cond && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    T *y = static_cast<T *>(p.y0);
    SweepFin<T, A, true> fin(p, load_ctx<A>(st), y, y);
    const int lane = threadIdx.x & 31;
    for (int u = 0; u < p.n; ++u) {
        const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
        A acc = 0;
        for (int i = a + lane; i < e; i += 32) acc += to_a<A>(ld_y<T, true>(y, p.row_idx[i]));
        acc = warp_sum(acc);
        if (lane == 0) fin(u, acc);
        __syncwarp();
    }
    block_partials<A>(st, fin.pt);
    if (last_block(st) && threadIdx.x == 0) close_sweep(p);
}

// ------------------------------------------------------------ init/output
// y <- stored form of x0 (or 1/n); sums of the start vector.
template <typename T, typename A>
__global__ void k_init(int32_t n, const double *x0, const int32_t *__restrict__ outdeg,
                       const A *__restrict__ inv, T *y, SolveState *st, int renorm)
{
    Part<A> pt;
    const double inv_n = st->inv_n;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const A x = static_cast<A>(x0 ? x0[u] : inv_n);
        const int od = outdeg[u];
        y[u] = static_cast<T>(od > 0 ? x * inv[u] : x);
        pt.sm += x;
        if (od == 0) pt.dm += x;
    }
    block_partials<A>(st, pt);
    if (last_block(st) && threadIdx.x == 0) {
        double res, resmax, dang, sum;
        take_sums(st, res, resmax, dang, sum);
        st->dang = dang;
        st->sum = sum;
        st->sigma = (renorm && sum > 0) ? 1.0 / sum : 1.0;
    }
}

// x_out <- x~ / sum(x~) from the current stored vector (Jacobi alternates
// buffers: after an odd number of sweeps the iterate is in y1).
template <typename T>
__global__ void k_output(int32_t n, const int32_t *__restrict__ outdeg, const T *__restrict__ y0,
                         const T *__restrict__ y1, int jacobi, const SolveState *st,
                         double *x_out)
{
    const double rs = 1.0 / st->sum;
    const T *y = (jacobi && (st->iter & 1)) ? y1 : y0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int od = outdeg[u];
        const double v = static_cast<double>(y[u]);
        x_out[u] = (od > 0 ? v * static_cast<double>(od) : v) * rs;
    }
}

}  // namespace fpr
