// sweep.cuh -- the fused PageRank sweep (one kernel per sweep).
//
// One launch gathers the stored contribution vector through the in-lists,
// applies teleport and dangling mass, writes the new stored value, and
// accumulates the sweep's L1/max error, dangling mass and total; the block
// that finishes last turns those sums into the next sweep's scalars and the
// stop decision (Algorithm 1/2 `while error > threshold`).
//
// Everything runs in the degree-ordered numbering (in-degree descending):
// hubs are the ids [0, nhub), and the most-gathered contributions share
// cache lines.  Stored vector y (one entry per vertex):
//   y_u = x~_u * inv_outdeg[u]   if u has out-edges (its contribution, the
//                                 paper's contributionList entry)
//   y_u = x~_u                    if u is dangling (never gathered), or for
//                                 weighted graphs (P is applied per in-edge)
// where the true rank is x_u = sigma * x~_u.  Reading a vertex's own old rank
// and gathering its in-neighbours touch the same array.
//
// Work items, in launch order (heavy first), taken round-robin by a
// persistent grid:
//   hub segment  hub_seg in-edges of one hub summed by a block; the block
//                finishing a hub's last segment adds the segment sums in order
//                and updates the hub (block per vertex)
//   tile         consecutive non-hub vertices with at most `tile` units of
//                work: all their in-edges are gathered into shared memory with
//                16-byte index loads (every gather of the tile in flight at
//                once), then reduced by a warp per vertex (in-degree > t_lo)
//                or a thread per vertex (in-degree <= t_lo)
// The per-vertex epilogue is a functor, so the same traversal serves the
// PageRank sweep, the correction sweep and the FP64 residual sweep of the
// defect-correction forms.
//
// Jacobi (Algorithm 1, Eq. 2): reads y[iter & 1], writes the other buffer.
// Fused (Algorithm 2, Eq. 9): one buffer updated in place with L2-coherent
// loads and stores, so a vertex sees whichever contribution is there (new if
// its in-neighbour was already updated in this sweep).  Inside a tile, the
// vertices are updated warp-vertices first, then thread-vertices in rounds;
// a later vertex reads the values of the tile's earlier vertices from shared
// memory.  After each fused sweep the iterate is rescaled to sum 1 by
// folding 1/sum into sigma.
#pragma once

#include "common.cuh"

namespace fpr {

constexpr int SWEEP_BS = 256;

struct SweepParams {
    int32_t n;
    const int32_t *__restrict__ col_ptr;  // relabelled in-lists
    const int32_t *__restrict__ row_idx;  // (padded by 4 entries)
    const int32_t *__restrict__ outdeg;
    const void *inv;              // A[n]: 1/outdeg in the arithmetic type
    const void *ew;               // A[m]: P per in-list slot (weighted) or null
    int32_t nhub;
    const int32_t *hubseg_start;  // [nhub + 1]
    int32_t nhubseg, hub_seg;
    double *seg_acc;              // [nhubseg]
    int32_t *hub_cnt;             // [nhub]
    int32_t ntiles, tile_c, maxe;
    const int32_t *tile_start;    // [ntiles + 1]
    const int32_t *tile_mid;      // [ntiles]
    int32_t stage;                // y[0, stage) is copied to shared memory at
                                  // the start of the sweep (hottest sources)
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
    return __ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __nv_bfloat16 ld_y<__nv_bfloat16, false>(const __nv_bfloat16 *p, int i)
{
    return __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __half ld_y<__half, true>(const __half *p, int i)
{
    return __ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __half ld_y<__half, false>(const __half *p, int i)
{
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p) + i));
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

// gathered term of in-list slot i whose source holds `val`
template <typename A, bool W>
__device__ __forceinline__ A edge_term(const SweepParams &p, int i, A val)
{
    if constexpr (W) return static_cast<const A *>(p.ew)[i] * val;
    else return val;
}

// Epilogue of the PageRank (or correction) sweep: new value of vertex u from
// its gathered sum `acc` (stored units); returns the stored value written.
template <typename T, typename A, bool GS, bool W>
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
        const A yo = to_a<A>(ld_y<T, GS>(yin, u));
        const A xold = (W || od == 0) ? yo : yo * static_cast<A>(od);  // stored units
        const A r = p.rhs ? static_cast<const A *>(p.rhs)[u] : c.base;
        const A xnew = r + c.d * (c.sig * (acc + c.dt));                 // true units
        const A diff = aabs(xnew - c.sig * xold);
        const A xs = xnew * c.rsig;                                       // stored units
        const A inv = static_cast<const A *>(p.inv)[u];
        const T yn = from_a<T>((W || od == 0) ? xs : xs * inv);
        st_y<T, GS>(yout, u, yn);
        pt.l1 += diff;
        pt.lmax = diff > pt.lmax ? diff : pt.lmax;
        pt.sm += xs;
        if (od == 0) pt.dm += xs;
        return yn;
    }
};

// Where a gathered contribution comes from: the copy of y[0, nstaged) in
// shared memory (the hottest sources in the degree-ordered ids), else y.
template <typename T, bool GS>
struct Src {
    const T *y;
    const T *staged;
    int nstaged;
    __device__ __forceinline__ T operator()(int v) const
    {
        return v < nstaged ? staged[v] : ld_y<T, GS>(y, v);
    }
};

// Sum over in-list slots [a, b) by one warp, 16-byte index loads in the body.
template <typename T, typename A, bool GS, bool W>
__device__ __forceinline__ A warp_gather(const SweepParams &p, const Src<T, GS> &y, int a, int b,
                                         int lane)
{
    const int32_t *__restrict__ row_idx = p.row_idx;
    A acc = 0;
    if (b - a < 64) {
        for (int i = a + lane; i < b; i += 32)
            acc += edge_term<A, W>(p, i, to_a<A>(y(row_idx[i])));
        return acc;
    }
    const int a4 = (a + 3) & ~3;
    const int b4 = b & ~3;
    if (lane < a4 - a) acc += edge_term<A, W>(p, a + lane, to_a<A>(y(row_idx[a + lane])));
    for (int i = a4 + 4 * lane; i < b4; i += 128) {
        const int4 q = __ldg(reinterpret_cast<const int4 *>(row_idx + i));
        const A s0 = edge_term<A, W>(p, i, to_a<A>(y(q.x)));
        const A s1 = edge_term<A, W>(p, i + 1, to_a<A>(y(q.y)));
        const A s2 = edge_term<A, W>(p, i + 2, to_a<A>(y(q.z)));
        const A s3 = edge_term<A, W>(p, i + 3, to_a<A>(y(q.w)));
        acc += (s0 + s1) + (s2 + s3);
    }
    if (lane < b - b4) acc += edge_term<A, W>(p, b4 + lane, to_a<A>(y(row_idx[b4 + lane])));
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

// Hub segment b: a block sums hub_seg in-edges of hub h; the block that
// completes the hub's last segment adds the segment sums in order and calls
// the epilogue (thread 0).
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void hub_segment(const SweepParams &p, int b, const Src<T, GS> &yin,
                                            Fin &fin)
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
    const int h = sh_h;  // hub vertex id (hubs are the first ids)
    const int s0 = p.hubseg_start[h];
    const int nseg = p.hubseg_start[h + 1] - s0;
    const int k = b - s0;
    const int a = p.col_ptr[h] + k * p.hub_seg;
    const int e = min(a + p.hub_seg, p.col_ptr[h + 1]);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const int per = (((e - a) + nw - 1) / nw + 3) & ~3;
    const int wa = min(e, a + warp * per), wb = min(e, wa + per);
    A acc = warp_gather<T, A, GS, W>(p, yin, wa, wb, lane);
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
            fin(h, static_cast<A>(all));
        }
    }
}

// Shared memory of a tile: gathered terms [maxe] (A); for the fused sweep
// also the source of each slot [maxe] (int) and the tile's new stored
// values [tile_c] (T).
template <typename T, typename A, bool GS>
__host__ __device__ constexpr size_t tile_smem_bytes(int maxe, int tile_c)
{
    return GS ? (size_t)maxe * sizeof(A) + (size_t)maxe * sizeof(int) + (size_t)tile_c * sizeof(T) + 64
              : (size_t)maxe * sizeof(A) + 16;
}

template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void tile_item(const SweepParams &p, int k, const Src<T, GS> &yin,
                                          Fin &fin, unsigned char *smem)
{
    const int v0 = p.tile_start[k], v1 = p.tile_start[k + 1];
    if (v0 >= v1) return;
    const int vm = p.tile_mid[k];
    const int ea = p.col_ptr[v0], eb = p.col_ptr[v1];
    const int ne = eb - ea;
    A *vals = reinterpret_cast<A *>(smem);
    int *sidx = reinterpret_cast<int *>(smem + (size_t)p.maxe * sizeof(A));
    T *fresh = reinterpret_cast<T *>(smem + (size_t)p.maxe * (sizeof(A) + sizeof(int)));

    // phase A: every in-edge of the tile; each thread loads two 16-byte index
    // vectors before issuing their eight gathers
    const int base = ea & ~3;
    const int span = eb - base;
    const int step = blockDim.x * 4;
    for (int j0 = threadIdx.x * 4; j0 < span; j0 += 2 * step) {
        const int j1 = j0 + step;
        const int4 q0 = __ldg(reinterpret_cast<const int4 *>(p.row_idx + base + j0));
        int4 q1 = make_int4(0, 0, 0, 0);
        if (j1 < span) q1 = __ldg(reinterpret_cast<const int4 *>(p.row_idx + base + j1));
        const int src[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        A got[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int sl = base + (c < 4 ? j0 + c : j1 + c - 4) - ea;
            got[c] = (sl >= 0 && sl < ne) ? to_a<A>(yin(src[c])) : A(0);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int sl = base + (c < 4 ? j0 + c : j1 + c - 4) - ea;
            if (sl >= 0 && sl < ne) {
                vals[sl] = edge_term<A, W>(p, ea + sl, got[c]);
                if constexpr (GS) sidx[sl] = src[c];
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // phase B1: in-degree > t_lo (the tile's first vertices): warp per vertex
    for (int u = v0 + warp; u < vm; u += nw) {
        const int a = p.col_ptr[u] - ea, e = p.col_ptr[u + 1] - ea;
        A acc = 0;
        for (int i = a + lane; i < e; i += 32) acc += vals[i];
        acc = warp_sum(acc);
        if (lane == 0) {
            const T yn = fin(u, acc);
            if constexpr (GS) fresh[u - v0] = yn;
        }
    }
    if constexpr (GS) __syncthreads();
    // phase B2: thread per vertex, in rounds of blockDim
    for (int u0 = vm; u0 < v1; u0 += blockDim.x) {
        const int u = u0 + threadIdx.x;
        if (u < v1) {
            const int a = p.col_ptr[u] - ea, e = p.col_ptr[u + 1] - ea;
            A acc = 0;
            for (int i = a; i < e; ++i) {
                A val = vals[i];
                if constexpr (GS) {
                    // in-tile source already updated in this sweep: fresh value
                    const int v = sidx[i];
                    if (v >= v0 && v < u0) val = edge_term<A, W>(p, ea + i, to_a<A>(fresh[v - v0]));
                }
                acc += val;
            }
            const T yn = fin(u, acc);
            if constexpr (GS) fresh[u - v0] = yn;
        }
        if constexpr (GS) __syncthreads();
    }
    __syncthreads();  // shared memory is reused by the next item
}

// Bytes of dynamic shared memory for the staged copy of y[0, stage).
template <typename T>
__host__ __device__ constexpr size_t stage_bytes(int stage)
{
    return ((size_t)stage * sizeof(T) + 15) & ~(size_t)15;
}

// Persistent loop: block b takes items b, b + G, b + 2G, ... (G = grid size)
// in that fixed order, so every block's partial sums are reproducible.  The
// block first copies the hottest contributions y[0, stage) into shared
// memory (16-byte loads); for the fused sweep that copy is a snapshot, i.e.
// those reads may see a value older than the one in y, as any asynchronous
// read may.
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void run_items(const SweepParams &p, const T *yin, Fin &fin)
{
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    T *staged = reinterpret_cast<T *>(dyn_smem);
    const int nst = p.stage;
    {
        const int4 *src = reinterpret_cast<const int4 *>(yin);
        int4 *dst = reinterpret_cast<int4 *>(dyn_smem);
        const int nvec = (int)(stage_bytes<T>(nst) / 16);
        for (int i = threadIdx.x; i < nvec; i += blockDim.x)
            dst[i] = GS ? __ldcg(src + i) : __ldg(src + i);
        __syncthreads();
    }
    Src<T, GS> s{yin, staged, nst};
    unsigned char *tile_smem = dyn_smem + stage_bytes<T>(nst);
    const int nitems = p.nhubseg + p.ntiles;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x) {
        if (item < p.nhubseg) {
            hub_segment<T, A, GS, W>(p, item, s, fin);
            __syncthreads();
        } else {
            tile_item<T, A, GS, W>(p, item - p.nhubseg, s, fin, tile_smem);
        }
    }
}

template <typename T, typename A, bool GS, bool W>
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
    SweepFin<T, A, GS, W> fin(p, load_ctx<A>(st), yin, yout);
    run_items<T, A, GS, W>(p, yin, fin);
    block_partials<A>(st, fin.pt);
    if (last_block(st) && threadIdx.x == 0) close_sweep(p);
}

// Fused sweep in strict increasing input-id order (Eq. 9 exactly): one warp,
// one vertex at a time, on the input-id in-lists.  For small graphs and
// checks only (unweighted).
template <typename T, typename A>
__global__ void k_sweep_serial(SweepParams p)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.use_cond && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    T *y = static_cast<T *>(p.y0);
    SweepFin<T, A, true, false> fin(p, load_ctx<A>(st), y, y);
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
// y <- stored form of the start vector (x0 in input ids, or 1/n), in the
// sweep's numbering (n2o maps it to input ids; null: same ids); sums of it.
template <typename T, typename A>
__global__ void k_init(int32_t n, const double *x0, const int32_t *__restrict__ n2o,
                       const int32_t *__restrict__ outdeg, const A *__restrict__ inv, T *y,
                       SolveState *st, int renorm, int weighted)
{
    Part<A> pt;
    const double inv_n = st->inv_n;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const A x = static_cast<A>(x0 ? x0[n2o ? n2o[u] : u] : inv_n);
        const int od = outdeg[u];
        y[u] = from_a<T>((weighted || od == 0) ? x : x * inv[u]);
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

__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return static_cast<double>(v); }
__device__ __forceinline__ double to_d(__nv_bfloat16 v) { return static_cast<double>(__bfloat162float(v)); }
__device__ __forceinline__ double to_d(__half v) { return static_cast<double>(__half2float(v)); }

// x_out (input ids) <- x~ / sum(x~) from the current stored vector (Jacobi
// alternates buffers: after an odd number of sweeps the iterate is in y1).
template <typename T>
__global__ void k_output(int32_t n, const int32_t *__restrict__ o2n,
                         const int32_t *__restrict__ outdeg, const T *__restrict__ y0,
                         const T *__restrict__ y1, int jacobi, const SolveState *st,
                         double *x_out, int weighted)
{
    const double rs = 1.0 / st->sum;
    const T *y = (jacobi && (st->iter & 1)) ? y1 : y0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int k = o2n ? o2n[u] : u;
        const int od = outdeg[k];
        const double v = to_d(y[k]);
        x_out[u] = ((weighted || od == 0) ? v : v * static_cast<double>(od)) * rs;
    }
}

}  // namespace fpr
