// sweep.cuh -- the fused PageRank sweep (one kernel per sweep).
//
// One launch gathers the stored contribution vector through the in-lists,
// applies teleport and dangling mass, writes the new stored value, and
// accumulates the sweep's L1/max error, dangling mass and total; the block
// that finishes last turns those sums into the next sweep's scalars and the
// stop decision (Algorithm 1/2 `while error > threshold`).
//
// Everything runs in the degree-ordered numbering (in-degree descending):
// hubs are the ids [0, nhub).  Stored vector y (one entry per vertex):
//   y_u = x~_u * inv_outdeg[u]   if u has out-edges (its contribution, the
//                                 paper's contributionList entry)
//   y_u = x~_u                    if u is dangling (never gathered), or for
//                                 weighted graphs (P is applied per in-edge)
// where the true rank is x_u = sigma * x~_u.  Reading a vertex's own old rank
// and gathering its in-neighbours touch the same array.
//
// Work items, in launch order (heavy first), each described by
// {v0, v1, ea, eb} (vertices [v0, v1), in-list slots [ea, eb)):
//   hub segment  hub_seg in-edges of one hub (v1 = v0 + 1) summed by a block;
//                the block finishing a hub's last segment adds the segment
//                sums in order and updates the hub (block per vertex)
//   tile         consecutive non-hub vertices with at most `tile` units of
//                work, reduced by a warp per vertex (in-degree > t_lo) or a
//                thread per vertex (in-degree <= t_lo)
// A persistent grid takes the items round-robin.  Each block double-buffers
// them in shared memory: while it works on one item, bulk copies (TMA,
// cp.async.bulk) bring the next item's contiguous streams -- in-list indices,
// offsets, out-degrees, 1/outdeg, old stored values, right-hand side, edge
// weights -- so the only memory latency left on the item's path is the random
// gather of the in-neighbours' contributions, all of which are in flight at
// once.  The per-vertex epilogue is a functor, so the same traversal serves
// the PageRank sweep, the correction sweep and the FP64 residual sweep of the
// defect-correction forms.
//
// Jacobi (Algorithm 1, Eq. 2): reads y[iter & 1], writes the other buffer.
// Fused (Algorithm 2, Eq. 9): one buffer updated in place with L2-coherent
// loads and stores, so a vertex sees whichever contribution is there (new if
// its in-neighbour was already updated in this sweep).  Inside a tile, the
// vertices are updated warp-vertices first, then thread-vertices in rounds;
// a later vertex reads the new values of the tile's earlier vertices from
// shared memory.  After each fused sweep the iterate is rescaled to sum 1 by
// folding 1/sum into sigma.
#pragma once

#include "common.cuh"
#include "tma.cuh"

namespace fpr {

constexpr int SWEEP_BS = 256;
constexpr uint32_t DEFAULT_WAIT_LIMIT = 1u << 22;

struct SweepParams {
    int32_t n;
    const int32_t *__restrict__ col_ptr;  // relabelled in-lists (padded)
    const int32_t *__restrict__ row_idx;
    const int32_t *__restrict__ outdeg;
    const void *inv;              // A[n]: 1/outdeg in the arithmetic type
    const void *ew;               // A[m]: P per in-list slot (weighted) or null
    const int4 *desc;             // [nhubseg + ntiles] item descriptors
    int32_t nhub, nhubseg, ntiles, t_lo;
    const int32_t *hubseg_start;  // [nhub + 1]
    double *seg_acc;              // [nhubseg]
    int32_t *hub_cnt;             // [nhub]
    int32_t idxcap, vcap;         // shared-memory capacity of one item
    int32_t stage;                // y[0, stage) is copied to shared memory
    uint32_t wait_limit;
    int32_t test_stall;
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

// Epilogue of the PageRank (or correction) sweep: new value of vertex u from
// its gathered sum `acc` (stored units), its out-degree, 1/outdeg, old stored
// value and right-hand side; returns the stored value written.
template <typename T, typename A, bool GS, bool W>
struct SweepFin {
    const SweepParams &p;
    Ctx<A> c;
    T *yout;
    Part<A> pt;
    __device__ SweepFin(const SweepParams &p_, const Ctx<A> &c_, T *yo) : p(p_), c(c_), yout(yo) {}
    __device__ __forceinline__ A base() const { return c.base; }
    __device__ __forceinline__ T operator()(int u, A acc, int od, A inv, T yold, A r)
    {
        const A yo = to_a<A>(yold);
        const A xold = (W || od == 0) ? yo : yo * static_cast<A>(od);  // stored units
        const A xnew = r + c.d * (c.sig * (acc + c.dt));                 // true units
        const A diff = aabs(xnew - c.sig * xold);
        const A xs = xnew * c.rsig;                                       // stored units
        const T yn = from_a<T>((W || od == 0) ? xs : xs * inv);
        st_y<T, GS>(yout, u, yn);
        pt.l1 += diff;
        pt.lmax = diff > pt.lmax ? diff : pt.lmax;
        pt.sm += xs;
        if (od == 0) pt.dm += xs;
        return yn;
    }
};

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
// scalars, history, stop test, loop condition.  A device-side error ends the
// loop with that status.
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
    const int error = *reinterpret_cast<volatile int *>(&st->error);
    if (!p.dc) {
        if (st->history) st->history[it - 1] = err;
        conv = err <= st->tau;
        stop = conv || it >= st->max_iter || error;
        st->status = error ? error : (conv ? PR_OK : PR_NOT_CONVERGED);
    } else {
        SolveState *so = p.st_outer;
        const int total = so->iter + 1;
        so->iter = total;
        st->inner_iter += 1;
        if (so->history) so->history[total - 1] = err;
        conv = err <= st->tau;
        stop = conv || it >= st->max_iter || total >= so->max_iter || error;
        if (error) {
            so->error = error;
            so->status = error;
            so->done = 1;
        }
    }
    st->done = stop ? 1 : 0;
    __threadfence();
    if (p.use_cond) cudaGraphSetConditional(p.cond, stop ? 0u : 1u);
}

// ------------------------------------------------------- shared memory
__host__ __device__ constexpr uint32_t a16(size_t b) { return (uint32_t)((b + 15) & ~(size_t)15); }

// Layout of the dynamic shared memory of a sweep block:
//   [staged y[0, stage)] [item buffer 0] [item buffer 1] [gathered terms]
//   [fused sweep: slot sources, new tile values] [barriers]
// and of one item buffer:
//   [descriptor int4] [indices] [offsets] [out-degrees] [1/outdeg]
//   [old stored values] [right-hand side] [edge weights]
struct Layout {
    uint32_t idx, cp, od, inv, yo, rhs, ew, buf;          // within a buffer
    uint32_t buf0, buf1, vals, sidx, fresh, bars, total;  // within the block
};

__host__ __device__ inline Layout make_layout(int idxcap, int vcap, int sa, int st, bool rhs,
                                              bool w, bool gs, int stage)
{
    Layout L;
    L.idx = 16;
    L.cp = L.idx + a16((size_t)idxcap * 4);
    L.od = L.cp + a16((size_t)vcap * 4);
    L.inv = L.od + a16((size_t)vcap * 4);
    L.yo = L.inv + a16((size_t)vcap * sa);
    L.rhs = L.yo + a16((size_t)vcap * st);
    L.ew = L.rhs + (rhs ? a16((size_t)vcap * sa) : 0);
    L.buf = L.ew + (w ? a16((size_t)idxcap * sa) : 0);
    L.buf0 = a16((size_t)stage * st);
    L.buf1 = L.buf0 + L.buf;
    L.vals = L.buf1 + L.buf;
    L.sidx = L.vals + a16((size_t)idxcap * sa);
    L.fresh = L.sidx + (gs ? a16((size_t)idxcap * 4) : 0);
    L.bars = L.fresh + (gs ? a16((size_t)vcap * st) : 0);
    L.total = L.bars + 32;  // three 8-byte barriers
    return L;
}

template <typename T, typename A, bool GS>
__host__ __device__ inline Layout layout_of(const SweepParams &p)
{
    return make_layout(p.idxcap, p.vcap, sizeof(A), sizeof(T), p.rhs != nullptr, p.ew != nullptr,
                       GS, p.stage);
}

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

// Thread 0: bulk copies of the item with descriptor d into `buf`, completing
// on `bar`.  Ranges are widened to 16-byte boundaries (the arrays are padded
// for it).
template <typename T, typename A>
__device__ __forceinline__ void issue_item(const SweepParams &p, const Layout &L, int4 d,
                                           unsigned char *buf, uint64_t *bar, const T *yin)
{
    *reinterpret_cast<int4 *>(buf) = d;
    const int v0 = d.x, v1 = d.y, ea = d.z, eb = d.w;
    // pass 0 sums the bytes announced on the barrier, pass 1 issues the copies
    uint32_t tx = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) mbar_expect_tx(bar, tx);
        auto range = [&](uint32_t off, const void *base, int elem, int lo, int hi) {
            const int al = 16 / elem;
            const int s = lo & ~(al - 1), e = (hi + al - 1) & ~(al - 1);
            if (e <= s) return;
            const uint32_t bytes = (uint32_t)(e - s) * (uint32_t)elem;
            if (pass == 0) tx += bytes;
            else bulk_load(buf + off, static_cast<const char *>(base) + (size_t)s * elem, bytes, bar);
        };
        range(L.idx, p.row_idx, 4, ea, eb);
        range(L.cp, p.col_ptr, 4, v0, v1 + 1);
        range(L.od, p.outdeg, 4, v0, v1);
        range(L.inv, p.inv, sizeof(A), v0, v1);
        range(L.yo, yin, sizeof(T), v0, v1);
        if (p.rhs) range(L.rhs, p.rhs, sizeof(A), v0, v1);
        if (p.ew) range(L.ew, p.ew, sizeof(A), ea, eb);
    }
}

// Works on one item whose streams are in `buf`.
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void do_item(const SweepParams &p, const Layout &L, int item,
                                        const unsigned char *buf, unsigned char *smem,
                                        const Src<T, GS> &src, Fin &fin)
{
    __shared__ double hub_red[SWEEP_BS / 32];
    const int4 d = *reinterpret_cast<const int4 *>(buf);
    const int v0 = d.x, v1 = d.y, ea = d.z, eb = d.w;
    const int ne = eb - ea;
    constexpr int alA = 16 / sizeof(A), alT = 16 / sizeof(T);
    const int *idx = reinterpret_cast<const int *>(buf + L.idx) - (ea & ~3);
    const int *cp = reinterpret_cast<const int *>(buf + L.cp) - (v0 & ~3);
    const int *od = reinterpret_cast<const int *>(buf + L.od) - (v0 & ~3);
    const A *inv = reinterpret_cast<const A *>(buf + L.inv) - (v0 & ~(alA - 1));
    const T *yo = reinterpret_cast<const T *>(buf + L.yo) - (v0 & ~(alT - 1));
    const A *rhs = reinterpret_cast<const A *>(buf + L.rhs) - (v0 & ~(alA - 1));
    const A *ew = reinterpret_cast<const A *>(buf + L.ew) - (ea & ~(alA - 1));
    A *vals = reinterpret_cast<A *>(smem + L.vals);
    int *sidx = reinterpret_cast<int *>(smem + L.sidx);
    T *fresh = reinterpret_cast<T *>(smem + L.fresh);
    const bool has_rhs = p.rhs != nullptr;

    // phase A: every in-edge, four independent gathers per thread per step
    for (int s0 = threadIdx.x; s0 < ne; s0 += 4 * SWEEP_BS) {
        int v[4];
        A got[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int s = s0 + c * SWEEP_BS;
            v[c] = s < ne ? idx[ea + s] : 0;
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int s = s0 + c * SWEEP_BS;
            got[c] = s < ne ? to_a<A>(src(v[c])) : A(0);
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int s = s0 + c * SWEEP_BS;
            if (s < ne) {
                vals[s] = W ? ew[ea + s] * got[c] : got[c];
                if constexpr (GS) sidx[s] = v[c];
            }
        }
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = SWEEP_BS / 32;

    if (v0 < p.nhub) {
        // hub segment: block sum, then the hub's last segment finishes it
        double s = 0;
        for (int i = threadIdx.x; i < ne; i += SWEEP_BS) s += static_cast<double>(vals[i]);
        s = warp_sum(s);
        if (lane == 0) hub_red[warp] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double tot = 0;
            for (int w = 0; w < nw; ++w) tot += hub_red[w];
            const int h = v0;
            p.seg_acc[item] = tot;
            __threadfence();
            const int s0 = p.hubseg_start[h];
            const int nseg = p.hubseg_start[h + 1] - s0;
            if (atomicAdd(&p.hub_cnt[h], 1) == nseg - 1) {
                __threadfence();
                const volatile double *sa = p.seg_acc;
                double all = 0;
                for (int j = 0; j < nseg; ++j) all += sa[s0 + j];
                p.hub_cnt[h] = 0;
                fin(h, static_cast<A>(all), od[h], inv[h], yo[h], has_rhs ? rhs[h] : fin.base());
            }
        }
        return;
    }

    // tile: first vertex with in-degree <= t_lo (degrees are non-increasing)
    int vm;
    {
        int lo = v0, hi = v1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (cp[mid + 1] - cp[mid] <= p.t_lo) hi = mid;
            else lo = mid + 1;
        }
        vm = lo;
    }
    // phase B1: in-degree > t_lo: warp per vertex
    for (int u = v0 + warp; u < vm; u += nw) {
        const int a = cp[u] - ea, e = cp[u + 1] - ea;
        A acc = 0;
        for (int i = a + lane; i < e; i += 32) acc += vals[i];
        acc = warp_sum(acc);
        if (lane == 0) {
            const T yn = fin(u, acc, od[u], inv[u], yo[u], has_rhs ? rhs[u] : fin.base());
            if constexpr (GS) fresh[u - v0] = yn;
        }
    }
    if constexpr (GS) __syncthreads();
    // phase B2: thread per vertex, in rounds of the block size
    for (int u0 = vm; u0 < v1; u0 += SWEEP_BS) {
        const int u = u0 + threadIdx.x;
        if (u < v1) {
            const int a = cp[u] - ea, e = cp[u + 1] - ea;
            A acc = 0;
            for (int i = a; i < e; ++i) {
                A val = vals[i];
                if constexpr (GS) {
                    // in-tile source already updated in this sweep: new value
                    const int v = sidx[i];
                    if (v >= v0 && v < u0) {
                        const A nv = to_a<A>(fresh[v - v0]);
                        val = W ? ew[ea + i] * nv : nv;
                    }
                }
                acc += val;
            }
            const T yn = fin(u, acc, od[u], inv[u], yo[u], has_rhs ? rhs[u] : fin.base());
            if constexpr (GS) fresh[u - v0] = yn;
        }
        if constexpr (GS) __syncthreads();
    }
}

// Persistent, double-buffered loop over the items of this block (items
// blockIdx, blockIdx + G, ... in that fixed order, so every block's partial
// sums are reproducible).  Returns false if a copy wait gave up.
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void run_items(const SweepParams &p, const T *yin, Fin &fin)
{
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const Layout L = layout_of<T, A, GS>(p);
    uint64_t *bars = reinterpret_cast<uint64_t *>(dyn_smem + L.bars);
    unsigned char *const buf0 = dyn_smem + L.buf0, *const buf1 = dyn_smem + L.buf1;
    const int nitems = p.nhubseg + p.ntiles;
    const uint32_t limit = p.wait_limit ? p.wait_limit : DEFAULT_WAIT_LIMIT;
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        mbar_init(&bars[2], 1);  // nothing ever arrives here (timeout test)
        mbar_init_fence();
    }
    // staged copy of the hottest contributions (snapshot for the fused sweep)
    if (p.stage > 0) {
        const int4 *s = reinterpret_cast<const int4 *>(yin);
        int4 *dst = reinterpret_cast<int4 *>(dyn_smem);
        const int nvec = (int)(a16((size_t)p.stage * sizeof(T)) / 16);
        for (int i = threadIdx.x; i < nvec; i += SWEEP_BS) dst[i] = GS ? __ldcg(s + i) : __ldg(s + i);
    }
    __syncthreads();
    const Src<T, GS> src{yin, reinterpret_cast<const T *>(dyn_smem), p.stage};
    // thread 0 keeps the descriptor of the item after next in a register, so
    // no descriptor load sits on an item's path
    int4 dnext = make_int4(0, 0, 0, 0);
    if (threadIdx.x == 0 && (int)blockIdx.x < nitems) {
        issue_item<T, A>(p, L, __ldg(p.desc + blockIdx.x), buf0, &bars[0], yin);
        if ((int)(blockIdx.x + gridDim.x) < nitems) dnext = __ldg(p.desc + blockIdx.x + gridDim.x);
    }
    int k = 0;
    bool timed_out = false;
    for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++k) {
        const int b = k & 1;
        const int next = item + gridDim.x;
        if (threadIdx.x == 0 && next < nitems) {
            fence_async_smem();  // generic reads of that buffer precede the copy
            issue_item<T, A>(p, L, dnext, b ? buf0 : buf1, &bars[b ^ 1], yin);
            if (next + (int)gridDim.x < nitems) dnext = __ldg(p.desc + next + gridDim.x);
        }
        bool ok = mbar_wait(&bars[b], (k >> 1) & 1, limit);
        if (p.test_stall && k == 0) ok = ok && mbar_wait(&bars[2], 0, limit);
        if (__syncthreads_or(!ok)) {
            // drain this block's copies still in flight, then report
            mbar_wait(&bars[b], (k >> 1) & 1, limit);
            if (next < nitems) mbar_wait(&bars[b ^ 1], ((k + 1) >> 1) & 1, limit);
            timed_out = true;
            break;
        }
        do_item<T, A, GS, W>(p, L, item, b ? buf1 : buf0, dyn_smem, src, fin);
        __syncthreads();  // the buffer and the gathered terms are reused
    }
    if (timed_out && threadIdx.x == 0) atomicCAS(&p.st->error, 0, (int)PR_ERR_TIMEOUT);
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
    SweepFin<T, A, GS, W> fin(p, load_ctx<A>(st), yout);
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
    SweepFin<T, A, true, false> fin(p, load_ctx<A>(st), y);
    const A *inv = static_cast<const A *>(p.inv);
    const A *rhs = static_cast<const A *>(p.rhs);
    const int lane = threadIdx.x & 31;
    for (int u = 0; u < p.n; ++u) {
        const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
        A acc = 0;
        for (int i = a + lane; i < e; i += 32) acc += to_a<A>(ld_y<T, true>(y, p.row_idx[i]));
        acc = warp_sum(acc);
        if (lane == 0)
            fin(u, acc, p.outdeg[u], inv[u], ld_y<T, true>(y, u), rhs ? rhs[u] : fin.base());
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
