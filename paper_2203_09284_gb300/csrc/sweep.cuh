// sweep.cuh -- the fused PageRank sweep.
//
// One sweep gathers the stored contribution vector through the in-lists,
// applies teleport and dangling mass, writes the new stored value, and
// accumulates the sweep's L1/max error, dangling mass and total; the block
// that finishes last turns those sums into the next sweep's scalars and the
// stop decision (Algorithm 1/2 `while error > threshold`).
//
// Everything runs in the degree-ordered numbering (in-degree descending), so
// the in-degree classes are contiguous ranges of ids:
//   hubs  [0, nhub)               in-degree > t_hub
//   mid   [nhub, nhub + nmid)     t_lo < in-degree <= t_hub
//   low   [nhub + nmid, n)        in-degree <= t_lo
// and the most-gathered contributions (in R-MAT-like graphs, the sources of
// about half of all edges) sit in the first few tens of thousands of ids.
//
// Stored vector y (one entry per vertex):
//   y_u = x~_u * inv_outdeg[u]   if u has out-edges (its contribution, the
//                                 paper's contributionList entry)
//   y_u = x~_u                    if u is dangling (never gathered), or for
//                                 weighted graphs (P is applied per in-edge)
// where the true rank is x_u = sigma * x~_u.
//
// Launch shape: one persistent block of 1024 threads per SM.  The block first
// copies y[0, stage) into shared memory with one bulk (TMA) copy completed on
// an mbarrier, so every warp of the SM reads the hottest contributions from
// shared memory; all other gathers go to L2/HBM.  Then each warp works on its
// own items with no block-wide synchronisation (items taken round-robin by
// warp, a fixed order, so the sweep's sums are reproducible):
//   hub segment  hub_seg in-edges of one hub, summed by a warp (16-byte index
//                loads, eight gathers in flight per lane); the warp finishing
//                a hub's last segment adds the segment sums in order and
//                updates the hub
//   mid group    32/G consecutive mid vertices, G lanes per vertex (G = 32,
//                16, 8 or 4 as the in-degree falls: more than mid_wide,
//                mid_wide/2, mid_wide/4, else; by default 1024, 512, 256),
//                same streaming gather, then a G-lane reduction
//   low tile     consecutive low-degree vertices with at most `tile` units of
//                work: the warp gathers all their in-edges into its slice of
//                shared memory, then one lane per vertex adds its own
// The per-vertex epilogue is a functor, so the same traversal serves the
// PageRank sweep, the correction sweep and the FP64 residual sweep of the
// defect-correction forms.
//
// Jacobi (Algorithm 1, Eq. 2): reads y[iter & 1], writes the other buffer.
// Fused (Algorithm 2, Eq. 9): one buffer updated in place, so a vertex sees
// whichever contribution is there (new if its in-neighbour was already
// updated in this sweep and the store has reached the load's cache level).
// The hottest vertices (hubs and the mid vertices with more than 128
// in-edges) are updated by a first launch, so the second launch's
// shared-memory copy and loads already see their new values; a low tile's
// in-edges are all gathered before any of its vertices is updated.  After
// each fused sweep the iterate is rescaled to sum 1 by folding 1/sum into
// sigma (unless the solve asks for the literal Algorithm 2).
// Perforated Jacobi (loop perforation): the epilogue functor decides per
// vertex whether it keeps its value; a kept vertex's in-edges are not
// gathered (low tiles mark their slots in a per-warp bit mask).
#pragma once

#include <type_traits>

#include "common.cuh"
#include "tma.cuh"

namespace fpr {

// One 1024-thread block per SM: 64 registers a thread fill the register file
// (smaller blocks at 2-6 per SM with fewer registers measured slower).
constexpr int SWEEP_BS = 1024;  // threads per sweep block
constexpr int SWEEP_MINB = 1;   // resident sweep blocks per SM
constexpr int SWEEP_WARPS = SWEEP_BS / 32;
constexpr uint32_t DEFAULT_WAIT_LIMIT = 1u << 22;


struct SweepParams {
    int32_t n;
    const int32_t *__restrict__ col_ptr;  // relabelled in-lists (padded)
    const int32_t *__restrict__ row_idx;
    const int32_t *__restrict__ outdeg;
    const void *inv;              // A[n]: 1/outdeg in the arithmetic type
    const void *ew;               // A[m]: P per in-list slot (weighted) or null
    int32_t nhub;                 // hubs are [0, nhub)
    const int4 *desc;             // [nhubseg + mi[4] + nlt] item descriptors, in
                                  // item order: hub segments {hub, 0, ea, eb},
                                  // mid groups and low tiles {v0, v1, ea, eb}
                                  // (vertices [v0, v1), in-list slots [ea, eb))
    int32_t nhubseg;
    const int32_t *hubseg_start;  // [nhub + 1]
    double *seg_acc;              // [nhubseg]
    int32_t *hub_cnt;             // [nhub]
    int32_t mi[5];                // mid items before sub-range k (32 >> k lanes
                                  // per vertex; mi[4]: all mid items)
    int32_t nlt;
    int32_t lcap;                 // per-warp slots for a low tile's in-edges
    int32_t stage;                // y[0, stage) is copied to shared memory
    int32_t item_lo, item_hi;     // this launch's items [item_lo, item_hi)
    int32_t write_alt;            // fused sweep: write the new values to y1, not y0
    int32_t close;                // this launch closes the sweep
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
    int32_t shift;                // correction sweep: restore the exact sum of e
    void *last;                   // perforated sweep: A[n] last change per vertex
};

// Loads of the stored vector.  Jacobi: read-only path (the kernel never
// writes the buffer it gathers from).  Fused: plain loads, cached in L1 (the
// buffer is updated in place by other warps; a load returns the value before
// or after a concurrent update, both of which the fused sweep allows).
// ld_l2 reads from L2, where a value this warp stored earlier in the sweep
// (st_y, also through L2) is visible after a __syncwarp.
template <typename T, bool GS>
__device__ __forceinline__ T ld_y(const T *p, int i)
{
    if constexpr (GS) return p[i];
    else return __ldg(p + i);
}

template <typename T>
__device__ __forceinline__ T ld_l2(const T *p, int i) { return __ldcg(p + i); }

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
    return __ushort_as_bfloat16(reinterpret_cast<const unsigned short *>(p)[i]);
}
template <>
__device__ __forceinline__ __nv_bfloat16 ld_y<__nv_bfloat16, false>(const __nv_bfloat16 *p, int i)
{
    return __ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __half ld_y<__half, true>(const __half *p, int i)
{
    return __ushort_as_half(reinterpret_cast<const unsigned short *>(p)[i]);
}
template <>
__device__ __forceinline__ __half ld_y<__half, false>(const __half *p, int i)
{
    return __ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __nv_bfloat16 ld_l2<__nv_bfloat16>(const __nv_bfloat16 *p, int i)
{
    return __ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short *>(p) + i));
}
template <>
__device__ __forceinline__ __half ld_l2<__half>(const __half *p, int i)
{
    return __ushort_as_half(__ldcg(reinterpret_cast<const unsigned short *>(p) + i));
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

// Cache policy of the index stream: each in-list slot is read once per
// sweep, so it is kept out of L1 and leaves L2 first (the gathered vector,
// reused, stays).
__device__ __forceinline__ uint64_t policy_stream()
{
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ int4 ld_idx4(const int32_t *p, uint64_t pol)
{
    int4 r;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p), "l"(pol));
    return r;
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
    A ds;       // d * sigma: weight of a gathered sum (stored units)
    A cst;      // d * sigma * dt: the dangling term every vertex receives
    A bc;       // base + cst: a new value's constant part without a rhs
    bool linf;  // the stop rule takes the largest change
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
    const double cst = st->d * st->sigma * (st->dang * st->inv_n);
    c.ds = static_cast<A>(st->d * st->sigma);
    c.cst = static_cast<A>(cst);
    c.bc = static_cast<A>(st->base + cst);
    c.linf = st->norm != 0;
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
    // constant part of vertex u's new value (true units): the teleport term
    // or the right-hand side, plus the dangling term
    __device__ __forceinline__ A rterm(const SweepParams &q, int u) const
    {
        return q.rhs ? static_cast<const A *>(q.rhs)[u] + c.cst : c.bc;
    }
    // r = rterm(u); new value x' = r + d sigma (acc + dt), acc in stored units
    __device__ __forceinline__ T operator()(int u, A acc, int od, A inv, T yold, A r)
    {
        const A yo = to_a<A>(yold);
        const A xold = (W || od == 0) ? yo : yo * static_cast<A>(od);  // stored units
        const A xnew = fma(c.ds, acc, r);                                // true units
        const A diff = aabs(xnew - c.sig * xold);
        const A xs = xnew * c.rsig;                                       // stored units
        const T yn = from_a<T>((W || od == 0) ? xs : xs * inv);
        st_y<T, GS>(yout, u, yn);
        pt.l1 += diff;
        if (c.linf) pt.lmax = diff > pt.lmax ? diff : pt.lmax;
        pt.sm += xs;
        if (od == 0) pt.dm += xs;
        return yn;
    }
};

// Perforated Jacobi sweep: a vertex whose change at its last computation was
// below eps times its value keeps the value in a perforated sweep (keep():
// no gather; its stored value is carried to the output buffer); computed
// vertices record their change.  The first sweep and every period-th are
// full (st->perf_period).
template <typename F, typename = void>
struct perf_of : std::false_type {};
template <typename F>
struct perf_of<F, std::void_t<decltype(F::PERF)>> : std::bool_constant<F::PERF> {};

template <typename T, typename A>
struct SweepFinPerf : SweepFin<T, A, false, false> {
    static constexpr bool PERF = true;
    A *last;        // [n] change at the last computation (true units)
    A eps;
    bool full;
    unsigned long long gath = 0;  // in-list entries this thread summed
    __device__ SweepFinPerf(const SweepParams &p_, const Ctx<A> &c_, T *yo, A *last_, A eps_,
                            bool full_)
        : SweepFin<T, A, false, false>(p_, c_, yo), last(last_), eps(eps_), full(full_) {}
    __device__ __forceinline__ bool skip(int u, int od, T yold) const
    {
        if (full) return false;
        const A yo = to_a<A>(yold);
        const A x = this->c.sig * (od == 0 ? yo : yo * static_cast<A>(od));
        return last[u] < eps * x;
    }
    __device__ __forceinline__ T operator()(int u, A acc, int od, A inv, T yold, A r)
    {
        const A yo = to_a<A>(yold);
        const A xold = od == 0 ? yo : yo * static_cast<A>(od);
        const A xnew = fma(this->c.ds, acc, r);
        const A diff = aabs(xnew - this->c.sig * xold);
        const A xs = xnew * this->c.rsig;
        const T yn = from_a<T>(od == 0 ? xs : xs * inv);
        this->yout[u] = yn;
        last[u] = diff;
        this->pt.l1 += diff;
        if (this->c.linf) this->pt.lmax = diff > this->pt.lmax ? diff : this->pt.lmax;
        this->pt.sm += xs;
        if (od == 0) this->pt.dm += xs;
        return yn;
    }
    __device__ __forceinline__ void keep(int u, int od, T yold)
    {
        const A yo = to_a<A>(yold);
        const A xs = od == 0 ? yo : yo * static_cast<A>(od);
        this->yout[u] = yold;
        this->pt.sm += xs;
        if (od == 0) this->pt.dm += xs;
    }
};

// Reduces the block's partial sums and adds them to the sweep accumulators.
template <typename A>
__device__ __forceinline__ void block_partials(SolveState *st, const Part<A> &pt)
{
    __shared__ double red[4][32];
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

// Reads and clears the sweep accumulators and the block ticket.  Called by
// all 32 lanes of one warp: lane k takes slot k (one round trip for all
// slots, through L2 where the atomics landed) and every lane gets the
// totals.  The words are integers, so the tree of adds gives the same totals
// as any other order.
__device__ __forceinline__ void take_sums(SolveState *st, double &res, double &resmax,
                                          double &dang, double &sum)
{
    static_assert(ACC_SLOTS == 32, "one accumulator slot per lane");
    __threadfence();
    const int lane = threadIdx.x & 31;
    longlong2 *slot = reinterpret_cast<longlong2 *>(&st->acc[lane]);
    const longlong2 r = __ldcg(slot), dd = __ldcg(slot + 1), s = __ldcg(slot + 2),
                    m = __ldcg(slot + 3);
    const longlong2 zero = make_longlong2(0, 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) __stcg(slot + k, zero);
    long long rh = r.x, rl = r.y, dh = dd.x, dl = dd.y, sh = s.x, sl = s.y;
    unsigned long long mx = static_cast<unsigned long long>(m.x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        rh += __shfl_xor_sync(FULL, rh, o);
        rl += __shfl_xor_sync(FULL, rl, o);
        dh += __shfl_xor_sync(FULL, dh, o);
        dl += __shfl_xor_sync(FULL, dl, o);
        sh += __shfl_xor_sync(FULL, sh, o);
        sl += __shfl_xor_sync(FULL, sl, o);
        const unsigned long long m2 = __shfl_xor_sync(FULL, mx, o);
        mx = m2 > mx ? m2 : mx;
    }
    res = fx_value(rh, rl);
    resmax = __longlong_as_double(static_cast<long long>(mx));
    dang = fx_value(dh, dl);
    sum = fx_value(sh, sl);
    if (lane == 0) st->ticket = 0;
}

// Closes a PageRank sweep (dc == 0) or a correction sweep (dc != 0): next
// scalars, history, stop test, loop condition.  A device-side error ends the
// loop with that status.  Called by all lanes of one warp (take_sums); lane
// 0 does the rest.
__device__ __forceinline__ void close_sweep(const SweepParams &p)
{
    SolveState *st = p.st;
    double res, resmax, dang, sum;
    take_sums(st, res, resmax, dang, sum);
    if (threadIdx.x & 31) return;
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
        // a perforated solve with a period stops only after a full sweep
        if (st->perf && st->perf_period > 0) conv = conv && ((it - 1) % st->perf_period == 0);
        stop = conv || it >= st->max_iter || error;
        st->status = error ? error : (conv ? PR_OK : PR_NOT_CONVERGED);
    } else {
        SolveState *so = p.st_outer;
        const int total = so->iter + 1;
        so->iter = total;
        st->inner_iter += 1;
        if (so->history) so->history[total - 1] = err;
        conv = err <= st->tau;
        // an inner solve whose change stops falling has reached the
        // correction's storage precision: hand over to the FP64 step
        if (err < st->best) {
            st->best = err;
            st->since = 0;
        } else {
            st->since += 1;
        }
        const bool stalled = st->since >= 8;
        stop = conv || stalled || it >= st->max_iter || total >= so->max_iter || error;
        if (p.shift) {
            // e <- e + beta x with sum(e) = mass_target afterwards; in stored
            // units e~ += gamma Y64 (the shift kernel applies it), so the
            // dangling mass and sum of e~ move by gamma times those of x~
            const double beta = (st->mass_target - st->sigma * sum) / (so->sigma * so->sum);
            const double gam = beta * so->sigma / st->sigma;
            st->shift = gam;
            st->dang = dang + gam * so->dang;
            st->sum = sum + gam * so->sum;
        }
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

// Dynamic shared memory of a sweep block:
//   [staged y[0, stage)] [barriers] [32 warp slices]
// and of one warp slice: [gathered terms, lcap] [perforated sweeps: one bit
// per term, set for the in-edges of vertices that keep their value].
struct Layout {
    uint32_t bars, warps, wmask, wbytes, total;
};

__host__ __device__ inline Layout make_layout(int lcap, int sa, int st, bool perf, int stage)
{
    Layout L;
    L.bars = a16((size_t)stage * st);
    L.warps = L.bars + 32;
    L.wmask = a16((size_t)lcap * sa);
    L.wbytes = L.wmask + (perf ? a16((size_t)((lcap + 31) / 32) * 4) : 0);
    L.total = L.warps + SWEEP_WARPS * L.wbytes;
    return L;
}

template <typename T, typename A, bool PERF>
__host__ __device__ inline Layout layout_of(const SweepParams &p)
{
    return make_layout(p.lcap, sizeof(A), sizeof(T), PERF, p.stage);
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

// This lane's share of the sum over in-list slots [a, e) when G lanes (gl =
// lane index among them) stream one list: 16-byte index loads, two of them
// (eight gathers) in flight per lane.
template <int G, typename T, typename A, bool GS, bool W>
__device__ __forceinline__ A group_stream(const SweepParams &p, const Src<T, GS> &src, int a,
                                          int e, int gl)
{
    A acc = 0;
    const A *ew = static_cast<const A *>(p.ew);
    const uint64_t pol = policy_stream();
    // the next step's indices are loaded while this step's gathers are in
    // flight, so a long in-list costs one round trip per step, not two
    const int4 zero = make_int4(0, 0, 0, 0);
    int j0 = (a & ~3) + 4 * gl;
    int4 q0 = j0 < e ? ld_idx4(p.row_idx + j0, pol) : zero;
    int4 q1 = j0 + 4 * G < e ? ld_idx4(p.row_idx + j0 + 4 * G, pol) : zero;
    for (; j0 < e; j0 += 8 * G) {
        const int j1 = j0 + 4 * G;
        const int n0 = j0 + 8 * G, n1 = n0 + 4 * G;
        const int4 r0 = n0 < e ? ld_idx4(p.row_idx + n0, pol) : zero;
        const int4 r1 = n1 < e ? ld_idx4(p.row_idx + n1, pol) : zero;
        const int v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        A got[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int s = (c < 4 ? j0 : j1) + (c & 3);
            got[c] = (s >= a && s < e) ? to_a<A>(src(v[c])) : A(0);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int s = (c < 4 ? j0 : j1) + (c & 3);
            if constexpr (W) got[c] = (s >= a && s < e) ? ew[s] * got[c] : A(0);
            acc += got[c];
        }
        q0 = r0;
        q1 = r1;
    }
    return acc;
}

template <int G, typename A>
__device__ __forceinline__ A group_sum(A v)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// hub segment i (one warp)
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void hub_item(const SweepParams &p, int i, const int4 &d,
                                         const Src<T, GS> &src, Fin &fin, int lane)
{
    const int h = d.x;
    bool sk = false;
    if constexpr (perf_of<Fin>::value) sk = fin.skip(h, __ldg(p.outdeg + h), ld_y<T, GS>(src.y, h));
    A acc = sk ? A(0) : group_stream<32, T, A, GS, W>(p, src, d.z, d.w, lane);
    const double s = warp_sum(static_cast<double>(acc));
    if (lane == 0) {
        if constexpr (perf_of<Fin>::value) {
            if (!sk) fin.gath += (unsigned long long)(d.w - d.z);
        }
        p.seg_acc[i] = s;
        __threadfence();
        const int s0 = p.hubseg_start[h];
        const int nseg = p.hubseg_start[h + 1] - s0;
        if (atomicAdd(&p.hub_cnt[h], 1) == nseg - 1) {
            __threadfence();
            const volatile double *sa = p.seg_acc;
            double all = 0;
            for (int j = 0; j < nseg; ++j) all += sa[s0 + j];
            p.hub_cnt[h] = 0;
            if (sk) {
                if constexpr (perf_of<Fin>::value) fin.keep(h, p.outdeg[h], ld_y<T, GS>(src.y, h));
            } else {
                fin(h, static_cast<A>(all), p.outdeg[h], static_cast<const A *>(p.inv)[h],
                    ld_y<T, GS>(src.y, h), fin.rterm(p, h));
            }
        }
    }
}

// mid vertices [v0, min(v0 + 32 / G, v_end)): G lanes per vertex
template <int G, typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void mid_group(const SweepParams &p, int v0, int v_end,
                                          const Src<T, GS> &src, Fin &fin, int lane)
{
    const int gl = lane & (G - 1);
    const int u = v0 + lane / G;
    const bool act = u < v_end;
    int a = 0, e = 0, od = 0;
    A inv = 0, r = 0;
    T yo{};
    if (act) {
        a = __ldg(p.col_ptr + u);
        e = __ldg(p.col_ptr + u + 1);
        if (gl == 0) {  // the epilogue's inputs, issued before the gathers
            od = __ldg(p.outdeg + u);
            inv = __ldg(static_cast<const A *>(p.inv) + u);
            yo = ld_y<T, GS>(src.y, u);
            r = fin.rterm(p, u);
        }
    }
    bool sk = false;
    if constexpr (perf_of<Fin>::value) {
        // the group's first lane decides; a kept vertex gathers nothing
        sk = __shfl_sync(FULL, (act && gl == 0) ? fin.skip(u, od, yo) : false, lane & ~(G - 1));
        if (sk) e = a;
        if (act && gl == 0 && !sk) fin.gath += (unsigned long long)(e - a);
    }
    A acc = group_stream<G, T, A, GS, W>(p, src, a, e, gl);
    acc = group_sum<G>(acc);
    if (act && gl == 0) {
        if (sk) {
            if constexpr (perf_of<Fin>::value) fin.keep(u, od, yo);
        } else {
            fin(u, acc, od, inv, yo, r);
        }
    }
}

// low tile k (one warp): in-edges gathered into the warp's shared slice,
// then one lane per vertex
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void low_item(const SweepParams &p, const int4 &d,
                                         const Src<T, GS> &src, Fin &fin, int lane,
                                         unsigned char *slice, const Layout &L)
{
    const int v0 = d.x, v1 = d.y, ea = d.z, eb = d.w;
    constexpr bool PF = perf_of<Fin>::value;
    if (!PF && ea == eb) {
        // a tile of vertices without in-edges (the tail of the degree-ordered
        // ids): nothing to gather and no offsets to read; two rounds of
        // vertex inputs in flight at a time
        for (int u0 = v0; u0 < v1; u0 += 64) {
            const int ua = u0 + lane, ub = ua + 32;
            int oda = 0, odb = 0;
            A inva = 0, invb = 0, ra = 0, rb = 0;
            T ya{}, yb{};
            if (ua < v1) {
                oda = __ldg(p.outdeg + ua);
                inva = __ldg(static_cast<const A *>(p.inv) + ua);
                ya = ld_y<T, GS>(src.y, ua);
                ra = fin.rterm(p, ua);
            }
            if (ub < v1) {
                odb = __ldg(p.outdeg + ub);
                invb = __ldg(static_cast<const A *>(p.inv) + ub);
                yb = ld_y<T, GS>(src.y, ub);
                rb = fin.rterm(p, ub);
            }
            if (ua < v1) fin(ua, A(0), oda, inva, ya, ra);
            if (ub < v1) fin(ub, A(0), odb, invb, yb, rb);
        }
        return;
    }
    A *vals = reinterpret_cast<A *>(slice);
    uint32_t *mask = reinterpret_cast<uint32_t *>(slice + L.wmask);
    const A *ew = static_cast<const A *>(p.ew);
    // inputs of this lane's first vertex, issued before the gathers
    int u = v0 + lane;
    int a0 = 0, e0 = 0, od0 = 0;
    A inv0 = 0, r0 = 0;
    T yo0{};
    if (u < v1) {
        a0 = __ldg(p.col_ptr + u);
        e0 = __ldg(p.col_ptr + u + 1);
        od0 = __ldg(p.outdeg + u);
        inv0 = __ldg(static_cast<const A *>(p.inv) + u);
        yo0 = ld_y<T, GS>(src.y, u);
        r0 = fin.rterm(p, u);
    }
    if constexpr (PF) {
        // slots of the vertices that keep their value: one bit each (a low
        // vertex has at most 32 in-edges, so its run spans at most 2 words)
        for (int w = lane; w < ((eb - ea + 31) >> 5); w += 32) mask[w] = 0;
        __syncwarp();
        for (int u0 = v0; u0 < v1; u0 += 32) {
            const int uu = u0 + lane;
            if (uu < v1) {
                int a = a0, e = e0;
                bool sk;
                if (u0 == v0) {
                    sk = fin.skip(uu, od0, yo0);
                } else {
                    a = __ldg(p.col_ptr + uu);
                    e = __ldg(p.col_ptr + uu + 1);
                    sk = fin.skip(uu, __ldg(p.outdeg + uu), ld_y<T, GS>(src.y, uu));
                }
                if (sk && e > a) {
                    const int lo = a - ea, hi = e - ea, len = hi - lo;
                    const uint32_t run = len >= 32 ? ~0u : ((1u << len) - 1u);
                    atomicOr(&mask[lo >> 5], run << (lo & 31));
                    if (((hi - 1) >> 5) != (lo >> 5)) {
                        const int rem = hi - ((hi - 1) >> 5) * 32;
                        atomicOr(&mask[(hi - 1) >> 5], rem >= 32 ? ~0u : ((1u << rem) - 1u));
                    }
                }
            }
        }
        __syncwarp();
    }
    // gathers: eight slots per lane in flight
    const uint64_t pol = policy_stream();
    for (int j0 = (ea & ~3) + 4 * lane; j0 < eb; j0 += 256) {
        const int j1 = j0 + 128;
        const int4 q0 = ld_idx4(p.row_idx + j0, pol);
        const int4 q1 = j1 < eb ? ld_idx4(p.row_idx + j1, pol) : make_int4(0, 0, 0, 0);
        const int v[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
        A got[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int s = (c < 4 ? j0 : j1) + (c & 3);
            bool take = s >= ea && s < eb;
            if constexpr (PF) take = take && !((mask[(s - ea) >> 5] >> ((s - ea) & 31)) & 1u);
            got[c] = take ? to_a<A>(src(v[c])) : A(0);
        }
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int s = (c < 4 ? j0 : j1) + (c & 3);
            if (s >= ea && s < eb) {
                vals[s - ea] = W ? ew[s] * got[c] : got[c];
            }
        }
    }
    __syncwarp();
    for (int u0 = v0; u0 < v1; u0 += 32) {
        u = u0 + lane;
        if (u < v1) {
            int a, e, od;
            A inv, r;
            T yo;
            if (u0 == v0) {
                a = a0, e = e0, od = od0, inv = inv0, r = r0, yo = yo0;
            } else {
                a = __ldg(p.col_ptr + u);
                e = __ldg(p.col_ptr + u + 1);
                od = __ldg(p.outdeg + u);
                inv = __ldg(static_cast<const A *>(p.inv) + u);
                yo = ld_y<T, GS>(src.y, u);
                r = fin.rterm(p, u);
            }
            bool kept = false;
            if constexpr (PF) {
                kept = fin.skip(u, od, yo);
                if (kept) fin.keep(u, od, yo);
                else fin.gath += (unsigned long long)(e - a);
            }
            if (!kept) {
                A acc = 0;
                for (int i = a - ea; i < e - ea; ++i) acc += vals[i];
                fin(u, acc, od, inv, yo, r);
            }
        }
        __syncwarp();
    }
}

// mid item j (vertices [d.x, d.y) of one sub-range)
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void mid_item(const SweepParams &p, int j, const int4 &d,
                                         const Src<T, GS> &src, Fin &fin, int lane)
{
    if (j < p.mi[1]) mid_group<32, T, A, GS, W>(p, d.x, d.y, src, fin, lane);
    else if (j < p.mi[2]) mid_group<16, T, A, GS, W>(p, d.x, d.y, src, fin, lane);
    else if (j < p.mi[3]) mid_group<8, T, A, GS, W>(p, d.x, d.y, src, fin, lane);
    else mid_group<4, T, A, GS, W>(p, d.x, d.y, src, fin, lane);
}

// The persistent sweep body: staging, then this warp's share of the launch's
// items [item_lo, item_hi) (in item order: hub segments, mid groups, low
// tiles), taken round-robin by global warp index.  If a bounded wait gives
// up, the error is recorded in the state and the block skips its items.
template <typename T, typename A, bool GS, bool W, typename Fin>
__device__ __forceinline__ void run_items(const SweepParams &p, const T *yin, Fin &fin)
{
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    const Layout L = layout_of<T, A, perf_of<Fin>::value>(p);
    uint64_t *bars = reinterpret_cast<uint64_t *>(dyn_smem + L.bars);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t limit = p.wait_limit ? p.wait_limit : DEFAULT_WAIT_LIMIT;
    // staged copy of the hottest contributions: one bulk copy (a snapshot,
    // for the fused sweep)
    const uint32_t sbytes = a16((size_t)p.stage * sizeof(T));
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);  // nothing ever arrives here (timeout test)
        mbar_init_fence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bars[0], sbytes);
        if (sbytes) bulk_load(dyn_smem, yin, sbytes, &bars[0]);
    }
    bool ok = mbar_wait(&bars[0], 0, limit);
    if (p.test_stall) ok = ok && mbar_wait(&bars[1], 0, limit);
    if (__syncthreads_or(!ok)) {
        mbar_wait(&bars[0], 0, limit);  // drain the copy before leaving
        if (threadIdx.x == 0) atomicCAS(&p.st->error, 0, (int)PR_ERR_TIMEOUT);
        return;
    }
    const Src<T, GS> src{yin, reinterpret_cast<const T *>(dyn_smem), p.stage};
    unsigned char *slice = dyn_smem + L.warps + warp * L.wbytes;
    // global warp index, blocks interleaved: neighbouring positions of a
    // round (items of like cost) go to different SMs, so that no SM holds a
    // run of the dearest items
    const int gw = warp * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * SWEEP_WARPS;
    const int nh = p.nhubseg, nm = p.mi[4];
    const int first = p.item_lo;
    const int total = p.item_hi - p.item_lo;
    // round r gives warp gw item r*nw + gw (r even) or r*nw + nw-1-gw (r odd):
    // the items' cost falls within each class, and alternating the direction
    // keeps any warp from always taking the dearest item of a round
    auto item_at = [&](int r) { return r * nw + ((r & 1) ? nw - 1 - gw : gw); };
    // descriptors are loaded two items ahead
    const int4 none = make_int4(0, 0, 0, 0);
    int4 dcur = item_at(0) < total ? __ldg(p.desc + first + item_at(0)) : none;
    int4 dnext = item_at(1) < total ? __ldg(p.desc + first + item_at(1)) : none;
    for (int r = 0;; ++r) {
        const int i = item_at(r);
        if (i >= total) break;
        const int i2 = item_at(r + 2);
        const int4 dnext2 = i2 < total ? __ldg(p.desc + first + i2) : none;
        const int k = first + i;
        if (k < nh) hub_item<T, A, GS, W>(p, k, dcur, src, fin, lane);
        else if (k < nh + nm) mid_item<T, A, GS, W>(p, k - nh, dcur, src, fin, lane);
        else low_item<T, A, GS, W>(p, dcur, src, fin, lane, slice, L);
        dcur = dnext;
        dnext = dnext2;
    }
}

template <typename T, typename A, bool GS, bool W>
__global__ void __launch_bounds__(SWEEP_BS, SWEEP_MINB) k_sweep(SweepParams p)
{
    SolveState *st = p.st;
    if (st->done) {
        if (p.close && p.use_cond && blockIdx.x == 0 && threadIdx.x == 0)
            cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    const int iter = st->iter;
    const T *yin;
    T *yout;
    if constexpr (GS) {
        yin = static_cast<const T *>(p.y0);
        yout = static_cast<T *>(p.write_alt ? p.y1 : p.y0);
    } else {
        yin = static_cast<const T *>((iter & 1) ? p.y1 : p.y0);
        yout = static_cast<T *>((iter & 1) ? p.y0 : p.y1);
    }
    SweepFin<T, A, GS, W> fin(p, load_ctx<A>(st), yout);
    run_items<T, A, GS, W>(p, yin, fin);
    block_partials<A>(st, fin.pt);
    if (p.close && last_block(st) && threadIdx.x < 32) close_sweep(p);
}

// Perforated Jacobi sweep (one launch per sweep).  The counts of gathered
// in-list entries are added to st->gathered.
template <typename T, typename A>
__global__ void __launch_bounds__(SWEEP_BS, SWEEP_MINB) k_sweep_perf(SweepParams p)
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
    const bool full = iter == 0 || (st->perf_period > 0 && iter % st->perf_period == 0);
    SweepFinPerf<T, A> fin(p, load_ctx<A>(st), yout, static_cast<A *>(p.last),
                           static_cast<A>(st->perf_eps), full);
    run_items<T, A, false, false>(p, yin, fin);
    unsigned long long g = fin.gath;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(FULL, g, o);
    if ((threadIdx.x & 31) == 0 && g) atomicAdd(&st->gathered, g);
    block_partials<A>(st, fin.pt);
    if (p.close && last_block(st) && threadIdx.x < 32) close_sweep(p);
}

// Between the two launches of a fused sweep: the first launch's vertices
// [0, n) wrote their new values to y1 (so that launch gathered from an array
// nobody was writing); they join y0 here, before the second launch reads
// them.  Nothing to do once the solve has stopped.
template <typename T>
__global__ void k_copy_front(const SolveState *st, const T *__restrict__ src, T *__restrict__ dst,
                             int32_t n)
{
    if (st->done) return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = src[i];
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
    const int lane = threadIdx.x & 31;
    for (int u = 0; u < p.n; ++u) {
        const int a = p.col_ptr[u], e = p.col_ptr[u + 1];
        A acc = 0;
        for (int i = a + lane; i < e; i += 32) acc += to_a<A>(ld_l2<T>(y, p.row_idx[i]));
        acc = warp_sum(acc);
        if (lane == 0) fin(u, acc, p.outdeg[u], inv[u], ld_l2<T>(y, u), fin.rterm(p, u));
        __syncwarp();
    }
    block_partials<A>(st, fin.pt);
    if (last_block(st) && threadIdx.x < 32) close_sweep(p);
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
    if (last_block(st) && threadIdx.x < 32) {
        double res, resmax, dang, sum;
        take_sums(st, res, resmax, dang, sum);
        if (threadIdx.x != 0) return;
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
