// batched.cu -- personalised PageRank for many teleport vectors at once (a
// multi-right-hand-side sweep).
//
// Column b of X (n x B, vertex-major) teleports to the single vertex s_b and
// sends its dangling mass there too (Eq. 1 with the uniform teleport 1/n
// replaced by the unit vector of s_b):
//   x'_b(u) = d * sum_{v in in(u)} P_vu x_b(v) + [u == s_b] ((1-d) + d D_b),
//   D_b     = sum_{v dangling} x_b(v),
// or, with dense teleport vectors V (column b sums to 1), along V:
//   x'_b(u) = d * sum_{v in in(u)} P_vu x_b(v) + V_b(u) ((1-d) + d D_b).
// The sweep is Jacobi (Algorithm 1 applied to every column) in FP32 or FP64
// (rows and sums in that type).  A column stops after the sweep whose L1
// change is <= threshold and keeps that iterate (later sweeps copy it
// unchanged); an FP32 column whose change has not fallen below its smallest
// value for STALL_SWEEPS sweeps has reached its rounding floor and stops as
// not converged.  The loop ends once every column has stopped or after
// max_iter sweeps.
//
// Layout: X rows of Bp = 32, 64, 128 or 256 elements (B is padded; wider
// batches run as several passes of at most 256 FP32 or 128 FP64 columns).
// A pass whose running columns have fallen to Bp/2 + Bp/8 hands them on to
// narrower passes (Bp/2 and 32 columns), since a sweep costs what its row
// width does.
// One warp owns a vertex row: lane l holds the columns l*w + k of every
// 32*w-wide chunk (w = elements per 16-byte access), so each gathered row is
// one contiguous, fully used read of 128 to 1024 bytes.  Rows are gathered
// in the degree-ordered ids.  Vertices with more than BATCH_SEG in-edges are
// split into segments; the warp that finishes a vertex's last segment adds
// the partial rows in segment order.  Per-column sums (L1 change, dangling
// mass) are kept per warp in shared memory, added over the warps in a fixed
// order and accumulated in exact fixed point, so the result does not depend
// on timing.
#include <string.h>

#include <algorithm>

#include "solve_impl.cuh"

namespace fpr {

constexpr int BATCH_BS = 1024;
constexpr int BATCH_WARPS = BATCH_BS / 32;
constexpr int BATCH_SEG = 256;   // in-edges per segment of a split vertex
constexpr int BATCH_COLS = 256;  // per-column state entries (largest pass)
constexpr int STALL_SWEEPS = 16; // FP32: sweeps without a new smallest change

struct BatchState {
    unsigned int ticket;
    int iter;
    int done;
    int max_iter;
    int error;
    int ncols;  // real columns of this pass
    double tau, d;
    int paused;  // the loop ended early to split the pass (done is set too)
};

struct BatchParams {
    int32_t n;
    const int32_t *__restrict__ col_ptr;
    const int32_t *__restrict__ row_idx;
    const int32_t *__restrict__ outdeg;
    const void *inv;          // E[n] 1/outdeg per source (unweighted graphs)
    const void *ew;           // E[m] P per in-list slot (weighted graphs) or null
    int32_t nhub;             // vertices [0, nhub) are split into segments
    const int4 *sdesc;        // [nseg] {vertex, its first segment, a, e}
    int32_t nseg;
    const int32_t *seg_start; // [nhub + 1]
    int32_t *seg_cnt;         // [nhub] segments finished in this sweep
    void *part;               // E[nseg][Bp] partial rows
    void *x0, *x1;            // E[n][Bp] iterates
    long long *acc;           // [Bp][4] L1 change hi/lo, dangling mass hi/lo
    double *dang;             // [Bp] dangling mass of the current iterate
    double *err;              // [Bp] last L1 change of an active column
    int32_t *conv;            // [Bp] sweep after which the column stopped
                              // (0: active, -1: padding)
    int32_t *seed;            // [Bp] seed in the degree-ordered ids (-1: padding)
    double *best;             // [Bp] smallest L1 change so far
    int32_t *since;           // [Bp] sweeps since the smallest change
    int32_t stall;            // stop columns at their rounding floor (FP32)
    const void *tele_rows;    // E[n][Bp] dense teleport rows (degree-ordered ids)
                              // or null: one-hot seeds
    int32_t pause_at;         // end the loop early (paused) once at most this
                              // many columns are still running (-1: never)
    BatchState *st;
    cudaGraphConditionalHandle cond;
    int32_t use_cond;
};

// 16-byte (or narrower) vector of W elements of E.
template <typename E, int W> struct Vec;
template <> struct Vec<float, 4> { using type = float4; };
template <> struct Vec<float, 2> { using type = float2; };
template <> struct Vec<float, 1> { using type = float; };
template <> struct Vec<double, 2> { using type = double2; };
template <> struct Vec<double, 1> { using type = double; };

template <typename V, typename E>
__device__ __forceinline__ void unpack(const V &v, E *r)
{
    if constexpr (sizeof(V) == sizeof(E)) {
        r[0] = v;
    } else if constexpr (sizeof(V) == 2 * sizeof(E)) {
        r[0] = v.x;
        r[1] = v.y;
    } else {
        r[0] = v.x;
        r[1] = v.y;
        r[2] = v.z;
        r[3] = v.w;
    }
}
template <typename V, typename E>
__device__ __forceinline__ V pack(const E *r)
{
    V v;
    if constexpr (sizeof(V) == sizeof(E)) {
        v = r[0];
    } else if constexpr (sizeof(V) == 2 * sizeof(E)) {
        v.x = r[0];
        v.y = r[1];
    } else {
        v.x = r[0];
        v.y = r[1];
        v.z = r[2];
        v.w = r[3];
    }
    return v;
}

// Row access for VEC columns of type E per lane.
template <typename E, int VEC>
struct RowIO {
    static constexpr int WMAX = 16 / (int)sizeof(E);
    static constexpr int WV = VEC < WMAX ? VEC : WMAX;  // elements per access
    static constexpr int NCH = VEC / WV;               // chunks of 32 * WV columns
    static constexpr int BP = 32 * VEC;
    using V = typename Vec<E, WV>::type;
    __device__ static __forceinline__ int col(int lane, int k)
    {
        return (k / WV) * (32 * WV) + lane * WV + (k % WV);
    }
    template <bool CG>
    __device__ static __forceinline__ void load(const E *row, int lane, E (&r)[VEC])
    {
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            const V *q = reinterpret_cast<const V *>(row + c * 32 * WV + lane * WV);
            const V v = CG ? __ldcg(q) : __ldg(q);
            unpack(v, &r[c * WV]);
        }
    }
    __device__ static __forceinline__ void store(E *row, int lane, const E (&r)[VEC])
    {
#pragma unroll
        for (int c = 0; c < NCH; ++c)
            *reinterpret_cast<V *>(row + c * 32 * WV + lane * WV) = pack<V>(&r[c * WV]);
    }
};

// acc += sum over in-list slots [a, e) of P * row(source): indices and
// coefficients loaded 32 at a time (one per lane) and broadcast; U rows in
// flight per warp (U chosen so the rows fit the registers).
template <typename E, int VEC, bool W>
__device__ __forceinline__ void gather_rows(const BatchParams &p, const E *x, int a, int e,
                                            int lane, E (&acc)[VEC])
{
    using IO = RowIO<E, VEC>;
    constexpr int BP = IO::BP;
    constexpr int U = VEC * sizeof(E) >= 32 ? 2 : 4;
    const E *ew = static_cast<const E *>(p.ew);
    const E *inv = static_cast<const E *>(p.inv);
    for (int base = a; base < e; base += 32) {
        const int cnt = min(32, e - base);
        int myv = 0;
        E myc = E(0);
        if (lane < cnt) {
            myv = __ldg(p.row_idx + base + lane);
            myc = W ? __ldg(ew + base + lane) : __ldg(inv + myv);
        }
        int j = 0;
        for (; j + U <= cnt; j += U) {
            E r[U][VEC];
            E c[U];
#pragma unroll
            for (int t = 0; t < U; ++t) {
                const int v = __shfl_sync(FULL, myv, j + t);
                c[t] = __shfl_sync(FULL, myc, j + t);
                IO::template load<false>(x + (size_t)v * BP, lane, r[t]);
            }
#pragma unroll
            for (int k = 0; k < VEC; ++k)
#pragma unroll
                for (int t = 0; t < U; ++t) acc[k] += c[t] * r[t][k];
        }
        for (; j < cnt; ++j) {
            E r0[VEC];
            const int v0 = __shfl_sync(FULL, myv, j);
            const E c0 = __shfl_sync(FULL, myc, j);
            IO::template load<false>(x + (size_t)v0 * BP, lane, r0);
#pragma unroll
            for (int k = 0; k < VEC; ++k) acc[k] += c0 * r0[k];
        }
    }
}

template <typename E>
struct BatchShared {
    double *werr, *wdang;  // this warp's per-column sums [Bp]
    const int *seed;       // [Bp]
    const E *tele;         // [Bp] (1-d) + d D_b
    const int *frozen;     // [Bp]
};

// New row of vertex u from its gathered sums; adds the L1 change and (for a
// dangling u) the new values to the warp's per-column sums.
template <typename E, int VEC>
__device__ __forceinline__ void batch_fin(const BatchParams &p, int u, const E (&acc)[VEC],
                                          const E *xin, E *xout, int lane, E d,
                                          const BatchShared<E> &sh)
{
    using IO = RowIO<E, VEC>;
    constexpr int BP = IO::BP;
    E xo[VEC], xn[VEC], tv[VEC];
    IO::template load<false>(xin + (size_t)u * BP, lane, xo);
    const E *trow = static_cast<const E *>(p.tele_rows);
    if (trow) IO::template load<false>(trow + (size_t)u * BP, lane, tv);
    const bool dangling = __ldg(p.outdeg + u) == 0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int b = IO::col(lane, k);
        E v = d * acc[k];
        if (trow) v += tv[k] * sh.tele[b];
        else if (sh.seed[b] == u) v += sh.tele[b];
        if (sh.frozen[b]) v = xo[k];
        xn[k] = v;
        sh.werr[b] += fabs((double)v - (double)xo[k]);
        if (dangling) sh.wdang[b] += (double)v;
    }
    IO::store(xout + (size_t)u * BP, lane, xn);
}

template <typename E, int VEC, bool W>
__global__ void __launch_bounds__(BATCH_BS, 1) k_batch_sweep(BatchParams p)
{
    using IO = RowIO<E, VEC>;
    constexpr int BP = IO::BP;
    extern __shared__ __align__(16) unsigned char bsm[];
    double *wsum = reinterpret_cast<double *>(bsm);  // [warps][2][Bp]
    E *s_tele = reinterpret_cast<E *>(bsm + (size_t)BATCH_WARPS * 2 * BP * sizeof(double));
    int *s_seed = reinterpret_cast<int *>(s_tele + BP);
    int *s_frozen = s_seed + BP;
    __shared__ bool is_last;
    BatchState *st = p.st;
    if (st->done) {
        if (p.use_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(p.cond, 0u);
        return;
    }
    const int iter = st->iter;
    const double dd = st->d;
    const E d = (E)dd;
    const E *xin = static_cast<const E *>((iter & 1) ? p.x1 : p.x0);
    E *xout = static_cast<E *>((iter & 1) ? p.x0 : p.x1);
    E *part = static_cast<E *>(p.part);
    for (int t = threadIdx.x; t < BP; t += blockDim.x) {
        s_seed[t] = p.seed[t];
        s_tele[t] = (E)((1.0 - dd) + dd * p.dang[t]);
        s_frozen[t] = p.conv[t] != 0;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    BatchShared<E> sh;
    sh.werr = wsum + (size_t)warp * 2 * BP;
    sh.wdang = sh.werr + BP;
    sh.seed = s_seed;
    sh.tele = s_tele;
    sh.frozen = s_frozen;
    for (int k = lane; k < 2 * BP; k += 32) sh.werr[k] = 0.0;
    __syncthreads();

    // blocks interleaved: neighbouring items (like cost) go to different SMs
    const int gw = warp * gridDim.x + blockIdx.x, nw = gridDim.x * BATCH_WARPS;
    const int nitems = p.nseg + (p.n - p.nhub);
    for (int r = 0;; ++r) {
        const int i = r * nw + ((r & 1) ? nw - 1 - gw : gw);
        if (i >= nitems) break;
        E acc[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) acc[k] = E(0);
        if (i < p.nseg) {
            const int4 dsc = __ldg(p.sdesc + i);
            gather_rows<E, VEC, W>(p, xin, dsc.z, dsc.w, lane, acc);
            IO::store(part + (size_t)i * BP, lane, acc);
            __syncwarp();
            __threadfence();
            const int h = dsc.x, s0 = dsc.y;
            const int nsg = p.seg_start[h + 1] - s0;
            int last = 0;
            if (lane == 0) last = atomicAdd(&p.seg_cnt[h], 1) == nsg - 1;
            last = __shfl_sync(FULL, last, 0);
            if (last) {
                __threadfence();
#pragma unroll
                for (int k = 0; k < VEC; ++k) acc[k] = E(0);
                for (int j = 0; j < nsg; ++j) {
                    E rr[VEC];
                    IO::template load<true>(part + (size_t)(s0 + j) * BP, lane, rr);
#pragma unroll
                    for (int k = 0; k < VEC; ++k) acc[k] += rr[k];
                }
                if (lane == 0) p.seg_cnt[h] = 0;
                batch_fin<E, VEC>(p, h, acc, xin, xout, lane, d, sh);
            }
        } else {
            const int u = p.nhub + (i - p.nseg);
            gather_rows<E, VEC, W>(p, xin, __ldg(p.col_ptr + u), __ldg(p.col_ptr + u + 1), lane,
                                   acc);
            batch_fin<E, VEC>(p, u, acc, xin, xout, lane, d, sh);
        }
    }
    __syncthreads();
    // this block's per-column sums, over the warps in order
    for (int t = threadIdx.x; t < BP; t += blockDim.x) {
        double e = 0.0, dm = 0.0;
        for (int w = 0; w < BATCH_WARPS; ++w) {
            e += wsum[(size_t)w * 2 * BP + t];
            dm += wsum[(size_t)w * 2 * BP + BP + t];
        }
        if (e != 0.0) fx_add(&p.acc[4 * t], &p.acc[4 * t + 1], e);
        if (dm != 0.0) fx_add(&p.acc[4 * t + 2], &p.acc[4 * t + 3], dm);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last) return;
    // the last block closes the sweep: per-column stop test
    __threadfence();
    int active = 0;
    for (int t = threadIdx.x; t < BP; t += blockDim.x) {
        volatile long long *a = p.acc + 4 * t;
        const double e = fx_value(a[0], a[1]);
        const double dm = fx_value(a[2], a[3]);
        a[0] = 0;
        a[1] = 0;
        a[2] = 0;
        a[3] = 0;
        if (p.conv[t] == 0) {
            p.err[t] = e;
            p.dang[t] = dm;
            if (e <= st->tau) {
                p.conv[t] = iter + 1;
            } else if (p.stall && e >= p.best[t] && ++p.since[t] >= STALL_SWEEPS) {
                p.conv[t] = -2 - iter;  // stopped at the rounding floor after sweep iter + 1
            } else {
                if (e < p.best[t]) {
                    p.best[t] = e;
                    p.since[t] = 0;
                }
                active = 1;
            }
        }
    }
    const int n_active = __syncthreads_count(active);
    if (threadIdx.x == 0) {
        st->ticket = 0;
        st->iter = iter + 1;
        const bool stop = n_active == 0 || iter + 1 >= st->max_iter;
        // enough columns stopped: end the loop so the host moves the running
        // ones into narrower passes
        const bool pause = !stop && n_active <= p.pause_at;
        st->done = (stop || pause) ? 1 : 0;
        st->paused = pause ? 1 : 0;
        __threadfence();
        if (p.use_cond) cudaGraphSetConditional(p.cond, (stop || pause) ? 0u : 1u);
    }
}

// ------------------------------------------------------------ set-up
__global__ void k_count_above(int32_t n, const int32_t *__restrict__ col_ptr, int t,
                              int32_t *count)
{
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const bool big = u < n && col_ptr[u + 1] - col_ptr[u] > t;
    const unsigned b = __ballot_sync(FULL, big);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(count, __popc(b));
}

__global__ void k_seg_count(int32_t nhub, const int32_t *__restrict__ col_ptr, int seg,
                            int32_t *nseg)
{
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < nhub) nseg[h] = (col_ptr[h + 1] - col_ptr[h] + seg - 1) / seg;
}

__global__ void k_seg_desc(int32_t nseg, int32_t nhub, const int32_t *__restrict__ seg_start,
                           int seg, const int32_t *__restrict__ col_ptr, int4 *desc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int lo = 0, hi = nhub - 1;  // vertex owning segment i
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (seg_start[mid] <= i) lo = mid;
        else hi = mid - 1;
    }
    const int a = col_ptr[lo] + (i - seg_start[lo]) * seg;
    desc[i] = make_int4(lo, seg_start[lo], a, min(a + seg, col_ptr[lo + 1]));
}

// x0 <- 1/n everywhere; per-column state; seeds mapped to the degree-ordered
// ids (flag 1 in *bad if one lies outside [0, n)).
template <typename E, int BP>
__global__ void k_batch_init(BatchParams p, const int32_t *__restrict__ seeds,
                             const int32_t *__restrict__ o2n, int ncols, double dang0,
                             int32_t *bad)
{
    const E x = (E)(1.0 / (double)p.n);
    E *x0 = static_cast<E *>(p.x0);
    const size_t total = (size_t)p.n * BP;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x)
        x0[i] = x;
    if (blockIdx.x == 0)
        for (int t = threadIdx.x; t < BP; t += blockDim.x) {
            int sd = -1;
            if (t < ncols && seeds) {
                const int s = seeds[t];
                if (s < 0 || s >= p.n) atomicOr(bad, 1);
                else sd = o2n[s];
            }
            p.seed[t] = sd;
            p.conv[t] = t < ncols ? 0 : -1;
            p.dang[t] = dang0;
            p.err[t] = 0.0;
            p.best[t] = INFINITY;
            p.since[t] = 0;
            p.acc[4 * t] = p.acc[4 * t + 1] = p.acc[4 * t + 2] = p.acc[4 * t + 3] = 0;
        }
}

// Dense teleport rows of the pass in the degree-ordered ids:
// out[k][b] = V[n2o[k]][c0 + cols[b]] for the pass's row positions b (cols
// null: cols[b] = b for b < ncols; a negative column: padding, 0); flag 2
// in *bad for a negative or non-finite entry.
template <typename E, int BP>
__global__ void k_batch_tele(int32_t n, const E *__restrict__ V, int ld, int c0, int ncols,
                             const int32_t *__restrict__ n2o, E *out, int32_t *bad,
                             const int32_t *__restrict__ cols)
{
    const size_t total = (size_t)n * BP;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / BP), b = (int)(i % BP);
        const int col = cols ? cols[b] : (b < ncols ? b : -1);
        E v = E(0);
        if (col >= 0) {
            v = V[(size_t)n2o[k] * ld + c0 + col];
            if (!(v >= E(0)) || isinf((double)v)) atomicOr(bad, 2);
        }
        out[i] = v;
    }
}

// Column sums of the final iterate (exact fixed-point accumulation).
template <typename E, int VEC>
__global__ void __launch_bounds__(BATCH_BS, 1) k_batch_colsum(BatchParams p, const E *x)
{
    using IO = RowIO<E, VEC>;
    constexpr int BP = IO::BP;
    extern __shared__ __align__(16) unsigned char bsm[];
    double *ws = reinterpret_cast<double *>(bsm);  // [warps][Bp]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double sm[VEC];
#pragma unroll
    for (int k = 0; k < VEC; ++k) sm[k] = 0.0;
    for (int u = blockIdx.x * BATCH_WARPS + warp; u < p.n; u += gridDim.x * BATCH_WARPS) {
        E r[VEC];
        IO::template load<false>(x + (size_t)u * BP, lane, r);
#pragma unroll
        for (int k = 0; k < VEC; ++k) sm[k] += (double)r[k];
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) ws[(size_t)warp * BP + IO::col(lane, k)] = sm[k];
    __syncthreads();
    for (int t = threadIdx.x; t < BP; t += blockDim.x) {
        double a = 0.0;
        for (int w = 0; w < BATCH_WARPS; ++w) a += ws[(size_t)w * BP + t];
        if (a != 0.0) fx_add(&p.acc[4 * t], &p.acc[4 * t + 1], a);
    }
}

// X_out[u][c0 + outmap[b]] = x[o2n[u]][b] / sum_b for the row positions b
// with outmap[b] >= 0 (the columns written now).
template <typename E, int BP>
__global__ void k_batch_out(BatchParams p, const E *x, const int32_t *__restrict__ o2n,
                            const int32_t *__restrict__ outmap, int ld, int c0, E *X_out)
{
    const size_t total = (size_t)p.n * BP;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const int u = (int)(i / BP), b = (int)(i % BP);
        const int col = outmap[b];
        if (col < 0) continue;
        const double sum = fx_value(p.acc[4 * b], p.acc[4 * b + 1]);
        X_out[(size_t)u * ld + c0 + col] = (E)((double)x[(size_t)o2n[u] * BP + b] / sum);
    }
}

// A narrower pass's first iterate from its parent's rows: y[u][i] =
// x[u][from[i]] (x rows of bp_src entries; from[i] < 0: padding, 0).
template <typename E, int BP>
__global__ void k_batch_take(int32_t n, const E *__restrict__ x, int bp_src,
                             const int32_t *__restrict__ from, E *y)
{
    const size_t total = (size_t)n * BP;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (size_t)gridDim.x * blockDim.x) {
        const size_t u = i / BP;
        const int b = (int)(i % BP);
        const int f = from[b];
        y[i] = f >= 0 ? x[u * (size_t)bp_src + f] : E(0);
    }
}

// Segments of the vertices with more than BATCH_SEG in-edges (built once).
static pr_status ensure_batch_items(pr_graph *g, cudaStream_t s)
{
    if (g->bnhub >= 0) return PR_OK;
    const int32_t n = g->n;
    const int32_t *rcp = g->r_col_ptr.as<int32_t>();
    PR_TRY(buf_alloc(g, g->bseg_start, sizeof(int32_t) * ((size_t)n + 1), s));
    int32_t *cnt = g->bseg_start.as<int32_t>() + n;  // scratch word
    PR_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int32_t), s));
    k_count_above<<<(n + 255) / 256, 256, 0, s>>>(n, rcp, BATCH_SEG, cnt);
    note_launch();
    PR_LAUNCH_CHECK();
    int32_t nhub = 0;
    PR_CUDA(cudaMemcpyAsync(&nhub, cnt, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    int32_t nseg = 0;
    PR_TRY(buf_alloc(g, g->bseg_cnt, sizeof(int32_t) * (size_t)std::max(nhub, 1), s));
    PR_CUDA(cudaMemsetAsync(g->bseg_cnt.p, 0, sizeof(int32_t) * (size_t)std::max(nhub, 1), s));
    if (nhub > 0) {
        k_seg_count<<<(nhub + 255) / 256, 256, 0, s>>>(nhub, rcp, BATCH_SEG,
                                                        g->bseg_start.as<int32_t>());
        note_launch();
        PR_LAUNCH_CHECK();
        PR_TRY(scan_exclusive(g, g->bseg_start.as<int32_t>(), g->bseg_start.as<int32_t>(), nhub,
                              s));
        PR_CUDA(cudaMemcpyAsync(&nseg, g->bseg_start.as<int32_t>() + nhub, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
    }
    PR_TRY(buf_alloc(g, g->bseg_desc, sizeof(int4) * (size_t)std::max(nseg, 1), s));
    if (nseg > 0) {
        k_seg_desc<<<(nseg + 255) / 256, 256, 0, s>>>(nseg, nhub, g->bseg_start.as<int32_t>(),
                                                       BATCH_SEG, rcp, g->bseg_desc.as<int4>());
        note_launch();
        PR_LAUNCH_CHECK();
    }
    PR_CUDA(cudaStreamSynchronize(s));
    g->bnhub = nhub;
    g->bnseg = nseg;
    return PR_OK;
}

// Per-column state in one buffer: acc [Bp][4] int64, dang/err/best [Bp]
// double, conv/seed/since [Bp] int32, then the BatchState (and the error
// word), then two [Bp] int32 maps of row positions to columns.
constexpr size_t COLS_STATE = (size_t)BATCH_COLS * (32 + 3 * 8 + 3 * 4);
constexpr size_t COLS_MAPS = COLS_STATE + 256;
static size_t cols_bytes() { return COLS_MAPS + 2 * sizeof(int32_t) * BATCH_COLS; }

// The state a narrower pass starts from: the columns still running when its
// parent pass paused, their rows in the parent's iterate and their
// per-column sums and counters.
struct BatchResume {
    int iter;                      // sweeps done
    const void *x;                 // parent iterate, rows of bp_src entries
    int bp_src;
    void *x0, *x1;                 // this pass's iterates (each n x Bp)
    int count;                     // columns taken over
    int32_t from[BATCH_COLS];      // their positions in the parent's rows
    int32_t cols[BATCH_COLS];      // their columns (c0 + cols[i] in X_out)
    int32_t seed[BATCH_COLS], since[BATCH_COLS];
    double dang[BATCH_COLS], err[BATCH_COLS], best[BATCH_COLS];
};

// One pass over up to Bp = 32 * VEC columns: from the start (rs null) or
// from a parent pass's state.  Once few enough columns are still running
// (at most Bp/2 + Bp/8), the loop pauses: the stopped columns are written
// out and the running ones go on in narrower passes (Bp/2 wide, and 32 wide
// for the rest), which gather half the row bytes or less per in-edge (the
// batched sweep's time follows its row width; a column's arithmetic does
// not depend on the pass it is in, so its result is the same).
template <typename E, int VEC>
static pr_status batch_pass(pr_graph *g, const pr_options *o, const int32_t *seeds, const E *V,
                            int ncols, int ld, int c0, E *X_out, pr_result *res, cudaStream_t s,
                            const BatchResume *rs = nullptr)
{
    constexpr int BP = 32 * VEC;
    constexpr bool fp64 = sizeof(E) == 8;
    const int32_t n = g->n;
    const bool weighted = g->weighted;
    BatchParams p;
    memset(&p, 0, sizeof(p));
    p.n = n;
    p.col_ptr = g->r_col_ptr.as<int32_t>();
    p.row_idx = g->r_row_idx.as<int32_t>();
    p.outdeg = g->r_outdeg.as<int32_t>();
    p.inv = fp64 ? g->r_inv64.p : g->r_inv32.p;
    p.ew = weighted ? (fp64 ? g->p64_csc.p : g->p32_csc.p) : nullptr;
    p.nhub = g->bnhub;
    p.sdesc = g->bseg_desc.as<int4>();
    p.nseg = g->bnseg;
    p.seg_start = g->bseg_start.as<int32_t>();
    p.seg_cnt = g->bseg_cnt.as<int32_t>();
    p.part = g->bpart.p;
    p.x0 = rs ? rs->x0 : g->bx0.p;
    p.x1 = rs ? rs->x1 : g->bx1.p;
    p.stall = fp64 ? 0 : 1;
    p.pause_at = VEC > 1 ? BP / 2 + BP / 8 : -1;
    char *cb = static_cast<char *>(g->bcols.p);
    p.acc = reinterpret_cast<long long *>(cb);
    p.dang = reinterpret_cast<double *>(cb + BATCH_COLS * 32);
    p.err = p.dang + BATCH_COLS;
    p.best = p.err + BATCH_COLS;
    p.conv = reinterpret_cast<int32_t *>(p.best + BATCH_COLS);
    p.seed = p.conv + BATCH_COLS;
    p.since = p.seed + BATCH_COLS;
    p.st = reinterpret_cast<BatchState *>(cb + BATCH_COLS * 68);
    int32_t *d_map = reinterpret_cast<int32_t *>(cb + COLS_MAPS);   // [Bp]
    int32_t *d_map2 = d_map + BATCH_COLS;                            // [Bp]

    // row position b holds column cols[b] of the pass (-1: padding)
    int32_t cols[BATCH_COLS];
    for (int b = 0; b < BP; ++b) cols[b] = rs ? (b < rs->count ? rs->cols[b] : -1) : (b < ncols ? b : -1);

    BatchState hs;
    memset(&hs, 0, sizeof(hs));
    hs.max_iter = o->max_iter;
    hs.tau = o->threshold;
    hs.d = o->d;
    hs.ncols = rs ? rs->count : ncols;
    hs.iter = rs ? rs->iter : 0;
    PR_CUDA(cudaMemcpyAsync(p.st, &hs, sizeof(hs), cudaMemcpyHostToDevice, s));
    int32_t *bad = reinterpret_cast<int32_t *>(p.st + 1);
    PR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int32_t), s));
    const int ib = std::max(1, std::min<int>((int)(((size_t)n * BP + 255) / 256), g->num_sms * 8));
    if (!rs) {
        const double dang0 = (double)g->n_dangling * (double)(E)(1.0 / (double)n);
        k_batch_init<E, BP><<<ib, 256, 0, s>>>(p, seeds ? seeds + c0 : nullptr,
                                               g->o2n.as<int32_t>(), ncols, dang0, bad);
        note_launch();
    } else {
        int32_t conv[BATCH_COLS], seed[BATCH_COLS], since[BATCH_COLS];
        double dang[BATCH_COLS], err[BATCH_COLS], best[BATCH_COLS];
        int32_t from[BATCH_COLS];
        for (int b = 0; b < BP; ++b) {
            const bool real = b < rs->count;
            from[b] = real ? rs->from[b] : -1;
            conv[b] = real ? 0 : -1;
            seed[b] = real ? rs->seed[b] : -1;
            since[b] = real ? rs->since[b] : 0;
            dang[b] = real ? rs->dang[b] : 0.0;
            err[b] = real ? rs->err[b] : 0.0;
            best[b] = real ? rs->best[b] : INFINITY;
        }
        PR_CUDA(cudaMemcpyAsync(d_map2, from, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
        k_batch_take<E, BP><<<ib, 256, 0, s>>>(n, static_cast<const E *>(rs->x), rs->bp_src,
                                               d_map2, static_cast<E *>(p.x0));
        note_launch();
        PR_CUDA(cudaMemcpyAsync(p.conv, conv, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(p.seed, seed, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(p.since, since, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(p.dang, dang, sizeof(double) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(p.err, err, sizeof(double) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemcpyAsync(p.best, best, sizeof(double) * BP, cudaMemcpyHostToDevice, s));
        PR_CUDA(cudaMemsetAsync(p.acc, 0, sizeof(long long) * 4 * BP, s));
        // the first sweep reads x0: an even sweep count here, else swap
        if (hs.iter & 1) std::swap(p.x0, p.x1);
        PR_CUDA(cudaStreamSynchronize(s));  // the host arrays above go out of scope
    }
    if (V) {
        PR_TRY(buf_alloc(g, g->btele, (size_t)n * BP * sizeof(E), s));
        PR_CUDA(cudaMemcpyAsync(d_map, cols, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
        k_batch_tele<E, BP><<<ib, 256, 0, s>>>(n, V, ld, c0, ncols, g->n2o.as<int32_t>(),
                                               g->btele.as<E>(), bad, d_map);
        note_launch();
        p.tele_rows = g->btele.p;
    }
    PR_LAUNCH_CHECK();
    int32_t hbad = 0;
    PR_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    if (hbad) {
        if (hbad & 1) set_error("pr_solve_batched: a seed lies outside [0, %d)", n);
        else set_error("pr_solve_batched: teleport entries must be finite and non-negative");
        return PR_ERR_INVALID_ARG;
    }

    const void *func = weighted ? reinterpret_cast<const void *>(&k_batch_sweep<E, VEC, true>)
                                : reinterpret_cast<const void *>(&k_batch_sweep<E, VEC, false>);
    const size_t smem = (size_t)BATCH_WARPS * 2 * BP * sizeof(double) + (size_t)BP * (sizeof(E) + 8);
    PR_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const int nitems = p.nseg + (n - p.nhub);
    const unsigned grid =
        (unsigned)std::max(1, std::min((nitems + BATCH_WARPS - 1) / BATCH_WARPS, g->num_sms));
    const int iter0 = hs.iter;
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
            p.cond = h;
            p.use_cond = 1;
            void *args[] = {&p};
            cudaKernelNodeParams kp = {};
            kp.func = const_cast<void *>(func);
            kp.gridDim = dim3(grid);
            kp.blockDim = dim3(BATCH_BS);
            kp.sharedMemBytes = (unsigned)smem;
            kp.kernelParams = args;
            e = cudaGraphAddKernelNode(&knode, cp.conditional.phGraph_out[0], nullptr, 0, &kp);
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) e = cudaGraphLaunch(exec, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (exec) cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_status(e, "batched loop graph", __FILE__, __LINE__);
        PR_CUDA(cudaMemcpyAsync(&hs, p.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        note_launch((uint64_t)(hs.iter - iter0) + 1);
    } else {
        p.use_cond = 0;
        void *args[] = {&p};
        while (hs.iter < o->max_iter) {
            const int batch = std::min(16, o->max_iter - hs.iter);
            for (int k = 0; k < batch; ++k) {
                PR_CUDA(cudaLaunchKernel(func, dim3(grid), dim3(BATCH_BS), args, smem, s));
                note_launch();
            }
            PR_CUDA(cudaMemcpyAsync(&hs, p.st, sizeof(hs), cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaStreamSynchronize(s));
            if (hs.done) break;
        }
    }

    // column sums of the iterate; the stopped columns (all of them at the
    // end) written out with their results
    const E *xf = static_cast<const E *>((hs.iter & 1) ? p.x1 : p.x0);
    E *xfree = static_cast<E *>((hs.iter & 1) ? p.x0 : p.x1);
    const bool split = hs.paused != 0;
    const size_t smem_s = (size_t)BATCH_WARPS * BP * sizeof(double);
    PR_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_batch_colsum<E, VEC>),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_s));
    k_batch_colsum<E, VEC><<<g->num_sms, BATCH_BS, smem_s, s>>>(p, xf);
    note_launch();
    long long acc[BATCH_COLS * 4];
    double err[BATCH_COLS];
    int32_t conv[BATCH_COLS];
    PR_CUDA(cudaMemcpyAsync(acc, p.acc, sizeof(long long) * 4 * BP, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(err, p.err, sizeof(double) * BP, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(conv, p.conv, sizeof(int32_t) * BP, cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    int32_t outmap[BATCH_COLS];
    for (int b = 0; b < BP; ++b) {
        const bool stopped = conv[b] > 0 || conv[b] <= -2;
        outmap[b] = (cols[b] >= 0 && (!split || stopped)) ? cols[b] : -1;
    }
    PR_CUDA(cudaMemcpyAsync(d_map, outmap, sizeof(int32_t) * BP, cudaMemcpyHostToDevice, s));
    k_batch_out<E, BP><<<g->num_sms * 8, 256, 0, s>>>(p, xf, g->o2n.as<int32_t>(), d_map, ld, c0,
                                                       X_out);
    note_launch();
    PR_LAUNCH_CHECK();
    pr_status all = PR_OK;
    for (int b = 0; b < BP; ++b) {
        if (outmap[b] < 0) continue;
        const int it = conv[b] > 0 ? conv[b] : conv[b] <= -2 ? -conv[b] - 1 : hs.iter;
        const pr_status cs = conv[b] > 0 ? PR_OK : PR_NOT_CONVERGED;
        if (cs != PR_OK) all = PR_NOT_CONVERGED;
        if (!res) continue;
        pr_result &r = res[c0 + outmap[b]];
        r.iters = it;
        r.outer_iters = 0;
        r.residual = err[b];
        r.sum_before_norm = (double)acc[4 * b] * 9.094947017729282e-13 +
                            (double)acc[4 * b + 1] * 8.271806125530277e-25;
        r.status = cs;
    }
    if constexpr (VEC > 1) {
        if (split) {
            // the running columns go on in a pass of Bp/2 columns and, for
            // those beyond, one of 32; both iterate in the free buffer of this
            // pass (two halves of n x Bp), reading their start from xf
            BatchResume *rr = new BatchResume;  // large: not on the stack
            rr->iter = hs.iter;
            rr->x = xf;
            rr->bp_src = BP;
            PR_CUDA(cudaMemcpyAsync(rr->seed, p.seed, sizeof(int32_t) * BP, cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaMemcpyAsync(rr->since, p.since, sizeof(int32_t) * BP, cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaMemcpyAsync(rr->dang, p.dang, sizeof(double) * BP, cudaMemcpyDeviceToHost, s));
            PR_CUDA(cudaMemcpyAsync(rr->best, p.best, sizeof(double) * BP, cudaMemcpyDeviceToHost, s));
            cudaError_t e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) {
                delete rr;
                return cuda_status(e, "batched split", __FILE__, __LINE__);
            }
            int run[BATCH_COLS], nrun = 0;
            for (int b = 0; b < BP; ++b)
                if (cols[b] >= 0 && conv[b] == 0) run[nrun++] = b;
            const size_t half = (size_t)n * (BP / 2);
            pr_status st = PR_OK;
            for (int first = 0; first < nrun;) {
                const int width = first == 0 ? BP / 2 : 32;
                const int cnt = std::min(width, nrun - first);
                BatchResume &q = *rr;
                // per-column arrays in the sub-pass's order (from the parent)
                int32_t seed2[BATCH_COLS], since2[BATCH_COLS];
                double dang2[BATCH_COLS], best2[BATCH_COLS], err2[BATCH_COLS];
                int32_t from2[BATCH_COLS], cols2[BATCH_COLS];
                for (int i = 0; i < cnt; ++i) {
                    const int b = run[first + i];
                    from2[i] = b;
                    cols2[i] = cols[b];
                    seed2[i] = q.seed[b];
                    since2[i] = q.since[b];
                    dang2[i] = q.dang[b];
                    best2[i] = q.best[b];
                    err2[i] = err[b];
                }
                BatchResume *sub = new BatchResume;
                sub->iter = hs.iter;
                sub->x = xf;
                sub->bp_src = BP;
                sub->x0 = xfree;
                sub->x1 = xfree + half;
                sub->count = cnt;
                memcpy(sub->from, from2, sizeof(int32_t) * cnt);
                memcpy(sub->cols, cols2, sizeof(int32_t) * cnt);
                memcpy(sub->seed, seed2, sizeof(int32_t) * cnt);
                memcpy(sub->since, since2, sizeof(int32_t) * cnt);
                memcpy(sub->dang, dang2, sizeof(double) * cnt);
                memcpy(sub->best, best2, sizeof(double) * cnt);
                memcpy(sub->err, err2, sizeof(double) * cnt);
                pr_status ss;
                if (first == 0)
                    ss = batch_pass<E, VEC / 2>(g, o, seeds, V, ncols, ld, c0, X_out, res, s, sub);
                else
                    ss = batch_pass<E, 1>(g, o, seeds, V, ncols, ld, c0, X_out, res, s, sub);
                delete sub;
                if (ss != PR_OK && ss != PR_NOT_CONVERGED) {
                    st = ss;
                    break;
                }
                if (ss == PR_NOT_CONVERGED) all = PR_NOT_CONVERGED;
                first += cnt;
            }
            delete rr;
            if (st != PR_OK) return st;
        }
    }
    return all;
}

template <typename E>
static pr_status solve_batched(pr_graph *g, const pr_options *o, int32_t B, const int32_t *seeds,
                               const E *V, E *X_out, pr_result *res, cudaStream_t s)
{
    constexpr int MAXC = sizeof(E) == 8 ? 128 : 256;  // columns per pass
    const int first = std::min<int>(B, MAXC);
    const int bp = first <= 32 ? 32 : first <= 64 ? 64 : first <= 128 ? 128 : 256;
    const size_t rows = (size_t)g->n * bp * sizeof(E);
    PR_TRY(buf_alloc(g, g->bx0, rows, s));
    PR_TRY(buf_alloc(g, g->bx1, rows, s));
    PR_TRY(buf_alloc(g, g->bpart, (size_t)std::max(g->bnseg, 1) * bp * sizeof(E), s));
    PR_TRY(buf_alloc(g, g->bcols, cols_bytes(), s));
    pr_status all = PR_OK;
    for (int c0 = 0; c0 < B; c0 += MAXC) {
        const int nc = std::min<int>(MAXC, B - c0);
        pr_status st;
        if (nc <= 32) st = batch_pass<E, 1>(g, o, seeds, V, nc, B, c0, X_out, res, s);
        else if (nc <= 64) st = batch_pass<E, 2>(g, o, seeds, V, nc, B, c0, X_out, res, s);
        else if (nc <= 128) st = batch_pass<E, 4>(g, o, seeds, V, nc, B, c0, X_out, res, s);
        else if constexpr (MAXC > 128) st = batch_pass<E, 8>(g, o, seeds, V, nc, B, c0, X_out, res, s);
        else st = PR_ERR_INVALID_ARG;
        if (st != PR_OK && st != PR_NOT_CONVERGED) return st;
        if (st == PR_NOT_CONVERGED) all = st;
    }
    return all;
}

}  // namespace fpr

using namespace fpr;

extern "C" pr_status pr_solve_batched(pr_graph *g, const pr_options *o, int32_t B,
                                      const int32_t *seeds, const void *V, void *X_out,
                                      pr_result *res, void *stream)
{
    if (res && B > 0) memset(res, 0, sizeof(pr_result) * (size_t)B);
    if (!g || !o || B < 1 || (!seeds == !V) || !X_out) {
        set_error("pr_solve_batched: need a graph, options, B >= 1, X_out and exactly one of "
                  "seeds and V");
        return PR_ERR_INVALID_ARG;
    }
    PR_TRY(validate_options(o));
    PR_TRY(check_device(g));
    if (o->variant != PR_JACOBI || (o->precision != PR_FP32 && o->precision != PR_FP64) ||
        o->norm != PR_NORM_L1) {
        set_error("pr_solve_batched: supports the Jacobi sweep in FP32 or FP64 with the L1 stop "
                  "rule");
        return PR_ERR_UNSUPPORTED;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    PR_TRY(ensure_batch_items(g, s));
    return o->precision == PR_FP64
               ? solve_batched<double>(g, o, B, seeds, static_cast<const double *>(V),
                                       static_cast<double *>(X_out), res, s)
               : solve_batched<float>(g, o, B, seeds, static_cast<const float *>(V),
                                      static_cast<float *>(X_out), res, s);
}
