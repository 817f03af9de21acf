// common.cuh -- internal declarations shared by the CUDA translation units of
// libfusedpr: the graph handle, device allocation through the caller's hooks,
// error reporting and small device helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/fusedpr.h"

namespace fpr {

constexpr unsigned FULL = 0xffffffffu;

// ---------------------------------------------------------------- errors --
void set_error(const char *fmt, ...);
// process-wide count of kernel launches issued by the library (diagnostics)
void note_launch(unsigned long long k = 1);
unsigned long long launches();
pr_status cuda_status(cudaError_t e, const char *what, const char *file, int line);

#define PR_CUDA(expr)                                                                    \
    do {                                                                                 \
        cudaError_t _e = (expr);                                                         \
        if (_e != cudaSuccess) return ::fpr::cuda_status(_e, #expr, __FILE__, __LINE__); \
    } while (0)

#define PR_TRY(expr)                          \
    do {                                              \
        pr_status _s = (expr);                        \
        if (_s != PR_OK) return _s;                   \
    } while (0)

#define PR_LAUNCH_CHECK() PR_CUDA(cudaGetLastError())

// ------------------------------------------------------------ allocation --
struct Mem {
    pr_allocator hooks{};
    bool has_hooks = false;
    cudaStream_t stream = nullptr;  // stream of the owner (used at destroy)
    void *alloc(size_t bytes, cudaStream_t s);
    void free(void *p, size_t bytes, cudaStream_t s);
};

// A device buffer owned by a graph (freed at destroy or on resize).
struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
    template <typename T>
    T *as() const { return static_cast<T *>(p); }
};

// Exact fixed-point accumulators of a sweep's partial sums (two words:
// integer part scaled by 2^40, fraction scaled by 2^80).  Blocks add into
// slot blockIdx % ACC_SLOTS so that same-address atomics do not serialise;
// integer sums make the total independent of the slot and of the order.
constexpr int ACC_SLOTS = 32;
struct alignas(64) AccSlot {
    long long res_hi, res_lo, dang_hi, dang_lo, sum_hi, sum_lo;
    unsigned long long res_max;  // bit pattern of the largest |x' - x| (>= 0)
    long long pad;
};

// Device state of one solve: scalars read by every block at the start of a
// sweep and rewritten by the block that finishes the sweep last.
struct SolveState {
    AccSlot acc[ACC_SLOTS];      // reset by the finishing block
    unsigned int ticket;         // blocks finished in this sweep
    int iter;                    // sweeps completed
    int done;                    // 1: stop (converged or out of sweeps)
    int status;                  // PR_OK / PR_NOT_CONVERGED / error
    int norm;
    int max_iter;
    int record;                  // history != nullptr
    int phase;                   // defect correction: 0 inner sweeps, 1 outer step
    int inner_iter;              // defect correction: sweeps in this inner solve
    int outer_iter;              // defect correction: residual evaluations
    int max_outer;
    int error;                   // set by a block whose bounded wait gave up
    double tau;
    double d;
    double base;      // (1-d)/n
    double inv_n;     // 1/n
    double dang;      // dangling mass of the current iterate (stored units)
    double sigma;     // true value = sigma * stored value (fused sweep rescale)
    double res;       // last sweep's L1 error (true units)
    double resmax;    // last sweep's max error
    double sum;       // sum of the current iterate (stored units)
    double scale;     // defect correction: power-of-two scale of the correction
    double rnorm;     // defect correction: ||r||_1 of the current outer step
    double inner_tol; // defect correction: inner stop threshold (true units)
    double inner_rel;
    double inner_floor; // defect correction: an inner solve stops no lower
                        // than inner_floor * tau
    double best;        // defect correction: smallest inner change so far
    int since;          // defect correction: inner sweeps since it
    double mass_target; // defect correction: exact sum of the correction,
                        // sum(r) / (1-d), in true units
    double shift;       // fused defect correction: e += shift * Y64 pending
                        // (stored units), set by the sweep's last block
    unsigned int shift_ticket;  // blocks of the shift kernel done
    double *history;
    // loop perforation (Jacobi): sweep k is full when k == 0 or
    // (perf_period > 0 and k % perf_period == 0); a perforated sweep skips a
    // vertex whose last change was below perf_eps times its value
    int perf;                   // 1: perforated solve
    int perf_period;
    double perf_eps;
    unsigned long long gathered;  // in-list entries summed (perforated solves)
};

// Work decomposition of a sweep in the degree-ordered ids (in-degree
// descending, so the in-degree classes are contiguous ranges):
//   hubs  [0, nhub)               in-degree > t_hub: segments of hub_seg
//                                 in-edges, one warp each
//   mid   [nhub, nhub + nmid)     t_lo < in-degree <= t_hub: four sub-ranges
//                                 [mb[k], mb[k+1]) of 32 >> k lanes per vertex
//                                 (in-degree > mid_wide, > mid_wide / 2,
//                                 > mid_wide / 4, the rest)
//   low   [nhub + nmid, n)        in-degree <= t_lo: tiles of consecutive
//                                 vertices with at most tile_c units of work
//                                 (in-edges + vertices), one warp each
struct Items {
    int32_t t_lo = -1, t_hub = -1, hub_seg = 0, tile_c = 0, mid_wide = 0;
    int32_t nhub = 0, nmid = 0, nlow = 0;
    int32_t nhubseg = 0;          // hub segments
    int32_t mb[5] = {0, 0, 0, 0, 0};  // mid sub-range bounds
    int32_t mi[5] = {0, 0, 0, 0, 0};  // mid items before each sub-range
    int32_t nlt = 0;              // low tiles
    int32_t lcap = 0;             // largest in-edge count of a low tile (+ slack)
    int32_t stage_kb = 0;         // shared-memory copy of the hottest sources
                                  // (KB; <= 0: none)
    int32_t wait_limit = 0;       // copy-barrier polls before a timeout (0: default)
    int32_t test_stall = 0;       // testing only (FUSEDPR_TEST_STALL): force the
                                  // timeout path
    int32_t fused_split = 0;      // fused sweep launches (pr_tune.fused_split)
    Buf hubseg_start;             // [nhub + 1] first segment of each hub
    Buf seg_acc;                  // [nhubseg] double partial sums
    Buf hub_cnt;                  // [nhub] segments finished this sweep
    Buf desc;                     // [nhubseg + mi[4] + nlt] int4: hub
                                  // segments {hub, 0, ea, eb}, then mid
                                  // groups and low tiles {v0, v1, ea, eb}:
                                  // vertices [v0, v1), in-list slots [ea, eb)
};

}  // namespace fpr

// Opaque handle of the C ABI.
struct pr_graph {
    int device = 0;
    int num_sms = 0;
    int max_smem = 0;  // opt-in dynamic shared memory per block (bytes)
    int32_t n = 0;
    int64_t m = 0;     // edges of the graph (after PR_DEDUP)
    int64_t m_in = 0;  // edges of the input list (pr_graph_create's m)
    int32_t n_dangling = 0;
    fpr::Mem mem;
    std::vector<fpr::Buf *> owned;

    // build products in the input ids
    fpr::Buf outdeg, indeg, col_ptr, row_idx, csc_eid;
    fpr::Buf row_ptr, col_idx, csr_eid;  // out-lists (lazy)
    fpr::Buf inv64;                      // 1/outdeg (0 for dangling)
    // degree-ordered ids used by the sweeps (r_ = relabelled)
    fpr::Buf n2o, o2n;                   // new -> old, old -> new
    fpr::Buf r_outdeg, r_col_ptr, r_row_idx, r_csc_eid, r_inv64, r_inv32;
    fpr::Items items;
    pr_tune tune{};

    // weighted graphs: raw weights, row sums (input ids) and P per
    // relabelled in-list slot
    bool weighted = false;
    fpr::Buf w, rowsum, p64_csc, p32_csc;

    // solve workspace (grown on demand)
    fpr::Buf ybuf;      // 2 x n x 8 bytes: stored vectors
    fpr::Buf xbuf;      // n doubles: FP64 iterate for defect correction
    fpr::Buf rbuf;      // n x 8 bytes: residual / right-hand side
    fpr::Buf state;     // SolveState
    fpr::Buf aux;       // scratch for batched / multi / adjoint
    fpr::Buf lastbuf;   // perforated solves: last change per vertex

    // batched personalised PageRank: hub segments of the row gather
    // (vertices [0, bnhub) with more than BATCH_SEG in-edges), iterates and
    // per-column state
    int32_t bnhub = -1, bnseg = 0;
    fpr::Buf bseg_start, bseg_cnt, bseg_desc;
    fpr::Buf bx0, bx1, bpart, bcols, btele;
    fpr::SolveState *host_state = nullptr;  // pinned mirror

    // reverse mode: the graph with every edge reversed (its in-lists are
    // this graph's out-lists), built on the first pr_backward, and
    // P_uv = w_uv / s_u per slot of its degree-ordered in-lists
    pr_graph *rev = nullptr;
    fpr::Buf adj_p64, adj_p32;  // P_uv per reversed slot
    fpr::Buf adj_s;             // s_u (sum of u's raw out-weights) per reversed id

    // cached CUDA graphs of the solve loop
    struct Cached {
        int key = -1;
        cudaGraphExec_t exec = nullptr;
        cudaGraph_t graph = nullptr;
    };
    std::vector<Cached> graphs;
};

namespace fpr {

pr_status buf_alloc(pr_graph *g, Buf &b, size_t bytes, cudaStream_t s);
void buf_free(pr_graph *g, Buf &b, cudaStream_t s);
pr_status ensure_items(pr_graph *g, const pr_tune &t, cudaStream_t s);
pr_status ensure_csr(pr_graph *g, cudaStream_t s);
pr_tune effective_tune(const pr_graph *g, const pr_tune *t);
int test_stall_requested();
void release_graphs(pr_graph *g);

// exclusive scan of `count` int32 values; out[count] receives the total.
pr_status scan_exclusive(pr_graph *g, const int32_t *in, int32_t *out, int64_t count,
                         cudaStream_t s);
// stable LSD radix sort of (key, value) pairs by the 8-bit digits at `shifts`
// (alt_k/alt_v: same-size scratch).  With kres/vres the result stays where
// the last pass put it (keys/vals or alt_k/alt_v) and they receive it; else
// it is copied back into keys/vals.
pr_status radix_sort(pr_graph *g, uint64_t *keys, int32_t *vals, uint64_t *alt_k, int32_t *alt_v,
                     int64_t m, const std::vector<int> &shifts, cudaStream_t s,
                     uint64_t **kres = nullptr, int32_t **vres = nullptr);
// digit shifts covering ids < n, starting at bit `offset`
std::vector<int> digit_shifts(int32_t n, int offset);

// primitives.cu kernels launched by the graph assembly
__global__ void k_run_degrees(int64_t m, const uint64_t *__restrict__ keys, int high,
                              int32_t *deg, int32_t *low32);
__global__ void k_make_csc_keys(int64_t m, const int32_t *__restrict__ src,
                                const int32_t *__restrict__ dst, int32_t n, uint64_t *keys,
                                int32_t *vals, int32_t *err);
__global__ void k_make_csr_keys(int32_t n, const int32_t *__restrict__ col_ptr,
                                const int32_t *__restrict__ row_idx,
                                const int32_t *__restrict__ csc_eid, uint64_t *keys, int32_t *vals);
__global__ void k_split_csr(int64_t m, const uint64_t *__restrict__ keys, int32_t *col_idx);
const char *last_error();

// ------------------------------------------------------------ device side --
__device__ __forceinline__ double warp_sum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

// Adds p (|p| < 2^20) into a two-word fixed-point accumulator: the integer
// part of p * 2^40 and the remaining fraction scaled by a further 2^40
// (truncated below 2^-80).  Integer addition is associative, so totals do not
// depend on the order in which blocks finish; up to 2^23 terms fit.
__device__ __forceinline__ void fx_add(long long *hi, long long *lo, double p)
{
    double t = p * 1099511627776.0;  // 2^40, exact
    double h = floor(t);
    double f = t - h;                // exact, in [0, 1)
    atomicAdd(reinterpret_cast<unsigned long long *>(hi),
              static_cast<unsigned long long>(static_cast<long long>(h)));
    atomicAdd(reinterpret_cast<unsigned long long *>(lo),
              static_cast<unsigned long long>(static_cast<long long>(f * 1099511627776.0)));
}
__device__ __forceinline__ double fx_value(long long hi, long long lo)
{
    return static_cast<double>(hi) * 9.094947017729282e-13 +   // 2^-40
           static_cast<double>(lo) * 8.271806125530277e-25;    // 2^-80
}

}  // namespace fpr
