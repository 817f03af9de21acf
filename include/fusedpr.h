/*
 * fusedpr.h -- C ABI of the GB300 fused PageRank library (libfusedpr.so).
 *
 * Problem (the paper's Sec. 3 and Eq. 1): a directed graph G(V, E) given as a
 * list of (u, v) tuples, each an out-link of u and an in-link of v; the
 * PageRank vector solves
 *     pr_u = (1-d)/n + d * ( sum_{v in inlink(u)} pr_v / d_o(v) + D/n ),
 * where D is the rank held by dangling vertices (out-degree 0), spread
 * uniformly (the paper's Eq. 1 has no dangling term; this library adds the
 * uniform redistribution and normalises the result to sum 1).  Two sweeps:
 *   PR_JACOBI    Algorithm 1 / Eq. 2: every vertex reads the previous sweep.
 *   PR_FUSED_GS  Algorithm 2 / Eq. 9 (FusEd-PageRank): a vertex's new
 *                contribution is written immediately and later readers in the
 *                same sweep may see it (asynchronous Gauss-Seidel, as the
 *                paper's parallel version).  Each sweep is followed by a
 *                rescale to sum 1, folded into the next sweep as a scalar.
 * Stop rule (Algorithm 1/2 `while error > threshold`, Eq. 3): the L1 (or
 * max) distance between successive iterates; a sweep whose error is <= the
 * threshold ends the solve.
 *
 * Conventions for every call:
 *   - Pointers documented "device" are CUDA device pointers on the current
 *     device; "host" pointers are ordinary host memory.  Inputs are only read
 *     and stay owned by the caller; outputs are caller-allocated.
 *   - All device work is ordered on `stream` (a cudaStream_t, NULL = legacy
 *     default stream).  Calls return after their result scalars are on the
 *     host (one stream synchronisation), so device outputs are complete too.
 *   - Every call returns a pr_status; nothing aborts or traps.  Device-side
 *     errors (bad vertex ids, timeouts) come back through status words.
 *     pr_last_error() gives a readable message for the calling thread.
 *   - Indices are int32 (n < 2^31); edge counts are int64 but must be
 *     < 2^31 (offsets are int32).
 *   - There is no CPU fallback: without a usable CUDA device every call
 *     returns PR_ERR_CUDA.
 */
#ifndef FUSEDPR_H
#define FUSEDPR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pr_graph pr_graph; /* opaque; owns its device buffers */

typedef enum {
    PR_OK = 0,
    PR_ERR_INVALID_ARG = 1, /* bad argument or vertex id (device-checked) */
    PR_ERR_OOM = 2,         /* allocation failed (allocator or CUDA) */
    PR_ERR_CUDA = 3,        /* CUDA runtime error; see pr_last_error() */
    PR_NOT_CONVERGED = 4,   /* max_iter reached; outputs hold the last iterate */
    PR_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    PR_ERR_UNSUPPORTED = 6, /* option combination not implemented */
    PR_ERR_NUMERIC = 7      /* a non-finite value appeared in the iterate */
} pr_status;

typedef enum { PR_JACOBI = 0, PR_FUSED_GS = 1 } pr_variant;

/* Arithmetic of the sweep.  *_DC forms run the cheap sweep on a correction
 * and recompute the residual in FP64 between inner solves (defect
 * correction); the stop value is then the FP64 residual
 * || (1-d)/n + d M x - x ||_1.  The correction is stored in FP32, BF16 or
 * FP16 (FP16 scaled by a power of two that keeps every entry below 2^14)
 * with FP32 accumulation. */
typedef enum {
    PR_FP64 = 0,
    PR_FP32 = 1,
    PR_FP32_DC = 2,
    PR_BF16_DC = 3,
    PR_FP16_DC = 4
} pr_precision;

typedef enum { PR_NORM_L1 = 0, PR_NORM_LINF = 1 } pr_norm;

/* Device allocator hooks (e.g. a framework's caching allocator).  alloc
 * returns a device pointer of at least `bytes` usable on `stream`, or NULL;
 * free releases it.  When the pr_allocator pointer passed to
 * pr_graph_create is NULL the library allocates stream-ordered from its own
 * memory pool of the device (cudaMallocFromPoolAsync/cudaFreeAsync), which
 * keeps freed memory for later builds and solves until the process exits,
 * like a caching allocator. */
typedef struct {
    void *(*alloc)(size_t bytes, void *stream, void *ctx);
    void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
    void *ctx;
} pr_allocator;

/* Launch parameters of the sweep (chosen by the autotuner; zero fields take
 * the library defaults).  The sweep works in a degree-ordered numbering
 * (in-degree descending), where the in-degree bins are contiguous. */
typedef struct {
    int32_t t_lo;      /* in-degree <= t_lo: low-degree tiles, one lane per
                          vertex (default 32, at most 32) */
    int32_t t_hub;     /* in-degree >  t_hub: hub, split into segments of
                          hub_seg in-edges, a warp per segment (default
                          4096); in between: 4 to 32 lanes per vertex */
    int32_t hub_seg;   /* in-edges per hub segment (default 2048, 256 to
                          8192) */
    int32_t tile;      /* work units (in-edges + vertices) per low-degree
                          tile, whose in-edges a warp gathers into shared
                          memory (default 256, 32 to 512) */
    int32_t deterministic_gs; /* 1: fused sweep in strict input id order on
                                 one warp (reproduces Eq. 9; n <= 65536) */
    int32_t stage_kb;  /* shared memory (KB) per block for a copy of the
                          stored vector's first entries, the most-gathered
                          contributions in the degree-ordered ids (0:
                          the default, 64; -1: none; > 0: that many KB, at
                          most the room the tiles leave) */
    int32_t wait_limit;/* polls of a copy barrier before a device-side wait
                          gives up with PR_ERR_TIMEOUT (0: 4M) */
    int32_t fused_split; /* launches of one fused sweep: 0 (default) or 1
                          two (the hub segments and the widest mid groups
                          first, so the rest reads their new values; with a
                          4- or 2-byte stored vector the first launch writes
                          its new values aside and they are copied in
                          before the second), 2 one.  Changes which values
                          a fused sweep reads fresh, hence its sweep count,
                          not the fixed point. */
    int32_t mid_wide;  /* mid vertices (t_lo < in-degree <= t_hub) get 32
                          lanes above mid_wide in-edges, 16 above
                          mid_wide / 2, 8 above mid_wide / 4 and 4 below
                          (default 1024; 16 to 2^20) */
    int32_t blocking;  /* 1: Jacobi sweeps (PR_FP64 / PR_FP32, unweighted, no
                          perforation) run propagation-blocked: contributions
                          scattered into bins of 16384 destinations, then
                          summed per bin in shared memory (the locality
                          technique the paper's related work cites for
                          vectors that do not fit in cache; built on first
                          use, about 20 bytes per edge).  Sums are added with
                          atomics, so results vary at rounding level.  0
                          (default): the in-list gather sweep. */
} pr_tune;

typedef struct {
    double d;               /* damping factor, 0 <= d < 1 (paper: 0.85) */
    double threshold;       /* stop when the sweep error <= threshold */
    int32_t max_iter;       /* >= 1; sweeps (inner sweeps for *_DC) */
    pr_variant variant;
    pr_precision precision;
    pr_norm norm;           /* error of a sweep: L1 or max norm (Eq. 3) */
    const double *x0;       /* device [n] start vector (sum 1) or NULL: 1/n */
    double *history;        /* device [max_iter] per-sweep error or NULL */
    int32_t use_graph;      /* 1 (default): CUDA-graph loop with the stop test
                               on the device; 0: host-driven loop */
    int32_t max_outer;      /* *_DC: max FP64 residual evaluations (default 8) */
    double inner_rel;       /* *_DC: inner stop, relative to ||r||_1 (0: auto:
                               FP32 1e-5 Jacobi / 3e-5 fused, FP16 and BF16
                               1e-2); an inner solve also stops once its
                               change has not fallen for 8 sweeps */
    const pr_tune *tune;    /* NULL: the graph's defaults */
    int32_t no_rescale;     /* PR_FUSED_GS with PR_FP64 / PR_FP32: 1 runs the
                               literal Algorithm 2, with no rescale of the
                               iterate to sum 1 after each sweep (the result
                               is still normalised once at the end); 0
                               (default) rescales.  Ignored by Jacobi and the
                               *_DC forms. */
    double perforate_eps;   /* > 0: loop-perforated Jacobi (the loop perforation
                               the paper's related work and conclusion name;
                               PR_JACOBI, PR_FP64 / PR_FP32, unweighted): in a
                               perforated sweep a vertex whose change at its
                               last computation was below perforate_eps times
                               its value keeps that value and its in-edges are
                               not gathered.  0 (default): plain Jacobi. */
    int32_t perforate_period; /* with perforate_eps > 0: sweep k (from 0) is a
                               full Jacobi sweep when k == 0 or k is a multiple
                               of perforate_period, and only full sweeps can
                               stop (the stop rule's bound then holds); 0: no
                               forced full sweeps, any sweep can stop (an
                               approximate result: skipped vertices count as
                               unchanged in the error). */
} pr_options;

typedef struct {
    int32_t iters;          /* sweeps run (all inner sweeps for *_DC) */
    int32_t outer_iters;    /* FP64 residual evaluations (*_DC), else 0 */
    double residual;        /* final stop value */
    double sum_before_norm; /* sum of the iterate before the final x /= sum */
    pr_status status;
    int64_t gathered;       /* pr_solve: in-list entries summed by its sweeps
                               (inner, and FP64 residual sweeps for *_DC;
                               fewer than sweeps x m when perforated) */
} pr_result;

/* Fills `o` with the defaults: d 0.85, threshold 1e-10, max_iter 1000,
 * Jacobi, FP64, L1, no x0/history, CUDA-graph loop. */
pr_status pr_options_default(pr_options *o);

/*
 * Builds the graph on the device from an edge list (Sec. 3 storage):
 * out/in-degree histograms, the in-lists (CSC: column u = sources of u's
 * in-edges, ascending, ties by input position), inverse out-degrees
 * (IEEE 1.0/deg, 0 for dangling), and the sweep's working copy in a
 * degree-ordered numbering: vertices sorted by in-degree, largest first (ties
 * by id), each in-list kept in its input-id order with its sources renamed
 * to the new ids.  That puts the in-degree bins in
 * contiguous ranges and packs the most-gathered contributions together.
 * Results of every solve are returned in the input ids.
 *   n       vertices, >= 1
 *   m       edges, 0 <= m < 2^31
 *   src,dst int32 [m] in device (or managed) memory, or in page-locked host
 *           memory, which the build reads once over the host link (no
 *           separate copy); pageable host memory is refused
 *           (PR_ERR_INVALID_ARG).  Ids must lie in [0, n) (checked on the
 *           device: PR_ERR_INVALID_ARG otherwise).  Self-loops and repeated
 *           edges are kept as ordinary edges.
 *   w       float [m] raw positive edge weights (same memory rules), or NULL
 *           (unweighted).
 *           Weighted graphs use P_uv = w_uv / sum_v' w_uv'.
 *   flags   PR_BUILD_CSR also builds the out-lists (needed by pr_backward;
 *           built lazily otherwise).  PR_DEDUP keeps only the first
 *           occurrence (lowest input position) of each repeated (u, v) pair
 *           (the paper's workloads are simple graphs, Sec. 5.2); the graph's
 *           edge count (pr_graph_info, the exported lists) is then the number
 *           kept, csc_eid/csr_eid still give input positions, weights of
 *           dropped edges are ignored and their pr_backward gradient is 0.
 *           Without it repeated edges count with multiplicity.
 *   alloc   allocator hooks or NULL (the library's pool); kept by the graph.
 *   out     receives the handle (NULL on error).
 */
#define PR_BUILD_CSR 1u
#define PR_DEDUP 2u
pr_status pr_graph_create(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                          const float *w, uint32_t flags, const pr_allocator *alloc,
                          void *stream, pr_graph **out);

/* Releases the graph and its buffers (NULL is ignored). */
void pr_graph_destroy(pr_graph *g);

/* Host outputs (each nullable): vertex and edge counts, dangling vertices,
 * and the sizes of the low/mid/hub in-degree bins under the graph's current
 * thresholds (low: in-degree <= t_lo, hub: > t_hub). */
pr_status pr_graph_info(const pr_graph *g, int32_t *n, int64_t *m, int32_t *n_dangling,
                        int32_t *bin_counts3);

/*
 * Copies the build products to caller device buffers (each nullable), for
 * bit-exact checks: outdeg/indeg [n], col_ptr/row_ptr [n+1], row_idx/csc_eid
 * [m] (in-lists), col_idx/csr_eid [m] (out-lists, ordered by (dst, input
 * position); built on demand), inv_outdeg [n] (FP64); the degree-ordered
 * numbering: new_to_old [n], rcol_ptr [n+1], rrow_idx [m] (the in-list of
 * new vertex k is the input-id in-list of new_to_old[k], in the same order,
 * with its sources renamed to new ids).
 */
pr_status pr_graph_export(pr_graph *g, int32_t *outdeg, int32_t *indeg, int32_t *col_ptr,
                          int32_t *row_idx, int32_t *csc_eid, int32_t *row_ptr,
                          int32_t *col_idx, int32_t *csr_eid, double *inv_outdeg,
                          int32_t *new_to_old, int32_t *rcol_ptr, int32_t *rrow_idx,
                          void *stream);

/*
 * Solves for the PageRank vector.
 *   x_out  device double [n]: the result, normalised to sum 1.
 *   res    host, nullable: sweeps, stop value, status.
 * Returns PR_OK, PR_NOT_CONVERGED (x_out holds the last iterate,
 * normalised), or an error.
 */
pr_status pr_solve(pr_graph *g, const pr_options *o, double *x_out, pr_result *res,
                   void *stream);

/*
 * Personalised PageRank for B teleport vectors at once (multi right-hand
 * side sweep): Eq. 1 with the uniform teleport (1-d)/n replaced by
 * (1-d) v_b for each column b.  Either seeds (column b teleports to the
 * single vertex seeds[b]) or V (dense teleport vectors) is given, not both;
 * a column's dangling mass is redistributed along its own teleport vector,
 * so every column sums to 1.  Jacobi sweep in FP32 or FP64 (o->precision
 * PR_FP32 or PR_FP64, o->variant PR_JACOBI, L1 norm); each column stops on
 * its own L1 change and keeps that iterate.  An FP32 column whose change
 * stops decreasing above the threshold (its rounding floor) stops too, with
 * status PR_NOT_CONVERGED.  Start vector 1/n.
 *   seeds  device int32 [B], ids in [0, n), or NULL
 *   V      device [n][B] (vertex-major, column b at stride B) of float for
 *          PR_FP32 or double for PR_FP64, or NULL: teleport vectors, entries
 *          finite and >= 0 (PR_ERR_INVALID_ARG otherwise), each column
 *          summing to 1 (not checked; a column with another sum S solves the
 *          problem with teleport mass S(1-d))
 *   X_out  device [n][B] (same layout and type as V): each column
 *          normalised to sum 1
 *   res    host [B], nullable: per-column sweeps, last change, status
 * Returns PR_OK if every column converged, else PR_NOT_CONVERGED (outputs
 * still written) or an error.  Columns run in passes of at most 256 (FP32)
 * or 128 (FP64); the handle keeps two n x pass-width iterates (and the
 * pass's teleport rows when V is given).
 */
pr_status pr_solve_batched(pr_graph *g, const pr_options *o, int32_t B, const int32_t *seeds,
                           const void *V, void *X_out, pr_result *res, void *stream);

/*
 * Solves G independent graphs in one sequence of launches (each sweep is one
 * kernel over the work items of every graph that has not converged yet):
 * Algorithm 1 (PR_JACOBI) or Algorithm 2 / Eq. 9 (PR_FUSED_GS, in place,
 * rescaled after each sweep unless o->no_rescale) per graph, with each
 * graph's own stop rule.
 *   graphs  host [G] handles (distinct, on one device)
 *   x_out   host [G] array of device double pointers, x_out[i] of size n_i
 *   res     host [G], nullable
 * o->precision must be PR_FP64 or PR_FP32, o->x0 NULL, no perforation
 * (PR_ERR_UNSUPPORTED otherwise).
 */
pr_status pr_solve_multi(pr_graph *const *graphs, int32_t G, const pr_options *o,
                         double *const *x_out, pr_result *res, void *stream);

/*
 * Reverse mode of pr_solve at its fixed point (the paper has no gradients:
 * this differentiates the fixed point of Eq. 1, x = (1-d)/n + d M x, with
 * M = P^T + dangling redistribution).  Given x (the forward result)
 * and grad_x = dL/dx, solves the transposed system
 *     (I - d M)^T lambda = grad_x
 * by iteration over the out-lists, then
 *     dL/dw_e = (d x_u / s_u) (lambda_v - sum_v' P_uv' lambda_v')  for e = u->v
 *     dL/dd   = lambda^T (M x - 1/n)
 * (raw weights w with row sums s_u; unweighted graphs use w = 1).
 *   x, grad_x  device double [n]
 *   grad_w     device double [m] in input edge order (m = pr_graph_create's
 *              edge count), or NULL
 *   grad_d     device double [1], or NULL
 * o->threshold applies to the L1 change of lambda per sweep.
 */
pr_status pr_backward(pr_graph *g, const pr_options *o, const double *x, const double *grad_x,
                      double *grad_w, double *grad_d, pr_result *res, void *stream);

/*
 * Exclusive prefix sum of int32 values without any device allocation (the
 * paper has no counterpart: this is the offsets step of the graph build,
 * col_ptr from in-degrees, offered for callers that must not allocate, e.g.
 * inside a memory-capped or preallocated runtime).
 *   in     device int32 [count] (read only; may be NULL if count == 0)
 *   out    device int32 [count + 1]: out[i] = in[0] + ... + in[i-1],
 *          out[count] = the total (sums must fit in int32)
 *   count  0 <= count <= 134217728 (65536 blocks of 2048); larger counts
 *          return PR_ERR_INVALID_ARG before any device work
 * Scratch: the per-block totals live in one fixed 256 KB __device__ array
 * of the library (one copy per device), located once per device with
 * cudaGetSymbolAddress; nothing is allocated or freed.  All calls on a
 * device share that array: calls that overlap in time (on different
 * streams or threads) race and give wrong results, so serialise them.  The
 * first call on a device does the one-time lookup; make it before any
 * stream capture.  Work is ordered on `stream`; the function returns
 * without synchronising.
 */
pr_status pr_scan_exclusive_noalloc(const int32_t *in, int32_t *out, int64_t count,
                                    void *stream);

/* Static string for a status code. */
const char *pr_status_string(pr_status s);

/* Message of the last error raised on the calling thread ("" if none). */
const char *pr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* FUSEDPR_H */
