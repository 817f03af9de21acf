/*
 * oracle.c -- plain, slow, single-threaded FP64 reference of the fused
 * PageRank hot path.  TEST INFRASTRUCTURE ONLY: it exists so that the CUDA
 * library can be checked against something obviously correct.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg may load it;
 * the product path never calls it and shares no code with it.
 *
 * Every routine is the textbook definition or the paper's algorithm written
 * out in the paper's order, with no blocking, fusion or reordering:
 *
 *   orc_build        storage of Sec. 3: out/in degrees, the out-list (CSR,
 *                    the paper's offsetList grouping) and the in-list (CSC,
 *                    the paper's contributionList grouping), inverse
 *                    out-degree.  Two stable counting sorts.
 *   orc_bins         stable partition of vertices by in-degree.
 *   orc_jacobi       Algorithm 1 (edge-centric baseline, Eq. 2) with the
 *                    dangling-mass term added; L1 or max-norm stop (Eq. 3).
 *   orc_gauss_seidel Algorithm 2 (FusEd-PageRank), i.e. Eq. 9 taken in
 *                    increasing vertex id order.
 *   orc_perforated   loop-perforated Jacobi (the loop perforation the paper
 *                    names in its related work and future work): vertices
 *                    of minor importance skip their in-list sums in some
 *                    sweeps.
 *   orc_adjoint      transposed fixed point of the same operator.
 *   orc_gradients    chain rule of the fixed point w.r.t. raw edge weights
 *                    and the damping factor d.
 *   orc_dense_*      dense Google-matrix system for tiny graphs, solved by
 *                    Gaussian elimination with partial pivoting.
 *
 * Readings of the paper that this file fixes (the paper is silent):
 *   - dangling vertices (out-degree 0) spread their rank uniformly (or along
 *     the teleport vector for personalised PageRank); the mass D is taken
 *     from the iterate at the start of the sweep;
 *   - the contribution of v is x_v * inv_outdeg[v] with inv_outdeg = 1.0/deg
 *     rounded once (a multiply, not a divide, per sweep);
 *   - `while error > threshold` means a sweep whose error is <= tau stops;
 *   - the result is normalised once, at the end (x /= sum x);
 *   - the fused sweep is followed by a rescale to sum 1 (its in-place
 *     updates do not conserve the sum; the fixed point has sum 1, so this
 *     changes the path, not the limit).  Jacobi conserves the sum exactly.
 *
 * Parity status: every function here is pinned by the CPU test suite
 * (closed forms, dense solves cross-checked by numpy, complex-step
 * derivatives, exact rational arithmetic, numpy stable sorts).
 *
 * Compiled with -ffp-contract=off so that no multiply-add is fused and the
 * results are the same on x86-64 and AArch64 hosts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_OOM 2
#define ORC_NOT_CONVERGED 4

/* ------------------------------------------------------------------------ */
/* Graph build (Sec. 3: inList/outList, contributionList, offsetList)        */
/* ------------------------------------------------------------------------ */

/* Stable counting sort of the item sequence `in` (length m) by key[in[i]]
 * with keys in [0, nkeys).  `start` receives the nkeys+1 bucket offsets. */
static int counting_sort(int64_t m, int32_t nkeys, const int32_t *key,
                         const int32_t *in, int32_t *out, int32_t *start)
{
    int64_t *next = (int64_t *)calloc((size_t)nkeys + 1, sizeof(int64_t));
    if (!next) return ORC_ERR_OOM;
    for (int64_t i = 0; i < m; ++i) next[key[in[i]] + 1] += 1;
    for (int32_t k = 0; k < nkeys; ++k) next[k + 1] += next[k];
    if (start)
        for (int32_t k = 0; k <= nkeys; ++k) start[k] = (int32_t)next[k];
    for (int64_t i = 0; i < m; ++i) {
        int32_t e = in[i];
        out[next[key[e]]++] = e;
    }
    free(next);
    return ORC_OK;
}

/*
 * Builds both adjacency layouts of the directed edge list (src[e] -> dst[e]).
 *   CSR  (out-lists): row u holds u's out-edges ordered by (dst, edge id).
 *   CSC  (in-lists):  column u holds u's in-edges ordered by (src, edge id).
 * Duplicate edges and self-loops are kept as ordinary edges.
 * inv_outdeg[u] = 1.0 / outdeg[u] (one IEEE division), 0.0 for dangling u.
 * Returns ORC_ERR_ARG for n < 1, m < 0, m >= 2^31 or an id outside [0, n).
 */
int orc_build(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
              int32_t *outdeg, int32_t *indeg,
              int32_t *row_ptr, int32_t *col_idx, int32_t *csr_eid,
              int32_t *col_ptr, int32_t *row_idx, int32_t *csc_eid,
              double *inv_outdeg)
{
    if (n < 1 || m < 0 || m >= ((int64_t)1 << 31)) return ORC_ERR_ARG;
    for (int64_t e = 0; e < m; ++e)
        if (src[e] < 0 || src[e] >= n || dst[e] < 0 || dst[e] >= n) return ORC_ERR_ARG;

    memset(outdeg, 0, sizeof(int32_t) * (size_t)n);
    memset(indeg, 0, sizeof(int32_t) * (size_t)n);
    for (int64_t e = 0; e < m; ++e) {
        outdeg[src[e]] += 1;
        indeg[dst[e]] += 1;
    }

    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *by_dst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!ids || !by_dst) { free(ids); free(by_dst); return ORC_ERR_OOM; }
    for (int64_t e = 0; e < m; ++e) ids[e] = (int32_t)e;

    /* out-lists: sort by dst (ties by id), then stably by src. */
    int rc = counting_sort(m, n, dst, ids, by_dst, NULL);
    if (rc == ORC_OK) rc = counting_sort(m, n, src, by_dst, csr_eid, row_ptr);
    if (rc == ORC_OK)
        for (int64_t p = 0; p < m; ++p) col_idx[p] = dst[csr_eid[p]];
    /* in-lists: the out-list stream (src, dst, id) sorted stably by dst. */
    if (rc == ORC_OK) rc = counting_sort(m, n, dst, csr_eid, csc_eid, col_ptr);
    if (rc == ORC_OK)
        for (int64_t q = 0; q < m; ++q) row_idx[q] = src[csc_eid[q]];
    free(ids);
    free(by_dst);
    if (rc != ORC_OK) return rc;

    for (int32_t u = 0; u < n; ++u)
        inv_outdeg[u] = outdeg[u] > 0 ? 1.0 / (double)outdeg[u] : 0.0;
    return ORC_OK;
}

/*
 * Degree-ordered relabelling used by the GPU sweep (an internal order; the
 * results are returned in the original ids).  new_to_old lists the vertices
 * by in-degree, largest first, ties in increasing id (a stable sort); the
 * relabelled in-lists hold, for new column u' = old vertex new_to_old[u'],
 * the new ids of its in-neighbours in ascending new id, ties by edge id.
 * rcol_ptr has n+1 entries, rrow_idx and rcsc_eid m each.
 */
int orc_relabel(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                const int32_t *indeg, int32_t *new_to_old, int32_t *rcol_ptr,
                int32_t *rrow_idx, int32_t *rcsc_eid)
{
    int32_t maxd = 0;
    for (int32_t u = 0; u < n; ++u) if (indeg[u] > maxd) maxd = indeg[u];
    /* counting sort of vertex ids by key maxd - indeg (stable) */
    int32_t *key = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *o2n = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *nsrc = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *ndst = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *eids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    int rc = ORC_OK;
    if (!key || !ids || !o2n || !nsrc || !ndst || !eids || !tmp) rc = ORC_ERR_OOM;
    if (rc == ORC_OK) {
        for (int32_t u = 0; u < n; ++u) { key[u] = maxd - indeg[u]; ids[u] = u; }
        rc = counting_sort(n, maxd + 1, key, ids, new_to_old, NULL);
    }
    if (rc == ORC_OK) {
        for (int32_t k = 0; k < n; ++k) o2n[new_to_old[k]] = k;
        for (int64_t e = 0; e < m; ++e) {
            nsrc[e] = o2n[src[e]];
            ndst[e] = o2n[dst[e]];
            eids[e] = (int32_t)e;
        }
        /* in-lists by (new dst, input src, edge id): each new in-list is
         * the input-id in-list of the same vertex, in the same order, with
         * its sources renamed: sort by input src, then stably by new dst */
        rc = counting_sort(m, n, src, eids, tmp, NULL);
    }
    if (rc == ORC_OK) rc = counting_sort(m, n, ndst, tmp, rcsc_eid, rcol_ptr);
    if (rc == ORC_OK)
        for (int64_t q = 0; q < m; ++q) rrow_idx[q] = nsrc[rcsc_eid[q]];
    free(key); free(ids); free(o2n); free(nsrc); free(ndst); free(eids); free(tmp);
    return rc;
}

/* Stable partition of vertex ids by in-degree: low (<= t_lo), mid
 * (t_lo < deg <= t_hub) and hub (> t_hub), each list in ascending id order.
 * counts[0..2] receive the list lengths. */
void orc_bins(int32_t n, const int32_t *indeg, int32_t t_lo, int32_t t_hub,
              int32_t *low, int32_t *mid, int32_t *hub, int32_t *counts)
{
    int32_t a = 0, b = 0, c = 0;
    for (int32_t u = 0; u < n; ++u) {
        if (indeg[u] <= t_lo) low[a++] = u;
        else if (indeg[u] <= t_hub) mid[b++] = u;
        else hub[c++] = u;
    }
    counts[0] = a;
    counts[1] = b;
    counts[2] = c;
}

/* ------------------------------------------------------------------------ */
/* Stationary PageRank iterations                                           */
/* ------------------------------------------------------------------------ */
/*
 * Both iterations below solve  x = r + d * M x,  M = P^T + w * a^T, where
 *   P_vu  = inv_outdeg[v]          (unweighted)   or csc_p[slot] (weighted),
 *   a     = indicator of dangling vertices (outdeg == 0),
 *   w     = uniform 1/n            (tele == NULL or dangling_along_tele == 0)
 *           or the teleport vector (dangling_along_tele != 0),
 *   r     = (1-d)/n                (tele == NULL, Eq. 1/Eq. 2)
 *           or (1-d) * tele        (personalised PageRank),
 *   rhs   when given, replaces r entirely (used for correction solves).
 */
typedef struct {
    int32_t n;
    const int32_t *col_ptr, *row_idx, *outdeg;
    const double *inv_outdeg, *csc_p;
    double d;
    const double *tele, *rhs;
    int32_t dangling_along_tele;
} orc_problem;

static double r_of(const orc_problem *p, int32_t u, double base)
{
    if (p->rhs) return p->rhs[u];
    if (p->tele) return (1.0 - p->d) * p->tele[u];
    return base;
}

static double w_of(const orc_problem *p, int32_t u, double inv_n)
{
    if (p->tele && p->dangling_along_tele) return p->tele[u];
    return inv_n;
}

/*
 * Global sums over all vertices (the dangling mass D, the total sum x, the L1
 * error of a sweep) are exact sums in the method.  A plain running sum of n
 * terms carries up to (n-1) eps of rounding, and on R-MAT graphs that error is
 * biased (4e-13 at n = 65536), so these sums are compensated (Neumaier's
 * variant of Kahan summation; error about 2 eps, independent of n).  The short
 * per-vertex in-list sums stay plain running sums, as in the algorithms.
 */
typedef struct { double s, c; } ksum;

static void ks_add(ksum *k, double v)
{
    double t = k->s + v;
    if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
    else k->c += (v - t) + k->s;
    k->s = t;
}

static double ks_get(const ksum *k) { return k->s + k->c; }

static double dangling_mass(const orc_problem *p, const double *x)
{
    ksum D = {0.0, 0.0};
    for (int32_t u = 0; u < p->n; ++u)
        if (p->outdeg[u] == 0) ks_add(&D, x[u]);
    return ks_get(&D);
}

static double total(const double *x, int32_t n)
{
    ksum s = {0.0, 0.0};
    for (int32_t u = 0; u < n; ++u) ks_add(&s, x[u]);
    return ks_get(&s);
}

/*
 * One Jacobi sweep (Algorithm 1, phase 1 then phase 2):
 *   phase 1: contribution c_v = x_v * inv_outdeg[v]            (unweighted)
 *   phase 2: x'_u = r_u + d * (sum_{v in inlink(u)} c_v + D * w_u)
 * For weighted graphs the in-edge term is csc_p[slot] * x_v.
 * Returns the L1 (norm 0) or max (norm 1) distance between x' and x.
 */
static double jacobi_sweep(const orc_problem *p, const double *x, double *xn, double *c,
                           int32_t norm)
{
    const int32_t n = p->n;
    const double base = (1.0 - p->d) / (double)n;
    const double inv_n = 1.0 / (double)n;
    const double D = dangling_mass(p, x);
    if (!p->csc_p)
        for (int32_t v = 0; v < n; ++v) c[v] = x[v] * p->inv_outdeg[v];
    ksum l1 = {0.0, 0.0};
    double mx = 0.0;
    for (int32_t u = 0; u < n; ++u) {
        double sum = 0.0;
        for (int32_t q = p->col_ptr[u]; q < p->col_ptr[u + 1]; ++q) {
            int32_t v = p->row_idx[q];
            sum += p->csc_p ? p->csc_p[q] * x[v] : c[v];
        }
        xn[u] = r_of(p, u, base) + p->d * (sum + D * w_of(p, u, inv_n));
        double diff = fabs(xn[u] - x[u]);
        ks_add(&l1, diff);
        if (diff > mx) mx = diff;
    }
    return norm == 0 ? ks_get(&l1) : mx;
}

/*
 * One sequential fused sweep (Algorithm 2 / Eq. 9): vertices in increasing id
 * order; each reads the contribution list as it stands (already rewritten for
 * in-neighbours j < i, old for j >= i including a self-loop), computes its new
 * rank and immediately rewrites its own contribution.  D is the dangling mass
 * at the start of the sweep.  The error compares each new rank with the
 * (normalised) rank it replaces.  The caller renormalises after the sweep.
 */
static double gs_sweep(const orc_problem *p, double *x, double *c, int32_t norm)
{
    const int32_t n = p->n;
    const double base = (1.0 - p->d) / (double)n;
    const double inv_n = 1.0 / (double)n;
    const double D = dangling_mass(p, x);
    ksum l1 = {0.0, 0.0};
    double mx = 0.0;
    for (int32_t u = 0; u < n; ++u) {
        double prev = x[u];
        double sum = 0.0;
        for (int32_t q = p->col_ptr[u]; q < p->col_ptr[u + 1]; ++q) {
            int32_t v = p->row_idx[q];
            sum += p->csc_p ? p->csc_p[q] * x[v] : c[v];
        }
        x[u] = r_of(p, u, base) + p->d * (sum + D * w_of(p, u, inv_n));
        if (!p->csc_p) c[u] = x[u] * p->inv_outdeg[u];
        double diff = fabs(x[u] - prev);
        ks_add(&l1, diff);
        if (diff > mx) mx = diff;
    }
    return norm == 0 ? ks_get(&l1) : mx;
}

/*
 * Runs Jacobi (gs == 0) or sequential fused Gauss-Seidel (gs != 0; with
 * renorm != 0 each sweep is followed by x /= sum x) from x0
 * (NULL: uniform 1/n, as in Algorithms 1 and 2) until a sweep's error is
 * <= tau or max_iter sweeps have run.  err_hist (nullable, max_iter slots)
 * receives each sweep's error.  With normalize != 0 the result is divided by
 * its sum, which is reported in *sum_before.
 */
static int run_iteration(const orc_problem *p, int gs, int renorm, const double *x0, double tau,
                         int32_t max_iter, int32_t norm, int32_t normalize, double *x_out,
                         int32_t *iters, double *err_last, double *err_hist, double *sum_before)
{
    const int32_t n = p->n;
    if (n < 1 || max_iter < 0) return ORC_ERR_ARG;
    double *x = x_out;
    double *xn = (double *)malloc(sizeof(double) * (size_t)n);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xn || !c) { free(xn); free(c); return ORC_ERR_OOM; }
    for (int32_t u = 0; u < n; ++u) x[u] = x0 ? x0[u] : 1.0 / (double)n;
    if (gs && !p->csc_p)
        for (int32_t v = 0; v < n; ++v) c[v] = x[v] * p->inv_outdeg[v];

    int32_t k = 0;
    double err = INFINITY;
    int converged = 0;
    while (k < max_iter) {
        if (gs) {
            /* In-place updates do not conserve sum(x) (some in-neighbours read
             * the new contribution, some the old), and that drift decays
             * slowly.  The fixed point has sum 1, so each sweep ends by
             * rescaling to sum 1; Jacobi conserves the sum exactly and is left
             * alone until the end. */
            err = gs_sweep(p, x, c, norm);
            if (renorm && p->rhs == NULL) {
                const double s = total(x, n);
                for (int32_t u = 0; u < n; ++u) x[u] = x[u] / s;
                if (!p->csc_p)
                    for (int32_t v = 0; v < n; ++v) c[v] = x[v] * p->inv_outdeg[v];
            }
        } else {
            err = jacobi_sweep(p, x, xn, c, norm);
            memcpy(x, xn, sizeof(double) * (size_t)n);
        }
        if (err_hist) err_hist[k] = err;
        ++k;
        if (err <= tau) { converged = 1; break; }
    }
    const double s = total(x, n);
    if (sum_before) *sum_before = s;
    if (normalize)
        for (int32_t u = 0; u < n; ++u) x[u] = x[u] / s;
    *iters = k;
    *err_last = err;
    free(xn);
    free(c);
    return converged ? ORC_OK : ORC_NOT_CONVERGED;
}

#define PROBLEM_ARGS                                                                       \
    int32_t n, const int32_t *col_ptr, const int32_t *row_idx, const int32_t *outdeg,      \
        const double *inv_outdeg, const double *csc_p, double d, const double *tele,        \
        const double *rhs, int32_t dangling_along_tele
#define MAKE_PROBLEM                                                                        \
    orc_problem p = {n, col_ptr, row_idx, outdeg, inv_outdeg, csc_p, d, tele, rhs,          \
                     dangling_along_tele}

int orc_jacobi(PROBLEM_ARGS, const double *x0, double tau, int32_t max_iter, int32_t norm,
               int32_t normalize, double *x_out, int32_t *iters, double *err_last,
               double *err_hist, double *sum_before)
{
    MAKE_PROBLEM;
    return run_iteration(&p, 0, 0, x0, tau, max_iter, norm, normalize, x_out, iters, err_last,
                         err_hist, sum_before);
}

int orc_gauss_seidel(PROBLEM_ARGS, int32_t renorm, const double *x0, double tau,
                     int32_t max_iter, int32_t norm, int32_t normalize, double *x_out,
                     int32_t *iters, double *err_last, double *err_hist, double *sum_before)
{
    MAKE_PROBLEM;
    return run_iteration(&p, 1, renorm, x0, tau, max_iter, norm, normalize, x_out, iters,
                         err_last, err_hist, sum_before);
}

/*
 * Loop-perforated Jacobi.  The paper names loop perforation (related work:
 * skipping the computations on vertices of minor importance, an approximate
 * computing technique; conclusion: future work) without defining it; the
 * reading implemented here:
 *   - a vertex whose change at its last computation was below eps times its
 *     current value (|x_new - x_old| < eps * x) has (nearly) stopped moving:
 *     in a perforated sweep it keeps its value and its in-list is not summed;
 *     every other vertex takes the Jacobi update of Algorithm 1 (the dangling
 *     mass D and the contributions come from the whole iterate at the start
 *     of the sweep, as in orc_jacobi);
 *   - with period > 0, sweep k (k = 0, 1, ...) is a full Jacobi sweep when k
 *     is a multiple of period, and only a full sweep can stop the iteration;
 *     with period 0 every sweep but the first is perforated and any sweep can
 *     stop (the approximate-computing form: the error of a sweep counts the
 *     vertices it computed, a skipped vertex changes by 0);
 *   - the stop rule is Algorithm 1's, and the result is normalised at the end.
 * Before its first computation a vertex has an infinite last change, so the
 * first sweep is always full; eps 0 or period 1 is plain Jacobi.  *gathered
 * receives the number of in-list entries summed over all sweeps.
 */
int orc_perforated(PROBLEM_ARGS, double eps, int32_t period, const double *x0, double tau,
                   int32_t max_iter, int32_t norm, int32_t normalize, double *x_out,
                   int32_t *iters, double *err_last, double *err_hist, double *sum_before,
                   int64_t *gathered)
{
    MAKE_PROBLEM;
    if (n < 1 || max_iter < 0 || period < 0 || !(eps >= 0.0)) return ORC_ERR_ARG;
    double *x = x_out;
    double *xn = (double *)malloc(sizeof(double) * (size_t)n);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    double *last = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xn || !c || !last) { free(xn); free(c); free(last); return ORC_ERR_OOM; }
    for (int32_t u = 0; u < n; ++u) {
        x[u] = x0 ? x0[u] : 1.0 / (double)n;
        last[u] = INFINITY;
    }
    const double base = (1.0 - p.d) / (double)n;
    const double inv_n = 1.0 / (double)n;
    int64_t edges = 0;
    int32_t k = 0;
    double err = INFINITY;
    int converged = 0;
    while (k < max_iter) {
        const int full = period > 0 && (k % period) == 0;
        const double D = dangling_mass(&p, x);
        if (!p.csc_p)
            for (int32_t v = 0; v < n; ++v) c[v] = x[v] * p.inv_outdeg[v];
        ksum l1 = {0.0, 0.0};
        double mx = 0.0;
        for (int32_t u = 0; u < n; ++u) {
            if (!full && last[u] < eps * x[u]) {
                xn[u] = x[u];
                continue;
            }
            double sum = 0.0;
            for (int32_t q = p.col_ptr[u]; q < p.col_ptr[u + 1]; ++q) {
                int32_t v = p.row_idx[q];
                sum += p.csc_p ? p.csc_p[q] * x[v] : c[v];
            }
            edges += p.col_ptr[u + 1] - p.col_ptr[u];
            xn[u] = r_of(&p, u, base) + p.d * (sum + D * w_of(&p, u, inv_n));
            const double diff = fabs(xn[u] - x[u]);
            last[u] = diff;
            ks_add(&l1, diff);
            if (diff > mx) mx = diff;
        }
        memcpy(x, xn, sizeof(double) * (size_t)n);
        err = norm == 0 ? ks_get(&l1) : mx;
        if (err_hist) err_hist[k] = err;
        ++k;
        if ((full || period == 0) && err <= tau) { converged = 1; break; }
    }
    const double s = total(x, n);
    if (sum_before) *sum_before = s;
    if (normalize)
        for (int32_t u = 0; u < n; ++u) x[u] = x[u] / s;
    *iters = k;
    *err_last = err;
    if (gathered) *gathered = edges;
    free(xn);
    free(c);
    free(last);
    return converged ? ORC_OK : ORC_NOT_CONVERGED;
}

/*
 * Tight fixed point x* by Jacobi: sweeps until the L1 successive difference
 * is <= floor_tau or has not decreased for `patience` sweeps (round-off
 * stagnation) or max_iter is hit.  The returned iterate satisfies
 * ||x - x*||_1 <= d/(1-d) * err_last (contraction of d*M in the 1-norm).
 */
int orc_fixed_point(PROBLEM_ARGS, const double *x0, double floor_tau, int32_t patience,
                    int32_t max_iter, int32_t normalize, double *x_out, int32_t *iters,
                    double *err_last, double *sum_before)
{
    MAKE_PROBLEM;
    if (n < 1) return ORC_ERR_ARG;
    double *x = x_out;
    double *xn = (double *)malloc(sizeof(double) * (size_t)n);
    double *c = (double *)malloc(sizeof(double) * (size_t)n);
    if (!xn || !c) { free(xn); free(c); return ORC_ERR_OOM; }
    for (int32_t u = 0; u < n; ++u) x[u] = x0 ? x0[u] : 1.0 / (double)n;
    double best = INFINITY, err = INFINITY;
    int32_t since_best = 0, k = 0;
    while (k < max_iter) {
        err = jacobi_sweep(&p, x, xn, c, 0);
        memcpy(x, xn, sizeof(double) * (size_t)n);
        ++k;
        if (err <= floor_tau) break;
        if (err < best) { best = err; since_best = 0; }
        else if (++since_best >= patience) break;
    }
    const double s = total(x, n);
    if (sum_before) *sum_before = s;
    if (normalize)
        for (int32_t u = 0; u < n; ++u) x[u] = x[u] / s;
    *iters = k;
    *err_last = err;
    free(xn);
    free(c);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Weighted graphs: row normalisation of raw edge weights                   */
/* ------------------------------------------------------------------------ */
/*
 * s[u] = sum of the raw weights on u's out-edges, summed in out-list order;
 * csr_p[slot] = w / s[u] for each out-list slot, csc_p[slot] the same value
 * placed at the in-list slot of the same edge.  Weights must be > 0.
 */
int orc_row_normalize(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *csr_eid,
                      const int32_t *csc_eid, const int32_t *row_idx, const float *w,
                      double *s, double *csr_p, double *csc_p)
{
    for (int32_t u = 0; u < n; ++u) {
        double acc = 0.0;
        for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q) acc += (double)w[csr_eid[q]];
        s[u] = acc;
        for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q)
            csr_p[q] = (double)w[csr_eid[q]] / acc;
    }
    for (int64_t q = 0; q < m; ++q) {
        int32_t u = row_idx[q];
        csc_p[q] = (double)w[csc_eid[q]] / s[u];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Adjoint and gradients                                                    */
/* ------------------------------------------------------------------------ */
/*
 * Transposed fixed point (I - d M)^T lambda = g for uniform teleport and
 * uniform dangling redistribution, iterated on the out-lists:
 *   lambda'_u = g_u + d * (sum_{v in outlink(u)} P_uv lambda_v
 *                          + [u dangling] * (sum_v lambda_v) / n).
 * csr_p == NULL means P_uv = inv_outdeg[u].  Stops like orc_fixed_point.
 */
int orc_adjoint(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                const int32_t *outdeg, const double *inv_outdeg, const double *csr_p, double d,
                const double *g, double floor_tau, int32_t patience, int32_t max_iter,
                double *lambda, int32_t *iters, double *err_last)
{
    double *ln = (double *)malloc(sizeof(double) * (size_t)n);
    if (!ln) return ORC_ERR_OOM;
    for (int32_t u = 0; u < n; ++u) lambda[u] = g[u];
    double best = INFINITY, err = INFINITY;
    int32_t since_best = 0, k = 0;
    while (k < max_iter) {
        const double S = total(lambda, n);
        ksum l1 = {0.0, 0.0};
        for (int32_t u = 0; u < n; ++u) {
            double acc = 0.0;
            for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q) {
                double puv = csr_p ? csr_p[q] : inv_outdeg[u];
                acc += puv * lambda[col_idx[q]];
            }
            if (outdeg[u] == 0) acc += S / (double)n;
            ln[u] = g[u] + d * acc;
            ks_add(&l1, fabs(ln[u] - lambda[u]));
        }
        err = ks_get(&l1);
        memcpy(lambda, ln, sizeof(double) * (size_t)n);
        ++k;
        if (err <= floor_tau) break;
        if (err < best) { best = err; since_best = 0; }
        else if (++since_best >= patience) break;
    }
    *iters = k;
    *err_last = err;
    free(ln);
    return ORC_OK;
}

/*
 * Gradients of L(x*) given x* (forward fixed point, un-normalised sum 1) and
 * lambda (adjoint of g = dL/dx), for x = (1-d)/n + d M x:
 *   dL/dP_uv = d * lambda_v * x_u,
 *   dL/dw_e  = (d x_u / s_u) (lambda_v - sum_{v'} P_uv' lambda_v')  for e = u->v
 *              (row normalisation P_uv = w_uv / s_u by the chain rule),
 *   dL/dd    = lambda^T (M x - 1/n).
 * w == NULL means all raw weights are 1 (then s_u = outdeg, P_uv = 1/outdeg).
 * grad_w is written in input edge order (csr_eid maps out-list slots to ids).
 */
int orc_gradients(int32_t n, int64_t m, const int32_t *row_ptr, const int32_t *col_idx,
                  const int32_t *csr_eid, const int32_t *outdeg, const float *w, double d,
                  const double *x, const double *lambda, double *grad_w, double *grad_d)
{
    (void)m;
    double *Mx = (double *)calloc((size_t)n, sizeof(double));
    if (!Mx) return ORC_ERR_OOM;
    ksum Dk = {0.0, 0.0};
    for (int32_t u = 0; u < n; ++u) {
        if (outdeg[u] == 0) { ks_add(&Dk, x[u]); continue; }
        double s = 0.0;
        for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q)
            s += w ? (double)w[csr_eid[q]] : 1.0;
        double plam = 0.0;
        for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q) {
            double puv = (w ? (double)w[csr_eid[q]] : 1.0) / s;
            plam += puv * lambda[col_idx[q]];
            Mx[col_idx[q]] += puv * x[u];
        }
        for (int32_t q = row_ptr[u]; q < row_ptr[u + 1]; ++q)
            grad_w[csr_eid[q]] = (d * x[u] / s) * (lambda[col_idx[q]] - plam);
    }
    const double D = ks_get(&Dk);
    ksum gd = {0.0, 0.0};
    for (int32_t u = 0; u < n; ++u)
        ks_add(&gd, lambda[u] * (Mx[u] + D / (double)n - 1.0 / (double)n));
    *grad_d = ks_get(&gd);
    free(Mx);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Dense systems for tiny graphs                                            */
/* ------------------------------------------------------------------------ */
/*
 * Dense column-stochastic operator of the graph:
 *   M[v][u] += w_e / s_u for every edge e = u->v (w == NULL: weight 1),
 *   M[v][u]  = tele_v (or 1/n) for every dangling u,
 * then A = I - d M and b = (1-d) tele (or (1-d)/n).  Row-major n x n.
 */
int orc_dense_system(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                     const double *w, double d, const double *tele,
                     int32_t dangling_along_tele, double *A, double *b)
{
    double *s = (double *)calloc((size_t)n, sizeof(double));
    double *M = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    if (!s || !M) { free(s); free(M); return ORC_ERR_OOM; }
    for (int64_t e = 0; e < m; ++e) s[src[e]] += w ? w[e] : 1.0;
    for (int64_t e = 0; e < m; ++e)
        M[(size_t)dst[e] * n + src[e]] += (w ? w[e] : 1.0) / s[src[e]];
    for (int32_t u = 0; u < n; ++u) {
        if (s[u] != 0.0) continue;
        for (int32_t v = 0; v < n; ++v)
            M[(size_t)v * n + u] =
                (tele && dangling_along_tele) ? tele[v] : 1.0 / (double)n;
    }
    for (int32_t i = 0; i < n; ++i) {
        for (int32_t j = 0; j < n; ++j)
            A[(size_t)i * n + j] = (i == j ? 1.0 : 0.0) - d * M[(size_t)i * n + j];
        b[i] = tele ? (1.0 - d) * tele[i] : (1.0 - d) / (double)n;
    }
    free(s);
    free(M);
    return ORC_OK;
}

/* Gaussian elimination with partial pivoting; A (row-major, n x n) and b are
 * overwritten.  Returns ORC_ERR_ARG for a singular matrix. */
int orc_dense_solve(int32_t n, double *A, double *b, double *x)
{
    for (int32_t k = 0; k < n; ++k) {
        int32_t piv = k;
        for (int32_t i = k + 1; i < n; ++i)
            if (fabs(A[(size_t)i * n + k]) > fabs(A[(size_t)piv * n + k])) piv = i;
        if (A[(size_t)piv * n + k] == 0.0) return ORC_ERR_ARG;
        if (piv != k) {
            for (int32_t j = 0; j < n; ++j) {
                double t = A[(size_t)k * n + j];
                A[(size_t)k * n + j] = A[(size_t)piv * n + j];
                A[(size_t)piv * n + j] = t;
            }
            double t = b[k]; b[k] = b[piv]; b[piv] = t;
        }
        for (int32_t i = k + 1; i < n; ++i) {
            double f = A[(size_t)i * n + k] / A[(size_t)k * n + k];
            for (int32_t j = k; j < n; ++j) A[(size_t)i * n + j] -= f * A[(size_t)k * n + j];
            b[i] -= f * b[k];
        }
    }
    for (int32_t i = n - 1; i >= 0; --i) {
        double acc = b[i];
        for (int32_t j = i + 1; j < n; ++j) acc -= A[(size_t)i * n + j] * x[j];
        x[i] = acc / A[(size_t)i * n + i];
    }
    return ORC_OK;
}
