// graph.cu -- pr_graph_create and friends: assembles the graph on the device
// (the paper's Sec. 3 storage: in-lists grouped by destination) and the
// sweep's working copy in a degree-ordered numbering.
//
// Build steps (all on the device, all deterministic):
//   1. edge keys and id validation                         (k_make_csc_keys)
//   2. in-lists in the input ids: stable radix sort of (dst, src) keys,
//      out/in-degrees from the runs of the half-sorted and sorted keys
//   3. 1/outdeg, dangling count, largest in-degree          (k_vertex_init)
//   4. degree-ordered ids: stable radix sort of vertices by in-degree,
//      largest first; each in-list copied with its sources renamed
//   5. work items: hub segments over [0, nhub), mid sub-ranges, low tiles
//   6. (on demand) out-lists; (weighted graphs) row sums and P per slot
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include "../../include/fusedpr_diag.h"
#include "common.cuh"

namespace fpr {

// ----------------------------------------------------- per-vertex data
// 1/outdeg in FP64 (IEEE quotient), dangling count, largest in-degree.
// Grid-stride; one pair of atomics per block (per-warp atomics on the two
// counters serialised at L2 and took ~170 us at 4M vertices).
__global__ void k_vertex_init(int32_t n, const int32_t *__restrict__ outdeg,
                              const int32_t *__restrict__ indeg, double *inv64,
                              int32_t *n_dangling, int32_t *max_indeg)
{
    __shared__ int s_dang[32], s_max[32];
    int dang = 0, di = 0;
    for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
        const int k = outdeg[u];
        inv64[u] = k > 0 ? 1.0 / (double)k : 0.0;
        dang += k == 0;
        di = max(di, indeg[u]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        dang += __shfl_xor_sync(FULL, dang, o);
        di = max(di, __shfl_xor_sync(FULL, di, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) {
        s_dang[warp] = dang;
        s_max[warp] = di;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int a = 0, b = 0;
        for (int w = 0; w < nw; ++w) {
            a += s_dang[w];
            b = max(b, s_max[w]);
        }
        if (a) atomicAdd(n_dangling, a);
        atomicMax(max_indeg, b);
    }
}

// ------------------------------------------------------------ relabelling
// key = (maxd - indeg) in the high word: ascending key = in-degree descending;
// the stable sort keeps ties in increasing id.
__global__ void k_perm_keys(int32_t n, const int32_t *__restrict__ indeg, int32_t maxd,
                            uint64_t *keys, int32_t *vals)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    keys[u] = (uint64_t)(uint32_t)(maxd - indeg[u]) << 32;
    vals[u] = u;
}

__global__ void k_invert_perm(int32_t n, const int32_t *__restrict__ n2o, int32_t *o2n)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) o2n[n2o[k]] = k;
}

__global__ void k_relabel_vertex(int32_t n, const int32_t *__restrict__ n2o,
                                 const int32_t *__restrict__ outdeg,
                                 const int32_t *__restrict__ indeg, int32_t *r_outdeg,
                                 int32_t *r_indeg, double *r_inv64, float *r_inv32)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int u = n2o[k];
    const int od = outdeg[u];
    r_outdeg[k] = od;
    r_indeg[k] = indeg[u];
    r_inv64[k] = od > 0 ? 1.0 / (double)od : 0.0;
    r_inv32[k] = od > 0 ? 1.0f / (float)od : 0.0f;
}

// The in-list of new vertex k is the input-id in-list of n2o[k], in the same
// order, with its sources renamed.  The copy is flat over the output slots:
// a warp takes a chunk of RL_SLOTS consecutive slots (coalesced writes) and
// each lane finds the vertex of its slot by binary search of r_col_ptr
// between the chunk's first and last owners.
constexpr int RL_SLOTS = 1024;

// owner[c]: the vertex whose in-list holds slot min(c * RL_SLOTS, m - 1)
// (the largest k with r_col_ptr[k] <= that slot), c in [0, nchunks].
__global__ void k_chunk_owner(int32_t n, int64_t m, int64_t nchunks,
                              const int32_t *__restrict__ r_col_ptr, int32_t *owner)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c > nchunks) return;
    const int64_t slot = min(c * RL_SLOTS, m - 1);
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = lo + ((hi - lo + 1) >> 1);
        if (r_col_ptr[mid] <= slot) lo = mid;
        else hi = mid - 1;
    }
    owner[c] = lo;
}

__global__ void k_relabel_lists(int64_t m, int64_t nchunks, const int32_t *__restrict__ owner,
                                const int32_t *__restrict__ n2o,
                                const int32_t *__restrict__ o2n,
                                const int32_t *__restrict__ col_ptr,
                                const int32_t *__restrict__ row_idx,
                                const int32_t *__restrict__ csc_eid,
                                const int32_t *__restrict__ r_col_ptr, int32_t *r_row_idx,
                                int32_t *r_csc_eid)
{
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < nchunks; c += nw) {
        const int ka = owner[c], kb = owner[c + 1];
        const int64_t s1 = min(m, (c + 1) * RL_SLOTS);
        for (int64_t j = c * RL_SLOTS + lane; j < s1; j += 32) {
            int lo = ka, hi = kb;
            while (lo < hi) {
                const int mid = lo + ((hi - lo + 1) >> 1);
                if (__ldg(r_col_ptr + mid) <= j) lo = mid;
                else hi = mid - 1;
            }
            const int64_t pos = (int64_t)__ldg(col_ptr + __ldg(n2o + lo)) + (j - __ldg(r_col_ptr + lo));
            r_row_idx[j] = o2n[row_idx[pos]];
            r_csc_eid[j] = csc_eid[pos];
        }
    }
}

// -------------------------------------------------------------- work items
// counts[0]: in-degree > t_hub; counts[1]: t_lo < in-degree <= t_hub;
// counts[2..4]: of those, in-degree > max(t_lo, 128 / 64 / 32).
__global__ void k_count_classes(int32_t n, const int32_t *__restrict__ col_ptr, int t_lo,
                                int t_hub, int w32, int32_t *counts)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    int deg = u < n ? col_ptr[u + 1] - col_ptr[u] : -1;
    const bool mid = deg > t_lo && deg <= t_hub;
    unsigned b[5] = {__ballot_sync(FULL, deg > t_hub), __ballot_sync(FULL, mid),
                     __ballot_sync(FULL, mid && deg > w32),
                     __ballot_sync(FULL, mid && deg > w32 / 2),
                     __ballot_sync(FULL, mid && deg > w32 / 4)};
    if ((threadIdx.x & 31) == 0)
        for (int k = 0; k < 5; ++k)
            if (b[k]) atomicAdd(&counts[k], __popc(b[k]));
}

__global__ void k_hub_segments(int32_t nhub, const int32_t *__restrict__ col_ptr, int hub_seg,
                               int32_t *nseg)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < nhub) nseg[h] = (col_ptr[h + 1] - col_ptr[h] + hub_seg - 1) / hub_seg;
}

// Tile k starts at the first vertex u >= first whose work prefix (in-edges +
// vertices before it, counted from `first`) reaches k * c.
__global__ void k_tile_starts(int32_t ntiles, int32_t first, int32_t n,
                              const int32_t *__restrict__ col_ptr, int32_t c, int32_t *tile_start)
{
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > ntiles) return;
    if (k == ntiles) {
        tile_start[k] = n;
        return;
    }
    const int64_t target = (int64_t)k * c;
    const int32_t e0 = col_ptr[first];
    int lo = first, hi = n;  // answer in [first, n]
    while (lo < hi) {
        int mid = lo + ((hi - lo) >> 1);
        int64_t cost = (int64_t)(col_ptr[mid] - e0) + (mid - first);
        if (cost >= target) hi = mid;
        else lo = mid + 1;
    }
    tile_start[k] = lo;
}

struct MidRanges {
    int32_t mb[5], mi[5];
};

// Item descriptors in item order: hub segments {hub, 0, ea, eb}, mid groups
// (32 >> k lanes per vertex, 1 << k vertices of sub-range k) and low tiles,
// both {v0, v1, ea, eb}.
__global__ void k_item_desc(int32_t nhubseg, int32_t nhub, const int32_t *__restrict__ hubseg_start,
                            int hub_seg, MidRanges mr, int32_t ntiles,
                            const int32_t *__restrict__ tile_start,
                            const int32_t *__restrict__ col_ptr, int4 *desc)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int nmid = mr.mi[4];
    if (i >= nhubseg + nmid + ntiles) return;
    if (i >= nhubseg && i < nhubseg + nmid) {
        const int j = i - nhubseg;
        int k = 0;
        while (k < 3 && j >= mr.mi[k + 1]) ++k;
        const int v0 = mr.mb[k] + (j - mr.mi[k]) * (1 << k);
        const int v1 = min(v0 + (1 << k), mr.mb[k + 1]);
        desc[i] = make_int4(v0, v1, col_ptr[v0], col_ptr[v1]);
        return;
    }
    if (i < nhubseg) {
        int lo = 0, hi = nhub - 1;  // hub owning segment i
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (hubseg_start[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const int h = lo;
        const int a = col_ptr[h] + (i - hubseg_start[h]) * hub_seg;
        desc[i] = make_int4(h, 0, a, min(a + hub_seg, col_ptr[h + 1]));
    } else {
        const int k = i - nhubseg - nmid;
        const int v0 = tile_start[k], v1 = tile_start[k + 1];
        desc[i] = make_int4(v0, v1, col_ptr[v0], col_ptr[v1]);
    }
}

pr_tune effective_tune(const pr_graph *g, const pr_tune *t)
{
    pr_tune r = g->tune;
    if (t) {
        if (t->t_lo > 0) r.t_lo = t->t_lo;
        if (t->t_hub > 0) r.t_hub = t->t_hub;
        if (t->hub_seg > 0) r.hub_seg = t->hub_seg;
        if (t->tile > 0) r.tile = t->tile;
        if (t->stage_kb != 0) r.stage_kb = t->stage_kb;
        r.deterministic_gs = t->deterministic_gs;
        r.wait_limit = t->wait_limit > 0 ? t->wait_limit : 0;
        r.fused_split = t->fused_split;
        r.blocking = t->blocking ? 1 : 0;
        if (t->mid_wide > 0) r.mid_wide = t->mid_wide;
    }
    r.mid_wide = std::max(16, std::min(r.mid_wide, 1 << 20));
    r.fused_split = std::max(0, std::min(r.fused_split, 2));
    r.stage_kb = r.stage_kb < 0 ? -1 : std::min(r.stage_kb, 227);
    // a low tile's in-edges (at most tile + t_lo) sit in one warp's slice of
    // shared memory, and a lane adds up to t_lo of them
    r.t_lo = std::max(0, std::min(r.t_lo, 32));
    r.t_hub = std::max(r.t_lo, std::min(r.t_hub, 1 << 20));
    r.hub_seg = std::max(256, std::min(r.hub_seg, 8192));
    r.tile = std::max(32, std::min(r.tile, 512));
    return r;
}

// the blocked sweep's layout of a graph (blocked.cu), released at destroy
void release_blocked(pr_graph *g);

// Fault-injection hook for the tests of the bounded device waits (not part
// of the C ABI): with FUSEDPR_TEST_STALL=1 in the environment, every sweep
// block's first wait also waits on a barrier nothing arrives at, so the wait
// runs out and the solve returns PR_ERR_TIMEOUT with the device still usable.
int test_stall_requested()
{
    const char *v = getenv("FUSEDPR_TEST_STALL");
    return (v && v[0] == '1') ? 1 : 0;
}

static void drop_temp(pr_graph *g, Buf &b, cudaStream_t s)
{
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &b), g->owned.end());
    buf_free(g, b, s);
}

// Scratch device memory freed when it goes out of scope (on every return
// path); never registered with the graph.
struct Scratch {
    pr_graph *g;
    cudaStream_t s;
    Buf b;
    Scratch(pr_graph *g_, cudaStream_t s_) : g(g_), s(s_) {}
    ~Scratch() { buf_free(g, b, s); }
    pr_status alloc(size_t bytes)
    {
        b.p = g->mem.alloc(bytes, s);
        if (!b.p) {
            set_error("device allocation of %zu bytes failed", bytes);
            return PR_ERR_OOM;
        }
        b.bytes = bytes ? bytes : 16;
        return PR_OK;
    }
    template <typename T>
    T *as() const { return b.as<T>(); }
};

// (Re)computes the classes, hub segments, mid sub-ranges and low tiles for
// the thresholds.
pr_status ensure_items(pr_graph *g, const pr_tune &t, cudaStream_t s)
{
    Items &it = g->items;
    it.stage_kb = t.stage_kb;
    it.wait_limit = t.wait_limit;
    it.test_stall = test_stall_requested();
    it.fused_split = t.fused_split;
    if (it.t_lo == t.t_lo && it.t_hub == t.t_hub && it.hub_seg == t.hub_seg &&
        it.tile_c == t.tile && it.mid_wide == t.mid_wide)
        return PR_OK;
    const int32_t n = g->n;
    const int32_t *rcp = g->r_col_ptr.as<int32_t>();
    Scratch tmp(g, s);
    PR_TRY(tmp.alloc(sizeof(int32_t) * 8));
    PR_CUDA(cudaMemsetAsync(tmp.b.p, 0, sizeof(int32_t) * 8, s));
    k_count_classes<<<(n + 255) / 256, 256, 0, s>>>(n, rcp, t.t_lo, t.t_hub, t.mid_wide,
                                                      tmp.as<int32_t>());
    note_launch();
    PR_LAUNCH_CHECK();
    int32_t h[8];
    PR_CUDA(cudaMemcpyAsync(h, tmp.b.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    it.nhub = h[0];
    it.nmid = h[1];
    it.nlow = n - h[0] - h[1];
    // mid sub-ranges: 32, 16, 8, 4 lanes per vertex
    const int32_t bounds[5] = {it.nhub, it.nhub + h[2], it.nhub + h[3], it.nhub + h[4],
                               it.nhub + h[1]};
    it.mi[0] = 0;
    for (int k = 0; k < 4; ++k) {
        const int per = 1 << k;  // vertices per warp
        it.mb[k] = bounds[k];
        it.mi[k + 1] = it.mi[k] + (bounds[k + 1] - bounds[k] + per - 1) / per;
    }
    it.mb[4] = bounds[4];

    // hub segments
    PR_TRY(buf_alloc(g, it.hubseg_start, sizeof(int32_t) * (size_t)(it.nhub + 1), s));
    PR_TRY(buf_alloc(g, it.hub_cnt, sizeof(int32_t) * (size_t)std::max(it.nhub, 1), s));
    PR_CUDA(cudaMemsetAsync(it.hub_cnt.p, 0, sizeof(int32_t) * (size_t)std::max(it.nhub, 1), s));
    it.nhubseg = 0;
    if (it.nhub > 0) {
        k_hub_segments<<<(it.nhub + 255) / 256, 256, 0, s>>>(it.nhub, rcp, t.hub_seg,
                                                            it.hubseg_start.as<int32_t>());
        note_launch();
        PR_LAUNCH_CHECK();
        PR_TRY(scan_exclusive(g, it.hubseg_start.as<int32_t>(), it.hubseg_start.as<int32_t>(),
                              it.nhub, s));
        PR_CUDA(cudaMemcpyAsync(&it.nhubseg, it.hubseg_start.as<int32_t>() + it.nhub,
                                sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    } else {
        PR_CUDA(cudaMemsetAsync(it.hubseg_start.p, 0, sizeof(int32_t), s));
    }
    PR_TRY(buf_alloc(g, it.seg_acc, sizeof(double) * (size_t)std::max(it.nhubseg, 1), s));

    // low tiles over [nhub + nmid, n)
    const int32_t first = it.nhub + it.nmid;
    int32_t ends[2] = {0, 0};
    PR_CUDA(cudaMemcpyAsync(&ends[0], rcp + first, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaMemcpyAsync(&ends[1], rcp + n, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    const int64_t work = (int64_t)(ends[1] - ends[0]) + (n - first);
    it.nlt = (int32_t)((work + t.tile - 1) / t.tile);
    Scratch tile_start(g, s);
    PR_TRY(tile_start.alloc(sizeof(int32_t) * (size_t)(it.nlt + 1)));
    k_tile_starts<<<(it.nlt + 256) / 256, 256, 0, s>>>(it.nlt, first, n, rcp, t.tile,
                                                       tile_start.as<int32_t>());
    note_launch();
    const int nitems = it.nhubseg + it.mi[4] + it.nlt;
    PR_TRY(buf_alloc(g, it.desc, sizeof(int4) * (size_t)std::max(nitems, 1), s));
    if (nitems > 0) {
        MidRanges mr;
        for (int k = 0; k < 5; ++k) {
            mr.mb[k] = it.mb[k];
            mr.mi[k] = it.mi[k];
        }
        k_item_desc<<<(nitems + 255) / 256, 256, 0, s>>>(
            it.nhubseg, it.nhub, it.hubseg_start.as<int32_t>(), t.hub_seg, mr, it.nlt,
            tile_start.as<int32_t>(), rcp, it.desc.as<int4>());
        note_launch();
    }
    PR_LAUNCH_CHECK();
    // a low tile holds fewer than tile + t_lo + 1 in-edges
    it.lcap = (t.tile + t.t_lo + 8) & ~7;
    it.t_lo = t.t_lo;
    it.t_hub = t.t_hub;
    it.hub_seg = t.hub_seg;
    it.tile_c = t.tile;
    it.mid_wide = t.mid_wide;
    PR_CUDA(cudaStreamSynchronize(s));
    return PR_OK;
}

// Builds the out-lists from the input-id in-lists: the in-list stream is
// ordered by (dst, src, id); a stable sort by src gives (src, dst, id).
pr_status ensure_csr(pr_graph *g, cudaStream_t s)
{
    if (g->col_idx.p) return PR_OK;
    const int64_t m = g->m;
    const int32_t n = g->n;
    PR_TRY(buf_alloc(g, g->row_ptr, sizeof(int32_t) * (size_t)(n + 1), s));
    PR_TRY(buf_alloc(g, g->col_idx, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), s));
    PR_TRY(buf_alloc(g, g->csr_eid, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), s));
    PR_TRY(scan_exclusive(g, g->outdeg.as<int32_t>(), g->row_ptr.as<int32_t>(), n, s));
    if (m == 0) return PR_OK;
    Buf k1, k2, v2;
    pr_status st = buf_alloc(g, k1, sizeof(uint64_t) * (size_t)m, s);
    if (st == PR_OK) st = buf_alloc(g, k2, sizeof(uint64_t) * (size_t)m, s);
    if (st == PR_OK) st = buf_alloc(g, v2, sizeof(int32_t) * (size_t)m, s);
    if (st == PR_OK) {
        int blocks = (int)std::min<int64_t>((n + 7) / 8, 1 << 20);
        k_make_csr_keys<<<std::max(blocks, 1), 256, 0, s>>>(n, g->col_ptr.as<int32_t>(),
                                                            g->row_idx.as<int32_t>(),
                                                            g->csc_eid.as<int32_t>(),
                                                            k1.as<uint64_t>(),
                                                            g->csr_eid.as<int32_t>());
        note_launch();
        st = radix_sort(g, k1.as<uint64_t>(), g->csr_eid.as<int32_t>(), k2.as<uint64_t>(),
                        v2.as<int32_t>(), m, digit_shifts(n, 32), s);
    }
    if (st == PR_OK) {
        k_split_csr<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, k1.as<uint64_t>(),
                                                                g->col_idx.as<int32_t>());
        note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "csr split", __FILE__, __LINE__);
    }
    drop_temp(g, k1, s);
    drop_temp(g, k2, s);
    drop_temp(g, v2, s);
    if (st == PR_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "csr build", __FILE__, __LINE__);
    }
    return st;
}

// --------------------------------------------------------------- weights
__global__ void k_rowsum(int32_t n, const int32_t *__restrict__ row_ptr,
                         const int32_t *__restrict__ csr_eid, const float *__restrict__ w,
                         double *rowsum)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    double s = 0.0;
    for (int q = row_ptr[u]; q < row_ptr[u + 1]; ++q) s += (double)w[csr_eid[q]];
    rowsum[u] = s;
}

// P per relabelled in-list slot: w_e / rowsum(source), source in input ids.
__global__ void k_csc_p(int64_t m, const int32_t *__restrict__ r_row_idx,
                        const int32_t *__restrict__ r_csc_eid, const int32_t *__restrict__ n2o,
                        const float *__restrict__ w, const double *__restrict__ rowsum,
                        double *p64, float *p32)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    double p = (double)w[r_csc_eid[q]] / rowsum[n2o[r_row_idx[q]]];
    p64[q] = p;
    p32[q] = (float)p;
}

__global__ void k_check_weights(int64_t m, const float *__restrict__ w, int32_t *err)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) {
        float x = w[e];
        if (!(x > 0.0f) || !isfinite(x)) atomicOr(err, 2);
    }
}

static void destroy_impl(pr_graph *g)
{
    if (!g) return;
    cudaStream_t s = g->mem.stream;
    cudaStreamSynchronize(s);
    pr_graph_destroy(g->rev);  // built by pr_graph_create (adjoint)
    g->rev = nullptr;
    release_graphs(g);
    for (Buf *b : g->owned) buf_free(g, *b, s);
    release_blocked(g);
    cudaStreamSynchronize(s);
    if (g->host_state) cudaFreeHost(g->host_state);
    cudaGetLastError();
    delete g;
}

// Sorts (keys, vals) by the given digits with scratch of the same size.
static pr_status sort_pairs(pr_graph *g, uint64_t *keys, int32_t *vals, int64_t m,
                            const std::vector<int> &shifts, cudaStream_t s)
{
    Buf k2, v2;
    pr_status st = buf_alloc(g, k2, sizeof(uint64_t) * (size_t)std::max<int64_t>(m, 1), s);
    if (st == PR_OK) st = buf_alloc(g, v2, sizeof(int32_t) * (size_t)std::max<int64_t>(m, 1), s);
    if (st == PR_OK)
        st = radix_sort(g, keys, vals, k2.as<uint64_t>(), v2.as<int32_t>(), m, shifts, s);
    drop_temp(g, k2, s);
    drop_temp(g, v2, s);
    return st;
}

// PR_DEDUP: 1 where the sorted (dst, src) key starts a run of equal keys
// (the run's first entry is the edge's first occurrence: the sort is stable)
__global__ void k_first_of_run(int64_t m, const uint64_t *__restrict__ keys, int32_t *flag)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        flag[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

__global__ void k_compact_runs(int64_t m, const uint64_t *__restrict__ keys,
                               const int32_t *__restrict__ vals, const int32_t *__restrict__ flag,
                               const int32_t *__restrict__ pos, uint64_t *kout, int32_t *vout)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        if (flag[i]) {
            kout[pos[i]] = keys[i];
            vout[pos[i]] = vals[i];
        }
}

// out-degrees of the kept edges (sources in the low 32 bits of the keys)
__global__ void k_count_sources(int64_t m, const uint64_t *__restrict__ keys, int32_t *outdeg)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride)
        atomicAdd(&outdeg[(uint32_t)keys[i]], 1);
}

static pr_status build_all(pr_graph *g, const int32_t *src, const int32_t *dst, const float *w,
                           uint32_t flags, cudaStream_t s)
{
    const int32_t n = g->n;
    int64_t m = g->m;
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    for (auto pb : {std::make_pair(&g->outdeg, sizeof(int32_t) * (size_t)n),
                    std::make_pair(&g->indeg, sizeof(int32_t) * (size_t)n),
                    std::make_pair(&g->col_ptr, sizeof(int32_t) * (size_t)(n + 1)),
                    std::make_pair(&g->row_idx, sizeof(int32_t) * mm),
                    std::make_pair(&g->csc_eid, sizeof(int32_t) * mm),
                    std::make_pair(&g->inv64, sizeof(double) * (size_t)n),
                    std::make_pair(&g->n2o, sizeof(int32_t) * (size_t)n),
                    std::make_pair(&g->o2n, sizeof(int32_t) * (size_t)n),
                    // the sweep's arrays are padded by 16 entries: its bulk
                    // copies widen every range to 16-byte boundaries
                    std::make_pair(&g->r_outdeg, sizeof(int32_t) * ((size_t)n + 16)),
                    std::make_pair(&g->r_col_ptr, sizeof(int32_t) * ((size_t)n + 17)),
                    std::make_pair(&g->r_row_idx, sizeof(int32_t) * (mm + 16)),
                    std::make_pair(&g->r_csc_eid, sizeof(int32_t) * mm),
                    std::make_pair(&g->r_inv64, sizeof(double) * ((size_t)n + 16)),
                    std::make_pair(&g->r_inv32, sizeof(float) * ((size_t)n + 16)),
                    std::make_pair(&g->state, 2 * sizeof(SolveState) + 64)})
        PR_TRY(buf_alloc(g, *pb.first, pb.second, s));
    PR_CUDA(cudaMallocHost(&g->host_state, 2 * sizeof(SolveState) + 64));
    int32_t *flags_dev = g->state.as<int32_t>();  // [err, n_dangling, max_indeg]
    PR_CUDA(cudaMemsetAsync(g->outdeg.p, 0, sizeof(int32_t) * n, s));
    PR_CUDA(cudaMemsetAsync(g->indeg.p, 0, sizeof(int32_t) * n, s));
    PR_CUDA(cudaMemsetAsync(flags_dev, 0, 4 * sizeof(int32_t), s));
    PR_CUDA(cudaMemsetAsync(g->r_row_idx.p, 0, sizeof(int32_t) * (mm + 16), s));
    PR_CUDA(cudaMemsetAsync(g->r_col_ptr.p, 0, sizeof(int32_t) * ((size_t)n + 17), s));
    PR_CUDA(cudaMemsetAsync(g->r_outdeg.p, 0, sizeof(int32_t) * ((size_t)n + 16), s));
    PR_CUDA(cudaMemsetAsync(g->r_inv64.p, 0, sizeof(double) * ((size_t)n + 16), s));
    PR_CUDA(cudaMemsetAsync(g->r_inv32.p, 0, sizeof(float) * ((size_t)n + 16), s));

    // 1. edge keys (dst << 32 | src) with their input positions, id and
    // weight validation
    Buf k1;
    PR_TRY(buf_alloc(g, k1, sizeof(uint64_t) * std::max(mm, (size_t)n), s));
    if (m > 0) {
        k_make_csc_keys<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
            m, src, dst, n, k1.as<uint64_t>(), g->csc_eid.as<int32_t>(), flags_dev);
        note_launch();
        if (w) {
            k_check_weights<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, w, flags_dev);
            note_launch();
        }
    }
    PR_LAUNCH_CHECK();
    int32_t herr = 0;
    PR_CUDA(cudaMemcpyAsync(&herr, flags_dev, sizeof(herr), cudaMemcpyDeviceToHost, s));
    PR_CUDA(cudaStreamSynchronize(s));
    if (herr & 3) {
        drop_temp(g, k1, s);
        if (herr & 1) set_error("pr_graph_create: an edge endpoint lies outside [0, %d)", n);
        else set_error("pr_graph_create: edge weights must be positive and finite");
        return PR_ERR_INVALID_ARG;
    }

    // 2. in-lists in the input ids: stable radix sort by the source digits,
    // then by the destination digits; out-degrees are the runs of equal
    // sources after the first half, in-degrees the runs of equal
    // destinations at the end
    pr_status st = PR_OK;
    if (m > 0) {
        Buf k2, v2;
        st = buf_alloc(g, k2, sizeof(uint64_t) * mm, s);
        if (st == PR_OK) st = buf_alloc(g, v2, sizeof(int32_t) * mm, s);
        uint64_t *ka = nullptr, *kb = nullptr;
        int32_t *va = nullptr, *vb = nullptr;
        int32_t *eid = g->csc_eid.as<int32_t>();
        const unsigned rb = (unsigned)std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 32);
        if (st == PR_OK)
            st = radix_sort(g, k1.as<uint64_t>(), eid, k2.as<uint64_t>(), v2.as<int32_t>(), m,
                            digit_shifts(n, 0), s, &ka, &va);
        if (st == PR_OK) {
            k_run_degrees<<<rb, 256, 0, s>>>(m, ka, 0, g->outdeg.as<int32_t>(), nullptr);
            note_launch();
            uint64_t *kalt = ka == k1.as<uint64_t>() ? k2.as<uint64_t>() : k1.as<uint64_t>();
            int32_t *valt = va == eid ? v2.as<int32_t>() : eid;
            st = radix_sort(g, ka, va, kalt, valt, m, digit_shifts(n, 32), s, &kb, &vb);
        }
        if (st == PR_OK && (flags & PR_DEDUP)) {
            // repeated (src, dst) pairs are adjacent after the sort, first
            // occurrence first: keep each run's first entry, then count the
            // out-degrees of what is kept
            Buf fl, pos;
            st = buf_alloc(g, fl, sizeof(int32_t) * mm, s);
            if (st == PR_OK) st = buf_alloc(g, pos, sizeof(int32_t) * (mm + 1), s);
            uint64_t *kc = kb == k1.as<uint64_t>() ? k2.as<uint64_t>() : k1.as<uint64_t>();
            int32_t *vc = vb == eid ? v2.as<int32_t>() : eid;
            if (st == PR_OK) {
                k_first_of_run<<<rb, 256, 0, s>>>(m, kb, fl.as<int32_t>());
                note_launch();
                st = scan_exclusive(g, fl.as<int32_t>(), pos.as<int32_t>(), m, s);
            }
            int32_t kept = 0;
            if (st == PR_OK) {
                k_compact_runs<<<rb, 256, 0, s>>>(m, kb, vb, fl.as<int32_t>(), pos.as<int32_t>(),
                                                  kc, vc);
                note_launch();
                PR_CUDA(cudaMemcpyAsync(&kept, pos.as<int32_t>() + m, sizeof(int32_t),
                                        cudaMemcpyDeviceToHost, s));
                PR_CUDA(cudaMemsetAsync(g->outdeg.p, 0, sizeof(int32_t) * (size_t)n, s));
                PR_CUDA(cudaStreamSynchronize(s));
                m = kept;
                g->m = kept;
                kb = kc;
                vb = vc;
                if (m > 0) {
                    k_count_sources<<<rb, 256, 0, s>>>(m, kb, g->outdeg.as<int32_t>());
                    note_launch();
                }
            }
            drop_temp(g, fl, s);
            drop_temp(g, pos, s);
        }
        if (st == PR_OK && m > 0) {
            k_run_degrees<<<rb, 256, 0, s>>>(m, kb, 1, g->indeg.as<int32_t>(),
                                             g->row_idx.as<int32_t>());
            note_launch();
            if (vb != eid)
                PR_CUDA(cudaMemcpyAsync(eid, vb, sizeof(int32_t) * (size_t)m,
                                        cudaMemcpyDeviceToDevice, s));
        }
        drop_temp(g, k2, s);
        drop_temp(g, v2, s);
    }
    if (st != PR_OK) {
        drop_temp(g, k1, s);
        return st;
    }
    const unsigned vib = (unsigned)std::max(1, std::min((n + 255) / 256, g->num_sms * 8));
    k_vertex_init<<<vib, 256, 0, s>>>(n, g->outdeg.as<int32_t>(), g->indeg.as<int32_t>(),
                                      g->inv64.as<double>(), flags_dev + 1, flags_dev + 2);
    note_launch();
    PR_LAUNCH_CHECK();
    int32_t hflags[3] = {0, 0, 0};
    PR_CUDA(cudaMemcpyAsync(hflags, flags_dev, sizeof(hflags), cudaMemcpyDeviceToHost, s));
    st = scan_exclusive(g, g->indeg.as<int32_t>(), g->col_ptr.as<int32_t>(), n, s);
    if (st == PR_OK) PR_CUDA(cudaStreamSynchronize(s));
    g->n_dangling = hflags[1];
    const int32_t maxd = hflags[2];
    // 4. degree-ordered ids
    Buf r_indeg;
    if (st == PR_OK) st = buf_alloc(g, r_indeg, sizeof(int32_t) * (size_t)n, s);
    if (st == PR_OK) {
        k_perm_keys<<<(n + 255) / 256, 256, 0, s>>>(n, g->indeg.as<int32_t>(), maxd,
                                                    k1.as<uint64_t>(), g->n2o.as<int32_t>());
        note_launch();
        st = sort_pairs(g, k1.as<uint64_t>(), g->n2o.as<int32_t>(), n,
                        digit_shifts(maxd + 1, 32), s);
    }
    if (st == PR_OK) {
        k_invert_perm<<<(n + 255) / 256, 256, 0, s>>>(n, g->n2o.as<int32_t>(),
                                                      g->o2n.as<int32_t>());
        note_launch();
        k_relabel_vertex<<<(n + 255) / 256, 256, 0, s>>>(
            n, g->n2o.as<int32_t>(), g->outdeg.as<int32_t>(), g->indeg.as<int32_t>(),
            g->r_outdeg.as<int32_t>(), r_indeg.as<int32_t>(), g->r_inv64.as<double>(),
            g->r_inv32.as<float>());
        note_launch();
        st = scan_exclusive(g, r_indeg.as<int32_t>(), g->r_col_ptr.as<int32_t>(), n, s);
    }
    if (st == PR_OK && m > 0) {
        const int64_t nchunks = (m + RL_SLOTS - 1) / RL_SLOTS;
        Buf owner;
        st = buf_alloc(g, owner, sizeof(int32_t) * (size_t)(nchunks + 1), s);
        if (st == PR_OK) {
            k_chunk_owner<<<(unsigned)((nchunks + 256) / 256), 256, 0, s>>>(
                n, m, nchunks, g->r_col_ptr.as<int32_t>(), owner.as<int32_t>());
            note_launch();
            const unsigned rb = (unsigned)std::min<int64_t>((nchunks + 7) / 8, (int64_t)g->num_sms * 8);
            k_relabel_lists<<<rb, 256, 0, s>>>(
                m, nchunks, owner.as<int32_t>(), g->n2o.as<int32_t>(), g->o2n.as<int32_t>(),
                g->col_ptr.as<int32_t>(), g->row_idx.as<int32_t>(), g->csc_eid.as<int32_t>(),
                g->r_col_ptr.as<int32_t>(), g->r_row_idx.as<int32_t>(),
                g->r_csc_eid.as<int32_t>());
            note_launch();
        }
        drop_temp(g, owner, s);
    }
    drop_temp(g, k1, s);
    drop_temp(g, r_indeg, s);
    if (st != PR_OK) return st;
    PR_LAUNCH_CHECK();

    // 5. work items for the default thresholds
    PR_TRY(ensure_items(g, effective_tune(g, nullptr), s));
    // 6. out-lists, weights
    if ((flags & PR_BUILD_CSR) || w) PR_TRY(ensure_csr(g, s));
    if (w && m > 0) {
        g->weighted = true;
        for (auto pb : {std::make_pair(&g->w, sizeof(float) * (size_t)g->m_in),
                        std::make_pair(&g->rowsum, sizeof(double) * (size_t)n),
                        std::make_pair(&g->p64_csc, sizeof(double) * ((size_t)m + 16)),
                        std::make_pair(&g->p32_csc, sizeof(float) * ((size_t)m + 16))})
            PR_TRY(buf_alloc(g, *pb.first, pb.second, s));
        PR_CUDA(cudaMemcpyAsync(g->w.p, w, sizeof(float) * (size_t)g->m_in, cudaMemcpyDefault,
                                s));
        k_rowsum<<<(n + 255) / 256, 256, 0, s>>>(n, g->row_ptr.as<int32_t>(),
                                                 g->csr_eid.as<int32_t>(), g->w.as<float>(),
                                                 g->rowsum.as<double>());
        note_launch();
        k_csc_p<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
            m, g->r_row_idx.as<int32_t>(), g->r_csc_eid.as<int32_t>(), g->n2o.as<int32_t>(),
            g->w.as<float>(), g->rowsum.as<double>(), g->p64_csc.as<double>(),
            g->p32_csc.as<float>());
        note_launch();
        PR_LAUNCH_CHECK();
    }
    PR_CUDA(cudaStreamSynchronize(s));
    return PR_OK;
}

}  // namespace fpr

using namespace fpr;

extern "C" const char *pr_last_error(void) { return fpr::last_error(); }

extern "C" uint64_t pr_kernel_launches(void) { return fpr::launches(); }

extern "C" pr_status pr_graph_create(int32_t n, int64_t m, const int32_t *src, const int32_t *dst,
                                     const float *w, uint32_t flags, const pr_allocator *alloc,
                                     void *stream, pr_graph **out)
{
    if (!out) {
        set_error("pr_graph_create: out is NULL");
        return PR_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (n < 1 || m < 0 || m >= ((int64_t)1 << 31) || (m > 0 && (!src || !dst))) {
        set_error("pr_graph_create: need n >= 1, 0 <= m < 2^31 and edge arrays");
        return PR_ERR_INVALID_ARG;
    }
    if (alloc && (!alloc->alloc || !alloc->free)) {
        set_error("pr_graph_create: allocator hooks incomplete");
        return PR_ERR_INVALID_ARG;
    }
    if (flags & ~(PR_BUILD_CSR | PR_DEDUP)) {
        set_error("pr_graph_create: unknown flags 0x%x", flags);
        return PR_ERR_INVALID_ARG;
    }
    // the edge arrays are read by kernels: device (or managed) memory, or
    // page-locked host memory, which the kernels read over the host link
    // through its device address; pageable host memory is refused
    if (m > 0) {
        const void *in[3] = {src, dst, w};
        const void *dev[3] = {nullptr, nullptr, nullptr};
        for (int k = 0; k < 3; ++k) {
            if (!in[k]) continue;
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, in[k]) != cudaSuccess ||
                a.type == cudaMemoryTypeUnregistered || !a.devicePointer) {
                cudaGetLastError();
                set_error("pr_graph_create: edge array %d is not device-accessible (device, managed "
                          "or page-locked host memory)", k);
                return PR_ERR_INVALID_ARG;
            }
            dev[k] = a.devicePointer;
        }
        src = static_cast<const int32_t *>(dev[0]);
        dst = static_cast<const int32_t *>(dev[1]);
        w = static_cast<const float *>(dev[2]);
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pr_graph *g = new pr_graph();
    g->n = n;
    g->m = m;
    g->m_in = m;
    g->mem.stream = s;
    if (alloc) {
        g->mem.hooks = *alloc;
        g->mem.has_hooks = true;
    }
    g->tune.t_lo = 32;
    g->tune.t_hub = 4096;
    g->tune.hub_seg = 2048;
    g->tune.tile = 256;
    g->tune.deterministic_gs = 0;
    g->tune.stage_kb = 64;
    g->tune.wait_limit = 0;
    g->tune.mid_wide = 1024;
    pr_status st = PR_OK;
    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&g->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                   g->device);
    if (e != cudaSuccess) st = cuda_status(e, "device query", __FILE__, __LINE__);
    if (st == PR_OK) st = build_all(g, src, dst, w, flags, s);
    if (st != PR_OK) {
        pr_graph_destroy(g);
        return st;
    }
    *out = g;
    return PR_OK;
}

extern "C" void pr_graph_destroy(pr_graph *g) { fpr::destroy_impl(g); }

extern "C" pr_status pr_graph_info(const pr_graph *g, int32_t *n, int64_t *m, int32_t *n_dangling,
                                   int32_t *bin_counts3)
{
    if (!g) {
        set_error("pr_graph_info: graph is NULL");
        return PR_ERR_INVALID_ARG;
    }
    if (n) *n = g->n;
    if (m) *m = g->m;
    if (n_dangling) *n_dangling = g->n_dangling;
    if (bin_counts3) {
        bin_counts3[0] = g->items.nlow;
        bin_counts3[1] = g->items.nmid;
        bin_counts3[2] = g->items.nhub;
    }
    return PR_OK;
}

extern "C" pr_status pr_graph_export(pr_graph *g, int32_t *outdeg, int32_t *indeg,
                                     int32_t *col_ptr, int32_t *row_idx, int32_t *csc_eid,
                                     int32_t *row_ptr, int32_t *col_idx, int32_t *csr_eid,
                                     double *inv_outdeg, int32_t *new_to_old, int32_t *rcol_ptr,
                                     int32_t *rrow_idx, void *stream)
{
    if (!g) {
        set_error("pr_graph_export: graph is NULL");
        return PR_ERR_INVALID_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t n = (size_t)g->n, m = (size_t)g->m;
    if (row_ptr || col_idx || csr_eid) PR_TRY(ensure_csr(g, s));
    auto cp = [&](void *dst, const Buf &b, size_t bytes) -> pr_status {
        if (dst && bytes) PR_CUDA(cudaMemcpyAsync(dst, b.p, bytes, cudaMemcpyDeviceToDevice, s));
        return PR_OK;
    };
    PR_TRY(cp(outdeg, g->outdeg, 4 * n));
    PR_TRY(cp(indeg, g->indeg, 4 * n));
    PR_TRY(cp(col_ptr, g->col_ptr, 4 * (n + 1)));
    PR_TRY(cp(row_idx, g->row_idx, 4 * m));
    PR_TRY(cp(csc_eid, g->csc_eid, 4 * m));
    PR_TRY(cp(row_ptr, g->row_ptr, 4 * (n + 1)));
    PR_TRY(cp(col_idx, g->col_idx, 4 * m));
    PR_TRY(cp(csr_eid, g->csr_eid, 4 * m));
    PR_TRY(cp(inv_outdeg, g->inv64, 8 * n));
    PR_TRY(cp(new_to_old, g->n2o, 4 * n));
    PR_TRY(cp(rcol_ptr, g->r_col_ptr, 4 * (n + 1)));
    PR_TRY(cp(rrow_idx, g->r_row_idx, 4 * m));
    PR_CUDA(cudaStreamSynchronize(s));
    return PR_OK;
}
