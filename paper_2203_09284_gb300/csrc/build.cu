// build.cu -- device-side graph build (the paper's Sec. 3 storage, rebuilt
// for the GPU): out/in-degree histograms, exclusive scans into offsets, a
// stable LSD radix sort that turns the edge list into in-lists (CSC) and,
// on demand, out-lists (CSR), inverse out-degrees, in-degree bins and the
// hub segments of the sweep.  All integer work is deterministic.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "common.cuh"

namespace fpr {

// ------------------------------------------------------------------ errors
static thread_local char g_last_error[512] = {0};

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
}

pr_status cuda_status(cudaError_t e, const char *what, const char *file, int line)
{
    set_error("%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    return e == cudaErrorMemoryAllocation ? PR_ERR_OOM : PR_ERR_CUDA;
}

const char *last_error() { return g_last_error; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

// --------------------------------------------------------------- memory
void *Mem::alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    if (has_hooks) return hooks.alloc(bytes, reinterpret_cast<void *>(s), hooks.ctx);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Mem::free(void *p, size_t bytes, cudaStream_t s)
{
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (has_hooks) hooks.free(p, bytes, reinterpret_cast<void *>(s), hooks.ctx);
    else cudaFreeAsync(p, s);
}

pr_status buf_alloc(pr_graph *g, Buf &b, size_t bytes, cudaStream_t s)
{
    if (b.p && b.bytes >= bytes) return PR_OK;
    buf_free(g, b, s);
    b.p = g->mem.alloc(bytes, s);
    if (!b.p) {
        set_error("device allocation of %zu bytes failed", bytes);
        return PR_ERR_OOM;
    }
    b.bytes = bytes ? bytes : 16;
    if (std::find(g->owned.begin(), g->owned.end(), &b) == g->owned.end()) g->owned.push_back(&b);
    return PR_OK;
}

void buf_free(pr_graph *g, Buf &b, cudaStream_t s)
{
    if (b.p) g->mem.free(b.p, b.bytes, s);
    b.p = nullptr;
    b.bytes = 0;
}

// ------------------------------------------------------------------ scan
// Three-kernel exclusive scan: per-block totals, a single-block scan of the
// totals, then per-block scans with the block offsets added.
constexpr int SCAN_BS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BS * SCAN_ITEMS;

__device__ __forceinline__ int block_exclusive_sum(int v, int *smem_warp, int *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) smem_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? smem_warp[lane] : 0;
        int wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            int t = __shfl_up_sync(FULL, wi, o);
            if (lane >= o) wi += t;
        }
        if (lane < nw) smem_warp[lane] = wi - w;
        if (lane == nw - 1) smem_warp[32] = wi;
    }
    __syncthreads();
    int r = smem_warp[warp] + incl - v;
    if (total) *total = smem_warp[32];
    __syncthreads();
    return r;
}

__global__ void k_scan_reduce(const int32_t *in, int64_t count, int32_t *bsum)
{
    __shared__ int sw[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k)
        if (base + k < count) s += in[base + k];
    int total;
    block_exclusive_sum(s, sw, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_spine(int32_t *bsum, int64_t nb, int32_t *total_out)
{
    __shared__ int sw[33];
    int carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
        int64_t i = b0 + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int ex = block_exclusive_sum(v, sw, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

__global__ void k_scan_down(const int32_t *in, int32_t *out, int64_t count, const int32_t *boff)
{
    __shared__ int sw[33];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int v[SCAN_ITEMS];
    int s = 0;
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        v[k] = base + k < count ? in[base + k] : 0;
        s += v[k];
    }
    int ex = block_exclusive_sum(s, sw, nullptr) + boff[blockIdx.x];
#pragma unroll
    for (int k = 0; k < SCAN_ITEMS; ++k) {
        if (base + k < count) out[base + k] = ex;
        ex += v[k];
    }
}

pr_status scan_exclusive(pr_graph *g, const int32_t *in, int32_t *out, int64_t count,
                         cudaStream_t s)
{
    int64_t nb = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) {
        PR_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return PR_OK;
    }
    Buf tmp;
    PR_TRY(buf_alloc(g, tmp, sizeof(int32_t) * (size_t)nb, s));
    k_scan_reduce<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, count, tmp.as<int32_t>()); note_launch();
    k_scan_spine<<<1, 1024, 0, s>>>(tmp.as<int32_t>(), nb, out + count); note_launch();
    k_scan_down<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, out, count, tmp.as<int32_t>()); note_launch();
    cudaError_t e = cudaGetLastError();
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &tmp), g->owned.end());
    buf_free(g, tmp, s);
    if (e != cudaSuccess) return cuda_status(e, "scan launch", __FILE__, __LINE__);
    return PR_OK;
}

// ------------------------------------------------------------- degrees
// Out/in-degree histograms with warp-aggregated atomics (R-MAT hubs put many
// edges of one warp on the same vertex); ids outside [0, n) raise err.
__global__ void k_degrees(int64_t m, const int32_t *__restrict__ src,
                          const int32_t *__restrict__ dst, int32_t n, int32_t *outdeg,
                          int32_t *indeg, int32_t *err)
{
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e0 = (int64_t)blockIdx.x * blockDim.x; e0 < m; e0 += stride) {
        int64_t e = e0 + threadIdx.x;
        bool valid = e < m;
        int s = valid ? src[e] : 0;
        int t = valid ? dst[e] : 0;
        bool ok = valid && s >= 0 && s < n && t >= 0 && t < n;
        if (valid && !ok) atomicOr(err, 1);
        unsigned okmask = __ballot_sync(FULL, ok);
        if (ok) {
            unsigned peers = __match_any_sync(okmask, s);
            if (lane == __ffs(peers) - 1) atomicAdd(&outdeg[s], __popc(peers));
            peers = __match_any_sync(okmask, t);
            if (lane == __ffs(peers) - 1) atomicAdd(&indeg[t], __popc(peers));
        }
    }
}

// ----------------------------------------------------------- radix sort
// Stable LSD radix sort of (64-bit key, int32 value) pairs, 8 bits a pass.
// A block owns a tile of 4096 pairs; warp w owns the w-th 512-pair run and
// ranks it in 16 rounds of 32 with __match_any_sync, so the order within a
// tile is preserved.
constexpr int RS_BS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_BS * RS_ROUNDS;
constexpr int RS_WARPS = RS_BS / 32;

__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t m, int shift,
                             int32_t *counts, int nblocks)
{
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * RS_TILE;
#pragma unroll 4
    for (int j = 0; j < RS_ROUNDS; ++j) {
        int64_t i = base + (int64_t)j * RS_BS + threadIdx.x;
        if (i < m) atomicAdd(&hist[(keys[i] >> shift) & 0xFF], 1);
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * nblocks + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(RS_BS) k_radix_scatter(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, int64_t m, int shift, const int32_t *__restrict__ offsets,
    int nblocks)
{
    __shared__ int wcnt[RS_WARPS][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_BS) (&wcnt[0][0])[i] = 0;
    __syncthreads();
    const unsigned lt = (1u << lane) - 1u;
    int64_t base = (int64_t)blockIdx.x * RS_TILE + (int64_t)warp * (RS_ROUNDS * 32);
    uint64_t k[RS_ROUNDS];
    int32_t v[RS_ROUNDS];
    int rank[RS_ROUNDS];
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        int64_t i = base + j * 32 + lane;
        bool valid = i < m;
        k[j] = valid ? kin[i] : 0;
        v[j] = valid ? vin[i] : 0;
        int dg = (int)((k[j] >> shift) & 0xFF);
        unsigned vmask = __ballot_sync(FULL, valid);
        int before = 0, r = 0;
        unsigned peers = 0;
        if (valid) {
            peers = __match_any_sync(vmask, dg);
            r = __popc(peers & lt);
            before = wcnt[warp][dg];
        }
        __syncwarp();
        if (valid && r == 0) wcnt[warp][dg] = before + __popc(peers);
        __syncwarp();
        rank[j] = valid ? before + r : -1;
    }
    __syncthreads();
    {   // exclusive prefix over warps for digit threadIdx.x
        int run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            int t = wcnt[w][threadIdx.x];
            wcnt[w][threadIdx.x] = run;
            run += t;
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        if (rank[j] < 0) continue;
        int dg = (int)((k[j] >> shift) & 0xFF);
        int64_t pos = (int64_t)offsets[(int64_t)dg * nblocks + blockIdx.x] + wcnt[warp][dg] + rank[j];
        kout[pos] = k[j];
        vout[pos] = v[j];
    }
}

// Sorts (keys, vals) in place by the 8-bit digits starting at each shift in
// `shifts`; alt_k/alt_v are same-size scratch.  Result ends in keys/vals.
static pr_status radix_sort(pr_graph *g, uint64_t *keys, int32_t *vals, uint64_t *alt_k,
                            int32_t *alt_v, int64_t m, const std::vector<int> &shifts,
                            cudaStream_t s)
{
    if (m <= 1 || shifts.empty()) return PR_OK;
    int nblocks = (int)((m + RS_TILE - 1) / RS_TILE);
    int64_t ncount = (int64_t)256 * nblocks;
    Buf counts;
    PR_TRY(buf_alloc(g, counts, sizeof(int32_t) * (size_t)(ncount + 1), s));
    uint64_t *ka = keys, *kb = alt_k;
    int32_t *va = vals, *vb = alt_v;
    pr_status st = PR_OK;
    for (int sh : shifts) {
        k_radix_hist<<<nblocks, RS_BS, 0, s>>>(ka, m, sh, counts.as<int32_t>(), nblocks); note_launch();
        st = scan_exclusive(g, counts.as<int32_t>(), counts.as<int32_t>(), ncount, s);
        if (st != PR_OK) break;
        k_radix_scatter<<<nblocks, RS_BS, 0, s>>>(ka, va, kb, vb, m, sh, counts.as<int32_t>(),
                                                  nblocks); note_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    cudaError_t e = cudaGetLastError();
    if (st == PR_OK && e != cudaSuccess) st = cuda_status(e, "radix sort", __FILE__, __LINE__);
    if (st == PR_OK && ka != keys) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * (size_t)m,
                                         cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, va, sizeof(int32_t) * (size_t)m,
                                         cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            st = cuda_status(e1 != cudaSuccess ? e1 : e2, "radix copy", __FILE__, __LINE__);
    }
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &counts), g->owned.end());
    buf_free(g, counts, s);
    return st;
}

static std::vector<int> digit_shifts(int32_t n, int offset)
{
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    std::vector<int> out;
    for (int b = 0; b < bits; b += 8) out.push_back(offset + b);
    return out;
}

__global__ void k_make_csc_keys(int64_t m, const int32_t *__restrict__ src,
                                const int32_t *__restrict__ dst, uint64_t *keys, int32_t *vals)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    keys[e] = ((uint64_t)(uint32_t)dst[e] << 32) | (uint64_t)(uint32_t)src[e];
    vals[e] = (int32_t)e;
}

__global__ void k_split_keys(int64_t m, const uint64_t *__restrict__ keys, int32_t *low32)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) low32[i] = (int32_t)(uint32_t)(keys[i] & 0xffffffffu);
}

// key = (source << 32) | destination for every in-list slot (warp per vertex)
__global__ void k_make_csr_keys(int32_t n, const int32_t *__restrict__ col_ptr,
                                const int32_t *__restrict__ row_idx,
                                const int32_t *__restrict__ csc_eid, uint64_t *keys, int32_t *vals)
{
    const int lane = threadIdx.x & 31;
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = warp; u < n; u += nwarps) {
        int a = col_ptr[u], b = col_ptr[u + 1];
        for (int i = a + lane; i < b; i += 32) {
            keys[i] = ((uint64_t)(uint32_t)row_idx[i] << 32) | (uint64_t)(uint32_t)u;
            vals[i] = csc_eid[i];
        }
    }
}

__global__ void k_split_csr(int64_t m, const uint64_t *__restrict__ keys, int32_t *col_idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < m) col_idx[i] = (int32_t)(uint32_t)(keys[i] & 0xffffffffu);
}

// ----------------------------------------------------- per-vertex data
__global__ void k_vertex_init(int32_t n, const int32_t *__restrict__ outdeg, double *inv64,
                              float *inv32, int32_t *n_dangling)
{
    int u = blockIdx.x * blockDim.x + threadIdx.x;
    bool dang = false;
    if (u < n) {
        int k = outdeg[u];
        inv64[u] = k > 0 ? 1.0 / (double)k : 0.0;
        inv32[u] = k > 0 ? 1.0f / (float)k : 0.0f;
        dang = k == 0;
    }
    unsigned b = __ballot_sync(FULL, dang);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(n_dangling, __popc(b));
}

// ---------------------------------------------------------------- bins
// Stable three-way partition of vertex ids by in-degree.
constexpr int BIN_BS = 256;

__device__ __forceinline__ int bin_of(int deg, int t_lo, int t_hub)
{
    return deg <= t_lo ? 0 : (deg <= t_hub ? 1 : 2);
}

__global__ void k_bin_count(int32_t n, const int32_t *__restrict__ indeg, int t_lo, int t_hub,
                            int32_t *counts, int nblocks)
{
    __shared__ int c[3];
    if (threadIdx.x < 3) c[threadIdx.x] = 0;
    __syncthreads();
    int u = blockIdx.x * BIN_BS + threadIdx.x;
    if (u < n) atomicAdd(&c[bin_of(indeg[u], t_lo, t_hub)], 1);
    __syncthreads();
    if (threadIdx.x < 3) counts[threadIdx.x * nblocks + blockIdx.x] = c[threadIdx.x];
}

__global__ void k_bin_scatter(int32_t n, const int32_t *__restrict__ indeg, int t_lo, int t_hub,
                              const int32_t *__restrict__ offsets, int nblocks, int32_t *bins)
{
    __shared__ int wc[3][BIN_BS / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int u = blockIdx.x * BIN_BS + threadIdx.x;
    int b = u < n ? bin_of(indeg[u], t_lo, t_hub) : 3;
    unsigned masks[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        masks[c] = __ballot_sync(FULL, b == c);
        if (lane == 0) wc[c][warp] = __popc(masks[c]);
    }
    __syncthreads();
    if (b < 3) {
        int before = 0;
        for (int w = 0; w < warp; ++w) before += wc[b][w];
        int pos = offsets[b * nblocks + blockIdx.x] + before + __popc(masks[b] & ((1u << lane) - 1u));
        bins[pos] = u;
    }
}

__global__ void k_hub_segments(int32_t nhub, const int32_t *__restrict__ hubs,
                               const int32_t *__restrict__ indeg, int hub_seg, int32_t *nseg)
{
    int h = blockIdx.x * blockDim.x + threadIdx.x;
    if (h < nhub) nseg[h] = (indeg[hubs[h]] + hub_seg - 1) / hub_seg;
}

pr_tune effective_tune(const pr_graph *g, const pr_tune *t)
{
    pr_tune r = g->tune;
    if (t) {
        if (t->t_lo > 0) r.t_lo = t->t_lo;
        if (t->t_hub > 0) r.t_hub = t->t_hub;
        if (t->hub_seg > 0) r.hub_seg = t->hub_seg;
        if (t->low_rounds > 0) r.low_rounds = t->low_rounds;
        if (t->mid_per_warp > 0) r.mid_per_warp = t->mid_per_warp;
        r.deterministic_gs = t->deterministic_gs;
    }
    if (r.t_hub < r.t_lo) r.t_hub = r.t_lo;
    if (r.hub_seg < 256) r.hub_seg = 256;
    return r;
}

// (Re)computes the bins and hub segments for the given thresholds.
pr_status ensure_items(pr_graph *g, const pr_tune &t, cudaStream_t s)
{
    Items &it = g->items;
    it.low_rounds = std::max(1, std::min(8, (int)t.low_rounds));
    it.mid_per_warp = std::max(1, std::min(16, (int)t.mid_per_warp));
    if (it.t_lo == t.t_lo && it.t_hub == t.t_hub && it.hub_seg == t.hub_seg) return PR_OK;
    const int32_t n = g->n;
    int nb = (n + BIN_BS - 1) / BIN_BS;
    Buf counts;
    PR_TRY(buf_alloc(g, counts, sizeof(int32_t) * (size_t)(3 * nb + 1), s));
    PR_TRY(buf_alloc(g, it.bins, sizeof(int32_t) * (size_t)n, s));
    k_bin_count<<<nb, BIN_BS, 0, s>>>(n, g->indeg.as<int32_t>(), t.t_lo, t.t_hub,
                                      counts.as<int32_t>(), nb); note_launch();
    PR_LAUNCH_CHECK();
    // keep the per-class totals: counts of class c start at c * nb
    std::vector<int32_t> h_counts(3 * nb);
    PR_CUDA(cudaMemcpyAsync(h_counts.data(), counts.p, sizeof(int32_t) * 3 * nb,
                            cudaMemcpyDeviceToHost, s));
    PR_TRY(scan_exclusive(g, counts.as<int32_t>(), counts.as<int32_t>(), 3 * (int64_t)nb, s));
    k_bin_scatter<<<nb, BIN_BS, 0, s>>>(n, g->indeg.as<int32_t>(), t.t_lo, t.t_hub,
                                        counts.as<int32_t>(), nb, it.bins.as<int32_t>()); note_launch();
    PR_LAUNCH_CHECK();
    PR_CUDA(cudaStreamSynchronize(s));
    int64_t c3[3] = {0, 0, 0};
    for (int c = 0; c < 3; ++c)
        for (int b = 0; b < nb; ++b) c3[c] += h_counts[c * nb + b];
    it.nlow = (int32_t)c3[0];
    it.nmid = (int32_t)c3[1];
    it.nhub = (int32_t)c3[2];
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &counts), g->owned.end());
    buf_free(g, counts, s);

    // hub segments
    PR_TRY(buf_alloc(g, it.hubseg_start, sizeof(int32_t) * (size_t)(it.nhub + 1), s));
    PR_TRY(buf_alloc(g, it.hub_cnt, sizeof(int32_t) * (size_t)std::max(it.nhub, 1), s));
    PR_CUDA(cudaMemsetAsync(it.hub_cnt.p, 0, sizeof(int32_t) * (size_t)std::max(it.nhub, 1), s));
    it.nhubseg = 0;
    if (it.nhub > 0) {
        const int32_t *hubs = it.bins.as<int32_t>() + it.nlow + it.nmid;
        k_hub_segments<<<(it.nhub + 255) / 256, 256, 0, s>>>(it.nhub, hubs, g->indeg.as<int32_t>(),
                                                            t.hub_seg, it.hubseg_start.as<int32_t>()); note_launch();
        PR_LAUNCH_CHECK();
        PR_TRY(scan_exclusive(g, it.hubseg_start.as<int32_t>(), it.hubseg_start.as<int32_t>(),
                              it.nhub, s));
        int32_t total = 0;
        PR_CUDA(cudaMemcpyAsync(&total, it.hubseg_start.as<int32_t>() + it.nhub, sizeof(int32_t),
                                cudaMemcpyDeviceToHost, s));
        PR_CUDA(cudaStreamSynchronize(s));
        it.nhubseg = total;
    }
    PR_TRY(buf_alloc(g, it.seg_acc, sizeof(double) * (size_t)std::max(it.nhubseg, 1), s));
    it.t_lo = t.t_lo;
    it.t_hub = t.t_hub;
    it.hub_seg = t.hub_seg;
    return PR_OK;
}

// Builds the out-lists from the in-lists: the in-list stream is ordered by
// (dst, src, id); a stable sort by src gives (src, dst, id).
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
                                                            g->csr_eid.as<int32_t>()); note_launch();
        st = radix_sort(g, k1.as<uint64_t>(), g->csr_eid.as<int32_t>(), k2.as<uint64_t>(),
                        v2.as<int32_t>(), m, digit_shifts(n, 32), s);
    }
    if (st == PR_OK) {
        k_split_csr<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, k1.as<uint64_t>(),
                                                                g->col_idx.as<int32_t>()); note_launch();
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_status(e, "csr split", __FILE__, __LINE__);
    }
    for (Buf *b : {&k1, &k2, &v2}) {
        g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), b), g->owned.end());
        buf_free(g, *b, s);
    }
    if (st == PR_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_status(e, "csr build", __FILE__, __LINE__);
    }
    return st;
}

static void destroy_impl(pr_graph *g);

// Row sums of raw weights in out-list order and P per in-list slot.
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

__global__ void k_csc_p(int64_t m, const int32_t *__restrict__ row_idx,
                        const int32_t *__restrict__ csc_eid, const float *__restrict__ w,
                        const double *__restrict__ rowsum, double *p64, float *p32)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= m) return;
    double p = (double)w[csc_eid[q]] / rowsum[row_idx[q]];
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
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    pr_graph *g = new pr_graph();
    g->n = n;
    g->m = m;
    g->mem.stream = s;
    if (alloc) {
        g->mem.hooks = *alloc;
        g->mem.has_hooks = true;
    }
    g->tune.t_lo = 8;
    g->tune.t_hub = 2048;
    g->tune.hub_seg = 8192;
    g->tune.low_rounds = 4;
    g->tune.mid_per_warp = 4;
    g->tune.deterministic_gs = 0;

    auto fail = [&](pr_status st) {
        destroy_impl(g);
        return st;
    };
    cudaError_t e = cudaGetDevice(&g->device);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaGetDevice", __FILE__, __LINE__));
    e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e != cudaSuccess) return fail(cuda_status(e, "device query", __FILE__, __LINE__));

    pr_status st = PR_OK;
    const size_t mm = (size_t)std::max<int64_t>(m, 1);
    for (auto pb : {std::make_pair(&g->outdeg, sizeof(int32_t) * (size_t)n),
                    std::make_pair(&g->indeg, sizeof(int32_t) * (size_t)n),
                    std::make_pair(&g->col_ptr, sizeof(int32_t) * (size_t)(n + 1)),
                    std::make_pair(&g->row_idx, sizeof(int32_t) * mm),
                    std::make_pair(&g->csc_eid, sizeof(int32_t) * mm),
                    std::make_pair(&g->inv64, sizeof(double) * (size_t)n),
                    std::make_pair(&g->inv32, sizeof(float) * (size_t)n),
                    std::make_pair(&g->state, 2 * sizeof(SolveState) + 64)}) {
        st = buf_alloc(g, *pb.first, pb.second, s);
        if (st != PR_OK) return fail(st);
    }
    e = cudaMallocHost(&g->host_state, 2 * sizeof(SolveState) + 64);
    if (e != cudaSuccess) return fail(cuda_status(e, "cudaMallocHost", __FILE__, __LINE__));
    int32_t *flags_dev = g->state.as<int32_t>();  // reuse as [err, n_dangling]
    if (cudaMemsetAsync(g->outdeg.p, 0, sizeof(int32_t) * n, s) != cudaSuccess ||
        cudaMemsetAsync(g->indeg.p, 0, sizeof(int32_t) * n, s) != cudaSuccess ||
        cudaMemsetAsync(flags_dev, 0, 2 * sizeof(int32_t), s) != cudaSuccess)
        return fail(cuda_status(cudaGetLastError(), "memset", __FILE__, __LINE__));

    if (m > 0) {
        int blocks = (int)std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 16);
        k_degrees<<<blocks, 256, 0, s>>>(m, src, dst, n, g->outdeg.as<int32_t>(),
                                         g->indeg.as<int32_t>(), flags_dev); note_launch();
        if (w) {
            k_check_weights<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, w, flags_dev);
            note_launch();
        }
    }
    k_vertex_init<<<(n + 255) / 256, 256, 0, s>>>(n, g->outdeg.as<int32_t>(), g->inv64.as<double>(),
                                                  g->inv32.as<float>(), flags_dev + 1); note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(cuda_status(e, "degree kernels", __FILE__, __LINE__));
    int32_t hflags[2] = {0, 0};
    e = cudaMemcpyAsync(hflags, flags_dev, sizeof(hflags), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_status(e, "degree check", __FILE__, __LINE__));
    if (hflags[0] & 1) {
        set_error("pr_graph_create: an edge endpoint lies outside [0, %d)", n);
        return fail(PR_ERR_INVALID_ARG);
    }
    if (hflags[0] & 2) {
        set_error("pr_graph_create: edge weights must be positive and finite");
        return fail(PR_ERR_INVALID_ARG);
    }
    g->n_dangling = hflags[1];

    st = scan_exclusive(g, g->indeg.as<int32_t>(), g->col_ptr.as<int32_t>(), n, s);
    if (st != PR_OK) return fail(st);

    if (m > 0) {
        Buf k1, k2, v2;
        st = buf_alloc(g, k1, sizeof(uint64_t) * (size_t)m, s);
        if (st == PR_OK) st = buf_alloc(g, k2, sizeof(uint64_t) * (size_t)m, s);
        if (st == PR_OK) st = buf_alloc(g, v2, sizeof(int32_t) * (size_t)m, s);
        if (st == PR_OK) {
            k_make_csc_keys<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
                m, src, dst, k1.as<uint64_t>(), g->csc_eid.as<int32_t>()); note_launch();
            std::vector<int> shifts = digit_shifts(n, 0);
            for (int sh : digit_shifts(n, 32)) shifts.push_back(sh);
            st = radix_sort(g, k1.as<uint64_t>(), g->csc_eid.as<int32_t>(), k2.as<uint64_t>(),
                            v2.as<int32_t>(), m, shifts, s);
        }
        if (st == PR_OK) {
            k_split_keys<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(m, k1.as<uint64_t>(),
                                                                     g->row_idx.as<int32_t>()); note_launch();
            e = cudaGetLastError();
            if (e != cudaSuccess) st = cuda_status(e, "csc split", __FILE__, __LINE__);
        }
        for (Buf *b : {&k1, &k2, &v2}) {
            g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), b), g->owned.end());
            buf_free(g, *b, s);
        }
        if (st != PR_OK) return fail(st);
    }

    st = ensure_items(g, effective_tune(g, nullptr), s);
    if (st != PR_OK) return fail(st);
    if ((flags & PR_BUILD_CSR) || w) {
        st = ensure_csr(g, s);
        if (st != PR_OK) return fail(st);
    }
    if (w && m > 0) {
        g->weighted = true;
        for (auto pb : {std::make_pair(&g->w, sizeof(float) * (size_t)m),
                        std::make_pair(&g->rowsum, sizeof(double) * (size_t)n),
                        std::make_pair(&g->p64_csc, sizeof(double) * (size_t)m),
                        std::make_pair(&g->p32_csc, sizeof(float) * (size_t)m)}) {
            st = buf_alloc(g, *pb.first, pb.second, s);
            if (st != PR_OK) return fail(st);
        }
        e = cudaMemcpyAsync(g->w.p, w, sizeof(float) * (size_t)m, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(cuda_status(e, "weights copy", __FILE__, __LINE__));
        k_rowsum<<<(n + 255) / 256, 256, 0, s>>>(n, g->row_ptr.as<int32_t>(),
                                                 g->csr_eid.as<int32_t>(), g->w.as<float>(),
                                                 g->rowsum.as<double>()); note_launch();
        k_csc_p<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(
            m, g->row_idx.as<int32_t>(), g->csc_eid.as<int32_t>(), g->w.as<float>(),
            g->rowsum.as<double>(), g->p64_csc.as<double>(), g->p32_csc.as<float>()); note_launch();
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(cuda_status(e, "weights", __FILE__, __LINE__));
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(cuda_status(e, "graph build", __FILE__, __LINE__));
    *out = g;
    return PR_OK;
}

namespace fpr {
static void destroy_impl(pr_graph *g)
{
    if (!g) return;
    cudaStream_t s = g->mem.stream;
    cudaStreamSynchronize(s);
    release_graphs(g);
    for (Buf *b : g->owned) buf_free(g, *b, s);
    buf_free(g, g->items.bins, s);
    cudaStreamSynchronize(s);
    if (g->host_state) cudaFreeHost(g->host_state);
    cudaGetLastError();
    delete g;
}
}  // namespace fpr

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
                                     double *inv_outdeg, int32_t *bins, void *stream)
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
    PR_TRY(cp(bins, g->items.bins, 4 * n));
    PR_CUDA(cudaStreamSynchronize(s));
    return PR_OK;
}
