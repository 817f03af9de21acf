// primitives.cu -- building blocks of the device graph build (the paper's
// Sec. 3 storage): error reporting, allocation through the caller's hooks,
// out/in-degree histograms, exclusive scans and a stable LSD radix sort of
// (64-bit key, int32 value) pairs.  All integer work is deterministic.

#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <atomic>

#include "common.cuh"
#include "tma.cuh"

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
// Without allocator hooks, device memory comes from the library's own
// stream-ordered pool of the device, which keeps what is freed for later
// builds and solves until the process exits, like a caching allocator.  (The
// default pool hands freed memory back at every synchronisation, so each
// build mapped its temporaries again: 9.6 against 5.5 ms at R-MAT scale 22;
// trimming the pool whenever its last graph was destroyed still cost 7.5 ms
// for a build-solve-destroy loop.)
constexpr int POOL_MAX_DEVICES = 64;
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[POOL_MAX_DEVICES];

static cudaMemPool_t lib_pool(int dev)
{
    if (dev < 0 || dev >= POOL_MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pool[dev] = pool;
    }
    return g_pool[dev];
}

void *Mem::alloc(size_t bytes, cudaStream_t s)
{
    if (bytes == 0) bytes = 16;
    if (has_hooks) return hooks.alloc(bytes, reinterpret_cast<void *>(s), hooks.ctx);
    void *p = nullptr;
    int device = 0;
    cudaGetDevice(&device);  // the graph's device (checked by every entry point)
    cudaMemPool_t pool = lib_pool(device);
    const cudaError_t e =
        pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMallocAsync(&p, bytes, s);
    if (e != cudaSuccess) {
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

// ------------------------------------------------- scan without allocation
// Block totals of pr_scan_exclusive_noalloc live in this fixed array (one
// copy per device, 256 KB) instead of allocated scratch.  Every call on a
// device uses the same array, so calls must not overlap in time.
constexpr int64_t NOALLOC_SCAN_BLOCKS = 65536;
static __device__ __align__(256) int32_t g_scan_blocks[NOALLOC_SCAN_BLOCKS];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_scan_mu;
static int32_t *g_scan_addr[NOALLOC_MAX_DEVICES];  // device address, per device

}  // namespace fpr

extern "C" pr_status pr_scan_exclusive_noalloc(const int32_t *in, int32_t *out, int64_t count,
                                               void *stream)
{
    using namespace fpr;
    if (count < 0 || !out || (count > 0 && !in)) {
        set_error("pr_scan_exclusive_noalloc: need count >= 0, in (if count > 0) and out");
        return PR_ERR_INVALID_ARG;
    }
    if (count > NOALLOC_SCAN_BLOCKS * SCAN_TILE) {
        set_error("pr_scan_exclusive_noalloc: count %lld exceeds the limit %lld",
                  (long long)count, (long long)(NOALLOC_SCAN_BLOCKS * SCAN_TILE));
        return PR_ERR_INVALID_ARG;
    }
    int dev = -1;
    PR_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("pr_scan_exclusive_noalloc: device %d out of range", dev);
        return PR_ERR_UNSUPPORTED;
    }
    int32_t *scratch;
    {
        std::lock_guard<std::mutex> lock(g_scan_mu);
        if (!g_scan_addr[dev]) {
            void *p = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&p, g_scan_blocks);
            if (e != cudaSuccess)
                return cuda_status(e, "cudaGetSymbolAddress(scan scratch)", __FILE__, __LINE__);
            g_scan_addr[dev] = static_cast<int32_t *>(p);
        }
        scratch = g_scan_addr[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t nb = (count + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 0) {
        PR_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), s));
        return PR_OK;
    }
    k_scan_reduce<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, count, scratch);
    note_launch();
    k_scan_spine<<<1, 1024, 0, s>>>(scratch, nb, out + count);
    note_launch();
    k_scan_down<<<(unsigned)nb, SCAN_BS, 0, s>>>(in, out, count, scratch);
    note_launch();
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}

namespace fpr {

// ------------------------------------------------------------- degrees
// Degrees from keys sorted by one endpoint (the high or the low word): each
// run of equal ids adds its length (end - start, written by the threads at
// its two ends); with `low32` also the low words (the in-list sources).
__global__ void k_run_degrees(int64_t m, const uint64_t *__restrict__ keys, int high,
                              int32_t *deg, int32_t *low32)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t k = keys[i];
        const uint32_t v = high ? (uint32_t)(k >> 32) : (uint32_t)k;
        if (low32) low32[i] = (int32_t)(uint32_t)k;
        const bool first = i == 0 || (high ? (uint32_t)(keys[i - 1] >> 32) : (uint32_t)keys[i - 1]) != v;
        const bool last = i == m - 1 || (high ? (uint32_t)(keys[i + 1] >> 32) : (uint32_t)keys[i + 1]) != v;
        if (first) atomicSub(&deg[v], (int32_t)i);
        if (last) atomicAdd(&deg[v], (int32_t)(i + 1));
    }
}

// ----------------------------------------------------------- radix sort
// Stable LSD radix sort of (64-bit key, int32 value) pairs, 8 bits a pass.
// Per pass: per-tile digit counts (tiles of 4096 pairs), one exclusive scan
// of them in digit-major order (the output start of each (digit, tile)),
// then the scatter: persistent blocks take tiles round-robin; a block ranks
// its tile by digit (stable: warp w ranks the w-th 512-pair run in 16 rounds
// of 32, a lane's peers found with one ballot per digit bit), reorders it by
// digit in shared memory and writes each digit's run to its place, while
// the bulk copy (TMA) of its next tile lands in shared memory.  Every copy
// wait is bounded.
constexpr int RS_BS = 256;
constexpr int RS_ROUNDS = 16;
constexpr int RS_TILE = RS_BS * RS_ROUNDS;
constexpr int RS_WARPS = RS_BS / 32;
constexpr int RS_BLOCKS_PER_SM = 2;
constexpr uint32_t RS_WAIT_LIMIT = 1u << 22;

// Digit counts of tile blockIdx.x: all 16 keys of a thread are loaded
// (streaming, read once) before the shared-memory increments.
__global__ void k_radix_hist(const uint64_t *__restrict__ keys, int64_t m, int shift,
                             int32_t *counts, int64_t ntiles, unsigned *used)
{
    __shared__ int hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    int dg[RS_ROUNDS];
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j) {
        const int64_t i = base + (int64_t)j * RS_BS + threadIdx.x;
        dg[j] = i < m ? (int)((__ldcs(keys + i) >> shift) & 0xFF) : -1;
    }
#pragma unroll
    for (int j = 0; j < RS_ROUNDS; ++j)
        if (dg[j] >= 0) atomicAdd(&hist[dg[j]], 1);
    __syncthreads();
    const int c = hist[threadIdx.x];
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = c;
    // OR of the digits present (the scatter picks its ranking method by it);
    // an atomic only where it adds a bit, so the word does not serialise
    // every block
    const unsigned o = __reduce_or_sync(FULL, c ? (unsigned)threadIdx.x : 0u);
    if ((threadIdx.x & 31) == 0 && (o & ~__ldcg(used))) atomicOr(used, o);
}

struct RadixSmem {
    uint64_t ik[RS_TILE];  // next tile, landed by the bulk copy
    int32_t iv[RS_TILE];
    uint64_t ok[RS_TILE];  // the current tile reordered by digit
    int32_t ov[RS_TILE];
    int wcnt[RS_WARPS][256];
    int bstart[256];
    int dbase[256];  // output position of reordered slot q: dbase[digit] + q
    int sw[33];
    uint64_t bar;
    int bad;
};

__global__ void __launch_bounds__(RS_BS, RS_BLOCKS_PER_SM) k_radix_scatter(
    const uint64_t *__restrict__ kin, const int32_t *__restrict__ vin, uint64_t *__restrict__ kout,
    int32_t *__restrict__ vout, int64_t m, int shift, const int32_t *__restrict__ offsets,
    int32_t *err, const unsigned *used)
{
    extern __shared__ __align__(16) unsigned char rs_smem[];
    RadixSmem &sm = *reinterpret_cast<RadixSmem *>(rs_smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const bool few = *used < 64u;  // every digit of this pass below 64
    const int64_t ntiles = (m + RS_TILE - 1) / RS_TILE;
    auto is_full = [&](int64_t t) { return t < ntiles && (t + 1) * RS_TILE <= m; };
    // a full tile arrives by bulk copy (16-byte aligned, 48 KB), the last
    // partial one by plain loads
    auto issue = [&](int64_t t) {
        if (is_full(t)) {
            mbar_expect_tx(&sm.bar, RS_TILE * 12);
            bulk_load(sm.ik, kin + t * RS_TILE, RS_TILE * 8, &sm.bar);
            bulk_load(sm.iv, vin + t * RS_TILE, RS_TILE * 4, &sm.bar);
        }
    };
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        mbar_init_fence();
        sm.bad = 0;
        issue(blockIdx.x);
    }
    __syncthreads();
    uint32_t parity = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        const int64_t tile0 = t * RS_TILE;
        const bool full = is_full(t);
        const int nvalid = (int)min((int64_t)RS_TILE, m - tile0);
        if (full) {
            if (!mbar_wait(&sm.bar, parity, RS_WAIT_LIMIT)) {
                atomicOr(err, 1);
                sm.bad = 1;
            }
            parity ^= 1;
        }
        for (int i = threadIdx.x; i < RS_WARPS * 256; i += RS_BS) (&sm.wcnt[0][0])[i] = 0;
        // this tile's output start of digit threadIdx.x
        const int dstart = offsets[(int64_t)threadIdx.x * ntiles + t];
        uint64_t k[RS_ROUNDS];
        int32_t v[RS_ROUNDS];
        int rank[RS_ROUNDS];
#pragma unroll
        for (int j = 0; j < RS_ROUNDS; ++j) {
            const int q = warp * (RS_ROUNDS * 32) + j * 32 + lane;
            const bool valid = q < nvalid;
            k[j] = valid ? (full ? sm.ik[q] : kin[tile0 + q]) : 0;
            v[j] = valid ? (full ? sm.iv[q] : vin[tile0 + q]) : 0;
        }
        __syncthreads();  // input buffer read, counters zero
        if (sm.bad) {
            // the copy did not land in time: wait once more (bounded) for it
            // before leaving, so nothing is in flight at exit
            mbar_wait(&sm.bar, parity ^ 1, RS_WAIT_LIMIT);
            break;
        }
        if (threadIdx.x == 0) {
            fence_async_smem();
            issue(t + gridDim.x);
        }
#pragma unroll
        for (int j = 0; j < RS_ROUNDS; ++j) {
            const bool valid = warp * (RS_ROUNDS * 32) + j * 32 + lane < nvalid;
            const int dg = (int)((k[j] >> shift) & 0xFF);
            // the valid lanes with this lane's digit: with at most 64
            // digits present in the pass, match.any; else one ballot per
            // digit bit (match.any kept the SM's address-divergence unit 80%
            // busy on full 8-bit digits and bound the pass; it is the faster
            // of the two when most lanes share few digits)
            const unsigned vmask = __ballot_sync(FULL, valid);
            unsigned peers;
            if (few) {
                peers = valid ? __match_any_sync(vmask, dg) : 0u;
            } else {
                peers = vmask;
#pragma unroll
                for (int b = 0; b < 8; ++b) {
                    const bool bit = (dg >> b) & 1;
                    const unsigned mb = __ballot_sync(FULL, bit);
                    peers &= bit ? mb : ~mb;
                }
            }
            int before = 0, r = 0;
            if (valid) {
                r = __popc(peers & lt);
                before = sm.wcnt[warp][dg];
            }
            __syncwarp();
            if (valid && r == 0) sm.wcnt[warp][dg] = before + __popc(peers);
            __syncwarp();
            rank[j] = valid ? before + r : -1;
        }
        __syncthreads();
        {   // digit d = threadIdx.x: prefix over warps, then over digits
            const int d = threadIdx.x;
            int run = 0;
#pragma unroll
            for (int w = 0; w < RS_WARPS; ++w) {
                const int c = sm.wcnt[w][d];
                sm.wcnt[w][d] = run;
                run += c;
            }
            const int bst = block_exclusive_sum(run, sm.sw, nullptr);
            sm.bstart[d] = bst;
            sm.dbase[d] = dstart - bst;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RS_ROUNDS; ++j) {
            if (rank[j] < 0) continue;
            const int dg = (int)((k[j] >> shift) & 0xFF);
            const int q = sm.bstart[dg] + sm.wcnt[warp][dg] + rank[j];
            sm.ok[q] = k[j];
            sm.ov[q] = v[j];
        }
        __syncthreads();
        for (int q = threadIdx.x; q < nvalid; q += RS_BS) {
            const uint64_t kk = sm.ok[q];
            const int64_t pos = (int64_t)sm.dbase[(kk >> shift) & 0xFF] + q;
            if (pos >= 0 && pos < m) {
                kout[pos] = kk;
                vout[pos] = sm.ov[q];
            }
        }
        __syncthreads();  // reordered tile and counters free for the next tile
    }
}

// Sorts (keys, vals) by the 8-bit digits starting at each shift in `shifts`;
// alt_k/alt_v are same-size scratch.  The result ends in keys/vals unless
// kres/vres are given (then it stays where the last pass wrote it).
pr_status radix_sort(pr_graph *g, uint64_t *keys, int32_t *vals, uint64_t *alt_k,
                     int32_t *alt_v, int64_t m, const std::vector<int> &shifts, cudaStream_t s,
                     uint64_t **kres, int32_t **vres)
{
    if (kres) *kres = keys;
    if (vres) *vres = vals;
    if (m <= 1 || shifts.empty()) return PR_OK;
    if ((reinterpret_cast<uintptr_t>(keys) | reinterpret_cast<uintptr_t>(vals) |
         reinterpret_cast<uintptr_t>(alt_k) | reinterpret_cast<uintptr_t>(alt_v)) & 15) {
        set_error("radix_sort: buffers must be 16-byte aligned (bulk copies)");
        return PR_ERR_INVALID_ARG;
    }
    const int64_t ntiles = (m + RS_TILE - 1) / RS_TILE;
    const int64_t ncount = 256 * ntiles;
    // scratch: counts [256][ntiles] (+ total), error word, one word per pass
    // for the OR of the digits present
    Buf scratch;
    PR_TRY(buf_alloc(g, scratch, sizeof(int32_t) * (size_t)(ncount + 2 + shifts.size()), s));
    int32_t *counts = scratch.as<int32_t>();
    int32_t *err = counts + ncount + 1;
    unsigned *used = reinterpret_cast<unsigned *>(counts + ncount + 2);
    pr_status st = PR_OK;
    cudaError_t e = cudaMemsetAsync(err, 0, sizeof(int32_t) * (1 + shifts.size()), s);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_radix_scatter),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(RadixSmem));
    uint64_t *ka = keys, *kb = alt_k;
    int32_t *va = vals, *vb = alt_v;
    const unsigned grid = (unsigned)std::min<int64_t>(ntiles, (int64_t)g->num_sms * RS_BLOCKS_PER_SM);
    for (size_t p = 0; p < shifts.size() && e == cudaSuccess && st == PR_OK; ++p) {
        k_radix_hist<<<(unsigned)ntiles, RS_BS, 0, s>>>(ka, m, shifts[p], counts, ntiles,
                                                        used + p);
        note_launch();
        st = scan_exclusive(g, counts, counts, ncount, s);
        if (st != PR_OK) break;
        k_radix_scatter<<<grid, RS_BS, sizeof(RadixSmem), s>>>(ka, va, kb, vb, m, shifts[p],
                                                             counts, err, used + p);
        note_launch();
        std::swap(ka, kb);
        std::swap(va, vb);
        e = cudaGetLastError();
    }
    int32_t herr = 0;
    if (st == PR_OK && e == cudaSuccess)
        e = cudaMemcpyAsync(&herr, err, sizeof(herr), cudaMemcpyDeviceToHost, s);
    if (st == PR_OK && e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (st == PR_OK && e != cudaSuccess) st = cuda_status(e, "radix sort", __FILE__, __LINE__);
    if (st == PR_OK && herr) {
        set_error("radix_sort: a bounded copy wait gave up");
        st = PR_ERR_TIMEOUT;
    }
    if (st == PR_OK && kres) {  // the caller takes the result where it ends
        *kres = ka;
        *vres = va;
    } else if (st == PR_OK && ka != keys) {
        cudaError_t e1 = cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * (size_t)m,
                                         cudaMemcpyDeviceToDevice, s);
        cudaError_t e2 = cudaMemcpyAsync(vals, va, sizeof(int32_t) * (size_t)m,
                                         cudaMemcpyDeviceToDevice, s);
        if (e1 != cudaSuccess || e2 != cudaSuccess)
            st = cuda_status(e1 != cudaSuccess ? e1 : e2, "radix copy", __FILE__, __LINE__);
    }
    g->owned.erase(std::remove(g->owned.begin(), g->owned.end(), &scratch), g->owned.end());
    buf_free(g, scratch, s);
    return st;
}

std::vector<int> digit_shifts(int32_t n, int offset)
{
    int bits = 0;
    while (bits < 31 && ((int64_t)1 << bits) < (int64_t)n) ++bits;
    std::vector<int> out;
    for (int b = 0; b < bits; b += 8) out.push_back(offset + b);
    return out;
}

// key = (dst << 32) | src, value = input position; ids outside [0, n) set
// bit 0 of err.
__global__ void k_make_csc_keys(int64_t m, const int32_t *__restrict__ src,
                                const int32_t *__restrict__ dst, int32_t n, uint64_t *keys,
                                int32_t *vals, int32_t *err)
{
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= m) return;
    const int32_t a = src[e], b = dst[e];
    if (a < 0 || a >= n || b < 0 || b >= n) atomicOr(err, 1);
    keys[e] = ((uint64_t)(uint32_t)b << 32) | (uint64_t)(uint32_t)a;
    vals[e] = (int32_t)e;
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


}  // namespace fpr
