// probe.cu -- pr_gather_probe: the sweep's irregular gathers alone (sum of
// y[idx[j]] over an index stream), a measured ceiling for the gather part of
// a sweep on this device.  Diagnostic; it computes nothing of the method.
//
// Same access pattern as the sweep: 16-byte index loads kept out of L1 and
// first out of L2, eight gathers in flight per lane, the first `hot` entries
// of y copied to shared memory, one persistent 1024-thread block per SM.
#include "../../include/fusedpr_diag.h"
#include "common.cuh"

namespace fpr {

constexpr int PROBE_BS = 1024;

__global__ void __launch_bounds__(PROBE_BS, 1)
    k_gather_probe(const int32_t *__restrict__ idx, int64_t m, const float *__restrict__ y,
                   int32_t n, int32_t hot, float *sink)
{
    extern __shared__ float sy[];
    for (int i = threadIdx.x; i < hot; i += blockDim.x) sy[i] = y[i];
    __syncthreads();
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    float acc = 0.f;
    const int64_t nq = m >> 2;  // whole int4 groups; the tail is added below
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += 2 * stride) {
        int4 a, b = make_int4(0, 0, 0, 0);
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
            : "=r"(a.x), "=r"(a.y), "=r"(a.z), "=r"(a.w)
            : "l"(idx + 4 * q), "l"(pol));
        const bool two = q + stride < nq;
        if (two)
            asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0, %1, %2, %3}, [%4], %5;"
                : "=r"(b.x), "=r"(b.y), "=r"(b.z), "=r"(b.w)
                : "l"(idx + 4 * (q + stride)), "l"(pol));
        // an entry outside [0, n) reads y[0] instead (never out of bounds)
        int v[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int c = 0; c < 8; ++c) v[c] = (unsigned)v[c] < (unsigned)n ? v[c] : 0;
        float got[8];
#pragma unroll
        for (int c = 0; c < 8; ++c)
            got[c] = (c < 4 || two) ? (v[c] < hot ? sy[v[c]] : __ldg(y + v[c])) : 0.f;
#pragma unroll
        for (int c = 0; c < 8; ++c) acc += got[c];
    }
    for (int64_t j = 4 * nq + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
        const int v = idx[j];
        acc += __ldg(y + ((unsigned)v < (unsigned)n ? v : 0));
    }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) atomicAdd(sink, acc);
}

}  // namespace fpr

using namespace fpr;

extern "C" pr_status pr_gather_probe(const int32_t *idx, int64_t m, const float *y, int32_t n,
                                     int32_t hot, float *sink, void *stream)
{
    if (m < 0 || n < 1 || !sink || (m > 0 && (!idx || !y)) || hot < 0 || hot > n ||
        hot > 49152) {
        set_error("pr_gather_probe: need m >= 0, n >= 1, 0 <= hot <= min(n, 49152) and buffers");
        return PR_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(idx) & 15) {  // 16-byte index loads
        set_error("pr_gather_probe: idx must be 16-byte aligned");
        return PR_ERR_INVALID_ARG;
    }
    int dev = 0, sms = 0;
    PR_CUDA(cudaGetDevice(&dev));
    PR_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t smem = sizeof(float) * (size_t)hot;
    PR_CUDA(cudaFuncSetAttribute(reinterpret_cast<const void *>(&k_gather_probe),
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_gather_probe<<<sms, PROBE_BS, smem, s>>>(idx, m, y, n, hot, sink);
    note_launch();
    PR_CUDA(cudaGetLastError());
    return PR_OK;
}
