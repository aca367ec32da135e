// probe.cu -- a STREAM-style copy kernel that measures the bandwidth of one
// level of the memory hierarchy on the device it runs on, used as the
// denominator of the trace kernel's L2 roofline (the paper has no
// counterpart; it is measurement support only).
//
// Every block copies its grid-stride share of `bytes` from src to dst,
// `repeats` times, with 16-byte loads and stores that bypass L1
// (ld.global.cg / st.global.cg), four in flight per thread. With a working
// set (src + dst) well inside L2 every repeat after the first is served by
// L2, so (2 * bytes * repeats) / time is the L2 copy bandwidth; with a
// working set far beyond L2 it is the DRAM copy bandwidth. The accesses are
// volatile so the compiler keeps every repeat.
#include <cuda_runtime.h>
#include <stdint.h>

#include "gsrt_internal.cuh"

namespace gsrt {
namespace {

__device__ __forceinline__ uint4 load_cg(const uint4 *p) {
    uint4 v;
    asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ void store_cg(uint4 *p, const uint4 &v) {
    asm volatile("st.global.cg.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

constexpr int kProbeThreads = 256;
constexpr int kProbeUnroll = 4;

__global__ void __launch_bounds__(kProbeThreads) k_copy(const uint4 *__restrict__ src,
                                                        uint4 *__restrict__ dst, int64_t n,
                                                        int repeats) {
    const int64_t stride = (int64_t)gridDim.x * kProbeThreads * kProbeUnroll;
    const int64_t first = (int64_t)blockIdx.x * kProbeThreads * kProbeUnroll + threadIdx.x;
    for (int r = 0; r < repeats; ++r) {
        for (int64_t i = first; i < n; i += stride) {
            uint4 v[kProbeUnroll];
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) {
                const int64_t j = i + (int64_t)u * kProbeThreads;
                if (j < n) v[u] = load_cg(src + j);
            }
#pragma unroll
            for (int u = 0; u < kProbeUnroll; ++u) {
                const int64_t j = i + (int64_t)u * kProbeThreads;
                if (j < n) store_cg(dst + j, v[u]);
            }
        }
    }
}

}  // namespace
}  // namespace gsrt

using namespace gsrt;

extern "C" gs_status gs_probe_copy(const void *src, void *dst, int64_t bytes, int32_t repeats,
                                   void *stream) {
    if (!src || !dst) return fail(GS_ERR_INVALID_ARG, "src or dst is NULL");
    if (bytes <= 0 || (bytes & 15) != 0)
        return fail(GS_ERR_INVALID_ARG, "bytes=%lld must be a positive multiple of 16",
                    (long long)bytes);
    if (((uintptr_t)src & 15u) || ((uintptr_t)dst & 15u))
        return fail(GS_ERR_INVALID_ARG, "src and dst must be 16-byte aligned");
    if (repeats < 1 || repeats > (1 << 20))
        return fail(GS_ERR_INVALID_ARG, "repeats=%d not in 1..2^20", repeats);
    if (!is_device_ptr(src) || !is_device_ptr(dst))
        return fail(GS_ERR_INVALID_ARG, "src and dst must be device pointers");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "probe setup");
    const int64_t n = bytes / 16;
    // eight blocks of 256 threads per SM, fewer when the copy is small
    int64_t blocks = (int64_t)sms * 8;
    const int64_t need = (n + kProbeThreads * kProbeUnroll - 1) / (kProbeThreads * kProbeUnroll);
    if (blocks > need) blocks = need;
    k_copy<<<(unsigned)blocks, kProbeThreads, 0, (cudaStream_t)stream>>>(
        static_cast<const uint4 *>(src), static_cast<uint4 *>(dst), n, repeats);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "probe launch");
    return GS_OK;
}
