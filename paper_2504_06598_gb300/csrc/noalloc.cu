// noalloc.cu -- hierarchy build that allocates no device memory.
//
// Same kernels and results as gs_build_bvh, for callers that must not call
// cudaMalloc: the caller passes the output buffers, and the build scratch
// (sort keys and ids, parents, arrival counters, boxes, histograms, scan
// block sums) lives in one file-scope __device__ array sized for at most
// kNoAllocMaxGaussians Gaussians. Every GPU that loads this library holds
// that array (about 4 MB) until the process exits. The caller's status word
// receives the build's error bits, so it is required: with no word of its
// own a caller would never learn of a non-finite parameter.
#include <cuda_runtime.h>

#include <mutex>

#include "gsrt_internal.cuh"

namespace gsrt {
namespace {

constexpr int64_t kNoAllocMaxGaussians = 65536;
constexpr size_t kAlign = 256;

constexpr size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Byte offsets of the pieces of the scratch array.
constexpr size_t kCodes0 = 0;
constexpr size_t kCodes1 = kCodes0 + align_up(8 * kNoAllocMaxGaussians);
constexpr size_t kVals0 = kCodes1 + align_up(8 * kNoAllocMaxGaussians);
constexpr size_t kVals1 = kVals0 + align_up(4 * kNoAllocMaxGaussians);
constexpr size_t kParent = kVals1 + align_up(4 * kNoAllocMaxGaussians);
constexpr size_t kArrive = kParent + align_up(4 * (2 * kNoAllocMaxGaussians + 2));
constexpr size_t kAabb = kArrive + align_up(4 * kNoAllocMaxGaussians);
constexpr size_t kBounds = kAabb + align_up(24 * kNoAllocMaxGaussians);
constexpr size_t kHist = kBounds + align_up(64);
constexpr size_t kHistEntries = 256 * ((kNoAllocMaxGaussians + 2047) / 2048);
constexpr size_t kScanTmp = kHist + align_up(4 * kHistEntries);
constexpr size_t kScanTmpEntries = kHistEntries / 1024 + 2;
constexpr size_t kScratchBytes = kScanTmp + align_up(4 * kScanTmpEntries);

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the symbol's host-side name is not a device address). With
// CUDA's lazy module loading this first lookup is also what loads the
// library's module on that device, which can allocate and synchronise; the
// cached address is that of the device's primary context and is stale after
// a cudaDeviceReset.
gs_status scratch_address(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(GS_ERR_CUDA, "device index %d too large", dev);
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the build scratch");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
    return GS_OK;
}

}  // namespace
}  // namespace gsrt

using namespace gsrt;

extern "C" gs_status gs_build_bvh_noalloc(const gs_gaussians *g, void *nodes_out,
                                          void *prims_out, uint32_t *status_out, void *stream) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->M < 0) return fail(GS_ERR_INVALID_ARG, "M=%lld is negative", (long long)g->M);
    if (g->M > kNoAllocMaxGaussians)
        return fail(GS_ERR_INVALID_ARG,
                    "M=%lld exceeds the %lld Gaussians this allocation-free build supports; "
                    "use gs_build_bvh",
                    (long long)g->M, (long long)kNoAllocMaxGaussians);
    if (g->M == 0) return GS_OK;
    if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits)
        return fail(GS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
    if (!nodes_out || !prims_out) return fail(GS_ERR_INVALID_ARG, "nodes_out or prims_out is NULL");
    if (((uintptr_t)nodes_out & 15u) || ((uintptr_t)prims_out & 15u))
        return fail(GS_ERR_INVALID_ARG, "nodes_out and prims_out must be 16-byte aligned");
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(GS_ERR_NO_DEVICE, "no CUDA device available");
    }
    const void *ptrs[6] = {g->means, g->log_scales, g->quats, g->opacity_logits, nodes_out,
                           prims_out};
    for (const void *p : ptrs)
        if (!is_device_ptr(p)) return fail(GS_ERR_INVALID_ARG, "an argument is not a device pointer");
    if (!status_out)
        return fail(GS_ERR_INVALID_ARG,
                    "status_out is NULL: the build reports non-finite parameters through it");
    if (!is_device_ptr(status_out))
        return fail(GS_ERR_INVALID_ARG, "status_out is not a device pointer");

    unsigned char *s = nullptr;
    gs_status st = scratch_address(&s);
    if (st != GS_OK) return st;
    gs_bvh b = {};
    cudaGetDevice(&b.device);
    b.capacity = kNoAllocMaxGaussians;
    b.nodes = static_cast<Node *>(nodes_out);
    b.prims = static_cast<PrimRec *>(prims_out);
    b.codes[0] = reinterpret_cast<unsigned long long *>(s + kCodes0);
    b.codes[1] = reinterpret_cast<unsigned long long *>(s + kCodes1);
    b.vals[0] = reinterpret_cast<uint32_t *>(s + kVals0);
    b.vals[1] = reinterpret_cast<uint32_t *>(s + kVals1);
    b.parent = reinterpret_cast<uint32_t *>(s + kParent);
    b.arrive = reinterpret_cast<uint32_t *>(s + kArrive);
    b.aabb = reinterpret_cast<float *>(s + kAabb);
    b.bounds = reinterpret_cast<unsigned int *>(s + kBounds);
    b.hist = reinterpret_cast<uint32_t *>(s + kHist);
    b.hist_len = (int64_t)kHistEntries;
    b.scan_tmp = reinterpret_cast<uint32_t *>(s + kScanTmp);
    b.node_format = GS_NODES_BINARY;
    b.status = status_out;
    return build_into(&b, g, (cudaStream_t)stream);
}
