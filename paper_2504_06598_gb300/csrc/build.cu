// build.cu -- hierarchy construction over the Gaussians' bounding boxes
// (Sec. 3.2 builds a BVH over the boxes of Eq. 2; the paper delegates it to
// Embree/OptiX, here it is a linear BVH built on the GPU):
//   k_preprocess  box of each Gaussian's bounding ellipsoid + scene bounds
//   k_morton      63-bit key: Morton code of each mean in the scene bounds
//                 with a size class of the Gaussian's box below the top
//                 two octree levels
//   radix sort    stable LSD sort of (code, id), 8 passes of 8 bits
//   k_karras      binary radix tree over the sorted codes (Karras 2012),
//                 equal codes split by position
//   k_leaves      per-Gaussian record in tree order, then bottom-up box
//                 refit with one arrival counter per node
#include <cuda_runtime.h>
#include <math.h>

#include "gsrt_internal.cuh"

namespace gsrt {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;

// Order-preserving map float -> uint32 (for atomicMin / atomicMax).
__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

struct Activated {
    float mu[3];
    float opacity;
    float R[9];  // R_q, local to world, row-major
    float inv_s[3];
    float s[3];
    bool finite;
};

// Eq. 1 activation in float32: normalised quaternion -> rotation,
// exp of log-scales, sigmoid of the opacity logit.
__device__ __forceinline__ Activated activate(const float *means, const float *log_scales,
                                              const float *quats, const float *logits,
                                              int64_t g) {
    Activated a;
    float qw = quats[4 * g + 0], qx = quats[4 * g + 1], qy = quats[4 * g + 2],
          qz = quats[4 * g + 3];
    float n2 = qw * qw + qx * qx + qy * qy + qz * qz;
    float inv = 1.0f / sqrtf(n2);
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    a.R[0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    a.R[1] = 2.0f * (qx * qy - qw * qz);
    a.R[2] = 2.0f * (qx * qz + qw * qy);
    a.R[3] = 2.0f * (qx * qy + qw * qz);
    a.R[4] = 1.0f - 2.0f * (qx * qx + qz * qz);
    a.R[5] = 2.0f * (qy * qz - qw * qx);
    a.R[6] = 2.0f * (qx * qz - qw * qy);
    a.R[7] = 2.0f * (qy * qz + qw * qx);
    a.R[8] = 1.0f - 2.0f * (qx * qx + qy * qy);
    bool fin = isfinite(n2) && n2 > 0.0f;
    for (int k = 0; k < 3; ++k) {
        float ls = log_scales[3 * g + k];
        a.mu[k] = means[3 * g + k];
        a.s[k] = expf(ls);
        a.inv_s[k] = expf(-ls);
        fin = fin && isfinite(ls) && isfinite(a.mu[k]) && a.s[k] > 0.0f && isfinite(a.s[k]) &&
              isfinite(a.inv_s[k]);
    }
    float lg = logits[g];
    fin = fin && isfinite(lg);
    a.opacity = 1.0f / (1.0f + expf(-lg));
    a.finite = fin;
    return a;
}

// Box of the ellipsoid |S^-1 R_q^T (x - mu)| <= s: half extent along world
// axis i is s * sqrt(sum_k R_ik^2 s_k^2). Padded outward (relative 2^-10 of
// the extent plus 2^-18 of the coordinate magnitude) so that float32
// rounding in the ellipsoid and slab tests never loses a valid hit.
__device__ __forceinline__ void ellipsoid_box(const Activated &a, float box[6]) {
    const float s_cut = 2.8284271247461903f;
    for (int i = 0; i < 3; ++i) {
        float v = 0.0f;
        for (int k = 0; k < 3; ++k) {
            float r = a.R[3 * i + k] * a.s[k];
            v = fmaf(r, r, v);
        }
        float h = s_cut * sqrtf(v);
        float pad = h * 0x1p-10f + (fabsf(a.mu[i]) + h) * 0x1p-18f;
        box[i] = a.mu[i] - (h + pad);
        box[3 + i] = a.mu[i] + (h + pad);
    }
}

__global__ void k_preprocess(int64_t M, const float *__restrict__ means,
                             const float *__restrict__ log_scales, const float *__restrict__ quats,
                             const float *__restrict__ logits, float *__restrict__ aabb,
                             unsigned int *__restrict__ bounds, uint32_t *__restrict__ status) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (g < M) {
        Activated a = activate(means, log_scales, quats, logits, g);
        float box[6];
        if (a.finite) {
            ellipsoid_box(a, box);
            for (int k = 0; k < 3; ++k) {
                lo[k] = a.mu[k];
                hi[k] = a.mu[k];
            }
        } else {
            // A non-finite Gaussian gets an empty box: it is never hit.
            for (int k = 0; k < 3; ++k) {
                box[k] = NAN;
                box[3 + k] = NAN;
            }
            atomicOr(status, kErrNonfinite);
        }
        for (int k = 0; k < 6; ++k) aabb[6 * g + k] = box[k];
    }
    // warp reduction of the finite means, then one atomic per warp
    for (int k = 0; k < 3; ++k) {
        for (int off = 16; off > 0; off >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], off));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], off));
        }
    }
    if ((threadIdx.x & 31) == 0 && lo[0] <= hi[0]) {
        for (int k = 0; k < 3; ++k) {
            atomicMin(&bounds[k], f2ord(lo[k]));
            atomicMax(&bounds[3 + k], f2ord(hi[k]));
        }
    }
}

// Spread the low 21 bits of v to every third bit of a 64-bit word.
__device__ __forceinline__ unsigned long long spread3(unsigned long long v) {
    v &= 0x1fffffull;
    v = (v | (v << 32)) & 0x1f00000000ffffull;
    v = (v | (v << 16)) & 0x1f0000ff0000ffull;
    v = (v | (v << 8)) & 0x100f00f00f00f00full;
    v = (v | (v << 4)) & 0x10c30c30c30c30c3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

// Sort key of one Gaussian: its 63-bit Morton code with a 4-bit size class
// inserted below the top two octree levels (6 bits). Gaussians of very
// different extent then fall into different subtrees below the coarse
// spatial split, so a few large Gaussians no longer inflate the boxes of
// the many small ones around them. Size class = floor(-2 log2(e / E)),
// clamped to 0..15, with e the largest box edge of the Gaussian and E the
// largest edge of the bounds of the means (large Gaussians sort first).
constexpr int kKeyTopBits = 6;
constexpr int kKeySizeBits = 4;

__global__ void k_morton(int64_t M, const float *__restrict__ means,
                         const unsigned int *__restrict__ bounds, const float *__restrict__ aabb,
                         unsigned long long *__restrict__ codes, uint32_t *__restrict__ vals) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M) return;
    unsigned long long q[3];
    float scene = 0.0f, edge = 0.0f;
    for (int k = 0; k < 3; ++k) {
        float lo = ord2f(bounds[k]), hi = ord2f(bounds[3 + k]);
        float ext = hi - lo;
        scene = fmaxf(scene, ext);
        edge = fmaxf(edge, aabb[6 * g + 3 + k] - aabb[6 * g + k]);
        float x = means[3 * g + k];
        float u = (ext > 0.0f) ? (x - lo) / ext : 0.0f;
        u = fminf(fmaxf(u, 0.0f), 1.0f);  // NaN -> 0
        q[k] = (unsigned long long)(u * 2097151.0f);
    }
    const unsigned long long morton = (spread3(q[0]) << 2) | (spread3(q[1]) << 1) | spread3(q[2]);
    int cls = 0;
    if (scene > 0.0f && edge > 0.0f) {
        const float c = floorf(-2.0f * log2f(edge / scene));
        cls = (int)fminf(fmaxf(c, 0.0f), (float)((1 << kKeySizeBits) - 1));
    }
    const int low = 63 - kKeyTopBits - kKeySizeBits;
    const unsigned long long top = morton >> (63 - kKeyTopBits);
    const unsigned long long rest = (morton & ((1ull << (63 - kKeyTopBits)) - 1ull)) >> kKeySizeBits;
    codes[g] = (top << (63 - kKeyTopBits)) | ((unsigned long long)cls << low) | rest;
    vals[g] = (uint32_t)g;
}

// ---------------------------------------------------------------- radix sort

__global__ void __launch_bounds__(kSortThreads)
    k_radix_hist(int64_t n, const unsigned long long *__restrict__ keys, int shift,
                 uint32_t *__restrict__ hist, int64_t tiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = base + r * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * tiles + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan in three launches: per-block sums, a scan of the block
// sums by one block, then each block scans its own items and adds its
// block's offset. kScanItems consecutive entries per block.
constexpr int kScanItems = 1024;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = v;
    for (int off = 1; off < 32; off <<= 1) {
        uint32_t u = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += u;
    }
    if (lane == 31) warp_sums[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0u;
        for (int off = 1; off < 32; off <<= 1) {
            uint32_t u = __shfl_up_sync(0xffffffffu, w, off);
            if (lane >= off) w += u;
        }
        warp_sums[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = incl - v + (warp > 0 ? warp_sums[warp - 1] : 0u);
    if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(256) k_scan_reduce(const uint32_t *__restrict__ a, int64_t n,
                                                     uint32_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    uint32_t v = 0;
    for (int k = 0; k < kScanItems / 256; ++k) {
        const int64_t i = base + k * 256 + threadIdx.x;
        if (i < n) v += a[i];
    }
    uint32_t total = 0;
    block_exclusive_scan(v, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t *__restrict__ sums, int64_t nb) {
    const int64_t chunk = (nb + 1023) / 1024;
    const int64_t b0 = threadIdx.x * chunk, b1 = min(b0 + chunk, nb);
    uint32_t v = 0;
    for (int64_t i = b0; i < b1; ++i) v += sums[i];
    uint32_t run = block_exclusive_scan(v, nullptr);
    for (int64_t i = b0; i < b1; ++i) {
        const uint32_t t = sums[i];
        sums[i] = run;
        run += t;
    }
}

__global__ void __launch_bounds__(256) k_scan_apply(uint32_t *__restrict__ a, int64_t n,
                                                    const uint32_t *__restrict__ sums) {
    const int64_t base = (int64_t)blockIdx.x * kScanItems;
    constexpr int P = kScanItems / 256;  // items per thread, consecutive
    uint32_t v[P];
    uint32_t local = 0;
    for (int k = 0; k < P; ++k) {
        const int64_t i = base + threadIdx.x * P + k;
        v[k] = i < n ? a[i] : 0u;
        local += v[k];
    }
    uint32_t run = block_exclusive_scan(local, nullptr) + sums[blockIdx.x];
    for (int k = 0; k < P; ++k) {
        const int64_t i = base + threadIdx.x * P + k;
        if (i < n) a[i] = run;
        run += v[k];
    }
}

void scan_exclusive(uint32_t *a, int64_t n, uint32_t *sums, cudaStream_t s) {
    const int64_t nb = (n + kScanItems - 1) / kScanItems;
    k_scan_reduce<<<(unsigned)nb, 256, 0, s>>>(a, n, sums);
    k_scan_top<<<1, 1024, 0, s>>>(sums, nb);
    k_scan_apply<<<(unsigned)nb, 256, 0, s>>>(a, n, sums);
}

// Stable scatter: keys of a tile are ranked in input order, round by round
// (256 keys per round), with warp-level digit matching and a per-digit
// prefix over the warps of the block.
__global__ void __launch_bounds__(kSortThreads)
    k_radix_scatter(int64_t n, const unsigned long long *__restrict__ kin,
                    const uint32_t *__restrict__ vin, unsigned long long *__restrict__ kout,
                    uint32_t *__restrict__ vout, int shift, const uint32_t *__restrict__ offs,
                    int64_t tiles) {
    constexpr int W = kSortThreads / 32;
    __shared__ uint32_t base[256];
    __shared__ uint32_t wcount[W][256];
    __shared__ uint32_t pref[W][256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    base[tid] = offs[(int64_t)tid * tiles + blockIdx.x];
    for (int w = 0; w < W; ++w) wcount[w][tid] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
    for (int r = 0; r < kSortItems; ++r) {
        int64_t i = tile0 + r * kSortThreads + tid;
        bool valid = i < n;
        unsigned long long key = valid ? kin[i] : 0ull;
        uint32_t val = (valid && vin) ? vin[i] : 0u;
        uint32_t digit = valid ? ((uint32_t)(key >> shift) & 255u) : (256u + lane);
        uint32_t peers = __match_any_sync(0xffffffffu, digit);
        uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid && rank == 0) wcount[warp][digit] = __popc(peers);
        __syncthreads();
        uint32_t run = base[tid];
        for (int w = 0; w < W; ++w) {
            uint32_t c = wcount[w][tid];
            pref[w][tid] = run;
            wcount[w][tid] = 0;
            run += c;
        }
        base[tid] = run;
        __syncthreads();
        if (valid) {
            uint32_t pos = pref[warp][digit] + rank;
            kout[pos] = key;
            if (vout) vout[pos] = val;
        }
    }
}

// ---------------------------------------------------------------- hierarchy

// Common-prefix length of sorted keys i and j, extended by the index bits
// when the codes are equal; -1 outside [0, n).
__device__ __forceinline__ int delta(const unsigned long long *__restrict__ codes, int64_t n,
                                     int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    unsigned long long a = codes[i], b = codes[j];
    if (a == b) return 64 + __clz((uint32_t)(i ^ j));
    return __clzll(a ^ b);
}

__global__ void k_karras(int64_t n, const unsigned long long *__restrict__ codes,
                         Node *__restrict__ nodes, uint32_t *__restrict__ parent_int,
                         uint32_t *__restrict__ parent_leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (delta(codes, n, i, i + 1) - delta(codes, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = delta(codes, n, i, i - d);
    int64_t lmax = 2;
    while (delta(codes, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int64_t l = 0;
    for (int64_t t = lmax >> 1; t >= 1; t >>= 1)
        if (delta(codes, n, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = delta(codes, n, i, j);
    int64_t s = 0;
    for (int64_t div = 2;; div <<= 1) {
        int64_t t = (l + div - 1) / div;
        if (delta(codes, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    uint32_t left = (lo == gamma) ? (kLeafBit | (uint32_t)gamma) : (uint32_t)gamma;
    uint32_t right = (hi == gamma + 1) ? (kLeafBit | (uint32_t)(gamma + 1)) : (uint32_t)(gamma + 1);
    Node &nd = nodes[i];
    nd.child[0] = left;
    nd.child[1] = right;
    nd.leaf_range[0] = (uint32_t)lo;
    nd.leaf_range[1] = (uint32_t)hi;
    if (left & kLeafBit) parent_leaf[gamma] = (uint32_t)i; else parent_int[gamma] = (uint32_t)i;
    if (right & kLeafBit) parent_leaf[gamma + 1] = (uint32_t)i; else parent_int[gamma + 1] = (uint32_t)i;
}

__device__ __forceinline__ void write_record(PrimRec *__restrict__ prims, int64_t i, uint32_t g,
                                             const Activated &a) {
    PrimRec r;
    for (int k = 0; k < 3; ++k) r.mu[k] = a.mu[k];
    r.opacity = a.opacity;
    // M = S^-1 R_q^T: row k is column k of R_q divided by s_k
    for (int k = 0; k < 3; ++k)
        for (int j = 0; j < 3; ++j) r.m[3 * k + j] = a.R[3 * j + k] * a.inv_s[k];
    if (!a.finite)
        for (int k = 0; k < 9; ++k) r.m[k] = NAN;
    r.gid = g;
    r.pad[0] = 0.0f;
    r.pad[1] = 0.0f;
    float4 *dst = reinterpret_cast<float4 *>(prims + i);
    const float4 *src = reinterpret_cast<const float4 *>(&r);
    for (int k = 0; k < 4; ++k) dst[k] = src[k];
}

// One thread per leaf (tree position i): write the Gaussian record, then
// carry boxes towards the root; the second thread to reach a node merges
// both child boxes and continues.
__global__ void k_leaves(int64_t n, const uint32_t *__restrict__ order,
                         const float *__restrict__ means, const float *__restrict__ log_scales,
                         const float *__restrict__ quats, const float *__restrict__ logits,
                         const float *__restrict__ aabb, PrimRec *__restrict__ prims,
                         Node *__restrict__ nodes, const uint32_t *__restrict__ parent_int,
                         const uint32_t *__restrict__ parent_leaf, uint32_t *__restrict__ arrive) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t g = order[i];
    Activated a = activate(means, log_scales, quats, logits, g);
    write_record(prims, i, g, a);
    float box[6];
    for (int k = 0; k < 6; ++k) box[k] = aabb[6 * (int64_t)g + k];
    uint32_t ref = kLeafBit | (uint32_t)i;
    uint32_t p = parent_leaf[i];
    for (int guard = 0; guard < 4096; ++guard) {
        Node *nd = nodes + p;
        int side = (__ldcg(&nd->child[0]) == ref) ? 0 : 1;
        for (int k = 0; k < 6; ++k) __stcg(&nd->box[side][k], box[k]);
        __threadfence();
        if (atomicAdd(&arrive[p], 1u) == 0u) return;
        __threadfence();
        for (int k = 0; k < 3; ++k) {
            box[k] = fminf(box[k], __ldcg(&nd->box[1 - side][k]));
            box[3 + k] = fmaxf(box[3 + k], __ldcg(&nd->box[1 - side][3 + k]));
        }
        if (p == 0) return;
        ref = p;
        p = parent_int[p];
    }
}

// M == 1: a root whose two children are the same leaf. Draws are keyed by
// (ray, Gaussian, sample), so testing the leaf twice gives the same answer.
__global__ void k_single(const uint32_t *__restrict__ order, const float *__restrict__ means,
                         const float *__restrict__ log_scales, const float *__restrict__ quats,
                         const float *__restrict__ logits, const float *__restrict__ aabb,
                         PrimRec *__restrict__ prims, Node *__restrict__ nodes) {
    uint32_t g = order[0];
    Activated a = activate(means, log_scales, quats, logits, g);
    write_record(prims, 0, g, a);
    Node nd;
    for (int s = 0; s < 2; ++s) {
        for (int k = 0; k < 6; ++k) nd.box[s][k] = aabb[6 * (int64_t)g + k];
        nd.child[s] = kLeafBit;
    }
    nd.leaf_range[0] = nd.leaf_range[1] = 0;
    nodes[0] = nd;
}

// Depth of every internal binary node (walk to the root).
__global__ void k_depth(int64_t n_int, const uint32_t *__restrict__ parent_int,
                        uint32_t *__restrict__ depth, uint32_t *__restrict__ flag) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    uint32_t d = 0, p = (uint32_t)i;
    while (p != 0 && d < 4096) {
        p = parent_int[p];
        ++d;
    }
    depth[i] = d;
    flag[i] = (d & 1u) ? 0u : 1u;  // wide nodes sit at even binary depth
}

// Quantisation of one axis of a node: planes origin + q * 2^e, q in 0..255.
__device__ __forceinline__ int quant_exponent(float ext) {
    if (!(ext > 0.0f)) return -120;
    int e = (int)ceilf(log2f(ext / 254.0f));
    e = max(e, -120);
    while (254.0f * ldexpf(1.0f, e) < ext) ++e;  // one unit of slack
    return min(e, 120);
}

__device__ __forceinline__ unsigned char quant_lo(float v, float origin, float scale) {
    if (!(v == v)) return 0;  // NaN box: full range
    float q = floorf((v - origin) / scale);
    q = fminf(fmaxf(q, 0.0f), 255.0f);
    while (q > 0.0f && __fadd_rn(origin, q * scale) > v) q -= 1.0f;
    return (unsigned char)q;
}

__device__ __forceinline__ unsigned char quant_hi(float v, float origin, float scale) {
    if (!(v == v)) return 255;
    float q = ceilf((v - origin) / scale);
    q = fminf(fmaxf(q, 0.0f), 255.0f);
    while (q < 255.0f && __fadd_rn(origin, q * scale) < v) q += 1.0f;
    return (unsigned char)q;
}

// One wide node per even-depth binary node: its children, or grandchildren
// where a child is internal; written at its compact index.
template <int FMT>
__global__ void k_collapse(int64_t n_int, const Node *__restrict__ nodes,
                           const uint32_t *__restrict__ depth, const uint32_t *__restrict__ wmap,
                           void *__restrict__ wide) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || (depth[i] & 1u)) return;
    float lo[3][4], hi[3][4];
    uint32_t child[4];
    int k = 0;
    const Node nd = nodes[i];
    for (int side = 0; side < 2; ++side) {
        const uint32_t c = nd.child[side];
        if (c & kLeafBit) {
            for (int a = 0; a < 3; ++a) { lo[a][k] = nd.box[side][a]; hi[a][k] = nd.box[side][3 + a]; }
            child[k++] = c;
        } else {
            const Node cn = nodes[c];
            for (int s2 = 0; s2 < 2; ++s2) {
                for (int a = 0; a < 3; ++a) { lo[a][k] = cn.box[s2][a]; hi[a][k] = cn.box[s2][3 + a]; }
                const uint32_t gc = cn.child[s2];
                child[k++] = (gc & kLeafBit) ? gc : wmap[gc];
            }
        }
    }
    const int used = k;
    for (; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) { lo[a][k] = INFINITY; hi[a][k] = INFINITY; }
        child[k] = kEmpty;
    }
    const uint32_t w = wmap[i];
    if (FMT == GS_NODES_WIDE4) {
        Node4 n;
        for (int a = 0; a < 3; ++a)
            for (int j = 0; j < 4; ++j) { n.lo[a][j] = lo[a][j]; n.hi[a][j] = hi[a][j]; }
        for (int j = 0; j < 4; ++j) { n.child[j] = child[j]; n.reserved[j] = 0; }
        reinterpret_cast<Node4 *>(wide)[w] = n;
    } else {
        NodeQ4 n;
        n.used = (unsigned char)((1u << used) - 1u);
        for (int a = 0; a < 3; ++a) {
            float nlo = INFINITY, nhi = -INFINITY;
            for (int j = 0; j < used; ++j) { nlo = fminf(nlo, lo[a][j]); nhi = fmaxf(nhi, hi[a][j]); }
            if (!(nlo <= nhi)) { nlo = 0.0f; nhi = 0.0f; }
            const int e = quant_exponent(nhi - nlo);
            const float scale = ldexpf(1.0f, e);
            n.origin[a] = nlo;
            n.exp[a] = (signed char)e;
            for (int j = 0; j < 4; ++j) {
                if (j < used) {
                    n.qlo[a][j] = quant_lo(lo[a][j], nlo, scale);
                    n.qhi[a][j] = quant_hi(hi[a][j], nlo, scale);
                } else {
                    n.qlo[a][j] = 255;
                    n.qhi[a][j] = 0;
                }
            }
        }
        for (int j = 0; j < 4; ++j) n.child[j] = child[j];
        n.reserved[0] = n.reserved[1] = 0;
        reinterpret_cast<NodeQ4 *>(wide)[w] = n;
    }
}

// The W-wide hierarchies (W = 2^LEVELS). The wide nodes sit at binary
// internal nodes of depth 0 mod LEVELS; a wide node covering at most W
// leaves has those leaves as its children (and no wide node below it),
// any other has its descendants LEVELS levels down, or the leaves met
// before. So a binary node is a wide root when it is the root, or when its
// depth is 0 mod LEVELS and its ancestor LEVELS levels up covers more than
// W leaves. expand_wide lists the LEVELS-level children, left to right,
// with their boxes.
template <int LEVELS>
__device__ __forceinline__ int expand_wide(const Node *__restrict__ nodes, uint32_t i,
                                           uint32_t ref[1 << LEVELS], float box[1 << LEVELS][6]) {
    int n = 0;
    const Node nd = nodes[i];
    for (int sd = 0; sd < 2; ++sd) {
        ref[n] = nd.child[sd];
        for (int q = 0; q < 6; ++q) box[n][q] = nd.box[sd][q];
        ++n;
    }
    for (int level = 1; level < LEVELS; ++level) {
        // expand in place from the back so entries keep left-to-right order
        int m = n;
        for (int j = 0; j < n; ++j)
            if (!(ref[j] & kLeafBit)) ++m;
        for (int j = n - 1, dst = m - 1; j >= 0; --j) {
            if (ref[j] & kLeafBit) {
                ref[dst] = ref[j];
                for (int q = 0; q < 6; ++q) box[dst][q] = box[j][q];
                --dst;
            } else {
                const Node cn = nodes[ref[j]];
                for (int sd = 1; sd >= 0; --sd) {
                    ref[dst] = cn.child[sd];
                    for (int q = 0; q < 6; ++q) box[dst][q] = cn.box[sd][q];
                    --dst;
                }
            }
        }
        n = m;
    }
    return n;
}

// Depth of every binary internal node (walk to the root).
__global__ void k_node_depth(int64_t n_int, const uint32_t *__restrict__ parent_int,
                             uint32_t *__restrict__ depth) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    uint32_t d = 0, p = (uint32_t)i;
    while (p != 0 && d < 4096) {
        p = parent_int[p];
        ++d;
    }
    depth[i] = d;
}

__device__ __forceinline__ uint32_t leaves_under(const Node &nd) {
    return nd.leaf_range[1] - nd.leaf_range[0] + 1u;
}

// Children of the wide node at each binary internal node (0 where none);
// the same count, plus `header` units where a node exists, seeds the
// offsets.
template <int LEVELS>
__global__ void k_count_wide(int64_t n_int, const Node *__restrict__ nodes,
                             const uint32_t *__restrict__ depth,
                             const uint32_t *__restrict__ parent_int, uint32_t *__restrict__ cnt,
                             uint32_t *__restrict__ off, uint32_t header) {
    constexpr uint32_t W = 1u << LEVELS;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    uint32_t c = 0;
    bool root = i == 0;
    if (!root && depth[i] % (uint32_t)LEVELS == 0u) {
        uint32_t p = (uint32_t)i;
        for (int k = 0; k < LEVELS; ++k) p = parent_int[p];
        root = leaves_under(nodes[p]) > W;
    }
    if (root) {
        const uint32_t n_leaves = leaves_under(nodes[i]);
        if (n_leaves <= W) {
            c = n_leaves;
        } else {
            uint32_t ref[1 << LEVELS];
            float box[1 << LEVELS][6];
            c = (uint32_t)expand_wide<LEVELS>(nodes, (uint32_t)i, ref, box);
        }
    }
    cnt[i] = c;
    off[i] = c ? c + header : 0u;
}

// Writes the child records of every wide node at its offset.
template <int LEVELS>
__global__ void k_collapse_wide(int64_t n_int, const Node *__restrict__ nodes,
                                const uint32_t *__restrict__ cnt, const uint32_t *__restrict__ off,
                                const uint32_t *__restrict__ order, const float *__restrict__ aabb,
                                ChildRec *__restrict__ rec) {
    constexpr uint32_t W = 1u << LEVELS;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || cnt[i] == 0u) return;
    ChildRec *dst = rec + off[i];
    const Node ndi = nodes[i];
    if (leaves_under(ndi) <= W) {
        // every leaf of the node, with the box its parent node holds for it
        for (uint32_t k = ndi.leaf_range[0]; k <= ndi.leaf_range[1]; ++k) {
            ChildRec c;
            const float *b = aabb + 6 * (int64_t)order[k];
            for (int q = 0; q < 3; ++q) { c.lo[q] = b[q]; c.hi[q] = b[3 + q]; }
            c.child = kLeafBit | k;
            c.reserved = 0;
            *dst++ = c;
        }
        return;
    }
    uint32_t ref[1 << LEVELS];
    float box[1 << LEVELS][6];
    const int n = expand_wide<LEVELS>(nodes, (uint32_t)i, ref, box);
    for (int j = 0; j < n; ++j) {
        ChildRec c;
        for (int q = 0; q < 3; ++q) { c.lo[q] = box[j][q]; c.hi[q] = box[j][3 + q]; }
        const uint32_t r = ref[j];
        c.child = (r & kLeafBit) ? r : (((cnt[r] - 1u) << kWideCountShift) | off[r]);
        c.reserved = 0;
        dst[j] = c;
    }
}

// 8-bit planes of one child box against its node's frame (origin, scale):
// lower planes rounded down and upper planes rounded up, each by one more
// quantum, so that the traversal's decoding (whose rounding stays under
// half a quantum) still covers the FP32 box. A non-finite box is flagged.
__device__ __forceinline__ void quant_child(const float b[6], const float origin[3],
                                            const float scale[3], uint32_t &q0, uint32_t &q1) {
    uint32_t lo[3], hi[3];
    bool finite = true;
    for (int a = 0; a < 3; ++a) finite = finite && isfinite(b[a]) && isfinite(b[3 + a]);
    for (int a = 0; a < 3; ++a) {
        float ql = floorf((b[a] - origin[a]) / scale[a]) - 1.0f;
        float qh = ceilf((b[3 + a] - origin[a]) / scale[a]) + 1.0f;
        // exact checks in the frame (q * scale is exact for a power-of-two
        // scale): one quantum of room below lo and above hi
        while (ql > 0.0f && !(__fadd_rn(origin[a], (ql + 1.0f) * scale[a]) <= b[a])) ql -= 1.0f;
        while (qh < 255.0f && !(__fadd_rn(origin[a], (qh - 1.0f) * scale[a]) >= b[3 + a])) qh += 1.0f;
        lo[a] = finite ? (uint32_t)fminf(fmaxf(ql, 0.0f), 255.0f) : 0u;
        hi[a] = finite ? (uint32_t)fminf(fmaxf(qh, 0.0f), 255.0f) : 0u;
    }
    q0 = lo[0] | lo[1] << 8 | lo[2] << 16 | hi[0] << 24;
    q1 = hi[1] | hi[2] << 8 | (finite ? 0u : kQ8Skip);
}

// Frame of an 8-bit wide node from the union of its children's boxes:
// per axis a power-of-two scale with the extent plus two spare quanta
// within 255 quanta, and the origin one quantum below the lower bound.
__device__ __forceinline__ void quant_frame(const float lo[3], const float hi[3], float origin[3],
                                            float scale[3]) {
    for (int a = 0; a < 3; ++a) {
        float l = lo[a], h = hi[a];
        if (!(l <= h)) { l = 0.0f; h = 0.0f; }
        const float ext = h - l;
        int e = ext > 0.0f ? (int)ceilf(log2f(ext / 251.0f)) : -120;
        e = max(e, -120);
        while (251.0f * ldexpf(1.0f, e) < ext) ++e;
        e = min(e, 120);
        scale[a] = ldexpf(1.0f, e);
        origin[a] = l - scale[a];
    }
}

// Writes every wide node of the 8-bit form at its offset: the header from
// the children's union box, then one unit per child.
template <int LEVELS>
__global__ void k_collapse_wide_q8(int64_t n_int, const Node *__restrict__ nodes,
                                   const uint32_t *__restrict__ cnt,
                                   const uint32_t *__restrict__ off,
                                   const uint32_t *__restrict__ order,
                                   const float *__restrict__ aabb, uint4 *__restrict__ units) {
    constexpr uint32_t W = 1u << LEVELS;
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || cnt[i] == 0u) return;
    uint4 *dst = units + off[i];
    const Node ndi = nodes[i];
    float ulo[3] = {INFINITY, INFINITY, INFINITY}, uhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float origin[3], scale[3];
    if (leaves_under(ndi) <= W) {
        for (uint32_t k = ndi.leaf_range[0]; k <= ndi.leaf_range[1]; ++k) {
            const float *b = aabb + 6 * (int64_t)order[k];
            for (int q = 0; q < 3; ++q) { ulo[q] = fminf(ulo[q], b[q]); uhi[q] = fmaxf(uhi[q], b[3 + q]); }
        }
        quant_frame(ulo, uhi, origin, scale);
        uint32_t j = kGroupQHeaderUnits;
        for (uint32_t k = ndi.leaf_range[0]; k <= ndi.leaf_range[1]; ++k, ++j) {
            const float *b = aabb + 6 * (int64_t)order[k];
            const float bx[6] = {b[0], b[1], b[2], b[3], b[4], b[5]};
            uint32_t q0, q1;
            quant_child(bx, origin, scale, q0, q1);
            dst[j] = make_uint4(q0, q1, kLeafBit | k, 0u);
        }
    } else {
        uint32_t ref[1 << LEVELS];
        float box[1 << LEVELS][6];
        const int n = expand_wide<LEVELS>(nodes, (uint32_t)i, ref, box);
        for (int j = 0; j < n; ++j)
            for (int q = 0; q < 3; ++q) { ulo[q] = fminf(ulo[q], box[j][q]); uhi[q] = fmaxf(uhi[q], box[j][3 + q]); }
        quant_frame(ulo, uhi, origin, scale);
        for (int j = 0; j < n; ++j) {
            uint32_t q0, q1;
            quant_child(box[j], origin, scale, q0, q1);
            const uint32_t r = ref[j];
            const uint32_t c = (r & kLeafBit) ? r : (((cnt[r] - 1u) << kWideCountShift) | off[r]);
            dst[kGroupQHeaderUnits + j] = make_uint4(q0, q1, c, 0u);
        }
    }
    dst[0] = make_uint4(__float_as_uint(origin[0]), __float_as_uint(origin[1]),
                        __float_as_uint(origin[2]), __float_as_uint(scale[0]));
    dst[1] = make_uint4(__float_as_uint(scale[1]), __float_as_uint(scale[2]), 0u, 0u);
}

inline unsigned grid_for(int64_t n, int threads) {
    return (unsigned)((n + threads - 1) / threads);
}

}  // namespace

int64_t radix_tiles(int64_t n) { return (n + kSortTile - 1) / kSortTile; }

int sort_keys64(unsigned long long *keys[2], int64_t n, int lo_bit, uint32_t *hist,
                uint32_t *scan_tmp, cudaStream_t s) {
    const int64_t tiles = radix_tiles(n);
    int cur = 0;
    for (int shift = lo_bit; shift < 64; shift += 8) {
        k_radix_hist<<<(unsigned)tiles, kSortThreads, 0, s>>>(n, keys[cur], shift, hist, tiles);
        scan_exclusive(hist, 256 * tiles, scan_tmp, s);
        k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, s>>>(n, keys[cur], nullptr, keys[1 - cur],
                                                                 nullptr, shift, hist, tiles);
        cur = 1 - cur;
    }
    return cur;
}

int64_t scan_tmp_entries(int64_t n) { return (n + kScanItems - 1) / kScanItems + 1; }

gs_status build_into(gs_bvh *b, const gs_gaussians *g, cudaStream_t s) {
    const int64_t M = g->M;
    b->M = M;
    b->n_nodes = M == 0 ? 0 : (M == 1 ? 1 : M - 1);
    if (M == 0) return GS_OK;
    cudaError_t e;
    // bounds: mins start at the largest ordered value, maxes at the smallest
    if ((e = cudaMemsetAsync(b->bounds, 0xff, 3 * sizeof(unsigned int), s)) != cudaSuccess)
        return cuda_fail(e, "memset bounds");
    if ((e = cudaMemsetAsync(b->bounds + 3, 0, 3 * sizeof(unsigned int), s)) != cudaSuccess)
        return cuda_fail(e, "memset bounds");
    k_preprocess<<<grid_for(M, 256), 256, 0, s>>>(M, g->means, g->log_scales, g->quats,
                                                   g->opacity_logits, b->aabb, b->bounds, b->status);
    k_morton<<<grid_for(M, 256), 256, 0, s>>>(M, g->means, b->bounds, b->aabb, b->codes[0],
                                               b->vals[0]);
    const int64_t tiles = radix_tiles(M);
    int cur = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        k_radix_hist<<<(unsigned)tiles, kSortThreads, 0, s>>>(M, b->codes[cur], shift, b->hist, tiles);
        scan_exclusive(b->hist, 256 * tiles, b->scan_tmp, s);
        k_radix_scatter<<<(unsigned)tiles, kSortThreads, 0, s>>>(
            M, b->codes[cur], b->vals[cur], b->codes[1 - cur], b->vals[1 - cur], shift, b->hist,
            tiles);
        cur = 1 - cur;
    }
    b->final_buf = cur;
    const uint32_t *order = b->vals[cur];
    if (M == 1) {
        k_single<<<1, 1, 0, s>>>(order, g->means, g->log_scales, g->quats, g->opacity_logits,
                                 b->aabb, b->prims, b->nodes);
    } else {
        uint32_t *parent_int = b->parent, *parent_leaf = b->parent + M;
        k_karras<<<grid_for(M - 1, 256), 256, 0, s>>>(M, b->codes[cur], b->nodes, parent_int,
                                                       parent_leaf);
        if ((e = cudaMemsetAsync(b->arrive, 0, (size_t)M * sizeof(uint32_t), s)) != cudaSuccess)
            return cuda_fail(e, "memset arrive");
        k_leaves<<<grid_for(M, 256), 256, 0, s>>>(M, order, g->means, g->log_scales, g->quats,
                                                   g->opacity_logits, b->aabb, b->prims, b->nodes,
                                                   parent_int, parent_leaf, b->arrive);
    }
    if (b->node_format == GS_NODES_WIDE4 || b->node_format == GS_NODES_WIDE4_Q8) {
        const int64_t n_int = b->n_nodes;
        if (M == 1) {
            if ((e = cudaMemsetAsync(b->depth, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset depth");
            if ((e = cudaMemsetAsync(b->wmap, 0, 4, s)) != cudaSuccess) return cuda_fail(e, "memset map");
        } else {
            k_depth<<<grid_for(n_int, 256), 256, 0, s>>>(n_int, b->parent, b->depth, b->wmap);
            scan_exclusive(b->wmap, n_int, b->scan_tmp, s);
        }
        if (b->node_format == GS_NODES_WIDE4)
            k_collapse<GS_NODES_WIDE4><<<grid_for(n_int, 256), 256, 0, s>>>(n_int, b->nodes, b->depth,
                                                                            b->wmap, b->wide);
        else
            k_collapse<GS_NODES_WIDE4_Q8><<<grid_for(n_int, 256), 256, 0, s>>>(
                n_int, b->nodes, b->depth, b->wmap, b->wide);
    }
    if (b->node_depth) {
        const int64_t n_int = b->n_nodes;
        const bool q8 = b->node_format == GS_NODES_BINARY_Q8;
        const uint32_t hdr = q8 ? (uint32_t)kGroupQHeaderUnits : 0u;
        k_node_depth<<<grid_for(n_int, 256), 256, 0, s>>>(n_int, b->parent, b->node_depth);
        const GroupTree *t = b->group;
        k_count_wide<3><<<grid_for(n_int, 256), 256, 0, s>>>(n_int, b->nodes, b->node_depth, b->parent,
                                                            t[0].cnt, t[0].off, hdr);
        scan_exclusive(t[0].off, n_int, b->scan_tmp, s);
        if (q8)
            k_collapse_wide_q8<3><<<grid_for(n_int, 256), 256, 0, s>>>(
                n_int, b->nodes, t[0].cnt, t[0].off, order, b->aabb, static_cast<uint4 *>(t[0].rec));
        else
            k_collapse_wide<3><<<grid_for(n_int, 256), 256, 0, s>>>(
                n_int, b->nodes, t[0].cnt, t[0].off, order, b->aabb, static_cast<ChildRec *>(t[0].rec));
        k_count_wide<4><<<grid_for(n_int, 128), 128, 0, s>>>(n_int, b->nodes, b->node_depth, b->parent,
                                                            t[1].cnt, t[1].off, hdr);
        scan_exclusive(t[1].off, n_int, b->scan_tmp, s);
        if (q8)
            k_collapse_wide_q8<4><<<grid_for(n_int, 128), 128, 0, s>>>(
                n_int, b->nodes, t[1].cnt, t[1].off, order, b->aabb, static_cast<uint4 *>(t[1].rec));
        else
            k_collapse_wide<4><<<grid_for(n_int, 128), 128, 0, s>>>(
                n_int, b->nodes, t[1].cnt, t[1].off, order, b->aabb, static_cast<ChildRec *>(t[1].rec));
        k_count_wide<5><<<grid_for(n_int, 128), 128, 0, s>>>(n_int, b->nodes, b->node_depth, b->parent,
                                                            t[2].cnt, t[2].off, hdr);
        scan_exclusive(t[2].off, n_int, b->scan_tmp, s);
        if (q8)
            k_collapse_wide_q8<5><<<grid_for(n_int, 128), 128, 0, s>>>(
                n_int, b->nodes, t[2].cnt, t[2].off, order, b->aabb, static_cast<uint4 *>(t[2].rec));
        else
            k_collapse_wide<5><<<grid_for(n_int, 128), 128, 0, s>>>(
                n_int, b->nodes, t[2].cnt, t[2].off, order, b->aabb, static_cast<ChildRec *>(t[2].rec));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "build launch");
    return GS_OK;
}

}  // namespace gsrt
