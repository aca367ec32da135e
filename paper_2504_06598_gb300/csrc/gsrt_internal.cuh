// gsrt_internal.cuh -- device records, helpers and launch declarations shared
// by the build, trace and API translation units of the GB300 library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gsrt.h"

namespace gsrt {

// --------------------------------------------------------------------------
// Records in device memory
// --------------------------------------------------------------------------

// One Gaussian, in hierarchy (Morton) order, 64 bytes = four 16-byte loads.
// m[] is the local transform M = S^-1 R_q^T (row-major): for a world vector
// v, |M v|^2 is the Mahalanobis form of Eq. 1, so the bounding ellipsoid of
// Eq. 2 is |M (x - mu)| <= s.
struct __align__(16) PrimRec {
    float mu[3];
    float opacity;
    float m[9];
    uint32_t gid;
    float pad[2];
};
static_assert(sizeof(PrimRec) == 64, "PrimRec must be 64 bytes");

// Binary node, 64 bytes: boxes of both children and their references.
struct __align__(16) Node {
    float box[2][6];  // {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z} left, right
    uint32_t child[2];
    uint32_t leaf_range[2];  // first and last sorted leaf the node covers
};
static_assert(sizeof(Node) == 64, "Node must be 64 bytes");

// 4-wide node, 128 bytes: child boxes as structure of arrays (FP32).
struct __align__(16) Node4 {
    float lo[3][4];  // lo[axis][slot]
    float hi[3][4];
    uint32_t child[4];
    uint32_t reserved[4];
};
static_assert(sizeof(Node4) == 128, "Node4 must be 128 bytes");

// Child record of the W-wide hierarchies (W = 8, 16, 32) that groups of W
// lanes traverse, 32 bytes, one lane's load. A wide node is the run of its
// children's records (2 to W) at its offset; an internal child is
// referenced as (count - 1) << 26 | offset, a leaf as kLeafBit | primitive
// index.
struct __align__(16) ChildRec {
    float lo[3];
    float hi[3];
    uint32_t child;
    uint32_t reserved;
};
static_assert(sizeof(ChildRec) == 32, "ChildRec must be 32 bytes");
// 8-bit form of the W-wide records (handles built with
// GS_NODES_BINARY_Q8), in 16-byte units: a wide node is a two-unit header
// (GroupQHeader) followed by one unit per child (ChildQ8). Plane q of axis
// a of a child decodes to origin[a] + q * scale[a] (scale a power of two);
// the build rounds lower planes down and upper planes up with one spare
// quantum on each side, so the decoded box contains the child's FP32 box
// with room for the traversal's rounding. An internal child is referenced
// as (count - 1) << 26 | unit of its node's header.
struct __align__(16) GroupQHeader {
    float origin[3];
    float scale[3];
    uint32_t reserved[2];
};
static_assert(sizeof(GroupQHeader) == 32, "GroupQHeader must be 32 bytes");
struct __align__(16) ChildQ8 {
    uint32_t q0;     // qlo.x | qlo.y << 8 | qlo.z << 16 | qhi.x << 24
    uint32_t q1;     // qhi.y | qhi.z << 8 | flags << 16 (bit 0: never entered)
    uint32_t child;
    uint32_t reserved;
};
static_assert(sizeof(ChildQ8) == 16, "ChildQ8 must be 16 bytes");
constexpr int kGroupQHeaderUnits = 2;
constexpr uint32_t kQ8Skip = 1u << 16;  // q1 flag: a child with a non-finite box
constexpr int kWideCountShift = 26;
constexpr uint32_t kWideOffsetMask = (1u << kWideCountShift) - 1u;
constexpr int kGroupTrees = 3;  // W = 8 << i: collapses of 3, 4 and 5 binary levels

// One W-wide hierarchy: records (ChildRec, or 16-byte units of the 8-bit
// form), and per binary internal node the child count of the wide node
// there (0 where none) and its first record or unit.
struct GroupTree {
    void *rec;
    uint32_t *cnt;
    uint32_t *off;
};

// 4-wide node, 64 bytes, child boxes quantised to 8 bits per plane against
// the node's own box: plane = origin[a] + q * 2^exp[a], with the lower
// planes rounded down and the upper planes rounded up so every decoded box
// contains the child's FP32 box.
struct __align__(16) NodeQ4 {
    float origin[3];
    signed char exp[3];
    unsigned char used;   // bit k: slot k holds a child
    unsigned char qlo[3][4];
    unsigned char qhi[3][4];
    uint32_t child[4];
    uint32_t reserved[2];
};
static_assert(sizeof(NodeQ4) == 64, "NodeQ4 must be 64 bytes");

constexpr uint32_t kLeafBit = 0x80000000u;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kMaxStack = 96;
constexpr uint32_t kStepLimit = 1u << 22;  // node visits per ray and pass

// Device status word bits.
constexpr uint32_t kErrStack = 1u << 0;
constexpr uint32_t kErrSteps = 1u << 1;
constexpr uint32_t kErrNonfinite = 1u << 2;
constexpr uint32_t kErrKeys = 1u << 3;  // a stored sample key named no Gaussian of the handle

// s^2 of Eq. 2 with s = 2 sqrt(2).
constexpr float kS2 = 8.0f;

}  // namespace gsrt

// --------------------------------------------------------------------------
// Handle (host side)
// --------------------------------------------------------------------------
struct gs_bvh {
    int device;
    int64_t M;
    int64_t capacity;
    int64_t n_nodes;
    int64_t device_bytes;
    // persistent outputs
    gsrt::Node *nodes;
    gsrt::PrimRec *prims;
    uint32_t *status;  // device status word
    // build scratch (kept for rebuilds)
    unsigned long long *codes[2];
    uint32_t *vals[2];
    uint32_t *parent;   // [2M]: parents of internal nodes (0..M-2) then leaves
    uint32_t *arrive;   // [M] refit arrival counters
    float *aabb;        // [M][6] in Gaussian-id order
    unsigned int *bounds;  // [6] ordered-int scene bounds of the means
    uint32_t *hist;     // radix histograms [256 * tiles]
    int64_t hist_len;
    uint32_t *scan_tmp; // block sums of the multi-block scan
    int final_buf;      // which of codes/vals holds the sorted result
    // traversal nodes other than the binary ones
    int node_format;    // GS_NODES_*
    void *wide;         // Node4 or NodeQ4 array, compact
    uint32_t *depth;    // depth of every internal binary node
    uint32_t *wmap;     // binary internal node -> wide node index
    // W-wide hierarchies for groups of lanes sharing one ray (binary format
    // only): W = 8, 16, 32, each at most M + (M - 1) records
    gsrt::GroupTree group[gsrt::kGroupTrees];
    uint32_t *node_depth;  // depth of every binary internal node
    // scratch of the batched form's deferred bounce rays, grown on demand
    int64_t wave_cap;                    // sample slots (pixels x spp) held
    int64_t wave_bytes;                  // device bytes of the scratch below
    unsigned long long *wave_codes[2];   // one sort code per slot
    float *wave_bounce;                  // [slots][3] albedo x bounce radiance
    uint32_t *wave_hist;                 // radix histograms of the codes
    uint32_t *wave_scan;                 // scan block sums
};

namespace gsrt {

// Host-side helpers (api.cu)
gs_status fail(gs_status s, const char *fmt, ...);
gs_status cuda_fail(cudaError_t e, const char *what);
bool is_device_ptr(const void *p);

// Build pipeline (build.cu)
gs_status build_into(gs_bvh *b, const gs_gaussians *g, cudaStream_t s);
int64_t radix_tiles(int64_t n);
int64_t scan_tmp_entries(int64_t n);
// Stable LSD radix sort of n 64-bit keys on bits [lo_bit, 64), 8 bits per
// pass, ping-ponging between keys[0] and keys[1]; returns the index of the
// buffer holding the result. hist: 256 * radix_tiles(n) entries, scan_tmp:
// scan_tmp_entries(256 * radix_tiles(n)).
int sort_keys64(unsigned long long *keys[2], int64_t n, int lo_bit, uint32_t *hist,
                uint32_t *scan_tmp, cudaStream_t s);

// Batched form (wavefront.cu): grows the handle's deferred-bounce scratch to
// `slots` sample slots (synchronous allocation; refused while the stream is
// capturing a graph).
gs_status reserve_wave_scratch(gs_bvh *b, int64_t slots, cudaStream_t s);
// Sample slots the batched form needs for these views and options (0 when
// the bounce is traced inline).
int64_t wave_slots(const gs_pinhole *cams, int n_views, const gs_scene_extras *ex,
                   const gs_trace_params *p);

// Backward (backward.cu)
// keys: the rendering's per-sample payloads, or null to trace them again.
gs_status launch_backward(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                          const gs_trace_params *p, const gs_sample_key *keys, const float *d_rgb,
                          float *d_means, float *d_log_scales, float *d_quats, float *d_logits,
                          float *d_sh, cudaStream_t s);

// Wavefront (wavefront.cu)
gs_status launch_render_views(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cams,
                              int n_views, const gs_scene_extras *ex, const gs_trace_params *p,
                              const gs_launch_options *opt, float *rgb, unsigned long long *counters,
                              int32_t *samples, cudaStream_t s);

// Trace (trace.cu)
// How a trace with these options maps samples to lanes: S samples per lane,
// spp_eff passes, 2^lpp_log2 lanes per pixel, grouped (cooperative) traversal.
void trace_layout(const gs_bvh *b, const gs_trace_params *p, int *S, int *spp_eff,
                  int *lpp_log2, bool *grouped);
gs_status launch_trace(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                       const gs_trace_params *p, float *rgb, int32_t *hit_id, float *hit_t,
                       gs_sample_key *keys, cudaStream_t s);

}  // namespace gsrt
