/*
 * gsrt.h -- C ABI of the GB300 library for stochastic ray tracing of
 * transparent 3D Gaussians (arXiv 2504.06598).
 *
 * One ray walks a bounding volume hierarchy over the Gaussians' bounding
 * boxes once (Sec. 3.2), evaluates each overlapped Gaussian's 1D Gaussian
 * along the ray (Sec. 3.1), accepts it at random with probability alpha
 * (Eq. 4, Alg. 1), keeps the closest accepted intersection (Eq. 6) or N of
 * them (Eq. 7, Sec. 3.5), and shades it with view-dependent spherical
 * harmonics. The result is an unbiased estimate of the depth-sorted blend
 * (Eq. 3).
 *
 * Conventions shared by every call
 *   - Pointers named in a struct or argument list as "device" must point to
 *     CUDA device memory of the current device; "host" pointers to host
 *     memory. Arrays are dense, row-major, 16-byte aligned (as returned by
 *     cudaMalloc or a PyTorch allocation).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream). Every call only enqueues work on it and returns without
 *     waiting, except where stated.
 *   - Argument errors are returned before anything is enqueued and leave
 *     all outputs untouched. gs_last_error() then describes the problem.
 *   - Errors found by a kernel (stack overflow, traversal step limit,
 *     non-finite parameters) are recorded in a status word owned by the BVH
 *     handle and are returned by gs_bvh_sync_status().
 *   - No call throws, traps, or waits on the device without a bound.
 *
 * Random draws: xi for (ray r, Gaussian g, sample s) is lane (s & 3) of
 * Philox-4x32-10 with key (seed low word, seed high word) and counter
 * (r, g, s >> 2, stream_tag), mapped to [0,1) as (u >> 8) * 2^-24. A hit
 * is accepted iff xi < alpha. Results therefore depend only on (seed, ray
 * id, Gaussian id, sample index), not on the hierarchy or launch shape.
 */
#ifndef GSRT_H
#define GSRT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1,    /* a pointer, size or option was rejected */
    GS_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    GS_ERR_OOM = 3,            /* device allocation failed */
    GS_ERR_STACK_OVERFLOW = 4, /* a ray needed more than stack_depth entries */
    GS_ERR_STEP_LIMIT = 5,     /* a ray exceeded the traversal step bound */
    GS_ERR_NONFINITE = 6,      /* a Gaussian parameter was NaN or infinite */
    GS_ERR_NO_DEVICE = 7       /* no CUDA device is available */
} gs_status;

/* Storage type of the spherical-harmonic coefficients. */
enum { GS_SH_F32 = 0, GS_SH_F16 = 1, GS_SH_BF16 = 2 };

/* Gaussian parameters (Eq. 1). All device pointers, caller-owned.
 *   means          [M][3] float  mu
 *   log_scales     [M][3] float  S = diag(exp(log_scales))
 *   quats          [M][4] float  (w,x,y,z), normalised by the library; the
 *                                 rotation R_q maps local to world and the
 *                                 paper's R equals R_q^T, so
 *                                 Sigma = R_q S^2 R_q^T
 *   opacity_logits [M]    float  opacity = sigmoid(logit)
 *   sh             [M][K][3]     K = (sh_degree+1)^2 coefficients per
 *                                 channel, type sh_dtype; colour
 *                                 c = max(0, k_0 + sum_{l>=1,m} Y_lm(d) k_lm)
 *                                 with real SH (Condon-Shortley phase),
 *                                 m = -l..l, d the unit ray direction; the
 *                                 DC term k_0 is stored pre-multiplied.
 *   M >= 0, M < 2^31; sh_degree in 0..3. */
typedef struct gs_gaussians {
    const float *means;
    const float *log_scales;
    const float *quats;
    const float *opacity_logits;
    const void *sh;
    int64_t M;
    int32_t sh_degree;
    int32_t sh_dtype;
} gs_gaussians;

/* Pinhole camera. The ray through pixel (x, y), row 0 at the top, is
 * defined in float32 by this exact sequence (each operation rounded once,
 * no fused multiply-add):
 *   th = (float) tan((double) fov_y_deg * pi / 360)
 *   f = normalise(look_at - eye), r = normalise(f x up), u = r x f
 *   s = th / height, ux = (2x + 1 - width) * s, uy = (height - 1 - 2y) * s
 *   d = normalise((f + ux * r) + uy * u), origin = eye,
 * normalise(v) = v / sqrt((v.x*v.x + v.y*v.y) + v.z*v.z).
 * Ray ids are ray_id_offset + y * width + x and must fit in 32 bits. */
typedef struct gs_pinhole {
    float eye[3];
    float look_at[3];
    float up[3];
    float fov_y_deg;
    int32_t width;
    int32_t height;
    uint32_t ray_id_offset;
    int32_t reserved;
} gs_pinhole;

/* Options of one trace (Alg. 1, Eq. 7).
 *   spp           passes: full traversals per pixel, >= 1
 *   n_hits        N, samples kept per traversal: 1, 2, 4 or 8
 *                 sample index s = pass * n_hits + k
 *   t_min, t_max  valid ray range, candidates need t_min < t < t_max
 *   bg            background colour of samples with no accepted hit
 *   depth_mode    0: depth is the mean of the 1D Gaussian (Sec. 3.1)
 *                 1: depth is the centre projected on the camera's forward
 *                    axis (Sec. 4.1); alpha stays the 1D peak
 *                    (gs_trace_stochastic only; this depth is not a ray
 *                    parameter, so accepted hits do not clip the traversal)
 *   stack_depth   traversal stack entries per ray, 1..96 (0 = 96), for
 *                 the per-lane stacks; the grouped traversal (see
 *                 gs_trace_stochastic) keeps 128 entries per group instead
 *   stream_tag    fourth Philox counter word, separates ray streams
 *   rng_mode      0: keyed Philox (above); 1: the trigonometric hash of
 *                 the hit point of Eq. 8-9, moved per sample by
 *                 1e-3 * frac(s * (0.8191725134, 0.6710436067,
 *                 0.5497004779)) - 5e-4 (gs_trace_stochastic only; float32,
 *                 not reproducible bit for bit)
 *   samples_per_lane
 *                 how many consecutive samples one lane of a traversal
 *                 carries (gs_trace_stochastic and gs_trace_backward,
 *                 each with its own choice for 0): 1, 2, 4 or 8 with
 *                 n_hits * samples_per_lane <= 8, or 0 to let the library
 *                 choose. The pixel then takes ceil(spp / S) passes, each
 *                 with n_hits * S slots (samples pass*n_hits*S + k),
 *                 so the S samples share one walk and one Philox call
 *                 serves four of their draws. Per-sample hits do not depend
 *                 on S; rgb_out may differ in the last bits (summation
 *                 order). The counters then count each lane's walk (the
 *                 union of its S samples' traversals); pass 1 for counts of
 *                 one sample's own traversal.
 *   counters      optional device uint64[7], incremented by the launch:
 *                 {nodes entered by each ray's own traversal, Gaussians
 *                 tested (Alg. 1 runs), Philox calls, rays (pixels),
 *                 samples shaded with a Gaussian's colour, node records
 *                 fetched by warps, Gaussian records fetched by warps};
 *                 in the grouped traversal the first and the sixth count
 *                 32-byte child records (of the wide nodes each ray
 *                 enters, and that each group fetches); NULL disables
 *                 counting (the default fast path). */
typedef struct gs_trace_params {
    uint64_t seed;
    int32_t spp;
    int32_t n_hits;
    float t_min;
    float t_max;
    float bg[3];
    int32_t depth_mode;
    int32_t stack_depth;
    uint32_t stream_tag;
    int32_t rng_mode;
    int32_t samples_per_lane;
    unsigned long long *counters;
} gs_trace_params;

/* Opaque hierarchy handle: library-owned device buffers holding the
 * per-Gaussian records (in hierarchy order), the nodes, build scratch and
 * the device status word. */
typedef struct gs_bvh gs_bvh;

/* Node format the traversal reads (the binary tree is always built too).
 *   GS_NODES_BINARY    64-byte binary nodes, FP32 child boxes; the handle
 *                      also holds 8-, 16- and 32-wide copies (one 32-byte
 *                      FP32 record per child, M + (M - 1) records at most
 *                      each, from 3, 4 and 5 binary levels) for the grouped
 *                      traversal, unless M > 2^25
 *   GS_NODES_WIDE4     128-byte 4-wide nodes, FP32 child boxes
 *   GS_NODES_WIDE4_Q8  64-byte 4-wide nodes, child boxes quantised to 8 bits
 *                      per plane with outward rounding (a decoded box always
 *                      contains the FP32 box, so no hit is lost and every
 *                      result equals the FP32 traversal's)
 *   GS_NODES_BINARY_Q8 binary nodes as GS_NODES_BINARY, with the 8-, 16- and
 *                      32-wide copies in 8-bit form: per wide node a 32-byte
 *                      header (origin, power-of-two scale per axis), then 16
 *                      bytes per child (six 8-bit planes rounded outward
 *                      with one spare quantum, the reference); unless
 *                      M > 2^24. Every result equals GS_NODES_BINARY's. */
enum { GS_NODES_BINARY = 0, GS_NODES_WIDE4 = 1, GS_NODES_WIDE4_Q8 = 2, GS_NODES_BINARY_Q8 = 3 };

typedef struct gs_build_options {
    int32_t node_format; /* GS_NODES_* */
    int32_t reserved[7]; /* zero */
} gs_build_options;

typedef struct gs_bvh_info {
    int64_t M;            /* Gaussians indexed */
    int64_t n_nodes;      /* internal binary nodes (max(M-1, 1), 0 when M = 0) */
    int64_t capacity;     /* largest M a rebuild can take without allocating */
    int64_t device_bytes; /* device memory held by the handle (including the
                             batched form's scratch, once allocated) */
    int32_t node_bytes;   /* bytes per binary node record */
    int32_t prim_bytes;   /* bytes per Gaussian record */
    int32_t node_format;  /* GS_NODES_* the traversal uses */
    int32_t wide_node_bytes; /* bytes per wide node (0 for binary) */
} gs_bvh_info;

/* Build the hierarchy over the Gaussians' bounding boxes (Sec. 3.2; the box
 * bounds the ellipsoid of Eq. 2 with s = 2 sqrt(2), tightly, then padded
 * outward so that no valid intersection is lost).
 *   g      Gaussian parameters (device arrays, read during the call's
 *          kernels only; SH is not read)
 *   out    receives a new handle (host pointer to a handle pointer)
 *   stream build kernels are enqueued here
 * Allocates the handle's device memory (synchronously). Parameters must be
 * unchanged until the build's kernels have run. Returns GS_ERR_INVALID_ARG
 * for bad sizes or pointers, GS_ERR_OOM / GS_ERR_CUDA / GS_ERR_NO_DEVICE on
 * CUDA failures. Non-finite parameters are reported by gs_bvh_sync_status. */
gs_status gs_build_bvh(const gs_gaussians *g, gs_bvh **out, void *stream);

/* gs_build_bvh with options (NULL = defaults: binary nodes). Same rules and
 * errors as gs_build_bvh; an unknown node_format returns
 * GS_ERR_INVALID_ARG. Rebuilds keep the handle's node format. */
gs_status gs_build_bvh_ex(const gs_gaussians *g, const gs_build_options *opt, gs_bvh **out,
                          void *stream);

/* Rebuild an existing handle for new parameters with M <= capacity, with no
 * allocation (the usual per-frame call when Gaussians move). Same rules as
 * gs_build_bvh; M > capacity returns GS_ERR_INVALID_ARG. */
gs_status gs_bvh_rebuild(gs_bvh *bvh, const gs_gaussians *g, void *stream);

/* Release the handle and its device memory (synchronises the device first).
 * NULL is accepted. */
gs_status gs_bvh_free(gs_bvh *bvh);

/* Fill *info (host struct) about the handle. */
gs_status gs_bvh_get_info(const gs_bvh *bvh, gs_bvh_info *info);

/* Wait for `stream`, then return and clear the device status word: GS_OK or
 * the first error a build or trace kernel recorded since the last call. */
gs_status gs_bvh_sync_status(gs_bvh *bvh, void *stream);

/* Copy the hierarchy to host memory for inspection (synchronous).
 *   nodes_out  host, n_nodes * node_bytes bytes, or NULL
 *   prims_out  host, M * prim_bytes bytes, or NULL
 *   codes_out  host uint64[M]: sorted Morton codes, or NULL
 *   order_out  host uint32[M]: Gaussian id of each leaf position, or NULL
 * Node record (64 bytes): float box[2][6] as {lo.x,lo.y,lo.z,hi.x,hi.y,
 * hi.z} of the left then right child, uint32 child[2], uint32 leaf_range[2]
 * (the first and last leaf position the node covers);
 * a child reference with bit 31 set is leaf (ref & 0x7fffffff), else an
 * internal node index; node 0 is the root. */
gs_status gs_bvh_export(const gs_bvh *bvh, void *nodes_out, void *prims_out,
                        uint64_t *codes_out, uint32_t *order_out);

/* Copy the wide nodes of a GS_NODES_WIDE4 or GS_NODES_WIDE4_Q8 handle to
 * host memory (synchronous). *n_out receives the number of wide nodes; at
 * most `capacity` of them are written to out (wide_node_bytes each), so a
 * call with capacity 0 queries the count. Node 0 is the root; a child
 * reference is a Gaussian record (bit 31 set), a wide node index, or
 * 0xffffffff for an unused slot. */
gs_status gs_bvh_export_wide(const gs_bvh *bvh, void *out, int64_t capacity, int64_t *n_out);

/* Render one pinhole view by stochastic ray tracing (Alg. 1, Eq. 4-7).
 *   bvh        built from the same Gaussians `g` (unchanged since)
 *   g          Gaussian parameters; only sh/sh_degree/sh_dtype are read here
 *   cam        host struct, width and height >= 1
 *   p          host struct of options
 *   rgb_out    device float[height][width][3]: mean over spp * n_hits
 *              samples of the closest accepted hit's colour (bg if none)
 *   hit_id_out device int32[spp][n_hits][height][width] Gaussian id of each
 *              sample's hit or -1; NULL to skip
 *   hit_t_out  device float[spp][n_hits][height][width] depth of each
 *              sample's hit (ray parameter, d is unit length) or +inf;
 *              NULL to skip
 * The 32 lanes of a warp split into pixels x samples: the L lanes of a pixel
 * (L the largest power of two not above ceil(spp / S), at most 32, S =
 * samples_per_lane) trace passes j*L + lane of the same ray. With L >= 8 and a GS_NODES_BINARY handle a
 * group of L lanes traverses the L-wide copy together (each lane tests one
 * child box, evaluates one hit Gaussian's depth and alpha, and draws for its
 * own samples); otherwise each lane traverses the nodes of the handle's
 * format in a warp packet. Every form returns the same hits.
 * Deterministic: identical inputs give bit-identical outputs. Traces that use
 * the same handle share its tile counter and status word, so they must not
 * overlap on the GPU: issue them on one stream (or order their streams). */
gs_status gs_trace_stochastic(const gs_bvh *bvh, const gs_gaussians *g, const gs_pinhole *cam,
                              const gs_trace_params *p, float *rgb_out, int32_t *hit_id_out,
                              float *hit_t_out, void *stream);

/* The payload of one sample after its traversal (Eq. 6): the depth key of
 * its closest accepted hit, split as the base-point parameter tc and the 1D
 * mean relative to the base point tau (the hit depth is tc + tau, rounded
 * once), and that Gaussian's id; {+inf, 0, 0xffffffff} when the sample
 * accepted nothing. 12 bytes, 4-byte aligned. */
typedef struct gs_sample_key {
    float tc;
    float tau;
    uint32_t gid;
} gs_sample_key;

/* gs_trace_stochastic that also stores every sample's payload, so that
 * gs_trace_backward_keys can take the gradient without tracing again.
 *   rgb_out   as in gs_trace_stochastic
 *   keys_out  device gs_sample_key[height][width][spp * n_hits]: entry s of
 *             a pixel is its sample s, the same sample index as the first
 *             two dimensions of gs_trace_stochastic's hit_id_out (sample
 *             pass i, slot h: s = i * n_hits + h); key.gid and
 *             key.tc + key.tau are that sample's hit_id_out and hit_t_out
 * Same rules, options and errors as gs_trace_stochastic; keys_out NULL,
 * not a device pointer or not 4-byte aligned returns GS_ERR_INVALID_ARG.
 * The image equals gs_trace_stochastic's for the same arguments. */
gs_status gs_trace_stochastic_keys(const gs_bvh *bvh, const gs_gaussians *g,
                                   const gs_pinhole *cam, const gs_trace_params *p, float *rgb_out,
                                   gs_sample_key *keys_out, void *stream);

/* How gs_trace_stochastic(bvh, ..., p, ...) maps samples to lanes (host
 * call, nothing is enqueued). layout_out (host int32[4]) receives
 * {samples per lane S, lanes per pixel L, passes ceil(spp / S) of
 * n_hits * S slots each, 1 if a group of L lanes walks the L-wide copy
 * together else 0}: one walk
 * of the hierarchy serves L * S samples of one ray when grouped, S samples
 * otherwise. Returns GS_ERR_INVALID_ARG for NULL pointers or options
 * gs_trace_stochastic would reject. */
gs_status gs_trace_layout(const gs_bvh *bvh, const gs_trace_params *p, int32_t *layout_out);

/* Measurement support (the paper has no counterpart): copy `bytes` from
 * src to dst `repeats` times in one kernel with 16-byte loads and stores
 * that bypass L1, enqueued on `stream`. src and dst are device pointers,
 * 16-byte aligned, bytes a positive multiple of 16, repeats in 1..2^20.
 * With src + dst well inside L2 the copy measures L2 bandwidth (the
 * denominator of the trace kernel's L2 roofline), beyond L2 it measures
 * DRAM bandwidth. The caller times it (for example with CUDA events). */
gs_status gs_probe_copy(const void *src, void *dst, int64_t bytes, int32_t repeats, void *stream);

/* Unbiased stochastic gradient of an image loss (the differentiable
 * rendering extension named at the end of the paper, Sec. 6). For each
 * sample with closest accepted hit k (colour c_k, or bg):
 *   dLoss/dc_k += g,  dLoss/dalpha_i += g . (c_i - c_k) / (1 - alpha_i)
 * for every valid Gaussian i in front of k, with g = d_rgb / (spp*n_hits);
 * alpha's dependence on the mean, log-scales, quaternion and opacity logit,
 * and the colour's on the SH coefficients, are then chained through. The
 * expectation is the gradient of the sorted blend of Eq. 3 (depth-order
 * swaps and the ellipsoid cutoff are not differentiated). Hits are
 * recomputed with the same keys as gs_trace_stochastic(bvh, g, cam, p), so
 * the samples are the ones that trace rendered; nothing is stored between
 * the two calls (gs_trace_backward_keys takes the stored payloads instead).
 *   d_rgb            device float[height][width][3], dLoss/d(rgb_out)
 *   d_means          device float[M][3]     } gradients, ACCUMULATED (+=),
 *   d_log_scales     device float[M][3]     } float32 whatever sh_dtype is;
 *   d_quats          device float[M][4]     } the caller zeroes them
 *   d_opacity_logits device float[M]        }
 *   d_sh             device float[M][K][3]  }
 * quats must be 16-byte aligned. Accumulation uses atomics, so the summation
 * order, and the last bits of the gradients, vary from run to run. Shares
 * the handle's tile counter with gs_trace_stochastic: order the calls on one
 * stream. */
gs_status gs_trace_backward(const gs_bvh *bvh, const gs_gaussians *g, const gs_pinhole *cam,
                            const gs_trace_params *p, const float *d_rgb, float *d_means,
                            float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_sh, void *stream);

/* gs_trace_backward with each sample's payload taken from `keys` instead
 * of a second forward traversal (the rendering's traversal is skipped;
 * the enumeration of the Gaussians in front of each winner remains).
 *   keys  device gs_sample_key[height][width][spp * n_hits], written by
 *         gs_trace_stochastic_keys with the same bvh, g, cam and p (seed,
 *         spp, n_hits, t range, stream_tag); samples_per_lane may differ
 * Other arguments, rules and errors as gs_trace_backward; keys NULL, not a
 * device pointer or not 4-byte aligned returns GS_ERR_INVALID_ARG. Given
 * the keys of that call, the gradients are those of gs_trace_backward (up
 * to the atomics' summation order). A key whose gid is neither 0xffffffff
 * nor below M is treated as no hit and makes gs_bvh_sync_status return
 * GS_ERR_INVALID_ARG. */
gs_status gs_trace_backward_keys(const gs_bvh *bvh, const gs_gaussians *g, const gs_pinhole *cam,
                                 const gs_trace_params *p, const gs_sample_key *keys,
                                 const float *d_rgb, float *d_means, float *d_log_scales,
                                 float *d_quats, float *d_opacity_logits, float *d_sh,
                                 void *stream);

/* Allocation-free variant of gs_build_bvh. The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- for
 * example a renderer thread that must never trigger the implicit device
 * synchronisation an allocation can cause, or a host application that hands
 * every byte of device memory to its own pool allocator up front.
 *
 * It runs the same kernels as gs_build_bvh and writes the same hierarchy,
 * byte for byte, into buffers the caller owns:
 *   g          Gaussian parameters (device arrays), 0 <= M <= 65536;
 *              larger M returns GS_ERR_INVALID_ARG (use gs_build_bvh)
 *   nodes_out  device, max(M-1, 1) * 64 bytes, 16-byte aligned: node
 *              records in the gs_bvh_export layout, node 0 the root
 *   prims_out  device, M * 64 bytes, 16-byte aligned: Gaussian records
 *   status_out device uint32, required (NULL returns GS_ERR_INVALID_ARG):
 *              the caller clears it; the build ORs error bits into it
 *              (non-zero means a non-finite parameter)
 *   stream     where the kernels are enqueued
 * Scratch memory lives in one statically allocated device array of this
 * library (about 4 MB on every GPU that loads the library, held until the
 * process exits). The first call on each device loads the library's module
 * there (CUDA loads modules lazily) and looks up that array's device address
 * (cudaGetSymbolAddress); loading a module may itself allocate and
 * synchronise, so make one warm-up call per device before the region that
 * must not allocate, and before any stream capture. The address is cached
 * per device and is invalid after cudaDeviceReset. Every call shares the
 * array: calls whose work overlaps on the GPU (different streams, or
 * different host threads) race and corrupt each other; serialise them, for
 * example on one stream. No cudaMalloc, cudaFree or other allocating call is
 * made. */
gs_status gs_build_bvh_noalloc(const gs_gaussians *g, void *nodes_out, void *prims_out,
                               uint32_t *status_out, void *stream);

/* ---------------------------------------------------------------------
 * Batched wavefront rendering: many views, shadows and one bounce.
 *
 * The Gaussians are emissive (their SH colour is their radiance, as the
 * paper assumes for Gaussians mixed with other assets, Sec. 5-6), placed
 * above an optional Lambertian ground quad (plane y = ground_y, normal +y,
 * |x|, |z| <= ground_half_extent) lit by point lights. Per sample of pixel
 * (x, y) of view v (ray id cams[v].ray_id_offset + y * width + x, sample s):
 *   camera ray (Philox stream tag 0): closest accepted Gaussian (t_g) or the
 *     ground (t_q); the nearer one shades the sample, the background if none;
 *   ground point p (float32: t_q = (ground_y - o.y) / d.y, p = o + t_q d with
 *     p.y = ground_y): radiance = albedo / pi * sum_l I_l V_l cos_l / r_l^2
 *     + albedo * L_b, where
 *   V_l (shadow ray to light l, stream tag 1 + l): 1 if no Gaussian is
 *     accepted on the open segment, i.e. Gaussians cast stochastic soft
 *     shadows; cos_l = max(0, omega_l.y), omega_l = normalise(light_l - p);
 *   L_b (bounce ray, stream tag 9, only if bounce != 0): colour of the
 *     closest accepted Gaussian along d_b, else the background; d_b =
 *     normalise((0,1,0) + u) with u uniform on the unit sphere, drawn by
 *     rejection from Philox-4x32-10 lanes (key = seed, counter = (ray id,
 *     attempt, s, 16), coordinate 2 * (w >> 8) * 2^-24 - 1, accepted when
 *     1e-8 < |v|^2 <= 1, up to 16 attempts, else u = (0,1,0)), a
 *     cosine-weighted direction.
 * Secondary rays start at p with t_min = shadow_eps; every vector above is
 * float32, each operation rounded once (normalise as for camera rays).
 * --------------------------------------------------------------------- */
typedef struct gs_light {
    float position[3];
    float intensity[3];
} gs_light;

typedef struct gs_scene_extras {
    int32_t n_lights;           /* 0..8 */
    gs_light lights[8];
    int32_t has_ground;         /* 0 or 1 */
    float ground_y;
    float ground_half_extent;
    float ground_albedo[3];
    int32_t bounce;             /* 0 or 1 */
    float shadow_eps;           /* t_min of shadow and bounce rays, > 0 */
} gs_scene_extras;

/* Launch shape of the wavefront kernel (picked by an autotuner).
 *   block_threads  threads per block: 64, 128 or 256 (0 = 128)
 *   stack_entries  traversal stack capacity: 48 or 96 (0 = 96) */
typedef struct gs_launch_options {
    int32_t block_threads;
    int32_t stack_entries;
    int32_t reserved[6];
} gs_launch_options;

/* Render n_views pinhole views (1..32, uneven sizes allowed). Warps take
 * pixel tiles from one queue over all views, the lanes of a pixel taking
 * its samples as in gs_trace_stochastic; below 64 samples per pixel (and
 * without counters or an inline bounce) a lane carries several consecutive
 * samples (8 from spp 8, 4 at spp 4-7, 2 at spp 2-3) as slots of one camera
 * walk and of one
 * shadow walk per light (a shadow slot ends at its first accepted
 * Gaussian); per-sample outcomes do not depend on it. Camera and shadow
 * rays are one ray per pixel (grouped traversal of the wide copies on
 * binary handles with 8 or more lanes per pixel, warp packets otherwise). When the ground and
 * the bounce are on (and the views hold fewer than 2^24 - 1 pixels, spp <=
 * 1024, pixels x spp <= 2^32 - 2^20) the bounce rays are deferred: each
 * sample slot gets a sort code (direction bin, then ground cell), the codes
 * are radix-sorted, and a second pass traces the bounce rays in that order,
 * on binary nodes each lane its own ray, taking the next code as soon as
 * its walk ends (a warp packet of 32 codes on 4-wide nodes), and
 * adds each pixel's bounce radiance in sample order; otherwise each lane
 * traces its bounce ray inline, the same way. The
 * deferred pass needs 28 bytes of device scratch per sample slot (total
 * pixels x spp), held by the handle and grown on first use (a synchronous
 * allocation; refused with GS_ERR_INVALID_ARG while `stream` is capturing
 * a graph: gs_graph_capture_views reserves it before capturing). The call
 * therefore modifies the handle's scratch, and calls on one handle must not
 * overlap on the GPU.
 *   bvh, g      as for gs_trace_stochastic (any node format)
 *   cams        host array [n_views]; ray ids must not overlap
 *   ex          host struct (above); NULL = no ground, lights or bounce
 *   p           spp >= 1 passes, n_hits must be 1; bg is the background
 *   opt         host struct or NULL for defaults
 *   rgb_out     device float[sum_v width_v * height_v][3], view v starting
 *               at pixel sum_{u<v} width_u * height_u
 *   counters    optional device uint64[4] incremented by the launch:
 *               {camera rays, shadow rays, bounce rays, node fetches by
 *               warps (child records fetched by groups in the grouped
 *               traversal)}
 *   samples_out optional device int32[spp][total pixels][3], per sample:
 *               camera hit (Gaussian id, -2 ground, -1 nothing), bounce hit
 *               (Gaussian id or -1), bit l set when light l was visible
 * Shares the handle's tile counter with gs_trace_stochastic. */
gs_status gs_render_views(const gs_bvh *bvh, const gs_gaussians *g, const gs_pinhole *cams,
                          int32_t n_views, const gs_scene_extras *ex, const gs_trace_params *p,
                          const gs_launch_options *opt, float *rgb_out,
                          unsigned long long *counters, int32_t *samples_out, void *stream);

/* A captured frame of the batched form: optionally the hierarchy rebuild
 * (parameters re-read from the same device arrays at every replay), then
 * the gs_render_views launch, recorded once as a CUDA graph and replayed
 * with gs_graph_launch. Arguments as for gs_render_views; `stream` must be
 * a non-default stream (the legacy default stream cannot be captured). The
 * deferred bounce's scratch is reserved before the capture starts. Every
 * replay renders the same rays with the same keys. */
typedef struct gs_graph gs_graph;

gs_status gs_graph_capture_views(gs_bvh *bvh, const gs_gaussians *g, int32_t rebuild,
                                 const gs_pinhole *cams, int32_t n_views,
                                 const gs_scene_extras *ex, const gs_trace_params *p,
                                 const gs_launch_options *opt, float *rgb_out, void *stream,
                                 gs_graph **out);

/* Replay a captured frame on `stream` (asynchronous). */
gs_status gs_graph_launch(gs_graph *graph, void *stream);

/* Release a captured frame. NULL is accepted. */
gs_status gs_graph_free(gs_graph *graph);

/* Short description of a status code (static string). */
const char *gs_status_string(gs_status s);

/* Detail of the last error returned on the calling thread (static buffer,
 * valid until the next call on that thread). */
const char *gs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* GSRT_H */
