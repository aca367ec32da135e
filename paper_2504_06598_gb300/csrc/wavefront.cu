// wavefront.cu -- many views, shadows and one diffuse bounce in one
// persistent launch (the path-tracing integration of Sec. 5: Gaussians
// among other assets cast soft shadows and light their surroundings).
//
// Warps take pixel tiles from one queue spanning every view (views of
// uneven size balance through the queue). As in the single-view trace a
// lane carries K consecutive samples (slots) and the L lanes of a pixel
// take interleaved passes of it. For each round a warp traces the camera
// ray of its lanes (K slots each); for the samples whose camera ray reaches
// the ground first, one shadow walk per light (any-hit: a slot stops at its
// first accepted Gaussian); the bounce ray of each such sample is deferred
// to a sorted pass of its own (or traced here, one sample per lane). Each
// ray type has its own Philox stream tag, so the draws of the different
// rays of a sample are independent.
#include <cuda_runtime.h>
#include <math.h>

#include "trace_common.cuh"

namespace gsrt {
namespace {

constexpr int kMaxViews = 32;
constexpr int kMaxLights = 8;
constexpr uint32_t kTagShadow = 1, kTagBounce = 9, kTagBounceDir = 16;

struct ViewDesc {
    float eye[3], look_at[3], up[3];
    float tan_half;
    int width, height;
    uint32_t ray_id_offset;
    uint32_t tile_begin;  // first tile of this view in the global queue
    uint32_t tiles_x;
    int64_t pix_begin;    // first pixel of this view in the packed output
};

struct WaveArgs {
    TraceArgs t;
    ViewDesc views[kMaxViews];
    int n_views;
    uint32_t total_tiles;
    int n_lights;
    float light_pos[kMaxLights][3];
    float light_int[kMaxLights][3];
    int has_ground;
    float ground_y, ground_half;
    float albedo[3];
    float albedo_over_pi[3];
    int bounce;
    float eps;
    unsigned long long *counters;
    int32_t *samples;  // optional [spp][n_pix][3] diagnostics
    int64_t n_pix;
    // deferred bounce: the camera pass writes one sort code per sample slot
    // (pixel * spp + sample); the bounce pass writes albedo x radiance
    int deferred;
    unsigned long long *codes;
    float *bounce_rgb;
    int spl;  // samples per lane of the camera and shadow pass (1, 2, 4 or 8)
};

// Sort code of a deferred bounce ray: 28 key bits (direction bin in an
// octahedral 64x64 map of the upper hemisphere, then the Morton order of
// the ground point on a 256x256 grid) above the pixel (24 bits) and the
// sample (10 bits). Codes of samples without a bounce are all ones; a
// bounce code is below 2^62, so on the sorted bits 32..63 it is strictly
// below every empty code and all empty codes sort last.
__device__ __forceinline__ uint32_t spread10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 8)) & 0x00ff00ffu;
    v = (v | (v << 4)) & 0x0f0f0f0fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ unsigned long long bounce_code(const WaveArgs &w, const float p[3],
                                                          const float d[3], int64_t gpix, int s) {
    const float l1 = fabsf(d[0]) + fabsf(d[1]) + fabsf(d[2]);
    const float u = d[0] / l1, v = d[2] / l1;
    const uint32_t qu = (uint32_t)min(63, max(0, (int)((u + 1.0f) * 32.0f)));
    const uint32_t qv = (uint32_t)min(63, max(0, (int)((v + 1.0f) * 32.0f)));
    const float inv = w.ground_half > 0.0f ? 1.0f / w.ground_half : 0.0f;
    const uint32_t qx = (uint32_t)min(255, max(0, (int)((p[0] * inv + 1.0f) * 128.0f)));
    const uint32_t qz = (uint32_t)min(255, max(0, (int)((p[2] * inv + 1.0f) * 128.0f)));
    const uint32_t key = (((qu << 6) | qv) << 16) | spread10(qx) | (spread10(qz) << 1);
    return ((unsigned long long)key << 34) | ((unsigned long long)gpix << 10) |
           (unsigned long long)s;
}

// Bounce direction: cosine-weighted about +y, normalise(n + u) with u
// uniform on the unit sphere by rejection from Philox lanes.
__device__ __forceinline__ void bounce_dir(const TraceArgs &a, uint32_t ray_id, uint32_t s,
                                           float d[3]) {
    float u[3] = {0.0f, 1.0f, 0.0f};
    for (uint32_t attempt = 0; attempt < 16; ++attempt) {
        const uint4 w = philox10(make_uint4(ray_id, attempt, s, kTagBounceDir), a.key0, a.key1);
        const uint32_t ws[3] = {w.x, w.y, w.z};
        float v[3];
        for (int i = 0; i < 3; ++i)
            v[i] = __fsub_rn(__fmul_rn(2.0f, (float)(ws[i] >> 8) * 0x1p-24f), 1.0f);
        float r2 = __fmul_rn(v[0], v[0]);
        r2 = __fadd_rn(r2, __fmul_rn(v[1], v[1]));
        r2 = __fadd_rn(r2, __fmul_rn(v[2], v[2]));
        if (r2 > 1e-8f && r2 <= 1.0f) {
            const float n = __fsqrt_rn(r2);
            for (int i = 0; i < 3; ++i) u[i] = __fdiv_rn(v[i], n);
            break;
        }
    }
    float b[3] = {u[0], __fadd_rn(1.0f, u[1]), u[2]};
    float n2 = __fmul_rn(b[0], b[0]);
    n2 = __fadd_rn(n2, __fmul_rn(b[1], b[1]));
    n2 = __fadd_rn(n2, __fmul_rn(b[2], b[2]));
    if (!(n2 > 1e-12f)) {
        d[0] = 0.0f; d[1] = 1.0f; d[2] = 0.0f;
        return;
    }
    const float n = __fsqrt_rn(n2);
    for (int i = 0; i < 3; ++i) d[i] = __fdiv_rn(b[i], n);
}

template <int FMT, bool COUNT, int K = 1>
__device__ __forceinline__ void trace_packet(const TraceArgs &a, Ray<K> &r, int pass,
                                             uint32_t *stack, float *stack_t, uint32_t &err,
                                             Counts &cnt) {
    if (a.n_nodes == 0) return;
    if constexpr (FMT == GS_NODES_BINARY || FMT == GS_NODES_BINARY_Q8)
        traverse_packet<K, COUNT>(a, r, pass, stack, stack_t, err, cnt);
    else traverse_packet_wide<K, COUNT, FMT>(a, r, pass, stack, stack_t, err, cnt);
}

// Bounce rays leave each lane in its own direction: on binary nodes each
// lane traverses alone instead of as a packet.
template <int FMT, bool COUNT>
__device__ __forceinline__ void trace_own_ray(const TraceArgs &a, Ray<1> &r, int pass,
                                              uint32_t *stack, float *stack_t, uint32_t &err,
                                              Counts &cnt) {
    if (a.n_nodes == 0) return;
    if constexpr (FMT == GS_NODES_BINARY || FMT == GS_NODES_BINARY_Q8)
        traverse_lane<1, COUNT>(a, r, pass, stack, stack_t, err, cnt);
    else traverse_packet_wide<1, COUNT, FMT>(a, r, pass, stack, stack_t, err, cnt);
}

// Camera and shadow rays are one ray for all lanes of a pixel: with groups
// of 2^GLG >= 8 lanes they take the grouped traversal of the wide copy.
template <int FMT, int GLG, bool COUNT, int K = 1>
__device__ __forceinline__ void trace_pixel_ray(const TraceArgs &a, Ray<K> &r, int pass,
                                                uint32_t *stack, float *stack_t, uint32_t *g_ref,
                                                float *g_t, uint32_t &err, Counts &cnt) {
    if (a.n_nodes == 0) return;
    if constexpr (GLG >= 3)
        traverse_group<K, COUNT, GLG, false, FMT == GS_NODES_BINARY_Q8>(a, r, pass, g_ref, g_t, err,
                                                                        cnt);
    else trace_packet<FMT, COUNT, K>(a, r, pass, stack, stack_t, err, cnt);
}

// Slots of pass `pass` of a lane carrying K samples: sample pass * K + k is
// live below the pixel's sample count, the others sit at -inf (nothing is
// closer, they never set the clip).
template <int K>
__device__ __forceinline__ void reset_live_slots(Ray<K> &r, int pass, int n_samples,
                                                 const bool need[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
        r.slot[k] = need[k] && pass * K + k < n_samples ? Slot{INFINITY, 0.0f, 0xffffffffu}
                                                        : Slot{-INFINITY, 0.0f, 0xffffffffu};
}

// Both passes of the batched form are latency-bound; they are built for 64
// registers (four 256-thread or eight 128-thread blocks per SM), measured
// faster than 80 or 105 registers at fewer blocks.
constexpr int kWaveMaxThreads = 256;
constexpr int kWaveMinBlocks = 4;

// GLG: log2 of the lanes per pixel when the grouped traversal is used, else
// 0. The group stacks are dynamic shared memory: per warp kGroupPool
// references then kGroupPool entry distances. K: samples a lane carries
// (slots of its camera and shadow rays); pass j of a lane holds samples
// j * K .. j * K + K - 1 of its pixel, each with its own keys, outcome and
// deferred bounce slot, exactly as K lanes with one sample each. Built
// for four 256-thread blocks per SM with every K (eight slots, 16-view
// frame at spp 8, 16 and 32: 202.4, 381.8 and 737.7 ms against 205.5,
// 386.9 and 747.4 with three blocks; 423.7 with two at spp 16).
template <int FMT, int STACK, bool COUNT, int GLG, int K = 1>
__global__ void __launch_bounds__(kWaveMaxThreads, kWaveMinBlocks)
    k_render_views(const WaveArgs w) {
    const TraceArgs &a = w.t;
    const int lane = threadIdx.x & 31;
    const uint32_t kAll = 0xffffffffu;
    extern __shared__ uint32_t wave_smem[];
    uint32_t *g_ref = nullptr;
    float *g_t = nullptr;
    if constexpr (GLG >= 3) {
        uint32_t *pool = wave_smem + (size_t)(threadIdx.x >> 5) * 2 * kGroupPool;
        const int off = (lane >> GLG) * (kGroupPool >> (5 - GLG));
        g_ref = pool + off;
        g_t = reinterpret_cast<float *>(pool + kGroupPool) + off;
    }
    const int lg = a.lpp_log2, L = 1 << lg;
    const int tw_lg = tile_w_log2(lg), th_lg = 5 - lg - tw_lg;
    const int sub = lane & (L - 1), pl = lane >> lg;
    const int S = a.n_samples;  // samples per pixel
    uint32_t stack[STACK];
    float stack_t[STACK];
    uint32_t err = 0;
    Counts cnt;
    unsigned long long n_cam = 0, n_shadow = 0, n_bounce = 0;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(a.work, 1u);
        tile = __shfl_sync(kAll, tile, 0);
        if (tile >= w.total_tiles) break;
        int v = 0;
        while (v + 1 < w.n_views && w.views[v + 1].tile_begin <= tile) ++v;
        const ViewDesc &vw = w.views[v];
        const uint32_t lt = tile - vw.tile_begin;
        const int x = (int)(((lt % vw.tiles_x) << tw_lg) + (pl & ((1 << tw_lg) - 1)));
        const int y = (int)(((lt / vw.tiles_x) << th_lg) + (pl >> tw_lg));
        const bool valid = x < vw.width && y < vw.height;
        const int64_t lpix = valid ? (int64_t)y * vw.width + x : 0;
        const uint32_t ray_id = vw.ray_id_offset + (uint32_t)lpix;
        float d0[3];
        camera_ray_view(vw.eye, vw.look_at, vw.up, vw.tan_half, vw.width, vw.height,
                        valid ? x : 0, valid ? y : 0, d0);
        float Y0[16];
        sh_basis(a.sh_degree, d0, Y0);
        // ground hit of the camera ray (fixed for the pixel)
        bool ground = false;
        float tq = INFINITY, p[3] = {0.0f, 0.0f, 0.0f};
        if (w.has_ground && valid && d0[1] != 0.0f) {
            tq = __fdiv_rn(__fsub_rn(w.ground_y, vw.eye[1]), d0[1]);
            p[0] = __fadd_rn(vw.eye[0], __fmul_rn(tq, d0[0]));
            p[1] = w.ground_y;
            p[2] = __fadd_rn(vw.eye[2], __fmul_rn(tq, d0[2]));
            ground = tq > a.t_min && fabsf(p[0]) <= w.ground_half && fabsf(p[2]) <= w.ground_half;
            if (!ground) tq = INFINITY;
        }
        float acc[3] = {0.0f, 0.0f, 0.0f};
        const int n_rounds = (a.spp + L - 1) >> lg;
        for (int j = 0; j < n_rounds; ++j) {
            const int pass = (j << lg) + sub;
            bool live[K];
#pragma unroll
            for (int k = 0; k < K; ++k) live[k] = valid && pass * K + k < S;
            // camera ray: K samples of the pixel's ray
            Ray<K> r;
            set_ray(r, vw.eye, d0);
            r.ray_id = ray_id;
            r.stream_tag = a.stream_tag;
            r.t_min = a.t_min;
            r.t_max = a.t_max;
            r.any_hit = false;
            reset_live_slots<K>(r, pass, S, live);
            update_clip(r, r.t_max);
            if (!live[0]) r.t_far = -INFINITY;
            trace_pixel_ray<FMT, GLG, COUNT, K>(a, r, pass, stack, stack_t, g_ref, g_t, err, cnt);
            float c[K][3];
            bool on_ground[K];
            int32_t diag_cam[K], diag_bounce[K], diag_vis[K];
#pragma unroll
            for (int k = 0; k < K; ++k) {
                n_cam += live[k];
                const bool gauss = live[k] && r.slot[k].gid != 0xffffffffu && r.slot[k].t() < tq;
                on_ground[k] = live[k] && ground && !gauss;
                c[k][0] = a.bg[0]; c[k][1] = a.bg[1]; c[k][2] = a.bg[2];
                diag_cam[k] = -1; diag_bounce[k] = -1; diag_vis[k] = 0;
                if (gauss) {
                    sh_colour(a, r.slot[k].gid, Y0, c[k]);
                    diag_cam[k] = (int32_t)r.slot[k].gid;
                }
                if (on_ground[k]) {
                    c[k][0] = c[k][1] = c[k][2] = 0.0f;
                    diag_cam[k] = -2;
                }
            }
            // one shadow packet per light
            for (int l = 0; l < w.n_lights; ++l) {
                float wl[3], omega[3];
                for (int i = 0; i < 3; ++i) wl[i] = __fsub_rn(w.light_pos[l][i], p[i]);
                float dist2 = __fmul_rn(wl[0], wl[0]);
                dist2 = __fadd_rn(dist2, __fmul_rn(wl[1], wl[1]));
                dist2 = __fadd_rn(dist2, __fmul_rn(wl[2], wl[2]));
                const float dist = __fsqrt_rn(dist2);
                for (int i = 0; i < 3; ++i) omega[i] = __fdiv_rn(wl[i], dist);
                const bool lit = omega[1] > 0.0f && dist2 > 0.0f;
                bool need[K];
                bool any_need = false;
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    need[k] = on_ground[k] && lit;
                    any_need |= need[k];
                }
                if (!__any_sync(kAll, any_need)) continue;
                // one ray for the pixel's lanes (the grouped traversal tests
                // each child against the group's ray), one slot per sample
                const bool pix_ok = ground && dist2 > 0.0f;
                Ray<K> sr;
                set_ray(sr, p, pix_ok ? omega : d0);
                sr.ray_id = ray_id;
                sr.stream_tag = kTagShadow + (uint32_t)l;
                sr.t_min = w.eps;
                sr.t_max = dist;
                sr.any_hit = true;
                reset_live_slots<K>(sr, pass, S, need);
                update_clip(sr, sr.t_max);
                if (!any_need) sr.t_far = -INFINITY;
                trace_pixel_ray<FMT, GLG, COUNT, K>(a, sr, pass, stack, stack_t, g_ref, g_t, err, cnt);
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    n_shadow += need[k];
                    if (need[k] && sr.slot[k].gid == 0xffffffffu) {
                        diag_vis[k] |= 1 << l;
                        const float kk = __fdiv_rn(omega[1], dist2);
                        for (int i = 0; i < 3; ++i)
                            c[k][i] = fmaf(w.albedo_over_pi[i] * w.light_int[l][i], kk, c[k][i]);
                    }
                }
            }
            // one diffuse bounce: deferred to the sorted bounce pass, or
            // traced here (one sample per lane only)
            if (w.bounce && w.deferred) {
#pragma unroll
                for (int k = 0; k < K; ++k) {
                    if (!live[k]) continue;
                    const int s = pass * K + k;
                    const int64_t gpix = vw.pix_begin + lpix;
                    const int64_t slot = gpix * S + s;
                    unsigned long long code = ~0ull;
                    if (on_ground[k]) {
                        float db[3] = {0.0f, 1.0f, 0.0f};
                        bounce_dir(a, ray_id, (uint32_t)s, db);
                        code = bounce_code(w, p, db, gpix, s);
                        ++n_bounce;
                    }
                    w.codes[slot] = code;
                    w.bounce_rgb[3 * slot] = 0.0f;
                    w.bounce_rgb[3 * slot + 1] = 0.0f;
                    w.bounce_rgb[3 * slot + 2] = 0.0f;
                }
            } else if constexpr (K == 1) {
                if (w.bounce) {
                    const int s = pass;
                    float db[3] = {0.0f, 1.0f, 0.0f};
                    if (on_ground[0]) bounce_dir(a, ray_id, (uint32_t)s, db);
                    const bool need = on_ground[0];
                    if (__any_sync(kAll, need)) {
                        Ray<1> br;
                        set_ray(br, p, db);
                        br.ray_id = ray_id;
                        br.stream_tag = kTagBounce;
                        br.t_min = w.eps;
                        br.t_max = INFINITY;
                        br.any_hit = false;
                        reset_slots(br);
                        update_clip(br, br.t_max);
                        if (!need) br.t_far = -INFINITY;
                        trace_own_ray<FMT, COUNT>(a, br, s, stack, stack_t, err, cnt);
                        n_bounce += need;
                        if (need) {
                            float lb[3] = {a.bg[0], a.bg[1], a.bg[2]};
                            if (br.slot[0].gid != 0xffffffffu) {
                                float Yb[16];
                                sh_basis(a.sh_degree, db, Yb);
                                sh_colour(a, br.slot[0].gid, Yb, lb);
                                diag_bounce[0] = (int32_t)br.slot[0].gid;
                            }
                            for (int i = 0; i < 3; ++i) c[0][i] = fmaf(w.albedo[i], lb[i], c[0][i]);
                        }
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < K; ++k) {
                if (!live[k]) continue;
                acc[0] += c[k][0];
                acc[1] += c[k][1];
                acc[2] += c[k][2];
                if (w.samples) {
                    const int64_t o = ((int64_t)(pass * K + k) * w.n_pix + vw.pix_begin + lpix) * 3;
                    w.samples[o] = diag_cam[k];
                    w.samples[o + 1] = diag_bounce[k];
                    w.samples[o + 2] = diag_vis[k];
                }
            }
            __syncwarp();
        }
        // the pixel's lanes add their partial sums
        for (int o = L >> 1; o >= 1; o >>= 1) {
            acc[0] += __shfl_xor_sync(kAll, acc[0], o);
            acc[1] += __shfl_xor_sync(kAll, acc[1], o);
            acc[2] += __shfl_xor_sync(kAll, acc[2], o);
        }
        if (valid && sub == 0) {
            const float inv_n = 1.0f / (float)S;
            const int64_t o = 3 * (vw.pix_begin + lpix);
            a.rgb[o] = acc[0] * inv_n;
            a.rgb[o + 1] = acc[1] * inv_n;
            a.rgb[o + 2] = acc[2] * inv_n;
        }
    }
    if (err) atomicOr(a.status, err);
    if (COUNT) {
        atomicAdd(w.counters + 0, n_cam);
        atomicAdd(w.counters + 1, n_shadow);
        atomicAdd(w.counters + 2, n_bounce);
        atomicAdd(w.counters + 3, cnt.node_fetch);
    }
}

// The bounce ray of a deferred sample code: the sample's ground point and
// bounce direction rebuilt with the camera pass's arithmetic.
__device__ __forceinline__ void bounce_ray(const WaveArgs &w, unsigned long long code, Ray<1> &br,
                                           int64_t &gpix, int &s) {
    gpix = (int64_t)((code >> 10) & 0xffffffull);
    s = (int)(code & 1023ull);
    int v = 0;
    while (v + 1 < w.n_views && w.views[v + 1].pix_begin <= gpix) ++v;
    const ViewDesc &vw = w.views[v];
    const int64_t lpix = gpix - vw.pix_begin;
    const int x = (int)(lpix % vw.width), y = (int)(lpix / vw.width);
    const uint32_t ray_id = vw.ray_id_offset + (uint32_t)lpix;
    float d0[3];
    camera_ray_view(vw.eye, vw.look_at, vw.up, vw.tan_half, vw.width, vw.height, x, y, d0);
    float p[3] = {0.0f, w.ground_y, 0.0f};
    float db[3] = {0.0f, 1.0f, 0.0f};
    const float tq = __fdiv_rn(__fsub_rn(w.ground_y, vw.eye[1]), d0[1]);
    p[0] = __fadd_rn(vw.eye[0], __fmul_rn(tq, d0[0]));
    p[2] = __fadd_rn(vw.eye[2], __fmul_rn(tq, d0[2]));
    bounce_dir(w.t, ray_id, (uint32_t)s, db);
    set_ray(br, p, db);
    br.ray_id = ray_id;
    br.stream_tag = kTagBounce;
    br.t_min = w.eps;
    br.t_max = INFINITY;
    br.any_hit = false;
    reset_slots(br);
    update_clip(br, br.t_max);
}

// Shades a finished bounce ray and writes albedo x radiance to its slot.
__device__ __forceinline__ void bounce_finish(const WaveArgs &w, const Ray<1> &br, int64_t gpix,
                                              int s) {
    const TraceArgs &a = w.t;
    float lb[3] = {a.bg[0], a.bg[1], a.bg[2]};
    if (br.slot[0].gid != 0xffffffffu) {
        float Yb[16];
        sh_basis(a.sh_degree, br.d, Yb);
        sh_colour(a, br.slot[0].gid, Yb, lb);
        if (w.samples) w.samples[((int64_t)s * w.n_pix + gpix) * 3 + 1] = (int32_t)br.slot[0].gid;
    }
    const int64_t slot = gpix * a.n_samples + s;
    for (int c = 0; c < 3; ++c) w.bounce_rgb[3 * slot + c] = w.albedo[c] * lb[c];
}

// One step of traverse_lane's walk of the binary nodes, its state (node,
// stack depth, steps) held by the caller: false once the walk has ended.
template <bool COUNT>
__device__ __forceinline__ bool lane_step(const TraceArgs &a, Ray<1> &r, int pass, uint32_t &node,
                                          int &sp, uint32_t &steps, uint32_t *stack,
                                          float *stack_t, uint32_t &err, Counts &cnt) {
    if (++steps > a.step_limit) {
        err |= kErrSteps;
        return false;
    }
    if (COUNT) {
        ++cnt.nodes;
        ++cnt.node_fetch;
    }
    const float4 *np = reinterpret_cast<const float4 *>(a.nodes + node);
    const float4 b0 = __ldg(np), b1 = __ldg(np + 1), b2 = __ldg(np + 2);
    const uint4 cref = __ldg(reinterpret_cast<const uint4 *>(np + 3));
    const float boxL[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
    const float boxR[6] = {b1.z, b1.w, b2.x, b2.y, b2.z, b2.w};
    float tL, tR;
    bool hL = slab(boxL, r.inv, r.oinv, r.t_min, r.t_far, tL);
    bool hR = slab(boxR, r.inv, r.oinv, r.t_min, r.t_far, tR);
    const bool leafL = (cref.x & kLeafBit) != 0u, leafR = (cref.y & kLeafBit) != 0u;
    if ((leafL && hL) || (leafR && hR)) {
        const bool swap = leafL && leafR && hR && (!hL || tR < tL);
        for (int li = 0; li < 2; ++li) {
            const bool right = (li == 0) == swap;
            if (!(right ? leafR : leafL) || !(right ? hR : hL)) continue;
            if (COUNT) {
                ++cnt.prims;
                ++cnt.prim_fetch;
            }
            intersect<1, COUNT>(a, r, (right ? cref.y : cref.x) & ~kLeafBit, pass, cnt.draws);
        }
    }
    hL = hL && !leafL && tL <= r.t_far;
    hR = hR && !leafR && tR <= r.t_far;
    if (hL && hR) {
        if (sp >= a.stack_depth) {
            err |= kErrStack;
            return false;
        }
        const bool left_first = tL <= tR;
        stack[sp] = left_first ? cref.y : cref.x;
        stack_t[sp] = left_first ? tR : tL;
        ++sp;
        node = left_first ? cref.x : cref.y;
        return true;
    }
    if (hL) {
        node = cref.x;
        return true;
    }
    if (hR) {
        node = cref.y;
        return true;
    }
    while (sp > 0) {
        --sp;
        if (stack_t[sp] <= r.t_far) {
            node = stack[sp];
            return true;
        }
    }
    return false;
}

// Deferred bounce pass over the sorted codes (empty codes sort last), so
// that a warp holds bounce rays of nearby directions from nearby ground
// points (the path tracer's wavefront regrouping of secondary rays). On
// binary nodes each lane walks its own ray, one node per loop step, and a
// lane whose ray has ended takes the next code from the queue at once
// (lanes that need one share an atomic): a warp's lanes stay busy instead
// of waiting for its longest walk (the persistent traversal with ray
// replacement of Aila and Laine, HPG 2009). Each lane shades its ray when
// the walk ends and writes albedo x radiance to the sample's slot. On
// 4-wide nodes a warp takes 32 consecutive codes and walks them as a
// packet.
template <int FMT, int STACK, bool COUNT>
__global__ void __launch_bounds__(kWaveMaxThreads, kWaveMinBlocks)
    k_bounce(const WaveArgs w, const unsigned long long *__restrict__ codes, int64_t n_slots) {
    const TraceArgs &a = w.t;
    const int lane = threadIdx.x & 31;
    const uint32_t kAll = 0xffffffffu;
    uint32_t stack[STACK];
    float stack_t[STACK];
    uint32_t err = 0;
    Counts cnt;
    if constexpr (FMT == GS_NODES_BINARY || FMT == GS_NODES_BINARY_Q8) {
        // the work counter counts codes; the launcher keeps n_slots + the
        // launch's threads below 2^32
        bool active = false, more = true;
        int64_t gpix = 0;
        int s = 0;
        Ray<1> br;
        uint32_t node = 0, steps = 0;
        int sp = 0;
        for (;;) {
            const uint32_t idle = __ballot_sync(kAll, !active && more);
            if (idle) {
                const int leader = __ffs(idle) - 1;
                uint32_t first = 0;
                if (lane == leader) first = atomicAdd(a.work, (uint32_t)__popc(idle));
                first = __shfl_sync(kAll, first, leader);
                if (!active && more) {
                    const int64_t i = (int64_t)first + __popc(idle & ((1u << lane) - 1u));
                    const unsigned long long code = i < n_slots ? codes[i] : ~0ull;
                    if (code == ~0ull) {
                        more = false;
                    } else {
                        bounce_ray(w, code, br, gpix, s);
                        node = 0;
                        sp = 0;
                        steps = 0;
                        active = a.n_nodes > 0 && br.t_far >= br.t_min;
                        if (!active) bounce_finish(w, br, gpix, s);
                    }
                }
            }
            if (!__any_sync(kAll, active) && !__any_sync(kAll, more)) break;
            if (active && !lane_step<COUNT>(a, br, s, node, sp, steps, stack, stack_t, err, cnt)) {
                active = false;
                bounce_finish(w, br, gpix, s);
            }
        }
    } else {
        for (;;) {
            uint32_t tile = 0;
            if (lane == 0) tile = atomicAdd(a.work, 1u);
            tile = __shfl_sync(kAll, tile, 0);
            if ((int64_t)tile * 32 >= n_slots) break;
            const int64_t i = (int64_t)tile * 32 + lane;
            const unsigned long long code = i < n_slots ? codes[i] : ~0ull;
            const bool valid = code != ~0ull;
            if (!__any_sync(kAll, valid)) break;
            int64_t gpix = 0;
            int s = 0;
            Ray<1> br;
            if (valid) {
                bounce_ray(w, code, br, gpix, s);
            } else {
                const float p[3] = {0.0f, w.ground_y, 0.0f}, db[3] = {0.0f, 1.0f, 0.0f};
                set_ray(br, p, db);
                br.ray_id = 0;
                br.stream_tag = kTagBounce;
                br.t_min = w.eps;
                br.t_max = INFINITY;
                br.any_hit = false;
                reset_slots(br);
                br.t_far = -INFINITY;
            }
            trace_own_ray<FMT, COUNT>(a, br, s, stack, stack_t, err, cnt);
            if (valid) bounce_finish(w, br, gpix, s);
            __syncwarp();
        }
    }
    if (err) atomicOr(a.status, err);
    if (COUNT) atomicAdd(w.counters + 3, cnt.node_fetch);
}

// Adds each pixel's bounce radiance, in sample order, to its mean.
__global__ void k_combine(const WaveArgs w) {
    const int64_t px = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (px >= w.n_pix) return;
    const TraceArgs &a = w.t;
    float sum[3] = {0.0f, 0.0f, 0.0f};
    const float *b = w.bounce_rgb + 3 * px * a.n_samples;
    for (int s = 0; s < a.n_samples; ++s)
        for (int c = 0; c < 3; ++c) sum[c] += b[3 * s + c];
    const float inv_n = 1.0f / (float)a.n_samples;
    for (int c = 0; c < 3; ++c) a.rgb[3 * px + c] = fmaf(sum[c], inv_n, a.rgb[3 * px + c]);
}

template <int FMT, int STACK, bool COUNT>
gs_status launch_bounce(const WaveArgs &w, const unsigned long long *codes, int64_t n_slots,
                        int threads, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bounce<FMT, STACK, COUNT>,
                                                          threads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "bounce launch setup");
    const int64_t tiles = (n_slots + 31) / 32;
    const uint32_t warps_per_block = (uint32_t)threads / 32;
    uint32_t blocks = (uint32_t)sms * (uint32_t)(per > 0 ? per : 1);
    const int64_t max_blocks = (tiles + warps_per_block - 1) / warps_per_block;
    if ((int64_t)blocks > max_blocks) blocks = (uint32_t)max_blocks;
    if (blocks == 0) return GS_OK;
    if ((e = cudaMemsetAsync(w.t.work, 0, sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "reset work counter");
    k_bounce<FMT, STACK, COUNT><<<blocks, threads, 0, s>>>(w, codes, n_slots);
    k_combine<<<(unsigned)((w.n_pix + 255) / 256), 256, 0, s>>>(w);
    return GS_OK;
}

template <int FMT>
gs_status launch_bounce_f(const WaveArgs &w, const unsigned long long *codes, int64_t n_slots,
                          int threads, int stack, cudaStream_t s) {
    const bool count = w.counters != nullptr;
    if (stack == 48)
        return count ? launch_bounce<FMT, 48, true>(w, codes, n_slots, threads, s)
                     : launch_bounce<FMT, 48, false>(w, codes, n_slots, threads, s);
    return count ? launch_bounce<FMT, 96, true>(w, codes, n_slots, threads, s)
                 : launch_bounce<FMT, 96, false>(w, codes, n_slots, threads, s);
}

template <int FMT, int STACK, bool COUNT, int GLG, int K = 1>
gs_status launch_views(const WaveArgs &w, int threads, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    const size_t smem = GLG >= 3 ? (size_t)(threads / 32) * 2 * kGroupPool * sizeof(uint32_t) : 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per, k_render_views<FMT, STACK, COUNT, GLG, K>, threads, smem);
    if (e != cudaSuccess) return cuda_fail(e, "render launch setup");
    const uint32_t warps_per_block = (uint32_t)threads / 32;
    uint32_t blocks = (uint32_t)sms * (uint32_t)(per > 0 ? per : 1);
    const uint32_t max_blocks = (w.total_tiles + warps_per_block - 1) / warps_per_block;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks == 0) return GS_OK;
    if ((e = cudaMemsetAsync(w.t.work, 0, sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "reset work counter");
    k_render_views<FMT, STACK, COUNT, GLG, K><<<blocks, threads, smem, s>>>(w);
    return GS_OK;
}

template <int FMT, int GLG>
gs_status launch_views_g(const WaveArgs &w, int threads, int stack, cudaStream_t s) {
    const bool count = w.counters != nullptr;
    // several samples per lane: packets only (fewer than 8 lanes a pixel),
    // never with counters
    if constexpr (GLG == 0) {
        if (!count && w.spl == 8)
            return stack == 48 ? launch_views<FMT, 48, false, 0, 8>(w, threads, s)
                               : launch_views<FMT, 96, false, 0, 8>(w, threads, s);
        if (!count && w.spl == 4)
            return stack == 48 ? launch_views<FMT, 48, false, 0, 4>(w, threads, s)
                               : launch_views<FMT, 96, false, 0, 4>(w, threads, s);
        if (!count && w.spl == 2)
            return stack == 48 ? launch_views<FMT, 48, false, 0, 2>(w, threads, s)
                               : launch_views<FMT, 96, false, 0, 2>(w, threads, s);
    }
    if (stack == 48)
        return count ? launch_views<FMT, 48, true, GLG>(w, threads, s)
                     : launch_views<FMT, 48, false, GLG>(w, threads, s);
    return count ? launch_views<FMT, 96, true, GLG>(w, threads, s)
                 : launch_views<FMT, 96, false, GLG>(w, threads, s);
}

template <int FMT>
gs_status launch_views_f(const WaveArgs &w, int threads, int stack, cudaStream_t s) {
    return launch_views_g<FMT, 0>(w, threads, stack, s);
}

// Binary handles with wide copies: pixels with 8 or more lanes group.
template <>
gs_status launch_views_f<GS_NODES_BINARY>(const WaveArgs &w, int threads, int stack, cudaStream_t s) {
    if (w.t.grec != nullptr) {
        switch (w.t.lpp_log2) {
            case 5: return launch_views_g<GS_NODES_BINARY, 5>(w, threads, stack, s);
            case 4: return launch_views_g<GS_NODES_BINARY, 4>(w, threads, stack, s);
            case 3: return launch_views_g<GS_NODES_BINARY, 3>(w, threads, stack, s);
            default: break;
        }
    }
    return launch_views_g<GS_NODES_BINARY, 0>(w, threads, stack, s);
}

// Binary handles with 8-bit wide copies: the groups read the 8-bit records;
// everything else is the binary form's.
template <>
gs_status launch_views_f<GS_NODES_BINARY_Q8>(const WaveArgs &w, int threads, int stack,
                                             cudaStream_t s) {
    if (w.t.grec != nullptr) {
        switch (w.t.lpp_log2) {
            case 5: return launch_views_g<GS_NODES_BINARY_Q8, 5>(w, threads, stack, s);
            case 4: return launch_views_g<GS_NODES_BINARY_Q8, 4>(w, threads, stack, s);
            case 3: return launch_views_g<GS_NODES_BINARY_Q8, 3>(w, threads, stack, s);
            default: break;
        }
    }
    return launch_views_g<GS_NODES_BINARY, 0>(w, threads, stack, s);
}

}  // namespace

int64_t wave_slots(const gs_pinhole *cams, int n_views, const gs_scene_extras *ex,
                   const gs_trace_params *p) {
    if (!ex || !ex->bounce || !ex->has_ground || p->spp < 1 || p->spp > 1024) return 0;
    int64_t pix = 0;
    for (int v = 0; v < n_views; ++v) pix += (int64_t)cams[v].width * cams[v].height;
    if (pix >= (int64_t)(1 << 24) - 1) return 0;  // the code's pixel field
    // the bounce pass counts codes in 32 bits, with room for its threads'
    // last fetches past the end
    if (pix * p->spp > (int64_t)0xFFFFFFFFll - (1 << 20)) return 0;
    return pix * p->spp;
}

gs_status reserve_wave_scratch(gs_bvh *b, int64_t slots, cudaStream_t s) {
    if (b->wave_cap >= slots) return GS_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
        return fail(GS_ERR_INVALID_ARG,
                    "the batched form's scratch must be reserved before a graph capture");
    void **bufs[] = {(void **)&b->wave_codes[0], (void **)&b->wave_codes[1],
                     (void **)&b->wave_bounce, (void **)&b->wave_hist, (void **)&b->wave_scan};
    for (void **q : bufs)
        if (*q) {
            cudaFree(*q);
            *q = nullptr;
        }
    b->device_bytes -= b->wave_bytes;
    b->wave_bytes = 0;
    b->wave_cap = 0;
    const int64_t tiles = radix_tiles(slots);
    const size_t sizes[] = {(size_t)slots * 8, (size_t)slots * 8, (size_t)slots * 12,
                            (size_t)tiles * 256 * 4, (size_t)scan_tmp_entries(256 * tiles) * 4};
    for (int k = 0; k < 5; ++k) {
        cudaError_t e = cudaMalloc(bufs[k], sizes[k]);
        if (e != cudaSuccess) {
            for (void **q : bufs)
                if (*q) {
                    cudaFree(*q);
                    *q = nullptr;
                }
            b->wave_cap = 0;
            return cuda_fail(e, "batched form scratch");
        }
    }
    b->wave_cap = slots;
    for (size_t z : sizes) b->wave_bytes += (int64_t)z;
    b->device_bytes += b->wave_bytes;
    return GS_OK;
}

gs_status launch_render_views(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cams,
                              int n_views, const gs_scene_extras *ex, const gs_trace_params *p,
                              const gs_launch_options *opt, float *rgb, unsigned long long *counters,
                              int32_t *samples, cudaStream_t s) {
    WaveArgs w = {};
    TraceArgs &a = w.t;
    a.nodes = b->nodes;
    a.wide = b->wide;
    a.prims = b->prims;
    a.sh = g->sh;
    a.n_nodes = b->n_nodes;
    a.sh_degree = g->sh_degree;
    a.sh_dtype = g->sh_dtype;
    for (int i = 0; i < 3; ++i) a.bg[i] = p->bg[i];
    a.key0 = (uint32_t)(p->seed & 0xffffffffu);
    a.key1 = (uint32_t)(p->seed >> 32);
    philox_round_keys(a.key0, a.key1, a.rk);
    a.stream_tag = p->stream_tag;
    // samples per lane of the camera and shadow pass: 8 from spp 8 to 63
    // (per-lane packets), 4 at spp 4-7, 2 at spp 2-3; one from spp 64 (grouped), with
    // counters, or with the bounce traced inline. Frame of 16 views 256^2
    // to 1080p with ground, four lights and a bounce, one sample per lane
    // -> four -> eight: spp 16 634 -> 472 -> 430 ms, spp 8 -> 269 -> 251,
    // spp 32 806 (one) -> 770 (eight).
    const int64_t bounce_slots = wave_slots(cams, n_views, ex, p);
    const bool inline_bounce = ex && ex->bounce && ex->has_ground && bounce_slots == 0;
    int K = 1;
    if (counters == nullptr && !inline_bounce && p->spp >= 2 && p->spp < 64)
        K = p->spp >= 8 ? 8 : (p->spp >= 4 ? 4 : 2);
    w.spl = K;
    a.spp = (p->spp + K - 1) / K;
    a.n_samples = p->spp;
    a.t_min = p->t_min;
    a.t_max = p->t_max;
    const int stack = (opt && opt->stack_entries == 48) ? 48 : 96;
    a.stack_depth = (p->stack_depth == 0 || p->stack_depth > stack) ? stack : p->stack_depth;
    a.step_limit = (uint32_t)(b->n_nodes + 8 < (int64_t)kStepLimit ? b->n_nodes + 8 : kStepLimit);
    a.rgb = rgb;
    a.status = b->status;
    a.work = b->status + 1;
    a.lpp_log2 = lanes_per_pixel_log2(a.spp);
    if (b->node_depth && a.lpp_log2 >= 3) {
        a.grec = b->group[a.lpp_log2 - 3].rec;
        a.gcnt = b->group[a.lpp_log2 - 3].cnt;
        a.gq8 = b->node_format == GS_NODES_BINARY_Q8;
    }
    const int tw_lg = tile_w_log2(a.lpp_log2), th_lg = 5 - a.lpp_log2 - tw_lg;
    uint32_t tiles = 0;
    int64_t pix = 0;
    for (int v = 0; v < n_views; ++v) {
        ViewDesc &d = w.views[v];
        for (int i = 0; i < 3; ++i) {
            d.eye[i] = cams[v].eye[i];
            d.look_at[i] = cams[v].look_at[i];
            d.up[i] = cams[v].up[i];
        }
        d.tan_half = (float)tan((double)cams[v].fov_y_deg * 3.14159265358979323846 / 360.0);
        d.width = cams[v].width;
        d.height = cams[v].height;
        d.ray_id_offset = cams[v].ray_id_offset;
        d.tiles_x = (uint32_t)((cams[v].width + (1 << tw_lg) - 1) >> tw_lg);
        d.tile_begin = tiles;
        d.pix_begin = pix;
        tiles += d.tiles_x * (uint32_t)((cams[v].height + (1 << th_lg) - 1) >> th_lg);
        pix += (int64_t)cams[v].width * cams[v].height;
    }
    w.n_views = n_views;
    w.total_tiles = tiles;
    w.n_pix = pix;
    if (ex) {
        w.n_lights = ex->n_lights;
        for (int l = 0; l < ex->n_lights; ++l)
            for (int i = 0; i < 3; ++i) {
                w.light_pos[l][i] = ex->lights[l].position[i];
                w.light_int[l][i] = ex->lights[l].intensity[i];
            }
        w.has_ground = ex->has_ground;
        w.ground_y = ex->ground_y;
        w.ground_half = ex->ground_half_extent;
        for (int i = 0; i < 3; ++i) {
            w.albedo[i] = ex->ground_albedo[i];
            w.albedo_over_pi[i] = (float)((double)ex->ground_albedo[i] / 3.14159265358979323846);
        }
        w.bounce = ex->bounce;
        w.eps = ex->shadow_eps;
    }
    w.counters = counters;
    w.samples = samples;
    const int threads = opt && opt->block_threads ? opt->block_threads : 128;
    // the bounce rays are sorted by direction and ground position and traced
    // in a pass of their own; the handle holds the scratch
    const int64_t slots = bounce_slots;
    gs_status st;
    if (slots > 0) {
        gs_bvh *mb = const_cast<gs_bvh *>(b);
        if ((st = reserve_wave_scratch(mb, slots, s)) != GS_OK) return st;
        w.deferred = 1;
        w.codes = mb->wave_codes[0];
        w.bounce_rgb = mb->wave_bounce;
    }
    switch (b->node_format) {
        case GS_NODES_WIDE4: st = launch_views_f<GS_NODES_WIDE4>(w, threads, stack, s); break;
        case GS_NODES_WIDE4_Q8: st = launch_views_f<GS_NODES_WIDE4_Q8>(w, threads, stack, s); break;
        case GS_NODES_BINARY_Q8: st = launch_views_f<GS_NODES_BINARY_Q8>(w, threads, stack, s); break;
        default: st = launch_views_f<GS_NODES_BINARY>(w, threads, stack, s); break;
    }
    if (st != GS_OK) return st;
    if (slots > 0) {
        gs_bvh *mb = const_cast<gs_bvh *>(b);
        const int cur = sort_keys64(mb->wave_codes, slots, 32, mb->wave_hist, mb->wave_scan, s);
        const unsigned long long *sorted = mb->wave_codes[cur];
        switch (b->node_format) {
            case GS_NODES_WIDE4:
                st = launch_bounce_f<GS_NODES_WIDE4>(w, sorted, slots, threads, stack, s);
                break;
            case GS_NODES_WIDE4_Q8:
                st = launch_bounce_f<GS_NODES_WIDE4_Q8>(w, sorted, slots, threads, stack, s);
                break;
            default: st = launch_bounce_f<GS_NODES_BINARY>(w, sorted, slots, threads, stack, s); break;
        }
        if (st != GS_OK) return st;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "render launch");
    return GS_OK;
}

}  // namespace gsrt
