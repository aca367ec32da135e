// trace.cu -- stochastic ray tracing of transparent Gaussians on sm_103a.
//
// One warp per tile of pixels. A lane carries S consecutive samples of its
// pixel (the launch's passes have N * S slots, see launch_trace); the 32
// lanes are split into pixels x lanes: the L lanes of one pixel trace passes
// sub, sub + L, ... of the same camera ray (L the largest power of two not
// above the passes, at most 32), so they share their ray and differ only in
// the random draws and the clips they cause; with one pass per pixel the
// tile is 8x4 pixels. With 8 or more lanes on a pixel the group walks the
// L-wide copy together (traverse_group), otherwise the warp traverses as a
// packet (traverse_packet). Each pass is one traversal of the hierarchy
// (Sec. 3.2) keeping its closest accepted intersections (Sec. 3.5). At every
// leaf the intersection routine of Alg. 1 runs:
//   t    mean of the 1D Gaussian along the ray (Sec. 3.1)
//   cull if t <= t_min or t is not before the slot's hit, or if the mean
//        lies outside the bounding ellipsoid (Eq. 2: q > s^2 = 8)
//   alpha = opacity * exp(-q/2), q the minimum of the Mahalanobis form
//   accept iff xi < alpha (Eq. 4, Fig. 2), replacing the slot (Eq. 6) and
//        clipping the traversal range to the farthest slot.
// After the traversal each slot is shaded once (SH colour, Sec. 3.2) or gets
// the background, and the pixel accumulates the mean of Eq. 7. On request
// every sample's slot {tc, tau, id} is also stored, [pixel][sample], for a
// gradient launch that reads it instead of tracing again.
//
// Float32 formulation of the 1D Gaussian. With o the ray origin, d the unit
// direction, mu the mean and M = S^-1 R_q^T:
//   o - mu = h + l exactly (h rounded, l its rounding error),
//   tc = -(h . d) puts the base point P = o + tc d near the mean,
//   w = P - mu = fma(tc, d, h) + l is accurate to the rounding of its own
//       (small) magnitude, whatever rounding tc carries, because q does not
//       depend on which point of the ray is used as base,
//   tau = -(Mw . Md) / |Md|^2 is the 1D mean relative to P,
//   w2 = w + tau d, q = |M w2|^2 - (M w2 . Md)^2 / |Md|^2.
// The depth is t = tc + tau; depths are compared through (tc, tau) pairs so
// that two nearby hits are ordered to the accuracy of tau, not of t.
#include <cuda_runtime.h>
#include <math.h>

#include "trace_common.cuh"

namespace gsrt {
namespace {

// Template values of FMT for the cooperative traversal of the W-wide records
// by groups of W = 8, 16, 32 lanes on one pixel: kFmtGroup + log2 W for the
// FP32 records, kFmtGroupQ8 + log2 W for the 8-bit ones; the others are
// GS_NODES_*.
constexpr int kFmtGroup = 8;
constexpr int kFmtGroupQ8 = 16;
__host__ __device__ constexpr bool is_group_fmt(int f) { return f >= kFmtGroup + 3; }
__host__ __device__ constexpr bool is_group_q8(int f) { return f >= kFmtGroupQ8 + 3; }

// Persistent kernel: each warp repeatedly takes the next tile (one atomic
// per tile, so the tail of the launch stays balanced), then runs all passes
// of its pixels. The grouped form is latency-bound and is built for eight
// resident blocks per SM with one or two slots per lane (64 registers),
// seven with four (72: fewer spills of the four slots), five with eight;
// the per-lane packet form for eight with up to four slots (against five:
// spp 1 4.77 -> 4.31 ms, spp 16 with four slots 16.9 -> 15.9 ms) and six
// with eight (85 registers; against one, four, five and eight blocks:
// spp 16 with eight slots 14.8, 13.3, 12.4, 11.7 and 12.1 ms).
constexpr int group_min_blocks(int n) { return n >= 8 ? 5 : (n >= 4 ? 7 : kGroupMinBlocks); }

template <int N, bool COUNT, int FMT>
__global__ void __launch_bounds__(kThreads, is_group_fmt(FMT) ? group_min_blocks(N)
                                                               : (N >= 8 ? 6 : 8))
    k_trace(const TraceArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t kAll = 0xffffffffu;
    const int lg = a.lpp_log2, L = 1 << lg;
    const int tw_lg = tile_w_log2(lg), th_lg = 5 - lg - tw_lg;
    const int sub = lane & (L - 1), pl = lane >> lg;
    const uint32_t tiles_x = (uint32_t)((a.width + (1 << tw_lg) - 1) >> tw_lg);
    const uint32_t tiles_y = (uint32_t)((a.height + (1 << th_lg) - 1) >> th_lg);
    const uint32_t n_tiles = tiles_x * tiles_y;
    const int64_t npix = (int64_t)a.width * a.height;
    uint32_t stack[kMaxStack];
    float stack_t[kMaxStack];
    uint32_t err = 0;
    Counts cnt;
    unsigned long long n_shaded = 0, n_rays = 0;
    // group stacks: each warp's pool split evenly among its groups
    constexpr bool grouped = is_group_fmt(FMT);
    constexpr int LG = grouped ? (FMT & 7) : 3;
    __shared__ uint32_t s_ref[grouped ? kThreads / 32 : 1][grouped ? kGroupPool : 1];
    __shared__ float s_t[grouped ? kThreads / 32 : 1][grouped ? kGroupPool : 1];
    const int grp_off = grouped ? (lane >> LG) * (kGroupPool >> (5 - LG)) : 0;
    uint32_t *grp_ref = s_ref[grouped ? threadIdx.x >> 5 : 0] + grp_off;
    float *grp_t = s_t[grouped ? threadIdx.x >> 5 : 0] + grp_off;
    for (;;) {
        uint32_t tile = 0;
        if (lane == 0) tile = atomicAdd(a.work, 1u);
        tile = __shfl_sync(kAll, tile, 0);
        if (tile >= n_tiles) break;
        const int x = (int)(((tile % tiles_x) << tw_lg) + (pl & ((1 << tw_lg) - 1)));
        const int y = (int)(((tile / tiles_x) << th_lg) + (pl >> tw_lg));
        const bool valid = x < a.width && y < a.height;
        const int64_t pix = valid ? (int64_t)y * a.width + x : 0;
        Ray<N> r;
        {
            float d[3];
            camera_ray(a, valid ? x : 0, valid ? y : 0, d);
            set_ray(r, a.eye, d);
        }
        r.ray_id = a.ray_id_offset + (uint32_t)pix;
        r.stream_tag = a.stream_tag;
        r.t_min = a.t_min;
        r.t_max = a.t_max;
        r.any_hit = false;
        float acc[3] = {0.0f, 0.0f, 0.0f};
        const int n_rounds = (a.spp + L - 1) >> lg;
        for (int j = 0; j < n_rounds; ++j) {
            const int pass = (j << lg) + sub;
            const bool live = valid && pass < a.spp;
            const int s0 = pass * N;
            // an unused slot (sample index beyond the pixel's count) sits
            // at -inf: no candidate is closer, and it never sets the clip
#pragma unroll
            for (int k = 0; k < N; ++k)
                r.slot[k] = s0 + k < a.n_samples ? Slot{INFINITY, 0.0f, 0xffffffffu}
                                                 : Slot{-INFINITY, 0.0f, 0xffffffffu};
            update_clip(r, a.t_max);
            if (!live) r.t_far = -INFINITY;  // lanes off the image never hit
            if (a.n_nodes > 0) {
                if constexpr (grouped)
                    traverse_group<N, COUNT, LG, true, is_group_q8(FMT)>(a, r, pass, grp_ref,
                                                                          grp_t, err, cnt);
                else if constexpr (FMT == GS_NODES_BINARY)
                    traverse_packet<N, COUNT>(a, r, pass, stack, stack_t, err, cnt);
                else
                    traverse_packet_wide<N, COUNT, FMT>(a, r, pass, stack, stack_t, err, cnt);
            }
            if (live) {
                // shade each slot once (Eq. 6) and accumulate (Eq. 7)
                float Y[16];
                sh_basis(a.sh_degree, r.d, Y);
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (s0 + k >= a.n_samples) continue;
                    float c[3];
                    if (r.slot[k].gid != 0xffffffffu) {
                        sh_colour(a, r.slot[k].gid, Y, c);
                        if (COUNT) ++n_shaded;
                    } else {
                        c[0] = a.bg[0]; c[1] = a.bg[1]; c[2] = a.bg[2];
                    }
                    acc[0] += c[0];
                    acc[1] += c[1];
                    acc[2] += c[2];
                    if (a.hit_id) {
                        const int64_t o = ((int64_t)s0 + k) * npix + pix;
                        a.hit_id[o] = r.slot[k].gid == 0xffffffffu ? -1 : (int32_t)r.slot[k].gid;
                        a.hit_t[o] = r.slot[k].t();
                    }
                }
                if (a.keys) {
                    gs_sample_key *key = a.keys + pix * a.n_samples + s0;
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        if (s0 + k >= a.n_samples) continue;
                        key[k].tc = r.slot[k].tc;
                        key[k].tau = r.slot[k].tau;
                        key[k].gid = r.slot[k].gid;
                    }
                }
            }
            __syncwarp();
        }
        // the pixel's lanes add their partial sums (Eq. 7)
        for (int o = L >> 1; o >= 1; o >>= 1) {
            acc[0] += __shfl_xor_sync(kAll, acc[0], o);
            acc[1] += __shfl_xor_sync(kAll, acc[1], o);
            acc[2] += __shfl_xor_sync(kAll, acc[2], o);
        }
        if (valid && sub == 0) {
            const float inv_n = 1.0f / (float)a.n_samples;
            a.rgb[3 * pix + 0] = acc[0] * inv_n;
            a.rgb[3 * pix + 1] = acc[1] * inv_n;
            a.rgb[3 * pix + 2] = acc[2] * inv_n;
            if (COUNT) ++n_rays;
        }
    }
    if (err) atomicOr(a.status, err);
    if (COUNT) {
        atomicAdd(a.counters + 0, cnt.nodes);
        atomicAdd(a.counters + 1, cnt.prims);
        atomicAdd(a.counters + 2, cnt.draws);
        atomicAdd(a.counters + 3, n_rays);
        atomicAdd(a.counters + 4, n_shaded);
        atomicAdd(a.counters + 5, cnt.node_fetch);
        atomicAdd(a.counters + 6, cnt.prim_fetch);
    }
}

template <int N, int FMT>
gs_status launch_nf(const TraceArgs &a, bool count, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = count ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace<N, true, FMT>, kThreads, 0)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_trace<N, false, FMT>, kThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "trace launch setup");
    // one resident grid; warps take tiles until none is left
    const int tw_lg = tile_w_log2(a.lpp_log2), th_lg = 5 - a.lpp_log2 - tw_lg;
    const uint32_t tiles = (uint32_t)(((a.width + (1 << tw_lg) - 1) >> tw_lg) *
                                      ((a.height + (1 << th_lg) - 1) >> th_lg));
    const uint32_t warps_needed = tiles;
    uint32_t blocks = (uint32_t)sms * (uint32_t)(per > 0 ? per : 1);
    const uint32_t max_blocks = (warps_needed + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    if ((e = cudaMemsetAsync(a.work, 0, sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "reset work counter");
    if (count) k_trace<N, true, FMT><<<blocks, kThreads, 0, s>>>(a);
    else k_trace<N, false, FMT><<<blocks, kThreads, 0, s>>>(a);
    return GS_OK;
}

template <int N>
gs_status launch_n(const TraceArgs &a, int format, bool count, cudaStream_t s) {
    // groups of 8 or more lanes on one pixel take the cooperative form
    if (format == GS_NODES_BINARY && a.grec != nullptr) {
        if (a.lpp_log2 == 5) return launch_nf<N, kFmtGroup + 5>(a, count, s);
        if (a.lpp_log2 == 4) return launch_nf<N, kFmtGroup + 4>(a, count, s);
        if (a.lpp_log2 == 3) return launch_nf<N, kFmtGroup + 3>(a, count, s);
    }
    if (format == GS_NODES_BINARY_Q8 && a.grec != nullptr) {
        if (a.lpp_log2 == 5) return launch_nf<N, kFmtGroupQ8 + 5>(a, count, s);
        if (a.lpp_log2 == 4) return launch_nf<N, kFmtGroupQ8 + 4>(a, count, s);
        if (a.lpp_log2 == 3) return launch_nf<N, kFmtGroupQ8 + 3>(a, count, s);
    }
    switch (format) {
        case GS_NODES_WIDE4: return launch_nf<N, GS_NODES_WIDE4>(a, count, s);
        case GS_NODES_WIDE4_Q8: return launch_nf<N, GS_NODES_WIDE4_Q8>(a, count, s);
        default: return launch_nf<N, GS_NODES_BINARY>(a, count, s);
    }
}

// Samples one lane carries when the caller leaves the choice to the
// library (samples_per_lane = 0). The time follows the number of walks a
// pixel needs and grows slowly with the slots a walk carries. Measured on
// the 1M-Gaussian shell at 1080p, trace ms for K = n_hits * S slots per
// lane and T = spp * n_hits samples per pixel (one sample per lane first):
//   T = 4:   K 1 14.1, 2 7.6, 4 5.4 (per-lane packets)
//   T = 8:   K 1 20.1, 4 8.8, 8 7.1
//   T = 16:  K 1 24.2, 4 15.9, 8 11.7
//   T = 32:  K 1 27.5, 2 27.0, 4 25.5 (8 lanes a pixel, grouped), 8 21.0
//   T = 64:  K 1 52.3, 2 30.4 (32 lanes, grouped), 4 30.5, 8 38.5
//   T = 128: K 2 59.8, 4 34.4, 8 46.4;  T = 256: K 4 67.5, 8 52.5
// K is never below n_hits.
int auto_samples_per_lane(int spp, int n_hits, int node_format) {
    (void)node_format;
    const int64_t T = (int64_t)spp * n_hits;
    int K;
    if (T <= 2) K = (int)T;
    else if (T < 8) K = 4;
    else if (T < 64) K = 8;
    else if (T < 128) K = 2;
    else if (T < 256) K = 4;
    else K = 8;
    if (K < n_hits) K = n_hits;
    return K / n_hits;
}

}  // namespace

void trace_layout(const gs_bvh *b, const gs_trace_params *p, int *S_out, int *spp_eff_out,
                  int *lpp_log2_out, bool *grouped_out) {
    // A lane carries S consecutive samples: the launch runs ceil(spp / S)
    // passes of n_hits * S slots; sample s = pass * n_hits * S + k either way.
    int S = p->samples_per_lane > 0 ? p->samples_per_lane
                                    : auto_samples_per_lane(p->spp, p->n_hits, b->node_format);
    while (S > 1 && S > p->spp) S >>= 1;
    *S_out = S;
    *spp_eff_out = (p->spp + S - 1) / S;
    *lpp_log2_out = lanes_per_pixel_log2(*spp_eff_out);
    *grouped_out = (b->node_format == GS_NODES_BINARY || b->node_format == GS_NODES_BINARY_Q8) &&
                   b->node_depth && *lpp_log2_out >= 3;
}

gs_status launch_trace(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                       const gs_trace_params *p, float *rgb, int32_t *hit_id, float *hit_t,
                       gs_sample_key *keys, cudaStream_t s) {
    int S = 1, spp_eff = 1, lpp_log2 = 0;
    bool grouped = false;
    trace_layout(b, p, &S, &spp_eff, &lpp_log2, &grouped);
    const int n_eff = p->n_hits * S;
    TraceArgs a;
    a.nodes = b->nodes;
    a.wide = b->wide;
    a.lpp_log2 = lpp_log2;
    if (b->node_depth && a.lpp_log2 >= 3) {
        a.grec = b->group[a.lpp_log2 - 3].rec;
        a.gcnt = b->group[a.lpp_log2 - 3].cnt;
    } else {
        a.grec = nullptr;
        a.gcnt = nullptr;
    }
    a.gq8 = b->node_format == GS_NODES_BINARY_Q8;
    a.prims = b->prims;
    a.sh = g->sh;
    a.n_nodes = b->n_nodes;
    a.sh_degree = g->sh_degree;
    a.sh_dtype = g->sh_dtype;
    a.width = cam->width;
    a.height = cam->height;
    a.ray_id_offset = cam->ray_id_offset;
    for (int i = 0; i < 3; ++i) {
        a.eye[i] = cam->eye[i];
        a.look_at[i] = cam->look_at[i];
        a.up[i] = cam->up[i];
        a.bg[i] = p->bg[i];
    }
    a.tan_half = (float)tan((double)cam->fov_y_deg * 3.14159265358979323846 / 360.0);
    a.key0 = (uint32_t)(p->seed & 0xffffffffu);
    a.key1 = (uint32_t)(p->seed >> 32);
    philox_round_keys(a.key0, a.key1, a.rk);
    a.stream_tag = p->stream_tag;
    a.spp = spp_eff;
    a.n_samples = p->spp * p->n_hits;
    a.t_min = p->t_min;
    a.t_max = p->t_max;
    a.stack_depth = p->stack_depth == 0 ? kMaxStack : p->stack_depth;
    // a valid traversal visits every internal node at most once per pass
    a.step_limit = (uint32_t)(b->n_nodes + 8 < (int64_t)kStepLimit ? b->n_nodes + 8 : kStepLimit);
    a.rgb = rgb;
    a.hit_id = hit_id;
    a.hit_t = hit_t;
    a.keys = keys;
    a.n_gauss = (uint32_t)b->M;
    a.counters = p->counters;
    a.status = b->status;
    a.work = b->status + 1;
    a.depth_mode = p->depth_mode;
    a.rng_mode = p->rng_mode;
    {
        // camera forward axis, float32 normalise as for the camera rays
        float f[3];
        for (int i = 0; i < 3; ++i) f[i] = cam->look_at[i] - cam->eye[i];
        float n2 = f[0] * f[0];
        n2 = n2 + f[1] * f[1];
        n2 = n2 + f[2] * f[2];
        const float n = sqrtf(n2);
        for (int i = 0; i < 3; ++i) a.fwd[i] = f[i] / n;
    }
    const bool count = p->counters != nullptr;
    gs_status st;
    switch (n_eff) {
        case 1: st = launch_n<1>(a, b->node_format, count, s); break;
        case 2: st = launch_n<2>(a, b->node_format, count, s); break;
        case 4: st = launch_n<4>(a, b->node_format, count, s); break;
        case 8: st = launch_n<8>(a, b->node_format, count, s); break;
        default: return fail(GS_ERR_INVALID_ARG, "n_hits must be 1, 2, 4 or 8");
    }
    if (st != GS_OK) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "trace launch");
    return GS_OK;
}

}  // namespace gsrt
