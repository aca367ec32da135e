// backward.cu -- unbiased stochastic gradients of an image loss (the
// differentiable-rendering extension the paper names in Sec. 6).
//
// For one sample whose closest accepted hit is k (colour c_k, or the
// background when nothing was accepted), with g = dLoss/dpixel / S:
//   dc_k          += g                      (colour of the selected hit)
//   dalpha_i      += g . (c_i - c_k) / (1 - alpha_i)
//                    for every valid Gaussian i in front of k in (t, id)
//                    order; those are exactly the ones the sample rejected.
// Both are unbiased for the gradient of the sorted blend of Eq. 3, whose
// dL/dalpha_i = T_i (c_i - B_i) and dL/dc_i = T_i alpha_i. Order swaps and
// the ellipsoid cutoff are not differentiated.
//
// Each pass takes its samples' winners either from the payloads the
// rendering stored (gs_trace_backward_keys) or by running the forward
// traversal again with the same Philox keys (identical winners); then a
// traversal clipped at the winners' depths enumerates the Gaussians in
// front of them. Gradients are accumulated with atomics: in
// the per-lane form reduced across the warp for the warp's shared leaf; in
// the grouped form (8 or more lanes on one pixel, the wide copy of that
// width) the chain rule runs once per Gaussian and group on the lanes'
// summed weights, and lanes whose slot holds the same Gaussian add its
// colour gradient once.
#include <cuda_runtime.h>
#include <math.h>

#include "trace_common.cuh"

namespace gsrt {
namespace {

// One candidate evaluated without acceptance, by the same formulas as
// intersect(): base point, 1D mean, and the local coordinates of the point
// on the ray at the mean.
// With RELOAD (the grouped enumeration) M and the opacity are not kept:
// grad_alpha re-reads them from the record (L1 still holds it), so fewer
// values stay live while the group sums the candidate's weight (spp 16
// 45.8 -> 43.4 ms, spp 64 60.7 -> 56.3); the per-lane form keeps them
// (re-reading cost it 6-20%).
struct Cand {
    float t, tc, tau, q, alpha, opacity;
    float v[3];  // x* - mu, world
    float u[3];  // M v = S^-1 R_q^T v
    float m[9];
    uint32_t idx;  // the Gaussian record
    uint32_t gid;
    bool valid;
};

template <bool RELOAD>
__device__ __forceinline__ Cand eval_cand(const TraceArgs &a, const float o[3], const float d[3],
                                          uint32_t idx) {
    Cand c;
    const float4 *pp = reinterpret_cast<const float4 *>(a.prims + idx);
    const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1), p2 = __ldg(pp + 2), p3 = __ldg(pp + 3);
    const float mu[3] = {p0.x, p0.y, p0.z};
    const float m[9] = {p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w, p3.x};
    c.gid = __float_as_uint(p3.y);
    c.idx = idx;
    if constexpr (!RELOAD) {
        c.opacity = p0.w;
#pragma unroll
        for (int i = 0; i < 9; ++i) c.m[i] = m[i];
    }
    float h[3], l[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float s = o[i] - mu[i];
        const float bp = s - o[i];
        const float ap = s - bp;
        l[i] = (o[i] - ap) + (-mu[i] - bp);
        h[i] = s;
    }
    const float tc = -fmaf(h[0], d[0], fmaf(h[1], d[1], h[2] * d[2]));
    float w[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) w[i] = fmaf(tc, d[i], h[i]) + l[i];
    float md[3], mw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        md[i] = fmaf(m[3 * i], d[0], fmaf(m[3 * i + 1], d[1], m[3 * i + 2] * d[2]));
        mw[i] = fmaf(m[3 * i], w[0], fmaf(m[3 * i + 1], w[1], m[3 * i + 2] * w[2]));
    }
    const float dd = fmaf(md[0], md[0], fmaf(md[1], md[1], md[2] * md[2]));
    const float wd = fmaf(mw[0], md[0], fmaf(mw[1], md[1], mw[2] * md[2]));
    const float inv_dd = 1.0f / dd;
    const float tau = -wd * inv_dd;
    const float t = tc + tau;
    float w2[3], mw2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) w2[i] = fmaf(tau, d[i], w[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        mw2[i] = fmaf(m[3 * i], w2[0], fmaf(m[3 * i + 1], w2[1], m[3 * i + 2] * w2[2]));
    const float ww = fmaf(mw2[0], mw2[0], fmaf(mw2[1], mw2[1], mw2[2] * mw2[2]));
    const float wd2 = fmaf(mw2[0], md[0], fmaf(mw2[1], md[1], mw2[2] * md[2]));
    const float q = fmaxf(ww - wd2 * wd2 * inv_dd, 0.0f);
    c.t = t;
    c.tc = tc;
    c.tau = tau;
    c.q = q;
    c.alpha = p0.w * expf(-0.5f * q);
    for (int i = 0; i < 3; ++i) {
        c.v[i] = w2[i];
        c.u[i] = mw2[i];
    }
    c.valid = (t > a.t_min) && (t < a.t_max) && (q <= kS2);
    return c;
}

// d alpha / d(mu, log s, quat, logit) of one candidate; alpha = o exp(-q/2),
// q = |u|^2 with u = S^-1 R_q^T v, and t held at the 1D mean (dq/dt = 0).
template <bool RELOAD>
__device__ void grad_alpha(const TraceArgs &a, const Cand &c, float out[11]) {
    float m[9], opacity;
    if constexpr (RELOAD) {
        const float4 *pp = reinterpret_cast<const float4 *>(a.prims + c.idx);
        const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1), p2 = __ldg(pp + 2), p3 = __ldg(pp + 3);
        m[0] = p1.x; m[1] = p1.y; m[2] = p1.z; m[3] = p1.w;
        m[4] = p2.x; m[5] = p2.y; m[6] = p2.z; m[7] = p2.w; m[8] = p3.x;
        opacity = p0.w;
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) m[i] = c.m[i];
        opacity = c.opacity;
    }
    const float dadq = -0.5f * c.alpha;
    // mean: dq/dmu = -2 M^T u
#pragma unroll
    for (int j = 0; j < 3; ++j)
        out[j] = dadq * -2.0f * fmaf(m[j], c.u[0], fmaf(m[3 + j], c.u[1], m[6 + j] * c.u[2]));
    // log-scales: dq/dlog s_k = -2 u_k^2
    float inv_s[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        out[3 + k] = dadq * -2.0f * c.u[k] * c.u[k];
        inv_s[k] = expf(-__ldg(a.log_scales + 3 * (int64_t)c.gid + k));
    }
    // rotation: dq/dR_jk = 2 v_j u_k / s_k, then R(q) and the normalisation
    float dR[9];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) dR[3 * j + k] = 2.0f * c.v[j] * c.u[k] * inv_s[k];
    const float4 qr = __ldg(reinterpret_cast<const float4 *>(a.quats) + c.gid);
    const float n = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float w = qr.x / n, x = qr.y / n, y = qr.z / n, z = qr.w / n;
    const float Dw[9] = {0.0f, -2 * z, 2 * y, 2 * z, 0.0f, -2 * x, -2 * y, 2 * x, 0.0f};
    const float Dx[9] = {0.0f, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x};
    const float Dy[9] = {-4 * y, 2 * x, 2 * w, 2 * x, 0.0f, 2 * z, -2 * w, 2 * z, -4 * y};
    const float Dz[9] = {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0.0f};
    float gq[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int e = 0; e < 9; ++e) {
        gq[0] = fmaf(dR[e], Dw[e], gq[0]);
        gq[1] = fmaf(dR[e], Dx[e], gq[1]);
        gq[2] = fmaf(dR[e], Dy[e], gq[2]);
        gq[3] = fmaf(dR[e], Dz[e], gq[3]);
    }
    const float qh[4] = {w, x, y, z};
    const float dot = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * z;
#pragma unroll
    for (int k = 0; k < 4; ++k) out[6 + k] = dadq * (gq[k] - dot * qh[k]) / n;
    out[10] = c.alpha * (1.0f - opacity);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Gradient of the leaf shared by the warp (same Gaussian for every lane
// that reaches it): each lane forms its contribution, the warp sums them,
// one lane adds the sums.
template <int N>
__device__ __forceinline__ void leaf_gradient(const TraceArgs &a, const Ray<N> &r, bool hit,
                                              uint32_t idx, const float ck[N][3], const float g[3],
                                              const float Y[16]) {
    const uint32_t kAll = 0xffffffffu;
    float contrib[11];
#pragma unroll
    for (int j = 0; j < 11; ++j) contrib[j] = 0.0f;
    uint32_t gid = 0;
    bool nz = false;
    if (hit) {
        const Cand c = eval_cand<false>(a, r.o, r.d, idx);
        gid = c.gid;
        if (c.valid) {
            float coef = 0.0f;
            bool any = false;
            float ci[3];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                if (!lex_closer(c.tc, c.tau, c.gid, r.slot[k])) continue;
                if (!any) {
                    sh_colour(a, c.gid, Y, ci);
                    any = true;
                }
                coef += g[0] * (ci[0] - ck[k][0]) + g[1] * (ci[1] - ck[k][1]) +
                        g[2] * (ci[2] - ck[k][2]);
            }
            if (any && coef != 0.0f) {
                // a rejected hit has alpha <= xi < 1
                coef /= (1.0f - c.alpha);
                grad_alpha<false>(a, c, contrib);
#pragma unroll
                for (int j = 0; j < 11; ++j) contrib[j] *= coef;
                nz = true;
            }
        }
    }
    const unsigned m = __ballot_sync(kAll, nz);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    gid = __shfl_sync(kAll, gid, leader);
    float sum[11];
#pragma unroll
    for (int j = 0; j < 11; ++j) sum[j] = warp_sum(contrib[j]);
    if ((int)(threadIdx.x & 31) == leader) {
        const int64_t gg = gid;
        for (int k = 0; k < 3; ++k) {
            atomicAdd(a.g_means + 3 * gg + k, sum[k]);
            atomicAdd(a.g_log_scales + 3 * gg + k, sum[3 + k]);
        }
        for (int k = 0; k < 4; ++k) atomicAdd(a.g_quats + 4 * gg + k, sum[6 + k]);
        atomicAdd(a.g_logits + gg, sum[10]);
    }
}

// Second traversal of a pass: every leaf the lane's ray reaches before its
// farthest slot (no acceptance, no clipping), in packet order.
template <int N>
__device__ void enumerate_packet(const TraceArgs &a, const Ray<N> &r, const float ck[N][3],
                                 const float g[3], const float Y[16], uint32_t *stack,
                                 float *stack_t, uint32_t &err) {
    const uint32_t kAll = 0xffffffffu;
    int sp = 0;
    uint32_t node = 0, steps = 0;
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
        }
        const float4 *np = reinterpret_cast<const float4 *>(a.nodes + node);
        const float4 b0 = __ldg(np), b1 = __ldg(np + 1), b2 = __ldg(np + 2);
        const uint4 cref = __ldg(reinterpret_cast<const uint4 *>(np + 3));
        const float boxL[6] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y};
        const float boxR[6] = {b1.z, b1.w, b2.x, b2.y, b2.z, b2.w};
        float tL, tR;
        bool hL = slab(boxL, r.inv, r.oinv, a.t_min, r.t_far, tL);
        bool hR = slab(boxR, r.inv, r.oinv, a.t_min, r.t_far, tR);
        if (cref.x & kLeafBit) {
            leaf_gradient<N>(a, r, hL, cref.x & ~kLeafBit, ck, g, Y);
            hL = false;
        }
        if (cref.y & kLeafBit) {
            leaf_gradient<N>(a, r, hR, cref.y & ~kLeafBit, ck, g, Y);
            hR = false;
        }
        const unsigned mL = __ballot_sync(kAll, hL), mR = __ballot_sync(kAll, hR);
        if (mL && mR) {
            const unsigned lf = __ballot_sync(kAll, hL && (!hR || tL <= tR));
            const bool left_first = 2 * __popc(lf) >= __popc(mL | mR);
            if (sp >= a.stack_depth) {
                err |= kErrStack;
                break;
            }
            stack[sp] = left_first ? cref.y : cref.x;
            stack_t[sp] = left_first ? (hR ? tR : INFINITY) : (hL ? tL : INFINITY);
            ++sp;
            node = left_first ? cref.x : cref.y;
            continue;
        }
        if (mL) { node = cref.x; continue; }
        if (mR) { node = cref.y; continue; }
        bool found = false;
        while (sp > 0) {
            --sp;
            if (__any_sync(kAll, stack_t[sp] <= r.t_far)) {
                node = stack[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}

// Grouped enumeration (groups of L = 2^LG lanes sharing one ray, the
// W-wide copy with W = L): the same leaves as enumerate_packet for each
// lane, visited once per group. The lane holding a hit leaf evaluates the
// candidate and its colour; every lane adds its own samples' weight
// sum_k g . (c_i - c_k) over the slots the candidate is in front of; the
// group's sum goes back to that lane, which chains it through alpha and
// adds the gradients once for the group.
template <int N, int LG, bool Q8>
__device__ void enumerate_group(const TraceArgs &a, const Ray<N> &r, const float ck[N][3],
                                const float g[3], const float Y[16], uint32_t *s_ref, float *s_t,
                                uint32_t &err) {
    constexpr int L = 1 << LG;
    constexpr int kCap = kGroupPool >> (5 - LG);
    constexpr uint32_t kLaneBits = L == 32 ? 0xffffffffu : ((1u << (L & 31)) - 1u);
    const int lane = threadIdx.x & 31;
    const int base = lane & ~(L - 1);
    const int sub = lane & (L - 1);
    const uint32_t gmask = kLaneBits << base;
    float G = r.t_far >= a.t_min ? r.t_far : -INFINITY;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) G = fmaxf(G, __shfl_xor_sync(gmask, G, o));
    if (!(G >= a.t_min)) return;
    int sp = 0;
    uint32_t node = (__ldg(a.gcnt) - 1u) << kWideCountShift;
    uint32_t steps = 0;
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
        }
        const int n_child = (int)((node >> kWideCountShift) & 31u) + 1;
        uint32_t ref = kEmpty;
        float te = INFINITY;
        bool hit = false;
        if (sub < n_child) hit = group_child<Q8>(a.grec, node, sub, r.inv, r.oinv, a.t_min, G, ref, te);
        const bool leaf = (ref & kLeafBit) != 0u;
        if ((__ballot_sync(gmask, hit && leaf) >> base) & kLaneBits) {
            Cand c;
            float ci[3] = {0.0f, 0.0f, 0.0f};
            bool ok = false;
            if (hit && leaf) {
                c = eval_cand<true>(a, r.o, r.d, ref & ~kLeafBit);
                // in front of some lane's winner only if t <= that lane's clip <= G
                ok = c.valid && c.t <= G;
                if (ok) {
                    if constexpr (N >= 4) {
                        // four or more slots: the basis is recomputed here
                        // instead of being held through the enumeration
                        // (N=4 spp 16 79.0 -> 69.4 ms; with two slots
                        // holding it measured 2% faster)
                        float Yl[16];
                        sh_basis(a.sh_degree, r.d, Yl);
                        sh_colour(a, c.gid, Yl, ci);
                    } else {
                        sh_colour(a, c.gid, Y, ci);
                    }
                }
            }
            float my_coef = 0.0f;
            const bool live = r.t_far >= a.t_min;  // lanes past the last pass add nothing
            for (uint32_t cm = (__ballot_sync(gmask, ok) >> base) & kLaneBits; cm; cm &= cm - 1u) {
                const int src = base + __ffs(cm) - 1;
                const float tc = __shfl_sync(gmask, c.tc, src);
                const float tau = __shfl_sync(gmask, c.tau, src);
                const uint32_t gid = __shfl_sync(gmask, c.gid, src);
                float cc[3];
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) cc[ch] = __shfl_sync(gmask, ci[ch], src);
                float coef = 0.0f;
#pragma unroll
                for (int k = 0; k < N; ++k) {
                    if (!live || !lex_closer(tc, tau, gid, r.slot[k])) continue;
                    coef += g[0] * (cc[0] - ck[k][0]) + g[1] * (cc[1] - ck[k][1]) +
                            g[2] * (cc[2] - ck[k][2]);
                }
#pragma unroll
                for (int o = 1; o < L; o <<= 1) coef += __shfl_xor_sync(gmask, coef, o);
                if (lane == src) my_coef = coef;
            }
            if (ok && my_coef != 0.0f) {
                // a rejected hit has alpha <= xi < 1
                const float w = my_coef / (1.0f - c.alpha);
                float d[11];
                grad_alpha<true>(a, c, d);
                const int64_t gg = c.gid;
                for (int k = 0; k < 3; ++k) {
                    atomicAdd(a.g_means + 3 * gg + k, d[k] * w);
                    atomicAdd(a.g_log_scales + 3 * gg + k, d[3 + k] * w);
                }
                for (int k = 0; k < 4; ++k) atomicAdd(a.g_quats + 4 * gg + k, d[6 + k] * w);
                atomicAdd(a.g_logits + gg, d[10] * w);
            }
        }
        const bool inner = hit && !leaf;
        const uint32_t im = (__ballot_sync(gmask, inner) >> base) & kLaneBits;
        if (im) {
            const uint32_t key = __reduce_min_sync(
                gmask, inner ? ((__float_as_uint(fmaxf(te, 0.0f)) & ~31u) | (uint32_t)sub)
                             : 0xffffffffu);
            const int nj = (int)(key & 31u);
            const uint32_t next = __shfl_sync(gmask, ref, base + nj);
            const uint32_t others = im & ~(1u << nj);
            const int npush = __popc(others);
            if (sp + npush > kCap) {
                err |= kErrStack;
                break;
            }
            __syncwarp(gmask);
            if (inner && sub != nj) {
                const int pos = sp + __popc(others & ((1u << sub) - 1u));
                s_ref[pos] = ref;
                s_t[pos] = te;
            }
            sp += npush;
            __syncwarp(gmask);
            node = next;
            continue;
        }
        if (sp == 0) break;
        --sp;  // no clip changes here: every pushed node is still needed
        node = s_ref[sp];
    }
}

// LG: log2 of the lanes per pixel when the grouped traversals are used, else
// 0. The grouped form is latency-bound and built for eight resident blocks
// per SM with up to two slots per lane, seven with four or more (72
// registers: N=4 spp 16 82.3 -> 79.0 ms; seven blocks cost 5-8% with two
// slots); the per-lane form for five (measured against three: 45.5 vs 48.5
// ms at N=4 spp 4, 10.4 vs 13.1 ms at spp 2; four blocks equal to five).
// KEYS: the winners come from the stored payloads (a.keys), and the
// forward traversal is not compiled in. Its per-lane form is built for six
// blocks per SM (N=4 spp 4: 20.9 ms against 21.2 with five or four); its
// grouped form keeps the re-tracing form's bounds (with two slots, seven
// and six blocks: spp 16 19.9 and 21.6 ms against 19.5).
template <int N, int LG, bool Q8, bool KEYS>
__global__ void __launch_bounds__(kThreads, LG >= 3 ? (N >= 4 ? 7 : kGroupMinBlocks)
                                                    : (KEYS ? 6 : 5))
    k_backward(const TraceArgs a) {
    const int lane = threadIdx.x & 31;
    const uint32_t kAll = 0xffffffffu;
    __shared__ uint32_t s_ref[LG >= 3 ? kThreads / 32 : 1][LG >= 3 ? kGroupPool : 1];
    __shared__ float s_t[LG >= 3 ? kThreads / 32 : 1][LG >= 3 ? kGroupPool : 1];
    const int grp_off = LG >= 3 ? (lane >> LG) * (kGroupPool >> (5 - (LG >= 3 ? LG : 5))) : 0;
    uint32_t *grp_ref = s_ref[LG >= 3 ? threadIdx.x >> 5 : 0] + grp_off;
    float *grp_t = s_t[LG >= 3 ? threadIdx.x >> 5 : 0] + grp_off;
    // pixels x samples per warp as in the forward trace
    const int lg = a.lpp_log2, L = 1 << lg;
    const int tw_lg = tile_w_log2(lg), th_lg = 5 - lg - tw_lg;
    const int sub = lane & (L - 1), pl = lane >> lg;
    const uint32_t tiles_x = (uint32_t)((a.width + (1 << tw_lg) - 1) >> tw_lg);
    const uint32_t tiles_y = (uint32_t)((a.height + (1 << th_lg) - 1) >> th_lg);
    const uint32_t n_tiles = tiles_x * tiles_y;
    const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
    uint32_t stack[kMaxStack];
    float stack_t[kMaxStack];
    uint32_t err = 0;
    Counts cnt;
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
        const float inv_s = 1.0f / (float)a.n_samples;
        float g[3] = {0.0f, 0.0f, 0.0f};
        if (valid)
            for (int ch = 0; ch < 3; ++ch) g[ch] = a.d_rgb[3 * pix + ch] * inv_s;
        const int n_rounds = (a.spp + L - 1) >> lg;
        for (int j = 0; j < n_rounds; ++j) {
            const int pass = (j << lg) + sub;
            const bool live = valid && pass < a.spp;
            // unused slots (sample index past the pixel's count) at -inf:
            // nothing is in front of them and they never set the clip
#pragma unroll
            for (int k = 0; k < N; ++k)
                r.slot[k] = pass * N + k < a.n_samples ? Slot{INFINITY, 0.0f, 0xffffffffu}
                                                       : Slot{-INFINITY, 0.0f, 0xffffffffu};
            update_clip(r, a.t_max);
            if (!live) r.t_far = -INFINITY;
            if (a.n_nodes == 0) continue;
            // 1) the winners: the rendering's stored payloads, or the forward
            // traversal again with the same keys (same winners)
            if constexpr (KEYS) {
                if (live) {
                    const gs_sample_key *kp = a.keys + pix * a.n_samples + pass * N;
#pragma unroll
                    for (int k = 0; k < N; ++k) {
                        if (pass * N + k >= a.n_samples) continue;
                        const float tc = __ldg(&kp[k].tc), tau = __ldg(&kp[k].tau);
                        const uint32_t gid = __ldg(&kp[k].gid);
                        if (gid == 0xffffffffu || gid < a.n_gauss) {
                            r.slot[k] = Slot{tc, tau, gid};
                        } else {
                            err |= kErrKeys;  // names no Gaussian: no hit
                        }
                    }
                }
            } else if constexpr (LG >= 3) {
                traverse_group<N, false, LG, false, Q8>(a, r, pass, grp_ref, grp_t, err, cnt);
            } else {
                traverse_packet<N, false>(a, r, pass, stack, stack_t, err, cnt);
            }
            // the SH basis of the pixel's direction, formed per pass so that it
            // need not stay live between passes
            float Y[16];
            sh_basis(a.sh_degree, r.d, Y);
            // 2) colours of the winners; dLoss/dk of the selected Gaussians
            float ck[N][3];
#pragma unroll
            for (int k = 0; k < N; ++k) {
                const uint32_t wid = live ? r.slot[k].gid : 0xffffffffu;
                float mult = 1.0f;
                bool leader = true;
                if constexpr (LG >= 3) {
                    // lanes of a pixel share g and Y: one lane adds for all
                    // lanes whose slot k holds the same Gaussian
                    constexpr uint32_t kBits = LG == 5 ? 0xffffffffu : ((1u << ((1 << LG) & 31)) - 1u);
                    const uint32_t gm = kBits << (lane & ~((1 << LG) - 1));
                    const uint32_t same = __match_any_sync(gm, wid);
                    mult = (float)__popc(same);
                    leader = (__ffs(same) - 1) == lane;
                }
                if (wid != 0xffffffffu) {
                    float raw[3];
                    sh_colour_raw(a, wid, Y, raw);
                    const int64_t base = (int64_t)wid * K * 3;
                    for (int ch = 0; ch < 3; ++ch) {
                        ck[k][ch] = fmaxf(raw[ch], 0.0f);
                        if (leader && raw[ch] > 0.0f && g[ch] != 0.0f)
                            for (int i = 0; i < K; ++i)
                                atomicAdd(a.g_sh + base + 3 * i + ch, mult * g[ch] * Y[i]);
                    }
                } else {
                    for (int ch = 0; ch < 3; ++ch) ck[k][ch] = a.bg[ch];
                }
            }
            // 3) every Gaussian in front of a winner
            update_clip(r, a.t_max);
            if (!live) r.t_far = -INFINITY;
            if constexpr (LG >= 3)
                enumerate_group<N, LG, Q8>(a, r, ck, g, Y, grp_ref, grp_t, err);
            else
                enumerate_packet<N>(a, r, ck, g, Y, stack, stack_t, err);
            __syncwarp();
        }
    }
    if (err) atomicOr(a.status, err);
}

template <int N, int LG, bool Q8, bool KEYS>
gs_status launch_backward_nl(const TraceArgs &a, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_backward<N, LG, Q8, KEYS>,
                                                          kThreads, 0);
    if (e != cudaSuccess) return cuda_fail(e, "backward launch setup");
    const int tw_lg = tile_w_log2(a.lpp_log2), th_lg = 5 - a.lpp_log2 - tw_lg;
    const uint32_t tiles = (uint32_t)(((a.width + (1 << tw_lg) - 1) >> tw_lg) *
                                      ((a.height + (1 << th_lg) - 1) >> th_lg));
    uint32_t blocks = (uint32_t)sms * (uint32_t)(per > 0 ? per : 1);
    const uint32_t max_blocks = (tiles + kThreads / 32 - 1) / (kThreads / 32);
    if (blocks > max_blocks) blocks = max_blocks;
    if ((e = cudaMemsetAsync(a.work, 0, sizeof(uint32_t), s)) != cudaSuccess)
        return cuda_fail(e, "reset work counter");
    k_backward<N, LG, Q8, KEYS><<<blocks, kThreads, 0, s>>>(a);
    return GS_OK;
}

// Groups of 8 or more lanes on one pixel use the wide copy of their width.
template <int N, bool KEYS>
gs_status launch_backward_nk(const TraceArgs &a, cudaStream_t s) {
    if (a.grec != nullptr && a.gq8) {
        switch (a.lpp_log2) {
            case 5: return launch_backward_nl<N, 5, true, KEYS>(a, s);
            case 4: return launch_backward_nl<N, 4, true, KEYS>(a, s);
            case 3: return launch_backward_nl<N, 3, true, KEYS>(a, s);
            default: break;
        }
    } else if (a.grec != nullptr) {
        switch (a.lpp_log2) {
            case 5: return launch_backward_nl<N, 5, false, KEYS>(a, s);
            case 4: return launch_backward_nl<N, 4, false, KEYS>(a, s);
            case 3: return launch_backward_nl<N, 3, false, KEYS>(a, s);
            default: break;
        }
    }
    return launch_backward_nl<N, 0, false, KEYS>(a, s);
}

template <int N>
gs_status launch_backward_n(const TraceArgs &a, cudaStream_t s) {
    return a.keys ? launch_backward_nk<N, true>(a, s) : launch_backward_nk<N, false>(a, s);
}

}  // namespace

// Samples one lane of the gradient launch carries when the caller leaves
// the choice to the library (samples_per_lane = 0). Measured on the
// 1M-Gaussian shell at 1080p (ms of gs_trace_backward, S = 1 against the
// choice): with T = spp * n_hits samples per pixel a lane takes K =
// n_hits * S slots, K = T up to 2, K = 4 below T = 16 (spp 4: 39.7 ->
// 15.0, per-lane packets), else K = 2 (spp 16: 49.4 -> 46.0, spp 64:
// 104.8 -> 59.8, 16- and 32-lane groups); never fewer than n_hits (N = 4
// at spp 4 and 16 keeps S = 1: 48.1 and 77.8 ms against 50.1 and 103.8).
static int auto_backward_samples_per_lane(int spp, int n_hits) {
    const int64_t T = (int64_t)spp * n_hits;
    int K = T <= 2 ? (int)T : (T < 16 ? 4 : 2);
    if (K < n_hits) K = n_hits;
    return K / n_hits;
}

gs_status launch_backward(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                          const gs_trace_params *p, const gs_sample_key *keys, const float *d_rgb,
                          float *d_means, float *d_log_scales, float *d_quats, float *d_logits,
                          float *d_sh, cudaStream_t s) {
    // a lane carries S consecutive samples: ceil(spp / S) passes of
    // n_hits * S slots, the same sample indices and keys as the forward
    int S = p->samples_per_lane > 0 ? p->samples_per_lane
                                    : auto_backward_samples_per_lane(p->spp, p->n_hits);
    while (S > 1 && S > p->spp) S >>= 1;
    const int spp_eff = (p->spp + S - 1) / S;
    TraceArgs a = {};
    a.nodes = b->nodes;
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
    a.step_limit = (uint32_t)(b->n_nodes + 8 < (int64_t)kStepLimit ? b->n_nodes + 8 : kStepLimit);
    a.status = b->status;
    a.work = b->status + 1;
    a.lpp_log2 = lanes_per_pixel_log2(spp_eff);
    if (b->node_depth && a.lpp_log2 >= 3) {
        a.grec = b->group[a.lpp_log2 - 3].rec;
        a.gcnt = b->group[a.lpp_log2 - 3].cnt;
        a.gq8 = b->node_format == GS_NODES_BINARY_Q8;
    }
    a.keys = const_cast<gs_sample_key *>(keys);  // read only here
    a.n_gauss = (uint32_t)b->M;
    a.d_rgb = d_rgb;
    a.log_scales = g->log_scales;
    a.quats = g->quats;
    a.g_means = d_means;
    a.g_log_scales = d_log_scales;
    a.g_quats = d_quats;
    a.g_logits = d_logits;
    a.g_sh = d_sh;
    gs_status st;
    switch (p->n_hits * S) {
        case 1: st = launch_backward_n<1>(a, s); break;
        case 2: st = launch_backward_n<2>(a, s); break;
        case 4: st = launch_backward_n<4>(a, s); break;
        case 8: st = launch_backward_n<8>(a, s); break;
        default: return fail(GS_ERR_INVALID_ARG, "n_hits must be 1, 2, 4 or 8");
    }
    if (st != GS_OK) return st;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "backward launch");
    return GS_OK;
}

}  // namespace gsrt
