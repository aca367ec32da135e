// trace_common.cuh -- device code shared by the forward trace (trace.cu)
// and the backward pass (backward.cu): launch arguments, Philox, camera
// rays, spherical harmonics, the Alg. 1 intersection routine, the slab test
// and the warp packet traversal. Both translation units compile the same
// source, so their per-candidate arithmetic is identical.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "gsrt_internal.cuh"

namespace gsrt {
namespace {

constexpr int kThreads = 128;

struct TraceArgs {
    const Node *nodes;
    const void *wide;  // Node4 or NodeQ4 when the handle has wide nodes
    const void *grec;      // W-wide records (ChildRec, or the 8-bit units) for the
                           // launch's group size, or null
    const uint32_t *gcnt;  // their per-node child counts (the root's at 0)
    int gq8;               // 1 when grec holds the 8-bit form
    const PrimRec *prims;
    const void *sh;
    int64_t n_nodes;
    int sh_degree;
    int sh_dtype;
    int width, height;
    uint32_t ray_id_offset;
    float eye[3], look_at[3], up[3];
    float tan_half;
    uint32_t key0, key1, stream_tag;
    uint32_t rk[20];  // Philox round keys (key0, key1) + r * (0x9E3779B9, 0xBB67AE85)
    int spp;        // passes per pixel of the launch (each with N slots)
    int n_samples;  // samples per pixel; slots at s = pass * N + k >= n_samples are unused
    float t_min, t_max;
    float bg[3];
    int stack_depth;
    uint32_t step_limit;
    float *rgb;
    int32_t *hit_id;
    float *hit_t;
    // per-sample payloads [pixel][sample]: written by the trace when set;
    // read by the backward when set, in place of its forward traversal
    gs_sample_key *keys;
    uint32_t n_gauss;  // Gaussians of the handle (bound on a stored key's id)
    unsigned long long *counters;
    uint32_t *status;
    uint32_t *work;  // tile counter of the persistent launch
    int lpp_log2;    // log2 of the lanes that trace samples of one pixel
    int depth_mode;  // 0: 1D mean; 1: centre projected on fwd (camera rays)
    int rng_mode;    // 0: Philox; 1: trigonometric hash of the hit point
    float fwd[3];    // camera forward axis (depth_mode 1)
    // backward pass only
    const float *d_rgb;        // [H][W][3] dLoss/d(pixel mean)
    const float *log_scales;   // raw parameters, for the scale and rotation
    const float *quats;        // derivatives
    float *g_means, *g_log_scales, *g_quats, *g_logits, *g_sh;
};

// A warp traces a tile of 32 >> lpp_log2 pixels, each pixel on 1 << lpp_log2
// consecutive lanes that take interleaved samples of the same camera ray.
// Tile width in pixels (a power of two); the height is the rest.
__host__ __device__ __forceinline__ int tile_w_log2(int lpp_log2) {
    const int px_log2 = 5 - lpp_log2;  // 32, 16, 8, 4, 2, 1 pixels
    return px_log2 >= 4 ? px_log2 - 2 : (px_log2 >= 2 ? px_log2 - 1 : px_log2);
}

// Lanes per pixel for a launch of spp passes: the largest power of two not
// above spp, at most the warp.
inline int lanes_per_pixel_log2(int spp) {
    int l = 0;
    while (l < 5 && (2 << l) <= spp) ++l;
    return l;
}

// ---------------------------------------------------------------- Philox
// Philox-4x32-10 (Salmon et al., SC'11): ten rounds, multipliers
// 0xD2511F53 and 0xCD9E8D57, key increments 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// The same generator with its ten round keys precomputed on the host
// (launch parameters), each round one 32x32->64-bit product per multiplier
// and two three-input exclusive ors.
__device__ __forceinline__ uint4 philox10_rk(uint4 c, const uint32_t rk[20]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53ull;
        const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57ull;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

// Round keys of philox10_rk for key (k0, k1).
inline void philox_round_keys(uint32_t k0, uint32_t k1, uint32_t rk[20]) {
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0 + (uint32_t)r * 0x9E3779B9u;
        rk[2 * r + 1] = k1 + (uint32_t)r * 0xBB67AE85u;
    }
}

__device__ __forceinline__ float lane_to_unit(uint32_t u) {
    return (float)(u >> 8) * 0x1p-24f;
}

__device__ __forceinline__ uint32_t pick(const uint4 &v, int lane) {
    return lane == 0 ? v.x : lane == 1 ? v.y : lane == 2 ? v.z : v.w;
}

// ---------------------------------------------------------------- camera
// Float32 camera ray with every operation rounded once (no contraction).
__device__ __forceinline__ void normalise_rn(float v[3]) {
    float n2 = __fmul_rn(v[0], v[0]);
    n2 = __fadd_rn(n2, __fmul_rn(v[1], v[1]));
    n2 = __fadd_rn(n2, __fmul_rn(v[2], v[2]));
    const float n = __fsqrt_rn(n2);
    v[0] = __fdiv_rn(v[0], n);
    v[1] = __fdiv_rn(v[1], n);
    v[2] = __fdiv_rn(v[2], n);
}

__device__ __forceinline__ void cross_rn(const float a[3], const float b[3], float c[3]) {
    c[0] = __fsub_rn(__fmul_rn(a[1], b[2]), __fmul_rn(a[2], b[1]));
    c[1] = __fsub_rn(__fmul_rn(a[2], b[0]), __fmul_rn(a[0], b[2]));
    c[2] = __fsub_rn(__fmul_rn(a[0], b[1]), __fmul_rn(a[1], b[0]));
}

__device__ __forceinline__ void camera_ray_view(const float eye[3], const float look_at[3],
                                                const float up[3], float tan_half, int width,
                                                int height, int x, int y, float d[3]) {
    float f[3], r[3], u[3];
    for (int i = 0; i < 3; ++i) f[i] = __fsub_rn(look_at[i], eye[i]);
    normalise_rn(f);
    cross_rn(f, up, r);
    normalise_rn(r);
    cross_rn(r, f, u);
    const float s = __fdiv_rn(tan_half, (float)height);
    const float ux = __fmul_rn((float)(2 * x + 1 - width), s);
    const float uy = __fmul_rn((float)(height - 1 - 2 * y), s);
    for (int i = 0; i < 3; ++i)
        d[i] = __fadd_rn(__fadd_rn(f[i], __fmul_rn(ux, r[i])), __fmul_rn(uy, u[i]));
    normalise_rn(d);
}

__device__ __forceinline__ void camera_ray(const TraceArgs &a, int x, int y, float d[3]) {
    camera_ray_view(a.eye, a.look_at, a.up, a.tan_half, a.width, a.height, x, y, d);
}

// ---------------------------------------------------------------- SH colour
__device__ __forceinline__ float load_coef(const void *sh, int dtype, int64_t i) {
    if (dtype == GS_SH_F32) return __ldg(static_cast<const float *>(sh) + i);
    const unsigned short raw = __ldg(static_cast<const unsigned short *>(sh) + i);
    if (dtype == GS_SH_F16) return __half2float(__ushort_as_half(raw));
    return __uint_as_float((uint32_t)raw << 16);  // bfloat16
}

// Real spherical harmonics with the Condon-Shortley phase as polynomials in
// the unit direction (x, y, z); constants are the normalisations
// sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!), times sqrt(2) for m != 0, times the
// Legendre polynomial coefficients. The DC term is pre-multiplied (basis 1).
__device__ void sh_basis(int deg, const float d[3], float Y[16]) {
    const float x = d[0], y = d[1], z = d[2];
    Y[0] = 1.0f;
    if (deg < 1) return;
    const float c1 = 0.48860251190291992f;  // sqrt(3/(4 pi))
    Y[1] = -c1 * y;
    Y[2] = c1 * z;
    Y[3] = -c1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    Y[4] = 1.0925484305920792f * x * y;              // sqrt(15/(4 pi))
    Y[5] = -1.0925484305920792f * y * z;
    Y[6] = 0.31539156525252005f * (3.0f * zz - 1.0f);  // sqrt(5/(16 pi))
    Y[7] = -1.0925484305920792f * x * z;
    Y[8] = 0.54627421529603959f * (xx - yy);          // sqrt(15/(16 pi))
    if (deg < 3) return;
    Y[9] = -0.59004358992664352f * y * (3.0f * xx - yy);  // sqrt(35/(32 pi))
    Y[10] = 2.8906114426405538f * x * y * z;               // sqrt(105/(4 pi))
    Y[11] = -0.45704579946446572f * y * (5.0f * zz - 1.0f);  // sqrt(21/(32 pi))
    Y[12] = 0.37317633259011540f * z * (5.0f * zz - 3.0f);   // sqrt(7/(16 pi))
    Y[13] = -0.45704579946446572f * x * (5.0f * zz - 1.0f);
    Y[14] = 1.4453057213202769f * z * (xx - yy);            // sqrt(105/(16 pi))
    Y[15] = -0.59004358992664352f * x * (xx - 3.0f * yy);
}

// Unclamped colour k_0 + sum Y_lm k_lm per channel.
__device__ __forceinline__ void sh_colour_raw(const TraceArgs &a, uint32_t gid, const float Y[16],
                                              float c[3]) {
    const int K = (a.sh_degree + 1) * (a.sh_degree + 1);
    const int64_t base = (int64_t)gid * K * 3;
    float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f;
    if (a.sh_dtype == GS_SH_F32 && K == 16) {
        const float4 *p = reinterpret_cast<const float4 *>(static_cast<const float *>(a.sh) + base);
        float v[48];
#pragma unroll
        for (int i = 0; i < 12; ++i) {
            const float4 q = __ldg(p + i);
            v[4 * i] = q.x; v[4 * i + 1] = q.y; v[4 * i + 2] = q.z; v[4 * i + 3] = q.w;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            acc0 = fmaf(Y[k], v[3 * k], acc0);
            acc1 = fmaf(Y[k], v[3 * k + 1], acc1);
            acc2 = fmaf(Y[k], v[3 * k + 2], acc2);
        }
    } else {
        for (int k = 0; k < K; ++k) {
            acc0 = fmaf(Y[k], load_coef(a.sh, a.sh_dtype, base + 3 * k), acc0);
            acc1 = fmaf(Y[k], load_coef(a.sh, a.sh_dtype, base + 3 * k + 1), acc1);
            acc2 = fmaf(Y[k], load_coef(a.sh, a.sh_dtype, base + 3 * k + 2), acc2);
        }
    }
    c[0] = acc0;
    c[1] = acc1;
    c[2] = acc2;
}

// View-dependent colour, clamped at zero.
__device__ __forceinline__ void sh_colour(const TraceArgs &a, uint32_t gid, const float Y[16],
                                          float c[3]) {
    sh_colour_raw(a, gid, Y, c);
    c[0] = fmaxf(c[0], 0.0f);
    c[1] = fmaxf(c[1], 0.0f);
    c[2] = fmaxf(c[2], 0.0f);
}

// ---------------------------------------------------------------- slots
struct Slot {
    float tc;   // base-point parameter
    float tau;  // 1D mean relative to the base point
    uint32_t gid;
    // the depth tc + tau, rounded once (range clipping and output); it is
    // exactly the candidate depth the slot was filled from
    __device__ __forceinline__ float t() const { return tc + tau; }
};

// (tc_a + tau_a, gid_a) < (tc_b + tau_b, gid_b), with the depth difference
// formed as (tc_a - tc_b) + (tau_a - tau_b).
__device__ __forceinline__ bool lex_closer(float tc, float tau, uint32_t gid, const Slot &s) {
    const float dt = (tc - s.tc) + (tau - s.tau);
    return dt < 0.0f || (dt == 0.0f && gid < s.gid);
}

template <int N>
struct Ray {
    float o[3], d[3], inv[3], oinv[3];
    uint32_t ray_id;
    uint32_t stream_tag;  // fourth Philox counter word
    float t_min, t_max;   // valid range of the 1D mean (Alg. 1)
    bool any_hit;         // stop at the first accepted hit (shadow rays)
    Slot slot[N];
    float t_far;  // conservative traversal clip
};

// Origin, unit direction and the slab-test reciprocals of a ray.
template <int N>
__device__ __forceinline__ void set_ray(Ray<N> &r, const float o[3], const float d[3]) {
    for (int i = 0; i < 3; ++i) {
        r.o[i] = o[i];
        r.d[i] = d[i];
        const float di = fabsf(d[i]) < 1e-30f ? copysignf(1e-30f, d[i]) : d[i];
        r.inv[i] = 1.0f / di;
        r.oinv[i] = r.o[i] * r.inv[i];
    }
}

template <int N>
__device__ __forceinline__ void reset_slots(Ray<N> &r) {
#pragma unroll
    for (int k = 0; k < N; ++k) r.slot[k] = Slot{INFINITY, 0.0f, 0xffffffffu};
}

template <int N>
__device__ __forceinline__ void update_clip(Ray<N> &r, float t_max) {
    float far = r.slot[0].t();
#pragma unroll
    for (int k = 1; k < N; ++k) far = fmaxf(far, r.slot[k].t());
    far = fminf(far, t_max);
    // expanded by 2^-19 relative so float32 slab rounding cannot cull a
    // node holding a hit that is (in exact arithmetic) not behind the clip
    r.t_far = far + fabsf(far) * 0x1p-19f;
}

// Trigonometric hash draw of Eq. 8-9 at hit point p for sample s (an
// alternative to Philox): xi = fract(b2 sin(a2 . (p_xy + r1(p_z)))), with
// r1(q) = fract(b1 sin(a1 q)), after moving p by a per-sample offset from
// the additive recurrence (fixed rays give no per-frame jitter here).
__device__ __forceinline__ float fract_f(float x) { return x - floorf(x); }

__device__ __forceinline__ float hash_xi(const float p[3], uint32_t s) {
    const float c[3] = {0.8191725134f, 0.6710436067f, 0.5497004779f};
    float q[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) q[i] = p[i] + 1e-3f * fract_f((float)s * c[i]) - 5e-4f;
    const float r1 = fract_f(47453.5453f * sinf(91.3458f * q[2]));
    return fract_f(43758.5453f * sinf(12.9898f * (q[0] + r1) + 78.233f * (q[1] + r1)));
}

// Alg. 1, split in three so that the cooperative traversal can evaluate
// the sample-independent part once per Gaussian and ray:
//   cand_depth  the record, the base point and the 1D mean (its depth key),
//               and the range test t_min < t < t_max;
//   cand_alpha  the refined minimum q, the ellipsoid test q <= s^2 and alpha;
//   accept      the draws of this lane's samples that are closer than their
//               slots, replacing slots and clipping.
// With RELOAD (the grouped traversal, whose leaf step is its register
// peak) cand_alpha re-reads M and the opacity from the record, which L1
// still holds, instead of keeping them live (measured 1-5% faster there;
// the per-lane packets keep them, 2% faster so).
struct CandGeom {
    float m[9];
    float w[3], md[3];
    float inv_dd, tau;
    float t, key_tc, key_tau;
    float opacity;
    uint32_t idx;
    uint32_t gid;
};

template <int N, bool RELOAD = false>
__device__ __forceinline__ bool cand_depth(const TraceArgs &a, const Ray<N> &r, uint32_t idx,
                                           CandGeom &c) {
    const float4 *pp = reinterpret_cast<const float4 *>(a.prims + idx);
    const float4 p0 = __ldg(pp), p1 = __ldg(pp + 1), p2 = __ldg(pp + 2), p3 = __ldg(pp + 3);
    const float mu[3] = {p0.x, p0.y, p0.z};
    const float m[9] = {p1.x, p1.y, p1.z, p1.w, p2.x, p2.y, p2.z, p2.w, p3.x};
    if constexpr (!RELOAD) {
#pragma unroll
        for (int i = 0; i < 9; ++i) c.m[i] = m[i];
        c.opacity = p0.w;
    }
    c.idx = idx;
    c.gid = __float_as_uint(p3.y);
    // o - mu = h + l exactly (two-sum)
    float h[3], l[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float s = r.o[i] - mu[i];
        const float bp = s - r.o[i];
        const float ap = s - bp;
        l[i] = (r.o[i] - ap) + (-mu[i] - bp);
        h[i] = s;
    }
    const float tc = -fmaf(h[0], r.d[0], fmaf(h[1], r.d[1], h[2] * r.d[2]));
#pragma unroll
    for (int i = 0; i < 3; ++i) c.w[i] = fmaf(tc, r.d[i], h[i]) + l[i];
    float mw[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        c.md[i] = fmaf(m[3 * i], r.d[0], fmaf(m[3 * i + 1], r.d[1], m[3 * i + 2] * r.d[2]));
        mw[i] = fmaf(m[3 * i], c.w[0], fmaf(m[3 * i + 1], c.w[1], m[3 * i + 2] * c.w[2]));
    }
    const float dd = fmaf(c.md[0], c.md[0], fmaf(c.md[1], c.md[1], c.md[2] * c.md[2]));
    const float wd = fmaf(mw[0], c.md[0], fmaf(mw[1], c.md[1], mw[2] * c.md[2]));
    c.inv_dd = 1.0f / dd;
    c.tau = -wd * c.inv_dd;
    c.t = tc + c.tau;
    // depth key (tc, tau); the projected-centre depth uses (centre, 0)
    c.key_tc = tc;
    c.key_tau = c.tau;
    if (a.depth_mode == 1) {
        const float hf = fmaf(h[0], a.fwd[0], fmaf(h[1], a.fwd[1], h[2] * a.fwd[2]));
        const float lf = fmaf(l[0], a.fwd[0], fmaf(l[1], a.fwd[1], l[2] * a.fwd[2]));
        c.t = -(hf + lf);
        c.key_tc = c.t;
        c.key_tau = 0.0f;
    }
    return (c.t > r.t_min) && (c.t < r.t_max);
}

// Refine the base point to the 1D mean, then the ellipsoid test (Eq. 2).
template <int N, bool RELOAD = false>
__device__ __forceinline__ bool cand_alpha(const TraceArgs &a, const Ray<N> &r, const CandGeom &c,
                                           float &alpha) {
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
    float w2[3], mw2[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) w2[i] = fmaf(c.tau, r.d[i], c.w[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        mw2[i] = fmaf(m[3 * i], w2[0], fmaf(m[3 * i + 1], w2[1], m[3 * i + 2] * w2[2]));
    const float ww = fmaf(mw2[0], mw2[0], fmaf(mw2[1], mw2[1], mw2[2] * mw2[2]));
    const float wd2 = fmaf(mw2[0], c.md[0], fmaf(mw2[1], c.md[1], mw2[2] * c.md[2]));
    const float q = fmaxf(ww - wd2 * wd2 * c.inv_dd, 0.0f);
    if (!(q <= kS2)) return false;
    alpha = opacity * expf(-0.5f * q);
    return true;
}

// Eq. 4 for the slots that the candidate is closer than: accept iff
// xi < alpha, replacing the slot (Eq. 6) and clipping the traversal range.
template <int N, bool COUNT>
__device__ __forceinline__ void accept(const TraceArgs &a, Ray<N> &r, int pass, const bool closer[N],
                                       float t, float key_tc, float key_tau, float alpha,
                                       uint32_t gid, unsigned long long &n_draws) {
    const uint32_t s0 = (uint32_t)pass * N;
    if (a.rng_mode == 1) {
        float ph[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) ph[i] = fmaf(t, r.d[i], r.o[i]);
#pragma unroll
        for (int k = 0; k < N; ++k) {
            if (!closer[k]) continue;
            if (hash_xi(ph, s0 + k) < alpha) {
                r.slot[k].tc = key_tc;
                r.slot[k].tau = key_tau;
                r.slot[k].gid = gid;
            }
        }
        update_clip(r, r.t_max);
        if (a.depth_mode == 1) r.t_far = r.t_max;
        return;
    }
    // one Philox call serves four consecutive samples
    uint4 u0 = make_uint4(0, 0, 0, 0), u1 = make_uint4(0, 0, 0, 0);
    u0 = philox10_rk(make_uint4(r.ray_id, gid, s0 >> 2, r.stream_tag), a.rk);
    if (N == 8) u1 = philox10_rk(make_uint4(r.ray_id, gid, (s0 >> 2) + 1, r.stream_tag), a.rk);
    if (COUNT) n_draws += 1 + (N == 8);
#pragma unroll
    for (int k = 0; k < N; ++k) {
        if (!closer[k]) continue;
        const uint32_t s = s0 + k;
        const uint32_t bits = (N == 8 && k >= 4) ? pick(u1, s & 3) : pick(u0, s & 3);
        if (lane_to_unit(bits) < alpha) {
            r.slot[k].tc = key_tc;
            r.slot[k].tau = key_tau;
            r.slot[k].gid = gid;
        }
    }
    if (r.any_hit) {
        // a sample's visibility is known at its first accepted hit: that
        // slot stops holding the clip and nothing is closer than it
#pragma unroll
        for (int k = 0; k < N; ++k)
            if (r.slot[k].gid != 0xffffffffu) r.slot[k].tc = -INFINITY;
    }
    update_clip(r, r.t_max);
    if (r.any_hit && !(r.t_far > -INFINITY)) r.t_far = -INFINITY;  // every sample known
    // A projected-centre depth is not a ray parameter, so it cannot clip the
    // box tests: every box on the ray stays open and order is decided here.
    if (a.depth_mode == 1) r.t_far = r.t_max;
}

// Which slots a candidate at depth key (key_tc, key_tau) is closer than,
// after the clip test t <= t_far (t_far only prunes hits behind every slot).
template <int N>
__device__ __forceinline__ bool closer_slots(const Ray<N> &r, float t, float key_tc, float key_tau,
                                             uint32_t gid, bool closer[N]) {
    if (!(t <= r.t_far)) return false;
    bool any = false;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        closer[k] = lex_closer(key_tc, key_tau, gid, r.slot[k]);
        any |= closer[k];
    }
    return any;
}

// Alg. 1 for primitive record idx against all N slots of the current pass.
template <int N, bool COUNT>
__device__ __forceinline__ void intersect(const TraceArgs &a, Ray<N> &r, uint32_t idx, int pass,
                                          unsigned long long &n_draws) {
    CandGeom c;
    if (!cand_depth<N>(a, r, idx, c)) return;
    bool closer[N];
    if (!closer_slots<N>(r, c.t, c.key_tc, c.key_tau, c.gid, closer)) return;
    float alpha;
    if (!cand_alpha<N>(a, r, c, alpha)) return;
    accept<N, COUNT>(a, r, pass, closer, c.t, c.key_tc, c.key_tau, alpha, c.gid, n_draws);
}

// Slab test of one child box against [t_min, t_far].
__device__ __forceinline__ bool slab(const float *lo_hi, const float inv[3], const float oinv[3],
                                     float t_min, float t_far, float &t_enter) {
    const float tx0 = fmaf(lo_hi[0], inv[0], -oinv[0]), tx1 = fmaf(lo_hi[3], inv[0], -oinv[0]);
    const float ty0 = fmaf(lo_hi[1], inv[1], -oinv[1]), ty1 = fmaf(lo_hi[4], inv[1], -oinv[1]);
    const float tz0 = fmaf(lo_hi[2], inv[2], -oinv[2]), tz1 = fmaf(lo_hi[5], inv[2], -oinv[2]);
    const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), t_min));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), t_far));
    t_enter = tn;
    return tn <= tf;
}

// Packet traversal of one 8x4 pixel tile by one warp (same pass for all
// lanes). The warp visits the union of the nodes its lanes need: every node
// is fetched once for the whole warp (one broadcast load), each lane
// slab-tests the children against its own clipped range and keeps its own
// slots, and the warp descends while any lane still needs a child. A lane's
// stack entry remembers its own entry distance, so a popped node is skipped
// once every lane's clip has passed it. Each lane runs Alg. 1 on exactly
// the leaves its own ray reaches, so per-lane results are those of an
// independent traversal.
struct Counts {
    unsigned long long nodes = 0;        // nodes entered by this lane's own ray
    unsigned long long prims = 0;        // Gaussians tested by this lane
    unsigned long long draws = 0;        // Philox calls
    unsigned long long node_fetch = 0;   // node records fetched by the warp
    unsigned long long prim_fetch = 0;   // Gaussian records fetched by the warp
};

template <int N, bool COUNT>
__device__ __forceinline__ void traverse_packet(const TraceArgs &a, Ray<N> &r, int pass,
                                                uint32_t *stack, float *stack_t, uint32_t &err,
                                                Counts &cnt) {
    const uint32_t kAll = 0xffffffffu;
    const bool lane0 = (threadIdx.x & 31) == 0;
    int sp = 0;
    uint32_t node = 0, steps = 0;
    bool active = r.t_far >= r.t_min;  // this lane's ray entered the node
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
        }
        if (COUNT) {
            cnt.nodes += active;
            cnt.node_fetch += lane0;
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
        if (leafL || leafR) {
            // Alg. 1 on the leaves this lane's ray reaches, nearer box first
            const bool swap = leafL && leafR && hR && (!hL || tR < tL);
            if (COUNT) {
                const unsigned wl = __ballot_sync(kAll, leafL && hL);
                const unsigned wr = __ballot_sync(kAll, leafR && hR);
                if (lane0) cnt.prim_fetch += (wl != 0u) + (wr != 0u);
            }
            for (int li = 0; li < 2; ++li) {
                const bool right = (li == 0) == swap;
                if (!(right ? leafR : leafL) || !(right ? hR : hL)) continue;
                if (COUNT) ++cnt.prims;
                intersect<N, COUNT>(a, r, (right ? cref.y : cref.x) & ~kLeafBit, pass, cnt.draws);
            }
            if (leafL) hL = false;
            if (leafR) hR = false;
            hL = hL && tL <= r.t_far;
            hR = hR && tR <= r.t_far;
        }
        const unsigned mL = __ballot_sync(kAll, hL), mR = __ballot_sync(kAll, hR);
        if (mL && mR) {
            // the child most lanes enter first is visited first
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
            active = left_first ? hL : hR;
            continue;
        }
        if (mL) { node = cref.x; active = hL; continue; }
        if (mR) { node = cref.y; active = hR; continue; }
        bool found = false;
        while (sp > 0) {
            --sp;
            const bool want = stack_t[sp] <= r.t_far;
            if (__any_sync(kAll, want)) {
                node = stack[sp];
                active = want;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}


// Child boxes of a wide node as FP32 planes. For the 8-bit form each plane
// is origin + q * 2^e rounded once, exactly as the build verified it, so a
// decoded box contains the FP32 box and the (monotone) slab test can only
// report more hits, never fewer.
template <int FMT>
__device__ __forceinline__ void load_wide(const TraceArgs &a, uint32_t node, float box[4][6],
                                          uint32_t child[4]) {
    if (FMT == GS_NODES_WIDE4) {
        const float4 *np = reinterpret_cast<const float4 *>(static_cast<const Node4 *>(a.wide) + node);
        const float4 lx = __ldg(np), ly = __ldg(np + 1), lz = __ldg(np + 2);
        const float4 hx = __ldg(np + 3), hy = __ldg(np + 4), hz = __ldg(np + 5);
        const uint4 c = __ldg(reinterpret_cast<const uint4 *>(np + 6));
        const float LX[4] = {lx.x, lx.y, lx.z, lx.w}, LY[4] = {ly.x, ly.y, ly.z, ly.w};
        const float LZ[4] = {lz.x, lz.y, lz.z, lz.w}, HX[4] = {hx.x, hx.y, hx.z, hx.w};
        const float HY[4] = {hy.x, hy.y, hy.z, hy.w}, HZ[4] = {hz.x, hz.y, hz.z, hz.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            box[k][0] = LX[k]; box[k][1] = LY[k]; box[k][2] = LZ[k];
            box[k][3] = HX[k]; box[k][4] = HY[k]; box[k][5] = HZ[k];
        }
        child[0] = c.x; child[1] = c.y; child[2] = c.z; child[3] = c.w;
    } else {
        const uint4 *np = reinterpret_cast<const uint4 *>(static_cast<const NodeQ4 *>(a.wide) + node);
        const uint4 v0 = __ldg(np), v1 = __ldg(np + 1), v2 = __ldg(np + 2), v3 = __ldg(np + 3);
        const float origin[3] = {__uint_as_float(v0.x), __uint_as_float(v0.y), __uint_as_float(v0.z)};
        float scale[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax) {
            const int e = (int)(signed char)((v0.w >> (8 * ax)) & 0xffu);
            scale[ax] = __uint_as_float((uint32_t)(e + 127) << 23);
        }
        const uint32_t used = (v0.w >> 24) & 0xffu;
        const uint32_t qlo[3] = {v1.x, v1.y, v1.z};
        const uint32_t qhi[3] = {v1.w, v2.x, v2.y};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const float ql = (float)((qlo[ax] >> (8 * k)) & 0xffu);
                const float qh = (float)((qhi[ax] >> (8 * k)) & 0xffu);
                box[k][ax] = __fadd_rn(origin[ax], ql * scale[ax]);
                box[k][3 + ax] = __fadd_rn(origin[ax], qh * scale[ax]);
            }
            if (!((used >> k) & 1u)) {
                box[k][0] = box[k][1] = box[k][2] = INFINITY;
                box[k][3] = box[k][4] = box[k][5] = INFINITY;
            }
        }
        child[0] = v2.z; child[1] = v2.w; child[2] = v3.x; child[3] = v3.y;
    }
}

// Packet traversal of a 4-wide hierarchy. Leaves are tested nearest first
// per lane; internal children are ordered for the whole warp by their
// nearest entry over the lanes that reach them, the nearest visited next and
// the others pushed with each lane's own entry distance.
template <int N, bool COUNT, int FMT>
__device__ __forceinline__ void traverse_packet_wide(const TraceArgs &a, Ray<N> &r, int pass,
                                                     uint32_t *stack, float *stack_t,
                                                     uint32_t &err, Counts &cnt) {
    const uint32_t kAll = 0xffffffffu;
    const bool lane0 = (threadIdx.x & 31) == 0;
    int sp = 0;
    uint32_t node = 0, steps = 0;
    bool active = r.t_far >= r.t_min;
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
        }
        if (COUNT) {
            cnt.nodes += active;
            cnt.node_fetch += lane0;
        }
        float box[4][6];
        uint32_t C[4];
        load_wide<FMT>(a, node, box, C);
        float t[4];
        bool h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) h[k] = slab(box[k], r.inv, r.oinv, r.t_min, r.t_far, t[k]);
        unsigned todo = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (C[k] != kEmpty && (C[k] & kLeafBit) && h[k]) todo |= 1u << k;
        if (COUNT) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const unsigned w = __ballot_sync(kAll, (todo >> k) & 1u);
                if (lane0 && w) ++cnt.prim_fetch;
            }
        }
        while (todo) {
            int best = 0;
            float bt = INFINITY;
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (((todo >> k) & 1u) && !(t[k] >= bt)) { best = k; bt = t[k]; }
            todo &= ~(1u << best);
            uint32_t leaf = C[0];
#pragma unroll
            for (int k = 1; k < 4; ++k) if (k == best) leaf = C[k];
            if (COUNT) ++cnt.prims;
            intersect<N, COUNT>(a, r, leaf & ~kLeafBit, pass, cnt.draws);
        }
        uint32_t key[4];
        int slot[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool in = C[k] != kEmpty && !(C[k] & kLeafBit);
            h[k] = in && h[k] && t[k] <= r.t_far;
            key[k] = __reduce_min_sync(kAll, h[k] ? __float_as_uint(fmaxf(t[k], 0.0f)) : 0xffffffffu);
            slot[k] = k;
        }
        // sort four (key, slot) pairs ascending; keys are uniform over the warp
#define GS_CSWAP(i, j)                                                   \
    if (key[j] < key[i]) {                                               \
        const uint32_t tk = key[i]; key[i] = key[j]; key[j] = tk;        \
        const int ts = slot[i]; slot[i] = slot[j]; slot[j] = ts;         \
    }
        GS_CSWAP(0, 1) GS_CSWAP(2, 3) GS_CSWAP(0, 2) GS_CSWAP(1, 3) GS_CSWAP(1, 2)
#undef GS_CSWAP
        if (key[0] != 0xffffffffu) {
            bool overflow = false;
#pragma unroll
            for (int j = 3; j >= 1; --j) {
                if (key[j] == 0xffffffffu) continue;
                if (sp >= a.stack_depth) { overflow = true; break; }
                uint32_t c = C[0];
                float tt = t[0];
                bool hh = h[0];
#pragma unroll
                for (int k = 1; k < 4; ++k)
                    if (k == slot[j]) { c = C[k]; tt = t[k]; hh = h[k]; }
                stack[sp] = c;
                stack_t[sp] = hh ? tt : INFINITY;
                ++sp;
            }
            if (overflow) {
                err |= kErrStack;
                break;
            }
            uint32_t c = C[0];
            bool hh = h[0];
#pragma unroll
            for (int k = 1; k < 4; ++k)
                if (k == slot[0]) { c = C[k]; hh = h[k]; }
            node = c;
            active = hh;
            continue;
        }
        bool found = false;
        while (sp > 0) {
            --sp;
            const bool want = stack_t[sp] <= r.t_far;
            if (__any_sync(kAll, want)) {
                node = stack[sp];
                active = want;
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}


// Independent traversal of the binary hierarchy by one lane (for rays
// whose directions differ from lane to lane, where a packet would visit the
// union of unrelated paths): near child first, the other pushed with its
// entry distance, pops skipped once the lane's clip has passed them.
template <int N, bool COUNT>
__device__ __forceinline__ void traverse_lane(const TraceArgs &a, Ray<N> &r, int pass,
                                              uint32_t *stack, float *stack_t, uint32_t &err,
                                              Counts &cnt) {
    if (!(r.t_far >= r.t_min)) return;
    int sp = 0;
    uint32_t node = 0, steps = 0;
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
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
                intersect<N, COUNT>(a, r, (right ? cref.y : cref.x) & ~kLeafBit, pass, cnt.draws);
            }
        }
        hL = hL && !leafL && tL <= r.t_far;
        hR = hR && !leafR && tR <= r.t_far;
        if (hL && hR) {
            if (sp >= a.stack_depth) {
                err |= kErrStack;
                break;
            }
            const bool left_first = tL <= tR;
            stack[sp] = left_first ? cref.y : cref.x;
            stack_t[sp] = left_first ? tR : tL;
            ++sp;
            node = left_first ? cref.x : cref.y;
            continue;
        }
        if (hL) { node = cref.x; continue; }
        if (hR) { node = cref.y; continue; }
        bool found = false;
        while (sp > 0) {
            --sp;
            if (stack_t[sp] <= r.t_far) {
                node = stack[sp];
                found = true;
                break;
            }
        }
        if (!found) break;
    }
}

// ---------------------------------------------------------------- groups
// Child `sub` of the wide node `node` slab-tested against [t_min, G]: its
// reference, its entry distance, and whether the ray enters its box. FP32
// records hold the box. In the 8-bit form plane q of axis a lies at
// origin + q * scale, i.e. at ray parameter q * A + B with A = scale * inv
// and B = origin * inv - o * inv; q enters as the float 2^23 + q (exact, one
// byte permute) and B as B - 2^23 A, rounded once (at most half a quantum of
// the ray parameter, within the spare quantum the build leaves on each side).
template <bool Q8>
__device__ __forceinline__ bool group_child(const void *grec, uint32_t node, int sub,
                                            const float inv[3], const float oinv[3], float t_min,
                                            float G, uint32_t &ref, float &te) {
    if constexpr (!Q8) {
        const float4 *cp = reinterpret_cast<const float4 *>(
            static_cast<const ChildRec *>(grec) + (node & kWideOffsetMask) + sub);
        const float4 q0 = __ldg(cp), q1 = __ldg(cp + 1);
        const float bx[6] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y};
        ref = __float_as_uint(q1.z);
        return slab(bx, inv, oinv, t_min, G, te);
    } else {
        const uint4 *u = static_cast<const uint4 *>(grec) + (node & kWideOffsetMask);
        const float4 h0 = __ldg(reinterpret_cast<const float4 *>(u));
        const float4 h1 = __ldg(reinterpret_cast<const float4 *>(u) + 1);
        const uint4 c = __ldg(u + kGroupQHeaderUnits + sub);
        ref = c.z;
        const float A0 = h0.w * inv[0], A1 = h1.x * inv[1], A2 = h1.y * inv[2];
        const float B0 = fmaf(-8388608.0f, A0, fmaf(h0.x, inv[0], -oinv[0]));
        const float B1 = fmaf(-8388608.0f, A1, fmaf(h0.y, inv[1], -oinv[1]));
        const float B2 = fmaf(-8388608.0f, A2, fmaf(h0.z, inv[2], -oinv[2]));
        const float lx = __uint_as_float(__byte_perm(c.x, 0x4B000000u, 0x7440u));
        const float ly = __uint_as_float(__byte_perm(c.x, 0x4B000000u, 0x7441u));
        const float lz = __uint_as_float(__byte_perm(c.x, 0x4B000000u, 0x7442u));
        const float hx = __uint_as_float(__byte_perm(c.x, 0x4B000000u, 0x7443u));
        const float hy = __uint_as_float(__byte_perm(c.y, 0x4B000000u, 0x7440u));
        const float hz = __uint_as_float(__byte_perm(c.y, 0x4B000000u, 0x7441u));
        const float tx0 = fmaf(lx, A0, B0), tx1 = fmaf(hx, A0, B0);
        const float ty0 = fmaf(ly, A1, B1), ty1 = fmaf(hy, A1, B1);
        const float tz0 = fmaf(lz, A2, B2), tz1 = fmaf(hz, A2, B2);
        const float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), t_min));
        const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), G));
        te = tn;
        return tn <= tf && !(c.y & kQ8Skip);
    }
}

constexpr int kGroupPool = 512;    // stack entries per warp, split among its groups
constexpr int kGroupMinBlocks = 8; // resident blocks per SM to build for

// Cooperative traversal of the W-wide hierarchy (W = L = 2^LG, 8 to 32) by a
// group of L lanes that trace different samples of one ray. The group
// visits a wide node in one step: lane k tests child k against the group's
// clip (the farthest of its lanes' clips). Lanes holding a hit leaf evaluate
// the sample-independent part of Alg. 1 for it (cand_depth, cand_alpha);
// every lane then draws for its own samples against each candidate
// (accept). The nearest hit inner child is visited next and the other hit
// inner children go to the group's stack in shared memory. Every node and
// leaf a lane's own ray needs is visited, and each lane keeps its own slots
// and clip, so per-lane results are those of an independent traversal.
// POP2 selects the two-stage pop of the group stack (below); both pop the
// same entries. Q8 reads the 8-bit form of the records.
template <int N, bool COUNT, int LG, bool POP2 = false, bool Q8 = false>
__device__ __forceinline__ void traverse_group(const TraceArgs &a, Ray<N> &r, int pass,
                                               uint32_t *s_ref, float *s_t, uint32_t &err,
                                               Counts &cnt) {
    constexpr int L = 1 << LG;
    constexpr int kCap = kGroupPool >> (5 - LG);  // this group's stack entries
    constexpr uint32_t kLaneBits = L == 32 ? 0xffffffffu : ((1u << (L & 31)) - 1u);
    const int lane = threadIdx.x & 31;
    const int base = lane & ~(L - 1);
    const int sub = lane & (L - 1);
    const uint32_t gmask = kLaneBits << base;
    float G = r.t_far >= r.t_min ? r.t_far : -INFINITY;
#pragma unroll
    for (int o = 1; o < L; o <<= 1) G = fmaxf(G, __shfl_xor_sync(gmask, G, o));
    if (!(G >= r.t_min)) return;  // no lane of the group is live
    int sp = 0;
    uint32_t node = (__ldg(a.gcnt) - 1u) << kWideCountShift;  // the root's records start at 0
    uint32_t steps = 0;
    float node_t = r.t_min;
    for (;;) {
        if (++steps > a.step_limit) {
            err |= kErrSteps;
            break;
        }
        const int n_child = (int)((node >> kWideCountShift) & 31u) + 1;
        if (COUNT) {
            // the child records of a wide node this lane's own ray enters
            cnt.nodes += node_t <= r.t_far ? n_child : 0;
            cnt.node_fetch += lane == base ? n_child : 0;
        }
        uint32_t ref = kEmpty;
        float te = INFINITY;
        bool hit = false;
        if (sub < n_child) hit = group_child<Q8>(a.grec, node, sub, r.inv, r.oinv, r.t_min, G, ref, te);
        const bool leaf = (ref & kLeafBit) != 0u;
        const uint32_t lm = (__ballot_sync(gmask, hit && leaf) >> base) & kLaneBits;
        if (lm) {
            if (COUNT) {
                for (uint32_t m2 = lm; m2; m2 &= m2 - 1u) {
                    const float tl = __shfl_sync(gmask, te, base + __ffs(m2) - 1);
                    cnt.prims += tl <= r.t_far;
                    cnt.prim_fetch += lane == base;
                }
            }
            // one lane per hit leaf: the part of Alg. 1 all samples share
            float ct = 0.0f, ck1 = 0.0f, ck2 = 0.0f, cal = 0.0f;
            uint32_t cgid = 0;
            bool ok = false;
            if (hit && leaf) {
                CandGeom c;
                ok = cand_depth<N, true>(a, r, ref & ~kLeafBit, c) && cand_alpha<N, true>(a, r, c, cal);
                ct = c.t;
                ck1 = c.key_tc;
                ck2 = c.key_tau;
                cgid = c.gid;
                // a lane takes a candidate only at t <= its own clip <= G
                ok = ok && ct <= G;
            }
            const float far0 = r.t_far;
            // every lane: its own draws against each candidate
            for (uint32_t cm = (__ballot_sync(gmask, ok) >> base) & kLaneBits; cm; cm &= cm - 1u) {
                const int src = base + __ffs(cm) - 1;
                const float t = __shfl_sync(gmask, ct, src);
                const float key_tc = __shfl_sync(gmask, ck1, src);
                const float key_tau = __shfl_sync(gmask, ck2, src);
                const float alpha = __shfl_sync(gmask, cal, src);
                const uint32_t gid = __shfl_sync(gmask, cgid, src);
                bool closer[N];
                if (closer_slots<N>(r, t, key_tc, key_tau, gid, closer))
                    accept<N, COUNT>(a, r, pass, closer, t, key_tc, key_tau, alpha, gid, cnt.draws);
            }
            // the group clip moves only when some lane's clip did
            if (__any_sync(gmask, r.t_far != far0)) {
                G = r.t_far >= r.t_min ? r.t_far : -INFINITY;
#pragma unroll
                for (int o = 1; o < L; o <<= 1) G = fmaxf(G, __shfl_xor_sync(gmask, G, o));
            }
        }
        const bool inner = hit && !leaf && te <= G;
        const uint32_t im = (__ballot_sync(gmask, inner) >> base) & kLaneBits;
        if (im) {
            // nearest inner child next (ties and the low five mantissa bits
            // of the entry distance broken by child index)
            const uint32_t key = __reduce_min_sync(
                gmask, inner ? ((__float_as_uint(fmaxf(te, 0.0f)) & ~31u) | (uint32_t)sub)
                             : 0xffffffffu);
            const int nj = (int)(key & 31u);
            const uint32_t next = __shfl_sync(gmask, ref, base + nj);
            const float next_t = __shfl_sync(gmask, te, base + nj);
            const uint32_t others = im & ~(1u << nj);
            const int npush = __popc(others);
            if (sp + npush > kCap) {
                err |= kErrStack;
                break;
            }
            __syncwarp(gmask);  // earlier reads of these entries are done
            if (inner && sub != nj) {
                const int pos = sp + __popc(others & ((1u << sub) - 1u));
                s_ref[pos] = ref;
                s_t[pos] = te;
            }
            sp += npush;
            __syncwarp(gmask);
            node = next;
            node_t = next_t;
            continue;
        }
        // pop the topmost entry within the group clip, dropping the ones
        // above it
        bool found = false;
        if constexpr (POP2) {
            // the top entry alone first (it usually holds); past it, lane k
            // checks the k-th entry below, one step per L culled entries
            if (sp > 0) {
                const float tt = s_t[sp - 1];
                if (tt <= G) {
                    --sp;
                    node = s_ref[sp];
                    node_t = tt;
                    found = true;
                } else {
                    --sp;
                }
            }
            if (!found)
                while (sp > 0) {
                    const int k = sp - 1 - sub;
                    const float tt = k >= 0 ? s_t[k] : INFINITY;
                    const uint32_t okm = (__ballot_sync(gmask, tt <= G) >> base) & kLaneBits;
                    if (okm) {
                        const int j = __ffs(okm) - 1;  // the lowest lane holds the topmost
                        sp = sp - 1 - j;
                        node = s_ref[sp];
                        node_t = s_t[sp];
                        found = true;
                        break;
                    }
                    sp = sp > L ? sp - L : 0;
                }
        } else {
            while (sp > 0) {
                --sp;
                const float tt = s_t[sp];
                if (tt <= G) {
                    node = s_ref[sp];
                    node_t = tt;
                    found = true;
                    break;
                }
            }
        }
        if (!found) break;
    }
}

}  // namespace
}  // namespace gsrt
