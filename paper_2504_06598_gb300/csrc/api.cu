// api.cu -- the C ABI of include/gsrt.h: argument validation, handle
// lifecycle, status reporting. Kernels live in build.cu and trace.cu.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "gsrt_internal.cuh"

namespace gsrt {

static thread_local char g_last_error[512] = "";

gs_status fail(gs_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return s;
}

gs_status cuda_fail(cudaError_t e, const char *what) {
    gs_status s = (e == cudaErrorMemoryAllocation) ? GS_ERR_OOM
                  : (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) ? GS_ERR_NO_DEVICE
                                                                                  : GS_ERR_CUDA;
    return fail(s, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static gs_status check_device() {
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess || n == 0) {
        cudaGetLastError();
        return fail(GS_ERR_NO_DEVICE, "no CUDA device available");
    }
    return GS_OK;
}

// Host-only checks of a parameter struct (no CUDA call).
static gs_status check_gaussians_host(const gs_gaussians *g, bool need_sh) {
    if (!g) return fail(GS_ERR_INVALID_ARG, "gaussians is NULL");
    if (g->M < 0 || g->M >= (int64_t)0x7fffffff)
        return fail(GS_ERR_INVALID_ARG, "M=%lld out of range [0, 2^31-1)", (long long)g->M);
    if (g->M > 0) {
        if (!g->means || !g->log_scales || !g->quats || !g->opacity_logits)
            return fail(GS_ERR_INVALID_ARG, "a Gaussian parameter pointer is NULL");
        if (need_sh && !g->sh) return fail(GS_ERR_INVALID_ARG, "sh is NULL");
    }
    if (g->sh_degree < 0 || g->sh_degree > 3)
        return fail(GS_ERR_INVALID_ARG, "sh_degree=%d not in 0..3", g->sh_degree);
    if (g->sh_dtype != GS_SH_F32 && g->sh_dtype != GS_SH_F16 && g->sh_dtype != GS_SH_BF16)
        return fail(GS_ERR_INVALID_ARG, "sh_dtype=%d unknown", g->sh_dtype);
    if (need_sh && g->M > 0 && g->sh_dtype == GS_SH_F32 && !aligned16(g->sh))
        return fail(GS_ERR_INVALID_ARG, "float32 sh must be 16-byte aligned");
    return GS_OK;
}

static gs_status check_gaussians_device(const gs_gaussians *g, bool need_sh) {
    if (g->M == 0) return GS_OK;
    const void *ptrs[5] = {g->means, g->log_scales, g->quats, g->opacity_logits, g->sh};
    const char *names[5] = {"means", "log_scales", "quats", "opacity_logits", "sh"};
    for (int i = 0; i < (need_sh ? 5 : 4); ++i)
        if (!is_device_ptr(ptrs[i]))
            return fail(GS_ERR_INVALID_ARG, "%s is not a device pointer", names[i]);
    return GS_OK;
}

static void release(gs_bvh *b) {
    if (!b) return;
    void *bufs[] = {b->nodes, b->prims, b->status, b->codes[0], b->codes[1], b->vals[0],
                    b->vals[1], b->parent, b->arrive, b->aabb, b->bounds, b->hist,
                    b->scan_tmp, b->wide, b->depth, b->wmap, b->node_depth};
    for (void *p : bufs)
        if (p) cudaFree(p);
    for (auto &t : b->group) {
        if (t.rec) cudaFree(t.rec);
        if (t.cnt) cudaFree(t.cnt);
        if (t.off) cudaFree(t.off);
    }
    void *wave[] = {b->wave_codes[0], b->wave_codes[1], b->wave_bounce, b->wave_hist, b->wave_scan};
    for (void *p : wave)
        if (p) cudaFree(p);
    free(b);
}

}  // namespace gsrt

using namespace gsrt;

extern "C" {

const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_OOM: return "out of device memory";
        case GS_ERR_STACK_OVERFLOW: return "traversal stack overflow";
        case GS_ERR_STEP_LIMIT: return "traversal step limit exceeded";
        case GS_ERR_NONFINITE: return "non-finite Gaussian parameter";
        case GS_ERR_NO_DEVICE: return "no CUDA device";
    }
    return "unknown status";
}

const char *gs_last_error(void) { return g_last_error; }

gs_status gs_build_bvh(const gs_gaussians *g, gs_bvh **out, void *stream) {
    return gs_build_bvh_ex(g, nullptr, out, stream);
}

gs_status gs_build_bvh_ex(const gs_gaussians *g, const gs_build_options *opt, gs_bvh **out,
                          void *stream) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    const int format = opt ? opt->node_format : GS_NODES_BINARY;
    if (format != GS_NODES_BINARY && format != GS_NODES_WIDE4 && format != GS_NODES_WIDE4_Q8 &&
        format != GS_NODES_BINARY_Q8)
        return fail(GS_ERR_INVALID_ARG, "node_format=%d unknown", format);
    if (opt)
        for (int i = 0; i < 7; ++i)
            if (opt->reserved[i] != 0) return fail(GS_ERR_INVALID_ARG, "reserved options must be zero");
    gs_status st = check_gaussians_host(g, false);
    if (st != GS_OK) return st;
    if ((st = check_device()) != GS_OK) return st;
    if ((st = check_gaussians_device(g, false)) != GS_OK) return st;
    gs_bvh *b = (gs_bvh *)calloc(1, sizeof(gs_bvh));
    if (!b) return fail(GS_ERR_OOM, "host allocation failed");
    cudaGetDevice(&b->device);
    const int64_t M = g->M;
    const int64_t cap = M > 0 ? M : 0;
    const int64_t nn = M > 1 ? M - 1 : 1;
    const int64_t tiles = radix_tiles(cap > 0 ? cap : 1);
    const int64_t scan_n = 256 * tiles > nn ? 256 * tiles : nn;
    const bool q8 = format == GS_NODES_BINARY_Q8;
    const bool wide = format == GS_NODES_WIDE4 || format == GS_NODES_WIDE4_Q8;
    const size_t wide_bytes = format == GS_NODES_WIDE4 ? sizeof(Node4) : sizeof(NodeQ4);
    // the W-wide records of the binary formats (at most one per leaf and
    // one per internal node, plus two header units per wide node in the
    // 8-bit form); offsets must fit 26 bits
    const int64_t recs = q8 ? cap + 3 * nn : cap + nn;
    const size_t rec_bytes = q8 ? sizeof(ChildQ8) : sizeof(ChildRec);
    const bool grouped = !wide && cap > 0 && recs <= (int64_t)kWideOffsetMask;
    b->node_format = format;
    struct Req { void **p; size_t bytes; } reqs[] = {
        {(void **)&b->status, 16},
        {(void **)&b->nodes, (size_t)nn * sizeof(Node)},
        {(void **)&b->prims, (size_t)(cap > 0 ? cap : 1) * sizeof(PrimRec)},
        {(void **)&b->codes[0], (size_t)(cap > 0 ? cap : 1) * 8},
        {(void **)&b->codes[1], (size_t)(cap > 0 ? cap : 1) * 8},
        {(void **)&b->vals[0], (size_t)(cap > 0 ? cap : 1) * 4},
        {(void **)&b->vals[1], (size_t)(cap > 0 ? cap : 1) * 4},
        {(void **)&b->parent, (size_t)(2 * cap + 2) * 4},
        {(void **)&b->arrive, (size_t)(cap > 0 ? cap : 1) * 4},
        {(void **)&b->aabb, (size_t)(cap > 0 ? cap : 1) * 24},
        {(void **)&b->bounds, 64},
        {(void **)&b->hist, (size_t)256 * tiles * 4},
        {(void **)&b->scan_tmp, (size_t)scan_tmp_entries(scan_n) * 4},
        {(void **)&b->wide, wide ? (size_t)nn * wide_bytes : 0},
        {(void **)&b->depth, wide ? (size_t)nn * 4 : 0},
        {(void **)&b->wmap, wide ? (size_t)nn * 4 : 0},
        {(void **)&b->node_depth, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[0].rec, grouped ? (size_t)recs * rec_bytes : 0},
        {(void **)&b->group[0].cnt, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[0].off, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[1].rec, grouped ? (size_t)recs * rec_bytes : 0},
        {(void **)&b->group[1].cnt, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[1].off, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[2].rec, grouped ? (size_t)recs * rec_bytes : 0},
        {(void **)&b->group[2].cnt, grouped ? (size_t)nn * 4 : 0},
        {(void **)&b->group[2].off, grouped ? (size_t)nn * 4 : 0},
    };
    int64_t total = 0;
    for (auto &r : reqs) {
        if (r.bytes == 0) continue;
        cudaError_t e = cudaMalloc(r.p, r.bytes);
        if (e != cudaSuccess) {
            release(b);
            return cuda_fail(e, "cudaMalloc");
        }
        total += (int64_t)r.bytes;
    }
    b->capacity = cap;
    b->hist_len = 256 * tiles;
    b->device_bytes = total;
    cudaError_t e = cudaMemsetAsync(b->status, 0, 16, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        release(b);
        return cuda_fail(e, "memset status");
    }
    st = build_into(b, g, (cudaStream_t)stream);
    if (st != GS_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        release(b);
        return st;
    }
    *out = b;
    return GS_OK;
}

gs_status gs_bvh_rebuild(gs_bvh *b, const gs_gaussians *g, void *stream) {
    if (!b) return fail(GS_ERR_INVALID_ARG, "bvh is NULL");
    gs_status st = check_gaussians_host(g, false);
    if (st != GS_OK) return st;
    if (g->M > b->capacity)
        return fail(GS_ERR_INVALID_ARG, "M=%lld exceeds capacity %lld", (long long)g->M,
                    (long long)b->capacity);
    if ((st = check_gaussians_device(g, false)) != GS_OK) return st;
    return build_into(b, g, (cudaStream_t)stream);
}

gs_status gs_bvh_free(gs_bvh *b) {
    if (!b) return GS_OK;
    cudaDeviceSynchronize();
    release(b);
    return GS_OK;
}

gs_status gs_bvh_get_info(const gs_bvh *b, gs_bvh_info *info) {
    if (!b || !info) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    info->M = b->M;
    info->n_nodes = b->n_nodes;
    info->capacity = b->capacity;
    info->device_bytes = b->device_bytes;
    info->node_bytes = (int32_t)sizeof(Node);
    info->prim_bytes = (int32_t)sizeof(PrimRec);
    info->node_format = b->node_format;
    info->wide_node_bytes = b->node_format == GS_NODES_WIDE4 ? (int32_t)sizeof(Node4)
                            : b->node_format == GS_NODES_WIDE4_Q8 ? (int32_t)sizeof(NodeQ4)
                                                                  : 0;
    return GS_OK;
}

gs_status gs_bvh_export_wide(const gs_bvh *b, void *out, int64_t capacity, int64_t *n_out) {
    if (!b || !n_out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
    if (b->node_format == GS_NODES_BINARY || b->node_format == GS_NODES_BINARY_Q8)
        return fail(GS_ERR_INVALID_ARG, "handle has binary nodes");
    if (capacity < 0) return fail(GS_ERR_INVALID_ARG, "negative capacity");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    *n_out = 0;
    if (b->M == 0) return GS_OK;
    // count = map of the last internal node + its own flag (even depth)
    uint32_t last_map = 0, last_depth = 0;
    const int64_t n_int = b->n_nodes;
    if ((e = cudaMemcpy(&last_map, b->wmap + n_int - 1, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy map");
    if ((e = cudaMemcpy(&last_depth, b->depth + n_int - 1, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy depth");
    const int64_t n = (int64_t)last_map + ((last_depth & 1u) ? 0 : 1);
    *n_out = n;
    const size_t bytes = b->node_format == GS_NODES_WIDE4 ? sizeof(Node4) : sizeof(NodeQ4);
    const int64_t k = n < capacity ? n : capacity;
    if (k > 0 && out &&
        (e = cudaMemcpy(out, b->wide, (size_t)k * bytes, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy wide nodes");
    return GS_OK;
}

gs_status gs_bvh_sync_status(gs_bvh *b, void *stream) {
    if (!b) return fail(GS_ERR_INVALID_ARG, "bvh is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    uint32_t word = 0;
    if ((e = cudaMemcpy(&word, b->status, 4, cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "read status");
    if (word) {
        if ((e = cudaMemset(b->status, 0, 4)) != cudaSuccess) return cuda_fail(e, "clear status");
    }
    if (word & kErrNonfinite) return fail(GS_ERR_NONFINITE, "non-finite Gaussian parameter(s)");
    if (word & kErrStack) return fail(GS_ERR_STACK_OVERFLOW, "a ray overflowed its stack");
    if (word & kErrSteps) return fail(GS_ERR_STEP_LIMIT, "a ray exceeded the step limit");
    if (word & kErrKeys)
        return fail(GS_ERR_INVALID_ARG, "a stored sample key named no Gaussian of the handle");
    return GS_OK;
}

gs_status gs_bvh_export(const gs_bvh *b, void *nodes_out, void *prims_out, uint64_t *codes_out,
                        uint32_t *order_out) {
    if (!b) return fail(GS_ERR_INVALID_ARG, "bvh is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "synchronize");
    if (b->M == 0) return GS_OK;
    if (nodes_out &&
        (e = cudaMemcpy(nodes_out, b->nodes, (size_t)b->n_nodes * sizeof(Node),
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy nodes");
    if (prims_out &&
        (e = cudaMemcpy(prims_out, b->prims, (size_t)b->M * sizeof(PrimRec),
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy prims");
    if (codes_out &&
        (e = cudaMemcpy(codes_out, b->codes[b->final_buf], (size_t)b->M * 8,
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy codes");
    if (order_out &&
        (e = cudaMemcpy(order_out, b->vals[b->final_buf], (size_t)b->M * 4,
                        cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(e, "copy order");
    return GS_OK;
}

static gs_status check_trace_args(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                                  const gs_trace_params *p) {
    if (!b) return fail(GS_ERR_INVALID_ARG, "bvh is NULL");
    gs_status st = check_gaussians_host(g, true);
    if (st != GS_OK) return st;
    if (g->M != b->M)
        return fail(GS_ERR_INVALID_ARG, "gaussians M=%lld differs from the hierarchy's M=%lld",
                    (long long)g->M, (long long)b->M);
    if (!cam || !p) return fail(GS_ERR_INVALID_ARG, "cam or params is NULL");
    if (cam->width < 1 || cam->height < 1 || cam->width > 65536 || cam->height > 65536)
        return fail(GS_ERR_INVALID_ARG, "image size %dx%d out of range", cam->width, cam->height);
    if ((uint64_t)cam->ray_id_offset + (uint64_t)cam->width * (uint64_t)cam->height >
        0x100000000ull)
        return fail(GS_ERR_INVALID_ARG, "ray ids exceed 32 bits");
    if (!(cam->fov_y_deg > 0.0f && cam->fov_y_deg < 180.0f))
        return fail(GS_ERR_INVALID_ARG, "fov_y_deg=%g not in (0, 180)", (double)cam->fov_y_deg);
    for (int i = 0; i < 3; ++i)
        if (!isfinite(cam->eye[i]) || !isfinite(cam->look_at[i]) || !isfinite(cam->up[i]))
            return fail(GS_ERR_INVALID_ARG, "camera vectors must be finite");
    if (p->spp < 1 || p->spp > (1 << 20)) return fail(GS_ERR_INVALID_ARG, "spp=%d out of range", p->spp);
    if (p->n_hits != 1 && p->n_hits != 2 && p->n_hits != 4 && p->n_hits != 8)
        return fail(GS_ERR_INVALID_ARG, "n_hits=%d must be 1, 2, 4 or 8", p->n_hits);
    if ((int64_t)p->spp * p->n_hits > (1ll << 30))
        return fail(GS_ERR_INVALID_ARG, "spp * n_hits too large");
    if (p->stack_depth < 0 || p->stack_depth > kMaxStack)
        return fail(GS_ERR_INVALID_ARG, "stack_depth=%d not in 0..%d", p->stack_depth, kMaxStack);
    if (p->depth_mode != 0 && p->depth_mode != 1)
        return fail(GS_ERR_INVALID_ARG, "depth_mode=%d unsupported", p->depth_mode);
    if (p->rng_mode != 0 && p->rng_mode != 1)
        return fail(GS_ERR_INVALID_ARG, "rng_mode=%d unsupported", p->rng_mode);
    {
        const int S = p->samples_per_lane;
        if (S != 0 && S != 1 && S != 2 && S != 4 && S != 8)
            return fail(GS_ERR_INVALID_ARG, "samples_per_lane=%d must be 0, 1, 2, 4 or 8", S);
        if (S * p->n_hits > 8)
            return fail(GS_ERR_INVALID_ARG, "n_hits * samples_per_lane = %d exceeds 8",
                        S * p->n_hits);
    }
    if (isnan(p->t_min) || isnan(p->t_max) || !(p->t_min < p->t_max))
        return fail(GS_ERR_INVALID_ARG, "need t_min < t_max");
    return GS_OK;
}

// The device-side checks gs_trace_stochastic and gs_trace_stochastic_keys
// share (after check_trace_args and the NULL checks of their outputs).
static gs_status check_trace_outputs(const gs_gaussians *g, const gs_trace_params *p,
                                     float *rgb_out) {
    gs_status st = check_device();
    if (st != GS_OK) return st;
    if ((st = check_gaussians_device(g, true)) != GS_OK) return st;
    if (!is_device_ptr(rgb_out)) return fail(GS_ERR_INVALID_ARG, "rgb_out is not a device pointer");
    if (p->counters && !is_device_ptr(p->counters))
        return fail(GS_ERR_INVALID_ARG, "counters is not a device pointer");
    return GS_OK;
}

// A sample-key array argument: present, on the device, 4-byte aligned.
static gs_status check_keys(const void *keys, const char *name) {
    if (!keys) return fail(GS_ERR_INVALID_ARG, "%s is NULL", name);
    if (((uintptr_t)keys & 3u) != 0) return fail(GS_ERR_INVALID_ARG, "%s is not 4-byte aligned", name);
    if (!is_device_ptr(keys)) return fail(GS_ERR_INVALID_ARG, "%s is not a device pointer", name);
    return GS_OK;
}

gs_status gs_trace_stochastic(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                              const gs_trace_params *p, float *rgb_out, int32_t *hit_id_out,
                              float *hit_t_out, void *stream) {
    gs_status st = check_trace_args(b, g, cam, p);
    if (st != GS_OK) return st;
    if (!rgb_out) return fail(GS_ERR_INVALID_ARG, "rgb_out is NULL");
    if ((hit_id_out == nullptr) != (hit_t_out == nullptr))
        return fail(GS_ERR_INVALID_ARG, "hit_id_out and hit_t_out go together");
    if ((st = check_trace_outputs(g, p, rgb_out)) != GS_OK) return st;
    if (hit_id_out && (!is_device_ptr(hit_id_out) || !is_device_ptr(hit_t_out)))
        return fail(GS_ERR_INVALID_ARG, "hit outputs must be device pointers");
    return launch_trace(b, g, cam, p, rgb_out, hit_id_out, hit_t_out, nullptr,
                        (cudaStream_t)stream);
}

gs_status gs_trace_stochastic_keys(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                                   const gs_trace_params *p, float *rgb_out,
                                   gs_sample_key *keys_out, void *stream) {
    gs_status st = check_trace_args(b, g, cam, p);
    if (st != GS_OK) return st;
    if (!rgb_out) return fail(GS_ERR_INVALID_ARG, "rgb_out is NULL");
    if (!keys_out) return fail(GS_ERR_INVALID_ARG, "keys_out is NULL");
    if ((st = check_trace_outputs(g, p, rgb_out)) != GS_OK) return st;
    if ((st = check_keys(keys_out, "keys_out")) != GS_OK) return st;
    return launch_trace(b, g, cam, p, rgb_out, nullptr, nullptr, keys_out, (cudaStream_t)stream);
}

gs_status gs_trace_layout(const gs_bvh *b, const gs_trace_params *p, int32_t *layout_out) {
    if (!b || !p || !layout_out) return fail(GS_ERR_INVALID_ARG, "bvh, params or layout_out is NULL");
    if (p->spp < 1 || p->spp > (1 << 20)) return fail(GS_ERR_INVALID_ARG, "spp=%d out of range", p->spp);
    if (p->n_hits != 1 && p->n_hits != 2 && p->n_hits != 4 && p->n_hits != 8)
        return fail(GS_ERR_INVALID_ARG, "n_hits=%d must be 1, 2, 4 or 8", p->n_hits);
    const int S0 = p->samples_per_lane;
    if ((S0 != 0 && S0 != 1 && S0 != 2 && S0 != 4 && S0 != 8) || S0 * p->n_hits > 8)
        return fail(GS_ERR_INVALID_ARG, "samples_per_lane=%d invalid for n_hits=%d", S0, p->n_hits);
    int S = 1, spp_eff = 1, lg = 0;
    bool grouped = false;
    trace_layout(b, p, &S, &spp_eff, &lg, &grouped);
    layout_out[0] = S;
    layout_out[1] = 1 << lg;
    layout_out[2] = spp_eff;
    layout_out[3] = grouped ? 1 : 0;
    return GS_OK;
}

// keyed: the caller is gs_trace_backward_keys, which requires keys.
static gs_status backward_common(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                                 const gs_trace_params *p, bool keyed, const gs_sample_key *keys,
                                 const float *d_rgb, float *d_means, float *d_log_scales,
                                 float *d_quats, float *d_opacity_logits, float *d_sh,
                                 void *stream) {
    gs_status st = check_trace_args(b, g, cam, p);
    if (st != GS_OK) return st;
    if (keyed && !keys) return fail(GS_ERR_INVALID_ARG, "keys is NULL");
    if (p->depth_mode != 0 || p->rng_mode != 0)
        return fail(GS_ERR_INVALID_ARG, "gradients need depth_mode 0 and rng_mode 0");
    if (!d_rgb || !d_means || !d_log_scales || !d_quats || !d_opacity_logits || !d_sh)
        return fail(GS_ERR_INVALID_ARG, "d_rgb and every gradient array are required");
    if (((uintptr_t)g->quats & 15u) != 0)
        return fail(GS_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    if ((st = check_device()) != GS_OK) return st;
    if ((st = check_gaussians_device(g, true)) != GS_OK) return st;
    const void *ptrs[6] = {d_rgb, d_means, d_log_scales, d_quats, d_opacity_logits, d_sh};
    for (const void *q : ptrs)
        if (!is_device_ptr(q)) return fail(GS_ERR_INVALID_ARG, "gradient arrays must be device pointers");
    if (keys && (st = check_keys(keys, "keys")) != GS_OK) return st;
    if (b->M == 0) return GS_OK;
    return launch_backward(b, g, cam, p, keys, d_rgb, d_means, d_log_scales, d_quats,
                           d_opacity_logits, d_sh, (cudaStream_t)stream);
}

gs_status gs_trace_backward(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                            const gs_trace_params *p, const float *d_rgb, float *d_means,
                            float *d_log_scales, float *d_quats, float *d_opacity_logits,
                            float *d_sh, void *stream) {
    return backward_common(b, g, cam, p, false, nullptr, d_rgb, d_means, d_log_scales, d_quats,
                           d_opacity_logits, d_sh, stream);
}

gs_status gs_trace_backward_keys(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cam,
                                 const gs_trace_params *p, const gs_sample_key *keys,
                                 const float *d_rgb, float *d_means, float *d_log_scales,
                                 float *d_quats, float *d_opacity_logits, float *d_sh,
                                 void *stream) {
    return backward_common(b, g, cam, p, true, keys, d_rgb, d_means, d_log_scales, d_quats,
                           d_opacity_logits, d_sh, stream);
}

static gs_status check_camera(const gs_pinhole *cam) {
    if (cam->width < 1 || cam->height < 1 || cam->width > 65536 || cam->height > 65536)
        return fail(GS_ERR_INVALID_ARG, "image size %dx%d out of range", cam->width, cam->height);
    if ((uint64_t)cam->ray_id_offset + (uint64_t)cam->width * (uint64_t)cam->height >
        0x100000000ull)
        return fail(GS_ERR_INVALID_ARG, "ray ids exceed 32 bits");
    if (!(cam->fov_y_deg > 0.0f && cam->fov_y_deg < 180.0f))
        return fail(GS_ERR_INVALID_ARG, "fov_y_deg=%g not in (0, 180)", (double)cam->fov_y_deg);
    for (int i = 0; i < 3; ++i)
        if (!isfinite(cam->eye[i]) || !isfinite(cam->look_at[i]) || !isfinite(cam->up[i]))
            return fail(GS_ERR_INVALID_ARG, "camera vectors must be finite");
    return GS_OK;
}

gs_status gs_render_views(const gs_bvh *b, const gs_gaussians *g, const gs_pinhole *cams,
                          int32_t n_views, const gs_scene_extras *ex, const gs_trace_params *p,
                          const gs_launch_options *opt, float *rgb_out,
                          unsigned long long *counters, int32_t *samples_out, void *stream) {
    if (!cams || n_views < 1 || n_views > 32)
        return fail(GS_ERR_INVALID_ARG, "need 1..32 views, got %d", n_views);
    gs_status st = check_trace_args(b, g, &cams[0], p);
    if (st != GS_OK) return st;
    if (p->n_hits != 1) return fail(GS_ERR_INVALID_ARG, "the wavefront form takes n_hits = 1");
    if (p->depth_mode != 0 || p->rng_mode != 0)
        return fail(GS_ERR_INVALID_ARG, "the wavefront form needs depth_mode 0 and rng_mode 0");
    for (int v = 0; v < n_views; ++v)
        if ((st = check_camera(&cams[v])) != GS_OK) return st;
    for (int v = 0; v < n_views; ++v)
        for (int u = v + 1; u < n_views; ++u) {
            const uint64_t a0 = cams[v].ray_id_offset,
                           a1 = a0 + (uint64_t)cams[v].width * cams[v].height;
            const uint64_t b0 = cams[u].ray_id_offset,
                           b1 = b0 + (uint64_t)cams[u].width * cams[u].height;
            if (a0 < b1 && b0 < a1)
                return fail(GS_ERR_INVALID_ARG, "ray ids of views %d and %d overlap", v, u);
        }
    if (ex) {
        if (ex->n_lights < 0 || ex->n_lights > 8) return fail(GS_ERR_INVALID_ARG, "0..8 lights");
        if ((ex->n_lights > 0 || ex->bounce) && !(ex->shadow_eps > 0.0f && isfinite(ex->shadow_eps)))
            return fail(GS_ERR_INVALID_ARG, "shadow_eps must be > 0");
        if (ex->has_ground && !(ex->ground_half_extent >= 0.0f && isfinite(ex->ground_y)))
            return fail(GS_ERR_INVALID_ARG, "bad ground plane");
        for (int l = 0; l < ex->n_lights; ++l)
            for (int i = 0; i < 3; ++i)
                if (!isfinite(ex->lights[l].position[i]) || !isfinite(ex->lights[l].intensity[i]))
                    return fail(GS_ERR_INVALID_ARG, "lights must be finite");
    }
    if (opt) {
        if (opt->block_threads != 0 && opt->block_threads != 64 && opt->block_threads != 128 &&
            opt->block_threads != 256)
            return fail(GS_ERR_INVALID_ARG, "block_threads must be 64, 128 or 256");
        if (opt->stack_entries != 0 && opt->stack_entries != 48 && opt->stack_entries != 96)
            return fail(GS_ERR_INVALID_ARG, "stack_entries must be 48 or 96");
    }
    if (!rgb_out) return fail(GS_ERR_INVALID_ARG, "rgb_out is NULL");
    if ((st = check_device()) != GS_OK) return st;
    if ((st = check_gaussians_device(g, true)) != GS_OK) return st;
    if (!is_device_ptr(rgb_out)) return fail(GS_ERR_INVALID_ARG, "rgb_out is not a device pointer");
    if (counters && !is_device_ptr(counters))
        return fail(GS_ERR_INVALID_ARG, "counters is not a device pointer");
    if (samples_out && !is_device_ptr(samples_out))
        return fail(GS_ERR_INVALID_ARG, "samples_out is not a device pointer");
    return launch_render_views(b, g, cams, n_views, ex, p, opt, rgb_out, counters, samples_out,
                               (cudaStream_t)stream);
}

struct gs_graph {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

gs_status gs_graph_capture_views(gs_bvh *b, const gs_gaussians *g, int32_t rebuild,
                                 const gs_pinhole *cams, int32_t n_views,
                                 const gs_scene_extras *ex, const gs_trace_params *p,
                                 const gs_launch_options *opt, float *rgb_out, void *stream,
                                 gs_graph **out) {
    if (!out) return fail(GS_ERR_INVALID_ARG, "out is NULL");
    if (!stream) return fail(GS_ERR_INVALID_ARG, "capture needs a non-default stream");
    if (rebuild) {
        gs_status st = check_gaussians_host(g, false);
        if (st != GS_OK) return st;
        if (!b || g->M > b->capacity) return fail(GS_ERR_INVALID_ARG, "rebuild exceeds capacity");
    }
    cudaStream_t s = (cudaStream_t)stream;
    // the deferred bounce's scratch cannot be allocated inside a capture
    if (b && cams && n_views >= 1 && n_views <= 32 && p) {
        const int64_t slots = wave_slots(cams, n_views, ex, p);
        if (slots > 0) {
            gs_status st = reserve_wave_scratch(b, slots, s);
            if (st != GS_OK) return st;
        }
    }
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(e, "begin capture");
    gs_status st = GS_OK;
    if (rebuild) {
        b->M = g->M;
        st = build_into(b, g, s);
    }
    if (st == GS_OK)
        st = gs_render_views(b, g, cams, n_views, ex, p, opt, rgb_out, nullptr, nullptr, stream);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(s, &graph);
    if (st != GS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "end capture");
    cudaGraphExec_t exec = nullptr;
    if ((e = cudaGraphInstantiate(&exec, graph, 0)) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return cuda_fail(e, "instantiate graph");
    }
    gs_graph *gr = (gs_graph *)calloc(1, sizeof(gs_graph));
    if (!gr) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return fail(GS_ERR_OOM, "host allocation failed");
    }
    gr->graph = graph;
    gr->exec = exec;
    *out = gr;
    return GS_OK;
}

gs_status gs_graph_launch(gs_graph *gr, void *stream) {
    if (!gr) return fail(GS_ERR_INVALID_ARG, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(gr->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "graph launch");
    return GS_OK;
}

gs_status gs_graph_free(gs_graph *gr) {
    if (!gr) return GS_OK;
    cudaGraphExecDestroy(gr->exec);
    cudaGraphDestroy(gr->graph);
    free(gr);
    return GS_OK;
}

}  // extern "C"
