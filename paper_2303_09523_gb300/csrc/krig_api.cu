// krig_api.cu -- host side of the C ABI declared in include/krig.h: plan
// creation (Algorithm 1 partition into Z sub-blocks and in-plane tiles,
// geometry-class enumeration, workspace layout), argument checking, kernel
// launches, device status and timing.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "krig_internal.h"

namespace {

thread_local std::string g_last_error;

krig_status fail(krig_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
krig_status fail(krig_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

krig_status cuda_fail(int err, const char* what)
{
    return fail(KRIG_ECUDA, "%s: %s", what, cudaGetErrorString((cudaError_t)err));
}

}  // namespace

void krig_internal_set_error(const char* msg) { g_last_error = msg ? msg : ""; }

namespace {

struct Timing {
    cudaEvent_t a, b;
    int kind;
};

}  // namespace

static_assert(sizeof(KrigLaunch) <= 32000, "kernel parameter block exceeds the 32 KB parameter limit");

struct krig_plan_s {
    std::vector<krig_volume_desc> desc;
    KrigLaunch L;
    int form = KRIG_FORM_DS;
    uint32_t flags = 0;
    int64_t ws_bytes = 0;
    unsigned char* ws = nullptr;
    int timing = 0;
    std::vector<Timing> pending;
    std::vector<cudaEvent_t> pool;
    DsTma tma;                              // tensor maps of the last call's slice pointers
    const void* tma_ptr[KRIG_TMA_VOLS] = {};
    double ms[KRIG_TIMING_KINDS] = {0, 0, 0, 0};
    int64_t launches[KRIG_TIMING_KINDS] = {0, 0, 0, 0};
};

// Descriptor limits of include/krig.h, shared by krig_plan_create and
// krig_interpolate_noalloc (declared in krig_internal.h).
krig_status krig_internal_check_desc(const krig_volume_desc& d, int i)
{
    if (d.H < 1 || d.H > 65536 || d.W < 1 || d.W > 65536)
        return fail(KRIG_EINVAL, "volume %d: H, W must be in [1, 65536] (got %d x %d)", i, d.H, d.W);
    if (d.n_known < 2 || d.n_known > 65536)
        return fail(KRIG_EINVAL, "volume %d: n_known must be in [2, 65536] (got %d)", i, d.n_known);
    if (d.zfactor < 1 || d.zfactor > KRIG_GMAX)
        return fail(KRIG_EINVAL, "volume %d: zfactor must be in [1, %d] (got %d)", i, KRIG_GMAX, d.zfactor);
    if (d.n_sub_blocks < 1 || d.n_sub_blocks > d.n_known - 1)
        return fail(KRIG_EINVAL, "volume %d: n_sub_blocks must be in [1, n_known-1] (got %d)", i, d.n_sub_blocks);
    if (d.half_w < 0 || d.half_w > KRIG_RMAX)
        return fail(KRIG_EUNSUPPORTED, "volume %d: half_w must be in [0, %d] (got %d)", i, KRIG_RMAX, d.half_w);
    if (d.in_dtype != KRIG_F64 && d.in_dtype != KRIG_F32 && d.in_dtype != KRIG_U16)
        return fail(KRIG_EINVAL, "volume %d: unknown in_dtype %d", i, d.in_dtype);
    if (d.in_dtype == KRIG_U16 && !(d.in_scale > 0.0f && d.in_scale < 3.0e38f))
        return fail(KRIG_EINVAL, "volume %d: in_scale must be finite and > 0", i);
    return KRIG_OK;
}

static krig_status record(krig_plan_t plan, cudaStream_t st, cudaEvent_t* ev)
{
    if (!plan->timing) return KRIG_OK;
    if (plan->pool.empty()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return fail(KRIG_ECUDA, "cudaEventCreate failed");
        plan->pool.push_back(e);
    }
    *ev = plan->pool.back();
    plan->pool.pop_back();
    if (cudaEventRecord(*ev, st) != cudaSuccess) return fail(KRIG_ECUDA, "cudaEventRecord failed");
    return KRIG_OK;
}

template <typename F>
static krig_status timed_launch(krig_plan_t plan, cudaStream_t st, int kind, F&& launch, const char* what)
{
    Timing t{nullptr, nullptr, kind};
    krig_status s = record(plan, st, &t.a);
    if (s != KRIG_OK) return s;
    int err = launch();
    if (err != 0) return cuda_fail(err, what);
    s = record(plan, st, &t.b);
    if (s != KRIG_OK) return s;
    if (plan->timing) plan->pending.push_back(t);
    return KRIG_OK;
}

extern "C" {

int32_t krig_version(void) { return 100; }

const char* krig_last_error(void) { return g_last_error.c_str(); }

krig_status krig_plan_create(krig_plan_t* plan, const krig_volume_desc* vols, int32_t n_vols, krig_form form,
                             uint32_t flags, size_t* workspace_bytes_out)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    *plan = nullptr;
    if (!vols) return fail(KRIG_EINVAL, "vols is NULL");
    if (n_vols < 1 || n_vols > KRIG_MAX_VOLUMES)
        return fail(KRIG_EINVAL, "n_vols must be in [1, %d] (got %d)", KRIG_MAX_VOLUMES, n_vols);
    if (form != KRIG_FORM_P64 && form != KRIG_FORM_PMX && form != KRIG_FORM_DS)
        return fail(KRIG_EINVAL, "unknown form %d", (int)form);
    const uint32_t known_flags = KRIG_FLAG_DS_FP64_SOLVE | KRIG_FLAG_FAULT_TIMEOUT | KRIG_FLAG_LOO | KRIG_FLAG_DRIFT_Z |
                                 KRIG_FLAG_DRIFT_XYZ | KRIG_FLAG_SLABS4 | KRIG_FLAG_CLAMP_BLOCK_MINMAX;
    if (flags & ~known_flags) return fail(KRIG_EINVAL, "unknown flag bits 0x%x", flags & ~known_flags);
    if ((flags & KRIG_FLAG_CLAMP_BLOCK_MINMAX) &&
        (form != KRIG_FORM_DS || (flags & (KRIG_FLAG_DRIFT_Z | KRIG_FLAG_DRIFT_XYZ | KRIG_FLAG_SLABS4))))
        return fail(KRIG_EUNSUPPORTED, "KRIG_FLAG_CLAMP_BLOCK_MINMAX applies to the DS form without drift flags");
    const uint32_t uk_flags = KRIG_FLAG_DRIFT_Z | KRIG_FLAG_DRIFT_XYZ | KRIG_FLAG_SLABS4;
    if (flags & uk_flags) {
        if ((flags & KRIG_FLAG_DRIFT_Z) && (flags & KRIG_FLAG_DRIFT_XYZ))
            return fail(KRIG_EINVAL, "KRIG_FLAG_DRIFT_Z and KRIG_FLAG_DRIFT_XYZ exclude each other");
        if (form != KRIG_FORM_DS) return fail(KRIG_EUNSUPPORTED, "universal kriging needs the DS form");
        if (flags & (KRIG_FLAG_LOO | KRIG_FLAG_DS_FP64_SOLVE | KRIG_FLAG_FAULT_TIMEOUT))
            return fail(KRIG_EUNSUPPORTED, "universal kriging plans take no LOO, FP64-solve or test flag");
        for (int i = 0; i < n_vols; ++i)
            if ((flags & KRIG_FLAG_DRIFT_XYZ) && (vols[i].half_w < 1 || vols[i].H < 2 || vols[i].W < 2))
                return fail(KRIG_EUNSUPPORTED,
                            "volume %d: the drift {1, x, y, z} needs half_w >= 1 and H, W >= 2 (else x or y is "
                            "constant over the window)", i);
    }
    for (int i = 0; i < n_vols; ++i) {
        krig_status st = krig_internal_check_desc(vols[i], i);
        if (st != KRIG_OK) return st;
        if ((flags & KRIG_FLAG_LOO) && vols[i].n_known < 3)
            return fail(KRIG_EINVAL, "volume %d: leave-one-slice-out needs n_known >= 3", i);
    }
    if ((flags & KRIG_FLAG_LOO) && form != KRIG_FORM_DS)
        return fail(KRIG_EUNSUPPORTED, "KRIG_FLAG_LOO needs the DS form");
    krig_plan_s* p = new (std::nothrow) krig_plan_s();
    if (!p) return fail(KRIG_ENOMEM, "out of host memory");
    memset(&p->tma, 0, sizeof(p->tma));
    p->desc.assign(vols, vols + n_vols);
    p->form = form;
    p->flags = flags;
    KrigLaunch& L = p->L;
    memset(&L, 0, sizeof(L));
    L.n_vols = n_vols;
    L.form = form;
    L.fault_timeout = (flags & KRIG_FLAG_FAULT_TIMEOUT) ? 1 : 0;
    int64_t off = 256;  // control block: status word
    int64_t items = 0, classes = 0, vox = 0, frames = 0;
    const int chunk = krig_pick_chunk(vols, n_vols);
    for (int i = 0; i < n_vols; ++i)
        krig_fill_vol(L.vol[i], vols[i], form, chunk, &off, &items, &classes, &vox, &frames);
    L.n_frame_units = frames;
    if (flags & KRIG_FLAG_LOO) {
        int64_t lc = 0, li = 0, la = 0;
        for (int i = 0; i < n_vols; ++i) krig_fill_loo(L.vol[i], &off, &lc, &li, &la);
        L.n_loo_classes = lc;
        L.n_loo_items = li;
        L.n_loo_adj = la;
    }
    if (flags & KRIG_FLAG_CLAMP_BLOCK_MINMAX) {
        L.clamp = 1;
        for (int i = 0; i < n_vols; ++i) {
            L.vol[i].mm_off = off;
            off = (off + 2LL * L.vol[i].k * (L.vol[i].dtype == KRIG_F64 ? 8 : 4) + 255) / 256 * 256;
            L.n_mm_blocks += L.vol[i].k;
        }
    }
    if (flags & (KRIG_FLAG_DRIFT_Z | KRIG_FLAG_DRIFT_XYZ | KRIG_FLAG_SLABS4)) {
        L.uk_drift = (flags & KRIG_FLAG_DRIFT_XYZ) ? 2 : ((flags & KRIG_FLAG_DRIFT_Z) ? 1 : 0);
        L.uk_slabs = (flags & KRIG_FLAG_SLABS4) ? 4 : 2;
        int64_t uc = 0, ui = 0;
        for (int i = 0; i < n_vols; ++i) krig_fill_uk(L.vol[i], L.uk_slabs, &off, &uc, &ui);
        L.n_uk_classes = uc;
        L.n_uk_items = ui;
    }
    L.n_items = items;
    L.n_classes = classes;
    L.n_vox = vox;
    krig_ds_order(L);
    p->ws_bytes = off;
    if (workspace_bytes_out) *workspace_bytes_out = (size_t)off;
    *plan = p;
    return KRIG_OK;
}

krig_status krig_plan_set_workspace(krig_plan_t plan, void* d_workspace, size_t bytes)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (!d_workspace) return fail(KRIG_EWORKSPACE, "workspace is NULL");
    if ((uintptr_t)d_workspace % 256 != 0) return fail(KRIG_EWORKSPACE, "workspace must be 256-byte aligned");
    if ((int64_t)bytes < plan->ws_bytes)
        return fail(KRIG_EWORKSPACE, "workspace too small: %zu bytes, plan needs %lld", bytes,
                    (long long)plan->ws_bytes);
    cudaError_t e = cudaMemset(d_workspace, 0, 256);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the workspace control block");
    if (plan->flags & KRIG_FLAG_LOO) {
        // no LOO weights solved yet: the recorded variogram reads as NaN (matches nothing)
        for (int v = 0; v < plan->L.n_vols; ++v) {
            e = cudaMemset((unsigned char*)d_workspace + plan->L.vol[v].lvg_off, 0xff, sizeof(krig_variogram));
            if (e != cudaSuccess) return cuda_fail(e, "initialising the LOO variogram record");
        }
    }
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e, "clearing the workspace control block");
    plan->ws = (unsigned char*)d_workspace;
    plan->L.ws = plan->ws;
    plan->L.status = (uint32_t*)plan->ws;
    return KRIG_OK;
}

krig_status krig_interpolate(krig_plan_t plan, const void* const* d_slices, void* const* d_out, float* const* d_var,
                             const krig_variogram* d_params, void* stream)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (!plan->ws) return fail(KRIG_EWORKSPACE, "no workspace set (krig_plan_set_workspace)");
    if (!d_slices || !d_out) return fail(KRIG_EINVAL, "d_slices / d_out is NULL");
    if (!d_params) return fail(KRIG_EINVAL, "d_params is NULL");
    KrigLaunch& L = plan->L;
    for (int v = 0; v < L.n_vols; ++v) {
        if (!d_slices[v] || !d_out[v]) return fail(KRIG_EINVAL, "volume %d: null slice or output pointer", v);
        if ((uintptr_t)d_slices[v] % 16 || (uintptr_t)d_out[v] % 16)
            return fail(KRIG_EINVAL, "volume %d: slice and output buffers must be 16-byte aligned", v);
        if (d_var && d_var[v] && (uintptr_t)d_var[v] % 16)
            return fail(KRIG_EINVAL, "volume %d: variance buffer must be 16-byte aligned", v);
        L.in[v] = d_slices[v];
        L.out[v] = d_out[v];
        L.var[v] = d_var ? d_var[v] : nullptr;
    }
    L.vg = d_params;
    cudaStream_t st = (cudaStream_t)stream;
    if (L.uk_slabs) {
        krig_status s = timed_launch(plan, st, 0, [&] { return krig_launch_uk(L, st); }, "universal kriging launch");
        if (s != KRIG_OK) return s;
    } else if (plan->form == KRIG_FORM_DS) {
        const int fp64 = (plan->flags & KRIG_FLAG_DS_FP64_SOLVE) ? 1 : 0;
        if (L.clamp) {
            krig_status s = timed_launch(plan, st, 0, [&] { return krig_launch_block_minmax(L, st); },
                                         "block min/max launch");
            if (s != KRIG_OK) return s;
        }
        krig_status s = timed_launch(plan, st, 0, [&] { return krig_launch_ds_solve(L, fp64, st); }, "class solve launch");
        if (s != KRIG_OK) return s;
        for (int v = 0; v < L.n_vols && v < KRIG_TMA_VOLS; ++v) {
            if (plan->tma_ptr[v] != L.in[v]) {
                plan->tma.valid[v] = krig_encode_ds_tma(L.vol[v], L.in[v], &plan->tma.tm[v]) == 0 ? 1 : 0;
                plan->tma_ptr[v] = L.in[v];
            }
        }
        s = timed_launch(plan, st, 1, [&] { return krig_launch_ds_apply(L, plan->tma, st); }, "stencil launch");
        if (s != KRIG_OK) return s;
    } else {
        krig_status s = timed_launch(plan, st, 0, [&] { return krig_launch_voxel(L, plan->form, st); }, "voxel solve launch");
        if (s != KRIG_OK) return s;
    }
    return KRIG_OK;
}

static krig_status loo_common(krig_plan_t plan, const void* const* d_slices, const krig_variogram* d_params)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (!(plan->flags & KRIG_FLAG_LOO)) return fail(KRIG_EUNSUPPORTED, "plan was created without KRIG_FLAG_LOO");
    if (!plan->ws) return fail(KRIG_EWORKSPACE, "no workspace set (krig_plan_set_workspace)");
    if (!d_slices || !d_params) return fail(KRIG_EINVAL, "d_slices / d_params is NULL");
    KrigLaunch& L = plan->L;
    for (int v = 0; v < L.n_vols; ++v) {
        if (!d_slices[v]) return fail(KRIG_EINVAL, "volume %d: null slice pointer", v);
        if ((uintptr_t)d_slices[v] % 16) return fail(KRIG_EINVAL, "volume %d: slices must be 16-byte aligned", v);
        L.in[v] = d_slices[v];
        L.pred[v] = nullptr;
        L.grad_slices[v] = nullptr;
    }
    L.vg = d_params;
    return KRIG_OK;
}

krig_status krig_loo_forward(krig_plan_t plan, const void* const* d_slices, const krig_variogram* d_params,
                             float* const* d_pred, double* d_loss, void* stream)
{
    krig_status s = loo_common(plan, d_slices, d_params);
    if (s != KRIG_OK) return s;
    if (!d_loss) return fail(KRIG_EINVAL, "d_loss is NULL");
    KrigLaunch& L = plan->L;
    for (int v = 0; v < L.n_vols; ++v) L.pred[v] = d_pred ? d_pred[v] : nullptr;
    L.loss = d_loss;
    L.grad_loss = nullptr;
    L.grad_params = nullptr;
    L.accumulate = 0;
    cudaStream_t st = (cudaStream_t)stream;
    return timed_launch(plan, st, 2, [&] { return krig_launch_loo(L, 0, 0, 0, st); }, "loo forward launch");
}

krig_status krig_backward(krig_plan_t plan, const void* const* d_slices, const krig_variogram* d_params,
                          const double* d_grad_loss, float* const* d_grad_slices, double* d_grad_params,
                          int32_t accumulate, void* stream)
{
    krig_status s = loo_common(plan, d_slices, d_params);
    if (s != KRIG_OK) return s;
    if (!d_grad_loss) return fail(KRIG_EINVAL, "d_grad_loss is NULL");
    KrigLaunch& L = plan->L;
    int want_slices = 0;
    for (int v = 0; v < L.n_vols; ++v) {
        L.grad_slices[v] = d_grad_slices ? d_grad_slices[v] : nullptr;
        want_slices |= L.grad_slices[v] != nullptr;
    }
    L.grad_loss = d_grad_loss;
    L.grad_params = d_grad_params;
    L.loss = nullptr;
    L.accumulate = accumulate ? 1 : 0;
    cudaStream_t st = (cudaStream_t)stream;
    // d_grad_params is cleared (unless accumulating) by the first launch of the pass
    return timed_launch(plan, st, 3, [&] { return krig_launch_loo(L, 1, want_slices, d_grad_params != nullptr, st); },
                        "backward launch");
}

// Re-cut every volume's sub-blocks into work items of `chunk` gaps (the
// workspace layout does not depend on it).
static void set_chunk(krig_plan_t plan, int chunk)
{
    KrigLaunch& L = plan->L;
    for (int v = 0; v < L.n_vols; ++v) {
        KrigVol& V = L.vol[v];
        const int max_block = (V.n - 1 + V.k - 1) / V.k;
        V.chunk = chunk < 1 ? 1 : (chunk > max_block ? max_block : chunk);
        V.chunks = (max_block + V.chunk - 1) / V.chunk;
        V.mdiv_chunks = krig_udiv_magic((uint32_t)V.chunks);
    }
    krig_ds_order(L);
}

krig_status krig_plan_autotune(krig_plan_t plan, const void* const* d_slices, void* const* d_out,
                               const krig_variogram* d_params, int32_t iters, void* stream, int32_t* chunk_out)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (plan->form != KRIG_FORM_DS) return fail(KRIG_EUNSUPPORTED, "autotuning applies to the DS form");
    if (iters < 1) iters = 1;
    cudaStream_t st = (cudaStream_t)stream;
    int max_block = 1;
    for (int v = 0; v < plan->L.n_vols; ++v) {
        const KrigVol& V = plan->L.vol[v];
        max_block = std::max(max_block, (V.n - 1 + V.k - 1) / V.k);
    }
    const int cand[] = {1, 2, 3, 4, 6, 8, 12, 16, 1 << 20};
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess)
        return fail(KRIG_ECUDA, "cudaEventCreate failed");
    const int saved_timing = plan->timing;
    plan->timing = 0;
    int best = plan->L.vol[0].chunk, best_bps = plan->L.ds_blocks_per_sm, last = -1;
    float best_ms = 1e30f;
    krig_status s = KRIG_OK;
    for (int c : cand) {
        const int eff = std::min(c, max_block);
        if (eff == last) continue;
        last = eff;
        set_chunk(plan, eff);
        // launch shape: as many stencil blocks per SM as fit, or one
        for (int bps = 0; bps <= 1 && s == KRIG_OK; ++bps) {
            plan->L.ds_blocks_per_sm = bps;
            s = krig_interpolate(plan, d_slices, d_out, nullptr, d_params, stream);  // warm-up
            if (s != KRIG_OK) break;
            cudaEventRecord(a, st);
            for (int i = 0; i < iters && s == KRIG_OK; ++i)
                s = krig_interpolate(plan, d_slices, d_out, nullptr, d_params, stream);
            cudaEventRecord(b, st);
            if (s != KRIG_OK) break;
            if (cudaEventSynchronize(b) != cudaSuccess) {
                s = fail(KRIG_ECUDA, "autotune timing failed");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            if (ms < best_ms) {
                best_ms = ms;
                best = eff;
                best_bps = bps;
            }
        }
        if (s != KRIG_OK) break;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    plan->timing = saved_timing;
    set_chunk(plan, best);
    plan->L.ds_blocks_per_sm = best_bps;
    if (chunk_out) *chunk_out = best;
    return s;
}

krig_status krig_plan_set_schedule(krig_plan_t plan, int32_t chunk, int32_t blocks_per_sm)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (plan->form != KRIG_FORM_DS) return fail(KRIG_EUNSUPPORTED, "the schedule applies to the DS form");
    if (chunk < 1 || blocks_per_sm < 0) return fail(KRIG_EINVAL, "chunk must be >= 1 and blocks_per_sm >= 0");
    set_chunk(plan, chunk);
    plan->L.ds_blocks_per_sm = blocks_per_sm;
    return KRIG_OK;
}

krig_status krig_plan_schedule(krig_plan_t plan, int32_t* chunk_out, int32_t* blocks_per_sm_out)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (chunk_out) *chunk_out = plan->L.vol[0].chunk;
    if (blocks_per_sm_out) *blocks_per_sm_out = plan->L.ds_blocks_per_sm;
    return KRIG_OK;
}

krig_status krig_plan_device_status(krig_plan_t plan, void* stream)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (!plan->ws) return fail(KRIG_EWORKSPACE, "no workspace set");
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "stream synchronize");
    uint32_t bits = 0;
    e = cudaMemcpy(&bits, plan->ws, sizeof(bits), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the device status");
    if (bits) {
        e = cudaMemset(plan->ws, 0, sizeof(bits));
        if (e != cudaSuccess) return cuda_fail(e, "clearing the device status");
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "clearing the device status");
    }
    if (bits & KRIG_DEV_SINGULAR) return fail(KRIG_ESINGULAR, "a kriging system was singular (check nugget + sill > 0)");
    if (bits & KRIG_DEV_TIMEOUT) return fail(KRIG_ETIMEOUT, "a device-side wait timed out");
    return KRIG_OK;
}

krig_status krig_plan_set_timing(krig_plan_t plan, int32_t enable)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    plan->timing = enable ? 1 : 0;
    return KRIG_OK;
}

krig_status krig_plan_get_timing(krig_plan_t plan, double* ms_out, int64_t* launches_out)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    for (Timing& t : plan->pending) {
        cudaError_t e = cudaEventSynchronize(t.b);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t.a, t.b);
        if (e != cudaSuccess) return cuda_fail(e, "reading timing events");
        plan->ms[t.kind] += ms;
        plan->launches[t.kind] += 1;
        plan->pool.push_back(t.a);
        plan->pool.push_back(t.b);
    }
    plan->pending.clear();
    for (int k = 0; k < KRIG_TIMING_KINDS; ++k) {
        if (ms_out) ms_out[k] = plan->ms[k];
        if (launches_out) launches_out[k] = plan->launches[k];
        plan->ms[k] = 0;
        plan->launches[k] = 0;
    }
    return KRIG_OK;
}

krig_status krig_plan_variance_table(krig_plan_t plan, int32_t v, float* h_table, int32_t* h_cx, int32_t* h_cy,
                                     int32_t* ncx_out, int32_t* ncy_out, void* stream)
{
    if (!plan) return fail(KRIG_EINVAL, "plan is NULL");
    if (plan->form != KRIG_FORM_DS || plan->L.uk_slabs)
        return fail(KRIG_EUNSUPPORTED, "the variance class table belongs to DS plans without drift flags");
    if (!plan->ws) return fail(KRIG_EWORKSPACE, "no workspace set");
    if (v < 0 || v >= plan->L.n_vols) return fail(KRIG_EINVAL, "volume index %d out of range", v);
    const KrigVol& V = plan->L.vol[v];
    if (ncx_out) *ncx_out = V.ncx;
    if (ncy_out) *ncy_out = V.ncy;
    // class of each coordinate: the truncation slot of its window, mapped to the compact class
    if (h_cx)
        for (int x = 0; x < V.W; ++x) {
            const int l = x < V.r ? x : V.r, rr = (V.W - 1 - x) < V.r ? (V.W - 1 - x) : V.r;
            h_cx[x] = V.xmap[l * (V.r + 1) + rr];
        }
    if (h_cy)
        for (int y = 0; y < V.H; ++y) {
            const int l = y < V.r ? y : V.r, rr = (V.H - 1 - y) < V.r ? (V.H - 1 - y) : V.r;
            h_cy[y] = V.ymap[l * (V.r + 1) + rr];
        }
    if (h_table) {
        cudaStream_t st = (cudaStream_t)stream;
        cudaError_t e = cudaMemcpyAsync(h_table, plan->ws + V.vtab_off, (size_t)krig_vtab_bytes(V),
                                        cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "reading the variance table");
    }
    return KRIG_OK;
}

void krig_plan_destroy(krig_plan_t plan)
{
    if (!plan) return;
    for (Timing& t : plan->pending) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (cudaEvent_t e : plan->pool) cudaEventDestroy(e);
    delete plan;
}

}  // extern "C"
