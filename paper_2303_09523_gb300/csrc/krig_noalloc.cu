// krig_noalloc.cu -- krig_interpolate_noalloc: the DS interpolation of one
// volume without any device allocation by the caller or by the library.
//
// Who needs it: code that may not call cudaMalloc at all -- plugins hosted by
// an application that owns every device byte through its own memory pool,
// real-time pipelines that cannot afford cudaMalloc's implicit device-wide
// synchronisation in their frame loop, or services that run under a fixed
// device-memory budget enforced outside the library.  Such callers cannot
// provide the workspace that krig_plan_set_workspace expects.
//
// Instead the scratch (device status word, per-class weight and variance
// tables) lives in one file-scope __device__ array of KRIG_NOALLOC_SCRATCH_BYTES
// that every GPU loading the library keeps until the process exits.  Host code
// cannot pass that array's name to a kernel (on the host it only names a
// host-side stand-in), so the device address is looked up once per device with
// cudaGetSymbolAddress and cached.  The cache outlives the device's primary
// context: after cudaDeviceReset the module is loaded again at another
// address, so this entry point must not be called on that device again in
// the same process.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "krig_internal.h"

#define KRIG_NOALLOC_SCRATCH_BYTES (64 * 1024)
#define KRIG_NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) unsigned char g_krig_noalloc_scratch[KRIG_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_noalloc_mu;
void* g_noalloc_addr[KRIG_NOALLOC_MAX_DEVICES];

krig_status noalloc_fail(krig_status st, const std::string& msg)
{
    krig_internal_set_error(msg.c_str());  // reported by krig_last_error()
    return st;
}

// Device address of the static scratch on the current device (set-up on the
// first call per device).
krig_status noalloc_scratch(void** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(KRIG_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= KRIG_NOALLOC_MAX_DEVICES) return noalloc_fail(KRIG_EUNSUPPORTED, "device index too large");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_krig_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return noalloc_fail(KRIG_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return KRIG_OK;
}

}  // namespace

extern "C" krig_status krig_interpolate_noalloc(const krig_volume_desc* desc, const void* d_slices, void* d_out,
                                                float* d_var, const krig_variogram* d_params, int32_t check_status,
                                                void* stream)
{
    if (!desc || !d_slices || !d_out || !d_params)
        return noalloc_fail(KRIG_EINVAL, "desc, d_slices, d_out and d_params must not be NULL");
    const krig_volume_desc& d = *desc;
    krig_status chk = krig_internal_check_desc(d, 0);  // the same limits as krig_plan_create
    if (chk != KRIG_OK) return chk;
    if ((uintptr_t)d_slices % 16 || (uintptr_t)d_out % 16 || (d_var && (uintptr_t)d_var % 16))
        return noalloc_fail(KRIG_EINVAL, "slice, output and variance buffers must be 16-byte aligned");

    // The kernel parameter block is built on the stack.
    static_assert(sizeof(KrigLaunch) < 64 * 1024, "launch block too large for the stack");
    KrigLaunch L;
    memset(&L, 0, sizeof(L));
    L.n_vols = 1;
    L.form = KRIG_FORM_DS;
    KrigVol& V = L.vol[0];
    int64_t need = 256, items = 0, classes = 0, vox = 0, frames = 0;
    krig_fill_vol(V, d, KRIG_FORM_DS, krig_pick_chunk(&d, 1), &need, &items, &classes, &vox, &frames);
    L.n_frame_units = frames;
    if (need > KRIG_NOALLOC_SCRATCH_BYTES)
        return noalloc_fail(KRIG_EINVAL, "this volume needs " + std::to_string((long long)need) +
                                             " bytes of scratch; the static scratch holds " +
                                             std::to_string(KRIG_NOALLOC_SCRATCH_BYTES) +
                                             " (use krig_plan_create with a caller workspace instead)");
    L.n_items = items;
    L.n_classes = classes;
    L.n_vox = vox;
    krig_ds_order(L);

    void* scratch = nullptr;
    krig_status st = noalloc_scratch(&scratch);
    if (st != KRIG_OK) return st;
    L.ws = (unsigned char*)scratch;
    L.status = (uint32_t*)scratch;
    L.in[0] = d_slices;
    L.out[0] = d_out;
    L.var[0] = d_var;
    L.vg = d_params;

    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(scratch, 0, 256, s);  // the status word must start at zero
    if (e != cudaSuccess) return noalloc_fail(KRIG_ECUDA, std::string("clearing the status word: ") + cudaGetErrorString(e));
    int err = krig_launch_ds_solve(L, 0, s);
    if (err) return noalloc_fail(KRIG_ECUDA, std::string("class solve launch: ") + cudaGetErrorString((cudaError_t)err));
    DsTma tma;  // host-side encoding of the slice pointer, passed by value to the kernel
    memset(&tma, 0, sizeof(tma));
    tma.valid[0] = krig_encode_ds_tma(V, d_slices, &tma.tm[0]) == 0 ? 1 : 0;
    err = krig_launch_ds_apply(L, tma, s);
    if (err) return noalloc_fail(KRIG_ECUDA, std::string("stencil launch: ") + cudaGetErrorString((cudaError_t)err));
    if (check_status) {
        uint32_t bits = 0;
        e = cudaMemcpyAsync(&bits, scratch, sizeof(bits), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return noalloc_fail(KRIG_ECUDA, std::string("reading the status word: ") + cudaGetErrorString(e));
        if (bits & KRIG_DEV_SINGULAR) return noalloc_fail(KRIG_ESINGULAR, "a kriging system was singular");
        // a stencil wait that gave up left part of the output unwritten
        if (bits & KRIG_DEV_TIMEOUT) return noalloc_fail(KRIG_ETIMEOUT, "a device-side wait timed out");
    }
    return KRIG_OK;
}
