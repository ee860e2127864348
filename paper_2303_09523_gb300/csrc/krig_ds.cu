// krig_ds.cu -- launcher of the DS stencil apply (one kernel per input type
// present in the plan) and device queries.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "krig_internal.h"

int krig_launch_ds_apply_f32(const KrigLaunch& L, const DsTma& T, void* stream);
int krig_launch_ds_apply_u16(const KrigLaunch& L, const DsTma& T, void* stream);
int krig_launch_ds_apply_f64(const KrigLaunch& L, const DsTma& T, void* stream);

int krig_launch_ds_apply(const KrigLaunch& L, const DsTma& T, void* stream)
{
    if (L.n_items == 0) return 0;
    int e = krig_launch_ds_apply_f32(L, T, stream);
    if (e == 0) e = krig_launch_ds_apply_u16(L, T, stream);
    if (e == 0) e = krig_launch_ds_apply_f64(L, T, stream);
    return e;
}

static PFN_cuTensorMapEncodeTiled_v12000 tma_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    });
    return fn;
}

int krig_encode_ds_tma(const KrigVol& V, const void* ptr, CUtensorMap* out)
{
    const int esz = V.dtype == KRIG_F64 ? 8 : V.dtype == KRIG_F32 ? 4 : 2;
    if (((int64_t)V.W * esz) % 16 != 0 || ((uintptr_t)ptr % 16) != 0) return 1;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tma_encoder();
    if (!enc) return 2;
    // box: the tile's row span (shared-memory row pitch) x (tile rows + 2r) x 1 slice
    const int rp = V.dtype == KRIG_F64 ? 72 : V.dtype == KRIG_F32 ? 80 : 96;
    const CUtensorMapDataType dt = V.dtype == KRIG_F64   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                   : V.dtype == KRIG_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                         : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)V.W, (cuuint64_t)V.H, (cuuint64_t)V.n};
    const cuuint64_t strides[2] = {(cuuint64_t)V.W * esz, (cuuint64_t)V.W * V.H * esz};
    const cuuint32_t box[3] = {(cuuint32_t)rp, (cuuint32_t)(KRIG_TY + 2 * V.r), 1u};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(out, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : 3;
}

int krig_device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}
