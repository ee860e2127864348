// krig_ds.cu -- launcher of the DS stencil apply (one kernel per input type
// present in the plan) and device queries.
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "krig_internal.h"

int krig_launch_ds_apply_f32(const KrigLaunch& L, const DsTma& T, void* stream);
int krig_launch_ds_apply_u16(const KrigLaunch& L, const DsTma& T, void* stream);
int krig_launch_ds_apply_f64(const KrigLaunch& L, const DsTma& T, void* stream);

// Known-value range of each Z sub-block (Algorithm 1: "for each block, we calculate
// the maximum and minimum possible value"): the min and max over the block's known
// slices a_b .. a_{b+1} (boundary slices belong to both neighbours), in the
// stencil's value type (u16: float32(u) * scale).  One block of threads per
// sub-block; the result [k][2] at mm_off.
template <typename TI, typename TC>
__device__ void ds_block_minmax(const KrigLaunch& P, const KrigVol& V, int v, int b)
{
    __shared__ TC red[2][32];
    const int a0 = b * V.gq + min(b, V.grm), a1 = (b + 1) * V.gq + min(b + 1, V.grm);
    const int64_t plane = (int64_t)V.H * V.W;
    const TI* in = (const TI*)P.in[v] + (size_t)a0 * plane;
    const int64_t cnt = (int64_t)(a1 - a0 + 1) * plane;
    TC lo = TC(INFINITY), hi = TC(-INFINITY);
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
        const TC x = sizeof(TI) == 2 ? (TC)__fmul_rn((float)in[i], V.scale) : (TC)in[i];
        lo = x < lo ? x : lo;
        hi = x > hi ? x : hi;
    }
    for (int o = 16; o; o >>= 1) {
        const TC l2 = __shfl_xor_sync(0xffffffffu, lo, o), h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        lo = l2 < lo ? l2 : lo;
        hi = h2 > hi ? h2 : hi;
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = lo;
        red[1][threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = red[0][w] < lo ? red[0][w] : lo;
            hi = red[1][w] > hi ? red[1][w] : hi;
        }
        TC* mm = (TC*)(P.ws + V.mm_off) + 2 * b;
        mm[0] = lo;
        mm[1] = hi;
    }
}

__global__ void __launch_bounds__(1024) k_block_minmax(const __grid_constant__ KrigLaunch P)
{
    int64_t blk = blockIdx.x;
    int v = 0;
    while (v + 1 < P.n_vols && blk >= P.vol[v].k) blk -= P.vol[v++].k;
    const KrigVol& V = P.vol[v];
    if (V.dtype == KRIG_F64) ds_block_minmax<double, double>(P, V, v, (int)blk);
    else if (V.dtype == KRIG_F32) ds_block_minmax<float, float>(P, V, v, (int)blk);
    else ds_block_minmax<uint16_t, float>(P, V, v, (int)blk);
}

int krig_launch_block_minmax(const KrigLaunch& L, void* stream)
{
    if (!L.clamp || L.n_mm_blocks == 0) return 0;
    k_block_minmax<<<(unsigned)L.n_mm_blocks, 1024, 0, (cudaStream_t)stream>>>(L);
    return (int)cudaGetLastError();
}

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
