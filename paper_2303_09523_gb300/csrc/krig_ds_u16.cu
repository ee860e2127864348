// krig_ds_u16.cu -- DS stencil apply kernel for uint16_t input slices (see krig_ds_apply.cuh).
#include "krig_ds_apply.cuh"

int krig_launch_ds_apply_u16(const KrigLaunch& L, const DsTma& T, void* stream)
{
    return krig_launch_ds_apply_t<uint16_t>(L, T, (cudaStream_t)stream);
}
