// krig_ds_f32.cu -- DS stencil apply kernel for float input slices (see krig_ds_apply.cuh).
#include "krig_ds_apply.cuh"

int krig_launch_ds_apply_f32(const KrigLaunch& L, const DsTma& T, void* stream)
{
    return krig_launch_ds_apply_t<float>(L, T, (cudaStream_t)stream);
}
