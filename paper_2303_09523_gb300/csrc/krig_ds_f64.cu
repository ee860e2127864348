// krig_ds_f64.cu -- DS stencil apply kernel for double input slices (see krig_ds_apply.cuh).
#include "krig_ds_apply.cuh"

int krig_launch_ds_apply_f64(const KrigLaunch& L, const DsTma& T, void* stream)
{
    return krig_launch_ds_apply_t<double>(L, T, (cudaStream_t)stream);
}
