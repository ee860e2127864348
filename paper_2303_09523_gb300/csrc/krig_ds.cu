// krig_ds.cu -- launcher of the DS stencil apply (one kernel per input type
// present in the plan) and device queries.
#include <cuda_runtime.h>

#include "krig_internal.h"

int krig_launch_ds_apply_f32(const KrigLaunch& L, void* stream);
int krig_launch_ds_apply_u16(const KrigLaunch& L, void* stream);
int krig_launch_ds_apply_f64(const KrigLaunch& L, void* stream);

int krig_launch_ds_apply(const KrigLaunch& L, int grid, void* stream)
{
    (void)grid;
    if (L.n_items == 0) return 0;
    int e = krig_launch_ds_apply_f32(L, stream);
    if (e == 0) e = krig_launch_ds_apply_u16(L, stream);
    if (e == 0) e = krig_launch_ds_apply_f64(L, stream);
    return e;
}

int krig_device_sm_count()
{
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    return n;
}
