// krig_internal.h -- definitions shared by the host planner and the CUDA kernels.
//
// Nothing here is part of the public ABI (include/krig.h is).
#pragma once

#include <stdint.h>

#include "../../include/krig.h"

#define KRIG_GMAX 8                     // largest Z factor g; t slots padded to 8
#define KRIG_TSLOTS 8
#define KRIG_RMAX 2                     // largest half-width r
#define KRIG_KMAX (2 * (2 * KRIG_RMAX + 1) * (2 * KRIG_RMAX + 1))  // 50 points
#define KRIG_XCLS_MAX (2 * KRIG_RMAX + 1)  // compact in-plane truncation classes per axis

// DS stencil tile: TX x TY output pixels per work item; each thread owns PX
// adjacent pixels of one row.
#define KRIG_TX 64
#define KRIG_TY 16
#define KRIG_PX 4
#define KRIG_DS_THREADS ((KRIG_TX / KRIG_PX) * KRIG_TY)  // 256

// Device status bits (sticky, in the workspace control block).
#define KRIG_DEV_SINGULAR 0x1u
#define KRIG_DEV_TIMEOUT 0x2u

// Per-volume parameters, passed by value in the kernel parameter block.
struct KrigVol {
    int32_t H, W, n, g, k, r, dtype;
    float scale;              // u16 -> float scale (1 otherwise)
    int32_t ncx, ncy;         // compact truncation classes along x / y
    int32_t tiles_x, tiles_y; // DS tiles
    int8_t xmap[(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];  // slot lx*(r+1)+rx -> compact class
    int8_t ymap[(KRIG_RMAX + 1) * (KRIG_RMAX + 1)];
    int8_t xext[KRIG_XCLS_MAX][2];                   // compact class -> (left, right) extent
    int8_t yext[KRIG_XCLS_MAX][2];
    int64_t item_begin;       // first DS work item of this volume
    int64_t cls_begin;        // first xy-class of this volume (global index)
    int64_t vox_begin;        // first output voxel of this volume (per-voxel forms)
    int64_t wtab_off;         // byte offset of the DS weight table in the workspace
    int64_t vtab_off;         // byte offset of the DS variance table in the workspace
    int64_t lag_off;          // byte offset of the FP64 lag tables (per-voxel forms)
};

struct KrigLaunch {
    KrigVol vol[KRIG_MAX_VOLUMES];
    const void* in[KRIG_MAX_VOLUMES];
    void* out[KRIG_MAX_VOLUMES];
    float* var[KRIG_MAX_VOLUMES];
    const krig_variogram* vg;   // device, [n_vols]
    unsigned char* ws;          // workspace base
    uint32_t* status;           // device status word (in the workspace)
    int32_t n_vols;
    int32_t form;
    int64_t n_items;            // DS work items over all volumes
    int64_t n_classes;          // xy-classes over all volumes
    int64_t n_vox;              // output voxels over all volumes
};

// Kernel launchers (krig_ds.cu, krig_voxel.cu). Return cudaError_t as int.
int krig_launch_ds_solve(const KrigLaunch& L, int solve_fp64, void* stream);
int krig_launch_ds_apply(const KrigLaunch& L, int grid, void* stream);
int krig_launch_voxel(const KrigLaunch& L, int form, void* stream);
int krig_device_sm_count();

// Set the thread-local message returned by krig_last_error() (krig_api.cu).
__attribute__((visibility("hidden"))) void krig_internal_set_error(const char* msg);

// Table sizes (bytes) per volume for the DS form.
inline int64_t krig_wtab_bytes(const KrigVol& v)
{
    int64_t taps = 2LL * (2 * v.r + 1) * (2 * v.r + 1);
    int64_t esz = v.dtype == KRIG_F64 ? 8 : 4;
    return (int64_t)v.ncx * v.ncy * taps * KRIG_TSLOTS * esz;
}
inline int64_t krig_vtab_bytes(const KrigVol& v) { return (int64_t)v.ncx * v.ncy * KRIG_TSLOTS * 4; }
inline int64_t krig_lag_bytes(const KrigVol& v)
{
    return 8LL * (2 * (2 * v.r + 1) * (2 * v.r + 1) + (v.g > 1 ? v.g - 1 : 0) * 2 * (v.r + 1) * (v.r + 1));
}
