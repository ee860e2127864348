// krig_internal.h -- definitions shared by the host planner and the CUDA kernels.
//
// Nothing here is part of the public ABI (include/krig.h is).
#pragma once

#include <cuda.h>  // CUtensorMap (types only; the encoder is reached through the runtime's entry-point query)
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
// Byte offset in the (zeroed) workspace control block of the LOO forward
// launch's block ticket counter (reset by the launch's last block).
#define KRIG_CTRL_LOO_DONE 64
// Byte offset in the control block of the DS stencil's frame-unit tickets, one
// 32-bit counter per input type (krig_dtype), zeroed by the class solve.
#define KRIG_CTRL_FRAME_NEXT 128

// n / d for 0 <= n < 2^32 by one multiply-high with m = krig_udiv_magic(d):
// m = ceil(2^64 / d), and floor(n m / 2^64) = floor(n / d) because the error
// n (m d - 2^64) / (d 2^64) stays below 1/d (division by invariant integers
// using multiplication, Granlund and Montgomery 1994).  d = 1: m = 0.
inline uint64_t krig_udiv_magic(uint32_t d) { return d <= 1 ? 0ull : ~0ull / d + 1ull; }
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t krig_udiv(uint32_t n, uint64_t m)
{
    return m ? (uint32_t)__umul64hi((unsigned long long)n, (unsigned long long)m) : n;
}
#endif

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
    int64_t otab_off;         // byte offset of the interior-class orbit weights [2][6][8] (DS)
    int64_t mm_off;           // byte offset of [k][2] known-value min / max per sub-block (clamp plans)
    int32_t chunk;            // gaps per DS work item (a sub-block is cut into chunks)
    int32_t chunks;           // chunks per sub-block
    int32_t cint;             // interior xy-class index, or -1 if the slice is narrower than 2r+1
    int32_t n_frame;          // frame pixels (within r of the border) per slice (DS)
    int64_t frame_begin;      // first DS frame unit (32 frame pixels of one gap) of this volume, numbered
                              // among the volumes of its input type
    int32_t frame_units;      // frame units per gap
    int32_t gq;               // (n-1) / k: gaps of the smaller sub-blocks
    int32_t grm;              // (n-1) % k: the first grm sub-blocks have one gap more
    int32_t pad0;
    uint64_t mdiv_tiles;      // krig_udiv multipliers: by tiles_x * tiles_y,
    uint64_t mdiv_chunks;     //   by chunks,
    uint64_t mdiv_tx;         //   by tiles_x
    // leave-one-slice-out (plans created with KRIG_FLAG_LOO)
    int64_t loo_cls_begin;    // first LOO class block of this volume
    int64_t loo_item_begin;   // first LOO residual tile (target slices 1..n-2)
    int64_t loo_adj_begin;    // first LOO adjoint tile (slices 0..n-1)
    int64_t lw_off;           // LOO weights [ncy][ncx][2][2r+1][2r+1] float
    int64_t lbar_off;         // sum r S_k per class tap, same layout, double, KRIG_LOO_REP copies
    int64_t res_off;          // residuals (n-2) x H x W float
    int64_t lacc_off;         // loss accumulators, KRIG_LOO_REP doubles
    int64_t lorb_off;         // interior class: sum r * (orbit sum of both slices), [KRIG_LOO_REP][NORB] doubles
    int64_t lvg_off;          // variogram the LOO weights were last solved for (krig_variogram)
    // universal kriging (plans created with a drift or four-slab flag)
    int64_t uk_cls_begin;     // first UK class block of this volume
    int64_t uk_item_begin;    // first UK tile item (gap, tile)
    int64_t uk_wtab_off;      // UK weights [npat][ncy][ncx][slabs][2r+1][2r+1][8] (f64 for f64 input, else f32)
    int64_t uk_vtab_off;      // UK variance [npat][ncy][ncx][8] f32
    int32_t uk_tiles_x, uk_tiles_y;
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
    int64_t n_frame_units;      // DS frame units over all volumes
    int32_t ds_frame_units[3];  // DS frame units per input type (krig_dtype)
    int8_t ds_order[KRIG_MAX_VOLUMES];  // volumes in DS work-item order: by input type, then r, then g
    int32_t fault_timeout;      // test only: make one bounded device wait give up
    int32_t accumulate;         // LOO backward: add into grad_slices / grad_params
    int64_t n_loo_classes, n_loo_items, n_loo_adj;
    int32_t ds_blocks_per_sm;   // stencil blocks per SM (0: as many as fit; set by the autotuner)
    int32_t clamp;              // clamp DS estimates to their sub-block's known range
    int64_t n_mm_blocks;        // sub-blocks over all volumes (clamp plans)
    int32_t uk_drift;           // universal kriging drift: 0 {1}, 1 {1, z}, 2 {1, x, y, z}
    int32_t uk_slabs;           // known slices per neighbourhood: 2, or 4 (0: DS / per-voxel forms)
    int64_t n_uk_classes, n_uk_items;
    // per-call LOO arguments
    float* pred[KRIG_MAX_VOLUMES];
    float* grad_slices[KRIG_MAX_VOLUMES];
    const double* grad_loss;    // [n_vols]
    double* grad_params;        // [n_vols][3]
    double* loss;               // [n_vols]
};

// TMA tensor maps of the known-slice stacks for the DS stencil: one 3-D map
// (x, y, slice) per volume, box = one tile row span x (tile rows + halo) x 1
// slice, zeros outside the stack.  Volumes past KRIG_TMA_VOLS, or whose rows
// are not a 16-byte multiple, use the row-copy path.
#define KRIG_TMA_VOLS 16
struct DsTma {
    CUtensorMap tm[KRIG_TMA_VOLS];
    int32_t valid[KRIG_TMA_VOLS];
};
// Encode the map of volume V at device address ptr; 0 on success.
int krig_encode_ds_tma(const KrigVol& V, const void* ptr, CUtensorMap* out);

// Kernel launchers (krig_ds.cu, krig_voxel.cu). Return cudaError_t as int.
int krig_launch_ds_solve(const KrigLaunch& L, int solve_fp64, void* stream);
int krig_launch_ds_apply(const KrigLaunch& L, const DsTma& T, void* stream);
int krig_launch_voxel(const KrigLaunch& L, int form, void* stream);
int krig_launch_loo(const KrigLaunch& L, int backward, int want_grad_slices, int want_grad_params, void* stream);
int krig_launch_uk(const KrigLaunch& L, void* stream);
int krig_launch_block_minmax(const KrigLaunch& L, void* stream);
int krig_device_sm_count();

// Set the thread-local message returned by krig_last_error() (krig_api.cu).
__attribute__((visibility("hidden"))) void krig_internal_set_error(const char* msg);
// Check one volume descriptor against the limits of include/krig.h (volume
// index i for the message); sets the message and returns the status.
__attribute__((visibility("hidden"))) krig_status krig_internal_check_desc(const krig_volume_desc& d, int i);

// Table sizes (bytes) per volume for the DS form.
inline int64_t krig_wtab_bytes(const KrigVol& v)
{
    int64_t taps = 2LL * (2 * v.r + 1) * (2 * v.r + 1);
    int64_t esz = v.dtype == KRIG_F64 ? 8 : 4;
    return (int64_t)v.ncx * v.ncy * taps * KRIG_TSLOTS * esz;
}
inline int64_t krig_vtab_bytes(const KrigVol& v) { return (int64_t)v.ncx * v.ncy * KRIG_TSLOTS * 4; }
#define KRIG_NORB 6  // D4 orbits of a (2r+1)^2 window for r <= 2
// The LOO weight table [ncls][taps] is followed, at the next multiple of four
// floats, by the interior class's weight per D4 orbit (8 slots).
__host__ __device__ constexpr int loo_wo_off(int ntaps_all) { return (ntaps_all + 3) & ~3; }
inline int64_t krig_otab_bytes(const KrigVol& v) { return 2LL * KRIG_NORB * KRIG_TSLOTS * (v.dtype == KRIG_F64 ? 8 : 4); }
inline int64_t krig_lag_bytes(const KrigVol& v)
{
    return 8LL * (2 * (2 * v.r + 1) * (2 * v.r + 1) + (v.g > 1 ? v.g - 1 : 0) * 2 * (v.r + 1) * (v.r + 1));
}

// Truncation classes along one axis of length N for half-width r: slot
// l*(r+1)+rr (window p-l .. p+rr) -> compact class, in increasing position.
inline void krig_axis_classes(int N, int r, int8_t* map, int8_t (*ext)[2], int* count)
{
    int n = 0;
    for (int i = 0; i < (KRIG_RMAX + 1) * (KRIG_RMAX + 1); ++i) map[i] = -1;
    for (int p = 0; p < N; ++p) {
        if (p > r && p < N - r - 1) continue;  // interior positions repeat the class at p = r
        const int l = p < r ? p : r, rr = (N - 1 - p) < r ? (N - 1 - p) : r;
        const int slot = l * (r + 1) + rr;
        if (map[slot] < 0) {
            map[slot] = (int8_t)n;
            ext[n][0] = (int8_t)l;
            ext[n][1] = (int8_t)rr;
            ++n;
        }
    }
    *count = n;
}

// Fill the descriptor of one volume and lay its tables out in the workspace
// from byte offset *off (advanced, 256-byte aligned).  item/class/voxel
// counters are advanced too.  chunk = gaps per DS work item.
inline void krig_fill_vol(KrigVol& V, const krig_volume_desc& d, int form, int chunk, int64_t* off, int64_t* items,
                          int64_t* classes, int64_t* vox, int64_t* frame_units)
{
    V.H = d.H;
    V.W = d.W;
    V.n = d.n_known;
    V.g = d.zfactor;
    V.k = d.n_sub_blocks;
    V.r = d.half_w;
    V.dtype = d.in_dtype;
    V.scale = d.in_dtype == KRIG_U16 ? d.in_scale : 1.0f;
    krig_axis_classes(d.W, d.half_w, V.xmap, V.xext, &V.ncx);
    krig_axis_classes(d.H, d.half_w, V.ymap, V.yext, &V.ncy);
    const int islot = V.r * (V.r + 1) + V.r;
    V.cint = (V.xmap[islot] >= 0 && V.ymap[islot] >= 0) ? V.ymap[islot] * V.ncx + V.xmap[islot] : -1;
    // frame: pixels within r of the border (all pixels if there is no interior)
    if (V.cint < 0) V.n_frame = V.H * V.W;
    else V.n_frame = 2 * V.r * V.W + 2 * V.r * (V.H - 2 * V.r);
    V.frame_units = V.g >= 2 ? (V.n_frame + 31) / 32 : 0;
    V.frame_begin = *frame_units;
    *frame_units += (int64_t)(V.n - 1) * V.frame_units;
    V.tiles_x = (d.W + KRIG_TX - 1) / KRIG_TX;
    V.tiles_y = (d.H + KRIG_TY - 1) / KRIG_TY;
    const int gaps = V.n - 1;
    const int max_block = (gaps + V.k - 1) / V.k;
    V.chunk = chunk < 1 ? 1 : (chunk > max_block ? max_block : chunk);
    V.chunks = (max_block + V.chunk - 1) / V.chunk;
    V.gq = gaps / V.k;
    V.grm = gaps % V.k;
    V.mdiv_tiles = krig_udiv_magic((uint32_t)(V.tiles_x * V.tiles_y));
    V.mdiv_chunks = krig_udiv_magic((uint32_t)V.chunks);
    V.mdiv_tx = krig_udiv_magic((uint32_t)V.tiles_x);
    V.item_begin = *items;
    *items += (int64_t)V.k * V.chunks * V.tiles_x * V.tiles_y;
    V.cls_begin = *classes;
    if (V.g >= 2) *classes += (int64_t)V.ncx * V.ncy;
    V.vox_begin = *vox;
    *vox += ((int64_t)(V.n - 1) * V.g + 1) * V.H * V.W;
    const auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
    V.wtab_off = V.vtab_off = V.lag_off = V.otab_off = 0;
    if (form == KRIG_FORM_DS) {
        V.wtab_off = *off;
        *off = up(*off + krig_wtab_bytes(V));
        V.vtab_off = *off;
        *off = up(*off + krig_vtab_bytes(V));
        V.otab_off = *off;
        *off = up(*off + krig_otab_bytes(V));
    } else {
        V.lag_off = *off;
        *off = up(*off + krig_lag_bytes(V));
    }
    V.pad0 = 0;
}

// Leave-one-slice-out tables of one volume (plans with KRIG_FLAG_LOO).  The
// residual blocks add their loss and tap-sum partials into one of
// KRIG_LOO_REP copies (block index modulo KRIG_LOO_REP), so that no address
// takes more than a few dozen atomic adds; the readers sum the copies.
#define KRIG_LOO_REP 32
// Target slices per residual work item: an item walks a chain of consecutive
// targets of one tile, so each slice of the chain is read once.
#define KRIG_LOO_CHAIN 8
inline void krig_fill_loo(KrigVol& V, int64_t* off, int64_t* classes, int64_t* items, int64_t* adj)
{
    const auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
    const int64_t taps = 2LL * (2 * V.r + 1) * (2 * V.r + 1);
    const int64_t ncls = (int64_t)V.ncx * V.ncy;
    const int64_t tiles = (int64_t)V.tiles_x * V.tiles_y;
    V.loo_cls_begin = *classes;
    *classes += ncls;
    V.loo_item_begin = *items;
    *items += (int64_t)((V.n - 2 + KRIG_LOO_CHAIN - 1) / KRIG_LOO_CHAIN) * tiles;
    V.loo_adj_begin = *adj;
    *adj += (int64_t)V.n * tiles;
    V.lw_off = *off;
    *off = up(*off + (loo_wo_off((int)(ncls * taps)) + 8) * 4);
    V.lbar_off = *off;
    *off = up(*off + KRIG_LOO_REP * ncls * taps * 8);
    V.res_off = *off;
    *off = up(*off + (int64_t)(V.n - 2) * V.H * V.W * 4);
    V.lacc_off = *off;
    *off = up(*off + KRIG_LOO_REP * 8);
    V.lorb_off = *off;
    *off = up(*off + KRIG_LOO_REP * KRIG_NORB * 8);
    V.lvg_off = *off;
    *off = up(*off + sizeof(krig_variogram));
}

// Number the DS work items volume by volume in ds_order -- sorted by input
// type and stencil shape (r, g), so that the items of one kernel instance and
// shape are one contiguous range -- and the frame units per input type.
// Called whenever the item counts change (plan creation, a new chunk length).
inline void krig_ds_order(KrigLaunch& L)
{
    int n = 0;
    for (int dt = 0; dt < 3; ++dt)
        for (int r = 0; r <= KRIG_RMAX; ++r)
            for (int g = 1; g <= KRIG_GMAX; ++g)
                for (int v = 0; v < L.n_vols; ++v)
                    if (L.vol[v].dtype == dt && L.vol[v].r == r && L.vol[v].g == g) L.ds_order[n++] = (int8_t)v;
    int64_t items = 0;
    for (int k = 0; k < n; ++k) {
        KrigVol& V = L.vol[L.ds_order[k]];
        V.item_begin = items;
        items += (int64_t)V.k * V.chunks * V.tiles_x * V.tiles_y;
    }
    L.n_items = items;
    for (int dt = 0; dt < 3; ++dt) {
        int64_t f = 0;
        for (int v = 0; v < L.n_vols; ++v)
            if (L.vol[v].dtype == dt) {
                L.vol[v].frame_begin = f;
                f += (int64_t)(L.vol[v].n - 1) * L.vol[v].frame_units;
            }
        L.ds_frame_units[dt] = (int32_t)f;
    }
}

// Universal kriging (Appendix A with a drift): tile of the UK stencil, and the
// slab patterns of a gap -- with four slabs the first gap has no slice below
// and the last none above (bit 0: slice j-1 missing, bit 1: slice j+2 missing).
#define KRIG_UK_TX 32
#define KRIG_UK_TY 16
__host__ __device__ inline int krig_uk_npat(int slabs) { return slabs == 4 ? 4 : 1; }
__host__ __device__ inline int krig_uk_terms(int drift) { return drift == 0 ? 1 : (drift == 1 ? 2 : 4); }

// Tables of one volume for the UK path (plans with a drift or four slabs).
inline void krig_fill_uk(KrigVol& V, int slabs, int64_t* off, int64_t* classes, int64_t* items)
{
    const auto up = [](int64_t x) { return (x + 255) / 256 * 256; };
    const int64_t ncls = (int64_t)krig_uk_npat(slabs) * V.ncx * V.ncy;
    const int64_t taps = (int64_t)slabs * (2 * V.r + 1) * (2 * V.r + 1);
    V.uk_tiles_x = (V.W + KRIG_UK_TX - 1) / KRIG_UK_TX;
    V.uk_tiles_y = (V.H + KRIG_UK_TY - 1) / KRIG_UK_TY;
    V.uk_cls_begin = *classes;
    if (V.g >= 2) *classes += ncls;
    V.uk_item_begin = *items;
    *items += (int64_t)(V.n - 1) * V.uk_tiles_x * V.uk_tiles_y;
    V.uk_wtab_off = *off;
    *off = up(*off + ncls * taps * KRIG_TSLOTS * (V.dtype == KRIG_F64 ? 8 : 4));
    V.uk_vtab_off = *off;
    *off = up(*off + ncls * KRIG_TSLOTS * 4);
}

// Gaps per DS work item: enough items to keep every SM busy several times
// over, each item still covering as many gaps as possible.
inline int krig_pick_chunk(const krig_volume_desc* vols, int n_vols)
{
    int64_t gap_tiles = 0;
    for (int i = 0; i < n_vols; ++i)
        gap_tiles += (int64_t)(vols[i].n_known - 1) * ((vols[i].W + KRIG_TX - 1) / KRIG_TX) *
                     ((vols[i].H + KRIG_TY - 1) / KRIG_TY);
    const int64_t target = 2048;
    int64_t c = (gap_tiles + target - 1) / target;
    return (int)(c < 1 ? 1 : c);
}
