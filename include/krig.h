/*
 * krig.h -- C ABI of the GB300 kriging library (libkrig.so).
 *
 * Ordinary kriging of the missing inter-slice voxels of registered 2-D slice
 * stacks, after arXiv 2303.09523 ("Fast 3D Volumetric Image Reconstruction
 * from 2D MRI Slices by Parallel Processing"):
 *   - Algorithm 1 (input: n slices, the inter-slice gap, k): the stack is cut
 *     along Z into k sub-blocks of whole gaps, each block is filled, and the
 *     blocks are merged at their stored offsets (Sec. 4.2);
 *   - Sec. 4.1.2: every missing voxel is a weighted linear sum of known voxels
 *     in 3-D, with weights that minimise the estimation variance subject to
 *     unbiasedness;
 *   - Appendix A: the weights and the Lagrange multiplier solve the extended
 *     system; with one constant predictor this is ordinary kriging.
 *
 * Geometry.  A volume has n known slices of H x W pixels (x fastest) and a
 * Z-upsampling factor g.  The output has (n-1)g+1 slices; known slice j is
 * output slice j*g and is copied through bit-exactly.  The missing voxel
 * (x, y, j*g+t), 1 <= t < g, is estimated from the (2r+1)x(2r+1) in-plane
 * window around (x, y) in known slices j and j+1 (K = 2(2r+1)^2 points),
 * truncated at the in-plane border.  Distances are Euclidean in output-voxel
 * units (in-plane spacing 1, known slices g apart).
 *
 * Variogram (semivariogram, gamma(0) = 0; `sill` is the partial sill):
 *   spherical:   nugget + sill (1.5 h/a - 0.5 (h/a)^3) for h < a, else nugget + sill
 *   exponential: nugget + sill (1 - exp(-3h/a))
 *
 * Conventions for every entry point:
 *   - All slice, output and parameter buffers are caller-owned DEVICE memory
 *     unless stated.  The plan owns host metadata only; device scratch lives
 *     in a caller-owned workspace (krig_plan_set_workspace).
 *   - Calls are asynchronous on the given CUDA stream (a cudaStream_t passed
 *     as void*; NULL = legacy default stream).  Argument errors are returned
 *     before anything is enqueued.  Errors found on the device (a singular
 *     system, a timed-out wait) are sticky bits read by
 *     krig_plan_device_status.
 *   - No C++ exception crosses this boundary.  krig_last_error() gives a
 *     thread-local message for the last non-OK status of this thread.
 *   - Calls that share one plan (and so one workspace) must not overlap on
 *     the device: enqueue them on one stream or synchronise between them.
 */
#ifndef KRIG_H
#define KRIG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct krig_plan_s* krig_plan_t;

typedef enum {
    KRIG_OK = 0,
    KRIG_EINVAL = 1,        /* bad argument (null pointer, size out of range, ...) */
    KRIG_ENOMEM = 2,        /* host allocation failed */
    KRIG_ECUDA = 3,         /* a CUDA runtime call failed */
    KRIG_ESINGULAR = 4,     /* a kriging system was singular (e.g. nugget = sill = 0) */
    KRIG_ETIMEOUT = 5,      /* a bounded device-side wait gave up */
    KRIG_EWORKSPACE = 6,    /* no workspace, or one that is too small or misaligned */
    KRIG_EUNSUPPORTED = 7   /* valid request this build does not implement */
} krig_status;

typedef enum { KRIG_SPHERICAL = 0, KRIG_EXPONENTIAL = 1 } krig_model;

/* Storage type of the known slices.  Output type: float64 for KRIG_F64
 * input, float32 otherwise.  KRIG_U16 values are float32(u) * in_scale
 * (float32 multiply). */
typedef enum { KRIG_F64 = 0, KRIG_F32 = 1, KRIG_U16 = 2 } krig_dtype;

/* How the kriging systems are solved.
 *   P64: one FP64 system per missing voxel (the plain reference form).
 *   PMX: one system per missing voxel, FP32 factorisation plus one FP64
 *        iterative-refinement step.
 *   DS : one system per neighbourhood geometry class (FP32 factorisation,
 *        one refinement step with a float-float residual; FP64 throughout
 *        with KRIG_FLAG_DS_FP64_SOLVE), applied to every voxel of that class
 *        as an FP32 stencil (FP64 for KRIG_F64 input).
 *        A voxel's system depends only on t and on how its window is
 *        truncated at the border, so the solutions repeat across voxels. */
typedef enum { KRIG_FORM_P64 = 0, KRIG_FORM_PMX = 1, KRIG_FORM_DS = 2 } krig_form;

/* One slice stack.  Limits: H, W in [1, 65536]; 2 <= n_known <= 65536;
 * 1 <= zfactor <= 8; 1 <= n_sub_blocks <= n_known - 1; half_w in {0, 1, 2}. */
typedef struct {
    int32_t H, W;
    int32_t n_known;       /* n */
    int32_t zfactor;       /* g */
    int32_t n_sub_blocks;  /* k: Z sub-blocks of whole gaps (Algorithm 1, step 2) */
    int32_t half_w;        /* r: window (2r+1)^2 per bracketing slice */
    int32_t in_dtype;      /* krig_dtype */
    float in_scale;        /* KRIG_U16 only; ignored otherwise */
} krig_volume_desc;

/* Variogram parameters, one per volume, in DEVICE memory for the calls below
 * (so a captured CUDA graph can be replayed with new values). 32 bytes. */
typedef struct {
    int32_t model;   /* krig_model */
    int32_t pad;
    double nugget;   /* >= 0 */
    double sill;     /* partial sill, >= 0; nugget + sill > 0 */
    double range;    /* a > 0, in output-voxel units */
} krig_variogram;

/* Plan flags.
 *   KRIG_FLAG_DS_FP64_SOLVE: DS form only -- factorise the class systems in
 *   FP64 instead of FP32 followed by one refinement step whose residual is
 *   formed in float-float (about 48 significant bits). */
#define KRIG_FLAG_DS_FP64_SOLVE 0x1u
/*   KRIG_FLAG_FAULT_TIMEOUT: test only -- the DS stencil kernel waits once on a
 *   barrier that nothing completes, so its bounded wait gives up and the call's
 *   device status becomes KRIG_ETIMEOUT (exercises failure detection without a
 *   real fault; the outputs of that call are not valid). */
#define KRIG_FLAG_FAULT_TIMEOUT 0x100u
/*   KRIG_FLAG_LOO: also size the workspace for krig_loo_forward / krig_backward
 *   (DS form only; every volume needs n_known >= 3). */
#define KRIG_FLAG_LOO 0x2u
/*   Universal kriging (Appendix A with more than one predictor, one
 *   unbiasedness constraint and Lagrange multiplier each; Sec. 4.1.2 names the
 *   method universal kriging).  DS form only, every volume of the plan:
 *     KRIG_FLAG_DRIFT_Z:   drift {1, z} (z along the stack);
 *     KRIG_FLAG_DRIFT_XYZ: drift {1, x, y, z} (needs half_w >= 1, H, W >= 2);
 *     KRIG_FLAG_SLABS4:    the window in four known slices, j-1 .. j+2, those
 *                          that exist (the "64 neighbours" of Sec. 4.1.2 read
 *                          as 4 slices x the in-plane window), instead of the
 *                          bracketing pair j, j+1.
 *   Either drift flag, or KRIG_FLAG_SLABS4 alone (constant drift: ordinary
 *   kriging on four slices), selects the universal-kriging path: one class
 *   solve per geometry class (truncation, and which outer slices exist; FP32
 *   Cholesky factorisation, two refinement steps with float-float residuals)
 *   with all targets t of a gap, then the stencil with each class's weights.
 *   The kriging variance is w'gamma0 + mu'f0.  Not combinable with
 *   KRIG_FLAG_LOO, KRIG_FLAG_DS_FP64_SOLVE or KRIG_FLAG_FAULT_TIMEOUT. */
/*   KRIG_FLAG_CLAMP_BLOCK_MINMAX: DS form (without drift flags) -- Algorithm 1
 *   computes the maximum and minimum value of each block without saying what
 *   they are for; with this flag every interpolated voxel is clamped to the
 *   [min, max] of the known voxels of its Z sub-block (its known slices a_b ..
 *   a_{b+1}, boundary slices included).  Off by default.  NaN estimates stay NaN. */
#define KRIG_FLAG_CLAMP_BLOCK_MINMAX 0x20u
#define KRIG_FLAG_DRIFT_Z 0x4u
#define KRIG_FLAG_DRIFT_XYZ 0x8u
#define KRIG_FLAG_SLABS4 0x10u

#define KRIG_MAX_VOLUMES 64

/* Create a plan for n_vols volumes (1..KRIG_MAX_VOLUMES) solved in `form`.
 * Validates the descriptors, partitions each stack into its Z sub-blocks and
 * in-plane tiles, enumerates the geometry classes and sizes the workspace.
 * *plan receives the handle (NULL on error); *workspace_bytes_out (nullable)
 * the device workspace size that krig_plan_set_workspace needs.  Does not
 * touch the GPU.  Errors: KRIG_EINVAL, KRIG_EUNSUPPORTED, KRIG_ENOMEM. */
krig_status krig_plan_create(krig_plan_t* plan, const krig_volume_desc* vols, int32_t n_vols,
                             krig_form form, uint32_t flags, size_t* workspace_bytes_out);

/* Attach caller-owned device memory (>= the size reported above, 256-byte
 * aligned) as the plan's workspace and upload the plan's tables into it
 * (synchronous: returns after the upload, on the current device).  The
 * memory must stay valid until the plan is destroyed or another workspace
 * is set.  Errors: KRIG_EWORKSPACE, KRIG_ECUDA. */
krig_status krig_plan_set_workspace(krig_plan_t plan, void* d_workspace, size_t bytes);

/* Interpolate every volume (Algorithm 1 steps 2-4, Sec. 4.1.2, Appendix A).
 *   d_slices[v]: device, n x H x W of the volume's in_dtype (16-byte aligned).
 *   d_out[v]:    device, ((n-1)g+1) x H x W, float64 for KRIG_F64 input else
 *                float32 (16-byte aligned).  Known slices are copied through.
 *   d_var:       nullable host array of n_vols nullable device pointers, each
 *                ((n-1)g+1) x H x W float32: the kriging variance
 *                w^T gamma0 + mu of every voxel (0 at known slices).
 *   d_params:    device array of n_vols krig_variogram.
 * The host arrays d_slices / d_out / d_var are read during the call only.
 * Errors: KRIG_EINVAL, KRIG_EWORKSPACE, KRIG_ECUDA (launch). */
krig_status krig_interpolate(krig_plan_t plan, const void* const* d_slices, void* const* d_out,
                             float* const* d_var, const krig_variogram* d_params, void* stream);

/* Leave-one-slice-out cross-validation loss, the differentiable objective for
 * fitting the variogram (the paper fixes none).  Each interior known slice j
 * (1 <= j <= n-2) is predicted at its own z by ordinary kriging from slices
 * j-1 and j+1 (a gap of 2g, target in the middle; same window, truncation and
 * variogram as krig_interpolate), and
 *     L_v = 1/((n-2) H W) * sum_j sum_{x,y} (P_j(x,y) - S_j(x,y))^2.
 * Needs a plan created with KRIG_FLAG_LOO.
 *   d_slices, d_params: as krig_interpolate.
 *   d_pred: nullable host array of nullable device pointers, (n-2) x H x W
 *           float32 predictions.
 *   d_loss: device, [n_vols] float64 (overwritten).
 * Errors: KRIG_EINVAL, KRIG_EUNSUPPORTED (plan without the flag), KRIG_EWORKSPACE,
 * KRIG_ECUDA. */
krig_status krig_loo_forward(krig_plan_t plan, const void* const* d_slices, const krig_variogram* d_params,
                             float* const* d_pred, double* d_loss, void* stream);

/* Gradient of the LOO loss, scaled by the upstream gradient d_grad_loss[v]
 * (device float64 per volume), with respect to
 *   - every known-slice intensity (d_grad_slices: nullable host array of
 *     nullable device pointers, n x H x W float32), and
 *   - the variogram parameters (d_grad_params: nullable device float64
 *     [n_vols][3] = d/d(nugget, sill, range)).
 * With accumulate != 0 the gradients are added to the buffers; otherwise they
 * are overwritten.  The residuals are recomputed from the slices, not kept
 * from the forward pass; the LOO class weights are reused when the workspace
 * records that they were solved for the same variogram values (the forward
 * pass of the same step), and solved again otherwise; the class adjoint
 * systems are always solved again.
 * Errors: as krig_loo_forward. */
krig_status krig_backward(krig_plan_t plan, const void* const* d_slices, const krig_variogram* d_params,
                          const double* d_grad_loss, float* const* d_grad_slices, double* d_grad_params,
                          int32_t accumulate, void* stream);

/* Autotune the DS schedule on the caller's data: time krig_interpolate (iters
 * calls each, synchronously on `stream`) for several work-item lengths (gaps
 * per item: 1, 2, 3, 4, 6, 8, 12, 16 and whole sub-blocks), each with the
 * stencil launched at as many blocks per SM as fit or at one, and keep the
 * fastest pair.  The choice changes only the schedule: every choice gives
 * bit-identical results.  Writes to d_out.  Not capturable; call it before
 * capturing a graph.  *chunk_out (nullable) receives the chosen length
 * (krig_plan_schedule reports both choices).
 * Errors: as krig_interpolate; KRIG_EUNSUPPORTED for P64 / PMX plans. */
krig_status krig_plan_autotune(krig_plan_t plan, const void* const* d_slices, void* const* d_out,
                               const krig_variogram* d_params, int32_t iters, void* stream, int32_t* chunk_out);

/* The plan's DS schedule: gaps per work item (of volume 0; every volume uses the
 * same length, capped at its sub-block) and stencil blocks per SM (0: as many as
 * fit).  Either pointer nullable.  Errors: KRIG_EINVAL. */
krig_status krig_plan_schedule(krig_plan_t plan, int32_t* chunk_out, int32_t* blocks_per_sm_out);

/* Set the DS schedule directly (a result of krig_plan_autotune kept from an
 * earlier run): gaps per work item (>= 1; capped at each volume's sub-block)
 * and stencil blocks per SM (0: as many as fit).  Results are bit-identical for
 * every schedule.  Host only; call it before capturing a graph.
 * Errors: KRIG_EINVAL, KRIG_EUNSUPPORTED (P64 / PMX plans). */
krig_status krig_plan_set_schedule(krig_plan_t plan, int32_t chunk, int32_t blocks_per_sm);

/* Wait for the stream, then return and clear the plan's device error bits:
 * KRIG_OK, KRIG_ESINGULAR or KRIG_ETIMEOUT (the first set, in that order). */
krig_status krig_plan_device_status(krig_plan_t plan, void* stream);

/* Kernel timing (tracing).  While enabled, each launch of the plan is
 * bracketed by CUDA events on the call's stream; krig_plan_get_timing waits
 * for them and returns the summed milliseconds per kernel kind and the number
 * of launches, then resets the sums.  kinds: 0 class/voxel solve, 1 stencil
 * apply (DS), 2 loo forward, 3 backward.  Arrays have KRIG_TIMING_KINDS
 * entries (nullable). */
#define KRIG_TIMING_KINDS 4
krig_status krig_plan_set_timing(krig_plan_t plan, int32_t enable);
krig_status krig_plan_get_timing(krig_plan_t plan, double* ms_out, int64_t* launches_out);

/* Kriging variance as a class table (the variance of a missing voxel depends only
 * on its geometry class, like its weights): after krig_interpolate on a DS plan
 * without drift flags, the variance of voxel (x, y, j*g + t), 1 <= t < g, of
 * volume v is
 *     h_table[(h_cy[y] * ncx + h_cx[x]) * 8 + t - 1]
 * (0 at known slices) -- the same values krig_interpolate writes into d_var,
 * without the variance volume.  Fills (each nullable): h_table host float
 * [ncy][ncx][8] (waits for `stream`, then copies), h_cx host int32 [W], h_cy
 * host int32 [H] (class of each coordinate), *ncx_out, *ncy_out.
 * Errors: KRIG_EINVAL, KRIG_EUNSUPPORTED (P64 / PMX / drift plans),
 * KRIG_EWORKSPACE, KRIG_ECUDA. */
krig_status krig_plan_variance_table(krig_plan_t plan, int32_t v, float* h_table, int32_t* h_cx, int32_t* h_cy,
                                     int32_t* ncx_out, int32_t* ncy_out, void* stream);

/* Thread-local message for the last non-OK status returned on this thread. */
const char* krig_last_error(void);

/* Destroy the plan (host memory only; the workspace stays the caller's).
 * NULL is ignored. */
void krig_plan_destroy(krig_plan_t plan);

/* Interpolate ONE volume in the DS form without any device allocation.
 * The paper has no counterpart: this entry point exists for callers that may
 * not allocate device memory -- a plugin inside an application that owns all
 * device memory through its own pool, a real-time loop that cannot take
 * cudaMalloc's implicit device synchronisation, a service under a device
 * memory budget enforced outside this library.  They cannot supply the
 * workspace krig_plan_set_workspace needs.
 *
 * Scratch: a static device array of 64 KiB inside the library, held by every
 * GPU that loads the library until the process exits.  Volumes whose class
 * tables do not fit are rejected with KRIG_EINVAL and a message giving the
 * size needed (float64 input with half_w 2 needs about 81 KB; every float32 or
 * uint16 volume fits).  Every call shares that one array and leaves its last
 * contents in it; the call clears the device status word itself.  Calls whose
 * work overlaps on the GPU (other streams, other host threads) race on the
 * scratch and must be serialised by the caller.
 *
 * The first call on a device looks up the array's device address (a one-time
 * set-up per device, done with that device current); make that first call
 * before any stream capture.  The address is kept for the life of the
 * process: after cudaDeviceReset on a device, do not call this entry point on
 * that device again.
 *
 * Arguments: as one volume of krig_interpolate (desc, d_slices, d_out,
 * d_var nullable, d_params pointing at one device krig_variogram); the
 * descriptor limits and error codes are those of krig_plan_create.  With
 * check_status != 0 the call waits for the stream and returns KRIG_ESINGULAR
 * if a kriging system was singular, or KRIG_ETIMEOUT if a bounded device
 * wait gave up (part of the output is then not written); with 0 it returns
 * after enqueueing (a singular system then shows as NaN estimates).  No
 * cudaMalloc, cudaFree or other allocating call is made. */
krig_status krig_interpolate_noalloc(const krig_volume_desc* desc, const void* d_slices, void* d_out, float* d_var,
                                     const krig_variogram* d_params, int32_t check_status, void* stream);

/* Empirical variogram of the known slices: the method-of-moments estimate of
 * the variogram gamma(h) that Sec. 4.1.2 uses (the paper does not say how it is
 * obtained), i.e. the data a model (spherical, exponential) is fitted to.
 * For every lag vector (s, dy, dx), |dy|, |dx| <= L = max_lag, s = 0 (both
 * voxels in one known slice) or s = 1 (known slice k to known slice k + 1):
 *   d_sums[(s (2L+1) + dy+L) (2L+1) + dx+L]
 *       = sum over k, y, x with both voxels inside the stack of
 *         (S[k][y][x] - S[k+s][y+dy][x+dx])^2
 * (device float64, 2 (2L+1)^2 entries, overwritten) and, if h_counts is not
 * NULL, the number of such pairs in the same layout (host int64, filled before
 * the call returns); gamma = sums / (2 counts) where counts > 0.  The in-plane
 * lags are in pixels; slice k + 1 lies zfactor output voxels above slice k.
 *   desc: H, W, n_known, in_dtype, in_scale as for krig_plan_create
 *         (zfactor, n_sub_blocks and half_w are not used).
 *   d_slices: n_known x H x W of in_dtype (u16: value * in_scale).
 *   max_lag: 0..16.
 * Differences and squares in float32, summed over at most 64 pixels of a row
 * in float32 and above that in float64.  Asynchronous on `stream`; no
 * workspace, no allocation.  Errors: KRIG_EINVAL (before any launch),
 * KRIG_ECUDA. */
krig_status krig_empirical_variogram(const krig_volume_desc* desc, const void* d_slices, int32_t max_lag,
                                     double* d_sums, int64_t* h_counts, void* stream);

/* Similarity metrics of Appendix D between ground-truth images G and
 * reconstructed images R (the paper scores each slice cut from the
 * reconstructed volume against its ground-truth image): for every image i of a
 * stack of n_img images of H x W pixels,
 *   d_out[8 i + 0] = RMSE = sqrt(1/(HW) sum (R - G)^2)
 *   d_out[8 i + 1] = MI(G, R) = sum p_GR log2(p_GR / (p_G p_R))   (bits)
 *   d_out[8 i + 2] = MI(G, G) = the entropy of G on its own value range
 *   d_out[8 i + 3] = ED = |H(G) - H(R)| / H(G)
 *   d_out[8 i + 4] = SSIM = (2 mx my + c1)(2 sxy + c2) / ((mx^2 + my^2 + c1)(sx^2 + sy^2 + c2))
 *   d_out[8 i + 5..7] = H(G), H(R), H(G, R)
 * Appendix D fixes neither the histogram nor the SSIM constants; here:
 * 256 equal bins over the joint range [min(G,R), max(G,R)] of the pair (a
 * value's bin floor((x - lo) * s), s = 256 / (hi - lo), in FP64, clamped to
 * [0, 255]; all values in bin 0 when hi = lo), logarithms base 2, population moments
 * over the whole image, c1 = (0.01 L)^2, c2 = (0.03 L)^2, L = max(G) - min(G).
 *   d_G, d_R: device float32 [n_img][H][W].  d_out: device float64 [n_img][8].
 *   d_work: caller-owned device scratch, 256-byte aligned, at least
 *           krig_similarity_workspace_bytes(n_img, H, W) bytes (partial sums
 *           and the 256 x 256 joint histogram of every image).
 * Sums in FP64.  Asynchronous on `stream`; no allocation.  Errors: KRIG_EINVAL,
 * KRIG_EWORKSPACE (before any launch), KRIG_ECUDA. */
size_t krig_similarity_workspace_bytes(int32_t n_img, int32_t H, int32_t W);
krig_status krig_similarity(const float* d_G, const float* d_R, int32_t n_img, int32_t H, int32_t W, void* d_work,
                            size_t work_bytes, double* d_out, void* stream);

/* Marching cubes (Appendix C): the triangle mesh of the iso-surface v = iso of a
 * volume (for instance a reconstructed stack), into a caller-owned device
 * buffer.  Every cube of 2 x 2 x 2 neighbouring voxels is classified by which
 * corners are inside (v > iso); the surface crosses each edge between an
 * inside and an outside corner at the linear-interpolation point.  The paper
 * prints no case table; the one used is generated from the cube's geometry
 * (krig_marching_cubes_table): on each face the cut edges are joined in pairs,
 * a face with two diagonal inside corners cutting each of them off alone (so
 * neighbouring cubes agree and the surface is closed); the segments, directed
 * with the inside corners on their right as seen from outside the cube, close
 * into loops, and each loop is fanned into triangles from its vertex on the
 * edge of smallest index.  Triangle normals (right-hand rule) point out of the
 * inside region.
 *   d_vol: device float32 [D][H][W] (x fastest), D, H, W >= 2.
 *   d_tri: device float32 [max_tri][3 vertices][x, y, z] in voxel units (corner
 *          (x, y, z) of the volume at (x, y, z)); nullable when max_tri = 0.
 *   d_ntri: device int64, receives the number of triangles of the surface; only
 *           the first max_tri are written (call with max_tri = 0 to size d_tri).
 *   d_work: caller-owned device scratch, 256-byte aligned, at least
 *           krig_marching_cubes_workspace_bytes(D, H, W) bytes (one byte per cube
 *           and a count per block of 2048 cubes).
 * Triangles are in cube order (x fastest), a cube's in table order: the output
 * is deterministic.  Asynchronous on `stream`.  Errors: KRIG_EINVAL,
 * KRIG_EWORKSPACE (before any launch), KRIG_ECUDA. */
size_t krig_marching_cubes_workspace_bytes(int32_t D, int32_t H, int32_t W);
krig_status krig_marching_cubes(const float* d_vol, int32_t D, int32_t H, int32_t W, float iso, float* d_tri,
                                int64_t max_tri, int64_t* d_ntri, void* d_work, size_t work_bytes, void* stream);
/* The generated case table: tri_out[256][16] edge indices, three per triangle,
 * -1 after the last; ntri_out[256] triangles per case (either nullable).  Edge
 * e joins cube corners (kEdge): 0-3 along x, 4-7 along y, 8-11 along z; corner
 * i = dx + 2 dy + 4 dz.  Host only. */
void krig_marching_cubes_table(int8_t* tri_out, uint8_t* ntri_out);

/* Measure the device's fused multiply-add rate (GFLOP/s, 2 flops per FMA)
 * in FP32 (fp64 = 0) or FP64 (fp64 = 1) on the current device with a short
 * synchronous kernel.  Support routine: the roofline denominator for kernels
 * bound by arithmetic issue rather than memory.  Errors: KRIG_EINVAL,
 * KRIG_ECUDA. */
krig_status krig_measure_fma_peak(int32_t fp64, double* gflops_out);

/* Library version: major * 10000 + minor * 100 + patch. */
int32_t krig_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KRIG_H */
