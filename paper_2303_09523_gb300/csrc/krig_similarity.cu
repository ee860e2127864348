// krig_similarity.cu -- the similarity metrics of Appendix D between ground-truth
// and reconstructed 2-D images, on the device: RMSE, mutual information,
// entropy difference and SSIM, per image of a stack (the paper scores every
// slice cut from the reconstructed volume against its ground-truth image).
//
// Readings of the metrics (Appendix D is silent on them): histograms of 256
// equal bins over the joint value range [min(G, R), max(G, R)] of the image
// pair, one binning for both images, logarithms base 2; MI(G, G) uses G's own
// range; ED = |H(G) - H(R)| / H(G) on the joint binning; SSIM is the printed
// global formula with population moments, c1 = (0.01 L)^2, c2 = (0.03 L)^2 and
// L = max(G) - min(G).  A value's bin is floor((x - lo) * s) with s = 256 /
// (hi - lo) formed once per image, in FP64, clamped to [0, 255] (all zero when
// hi <= lo); one FP64 division per image instead of one per value.
//
// Four launches per call: per-block partial sums and extrema, per-image
// means and ranges (and the histograms zeroed), the histograms (joint
// 256 x 256 counts by global atomics, G's own-range counts in shared memory)
// with the centred second moments, and per-image entropies and metrics.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <string>

#include "krig_internal.h"

namespace {

constexpr int SIM_BINS = 256;
constexpr int SIM_THREADS = 256;
constexpr int SIM_PART = 10;   // doubles per block partial: 6 sums, min/max of G and R
constexpr int SIM_STATS = 12;  // doubles per image: 6 sums, joint lo/hi, G lo/hi, n, pad
constexpr int SIM_MAX_BLOCKS = 64;

struct SimWork {
    double* part;         // [n_img][nb][SIM_PART]
    double* stats;        // [n_img][SIM_STATS]
    unsigned* joint;      // [n_img][256][256]
    unsigned* own;        // [n_img][256]
};

__host__ __device__ inline size_t sim_align(size_t x) { return (x + 255) / 256 * 256; }

int sim_blocks(int64_t npix)
{
    int64_t nb = (npix + 8 * SIM_THREADS - 1) / (8 * SIM_THREADS);
    return (int)(nb < 1 ? 1 : (nb > SIM_MAX_BLOCKS ? SIM_MAX_BLOCKS : nb));
}

SimWork sim_layout(void* base, int n_img, int nb, size_t* total)
{
    unsigned char* p = (unsigned char*)base;
    size_t off = 0;
    SimWork w;
    w.part = (double*)(p + off);
    off = sim_align(off + (size_t)n_img * nb * SIM_PART * sizeof(double));
    w.stats = (double*)(p + off);
    off = sim_align(off + (size_t)n_img * SIM_STATS * sizeof(double));
    w.joint = (unsigned*)(p + off);
    off = sim_align(off + (size_t)n_img * SIM_BINS * SIM_BINS * sizeof(unsigned));
    w.own = (unsigned*)(p + off);
    off = sim_align(off + (size_t)n_img * SIM_BINS * sizeof(unsigned));
    *total = off;
    return w;
}

template <typename T>
__device__ __forceinline__ T block_reduce(T v, T* red, bool is_max, bool is_min)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) {
        const T u = __shfl_xor_sync(0xffffffffu, v, o);
        v = is_max ? (u > v ? u : v) : is_min ? (u < v ? u : v) : v + u;
    }
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < SIM_THREADS / 32 ? red[lane] : (is_max ? -INFINITY : is_min ? INFINITY : T(0));
        for (int o = 16; o; o >>= 1) {
            const T u = __shfl_xor_sync(0xffffffffu, v, o);
            v = is_max ? (u > v ? u : v) : is_min ? (u < v ? u : v) : v + u;
        }
    }
    return v;  // valid in thread 0
}

// Partial sums over one block's share of one image: sum G, R, G^2, R^2, GR,
// (R - G)^2 in FP64 (products of the exact float values), min / max of G, R
// (the means and the ranges; the variances come from a second, centred pass).
__global__ void __launch_bounds__(SIM_THREADS) k_sim_partial(const float* G, const float* R, int64_t npix, SimWork w)
{
    __shared__ double red[SIM_THREADS / 32];
    const int img = blockIdx.y, nb = gridDim.x;
    const float* g = G + (size_t)img * npix;
    const float* r = R + (size_t)img * npix;
    double s[6] = {0, 0, 0, 0, 0, 0};
    double mn[2] = {INFINITY, INFINITY}, mx[2] = {-INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)SIM_THREADS + threadIdx.x; i < npix; i += (int64_t)nb * SIM_THREADS) {
        const double a = g[i], b = r[i];
        s[0] += a;
        s[1] += b;
        s[2] += a * a;
        s[3] += b * b;
        s[4] += a * b;
        s[5] += (b - a) * (b - a);
        mn[0] = fmin(mn[0], a);
        mx[0] = fmax(mx[0], a);
        mn[1] = fmin(mn[1], b);
        mx[1] = fmax(mx[1], b);
    }
    double* out = w.part + ((size_t)img * nb + blockIdx.x) * SIM_PART;
    for (int k = 0; k < 6; ++k) {
        const double t = block_reduce<double>(s[k], red, false, false);
        if (threadIdx.x == 0) out[k] = t;
    }
    for (int k = 0; k < 2; ++k) {
        const double a = block_reduce<double>(mn[k], red, false, true);
        if (threadIdx.x == 0) out[6 + 2 * k] = a;
        const double b = block_reduce<double>(mx[k], red, true, false);
        if (threadIdx.x == 0) out[7 + 2 * k] = b;
    }
}

// Per image: the partials summed in block order, the ranges, and the
// histograms zeroed for the next launch.
__global__ void __launch_bounds__(SIM_THREADS) k_sim_stats(int nb, int64_t npix, SimWork w)
{
    const int img = blockIdx.x;
    if (threadIdx.x == 0) {
        const double* p = w.part + (size_t)img * nb * SIM_PART;
        double s[6] = {0, 0, 0, 0, 0, 0};
        double gmn = INFINITY, gmx = -INFINITY, rmn = INFINITY, rmx = -INFINITY;
        for (int b = 0; b < nb; ++b) {
            for (int k = 0; k < 6; ++k) s[k] += p[b * SIM_PART + k];
            gmn = fmin(gmn, p[b * SIM_PART + 6]);
            gmx = fmax(gmx, p[b * SIM_PART + 7]);
            rmn = fmin(rmn, p[b * SIM_PART + 8]);
            rmx = fmax(rmx, p[b * SIM_PART + 9]);
        }
        double* st = w.stats + (size_t)img * SIM_STATS;
        for (int k = 0; k < 6; ++k) st[k] = s[k];
        st[6] = fmin(gmn, rmn);
        st[7] = fmax(gmx, rmx);
        st[8] = gmn;
        st[9] = gmx;
        st[10] = (double)npix;
        st[11] = 0.0;
    }
    unsigned* j = w.joint + (size_t)img * SIM_BINS * SIM_BINS;
    for (int e = threadIdx.x; e < SIM_BINS * SIM_BINS; e += SIM_THREADS) j[e] = 0u;
    if (threadIdx.x < SIM_BINS) w.own[(size_t)img * SIM_BINS + threadIdx.x] = 0u;
}

// Bin of x: floor((x - lo) * scale), scale = 256 / (hi - lo) formed once per image
// (0 when hi <= lo: every value in bin 0).  FP64, the oracle's arithmetic.
__device__ __forceinline__ int sim_bin(double x, double lo, double scale)
{
    const double b = floor((x - lo) * scale);
    return b < 0.0 ? 0 : (b > SIM_BINS - 1 ? SIM_BINS - 1 : (int)b);
}
__device__ __forceinline__ double sim_scale(double lo, double hi)
{
    return hi > lo ? (double)SIM_BINS / (hi - lo) : 0.0;
}

// The histograms, and the centred sums sum (G - mx)^2, (R - my)^2, (G - mx)(R - my)
// per block (two-pass moments: a constant image has exactly zero variance).
__global__ void __launch_bounds__(SIM_THREADS) k_sim_hist(const float* G, const float* R, int64_t npix, SimWork w)
{
    __shared__ unsigned own[SIM_BINS];
    __shared__ double red[SIM_THREADS / 32];
    const int img = blockIdx.y, nb = gridDim.x;
    const double* st = w.stats + (size_t)img * SIM_STATS;
    const double lo = st[6], glo = st[8];
    const double sc = sim_scale(st[6], st[7]), gsc = sim_scale(st[8], st[9]);
    for (int e = threadIdx.x; e < SIM_BINS; e += SIM_THREADS) own[e] = 0u;
    __syncthreads();
    const float* g = G + (size_t)img * npix;
    const float* r = R + (size_t)img * npix;
    unsigned* joint = w.joint + (size_t)img * SIM_BINS * SIM_BINS;
    const double mx = st[0] / st[10], my = st[1] / st[10];
    double c[3] = {0.0, 0.0, 0.0};
    for (int64_t i = blockIdx.x * (int64_t)SIM_THREADS + threadIdx.x; i < npix; i += (int64_t)nb * SIM_THREADS) {
        const double a = g[i], b = r[i];
        atomicAdd(&joint[sim_bin(a, lo, sc) * SIM_BINS + sim_bin(b, lo, sc)], 1u);
        atomicAdd(&own[sim_bin(a, glo, gsc)], 1u);
        c[0] += (a - mx) * (a - mx);
        c[1] += (b - my) * (b - my);
        c[2] += (a - mx) * (b - my);
    }
    __syncthreads();
    for (int e = threadIdx.x; e < SIM_BINS; e += SIM_THREADS)
        if (own[e]) atomicAdd(&w.own[(size_t)img * SIM_BINS + e], own[e]);
    double* out = w.part + ((size_t)img * nb + blockIdx.x) * SIM_PART;  // the first pass's partials are spent
    for (int k = 0; k < 3; ++k) {
        const double t = block_reduce<double>(c[k], red, false, false);
        if (threadIdx.x == 0) out[k] = t;
    }
}

// Per image: marginals, entropies and the metrics.  out[img][8] = rmse, mi,
// mi_gg (= entropy of G on its own range), ed, ssim, h_g, h_r (joint binning), h_gr.
__global__ void __launch_bounds__(SIM_THREADS) k_sim_final(SimWork w, int nb, double* out)
{
    __shared__ double pg[SIM_BINS], pr[SIM_BINS];
    __shared__ double red[SIM_THREADS / 32];
    const int img = blockIdx.x, t = threadIdx.x;
    const double* st = w.stats + (size_t)img * SIM_STATS;
    const double n = st[10];
    const unsigned* joint = w.joint + (size_t)img * SIM_BINS * SIM_BINS;
    // marginal counts: row t (G bin t) and column t (R bin t)
    double rs = 0.0, cs = 0.0;
    for (int k = 0; k < SIM_BINS; ++k) {
        rs += (double)joint[t * SIM_BINS + k];
        cs += (double)joint[k * SIM_BINS + t];
    }
    pg[t] = rs / n;
    pr[t] = cs / n;
    __syncthreads();
    double mi = 0.0, hgr = 0.0;
    for (int k = 0; k < SIM_BINS; ++k) {
        const unsigned c = joint[t * SIM_BINS + k];
        if (c) {
            const double p = (double)c / n;
            mi += p * log2(p / (pg[t] * pr[k]));
            hgr -= p * log2(p);
        }
    }
    const double hg = pg[t] > 0.0 ? -pg[t] * log2(pg[t]) : 0.0;
    const double hr = pr[t] > 0.0 ? -pr[t] * log2(pr[t]) : 0.0;
    const unsigned co = w.own[(size_t)img * SIM_BINS + t];
    const double po = (double)co / n;
    const double hgg = co ? -po * log2(po) : 0.0;
    const double MI = block_reduce<double>(mi, red, false, false);
    const double HGR = block_reduce<double>(hgr, red, false, false);
    const double HG = block_reduce<double>(hg, red, false, false);
    const double HR = block_reduce<double>(hr, red, false, false);
    const double HGG = block_reduce<double>(hgg, red, false, false);
    if (t == 0) {
        const double mx = st[0] / n, my = st[1] / n;
        double cs[3] = {0.0, 0.0, 0.0};
        for (int b = 0; b < nb; ++b)
            for (int k = 0; k < 3; ++k) cs[k] += w.part[((size_t)img * nb + b) * SIM_PART + k];
        const double vx = cs[0] / n, vy = cs[1] / n, cxy = cs[2] / n;
        const double L = st[9] - st[8];
        const double c1 = (0.01 * L) * (0.01 * L), c2 = (0.03 * L) * (0.03 * L);
        double* o = out + (size_t)img * 8;
        o[0] = sqrt(st[5] / n);
        o[1] = MI;
        o[2] = HGG;
        o[3] = HG > 0.0 ? fabs(HG - HR) / HG : fabs(HG - HR);
        o[4] = ((2 * mx * my + c1) * (2 * cxy + c2)) / ((mx * mx + my * my + c1) * (vx + vy + c2));
        o[5] = HG;
        o[6] = HR;
        o[7] = HGR;
    }
}

krig_status sim_fail(krig_status st, const std::string& msg)
{
    krig_internal_set_error(msg.c_str());
    return st;
}

}  // namespace

extern "C" size_t krig_similarity_workspace_bytes(int32_t n_img, int32_t H, int32_t W)
{
    if (n_img < 1 || H < 1 || W < 1) return 0;
    size_t total = 0;
    sim_layout(nullptr, n_img, sim_blocks((int64_t)H * W), &total);
    return total;
}

extern "C" krig_status krig_similarity(const float* d_G, const float* d_R, int32_t n_img, int32_t H, int32_t W,
                                       void* d_work, size_t work_bytes, double* d_out, void* stream)
{
    if (!d_G || !d_R || !d_out || !d_work) return sim_fail(KRIG_EINVAL, "d_G, d_R, d_work and d_out must not be NULL");
    if (n_img < 1 || n_img > 65535 || H < 1 || W < 1 || (int64_t)H * W > (1LL << 31))
        return sim_fail(KRIG_EINVAL, "n_img must be in [1, 65535] and H * W in [1, 2^31]");
    if ((uintptr_t)d_work % 256) return sim_fail(KRIG_EWORKSPACE, "workspace must be 256-byte aligned");
    const int64_t npix = (int64_t)H * W;
    const int nb = sim_blocks(npix);
    size_t need = 0;
    SimWork w = sim_layout(d_work, n_img, nb, &need);
    if (work_bytes < need)
        return sim_fail(KRIG_EWORKSPACE, "workspace too small: " + std::to_string(work_bytes) + " bytes, need " +
                                             std::to_string(need));
    cudaStream_t st = (cudaStream_t)stream;
    k_sim_partial<<<dim3(nb, n_img), SIM_THREADS, 0, st>>>(d_G, d_R, npix, w);
    k_sim_stats<<<n_img, SIM_THREADS, 0, st>>>(nb, npix, w);
    k_sim_hist<<<dim3(nb, n_img), SIM_THREADS, 0, st>>>(d_G, d_R, npix, w);
    k_sim_final<<<n_img, SIM_THREADS, 0, st>>>(w, nb, d_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sim_fail(KRIG_ECUDA, std::string("similarity launch: ") + cudaGetErrorString(e));
    return KRIG_OK;
}
