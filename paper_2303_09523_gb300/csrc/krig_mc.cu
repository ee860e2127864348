// krig_mc.cu -- marching cubes on the device (Appendix C): the triangle mesh of
// the iso-surface {v = iso} of a reconstructed volume, written as a triangle
// list into a caller-owned device buffer (no graphics API; the paper's display
// steps are outside this library).
//
// Appendix C describes the method: every cube of eight neighbouring voxels is
// classified by which corners lie inside (v > iso), one of 256 configurations
// held in a look-up table, and the surface crosses the cube's edges at the
// points found by linear interpolation of the corner values.  The paper prints
// no table.  Here the table is generated on the host from the cube's geometry:
//   * on each face of the cube the crossed edges are joined in pairs by
//     segments; a face with two diagonally opposite inside corners (the
//     ambiguous face) keeps the inside corners apart (each is cut off by its
//     own segment), a rule that depends only on the face, so neighbouring
//     cubes agree and the mesh has no holes;
//   * segments are directed so that, seen from outside the cube, the inside
//     corners lie on their right; every crossed edge then starts exactly one
//     segment (in one of its two faces) and ends one (in the other), and the
//     segments close into loops;
//   * each loop is cut into a fan of triangles from its vertex on the edge of
//     smallest index, in loop order; the triangles' normals (right-hand rule)
//     then point out of the inside region, from high values to low.
// Corner i of the cube at (x, y, z) is voxel (x + (i&1), y + ((i>>1)&1),
// z + (i>>2)); edge e joins the two corners listed in kEdge[e] (lower index
// first, one coordinate apart).  A vertex on edge (a, b) is at corner a plus
// t = (iso - v_a) / (v_b - v_a) along the edge (float32).
//
// Three launches: case of every cube and triangle counts per block of cubes;
// an exclusive scan of the block counts (one block); the triangles, each
// block placing its cubes' triangles in cube order after the earlier blocks'.
// The output order is deterministic: cubes in memory order (x fastest), a
// cube's triangles in table order.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>
#include <string>

#include "krig_internal.h"

namespace {

constexpr int MC_THREADS = 256;
constexpr int MC_PER_THREAD = 8;
constexpr int MC_CUBES = MC_THREADS * MC_PER_THREAD;  // cubes per block
constexpr int MC_SCAN_THREADS = 1024;

const int kEdge[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
// corners of each face in counter-clockwise order seen from outside the cube
const int kFace[6][4] = {{0, 4, 6, 2}, {1, 3, 7, 5}, {0, 1, 5, 4}, {2, 6, 7, 3}, {0, 2, 3, 1}, {4, 5, 7, 6}};

struct McTable {
    int8_t tri[256][16];  // edge indices, three per triangle, -1 after the last
    uint8_t ntri[256];
};

int edge_of(int a, int b)
{
    for (int e = 0; e < 12; ++e)
        if ((kEdge[e][0] == a && kEdge[e][1] == b) || (kEdge[e][0] == b && kEdge[e][1] == a)) return e;
    return -1;
}

void build_table(McTable& T)
{
    memset(&T, 0, sizeof(T));
    for (int c = 0; c < 256; ++c) {
        int next[12];
        for (int e = 0; e < 12; ++e) next[e] = -1;
        for (int f = 0; f < 6; ++f) {
            int in[4], E[4], cnt = 0;
            for (int i = 0; i < 4; ++i) {
                in[i] = (c >> kFace[f][i]) & 1;
                cnt += in[i];
                E[i] = edge_of(kFace[f][i], kFace[f][(i + 1) % 4]);  // between corner i and i + 1
            }
            if (cnt == 0 || cnt == 4) continue;
            if (cnt == 2 && in[0] == in[2]) {
                // ambiguous face: each inside corner i cut off alone, E_{i-1} -> E_i
                for (int i = 0; i < 4; ++i)
                    if (in[i]) next[E[(i + 3) % 4]] = E[i];
                continue;
            }
            // one run of inside corners a..b (cyclic): segment from the edge before the
            // run to the edge after it
            int a = 0;
            while (!(in[a] && !in[(a + 3) % 4])) ++a;
            int b = a;
            while (in[(b + 1) % 4]) b = (b + 1) % 4;
            next[E[(a + 3) % 4]] = E[b];
        }
        bool seen[12] = {false};
        int k = 0, nt = 0;
        for (int e0 = 0; e0 < 12; ++e0) {
            if (next[e0] < 0 || seen[e0]) continue;
            int loop[12], n = 0;
            for (int e = e0; !seen[e]; e = next[e]) {
                seen[e] = true;
                loop[n++] = e;
            }
            for (int i = 1; i + 1 < n; ++i) {
                T.tri[c][k++] = (int8_t)loop[0];
                T.tri[c][k++] = (int8_t)loop[i];
                T.tri[c][k++] = (int8_t)loop[i + 1];
                ++nt;
            }
        }
        for (; k < 16; ++k) T.tri[c][k] = -1;
        T.ntri[c] = (uint8_t)nt;
    }
}

const McTable& table()
{
    static McTable T;
    static std::once_flag once;
    std::call_once(once, [] { build_table(T); });
    return T;
}

struct McArgs {
    const float* vol;
    int D, H, W;
    float iso;
    int64_t ncubes;
    uint8_t* cases;      // [ncubes]
    int64_t* bsum;       // [nblocks + 1]: per-block triangle counts, then their exclusive scan
    float* tri;          // [max_tri][9]
    int64_t max_tri;
    int64_t* ntri;       // device, total
    uint64_t mcw, mch;   // krig_udiv multipliers: by W - 1, by H - 1
};

// Cube index -> (x, y, z), multiply-high divisions (cube < 2^32).
__device__ __forceinline__ void mc_xyz(const McArgs& a, int64_t cube, int& x, int& y, int& z)
{
    const uint32_t c = (uint32_t)cube;
    const uint32_t r = krig_udiv(c, a.mcw);
    x = (int)(c - r * (uint32_t)(a.W - 1));
    const uint32_t zz = krig_udiv(r, a.mch);
    y = (int)(r - zz * (uint32_t)(a.H - 1));
    z = (int)zz;
}

// Corner `end` (0: lower index, 1: upper) of edge e, the same list as kEdge:
// edges 0-3 run along x, 4-7 along y, 8-11 along z.
__device__ __forceinline__ int kEdgeDev(int e, int end)
{
    int a, d;
    if (e < 4) {
        a = 2 * e;
        d = 1;
    } else if (e < 8) {
        const int k = e - 4;
        a = (k & 1) + 4 * (k >> 1);
        d = 2;
    } else {
        a = e - 8;
        d = 4;
    }
    return end ? a + d : a;
}

__device__ __forceinline__ int mc_case(const McArgs& a, int64_t cube)
{
    int x, y, z;
    mc_xyz(a, cube, x, y, z);
    const size_t plane = (size_t)a.H * a.W;
    const float* p = a.vol + (size_t)z * plane + (size_t)y * a.W + x;
    int c = 0;
    c |= (p[0] > a.iso) << 0;
    c |= (p[1] > a.iso) << 1;
    c |= (p[a.W] > a.iso) << 2;
    c |= (p[a.W + 1] > a.iso) << 3;
    c |= (p[plane] > a.iso) << 4;
    c |= (p[plane + 1] > a.iso) << 5;
    c |= (p[plane + a.W] > a.iso) << 6;
    c |= (p[plane + a.W + 1] > a.iso) << 7;
    return c;
}

__global__ void __launch_bounds__(MC_THREADS) k_mc_classify(const McArgs a, const __grid_constant__ McTable T)
{
    __shared__ int red[MC_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * MC_CUBES;
    int cnt = 0;
    for (int k = 0; k < MC_PER_THREAD; ++k) {
        const int64_t cube = base + (int64_t)k * MC_THREADS + threadIdx.x;
        if (cube < a.ncubes) {
            const int c = mc_case(a, cube);
            a.cases[cube] = (uint8_t)c;
            cnt += T.ntri[c];
        }
    }
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int w = 0; w < MC_THREADS / 32; ++w) s += red[w];
        a.bsum[blockIdx.x] = s;
    }
}

// Exclusive scan of the nb block counts in place (one block), total into *ntri.
__global__ void __launch_bounds__(MC_SCAN_THREADS) k_mc_scan(const McArgs a, int64_t nb)
{
    __shared__ int64_t part[MC_SCAN_THREADS];
    const int t = threadIdx.x;
    const int64_t per = (nb + MC_SCAN_THREADS - 1) / MC_SCAN_THREADS;
    const int64_t lo = t * per, hi = lo + per < nb ? lo + per : nb;
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += a.bsum[i];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < MC_SCAN_THREADS; o <<= 1) {  // inclusive scan of the thread sums
        const int64_t v = t >= o ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = t > 0 ? part[t - 1] : 0;
    for (int64_t i = lo; i < hi; ++i) {
        const int64_t c = a.bsum[i];
        a.bsum[i] = run;
        run += c;
    }
    if (t == MC_SCAN_THREADS - 1) *a.ntri = part[t];
}

__global__ void __launch_bounds__(MC_THREADS) k_mc_emit(const McArgs a, const __grid_constant__ McTable T)
{
    __shared__ int wsum[MC_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * MC_CUBES;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // each thread owns MC_PER_THREAD consecutive cubes: the block's cubes in order
    int cs[MC_PER_THREAD], cnt = 0;
    for (int k = 0; k < MC_PER_THREAD; ++k) {
        const int64_t cube = base + (int64_t)threadIdx.x * MC_PER_THREAD + k;
        cs[k] = cube < a.ncubes ? a.cases[cube] : 0;
        cnt += T.ntri[cs[k]];
    }
    // exclusive scan of the thread counts across the block
    int incl = cnt;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    int woff = 0;
    for (int w = 0; w < warp; ++w) woff += wsum[w];
    int64_t out = a.bsum[blockIdx.x] + woff + incl - cnt;
    const size_t plane = (size_t)a.H * a.W;
    for (int k = 0; k < MC_PER_THREAD; ++k) {
        const int c = cs[k];
        if (!T.ntri[c]) continue;
        const int64_t cube = base + (int64_t)threadIdx.x * MC_PER_THREAD + k;
        int x, y, z;
        mc_xyz(a, cube, x, y, z);
        const float* p = a.vol + (size_t)z * plane + (size_t)y * a.W + x;
        float v[8];
        v[0] = p[0];
        v[1] = p[1];
        v[2] = p[a.W];
        v[3] = p[a.W + 1];
        v[4] = p[plane];
        v[5] = p[plane + 1];
        v[6] = p[plane + a.W];
        v[7] = p[plane + a.W + 1];
        for (int q = 0; q < T.ntri[c]; ++q, ++out) {
            if (out >= a.max_tri) continue;
            float* o = a.tri + out * 9;
            for (int m = 0; m < 3; ++m) {
                const int e = T.tri[c][3 * q + m];
                const int ca = kEdgeDev(e, 0), cb = kEdgeDev(e, 1);
                const float t = (a.iso - v[ca]) / (v[cb] - v[ca]);
                const int bit = ca ^ cb;  // the axis the edge runs along
                o[3 * m + 0] = (float)(x + (ca & 1)) + (bit == 1 ? t : 0.0f);
                o[3 * m + 1] = (float)(y + ((ca >> 1) & 1)) + (bit == 2 ? t : 0.0f);
                o[3 * m + 2] = (float)(z + (ca >> 2)) + (bit == 4 ? t : 0.0f);
            }
        }
    }
}

krig_status mc_fail(krig_status st, const std::string& msg)
{
    krig_internal_set_error(msg.c_str());
    return st;
}

size_t mc_layout(int64_t ncubes, int64_t* nblocks)
{
    const int64_t nb = (ncubes + MC_CUBES - 1) / MC_CUBES;
    *nblocks = nb;
    return ((size_t)ncubes + 255) / 256 * 256 + (size_t)(nb + 1) * sizeof(int64_t);
}

}  // namespace

extern "C" size_t krig_marching_cubes_workspace_bytes(int32_t D, int32_t H, int32_t W)
{
    if (D < 2 || H < 2 || W < 2) return 0;
    int64_t nb = 0;
    return mc_layout((int64_t)(D - 1) * (H - 1) * (W - 1), &nb);
}

extern "C" krig_status krig_marching_cubes(const float* d_vol, int32_t D, int32_t H, int32_t W, float iso, float* d_tri,
                                           int64_t max_tri, int64_t* d_ntri, void* d_work, size_t work_bytes,
                                           void* stream)
{
    if (!d_vol || !d_ntri || !d_work || (max_tri > 0 && !d_tri))
        return mc_fail(KRIG_EINVAL, "d_vol, d_ntri, d_work (and d_tri when max_tri > 0) must not be NULL");
    if (D < 2 || H < 2 || W < 2 || D > 65536 || H > 65536 || W > 65536)
        return mc_fail(KRIG_EINVAL, "D, H, W must be in [2, 65536]");
    if (max_tri < 0) return mc_fail(KRIG_EINVAL, "max_tri must be >= 0");
    if (!(iso == iso)) return mc_fail(KRIG_EINVAL, "iso must not be NaN");
    if ((uintptr_t)d_work % 256) return mc_fail(KRIG_EWORKSPACE, "workspace must be 256-byte aligned");
    const int64_t ncubes = (int64_t)(D - 1) * (H - 1) * (W - 1);
    int64_t nb = 0;
    const size_t need = mc_layout(ncubes, &nb);
    if (work_bytes < need)
        return mc_fail(KRIG_EWORKSPACE, "workspace too small: " + std::to_string(work_bytes) + " bytes, need " +
                                            std::to_string(need));
    if (ncubes >= (1LL << 32)) return mc_fail(KRIG_EINVAL, "volume too large: at most 2^32 - 1 cubes");
    McArgs a;
    a.vol = d_vol;
    a.D = D;
    a.H = H;
    a.W = W;
    a.iso = iso;
    a.ncubes = ncubes;
    a.cases = (uint8_t*)d_work;
    a.bsum = (int64_t*)((unsigned char*)d_work + ((size_t)ncubes + 255) / 256 * 256);
    a.tri = d_tri;
    a.max_tri = max_tri;
    a.ntri = d_ntri;
    a.mcw = krig_udiv_magic((uint32_t)(W - 1));
    a.mch = krig_udiv_magic((uint32_t)(H - 1));
    const McTable& T = table();
    cudaStream_t st = (cudaStream_t)stream;
    k_mc_classify<<<(unsigned)nb, MC_THREADS, 0, st>>>(a, T);
    k_mc_scan<<<1, MC_SCAN_THREADS, 0, st>>>(a, nb);
    k_mc_emit<<<(unsigned)nb, MC_THREADS, 0, st>>>(a, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mc_fail(KRIG_ECUDA, std::string("marching cubes launch: ") + cudaGetErrorString(e));
    return KRIG_OK;
}

// The generated case table (for tests and for callers that draw the mesh
// themselves): tri[256][16] edge indices (-1 terminated), ntri[256].
extern "C" void krig_marching_cubes_table(int8_t* tri_out, uint8_t* ntri_out)
{
    const McTable& T = table();
    if (tri_out) memcpy(tri_out, T.tri, sizeof(T.tri));
    if (ntri_out) memcpy(ntri_out, T.ntri, sizeof(T.ntri));
}
