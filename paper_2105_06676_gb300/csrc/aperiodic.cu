// StencilFFT-A for zero-Dirichlet grids (paper Sec. 5, Fig.
// "stencil-fft-algorithm-1D-aperiodic").
//
// The boundary's region of influence after T steps is the set of cells with
// dist <= sigma T, where dist(i) = min_a min(i_a + 1, l_a - i_a) and sigma is
// the stencil radius (Sec. 5.1). The result is assembled from
//   * the interior (dist > sigma T): the periodic solve of the whole grid,
//     whose spectrum is taken from the untouched input before the boundary
//     work starts and whose inverse writes only interior cells;
//   * the frame (dist <= sigma T): RecursiveBoundary, run in place on the grid.
//
// RecursiveBoundary(T) reads the grid at dist <= 2 sigma T and leaves the grid
// at time +T on dist <= sigma T (cells in (sigma T, 2 sigma T] are scratch
// afterwards). With T1 = floor(T/2) and T2 = T - T1 (odd T split as the
// paper's T/2 halves):
//   Step 1  P1: periodic solve for T1 of the strips holding dist <= 2 sigma T,
//               kept on sigma T1 < dist <= sigma T + sigma T2 (stashed);
//           RecursiveBoundary(T1) in place -> dist <= sigma T1 at time T1;
//           scatter P1 -> the grid holds time T1 on dist <= sigma T + sigma T2.
//   Step 2  P2: periodic solve for T2 of the strips holding that region, kept
//               on sigma T2 < dist <= sigma T (stashed);
//           RecursiveBoundary(T2) in place -> dist <= sigma T2 at time T;
//           scatter P2.
// Base case (T < cutoff): the direct loop with zero ghosts, temporally blocked
// in shared memory.
//
// A "periodic solve of the region" (the paper's Periodic(s, A, l_1..l_d, T/2))
// runs on face strips: for face (a, side) the box covering axis a over the
// region's width W (zero-padded to a power of two) and every other axis in
// full. A kept cell's dependence cone (radius sigma T_k) stays inside the
// strip and never crosses the grid boundary, so the periodic wrap of the box
// never reaches it. When a strip would span half an axis or more, one
// whole-grid solve replaces the 2d strips.
//
// Every strip is stored with its face-normal axis first (the grid region is
// gathered transposed when needed and solved with correspondingly permuted
// weights), so the long axes stay contiguous and all strips of a step with the
// same box shape run as one batched launch per pass.
//
// Execution: RecursiveBoundary's "parallel" blocks become concurrent streams.
// Each periodic solve's gather runs on the main stream (it reads the grid,
// which later main-stream work overwrites); its FFT passes run on a per-level
// branch stream and rejoin the main stream before the scatter that consumes
// them. From the second run for a given T and grid the whole schedule is
// replayed as one CUDA graph captured from those streams.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

namespace {

constexpr int kNoHi = 0x3fffffff;

// One strip (batch item): box axis a is grid axis perm[a]; box cell q is grid
// cell g with g[perm[a]] = off[perm[a]] + q[a] when q[a] < valid[a].
struct ItemGeom {
    int perm[3];
    int off[3];      // by grid axis
    int valid[3];    // by box axis
    int face_axis;   // grid face of the strip, -1 for the whole grid
    int face_side;
};

// Faces are numbered f = 2 a + side; the distance of cell g to face f is
// g_a + 1 (side 0) or l_a - g_a (side 1). A scatter writes the cells that are
// clear of every face (distance > lo[f] for all f) and within hi[f] of some
// face f (of its own face for a strip).
struct BatchGeom {
    int ndim;
    int gdims[3];
    int bdims[3];
    long long box_cells;
    int items;
    int lo[6], hi[6];
    ItemGeom it[kMaxItems];
};

// Some face f of the first ndim axes with distance(g, f) <= w[f].
__device__ __forceinline__ bool near_face(const int* g, const int* gd, int ndim, const int* w) {
    bool n = false;
    for (int a = 0; a < ndim; ++a) n |= (g[a] + 1 <= w[2 * a]) | (gd[a] - g[a] <= w[2 * a + 1]);
    return n;
}

__device__ __forceinline__ int face_distance(const int* g, const int* gd, int f) {
    return (f & 1) ? gd[f >> 1] - g[f >> 1] : g[f >> 1] + 1;
}

__device__ __forceinline__ bool item_cell(const BatchGeom& b, long long e, int* item, int* g) {
    *item = (int)(e / b.box_cells);
    long long rest = e - (long long)(*item) * b.box_cells;
    const ItemGeom& it = b.it[*item];
    bool in = true;
    for (int a = b.ndim - 1; a >= 0; --a) {
        const int q = (int)(rest % b.bdims[a]);
        rest /= b.bdims[a];
        in &= q < it.valid[a];
        g[it.perm[a]] = it.off[it.perm[a]] + q;
    }
    return in;
}

__device__ __forceinline__ long long grid_index(const int* g, const BatchGeom& b) {
    long long idx = 0;
    for (int a = 0; a < b.ndim; ++a) idx = idx * b.gdims[a] + g[a];
    return idx;
}

template <typename R>
__global__ void k_gather(const R* __restrict__ X, R* __restrict__ S,
                         const __grid_constant__ BatchGeom b, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int item, g[3];
        const bool in = item_cell(b, e, &item, g);
        S[e] = in ? X[grid_index(g, b)] : R(0);
    }
}

template <typename R>
__global__ void k_scatter(const R* __restrict__ S, R* __restrict__ X,
                          const __grid_constant__ BatchGeom b, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int item, g[3];
        if (!item_cell(b, e, &item, g)) continue;
        if (near_face(g, b.gdims, b.ndim, b.lo)) continue;
        const ItemGeom& it = b.it[item];
        if (it.face_axis >= 0) {
            const int f = 2 * it.face_axis + it.face_side;
            if (face_distance(g, b.gdims, f) > b.hi[f]) continue;
        } else if (!near_face(g, b.gdims, b.ndim, b.hi)) {
            continue;
        }
        X[grid_index(g, b)] = S[e];
    }
}

// ---------------------------------------------------------------------------
// base case: temporally blocked direct loop over output tiles of the frame
// ---------------------------------------------------------------------------
struct BaseTile {
    int lo[3], hi[3];  // output box in grid coordinates (hi exclusive)
};

struct BaseParams {
    int ndim;
    int gdims[3];
    int Tb;
    int mirror;       // reflecting boundary: ghosts mirror the cells inside (else zero)
    int wout[6];      // write cells within wout[f] of some face f
    double w[kMaxWeights];
    float wf[kMaxWeights];
};

template <typename R>
__device__ __forceinline__ R base_weight(const BaseParams& p, int i);
template <>
__device__ __forceinline__ float base_weight<float>(const BaseParams& p, int i) { return p.wf[i]; }
template <>
__device__ __forceinline__ double base_weight<double>(const BaseParams& p, int i) { return p.w[i]; }

template <typename R, int RAD>
__global__ void __launch_bounds__(512)
k_base_tiles(const R* __restrict__ X, R* __restrict__ Y, const BaseTile* __restrict__ tiles,
             const __grid_constant__ BaseParams p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int W = 2 * RAD + 1;
    const BaseTile t = tiles[blockIdx.x];
    const int h = RAD * p.Tb;
    int ilo[3] = {0, 0, 0}, ihi[3] = {1, 1, 1}, ext[3] = {1, 1, 1};
    const int off = 3 - p.ndim;  // work in 3-D with leading unit axes
    int olo[3] = {0, 0, 0}, ohi[3] = {1, 1, 1}, gd[3] = {1, 1, 1};
    for (int a = 0; a < p.ndim; ++a) {
        gd[off + a] = p.gdims[a];
        olo[off + a] = t.lo[a];
        ohi[off + a] = t.hi[a];
        ilo[off + a] = max(t.lo[a] - h, 0);
        ihi[off + a] = min(t.hi[a] + h, p.gdims[a]);
    }
    for (int a = 0; a < 3; ++a) ext[a] = ihi[a] - ilo[a];
    const int vol = ext[0] * ext[1] * ext[2];
    R* b0 = reinterpret_cast<R*>(smraw);
    R* b1 = b0 + vol;
    for (int e = threadIdx.x; e < vol; e += blockDim.x) {
        const int z = e / (ext[1] * ext[2]), y = (e / ext[2]) % ext[1], x = e % ext[2];
        const long long gi = ((long long)(ilo[0] + z) * gd[1] + (ilo[1] + y)) * gd[2] + (ilo[2] + x);
        b0[e] = X[gi];
    }
    __syncthreads();
    const int r0 = p.ndim >= 3 ? RAD : 0, r1 = p.ndim >= 2 ? RAD : 0;
    for (int step = 1; step <= p.Tb; ++step) {
        // cells within (Tb - step) * RAD of the output box are still needed
        const int reach = (p.Tb - step) * RAD;
        int clo[3], chi[3];
        for (int a = 0; a < 3; ++a) {
            clo[a] = max(olo[a] - reach, ilo[a]) - ilo[a];
            chi[a] = min(ohi[a] + reach, ihi[a]) - ilo[a];
        }
        const int cx = chi[2] - clo[2], cy = chi[1] - clo[1], cz = chi[0] - clo[0];
        const int cvol = cx * cy * cz;
        for (int e = threadIdx.x; e < cvol; e += blockDim.x) {
            const int z = clo[0] + e / (cx * cy), y = clo[1] + (e / cx) % cy, x = clo[2] + e % cx;
            R acc = 0;
            int wi = 0;
            for (int m0 = -r0; m0 <= r0; ++m0) {
                const int zz = z + m0;
                const bool zin = zz >= 0 && zz < ext[0];
                for (int m1 = -r1; m1 <= r1; ++m1) {
                    const int yy = y + m1;
                    const bool yin = zin && yy >= 0 && yy < ext[1];
#pragma unroll
                    for (int m2 = -RAD; m2 <= RAD; ++m2, ++wi) {
                        const int xx = x + m2;
                        if (yin && xx >= 0 && xx < ext[2])
                            acc += (R)p.w[wi] * b0[(zz * ext[1] + yy) * ext[2] + xx];
                    }
                }
            }
            b1[(z * ext[1] + y) * ext[2] + x] = acc;
        }
        __syncthreads();
        R* tmp = b0;
        b0 = b1;
        b1 = tmp;
    }
    (void)W;
    const int ox = ohi[2] - olo[2], oy = ohi[1] - olo[1], oz = ohi[0] - olo[0];
    const int ovol = ox * oy * oz;
    for (int e = threadIdx.x; e < ovol; e += blockDim.x) {
        int g3[3] = {olo[0] + e / (ox * oy), olo[1] + (e / ox) % oy, olo[2] + e % ox};
        if (!near_face(g3 + off, gd + off, p.ndim, p.wout)) continue;
        const int z = g3[0] - ilo[0], y = g3[1] - ilo[1], x = g3[2] - ilo[2];
        const long long gi = ((long long)g3[0] * gd[1] + g3[1]) * gd[2] + g3[2];
        Y[gi] = b0[(z * ext[1] + y) * ext[2] + x];
    }
}

template <typename R>
__global__ void k_tile_copy(const R* __restrict__ Y, R* __restrict__ X,
                            const BaseTile* __restrict__ tiles, const __grid_constant__ BaseParams p) {
    const BaseTile t = tiles[blockIdx.x];
    int lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1}, gd[3] = {1, 1, 1};
    const int off = 3 - p.ndim;
    for (int a = 0; a < p.ndim; ++a) {
        lo[off + a] = t.lo[a];
        hi[off + a] = t.hi[a];
        gd[off + a] = p.gdims[a];
    }
    const int ox = hi[2] - lo[2], oy = hi[1] - lo[1], oz = hi[0] - lo[0];
    for (int e = threadIdx.x; e < ox * oy * oz; e += blockDim.x) {
        int g3[3] = {lo[0] + e / (ox * oy), lo[1] + (e / ox) % oy, lo[2] + e % ox};
        if (!near_face(g3 + off, gd + off, p.ndim, p.wout)) continue;
        const long long gi = ((long long)g3[0] * gd[1] + g3[1]) * gd[2] + g3[2];
        X[gi] = Y[gi];
    }
}

// Reflecting boundary in the zero-ring tile layout: before every step the
// ring cells that lie outside the grid take the current value of their mirror
// image (ghost -1-k <- cell k, ghost l+k <- cell l-1-k), axis by axis so that
// corner ghosts mirror in every axis. `padded` is the tile's extent plus the
// ring per axis (3 axes, leading unit axes for 1-D / 2-D tiles), `lo_out` /
// `hi_out` say which sides of the tile touch the grid boundary; the mirror
// images lie inside the tile (it covers the first / last RAD cells of an axis
// it touches). Contains CTA barriers: call it from every thread.
template <typename R, int RAD>
__device__ __forceinline__ void mirror_ring(R* b, const int* padded, const bool* lo_out,
                                            const bool* hi_out) {
    const int px = padded[2], py = padded[1], pz = padded[0];
    for (int ax = 2; ax >= 0; --ax) {
        if (!lo_out[ax] && !hi_out[ax]) continue;
        const int len = padded[ax];
        // lines along the other two axes: every cell of the padded box whose
        // coordinate on ax is a ghost of a boundary side
        const int others = (pz * py * px) / len;
        for (int e = threadIdx.x; e < others * 2 * RAD; e += blockDim.x) {
            const int line = e / (2 * RAD), g = e - line * 2 * RAD;
            const bool low = g < RAD;
            const int k = low ? g : g - RAD;
            if (low ? !lo_out[ax] : !hi_out[ax]) continue;
            const int dst = low ? RAD - 1 - k : len - RAD + k;
            const int src = low ? RAD + k : len - RAD - 1 - k;
            int c[3];
            // split `line` over the two axes other than ax
            int rest = line;
            for (int a = 2; a >= 0; --a) {
                if (a == ax) continue;
                c[a] = rest % padded[a];
                rest /= padded[a];
            }
            c[ax] = dst;
            const int di = (c[0] * py + c[1]) * px + c[2];
            c[ax] = src;
            const int si = (c[0] * py + c[1]) * px + c[2];
            b[di] = b[si];
        }
        __syncthreads();
    }
}

// 2-D base case: the tile (output box plus a halo of RAD*T_b, clipped to the
// grid) lives in shared memory with a ring of RAD zero cells around it, so the
// stencil reads need no bounds tests; each thread owns columns of the tile and
// walks its rows. Reads beyond the tile are the zero ring: outside the grid
// that is the boundary condition, inside the grid it only reaches cells whose
// values never propagate to the output box within T_b steps.
// Rows of outputs one thread computes per item of the 2-D base case.
constexpr int kBaseRun = 8;

template <typename R, int RAD>
__global__ void __launch_bounds__(512)
k_base_2d(const R* __restrict__ X, R* __restrict__ Y, const BaseTile* __restrict__ tiles,
          const __grid_constant__ BaseParams p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int W = 2 * RAD + 1;
    const BaseTile t = tiles[blockIdx.x];
    const int L0 = p.gdims[0], L1 = p.gdims[1];
    const int h = RAD * p.Tb;
    const int iy0 = max(t.lo[0] - h, 0), iy1 = min(t.hi[0] + h, L0);
    const int ix0 = max(t.lo[1] - h, 0), ix1 = min(t.hi[1] + h, L1);
    const int ey = iy1 - iy0, ex = ix1 - ix0;
    const int pitch = ex + 2 * RAD;
    const int cells = (ey + 2 * RAD) * pitch;
    R* b0 = reinterpret_cast<R*>(smraw);
    R* b1 = b0 + cells;
    for (int e = threadIdx.x; e < 2 * cells; e += blockDim.x) b0[e] = R(0);
    __syncthreads();
    for (int e = threadIdx.x; e < ey * ex; e += blockDim.x) {
        const int y = e / ex, x = e - y * ex;
        b0[(y + RAD) * pitch + x + RAD] = X[(long long)(iy0 + y) * L1 + ix0 + x];
    }
    R w[W * W];
#pragma unroll
    for (int i = 0; i < W * W; ++i) w[i] = (R)p.w[i];
    __syncthreads();
    const bool lo_out[3] = {false, iy0 == 0, ix0 == 0}, hi_out[3] = {false, iy1 == L0, ix1 == L1};
    const int padded[3] = {1, ey + 2 * RAD, pitch};
    const bool refl = p.mirror && (lo_out[1] || lo_out[2] || hi_out[1] || hi_out[2]);
    for (int step = 1; step <= p.Tb; ++step) {
        if (refl) mirror_ring<R, RAD>(b0, padded, lo_out, hi_out);
        const int reach = (p.Tb - step) * RAD;
        const int cy0 = max(t.lo[0] - reach, iy0) - iy0, cy1 = min(t.hi[0] + reach, iy1) - iy0;
        const int cx0 = max(t.lo[1] - reach, ix0) - ix0, cx1 = min(t.hi[1] + reach, ix1) - ix0;
        // each item is a column x and a run of kBaseRun rows: the W neighbours
        // of an input row are read once and added, slice by slice, into a
        // window of W accumulators; while padded input row yi is added, acc[i]
        // is output row yi - 2 RAD + i, and after it acc[0] is complete
        const int nx = cx1 - cx0, nruns = (cy1 - cy0 + kBaseRun - 1) / kBaseRun;
        for (int item = threadIdx.x; item < nx * nruns; item += blockDim.x) {
            const int run = item / nx, x = cx0 + item - run * nx;
            const int ya = cy0 + run * kBaseRun, yb = min(ya + kBaseRun, cy1);
            R acc[W];
#pragma unroll
            for (int i = 0; i < W; ++i) acc[i] = R(0);
            // padded input rows ya .. yb + 2 RAD - 1 feed outputs ya .. yb - 1
            for (int yi = ya; yi < yb + 2 * RAD; ++yi) {
                const R* src = b0 + yi * pitch + x;
                R nb[W];
#pragma unroll
                for (int m1 = 0; m1 < W; ++m1) nb[m1] = src[m1];
#pragma unroll
                for (int i = 0; i < W; ++i) {
                    R sacc = 0;
#pragma unroll
                    for (int m1 = 0; m1 < W; ++m1) sacc += w[(W - 1 - i) * W + m1] * nb[m1];
                    acc[i] += sacc;
                }
                const int yo = yi - 2 * RAD;    // output row whose window closed
                if (yo >= ya) b1[(yo + RAD) * pitch + x + RAD] = acc[0];
#pragma unroll
                for (int i = 0; i + 1 < W; ++i) acc[i] = acc[i + 1];
                acc[W - 1] = R(0);
            }
        }
        __syncthreads();
        R* tmp = b0;
        b0 = b1;
        b1 = tmp;
    }
    const int oy = t.hi[0] - t.lo[0], ox = t.hi[1] - t.lo[1];
    for (int e = threadIdx.x; e < oy * ox; e += blockDim.x) {
        const int gy = t.lo[0] + e / ox, gx = t.lo[1] + e % ox;
        const int g2[2] = {gy, gx};
        if (!near_face(g2, p.gdims, 2, p.wout)) continue;
        Y[(long long)gy * L1 + gx] = b0[(gy - iy0 + RAD) * pitch + gx - ix0 + RAD];
    }
}

// 1-D and 3-D base cases with the same zero-ring layout as k_base_2d (no
// bounds tests in the stencil loop, no divisions per cell).
template <typename R, int RAD>
__global__ void __launch_bounds__(256)
k_base_1d(const R* __restrict__ X, R* __restrict__ Y, const BaseTile* __restrict__ tiles,
          const __grid_constant__ BaseParams p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int W = 2 * RAD + 1;
    const BaseTile t = tiles[blockIdx.x];
    const int L = p.gdims[0];
    const int h = RAD * p.Tb;
    const int i0 = max(t.lo[0] - h, 0), i1 = min(t.hi[0] + h, L);
    const int ex = i1 - i0;
    const int cells = ex + 2 * RAD;
    R* b0 = reinterpret_cast<R*>(smraw);
    R* b1 = b0 + cells;
    for (int e = threadIdx.x; e < 2 * cells; e += blockDim.x) b0[e] = R(0);
    __syncthreads();
    for (int e = threadIdx.x; e < ex; e += blockDim.x) b0[e + RAD] = X[i0 + e];
    R w[W];
#pragma unroll
    for (int i = 0; i < W; ++i) w[i] = (R)p.w[i];
    __syncthreads();
    const bool lo_out[3] = {false, false, i0 == 0}, hi_out[3] = {false, false, i1 == L};
    const int padded[3] = {1, 1, cells};
    const bool refl = p.mirror && (lo_out[2] || hi_out[2]);
    for (int step = 1; step <= p.Tb; ++step) {
        if (refl) mirror_ring<R, RAD>(b0, padded, lo_out, hi_out);
        const int reach = (p.Tb - step) * RAD;
        const int c0 = max(t.lo[0] - reach, i0) - i0, c1 = min(t.hi[0] + reach, i1) - i0;
        for (int x = c0 + threadIdx.x; x < c1; x += blockDim.x) {
            R acc = 0;
#pragma unroll
            for (int m = 0; m < W; ++m) acc += w[m] * b0[x + m];
            b1[x + RAD] = acc;
        }
        __syncthreads();
        R* tmp = b0;
        b0 = b1;
        b1 = tmp;
    }
    for (int g = t.lo[0] + threadIdx.x; g < t.hi[0]; g += blockDim.x) {
        if (g + 1 <= p.wout[0] || L - g <= p.wout[1]) Y[g] = b0[g - i0 + RAD];
    }
}

template <typename R, int RAD>
__global__ void __launch_bounds__(256)
k_base_3d(const R* __restrict__ X, R* __restrict__ Y, const BaseTile* __restrict__ tiles,
          const __grid_constant__ BaseParams p) {
    extern __shared__ __align__(16) unsigned char smraw[];
    constexpr int W = 2 * RAD + 1;
    const BaseTile t = tiles[blockIdx.x];
    const int L0 = p.gdims[0], L1 = p.gdims[1], L2 = p.gdims[2];
    const int h = RAD * p.Tb;
    int lo[3], hi[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        lo[a] = max(t.lo[a] - h, 0);
        hi[a] = min(t.hi[a] + h, p.gdims[a]);
        ext[a] = hi[a] - lo[a];
    }
    const int px = ext[2] + 2 * RAD, py = ext[1] + 2 * RAD;
    const int plane = px * py;
    const int cells = (ext[0] + 2 * RAD) * plane;
    R* b0 = reinterpret_cast<R*>(smraw);
    R* b1 = b0 + cells;
    for (int e = threadIdx.x; e < 2 * cells; e += blockDim.x) b0[e] = R(0);
    __syncthreads();
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5, ny = blockDim.x >> 5;
    for (int zy = ty; zy < ext[0] * ext[1]; zy += ny) {
        const int z = zy / ext[1], y = zy - z * ext[1];
        for (int x = tx; x < ext[2]; x += 32)
            b0[(z + RAD) * plane + (y + RAD) * px + x + RAD] =
                X[((long long)(lo[0] + z) * L1 + lo[1] + y) * L2 + lo[2] + x];
    }
    __syncthreads();
    bool lo_out[3], hi_out[3];
    bool any_out = false;
    for (int a = 0; a < 3; ++a) {
        lo_out[a] = lo[a] == 0;
        hi_out[a] = hi[a] == p.gdims[a];
        any_out |= lo_out[a] || hi_out[a];
    }
    const int padded[3] = {ext[0] + 2 * RAD, py, px};
    const bool refl = p.mirror && any_out;
    for (int step = 1; step <= p.Tb; ++step) {
        if (refl) mirror_ring<R, RAD>(b0, padded, lo_out, hi_out);
        const int reach = (p.Tb - step) * RAD;
        int c0[3], c1[3];
        for (int a = 0; a < 3; ++a) {
            c0[a] = max(t.lo[a] - reach, lo[a]) - lo[a];
            c1[a] = min(t.hi[a] + reach, hi[a]) - lo[a];
        }
        const int cy = c1[1] - c0[1], cz = c1[0] - c0[0];
        for (int zy = ty; zy < cz * cy; zy += ny) {
            const int z = c0[0] + zy / cy, y = c0[1] + zy % cy;
            for (int x = c0[2] + tx; x < c1[2]; x += 32) {
                const R* src = b0 + z * plane + y * px + x;
                R acc = 0;
#pragma unroll
                for (int m0 = 0; m0 < W; ++m0)
#pragma unroll
                    for (int m1 = 0; m1 < W; ++m1)
#pragma unroll
                        for (int m2 = 0; m2 < W; ++m2)
                            acc += base_weight<R>(p, (m0 * W + m1) * W + m2) *
                                   src[m0 * plane + m1 * px + m2];
                b1[(z + RAD) * plane + (y + RAD) * px + x + RAD] = acc;
            }
        }
        __syncthreads();
        R* tmp = b0;
        b0 = b1;
        b1 = tmp;
    }
    const int oy = t.hi[1] - t.lo[1], oz = t.hi[0] - t.lo[0];
    for (int zy = ty; zy < oz * oy; zy += ny) {
        const int gz = t.lo[0] + zy / oy, gy = t.lo[1] + zy % oy;
        for (int gx = t.lo[2] + tx; gx < t.hi[2]; gx += 32) {
            const int g3[3] = {gz, gy, gx};
            if (!near_face(g3, p.gdims, 3, p.wout)) continue;
            Y[((long long)gz * L1 + gy) * L2 + gx] =
                b0[(gz - lo[0] + RAD) * plane + (gy - lo[1] + RAD) * px + gx - lo[2] + RAD];
        }
    }
}

// One step of the loop on the whole 3-D grid with zero ghosts, one output per
// thread gathered directly (used for FP64, where the double-precision FMA
// rate, not the loads, sets the time and a streamed chunk's recomputed halo
// planes would cost FMAs).
template <typename R, int RAD>
__global__ void __launch_bounds__(256)
k_step_3d(const R* __restrict__ A, R* __restrict__ B, const __grid_constant__ BaseParams p) {
    constexpr int W = 2 * RAD + 1;
    const int L0 = p.gdims[0], L1 = p.gdims[1], L2 = p.gdims[2];
    const long long n = (long long)L0 * L1 * L2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n;
         e += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(e % L2);
        const long long zy = e / L2;
        const int y = (int)(zy % L1), z = (int)(zy / L1);
        R acc = 0;
#pragma unroll
        for (int m0 = 0; m0 < W; ++m0) {
            const int zz = z + m0 - RAD;
            if (zz < 0 || zz >= L0) continue;
#pragma unroll
            for (int m1 = 0; m1 < W; ++m1) {
                const int yy = y + m1 - RAD;
                if (yy < 0 || yy >= L1) continue;
                const R* row = A + ((long long)zz * L1 + yy) * L2;
#pragma unroll
                for (int m2 = 0; m2 < W; ++m2) {
                    const int xx = x + m2 - RAD;
                    if (xx >= 0 && xx < L2)
                        acc += base_weight<R>(p, (m0 * W + m1) * W + m2) * __ldg(row + xx);
                }
            }
        }
        B[e] = acc;
    }
}

// One step of the loop on the whole 3-D grid, streamed along axis 0: a CTA
// owns a TY x TX tile of (axis 1, axis 2), TX x TY = 256 with TX matched to
// the grid's contiguous axis, and a chunk of axis-0
// planes. Each input plane (with an r-cell halo, zeros outside the grid) is
// staged once in shared memory; every thread reads its (2r+1)^2 neighbours
// into registers and adds them, slice by slice, into a window of 2r+1
// accumulators for the outputs z = p - r .. p + r. The oldest one is complete
// after plane p and is stored. Per output: (2r+1)^2 shared loads and (2r+1)^3
// FMAs, against (2r+1)^3 global loads for a direct gather.
constexpr int kStepThreads = 256;

template <typename R, int RAD, int TX>
__global__ void __launch_bounds__(kStepThreads)
k_step_3d_stream(const R* __restrict__ A, R* __restrict__ B, const __grid_constant__ BaseParams p,
                 int zchunk) {
    constexpr int W = 2 * RAD + 1;
    constexpr int TY = kStepThreads / TX;
    constexpr int PX = TX + 2 * RAD, PY = TY + 2 * RAD;
    __shared__ R plane[PY][PX];
    const int L0 = p.gdims[0], L1 = p.gdims[1], L2 = p.gdims[2];
    const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * zchunk, z1 = min(L0, z0 + zchunk);
    const int x = x0 + tx, y = y0 + ty;
    R acc[W];
#pragma unroll
    for (int i = 0; i < W; ++i) acc[i] = 0;
    for (int pz = z0 - RAD; pz < z1 + RAD; ++pz) {
        const bool in = pz >= 0 && pz < L0;
        if (in) {
            const R* src = A + (long long)pz * L1 * L2;
            for (int e = threadIdx.x; e < PX * PY; e += kStepThreads) {
                const int py = e / PX, px = e - py * PX;
                const int gy = y0 + py - RAD, gx = x0 + px - RAD;
                plane[py][px] = (gy >= 0 && gy < L1 && gx >= 0 && gx < L2)
                                    ? __ldg(src + (long long)gy * L2 + gx) : R(0);
            }
        }
        __syncthreads();
        if (in) {
            R nb[W][W];
#pragma unroll
            for (int m1 = 0; m1 < W; ++m1)
#pragma unroll
                for (int m2 = 0; m2 < W; ++m2) nb[m1][m2] = plane[ty + m1][tx + m2];
            // acc[i] is output z = pz - RAD + i, which takes this plane with m0 = RAD - i
#pragma unroll
            for (int i = 0; i < W; ++i) {
                R s = 0;
#pragma unroll
                for (int m1 = 0; m1 < W; ++m1)
#pragma unroll
                    for (int m2 = 0; m2 < W; ++m2)
                        s += base_weight<R>(p, ((W - 1 - i) * W + m1) * W + m2) * nb[m1][m2];
                acc[i] += s;
            }
        }
        __syncthreads();
        const int zo = pz - RAD;
        if (zo >= z0 && zo < z1 && y < L1 && x < L2)
            B[((long long)zo * L1 + y) * L2 + x] = acc[0];
#pragma unroll
        for (int i = 0; i + 1 < W; ++i) acc[i] = acc[i + 1];
        acc[W - 1] = 0;
    }
}

// The whole loop (paper Sec. 1 "Problem Specification", zero ghosts) for a
// grid small enough to live in the shared memory of one thread-block cluster:
// CTA `rank` keeps planes [rank S, (rank + 1) S) of axis 0 plus r ghost planes
// on each side, every plane padded with a zero ring of width r, in two
// buffers. Each step computes the CTA's own planes from `cur` into `nxt`
// (axis-0 register window as in k_step_3d_stream), pushes its first and last
// r planes into the neighbours' `nxt` ghost planes through distributed shared
// memory, and meets the cluster at one barrier; the grid is read once at the
// start and written once at the end. Ghost planes beyond the grid and the
// rings are never written, so they stay zero.
namespace cgx = cooperative_groups;

constexpr int kClusterThreads = 512;

struct ClusterGeom {
    int S;          // own planes (axis 0) per CTA
    int L1p, L2p;   // padded plane extents (1 for absent axes)
    int P;          // elements per padded plane
    int Q;          // interior cells per plane
    int G;          // axis-0 groups of threads per CTA
};

struct ClusterPlan {
    bool ok = false;
    int cs = 0;        // CTAs in the cluster
    ClusterGeom g{};
    size_t smem = 0;   // dynamic shared memory per CTA
};

constexpr int kClusterSmemMax = 226 * 1024;

template <typename R, int RAD, int D>
__global__ void __launch_bounds__(kClusterThreads)
k_loop_cluster(R* __restrict__ grid, const __grid_constant__ BaseParams p,
               const __grid_constant__ ClusterGeom cg, long long T) {
    constexpr int W = 2 * RAD + 1;
    constexpr int RY = D >= 2 ? RAD : 0, RX = D == 3 ? RAD : 0;
    extern __shared__ __align__(16) unsigned char smraw[];
    cgx::cluster_group cluster = cgx::this_cluster();
    const int rank = (int)cluster.block_rank(), nrank = (int)cluster.num_blocks();
    const int planes = cg.S + 2 * RAD;
    const int bufsz = planes * cg.P;
    R* cur = reinterpret_cast<R*>(smraw);
    R* nxt = cur + bufsz;
    const int L0 = p.gdims[0], L1 = D >= 2 ? p.gdims[1] : 1, L2 = D == 3 ? p.gdims[2] : 1;
    const int z0 = rank * cg.S;   // grid plane of local plane RAD
    for (int e = threadIdx.x; e < 2 * bufsz; e += blockDim.x) cur[e] = R(0);
    __syncthreads();
    for (int e = threadIdx.x; e < planes * cg.Q; e += blockDim.x) {
        const int pl = e / cg.Q, qi = e - pl * cg.Q;
        const int gz = z0 + pl - RAD;
        if (gz < 0 || gz >= L0) continue;
        const int y = qi / L2, x = qi - (qi / L2) * L2;
        cur[pl * cg.P + (y + RY) * cg.L2p + x + RX] = grid[((long long)gz * L1 + y) * L2 + x];
    }
    // every CTA's buffers are initialised before any neighbour pushes into them
    cluster.sync();
    for (long long t = 0; t < T; ++t) {
        for (int item = threadIdx.x; item < cg.G * cg.Q; item += blockDim.x) {
            const int g = item / cg.Q, qi = item - g * cg.Q;
            const int za = g * cg.S / cg.G, zb = (g + 1) * cg.S / cg.G;
            const int y = qi / L2, x = qi - (qi / L2) * L2;
            const int c0 = (y + RY) * cg.L2p + x + RX;
            R acc[W];
#pragma unroll
            for (int i = 0; i < W; ++i) acc[i] = R(0);
            // output plane o (local) takes input planes o - r .. o + r; while
            // input plane pl is added, acc[i] is output plane pl - r + i, and
            // after it acc[0] (plane pl - r) is complete
            for (int pl = za; pl < zb + 2 * RAD; ++pl) {
                const R* src = cur + pl * cg.P + c0;
                if constexpr (D == 3) {
                    R nb[W][W];
#pragma unroll
                    for (int m1 = 0; m1 < W; ++m1)
#pragma unroll
                        for (int m2 = 0; m2 < W; ++m2) nb[m1][m2] = src[(m1 - RAD) * cg.L2p + m2 - RAD];
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        R sacc = 0;
#pragma unroll
                        for (int m1 = 0; m1 < W; ++m1)
#pragma unroll
                            for (int m2 = 0; m2 < W; ++m2)
                                sacc += base_weight<R>(p, ((W - 1 - i) * W + m1) * W + m2) * nb[m1][m2];
                        acc[i] += sacc;
                    }
                } else if constexpr (D == 2) {
                    R nb[W];
#pragma unroll
                    for (int m1 = 0; m1 < W; ++m1) nb[m1] = src[m1 - RAD];
#pragma unroll
                    for (int i = 0; i < W; ++i) {
                        R sacc = 0;
#pragma unroll
                        for (int m1 = 0; m1 < W; ++m1)
                            sacc += base_weight<R>(p, (W - 1 - i) * W + m1) * nb[m1];
                        acc[i] += sacc;
                    }
                } else {
                    const R v = src[0];
#pragma unroll
                    for (int i = 0; i < W; ++i) acc[i] += base_weight<R>(p, W - 1 - i) * v;
                }
                if (pl >= za + 2 * RAD) nxt[(pl - RAD) * cg.P + c0] = acc[0];
#pragma unroll
                for (int i = 0; i + 1 < W; ++i) acc[i] = acc[i + 1];
                acc[W - 1] = R(0);
            }
        }
        __syncthreads();
        // own first r planes -> lower neighbour's upper ghosts, own last r
        // planes -> upper neighbour's lower ghosts
        if (RAD > 0) {
            const int span = RAD * cg.P;
            if (rank > 0) {
                R* dst = cluster.map_shared_rank(nxt, rank - 1) + (cg.S + RAD) * cg.P;
                const R* srcp = nxt + RAD * cg.P;
                for (int e = threadIdx.x; e < span; e += blockDim.x) dst[e] = srcp[e];
            }
            if (rank + 1 < nrank) {
                R* dst = cluster.map_shared_rank(nxt, rank + 1);
                const R* srcp = nxt + cg.S * cg.P;
                for (int e = threadIdx.x; e < span; e += blockDim.x) dst[e] = srcp[e];
            }
        }
        cluster.sync();
        R* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    for (int e = threadIdx.x; e < cg.S * cg.Q; e += blockDim.x) {
        const int pl = e / cg.Q, qi = e - pl * cg.Q;
        const int y = qi / L2, x = qi - (qi / L2) * L2;
        grid[((long long)(z0 + pl) * L1 + y) * L2 + x] =
            cur[(pl + RAD) * cg.P + (y + RY) * cg.L2p + x + RX];
    }
}

// 2-D gather and scatter of batch items in 32 x 32 tiles of the box. A
// transposed item (perm = (1, 0)) goes through a shared tile so that both the
// grid side and the box side are accessed along their contiguous axis.
template <typename R, bool SCATTER>
__global__ void __launch_bounds__(256)
k_copy_2d(R* __restrict__ X, R* __restrict__ S, const __grid_constant__ BatchGeom b) {
    __shared__ R tile[32][33];
    const int item = blockIdx.z;
    const ItemGeom& it = b.it[item];
    const int B0 = b.bdims[0], B1 = b.bdims[1];
    const int L0 = b.gdims[0], L1 = b.gdims[1];
    R* Sb = S + (long long)item * b.box_cells;
    const int q0b = blockIdx.y * 32, q1b = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
    const bool transposed = it.perm[0] == 1;
    if (SCATTER && it.face_axis >= 0) {
        // kept cells have distance to the strip's face in (lo[f], hi[f]]; the
        // face normal is box axis 0, so only box rows in that band can be written
        const int a = it.face_axis, offn = it.off[a], Ln = a == 0 ? L0 : L1;
        const int f = 2 * a + it.face_side;
        const int klo = it.face_side == 0 ? b.lo[f] - offn : Ln - offn - b.hi[f];
        const int khi = it.face_side == 0 ? b.hi[f] - offn : Ln - offn - b.lo[f];
        if (q0b >= khi || q0b + 32 <= klo) return;
    }
    auto keep = [&](int g0, int g1) {
        const int g[2] = {g0, g1};
        if (near_face(g, b.gdims, 2, b.lo)) return false;
        if (it.face_axis >= 0) {
            const int f = 2 * it.face_axis + it.face_side;
            return face_distance(g, b.gdims, f) <= b.hi[f];
        }
        return near_face(g, b.gdims, 2, b.hi);
    };
    if (!transposed) {
        for (int r = ty; r < 32; r += 8) {
            const int q0 = q0b + r, q1 = q1b + tx;
            if (q0 >= B0 || q1 >= B1) continue;
            const bool in = q0 < it.valid[0] && q1 < it.valid[1];
            const int g0 = it.off[0] + q0, g1 = it.off[1] + q1;
            if (!SCATTER) {
                Sb[(long long)q0 * B1 + q1] = in ? X[(long long)g0 * L1 + g1] : R(0);
            } else if (in && keep(g0, g1)) {
                X[(long long)g0 * L1 + g1] = Sb[(long long)q0 * B1 + q1];
            }
        }
        return;
    }
    // transposed: box (q0, q1) <-> grid (g0 = off0 + q1, g1 = off1 + q0)
    if (!SCATTER) {
        for (int r = ty; r < 32; r += 8) {
            const int q1 = q1b + r, q0 = q0b + tx;       // read grid row g0 = off0 + q1 along g1
            R v = R(0);
            if (q0 < it.valid[0] && q1 < it.valid[1])
                v = X[(long long)(it.off[0] + q1) * L1 + it.off[1] + q0];
            tile[r][tx] = v;
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int q0 = q0b + r, q1 = q1b + tx;
            if (q0 < B0 && q1 < B1) Sb[(long long)q0 * B1 + q1] = tile[tx][r];
        }
    } else {
        for (int r = ty; r < 32; r += 8) {
            const int q0 = q0b + r, q1 = q1b + tx;       // read box row q0 along q1
            tile[r][tx] = (q0 < B0 && q1 < B1) ? Sb[(long long)q0 * B1 + q1] : R(0);
        }
        __syncthreads();
        for (int r = ty; r < 32; r += 8) {
            const int q1 = q1b + r, q0 = q0b + tx;
            if (q0 >= it.valid[0] || q1 >= it.valid[1]) continue;
            const int g0 = it.off[0] + q1, g1 = it.off[1] + q0;
            if (keep(g0, g1)) X[(long long)g0 * L1 + g1] = tile[tx][r];
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(256)
k_tile_copy_2d(const R* __restrict__ Y, R* __restrict__ X, const BaseTile* __restrict__ tiles,
               const __grid_constant__ BaseParams p) {
    const BaseTile t = tiles[blockIdx.x];
    const int L0 = p.gdims[0], L1 = p.gdims[1];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    for (int y = t.lo[0] + ty; y < t.hi[0]; y += 8)
        for (int x = t.lo[1] + tx; x < t.hi[1]; x += 32) {
            const int g2[2] = {y, x};
            if (!near_face(g2, p.gdims, 2, p.wout)) continue;
            const long long gi = (long long)y * L1 + x;
            X[gi] = Y[gi];
        }
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

int grid_blocks(long long total) {
    long long b = (total + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 16));
}

}  // namespace

// ---------------------------------------------------------------------------
// host: schedule, buffers, streams, graphs
// ---------------------------------------------------------------------------
struct Batch {                 // items of one step with equal box shape
    int64_t bdims[3];
    BatchGeom geom;
    int norient;
    int perms[kMaxOrient][3];
    int orient[kMaxItems];
    size_t s_off, h_off;       // byte offsets into the level's buffers
    int vt[kMaxOrient];        // multiplier table per orientation (-1: none)
};

// Lambda^T / N for one (T, box shape, orientation), built once per run and
// shared by every strip solve with those parameters.
struct VTable {
    int64_t T;
    int64_t bdims[3];
    int perm[3];
    void* buf = nullptr;
};

struct Step {                  // all periodic solves of one P1 or P2 step
    int level;
    int64_t T;
    std::vector<Batch> batches;
};

struct Op {
    // SOLVE / SCATTER: a periodic strip solve and its write-back (step index);
    // BASE: a RecursiveBoundary leaf, T steps of the loop on the frame;
    // LOOP: T steps of the loop on the whole grid (temporally blocked tiles);
    // STEP: T single-step launches of the loop on the whole grid (3-D);
    // CLUSTER: T steps of the loop in one thread-block cluster's shared memory
    enum Kind { SOLVE, SCATTER, BASE, LOOP, STEP, CLUSTER } kind;
    int step;
    int64_t T;
};

struct BaseSet {
    void* tiles = nullptr;     // device BaseTile[count]
    int count = 0;
    size_t smem = 0;
};

struct Schedule {
    std::vector<Step> steps;
    std::vector<Op> ops;
    std::vector<VTable> tables;
    bool loop = false;         // the plain loop over the whole grid (no interior solve)
    ClusterPlan cluster;       // launch shape of an Op::CLUSTER
};

struct LevelBuffers {
    void* S = nullptr;
    void* H = nullptr;
    size_t S_bytes = 0, H_bytes = 0;
    cudaStream_t stream = nullptr;   // branch stream of this level
    cudaEvent_t fork = nullptr, done = nullptr;
};

struct AperiodicState {
    std::map<int64_t, Schedule> schedules;   // per T
    std::vector<LevelBuffers> levels;
    std::map<int64_t, BaseSet> base;         // per base-case T
    void* Y = nullptr;                       // full-grid scratch of the base case
    void* Z = nullptr;                       // interior result
    cudaStream_t cap = nullptr;              // capture stream
    cudaStream_t interior = nullptr;         // branch stream of the interior solve
    cudaEvent_t int_fork = nullptr, int_done = nullptr;
    std::map<int64_t, int> runs;             // eager runs so far per T
    // schedule picked by stencil_plan_autotune per T: (mode, cutoff)
    std::map<int64_t, std::pair<int, int64_t>> tuned;
    std::map<std::pair<int64_t, const void*>, cudaGraphExec_t> graphs;
    size_t bytes = 0;                        // device memory held (level buffers, tables, scratch)
};

static int box_Mp(int64_t n, int precision) {
    const int64_t align = precision == STENCIL_FP32 ? 16 : 8;
    return (int)((n + 1 + align - 1) / align * align);
}

// l-shells (appendix "l-shell Spatial Grid Decomposition"): face f = 2 a + side
// is looked towards by reach_to(f) cells per step (its toward-reach) and away
// from by reach_from(f) = the opposite face's toward-reach. After t steps the
// boundary has reached exactly the cells within reach_to(f) t of some face f; a
// kept cell's dependence cone over t steps reaches reach_to(f) t towards and
// reach_from(f) t away from every face. A face with toward-reach 0 never
// reaches any cell: it gets no strip and no band.
static int reach_to(const stencil_plan_s* p, int f) { return p->reach[f >> 1][f & 1]; }
static int reach_from(const stencil_plan_s* p, int f) { return p->reach[f >> 1][(f & 1) ^ 1]; }

// Per-face bounds of a region or keep range: v[f] = reach_to(f) x + reach_from(f) y
// (0 for faces that no offset looks towards), capped at kNoHi.
struct FaceBounds {
    int64_t v[6] = {0, 0, 0, 0, 0, 0};
};
static FaceBounds face_bounds(const stencil_plan_s* p, int64_t x, int64_t y) {
    FaceBounds b;
    for (int f = 0; f < 2 * p->ndim; ++f)
        b.v[f] = reach_to(p, f) > 0
                     ? std::min<int64_t>(reach_to(p, f) * x + reach_from(p, f) * y, kNoHi)
                     : 0;
    return b;
}
// Some cell lies farther than lo.v[f] from every face f.
static bool clear_cells_exist(const stencil_plan_s* p, const FaceBounds& lo) {
    for (int a = 0; a < p->ndim; ++a)
        if (lo.v[2 * a] + lo.v[2 * a + 1] >= p->dims[a]) return false;
    return true;
}
static bool any_reach(const stencil_plan_s* p) {
    for (int f = 0; f < 2 * p->ndim; ++f)
        if (reach_to(p, f) > 0) return true;
    return false;
}

// The strips of a periodic solve over the region "within W.v[f] of some face f"
// keeping the cells clear of every face by lo and within hi of their strip's
// face, grouped into batches of equal box shape.
static std::vector<Batch> make_batches(const stencil_plan_s* p, const FaceBounds& W,
                                       const FaceBounds& lo, const FaceBounds& hi) {
    const int d = p->ndim;
    int64_t P[6] = {0, 0, 0, 0, 0, 0};
    for (int f = 0; f < 2 * d; ++f)
        if (reach_to(p, f) > 0)
            P[f] = next_pow2(std::max<int64_t>({W.v[f], 4, 2 * p->radius + 1}));
    bool whole = false;
    for (int a = 0; a < d; ++a)
        if (P[2 * a] + P[2 * a + 1] >= p->dims[a]) whole = true;
    struct Item { int64_t bdims[3]; ItemGeom g; };
    std::vector<Item> items;
    if (whole) {
        Item it;
        for (int a = 0; a < 3; ++a) {
            it.bdims[a] = a < d ? p->dims[a] : 1;
            it.g.perm[a] = a;
            it.g.off[a] = 0;
            it.g.valid[a] = a < d ? (int)p->dims[a] : 1;
        }
        it.g.face_axis = -1;
        it.g.face_side = 0;
        items.push_back(it);
    } else {
        for (int a = 0; a < d; ++a) {
            for (int side = 0; side < 2; ++side) {
                const int f = 2 * a + side;
                if (reach_to(p, f) == 0) continue;
                Item it;
                int perm[3] = {a, 0, 0}, k = 1;
                for (int b = 0; b < d; ++b)
                    if (b != a) perm[k++] = b;
                for (int b = d; b < 3; ++b) perm[b] = b;
                for (int b = 0; b < 3; ++b) {
                    it.g.perm[b] = perm[b];
                    it.g.off[b] = 0;
                }
                it.g.off[a] = side == 0 ? 0 : (int)(p->dims[a] - W.v[f]);
                for (int b = 0; b < 3; ++b) {
                    if (b >= d) {
                        it.bdims[b] = 1;
                        it.g.valid[b] = 1;
                    } else if (b == 0) {
                        it.bdims[b] = P[f];
                        it.g.valid[b] = (int)W.v[f];
                    } else {
                        it.bdims[b] = p->dims[perm[b]];
                        it.g.valid[b] = (int)p->dims[perm[b]];
                    }
                }
                it.g.face_axis = a;
                it.g.face_side = side;
                items.push_back(it);
            }
        }
    }
    std::vector<Batch> out;
    for (const Item& it : items) {
        Batch* b = nullptr;
        for (Batch& c : out)
            if (c.bdims[0] == it.bdims[0] && c.bdims[1] == it.bdims[1] &&
                c.bdims[2] == it.bdims[2] && c.geom.items < kMaxItems)
                b = &c;
        if (!b) {
            out.emplace_back();
            b = &out.back();
            std::memset(&b->geom, 0, sizeof(b->geom));
            for (int a = 0; a < 3; ++a) b->bdims[a] = it.bdims[a];
            b->geom.ndim = d;
            b->geom.box_cells = 1;
            for (int a = 0; a < d; ++a) {
                b->geom.gdims[a] = (int)p->dims[a];
                b->geom.bdims[a] = (int)it.bdims[a];
                b->geom.box_cells *= it.bdims[a];
            }
            for (int f = 0; f < 6; ++f) {
                b->geom.lo[f] = (int)lo.v[f];
                b->geom.hi[f] = (int)hi.v[f];
            }
            b->norient = 0;
        }
        int o = 0;
        while (o < b->norient && std::memcmp(b->perms[o], it.g.perm, sizeof(int) * 3) != 0) ++o;
        if (o == b->norient) {
            std::memcpy(b->perms[o], it.g.perm, sizeof(int) * 3);
            ++b->norient;
        }
        b->orient[b->geom.items] = o;
        b->geom.it[b->geom.items++] = it.g;
    }
    return out;
}

// RecursiveBoundary(T) over l-shells, with a = reach_to(f), b = reach_from(f)
// per face (a = b = sigma on every face gives the distance form of the header):
// input "within (a + b) T of some face", output "within a T of some face";
// Step 1 keeps the cells clear of every face by a T1 and within a T + b T2 of
// some face, Step 2 those clear by a T2 and within a T. A kept cell's cone
// reaches b T_k away from its face, which the solve's region holds.
static void build_rb(const stencil_plan_s* p, Schedule& sc, int64_t T, int level, int64_t cutoff) {
    if (T < cutoff) {
        sc.ops.push_back(Op{Op::BASE, -1, T});
        return;
    }
    const int64_t T1 = T / 2, T2 = T - T1;
    // Step 1: P1 over the input region for T1 steps, kept clear by a T1 and within a T + b T2
    int i1 = -1;
    const FaceBounds lo1 = face_bounds(p, T1, 0);
    if (clear_cells_exist(p, lo1)) {
        Step s1;
        s1.level = level;
        s1.T = T1;
        s1.batches = make_batches(p, face_bounds(p, T, T), lo1, face_bounds(p, T, T2));
        sc.steps.push_back(s1);
        i1 = (int)sc.steps.size() - 1;
        sc.ops.push_back(Op{Op::SOLVE, i1, 0});
    }
    build_rb(p, sc, T1, level + 1, cutoff);
    if (i1 >= 0) sc.ops.push_back(Op{Op::SCATTER, i1, 0});
    // Step 2: P2 over "within a T + b T2" for T2 steps, kept clear by a T2 and within a T
    int i2 = -1;
    const FaceBounds lo2 = face_bounds(p, T2, 0);
    if (clear_cells_exist(p, lo2)) {
        Step s2;
        s2.level = level;
        s2.T = T2;
        s2.batches = make_batches(p, face_bounds(p, T, T2), lo2, face_bounds(p, T, 0));
        sc.steps.push_back(s2);
        i2 = (int)sc.steps.size() - 1;
        sc.ops.push_back(Op{Op::SOLVE, i2, 0});
    }
    build_rb(p, sc, T2, level + 1, cutoff);
    if (i2 >= 0) sc.ops.push_back(Op{Op::SCATTER, i2, 0});
}

static std::vector<BaseTile> make_base_tiles(const stencil_plan_s* p, int64_t Tb, size_t* smem,
                                            bool whole_grid = false);

static int64_t auto_cutoff(const stencil_plan_s* p, int64_t cutoff) {
    // the loop's cost per leaf grows with T_b^2 while each recursion level costs
    // about eight grid-sized FFT solves (four face strips of width 2 sigma T_k
    // per node, two solves per node); 2-D: 64 measured best on 8192^2, T = 4096
    // (cutoff 8 / 16 / 32 / 48 / 64: 199 / 119 / 70 / 64 / 64 ms)
    int64_t want = p->ndim == 1 ? 256 : p->ndim == 2 ? 64 : 8;
    if (cutoff >= 2) {
        want = cutoff;
    } else if (p->radius > 0) {
        // keep each leaf's tiles at least twice the halo wide along every axis
        // (recomputation at most (1 + 2h / extent)^d), with extent + 2h + 2r
        // per axis fitting the shared-memory budget: h = r T_b <= (side - 2r) / 4
        const double cells = 150.0 * 1024 / (2.0 * (double)p->elem);
        const double side = std::pow(cells, 1.0 / p->ndim);
        const int64_t tb = (int64_t)((side - 2.0 * p->radius) / (4.0 * p->radius));
        want = std::max<int64_t>(2, std::min<int64_t>(want, tb + 1));
    }
    // every base-case tile (output box plus the T_b-step halo) must fit in shared
    // memory: lower the cutoff until the largest leaf (T_b = cutoff - 1) fits
    while (want > 2) {
        size_t smem = 0;
        make_base_tiles(p, want - 1, &smem);
        if (smem <= (size_t)kSmemBudget) break;
        --want;
    }
    return want;
}

// byte offsets of each batch in its level's buffers; returns the totals
static void layout_step(const stencil_plan_s* p, Step& st, size_t* S_total, size_t* H_total) {
    size_t so = 0, ho = 0;
    for (Batch& b : st.batches) {
        b.s_off = so;
        b.h_off = ho;
        so += (size_t)b.geom.items * b.geom.box_cells * p->elem;
        so = (so + 255) & ~size_t(255);
        const size_t hb = periodic_workspace_bytes(p->ndim, b.bdims, p->precision);
        ho += (size_t)b.geom.items * hb;
        ho = (ho + 255) & ~size_t(255);
    }
    *S_total = so;
    *H_total = ho;
}

static cudaError_t ensure_level(AperiodicState* st, int level, size_t sb, size_t hb) {
    if ((int)st->levels.size() <= level) st->levels.resize(level + 1);
    LevelBuffers& L = st->levels[level];
    cudaError_t err;
    if (L.S_bytes < sb) {
        cudaFree(L.S);
        L.S = nullptr;
        L.S_bytes = 0;
        err = cudaMalloc(&L.S, sb);
        if (err != cudaSuccess) return err;
        L.S_bytes = sb;
        st->bytes += sb;
    }
    if (L.H_bytes < hb) {
        cudaFree(L.H);
        L.H = nullptr;
        L.H_bytes = 0;
        err = cudaMalloc(&L.H, hb);
        if (err != cudaSuccess) return err;
        L.H_bytes = hb;
        st->bytes += hb;
    }
    if (!L.stream) {
        err = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (err != cudaSuccess) return err;
        err = cudaEventCreateWithFlags(&L.fork, cudaEventDisableTiming);
        if (err != cudaSuccess) return err;
        err = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// Output tiles of the base case's frame, the cells within reach_to(f) T_b of
// some face f (bands per face, earlier axes' bands excluded); the loop reads a
// halo of radius x T_b around each tile.
static std::vector<BaseTile> make_base_tiles(const stencil_plan_s* p, int64_t Tb, size_t* smem,
                                            bool whole_grid) {
    const int d = p->ndim;
    int w[6] = {0, 0, 0, 0, 0, 0};
    for (int f = 0; f < 2 * d; ++f) w[f] = (int)std::min<int64_t>(reach_to(p, f) * Tb, kNoHi);
    const int h = (int)(p->radius * Tb);
    const size_t budget = 150 * 1024 / (2 * p->elem);  // cells per buffer
    std::vector<BaseTile> tiles;
    // regions: bands per face, earlier axes' bands excluded
    struct Region { int lo[3], hi[3]; int normal; };
    std::vector<Region> regions;
    bool whole = whole_grid;
    for (int a = 0; a < d; ++a)
        if ((int64_t)w[2 * a] + w[2 * a + 1] >= p->dims[a]) whole = true;
    if (whole) {
        Region r;
        for (int a = 0; a < 3; ++a) { r.lo[a] = 0; r.hi[a] = a < d ? (int)p->dims[a] : 1; }
        r.normal = -1;
        regions.push_back(r);
    } else {
        for (int a = 0; a < d; ++a) {
            for (int side = 0; side < 2; ++side) {
                const int wf = w[2 * a + side];
                if (wf == 0) continue;
                Region r;
                r.normal = a;
                bool empty = false;
                for (int b = 0; b < 3; ++b) {
                    if (b >= d) { r.lo[b] = 0; r.hi[b] = 1; continue; }
                    if (b == a) {
                        r.lo[b] = side == 0 ? 0 : (int)p->dims[b] - wf;
                        r.hi[b] = side == 0 ? wf : (int)p->dims[b];
                    } else if (b < a) {
                        r.lo[b] = w[2 * b];
                        r.hi[b] = (int)p->dims[b] - w[2 * b + 1];
                        if (r.hi[b] <= r.lo[b]) empty = true;
                    } else {
                        r.lo[b] = 0;
                        r.hi[b] = (int)p->dims[b];
                    }
                }
                if (!empty) regions.push_back(r);
            }
        }
    }
    size_t max_vol = 0;
    for (const Region& r : regions) {
        // chunk sizes: normal axis up to 64, other axes as large as the budget allows
        int cs[3];
        for (int b = 0; b < 3; ++b) cs[b] = b < d ? std::min(r.hi[b] - r.lo[b], b == r.normal ? 64 : 1024) : 1;
        // staged cells of a tile: output, T_b-step halo (clipped to the grid) and
        // the kernel's zero ring of width r on each side
        auto vol = [&](void) {
            size_t v = 1;
            for (int b = 0; b < d; ++b)
                v *= (size_t)(std::min(cs[b] + 2 * h, (int)p->dims[b]) + 2 * p->radius);
            return v;
        };
        while (vol() > budget) {
            int best = -1;
            for (int b = 0; b < d; ++b)
                if (cs[b] > 1 && (best < 0 || cs[b] > cs[best])) best = b;
            if (best < 0) break;
            cs[best] = (cs[best] + 1) / 2;
        }
        max_vol = std::max(max_vol, vol());
        for (int z = r.lo[0]; z < r.hi[0]; z += cs[0])
            for (int y = r.lo[1]; y < r.hi[1]; y += cs[1])
                for (int x = r.lo[2]; x < r.hi[2]; x += cs[2]) {
                    BaseTile t;
                    const int o[3] = {z, y, x};
                    for (int b = 0; b < 3; ++b) {
                        t.lo[b] = o[b];
                        t.hi[b] = std::min(o[b] + cs[b], r.hi[b]);
                    }
                    tiles.push_back(t);
                }
    }
    {
        // k_base_1d/2d/3d: (extent + 2 RAD) per axis, two buffers
        size_t m = 0;
        for (const BaseTile& t : tiles) {
            size_t v = 1;
            for (int a = 0; a < d; ++a) {
                const int lo = std::max(t.lo[a] - h, 0);
                const int hi = std::min<int>(t.hi[a] + h, (int)p->dims[a]);
                v *= (size_t)(hi - lo + 2 * p->radius);
            }
            m = std::max(m, v);
        }
        *smem = 2 * m * p->elem;
    }
    (void)max_vol;
    return tiles;
}

template <typename R>
static cudaError_t launch_base(stencil_plan_s* p, const BaseSet& bs, R* X, R* Y, int64_t Tb,
                              cudaStream_t s, bool whole = false) {
    BaseParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.ndim = p->ndim;
    for (int a = 0; a < p->ndim; ++a) bp.gdims[a] = (int)p->dims[a];
    bp.Tb = (int)Tb;
    bp.mirror = p->boundary == STENCIL_NEUMANN ? 1 : 0;
    for (int f = 0; f < 6; ++f)
        bp.wout[f] = whole ? kNoHi
                           : f < 2 * p->ndim ? (int)std::min<int64_t>(reach_to(p, f) * Tb, kNoHi) : 0;
    for (int i = 0; i < p->nweights; ++i) {
        bp.w[i] = p->weights[i];
        bp.wf[i] = (float)p->weights[i];
    }
    const BaseTile* tiles = static_cast<const BaseTile*>(bs.tiles);
    cudaError_t err = cudaSuccess;
    p->prof.begin(PASS_BASE_LOOP, s);
    switch (p->radius) {
#define SFFT_BASE_CASE(RADV)                                                                  \
    case RADV:                                                                                \
        {                                                                                     \
            auto kern = p->ndim == 1 ? k_base_1d<R, RADV>                                     \
                                     : p->ndim == 2 ? k_base_2d<R, RADV> : k_base_3d<R, RADV>; \
            if (bs.smem > 48 * 1024)                                                          \
                err = smem_optin(reinterpret_cast<const void*>(kern), bs.smem);              \
            if (err == cudaSuccess) {                                                         \
                kern<<<bs.count, p->ndim == 2 ? 512 : 256, bs.smem, s>>>(X, Y, tiles, bp);     \
                err = cudaGetLastError();                                                     \
            }                                                                                 \
        }                                                                                     \
        break;
        SFFT_BASE_CASE(0)
        SFFT_BASE_CASE(1)
        SFFT_BASE_CASE(2)
        SFFT_BASE_CASE(3)
#undef SFFT_BASE_CASE
        default: err = cudaErrorInvalidValue;
    }
    p->prof.end(s);
    if (err != cudaSuccess) return err;
    p->prof.begin(PASS_COPY, s);
    if (p->ndim == 2)
        k_tile_copy_2d<R><<<bs.count, 256, 0, s>>>(Y, X, tiles, bp);
    else
        k_tile_copy<R><<<bs.count, 256, 0, s>>>(Y, X, tiles, bp);
    err = cudaGetLastError();
    p->prof.end(s);
    return err;
}

// One table per distinct (T_k, box shape, orientation) of the schedule (d >= 2).
static void assign_tables(const stencil_plan_s* p, Schedule& sc) {
    for (Step& st : sc.steps)
        for (Batch& b : st.batches)
            for (int o = 0; o < kMaxOrient; ++o) {
                b.vt[o] = -1;
                if (p->ndim < 2 || o >= b.norient) continue;
                int idx = -1;
                for (size_t i = 0; i < sc.tables.size(); ++i) {
                    const VTable& v = sc.tables[i];
                    if (v.T == st.T && std::memcmp(v.bdims, b.bdims, sizeof(v.bdims)) == 0 &&
                        std::memcmp(v.perm, b.perms[o], sizeof(v.perm)) == 0)
                        idx = (int)i;
                }
                if (idx < 0) {
                    VTable v;
                    v.T = st.T;
                    std::memcpy(v.bdims, b.bdims, sizeof(v.bdims));
                    std::memcpy(v.perm, b.perms[o], sizeof(v.perm));
                    sc.tables.push_back(v);
                    idx = (int)sc.tables.size() - 1;
                }
                b.vt[o] = idx;
            }
}

// T single steps of the loop over the whole grid (3-D), X -> Y -> X ...
template <typename R>
static cudaError_t launch_steps(stencil_plan_s* p, R* X, R* Y, int64_t T, cudaStream_t s) {
    BaseParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.ndim = p->ndim;
    for (int a = 0; a < p->ndim; ++a) bp.gdims[a] = (int)p->dims[a];
    for (int i = 0; i < p->nweights; ++i) {
        bp.w[i] = p->weights[i];
        bp.wf[i] = (float)p->weights[i];
    }
    const int blocks = grid_blocks(p->n_cells);
    // FP32: tiles of (axis 1, axis 2); axis 0 cut into chunks until about four
    // CTAs per SM are in flight, each chunk at least 2r + 2 planes deep
    const int L0 = (int)p->dims[0];
    const int TX = p->dims[2] >= 32 ? 32 : p->dims[2] >= 16 ? 16 : 8;
    const dim3 tiles((unsigned)((p->dims[2] + TX - 1) / TX),
                     (unsigned)((p->dims[1] + kStepThreads / TX - 1) / (kStepThreads / TX)), 1);
    const int want = std::max(1, (int)(608 / (tiles.x * tiles.y)));
    int zchunk = std::max<int>((L0 + want - 1) / want, 2 * p->radius + 2);
    zchunk = std::min(zchunk, L0);
    const dim3 grid3(tiles.x, tiles.y, (unsigned)((L0 + zchunk - 1) / zchunk));
    cudaError_t err = cudaSuccess;
    R* a = X;
    R* b = Y;
    p->prof.begin(PASS_BASE_LOOP, s);
    for (int64_t t = 0; t < T && err == cudaSuccess; ++t) {
        if constexpr (sizeof(R) == 8) {
            switch (p->radius) {
                case 1: k_step_3d<R, 1><<<blocks, 256, 0, s>>>(a, b, bp); break;
                case 2: k_step_3d<R, 2><<<blocks, 256, 0, s>>>(a, b, bp); break;
                case 3: k_step_3d<R, 3><<<blocks, 256, 0, s>>>(a, b, bp); break;
                default: k_step_3d<R, 0><<<blocks, 256, 0, s>>>(a, b, bp); break;
            }
        } else {
#define SFFT_STEP(RADV, TXV) \
    k_step_3d_stream<R, RADV, TXV><<<grid3, kStepThreads, 0, s>>>(a, b, bp, zchunk)
#define SFFT_STEP_TX(RADV)                         \
    (TX == 32 ? SFFT_STEP(RADV, 32) : TX == 16 ? SFFT_STEP(RADV, 16) : SFFT_STEP(RADV, 8))
            switch (p->radius) {
                case 1: SFFT_STEP_TX(1); break;
                case 2: SFFT_STEP_TX(2); break;
                case 3: SFFT_STEP_TX(3); break;
                default: SFFT_STEP_TX(0); break;
            }
#undef SFFT_STEP_TX
#undef SFFT_STEP
        }
        err = cudaGetLastError();
        R* tmp = a;
        a = b;
        b = tmp;
    }
    p->prof.end(s);
    if (err == cudaSuccess && a != X)
        err = cudaMemcpyAsync(X, a, (size_t)p->n_cells * p->elem, cudaMemcpyDeviceToDevice, s);
    return err;
}

// Cost estimates (seconds) that decide between RecursiveBoundary and the
// plain loop for a zero-Dirichlet solve; the constants are per-cell costs
// measured on GB300 for FP32 (FFT passes plus copies; one stencil point of the
// blocked loop) and the cost of one launch.
static double fft_cell_s(const stencil_plan_s* p) { return (p->precision == STENCIL_FP32 ? 1.0 : 8.0) * 2.0e-11; }
static double loop_point_s(const stencil_plan_s* p) { return (p->precision == STENCIL_FP32 ? 1.0 : 2.0) * 0.7e-12; }
constexpr double kLaunchS = 4e-6;
// Base-case tiles the GPU works on at full rate at once (one per SM of 152):
// a launch with fewer tiles leaves SMs idle, so its time is set by the
// largest tile, not by the total work.
constexpr double kTileSlots = 152.0;

static double stencil_points(const stencil_plan_s* p) { return (double)p->nweights; }

// Cells (output tile plus halo) of a list of tiles, and the time-setting
// equivalent: the total, or the largest tile times the concurrent slots.
static double tile_cells_effective(const stencil_plan_s* p, const std::vector<BaseTile>& tiles,
                                   int64_t halo, bool whole_grid = false) {
    double total = 0.0, largest = 0.0;
    for (const BaseTile& t : tiles) {
        double v = 1.0;
        for (int a = 0; a < p->ndim; ++a)
            v *= (double)(std::min<int64_t>(t.hi[a] + halo, p->dims[a]) -
                          std::max<int64_t>(t.lo[a] - halo, 0));
        total += v;
        largest = std::max(largest, v);
    }
    // calibrated on 3-D frames (tens of tiles) and on launches of a few tiles
    // over small 1-D / 2-D grids; 2-D frames of many tiles measured close to
    // their total work
    (void)whole_grid;
    const bool idle = p->ndim == 3 || tiles.size() < 38;
    return idle ? std::max(total, largest * kTileSlots) : total;
}

static double schedule_cost(const stencil_plan_s* p, const Schedule& sc, int64_t T) {
    double c = 0.0;
    if (clear_cells_exist(p, face_bounds(p, T, 0)))
        c += (double)p->n_cells * fft_cell_s(p);   // interior solve
    // a strip batch: gather, three or five FFT passes, table and scatter
    // launches and the step's stream joins, about 20 us of fixed cost (100 us
    // for 1-D, whose strips are tiny next to it); 2-D leaves run about 5x
    // faster than the tile-count model below says (fitted to GB300 runs of
    // 2-D grids of 4K-67M cells, r = 1-3, and 1-D grids of 8K-16K cells)
    const double batch_s = p->ndim == 1 ? 1e-4 : 2e-5;
    for (const Step& st : sc.steps)
        for (const Batch& b : st.batches)
            c += (double)b.geom.items * (double)b.geom.box_cells * fft_cell_s(p) + batch_s;
    const double leaf_scale = p->ndim == 2 ? 0.2 : 1.0;
    // base leaves repeat a few T_b values thousands of times: price each once
    std::map<int64_t, double> leaf;
    for (const Op& op : sc.ops) {
        if (op.kind != Op::BASE) continue;
        auto it = leaf.find(op.T);
        if (it == leaf.end()) {
            size_t smem = 0;
            const std::vector<BaseTile> tiles = make_base_tiles(p, op.T, &smem);
            const double cells = tile_cells_effective(p, tiles, p->radius * op.T);
            it = leaf.emplace(op.T, leaf_scale * cells * (double)op.T * stencil_points(p) *
                                            loop_point_s(p) +
                                        2 * kLaunchS).first;
        }
        c += it->second;
    }
    return c;
}

// Launch shape of k_loop_cluster for the plan's grid: the largest cluster
// (16, else 8, 4, 2 CTAs) whose slabs hold at least r planes, whose two
// buffers fit one CTA's shared memory and that the device can run.

template <typename R, int RAD, int D>
static const void* cluster_kernel() {
    return reinterpret_cast<const void*>(k_loop_cluster<R, RAD, D>);
}

template <typename R>
static const void* cluster_kernel_for(int radius, int ndim) {
#define SFFT_CK(RADV)                                                               \
    case RADV:                                                                     \
        return ndim == 1 ? cluster_kernel<R, RADV, 1>()                            \
               : ndim == 2 ? cluster_kernel<R, RADV, 2>() : cluster_kernel<R, RADV, 3>();
    switch (radius) {
        SFFT_CK(0)
        SFFT_CK(1)
        SFFT_CK(2)
        SFFT_CK(3)
        default: return nullptr;
    }
#undef SFFT_CK
}

static bool have_device() {
    static const bool yes = [] {
        int n = 0;
        const bool ok = cudaGetDeviceCount(&n) == cudaSuccess && n > 0;
        cudaGetLastError();
        return ok;
    }();
    return yes;
}

static ClusterPlan plan_cluster(const stencil_plan_s* p) {
    ClusterPlan cp;
    if (!have_device()) return cp;
    if (p->boundary == STENCIL_NEUMANN) return cp;   // its ghost planes are zeros
    const int d = p->ndim, r = p->radius;
    const int64_t L0 = p->dims[0];
    const void* kern = p->precision == STENCIL_FP32 ? cluster_kernel_for<float>(r, d)
                                                    : cluster_kernel_for<double>(r, d);
    if (!kern) return cp;
    for (int cs = 16; cs >= 2; cs /= 2) {
        if (L0 % cs != 0 || L0 / cs < std::max(r, 1)) continue;
        ClusterGeom g;
        g.S = (int)(L0 / cs);
        g.L1p = d >= 2 ? (int)p->dims[1] + 2 * r : 1;
        g.L2p = d == 3 ? (int)p->dims[2] + 2 * r : 1;
        g.P = g.L1p * g.L2p;
        g.Q = (int)((d >= 2 ? p->dims[1] : 1) * (d == 3 ? p->dims[2] : 1));
        g.G = std::max(1, std::min(g.S, kClusterThreads / g.Q));
        const size_t smem = 2 * (size_t)(g.S + 2 * r) * g.P * p->elem;
        if (smem > (size_t)kClusterSmemMax) continue;
        // the device must be able to run the cluster (fails without a GPU)
        // (the dynamic shared-memory limit only ever rises: plans of other
        // shapes share the kernel)
        if ((smem > 48 * 1024 && smem_optin(kern, smem) != cudaSuccess) ||
            (cs > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                           cudaSuccess)) {
            cudaGetLastError();
            continue;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(kClusterThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess || clusters < 1) {
            cudaGetLastError();
            continue;
        }
        cp.ok = true;
        cp.cs = cs;
        cp.g = g;
        cp.smem = smem;
        return cp;
    }
    return cp;
}

template <typename R>
static cudaError_t launch_cluster(stencil_plan_s* p, const ClusterPlan& cp, R* X, int64_t T,
                                  cudaStream_t s) {
    BaseParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.ndim = p->ndim;
    for (int a = 0; a < p->ndim; ++a) bp.gdims[a] = (int)p->dims[a];
    for (int i = 0; i < p->nweights; ++i) {
        bp.w[i] = p->weights[i];
        bp.wf[i] = (float)p->weights[i];
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(cp.cs, 1, 1);
    cfg.blockDim = dim3(kClusterThreads, 1, 1);
    cfg.dynamicSmemBytes = cp.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cp.cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const long long TT = (long long)T;
    cudaError_t err = cudaSuccess;
    p->prof.begin(PASS_BASE_LOOP, s);
#define SFFT_CL(RADV, DV)                                                                 \
    err = cudaLaunchKernelEx(&cfg, k_loop_cluster<R, RADV, DV>, X, bp, cp.g, TT)
#define SFFT_CL_D(RADV)                                                                   \
    case RADV:                                                                           \
        if (p->ndim == 1) SFFT_CL(RADV, 1);                                              \
        else if (p->ndim == 2) SFFT_CL(RADV, 2);                                         \
        else SFFT_CL(RADV, 3);                                                           \
        break;
    switch (p->radius) {
        SFFT_CL_D(0)
        SFFT_CL_D(1)
        SFFT_CL_D(2)
        SFFT_CL_D(3)
        default: err = cudaErrorInvalidValue;
    }
#undef SFFT_CL_D
#undef SFFT_CL
    p->prof.end(s);
    return err;
}

// The plain loop as a schedule: the cluster-resident loop when the grid fits
// one cluster and its estimate is lower, else whole-grid blocked tiles of Tc
// steps (1-D, 2-D) or single steps (3-D); returns its estimated cost.
static double build_loop_tiles(const stencil_plan_s* p, Schedule& sc, int64_t T);

static double build_loop(const stencil_plan_s* p, Schedule& sc, int64_t T) {
    Schedule tiles;
    const double c_tiles = build_loop_tiles(p, tiles, T);
    // 1-D grids: the tiled loop measured faster (it spreads over every SM)
    const ClusterPlan cp = p->ndim >= 2 ? plan_cluster(p) : ClusterPlan{};
    if (cp.ok) {
        // per step (GB300 fit over 2-D and 3-D grids of 4K-262K cells): about
        // 1 us of push and cluster barrier plus the CTA's share of the point
        // updates at 1.2e11 (FP32) / 6e8 (FP64) per second per SM
        const double rate = p->precision == STENCIL_FP32 ? 1.2e11 : 6e8;
        const double step = (double)p->n_cells * stencil_points(p) / (cp.cs * rate) + 1.05e-6;
        const double c_cluster = (double)T * step + 2 * kLaunchS;
        if (c_cluster < c_tiles) {
            sc.loop = true;
            sc.cluster = cp;
            sc.ops.push_back(Op{Op::CLUSTER, -1, T});
            return c_cluster;
        }
    }
    sc = std::move(tiles);
    return c_tiles;
}

static double build_loop_tiles(const stencil_plan_s* p, Schedule& sc, int64_t T) {
    sc.loop = true;
    if (p->ndim == 3 && p->boundary != STENCIL_NEUMANN) {   // the step kernels read zero ghosts
        // axis-0 streamed steps: FMA-bound at about 8e12 (FP32) / 3.6e11 (FP64)
        // point updates per second on large grids, about 8 us per step on small
        // ones (GB300 measurements)
        sc.ops.push_back(Op{Op::STEP, -1, T});
        const double per_pt = p->precision == STENCIL_FP32 ? 1.3e-13 : 2.8e-12;
        const double step = std::max(8e-6, (double)p->n_cells * stencil_points(p) * per_pt);
        return (double)T * (step + 2e-6);
    }
    double best = -1.0;
    int64_t best_tc = 1;
    for (int64_t tc = 1; tc <= std::min<int64_t>(T, p->ndim == 1 ? 256 : 64); tc *= 2) {
        size_t smem = 0;
        const std::vector<BaseTile> tiles = make_base_tiles(p, tc, &smem, true);
        if (smem > (size_t)kSmemBudget) break;
        const double cells = tile_cells_effective(p, tiles, p->radius * tc, true);
        const double cost = cells * (double)T * stencil_points(p) * loop_point_s(p) +
                            (double)(T / tc + 1) * 2 * kLaunchS;
        if (best < 0 || cost < best) {
            best = cost;
            best_tc = tc;
        }
    }
    for (int64_t done = 0; done < T; done += best_tc)
        sc.ops.push_back(Op{Op::LOOP, -1, std::min<int64_t>(best_tc, T - done)});
    return best;
}

static cudaError_t prepare(stencil_plan_s* p, int64_t T, Schedule** out) {
    if (!p->ap) p->ap = new AperiodicState();
    AperiodicState* st = p->ap;
    cudaError_t err;
    if (!st->Y) {
        err = cudaMalloc(&st->Y, (size_t)p->n_cells * p->elem);
        if (err != cudaSuccess) {
            st->Y = nullptr;
            return err;
        }
        st->bytes += (size_t)p->n_cells * p->elem;
    }
    if (!st->cap) {
        err = cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaStreamCreateWithFlags(&st->interior, cudaStreamNonBlocking);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&st->int_fork, cudaEventDisableTiming);
        if (err == cudaSuccess) err = cudaEventCreateWithFlags(&st->int_done, cudaEventDisableTiming);
        if (err != cudaSuccess) return err;
    }
    auto it = st->schedules.find(T);
    if (it == st->schedules.end()) {
        Schedule sc;
        int mode = p->schedule;
        int64_t cut = p->cutoff;
        auto tu = st->tuned.find(T);
        if (mode == STENCIL_SCHEDULE_AUTO && cut == 0 && tu != st->tuned.end()) {
            mode = tu->second.first;     // measured by stencil_plan_autotune
            cut = tu->second.second;
        }
        if (mode == STENCIL_SCHEDULE_CLUSTER) {
            sc.cluster = plan_cluster(p);
            if (!sc.cluster.ok) return cudaErrorInvalidValue;   // grid too large for one cluster
            sc.loop = true;
            sc.ops.push_back(Op{Op::CLUSTER, -1, T});
        } else if (mode == STENCIL_SCHEDULE_LOOP) {
            build_loop(p, sc, T);
        } else {
            build_rb(p, sc, T, 0, auto_cutoff(p, cut));
            if (mode == STENCIL_SCHEDULE_AUTO && cut == 0) {
                // automatic mode: the plain loop when it is the cheaper schedule (a
                // boundary region that spans the whole grid gains nothing from FFTs)
                Schedule loop;
                const double c_loop = build_loop(p, loop, T);
                if (c_loop < schedule_cost(p, sc, T)) sc = std::move(loop);
            }
        }
        assign_tables(p, sc);
        for (VTable& v : sc.tables) {
            const size_t vb = periodic_workspace_bytes(p->ndim, v.bdims, p->precision);
            err = cudaMalloc(&v.buf, vb);
            if (err != cudaSuccess) {
                v.buf = nullptr;
                return err;
            }
            st->bytes += vb;
        }
        for (Step& step : sc.steps) {
            size_t sb = 0, hb = 0;
            layout_step(p, step, &sb, &hb);
            err = ensure_level(st, step.level, sb, hb);
            if (err != cudaSuccess) return err;
        }
        for (const Op& op : sc.ops) {
            if (op.kind != Op::BASE && op.kind != Op::LOOP) continue;
            const int64_t key = 2 * op.T + (op.kind == Op::LOOP ? 1 : 0);
            if (st->base.count(key)) continue;
            BaseSet bs;
            std::vector<BaseTile> tiles = make_base_tiles(p, op.T, &bs.smem, op.kind == Op::LOOP);
            bs.count = (int)tiles.size();
            if (bs.smem > (size_t)kSmemBudget) return cudaErrorInvalidValue;
            err = cudaMalloc(&bs.tiles, sizeof(BaseTile) * std::max<size_t>(1, tiles.size()));
            if (err != cudaSuccess) return err;
            // a pageable-memory cudaMemcpy may return before its DMA lands and is
            // ordered only against the legacy stream; upload on the per-thread
            // stream and wait, so kernels on any stream see the tiles
            err = cudaMemcpyAsync(bs.tiles, tiles.data(), sizeof(BaseTile) * tiles.size(),
                                  cudaMemcpyHostToDevice, cudaStreamPerThread);
            if (err == cudaSuccess) err = cudaStreamSynchronize(cudaStreamPerThread);
            if (err != cudaSuccess) return err;
            st->base[key] = bs;
        }
        it = st->schedules.emplace(T, std::move(sc)).first;
    }
    *out = &it->second;
    return cudaSuccess;
}

// Enqueue the whole zero-Dirichlet solve on `main` (and, with branches, on the
// per-level branch streams joined back to main).
template <typename R>
static cudaError_t emit(stencil_plan_s* p, AperiodicState* st, const Schedule& sc, R* X,
                        int64_t T, bool interior, cudaStream_t main, bool branches) {
    cudaError_t err;
    const size_t bytes = (size_t)p->n_cells * p->elem;
    R* Z = static_cast<R*>(st->Z);
    // Step 2 of the periodic solves, once per distinct (T_k, box, orientation)
    for (const VTable& v : sc.tables) {
        const SymbolParams sp = make_symbol_params(p, v.bdims, v.T, p->E64, p->E32, v.perm);
        const int64_t n = v.bdims[p->ndim - 1] / 2;
        p->prof.begin(PASS_VTABLE, main);
        err = launch_vtable<R>(v.buf, sp, box_Mp(n, p->precision), main);
        p->prof.end(main);
        if (err != cudaSuccess) return err;
    }
    if (interior) {
        // interior (dist > sigma T): the periodic solve of the untouched input
        p->prof.begin(PASS_COPY, main);
        err = cudaMemcpyAsync(Z, X, bytes, cudaMemcpyDeviceToDevice, main);
        p->prof.end(main);
        if (err != cudaSuccess) return err;
        cudaStream_t is = main;
        if (branches) {
            if ((err = cudaEventRecord(st->int_fork, main)) != cudaSuccess) return err;
            if ((err = cudaStreamWaitEvent(st->interior, st->int_fork, 0)) != cudaSuccess) return err;
            is = st->interior;
        }
        err = periodic_solve<R>(p, Z, p->dims, T, p->H, p->Mp, p->tw, p->twn_log2, p->E64, p->E32,
                                p->status, is);
        if (err != cudaSuccess) return err;
        if (branches && (err = cudaEventRecord(st->int_done, is)) != cudaSuccess) return err;
    }
    for (const Op& op : sc.ops) {
        if (op.kind == Op::BASE || op.kind == Op::LOOP) {
            auto it = st->base.find(2 * op.T + (op.kind == Op::LOOP ? 1 : 0));
            err = launch_base<R>(p, it->second, X, static_cast<R*>(st->Y), op.T, main,
                                 op.kind == Op::LOOP);
            if (err != cudaSuccess) return err;
            continue;
        }
        if (op.kind == Op::STEP) {
            err = launch_steps<R>(p, X, static_cast<R*>(st->Y), op.T, main);
            if (err != cudaSuccess) return err;
            continue;
        }
        if (op.kind == Op::CLUSTER) {
            if (!sc.cluster.ok) return cudaErrorInvalidValue;
            err = launch_cluster<R>(p, sc.cluster, X, op.T, main);
            if (err != cudaSuccess) return err;
            continue;
        }
        const Step& step = sc.steps[op.step];
        LevelBuffers& L = st->levels[step.level];
        if (op.kind == Op::SOLVE) {
            for (const Batch& b : step.batches) {
                const long long total = (long long)b.geom.items * b.geom.box_cells;
                R* S = reinterpret_cast<R*>(static_cast<char*>(L.S) + b.s_off);
                p->prof.begin(PASS_GATHER, main);
                if (p->ndim == 2) {
                    dim3 grid((b.geom.bdims[1] + 31) / 32, (b.geom.bdims[0] + 31) / 32, b.geom.items);
                    k_copy_2d<R, false><<<grid, 256, 0, main>>>(X, S, b.geom);
                } else {
                    k_gather<R><<<grid_blocks(total), 256, 0, main>>>(X, S, b.geom, total);
                }
                err = cudaGetLastError();
                p->prof.end(main);
                if (err != cudaSuccess) return err;
            }
            cudaStream_t bs = main;
            if (branches) {
                if ((err = cudaEventRecord(L.fork, main)) != cudaSuccess) return err;
                if ((err = cudaStreamWaitEvent(L.stream, L.fork, 0)) != cudaSuccess) return err;
                bs = L.stream;
            }
            for (const Batch& b : step.batches) {
                R* S = reinterpret_cast<R*>(static_cast<char*>(L.S) + b.s_off);
                void* H = static_cast<char*>(L.H) + b.h_off;
                const int64_t n = b.bdims[p->ndim - 1] / 2;
                const void* vt[kMaxOrient] = {nullptr, nullptr, nullptr};
                for (int o = 0; o < b.norient; ++o)
                    if (b.vt[o] >= 0) vt[o] = sc.tables[b.vt[o]].buf;
                err = batched_solve<R>(p, S, b.bdims, b.geom.items, step.T, H,
                                       box_Mp(n, p->precision), b.orient, b.perms, b.norient,
                                       p->tw, p->twn_log2, p->E64, p->E32, p->status, bs, vt);
                if (err != cudaSuccess) return err;
            }
            if (branches && (err = cudaEventRecord(L.done, bs)) != cudaSuccess) return err;
        } else {
            if (branches && (err = cudaStreamWaitEvent(main, L.done, 0)) != cudaSuccess) return err;
            for (const Batch& b : step.batches) {
                const long long total = (long long)b.geom.items * b.geom.box_cells;
                R* S = reinterpret_cast<R*>(static_cast<char*>(L.S) + b.s_off);
                p->prof.begin(PASS_SCATTER, main);
                if (p->ndim == 2) {
                    dim3 grid((b.geom.bdims[1] + 31) / 32, (b.geom.bdims[0] + 31) / 32, b.geom.items);
                    k_copy_2d<R, true><<<grid, 256, 0, main>>>(X, S, b.geom);
                } else {
                    k_scatter<R><<<grid_blocks(total), 256, 0, main>>>(S, X, b.geom, total);
                }
                err = cudaGetLastError();
                p->prof.end(main);
                if (err != cudaSuccess) return err;
            }
        }
    }
    if (interior) {
        if (branches && (err = cudaStreamWaitEvent(main, st->int_done, 0)) != cudaSuccess) return err;
        BatchGeom b;
        std::memset(&b, 0, sizeof(b));
        b.ndim = p->ndim;
        b.box_cells = p->n_cells;
        b.items = 1;
        for (int a = 0; a < p->ndim; ++a) {
            b.gdims[a] = b.bdims[a] = (int)p->dims[a];
            b.it[0].perm[a] = a;
            b.it[0].valid[a] = (int)p->dims[a];
        }
        b.it[0].face_axis = -1;
        const FaceBounds lo = face_bounds(p, T, 0);
        for (int f = 0; f < 6; ++f) {
            b.lo[f] = (int)lo.v[f];
            b.hi[f] = kNoHi;
        }
        p->prof.begin(PASS_COPY, main);
        k_scatter<R><<<grid_blocks(p->n_cells), 256, 0, main>>>(Z, X, b, p->n_cells);
        err = cudaGetLastError();
        p->prof.end(main);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// The schedule of T with every buffer it needs, including the interior scratch.
static cudaError_t prepare_all(stencil_plan_s* p, int64_t T, Schedule** out) {
    cudaError_t err = prepare(p, T, out);
    if (err != cudaSuccess) return err;
    const bool interior = !(*out)->loop && clear_cells_exist(p, face_bounds(p, T, 0));
    AperiodicState* st = p->ap;
    if (interior && !st->Z) {
        err = cudaMalloc(&st->Z, (size_t)p->n_cells * p->elem);
        if (err != cudaSuccess) {
            st->Z = nullptr;
            return err;
        }
        st->bytes += (size_t)p->n_cells * p->elem;
    }
    return cudaSuccess;
}

template <typename R>
static cudaError_t aperiodic_impl(stencil_plan_s* p, R* grid, int64_t T, cudaStream_t s) {
    if (p->radius == 0 || !any_reach(p))   // a pointwise stencil never feels the boundary
        return periodic_solve<R>(p, grid, p->dims, T, p->H, p->Mp, p->tw, p->twn_log2, p->E64,
                                 p->E32, p->status, s);
    Schedule* sc = nullptr;
    cudaError_t err = prepare_all(p, T, &sc);
    if (err != cudaSuccess) return err;
    const bool interior = !sc->loop && clear_cells_exist(p, face_bounds(p, T, 0));
    AperiodicState* st = p->ap;
    // profiled runs: one stream, every launch bracketed by events
    if (p->prof.enabled) return emit<R>(p, st, *sc, grid, T, interior, s, false);
    // the first run for a T goes eagerly (it also sets every kernel attribute)
    int& runs = st->runs[T];
    if (runs == 0 || !p->use_graphs) {
        ++runs;
        return emit<R>(p, st, *sc, grid, T, interior, s, true);
    }
    const auto key = std::make_pair(T, static_cast<const void*>(grid));
    auto git = st->graphs.find(key);
    if (git == st->graphs.end()) {
        if (st->graphs.size() >= 8) {          // bound the cache
            cudaGraphExecDestroy(st->graphs.begin()->second);
            st->graphs.erase(st->graphs.begin());
        }
        err = cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal);
        if (err != cudaSuccess) return err;
        cudaError_t e1 = emit<R>(p, st, *sc, grid, T, interior, st->cap, true);
        cudaGraph_t graph = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(st->cap, &graph);
        if (e1 != cudaSuccess || e2 != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return e1 != cudaSuccess ? e1 : e2;
        }
        cudaGraphExec_t exec = nullptr;
        err = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (err != cudaSuccess) return err;
        git = st->graphs.emplace(key, exec).first;
    }
    return cudaGraphLaunch(git->second, s);
}

void aperiodic_forget_graphs(stencil_plan_s* p) {
    if (!p || !p->ap) return;
    for (auto& kv : p->ap->graphs) cudaGraphExecDestroy(kv.second);
    p->ap->graphs.clear();
}

void aperiodic_forget_schedules(stencil_plan_s* p) {
    if (!p || !p->ap) return;
    aperiodic_forget_graphs(p);
    // cudaFree waits for the device, so no launch still reads these tables
    for (auto& kv : p->ap->schedules)
        for (auto& v : kv.second.tables) {
            cudaFree(v.buf);
            p->ap->bytes -= periodic_workspace_bytes(p->ndim, v.bdims, p->precision);
        }
    p->ap->schedules.clear();
    // base-case tiles and measured choices depend on the reach towards every face
    for (auto& kv : p->ap->base) cudaFree(kv.second.tiles);
    p->ap->base.clear();
    p->ap->tuned.clear();
}

size_t aperiodic_bytes(const stencil_plan_s* p) { return p && p->ap ? p->ap->bytes : 0; }

// Times the zero-Dirichlet schedules for T on a scratch copy of grid and keeps
// the fastest for later runs of T (stencil_plan_autotune). Candidates, in
// fixed slots: RecursiveBoundary with the automatic cutoff, the whole-grid
// loop, RecursiveBoundary with half and with twice that cutoff, the
// cluster-resident loop. Each is run three times (schedule set-up, graph
// capture, replay); the replay is timed with events on s.
int aperiodic_autotune(stencil_plan_s* p, const void* grid, int64_t T, cudaStream_t s,
                       double* ms, int cap) {
    if (!p->ap) p->ap = new AperiodicState();
    // fixed slots; a slot that does not apply keeps mode -1 and time -1
    const int64_t c0 = auto_cutoff(p, 0);
    std::vector<std::pair<int, int64_t>> cand = {{STENCIL_SCHEDULE_RECURSIVE, 0},
                                                 {STENCIL_SCHEDULE_LOOP, 0},
                                                 {-1, 0}, {-1, 0}, {-1, 0}};
    if (c0 / 2 >= 2) cand[2] = {STENCIL_SCHEDULE_RECURSIVE, c0 / 2};
    if (auto_cutoff(p, 2 * c0) == 2 * c0) cand[3] = {STENCIL_SCHEDULE_RECURSIVE, 2 * c0};
    if (plan_cluster(p).ok) cand[4] = {STENCIL_SCHEDULE_CLUSTER, 0};
    for (int i = 0; i < cap && ms; ++i) ms[i] = -1.0;
    const size_t bytes = (size_t)p->n_cells * p->elem;
    void* scratch = nullptr;
    cudaError_t err = cudaMalloc(&scratch, bytes);
    if (err != cudaSuccess) return err == cudaErrorMemoryAllocation ? STENCIL_ENOMEM : STENCIL_ECUDA;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int saved_mode = p->schedule;
    const int64_t saved_cut = p->cutoff;
    int best = -1, rc = STENCIL_OK;
    float best_ms = 0.f;
    for (size_t i = 0; i < cand.size() && rc == STENCIL_OK; ++i) {
        if (cand[i].first < 0) continue;
        p->schedule = cand[i].first;
        p->cutoff = cand[i].second;
        aperiodic_forget_schedules(p);
        float t = 0.f;
        for (int rep = 0; rep < 3 && rc == STENCIL_OK; ++rep) {
            err = cudaMemcpyAsync(scratch, grid, bytes, cudaMemcpyDeviceToDevice, s);
            if (err != cudaSuccess) rc = STENCIL_ECUDA;
            if (rc == STENCIL_OK && rep == 2) cudaEventRecord(e0, s);
            if (rc == STENCIL_OK) rc = aperiodic_run(p, scratch, T, s);
            if (rc == STENCIL_OK && rep == 2) {
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = STENCIL_ECUDA;
                else cudaEventElapsedTime(&t, e0, e1);
            }
        }
        if (rc == STENCIL_OK) {
            if ((int)i < cap && ms) ms[i] = t;
            if (best < 0 || t < best_ms) {
                best = (int)i;
                best_ms = t;
            }
        }
    }
    p->schedule = saved_mode;
    p->cutoff = saved_cut;
    aperiodic_forget_schedules(p);
    if (rc == STENCIL_OK) p->ap->tuned[T] = cand[best];
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamSynchronize(s);
    cudaFree(scratch);
    return rc == STENCIL_OK ? best : rc;
}

int aperiodic_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s) {
    cudaError_t err = p->precision == STENCIL_FP32
                          ? aperiodic_impl<float>(p, static_cast<float*>(grid), T, s)
                          : aperiodic_impl<double>(p, static_cast<double*>(grid), T, s);
    if (err == cudaSuccess) return STENCIL_OK;
    note_cuda_error(err);
    if (err == cudaErrorMemoryAllocation) return STENCIL_ENOMEM;
    if (err == cudaErrorInvalidValue) return STENCIL_EUNSUPPORTED;
    return STENCIL_ECUDA;
}

int aperiodic_prepare(stencil_plan_s* p, int64_t T) {
    if (p->radius == 0 || !any_reach(p)) return STENCIL_OK;   // solved by the periodic path
    Schedule* sc = nullptr;
    const cudaError_t err = prepare_all(p, T, &sc);
    if (err == cudaSuccess) return STENCIL_OK;
    note_cuda_error(err);
    if (err == cudaErrorMemoryAllocation) return STENCIL_ENOMEM;
    if (err == cudaErrorInvalidValue) return STENCIL_EUNSUPPORTED;
    return STENCIL_ECUDA;
}

void aperiodic_release(stencil_plan_s* p) {
    if (!p || !p->ap) return;
    AperiodicState* st = p->ap;
    for (auto& kv : st->graphs) cudaGraphExecDestroy(kv.second);
    for (auto& L : st->levels) {
        cudaFree(L.S);
        cudaFree(L.H);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.fork) cudaEventDestroy(L.fork);
        if (L.done) cudaEventDestroy(L.done);
    }
    for (auto& kv : st->base) cudaFree(kv.second.tiles);
    for (auto& kv : st->schedules)
        for (auto& v : kv.second.tables) cudaFree(v.buf);
    cudaFree(st->Y);
    cudaFree(st->Z);
    if (st->cap) cudaStreamDestroy(st->cap);
    if (st->interior) cudaStreamDestroy(st->interior);
    if (st->int_fork) cudaEventDestroy(st->int_fork);
    if (st->int_done) cudaEventDestroy(st->int_done);
    delete st;
    p->ap = nullptr;
}

// Host-only export of the zero-Dirichlet schedule (see stencilfft.h).
extern "C" int64_t stencil_debug_schedule_reach(int ndim, const int64_t* dims, int radius,
                                                const int* reach, int64_t T, int64_t cutoff,
                                                int64_t* out, int64_t cap) {
    if (ndim < 1 || ndim > 3 || !dims || radius < 1 || radius > kMaxRadius || T < 1 ||
        (cutoff != 0 && cutoff < 2))
        return -1;
    stencil_plan_s p;
    p.ndim = ndim;
    p.radius = radius;
    p.elem = sizeof(float);
    p.precision = STENCIL_FP32;
    p.cutoff = cutoff;
    for (int a = 0; a < ndim; ++a) {
        if (dims[a] < 4 || ilog2_exact(dims[a]) < 0) return -1;
        p.dims[a] = dims[a];
        for (int side = 0; side < 2; ++side) {
            const int v = reach ? reach[2 * a + side] : radius;
            if (v < 0 || v > radius) return -1;
            p.reach[a][side] = v;
        }
    }
    if (!any_reach(&p)) return -1;
    p.n_cells = 1;
    for (int a = 0; a < ndim; ++a) p.n_cells *= dims[a];
    p.nweights = 1;
    for (int a = 0; a < ndim; ++a) p.nweights *= 2 * radius + 1;
    Schedule sc;
    build_rb(&p, sc, T, 0, auto_cutoff(&p, p.cutoff));
    if (cutoff == 0) {
        Schedule loop;
        const double c_loop = build_loop(&p, loop, T);
        if (c_loop < schedule_cost(&p, sc, T)) sc = std::move(loop);
    }
    std::vector<int64_t> v;
    for (const Op& op : sc.ops) {
        if (op.kind == Op::LOOP || op.kind == Op::STEP || op.kind == Op::CLUSTER) {
            v.push_back(op.kind == Op::LOOP ? 4 : op.kind == Op::STEP ? 5 : 6);
            v.push_back(op.T);
            continue;
        }
        if (op.kind == Op::BASE) {
            size_t smem = 0;
            std::vector<BaseTile> tiles = make_base_tiles(&p, op.T, &smem);
            v.push_back(3);
            v.push_back(op.T);
            for (int f = 0; f < 6; ++f)
                v.push_back(f < 2 * ndim ? std::min<int64_t>(reach_to(&p, f) * op.T, kNoHi) : 0);
            v.push_back((int64_t)tiles.size());
            for (const BaseTile& t : tiles)
                for (int a = 0; a < 3; ++a) {
                    v.push_back(t.lo[a]);
                    v.push_back(t.hi[a]);
                }
            continue;
        }
        const Step& st = sc.steps[op.step];
        if (op.kind == Op::SCATTER) {
            v.push_back(2);
            v.push_back(op.step);
            continue;
        }
        int nitems = 0;
        for (const Batch& b : st.batches) nitems += b.geom.items;
        v.push_back(1);
        v.push_back(op.step);
        v.push_back(st.T);
        v.push_back(st.level);
        v.push_back(nitems);
        for (const Batch& b : st.batches) {
            for (int i = 0; i < b.geom.items; ++i) {
                const ItemGeom& g = b.geom.it[i];
                for (int a = 0; a < 3; ++a) v.push_back(b.bdims[a]);
                for (int a = 0; a < 3; ++a) v.push_back(g.off[a]);
                for (int a = 0; a < 3; ++a) v.push_back(g.valid[a]);
                for (int a = 0; a < 3; ++a) v.push_back(g.perm[a]);
                for (int f = 0; f < 6; ++f) v.push_back(b.geom.lo[f]);
                for (int f = 0; f < 6; ++f) v.push_back(b.geom.hi[f]);
                v.push_back(g.face_axis);
                v.push_back(g.face_side);
            }
        }
    }
    if (out && cap > 0)
        for (int64_t i = 0; i < (int64_t)v.size() && i < cap; ++i) out[i] = v[i];
    return (int64_t)v.size();
}

extern "C" int64_t stencil_debug_schedule(int ndim, const int64_t* dims, int radius, int64_t T,
                                          int64_t cutoff, int64_t* out, int64_t cap) {
    return stencil_debug_schedule_reach(ndim, dims, radius, nullptr, T, cutoff, out, cap);
}
