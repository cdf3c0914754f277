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
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <vector>

#include "../../include/stencilfft.h"
#include "internal.h"
#include "plan_impl.h"

using namespace sfft;

namespace {

constexpr int kNoHi = 0x3fffffff;

// A box of the grid: box cell q (row-major over bdims) maps to grid cell
// off + q when q_a < valid_a on every axis.
struct BoxGeom {
    int ndim;
    int gdims[3];
    int bdims[3];
    int off[3];
    int valid[3];
};

// Which cells a scatter writes: dist in (lo, hi]; with face_axis >= 0 also
// the distance to that face must be <= hi.
struct CellMask {
    int lo, hi;
    int face_axis, face_side;
};

__device__ __forceinline__ int cell_dist(const int* g, const int* gd, int ndim) {
    int d = 0x7fffffff;
    for (int a = 0; a < ndim; ++a) d = min(d, min(g[a] + 1, gd[a] - g[a]));
    return d;
}

__device__ __forceinline__ bool mask_ok(const int* g, const BoxGeom& b, const CellMask& m) {
    const int d = cell_dist(g, b.gdims, b.ndim);
    if (d <= m.lo || d > m.hi) return false;
    if (m.face_axis >= 0) {
        const int a = m.face_axis;
        const int df = m.face_side == 0 ? g[a] + 1 : b.gdims[a] - g[a];
        if (df > m.hi) return false;
    }
    return true;
}

__device__ __forceinline__ void box_coords(long long e, const BoxGeom& b, int* q) {
    for (int a = b.ndim - 1; a >= 0; --a) {
        q[a] = (int)(e % b.bdims[a]);
        e /= b.bdims[a];
    }
}

__device__ __forceinline__ long long grid_index(const int* g, const BoxGeom& b) {
    long long idx = 0;
    for (int a = 0; a < b.ndim; ++a) idx = idx * b.gdims[a] + g[a];
    return idx;
}

template <typename R>
__global__ void k_gather(const R* __restrict__ X, R* __restrict__ S,
                         const __grid_constant__ BoxGeom b, long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int q[3], g[3];
        box_coords(e, b, q);
        bool in = true;
        for (int a = 0; a < b.ndim; ++a) {
            in &= q[a] < b.valid[a];
            g[a] = b.off[a] + q[a];
        }
        S[e] = in ? X[grid_index(g, b)] : R(0);
    }
}

template <typename R>
__global__ void k_scatter(const R* __restrict__ S, R* __restrict__ X,
                          const __grid_constant__ BoxGeom b, const __grid_constant__ CellMask m,
                          long long total) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        int q[3], g[3];
        box_coords(e, b, q);
        bool in = true;
        for (int a = 0; a < b.ndim; ++a) {
            in &= q[a] < b.valid[a];
            g[a] = b.off[a] + q[a];
        }
        if (in && mask_ok(g, b, m)) X[grid_index(g, b)] = S[e];
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
    int wout;         // write cells with dist <= wout
    double w[kMaxWeights];
};

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
        int d = 0x7fffffff;
        for (int a = 3 - p.ndim; a < 3; ++a) d = min(d, min(g3[a] + 1, gd[a] - g3[a]));
        if (d > p.wout) continue;
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
        int d = 0x7fffffff;
        for (int a = off; a < 3; ++a) d = min(d, min(g3[a] + 1, gd[a] - g3[a]));
        if (d > p.wout) continue;
        const long long gi = ((long long)g3[0] * gd[1] + g3[1]) * gd[2] + g3[2];
        X[gi] = Y[gi];
    }
}

int64_t next_pow2(int64_t v) {
    int64_t p = 1;
    while (p < v) p <<= 1;
    return p;
}

}  // namespace

// ---------------------------------------------------------------------------
// host: schedule and buffers
// ---------------------------------------------------------------------------
struct StripSolve {
    int64_t bdims[3];
    BoxGeom geom;
    CellMask mask;
};

struct StripStep {       // all periodic solves of one P1 or P2 step
    int level;
    int64_t T;           // steps of this periodic solve
    std::vector<StripSolve> strips;
};

struct Op {
    enum Kind { SOLVE, SCATTER, BASE } kind;
    int step;            // index into steps (SOLVE / SCATTER)
    int64_t T;           // BASE: steps
};

struct LevelBuffers {
    std::vector<void*> S;      // strip real buffers
    std::vector<void*> H;      // strip half-spectrum workspaces
    std::vector<size_t> S_bytes, H_bytes;
};

struct BaseSet {
    void* tiles = nullptr;     // device BaseTile[count]
    int count = 0;
    size_t smem = 0;
};

struct Schedule {
    std::vector<StripStep> steps;
    std::vector<Op> ops;
};

struct AperiodicState {
    std::map<int64_t, Schedule> schedules;   // per T
    std::vector<LevelBuffers> levels;
    std::map<int64_t, BaseSet> base;         // per base-case T
    void* Y = nullptr;                       // full-grid scratch of the base case
    void* Z = nullptr;                       // interior result
};

static int box_Mp(int64_t n, int precision) {
    const int64_t align = precision == STENCIL_FP32 ? 16 : 8;
    return (int)((n + 1 + align - 1) / align * align);
}

// The strips of a periodic solve over the region dist <= W, keeping (lo, hi].
static std::vector<StripSolve> make_strips(const stencil_plan_s* p, int64_t W, int lo, int hi) {
    std::vector<StripSolve> out;
    const int d = p->ndim;
    bool whole = false;
    for (int a = 0; a < d; ++a) {
        const int64_t P = next_pow2(std::max<int64_t>({W, 4, 2 * p->radius + 1}));
        if (2 * P >= p->dims[a]) whole = true;
    }
    BoxGeom base;
    std::memset(&base, 0, sizeof(base));
    base.ndim = d;
    for (int a = 0; a < d; ++a) {
        base.gdims[a] = (int)p->dims[a];
        base.bdims[a] = (int)p->dims[a];
        base.off[a] = 0;
        base.valid[a] = (int)p->dims[a];
    }
    if (whole) {
        StripSolve s;
        s.geom = base;
        for (int a = 0; a < 3; ++a) s.bdims[a] = a < d ? p->dims[a] : 1;
        s.mask = CellMask{lo, hi, -1, 0};
        out.push_back(s);
        return out;
    }
    for (int a = 0; a < d; ++a) {
        for (int side = 0; side < 2; ++side) {
            StripSolve s;
            s.geom = base;
            const int64_t P = next_pow2(std::max<int64_t>({W, 4, 2 * p->radius + 1}));
            s.geom.bdims[a] = (int)P;
            s.geom.valid[a] = (int)W;
            s.geom.off[a] = side == 0 ? 0 : (int)(p->dims[a] - W);
            for (int b = 0; b < 3; ++b) s.bdims[b] = b < d ? s.geom.bdims[b] : 1;
            s.mask = CellMask{lo, hi, a, side};
            out.push_back(s);
        }
    }
    return out;
}

static void build_rb(const stencil_plan_s* p, Schedule& sc, int64_t T, int level, int64_t cutoff) {
    const int sigma = p->radius;
    if (T < cutoff) {
        sc.ops.push_back(Op{Op::BASE, -1, T});
        return;
    }
    const int64_t T1 = T / 2, T2 = T - T1;
    // Step 1
    StripStep s1;
    s1.level = level;
    s1.T = T1;
    s1.strips = make_strips(p, 2 * sigma * T, (int)(sigma * T1),
                            (int)std::min<int64_t>(sigma * T + sigma * T2, kNoHi));
    sc.steps.push_back(s1);
    const int i1 = (int)sc.steps.size() - 1;
    sc.ops.push_back(Op{Op::SOLVE, i1, 0});
    build_rb(p, sc, T1, level + 1, cutoff);
    sc.ops.push_back(Op{Op::SCATTER, i1, 0});
    // Step 2
    StripStep s2;
    s2.level = level;
    s2.T = T2;
    s2.strips = make_strips(p, sigma * T + sigma * T2, (int)(sigma * T2), (int)(sigma * T));
    sc.steps.push_back(s2);
    const int i2 = (int)sc.steps.size() - 1;
    sc.ops.push_back(Op{Op::SOLVE, i2, 0});
    build_rb(p, sc, T2, level + 1, cutoff);
    sc.ops.push_back(Op{Op::SCATTER, i2, 0});
}

static int64_t auto_cutoff(const stencil_plan_s* p) {
    if (p->cutoff >= 2) return p->cutoff;
    // the loop's cost per leaf grows with T_b^2 while each recursion level costs
    // about three frame-sized FFT solves; these values balance the two on GB300
    if (p->ndim == 1) return 256;
    if (p->ndim == 2) return 32;
    return 8;
}

static cudaError_t ensure_level(stencil_plan_s* p, AperiodicState* st, const StripStep& step) {
    if ((int)st->levels.size() <= step.level) st->levels.resize(step.level + 1);
    LevelBuffers& L = st->levels[step.level];
    const size_t n = step.strips.size();
    if (L.S.size() < n) {
        L.S.resize(n, nullptr);
        L.H.resize(n, nullptr);
        L.S_bytes.resize(n, 0);
        L.H_bytes.resize(n, 0);
    }
    for (size_t j = 0; j < n; ++j) {
        const StripSolve& s = step.strips[j];
        int64_t cells = 1;
        for (int a = 0; a < p->ndim; ++a) cells *= s.bdims[a];
        const size_t sb = (size_t)cells * p->elem;
        const size_t hb = periodic_workspace_bytes(p->ndim, s.bdims, p->precision);
        if (L.S_bytes[j] < sb) {
            cudaFree(L.S[j]);
            L.S[j] = nullptr;
            cudaError_t err = cudaMalloc(&L.S[j], sb);
            if (err != cudaSuccess) return err;
            L.S_bytes[j] = sb;
        }
        if (L.H_bytes[j] < hb) {
            cudaFree(L.H[j]);
            L.H[j] = nullptr;
            cudaError_t err = cudaMalloc(&L.H[j], hb);
            if (err != cudaSuccess) return err;
            L.H_bytes[j] = hb;
        }
    }
    return cudaSuccess;
}

// Output tiles of the frame dist <= w for the base case.
static std::vector<BaseTile> make_base_tiles(const stencil_plan_s* p, int64_t Tb, size_t* smem) {
    const int d = p->ndim;
    const int w = (int)(p->radius * Tb);
    const int h = w;
    const size_t budget = 160 * 1024 / (2 * p->elem);  // cells per buffer
    std::vector<BaseTile> tiles;
    // regions: bands per face, earlier axes' bands excluded
    struct Region { int lo[3], hi[3]; int normal; };
    std::vector<Region> regions;
    bool whole = false;
    for (int a = 0; a < d; ++a)
        if (2 * (int64_t)w >= p->dims[a]) whole = true;
    if (whole) {
        Region r;
        for (int a = 0; a < 3; ++a) { r.lo[a] = 0; r.hi[a] = a < d ? (int)p->dims[a] : 1; }
        r.normal = -1;
        regions.push_back(r);
    } else {
        for (int a = 0; a < d; ++a) {
            for (int side = 0; side < 2; ++side) {
                Region r;
                r.normal = a;
                bool empty = false;
                for (int b = 0; b < 3; ++b) {
                    if (b >= d) { r.lo[b] = 0; r.hi[b] = 1; continue; }
                    if (b == a) {
                        r.lo[b] = side == 0 ? 0 : (int)p->dims[b] - w;
                        r.hi[b] = side == 0 ? w : (int)p->dims[b];
                    } else if (b < a) {
                        r.lo[b] = w;
                        r.hi[b] = (int)p->dims[b] - w;
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
        auto vol = [&](void) {
            size_t v = 1;
            for (int b = 0; b < d; ++b) v *= (size_t)std::min(cs[b] + 2 * h, (int)p->dims[b]);
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
    *smem = 2 * max_vol * p->elem;
    return tiles;
}

template <typename R>
static cudaError_t launch_base(stencil_plan_s* p, const BaseSet& bs, R* X, R* Y, int64_t Tb,
                              cudaStream_t s) {
    BaseParams bp;
    std::memset(&bp, 0, sizeof(bp));
    bp.ndim = p->ndim;
    for (int a = 0; a < p->ndim; ++a) bp.gdims[a] = (int)p->dims[a];
    bp.Tb = (int)Tb;
    bp.wout = (int)(p->radius * Tb);
    for (int i = 0; i < p->nweights; ++i) bp.w[i] = p->weights[i];
    const BaseTile* tiles = static_cast<const BaseTile*>(bs.tiles);
    cudaError_t err = cudaSuccess;
    p->prof.begin(PASS_BASE_LOOP, s);
    switch (p->radius) {
#define SFFT_BASE_CASE(RADV)                                                                  \
    case RADV:                                                                                \
        if (bs.smem > 48 * 1024)                                                              \
            err = cudaFuncSetAttribute(k_base_tiles<R, RADV>,                                 \
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs.smem); \
        if (err == cudaSuccess) {                                                             \
            k_base_tiles<R, RADV><<<bs.count, 256, bs.smem, s>>>(X, Y, tiles, bp);            \
            err = cudaGetLastError();                                                         \
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
    k_tile_copy<R><<<bs.count, 256, 0, s>>>(Y, X, tiles, bp);
    err = cudaGetLastError();
    p->prof.end(s);
    return err;
}

static int grid_blocks(long long total) {
    long long b = (total + 255) / 256;
    return (int)std::max<long long>(1, std::min<long long>(b, 152 * 16));
}

template <typename R>
static cudaError_t run_schedule(stencil_plan_s* p, AperiodicState* st, const Schedule& sc, R* X,
                                cudaStream_t s) {
    cudaError_t err;
    for (const Op& op : sc.ops) {
        if (op.kind == Op::BASE) {
            auto it = st->base.find(op.T);
            err = launch_base<R>(p, it->second, X, static_cast<R*>(st->Y), op.T, s);
            if (err != cudaSuccess) return err;
            continue;
        }
        const StripStep& step = sc.steps[op.step];
        LevelBuffers& L = st->levels[step.level];
        for (size_t j = 0; j < step.strips.size(); ++j) {
            const StripSolve& ss = step.strips[j];
            long long total = 1;
            for (int a = 0; a < p->ndim; ++a) total *= ss.bdims[a];
            R* S = static_cast<R*>(L.S[j]);
            if (op.kind == Op::SOLVE) {
                p->prof.begin(PASS_COPY, s);
                k_gather<R><<<grid_blocks(total), 256, 0, s>>>(X, S, ss.geom, total);
                err = cudaGetLastError();
                p->prof.end(s);
                if (err != cudaSuccess) return err;
                const int64_t n = ss.bdims[p->ndim - 1] / 2;
                err = periodic_solve<R>(p, S, ss.bdims, step.T, L.H[j], box_Mp(n, p->precision),
                                        p->tw, p->twn_log2, p->E64, p->E32, p->status, s);
                if (err != cudaSuccess) return err;
            } else {
                p->prof.begin(PASS_COPY, s);
                k_scatter<R><<<grid_blocks(total), 256, 0, s>>>(S, X, ss.geom, ss.mask, total);
                err = cudaGetLastError();
                p->prof.end(s);
                if (err != cudaSuccess) return err;
            }
        }
    }
    return cudaSuccess;
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
    }
    auto it = st->schedules.find(T);
    if (it == st->schedules.end()) {
        Schedule sc;
        build_rb(p, sc, T, 0, auto_cutoff(p));
        for (const StripStep& step : sc.steps) {
            err = ensure_level(p, st, step);
            if (err != cudaSuccess) return err;
        }
        for (const Op& op : sc.ops) {
            if (op.kind != Op::BASE || st->base.count(op.T)) continue;
            BaseSet bs;
            std::vector<BaseTile> tiles = make_base_tiles(p, op.T, &bs.smem);
            bs.count = (int)tiles.size();
            if (bs.smem > (size_t)kSmemBudget) return cudaErrorInvalidValue;
            err = cudaMalloc(&bs.tiles, sizeof(BaseTile) * std::max<size_t>(1, tiles.size()));
            if (err != cudaSuccess) return err;
            err = cudaMemcpy(bs.tiles, tiles.data(), sizeof(BaseTile) * tiles.size(),
                             cudaMemcpyHostToDevice);
            if (err != cudaSuccess) return err;
            st->base[op.T] = bs;
        }
        it = st->schedules.emplace(T, std::move(sc)).first;
    }
    *out = &it->second;
    return cudaSuccess;
}

template <typename R>
static cudaError_t aperiodic_impl(stencil_plan_s* p, R* grid, int64_t T, cudaStream_t s) {
    const int sigma = p->radius;
    if (sigma == 0)  // a pointwise stencil never feels the boundary
        return periodic_solve<R>(p, grid, p->dims, T, p->H, p->Mp, p->tw, p->twn_log2, p->E64,
                                 p->E32, p->status, s);
    int64_t maxdist = p->dims[0] / 2;
    for (int a = 1; a < p->ndim; ++a) maxdist = std::min(maxdist, p->dims[a] / 2);
    const bool interior = sigma * T < maxdist;
    Schedule* sc = nullptr;
    cudaError_t err = prepare(p, T, &sc);
    if (err != cudaSuccess) return err;
    AperiodicState* st = p->ap;
    const size_t bytes = (size_t)p->n_cells * p->elem;
    R* Z = nullptr;
    if (interior) {
        if (!st->Z) {
            err = cudaMalloc(&st->Z, bytes);
            if (err != cudaSuccess) {
                st->Z = nullptr;
                return err;
            }
        }
        Z = static_cast<R*>(st->Z);
        // interior (dist > sigma T): the periodic solve of the untouched input
        p->prof.begin(PASS_COPY, s);
        err = cudaMemcpyAsync(Z, grid, bytes, cudaMemcpyDeviceToDevice, s);
        p->prof.end(s);
        if (err != cudaSuccess) return err;
        err = periodic_solve<R>(p, Z, p->dims, T, p->H, p->Mp, p->tw, p->twn_log2, p->E64, p->E32,
                                p->status, s);
        if (err != cudaSuccess) return err;
    }
    // boundary region (dist <= sigma T): RecursiveBoundary in place
    err = run_schedule<R>(p, st, *sc, grid, s);
    if (err != cudaSuccess) return err;
    if (interior) {
        BoxGeom b;
        std::memset(&b, 0, sizeof(b));
        b.ndim = p->ndim;
        for (int a = 0; a < p->ndim; ++a) {
            b.gdims[a] = b.bdims[a] = b.valid[a] = (int)p->dims[a];
            b.off[a] = 0;
        }
        const CellMask m{(int)(sigma * T), kNoHi, -1, 0};
        p->prof.begin(PASS_COPY, s);
        k_scatter<R><<<grid_blocks(p->n_cells), 256, 0, s>>>(Z, grid, b, m, p->n_cells);
        err = cudaGetLastError();
        p->prof.end(s);
        if (err != cudaSuccess) return err;
    }
    return cudaSuccess;
}

int aperiodic_run(stencil_plan_s* p, void* grid, int64_t T, cudaStream_t s) {
    cudaError_t err = p->precision == STENCIL_FP32
                          ? aperiodic_impl<float>(p, static_cast<float*>(grid), T, s)
                          : aperiodic_impl<double>(p, static_cast<double*>(grid), T, s);
    if (err == cudaSuccess) return STENCIL_OK;
    if (err == cudaErrorMemoryAllocation) return STENCIL_ENOMEM;
    if (err == cudaErrorInvalidValue) return STENCIL_EUNSUPPORTED;
    return STENCIL_ECUDA;
}

void aperiodic_release(stencil_plan_s* p) {
    if (!p || !p->ap) return;
    AperiodicState* st = p->ap;
    for (auto& L : st->levels) {
        for (void* b : L.S) cudaFree(b);
        for (void* b : L.H) cudaFree(b);
    }
    for (auto& kv : st->base) cudaFree(kv.second.tiles);
    cudaFree(st->Y);
    cudaFree(st->Z);
    delete st;
    p->ap = nullptr;
}

// Host-only export of the zero-Dirichlet schedule (see stencilfft.h).
extern "C" int64_t stencil_debug_schedule(int ndim, const int64_t* dims, int radius, int64_t T,
                                          int64_t cutoff, int64_t* out, int64_t cap) {
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
    }
    Schedule sc;
    build_rb(&p, sc, T, 0, auto_cutoff(&p));
    std::vector<int64_t> v;
    for (const Op& op : sc.ops) {
        if (op.kind == Op::BASE) {
            size_t smem = 0;
            std::vector<BaseTile> tiles = make_base_tiles(&p, op.T, &smem);
            v.push_back(3);
            v.push_back(op.T);
            v.push_back((int64_t)tiles.size());
            for (const BaseTile& t : tiles)
                for (int a = 0; a < 3; ++a) {
                    v.push_back(t.lo[a]);
                    v.push_back(t.hi[a]);
                }
            continue;
        }
        const StripStep& st = sc.steps[op.step];
        if (op.kind == Op::SCATTER) {
            v.push_back(2);
            v.push_back(op.step);
            continue;
        }
        v.push_back(1);
        v.push_back(op.step);
        v.push_back(st.T);
        v.push_back(st.level);
        v.push_back((int64_t)st.strips.size());
        for (const StripSolve& s : st.strips) {
            for (int a = 0; a < 3; ++a) v.push_back(s.geom.bdims[a]);
            for (int a = 0; a < 3; ++a) v.push_back(s.geom.off[a]);
            for (int a = 0; a < 3; ++a) v.push_back(s.geom.valid[a]);
            v.push_back(s.mask.lo);
            v.push_back(s.mask.hi);
            v.push_back(s.mask.face_axis);
            v.push_back(s.mask.face_side);
        }
    }
    if (out && cap > 0)
        for (int64_t i = 0; i < (int64_t)v.size() && i < cap; ++i) out[i] = v[i];
    return (int64_t)v.size();
}
