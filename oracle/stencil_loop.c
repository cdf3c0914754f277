/*
 * Oracle: plain FP64 nested-loop stencil evolution on the CPU.
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously correct
 * definition the GPU path is checked against. Only tests, the smoke check
 * and the bench's CPU-baseline leg may build, load or call it. It shares no
 * code, header, table or helper with the CUDA library.
 *
 * What it computes (paper Sec. 1, "Problem Specification"; looping codes of
 * Fig. "looping-code", PStencil-Loop / AStencil-Loop; d-D indexing of the
 * appendix "Supporting d-D Spatial Grids"):
 *
 *     a_{t+1}[i] = sum over m in [-r, r]^d of  w[m] * a_t[i + m]
 *
 * for t = 0 .. T-1, where
 *   - periodic grids (boundary 0) wrap every index modulo the axis length
 *     (the grid is a torus, Sec. 1);
 *   - zero-Dirichlet grids (boundary 1) read a_t[j] = 0 for every j outside
 *     the grid: every one of the N cells evolves, and a ring of ghost cells
 *     held at 0 supplies the missing neighbours. This is the aperiodic loop of
 *     Fig. "looping-code" with the boundary condition "cells beyond the grid
 *     are zero" (the paper leaves the condition generic).
 *   - reflecting (zero-flux Neumann) grids (boundary 2) read the mirror image
 *     across the cell face: index -1-k reads cell k, index l+k reads cell
 *     l-1-k (half-sample symmetric ghosts, refreshed every step from the
 *     current values). Sec. 5.1 names Neumann among the aperiodic conditions
 *     the method covers; the radius must not exceed the axis length.
 *
 * The weights are the stencil coefficients over the box [-r, r]^d in
 * row-major order, entry (m_1 + r, ..., m_d + r). In the paper's
 * circulant form (Sec. 4, "Mathematical Formulation") the first column of S
 * is s[(-m) mod l] = w[m].
 *
 * Summation order is fixed: m in row-major order. Double buffering, T
 * sequential steps, and an OpenMP parallel loop over cells, as in the paper's
 * looping codes (their inner loops are "parallel for" over i).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static int64_t wrap(int64_t i, int64_t n) {
    int64_t q = i % n;
    return q < 0 ? q + n : q;
}

/* Mirror image of an index at most n cells outside [0, n). */
static int64_t mirror(int64_t i, int64_t n) {
    if (i < 0) return -1 - i;
    if (i >= n) return 2 * n - 1 - i;
    return i;
}

/* One step b = S a. Grid shape l0 x l1 x l2 (unused leading axes have
 * length 1 and radius 0). r[k] is the stencil radius along axis k, and the
 * weights are (2r0+1) x (2r1+1) x (2r2+1) row-major. */
static void one_step(const int64_t l[3], const int r[3], const double* w,
                     int boundary, const double* a, double* b) {
    const int64_t n = l[0] * l[1] * l[2];
    const int w1 = 2 * r[1] + 1, w2 = 2 * r[2] + 1;
#pragma omp parallel for schedule(static)
    for (int64_t cell = 0; cell < n; ++cell) {
        const int64_t i0 = cell / (l[1] * l[2]);
        const int64_t i1 = (cell / l[2]) % l[1];
        const int64_t i2 = cell % l[2];
        double acc = 0.0;
        for (int m0 = -r[0]; m0 <= r[0]; ++m0) {
            for (int m1 = -r[1]; m1 <= r[1]; ++m1) {
                for (int m2 = -r[2]; m2 <= r[2]; ++m2) {
                    int64_t j0 = i0 + m0, j1 = i1 + m1, j2 = i2 + m2;
                    if (boundary == 0) {
                        j0 = wrap(j0, l[0]);
                        j1 = wrap(j1, l[1]);
                        j2 = wrap(j2, l[2]);
                    } else if (boundary == 2) {
                        j0 = mirror(j0, l[0]);
                        j1 = mirror(j1, l[1]);
                        j2 = mirror(j2, l[2]);
                    } else if (j0 < 0 || j0 >= l[0] || j1 < 0 || j1 >= l[1] ||
                               j2 < 0 || j2 >= l[2]) {
                        continue; /* ghost cell: value 0 */
                    }
                    const double wm =
                        w[((m0 + r[0]) * w1 + (m1 + r[1])) * w2 + (m2 + r[2])];
                    acc += wm * a[(j0 * l[1] + j1) * l[2] + j2];
                }
            }
        }
        b[cell] = acc;
    }
}

/*
 * Evolve a0 by T steps into out (both hold prod(dims) doubles, row-major,
 * last axis contiguous). ndim in 1..3, radius >= 0, boundary 0 = periodic,
 * 1 = zero Dirichlet, 2 = reflecting (radius <= every axis length).
 * nthreads <= 0 keeps the OpenMP default.
 * Returns 0 on success, -1 on bad arguments, -2 if scratch allocation fails.
 */
int oracle_stencil_loop(int ndim, const int64_t* dims, int radius,
                        const double* weights, int boundary, int64_t T,
                        const double* a0, double* out, int nthreads) {
    if (ndim < 1 || ndim > 3 || radius < 0 || T < 0 || !dims || !weights ||
        !a0 || !out || boundary < 0 || boundary > 2)
        return -1;
    int64_t l[3] = {1, 1, 1};
    int r[3] = {0, 0, 0};
    for (int k = 0; k < ndim; ++k) {
        if (dims[k] < 1 || (boundary == 2 && radius > dims[k])) return -1;
        l[3 - ndim + k] = dims[k];
        r[3 - ndim + k] = radius;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    const int64_t n = l[0] * l[1] * l[2];
    double* cur = (double*)malloc((size_t)n * sizeof(double));
    double* nxt = (double*)malloc((size_t)n * sizeof(double));
    if (!cur || !nxt) {
        free(cur);
        free(nxt);
        return -2;
    }
    memcpy(cur, a0, (size_t)n * sizeof(double));
    for (int64_t t = 0; t < T; ++t) {
        one_step(l, r, weights, boundary, cur, nxt);
        double* tmp = cur;
        cur = nxt;
        nxt = tmp;
    }
    memcpy(out, cur, (size_t)n * sizeof(double));
    free(cur);
    free(nxt);
    return 0;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
