/*
 * FP64 exact ray/voxel intersection lengths (the system matrix H of the
 * forward model, Sec. II: h(y|x) is the length of the intersection of ray
 * path y with voxel x).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is part of the CPU oracle: only the
 * tests, the smoke check and the CPU-baseline leg of the benchmark may load
 * it.  It shares no code with the CUDA path.
 *
 * Method: Siddon's parametric traversal, in its plainest form.  A ray is the
 * segment P(a) = P1 + a (P2 - P1), a in [0, 1].  Every parameter value at
 * which it crosses a grid plane is collected, the list is sorted, and each
 * pair of consecutive values bounds one piece of the ray that lies inside one
 * voxel; that voxel is found from the piece's midpoint and the piece's length
 * is (a_{k+1} - a_k) |P2 - P1|.  No incremental stepping, no blocking.
 *
 * Grid: nx * ny (* nz) voxels of size vx * vy (* vz) mm, centred at the
 * origin, voxel index (iz * ny + iy) * nx + ix (x fastest).  A voxel owns the
 * half-open box [x_i, x_{i+1}) x [y_j, y_{j+1}) (x [z_k, z_{k+1})), so a ray
 * lying exactly on a grid plane is given to the voxel above that plane.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_double(const void* a, const void* b)
{
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* Range of the parameter a for which coordinate p1 + a*dp lies in [lo, hi).
 * Returns 0 if the ray never enters the slab. */
static int slab_range(double p1, double dp, double lo, double hi, double* amin, double* amax)
{
    if (dp == 0.0) {
        if (p1 >= lo && p1 < hi) { *amin = -INFINITY; *amax = INFINITY; return 1; }
        return 0;
    }
    double a0 = (lo - p1) / dp, a1 = (hi - p1) / dp;
    *amin = a0 < a1 ? a0 : a1;
    *amax = a0 < a1 ? a1 : a0;
    return 1;
}

/*
 * Intersections of one segment with the grid.  dims = 2 or 3.  p1, p2 hold
 * (x, y[, z]).  Writes up to the returned count of (voxel, length) pairs, in
 * order along the ray, into idx/len when they are non-NULL.  work must hold
 * nx + ny + nz + 8 doubles.
 */
static int64_t siddon(int dims, const double* p1, const double* p2, const int* n, const double* v,
                      int64_t* idx, double* len, double* work)
{
    double d[3] = {0, 0, 0}, lo[3], amin = 0.0, amax = 1.0, length = 0.0;
    for (int k = 0; k < dims; ++k) {
        d[k] = p2[k] - p1[k];
        length += d[k] * d[k];
        lo[k] = -0.5 * n[k] * v[k];
    }
    length = sqrt(length);
    for (int k = 0; k < dims; ++k) {
        double a0, a1;
        if (!slab_range(p1[k], d[k], lo[k], lo[k] + n[k] * v[k], &a0, &a1)) return 0;
        if (a0 > amin) amin = a0;
        if (a1 < amax) amax = a1;
    }
    if (!(amax > amin)) return 0;

    int m = 0;
    work[m++] = amin;
    work[m++] = amax;
    for (int k = 0; k < dims; ++k) {
        if (d[k] == 0.0) continue;
        for (int i = 0; i <= n[k]; ++i) {
            double a = (lo[k] + i * v[k] - p1[k]) / d[k];
            if (a > amin && a < amax) work[m++] = a;
        }
    }
    qsort(work, (size_t)m, sizeof(double), cmp_double);

    int64_t count = 0;
    for (int s = 0; s + 1 < m; ++s) {
        double a0 = work[s], a1 = work[s + 1];
        if (!(a1 > a0)) continue;
        double mid = 0.5 * (a0 + a1);
        int64_t flat = 0, stride = 1, inside = 1;
        for (int k = 0; k < dims; ++k) {
            double c = p1[k] + mid * d[k];
            int64_t i = (int64_t)floor((c - lo[k]) / v[k]);
            if (i < 0 || i >= n[k]) { inside = 0; break; }
            flat += i * stride;
            stride *= n[k];
        }
        if (!inside) continue;
        if (idx) { idx[count] = flat; len[count] = (a1 - a0) * length; }
        ++count;
    }
    return count;
}

/* Number of intersected voxels of each ray.  seg: nrays * 2*dims doubles,
 * (p1, p2) per ray. */
void or_siddon_counts(int dims, int64_t nrays, const double* seg, const int* n, const double* v,
                      int64_t* counts)
{
    int64_t wn = (int64_t)n[0] + n[1] + (dims == 3 ? n[2] : 0) + 8;
#pragma omp parallel
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)wn);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nrays; ++r)
            counts[r] = siddon(dims, seg + r * 2 * dims, seg + r * 2 * dims + dims, n, v, NULL, NULL, work);
        free(work);
    }
}

/* Fill the CSR arrays of H given row pointers from or_siddon_counts. */
void or_siddon_fill(int dims, int64_t nrays, const double* seg, const int* n, const double* v,
                    const int64_t* rowptr, int64_t* cols, double* vals)
{
    int64_t wn = (int64_t)n[0] + n[1] + (dims == 3 ? n[2] : 0) + 8;
#pragma omp parallel
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)wn);
#pragma omp for schedule(dynamic, 64)
        for (int64_t r = 0; r < nrays; ++r)
            siddon(dims, seg + r * 2 * dims, seg + r * 2 * dims + dims, n, v, cols + rowptr[r], vals + rowptr[r],
                   work);
        free(work);
    }
}
