// 3-D circular cone-beam kernels (sm_103a, FP32 bulk, FP64 cost and
// update): the same steps as the 2-D path (Algorithm 1 with the Results
// section's tree growth) for a volume, with either the 3-D Haar transform
// (octree blocks, seven details) or the 2-D Haar transform of each z-slice
// under one shared tree (the paper's own 3-D setting).  All sums run in a
// fixed order.
#include <type_traits>
#include "cone3d.cuh"

#include <cmath>
#include "wam_kernels.h"

#include <math.h>

namespace wam {

namespace {

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

template <typename V>
__device__ __forceinline__ V wsum(V x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}
template <typename V>
__device__ __forceinline__ V wmax(V x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const V y = __shfl_down_sync(0xffffffffu, x, o);
        x = x > y ? x : y;
    }
    return x;
}

__device__ __forceinline__ void add_work3(unsigned long long* work, unsigned cnt)
{
    if (!work) return;
    const unsigned m = __activemask();
    const unsigned tot = __reduce_add_sync(m, cnt);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicAdd(work, (unsigned long long)tot);
}

// x with its sign flipped where sgn < 0
__device__ __forceinline__ float flipf(float x, float sgn)
{
    return __int_as_float(__float_as_int(x) ^ (__float_as_int(sgn) & 0x80000000));
}

// 2^-k exactly
__host__ __device__ __forceinline__ double exp2m(int k)
{
#ifdef __CUDA_ARCH__
    return __hiloint2double((1023 - k) << 20, 0);
#else
    return std::ldexp(1.0, -k);
#endif
}

// 2^(-3l/2) (3-D Haar) or 2^-l (2-D Haar per slice), without a division:
// for odd l, 2^(-3l/2) = 2^(-(3l-1)/2) / sqrt(2)
__host__ __device__ __forceinline__ double basis_scale(int z3, int l)
{
    if (!z3) return exp2m(l);
    return (l & 1) ? exp2m((3 * l - 1) / 2) * (1.0 / sqrt(2.0)) : exp2m(3 * l / 2);
}

// ---------------------------------------------------------------------------
// one cone-beam ray: P(t) = P0 + t dir, |dir| = 1, P0 the ray's point in the
// plane through the rotation axis normal to e (|P0| <= the image reach)
// ---------------------------------------------------------------------------
struct Ray3 {
    float px, py, pz, dx, dy, dz, idx, idy, idz, tin, tout;
};

__device__ __forceinline__ float srcp(float d)
{
    float a = fabsf(d);
    a = a < 1e-30f ? 1e-30f : a;
    const float r = 1.0f / a;
    return signbit(d) ? -r : r;
}

__device__ __forceinline__ bool make_ray3(const Geom3& g, int v, int r, int b, Ray3& ray)
{
    const float c = g.cs[2 * v], s = g.cs[2 * v + 1];
    const float ub = ((float)b - g.ucen) * g.pitch;
    const float vr = ((float)r - g.rcen) * g.rpitch;
    const float Dx = -g.sdd * c - ub * s, Dy = -g.sdd * s + ub * c, Dz = vr;
    const float n = g.dlen[(size_t)r * g.B + b];
    const float in = 1.0f / n;
    ray.dx = Dx * in;
    ray.dy = Dy * in;
    ray.dz = Dz * in;
    const float al = g.sod / g.sdd;
    ray.px = -al * ub * s;
    ray.py = al * ub * c;
    ray.pz = al * vr;
    const float tlo = -al * n, thi = (1.0f - al) * n;
    ray.idx = srcp(ray.dx);
    ray.idy = srcp(ray.dy);
    ray.idz = srcp(ray.dz);
    const float X1 = g.X0 + g.nx * g.vx, Y1 = g.Y0 + g.ny * g.vy, Z1 = g.Z0 + g.nz * g.vz;
    const float a0 = (g.X0 - ray.px) * ray.idx, a1 = (X1 - ray.px) * ray.idx;
    const float b0 = (g.Y0 - ray.py) * ray.idy, b1 = (Y1 - ray.py) * ray.idy;
    const float e0 = (g.Z0 - ray.pz) * ray.idz, e1 = (Z1 - ray.pz) * ray.idz;
    ray.tin = fmaxf(tlo, fmaxf(fmaxf(fminf(a0, a1), fminf(b0, b1)), fminf(e0, e1)));
    ray.tout = fminf(thi, fminf(fminf(fmaxf(a0, a1), fmaxf(b0, b1)), fmaxf(e0, e1)));
    return ray.tout > ray.tin;
}

// Visit the leaf blocks crossed by the ray.  leaf: level per voxel (z3) or
// per (ix, iy) (slices); null: every voxel is a leaf.  visit(ix, iy, iz,
// lam, bx0, by0, bz0, chord).  Each step crosses one grid plane forward.
template <typename F>
__device__ __forceinline__ void walk3(const Geom3& g, const uint8_t* __restrict__ leaf, int z3, const Ray3& r,
                                      F&& visit)
{
    float t = r.tin;
    int ix = clampi((int)floorf((r.px + t * r.dx - g.X0) * g.ivx), 0, g.nx - 1);
    int iy = clampi((int)floorf((r.py + t * r.dy - g.Y0) * g.ivy), 0, g.ny - 1);
    int iz = clampi((int)floorf((r.pz + t * r.dz - g.Z0) * g.ivz), 0, g.nz - 1);
    const bool xp = r.idx > 0.0f, yp = r.idy > 0.0f, zp = r.idz > 0.0f;
    const int max_steps = g.nx + g.ny + g.nz + 6;
    for (int step = 0; step < max_steps; ++step) {
        int lam = 0;
        if (leaf) lam = z3 ? (int)leaf[((size_t)iz * g.ny + iy) * g.nx + ix] : (int)leaf[(size_t)iy * g.nx + ix];
        const int bs = 1 << lam, bsz = z3 ? bs : 1;
        const int bx0 = (ix >> lam) << lam, by0 = (iy >> lam) << lam;
        const int bz0 = z3 ? (iz >> lam) << lam : iz;
        const float tx = (g.X0 + (float)(xp ? bx0 + bs : bx0) * g.vx - r.px) * r.idx;
        const float ty = (g.Y0 + (float)(yp ? by0 + bs : by0) * g.vy - r.py) * r.idy;
        const float tz = (g.Z0 + (float)(zp ? bz0 + bsz : bz0) * g.vz - r.pz) * r.idz;
        float te = fminf(fminf(fminf(tx, ty), tz), r.tout);
        te = fmaxf(te, t);
        visit(ix, iy, iz, lam, bx0, by0, bz0, te - t);
        t = te;
        if (te >= r.tout) break;
        const float ex = r.px + te * r.dx, ey = r.py + te * r.dy, ez = r.pz + te * r.dz;
        if (tx <= ty && tx <= tz) {
            ix = xp ? bx0 + bs : bx0 - 1;
            iy = clampi((int)floorf((ey - g.Y0) * g.ivy), by0, by0 + bs - 1);
            iz = clampi((int)floorf((ez - g.Z0) * g.ivz), bz0, bz0 + bsz - 1);
        } else if (ty <= tz) {
            iy = yp ? by0 + bs : by0 - 1;
            ix = clampi((int)floorf((ex - g.X0) * g.ivx), bx0, bx0 + bs - 1);
            iz = clampi((int)floorf((ez - g.Z0) * g.ivz), bz0, bz0 + bsz - 1);
        } else {
            iz = zp ? bz0 + bsz : bz0 - 1;
            ix = clampi((int)floorf((ex - g.X0) * g.ivx), bx0, bx0 + bs - 1);
            iy = clampi((int)floorf((ey - g.Y0) * g.ivy), by0, by0 + bs - 1);
        }
        if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny || (unsigned)iz >= (unsigned)g.nz)
            break;
    }
}

// Exact voxel walk by in-plane strips: the 2-D strip walk with z as a second
// minor axis.  The major axis is the in-plane one whose grid lines the ray
// crosses most often per unit length; when z's lines are crossed no more often
// (strip3_ok), a strip holds at most one crossing of the in-plane minor axis
// and one of z, so one to three voxels, visited in travel order: the crossing
// with the longer piece beyond it comes first.  Both minor positions are
// tracked in oriented voxel units from the entry voxel's edges; the two end
// strips are peeled.  Voxels are addressed in a volume with a one-voxel zero
// apron on every side, (nz + 2) slabs of (nm + 2) strips of (nn + 2):
// lin = ((k + 1)(nm + 2) + (j + 1))(nn + 2) + (c + 1), j the strip, c the minor
// index, k the slice; x-major rays read a copy with x and y exchanged.  A step
// across a face of the volume (only in the exit strip) lands on the apron
// and reads 0, so no range test is needed.  visit(la, ca, lb, cb, lc, cc)
// once per strip.
__device__ __forceinline__ bool strip3_ok(const Geom3& g, const Ray3& r, bool& ymaj)
{
    const float ax = fabsf(r.dx) * g.ivx, ay = fabsf(r.dy) * g.ivy, az = fabsf(r.dz) * g.ivz;
    ymaj = ay >= ax;
    return az <= fmaxf(ax, ay);
}

template <typename F>
__device__ __forceinline__ void traverse_strips3(const Geom3& g, const Ray3& r, bool ymaj, F&& visit)
{
    const float pm = ymaj ? r.py : r.px, pn = ymaj ? r.px : r.py;
    const float dm = ymaj ? r.dy : r.dx, dn = ymaj ? r.dx : r.dy;
    const float vm = ymaj ? g.vy : g.vx, vn = ymaj ? g.vx : g.vy;
    const float ivm = ymaj ? g.ivy : g.ivx, ivn = ymaj ? g.ivx : g.ivy;
    const float M0 = ymaj ? g.Y0 : g.X0, N0 = ymaj ? g.X0 : g.Y0;
    const int nm = ymaj ? g.ny : g.nx, nn = ymaj ? g.nx : g.ny;
    const float idm = ymaj ? r.idy : r.idx, idn = ymaj ? r.idx : r.idy;
    const float sec = fabsf(idm);                      // length per unit of major coordinate
    const float vkn = vn * fabsf(idn), vkz = g.vz * fabsf(r.idz);
    const float sn = dn * idm, sz = r.dz * idm;        // dn / dm, dz / dm
    const float s_in = pm + r.tin * dm, s_out = pm + r.tout * dm;
    const float s_lo = fminf(s_in, s_out), s_hi = fmaxf(s_in, s_out);
    const float n0 = pn - pm * sn, z0 = r.pz - pm * sz;   // minor and z coordinates at major 0
    const bool upn = sn >= 0.0f, upz = sz >= 0.0f;
    const int j0 = clampi((int)floorf((s_lo - M0) * ivm), 0, nm - 1);
    const int j1 = clampi((int)floorf((s_hi - M0) * ivm), 0, nm - 1);
    const int c0 = clampi((int)floorf((fmaf(s_lo, sn, n0) - N0) * ivn), 0, nn - 1);
    const int k0 = clampi((int)floorf((fmaf(s_lo, sz, z0) - g.Z0) * g.ivz), 0, g.nz - 1);
    const float Nc = fmaf((float)c0, vn, N0), Zc = fmaf((float)k0, g.vz, g.Z0);
    const float Gn = fabsf(sn) * ivn, Gz = fabsf(sz) * g.ivz;
    const float Un = (upn ? n0 - Nc : Nc - n0) * ivn, Uz = (upz ? z0 - Zc : Zc - z0) * g.ivz;
    const int sM = nn + 2, sZ = (nm + 2) * (nn + 2);
    const int dln = upn ? 1 : -1, dlz = upz ? sZ : -sZ;
    const float fn0 = upn ? 1.0f : 0.0f, fz0 = upz ? 1.0f : 0.0f;   // the first grid lines ahead, oriented
    int lin = ((k0 + 1) * (nm + 2) + (j0 + 1)) * sM + c0 + 1;
    // One strip: en, ez = the minor and z positions at the strip's end minus
    // the next oriented grid lines; a crossing (e >= 0) puts the last e vk of
    // the chord beyond that line.  En, Ez carry them to the next strip (one
    // line further on a crossing).  In a full strip a piece past a crossing
    // (0 <= e < D) is below the chord D vk, so only the end strips clamp it.
    float En = 0.0f, Ez = 0.0f;
    auto strip = [&](float chord, float en, float ez, auto clamp) {
        const bool cn = en >= 0.0f, cz = ez >= 0.0f;
        const float pn = en * vkn, pz = ez * vkz;
        const float ln = cn ? (decltype(clamp)::value ? fminf(pn, chord) : pn) : 0.0f;   // piece beyond the minor line
        const float lz = cz ? (decltype(clamp)::value ? fminf(pz, chord) : pz) : 0.0f;   // piece beyond the z plane
        const float hi = fmaxf(ln, lz), lo = fminf(ln, lz);
        const int lb = ln > lz ? lin + dln : (cz ? lin + dlz : lin);
        const int lc = lin + (cn ? dln : 0) + (cz ? dlz : 0);
        visit(lin, chord - hi, lb, hi - lo, lc, lo);
        En = cn ? en - 1.0f : en;
        Ez = cz ? ez - 1.0f : ez;
        lin = lc + sM;
    };
    if (j1 == j0) {
        strip((s_hi - s_lo) * sec, fmaf(s_hi, Gn, Un) - fn0, fmaf(s_hi, Gz, Uz) - fz0, std::true_type());
        return;
    }
    const float An = fmaf(Gn, M0, Un), Dn = Gn * vm, Az = fmaf(Gz, M0, Uz), Dz = Gz * vm;
    const float fj = (float)(j0 + 1);
    strip(fmaxf(fmaf(fj, vm, M0) - s_lo, 0.0f) * sec, fmaf(fj, Dn, An) - fn0, fmaf(fj, Dz, Az) - fz0,
          std::true_type());
    const float full = vm * sec;
#pragma unroll 4
    for (int k = j1 - j0 - 1; k > 0; --k) strip(full, En + Dn, Ez + Dz, std::false_type());
    // the last strip ends at the exit point, past the end of strip j1 - 1 by
    // u - A - j1 D on each minor axis
    strip(fmaxf(s_hi - fmaf((float)j1, vm, M0), 0.0f) * sec, En + (fmaf(s_hi, Gn, Un) - fmaf((float)j1, Dn, An)),
          Ez + (fmaf(s_hi, Gz, Uz) - fmaf((float)j1, Dz, Az)), std::true_type());
}

}  // namespace

// The strip walk's two apron-padded volumes: py (z, y, x) and px (z, x, y),
// each (nz + 2)(ny + 2)(nx + 2) with a zero border.  One thread per padded
// voxel; the x-y transposition goes through a 32x32 shared tile per slice.
// Cells of 2^lam x 2^lam x 2^lamz voxels (mu constant on them; lam = 0:
// voxels): nx, ny, nz count cells, nxf, nyf are mu's row and slice sizes, and
// a cell's value is read at its first voxel.
__global__ void k_pad3(const float* __restrict__ mu, int nxf, int nyf, int lam, int lamz, int nx, int ny, int nz,
                       float* __restrict__ py, float* __restrict__ px)
{
    __shared__ float tile[32][33];
    const int x0 = (int)blockIdx.x * 32 - 1, y0 = (int)blockIdx.y * 32 - 1, z = (int)blockIdx.z - 1;
    const size_t slab = (size_t)(nx + 2) * (ny + 2);
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int x = x0 + threadIdx.x, y = y0 + k;
        float v = 0.0f;
        if (x >= 0 && x < nx && y >= 0 && y < ny && z >= 0 && z < nz)
            v = mu[(((size_t)z << lamz) * nyf + ((size_t)y << lam)) * nxf + ((size_t)x << lam)];
        tile[k][threadIdx.x] = v;
        if (x <= nx && y <= ny) py[(size_t)(z + 1) * slab + (size_t)(y + 1) * (nx + 2) + (x + 1)] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int y = y0 + threadIdx.x, x = x0 + k;
        if (x <= nx && y <= ny) px[(size_t)(z + 1) * slab + (size_t)(x + 1) * (ny + 2) + (y + 1)] = tile[threadIdx.x][k];
    }
}

// ---------------------------------------------------------------------------
// a2 + a3: projection (leaf or voxel walk), Beer's law, FP64 cost terms
// ---------------------------------------------------------------------------
template <bool STRIP, bool WORK>
__global__ void __launch_bounds__(kFwdTPB)
k_forward3(Geom3 g, const float* __restrict__ mu, const float* __restrict__ pad, const uint8_t* __restrict__ leaf,
           int z3, const float* __restrict__ d, const double* __restrict__ dterm, const float* __restrict__ I0,
           float* __restrict__ qhat, float* __restrict__ p_out, double* __restrict__ cost_part,
           unsigned long long* __restrict__ work)
{
    const int v = blockIdx.z, r = blockIdx.y;
    const int b = blockIdx.x * kFwdTPB + threadIdx.x;
    double term = 0.0;
    unsigned steps = 0;
    if (b < g.B) {
        Ray3 ray;
        float acc = 0.0f;
        bool ymaj = false;
        if (make_ray3(g, v, r, b, ray)) {
            if (STRIP && strip3_ok(g, ray, ymaj)) {
                // padded volumes: loads run one strip ahead of their use; the
                // sum keeps the walk's order
                const float* img = ymaj ? pad : pad + (size_t)(g.nx + 2) * (g.ny + 2) * (g.nz + 2);
                float pa = 0.0f, va = 0.0f, pb = 0.0f, vb = 0.0f, pc = 0.0f, vc = 0.0f;
                traverse_strips3(g, ray, ymaj, [&](int la, float ca, int lb, float cb, int lc, float cc) {
                    const float wa = __ldg(img + la), wb = __ldg(img + lb), wc = __ldg(img + lc);
                    acc += pa * va;
                    acc += pb * vb;
                    acc += pc * vc;
                    pa = ca; va = wa;
                    pb = cb; vb = wb;
                    pc = cc; vc = wc;
                    if (WORK) steps += (ca > 0.0f) + (cb > 0.0f) + (cc > 0.0f);
                });
                acc += pa * va;
                acc += pb * vb;
                acc += pc * vc;
            } else if (STRIP) {
                // a ray steeper in z than the strip walk allows: the cell walk on
                // the same (possibly coarse) grid, reading the padded row-major copy
                walk3(g, nullptr, z3, ray, [&](int ix, int iy, int iz, int, int, int, int, float c) {
                    acc += c * __ldg(pad + (((size_t)iz + 1) * (g.ny + 2) + iy + 1) * (g.nx + 2) + ix + 1);
                    if (WORK) ++steps;
                });
            } else {
                walk3(g, leaf, z3, ray, [&](int ix, int iy, int iz, int, int, int, int, float c) {
                    acc += c * __ldg(mu + ((size_t)iz * g.ny + iy) * g.nx + ix);
                    if (WORK) ++steps;
                });
            }
        }
        const size_t y = ((size_t)v * g.R + r) * g.B + b;
        if (p_out) p_out[y] = acc;
        if (qhat) {
            const float q = I0[y] * expf(-acc);
            qhat[y] = q;
            term = dterm[y] + (double)d[y] * (double)acc + (double)q;
        }
    }
    if (WORK) add_work3(work, steps);
    if (cost_part) {
        term = wsum(term);
        if ((threadIdx.x & 31) == 0)
            cost_part[(((size_t)v * g.R + r) * gridDim.x + blockIdx.x) * (kFwdTPB / 32) + (threadIdx.x >> 5)] = term;
    }
}

int forward3_parts(const Geom3& g) { return (int)nb(g.B, kFwdTPB) * g.V * g.R * (kFwdTPB / 32); }

cudaError_t launch_forward3(const Geom3& g, const float* mu, float* pad, const uint8_t* leaf, int lam, int z3,
                            const float* d, const double* dterm, const float* I0, float* qhat, float* p_out,
                            double* cost_part, unsigned long long* work, cudaStream_t st)
{
    dim3 grid(nb(g.B, kFwdTPB), g.R, g.V);
    if (!leaf && pad) {
        // the strip walk over the padded cells of 2^lam voxels (2^lam x 2^lam x 1
        // per slice when z3 = 0): same box, larger cells
        const int lamz = z3 ? lam : 0;
        if (lam < 0 || (g.nx >> lam) << lam != g.nx || (g.ny >> lam) << lam != g.ny ||
            (g.nz >> lamz) << lamz != g.nz)
            return cudaErrorInvalidValue;
        Geom3 gc = g;
        gc.nx = g.nx >> lam;
        gc.ny = g.ny >> lam;
        gc.nz = g.nz >> lamz;
        gc.vx = g.vx * (float)(1 << lam);
        gc.vy = g.vy * (float)(1 << lam);
        gc.vz = g.vz * (float)(1 << lamz);
        gc.ivx = g.ivx / (float)(1 << lam);
        gc.ivy = g.ivy / (float)(1 << lam);
        gc.ivz = g.ivz / (float)(1 << lamz);
        count_launch();
        k_pad3<<<dim3(nb(gc.nx + 2, 32), nb(gc.ny + 2, 32), gc.nz + 2), dim3(32, 8), 0, st>>>(
            mu, g.nx, g.ny, lam, lamz, gc.nx, gc.ny, gc.nz, pad, pad + (size_t)(gc.nx + 2) * (gc.ny + 2) * (gc.nz + 2));
        count_launch();
        if (work)
            k_forward3<true, true><<<grid, kFwdTPB, 0, st>>>(gc, mu, pad, leaf, z3, d, dterm, I0, qhat, p_out,
                                                              cost_part, work);
        else
            k_forward3<true, false><<<grid, kFwdTPB, 0, st>>>(gc, mu, pad, leaf, z3, d, dterm, I0, qhat, p_out,
                                                               cost_part, work);
    } else {
        count_launch();
        if (work)
            k_forward3<false, true><<<grid, kFwdTPB, 0, st>>>(g, mu, nullptr, leaf, z3, d, dterm, I0, qhat, p_out,
                                                               cost_part, work);
        else
            k_forward3<false, false><<<grid, kFwdTPB, 0, st>>>(g, mu, nullptr, leaf, z3, d, dterm, I0, qhat, p_out,
                                                                cost_part, work);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a0, a4: voxel-driven split back-projection.  CTA = 32 items x 8 warps (each
// warp its own views).  Per (block, view) the shadow (bins x rows) from the 8
// corners; per ray the chords through the children in crossing-ordered form
// (parameter tau along D = -SDD e + u_b u + v_r z; chords in mm = dtau |D|):
//   x halves [a - Ax, a], [a, a + Ax], y halves [b - Ay, b], [b, b + Ay],
//   z halves [c - Az, c], [c, c + Az]  (first / second along the ray).
// Modes: octet (voxel basis, 2x2x2 voxels: the 8 voxel chords in physical
// order, sums of non-negative terms), 3-D Haar (approximation + 7 details,
// from the centre-plane crossings clamped to the ray's interval in the block,
// no octant chords), per-slice 2-D Haar (the same in the slice's z slab:
// approximation + 3 details), or a single block chord.  Details accumulate
// the signed sum and the absolute sum of qhat * phi, turned into the + and -
// parts after the view loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void decode3(const Segment3& S, int item, int& bx, int& by, int& bz)
{
    if (S.items) {
        const uint32_t w = S.items[S.rep > 0 ? item % S.rep : item];
        bx = (int)(w & 1023u);
        by = (int)((w >> 10) & 1023u);
        bz = S.rep > 0 ? item / S.rep : (int)(w >> 20);
    } else {
        bx = item % S.gw;
        const int rest = item / S.gw;
        by = rest % S.gh;
        bz = rest / S.gh;
    }
}

// Item kinds of a cone-beam back-projection segment.
enum { kBp3Block = 0, kBp3Oct = 1, kBp3Quad = 2, kBp3Octet = 3 };

// The view, row and bin loops of one item, specialised by item kind and work
// counting (no run-time switch in the inner loop; the bin loop is not
// unrolled and the ray offset from the block centre is linear in the bin).
template <int MODE, bool WORK>
__device__ __forceinline__ void bp3_item(const Geom3& g, const Segment3& S, int z3, int bx, int by, int bz,
                                         int chunk, int wv, const float* __restrict__ sino, float (&acc)[kSlots3],
                                         unsigned& evals)
{
    const bool oct = MODE == kBp3Octet;
    const int l = S.level;
    const int bs = 1 << l;
    const int bsz = oct ? 2 : (z3 ? bs : 1);
    const float hx = 0.5f * bs * g.vx, hy = 0.5f * bs * g.vy, hz = 0.5f * bsz * g.vz;
    const float cx = g.X0 + (2 * bx + 1) * hx, cy = g.Y0 + (2 * by + 1) * hy;
    const float cz = g.Z0 + (2 * bz + 1) * hz;
    const float scale = oct ? 1.0f : (float)basis_scale(z3, l);
    const int v0 = chunk * S.vpc, v1 = min(g.V, v0 + S.vpc);
    const float isdd = 1.0f / g.sdd, ipitch = 1.0f / g.pitch, irp = 1.0f / g.rpitch;
    for (int v = v0 + wv; v < v1; v += kViewLanes) {
        const float c = __ldg(g.cs + 2 * v), s = __ldg(g.cs + 2 * v + 1);
        const float ac = cx * c + cy * s, wc = -cx * s + cy * c;
        float umin = 1e30f, umax = -1e30f, vmin = 1e30f, vmax = -1e30f;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float ox = (k & 1) ? hx : -hx, oy = (k & 2) ? hy : -hy, oz = (k & 4) ? hz : -hz;
            const float den = __fdividef(g.sdd, g.sod - (ac + ox * c + oy * s));
            const float uu = (wc - ox * s + oy * c) * den, vv = (cz + oz) * den;
            umin = fminf(umin, uu); umax = fmaxf(umax, uu);
            vmin = fminf(vmin, vv); vmax = fmaxf(vmax, vv);
        }
        // the bins and rows whose rays pass through the shadow; a margin of
        // 1e-3 bin (row) covers the fast division's rounding
        const int blo = max(0, (int)ceilf(umin * ipitch + g.ucen - 1e-3f));
        const int bhi = min(g.B - 1, (int)floorf(umax * ipitch + g.ucen + 1e-3f));
        const int rlo = max(0, (int)ceilf(vmin * irp + g.rcen - 1e-3f));
        const int rhi = min(g.R - 1, (int)floorf(vmax * irp + g.rcen + 1e-3f));
        if (blo > bhi || rlo > rhi) continue;
        const float kappa = (g.sod - ac) * isdd;
        const float dw0 = (((float)blo - g.ucen) * g.pitch) * kappa - wc, dstep = g.pitch * kappa;
        const float4* drow = g.dirt + (size_t)v * g.B;
        for (int rr = rlo; rr <= rhi; ++rr) {
            const float vr = ((float)rr - g.rcen) * g.rpitch;
            const float ri = __ldg(g.rowinv + rr);
            // z intervals (in tau) of the first / second z half and of the whole
            // block; for voxel octets the lower / upper half in physical order
            float z0l, z0h, z1l, z1h, zsl, zsh, zc;
            if (vr != 0.0f) {
                const float cc = -(vr * kappa - cz) * ri;      // z centre-plane crossing
                zc = cc;
                if (oct) {
                    const float Hz = 0.5f * hz, uz = fabsf(ri) + ri, wz = fabsf(ri) - ri;
                    z0l = fmaf(-Hz, uz, cc); z0h = fmaf(Hz, wz, cc);      // lower z half
                    z1l = fmaf(-Hz, wz, cc); z1h = fmaf(Hz, uz, cc);      // upper z half
                    zsl = zsh = 0.0f;
                } else {
                    const float Az = hz * fabsf(ri);
                    z0l = cc - Az; z0h = cc; z1l = cc; z1h = cc + Az; zsl = cc - Az; zsh = cc + Az;
                }
            } else {
                // the ray stays in the plane z = 0: it belongs to the half (block)
                // whose half-open z range [lo, hi) holds 0; 1/v_r = +inf, so the
                // first half is the lower one
                const float B = 1e30f;
                const bool lo = (cz - hz <= 0.0f) && (0.0f < cz), hi = (cz <= 0.0f) && (0.0f < cz + hz);
                const bool in = (cz - hz <= 0.0f) && (0.0f < cz + hz);
                z0l = lo ? -B : B; z0h = lo ? B : -B;
                z1l = hi ? -B : B; z1h = hi ? B : -B;
                zsl = in ? -B : B; zsh = in ? B : -B;
                zc = lo ? B : -B;      // the ray lies wholly in the first (lower) or second z half
            }
            const float* row = sino + ((size_t)v * g.R + rr) * g.B;
            const float* dl = g.dlen + (size_t)rr * g.B;
            float fk = 0.0f;
#pragma unroll 1
            for (int bb = blo; bb <= bhi; ++bb, fk += 1.0f) {
                const float dw = fmaf(fk, dstep, dw0);
                const float4 T = __ldg(drow + bb);
                const float a = dw * T.x, b = dw * T.y;
                const float q = __ldg(row + bb) * __ldg(dl + bb);
                if (MODE == kBp3Block) {
                    const float Ax = hx * fabsf(T.z), Ay = hy * fabsf(T.w);
                    const float ch = fmaxf(fminf(fminf(a + Ax, b + Ay), zsh) -
                                           fmaxf(fmaxf(a - Ax, b - Ay), zsl), 0.0f);
                    acc[0] = fmaf(q, ch, acc[0]);
                    if (WORK) evals += ch > 0.0f;
                } else if (MODE == kBp3Quad) {
                    // the split of the block within the slice's z slab from the
                    // clamped centre-line crossings, as in 2-D: [lo, hi] the ray's
                    // interval in block and slab, ca, cb its x and y centre-plane
                    // crossings clamped to it; first-minus-second half differences
                    // 2 ca - (lo + hi), 2 cb - (lo + hi), diagonal (hi - lo) - 2|ca - cb|
                    const float Ax = hx * fabsf(T.z), Ay = hy * fabsf(T.w);
                    const float lo = fmaxf(fmaxf(a - Ax, b - Ay), zsl);
                    const float hi = fmaxf(fminf(fminf(a + Ax, b + Ay), zsh), lo);
                    const float ca = fminf(fmaxf(a, lo), hi), cb = fminf(fmaxf(b, lo), hi);
                    const float sm = lo + hi;
                    if (WORK) {
                        const float xl[2] = {a - Ax, a}, xh[2] = {a, a + Ax};
                        const float yl[2] = {b - Ay, b}, yh[2] = {b, b + Ay};
#pragma unroll
                        for (int j = 0; j < 2; ++j)
#pragma unroll
                            for (int i = 0; i < 2; ++i)
                                evals += fminf(fminf(xh[i], yh[j]), zsh) - fmaxf(fmaxf(xl[i], yl[j]), zsl) > 0.0f;
                    }
                    acc[0] = fmaf(q, hi - lo, acc[0]);
                    // + on the lower halves: t = 1 x, 2 y, 3 xy; the signed sum of
                    // q phi and the sum of q |phi| (q >= 0), split after the loops
                    const float W[3] = {flipf(fmaf(2.0f, ca, -sm), T.z), flipf(fmaf(2.0f, cb, -sm), T.w),
                                        flipf(flipf(fmaf(-2.0f, fabsf(ca - cb), hi - lo), T.z), T.w)};
#pragma unroll
                    for (int t = 0; t < 3; ++t) {
                        acc[1 + 2 * t] = fmaf(q, W[t], acc[1 + 2 * t]);
                        acc[2 + 2 * t] = fmaf(q, fabsf(W[t]), acc[2 + 2 * t]);
                    }
                } else if (MODE == kBp3Octet) {
                    // voxel basis: chords of the 8 voxels in physical order (index
                    // x + 2 y + 4 z, 0 = lower half), select-free: the lower-x voxel
                    // spans [a - H(|1/Dx| + 1/Dx), a + H(|1/Dx| - 1/Dx)], H half its size
                    const float Hx = 0.5f * hx, Hy = 0.5f * hy;
                    const float ux = fabsf(T.z) + T.z, wx = fabsf(T.z) - T.z;
                    const float uy = fabsf(T.w) + T.w, wy = fabsf(T.w) - T.w;
                    const float xl[2] = {fmaf(-Hx, ux, a), fmaf(-Hx, wx, a)};
                    const float xh[2] = {fmaf(Hx, wx, a), fmaf(Hx, ux, a)};
                    const float yl[2] = {fmaf(-Hy, uy, b), fmaf(-Hy, wy, b)};
                    const float yh[2] = {fmaf(Hy, wy, b), fmaf(Hy, uy, b)};
                    const float zl[2] = {z0l, z1l}, zh[2] = {z0h, z1h};
#pragma unroll
                    for (int j = 0; j < 2; ++j)
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const float lo = fmaxf(xl[i], yl[j]), hi = fminf(xh[i], yh[j]);
#pragma unroll
                            for (int k = 0; k < 2; ++k) {
                                const float ch = fmaxf(fminf(hi, zh[k]) - fmaxf(lo, zl[k]), 0.0f);
                                acc[i + 2 * j + 4 * k] += q * ch;
                                if (WORK) evals += ch > 0.0f;
                            }
                        }
                } else {
                    // The 3-D Haar split without the eight octant chords: with [lo, hi]
                    // the ray's interval in the block and ca, cb, cc its x, y and z
                    // centre-plane crossings clamped to it, the ray is in the first
                    // half along an axis before that axis' crossing, so the products
                    // of the half signs (+1 first, -1 second) integrate to
                    // 2 c - (lo + hi) for one axis, (hi - lo) - 2 |ci - cj| for two
                    // (the stretch between the crossings has mixed signs), and for
                    // all three, whose product flips at each of the sorted crossings
                    // p1 <= p2 <= p3: 2 (p1 - p2 + p3) - (lo + hi), with
                    // p2 = ca + cb + cc - p1 - p3.  w[t]: bit 1 x, 2 y, 4 z.
                    const float Ax = hx * fabsf(T.z), Ay = hy * fabsf(T.w);
                    const float lo = fmaxf(fmaxf(a - Ax, b - Ay), zsl);
                    const float hi = fmaxf(fminf(fminf(a + Ax, b + Ay), zsh), lo);
                    const float ca = fminf(fmaxf(a, lo), hi), cb = fminf(fmaxf(b, lo), hi);
                    const float cc = fminf(fmaxf(zc, lo), hi);
                    const float A = hi - lo, sm = lo + hi;
                    const float p1 = fminf(fminf(ca, cb), cc), p3 = fmaxf(fmaxf(ca, cb), cc);
                    float w[8];
                    w[0] = A;
                    w[1] = fmaf(2.0f, ca, -sm);
                    w[2] = fmaf(2.0f, cb, -sm);
                    w[4] = fmaf(2.0f, cc, -sm);
                    w[3] = fmaf(-2.0f, fabsf(ca - cb), A);
                    w[5] = fmaf(-2.0f, fabsf(ca - cc), A);
                    w[6] = fmaf(-2.0f, fabsf(cb - cc), A);
                    w[7] = fmaf(4.0f, p1 + p3, -fmaf(2.0f, ca + cb + cc, sm));
                    if (WORK) {
                        const float xl[2] = {a - Ax, a}, xh[2] = {a, a + Ax};
                        const float yl[2] = {b - Ay, b}, yh[2] = {b, b + Ay};
                        const float zl[2] = {z0l, z1l}, zh[2] = {z0h, z1h};
#pragma unroll
                        for (int j = 0; j < 2; ++j)
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const float l2 = fmaxf(xl[i], yl[j]), h2 = fminf(xh[i], yh[j]);
#pragma unroll
                                for (int k = 0; k < 2; ++k) evals += fminf(h2, zh[k]) - fmaxf(l2, zl[k]) > 0.0f;
                            }
                    }
                    acc[0] = fmaf(q, w[0], acc[0]);
#pragma unroll
                    for (int t = 1; t < 8; ++t) {
                        float wt = w[t];
                        if (t & 1) wt = flipf(wt, T.z);
                        if (t & 2) wt = flipf(wt, T.w);
                        if (t & 4) wt = flipf(wt, ri);
                        // signed and absolute sums (q >= 0), split after the loops
                        acc[2 * t - 1] = fmaf(q, wt, acc[2 * t - 1]);
                        acc[2 * t] = fmaf(q, fabsf(wt), acc[2 * t]);
                    }
                }
            }
        }
    }
    if (MODE != kBp3Octet) {
        // the basis scale, and (signed sum s, absolute sum a) -> + part
        // (s + a) / 2 and - part (s - a) / 2, clamped to their signs
        acc[0] *= scale;
        if (MODE == kBp3Oct || MODE == kBp3Quad) {
            constexpr int nd = MODE == kBp3Oct ? 7 : 3;
#pragma unroll
            for (int t = 1; t <= nd; ++t) {
                const float sg = acc[2 * t - 1] * scale, ab = acc[2 * t] * scale;
                acc[2 * t - 1] = fmaxf(0.5f * (sg + ab), 0.0f);
                acc[2 * t] = fminf(0.5f * (sg - ab), 0.0f);
            }
        }
    }
}

template <bool WORK>
__device__ __forceinline__ void bp3_dispatch(const Geom3& g, const Segment3& S, int z3, int bx, int by, int bz,
                                             int chunk, int wv, const float* sino, float (&acc)[kSlots3],
                                             unsigned& evals)
{
    const bool det = S.has_details != 0;
    if (S.octet) bp3_item<kBp3Octet, WORK>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
    else if (det && z3) bp3_item<kBp3Oct, WORK>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
    else if (det) bp3_item<kBp3Quad, WORK>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
    else bp3_item<kBp3Block, WORK>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
}

__global__ void __launch_bounds__(kBackTPB)
k_backproject3(Geom3 g, SegTable3 tab, int z3, const float* __restrict__ sino, float* __restrict__ part,
               unsigned long long* __restrict__ work)
{
    __shared__ float red[kViewLanes][kSlots3][kItemsPerCta];
    const int cta = blockIdx.x;
    int si = 0;
    while (si + 1 < tab.n && cta >= tab.s[si + 1].cta_begin) ++si;
    const Segment3& S = tab.s[si];
    const int local = cta - S.cta_begin;
    const int chunk = local / S.tiles, tile = local - chunk * S.tiles;
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int item = tile * kItemsPerCta + lane;
    const bool oct = S.octet != 0, det = S.has_details != 0;
    float acc[kSlots3];
#pragma unroll
    for (int k = 0; k < kSlots3; ++k) acc[k] = 0.0f;
    unsigned evals = 0;
    if (item < S.n_items) {
        int bx, by, bz;
        decode3(S, item, bx, by, bz);
        if (work) bp3_dispatch<true>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
        else bp3_dispatch<false>(g, S, z3, bx, by, bz, chunk, wv, sino, acc, evals);
    }
    add_work3(work, evals);
#pragma unroll
    for (int k = 0; k < kSlots3; ++k) red[wv][k][lane] = acc[k];
    __syncthreads();
    for (int t = threadIdx.x; t < kSlots3 * kItemsPerCta; t += kBackTPB) {
        const int k = t / kItemsPerCta, l = t - k * kItemsPerCta;
        const int it = tile * kItemsPerCta + l;
        if (it >= S.n_items) continue;
        if (oct) {
            if (k >= 8) continue;
            // voxel k = cx + 2 cy + 4 cz
            float v = red[0][k][l];
#pragma unroll
            for (int w = 1; w < kViewLanes; ++w) v += red[w][k][l];
            part[S.part_off + ((size_t)chunk * S.n_slots + k) * S.n_items + it] = v;
        } else {
            const int ndet = z3 ? 7 : 3;
            int slot;
            if (k == 0) {
                if (!S.has_approx) continue;
                slot = 0;
            } else {
                if (!det || k > 2 * ndet) continue;
                slot = S.has_approx + (k - 1);
            }
            float sum = red[0][k][l];
#pragma unroll
            for (int w = 1; w < kViewLanes; ++w) sum += red[w][k][l];
            part[S.part_off + ((size_t)chunk * S.n_slots + slot) * S.n_items + it] = sum;
        }
    }
}

cudaError_t launch_backproject3(const Geom3& g, const SegTable3& tab, int z3, const float* sino, float* part,
                                unsigned long long* work, cudaStream_t st)
{
    if (tab.total_ctas == 0) return cudaSuccess;
    count_launch();
    k_backproject3<<<tab.total_ctas, kBackTPB, 0, st>>>(g, tab, z3, sino, part, work);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// coefficient indices
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long approx3(const Layout3& lay, int bx, int by, int bz)
{
    const int L = lay.L;
    if (lay.z3) return ((long long)bz * lay.gh[L] + by) * lay.gw[L] + bx;
    return (long long)bz * lay.nslice + (long long)by * lay.gw[L] + bx;
}

// detail t: z3: t = 1..7 (bit mask x 1, y 2, z 4); slices: t = 1 (x, "v"),
// 2 (y, "h"), 3 (xy, "d") stored in the 2-D plane order h, v, d
__device__ __forceinline__ long long detail3(const Layout3& lay, int l, int t, int bx, int by, int bz)
{
    if (lay.z3) {
        const long long n = (long long)lay.gw[l] * lay.gh[l] * lay.gd[l];
        return lay.coff[l] + (long long)(t - 1) * n + ((long long)bz * lay.gh[l] + by) * lay.gw[l] + bx;
    }
    const long long n = (long long)lay.gw[l] * lay.gh[l];
    const int plane = (t == 2) ? 0 : (t == 1 ? 1 : 2);
    return (long long)bz * lay.nslice + lay.coff[l] + plane * n + (long long)by * lay.gw[l] + bx;
}

__device__ __forceinline__ float sum_slot3(const Segment3& S, const float* __restrict__ part, int item, int slot)
{
    float s = 0.0f;
    const float* p = part + S.part_off + (size_t)slot * S.n_items + item;
    const size_t stride = (size_t)S.n_slots * S.n_items;
    for (int c = 0; c < S.n_chunks; ++c) s += p[c * stride];
    return s;
}

// the AM root of Eq. 1.9 in FP32 on b, bp, bm divided by the largest of
// |b|, bp, -bm (the root is a ratio; nothing overflows, no FP64 arithmetic)
__device__ __forceinline__ double am_delta32(double b, float bp, float bm, double z0, float iz0, double clamp)
{
    float bf = (float)b;
    const float sc = fmaxf(fmaxf(bp, -bm), fabsf(bf));
    float t = 0.0f;
    if (sc > 0.0f) {
        const float r = 1.0f / fmaxf(sc, 1e-30f);
        bf *= r;
        bp *= r;
        bm *= r;
        if (bp > 0.0f) {
            const float disc = sqrtf(bf * bf - 4.0f * bp * bm);
            const float u = (bf >= 0.0f) ? (bf + disc) / (2.0f * bp) : 2.0f * bm / (bf - disc);
            t = (u > 0.0f) ? -logf(u) : (float)clamp;
        } else if (bm < 0.0f) {
            t = (bf < 0.0f) ? -logf(bm / bf) : -(float)clamp;
        }
    }
    t = fminf(fmaxf(t, -(float)clamp), (float)clamp);
    return (double)(t * iz0);
}

// One thread per coefficient: thread 8 i + k of item i takes voxel k of an
// octet, or (k = 0) the approximation and (k = 1..7) detail type k of a block
// (types 1..3 only for the per-slice 2-D tree).
__global__ void k_update3(SegTable3 tab, Layout3 lay, const float* __restrict__ part, const double* __restrict__ bvec,
                          const double* __restrict__ z0p, double clamp, double* __restrict__ beta, int nonneg)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= 8LL * tab.total_items) return;
    const int it = (int)(gid >> 3), k = (int)(gid & 7);
    int si = 0;
    while (si + 1 < tab.n && it >= tab.s[si + 1].item_begin) ++si;
    const Segment3& S = tab.s[si];
    const int item = it - S.item_begin;
    int bx, by, bz;
    decode3(S, item, bx, by, bz);
    const double z0 = *z0p;
    const float iz0 = 1.0f / (float)z0;
    if (S.octet) {
        const long long z = ((long long)(2 * bz + (k >> 2)) * lay.ny + 2 * by + ((k >> 1) & 1)) * lay.nx +
                            2 * bx + (k & 1);
        const double nb = beta[z] + am_delta32(bvec[z], sum_slot3(S, part, item, k), 0.0f, z0, iz0, clamp);
        beta[z] = nonneg ? fmax(nb, 0.0) : nb;       // plain AM kept nonnegative: the step ends at 0
        return;
    }
    if (k == 0) {
        if (!S.has_approx) return;
        const long long z = approx3(lay, bx, by, bz);
        const double nb = beta[z] + am_delta32(bvec[z], sum_slot3(S, part, item, 0), 0.0f, z0, iz0, clamp);
        beta[z] = (nonneg && S.level == 0) ? fmax(nb, 0.0) : nb;
        return;
    }
    if (!S.has_details || k > (lay.z3 ? 7 : 3)) return;
    const int slot = (S.has_approx ? 1 : 0) + 2 * (k - 1);
    const long long z = detail3(lay, S.level, k, bx, by, bz);
    beta[z] += am_delta32(bvec[z], sum_slot3(S, part, item, slot), sum_slot3(S, part, item, slot + 1), z0, iz0,
                          clamp);
}

cudaError_t launch_update3(const SegTable3& tab, const Layout3& lay, const float* part, const double* b,
                           const double* z0, double clamp, double* beta, int nonneg, cudaStream_t st)
{
    if (tab.total_items == 0) return cudaSuccess;
    count_launch();
    k_update3<<<nb(8LL * tab.total_items, 256), 256, 0, st>>>(tab, lay, part, b, z0, clamp, beta, nonneg);
    return cudaGetLastError();
}

// voxel-basis back-projection (octet segment) into a volume
__global__ void k_reduce_voxels3(SegTable3 tab, Layout3 lay, const float* __restrict__ part, double* __restrict__ out,
                                 float* __restrict__ outf)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)lay.nx * lay.ny * lay.nz;
    if (p >= N) return;
    const Segment3& S = tab.s[0];
    const int ix = (int)(p % lay.nx);
    const long long r = p / lay.nx;
    const int iy = (int)(r % lay.ny), iz = (int)(r / lay.ny);
    const int item = ((iz >> 1) * S.gh + (iy >> 1)) * S.gw + (ix >> 1);
    const float v = sum_slot3(S, part, item, (ix & 1) + 2 * (iy & 1) + 4 * (iz & 1));
    if (out) out[p] = (double)v;
    if (outf) outf[p] = v;
}

cudaError_t launch_reduce_voxels3(const SegTable3& tab, const Layout3& lay, const float* part, double* out,
                                  float* outf, cudaStream_t st)
{
    const long long N = (long long)lay.nx * lay.ny * lay.nz;
    count_launch();
    k_reduce_voxels3<<<nb(N, 256), 256, 0, st>>>(tab, lay, part, out, outf);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a5: Z0 row sums over the tree (ancestor accumulators as in 2-D; octants for
// the 3-D Haar, quadrants of the ray's current slice for the slices mode)
// ---------------------------------------------------------------------------
constexpr int kMaxL3 = 5;

// c negated where bit li of `bits` is set (a sign-bit flip).
__device__ __forceinline__ float flip_bit3(float c, int bits, int li)
{
    return __int_as_float(__float_as_int(c) ^ ((bits << (31 - li)) & 0x80000000));
}

// Z3: the 3-D tree (seven signed detail sums per level); else the per-slice
// 2-D tree (three, as in 2-D)
template <bool Z3>
__global__ void __launch_bounds__(kFwdTPB)
k_z03(Geom3 g, Layout3 lay, const uint8_t* __restrict__ leaf, double* __restrict__ part)
{
    const int v = blockIdx.z, r = blockIdx.y;
    const int b = blockIdx.x * kFwdTPB + threadIdx.x;
    double rowsum = 0.0;
    if (b < g.B) {
        Ray3 ray;
        if (make_ray3(g, v, r, b, ray)) {
            const int L = lay.L, z3 = Z3 ? 1 : 0;
            // per level, the ray's signed detail sums of its current block: the
            // 3-D tree's seven (x, y, xy, z, xz, yz, xyz half-sign products) or
            // the slice's three (x, y, xy); they stay zero in blocks that are
            // not expanded
            constexpr int ND = Z3 ? 7 : 3;
            float acc[kMaxL3][ND];
#pragma unroll
            for (int l = 0; l < kMaxL3; ++l)
#pragma unroll
                for (int k = 0; k < ND; ++k) acc[l][k] = 0.0f;
            float total = 0.0f, rs = 0.0f;
            auto flush = [&](int li) {
                float sa = 0.0f;
#pragma unroll
                for (int t = 0; t < ND; ++t) sa += fabsf(acc[li][t]);
                rs += (float)basis_scale(z3, li + 1) * sa;
#pragma unroll
                for (int k = 0; k < ND; ++k) acc[li][k] = 0.0f;
            };
            // the previous leaf's voxel: the level-l block changes exactly when bit
            // l or a higher one of x or y (3-D tree: or z) changes, and in the
            // slices mode with any change of slice (the start flushes zero sums)
            int pix = -1, piy = -1, piz = -1;
            walk3(g, leaf, z3, ray, [&](int ix, int iy, int iz, int lam, int, int, int, float c) {
                total += c;
                const int mz = Z3 ? (iz ^ piz) : (iz != piz ? -1 : 0);
                const int hb = 31 - __clz((ix ^ pix) | (iy ^ piy) | mz);
                pix = ix;
                piy = iy;
                piz = iz;
#pragma unroll
                for (int li = 0; li < kMaxL3; ++li) {
                    const int l = li + 1;
                    if (l <= hb && l <= L) flush(li);
                    if (l > lam && l <= L) {
                        // the leaf's half along each axis in its level-l ancestor:
                        // bit l - 1 of the voxel (the leaf is aligned to 2^lam)
                        acc[li][0] += flip_bit3(c, ix, li);
                        acc[li][1] += flip_bit3(c, iy, li);
                        acc[li][2] += flip_bit3(c, ix ^ iy, li);
                        if (Z3) {
                            acc[li][3 % ND] += flip_bit3(c, iz, li);
                            acc[li][4 % ND] += flip_bit3(c, ix ^ iz, li);
                            acc[li][5 % ND] += flip_bit3(c, iy ^ iz, li);
                            acc[li][6 % ND] += flip_bit3(c, ix ^ iy ^ iz, li);
                        }
                    }
                }
            });
#pragma unroll
            for (int li = 0; li < kMaxL3; ++li)
                if (li + 1 <= L) flush(li);
            rowsum = (double)rs + (double)total * basis_scale(z3, L);
        }
    }
    rowsum = wmax(rowsum);
    if ((threadIdx.x & 31) == 0)
        part[(((size_t)v * g.R + r) * gridDim.x + blockIdx.x) * (kFwdTPB / 32) + (threadIdx.x >> 5)] = rowsum;
}

cudaError_t launch_z03(const Geom3& g, const Layout3& lay, const uint8_t* leaf, double* part, cudaStream_t st)
{
    if (lay.L > kMaxL3) return cudaErrorInvalidValue;
    count_launch();
    dim3 grid(nb(g.B, kFwdTPB), g.R, g.V);
    if (lay.z3) k_z03<true><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part);
    else k_z03<false><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// a1 synthesis, leaf map, a7 expansion, block lists, full analysis
// ---------------------------------------------------------------------------
__global__ void k_synth3(Layout3 lay, const uint8_t* __restrict__ leaf, const double* __restrict__ beta,
                         float* __restrict__ mu)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)lay.nx * lay.ny * lay.nz;
    if (p >= N) return;
    const int ix = (int)(p % lay.nx);
    const long long rr = p / lay.nx;
    const int iy = (int)(rr % lay.ny), iz = (int)(rr / lay.ny);
    const int L = lay.L;
    if (L == 0) {
        mu[p] = (float)beta[p];
        return;
    }
    const int lam = leaf ? (lay.z3 ? (int)leaf[p] : (int)leaf[(long long)iy * lay.nx + ix]) : 0;
    double v = beta[approx3(lay, ix >> L, iy >> L, lay.z3 ? iz >> L : iz)] * basis_scale(lay.z3, L);
    for (int l = L; l > lam; --l) {
        const int bx = ix >> l, by = iy >> l, bz = lay.z3 ? iz >> l : iz;
        const int cx = (ix >> (l - 1)) & 1, cy = (iy >> (l - 1)) & 1, cz = lay.z3 ? (iz >> (l - 1)) & 1 : 0;
        const int nt = lay.z3 ? 7 : 3;
        double s = 0.0;
        for (int t = 1; t <= nt; ++t) {
            const int par = ((t & 1) & cx) ^ (((t >> 1) & 1) & cy) ^ (((t >> 2) & 1) & cz);
            const double bz_ = beta[detail3(lay, l, t, bx, by, bz)];
            s += par ? -bz_ : bz_;
        }
        v += s * basis_scale(lay.z3, l);
    }
    mu[p] = (float)v;
}

cudaError_t launch_synth3(const Layout3& lay, const uint8_t* leaf, const double* beta, float* mu, cudaStream_t st)
{
    const long long N = (long long)lay.nx * lay.ny * lay.nz;
    count_launch();
    k_synth3<<<nb(N, 256), 256, 0, st>>>(lay, leaf, beta, mu);
    return cudaGetLastError();
}

__global__ void k_leafmap3(Layout3 lay, const uint8_t* __restrict__ mask, uint8_t* __restrict__ leaf)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = lay.z3 ? (long long)lay.nx * lay.ny * lay.nz : lay.nslice;
    if (p >= n) return;
    const int ix = (int)(p % lay.nx);
    const long long rr = p / lay.nx;
    const int iy = (int)(rr % lay.ny), iz = lay.z3 ? (int)(rr / lay.ny) : 0;
    int lam = lay.L;
    for (int l = lay.L; l >= 1; --l) {
        const long long m = lay.moff[l] + (((long long)(iz >> l)) * lay.gh[l] + (iy >> l)) * lay.gw[l] + (ix >> l);
        if (mask[m]) lam = l - 1;
        else break;
    }
    leaf[p] = (uint8_t)lam;
}

cudaError_t launch_leafmap3(const Layout3& lay, const uint8_t* mask, uint8_t* leaf, cudaStream_t st)
{
    const long long n = lay.z3 ? (long long)lay.nx * lay.ny * lay.nz : lay.nslice;
    count_launch();
    k_leafmap3<<<nb(n, 256), 256, 0, st>>>(lay, mask, leaf);
    return cudaGetLastError();
}

// S = sum over z of mu (slices mode), fixed order
__global__ void k_zsum(Layout3 lay, const float* __restrict__ mu, float* __restrict__ s2d)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= lay.nslice) return;
    float s = 0.0f;
    for (int z = 0; z < lay.nz; ++z) s += mu[(long long)z * lay.nslice + p];
    s2d[p] = s;
}

__global__ void k_max3(const float* __restrict__ S, long long n, double* __restrict__ part)
{
    double m = -INFINITY;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, (double)S[i]);
    __shared__ double sh[32];
    m = wmax(m);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = -INFINITY;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, sh[w]);
        part[blockIdx.x] = r;
    }
}

__global__ void k_thr3(const double* __restrict__ part, int n, double tau, double* __restrict__ thr)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double m = -INFINITY;
        for (int i = 0; i < n; ++i) m = fmax(m, part[i]);
        *thr = tau * m;
    }
}

__global__ void k_mark3(Layout3 lay, const float* __restrict__ S, const double* __restrict__ thr, int all,
                        const uint8_t* __restrict__ leaf_old, uint8_t* __restrict__ mask_new)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = lay.z3 ? (long long)lay.nx * lay.ny * lay.nz : lay.nslice;
    if (p >= n) return;
    const int lam = leaf_old[p];
    if (lam < 1) return;
    if (!all && !((double)S[p] > *thr)) return;
    const int ix = (int)(p % lay.nx);
    const long long rr = p / lay.nx;
    const int iy = (int)(rr % lay.ny), iz = lay.z3 ? (int)(rr / lay.ny) : 0;
    mask_new[lay.moff[lam] + (((long long)(iz >> lam)) * lay.gh[lam] + (iy >> lam)) * lay.gw[lam] + (ix >> lam)] = 1;
}

cudaError_t launch_expand3(const Layout3& lay, const float* mu, double tau, const uint8_t* leaf_old,
                           uint8_t* mask_new, float* s2d, double* scratch, cudaStream_t st)
{
    const float* S = mu;
    long long n = (long long)lay.nx * lay.ny * lay.nz;
    if (!lay.z3) {
        count_launch();
        k_zsum<<<nb(lay.nslice, 256), 256, 0, st>>>(lay, mu, s2d);
        S = s2d;
        n = lay.nslice;
    }
    const int parts = 256;
    count_launch();
    k_max3<<<parts, 256, 0, st>>>(S, n, scratch);
    count_launch();
    k_thr3<<<1, 32, 0, st>>>(scratch, parts, tau, scratch + parts);
    count_launch();
    k_mark3<<<nb(n, 256), 256, 0, st>>>(lay, S, scratch + parts, tau < 0.0 ? 1 : 0, leaf_old, mask_new);
    return cudaGetLastError();
}

// Block lists in Morton order: list 0 level-L blocks not expanded, list 1
// level-L expanded, list 1 + k expanded blocks of level L - k.  Entries
// (bx | by << 10 | bz << 20); in the slices mode the lists hold 2-D blocks
// (bz = 0) and the host code repeats them over the slices.
__device__ __forceinline__ uint32_t part1by2(uint32_t x, int sh)
{
    uint32_t r = 0;
    for (int i = 0; i < 10; ++i) r |= ((x >> (3 * i + sh)) & 1u) << i;
    return r;
}

__global__ void __launch_bounds__(1024) k_compact3(Layout3 lay, const uint8_t* __restrict__ mask,
                                                   uint32_t* __restrict__ lists, long long stride,
                                                   int* __restrict__ counts)
{
    const int list = blockIdx.x;
    const int level = list <= 1 ? lay.L : lay.L - (list - 1);
    const int want = list == 0 ? 0 : 1;
    const int gw = lay.gw[level], gh = lay.gh[level], gd = lay.z3 ? lay.gd[level] : 1;
    int side = 1;
    while (side < gw || side < gh || side < gd) side <<= 1;
    const long long ncode = lay.z3 ? (long long)side * side * side : (long long)side * side;
    uint32_t* out = lists + stride * list;
    __shared__ int wc[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long long m0 = 0; m0 < ncode; m0 += blockDim.x) {
        const long long m = m0 + threadIdx.x;
        bool keep = false;
        int bx = 0, by = 0, bz = 0;
        if (m < ncode) {
            if (lay.z3) {
                bx = (int)part1by2((uint32_t)m, 0);
                by = (int)part1by2((uint32_t)m, 1);
                bz = (int)part1by2((uint32_t)m, 2);
            } else {
                uint32_t x = (uint32_t)m, y = (uint32_t)(m >> 1);
                uint32_t rx = 0, ry = 0;
                for (int i = 0; i < 16; ++i) {
                    rx |= ((x >> (2 * i)) & 1u) << i;
                    ry |= ((y >> (2 * i)) & 1u) << i;
                }
                bx = (int)rx;
                by = (int)ry;
            }
            if (bx < gw && by < gh && bz < gd) {
                const int e = mask[lay.moff[level] + ((long long)bz * gh + by) * gw + bx] ? 1 : 0;
                keep = (e == want);
            }
        }
        const unsigned bal = __ballot_sync(0xffffffffu, keep);
        if (lane == 0) wc[wid] = __popc(bal);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            if (w < wid) off += wc[w];
            tot += wc[w];
        }
        if (keep)
            out[base + off + __popc(bal & ((1u << lane) - 1u))] =
                (uint32_t)bx | ((uint32_t)by << 10) | ((uint32_t)bz << 20);
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) counts[list] = base;
}

cudaError_t launch_compact3(const Layout3& lay, const uint8_t* mask, uint32_t* lists, long long stride, int* counts,
                            cudaStream_t st)
{
    count_launch();
    k_compact3<<<lay.L + 1, 1024, 0, st>>>(lay, mask, lists, stride, counts);
    return cudaGetLastError();
}

// analysis of one level: z3 from the (nz>>(l-1), ...) approximation volume,
// slices from per-slice (ny>>(l-1), nx>>(l-1)) images stacked in z
__global__ void k_haar3_level(Layout3 lay, int l, const double* __restrict__ a, double* __restrict__ a_next,
                              double* __restrict__ coef)
{
    const int gw = lay.gw[l], gh = lay.gh[l], gd = lay.z3 ? lay.gd[l] : lay.nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)gw * gh * gd) return;
    const int bx = (int)(i % gw);
    const long long r = i / gw;
    const int by = (int)(r % gh), bz = (int)(r / gh);
    const int w = 2 * gw, h = 2 * gh;
    if (lay.z3) {
        double c[8];
        for (int k = 0; k < 8; ++k)
            c[k] = a[(((long long)(2 * bz + (k >> 2))) * h + 2 * by + ((k >> 1) & 1)) * w + 2 * bx + (k & 1)];
        const double s = 1.0 / (2.0 * sqrt(2.0));
        const long long n = (long long)gw * gh * gd;
        for (int t = 0; t < 8; ++t) {
            double acc = 0.0;
            for (int k = 0; k < 8; ++k) acc += (__popc(t & k) & 1) ? -c[k] : c[k];
            if (t == 0) a_next[i] = acc * s;
            else coef[lay.coff[l] + (long long)(t - 1) * n + i] = acc * s;
        }
    } else {
        const long long base = (long long)bz * h * w;
        const double ll = a[base + (2 * by) * w + 2 * bx], lh = a[base + (2 * by) * w + 2 * bx + 1];
        const double hl = a[base + (2 * by + 1) * w + 2 * bx], hh = a[base + (2 * by + 1) * w + 2 * bx + 1];
        const long long n = (long long)gw * gh;
        const long long j = (long long)by * gw + bx;
        a_next[(long long)bz * n + j] = 0.5 * (ll + lh + hl + hh);
        double* cs = coef + (long long)bz * lay.nslice + lay.coff[l];
        cs[j] = 0.5 * (ll + lh - hl - hh);
        cs[n + j] = 0.5 * (ll - lh + hl - hh);
        cs[2 * n + j] = 0.5 * (ll - lh - hl + hh);
    }
}

// copy the level-L approximations into the coefficient vector
__global__ void k_haar3_approx(Layout3 lay, const double* __restrict__ a, double* __restrict__ coef)
{
    const int L = lay.L;
    const long long nA = (long long)lay.gw[L] * lay.gh[L];
    const long long n = lay.z3 ? nA * lay.gd[L] : nA * lay.nz;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (lay.z3) coef[i] = a[i];
    else coef[(i / nA) * lay.nslice + (i % nA)] = a[i];
}

cudaError_t launch_haar3(const Layout3& lay, const double* img, double* coef, double* ta, double* tb,
                         cudaStream_t st)
{
    const long long N = (long long)lay.nx * lay.ny * lay.nz;
    if (lay.L == 0) return cudaMemcpyAsync(coef, img, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    const double* a = img;
    double* bufs[2] = {ta, tb};
    for (int l = 1; l <= lay.L; ++l) {
        double* an = bufs[l & 1];
        const long long n = (long long)lay.gw[l] * lay.gh[l] * (lay.z3 ? lay.gd[l] : lay.nz);
        count_launch();
        k_haar3_level<<<nb(n, 256), 256, 0, st>>>(lay, l, a, an, coef);
        a = an;
    }
    const long long nA = (long long)lay.gw[lay.L] * lay.gh[lay.L] * (lay.z3 ? lay.gd[lay.L] : lay.nz);
    count_launch();
    k_haar3_approx<<<nb(nA, 256), 256, 0, st>>>(lay, a, coef);
    return cudaGetLastError();
}

}  // namespace wam
