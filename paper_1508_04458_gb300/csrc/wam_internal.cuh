// Internal device/host declarations of libwam (not part of the C-ABI).
//
// Geometry, tree layout and the two exact-intersection primitives shared by
// the kernels:
//   * ray traversal over the leaf blocks of the wavelet tree (ray-driven
//     projector and Z0), and
//   * closed-form chords of one ray through a block and its four children
//     (voxel-driven back-projectors).
// Both evaluate h(y|x) = length of ray y inside voxel x (Sec. II) and its
// block sums, which by Eq. 1.2 give phi(y|z) = sum_x h(y|x) omega(x|z).
#pragma once
#include <type_traits>

#include <cuda_runtime.h>
#include <stdint.h>

namespace wam {

constexpr int kMaxLevels = 8;
constexpr int kMaxSegs = 2 * kMaxLevels + 4;
constexpr int kItemsPerCta = 32;  // back-projector: items (blocks) per CTA, one per lane
constexpr int kViewLanes = 8;     // back-projector: warps per CTA, each on its own views
constexpr int kBackTPB = kItemsPerCta * kViewLanes;
constexpr int kFwdTPB = 128;      // threads per CTA of the ray-driven kernels
constexpr int kMaxBags = 128;     // bags of one persistent batched iteration

// Scan geometry in the kernel's precision T.  X0, Y0: lower-left image corner.
template <typename T>
struct Geom {
    int kind, nx, ny, V, B;
    int stage_rows;               // staged forward: strips per shared-memory stage (16, 24, 32), 0: none
    T vx, vy, X0, Y0, ivx, ivy;
    T pitch, ucen, sod, sdd;
    const T* cs;                  // device [V][2]: cos, sin of each view angle
};

// Tree / coefficient layout for L levels (see wam.h).
struct Layout {
    int L, nx, ny;
    int gw[kMaxLevels + 1], gh[kMaxLevels + 1];     // block grid per level
    long long coff[kMaxLevels + 1];                 // first detail plane of level l
    long long moff[kMaxLevels + 1];                 // mask offset of level l
    long long mask_bytes;
};

// One homogeneous group of back-projection items (blocks of one level and
// one kind), split into `n_chunks` view ranges of `vpc` views each.
struct Segment {
    int level;          // 0: pixel basis (Omega = I); 1..L: Haar level
    int has_approx;     // accumulates the (unsigned) approximation slot
    int has_details;    // accumulates h+, h-, v+, v-, d+, d-
    int quad;           // pixel basis, item = 2x2 pixels: slots = the four pixel sums
    int n_items;
    const uint32_t* items;   // packed (by << 16) | bx, or null: implicit row-major
    int gw;             // block-grid width for implicit items
    int n_chunks, vpc;
    int tiles;
    int cta_begin;      // first CTA of this segment in the back-projection grid
    int item_begin;     // first thread of this segment in the update grid
    int n_slots;
    long long part_off; // first partial of this segment
};

struct SegTable {
    int n;
    int total_ctas;
    int total_items;
    Segment s[kMaxSegs];
};

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename T> __device__ __forceinline__ T tiny_dir();
template <> __device__ __forceinline__ float tiny_dir<float>() { return 1e-30f; }
template <> __device__ __forceinline__ double tiny_dir<double>() { return 1e-200; }

// Finite reciprocal of a direction component: |d| is clamped to a tiny value
// (sign kept, +0 for a zero) so that plane-crossing parameters stay finite.
template <typename T>
__device__ __forceinline__ T safe_rcp(T d)
{
    T a = fabs(d);
    a = a < tiny_dir<T>() ? tiny_dir<T>() : a;
    T r = T(1) / a;
    return signbit(d) ? -r : r;
}

template <typename T> __device__ __forceinline__ T rsqrt_t(T x);
template <> __device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

// ---------------------------------------------------------------------------
// one ray in parametric form P(t) = P0 + t * dir, |dir| = 1, P0 the point of
// the ray closest to the origin; [tin, tout] is its part inside the image.
// ---------------------------------------------------------------------------
template <typename T>
struct Ray {
    T px, py, dx, dy, idx, idy, tin, tout;
};

template <typename T>
__device__ __forceinline__ bool make_ray(const Geom<T>& g, int v, int b, Ray<T>& r)
{
    const T c = g.cs[2 * v], s = g.cs[2 * v + 1];
    const T ub = (T(b) - g.ucen) * g.pitch;
    T tlo, thi;
    if (g.kind == 0) {
        // line through ub*u, u = (-s, c), direction e = (c, s)
        r.dx = c; r.dy = s;
        r.px = -ub * s; r.py = ub * c;
        tlo = T(-1e30); thi = T(1e30);
    } else {
        // source SOD e, detector point -(SDD-SOD) e + ub u
        const T n2 = g.sdd * g.sdd + ub * ub;
        const T rn = rsqrt_t<T>(n2);
        r.dx = (-g.sdd * c - ub * s) * rn;
        r.dy = (-g.sdd * s + ub * c) * rn;
        const T k = g.sod * ub / n2;               // P0 = k (ub e + SDD u)
        r.px = k * (ub * c - g.sdd * s);
        r.py = k * (ub * s + g.sdd * c);
        tlo = -g.sod * g.sdd * rn;                 // the source
        thi = tlo + n2 * rn;                       // the detector
    }
    r.idx = safe_rcp(r.dx);
    r.idy = safe_rcp(r.dy);
    const T X1 = g.X0 + T(g.nx) * g.vx, Y1 = g.Y0 + T(g.ny) * g.vy;
    T a0 = (g.X0 - r.px) * r.idx, a1 = (X1 - r.px) * r.idx;
    T b0 = (g.Y0 - r.py) * r.idy, b1 = (Y1 - r.py) * r.idy;
    r.tin = fmax(tlo, fmax(fmin(a0, a1), fmin(b0, b1)));
    r.tout = fmin(thi, fmin(fmax(a0, a1), fmax(b0, b1)));
    return r.tout > r.tin;
}

// Visit the leaf blocks crossed by the ray, in order.  leaf[iy*nx+ix] is the
// level of the leaf holding pixel (ix, iy) (null: every pixel is a leaf).
// visit(ix, iy, lam, bx0, by0, chord): (ix, iy) the pixel where the ray
// enters the leaf, (bx0, by0) the leaf's first pixel, chord its length (mm).
// Every step crosses one grid line in the travel direction, so nx + ny + 4
// steps bound the walk.
template <typename T, typename F>
__device__ __forceinline__ void traverse(const Geom<T>& g, const uint8_t* __restrict__ leaf,
                                         const Ray<T>& r, F&& visit)
{
    T t = r.tin;
    int ix = clampi((int)floor((r.px + t * r.dx - g.X0) * g.ivx), 0, g.nx - 1);
    int iy = clampi((int)floor((r.py + t * r.dy - g.Y0) * g.ivy), 0, g.ny - 1);
    const bool xpos = r.idx > T(0), ypos = r.idy > T(0);
    const int max_steps = g.nx + g.ny + 4;
    for (int step = 0; step < max_steps; ++step) {
        const int lam = leaf ? (int)leaf[iy * g.nx + ix] : 0;
        const int bs = 1 << lam;
        const int bx0 = (ix >> lam) << lam, by0 = (iy >> lam) << lam;
        const int xe = xpos ? bx0 + bs : bx0;
        const int ye = ypos ? by0 + bs : by0;
        const T tx = (g.X0 + T(xe) * g.vx - r.px) * r.idx;
        const T ty = (g.Y0 + T(ye) * g.vy - r.py) * r.idy;
        T te = fmin(fmin(tx, ty), r.tout);
        te = fmax(te, t);
        visit(ix, iy, lam, bx0, by0, te - t);
        t = te;
        if (te >= r.tout) break;
        if (tx <= ty) {
            ix = xpos ? bx0 + bs : bx0 - 1;
            iy = clampi((int)floor((r.py + te * r.dy - g.Y0) * g.ivy), by0, by0 + bs - 1);
        } else {
            iy = ypos ? by0 + bs : by0 - 1;
            ix = clampi((int)floor((r.px + te * r.dx - g.X0) * g.ivx), bx0, bx0 + bs - 1);
        }
        if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny) break;
    }
}

// Incremental Siddon walk over single pixels (every pixel a leaf).  The next
// crossing of each axis is recomputed from the first one and an integer count
// (t = t_first + k * t_per_pixel), so rounding does not accumulate along the
// ray.  visit(ix, iy, chord).
template <typename T, typename F>
__device__ __forceinline__ void traverse_pixels(const Geom<T>& g, const Ray<T>& r, F&& visit)
{
    T t = r.tin;
    int ix = clampi((int)floor((r.px + t * r.dx - g.X0) * g.ivx), 0, g.nx - 1);
    int iy = clampi((int)floor((r.py + t * r.dy - g.Y0) * g.ivy), 0, g.ny - 1);
    const bool xpos = r.idx > T(0), ypos = r.idy > T(0);
    const int sx = xpos ? 1 : -1, sy = ypos ? 1 : -1;
    const T ax = fabs(r.idx) * g.vx, ay = fabs(r.idy) * g.vy;
    const T tx0 = (g.X0 + T(ix + (xpos ? 1 : 0)) * g.vx - r.px) * r.idx;
    const T ty0 = (g.Y0 + T(iy + (ypos ? 1 : 0)) * g.vy - r.py) * r.idy;
    T tx = tx0, ty = ty0;
    T kx = T(0), ky = T(0);     // crossing counts, exact in T
    const int max_steps = g.nx + g.ny + 4;
    for (int step = 0; step < max_steps; ++step) {
        T te = fmin(fmin(tx, ty), r.tout);
        te = fmax(te, t);
        visit(ix, iy, te - t);
        t = te;
        if (te >= r.tout) break;
        if (tx <= ty) {
            ix += sx;
            kx += T(1);
            tx = tx0 + kx * ax;
        } else {
            iy += sy;
            ky += T(1);
            ty = ty0 + ky * ay;
        }
        if ((unsigned)ix >= (unsigned)g.nx || (unsigned)iy >= (unsigned)g.ny) break;
    }
}

// Exact pixel walk by strips.  The ray's major axis is the one whose grid
// lines it crosses most often per unit length (|d|/v larger), so within one
// pixel strip across that axis it crosses at most one line of the other
// axis: a strip holds one or two pixels.  Strips are visited in increasing
// major coordinate, the two pixels of a strip in the same order.
//
// The minor coordinate is tracked in pixel units oriented along the ray's
// minor travel and counted from the edge of the entry pixel c0
// (u = +-(n - N0 - c0 v_minor) / v_minor), so the next grid line is an
// integer ahead; the walk carries e = u - (that line) at the end of each
// strip, which grows by the constant D per full strip and drops by one at a
// crossing (e >= 0); the piece beyond a crossing is e v_minor / |d_minor| (no
// division in the loop).  Counting from c0 keeps u small for rays near an
// axis, whose crossing points are the most sensitive to rounding in u.  The
// two partial end strips are peeled (e from the entry and exit points);
// interior strips have the constant chord v_major / |d_major|.
//
// Pixels are addressed in an image with a one-pixel zero apron on every side,
// (nm + 2) strips of sM = pad_row(nn): lin = (j + 1) sM + (c + 1).  A step
// across the image's minor edge (possible only in the exit strip, where the
// ray leaves through that edge) lands on the apron and reads 0, so the walk
// needs no range test; the apron also keeps any index the walk can form
// inside the allocation.  visit(la, ca, lb, cb) once per strip: first pixel
// and chord, second pixel and chord (cb = 0, lb = la for a one-pixel strip).
// Row length of an apron-padded copy with n cells per row: n + 2 rounded up
// to a multiple of 4 elements, so that every row starts on a 16-byte
// boundary (the tensor-memory-access copies of the staged forward need it).
// The elements past n + 2 are never read by a walk.
__host__ __device__ __forceinline__ int pad_row(int n) { return (n + 2 + 3) & ~3; }

template <typename T>
__device__ __forceinline__ bool strip_major_y(const Geom<T>& g, const Ray<T>& r)
{
    return fabs(r.dy) * g.ivy >= fabs(r.dx) * g.ivx;
}

template <typename T, typename F>
__device__ __forceinline__ void traverse_strips(const Geom<T>& g, const Ray<T>& r, bool ymaj, F&& visit)
{
    const T pm = ymaj ? r.py : r.px, pn = ymaj ? r.px : r.py;
    const T dm = ymaj ? r.dy : r.dx, dn = ymaj ? r.dx : r.dy;
    const T vm = ymaj ? g.vy : g.vx, vn = ymaj ? g.vx : g.vy;
    const T ivm = ymaj ? g.ivy : g.ivx, ivn = ymaj ? g.ivx : g.ivy;
    const T M0 = ymaj ? g.Y0 : g.X0, N0 = ymaj ? g.X0 : g.Y0;
    const int nm = ymaj ? g.ny : g.nx, nn = ymaj ? g.nx : g.ny;
    const T sec = fabs(ymaj ? r.idy : r.idx);          // length per unit of major coordinate
    const T vk = vn * fabs(ymaj ? r.idx : r.idy);      // length per minor pixel unit
    const T slope = dn * (ymaj ? r.idy : r.idx);       // dn / dm
    const T s_in = pm + r.tin * dm, s_out = pm + r.tout * dm;
    const T s_lo = fmin(s_in, s_out), s_hi = fmax(s_in, s_out);
    const T n0 = pn - pm * slope;                      // minor coordinate at major 0
    const bool up = slope >= T(0);
    const int j0 = clampi((int)floor((s_lo - M0) * ivm), 0, nm - 1);
    const int j1 = clampi((int)floor((s_hi - M0) * ivm), 0, nm - 1);
    const int c0 = clampi((int)floor((fma(s_lo, slope, n0) - N0) * ivn), 0, nn - 1);
    const T Nc = fma(T(c0), vn, N0);                   // lower edge of the entry pixel
    const T G = fabs(slope) * ivn;                     // oriented minor units per unit major
    const T U0 = (up ? n0 - Nc : Nc - n0) * ivn;       // u at major 0
    const int sM = pad_row(nn), dlin = up ? 1 : -1;
    const T fbo0 = up ? T(1) : T(0);                   // the first minor grid line ahead, oriented
    int lin = (j0 + 1) * sM + c0 + 1;
    // One strip: e = u - (the next oriented minor grid line) at the strip's
    // end; a crossing (e >= 0) puts the last e * vk of the chord in the next
    // cell.  Returns e for the next line (one line further on a crossing).
    // (In a full strip the piece past a crossing, e vk with 0 <= e < D, is
    // below the chord D vk, so only the partial end strips clamp it.)
    auto strip = [&](T chord, T e, auto clamp) {
        const bool cross = e >= T(0);
        const T cb = cross ? (decltype(clamp)::value ? fmin(e * vk, chord) : e * vk) : T(0);
        const int lb = cross ? lin + dlin : lin;
        visit(lin, chord - cb, lb, cb);
        lin = lb + sM;
        return cross ? e - T(1) : e;
    };
    using Clamp = std::true_type;
    using NoClamp = std::false_type;
    if (j1 == j0) {
        strip((s_hi - s_lo) * sec, fma(s_hi, G, U0) - fbo0, Clamp());
        return;
    }
    const T A = fma(G, M0, U0), D = G * vm;            // u at the end of strip j: A + (j + 1) D
    T E = strip(fmax(fma(T(j0 + 1), vm, M0) - s_lo, T(0)) * sec, fma(T(j0 + 1), D, A) - fbo0, Clamp());
    const T full = vm * sec;
#pragma unroll 4
    for (int k = j1 - j0 - 1; k > 0; --k) E = strip(full, E + D, NoClamp());
    // the last strip ends at the exit point, u - A - j1 D past the end of strip j1 - 1
    strip(fmax(s_hi - fma(T(j1), vm, M0), T(0)) * sec, E + (fma(s_hi, G, U0) - fma(T(j1), D, A)), Clamp());
}

// ---------------------------------------------------------------------------
// closed-form chords through an axis-aligned block
// ---------------------------------------------------------------------------
// Chords in crossing order.  Measured along the unit
// direction from a point of the ray, the ray crosses the block's centre lines
// x = cx at t = a and y = cy at t = b, and its faces at a -+ Ax (x) and
// b -+ Ay (y), Ax = hx |1/dx|, Ay = hy |1/dy|, always in this order.  The
// half it crosses first along x is "F", the other "S" (likewise along y), so
// the four child chords need no sorting:
//   cFF = [max(a - Ax, b - Ay), min(a, b)]        (first x half, first y half)
//   cFS = [max(a - Ax, b), min(a, b + Ay)]
//   cSF = [max(a, b - Ay), min(a + Ax, b)]
//   cSS = [max(a, b), min(a + Ax, b + Ay)]
// (interval lengths, clamped at 0).  The first half along x is the lower one
// when 1/dx > 0, the upper one otherwise (likewise y).
template <typename T>
__device__ __forceinline__ T block_chord_ab(T a, T b, T Ax, T Ay)
{
    return fmax(fmin(a + Ax, b + Ay) - fmax(a - Ax, b - Ay), T(0));
}

// Chords of a ray through the four children of a block in physical order
// (l/h: lower/upper half along x, then y).  a, b: the ray parameters where it
// crosses the block's centre lines x = cx, y = cy; ix = 1/dx, iy = 1/dy
// (signed); Hx, Hy: half the block's half-sizes.  The child on the lower-x
// side spans the parameters between the lines x = cx - 2 Hx and x = cx, i.e.
// [a - Hx (|ix| + ix), a + Hx (|ix| - ix)] whatever the sign of dx, so no
// selects are needed.
template <typename T>
__device__ __forceinline__ void child_chords_phys(T a, T b, T Hx, T Hy, T ix, T iy, T& cll, T& chl, T& clh,
                                                  T& chh)
{
    const T ux = fabs(ix) + ix, wx = fabs(ix) - ix, uy = fabs(iy) + iy, wy = fabs(iy) - iy;
    const T xl0 = fma(-Hx, ux, a), xl1 = fma(Hx, wx, a), xh0 = fma(-Hx, wx, a), xh1 = fma(Hx, ux, a);
    const T yl0 = fma(-Hy, uy, b), yl1 = fma(Hy, wy, b), yh0 = fma(-Hy, wy, b), yh1 = fma(Hy, uy, b);
    cll = fmax(fmin(xl1, yl1) - fmax(xl0, yl0), T(0));
    chl = fmax(fmin(xh1, yl1) - fmax(xh0, yl0), T(0));
    clh = fmax(fmin(xl1, yh1) - fmax(xl0, yh0), T(0));
    chh = fmax(fmin(xh1, yh1) - fmax(xh0, yh0), T(0));
}

// The same for a ray taken with dx >= 0 (ix = 1/dx >= 0): the lower-x child
// spans [a - 2 Hx ix, a] and the upper one [a, a + 2 Hx ix].
template <typename T>
__device__ __forceinline__ void child_chords_phys_xpos(T a, T b, T Hx, T Hy, T ix, T iy, T& cll, T& chl, T& clh,
                                                       T& chh)
{
    const T uy = fabs(iy) + iy, wy = fabs(iy) - iy;
    const T xl0 = fma(-2 * Hx, ix, a), xh1 = fma(2 * Hx, ix, a);
    const T yl0 = fma(-Hy, uy, b), yl1 = fma(Hy, wy, b), yh0 = fma(-Hy, wy, b), yh1 = fma(Hy, uy, b);
    cll = fmax(fmin(a, yl1) - fmax(xl0, yl0), T(0));
    chl = fmax(fmin(xh1, yl1) - fmax(a, yl0), T(0));
    clh = fmax(fmin(a, yh1) - fmax(xl0, yh0), T(0));
    chh = fmax(fmin(xh1, yh1) - fmax(a, yh0), T(0));
}

// The Haar split of a ray through a block without its four child chords:
// with [lo, hi] the ray's parameter interval inside the block (a, b, Ax, Ay
// as in child_chords_ab) and ca, cb the centre-line crossings clamped to it,
// the chord is A = hi - lo, the first x half minus the second is
// 2 ca - (lo + hi), likewise in y with cb, and the diagonal difference
// (FF + SS) - (FS + SF) is A - 2 |ca - cb| (the part between the two
// crossings lies in the mixed children).  A miss gives hi = lo: all zero.
template <typename T>
__device__ __forceinline__ void haar_split(T a, T b, T Ax, T Ay, T& A, T& dx, T& dy, T& dg)
{
    const T lo = fmax(a - Ax, b - Ay);
    const T hi = fmax(fmin(a + Ax, b + Ay), lo);
    const T ca = fmin(fmax(a, lo), hi), cb = fmin(fmax(b, lo), hi);
    const T s = lo + hi;
    A = hi - lo;
    dx = fma(T(2), ca, -s);
    dy = fma(T(2), cb, -s);
    dg = fma(T(-2), fabs(ca - cb), A);
}

template <typename T>
__device__ __forceinline__ void child_chords_ab(T a, T b, T Ax, T Ay, T& cFF, T& cFS, T& cSF, T& cSS)
{
    const T a0 = a - Ax, a2 = a + Ax, b0 = b - Ay, b2 = b + Ay;
    cFF = fmax(fmin(a, b) - fmax(a0, b0), T(0));
    cFS = fmax(fmin(a, b2) - fmax(a0, b), T(0));
    cSF = fmax(fmin(a2, b) - fmax(a, b0), T(0));
    cSS = fmax(fmin(a2, b2) - fmax(a, b), T(0));
}

}  // namespace wam
