// CUDA kernels of libwam (sm_103a).  Each kernel is one step of the
// multiresolution AM iteration (Algorithm 1 and the Results section's tree
// growth).  All reductions run in a fixed order: results are deterministic.
#include "wam_internal.cuh"
#include "wam_kernels.h"

#include <cuda.h>
#include <math.h>

#include <atomic>
#include <mutex>
#include <type_traits>

namespace wam {

// ---------------------------------------------------------------------------
// deterministic block reductions
// ---------------------------------------------------------------------------

template <typename V, typename Op>
__device__ __forceinline__ V warp_reduce(V x, Op op)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = op(x, __shfl_down_sync(0xffffffffu, x, o));
    return x;
}

// Reduce over the CTA; the result is valid in thread 0.  Fixed tree order.
template <typename V, typename Op>
__device__ __forceinline__ V block_reduce(V x, Op op, V identity)
{
    __shared__ V sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    x = warp_reduce(x, op);
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    const int nw = (blockDim.x + 31) >> 5;
    x = (threadIdx.x < nw) ? sh[threadIdx.x] : identity;
    if (wid == 0) x = warp_reduce(x, op);
    __syncthreads();
    return x;
}

// Warp-aggregated add of a per-thread count into a 64-bit device counter.
__device__ __forceinline__ void add_work(unsigned long long* work, unsigned cnt)
{
    if (!work) return;
    const unsigned m = __activemask();
    const unsigned tot = __reduce_add_sync(m, cnt);
    if ((threadIdx.x & 31) == (unsigned)(__ffs(m) - 1)) atomicAdd(work, (unsigned long long)tot);
}

// 2^-l exactly (l = 0..1022), built from its exponent bits
__device__ __forceinline__ double pow2m(int l) { return __hiloint2double((1023 - l) << 20, 0); }

struct OpSum {
    template <typename V> __device__ V operator()(V a, V b) const { return a + b; }
};
struct OpMax {
    template <typename V> __device__ V operator()(V a, V b) const { return a > b ? a : b; }
};

// ---------------------------------------------------------------------------
// a2 + a3: ray-driven forward projection over the tree's leaves, fused with
// Beer's law and the I-divergence terms (Sec. II and its footnote).
// One thread per ray; CTA = (bin tile, view).
// ---------------------------------------------------------------------------
// The two apron-padded copies the pixel walk reads, on the grid of cells of
// 2^lam x 2^lam pixels (mu constant on each cell; lam = 0: the pixels):
// py = the cell values with a zero border ((ny + 2) rows of nx + 2 used
// elements at the stride pad_row(nx); nx, ny counted in cells), px = its
// transpose with a zero border ((nx + 2) rows of ny + 2 at the stride
// pad_row(ny)).  A cell's value is read at its first pixel; nxf is mu's row
// length.  One thread per padded cell (x, y) in [-1, nx] x [-1, ny]; both
// writes coalesced through a 32x32 shared tile.
template <typename T>
__global__ void k_pad2(const T* __restrict__ mu, int nxf, int lam, int nx, int ny, T* __restrict__ py,
                       T* __restrict__ px)
{
    __shared__ T tile[32][33];
    const int x0 = (int)blockIdx.x * 32 - 1, y0 = (int)blockIdx.y * 32 - 1;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int x = x0 + threadIdx.x, y = y0 + k;
        T v = T(0);
        if (x >= 0 && x < nx && y >= 0 && y < ny) v = mu[((size_t)y << lam) * nxf + ((size_t)x << lam)];
        tile[k][threadIdx.x] = v;
        if (x <= nx && y <= ny) py[(size_t)(y + 1) * pad_row(nx) + (x + 1)] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int y = y0 + threadIdx.x, x = x0 + k;
        if (x <= nx && y <= ny) px[(size_t)(x + 1) * pad_row(ny) + (y + 1)] = tile[threadIdx.x][k];
    }
}

// Per-ray I-divergence term dterm + d p + q of the cost.  FP64: as written.
// FP32: the three addends are of order d |log(d/I0)| while their sum is of
// order one, so they are added in float-float (the exact product d p by an
// FMA, exact sums by Knuth's two-sum) and only the sum is rounded to float;
// the warp sums of these terms are then FP32 and the CTA's in FP64.
template <typename T> struct CostAccT { using type = double; };
template <> struct CostAccT<float> { using type = float; };
template <typename T> using CostAcc = typename CostAccT<T>::type;

__device__ __forceinline__ double cost_term(double dt, float d, double p, double q)
{
    return dt + (double)d * p + q;
}

// s + e = a + b exactly (round-to-nearest, no contraction)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ float cost_term(float2 dt, float d, float p, float q)
{
    const float ph = __fmul_rn(d, p);
    const float pl = __fmaf_rn(d, p, -ph);      // d p = ph + pl exactly
    float s1, e1, s2, e2;
    two_sum(dt.x, ph, s1, e1);
    two_sum(s1, q, s2, e2);
    return __fadd_rn(s2, __fadd_rn(__fadd_rn(dt.y, pl), __fadd_rn(e1, e2)));
}

// The epilogue of a ray's projection p = acc: p (optional), qhat = I0 e^-p,
// the residual d - qhat (optional), and the ray's cost term.
template <typename T>
__device__ __forceinline__ CostAcc<T> forward_ray_out(const Geom<T>& g, int v, int b, T acc, const float* __restrict__ d,
                                                      const typename CostTerm<T>::type* __restrict__ dterm,
                                                      const float* __restrict__ I0, T* __restrict__ qhat,
                                                      T* __restrict__ p_out, T* __restrict__ resid)
{
    CostAcc<T> term = 0;
    const size_t y = (size_t)v * g.B + b;
    if (p_out) p_out[y] = acc;
    if (qhat || resid) {
        const T q = T(I0[y]) * exp(-acc);
        if (qhat) qhat[y] = q;
        if (resid) resid[y] = T(d[y]) - q;   // dI/dp = d - q
        // d log(d/q) - d + q = [d (log d - log I0) - d] + d p + q
        term = cost_term(dterm[y], d[y], acc, q);
    }
    return term;
}

// One cost partial per CTA: warp sums, then the warps in a fixed order (a
// CTA's slot frees only when its last warp ends, so the barrier costs no
// occupancy).  Every thread of the CTA must call it.
template <typename V>
__device__ __forceinline__ void forward_cost_partial(V term, double* __restrict__ cost_part, int slot)
{
    if (!cost_part) return;
    __shared__ V wsum[kFwdTPB / 32];
    term = warp_reduce(term, OpSum());
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = wsum[0];
#pragma unroll
        for (int w = 1; w < kFwdTPB / 32; ++w) t += wsum[w];
        cost_part[slot] = t;
    }
}

// The rays of bin tile `tile` of view v (one per thread), their cost terms
// summed into cost_part[slot].  Every thread of the CTA must call it.
template <typename T, bool PIX, bool WORK>
__device__ __forceinline__ void forward_body(const Geom<T>& g, const T* __restrict__ mu, const T* __restrict__ pad,
                                             const uint8_t* __restrict__ leaf, const float* __restrict__ d,
                                             const typename CostTerm<T>::type* __restrict__ dterm,
                                             const float* __restrict__ I0, T* __restrict__ qhat,
                                             T* __restrict__ p_out, T* __restrict__ resid,
                                             double* __restrict__ cost_part, unsigned long long* __restrict__ work,
                                             int v, int tile, int slot)
{
    const int b = tile * kFwdTPB + threadIdx.x;
    CostAcc<T> term = 0;
    unsigned steps = 0;
    if (b < g.B) {
        Ray<T> r;
        T acc = T(0);
        if (make_ray(g, v, b, r)) {
            if (PIX) {
                // y-major rays walk rows of the padded mu, x-major rays rows
                // of the padded transpose.  Loads run one strip ahead of their
                // use; the sum keeps the walk's order.
                const bool ymaj = strip_major_y(g, r);
                const T* img = ymaj ? pad : pad + (size_t)pad_row(g.nx) * (g.ny + 2);
                T pca = T(0), pva = T(0), pcb = T(0), pvb = T(0);
                traverse_strips(g, r, ymaj, [&](int la, T ca, int lb, T cb) {
                    const T va = __ldg(img + la), vb = __ldg(img + lb);
                    acc += pca * pva;
                    acc += pcb * pvb;
                    pca = ca; pva = va;
                    pcb = cb; pvb = vb;
                    if (WORK) steps += (ca > T(0)) + (cb > T(0));
                });
                acc += pca * pva;
                acc += pcb * pvb;
            } else {
                traverse(g, leaf, r, [&](int ix, int iy, int, int, int, T c) {
                    acc += c * __ldg(mu + iy * g.nx + ix);
                    if (WORK) ++steps;
                });
            }
        }
        term = forward_ray_out(g, v, b, acc, d, dterm, I0, qhat, p_out, resid);
    }
    if (WORK) add_work(work, steps);
    forward_cost_partial(term, cost_part, slot);
}

// Sixteen CTAs per SM (at most 32 registers): a full SM of warps to cover
// the image-row loads that miss L1.
template <typename T, bool PIX, bool WORK>
__global__ void __launch_bounds__(kFwdTPB, 16)
k_forward(Geom<T> g, const T* __restrict__ mu, const T* __restrict__ pad, const uint8_t* __restrict__ leaf,
          const float* __restrict__ d, const typename CostTerm<T>::type* __restrict__ dterm,
          const float* __restrict__ I0, T* __restrict__ qhat, T* __restrict__ p_out,
          T* __restrict__ resid, double* __restrict__ cost_part, unsigned long long* __restrict__ work)
{
    forward_body<T, PIX, WORK>(g, mu, pad, leaf, d, dterm, I0, qhat, p_out, resid, cost_part, work, blockIdx.y,
                               blockIdx.x, blockIdx.y * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------------------
// a2 + a3 with the image band staged in shared memory by the tensor memory
// accelerator.  The 128 rays of a CTA (consecutive bins of one view) come
// from one source (or are parallel), so they never cross inside the image:
// at every strip of the walk their cells lie between those of the CTA's
// first and last ray.  When all the CTA's rays share the walk's major axis,
// the CTA copies its band kStageRows strips at a time (a window of
// kStageCols cells, double buffered, one cp.async.bulk.tensor per stage on an
// mbarrier) and every ray walks its strips of that stage from shared memory.
// The walk, its chords and the order of its sums are those of
// traverse_strips, so the result equals the unstaged kernel's bit for bit.
// A ray's partial first and last strips are read from global memory, its
// interior strips stage by stage; a ray whose columns in a stage would leave
// the window reads that stage from global memory instead; CTAs with mixed
// major axes, or bands wider than the window, walk global memory throughout.
// Staging removes the long-scoreboard stalls of the unstaged walk (L1 misses
// on the image rows) but adds per-stage bookkeeping and holds 21-41 KB of
// shared memory per CTA; on the 512 x 512 scan the two come out about even,
// on scans whose bands overflow the window it is slower, so it is a tuning
// choice per geometry (off by default).
// ---------------------------------------------------------------------------
constexpr int kStageCols = 160;               // 640 B: a multiple of 16 B
constexpr int kMaxStrips = 1536;              // bands of up to 1536 strips are staged
constexpr long long kWaitCycles = 1LL << 31;  // ~1 s at 2 GHz: a copy that takes longer is an error

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with this parity to complete, for at most kWaitCycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > kWaitCycles) return false;
    return true;
}

// 2-D tile (x = column, y = row, in elements) of the tensor into shared memory.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_addr(dst)), "l"(reinterpret_cast<uint64_t>(tm)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// kStageRows strips per stage: a tile shape the autotuner chooses per geometry.
template <int kStageRows, bool WORK>
__global__ void __launch_bounds__(kFwdTPB, 10)
k_forward_staged(Geom<float> g, const float* __restrict__ pad, const __grid_constant__ CUtensorMap tmy,
                 const __grid_constant__ CUtensorMap tmx, const float* __restrict__ d,
                 const float2* __restrict__ dterm, const float* __restrict__ I0, float* __restrict__ qhat,
                 float* __restrict__ p_out, float* __restrict__ resid, double* __restrict__ cost_part,
                 unsigned long long* __restrict__ work, int* __restrict__ err)
{
    constexpr int kMaxStages = (kMaxStrips + kStageRows - 1) / kStageRows;
    __shared__ __align__(128) float buf[2][kStageRows * kStageCols];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ int s_x0[kMaxStages];
    __shared__ int s_jlo, s_jhi, s_staged;
    __shared__ float s_line[2][2];            // (n0, slope) of the CTA's first and last ray

    const int v = blockIdx.y;
    const int b = blockIdx.x * kFwdTPB + threadIdx.x;
    const int bl = min(b, g.B - 1);           // rays past the last bin still give the band's edge
    Ray<float> r;
    const bool inside = make_ray(g, v, bl, r);
    const bool hit = inside && b < g.B;
    const bool ymaj = strip_major_y(g, r);
    const int allY = __syncthreads_and(!hit || ymaj);
    const int allX = __syncthreads_and(!hit || !ymaj);
    const bool Y = allY ? true : (allX ? false : ymaj);
    const bool uniform = allY || allX;

    // the walk of traverse_strips, in the frame of the major axis
    const float pm = Y ? r.py : r.px, pn = Y ? r.px : r.py;
    const float dm = Y ? r.dy : r.dx, dn = Y ? r.dx : r.dy;
    const float vm = Y ? g.vy : g.vx, vn = Y ? g.vx : g.vy;
    const float ivm = Y ? g.ivy : g.ivx, ivn = Y ? g.ivx : g.ivy;
    const float M0 = Y ? g.Y0 : g.X0, N0 = Y ? g.X0 : g.Y0;
    const int nm = Y ? g.ny : g.nx, nn = Y ? g.nx : g.ny;
    const float sec = fabsf(Y ? r.idy : r.idx);
    const float vk = vn * fabsf(Y ? r.idx : r.idy);
    const float slope = dn * (Y ? r.idy : r.idx);
    const float s_in = pm + r.tin * dm, s_out = pm + r.tout * dm;
    const float s_lo = fminf(s_in, s_out), s_hi = fmaxf(s_in, s_out);
    const float n0 = pn - pm * slope;
    const bool up = slope >= 0.0f;
    const int j0 = clampi((int)floorf((s_lo - M0) * ivm), 0, nm - 1);
    const int j1 = clampi((int)floorf((s_hi - M0) * ivm), 0, nm - 1);
    const int c0 = clampi((int)floorf((fmaf(s_lo, slope, n0) - N0) * ivn), 0, nn - 1);
    const float Nc = fmaf((float)c0, vn, N0);
    const float G = fabsf(slope) * ivn;
    const float U0 = (up ? n0 - Nc : Nc - n0) * ivn;
    const int sM = pad_row(nn), dlin = up ? 1 : -1;
    const float A = fmaf(G, M0, U0), D = G * vm;
    const float full = vm * sec;
    const float* img = Y ? pad : pad + (size_t)pad_row(g.nx) * (g.ny + 2);

    if (threadIdx.x == 0) {
        s_jlo = 1 << 30;
        s_jhi = -1;
        s_staged = uniform ? 1 : 0;
    }
    if (threadIdx.x == 0 || b == g.B - 1 || threadIdx.x == kFwdTPB - 1) {
        // the band's edges: the CTA's first ray and its last ray within the scan
        const int k = threadIdx.x == 0 ? 0 : 1;
        if (k == 0 || b == g.B - 1 || (threadIdx.x == kFwdTPB - 1 && b < g.B)) {
            s_line[k][0] = n0;
            s_line[k][1] = slope;
        }
    }
    __syncthreads();
    if (hit) {
        atomicMin(&s_jlo, j0);
        atomicMax(&s_jhi, j1);
    }
    __syncthreads();
    const int Jlo = s_jlo, Jhi = s_jhi;
    const int nst = Jhi >= Jlo ? (Jhi - Jlo) / kStageRows + 1 : 0;
    if (threadIdx.x < 32 && s_staged) {
        // each stage's window: the cells of the two edge rays over its strips, 2 cells of margin
        bool ok = nst <= kMaxStages;
        for (int st = threadIdx.x; ok && st < nst; st += 32) {
            const int ja = Jlo + st * kStageRows, jb = min(Jhi, ja + kStageRows - 1);
            const float Ma = fmaf((float)ja, vm, M0), Mb = fmaf((float)(jb + 1), vm, M0);
            float lo = 3e38f, hi = -3e38f;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float na = fmaf(Ma, s_line[k][1], s_line[k][0]), nb = fmaf(Mb, s_line[k][1], s_line[k][0]);
                lo = fminf(lo, fminf(na, nb));
                hi = fmaxf(hi, fmaxf(na, nb));
            }
            const float clo = fmaxf((lo - N0) * ivn, -8.0f), chi = fminf((hi - N0) * ivn, (float)nn + 8.0f);
            const int x0 = ((int)floorf(clo) + 1 - 2) & ~3;              // padded column, 16-byte aligned
            const int x1 = (int)floorf(chi) + 1 + 2;
            if (x1 - x0 >= kStageCols) ok = false;
            else s_x0[st] = x0;
        }
        if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) s_staged = 0;
    }
    if (threadIdx.x == 0 && s_staged && nst > 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const CUtensorMap* tm = Y ? &tmy : &tmx;
        for (int st = 0; st < min(2, nst); ++st) {
            mbar_expect_tx(&bar[st], kStageRows * kStageCols * sizeof(float));
            tma_load_2d(buf[st], tm, s_x0[st], Jlo + st * kStageRows + 1, &bar[st]);
        }
    }
    __syncthreads();
    const bool staged = s_staged != 0;

    float acc = 0.0f;
    unsigned steps = 0;
    // walk state: the padded column colp of the next strip's first cell, and
    // E = u - (the next oriented minor grid line) after the last strip walked
    // (traverse_strips' running form: the same values, the same sums)
    int colp = c0 + 1;
    const float fbo0 = up ? 1.0f : 0.0f;
    float E = 0.0f;
    auto strip = [&](const float* base, int rs, int& p, float chord, float e, auto clamp) {
        const bool cross = e >= 0.0f;
        const float cb = cross ? (decltype(clamp)::value ? fminf(e * vk, chord) : e * vk) : 0.0f;
        const int pb = cross ? p + dlin : p;
        const float ca = chord - cb;
        acc += ca * base[p];
        acc += cb * base[pb];
        if (WORK) steps += (ca > 0.0f) + (cb > 0.0f);
        E = cross ? e - 1.0f : e;
        p = pb + rs;
    };
    // interior strips ja..jb (full chords) from base (row stride rs), p the
    // index of strip ja's first cell; returns the index one row past jb
    auto interior = [&](const float* base, int rs, int p, int ja, int jb) {
#pragma unroll 4
        for (int jj = ja; jj <= jb; ++jj) strip(base, rs, p, full, E + D, std::false_type());
        return p;
    };
    // the partial first strip (the whole walk when it is one strip), from global memory
    if (hit) {
        int p = (j0 + 1) * sM + colp;
        if (j0 == j1) strip(img, sM, p, (s_hi - s_lo) * sec, fmaf(s_hi, G, U0) - fbo0, std::true_type());
        else strip(img, sM, p, fmaxf(fmaf((float)(j0 + 1), vm, M0) - s_lo, 0.0f) * sec,
                   fmaf((float)(j0 + 1), D, A) - fbo0, std::true_type());
        colp = p - (j0 + 2) * sM;
    }
    const int i0 = j0 + 1, i1 = j1 - 1;          // the interior strips
    if (!staged) {
        if (hit && i0 <= i1) {
            const int pe = interior(img, sM, (i0 + 1) * sM + colp, i0, i1);
            colp = pe - (i1 + 2) * sM;
        }
    } else {
        const CUtensorMap* tm = Y ? &tmy : &tmx;
        int failed = -1;                      // the stage whose copy timed out
        for (int st = 0; st < nst; ++st) {
            const int bi = st & 1;
            const int ra = Jlo + st * kStageRows, rb = min(Jhi, ra + kStageRows - 1);
            const bool timed_out = !mbar_wait_bounded(&bar[bi], (st >> 1) & 1);
            const int ja = max(i0, ra), jb = min(i1, rb);
            if (hit && ja <= jb && !timed_out) {
                // the columns this ray reaches in the stage: its column now and
                // after the crossings up to strip jb (at most one per strip)
                // (E + (jb + 1 - ja) D rounded down, plus one, up to one off by
                // rounding: inside the window's two-cell margin)
                const int ncross = max(0, (int)floorf(fmaf((float)(jb + 1 - ja), D, E)) + 1);
                const int cend = colp + dlin * ncross;
                const int x0 = s_x0[st];
                if (min(colp, cend) - 2 >= x0 && max(colp, cend) + 2 < x0 + kStageCols) {
                    const int pe = interior(buf[bi], kStageCols, (ja - ra) * kStageCols + (colp - x0), ja, jb);
                    colp = pe - (jb + 1 - ra) * kStageCols + x0;
                } else {
                    const int pe = interior(img, sM, (ja + 1) * sM + colp, ja, jb);
                    colp = pe - (jb + 2) * sM;
                }
            }
            // the stage's barrier, and a vote that every thread takes alike
            if (__syncthreads_or(timed_out)) {
                failed = st;
                break;
            }
            if (threadIdx.x == 0 && st + 2 < nst) {
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_expect_tx(&bar[bi], kStageRows * kStageCols * sizeof(float));
                tma_load_2d(buf[bi], tm, s_x0[st + 2], Jlo + (st + 2) * kStageRows + 1, &bar[bi]);
            }
        }
        if (failed >= 0 && threadIdx.x == 0) {
            // record the failure; wait (bounded) for this CTA's copies still in
            // flight, stages `failed` and failed + 1, before the CTA ends
            atomicOr(err, 1);
            for (int st = failed; st < min(nst, failed + 2); ++st) mbar_wait_bounded(&bar[st & 1], (st >> 1) & 1);
        }
    }
    // the partial last strip, from global memory
    if (hit && j1 > j0) {
        int p = (j1 + 1) * sM + colp;
        strip(img, sM, p, fmaxf(s_hi - fmaf((float)j1, vm, M0), 0.0f) * sec,
              E + (fmaf(s_hi, G, U0) - fmaf((float)j1, D, A)), std::true_type());
    }
    CostAcc<float> term = 0;
    if (b < g.B) term = forward_ray_out(g, v, b, inside ? acc : 0.0f, d, dterm, I0, qhat, p_out, resid);
    if (WORK) add_work(work, steps);
    forward_cost_partial(term, cost_part, blockIdx.y * gridDim.x + blockIdx.x);
}

// Sum n partials in a fixed order (one CTA of 256 threads).
__global__ void k_sum_final(const double* __restrict__ part, int n, double* __restrict__ out)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_reduce(s, OpSum(), 0.0);
    if (threadIdx.x == 0) *out = s;
}

// Same, written to out[*counter], then the counter advances (graph replays).
// CTAs of 1024 threads (the order of the sum depends on it).
__device__ __forceinline__ void sum_at_body(const double* __restrict__ part, int n, double* __restrict__ out,
                                            int* __restrict__ counter)
{
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_reduce(s, OpSum(), 0.0);
    if (threadIdx.x == 0) {
        out[*counter] = s;
        *counter += 1;
    }
}

__global__ void k_sum_at(const double* __restrict__ part, int n, double* __restrict__ out, int* __restrict__ counter)
{
    sum_at_body(part, n, out, counter);
}

__global__ void k_max_final(const double* __restrict__ part, int n, double* __restrict__ out)
{
    double s = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s = fmax(s, part[i]);
    s = block_reduce<double>(s, OpMax(), -INFINITY);
    if (threadIdx.x == 0) *out = s;
}

// c negated where bit li of `bits` is set (a sign-bit flip in FP32).
__device__ __forceinline__ float flip_bit(float c, int bits, int li)
{
    return __int_as_float(__float_as_int(c) ^ ((bits << (31 - li)) & 0x80000000));
}
__device__ __forceinline__ double flip_bit(double c, int bits, int li) { return ((bits >> li) & 1) ? -c : c; }

// ---------------------------------------------------------------------------
// a5, Eq. 1.61: per ray sum over active z of |phi(y|z)|, then max over rays.
// The ray walks the leaves; each leaf's chord is added, with the Haar signs of
// the quadrant it lies in, to the three detail sums of every expanded ancestor
// block.  A convex block is crossed in one contiguous run of leaves, so a
// block's |phi| terms are final when the ray's pixel leaves it.
// ---------------------------------------------------------------------------
template <typename T, int LM>
__global__ void __launch_bounds__(kFwdTPB)
k_z0(Geom<T> g, Layout lay, const uint8_t* __restrict__ leaf, double* __restrict__ part)
{
    // LM = the tree's level count (0..kMaxLevels): the per-level loops unroll
    // exactly, with compile-time bounds
    const int v = blockIdx.y;
    const int b = blockIdx.x * kFwdTPB + threadIdx.x;
    double rowsum = 0.0;
    if (b < g.B) {
        Ray<T> r;
        if (make_ray(g, v, b, r)) {
            // per level, the ray's three Haar detail sums of its current block
            // (lower minus upper half, left minus right, diagonal); they stay
            // zero in blocks that are not expanded
            T hs[LM > 0 ? LM : 1], vs[LM > 0 ? LM : 1], ds[LM > 0 ? LM : 1];
#pragma unroll
            for (int l = 0; l < LM; ++l) hs[l] = vs[l] = ds[l] = T(0);
            T total = T(0), rs = T(0);
            const int L = LM;
            auto flush = [&](int li) {
                const T s = T(1) / T(1 << (li + 1));
                rs += s * (fabs(hs[li]) + fabs(vs[li]) + fabs(ds[li]));
                hs[li] = vs[li] = ds[li] = T(0);
            };
            // the previous leaf's pixel: the level-l block changes between two
            // leaves exactly when bit l or a higher one of x or y changes, i.e.
            // for every l up to the highest changed bit (the start flushes the
            // zero sums of every level)
            int pix = -1, piy = -1;
            traverse(g, leaf, r, [&](int ix, int iy, int lam, int, int, T c) {
                total += c;
                const int hb = 31 - __clz((ix ^ pix) | (iy ^ piy));
                pix = ix;
                piy = iy;
#pragma unroll
                for (int li = 0; li < LM; ++li) {
                    const int l = li + 1;
                    if (l <= hb) flush(li);
                    if (l > lam) {
                        // the leaf's quadrant in its level-l ancestor: bit l - 1 of
                        // the pixel (the leaf is aligned to 2^lam, lam < l)
                        hs[li] += flip_bit(c, iy, li);
                        vs[li] += flip_bit(c, ix, li);
                        ds[li] += flip_bit(c, ix ^ iy, li);
                    }
                }
            });
#pragma unroll
            for (int li = 0; li < LM; ++li) flush(li);
            rowsum = (double)rs + (double)total * pow2m(L);
        }
    }
    rowsum = warp_reduce(rowsum, OpMax());
    if ((threadIdx.x & 31) == 0)
        part[(blockIdx.y * gridDim.x + blockIdx.x) * (kFwdTPB / 32) + (threadIdx.x >> 5)] = rowsum;
}

// ---------------------------------------------------------------------------
// a4 (Eq. 1.10) and H^T: voxel-driven split back-projection.
// CTA = 32 consecutive items (blocks of one level, Morton order) x 8 warps;
// lane i of every warp holds item i, warp w takes views v0 + w, v0 + w + 8,
// ... of the CTA's view range.  For each view the block's shadow on the
// detector is found from its corners; for each ray in it the Haar split
// (haar_split: the block chord and the three half differences, from the
// centre-line crossings clamped to the ray's interval in the block) gives phi
// for the approximation (all +) and the three details, and the signed sum of
// qhat*phi and the sum of qhat*|phi| are accumulated; after the view loop they
// become the + and - parts of Eq. 1.10.  The 8 warps' sums are added in a fixed
// order in shared memory and one partial per (item, view range) is written;
// partials are summed in a fixed order by the consumer.  dirtab (optional)
// holds per ray the reciprocal unit direction (1/dx, ry/dy) and its products
// with the view's sin and -cos.
// ---------------------------------------------------------------------------
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_16a; };

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }
__device__ __forceinline__ double4_16a ld4(const double4_16a* p)
{
    const double2 lo = __ldg(reinterpret_cast<const double2*>(p));
    const double2 hi = __ldg(reinterpret_cast<const double2*>(p) + 1);
    double4_16a r;
    r.x = lo.x;
    r.y = lo.y;
    r.z = hi.x;
    r.w = hi.y;
    return r;
}

__device__ __forceinline__ float2 ld2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ double2 ld2(const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); }

__device__ __forceinline__ float fast_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double fast_div(double a, double b) { return a / b; }

// x with the sign flipped where `sgn` is negative (one logic op in FP32).
__device__ __forceinline__ float flip(float x, float sgn)
{
    return __int_as_float(__float_as_int(x) ^ (__float_as_int(sgn) & 0x80000000));
}
__device__ __forceinline__ double flip(double x, double sgn) { return signbit(sgn) ? -x : x; }
__device__ __forceinline__ float flip2(float x, float s1, float s2)
{
    return __int_as_float(__float_as_int(x) ^ ((__float_as_int(s1) ^ __float_as_int(s2)) & 0x80000000));
}
__device__ __forceinline__ double flip2(double x, double s1, double s2)
{
    return (signbit(s1) != signbit(s2)) ? -x : x;
}

// dirtab[v][b] = (s/dx, -c/dy, 1/dx, ry/dy) of ray (v, b), c, s = cos, sin of
// the view, ry = vy / vx, the ray oriented so that dx >= 0: with delta the
// ray's offset from a block centre along u, the centre-line crossings are
// a = delta s/dx and b = -delta c/dy.
// Item kinds of a back-projection segment.
enum { kBpBlock = 0, kBpSplit = 1, kBpQuad = 2 };

// The view and bin loops of one item (block bx, by of segment S) over the
// views of its chunk taken by this warp, specialised by item kind, by the
// direction table's presence and by work counting, so that the inner loop
// carries no run-time switch.  acc: A, h+, h-, v+, v-, d+, d- of the Haar
// split; a pixel quad keeps its four pixel sums in the first four.
template <typename T, int MODE, bool TABLE, bool WORK>
__device__ __forceinline__ void bp_item(const Geom<T>& g, const Segment& S, int bx, int by, int chunk, int wv,
                                        const T* __restrict__ sino,
                                        const typename Vec4<T>::type* __restrict__ dirtab, T (&acc)[7],
                                        unsigned& evals)
{
    const int bsz = 1 << S.level;
    const T hx = T(0.5) * T(bsz) * g.vx, hy = T(0.5) * T(bsz) * g.vy;
    const T cx = g.X0 + (T(2 * bx + 1)) * hx, cy = g.Y0 + (T(2 * by + 1)) * hy;
    // The ray parameters are measured in units of hx: the block spans
    // [a - 1/dx, a + 1/dx] along x and [b - ry/|dy|, b + ry/|dy|] along y
    // (ry = vy / vx, folded into the table's fourth entry), so no per-bin
    // scaling; the sums are multiplied by hx once after the loops.
    const T ihx = T(1) / hx, ry = g.vy * g.ivx;
    // the block's centre and the source distance in the same units (the
    // shadow's corners are ratios, the same in any unit)
    const T cxn = cx * ihx, cyn = cy * ihx, sodn = g.sod * ihx;
    const int v0 = chunk * S.vpc;
    const int v1 = min(g.V, v0 + S.vpc);
    const bool fan = g.kind != 0;
    const T isdd = T(1) / g.sdd, ipitch = T(1) / g.pitch;
    const T u0 = -g.ucen * g.pitch;
    // detector coordinate -> bin: u * ku + ucen (fan: u = sdd w / (sod - a),
    // a ratio; parallel: u = w, here in units of hx)
    const T ku = fan ? g.sdd * ipitch : hx * ipitch;
    for (int v = v0 + wv; v < v1; v += kViewLanes) {
        const auto csv = ld2(g.cs + 2 * v);
        const T c = csv.x, s = csv.y;
        const T ac = cxn * c + cyn * s;      // block centre along e (units of hx)
        const T wc = -cxn * s + cyn * c;     // ... along u
        // shadow of the block from its four corners (+-1, +-ry): along u the
        // corners sit at wc +- (ry c - s) and wc +- (s + ry c), along e at
        // ac +- (c + ry s) and ac +- (c - ry s) respectively
        const T w1 = fma(ry, c, -s), e1 = fma(ry, s, c);
        const T w2 = fma(ry, c, s), e2 = fma(-ry, s, c);
        T umin, umax;
        const T D = sodn - ac;
        if (fan) {
            const T r0 = fast_div(wc - w1, D + e1), r1 = fast_div(wc + w1, D - e1);
            const T r2 = fast_div(wc - w2, D - e2), r3 = fast_div(wc + w2, D + e2);
            umin = fmin(fmin(r0, r1), fmin(r2, r3));
            umax = fmax(fmax(r0, r1), fmax(r2, r3));
        } else {
            const T e = fmax(fabs(w1), fabs(w2));
            umin = wc - e;
            umax = wc + e;
        }
        // the rays through the shadow (umin, umax); a margin of 1e-3 bin
        // covers the fast division's rounding (~1e-4 bin at the detector edge)
        const int blo = max(0, (int)ceil(fma(umin, ku, g.ucen - T(1e-3))));
        const int bhi = min(g.B - 1, (int)floor(fma(umax, ku, g.ucen + T(1e-3))));
        // kappa: detector length per unit of hx at the block's depth
        const T kappa = fan ? D * isdd : ihx;
        // ray offset from the block centre along u (in units of hx), linear in the bin
        T delta = fma(T(blo) * g.pitch + u0, kappa, -wc);
        const T dstep = g.pitch * kappa;
        const T* row = sino + (size_t)v * g.B;
        const typename Vec4<T>::type* drow = TABLE ? dirtab + (size_t)v * g.B : nullptr;
#pragma unroll 1
        for (int bb = blo; bb <= bhi; ++bb, delta += dstep) {
            typename Vec4<T>::type dd;
            if (TABLE) {
                dd = ld4(drow + bb);
            } else {
                // no table: the same four numbers from the ray's direction,
                // oriented so that dx >= 0 like the table's
                const T ub = T(bb) * g.pitch + u0;
                T dx = c, dy = s;
                if (fan) {
                    const T rn = rsqrt_t<T>(g.sdd * g.sdd + ub * ub);
                    dx = (-g.sdd * c - ub * s) * rn;
                    dy = (-g.sdd * s + ub * c) * rn;
                }
                if (signbit(dx)) {
                    dx = -dx;
                    dy = -dy;
                }
                const T iy = safe_rcp(dy);
                dd.z = safe_rcp(dx);
                dd.w = iy * ry;
                dd.x = s * dd.z;
                dd.y = -c * iy;
            }
            const T a = delta * dd.x, b = delta * dd.y;
            const T q = __ldg(row + bb);
            if (MODE == kBpQuad) {
                // pixel basis: the four pixels' chords in physical order, select-free:
                // pixel (ylo,xlo), (ylo,xhi), (yhi,xlo), (yhi,xhi) sums
                T cll, chl, clh, chh;
                child_chords_phys_xpos(a, b, T(0.5), T(0.5), dd.z, dd.w, cll, chl, clh, chh);
                acc[0] += q * cll;
                acc[1] += q * chl;
                acc[2] += q * clh;
                acc[3] += q * chh;
                if (WORK) evals += (cll > T(0)) + (chl > T(0)) + (clh > T(0)) + (chh > T(0));
            } else if (MODE == kBpSplit) {
                // Haar split: the block chord and the three first-minus-second
                // half differences along the travel direction (haar_split).
                // The travel has dx >= 0, so its first x half is the lower one;
                // along y the first half is the lower one when 1/dy > 0
                T A, dx, dy, dg;
                haar_split(a, b, dd.z, fabs(dd.w), A, dx, dy, dg);
                const T qy = flip(q, dd.w);        // q with the sign that orders the y halves
                acc[0] = fma(q, A, acc[0]);
                // lower half minus upper half: the signed sum of q phi and the
                // sum of q |phi| (q >= 0), turned into the + and - parts below
                acc[1] = fma(qy, dy, acc[1]);
                acc[2] = fma(q, fabs(dy), acc[2]);
                acc[3] = fma(q, dx, acc[3]);
                acc[4] = fma(q, fabs(dx), acc[4]);
                acc[5] = fma(qy, dg, acc[5]);
                acc[6] = fma(q, fabs(dg), acc[6]);
                if (WORK) {
                    T cFF, cFS, cSF, cSS;
                    child_chords_ab(a, b, dd.z, fabs(dd.w), cFF, cFS, cSF, cSS);
                    evals += (cFF > T(0)) + (cFS > T(0)) + (cSF > T(0)) + (cSS > T(0));
                }
            } else {
                const T ch = block_chord_ab(a, b, dd.z, fabs(dd.w));
                acc[0] = fma(q, ch, acc[0]);
                if (WORK) evals += ch > T(0);
            }
        }
    }
    if (MODE == kBpQuad) {
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] *= hx;
    } else {
        // hx times the block scale 2^-level; (signed sum s, absolute sum a)
        // -> + part (s + a) / 2 and - part (s - a) / 2, clamped to their
        // signs against rounding
        const T scale = hx / T(bsz);
        acc[0] *= scale;
        if (MODE == kBpSplit) {
#pragma unroll
            for (int k = 1; k < 7; k += 2) {
                const T sg = acc[k] * scale, ab = acc[k + 1] * scale;
                acc[k] = fmax(T(0.5) * (sg + ab), T(0));
                acc[k + 1] = fmin(T(0.5) * (sg - ab), T(0));
            }
        }
    }
}

template <typename T, bool TABLE, bool WORK>
__device__ __forceinline__ void bp_dispatch(const Geom<T>& g, const Segment& S, int bx, int by, int chunk, int wv,
                                            const T* sino, const typename Vec4<T>::type* dirtab, T (&acc)[7],
                                            unsigned& evals)
{
    if (S.quad) bp_item<T, kBpQuad, TABLE, WORK>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
    else if (S.has_details) bp_item<T, kBpSplit, TABLE, WORK>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
    else bp_item<T, kBpBlock, TABLE, WORK>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
}

// a4 (Eq. 1.10) and a0: one CTA = kItemsPerCta items (lanes) x kViewLanes
// warps, each warp taking every kViewLanes-th view of the CTA's view chunk;
// the warps' sums meet in shared memory in a fixed order and leave one
// partial per (item, chunk, slot).
// CTA number `cta` of the back-projection plan tab.  Every thread of the CTA
// must call it.
template <typename T>
__device__ __forceinline__ void bp_body(const Geom<T>& g, const SegTable& tab, int cta, const T* __restrict__ sino,
                                        const typename Vec4<T>::type* __restrict__ dirtab, T* __restrict__ part,
                                        unsigned long long* __restrict__ work)
{
    __shared__ T red[kViewLanes][7][kItemsPerCta];
    int si = 0;
    while (si + 1 < tab.n && cta >= tab.s[si + 1].cta_begin) ++si;
    const Segment& S = tab.s[si];
    const int local = cta - S.cta_begin;
    const int chunk = local / S.tiles, tile = local - chunk * S.tiles;
    const int lane = threadIdx.x & 31, wv = threadIdx.x >> 5;
    const int item = tile * kItemsPerCta + lane;
    const bool quad = S.quad != 0;
    const bool det = S.has_details != 0;
    T acc[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};
    unsigned evals = 0;
    if (item < S.n_items) {
        int bx, by;
        if (S.items) {
            const uint32_t w = S.items[item];
            bx = (int)(w & 0xffffu);
            by = (int)(w >> 16);
        } else {
            bx = item % S.gw;
            by = item / S.gw;
        }
        if (dirtab) {
            if (work) bp_dispatch<T, true, true>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
            else bp_dispatch<T, true, false>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
        } else {
            if (work) bp_dispatch<T, false, true>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
            else bp_dispatch<T, false, false>(g, S, bx, by, chunk, wv, sino, dirtab, acc, evals);
        }
    }
    const T aA = acc[0], hP = acc[1], hM = acc[2], vP = acc[3], vM = acc[4], dP = acc[5], dM = acc[6];
    add_work(work, evals);
    // fixed-order sum of the 8 view lanes, one partial per (item, view range)
    red[wv][0][lane] = aA;
    red[wv][1][lane] = hP; red[wv][2][lane] = hM;
    red[wv][3][lane] = vP; red[wv][4][lane] = vM;
    red[wv][5][lane] = dP; red[wv][6][lane] = dM;
    __syncthreads();
    const int t = threadIdx.x;
    if (t < 7 * kItemsPerCta) {
        const int k = t / kItemsPerCta, l = t - k * kItemsPerCta;
        const int it = tile * kItemsPerCta + l;
        if (it < S.n_items) {
            if (quad) {
                // pixel k = (ylo,xlo), (ylo,xhi), (yhi,xlo), (yhi,xhi) in slots 0..3
                if (k < 4) {
                    T sumk = red[0][k][l];
#pragma unroll
                    for (int w = 1; w < kViewLanes; ++w) sumk += red[w][k][l];
                    part[S.part_off + ((size_t)chunk * S.n_slots + k) * S.n_items + it] = sumk;
                }
            } else {
                // slot k of the segment: 0 = approximation when present, then h+ .. d-
                const int slot = S.has_approx ? k : k - 1;
                const bool used = (k == 0) ? S.has_approx != 0 : det;
                if (used) {
                    T sumk = red[0][k][l];
#pragma unroll
                    for (int w = 1; w < kViewLanes; ++w) sumk += red[w][k][l];
                    part[S.part_off + ((size_t)chunk * S.n_slots + slot) * S.n_items + it] = sumk;
                }
            }
        }
    }
}

// Six CTAs per SM (at most 40 registers): the extra warps hide more of the
// gathers' latency than the tighter allocation costs.
template <typename T>
__global__ void __launch_bounds__(kBackTPB, 6)
k_backproject(Geom<T> g, SegTable tab, const T* __restrict__ sino,
              const typename Vec4<T>::type* __restrict__ dirtab, T* __restrict__ part,
              unsigned long long* __restrict__ work)
{
    bp_body<T>(g, tab, blockIdx.x, sino, dirtab, part, work);
}

// ---------------------------------------------------------------------------
// helpers over segment items
// ---------------------------------------------------------------------------

__device__ __forceinline__ int find_item_segment(const SegTable& tab, int gid)
{
    int si = 0;
    while (si + 1 < tab.n && gid >= tab.s[si + 1].item_begin) ++si;
    return si;
}

__device__ __forceinline__ void item_block(const Segment& S, int item, int& bx, int& by)
{
    if (S.items) {
        const uint32_t w = S.items[item];
        bx = (int)(w & 0xffffu);
        by = (int)(w >> 16);
    } else {
        bx = item % S.gw;
        by = item / S.gw;
    }
}

// Sum of one slot of an item over its view ranges, in a fixed order, in the
// kernel precision T.
template <typename T>
__device__ __forceinline__ T sum_slot(const Segment& S, const T* __restrict__ part, int item, int slot)
{
    T s = T(0);
    const T* p = part + S.part_off + (size_t)slot * S.n_items + item;
    const size_t stride = (size_t)S.n_slots * S.n_items;
    for (int c = 0; c < S.n_chunks; ++c) s += p[c * stride];
    return s;
}

__device__ __forceinline__ long long approx_index(const Layout& lay, int level, int bx, int by)
{
    return level == 0 ? (long long)by * lay.nx + bx : (long long)by * lay.gw[lay.L] + bx;
}

__device__ __forceinline__ long long detail_index(const Layout& lay, int level, int t, int bx, int by)
{
    return lay.coff[level] + (long long)t * lay.gw[level] * lay.gh[level] + (long long)by * lay.gw[level] + bx;
}

// Eq. 1.9 = 0 solved for Delta = beta~ - betahat.  With u = exp(-Z0 Delta):
// bp u^2 - b u + bm = 0, bp >= 0 >= bm, whose positive root is taken in the
// form free of cancellation for the sign of b.  root_t returns t = Z0 Delta
// = -ln u, or +-big where the minimiser is at +-infinity (u = 0 or u = inf);
// no ray weight (bp = bm = 0): 0.
__device__ __forceinline__ double root_t(double b, double bp, double bm, double big)
{
    if (bp > 0.0) {
        const double disc = sqrt(b * b - 4.0 * bp * bm);
        const double u = (b >= 0.0) ? (b + disc) / (2.0 * bp) : 2.0 * bm / (b - disc);
        return (u > 0.0) ? -log(u) : big;
    }
    if (bm < 0.0) return (b < 0.0) ? -log(bm / b) : -big;
    return 0.0;
}

// The same in FP32.  The root u is a ratio, so b, bp and bm are first
// divided by the largest of |b|, bp, -bm (at least 1e-30, for q-hat
// underflowing behind metal): no square or product can overflow, and no case
// needs FP64 arithmetic (GB300's FP64 rate is a small fraction of its FP32
// rate).  A square that underflows leaves u at most a factor 2 off where
// -ln u > 43, i.e. beyond any clamp.
__device__ __forceinline__ float root_t32(float bf, float bp, float bm, float big)
{
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
            t = (u > 0.0f) ? -logf(u) : big;
        } else if (bm < 0.0f) {
            t = (bf < 0.0f) ? -logf(bm / bf) : -big;
        }
    }
    return t;
}

// A minimiser at +-infinity is clamped to |Z0 Delta| = clamp (hit reports
// that the step sits at the clamp).
__device__ __forceinline__ double am_delta(double b, double bp, double bm, double z0, double clamp, bool& hit)
{
    double t = root_t(b, bp, bm, clamp);   // = Z0 * Delta
    t = fmin(fmax(t, -clamp), clamp);
    hit = fabs(t) >= clamp;
    return t / z0;
}

// FP32 root (iz0 = 1 / Z0 in FP32).
__device__ __forceinline__ double am_delta_f32(double b, float bp, float bm, double z0, float iz0, double clamp,
                                               bool& hit)
{
    float t = root_t32((float)b, bp, bm, (float)clamp);
    t = fminf(fmaxf(t, -(float)clamp), (float)clamp);
    hit = fabsf(t) >= (float)clamp;
    return (double)(t * iz0);
}

__device__ __forceinline__ double am_step(double b, float bp, float bm, double z0, float iz0, double clamp, bool& hit)
{
    return am_delta_f32(b, bp, bm, z0, iz0, clamp, hit);
}

__device__ __forceinline__ double am_step(double b, double bp, double bm, double z0, float, double clamp, bool& hit)
{
    return am_delta(b, bp, bm, z0, clamp, hit);
}

// The step with an L1 penalty lam |beta| on the coefficient (Eq. 1.1 with
// R = the l1 norm of the detail coefficients): the minimiser of the
// one-coefficient surrogate of Eq. 1.8 plus lam |betahat + Delta|, a convex
// function with a kink at t0 = -Z0 betahat (beta = 0).  Eq. 1.9's left side
// increases in Delta, so the minimiser is the root for b + lam if it lies
// beyond the kink, the root for b - lam if it lies before it, else the kink
// itself (zero = true: beta becomes exactly 0).  The decision uses the
// unclamped roots; the step is then clamped like the others.
__device__ __forceinline__ double am_step_l1(double b, double bp, double bm, double z0, float, double clamp,
                                             double bhat, double lam, bool& hit, bool& zero)
{
    const double big = 1e300;
    const double up = root_t(b + lam, bp, bm, big), dn = root_t(b - lam, bp, bm, big);
    const double t0 = -z0 * bhat;
    double t = up > t0 ? up : (dn < t0 ? dn : t0);
    zero = !(up > t0) && !(dn < t0) && fabs(t0) <= clamp;
    t = fmin(fmax(t, -clamp), clamp);
    hit = fabs(t) >= clamp;
    return t / z0;
}

__device__ __forceinline__ double am_step_l1(double b, float bp, float bm, double z0, float iz0, double clamp,
                                             double bhat, double lam, bool& hit, bool& zero)
{
    const float big = 3e38f;
    const float up = root_t32((float)(b + lam), bp, bm, big), dn = root_t32((float)(b - lam), bp, bm, big);
    const float t0 = (float)(-z0 * bhat);
    float t = up > t0 ? up : (dn < t0 ? dn : t0);
    zero = !(up > t0) && !(dn < t0) && fabsf(t0) <= (float)clamp;
    t = fminf(fmaxf(t, -(float)clamp), (float)clamp);
    hit = fabsf(t) >= (float)clamp;
    return (double)(t * iz0);
}

// Sum of one slot of an item over the view chunks c = lane, lane + G, ... of
// one lane of a group of G (fixed order within the lane).
template <typename T>
__device__ __forceinline__ T sum_slot_lane(const Segment& S, const T* __restrict__ part, int item, int slot, int lane,
                                           int G)
{
    T s = T(0);
    const T* p = part + S.part_off + (size_t)slot * S.n_items + item;
    const size_t stride = (size_t)S.n_slots * S.n_items;
#pragma unroll 4
    for (int c = lane; c < S.n_chunks; c += G) s += p[c * stride];
    return s;
}

// The G lanes' sums of a group added by a fixed butterfly (every lane gets
// the same total).
template <int G, typename T>
__device__ __forceinline__ T group_sum(T x)
{
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// a6: reduce the partials of each item and apply the AM update to beta.  One
// group of G lanes per coefficient: coefficient 4 i + k of item i is pixel k
// of a quad, or (k = 0) the approximation and (k = 1..3) detail type k of a
// block; the lanes split the item's view-chunk partials, a fixed butterfly
// adds them, and lane 0 applies the update.  G is chosen per segment: 8 when
// its items carry 8 or more view chunks (coarse levels), else 1.
__host__ __device__ __forceinline__ int upd_lanes(const Segment& S) { return S.n_chunks >= 8 ? 8 : 1; }
// Threads of a segment in the update grid: 4 coefficients per item, its lanes
// each, padded to whole warps (a warp never spans two segments).
__host__ __device__ __forceinline__ long long upd_threads(const Segment& S)
{
    return (4LL * S.n_items * upd_lanes(S) + 31) / 32 * 32;
}

// Thread gid of the update grid of plan tab (threads of whole warps).
template <typename T>
__device__ __forceinline__ void update_body(const SegTable& tab, const Layout& lay, const T* __restrict__ part,
                                            const double* __restrict__ bvec, const double* __restrict__ z0p,
                                            double clamp, double* __restrict__ beta, float* __restrict__ beta32,
                                            int nonneg, double lam, unsigned long long* __restrict__ hits,
                                            long long gid)
{
    int si = 0;
    long long first = 0;
    while (si < tab.n && gid >= first + upd_threads(tab.s[si])) first += upd_threads(tab.s[si++]);
    if (si >= tab.n) return;                 // whole warps past the last segment
    const Segment& S = tab.s[si];
    const int G = upd_lanes(S);              // uniform over the warp
    const long long local = gid - first;
    const long long cf = local / G;
    const int lane8 = (int)(local % G);
    long long z = -1;
    T bp = T(0), bm = T(0);
    const bool pix = S.quad || S.level == 0;   // a pixel coefficient (pixel basis)
    if (cf < 4LL * S.n_items) {              // every lane reaches the shuffles below
        const int item = (int)(cf >> 2), k = (int)(cf & 3);
        int bx, by;
        item_block(S, item, bx, by);
        if (S.quad) {
            z = (long long)(2 * by + (k >> 1)) * lay.nx + 2 * bx + (k & 1);
            bp = sum_slot_lane(S, part, item, k, lane8, G);
        } else if (k == 0) {
            if (S.has_approx) {
                z = approx_index(lay, S.level, bx, by);
                bp = sum_slot_lane(S, part, item, 0, lane8, G);
            }
        } else if (S.has_details) {
            const int t = k - 1, slot = (S.has_approx ? 1 : 0) + 2 * t;
            z = detail_index(lay, S.level, t, bx, by);
            bp = sum_slot_lane(S, part, item, slot, lane8, G);
            bm = sum_slot_lane(S, part, item, slot + 1, lane8, G);
        }
    }
    if (G == 8) {
        bp = group_sum<8>(bp);
        bm = group_sum<8>(bm);
    }
    if (z < 0 || lane8 != 0) return;
    const double z0 = *z0p;
    const float iz0 = 1.0f / (float)z0;
    bool hit = false;
    double nb;
    if (lam > 0.0 && !pix && (cf & 3) != 0) {
        // a detail coefficient under the L1 penalty
        bool zero = false;
        const double bh = beta[z];
        nb = bh + am_step_l1(bvec[z], bp, bm, z0, iz0, clamp, bh, lam, hit, zero);
        if (zero) nb = 0.0;
    } else {
        nb = beta[z] + am_step(bvec[z], bp, bm, z0, iz0, clamp, hit);
    }
    // plain AM kept nonnegative: the pixel's step ends at mu = 0 (the
    // separable surrogate's minimiser over mu >= 0)
    if (nonneg && pix) nb = fmax(nb, 0.0);
    beta[z] = nb;
    if (beta32) beta32[z] = (float)nb;
    add_work(hits, hit ? 1u : 0u);     // steps at the clamp |Z0 Delta| = clamp
}

template <typename T>
__global__ void k_update(SegTable tab, Layout lay, const T* __restrict__ part, const double* __restrict__ bvec,
                         const double* __restrict__ z0p, double clamp, double* __restrict__ beta,
                         float* __restrict__ beta32, int nonneg, double lam, unsigned long long* __restrict__ hits)
{
    update_body<T>(tab, lay, part, bvec, z0p, clamp, beta, beta32, nonneg, lam, hits,
                   (long long)blockIdx.x * blockDim.x + threadIdx.x);
}

// Scatter the reduced bhat+ / bhat- of each item into coefficient layout.
template <typename T>
__global__ void k_split_out(SegTable tab, Layout lay, const T* __restrict__ part, double* __restrict__ bplus,
                            double* __restrict__ bminus)
{
    const int gid = blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= tab.total_items) return;
    const Segment& S = tab.s[find_item_segment(tab, gid)];
    const int item = gid - S.item_begin;
    int bx, by;
    item_block(S, item, bx, by);
    if (S.quad) {
        for (int k = 0; k < 4; ++k) {
            const long long z = (long long)(2 * by + (k >> 1)) * lay.nx + 2 * bx + (k & 1);
            bplus[z] = (double)sum_slot(S, part, item, k);
            if (bminus) bminus[z] = 0.0;
        }
        return;
    }
    int slot = 0;
    if (S.has_approx) {
        const long long z = approx_index(lay, S.level, bx, by);
        bplus[z] = (double)sum_slot(S, part, item, 0);
        if (bminus) bminus[z] = 0.0;
        slot = 1;
    }
    if (S.has_details) {
        for (int t = 0; t < 3; ++t) {
            const long long z = detail_index(lay, S.level, t, bx, by);
            bplus[z] = (double)sum_slot(S, part, item, slot + 2 * t);
            if (bminus) bminus[z] = (double)sum_slot(S, part, item, slot + 2 * t + 1);
        }
    }
}

// Pixel-basis back-projection result (level-0 segment) into an image.
template <typename T, typename O>
__global__ void k_reduce_pixels(SegTable tab, int nx, long long npix, const T* __restrict__ part,
                                O* __restrict__ out)
{
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const Segment& S = tab.s[0];
    if (S.quad) {
        const int ix = (int)(p % nx), iy = (int)(p / nx);
        const int item = (iy >> 1) * S.gw + (ix >> 1);
        out[p] = (O)sum_slot(S, part, item, ((iy & 1) << 1) | (ix & 1));
    } else {
        out[p] = (O)sum_slot(S, part, (int)p, 0);
    }
}

// ---------------------------------------------------------------------------
// a1, Eq. 1.2: mu = Omega beta over the tree.  Per pixel, only the levels
// above its leaf carry active details; below they are inactive (zero).
// ---------------------------------------------------------------------------
// a1, Eq. 1.2: mu at pixel (ix, iy) = the sum over the active coefficients
// whose support holds it, i.e. the level-L approximation and the details of
// the expanded ancestors above its leaf level lam, in FP64.
__device__ __forceinline__ double synth_at(const Layout& lay, const double* __restrict__ beta, int ix, int iy,
                                           int lam)
{
    const int L = lay.L;
    double v = beta[(long long)(iy >> L) * lay.gw[L] + (ix >> L)] * pow2m(L);
    for (int l = L; l > lam; --l) {
        const int bx = ix >> l, by = iy >> l;
        const double sh = ((iy >> (l - 1)) & 1) ? -1.0 : 1.0;
        const double sv = ((ix >> (l - 1)) & 1) ? -1.0 : 1.0;
        const long long n = (long long)lay.gw[l] * lay.gh[l];
        const long long z = lay.coff[l] + (long long)by * lay.gw[l] + bx;
        v += (sh * beta[z] + sv * beta[z + n] + sh * sv * beta[z + 2 * n]) * pow2m(l);
    }
    return v;
}

// The same sum in FP32 from the float copy of the coefficients (the FP32
// forward's input; 2^-l applied exactly).
__device__ __forceinline__ float pow2mf(int l) { return __int_as_float((127 - l) << 23); }

__device__ __forceinline__ float synth_at(const Layout& lay, const float* __restrict__ beta, int ix, int iy, int lam)
{
    const int L = lay.L;
    float v = beta[(long long)(iy >> L) * lay.gw[L] + (ix >> L)] * pow2mf(L);
    for (int l = L; l > lam; --l) {
        const int bx = ix >> l, by = iy >> l;
        const float sh = ((iy >> (l - 1)) & 1) ? -1.0f : 1.0f;
        const float sv = ((ix >> (l - 1)) & 1) ? -1.0f : 1.0f;
        const long long n = (long long)lay.gw[l] * lay.gh[l];
        const long long z = lay.coff[l] + (long long)by * lay.gw[l] + bx;
        v += (sh * beta[z] + sv * beta[z + n] + sh * sv * beta[z + 2 * n]) * pow2mf(l);
    }
    return v;
}

template <typename T>
__global__ void k_synth(Layout lay, const uint8_t* __restrict__ leaf, const double* __restrict__ beta,
                        T* __restrict__ mu)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= lay.nx * lay.ny) return;
    if (lay.L == 0) {
        mu[p] = (T)beta[p];
        return;
    }
    const int ix = p % lay.nx, iy = p / lay.nx;
    mu[p] = (T)synth_at(lay, beta, ix, iy, leaf ? (int)leaf[p] : 0);
}

// a1 fused with the strip walk's input: the apron-padded copies of k_pad2
// (cells of 2^lam pixels, row-major and transposed) filled straight from the
// coefficients; a cell's value is mu at its first pixel.
// Tile (tx, ty) of 32 x 32 padded cells; CTAs of 32 x 8 threads.
template <typename T>
__device__ __forceinline__ void synth_pad2_body(const Layout& lay, const uint8_t* __restrict__ leaf,
                                                const typename SynthCoef<T>::type* __restrict__ beta, int lam,
                                                int nx, int ny, T* __restrict__ py, T* __restrict__ px, int tx,
                                                int ty)
{
    __shared__ T tile[32][33];
    const int x0 = tx * 32 - 1, y0 = ty * 32 - 1;
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int x = x0 + threadIdx.x, y = y0 + k;
        T v = T(0);
        if (x >= 0 && x < nx && y >= 0 && y < ny) {
            const int ix = x << lam, iy = y << lam;
            v = lay.L == 0 ? (T)beta[(long long)iy * lay.nx + ix]
                           : (T)synth_at(lay, beta, ix, iy, leaf ? (int)leaf[(long long)iy * lay.nx + ix] : 0);
        }
        tile[k][threadIdx.x] = v;
        if (x <= nx && y <= ny) py[(size_t)(y + 1) * pad_row(nx) + (x + 1)] = v;
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += 8) {
        const int y = y0 + threadIdx.x, x = x0 + k;
        if (x <= nx && y <= ny) px[(size_t)(x + 1) * pad_row(ny) + (y + 1)] = tile[threadIdx.x][k];
    }
}

template <typename T>
__global__ void k_synth_pad2(Layout lay, const uint8_t* __restrict__ leaf,
                             const typename SynthCoef<T>::type* __restrict__ beta, int lam, int nx, int ny,
                             T* __restrict__ py, T* __restrict__ px)
{
    synth_pad2_body<T>(lay, leaf, beta, lam, nx, ny, py, px, blockIdx.x, blockIdx.y);
}

// Leaf level of every pixel from the masks.
__global__ void k_leafmap(Layout lay, const uint8_t* __restrict__ mask, uint8_t* __restrict__ leaf)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= lay.nx * lay.ny) return;
    const int ix = p % lay.nx, iy = p / lay.nx;
    int lam = lay.L;
    for (int l = lay.L; l >= 1; --l) {
        if (mask[lay.moff[l] + (long long)(iy >> l) * lay.gw[l] + (ix >> l)]) lam = l - 1;
        else break;
    }
    leaf[p] = (uint8_t)lam;
}

// ---------------------------------------------------------------------------
// a7: the tree-growth criterion (Results section)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_max_partial(const T* __restrict__ S, int n, double* __restrict__ part)
{
    double m = -INFINITY;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        m = fmax(m, (double)S[i]);
    m = block_reduce<double>(m, OpMax(), -INFINITY);
    if (threadIdx.x == 0) part[blockIdx.x] = m;
}

// thr = tau * max S, in FP64
__global__ void k_threshold(const double* __restrict__ part, int n, double tau, double* __restrict__ thr)
{
    double m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, part[i]);
    m = block_reduce<double>(m, OpMax(), -INFINITY);
    if (threadIdx.x == 0) *thr = tau * m;
}

// Every selected pixel marks its leaf block (leaf read from the tree before
// the step) as expanded in the new mask.  Stores of 1 are idempotent.
template <typename T>
__global__ void k_expand_mark(Layout lay, const T* __restrict__ S, const double* __restrict__ thr, int all,
                              const uint8_t* __restrict__ leaf_old, uint8_t* __restrict__ mask_new)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= lay.nx * lay.ny) return;
    const int lam = leaf_old[p];
    if (lam < 1) return;
    if (!all && !((double)S[p] > *thr)) return;
    const int ix = p % lay.nx, iy = p / lay.nx;
    mask_new[lay.moff[lam] + (long long)(iy >> lam) * lay.gw[lam] + (ix >> lam)] = 1;
}

// Compacted block lists, one CTA per list, blocks in Morton (Z) order so
// that neighbouring threads of the back-projector hold neighbouring blocks.
// List 0: level-L blocks not expanded; list 1: level-L blocks expanded;
// list 1 + k (k = 1..L-1): expanded blocks of level L - k.
__device__ __forceinline__ uint32_t compact_bits(uint32_t x)
{
    x &= 0x55555555u;
    x = (x | (x >> 1)) & 0x33333333u;
    x = (x | (x >> 2)) & 0x0f0f0f0fu;
    x = (x | (x >> 4)) & 0x00ff00ffu;
    x = (x | (x >> 8)) & 0x0000ffffu;
    return x;
}

// A list's Morton codes go by chunks of 1024, one CTA each: a first launch
// counts each chunk's kept blocks, a second one writes them at the offset the
// chunks before it sum to (the same order as one sequential pass).
struct CompactList {
    int level, want, gw, gh;
    long long ncode;
};

__device__ __forceinline__ CompactList compact_list(const Layout& lay, int list)
{
    CompactList c;
    c.level = list <= 1 ? lay.L : lay.L - (list - 1);
    c.want = list == 0 ? 0 : 1;
    c.gw = lay.gw[c.level];
    c.gh = lay.gh[c.level];
    int side = 1;
    while (side < c.gw || side < c.gh) side <<= 1;
    c.ncode = (long long)side * side;
    return c;
}

// kept blocks of chunk `chunk` of list `list`: this thread's flag and code,
// the CTA's total and this thread's rank among the kept (in code order)
__device__ __forceinline__ void compact_chunk(const Layout& lay, const uint8_t* __restrict__ mask,
                                              const CompactList& cl, int chunk, bool& keep, uint32_t& code,
                                              int& rank, int& total)
{
    __shared__ int warp_cnt[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const long long m = (long long)chunk * 1024 + threadIdx.x;
    keep = false;
    code = 0;
    if (m < cl.ncode) {
        const int bx = (int)compact_bits((uint32_t)m), by = (int)compact_bits((uint32_t)(m >> 1));
        if (bx < cl.gw && by < cl.gh) {
            const int e = mask[lay.moff[cl.level] + (long long)by * cl.gw + bx] ? 1 : 0;
            keep = (e == cl.want);
            code = ((uint32_t)by << 16) | (uint32_t)bx;
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    int off = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
        const int n = warp_cnt[w];
        off += w < wid ? n : 0;
        tot += n;
    }
    rank = off + __popc(bal & ((1u << lane) - 1u));
    total = tot;
}

__global__ void __launch_bounds__(1024) k_compact_count(Layout lay, const uint8_t* __restrict__ mask,
                                                        int* __restrict__ chunk_cnt, int max_chunks)
{
    const int list = blockIdx.y, chunk = blockIdx.x;
    const CompactList cl = compact_list(lay, list);
    if ((long long)chunk * 1024 >= cl.ncode) return;
    bool keep;
    uint32_t code;
    int rank, total;
    compact_chunk(lay, mask, cl, chunk, keep, code, rank, total);
    if (threadIdx.x == 0) chunk_cnt[list * max_chunks + chunk] = total;
}

__global__ void __launch_bounds__(1024) k_compact(Layout lay, const uint8_t* __restrict__ mask,
                                                  uint32_t* __restrict__ lists, long long list_stride,
                                                  const int* __restrict__ chunk_cnt, int max_chunks,
                                                  int* __restrict__ counts)
{
    const int list = blockIdx.y, chunk = blockIdx.x;
    const CompactList cl = compact_list(lay, list);
    const int nchunk = (int)((cl.ncode + 1023) / 1024);
    if (chunk >= nchunk) return;
    __shared__ int base;
    if (threadIdx.x < 32) {                  // the earlier chunks' counts, summed by one warp
        int b = 0;
        for (int c = threadIdx.x; c < chunk; c += 32) b += chunk_cnt[list * max_chunks + c];
        b = warp_reduce(b, OpSum());
        if (threadIdx.x == 0) base = b;
    }
    bool keep;
    uint32_t code;
    int rank, total;
    compact_chunk(lay, mask, cl, chunk, keep, code, rank, total);   // its barrier publishes base
    if (keep) lists[list_stride * list + base + rank] = code;
    if (chunk == nchunk - 1 && threadIdx.x == 0) counts[list] = base + total;
}

// ---------------------------------------------------------------------------
// full orthonormal Haar transform, one level per launch (FP64)
// ---------------------------------------------------------------------------
// analysis of level l: `a` is the level l-1 approximation image (w x h,
// w = nx >> (l-1)); writes the level-l approximation into a_next and the
// three detail planes into coef.
__global__ void k_haar_analysis(Layout lay, int l, const double* __restrict__ a, double* __restrict__ a_next,
                                double* __restrict__ coef)
{
    const int gw = lay.gw[l], gh = lay.gh[l];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gw * gh) return;
    const int bx = i % gw, by = i / gw;
    const int w = 2 * gw;
    const double ll = a[(2 * by) * w + 2 * bx], lh = a[(2 * by) * w + 2 * bx + 1];
    const double hl = a[(2 * by + 1) * w + 2 * bx], hh = a[(2 * by + 1) * w + 2 * bx + 1];
    a_next[i] = 0.5 * (ll + lh + hl + hh);
    const long long n = (long long)gw * gh;
    double* c = coef + lay.coff[l];
    c[i] = 0.5 * (ll + lh - hl - hh);
    c[n + i] = 0.5 * (ll - lh + hl - hh);
    c[2 * n + i] = 0.5 * (ll - lh - hl + hh);
}

__global__ void k_haar_synthesis(Layout lay, int l, const double* __restrict__ a, const double* __restrict__ coef,
                                 double* __restrict__ a_prev)
{
    const int gw = lay.gw[l], gh = lay.gh[l];
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= gw * gh) return;
    const int bx = i % gw, by = i / gw;
    const int w = 2 * gw;
    const long long n = (long long)gw * gh;
    const double* c = coef + lay.coff[l];
    const double A = a[i], h = c[i], v = c[n + i], d = c[2 * n + i];
    a_prev[(2 * by) * w + 2 * bx] = 0.5 * (A + h + v + d);
    a_prev[(2 * by) * w + 2 * bx + 1] = 0.5 * (A + h - v - d);
    a_prev[(2 * by + 1) * w + 2 * bx] = 0.5 * (A - h + v - d);
    a_prev[(2 * by + 1) * w + 2 * bx + 1] = 0.5 * (A - h - v + d);
}

// per-ray constant of the cost: d (log d - log I0) - d, 0 log 0 = 0
__global__ void k_dterm(const float* __restrict__ d, const float* __restrict__ I0, long long n,
                        double* __restrict__ out, float2* __restrict__ out2)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double dd = d[i];
    const double t = dd > 0.0 ? dd * (log(dd) - log((double)I0[i])) - dd : 0.0;
    out[i] = t;
    const float hi = (float)t;
    out2[i] = make_float2(hi, (float)(t - (double)hi));
}

__global__ void k_fill_f32(float* __restrict__ x, long long n, float v)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = v;
}

template <typename A, typename B>
__global__ void k_convert(const A* __restrict__ x, B* __restrict__ y, long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = (B)x[i];
}

// ---------------------------------------------------------------------------
// host launchers
// ---------------------------------------------------------------------------
// dst row k = src row perm[k] (rows of B elements): a scan's views in
// another order
template <typename E>
__global__ void k_permute_rows(const E* __restrict__ src, E* __restrict__ dst, const int* __restrict__ perm,
                               int V, int B)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)V * B) return;
    const int k = (int)(i / B), b = (int)(i - (long long)k * B);
    dst[i] = src[(long long)perm[k] * B + b];
}

static inline unsigned nblk(long long n, int t) { return (unsigned)((n + t - 1) / t); }


static std::atomic<unsigned long long> g_launches{0};
unsigned long long kernel_launches() { return g_launches.load(); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
#define COUNT_LAUNCH() g_launches.fetch_add(1, std::memory_order_relaxed)

template <typename E>
cudaError_t launch_permute_rows(const E* src, E* dst, const int* perm, int V, int B, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_permute_rows<E><<<nblk((long long)V * B, 256), 256, 0, st>>>(src, dst, perm, V, B);
    return cudaGetLastError();
}
template cudaError_t launch_permute_rows<float>(const float*, float*, const int*, int, int, cudaStream_t);
template cudaError_t launch_permute_rows<double>(const double*, double*, const int*, int, int, cudaStream_t);
template cudaError_t launch_permute_rows<float2>(const float2*, float2*, const int*, int, int, cudaStream_t);

// ---------------------------------------------------------------------------
// P2: one iteration of many bags in five launches.  The forward and the
// back-projector are persistent: a grid of about one wave pulls work items
// (bag, view, bin tile) or (bag, CTA of the bag's plan) from a global
// counter, the largest bags first; each item runs the single-bag kernel's
// body, so every partial and every sum is formed as the per-bag kernels form
// it (in other kernels, where the compiler may contract multiply-adds
// differently: the results agree to FP32 rounding).
// ---------------------------------------------------------------------------

// bag k owns items pre[k] .. pre[k+1]-1
__device__ __forceinline__ int bag_of(const int* __restrict__ pre, int n, int item)
{
    int k = 0;
    while (k + 1 < n && item >= pre[k + 1]) ++k;
    return k;
}

// A CTA's walk over the work queue: thread 0 takes the next item from the
// counter while the CTA works on the current one (the atomic's latency
// overlaps the work), and a barrier hands it on.  body(item) must contain a
// CTA barrier after its last read of shared memory.
template <typename F>
__device__ __forceinline__ void for_each_item(int* __restrict__ counter, int total, F&& body)
{
    __shared__ int s_item;
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    int cur = s_item;
    while (cur < total) {
        int nxt = 0;
        if (threadIdx.x == 0) nxt = atomicAdd(counter, 1);
        body(cur);
        __syncthreads();                   // every thread has read s_item and finished the item
        if (threadIdx.x == 0) s_item = nxt;
        __syncthreads();
        cur = s_item;
    }
}

__global__ void k_multi_synth(const BagDev* __restrict__ bags, const BatchPrefix* __restrict__ pre)
{
    const int item = blockIdx.x;
    const int k = bag_of(pre->syn, pre->n, item);
    const BagDev& B = bags[k];
    const int local = item - pre->syn[k];
    synth_pad2_body<float>(B.lay, B.lay.L > 0 ? B.leaf : nullptr, B.beta32, B.lam, B.gc.nx, B.gc.ny, B.pad,
                           B.pad + (size_t)pad_row(B.gc.nx) * (B.gc.ny + 2), local % B.syn_tx, local / B.syn_tx);
}

__global__ void __launch_bounds__(kFwdTPB) k_multi_forward(const BagDev* __restrict__ bags,
                                                           const BatchPrefix* __restrict__ pre,
                                                           int* __restrict__ counter)
{
    for_each_item(counter, pre->fwd[pre->n], [&](int item) {
        const int k = bag_of(pre->fwd, pre->n, item);
        const BagDev& B = bags[k];
        const int local = item - pre->fwd[k];
        const int v = local / B.fwd_tiles, t = local - v * B.fwd_tiles;
        forward_body<float, true, false>(B.gc, nullptr, B.pad, nullptr, B.d, B.dterm, B.I0, B.q, nullptr, nullptr,
                                         B.cpart, nullptr, v, t, v * B.fwd_tiles + t);
    });
}

__global__ void __launch_bounds__(1024) k_multi_sum(const BagDev* __restrict__ bags)
{
    const BagDev& B = bags[blockIdx.x];
    sum_at_body(B.cpart, B.ncost, B.costs, B.counter);
}

__global__ void __launch_bounds__(kBackTPB) k_multi_backproject(const BagDev* __restrict__ bags,
                                                                const BatchPrefix* __restrict__ pre,
                                                                int* __restrict__ counter)
{
    for_each_item(counter, pre->bp[pre->n], [&](int item) {
        const int k = bag_of(pre->bp, pre->n, item);
        const BagDev& B = bags[k];
        bp_body<float>(B.g, B.tab, item - pre->bp[k], B.q, B.dirt, B.part, nullptr);
    });
}

__global__ void k_multi_update(const BagDev* __restrict__ bags, const BatchPrefix* __restrict__ pre)
{
    const long long gid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= pre->upd[pre->n]) return;   // whole warps (every bag's share is)
    const int k = bag_of(pre->upd, pre->n, (int)gid);
    const BagDev& B = bags[k];
    update_body<float>(B.tab, B.lay, B.part, B.bvec, B.z0, B.clamp, B.beta, const_cast<float*>(B.beta32), B.nonneg,
                       0.0, nullptr, gid - pre->upd[k]);
}

int batch_launches_per_iteration() { return 5; }

long long update_threads(const SegTable& tab)
{
    long long t = 0;
    for (int i = 0; i < tab.n; ++i) t += upd_threads(tab.s[i]);
    return t;
}

cudaError_t launch_batch_iteration(const BagDev* bags, const BatchPrefix* pre_dev, const BatchPrefix& pre,
                                   int* counters, cudaStream_t st)
{
    static int grid_fwd = 0, grid_bp = 0;
    if (!grid_fwd) {
        int dev = 0, sms = 0, of = 0, ob = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&of, k_multi_forward, kFwdTPB, 0) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ob, k_multi_backproject, kBackTPB, 0) != cudaSuccess)
            return cudaGetLastError();
        grid_fwd = std::max(1, sms * of);
        grid_bp = std::max(1, sms * ob);
    }
    cudaError_t e = cudaMemsetAsync(counters, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (pre.syn[pre.n] > 0) {
        COUNT_LAUNCH();
        k_multi_synth<<<pre.syn[pre.n], dim3(32, 8), 0, st>>>(bags, pre_dev);
    }
    COUNT_LAUNCH();
    k_multi_forward<<<std::min(grid_fwd, std::max(1, pre.fwd[pre.n])), kFwdTPB, 0, st>>>(bags, pre_dev, counters);
    COUNT_LAUNCH();
    k_multi_sum<<<pre.n, 1024, 0, st>>>(bags);
    COUNT_LAUNCH();
    k_multi_backproject<<<std::min(grid_bp, std::max(1, pre.bp[pre.n])), kBackTPB, 0, st>>>(bags, pre_dev,
                                                                                            counters + 1);
    if (pre.upd[pre.n] > 0) {
        COUNT_LAUNCH();
        k_multi_update<<<nblk(pre.upd[pre.n], 256), 256, 0, st>>>(bags, pre_dev);
    }
    return cudaGetLastError();
}

// ---- the staged forward's host side -----------------------------------------

// Raised by a staged forward whose tensor copy did not complete in time; one
// word per device, read and cleared by the host code after a reconstruction.
__device__ int g_stage_err;

int* stage_error_word()
{
    static int* addr[64] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    if (!addr[dev] && cudaGetSymbolAddress((void**)&addr[dev], g_stage_err) != cudaSuccess) {
        cudaGetLastError();
        addr[dev] = nullptr;
    }
    return addr[dev];
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled()
{
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(f);
        else
            cudaGetLastError();
    });
    return fn;
}

// The tensor map of one apron-padded copy: rows of `cols` used elements at
// the stride pad_row(cols - 2), `rows` rows; tiles of stage_rows x kStageCols,
// out-of-range elements read as zero.
static bool pad_map(CUtensorMap* m, const float* base, int cols, int rows, int stage_rows)
{
    EncodeTiledFn fn = encode_tiled();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)pad_row(cols - 2) * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)kStageCols, (cuuint32_t)stage_rows};
    const cuuint32_t es[2] = {1, 1};
    return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, es,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The strip walk over the padded copies in pad (cell grid gc): staged when the
// tensor maps can be made, else from global memory.  FP32 only.
template <typename T>
static void launch_strip_walk(const Geom<T>& gc, T* pad, const float* d, const typename CostTerm<T>::type* dterm,
                              const float* I0, T* qhat, T* p_out, T* resid, double* cost_part,
                              unsigned long long* work, cudaStream_t st)
{
    const dim3 grid(nblk(gc.B, kFwdTPB), gc.V);
    if constexpr (std::is_same<T, float>::value) {
        CUtensorMap my, mx;
        int* err = stage_error_word();
        // staged tiles pay off from 128-cell grids up (coarser grids' bands are
        // a few cells wide and their walks a few stages long)
        const int R = std::min(gc.nx, gc.ny) >= 128 ? gc.stage_rows : 0;
        if ((R == 16 || R == 24 || R == 32) && err && pad_map(&my, pad, gc.nx + 2, gc.ny + 2, R) &&
            pad_map(&mx, pad + (size_t)pad_row(gc.nx) * (gc.ny + 2), gc.ny + 2, gc.nx + 2, R)) {
            COUNT_LAUNCH();
#define WAM_STAGED(RR, WW)                                                                                  \
    k_forward_staged<RR, WW><<<grid, kFwdTPB, 0, st>>>(gc, pad, my, mx, d, dterm, I0, qhat, p_out, resid, cost_part, \
                                                       work, err)
            if (R == 16) { if (work) WAM_STAGED(16, true); else WAM_STAGED(16, false); }
            else if (R == 24) { if (work) WAM_STAGED(24, true); else WAM_STAGED(24, false); }
            else { if (work) WAM_STAGED(32, true); else WAM_STAGED(32, false); }
#undef WAM_STAGED
            return;
        }
    }
    COUNT_LAUNCH();
    if (work)
        k_forward<T, true, true><<<grid, kFwdTPB, 0, st>>>(gc, nullptr, pad, nullptr, d, dterm, I0, qhat, p_out, resid,
                                                           cost_part, work);
    else
        k_forward<T, true, false><<<grid, kFwdTPB, 0, st>>>(gc, nullptr, pad, nullptr, d, dterm, I0, qhat, p_out,
                                                            resid, cost_part, work);
}

template <typename T>
cudaError_t launch_forward(const Geom<T>& g, const T* mu, T* pad, const uint8_t* leaf, int lam, const float* d,
                           const typename CostTerm<T>::type* dterm, const float* I0, T* qhat, T* p_out, T* resid,
                           double* cost_part, unsigned long long* work, cudaStream_t st)
{
    dim3 grid(nblk(g.B, kFwdTPB), g.V);
    if (leaf) {
        COUNT_LAUNCH();
        if (work)
            k_forward<T, false, true><<<grid, kFwdTPB, 0, st>>>(g, mu, nullptr, leaf, d, dterm, I0, qhat, p_out,
                                                                resid, cost_part, work);
        else
            k_forward<T, false, false><<<grid, kFwdTPB, 0, st>>>(g, mu, nullptr, leaf, d, dterm, I0, qhat, p_out,
                                                                 resid, cost_part, work);
    } else {
        if (!pad || lam < 0 || (g.nx >> lam) << lam != g.nx || (g.ny >> lam) << lam != g.ny)
            return cudaErrorInvalidValue;
        const Geom<T> gc = cell_grid(g, lam);
        COUNT_LAUNCH();
        k_pad2<T><<<dim3(nblk(gc.nx + 2, 32), nblk(gc.ny + 2, 32)), dim3(32, 8), 0, st>>>(
            mu, g.nx, lam, gc.nx, gc.ny, pad, pad + (size_t)pad_row(gc.nx) * (gc.ny + 2));
        launch_strip_walk(gc, pad, d, dterm, I0, qhat, p_out, resid, cost_part, work, st);
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_forward_tree(const Geom<T>& g, const Layout& lay, const uint8_t* leaf,
                                const typename SynthCoef<T>::type* beta, int lam, T* pad, const float* d, const typename CostTerm<T>::type* dterm,
                                const float* I0, T* qhat, T* p_out, T* resid, double* cost_part,
                                unsigned long long* work, cudaStream_t st)
{
    if (!pad || lam < 0 || (g.nx >> lam) << lam != g.nx || (g.ny >> lam) << lam != g.ny)
        return cudaErrorInvalidValue;
    const Geom<T> gc = cell_grid(g, lam);
    COUNT_LAUNCH();
    k_synth_pad2<T><<<dim3(nblk(gc.nx + 2, 32), nblk(gc.ny + 2, 32)), dim3(32, 8), 0, st>>>(
        lay, leaf, beta, lam, gc.nx, gc.ny, pad, pad + (size_t)pad_row(gc.nx) * (gc.ny + 2));
    launch_strip_walk(gc, pad, d, dterm, I0, qhat, p_out, resid, cost_part, work, st);
    return cudaGetLastError();
}

int forward_parts(int V, int B) { return (int)nblk(B, kFwdTPB) * V * (kFwdTPB / 32); }
int forward_cost_parts(int V, int B) { return (int)nblk(B, kFwdTPB) * V; }

cudaError_t launch_sum_final(const double* part, int n, double* out, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_sum_final<<<1, 1024, 0, st>>>(part, n, out);
    return cudaGetLastError();
}

cudaError_t launch_sum_at(const double* part, int n, double* out, int* counter, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_sum_at<<<1, 1024, 0, st>>>(part, n, out, counter);
    return cudaGetLastError();
}

cudaError_t launch_max_final(const double* part, int n, double* out, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_max_final<<<1, 1024, 0, st>>>(part, n, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_z0(const Geom<T>& g, const Layout& lay, const uint8_t* leaf, double* part, cudaStream_t st)
{
    dim3 grid(nblk(g.B, kFwdTPB), g.V);
    COUNT_LAUNCH();
    switch (lay.L) {
    case 0: k_z0<T, 0><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 1: k_z0<T, 1><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 2: k_z0<T, 2><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 3: k_z0<T, 3><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 4: k_z0<T, 4><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 5: k_z0<T, 5><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 6: k_z0<T, 6><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 7: k_z0<T, 7><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    case 8: k_z0<T, 8><<<grid, kFwdTPB, 0, st>>>(g, lay, leaf, part); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_backproject(const Geom<T>& g, const SegTable& tab, const T* sino, const void* dirtab, T* part,
                               unsigned long long* work, cudaStream_t st)
{
    if (tab.total_ctas == 0) return cudaSuccess;
    COUNT_LAUNCH();
    k_backproject<T><<<tab.total_ctas, kBackTPB, 0, st>>>(
        g, tab, sino, static_cast<const typename Vec4<T>::type*>(dirtab), part, work);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update(const SegTable& tab, const Layout& lay, const T* part, const double* b,
                          const double* z0, double clamp, double* beta, float* beta32, int nonneg, double lam,
                          unsigned long long* hits, cudaStream_t st)
{
    if (tab.total_items == 0) return cudaSuccess;
    long long threads = 0;
    for (int i = 0; i < tab.n; ++i) threads += upd_threads(tab.s[i]);
    COUNT_LAUNCH();
    k_update<T><<<nblk(threads, 256), 256, 0, st>>>(tab, lay, part, b, z0, clamp, beta, beta32, nonneg, lam, hits);
    return cudaGetLastError();
}

// lam * sum of |beta| over the detail coefficients (indices from the count
// of level-L approximations on; inactive ones are 0): one FP64 partial per
// CTA of 256 threads, each thread summing 4 coefficients in a fixed order.
__global__ void k_l1_sum(const double* __restrict__ beta, long long first, long long n, double lam,
                         double* __restrict__ part)
{
    double s = 0.0;
    const long long base = first + ((long long)blockIdx.x * blockDim.x + threadIdx.x) * 4;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < n) s += fabs(beta[base + k]);
    s = block_reduce(s, OpSum(), 0.0);
    if (threadIdx.x == 0) part[blockIdx.x] = lam * s;
}

int l1_parts(const Layout& lay)
{
    const long long nA = (long long)lay.gw[lay.L] * lay.gh[lay.L];
    const long long nd = (long long)lay.nx * lay.ny - nA;
    return (int)std::max(1LL, (nd + 1023) / 1024);
}

cudaError_t launch_l1_sum(const Layout& lay, const double* beta, double lam, double* part, cudaStream_t st)
{
    const long long nA = (long long)lay.gw[lay.L] * lay.gh[lay.L];
    COUNT_LAUNCH();
    k_l1_sum<<<l1_parts(lay), 256, 0, st>>>(beta, nA, (long long)lay.nx * lay.ny, lam, part);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_split_out(const SegTable& tab, const Layout& lay, const T* part, double* bp, double* bm,
                             cudaStream_t st)
{
    if (tab.total_items == 0) return cudaSuccess;
    COUNT_LAUNCH();
    k_split_out<T><<<nblk(tab.total_items, 256), 256, 0, st>>>(tab, lay, part, bp, bm);
    return cudaGetLastError();
}

template <typename T, typename O>
cudaError_t launch_reduce_pixels(const SegTable& tab, int nx, long long npix, const T* part, O* out,
                                 cudaStream_t st)
{
    COUNT_LAUNCH();
    k_reduce_pixels<T, O><<<nblk(npix, 256), 256, 0, st>>>(tab, nx, npix, part, out);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_synth(const Layout& lay, const uint8_t* leaf, const double* beta, T* mu, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_synth<T><<<nblk((long long)lay.nx * lay.ny, 256), 256, 0, st>>>(lay, leaf, beta, mu);
    return cudaGetLastError();
}

cudaError_t launch_leafmap(const Layout& lay, const uint8_t* mask, uint8_t* leaf, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_leafmap<<<nblk((long long)lay.nx * lay.ny, 256), 256, 0, st>>>(lay, mask, leaf);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_expand(const Layout& lay, const T* S, double tau, const uint8_t* leaf_old,
                          uint8_t* mask_new, double* scratch /* >= 257 doubles */, cudaStream_t st)
{
    const int n = lay.nx * lay.ny;
    const int nb = 256;
    COUNT_LAUNCH();
    k_max_partial<T><<<nb, 256, 0, st>>>(S, n, scratch);
    COUNT_LAUNCH();
    k_threshold<<<1, 256, 0, st>>>(scratch, nb, tau, scratch + nb);
    COUNT_LAUNCH();
    k_expand_mark<T><<<nblk(n, 256), 256, 0, st>>>(lay, S, scratch + nb, tau < 0.0 ? 1 : 0, leaf_old, mask_new);
    return cudaGetLastError();
}

int compact_chunks(const Layout& lay)
{
    int gw = 1, gh = 1;
    for (int l = 1; l <= lay.L; ++l) {
        gw = std::max(gw, lay.gw[l]);
        gh = std::max(gh, lay.gh[l]);
    }
    long long side = 1;
    while (side < gw || side < gh) side <<= 1;
    return (int)((side * side + 1023) / 1024);
}

cudaError_t launch_compact(const Layout& lay, const uint8_t* mask, uint32_t* lists, long long list_stride,
                           int* counts, int* chunk_cnt, cudaStream_t st)
{
    const int nlists = lay.L + 1, maxc = compact_chunks(lay);
    COUNT_LAUNCH();
    k_compact_count<<<dim3(maxc, nlists), 1024, 0, st>>>(lay, mask, chunk_cnt, maxc);
    COUNT_LAUNCH();
    k_compact<<<dim3(maxc, nlists), 1024, 0, st>>>(lay, mask, lists, list_stride, chunk_cnt, maxc, counts);
    return cudaGetLastError();
}

cudaError_t launch_haar(const Layout& lay, const double* in, double* out, int inverse, double* tmp_a,
                        double* tmp_b, cudaStream_t st)
{
    const long long N = (long long)lay.nx * lay.ny;
    if (lay.L == 0) return cudaMemcpyAsync(out, in, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (!inverse) {
        const double* a = in;
        double* bufs[2] = {tmp_a, tmp_b};
        for (int l = 1; l <= lay.L; ++l) {
            double* an = (l == lay.L) ? out : bufs[l & 1];   // level-L approximations go first in `out`
            COUNT_LAUNCH();
            k_haar_analysis<<<nblk((long long)lay.gw[l] * lay.gh[l], 256), 256, 0, st>>>(lay, l, a, an, out);
            a = an;
        }
    } else {
        // start from the level-L approximations stored at the front of `in`
        const double* a = in;
        double* bufs[2] = {tmp_a, tmp_b};
        for (int l = lay.L; l >= 1; --l) {
            double* ap = (l == 1) ? out : bufs[l & 1];
            COUNT_LAUNCH();
            k_haar_synthesis<<<nblk((long long)lay.gw[l] * lay.gh[l], 256), 256, 0, st>>>(lay, l, a, in, ap);
            a = ap;
        }
    }
    return cudaGetLastError();
}

cudaError_t launch_dterm(const float* d, const float* I0, long long n, double* out, float2* out2, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_dterm<<<nblk(n, 256), 256, 0, st>>>(d, I0, n, out, out2);
    return cudaGetLastError();
}

cudaError_t launch_fill_f32(float* x, long long n, float v, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_fill_f32<<<nblk(n, 256), 256, 0, st>>>(x, n, v);
    return cudaGetLastError();
}

template <typename A, typename B>
cudaError_t launch_convert(const A* x, B* y, long long n, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_convert<A, B><<<nblk(n, 256), 256, 0, st>>>(x, y, n);
    return cudaGetLastError();
}

// out = a - (float)b (the subtraction of an FP64 vector rounded to float)
__global__ void k_sub_f64(const float* __restrict__ a, const double* __restrict__ b, float* __restrict__ out,
                          long long n)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = a[i] - (float)b[i];
}

cudaError_t launch_sub_f64(const float* a, const double* b, float* out, long long n, cudaStream_t st)
{
    COUNT_LAUNCH();
    k_sub_f64<<<nblk(n, 256), 256, 0, st>>>(a, b, out, n);
    return cudaGetLastError();
}

// a6 on dense coefficient arrays (the step-level entry point): every active
// coefficient gets its AM step from given b, bhat+, bhat-.
__global__ void k_update_dense(Layout lay, const uint8_t* __restrict__ mask, const double* __restrict__ bvec,
                               const double* __restrict__ bp, const double* __restrict__ bm,
                               const double* __restrict__ z0p, double clamp, double* __restrict__ beta)
{
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long N = (long long)lay.nx * lay.ny;
    if (z >= N) return;
    const int L = lay.L;
    const long long nA = (long long)lay.gw[L] * lay.gh[L];
    if (L > 0 && z >= nA) {
        int l = L;
        while (l > 1 && z >= lay.coff[l - 1]) --l;
        const long long n = (long long)lay.gw[l] * lay.gh[l];
        const long long r = (z - lay.coff[l]) % n;
        const int bx = (int)(r % lay.gw[l]), by = (int)(r / lay.gw[l]);
        if (!mask[lay.moff[l] + (long long)by * lay.gw[l] + bx]) return;
    }
    bool hit = false;
    beta[z] += am_delta(bvec[z], bp[z], bm ? bm[z] : 0.0, *z0p, clamp, hit);
}

// a6 per coefficient on flat arrays, with the same root the reconstruction's
// k_update<T> applies (am_step: FP32 on normalised inputs for T = float, FP64
// for T = double; am_step_l1 where lam > 0): the step-level view of the AM
// update.
template <typename T>
__global__ void k_am_delta(long long n, const double* __restrict__ bvec, const double* __restrict__ bp,
                           const double* __restrict__ bm, const double* __restrict__ bhat, double lam, double z0,
                           double clamp, double* __restrict__ delta, int* __restrict__ at_clamp)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    bool hit = false;
    const float iz0 = 1.0f / (float)z0;
    double dl;
    if (lam > 0.0) {
        bool zero = false;
        dl = am_step_l1(bvec[i], (T)bp[i], (T)bm[i], z0, iz0, clamp, bhat[i], lam, hit, zero);
        if (zero) dl = -bhat[i];
    } else {
        dl = am_step(bvec[i], (T)bp[i], (T)bm[i], z0, iz0, clamp, hit);
    }
    delta[i] = dl;
    if (at_clamp) at_clamp[i] = hit ? 1 : 0;
}

cudaError_t launch_am_delta(int precision, long long n, const double* b, const double* bp, const double* bm,
                            const double* bhat, double lam, double z0, double clamp, double* delta, int* at_clamp,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    COUNT_LAUNCH();
    if (precision == 32)
        k_am_delta<float><<<nblk(n, 256), 256, 0, st>>>(n, b, bp, bm, bhat, lam, z0, clamp, delta, at_clamp);
    else
        k_am_delta<double><<<nblk(n, 256), 256, 0, st>>>(n, b, bp, bm, bhat, lam, z0, clamp, delta, at_clamp);
    return cudaGetLastError();
}

cudaError_t launch_update_dense(const Layout& lay, const uint8_t* mask, const double* b, const double* bp,
                                const double* bm, const double* z0, double clamp, double* beta, cudaStream_t st)
{
    const long long N = (long long)lay.nx * lay.ny;
    COUNT_LAUNCH();
    k_update_dense<<<nblk(N, 256), 256, 0, st>>>(lay, mask, b, bp, bm, z0, clamp, beta);
    return cudaGetLastError();
}

// explicit instantiations
#define WAM_INST(T)                                                                                              \
    template cudaError_t launch_forward_tree<T>(const Geom<T>&, const Layout&, const uint8_t*,                      \
                                                const typename SynthCoef<T>::type*, int, T*,                          \
                                                const float*, const typename CostTerm<T>::type*, const float*, T*,    \
                                                T*, T*, double*, unsigned long long*, cudaStream_t);                  \
    template cudaError_t launch_forward<T>(const Geom<T>&, const T*, T*, const uint8_t*, int, const float*,          \
                                           const typename CostTerm<T>::type*, const float*, T*, T*, T*, double*,      \
                                           unsigned long long*, cudaStream_t);                                        \
    template cudaError_t launch_z0<T>(const Geom<T>&, const Layout&, const uint8_t*, double*, cudaStream_t);     \
    template cudaError_t launch_backproject<T>(const Geom<T>&, const SegTable&, const T*, const void*, T*,       \
                                               unsigned long long*, cudaStream_t);                              \
    template cudaError_t launch_update<T>(const SegTable&, const Layout&, const T*, const double*, const double*, \
                                          double, double*, float*, int, double, unsigned long long*,             \
                                          cudaStream_t);                                                         \
    template cudaError_t launch_split_out<T>(const SegTable&, const Layout&, const T*, double*, double*,         \
                                             cudaStream_t);                                                      \
    template cudaError_t launch_synth<T>(const Layout&, const uint8_t*, const double*, T*, cudaStream_t);        \
    template cudaError_t launch_expand<T>(const Layout&, const T*, double, const uint8_t*, uint8_t*, double*,    \
                                          cudaStream_t);
WAM_INST(float)
WAM_INST(double)
#undef WAM_INST
template cudaError_t launch_reduce_pixels<float, float>(const SegTable&, int, long long, const float*, float*,
                                                       cudaStream_t);
template cudaError_t launch_reduce_pixels<float, double>(const SegTable&, int, long long, const float*, double*,
                                                        cudaStream_t);
template cudaError_t launch_reduce_pixels<double, double>(const SegTable&, int, long long, const double*, double*,
                                                         cudaStream_t);
template cudaError_t launch_convert<float, double>(const float*, double*, long long, cudaStream_t);
template cudaError_t launch_convert<double, float>(const double*, float*, long long, cudaStream_t);

}  // namespace wam
