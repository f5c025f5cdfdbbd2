// Kernels for differentiating through the method: the sign-split projection
// Phi+ a + Phi- c (the linearisation of bhat+-(beta), Eq. 1.10), the
// derivatives of the AM root (Eq. 1.9) with respect to bhat+ and bhat-, and
// the L1 term of an I-divergence + lambda ||beta_detail||_1 loss.
#include "wam_internal.cuh"
#include "wam_kernels.h"

namespace wam {

namespace {

template <typename V>
__device__ __forceinline__ V warp_sum(V x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    return x;
}

inline unsigned nb(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// Per ray y: out(y) = qhat(y) * sum over every coefficient z of the full
// L-level basis of [max(phi, 0) gbar dplus + min(phi, 0) gbar dminus](y, z).
// The ray walks single pixels; a level-l block's detail phi values are built
// from the chords of its four children as in the Z0 kernel (a block is
// crossed in one run of pixels, so its terms are final when the next block
// of that level appears); the approximation's phi = 2^-L chord >= 0 is added
// pixel by pixel.
__global__ void __launch_bounds__(kFwdTPB)
k_phi_project(Geom<float> g, Layout lay, const float* __restrict__ gbar, const float* __restrict__ dplus,
              const float* __restrict__ dminus, const float* __restrict__ qhat, float* __restrict__ out)
{
    const int v = blockIdx.y;
    const int b = blockIdx.x * kFwdTPB + threadIdx.x;
    if (b >= g.B) return;
    const int L = lay.L;
    Ray<float> r;
    float total = 0.0f;
    if (make_ray(g, v, b, r)) {
        float acc[kMaxLevels][4];
        int cur[kMaxLevels];
#pragma unroll
        for (int l = 0; l < kMaxLevels; ++l) {
            cur[l] = -1;
            acc[l][0] = acc[l][1] = acc[l][2] = acc[l][3] = 0.0f;
        }
        const float sA = 1.0f / (float)(1 << L);
        auto flush = [&](int li) {
            if (cur[li] >= 0) {
                const int l = li + 1;
                const float* a = acc[li];
                const float s = 1.0f / (float)(1 << l);
                const int bx = cur[li] & 0xffff, by = cur[li] >> 16;
                const long long n = (long long)lay.gw[l] * lay.gh[l];
                const long long z0 = lay.coff[l] + (long long)by * lay.gw[l] + bx;
                const float ph[3] = {s * (a[0] + a[1] - a[2] - a[3]), s * (a[0] - a[1] + a[2] - a[3]),
                                     s * (a[0] - a[1] - a[2] + a[3])};
#pragma unroll
                for (int t = 0; t < 3; ++t) {
                    const long long z = z0 + t * n;
                    const float gz = __ldg(gbar + z);
                    total += ph[t] > 0.0f ? ph[t] * gz * __ldg(dplus + z) : ph[t] * gz * __ldg(dminus + z);
                }
            }
            acc[li][0] = acc[li][1] = acc[li][2] = acc[li][3] = 0.0f;
        };
        traverse_pixels(g, r, [&](int ix, int iy, float c) {
            const long long zA = (long long)(iy >> L) * lay.gw[L] + (ix >> L);
            total += sA * c * __ldg(gbar + zA) * __ldg(dplus + zA);
#pragma unroll
            for (int li = 0; li < kMaxLevels; ++li) {
                const int l = li + 1;
                if (l <= L) {
                    const int id = ((iy >> l) << 16) | (ix >> l);
                    if (id != cur[li]) {
                        flush(li);
                        cur[li] = id;
                    }
                    const int q = (((iy >> li) & 1) << 1) | ((ix >> li) & 1);
                    acc[li][0] += q == 0 ? c : 0.0f;
                    acc[li][1] += q == 1 ? c : 0.0f;
                    acc[li][2] += q == 2 ? c : 0.0f;
                    acc[li][3] += q == 3 ? c : 0.0f;
                }
            }
        });
#pragma unroll
        for (int li = 0; li < kMaxLevels; ++li) flush(li);
    }
    const size_t y = (size_t)v * g.B + b;
    out[y] = qhat ? qhat[y] * total : total;
}

// dDelta/dbhat+ and dDelta/dbhat- of the AM step (FP64 root, FP32 result).
// With u the positive root of bp u^2 - b u + bm = 0 and sqrt(D) =
// sqrt(b^2 - 4 bp bm) = 2 bp u - b:  du/dbp = -u^2/sqrt(D), du/dbm = -1/sqrt(D),
// Delta = -ln(u)/Z0, so dDelta/dbp = u/(Z0 sqrt(D)), dDelta/dbm = 1/(Z0 u sqrt(D)).
// Clamped or degenerate steps have zero derivative.
__global__ void k_am_derivs(long long n, const double* __restrict__ bvec, const double* __restrict__ bp,
                            const double* __restrict__ bm, const double* __restrict__ z0p, double clamp,
                            float* __restrict__ dplus, float* __restrict__ dminus)
{
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= n) return;
    const double b = bvec[z], p = bp[z], m = bm ? bm[z] : 0.0, Z0 = *z0p;
    double u = 0.0;
    bool ok = false;
    if (p > 0.0) {
        const double disc = sqrt(b * b - 4.0 * p * m);
        u = (b >= 0.0) ? (b + disc) / (2.0 * p) : 2.0 * m / (b - disc);
        ok = u > 0.0;
    } else if (m < 0.0 && b < 0.0) {
        u = m / b;
        ok = true;
    }
    float fp = 0.0f, fm = 0.0f;
    if (ok && fabs(log(u)) < clamp) {
        const double sd = sqrt(b * b - 4.0 * p * m);
        if (sd > 0.0) {
            fp = (float)(u / (Z0 * sd));
            fm = (float)(1.0 / (Z0 * u * sd));
        }
    }
    dplus[z] = fp;
    dminus[z] = fm;
}

// grad = g + lambda sign(beta) on the detail coefficients (index >= nA);
// part[cta] = lambda * sum |beta_detail| of the CTA's coefficients.
__global__ void k_l1(long long n, long long nA, const float* __restrict__ beta, const double* __restrict__ gin,
                     float lambda, float* __restrict__ grad, double* __restrict__ part)
{
    const long long z = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l1 = 0.0;
    if (z < n) {
        float gz = (float)gin[z];
        if (z >= nA) {
            const float bz = beta[z];
            gz += bz > 0.0f ? lambda : (bz < 0.0f ? -lambda : 0.0f);
            l1 = (double)lambda * fabs((double)bz);
        }
        grad[z] = gz;
    }
    __shared__ double sh[32];
    l1 = warp_sum(l1);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = l1;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
        part[blockIdx.x] = s;
    }
}

cudaError_t launch_phi_project(const Geom<float>& g, const Layout& lay, const float* gbar, const float* dplus,
                               const float* dminus, const float* qhat, float* out, cudaStream_t st)
{
    count_launch();
    dim3 grid(nb(g.B, kFwdTPB), g.V);
    k_phi_project<<<grid, kFwdTPB, 0, st>>>(g, lay, gbar, dplus, dminus, qhat, out);
    return cudaGetLastError();
}

cudaError_t launch_am_derivs(const Layout& lay, const double* b, const double* bp, const double* bm,
                             const double* z0, double clamp, float* dplus, float* dminus, cudaStream_t st)
{
    const long long n = (long long)lay.nx * lay.ny;
    count_launch();
    k_am_derivs<<<nb(n, 256), 256, 0, st>>>(n, b, bp, bm, z0, clamp, dplus, dminus);
    return cudaGetLastError();
}

cudaError_t launch_l1(const Layout& lay, const float* beta, const double* g, float lambda, float* grad,
                      double* part, int nparts, cudaStream_t st)
{
    const long long n = (long long)lay.nx * lay.ny;
    const long long nA = (long long)lay.gw[lay.L] * lay.gh[lay.L];
    if ((long long)nparts < (long long)nb(n, 256)) return cudaErrorInvalidValue;
    count_launch();
    k_l1<<<nb(n, 256), 256, 0, st>>>(n, nA, beta, g, lambda, grad, part);
    return cudaGetLastError();
}

}  // namespace wam
