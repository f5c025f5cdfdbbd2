// Host-side launchers of the libwam kernels (internal).
#pragma once

#include "../../include/wam.h"
#include "wam_internal.cuh"

#include <string>

namespace wam {

// WAM_OK for a geometry wam_create accepts, else WAM_ERR_ARG with the reason
// in *why (wam_api.cu).
wam_status check_geometry(const wam_geometry* g, std::string* why);

// The per-ray cost constant d (log d - log I0) - d as the forward of type T
// reads it: FP64 for T = double; for T = float a pair (hi, lo) of floats
// with hi + lo equal to the FP64 value to about 2^-48 relative (the FP32
// forward then forms the cancelling sum dterm + d p + q in float-float and
// needs no FP64 arithmetic per ray).
template <typename T> struct CostTerm { using type = double; };
template <> struct CostTerm<float> { using type = float2; };

// The coefficients the strip-walk forward of type T synthesises its cells
// from: FP64 for T = double; for T = float the float copy of beta that the
// FP32 update keeps beside it (no FP64 arithmetic per cell).
template <typename T> struct SynthCoef { using type = double; };
template <> struct SynthCoef<float> { using type = float; };

template <typename T>
// leaf: the leaf walk over the tree's leaf map; null: the strip walk over the
// grid of 2^lam-pixel cells (mu must be constant on them; lam = 0: pixels).
// pad: scratch of 2 (nx + 2)(ny + 2) elements, required when leaf is null
// (the strip walk reads apron-padded copies of the cell values written there).
cudaError_t launch_forward(const Geom<T>& g, const T* mu, T* pad, const uint8_t* leaf, int lam, const float* d,
                           const typename CostTerm<T>::type* dterm, const float* I0, T* qhat, T* p_out, T* resid, double* cost_part,
                           unsigned long long* work, cudaStream_t st);
// a1 + a2 + a3 for the strip walk: the padded cell images of 2^lam pixels
// synthesised from the coefficients beta over the tree (leaf map; null when
// L = 0) straight into pad, then the forward pass.
template <typename T>
cudaError_t launch_forward_tree(const Geom<T>& g, const Layout& lay, const uint8_t* leaf,
                                const typename SynthCoef<T>::type* beta, int lam, T* pad, const float* d, const typename CostTerm<T>::type* dterm,
                                const float* I0, T* qhat, T* p_out, T* resid, double* cost_part,
                                unsigned long long* work, cudaStream_t st);
int forward_parts(int V, int B);
int forward_cost_parts(int V, int B);   // cost partials a forward launch writes (one per CTA)
// dst row k = src row perm[k], rows of B elements (views of a scan reordered)
template <typename E>
cudaError_t launch_permute_rows(const E* src, E* dst, const int* perm, int V, int B, cudaStream_t st);
cudaError_t launch_sum_final(const double* part, int n, double* out, cudaStream_t st);
cudaError_t launch_max_final(const double* part, int n, double* out, cudaStream_t st);
cudaError_t launch_sum_at(const double* part, int n, double* out, int* counter, cudaStream_t st);
template <typename T>
cudaError_t launch_z0(const Geom<T>& g, const Layout& lay, const uint8_t* leaf, double* part, cudaStream_t st);
template <typename T>
cudaError_t launch_backproject(const Geom<T>& g, const SegTable& tab, const T* sino, const void* dirtab, T* part,
                               unsigned long long* work, cudaStream_t st);
template <typename T>
// beta32 (optional): the float copy of beta, rewritten for every updated
// coefficient; nonneg: pixel coefficients end their step at 0 (plain AM);
// lam > 0: detail coefficients take the L1-penalised step
cudaError_t launch_update(const SegTable& tab, const Layout& lay, const T* part, const double* b, const double* z0,
                          double clamp, double* beta, float* beta32, int nonneg, double lam, unsigned long long* hits,
                          cudaStream_t st);
// lam * sum |beta| over the detail coefficients as l1_parts(lay) FP64 partials
int l1_parts(const Layout& lay);
cudaError_t launch_l1_sum(const Layout& lay, const double* beta, double lam, double* part, cudaStream_t st);
template <typename T>
cudaError_t launch_split_out(const SegTable& tab, const Layout& lay, const T* part, double* bp, double* bm,
                             cudaStream_t st);
template <typename T, typename O>
cudaError_t launch_reduce_pixels(const SegTable& tab, int nx, long long npix, const T* part, O* out,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_synth(const Layout& lay, const uint8_t* leaf, const double* beta, T* mu, cudaStream_t st);
cudaError_t launch_leafmap(const Layout& lay, const uint8_t* mask, uint8_t* leaf, cudaStream_t st);
template <typename T>
cudaError_t launch_expand(const Layout& lay, const T* S, double tau, const uint8_t* leaf_old, uint8_t* mask_new,
                          double* scratch, cudaStream_t st);
// chunk_cnt: scratch of (L + 1) * compact_chunks(lay) ints
int compact_chunks(const Layout& lay);
cudaError_t launch_compact(const Layout& lay, const uint8_t* mask, uint32_t* lists, long long list_stride,
                           int* counts, int* chunk_cnt, cudaStream_t st);
cudaError_t launch_haar(const Layout& lay, const double* in, double* out, int inverse, double* tmp_a,
                        double* tmp_b, cudaStream_t st);
// dterm of every ray in FP64 (out) and as float pairs (out2)
cudaError_t launch_dterm(const float* d, const float* I0, long long n, double* out, float2* out2, cudaStream_t st);
cudaError_t launch_fill_f32(float* x, long long n, float v, cudaStream_t st);
template <typename A, typename B>
cudaError_t launch_convert(const A* x, B* y, long long n, cudaStream_t st);
cudaError_t launch_update_dense(const Layout& lay, const uint8_t* mask, const double* b, const double* bp,
                                const double* bm, const double* z0, double clamp, double* beta, cudaStream_t st);

// Eq. 1.9's step per coefficient on flat arrays with the reconstruction's own
// root (precision 32: bp, bm rounded to float and the FP32 root; 64: FP64;
// lam > 0: the L1-penalised step from the current values bhat)
cudaError_t launch_am_delta(int precision, long long n, const double* b, const double* bp, const double* bm,
                            const double* bhat, double lam, double z0, double clamp, double* delta, int* at_clamp,
                            cudaStream_t st);

// The strip walk's grid of 2^lam-pixel cells: the same box, cells 2^lam times larger.
template <typename T>
inline Geom<T> cell_grid(const Geom<T>& g, int lam)
{
    Geom<T> gc = g;
    gc.nx = g.nx >> lam;
    gc.ny = g.ny >> lam;
    gc.vx = g.vx * T(1 << lam);
    gc.vy = g.vy * T(1 << lam);
    gc.ivx = g.ivx / T(1 << lam);
    gc.ivy = g.ivy / T(1 << lam);
    return gc;
}

// Threads of the update grid of a plan (whole warps per segment).
long long update_threads(const SegTable& tab);

// One bag of a persistent batched iteration (FP32, strip-walk forward): what
// its five kernels read and write, and its share of their work.  Built on
// the host per tree epoch, read by the multi-bag kernels from device memory.
struct BagDev {
    Geom<float> g;          // the scan (the back-projector's geometry)
    Geom<float> gc;         // the strip walk's grid of 2^lam-pixel cells
    Layout lay;
    SegTable tab;           // the back-projection / update plan of the tree
    const uint8_t* leaf;    // leaf map (null when L = 0)
    const float* beta32;    // the float copy of beta the cells are synthesised from
    float* pad;             // apron-padded cell copies (row-major, then transposed)
    int lam;                // cells of 2^lam pixels
    int syn_tx, syn_ty;     // 32 x 32 cell tiles of the padded copies
    int fwd_tiles;          // bin tiles of kFwdTPB rays per view
    const float* d;
    const float2* dterm;
    const float* I0;
    float* q;               // q-hat
    double* cpart;          // the forward's cost partials (one per CTA of the per-bag launch)
    int ncost;              // how many
    const float4* dirt;     // direction table
    float* part;            // back-projection partials
    const double* bvec;     // b = Phi^T d
    const double* z0;
    double clamp;
    double* beta;
    int nonneg;
    double* costs;          // cost history
    int* counter;           // its slot counter
};

// The work of all bags in prefix form: bag k owns items pre[k] .. pre[k+1]-1
// (forward: view x bin tile; back-projection: CTAs of its plan; update:
// threads, whole warps; synthesis: cell tiles), bags in decreasing order of
// work so that the persistent kernels start the largest first.
struct BatchPrefix {
    int n;
    int fwd[kMaxBags + 1], bp[kMaxBags + 1], upd[kMaxBags + 1], syn[kMaxBags + 1];
};

// One iteration of every bag: cell synthesis, forward (persistent CTAs over
// a global item counter), cost sums, back-projection (persistent), update.
// counters: two device ints, reset on st before the kernels.  Results agree
// with the per-bag kernels' to FP32 rounding.
cudaError_t launch_batch_iteration(const BagDev* bags, const BatchPrefix* pre_dev, const BatchPrefix& pre,
                                   int* counters, cudaStream_t st);
int batch_launches_per_iteration();

// Device word raised by a staged forward whose shared-memory copy did not
// complete within its wait budget (then its results are invalid); null if
// the word cannot be located on the current device.
int* stage_error_word();

// out = a - (float)b, n elements
cudaError_t launch_sub_f64(const float* a, const double* b, float* out, long long n, cudaStream_t st);

unsigned long long kernel_launches();
// kernels run by graph replays (counted once when captured)
void add_launches(unsigned long long n);
void count_launch();

// grad.cu: operators for the gradient and the unrolled-AM patterns
cudaError_t launch_phi_project(const Geom<float>& g, const Layout& lay, const float* gbar, const float* dplus,
                               const float* dminus, const float* qhat, float* out, cudaStream_t st);
cudaError_t launch_am_derivs(const Layout& lay, const double* b, const double* bp, const double* bm,
                             const double* z0, double clamp, float* dplus, float* dminus, cudaStream_t st);
cudaError_t launch_l1(const Layout& lay, const float* beta, const double* g, float lambda, float* grad,
                      double* part, int nparts, cudaStream_t st);

}  // namespace wam
