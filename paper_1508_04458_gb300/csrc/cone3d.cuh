// Internal declarations of the 3-D circular cone-beam path (FP32 bulk).
//
// Volume nx*ny*nz voxels, index (iz*ny + iy)*nx + ix; sinogram
// [view][row][bin].  Two wavelet modes: the 3-D Haar transform (octree,
// seven details per block; "z3") and the 2-D Haar transform of every
// z-slice with one tree shared by all slices ("slices").
#pragma once

#include "wam_internal.cuh"

namespace wam {

struct Geom3 {
    int nx, ny, nz, V, R, B;
    float vx, vy, vz, X0, Y0, Z0, ivx, ivy, ivz;
    float pitch, ucen, rpitch, rcen, sod, sdd;
    const float* cs;      // [V][2] cos, sin
    const float4* dirt;   // [V][B] (s/Dx, -c/Dy, 1/Dx, 1/Dy) of the in-plane direction (-SDD e + u_b u)
    const float* rowinv;  // [R] 1/v_r (finite)
    const float* dlen;    // [R][B] |D| = sqrt(SDD^2 + u_b^2 + v_r^2)
};

struct Layout3 {
    int L, nx, ny, nz, z3;
    int gw[kMaxLevels + 1], gh[kMaxLevels + 1], gd[kMaxLevels + 1];
    long long coff[kMaxLevels + 1];   // z3: first detail plane of level l; slices: within one slice
    long long moff[kMaxLevels + 1];   // mask offset of level l
    long long mask_bytes;
    long long nslice;                 // nx*ny
};

// items: (bx | by << 10 | bz << 20); bz is the slice index in the per-slice mode
struct Segment3 {
    int level, has_approx, has_details, octet;   // octet: voxel basis, item = 2x2x2 voxels
    int n_items;
    const uint32_t* items;            // null: implicit (x fastest) over gw x gh x gd
    int rep;                          // > 0: item i is items[i % rep] in slice i / rep
    int gw, gh;
    int n_chunks, vpc, tiles, cta_begin, item_begin, n_slots;
    long long part_off;
};

struct SegTable3 {
    int n, total_ctas, total_items;
    Segment3 s[2 * kMaxLevels + 4];
};

constexpr int kSlots3 = 15;           // approximation + 7 details x (+, -)

// launchers (cone3d.cu)
// leaf null and pad non-null: the strip walk over apron-padded copies of the
// cells of 2^lam voxels (2^lam x 2^lam x 1 when z3 = 0; mu must be constant on
// them) written to pad (2 (nx + 2)(ny + 2)(nz + 2) floats at most); else the
// leaf / voxel walk.
cudaError_t launch_forward3(const Geom3& g, const float* mu, float* pad, const uint8_t* leaf, int lam, int z3,
                            const float* d, const double* dterm, const float* I0, float* qhat, float* p_out,
                            double* cost_part, unsigned long long* work, cudaStream_t st);
int forward3_parts(const Geom3& g);
cudaError_t launch_backproject3(const Geom3& g, const SegTable3& tab, int z3, const float* sino, float* part,
                                unsigned long long* work, cudaStream_t st);
// nonneg: voxel coefficients (plain AM) end their step at 0
cudaError_t launch_update3(const SegTable3& tab, const Layout3& lay, const float* part, const double* b,
                           const double* z0, double clamp, double* beta, int nonneg, cudaStream_t st);
cudaError_t launch_reduce_voxels3(const SegTable3& tab, const Layout3& lay, const float* part, double* out,
                                  float* outf, cudaStream_t st);
cudaError_t launch_z03(const Geom3& g, const Layout3& lay, const uint8_t* leaf, double* part, cudaStream_t st);
cudaError_t launch_synth3(const Layout3& lay, const uint8_t* leaf, const double* beta, float* mu, cudaStream_t st);
cudaError_t launch_leafmap3(const Layout3& lay, const uint8_t* mask, uint8_t* leaf, cudaStream_t st);
cudaError_t launch_expand3(const Layout3& lay, const float* mu, double tau, const uint8_t* leaf_old,
                           uint8_t* mask_new, float* s2d, double* scratch, cudaStream_t st);
cudaError_t launch_compact3(const Layout3& lay, const uint8_t* mask, uint32_t* lists, long long stride,
                            int* counts, cudaStream_t st);
cudaError_t launch_haar3(const Layout3& lay, const double* img, double* coef, double* ta, double* tb,
                         cudaStream_t st);

}  // namespace wam
