// wam_backproject_static: H^T s for callers that must not allocate device
// memory.  Everything the back-projection needs besides its input and output
// (the per-view cos/sin table and the per-view-range partial sums) lives in
// one file-scope static device array, so this call performs no cudaMalloc,
// cudaFree or other allocating call.
#include "../../include/wam.h"
#include "wam_internal.cuh"
#include "wam_kernels.h"

#include <algorithm>
#include <cmath>
#include <string>

namespace {

// Shared scratch of every call on a device; held by each device that loads
// the library until the process exits.
constexpr size_t kStaticBytes = WAM_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_wam_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
// Device address of g_wam_static_scratch per device, found once per device.
void* g_scratch_addr[kMaxDevices] = {nullptr};

wam_status scratch_address(int dev, float** out)
{
    if (dev < 0 || dev >= kMaxDevices) return WAM_ERR_ARG;
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_wam_static_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return WAM_ERR_CUDA;
        }
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<float*>(g_scratch_addr[dev]);
    return WAM_OK;
}

// The per-view cos/sin table, written on the device into the scratch: the
// angle in FP64 exactly as the context path forms it (angle0 + k * span / V),
// its cosine and sine in FP64, each rounded once to float.
__global__ void k_static_views(float* __restrict__ cs, int V, double angle0, double step)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= V) return;
    const double th = angle0 + k * step;
    double sn, c;
    sincos(th, &sn, &c);
    cs[2 * k] = (float)c;
    cs[2 * k + 1] = (float)sn;
}

}  // namespace

extern "C" wam_status wam_backproject_static(const wam_geometry* w, const float* s, float* out, void* stream)
{
    using namespace wam;
    if (!w || !s || !out) return WAM_ERR_ARG;
    std::string why;
    if (check_geometry(w, &why) != WAM_OK || w->kind == WAM_CONE3D_FLAT_CIRCULAR) return WAM_ERR_ARG;
    const long long N = (long long)w->nx * w->ny;
    const int V = w->n_views;

    // one segment: every pixel (level 0), its views split into ranges so that
    // the grid holds about 1024 threads per SM
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return WAM_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
        cudaGetLastError();
        sms = 148;
    }
    const double mag = (w->kind == WAM_FAN2D_FLAT) ? 1.2 * w->sdd / w->sod : 1.0;
    const double shadow = std::sqrt(w->vx * w->vx + w->vy * w->vy) * mag / w->bin_pitch + 1.0;
    const double per_thread = std::max((double)N * V * shadow / (sms * 1024.0), 256.0);
    int vpc = std::max(1, std::min((int)std::lround(per_thread / shadow), V));
    SegTable tab{};
    Segment& sg = tab.s[0];
    tab.n = 1;
    sg.level = 0;
    sg.has_approx = 1;
    sg.has_details = 0;
    sg.n_items = (int)N;
    sg.items = nullptr;
    sg.gw = w->nx;
    // at most V / (view lanes) ranges, each a whole number of view lanes long
    // (capped at V), so that the CTA's warps get equal view counts
    const int chunks = std::max(1, std::min((V + vpc - 1) / vpc, std::max(1, V / kViewLanes)));
    sg.vpc = (V + chunks - 1) / chunks;
    sg.vpc = std::min(V, (sg.vpc + kViewLanes - 1) / kViewLanes * kViewLanes);
    sg.n_chunks = (V + sg.vpc - 1) / sg.vpc;
    sg.tiles = (int)((N + kItemsPerCta - 1) / kItemsPerCta);
    sg.cta_begin = 0;
    sg.item_begin = 0;
    sg.n_slots = 1;
    sg.part_off = 0;
    tab.total_ctas = sg.tiles * sg.n_chunks;
    tab.total_items = (int)N;

    // scratch layout: [2V floats: cos, sin per view][pad to 256 B][partials]
    const size_t cs_bytes = ((size_t)2 * V * sizeof(float) + 255) & ~(size_t)255;
    const size_t part_bytes = (size_t)sg.n_chunks * (size_t)N * sizeof(float);
    if (cs_bytes + part_bytes > kStaticBytes) return WAM_ERR_ARG;   // beyond the fixed scratch

    float* base = nullptr;
    wam_status st = scratch_address(dev, &base);
    if (st != WAM_OK) return st;
    float* cs = base;
    float* part = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(base) + cs_bytes);

    cudaStream_t cst = static_cast<cudaStream_t>(stream);
    // the view table is written on the device: no host-to-device copy
    count_launch();
    k_static_views<<<(V + 127) / 128, 128, 0, cst>>>(cs, V, w->angle0, w->angle_span / V);
    if (cudaGetLastError() != cudaSuccess) return WAM_ERR_CUDA;

    Geom<float> g;
    g.kind = w->kind;
    g.stage_rows = 0;
    g.nx = w->nx;
    g.ny = w->ny;
    g.V = V;
    g.B = w->n_bins;
    g.vx = (float)w->vx;
    g.vy = (float)w->vy;
    g.X0 = (float)(-0.5 * w->nx * w->vx);
    g.Y0 = (float)(-0.5 * w->ny * w->vy);
    g.ivx = (float)(1.0 / w->vx);
    g.ivy = (float)(1.0 / w->vy);
    g.pitch = (float)w->bin_pitch;
    g.ucen = (float)(0.5 * (w->n_bins - 1));
    g.sod = (float)w->sod;
    g.sdd = (float)w->sdd;
    g.cs = cs;
    // every partial of every (pixel, view range) is written before it is read:
    // nothing in the scratch needs clearing
    if (launch_backproject<float>(g, tab, s, nullptr, part, nullptr, cst) != cudaSuccess) return WAM_ERR_CUDA;
    if (launch_reduce_pixels<float, float>(tab, w->nx, N, part, out, cst) != cudaSuccess) return WAM_ERR_CUDA;
    return WAM_OK;
}
