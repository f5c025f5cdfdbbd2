// C-ABI of libwam: context, data, the reconstruction driver (Algorithm 1 with
// the Results section's tree growth, or plain AM) and the step-level calls.
// No exception crosses the boundary; every call returns a wam_status.
#include "../../include/wam.h"
#include "cone3d.cuh"
#include "wam_internal.cuh"
#include "wam_kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

using namespace wam;

namespace {

struct Buf {
    void* p = nullptr;
    size_t bytes = 0;
};

enum BufId {
    B_CS32, B_CS64, B_D, B_I0, B_DTERM,
    B_Q, B_MU, B_BETA, B_BVEC, B_MASK_A, B_MASK_B, B_LEAF, B_LISTS, B_COUNTS,
    B_PART, B_COSTPART, B_COSTS, B_Z0, B_SCRATCH, B_TMPA, B_TMPB, B_GIMG, B_SINO,
    B_DIR32, B_DIR64, B_GBETA, B_GMU, B_GRES, B_GCOEF, B_L1PART,
    B_DIR3, B_ROWINV, B_DLEN, B_S2D, B_COUNTER, B_MUT,
    B_PERM, B_CSP32, B_CSP64, B_DIRP32, B_DIRP64, B_DP, B_I0P, B_DTP, B_BSUB, B_Z0SUB, B_SINOP,
    B_DTERM2, B_BETA32, B_BATCH, B_VJP, B_VJPQ, B_VJPR, B_VJPD, B_VJPB,
    B_NBUF
};

}  // namespace

struct ProfPending {
    int k;
    cudaEvent_t a, b;
};

// Algorithm 1's state after a run (for wam_checkpoint) or loaded from a file
// (wam_resume, consumed by the next wam_reconstruct).
struct RunRecord {
    bool valid = false;
    int levels = 0, dims = 2, zsum = 0, precision = 32, full_am = 0;
    double clamp = 30.0;
    std::vector<int> expand_at;
    std::vector<double> tau;
    int iters_done = 0, expansions_done = 0, n_subsets = 1, nonneg = 0;
    double tuning = 32.0;
    double lambda = 0.0;
    std::vector<double> beta, hist;     // host copies (loaded state only)
    std::vector<uint8_t> mask;
};

struct wam_ctx {
    wam_geometry g{};
    RunRecord last;                        // last finished reconstruction (device buffers hold its arrays)
    RunRecord pending;                     // state loaded by wam_resume
    // profiling
    bool prof = false;                     // CUDA events around each kernel
    bool prof_work = false;                // work counters in the kernels
    std::vector<cudaEvent_t> ev_pool;
    std::vector<ProfPending> pend;
    wam_stats stats{};
    unsigned long long* dwork = nullptr;   // device [WAM_NKERNEL]
    long long last_leaves = 0;             // leaves of the tree last planned
    int last_lmin = 0;                     // ... and its finest leaf level
    // tuning
    double back_ctas_per_sm = 32.0;        // back-projector work split: CTAs per SM per launch
    int fwd_stage_rows = 0;                // forward: strips per staged image tile (0: no staging)
    bool graphs = true;                    // replay each tree epoch's iteration as a CUDA graph
    cudaStream_t prof_stream = nullptr;
    int device = 0;
    int num_sms = 148;
    std::string err;
    bool has_data = false;
    long long M = 0, N = 0;
    Buf buf[B_NBUF];
};

namespace {

wam_status fail(wam_ctx* c, wam_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

// Return the status of a failing CUDA call (WCK) or library step (WST).  The
// locals carry names no caller uses, so a macro argument can never see them.
#define WCK(ctx, call)                                                                              \
    do {                                                                                            \
        cudaError_t wck_err_local = (call);                                                         \
        if (wck_err_local != cudaSuccess)                                                           \
            return fail(ctx, WAM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(wck_err_local)); \
    } while (0)

#define WST(call)                                                    \
    do {                                                             \
        wam_status wst_status_local = (call);                        \
        if (wst_status_local != WAM_OK) return wst_status_local;     \
    } while (0)

// Grow-only device buffer.
wam_status ensure(wam_ctx* c, BufId id, size_t bytes, void** out)
{
    Buf& b = c->buf[id];
    if (b.bytes < bytes) {
        if (b.p) cudaFree(b.p);
        b.p = nullptr;
        b.bytes = 0;
        cudaError_t e = cudaMalloc(&b.p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(c, WAM_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
        }
        b.bytes = bytes;
    }
    *out = b.p;
    return WAM_OK;
}

template <typename P>
wam_status ensure_t(wam_ctx* c, BufId id, size_t count, P** out)
{
    void* p = nullptr;
    WST(ensure(c, id, count * sizeof(P), &p));
    *out = static_cast<P*>(p);
    return WAM_OK;
}

// the per-ray cost constant in the form the forward of type T reads
template <typename T>
const typename CostTerm<T>::type* dterm_buf(const wam_ctx* c)
{
    return static_cast<const typename CostTerm<T>::type*>(c->buf[sizeof(T) == 4 ? B_DTERM2 : B_DTERM].p);
}

// Elements of the strip walk's two apron-padded image (2-D) or volume
// (cone beam) copies.
size_t pad_elems(const wam_ctx* c)
{
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR)
        return 2 * (size_t)(c->g.nx + 2) * (size_t)(c->g.ny + 2) * (size_t)(c->g.nz + 2);
    // row-major copy (ny + 2 rows) and transposed copy (nx + 2 rows), rows at 16-byte strides
    return (size_t)pad_row(c->g.nx) * (c->g.ny + 2) + (size_t)pad_row(c->g.ny) * (c->g.nx + 2);
}

// --- run state ---------------------------------------------------------------
double eff_clamp(const wam_schedule* sc) { return sc->dmax_clamp > 0 ? sc->dmax_clamp : 30.0; }

int eff_dims(const wam_ctx* c, const wam_schedule* sc)
{
    return c->g.kind == WAM_CONE3D_FLAT_CIRCULAR ? sc->dims : 2;
}

void record_run(wam_ctx* c, const wam_schedule* sc, int iters, int expansions)
{
    RunRecord& r = c->last;
    r = RunRecord{};
    r.valid = true;
    r.levels = sc->full_am ? 0 : sc->levels;
    r.dims = eff_dims(c, sc);
    r.zsum = sc->zsum_criterion;
    r.precision = sc->precision;
    r.full_am = sc->full_am;
    r.clamp = eff_clamp(sc);
    r.expand_at.assign(sc->expand_at, sc->expand_at + sc->n_expand);
    r.tau.assign(sc->tau, sc->tau + sc->n_expand);
    r.iters_done = iters;
    r.expansions_done = expansions;
    r.n_subsets = std::max(1, sc->n_subsets);
    r.nonneg = sc->nonneg != 0;
    r.lambda = sc->lambda;
    r.tuning = c->back_ctas_per_sm;
    c->pending = RunRecord{};
}

// A schedule may continue the pending state when it ran the same method and
// the same expansions up to the iterations done.
wam_status check_resume(wam_ctx* c, const wam_schedule* sc)
{
    const RunRecord& r = c->pending;
    if (!r.valid) return WAM_OK;
    const int L = sc->full_am ? 0 : sc->levels;
    if (L != r.levels || sc->full_am != r.full_am || sc->precision != r.precision || eff_dims(c, sc) != r.dims ||
        sc->zsum_criterion != r.zsum || eff_clamp(sc) != r.clamp || std::max(1, sc->n_subsets) != r.n_subsets ||
        (sc->nonneg != 0) != (r.nonneg != 0) || sc->lambda != r.lambda)
        return fail(c, WAM_ERR_STATE, "resume: the schedule's method differs from the checkpoint's");
    if (sc->n_iters < r.iters_done) return fail(c, WAM_ERR_STATE, "resume: n_iters is below the iterations done");
    if (L > 0) {
        if (sc->n_expand < r.expansions_done) return fail(c, WAM_ERR_STATE, "resume: fewer expansions than done");
        for (int k = 0; k < r.expansions_done; ++k)
            if (sc->expand_at[k] != r.expand_at[k] || sc->tau[k] != r.tau[k])
                return fail(c, WAM_ERR_STATE, "resume: the expansions done differ from the schedule's");
        if (sc->n_expand > r.expansions_done && sc->expand_at[r.expansions_done] <= r.iters_done)
            return fail(c, WAM_ERR_STATE, "resume: the schedule expands at or before the iterations done");
    }
    return WAM_OK;
}

// --- profiling ---------------------------------------------------------------
cudaEvent_t take_event(wam_ctx* c)
{
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

struct ProfScope {
    wam_ctx* c;
    int k;
    cudaStream_t st;
    cudaEvent_t a = nullptr;
    ProfScope(wam_ctx* c_, int k_, cudaStream_t st_) : c(c_), k(k_), st(st_)
    {
        if (c->prof) {
            a = take_event(c);
            if (a) cudaEventRecord(a, st);
        }
    }
    ~ProfScope()
    {
        if (!c->prof || !a) return;
        cudaEvent_t b = take_event(c);
        if (!b) {
            c->ev_pool.push_back(a);
            return;
        }
        cudaEventRecord(b, st);
        c->pend.push_back({k, a, b});
        c->stats.launches[k] += 1;
        c->prof_stream = st;
    }
};

unsigned long long* work_ptr(wam_ctx* c, int k) { return c->prof_work && c->dwork ? c->dwork + k : nullptr; }

wam_status prof_resolve(wam_ctx* c)
{
    if (c->pend.empty() && !c->dwork) return WAM_OK;
    WCK(c, cudaStreamSynchronize(c->prof_stream));
    for (auto& p : c->pend) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) c->stats.ms[p.k] += ms;
        else cudaGetLastError();
        c->ev_pool.push_back(p.a);
        c->ev_pool.push_back(p.b);
    }
    c->pend.clear();
    if (c->dwork) {
        unsigned long long h[WAM_NKERNEL];
        WCK(c, cudaMemcpy(h, c->dwork, sizeof(h), cudaMemcpyDeviceToHost));
        WCK(c, cudaMemset(c->dwork, 0, sizeof(h)));
        for (int k = 0; k < WAM_NKERNEL; ++k) c->stats.work[k] += h[k];
    }
    return WAM_OK;
}

#define PROF(K) ProfScope prof_scope_##K(c, K, st)

template <typename T>
wam_status make_geom(wam_ctx* c, Geom<T>* g)
{
    const wam_geometry& w = c->g;
    g->kind = w.kind;
    g->stage_rows = c->fwd_stage_rows;
    g->nx = w.nx;
    g->ny = w.ny;
    g->V = w.n_views;
    g->B = w.n_bins;
    g->vx = (T)w.vx;
    g->vy = (T)w.vy;
    g->X0 = (T)(-0.5 * w.nx * w.vx);
    g->Y0 = (T)(-0.5 * w.ny * w.vy);
    g->ivx = (T)(1.0 / w.vx);
    g->ivy = (T)(1.0 / w.vy);
    g->pitch = (T)w.bin_pitch;
    g->ucen = (T)(0.5 * (w.n_bins - 1));
    g->sod = (T)w.sod;
    g->sdd = (T)w.sdd;
    T* cs = nullptr;
    WST(ensure_t(c, sizeof(T) == 4 ? B_CS32 : B_CS64, 2 * (size_t)w.n_views, &cs));
    g->cs = cs;
    return WAM_OK;
}

wam_status upload_views(wam_ctx* c)
{
    const wam_geometry& w = c->g;
    std::vector<double> cs64(2 * (size_t)w.n_views);
    std::vector<float> cs32(cs64.size());
    for (int k = 0; k < w.n_views; ++k) {
        const double th = w.angle0 + k * (w.angle_span / w.n_views);
        cs64[2 * k] = std::cos(th);
        cs64[2 * k + 1] = std::sin(th);
        cs32[2 * k] = (float)cs64[2 * k];
        cs32[2 * k + 1] = (float)cs64[2 * k + 1];
    }
    double* d64 = nullptr;
    float* d32 = nullptr;
    WST(ensure_t(c, B_CS64, cs64.size(), &d64));
    WST(ensure_t(c, B_CS32, cs32.size(), &d32));
    WCK(c, cudaMemcpy(d64, cs64.data(), cs64.size() * sizeof(double), cudaMemcpyHostToDevice));
    WCK(c, cudaMemcpy(d32, cs32.data(), cs32.size() * sizeof(float), cudaMemcpyHostToDevice));
    return WAM_OK;
}

wam_status make_layout(wam_ctx* c, int L, Layout* lay)
{
    const wam_geometry& w = c->g;
    if (L < 0 || L > WAM_MAX_LEVELS) return fail(c, WAM_ERR_ARG, "levels must be in 0..8");
    if (w.nx % (1 << L) || w.ny % (1 << L))
        return fail(c, WAM_ERR_ARG, "nx and ny must be divisible by 2^levels");
    if ((w.nx >> 1) > 65535 || (w.ny >> 1) > 65535) return fail(c, WAM_ERR_ARG, "image too large");
    std::memset(lay, 0, sizeof(*lay));
    lay->L = L;
    lay->nx = w.nx;
    lay->ny = w.ny;
    for (int l = 0; l <= L; ++l) {
        lay->gw[l] = w.nx >> l;
        lay->gh[l] = w.ny >> l;
    }
    long long off = (long long)lay->gw[L] * lay->gh[L];
    long long moff = 0;
    for (int l = L; l >= 1; --l) {
        lay->coff[l] = off;
        off += 3LL * lay->gw[l] * lay->gh[l];
        lay->moff[l] = moff;
        moff += (long long)lay->gw[l] * lay->gh[l];
    }
    lay->mask_bytes = moff;
    return WAM_OK;
}

// --- back-projection work plan ------------------------------------------------

struct ListInfo {
    int level, has_approx, has_details, n;
    const uint32_t* items;
    int gw;
    int quad = 0;
};

// Split every list into view ranges so that the grid holds about
// back_ctas_per_sm 256-thread CTAs per SM (a tuning value, default 32) with
// similar work (chord evaluations) each.
template <typename T>
wam_status plan_segments(wam_ctx* c, const std::vector<ListInfo>& lists, SegTable* tab, T** part_out, int nv = 0)
{
    const wam_geometry& w = c->g;
    const int V = nv > 0 ? nv : w.n_views;     // views of the scan (or view subset) back-projected
    std::memset(tab, 0, sizeof(*tab));
    const double mag = (w.kind == WAM_FAN2D_FLAT) ? 1.2 * w.sdd / w.sod : 1.0;
    const double diag = std::sqrt(w.vx * w.vx + w.vy * w.vy);
    std::vector<double> cost(lists.size());
    double total = 0.0;
    for (size_t i = 0; i < lists.size(); ++i) {
        const double shadow = (double)(1 << lists[i].level) * diag * mag / w.bin_pitch + 1.0;
        cost[i] = shadow * ((lists[i].has_details || lists[i].quad) ? 3.0 : 1.0);
        total += (double)lists[i].n * V * cost[i];
    }
    const double target_ctas = (double)c->num_sms * c->back_ctas_per_sm;
    const double per_cta = std::max(total / target_ctas, 1.0);
    const int max_chunks = std::max(1, V / kViewLanes);
    int cta = 0, items = 0;
    long long part = 0;
    for (size_t i = 0; i < lists.size(); ++i) {
        const ListInfo& li = lists[i];
        if (li.n == 0) continue;
        if (tab->n >= kMaxSegs) return fail(c, WAM_ERR_ARG, "too many segments");
        Segment& s = tab->s[tab->n++];
        s.level = li.level;
        s.has_approx = li.has_approx;
        s.has_details = li.has_details;
        s.quad = li.quad;
        s.n_items = li.n;
        s.items = li.items;
        s.gw = li.gw;
        const double full = (double)kItemsPerCta * V * cost[i];
        int chunks = (int)std::ceil(full / per_cta);
        chunks = std::max(1, std::min(chunks, max_chunks));
        // views per chunk a multiple of the CTA's view lanes, so that its warps
        // get equal view counts and meet at the final barrier together
        s.vpc = (V + chunks - 1) / chunks;
        s.vpc = std::min(V, (s.vpc + kViewLanes - 1) / kViewLanes * kViewLanes);
        s.n_chunks = (V + s.vpc - 1) / s.vpc;
        s.tiles = (li.n + kItemsPerCta - 1) / kItemsPerCta;
        s.cta_begin = cta;
        s.item_begin = items;
        s.n_slots = li.quad ? 4 : li.has_approx + 6 * li.has_details;
        s.part_off = part;
        cta += s.tiles * s.n_chunks;
        items += li.n;
        part += (long long)s.n_slots * s.n_chunks * li.n;
    }
    tab->total_ctas = cta;
    tab->total_items = items;
    return ensure_t(c, B_PART, (size_t)std::max<long long>(part, 1), part_out);
}

// Per ray (s/dx, -c/dy, 1/dx, ry/dy), ry = vy / vx: the reciprocal unit
// direction (its y part times the pixel's aspect ratio, the back-projector
// measuring lengths in units of a block's half-width) and its products with
// the view's sin and -cos, computed in FP64 on the host once
// per context and precision.  Every ray is taken in the orientation with
// dx >= 0 (a line's two orientations cross the same voxels), so the
// back-projector's first x half along the travel is always the lower one.
template <typename T>
wam_status dir_table(wam_ctx* c, const void** out, const std::vector<int>* order = nullptr)
{
    const BufId id = order ? (sizeof(T) == 4 ? B_DIRP32 : B_DIRP64) : (sizeof(T) == 4 ? B_DIR32 : B_DIR64);
    const wam_geometry& w = c->g;
    const size_t n = (size_t)w.n_views * w.n_bins;
    if (!order && c->buf[id].p && c->buf[id].bytes >= n * 4 * sizeof(T)) {
        *out = c->buf[id].p;
        return WAM_OK;
    }
    std::vector<T> h(4 * n);
    const double tiny = sizeof(T) == 4 ? 1e-30 : 1e-200;
    auto rcp = [tiny](double d) {
        double a = std::fabs(d);
        a = a < tiny ? tiny : a;
        return std::signbit(d) ? -1.0 / a : 1.0 / a;
    };
    const double ry = w.vy / w.vx;                    // the pixel's aspect ratio
    for (int k = 0; k < w.n_views; ++k) {
        const int view = order ? (*order)[k] : k;     // row k of the table holds this view
        const double th = w.angle0 + view * (w.angle_span / w.n_views);
        const double cs = std::cos(th), sn = std::sin(th);
        for (int b = 0; b < w.n_bins; ++b) {
            double dx = cs, dy = sn;
            if (w.kind == WAM_FAN2D_FLAT) {
                const double ub = (b - 0.5 * (w.n_bins - 1)) * w.bin_pitch;
                const double rn = 1.0 / std::sqrt(w.sdd * w.sdd + ub * ub);
                dx = (-w.sdd * cs - ub * sn) * rn;
                dy = (-w.sdd * sn + ub * cs) * rn;
            }
            if (std::signbit(dx)) {
                dx = -dx;
                dy = -dy;
            }
            const double ix = rcp(dx), iy = rcp(dy);
            T* e = &h[4 * ((size_t)k * w.n_bins + b)];
            e[0] = (T)(sn * ix);
            e[1] = (T)(-cs * iy);
            e[2] = (T)ix;
            e[3] = (T)(ry * iy);
        }
    }
    T* d = nullptr;
    WST(ensure_t(c, id, 4 * n, &d));
    WCK(c, cudaMemcpy(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = d;
    return WAM_OK;
}

// Pixel basis (Omega = I): items are 2x2 pixel quads when both sides are
// even (one shadow per quad, four chords per ray), else single pixels.
template <typename T>
wam_status plan_pixels(wam_ctx* c, SegTable* tab, T** part, int nv = 0)
{
    const int nx = c->g.nx, ny = c->g.ny;
    std::vector<ListInfo> lists;
    if (nx % 2 == 0 && ny % 2 == 0) {
        ListInfo li{1, 0, 0, (nx / 2) * (ny / 2), nullptr, nx / 2};
        li.quad = 1;
        lists.push_back(li);
    } else {
        lists.push_back({0, 1, 0, (int)c->N, nullptr, nx});
    }
    return plan_segments<T>(c, lists, tab, part, nv);
}

// Rebuild leaf map, block lists and work plan from the mask (device); reads
// the list lengths back (one small synchronous copy).
template <typename T>
wam_status plan_tree(wam_ctx* c, const Layout& lay, const uint8_t* mask, uint8_t* leaf, SegTable* tab, T** part,
                     cudaStream_t st, int nv = 0)
{
    PROF(WAM_K_TREE);
    WCK(c, launch_leafmap(lay, mask, leaf, st));
    const int L = lay.L;
    const long long stride = (long long)lay.gw[1] * lay.gh[1];
    uint32_t* lists = nullptr;
    int* counts = nullptr;
    WST(ensure_t(c, B_LISTS, (size_t)stride * (L + 1), &lists));
    const int maxc = compact_chunks(lay);
    WST(ensure_t(c, B_COUNTS, (size_t)(L + 1) * (1 + maxc), &counts));
    WCK(c, launch_compact(lay, mask, lists, stride, counts, counts + (L + 1), st));
    std::vector<int> h(L + 1);
    WCK(c, cudaMemcpyAsync(h.data(), counts, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, st));
    WCK(c, cudaStreamSynchronize(st));
    // leaves: each expanded block turns one leaf into four
    long long leaves = (long long)lay.gw[L] * lay.gh[L];
    for (int k = 1; k <= L; ++k) leaves += 3LL * h[k];
    c->last_leaves = leaves;
    // h[k] counts the expanded blocks of level L - k + 1, whose children are
    // leaves of level L - k (or finer)
    c->last_lmin = L;
    for (int k = 1; k <= L; ++k)
        if (h[k] > 0) c->last_lmin = L - k;
    std::vector<ListInfo> li;
    li.push_back({L, 1, 0, h[0], lists, lay.gw[L]});
    li.push_back({L, 1, 1, h[1], lists + stride, lay.gw[L]});
    for (int k = 1; k < L; ++k) li.push_back({L - k, 0, 1, h[k + 1], lists + stride * (k + 1), lay.gw[L - k]});
    return plan_segments<T>(c, li, tab, part, nv);
}

template <typename T>
wam_status compute_z0(wam_ctx* c, const Geom<T>& g, const Layout& lay, const uint8_t* leaf, double* z0,
                      cudaStream_t st)
{
    const int np = forward_parts(g.V, g.B);
    double* part = nullptr;
    WST(ensure_t(c, B_COSTPART, (size_t)np, &part));
    WCK(c, launch_z0(g, lay, leaf, part, st));
    WCK(c, launch_max_final(part, np, z0, st));
    return WAM_OK;
}

}  // namespace

// Shared with the non-allocating back-projector (wam_static.cu), so both entry
// points accept the same 2-D geometries.
wam_status wam::check_geometry(const wam_geometry* g, std::string* why)
{
    if (!g) { *why = "geometry is NULL"; return WAM_ERR_ARG; }
    if (g->kind == WAM_CONE3D_FLAT_CIRCULAR) {
        if (g->nx <= 0 || g->ny <= 0 || g->nz <= 0 || g->n_views <= 0 || g->n_bins <= 0 || g->n_rows <= 0) {
            *why = "sizes must be positive"; return WAM_ERR_ARG;
        }
        if (!(g->vx > 0) || !(g->vy > 0) || !(g->vz > 0) || !(g->bin_pitch > 0) || !(g->row_pitch > 0)) {
            *why = "voxel sizes and pitches must be > 0"; return WAM_ERR_ARG;
        }
        if (g->nx > 2046 || g->ny > 2046 || g->nz > 1022) { *why = "volume too large"; return WAM_ERR_ARG; }
        if ((long long)g->nx * g->ny * g->nz > (1LL << 31) - 1 ||
            (long long)g->n_views * g->n_rows * g->n_bins > (1LL << 31) - 1) {
            *why = "problem too large for 32-bit indices"; return WAM_ERR_ARG;
        }
        const double r = 0.5 * std::hypot(g->nx * g->vx, g->ny * g->vy);
        if (!(g->sod > r) || !(g->sdd - g->sod > r)) {
            *why = "cone beam: source and detector must lie outside the volume's circumradius"; return WAM_ERR_ARG;
        }
        return WAM_OK;
    }
    if (g->kind != WAM_PARALLEL2D && g->kind != WAM_FAN2D_FLAT) { *why = "unsupported geometry kind"; return WAM_ERR_ARG; }
    if (g->nx <= 0 || g->ny <= 0 || g->n_views <= 0 || g->n_bins <= 0) { *why = "sizes must be positive"; return WAM_ERR_ARG; }
    if (g->nz > 1 || g->n_rows > 1) { *why = "2-D geometry expected (nz = n_rows = 1)"; return WAM_ERR_ARG; }
    if (!(g->vx > 0) || !(g->vy > 0) || !(g->bin_pitch > 0)) { *why = "voxel size and bin pitch must be > 0"; return WAM_ERR_ARG; }
    if (!std::isfinite(g->angle0) || !std::isfinite(g->angle_span)) { *why = "angles must be finite"; return WAM_ERR_ARG; }
    if ((long long)g->nx * g->ny > (1LL << 31) - 1 || (long long)g->n_views * g->n_bins > (1LL << 31) - 1) {
        *why = "problem too large for 32-bit indices"; return WAM_ERR_ARG;
    }
    if (g->nx > 65536 || g->ny > 65536) { *why = "image side above 65536"; return WAM_ERR_ARG; }
    if (g->kind == WAM_FAN2D_FLAT) {
        const double r = 0.5 * std::hypot(g->nx * g->vx, g->ny * g->vy);
        if (!(g->sod > r)) { *why = "fan beam: SOD must exceed the image circumradius"; return WAM_ERR_ARG; }
        if (!(g->sdd - g->sod > r)) { *why = "fan beam: the detector must lie outside the image"; return WAM_ERR_ARG; }
    }
    return WAM_OK;
}

namespace {

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }



// ---------------------------------------------------------------------------
// the reconstruction driver
// ---------------------------------------------------------------------------
// One reconstruction split into phases.  iteration() and final_cost() only
// launch kernels on the given stream (no allocation, no host wait), so a
// batch of runs can capture them in a CUDA graph; expand() reads the new
// block-list lengths back to the host.
template <typename T>
struct Run {
    wam_ctx* c = nullptr;
    const wam_schedule* sc = nullptr;
    int L = 0, J = 0, np = 0, npc = 0;   // partial buffer size; cost partials of one forward
    int nl1 = 0;                // lam > 0: partials of the penalty after the forward's
    double clamp = 30.0;
    double lam = 0.0;           // L1 penalty on the detail coefficients (0: Algorithm 1 as stated)
    long long N = 0, M = 0;
    Layout lay{};
    Geom<T> g{};
    T *q = nullptr, *mu = nullptr, *mut = nullptr, *sino = nullptr, *part = nullptr;
    double *beta = nullptr, *bvec = nullptr, *costs = nullptr, *z0 = nullptr, *scratch = nullptr;
    double *tmpa = nullptr, *tmpb = nullptr, *gimg = nullptr, *cpart = nullptr;
    float* beta32 = nullptr;    // FP32 runs: the float copy of beta the forward synthesises from
    uint8_t *mask = nullptr, *mask2 = nullptr, *leaf = nullptr;
    int* counter = nullptr;
    const float *dsino = nullptr, *I0 = nullptr;
    const typename CostTerm<T>::type* dterm = nullptr;
    const void* dirt = nullptr;
    SegTable tab{};
    const uint8_t* fwd_leaf = nullptr;
    int fwd_lam = 0;
    std::vector<int> exp_at;
    size_t next_exp = 0;
    int j0 = 0;                 // first iteration to run (> 0 when resuming)
    // ordered subsets of views: the scan is held in subset-major view order
    // (subset s = views k with k mod S = s, rows sv0[s] .. sv0[s] + svn[s] - 1)
    int S = 1;
    std::vector<int> sv0, svn;
    std::vector<Geom<T>> gsub;  // each subset as a scan of its own
    Geom<T> gperm{};            // the whole scan in subset-major order
    const float *dP = nullptr, *I0P = nullptr;
    const typename CostTerm<T>::type* dtP = nullptr;
    const void* dirP = nullptr;
    double *bsub = nullptr, *z0sub = nullptr;   // per subset: b (Eq. 1.6 on its rays), Z0

    // How a2 walks the tree's image mu, which is constant on the leaves and
    // so on the cells of the finest leaf level lam: the strip walk over the
    // grid of those cells (exact for such an image), unless the tree is so
    // uneven that the leaves are fewer than a ninth of the cells.  A ray then
    // meets about 3 times fewer leaves than cells, which pays for the leaf
    // walk's dearer steps (a leaf-map read and a division per leaf).
    const uint8_t* pick_leaf()
    {
        fwd_lam = L > 0 ? c->last_lmin : 0;
        const long long cells = N >> (2 * fwd_lam);
        if (L > 0 && cells > 9 * c->last_leaves) {
            fwd_lam = 0;
            return leaf;
        }
        return nullptr;
    }

    wam_status setup(wam_ctx* ctx, const wam_schedule* sched, cudaStream_t st)
    {
        c = ctx;
        sc = sched;
        L = sc->full_am ? 0 : sc->levels;
        J = sc->n_iters;
        clamp = sc->dmax_clamp > 0 ? sc->dmax_clamp : 30.0;
        lam = sc->lambda;
        WST(make_layout(c, L, &lay));
        WST(make_geom<T>(c, &g));
        N = c->N;
        M = c->M;
        WST(ensure_t(c, B_Q, (size_t)M, &q));
        WST(ensure_t(c, B_MU, (size_t)N, &mu));
        WST(ensure_t(c, B_MUT, pad_elems(c), &mut));
        WST(ensure_t(c, B_BETA, (size_t)N, &beta));
        if (sizeof(T) == 4) WST(ensure_t(c, B_BETA32, (size_t)N, &beta32));
        WST(ensure_t(c, B_BVEC, (size_t)N, &bvec));
        WST(ensure_t(c, B_COSTS, (size_t)J + 1, &costs));
        WST(ensure_t(c, B_Z0, 1, &z0));
        WST(ensure_t(c, B_SCRATCH, 1024, &scratch));
        WST(ensure_t(c, B_TMPA, (size_t)N, &tmpa));
        WST(ensure_t(c, B_TMPB, (size_t)N, &tmpb));
        WST(ensure_t(c, B_GIMG, (size_t)N, &gimg));
        WST(ensure_t(c, B_COUNTER, 1, &counter));
        np = forward_parts(g.V, g.B);
        npc = forward_cost_parts(g.V, g.B);
        nl1 = lam > 0 ? l1_parts(lay) : 0;
        WST(ensure_t(c, B_COSTPART, (size_t)std::max(np, npc + nl1), &cpart));
        if (L > 0) {
            WST(ensure_t(c, B_MASK_A, (size_t)lay.mask_bytes, &mask));
            WST(ensure_t(c, B_MASK_B, (size_t)lay.mask_bytes, &mask2));
            WST(ensure_t(c, B_LEAF, (size_t)N, &leaf));
        }
        dsino = static_cast<const float*>(c->buf[B_D].p);
        I0 = static_cast<const float*>(c->buf[B_I0].p);
        dterm = dterm_buf<T>(c);
        WST(dir_table<T>(c, &dirt));

        // a0, Eq. 1.6: b = Phi^T d = Omega^T (H^T d) for every coefficient
        SegTable pix;
        WST(plan_pixels<T>(c, &pix, &part));
        const T* dT;
        if (sizeof(T) == sizeof(float)) {
            dT = reinterpret_cast<const T*>(dsino);
        } else {
            WST(ensure_t(c, B_SINO, (size_t)M, &sino));
            WCK(c, (launch_convert<float, double>(dsino, reinterpret_cast<double*>(sino), M, st)));
            dT = sino;
        }
        {
            PROF(WAM_K_BACKPROJECT);
            WCK(c, launch_backproject(g, pix, dT, dirt, part, work_ptr(c, WAM_K_BACKPROJECT), st));
        }
        {
            PROF(WAM_K_TREE);
            WCK(c, (launch_reduce_pixels<T, double>(pix, c->g.nx, N, part, gimg, st)));
            WCK(c, launch_haar(lay, gimg, bvec, 0, tmpa, tmpb, st));
        }
        // beta^(0) = 0; the tree holds the approximations only
        WCK(c, cudaMemsetAsync(beta, 0, N * sizeof(double), st));
        if (beta32) WCK(c, cudaMemsetAsync(beta32, 0, N * sizeof(float), st));
        WCK(c, cudaMemsetAsync(counter, 0, sizeof(int), st));
        if (L > 0) {
            WCK(c, cudaMemsetAsync(mask, 0, lay.mask_bytes, st));
            WST(plan_tree<T>(c, lay, mask, leaf, &tab, &part, st));
        } else {
            tab = pix;
        }
        {
            PROF(WAM_K_Z0);
            WST(compute_z0<T>(c, g, lay, leaf, z0, st));
        }
        fwd_leaf = pick_leaf();
        exp_at.assign(sc->n_expand > 0 ? sc->expand_at : nullptr,
                      sc->n_expand > 0 ? sc->expand_at + sc->n_expand : nullptr);
        next_exp = 0;
        j0 = 0;
        S = std::max(1, sc->n_subsets);
        if (S > 1) WST(setup_subsets(st));
        if (c->pending.valid) WST(load_pending(st));
        return WAM_OK;
    }

    // The views in subset-major order (cos/sin, direction table, d, I0, the
    // cost constants), each subset's b and the block plan for a subset's
    // view count; then the subsets' Z0.
    wam_status setup_subsets(cudaStream_t st)
    {
        const wam_geometry& w = c->g;
        const int V = w.n_views, B = w.n_bins;
        std::vector<int> perm;
        perm.reserve(V);
        sv0.assign(S, 0);
        svn.assign(S, 0);
        for (int ss = 0; ss < S; ++ss) {
            sv0[ss] = (int)perm.size();
            for (int k = ss; k < V; k += S) perm.push_back(k);
            svn[ss] = (int)perm.size() - sv0[ss];
        }
        int* dperm = nullptr;
        WST(ensure_t(c, B_PERM, (size_t)V, &dperm));
        WCK(c, cudaMemcpyAsync(dperm, perm.data(), V * sizeof(int), cudaMemcpyHostToDevice, st));
        std::vector<T> csh(2 * (size_t)V);
        for (int k = 0; k < V; ++k) {
            const double th = w.angle0 + perm[k] * (w.angle_span / V);
            csh[2 * k] = (T)std::cos(th);
            csh[2 * k + 1] = (T)std::sin(th);
        }
        T* csp = nullptr;
        WST(ensure_t(c, sizeof(T) == 4 ? B_CSP32 : B_CSP64, csh.size(), &csp));
        WCK(c, cudaMemcpyAsync(csp, csh.data(), csh.size() * sizeof(T), cudaMemcpyHostToDevice, st));
        float *dp = nullptr, *ip = nullptr;
        typename CostTerm<T>::type* dtp = nullptr;
        WST(ensure_t(c, B_DP, (size_t)M, &dp));
        WST(ensure_t(c, B_I0P, (size_t)M, &ip));
        WST(ensure_t(c, B_DTP, (size_t)M, &dtp));
        WCK(c, launch_permute_rows<float>(dsino, dp, dperm, V, B, st));
        WCK(c, launch_permute_rows<float>(I0, ip, dperm, V, B, st));
        WCK(c, launch_permute_rows<typename CostTerm<T>::type>(dterm, dtp, dperm, V, B, st));
        dP = dp;
        I0P = ip;
        dtP = dtp;
        WST(dir_table<T>(c, &dirP, &perm));
        gperm = g;
        gperm.cs = csp;
        gsub.assign(S, g);
        for (int ss = 0; ss < S; ++ss) {
            gsub[ss].V = svn[ss];
            gsub[ss].cs = csp + 2 * (size_t)sv0[ss];
        }
        // b_s = Phi_s^T d_s = Omega^T (H_s^T d_s) for every coefficient
        WST(ensure_t(c, B_BSUB, (size_t)S * N, &bsub));
        WST(ensure_t(c, B_Z0SUB, (size_t)S, &z0sub));
        const T* dTP;
        if (sizeof(T) == sizeof(float)) {
            dTP = reinterpret_cast<const T*>(dp);
        } else {
            T* sp = nullptr;
            WST(ensure_t(c, B_SINOP, (size_t)M, &sp));
            WCK(c, launch_permute_rows<T>(sino, sp, dperm, V, B, st));
            dTP = sp;
        }
        SegTable pix;
        T* ppart = nullptr;
        WST(plan_pixels<T>(c, &pix, &ppart, svn[0]));
        for (int ss = 0; ss < S; ++ss) {
            const size_t off = (size_t)sv0[ss] * B;
            {
                PROF(WAM_K_BACKPROJECT);
                WCK(c, launch_backproject(gsub[ss], pix, dTP + off, dir_rows(off), ppart,
                                          work_ptr(c, WAM_K_BACKPROJECT), st));
            }
            PROF(WAM_K_TREE);
            WCK(c, (launch_reduce_pixels<T, double>(pix, c->g.nx, N, ppart, gimg, st)));
            WCK(c, launch_haar(lay, gimg, bsub + (size_t)ss * N, 0, tmpa, tmpb, st));
        }
        if (L == 0) {
            WST(plan_pixels<T>(c, &tab, &part, svn[0]));
            PROF(WAM_K_Z0);
            for (int ss = 0; ss < S; ++ss) WST(compute_z0<T>(c, gsub[ss], lay, leaf, z0sub + ss, st));
            return WAM_OK;
        }
        return replan(st);
    }

    // direction-table rows from ray `off` of the subset-major table
    const void* dir_rows(size_t off) const
    {
        return static_cast<const void*>(static_cast<const T*>(dirP) + 4 * off);
    }

    // block plan, forward walk and Z0 (per subset) for the current tree
    wam_status replan(cudaStream_t st)
    {
        if (L > 0) {
            WST(plan_tree<T>(c, lay, mask, leaf, &tab, &part, st, S > 1 ? svn[0] : 0));
            fwd_leaf = pick_leaf();
        }
        PROF(WAM_K_Z0);
        if (S > 1) {
            for (int ss = 0; ss < S; ++ss) WST(compute_z0<T>(c, gsub[ss], lay, leaf, z0sub + ss, st));
        } else {
            WST(compute_z0<T>(c, g, lay, leaf, z0, st));                                  // a5
        }
        return WAM_OK;
    }

    // the coefficients the strip-walk forward synthesises its cells from
    const typename SynthCoef<T>::type* synth_src() const
    {
        return reinterpret_cast<const typename SynthCoef<T>::type*>(sizeof(T) == 4 ? (const void*)beta32
                                                                                   : (const void*)beta);
    }

    // a1 + a2 + a3 on a scan (the whole one or a subset): qhat into qq and,
    // with cp, the cost partials
    wam_status fwd(const Geom<T>& gg, const float* dd, const typename CostTerm<T>::type* dt, const float* ii, T* qq,
                   double* cp,
                   cudaStream_t st)
    {
        if (fwd_leaf) {
            {
                PROF(WAM_K_SYNTH);
                WCK(c, launch_synth(lay, leaf, beta, mu, st));
            }
            PROF(WAM_K_FORWARD);
            WCK(c, launch_forward(gg, mu, mut, fwd_leaf, 0, dd, dt, ii, qq, (T*)nullptr, (T*)nullptr, cp,
                                  work_ptr(c, WAM_K_FORWARD), st));
        } else {
            PROF(WAM_K_FORWARD);
            WCK(c, launch_forward_tree(gg, lay, L > 0 ? leaf : nullptr, synth_src(), fwd_lam, mut, dd, dt, ii, qq,
                                       (T*)nullptr, (T*)nullptr, cp, work_ptr(c, WAM_K_FORWARD), st));
        }
        return WAM_OK;
    }

    // one iteration with ordered subsets: the full cost at beta^(j) (its qhat
    // rows of subset 0 serve the first sub-iteration), then per subset a2-a4
    // on its rays and a6 with its b and Z0
    wam_status iteration_os(int j, cudaStream_t st)
    {
        const int B = c->g.n_bins;
        WST(fwd(gperm, dP, dtP, I0P, q, cpart, st));
        {
            PROF(WAM_K_FORWARD);
            WCK(c, launch_sum_final(cpart, npc, costs + j, st));
        }
        for (int ss = 0; ss < S; ++ss) {
            const size_t off = (size_t)sv0[ss] * B;
            if (ss > 0) WST(fwd(gsub[ss], dP + off, dtP + off, I0P + off, q + off, nullptr, st));
            {
                PROF(WAM_K_BACKPROJECT);
                WCK(c, launch_backproject(gsub[ss], tab, q + off, dir_rows(off), part,
                                          work_ptr(c, WAM_K_BACKPROJECT), st));
            }
            PROF(WAM_K_UPDATE);
            WCK(c, launch_update(tab, lay, part, bsub + (size_t)ss * N, z0sub + ss, clamp, beta, beta32, sc->nonneg, 0.0,
                                 work_ptr(c, WAM_K_UPDATE), st));
        }
        return WAM_OK;
    }

    // continue from the state of wam_resume: beta, the tree (its block lists
    // and Z0 rebuilt), the cost history so far and the expansions done
    wam_status load_pending(cudaStream_t st)
    {
        const RunRecord& r = c->pending;
        if (r.beta.size() != (size_t)N || r.hist.size() != (size_t)r.iters_done + 1 ||
            r.mask.size() != (L > 0 ? (size_t)lay.mask_bytes : 0))
            return fail(c, WAM_ERR_STATE, "resume: the checkpoint's sizes do not fit this schedule");
        WCK(c, cudaMemcpyAsync(beta, r.beta.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
        if (beta32) WCK(c, (launch_convert<double, float>(beta, beta32, N, st)));
        WCK(c, cudaMemcpyAsync(costs, r.hist.data(), r.hist.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        if (L > 0) {
            WCK(c, cudaMemcpyAsync(mask, r.mask.data(), lay.mask_bytes, cudaMemcpyHostToDevice, st));
            WST(replan(st));
        }
        next_exp = (size_t)r.expansions_done;
        j0 = r.iters_done;
        return WAM_OK;
    }

    // a1 - a6 of iteration j; with use_counter the cost goes to
    // costs[*counter] (then counter + 1) instead of costs[j]
    wam_status iteration(int j, cudaStream_t st, bool use_counter)
    {
        if (S > 1) return iteration_os(j, st);
        if (fwd_leaf) {
            PROF(WAM_K_SYNTH);
            WCK(c, launch_synth(lay, leaf, beta, mu, st));                                  // a1
        }
        {
            PROF(WAM_K_FORWARD);                                                            // (a1,) a2, a3
            if (fwd_leaf)
                WCK(c, launch_forward(g, mu, mut, fwd_leaf, 0, dsino, dterm, I0, q, (T*)nullptr, (T*)nullptr, cpart,
                                      work_ptr(c, WAM_K_FORWARD), st));
            else
                WCK(c, launch_forward_tree(g, lay, L > 0 ? leaf : nullptr, synth_src(), fwd_lam, mut, dsino, dterm, I0, q,
                                           (T*)nullptr, (T*)nullptr, cpart, work_ptr(c, WAM_K_FORWARD), st));
            WST(cost_out(costs + j, use_counter, st));
        }
        {
            PROF(WAM_K_BACKPROJECT);                                                        // a4
            WCK(c, launch_backproject(g, tab, q, dirt, part, work_ptr(c, WAM_K_BACKPROJECT), st));
        }
        {
            PROF(WAM_K_UPDATE);                                                             // a6
            WCK(c, launch_update(tab, lay, part, bvec, z0, clamp, beta, beta32, sc->nonneg, lam, work_ptr(c, WAM_K_UPDATE),
                                 st));
        }
        return WAM_OK;
    }

    bool expands_after(int j) const
    {
        return L > 0 && next_exp < exp_at.size() && exp_at[next_exp] == j + 1;
    }

    // a7 (+ new block lists and a5); call when expands_after(j)
    wam_status expand(cudaStream_t st)
    {
        const double tau = sc->tau[next_exp];
        ++next_exp;
        {
            PROF(WAM_K_TREE);
            WCK(c, launch_synth(lay, leaf, beta, mu, st));
            WCK(c, cudaMemcpyAsync(mask2, mask, lay.mask_bytes, cudaMemcpyDeviceToDevice, st));
            WCK(c, launch_expand<T>(lay, mu, tau, leaf, mask2, scratch, st));
        }
        std::swap(mask, mask2);
        std::swap(c->buf[B_MASK_A], c->buf[B_MASK_B]);
        return replan(st);
    }

    // the image out (FP64 synthesis) and the last cost, on the forward path
    // of the iterations (so that the history is that of one run, cut or not)
    wam_status final_cost(cudaStream_t st, bool use_counter)
    {
        {
            PROF(WAM_K_SYNTH);
            WCK(c, launch_synth(lay, leaf, beta, mu, st));
        }
        {
            PROF(WAM_K_FORWARD);
            if (fwd_leaf)
                WCK(c, launch_forward(g, mu, mut, fwd_leaf, 0, dsino, dterm, I0, q, (T*)nullptr, (T*)nullptr, cpart,
                                      work_ptr(c, WAM_K_FORWARD), st));
            else
                WCK(c, launch_forward_tree(g, lay, L > 0 ? leaf : nullptr, synth_src(), fwd_lam, mut, dsino, dterm,
                                           I0, q, (T*)nullptr, (T*)nullptr, cpart, work_ptr(c, WAM_K_FORWARD), st));
            WST(cost_out(costs + J, use_counter, st));
        }
        return WAM_OK;
    }

    // the forward's cost partials (and, with lam > 0, the penalty of the same
    // beta) summed into `at`, or into costs[*counter] with use_counter
    wam_status cost_out(double* at, bool use_counter, cudaStream_t st)
    {
        if (nl1 > 0) WCK(c, launch_l1_sum(lay, beta, lam, cpart + npc, st));
        if (use_counter) WCK(c, launch_sum_at(cpart, npc + nl1, costs, counter, st));
        else WCK(c, launch_sum_final(cpart, npc + nl1, at, st));
        return WAM_OK;
    }

    // copies results out (on st) and returns the cost history on the host
    wam_status copy_out(void* mu_out, double* hist, unsigned char* mask_out, int on_device, std::vector<double>* h,
                        cudaStream_t st)
    {
        const cudaMemcpyKind k2 = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (mu_out) WCK(c, cudaMemcpyAsync(mu_out, mu, N * sizeof(T), k2, st));
        if (mask_out && L > 0) WCK(c, cudaMemcpyAsync(mask_out, mask, lay.mask_bytes, k2, st));
        h->resize(J + 1);
        WCK(c, cudaMemcpyAsync(h->data(), costs, (J + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (hist) WCK(c, cudaMemcpyAsync(hist, costs, (J + 1) * sizeof(double), k2, st));
        return WAM_OK;
    }

    wam_status monotone(const std::vector<double>& h) const
    {
        const double band = sizeof(T) == sizeof(float) ? 1e-6 : 1e-11;
        for (int j = 0; j < J; ++j)
            if (h[j + 1] > h[j] + band * std::fabs(h[j])) return WAM_WARN_NONMONOTONE;
        return WAM_OK;
    }
};

// A staged forward whose shared-memory copy did not complete within its wait
// budget raised the device's stage-error word: the run's results are invalid.
// Reads and clears the word (the stream has been synchronised).
wam_status check_stage_error(wam_ctx* c)
{
    int* w = stage_error_word();
    if (!w) return WAM_OK;
    int v = 0;
    WCK(c, cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v == 0) return WAM_OK;
    WCK(c, cudaMemset(w, 0, sizeof(int)));
    return fail(c, WAM_ERR_TIMEOUT, "a staged image copy of the forward projector did not complete in time");
}

// Iterations j0 .. J-1 of a run by tree epochs: the iterations between two
// expansions launch the same kernels (the cost slot comes from the device
// counter), so one of them is captured in a CUDA graph and the graph is
// replayed for the rest of the epoch.  Capture needs a stream other than the
// legacy default one: the work runs on a private stream ordered after st, and
// st waits for it at the end.
template <typename T>
wam_status iterate_graphs(wam_ctx* c, Run<T>& run, cudaStream_t st)
{
    cudaStream_t gs = nullptr;
    cudaEvent_t ev = nullptr;
    auto done = [&](wam_status s) {
        if (gs && ev && cudaEventRecord(ev, gs) == cudaSuccess) cudaStreamWaitEvent(st, ev, 0);
        if (gs) cudaStreamDestroy(gs);
        if (ev) cudaEventDestroy(ev);
        if (s != WAM_OK) cudaGetLastError();
        return s;
    };
    if (cudaStreamCreateWithFlags(&gs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess || cudaEventRecord(ev, st) != cudaSuccess ||
        cudaStreamWaitEvent(gs, ev, 0) != cudaSuccess)
        return done(fail(c, WAM_ERR_CUDA, "stream or event creation failed"));
    const int j0 = run.j0;
    if (cudaMemcpyAsync(run.counter, &j0, sizeof(int), cudaMemcpyHostToDevice, gs) != cudaSuccess)
        return done(fail(c, WAM_ERR_CUDA, "counter copy failed"));
    int j = j0;
    while (j < run.J) {
        int e = run.J;
        if (run.L > 0 && run.next_exp < run.exp_at.size()) e = std::min(run.J, run.exp_at[run.next_exp]);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        const unsigned long long n0 = kernel_launches();
        if (cudaStreamBeginCapture(gs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
            return done(fail(c, WAM_ERR_CUDA, "stream capture could not start"));
        wam_status s = run.iteration(j, gs, true);
        const cudaError_t ec = cudaStreamEndCapture(gs, &graph);
        if (s != WAM_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return done(s != WAM_OK ? s : fail(c, WAM_ERR_CUDA, "stream capture failed"));
        }
        if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
            cudaGraphDestroy(graph);
            return done(fail(c, WAM_ERR_CUDA, "graph instantiation failed"));
        }
        const unsigned long long per_iter = kernel_launches() - n0;
        for (int k = j; k < e && s == WAM_OK; ++k)
            if (cudaGraphLaunch(exec, gs) != cudaSuccess) s = fail(c, WAM_ERR_CUDA, "graph launch failed");
        add_launches(per_iter * (unsigned long long)(e - j - 1));
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        if (s != WAM_OK) return done(s);
        j = e;
        if (run.expands_after(j - 1)) {
            s = run.expand(gs);
            if (s != WAM_OK) return done(s);
        }
    }
    return done(WAM_OK);
}

template <typename T>
wam_status reconstruct_impl(wam_ctx* c, const wam_schedule* sc, void* mu_out, double* hist, unsigned char* mask_out,
                            int on_device, cudaStream_t st)
{
    WST(check_resume(c, sc));
    c->last.valid = false;
    Run<T> run;
    WST(run.setup(c, sc, st));
    if (c->graphs && !c->prof && !c->prof_work && run.S == 1 && run.j0 < run.J) {
        WST(iterate_graphs(c, run, st));
    } else {
        for (int j = run.j0; j < run.J; ++j) {
            WST(run.iteration(j, st, false));
            if (run.expands_after(j)) WST(run.expand(st));
        }
    }
    WST(run.final_cost(st, false));
    std::vector<double> h;
    WST(run.copy_out(mu_out, hist, mask_out, on_device, &h, st));
    WCK(c, cudaStreamSynchronize(st));
    WST(check_stage_error(c));
    if (c->prof || c->prof_work) WST(prof_resolve(c));
    record_run(c, sc, run.J, (int)run.next_exp);
    return run.monotone(h);
}

template <typename T>
wam_status project_impl(wam_ctx* c, const T* mu, T* p, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!mu || !p) return fail(c, WAM_ERR_ARG, "null pointer");
    Geom<T> g;
    WST(make_geom<T>(c, &g));
    T* mut = nullptr;
    WST(ensure_t(c, B_MUT, pad_elems(c), &mut));
    WCK(c, launch_forward<T>(g, mu, mut, nullptr, 0, nullptr, nullptr, nullptr, nullptr, p, nullptr, nullptr, nullptr,
                             as_stream(stream)));
    return WAM_OK;
}

template <typename T>
wam_status backproject_impl(wam_ctx* c, const T* s, T* out, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!s || !out) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Geom<T> g;
        WST(make_geom<T>(c, &g));
        SegTable tab;
        T* part = nullptr;
        WST(plan_pixels<T>(c, &tab, &part));
        cudaStream_t st = as_stream(stream);
        const void* dirt = nullptr;
        WST(dir_table<T>(c, &dirt));
        WCK(c, launch_backproject(g, tab, s, dirt, part, nullptr, st));
        WCK(c, (launch_reduce_pixels<T, T>(tab, c->g.nx, c->N, part, out, st)));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status leaf_from_masks(wam_ctx* c, const Layout& lay, const unsigned char* masks, uint8_t** leaf,
                                  cudaStream_t st)
{
    *leaf = nullptr;
    if (lay.L == 0 || !masks) return WAM_OK;
    WST(ensure_t(c, B_LEAF, (size_t)c->N, leaf));
    WCK(c, launch_leafmap(lay, masks, *leaf, st));
    return WAM_OK;
}

template <typename T>
wam_status forward_impl(wam_ctx* c, int levels, const unsigned char* masks, const T* mu, T* qhat,
                               double* cost, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    if (!mu || !qhat || !cost) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    Geom<T> g;
    WST(make_geom<T>(c, &g));
    cudaStream_t st = as_stream(stream);
    uint8_t* leaf = nullptr;
    WST(leaf_from_masks(c, lay, masks, &leaf, st));
    const int np = forward_parts(g.V, g.B);
    double* cpart = nullptr;
    WST(ensure_t(c, B_COSTPART, (size_t)np, &cpart));
    T* mut = nullptr;
    WST(ensure_t(c, B_MUT, pad_elems(c), &mut));
    WCK(c, launch_forward<T>(g, mu, mut, leaf, 0, static_cast<const float*>(c->buf[B_D].p),
                             dterm_buf<T>(c), static_cast<const float*>(c->buf[B_I0].p), qhat, nullptr, nullptr,
                             cpart, nullptr,
                             st));
    WCK(c, launch_sum_final(cpart, forward_cost_parts(g.V, g.B), cost, st));
    return WAM_OK;
}

// ---------------------------------------------------------------------------
// 3-D circular cone beam
// ---------------------------------------------------------------------------

// Tables of the cone geometry, computed in FP64 on the host once:
// in-plane direction D_xy = -SDD e + u_b u per (view, bin) as
// (s/Dx, -c/Dy, 1/Dx, 1/Dy); 1/v_r per row; |D| per (row, bin).
wam_status make_geom3(wam_ctx* c, Geom3* g)
{
    const wam_geometry& w = c->g;
    g->nx = w.nx; g->ny = w.ny; g->nz = w.nz; g->V = w.n_views; g->R = w.n_rows; g->B = w.n_bins;
    g->vx = (float)w.vx; g->vy = (float)w.vy; g->vz = (float)w.vz;
    g->X0 = (float)(-0.5 * w.nx * w.vx); g->Y0 = (float)(-0.5 * w.ny * w.vy); g->Z0 = (float)(-0.5 * w.nz * w.vz);
    g->ivx = (float)(1.0 / w.vx); g->ivy = (float)(1.0 / w.vy); g->ivz = (float)(1.0 / w.vz);
    g->pitch = (float)w.bin_pitch; g->ucen = (float)(0.5 * (w.n_bins - 1));
    g->rpitch = (float)w.row_pitch; g->rcen = (float)(0.5 * (w.n_rows - 1));
    g->sod = (float)w.sod; g->sdd = (float)w.sdd;
    g->cs = static_cast<const float*>(c->buf[B_CS32].p);
    const size_t nvb = (size_t)w.n_views * w.n_bins, nrb = (size_t)w.n_rows * w.n_bins;
    if (!c->buf[B_DIR3].p || c->buf[B_DIR3].bytes < nvb * 16) {
        auto rcp = [](double d) {
            double a = std::fabs(d);
            a = a < 1e-30 ? 1e-30 : a;
            return std::signbit(d) ? -1.0 / a : 1.0 / a;
        };
        std::vector<float> dir(4 * nvb), rinv(w.n_rows), dl(nrb);
        for (int k = 0; k < w.n_views; ++k) {
            const double th = w.angle0 + k * (w.angle_span / w.n_views);
            const double cs = std::cos(th), sn = std::sin(th);
            for (int b = 0; b < w.n_bins; ++b) {
                const double ub = (b - 0.5 * (w.n_bins - 1)) * w.bin_pitch;
                const double ix = rcp(-w.sdd * cs - ub * sn), iy = rcp(-w.sdd * sn + ub * cs);
                float* e = &dir[4 * ((size_t)k * w.n_bins + b)];
                e[0] = (float)(sn * ix); e[1] = (float)(-cs * iy); e[2] = (float)ix; e[3] = (float)iy;
            }
        }
        for (int r = 0; r < w.n_rows; ++r) {
            const double vr = (r - 0.5 * (w.n_rows - 1)) * w.row_pitch;
            rinv[r] = (float)rcp(vr);
            for (int b = 0; b < w.n_bins; ++b) {
                const double ub = (b - 0.5 * (w.n_bins - 1)) * w.bin_pitch;
                dl[(size_t)r * w.n_bins + b] = (float)std::sqrt(w.sdd * w.sdd + ub * ub + vr * vr);
            }
        }
        float *d1 = nullptr, *d2 = nullptr, *d3 = nullptr;
        WST(ensure_t(c, B_DIR3, 4 * nvb, &d1));
        WST(ensure_t(c, B_ROWINV, (size_t)w.n_rows, &d2));
        WST(ensure_t(c, B_DLEN, nrb, &d3));
        WCK(c, cudaMemcpy(d1, dir.data(), dir.size() * 4, cudaMemcpyHostToDevice));
        WCK(c, cudaMemcpy(d2, rinv.data(), rinv.size() * 4, cudaMemcpyHostToDevice));
        WCK(c, cudaMemcpy(d3, dl.data(), dl.size() * 4, cudaMemcpyHostToDevice));
    }
    g->dirt = static_cast<const float4*>(c->buf[B_DIR3].p);
    g->rowinv = static_cast<const float*>(c->buf[B_ROWINV].p);
    g->dlen = static_cast<const float*>(c->buf[B_DLEN].p);
    return WAM_OK;
}

wam_status make_layout3(wam_ctx* c, int L, int z3, Layout3* lay)
{
    const wam_geometry& w = c->g;
    if (L < 0 || L > 5) return fail(c, WAM_ERR_ARG, "cone beam: levels must be in 0..5");
    if (w.nx % (1 << L) || w.ny % (1 << L) || (z3 && w.nz % (1 << L)))
        return fail(c, WAM_ERR_ARG, "volume sides must be divisible by 2^levels");
    if (w.nx % 2 || w.ny % 2 || w.nz % 2) return fail(c, WAM_ERR_ARG, "cone beam: nx, ny, nz must be even");
    std::memset(lay, 0, sizeof(*lay));
    lay->L = L; lay->nx = w.nx; lay->ny = w.ny; lay->nz = w.nz; lay->z3 = z3;
    lay->nslice = (long long)w.nx * w.ny;
    for (int l = 0; l <= L; ++l) {
        lay->gw[l] = w.nx >> l; lay->gh[l] = w.ny >> l; lay->gd[l] = z3 ? (w.nz >> l) : w.nz;
    }
    const int nd = z3 ? 7 : 3;
    long long off = (long long)lay->gw[L] * lay->gh[L] * (z3 ? lay->gd[L] : 1);
    long long moff = 0;
    for (int l = L; l >= 1; --l) {
        const long long nbk = (long long)lay->gw[l] * lay->gh[l] * (z3 ? lay->gd[l] : 1);
        lay->coff[l] = off;
        off += nd * nbk;
        lay->moff[l] = moff;
        moff += nbk;
    }
    lay->mask_bytes = moff;
    return WAM_OK;
}

struct ListInfo3 {
    int level, has_approx, has_details, octet, n;
    const uint32_t* items;
    int rep, gw, gh;
};

wam_status plan3(wam_ctx* c, int z3, const std::vector<ListInfo3>& lists, SegTable3* tab, float** part_out)
{
    const wam_geometry& w = c->g;
    std::memset(tab, 0, sizeof(*tab));
    const double mag = 1.3 * w.sdd / w.sod;
    std::vector<double> cost(lists.size());
    double total = 0.0;
    for (size_t i = 0; i < lists.size(); ++i) {
        const ListInfo3& li = lists[i];
        const double sxy = (double)(1 << li.level) * std::hypot(w.vx, w.vy);
        const double sz = (li.octet ? 2.0 : (z3 ? (double)(1 << li.level) : 1.0)) * w.vz;
        const double rays = (sxy * mag / w.bin_pitch + 1.0) * (sz * mag / w.row_pitch + 1.0);
        cost[i] = rays * ((li.has_details || li.octet) ? 4.0 : 1.0);
        total += (double)li.n * w.n_views * cost[i];
    }
    const double per_cta = std::max(total / ((double)c->num_sms * c->back_ctas_per_sm), 1.0);
    const int max_chunks = std::max(1, w.n_views / kViewLanes);
    int cta = 0, items = 0;
    long long part = 0;
    const int nd = z3 ? 7 : 3;
    for (size_t i = 0; i < lists.size(); ++i) {
        const ListInfo3& li = lists[i];
        if (li.n == 0) continue;
        Segment3& s = tab->s[tab->n++];
        s.level = li.level; s.has_approx = li.has_approx; s.has_details = li.has_details; s.octet = li.octet;
        s.n_items = li.n; s.items = li.items; s.rep = li.rep; s.gw = li.gw; s.gh = li.gh;
        int chunks = (int)std::ceil((double)kItemsPerCta * w.n_views * cost[i] / per_cta);
        chunks = std::max(1, std::min(chunks, max_chunks));
        s.vpc = (w.n_views + chunks - 1) / chunks;
        s.n_chunks = (w.n_views + s.vpc - 1) / s.vpc;
        s.tiles = (li.n + kItemsPerCta - 1) / kItemsPerCta;
        s.cta_begin = cta; s.item_begin = items;
        s.n_slots = li.octet ? 8 : li.has_approx + 2 * nd * li.has_details;
        s.part_off = part;
        cta += s.tiles * s.n_chunks;
        items += li.n;
        part += (long long)s.n_slots * s.n_chunks * li.n;
    }
    tab->total_ctas = cta;
    tab->total_items = items;
    return ensure_t(c, B_PART, (size_t)std::max<long long>(part, 1), part_out);
}

wam_status plan_voxels3(wam_ctx* c, int z3, SegTable3* tab, float** part)
{
    const wam_geometry& w = c->g;
    std::vector<ListInfo3> li = {{1, 0, 0, 1, (w.nx / 2) * (w.ny / 2) * (w.nz / 2), nullptr, 0, w.nx / 2, w.ny / 2}};
    return plan3(c, z3, li, tab, part);
}

wam_status plan_tree3(wam_ctx* c, const Layout3& lay, const uint8_t* mask, uint8_t* leaf, SegTable3* tab,
                      float** part, long long* leaves, cudaStream_t st)
{
    PROF(WAM_K_TREE);
    WCK(c, launch_leafmap3(lay, mask, leaf, st));
    const int L = lay.L;
    const long long stride = (long long)lay.gw[1] * lay.gh[1] * (lay.z3 ? lay.gd[1] : 1);
    uint32_t* lists = nullptr;
    int* counts = nullptr;
    WST(ensure_t(c, B_LISTS, (size_t)stride * (L + 1), &lists));
    WST(ensure_t(c, B_COUNTS, (size_t)(L + 1), &counts));
    WCK(c, launch_compact3(lay, mask, lists, stride, counts, st));
    std::vector<int> h(L + 1);
    WCK(c, cudaMemcpyAsync(h.data(), counts, sizeof(int) * (L + 1), cudaMemcpyDeviceToHost, st));
    WCK(c, cudaStreamSynchronize(st));
    const int rep = lay.z3 ? 0 : 1;
    const int nzr = lay.z3 ? 1 : lay.nz;
    const int nd = lay.z3 ? 7 : 3;
    long long lv = (long long)lay.gw[L] * lay.gh[L] * (lay.z3 ? lay.gd[L] : 1);
    for (int k = 1; k <= L; ++k) lv += (long long)nd * h[k];
    *leaves = lv * nzr;
    // finest leaf level: h[k] counts the expanded blocks of level L - k + 1
    c->last_lmin = L;
    for (int k = 1; k <= L; ++k)
        if (h[k] > 0) c->last_lmin = L - k;
    std::vector<ListInfo3> li;
    li.push_back({L, 1, 0, 0, h[0] * nzr, lists, rep ? h[0] : 0, lay.gw[L], lay.gh[L]});
    li.push_back({L, 1, 1, 0, h[1] * nzr, lists + stride, rep ? h[1] : 0, lay.gw[L], lay.gh[L]});
    for (int k = 1; k < L; ++k)
        li.push_back({L - k, 0, 1, 0, h[k + 1] * nzr, lists + stride * (k + 1), rep ? h[k + 1] : 0, lay.gw[L - k],
                      lay.gh[L - k]});
    return plan3(c, lay.z3, li, tab, part);
}

wam_status compute_z03(wam_ctx* c, const Geom3& g, const Layout3& lay, const uint8_t* leaf, double* z0,
                       cudaStream_t st)
{
    const int np = forward3_parts(g);
    double* part = nullptr;
    WST(ensure_t(c, B_COSTPART, (size_t)np, &part));
    WCK(c, launch_z03(g, lay, leaf, part, st));
    WCK(c, launch_max_final(part, np, z0, st));
    return WAM_OK;
}

wam_status reconstruct3_impl(wam_ctx* c, const wam_schedule* sc, void* mu_out, double* hist,
                             unsigned char* mask_out, int on_device, cudaStream_t st)
{
    if (sc->precision != 32) return fail(c, WAM_ERR_ARG, "cone beam: precision 32 only");
    WST(check_resume(c, sc));
    c->last.valid = false;
    const int L = sc->full_am ? 0 : sc->levels;
    int z3 = 1;
    if (!sc->full_am && L > 0) {
        if (sc->dims == 3) z3 = 1;
        else if (sc->dims == 2 && sc->zsum_criterion) z3 = 0;
        else return fail(c, WAM_ERR_ARG, "cone beam: dims 3, or dims 2 with zsum_criterion = 1");
    }
    Layout3 lay;
    WST(make_layout3(c, L, z3, &lay));
    Geom3 g;
    WST(make_geom3(c, &g));
    const long long N = c->N, M = c->M;
    const int J = sc->n_iters;
    const double clamp = sc->dmax_clamp > 0 ? sc->dmax_clamp : 30.0;
    float *q = nullptr, *mu = nullptr, *s2d = nullptr;
    double *beta = nullptr, *bvec = nullptr, *costs = nullptr, *z0 = nullptr, *scratch = nullptr;
    double *tmpa = nullptr, *tmpb = nullptr, *gimg = nullptr, *cpart = nullptr;
    uint8_t *mask = nullptr, *mask2 = nullptr, *leaf = nullptr;
    WST(ensure_t(c, B_Q, (size_t)M, &q));
    WST(ensure_t(c, B_MU, (size_t)N, &mu));
    WST(ensure_t(c, B_BETA, (size_t)N, &beta));
    WST(ensure_t(c, B_BVEC, (size_t)N, &bvec));
    WST(ensure_t(c, B_COSTS, (size_t)J + 1, &costs));
    WST(ensure_t(c, B_Z0, 1, &z0));
    WST(ensure_t(c, B_SCRATCH, 1024, &scratch));
    WST(ensure_t(c, B_TMPA, (size_t)N, &tmpa));
    WST(ensure_t(c, B_TMPB, (size_t)N, &tmpb));
    WST(ensure_t(c, B_GIMG, (size_t)N, &gimg));
    WST(ensure_t(c, B_S2D, (size_t)lay.nslice, &s2d));
    float* pad3 = nullptr;
    WST(ensure_t(c, B_MUT, pad_elems(c), &pad3));
    const int np = forward3_parts(g);
    WST(ensure_t(c, B_COSTPART, (size_t)np, &cpart));
    if (L > 0) {
        WST(ensure_t(c, B_MASK_A, (size_t)lay.mask_bytes, &mask));
        WST(ensure_t(c, B_MASK_B, (size_t)lay.mask_bytes, &mask2));
        WST(ensure_t(c, B_LEAF, (size_t)N, &leaf));
    }
    const float* dsino = static_cast<const float*>(c->buf[B_D].p);
    const float* I0 = static_cast<const float*>(c->buf[B_I0].p);
    const double* dterm = static_cast<const double*>(c->buf[B_DTERM].p);

    // a0: b = Omega^T H^T d
    SegTable3 vox;
    float* part = nullptr;
    WST(plan_voxels3(c, z3, &vox, &part));
    {
        PROF(WAM_K_BACKPROJECT);
        WCK(c, launch_backproject3(g, vox, z3, dsino, part, work_ptr(c, WAM_K_BACKPROJECT), st));
    }
    {
        PROF(WAM_K_TREE);
        WCK(c, launch_reduce_voxels3(vox, lay, part, gimg, nullptr, st));
        WCK(c, launch_haar3(lay, gimg, bvec, tmpa, tmpb, st));
    }
    WCK(c, cudaMemsetAsync(beta, 0, N * sizeof(double), st));
    SegTable3 tab;
    long long leaves = N;
    if (L > 0) {
        WCK(c, cudaMemsetAsync(mask, 0, lay.mask_bytes, st));
        WST(plan_tree3(c, lay, mask, leaf, &tab, &part, &leaves, st));
    } else {
        tab = vox;
    }
    {
        PROF(WAM_K_Z0);
        WST(compute_z03(c, g, lay, leaf, z0, st));
    }
    // a2 walks the volume mu, constant on the leaves and so on the cells of the
    // finest leaf level lam (2^lam cubes for the 3-D tree, 2^lam x 2^lam x 1
    // per slice): the strip walk over those cells, unless the leaves are fewer
    // than a ninth of the cells (then the leaf walk meets fewer boundaries)
    int flam = 0;
    auto pick = [&]() -> const uint8_t* {
        flam = L > 0 ? c->last_lmin : 0;
        const long long cells = N >> ((z3 ? 3 : 2) * flam);
        if (L > 0 && cells > 9 * leaves) {
            flam = 0;
            return leaf;
        }
        return nullptr;
    };
    const uint8_t* fleaf = pick();
    std::vector<int> exp_at(sc->n_expand > 0 ? sc->expand_at : nullptr,
                            sc->n_expand > 0 ? sc->expand_at + sc->n_expand : nullptr);
    size_t next_exp = 0;
    int j0 = 0;
    if (c->pending.valid) {
        // continue from the state of wam_resume (as in the 2-D driver)
        const RunRecord& r = c->pending;
        if (r.beta.size() != (size_t)N || r.hist.size() != (size_t)r.iters_done + 1 ||
            r.mask.size() != (L > 0 ? (size_t)lay.mask_bytes : 0))
            return fail(c, WAM_ERR_STATE, "resume: the checkpoint's sizes do not fit this schedule");
        WCK(c, cudaMemcpyAsync(beta, r.beta.data(), N * sizeof(double), cudaMemcpyHostToDevice, st));
        WCK(c, cudaMemcpyAsync(costs, r.hist.data(), r.hist.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        if (L > 0) {
            WCK(c, cudaMemcpyAsync(mask, r.mask.data(), lay.mask_bytes, cudaMemcpyHostToDevice, st));
            WST(plan_tree3(c, lay, mask, leaf, &tab, &part, &leaves, st));
            fleaf = pick();
            PROF(WAM_K_Z0);
            WST(compute_z03(c, g, lay, leaf, z0, st));
        }
        next_exp = (size_t)r.expansions_done;
        j0 = r.iters_done;
    }
    for (int j = j0; j <= J; ++j) {
        {
            PROF(WAM_K_SYNTH);
            WCK(c, launch_synth3(lay, leaf, beta, mu, st));
        }
        {
            PROF(WAM_K_FORWARD);
            WCK(c, launch_forward3(g, mu, pad3, fleaf, flam, z3, dsino, dterm, I0, q, nullptr, cpart, work_ptr(c, WAM_K_FORWARD),
                                   st));
            WCK(c, launch_sum_final(cpart, np, costs + j, st));
        }
        if (j == J) break;
        {
            PROF(WAM_K_BACKPROJECT);
            WCK(c, launch_backproject3(g, tab, z3, q, part, work_ptr(c, WAM_K_BACKPROJECT), st));
        }
        {
            PROF(WAM_K_UPDATE);
            WCK(c, launch_update3(tab, lay, part, bvec, z0, clamp, beta, sc->nonneg, st));
        }
        if (L > 0 && next_exp < exp_at.size() && exp_at[next_exp] == j + 1) {
            const double tau = sc->tau[next_exp];
            ++next_exp;
            {
                PROF(WAM_K_TREE);
                WCK(c, launch_synth3(lay, leaf, beta, mu, st));
                WCK(c, cudaMemcpyAsync(mask2, mask, lay.mask_bytes, cudaMemcpyDeviceToDevice, st));
                WCK(c, launch_expand3(lay, mu, tau, leaf, mask2, s2d, scratch, st));
            }
            std::swap(mask, mask2);
            std::swap(c->buf[B_MASK_A], c->buf[B_MASK_B]);
            WST(plan_tree3(c, lay, mask, leaf, &tab, &part, &leaves, st));
            fleaf = pick();
            {
                PROF(WAM_K_Z0);
                WST(compute_z03(c, g, lay, leaf, z0, st));
            }
        }
    }
    const cudaMemcpyKind k2 = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (mu_out) WCK(c, cudaMemcpyAsync(mu_out, mu, N * sizeof(float), k2, st));
    if (mask_out && L > 0) WCK(c, cudaMemcpyAsync(mask_out, mask, lay.mask_bytes, k2, st));
    std::vector<double> h(J + 1);
    WCK(c, cudaMemcpyAsync(h.data(), costs, (J + 1) * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (hist) WCK(c, cudaMemcpyAsync(hist, costs, (J + 1) * sizeof(double), k2, st));
    WCK(c, cudaStreamSynchronize(st));
    if (c->prof || c->prof_work) WST(prof_resolve(c));
    record_run(c, sc, J, (int)next_exp);
    for (int j = 0; j < J; ++j)
        if (h[j + 1] > h[j] + 1e-6 * std::fabs(h[j])) return WAM_WARN_NONMONOTONE;
    return WAM_OK;
}

// ---- checkpoint files ----------------------------------------------------------
// CRC-32 (the reflected IEEE 802.3 polynomial 0xEDB88320, initial value and
// final xor 0xFFFFFFFF), byte-wise with a 256-entry table.
uint32_t crc32_update(uint32_t crc, const void* data, size_t n)
{
    static uint32_t table[256];
    static bool ready = false;
    if (!ready) {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t r = i;
            for (int k = 0; k < 8; ++k) r = (r & 1u) ? (r >> 1) ^ 0xEDB88320u : r >> 1;
            table[i] = r;
        }
        ready = true;
    }
    const unsigned char* p = static_cast<const unsigned char*>(data);
    crc = ~crc;
    for (size_t i = 0; i < n; ++i) crc = table[(crc ^ p[i]) & 0xffu] ^ (crc >> 8);
    return ~crc;
}

// CRC-32 of the context's d and I0 (device copies read back)
wam_status data_crc(wam_ctx* c, uint32_t* cd, uint32_t* ci)
{
    std::vector<float> h((size_t)c->M);
    WCK(c, cudaMemcpy(h.data(), c->buf[B_D].p, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    *cd = crc32_update(0, h.data(), h.size() * sizeof(float));
    WCK(c, cudaMemcpy(h.data(), c->buf[B_I0].p, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    *ci = crc32_update(0, h.data(), h.size() * sizeof(float));
    return WAM_OK;
}

struct CkptWriter {
    std::vector<unsigned char> b;
    void raw(const void* p, size_t n)
    {
        const unsigned char* q = static_cast<const unsigned char*>(p);
        b.insert(b.end(), q, q + n);
    }
    void i64(long long v)
    {
        const int64_t x = v;
        raw(&x, 8);
    }
    void f64(double v) { raw(&v, 8); }
};

struct CkptReader {
    const unsigned char* p;
    size_t n, at = 0;
    bool raw(void* dst, size_t k)
    {
        if (k > n - at) return false;
        std::memcpy(dst, p + at, k);
        at += k;
        return true;
    }
    bool i64(long long* v)
    {
        int64_t x;
        if (!raw(&x, 8)) return false;
        *v = x;
        return true;
    }
    bool f64(double* v) { return raw(v, 8); }
};

const char kCkptMagic[8] = {'W', 'A', 'M', 'C', 'K', 'P', 'T', '1'};

}  // namespace

// ===========================================================================
// C-ABI
// ===========================================================================
extern "C" {

wam_status wam_create(const wam_geometry* g, wam_ctx** out)
{
    if (!out) return WAM_ERR_ARG;
    *out = nullptr;
    std::string why;
    if (check_geometry(g, &why) != WAM_OK) return WAM_ERR_ARG;
    try {
        wam_ctx* c = new wam_ctx();
        c->g = *g;
        const bool cone = g->kind == WAM_CONE3D_FLAT_CIRCULAR;
        c->N = (long long)g->nx * g->ny * (cone ? g->nz : 1);
        c->M = (long long)g->n_views * g->n_bins * (cone ? g->n_rows : 1);
        if (cudaGetDevice(&c->device) != cudaSuccess) {
            cudaGetLastError();
            delete c;
            return WAM_ERR_CUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) == cudaSuccess && sms > 0)
            c->num_sms = sms;
        wam_status s = upload_views(c);
        if (s != WAM_OK) {
            wam_destroy(c);
            return s;
        }
        *out = c;
        return WAM_OK;
    } catch (...) {
        return WAM_ERR_OOM;
    }
}

void wam_destroy(wam_ctx* c)
{
    if (!c) return;
    for (auto& b : c->buf)
        if (b.p) cudaFree(b.p);
    for (auto& p : c->pend) {
        cudaEventDestroy(p.a);
        cudaEventDestroy(p.b);
    }
    for (auto e : c->ev_pool) cudaEventDestroy(e);
    if (c->dwork) cudaFree(c->dwork);
    delete c;
}

const char* wam_last_error(const wam_ctx* c) { return c ? c->err.c_str() : "null context"; }

size_t wam_mask_bytes_dims(const wam_ctx* c, int levels, int dims)
{
    if (!c || levels < 0 || levels > WAM_MAX_LEVELS) return 0;
    if (dims != 3) return wam_mask_bytes(c, levels);
    size_t s = 0;
    for (int l = 1; l <= levels; ++l)
        s += (size_t)(c->g.nx >> l) * (size_t)(c->g.ny >> l) * (size_t)(c->g.nz >> l);
    return s;
}

size_t wam_mask_bytes(const wam_ctx* c, int levels)
{
    if (!c || levels < 0 || levels > WAM_MAX_LEVELS) return 0;
    size_t s = 0;
    for (int l = 1; l <= levels; ++l) s += (size_t)(c->g.nx >> l) * (size_t)(c->g.ny >> l);
    return s;
}

wam_status wam_set_data(wam_ctx* c, const float* d, const float* I0, int I0_is_scalar, int on_device, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (!d || !I0) return fail(c, WAM_ERR_ARG, "d and I0 must not be NULL");
    try {
        cudaStream_t st = as_stream(stream);
        const long long M = c->M;
        float *dd = nullptr, *ii = nullptr;
        double* dt = nullptr;
        WST(ensure_t(c, B_D, (size_t)M, &dd));
        WST(ensure_t(c, B_I0, (size_t)M, &ii));
        WST(ensure_t(c, B_DTERM, (size_t)M, &dt));
        float2* dt2 = nullptr;
        WST(ensure_t(c, B_DTERM2, (size_t)M, &dt2));
        // validate on the host (device data are copied back once)
        std::vector<float> hd((size_t)M), hi(I0_is_scalar ? 1 : (size_t)M);
        const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        WCK(c, cudaMemcpyAsync(hd.data(), d, M * sizeof(float), kin, st));
        WCK(c, cudaMemcpyAsync(hi.data(), I0, hi.size() * sizeof(float), kin, st));
        WCK(c, cudaStreamSynchronize(st));
        for (float x : hd)
            if (!(x >= 0.0f) || !std::isfinite(x)) return fail(c, WAM_ERR_ARG, "d must be finite and >= 0");
        for (float x : hi)
            if (!(x > 0.0f) || !std::isfinite(x)) return fail(c, WAM_ERR_ARG, "I0 must be finite and > 0");
        WCK(c, cudaMemcpyAsync(dd, hd.data(), M * sizeof(float), cudaMemcpyHostToDevice, st));
        if (I0_is_scalar) {
            WCK(c, launch_fill_f32(ii, M, hi[0], st));
        } else {
            WCK(c, cudaMemcpyAsync(ii, hi.data(), M * sizeof(float), cudaMemcpyHostToDevice, st));
        }
        WCK(c, launch_dterm(dd, ii, M, dt, dt2, st));
        WCK(c, cudaStreamSynchronize(st));
        c->has_data = true;
        c->last = RunRecord{};
        c->pending = RunRecord{};
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_reconstruct(wam_ctx* c, const wam_schedule* sc, void* mu_out, double* hist, unsigned char* mask_out,
                           int on_device, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (!sc) return fail(c, WAM_ERR_ARG, "schedule is NULL");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    if (sc->n_iters < 0) return fail(c, WAM_ERR_ARG, "n_iters must be >= 0");
    if (sc->precision != 32 && sc->precision != 64) return fail(c, WAM_ERR_ARG, "precision must be 32 or 64");
    if (sc->n_subsets < 0 || sc->n_subsets > c->g.n_views)
        return fail(c, WAM_ERR_ARG, "n_subsets must be in 0..n_views");
    if (sc->n_subsets > 1 && c->g.kind == WAM_CONE3D_FLAT_CIRCULAR)
        return fail(c, WAM_ERR_ARG, "ordered subsets: 2-D contexts only");
    if (sc->nonneg != 0 && sc->nonneg != 1) return fail(c, WAM_ERR_ARG, "nonneg must be 0 or 1");
    if (sc->nonneg && !sc->full_am && sc->levels != 0)
        return fail(c, WAM_ERR_ARG, "nonneg applies to plain AM (full_am or levels = 0) only");
    if (!(sc->lambda >= 0.0) || !std::isfinite(sc->lambda)) return fail(c, WAM_ERR_ARG, "lambda must be finite and >= 0");
    if (sc->lambda > 0.0 && (sc->full_am || sc->levels == 0 || sc->n_subsets > 1 ||
                             c->g.kind == WAM_CONE3D_FLAT_CIRCULAR))
        return fail(c, WAM_ERR_ARG, "lambda > 0 needs a 2-D Haar tree (levels > 0) without ordered subsets");
    if (sc->n_expand < 0 || (sc->n_expand > 0 && (!sc->expand_at || !sc->tau)))
        return fail(c, WAM_ERR_ARG, "expand_at/tau missing");
    for (int k = 0; k < sc->n_expand; ++k) {
        if (sc->expand_at[k] < 1 || (k > 0 && sc->expand_at[k] <= sc->expand_at[k - 1]))
            return fail(c, WAM_ERR_ARG, "expand_at must be increasing and >= 1");
        if (!std::isfinite(sc->tau[k])) return fail(c, WAM_ERR_ARG, "tau must be finite");
    }
    try {
        cudaStream_t st = as_stream(stream);
        if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR)
            return reconstruct3_impl(c, sc, mu_out, hist, mask_out, on_device, st);
        if (sc->precision == 32) return reconstruct_impl<float>(c, sc, mu_out, hist, mask_out, on_device, st);
        return reconstruct_impl<double>(c, sc, mu_out, hist, mask_out, on_device, st);
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

// ---- checkpoint / resume ----------------------------------------------------

wam_status wam_checkpoint(wam_ctx* c, const char* path)
{
    if (!c) return WAM_ERR_ARG;
    if (!path || !*path) return fail(c, WAM_ERR_ARG, "path is empty");
    if (!c->last.valid || !c->has_data) return fail(c, WAM_ERR_STATE, "no finished reconstruction to checkpoint");
    try {
        const RunRecord& r = c->last;
        const size_t mb = r.levels > 0 ? wam_mask_bytes_dims(c, r.levels, r.dims) : 0;
        std::vector<double> beta((size_t)c->N), hist((size_t)r.iters_done + 1);
        std::vector<unsigned char> mask(mb);
        WCK(c, cudaMemcpy(beta.data(), c->buf[B_BETA].p, beta.size() * sizeof(double), cudaMemcpyDeviceToHost));
        WCK(c, cudaMemcpy(hist.data(), c->buf[B_COSTS].p, hist.size() * sizeof(double), cudaMemcpyDeviceToHost));
        if (mb) WCK(c, cudaMemcpy(mask.data(), c->buf[B_MASK_A].p, mb, cudaMemcpyDeviceToHost));
        uint32_t cd = 0, ci = 0;
        WST(data_crc(c, &cd, &ci));
        const wam_geometry& g = c->g;
        CkptWriter w;
        w.raw(kCkptMagic, 8);
        const uint32_t version = 3, zero = 0;
        w.raw(&version, 4);
        w.raw(&zero, 4);
        const long long ints[22] = {g.kind, g.nx, g.ny, g.nz, g.n_views, g.n_bins, g.n_rows, r.levels, r.dims,
                                    r.zsum, r.precision, r.full_am, (long long)r.expand_at.size(), r.iters_done,
                                    r.expansions_done, c->N, (long long)mb, (long long)hist.size(), cd, ci,
                                    r.n_subsets, r.nonneg};
        for (long long v : ints) w.i64(v);
        const double dbl[12] = {g.vx, g.vy, g.vz, g.angle0, g.angle_span, g.bin_pitch, g.row_pitch, g.sod, g.sdd,
                                r.clamp, r.tuning, r.lambda};
        for (double v : dbl) w.f64(v);
        for (int v : r.expand_at) w.i64(v);
        for (double v : r.tau) w.f64(v);
        w.raw(beta.data(), beta.size() * sizeof(double));
        w.raw(mask.data(), mask.size());
        w.raw(hist.data(), hist.size() * sizeof(double));
        const uint32_t crc = crc32_update(0, w.b.data(), w.b.size());
        w.raw(&crc, 4);
        const std::string tmp = std::string(path) + ".tmp";
        std::FILE* f = std::fopen(tmp.c_str(), "wb");
        if (!f) return fail(c, WAM_ERR_IO, "cannot open " + tmp + " for writing");
        const bool ok = std::fwrite(w.b.data(), 1, w.b.size(), f) == w.b.size() && std::fflush(f) == 0;
        if (std::fclose(f) != 0 || !ok) {
            std::remove(tmp.c_str());
            return fail(c, WAM_ERR_IO, "writing " + tmp + " failed");
        }
        if (std::rename(tmp.c_str(), path) != 0) {
            std::remove(tmp.c_str());
            return fail(c, WAM_ERR_IO, std::string("renaming to ") + path + " failed");
        }
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_resume(wam_ctx* c, const char* path)
{
    if (!c) return WAM_ERR_ARG;
    if (!path || !*path) return fail(c, WAM_ERR_ARG, "path is empty");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    try {
        std::FILE* f = std::fopen(path, "rb");
        if (!f) return fail(c, WAM_ERR_IO, std::string("cannot open ") + path);
        std::vector<unsigned char> buf;
        unsigned char chunk[1 << 16];
        size_t k;
        while ((k = std::fread(chunk, 1, sizeof chunk, f)) > 0) buf.insert(buf.end(), chunk, chunk + k);
        const bool rerr = std::ferror(f) != 0;
        std::fclose(f);
        if (rerr) return fail(c, WAM_ERR_IO, std::string("reading ") + path + " failed");
        if (buf.size() < 16 + 4 || std::memcmp(buf.data(), kCkptMagic, 8) != 0)
            return fail(c, WAM_ERR_IO, "not a checkpoint file (magic)");
        uint32_t crc_file;
        std::memcpy(&crc_file, buf.data() + buf.size() - 4, 4);
        if (crc32_update(0, buf.data(), buf.size() - 4) != crc_file)
            return fail(c, WAM_ERR_IO, "checkpoint file is corrupt (CRC mismatch)");
        CkptReader rd{buf.data(), buf.size() - 4};
        rd.at = 8;
        uint32_t version = 0, zero = 0;
        if (!rd.raw(&version, 4) || !rd.raw(&zero, 4) || (version != 2 && version != 3))
            return fail(c, WAM_ERR_IO, "unsupported checkpoint version");
        long long v[22];
        double d[12] = {0};                   // version 2 files carry no lambda (0)
        for (long long& x : v)
            if (!rd.i64(&x)) return fail(c, WAM_ERR_IO, "checkpoint header truncated");
        for (int k = 0; k < (version == 3 ? 12 : 11); ++k)
            if (!rd.f64(&d[k])) return fail(c, WAM_ERR_IO, "checkpoint header truncated");
        const wam_geometry& g = c->g;
        const bool same_geom = v[0] == g.kind && v[1] == g.nx && v[2] == g.ny && v[3] == g.nz && v[4] == g.n_views &&
                               v[5] == g.n_bins && v[6] == g.n_rows && d[0] == g.vx && d[1] == g.vy &&
                               d[2] == g.vz && d[3] == g.angle0 && d[4] == g.angle_span && d[5] == g.bin_pitch &&
                               d[6] == g.row_pitch && d[7] == g.sod && d[8] == g.sdd;
        if (!same_geom) return fail(c, WAM_ERR_STATE, "checkpoint geometry differs from the context's");
        uint32_t cd = 0, ci = 0;
        WST(data_crc(c, &cd, &ci));
        if (v[18] != (long long)cd || v[19] != (long long)ci)
            return fail(c, WAM_ERR_STATE, "checkpoint data (d, I0) differ from the context's");
        RunRecord r;
        r.levels = (int)v[7];
        r.dims = (int)v[8];
        r.zsum = (int)v[9];
        r.precision = (int)v[10];
        r.full_am = (int)v[11];
        const long long n_expand = v[12];
        r.iters_done = (int)v[13];
        r.expansions_done = (int)v[14];
        r.n_subsets = (int)v[20];
        r.nonneg = (int)v[21];
        r.clamp = d[9];
        r.tuning = d[10];
        r.lambda = d[11];
        const size_t mb = r.levels > 0 ? wam_mask_bytes_dims(c, r.levels, r.dims) : 0;
        if (r.levels < 0 || r.levels > WAM_MAX_LEVELS || n_expand < 0 || n_expand > 4096 || r.iters_done < 0 ||
            r.expansions_done < 0 || r.expansions_done > n_expand || v[15] != c->N || v[16] != (long long)mb ||
            v[17] != (long long)r.iters_done + 1 || !(r.tuning >= 0.25 && r.tuning <= 256.0) || r.n_subsets < 1 ||
            r.n_subsets > c->g.n_views || (r.nonneg != 0 && r.nonneg != 1) || !(r.lambda >= 0.0) ||
            !std::isfinite(r.lambda))
            return fail(c, WAM_ERR_IO, "checkpoint header is inconsistent with this context");
        r.expand_at.resize((size_t)n_expand);
        r.tau.resize((size_t)n_expand);
        for (int& x : r.expand_at) {
            long long t;
            if (!rd.i64(&t)) return fail(c, WAM_ERR_IO, "checkpoint truncated");
            x = (int)t;
        }
        for (double& x : r.tau)
            if (!rd.f64(&x)) return fail(c, WAM_ERR_IO, "checkpoint truncated");
        r.beta.resize((size_t)c->N);
        r.mask.resize(mb);
        r.hist.resize((size_t)r.iters_done + 1);
        if (!rd.raw(r.beta.data(), r.beta.size() * sizeof(double)) || !rd.raw(r.mask.data(), mb) ||
            !rd.raw(r.hist.data(), r.hist.size() * sizeof(double)) || rd.at != rd.n)
            return fail(c, WAM_ERR_IO, "checkpoint size does not match its header");
        r.valid = true;
        c->back_ctas_per_sm = r.tuning;
        c->pending = std::move(r);
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

// ---- steps ------------------------------------------------------------------

wam_status wam_project(wam_ctx* c, const float* mu, float* p, void* s)
{
    if (c && c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) {
        if (!mu || !p) return fail(c, WAM_ERR_ARG, "null pointer");
        Geom3 g;
        WST(make_geom3(c, &g));
        float* pad3 = nullptr;
        WST(ensure_t(c, B_MUT, pad_elems(c), &pad3));
        WCK(c, launch_forward3(g, mu, pad3, nullptr, 0, 1, nullptr, nullptr, nullptr, nullptr, p, nullptr, nullptr,
                               as_stream(s)));
        return WAM_OK;
    }
    return project_impl<float>(c, mu, p, s);
}
wam_status wam_project_f64(wam_ctx* c, const double* mu, double* p, void* s) { return project_impl<double>(c, mu, p, s); }

wam_status wam_backproject(wam_ctx* c, const float* s, float* gout, void* st)
{
    if (c && c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) {
        if (!s || !gout) return fail(c, WAM_ERR_ARG, "null pointer");
        try {
            Layout3 lay;
            WST(make_layout3(c, 0, 1, &lay));
            Geom3 g;
            WST(make_geom3(c, &g));
            SegTable3 tab;
            float* part = nullptr;
            WST(plan_voxels3(c, 1, &tab, &part));
            WCK(c, launch_backproject3(g, tab, 1, s, part, nullptr, as_stream(st)));
            WCK(c, launch_reduce_voxels3(tab, lay, part, nullptr, gout, as_stream(st)));
            return WAM_OK;
        } catch (...) {
            return fail(c, WAM_ERR_OOM, "host allocation failed");
        }
    }
    return backproject_impl<float>(c, s, gout, st);
}
wam_status wam_backproject_f64(wam_ctx* c, const double* s, double* g, void* st)
{
    return backproject_impl<double>(c, s, g, st);
}

wam_status wam_haar(wam_ctx* c, int levels, const double* in, double* out, int inverse, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!in || !out || in == out) return fail(c, WAM_ERR_ARG, "in and out must be distinct non-null arrays");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    double *ta = nullptr, *tb = nullptr;
    WST(ensure_t(c, B_TMPA, (size_t)c->N, &ta));
    WST(ensure_t(c, B_TMPB, (size_t)c->N, &tb));
    WCK(c, launch_haar(lay, in, out, inverse, ta, tb, as_stream(stream)));
    return WAM_OK;
}

wam_status wam_synthesize(wam_ctx* c, int levels, const unsigned char* masks, const double* beta, float* mu,
                          void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!beta || !mu || (levels > 0 && !masks)) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    cudaStream_t st = as_stream(stream);
    uint8_t* leaf = nullptr;
    WST(leaf_from_masks(c, lay, masks, &leaf, st));
    WCK(c, launch_synth<float>(lay, leaf, beta, mu, st));
    return WAM_OK;
}

wam_status wam_forward(wam_ctx* c, int levels, const unsigned char* masks, const float* mu, float* qhat,
                       double* cost, void* st)
{
    return forward_impl<float>(c, levels, masks, mu, qhat, cost, st);
}

wam_status wam_forward_f64(wam_ctx* c, int levels, const unsigned char* masks, const double* mu, double* qhat,
                           double* cost, void* st)
{
    return forward_impl<double>(c, levels, masks, mu, qhat, cost, st);
}

wam_status wam_split_backproject(wam_ctx* c, int levels, const unsigned char* masks, const float* qhat,
                                 double* bplus, double* bminus, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!qhat || !bplus || !bminus || (levels > 0 && !masks)) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        Geom<float> g;
        WST(make_geom<float>(c, &g));
        cudaStream_t st = as_stream(stream);
        SegTable tab;
        float* part = nullptr;
        if (levels == 0) {
            WST(plan_pixels<float>(c, &tab, &part));
        } else {
            uint8_t* leaf = nullptr;
            WST(ensure_t(c, B_LEAF, (size_t)c->N, &leaf));
            WST(plan_tree<float>(c, lay, masks, leaf, &tab, &part, st));
        }
        WCK(c, cudaMemsetAsync(bplus, 0, c->N * sizeof(double), st));
        WCK(c, cudaMemsetAsync(bminus, 0, c->N * sizeof(double), st));
        const void* dirt = nullptr;
        WST(dir_table<float>(c, &dirt));
        WCK(c, launch_backproject(g, tab, qhat, dirt, part, nullptr, st));
        WCK(c, launch_split_out(tab, lay, part, bplus, bminus, st));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_z0(wam_ctx* c, int levels, const unsigned char* masks, double* z0, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!z0 || (levels > 0 && !masks)) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    Geom<float> g;
    WST(make_geom<float>(c, &g));
    cudaStream_t st = as_stream(stream);
    uint8_t* leaf = nullptr;
    WST(leaf_from_masks(c, lay, masks, &leaf, st));
    return compute_z0<float>(c, g, lay, leaf, z0, st);
}

wam_status wam_update(wam_ctx* c, int levels, const unsigned char* masks, const double* b, const double* bplus,
                      const double* bminus, const double* z0, double clamp, double* beta, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!b || !bplus || !bminus || !z0 || !beta || (levels > 0 && !masks)) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    WCK(c, launch_update_dense(lay, masks, b, bplus, bminus, z0, clamp > 0 ? clamp : 30.0, beta, as_stream(stream)));
    return WAM_OK;
}

wam_status wam_am_delta(long long n, const double* b, const double* bplus, const double* bminus,
                        const double* beta, double lambda, double z0, double clamp, int precision, double* delta,
                        int* at_clamp, void* stream)
{
    if (n < 0 || (n > 0 && (!b || !bplus || !bminus || !delta))) return WAM_ERR_ARG;
    if (precision != 32 && precision != 64) return WAM_ERR_ARG;
    if (!(z0 > 0) || !std::isfinite(z0) || std::isnan(clamp)) return WAM_ERR_ARG;
    if (!(lambda >= 0.0) || !std::isfinite(lambda) || (lambda > 0.0 && n > 0 && !beta)) return WAM_ERR_ARG;
    if (launch_am_delta(precision, n, b, bplus, bminus, beta, lambda, z0, clamp > 0 ? clamp : 30.0, delta, at_clamp,
                        as_stream(stream)) != cudaSuccess) {
        cudaGetLastError();
        return WAM_ERR_CUDA;
    }
    return WAM_OK;
}

wam_status wam_expand(wam_ctx* c, int levels, const float* S, double tau, const unsigned char* mask_in,
                      unsigned char* mask_out, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (levels < 1) return fail(c, WAM_ERR_ARG, "levels must be >= 1");
    if (!S || !mask_in || !mask_out || mask_in == mask_out) return fail(c, WAM_ERR_ARG, "bad pointers");
    if (!std::isfinite(tau)) return fail(c, WAM_ERR_ARG, "tau must be finite");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    cudaStream_t st = as_stream(stream);
    uint8_t* leaf = nullptr;
    double* scratch = nullptr;
    WST(leaf_from_masks(c, lay, mask_in, &leaf, st));
    WST(ensure_t(c, B_SCRATCH, 1024, &scratch));
    WCK(c, cudaMemcpyAsync(mask_out, mask_in, lay.mask_bytes, cudaMemcpyDeviceToDevice, st));
    WCK(c, launch_expand<float>(lay, S, tau, leaf, mask_out, scratch, st));
    return WAM_OK;
}

wam_status wam_profile(wam_ctx* c, int enable)
{
    if (!c) return WAM_ERR_ARG;
    if (enable < WAM_PROFILE_OFF || enable > WAM_PROFILE_WORK) return fail(c, WAM_ERR_ARG, "unknown profile mode");
    if (enable) {
        if (!c->dwork) {
            if (cudaMalloc(&c->dwork, sizeof(unsigned long long) * WAM_NKERNEL) != cudaSuccess) {
                cudaGetLastError();
                c->dwork = nullptr;
                return fail(c, WAM_ERR_OOM, "profiling counters");
            }
        }
        WCK(c, cudaDeviceSynchronize());
        for (auto& p : c->pend) {
            c->ev_pool.push_back(p.a);
            c->ev_pool.push_back(p.b);
        }
        c->pend.clear();
        WCK(c, cudaMemset(c->dwork, 0, sizeof(unsigned long long) * WAM_NKERNEL));
        std::memset(&c->stats, 0, sizeof(c->stats));
    }
    c->prof = enable == WAM_PROFILE_ALL || enable == WAM_PROFILE_TIME;
    c->prof_work = enable == WAM_PROFILE_ALL || enable == WAM_PROFILE_WORK;
    return WAM_OK;
}

wam_status wam_get_stats(wam_ctx* c, wam_stats* out)
{
    if (!c || !out) return WAM_ERR_ARG;
    WST(prof_resolve(c));
    *out = c->stats;
    return WAM_OK;
}

unsigned long long wam_kernel_launches(void) { return wam::kernel_launches(); }

wam_status wam_set_tuning(wam_ctx* c, int key, double value)
{
    if (!c) return WAM_ERR_ARG;
    if (key == WAM_TUNE_BACK_CTAS_PER_SM) {
        if (!(value >= 0.25 && value <= 256.0)) return fail(c, WAM_ERR_ARG, "CTAs per SM must be in [0.25, 256]");
        c->back_ctas_per_sm = value;
        return WAM_OK;
    }
    if (key == WAM_TUNE_FWD_STAGE_ROWS) {
        if (value != 0.0 && value != 16.0 && value != 24.0 && value != 32.0)
            return fail(c, WAM_ERR_ARG, "WAM_TUNE_FWD_STAGE_ROWS must be 0, 16, 24 or 32");
        c->fwd_stage_rows = (int)value;
        return WAM_OK;
    }
    if (key == WAM_TUNE_GRAPHS) {
        if (value != 0.0 && value != 1.0) return fail(c, WAM_ERR_ARG, "graphs: 0 or 1");
        c->graphs = value != 0.0;
        return WAM_OK;
    }
    return fail(c, WAM_ERR_ARG, "unknown tuning key");
}

wam_status wam_reconstruct_batch(wam_ctx* const* ctxs, int n, const wam_schedule* sc, void* const* mu_out,
                                 double* const* hist, int on_device, int use_graph, void* stream)
{
    if (!ctxs || n <= 0 || !sc) return WAM_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        if (!ctxs[i]) return WAM_ERR_ARG;
        if (ctxs[i]->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(ctxs[i], WAM_ERR_ARG, "2-D contexts only");
        if (!ctxs[i]->has_data) return fail(ctxs[i], WAM_ERR_STATE, "wam_set_data must be called first");
        if (ctxs[i]->pending.valid)
            return fail(ctxs[i], WAM_ERR_STATE, "a resumed state is pending: continue it with wam_reconstruct");
        for (int k = 0; k < i; ++k)
            if (ctxs[k] == ctxs[i]) return fail(ctxs[i], WAM_ERR_ARG, "a context appears twice in the batch");
    }
    wam_ctx* c0 = ctxs[0];
    if (use_graph < 0 || use_graph > 2) return fail(c0, WAM_ERR_ARG, "use_graph must be 0, 1 or 2");
    if (sc->precision != 32) return fail(c0, WAM_ERR_ARG, "batched reconstruction runs in precision 32");
    if (sc->n_subsets > 1) return fail(c0, WAM_ERR_ARG, "batched reconstruction has no ordered subsets");
    if (sc->nonneg != 0 && sc->nonneg != 1) return fail(c0, WAM_ERR_ARG, "nonneg must be 0 or 1");
    if (sc->nonneg && !sc->full_am && sc->levels != 0)
        return fail(c0, WAM_ERR_ARG, "nonneg applies to plain AM (full_am or levels = 0) only");
    if (!(sc->lambda >= 0.0) || !std::isfinite(sc->lambda) || (sc->lambda > 0.0 && (sc->full_am || sc->levels == 0)))
        return fail(c0, WAM_ERR_ARG, "lambda must be finite and >= 0, and > 0 only with a Haar tree");
    if (sc->n_iters < 0 || sc->n_expand < 0 || (sc->n_expand > 0 && (!sc->expand_at || !sc->tau)))
        return fail(c0, WAM_ERR_ARG, "bad schedule");
    for (int k = 0; k < sc->n_expand; ++k)
        if (sc->expand_at[k] < 1 || (k > 0 && sc->expand_at[k] <= sc->expand_at[k - 1]) || !std::isfinite(sc->tau[k]))
            return fail(c0, WAM_ERR_ARG, "expand_at must be increasing and >= 1, tau finite");
    // the batch runs on its own non-blocking stream `st` (graph capture is not
    // possible on the legacy default stream), ordered after the caller's
    // stream; the caller's stream waits for it at the end
    const cudaStream_t user = as_stream(stream);
    cudaStream_t st = nullptr;
    std::vector<cudaStream_t> ss(n, nullptr);
    std::vector<cudaEvent_t> joins(n, nullptr);
    cudaEvent_t fork = nullptr;
    std::vector<bool> prof(n);
    for (int i = 0; i < n; ++i) prof[i] = ctxs[i]->prof;
    wam_status ret = WAM_OK;
    auto cleanup = [&]() {
        if (st && fork && cudaEventRecord(fork, st) == cudaSuccess) cudaStreamWaitEvent(user, fork, 0);
        for (int i = 0; i < n; ++i) {
            if (ss[i]) cudaStreamDestroy(ss[i]);
            if (joins[i]) cudaEventDestroy(joins[i]);
            ctxs[i]->prof = prof[i];
        }
        if (st) cudaStreamDestroy(st);
        if (fork) cudaEventDestroy(fork);
        cudaGetLastError();
    };
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(fork, user) != cudaSuccess || cudaStreamWaitEvent(st, fork, 0) != cudaSuccess) {
        cleanup();
        return fail(c0, WAM_ERR_CUDA, "stream or event creation failed");
    }
    try {
        std::vector<Run<float>> runs(n);
        for (int i = 0; i < n; ++i) {
            ctxs[i]->prof = false;
            ctxs[i]->last.valid = false;
        }
        for (int i = 0; i < n; ++i) {
            wam_status s = runs[i].setup(ctxs[i], sc, st);
            if (s != WAM_OK) { cleanup(); return s; }
        }
        // the bags' branches (modes 0 and 1) run concurrently: a staged forward
        // tile, chosen for a bag run alone, slows the shared GPU down there, so
        // the branches take the global-memory walk
        if (use_graph != 2)
            for (auto& r : runs) {
                r.g.stage_rows = 0;
                r.gperm.stage_rows = 0;
                for (auto& gs : r.gsub) gs.stage_rows = 0;
            }
        bool ok = true;
        for (int i = 0; i < n && ok; ++i)
            ok = cudaStreamCreateWithFlags(&ss[i], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&joins[i], cudaEventDisableTiming) == cudaSuccess;
        if (!ok) {
            cudaGetLastError();
            cleanup();
            return fail(c0, WAM_ERR_CUDA, "stream or event creation failed");
        }
        // one step of every run, each on its own stream, forked from and joined into st
        auto step_all = [&](bool final_step) -> wam_status {
            if (cudaEventRecord(fork, st) != cudaSuccess) return fail(c0, WAM_ERR_CUDA, "event record");
            for (int i = 0; i < n; ++i) {
                if (cudaStreamWaitEvent(ss[i], fork, 0) != cudaSuccess) return fail(c0, WAM_ERR_CUDA, "stream wait");
                wam_status s = final_step ? runs[i].final_cost(ss[i], true) : runs[i].iteration(0, ss[i], true);
                if (s != WAM_OK) return s;
                if (cudaEventRecord(joins[i], ss[i]) != cudaSuccess) return fail(c0, WAM_ERR_CUDA, "event record");
                if (cudaStreamWaitEvent(st, joins[i], 0) != cudaSuccess) return fail(c0, WAM_ERR_CUDA, "stream wait");
            }
            return WAM_OK;
        };
        // persistent multi-bag kernels (use_graph = 2): the descriptors of every
        // bag for the current tree epoch, in decreasing order of work; false
        // when some run needs the per-bag path this epoch (a leaf-walk
        // forward, the l1 penalty, ordered subsets, too many bags)
        std::vector<BagDev> hb;
        BatchPrefix hp{};
        auto build_bags = [&]() -> bool {
            if (n > kMaxBags) return false;
            for (int i = 0; i < n; ++i)
                if (runs[i].fwd_leaf || runs[i].lam > 0.0 || runs[i].S > 1) return false;
            std::vector<int> order(n);
            std::vector<double> work(n);
            for (int i = 0; i < n; ++i) {
                order[i] = i;
                work[i] = (double)runs[i].tab.total_ctas * kBackTPB + (double)runs[i].g.V * runs[i].g.B;
            }
            std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
            hb.assign(n, BagDev{});
            hp = BatchPrefix{};
            hp.n = n;
            for (int k = 0; k < n; ++k) {
                const Run<float>& r = runs[order[k]];
                BagDev& B = hb[k];
                B.g = r.g;
                B.gc = cell_grid(r.g, r.fwd_lam);
                B.lay = r.lay;
                B.tab = r.tab;
                B.leaf = r.L > 0 ? r.leaf : nullptr;
                B.beta32 = r.beta32;
                B.pad = r.mut;
                B.lam = r.fwd_lam;
                B.syn_tx = (B.gc.nx + 2 + 31) / 32;
                B.syn_ty = (B.gc.ny + 2 + 31) / 32;
                B.fwd_tiles = (r.g.B + kFwdTPB - 1) / kFwdTPB;
                B.d = r.dsino;
                B.dterm = r.dterm;
                B.I0 = r.I0;
                B.q = r.q;
                B.cpart = r.cpart;
                B.ncost = r.npc;
                B.dirt = static_cast<const float4*>(r.dirt);
                B.part = r.part;
                B.bvec = r.bvec;
                B.z0 = r.z0;
                B.clamp = r.clamp;
                B.beta = r.beta;
                B.nonneg = r.sc->nonneg;
                B.costs = r.costs;
                B.counter = r.counter;
                hp.fwd[k + 1] = hp.fwd[k] + r.g.V * B.fwd_tiles;
                hp.bp[k + 1] = hp.bp[k] + r.tab.total_ctas;
                hp.upd[k + 1] = hp.upd[k] + (int)update_threads(r.tab);
                hp.syn[k + 1] = hp.syn[k] + B.syn_tx * B.syn_ty;
            }
            return true;
        };
        const int J = sc->n_iters;
        int j = 0;
        while (j < J) {
            int e = J;
            const Run<float>& r0 = runs[0];
            if (r0.L > 0 && r0.next_exp < r0.exp_at.size()) e = std::min(J, r0.exp_at[r0.next_exp]);
            // iterations j .. e-1 share one tree per run
            if (use_graph == 2 && build_bags()) {
                // descriptors, prefixes and two item counters in one device block
                const size_t nb = sizeof(BagDev) * n, np = sizeof(BatchPrefix);
                void* blk = nullptr;
                wam_status s = ensure(c0, B_BATCH, nb + np + 2 * sizeof(int), &blk);
                if (s != WAM_OK) { cleanup(); return s; }
                BagDev* dbags = static_cast<BagDev*>(blk);
                BatchPrefix* dpre = reinterpret_cast<BatchPrefix*>(static_cast<char*>(blk) + nb);
                int* counters = reinterpret_cast<int*>(static_cast<char*>(blk) + nb + np);
                if (cudaMemcpyAsync(dbags, hb.data(), nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
                    cudaMemcpyAsync(dpre, &hp, np, cudaMemcpyHostToDevice, st) != cudaSuccess) {
                    cleanup();
                    return fail(c0, WAM_ERR_CUDA, "batch descriptor upload failed");
                }
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                    cudaGetLastError();
                    cleanup();
                    return fail(c0, WAM_ERR_CUDA, "stream capture could not start");
                }
                const cudaError_t el = launch_batch_iteration(dbags, dpre, hp, counters, st);
                const cudaError_t ec = cudaStreamEndCapture(st, &graph);
                if (el != cudaSuccess || ec != cudaSuccess ||
                    cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                    cudaGetLastError();
                    if (graph) cudaGraphDestroy(graph);
                    cleanup();
                    return fail(c0, WAM_ERR_CUDA, "persistent batch iteration could not be captured");
                }
                for (int k = j; k < e && s == WAM_OK; ++k)
                    if (cudaGraphLaunch(exec, st) != cudaSuccess) s = fail(c0, WAM_ERR_CUDA, "graph launch failed");
                add_launches((unsigned long long)batch_launches_per_iteration() * (unsigned long long)std::max(0, e - j - 1));
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                if (s != WAM_OK) { cleanup(); return s; }
            } else if (use_graph) {
                cudaGraph_t graph = nullptr;
                cudaGraphExec_t exec = nullptr;
                if (cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
                    cudaGetLastError();
                    cleanup();
                    return fail(c0, WAM_ERR_CUDA, "stream capture could not start");
                }
                wam_status s = step_all(false);
                const cudaError_t ec = cudaStreamEndCapture(st, &graph);
                if (s != WAM_OK || ec != cudaSuccess) {
                    cudaGetLastError();
                    if (graph) cudaGraphDestroy(graph);
                    cleanup();
                    return s != WAM_OK ? s : fail(c0, WAM_ERR_CUDA, "stream capture failed");
                }
                if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
                    cudaGetLastError();
                    cudaGraphDestroy(graph);
                    cleanup();
                    return fail(c0, WAM_ERR_CUDA, "graph instantiation failed");
                }
                for (int k = j; k < e && s == WAM_OK; ++k)
                    if (cudaGraphLaunch(exec, st) != cudaSuccess) s = fail(c0, WAM_ERR_CUDA, "graph launch failed");
                cudaGraphExecDestroy(exec);
                cudaGraphDestroy(graph);
                if (s != WAM_OK) { cleanup(); return s; }
            } else {
                for (int k = j; k < e; ++k) {
                    wam_status s = step_all(false);
                    if (s != WAM_OK) { cleanup(); return s; }
                }
            }
            j = e;
            if (j < J || (j == J && runs[0].expands_after(J - 1))) {
                for (int i = 0; i < n; ++i) {
                    if (!runs[i].expands_after(j - 1)) continue;
                    wam_status s = runs[i].expand(st);
                    if (s != WAM_OK) { cleanup(); return s; }
                }
            }
        }
        wam_status s = step_all(true);
        if (s != WAM_OK) { cleanup(); return s; }
        std::vector<std::vector<double>> hs(n);
        for (int i = 0; i < n; ++i) {
            s = runs[i].copy_out(mu_out ? mu_out[i] : nullptr, hist ? hist[i] : nullptr, nullptr, on_device, &hs[i],
                                 st);
            if (s != WAM_OK) { cleanup(); return s; }
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) {
            cleanup();
            return fail(c0, WAM_ERR_CUDA, "synchronisation failed");
        }
        s = check_stage_error(c0);
        if (s != WAM_OK) { cleanup(); return s; }
        for (int i = 0; i < n; ++i) {
            record_run(ctxs[i], sc, J, (int)runs[i].next_exp);
            if (runs[i].monotone(hs[i]) != WAM_OK) ret = WAM_WARN_NONMONOTONE;
        }
    } catch (...) {
        cleanup();
        return fail(c0, WAM_ERR_OOM, "host allocation failed");
    }
    cleanup();
    return ret;
}

}  // extern "C"

// ---- operators of the full Haar basis and the gradient pieces ---------------

namespace {

// mu = Omega beta (full L-level basis), float in and out; FP64 synthesis
wam_status coef_to_image(wam_ctx* c, const Layout& lay, const float* beta, float** mu, cudaStream_t st)
{
    double* b64 = nullptr;
    WST(ensure_t(c, B_GBETA, (size_t)c->N, &b64));
    WST(ensure_t(c, B_GMU, (size_t)c->N, mu));
    WCK(c, (launch_convert<float, double>(beta, b64, c->N, st)));
    WCK(c, launch_synth<float>(lay, nullptr, b64, *mu, st));
    return WAM_OK;
}

// coef (FP64) = Omega^T H^T s
wam_status sino_to_coef(wam_ctx* c, const Layout& lay, const float* s, double** coef, cudaStream_t st)
{
    Geom<float> g;
    WST(make_geom<float>(c, &g));
    const void* dirt = nullptr;
    WST(dir_table<float>(c, &dirt));
    SegTable tab;
    float* part = nullptr;
    WST(plan_pixels<float>(c, &tab, &part));
    double *gimg = nullptr, *ta = nullptr, *tb = nullptr;
    WST(ensure_t(c, B_GIMG, (size_t)c->N, &gimg));
    WST(ensure_t(c, B_TMPA, (size_t)c->N, &ta));
    WST(ensure_t(c, B_TMPB, (size_t)c->N, &tb));
    WST(ensure_t(c, B_GCOEF, (size_t)c->N, coef));
    {
        PROF(WAM_K_BACKPROJECT);
        WCK(c, launch_backproject(g, tab, s, dirt, part, work_ptr(c, WAM_K_BACKPROJECT), st));
    }
    PROF(WAM_K_TREE);
    WCK(c, (launch_reduce_pixels<float, double>(tab, c->g.nx, c->N, part, gimg, st)));
    WCK(c, launch_haar(lay, gimg, *coef, 0, ta, tb, st));
    return WAM_OK;
}

}  // namespace

extern "C" {

wam_status wam_project_coef(wam_ctx* c, int levels, const float* beta, float* p, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!beta || !p) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        cudaStream_t st = as_stream(stream);
        float* mu = nullptr;
        WST(coef_to_image(c, lay, beta, &mu, st));
        Geom<float> g;
        WST(make_geom<float>(c, &g));
        float* mut = nullptr;
        WST(ensure_t(c, B_MUT, pad_elems(c), &mut));
        PROF(WAM_K_FORWARD);
        WCK(c, launch_forward<float>(g, mu, mut, nullptr, 0, nullptr, nullptr, nullptr, nullptr, p, nullptr, nullptr,
                                     work_ptr(c, WAM_K_FORWARD), st));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_backproject_coef(wam_ctx* c, int levels, const float* s, float* gout, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!s || !gout) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        cudaStream_t st = as_stream(stream);
        double* coef = nullptr;
        WST(sino_to_coef(c, lay, s, &coef, st));
        WCK(c, (launch_convert<double, float>(coef, gout, c->N, st)));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_idiv_grad(wam_ctx* c, int levels, const float* beta, float lambda, double* loss, float* grad,
                         float* qhat, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    if (!beta || !loss || !grad) return fail(c, WAM_ERR_ARG, "null pointer");
    if (!(lambda >= 0.0f) || !std::isfinite(lambda)) return fail(c, WAM_ERR_ARG, "lambda must be finite and >= 0");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        cudaStream_t st = as_stream(stream);
        float* mu = nullptr;
        WST(coef_to_image(c, lay, beta, &mu, st));
        Geom<float> g;
        WST(make_geom<float>(c, &g));
        const int np = forward_parts(g.V, g.B);
        double* cpart = nullptr;
        float* res = nullptr;
        WST(ensure_t(c, B_COSTPART, (size_t)np, &cpart));
        WST(ensure_t(c, B_GRES, (size_t)c->M, &res));
        float* mut = nullptr;
        WST(ensure_t(c, B_MUT, pad_elems(c), &mut));
        {
            PROF(WAM_K_FORWARD);
            WCK(c, launch_forward<float>(g, mu, mut, nullptr, 0, static_cast<const float*>(c->buf[B_D].p),
                                         dterm_buf<float>(c), static_cast<const float*>(c->buf[B_I0].p), qhat,
                                         nullptr, res, cpart, work_ptr(c, WAM_K_FORWARD), st));
        }
        double* coef = nullptr;
        WST(sino_to_coef(c, lay, res, &coef, st));
        const int nl1 = (int)((c->N + 255) / 256);
        double* l1 = nullptr;
        const int npc = forward_cost_parts(g.V, g.B);
        WST(ensure_t(c, B_L1PART, (size_t)nl1 + npc, &l1));
        WCK(c, launch_l1(lay, beta, coef, lambda, grad, l1, nl1, st));
        // loss = sum of the cost partials and the L1 partials, fixed order
        WCK(c, cudaMemcpyAsync(l1 + nl1, cpart, npc * sizeof(double), cudaMemcpyDeviceToDevice, st));
        WCK(c, launch_sum_final(l1, nl1 + npc, loss, st));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_am_derivs(wam_ctx* c, int levels, const double* b, const double* bplus, const double* bminus,
                         const double* z0, double clamp, float* dplus, float* dminus, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!b || !bplus || !bminus || !z0 || !dplus || !dminus) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    WCK(c, launch_am_derivs(lay, b, bplus, bminus, z0, clamp > 0 ? clamp : 30.0, dplus, dminus,
                            as_stream(stream)));
    return WAM_OK;
}

wam_status wam_precompute_b(wam_ctx* c, int levels, double* b, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    if (!b) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        cudaStream_t st = as_stream(stream);
        Geom<float> g;
        WST(make_geom<float>(c, &g));
        const void* dirt = nullptr;
        WST(dir_table<float>(c, &dirt));
        SegTable pix;
        float* part = nullptr;
        WST(plan_pixels<float>(c, &pix, &part));
        double *gimg = nullptr, *ta = nullptr, *tb = nullptr;
        WST(ensure_t(c, B_GIMG, (size_t)c->N, &gimg));
        WST(ensure_t(c, B_TMPA, (size_t)c->N, &ta));
        WST(ensure_t(c, B_TMPB, (size_t)c->N, &tb));
        // the same launches as the reconstruction's precompute (a0)
        WCK(c, launch_backproject(g, pix, static_cast<const float*>(c->buf[B_D].p), dirt, part, nullptr, st));
        WCK(c, (launch_reduce_pixels<float, double>(pix, c->g.nx, c->N, part, gimg, st)));
        WCK(c, launch_haar(lay, gimg, b, 0, ta, tb, st));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_am_step_vjp(wam_ctx* c, int levels, const double* beta, const double* b, const double* z0,
                           double clamp, const float* gbar, float* gout, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!c->has_data) return fail(c, WAM_ERR_STATE, "wam_set_data must be called first");
    if (!beta || !b || !z0 || !gbar || !gout) return fail(c, WAM_ERR_ARG, "null pointer");
    try {
        Layout lay;
        WST(make_layout(c, levels, &lay));
        cudaStream_t st = as_stream(stream);
        const long long N = c->N, M = c->M;
        // the full tree: every detail active
        uint8_t* masks = nullptr;
        WST(ensure_t(c, B_VJP, (size_t)lay.mask_bytes + 1, &masks));
        WCK(c, cudaMemsetAsync(masks, 1, (size_t)lay.mask_bytes, st));
        // qhat at beta and its split back-projections
        float *mu = nullptr, *q = nullptr, *dp = nullptr, *dm = nullptr, *r = nullptr;
        double *cost = nullptr, *bp = nullptr, *bm = nullptr;
        WST(ensure_t(c, B_GMU, (size_t)N, &mu));
        WST(ensure_t(c, B_VJPQ, (size_t)M, &q));
        WST(ensure_t(c, B_VJPR, (size_t)M, &r));
        WST(ensure_t(c, B_VJPD, 2 * (size_t)N, &dp));
        dm = dp + N;
        WST(ensure_t(c, B_VJPB, 2 * (size_t)N + 1, &bp));
        bm = bp + N;
        cost = bm + N;
        WST(wam_synthesize(c, levels, masks, beta, mu, stream));
        WST(wam_forward(c, levels, masks, mu, q, cost, stream));
        WST(wam_split_backproject(c, levels, masks, q, bp, bm, stream));
        // the derivatives of the root of Eq. 1.9 with respect to bhat+ and bhat-
        WST(wam_am_derivs(c, levels, b, bp, bm, z0, clamp, dp, dm, stream));
        // r = Q (Phi+ D+ gbar + Phi- D- gbar), then gout = gbar - Phi^T r
        WST(wam_phi_split_project(c, levels, gbar, dp, dm, q, r, stream));
        double* coef = nullptr;
        WST(sino_to_coef(c, lay, r, &coef, st));
        WCK(c, launch_sub_f64(gbar, coef, gout, N, st));
        return WAM_OK;
    } catch (...) {
        return fail(c, WAM_ERR_OOM, "host allocation failed");
    }
}

wam_status wam_idiv_grad_batch(wam_ctx* c, int levels, int n, const float* beta, float lambda, double* loss,
                               float* grad, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (n < 0 || (n > 0 && (!beta || !loss || !grad))) return fail(c, WAM_ERR_ARG, "bad batch");
    for (int i = 0; i < n; ++i)
        WST(wam_idiv_grad(c, levels, beta + (size_t)i * c->N, lambda, loss + i, grad + (size_t)i * c->N, nullptr,
                          stream));
    return WAM_OK;
}

wam_status wam_project_coef_batch(wam_ctx* c, int levels, int n, const float* beta, float* p, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (n < 0 || (n > 0 && (!beta || !p))) return fail(c, WAM_ERR_ARG, "bad batch");
    for (int i = 0; i < n; ++i)
        WST(wam_project_coef(c, levels, beta + (size_t)i * c->N, p + (size_t)i * c->M, stream));
    return WAM_OK;
}

wam_status wam_backproject_coef_batch(wam_ctx* c, int levels, int n, const float* s, float* g, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (n < 0 || (n > 0 && (!s || !g))) return fail(c, WAM_ERR_ARG, "bad batch");
    for (int i = 0; i < n; ++i)
        WST(wam_backproject_coef(c, levels, s + (size_t)i * c->M, g + (size_t)i * c->N, stream));
    return WAM_OK;
}

wam_status wam_phi_split_project(wam_ctx* c, int levels, const float* gbar, const float* dplus,
                                 const float* dminus, const float* qhat, float* out, void* stream)
{
    if (!c) return WAM_ERR_ARG;
    if (c->g.kind == WAM_CONE3D_FLAT_CIRCULAR) return fail(c, WAM_ERR_ARG, "not available for cone-beam contexts");
    if (!gbar || !dplus || !dminus || !out) return fail(c, WAM_ERR_ARG, "null pointer");
    Layout lay;
    WST(make_layout(c, levels, &lay));
    Geom<float> g;
    WST(make_geom<float>(c, &g));
    WCK(c, launch_phi_project(g, lay, gbar, dplus, dminus, qhat, out, as_stream(stream)));
    return WAM_OK;
}

}  // extern "C"
