"""Benchmark: multiresolution (wavelet-tree) AM on the 2-D fan-beam baggage
workload (512x512 at 1 mm, 720 views over 360 deg, 1024 bins x 1.2 mm, I0 1e5,
4-level Haar tree with the adaptive threshold schedule, 100 iterations).

One step = one complete reconstruction through the C-ABI (precompute of
b = Phi^T d, then per iteration: tree-masked synthesis, ray-driven projection
with Beer's law and the FP64 I-divergence, split back-projection, AM update;
tree expansions with Z0 recomputation after iterations 8, 16, 32, 64).
value = AM iterations per second over all ranks (weak scaling: every rank
reconstructs its own seeded bag; no collective on the data path).

Also reported: the same rate end to end from host buffers (e2e), plain
full-image AM's rate, time to reach plain AM's final I-divergence, the
dominant kernel's roofline, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl wam|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-target I-divergence and AM iters/s, multires vs full AM; projector GB/s"
WORKLOAD = "fan512: 2-D fan beam 512x512 @1 mm, 720 views x 1024 bins, I0 1e5, L=4 Haar tree, 100 AM iterations"
L_LEVELS = 4
N_ITERS = 100
EXPAND_AT = (8, 16, 32, 64)
TAU = (0.1, 0.03, 0.01, -1.0)       # adaptive threshold: last expansion takes every leaf
TTT_MAX_ITERS = 300                 # multires iterations allowed to reach the target


def workload_config():
    """The benchmark workload, the same for the GPU arm and the reference arm."""
    return {"workload": WORKLOAD, "levels": L_LEVELS, "iterations": N_ITERS, "expand_after": list(EXPAND_AT),
            "tau": list(TAU), "seed": 1509, "l2": "flushed between steps (256 MiB write)",
            "cost_precision": "f64"}
K_MIN = 10                          # FP32 instructions per ray-rectangle intersection (floor)


def _env_int(name, default):
    try:
        return int(os.environ.get(name, default))
    except ValueError:
        return default


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p is not None:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except Exception:
                self.p.kill()
                out = ""
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------

def sample_scan(problem, view_stride: int):
    """Every view_stride-th view of the workload's scan: its geometry and counts."""
    from paper_1508_04458_gb300 import inputs as I
    g = problem.geom
    nv = g.n_views // view_stride
    sub = I.Geometry(**{**g.__dict__, "n_views": nv,
                        "angle_span": g.angle_span * (nv * view_stride) / g.n_views})
    return sub, np.ascontiguousarray(problem.d[::view_stride][:nv])


def sample_schedule(n_iters: int):
    """The benchmark's expansions at the same fractions of a shorter run."""
    exp_at = tuple(sorted(set(max(1, round(n_iters * e / N_ITERS)) for e in EXPAND_AT)))
    return exp_at, TAU[: len(exp_at)]


def oracle_sample(problem, view_stride: int, n_iters: int):
    """Time the FP64 oracle's Algorithm 1 on every view_stride-th view of the
    workload (full image; the schedule scaled to n_iters, i.e. expansions
    after n_iters * (8, 16, 32, 64) / 100 iterations, so the tree spends the
    same share of iterations at each size).  Its cost per iteration is linear
    in the number of rays, so the rate is scaled by view_stride to the full
    workload."""
    from oracle import am
    from oracle import system_matrix as smx

    g = problem.geom
    sub, d = sample_scan(problem, view_stride)
    t0 = time.perf_counter()
    H = smx.system_matrix(sub)
    exp_at, taus = sample_schedule(n_iters)
    r = am.wavelet_am(H, d, problem.I0, g.nx, g.ny, L_LEVELS, n_iters, expand_at=exp_at, taus=taus)
    dt = time.perf_counter() - t0
    rate = n_iters / dt / view_stride
    return rate, dt, r


def gpu_error_vs_oracle(problem, view_stride: int, n_iters: int, ref):
    """The GPU path (FP32, through the C-ABI) on the oracle's own sample scan
    and schedule, against the oracle's result: relative L2 error of mu, the
    largest relative deviation of the I-divergence history, and whether the
    final trees agree."""
    from paper_1508_04458_gb300 import wam
    sub, d = sample_scan(problem, view_stride)
    g = problem.geom
    exp_at, taus = sample_schedule(n_iters)
    ctx = wam.Context(sub)
    ctx.set_data(d.astype(np.float32), problem.I0)
    mu, hist, masks, st = ctx.reconstruct(L_LEVELS, n_iters, exp_at, taus, precision=32)
    ctx.close()
    ref_masks = np.concatenate([ref.tree[l - 1].astype(np.uint8).ravel() for l in range(L_LEVELS, 0, -1)])
    mu_rel = float(np.linalg.norm(mu.astype(np.float64) - ref.mu.ravel()) / np.linalg.norm(ref.mu))
    cost_rel = float(np.max(np.abs(hist - ref.cost) / np.abs(ref.cost)))
    return {"mu_rel_l2": mu_rel, "idiv_max_rel": cost_rel, "trees_equal": bool(np.array_equal(masks, ref_masks)),
            "status": int(st), "bound": {"mu_rel_l2": 1e-4, "idiv_max_rel": 1e-4},
            "sample": "the cpu_baseline sample: every %dth view (%d of %d), full %dx%d image, %d iterations, "
                      "expansions after %s" % (view_stride, sub.n_views, g.n_views, g.nx, g.ny, n_iters,
                                               list(exp_at))}


def run_reference(args, problem, world):
    rank = _env_int("RANK", 0)
    if rank != 0:
        return
    stride, iters = 30, 25
    for _ in range(args.warmup):
        oracle_sample(problem, stride, iters)
    times = []
    for _ in range(args.steps):
        rate, dt, _ = oracle_sample(problem, stride, iters)
        times.append(dt)
    total = sum(times)
    value = args.steps * iters / total / stride
    cores = os.cpu_count()
    sample = ("every %dth view (%d of %d), full 512x512 image, %d iterations, expansions at the same "
              "fractions of the run; rate scaled by %d" % (stride, problem.geom.n_views // stride,
                                                          problem.geom.n_views, iters, stride))
    line = {"metric": METRIC, "value": value, "unit": "AM iters/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(),
            "cpu_baseline": {"value": value, "unit": "AM iters/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "AM iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def difference_image(problem, pair, save_dir=None):
    """The analogue of the paper's Figs 2-4 (Results section): the images of
    plain AM after k iterations and of multiresolution AM after the j
    iterations it needs to reach the same I-divergence, and their difference
    (multires minus plain).  Summaries over the true phantom's structure:
    the edge band (pixels whose 3x3 neighbourhood in the rasterised phantom
    spans more than 0.005 /mm) and the flat regions (the other pixels inside
    the objects), the difference's RMS in each, and each image's mean
    gradient magnitude in the edge band (a sharper edge has a larger one)."""
    k, j, mu_plain, mu_mr = pair
    g = problem.geom
    a = mu_plain.reshape(g.ny, g.nx).astype(np.float64)
    m = mu_mr.reshape(g.ny, g.nx).astype(np.float64)
    t = np.asarray(problem.mu_true, dtype=np.float64).reshape(g.ny, g.nx)
    pad = np.pad(t, 1, mode="edge")
    win = np.stack([pad[dy:dy + g.ny, dx:dx + g.nx] for dy in range(3) for dx in range(3)])
    edge = (win.max(axis=0) - win.min(axis=0)) > 0.005
    flat = (~edge) & (t > 0.005)
    diff = m - a

    def grad(x):
        gy, gx = np.gradient(x)
        return np.hypot(gx, gy)

    rms = lambda x, sel: float(np.sqrt(np.mean(x[sel] ** 2))) if sel.any() else None
    out = {"plain_am_iters": k, "multires_iters": j, "edge_pixels": int(edge.sum()),
           "flat_pixels": int(flat.sum()), "rms_diff_edge": rms(diff, edge), "rms_diff_flat": rms(diff, flat),
           "rms_err_edge": {"plain_am": rms(a - t, edge), "multires": rms(m - t, edge)},
           "rms_err_flat": {"plain_am": rms(a - t, flat), "multires": rms(m - t, flat)},
           "mean_grad_edge": {"plain_am": float(grad(a)[edge].mean()), "multires": float(grad(m)[edge].mean()),
                              "phantom": float(grad(t)[edge].mean())}}
    if save_dir:
        os.makedirs(save_dir, exist_ok=True)
        np.savez_compressed(os.path.join(save_dir, "equal_objective_images.npz"), plain_am=a.astype(np.float32),
                            multires=m.astype(np.float32), difference=diff.astype(np.float32),
                            edge=edge, flat=flat)
        out["saved"] = "equal_objective_images.npz"
    return out


def roofline_of(stats, sms: int, what: str = "ray-rectangle"):
    """ALU roofline of the dominant kernel class (forward or back-projector):
    its counted intersections per launch over its event-timed launch duration,
    against SMs x 128 FP32 lanes x the maximum SM clock / K_MIN."""
    dom = max(("forward", "backproject"), key=lambda k: stats[k]["ms"])
    sd = stats[dom]
    clk_mhz = float(_peaks().get("sm_max_mhz", 2070.0))
    peak = sms * 128 * clk_mhz * 1e6 / K_MIN / 1e9            # G intersections / s
    per_launch_work = sd["work"] / max(1, sd["launches"])
    per_launch_ms = sd["ms"] / max(1, sd["launches"])
    achieved = per_launch_work / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0
    return {"bound": "alu", "kernel": "k_" + dom, "achieved": achieved, "peak": peak,
            "unit": "G %s intersections/s" % what, "frac": achieved / peak if peak else None,
            "peak_basis": "%d SMs x 128 FP32 lanes x %.0f MHz (MEASURED_PEAKS sm_max_mhz) / %d "
                          "instructions per intersection" % (sms, clk_mhz, K_MIN),
            "work_per_launch": per_launch_work, "ms_per_launch": per_launch_ms}


def profiled(ctx, fn):
    """Per-kernel-class times (events only) and work (counters only, a second
    run) of one call of fn on ctx."""
    from paper_1508_04458_gb300 import wam
    ctx.profile(mode=wam.WAM_PROFILE_TIME)
    fn()
    st = ctx.stats()
    ctx.profile(mode=wam.WAM_PROFILE_WORK)
    fn()
    w = ctx.stats()
    ctx.profile(False)
    for k in st:
        st[k]["work"] = w[k]["work"]
    return st


def run_wam(args, problem, world, rank, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1508_04458_gb300 import wam

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    g = problem.geom
    N, M = g.nx * g.ny, g.n_views * g.n_bins
    ctx = wam.Context(g)
    d_dev = torch.from_numpy(problem.d.astype(np.float32).ravel()).to(dev)
    ctx.set_data(d_dev, problem.I0)
    # the tile shapes for this geometry class (the autotuner's cached choice)
    tuned = None
    if not args.no_tune:
        from paper_1508_04458_gb300 import autotune
        cache = os.path.join(ROOT, "_build", "tune.json")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        tuned = autotune.tune(ctx, cache=cache)

    def step(n_iters=N_ITERS, levels=L_LEVELS, full=False, n_subsets=1):
        return ctx.reconstruct(levels, n_iters, () if full else EXPAND_AT, () if full else TAU,
                               precision=32, full_am=full, device_out=True, n_subsets=n_subsets)

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # > L2 (129 MB)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K complete reconstructions, L2 flushed between them,
    # no instrumentation inside the library (events only around each step)
    ctx.profile(False)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = wam.kernel_launches()
    with ClockSampler(local_rank) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            mu, hist, masks, st = step()
            ends[k].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    launches = wam.kernel_launches() - launches0
    # the kernel-timing pass: K more steps of the same workload (L2 flushed
    # between them) with CUDA events on the library's stream around every
    # kernel class, for the per-kernel times and the roofline
    ctx.profile(mode=wam.WAM_PROFILE_TIME)
    for k in range(args.steps):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    stats = ctx.stats()
    # the same step once more with the kernels' work counters (outside the
    # timed region: counting adds instructions); the work is deterministic
    ctx.profile(mode=wam.WAM_PROFILE_WORK)
    step()
    work1 = ctx.stats()
    ctx.profile(False)
    for k in stats:
        stats[k]["work"] = work1[k]["work"] * args.steps
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    dev_ms = float(sum(step_ms))
    t_max = torch.tensor([dev_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    dev_ms_max = float(t_max.item())
    value = world * args.steps * N_ITERS / (dev_ms_max / 1e3)
    hist_mr = hist.cpu().numpy()

    # ---- plain full-image AM and time to target (outside the timed region)
    def timed(fn):
        torch.cuda.synchronize()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        out = fn()
        b.record(stream)
        torch.cuda.synchronize()
        return out, a.elapsed_time(b)

    step(full=True, levels=0)
    (mu_f, hist_f, _, _), full_ms = timed(lambda: step(full=True, levels=0))
    hist_f = hist_f.cpu().numpy()
    target = float(hist_f[-1]) * (1.0 + 1e-3)
    (_, hist_long, _, _), long_ms = timed(lambda: step(n_iters=TTT_MAX_ITERS))
    hist_long = hist_long.cpu().numpy()
    hit = np.nonzero(hist_long <= target)[0]
    ttt_mr = None
    j_hit = None
    if hit.size:
        j_hit = int(hit[0])
        _, ttt_mr = timed(lambda: step(n_iters=j_hit))
    # plain AM's own time to its final value is its full run
    (_, _, _, _), full_ms2 = timed(lambda: step(full=True, levels=0))
    # objective-versus-time comparison: time for each method to reach plain
    # AM's cost after k iterations (+1e-3), k = 10, 20, 50, 100
    curve = []
    equal_pair = None
    for k in (10, 20, 50, 100):
        tgt = float(hist_f[k]) * (1.0 + 1e-3)
        (mu_k, _, _, _), t_full = timed(lambda: step(n_iters=k, full=True, levels=0))
        jh = np.nonzero(hist_long <= tgt)[0]
        t_mr = None
        if jh.size:
            (mu_j, _, _, _), t_mr = timed(lambda: step(n_iters=int(jh[0])))
            equal_pair = (k, int(jh[0]), mu_k.cpu().numpy(), mu_j.cpu().numpy())
        curve.append({"full_am_iters": k, "target_idiv": tgt, "full_am_ms": t_full,
                      "multires_iters": int(jh[0]) if jh.size else None, "multires_ms": t_mr})
    difference = difference_image(problem, equal_pair, args.save_dir) if equal_pair else None

    # ---- ordered subsets of views (the Conclusion's combination with ordered
    # subsets): the same schedules with S interleaved view subsets, time to
    # plain AM's final cost (+1e-3)
    def os_run(full, n_sub, n_max):
        step(n_iters=N_ITERS, full=full, levels=0 if full else L_LEVELS, n_subsets=n_sub)
        (_, h100, _, _), ms100 = timed(lambda: step(n_iters=N_ITERS, full=full, levels=0 if full else L_LEVELS,
                                                    n_subsets=n_sub))
        h = h100.cpu().numpy()
        if n_max > N_ITERS:
            (_, hl, _, _), _ = timed(lambda: step(n_iters=n_max, full=full, levels=0 if full else L_LEVELS,
                                                  n_subsets=n_sub))
            h = hl.cpu().numpy()
        jh = np.nonzero(h <= target)[0]
        t_hit = None
        if jh.size:
            _, t_hit = timed(lambda: step(n_iters=int(jh[0]), full=full, levels=0 if full else L_LEVELS,
                                          n_subsets=n_sub))
        return {"n_subsets": n_sub, "iters_per_s": N_ITERS / (ms100 / 1e3),
                "idiv_after_%d" % N_ITERS: float(h100.cpu().numpy()[-1]),
                "iters_to_target": int(jh[0]) if jh.size else None, "time_to_target_ms": t_hit}
    ordered = {"multires": os_run(False, 16, TTT_MAX_ITERS), "full_am": os_run(True, 8, N_ITERS)}

    # ---- the projector pair at full resolution (plain AM's kernels): per-launch
    # time (events), exact nonzero intersections (counters, a separate run),
    # and the bandwidth a stored sparse H (8 B per nonzero) would need to match
    ctx.profile(mode=wam.WAM_PROFILE_TIME)
    step(full=True, levels=0)
    t_st = ctx.stats()
    ctx.profile(mode=wam.WAM_PROFILE_WORK)
    step(full=True, levels=0)
    w_st = ctx.stats()
    ctx.profile(False)
    projector = {}
    for k in ("forward", "backproject"):
        nl = max(1, t_st[k]["launches"])
        ms_l = t_st[k]["ms"] / nl
        nnz = w_st[k]["work"] / nl
        projector[k] = {"ms_per_launch": ms_l, "intersections_per_launch": nnz,
                        "G_intersections_per_s": nnz / (ms_l * 1e6) if ms_l > 0 else None,
                        "stored_matrix_equiv_GBps": 8.0 * nnz / (ms_l * 1e6) if ms_l > 0 else None}

    # ---- e2e through the C-ABI from host buffers
    d_host = np.ascontiguousarray(problem.d.astype(np.float32).ravel())
    torch.cuda.synchronize()
    e0 = time.perf_counter()
    for _ in range(args.steps):
        ctx.set_data(d_host, problem.I0)
        mu_h, hist_h, masks_h, _ = ctx.reconstruct(L_LEVELS, N_ITERS, EXPAND_AT, TAU, precision=32)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - e0
    e2e = {"value": args.steps * N_ITERS / e2e_s, "unit": "AM iters/s",
           "h2d_bytes_per_step": int(d_host.nbytes + 4),
           "d2h_bytes_per_step": int(mu_h.nbytes + hist_h.nbytes + masks_h.nbytes)}
    if world > 1:
        t = torch.tensor([e2e_s], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e["value"] = world * args.steps * N_ITERS / float(t.item())

    # ---- roofline of the dominant kernel (ALU bound: ray-rectangle intersections)
    peaks = _peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    roofline = roofline_of(stats, sms)
    dom = roofline["kernel"][2:]
    per_launch_ms = roofline["ms_per_launch"]
    traffic = None
    tpath = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tpath):
        try:
            tj = json.load(open(tpath))
            traffic = tj.get(dom, {}).get("dram_bytes_per_launch")
        except Exception:
            traffic = None
    roofline["traffic"] = traffic
    if traffic and per_launch_ms > 0:
        # the HBM side of the same kernel: its DRAM bytes per launch (ncu, cold replay) over its live
        # launch time, against the measured copy rate -- small, since the working set lives in L2
        gbps = traffic / (per_launch_ms / 1e3) / 1e9
        hbm = float(peaks.get("hbm_gbs", 6746.0))
        roofline["dram"] = {"GBps": gbps, "peak_GBps": hbm, "frac": gbps / hbm,
                            "basis": "dram__bytes per launch (ncu) / live launch time; peak = MEASURED_PEAKS hbm_gbs"}

    # ---- CPU oracle on a bounded sample (rank 0, N = 1 only)
    cpu = None
    err_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu:
        stride, iters = 15, 25
        rate, dt, ref = oracle_sample(problem, stride, iters)
        cpu = {"value": rate, "unit": "AM iters/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": "every %dth view (%d of %d), full 512x512 image, %d iterations, expansions at the "
                         "same fractions of the run, %.1f s; rate scaled by %d" % (stride, g.n_views // stride,
                                                                                 g.n_views, iters, dt, stride)}
        err_vs_oracle = gpu_error_vs_oracle(problem, stride, iters, ref)

    # ---- the other workloads, as compact sub-records (rank 0, one GPU)
    extra = {}
    if rank == 0 and world == 1 and not args.no_extra:
        for name, fn in (("cone256", sub_cone256), ("batch32", sub_batch32), ("autograd", sub_autograd)):
            with ClockSampler(local_rank) as ck:
                rec = fn(args, quick=True)
            rec["clocks"] = ck.summary()
            extra[name] = rec

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "AM iters/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": dev_ms_max / args.steps,
            "ms_per_step_median": float(np.median(step_ms)), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": workload_config(), "tile_shapes": tuned,
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
            "roofline": roofline, "cpu_baseline": cpu, "err_vs_oracle": err_vs_oracle,
            "multires": {"final_idiv": float(hist_mr[-1]), "ms_per_iter": dev_ms_max / args.steps / N_ITERS,
                         "time_to_target_ms": ttt_mr, "iters_to_target": j_hit,
                         "idiv_after_%d" % TTT_MAX_ITERS: float(hist_long[-1]),
                         "ms_%d_iters" % TTT_MAX_ITERS: long_ms},
            "full_am": {"iters_per_s": N_ITERS / (full_ms2 / 1e3), "final_idiv": float(hist_f[-1]),
                        "ms_per_iter": full_ms2 / N_ITERS, "time_to_target_ms": full_ms2},
            "target_idiv": target,
            "time_to_equal_objective": curve,
            "difference_at_equal_objective": difference,
            "ordered_subsets": ordered,
            "projector": projector,
            "clamp_hits_per_reconstruction": int(work1["update"]["work"]),
            "kernels": {k: {"ms": round(v["ms"], 3), "launches": v["launches"], "work": v["work"]}
                        for k, v in stats.items()},
            "wall_s_timed": wall,
            **extra,
        }
        print(json.dumps(line), flush=True)
    ctx.close()


def _timed(fn, stream=None):
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    out = fn()
    b.record()
    torch.cuda.synchronize()
    return out, a.elapsed_time(b)


def sub_batch32(args, quick: bool = False):
    """32 seeded bags of uneven size (256^2..768^2, 360..1440 views,
    512..1536 bins, I0 1e4..1e5), 100 multiresolution iterations each:
    batched (one CUDA graph per tree epoch) against the per-bag loop."""
    import torch
    from paper_1508_04458_gb300 import autotune, inputs as I, wam
    bags = I.batch_bags(32, device="cuda")
    ctxs = []
    for p in bags:
        c = wam.Context(p.geom)
        c.set_data(torch.from_numpy(p.d.astype(np.float32).ravel()).cuda(), p.I0)
        ctxs.append(c)
    tuned = {}
    if not args.no_tune:
        cache = os.path.join(ROOT, "_build", "tune.json")
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        for c in ctxs:
            tuned[autotune.geometry_class(c.geom)] = autotune.tune(c, cache=cache)
    loop = lambda: [c.reconstruct(L_LEVELS, N_ITERS, EXPAND_AT, TAU, device_out=True) for c in ctxs]
    batch = lambda: wam.reconstruct_batch(ctxs, L_LEVELS, N_ITERS, EXPAND_AT, TAU, use_graph=wam.BATCH_GRAPH)
    persistent = lambda: wam.reconstruct_batch(ctxs, L_LEVELS, N_ITERS, EXPAND_AT, TAU,
                                               use_graph=wam.BATCH_PERSISTENT)
    steps = 2 if quick else args.steps
    for _ in range(1 if quick else max(1, args.warmup)):
        loop()
        batch()
        persistent()
    t_loop = min(_timed(loop)[1] for _ in range(steps))
    t_graph = min(_timed(batch)[1] for _ in range(steps))
    t_batch = min(_timed(persistent)[1] for _ in range(steps))
    # kernel classes of one pass over the bags (the same kernels the batch runs)
    agg = None
    for c in ctxs:
        st = profiled(c, lambda: c.reconstruct(L_LEVELS, N_ITERS, EXPAND_AT, TAU, device_out=True))
        if agg is None:
            agg = st
        else:
            for k in agg:
                for f in ("ms", "launches", "work"):
                    agg[k][f] += st[k][f]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    iters = 32 * N_ITERS
    out = {"workload": "batch32: 32 fan-beam bags 256..768 px, 360..1440 views, 512..1536 bins, "
                       "L=4, 100 iterations; persistent multi-bag kernels, one graph per epoch with per-bag "
                       "stream branches, and the per-bag loop (iters_per_s: the fastest batched mode)",
           "unit": "AM iters/s (all bags)",
           "iters_per_s": iters / (min(t_batch, t_graph) / 1e3),
           "fastest_mode": "persistent" if t_batch < t_graph else "graph_per_bag_branches",
           "persistent": iters / (t_batch / 1e3),
           "batched_graph": iters / (t_graph / 1e3), "per_bag_loop": iters / (t_loop / 1e3),
           "ms_persistent": t_batch, "ms_graph": t_graph, "ms_loop": t_loop, "speedup": t_loop / t_batch,
           "speedup_graph": t_loop / t_graph,
           "roofline": roofline_of(agg, sms),
           "autotuned_back_ctas_per_sm": tuned, "pixels": int(sum(p.geom.nx * p.geom.ny for p in bags)),
           "rays": int(sum(p.geom.n_views * p.geom.n_bins for p in bags))}
    for c in ctxs:
        c.close()
    return out


def sub_autograd(args, quick: bool = False):
    """The differentiation workload: a batch of 8 coefficient vectors on a
    256x256 fan-beam bag (360 views x 512 bins, L = 4 Haar levels): the
    I-divergence + l1 loss with its gradient for the whole batch, and 10
    unrolled AM steps (full tree) differentiated with respect to beta^(0)."""
    import torch
    from paper_1508_04458_gb300 import inputs as I, wam
    from paper_1508_04458_gb300.autograd import AMUnroll, IDivLoss, Operators
    prob = I.problem_fan(256, 360, 512, 1e5, seed=I.SEED_BASE + 3)
    L, B, steps = 4, 8, 10
    ctx = wam.Context(prob.geom)
    ctx.set_data(prob.d.astype(np.float32), prob.I0)
    ops = Operators(ctx, L)
    ops.setup(torch.from_numpy(prob.d.astype(np.float32).ravel()).cuda())
    rng = np.random.default_rng(4)
    N = prob.geom.nx * prob.geom.ny
    nA = (prob.geom.nx >> L) * (prob.geom.ny >> L)
    betas = np.zeros((B, N), np.float32)
    betas[:, :nA] = 0.02 * (1 << L)
    betas[:, nA:] = rng.normal(0.0, 1e-3, (B, N - nA))
    bt = torch.tensor(betas, device="cuda", requires_grad=True)

    def loss_grad():
        bt.grad = None
        IDivLoss.apply(bt, ops, 1.0).sum().backward()

    def unrolled():
        b0 = torch.tensor(betas[0], device="cuda", requires_grad=True)
        IDivLoss.apply(AMUnroll.apply(b0, ops, steps), ops, 1.0).backward()

    out = {}
    reps = 3 if quick else args.steps
    for name, fn, items in (("loss_grad_batch8", loss_grad, B), ("unroll10_grad", unrolled, 1)):
        for _ in range(2 if quick else max(2, args.warmup)):
            fn()
        (_, ms) = _timed(lambda: [fn() for _ in range(reps)])
        out[name] = {"ms_per_call": ms / reps, "items_per_s": items * reps / (ms / 1e3)}
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    st = profiled(ctx, loss_grad)
    rec = {"workload": "autograd: batch 8 x 256x256 fan beam (360 views x 512 bins), L=4 Haar, "
                       "loss + l1 gradient; 10 unrolled AM steps with their gradient",
           "unit": "items/s", "iters_per_s": out["loss_grad_batch8"]["items_per_s"], **out,
           "roofline": roofline_of(st, sms)}
    ctx.close()
    return rec


def sub_cone256(args, quick: bool = False):
    """3-D circular cone beam 256x256x128 @1.5 mm, 900 views, 64 x 768,
    I0 5e4: plain AM and multiresolution AM (3-D Haar, L=3, expansions
    after 8, 16, 32) and the per-slice 2-D Haar mode, 60 iterations."""
    import torch
    from paper_1508_04458_gb300 import inputs as I, wam
    p = I.problem_cone256(device="cuda")
    ctx = wam.Context(p.geom)
    ctx.set_data(torch.from_numpy(p.d.astype(np.float32).ravel()).cuda(), p.I0)
    J, ea, tau = 60, (8, 16, 32), (0.1, 0.03, -1.0)
    modes = [("multires_3d_haar", dict(levels=3, n_iters=J, expand_at=ea, tau=tau, dims=3)),
             ("full_am", dict(levels=0, n_iters=J, full_am=True)),
             ("multires_per_slice", dict(levels=3, n_iters=J, expand_at=ea, tau=tau, dims=2, zsum=True))]
    if quick:
        modes = modes[:2]
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    res = {}
    for name, kw in modes:
        ctx.reconstruct(**kw, device_out=True)
        (mu, hist, _, st), ms = _timed(lambda: ctx.reconstruct(**kw, device_out=True))
        # the kernel split (events only) and the work (counters only) in two more runs
        k = profiled(ctx, lambda: ctx.reconstruct(**kw, device_out=True))
        h = hist.cpu().numpy()
        res[name] = {"ms": ms, "iters_per_s": J / (ms / 1e3), "status": st, "idiv0": float(h[0]),
                     "idiv_final": float(h[-1]), "roofline": roofline_of(k, sms, "ray-cell"),
                     "kernels": {n: {"ms": round(v["ms"], 2), "launches": v["launches"], "work": v["work"]}
                                 for n, v in k.items()}}
    ctx.close()
    return {"workload": "cone256: 256x256x128 @1.5 mm, 900 views x 64 rows x 768 bins, I0 5e4, 60 iterations",
            "unit": "AM iters/s", "iters_per_s": res["multires_3d_haar"]["iters_per_s"],
            "roofline": res["multires_3d_haar"]["roofline"], **res}


def profile_case(case: str, n: int = 256):
    """A case of the same kernels for kernel profiling: an n x n bag with
    n * 1.40625 views x 2n bins (256: 360 x 512; 512: 720 x 1024, the
    benchmark's own scan).  multires / full: two reconstructions of the
    benchmark's schedule (multiresolution AM / plain AM).  fulltree: one
    8-iteration multiresolution run whose expansions after iterations 1-4
    take every leaf, so launches 6 to 8 of the back-projector run the full
    4-level tree (the same items whatever the data); it prints the library's
    work count (child chords) and CUDA-event time per launch of that phase.
    forward: three pixel-basis forward projections of a constant image
    with the global-memory strip walk, then three with the walk staged in
    shared memory 24 strips at a time."""
    import json
    import torch
    from paper_1508_04458_gb300 import inputs as I
    from paper_1508_04458_gb300 import wam
    p = I.problem_fan(256, 360, 512, 1e5, seed=I.SEED_BASE + 3) if n == 256 else I.problem_fan512()
    ctx = wam.Context(p.geom)
    ctx.set_data(p.d.astype(np.float32), p.I0)
    if case == "fulltree":
        ea, tau = (1, 2, 3, 4), (-1.0, -1.0, -1.0, -1.0)
        ctx.reconstruct(4, 8, ea, tau, precision=32, device_out=True)
        torch.cuda.synchronize()
        per = {}
        for mode, key in ((wam.WAM_PROFILE_WORK, "work"), (wam.WAM_PROFILE_TIME, "ms")):
            for iters in (8, 6):
                ctx.profile(mode=mode)
                ctx.reconstruct(4, iters, ea, tau, precision=32, device_out=True)
                per[(key, iters)] = ctx.stats()["backproject"][key]
                ctx.profile(False)
        print(json.dumps({"case": "fulltree fan%d" % n,
                          "backproject_work_per_launch": (per[("work", 8)] - per[("work", 6)]) / 2,
                          "backproject_ms_per_launch": (per[("ms", 8)] - per[("ms", 6)]) / 2}))
    elif case == "forward":
        g = p.geom
        mu = torch.full((g.nx * g.ny,), 0.02, dtype=torch.float32, device="cuda")
        q = torch.empty(g.n_views * g.n_bins, dtype=torch.float32, device="cuda")
        cost = torch.empty(1, dtype=torch.float64, device="cuda")
        for rows in (0, 24):
            ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, float(rows)))
            for _ in range(3):
                ctx.check(wam.wam_forward(ctx.h, 0, None, wam.ptr(mu), wam.ptr(q), wam.ptr(cost),
                                          wam.current_stream()))
    else:
        for _ in range(2):
            if case == "full":
                ctx.reconstruct(0, N_ITERS, precision=32, full_am=True, device_out=True)
            else:
                ctx.reconstruct(L_LEVELS, N_ITERS, EXPAND_AT, TAU, precision=32, device_out=True)
    torch.cuda.synchronize()
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("wam", "reference"), default="wam")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle sample")
    ap.add_argument("--no-tune", action="store_true", help="batch32: skip the autotuner")
    ap.add_argument("--save-dir", default=None,
                    help="write the equal-objective images (plain AM, multires, difference) here as .npz")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the cone256 / batch32 / autograd sub-records of the default line")
    ap.add_argument("--workload", choices=("fan512", "batch32", "cone256", "autograd"), default="fan512",
                    help="fan512 (default): the benchmark line; batch32 / cone256 / autograd: secondary "
                         "measurements of the batched, 3-D cone-beam and differentiation paths "
                         "(one JSON line each)")
    ap.add_argument("--profile-case", choices=("multires", "full", "fulltree", "forward"), default=None,
                    help="kernel profiling cases on a fan-beam bag (--profile-n): two reconstructions "
                         "(multires or plain AM, print nothing); fulltree: the full 4-level tree, prints the "
                         "back-projector's work and time per launch; forward: pixel-basis projections, "
                         "unstaged then staged")
    ap.add_argument("--profile-n", type=int, choices=(256, 512), default=256,
                    help="image side of --profile-case (512: the benchmark's own bag and scan)")
    args = ap.parse_args()
    if args.profile_case:
        profile_case(args.profile_case, args.profile_n)
        return
    subs = {"batch32": sub_batch32, "cone256": sub_cone256, "autograd": sub_autograd}
    if args.workload in subs:
        print(json.dumps(subs[args.workload](args)), flush=True)
        return

    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local_rank = _env_int("LOCAL_RANK", 0)
    from paper_1508_04458_gb300 import inputs as I
    problem = I.problem_fan512(seed=I.SEED_BASE + 1 + rank)

    if args.impl == "reference":
        run_reference(args, problem, world)
        return
    import torch
    import torch.distributed as dist
    if world > 1:
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        run_wam(args, problem, world, rank, local_rank)
    finally:
        if world > 1:
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
