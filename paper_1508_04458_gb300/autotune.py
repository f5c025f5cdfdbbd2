"""Autotuner of libwam's tile shapes, per geometry class.

Two shapes are tuned, each by timing a short multiresolution reconstruction
per candidate with the library's own CUDA-event profile:

* the back-projector's views per CTA (WAM_TUNE_BACK_CTAS_PER_SM: the launch
  aims at that many 256-thread CTAs per SM by splitting every block list's
  views into ranges), timed on k_backproject's ms per launch;
* the forward projector's staged image tile (WAM_TUNE_FWD_STAGE_ROWS: 16, 24
  or 32 strips of 160 cells per shared-memory stage, or 0 for no staging),
  timed on the forward's ms per launch.

A geometry class is the image side and the ray count rounded up to powers of
two; results are cached in a JSON file keyed by the class and the device
name.  The back-projector knob only changes how views are split across CTAs
(the order of fixed partial sums), the forward knob nothing that is
computed.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

from . import wam

CANDIDATES = (4.0, 8.0, 16.0, 32.0, 64.0, 128.0)
STAGE_ROWS = (0, 16, 24, 32)


def geometry_class(g) -> str:
    side = 1 << max(0, (max(g.nx, g.ny) - 1).bit_length())
    vb = 1 << max(0, (g.n_views * g.n_bins - 1).bit_length())
    return "k%d_s%d_r%d" % (g.kind, side, vb)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(0).replace(" ", "_")


def _timed(ctx: "wam.Context", kernel: str, levels: int, n_iters: int, expand_at, tau, reps: int = 3) -> float:
    """ms per launch of one kernel class: the fastest of `reps` profiled
    reconstructions after a warm-up (close candidates differ by a few
    percent, about the spread of a single run)."""
    ctx.reconstruct(levels, n_iters, expand_at, tau, device_out=True)      # warm-up
    best = float("inf")
    for _ in range(reps):
        ctx.profile(mode=wam.WAM_PROFILE_TIME)
        ctx.reconstruct(levels, n_iters, expand_at, tau, device_out=True)
        st = ctx.stats()[kernel]
        ctx.profile(False)
        best = min(best, st["ms"] / max(1, st["launches"]))
    return best


def measure(ctx: "wam.Context", value: float, levels: int, n_iters: int, expand_at, tau) -> float:
    """k_backproject ms per launch with the back-projector knob at `value`."""
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, float(value)))
    return _timed(ctx, "backproject", levels, n_iters, expand_at, tau)


def measure_forward(ctx: "wam.Context", rows: int, levels: int, n_iters: int, expand_at, tau) -> float:
    """The forward's ms per launch with the staged tile at `rows` strips (0: none)."""
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, float(rows)))
    return _timed(ctx, "forward", levels, n_iters, expand_at, tau)


def tune(ctx: "wam.Context", levels: int = 4, n_iters: int = 12, expand_at=(2, 4, 6, 8),
         tau=(0.1, 0.03, 0.01, -1.0), candidates: Sequence[float] = CANDIDATES,
         stage_rows: Sequence[int] = STAGE_ROWS, cache: Optional[str] = None) -> Dict[str, float]:
    """Best tile shapes for ctx's geometry class (cached); ctx is left set to
    them.  Returns {"back_ctas_per_sm": ..., "fwd_stage_rows": ...}.  ctx
    must have data set."""
    key = geometry_class(ctx.geom) + "@" + _device_name()
    table: Dict[str, dict] = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    entry = table.get(key)
    if entry is None or "fwd_stage_rows" not in entry:
        times = {c: measure(ctx, c, levels, n_iters, expand_at, tau) for c in candidates}
        best = min(times, key=times.get)
        ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, best))
        ftimes = {r: measure_forward(ctx, r, levels, n_iters, expand_at, tau) for r in stage_rows}
        rows = min(ftimes, key=ftimes.get)
        entry = {"back_ctas_per_sm": best, "ms_per_launch": {str(k): v for k, v in times.items()},
                 "fwd_stage_rows": rows, "fwd_ms_per_launch": {str(k): v for k, v in ftimes.items()}}
        table[key] = entry
        if cache:
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
    out = {"back_ctas_per_sm": float(entry["back_ctas_per_sm"]), "fwd_stage_rows": int(entry["fwd_stage_rows"])}
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, out["back_ctas_per_sm"]))
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_FWD_STAGE_ROWS, float(out["fwd_stage_rows"])))
    return out
