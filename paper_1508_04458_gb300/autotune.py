"""Autotuner of libwam's back-projector work split (WAM_TUNE_BACK_CTAS_PER_SM).

For a geometry class (image side and view count rounded to buckets) it
times a short multiresolution reconstruction per candidate with the
library's own CUDA-event profile (k_backproject time per launch) and keeps
the fastest; results are cached in a JSON file keyed by the class and the
device name.  The knob only changes how views are split across CTAs (the
order of fixed partial sums), never what is computed.
"""
from __future__ import annotations

import json
import os
from typing import Dict, Optional, Sequence

from . import wam

CANDIDATES = (4.0, 8.0, 16.0, 32.0, 64.0, 128.0)


def geometry_class(g) -> str:
    side = 1 << max(0, (max(g.nx, g.ny) - 1).bit_length())
    vb = 1 << max(0, (g.n_views * g.n_bins - 1).bit_length())
    return "k%d_s%d_r%d" % (g.kind, side, vb)


def _device_name() -> str:
    import torch
    return torch.cuda.get_device_name(0).replace(" ", "_")


def measure(ctx: "wam.Context", value: float, levels: int, n_iters: int, expand_at, tau) -> float:
    """k_backproject ms per launch with the knob at `value`."""
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, float(value)))
    ctx.reconstruct(levels, n_iters, expand_at, tau, device_out=True)      # warm-up
    ctx.profile(mode=wam.WAM_PROFILE_TIME)
    ctx.reconstruct(levels, n_iters, expand_at, tau, device_out=True)
    st = ctx.stats()["backproject"]
    ctx.profile(False)
    return st["ms"] / max(1, st["launches"])


def tune(ctx: "wam.Context", levels: int = 4, n_iters: int = 12, expand_at=(2, 4, 6, 8),
         tau=(0.1, 0.03, 0.01, -1.0), candidates: Sequence[float] = CANDIDATES,
         cache: Optional[str] = None) -> float:
    """Best knob value for ctx's geometry class (cached); ctx is left set to it.
    ctx must have data set."""
    key = geometry_class(ctx.geom) + "@" + _device_name()
    table: Dict[str, dict] = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
    if key in table:
        best = float(table[key]["back_ctas_per_sm"])
    else:
        times = {c: measure(ctx, c, levels, n_iters, expand_at, tau) for c in candidates}
        best = min(times, key=times.get)
        table[key] = {"back_ctas_per_sm": best, "ms_per_launch": {str(k): v for k, v in times.items()}}
        if cache:
            tmp = cache + ".tmp"
            with open(tmp, "w") as f:
                json.dump(table, f, indent=1, sort_keys=True)
            os.replace(tmp, cache)
    ctx.check(wam.wam_set_tuning(ctx.h, wam.WAM_TUNE_BACK_CTAS_PER_SM, best))
    return best
