"""Thin Python binding of libwam (ctypes; argument marshalling only).

Every function of include/wam.h is exported here under the same name with
the same arguments (pointers as integers: use `ptr(tensor)` for torch
tensors, `hptr(ndarray)` for numpy arrays).  `Context` is a convenience
wrapper that owns a wam_ctx and converts torch tensors / numpy arrays; every
step of the method runs in libwam's CUDA kernels.

Importing this module loads libwam.so and raises ImportError when it has
not been built (python -c "import __graft_entry__ as g; g.build()").
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwam.so")

if not os.path.exists(LIB_PATH):
    raise ImportError("libwam.so is missing at %s: build it first "
                      "(paper_1508_04458_gb300/build.py)" % LIB_PATH)
lib = ctypes.CDLL(LIB_PATH)

WAM_OK = 0
WAM_ERR_ARG = -1
WAM_ERR_OOM = -2
WAM_ERR_CUDA = -3
WAM_ERR_TIMEOUT = -4
WAM_ERR_STATE = -5
WAM_ERR_IO = -6
WAM_WARN_NONMONOTONE = 1
WAM_MAX_LEVELS = 8
WAM_TUNE_BACK_CTAS_PER_SM = 1
WAM_TUNE_GRAPHS = 2
WAM_TUNE_FWD_STAGE_ROWS = 3
WAM_PROFILE_OFF, WAM_PROFILE_ALL, WAM_PROFILE_TIME, WAM_PROFILE_WORK = 0, 1, 2, 3


class wam_geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angle0", ctypes.c_double), ("angle_span", ctypes.c_double),
                ("n_bins", ctypes.c_int), ("n_rows", ctypes.c_int),
                ("bin_pitch", ctypes.c_double), ("row_pitch", ctypes.c_double),
                ("sod", ctypes.c_double), ("sdd", ctypes.c_double)]


class wam_schedule(ctypes.Structure):
    _fields_ = [("levels", ctypes.c_int), ("dims", ctypes.c_int), ("n_iters", ctypes.c_int),
                ("n_expand", ctypes.c_int), ("expand_at", ctypes.POINTER(ctypes.c_int)),
                ("tau", ctypes.POINTER(ctypes.c_double)), ("zsum_criterion", ctypes.c_int),
                ("precision", ctypes.c_int), ("full_am", ctypes.c_int), ("dmax_clamp", ctypes.c_double),
                ("n_subsets", ctypes.c_int), ("nonneg", ctypes.c_int), ("lambda_", ctypes.c_double)]


WAM_K_FORWARD, WAM_K_BACKPROJECT, WAM_K_UPDATE, WAM_K_Z0, WAM_K_SYNTH, WAM_K_TREE = range(6)
WAM_NKERNEL = 6
KERNEL_NAMES = ("forward", "backproject", "update", "z0", "synth", "tree")


class wam_stats(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_double * WAM_NKERNEL),
                ("launches", ctypes.c_ulonglong * WAM_NKERNEL),
                ("work", ctypes.c_ulonglong * WAM_NKERNEL)]


_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_S = ctypes.c_int  # wam_status

_PROTOS = {
    "wam_create": (_S, [ctypes.POINTER(wam_geometry), ctypes.POINTER(_P)]),
    "wam_destroy": (None, [_P]),
    "wam_last_error": (ctypes.c_char_p, [_P]),
    "wam_mask_bytes": (ctypes.c_size_t, [_P, _I]),
    "wam_mask_bytes_dims": (ctypes.c_size_t, [_P, _I, _I]),
    "wam_set_data": (_S, [_P, _P, _P, _I, _I, _P]),
    "wam_reconstruct": (_S, [_P, ctypes.POINTER(wam_schedule), _P, _P, _P, _I, _P]),
    "wam_project": (_S, [_P, _P, _P, _P]),
    "wam_project_f64": (_S, [_P, _P, _P, _P]),
    "wam_backproject": (_S, [_P, _P, _P, _P]),
    "wam_backproject_f64": (_S, [_P, _P, _P, _P]),
    "wam_haar": (_S, [_P, _I, _P, _P, _I, _P]),
    "wam_synthesize": (_S, [_P, _I, _P, _P, _P, _P]),
    "wam_forward": (_S, [_P, _I, _P, _P, _P, _P, _P]),
    "wam_forward_f64": (_S, [_P, _I, _P, _P, _P, _P, _P]),
    "wam_split_backproject": (_S, [_P, _I, _P, _P, _P, _P, _P]),
    "wam_z0": (_S, [_P, _I, _P, _P, _P]),
    "wam_update": (_S, [_P, _I, _P, _P, _P, _P, _P, _D, _P, _P]),
    "wam_expand": (_S, [_P, _I, _P, _D, _P, _P, _P]),
    "wam_am_delta": (_S, [ctypes.c_longlong, _P, _P, _P, _P, _D, _D, _D, _I, _P, _P, _P]),
    "wam_project_coef": (_S, [_P, _I, _P, _P, _P]),
    "wam_backproject_coef": (_S, [_P, _I, _P, _P, _P]),
    "wam_idiv_grad": (_S, [_P, _I, _P, ctypes.c_float, _P, _P, _P, _P]),
    "wam_am_derivs": (_S, [_P, _I, _P, _P, _P, _P, _D, _P, _P, _P]),
    "wam_phi_split_project": (_S, [_P, _I, _P, _P, _P, _P, _P, _P]),
    "wam_idiv_grad_batch": (_S, [_P, _I, _I, _P, ctypes.c_float, _P, _P, _P]),
    "wam_project_coef_batch": (_S, [_P, _I, _I, _P, _P, _P]),
    "wam_backproject_coef_batch": (_S, [_P, _I, _I, _P, _P, _P]),
    "wam_precompute_b": (_S, [_P, _I, _P, _P]),
    "wam_am_step_vjp": (_S, [_P, _I, _P, _P, _P, _D, _P, _P, _P]),
    "wam_backproject_static": (_S, [ctypes.POINTER(wam_geometry), _P, _P, _P]),
    "wam_reconstruct_batch": (_S, [ctypes.POINTER(_P), _I, ctypes.POINTER(wam_schedule), ctypes.POINTER(_P),
                                   ctypes.POINTER(_P), _I, _I, _P]),
    "wam_set_tuning": (_S, [_P, _I, _D]),
    "wam_checkpoint": (_S, [_P, ctypes.c_char_p]),
    "wam_resume": (_S, [_P, ctypes.c_char_p]),
    "wam_profile": (_S, [_P, _I]),
    "wam_get_stats": (_S, [_P, _P]),
    "wam_kernel_launches": (ctypes.c_ulonglong, []),
}

for _name, (_res, _args) in _PROTOS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f

EXPORTED = tuple(_PROTOS)


class WamError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("libwam status %d: %s" % (status, msg))
        self.status = status


def ptr(t) -> int:
    """Device (or host) address of a contiguous torch tensor; 0 for None."""
    if t is None:
        return 0
    assert t.is_contiguous(), "tensor must be contiguous"
    return t.data_ptr()


def hptr(a: Optional[np.ndarray]) -> int:
    if a is None:
        return 0
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def current_stream() -> int:
    import torch
    return torch.cuda.current_stream().cuda_stream


def geometry(g) -> wam_geometry:
    """wam_geometry from any object with the same field names."""
    return wam_geometry(*(getattr(g, f) for f, _ in wam_geometry._fields_))


def schedule(levels: int, n_iters: int, expand_at: Sequence[int] = (), tau: Sequence[float] = (),
             precision: int = 32, full_am: bool = False, clamp: float = 30.0, dims: int = 2,
             zsum: bool = False, n_subsets: int = 1, nonneg: bool = False, lam: float = 0.0):
    """wam_schedule plus the arrays it points to (keep the tuple alive)."""
    ea = (ctypes.c_int * max(1, len(expand_at)))(*expand_at)
    ta = (ctypes.c_double * max(1, len(tau)))(*tau)
    s = wam_schedule(levels=levels, dims=dims, n_iters=n_iters, n_expand=len(expand_at),
                     expand_at=ctypes.cast(ea, ctypes.POINTER(ctypes.c_int)),
                     tau=ctypes.cast(ta, ctypes.POINTER(ctypes.c_double)), zsum_criterion=1 if zsum else 0,
                     precision=precision, full_am=1 if full_am else 0, dmax_clamp=clamp, n_subsets=n_subsets,
                     nonneg=1 if nonneg else 0, lambda_=float(lam))
    return s, (ea, ta)


class Context:
    """Owns one wam_ctx for one scan geometry on the current CUDA device."""

    def __init__(self, geom):
        self.geom = geom
        self._g = geometry(geom)
        h = _P()
        st = wam_create(ctypes.byref(self._g), ctypes.byref(h))
        if st != WAM_OK:
            raise WamError(st, "wam_create failed (geometry rejected or no CUDA device)")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            wam_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, st: int, allow=(WAM_OK,)) -> int:
        if st not in allow:
            raise WamError(st, (wam_last_error(self.h) or b"").decode())
        return st

    def mask_bytes(self, levels: int, dims: int = 2) -> int:
        return int(wam_mask_bytes_dims(self.h, levels, dims))

    def set_data(self, d, I0, stream: Optional[int] = None):
        """d: numpy (host) or torch (device) float32 [V][B]; I0 scalar or array."""
        import torch
        if isinstance(d, torch.Tensor):
            scalar = not isinstance(I0, torch.Tensor)
            i0 = torch.tensor([float(I0)], dtype=torch.float32, device=d.device) if scalar else I0
            if scalar:
                i0 = i0.expand(1).contiguous()
            s = current_stream() if stream is None else stream
            return self.check(wam_set_data(self.h, ptr(d), ptr(i0), int(scalar), 1, s))
        d = np.ascontiguousarray(d, dtype=np.float32)
        scalar = np.ndim(I0) == 0
        i0 = np.ascontiguousarray(np.atleast_1d(np.asarray(I0, dtype=np.float32)))
        s = current_stream() if stream is None else stream
        return self.check(wam_set_data(self.h, hptr(d), hptr(i0), int(scalar), 0, s))

    def reconstruct(self, levels: int, n_iters: int, expand_at=(), tau=(), precision: int = 32,
                    full_am: bool = False, device_out: bool = False, stream: Optional[int] = None,
                    dims: int = 2, zsum: bool = False, n_subsets: int = 1, nonneg: bool = False,
                    lam: float = 0.0):
        """Run the method; returns (mu, idiv history, masks, status).  Cone-beam
        contexts: dims = 3 (3-D Haar) or dims = 2 with zsum (per-slice Haar).
        n_subsets > 1: ordered subsets of views (2-D).  nonneg: plain AM with
        mu >= 0 (each pixel's step ends at 0).  lam > 0: the L1 penalty on the
        detail coefficients (wam_schedule.lambda)."""
        import torch
        sc, keep = schedule(levels, n_iters, expand_at, tau, precision, full_am, dims=dims, zsum=zsum,
                            n_subsets=n_subsets, nonneg=nonneg, lam=lam)
        L = 0 if full_am else levels
        N = self.geom.nx * self.geom.ny * max(1, getattr(self.geom, "nz", 1))
        s = current_stream() if stream is None else stream
        if device_out:
            dt = torch.float32 if precision == 32 else torch.float64
            mu = torch.empty(N, dtype=dt, device="cuda")
            hist = torch.empty(n_iters + 1, dtype=torch.float64, device="cuda")
            masks = torch.empty(max(1, self.mask_bytes(L, dims)), dtype=torch.uint8, device="cuda")
            st = wam_reconstruct(self.h, ctypes.byref(sc), ptr(mu), ptr(hist), ptr(masks), 1, s)
        else:
            mu = np.empty(N, dtype=np.float32 if precision == 32 else np.float64)
            hist = np.empty(n_iters + 1, dtype=np.float64)
            masks = np.empty(max(1, self.mask_bytes(L, dims)), dtype=np.uint8)
            st = wam_reconstruct(self.h, ctypes.byref(sc), hptr(mu), hptr(hist), hptr(masks), 0, s)
        del keep
        self.check(st, allow=(WAM_OK, WAM_WARN_NONMONOTONE))
        return mu, hist, masks[: self.mask_bytes(L, dims)], st

    def checkpoint(self, path: str):
        """Write the state of the last finished reconstruct() to path."""
        return self.check(wam_checkpoint(self.h, os.fsencode(path)))

    def resume(self, path: str):
        """Load a checkpoint; the next reconstruct() continues from it."""
        return self.check(wam_resume(self.h, os.fsencode(path)))

    def profile(self, enable: bool = True, mode: Optional[int] = None):
        """Reset and enable (or stop) per-kernel event timing and work counting
        of reconstruct(); mode = WAM_PROFILE_TIME / _WORK selects one of them."""
        m = mode if mode is not None else (WAM_PROFILE_ALL if enable else WAM_PROFILE_OFF)
        self.check(wam_profile(self.h, m))

    def stats(self) -> dict:
        st = wam_stats()
        self.check(wam_get_stats(self.h, ctypes.byref(st)))
        return {name: {"ms": st.ms[k], "launches": int(st.launches[k]), "work": int(st.work[k])}
                for k, name in enumerate(KERNEL_NAMES)}


def kernel_launches() -> int:
    """Kernels launched by libwam in this process so far."""
    return int(wam_kernel_launches())


BATCH_DIRECT, BATCH_GRAPH, BATCH_PERSISTENT = 0, 1, 2


def reconstruct_batch(ctxs, levels: int, n_iters: int, expand_at=(), tau=(), use_graph=True,
                      stream: Optional[int] = None):
    """wam_reconstruct_batch on device outputs; returns ([mu], [hist], status).
    use_graph: False / BATCH_DIRECT, True / BATCH_GRAPH (one graph per tree
    epoch, every bag on its own stream branch) or BATCH_PERSISTENT (one graph
    per epoch of five multi-bag kernels, the forward and back-projector
    persistent over a work queue)."""
    import torch
    sc, keep = schedule(levels, n_iters, expand_at, tau, 32, False)
    n = len(ctxs)
    mus = [torch.empty(c.geom.nx * c.geom.ny, dtype=torch.float32, device="cuda") for c in ctxs]
    hists = [torch.empty(n_iters + 1, dtype=torch.float64, device="cuda") for _ in ctxs]
    harr = (_P * n)(*[c.h for c in ctxs])
    marr = (_P * n)(*[ptr(m) for m in mus])
    qarr = (_P * n)(*[ptr(h) for h in hists])
    s = current_stream() if stream is None else stream
    mode = int(use_graph) if not isinstance(use_graph, bool) else (1 if use_graph else 0)
    st = wam_reconstruct_batch(harr, n, ctypes.byref(sc), marr, qarr, 1, mode, s)
    del keep
    if st not in (WAM_OK, WAM_WARN_NONMONOTONE):
        msgs = [(wam_last_error(c.h) or b"").decode() for c in ctxs]
        raise WamError(st, "; ".join(m for m in msgs if m))
    return mus, hists, st
