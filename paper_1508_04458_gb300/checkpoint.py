"""Reader of the checkpoint files written by wam_checkpoint (host only, no
GPU): the state of Algorithm 1 after some iterations, i.e. the coefficient
vector beta, the tree masks and the cost history, with the geometry and the
schedule that produced them.  The layout is the one documented beside
wam_checkpoint in include/wam.h (little endian, CRC-32 at the end)."""
from __future__ import annotations

import struct
import zlib

import numpy as np

MAGIC = b"WAMCKPT1"
INT_FIELDS = ("kind", "nx", "ny", "nz", "n_views", "n_bins", "n_rows", "levels", "dims", "zsum_criterion",
              "precision", "full_am", "n_expand", "iters_done", "expansions_done", "n_coef", "mask_bytes",
              "n_hist", "crc_d", "crc_I0", "n_subsets", "nonneg")
DBL_FIELDS = ("vx", "vy", "vz", "angle0", "angle_span", "bin_pitch", "row_pitch", "sod", "sdd", "dmax_clamp",
              "tuning", "lambda")


class CheckpointError(ValueError):
    pass


def parse(buf: bytes) -> dict:
    """Decode a checkpoint held in memory; raises CheckpointError when the
    magic, the version, the CRC or the sizes do not check out."""
    if len(buf) < 20 or buf[:8] != MAGIC:
        raise CheckpointError("not a checkpoint file (magic)")
    (crc,) = struct.unpack_from("<I", buf, len(buf) - 4)
    if zlib.crc32(buf[:-4]) & 0xFFFFFFFF != crc:
        raise CheckpointError("CRC mismatch")
    version, _ = struct.unpack_from("<II", buf, 8)
    if version not in (2, 3):
        raise CheckpointError("unsupported version %d" % version)
    dbl = DBL_FIELDS if version == 3 else DBL_FIELDS[:-1]     # version 2 has no lambda
    at = 16
    head = 8 * (len(INT_FIELDS) + len(dbl))
    if at + head > len(buf) - 4:
        raise CheckpointError("header truncated")
    out = dict(zip(INT_FIELDS, struct.unpack_from("<%dq" % len(INT_FIELDS), buf, at)))
    at += 8 * len(INT_FIELDS)
    out.update(zip(dbl, struct.unpack_from("<%dd" % len(dbl), buf, at)))
    out.setdefault("lambda", 0.0)
    out["version"] = version
    at += 8 * len(dbl)
    ne, n, mb, nh = out["n_expand"], out["n_coef"], out["mask_bytes"], out["n_hist"]
    if min(ne, n, mb, nh) < 0 or nh != out["iters_done"] + 1:
        raise CheckpointError("inconsistent header")
    need = 16 * ne + 8 * n + mb + 8 * nh
    if at + need != len(buf) - 4:
        raise CheckpointError("size does not match the header")
    out["expand_at"] = np.frombuffer(buf, "<i8", ne, at).astype(int).tolist()
    at += 8 * ne
    out["tau"] = np.frombuffer(buf, "<f8", ne, at).tolist()
    at += 8 * ne
    out["beta"] = np.frombuffer(buf, "<f8", n, at).copy()
    at += 8 * n
    out["masks"] = np.frombuffer(buf, np.uint8, mb, at).copy()
    at += mb
    out["hist"] = np.frombuffer(buf, "<f8", nh, at).copy()
    return out


def read(path: str) -> dict:
    with open(path, "rb") as f:
        return parse(f.read())
