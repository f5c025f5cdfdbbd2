"""The checkpoint file layout on the host: a file assembled here field by
field from the documented layout decodes to the same values, and a flipped
byte, a truncation or a wrong magic is rejected."""
import struct
import zlib

import numpy as np
import pytest

from paper_1508_04458_gb300 import checkpoint as ck


def _assemble(ints, dbls, expand_at, tau, beta, masks, hist):
    version = 3 if len(dbls) == 12 else 2          # version 3 adds lambda after tuning
    b = bytearray(b"WAMCKPT1") + struct.pack("<II", version, 0)
    b += struct.pack("<22q", *ints) + struct.pack("<%dd" % len(dbls), *dbls)
    b += struct.pack("<%dq" % len(expand_at), *expand_at) + struct.pack("<%dd" % len(tau), *tau)
    b += np.asarray(beta, "<f8").tobytes() + np.asarray(masks, np.uint8).tobytes()
    b += np.asarray(hist, "<f8").tobytes()
    b += struct.pack("<I", zlib.crc32(bytes(b)) & 0xFFFFFFFF)
    return bytes(b)


def _example():
    rng = np.random.default_rng(0)
    nx, ny, L = 16, 8, 2
    N = nx * ny
    mb = (nx >> 1) * (ny >> 1) + (nx >> 2) * (ny >> 2)
    beta = rng.normal(size=N)
    masks = (rng.random(mb) < 0.5).astype(np.uint8)
    hist = np.sort(rng.random(7))[::-1] * 1e5
    ints = [1, nx, ny, 1, 30, 41, 1, L, 2, 0, 32, 0, 2, 6, 1, N, mb, 7, 123456789, 987654321, 4, 0]
    dbls = [1.0, 1.0, 1.0, 0.0, 6.283185307179586, 1.2, 1.0, 500.0, 800.0, 30.0, 32.0, 0.25]
    return _assemble(ints, dbls, [3, 9], [0.1, -1.0], beta, masks, hist), beta, masks, hist


def test_round_trip():
    buf, beta, masks, hist = _example()
    c = ck.parse(buf)
    assert (c["nx"], c["ny"], c["levels"], c["iters_done"], c["expansions_done"]) == (16, 8, 2, 6, 1)
    assert c["expand_at"] == [3, 9] and c["tau"] == [0.1, -1.0]
    assert c["crc_d"] == 123456789 and c["sdd"] == 800.0 and c["tuning"] == 32.0 and c["n_subsets"] == 4
    assert c["nonneg"] == 0 and c["lambda"] == 0.25 and c["version"] == 3
    np.testing.assert_array_equal(c["beta"], beta)
    np.testing.assert_array_equal(c["masks"], masks)
    np.testing.assert_array_equal(c["hist"], hist)


@pytest.mark.parametrize("where", [0, 20, 200, -5])
def test_corruption_is_rejected(where):
    buf = bytearray(_example()[0])
    buf[where] ^= 0x40
    with pytest.raises(ck.CheckpointError):
        ck.parse(bytes(buf))


def test_truncation_is_rejected():
    buf = _example()[0]
    for n in (10, 100, len(buf) - 1):
        with pytest.raises(ck.CheckpointError):
            ck.parse(buf[:n])


def test_version_and_nonneg_field():
    buf, beta, masks, hist = _example()
    # the nonnegativity flag is the 22nd integer field
    b = bytearray(buf[:-4])
    struct.pack_into("<q", b, 16 + 8 * 21, 1)
    b += struct.pack("<I", zlib.crc32(bytes(b)) & 0xFFFFFFFF)
    assert ck.parse(bytes(b))["nonneg"] == 1
    # an older layout (version 1) is refused, CRC intact
    old = bytearray(buf[:-4])
    struct.pack_into("<I", old, 8, 1)
    old += struct.pack("<I", zlib.crc32(bytes(old)) & 0xFFFFFFFF)
    with pytest.raises(ck.CheckpointError):
        ck.parse(bytes(old))


def test_version_2_layout_reads_as_lambda_zero():
    # the earlier layout: 11 doubles (no lambda); it still decodes, with lambda = 0
    rng = np.random.default_rng(1)
    nx, ny, L = 8, 8, 1
    N, mb = nx * ny, (nx >> 1) * (ny >> 1)
    ints = [1, nx, ny, 1, 10, 17, 1, L, 2, 0, 32, 0, 0, 2, 0, N, mb, 3, 1, 2, 1, 0]
    dbls = [1.0, 1.0, 1.0, 0.0, 6.283185307179586, 1.2, 1.0, 500.0, 800.0, 30.0, 32.0]
    buf = _assemble(ints, dbls, [], [], rng.normal(size=N), np.zeros(mb, np.uint8), [3.0, 2.0, 1.0])
    c = ck.parse(buf)
    assert c["version"] == 2 and c["lambda"] == 0.0 and c["tuning"] == 32.0
