"""CPU oracle for the multiresolution AM method (FP64, plain and slow).

TEST INFRASTRUCTURE ONLY.  Only the tests, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` may import, call, link or execute anything in
this package.  It shares no code with the CUDA path and never calls it.

  system_matrix  H from exact ray/voxel intersection lengths (Siddon, C)
  haar, haar3d   orthonormal 2-D / 3-D Haar Omega: butterfly and explicit basis
  am             Algorithm 1 (wavelet AM with tree expansion) and plain AM

Every function cites the passage of the paper it follows.  Pins (tests that
tie the oracle to the mathematics rather than to itself) live in
tests/test_oracle_*.py.
"""
from . import am, haar, haar3d, system_matrix  # noqa: F401
