"""GB300-native multiresolution (wavelet-tree) alternating minimisation for
transmission CT (Degirmenci, O'Sullivan, Politte, arXiv 1508.04458).

`paper_1508_04458_gb300.wam` is the thin binding of the C-ABI library libwam
(CUDA kernels for sm_103a); `paper_1508_04458_gb300.inputs` draws the seeded
synthetic scans.  Importing `wam` loads libwam and fails loudly when it has
not been built.
"""
__all__ = ["inputs", "wam"]
