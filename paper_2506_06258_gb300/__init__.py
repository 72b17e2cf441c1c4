"""GB300-native restarted PDHCG for linear Fisher markets and the Arrow-Debreu
fixed point (Liu, Huang, Li, Ge, Ye, arXiv 2506.06258).

The compute path is ``libpdhcg.so`` (hand-written CUDA for sm_103a, C ABI in
``include/pdhcg.h``); :mod:`capi` binds it with the same names and
:mod:`api` adds a small PyTorch-facing layer.  :mod:`synth` generates seeded
synthetic markets.
"""
__all__ = ["api", "capi", "synth", "build"]
