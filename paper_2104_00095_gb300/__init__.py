"""GB300-native per-step grid update of the 3D reference map technique (arXiv 2104.00095).

The compute path lives in the CUDA library ``librmt.so`` (sources in ``csrc/``, C ABI in
``include/rmt.h``); :mod:`paper_2104_00095_gb300.rmt` is a thin ctypes binding with the same
names.  :mod:`paper_2104_00095_gb300.scenes` draws the seeded synthetic inputs.
"""
__all__ = ["rmt", "scenes"]
