"""Single-GPU (B300, sm_103a) MPdist-profile engine for PaSTiLa (arXiv 2401.13680).

The compute lives in ``libpastila.so`` (hand-written CUDA, C ABI declared in
``include/pastila.h``); ``pastila`` is its thin ctypes binding.
"""
