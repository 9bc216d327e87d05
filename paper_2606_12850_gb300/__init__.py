"""GB300-native spectral-element elastic wave solver (arXiv 2606.12850 hot path).

``paper_2606_12850_gb300.sem`` is the ctypes binding of the C-ABI library ``libsemgb.so``
(declared in ``include/sem.h``); ``paper_2606_12850_gb300.inputs`` builds seeded synthetic
meshes and workloads. The binding loads the CUDA library on first use and raises if it is
missing: there is no CPU fallback.
"""
