"""GB300-native ReaxFF timestep: CUDA kernels behind the C ABI in include/reaxff.h.

`paper_1706_07772_gb300.reaxff` is the Python binding of libreaxff.so; the library is
built in-tree by `python -m paper_1706_07772_gb300.build`.
"""
