"""GB300-native data-parallel hot path of the enhanced DPSO inspection planner
(Phung et al., arXiv:1706.04399).

The compute lives in the CUDA library ``libdpso_gb300.so`` (built from
``csrc/``) behind the C ABI declared in ``include/dpso.h``; ``dpso`` is its
thin ctypes binding.  ``inputs`` holds the seeded synthetic workloads.
Importing the package does not load the library; the first call into
``dpso`` does, and raises if it has not been built.
"""
