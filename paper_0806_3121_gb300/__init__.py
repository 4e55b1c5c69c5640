"""GB300-native Huang-Abraham ABFT matrix multiplication (Bosilca, Delmas, Dongarra,
Langou 2008): C-ABI library libabft (include/abft.h) with hand-written sm_103a kernels,
a thin ctypes binding (``abft``), its nvcc build (``build``) and seeded synthetic
workloads (``workloads``)."""
__all__ = ["abft", "build", "workloads"]
