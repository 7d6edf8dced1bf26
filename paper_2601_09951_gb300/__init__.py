"""GB300-native state-vector VQE hot path (energy, adjoint gradient, batched and served).

The compute path is the CUDA library ``libsvqe.so`` behind the C ABI in ``include/svqe.h``;
``paper_2601_09951_gb300.svqe`` is its ctypes binding.  Importing the package loads nothing;
the library is opened on first use and a missing library is an error, never a fallback.
"""
__all__ = ["svqe", "workloads"]
