"""Lazy qubit reordering (arXiv 2410.04252) on one GB300: QSU, EVC and the
adjoint VQE gradient on a 2^n state vector split into 2^g virtual chunks.

Submodules:
  workloads  seeded synthetic circuits, parameters and Hamiltonians
  sv         ctypes binding of the C-ABI library libsv.so (CUDA, sm_103a)
  autograd   torch.autograd.Function over sv_grad
  dist       the state sharded over ranks: QRs as pairwise exchanges

The binding is imported on first use of a name it defines, so that the
input generators can be used without loading CUDA.
"""
__all__ = ["workloads", "sv", "autograd", "dist"]


def __getattr__(name):
    if name in ("sv", "autograd"):
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
