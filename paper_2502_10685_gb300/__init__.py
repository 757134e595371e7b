"""GB300 Pauli-coefficient propagation (arXiv 2502.10685, extended stabilizer formalism).

Submodules:
  workloads  seeded synthetic circuits, observables, batches and traces (numpy only)
  stab       Python binding of the C interface in include/stab.h (loads libstab.so)
  autograd   torch.autograd.Function over stab_expect / stab_grad
  build      nvcc build of libstab.so for sm_103a

Importing the package does not load the CUDA library; the binding loads it on
first use and raises if it is missing (there is no CPU fallback).
"""
import importlib

__all__ = ["workloads", "stab", "autograd", "build", "Stab"]


def __getattr__(name):
    if name in ("stab", "autograd", "build", "workloads", "serve", "batch"):
        return importlib.import_module("." + name, __name__)
    if name == "Stab":
        return importlib.import_module(".stab", __name__).Stab
    raise AttributeError(name)
