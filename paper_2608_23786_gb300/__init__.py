"""GB300-native Monte Carlo KBC lattice Boltzmann ensembles (D3Q19, sm_103a).

The compute path is libmclbm (hand-written CUDA kernels behind the C ABI in
include/mclbm.h); ``mclbm`` is its ctypes binding and ``Ensemble`` a thin
PyTorch-memory wrapper.  Importing the package does not load the library;
the first call that needs it loads it and raises if it has not been built.
"""
from . import build, mclbm  # noqa: F401

__all__ = ["build", "mclbm", "Ensemble"]


def __getattr__(name):
    if name == "Ensemble":
        from .ensemble import Ensemble
        return Ensemble
    raise AttributeError(name)
