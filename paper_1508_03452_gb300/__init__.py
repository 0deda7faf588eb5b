"""GB300-native lattice Boltzmann solver for resistive relativistic MHD
(Mohseni, Mendoza, Succi, Herrmann; arXiv:1508.03452).

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lbrmhd.h``); ``lbrmhd`` is its Python binding and ``workloads`` holds
the seeded synthetic initial fields of the paper's test problems. Importing the
package does not load the CUDA library; ``lbrmhd.load()`` or the first
``lbrmhd.Solver`` does.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "lbrmhd", "build"]


def __getattr__(name):
    if name in ("lbrmhd", "build"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
