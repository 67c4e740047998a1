"""GB300-native differentiable magneto-elastic MLS-MPM (arxiv 2503.22767).

The substep (sort, P2G with neo-Hookean + hard-magnetic stress, grid
operation, G2P) and its reverse-mode adjoint run as hand-written CUDA kernels
for sm_103a behind the C ABI declared in ``include/mpm.h``.  This package is
the thin Python side: ``binding`` loads the library and marshals arguments,
``sim`` wraps it in a ``torch.autograd.Function``, ``design`` maps design
parameters (angles, Fourier coefficients) onto the ABI's inputs, and
``workloads`` draws seeded synthetic problems.

Submodules are imported lazily so that ``workloads`` works without a GPU.
"""
import importlib

__all__ = ["binding", "sim", "design", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
