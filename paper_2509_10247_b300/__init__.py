"""B300-native fused, batched, differentiable quadrotor environment step
(DiffAero, arXiv 2509.10247): sm_103a CUDA behind the C ABI of
include/diffsim.h, with a ctypes binding and torch.autograd wrappers.

Submodules load lazily: ``synth`` (seeded inputs, numpy only), ``binding``
(the C-ABI calls), ``autograd`` (DiffSimRollout, DiffSimStep), ``build``,
``autotune`` (launch-shape search with a bitwise parity gate and a JSON cache).
"""
import importlib

__all__ = ["synth", "binding", "autograd", "build", "autotune"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
