"""GB300-native event-driven spiking-network hot path of BrainPy (ICLR 2024).

The compute lives in libbp (hand-written CUDA for sm_103a behind the C ABI in
include/bp.h).  ``binding`` marshals torch tensors into those calls;
``network`` wraps the E/I network object; ``workloads`` draws the seeded
synthetic inputs.  Importing the package does not load the library; the first
call into ``binding`` does, and fails loudly if it was not built.
"""
from . import workloads  # noqa: F401

__all__ = ["binding", "network", "workloads", "build"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name in ("binding", "network", "snn"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
