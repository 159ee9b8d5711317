"""GB300 (sm_103a) multi-level tunnelling ionization: ADK rates and the
analytic, locally reduced charge-state update of Cheng & Samulyak
(arXiv 2202.10647), as a CUDA library with a C ABI (include/ionize.h) and a
thin Python binding (``ionize``)."""
from . import build  # noqa: F401

__all__ = ["build", "ionize", "workloads"]


def __getattr__(name):
    if name in ("ionize", "workloads"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
