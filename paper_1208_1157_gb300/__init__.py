"""GB300-native (sm_103a) FP64 integrator for large ensembles of few-body systems:
the Hermite-4 and mixed-variable symplectic methods of Swarm-NG (arXiv:1208.1157)
behind a C ABI (include/swarm.h), with this package as its thin Python binding.

  ics    seeded synthetic planetary ensembles (inputs only)
  swarm  ctypes binding of libswarm_gb300.so (Ensemble, fp64_peak, tuner)
  build  nvcc build of the library
"""
from . import ics  # noqa: F401

__all__ = ["ics", "swarm", "build"]


def __getattr__(name):
    if name in ("swarm", "build", "server"):
        import importlib

        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
