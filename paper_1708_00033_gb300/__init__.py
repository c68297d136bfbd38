"""GB300-native (sm_103a) direct-SCF Fock build.

The hot path of Mironov et al. (SC17) Hartree-Fock: Schwarz-screened unique
shell quartets (Algorithm 1), electron-repulsion integrals, and their
digestion into J and K (Eq. 1a-1f), as hand-written CUDA behind the C-ABI of
include/hf.h.  ``inputs`` draws the seeded synthetic workloads; ``hf`` is the
ctypes binding of the library.
"""
from . import inputs  # noqa: F401


def build(verbose: bool = False) -> str:
    """Compile libhf.so for sm_103a (needs nvcc) and return its path."""
    from ._build import build as _build
    return _build(verbose=verbose)


def __getattr__(name):
    if name in ("hf",):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
