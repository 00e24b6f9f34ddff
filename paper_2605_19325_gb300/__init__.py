"""GB300-native exterior NMF (eNMF): C-ABI CUDA library plus a thin binding.

The factorisation runs in libenmf.so (hand-written sm_103a kernels); this
package only loads it and marshals tensors.  Build it with
``paper_2605_19325_gb300.build.build()``.
"""
from . import binding  # noqa: F401  (raises if libenmf.so is missing)

__all__ = ["binding", "solver"]


def __getattr__(name):
    if name == "solver":
        from . import solver
        return solver
    if name in ("Solver", "solve"):
        from . import solver
        return getattr(solver, name)
    raise AttributeError(name)
