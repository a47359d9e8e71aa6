"""GB300-native POD-augmented conjugate gradient for sequences of sparse SPD systems.

The compute path is the CUDA library ``lib/libpodcg.so`` (C ABI in ``include/pod_cg.h``);
this package holds its thin Python binding (:mod:`.solver`), the in-tree build
(:mod:`._build`), the sequence driver (:mod:`.sequence`) and the seeded synthetic workloads
(:mod:`.workloads`). Importing the package does not load the library; the first solver
call does, and fails loudly if it has not been built.
"""

__all__ = ["build", "solver", "workloads"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)
