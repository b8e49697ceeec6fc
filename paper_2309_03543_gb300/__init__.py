"""GB300-native corrector-step solver (arXiv 2309.03543, Sec. 3.2.2-3.2.3).

Assembly of the CP1/CP2 matrices on Delaunay triangle meshes and their
preconditioned conjugate-gradient solves, as hand-written sm_103a CUDA kernels
behind the C ABI of include/cps.h.  This package is the Python binding:
``Context.assemble`` -> ``System.solve`` / ``System.adjoint`` /
``solve_batch``, and the autograd wrapper ``CorrectorSolve``.
"""
from ._cps import (BATCH_GRAPH, BATCH_ONE_LAUNCH, CP1_HOST, CP1_ONE_LAUNCH, FP64, KIND_CP1_X, KIND_CP1_Y, KIND_CP2, MIXED, PATH_AUTO, PATH_CLUSTER,  # noqa: F401
                   PATH_CLUSTER_1RED, PATH_CLUSTER_PIPE, PATH_CLUSTER_SSTEP2, PATH_CLUSTER_SSTEP3, PATH_PERSISTENT, PATH_PERSISTENT_1RED, PATH_PERSISTENT_1RED_L2, PATH_PERSISTENT_L2, PATH_STREAM, PATH_STREAM_1RED, PATH_STREAM_1RED_L2, PATH_STREAM_L2, PC_IC0, PC_JACOBI, PC_REDUCED, PER_CELL, PER_CELL_LOGK, PER_VERTEX, LIB_PATH)
from .api import Context, CpsError, SolveStats, System, cp1_setup, cp1_step, set_cp1_path, solve_batch  # noqa: F401
from .autograd import CorrectorSolve, LogPermeabilityCorrector, chained_solve  # noqa: F401


def build(force: bool = False) -> str:
    from .build import build as _b
    return _b(force=force)
