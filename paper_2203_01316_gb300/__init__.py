"""GB300 (sm_103a) thermal lattice Boltzmann library: the coupled f+h
stream+collide step of arXiv 2203.01316 behind a C ABI (include/lbm.h).

`Solver` (paper_2203_01316_gb300.lbm) is the Python binding; `inputs` builds
seeded synthetic geometries and fields; `build` compiles the CUDA library.
"""
from .lbm import LBMError, Solver, lib  # noqa: F401
