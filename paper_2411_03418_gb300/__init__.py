"""GB300-native line-by-line absorption (MARFA's eleven-grid path, arXiv 2411.03418).

The compute path is libmarfa (CUDA, sm_103a) behind the C-ABI of include/marfa.h;
``paper_2411_03418_gb300.marfa`` is its ctypes binding and
``paper_2411_03418_gb300.build`` compiles it in-tree.
"""
from . import build  # noqa: F401
