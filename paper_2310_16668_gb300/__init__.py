"""GB300-native skeletonized fast multipole apply (strong recursive
skeletonization FMM, arXiv 2310.16668).

The compute lives in ``libskel.so`` (C-ABI in ``include/skel.h``): the tree
on the host, the interpolative decompositions on the host or the GPU (FP64),
sm_103a CUDA kernels for the apply. This package is the thin Python binding,
plus ``gmres`` (restarted GMRES with the apply as the product).
"""
from .api import SkelApply, SkelBatch, SkelFMM, skel_apply  # noqa: F401
from .solve import gmres  # noqa: F401
