"""GB300-native skeletonized fast multipole apply (strong recursive
skeletonization FMM, arXiv 2310.16668).

The compute lives in ``libskel.so`` (C-ABI in ``include/skel.h``): host FP64
tree + interpolative decompositions, sm_103a CUDA kernels for the apply.
This package is the thin Python binding.
"""
from .api import SkelApply, SkelBatch, SkelFMM, skel_apply  # noqa: F401
