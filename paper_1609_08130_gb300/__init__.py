"""GB300 (sm_103a) implementation of the strong recursive skeletonization
factorization (RS-S) of Minden, Ho, Damle & Ying (arXiv:1609.08130).

The compute path is the CUDA library ``librss.so`` (C ABI in
``include/rss.h``); :mod:`.rss` is its thin Python binding and
:mod:`.inputs` makes seeded synthetic workloads.
"""
from . import inputs  # noqa: F401
from .rss import (FP64, MIXED, LAPLACE2D_LOG, LAPLACE3D_INV, Factorization, Mlp, RSSError, Tree,  # noqa: F401
                  autotune_elim_table, autotune_table, build, kernel_launches, lib)
