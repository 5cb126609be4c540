"""GB300-native (sm_103a) Monte Carlo engine for 1+1-d KPZ growth mapped onto
a bit-packed ASEP lattice gas (arXiv:1012.0385, Schulz, Odor, Odor, Nagy).

The compute path is ``libasep.so`` (hand-written CUDA, C ABI in
``include/asep.h``); :mod:`paper_1012_0385_gb300.asep` is its Python binding.
"""
from . import asep  # noqa: F401
from .asep import *  # noqa: F401,F403

__all__ = ["asep"]
