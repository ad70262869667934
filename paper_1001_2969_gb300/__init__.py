"""GB300-native implicit electrostatic PIC/MC timestep in axisymmetric r-z
geometry (Wang, Jiang & Wang, arXiv:1001.2969).

The compute lives in ``libpic.so`` (CUDA for sm_103a, C ABI in
``include/pic.h``); ``paper_1001_2969_gb300.pic`` is its thin binding.
"""
from .build import build  # noqa: F401
