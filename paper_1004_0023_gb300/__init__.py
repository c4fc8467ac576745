"""GB300-native parallel-tempering quantum Monte Carlo (PT-QMC) hot path.

The compute path lives in a C-ABI shared library built from ``csrc/`` (hand-written
sm_103a CUDA). ``pt`` is a thin ctypes binding with the same names as the C entry
points; ``instances`` holds the seeded synthetic problem generators.
"""
__all__ = ["instances", "pt"]
