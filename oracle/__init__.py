"""Plain CPU oracle for the PT-QMC hot path (test infrastructure only)."""
from .oracle import Oracle, build, det_exp, load, philox  # noqa: F401
