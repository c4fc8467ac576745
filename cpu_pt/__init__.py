"""The paper's multi-threaded CPU Parallel Tempering (Sec. 4) as a CPU comparison baseline."""
from .cpu_pt import CpuPT, build, load  # noqa: F401
