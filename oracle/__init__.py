"""FP64 CPU oracle for the gather-and-refine scoring path and for Token-Aware Clustering's
centroid allotment (`oracle.tac`) (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg may
import this package. The CUDA library never calls it, and it shares no code
with the CUDA path.
"""
from .oracle import Oracle, build, lib_path  # noqa: F401
