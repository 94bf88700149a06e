"""GB300 BERN-NN: sound polynomial bounds of ReLU networks over input boxes
(arxiv 2211.14438), computed by hand-written sm_103a CUDA kernels behind a
C ABI (include/bern.h).  ``bern`` is the Python binding; ``workloads`` holds
the seeded synthetic inputs."""
from . import workloads  # noqa: F401

__all__ = ["bern", "workloads", "build"]
