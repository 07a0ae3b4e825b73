"""GB300-native multidimensional range query (MDRQ) scan.

The query path is the C-ABI library ``libmdrq.so`` (CUDA kernels for sm_103a, built
from ``csrc/``) reached through the ctypes binding in ``mdrq.py``. Importing this
package does not load the library; the first call into ``mdrq`` does, and raises if it
is missing. ``workloads`` makes seeded synthetic inputs and needs no GPU.
"""
__all__ = ["mdrq", "workloads"]
