"""perc5d: exact batched first-spanning search and largest-cluster mass for random site
percolation on the 5D simple cubic lattice with complex neighborhoods, on B300 (sm_103a).

Layers: ``include/perc.h`` (C ABI of ``libperc.so``, CUDA kernels in ``csrc/``), ``perc`` (the
ctypes binding), ``driver`` (batched workloads: ranking, sample tables, plain or learned bracket),
``bracket`` (training of the bracket network on the GPU), ``workloads`` (seeded inputs).
"""
from . import workloads  # noqa: F401

__all__ = ["perc", "driver", "bracket", "workloads", "build"]
