"""GB300-native short-range particle-particle solver of CRK-HACC
(arXiv 2510.03557): Morton-sorted leaves, leaf-pair lists, the CRKSPH passes
and short-range gravity, in hand-written sm_103a CUDA behind a C ABI.

The native library is loaded lazily by ``paper_2510_03557_gb300.crk``; the
input generators in ``workloads`` need no GPU.
"""
