"""GB300-native (sm_103a) lattice Boltzmann inkjet model of He et al.
(arXiv:1702.04487): the fused per-step lattice update behind a C ABI.

Importing the package does not load the CUDA library; ``inkjet`` (the
binding) does, and fails loudly when it is missing.
"""
