"""GB300-native field + tracking-step engine for the OuroborosBEM method
(arXiv 2110.09214): BEM panel field + all-pairs space charge at every charge,
fused with the null-collision Monte Carlo step, behind the C ABI of
``include/obem.h``.

Importing the package is cheap; the CUDA library is loaded on first use by
``paper_2110_09214_gb300.obem``.
"""
__all__ = ["inputs", "obem", "swarm"]
