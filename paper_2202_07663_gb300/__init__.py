"""GB300-native batched lens-model log-likelihood and gradient (GIGA-Lens,
arXiv:2202.07663).

Importing the package loads nothing heavy. The CUDA library is loaded on
first use by :mod:`paper_2202_07663_gb300.abi`; if it is missing the call
fails loudly (there is no CPU fallback).
"""

__all__ = ["abi", "inputs"]
