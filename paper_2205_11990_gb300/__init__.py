"""GB300-native matrix-product-state Vlasov-Poisson solver (Ye & Loureiro, arXiv:2205.11990).

Importing the package is cheap; the CUDA library is loaded on first use by
:mod:`paper_2205_11990_gb300.vpmps`.
"""
__all__ = ["inputs", "vpmps"]
