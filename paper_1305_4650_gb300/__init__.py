"""GB300-native Chebyshev-interpolation butterfly (sm_103a CUDA behind a C ABI).

Importing the package is cheap: the CUDA library is loaded on first use of
``paper_1305_4650_gb300.bf`` (see ``bf.py``).
"""
__all__ = ["workloads"]
