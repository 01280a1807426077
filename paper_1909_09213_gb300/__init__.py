"""GB300-native CUBICS hot path: bitset constraint propagation with on-device search.

Importing the package is cheap: the CUDA library is loaded on first use by
``paper_1909_09213_gb300.cubics`` and the import fails loudly if it is missing.
"""
