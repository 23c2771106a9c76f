"""GB300-native hybrid compressor hot path (arXiv:2212.10733).

The CUDA library and its binding live in :mod:`paper_2212_10733_gb300.aeqc`;
importing this package alone loads nothing native.
"""
