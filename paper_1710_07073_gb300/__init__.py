"""GB300-native LBGK-LPT bubble-column hot path (arXiv:1710.07073).

The coupled step runs in the CUDA library liblbm.so (C ABI in include/lbm.h);
``paper_1710_07073_gb300.lbm`` is its Python binding and
``paper_1710_07073_gb300.build`` compiles it for sm_103a.
"""
