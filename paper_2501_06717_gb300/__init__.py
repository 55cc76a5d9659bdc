"""GB300-native hot path of a block-adaptive ideal-MHD solver (arXiv 2501.06717).

The compute path lives in the CUDA library ``libbats`` (C-ABI, ``include/bats.h``);
``paper_2501_06717_gb300.bats`` is its thin ctypes binding.  Import it
explicitly: importing this package loads nothing compiled.
"""
