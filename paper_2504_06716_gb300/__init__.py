"""GSta training hot path for GB300 (sm_103a): 3-D Gaussian splatting with
gradient-norm freezing, as hand-written CUDA behind a C ABI.

Importing the package loads nothing; the CUDA library is loaded by
``paper_2504_06716_gb300.lib`` on first use and fails loudly if absent.
"""
