"""GB300-native QED Monte Carlo event generator (arXiv:2008.10468).

The compute path lives in the CUDA library ``csrc/libqed.so`` behind a C ABI
(``include/qed.h``); ``paper_2008_10468_gb300.qed`` is its thin ctypes binding.
``paper_2008_10468_gb300.inputs`` generates the seeded synthetic workloads.
Importing the package itself loads nothing; import the submodule you need.
"""
