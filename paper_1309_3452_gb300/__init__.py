"""GB300-native staggered space-time leap-frog Dirac stepper (arXiv:1309.3452).

`paper_1309_3452_gb300.dirac` is the binding of the C-ABI CUDA library
(`libdirac.so`); `paper_1309_3452_gb300.workloads` builds seeded synthetic
inputs.  Importing this package loads nothing; importing `dirac` loads the
CUDA library and fails loudly when it has not been built.
"""
