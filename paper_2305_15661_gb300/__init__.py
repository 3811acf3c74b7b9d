"""GB300-native EQP-IFT hot path (arXiv 2305.15661): element residual/Jacobian
kernels, weighted reduced contraction, hyperreduced gather and LM solve, behind
the C ABI in include/ift.h. ``ift`` is the Python binding, ``workloads`` the
seeded synthetic inputs, ``build`` the in-tree compiler driver."""
