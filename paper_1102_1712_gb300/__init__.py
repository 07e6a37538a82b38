"""GB300-native single-projection PCA lung-motion solver (Li et al., arXiv:1102.1712).

The compute path is the C-ABI library ``libpcasolve.so`` built from ``csrc/``
(hand-written CUDA for sm_103a); ``pcasolve`` is its thin ctypes binding.
``synth`` generates seeded synthetic inputs.  Nothing here imports the oracle.
"""
