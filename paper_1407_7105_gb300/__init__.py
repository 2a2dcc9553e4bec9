"""GB300-native connected-component (CC) Hamiltonian-splitting N-body
integrator hot path (Jaenes, Pelupessy & Portegies Zwart, arXiv:1407.7105).

The compute path is the CUDA library ``libcc.so`` built from ``csrc/``;
``cc`` is its thin ctypes binding and ``ics`` the seeded initial-condition
generators.
"""
