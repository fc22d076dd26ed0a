"""GB300-native Memetic Phase Retrieval (MPR) hot path.

The compute runs in hand-written CUDA kernels for sm_103a inside ``libspring.so``;
:mod:`paper_2409_07413_gb300.spring` is the thin ctypes binding over its C ABI
(``include/spring.h``).  :mod:`paper_2409_07413_gb300.synthetic` draws seeded inputs.
"""
