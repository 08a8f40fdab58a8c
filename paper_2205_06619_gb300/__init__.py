"""FastSTMF hot path on GB300 (sm_103a): masked max-plus product with top-2
tracking and the ByRow/TD_A factor-update sweep, as CUDA kernels behind a
C ABI (``include/stmf.h``).  The native library is loaded lazily on first
use by :mod:`paper_2205_06619_gb300.api`; importing this package never
touches the GPU."""
