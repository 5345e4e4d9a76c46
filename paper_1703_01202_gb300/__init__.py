"""GB300-native Newton-Krylov-Schwarz time stepper for the phase field crystal
equation (Wei, Yang & Huang, arXiv:1703.01202).  The compute path is the C-ABI
library ``libpfc.so`` (hand-written CUDA for sm_103a); this package holds its
Python binding (``pfc``), its build step and the seeded input generators."""
