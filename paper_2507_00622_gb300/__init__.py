"""GB300 (sm_103a) library for ensembles of Hamiltonian orbits with their
variational equations and the chaos indicators of arXiv 2507.00622
(SALI, GALI_k, Lagrangian-descriptor indicators, Lyapunov spectrum by QR).

The compute path is ``libchs.so`` (CUDA, C ABI in ``include/chs.h``); the
``chs`` module is its ctypes binding.  Importing this package loads nothing;
``paper_2507_00622_gb300.chs.load()`` loads the library and fails loudly when
it has not been built.
"""
__version__ = "0.1.0"
