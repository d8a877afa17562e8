"""GB300 (sm_103a) two-grid MLQMC level evaluation for random elliptic eigenvalue problems.

The compute path is the CUDA library ``lib/libmlqmc_evp.so`` (sources in ``csrc/``, C ABI in
``include/mlqmc_evp.h``); ``binding`` marshals arguments to it with ctypes.  Import
``paper_2103_03407_gb300.binding`` explicitly: importing the package itself loads nothing.
"""
