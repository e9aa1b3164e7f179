"""B300-native H-M-H Strang step for 2.5D ideal MHD (FP64 CUDA kernels behind a C ABI).

``paper_2609_10849_b300.mhd`` is the ctypes binding of ``libmhd.so``;
``paper_2609_10849_b300.workloads`` generates the seeded synthetic initial
states.  Importing the package does not load the CUDA library.
"""
