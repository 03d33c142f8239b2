"""rmgtd: GB300-native real-time TDDFT hot path (arXiv:2410.09189, Algorithm 1).

The compute lives in the CUDA library ``librmgtd.so`` behind the C ABI of
``include/rmgtd.h``; ``paper_2410_09189_gb300.rmgtd`` is its thin ctypes binding and
``paper_2410_09189_gb300.inputs`` the seeded input generators.  Importing the package
loads nothing; the library is loaded on first use of the binding.
"""
