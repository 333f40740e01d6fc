"""GB300-native sparse-grid Krylov IIF DG solver (Liu, Cheng, Chen, Zhang, arXiv:1810.11111).

The compute path lives in the CUDA library ``libsgkiif.so`` built from
``csrc/``; ``sgkiif`` is its thin ctypes binding and ``workloads`` holds the
seeded synthetic inputs.  Importing this package loads nothing; the binding
loads the library on first use and raises if it has not been built.
"""
