"""GB300 (sm_103a) D3Q19 TRT lattice Boltzmann sweep behind a C ABI.

The compute path is the CUDA library ``liblbm_gb300.so`` built from ``csrc/``;
``lbm`` is its thin ctypes binding (argument marshalling only) and ``inputs``
holds the seeded synthetic workloads. Importing this package loads nothing:
``lbm`` loads the library on first use and raises if it is missing.
"""
