"""B300-native sparse truncated state-vector simulator for peaked circuits.

The compute path is the CUDA library ``libsv.so`` (built from ``csrc/``)
behind the C ABI declared in ``include/sv.h``; ``paper_2607_07816_b300.sv``
is its thin Python binding.  ``paper_2607_07816_b300.circuits`` holds the
seeded synthetic workload generators.  Submodules are imported on demand so
that the input generators can be used without the CUDA library.
"""
