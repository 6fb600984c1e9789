"""GB300-native Mosaic Flow sweep engine (Feeney et al., SC '23, arXiv 2308.14258).

The compute path lives in the sm_103a shared library built from ``csrc/`` and is
reached through the ctypes binding in :mod:`paper_2308_14258_gb300.mosaicflow`.
Importing this package does not load the library; :mod:`.inputs` holds the seeded
synthetic workload generators.
"""
