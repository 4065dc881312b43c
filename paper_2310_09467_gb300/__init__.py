"""GB300 (sm_103a) implementation of the PC-bzip2 compression path for raw
light-field microscopy frames.

- ``lfc``   : Python binding of the C ABI in ``include/lfc.h`` (liblfc.so).
- ``build`` : compiles liblfc.so in-tree with nvcc for sm_103a.
- ``synth`` : seeded synthetic LFM frames (inputs only).
"""
