"""Tucker-compressed FMM far-fields on one GB300 (arXiv 2103.05822).

``tfmm``    - Python binding of the C ABI in ``include/tfmm.h`` (libtfmm.so).
``inputs``  - seeded synthetic meshes and vectors shared by tests and benchmark.
``build``   - in-tree nvcc build of libtfmm.so for sm_103a.
"""
