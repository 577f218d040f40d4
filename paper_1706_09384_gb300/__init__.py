"""GB300-native H-matrix hot path for 3D elastodynamic Green's tensors
(arXiv:1706.09384): cluster tree, block partition, Green's-tensor near field,
vector ACA + QR/SVD recompression, H-matvec and GMRES, all as sm_103a CUDA
kernels behind the C ABI declared in ``include/hm.h``.

``inputs`` (seeded synthetic clouds) is importable without a GPU; the CUDA
binding lives in ``paper_1706_09384_gb300.hm`` and loads ``libhm.so`` lazily.
"""
