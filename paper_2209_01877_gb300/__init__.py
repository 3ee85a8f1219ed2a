"""GB300 (sm_103a) modal DG residual and SSP-RK3 for the 3D Euler equations on
tetrahedra, behind the C ABI of include/dg.h.

Modules: ``dg`` (ctypes binding of libdg.so), ``inputs`` (seeded synthetic
meshes and fields), ``build`` (nvcc build of libdg.so).
"""
