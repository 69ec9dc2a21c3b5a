"""GB300 (sm_103a) solver for the vacuum quark gap equation with the Ball-Chiu vertex
(arXiv:2012.03667): batched successive approximation, mixed-precision refinement and an implicit
adjoint, behind the C interface include/qdse.h.

``qdse``      ctypes binding of libqdse.so (same entry-point names as the C interface)
``autograd``  torch.autograd.Function wrappers (solve -> A, B; condensate)
``inputs``    seeded synthetic workload generators (no solver arithmetic)
``build``     in-tree nvcc build of libqdse.so
"""
