"""GB300-native (sm_103a) auxiliary-grid AMG: quadtree aggregation, Galerkin coarse operators
and the nonlinear AMLI-cycle solve, as CUDA kernels behind a C ABI (include/amg.h).

The binding (``paper_1209_5421_gb300.amg``) is imported lazily so that the synthetic
workload generator (``paper_1209_5421_gb300.meshes``) can be used without the CUDA library.
"""
