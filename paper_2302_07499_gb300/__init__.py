"""GB300-native nonlocal P1 tetrahedral assembly and solve (nlfem).

Chen, Ma & Zhang, "High performance implementation of 3D FEM for nonlocal
Poisson problem with different ball approximation strategies": assembly of
the nonlocal stiffness matrix and right-hand side with the nocaps,
approxcaps and fullcaps ball approximations (Sec. 3.3, 4.3), and the CG
solve of the volume-constrained system (Alg. 5).  All compute runs in the
CUDA kernels of libnlfem.so (C-ABI declared in include/nlfem.h); this
package is the Python binding.
"""
from ._binding import (APPROXCAPS, BARYCENTER, INSIDE, OVERLAP, DEVICE, FP32_COMP, FP64, FULLCAPS, FULLCAPS_QMC, HOST, MAT_A, MAT_K, MAT_LIFT, NOCAPS, Device,  # noqa
                       Mesh, NlError, Pairs, System, lib, probe_moments, probe_philox, EXPORTED, LIB_PATH,
                       kernel_launches, Batch, Server, mesh_box, probe_mc_samples,
                       probe_alu_rates)
