// Hot kernels instantiated for D=3, M=2, PDE=2 (0 Euler, 1 MHD-GLM, 2 linear advection).
#include "aw_inst.cuh"
AW_INSTANTIATE(3, 2, 2)
