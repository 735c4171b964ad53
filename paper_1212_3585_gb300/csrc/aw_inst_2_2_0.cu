// Hot kernels instantiated for D=2, M=2, PDE=0 (0 Euler, 1 MHD-GLM, 2 linear advection).
#include "aw_inst.cuh"
AW_INSTANTIATE(2, 2, 0)
