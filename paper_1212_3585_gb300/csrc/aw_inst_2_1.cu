// Hot kernels instantiated for D=2, M=1 (the second-order scheme): PDE=0 Euler and PDE=2 linear
// advection.
#include "aw_inst.cuh"
AW_INSTANTIATE(2, 1, 0)
AW_INSTANTIATE(2, 1, 2)
