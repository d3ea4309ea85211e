// Instantiation of the 3D sweep and init kernels for L = 14.
#include "pa_sweep3d.cuh"
PA_INSTANTIATE_SWEEP3D(14)
