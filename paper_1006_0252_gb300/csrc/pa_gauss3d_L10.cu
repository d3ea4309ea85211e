// Instantiation of the Gaussian-coupling 3D sweep kernel for L = 10.
#include "pa_gauss3d.cuh"
PA_INSTANTIATE_GAUSS3D(10)
