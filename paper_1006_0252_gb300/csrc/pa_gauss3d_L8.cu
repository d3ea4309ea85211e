// Instantiation of the Gaussian-coupling 3D sweep kernels for L = 8 (with
// the threshold-table kernel for blocks of 512 and 1024 threads).
#include "pa_gauss3d_tab.cuh"
PA_INSTANTIATE_GAUSS3D_TAB(8)
