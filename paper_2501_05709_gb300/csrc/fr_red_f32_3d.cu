// Reduced-degree element kernels instantiated for float in 3D.
#define FR_REAL float
#define FR_DIM 3
#include "fr_reduced_launch.cuh"
