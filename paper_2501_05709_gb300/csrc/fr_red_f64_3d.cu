// Reduced-degree element kernels instantiated for double in 3D.
#define FR_REAL double
#define FR_DIM 3
#include "fr_reduced_launch.cuh"
