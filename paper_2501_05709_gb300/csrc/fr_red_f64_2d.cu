// Reduced-degree element kernels instantiated for double in 2D.
#define FR_REAL double
#define FR_DIM 2
#include "fr_reduced_launch.cuh"
