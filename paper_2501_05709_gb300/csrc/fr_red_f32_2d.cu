// Reduced-degree element kernels instantiated for float in 2D.
#define FR_REAL float
#define FR_DIM 2
#include "fr_reduced_launch.cuh"
