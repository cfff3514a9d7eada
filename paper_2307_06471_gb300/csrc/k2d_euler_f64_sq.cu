// The FP64 2D Euler step for square cells (kernels_2d_sq.inc)
#define CRK_T double
#define CRK_NAME euler_f64
#include "kernels_2d_sq.inc"
