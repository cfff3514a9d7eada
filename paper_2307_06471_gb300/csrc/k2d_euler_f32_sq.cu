// The FP32 2D Euler step for square cells (kernels_2d_sq.inc)
#define CRK_T float
#define CRK_NAME euler_f32
#include "kernels_2d_sq.inc"
