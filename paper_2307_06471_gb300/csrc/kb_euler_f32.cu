// batched 2D Euler step in float
#define CRK_T float
#define CRK_NAME euler_f32
#include "batch_kernels.inc"
