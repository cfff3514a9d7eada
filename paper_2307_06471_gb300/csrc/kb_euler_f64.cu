// batched 2D Euler step in double
#define CRK_T double
#define CRK_NAME euler_f64
#include "batch_kernels.inc"
