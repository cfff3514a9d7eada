// 2D kernels: PHYS_EULER in float
#define CRK_T float
#define CRK_PHYS crk::PHYS_EULER
#define CRK_NAME euler_f32
#include "kernels_2d.inc"
