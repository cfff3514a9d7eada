// 2D kernels: PHYS_EULER in double
#define CRK_T double
#define CRK_PHYS crk::PHYS_EULER
#define CRK_NAME euler_f64
#include "kernels_2d.inc"
