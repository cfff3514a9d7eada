// 2D kernels: PHYS_ADV in double
#define CRK_T double
#define CRK_PHYS crk::PHYS_ADV
#define CRK_NAME adv_f64
#include "kernels_2d.inc"
