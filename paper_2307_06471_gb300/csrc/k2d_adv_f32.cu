// 2D kernels: PHYS_ADV in float
#define CRK_T float
#define CRK_PHYS crk::PHYS_ADV
#define CRK_NAME adv_f32
#include "kernels_2d.inc"
