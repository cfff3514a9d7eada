// 2D kernels: PHYS_EULER in float
#define CRK_T float
#define CRK_PHYS crk::PHYS_EULER
#define CRK_NAME euler_f32
// square cells take the square-cell form of the step (k2d_euler_f32_sq.cu);
// CRK_SQ_STEP_OFF keeps them on the general form (tuning knob)
#ifndef CRK_SQ_STEP_OFF
#define CRK_SQ_STEP 1
#endif
#include "kernels_2d.inc"
