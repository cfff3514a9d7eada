// 2D kernels: PHYS_EULER in double
#define CRK_T double
#define CRK_PHYS crk::PHYS_EULER
#define CRK_NAME euler_f64
// square cells take the square-cell form of the step (k2d_euler_f64_sq.cu);
// CRK_SQ_STEP_OFF keeps them on the general form (tuning knob)
#ifndef CRK_SQ_STEP_OFF
#define CRK_SQ_STEP 1
#endif
#include "kernels_2d.inc"
