"""Named explicit Butcher tableaux (eq. (2.5)) for crkdg_create.

  MIDPOINT  eq. (2.9)   second-order cRKDG (a21 = 1/2, b = (0, 1))
  HEUN2     eq. (3.3)   Butcher form of SSP-RK2 (a21 = 1, b = (1/2, 1/2))
  HEUN3     eq. (2.10)  third-order cRKDG (a21 = 1/3, a32 = 2/3, b = (1/4, 0, 3/4))
  SSPRK3                SSP-RK3 in Butcher form (a21 = 1, a31 = a32 = 1/4, b = (1/6, 1/6, 2/3))
  RK4                   classical four-stage fourth-order method (Remark 2.1)
  EULER                 forward Euler (one stage)
"""

MIDPOINT = ([[0.0, 0.0], [0.5, 0.0]], [0.0, 1.0])
HEUN2 = ([[0.0, 0.0], [1.0, 0.0]], [0.5, 0.5])
HEUN3 = ([[0.0, 0.0, 0.0], [1.0 / 3.0, 0.0, 0.0], [0.0, 2.0 / 3.0, 0.0]], [0.25, 0.0, 0.75])
SSPRK3 = ([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.25, 0.25, 0.0]], [1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0])
RK4 = ([[0.0, 0.0, 0.0, 0.0], [0.5, 0.0, 0.0, 0.0], [0.0, 0.5, 0.0, 0.0], [0.0, 0.0, 1.0, 0.0]],
       [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0])
EULER = ([[0.0]], [1.0])

BY_NAME = {"midpoint": MIDPOINT, "heun2": HEUN2, "heun3": HEUN3, "ssprk3": SSPRK3, "rk4": RK4,
           "euler": EULER}
