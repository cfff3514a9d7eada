"""Butcher tableaux (eq. (2.5)): c | A over b, A strictly lower triangular.

Test infrastructure only: the CUDA library receives tableaux as input arrays
and defines none of its own.
"""
import numpy as np


def tableau(A, b):
    A = np.array(A, dtype=np.float64)
    b = np.array(b, dtype=np.float64)
    c = A.sum(axis=1)
    return {"A": A, "b": b, "c": c, "s": len(b)}


# forward Euler (one stage)
EULER = tableau([[0.0]], [1.0])
# Eq. (2.9): second-order cRKDG, explicit midpoint (a21 = 1/2, b = (0, 1))
MIDPOINT = tableau([[0, 0], [0.5, 0]], [0.0, 1.0])
# Eq. (3.3): Butcher form of SSP-RK2 (Heun): a21 = 1, b = (1/2, 1/2)
HEUN = tableau([[0, 0], [1.0, 0]], [0.5, 0.5])
# Eq. (2.10): third-order cRKDG (Heun's third-order method)
HEUN3 = tableau([[0, 0, 0], [1 / 3, 0, 0], [0, 2 / 3, 0]], [0.25, 0.0, 0.75])
# SSP-RK3 of Shu and Osher written in Butcher form (Sec. 3.2.1 / Table 4.3)
SSPRK3 = tableau([[0, 0, 0], [1.0, 0, 0], [0.25, 0.25, 0]], [1 / 6, 1 / 6, 2 / 3])
# classical four-stage fourth-order RK (Remark 2.1, Sec. 4)
RK4 = tableau([[0, 0, 0, 0], [0.5, 0, 0, 0], [0, 0.5, 0, 0], [0, 0, 1.0, 0]],
              [1 / 6, 1 / 3, 1 / 3, 1 / 6])
# a second four-stage fourth-order method (Kutta's 3/8 rule), used only to
# show that the linear update does not depend on the tableau (Sec. 3.5.1)
RK38 = tableau([[0, 0, 0, 0], [1 / 3, 0, 0, 0], [-1 / 3, 1.0, 0, 0], [1.0, -1.0, 1.0, 0]],
               [1 / 8, 3 / 8, 3 / 8, 1 / 8])
