"""GB300 (sm_103a) implementation of the compact RKDG time step
(Chen, Sun, Xing, arXiv 2307.06471).

  binding   ctypes binding of the C ABI in include/crkdg.h (libcrkdg.so)
  build     in-tree nvcc build of libcrkdg.so
  tableaux  named Butcher tableaux
"""
