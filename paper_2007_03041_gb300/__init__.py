"""GB300 (sm_103a) fast summation of the method-of-lines-transpose operator
L^{-1} and the successive-convolution partial sums of D = I - L^{-1}
(arXiv 2007.03041), behind the C ABI of include/molt.h.

``molt``      -- ctypes binding with the C names (molt_create, molt_apply_D,
                 molt_step, molt_destroy).
``workloads`` -- seeded synthetic inputs.
``build``     -- compiles libmolt.so in-tree with nvcc for sm_103a.
"""
