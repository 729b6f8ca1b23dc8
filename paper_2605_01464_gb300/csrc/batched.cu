// batched.cu -- host side of qpinv_solve_batched (descriptors, ordering,
// CUDA graph capture and replay); the kernel is instantiated per tile shape
// in batched_tile<t>.cu.  The code lives in batched_impl.cuh.
#include "batched_impl.cuh"
