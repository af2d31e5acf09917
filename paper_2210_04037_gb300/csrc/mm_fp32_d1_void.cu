// FP32-split instantiation of the step kernels for 1D grids holding a void
// material (the void volume fraction of Sec. 2.1, opened at critically
// damaged faces in tension, Sec. 3.1): two or three materials, one plastic.
#include "mm_launch.cuh"

cudaError_t mm_p32_d1_void(int what, int axis, int flag, const KArgs& a, double* out,
                           int nblocks, cudaStream_t s) {
  return mm::Launch<mm::P32V>::by_mat_void<1>(what, axis, flag, a, out, nblocks, s);
}
