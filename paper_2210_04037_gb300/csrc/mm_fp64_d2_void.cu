// FP64 (compiled with --fmad=false, as the other FP64 units) instantiation of the step kernels for 2D grids holding a void
// material (the void volume fraction of Sec. 2.1, opened at critically
// damaged faces in tension, Sec. 3.1): two or three materials, one plastic.
#include "mm_launch.cuh"

cudaError_t mm_p64_d2_void(int what, int axis, int flag, const KArgs& a, double* out,
                           int nblocks, cudaStream_t s) {
  return mm::Launch<mm::P64V>::by_mat_void<2>(what, axis, flag, a, out, nblocks, s);
}
