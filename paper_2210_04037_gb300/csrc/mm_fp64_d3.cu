// FP64 instantiation of the step kernels for 3D grids.  Compiled with
// --fmad=false so every product and sum is rounded separately, as in the
// CPU reference arithmetic.
#include "mm_launch.cuh"

cudaError_t mm_p64_d3(int what, int axis, int flag, const KArgs& a, double* out, int nblocks,
                      cudaStream_t s) {
  return mm::Launch<mm::P64>::by_mat<3>(what, axis, flag, a, out, nblocks, s);
}
