// FP32-split instantiation of the step kernels for 2D grids:
// reconstruction, fluxes and closures in FP32; total energy, its recovery,
// the plastic-return iteration and the totals in FP64.
#include "mm_launch.cuh"

cudaError_t mm_p32_d2(int what, int axis, int flag, const KArgs& a, double* out, int nblocks,
                      cudaStream_t s) {
  return mm::Launch<mm::P32>::by_mat<2>(what, axis, flag, a, out, nblocks, s);
}
