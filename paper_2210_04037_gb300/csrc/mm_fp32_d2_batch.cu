// FP32-split batched kernels for 2D grids: one launch per kernel kind over
// every member of a batch (same cell arithmetic as the single-grid kernels).
#include "mm_launch.cuh"

cudaError_t mm_p32_d2_batch(int what, int axis, int variant, int nmat, int nhist, const BatchK& b,
                   cudaStream_t s) {
  return mm::Launch<mm::P32>::by_mat_batch<2>(what, axis, variant, nmat, nhist, b, s);
}

long long mm_p32_d2_batch_tiles(int axis, int variant, const int n[3]) {
  return mm::Launch<mm::P32>::tiles<2>(axis, mm::P32::split ? variant : 0, n);
}
