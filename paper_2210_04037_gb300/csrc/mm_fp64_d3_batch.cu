// FP64 batched kernels for 3D grids: one launch per kernel kind over
// every member of a batch (same cell arithmetic as the single-grid kernels).
#include "mm_launch.cuh"

cudaError_t mm_p64_d3_batch(int what, int axis, int variant, int nmat, int nhist, const BatchK& b,
                   cudaStream_t s) {
  return mm::Launch<mm::P64>::by_mat_batch<3>(what, axis, variant, nmat, nhist, b, s);
}

long long mm_p64_d3_batch_tiles(int axis, int variant, const int n[3]) {
  return mm::Launch<mm::P64>::tiles<3>(axis, mm::P64::split ? variant : 0, n);
}
