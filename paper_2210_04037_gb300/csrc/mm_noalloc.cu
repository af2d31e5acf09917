// Conserved totals of a caller-held device state, with no allocation.
//
// Callers that cannot allocate device memory -- a serving loop that owns a
// fixed memory pool and must not let a library call cudaMalloc (which can
// synchronise the device and fragment the pool), or code running where the
// CUDA allocator is off limits -- use mm_conserved_totals_noalloc.  Its block
// partial sums live in one file-scope device array of fixed size that every
// GPU which loads this library keeps until the process exits.  The host
// code must not pass the array's name to a kernel (in host code it names a
// host-side stand-in); it resolves the device address with
// cudaGetSymbolAddress at every call and passes that.
#include <cuda_runtime.h>

#include <cstdio>

#include "mm_internal.h"
#include "mmfrac.h"

namespace {

constexpr int kNoallocBlocks = 1024;                 // partial rows
constexpr int kNoallocQuantities = MM_MAXMAT + 4;    // N masses, 3 momenta, energy

// Shared by every call on a device; each call overwrites every row it
// reads, so nothing has to be cleared between calls.
static __device__ __align__(256) double mm_noalloc_partial[kNoallocBlocks * kNoallocQuantities];

// Device address of the scratch array in the current context.  Looked up at
// every call (a host-side table lookup once the module is loaded) rather
// than cached, so that it stays right after a context is reset and the
// module loaded again at another address.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, mm_noalloc_partial);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

// Per-block sums of (phi rho)_l, rho u_k and rho E over [field][cell] FP64
// conserved fields; block b writes row b of the scratch.
__global__ void __launch_bounds__(256)
    k_noalloc_partial(const double* U, long long ncell, int nmat, int o_mom, int dim, int o_E,
                      double* partial) {
  double acc[kNoallocQuantities];
  for (int q = 0; q < kNoallocQuantities; ++q) acc[q] = 0.0;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    for (int l = 0; l < nmat; ++l) acc[l] += U[(long long)(nmat - 1 + l) * ncell + c];
    for (int k = 0; k < dim; ++k) acc[nmat + k] += U[(long long)(o_mom + k) * ncell + c];
    acc[nmat + 3] += U[(long long)o_E * ncell + c];
  }
  __shared__ double red[8][kNoallocQuantities];
  const int nq = nmat + 4;
  for (int q = 0; q < nq; ++q) {
    double v = acc[q];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < nq) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
    partial[(long long)blockIdx.x * nq + threadIdx.x] = s;
  }
}

// One warp per quantity sums the block rows into the caller's output.
__global__ void k_noalloc_final(const double* partial, int nblocks, int nq, double dV,
                                double* out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= nq) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * nq + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[q] = s * dV;
}

mm_status reject(mm_status st, const char* msg) {
  mm_internal_set_error(msg);
  return st;
}

}  // namespace

extern "C" mm_status mm_conserved_totals_noalloc(const double* d_cons, int dim, int64_t ncell,
                                                 int n_materials, int n_plastic,
                                                 const double dx[3], double* d_out,
                                                 void* cuda_stream) {
  char msg[256];
  if (!d_cons || !d_out || !dx) return reject(MM_EINVAL, "mm_conserved_totals_noalloc: null argument");
  if (dim < 1 || dim > 3 || ncell < 1 || n_plastic < 0 || n_plastic > n_materials)
    return reject(MM_EINVAL, "mm_conserved_totals_noalloc: bad dim, ncell or n_plastic");
  if (n_materials < 1 || n_materials + 4 > kNoallocQuantities) {
    snprintf(msg, sizeof msg,
             "mm_conserved_totals_noalloc: %d materials exceed the fixed scratch of %d "
             "quantities x %d blocks (at most %d materials)",
             n_materials, kNoallocQuantities, kNoallocBlocks, kNoallocQuantities - 4);
    return reject(MM_EINVAL, msg);
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "mm_conserved_totals_noalloc: cudaGetSymbolAddress: %s",
             cudaGetErrorString(e));
    return reject(MM_ECUDA, msg);
  }
  const int o_mom = (n_materials - 1) + n_materials;
  const int o_E = o_mom + dim;
  long long nb = (ncell + 255) / 256;
  if (nb > kNoallocBlocks) nb = kNoallocBlocks;
  double dV = 1.0;
  for (int k = 0; k < dim; ++k) dV *= dx[k];
  cudaStream_t s = (cudaStream_t)cuda_stream;
  k_noalloc_partial<<<(unsigned)nb, 256, 0, s>>>(d_cons, ncell, n_materials, o_mom, dim, o_E,
                                                 scratch);
  k_noalloc_final<<<1, 32 * (n_materials + 4), 0, s>>>(scratch, (int)nb, n_materials + 4, dV,
                                                        d_out);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    snprintf(msg, sizeof msg, "mm_conserved_totals_noalloc: launch: %s", cudaGetErrorString(e));
    return reject(MM_ECUDA, msg);
  }
  return MM_OK;
}
