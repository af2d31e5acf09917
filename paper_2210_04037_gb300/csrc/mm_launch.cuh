// Host-side launchers: dispatch a runtime (dim, materials, plastic
// materials) triple to the kernel instantiations of one precision policy.
#pragma once

#include "mm_kernels.cuh"

namespace mm {

__global__ void k_totals_final(const double* partial, int nblocks, int nq, double dV, double* out);

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

template <class P>
struct Launch {
  template <int DIM, int NMAT, int NH, int AX>
  static cudaError_t sweep_ax(KArgs a, cudaStream_t s) {
    typedef SweepShape<P, DIM, NMAT, NH, AX> SH;
    constexpr int TD = (AX == 0) ? 1 : 0;
    constexpr int RD = 3 - AX - TD;
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_sweep<P, DIM, NMAT, NH, AX>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SH::smem);
      if (e != cudaSuccess) return e;
      attr = true;
    }
    a.tiles[0] = (a.n[AX] + SH::TL - 1) / SH::TL;
    a.tiles[1] = (a.n[TD] + SH::TW - 1) / SH::TW;
    a.tiles[2] = a.n[RD];
    const long long nb = (long long)a.tiles[0] * a.tiles[1] * a.tiles[2];
    k_sweep<P, DIM, NMAT, NH, AX><<<(unsigned)nb, SH::NT, SH::smem, s>>>(a);
    return cudaGetLastError();
  }

  template <int DIM, int NMAT, int NH>
  static cudaError_t sweep_t(int axis, KArgs a, cudaStream_t s) {
    if (axis == 0) return sweep_ax<DIM, NMAT, NH, 0>(a, s);
    if constexpr (DIM >= 2)
      if (axis == 1) return sweep_ax<DIM, NMAT, NH, 1>(a, s);
    if constexpr (DIM >= 3)
      if (axis == 2) return sweep_ax<DIM, NMAT, NH, 2>(a, s);
    return cudaErrorInvalidValue;
  }

  template <int DIM, int NMAT, int NH>
  static cudaError_t run(int what, int axis, int flag, KArgs a, double* out, int nblocks,
                         cudaStream_t s) {
    switch (what) {
      case 0: {
        k_init<P, DIM, NMAT, NH><<<grid_for(a.ncell, 128), 128, 0, s>>>(a);
        break;
      }
      case 1: {
        k_read<P, DIM, NMAT, NH><<<grid_for(a.ncell, 128), 128, 0, s>>>(a, flag);
        break;
      }
      case 2: {
        k_cfl<P, DIM, NMAT, NH><<<grid_for(a.ncell, 256), 256, 0, s>>>(a);
        break;
      }
      case 3:
        return sweep_t<DIM, NMAT, NH>(axis, a, s);
      case 4: {
        k_sources<P, DIM, NMAT, NH><<<grid_for(a.ncell, 128), 128, 0, s>>>(a);
        break;
      }
      case 5: {
        k_totals<P, DIM, NMAT, NH><<<nblocks, 256, 0, s>>>(a);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        double dV = 1.0;
        for (int k = 0; k < DIM; ++k) dV *= a.dx[k];
        k_totals_final<<<1, 32 * (NMAT + 4), 0, s>>>(a.partial, nblocks, NMAT + 4, dV, out);
        break;
      }
      default:
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }

  template <int DIM>
  static cudaError_t by_mat(int what, int axis, int flag, KArgs a, double* out, int nblocks,
                            cudaStream_t s) {
    if (a.nmat == 1 && a.nhist == 0) return run<DIM, 1, 0>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 1 && a.nhist == 1) return run<DIM, 1, 1>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 2 && a.nhist == 0) return run<DIM, 2, 0>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 2 && a.nhist == 1) return run<DIM, 2, 1>(what, axis, flag, a, out, nblocks, s);
    return cudaErrorInvalidValue;
  }

};

}  // namespace mm
