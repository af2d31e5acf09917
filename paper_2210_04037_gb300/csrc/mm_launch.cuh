// Host-side launchers: dispatch a runtime (dim, materials, plastic
// materials) triple to the kernel instantiations of one precision policy.
#pragma once

#include <atomic>

#include "mm_kernels.cuh"

namespace mm {

__global__ void k_totals_final(const double* partial, int nblocks, int nq, double dV, double* out);

// Batches of 128 cells each source CTA takes at least: the queue of
// yielding cells fills across them, so fewer returns run on part-filled
// warps.  Measured on the 512^2 ring (source kernel): 1 batch 42 us, 2: 42,
// 4: 36, 8: 50, 16: 75.  Grids of more than 2432 x 4 x 128 cells are capped
// at 2432 CTAs anyway.
#ifndef MM_SRC_BATCHES
#define MM_SRC_BATCHES 4
#endif

// Whole waves of resident CTAs the bounded FP32-split source kernel runs
// as (0: the 2432-CTA cap, 3.2 waves at 5 CTAs per SM, whose last part-wave
// left most SMs idle).  Measured on the 256^3 cylinder (steps 6-35): cap
// 1.66 ms, one wave 1.48, two 1.53, four 1.55.
#ifndef MM_SRC_WAVES
#define MM_SRC_WAVES 1
#endif

inline int grid_for(long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  if (b > 152LL * 16) b = 152LL * 16;
  if (b < 1) b = 1;
  return (int)b;
}

// Opt a kernel in to `smem` bytes of dynamic shared memory once per device
// and kernel (a bit per device, set after the call: threads that race both
// make the same call).  The kernel is a template argument so that every
// kernel has its own flags (kernels of one signature share a pointer type).
template <auto Kernel>
cudaError_t smem_attr(size_t smem) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_acquire) & bit) return cudaSuccess;
  e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done.fetch_or(bit, std::memory_order_release);
  return e;
}

template <class P>
struct Launch {
  template <int DIM, int NMAT, int NH, int AX>
  static cudaError_t sweep_ax(KArgs a, cudaStream_t s) {
    typedef SweepShape<P, DIM, NMAT, NH, AX> SH;
    constexpr int TD = (AX == 0) ? 1 : 0;
    constexpr int RD = 3 - AX - TD;
    const long long nta = (a.n[AX] + SH::TL - 1) / SH::TL;
    const long long cols = (long long)((a.n[TD] + SH::TW - 1) / SH::TW) * a.n[RD];
    // 3D y and z sweeps: chunks of K tiles along the sweep axis per CTA while
    // about 2432 CTAs (16 per SM) remain; K = 1 is one CTA per tile.  Measured
    // on GB300: the 256^3 z sweep 3.99 -> 3.57 ms, y 3.72 -> 3.67; x tiles are
    // long (halo 4 of TL + 4) and lost (3.63 -> 4.01), the 2048^2 2D y sweep
    // lost (0.50 -> 0.58 ms): those keep one tile per CTA
    long long K = (DIM == 3 && AX != 0) ? nta * cols / (152LL * 16) : 1;
    if (K > nta) K = nta;
    if (K <= 1) {
      cudaError_t e = smem_attr<k_sweep<P, DIM, NMAT, NH, AX>>(SH::smem);
      if (e != cudaSuccess) return e;
      k_sweep<P, DIM, NMAT, NH, AX><<<(unsigned)(nta * cols), SH::NT, SH::smem, s>>>(a);
      return cudaGetLastError();
    }
    const long long nch = (nta + K - 1) / K;
    if constexpr (std::is_same<P, P32>::value && DIM == 3 && AX != 0 && NMAT == 2 && NH <= 1) {
      // tiles staged by TMA where the grid has maps for this state buffer
      // (two materials; mm_fp32_d3_tma.cu)
      typedef StageShape<P, DIM, NMAT, NH, AX> CS;
      const SweepTmaSet* ts = static_cast<const SweepTmaSet*>(a.tma);
      const int b = !ts ? -1 : (a.Uin == ts->U[0] ? 0 : (a.Uin == ts->U[1] ? 1 : -1));
      if (b >= 0 && ts->nlo == CS::NLO && ts->nhi == CS::NHI && ts->TL[AX - 1] == SH::TL &&
          ts->TW == SH::TW)
        return mm_p32_d3_col_tma(NH, AX, a, (int)K, (unsigned)(nch * cols), ts->m[b][AX - 1], s);
    }
    cudaError_t e = smem_attr<k_sweep_col<P, DIM, NMAT, NH, AX>>(SH::smem);
    if (e != cudaSuccess) return e;
    k_sweep_col<P, DIM, NMAT, NH, AX><<<(unsigned)(nch * cols), SH::NT, SH::smem, s>>>(a, (int)K);
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
        // one wave of resident CTAs (the grid strides over the cells)
        int dev = 0, sms = 0, per = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
          e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_cfl<P, DIM, NMAT, NH>, 256, 0);
        if (e != cudaSuccess) return e;
        const int wave = sms * (per > 0 ? per : 1);
        const int need = grid_for(a.ncell, 256);
        k_cfl<P, DIM, NMAT, NH><<<need < wave ? need : wave, 256, 0, s>>>(a);
        break;
      }
      case 3:
        return sweep_t<DIM, NMAT, NH>(axis, a, s);
      case 6: {
        k_xvel<P, DIM, NMAT, NH><<<grid_for(a.ncell, 256), 256, 0, s>>>(a);
        break;
      }
      case 7: {
        k_xstage<P, DIM, NMAT, NH><<<grid_for(a.ncell, 256), 256, 0, s>>>(a, flag);
        break;
      }
      case 8: {
        k_frag_mark<P, DIM, NMAT, NH><<<grid_for(a.ncell, 256), 256, 0, s>>>(a);
        break;
      }
      case 9: {
        if constexpr (Voidable<P>::value)
          k_seed<P, DIM, NMAT, NH><<<grid_for(a.ncell, 256), 256, 0, s>>>(a);
        else
          return cudaErrorInvalidValue;
        break;
      }
      case 4: {
        const int g = grid_for(a.ncell, 128 * MM_SRC_BATCHES);
        bool bounded = false;
        if constexpr (P::split) {
          if (a.ncell >= 152LL * 16 * 128 * MM_SRC_BATCHES) {
            // MM_SRC_WAVES whole waves of resident CTAs (> 0), or the
            // 2432-CTA cap (0)
            int gw = g;
            if (MM_SRC_WAVES > 0) {
              int dev = 0, sms = 0, per = 0;
              cudaError_t e = cudaGetDevice(&dev);
              if (e == cudaSuccess)
                e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
              if (e == cudaSuccess)
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                    &per, k_sources<P, DIM, NMAT, NH, 5>, 128, 0);
              if (e != cudaSuccess) return e;
              gw = sms * (per > 0 ? per : 1) * MM_SRC_WAVES;
            }
            k_sources<P, DIM, NMAT, NH, 5><<<gw, 128, 0, s>>>(a);
            bounded = true;
          }
        }
        if (!bounded) k_sources<P, DIM, NMAT, NH, 1><<<g, 128, 0, s>>>(a);
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

  // ---- batched launches: persistent CTAs, one wave at full occupancy
  template <class K>
  static cudaError_t persistent(K kernel, int threads, size_t smem, BatchK b, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
    if (e != cudaSuccess) return e;
    if (per < 1) per = 1;
    if (b.cta_per_sm > 0 && b.cta_per_sm < per) per = b.cta_per_sm;
    long long grid = (long long)sms * per;
    if (grid > b.total - b.base) grid = b.total - b.base;
    if (grid < 1) return cudaSuccess;
    kernel<<<(unsigned)grid, threads, smem, s>>>(b);
    return cudaGetLastError();
  }

  template <int DIM, int NMAT, int NH, int AX, int V>
  static cudaError_t sweep_batch(BatchK b, cudaStream_t s) {
    typedef SweepShape<P, DIM, NMAT, NH, AX, V> SH;
    cudaError_t e = smem_attr<k_sweep_batch<P, DIM, NMAT, NH, AX, V>>(SH::smem);
    if (e != cudaSuccess) return e;
    return persistent(k_sweep_batch<P, DIM, NMAT, NH, AX, V>, SH::NT, SH::smem, b, s);
  }

  template <int DIM, int NMAT, int NH>
  static cudaError_t run_batch(int what, int axis, int variant, BatchK b, cudaStream_t s) {
    if (what == 0) return persistent(k_cfl_batch<P, DIM, NMAT, NH>, 256, 0, b, s);
    if (what == 2) return persistent(k_sources_batch<P, DIM, NMAT, NH>, 128, 0, b, s);
    if (what != 1) return cudaErrorInvalidValue;
#define MM_SWEEP_BATCH(AXIS)                                                     \
  if (axis == AXIS) {                                                            \
    if constexpr (P::split)                                                      \
      if (variant == 1) return sweep_batch<DIM, NMAT, NH, AXIS, 1>(b, s);        \
    return sweep_batch<DIM, NMAT, NH, AXIS, 0>(b, s);                            \
  }
    MM_SWEEP_BATCH(0)
    if constexpr (DIM >= 2) { MM_SWEEP_BATCH(1) }
    if constexpr (DIM >= 3) { MM_SWEEP_BATCH(2) }
#undef MM_SWEEP_BATCH
    return cudaErrorInvalidValue;
  }

  template <int DIM>
  static cudaError_t by_mat_batch(int what, int axis, int variant, int nmat, int nhist, BatchK b,
                                  cudaStream_t s) {
    if (!P::split) variant = 0;  // one FP64 tile shape
    if (nmat == 2 && nhist == 0) return run_batch<DIM, 2, 0>(what, axis, variant, b, s);
    if (nmat == 2 && nhist == 1) return run_batch<DIM, 2, 1>(what, axis, variant, b, s);
    return cudaErrorInvalidValue;
  }

  // Tiles of one sweep of a grid with n cells per axis (the tile shape does
  // not depend on the materials).
  template <int DIM>
  static long long tiles(int axis, int variant, const int n[3]) {
    int TL = 0, TW = 0;
#define MM_TILE_OF(AXIS)                                                                  \
  if (axis == AXIS) {                                                                     \
    TL = variant == 0 ? Tile<P, DIM, AXIS, 0>::TL : Tile<P, DIM, AXIS, 1>::TL;            \
    TW = variant == 0 ? Tile<P, DIM, AXIS, 0>::TW : Tile<P, DIM, AXIS, 1>::TW;            \
  }
    MM_TILE_OF(0)
    if constexpr (DIM >= 2) { MM_TILE_OF(1) }
    if constexpr (DIM >= 3) { MM_TILE_OF(2) }
#undef MM_TILE_OF
    if (TL == 0) return 0;
    const int TD = axis == 0 ? 1 : 0, RD = 3 - axis - TD;
    return (long long)((n[axis] + TL - 1) / TL) * ((n[TD] + TW - 1) / TW) * n[RD];
  }

  // grids with a void material: two or three materials, one plastic
  template <int DIM>
  static cudaError_t by_mat_void(int what, int axis, int flag, KArgs a, double* out,
                                 int nblocks, cudaStream_t s) {
    if (a.nmat == 2 && a.nhist == 1) return run<DIM, 2, 1>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 3 && a.nhist == 1) return run<DIM, 3, 1>(what, axis, flag, a, out, nblocks, s);
    return cudaErrorInvalidValue;
  }

  template <int DIM>
  static cudaError_t by_mat(int what, int axis, int flag, KArgs a, double* out, int nblocks,
                            cudaStream_t s) {
    if (a.nmat == 1 && a.nhist == 0) return run<DIM, 1, 0>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 1 && a.nhist == 1) return run<DIM, 1, 1>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 2 && a.nhist == 0) return run<DIM, 2, 0>(what, axis, flag, a, out, nblocks, s);
    if (a.nmat == 2 && a.nhist == 1) return run<DIM, 2, 1>(what, axis, flag, a, out, nblocks, s);
    // two plastic solids (with or without a gas), 1D and 2D grids
    if constexpr (DIM <= 2) {
      if (a.nmat == 2 && a.nhist == 2) return run<DIM, 2, 2>(what, axis, flag, a, out, nblocks, s);
      if (a.nmat == 3 && a.nhist == 2) return run<DIM, 3, 2>(what, axis, flag, a, out, nblocks, s);
    }
    return cudaErrorInvalidValue;
  }

};

}  // namespace mm
