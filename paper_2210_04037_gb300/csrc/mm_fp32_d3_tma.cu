// The TMA-staged y and z sweeps of 3D FP32-split grids of two materials and
// the encoder of their tensor maps (a unit of its own, so that it compiles
// beside mm_fp32_d3.cu; the same FP32 flags, the same sweep code).
#include <cstring>

#include "mm_launch.cuh"

using namespace mm;

namespace {

template <int NH, int AX>
cudaError_t col_tma(const KArgs& a, int K, unsigned grid, const ColTma& tm, cudaStream_t s) {
  typedef SweepShape<P32, 3, 2, NH, AX, 0> SH;
  cudaError_t e = smem_attr<k_sweep_col_tma<P32, 3, 2, NH, AX>>(SH::smem);
  if (e != cudaSuccess) return e;
  k_sweep_col_tma<P32, 3, 2, NH, AX><<<grid, SH::NT, SH::smem, s>>>(a, K, tm);
  return cudaGetLastError();
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// cuTensorMapEncodeTiled through the runtime's driver entry points (the
// library links no driver library); null where it is unavailable.
EncodeTiled encoder() {
  static const EncodeTiled fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return EncodeTiled(nullptr);
    return reinterpret_cast<EncodeTiled>(p);
  }();
  return fn;
}

}  // namespace

cudaError_t mm_p32_d3_col_tma(int nhist, int axis, const KArgs& a, int K, unsigned grid,
                              const ColTma& tm, cudaStream_t s) {
  if (nhist == 0) return axis == 1 ? col_tma<0, 1>(a, K, grid, tm, s) : col_tma<0, 2>(a, K, grid, tm, s);
  return axis == 1 ? col_tma<1, 1>(a, K, grid, tm, s) : col_tma<1, 2>(a, K, grid, tm, s);
}

bool mm_p32_d3_tma_encode(SweepTmaSet* out, void* const U[2], double* const E[2], const int n[3],
                          int nmat, int nhist) {
  // rows of 16-byte multiples (float rows: n0 a multiple of 4)
  if (nmat != 2 || nhist < 0 || nhist > 1 || n[0] % 4 != 0) return false;
  const EncodeTiled enc = encoder();
  if (!enc) return false;
  const int oE = (nmat - 1) + nmat + 3;
  const int NF = oE + 1 + 9 + 2 * nhist + 3;  // float slots 0 .. NF (slot NF: last fraction)
  static_assert(Tile<P32, 3, 1>::TW == Tile<P32, 3, 2>::TW, "one box width");
  const cuuint32_t TW = Tile<P32, 3, 1>::TW;
  const cuuint32_t TLs[2] = {Tile<P32, 3, 1>::TL, Tile<P32, 3, 2>::TL};
  const cuuint64_t n0 = n[0], n1 = n[1], n2 = n[2], ncell = n0 * n1 * n2;
  SweepTmaSet t;
  memset(&t, 0, sizeof t);
  const cuuint32_t one[4] = {1, 1, 1, 1};
  for (int b = 0; b < 2; ++b) {
    t.U[b] = U[b];
    for (int ax = 1; ax <= 2; ++ax) {
      const cuuint32_t TL = TLs[ax - 1];
      const cuuint32_t by = ax == 1 ? TL : 1, bz = ax == 2 ? TL : 1;
      const cuuint64_t dimf[4] = {n0, n1, n2, cuuint64_t(NF + 1)};
      const cuuint64_t strf[3] = {n0 * 4, n0 * n1 * 4, ncell * 4};
      const cuuint32_t boxlo[4] = {TW, by, bz, cuuint32_t(oE)};
      const cuuint32_t boxhi[4] = {TW, by, bz, cuuint32_t(NF - oE)};
      const cuuint64_t dime[3] = {n0, n1, n2};
      const cuuint64_t stre[2] = {n0 * 8, n0 * n1 * 8};
      const cuuint32_t boxe[3] = {TW, by, bz};
      ColTma& m = t.m[b][ax - 1];
      if (enc(&m.lo, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, U[b], dimf, strf, boxlo, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
          enc(&m.hi, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, U[b], dimf, strf, boxhi, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
          enc(&m.e, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, E[b], dime, stre, boxe, one,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    }
  }
  t.nlo = oE;
  t.nhi = NF - oE;
  t.TL[0] = int(TLs[0]);
  t.TL[1] = int(TLs[1]);
  t.TW = int(TW);
  *out = t;
  return true;
}
