// Kernels of one explicit step: CFL reduction, the dimensionally split
// MUSCL-Hancock sweeps (shared-memory tiles along the sweep axis), the
// per-cell sources (perturbed plastic return + RK4 damage), initial-state
// conversion, field read-back and FP64 totals.  Included by the precision
// translation units, which instantiate them for FP64 and FP32-split.
#pragma once

#include <type_traits>

#include "mm_phys.cuh"

namespace mm {

enum { ST_ECUDA = -3, ST_ENONFINITE = -4, ST_ENOCONV = -5, ST_EDT = -6, ST_ETIMEOUT = -7 };
enum { BC_T = 0, BC_P = 1, BC_R = 2 };

__device__ __forceinline__ void report(DevErr* e, int code, long long cell, long long step) {
  if (atomicCAS(&e->code, 0, code) == 0) {
    e->cell = cell;
    e->step = step;
  }
}

// ------------------------------------------------ TMA and mbarrier (PTX) ----
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// One-arrival mbarrier at shared address bar, made visible to the async
// proxy (TMA) before its first use.
__device__ __forceinline__ void mbar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The arrival of the phase, expecting `bytes` of TMA writes before it completes.
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Orders the CTA's earlier generic accesses of shared memory (a barrier
// before it makes every thread's visible) before later TMA writes there.
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Tiled TMA loads of a box at element coordinates (x first) into shared
// memory at dst, completing `box bytes` on the mbarrier at bar.  The map is
// a kernel parameter (__grid_constant__).  x times the element size is a
// multiple of 16 bytes at every call site; boxes reaching outside the
// tensor read zeros there.
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* m, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* m, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(m)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

// Waits until the phase of the given parity of the mbarrier at bar has
// completed, for at most one second of the global timer (and 2^26 tries);
// false when the wait gave up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  unsigned long long t0 = 0;
  for (long long it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (it == 0)
      t0 = t;
    else if (t - t0 > 1000000000ull || it > (1LL << 26))
      return false;
  }
}

// Derived quantities of a state kept beside it in shared memory: the stress
// column and row (the FP64 path keeps both, which differ in the last ulp;
// the split path keeps the column of the symmetric stress only), density,
// c_L and G.  NAUX values.
template <class P>
struct AuxRec {
  static constexpr int N = P::split ? 6 : 9;
};

template <class P, class R>
__device__ __forceinline__ void put_aux(R* q, const Aux<R>& ax) {
  constexpr int o = P::split ? 3 : 6;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    q[k] = ax.sd[k];
    if (!P::split) q[3 + k] = ax.sr[k];
  }
  q[o] = ax.rho;
  q[o + 1] = ax.cL;
  q[o + 2] = ax.G;
}

template <class P, class R>
__device__ __forceinline__ void get_aux(const R* q, Aux<R>& ax) {
  constexpr int o = P::split ? 3 : 6;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    ax.sd[k] = q[k];
    ax.sr[k] = P::split ? q[k] : q[3 + k];
  }
  ax.rho = q[o];
  ax.cL = q[o + 1];
  ax.G = q[o + 2];
}

template <class R>
__device__ __forceinline__ R van_leer(R a, R b) {
  return (a * b > R(0)) ? R(2) * a * b / (a + b) : R(0);
}

__device__ __forceinline__ long long cell_index(const KArgs& a, int x, int y, int z) {
  return (long long)x + (long long)a.n[0] * ((long long)y + (long long)a.n[1] * z);
}

// Storage of the second block.  FP64: rho E and phi_0..phi_{N-2} in their
// slots of the field array.  FP32-split: rho E in the FP64 side array, the N
// volume fractions as floats in the phi slots plus one extra slot NF.
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ long long phislot(const KArgs& a, int l, long long idx) {
  typedef Lay<DIM, NMAT, NH> L;
  return (long long)(l < L::NPHI ? L::oPHI + l : L::NF) * a.ncell + idx;
}

template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void load_at(const KArgs& a, long long idx, typename P::R* c,
                                        typename P::X* cx, double* rhoE) {
  typedef typename P::R R;
  typedef typename P::S S;
  typedef typename P::X XT;
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int NPX = Phys<P, DIM, NMAT, NH>::NPX;
  const S* U = (const S*)a.Uin;
#pragma unroll
  for (int f = 0; f < L::NF; ++f)
    c[f] = (f == L::oE || f < L::oARHO) ? R(0) : R(U[(long long)f * a.ncell + idx]);
#pragma unroll
  for (int l = 0; l < NPX; ++l) cx[1 + l] = XT(U[phislot<P, DIM, NMAT, NH>(a, l, idx)]);
  const double e = P::split ? a.Ein[idx] : double(U[(long long)L::oE * a.ncell + idx]);
  cx[0] = XT(e);
  *rhoE = e;
}

// Load the conserved state of the cell at axis position gi (ghost cells via
// the boundary rule of that side), transverse position gw, rest rr.
template <class P, int DIM, int NMAT, int NH, int AX>
__device__ __forceinline__ long long load_cell(const KArgs& a, int gi, int gw, int rr,
                                               typename P::R* c, typename P::X* cx,
                                               double* rhoE) {
  typedef typename P::R R;
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int TD = (AX == 0) ? 1 : 0;
  constexpr int RD = 3 - AX - TD;
  const int n = a.n[AX];
  int src = gi, side = -1, kind = BC_T;
  if (gi < 0) {
    side = 0;
    kind = a.bc[AX][0];
    src = kind == BC_P ? gi + n : (kind == BC_R ? -1 - gi : 0);
  } else if (gi >= n) {
    side = 1;
    kind = a.bc[AX][1];
    src = kind == BC_P ? gi - n : (kind == BC_R ? 2 * n - 1 - gi : n - 1);
  }
  src = src < 0 ? 0 : (src > n - 1 ? n - 1 : src);
  int co[3];
  co[AX] = src;
  co[TD] = gw;
  co[RD] = rr;
  const long long idx = cell_index(a, co[0], co[1], co[2]);
  load_at<P, DIM, NMAT, NH>(a, idx, c, cx, rhoE);
  if (side >= 0 && kind == BC_P) {
    const R Lx = R(a.hi[AX] - a.lo[AX]);
    c[L::oX + AX] += side == 0 ? -Lx : Lx;
  } else if (side >= 0 && kind == BC_R) {
    c[L::oMOM + AX] = -c[L::oMOM + AX];
#pragma unroll
    for (int k = 0; k < L::NFC; ++k) {
      const int i = FC<DIM>::idx(k) / 3, j = FC<DIM>::idx(k) % 3;
      if ((i == AX) != (j == AX)) c[L::oF + k] = -c[L::oF + k];
    }
    const R wall = R(side == 0 ? a.lo[AX] : a.hi[AX]);
    c[L::oX + AX] = R(2) * wall - c[L::oX + AX];
  }
  return idx;
}

template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void store_cell(const KArgs& a, long long idx, const typename P::R* c,
                                           const typename P::X* cx, double rhoE) {
  typedef typename P::S S;
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int NPX = Phys<P, DIM, NMAT, NH>::NPX;
  S* U = (S*)a.Uout;
#pragma unroll
  for (int f = 0; f < L::NF; ++f)
    if (f != L::oE && f >= L::oARHO) U[(long long)f * a.ncell + idx] = S(c[f]);
#pragma unroll
  for (int l = 0; l < NPX; ++l) U[phislot<P, DIM, NMAT, NH>(a, l, idx)] = S(cx[1 + l]);
  if (P::split)
    a.Eout[idx] = rhoE;
  else
    U[(long long)L::oE * a.ncell + idx] = S(rhoE);
}

// In-place store of the deformation tensor (and optionally the history) of
// one cell: the fields the source step changes.
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void store_sources(const KArgs& a, long long idx,
                                              const typename P::R* c, bool hist) {
  typedef typename P::S S;
  typedef Lay<DIM, NMAT, NH> L;
  S* U = (S*)a.Uout;
#pragma unroll
  for (int k = 0; k < L::NFC; ++k) U[(long long)(L::oF + k) * a.ncell + idx] = S(c[L::oF + k]);
  if (hist) {
#pragma unroll
    for (int k = 0; k < 2 * NH; ++k) U[(long long)(L::oH + k) * a.ncell + idx] = S(c[L::oH + k]);
  }
}

// Still state: zero velocity, and every field but X equal to the reference
// state (exact comparisons; -0 equals +0).  A line of cells in such states
// keeps them through a sweep bit for bit, up to the sign of a zero: every
// slope but those of X is zero, both face states are the cell's, the
// Riemann problems between them are contacts at rest with equal sides, and
// the update adds lam (F - F + 0) = 0 to each field (X moves with u = 0).
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ bool same_state(const typename P::R* c, const typename P::X* cx,
                                           double e, const typename P::R* cr,
                                           const typename P::X* cxr, double er) {
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int NX = Phys<P, DIM, NMAT, NH>::NX;
  bool s = e == er;
#pragma unroll
  for (int f = 0; f < L::oX; ++f) s = s && c[f] == cr[f];
#pragma unroll
  for (int k = 0; k < NX; ++k) s = s && cx[k] == cxr[k];
  return s;
}

template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ bool same_still(const typename P::R* c, const typename P::X* cx,
                                           double e, const typename P::R* cr,
                                           const typename P::X* cxr, double er) {
  typedef Lay<DIM, NMAT, NH> L;
  bool s = true;
#pragma unroll
  for (int k = 0; k < DIM; ++k) s = s && c[L::oMOM + k] == 0;
  return s && same_state<P, DIM, NMAT, NH>(c, cx, e, cr, cxr, er);
}

// ------------------------------------------------------------------ sweep ----
template <class P, int DIM, int AX, int V = 0> struct Tile;
// The halo-extended tile (TL + 4) x TW equals the CTA, so each phase is one
// pass of the threads (phases 2-4 have 2, 3 and 4 fewer rows of items).
// FP64 (compute bound on GB300's FP64 rate): 64-thread CTAs.
template <> struct Tile<P64, 1, 0> { static constexpr int TL = 60, TW = 1, NT = 64; };
template <> struct Tile<P64, 2, 0> { static constexpr int TL = 28, TW = 2, NT = 64; };
template <> struct Tile<P64, 2, 1> { static constexpr int TL = 12, TW = 4, NT = 64; };
template <> struct Tile<P64, 3, 0> { static constexpr int TL = 28, TW = 2, NT = 64; };
template <> struct Tile<P64, 3, 1> { static constexpr int TL = 12, TW = 4, NT = 64; };
template <> struct Tile<P64, 3, 2> { static constexpr int TL = 12, TW = 4, NT = 64; };
// FP32-split 1D and 2D: 128-thread CTAs (256 for the 2D y sweep).
// 3D: 192-thread CTAs, two per SM (the same twelve warps as three of 128,
// which the registers and shared memory allow either way).  The x sweep's
// tile is one 32-cell row per warp in phase 1 (28 x 6); the y and z sweeps
// run columns of 12 x 16 tiles (each tile's 192 new cells, one per thread,
// in rows of 64 bytes along x).  Measured on the 256^3 cylinder over steps
// 16-25 (per-kernel CUDA events, identical results): x 28 x 4 -> 28 x 6
// 3.81 -> 3.66 ms; y 16 x 8 -> 12 x 16 3.62 -> 3.08, z 3.07 -> 2.89 (these
// two with the log series' finer tiers, which gave x 3.63).  Not
// kept: one 384-thread CTA per SM (x 28 x 12: 3.91; y, z 16 x 24: 3.41,
// 3.05), 16 x 12 (y 3.10, z 2.94), 8 x 24 (y 4.80, z 4.39), 16 x 16 with
// 256 threads and one CTA per SM (y 3.66, z 3.29), x 60 x 3 (4.07).
template <> struct Tile<P32, 1, 0> { static constexpr int TL = 124, TW = 1, NT = 128; };
template <> struct Tile<P32, 2, 0> { static constexpr int TL = 60, TW = 2, NT = 128; };
template <> struct Tile<P32, 2, 1> { static constexpr int TL = 28, TW = 8, NT = 256; };
template <> struct Tile<P32, 3, 0> { static constexpr int TL = 28, TW = 6, NT = 192; };
template <> struct Tile<P32, 3, 1> { static constexpr int TL = 12, TW = 16, NT = 192; };
template <> struct Tile<P32, 3, 2> { static constexpr int TL = 12, TW = 16, NT = 192; };
// Second shape per axis, one of the two the batched sweep's autotuner times
// (the cell arithmetic does not depend on the tile, so either gives the same
// bits): longer tiles along the sweep, narrower across it.
template <class P, int DIM, int AX> struct Tile<P, DIM, AX, 1> : Tile<P, DIM, AX, 0> {};
// grids that can open void take the single-grid tiles of their precision
template <int DIM, int AX> struct Tile<P64V, DIM, AX, 0> : Tile<P64, DIM, AX, 0> {};
template <int DIM, int AX> struct Tile<P32V, DIM, AX, 0> : Tile<P32, DIM, AX, 0> {};
// but 3D void grids keep 128-thread CTAs: their column kernels take 218-228
// registers, so a 192-thread CTA would run alone on an SM
template <> struct Tile<P32V, 3, 0> { static constexpr int TL = 28, TW = 4, NT = 128; };
template <> struct Tile<P32V, 3, 1> { static constexpr int TL = 16, TW = 8, NT = 128; };
template <> struct Tile<P32V, 3, 2> { static constexpr int TL = 16, TW = 8, NT = 128; };
template <> struct Tile<P32, 1, 0, 1> { static constexpr int TL = 60, TW = 1, NT = 64; };
template <> struct Tile<P32, 2, 0, 1> { static constexpr int TL = 60, TW = 2, NT = 128; };
template <> struct Tile<P32, 2, 1, 1> { static constexpr int TL = 28, TW = 4, NT = 128; };
template <> struct Tile<P32, 3, 0, 1> { static constexpr int TL = 60, TW = 2, NT = 128; };
template <> struct Tile<P32, 3, 1, 1> { static constexpr int TL = 28, TW = 4, NT = 128; };
template <> struct Tile<P32, 3, 2, 1> { static constexpr int TL = 28, TW = 4, NT = 128; };

template <class P, int DIM, int NMAT, int NH, int AX, int V = 0>
struct SweepShape {
  typedef typename P::R R;
  static constexpr int TL = Tile<P, DIM, AX, V>::TL, TW = Tile<P, DIM, AX, V>::TW;
  static constexpr int NT = Tile<P, DIM, AX, V>::NT;
  static constexpr int NF = Lay<DIM, NMAT, NH>::NF;
  static constexpr int C1 = NF + AuxRec<P>::N, C2 = NF + AuxRec<P>::N, C3 = NF + 4;
  static constexpr int N1 = (TL + 4) * TW, N2 = (TL + 2) * TW, N3 = (TL + 1) * TW, N4 = TL * TW;
  static constexpr int NX = Phys<P, DIM, NMAT, NH>::NX;
  // face records per face: one, or (grids that can open void) the record
  // the cell left of the face takes and the one the cell right of it takes
  static constexpr int NR = Voidable<P>::value ? 2 : 1;
  static constexpr size_t smem = sizeof(typename P::X) * NX * (size_t(N1) + 2 * size_t(N2) + NR * size_t(N3)) +
                                 sizeof(R) * (size_t(N1) * C1 + 2 * size_t(N2) * C2 + NR * size_t(N3) * C3);
  __device__ static __forceinline__ int idx(int p, int w, int len) {
    return AX == 0 ? w * len + p : p * TW + w;
  }
  __device__ static __forceinline__ void pos(int it, int len, int& p, int& w) {
    if (AX == 0) {
      p = it % len;
      w = it / len;
    } else {
      w = it % TW;
      p = it / TW;
    }
  }
};

// TMA staging of the y and z sweeps' tiles (3D FP32-split; columns of
// tiles per CTA, k_sweep_col_tma): the TL new cells x TW of a tile (axis
// positions 4 .. TL + 3, the rows a0 + 2 .. a0 + TL + 1) as three boxes of
// BE = TL TW elements per slot, each starting on a 128-byte boundary as the
// copies require: float slots 0 .. oE - 1 (at 0), slots oE + 1 .. NF (at
// OHI; slot oE is unused in the split form), then rho E (doubles, at OE);
// element (slot s, position p, column w) at s BE + (p - 4) TW + w.  The
// boxes sit in the half-step records (r2) between the two items carried at
// the front and the two carried from the end, which are dead from phase 4
// of one tile (when the next tile's copy is issued) to phase 1 of the next
// (when it is read).
template <class P, int DIM, int NMAT, int NH, int AX>
struct StageShape {
  typedef SweepShape<P, DIM, NMAT, NH, AX, 0> SH;
  static_assert(P::split && sizeof(typename P::R) == 4 && sizeof(typename P::X) == 4 &&
                    DIM == 3 && AX != 0,
                "staging of the 3D FP32-split y and z sweeps");
  typedef Lay<DIM, NMAT, NH> L;
  static constexpr int NLO = L::oE, NHI = L::NF - L::oE;
  static constexpr int BE = SH::TL * SH::TW;
  static constexpr uint32_t SLOT = uint32_t(BE) * 4;
  static constexpr uint32_t OHI = (NLO * SLOT + 127u) & ~127u;
  static constexpr uint32_t OE = (OHI + NHI * SLOT + 127u) & ~127u;
  static constexpr uint32_t bytes = (NLO + NHI) * SLOT + uint32_t(BE) * 8;  // the copies deliver
  static constexpr uint32_t span = OE + uint32_t(BE) * 8;                    // the boxes take
  static constexpr size_t r2 = 4 * size_t(SH::NX) * (size_t(SH::N1) + 2 * size_t(SH::N2) +
                                                     SH::NR * size_t(SH::N3)) +
                               4 * size_t(SH::N1) * SH::C1;
  // first byte past the front carried items, and the start of the end ones
  static constexpr size_t lo = r2 + 4 * size_t(4 * SH::TW) * SH::C2;
  static constexpr size_t hi = r2 + 4 * size_t(2 * SH::TL * SH::TW) * SH::C2;
  static_assert(lo + 127 + span <= hi, "the staged boxes fit between the carried records");
  __device__ static __forceinline__ int pos(int p, int w) { return (p - 4) * SH::TW + w; }
};

// The staging state of a CTA: maps, mbarrier, the wait's phase parity (per
// thread), the boxes' offset from the dynamic shared memory, whether every
// wait so far completed, and the tile whose copy the current tile issues
// (next: there is one; its axis tile, first transverse cell, remaining
// index).
struct ColStage {
  const ColTma* tm;
  DevErr* err;
  uint32_t bar;
  uint32_t parity;
  uint32_t dst;  // shared address of the boxes (128-byte aligned)
  uint32_t off;  // dst - shared address of the dynamic shared memory
  bool ok;
  bool next;
  int nta, nw0, nrr;
};

// Issues the copies of the new cells of tile (ta, w0, rr) (one thread;
// after a barrier that ends every generic access of the boxes' bytes).
template <class P, int DIM, int NMAT, int NH, int AX>
__device__ __forceinline__ void stage_issue(const ColStage& st, int ta, int w0, int rr) {
  typedef StageShape<P, DIM, NMAT, NH, AX> CS;
  const int r0 = ta * CS::SH::TL + 2;
  const int x = w0, y = AX == 1 ? r0 : rr, z = AX == 1 ? rr : r0;
  static_assert(CS::OHI % 128 == 0 && CS::OE % 128 == 0, "box starts on 128-byte boundaries");
  fence_async_shared();
  if (st.dst & 127u) {
    // never by construction; the copies would fault: complete the phase
    // without them and report
    report(st.err, ST_ECUDA, 0, 0);
    mbar_expect_tx(st.bar, 0);
    return;
  }
  mbar_expect_tx(st.bar, CS::bytes);
  tma_load_4d(st.dst, &st.tm->lo, x, y, z, 0, st.bar);
  tma_load_4d(st.dst + CS::OHI, &st.tm->hi, x, y, z, CS::NLO + 1, st.bar);
  tma_load_3d(st.dst + CS::OE, &st.tm->e, x, y, z, st.bar);
}

// The conserved state of a staged cell (box position pos): the values
// load_at reads from global memory.
template <class P, int DIM, int NMAT, int NH, int AX>
__device__ __forceinline__ void stage_at(const unsigned char* box, int pos, typename P::R* c,
                                         typename P::X* cx, double* rhoE) {
  typedef StageShape<P, DIM, NMAT, NH, AX> CS;
  typedef Lay<DIM, NMAT, NH> L;
  typedef typename P::R R;
  typedef typename P::X XT;
  constexpr int NPX = Phys<P, DIM, NMAT, NH>::NPX, BE = CS::BE;
  const float* lo = reinterpret_cast<const float*>(box);
  const float* hi = reinterpret_cast<const float*>(box + CS::OHI);
  const double* ev = reinterpret_cast<const double*>(box + CS::OE);
#pragma unroll
  for (int f = 0; f < L::NF; ++f)
    c[f] = (f == L::oE || f < L::oARHO) ? R(0)
                                        : R(f < L::oE ? lo[f * BE + pos]
                                                      : hi[(f - L::oE - 1) * BE + pos]);
#pragma unroll
  for (int l = 0; l < NPX; ++l) {
    const int slot = l < L::NPHI ? L::oPHI + l : L::NF;
    cx[1 + l] = XT(slot < L::oE ? lo[slot * BE + pos] : hi[(slot - L::oE - 1) * BE + pos]);
  }
  const double e = ev[pos];
  cx[0] = XT(e);
  *rhoE = e;
}

// One tile of one sweep along AX: Uin -> Uout.  Phases over the tile (each
// a pass of the CTA's threads over its items, separated by barriers):
//   1. load + primitive recovery of the tile cells with a halo of two,
//   2. van Leer reconstruction + MUSCL-Hancock half step (face states),
//   3. Riemann problem at each face,
//   4. conservative update with the non-conservative terms, store.
// (ta, tw, rr): tile along AX, across it, and the index along the remaining
// axis; smem: SH::smem bytes; ok1, ok2: SH::N1, SH::N2 flags.  first = false:
// the tile follows tile ta - 1 of the same CTA, whose last four recovered
// cells, last two half-stepped cells and last face are already in place
// (carried), so each phase computes only the tile's new items.  carry: move
// those records to the front for tile ta + 1 at the end.  All threads of the
// CTA call it together.
//
// Still tiles: when every cell of the halo-extended tile holds one still
// state (same_still against the tile's first cell), the sweep leaves the
// tile's cells as they are; they are copied to Uout and nothing is
// computed.  Returns false then (no records to carry), true otherwise.
//
// TM = 1 (k_sweep_col_tma): the tile's new in-grid cells come from the
// boxes TMA copied (sc), whose copy was issued before the call; the copy of
// the tile sc names next is issued here (after phase 3, or at once for a
// still tile).  A wait that gives up reports MM_ETIMEOUT and clears sc->ok;
// the call then returns false and the CTA stops.
template <class P, int DIM, int NMAT, int NH, int AX, int V, int TM = 0>
__device__ __forceinline__ bool sweep_tile(const KArgs& a, int ta, int tw, int rr, bool first,
                                           bool carry, unsigned char* smem, unsigned char* ok1,
                                           unsigned char* ok2, ColStage* sc = nullptr) {
  typedef typename P::R R;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  typedef SweepShape<P, DIM, NMAT, NH, AX, V> SH;
  typedef typename P::X XT;
  constexpr int NF = L::NF, NX = SH::NX, TL = SH::TL, TW = SH::TW, NT = SH::NT;
  constexpr int C1 = SH::C1, C2 = SH::C2, C3 = SH::C3, NR = SH::NR;
  constexpr int N1 = SH::N1, N2 = SH::N2, N3 = SH::N3, N4 = SH::N4;
  constexpr int TD = (AX == 0) ? 1 : 0;
  XT* x1 = reinterpret_cast<XT*>(smem);  // N1 * NX
  XT* x2 = x1 + N1 * NX;                  // 2 * N2 * NX
  XT* x3 = x2 + 2 * N2 * NX;              // NR * N3 * NX
  R* r1 = reinterpret_cast<R*>(x3 + NR * N3 * NX);
  R* r2 = r1 + N1 * C1;
  R* r3 = r2 + 2 * N2 * C2;

  const int na = a.n[AX], ntw = a.n[TD];
  const int a0 = ta * TL, w0 = tw * TW;
  const long long step = a.info->steps;
  const R lam = R(a.info->lam[AX]);  // dt / dx_AX of the step

  // 0. still tile?  The reference is the tile's first cell (read by every
  // thread, one broadcast); each thread tests its cells, velocity first.
  {
    R cr[NF];
    XT cxr[NX];
    double er;
    load_cell<P, DIM, NMAT, NH, AX>(a, a0 - 2, w0, rr, cr, cxr, &er);
    bool still = true;
#pragma unroll
    for (int k = 0; k < DIM; ++k) still = still && cr[L::oMOM + k] == R(0);
    if (still) {
      for (int it0 = threadIdx.x; it0 < (TL + 4) * TW && still; it0 += NT) {
        int p, w;
        SH::pos(it0, TL + 4, p, w);
        const int gi = a0 - 2 + p;
        if (w0 + w < ntw && gi >= -2 && gi < na + 2) {
          R c[NF];
          XT cx[NX];
          double eE;
          load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
          still = same_still<P, DIM, NMAT, NH>(c, cx, eE, cr, cxr, er);
        }
      }
    }
    if (__syncthreads_and(still)) {
      if constexpr (TM) {
        // the staged boxes are not needed; the next tile's copy reuses them
        const bool got = mbar_wait(sc->bar, sc->parity);
        sc->parity ^= 1u;
        if (__syncthreads_or(!got)) {
          if (threadIdx.x == 0) report(a.err, ST_ETIMEOUT, cell_index(a, w0, 0, 0), step);
          sc->ok = false;
          return false;
        }
        if (sc->next && threadIdx.x == 0)
          stage_issue<P, DIM, NMAT, NH, AX>(*sc, sc->nta, sc->nw0, sc->nrr);
      }
      for (int it = threadIdx.x; it < N4; it += NT) {
        int p4, w;
        SH::pos(it, TL, p4, w);
        const int gi = a0 + p4;
        if (w0 + w < ntw && gi < na) {
          R c[NF];
          XT cx[NX];
          double eE;
          const long long idx = load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
          store_cell<P, DIM, NMAT, NH>(a, idx, c, cx, eE);
        }
      }
      return false;
    }
  }

  // 1. primitive recovery of every tile cell, halo of two included
  // (positions 0..3 carried when the tile follows one of the same CTA)
  const int s1 = first ? 0 : 4;
  if constexpr (TM) {
    const bool got = mbar_wait(sc->bar, sc->parity);
    sc->parity ^= 1u;
    if (__syncthreads_or(!got)) {
      if (threadIdx.x == 0) report(a.err, ST_ETIMEOUT, cell_index(a, w0, 0, 0), step);
      sc->ok = false;
      return false;
    }
  }
  for (int it0 = threadIdx.x; it0 < (TL + 4 - s1) * TW; it0 += NT) {
    int p, w;
    SH::pos(it0, TL + 4 - s1, p, w);
    p += s1;
    const int it = SH::idx(p, w, TL + 4);
    const int gi = a0 - 2 + p;
    unsigned char okv = 0;
    if (w0 + w < ntw && gi >= -2 && gi < na + 2) {
      R c[NF];
      XT cx[NX];
      double eE;
      long long idx = 0;
      bool staged = false;
      if constexpr (TM) {
        typedef StageShape<P, DIM, NMAT, NH, AX> CS;
        if (p >= 4 && gi < na) {
          int co[3];
          co[AX] = gi;
          co[TD] = w0 + w;
          co[3 - AX - TD] = rr;
          idx = cell_index(a, co[0], co[1], co[2]);
          stage_at<P, DIM, NMAT, NH, AX>(smem + sc->off, CS::pos(p, w), c, cx, &eE);
          staged = true;
        }
      }
      if (!staged) idx = load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
      R* rec = r1 + it * C1;
      Aux<R> ax;
      if (PH::template u2w<AX>(a, c, cx, rec, x1 + it * NX, ax, &eE)) {
        put_aux<P>(rec + NF, ax);
        okv = 1;
      } else {
        report(a.err, ST_ENONFINITE, idx, step);
        okv = 2;
      }
    }
    ok1[it] = okv;
  }
  __syncthreads();

  // 2. van Leer reconstruction and MUSCL-Hancock half step on cells -1..TL
  // (items 0, 1 carried)
  const int s2 = first ? 0 : 2;
  for (int it0 = threadIdx.x; it0 < (TL + 2 - s2) * TW; it0 += NT) {
    int p2, w;
    SH::pos(it0, TL + 2 - s2, p2, w);
    p2 += s2;
    const int it = SH::idx(p2, w, TL + 2);
    const int gi = a0 - 1 + p2;
    const int im = SH::idx(p2, w, TL + 4), ic = SH::idx(p2 + 1, w, TL + 4),
              ip = SH::idx(p2 + 2, w, TL + 4);
    unsigned char okv = 0;
    if (w0 + w < ntw && gi >= -1 && gi <= na && ok1[im] == 1 && ok1[ic] == 1 && ok1[ip] == 1) {
      const R* wm = r1 + im * C1;
      const R* wc = r1 + ic * C1;
      const R* wp = r1 + ip * C1;
      const XT* xm = x1 + im * NX;
      const XT* xc = x1 + ic * NX;
      const XT* xp = x1 + ip * NX;
      R uc[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) uc[k] = k < DIM ? wc[L::oMOM + k] : R(0);
      R sl[NF];
      XT slx[NX];
      bool flat = true;
#pragma unroll
      for (int k = 0; k < NF; ++k) {
        sl[k] = van_leer(wc[k] - wm[k], wp[k] - wc[k]);
        if (k < L::oX) flat = flat && sl[k] == R(0);
      }
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        slx[k] = van_leer(xc[k] - xm[k], xp[k] - xc[k]);
        flat = flat && slx[k] == XT(0);
      }
      // face states: slot 2 it is the left face (w - slope/2), 2 it + 1 the right
      R* const q0 = r2 + (2 * it) * C2;
      XT* const qx0 = x2 + (2 * it) * NX;
      bool done = false;
      if (P::split && flat) {
        // Split path: with every slope but those of X zero, both face states
        // equal the cell state except in X, and the half step changes only X
        // (X enters no closure): X_L,R += lam/2 (X_L - X_R) u_d.
        R c[NF];
        XT cx[NX];
        double eE;
        load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
        Aux<R> xa;
        get_aux<P>(wc + NF, xa);
#pragma unroll
        for (int k = 0; k < 3; ++k) xa.u[k] = uc[k];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          R* q = q0 + s * C2;
#pragma unroll
          for (int k = 0; k < NF; ++k) q[k] = c[k];
#pragma unroll
          for (int k = 0; k < DIM; ++k) {
            const R inc = R(0.5) * lam * ((wc[L::oX + k] - R(0.5) * sl[L::oX + k]) -
                                          (wc[L::oX + k] + R(0.5) * sl[L::oX + k])) * uc[AX];
            q[L::oX + k] = (s == 0 ? wc[L::oX + k] - R(0.5) * sl[L::oX + k]
                                   : wc[L::oX + k] + R(0.5) * sl[L::oX + k]) + inc;
          }
          put_aux<P>(q + NF, xa);
#pragma unroll
          for (int k = 0; k < NX; ++k) qx0[s * NX + k] = cx[k];
        }
        done = true;
      } else {
        // MUSCL-Hancock: one pass per face state (one code site for the
        // state conversions), accumulating F_L - F_R and the jumps the
        // non-conservative terms need; the half-step states go to shared memory.
        bool good = true;
        R dfl[NF], dF[3], du = R(0);
        XT dfx[NX];
#pragma unroll
        for (int k = 0; k < NF; ++k) dfl[k] = R(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) dfx[k] = XT(0);
#pragma unroll
        for (int j = 0; j < 3; ++j) dF[j] = R(0);
#pragma unroll 1
        for (int s = 0; s < 2; ++s) {
          const R hs = s == 0 ? R(-0.5) : R(0.5);
          const R sg = s == 0 ? R(1) : R(-1);
          R wv[NF], cs[NF], f[NF], row[3];
          XT wxv[NX], cxs[NX], fx[NX];
#pragma unroll
          for (int k = 0; k < NF; ++k) wv[k] = wc[k] + hs * sl[k];
#pragma unroll
          for (int k = 0; k < NX; ++k) wxv[k] = xc[k] + XT(hs) * slx[k];
          if constexpr (NR == 2) {
            // the limited slope keeps a face value between the neighbours'
            // up to rounding: a void fraction a rounding below zero is zero
#pragma unroll
            for (int l = 0; l < PH::NPX; ++l)
              if (l == a.void_l && wxv[1 + l] < XT(0)) wxv[1 + l] = XT(0);
          }
          Aux<R> xs;
          if (!PH::template w2u<AX>(a, wv, wxv, cs, cxs, xs)) {
            good = false;
            break;
          }
          PH::template flux<AX>(cs, cxs, xs, f, fx);
          PH::template frow<AX>(cs, row);
#pragma unroll
          for (int k = 0; k < NF; ++k) dfl[k] += sg * f[k];
#pragma unroll
          for (int k = 0; k < NX; ++k) dfx[k] += XT(sg) * fx[k];
#pragma unroll
          for (int j = 0; j < 3; ++j) dF[j] -= sg * row[j];
          du -= sg * xs.u[AX];
          R* q = q0 + s * C2;
#pragma unroll
          for (int k = 0; k < NF; ++k) q[k] = cs[k];
#pragma unroll
          for (int k = 0; k < NX; ++k) qx0[s * NX + k] = cxs[k];
        }
        if (good) {
          R nc[NF];
          XT ncx[NX];
          PH::template noncons<AX>(wc, xc, uc, du, dF, nc, ncx);
#pragma unroll 1
          for (int s = 0; s < 2; ++s) {
            R* q = q0 + s * C2;
            XT* qx = qx0 + s * NX;
            R cs[NF], tmp[NF];
            XT cxs[NX], tmpx[NX];
#pragma unroll
            for (int k = 0; k < NF; ++k) cs[k] = q[k] + R(0.5) * lam * (dfl[k] + nc[k]);
#pragma unroll
            for (int k = 0; k < NX; ++k) cxs[k] = qx[k] + XT(0.5) * XT(lam) * (dfx[k] + ncx[k]);
            if constexpr (NR == 2) {
              // a void fraction a rounding below zero is zero, as in the update
#pragma unroll
              for (int l = 0; l < PH::NPX; ++l)
                if (l == a.void_l && cxs[1 + l] < XT(0)) cxs[1 + l] = XT(0);
            }
            Aux<R> xs;
            if (!PH::template u2w<AX>(a, cs, cxs, tmp, tmpx, xs)) {
              good = false;
              break;
            }
            // A half step changes ln(rho_l) by (dt/2)|du/dx| <= cfl <= 1 (dt <=
            // cfl dx / S, |u_R - u_L| <= 2 S).  A larger change of a phase
            // density comes from the near-cancelling increments of phi_l and
            // phi_l rho_l at a trace fraction, and the face falls back.
            const R hs = s == 0 ? R(-0.5) : R(0.5);
            const R eb = R(2.718281828459045);
#pragma unroll
            for (int l = 0; l < NMAT; ++l) {
              const R r0 = wc[L::oARHO + l] + hs * sl[L::oARHO + l];
              const R r1 = tmp[L::oARHO + l];
              good = good && r1 <= eb * r0 && r0 <= eb * r1;
            }
            if (!good) break;
#pragma unroll
            for (int k = 0; k < NF; ++k) q[k] = cs[k];
#pragma unroll
            for (int k = 0; k < NX; ++k) qx[k] = cxs[k];
            put_aux<P>(q + NF, xs);
          }
        }
        done = good;
      }
      if (!done) {
        // first order: both faces take the cell average
        R c[NF];
        XT cx[NX];
        double eE;
        load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
        Aux<R> xa;
        get_aux<P>(wc + NF, xa);
#pragma unroll
        for (int k = 0; k < 3; ++k) xa.u[k] = uc[k];
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
          for (int k = 0; k < NF; ++k) q0[s * C2 + k] = c[k];
          put_aux<P>(q0 + s * C2 + NF, xa);
#pragma unroll
          for (int k = 0; k < NX; ++k) qx0[s * NX + k] = cx[k];
        }
      }
      okv = 1;
    }
    ok2[it] = okv;
  }
  __syncthreads();

  // 3. Riemann problem at faces -1/2 .. TL-1/2 (face 0 carried)
  const int s3 = first ? 0 : 1;
  for (int it0 = threadIdx.x; it0 < (TL + 1 - s3) * TW; it0 += NT) {
    int f, w;
    SH::pos(it0, TL + 1 - s3, f, w);
    f += s3;
    const int it = SH::idx(f, w, TL + 1);
    const int il = SH::idx(f, w, TL + 2), ir = SH::idx(f + 1, w, TL + 2);
    if (ok2[il] == 1 && ok2[ir] == 1) {
      const R* ql = r2 + (2 * il + 1) * C2;  // right face state of the left cell
      const R* qr = r2 + (2 * ir) * C2;      // left face state of the right cell
      Aux<R> xl, xr;
      get_aux<P>(ql + NF, xl);
      get_aux<P>(qr + NF, xr);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        xl.u[k] = k < DIM ? ql[L::oMOM + k] / xl.rho : R(0);
        xr.u[k] = k < DIM ? qr[L::oMOM + k] / xr.rho : R(0);
      }
      R fo[NF], row[3], uf;
      XT fox[NX];
      if constexpr (NR == 2) {
        // the record the right cell takes goes to slot 1 first, then the
        // left cell's to slot 0
        R* q3 = r3 + (2 * it + 1) * C3;
        R uf1, row1[3];
        PH::template riemann2<AX>(a, ql, x2 + (2 * il + 1) * NX, xl, qr, x2 + (2 * ir) * NX, xr,
                                  fo, fox, uf, row, q3, x3 + (2 * it + 1) * NX, uf1, row1);
        q3[NF] = uf1;
        q3[NF + 1] = row1[0];
        q3[NF + 2] = row1[1];
        q3[NF + 3] = row1[2];
      } else {
        PH::template riemann<AX>(ql, x2 + (2 * il + 1) * NX, xl, qr, x2 + (2 * ir) * NX, xr, fo,
                                 fox, uf, row);
      }
      R* q3 = r3 + NR * it * C3;
#pragma unroll
      for (int k = 0; k < NF; ++k) q3[k] = fo[k];
      q3[NF] = uf;
      q3[NF + 1] = row[0];
      q3[NF + 2] = row[1];
      q3[NF + 3] = row[2];
#pragma unroll
      for (int k = 0; k < NX; ++k) x3[NR * it * NX + k] = fox[k];
    }
  }
  __syncthreads();

  // the next tile's boxes are copied while this one is updated
  if constexpr (TM)
    if (sc->next && threadIdx.x == 0)
      stage_issue<P, DIM, NMAT, NH, AX>(*sc, sc->nta, sc->nw0, sc->nrr);

  // 4. conservative update with the non-conservative terms
  for (int it = threadIdx.x; it < N4; it += NT) {
    int p4, w;
    SH::pos(it, TL, p4, w);
    const int gi = a0 + p4;
    if (w0 + w < ntw && gi < na) {
      const int fl = SH::idx(p4, w, TL + 1), fr = SH::idx(p4 + 1, w, TL + 1);
      const int ic = SH::idx(p4 + 2, w, TL + 4);
      if (ok1[ic] != 1) continue;
      R c[NF];
      XT cx[NX];
      double eE;
      const long long idx = load_cell<P, DIM, NMAT, NH, AX>(a, gi, w0 + w, rr, c, cx, &eE);
      const R* wc = r1 + ic * C1;
      const XT* xc = x1 + ic * NX;
      // the left face's record as a right cell takes it, the right face's as
      // a left cell does (one record each where the void cannot open)
      const R* ql = r3 + (NR * fl + NR - 1) * C3;
      const R* qr = r3 + NR * fr * C3;
      const XT* xql = x3 + (NR * fl + NR - 1) * NX;
      const XT* xqr = x3 + NR * fr * NX;
      R uc[3], dF[3], nc[NF];
      XT ncx[NX];
#pragma unroll
      for (int k = 0; k < 3; ++k) uc[k] = k < DIM ? wc[L::oMOM + k] : R(0);
#pragma unroll
      for (int j = 0; j < 3; ++j) dF[j] = qr[NF + 1 + j] - ql[NF + 1 + j];
      PH::template noncons<AX>(wc, xc, uc, qr[NF] - ql[NF], dF, nc, ncx);
#pragma unroll
      for (int k = 0; k < NF; ++k) c[k] = c[k] + lam * ((ql[k] - qr[k]) + nc[k]);
#pragma unroll
      for (int k = 1; k < NX; ++k) cx[k] = cx[k] + XT(lam) * ((xql[k] - xqr[k]) + ncx[k]);
      if constexpr (NR == 2) {
        // the void fraction is created only where the void opens; its
        // transport of traces can leave it a rounding below zero: zero
#pragma unroll
        for (int l = 0; l < PH::NPX; ++l)
          if (l == a.void_l && cx[1 + l] < XT(0)) cx[1 + l] = XT(0);
      }
      // total energy updated in FP64 (the stored state)
      // (the face fluxes differenced in FP64 telescope exactly over the
      // cells, which keeps the total energy conserved to FP64 rounding)
      eE = eE + double(lam) * ((double(xql[0]) - double(xqr[0])) + double(ncx[0]));
      store_cell<P, DIM, NMAT, NH>(a, idx, c, cx, eE);
    }
  }
  if (carry) {
    // the next tile's first recovered cells (4), half-stepped cells (2) and
    // face (1) are this tile's last ones
    __syncthreads();
    for (int it0 = threadIdx.x; it0 < 7 * TW; it0 += NT) {
      const int w = it0 % TW, kind = it0 / TW;
      if (kind < 4) {
        const int d = SH::idx(kind, w, TL + 4), sidx = SH::idx(kind + TL, w, TL + 4);
        for (int k = 0; k < C1; ++k) r1[d * C1 + k] = r1[sidx * C1 + k];
        for (int k = 0; k < NX; ++k) x1[d * NX + k] = x1[sidx * NX + k];
        ok1[d] = ok1[sidx];
      } else if (kind < 6) {
        const int j = kind - 4;
        const int d = SH::idx(j, w, TL + 2), sidx = SH::idx(j + TL, w, TL + 2);
        for (int k = 0; k < 2 * C2; ++k) r2[2 * d * C2 + k] = r2[2 * sidx * C2 + k];
        for (int k = 0; k < 2 * NX; ++k) x2[2 * d * NX + k] = x2[2 * sidx * NX + k];
        ok2[d] = ok2[sidx];
      } else {
        const int d = SH::idx(0, w, TL + 1), sidx = SH::idx(TL, w, TL + 1);
        for (int k = 0; k < NR * C3; ++k) r3[NR * d * C3 + k] = r3[NR * sidx * C3 + k];
        for (int k = 0; k < NR * NX; ++k) x3[NR * d * NX + k] = x3[NR * sidx * NX + k];
      }
    }
    __syncthreads();
  }
  return true;
}

// Tile coordinates of tile index b of a sweep (along AX fastest, then
// across, then the remaining axis).
template <int AX, int TL, int TW>
__device__ __forceinline__ void tile_of(const KArgs& a, long long b, int& ta, int& tw, int& rr) {
  constexpr int TD = (AX == 0) ? 1 : 0;
  const int nta = (a.n[AX] + TL - 1) / TL, ntt = (a.n[TD] + TW - 1) / TW;
  ta = int(b % nta);
  b /= nta;
  tw = int(b % ntt);
  rr = int(b / ntt);
}

// One CTA per tile of one grid.
template <class P, int DIM, int NMAT, int NH, int AX>
__global__ void __launch_bounds__(Tile<P, DIM, AX>::NT) k_sweep(KArgs a) {
  typedef SweepShape<P, DIM, NMAT, NH, AX, 0> SH;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned char ok1[SH::N1], ok2[SH::N2];
  int ta, tw, rr;
  tile_of<AX, SH::TL, SH::TW>(a, blockIdx.x, ta, tw, rr);
  sweep_tile<P, DIM, NMAT, NH, AX, 0>(a, ta, tw, rr, true, false, smem, ok1, ok2);
}

// One CTA per chunk of K consecutive tiles along the sweep axis (large
// grids): each tile after the chunk's first reuses the overlap its
// predecessor recovered and half-stepped, so no halo cell is computed twice
// inside a chunk.  Blocks: chunk fastest, then across, then the remaining axis.
template <class P, int DIM, int NMAT, int NH, int AX>
__global__ void __launch_bounds__(Tile<P, DIM, AX>::NT) k_sweep_col(KArgs a, int K) {
  typedef SweepShape<P, DIM, NMAT, NH, AX, 0> SH;
  constexpr int TD = (AX == 0) ? 1 : 0;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned char ok1[SH::N1], ok2[SH::N2];
  const int nta = (a.n[AX] + SH::TL - 1) / SH::TL, ntt = (a.n[TD] + SH::TW - 1) / SH::TW;
  const int nch = (nta + K - 1) / K;
  long long b = blockIdx.x;
  const int ch = int(b % nch);
  b /= nch;
  const int tw = int(b % ntt), rr = int(b / ntt);
  const int t0 = ch * K, t1 = t0 + K < nta ? t0 + K : nta;
  // a tile after a still one starts afresh (nothing was carried)
  bool first = true;
  for (int ta = t0; ta < t1; ++ta)
    first = !sweep_tile<P, DIM, NMAT, NH, AX, 0>(a, ta, tw, rr, first, ta + 1 < t1, smem, ok1,
                                                 ok2);
}

// Setup of the staged sweep kernel: the map's alignment (a map the
// TMA unit reads must sit on a 64-byte boundary; parameters keep the type's
// 128-byte alignment, checked, not assumed), the mbarrier, the boxes'
// place.  False (error reported) if the map is misaligned.
template <class P, int DIM, int NMAT, int NH, int AX>
__device__ __forceinline__ bool stage_setup(const KArgs& a, const ColTma& tm, ColStage& sc,
                                            unsigned char* smem, unsigned long long* bar) {
  if (reinterpret_cast<uintptr_t>(&tm) & 63) {
    if (threadIdx.x == 0) report(a.err, ST_ECUDA, blockIdx.x, a.info->steps);
    return false;
  }
  sc.tm = &tm;
  sc.err = a.err;
  sc.bar = smem_u32(bar);
  sc.parity = 0;
  const uint32_t base = smem_u32(smem);
  sc.dst = (base + uint32_t(StageShape<P, DIM, NMAT, NH, AX>::lo) + 127u) & ~127u;
  sc.off = sc.dst - base;
  sc.ok = true;
  sc.next = false;
  if (threadIdx.x == 0) mbar_init(sc.bar);
  __syncthreads();
  return true;
}

// k_sweep_col with the tiles' new cells staged by TMA (3D FP32-split y and
// z sweeps; maps of the launch's Uin and Ein in tm): the copy of a CTA's
// first tile is issued before its loop, each later one during the update
// of the tile before it, so a tile's loads overlap the previous tile's work.
// Registers bounded for two 192-thread CTAs per SM, as many as the shared
// memory of the 12 x 16 tiles holds (unbounded, ptxas took about 210).
template <class P, int DIM, int NMAT, int NH, int AX>
__global__ void __launch_bounds__(Tile<P, DIM, AX>::NT, 2)
    k_sweep_col_tma(const __grid_constant__ KArgs a, int K, const __grid_constant__ ColTma tm) {
  typedef SweepShape<P, DIM, NMAT, NH, AX, 0> SH;
  constexpr int TD = 0;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned char ok1[SH::N1], ok2[SH::N2];
  __shared__ __align__(8) unsigned long long bar;
  const int nta = (a.n[AX] + SH::TL - 1) / SH::TL, ntt = (a.n[TD] + SH::TW - 1) / SH::TW;
  const int nch = (nta + K - 1) / K;
  long long b = blockIdx.x;
  const int ch = int(b % nch);
  b /= nch;
  const int tw = int(b % ntt), rr = int(b / ntt);
  const int t0 = ch * K, t1 = t0 + K < nta ? t0 + K : nta;
  ColStage sc;
  if (!stage_setup<P, DIM, NMAT, NH, AX>(a, tm, sc, smem, &bar)) return;
  if (threadIdx.x == 0) stage_issue<P, DIM, NMAT, NH, AX>(sc, t0, tw * SH::TW, rr);
  sc.nw0 = tw * SH::TW;
  sc.nrr = rr;
  bool first = true;
  for (int ta = t0; ta < t1 && sc.ok; ++ta) {
    sc.next = ta + 1 < t1;
    sc.nta = ta + 1;
    first = !sweep_tile<P, DIM, NMAT, NH, AX, 0, 1>(a, ta, tw, rr, first, sc.next, smem, ok1,
                                                    ok2, &sc);
  }
}

// ------------------------------------------------------------ batches ----
// Work of a batched launch: member m owns units [start[m], start[m+1]) of
// the concatenated list; persistent CTAs take units from a counter.
__device__ __forceinline__ int batch_member(const BatchK& bk, long long u) {
  int lo = 0, hi = bk.M - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (bk.start[mid] <= u) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Next unit for the CTA (uniform); ka <- the arguments of its member,
// copied only when the member differs from the previous unit's (s_m, -1 at
// the start): a CTA's units are mostly of one member.  GRAB units are taken
// from the counter at a time (s_unit the next one, s_end the end of the
// taken range; both -1 at the start), which spreads the atomic's latency
// over them.
template <int GRAB = 1>
__device__ __forceinline__ bool batch_next(const BatchK& bk, KArgs& ka, long long& unit,
                                           long long& s_unit, long long& s_end, int& s_m) {
  __syncthreads();  // the previous unit is finished by every thread
  if (threadIdx.x == 0) {
    if (s_unit < 0 || s_unit >= s_end) {
      s_unit = bk.base + (long long)atomicAdd(bk.counter, (unsigned long long)GRAB);
      s_end = s_unit + GRAB;
    }
  }
  __syncthreads();
  const long long u = s_unit;
  if (u >= bk.total) return false;
  const int m = batch_member(bk, u);
  unit = u - bk.start[m];
  __syncthreads();  // every thread has read s_unit
  if (threadIdx.x == 0) s_unit = u + 1;
  if (m != s_m) {
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(bk.args + m);
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(&ka);
    for (int i = threadIdx.x; i < int(sizeof(KArgs) / 8); i += blockDim.x) dst[i] = src[i];
    __syncthreads();  // every thread has read s_m before it changes
    if (threadIdx.x == 0) s_m = m;
    __syncthreads();
  }
  return true;
}

// One sweep along AX over the tiles of every member of a batch.
template <class P, int DIM, int NMAT, int NH, int AX, int V>
__global__ void __launch_bounds__(Tile<P, DIM, AX, V>::NT) k_sweep_batch(BatchK bk) {
  typedef SweepShape<P, DIM, NMAT, NH, AX, V> SH;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ unsigned char ok1[SH::N1], ok2[SH::N2];
  __shared__ KArgs ka;
  __shared__ long long s_unit, s_end;
  __shared__ int s_m;
  if (threadIdx.x == 0) {
    s_m = -1;
    s_unit = -1;
    s_end = -1;
  }
  long long t;
  while (batch_next<4>(bk, ka, t, s_unit, s_end, s_m)) {
    int ta, tw, rr;
    tile_of<AX, SH::TL, SH::TW>(ka, t, ta, tw, rr);
    sweep_tile<P, DIM, NMAT, NH, AX, V>(ka, ta, tw, rr, true, false, smem, ok1, ok2);
  }
}

// ------------------------------------------------------------- sources ----
// Perturbation lookup phi(x) = phi0(X): multilinear, 1 outside the lattice.
// T = double (FP64 path) or float (FP32-split).
template <int DIM, class T>
__device__ __forceinline__ T lookup(const KArgs& a, const T X[3]) {
  if (!a.phi0) return T(1);
  // lattice of at most 2^31 - 1 points (checked on the host): int indices
  int i0[3] = {0, 0, 0};
  T w[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int k = 0; k < DIM; ++k) {
    const T lo = sizeof(T) == 4 ? T(a.plof[k]) : T(a.plo[k]);
    const T h = sizeof(T) == 4 ? T(a.phf[k]) : T(a.ph[k]);
    const T s = (X[k] - lo) / h;
    if (!(s >= T(0)) || !(s <= T(a.pn[k] - 1))) return T(1);
    int i = int(floor(s));
    if (i > a.pn[k] - 2) i = a.pn[k] - 2;
    i0[k] = i;
    w[k] = s - T(i);
  }
  T v = T(0);
#pragma unroll
  for (int c = 0; c < (1 << DIM); ++c) {
    T wt = T(1);
    int idx = 0, str = 1;
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const int bit = (c >> k) & 1;
      wt *= bit ? w[k] : T(1) - w[k];
      idx += (i0[k] + bit) * str;
      str *= a.pn[k];
    }
    v += wt * T(__ldg(a.phi0 + idx));
  }
  return v;
}

// Mixture yield stress sum_l phi_l phi (1-D_l) sigma_Y,l (Johnson-Cook, rate
// factor floored at 1, zero at critical damage D >= D_cut) and its
// derivative in dl.
// The Johnson-Cook powers and logarithm are evaluated in T (FP64 on the FP64
// path, FP32 on the split path); the sums are FP64.
template <int NMAT, class T>
__device__ __forceinline__ double yield_mix(const KArgs& a, const double* phi, const double* eps,
                                            const double* D, double phihat, double dt, double dl,
                                            double* dY) {
  double Y = 0.0, dYs = 0.0;
#pragma unroll
  for (int l = 0; l < NMAT; ++l) {
    const MatK& m = a.mat[l];
    if (m.plasticity != 1) continue;
    // critical damage at the threshold in the path's precision
    const double dcut = sizeof(T) == sizeof(float) ? double(a.matf[l].D_cut) : m.D_cut;
    if (m.damage != 0 && D[l] >= dcut) continue;
    const double psi = m.damage != 0 ? 1.0 - D[l] : 1.0;
    const double e = (eps[l] > 0.0 ? eps[l] : 0.0) + dl;
    double hard = m.c1, dhard = 0.0;
    if (m.c2 != 0.0) {
      hard += m.c2 * double(mpow(T(e), T(m.n_hard)));
      if (e > 0.0) dhard = m.c2 * m.n_hard * double(mpow(T(e), T(m.n_hard - 1.0)));
    }
    double Rr = 1.0, dR = 0.0;
    if (m.c3 != 0.0 && dl > 0.0) {
      const double r = 1.0 + m.c3 * double(mlog(T(dl / (dt * m.edot0))));
      if (r > 1.0) {
        Rr = r;
        dR = m.c3 / dl;
      }
    }
    const double wgt = phi[l] * phihat * psi;
    Y += wgt * hard * Rr;
    dYs += wgt * (dhard * Rr + hard * dR);
  }
  if (dY) *dY = dYs;
  return Y;
}

// The same yield stress and derivative evaluated wholly in FP32 (split
// path): the Newton iterate and residual stay FP64, the function values and
// the step quotient are FP32.
template <int NMAT>
__device__ __forceinline__ float yield_mix_f32(const KArgs& a, const float* phi, const float* eps,
                                               const float* D, float phihat, float inv_dt,
                                               float dl, float* dY) {
  float Y = 0.f, dYs = 0.f;
#pragma unroll
  for (int l = 0; l < NMAT; ++l) {
    const MatKf& m = a.matf[l];
    if (m.plasticity != 1) continue;
    if (m.damage != 0 && D[l] >= m.D_cut) continue;
    const float psi = m.damage != 0 ? 1.f - D[l] : 1.f;
    const float e = (eps[l] > 0.f ? eps[l] : 0.f) + dl;
    float hard = m.c1, dhard = 0.f;
    if (m.c2 != 0.f) {
      const float en = mpow(e, m.n_hard);
      hard += m.c2 * en;
      if (e > 0.f) dhard = m.c2n * en / e;
    }
    float Rr = 1.f, dR = 0.f;
    if (m.c3 != 0.f && dl > 0.f) {
      const float r = 1.f + m.c3 * __logf(dl * inv_dt / m.edot0);
      if (r > 1.f) {
        Rr = r;
        dR = m.c3 / dl;
      }
    }
    const float wgt = phi[l] * phihat * psi;
    Y += wgt * hard * Rr;
    dYs += wgt * (dhard * Rr + hard * dR);
  }
  *dY = dYs;
  return Y;
}

// Triaxiality-dependent threshold strain; eps_c^(2n), eps_t^(2n) precomputed.
template <class T, class M>
__device__ __forceinline__ T eps_thresh(const M& m, T Rt) {
  const T n = T(m.n_hard), et = T(m.eps_t), ec = T(m.eps_c);
  const T num = T(m.bon_ec2n) - T(m.bon_et2n);
  const T den = mpow(ec, T(2) * n / Rt) - mpow(et, T(2) * n / Rt);
  return mpow(et, T(1) / Rt) / mpow(Rt, T(1) / n) * mpow(num / den, T(1) / (T(2) * n));
}

template <class T, class M>
__device__ __forceinline__ T dmg_rate(const M& m, T D, T eps, T ed, T Rt, T th, bool tension) {
  if (m.damage == 2) return T(m.Ddot0) * (T(1) - D) * ed;
  if (!tension || !(eps > th)) return T(0);
  if (D >= T(m.D_crit)) return T(0);
  const T aD = T(m.alpha_D), Dc = T(m.D_crit);
  return T(m.bon_k) * Rt * mpow(Dc - D, (aD - T(1)) / aD) * ed / eps;
}

// RK4 over the step of the damage rate with eps_p(t) linear in t (the
// plastic increment deps over dt), p and sigma_eq held at the returned
// state; clamped to [0, D_crit].  Bonora: zero unless p < 0 (checked first).
template <class T, class M>
__device__ __forceinline__ T damage_rk4(const M& m, T D, T eps0, T deps, T dt, T p, T seq,
                                        T rho) {
  if (m.damage == 0 || !(deps > T(0))) return D;
  T Rt = T(1), th = T(0);
  const bool tension = p < T(0);
  if (m.damage == 1) {
    if (!(seq > T(0))) return D;
    if (!tension) return D < T(0) ? T(0) : (D > T(m.D_crit) ? T(m.D_crit) : D);
    const T x = p / seq;
    Rt = T(2) / T(3) * (T(1) + T(m.poisson)) +
         T(3) * (T(1) - T(2) * T(m.poisson)) * (T(m.rho0) / rho) * (x * x);
    th = eps_thresh<T, M>(m, Rt);
  }
  const T ed = deps / dt;
  const T k1 = dmg_rate<T, M>(m, D, eps0, ed, Rt, th, tension);
  const T k2 = dmg_rate<T, M>(m, D + T(0.5) * dt * k1, eps0 + T(0.5) * deps, ed, Rt, th, tension);
  const T k3 = dmg_rate<T, M>(m, D + T(0.5) * dt * k2, eps0 + T(0.5) * deps, ed, Rt, th, tension);
  const T k4 = dmg_rate<T, M>(m, D + dt * k3, eps0 + deps, ed, Rt, th, tension);
  T Dn = D + dt / T(6) * (k1 + T(2) * k2 + T(2) * k3 + k4);
  if (Dn < T(0)) Dn = T(0);
  if (Dn > T(m.D_crit)) Dn = T(m.D_crit);
  return Dn;
}

// The full source step of one cell: det Fbar = 1, the radial return to the
// perturbed yield stress (FP64 Newton) and RK4 damage, then the in-place
// store.  Out of line: in the split path only cells at or above yield come
// here, so the common elastic path of k_sources stays compact.
template <class P, int DIM, int NMAT, int NH>
__device__ __noinline__ void source_full(const KArgs& a, long long cell, typename P::R* c,
                                         const typename P::X* cx, double eE,
                                         const typename P::R* rho, const typename P::R* Dr,
                                         const typename P::R* phir, const typename P::R* Er,
                                         typename P::R phihat_r, typename P::R Gm_r,
                                         bool can_yield, double dt, long long step) {
  typedef typename P::R R;
  typedef typename P::X XT;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int NF = L::NF, NX = PH::NX;
  (void)NX;
  // the return and the damage take the fractions, strains and damage in FP64
  double phi[NMAT], eps[NMAT], Dm[NMAT];
#pragma unroll
  for (int l = 0; l < NMAT; ++l) {
    phi[l] = double(phir[l]);
    eps[l] = double(Er[l]);
    Dm[l] = double(Dr[l]);
  }
  const double phihat = double(phihat_r), Gm = double(Gm_r);
  // det Fbar = 1
  R X[9];
  PH::fullX(c, X);
  if (P::aform) {
    // A <- (I + A)/cbrt(det) - I with det - 1 expanded in A
    const R ed = (X[0] + X[4] + X[8]) +
                 (X[0] * X[4] - X[1] * X[3] + X[0] * X[8] - X[2] * X[6] + X[4] * X[8] -
                  X[5] * X[7]) +
                 (X[0] * (X[4] * X[8] - X[5] * X[7]) - X[1] * (X[3] * X[8] - X[5] * X[6]) +
                  X[2] * (X[3] * X[7] - X[4] * X[6]));
    const R cm1 = mexpm1(mlog1p(ed) / R(3));
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] = (X[k] - ((k % 4 == 0) ? cm1 : R(0))) / (R(1) + cm1);
  } else {
    const R det = X[0] * (X[4] * X[8] - X[5] * X[7]) - X[1] * (X[3] * X[8] - X[5] * X[6]) +
                  X[2] * (X[3] * X[7] - X[4] * X[6]);
    const R c3 = mcbrt(det);
#pragma unroll
    for (int k = 0; k < 9; ++k) X[k] /= c3;
  }
  // dev(H), |dev(H)|, and (for the return) either eigen-pairs or the
  // series form of exp((k-1) dev(H)) - I
  // (only a cell that can yield and carries shear needs them)
  const bool yieldable = can_yield && Gm > 0.0;
  R devH[9], h[3], V[9];
  R J2 = R(0);
  bool series = false;
  if (yieldable) {
    if constexpr (P::split) {
      // series form while the stretch is small (|dev(H)|_F <= 0.05), else
      // the eigen-pairs are taken below
      R dH[9], j2;
      if (hencky_fast(X, dH, j2) && j2 <= R(2.5e-3)) {
#pragma unroll
        for (int q = 0; q < 9; ++q) devH[q] = dH[q];
        J2 = j2;
        series = true;
      }
    }
    if (!series) {
      if (!hencky<P::aform>(X, devH, h, V)) {
        report(a.err, ST_ENONFINITE, cell, step);
        return;
      }
      J2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
    }
  }
  double dl = 0.0;
  R km1 = R(0);  // k - 1 of the return factor k = 1 - 3 G dl / sigma_eq
  if (yieldable) {
    // Split path: the equivalent stress, the bracket, the start and the
    // yield-function inputs come from FP32 quantities and are formed in FP32
    // (this part's FP64 pipe is narrow); the Newton iterate and residual
    // stay FP64.
    float phf[NMAT], epf[NMAT], Dmf[NMAT];
    float inv_dt = 0.f, strf = 0.f;
    double str;
    if constexpr (P::split) {
#pragma unroll
      for (int l = 0; l < NMAT; ++l) {
        phf[l] = phir[l];
        epf[l] = Er[l];
        Dmf[l] = Dr[l];
      }
      const float Jf = series ? sqrtf(J2) : sqrtf(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
      strf = 2.4494897f * Gm_r * Jf;  // sqrt(6) G |dev H|
      str = double(strf);
      inv_dt = 1.0f / float(dt);
    } else {
      const double J = series ? sqrt(double(J2))
                              : sqrt(double(h[0]) * double(h[0]) + double(h[1]) * double(h[1]) +
                                     double(h[2]) * double(h[2]));
      str = sqrt(6.0) * Gm * J;
    }
    float dYf0;
    const double Y0 =
        P::split ? double(yield_mix_f32<NMAT>(a, phf, epf, Dmf, float(phihat_r), inv_dt, 0.f, &dYf0))
                 : yield_mix<NMAT, R>(a, phi, eps, Dm, phihat, dt, 0.0, nullptr);
    if (str > Y0) {
      // stopping rule at the accuracy of the yield-stress evaluation
      const double gtol = P::split ? 1e-6 : 8.0 * 2.220446049250313e-16;
      const double xtol = P::split ? 1e-7 : 4.0 * 2.220446049250313e-16;
      double b0, x;
      if constexpr (P::split) {
        const float g3 = 3.0f * Gm_r;
        b0 = double(strf / g3);
        x = double((strf - float(Y0)) / g3);
      } else {
        b0 = str / (3.0 * Gm);
        x = (str - Y0) / (3.0 * Gm);
      }
      double lo = 0.0, hi = b0;
      bool conv = false;
      for (int it = 0; it < 200; ++it) {
        double dY = 0.0, Y;
        float dYf = 0.f;
        if (P::split) {
          Y = double(yield_mix_f32<NMAT>(a, phf, epf, Dmf, float(phihat_r), inv_dt, float(x), &dYf));
        } else {
          Y = yield_mix<NMAT, R>(a, phi, eps, Dm, phihat, dt, x, &dY);
        }
        const double g = str - 3.0 * Gm * x - Y;
        if (fabs(g) <= gtol * str) {
          conv = true;
          break;
        }
        if (g > 0.0) lo = x; else hi = x;
        double nx = P::split ? x - double(float(g) / (-3.0f * Gm_r - dYf))
                             : x - g / (-3.0 * Gm - dY);
        if (!(nx > lo && nx < hi)) nx = 0.5 * (lo + hi);
        if (fabs(nx - x) <= xtol * b0) {
          x = nx;
          conv = true;
          break;
        }
        x = nx;
      }
      if (!conv) {
        report(a.err, ST_ENOCONV, cell, step);
        return;
      }
      dl = x;
      // split path: k - 1 itself in FP32 (k rounded to FP32 would leave
      // k - 1 with a relative error of 6e-8 / |k - 1|)
      if constexpr (P::split)
        km1 = -(3.0f * Gm_r * float(dl)) / strf;
      else
        km1 = R((str - 3.0 * Gm * dl) / str) - R(1);
      // Fbar <- S Fbar, S = exp((k-1) dev(H)) (the rotation is kept); in A
      // form A <- (S - I)(I + A) + A
      R Sm[9], Xn[9];
      if (series) {
        R Y[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) Y[q] = km1 * devH[q];
        expm1_series(Y, Sm);
      } else {
        R m1[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) m1[q] = P::aform ? mexpm1(km1 * h[q]) : mexp(km1 * h[q]);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j)
            Sm[3 * i + j] = V[3 * i + 0] * m1[0] * V[3 * j + 0] + V[3 * i + 1] * m1[1] * V[3 * j + 1] +
                            V[3 * i + 2] * m1[2] * V[3 * j + 2];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const R sx = Sm[3 * i + 0] * X[0 + j] + Sm[3 * i + 1] * X[3 + j] + Sm[3 * i + 2] * X[6 + j];
          Xn[3 * i + j] = P::aform ? Sm[3 * i + j] + sx + X[3 * i + j] : sx;
        }
#pragma unroll
      for (int k2 = 0; k2 < 9; ++k2) X[k2] = Xn[k2];
    }
  }
#pragma unroll
  for (int k = 0; k < L::NFC; ++k) c[L::oF + k] = X[FC<DIM>::idx(k)];
  if (dl > 0.0) {
    R w2[NF];
    XT wx2[NX];
    Aux<R> as;
    // the recovery's mixture is that of the returned state (same fractions,
    // densities and damage, Fbar = X)
    typename PH::Mix mx;
    if (!PH::template u2w<0>(a, c, cx, w2, wx2, as, &eE, &mx)) {
      report(a.err, ST_ENONFINITE, cell, step);
      return;
    }
    R seq;
    if constexpr (P::split)
      seq = 2.4494897f * mx.Gm * sqrtf(mx.J2);
    else
      seq = R(sqrt(6.0) * double(mx.Gm) * sqrt(double(mx.J2)));
#pragma unroll
    for (int l = 0; l < NMAT; ++l) {
#pragma unroll
      for (int hh = 0; hh < NH; ++hh)
        if (a.hslot[l] == hh) {
          const R arho = c[L::oARHO + l];
          if constexpr (P::split) {
            const R Dn = damage_rk4<R>(matp<R>(a, l), Dr[l], Er[l], R(dl), R(dt), R(wx2[0]), seq,
                                       rho[l]);
            c[L::oH + 2 * hh] = arho * (Er[l] + R(dl));
            c[L::oH + 2 * hh + 1] = arho * Dn;
          } else {
            const double Dn = double(damage_rk4<R>(matp<R>(a, l), R(Dm[l]), R(eps[l]), R(dl),
                                                   R(dt), R(wx2[0]), seq, rho[l]));
            c[L::oH + 2 * hh] = R(double(arho) * (eps[l] + dl));
            c[L::oH + 2 * hh + 1] = R(double(arho) * Dn);
          }
        }
    }
  }
  store_sources<P, DIM, NMAT, NH>(a, cell, c, dl > 0.0);
}

// Queue of cells at yield (split path), one per CTA in shared memory, as
// [quantity][slot] columns: the conserved state of the cell and what the
// yield test derived from it (rho_l, D_l, phi_l, eps_l, phi(X), G_mix).
template <class P, int DIM, int NMAT, int NH>
struct SrcQueue {
  typedef typename P::R R;
  typedef typename P::X XT;
  static constexpr int NF = Lay<DIM, NMAT, NH>::NF, NX = Phys<P, DIM, NMAT, NH>::NX;
  static constexpr int NT = 128, CAP = 2 * NT, NV = 4 * NMAT + 2;
  R c[NF][CAP];
  XT cx[NX][CAP];
  R v[NV][CAP];
  double eE[CAP];
  long long cell[CAP];
  unsigned char cy[CAP];
  int n;
};

template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void src_dequeue(const KArgs& a, SrcQueue<P, DIM, NMAT, NH>& q, int s,
                                            double dt, long long step) {
  typedef SrcQueue<P, DIM, NMAT, NH> Q;
  typename Q::R c[Q::NF], rho[NMAT], Dr[NMAT], phir[NMAT], Er[NMAT];
  typename Q::XT cx[Q::NX];
#pragma unroll
  for (int k = 0; k < Q::NF; ++k) c[k] = q.c[k][s];
#pragma unroll
  for (int k = 0; k < Q::NX; ++k) cx[k] = q.cx[k][s];
#pragma unroll
  for (int l = 0; l < NMAT; ++l) {
    rho[l] = q.v[l][s];
    Dr[l] = q.v[NMAT + l][s];
    phir[l] = q.v[2 * NMAT + l][s];
    Er[l] = q.v[3 * NMAT + l][s];
  }
  source_full<P, DIM, NMAT, NH>(a, q.cell[s], c, cx, q.eE[s], rho, Dr, phir, Er,
                                q.v[4 * NMAT][s], q.v[4 * NMAT + 1][s], q.cy[s] != 0, dt, step);
}

// L2 prefetch of the stored state of the 32 cells c0 .. c0 + 31 (FP32-split
// single grids; c0 < ncell): lane k of the warp asks for the line of float
// slot k (slot oE holds nothing in the split form), two lanes for the FP64
// rho E.  A hint only: nothing is read into registers, and every address lies
// inside the state arrays.
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void prefetch_cells_l2(const KArgs& a, long long c0) {
  typedef Lay<DIM, NMAT, NH> L;
  static_assert(P::split && sizeof(typename P::S) == 4 && L::NF + 2 < 32, "one lane per slot");
  const int lane = threadIdx.x & 31;
  const void* p = nullptr;
  if (lane <= L::NF && lane != L::oE && lane < a.nfield)
    p = static_cast<const float*>(a.Uin) + (long long)lane * a.ncell + c0;
  else if (lane == L::NF + 1)
    p = a.Ein + c0;
  else if (lane == L::NF + 2)
    p = a.Ein + (c0 + 16 < a.ncell ? c0 + 16 : a.ncell - 1);
  if (p) asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// Per-cell sources after the sweeps (in place): renormalise det Fbar = 1,
// radial return in Hencky space to the perturbed yield stress (Newton on
// the plastic increment in FP64), then RK4 damage.  Split path: cells
// inside the yield surface take the short path at once; cells at yield are
// queued and returned 128 at a time, so the return runs on full warps
// wherever the yielding cells lie.
//
// sources_cells: cells [base, base + 128) of one grid, one per thread of the
// 128-thread CTA, then the queue drained if it holds a full batch;
// sources_flush: the rest of the queue.  All threads call both together.
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void sources_cells(
    const KArgs& a, long long base,
    typename std::conditional<P::split, SrcQueue<P, DIM, NMAT, NH>, int>::type& qs, double dt,
    long long step) {
  typedef typename P::R R;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  typedef typename P::X XT;
  typedef SrcQueue<P, DIM, NMAT, NH> Q;
  constexpr int NF = L::NF, NX = PH::NX;
  const long long cell = base + threadIdx.x;
    do {
      if (cell >= a.ncell) break;
      R c[NF], w[NF];
      XT cx[NX], wx[NX];
      double eE;
      load_at<P, DIM, NMAT, NH>(a, cell, c, cx, &eE);
      {
        // Fbar = I exactly (A = 0 in the split form): det Fbar = 1 and
        // dev(H) = 0, so no trial stress, no plastic increment and no
        // damage; the source step leaves the cell as it is
        bool ident = true;
#pragma unroll
        for (int k = 0; k < L::NFC; ++k)
          ident = ident && c[L::oF + k] == ((!P::aform && FC<DIM>::idx(k) % 4 == 0) ? R(1) : R(0));
        if (ident) break;
      }
      Aux<R> ax;
      typename PH::Mix mx0;
      if (!PH::template u2w<0>(a, c, cx, w, wx, ax, &eE, &mx0)) {
        report(a.err, ST_ENONFINITE, cell, step);
        break;
      }
      R rho[NMAT], Dr[NMAT], phir[NMAT], Er[NMAT];
      {
        XT phx[NMAT];
        PH::fractions(cx, phx);
#pragma unroll
        for (int l = 0; l < NMAT; ++l) phir[l] = R(phx[l]);
      }
#pragma unroll
      for (int l = 0; l < NMAT; ++l) {
        rho[l] = w[L::oARHO + l];
        Er[l] = R(0);
        Dr[l] = R(0);
#pragma unroll
        for (int h = 0; h < NH; ++h)
          if (a.hslot[l] == h) {
            Er[l] = w[L::oH + 2 * h];
            Dr[l] = w[L::oH + 2 * h + 1];
          }
      }
      R Xc[3] = {R(0), R(0), R(0)};
#pragma unroll
      for (int k = 0; k < DIM; ++k) Xc[k] = w[L::oX + k];
      const R phihat = lookup<DIM, R>(a, Xc);
      // shear modulus of the mixture; whether the cell may yield
      R Gm = R(0);
      bool can_yield = true;
#pragma unroll
      for (int l = 0; l < NMAT; ++l) {
        const auto& m = matp<R>(a, l);
        if (m.eos == 1 && m.G0 > 0 && m.plasticity != 1) can_yield = false;
        if constexpr (!P::split) {
          R te, tp, tdp, tG;
          R tga, tdg;
          thermo(m, rho[l], m.damage != 0 ? R(1) - Dr[l] : R(1), R(0), te, tp, tdp, tG, tga, tdg);
          Gm += phir[l] * tG;
        }
      }
      if constexpr (P::split) {
        // G_mix of the recovery (G does not depend on J2)
        Gm = mx0.Gm;
        // FP32 yield test against the rate-free yield stress; cells clearly
        // inside the yield surface only get det Fbar = 1 (and nothing is
        // written when that leaves Fbar as it is)
        R y0 = R(0);
#pragma unroll
        for (int l = 0; l < NMAT; ++l) {
          const auto& m = matp<R>(a, l);
          if (m.plasticity != 1 || (m.damage != 0 && Dr[l] >= R(m.D_cut))) continue;
          const R e = Er[l] > R(0) ? Er[l] : R(0);
          R hard = R(m.c1);
          if (m.c2 != 0) hard += R(m.c2) * mpow(e, R(m.n_hard));
          y0 += phir[l] * phihat * (m.damage != 0 ? R(1) - Dr[l] : R(1)) * hard;
        }
        const R strf = R(2.449489743f) * mx0.Gm * msqrt(mx0.J2);
        if (!can_yield || !(mx0.Gm > R(0)) || !(strf > y0 * R(0.9999))) {
          R X[9];
          PH::fullX(c, X);
          const R ed = (X[0] + X[4] + X[8]) +
                       (X[0] * X[4] - X[1] * X[3] + X[0] * X[8] - X[2] * X[6] + X[4] * X[8] -
                        X[5] * X[7]) +
                       (X[0] * (X[4] * X[8] - X[5] * X[7]) - X[1] * (X[3] * X[8] - X[5] * X[6]) +
                        X[2] * (X[3] * X[7] - X[4] * X[6]));
          if (ed != R(0)) {
            const R cm1 = mexpm1(mlog1p(ed) / R(3));
#pragma unroll
            for (int k = 0; k < L::NFC; ++k) {
              const int q = FC<DIM>::idx(k);
              c[L::oF + k] = (X[q] - ((q % 4 == 0) ? cm1 : R(0))) / (R(1) + cm1);
            }
            store_sources<P, DIM, NMAT, NH>(a, cell, c, false);
          }
          break;
        }
        // at yield: queue the cell (at most 2 x 128 - 1 entries: the queue is
        // drained below whenever it holds 128)
        const int sl = atomicAdd(&qs.n, 1);
#pragma unroll
        for (int k = 0; k < NF; ++k) qs.c[k][sl] = c[k];
#pragma unroll
        for (int k = 0; k < NX; ++k) qs.cx[k][sl] = cx[k];
#pragma unroll
        for (int l = 0; l < NMAT; ++l) {
          qs.v[l][sl] = rho[l];
          qs.v[NMAT + l][sl] = Dr[l];
          qs.v[2 * NMAT + l][sl] = phir[l];
          qs.v[3 * NMAT + l][sl] = Er[l];
        }
        qs.v[4 * NMAT][sl] = phihat;
        qs.v[4 * NMAT + 1][sl] = Gm;
        qs.eE[sl] = eE;
        qs.cell[sl] = cell;
        qs.cy[sl] = can_yield ? 1 : 0;
      } else {
        source_full<P, DIM, NMAT, NH>(a, cell, c, cx, eE, rho, Dr, phir, Er, phihat, Gm,
                                      can_yield, dt, step);
      }
    } while (false);
  if constexpr (P::split) {
    __syncthreads();
    const int n = qs.n;
    if (n >= Q::NT) {
      src_dequeue<P, DIM, NMAT, NH>(a, qs, n - Q::NT + (int)threadIdx.x, dt, step);
      __syncthreads();
      if (threadIdx.x == 0) qs.n = n - Q::NT;
      __syncthreads();
    }
  }
}

template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ void sources_flush(
    const KArgs& a,
    typename std::conditional<P::split, SrcQueue<P, DIM, NMAT, NH>, int>::type& qs, double dt,
    long long step) {
  if constexpr (P::split) {
    // sources_cells ended on a barrier after the last update of the count
    const int n = qs.n;
    if ((int)threadIdx.x < n) src_dequeue<P, DIM, NMAT, NH>(a, qs, (int)threadIdx.x, dt, step);
    __syncthreads();
    if (threadIdx.x == 0) qs.n = 0;
    __syncthreads();
  }
}

// One grid: the CTA strides over the cells in batches of 128 (uniform trip
// count: the barriers are reached by all).
// MINB: CTAs per SM the registers must allow (launch bound).  The launcher
// takes 5 for FP32-split grids large enough to fill 2432 CTAs (96 instead
// of 104 registers, 5 CTAs per SM instead of 4: 2048^2 ring 235 -> 213 us,
// 256^3 cylinder 1.53 -> 1.48 ms) and 1 below (512^2 ring 36.6 us against
// 37.6 with the bound).
template <class P, int DIM, int NMAT, int NH, int MINB = 1>
__global__ void __launch_bounds__(128, MINB) k_sources(KArgs a) {
  static_assert(SrcQueue<P, DIM, NMAT, NH>::NT == 128, "queue batch = CTA size");
  __shared__ typename std::conditional<P::split, SrcQueue<P, DIM, NMAT, NH>, int>::type qs;
  const double dt = a.info->dt;
  const long long step = a.info->steps;
  if constexpr (P::split) {
    if (threadIdx.x == 0) qs.n = 0;
    __syncthreads();
  }
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < a.ncell; base += stride) {
    // the warp's cells of the next pass are asked into L2 while this pass
    // computes.  Measured on the 256^3 cylinder (one wave, 5 CTAs per SM),
    // ms per step over steps 6-15 / 16-25 / 26-35: 1.09 / 1.38 / 1.93 ->
    // 1.03 / 1.32 / 1.89 (the same prefetch in the CFL kernel, 64 registers,
    // made it slower: 0.447 -> 0.529 ms; in the x sweep, one wave of tiles
    // ahead, it gained 1 %).  Only the one-wave instantiation (MINB 5) takes
    // it: on the 512^2 ring (512 CTAs, four passes each) it cost 2-3 % of
    // the source kernel (44.4 / 48.0 / 51.3 -> 45.6 / 49.3 / 52.8 us).
    if constexpr (std::is_same<P, P32>::value && MINB > 1) {
      const long long nb = base + stride + (threadIdx.x & ~31);
      if (nb < a.ncell) prefetch_cells_l2<P, DIM, NMAT, NH>(a, nb);
    }
    sources_cells<P, DIM, NMAT, NH>(a, base, qs, dt, step);
  }
  sources_flush<P, DIM, NMAT, NH>(a, qs, dt, step);
}

// Every member of a batch: units are chunks of bk.chunk cells (a multiple of
// 128) of one member; the queue is drained at the end of each chunk.
// FP32-split: 5 CTAs per SM (96 registers): the 64-ring ensemble's batched
// sources 1.056 -> 0.951 ms per step.
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(128, P::split ? 5 : 1) k_sources_batch(BatchK bk) {
  __shared__ typename std::conditional<P::split, SrcQueue<P, DIM, NMAT, NH>, int>::type qs;
  __shared__ KArgs ka;
  __shared__ long long s_unit, s_end;
  __shared__ int s_m;
  if (threadIdx.x == 0) {
    s_m = -1;
    s_unit = -1;
    s_end = -1;
  }
  if constexpr (P::split) {
    if (threadIdx.x == 0) qs.n = 0;
  }
  long long ch;
  while (batch_next(bk, ka, ch, s_unit, s_end, s_m)) {
    const double dt = ka.info->dt;
    const long long step = ka.info->steps;
    const long long b0 = ch * bk.chunk;
    const long long b1 = b0 + bk.chunk < ka.ncell ? b0 + bk.chunk : ka.ncell;
    for (long long base = b0; base < b1; base += 128)
      sources_cells<P, DIM, NMAT, NH>(ka, base, qs, dt, step);
    sources_flush<P, DIM, NMAT, NH>(ka, qs, dt, step);
  }
}

// --------------------------------------------------------------- CFL ----
// Largest max_d |u_d| + c_L over cells begin, begin + stride, ... < end.
template <class P, int DIM, int NMAT, int NH>
__device__ __forceinline__ double cfl_max(const KArgs& a, long long begin, long long end,
                                          long long stride, long long step) {
  typedef typename P::R R;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef typename P::X XT;
  constexpr int NF = Lay<DIM, NMAT, NH>::NF, NX = PH::NX;
  double smax = 0.0;
  for (long long cell = begin; cell < end; cell += stride) {
    R c[NF], w[NF];
    XT cx[NX], wx[NX];
    double eE;
    load_at<P, DIM, NMAT, NH>(a, cell, c, cx, &eE);
    Aux<R> ax;
    if (!PH::template u2w<0>(a, c, cx, w, wx, ax, &eE)) {
      report(a.err, ST_ENONFINITE, cell, step);
      continue;
    }
    R v = R(0);
#pragma unroll
    for (int k = 0; k < DIM; ++k) v = mabs(ax.u[k]) > v ? mabs(ax.u[k]) : v;
    const double s = double(v + ax.cL);
    smax = s > smax ? s : smax;
  }
  return smax;
}

// CTA maximum of a non-negative value into *dst (bits of a double); all
// threads call it together.
__device__ __forceinline__ void cta_max_to(unsigned long long* dst, double smax) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) smax = fmax(smax, __shfl_xor_sync(0xffffffffu, smax, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) m = fmax(m, red[i]);
    atomicMax(dst, (unsigned long long)__double_as_longlong(m));
  }
}

// The CFL reduction of one grid; the last CTA to finish (counted with an
// atomic after a fence, no waiting) forms dt for the step.
// FP32-split: four 256-thread CTAs per SM (64 registers, 16 bytes spilled);
// the FP64 recovery would spill 260 bytes under that cap, so it has none.
// Launched as one wave of resident CTAs that stride over the cells.
// Measured on the 512^2 ring: 29.8 us with 3 CTAs per SM over 2.25 waves,
// 24.0 with the cap, 22.9 in one wave, 19.7 with both.
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256, P::split ? 4 : 1) k_cfl(KArgs a) {
  const double smax = cfl_max<P, DIM, NMAT, NH>(a, blockIdx.x * (long long)blockDim.x + threadIdx.x,
                                                a.ncell, (long long)gridDim.x * blockDim.x,
                                                a.info->steps);
  cta_max_to(&a.info->smax_bits, smax);
  __shared__ bool last;
  if (threadIdx.x == 0) {
    __threadfence();  // this CTA's atomicMax before its count
    last = atomicAdd(&a.info->cfl_done, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();  // every other CTA's atomicMax before the read
    a.info->cfl_done = 0u;
    dt_update(a.info, a.err, a.cfl, a.dxmin, a.dx, a.dim);
  }
}

// Every member of a batch, in chunks of bk.chunk cells.
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_cfl_batch(BatchK bk) {
  __shared__ KArgs ka;
  __shared__ long long s_unit, s_end;
  __shared__ int s_m;
  if (threadIdx.x == 0) {
    s_m = -1;
    s_unit = -1;
    s_end = -1;
  }
  long long ch;
  while (batch_next(bk, ka, ch, s_unit, s_end, s_m)) {
    const long long b0 = ch * bk.chunk;
    const long long b1 = b0 + bk.chunk < ka.ncell ? b0 + bk.chunk : ka.ncell;
    const double smax = cfl_max<P, DIM, NMAT, NH>(ka, b0 + threadIdx.x, b1, blockDim.x,
                                                  ka.info->steps);
    cta_max_to(&ka.info->smax_bits, smax);
  }
}

// ------------------------------------- X by WENO3 + RK3 (Sec. 3.2.1) ----
// The alternative to carrying X in the sweeps:
//   dX/dt = -sum_d [u_{d,i+1/2} (X_{i+1/2} - X_i) - u_{d,i-1/2} (X_{i-1/2} - X_i)] / dx_d
// (the difference of the fluxes X u_d plus X div(u), so DX/Dt = 0), face
// velocity the mean of the two cell velocities, face X the third-order WENO
// value reconstructed in the upwind cell, Shu and Osher's three-stage TVD
// Runge-Kutta scheme with the velocities of the step's start; ghosts follow
// the sweeps' boundary rules.  All before the sweeps; the result replaces X
// after them.

// Cell velocities of the step's start into xs[0].
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_xvel(KArgs a) {
  typedef typename P::R R;
  typedef Lay<DIM, NMAT, NH> L;
  const R* U = static_cast<const R*>(a.Uin);
  R* V = static_cast<R*>(a.xs[0]);
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < a.ncell;
       c += (long long)gridDim.x * blockDim.x) {
    R rho = R(0);
#pragma unroll
    for (int l = 0; l < NMAT; ++l) rho += U[(long long)(L::oARHO + l) * a.ncell + c];
#pragma unroll
    for (int d = 0; d < DIM; ++d) V[(long long)d * a.ncell + c] = U[(long long)(L::oMOM + d) * a.ncell + c] / rho;
  }
}

// WENO3 value at the face between cells b and c reconstructed in cell b
// from its neighbours a (away from the face) and c (across it): candidates
// -a/2 + 3b/2 and (b + c)/2, linear weights 1/3 and 2/3, smoothness
// ((b - a)/dx)^2 and ((c - b)/dx)^2, eps = 1e-6 (Jiang and Shu).
template <class R>
__device__ __forceinline__ R weno3_face(R a, R b, R c, R dx) {
  const R q0 = R(-0.5) * a + R(1.5) * b;
  const R q1 = R(0.5) * b + R(0.5) * c;
  const R s0 = (b - a) / dx, s1 = (c - b) / dx;
  const R e0 = R(1e-6) + s0 * s0, e1 = R(1e-6) + s1 * s1;
  const R a0 = (R(1) / R(3)) / (e0 * e0);
  const R a1 = (R(2) / R(3)) / (e1 * e1);
  return (a0 * q0 + a1 * q1) / (a0 + a1);
}

// One RK stage (1, 2, 3): stage s reads X from src (stage 1: the state)
// and writes dst = X0 + dt L (1), 3/4 X0 + 1/4 (X1 + dt L) (2),
// 1/3 X0 + 2/3 (X2 + dt L) (3), X0 the state's X.
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_xstage(KArgs a, int stage) {
  typedef typename P::R R;
  typedef Lay<DIM, NMAT, NH> L;
  const long long nc = a.ncell;
  const R* X0 = static_cast<const R*>(a.Uin) + (long long)L::oX * nc;
  const R* V = static_cast<const R*>(a.xs[0]);
  const R* src = stage == 1 ? X0 : static_cast<const R*>(a.xs[stage - 1]);
  R* dst = static_cast<R*>(a.xs[stage == 2 ? 2 : 1]);
  const R dt = R(a.info->dt);
  // grids here hold fewer than 2^31 cells (checked on the host): 32-bit indices
  const int n0 = a.n[0], n1 = a.n[1];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < (int)nc; c += gridDim.x * blockDim.x) {
    const int idx[3] = {c % n0, (c / n0) % n1, c / (n0 * n1)};
    R Lk[DIM];
#pragma unroll
    for (int k = 0; k < DIM; ++k) Lk[k] = R(0);
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      const int n = a.n[d];
      const int stride = d == 0 ? 1 : (d == 1 ? n0 : n0 * n1);
      const bool inner = idx[d] >= 2 && idx[d] + 2 < n;  // the whole stencil inside the grid
      // velocity component d on the stencil (negated across a mirror wall)
      R u[5];
#pragma unroll
      for (int o = -2; o <= 2; ++o) {
        if (inner) {
          u[o + 2] = V[(long long)d * nc + c + o * stride];
        } else {
          int j = idx[d] + o;
          bool mirror = false;
          if (j < 0 || j >= n) {
            const int side = j < 0 ? 0 : 1;
            const int bc = a.bc[d][side];
            if (bc == BC_P) j = side == 0 ? j + n : j - n;
            else if (bc == BC_R) { mirror = true; j = side == 0 ? -1 - j : 2 * n - 1 - j; }
            else j = side == 0 ? 0 : n - 1;
          }
          const R uv = V[(long long)d * nc + c + (j - idx[d]) * stride];
          u[o + 2] = mirror ? -uv : uv;
        }
      }
      const R dx = R(a.dx[d]);
      const R uL = R(0.5) * (u[1] + u[2]), uR = R(0.5) * (u[2] + u[3]);
      const bool pr = uR >= R(0), pl = uL >= R(0);
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        R x[5];
#pragma unroll
        for (int o = -2; o <= 2; ++o) {
          if (inner) {
            x[o + 2] = src[(long long)k * nc + c + o * stride];
          } else {
            int j = idx[d] + o;
            R shift = R(0);
            bool mirror = false;
            int side = 0;
            if (j < 0 || j >= n) {
              side = j < 0 ? 0 : 1;
              const int bc = a.bc[d][side];
              if (bc == BC_P) {
                shift = side == 0 ? -R(a.hi[d] - a.lo[d]) : R(a.hi[d] - a.lo[d]);
                j = side == 0 ? j + n : j - n;
              } else if (bc == BC_R) {
                mirror = true;
                j = side == 0 ? -1 - j : 2 * n - 1 - j;
              } else {
                j = side == 0 ? 0 : n - 1;
              }
            }
            R xv = src[(long long)k * nc + c + (j - idx[d]) * stride];
            if (k == d) {
              if (mirror) xv = R(2) * R(side == 0 ? a.lo[d] : a.hi[d]) - xv;
              xv += shift;
            }
            x[o + 2] = xv;
          }
        }
        // the upwind cell's stencil first, then one reconstruction per face
        const R XR = weno3_face(pr ? x[1] : x[4], pr ? x[2] : x[3], pr ? x[3] : x[2], dx);
        const R XL = weno3_face(pl ? x[0] : x[3], pl ? x[1] : x[2], pl ? x[2] : x[1], dx);
        Lk[k] -= (uR * (XR - x[2]) - uL * (XL - x[2])) / dx;
      }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) {
      const long long q = (long long)k * nc + c;
      if (stage == 1)
        dst[q] = X0[q] + dt * Lk[k];
      else if (stage == 2)
        dst[q] = R(0.75) * X0[q] + R(0.25) * (src[q] + dt * Lk[k]);
      else
        dst[q] = (R(1) / R(3)) * X0[q] + (R(2) / R(3)) * (src[q] + dt * Lk[k]);
    }
  }
}

// ------------------------------------------------------------ seeding ----
// Lagrangian seeding into void (Sec. 3.2.1 seeding routine): each cell with
// void fraction nu > 1/2 and a normal (|grad nu| h > 1e-6) takes
// X = X(p) - (p - c), c its centre, p = c + 1.5 h n the probe, n =
// -grad nu / |grad nu| (pointing into the material), h the largest cell
// size, X(p) multilinear in the cell-centred X of the step's start.  Cells
// outside the grid follow the sweeps' ghost rules (periodic: wrapped, X
// shifted by the period; reflective: mirrored, X reflected about the wall;
// transmissive: the edge cell).  The geometry and the interpolation run in
// FP64 on both paths, in the order of their definition; every cell's X
// (seeded or not) goes to a.xseed, copied over the state's X afterwards.

// Index along d mapped into the grid; X_d of that cell maps to the ghost by
// X -> 2 wall - X (mirror) and + shift.
__device__ __forceinline__ long long seed_map(const KArgs& a, int d, long long i, double& shift,
                                              bool& mirror, double& wall) {
  const long long n = a.n[d];
  shift = 0.0;
  mirror = false;
  wall = 0.0;
  if (i >= 0 && i < n) return i;
  const int side = i < 0 ? 0 : 1;
  const int bc = a.bc[d][side];
  if (bc == BC_P) {
    shift = side == 0 ? -(a.hi[d] - a.lo[d]) : (a.hi[d] - a.lo[d]);
    return side == 0 ? i + n : i - n;
  }
  if (bc == BC_R) {
    mirror = true;
    wall = side == 0 ? a.lo[d] : a.hi[d];
    return side == 0 ? -1 - i : 2 * n - 1 - i;
  }
  return side == 0 ? 0 : n - 1;
}

template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_seed(KArgs a) {
  typedef typename P::S S;
  typedef Lay<DIM, NMAT, NH> L;
  const S* U = static_cast<const S*>(a.Uin);
  S* out = static_cast<S*>(a.xseed);
  const long long nc = a.ncell;
  const long long nuo = phislot<P, DIM, NMAT, NH>(a, a.void_l, 0);
  double h = 0.0;
#pragma unroll
  for (int d = 0; d < DIM; ++d) h = a.dx[d] > h ? a.dx[d] : h;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < nc;
       c += (long long)gridDim.x * blockDim.x) {
    const long long ix[3] = {c % a.n[0], (c / a.n[0]) % a.n[1], c / ((long long)a.n[0] * a.n[1])};
    bool seed = double(U[nuo + c]) > 0.5;
    double gr[3] = {0.0, 0.0, 0.0}, gn = 0.0;
    if (seed) {
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        double sh, wl;
        bool mr;
        long long q[2];
#pragma unroll
        for (int o = 0; o < 2; ++o) {
          long long j[3] = {ix[0], ix[1], ix[2]};
          j[d] = seed_map(a, d, ix[d] + (o == 0 ? -1 : 1), sh, mr, wl);
          q[o] = j[0] + (long long)a.n[0] * (j[1] + (long long)a.n[1] * j[2]);
        }
        gr[d] = (double(U[nuo + q[1]]) - double(U[nuo + q[0]])) / (2.0 * a.dx[d]);
        gn += gr[d] * gr[d];
      }
      gn = sqrt(gn);
      seed = gn * h > 1e-6;
    }
    if (!seed) {
#pragma unroll
      for (int k = 0; k < DIM; ++k) out[(long long)k * nc + c] = U[(long long)(L::oX + k) * nc + c];
      continue;
    }
    double cc[3], p[3], f[3];
    long long i0[3] = {0, 0, 0};
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
      cc[d] = a.lo[d] + (double(ix[d]) + 0.5) * a.dx[d];
      p[d] = cc[d] + 1.5 * h * (-gr[d] / gn);
      const double s = (p[d] - a.lo[d]) / a.dx[d] - 0.5;
      const double fl = floor(s);
      i0[d] = (long long)fl;
      f[d] = s - fl;
    }
    double Xi[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int corner = 0; corner < (1 << DIM); ++corner) {
      long long j[3] = {0, 0, 0};
      double shift[3] = {0.0, 0.0, 0.0}, wall[3] = {0.0, 0.0, 0.0};
      bool mirror[3] = {false, false, false};
      double w = 1.0;
#pragma unroll
      for (int d = 0; d < DIM; ++d) {
        const int b = (corner >> d) & 1;
        j[d] = seed_map(a, d, i0[d] + b, shift[d], mirror[d], wall[d]);
        w *= b ? f[d] : 1.0 - f[d];
      }
      const long long q = j[0] + (long long)a.n[0] * (j[1] + (long long)a.n[1] * j[2]);
#pragma unroll
      for (int k = 0; k < DIM; ++k) {
        double x = double(U[(long long)(L::oX + k) * nc + q]);
        if (mirror[k]) x = 2.0 * wall[k] - x;
        Xi[k] += w * (x + shift[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < DIM; ++k) out[(long long)k * nc + c] = S(Xi[k] - (p[k] - cc[k]));
  }
}

// ------------------------------------------------------ init and read ----
template <class P, int DIM, int NMAT, int NH>
__global__ void k_init(KArgs a) {
  typedef typename P::R R;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  typedef typename P::X XT;
  constexpr int NF = L::NF, NX = PH::NX;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < a.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    R w[NF], c[NF];
    XT wx[NX], cx[NX];
    double phisum = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double v = a.prim[(long long)f * a.ncell + cell];
      if (P::aform && f >= L::oF && f < L::oF + L::NFC) {
        const int ij = FC<DIM>::idx(f - L::oF);
        if (ij % 4 == 0) v -= 1.0;
      }
      w[f] = R(v);
      if (f == L::oE) wx[0] = XT(v);
      if (f < L::oARHO) {
        wx[1 + f] = XT(v);
        phisum += v;
      }
    }
    // all N fractions carried: the last one formed once, here, in FP64
    if (P::allphi) wx[NX - 1] = XT(1.0 - phisum);
    Aux<R> ax;
    double eE = 0.0;
    if (!PH::template w2u<0>(a, w, wx, c, cx, ax, &eE)) report(a.err, ST_ENONFINITE, cell, 0);
    store_cell<P, DIM, NMAT, NH>(a, cell, c, cx, eE);
  }
}

template <class P, int DIM, int NMAT, int NH>
__global__ void k_read(KArgs a, int primitive) {
  typedef typename P::R R;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  typedef typename P::X XT;
  constexpr int NF = L::NF, NX = PH::NX;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < a.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    R c[NF], w[NF];
    XT cx[NX], wx[NX];
    double eE;
    load_at<P, DIM, NMAT, NH>(a, cell, c, cx, &eE);
    const R* src = c;
    const XT* srcx = cx;
    if (primitive) {
      Aux<R> ax;
      if (!PH::template u2w<0>(a, c, cx, w, wx, ax, &eE)) report(a.err, ST_ENONFINITE, cell, 0);
      src = w;
      srcx = wx;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      double v = double(src[f]);
      if (f == L::oE) v = primitive ? double(srcx[0]) : eE;
      if (f < L::oARHO) v = double(srcx[1 + f]);
      if (P::aform && f >= L::oF && f < L::oF + L::NFC) {
        const int ij = FC<DIM>::idx(f - L::oF);
        if (ij % 4 == 0) v += 1.0;
      }
      a.prim[(long long)f * a.ncell + cell] = v;
    }
  }
}

// ------------------------------------------------------------ totals ----
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_totals(KArgs a) {
  typedef Lay<DIM, NMAT, NH> L;
  typedef typename P::S S;
  constexpr int NQ = NMAT + 4;
  double acc[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) acc[q] = 0.0;
  const S* U = (const S*)a.Uin;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < a.ncell;
       cell += (long long)gridDim.x * blockDim.x) {
#pragma unroll
    for (int l = 0; l < NMAT; ++l) acc[l] += double(U[(long long)(L::oARHO + l) * a.ncell + cell]);
#pragma unroll
    for (int k = 0; k < DIM; ++k)
      acc[NMAT + k] += double(U[(long long)(L::oMOM + k) * a.ncell + cell]);
    acc[NMAT + 3] += P::split ? a.Ein[cell] : double(U[(long long)L::oE * a.ncell + cell]);
  }
  __shared__ double red[8][NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5][q] = v;
  }
  __syncthreads();
  if (threadIdx.x < NQ) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i][threadIdx.x];
    a.partial[(long long)blockIdx.x * NQ + threadIdx.x] = s;
  }
}

// ----------------------------------------------------------- fragments ----
// Marks the cells of fragments at void cut-off a.fcut (Sec. 4.2, 4.3
// demarcate fragments by a contour of the void fraction; in this gas-filled
// model a cell is in a fragment when its solid fraction exceeds 1 - theta
// and no solid in it is critically damaged, D >= D_crit (1 - 1e-4) as in
// the yield stress): a.frag[cell] = cell there and
// -1 elsewhere; a.fmass[cell] = dV sum (phi rho) over the solids on those
// cells (left as it is elsewhere).  Each
// warp also links the runs of fragment cells along x within its 32 cells:
// a member points at the first member of its run (a run stops at a
// non-member, at the first cell of a row and at the warp's first lane), so
// the union pass needs no x-links inside a warp.  Requires ncell < 2^31.
template <class P, int DIM, int NMAT, int NH>
__global__ void __launch_bounds__(256) k_frag_mark(KArgs a) {
  typedef typename P::R R;
  typedef typename P::S S;
  typedef typename P::X XT;
  typedef Phys<P, DIM, NMAT, NH> PH;
  typedef Lay<DIM, NMAT, NH> L;
  constexpr int NX = PH::NX;
  const S* U = (const S*)a.Uin;
  // The cut: the FP64 path compares in FP64 with 1 - theta (a.fthr).  The
  // FP32-split path compares its FP32 fractions with the largest float not
  // above 1 - theta (a.fthrf), which for one solid (its fraction one stored
  // float) decides exactly as the FP64 comparison; the scarce FP64 pipe is
  // left to the members' masses.  The constants come with the launch.
  // whole warps run the loop (bound rounded up to the warp) for the ballots
  const long long end = (a.ncell + 31) / 32 * 32;
  const int lane = threadIdx.x & 31;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < end;
       cell += (long long)gridDim.x * blockDim.x) {
    bool in = false;
    R arho[NMAT];
    if (cell < a.ncell) {
      XT cx[NX], phid[NMAT];
      cx[0] = XT(0);
#pragma unroll
      for (int l = 0; l < PH::NPX; ++l) cx[1 + l] = XT(U[phislot<P, DIM, NMAT, NH>(a, l, cell)]);
      PH::fractions(cx, phid);
      XT phis = XT(0);
      bool crit = false;
#pragma unroll
      for (int l = 0; l < NMAT; ++l) {
        arho[l] = R(0);
        if (a.mat[l].eos != 1) continue;
        phis += phid[l];
        arho[l] = R(U[(long long)(L::oARHO + l) * a.ncell + cell]);
#pragma unroll
        for (int h = 0; h < NH; ++h)
          if (h == a.hslot[l] && a.mat[l].damage != 0) {
            const R D = R(U[(long long)(L::oH + 2 * h + 1) * a.ncell + cell]) / arho[l];
            crit = crit || D >= (P::split ? R(a.fdcritf[l]) : R(a.fdcrit[l]));
          }
      }
      if constexpr (P::split)
        in = float(phis) > a.fthrf && !crit;
      else
        in = double(phis) > a.fthr && !crit;
    }
    const unsigned mem = __ballot_sync(0xffffffffu, in);
    const unsigned rows = __ballot_sync(0xffffffffu, cell < a.ncell && (int)cell % a.n[0] == 0);
    // run starts: members whose left lane is not a member, or that begin a row
    const unsigned starts = mem & (~(mem << 1) | rows);
    const unsigned upto = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
    const int s = 31 - __clz(starts & upto);
    if (cell < a.ncell) {
      a.frag[cell] = in ? (int)(cell - lane + s) : -1;
      if (in) {  // read for fragment cells only
        double ms = 0.0;
#pragma unroll
        for (int l = 0; l < NMAT; ++l)
          if (a.mat[l].eos == 1) ms += double(arho[l]) * a.fdV;
        a.fmass[cell] = ms;
      }
    }
  }
}

}  // namespace mm
