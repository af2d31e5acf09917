// Internal declarations shared by the host API (mm_api.cu) and the kernel
// translation units (mm_fp64.cu, mm_fp32.cu).  Not part of the public ABI.
#pragma once

#include <cuda.h>  // CUtensorMap (type only; the encoder is reached through the runtime)
#include <cuda_runtime.h>
#include <stdint.h>

#include "mmfrac.h"

#define MM_MAXMAT 3

// Material constants as the kernels use them (copied from mm_material, plus
// derived values computed once on the host).
struct MatK {
  int eos, plasticity, damage, shear_model;  // shear_model: 0 Romenskii, 1 Steinberg
  double rho0, K0, G0, alpha, beta, Gamma0, gamma_gas;
  double c1, c2, c3, n_hard, edot0;
  double D_crit, eps_t, eps_c, alpha_D, poisson, Ddot0;
  double xi;     // 1 / Grueneisen coefficient (ideal gas: 1/(gamma-1))
  double Gamma;  // Grueneisen coefficient (ideal gas: gamma - 1)
  // Bonora constants: alpha_D D_c^(1/alpha_D) / ln(eps_c/eps_t), and
  // eps_c^(2n), eps_t^(2n) of the threshold law (n the hardening exponent)
  double bon_k, bon_ec2n, bon_et2n;
  // critical damage threshold D_crit (1 - 1e-4): D comes back as the ratio
  // (phi rho D) / (phi rho) of two transported quantities, so a capped
  // state reads below D_crit by rounding (FP32 storage: about 1e-7 a step)
  // or by a trace of undamaged material mixed in
  double D_cut;
  // Steinberg shear modulus and Grueneisen function (shear_model 1)
  double Gp, Gamma1, Gamma2, gamma_s;
};

// The same constants in FP32 for the FP32-split kernels, which read them as
// operands straight from the parameter bank (a double constant would cost a
// conversion on the FP64 pipe at every use), plus ratios the FP32 closure
// uses in place of divisions.
struct MatKf {
  int eos, plasticity, damage, alpha_one;  // alpha_one: alpha == 1
  float rho0, K0, G0, alpha, beta, Gamma0, gamma_gas;
  float c1, c2, c3, n_hard, edot0;
  float D_crit, eps_t, eps_c, alpha_D, poisson, Ddot0;
  float xi, Gamma, bon_k, bon_ec2n, bon_et2n;
  float inv_rho0;  // 1 / rho0
  float K0_2a2;    // K0 / (2 alpha^2)
  float K0_arho0;  // K0 / (alpha rho0)
  float c2n;       // c2 n_hard
  float D_cut;     // the FP64 threshold rounded to FP32
  int shear_model;
  float Gp, Gamma1, Gamma2, gamma_s;
};

// First failure seen on the device (sticky until the host clears it).
struct DevErr {
  int code;       // 0 or an mm_status
  int pad;
  long long cell; // linear cell index
  long long step; // step counter at the failure
};

// Device-resident step bookkeeping; dt never leaves the device inside a step.
struct DevInfo {
  double t, dt, smax;
  unsigned int cfl_done;         // CTAs of the CFL reduction finished this step (reset by the last)
  unsigned int pad;
  long long steps;
  unsigned long long smax_bits;  // running max of the signal speed (bits of a >= 0 double)
  double lam[3];                 // dt / dx_k of the step (0 for an axis the grid lacks)
};

// dt = cfl dx_min / s_max from the finished CFL reduction; advances t and
// the step count, forms the sweeps' dt / dx_k, clears the running maximum.
// The maximum is read past L1 (other CTAs raised it by atomics).
__device__ __forceinline__ void dt_update(DevInfo* info, DevErr* err, double cfl, double dxmin,
                                          const double* dx, int dim) {
  const unsigned long long bits = *(volatile unsigned long long*)&info->smax_bits;
  const double smax = __longlong_as_double((long long)bits);
  info->smax_bits = 0ull;
  info->steps += 1;
  const double dt = cfl * dxmin / smax;
  if (!(dt > 0.0) || !isfinite(dt)) {
    if (atomicCAS(&err->code, 0, MM_EDT) == 0) {
      err->cell = -1;
      err->step = info->steps;
    }
  }
  info->dt = dt;
  info->smax = smax;
  info->t += dt;
  for (int k = 0; k < 3; ++k) info->lam[k] = k < dim ? dt / dx[k] : 0.0;
}

// Everything a kernel needs, passed by value.
struct KArgs {
  int dim, nmat, nhist, nfield;
  int n[3];
  long long ncell;
  double dx[3], lo[3], hi[3];
  int bc[3][2];
  int hslot[MM_MAXMAT];
  int void_l;          // index of the void material (eos 2), or -1
  int pad_void;
  MatK mat[MM_MAXMAT];
  MatKf matf[MM_MAXMAT];
  const void* Uin;     // conserved fields [nfield][ncell] (double or float)
  void* Uout;
  const double* Ein;   // rho E [ncell] (FP32-split storage only)
  double* Eout;
  const float* phi0;
  int pn[3];
  double plo[3], ph[3];
  float plof[3], phf[3];  // plo, ph in FP32
  DevInfo* info;
  DevErr* err;
  double cfl, dxmin;
  double* prim;        // [nfield][ncell] doubles for init / read
  double* partial;     // per-block partial totals
  void* xs[3];         // X by WENO3 + RK3: cell velocities, stage 1, stage 2 ([dim][ncell], R)
  void* xseed;         // Lagrangian seeding (void grids): X after seeding ([dim][ncell], S)
  const void* tma;     // host address of the grid's SweepTmaSet, or null (read by the host
                       // launcher only, which passes the maps of Uin to the kernel)
  int* frag;           // fragment labelling: per-cell parent index, -1 outside fragments
  double* fmass;       // fragment labelling: per-cell solid mass dV sum (phi rho)_solid
  double fcut;         // fragment labelling: void cut-off theta
  // fragment labelling constants of the launch (set on the host): 1 - theta,
  // the largest float not above it, D_crit (1 - 1e-4) per material in FP64
  // and FP32, the cell volume
  double fthr, fdV;
  double fdcrit[MM_MAXMAT];
  float fthrf;
  float fdcritf[MM_MAXMAT];
  float fpad;
};

static_assert(sizeof(KArgs) % 8 == 0, "KArgs is copied as 8-byte words");

// Fragment labelling (mm_frag.cu), after the marking kernel has set
// a.frag[i] = i on fragment cells and -1 elsewhere (a.ncell < 2^31):
// mm_frag_label joins face neighbours (periodic faces wrap) by union-find
// with links to the smaller root, then points every cell at its root, the
// smallest cell index of its fragment.  mm_frag_count writes, per block of
// MM_FRAG_CELLS cells, the exclusive count of roots before it (boff[b],
// nblocks + 1 entries) and the total to boff[nblocks].  mm_frag_collect
// numbers the roots in index order (fid) and accumulates each fragment's
// label, cell count and mass.
#define MM_FRAG_CELLS 2048
cudaError_t mm_frag_label(const KArgs& a, cudaStream_t s);
cudaError_t mm_frag_count(const KArgs& a, int* boff, cudaStream_t s);
cudaError_t mm_frag_collect(const KArgs& a, const int* boff, int* fid, long long* flabel,
                            unsigned long long* fcells, double* fmass, cudaStream_t s);

// One batched launch over the members of a batch: member m owns work units
// [start[m], start[m+1]) (tiles of a sweep, or chunks of `chunk` cells) and
// its arguments args[m]; persistent CTAs take units from *counter (zero at
// launch).
struct BatchK {
  const KArgs* args;
  const long long* start;
  unsigned long long* counter;
  long long base;    // units before the launch's first member (start[0])
  long long total;   // start[M]
  long long chunk;   // cells per unit of the CFL and source launches (multiple of 128)
  int M;
  int cta_per_sm;    // persistent CTAs per SM (0: as many as fit)
};

// Sets the message mm_last_error() returns on the calling thread.
void mm_internal_set_error(const char* msg);

// Launchers implemented in the precision x dimension translation units
// (mm_fp64_d{1,2,3}.cu, mm_fp32_d{1,2,3}.cu).  what: 0 init, 1 read
// (flag = primitive), 2 CFL reduction, 3 sweep along axis, 4 sources,
// 5 totals into out (nblocks partials), 6 cell velocities for X, 7 X stage
// (flag = 1, 2, 3).
#define MM_DECLARE_LAUNCHER(name)                                                          \
  cudaError_t name(int what, int axis, int flag, const KArgs& a, double* out, int nblocks, \
                   cudaStream_t s);
MM_DECLARE_LAUNCHER(mm_p64_d1)
MM_DECLARE_LAUNCHER(mm_p64_d2)
MM_DECLARE_LAUNCHER(mm_p64_d3)
MM_DECLARE_LAUNCHER(mm_p32_d1)
MM_DECLARE_LAUNCHER(mm_p32_d2)
MM_DECLARE_LAUNCHER(mm_p32_d3)
// grids with a void material (mm_fp{64,32}_d{1,2,3}_void.cu): two or three
// materials, one of them plastic
MM_DECLARE_LAUNCHER(mm_p64_d1_void)
MM_DECLARE_LAUNCHER(mm_p64_d2_void)
MM_DECLARE_LAUNCHER(mm_p64_d3_void)
MM_DECLARE_LAUNCHER(mm_p32_d1_void)
MM_DECLARE_LAUNCHER(mm_p32_d2_void)
MM_DECLARE_LAUNCHER(mm_p32_d3_void)
#undef MM_DECLARE_LAUNCHER

// Batched launchers (mm_fp{64,32}_d{1,2,3}_batch.cu): what 0 CFL, 1 sweep
// along axis with tile variant `variant` (0 or 1; FP64 has one shape), 2
// sources; two materials (nhist 0 or 1); persistent CTAs, one wave at full
// occupancy.  name_tiles: tiles of one sweep of a grid of n cells per axis.
#define MM_DECLARE_BATCH_LAUNCHER(name)                                                     \
  cudaError_t name(int what, int axis, int variant, int nmat, int nhist, const BatchK& b, \
                   cudaStream_t s);                                                         \
  long long name##_tiles(int axis, int variant, const int n[3]);
MM_DECLARE_BATCH_LAUNCHER(mm_p64_d1_batch)
MM_DECLARE_BATCH_LAUNCHER(mm_p64_d2_batch)
MM_DECLARE_BATCH_LAUNCHER(mm_p64_d3_batch)
MM_DECLARE_BATCH_LAUNCHER(mm_p32_d1_batch)
MM_DECLARE_BATCH_LAUNCHER(mm_p32_d2_batch)
MM_DECLARE_BATCH_LAUNCHER(mm_p32_d3_batch)
#undef MM_DECLARE_BATCH_LAUNCHER

// TMA tile loads of the 3D FP32-split y and z sweeps (k_sweep_col_tma): one
// tensor map per part of the state a tile reads, with a box of TW cells
// along x, TL along the sweep axis and one along the remaining axis: the
// float slots 0 .. oE - 1 (lo) and oE + 1 .. NF (hi; slot oE is unused in
// the split form) of the [slot][z][y][x] float array, and the FP64 rho E
// array (e).  Maps live in kernel parameters (__grid_constant__).
struct ColTma {
  CUtensorMap lo, hi, e;
};

// A grid's maps: per state buffer U[b] (E[b]) and sweep axis 1, 2.  nlo,
// nhi, TL, TW: the box the maps were encoded with; the launcher uses them
// only when they equal its kernel's (so the bytes a tile expects are the
// bytes the copies deliver).
struct SweepTmaSet {
  const void* U[2];
  ColTma m[2][2];
  int nlo, nhi, TL[2], TW;
};

// Launches the staged column sweep of a 3D FP32-split grid of two materials
// (nhist 0 or 1) along axis 1 or 2: K tiles per CTA, grid CTAs, maps tm.
cudaError_t mm_p32_d3_col_tma(int nhist, int axis, const KArgs& a, int K, unsigned grid,
                              const ColTma& tm, cudaStream_t s);

// Encodes s for a 3D FP32-split grid without void of n cells per axis,
// nmat materials and nhist plastic materials whose state buffers are U[b]
// ([nfield + 1][ncell] floats) and E[b] ([ncell] doubles).  Returns false
// (s untouched) where a map cannot describe the grid: n[0] not a multiple
// of 4 (row strides of 16 bytes), an encoder that is unavailable or refuses.
bool mm_p32_d3_tma_encode(SweepTmaSet* s, void* const U[2], double* const E[2], const int n[3],
                          int nmat, int nhist);
