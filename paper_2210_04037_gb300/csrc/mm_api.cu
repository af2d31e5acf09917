// C-ABI host side of the mmfrac library: grid lifetime, initial state,
// the step driver loop (dt stays on the device), read-back and totals.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "mm_internal.h"
#include "mmfrac.h"

namespace {

thread_local std::string g_error;

mm_status fail(mm_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_error = buf;
  return s;
}

#define CUDA_TRY(call)                                                          \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return fail(MM_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

// The same for every member of a batch (one thread per member).
__global__ void k_dt_batch(const KArgs* args, int M, double cfl) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m < M) dt_update(args[m].info, args[m].err, cfl, args[m].dxmin, args[m].dx, args[m].dim);
}

}  // namespace

void mm_internal_set_error(const char* msg) { g_error = msg; }

namespace mm {
// Sum of the per-block partial totals, one warp per quantity, scaled by dV.
__global__ void k_totals_final(const double* partial, int nblocks, int nq, double dV,
                               double* out) {
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= nq) return;
  double s = 0.0;
  for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * nq + q];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) out[q] = s * dV;
}
}  // namespace mm

struct mm_grid {
  mm_grid_desc desc;
  int dim = 0, nmat = 0, nhist = 0, nfield = 0, prec = 0;
  long long ncell = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* U[2] = {nullptr, nullptr};
  double* E[2] = {nullptr, nullptr};
  int cur = 0;
  DevInfo* info = nullptr;
  DevErr* err = nullptr;
  double* prim = nullptr;
  double* partial = nullptr;
  double* tot = nullptr;
  int tot_blocks = 0;
  float* phi0 = nullptr;
  bool ready = false;
  long long launches = 0;
  KArgs base;
  // a step replayed from a CUDA graph, one per parity of the ping-pong
  // buffers at the step's start (recaptured when cfl changes)
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  double gcfl[2] = {0.0, 0.0};
  long long glaunches = 0;  // kernels in one captured step
  bool gwarm = false;       // a step ran uncaptured (kernel attributes are set)
  bool nograph = false;     // capture refused on this stream: launch directly
  // kernel timing
  bool prof = false;
  std::vector<cudaEvent_t> ev;      // pool, two per timed launch
  std::vector<int> ev_kind;         // kind of each started pair
  double prof_ms[MM_K_COUNT] = {};
  long long prof_n[MM_K_COUNT] = {};
  // X by WENO3 + RK3: scheme and its scratch (velocities, two stages)
  int xscheme = MM_X_SWEEP;
  void* xs[3] = {nullptr, nullptr, nullptr};
  void* xseed = nullptr;    // Lagrangian seeding scratch (grids with void)
  bool seed_x = true;       // seeding before each step (grids with void)
  // tensor maps of the TMA-staged y and z sweeps (3D FP32-split grids of
  // two materials without void, n[0] a multiple of 4), and their switch
  SweepTmaSet* tma = nullptr;
  bool tma_on = true;
  // fragment labelling scratch (allocated on the first mm_fragments):
  // per-cell parents, fragment numbers of the roots and solid masses, the
  // per-block root offsets, and per-fragment labels, cell counts and masses
  int* fparent = nullptr;
  int* ffid = nullptr;
  double* fcm = nullptr;
  int* fboff = nullptr;
  long long* flab = nullptr;
  unsigned long long* fcnt = nullptr;
  double* fmas = nullptr;
  long long fcap = 0;
};

namespace {

size_t elem_size(const mm_grid* g) { return g->prec == MM_FP64 ? sizeof(double) : sizeof(float); }

void drop_graphs(mm_grid* g) {
  for (int p = 0; p < 2; ++p) {
    if (g->gexec[p]) cudaGraphExecDestroy(g->gexec[p]);
    g->gexec[p] = nullptr;
  }
}

void free_state(mm_grid* g) {
  drop_graphs(g);  // they hold the state's addresses
  for (int i = 0; i < 2; ++i) {
    cudaFree(g->U[i]);
    cudaFree(g->E[i]);
    g->U[i] = nullptr;
    g->E[i] = nullptr;
  }
  delete g->tma;  // maps of the freed buffers
  g->tma = nullptr;
  cudaFree(g->prim);
  cudaFree(g->phi0);
  g->prim = nullptr;
  g->phi0 = nullptr;
  g->ready = false;
}

cudaError_t go(mm_grid* g, int what, int axis, int flag, const KArgs& a, double* out = nullptr,
               int nblocks = 0) {
  g->launches += (what == 5) ? 2 : 1;
  typedef cudaError_t (*launcher)(int, int, int, const KArgs&, double*, int, cudaStream_t);
  static const launcher table[2][2][3] = {
      {{mm_p64_d1, mm_p64_d2, mm_p64_d3}, {mm_p32_d1, mm_p32_d2, mm_p32_d3}},
      {{mm_p64_d1_void, mm_p64_d2_void, mm_p64_d3_void},
       {mm_p32_d1_void, mm_p32_d2_void, mm_p32_d3_void}}};
  return table[a.void_l >= 0 ? 1 : 0][g->prec == MM_FP64 ? 0 : 1][g->dim - 1](
      what, axis, flag, a, out, nblocks, g->stream);
}

mm_status check_device_error(mm_grid* g, const char* where) {
  DevErr e;
  cudaError_t ce = cudaMemcpyAsync(&e, g->err, sizeof e, cudaMemcpyDeviceToHost, g->stream);
  if (ce == cudaSuccess) ce = cudaStreamSynchronize(g->stream);
  if (ce != cudaSuccess) return fail(MM_ECUDA, "%s: %s", where, cudaGetErrorString(ce));
  if (e.code != 0) {
    cudaMemsetAsync(g->err, 0, sizeof(DevErr), g->stream);
    const char* what = e.code == MM_ENONFINITE ? "inadmissible state"
                       : e.code == MM_ENOCONV  ? "plastic return did not converge"
                       : e.code == MM_EDT      ? "non-positive time step"
                       : e.code == MM_ETIMEOUT ? "a bounded wait in a kernel gave up"
                                               : "device error";
    return fail((mm_status)e.code, "%s: %s at cell %lld, step %lld", where, what, e.cell, e.step);
  }
  return MM_OK;
}

// Start / stop the timing of one launch of the given kind (G: a grid or a
// batch, both carrying the same timing fields).
template <class G>
void prof_begin(G* g, int kind) {
  if (!g->prof) return;
  const size_t i = g->ev_kind.size();
  while (g->ev.size() < 2 * (i + 1)) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    g->ev.push_back(e);
  }
  g->ev_kind.push_back(kind);
  cudaEventRecord(g->ev[2 * i], g->stream);
}

template <class G>
void prof_end(G* g) {
  if (!g->prof) return;
  cudaEventRecord(g->ev[2 * (g->ev_kind.size() - 1) + 1], g->stream);
}

// After a stream synchronisation: accumulate the recorded pairs.
template <class G>
void prof_collect(G* g) {
  if (!g->prof) return;
  for (size_t i = 0; i < g->ev_kind.size(); ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, g->ev[2 * i], g->ev[2 * i + 1]) == cudaSuccess) {
      g->prof_ms[g->ev_kind[i]] += ms;
      g->prof_n[g->ev_kind[i]] += 1;
    }
  }
  g->ev_kind.clear();
}

KArgs args_for(mm_grid* g) {
  KArgs a = g->base;
  a.Uin = g->U[g->cur];
  a.Uout = g->U[g->cur];
  a.Ein = g->E[g->cur];
  a.Eout = g->E[g->cur];
  a.tma = g->tma_on ? g->tma : nullptr;
  return a;
}

}  // namespace

extern "C" {

const char* mm_last_error(void) { return g_error.c_str(); }

mm_status mm_create_grid(const mm_grid_desc* desc, void* cuda_stream, mm_grid** out) {
  if (!desc || !out) return fail(MM_EINVAL, "mm_create_grid: null argument");
  *out = nullptr;
  if (desc->dim < 1 || desc->dim > 3) return fail(MM_EINVAL, "dim must be 1, 2 or 3");
  if (desc->n_materials < 1 || desc->n_materials > MM_MAXMAT)
    return fail(MM_EINVAL, "n_materials must be 1..%d", MM_MAXMAT);
  if (desc->precision != MM_FP64 && desc->precision != MM_FP32_SPLIT)
    return fail(MM_EINVAL, "precision must be MM_FP64 or MM_FP32_SPLIT");
  long long ncell = 1;
  for (int k = 0; k < desc->dim; ++k) {
    if (desc->n[k] < 2 || desc->n[k] > (1 << 24)) return fail(MM_EINVAL, "n[%d] out of range", k);
    if (!(desc->hi[k] > desc->lo[k])) return fail(MM_EINVAL, "hi[%d] must exceed lo[%d]", k, k);
    for (int s = 0; s < 2; ++s)
      if (desc->bc[k][s] < 0 || desc->bc[k][s] > 2) return fail(MM_EINVAL, "bad boundary kind");
    if ((desc->bc[k][0] == MM_BC_PERIODIC) != (desc->bc[k][1] == MM_BC_PERIODIC))
      return fail(MM_EINVAL, "periodic boundaries must be set on both sides");
    ncell *= desc->n[k];
  }
  if (ncell > (1LL << 31)) return fail(MM_EINVAL, "too many cells");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1)
    return fail(MM_ECUDA, "no CUDA device available");
  mm_grid* g = new mm_grid();
  g->desc = *desc;
  g->dim = desc->dim;
  g->nmat = desc->n_materials;
  g->prec = desc->precision;
  g->ncell = ncell;
  if (cuda_stream) {
    g->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete g;
      return fail(MM_ECUDA, "cudaStreamCreate failed");
    }
    g->own_stream = true;
  }
  // totals: at least 8 cells per thread, at most 1024 blocks of 256.  Each
  // warp's FP64 reduction of the N + 4 sums costs about as much as a thread
  // accumulating 8 cells on this part's narrow FP64 pipe, so one cell per
  // thread (1024 blocks on a 512^2 grid) spent most of the time reducing.
  {
    long long nb = ncell / (256LL * 8);
    g->tot_blocks = (int)(nb < 1 ? 1 : (nb > 1024 ? 1024 : nb));
  }
  if (cudaMalloc(&g->info, sizeof(DevInfo)) != cudaSuccess ||
      cudaMalloc(&g->err, sizeof(DevErr)) != cudaSuccess ||
      cudaMalloc(&g->partial, sizeof(double) * g->tot_blocks * (MM_MAXMAT + 4)) != cudaSuccess ||
      cudaMalloc(&g->tot, sizeof(double) * (MM_MAXMAT + 4)) != cudaSuccess) {
    mm_destroy(g);
    return fail(MM_ENOMEM, "device allocation failed");
  }
  cudaMemsetAsync(g->info, 0, sizeof(DevInfo), g->stream);
  cudaMemsetAsync(g->err, 0, sizeof(DevErr), g->stream);
  KArgs& a = g->base;
  memset(&a, 0, sizeof a);
  a.void_l = -1;
  a.dim = g->dim;
  a.nmat = g->nmat;
  a.ncell = ncell;
  a.dxmin = 1e300;
  for (int k = 0; k < 3; ++k) {
    a.n[k] = k < g->dim ? (int)desc->n[k] : 1;
    a.lo[k] = k < g->dim ? desc->lo[k] : 0.0;
    a.hi[k] = k < g->dim ? desc->hi[k] : 1.0;
    a.dx[k] = (a.hi[k] - a.lo[k]) / a.n[k];
    a.bc[k][0] = k < g->dim ? desc->bc[k][0] : 0;
    a.bc[k][1] = k < g->dim ? desc->bc[k][1] : 0;
    if (k < g->dim && a.dx[k] < a.dxmin) a.dxmin = a.dx[k];
  }
  a.info = g->info;
  a.err = g->err;
  a.partial = g->partial;
  *out = g;
  return MM_OK;
}

mm_status mm_set_materials(mm_grid* g, const mm_material* mats, int n, const mm_init* init) {
  if (!g || !mats || !init || !init->prim) return fail(MM_EINVAL, "mm_set_materials: null argument");
  if (n != g->nmat) return fail(MM_EINVAL, "expected %d materials, got %d", g->nmat, n);
  int nhist = 0, void_l = -1;
  int hslot[MM_MAXMAT] = {-1, -1, -1};
  MatK mk[MM_MAXMAT];
  memset(mk, 0, sizeof mk);
  for (int l = 0; l < n; ++l) {
    const mm_material& m = mats[l];
    if (m.eos != MM_EOS_IDEAL_GAS && m.eos != MM_EOS_ROMENSKII && m.eos != MM_EOS_VOID)
      return fail(MM_EINVAL, "material %d: unknown eos", l);
    if (m.eos == MM_EOS_VOID) {
      if (void_l >= 0 || l == n - 1 || m.plasticity != MM_PL_NONE || m.damage != MM_DMG_NONE)
        return fail(MM_EINVAL,
                    "material %d: one void at most, not the last material, without plasticity "
                    "or damage", l);
      void_l = l;
    }
    if (m.eos == MM_EOS_IDEAL_GAS && !(m.gamma_gas > 1.0))
      return fail(MM_EINVAL, "material %d: gamma_gas must exceed 1", l);
    if (m.eos == MM_EOS_ROMENSKII &&
        !(m.rho0 > 0 && m.K0 > 0 && m.G0 >= 0 && m.alpha > 0 && m.Gamma0 > 0))
      return fail(MM_EINVAL, "material %d: Romenskii parameters out of range", l);
    if (m.shear_model != MM_SHEAR_ROMENSKII && m.shear_model != MM_SHEAR_STEINBERG)
      return fail(MM_EINVAL, "material %d: unknown shear model", l);
    if (m.shear_model == MM_SHEAR_STEINBERG &&
        !(m.eos == MM_EOS_ROMENSKII && m.Gp >= 0 && m.gamma_s > 0 &&
          m.Gamma0 + m.Gamma1 + m.Gamma2 > 0 && m.Gamma0 > 0 && m.Gamma1 >= 0 && m.Gamma2 >= 0))
      return fail(MM_EINVAL,
                  "material %d: the Steinberg model takes a Romenskii solid, Gp >= 0, "
                  "Gamma0 > 0, Gamma1, Gamma2 >= 0, gamma_s > 0", l);
    if (m.plasticity != MM_PL_NONE && m.plasticity != MM_PL_JOHNSON_COOK)
      return fail(MM_EINVAL, "material %d: unknown plasticity model", l);
    if (m.plasticity == MM_PL_JOHNSON_COOK && !(m.c1 >= 0 && m.c2 >= 0 && m.edot0 > 0))
      return fail(MM_EINVAL, "material %d: Johnson-Cook parameters out of range", l);
    if (m.damage != MM_DMG_NONE && m.damage != MM_DMG_BONORA && m.damage != MM_DMG_SIMPLE)
      return fail(MM_EINVAL, "material %d: unknown damage model", l);
    if (m.damage != MM_DMG_NONE && m.plasticity != MM_PL_JOHNSON_COOK)
      return fail(MM_EINVAL, "material %d: damage needs a plasticity model", l);
    if (m.damage == MM_DMG_BONORA &&
        !(m.D_crit > 0 && m.D_crit < 1 && m.eps_c > m.eps_t && m.eps_t > 0 && m.alpha_D > 0 &&
          m.n_hard > 0))
      return fail(MM_EINVAL, "material %d: Bonora parameters out of range", l);
    if (m.damage == MM_DMG_SIMPLE && !(m.D_crit > 0 && m.D_crit < 1))
      return fail(MM_EINVAL, "material %d: D_crit out of range", l);
    MatK& k = mk[l];
    k.eos = m.eos;
    k.plasticity = m.plasticity;
    k.damage = m.damage;
    k.shear_model = m.eos == MM_EOS_ROMENSKII ? m.shear_model : MM_SHEAR_ROMENSKII;
    k.Gp = m.Gp;
    k.Gamma1 = m.Gamma1;
    k.Gamma2 = m.Gamma2;
    k.gamma_s = m.gamma_s;
    k.rho0 = m.rho0;
    k.K0 = m.K0;
    k.G0 = m.G0;
    k.alpha = m.alpha;
    k.beta = m.beta;
    k.Gamma0 = m.Gamma0;
    k.gamma_gas = m.gamma_gas;
    k.c1 = m.c1;
    k.c2 = m.c2;
    k.c3 = m.c3;
    k.n_hard = m.n_hard;
    k.edot0 = m.edot0;
    k.D_crit = m.D_crit;
    k.D_cut = m.D_crit * (1.0 - 1e-4);
    k.eps_t = m.eps_t;
    k.eps_c = m.eps_c;
    k.alpha_D = m.alpha_D;
    k.poisson = m.poisson;
    k.Ddot0 = m.Ddot0;
    k.Gamma = m.eos == MM_EOS_IDEAL_GAS ? m.gamma_gas - 1.0
              : m.eos == MM_EOS_VOID     ? 1.0
                                         : m.Gamma0;
    k.xi = m.eos == MM_EOS_VOID ? 0.0 : 1.0 / k.Gamma;
    if (m.damage == MM_DMG_BONORA) {
      k.bon_k = m.alpha_D * pow(m.D_crit, 1.0 / m.alpha_D) / log(m.eps_c / m.eps_t);
      k.bon_ec2n = pow(m.eps_c, 2.0 * m.n_hard);
      k.bon_et2n = pow(m.eps_t, 2.0 * m.n_hard);
    }
    if (m.plasticity == MM_PL_JOHNSON_COOK) hslot[l] = nhist++;
  }
  if (nhist > 2) return fail(MM_EINVAL, "at most two plastic materials are supported");
  if (nhist == 2 && (g->dim > 2 || void_l >= 0))
    return fail(MM_EINVAL, "two plastic materials are supported on 1D and 2D grids without void");
  if (void_l >= 0 && nhist != 1)
    return fail(MM_EINVAL, "a grid with void needs exactly one plastic material");
  if (n == 3 && void_l < 0 && nhist != 2)
    return fail(MM_EINVAL,
                "three materials are supported with one of them void, or with two plastic "
                "solids (1D, 2D)");
  const int nF = g->dim == 1 ? 3 : (g->dim == 2 ? 5 : 9);
  const int nfield = (g->nmat - 1) + g->nmat + g->dim + 1 + nF + 2 * nhist + g->dim;
  if (init->phi0) {
    long long np = 1;
    for (int k = 0; k < g->dim; ++k) {
      if (init->phi0_n[k] < 2 || !(init->phi0_h[k] > 0))
        return fail(MM_EINVAL, "perturbation lattice needs >= 2 points and h > 0 per axis");
      if (init->phi0_n[k] > 0x7fffffffLL / np)
        return fail(MM_EINVAL, "perturbation lattice exceeds 2^31 - 1 points");
      np *= init->phi0_n[k];
    }
  }
  free_state(g);
  g->nhist = nhist;
  g->nfield = nfield;
  const size_t es = elem_size(g);
  // FP32-split: one more float field (the last volume fraction is carried,
  // not formed as 1 - sum) and rho E in an FP64 side array
  const size_t nstore = g->prec == MM_FP32_SPLIT ? nfield + 1 : nfield;
  for (int i = 0; i < 2; ++i) {
    if (cudaMalloc(&g->U[i], es * nstore * g->ncell) != cudaSuccess) {
      free_state(g);
      return fail(MM_ENOMEM, "device allocation of the state failed");
    }
    if (g->prec == MM_FP32_SPLIT &&
        cudaMalloc(&g->E[i], sizeof(double) * g->ncell) != cudaSuccess) {
      free_state(g);
      return fail(MM_ENOMEM, "device allocation of the state failed");
    }
  }
  if (cudaMalloc(&g->prim, sizeof(double) * nfield * g->ncell) != cudaSuccess) {
    free_state(g);
    return fail(MM_ENOMEM, "device allocation of the staging buffer failed");
  }
  if (g->prec == MM_FP32_SPLIT && g->dim == 3 && void_l < 0) {
    // maps for the TMA-staged y and z sweeps, where they describe the grid
    SweepTmaSet t;
    const int n3[3] = {(int)g->desc.n[0], (int)g->desc.n[1], (int)g->desc.n[2]};
    if (mm_p32_d3_tma_encode(&t, g->U, g->E, n3, g->nmat, nhist)) g->tma = new SweepTmaSet(t);
  }
  KArgs& a = g->base;
  a.nhist = nhist;
  a.nfield = nfield;
  a.void_l = void_l;
  if (void_l >= 0 && !g->xseed &&
      cudaMalloc(&g->xseed, elem_size(g) * (size_t)g->dim * g->ncell) != cudaSuccess) {
    g->xseed = nullptr;
    return fail(MM_ENOMEM, "device allocation of the seeding scratch failed");
  }
  a.xseed = g->xseed;
  for (int l = 0; l < MM_MAXMAT; ++l) {
    const MatK& k = mk[l];
    a.mat[l] = k;
    a.hslot[l] = hslot[l];
    MatKf& f = a.matf[l];
    f.eos = k.eos;
    f.plasticity = k.plasticity;
    f.damage = k.damage;
    f.alpha_one = k.alpha == 1.0;
    f.rho0 = float(k.rho0);
    f.K0 = float(k.K0);
    f.G0 = float(k.G0);
    f.alpha = float(k.alpha);
    f.beta = float(k.beta);
    f.Gamma0 = float(k.Gamma0);
    f.gamma_gas = float(k.gamma_gas);
    f.c1 = float(k.c1);
    f.c2 = float(k.c2);
    f.c3 = float(k.c3);
    f.n_hard = float(k.n_hard);
    f.edot0 = float(k.edot0);
    f.D_crit = float(k.D_crit);
    f.D_cut = float(k.D_cut);
    f.shear_model = k.shear_model;
    f.Gp = float(k.Gp);
    f.Gamma1 = float(k.Gamma1);
    f.Gamma2 = float(k.Gamma2);
    f.gamma_s = float(k.gamma_s);
    f.eps_t = float(k.eps_t);
    f.eps_c = float(k.eps_c);
    f.alpha_D = float(k.alpha_D);
    f.poisson = float(k.poisson);
    f.Ddot0 = float(k.Ddot0);
    f.xi = float(k.xi);
    f.Gamma = float(k.Gamma);
    f.bon_k = float(k.bon_k);
    f.bon_ec2n = float(k.bon_ec2n);
    f.bon_et2n = float(k.bon_et2n);
    f.inv_rho0 = k.rho0 > 0 ? float(1.0 / k.rho0) : 0.f;
    f.K0_2a2 = k.alpha > 0 ? float(k.K0 / (2.0 * k.alpha * k.alpha)) : 0.f;
    f.K0_arho0 = k.alpha > 0 && k.rho0 > 0 ? float(k.K0 / (k.alpha * k.rho0)) : 0.f;
    f.c2n = float(k.c2 * k.n_hard);
  }
  a.prim = g->prim;
  a.phi0 = nullptr;
  if (init->phi0) {
    long long np = 1;
    for (int k = 0; k < g->dim; ++k) {
      a.pn[k] = (int)init->phi0_n[k];
      a.plo[k] = init->phi0_lo[k];
      a.ph[k] = init->phi0_h[k];
      a.plof[k] = float(init->phi0_lo[k]);
      a.phf[k] = float(init->phi0_h[k]);
      np *= init->phi0_n[k];
    }
    if (cudaMalloc(&g->phi0, sizeof(float) * np) != cudaSuccess) {
      free_state(g);
      return fail(MM_ENOMEM, "device allocation of the lattice failed");
    }
    CUDA_TRY(cudaMemcpyAsync(g->phi0, init->phi0, sizeof(float) * np, cudaMemcpyHostToDevice,
                             g->stream));
    a.phi0 = g->phi0;
  }
  CUDA_TRY(cudaMemcpyAsync(g->prim, init->prim, sizeof(double) * nfield * g->ncell,
                           cudaMemcpyHostToDevice, g->stream));
  CUDA_TRY(cudaMemsetAsync(g->info, 0, sizeof(DevInfo), g->stream));
  CUDA_TRY(cudaMemsetAsync(g->err, 0, sizeof(DevErr), g->stream));
  g->cur = 0;
  KArgs b = args_for(g);
  CUDA_TRY(go(g, 0, 0, 0, b));
  mm_status st = check_device_error(g, "mm_set_materials");
  if (st != MM_OK) return st;
  g->ready = true;
  return MM_OK;
}

namespace {

mm_status step_args(mm_grid* g, int n_steps, double cfl, const char* who) {
  if (!g) return fail(MM_EINVAL, "%s: null grid", who);
  if (!g->ready) return fail(MM_ESTATE, "%s before mm_set_materials", who);
  if (n_steps < 0) return fail(MM_EINVAL, "n_steps must be >= 0");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return fail(MM_EINVAL, "cfl must be in (0, 1]");
  return MM_OK;
}

// Enqueue one step on the grid's stream: CFL reduction, dt, the split
// sweeps, the sources.  dt stays on the device.
mm_status enqueue_one(mm_grid* g, double cfl) {
  {
    KArgs a = args_for(g);
    a.cfl = cfl;
    if (a.void_l >= 0 && g->seed_x) {
      // Lagrangian seeding into void from the step's start (all cells read
      // the old X; the new X are copied over after every cell is done)
      prof_begin(g, MM_K_XTRANSPORT);
      CUDA_TRY(go(g, 9, 0, 0, a));
      const size_t es = elem_size(g);
      CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(g->U[g->cur]) + es * (size_t)(g->nfield - g->dim) * g->ncell,
                               g->xseed, es * (size_t)g->dim * g->ncell, cudaMemcpyDeviceToDevice,
                               g->stream));
      prof_end(g);
    }
    // the CFL reduction's last CTA also forms dt (no separate launch)
    prof_begin(g, MM_K_CFL);
    CUDA_TRY(go(g, 2, 0, 0, a));
    prof_end(g);
    if (g->xscheme == MM_X_WENO3_RK3) {
      // X of the step's end from its start (the state the sweeps read)
      prof_begin(g, MM_K_XTRANSPORT);
      CUDA_TRY(go(g, 6, 0, 0, a));
      for (int st = 1; st <= 3; ++st) CUDA_TRY(go(g, 7, 0, st, a));
      prof_end(g);
    }
    for (int d = 0; d < g->dim; ++d) {
      KArgs b = args_for(g);
      b.Uout = g->U[1 - g->cur];
      b.Eout = g->E[1 - g->cur];
      prof_begin(g, MM_K_SWEEP_X + d);
      CUDA_TRY(go(g, 3, d, 0, b));
      prof_end(g);
      g->cur = 1 - g->cur;
    }
    if (g->xscheme == MM_X_WENO3_RK3) {
      // the sweeps' X is replaced (X are the last dim fields of the layout)
      const size_t es = elem_size(g);
      prof_begin(g, MM_K_XTRANSPORT);
      CUDA_TRY(cudaMemcpyAsync(static_cast<char*>(g->U[g->cur]) + es * (size_t)(g->nfield - g->dim) * g->ncell,
                               g->xs[1], es * (size_t)g->dim * g->ncell, cudaMemcpyDeviceToDevice,
                               g->stream));
      prof_end(g);
    }
    KArgs c = args_for(g);
    prof_begin(g, MM_K_SOURCES);
    CUDA_TRY(go(g, 4, 0, 0, c));
    prof_end(g);
  }
  return MM_OK;
}

// Enqueue n_steps steps.  The first step after the state is set runs
// launch by launch; later ones replay a captured step (not while kernel
// timing is on, which times each launch).
mm_status enqueue_steps(mm_grid* g, int n_steps, double cfl) {
  g->launches = 0;
  for (int s = 0; s < n_steps; ++s) {
    if (g->prof || !g->gwarm || g->nograph) {
      mm_status st = enqueue_one(g, cfl);
      if (st != MM_OK) return st;
      g->gwarm = true;
      continue;
    }
    const int p = g->cur;
    if (!g->gexec[p] || g->gcfl[p] != cfl) {
      if (g->gexec[p]) cudaGraphExecDestroy(g->gexec[p]);
      g->gexec[p] = nullptr;
      if (cudaStreamBeginCapture(g->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        g->nograph = true;
        --s;
        continue;
      }
      const long long l0 = g->launches;
      mm_status st = enqueue_one(g, cfl);
      cudaGraph_t graph = nullptr;
      cudaError_t e = cudaStreamEndCapture(g->stream, &graph);
      g->cur = p;  // the capture advanced the buffers; the launch below does it
      g->glaunches = g->launches - l0;
      g->launches = l0;
      if (st != MM_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return st != MM_OK ? st : fail(MM_ECUDA, "step capture: %s", cudaGetErrorString(e));
      }
      e = cudaGraphInstantiate(&g->gexec[p], graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) {
        g->gexec[p] = nullptr;
        return fail(MM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
      }
      g->gcfl[p] = cfl;
    }
    CUDA_TRY(cudaGraphLaunch(g->gexec[p], g->stream));
    g->launches += g->glaunches;
    if (g->dim & 1) g->cur ^= 1;
  }
  return MM_OK;
}

// Synchronise, report a latched device failure, fill info.
mm_status finish_steps(mm_grid* g, const char* who, mm_step_info* info) {
  mm_status st = check_device_error(g, who);
  prof_collect(g);
  if (info) {
    DevInfo h;
    CUDA_TRY(cudaMemcpy(&h, g->info, sizeof h, cudaMemcpyDeviceToHost));
    info->t = h.t;
    info->dt_last = h.dt;
    info->smax = h.smax;
    info->steps_done = h.steps;
    info->bad_cell = -1;
    if (st != MM_OK) {
      // the message carries the cell; keep the struct consistent
      const char* m = g_error.c_str();
      const char* p = strstr(m, "cell ");
      if (p) info->bad_cell = atoll(p + 5);
    }
  }
  return st;
}

}  // namespace

mm_status mm_step(mm_grid* g, int n_steps, double cfl, mm_step_info* info) {
  mm_status st = step_args(g, n_steps, cfl, "mm_step");
  if (st != MM_OK) return st;
  st = enqueue_steps(g, n_steps, cfl);
  if (st != MM_OK) return st;
  return finish_steps(g, "mm_step", info);
}

mm_status mm_step_async(mm_grid* g, int n_steps, double cfl) {
  mm_status st = step_args(g, n_steps, cfl, "mm_step_async");
  if (st != MM_OK) return st;
  return enqueue_steps(g, n_steps, cfl);
}

mm_status mm_synchronize(mm_grid* g, mm_step_info* info) {
  if (!g) return fail(MM_EINVAL, "mm_synchronize: null grid");
  if (!g->ready) return fail(MM_ESTATE, "mm_synchronize before mm_set_materials");
  return finish_steps(g, "mm_synchronize", info);
}

mm_status mm_read_fields(mm_grid* g, uint64_t field_mask, int primitive, double* host_dst,
                         size_t dst_len) {
  if (!g || !host_dst) return fail(MM_EINVAL, "mm_read_fields: null argument");
  if (!g->ready) return fail(MM_ESTATE, "mm_read_fields before mm_set_materials");
  int nsel = 0;
  for (int f = 0; f < g->nfield; ++f)
    if (field_mask >> f & 1ull) ++nsel;
  if ((size_t)nsel * (size_t)g->ncell > dst_len)
    return fail(MM_EINVAL, "destination holds %zu doubles, need %lld", dst_len,
                (long long)nsel * g->ncell);
  KArgs a = args_for(g);
  CUDA_TRY(go(g, 1, 0, primitive ? 1 : 0, a));
  int o = 0;
  for (int f = 0; f < g->nfield; ++f) {
    if (!(field_mask >> f & 1ull)) continue;
    CUDA_TRY(cudaMemcpyAsync(host_dst + (size_t)o * g->ncell, g->prim + (size_t)f * g->ncell,
                             sizeof(double) * g->ncell, cudaMemcpyDeviceToHost, g->stream));
    ++o;
  }
  return check_device_error(g, "mm_read_fields");
}

mm_status mm_conserved_totals(mm_grid* g, double* out, size_t out_len) {
  if (!g || !out) return fail(MM_EINVAL, "mm_conserved_totals: null argument");
  if (!g->ready) return fail(MM_ESTATE, "mm_conserved_totals before mm_set_materials");
  if (out_len < (size_t)g->nmat + 4) return fail(MM_EINVAL, "out_len must be >= %d", g->nmat + 4);
  KArgs a = args_for(g);
  CUDA_TRY(go(g, 5, 0, 0, a, g->tot, g->tot_blocks));
  CUDA_TRY(cudaMemcpyAsync(out, g->tot, sizeof(double) * (g->nmat + 4), cudaMemcpyDeviceToHost,
                           g->stream));
  CUDA_TRY(cudaStreamSynchronize(g->stream));
  return MM_OK;
}

int mm_num_fields(const mm_grid* g) { return g ? g->nfield : 0; }
int64_t mm_num_cells(const mm_grid* g) { return g ? g->ncell : 0; }
int64_t mm_kernel_launches(const mm_grid* g) { return g ? g->launches : 0; }

mm_status mm_profile_enable(mm_grid* g, int enable) {
  if (!g) return fail(MM_EINVAL, "mm_profile_enable: null grid");
  g->prof = enable != 0;
  return MM_OK;
}

mm_status mm_profile_read(mm_grid* g, double* ms, int64_t* counts, int n, int reset) {
  if (!g || n < 0) return fail(MM_EINVAL, "mm_profile_read: bad argument");
  for (int k = 0; k < n && k < MM_K_COUNT; ++k) {
    if (ms) ms[k] = g->prof_ms[k];
    if (counts) counts[k] = g->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < MM_K_COUNT; ++k) {
      g->prof_ms[k] = 0.0;
      g->prof_n[k] = 0;
    }
  return MM_OK;
}

mm_status mm_set_lagrangian_seeding(mm_grid* g, int on) {
  if (!g) return fail(MM_EINVAL, "mm_set_lagrangian_seeding: null grid");
  if (on != 0 && on != 1) return fail(MM_EINVAL, "mm_set_lagrangian_seeding: on must be 0 or 1");
  g->seed_x = on != 0;
  drop_graphs(g);
  return MM_OK;
}

mm_status mm_set_tma_loads(mm_grid* g, int on, int* active) {
  if (!g) return fail(MM_EINVAL, "mm_set_tma_loads: null grid");
  if (on < -1 || on > 1) return fail(MM_EINVAL, "mm_set_tma_loads: on must be -1, 0 or 1");
  if (on >= 0 && g->tma_on != (on != 0)) {
    g->tma_on = on != 0;
    drop_graphs(g);  // they hold the launches of the other kernels
  }
  if (active) *active = g->tma_on && g->tma ? 1 : 0;
  return MM_OK;
}

mm_status mm_set_x_transport(mm_grid* g, int scheme) {
  if (!g) return fail(MM_EINVAL, "mm_set_x_transport: null grid");
  if (scheme != MM_X_SWEEP && scheme != MM_X_WENO3_RK3)
    return fail(MM_EINVAL, "mm_set_x_transport: unknown scheme %d", scheme);
  if (scheme == MM_X_WENO3_RK3 && g->ncell >= (1ll << 31))
    return fail(MM_EINVAL, "mm_set_x_transport: WENO3 + RK3 takes grids of fewer than 2^31 cells");
  if (scheme == MM_X_WENO3_RK3 && !g->xs[0]) {
    const size_t bytes = elem_size(g) * (size_t)g->dim * g->ncell;
    for (int i = 0; i < 3; ++i) {
      if (cudaMalloc(&g->xs[i], bytes) != cudaSuccess) {
        for (int j = 0; j <= i; ++j) {
          cudaFree(g->xs[j]);
          g->xs[j] = nullptr;
        }
        return fail(MM_ENOMEM, "device allocation of the X scratch failed");
      }
    }
    for (int i = 0; i < 3; ++i) g->base.xs[i] = g->xs[i];
  }
  g->xscheme = scheme;
  drop_graphs(g);
  return MM_OK;
}

mm_status mm_fragments(mm_grid* g, double theta, int64_t* labels, size_t labels_len,
                       mm_fragment* frags, size_t max_frags, int64_t* n_frags) {
  if (!g || !n_frags) return fail(MM_EINVAL, "mm_fragments: null argument");
  if (!(theta > 0.0 && theta <= 1.0))
    return fail(MM_EINVAL, "mm_fragments: the cut-off must lie in (0, 1], got %g", theta);
  if (!g->ready) return fail(MM_ESTATE, "mm_fragments before mm_set_materials");
  if (labels && labels_len != (size_t)g->ncell)
    return fail(MM_EINVAL, "mm_fragments: labels holds %zu entries, the grid %lld cells",
                labels_len, g->ncell);
  if (max_frags > 0 && !frags) return fail(MM_EINVAL, "mm_fragments: null fragment array");
  if (g->ncell >= (1ll << 31))
    return fail(MM_EINVAL, "mm_fragments takes grids of fewer than 2^31 cells");
  const long long nblk = (g->ncell + MM_FRAG_CELLS - 1) / MM_FRAG_CELLS;
  if (!g->fparent) {
    const size_t n = (size_t)g->ncell;
    if (cudaMalloc(&g->fparent, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&g->ffid, sizeof(int) * n) != cudaSuccess ||
        cudaMalloc(&g->fcm, sizeof(double) * n) != cudaSuccess ||
        cudaMalloc(&g->fboff, sizeof(int) * (size_t)(nblk + 1)) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(g->fparent);
      cudaFree(g->ffid);
      cudaFree(g->fcm);
      cudaFree(g->fboff);
      g->fparent = g->ffid = g->fboff = nullptr;
      g->fcm = nullptr;
      return fail(MM_ENOMEM, "device allocation of the fragment scratch failed");
    }
  }
  KArgs a = args_for(g);
  a.frag = g->fparent;
  a.fmass = g->fcm;
  a.fcut = theta;
  a.fthr = 1.0 - theta;
  a.fthrf = (float)a.fthr;
  if ((double)a.fthrf > a.fthr) a.fthrf = std::nextafter(a.fthrf, -1.0f);
  a.fdV = 1.0;
  for (int k = 0; k < g->dim; ++k) a.fdV *= a.dx[k];
  for (int l = 0; l < MM_MAXMAT; ++l) {
    a.fdcrit[l] = l < g->nmat ? a.mat[l].D_cut : 0.0;
    a.fdcritf[l] = l < g->nmat ? a.matf[l].D_cut : 0.0f;
  }
  a.fpad = 0.0f;
  prof_begin(g, MM_K_FRAG_MARK);
  CUDA_TRY(go(g, 8, 0, 0, a));
  prof_end(g);
  prof_begin(g, MM_K_FRAG_UNION);
  CUDA_TRY(mm_frag_label(a, g->stream));
  prof_end(g);
  prof_begin(g, MM_K_FRAG_COUNT);
  CUDA_TRY(mm_frag_count(a, g->fboff, g->stream));
  prof_end(g);
  g->launches += 4;
  int nf = 0;
  CUDA_TRY(cudaMemcpyAsync(&nf, g->fboff + nblk, sizeof(int), cudaMemcpyDeviceToHost, g->stream));
  mm_status st = check_device_error(g, "mm_fragments");
  if (st != MM_OK) return st;
  if (nf > g->fcap) {
    cudaFree(g->flab);
    cudaFree(g->fcnt);
    cudaFree(g->fmas);
    g->flab = nullptr;
    g->fcnt = nullptr;
    g->fmas = nullptr;
    g->fcap = 0;
    const long long cap = nf + nf / 4 + 64;
    if (cudaMalloc(&g->flab, sizeof(long long) * cap) != cudaSuccess ||
        cudaMalloc(&g->fcnt, sizeof(unsigned long long) * cap) != cudaSuccess ||
        cudaMalloc(&g->fmas, sizeof(double) * cap) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(g->flab);
      cudaFree(g->fcnt);
      cudaFree(g->fmas);
      g->flab = nullptr;
      g->fcnt = nullptr;
      g->fmas = nullptr;
      return fail(MM_ENOMEM, "device allocation of %d fragment records failed", nf);
    }
    g->fcap = cap;
  }
  if (nf > 0) {
    CUDA_TRY(cudaMemsetAsync(g->fcnt, 0, sizeof(unsigned long long) * nf, g->stream));
    CUDA_TRY(cudaMemsetAsync(g->fmas, 0, sizeof(double) * nf, g->stream));
    prof_begin(g, MM_K_FRAG_COLLECT);
    CUDA_TRY(mm_frag_collect(a, g->fboff, g->ffid, g->flab, g->fcnt, g->fmas, g->stream));
    prof_end(g);
    g->launches += 2;
  }
  const size_t k = max_frags < (size_t)nf ? max_frags : (size_t)nf;
  std::vector<long long> hl(k);
  std::vector<unsigned long long> hc(k);
  std::vector<double> hm(k);
  std::vector<int> hp(labels ? (size_t)g->ncell : 0);
  if (k > 0) {
    CUDA_TRY(cudaMemcpyAsync(hl.data(), g->flab, sizeof(long long) * k, cudaMemcpyDeviceToHost,
                             g->stream));
    CUDA_TRY(cudaMemcpyAsync(hc.data(), g->fcnt, sizeof(unsigned long long) * k,
                             cudaMemcpyDeviceToHost, g->stream));
    CUDA_TRY(cudaMemcpyAsync(hm.data(), g->fmas, sizeof(double) * k, cudaMemcpyDeviceToHost,
                             g->stream));
  }
  if (labels)
    CUDA_TRY(cudaMemcpyAsync(hp.data(), g->fparent, sizeof(int) * (size_t)g->ncell,
                             cudaMemcpyDeviceToHost, g->stream));
  st = check_device_error(g, "mm_fragments");
  if (st != MM_OK) return st;
  for (size_t i = 0; i < k; ++i) {
    frags[i].label = hl[i];
    frags[i].cells = (int64_t)hc[i];
    frags[i].mass = hm[i];
  }
  if (labels)
    for (long long c = 0; c < g->ncell; ++c) labels[c] = hp[(size_t)c];
  *n_frags = nf;
  prof_collect(g);
  return MM_OK;
}

mm_status mm_destroy(mm_grid* g) {
  if (!g) return MM_OK;
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  for (int i = 0; i < 3; ++i) cudaFree(g->xs[i]);
  cudaFree(g->xseed);
  cudaFree(g->fparent);
  cudaFree(g->ffid);
  cudaFree(g->fcm);
  cudaFree(g->fboff);
  cudaFree(g->flab);
  cudaFree(g->fcnt);
  cudaFree(g->fmas);
  free_state(g);
  cudaFree(g->info);
  cudaFree(g->err);
  cudaFree(g->partial);
  cudaFree(g->tot);
  if (g->own_stream && g->stream) cudaStreamDestroy(g->stream);
  delete g;
  return MM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ batches ----
// Several grids stepped together: one launch per kernel kind covers every
// member (persistent CTAs over the concatenated tiles or cell chunks), each
// member with its own dt; a step is captured in a CUDA graph and replayed.

namespace {

constexpr long long kChunk = 8192;  // cells per unit of the CFL and source launches
constexpr int kPhases = 5;          // CFL, sweeps x, y, z, sources

typedef cudaError_t (*batch_launcher)(int, int, int, int, int, const BatchK&, cudaStream_t);
typedef long long (*tiles_fn)(int, int, const int[3]);

batch_launcher batch_launch_of(int prec, int dim) {
  static const batch_launcher t[2][3] = {{mm_p64_d1_batch, mm_p64_d2_batch, mm_p64_d3_batch},
                                         {mm_p32_d1_batch, mm_p32_d2_batch, mm_p32_d3_batch}};
  return t[prec == MM_FP64 ? 0 : 1][dim - 1];
}

tiles_fn tiles_of(int prec, int dim) {
  static const tiles_fn t[2][3] = {
      {mm_p64_d1_batch_tiles, mm_p64_d2_batch_tiles, mm_p64_d3_batch_tiles},
      {mm_p32_d1_batch_tiles, mm_p32_d2_batch_tiles, mm_p32_d3_batch_tiles}};
  return t[prec == MM_FP64 ? 0 : 1][dim - 1];
}

KArgs args_at(const mm_grid* g, int c) {
  KArgs a = g->base;
  a.Uin = g->U[c];
  a.Uout = g->U[c];
  a.Ein = g->E[c];
  a.Eout = g->E[c];
  return a;
}

}  // namespace

struct mm_batch {
  std::vector<mm_grid*> m;
  int M = 0, dim = 0, prec = 0, nmat = 0, nhist = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  KArgs* args = nullptr;                  // [2 parities][kPhases][M] member arguments
  long long* tstart = nullptr;            // [3 axes][2 variants][M + 1] tile prefix
  long long* cstart = nullptr;            // [M + 1] chunk prefix
  unsigned long long* counter = nullptr;  // [8] work counters of one step
  std::vector<long long> h_tstart, h_cstart;
  int variant[3] = {0, 0, 0};
  int cps[3] = {0, 0, 0};  // persistent sweep CTAs per SM per axis (0: as many as fit)
  int cps_src = 0;         // the same for the source kernel
  // groups of members stepped one after another (each group's state sized
  // to stay in L2 between its launches): member index bounds, ngroups + 1
  std::vector<int> gstart;
  int parity = 0;  // flips with every sweep: the members' buffers relative to creation
  int use_graph = 1;
  bool warmed = false;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  double exec_cfl[2] = {0.0, 0.0};
  // kernel timing (steps are launched one kernel at a time while it is on)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;
  double prof_ms[MM_K_COUNT] = {};
  long long prof_n[MM_K_COUNT] = {};
};

namespace {

void batch_free(mm_batch* b) {
  for (int p = 0; p < 2; ++p)
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
  for (cudaEvent_t e : b->ev) cudaEventDestroy(e);
  cudaFree(b->args);
  cudaFree(b->tstart);
  cudaFree(b->cstart);
  cudaFree(b->counter);
  if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
  delete b;
}

void batch_drop_graphs(mm_batch* b) {
  for (int p = 0; p < 2; ++p) {
    if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
    b->exec[p] = nullptr;
  }
}

BatchK batch_k(const mm_batch* b, int phase, const long long* start, long long total) {
  BatchK k;
  k.args = b->args + ((size_t)b->parity * kPhases + phase) * b->M;
  k.start = start;
  k.counter = b->counter + phase;
  k.total = total;
  k.chunk = kChunk;
  k.M = b->M;
  k.cta_per_sm = 0;
  k.base = 0;
  return k;
}

// The same launch restricted to members [g0, g1) of group gi (its own work
// counter; unit numbers stay those of the whole batch).
BatchK batch_kg(const mm_batch* b, int phase, const long long* start, const long long* h_start,
                int g0, int g1, int gi) {
  BatchK k = batch_k(b, phase, start + g0, h_start[g1]);
  k.args += g0;
  k.counter = b->counter + 8 * gi + phase;
  k.base = h_start[g0];
  k.M = g1 - g0;
  return k;
}

// The launches of one step at the current parity (capturable).
cudaError_t batch_enqueue(mm_batch* b, double cfl) {
  batch_launcher L = batch_launch_of(b->prec, b->dim);
  const int M = b->M;
  const int G = (int)b->gstart.size() - 1;
  cudaError_t e = cudaMemsetAsync(b->counter, 0, 8 * sizeof(unsigned long long) * G, b->stream);
  if (e != cudaSuccess) return e;
  // one group after another: every launch of a step on a group's members
  // (whose state then stays in L2), members independent of one another
  for (int gi = 0; gi < G; ++gi) {
    const int g0 = b->gstart[gi], g1 = b->gstart[gi + 1];
    prof_begin(b, MM_K_CFL);
    e = L(0, 0, 0, b->nmat, b->nhist, batch_kg(b, 0, b->cstart, b->h_cstart.data(), g0, g1, gi),
          b->stream);
    prof_end(b);
    if (e != cudaSuccess) return e;
    prof_begin(b, MM_K_DT);
    k_dt_batch<<<(g1 - g0 + 127) / 128, 128, 0, b->stream>>>(
        b->args + (size_t)b->parity * kPhases * M + g0, g1 - g0, cfl);
    prof_end(b);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    for (int d = 0; d < b->dim; ++d) {
      const int v = b->variant[d];
      const size_t o = (size_t)(d * 2 + v) * (M + 1);
      prof_begin(b, MM_K_SWEEP_X + d);
      BatchK k = batch_kg(b, 1 + d, b->tstart + o, b->h_tstart.data() + o, g0, g1, gi);
      k.cta_per_sm = b->cps[d];
      e = L(1, d, v, b->nmat, b->nhist, k, b->stream);
      prof_end(b);
      if (e != cudaSuccess) return e;
    }
    prof_begin(b, MM_K_SOURCES);
    BatchK ks = batch_kg(b, 4, b->cstart, b->h_cstart.data(), g0, g1, gi);
    ks.cta_per_sm = b->cps_src;
    e = L(2, 0, 0, b->nmat, b->nhist, ks, b->stream);
    prof_end(b);
    if (e != cudaSuccess) return e;
  }
  return e;
}

// Greedy groups of consecutive members whose state copies (both buffers)
// sum to at most `bytes` each (a larger member is a group of its own);
// bytes <= 0: one group of every member.
void batch_group(mm_batch* b, long long bytes) {
  b->gstart.assign(1, 0);
  long long acc = 0;
  for (int i = 0; i < b->M; ++i) {
    const mm_grid* g = b->m[i];
    const long long mb = 2 * (long long)(elem_size(g) * (size_t)(g->nfield + 1) * g->ncell +
                                         (g->prec == MM_FP64 ? 0 : sizeof(double) * g->ncell));
    if (bytes > 0 && i > b->gstart.back() && acc + mb > bytes) {
      b->gstart.push_back(i);
      acc = 0;
    }
    acc += mb;
  }
  b->gstart.push_back(b->M);
}

// Default group budget: 60 % of the device's L2 cache.
long long default_group_bytes() {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess || l2 <= 0)
    return 0;
  return (long long)l2 * 6 / 10;
}

void batch_advance(mm_batch* b) {
  if (b->dim & 1) {
    b->parity ^= 1;
    for (mm_grid* g : b->m) g->cur ^= 1;
  }
}

}  // namespace

mm_status mm_batch_create(mm_grid* const* grids, int n, void* cuda_stream, mm_batch** out) {
  if (!grids || !out || n < 1) return fail(MM_EINVAL, "mm_batch_create: null argument or n < 1");
  *out = nullptr;
  const mm_grid* g0 = grids[0];
  for (int i = 0; i < n; ++i) {
    const mm_grid* g = grids[i];
    if (!g) return fail(MM_EINVAL, "mm_batch_create: member %d is null", i);
    if (!g->ready) return fail(MM_ESTATE, "mm_batch_create: member %d has no materials", i);
    if (g->dim != g0->dim || g->prec != g0->prec || g->nmat != g0->nmat || g->nhist != g0->nhist)
      return fail(MM_EINVAL,
                  "mm_batch_create: member %d differs from member 0 in dimension, precision or "
                  "material layout", i);
    for (int j = 0; j < i; ++j)
      if (grids[j] == g) return fail(MM_EINVAL, "mm_batch_create: member %d repeats member %d", i, j);
  }
  if (g0->nmat != 2 || g0->nhist > 1)
    return fail(MM_EINVAL,
                "mm_batch_create: batches are built for two materials, at most one plastic");
  for (int i = 0; i < n; ++i)
    if (grids[i]->base.void_l >= 0)
      return fail(MM_EINVAL, "mm_batch_create: member %d holds void; void grids run alone", i);
  for (int i = 0; i < n; ++i)
    if (grids[i]->xscheme != MM_X_SWEEP)
      return fail(MM_EINVAL, "mm_batch_create: member %d transports X by WENO3 + RK3; batches "
                  "carry X in the sweeps", i);
  for (int i = 0; i < n; ++i) CUDA_TRY(cudaStreamSynchronize(grids[i]->stream));
  mm_batch* b = new mm_batch();
  b->m.assign(grids, grids + n);
  b->M = n;
  b->dim = g0->dim;
  b->prec = g0->prec;
  b->nmat = g0->nmat;
  b->nhist = g0->nhist;
  if (cuda_stream) {
    b->stream = (cudaStream_t)cuda_stream;
  } else {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
      batch_free(b);
      return fail(MM_ECUDA, "cudaStreamCreate failed");
    }
    b->own_stream = true;
  }
  // member arguments per step-start parity and phase
  std::vector<KArgs> A((size_t)2 * kPhases * n);
  for (int p = 0; p < 2; ++p)
    for (int i = 0; i < n; ++i) {
      const mm_grid* g = grids[i];
      const int c0 = g->cur ^ p;
      A[((size_t)p * kPhases + 0) * n + i] = args_at(g, c0);
      for (int d = 0; d < 3; ++d) {
        const int ci = c0 ^ (d & 1);
        KArgs a = args_at(g, ci);
        a.Uout = g->U[ci ^ 1];
        a.Eout = g->E[ci ^ 1];
        A[((size_t)p * kPhases + 1 + d) * n + i] = a;
      }
      A[((size_t)p * kPhases + 4) * n + i] = args_at(g, c0 ^ (g->dim & 1));
    }
  b->h_tstart.assign((size_t)3 * 2 * (n + 1), 0);
  tiles_fn T = tiles_of(b->prec, b->dim);
  for (int d = 0; d < b->dim; ++d)
    for (int v = 0; v < 2; ++v) {
      long long* st = &b->h_tstart[(size_t)(d * 2 + v) * (n + 1)];
      for (int i = 0; i < n; ++i) {
        const int nn[3] = {(int)grids[i]->desc.n[0], (int)grids[i]->desc.n[1], (int)grids[i]->desc.n[2]};
        st[i + 1] = st[i] + T(d, v, nn);
      }
    }
  b->h_cstart.assign(n + 1, 0);
  for (int i = 0; i < n; ++i)
    b->h_cstart[i + 1] = b->h_cstart[i] + (grids[i]->ncell + kChunk - 1) / kChunk;
  if (cudaMalloc(&b->args, sizeof(KArgs) * A.size()) != cudaSuccess ||
      cudaMalloc(&b->tstart, sizeof(long long) * b->h_tstart.size()) != cudaSuccess ||
      cudaMalloc(&b->cstart, sizeof(long long) * b->h_cstart.size()) != cudaSuccess ||
      cudaMalloc(&b->counter, sizeof(unsigned long long) * 8 * n) != cudaSuccess) {
    batch_free(b);
    return fail(MM_ENOMEM, "device allocation of the batch tables failed");
  }
  cudaError_t e = cudaMemcpy(b->args, A.data(), sizeof(KArgs) * A.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->tstart, b->h_tstart.data(), sizeof(long long) * b->h_tstart.size(),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->cstart, b->h_cstart.data(), sizeof(long long) * b->h_cstart.size(),
                   cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    batch_free(b);
    return fail(MM_ECUDA, "mm_batch_create: %s", cudaGetErrorString(e));
  }
  batch_group(b, 0);
  *out = b;
  return MM_OK;
}

mm_status mm_batch_set_grouping(mm_batch* b, int64_t group_bytes) {
  if (!b) return fail(MM_EINVAL, "mm_batch_set_grouping: null batch");
  batch_group(b, group_bytes < 0 ? default_group_bytes() : group_bytes);  // (L2 budget)
  batch_drop_graphs(b);
  return MM_OK;
}

int mm_batch_num_groups(const mm_batch* b) { return b ? (int)b->gstart.size() - 1 : 0; }

mm_status mm_batch_set_options(mm_batch* b, int use_graph, const int tile_variant[3]) {
  if (!b) return fail(MM_EINVAL, "mm_batch_set_options: null batch");
  b->use_graph = use_graph != 0;
  if (tile_variant)
    for (int d = 0; d < 3; ++d) {
      if (tile_variant[d] != 0 && tile_variant[d] != 1)
        return fail(MM_EINVAL, "tile variants are 0 or 1");
      b->variant[d] = tile_variant[d];
    }
  batch_drop_graphs(b);
  return MM_OK;
}

mm_status mm_batch_step(mm_batch* b, int n_steps, double cfl) {
  if (!b) return fail(MM_EINVAL, "mm_batch_step: null batch");
  if (n_steps < 0) return fail(MM_EINVAL, "n_steps must be >= 0");
  if (!(cfl > 0.0) || !(cfl <= 1.0)) return fail(MM_EINVAL, "cfl must be in (0, 1]");
  for (int s = 0; s < n_steps; ++s) {
    const int p = b->parity;
    if (b->use_graph && b->warmed && !b->prof) {
      if (!b->exec[p] || b->exec_cfl[p] != cfl) {
        if (b->exec[p]) cudaGraphExecDestroy(b->exec[p]);
        b->exec[p] = nullptr;
        cudaGraph_t graph = nullptr;
        CUDA_TRY(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        cudaError_t e = batch_enqueue(b, cfl);
        cudaError_t e2 = cudaStreamEndCapture(b->stream, &graph);
        if (e != cudaSuccess || e2 != cudaSuccess) {
          if (graph) cudaGraphDestroy(graph);
          return fail(MM_ECUDA, "mm_batch_step: graph capture: %s",
                      cudaGetErrorString(e != cudaSuccess ? e : e2));
        }
        e = cudaGraphInstantiate(&b->exec[p], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
          b->exec[p] = nullptr;
          return fail(MM_ECUDA, "mm_batch_step: cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
        b->exec_cfl[p] = cfl;
      }
      CUDA_TRY(cudaGraphLaunch(b->exec[p], b->stream));
    } else {
      // the first step runs uncaptured (it sets the kernels' attributes)
      CUDA_TRY(batch_enqueue(b, cfl));
      b->warmed = true;
    }
    batch_advance(b);
  }
  return MM_OK;
}

namespace {

// Size class of a batch: log2 of its median member cell count.
int batch_size_class(const mm_batch* b) {
  std::vector<long long> n;
  for (const mm_grid* g : b->m) n.push_back(g->ncell);
  std::sort(n.begin(), n.end());
  const long long med = n[n.size() / 2];
  int c = 0;
  while ((2LL << c) <= med) ++c;
  return c;
}

// Cache key: the device, precision, dimension, material layout and size
// class of a batch.
std::string tune_key(const mm_batch* b, int size_class) {
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceProp p;
  std::string name = "unknown";
  int sms = 0;
  if (cudaGetDeviceProperties(&p, dev) == cudaSuccess) {
    name = p.name;
    sms = p.multiProcessorCount;
  }
  for (char& ch : name)
    if (ch == ' ' || ch == '|') ch = '_';
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s|%d|%s|%d|%d|%d|%d", name.c_str(), sms,
                b->prec == MM_FP64 ? "fp64" : "fp32split", b->dim, b->nmat, b->nhist, size_class);
  return buf;
}

// The cached choice for key: tile variant and CTAs per SM per axis.
bool tune_read(const char* path, const std::string& key, int v[3], int c[3]) {
  FILE* f = std::fopen(path, "r");
  if (!f) return false;
  char line[512];
  bool found = false;
  while (std::fgets(line, sizeof line, f)) {
    char k[300];
    int a[6];
    if (std::sscanf(line, "%299s %d %d %d %d %d %d", k, &a[0], &a[1], &a[2], &a[3], &a[4],
                    &a[5]) == 7 &&
        key == k) {
      for (int d = 0; d < 3; ++d) {
        v[d] = a[d];
        c[d] = a[3 + d];
      }
      found = true;  // the last line for a key wins
    }
  }
  std::fclose(f);
  return found;
}

// Appends the choice for key (a later line for the same key overrides).
bool tune_write(const char* path, const std::string& key, const int v[3], const int c[3]) {
  FILE* f = std::fopen(path, "a");
  if (!f) return false;
  std::fprintf(f, "%s %d %d %d %d %d %d\n", key.c_str(), v[0], v[1], v[2], c[0], c[1], c[2]);
  return std::fclose(f) == 0;
}

}  // namespace

mm_status mm_batch_autotune_ex(mm_batch* b, int reps, const char* cache_path, int force,
                               mm_tune* out) {
  if (!b) return fail(MM_EINVAL, "mm_batch_autotune_ex: null batch");
  if (reps < 1) reps = 1;
  const int cls = batch_size_class(b);
  const std::string key = tune_key(b, cls);
  int from_cache = 0;
  int v[3] = {0, 0, 0}, c[3] = {0, 0, 0};
  if (cache_path && !force && tune_read(cache_path, key, v, c)) {
    bool ok = true;
    for (int d = 0; d < 3; ++d)
      ok = ok && (v[d] == 0 || (v[d] == 1 && b->prec != MM_FP64)) && c[d] >= 0 && c[d] <= 64;
    if (ok) from_cache = 1;
  }
  if (!from_cache) {
    // search: tile variant x persistent CTAs per SM (as many as fit, 1, 2)
    // per sweep axis, each timed as a sweep from the current state into the
    // free buffer (phase 1 of the current parity), which leaves the state
    // as it is
    batch_launcher L = batch_launch_of(b->prec, b->dim);
    const int M = b->M;
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    const int cps_options[3] = {0, 1, 2};
    for (int d = 0; d < b->dim; ++d) {
      float best = -1.f;
      for (int vv = 0; vv < (b->prec == MM_FP64 ? 1 : 2); ++vv) {
        for (int ci = 0; ci < 3; ++ci) {
          const size_t o = (size_t)(d * 2 + vv) * (M + 1);
          BatchK k = batch_k(b, 1, b->tstart + o, b->h_tstart[o + M]);
          k.cta_per_sm = cps_options[ci];
          float ms = 0.f;
          for (int r = -1; r < reps; ++r) {
            CUDA_TRY(cudaMemsetAsync(b->counter + 1, 0, sizeof(unsigned long long), b->stream));
            CUDA_TRY(cudaEventRecord(e0, b->stream));
            CUDA_TRY(L(1, d, vv, b->nmat, b->nhist, k, b->stream));
            CUDA_TRY(cudaEventRecord(e1, b->stream));
            CUDA_TRY(cudaEventSynchronize(e1));
            float t = 0.f;
            CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
            if (r >= 0) ms += t;  // r = -1 warms up
          }
          if (best < 0.f || ms < best) {
            best = ms;
            v[d] = vv;
            c[d] = cps_options[ci];
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (mm_grid* g : b->m) {
      mm_status st = check_device_error(g, "mm_batch_autotune");
      if (st != MM_OK) return st;
    }
    if (cache_path && !tune_write(cache_path, key, v, c))
      return fail(MM_EINVAL, "mm_batch_autotune_ex: cannot write the cache file %s", cache_path);
  }
  for (int d = 0; d < 3; ++d) {
    b->variant[d] = v[d];
    b->cps[d] = c[d];
  }
  batch_drop_graphs(b);
  if (out) {
    for (int d = 0; d < 3; ++d) {
      out->variant[d] = v[d];
      out->cta_per_sm[d] = c[d];
    }
    out->from_cache = from_cache;
    out->size_class = cls;
  }
  return MM_OK;
}

mm_status mm_batch_autotune(mm_batch* b, int reps, int chosen[3]) {
  mm_tune t;
  mm_status st = mm_batch_autotune_ex(b, reps, nullptr, 1, &t);
  if (st != MM_OK) return st;
  if (chosen)
    for (int d = 0; d < 3; ++d) chosen[d] = t.variant[d];
  return MM_OK;
}

mm_status mm_batch_synchronize(mm_batch* b) {
  if (!b) return fail(MM_EINVAL, "mm_batch_synchronize: null batch");
  CUDA_TRY(cudaStreamSynchronize(b->stream));
  prof_collect(b);
  for (int i = 0; i < b->M; ++i) {
    mm_status st = check_device_error(b->m[i], "mm_batch_synchronize");
    if (st != MM_OK) {
      std::string msg = g_error;
      return fail(st, "member %d: %s", i, msg.c_str());
    }
  }
  return MM_OK;
}

mm_status mm_batch_profile_enable(mm_batch* b, int enable) {
  if (!b) return fail(MM_EINVAL, "mm_batch_profile_enable: null batch");
  b->prof = enable != 0;
  return MM_OK;
}

mm_status mm_batch_profile_read(mm_batch* b, double* ms, int64_t* counts, int n, int reset) {
  if (!b || n < 0) return fail(MM_EINVAL, "mm_batch_profile_read: bad argument");
  for (int k = 0; k < n && k < MM_K_COUNT; ++k) {
    if (ms) ms[k] = b->prof_ms[k];
    if (counts) counts[k] = b->prof_n[k];
  }
  if (reset)
    for (int k = 0; k < MM_K_COUNT; ++k) {
      b->prof_ms[k] = 0.0;
      b->prof_n[k] = 0;
    }
  return MM_OK;
}

mm_status mm_batch_destroy(mm_batch* b) {
  if (!b) return MM_OK;
  cudaStreamSynchronize(b->stream);
  batch_free(b);
  return MM_OK;
}
