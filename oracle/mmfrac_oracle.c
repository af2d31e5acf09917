/*
 * Plain FP64 CPU oracle of the explicit Eulerian diffuse-interface step of
 * Wallis, Barton & Nikiforakis (arXiv 2210.04037).  TEST INFRASTRUCTURE ONLY:
 * it is loaded by tests/, by __graft_entry__.smoke() and by the cpu_baseline
 * and reference legs of bench.py, never by the product path.  It shares no
 * code with the CUDA library.
 *
 * The paper states the governing system (Sec. 2.1), the closures (Sec. 2.1.1,
 * 2.1.2), the damage laws (Sec. 2.1.1, Sec. 4.3), the perturbation field
 * (Sec. 2.1.3, 3.2) and RK4 for damage (Sec. 3.1), and defers the hyperbolic
 * solver, the mixture rules and the plastic update to earlier papers (start
 * of Sec. 3).  The readings used for those are written out beside each
 * routine; every step is done plainly, one cell or one face at a time, in
 * the order the method takes them:
 *
 *   one time step = dt from the CFL rule (R-CFL)
 *                   -> sweep x -> sweep y -> sweep z  (dimensional split, R8)
 *                   -> per-cell sources: phi0(X) lookup, plastic return,
 *                      RK4 damage (Godunov split, R12)
 *   fragments     = membership at a void cut-off -> components under face
 *                   adjacency in cell order -> masses (Sec. 4.2, 4.3)
 *   one sweep     = primitive recovery -> van Leer slopes on primitives (R9)
 *                   -> MUSCL-Hancock half step (first order where a face
 *                      state is inadmissible or a phase density leaves the
 *                      half step's bound) -> HLLC flux (R11)
 *                   -> conservative update + non-conservative terms
 */
#include "oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXF 32
#define LDIM 3

struct or_grid {
  int dim, nmat, nhist, nF, nfield;
  long n[3], ncell;
  double lo[3], hi[3], dx[3];
  int bc[3][2];
  or_material mat[OR_MAXMAT];
  int hslot[OR_MAXMAT]; /* history slot of material l, or -1 */
  int void_l;           /* index of the void material (eos 2), or -1 */
  int Fidx[9];          /* row-major index (3i+j) of each stored Fbar comp */
  int o_phi, o_arho, o_mom, o_E, o_F, o_hist, o_X;
  double *U, *V; /* conserved state and sweep output, [nfield][ncell] */
  float *phi0;
  long pn[3];
  double plo[3], ph[3];
  double t, dt_last, smax;
  long steps, bad_cell;
  long nbound; /* faces sent to first order by the phase-density bound */
  int xscheme; /* 0: X carried by the sweeps (R20); 1: WENO3 + RK3 (R28) */
  int seed_x;  /* Lagrangian seeding into void before each step (R35; default on) */
};

/* Derived quantities of one state that the flux and the Riemann solver use. */
typedef struct {
  double u[3];     /* velocity */
  double sig[9];   /* Cauchy stress, tension positive (R5) */
  double F[9];     /* full deformation tensor Fbar */
  double rho, p, cL;
  double G;        /* mixture shear modulus */
} aux_t;

/* ------------------------------------------------------------------------ */
/* Closures: one material (Sec. 2.1.1 and 2.1.2, Romenskii forms)           */
/* ------------------------------------------------------------------------ */

/*
 * Reference curve of one material at phasic density rho, damage factor
 * psi = 1 - D and shear invariant J2 = tr(devH devH^T).
 *   e_ref = e_c + e_s,  p_ref = rho^2 d e_ref / d rho,  dp_ref/drho,
 *   G and the Grueneisen coefficient Gamma.
 * Romenskii cold energy, printed with 1/rho (Eq. Romenskii, R3):
 *   e_c = psi K0 / (2 rho alpha^2) (eta^alpha - 1)^2,  eta = rho/rho0,
 * degraded by (1-D) (Eq. coldCompressionDegradation); shear modulus
 *   G = psi G0 eta^(beta+1)  (Romenskii G, degraded linearly, Sec. 2.1.1);
 * shear energy e_s = G J^2 / rho (Eq. shearEnergy); theta = eta^Gamma0 gives
 * a constant Gamma = Gamma0, hence the Mie-Grueneisen form
 *   p = p_ref + rho Gamma (e - e_ref).
 * Steinberg variant (shear_model 1; Sec. 2.1.2 and the U-Nb closure of
 * Sec. 4.3, R36): G = psi (G0 + Gp p_c0(rho) eta^(-1/3)), p_c0 the undamaged
 * cold pressure, and the Debye temperature of Burakovsky and Preston, whose
 * logarithmic derivative is Gamma(rho) = Gamma0 + Gamma1 eta^(-1/3) +
 * Gamma2 eta^(-gamma_s); the same Mie-Grueneisen form then holds with
 * Gamma(rho), and the shear pressure is p_s = rho^2 d e_s/d rho =
 * J^2 (rho G' - G).  Where the form is negative (strong tension) G = 0.
 * out[5] = rho Gamma'(rho) / Gamma: the isentropic sound speed of the form
 *   c^2 = dp_ref/drho + (Gamma + 1 + rho Gamma'/Gamma) (p - p_ref) / rho.
 * Ideal gas is the G = 0 case with e_ref = p_ref = 0, Gamma = gamma - 1.
 */
void or_thermo(const or_material* m, double rho, double psi, double J2,
               double* out) {
  out[5] = 0.0;
  if (m->eos == 0) {
    out[0] = 0.0;
    out[1] = 0.0;
    out[2] = 0.0;
    out[3] = 0.0;
    out[4] = m->gamma_gas - 1.0;
    return;
  }
  if (m->eos == 2) {  /* void: no energy, no pressure, no shear */
    out[0] = out[1] = out[2] = out[3] = 0.0;
    out[4] = 1.0;
    return;
  }
  const double a = m->alpha;
  const double eta = rho / m->rho0;
  const double ea = pow(eta, a);
  const double q = ea - 1.0;
  /* cold energy and its pressure p_c = rho^2 de_c/drho */
  const double ec = psi * m->K0 / (2.0 * rho * a * a) * (q * q);
  const double pc = psi * m->K0 / (2.0 * a * a) * (2.0 * a * q * ea - q * q);
  /* d p_c / d rho = psi K0 eta^(a-1) ((2a-1) eta^a + 1 - a) / (a rho0) */
  const double dpc = psi * m->K0 * pow(eta, a - 1.0) *
                     ((2.0 * a - 1.0) * ea + (1.0 - a)) / (a * m->rho0);
  if (m->shear_model == 1) {
    /* Steinberg: G = psi (G0 + Gp q), q = p_c0 u, u = eta^(-1/3), with the
     * undamaged cold pressure p_c0 and its derivatives
     *   p_c0'  = K0 E ((2a-1) E + 1 - a) / (a rho),
     *   p_c0'' = K0 E ((2a-1)^2 E - (a-1)^2) / (a rho^2),  E = eta^a,
     * and u' = -u / (3 rho), u'' = 4 u / (9 rho^2). */
    const double pc0 = m->K0 / (2.0 * a * a) * (2.0 * a * q * ea - q * q);
    const double pc1 = m->K0 * ea * ((2.0 * a - 1.0) * ea + (1.0 - a)) / (a * rho);
    const double pc2 = m->K0 * ea * ((2.0 * a - 1.0) * (2.0 * a - 1.0) * ea -
                                     (a - 1.0) * (a - 1.0)) / (a * rho * rho);
    const double u = pow(eta, -1.0 / 3.0);
    const double qs = pc0 * u;
    const double q2 = u * (pc2 - 2.0 * pc1 / (3.0 * rho) + 4.0 * pc0 / (9.0 * rho * rho));
    const double q1 = u * (pc1 - pc0 / (3.0 * rho));
    /* the form turns negative in strong tension (p_c < -G0 / Gp eta^(1/3),
     * about 20 % expansion for U-Nb, where a trace phase in a gas cell can
     * go): there the material has no shear stiffness, G = G' = G'' = 0 */
    const int pos = m->G0 + m->Gp * qs > 0.0;
    const double G = pos ? psi * (m->G0 + m->Gp * qs) : 0.0;
    const double dG = pos ? psi * m->Gp * q1 : 0.0, d2G = pos ? psi * m->Gp * q2 : 0.0;
    const double es = G * J2 / rho;
    const double ps = J2 * (rho * dG - G);
    const double dps = J2 * rho * d2G;
    const double g2 = pow(eta, -m->gamma_s);
    const double Gam = m->Gamma0 + m->Gamma1 * u + m->Gamma2 * g2;
    out[0] = ec + es;
    out[1] = pc + ps;
    out[2] = dpc + dps;
    out[3] = G;
    out[4] = Gam;
    out[5] = (-m->Gamma1 * u / 3.0 - m->gamma_s * m->Gamma2 * g2) / Gam;
    return;
  }
  /* shear part: G(rho), e_s = G J2/rho, p_s = rho^2 de_s/drho = beta G J2 */
  const double G = psi * m->G0 * pow(eta, m->beta + 1.0);
  const double es = G * J2 / rho;
  const double ps = m->beta * G * J2;
  const double dps = m->beta * (m->beta + 1.0) * G * J2 / rho;
  out[0] = ec + es;
  out[1] = pc + ps;
  out[2] = dpc + dps;
  out[3] = G;
  out[4] = m->Gamma0;
}

/* ------------------------------------------------------------------------ */
/* Hencky strain devH = dev(ln Vbar) = dev(1/2 ln(Fbar Fbar^T)) (Sec. 2.1.1) */
/* by the cyclic Jacobi method (symmetric Schur rotations).                 */
/* ------------------------------------------------------------------------ */

static void jacobi_rotate(double a[9], double Q[9], int p, int q) {
  const double apq = a[3 * p + q];
  if (apq == 0.0) return;
  const double app = a[3 * p + p], aqq = a[3 * q + q];
  const double theta = (aqq - app) / (2.0 * apq);
  double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
  if (theta < 0.0) t = -t;
  const double c = 1.0 / sqrt(t * t + 1.0);
  const double s = t * c;
  a[3 * p + p] = app - t * apq;
  a[3 * q + q] = aqq + t * apq;
  a[3 * p + q] = 0.0;
  a[3 * q + p] = 0.0;
  const int r = 3 - p - q;
  const double arp = a[3 * r + p], arq = a[3 * r + q];
  a[3 * r + p] = a[3 * p + r] = c * arp - s * arq;
  a[3 * r + q] = a[3 * q + r] = s * arp + c * arq;
  for (int k = 0; k < 3; ++k) {
    const double qp = Q[3 * k + p], qq = Q[3 * k + q];
    Q[3 * k + p] = c * qp - s * qq;
    Q[3 * k + q] = s * qp + c * qq;
  }
}

/* Eigen-decomposition A = Q diag(lam) Q^T of a symmetric 3x3 matrix. */
static void jacobi3(const double A[9], double lam[3], double Q[9]) {
  double a[9];
  memcpy(a, A, sizeof a);
  for (int k = 0; k < 9; ++k) Q[k] = (k % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 50; ++sweep) {
    const double off = a[1] * a[1] + a[2] * a[2] + a[5] * a[5];
    const double dd = a[0] * a[0] + a[4] * a[4] + a[8] * a[8];
    if (off <= 1e-32 * dd) break;
    jacobi_rotate(a, Q, 0, 1);
    jacobi_rotate(a, Q, 0, 2);
    jacobi_rotate(a, Q, 1, 2);
  }
  lam[0] = a[0];
  lam[1] = a[4];
  lam[2] = a[8];
}

/* devH and its eigen-pairs: h = dev eigenvalues of 1/2 ln b, b = F F^T. */
static int hencky_eig(const double F[9], double devH[9], double h[3],
                      double Q[9], double lam[3]) {
  double b[9];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      const double s = F[3 * i + 0] * F[3 * j + 0] +
                       F[3 * i + 1] * F[3 * j + 1] +
                       F[3 * i + 2] * F[3 * j + 2];
      b[3 * i + j] = s;
      b[3 * j + i] = s;
    }
  jacobi3(b, lam, Q);
  for (int k = 0; k < 3; ++k)
    if (!(lam[k] > 0.0) || !isfinite(lam[k])) return -1;
  for (int k = 0; k < 3; ++k) h[k] = 0.5 * log(lam[k]);
  const double tr = (h[0] + h[1] + h[2]) / 3.0;
  for (int k = 0; k < 3; ++k) h[k] -= tr;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      devH[3 * i + j] = Q[3 * i + 0] * h[0] * Q[3 * j + 0] +
                        Q[3 * i + 1] * h[1] * Q[3 * j + 1] +
                        Q[3 * i + 2] * h[2] * Q[3 * j + 2];
  return 0;
}

int or_hencky(const double F[9], double devH[9], double lam[3], double Q[9]) {
  double h[3];
  return hencky_eig(F, devH, h, Q, lam);
}

/* ------------------------------------------------------------------------ */
/* Field layout                                                              */
/* ------------------------------------------------------------------------ */

static int is_damaged(const or_material* m) { return m->damage != 0; }

/* Critical damage (Sec. 3.1): D >= D_crit within 1e-4 (R34).  D comes back
 * as the ratio (phi rho D) / (phi rho) of two transported quantities, so a
 * cell the RK4 capped at D_crit reads below it after advection, by rounding
 * (in FP32 storage about 1e-7 a step) or by a trace of undamaged material
 * mixed in; the yield stress and the void-opening test both count a cell
 * within the band as critical, and a cell diluted further as healed (the
 * artificial healing of Sec. 3.1). */
static int is_critical(const or_material* m, double D) {
  return is_damaged(m) && D >= m->D_crit * (1.0 - 1e-4);
}

/* The void volume fraction nu (Sec. 2.1) is carried as a material of its
 * own (eos 2): its fraction is advected like the others, it has no mass, no
 * energy and no stress, and it takes no part in the pressure equilibrium of
 * the materials (R33). */
static int is_void(const or_material* m) { return m->eos == 2; }

/* Full local views of a stored state vector (inactive components: 0 / I). */
static void full_F(const or_grid* g, const double* w, double F[9]) {
  for (int k = 0; k < 9; ++k) F[k] = (k % 4 == 0) ? 1.0 : 0.0;
  for (int c = 0; c < g->nF; ++c) F[g->Fidx[c]] = w[g->o_F + c];
}

static void vol_fracs(const or_grid* g, const double* w, double phi[]) {
  double s = 0.0;
  for (int l = 0; l + 1 < g->nmat; ++l) {
    phi[l] = w[g->o_phi + l];
    s += phi[l];
  }
  phi[g->nmat - 1] = 1.0 - s;
}

/* ------------------------------------------------------------------------ */
/* Mixture (R7: Allaire isobaric closure, single Fbar, Sec. 2.1 and 2.1.2)  */
/* ------------------------------------------------------------------------ */

typedef struct {
  double th[OR_MAXMAT][6];
  double xi, Gmix;
  double devH[9], J2;
} mix_t;

static int mixture(const or_grid* g, const double* phi, const double* rho_l,
                   const double* Dl, const double F[9], mix_t* mx) {
  double h[3], Q[9], lam[3];
  if (hencky_eig(F, mx->devH, h, Q, lam) != 0) return -1;
  mx->J2 = h[0] * h[0] + h[1] * h[1] + h[2] * h[2];
  mx->xi = 0.0;
  mx->Gmix = 0.0;
  for (int l = 0; l < g->nmat; ++l) {
    const double psi = is_damaged(&g->mat[l]) ? 1.0 - Dl[l] : 1.0;
    or_thermo(&g->mat[l], rho_l[l], psi, mx->J2, mx->th[l]);
    if (is_void(&g->mat[l])) continue;
    mx->xi += phi[l] / mx->th[l][4];
    mx->Gmix += phi[l] * mx->th[l][3];
  }
  return 0;
}

/* Stress sigma = -p I + 2 G dev(H) (R5) and longitudinal sound speed (R6). */
static int finish_aux(const or_grid* g, const double* phi, const double* rho_l,
                      const double* arho, const mix_t* mx, aux_t* ax) {
  /* with void in the cell the materials fill 1 - nu of it and the pressure
   * part of the stress is theirs times that fraction (the void carries
   * none); the shear part is already weighted by the fractions (R33) */
  const double pm = g->void_l >= 0 ? ax->p * (1.0 - phi[g->void_l]) : ax->p;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      ax->sig[3 * i + j] =
          (i == j ? -pm : 0.0) + 2.0 * mx->Gmix * mx->devH[3 * i + j];
  /* frozen mixture sound speed: xi c^2 = sum_l y_l xi_l c_l^2, c_l^2 the
   * isentropic sound speed of material l (with rho Gamma'/Gamma for a
   * density-dependent Gamma, R36) */
  double s = 0.0;
  for (int l = 0; l < g->nmat; ++l) {
    if (is_void(&g->mat[l])) continue;
    const double Gam = mx->th[l][4];
    const double cl2 = mx->th[l][2] + (Gam + 1.0 + mx->th[l][5]) * (ax->p - mx->th[l][1]) /
                                          rho_l[l];
    s += (arho[l] / ax->rho) * (1.0 / Gam) * cl2;
  }
  (void)phi;
  const double c2 = s / mx->xi;
  ax->G = mx->Gmix;
  const double cL2 = c2 + (4.0 / 3.0) * mx->Gmix / ax->rho;
  if (!(cL2 > 0.0) || !isfinite(cL2)) return -1;
  ax->cL = sqrt(cL2);
  return 0;
}

/* Primitive W -> conserved U (+ derived quantities). Returns 0 if valid. */
static int w2u(const or_grid* g, const double* w, double* u, aux_t* ax) {
  double phi[OR_MAXMAT], rho_l[OR_MAXMAT], arho[OR_MAXMAT], Dl[OR_MAXMAT];
  vol_fracs(g, w, phi);
  ax->rho = 0.0;
  for (int l = 0; l < g->nmat; ++l) {
    Dl[l] = 0.0;
    if (is_void(&g->mat[l])) {
      /* no mass; the fraction may be zero */
      if (!(phi[l] >= 0.0)) return -1;
      rho_l[l] = 0.0;
      arho[l] = 0.0;
      continue;
    }
    if (!(phi[l] > 0.0)) return -1;
    rho_l[l] = w[g->o_arho + l];
    if (!(rho_l[l] > 0.0)) return -1;
    arho[l] = phi[l] * rho_l[l];
    ax->rho += arho[l];
    Dl[l] = g->hslot[l] >= 0 ? w[g->o_hist + 2 * g->hslot[l] + 1] : 0.0;
  }
  for (int k = 0; k < 3; ++k) ax->u[k] = k < g->dim ? w[g->o_mom + k] : 0.0;
  ax->p = w[g->o_E];
  full_F(g, w, ax->F);
  mix_t mx;
  if (mixture(g, phi, rho_l, Dl, ax->F, &mx) != 0) return -1;
  /* rho e = sum_l phi_l rho_l e_l with p = p_ref,l + rho_l Gamma_l (e_l - e_ref,l) */
  double rhoe = 0.0;
  for (int l = 0; l < g->nmat; ++l) {
    if (is_void(&g->mat[l])) continue; /* no energy, no part in the closure */
    rhoe += arho[l] * mx.th[l][0] + phi[l] * (ax->p - mx.th[l][1]) / mx.th[l][4];
  }
  const double ke = 0.5 * ax->rho *
                    (ax->u[0] * ax->u[0] + ax->u[1] * ax->u[1] + ax->u[2] * ax->u[2]);
  for (int l = 0; l + 1 < g->nmat; ++l) u[g->o_phi + l] = phi[l];
  for (int l = 0; l < g->nmat; ++l) u[g->o_arho + l] = arho[l];
  for (int k = 0; k < g->dim; ++k) u[g->o_mom + k] = ax->rho * ax->u[k];
  u[g->o_E] = rhoe + ke;
  for (int c = 0; c < g->nF; ++c) u[g->o_F + c] = w[g->o_F + c];
  for (int l = 0; l < g->nmat; ++l) {
    const int h = g->hslot[l];
    if (h < 0) continue;
    u[g->o_hist + 2 * h] = arho[l] * w[g->o_hist + 2 * h];
    u[g->o_hist + 2 * h + 1] = arho[l] * w[g->o_hist + 2 * h + 1];
  }
  for (int k = 0; k < g->dim; ++k) u[g->o_X + k] = w[g->o_X + k];
  return finish_aux(g, phi, rho_l, arho, &mx, ax);
}

/* Conserved U -> primitive W (+ derived quantities). Returns 0 if valid. */
static int u2w(const or_grid* g, const double* u, double* w, aux_t* ax) {
  double phi[OR_MAXMAT], rho_l[OR_MAXMAT], arho[OR_MAXMAT], Dl[OR_MAXMAT];
  vol_fracs(g, u, phi);
  ax->rho = 0.0;
  for (int l = 0; l < g->nmat; ++l) {
    arho[l] = u[g->o_arho + l];
    if (is_void(&g->mat[l])) {
      if (!(phi[l] >= 0.0)) return -1;
      rho_l[l] = 0.0;
      continue;
    }
    if (!(phi[l] > 0.0) || !(arho[l] > 0.0)) return -1;
    rho_l[l] = arho[l] / phi[l];
    ax->rho += arho[l];
  }
  for (int l = 0; l < g->nmat; ++l) {
    const int h = g->hslot[l];
    Dl[l] = 0.0;
    if (h < 0) continue;
    w[g->o_hist + 2 * h] = u[g->o_hist + 2 * h] / arho[l];
    w[g->o_hist + 2 * h + 1] = u[g->o_hist + 2 * h + 1] / arho[l];
    Dl[l] = w[g->o_hist + 2 * h + 1];
  }
  for (int k = 0; k < 3; ++k)
    ax->u[k] = k < g->dim ? u[g->o_mom + k] / ax->rho : 0.0;
  full_F(g, u, ax->F);
  mix_t mx;
  if (mixture(g, phi, rho_l, Dl, ax->F, &mx) != 0) return -1;
  const double ke = 0.5 * ax->rho *
                    (ax->u[0] * ax->u[0] + ax->u[1] * ax->u[1] + ax->u[2] * ax->u[2]);
  const double rhoe = u[g->o_E] - ke;
  double num = rhoe;
  for (int l = 0; l < g->nmat; ++l)
    num += -arho[l] * mx.th[l][0] + phi[l] * mx.th[l][1] / mx.th[l][4];
  ax->p = num / mx.xi;
  for (int l = 0; l + 1 < g->nmat; ++l) w[g->o_phi + l] = phi[l];
  for (int l = 0; l < g->nmat; ++l) w[g->o_arho + l] = rho_l[l];
  for (int k = 0; k < g->dim; ++k) w[g->o_mom + k] = ax->u[k];
  w[g->o_E] = ax->p;
  for (int c = 0; c < g->nF; ++c) w[g->o_F + c] = u[g->o_F + c];
  for (int k = 0; k < g->dim; ++k) w[g->o_X + k] = u[g->o_X + k];
  for (int k = 0; k < g->nfield; ++k)
    if (!isfinite(w[k]) || !isfinite(u[k])) return -1;
  return finish_aux(g, phi, rho_l, arho, &mx, ax);
}

/* ------------------------------------------------------------------------ */
/* Physical flux in direction d of the system of Sec. 2.1 (G4-G9, G13, R1)  */
/* ------------------------------------------------------------------------ */

static void phys_flux(const or_grid* g, int d, const double* u,
                      const aux_t* ax, double* f) {
  const double ud = ax->u[d];
  for (int l = 0; l + 1 < g->nmat; ++l) f[g->o_phi + l] = u[g->o_phi + l] * ud;
  for (int l = 0; l < g->nmat; ++l) f[g->o_arho + l] = u[g->o_arho + l] * ud;
  for (int k = 0; k < g->dim; ++k)
    f[g->o_mom + k] = u[g->o_mom + k] * ud - ax->sig[3 * k + d];
  f[g->o_E] = u[g->o_E] * ud -
              (ax->sig[3 * d + 0] * ax->u[0] + ax->sig[3 * d + 1] * ax->u[1] +
               ax->sig[3 * d + 2] * ax->u[2]);
  for (int c = 0; c < g->nF; ++c) {
    const int i = g->Fidx[c] / 3, j = g->Fidx[c] % 3;
    f[g->o_F + c] = (i == d) ? 0.0
                             : u[g->o_F + c] * ud - ax->F[3 * d + j] * ax->u[i];
  }
  for (int k = 0; k < 2 * g->nhist; ++k) f[g->o_hist + k] = u[g->o_hist + k] * ud;
  for (int k = 0; k < g->dim; ++k) f[g->o_X + k] = u[g->o_X + k] * ud;
}

/* ------------------------------------------------------------------------ */
/* Riemann solver (R11), HLLD type for the elastic mixture: Davis outer     */
/* longitudinal waves S_L, S_R; contact S*; in each star region a shear     */
/* wave S* -/+ c_s.  Every intermediate state follows from the Rankine-     */
/* Hugoniot conditions across its wave: across S_K the tangential velocity  */
/* and traction are unchanged; across the shear waves the normal velocity,  */
/* normal stress, densities and the row d of Fbar are unchanged; at the     */
/* contact the normal stress, the tangential velocity and traction are      */
/* continuous.  With G = 0 it is the HLLC solver.                           */
/* ------------------------------------------------------------------------ */

/* Flux through the face from the star side K (left = 1: the left star
 * region holds the face) of the subsonic Riemann fan: F_K + S_K (U*_K - U_K)
 * plus the jump across K's shear wave; the face velocity and the row d of
 * Fbar of that star region. */
static void star_side_flux(const or_grid* g, int d, int left, const double* UL,
                           const aux_t* aL, const double* UR, const aux_t* aR,
                           double SL, double SR, double Ss, double* Fo,
                           double* uface, double Frow[3]) {
  const double uL = aL->u[d], uR = aR->u[d];
  const double rL = aL->rho, rR = aR->rho;
  const double* UK = left ? UL : UR;
  const aux_t* aK = left ? aL : aR;
  const double SK = left ? SL : SR;
  double FK[MAXF];
  phys_flux(g, d, UK, aK, FK);
  const double uK = aK->u[d];
  for (int j = 0; j < 3; ++j) Frow[j] = aK->F[3 * d + j];
  /* star state of side K */
  const double chi = (SK - uK) / (SK - Ss);
  const double rK = aK->rho;
  double Us[MAXF];
  for (int l = 0; l + 1 < g->nmat; ++l) Us[g->o_phi + l] = UK[g->o_phi + l] * chi;
  for (int l = 0; l < g->nmat; ++l) Us[g->o_arho + l] = UK[g->o_arho + l] * chi;
  for (int k = 0; k < g->dim; ++k)
    Us[g->o_mom + k] = (k == d) ? rK * chi * Ss : UK[g->o_mom + k] * chi;
  Us[g->o_E] = chi * (UK[g->o_E] + rK * Ss * (Ss - uK) -
                      aK->sig[3 * d + d] * (Ss - uK) / (SK - uK));
  for (int c = 0; c < g->nF; ++c) {
    const int i = g->Fidx[c] / 3;
    Us[g->o_F + c] = (i == d) ? UK[g->o_F + c] : UK[g->o_F + c] * chi;
  }
  for (int k = 0; k < 2 * g->nhist; ++k) Us[g->o_hist + k] = UK[g->o_hist + k] * chi;
  for (int k = 0; k < g->dim; ++k) Us[g->o_X + k] = UK[g->o_X + k] * chi;
  for (int k = 0; k < g->nfield; ++k) Fo[k] = FK[k] + SK * (Us[k] - UK[k]);
  *uface = uK + SK * (chi - 1.0);
  /* shear waves: speeds from the star densities, kept inside [S_L, S_R] */
  const double rsL = rL * ((SL - uL) / (SL - Ss));
  const double rsR = rR * ((SR - uR) / (SR - Ss));
  double csL = sqrt(aL->G / rsL), csR = sqrt(aR->G / rsR);
  if (csL > Ss - SL) csL = Ss - SL;
  if (csR > SR - Ss) csR = SR - Ss;
  const double ZL = rsL * csL, ZR = rsR * csR;
  const double csK = left ? csL : csR;
  if (!(ZL + ZR > 0.0)) return;
  if (left ? !(Ss - csL < 0.0) : !(Ss + csR > 0.0)) return;
  /* a side without shear stiffness has no shear wave (it would coincide
   * with the contact; reachable at a contact at rest) */
  if (!(csK > 0.0)) return;
  double Uss[MAXF];
  for (int k = 0; k < g->nfield; ++k) Uss[k] = Us[k];
  const double sgn = left ? 1.0 : -1.0;
  const double rsK = left ? rsL : rsR;
  for (int t = 0; t < g->dim; ++t) {
    if (t == d) continue;
    const double uLt = aL->u[t], uRt = aR->u[t];
    const double tauL = aL->sig[3 * t + d], tauR = aR->sig[3 * t + d];
    const double uss = (tauR - tauL + ZL * uLt + ZR * uRt) / (ZL + ZR);
    const double tss = tauL + ZL * (uss - uLt);
    const double uKt = left ? uLt : uRt, tauK = left ? tauL : tauR;
    const double du = uss - uKt;
    Uss[g->o_mom + t] = rsK * uss;
    for (int c = 0; c < g->nF; ++c) {
      const int i = g->Fidx[c] / 3, j = g->Fidx[c] % 3;
      if (i == t) Uss[g->o_F + c] = Us[g->o_F + c] + sgn * aK->F[3 * d + j] * du / csK;
    }
    Uss[g->o_E] += sgn * (tss * uss - tauK * uKt) / csK;
  }
  const double SSK = left ? Ss - csL : Ss + csR;
  for (int k = 0; k < g->nfield; ++k) Fo[k] += SSK * (Uss[k] - Us[k]);
}

static void riemann_contact(const or_grid* g, int d, const double* UL, const aux_t* aL,
                            const double* UR, const aux_t* aR, double* Fo,
                            double* uface, double Frow[3]) {
  const double uL = aL->u[d], uR = aR->u[d];
  const double a1 = uL - aL->cL, a2 = uR - aR->cL;
  const double b1 = uL + aL->cL, b2 = uR + aR->cL;
  const double SL = a1 < a2 ? a1 : a2;
  const double SR = b1 > b2 ? b1 : b2;
  const double sL = aL->sig[3 * d + d], sR = aR->sig[3 * d + d];
  const double rL = aL->rho, rR = aR->rho;
  const double Ss = (sL - sR + rL * uL * (SL - uL) - rR * uR * (SR - uR)) /
                    (rL * (SL - uL) - rR * (SR - uR));
  if (SL >= 0.0 || SR <= 0.0) {
    const aux_t* aK = SL >= 0.0 ? aL : aR;
    phys_flux(g, d, SL >= 0.0 ? UL : UR, aK, Fo);
    *uface = aK->u[d];
    for (int j = 0; j < 3; ++j) Frow[j] = aK->F[3 * d + j];
    return;
  }
  /* A contact at rest (S* zero to within the rounding of the wave speeds, as
   * at a reflective wall or on any symmetry plane) lies on the face itself:
   * the face takes the mean of what the two star sides give (R31).  The two
   * agree in the conserved fields; in the tangential rows of Fbar, the row d
   * and the face velocity they differ, and the mean makes the face
   * independent of the sign of a rounded zero.  At a wall it gives the
   * kinematics of a free-slip wall: no flux of the tangential rows, row d
   * without tangential entries. */
  if (fabs(Ss) <= 16.0 * DBL_EPSILON * (SR - SL)) {
    double FL[MAXF], FR[MAXF], ufL, ufR, rowL[3], rowR[3];
    star_side_flux(g, d, 1, UL, aL, UR, aR, SL, SR, Ss, FL, &ufL, rowL);
    star_side_flux(g, d, 0, UL, aL, UR, aR, SL, SR, Ss, FR, &ufR, rowR);
    for (int k = 0; k < g->nfield; ++k) Fo[k] = 0.5 * (FL[k] + FR[k]);
    *uface = 0.5 * (ufL + ufR);
    for (int j = 0; j < 3; ++j) Frow[j] = 0.5 * (rowL[j] + rowR[j]);
    return;
  }
  star_side_flux(g, d, Ss >= 0.0, UL, aL, UR, aR, SL, SR, Ss, Fo, uface, Frow);
}

/* ------------------------------------------------------------------------ */
/* Void opening (Sec. 3.1: the void-opening flux modifier applied where     */
/* either face state is critically damaged and the two are in tension along */
/* the sweep, x^T (sigma_L + sigma_R) x > 0).  The modifier itself is in a  */
/* paper not available; reading R33: each side meets a traction-free        */
/* surface (the Riemann problem of a material against void), and where the  */
/* two surfaces separate, the gap between them is void.                     */
/* ------------------------------------------------------------------------ */

/* A damaged solid at critical damage (R34). */
static int critical_state(const or_grid* g, const double* U) {
  for (int l = 0; l < g->nmat; ++l) {
    const int h = g->hslot[l];
    if (h < 0 || !is_damaged(&g->mat[l])) continue;
    const double arho = U[g->o_arho + l];
    if (!(arho > 0.0)) continue;
    if (is_critical(&g->mat[l], U[g->o_hist + 2 * h + 1] / arho)) return 1;
  }
  return 0;
}

/* Speed of side K's traction-free surface: across K's longitudinal wave
 * S_K = u_K -/+ c_L,K the normal stress drops to zero,
 * 0 = sigma_K - rho_K (S_K - u_K)(S_f - u_K)  (HLLC jump relation). */
static double free_surface_speed(int d, int left, const aux_t* a) {
  const double SK = left ? a->u[d] - a->cL : a->u[d] + a->cL;
  return a->u[d] + a->sig[3 * d + d] / (a->rho * (SK - a->u[d]));
}

/* Flux of side K's fan against a traction-free surface: waves S_K, the
 * shear wave S_f -/+ c_s and the surface S_f; in the star regions the
 * normal stress and then the tangential tractions are zero.  at_face: the
 * region holding x/t = 0; otherwise the region just inside the surface.
 * Fo, uface, Frow as in the contact solver. */
static void free_surface_flux(const or_grid* g, int d, int left, const double* UK,
                              const aux_t* aK, int at_face, double* Fo, double* uface,
                              double Frow[3]) {
  const double uK = aK->u[d];
  const double SK = left ? uK - aK->cL : uK + aK->cL;
  const double Sf = free_surface_speed(d, left, aK);
  for (int j = 0; j < 3; ++j) Frow[j] = aK->F[3 * d + j];
  phys_flux(g, d, UK, aK, Fo);
  *uface = uK;
  if (at_face && (left ? SK >= 0.0 : SK <= 0.0)) return; /* region K */
  const double chi = (SK - uK) / (SK - Sf);
  const double rK = aK->rho;
  double Us[MAXF];
  for (int l = 0; l + 1 < g->nmat; ++l) Us[g->o_phi + l] = UK[g->o_phi + l] * chi;
  for (int l = 0; l < g->nmat; ++l) Us[g->o_arho + l] = UK[g->o_arho + l] * chi;
  for (int k = 0; k < g->dim; ++k)
    Us[g->o_mom + k] = (k == d) ? rK * chi * Sf : UK[g->o_mom + k] * chi;
  Us[g->o_E] = chi * (UK[g->o_E] + rK * Sf * (Sf - uK) -
                      aK->sig[3 * d + d] * (Sf - uK) / (SK - uK));
  for (int c = 0; c < g->nF; ++c) {
    const int i = g->Fidx[c] / 3;
    Us[g->o_F + c] = (i == d) ? UK[g->o_F + c] : UK[g->o_F + c] * chi;
  }
  for (int k = 0; k < 2 * g->nhist; ++k) Us[g->o_hist + k] = UK[g->o_hist + k] * chi;
  for (int k = 0; k < g->dim; ++k) Us[g->o_X + k] = UK[g->o_X + k] * chi;
  for (int k = 0; k < g->nfield; ++k) Fo[k] += SK * (Us[k] - UK[k]);
  *uface = uK + SK * (chi - 1.0);
  /* the shear wave: speed from the star density, kept between S_K and S_f */
  const double rs = rK * ((SK - uK) / (SK - Sf));
  double cs = sqrt(aK->G / rs);
  if (cs > fabs(Sf - SK)) cs = fabs(Sf - SK);
  if (!(cs > 0.0)) return;
  const double SSK = left ? Sf - cs : Sf + cs;
  if (at_face && (left ? SSK >= 0.0 : SSK <= 0.0)) return; /* region K* */
  const double Z = rs * cs, sgn = left ? 1.0 : -1.0;
  double Uss[MAXF];
  for (int k = 0; k < g->nfield; ++k) Uss[k] = Us[k];
  for (int t = 0; t < g->dim; ++t) {
    if (t == d) continue;
    const double tau = aK->sig[3 * t + d], ut = aK->u[t];
    /* zero traction behind the shear wave: tau + sgn Z (uss - ut) = 0 */
    const double uss = ut - sgn * tau / Z;
    const double du = uss - ut;
    Uss[g->o_mom + t] = rs * uss;
    for (int c = 0; c < g->nF; ++c) {
      const int i = g->Fidx[c] / 3, j = g->Fidx[c] % 3;
      if (i == t) Uss[g->o_F + c] = Us[g->o_F + c] + sgn * aK->F[3 * d + j] * du / cs;
    }
    Uss[g->o_E] += sgn * (0.0 * uss - tau * ut) / cs;
  }
  for (int k = 0; k < g->nfield; ++k) Fo[k] += SSK * (Uss[k] - Us[k]);
}

/* Riemann problem at a face: the face records of its left cell (FoL, ufL,
 * FrL: what the cell left of the face sees) and of its right cell.  They
 * are the same record (the contact solver) unless the void opens.  Where it
 * opens, each side's traction-free surface S_f,K sets that side's face
 * velocity, its Fbar and X transport; the conserved fields and the
 * material fractions take what crosses the face (nothing when the gap
 * holds the face; the fan of the side whose surface has passed it
 * otherwise), and the void fraction takes the rest, so that every side's
 * fractions stay summing to one: a side that receives the gap gets void at
 * the rate S_f,own - u_crossing. */
static void riemann(const or_grid* g, int d, const double* UL, const aux_t* aL,
                    const double* UR, const aux_t* aR, double* FoL, double* ufL,
                    double FrL[3], double* FoR, double* ufR, double FrR[3]) {
  const int nf = g->nfield;
  if (g->void_l >= 0 && (critical_state(g, UL) || critical_state(g, UR)) &&
      aL->sig[3 * d + d] + aR->sig[3 * d + d] > 0.0) {
    const double SfL = free_surface_speed(d, 1, aL), SfR = free_surface_speed(d, 0, aR);
    if (SfL < SfR) {
      double Fs[2][MAXF], ufs[2], rows[2][3], Fc[MAXF], ufc = 0.0, rowc[3];
      free_surface_flux(g, d, 1, UL, aL, 0, Fs[0], &ufs[0], rows[0]);
      free_surface_flux(g, d, 0, UR, aR, 0, Fs[1], &ufs[1], rows[1]);
      int cross = -1; /* the side whose fan holds the face, or none */
      for (int k = 0; k < nf; ++k) Fc[k] = 0.0;
      if (SfL > 0.0) {
        cross = 0;
        free_surface_flux(g, d, 1, UL, aL, 1, Fc, &ufc, rowc);
      } else if (SfR < 0.0) {
        cross = 1;
        free_surface_flux(g, d, 0, UR, aR, 1, Fc, &ufc, rowc);
      }
      for (int side = 0; side < 2; ++side) {
        double* Fo = side == 0 ? FoL : FoR;
        double* uf = side == 0 ? ufL : ufR;
        double* Fr = side == 0 ? FrL : FrR;
        for (int j = 0; j < 3; ++j) Fr[j] = rows[side][j];
        if (cross == side) {
          for (int k = 0; k < nf; ++k) Fo[k] = Fc[k];
          *uf = ufc;
          continue;
        }
        for (int k = 0; k < nf; ++k) Fo[k] = Fc[k];
        for (int c = 0; c < g->nF; ++c) Fo[g->o_F + c] = Fs[side][g->o_F + c];
        for (int k = 0; k < g->dim; ++k) Fo[g->o_X + k] = Fs[side][g->o_X + k];
        Fo[g->o_phi + g->void_l] += ufs[side] - ufc;
        *uf = ufs[side];
      }
      return;
    }
  }
  riemann_contact(g, d, UL, aL, UR, aR, FoL, ufL, FrL);
  for (int k = 0; k < nf; ++k) FoR[k] = FoL[k];
  *ufR = *ufL;
  for (int j = 0; j < 3; ++j) FrR[j] = FrL[j];
}

/* ------------------------------------------------------------------------ */
/* Reconstruction: van Leer slopes on primitives (R9), positivity fallback   */
/* to first order (R10).                                                     */
/* ------------------------------------------------------------------------ */

static double van_leer(double a, double b) {
  if (a * b > 0.0) return 2.0 * a * b / (a + b);
  return 0.0;
}

/* Non-conservative terms, per unit of 1/dx: phi and X take q_c * du; the
 * deformation tensor takes 2/3 F_ij du - u_i dF_dj (Eq. for Vbar, R1, R20). */
static void noncons(const or_grid* g, int d, const double* wc, const aux_t* ac,
                    double du, const double dFrow[3], double* nc) {
  for (int k = 0; k < g->nfield; ++k) nc[k] = 0.0;
  for (int l = 0; l + 1 < g->nmat; ++l) nc[g->o_phi + l] = wc[g->o_phi + l] * du;
  for (int k = 0; k < g->dim; ++k) nc[g->o_X + k] = wc[g->o_X + k] * du;
  for (int c = 0; c < g->nF; ++c) {
    const int i = g->Fidx[c] / 3, j = g->Fidx[c] % 3;
    nc[g->o_F + c] = (2.0 / 3.0) * ac->F[3 * i + j] * du - ac->u[i] * dFrow[j];
  }
  (void)d;
}

/* A half step of length dt/2 changes the log of a phase density by
 * (dt/2) |du/dx| at most, and with dt <= cfl dx / S (S = max |u| + c_L over the
 * grid, |u_R - u_L| <= 2 S, cfl <= 1) that is at most 1.  A half-stepped face
 * state whose phase density differs from the reconstructed one by more than a
 * factor e is therefore not the half step's compression: it comes from the
 * near-cancelling increments of phi_l and phi_l rho_l where phi_l is a trace
 * fraction, and it is treated as inadmissible. */
static int phase_density_in_bound(const or_grid* g, const double* w_rec,
                                  const double* w_half) {
  const double e = 2.718281828459045;
  for (int l = 0; l < g->nmat; ++l) {
    const double r0 = w_rec[g->o_arho + l], r1 = w_half[g->o_arho + l];
    if (!(r1 <= e * r0 && r0 <= e * r1)) return 0;
  }
  return 1;
}

/* Face states of one cell after the MUSCL-Hancock half step.  Falls back to
 * the cell average on both faces when a state leaves the admissible set or a
 * phase density leaves the half step's bound (phase_density_in_bound). */
static int face_states(const or_grid* g, int d, double lam, const double* wm,
                       const double* wc, const double* wp, const double* uc,
                       const aux_t* ac, double* UL, aux_t* aL, double* UR,
                       aux_t* aR) {
  int bound = 0;
  double wL[MAXF], wR[MAXF];
  for (int k = 0; k < g->nfield; ++k) {
    const double s = van_leer(wc[k] - wm[k], wp[k] - wc[k]);
    wL[k] = wc[k] - 0.5 * s;
    wR[k] = wc[k] + 0.5 * s;
  }
  /* the limited slope keeps a face value between the neighbours' values up
   * to rounding; a void fraction next to a zero one can come out a rounding
   * below zero, which is zero (R33) */
  if (g->void_l >= 0) {
    if (wL[g->o_phi + g->void_l] < 0.0) wL[g->o_phi + g->void_l] = 0.0;
    if (wR[g->o_phi + g->void_l] < 0.0) wR[g->o_phi + g->void_l] = 0.0;
  }
  double uL0[MAXF], uR0[MAXF];
  aux_t xL, xR;
  int ok = w2u(g, wL, uL0, &xL) == 0 && w2u(g, wR, uR0, &xR) == 0;
  if (ok) {
    double FL[MAXF], FR[MAXF], nc[MAXF], dF[3];
    phys_flux(g, d, uL0, &xL, FL);
    phys_flux(g, d, uR0, &xR, FR);
    for (int j = 0; j < 3; ++j) dF[j] = xR.F[3 * d + j] - xL.F[3 * d + j];
    noncons(g, d, wc, ac, xR.u[d] - xL.u[d], dF, nc);
    double uL1[MAXF], uR1[MAXF], wL1[MAXF], wR1[MAXF];
    for (int k = 0; k < g->nfield; ++k) {
      const double inc = 0.5 * lam * ((FL[k] - FR[k]) + nc[k]);
      uL1[k] = uL0[k] + inc;
      uR1[k] = uR0[k] + inc;
    }
    /* the void fraction's trace transport can leave it a rounding below
     * zero in the half step too: zero, as in the update (R33) */
    if (g->void_l >= 0) {
      if (uL1[g->o_phi + g->void_l] < 0.0) uL1[g->o_phi + g->void_l] = 0.0;
      if (uR1[g->o_phi + g->void_l] < 0.0) uR1[g->o_phi + g->void_l] = 0.0;
    }
    ok = u2w(g, uL1, wL1, aL) == 0 && u2w(g, uR1, wR1, aR) == 0;
    if (ok && !(phase_density_in_bound(g, wL, wL1) && phase_density_in_bound(g, wR, wR1))) {
      ok = 0;
      bound = 1;
    }
    if (ok) {
      memcpy(UL, uL1, sizeof(double) * g->nfield);
      memcpy(UR, uR1, sizeof(double) * g->nfield);
      return 0;
    }
  }
  memcpy(UL, uc, sizeof(double) * g->nfield);
  memcpy(UR, uc, sizeof(double) * g->nfield);
  *aL = *ac;
  *aR = *ac;
  return bound;
}

/* ------------------------------------------------------------------------ */
/* Boundaries: two ghost cells per side along the sweep axis.               */
/* ------------------------------------------------------------------------ */

static void mirror_state(const or_grid* g, int d, double* u, double wall) {
  u[g->o_mom + d] = -u[g->o_mom + d];
  for (int c = 0; c < g->nF; ++c) {
    const int i = g->Fidx[c] / 3, j = g->Fidx[c] % 3;
    if ((i == d) != (j == d)) u[g->o_F + c] = -u[g->o_F + c];
  }
  u[g->o_X + d] = 2.0 * wall - u[g->o_X + d];
}

/* ext[c+2] holds cell c of the line, c = -2 .. n+1. */
static void fill_ghosts(const or_grid* g, int d, long n, double* ext) {
  const int nf = g->nfield;
  const double L = g->hi[d] - g->lo[d];
  for (int side = 0; side < 2; ++side) {
    for (int m = 0; m < 2; ++m) {
      double* dst = side == 0 ? ext + (size_t)(1 - m) * nf
                              : ext + (size_t)(n + 2 + m) * nf;
      const int bc = g->bc[d][side];
      long src;
      if (bc == OR_BC_PERIODIC)
        src = side == 0 ? n - 1 - m : m;
      else if (bc == OR_BC_REFLECTIVE)
        src = side == 0 ? m : n - 1 - m;
      else
        src = side == 0 ? 0 : n - 1;
      if (src < 0) src = 0;
      if (src > n - 1) src = n - 1;
      memcpy(dst, ext + (size_t)(src + 2) * nf, sizeof(double) * nf);
      if (bc == OR_BC_PERIODIC)
        dst[g->o_X + d] += side == 0 ? -L : L;
      else if (bc == OR_BC_REFLECTIVE)
        mirror_state(g, d, dst, side == 0 ? g->lo[d] : g->hi[d]);
    }
  }
}

/* ------------------------------------------------------------------------ */
/* One sweep along axis d over one line of cells.                            */
/* ------------------------------------------------------------------------ */

static long line_stride(const or_grid* g, int d) {
  return d == 0 ? 1 : (d == 1 ? g->n[0] : g->n[0] * g->n[1]);
}

static long line_base(const or_grid* g, int d, long line) {
  if (d == 0) return line * g->n[0];
  if (d == 1) {
    const long i = line % g->n[0], k = line / g->n[0];
    return i + k * g->n[0] * g->n[1];
  }
  return line;
}

static int sweep_line(const or_grid* g, int d, double dt, long line,
                      long* bad, long* nbound) {
  const long n = g->n[d];
  const int nf = g->nfield;
  const long base = line_base(g, d, line), stride = line_stride(g, d);
  const double lam = dt / g->dx[d];
  const size_t ne = (size_t)n + 4;
  double* ext = malloc(sizeof(double) * ne * nf);
  double* W = malloc(sizeof(double) * ne * nf);
  aux_t* A = malloc(sizeof(aux_t) * ne);
  double* FS = malloc(sizeof(double) * ne * 2 * nf); /* face states per cell */
  aux_t* FA = malloc(sizeof(aux_t) * ne * 2);
  /* face records as the cell left of the face sees them, then as the cell
   * right of it sees them (the two differ only where the void opens) */
  double* FX = malloc(sizeof(double) * ne * nf * 2); /* face fluxes */
  double* UF = malloc(sizeof(double) * ne * 2);      /* face velocity */
  double* FR = malloc(sizeof(double) * ne * 6);      /* face Fbar row d */
  double* FXr = FX + ne * nf;
  double* UFr = UF + ne;
  double* FRr = FR + ne * 3;
  int rc = OR_OK;
  for (long c = 0; c < n; ++c)
    for (int k = 0; k < nf; ++k)
      ext[(size_t)(c + 2) * nf + k] = g->U[(size_t)k * g->ncell + base + c * stride];
  fill_ghosts(g, d, n, ext);
  /* 1. primitive recovery on every cell of the extended line */
  for (size_t e = 0; e < ne; ++e) {
    if (u2w(g, ext + e * nf, W + e * nf, &A[e]) != 0) {
      long c = (long)e - 2;
      if (c < 0) c = 0;
      if (c > n - 1) c = n - 1;
      *bad = base + c * stride;
      rc = OR_ENONFINITE;
      goto done;
    }
  }
  /* 2. reconstruction + half step on cells -1 .. n (ext 1 .. n+2) */
  for (size_t e = 1; e <= (size_t)n + 2; ++e) {
    *nbound += face_states(g, d, lam, W + (e - 1) * nf, W + e * nf, W + (e + 1) * nf,
                           ext + e * nf, &A[e], FS + (2 * e) * nf, &FA[2 * e],
                           FS + (2 * e + 1) * nf, &FA[2 * e + 1]);
  }
  /* 3. HLLC on faces between ext e and e+1, e = 1 .. n+1 */
  for (size_t e = 1; e <= (size_t)n + 1; ++e) {
    riemann(g, d, FS + (2 * e + 1) * nf, &FA[2 * e + 1], FS + (2 * (e + 1)) * nf,
            &FA[2 * (e + 1)], FX + e * nf, &UF[e], FR + 3 * e, FXr + e * nf, &UFr[e],
            FRr + 3 * e);
  }
  /* 4. update of cells 0 .. n-1 (ext 2 .. n+1): face e-1 is left, e right;
   * the cell takes the right-cell record of its left face and the
   * left-cell record of its right face */
  for (size_t e = 2; e <= (size_t)n + 1; ++e) {
    const double* uc = ext + e * nf;
    const double du = UF[e] - UFr[e - 1];
    double dF[3], nc[MAXF];
    for (int j = 0; j < 3; ++j) dF[j] = FR[3 * e + j] - FRr[3 * (e - 1) + j];
    noncons(g, d, W + e * nf, &A[e], du, dF, nc);
    const long cell = base + ((long)e - 2) * stride;
    for (int k = 0; k < nf; ++k)
      g->V[(size_t)k * g->ncell + cell] =
          uc[k] + lam * ((FXr[(e - 1) * nf + k] - FX[e * nf + k]) + nc[k]);
    /* the void fraction is created only where the void opens; its transport
     * of traces (ahead of an opening crack it falls off to 1e-300 and
     * below) can leave it a rounding below zero, which is taken as zero */
    if (g->void_l >= 0) {
      double* nu = &g->V[(size_t)(g->o_phi + g->void_l) * g->ncell + cell];
      if (*nu < 0.0) *nu = 0.0;
    }
  }
done:
  free(ext); free(W); free(A); free(FS); free(FA); free(FX); free(UF); free(FR);
  return rc;
}

static int sweep(or_grid* g, int d, double dt) {
  const long nlines = g->ncell / g->n[d];
  int rc = OR_OK;
  long bad = -1, nb = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : nb)
  for (long line = 0; line < nlines; ++line) {
    long b = -1;
    const int r = sweep_line(g, d, dt, line, &b, &nb);
    if (r != OR_OK) {
#pragma omp critical
      {
        if (rc == OR_OK || b < bad) { rc = r; bad = b; }
      }
    }
  }
  if (rc != OR_OK) {
    g->bad_cell = bad;
    return rc;
  }
  g->nbound += nb;
  double* t = g->U;
  g->U = g->V;
  g->V = t;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Lagrangian coordinates by third-order WENO and three-stage RK (Sec.      */
/* 3.2.1), the alternative to carrying X in the sweeps (R28):               */
/*   dX/dt = -sum_d [u_{d,i+1/2} (X_{i+1/2} - X_i)                          */
/*                   - u_{d,i-1/2} (X_{i-1/2} - X_i)] / dx_d,                */
/* the difference of the fluxes X u_d plus X div(u), so that DX/Dt = 0.     */
/* Face velocity: mean of the two cell velocities.  Face value of X: the    */
/* WENO3 value reconstructed in the upwind cell.  Time: Shu and Osher's     */
/* three-stage TVD Runge-Kutta scheme with the velocities of the step's     */
/* start.  Ghost cells follow the rules of the sweeps.                       */
/* ------------------------------------------------------------------------ */

/* WENO3 value at the face between cells b and c, reconstructed in cell b
   from its neighbours a (away from the face) and c (across it): candidates
   -a/2 + 3b/2 and (b + c)/2, linear weights 1/3 and 2/3, smoothness
   ((b - a)/dx)^2 and ((c - b)/dx)^2, eps = 1e-6 (Jiang and Shu). */
static double weno3_face(double a, double b, double c, double dx) {
  const double q0 = -0.5 * a + 1.5 * b;
  const double q1 = 0.5 * b + 0.5 * c;
  const double s0 = (b - a) / dx, s1 = (c - b) / dx;
  const double e0 = 1e-6 + s0 * s0, e1 = 1e-6 + s1 * s1;
  const double a0 = (1.0 / 3.0) / (e0 * e0);
  const double a1 = (2.0 / 3.0) / (e1 * e1);
  return (a0 * q0 + a1 * q1) / (a0 + a1);
}

/* Component k of X and velocity u_d of the cell o steps along axis d from
   the cell at linear index cell (coordinate i along d), ghosts included. */
static void x_at(const or_grid* g, const double* X, const double* vel, long cell,
                 long i, int d, int o, int k, double* Xk, double* ud) {
  const long n = g->n[d], stride = line_stride(g, d);
  long j = i + o;
  double shift = 0.0;
  int mirror = 0, side = 0;
  if (j < 0 || j >= n) {
    side = j < 0 ? 0 : 1;
    const int bc = g->bc[d][side];
    if (bc == OR_BC_PERIODIC) {
      shift = side == 0 ? -(g->hi[d] - g->lo[d]) : (g->hi[d] - g->lo[d]);
      j = side == 0 ? j + n : j - n;
    } else if (bc == OR_BC_REFLECTIVE) {
      mirror = 1;
      j = side == 0 ? -1 - j : 2 * n - 1 - j;
    } else {
      j = side == 0 ? 0 : n - 1;
    }
  }
  const long src = cell + (j - i) * stride;
  *Xk = X[(size_t)k * g->ncell + src];
  *ud = vel[(size_t)d * g->ncell + src];
  if (k == d) {
    if (mirror) *Xk = 2.0 * (side == 0 ? g->lo[d] : g->hi[d]) - *Xk;
    *Xk += shift;
  }
  if (mirror) *ud = -*ud;
}

/* The right-hand side of dX_k/dt at one cell. */
static double x_rhs(const or_grid* g, const double* X, const double* vel, long cell, int k) {
  long idx[3] = {cell % g->n[0], (cell / g->n[0]) % g->n[1], cell / (g->n[0] * g->n[1])};
  double L = 0.0;
  for (int d = 0; d < g->dim; ++d) {
    double x[5], u[5];
    for (int o = -2; o <= 2; ++o) x_at(g, X, vel, cell, idx[d], d, o, k, &x[o + 2], &u[o + 2]);
    const double uL = 0.5 * (u[1] + u[2]), uR = 0.5 * (u[2] + u[3]);
    const double XR = uR >= 0.0 ? weno3_face(x[1], x[2], x[3], g->dx[d])
                                : weno3_face(x[4], x[3], x[2], g->dx[d]);
    const double XL = uL >= 0.0 ? weno3_face(x[0], x[1], x[2], g->dx[d])
                                : weno3_face(x[3], x[2], x[1], g->dx[d]);
    L -= (uR * (XR - x[2]) - uL * (XL - x[2])) / g->dx[d];
  }
  return L;
}

/* X at the end of a step of length dt from the present state, into Xn
   ([dim][ncell]). */
static int x_weno_rk3(const or_grid* g, double dt, double* Xn) {
  const long nc = g->ncell;
  const size_t sz = sizeof(double) * (size_t)g->dim * nc;
  double* vel = malloc(sz);
  double* X0 = malloc(sz);
  double* X1 = malloc(sz);
  double* X2 = malloc(sz);
  if (!vel || !X0 || !X1 || !X2) {
    free(vel); free(X0); free(X1); free(X2);
    return OR_EINVAL;
  }
#pragma omp parallel for
  for (long c = 0; c < nc; ++c) {
    double rho = 0.0;
    for (int l = 0; l < g->nmat; ++l) rho += g->U[(size_t)(g->o_arho + l) * nc + c];
    for (int d = 0; d < g->dim; ++d) {
      vel[(size_t)d * nc + c] = g->U[(size_t)(g->o_mom + d) * nc + c] / rho;
      X0[(size_t)d * nc + c] = g->U[(size_t)(g->o_X + d) * nc + c];
    }
  }
#pragma omp parallel for
  for (long c = 0; c < nc; ++c)
    for (int k = 0; k < g->dim; ++k)
      X1[(size_t)k * nc + c] = X0[(size_t)k * nc + c] + dt * x_rhs(g, X0, vel, c, k);
#pragma omp parallel for
  for (long c = 0; c < nc; ++c)
    for (int k = 0; k < g->dim; ++k) {
      const size_t q = (size_t)k * nc + c;
      X2[q] = 0.75 * X0[q] + 0.25 * (X1[q] + dt * x_rhs(g, X1, vel, c, k));
    }
#pragma omp parallel for
  for (long c = 0; c < nc; ++c)
    for (int k = 0; k < g->dim; ++k) {
      const size_t q = (size_t)k * nc + c;
      Xn[q] = (1.0 / 3.0) * X0[q] + (2.0 / 3.0) * (X2[q] + dt * x_rhs(g, X2, vel, c, k));
    }
  free(vel); free(X0); free(X1); free(X2);
  return OR_OK;
}

int or_set_x_scheme(or_grid* g, int scheme) {
  if (!g || scheme < 0 || scheme > 1) return OR_EINVAL;
  g->xscheme = scheme;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Perturbation field phi(x,t) = phi0(X(x,t)) (Eq. for phi, Sec. 3.2.2):    */
/* multilinear interpolation on the lattice, 1 outside it (R13).            */
/* ------------------------------------------------------------------------ */

double or_lookup(int dim, const float* phi0, const long pn[3],
                 const double plo[3], const double ph[3], const double X[3]) {
  if (!phi0) return 1.0;
  long i0[3] = {0, 0, 0};
  double w[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < dim; ++k) {
    const double s = (X[k] - plo[k]) / ph[k];
    if (!(s >= 0.0) || !(s <= (double)(pn[k] - 1))) return 1.0;
    long i = (long)floor(s);
    if (i > pn[k] - 2) i = pn[k] - 2;
    i0[k] = i;
    w[k] = s - (double)i;
  }
  double v = 0.0;
  const int corners = 1 << dim;
  for (int c = 0; c < corners; ++c) {
    double wt = 1.0;
    long idx = 0, str = 1;
    for (int k = 0; k < dim; ++k) {
      const int b = (c >> k) & 1;
      wt *= b ? w[k] : 1.0 - w[k];
      idx += (i0[k] + b) * str;
      str *= pn[k];
    }
    v += wt * (double)phi0[idx];
  }
  return v;
}

/* ------------------------------------------------------------------------ */
/* Damage (Sec. 2.1.1: Bonora rate, Pirondi-Bonora gate, threshold;         */
/* Sec. 4.3: simple model), RK4 over the step (Sec. 3.1).                    */
/* ------------------------------------------------------------------------ */

/* Triaxiality-dependent threshold plastic strain (Eq. after the gate).
 * Pinned by two closed forms: it reduces to eps_thresh at R_t = 1, and it
 * tends to eps_thresh R_t^(-1/(2n)) as eps_crit -> eps_thresh for any R_t
 * (every power in it enters that limit). */
double or_eps_thresh(double eps_t, double eps_c, double n, double Rt) {
  const double num = pow(eps_c, 2.0 * n) - pow(eps_t, 2.0 * n);
  const double den = pow(eps_c, 2.0 * n / Rt) - pow(eps_t, 2.0 * n / Rt);
  return pow(eps_t, 1.0 / Rt) / pow(Rt, 1.0 / n) * pow(num / den, 1.0 / (2.0 * n));
}

/* Stress triaxiality function, first form with the hydrostatic pressure
 * (the R_t printed with rho0/rho, used with p instead of p_c, R17). */
double or_Rt(double poisson, double rho0, double rho, double p, double seq) {
  const double x = p / seq;
  return 2.0 / 3.0 * (1.0 + poisson) +
         3.0 * (1.0 - 2.0 * poisson) * (rho0 / rho) * (x * x);
}

static double damage_rate(const or_material* m, double D, double eps,
                          double epsdot, double p, double Rt, double thresh) {
  if (m->damage == 2) return m->Ddot0 * (1.0 - D) * epsdot;
  /* Bonora, D0 = 0 (R18); active only under tension above threshold */
  if (!(p < 0.0) || !(eps > thresh)) return 0.0;
  if (D >= m->D_crit) return 0.0;
  const double aD = m->alpha_D, Dc = m->D_crit;
  return aD * pow(Dc, 1.0 / aD) / log(m->eps_c / m->eps_t) * Rt *
         pow(Dc - D, (aD - 1.0) / aD) * epsdot / eps;
}

double or_damage_rk4(const or_material* m, double D, double eps0, double deps,
                     double dt, double p, double seq, double rho) {
  if (m->damage == 0 || !(deps > 0.0)) return D;
  double Rt = 1.0, thresh = 0.0;
  if (m->damage == 1) {
    if (!(seq > 0.0)) return D;
    Rt = or_Rt(m->poisson, m->rho0, rho, p, seq);
    thresh = or_eps_thresh(m->eps_t, m->eps_c, m->n_hard, Rt);
  }
  const double ed = deps / dt;
  const double k1 = damage_rate(m, D, eps0, ed, p, Rt, thresh);
  const double k2 = damage_rate(m, D + 0.5 * dt * k1, eps0 + 0.5 * deps, ed, p, Rt, thresh);
  const double k3 = damage_rate(m, D + 0.5 * dt * k2, eps0 + 0.5 * deps, ed, p, Rt, thresh);
  const double k4 = damage_rate(m, D + dt * k3, eps0 + deps, ed, p, Rt, thresh);
  double Dn = D + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4);
  if (Dn < 0.0) Dn = 0.0;
  if (Dn > m->D_crit) Dn = m->D_crit;
  return Dn;
}

/* ------------------------------------------------------------------------ */
/* Plastic return (Phi of Sec. 2.1 with chi -> infinity, R15): radial return */
/* in Hencky space to the perturbed, damaged Johnson-Cook yield stress      */
/* sigma'_Y = phi sigma_Y (Eq. perturbed yield), (1-D) (Sec. 2.1.1), and 0  */
/* at critical damage (Sec. 3.1).                                            */
/* ------------------------------------------------------------------------ */

static double yield_mix(const or_material* mats, int nmat, const double* phi,
                        const double* eps, const double* D, double phihat,
                        double dt, double dl, double* dY) {
  double Y = 0.0, dYs = 0.0;
  for (int l = 0; l < nmat; ++l) {
    const or_material* m = &mats[l];
    if (m->plasticity != 1) continue;
    if (is_critical(m, D[l])) continue;
    const double psi = is_damaged(m) ? 1.0 - D[l] : 1.0;
    /* advection can leave a rounding-level negative plastic strain; the
     * hardening law sees it as zero (R27) */
    const double e = (eps[l] > 0.0 ? eps[l] : 0.0) + dl;
    double hard = m->c1, dhard = 0.0;
    if (m->c2 != 0.0) {
      hard += m->c2 * pow(e, m->n_hard);
      if (e > 0.0) dhard = m->c2 * m->n_hard * pow(e, m->n_hard - 1.0);
    }
    double R = 1.0, dR = 0.0;
    if (m->c3 != 0.0 && dl > 0.0) {
      const double r = 1.0 + m->c3 * log(dl / (dt * m->edot0));
      if (r > 1.0) {
        R = r;
        dR = m->c3 / dl;
      }
    }
    const double wgt = phi[l] * phihat * psi;
    Y += wgt * hard * R;
    dYs += wgt * (dhard * R + hard * dR);
  }
  if (dY) *dY = dYs;
  return Y;
}

/* Solve sigma_tr - 3 G dl - Y(dl) = 0 for the plastic increment dl >= 0. */
static int return_increment(const or_material* mats, int nmat,
                            const double* phi, const double* eps,
                            const double* D, double phihat, double dt,
                            double G, double str, double* dl_out) {
  const double Y0 = yield_mix(mats, nmat, phi, eps, D, phihat, dt, 0.0, NULL);
  if (!(str > Y0)) {
    *dl_out = 0.0;
    return OR_OK;
  }
  /* Safeguarded Newton on the bracket [0, sigma_tr/(3G)], iterated down to
   * the rounding floor: the residual is a difference of terms no larger than
   * sigma_tr, so |g| <= 8 eps sigma_tr is converged; so is a step below the
   * rounding scale of the bracket. */
  const double b0 = str / (3.0 * G);
  double a = 0.0, b = b0;
  double dl = (str - Y0) / (3.0 * G);
  for (int it = 0; it < 200; ++it) {
    double dY;
    const double Y = yield_mix(mats, nmat, phi, eps, D, phihat, dt, dl, &dY);
    const double gv = str - 3.0 * G * dl - Y;
    if (fabs(gv) <= 8.0 * DBL_EPSILON * str) {
      *dl_out = dl;
      return OR_OK;
    }
    if (gv > 0.0) a = dl; else b = dl;
    double nx = dl - gv / (-3.0 * G - dY);
    if (!(nx > a && nx < b)) nx = 0.5 * (a + b);
    if (fabs(nx - dl) <= 4.0 * DBL_EPSILON * b0) {
      *dl_out = nx;
      return OR_OK;
    }
    dl = nx;
  }
  return OR_ENOCONV;
}

static double det3(const double F[9]) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* F <- exp((k-1) devH) F = Q diag(exp((k-1) h)) Q^T F */
static void scale_stretch(double F[9], const double Q[9], const double h[3],
                          double k) {
  double m[3], S[9], out[9];
  for (int i = 0; i < 3; ++i) m[i] = exp((k - 1.0) * h[i]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      S[3 * i + j] = Q[3 * i + 0] * m[0] * Q[3 * j + 0] +
                     Q[3 * i + 1] * m[1] * Q[3 * j + 1] +
                     Q[3 * i + 2] * m[2] * Q[3 * j + 2];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      out[3 * i + j] = S[3 * i + 0] * F[0 + j] + S[3 * i + 1] * F[3 + j] +
                       S[3 * i + 2] * F[6 + j];
  memcpy(F, out, sizeof out);
}

/* Shear modulus of the mixture G_mix = sum phi_l G_l and whether the cell
 * may yield (every material with G0 > 0 has a plasticity model). */
static int mix_shear(const or_material* mats, int nmat, const double* phi,
                     const double* rho, const double* D, double* Gmix) {
  int can_yield = 1;
  *Gmix = 0.0;
  for (int l = 0; l < nmat; ++l) {
    double th[6];
    const double psi = is_damaged(&mats[l]) ? 1.0 - D[l] : 1.0;
    or_thermo(&mats[l], rho[l], psi, 0.0, th);
    *Gmix += phi[l] * th[3];
    if (mats[l].eos == 1 && mats[l].G0 > 0.0 && mats[l].plasticity != 1)
      can_yield = 0;
  }
  return can_yield;
}

int or_plastic_return_cell(const or_material* mats, int nmat,
                           const double* phi, const double* rho,
                           const double* eps, const double* D, double phihat,
                           double dt, double F[9], double* dEps) {
  double Gm;
  const int can_yield = mix_shear(mats, nmat, phi, rho, D, &Gm);
  const double dt3 = cbrt(det3(F));
  for (int k = 0; k < 9; ++k) F[k] /= dt3;
  *dEps = 0.0;
  if (!can_yield || !(Gm > 0.0)) return OR_OK;
  double devH[9], h[3], Q[9], lam[3];
  if (hencky_eig(F, devH, h, Q, lam) != 0) return OR_ENONFINITE;
  const double J = sqrt(h[0] * h[0] + h[1] * h[1] + h[2] * h[2]);
  const double str = sqrt(6.0) * Gm * J;
  double dl;
  const int rc = return_increment(mats, nmat, phi, eps, D, phihat, dt, Gm, str, &dl);
  if (rc != OR_OK) return rc;
  if (dl > 0.0) {
    const double k = (str - 3.0 * Gm * dl) / str;
    scale_stretch(F, Q, h, k);
  }
  *dEps = dl;
  return OR_OK;
}

/* Sources of one cell after the sweeps (R12). */
static int source_cell(or_grid* g, long cell, double dt) {
  double u[MAXF], w[MAXF];
  aux_t ax;
  for (int k = 0; k < g->nfield; ++k) u[k] = g->U[(size_t)k * g->ncell + cell];
  if (u2w(g, u, w, &ax) != 0) return OR_ENONFINITE;
  double phi[OR_MAXMAT], rho[OR_MAXMAT], eps[OR_MAXMAT], D[OR_MAXMAT];
  vol_fracs(g, u, phi);
  for (int l = 0; l < g->nmat; ++l) {
    rho[l] = w[g->o_arho + l];
    const int h = g->hslot[l];
    eps[l] = h >= 0 ? w[g->o_hist + 2 * h] : 0.0;
    D[l] = h >= 0 ? w[g->o_hist + 2 * h + 1] : 0.0;
  }
  double X[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < g->dim; ++k) X[k] = w[g->o_X + k];
  const double phihat = or_lookup(g->dim, g->phi0, g->pn, g->plo, g->ph, X);
  double F[9];
  full_F(g, u, F);
  double dl;
  const int rc = or_plastic_return_cell(g->mat, g->nmat, phi, rho, eps, D,
                                        phihat, dt, F, &dl);
  if (rc != OR_OK) return rc;
  for (int c = 0; c < g->nF; ++c) u[g->o_F + c] = F[g->Fidx[c]];
  if (dl > 0.0) {
    /* pressure and equivalent stress of the returned state for the damage law */
    double ws[MAXF];
    aux_t as;
    if (u2w(g, u, ws, &as) != 0) return OR_ENONFINITE;
    mix_t mx;
    if (mixture(g, phi, rho, D, F, &mx) != 0) return OR_ENONFINITE;
    const double seq = sqrt(6.0) * mx.Gmix * sqrt(mx.J2);
    for (int l = 0; l < g->nmat; ++l) {
      const int h = g->hslot[l];
      if (h < 0) continue;
      const double arho = u[g->o_arho + l];
      const double Dn = or_damage_rk4(&g->mat[l], D[l], eps[l], dl, dt, as.p,
                                      seq, rho[l]);
      u[g->o_hist + 2 * h] = arho * (eps[l] + dl);
      u[g->o_hist + 2 * h + 1] = arho * Dn;
    }
  }
  for (int k = 0; k < g->nfield; ++k) g->U[(size_t)k * g->ncell + cell] = u[k];
  return OR_OK;
}

static int sources(or_grid* g, double dt) {
  int rc = OR_OK;
  long bad = -1;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->ncell; ++c) {
    const int r = source_cell(g, c, dt);
    if (r != OR_OK) {
#pragma omp critical
      {
        if (rc == OR_OK || c < bad) { rc = r; bad = c; }
      }
    }
  }
  if (rc != OR_OK) g->bad_cell = bad;
  return rc;
}

/* ------------------------------------------------------------------------ */
/* CFL time step: dt = cfl * min_d dx_d / max_cells (max_d |u_d| + c_L).    */
/* ------------------------------------------------------------------------ */

int or_cfl_dt(or_grid* g, double cfl, double* dt, double* smax) {
  double s = 0.0;
  int rc = OR_OK;
  long bad = -1;
#pragma omp parallel for reduction(max : s) schedule(static)
  for (long c = 0; c < g->ncell; ++c) {
    double u[MAXF], w[MAXF];
    aux_t ax;
    for (int k = 0; k < g->nfield; ++k) u[k] = g->U[(size_t)k * g->ncell + c];
    if (u2w(g, u, w, &ax) != 0) {
#pragma omp critical
      {
        if (rc == OR_OK || c < bad) { rc = OR_ENONFINITE; bad = c; }
      }
      continue;
    }
    double v = 0.0;
    for (int k = 0; k < g->dim; ++k) {
      const double a = fabs(ax.u[k]);
      if (a > v) v = a;
    }
    v += ax.cL;
    if (v > s) s = v;
  }
  if (rc != OR_OK) {
    g->bad_cell = bad;
    return rc;
  }
  double dxm = g->dx[0];
  for (int k = 1; k < g->dim; ++k)
    if (g->dx[k] < dxm) dxm = g->dx[k];
  *smax = s;
  *dt = cfl * dxm / s;
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* API                                                                       */
/* ------------------------------------------------------------------------ */

void or_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int or_nfield(const or_grid* g) { return g->nfield; }
long or_ncell(const or_grid* g) { return g->ncell; }

or_grid* or_create(int dim, const long n[3], const double lo[3],
                   const double hi[3], const int bc[6], int nmat,
                   const or_material* mats, const double* prim,
                   const float* phi0, const long pn[3], const double plo[3],
                   const double ph[3], int* status) {
  *status = OR_EINVAL;
  if (dim < 1 || dim > 3 || nmat < 1 || nmat > OR_MAXMAT) return NULL;
  or_grid* g = calloc(1, sizeof(or_grid));
  g->dim = dim;
  g->nmat = nmat;
  g->ncell = 1;
  for (int k = 0; k < 3; ++k) {
    g->n[k] = k < dim ? n[k] : 1;
    g->lo[k] = k < dim ? lo[k] : 0.0;
    g->hi[k] = k < dim ? hi[k] : 1.0;
    g->dx[k] = (g->hi[k] - g->lo[k]) / (double)g->n[k];
    g->ncell *= g->n[k];
    g->bc[k][0] = k < dim ? bc[2 * k] : 0;
    g->bc[k][1] = k < dim ? bc[2 * k + 1] : 0;
    if (k < dim && g->n[k] < 2) { free(g); return NULL; }
  }
  g->nhist = 0;
  g->void_l = -1;
  g->seed_x = 1;
  for (int l = 0; l < nmat; ++l) {
    g->mat[l] = mats[l];
    g->hslot[l] = mats[l].plasticity == 1 ? g->nhist++ : -1;
    if (mats[l].eos == 2) {
      /* one void at most, never the last material (whose fraction is
       * formed as one minus the others), with no strength or damage model */
      if (g->void_l >= 0 || l == nmat - 1 || mats[l].plasticity != 0 || mats[l].damage != 0) {
        free(g);
        return NULL;
      }
      g->void_l = l;
    }
  }
  static const int F1[] = {0, 4, 8};
  static const int F2[] = {0, 1, 3, 4, 8};
  g->nF = dim == 1 ? 3 : (dim == 2 ? 5 : 9);
  for (int c = 0; c < g->nF; ++c)
    g->Fidx[c] = dim == 1 ? F1[c] : (dim == 2 ? F2[c] : c);
  g->o_phi = 0;
  g->o_arho = nmat - 1;
  g->o_mom = g->o_arho + nmat;
  g->o_E = g->o_mom + dim;
  g->o_F = g->o_E + 1;
  g->o_hist = g->o_F + g->nF;
  g->o_X = g->o_hist + 2 * g->nhist;
  g->nfield = g->o_X + dim;
  g->U = malloc(sizeof(double) * g->nfield * g->ncell);
  g->V = malloc(sizeof(double) * g->nfield * g->ncell);
  if (phi0) {
    long np = 1;
    for (int k = 0; k < dim; ++k) {
      g->pn[k] = pn[k];
      g->plo[k] = plo[k];
      g->ph[k] = ph[k];
      np *= pn[k];
    }
    g->phi0 = malloc(sizeof(float) * np);
    memcpy(g->phi0, phi0, sizeof(float) * np);
  }
  g->bad_cell = -1;
  long bad = -1;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->ncell; ++c) {
    double w[MAXF], u[MAXF];
    aux_t ax;
    for (int k = 0; k < g->nfield; ++k) w[k] = prim[(size_t)k * g->ncell + c];
    if (w2u(g, w, u, &ax) != 0) {
#pragma omp critical
      {
        if (bad < 0 || c < bad) bad = c;
      }
    }
    for (int k = 0; k < g->nfield; ++k) g->U[(size_t)k * g->ncell + c] = u[k];
  }
  g->bad_cell = bad;
  *status = bad >= 0 ? OR_ENONFINITE : OR_OK;
  return g;
}

void or_destroy(or_grid* g) {
  if (!g) return;
  free(g->U);
  free(g->V);
  free(g->phi0);
  free(g);
}

/* ------------------------------------------------------------------------ */
/* Lagrangian seeding into void (Sec. 3.2.1 seeding routine, R35): in each  */
/* cell with nu > 1/2 and a normal, |grad nu| h > 1e-6 (h the largest cell  */
/* size; a void of uniform fraction up to rounding has none), the unit      */
/* normal n = -grad nu / |grad nu| (central differences; it points from    */
/* the void into the material), a probe at                                  */
/* p = c + 1.5 h n (c the cell centre) and                                  */
/* X_new = X(p) - (p - c), X(p) multilinear in the cell-centred X.  All     */
/* cells read the X of the step's start (the new values are written after   */
/* every cell is computed).  Cells outside the grid follow the sweeps'      */
/* ghost rules: periodic wraps (X shifted by the period), reflective        */
/* mirrors (X_d reflected about the wall), transmissive copies the edge.    */
/* ------------------------------------------------------------------------ */

/* Cell index i along d (at most two cells outside the grid) mapped into the
 * grid; *shift and *mirror say how X_d of that cell maps to the ghost. */
static long ghost_map(const or_grid* g, int d, long i, double* shift, int* mirror,
                      double* wall) {
  const long n = g->n[d];
  *shift = 0.0;
  *mirror = 0;
  *wall = 0.0;
  if (i >= 0 && i < n) return i;
  const int side = i < 0 ? 0 : 1;
  const int bc = g->bc[d][side];
  if (bc == OR_BC_PERIODIC) {
    *shift = side == 0 ? -(g->hi[d] - g->lo[d]) : (g->hi[d] - g->lo[d]);
    return side == 0 ? i + n : i - n;
  }
  if (bc == OR_BC_REFLECTIVE) {
    *mirror = 1;
    *wall = side == 0 ? g->lo[d] : g->hi[d];
    return side == 0 ? -1 - i : 2 * n - 1 - i;
  }
  return side == 0 ? 0 : n - 1;
}

static double void_at(const or_grid* g, const long ix[3]) {
  long j[3];
  for (int d = 0; d < 3; ++d) {
    double s, w;
    int m;
    j[d] = d < g->dim ? ghost_map(g, d, ix[d], &s, &m, &w) : 0;
  }
  const long c = j[0] + g->n[0] * (j[1] + g->n[1] * j[2]);
  return g->U[(size_t)(g->o_phi + g->void_l) * g->ncell + c];
}

/* X of the cell at integer position ix (ghosts by the rules above). */
static void x_of(const or_grid* g, const double* Xs, const long ix[3], double X[3]) {
  long j[3];
  double shift[3] = {0.0, 0.0, 0.0}, wall[3] = {0.0, 0.0, 0.0};
  int mirror[3] = {0, 0, 0};
  for (int d = 0; d < 3; ++d)
    j[d] = d < g->dim ? ghost_map(g, d, ix[d], &shift[d], &mirror[d], &wall[d]) : 0;
  const long c = j[0] + g->n[0] * (j[1] + g->n[1] * j[2]);
  for (int k = 0; k < g->dim; ++k) {
    double x = Xs[(size_t)k * g->ncell + c];
    if (mirror[k]) x = 2.0 * wall[k] - x;
    X[k] = x + shift[k];
  }
}

int or_seed_x(or_grid* g) {
  if (g->void_l < 0) return OR_OK;
  const int dim = g->dim;
  const size_t nX = (size_t)dim * g->ncell;
  double* Xs = malloc(sizeof(double) * nX);
  double* Xn = malloc(sizeof(double) * nX);
  if (!Xs || !Xn) {
    free(Xs);
    free(Xn);
    return OR_EINVAL;
  }
  memcpy(Xs, g->U + (size_t)g->o_X * g->ncell, sizeof(double) * nX);
  memcpy(Xn, Xs, sizeof(double) * nX);
  double h = 0.0;
  for (int d = 0; d < dim; ++d) h = g->dx[d] > h ? g->dx[d] : h;
#pragma omp parallel for schedule(static)
  for (long c = 0; c < g->ncell; ++c) {
    const long ix[3] = {c % g->n[0], (c / g->n[0]) % g->n[1], c / (g->n[0] * g->n[1])};
    if (!(void_at(g, ix) > 0.5)) continue;
    double gr[3] = {0.0, 0.0, 0.0}, gn = 0.0;
    for (int d = 0; d < dim; ++d) {
      long a[3] = {ix[0], ix[1], ix[2]}, b[3] = {ix[0], ix[1], ix[2]};
      a[d] -= 1;
      b[d] += 1;
      gr[d] = (void_at(g, b) - void_at(g, a)) / (2.0 * g->dx[d]);
      gn += gr[d] * gr[d];
    }
    gn = sqrt(gn);
    if (!(gn * h > 1e-6)) continue;
    double cc[3], p[3], f[3];
    long i0[3] = {0, 0, 0};
    for (int d = 0; d < dim; ++d) {
      cc[d] = g->lo[d] + ((double)ix[d] + 0.5) * g->dx[d];
      p[d] = cc[d] + 1.5 * h * (-gr[d] / gn);
      const double s = (p[d] - g->lo[d]) / g->dx[d] - 0.5;
      const double fl = floor(s);
      i0[d] = (long)fl;
      f[d] = s - fl;
    }
    double Xi[3] = {0.0, 0.0, 0.0};
    for (int corner = 0; corner < (1 << dim); ++corner) {
      long q[3] = {0, 0, 0};
      double w = 1.0;
      for (int d = 0; d < dim; ++d) {
        const int b = (corner >> d) & 1;
        q[d] = i0[d] + b;
        w *= b ? f[d] : 1.0 - f[d];
      }
      double Xq[3];
      x_of(g, Xs, q, Xq);
      for (int k = 0; k < dim; ++k) Xi[k] += w * Xq[k];
    }
    for (int k = 0; k < dim; ++k) Xn[(size_t)k * g->ncell + c] = Xi[k] - (p[k] - cc[k]);
  }
  memcpy(g->U + (size_t)g->o_X * g->ncell, Xn, sizeof(double) * nX);
  free(Xs);
  free(Xn);
  return OR_OK;
}

int or_set_seed_x(or_grid* g, int on) {
  if (on != 0 && on != 1) return OR_EINVAL;
  g->seed_x = on;
  return OR_OK;
}

int or_step(or_grid* g, int nsteps, double cfl, double dt_fixed, double* info) {
  int rc = OR_OK;
  for (int s = 0; s < nsteps; ++s) {
    double dt, smax = 0.0;
    /* X in the void from the material around it, before the step (R35) */
    if (g->void_l >= 0 && g->seed_x) {
      rc = or_seed_x(g);
      if (rc != OR_OK) break;
    }
    if (dt_fixed > 0.0) {
      dt = dt_fixed;
    } else {
      rc = or_cfl_dt(g, cfl, &dt, &smax);
      if (rc != OR_OK) break;
    }
    double* Xn = NULL;
    if (g->xscheme == 1) {
      /* X from the state at the step's start; the sweeps' X is replaced */
      Xn = malloc(sizeof(double) * (size_t)g->dim * g->ncell);
      rc = Xn ? x_weno_rk3(g, dt, Xn) : OR_EINVAL;
      if (rc != OR_OK) {
        free(Xn);
        break;
      }
    }
    for (int d = 0; d < g->dim && rc == OR_OK; ++d) rc = sweep(g, d, dt);
    if (Xn) {
      if (rc == OR_OK)
        memcpy(g->U + (size_t)g->o_X * g->ncell, Xn, sizeof(double) * (size_t)g->dim * g->ncell);
      free(Xn);
    }
    if (rc != OR_OK) break;
    rc = sources(g, dt);
    if (rc != OR_OK) break;
    g->t += dt;
    g->dt_last = dt;
    g->smax = smax;
    g->steps += 1;
  }
  if (info) {
    info[0] = g->t;
    info[1] = g->dt_last;
    info[2] = g->smax;
    info[3] = (double)g->steps;
    info[4] = (double)g->bad_cell;
    info[5] = (double)g->nbound;
  }
  return rc;
}

int or_read(const or_grid* g, int primitive, double* out) {
  if (!primitive) {
    memcpy(out, g->U, sizeof(double) * g->nfield * g->ncell);
    return OR_OK;
  }
  int rc = OR_OK;
  for (long c = 0; c < g->ncell; ++c) {
    double u[MAXF], w[MAXF];
    aux_t ax;
    for (int k = 0; k < g->nfield; ++k) u[k] = g->U[(size_t)k * g->ncell + c];
    if (u2w(g, u, w, &ax) != 0) rc = OR_ENONFINITE;
    for (int k = 0; k < g->nfield; ++k) out[(size_t)k * g->ncell + c] = w[k];
  }
  return rc;
}

int or_write_conserved(or_grid* g, const double* U) {
  memcpy(g->U, U, sizeof(double) * g->nfield * g->ncell);
  return OR_OK;
}

/* Totals sum dV (phi rho)_l, sum dV rho u (3 comps), sum dV rho E, each
 * with compensated (Kahan) summation. */
int or_totals(const or_grid* g, double* out) {
  double dV = 1.0;
  for (int k = 0; k < g->dim; ++k) dV *= g->dx[k];
  const int nq = g->nmat + 4;
  for (int q = 0; q < nq; ++q) {
    int field = -1;
    if (q < g->nmat) field = g->o_arho + q;
    else if (q < g->nmat + 3) field = (q - g->nmat) < g->dim ? g->o_mom + (q - g->nmat) : -1;
    else field = g->o_E;
    double s = 0.0, comp = 0.0;
    if (field >= 0)
      for (long c = 0; c < g->ncell; ++c) {
        const double y = g->U[(size_t)field * g->ncell + c] * dV - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
      }
    out[q] = s;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------------ */
/* Fragments (Sec. 4.2, 4.3): the paper demarcates fragments by a contour    */
/* nu = theta of the void volume fraction (theta = 0.25, 0.5, 0.75) and      */
/* reports each fragment's mass.  This model carries gas, not void, and a   */
/* crack is critically damaged solid (D >= D_crit, Sec. 3.1).  Reading: the  */
/* non-intact fraction of a cell is 1 - phi_s (phi_s the summed fraction of  */
/* the solid materials) where no solid is critically damaged, else 1; a     */
/* cell is in a fragment when that fraction is below theta, i.e.            */
/* phi_s > 1 - theta and no solid at D >= D_crit.  Fragments are the        */
/* components of such cells under face adjacency (periodic faces wrap);     */
/* a fragment's mass is the sum of dV (phi rho)_l over its cells and solid  */
/* materials.  Labels: the smallest cell index of the component.  Critical  */
/* means D >= D_crit (1 - 1e-4), as in the yield stress (R34).               */
/* ------------------------------------------------------------------------ */

static int in_fragment(const or_grid* g, double theta, long c) {
  const double* U = g->U;
  const long n = g->ncell;
  double phis = 0.0, last = 1.0;
  for (int l = 0; l < g->nmat; ++l) {
    const double phi = l + 1 < g->nmat ? U[(size_t)(g->o_phi + l) * n + c] : last;
    if (l + 1 < g->nmat) last -= phi;
    if (g->mat[l].eos != 1) continue;
    phis += phi;
    const int h = g->hslot[l];
    if (is_damaged(&g->mat[l]) && h >= 0) {
      const double arho = U[(size_t)(g->o_arho + l) * n + c];
      if (is_critical(&g->mat[l], U[(size_t)(g->o_hist + 2 * h + 1) * n + c] / arho)) return 0;
    }
  }
  return phis > 1.0 - theta;
}

long or_fragments(const or_grid* g, double theta, long* labels, long* frag_label,
                  long* frag_cells, double* frag_mass, long max_frag) {
  const long n = g->ncell;
  double dV = 1.0;
  for (int k = 0; k < g->dim; ++k) dV *= g->dx[k];
  long* lab = labels ? labels : malloc(sizeof(long) * (size_t)n);
  long* queue = malloc(sizeof(long) * (size_t)n);
  for (long c = 0; c < n; ++c) lab[c] = in_fragment(g, theta, c) ? n : -1; /* n: unvisited */
  long nfrag = 0;
  for (long c0 = 0; c0 < n; ++c0) {
    if (lab[c0] != n) continue;
    /* breadth-first search from the smallest unvisited member */
    long head = 0, tail = 0, cells = 0;
    double s = 0.0, comp = 0.0;
    lab[c0] = c0;
    queue[tail++] = c0;
    while (head < tail) {
      const long c = queue[head++];
      ++cells;
      for (int l = 0; l < g->nmat; ++l) {
        if (g->mat[l].eos != 1) continue;
        const double y = g->U[(size_t)(g->o_arho + l) * n + c] * dV - comp;
        const double t = s + y;
        comp = (t - s) - y;
        s = t;
      }
      long rest = c, stride = 1;
      for (int d = 0; d < g->dim; ++d) {
        const long nd = g->n[d];
        const long i = rest % nd;
        rest /= nd;
        for (int side = 0; side < 2; ++side) {
          long j = side == 0 ? i - 1 : i + 1;
          if (j < 0 || j >= nd) {
            if (g->bc[d][side] != OR_BC_PERIODIC) continue;
            j = j < 0 ? nd - 1 : 0;
          }
          const long nb = c + (j - i) * stride;
          if (lab[nb] == n) {
            lab[nb] = c0;
            queue[tail++] = nb;
          }
        }
        stride *= nd;
      }
    }
    if (nfrag < max_frag) {
      if (frag_label) frag_label[nfrag] = c0;
      if (frag_cells) frag_cells[nfrag] = cells;
      if (frag_mass) frag_mass[nfrag] = s;
    }
    ++nfrag;
  }
  free(queue);
  if (!labels) free(lab);
  return nfrag;
}
