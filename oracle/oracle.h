/*
 * Plain FP64 CPU oracle of the explicit Eulerian step of the diffuse-interface
 * multi-material elastoplastic method of Wallis, Barton & Nikiforakis,
 * "A multi-physics method for fracture and fragmentation at high strain-rates"
 * (arXiv 2210.04037).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference leg of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path under
 * paper_2210_04037_gb300/; the two agree only on the documented field order.
 *
 * What it computes (paper sections in brackets; where the paper defers to
 * earlier work the reading is named R<k> and listed in the design notes):
 *   - state and transport equations (Sec. 2.1, Eqs. for phi, phi*rho,
 *     phi*rho*alpha, rho*u, rho*E, the unimodular deformation tensor, X),
 *   - closures: Mie-Grueneisen split with the Romenskii cold energy, the
 *     Romenskii shear modulus with a constant Grueneisen coefficient or the
 *     Steinberg shear modulus with a density-dependent one, Hencky strain,
 *     shear energy G*J^2/rho, stress -p I + 2 G dev(H) (Sec. 2.1.1, 2.1.2),
 *   - ideal gas as the G=0 special case,
 *   - damage degradation of G and of the cold energy, the Bonora damage rate
 *     with the tension gate and the triaxiality-dependent threshold, the
 *     simple damage model of the expanding-ring test, RK4 integration
 *     (Sec. 2.1.1, Sec. 3.1, Sec. 4.3),
 *   - the yield stress perturbed by phi0(X) looked up on a lattice
 *     (Sec. 2.1.3, Sec. 3.2.2).
 * Parity unpinned parts: none of the functions below is without a pin; the
 * choice of MUSCL-Hancock + HLLC itself is a reading (the paper defers the
 * hyperbolic solver), pinned only through the closed-form tests.
 */
#ifndef MMFRAC_ORACLE_H
#define MMFRAC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAXMAT 4

/* Boundary kinds per face of the box. */
#define OR_BC_TRANSMISSIVE 0
#define OR_BC_PERIODIC 1
#define OR_BC_REFLECTIVE 2

/* Error codes. */
#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENONFINITE (-4)
#define OR_ENOCONV (-5)

typedef struct {
  int eos;                /* 0 ideal gas, 1 Romenskii solid, 2 void (massless,
                             stress-free; at most one, never the last material) */
  double rho0, K0, G0, alpha, beta, Gamma0, gamma_gas;
  int plasticity;         /* 0 none, 1 Johnson-Cook (no thermal term) */
  double c1, c2, c3, n_hard, edot0;
  int damage;             /* 0 none, 1 Bonora, 2 simple (Ddot0 (1-D) epsdot) */
  double D_crit, eps_t, eps_c, alpha_D, poisson, Ddot0;
  int shear_model;        /* Romenskii solids: 0 Romenskii G = G0 eta^(beta+1) with
                             constant Gamma0; 1 Steinberg G = G0 + Gp p_c eta^(-1/3)
                             with Gamma = Gamma0 + Gamma1 eta^(-1/3) + Gamma2
                             eta^(-gamma_s) (Sec. 2.1.2, Sec. 4.3) */
  double Gp, Gamma1, Gamma2, gamma_s;
} or_material;

typedef struct or_grid or_grid;

/* Create a grid and set its initial state from primitive fields.
 * prim: [nfield][ncell] doubles, x fastest, in the primitive field order
 * (phi_0..phi_{N-2}, rho_0..rho_{N-1}, u (dim), p, Fbar (active comps),
 *  (eps_p, D) per plastic material, X (dim)).
 * bc: [dim][2] flattened as bc[2*d + side].
 * phi0: perturbation lattice (float, x fastest) or NULL.              */
or_grid* or_create(int dim, const long n[3], const double lo[3],
                   const double hi[3], const int bc[6], int nmat,
                   const or_material* mats, const double* prim,
                   const float* phi0, const long pn[3], const double plo[3],
                   const double ph[3], int* status);
void or_destroy(or_grid* g);
int or_nfield(const or_grid* g);
long or_ncell(const or_grid* g);
/* Advance nsteps.  dt_fixed > 0 imposes that dt; otherwise the CFL rule. */
int or_step(or_grid* g, int nsteps, double cfl, double dt_fixed,
            double* info /* [t, dt_last, smax, steps, bad_cell, nbound] */);
/* nbound: faces, since creation, whose half step was replaced by the cell
 * average because a phase density left the half step's bound (a factor e). */
/* Time step the CFL rule gives for the present state. */
int or_cfl_dt(or_grid* g, double cfl, double* dt, double* smax);
int or_read(const or_grid* g, int primitive, double* out);
int or_write_conserved(or_grid* g, const double* U);
int or_totals(const or_grid* g, double* out /* N + 4 */);
void or_set_threads(int n);
/* Transport of the Lagrangian coordinates X: 0 (default) carried by the
 * sweeps like the volume fractions; 1 third-order WENO with three-stage RK
 * from the state at the step's start (Sec. 3.2.1).  OR_EINVAL otherwise. */
int or_set_x_scheme(or_grid* g, int scheme);

/* Lagrangian seeding into void (Sec. 3.2.1 seeding routine; reading in the
 * source): or_seed_x applies it once to the present state (grids with a
 * void material; no-op otherwise); or_set_seed_x(g, 0/1) turns off / on
 * (default) its application before every step. */
int or_seed_x(or_grid* g);
int or_set_seed_x(or_grid* g, int on);

/* Fragments at void cut-off theta (Sec. 4.2, 4.3; reading in the source):
 * labels[ncell] (may be NULL) gets each cell's fragment label, the smallest
 * cell index of its fragment, or -1; the first max_frag fragments in label
 * order get label, cell count and mass.  Returns the number of fragments. */
long or_fragments(const or_grid* g, double theta, long* labels, long* frag_label,
                  long* frag_cells, double* frag_mass, long max_frag);

/* ---- single-point routines exported for the pins ---- */
void or_thermo(const or_material* m, double rho, double psi, double J2,
               double* out /* e_ref, p_ref, dpref_drho, G, Gamma,
                              rho Gamma'(rho) / Gamma */);
int or_hencky(const double F[9], double devH[9], double lam[3], double Q[9]);
double or_lookup(int dim, const float* phi0, const long pn[3],
                 const double plo[3], const double ph[3], const double X[3]);
double or_eps_thresh(double eps_t, double eps_c, double n, double Rt);
double or_Rt(double poisson, double rho0, double rho, double p, double seq);
double or_damage_rk4(const or_material* m, double D, double eps0,
                     double deps, double dt, double p, double seq,
                     double rho);
int or_plastic_return_cell(const or_material* mats, int nmat,
                           const double* phi, const double* rho,
                           const double* eps, const double* D, double phihat,
                           double dt, double F[9], double* dEps);

#ifdef __cplusplus
}
#endif
#endif
