/*
 * mmfrac: GB300-native explicit Eulerian step of the diffuse-interface
 * multi-material elastoplastic method with damage and a perturbed yield
 * stress (Wallis, Barton & Nikiforakis, "A multi-physics method for fracture
 * and fragmentation at high strain-rates", arXiv 2210.04037).
 *
 * C ABI.  All device memory is owned by the library.  Host buffers passed to
 * a call belong to the caller and are only read or written during that call.
 * Every call is ordered on the grid's CUDA stream; calls that return data to
 * the host synchronise that stream.  All functions return MM_OK or a negative
 * mm_status; mm_last_error() gives a thread-local message for the last
 * failure.
 *
 * Problem statement (Sec. 2.1): per material l, volume fraction phi_l,
 * partial density phi_l rho_l and history phi_l rho_l (eps_p, D); shared
 * momentum rho u, total energy rho E, unimodular elastic deformation tensor
 * Fbar and Lagrangian coordinates X.  The step is dimensionally split
 * (x, y, z sweeps), followed by the per-cell plastic return to the perturbed
 * yield stress phi0(X) sigma_Y (Sec. 2.1.3) and RK4 damage growth with loss
 * of strength (Sec. 3.1).
 *
 * Field order (primitive / conserved), dim d, N materials, H plastic ones:
 *   phi_0..phi_{N-2} / same;  rho_0..rho_{N-1} / phi_l rho_l;
 *   u_0..u_{d-1} / rho u;     p / rho E;
 *   Fbar comps / same  (d=1: xx yy zz; d=2: xx xy yx yy zz; d=3: 9, row-major);
 *   (eps_p, D) per plastic material / phi rho (eps_p, D);  X_0..X_{d-1} / same.
 * Arrays of fields are [field][cell], cells x fastest, then y, then z.
 */
#ifndef MMFRAC_H
#define MMFRAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MM_OK = 0,
  MM_EINVAL = -1,     /* an argument is out of range or inconsistent */
  MM_ENOMEM = -2,     /* device allocation failed */
  MM_ECUDA = -3,      /* a CUDA call failed (no device, launch error, ...) */
  MM_ENONFINITE = -4, /* a cell left the admissible set (rho_l <= 0, phi_l <= 0,
                         c_L^2 <= 0 or a non-finite value) */
  MM_ENOCONV = -5,    /* the plastic return did not converge */
  MM_EDT = -6,        /* non-positive or non-finite time step */
  MM_ETIMEOUT = -7,   /* a bounded wait ended before the work finished */
  MM_ESTATE = -8      /* call out of order (e.g. step before set_materials) */
} mm_status;

enum { MM_BC_TRANSMISSIVE = 0, MM_BC_PERIODIC = 1, MM_BC_REFLECTIVE = 2 };
enum { MM_FP64 = 0, MM_FP32_SPLIT = 1 };
enum { MM_EOS_IDEAL_GAS = 0, MM_EOS_ROMENSKII = 1, MM_EOS_VOID = 2 };
enum { MM_PL_NONE = 0, MM_PL_JOHNSON_COOK = 1 };
enum { MM_DMG_NONE = 0, MM_DMG_BONORA = 1, MM_DMG_SIMPLE = 2 };

/* Grid: dim in {1,2,3}; n[k] cells on [lo[k], hi[k]] for k < dim (n[k] >= 2);
 * bc[k][side] one of MM_BC_*; precision MM_FP64 (every step in FP64) or
 * MM_FP32_SPLIT (reconstruction and fluxes in FP32, total energy, energy
 * recovery, plastic return iteration and totals in FP64); n_materials 1..2,
 * or 3 when one of them is void (MM_EOS_VOID); at most one material with a
 * plasticity model, or two on 1D and 2D grids without void (two or three
 * materials, e.g. two solids in a gas). */
typedef struct {
  int dim;
  int64_t n[3];
  double lo[3], hi[3];
  int bc[3][2];
  int precision;
  int n_materials;
} mm_grid_desc;

/* Material (Sec. 2.1.1-2.1.2 and the parameter tables): Romenskii cold
 * energy K0, rho0, alpha; shear modulus G0 (rho/rho0)^(beta+1); Grueneisen
 * Gamma0; ideal gas gamma_gas.  MM_EOS_VOID: the void volume fraction nu of
 * Sec. 2.1 as a material of its own (no mass, energy or stress; its
 * primitive density field is 0; other parameters unused): at most one, not
 * the last material, with no plasticity or damage model, beside exactly one
 * plastic material; its fraction may be 0.  Where either face state is
 * critically damaged (D >= D_crit (1 - 1e-4), the threshold at which the
 * yield stress is zero too) and the two are in tension
 * along the sweep, x^T (sigma_L + sigma_R) x > 0, such a grid opens void
 * (Sec. 3.1): each side meets a traction-free surface and the gap between
 * them becomes void.  Grids with void run on single grids only (not in
 * batches or on the server).  Johnson-Cook yield (c1 + c2 eps^n_hard)
 * max(1, 1 + c3 ln(epsdot/edot0)).  Damage: Bonora (D_crit, eps_t = the
 * threshold strain, eps_c = the critical strain, alpha_D, poisson) or the
 * simple law Ddot = Ddot0 (1-D) epsdot (Sec. 4.3).  Shear model of a
 * Romenskii solid: MM_SHEAR_ROMENSKII (G above, constant Gamma0) or
 * MM_SHEAR_STEINBERG (Sec. 2.1.2 and the U-Nb closure of Sec. 4.3):
 * G = G0 + Gp p_c eta^(-1/3), p_c the cold pressure, eta = rho/rho0, and
 * Gamma = Gamma0 + Gamma1 eta^(-1/3) + Gamma2 eta^(-gamma_s) (beta unused);
 * both degraded by (1 - D) as above.  SI units. */
enum { MM_SHEAR_ROMENSKII = 0, MM_SHEAR_STEINBERG = 1 };
typedef struct {
  int eos;
  double rho0, K0, G0, alpha, beta, Gamma0, gamma_gas;
  int plasticity;
  double c1, c2, c3, n_hard, edot0;
  int damage;
  double D_crit, eps_t, eps_c, alpha_D, poisson, Ddot0;
  int shear_model;
  double Gp, Gamma1, Gamma2, gamma_s;
} mm_material;

/* Initial state: prim = [nfield][ncell] primitive fields in the order above
 * (host, copied).  phi0 = perturbation lattice of phi0_n points per axis
 * (x fastest) with origin phi0_lo and spacing phi0_h (host, copied), or NULL
 * for phi = 1 everywhere (Sec. 3.2.2: phi(x) = phi0(X(x)), multilinear,
 * 1 outside the lattice).  At least 2 points per axis and at most 2^31 - 1
 * points in all (else MM_EINVAL). */
typedef struct {
  const double* prim;
  const float* phi0;
  int64_t phi0_n[3];
  double phi0_lo[3], phi0_h[3];
} mm_init;

typedef struct {
  double t, dt_last, smax;
  int64_t steps_done, bad_cell;
} mm_step_info;

typedef struct mm_grid mm_grid;

/* Create a grid and allocate its state on the current CUDA device.
 * cuda_stream: a cudaStream_t to order work on, or NULL for a stream the
 * library creates.  Errors: MM_EINVAL, MM_ENOMEM, MM_ECUDA (no device). */
mm_status mm_create_grid(const mm_grid_desc* desc, void* cuda_stream, mm_grid** out);

/* Set the materials and the initial state (Sec. 2.1; conversion of the
 * primitive state to the conserved one by the closures of Sec. 2.1.1).
 * n must equal desc.n_materials.  Errors: MM_EINVAL, MM_ENONFINITE (an
 * initial cell is inadmissible; bad_cell in mm_last_error). */
mm_status mm_set_materials(mm_grid* g, const mm_material* mats, int n, const mm_init* init);

/* Advance n_steps explicit steps with dt = cfl * min_k dx_k / max_cells
 * (max_k |u_k| + c_L), each step = sweeps x, y, z then the sources.  After
 * the first step on a state, steps are replayed from a captured CUDA graph
 * (the same kernels; launch by launch while kernel timing is on, or on a
 * stream that cannot be captured).  Calls on one grid must not overlap.
 * info (may be NULL) receives time, last dt, last signal speed, steps done
 * and the first bad cell.  On MM_ENONFINITE / MM_ENOCONV the state after
 * the failing step is undefined.  Errors: MM_ESTATE (no materials yet),
 * MM_EINVAL, MM_ENONFINITE, MM_ENOCONV, MM_EDT, MM_ECUDA. */
mm_status mm_step(mm_grid* g, int n_steps, double cfl, mm_step_info* info);

/* The same n_steps steps as mm_step, enqueued on the grid's stream without
 * waiting for them (no host synchronisation): for callers that overlap the
 * stepping with other work or time it with events on the stream.  Argument
 * and launch errors are returned at once (MM_ESTATE, MM_EINVAL, MM_ECUDA);
 * a failure inside a step (MM_ENONFINITE, MM_ENOCONV, MM_EDT) is latched on
 * the device (the first one, with its cell and step) and returned by the
 * next mm_synchronize, mm_step or mm_read_fields; the state after it is
 * undefined. */
mm_status mm_step_async(mm_grid* g, int n_steps, double cfl);

/* Wait for the work enqueued on the grid's stream and report the first
 * failure latched by the steps since the last report (errors as mm_step).
 * info (may be NULL) is filled as by mm_step. */
mm_status mm_synchronize(mm_grid* g, mm_step_info* info);

/* Transport of the Lagrangian coordinates X (Sec. 3.2.1).  MM_X_SWEEP
 * (default): X is carried by the split MUSCL-Hancock sweeps like the volume
 * fractions.  MM_X_WENO3_RK3: the scheme the paper states for X, third-order
 * WENO face values from the upwind cell and the three-stage TVD Runge-Kutta
 * scheme with the velocities of the step's start, computed before the sweeps
 * and replacing their X (dX/dt = -div(X u) + X div(u), face velocity the
 * mean of the cell velocities; ghosts follow the boundary rules).  The first
 * call with MM_X_WENO3_RK3 allocates 3 x dim x ncell values of scratch.
 * Grids in a batch must use MM_X_SWEEP; MM_X_WENO3_RK3 takes grids of fewer
 * than 2^31 cells.  Errors: MM_EINVAL, MM_ENOMEM. */
enum { MM_X_SWEEP = 0, MM_X_WENO3_RK3 = 1 };
mm_status mm_set_x_transport(mm_grid* g, int scheme);

/* Lagrangian seeding into void (Sec. 3.2.1 seeding routine), on grids with a
 * void material: before each step, every cell with void fraction nu > 1/2
 * and a normal (|grad nu| h > 1e-6, central differences) takes
 * X = X(p) - (p - c), c its
 * centre, p = c + 1.5 h n the probe point, n = -grad nu / |grad nu| (into
 * the material), h the largest cell size, X(p) multilinear in the
 * cell-centred X of the step's start; ghost cells follow the boundary rules.
 * on = 1 (default) or 0; no effect on grids without void (whose X the step
 * carries everywhere).  Grids with void hold dim x ncell values of scratch
 * for it from mm_set_materials on.  Errors: MM_EINVAL. */
mm_status mm_set_lagrangian_seeding(mm_grid* g, int on);

/* TMA tile loads in the y and z sweeps (the split update of Sec. 3.1 along
 * the second and third axes; no change to what a step computes).  3D
 * FP32-split grids of two materials without void whose n[0] is a multiple
 * of 4 get tensor maps of their state from mm_set_materials on; their y and
 * z sweeps, where they run as columns of tiles per CTA (large grids), then
 * stage each tile's new cells in shared memory with cp.async.bulk.tensor
 * copies issued one tile ahead instead of per-thread loads.  The staged
 * values are the stored ones, so both loads give the same bits.
 * on = 1 (default) uses the maps, 0 the per-thread loads, -1 leaves the
 * switch as it is.  active (may be null) receives 1 where the grid has maps
 * and the switch is on, else 0.  A staged tile whose copy has not arrived
 * within one second ends its CTA with MM_ETIMEOUT (reported by the next
 * synchronising call).  Errors: MM_EINVAL. */
mm_status mm_set_tma_loads(mm_grid* g, int on, int* active);

/* Fragments of the present state (Sec. 4.2, 4.3 demarcate fragments by the
 * contour nu = theta of the void volume fraction, theta = 0.25, 0.5, 0.75,
 * and report fragment masses).  A crack is critically damaged solid
 * (Sec. 3.1) and the space around the pieces holds gas, or void on grids
 * with a void material, so a cell belongs to a fragment when the summed
 * volume fraction of its solid (Romenskii) materials exceeds 1 - theta
 * (on a grid of solid and void alone: nu < theta) and no damaged solid in
 * it has D >= D_crit (1 - 1e-4), the threshold of the yield stress (D comes
 * back as (phi rho D)/(phi rho), below a cap at D_crit by rounding or a
 * trace mixed in).  Fragments are the components of such cells under
 * face adjacency; periodic faces wrap.  A fragment's label is its smallest
 * linear cell index (x fastest), its mass sum dV (phi rho) over its cells
 * and solids (FP64; summed in no fixed order).
 *   theta      cut-off in (0, 1].
 *   labels     host int64[labels_len] or NULL; labels_len must equal the
 *              cell count.  Receives each cell's label or -1.
 *   frags      host array of max_frags records or NULL (max_frags 0).
 *              Receives the first min(max_frags, *n_frags) fragments in
 *              label order.
 *   n_frags    receives the number of fragments (may exceed max_frags).
 * Runs on the grid's stream and synchronises.  The first call allocates
 * 16 bytes per cell of scratch, kept until mm_destroy.  Takes grids of
 * fewer than 2^31 cells.  Errors: MM_EINVAL (arguments), MM_ESTATE (before
 * mm_set_materials), MM_ENOMEM, MM_ETIMEOUT (a union that did not settle,
 * which the labelling's invariants exclude), MM_ECUDA. */
typedef struct {
  int64_t label; /* smallest cell index of the fragment */
  int64_t cells; /* number of cells */
  double mass;   /* solid mass, kg (per metre in 2D, per m^2 in 1D) */
} mm_fragment;
mm_status mm_fragments(mm_grid* g, double theta, int64_t* labels, size_t labels_len,
                       mm_fragment* frags, size_t max_frags, int64_t* n_frags);

/* Copy fields to host_dst ([popcount(field_mask)][ncell] doubles, fields
 * in order; bit f of field_mask selects field f, ~0 for all).
 * primitive = 1 returns the primitive fields, 0 the conserved ones.
 * dst_len is the capacity of host_dst in doubles.  Errors: MM_EINVAL. */
mm_status mm_read_fields(mm_grid* g, uint64_t field_mask, int primitive,
                         double* host_dst, size_t dst_len);

/* ---- Batched ensembles.  Sec. 4.3 notes that one run of the expanding
 * ring is a single sample and that fragment statistics need the model run
 * many times: a batch steps many grids (seeded realisations of the
 * perturbation field, of uneven size) together.  Each member keeps its own
 * state, dt and time; one launch per kernel kind covers every member (CTAs
 * take the members' tiles or cell chunks from a work counter), and from the
 * second step on a step is one CUDA graph launch.  A member's results are
 * those of mm_step on that member alone. */
typedef struct mm_batch mm_batch;

/* Batch the n grids (distinct, materials set, same dimension, precision and
 * material layout, two materials).  The batch references the grids, which
 * must outlive it; between mm_batch_step and mm_batch_synchronize the grids
 * must not be used on their own.  cuda_stream: stream to order the batch's
 * work on, or NULL for one the library creates.  Errors: MM_EINVAL,
 * MM_ESTATE (a member without materials), MM_ENOMEM, MM_ECUDA. */
mm_status mm_batch_create(mm_grid* const* grids, int n, void* cuda_stream, mm_batch** out);

/* use_graph: 1 (default) replays captured steps, 0 launches each kernel;
 * tile_variant (may be NULL): tile shape per sweep axis, 0 or 1 (FP32-split
 * has two shapes per axis, FP64 one).  Errors: MM_EINVAL. */
mm_status mm_batch_set_options(mm_batch* b, int use_graph, const int tile_variant[3]);

/* Enqueue n_steps steps of every member (each with its own dt = cfl dx_min
 * / s_max) without waiting.  Failures inside a step are latched per member
 * and returned by mm_batch_synchronize.  Errors: MM_EINVAL, MM_ECUDA. */
mm_status mm_batch_step(mm_batch* b, int n_steps, double cfl);

/* Time each launch configuration of each sweep axis on the batch's current
 * states (reps timed launches after one warm-up; a sweep into the free
 * buffer leaves the state unchanged), keep the fastest, and return the
 * chosen tile shapes in chosen (may be NULL).  The configurations: the
 * compiled tile shapes (FP32-split: 2 per axis; FP64: 1) times the
 * persistent CTAs per SM (as many as fit, 1, 2).  Blocks.  Errors:
 * MM_EINVAL, MM_ECUDA. */
mm_status mm_batch_autotune(mm_batch* b, int reps, int chosen[3]);

/* The same search with a persistent choice.  The batch's size class is
 * log2 of its median member cell count; the cache key is the device (name
 * and SM count), precision, dimension, material layout and size class.
 * With cache_path non-NULL and force 0, a choice cached under the key is
 * taken without timing; otherwise the search runs and its choice is
 * appended to the file (plain text, one line per key, the last line for a
 * key wins; not locked against other processes).  out (may be NULL)
 * receives the choice. */
typedef struct {
  int variant[3];     /* tile shape per sweep axis */
  int cta_per_sm[3];  /* persistent CTAs per SM per sweep axis (0: as many as fit) */
  int from_cache;     /* 1: read from the cache, 0: timed */
  int size_class;     /* log2 of the median member cell count */
} mm_tune;
mm_status mm_batch_autotune_ex(mm_batch* b, int reps, const char* cache_path, int force,
                               mm_tune* out);

/* Members stepped in groups, one group after another within a step: every
 * launch of a step runs on one group's members, whose state (both buffers)
 * then stays in the L2 cache between the launches.  Groups are consecutive
 * members, greedily up to group_bytes of state each (a larger member is a
 * group of its own); group_bytes 0 (the default): one group of all members;
 * negative: 60 % of the device's L2.  Results do not depend on the grouping.
 * (Measured on GB300 with the 64-ring ensemble: one group 7.5 ms per step,
 * 4 groups 8.8, 19 groups 17.5: the smaller launches fill the GPU less.)
 * Errors: MM_EINVAL. */
mm_status mm_batch_set_grouping(mm_batch* b, int64_t group_bytes);
/* Number of member groups of the batch (0 for NULL). */
int mm_batch_num_groups(const mm_batch* b);

/* Wait for the batch's work and report the first failure latched by a
 * member (its index in the message).  Errors as mm_step. */
mm_status mm_batch_synchronize(mm_batch* b);

/* Per-kernel timing of the batch's launches, as mm_profile_enable /
 * mm_profile_read for a grid (while it is on, steps are launched kernel by
 * kernel, not replayed from a graph; times are collected by
 * mm_batch_synchronize).  Errors: MM_EINVAL. */
mm_status mm_batch_profile_enable(mm_batch* b, int enable);
mm_status mm_batch_profile_read(mm_batch* b, double* ms, int64_t* counts, int n, int reset);

/* Wait for the batch's work and free the batch (not its grids). */
mm_status mm_batch_destroy(mm_batch* b);

/* ---- Served runs (continuous batching).  A server owns a scheduler thread
 * that admits submitted runs first come, first served while the device
 * memory they need fits its budget, steps all admitted runs together (one
 * batch per group of runs with the same dimension, precision, material
 * layout and CFL number, the groups on separate streams), and retires each
 * run when it has done its steps: its primitive fields go to host memory and
 * its device memory is freed, which admits the next runs.  Runs submitted
 * while others are on the GPU join them at the next tick (every
 * steps_per_tick steps).  A run's result is the same as that of the same
 * grid stepped alone with mm_step. */
typedef struct mm_server mm_server;

typedef struct {
  int64_t id;
  int32_t status;      /* mm_status of the run */
  int32_t nfield;      /* the result holds nfield x ncell doubles */
  int64_t ncell;
  int64_t steps_done;
  double t;            /* simulated time reached */
  double submit_s, admit_s, done_s;  /* seconds since the server was created */
} mm_run_info;

typedef struct {
  uint64_t budget_bytes, used_bytes;
  int64_t pending, admitted, retired;
} mm_server_info;

/* Create a server on the current device.  memory_budget: device bytes its
 * runs may hold at once (0: 90 % of the free memory now); steps_per_tick:
 * steps between admissions (<= 0: 8).  Errors: MM_EINVAL, MM_ECUDA. */
mm_status mm_server_create(size_t memory_budget, int steps_per_tick, mm_server** out);

/* Queue a run of n_steps steps at the given CFL number on the grid desc
 * with the materials and initial state given (as for mm_create_grid and
 * mm_set_materials; all host data are copied before the call returns).
 * Two materials.  *id receives the run's id.  Errors: MM_EINVAL (arguments,
 * or a run larger than the memory budget), MM_ESTATE (server shutting
 * down).  Errors of the run itself are returned by mm_server_wait. */
mm_status mm_server_submit(mm_server* s, const mm_grid_desc* desc, const mm_material* mats,
                           int n_mat, const mm_init* init, int n_steps, double cfl,
                           int64_t* id);

/* Wait up to timeout_ms (< 0: without limit) for run id.  On MM_ETIMEOUT
 * nothing changes.  When the run has finished, info (may be NULL) is filled;
 * a failed run returns its error and is released; a successful run copies
 * its primitive fields ([nfield][ncell], as mm_read_fields) to host_dst and
 * is released, or, with host_dst NULL, only fills info and stays available.
 * Errors: MM_EINVAL (unknown id, destination too small), MM_ETIMEOUT, the
 * run's own error. */
mm_status mm_server_wait(mm_server* s, int64_t id, int timeout_ms, mm_run_info* info,
                         double* host_dst, size_t dst_len);

/* Memory budget and use, and run counts.  Errors: MM_EINVAL. */
mm_status mm_server_stats(mm_server* s, mm_server_info* info);

/* Stop admitting, finish the admitted runs, cancel the queued ones (their
 * wait returns MM_ESTATE), join the scheduler and free the server. */
mm_status mm_server_destroy(mm_server* s);

/* Conserved totals sum_cells dV (phi rho)_l (N values), sum dV rho u
 * (3 values, 0 for k >= dim), sum dV rho E: N + 4 doubles, accumulated in
 * FP64.  out_len >= N + 4.  Errors: MM_EINVAL. */
mm_status mm_conserved_totals(mm_grid* g, double* out, size_t out_len);

/* Conserved totals of a state the caller holds in device memory, computed
 * without allocating anything (the paper has no counterpart; this is an
 * interface for callers that cannot allocate).  Some callers cannot call
 * cudaMalloc: a serving loop that owns a fixed pool of device memory and
 * must not let a library allocate (cudaMalloc can synchronise the device and
 * fragments the pool), or a runtime whose allocator is off limits at the
 * point of the call.  They pass the state and the output; the block partial
 * sums go to one file-scope device array of 1024 x 7 doubles (56 KiB: up
 * to 3 materials) that every GPU which loads the library keeps until the
 * process exits.
 *   d_cons   device pointer, FP64 conserved fields [nfield][ncell] in the
 *            field order above (mm_read_fields(..., primitive = 0) layout);
 *   dim, ncell, n_materials (1..3): the layout of d_cons; n_plastic
 *            (materials with a plasticity model) is only checked
 *            (0..n_materials): the totals read fields that come before the
 *            plastic ones, so their offsets do not depend on it;
 *   dx       host array, cell size per axis (dV = product over dim);
 *   d_out    device pointer to N + 4 doubles (as mm_conserved_totals);
 *   cuda_stream  stream to order the two kernels on (NULL: default stream).
 * The call is asynchronous on the stream.  Each call looks up the scratch
 * array's device address in the current context (cudaGetSymbolAddress).
 * The first call in a context loads the library's device code there if it
 * is not loaded yet (lazy module loading, the CUDA default), which
 * materialises the array: a one-time device allocation by the driver.  Make
 * that first call during setup, before any stream capture; later calls
 * allocate nothing.
 * Every call on a device shares the one array and overwrites every entry it
 * reads, so nothing carries over, but calls that overlap on the GPU (other
 * streams, other threads) race on it: order them.  More materials than the
 * scratch holds: MM_EINVAL.  Other errors: MM_EINVAL, MM_ECUDA. */
mm_status mm_conserved_totals_noalloc(const double* d_cons, int dim, int64_t ncell,
                                      int n_materials, int n_plastic, const double dx[3],
                                      double* d_out, void* cuda_stream);

/* Number of fields and cells of the grid (for sizing buffers). */
int mm_num_fields(const mm_grid* g);
int64_t mm_num_cells(const mm_grid* g);

/* Release every device resource of the grid. */
mm_status mm_destroy(mm_grid* g);

/* Message of the last failure on the calling thread ("" if none). */
const char* mm_last_error(void);

/* Kernels launched by the last mm_step or mm_step_async call (for launch
 * accounting). */
int64_t mm_kernel_launches(const mm_grid* g);

/* Kernel timing (tracing aid, no counterpart in the paper).  With enable = 1
 * every later mm_step brackets each of its launches with CUDA events on the
 * grid's stream and accumulates the elapsed device time per kernel kind:
 * MM_K_CFL (on a single grid it also forms dt), MM_K_DT (batches only: the
 * per-member dt launch), MM_K_SWEEP_X, MM_K_SWEEP_Y, MM_K_SWEEP_Z, MM_K_SOURCES,
 * MM_K_XTRANSPORT (the X update of MM_X_WENO3_RK3, its four launches and the
 * copy together); mm_fragments likewise: MM_K_FRAG_MARK (membership and
 * masses), MM_K_FRAG_UNION (the union and root passes), MM_K_FRAG_COUNT (the
 * ordered root count), MM_K_FRAG_COLLECT (numbering and per-fragment sums).
 * mm_profile_read copies min(n, MM_K_COUNT) accumulated milliseconds and
 * launch counts (either pointer may be NULL) and, if reset = 1, zeroes them.
 * Errors: MM_EINVAL, MM_ECUDA. */
enum { MM_K_CFL = 0, MM_K_DT = 1, MM_K_SWEEP_X = 2, MM_K_SWEEP_Y = 3, MM_K_SWEEP_Z = 4,
       MM_K_SOURCES = 5, MM_K_XTRANSPORT = 6, MM_K_FRAG_MARK = 7, MM_K_FRAG_UNION = 8,
       MM_K_FRAG_COUNT = 9, MM_K_FRAG_COLLECT = 10, MM_K_COUNT = 11 };
mm_status mm_profile_enable(mm_grid* g, int enable);
mm_status mm_profile_read(mm_grid* g, double* ms, int64_t* counts, int n, int reset);

#ifdef __cplusplus
}
#endif
#endif
