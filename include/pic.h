/*
 * pic.h -- C ABI of the GB300 implicit electrostatic PIC/MC timestep in
 * axisymmetric r-z geometry (Wang, Jiang & Wang, "Implicit and
 * electrostatic Particle-in-cell/Monte Carlo model in two-dimensional and
 * axisymmetric geometry I: analysis of numerical techniques",
 * arXiv:1001.2969).
 *
 * One handle holds one reactor: an r-z mesh, two species (electrons and
 * one ion species), their particles resident in GPU memory, the fields and
 * the multigrid workspace.  Every entry point returns a pic_status and
 * never aborts the process; pic_last_error() gives a one-line reason.
 * Grids are FP64, row-major [i][j] with i the z node (0..nz-1) and j the
 * r node (0..nr-1).  Units are SI (volts, metres, seconds, kilograms,
 * coulombs); energies in cross-section tables are in eV.
 *
 * Threading: a handle may be used from one host thread at a time.  All
 * device work of a handle is issued on the stream given in the config
 * (the legacy default stream when NULL).
 */
#ifndef PIC_H
#define PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pic_status {
    PIC_OK = 0,
    PIC_ERR_ARG = 1,           /* invalid argument or configuration          */
    PIC_ERR_CAPACITY = 2,      /* particle or births capacity exceeded        */
    PIC_ERR_CUDA = 3,          /* a CUDA runtime call failed                  */
    PIC_ERR_NOT_CONVERGED = 4, /* multigrid hit mg_max_cycles (non-fatal)    */
    PIC_ERR_NUMERIC = 5,       /* NaN/Inf in the particle state               */
    PIC_ERR_TIMEOUT = 6,       /* a bounded device wait gave up              */
    PIC_ERR_STATE = 7          /* call not valid in the handle's state        */
} pic_status;

enum { PIC_FP64 = 0, PIC_MIXED = 1 };
enum { PIC_WEIGHT_ZR2 = 0, PIC_WEIGHT_ZR = 1 };
enum { PIC_CHI_MAX = 0, PIC_CHI_MEAN = 1 };
/* starting value of each timestep's solve (pic_config.mg_guess) */
enum { PIC_GUESS_PREVIOUS = 0, PIC_GUESS_LINEAR = 1 };

/* pusher (Sec. 2.3): the local X-Y frame with a_theta dropped (the paper's
 * choice for its 2D runs), or the global X-Y-Z form, which carries a_theta */
enum { PIC_PUSH_LOCAL = 0, PIC_PUSH_XYZ = 1 };
enum { PIC_SCATTER_VS = 0, PIC_SCATTER_ISOTROPIC = 1 };
enum { PIC_XS_ELASTIC = 0, PIC_XS_EXCITE = 1, PIC_XS_IONIZE = 2, PIC_XS_CX = 3 };

#define PIC_MAX_CH 4

/* Counter slots returned by pic_moments (int64). */
#define PIC_C_COLL 0    /* [s*4+ch] real collisions of species s, channel ch */
#define PIC_C_CAND 8    /* [s] null-collision candidates                      */
#define PIC_C_NUOVER 10 /* [s] particles whose nu exceeded nu_max             */
#define PIC_C_BIRTHS 12 /* [s] particles born (ionisation and splitting)      */
#define PIC_C_SPLITS 14 /* [s] parents split                                  */
#define PIC_C_ABS 16    /* [s*3+wall] absorbed at z=0, z=L, r=R               */
#define PIC_C_MGCYC 22  /* multigrid V-cycles, summed over steps              */
#define PIC_C_STEPS 23  /* steps taken                                        */
#define PIC_C_PSTEPS 24 /* particles moved by the passes, summed over steps   */
#define PIC_NCOUNT 25

/* Mesh: uniform node-centred r-z mesh, z in [0, L], r in [0, R] (Sec. 2.4,
 * Sec. 3.2).  nz must be 2^k + 1 (z-semi-coarsening, Sec. 2.5); 3 <= nr <= 1025
 * (one r-line unknown per thread of a line solve). */
typedef struct pic_mesh {
    double R, L;
    int32_t nz, nr;
} pic_mesh;

/* Species [0] electrons, [1] ions: charge, mass, initial density n0
 * (m^-3), temperature (eV), initial macro-particle count and capacity. */
typedef struct pic_species {
    double q, m, n0, T_eV;
    int64_t n_init, capacity;
} pic_species;

/* Cross sections (Sec. 2.6): sigma_m2[ch * n_e + k] at E_k = k E_max/(n_e-1),
 * linearly interpolated, 1/E above E_max.  Electron channels may be
 * ELASTIC, EXCITE, IONIZE; the ion channel is CX (charge exchange).
 * B_eV is the ionisation energy-sharing parameter. */
typedef struct pic_xsec {
    int32_t n_e;
    double E_max_eV;
    int32_t n_ch;
    const double *sigma_m2;
    const double *threshold_eV;
    const int32_t *kind;
    double B_eV;
} pic_xsec;

/* rf source on the z = 0 electrode: V(t) = sum_k amp_k sin(2 pi f_k t + ph_k)
 * (Sec. 3 benchmark: 200 sin(w t) at 13.56 MHz). */
typedef struct pic_rf {
    int32_t n;
    const double *amp_V, *freq_Hz, *phase_rad;
} pic_rf;

/* Background gas (Sec. 2.6): pressure, temperature, atom mass. */
typedef struct pic_gas {
    double p_Pa, T_K, m_gas;
} pic_gas;

/* Device memory hooks.  alloc returns 256-byte aligned device memory or
 * NULL; free releases it.  When alloc is NULL the library uses cudaMalloc. */
typedef void *(*pic_alloc_fn)(size_t bytes, void *ctx, void *stream);
typedef void (*pic_free_fn)(void *ptr, size_t bytes, void *ctx, void *stream);

typedef struct pic_config {
    pic_mesh mesh;
    pic_species sp[2];
    pic_xsec xs[2];
    pic_rf rf;
    pic_gas gas;
    double dt;            /* time step (s) */
    uint64_t seed;        /* Philox key    */
    int32_t precision;    /* PIC_FP64 or PIC_MIXED                            */
    int32_t weighting;    /* PIC_WEIGHT_ZR2 (Eq. (9)) or PIC_WEIGHT_ZR (Eq. (8)) */
    int32_t chi_face;     /* PIC_CHI_MAX or PIC_CHI_MEAN (Sec. 2.5)            */
    int32_t scatter;      /* PIC_SCATTER_VS or PIC_SCATTER_ISOTROPIC           */
    int32_t split_every;  /* weight-split period in steps, 0 = never (Sec. 2.2) */
    int32_t mg_max_cycles;
    double mg_tol;        /* relative max-norm residual; <= 0: run mg_max_cycles */
    const double *phi_zL; /* nullable: nr potentials on z = L (else grounded)  */
    int64_t births_capacity; /* per species, 0 = capacity/2                  */
    int32_t eedf_bins;
    double eedf_emax_eV;
    int32_t load;         /* 1: load the species at init (uniform n0, weights ~ cell volume) */
    pic_alloc_fn alloc;
    pic_free_fn free;
    void *alloc_ctx;
    void *stream;         /* cudaStream_t */
    /* external circuit (Sec. 2.5, end): a blocking capacitor circuit_C (F)
     * between the rf source and the z = 0 electrode, solved by Vahedi's
     * superposition each step; 0 drives the electrode directly */
    double circuit_C;
    int32_t pusher;       /* PIC_PUSH_LOCAL or PIC_PUSH_XYZ (Sec. 2.3)          */
    /* ion subcycling (Sec. 2.7, Vahedi's method; the implicit form is this
     * library's reading): with K = ion_subcycle > 1 the ions move only in
     * the passes n with n mod K = K - 1, by one D1 cycle with dt_i = K dt
     * (final push, Monte Carlo with P_null = 1 - exp(-nu_max dt_i), first
     * push), and are held still, state and deposit, in the others; their
     * susceptibility enters the solve before a moving pass with dt_i^2 and
     * no other.  Ions born in any pass take their first push with dt_i.
     * 0 or 1: no subcycling.  split_every must be a multiple of K.  Not
     * with pic_batch_init or pic_window (PIC_ERR_ARG). */
    int32_t ion_subcycle;
    /* starting value w_0 of each timestep's V-cycles (Algorithm 1 leaves it
     * open): PIC_GUESS_PREVIOUS the last step's potential, PIC_GUESS_LINEAR
     * 2 phi^n - phi^(n-1) on the interior nodes, extrapolated from the last
     * two steps.  phi^(n-1) starts equal to phi (zero) at init, so the first
     * step starts from phi^n; checkpoints carry it.  With the external circuit
     * its two solves start from their previous solutions either way. */
    int32_t mg_guess;
} pic_config;

typedef struct pic_handle pic_handle;
typedef struct pic_batch pic_batch;

/* Host particle arrays, absolute coordinates, FP64.  cell (nullable) is
 * filled by pic_get_particles with the stored cell index j (nz-1) + i and
 * ignored by pic_set_particles.  at (nullable): a_theta, carried by the
 * X-Y-Z pusher only (zero for the local pusher; NULL on set: zeros). */
typedef struct pic_particles_view {
    int64_t n;
    double *r, *z, *vr, *vt, *vz, *ar, *az, *w;
    uint64_t *id;
    int32_t *cell;
    double *at;
} pic_particles_view;

typedef struct pic_solve_info {
    int32_t cycles;
    double rel_residual;
} pic_solve_info;

typedef struct pic_moments_out {
    double *ne, *ni, *phi, *Er, *Ez; /* [nz][nr] averages over steps, nullable */
    double *eedf;                    /* [eedf_bins] weighted electron energies per step */
    int64_t *counters;               /* [PIC_NCOUNT], nullable                  */
    double *charge;                  /* [3] absorbed charge at z=0, z=L, r=R     */
    int64_t nsamples;                /* out: steps averaged                     */
    int32_t on_device;               /* grids/eedf are device pointers          */
} pic_moments_out;

/*
 * pic_init -- validate cfg, allocate the handle's device state and, when
 * cfg->load is 1, load both species: uniform density n0 with weights
 * proportional to the cell volume (Sec. 2.2, Eq. (3)), particles spread
 * evenly over cells numbered c = j (nz-1) + i (remainder to the lowest
 * numbers), uniform in z and r^2 within a cell, Maxwellian velocities
 * (Philox draws keyed by the particle id), zero acceleration; then deposit
 * the charge (Sec. 2.4).  Arrays in cfg are copied; the caller keeps them.
 * Errors: PIC_ERR_ARG (bad mesh, species, tables, capacities),
 * PIC_ERR_CUDA (allocation or launch).  *out is NULL on error.
 */
pic_status pic_init(const pic_config *cfg, pic_handle **out);

/*
 * pic_step -- advance nsteps implicit timesteps (Sec. 2.1 cycle in its
 * merged form): rho and chi from the deposit at x~ (Sec. 2.1, 2.4), solve
 * div[(1+chi) grad phi] = -rho/eps0 by z-semi-coarsening multigrid
 * (Sec. 2.5, Algorithm 1), E = -grad phi, then one pass over the particles:
 * gather E, final push, axis reflection and wall absorption (Sec. 2.3),
 * null-collision Monte Carlo (Sec. 2.6), weight splitting on split steps
 * (Sec. 2.2), first push of the next step in the local X-Y frame with the
 * theta rotation (Sec. 2.3), deposit of rho and chi, and a re-sort of the
 * particles by cell (Sec. 2.1 merged cycle).  The steps run without host
 * synchronisation, each as one CUDA graph replay (captured on first use per
 * buffer parity, on a private stream ordered after and before the handle's
 * stream; launched one by one while profiling is on); the call synchronises
 * once at the end.  Returns the first non-OK status of the steps;
 * PIC_ERR_NOT_CONVERGED is non-fatal (the step completes).  On
 * PIC_ERR_CAPACITY and PIC_ERR_TIMEOUT the particle state is left at the last
 * completed step.  The last pass's re-sort is checked for capacity before
 * the call returns; its rank and births numbering run beside the next
 * step's solve, or at the start of the next call that reads or replaces the
 * particle state (pic_get_particles, pic_set_particles, pic_get_counts,
 * pic_set_step, pic_save, pic_load, pic_window).  Should that numbering time
 * out (PIC_ERR_TIMEOUT from that call), the pass is dropped and the state is
 * left at the step before it.
 */
pic_status pic_step(pic_handle *h, int32_t nsteps);

/*
 * Batched reactors (no counterpart in the paper, which runs one reactor).
 * pic_batch_init groups n distinct handles (each made by pic_init: any mesh,
 * particle count and precision); the caller keeps ownership of the handles
 * and must destroy the batch before them.  pic_batch_step advances every
 * reactor by nsteps timesteps: each step of all reactors is one CUDA graph
 * launch that forks into one branch per reactor (its whole timestep, as
 * pic_step would run it) and joins, so the GPU runs the reactors side by
 * side.  The work is ordered after `stream` (a cudaStream_t; NULL: the legacy
 * default stream) and after each handle's own stream, and before them again;
 * the call synchronises once.  statuses (NULL or n entries) receives what
 * pic_step would have returned for each handle; the return value is the
 * first non-OK one.  Handles must have profiling off.  Errors: PIC_ERR_ARG
 * (null, repeated handle, n < 1, a handle that subcycles its ions),
 * PIC_ERR_CUDA (streams, events).
 */
pic_status pic_batch_init(pic_handle *const *handles, int32_t n, void *stream, pic_batch **out);

/*
 * pic_tune -- choose the particle pass's shape per species (no counterpart
 * in the paper).  Shapes: 0 direct loads, 1 the chunk's particles prefetched
 * into shared memory (cp.async), 2 and 3 the same with 8 instead of 4
 * particles per thread; -1 the default (electrons 2, ions 1).  With
 * steps_per_variant > 0 every shape runs that many real steps of this
 * reactor (the simulation advances) with CUDA events around each species'
 * pass, the fastest per species is kept and, if variants is not NULL,
 * written to variants[0..1] (electrons, ions).  With steps_per_variant = 0
 * the shapes are set from variants[0..1].  Captured step graphs are dropped.
 * Errors: PIC_ERR_ARG, and any error of the timed steps.
 */
pic_status pic_tune(pic_handle *h, int32_t steps_per_variant, int32_t *variants);
pic_status pic_batch_step(pic_batch *b, int32_t nsteps, pic_status *statuses);
void pic_batch_destroy(pic_batch *b);

/*
 * pic_field_solve -- stand-alone solve of Eq. (2) (Sec. 2.1, 2.5) on the
 * handle's mesh: rho (C/m^3) and chi (dimensionless) in, phi (V) out, all
 * [nz][nr] FP64; z = 0 at potential V, z = L at the configured phi_zL (or
 * 0), r = R at 0.  Cold start (zero interior).  Pointers are host memory
 * unless on_device.  Does not touch the simulation's fields.  info may be
 * NULL.  Returns PIC_ERR_NOT_CONVERGED if mg_max_cycles was reached.
 */
pic_status pic_field_solve(pic_handle *h, const double *rho, const double *chi, double V,
                           double *phi, int32_t on_device, pic_solve_info *info);

/*
 * pic_field_solve_noalloc -- the same FP64 multigrid solve as pic_field_solve,
 * without a handle and without allocating any device memory.  The paper has
 * no counterpart: this entry point exists for callers that cannot allocate
 * when they need a solve -- hosts that give the library a fixed memory budget
 * at start-up and allow no growth afterwards, real-time loops that must not
 * stall on an allocation.
 *
 * rho, chi (in) and phi (out) are caller-owned DEVICE arrays [nz][nr]; phi_zL
 * is a device array of nr potentials on z = L or NULL (grounded); z = 0 is
 * at V, r = R grounded.  Cold start, at most max_cycles V-cycles, tolerance
 * tol as mg_tol in pic_config.  Work is issued on `stream` (a cudaStream_t,
 * NULL for the legacy stream); the residual is read back to the host after
 * every V-cycle, so the call synchronises `stream` and the solve is finished
 * when it returns.  info (host) may be NULL.
 *
 * Workspace: one fixed device array of 800,000 doubles (6.4 MB) compiled
 * into the library, held on every GPU that loads it until the process
 * exits; it fits meshes up to 129 x 513 nodes.  A larger mesh is rejected
 * with PIC_ERR_ARG and a message on stderr; bad arguments likewise.  The
 * first call on a device looks up the workspace's device address with that
 * device current and keeps it for the process; make that first call before
 * any stream capture begins.  The kept address does not survive a device
 * reset (cudaDeviceReset): do not call this entry point after one.  All
 * calls share the one workspace, which keeps the last call's contents: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller.  Errors: PIC_ERR_ARG, PIC_ERR_CUDA,
 * PIC_ERR_NOT_CONVERGED (non-fatal, phi holds the last iterate).
 */
pic_status pic_field_solve_noalloc(double R, double L, int32_t nz, int32_t nr, int32_t chi_face,
                                   const double *rho, const double *chi, double V,
                                   const double *phi_zL, double *phi, double tol,
                                   int32_t max_cycles, void *stream, pic_solve_info *info);

/*
 * pic_moments -- time averages over the steps since the last reset (Sec. 3:
 * results are averages over time) of n_e, n_i (m^-3, deposit over node
 * volumes, Eq. (10)), phi, E_r, E_z; the electron energy distribution
 * (weighted, after collisions) summed per step and divided by the steps;
 * counters and absorbed charge since the last reset.  Caller-owned
 * buffers; NULL members are skipped.  reset != 0 clears the averages and
 * counters after copying them out.
 */
pic_status pic_moments(pic_handle *h, pic_moments_out *out, int32_t reset);

/*
 * pic_get_particles -- copy the particles of species s (0 e, 1 ion) into
 * the host arrays of *view, at most `capacity` of them, in cell order;
 * view->n is set to the number copied.  Positions are the stored x~
 * (after the first push of the next step, Sec. 2.1).
 */
pic_status pic_get_particles(pic_handle *h, int32_t s, pic_particles_view *view,
                             int64_t capacity);

/*
 * pic_set_particles -- replace the particles of species s by view->n host
 * particles (absolute r, z, velocities, accelerations a_bar, weights, ids)
 * and redeposit both species.  Positions must be inside the domain.  The
 * next id given to a newborn is max(id) + 1.  PIC_ERR_CAPACITY if n is
 * larger than the species capacity.
 */
pic_status pic_set_particles(pic_handle *h, int32_t s, const pic_particles_view *view);

/* pic_set_step -- set the step index that keys the Philox draws (Sec. 2.6)
 * and the rf phase of the next solve (t = (step + 1) dt). */
pic_status pic_set_step(pic_handle *h, int64_t step);

/* pic_set_boundary -- set the nr potentials on z = L used by the next
 * solves (Sec. 2.5 Dirichlet data); phi_zL NULL grounds it again. */
pic_status pic_set_boundary(pic_handle *h, const double *phi_zL, int32_t on_device);

/* pic_get_fields -- copy rho, chi, phi, E_z, E_r of the last step ([nz][nr],
 * rho/chi are the ones of the deposit held now); NULL members skipped. */
pic_status pic_get_fields(pic_handle *h, double *rho, double *chi, double *phi, double *Ez,
                          double *Er, int32_t on_device);

/*
 * pic_get_deposit / pic_set_deposit -- the particle deposit the next step's
 * field solve takes, for a reactor whose particles are shared among
 * processes (Sec. 2.7: each process deposits its own particles, the sums are
 * all-reduced, and every process then solves the same field, as the paper's
 * MPI version does).  Ne, Ni: the electron and ion deposits, [nz][nr] FP64,
 * the sums over particles of weight x shape factor at each node (Eq. (10)
 * before the division by the node volume); q: 3 doubles, the charge
 * absorbed at z = 0, z = L and r = R since the last external-circuit solve
 * (the whole run without a circuit), which the circuit's electrode charge
 * takes.  Valid between calls that step: after pic_step returns they hold
 * this handle's deposit of its last pass; what pic_set_deposit writes is
 * what the next step solves with.  The time averages of pic_moments are
 * taken before any exchange, from this handle's own deposit, and add up
 * across processes.  NULL members are skipped; pointers are host memory
 * unless on_device (then device memory, ordered on the handle's stream).
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA.
 */
pic_status pic_get_deposit(pic_handle *h, double *Ne, double *Ni, double *q, int32_t on_device);
pic_status pic_set_deposit(pic_handle *h, const double *Ne, const double *Ni, const double *q,
                           int32_t on_device);

/*
 * pic_set_id_stride -- number this handle's newborns next_id[s] + stride x
 * (rank of their key) for species s, next_id advancing by stride x births
 * (no counterpart in the paper; the default is the stride 1 of the
 * canonical numbering).  With the particles of one reactor shared among P
 * processes, process r sets stride P and next_id[s] = N_s + r (N_s above
 * every id in use) so that newborn ids stay unique across the processes;
 * since every draw is keyed by the particle id, a newborn's history then
 * differs from the one-process run's, which is statistically the same.
 * next_id: 2 values, host.  Errors: PIC_ERR_ARG (stride 0, null).
 */
pic_status pic_set_id_stride(pic_handle *h, const uint64_t *next_id, uint64_t stride);

/* pic_get_counts -- particles alive per species, steps taken, next ids. */
pic_status pic_get_counts(pic_handle *h, int64_t *n_alive, int64_t *step, uint64_t *next_id);

/* pic_save / pic_load -- checkpoint: particles, phi and the step before's
 * phi (the solve's extrapolated start), the deposit, step, ids, and the
 * circuit state when there is one.  Resuming is bit-exact because every
 * draw is keyed by (id, step).  pic_load rejects (PIC_ERR_ARG) a file of
 * another mesh, pusher, subcycling or circuit setting, and one written in
 * an earlier format. */
/*
 * pic_get_circuit -- state of the external circuit after the last step:
 * out[0] electrode voltage V (V), out[1] electrode charge Q (C), out[2]
 * capacitor charge Q_c = circuit_C (V_rf - V) (C).  All zero without a
 * circuit.  out: 3 doubles, host memory.
 */
pic_status pic_get_circuit(pic_handle *h, double *out);

/*
 * pic_merge -- combine light particles of species s in pairs (Sec. 2.2 says
 * small particles sometimes need combining and gives no algorithm; this is
 * the library's reading).  Particles lighter than frac times the split's
 * reference weight of their radial cell are grouped by cell and by velocity
 * bin (each component's floor(v / dv), dv in m/s), taken in order of id
 * within a group, and merged in pairs into the lower id: weight summed; z,
 * r^2, v_r, v_z, a_r, a_z as weight-means; v_theta (and a_theta) so that the
 * angular momentum is kept at the merged radius.  Charge, the z and r^2
 * moments (hence the cell and the deposit's totals and first moments),
 * radial and axial momentum, angular momentum and sum w a are kept; the
 * kinetic energy of the pairs' velocity spread is lost and returned in
 * *energy_J (nullable), the pairs in *pairs (nullable).  The deposit is
 * redone.  Errors: PIC_ERR_ARG (s, frac or dv), PIC_ERR_CAPACITY (a cell
 * with more than 1024 light particles of s: that cell is left as it was),
 * PIC_ERR_CUDA.
 */
pic_status pic_merge(pic_handle *h, int32_t s, double frac, double dv, int64_t *pairs, double *energy_J);

/*
 * pic_window -- a collisionless window of the timestep and the gradient of a
 * time-averaged ion-density functional by a hand-written adjoint (the
 * paper's timestep, Sec. 2.1 merged cycle, with the Monte Carlo step of
 * Sec. 2.6 off: no collisions, births or splitting whatever the cross
 * sections; the adjoint has no counterpart in the paper).
 *
 * From the handle's current particles and step index, takes nsteps steps
 * with the first rf component's amplitude set to amp0 (V) and the z = L row
 * of the potential set to phi_zL (nr values, V, host; NULL: zeros), and
 * returns in *J the functional
 *     J = (1/nsteps) sum_{n=1..nsteps} sum_k w[k] N_i^n(k),
 * N_i^n the ion deposit after step n (the time average of the volume
 * integral of w n_i), w: nz*nr doubles, host, row-major [i][j].  With grad
 * != 0 also *dJ_damp = dJ/d amp0 and dJ_dphi_zL[0..nr-1] = dJ/d phi_zL
 * (host).  The forward runs in the handle's precision; the adjoint is
 * FP64.  The forward keeps the particle state every ckpt steps and the
 * backward recomputes one such segment at a time (memory: about
 * (nsteps/ckpt + ckpt) particle states).  Particles keep their slots (no
 * sort) and one that reaches a wall leaves the sums.  The handle's own
 * state (particles, fields, step, counters) is unchanged.
 * Errors: PIC_ERR_ARG (nsteps < 1, ckpt < 1, null w, no rf component, the
 * X-Y-Z pusher, ion subcycling), PIC_ERR_NOT_CONVERGED / PIC_ERR_TIMEOUT (a solve of the window),
 * PIC_ERR_CUDA (device memory).
 */
pic_status pic_window(pic_handle *h, int32_t nsteps, int32_t ckpt, const double *w, double amp0,
                      const double *phi_zL, int32_t grad, double *J, double *dJ_damp, double *dJ_dphi_zL);

pic_status pic_save(pic_handle *h, const char *path);
pic_status pic_load(pic_handle *h, const char *path);

/* pic_profile -- when on, steps launch one by one (no graph) and CUDA events
 * bracket each phase of every step on the handle's stream.  pic_timings
 * returns the accumulated milliseconds per phase [0 solve, 1 electron pass,
 * 2 ion pass, 3 sort and births, 4 moments and step end], the number of
 * particle-kernel launches, and the number of all kernel launches this
 * handle has made (graph nodes included). */
pic_status pic_profile(pic_handle *h, int32_t on);
pic_status pic_timings(pic_handle *h, double *ms, int64_t *particle_launches,
                       int64_t *all_launches, int32_t reset);

/*
 * pic_selftest_wait -- failure-detection self-test (no counterpart in the
 * paper).  Every wait of the library's cooperative kernels (grid barriers,
 * bulk-copy completions) gives up after a bounded number of polls and
 * reports PIC_ERR_TIMEOUT instead of hanging.  This runs that barrier with
 * one block waiting for a second participant that is never launched, with a
 * limit of `polls` (256 to the library's own limit): *gave_up = 1 when the
 * wait ran out and returned, as it must; the CUDA context stays usable.
 * Errors: PIC_ERR_ARG, PIC_ERR_CUDA.
 */
pic_status pic_selftest_wait(int64_t polls, int32_t *gave_up);

/*
 * pic_fp64_fma_rate -- measured FP64 rate of the current device (no
 * counterpart in the paper): a plain kernel of independent fused
 * multiply-add chains (8 per thread, `iters` FMAs each, 8 blocks of 256
 * threads per SM), timed with CUDA events after one warm-up launch; *gflops
 * = 2 x FMAs / time in GFLOP/s.  It is the peak the FP64 particle pass is
 * compared with.  Allocates and frees a small device buffer; synchronises
 * the device.  Errors: PIC_ERR_ARG (iters outside 16 .. 2^20, null
 * gflops), PIC_ERR_CUDA.
 */
pic_status pic_fp64_fma_rate(int32_t iters, double *gflops);

void pic_destroy(pic_handle *h);
const char *pic_last_error(const pic_handle *h);
const char *pic_status_string(pic_status s);

#ifdef __cplusplus
}
#endif
#endif
