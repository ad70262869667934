/*
 * oracle.h -- plain, serial, FP64 CPU oracle of one implicit electrostatic
 * PIC/MC timestep in axisymmetric r-z geometry (Wang, Jiang & Wang,
 * "Implicit and electrostatic Particle-in-cell/Monte Carlo model in
 * two-dimensional and axisymmetric geometry I", arXiv:1001.2969).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load this library.  The product
 * library shares no code, header, table or constant with it, and neither
 * includes nor links the other.
 *
 * Every function follows the paper in the paper's order and notation,
 * in absolute (r, z) coordinates and SI units.  Readings of the places
 * where the paper is silent or garbled are stated next to the code that
 * implements them.
 *
 * Parity status: every function is pinned by a test that does not reuse
 * the oracle's own formulas (closed forms, invariants, library routines,
 * published test vectors).  Nothing here is "parity unpinned".
 */
#ifndef ORC_ORACLE_H
#define ORC_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_MAX_CH 4

/* channel kinds (Sec. 2.6) */
#define ORC_ELASTIC 0
#define ORC_EXCITE 1
#define ORC_IONIZE 2
#define ORC_CX 3

/* shape functions (Sec. 2.4) */
#define ORC_ZR2 0
#define ORC_ZR 1

/* face susceptibility rule (Sec. 2.5) */
#define ORC_CHI_MAX 0
#define ORC_CHI_MEAN 1

/* scattering law */
#define ORC_SCATTER_VS 0
#define ORC_SCATTER_ISO 1

/* counter slots (int64) */
#define ORC_C_COLL 0        /* [s*4 + ch] real collisions, 8 slots   */
#define ORC_C_CAND 8        /* [s] null-collision candidates          */
#define ORC_C_NUOVER 10     /* [s] nu > nu_max events                 */
#define ORC_C_BIRTHS 12     /* [s] particles born (ionisation+split)  */
#define ORC_C_SPLITS 14     /* [s] parents that were split           */
#define ORC_C_ABS 16        /* [s*3 + wall] absorbed particles, 6     */
#define ORC_C_NCOUNT 24

/* charge slots (double): absorbed charge per wall z=0, z=L, r=R */
#define ORC_Q_NCOUNT 3

typedef struct {
    double R, L;
    int32_t nz, nr;
    /* species 0 = electrons, 1 = ions */
    double q[2], m[2], n0[2], T_eV[2];
    int64_t n_init[2];
    /* cross sections on the uniform grid E_k = k*E_max/(n_e-1) */
    int32_t xs_ne[2];
    double xs_emax[2];
    int32_t xs_nch[2];
    const double *xs_sigma[2]; /* [n_ch][n_e] */
    const double *xs_thr[2];   /* [n_ch] */
    const int32_t *xs_kind[2]; /* [n_ch] */
    double xs_B[2];            /* ionisation energy-sharing parameter (eV) */
    /* rf waveform on the z=0 electrode */
    int32_t rf_n;
    const double *rf_amp, *rf_freq, *rf_phase;
    /* background gas */
    double p_Pa, T_K, m_gas;
    double dt;
    uint64_t seed;
    int32_t weighting, chi_face, scatter, split_every, mg_max_cycles;
    double mg_tol;
    const double *phi_zL; /* nullable: nr potentials on z = L */
    int32_t eedf_bins;
    double eedf_emax;
    /* external circuit (Sec. 2.5, end): blocking capacitor (F) between the
     * rf source and the z = 0 electrode; 0 drives the electrode directly */
    double circuit_C;
    /* pusher (Sec. 2.3): 0 the local X-Y frame with a_theta dropped, 1 the
     * global X-Y-Z form (a_theta carried) */
    int32_t pusher;
    /* ion subcycling (Sec. 2.7): ions move in every K-th pass only, with
     * dt_i = K dt; 0 or 1 moves them every pass */
    int32_t ion_subcycle;
    /* starting value w_0 of a timestep's V-cycles (Algorithm 1 leaves it
     * open): 0 the last step's potential, 1 the linear extrapolation
     * 2 phi^n - phi^(n-1) from the last two steps on the interior nodes
     * (plain solves only; the circuit's two solves start from their last
     * solutions) */
    int32_t mg_guess;
} orc_config;

typedef struct orc_state orc_state;

/* lifetime */
orc_state *orc_create(const orc_config *cfg, int64_t capacity);
/* a_theta of species s (X-Y-Z pusher; zero otherwise and for set/loaded particles) */
void orc_get_at(const orc_state *st, int s, double *at);
void orc_set_at(orc_state *st, int s, const double *at);
void orc_destroy(orc_state *st);

/* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11) */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* particle store access (absolute FP64 coordinates) */
int64_t orc_count(const orc_state *st, int s);
void orc_set_particles(orc_state *st, int s, int64_t n, const double *r, const double *z,
                       const double *vr, const double *vt, const double *vz, const double *ar,
                       const double *az, const double *w, const uint64_t *id);
void orc_get_particles(const orc_state *st, int s, double *r, double *z, double *vr, double *vt,
                       double *vz, double *ar, double *az, double *w, uint64_t *id);
void orc_set_next_id(orc_state *st, int s, uint64_t next_id);
uint64_t orc_get_next_id(const orc_state *st, int s);
void orc_set_step(orc_state *st, int64_t step);
int64_t orc_get_step(const orc_state *st);
/* 1 when the next pass moves the ions (always without subcycling) */
int orc_ion_pass(const orc_state *st);
/* merge light particles of species s in pairs (see oracle.c); returns the
 * pairs merged, *energy_J the kinetic energy their velocity spread held */
int64_t orc_merge(orc_state *st, int s, double frac, double dv, double *energy_J);

/* external circuit state: out[0] electrode voltage V, out[1] electrode
 * charge Q, out[2] capacitor charge Q_c (C, after the last step) */
void orc_get_circuit(const orc_state *st, double out[3]);

/* loading: the whole load, or particles [p0, p1) of species s only */
void orc_load(orc_state *st);
void orc_load_range(const orc_state *st, int s, int64_t p0, int64_t p1, double *r, double *z,
                    double *vr, double *vt, double *vz, double *ar, double *az, double *w,
                    uint64_t *id);

/* grids, all [nz][nr] row-major */
void orc_deposit(orc_state *st);               /* N_s from the stored positions */
void orc_finalize(orc_state *st);              /* rho, chi from N_s               */
void orc_node_volumes(const orc_state *st, double *V);
void orc_get_grid(const orc_state *st, int which, double *out); /* 0 N_e,1 N_i,2 rho,3 chi,4 phi,5 Ez,6 Er */
void orc_set_grid(orc_state *st, int which, const double *in);

/* field solve of div[(1+chi) grad phi] = -rho/eps0 with phi(z=0)=V */
double orc_voltage(const orc_state *st, double t);
int orc_solve(orc_state *st, double V, double tol, int max_cycles, int *cycles, double *rel_res);
void orc_apply_A(const orc_state *st, const double *chi, const double *u, double *Au);
void orc_rhs(const orc_state *st, const double *rho, double *f);
void orc_efield(orc_state *st);

/* one merged particle pass with the stored E; then one full step */
void orc_particle_pass(orc_state *st);
void orc_step(orc_state *st, int nsteps, int *last_cycles, double *last_res);

/* diagnostics */
void orc_get_counters(const orc_state *st, int64_t *c, double *q);
void orc_reset_counters(orc_state *st);
void orc_get_moments(const orc_state *st, double *ne, double *ni, double *phi, double *Ez,
                     double *Er, double *eedf, int64_t *nsamples);
void orc_reset_moments(orc_state *st);

/* pieces exposed for pins */
double orc_sigma(const orc_state *st, int s, int ch, double E_eV);
double orc_nu_max(const orc_state *st, int s);
double orc_p_null(const orc_state *st, int s);
double orc_cos_chi(const orc_state *st, double eps_eV, double R);
void orc_scatter_dir(double ux, double uy, double uz, double cos_chi, double phi, double out[3]);
double orc_ejected_energy(double eps_eV, double thr_eV, double B_eV, double R);
double orc_w_ref(const orc_state *st, int s, int j);

#ifdef __cplusplus
}
#endif
#endif
