/*
 * oracle.c -- plain FP64 CPU oracle of the implicit electrostatic PIC/MC
 * timestep in axisymmetric r-z geometry (Wang, Jiang & Wang,
 * arXiv:1001.2969).  TEST INFRASTRUCTURE ONLY: used by the tests, the smoke
 * check and the CPU-baseline leg of the benchmark, never by the product.
 *
 * Written to be read against the paper: absolute coordinates, SI units,
 * serial loops, no blocking, fusion or reordering beyond the paper's own
 * step order.  Build: gcc -O2 -ffp-contract=off (no FMA contraction, so
 * the arithmetic is the plain IEEE sequence written here).
 *
 * Readings where the paper is silent or garbled are marked READING.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* CODATA 2018 values */
static const double ORC_E = 1.602176634e-19;    /* elementary charge, C */
static const double ORC_EPS0 = 8.8541878128e-12; /* vacuum permittivity, F/m */
static const double ORC_KB = 1.380649e-23;      /* Boltzmann constant, J/K */
static const double ORC_PI = 3.14159265358979323846;

#define ORC_SPLIT_NMAX 4096 /* READING: cap on copies per parent per split */

typedef struct {
    int64_t n;
    double *r, *z, *vr, *vt, *vz, *ar, *az, *w;
    double *at; /* a_theta: carried by the X-Y-Z pusher only */
    uint64_t *id;
} orc_store;

typedef struct {
    int ts;       /* species of the newborn              */
    int ps;       /* species of the parent               */
    uint64_t pid; /* parent id                           */
    int k;        /* birth slot within the parent's pass */
    double r, z, vr, vt, vz, ar, az, w, at;
} orc_birth;

struct orc_state {
    orc_config c;
    double *own_sigma[2], *own_thr[2], *own_rf, *own_phiL;
    int32_t *own_kind[2];
    double dz, dr;
    int64_t cap;
    orc_store p[2];
    uint64_t next_id[2];
    int64_t step;
    double *N[2], *rho, *chi, *phi, *Ez, *Er;
    double ng, nu_max[2], p_null[2];
    int64_t cnt[ORC_C_NCOUNT];
    double qabs[ORC_Q_NCOUNT];
    double qpass[ORC_Q_NCOUNT]; /* absorbed charge of the last particle pass */
    /* external circuit: superposition parts of phi and the circuit state */
    double *phiP, *phiL, *zero;
    double *phi_prev; /* the potential of the step before phi's (mg_guess) */
    double circ_V, circ_Q, circ_Qc;
    /* births of the current pass */
    orc_birth *b;
    int64_t nb, bcap;
    /* time-averaged moments */
    double *m_ne, *m_ni, *m_phi, *m_ez, *m_er, *m_eedf;
    int64_t m_n;
    double *eedf_pass;
};

/* ------------------------------------------------------------------ */
/* Philox4x32-10, from the definition in Salmon et al., SC'11:         */
/* round: (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2),                */
/*                         hi(M0*c0)^c3^k1, lo(M0*c0)),                */
/* key schedule k0 += 0x9E3779B9, k1 += 0xBB67AE85 between rounds.      */
/* ------------------------------------------------------------------ */
void orc_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* draws of particle `id` of species s at pass `step` on `stream` */
static void orc_draw(const orc_state *st, int s, uint64_t id, uint32_t step, int stream,
                     uint32_t x[4]) {
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, (uint32_t)(stream * 2 + s)};
    uint32_t key[2] = {(uint32_t)st->c.seed, (uint32_t)(st->c.seed >> 32)};
    orc_philox(ctr, key, x);
}

/* uniform on (0,1): ((x + 1/2) / 2^32) */
static double orc_u(uint32_t x) { return ((double)x + 0.5) * (1.0 / 4294967296.0); }

/* Box-Muller pair of standard normals from two words */
static void orc_normals(uint32_t xa, uint32_t xb, double *n0, double *n1) {
    double ua = orc_u(xa), ub = orc_u(xb);
    double rad = sqrt(-2.0 * log(ua));
    *n0 = rad * cos(2.0 * ORC_PI * ub);
    *n1 = rad * sin(2.0 * ORC_PI * ub);
}

/* ------------------------------------------------------------------ */
/* mesh                                                                 */
/* ------------------------------------------------------------------ */
#define IDX(i, j) ((int64_t)(i) * st->c.nr + (j))

static double zi(const orc_state *st, int i) { return i * st->dz; }
static double rj(const orc_state *st, int j) { return j * st->dr; }

static int cell_z(const orc_state *st, double z) {
    int i = (int)floor(z / st->dz);
    if (i < 0) i = 0;
    if (i > st->c.nz - 2) i = st->c.nz - 2;
    return i;
}
static int cell_r(const orc_state *st, double r) {
    int j = (int)floor(r / st->dr);
    if (j < 0) j = 0;
    if (j > st->c.nr - 2) j = st->c.nr - 2;
    return j;
}

/*
 * Shape factors of a particle at (r, z) in cell (i, j) (Sec. 2.4).
 * z: linear, (z_{i+1}-z)/(z_{i+1}-z_i).  r: z-r weighting, Eq. (8):
 * (r_{j+1}-r)/(r_{j+1}-r_j); z-r^2 weighting, Eq. (9):
 * (r_{j+1}^2-r^2)/(r_{j+1}^2-r_j^2).
 */
static void shape(const orc_state *st, double r, double z, int i, int j, double Sz[2],
                  double Sr[2]) {
    double z0 = zi(st, i), z1 = zi(st, i + 1);
    Sz[0] = (z1 - z) / (z1 - z0);
    Sz[1] = (z - z0) / (z1 - z0);
    double r0 = rj(st, j), r1 = rj(st, j + 1);
    if (st->c.weighting == ORC_ZR) {
        Sr[0] = (r1 - r) / (r1 - r0);
        Sr[1] = (r - r0) / (r1 - r0);
    } else {
        Sr[0] = (r1 * r1 - r * r) / (r1 * r1 - r0 * r0);
        Sr[1] = (r * r - r0 * r0) / (r1 * r1 - r0 * r0);
    }
}

/*
 * Node volumes V_{i,j} (Sec. 2.4, after Eq. (10)).
 * z-r:   V_j = pi/3 [r_{j+1}(r_j+r_{j+1}) - r_{j-1}(r_j+r_{j-1})] dz, V_0 = pi/3 r_1^2 dz
 * z-r^2: V_j = pi/2 (r_{j+1}^2 - r_{j-1}^2) dz,                     V_0 = pi/2 r_1^2 dz
 * READING: on the boundary rows i = 0, nz-1 only the inner half in z counts,
 * and on j = nr-1 only the inner part of the support in r (the part
 * inside the domain).  These are Dirichlet nodes; only diagnostics use them.
 */
void orc_node_volumes(const orc_state *st, double *V) {
    int nz = st->c.nz, nr = st->c.nr;
    for (int i = 0; i < nz; ++i) {
        double hz = (i == 0 || i == nz - 1) ? 0.5 * st->dz : st->dz;
        for (int j = 0; j < nr; ++j) {
            double v;
            double r = rj(st, j);
            if (st->c.weighting == ORC_ZR) {
                if (j == 0) {
                    double r1 = rj(st, 1);
                    v = ORC_PI / 3.0 * r1 * r1;
                } else if (j == nr - 1) {
                    /* inner part: int_{r_{j-1}}^{r_j} (r'-r_{j-1})/dr 2 pi r' dr' */
                    double rm = rj(st, j - 1);
                    v = ORC_PI / 3.0 * st->dr * (2.0 * r + rm);
                } else {
                    double rp = rj(st, j + 1), rm = rj(st, j - 1);
                    v = ORC_PI / 3.0 * (rp * (r + rp) - rm * (r + rm));
                }
            } else {
                if (j == 0) {
                    double r1 = rj(st, 1);
                    v = ORC_PI / 2.0 * r1 * r1;
                } else if (j == nr - 1) {
                    double rm = rj(st, j - 1);
                    v = ORC_PI / 2.0 * (r * r - rm * rm);
                } else {
                    double rp = rj(st, j + 1), rm = rj(st, j - 1);
                    v = ORC_PI / 2.0 * (rp * rp - rm * rm);
                }
            }
            V[IDX(i, j)] = v * hz;
        }
    }
}

/* ------------------------------------------------------------------ */
/* cross sections and collision frequencies (Sec. 2.6)                  */
/* ------------------------------------------------------------------ */

/* sigma_ch(E): linear interpolation on the table, 1/E law above it */
double orc_sigma(const orc_state *st, int s, int ch, double E) {
    int ne = st->c.xs_ne[s];
    double emax = st->c.xs_emax[s];
    const double *sg = st->c.xs_sigma[s] + (int64_t)ch * ne;
    if (E >= emax) return sg[ne - 1] * emax / E;
    if (E <= 0.0) return sg[0];
    double dE = emax / (ne - 1);
    double x = E / dE;
    int k = (int)floor(x);
    if (k > ne - 2) k = ne - 2;
    double f = x - k;
    return sg[k] + f * (sg[k + 1] - sg[k]);
}

static double orc_sigma_tot_node(const orc_state *st, int s, int k) {
    int ne = st->c.xs_ne[s];
    double t = 0.0;
    for (int ch = 0; ch < st->c.xs_nch[s]; ++ch) t += st->c.xs_sigma[s][(int64_t)ch * ne + k];
    return t;
}

/*
 * nu_max = n_g * max_E sigma_tot(E) g(E), g = sqrt(2 E e / m).  sigma_tot is
 * linear on each table segment, sigma = alpha + beta E, so on a falling
 * segment the product has its stationary point at E* = -alpha/(3 beta);
 * beyond the table nu falls as E^-1/2.  READING: a relative margin of 1e-6
 * keeps rounding in the per-particle nu below nu_max.
 */
static double orc_compute_nu_max(const orc_state *st, int s) {
    int ne = st->c.xs_ne[s];
    double emax = st->c.xs_emax[s];
    double dE = emax / (ne - 1);
    double m = st->c.m[s];
    double best = 0.0;
    for (int k = 0; k < ne; ++k) {
        double E = k * dE;
        double v = orc_sigma_tot_node(st, s, k) * sqrt(2.0 * E * ORC_E / m);
        if (v > best) best = v;
    }
    for (int k = 0; k + 1 < ne; ++k) {
        double s0 = orc_sigma_tot_node(st, s, k), s1 = orc_sigma_tot_node(st, s, k + 1);
        double beta = (s1 - s0) / dE;
        if (beta < 0.0) {
            double alpha = s0 - beta * (k * dE);
            double Es = -alpha / (3.0 * beta);
            if (Es > k * dE && Es < (k + 1) * dE) {
                double v = (alpha + beta * Es) * sqrt(2.0 * Es * ORC_E / m);
                if (v > best) best = v;
            }
        }
    }
    return st->ng * best * (1.0 + 1e-6);
}

double orc_nu_max(const orc_state *st, int s) { return st->nu_max[s]; }
double orc_p_null(const orc_state *st, int s) { return st->p_null[s]; }

/*
 * Scattering angle of an electron of energy eps (eV), Vahedi & Surendra
 * (1995) as cited in Sec. 2.6: cos chi = (2 + eps - 2 (1+eps)^R) / eps.
 * Below 1e-6 eV the law is isotropic, cos chi = 1 - 2R (its eps -> 0 limit).
 */
double orc_cos_chi(const orc_state *st, double eps, double R) {
    double c;
    if (st->c.scatter == ORC_SCATTER_ISO || eps < 1e-6)
        c = 1.0 - 2.0 * R;
    else
        c = (2.0 + eps - 2.0 * pow(1.0 + eps, R)) / eps;
    if (c > 1.0) c = 1.0;
    if (c < -1.0) c = -1.0;
    return c;
}

/*
 * New unit direction after scattering by (chi, phi) about the incident unit
 * vector u (Vahedi & Surendra 1995, with the z axis as reference):
 *   u' = cos(chi) u + sin(chi) [cos(phi) e1 + sin(phi) e2],
 *   e1 = (u_y, -u_x, 0)/s, e2 = u x e1 = (u_x u_z, u_y u_z, -s^2)/s,
 *   s = sqrt(u_x^2 + u_y^2).  When u is along z, e1 = x, e2 = (0, u_z, 0).
 */
void orc_scatter_dir(double ux, double uy, double uz, double cos_chi, double phi,
                     double out[3]) {
    double sin_chi = sqrt(fmax(0.0, 1.0 - cos_chi * cos_chi));
    double cp = cos(phi), sp = sin(phi);
    double s2 = ux * ux + uy * uy;
    if (s2 < 1e-24) {
        out[0] = sin_chi * cp;
        out[1] = sin_chi * sp * uz;
        out[2] = cos_chi * uz;
        return;
    }
    double s = sqrt(s2);
    out[0] = cos_chi * ux + sin_chi * (cp * uy + sp * ux * uz) / s;
    out[1] = cos_chi * uy + sin_chi * (-cp * ux + sp * uy * uz) / s;
    out[2] = cos_chi * uz + sin_chi * (-sp * s2) / s;
}

/*
 * Energy of the ejected electron in an ionisation, Opal's form as used by
 * Vahedi & Surendra: eps_ej = B tan(R atan((eps - thr)/(2B))).
 */
double orc_ejected_energy(double eps, double thr, double B, double R) {
    return B * tan(R * atan((eps - thr) / (2.0 * B)));
}

/* ------------------------------------------------------------------ */
/* lifetime                                                             */
/* ------------------------------------------------------------------ */
static void *xmalloc(size_t n) {
    void *p = calloc(1, n ? n : 1);
    return p;
}

static void store_alloc(orc_store *s, int64_t cap) {
    s->n = 0;
    s->r = xmalloc(cap * sizeof(double));
    s->z = xmalloc(cap * sizeof(double));
    s->vr = xmalloc(cap * sizeof(double));
    s->vt = xmalloc(cap * sizeof(double));
    s->vz = xmalloc(cap * sizeof(double));
    s->ar = xmalloc(cap * sizeof(double));
    s->az = xmalloc(cap * sizeof(double));
    s->w = xmalloc(cap * sizeof(double));
    s->at = xmalloc(cap * sizeof(double));
    s->id = xmalloc(cap * sizeof(uint64_t));
}

static void store_free(orc_store *s) {
    free(s->r);
    free(s->z);
    free(s->vr);
    free(s->vt);
    free(s->vz);
    free(s->ar);
    free(s->az);
    free(s->w);
    free(s->at);
    free(s->id);
}

/*
 * Ion subcycling (Sec. 2.7, Vahedi's method, named there without a form for
 * the implicit scheme).  READING: the ions move in the passes n with
 * n mod K = K - 1 (so a split pass, n mod split_every = split_every - 1
 * with K dividing split_every, is always one of them) and are held still,
 * state and deposit, in the others.  A moving pass takes the whole D1
 * cycle with dt_i = K dt: final push, Monte Carlo with
 * P_null = 1 - exp(-nu_max dt_i), first push.  So the ions respond to the
 * field only in the solves that precede their moving passes: their
 * susceptibility enters those solves with dt_i^2 and the others not at
 * all.  Ions born in any pass (ionisation by electrons, splits) take
 * their first push with dt_i, like the ions moved in a pass.
 */
static int subcycle(const orc_state *st) { return st->c.ion_subcycle > 1 ? st->c.ion_subcycle : 1; }

int orc_ion_pass(const orc_state *st) {
    const int K = subcycle(st);
    return (int)(st->step % K) == K - 1;
}

static double dt_of(const orc_state *st, int s) { return s == 1 ? st->c.dt * subcycle(st) : st->c.dt; }

orc_state *orc_create(const orc_config *cfg, int64_t capacity) {
    orc_state *st = xmalloc(sizeof(orc_state));
    st->c = *cfg;
    for (int s = 0; s < 2; ++s) {
        int64_t ns = (int64_t)cfg->xs_nch[s] * cfg->xs_ne[s];
        st->own_sigma[s] = xmalloc(ns * sizeof(double));
        memcpy(st->own_sigma[s], cfg->xs_sigma[s], ns * sizeof(double));
        st->own_thr[s] = xmalloc(cfg->xs_nch[s] * sizeof(double));
        memcpy(st->own_thr[s], cfg->xs_thr[s], cfg->xs_nch[s] * sizeof(double));
        st->own_kind[s] = xmalloc(cfg->xs_nch[s] * sizeof(int32_t));
        memcpy(st->own_kind[s], cfg->xs_kind[s], cfg->xs_nch[s] * sizeof(int32_t));
        st->c.xs_sigma[s] = st->own_sigma[s];
        st->c.xs_thr[s] = st->own_thr[s];
        st->c.xs_kind[s] = st->own_kind[s];
    }
    st->own_rf = xmalloc(3 * (cfg->rf_n > 0 ? cfg->rf_n : 1) * sizeof(double));
    for (int k = 0; k < cfg->rf_n; ++k) {
        st->own_rf[k] = cfg->rf_amp[k];
        st->own_rf[cfg->rf_n + k] = cfg->rf_freq[k];
        st->own_rf[2 * cfg->rf_n + k] = cfg->rf_phase[k];
    }
    st->c.rf_amp = st->own_rf;
    st->c.rf_freq = st->own_rf + cfg->rf_n;
    st->c.rf_phase = st->own_rf + 2 * cfg->rf_n;
    st->own_phiL = NULL;
    if (cfg->phi_zL) {
        st->own_phiL = xmalloc(cfg->nr * sizeof(double));
        memcpy(st->own_phiL, cfg->phi_zL, cfg->nr * sizeof(double));
    }
    st->c.phi_zL = st->own_phiL;

    st->dz = cfg->L / (cfg->nz - 1);
    st->dr = cfg->R / (cfg->nr - 1);
    st->cap = capacity;
    for (int s = 0; s < 2; ++s) {
        store_alloc(&st->p[s], capacity);
        st->next_id[s] = 0;
    }
    int64_t ng = (int64_t)cfg->nz * cfg->nr;
    for (int s = 0; s < 2; ++s) st->N[s] = xmalloc(ng * sizeof(double));
    st->rho = xmalloc(ng * sizeof(double));
    st->chi = xmalloc(ng * sizeof(double));
    st->phi = xmalloc(ng * sizeof(double));
    st->phi_prev = xmalloc(ng * sizeof(double)); /* zero, like phi */
    st->Ez = xmalloc(ng * sizeof(double));
    st->Er = xmalloc(ng * sizeof(double));
    st->phiP = xmalloc(ng * sizeof(double));
    st->phiL = xmalloc(ng * sizeof(double));
    st->zero = xmalloc(ng * sizeof(double));
    st->m_ne = xmalloc(ng * sizeof(double));
    st->m_ni = xmalloc(ng * sizeof(double));
    st->m_phi = xmalloc(ng * sizeof(double));
    st->m_ez = xmalloc(ng * sizeof(double));
    st->m_er = xmalloc(ng * sizeof(double));
    int nb = cfg->eedf_bins > 0 ? cfg->eedf_bins : 1;
    st->m_eedf = xmalloc(nb * sizeof(double));
    st->eedf_pass = xmalloc(nb * sizeof(double));

    /* background gas density n_g = p / (k_B T) */
    st->ng = cfg->p_Pa / (ORC_KB * cfg->T_K);
    for (int s = 0; s < 2; ++s) {
        st->nu_max[s] = orc_compute_nu_max(st, s);
        st->p_null[s] = 1.0 - exp(-st->nu_max[s] * dt_of(st, s));
    }
    st->bcap = 1024;
    st->b = xmalloc(st->bcap * sizeof(orc_birth));
    return st;
}

void orc_destroy(orc_state *st) {
    if (!st) return;
    for (int s = 0; s < 2; ++s) {
        store_free(&st->p[s]);
        free(st->own_sigma[s]);
        free(st->own_thr[s]);
        free(st->own_kind[s]);
        free(st->N[s]);
    }
    free(st->own_rf);
    free(st->own_phiL);
    free(st->rho);
    free(st->chi);
    free(st->phi);
    free(st->phi_prev);
    free(st->Ez);
    free(st->Er);
    free(st->phiP);
    free(st->phiL);
    free(st->zero);
    free(st->m_ne);
    free(st->m_ni);
    free(st->m_phi);
    free(st->m_ez);
    free(st->m_er);
    free(st->m_eedf);
    free(st->eedf_pass);
    free(st->b);
    free(st);
}

int64_t orc_count(const orc_state *st, int s) { return st->p[s].n; }
void orc_set_next_id(orc_state *st, int s, uint64_t v) { st->next_id[s] = v; }
uint64_t orc_get_next_id(const orc_state *st, int s) { return st->next_id[s]; }
void orc_set_step(orc_state *st, int64_t step) { st->step = step; }
int64_t orc_get_step(const orc_state *st) { return st->step; }


void orc_set_particles(orc_state *st, int s, int64_t n, const double *r, const double *z,
                       const double *vr, const double *vt, const double *vz, const double *ar,
                       const double *az, const double *w, const uint64_t *id) {
    orc_store *p = &st->p[s];
    if (n > st->cap) n = st->cap;
    p->n = n;
    memcpy(p->r, r, n * sizeof(double));
    memcpy(p->z, z, n * sizeof(double));
    memcpy(p->vr, vr, n * sizeof(double));
    memcpy(p->vt, vt, n * sizeof(double));
    memcpy(p->vz, vz, n * sizeof(double));
    memcpy(p->ar, ar, n * sizeof(double));
    memcpy(p->az, az, n * sizeof(double));
    memcpy(p->w, w, n * sizeof(double));
    memset(p->at, 0, n * sizeof(double));
    memcpy(p->id, id, n * sizeof(uint64_t));
    uint64_t mx = 0;
    for (int64_t k = 0; k < n; ++k)
        if (id[k] + 1 > mx) mx = id[k] + 1;
    st->next_id[s] = mx;
    orc_deposit(st);
}

void orc_get_at(const orc_state *st, int s, double *at) {
    memcpy(at, st->p[s].at, st->p[s].n * sizeof(double));
}

void orc_set_at(orc_state *st, int s, const double *at) {
    memcpy(st->p[s].at, at, st->p[s].n * sizeof(double));
}

void orc_get_particles(const orc_state *st, int s, double *r, double *z, double *vr, double *vt,
                       double *vz, double *ar, double *az, double *w, uint64_t *id) {
    const orc_store *p = &st->p[s];
    int64_t n = p->n;
    memcpy(r, p->r, n * sizeof(double));
    memcpy(z, p->z, n * sizeof(double));
    memcpy(vr, p->vr, n * sizeof(double));
    memcpy(vt, p->vt, n * sizeof(double));
    memcpy(vz, p->vz, n * sizeof(double));
    memcpy(ar, p->ar, n * sizeof(double));
    memcpy(az, p->az, n * sizeof(double));
    memcpy(w, p->w, n * sizeof(double));
    memcpy(id, p->id, n * sizeof(uint64_t));
}

/* ------------------------------------------------------------------ */
/* loading                                                              */
/* ------------------------------------------------------------------ */

/* reference macro-particle count per cell: the base count of the load */
static int64_t orc_ppc_ref(const orc_state *st, int s) {
    int64_t ncell = (int64_t)(st->c.nz - 1) * (st->c.nr - 1);
    int64_t b = st->c.n_init[s] / ncell;
    return b > 0 ? b : 1;
}

/*
 * Reference weight of radial cell j (Sec. 2.2, Eq. (3), w_p ~ 2 pi r dr dz,
 * in the cell-volume form): n0 pi (r_{j+1}^2 - r_j^2) dz / ppc_ref.
 */
double orc_w_ref(const orc_state *st, int s, int j) {
    double r0 = rj(st, j), r1 = rj(st, j + 1);
    return st->c.n0[s] * ORC_PI * (r1 * r1 - r0 * r0) * st->dz / (double)orc_ppc_ref(st, s);
}

/*
 * Load particles [p0, p1) of species s (READING of the configs: uniform
 * density n0 with weights proportional to the cell volume, Sec. 2.2).
 * Cells are numbered c = j (nz-1) + i.  The N particles are spread
 * N / N_c per cell with the remainder one each in the lowest-numbered
 * cells; particle p has id p.  Inside its cell a particle is uniform in
 * z and in r^2, r = sqrt(r_j^2 + u (r_{j+1}^2 - r_j^2)); its weight is
 * n0 pi (r_{j+1}^2 - r_j^2) dz / (particles in its cell); its velocity is
 * Maxwellian at T (three Box-Muller normals); its acceleration is zero.
 * Draws: stream 3 -> (u_z, u_r, normal pair), stream 4 -> one more pair,
 * at step 0xFFFFFFFF.
 */
void orc_load_range(const orc_state *st, int s, int64_t p0, int64_t p1, double *r, double *z,
                    double *vr, double *vt, double *vz, double *ar, double *az, double *w,
                    uint64_t *id) {
    int nzc = st->c.nz - 1;
    int64_t ncell = (int64_t)nzc * (st->c.nr - 1);
    int64_t N = st->c.n_init[s];
    int64_t base = N / ncell, rem = N % ncell;
    double sig = sqrt(st->c.T_eV[s] * ORC_E / st->c.m[s]);
    for (int64_t p = p0; p < p1; ++p) {
        int64_t c, ppc;
        if (p < rem * (base + 1)) {
            c = p / (base + 1);
        } else {
            c = rem + (p - rem * (base + 1)) / base;
        }
        ppc = base + (c < rem ? 1 : 0);
        int i = (int)(c % nzc), j = (int)(c / nzc);
        uint32_t x[4], y[4];
        orc_draw(st, s, (uint64_t)p, 0xFFFFFFFFu, 3, x);
        orc_draw(st, s, (uint64_t)p, 0xFFFFFFFFu, 4, y);
        double r0 = rj(st, j), r1 = rj(st, j + 1);
        double zz = zi(st, i) + orc_u(x[0]) * st->dz;
        double rr = sqrt(r0 * r0 + orc_u(x[1]) * (r1 * r1 - r0 * r0));
        double n0, n1, n2, n3;
        orc_normals(x[2], x[3], &n0, &n1);
        orc_normals(y[0], y[1], &n2, &n3);
        int64_t k = p - p0;
        r[k] = rr;
        z[k] = zz;
        vr[k] = sig * n0;
        vt[k] = sig * n1;
        vz[k] = sig * n2;
        ar[k] = 0.0;
        az[k] = 0.0;
        w[k] = st->c.n0[s] * ORC_PI * (r1 * r1 - r0 * r0) * st->dz / (double)ppc;
        id[k] = (uint64_t)p;
    }
}

void orc_load(orc_state *st) {
    for (int s = 0; s < 2; ++s) {
        orc_store *p = &st->p[s];
        int64_t n = st->c.n_init[s];
        if (n > st->cap) n = st->cap;
        orc_load_range(st, s, 0, n, p->r, p->z, p->vr, p->vt, p->vz, p->ar, p->az, p->w, p->id);
        p->n = n;
        st->next_id[s] = (uint64_t)n;
    }
    st->step = 0;
    orc_deposit(st);
}

/* ------------------------------------------------------------------ */
/* weighting (Sec. 2.4) and implicit susceptibility (Sec. 2.1)          */
/* ------------------------------------------------------------------ */

/* N_s[i][j] = sum_p w_p S (Eq. (8) or (9)) over the stored positions */
void orc_deposit(orc_state *st) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    for (int s = 0; s < 2; ++s) {
        memset(st->N[s], 0, ng * sizeof(double));
        orc_store *p = &st->p[s];
        for (int64_t k = 0; k < p->n; ++k) {
            int i = cell_z(st, p->z[k]), j = cell_r(st, p->r[k]);
            double Sz[2], Sr[2];
            shape(st, p->r[k], p->z[k], i, j, Sz, Sr);
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) st->N[s][IDX(i + a, j + b)] += p->w[k] * Sz[a] * Sr[b];
        }
    }
}

/*
 * rho = sum_s q_s N_s / V (Eq. (10)); chi = sum_s (q_s / m_s) rho_s dt^2 / 2
 * (Sec. 2.1) -- in SI units chi = dt^2/(2 eps0) sum_s q_s^2 N_s / (m_s V).
 * With ion subcycling the ions' term takes dt_i and counts only before a
 * pass that moves them (READING, at subcycle() above).
 */
void orc_finalize(orc_state *st) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    double *V = xmalloc(ng * sizeof(double));
    orc_node_volumes(st, V);
    const int moves_ions = orc_ion_pass(st);
    for (int64_t k = 0; k < ng; ++k) {
        double rho = 0.0, chi = 0.0;
        for (int s = 0; s < 2; ++s) {
            double rho_s = st->c.q[s] * st->N[s][k] / V[k];
            rho += rho_s;
            if (s == 1 && !moves_ions) continue;
            double dts = dt_of(st, s);
            chi += 0.5 * (st->c.q[s] / st->c.m[s]) * rho_s * dts * dts / ORC_EPS0;
        }
        st->rho[k] = rho;
        st->chi[k] = chi;
    }
    free(V);
}

void orc_get_grid(const orc_state *st, int which, double *out) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    const double *src = NULL;
    switch (which) {
    case 0: src = st->N[0]; break;
    case 1: src = st->N[1]; break;
    case 2: src = st->rho; break;
    case 3: src = st->chi; break;
    case 4: src = st->phi; break;
    case 5: src = st->Ez; break;
    case 6: src = st->Er; break;
    default: return;
    }
    memcpy(out, src, ng * sizeof(double));
}

void orc_set_grid(orc_state *st, int which, const double *in) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    double *dst = NULL;
    switch (which) {
    case 0: dst = st->N[0]; break;
    case 1: dst = st->N[1]; break;
    case 2: dst = st->rho; break;
    case 3: dst = st->chi; break;
    case 4: dst = st->phi; break;
    case 5: dst = st->Ez; break;
    case 6: dst = st->Er; break;
    default: return;
    }
    memcpy(dst, in, ng * sizeof(double));
    /* a potential set from outside has no history: the next extrapolation
     * starts from it unchanged */
    if (which == 4) memcpy(st->phi_prev, in, ng * sizeof(double));
}

/* ------------------------------------------------------------------ */
/* field solver (Sec. 2.5)                                              */
/* ------------------------------------------------------------------ */

/* one multigrid level: nodal chi, unknown u, right-hand side f */
typedef struct {
    int nz;
    double dz;
    double *chi, *u, *f, *r;
} orc_level;

static double face_chi(const orc_state *st, double a, double b) {
    /* Sec. 2.5: chi_{i+1/2} = max(chi_i, chi_{i+1}) or the mean */
    if (st->c.chi_face == ORC_CHI_MEAN) return 0.5 * (a + b);
    return a > b ? a : b;
}

/* z-face area of the control volume of radial node j */
static double area_z(const orc_state *st, int j) {
    double rp = (j + 0.5) * st->dr;
    double rm = j > 0 ? (j - 0.5) * st->dr : 0.0;
    return ORC_PI * (rp * rp - rm * rm);
}

/*
 * Five-point finite-volume coefficients of Eq. (11) (Sec. 2.5) at node
 * (i, j) of a level: -a u_{i-1,j} + b u_ij - c u_{i+1,j} - d u_{i,j-1}
 * - e u_{i,j+1} = f_ij.  READING (typo in Eq. (11): "c_{i+1,j} phi_{i,j}"
 * is c_{ij} phi_{i+1,j}): a, c are the z-face fluxes eps A_j / dz,
 * d, e the r-face fluxes eps 2 pi r_{j -/+ 1/2} dz / dr, d = 0 on the axis
 * (symmetry), b = a + c + d + e.
 */
static void coefs(const orc_state *st, const orc_level *lv, int i, int j, double *a,
                  double *b, double *c, double *d, double *e) {
    int nr = st->c.nr;
    const double *chi = lv->chi;
    double Aj = area_z(st, j);
    *a = (1.0 + face_chi(st, chi[(int64_t)(i - 1) * nr + j], chi[(int64_t)i * nr + j])) * Aj /
         lv->dz;
    *c = (1.0 + face_chi(st, chi[(int64_t)i * nr + j], chi[(int64_t)(i + 1) * nr + j])) * Aj /
         lv->dz;
    *e = (1.0 + face_chi(st, chi[(int64_t)i * nr + j], chi[(int64_t)i * nr + j + 1])) * 2.0 *
         ORC_PI * ((j + 0.5) * st->dr) * lv->dz / st->dr;
    if (j > 0)
        *d = (1.0 + face_chi(st, chi[(int64_t)i * nr + j - 1], chi[(int64_t)i * nr + j])) * 2.0 *
             ORC_PI * ((j - 0.5) * st->dr) * lv->dz / st->dr;
    else
        *d = 0.0;
    *b = *a + *c + *d + *e;
}

/* r = f - A u on interior nodes, 0 on Dirichlet nodes; returns max |r| */
static double residual(const orc_state *st, const orc_level *lv, double *r) {
    int nr = st->c.nr;
    double mx = 0.0;
    memset(r, 0, (size_t)lv->nz * nr * sizeof(double));
    for (int i = 1; i < lv->nz - 1; ++i)
        for (int j = 0; j < nr - 1; ++j) {
            double a, b, c, d, e;
            coefs(st, lv, i, j, &a, &b, &c, &d, &e);
            const double *u = lv->u;
            double Au = b * u[(int64_t)i * nr + j] - a * u[(int64_t)(i - 1) * nr + j] -
                        c * u[(int64_t)(i + 1) * nr + j] - e * u[(int64_t)i * nr + j + 1];
            if (j > 0) Au -= d * u[(int64_t)i * nr + j - 1];
            double v = lv->f[(int64_t)i * nr + j] - Au;
            r[(int64_t)i * nr + j] = v;
            if (fabs(v) > mx) mx = fabs(v);
        }
    return mx;
}

/*
 * Line relaxation of z-row i (Sec. 2.5, Eq. (12)): the r-line is solved
 * exactly with the neighbouring rows held at their current values:
 * -d u_{i,j-1} + b u_ij - e u_{i,j+1} = f_ij + a u_{i-1,j} + c u_{i+1,j}
 * for j = 0 .. nr-2, u_{i,nr-1} Dirichlet.  READING (typo in Eq. (12):
 * the last right-hand side reads f_{i,j}; it is f_{i,j+1}).  Thomas
 * algorithm.
 */
static void line_solve(const orc_state *st, orc_level *lv, int i) {
    int nr = st->c.nr, n = nr - 1;
    double *cp = xmalloc(n * sizeof(double)), *dp = xmalloc(n * sizeof(double));
    double *u = lv->u;
    for (int j = 0; j < n; ++j) {
        double a, b, c, d, e;
        coefs(st, lv, i, j, &a, &b, &c, &d, &e);
        double rhs = lv->f[(int64_t)i * nr + j] + a * u[(int64_t)(i - 1) * nr + j] +
                     c * u[(int64_t)(i + 1) * nr + j];
        if (j == n - 1) rhs += e * u[(int64_t)i * nr + nr - 1];
        double lower = -d, diag = b, upper = (j < n - 1) ? -e : 0.0;
        if (j == 0) {
            cp[j] = upper / diag;
            dp[j] = rhs / diag;
        } else {
            double den = diag - lower * cp[j - 1];
            cp[j] = upper / den;
            dp[j] = (rhs - lower * dp[j - 1]) / den;
        }
    }
    u[(int64_t)i * nr + n - 1] = dp[n - 1];
    for (int j = n - 2; j >= 0; --j) u[(int64_t)i * nr + j] = dp[j] - cp[j] * u[(int64_t)i * nr + j + 1];
    free(cp);
    free(dp);
}

/* zebra sweep: odd (red) rows first, then even (black) rows */
static void line_smooth(const orc_state *st, orc_level *lv) {
    for (int i = 1; i < lv->nz - 1; i += 2) line_solve(st, lv, i);
    for (int i = 2; i < lv->nz - 1; i += 2) line_solve(st, lv, i);
}

static void apply_bc(orc_state *st, double V) {
    int nz = st->c.nz, nr = st->c.nr;
    /* READING: z=0 powered at V(t) (corner with r=R grounded), z=L at
     * phi_zL or 0, r=R grounded (Sec. 3 benchmark geometry). */
    for (int j = 0; j < nr; ++j) {
        st->phi[IDX(0, j)] = (j == nr - 1) ? 0.0 : V;
        st->phi[IDX(nz - 1, j)] = st->c.phi_zL ? st->c.phi_zL[j] : 0.0;
    }
    for (int i = 1; i < nz - 1; ++i) st->phi[IDX(i, nr - 1)] = 0.0;
}

void orc_apply_A(const orc_state *st, const double *chi, const double *u, double *Au) {
    orc_level lv;
    int nz = st->c.nz, nr = st->c.nr;
    lv.nz = nz;
    lv.dz = st->dz;
    lv.chi = (double *)chi;
    lv.u = (double *)u;
    lv.f = xmalloc((size_t)nz * nr * sizeof(double));
    residual(st, &lv, Au); /* Au <- 0 - A u on interior */
    for (int64_t k = 0; k < (int64_t)nz * nr; ++k) Au[k] = -Au[k];
    free(lv.f);
}

/* f = rho * (control volume) / eps0, the FV form of -rho/eps0 (Sec. 2.5) */
void orc_rhs(const orc_state *st, const double *rho, double *f) {
    int nz = st->c.nz, nr = st->c.nr;
    for (int i = 0; i < nz; ++i)
        for (int j = 0; j < nr; ++j) f[IDX(i, j)] = rho[IDX(i, j)] * area_z(st, j) * st->dz / ORC_EPS0;
}

double orc_voltage(const orc_state *st, double t) {
    double v = 0.0;
    for (int k = 0; k < st->c.rf_n; ++k)
        v += st->c.rf_amp[k] * sin(2.0 * ORC_PI * st->c.rf_freq[k] * t + st->c.rf_phase[k]);
    return v;
}

/*
 * Multigrid solve (Sec. 2.5, Algorithm 1): z-only semi-coarsening,
 * V(0,1) cycles.  READING of the garbled algorithm:
 *  - the fine residual is restricted down; coarse levels start from zero
 *    with no pre-smoothing, so their right-hand sides are restrictions of
 *    the one above;
 *  - the coarsest level (nz = 3, one interior row) is solved exactly;
 *  - on the way up "u^l = u^l + I(u^l)" is read as u^l += P u^{l-1},
 *    followed by one zebra line sweep;
 *  - restriction is the [1/4 1/2 1/4] full weighting of Eq. (13) in z on
 *    the density form, i.e. [1/2 1 1/2] on the volume-integrated
 *    residuals used here; prolongation is linear interpolation in z;
 *  - the coarse operator "A^{l-1} = I A^l" is rediscretised from the
 *    z-full-weighted nodal chi with dz doubled.
 * Stops when max|f - A u| <= tol * max|b|, b the right-hand side with the
 * boundary values moved over; tol <= 0 runs exactly max_cycles cycles.
 * Warm start from the stored phi.  Returns 0 converged, 1 not.
 */
int orc_solve(orc_state *st, double V, double tol, int max_cycles, int *cycles,
              double *rel_res) {
    int nz = st->c.nz, nr = st->c.nr;
    int nlev = 0;
    int nzl[32];
    for (int n = nz; n >= 3; n = (n + 1) / 2) {
        nzl[nlev++] = n;
        if (n == 3) break;
    }
    if (nlev == 0) return 2;
    orc_level lv[32];
    for (int l = 0; l < nlev; ++l) {
        lv[l].nz = nzl[l];
        lv[l].dz = st->c.L / (nzl[l] - 1);
        size_t sz = (size_t)nzl[l] * nr * sizeof(double);
        lv[l].chi = xmalloc(sz);
        lv[l].u = l > 0 ? xmalloc(sz) : NULL;
        lv[l].f = xmalloc(sz);
        lv[l].r = xmalloc(sz);
    }
    memcpy(lv[0].chi, st->chi, (size_t)nz * nr * sizeof(double));
    for (int l = 1; l < nlev; ++l) {
        int nc = nzl[l];
        for (int I = 0; I < nc; ++I)
            for (int j = 0; j < nr; ++j) {
                double v;
                if (I == 0 || I == nc - 1)
                    v = lv[l - 1].chi[(int64_t)(2 * I) * nr + j];
                else
                    v = 0.25 * lv[l - 1].chi[(int64_t)(2 * I - 1) * nr + j] +
                        0.5 * lv[l - 1].chi[(int64_t)(2 * I) * nr + j] +
                        0.25 * lv[l - 1].chi[(int64_t)(2 * I + 1) * nr + j];
                lv[l].chi[(int64_t)I * nr + j] = v;
            }
    }
    apply_bc(st, V);
    orc_rhs(st, st->rho, lv[0].f);
    for (int i = 0; i < nz; ++i)
        for (int j = 0; j < nr; ++j)
            if (i == 0 || i == nz - 1 || j == nr - 1) lv[0].f[IDX(i, j)] = 0.0;

    /* |b|: residual of the boundary values with a zero interior */
    double bnorm;
    {
        double *ub = xmalloc((size_t)nz * nr * sizeof(double));
        for (int i = 0; i < nz; ++i)
            for (int j = 0; j < nr; ++j)
                ub[IDX(i, j)] = (i == 0 || i == nz - 1 || j == nr - 1) ? st->phi[IDX(i, j)] : 0.0;
        lv[0].u = ub;
        bnorm = residual(st, &lv[0], lv[0].r);
        free(ub);
    }
    lv[0].u = st->phi;

    int cyc = 0, status = 1;
    double rn = 0.0;
    if (bnorm == 0.0) {
        for (int i = 1; i < nz - 1; ++i)
            for (int j = 0; j < nr - 1; ++j) st->phi[IDX(i, j)] = 0.0;
        status = 0;
        rn = 0.0;
        bnorm = 1.0;
    } else {
        for (;;) {
            rn = residual(st, &lv[0], lv[0].r);
            if (tol > 0.0 && rn <= tol * bnorm) {
                status = 0;
                break;
            }
            if (cyc >= max_cycles) {
                status = tol > 0.0 ? 1 : 0;
                break;
            }
            /* restrict the residual down the levels */
            for (int l = 1; l < nlev; ++l) {
                const double *src = (l == 1) ? lv[0].r : lv[l - 1].f;
                int nc = nzl[l];
                memset(lv[l].f, 0, (size_t)nc * nr * sizeof(double));
                memset(lv[l].u, 0, (size_t)nc * nr * sizeof(double));
                for (int I = 1; I < nc - 1; ++I)
                    for (int j = 0; j < nr - 1; ++j)
                        lv[l].f[(int64_t)I * nr + j] = 0.5 * src[(int64_t)(2 * I - 1) * nr + j] +
                                                        src[(int64_t)(2 * I) * nr + j] +
                                                        0.5 * src[(int64_t)(2 * I + 1) * nr + j];
            }
            /* coarsest: one interior row, solved exactly */
            line_solve(st, &lv[nlev - 1], 1);
            /* prolong and correct, then one zebra sweep, going up */
            for (int l = nlev - 2; l >= 0; --l) {
                int nf = nzl[l];
                const double *uc = lv[l + 1].u;
                double *uf = lv[l].u;
                for (int i = 1; i < nf - 1; ++i)
                    for (int j = 0; j < nr - 1; ++j) {
                        double corr;
                        if (i % 2 == 0)
                            corr = uc[(int64_t)(i / 2) * nr + j];
                        else
                            corr = 0.5 * (uc[(int64_t)(i / 2) * nr + j] +
                                          uc[(int64_t)(i / 2 + 1) * nr + j]);
                        uf[(int64_t)i * nr + j] += corr;
                    }
                line_smooth(st, &lv[l]);
            }
            ++cyc;
        }
    }
    if (cycles) *cycles = cyc;
    if (rel_res) *rel_res = rn / bnorm;
    for (int l = 0; l < nlev; ++l) {
        free(lv[l].chi);
        if (l > 0) free(lv[l].u);
        free(lv[l].f);
        free(lv[l].r);
    }
    return status;
}

/*
 * E = -grad phi at the nodes.  READING (the paper does not say): central
 * differences inside, one-sided first-order differences on the boundary
 * rows and the r = R column, E_r = 0 on the axis (symmetry).
 */
void orc_efield(orc_state *st) {
    int nz = st->c.nz, nr = st->c.nr;
    const double *p = st->phi;
    for (int i = 0; i < nz; ++i)
        for (int j = 0; j < nr; ++j) {
            double ez, er;
            if (i == 0)
                ez = -(p[IDX(1, j)] - p[IDX(0, j)]) / st->dz;
            else if (i == nz - 1)
                ez = -(p[IDX(nz - 1, j)] - p[IDX(nz - 2, j)]) / st->dz;
            else
                ez = -(p[IDX(i + 1, j)] - p[IDX(i - 1, j)]) / (2.0 * st->dz);
            if (j == 0)
                er = 0.0;
            else if (j == nr - 1)
                er = -(p[IDX(i, nr - 1)] - p[IDX(i, nr - 2)]) / st->dr;
            else
                er = -(p[IDX(i, j + 1)] - p[IDX(i, j - 1)]) / (2.0 * st->dr);
            st->Ez[IDX(i, j)] = ez;
            st->Er[IDX(i, j)] = er;
        }
}

/* ------------------------------------------------------------------ */
/* particle pass (Sec. 2.1, 2.2, 2.3, 2.6)                              */
/* ------------------------------------------------------------------ */
typedef struct {
    double r, z, vr, vt, vz, ar, az, w;
    double at; /* a_theta (X-Y-Z pusher) */
} orc_p;

static void push_birth(orc_state *st, int ts, int ps, uint64_t pid, int k, const orc_p *q) {
    if (st->nb == st->bcap) {
        st->bcap *= 2;
        st->b = realloc(st->b, st->bcap * sizeof(orc_birth));
    }
    orc_birth *b = &st->b[st->nb++];
    b->ts = ts;
    b->ps = ps;
    b->pid = pid;
    b->k = k;
    b->r = q->r;
    b->z = q->z;
    b->vr = q->vr;
    b->vt = q->vt;
    b->vz = q->vz;
    b->ar = q->ar;
    b->az = q->az;
    b->w = q->w;
    b->at = q->at;
}

/* wall test on a position (READING: domain 0 < z < L, 0 <= r < R; the
 * z walls are tested first).  Returns -1 inside, else the wall index. */
static int wall_of(const orc_state *st, double r, double z) {
    if (z <= 0.0) return 0;
    if (z >= st->c.L) return 1;
    if (r >= st->c.R) return 2;
    return -1;
}

/*
 * First push in the local X-Y frame and rotation back to r-theta
 * (Sec. 2.3, Eqs. (4)-(5)).  Local pusher, READING: a_theta = 0 (the record
 * has no a_theta and its accumulation is ignored, Sec. 2.3), so
 * v_y' = v_theta and the rotated a_theta' is dropped.  X-Y-Z pusher (Sec.
 * 2.3, end), READING: the Cartesian push of a particle taken at azimuth 0
 * (the field is axisymmetric, so the azimuth itself never matters):
 * v_y' = v_theta + a_theta dt / 2, and both (v_x, v_y) and (a_r, a_theta)
 * rotate onto the new local frame.  At r' = 0, cos = 1 and sin = 0.
 */
static void first_push(const orc_state *st, orc_p *q, double dt) {
    const int xyz = st->c.pusher == 1;
    double vx = q->vr + 0.5 * q->ar * dt;
    double vy = xyz ? q->vt + 0.5 * q->at * dt : q->vt;
    double vz = q->vz + 0.5 * q->az * dt;
    double x = q->r + vx * dt;
    double y = vy * dt;
    double z = q->z + vz * dt;
    double r = sqrt(x * x + y * y);
    double c = 1.0, s = 0.0;
    if (r > 0.0) {
        c = x / r;
        s = y / r;
    }
    q->r = r;
    q->z = z;
    q->vr = vx * c + vy * s;
    q->vt = -vx * s + vy * c;
    q->vz = vz;
    if (xyz) {
        double ar = q->ar * c + q->at * s;
        q->at = -q->ar * s + q->at * c;
        q->ar = ar;
    } else {
        q->ar = q->ar * c;
    }
    /* a_z unchanged */
}

static void absorb(orc_state *st, int s, int wall, double w) {
    st->cnt[ORC_C_ABS + s * 3 + wall] += 1;
    st->qabs[wall] += st->c.q[s] * w;
    st->qpass[wall] += st->c.q[s] * w;
}

/* newborn: first push, wall test, record */
static void newborn(orc_state *st, int ts, int ps, uint64_t pid, int k, orc_p q) {
    st->cnt[ORC_C_BIRTHS + ts] += 1;
    first_push(st, &q, dt_of(st, ts));
    int wall = wall_of(st, q.r, q.z);
    if (wall >= 0) {
        absorb(st, ts, wall, q.w);
        return;
    }
    push_birth(st, ts, ps, pid, k, &q);
}

static int birth_cmp(const void *pa, const void *pb) {
    const orc_birth *a = pa, *b = pb;
    if (a->ts != b->ts) return a->ts < b->ts ? -1 : 1;
    if (a->ps != b->ps) return a->ps < b->ps ? -1 : 1;
    if (a->pid != b->pid) return a->pid < b->pid ? -1 : 1;
    if (a->k != b->k) return a->k < b->k ? -1 : 1;
    return 0;
}

/*
 * Null-collision Monte Carlo for one particle (Sec. 2.6).  READING:
 *  - candidate if u1 < P_null = 1 - exp(-nu_max dt), one real collision
 *    at most per step;
 *  - channel k if u2 nu_max < sum_{k' <= k} nu_k'(E), channel order as in
 *    the table, otherwise null;
 *  - electrons see the gas at rest: g = |v|, E = m g^2 / 2;
 *  - ions see a neutral drawn from the gas Maxwellian: g = |v - v_n|,
 *    E = m_ion g^2 / 2, charge exchange sets v = v_n;
 *  - elastic: Vahedi-Surendra angle, energy loss 2 (m/M)(1 - cos chi);
 *    excitation: E - thr, then scatter; ionisation: E - thr shared by
 *    Opal's form, both electrons scatter, the new ion is a gas atom at
 *    rest frame temperature; newborns copy the parent's weight and take
 *    a = a_parent (q_new m_parent)/(q_parent m_new) (Eq. (15)).
 *  - excitation or ionisation picked below its threshold (possible only by
 *    the table interpolation) is a null event.
 * Draws: stream 0 (u1, u2, R_chi, R_phi); stream 1 (ions: neutral normals;
 * ionisation: R_ej, R_chi2, R_phi2); stream 2 (new ion normals).
 */
static void collide(orc_state *st, int s, uint64_t id, orc_p *q, uint32_t step) {
    uint32_t x[4];
    orc_draw(st, s, id, step, 0, x);
    if (!(orc_u(x[0]) < st->p_null[s])) return;
    st->cnt[ORC_C_CAND + s] += 1;

    double m = st->c.m[s];
    double vnx = 0.0, vny = 0.0, vnz = 0.0;
    double gx = q->vr, gy = q->vt, gz = q->vz;
    if (s == 1) {
        uint32_t y[4];
        orc_draw(st, s, id, step, 1, y);
        double n0, n1, n2, n3;
        orc_normals(y[0], y[1], &n0, &n1);
        orc_normals(y[2], y[3], &n2, &n3);
        double sg = sqrt(ORC_KB * st->c.T_K / st->c.m_gas);
        vnx = sg * n0;
        vny = sg * n1;
        vnz = sg * n2;
        gx = q->vr - vnx;
        gy = q->vt - vny;
        gz = q->vz - vnz;
    }
    double g = sqrt(gx * gx + gy * gy + gz * gz);
    double E = 0.5 * m * g * g / ORC_E;

    int nch = st->c.xs_nch[s];
    double nu[ORC_MAX_CH], tot = 0.0;
    for (int ch = 0; ch < nch; ++ch) {
        nu[ch] = st->ng * orc_sigma(st, s, ch, E) * g;
        tot += nu[ch];
    }
    if (tot > st->nu_max[s]) st->cnt[ORC_C_NUOVER + s] += 1;
    double sel = orc_u(x[1]) * st->nu_max[s];
    double cum = 0.0;
    int ch = -1;
    for (int k = 0; k < nch; ++k) {
        cum += nu[k];
        if (sel < cum) {
            ch = k;
            break;
        }
    }
    if (ch < 0) return;
    int kind = st->c.xs_kind[s][ch];
    double thr = st->c.xs_thr[s][ch];
    if ((kind == ORC_EXCITE || kind == ORC_IONIZE) && E <= thr) return;
    st->cnt[ORC_C_COLL + s * 4 + ch] += 1;

    if (kind == ORC_CX) {
        q->vr = vnx;
        q->vt = vny;
        q->vz = vnz;
        return;
    }
    /* electron channels: incident direction of the electron */
    double ux = gx / g, uy = gy / g, uz = gz / g;
    double d1[3];
    if (kind == ORC_ELASTIC) {
        double cc = orc_cos_chi(st, E, orc_u(x[2]));
        orc_scatter_dir(ux, uy, uz, cc, 2.0 * ORC_PI * orc_u(x[3]), d1);
        double gn = g * sqrt(1.0 - 2.0 * m / st->c.m_gas * (1.0 - cc));
        q->vr = gn * d1[0];
        q->vt = gn * d1[1];
        q->vz = gn * d1[2];
    } else if (kind == ORC_EXCITE) {
        double Ep = E - thr;
        double cc = orc_cos_chi(st, Ep, orc_u(x[2]));
        orc_scatter_dir(ux, uy, uz, cc, 2.0 * ORC_PI * orc_u(x[3]), d1);
        double gn = sqrt(2.0 * Ep * ORC_E / m);
        q->vr = gn * d1[0];
        q->vt = gn * d1[1];
        q->vz = gn * d1[2];
    } else if (kind == ORC_IONIZE) {
        uint32_t y[4], zz[4];
        orc_draw(st, s, id, step, 1, y);
        orc_draw(st, s, id, step, 2, zz);
        double Eej = orc_ejected_energy(E, thr, st->c.xs_B[s], orc_u(y[0]));
        double Esc = E - thr - Eej;
        if (Esc < 0.0) Esc = 0.0;
        double c1 = orc_cos_chi(st, Esc, orc_u(x[2]));
        orc_scatter_dir(ux, uy, uz, c1, 2.0 * ORC_PI * orc_u(x[3]), d1);
        double c2 = orc_cos_chi(st, Eej, orc_u(y[1]));
        double d2[3];
        orc_scatter_dir(ux, uy, uz, c2, 2.0 * ORC_PI * orc_u(y[2]), d2);
        double g1 = sqrt(2.0 * Esc * ORC_E / m), g2 = sqrt(2.0 * Eej * ORC_E / m);
        orc_p e2 = *q;
        q->vr = g1 * d1[0];
        q->vt = g1 * d1[1];
        q->vz = g1 * d1[2];
        e2.vr = g2 * d2[0];
        e2.vt = g2 * d2[1];
        e2.vz = g2 * d2[2];
        /* new ion: gas atom velocity, weight of the incident particle */
        double n0, n1, n2, n3;
        orc_normals(zz[0], zz[1], &n0, &n1);
        orc_normals(zz[2], zz[3], &n2, &n3);
        double sg = sqrt(ORC_KB * st->c.T_K / st->c.m_gas);
        orc_p ion = *q;
        ion.vr = sg * n0;
        ion.vt = sg * n1;
        ion.vz = sg * n2;
        double fac = (st->c.q[1] * st->c.m[0]) / (st->c.q[0] * st->c.m[1]);
        ion.ar = q->ar * fac;
        ion.az = q->az * fac;
        ion.at = q->at * fac;
        newborn(st, 0, s, id, 0, e2);
        newborn(st, 1, s, id, 1, ion);
    }
}

/*
 * Weight-conserving split (Sec. 2.2): if w_p > w_r, N = [w_p / w_r] new
 * particles of weight w_r at the parent's phase point, the parent keeps
 * w_p - N w_r.  READING: w_r is the reference weight of the particle's
 * radial cell; when the remainder is not positive the parent keeps one
 * share (N - 1 copies); at most ORC_SPLIT_NMAX copies per parent per split.
 */
static void split(orc_state *st, int s, uint64_t id, orc_p *q) {
    int j = cell_r(st, q->r);
    double wr = orc_w_ref(st, s, j);
    if (!(q->w > wr)) return;
    double Nf = floor(q->w / wr);
    if (Nf > ORC_SPLIT_NMAX) Nf = ORC_SPLIT_NMAX;
    int N = (int)Nf;
    double rem = q->w - Nf * wr;
    if (!(rem > 0.0)) {
        N -= 1;
        rem = q->w - (double)N * wr;
    }
    if (N <= 0) return;
    st->cnt[ORC_C_SPLITS + s] += 1;
    orc_p copy = *q;
    copy.w = wr;
    q->w = rem;
    for (int k = 0; k < N; ++k) newborn(st, s, s, id, 2 + k, copy);
}

/*
 * Particle merging (Sec. 2.2 names the need to combine small particles
 * and points to a reference; it gives no algorithm).  READING: particles of
 * species s lighter than frac * w_r (w_r of their radial cell, as for the
 * split) are grouped by cell of x~ and by velocity bin, the bin of each
 * component being floor(v / dv) (clamped to +-2^20); inside a group they are
 * taken in order of id and merged in pairs, the odd last one left alone.
 * The pair (a, b), id a < id b, becomes one particle with id a and
 *   w = w_a + w_b,  z = <z>,  r^2 = <r^2>,  v_r = <v_r>,  v_z = <v_z>,
 *   a_r = <a_r>,  a_z = <a_z>,  v_theta = <r v_theta> / r  (and a_theta
 *   likewise), <x> = (w_a x_a + w_b x_b) / w,
 * which keeps the charge, the z and r^2 moments (so the cell, and the z-r^2
 * deposit's totals and first moments), the radial and axial momentum, the
 * angular momentum and the implicit current sum w a.  The kinetic energy
 * the velocity spread held, (m/2) w_a w_b / w |v_a - v_b|^2 in the local
 * components, is lost; *energy_J returns it.  The deposit of the stored
 * state is redone (the next solve takes it).  Returns the pairs merged.
 */
typedef struct {
    int64_t k;      /* index in the store */
    int64_t cell;   /* j (nz-1) + i       */
    uint64_t key;   /* velocity bin       */
    uint64_t id;
} orc_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const orc_cand *a = pa, *b = pb;
    if (a->cell != b->cell) return a->cell < b->cell ? -1 : 1;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1;
    return 0;
}

static uint64_t vbin(double v, double dv) {
    double b = floor(v / dv);
    if (b < -1048576.0) b = -1048576.0;
    if (b > 1048575.0) b = 1048575.0;
    return (uint64_t)((int64_t)b + 1048576);
}

int64_t orc_merge(orc_state *st, int s, double frac, double dv, double *energy_J) {
    orc_store *P = &st->p[s];
    orc_cand *c = xmalloc((P->n > 0 ? P->n : 1) * sizeof(orc_cand));
    int64_t nc = 0;
    for (int64_t k = 0; k < P->n; ++k) {
        int i = cell_z(st, P->z[k]), j = cell_r(st, P->r[k]);
        if (!(P->w[k] < frac * orc_w_ref(st, s, j))) continue;
        c[nc].k = k;
        c[nc].cell = (int64_t)j * (st->c.nz - 1) + i;
        c[nc].key = (vbin(P->vr[k], dv) << 42) | (vbin(P->vt[k], dv) << 21) | vbin(P->vz[k], dv);
        c[nc].id = P->id[k];
        ++nc;
    }
    qsort(c, nc, sizeof(orc_cand), cand_cmp);
    char *gone = calloc(P->n > 0 ? P->n : 1, 1);
    int64_t pairs = 0;
    double lost = 0.0;
    for (int64_t q = 0; q < nc;) {
        int64_t e = q + 1;
        while (e < nc && c[e].cell == c[q].cell && c[e].key == c[q].key) ++e;
        for (int64_t u = q; u + 1 < e; u += 2) {
            int64_t a = c[u].k, b = c[u + 1].k;
            double wa = P->w[a], wb = P->w[b], W = wa + wb;
            double ra = P->r[a], rb = P->r[b];
            double r = sqrt((wa * ra * ra + wb * rb * rb) / W);
            double vr = (wa * P->vr[a] + wb * P->vr[b]) / W;
            double vz = (wa * P->vz[a] + wb * P->vz[b]) / W;
            double Lt = wa * ra * P->vt[a] + wb * rb * P->vt[b];
            double Lat = wa * ra * P->at[a] + wb * rb * P->at[b];
            double vt = r > 0.0 ? Lt / (W * r) : (wa * P->vt[a] + wb * P->vt[b]) / W;
            double at = r > 0.0 ? Lat / (W * r) : (wa * P->at[a] + wb * P->at[b]) / W;
            double e0 = wa * (P->vr[a] * P->vr[a] + P->vt[a] * P->vt[a] + P->vz[a] * P->vz[a]) +
                        wb * (P->vr[b] * P->vr[b] + P->vt[b] * P->vt[b] + P->vz[b] * P->vz[b]);
            lost += 0.5 * st->c.m[s] * (e0 - W * (vr * vr + vt * vt + vz * vz));
            P->z[a] = (wa * P->z[a] + wb * P->z[b]) / W;
            P->r[a] = r;
            P->vr[a] = vr;
            P->vt[a] = vt;
            P->vz[a] = vz;
            P->ar[a] = (wa * P->ar[a] + wb * P->ar[b]) / W;
            P->az[a] = (wa * P->az[a] + wb * P->az[b]) / W;
            P->at[a] = at;
            P->w[a] = W;
            gone[b] = 1;
            ++pairs;
        }
        q = e;
    }
    int64_t out = 0;
    for (int64_t k = 0; k < P->n; ++k) {
        if (gone[k]) continue;
        P->r[out] = P->r[k];
        P->z[out] = P->z[k];
        P->vr[out] = P->vr[k];
        P->vt[out] = P->vt[k];
        P->vz[out] = P->vz[k];
        P->ar[out] = P->ar[k];
        P->az[out] = P->az[k];
        P->at[out] = P->at[k];
        P->w[out] = P->w[k];
        P->id[out] = P->id[k];
        ++out;
    }
    P->n = out;
    free(gone);
    free(c);
    if (energy_J) *energy_J = lost;
    /* the stored state's deposit follows the merged positions */
    orc_deposit(st);
    return pairs;
}

static int eedf_bin(const orc_state *st, double E) {
    if (st->c.eedf_bins <= 0 || !(E >= 0.0)) return -1;
    double x = E / st->c.eedf_emax * st->c.eedf_bins;
    if (x >= st->c.eedf_bins) return -1;
    return (int)x;
}

/*
 * One merged particle pass (Sec. 2.1: the final push of step n and the
 * first push of step n+1 are one pass; MC acts on x^{n+1}, Sec. 2.1 end).
 * Per particle: gather E at x~ -> final push (Sec. 2.1 finalpush, Sec. 2.3
 * final push in r-z) -> axis (|r|, |v_r|, |a_r|) -> walls -> MC -> split ->
 * first push -> walls.  Newborns get their first push at birth.  Births
 * are ordered by (species, parent species, parent id, slot) and numbered
 * from next_id; they are appended after the survivors.
 */
void orc_particle_pass(orc_state *st) {
    uint32_t step = (uint32_t)st->step;
    const int moves_ions = orc_ion_pass(st);
    int do_split = st->c.split_every > 0 && (st->step % st->c.split_every) == st->c.split_every - 1;
    st->nb = 0;
    memset(st->qpass, 0, sizeof(st->qpass));
    if (st->c.eedf_bins > 0) memset(st->eedf_pass, 0, st->c.eedf_bins * sizeof(double));
    for (int s = 0; s < 2; ++s) {
        if (s == 1 && !moves_ions) continue; /* held still (subcycling) */
        orc_store *P = &st->p[s];
        double qm = st->c.q[s] / st->c.m[s];
        double dt = dt_of(st, s);
        int64_t out = 0;
        for (int64_t k = 0; k < P->n; ++k) {
            orc_p q = {P->r[k], P->z[k], P->vr[k], P->vt[k], P->vz[k], P->ar[k], P->az[k], P->w[k], P->at[k]};
            uint64_t id = P->id[k];
            /* gather E at x~ (Sec. 2.4, same weights as the deposit) */
            int i = cell_z(st, q.z), j = cell_r(st, q.r);
            double Sz[2], Sr[2];
            shape(st, q.r, q.z, i, j, Sz, Sr);
            double Ez = 0.0, Er = 0.0;
            for (int a = 0; a < 2; ++a)
                for (int b = 0; b < 2; ++b) {
                    Ez += Sz[a] * Sr[b] * st->Ez[IDX(i + a, j + b)];
                    Er += Sz[a] * Sr[b] * st->Er[IDX(i + a, j + b)];
                }
            /* final push in r-z */
            q.z = q.z + 0.5 * qm * Ez * dt * dt;
            q.r = q.r + 0.5 * qm * Er * dt * dt;
            q.vz = q.vz + 0.5 * qm * Ez * dt;
            q.vr = q.vr + 0.5 * qm * Er * dt;
            q.az = 0.5 * (qm * Ez + q.az);
            q.ar = 0.5 * (qm * Er + q.ar);
            q.at = 0.5 * q.at; /* no E_theta */
            if (q.r < 0.0) {
                q.r = -q.r;
                if (st->c.pusher == 1) {
                    /* X-Y-Z: through the axis to the opposite azimuth, whose
                     * local r and theta directions are the reversed ones */
                    q.vr = -q.vr;
                    q.ar = -q.ar;
                    q.vt = -q.vt;
                    q.at = -q.at;
                } else {
                    /* axis crossing: absolute values in r (Sec. 2.3) */
                    q.vr = fabs(q.vr);
                    q.ar = fabs(q.ar);
                }
            }
            int wall = wall_of(st, q.r, q.z);
            if (wall >= 0) {
                absorb(st, s, wall, q.w);
                continue;
            }
            collide(st, s, id, &q, step);
            if (s == 0 && st->c.eedf_bins > 0) {
                double E = 0.5 * st->c.m[0] * (q.vr * q.vr + q.vt * q.vt + q.vz * q.vz) / ORC_E;
                int bi = eedf_bin(st, E);
                if (bi >= 0) st->eedf_pass[bi] += q.w;
            }
            if (do_split) split(st, s, id, &q);
            first_push(st, &q, dt);
            wall = wall_of(st, q.r, q.z);
            if (wall >= 0) {
                absorb(st, s, wall, q.w);
                continue;
            }
            P->r[out] = q.r;
            P->z[out] = q.z;
            P->vr[out] = q.vr;
            P->vt[out] = q.vt;
            P->vz[out] = q.vz;
            P->ar[out] = q.ar;
            P->az[out] = q.az;
            P->at[out] = q.at;
            P->w[out] = q.w;
            P->id[out] = id;
            ++out;
        }
        P->n = out;
    }
    /* canonical numbering of the births */
    qsort(st->b, st->nb, sizeof(orc_birth), birth_cmp);
    for (int64_t k = 0; k < st->nb; ++k) {
        orc_birth *b = &st->b[k];
        orc_store *P = &st->p[b->ts];
        if (P->n >= st->cap) continue;
        int64_t o = P->n++;
        P->r[o] = b->r;
        P->z[o] = b->z;
        P->vr[o] = b->vr;
        P->vt[o] = b->vt;
        P->vz[o] = b->vz;
        P->ar[o] = b->ar;
        P->at[o] = b->at;
        P->az[o] = b->az;
        P->w[o] = b->w;
        P->id[o] = st->next_id[b->ts]++;
    }
    st->step += 1;
}

/*
 * Charge on the z = 0 electrode (nodes j < nr-1; the corner belongs to the
 * grounded wall).  READING (the paper gives the circuit, not the discrete
 * charge): Gauss's law on the electrode row of the finite-volume mesh, i.e.
 * the displacement flux eps0 c_{0j} (phi_0j - phi_1j) through the z-face
 * into row 1, less the charge rho_0j V_0j of the half cell in front of the
 * electrode.
 */
static double electrode_charge(const orc_state *st, const double *phi, const double *rho,
                               const double *V) {
    int nr = st->c.nr;
    double q = 0.0;
    for (int j = 0; j < nr - 1; ++j) {
        double c0 = (1.0 + face_chi(st, st->chi[IDX(0, j)], st->chi[IDX(1, j)])) * area_z(st, j) / st->dz;
        q += ORC_EPS0 * c0 * (phi[IDX(0, j)] - phi[IDX(1, j)]) - rho[IDX(0, j)] * V[IDX(0, j)];
    }
    return q;
}

/*
 * External circuit (Sec. 2.5, end), Vahedi's superposition: with a blocking
 * capacitor C between the rf source and the z = 0 electrode, phi_P solves
 * the plasma's charge with the electrode at 0 (other boundaries as usual),
 * phi_L the charge-free problem with the electrode at 1 and every other
 * boundary at 0, both with the same coefficient 1 + chi (each warm-started
 * from its last solution).  The electrode charge is linear in its voltage,
 * Q = Q_P + V Q_L, and the circuit equation
 *   Q^t = Q^{t-1} + C (V_rf^t - V^t) - Q_c^{t-1} + Q_conv^t,
 * with Q_c^t = C (V_rf^t - V^t) and Q_conv the charge the electrode
 * collected in the last particle pass, fixes V^t; then
 * phi = phi_P + V^t phi_L.  READING: Q and Q_c start at 0.
 */
static void circuit_solve(orc_state *st, double Vrf, const double *V, int *cycles, double *rel_res) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    double *keep_phi = st->phi, *keep_rho = st->rho;
    const double *keep_zL = st->c.phi_zL;
    int c1 = 0, c2 = 0;
    double r1 = 0.0, r2 = 0.0;
    st->phi = st->phiP;
    orc_solve(st, 0.0, st->c.mg_tol, st->c.mg_max_cycles, &c1, &r1);
    st->phi = st->phiL;
    st->rho = st->zero;
    st->c.phi_zL = NULL;
    orc_solve(st, 1.0, st->c.mg_tol, st->c.mg_max_cycles, &c2, &r2);
    st->phi = keep_phi;
    st->rho = keep_rho;
    st->c.phi_zL = keep_zL;
    double QP = electrode_charge(st, st->phiP, st->rho, V);
    double QL = electrode_charge(st, st->phiL, st->zero, V);
    double C = st->c.circuit_C;
    double Vt = (st->circ_Q - st->circ_Qc + C * Vrf + st->qpass[0] - QP) / (QL + C);
    st->circ_V = Vt;
    st->circ_Q = QP + Vt * QL;
    st->circ_Qc = C * (Vrf - Vt);
    for (int64_t k = 0; k < ng; ++k) st->phi[k] = st->phiP[k] + Vt * st->phiL[k];
    if (cycles) *cycles = c1 + c2;
    if (rel_res) *rel_res = r1 > r2 ? r1 : r2;
}

void orc_get_circuit(const orc_state *st, double out[3]) {
    out[0] = st->circ_V;
    out[1] = st->circ_Q;
    out[2] = st->circ_Qc;
}

/*
 * One timestep (Sec. 2.1 cycle, merged form): rho, chi from the deposit at
 * x~ -> solve at t_{n+1} -> E -> particle pass -> deposit at the new x~ ->
 * time averages (Sec. 3: moments averaged over time).
 */
void orc_step(orc_state *st, int nsteps, int *last_cycles, double *last_res) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    double *V = xmalloc(ng * sizeof(double));
    orc_node_volumes(st, V);
    for (int n = 0; n < nsteps; ++n) {
        orc_finalize(st);
        double t = (double)(st->step + 1) * st->c.dt;
        int cyc = 0;
        double res = 0.0;
        if (st->c.circuit_C > 0.0)
            circuit_solve(st, orc_voltage(st, t), V, &cyc, &res);
        else {
            if (st->c.mg_guess == 1) {
                /* w_0 of Algorithm 1: phi^n + (phi^n - phi^(n-1)) on the
                 * interior nodes, the potential extrapolated linearly in
                 * time (the boundary values are set by the solve) */
                int nz = st->c.nz, nr = st->c.nr;
                for (int i = 1; i < nz - 1; ++i)
                    for (int j = 0; j < nr - 1; ++j) {
                        double now = st->phi[IDX(i, j)];
                        st->phi[IDX(i, j)] = 2.0 * now - st->phi_prev[IDX(i, j)];
                        st->phi_prev[IDX(i, j)] = now;
                    }
            }
            orc_solve(st, orc_voltage(st, t), st->c.mg_tol, st->c.mg_max_cycles, &cyc, &res);
        }
        if (last_cycles) *last_cycles = cyc;
        if (last_res) *last_res = res;
        orc_efield(st);
        orc_particle_pass(st);
        orc_deposit(st);
        for (int64_t k = 0; k < ng; ++k) {
            st->m_ne[k] += st->N[0][k] / V[k];
            st->m_ni[k] += st->N[1][k] / V[k];
            st->m_phi[k] += st->phi[k];
            st->m_ez[k] += st->Ez[k];
            st->m_er[k] += st->Er[k];
        }
        for (int b = 0; b < st->c.eedf_bins; ++b) st->m_eedf[b] += st->eedf_pass[b];
        st->m_n += 1;
    }
    free(V);
}

void orc_get_counters(const orc_state *st, int64_t *c, double *q) {
    if (c) memcpy(c, st->cnt, sizeof(st->cnt));
    if (q) memcpy(q, st->qabs, sizeof(st->qabs));
}

void orc_reset_counters(orc_state *st) {
    memset(st->cnt, 0, sizeof(st->cnt));
    memset(st->qabs, 0, sizeof(st->qabs));
}

void orc_get_moments(const orc_state *st, double *ne, double *ni, double *phi, double *Ez,
                     double *Er, double *eedf, int64_t *nsamples) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    double inv = st->m_n > 0 ? 1.0 / (double)st->m_n : 0.0;
    for (int64_t k = 0; k < ng; ++k) {
        if (ne) ne[k] = st->m_ne[k] * inv;
        if (ni) ni[k] = st->m_ni[k] * inv;
        if (phi) phi[k] = st->m_phi[k] * inv;
        if (Ez) Ez[k] = st->m_ez[k] * inv;
        if (Er) Er[k] = st->m_er[k] * inv;
    }
    if (eedf)
        for (int b = 0; b < st->c.eedf_bins; ++b) eedf[b] = st->m_eedf[b] * inv;
    if (nsamples) *nsamples = st->m_n;
}

void orc_reset_moments(orc_state *st) {
    int64_t ng = (int64_t)st->c.nz * st->c.nr;
    memset(st->m_ne, 0, ng * sizeof(double));
    memset(st->m_ni, 0, ng * sizeof(double));
    memset(st->m_phi, 0, ng * sizeof(double));
    memset(st->m_ez, 0, ng * sizeof(double));
    memset(st->m_er, 0, ng * sizeof(double));
    if (st->c.eedf_bins > 0) memset(st->m_eedf, 0, st->c.eedf_bins * sizeof(double));
    st->m_n = 0;
}
