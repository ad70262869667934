// pic_internal.cuh -- device data layout, kernel argument blocks and launcher
// declarations of the GB300 r-z implicit PIC/MC library (arXiv:1001.2969).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pic.h"

namespace pic {

// CODATA 2018 values
constexpr double kQe = 1.602176634e-19;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kKB = 1.380649e-23;
constexpr double kPi = 3.14159265358979323846;

constexpr int kMaxCh = PIC_MAX_CH;
constexpr int kSplitNMax = 4096;  // copies per parent per split, at most

// status bits raised by kernels
enum : int {
    ST_BIRTH_OVERFLOW = 1,
    ST_CAPACITY = 2,
    ST_NAN = 4,
    ST_TIMEOUT = 8,
};

// Step control on the device.  A timestep runs with no host
// synchronisation: the first failed check sets `halt`, every later kernel of
// the pic_step call returns at once, and the host reads this block once per
// call.  Step-dependent values (step number, electrode voltage, split flag)
// live here too, so a step's launches are the same every time (graph replay).
struct StepCtl {
    int32_t halt;         // a step failed: later step kernels do nothing
    int32_t halt_status;  // ST_* bits of the failure
    int64_t halt_step;    // number of the step that failed
    int64_t step;         // number of the step being taken
    double V;             // electrode voltage at the step's field time
    int32_t do_split;     // the step splits heavy particles
    int32_t mg_flags;     // bit 0: a solve stopped before the tolerance
    uint64_t next_id[2];  // next particle id per species
    unsigned long long mg_cycles;  // V-cycles of all solves so far
    int32_t mg_last_cycles;
    int32_t pad;
    double mg_last_res;   // relative residual of the last solve
    unsigned int bar;     // barrier counter of the births numbering
    int32_t bar_timeout;  // a bounded wait of the births numbering gave up
    double circ_V, circ_Q, circ_Qc;  // external circuit: electrode voltage and charge, capacitor charge
    // The cell sort of a pass (scan, capacity check, rank, births numbering)
    // runs in the next step beside its field solve, or before the particle
    // state is read (the end of a call runs its scans and capacity check
    // only): pending from the end of the pass until it is done.  A failed
    // sort (capacity, births overflow, a wait that gave up) also halts the
    // step.
    int32_t sort_pending;
    int32_t sort_fail;         // the sort failed: later sort kernels do nothing
    int32_t sort_fail_status;  // ST_* bits of the failure
    int32_t pad2;
    int64_t sort_fail_step;    // number of the step whose sort failed
    // newborns of one pass get ids next_id + id_stride * rank (0 means 1): a
    // reactor whose particles are shared among processes numbers each
    // process's newborns in its own residue class
    uint64_t id_stride;
};

// a sort kernel has nothing to do: no pass waits for it, or the sort failed
// (ctl null: a sort outside the timestep, always done)
__device__ __forceinline__ bool sort_skip(const StepCtl *ctl) {
    return ctl && (!ctl->sort_pending || ctl->sort_fail);
}

// a failure of the pending sort: the pass it sorts (the step before the one
// being taken) did not complete, and nothing after it runs
__device__ __forceinline__ void sort_failed(StepCtl *ctl, int status) {
    if (atomicExch(&ctl->sort_fail, 1) == 0) {
        ctl->sort_fail_status = status;
        ctl->sort_fail_step = ctl->step - 1;
    }
    ctl->halt = 1;
}

// ---- grid barrier of cooperative launches ----
// Thread 0 of each block adds 1 with release semantics and polls with
// acquire loads until the counter (which only grows) reaches `target`: the
// participants times the barriers of this kind the block has passed.  The
// block's writes before the barrier are visible to every participant after
// it.  The poll is bounded: after `limit` tries (kSpinLimit: a few seconds
// at most, against microseconds for a wait that ends), or once another block
// gave up, the block raises *timeout and the call returns false.
constexpr long long kSpinLimit = 1LL << 22;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void atom_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool count_barrier(unsigned *count, unsigned target, int *timeout,
                                              long long limit = kSpinLimit) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        atom_add_release(count, 1u);
        long long it = 0;
        while ((int)(ld_acquire(count) - target) < 0) {
            if ((++it & 255) == 0 && (it > limit || *(volatile int *)timeout)) {
                atomicExch(timeout, 1);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// four-wide vectors: float4 for the mixed path, two 16-byte halves for FP64
struct alignas(16) dbl4 {
    double x, y, z, w;
};
template <typename T>
struct V4;
template <>
struct V4<float> {
    using type = float4;
};
template <>
struct V4<double> {
    using type = dbl4;
};
template <typename T>
struct V2;
template <>
struct V2<float> {
    using type = float2;
};
template <>
struct V2<double> {
    using type = double2;
};

// Particle store of one species (structure of 128-bit vectors):
//   q0 = {dz offset in [0,1), dr offset in [0,1), v_r, v_theta}
//   q1 = {v_z, a_r, a_z, w}
//   cell = j (nz-1) + i of the stored position x~, -1 when dead
//   id = 64-bit identity that keys the Philox draws
template <typename T>
struct PBuf {
    typename V4<T>::type *q0;
    typename V4<T>::type *q1;
    int32_t *cell;
    uint64_t *id;
    T *at;  // a_theta (X-Y-Z pusher), null otherwise
};

// device-side scalars of one handle
struct DevScalars {
    int32_t n_alive[2];     // particles the next pass reads through perm
    int32_t n_main[2];      // main entries of the current set
    int32_t n_births[2][2]; // births in births buffer [set][species]
    int32_t status;
    int32_t pad;
    unsigned long long cnt[PIC_NCOUNT];
    double qabs[3];
    double qstep[3];  // absorbed charge per wall since the circuit last took it
    unsigned long long mg_res_bits;  // max |residual| of the last residual kernel
    unsigned long long mg_aux_bits;
    int32_t chunk_next[2];  // the particle pass's next unclaimed chunk, per species
};

template <typename T>
struct V4;
// cross-section block for the particle kernel
template <typename T>
struct Xs {
    const T *sigma;                       // [n_ch][n_e]
    const typename V4<T>::type *sig4;     // [n_e] {sigma_0..sigma_3}, zero-padded
    int n_e, n_ch;
    T emax, inv_dE;
    int kind[kMaxCh];
    T thr[kMaxCh];
    T B;
};

// per-launch arguments of the fused particle kernel (one species)
template <typename T>
struct StepArgs {
    int nz, nr, ncz, ncr;
    float inv_ncz;  // 1/ncz for the cell decode
    int s;          // species of this launch
    double qch[2];  // species charges (absorbed-charge tallies)
    int weighting;  // PIC_WEIGHT_*
    int scatter;    // PIC_SCATTER_*
    int xyz;        // the X-Y-Z pusher (a_theta carried)
    // final push: offsets/velocities/accelerations change per unit E
    T kz, kr, kv, ka;
    // first push
    T dt, dt_dz, dt_dr, dr, inv_dr;
    T bdt[2], bdt_dz[2];  // first push of a newborn of species t (ion subcycling: dt_i)
    // Monte Carlo
    unsigned long long t_null;  // candidate iff word < t_null
    T nu_max, ng, half_m_e;     // half_m_e = m / (2 e): E[eV] = half_m_e g^2
    T two_e_m;                  // 2 e / m: g^2 = two_e_m E[eV]
    T two_m_M;                  // 2 m / M_gas (elastic energy loss)
    T v_gas;                    // sqrt(k T_gas / M_gas)
    T ion_acc;                  // a_ion = a_e * ion_acc (newborn ion)
    Xs<T> xs;
    uint32_t key0, key1;
    const StepCtl *ctl;  // step number (Philox counter), split flag, halt
    // splitting
    const T *w_ref;  // [ncr]
    // fields at the nodes {E_z, E_r}
    const typename V2<T>::type *E;
    // input set, read through perm
    PBuf<T> src_main, src_births;
    const int32_t *n_main_src;
    const int32_t *perm;
    const int32_t *n_alive;
    // output set
    PBuf<T> dst_main;
    PBuf<T> births[2];
    uint64_t *bkey[2];
    int32_t *nb[2];
    int bcap;
    double *N[2];
    int32_t *counts[2];
    DevScalars *ds;
    int32_t *chunk_next;  // zero before the launch; blocks claim chunks from it
    double *eedf;
    int eedf_bins;
    T eedf_scale;  // bins per eV
};


// ---- launchers (particles.cu) ----
// variant: particle-pass shape (bit 0 shared-memory prefetch, bit 1 eight
// particles per thread), -1 the species' default
constexpr int kStepVariants = 4;
template <typename T>
void launch_step(const StepArgs<T> &a, int grid, int variant, cudaStream_t st);
template <typename T>
void launch_load(PBuf<T> dst, int64_t n, int s, int nz, int nr, double dz, double dr,
                 double n0, double T_eV, double m, uint32_t key0, uint32_t key1,
                 int64_t ncell_pop, cudaStream_t st);
// merges the light particles of each cell in pairs (k_merge in particles.cu);
// cursor: each cell's end in the permutation
template <typename T>
void launch_merge(PBuf<T> mainb, PBuf<T> births, const int32_t *nmain_dev, const int32_t *perm,
                  const int32_t *cursor, int ncell, int ncz, double dz, double dr, const T *w_ref, double frac,
                  double dv, double mass, int xyz, unsigned long long *pairs, double *energy, int *overflow,
                  cudaStream_t st);
template <typename T>
void launch_deposit(PBuf<T> src, const int32_t *n_dev, int nz, int nr, int weighting,
                    double *N, cudaStream_t st);
template <typename T>
void launch_from_abs(PBuf<T> dst, int64_t n, const double *r, const double *z, const double *vr,
                     const double *vt, const double *vz, const double *ar, const double *az,
                     const double *w, const uint64_t *id, const double *at, int nz, int nr, double dz,
                     double dr, cudaStream_t st);
template <typename T>
void launch_to_abs(PBuf<T> src_main, PBuf<T> src_births, const int32_t *n_main_src,
                   const int32_t *perm, int64_t n, double *r, double *z, double *vr, double *vt,
                   double *vz, double *ar, double *az, double *w, uint64_t *id, int32_t *cell,
                   double *at, int nz, double dz, double dr, cudaStream_t st);

// ---- launchers (sortk.cu) ----
template <typename T>
void launch_hist(PBuf<T> buf, const int32_t *n_dev, int32_t *counts, cudaStream_t st);
// exclusive scan of counts[ncell] into cursor, total into *n_alive, capacity check
void launch_scan(const int32_t *counts, int32_t *cursor, int ncell, int32_t *block_sums,
                 int32_t *n_alive, int64_t capacity, DevScalars *ds, const StepCtl *ctl,
                 cudaStream_t st);
// a failed check of the pending sort's pass (capacity, births overflow)
void launch_step_check(const DevScalars *ds, StepCtl *ctl, cudaStream_t st);
template <typename T>
void launch_rank(PBuf<T> main, const int32_t *n_main, PBuf<T> births, const int32_t *n_births,
                 int32_t *cursor, int32_t *perm, const int32_t *n_alive, int64_t cap,
                 const int32_t *status, const StepCtl *ctl, int ncell, cudaStream_t st);
// births of species s get ids next_id[s] + rank of their key among the
// *nb births (one cooperative launch; next_id[s] advances by *nb)
struct RadixTmp {
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    uint32_t *hist;
    int *flag;
    int max_n;
};
// the bounded-wait self-test (sortk.cu): 0 when it ran, *gave_up = 1 when
// the wait ran out as it must
int wait_selftest(long long limit, int *gave_up);
// numbers the births key/id[*nb0 .. *nb) (nb0 nullable: from 0), on at
// most max_grid blocks
void launch_birth_ids(const uint64_t *key, uint64_t *id, const int32_t *nb, const int32_t *nb0, StepCtl *ctl,
                      int s, RadixTmp tmp, cudaStream_t st, int max_grid = 1 << 30);

// ---- multigrid (field.cu) ----
struct MGLevel {
    int nz;
    double dz;
    double *chi, *cz, *cr, *u, *f;
    float *cz32, *cr32, *u32, *f32;
};
struct MGWork {
    int nlev;
    MGLevel lv[16];
    double *r;        // fine residual
    double *f0;       // fine right-hand side
    DevScalars *ds;   // residual max goes to ds->mg_res_bits
};
struct FieldDims {
    int nz, nr;
    double dz, dr, L;
    int chi_face;
};
// ctl (may be null): skip when the step has halted
void launch_finalize(const double *Ne, const double *Ni, const double *V, double q0, double q1,
                     double chi0, double chi1, double *rho, double *chi, int ng, const StepCtl *ctl,
                     cudaStream_t st);
// multigrid solve into phi (device); returns cycles, residual and the launch count
int mg_solve(const FieldDims &fd, MGWork &mg, const double *rho, const double *chi, double V,
             const double *phi_zL, double *phi, bool warm, bool mixed, double tol, int max_cycles,
             double *rel_res, int *launches, cudaStream_t st);
template <typename T>
void launch_efield(const double *phi, double *Ez, double *Er, typename V2<T>::type *E2, int nz,
                   int nr, double dz, double dr, const StepCtl *ctl, cudaStream_t st);
void launch_moments(const double *Ne, const double *Ni, const double *V, const double *phi,
                    const double *Ez, const double *Er, double *m_ne, double *m_ni,
                    double *m_phi, double *m_ez, double *m_er, int ng, const StepCtl *ctl,
                    cudaStream_t st);

}  // namespace pic
