// pic_api.cu -- C ABI of the GB300 r-z implicit PIC/MC library
// (Wang, Jiang & Wang, arXiv:1001.2969): configuration checks, device state,
// and the per-step orchestration of the field solve, the particle pass and
// the cell sort on the caller's stream.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "mg.cuh"
#include "pic_internal.cuh"
#include "window.cuh"

using namespace pic;

namespace {

constexpr int kNumTiming = 5;  // solve, particle pass e, particle pass i, sort+births, other

struct RawBuf {
    void *q0 = nullptr, *q1 = nullptr;
    int32_t *cell = nullptr;
    uint64_t *id = nullptr;
    void *at = nullptr;  // a_theta (X-Y-Z pusher only)
};

template <typename T>
PBuf<T> view(const RawBuf &b) {
    PBuf<T> p;
    p.q0 = reinterpret_cast<typename V4<T>::type *>(b.q0);
    p.q1 = reinterpret_cast<typename V4<T>::type *>(b.q1);
    p.cell = b.cell;
    p.id = b.id;
    p.at = reinterpret_cast<T *>(b.at);
    return p;
}

struct SpecDev {
    RawBuf main[2], births[2];
    uint64_t *bkey[2] = {nullptr, nullptr};
    int32_t *perm = nullptr, *counts = nullptr, *cursor = nullptr, *block_sums = nullptr;
    int32_t *d_nmain[2] = {nullptr, nullptr}, *d_nbirths[2] = {nullptr, nullptr};
    int32_t *d_nalive = nullptr, *d_ntotal = nullptr;
    // births already in the buffer when the last pass began (held ions
    // collect newborns over several passes; each pass numbers its own)
    int32_t *d_nb0 = nullptr;
    void *sigma = nullptr;  // T[n_ch][n_e]
    void *sig4 = nullptr;   // T[n_e][4], channels interleaved
    void *w_ref = nullptr;  // T[ncr]
    int64_t cap = 0, bcap = 0;
    uint64_t next_id = 0;  // host copy of the device's step control
};

struct EvRec {
    int phase;
    cudaEvent_t a, b;
};

// one timestep captured as a CUDA graph, per parity of the current buffer set
struct StepGraph {
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;  // kernels in the graph
    bool failed = false;   // capture or instantiation failed: launch directly
};

}  // namespace

struct pic_handle {
    pic_config cfg;
    std::vector<double> own_sigma[2], own_thr[2], own_rf, own_phiL;
    std::vector<int32_t> own_kind[2];
    int nz = 0, nr = 0, ncz = 0, ncr = 0, ncell = 0, ng = 0;
    double dz = 0, dr = 0;
    bool mixed = false;
    cudaStream_t st = nullptr;
    std::vector<std::pair<void *, size_t>> allocs;
    DevScalars *ds = nullptr;
    StepCtl *sctl = nullptr;  // step control (device)
    double *rf_d = nullptr;   // rf table on the device: amplitudes, frequencies, phases
    int32_t *scal = nullptr;  // per-species device scalars (n_main, n_births, n_alive, n_total)
    SpecDev sp[2];
    int cur = 0;    // buffer set holding the electrons (and, without subcycling, the ions)
    int cur_i = 0;  // buffer set holding the ions (flips only in passes that move them)
    int K = 1;      // ion subcycling: the ions move every K-th pass
    double *N[2] = {nullptr, nullptr};
    double *rho = nullptr, *chi = nullptr, *phi = nullptr, *Ez = nullptr, *Er = nullptr, *V = nullptr;
    void *E2 = nullptr;
    double *phiL_d = nullptr;
    bool has_phiL = false;
    // external circuit: the two superposition parts of phi and an empty charge grid
    double *phi_P = nullptr, *phi_L = nullptr, *zero_grid = nullptr;
    double *phi_prev = nullptr;  // the potential of the step before phi's (mg_guess)
    double *m_acc[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    double *eedf = nullptr;
    double *tmp_grid[3] = {nullptr, nullptr, nullptr};
    double *mom_stage = nullptr;  // the scaled time averages on their way to host buffers
    // pinned host copy of the step control and the status word, read once per call
    struct HostCtl {
        StepCtl c;
        int32_t status;
    } *host_ctl = nullptr;
    MGFast mgf;
    RadixTmp rtmp;
    int64_t step = 0;  // host copy of the device's step number (exact after each call)
    int64_t nsamples = 0;
    int64_t mg_cycles_total = 0, steps_total = 0;  // host copies (device step control)
    int last_cycles = 0;
    double last_res = 0.0;
    int step_grid = 1;  // blocks of the particle pass (they walk the chunks)
    int variant[2] = {-1, -1};  // particle-pass shape per species (-1: default)
    cudaStream_t user_st = nullptr;  // the caller's stream
    cudaStream_t gst = nullptr;      // private stream the step graphs are captured on and run on
    cudaStream_t gst2 = nullptr;     // the step graph's second branch (the previous pass's cell sort)
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork2 = nullptr, ev_join2 = nullptr;
    StepGraph graphs[8];       // per (cur, cur_i, the pass moves the ions)
    StepGraph sort_graphs[4];  // the last pass's cell sort at the end of a call, per (cur, cur_i)
    StepGraph check_graphs[4];  // its capacity check alone (the rest deferred), per (cur, cur_i)
    bool sort_deferred = false;  // the last pass's rank and births numbering are still to run
    bool in_batch = false;     // stepped with other reactors (pic_batch): narrow solves
    double ngas = 0.0, nu_max[2] = {0, 0}, p_null[2] = {0, 0};
    unsigned long long t_null[2] = {0, 0};
    std::string err;
    bool prof = false;
    std::vector<EvRec> ev_live;
    std::vector<cudaEvent_t> ev_pool;
    double t_ms[kNumTiming] = {0, 0, 0, 0, 0};
    int64_t launches = 0, particle_launches = 0;
};

// Several reactors stepped together: each step of all of them is one graph
// that forks into one branch per reactor (its whole timestep on the
// reactor's private stream) and joins, keyed by the buffer parities.
struct pic_batch {
    std::vector<pic_handle *> hs;
    cudaStream_t st = nullptr;      // the caller's stream
    cudaStream_t origin = nullptr;  // where the batch graphs are captured and run
    cudaEvent_t ev_in = nullptr, ev_out = nullptr, ev_fork = nullptr;
    std::vector<cudaEvent_t> ev_join;
    struct Graph {
        cudaGraphExec_t exec = nullptr;
        std::vector<int64_t> launches;  // kernels per reactor in the graph
        bool failed = false;
        pic::SolveJob *jobs_d = nullptr;  // the shared solve launches' job table (device)
    };
    cudaEvent_t ev_fork2 = nullptr;
    std::map<std::vector<char>, Graph> graphs;
};

namespace {

// Ion subcycling (Sec. 2.7, Vahedi's method; the implicit form is a
// reading): the ions move in the passes n with n mod K = K - 1, with
// dt_i = K dt, and are held still, state and deposit, in the others.
bool moves_ions(const pic_handle *h, int64_t step) {
    const int64_t K = h->K;
    return K == 1 || ((step % K) + K) % K == K - 1;
}
// passes that moved the ions among steps [0, n) (floor(n / K))
int64_t ion_passes_before(const pic_handle *h, int64_t n) {
    const int64_t K = h->K;
    return n >= 0 ? n / K : -((-n + K - 1) / K);
}
double dt_of(const pic_handle *h, int s) { return s == 1 ? h->cfg.dt * h->K : h->cfg.dt; }
// susceptibility factor q^2 dt_s^2 / (2 eps0 m) of species s before a pass
// (Sec. 2.1); zero for ions the pass holds still
double chi_coef(const pic_handle *h, int s, bool moves) {
    if (s == 1 && !moves) return 0.0;
    const double dt = dt_of(h, s);
    return h->cfg.sp[s].q * h->cfg.sp[s].q * dt * dt / (2.0 * kEps0 * h->cfg.sp[s].m);
}
// the buffer set holding species s
int par_of(const pic_handle *h, int s) { return s == 1 ? h->cur_i : h->cur; }

pic_status fail(pic_handle *h, pic_status s, const std::string &msg) {
    if (h) h->err = msg;
    return s;
}

void *dalloc(pic_handle *h, size_t bytes) {
    if (bytes == 0) bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (h->cfg.alloc) {
        p = h->cfg.alloc(bytes, h->cfg.alloc_ctx, (void *)h->st);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (!p) throw std::bad_alloc();
    h->allocs.push_back({p, bytes});
    return p;
}

void free_all(pic_handle *h) {
    for (auto &a : h->allocs) {
        if (h->cfg.free)
            h->cfg.free(a.first, a.second, h->cfg.alloc_ctx, (void *)h->st);
        else if (!h->cfg.alloc)
            cudaFree(a.first);
    }
    h->allocs.clear();
}

pic_status cuda_check(pic_handle *h, const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return fail(h, PIC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
    return PIC_OK;
}

bool pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }

// ---- null-collision frequency bound (Sec. 2.6) ----
// nu_max = n_g max_E sigma_tot(E) sqrt(2 E e / m) over the table: endpoints
// of every linear segment and, on falling segments, the stationary point of
// (alpha + beta E) sqrt(E) at E = -alpha / (3 beta); beyond the table nu
// falls as E^-1/2.  A relative margin of 1e-6 absorbs rounding.
double nu_max_of(const pic_handle *h, int s) {
    const int ne = h->cfg.xs[s].n_e, nch = h->cfg.xs[s].n_ch;
    const double emax = h->cfg.xs[s].E_max_eV, dE = emax / (ne - 1), m = h->cfg.sp[s].m;
    auto tot = [&](int k) {
        double t = 0.0;
        for (int ch = 0; ch < nch; ++ch) t += h->own_sigma[s][(size_t)ch * ne + k];
        return t;
    };
    double best = 0.0;
    for (int k = 0; k < ne; ++k) {
        const double E = k * dE;
        best = std::max(best, tot(k) * sqrt(2.0 * E * kQe / m));
    }
    for (int k = 0; k + 1 < ne; ++k) {
        const double s0 = tot(k), s1 = tot(k + 1);
        const double beta = (s1 - s0) / dE;
        if (beta < 0.0) {
            const double alpha = s0 - beta * (k * dE);
            const double Es = -alpha / (3.0 * beta);
            if (Es > k * dE && Es < (k + 1) * dE)
                best = std::max(best, (alpha + beta * Es) * sqrt(2.0 * Es * kQe / m));
        }
    }
    return h->ngas * best * (1.0 + 1e-6);
}

pic_status validate(const pic_config *c, std::string &why) {
    auto bad = [&](const char *m) {
        why = m;
        return PIC_ERR_ARG;
    };
    if (!(c->mesh.R > 0) || !(c->mesh.L > 0)) return bad("mesh R and L must be positive");
    if (c->mesh.nz < 3 || !pow2(c->mesh.nz - 1)) return bad("nz must be 2^k + 1 >= 3");
    if (c->mesh.nr < 3 || c->mesh.nr > 1025) return bad("nr must be in [3, 1025]");
    if ((int64_t)(c->mesh.nz - 1) * (c->mesh.nr - 1) >= (1LL << 24)) return bad("mesh too large (cells < 2^24)");
    if (!(c->dt > 0)) return bad("dt must be positive");
    if (c->precision != PIC_FP64 && c->precision != PIC_MIXED) return bad("precision");
    if (c->weighting != PIC_WEIGHT_ZR2 && c->weighting != PIC_WEIGHT_ZR) return bad("weighting");
    if (c->chi_face != PIC_CHI_MAX && c->chi_face != PIC_CHI_MEAN) return bad("chi_face");
    if (c->scatter != PIC_SCATTER_VS && c->scatter != PIC_SCATTER_ISOTROPIC) return bad("scatter");
    if (c->split_every < 0) return bad("split_every must be >= 0");
    if (c->mg_max_cycles < 1) return bad("mg_max_cycles must be >= 1");
    if (c->pusher != PIC_PUSH_LOCAL && c->pusher != PIC_PUSH_XYZ) return bad("pusher must be PIC_PUSH_LOCAL or PIC_PUSH_XYZ");
    if (c->ion_subcycle < 0 || c->ion_subcycle > 1024) return bad("ion_subcycle must be in [0, 1024]");
    if (c->mg_guess != PIC_GUESS_PREVIOUS && c->mg_guess != PIC_GUESS_LINEAR)
        return bad("mg_guess must be PIC_GUESS_PREVIOUS or PIC_GUESS_LINEAR");
    if (c->ion_subcycle > 1 && c->split_every % c->ion_subcycle != 0)
        return bad("split_every must be a multiple of ion_subcycle");
    if (!(c->circuit_C >= 0.0) || !std::isfinite(c->circuit_C))
        return bad("circuit_C must be finite and >= 0 (0: the electrode follows the source)");
    if (c->eedf_bins < 0 || c->eedf_bins > 4096) return bad("eedf_bins must be in [0, 4096]");
    if (c->eedf_bins > 0 && !(c->eedf_emax_eV > 0)) return bad("eedf_emax_eV must be positive");
    if (!(c->gas.T_K > 0) || !(c->gas.m_gas > 0) || c->gas.p_Pa < 0) return bad("gas");
    if (c->rf.n < 0 || (c->rf.n > 0 && (!c->rf.amp_V || !c->rf.freq_Hz || !c->rf.phase_rad)))
        return bad("rf");
    for (int s = 0; s < 2; ++s) {
        const pic_species &p = c->sp[s];
        if (!(p.m > 0) || p.q == 0 || p.n0 < 0 || p.T_eV < 0) return bad("species q, m, n0, T");
        if (p.n_init < 0 || p.capacity < p.n_init || p.capacity < 1) return bad("species capacity");
        const int64_t bc = c->births_capacity > 0 ? c->births_capacity : std::max<int64_t>(4096, p.capacity / 2);
        if (p.capacity + bc >= (1LL << 31) - 1) return bad("capacity too large for 32-bit indices");
        const pic_xsec &x = c->xs[s];
        if (x.n_e < 2 || !(x.E_max_eV > 0) || x.n_ch < 1 || x.n_ch > PIC_MAX_CH || !x.sigma_m2 ||
            !x.threshold_eV || !x.kind)
            return bad("cross-section table");
        for (int ch = 0; ch < x.n_ch; ++ch) {
            const int k = x.kind[ch];
            if (s == 0 && k != PIC_XS_ELASTIC && k != PIC_XS_EXCITE && k != PIC_XS_IONIZE)
                return bad("electron channels must be ELASTIC, EXCITE or IONIZE");
            if (s == 1 && k != PIC_XS_CX) return bad("ion channels must be CX");
            if (k == PIC_XS_IONIZE && !(x.B_eV > 0)) return bad("ionisation needs B_eV > 0");
        }
    }
    return PIC_OK;
}

// node volumes of Sec. 2.4 (z-r^2 or z-r), inner halves on the boundary rows
// and on r = R
void node_volumes(const pic_handle *h, std::vector<double> &V) {
    V.assign((size_t)h->ng, 0.0);
    for (int i = 0; i < h->nz; ++i) {
        const double hz = (i == 0 || i == h->nz - 1) ? 0.5 * h->dz : h->dz;
        for (int j = 0; j < h->nr; ++j) {
            const double r = j * h->dr, rp = (j + 1) * h->dr, rm = (j - 1) * h->dr, r1 = h->dr;
            double v;
            if (h->cfg.weighting == PIC_WEIGHT_ZR) {
                if (j == 0)
                    v = kPi / 3.0 * r1 * r1;
                else if (j == h->nr - 1)
                    v = kPi / 3.0 * h->dr * (2.0 * r + rm);
                else
                    v = kPi / 3.0 * (rp * (r + rp) - rm * (r + rm));
            } else {
                if (j == 0)
                    v = kPi / 2.0 * r1 * r1;
                else if (j == h->nr - 1)
                    v = kPi / 2.0 * (r * r - rm * rm);
                else
                    v = kPi / 2.0 * (rp * rp - rm * rm);
            }
            V[(size_t)i * h->nr + j] = v * hz;
        }
    }
}

__global__ void k_iota(int32_t *p, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) p[k] = k;
}

__global__ void k_scale(const double *src, double *dst, int n, double f) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = src[k] * f;
}

// step prologue: the field time's electrode voltage (Sec. 2.5 boundary data)
// and the split flag, from the step number on the device
__global__ void k_step_begin(StepCtl *c, const double *rf, int nrf, double dt, int split_every) {
    if (c->halt) return;
    const double t = (double)(c->step + 1) * dt;
    double v = 0.0;
    for (int k = 0; k < nrf; ++k) v += rf[k] * sin(2.0 * kPi * rf[nrf + k] * t + rf[2 * nrf + k]);
    c->V = v;
    c->do_split = split_every > 0 && (c->step % split_every) == split_every - 1;
}

// step epilogue: the pass wrote *nalive entries into the destination main
// buffers; their cell sort is pending, and the step advances
// nmain1 / nalive1 null: the pass held the ions still (subcycling)
__global__ void k_step_end(StepCtl *c, DevScalars *ds, int32_t *nmain0, const int32_t *nalive0, int32_t *nmain1,
                           const int32_t *nalive1) {
    if (c->halt) return;
    *nmain0 = *nalive0;
    unsigned long long n = (unsigned long long)(*nalive0);
    if (nmain1) {
        *nmain1 = *nalive1;
        n += (unsigned long long)(*nalive1);
    }
    ds->cnt[PIC_C_PSTEPS] += n;
    c->sort_pending = 1;
    c->step += 1;
}

// sort epilogue: the sorted counts take effect for the next pass
// a pass that holds the ions: the births its newborn ions join start at
// the buffer's present count (skipped once the step has failed, so that a
// dropped pass's newborns can be cut off again)
// zero what the particle passes accumulate into (null members skipped)
struct PassReset {
    double *N[2];
    int32_t *counts[2];
    int32_t *nbirths[2];
    int32_t *nb0;
    int32_t *chunk_next;  // [2]
    int ng, ncell;
};
__global__ void k_pass_reset(PassReset r) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    for (int s = 0; s < 2; ++s) {
        if (r.N[s])
            for (int k = t; k < r.ng; k += stride) r.N[s][k] = 0.0;
        if (r.counts[s])
            for (int k = t; k < r.ncell; k += stride) r.counts[s][k] = 0;
    }
    if (t == 0) {
        for (int s = 0; s < 2; ++s)
            if (r.nbirths[s]) *r.nbirths[s] = 0;
        if (r.nb0) *r.nb0 = 0;
        r.chunk_next[0] = r.chunk_next[1] = 0;
    }
}

__global__ void k_hold_ions(const StepCtl *c, int32_t *nb0, const int32_t *nb) {
    if (c->halt) return;
    *nb0 = *nb;
}
__global__ void k_sort_end(StepCtl *c, int32_t *nalive0, const int32_t *ntotal0, int32_t *nalive1,
                           const int32_t *ntotal1) {
    if (sort_skip(c)) return;
    *nalive0 = *ntotal0;
    *nalive1 = *ntotal1;
    c->sort_pending = 0;
}

// External circuit (Sec. 2.5, end), Vahedi's superposition: the charge on
// the z = 0 electrode (Gauss's law on the electrode row: displacement flux
// eps0 c_0j (phi_0j - phi_1j) into row 1 less the half-cell charge
// rho_0j V_0j, nodes j < nr - 1) is Q_P + V Q_L; the circuit equation
// Q^t = Q^{t-1} + C (V_rf^t - V^t) - Q_c^{t-1} + Q_conv^t then fixes V^t.
// One block.
__global__ void k_circuit(StepCtl *c, DevScalars *ds, const double *cz0, const double *phiP,
                          const double *phiL, const double *rho, const double *Vn, int nr, double C) {
    __shared__ double sP[32], sL[32];
    if (c->halt) return;
    double qp = 0.0, ql = 0.0;
    for (int j = threadIdx.x; j < nr - 1; j += blockDim.x) {
        qp += kEps0 * cz0[j] * (phiP[j] - phiP[nr + j]) - rho[j] * Vn[j];
        ql += kEps0 * cz0[j] * (phiL[j] - phiL[nr + j]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        qp += __shfl_xor_sync(0xffffffffu, qp, o);
        ql += __shfl_xor_sync(0xffffffffu, ql, o);
    }
    if ((threadIdx.x & 31) == 0) {
        sP[threadIdx.x >> 5] = qp;
        sL[threadIdx.x >> 5] = ql;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double QP = 0.0, QL = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            QP += sP[w];
            QL += sL[w];
        }
        const double Vrf = c->V;
        const double Vt = (c->circ_Q - c->circ_Qc + C * Vrf + ds->qstep[0] - QP) / (QL + C);
        c->circ_V = Vt;
        c->circ_Q = QP + Vt * QL;
        c->circ_Qc = C * (Vrf - Vt);
        // the collected charge is taken; the coming particle pass adds anew
        ds->qstep[0] = ds->qstep[1] = ds->qstep[2] = 0.0;
    }
}

// phi = phi_P + V phi_L
__global__ void k_superpose(const StepCtl *c, const double *phiP, const double *phiL, double *phi, int ng) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng || c->halt) return;
    phi[k] = phiP[k] + c->circ_V * phiL[k];
}

// host values the device's step control starts from
void push_ctl(pic_handle *h) {
    StepCtl c;
    cudaMemcpyAsync(&c, h->sctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    c.step = h->step;
    c.next_id[0] = h->sp[0].next_id;
    c.next_id[1] = h->sp[1].next_id;
    cudaMemcpyAsync(h->sctl, &c, sizeof(StepCtl), cudaMemcpyHostToDevice, h->st);
    cudaStreamSynchronize(h->st);
}

cudaEvent_t ev_get(pic_handle *h) {
    if (!h->ev_pool.empty()) {
        cudaEvent_t e = h->ev_pool.back();
        h->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct PhaseTimer {
    pic_handle *h;
    int phase;
    cudaEvent_t a = nullptr;
    PhaseTimer(pic_handle *hh, int ph) : h(hh), phase(ph) {
        if (h->prof) {
            a = ev_get(h);
            cudaEventRecord(a, h->st);
        }
    }
    ~PhaseTimer() {
        if (h->prof) {
            cudaEvent_t b = ev_get(h);
            cudaEventRecord(b, h->st);
            h->ev_live.push_back({phase, a, b});
        }
    }
};

void resolve_events(pic_handle *h) {
    if (h->ev_live.empty()) return;
    cudaStreamSynchronize(h->st);
    for (auto &r : h->ev_live) {
        float ms = 0;
        cudaEventElapsedTime(&ms, r.a, r.b);
        h->t_ms[r.phase] += ms;
        h->ev_pool.push_back(r.a);
        h->ev_pool.push_back(r.b);
    }
    h->ev_live.clear();
}

template <typename T>
void alloc_tables(pic_handle *h) {
    for (int s = 0; s < 2; ++s) {
        const pic_xsec &x = h->cfg.xs[s];
        std::vector<T> sg((size_t)x.n_ch * x.n_e);
        for (size_t k = 0; k < sg.size(); ++k) sg[k] = (T)h->own_sigma[s][k];
        h->sp[s].sigma = dalloc(h, sg.size() * sizeof(T));
        cudaMemcpyAsync(h->sp[s].sigma, sg.data(), sg.size() * sizeof(T), cudaMemcpyHostToDevice, h->st);
        std::vector<T> s4((size_t)x.n_e * 4, (T)0);
        for (int ch = 0; ch < x.n_ch; ++ch)
            for (int k = 0; k < x.n_e; ++k) s4[(size_t)k * 4 + ch] = (T)h->own_sigma[s][(size_t)ch * x.n_e + k];
        h->sp[s].sig4 = dalloc(h, s4.size() * sizeof(T));
        cudaMemcpyAsync(h->sp[s].sig4, s4.data(), s4.size() * sizeof(T), cudaMemcpyHostToDevice, h->st);
        cudaStreamSynchronize(h->st);
        // reference weight of radial cell j (Sec. 2.2): n0 pi (r_{j+1}^2 - r_j^2) dz / ppc_ref
        const int64_t base = h->cfg.sp[s].n_init / h->ncell;
        const double ppc = (double)(base > 0 ? base : 1);
        std::vector<T> wr(h->ncr);
        for (int j = 0; j < h->ncr; ++j) {
            const double r0 = j * h->dr, r1 = (j + 1) * h->dr;
            wr[j] = (T)(h->cfg.sp[s].n0 * kPi * (r1 * r1 - r0 * r0) * h->dz / ppc);
        }
        h->sp[s].w_ref = dalloc(h, wr.size() * sizeof(T));
        cudaMemcpyAsync(h->sp[s].w_ref, wr.data(), wr.size() * sizeof(T), cudaMemcpyHostToDevice, h->st);
    }
    cudaStreamSynchronize(h->st);
}

void alloc_rawbuf(pic_handle *h, RawBuf &b, int64_t n, size_t tsize) {
    b.q0 = dalloc(h, (size_t)n * 4 * tsize);
    b.q1 = dalloc(h, (size_t)n * 4 * tsize);
    b.cell = (int32_t *)dalloc(h, (size_t)n * sizeof(int32_t));
    b.id = (uint64_t *)dalloc(h, (size_t)n * sizeof(uint64_t));
    if (h->cfg.pusher == PIC_PUSH_XYZ) b.at = dalloc(h, (size_t)n * tsize);
}

void setup_device(pic_handle *h) {
    const size_t ts = h->mixed ? sizeof(float) : sizeof(double);
    h->ds = (DevScalars *)dalloc(h, sizeof(DevScalars));
    cudaMemsetAsync(h->ds, 0, sizeof(DevScalars), h->st);
    {
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        h->step_grid = std::max(1, nsm * 8);
    }
    h->sctl = (StepCtl *)dalloc(h, sizeof(StepCtl));
    cudaMemsetAsync(h->sctl, 0, sizeof(StepCtl), h->st);
    h->rf_d = (double *)dalloc(h, std::max<size_t>(1, h->own_rf.size()) * sizeof(double));
    if (!h->own_rf.empty())
        cudaMemcpyAsync(h->rf_d, h->own_rf.data(), h->own_rf.size() * sizeof(double), cudaMemcpyHostToDevice, h->st);
    h->scal = (int32_t *)dalloc(h, 2 * 8 * sizeof(int32_t));
    cudaMemsetAsync(h->scal, 0, 2 * 8 * sizeof(int32_t), h->st);
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        d.cap = h->cfg.sp[s].capacity;
        d.bcap = h->cfg.births_capacity > 0 ? h->cfg.births_capacity : std::max<int64_t>(4096, d.cap / 2);
        for (int k = 0; k < 2; ++k) {
            alloc_rawbuf(h, d.main[k], d.cap, ts);
            alloc_rawbuf(h, d.births[k], d.bcap, ts);
            d.bkey[k] = (uint64_t *)dalloc(h, (size_t)d.bcap * sizeof(uint64_t));
        }
        d.perm = (int32_t *)dalloc(h, (size_t)d.cap * sizeof(int32_t));
        d.counts = (int32_t *)dalloc(h, (size_t)h->ncell * sizeof(int32_t));
        d.cursor = (int32_t *)dalloc(h, (size_t)h->ncell * sizeof(int32_t));
        d.block_sums = (int32_t *)dalloc(h, (size_t)(h->ncell / 4096 + 2) * sizeof(int32_t));
        int32_t *sc = h->scal + s * 8;
        d.d_nmain[0] = sc + 0;
        d.d_nmain[1] = sc + 1;
        d.d_nbirths[0] = sc + 2;
        d.d_nbirths[1] = sc + 3;
        d.d_nalive = sc + 4;
        d.d_ntotal = sc + 5;
        d.d_nb0 = sc + 6;
    }
    const size_t gb = (size_t)h->ng * sizeof(double);
    for (int s = 0; s < 2; ++s) h->N[s] = (double *)dalloc(h, gb);
    h->rho = (double *)dalloc(h, gb);
    h->chi = (double *)dalloc(h, gb);
    h->phi = (double *)dalloc(h, gb);
    h->phi_prev = (double *)dalloc(h, gb);
    h->Ez = (double *)dalloc(h, gb);
    h->Er = (double *)dalloc(h, gb);
    h->V = (double *)dalloc(h, gb);
    for (int k = 0; k < 3; ++k) h->tmp_grid[k] = (double *)dalloc(h, gb);
    for (int k = 0; k < 5; ++k) h->m_acc[k] = (double *)dalloc(h, gb);
    h->E2 = dalloc(h, (size_t)h->ng * 2 * ts);
    h->phiL_d = (double *)dalloc(h, (size_t)h->nr * sizeof(double));
    if (h->cfg.circuit_C > 0.0) {
        h->phi_P = (double *)dalloc(h, gb);
        h->phi_L = (double *)dalloc(h, gb);
        h->zero_grid = (double *)dalloc(h, gb);
        cudaMemsetAsync(h->phi_P, 0, gb, h->st);
        cudaMemsetAsync(h->phi_L, 0, gb, h->st);
        cudaMemsetAsync(h->zero_grid, 0, gb, h->st);
    }
    h->eedf = (double *)dalloc(h, (size_t)std::max(1, h->cfg.eedf_bins) * sizeof(double));
    for (int s = 0; s < 2; ++s) cudaMemsetAsync(h->N[s], 0, gb, h->st);
    cudaMemsetAsync(h->phi, 0, gb, h->st);
    cudaMemsetAsync(h->phi_prev, 0, gb, h->st);  // = phi: the first step starts from phi
    cudaMemsetAsync(h->Ez, 0, gb, h->st);
    cudaMemsetAsync(h->Er, 0, gb, h->st);
    cudaMemsetAsync(h->rho, 0, gb, h->st);
    cudaMemsetAsync(h->chi, 0, gb, h->st);
    for (int k = 0; k < 5; ++k) cudaMemsetAsync(h->m_acc[k], 0, gb, h->st);
    cudaMemsetAsync(h->eedf, 0, (size_t)std::max(1, h->cfg.eedf_bins) * sizeof(double), h->st);
    if (h->has_phiL)
        cudaMemcpyAsync(h->phiL_d, h->own_phiL.data(), (size_t)h->nr * sizeof(double),
                        cudaMemcpyHostToDevice, h->st);
    std::vector<double> V;
    node_volumes(h, V);
    cudaMemcpyAsync(h->V, V.data(), gb, cudaMemcpyHostToDevice, h->st);
    // multigrid hierarchy: per level nodal chi and face coefficients, the
    // V-cycle's correction and right-hand side, and the r-line factors
    MGFast &m = h->mgf;
    memset(&m, 0, sizeof(m));
    const size_t line_fe = mg_line_factor_elems(h->nr);
    int nl = 0;
    for (int z = h->nz;; z = (z + 1) / 2) {
        const int l = nl++;
        m.nz[l] = z;
        m.dz[l] = h->cfg.mesh.L / (z - 1);
        const size_t g = (size_t)z * h->nr;
        m.chi[l] = (double *)dalloc(h, g * sizeof(double));
        m.cz[l] = (double *)dalloc(h, g * sizeof(double));
        m.cr[l] = (double *)dalloc(h, g * sizeof(double));
        if (h->mixed) {
            m.cz32[l] = (float *)dalloc(h, g * sizeof(float));
            m.cr32[l] = (float *)dalloc(h, g * sizeof(float));
            m.u32[l] = (float *)dalloc(h, g * sizeof(float));
            m.f32[l] = (float *)dalloc(h, g * sizeof(float));
        } else {
            m.u64[l] = (double *)dalloc(h, g * sizeof(double));
            m.f64[l] = (double *)dalloc(h, g * sizeof(double));
        }
        const size_t fe = (size_t)(z - 2) * line_fe;
        if (z == 3) {
            m.facc = (double *)dalloc(h, fe * sizeof(double));
            if (h->mixed) m.facc32 = (float *)dalloc(h, fe * sizeof(float));
        } else if (!h->mixed)
            m.fac64[l] = (double *)dalloc(h, fe * sizeof(double));
        else
            m.fac32[l] = (float *)dalloc(h, fe * sizeof(float));
        if (z == 3) break;
    }
    m.nlev = nl;
    {
        std::vector<double> geo;
        mg_fast_geometry(m, h->nr, h->dr, geo);
        double *g = (double *)dalloc(h, geo.size() * sizeof(double));
        cudaMemcpyAsync(g, geo.data(), geo.size() * sizeof(double), cudaMemcpyHostToDevice, h->st);
        for (int l = 0; l < nl; ++l) {
            m.gz[l] = g + (size_t)2 * l * h->nr;
            m.gr[l] = m.gz[l] + h->nr;
        }
        m.ga = g + (size_t)2 * nl * h->nr;
        cudaStreamSynchronize(h->st);  // geo is a local
    }
    m.fc64 = (double *)dalloc(h, (size_t)3 * h->nr * sizeof(double));
    m.f0 = (double *)dalloc(h, gb);
    m.dg0 = (double *)dalloc(h, gb);
    m.phi2 = (double *)dalloc(h, gb);
    if (h->mixed) {
        m.kr = (double *)dalloc(h, gb);
        m.kw = (double *)dalloc(h, gb);
        m.kzp = (double *)dalloc(h, gb);
        m.kwp = (double *)dalloc(h, gb);
        m.kpart = (double *)dalloc(h, (size_t)4 * 1024 * sizeof(double));
        for (double *z : {m.kr, m.kw, m.kzp, m.kwp}) cudaMemsetAsync(z, 0, gb, h->st);
    }
    m.ctl = (MGCtl *)dalloc(h, sizeof(MGCtl));
    m.self = (MGFast *)dalloc(h, sizeof(MGFast));
    mg_fast_upload(m, h->st);
    // births radix scratch
    int64_t bmax = std::max(h->sp[0].bcap, h->sp[1].bcap);
    h->rtmp.max_n = (int)bmax;
    h->rtmp.k0 = (uint64_t *)dalloc(h, (size_t)bmax * 8);
    h->rtmp.k1 = (uint64_t *)dalloc(h, (size_t)bmax * 8);
    h->rtmp.v0 = (uint32_t *)dalloc(h, (size_t)bmax * 4);
    h->rtmp.v1 = (uint32_t *)dalloc(h, (size_t)bmax * 4);
    h->rtmp.hist = (uint32_t *)dalloc(h, (size_t)256 * (bmax / 2048 + 2) * 4);
    h->rtmp.flag = (int *)dalloc(h, sizeof(int));
    if (h->mixed)
        alloc_tables<float>(h);
    else
        alloc_tables<double>(h);
}

template <typename T>
void deposit_current(pic_handle *h) {
    for (int s = 0; s < 2; ++s) cudaMemsetAsync(h->N[s], 0, (size_t)h->ng * sizeof(double), h->st);
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        const int c = par_of(h, s);
        launch_deposit<T>(view<T>(d.main[c]), d.d_nmain[c], h->nz, h->nr, h->cfg.weighting, h->N[s], h->st);
        launch_deposit<T>(view<T>(d.births[c]), d.d_nbirths[c], h->nz, h->nr, h->cfg.weighting, h->N[s],
                          h->st);
        h->launches += 2;
    }
}

template <typename T>
pic_status load_all(pic_handle *h) {
    const uint32_t k0 = (uint32_t)h->cfg.seed, k1 = (uint32_t)(h->cfg.seed >> 32);
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        const pic_species &p = h->cfg.sp[s];
        const int64_t n = h->cfg.load ? p.n_init : 0;
        launch_load<T>(view<T>(d.main[0]), n, s, h->nz, h->nr, h->dz, h->dr, p.n0, p.T_eV, p.m, k0,
                       k1, h->ncell, h->st);
        if (n > 0) k_iota<<<(unsigned)((n + 255) / 256), 256, 0, h->st>>>(d.perm, (int)n);
        const int32_t vals[8] = {(int32_t)n, 0, 0, 0, (int32_t)n, (int32_t)n, 0, 0};
        cudaMemcpyAsync(h->scal + s * 8, vals, sizeof(vals), cudaMemcpyHostToDevice, h->st);
        // the stored state's cell counts (held ions keep them until their
        // next moving pass; otherwise the first pass recounts)
        cudaMemsetAsync(d.counts, 0, (size_t)h->ncell * sizeof(int32_t), h->st);
        launch_hist<T>(view<T>(d.main[0]), d.d_nmain[0], d.counts, h->st);
        d.next_id = (uint64_t)n;
        h->launches += 3;
    }
    h->cur = h->cur_i = 0;
    deposit_current<T>(h);
    cudaStreamSynchronize(h->st);
    push_ctl(h);
    return cuda_check(h, "load");
}


// the pass of species s from buffer set src_set to dst_set; newborn ions go
// to the ions' set ion_set (the one their next moving pass reads)
template <typename T>
void fill_step_args(pic_handle *h, StepArgs<T> &a, int s, int src_set, int dst_set, int ion_set) {
    const pic_species &p = h->cfg.sp[s];
    const double dt = dt_of(h, s), qm = p.q / p.m;
    a.nz = h->nz;
    a.nr = h->nr;
    a.ncz = h->ncz;
    a.ncr = h->ncr;
    a.inv_ncz = 1.0f / (float)h->ncz;
    a.s = s;
    a.qch[0] = h->cfg.sp[0].q;
    a.qch[1] = h->cfg.sp[1].q;
    a.weighting = h->cfg.weighting;
    a.scatter = h->cfg.scatter;
    a.xyz = h->cfg.pusher == PIC_PUSH_XYZ ? 1 : 0;
    a.kz = (T)(0.5 * qm * dt * dt / h->dz);
    a.kr = (T)(0.5 * qm * dt * dt / h->dr);
    a.kv = (T)(0.5 * qm * dt);
    a.ka = (T)qm;
    a.dt = (T)dt;
    a.dt_dz = (T)(dt / h->dz);
    a.dt_dr = (T)(dt / h->dr);
    a.dr = (T)h->dr;
    a.inv_dr = (T)(1.0 / h->dr);
    a.t_null = h->t_null[s];
    a.nu_max = (T)h->nu_max[s];
    a.ng = (T)h->ngas;
    a.half_m_e = (T)(0.5 * p.m / kQe);
    a.two_e_m = (T)(2.0 * kQe / p.m);
    a.two_m_M = (T)(2.0 * p.m / h->cfg.gas.m_gas);
    a.v_gas = (T)sqrt(kKB * h->cfg.gas.T_K / h->cfg.gas.m_gas);
    a.ion_acc = (T)((h->cfg.sp[1].q * h->cfg.sp[0].m) / (h->cfg.sp[0].q * h->cfg.sp[1].m));
    const pic_xsec &x = h->cfg.xs[s];
    a.xs.sigma = (const T *)h->sp[s].sigma;
    a.xs.sig4 = (const typename V4<T>::type *)h->sp[s].sig4;
    a.xs.n_e = x.n_e;
    a.xs.n_ch = x.n_ch;
    a.xs.emax = (T)x.E_max_eV;
    a.xs.inv_dE = (T)((x.n_e - 1) / x.E_max_eV);
    for (int ch = 0; ch < kMaxCh; ++ch) {
        a.xs.kind[ch] = ch < x.n_ch ? h->own_kind[s][ch] : 0;
        a.xs.thr[ch] = ch < x.n_ch ? (T)h->own_thr[s][ch] : (T)0;
    }
    a.xs.B = (T)x.B_eV;
    a.key0 = (uint32_t)h->cfg.seed;
    a.key1 = (uint32_t)(h->cfg.seed >> 32);
    a.ctl = h->sctl;
    a.w_ref = (const T *)h->sp[s].w_ref;
    a.E = (const typename V2<T>::type *)h->E2;
    SpecDev &d = h->sp[s];
    a.src_main = view<T>(d.main[src_set]);
    a.src_births = view<T>(d.births[src_set]);
    a.n_main_src = d.d_nmain[src_set];
    a.perm = d.perm;
    a.n_alive = d.d_nalive;
    a.dst_main = view<T>(d.main[dst_set]);
    for (int t = 0; t < 2; ++t) {
        const int bs = t == 1 ? ion_set : dst_set;
        a.births[t] = view<T>(h->sp[t].births[bs]);
        a.bkey[t] = h->sp[t].bkey[bs];
        a.nb[t] = h->sp[t].d_nbirths[bs];
        a.N[t] = h->N[t];
        a.counts[t] = h->sp[t].counts;
        a.bdt[t] = (T)dt_of(h, t);
        a.bdt_dz[t] = (T)(dt_of(h, t) / h->dz);
    }
    a.bcap = (int)std::min(h->sp[0].bcap, h->sp[1].bcap);
    a.ds = h->ds;
    a.chunk_next = &h->ds->chunk_next[s];
    a.eedf = (s == 0 && h->cfg.eedf_bins > 0) ? h->eedf : nullptr;
    a.eedf_bins = h->cfg.eedf_bins;
    a.eedf_scale = h->cfg.eedf_bins > 0 ? (T)(h->cfg.eedf_bins / h->cfg.eedf_emax_eV) : (T)0;
}

// Enqueues one timestep (Sec. 2.1 merged cycle) without a host
// synchronisation; failures halt the step on the device (StepCtl) and are
// resolved by pic_step after the last step of the call.
// The cell sort of the last pass, whose output is the buffer set `par`
// (Sec. 2.7; a GPU necessity here): per species an exclusive scan of the
// pass's cell counts, the capacity check, the rank into the permutation the
// next pass reads through.  Regular kernels only, so it can run beside the
// cooperative field solve.
// With ion subcycling the ions are sorted only before a pass that moves
// them (ions = false otherwise): held ions keep their order, and their
// counts and births collect until then.
template <typename T>
void sort_branch(pic_handle *h, int par_e, int par_i, bool ions, cudaStream_t st) {
    const int ns = ions ? 2 : 1;
    for (int s = 0; s < ns; ++s) {
        SpecDev &d = h->sp[s];
        launch_scan(d.counts, d.cursor, h->ncell, d.block_sums, d.d_ntotal, d.cap, h->ds, h->sctl, st);
    }
    // capacity and births overflow: the sort fails before any permutation changes
    launch_step_check(h->ds, h->sctl, st);
    for (int s = 0; s < ns; ++s) {
        SpecDev &d = h->sp[s];
        const int par = s == 1 ? par_i : par_e;
        launch_rank<T>(view<T>(d.main[par]), d.d_nmain[par], view<T>(d.births[par]), d.d_nbirths[par],
                       d.cursor, d.perm, d.d_ntotal, d.cap, &h->ds->status, h->sctl, h->ncell, st);
    }
    h->launches += 4 * ns + 1;
}

// the rest of the sort: newborn numbering (a cooperative launch, after the
// field solve's), then the sorted counts take effect
void sort_finish(pic_handle *h, int par_e, int par_i, cudaStream_t st) {
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        const int par = s == 1 ? par_i : par_e;
        // in a batch: at most 8 blocks (a step's births are few; the numbering
        // is a cooperative launch, and a wide one waits for free SMs)
        launch_birth_ids(d.bkey[par], d.births[par].id, d.d_nbirths[par], d.d_nb0, h->sctl, s, h->rtmp, st,
                         h->in_batch ? 1 : 1 << 30);
    }
    k_sort_end<<<1, 1, 0, st>>>(h->sctl, h->sp[0].d_nalive, h->sp[0].d_ntotal, h->sp[1].d_nalive,
                                 h->sp[1].d_ntotal);
    h->launches += 3;
}

// Enqueue one timestep (Sec. 2.1, merged cycle) on h->st: the field at the
// new time (finalize, solve, E) beside the previous pass's cell sort (on
// sb, forked and joined; in order on h->st when sb is null), then the
// particle passes, the time averages and the step's end.  The pass's own
// sort is left pending for the next step or the end of the call.  mv: the
// pass moves the ions (always without subcycling); otherwise they stay in
// their buffer set with their deposit, and newborn ions join their births.
// part 0: the whole step; a batch whose reactors solve in shared launches
// splits it: part 1 ends after the solve's set-up (its solve described in
// *job), part 2 starts after the shared solve launch.
template <typename T>
void one_step(pic_handle *h, cudaStream_t sb, bool mv, int part = 0, SolveJob *job = nullptr) {
    cudaStream_t st = h->st;
    const int src = h->cur, dst = 1 - h->cur;
    const int isrc = h->cur_i, idst = mv ? 1 - h->cur_i : h->cur_i;
    if (part == 2) {
        mg_solve_done(h->mgf, h->sctl, true, st);
        launch_efield<T>(h->phi, h->Ez, h->Er, (typename V2<T>::type *)h->E2, h->nz, h->nr, h->dz,
                         h->dr, h->sctl, st);
        h->launches += 3;  // the shared solve's share, its report, E
    } else {
    k_step_begin<<<1, 1, 0, st>>>(h->sctl, h->rf_d, h->cfg.rf.n, h->cfg.dt, h->cfg.split_every);
    h->launches += 1;
    if (!sb) {
        PhaseTimer t(h, 3);
        sort_branch<T>(h, src, isrc, mv, st);
    }
    // with a second branch, the sort forks off right before the one-launch
    // solve (after its set-up): the solve, at the highest priority, takes
    // its SMs first and the sort's blocks fill the rest of the machine
    cudaEvent_t fork = sb ? h->ev_fork : nullptr;
    {
        PhaseTimer t(h, 0);
        launch_finalize(h->N[0], h->N[1], h->V, h->cfg.sp[0].q, h->cfg.sp[1].q, chi_coef(h, 0, true),
                        chi_coef(h, 1, mv), h->rho, h->chi, h->ng, h->sctl, st);
        FieldDims fd{h->nz, h->nr, h->dz, h->dr, h->cfg.mesh.L, h->cfg.chi_face};
        int L = 0;
        if (h->cfg.circuit_C > 0.0) {
            // phi_P: the plasma's charge, electrode at 0; phi_L: no charge,
            // electrode at 1, every other boundary at 0; same operator
            mg_fast_solve(fd, h->mgf, h->rho, h->chi, 0.0, h->has_phiL ? h->phiL_d : nullptr, h->phi_P,
                          true, h->mixed, h->cfg.mg_tol, h->cfg.mg_max_cycles, nullptr, &L, h->sctl, st,
                          false, true, fork, !h->in_batch);
            mg_fast_solve(fd, h->mgf, h->zero_grid, h->chi, 1.0, nullptr, h->phi_L, true, h->mixed,
                          h->cfg.mg_tol, h->cfg.mg_max_cycles, nullptr, &L, h->sctl, st, false, false, nullptr,
                          !h->in_batch);
            k_circuit<<<1, 256, 0, st>>>(h->sctl, h->ds, h->mgf.cz[0], h->phi_P, h->phi_L, h->rho, h->V,
                                         h->nr, h->cfg.circuit_C);
            k_superpose<<<(h->ng + 255) / 256, 256, 0, st>>>(h->sctl, h->phi_P, h->phi_L, h->phi, h->ng);
            L += 2;
        } else {
            mg_fast_solve(fd, h->mgf, h->rho, h->chi, 0.0, h->has_phiL ? h->phiL_d : nullptr, h->phi,
                          true, h->mixed, h->cfg.mg_tol, h->cfg.mg_max_cycles, nullptr, &L, h->sctl, st, true,
                          true, fork, !h->in_batch, part == 1 ? job : nullptr,
                          h->cfg.mg_guess == PIC_GUESS_LINEAR ? h->phi_prev : nullptr);
            if (part == 1) {
                h->launches += L;
                return;
            }
        }
        if (sb) {
            cudaStreamWaitEvent(sb, h->ev_fork, 0);
            sort_branch<T>(h, src, isrc, mv, sb);
            cudaEventRecord(h->ev_join, sb);
        }
        launch_efield<T>(h->phi, h->Ez, h->Er, (typename V2<T>::type *)h->E2, h->nz, h->nr, h->dz,
                         h->dr, h->sctl, st);
        h->launches += L + 2;
    }
    if (sb) cudaStreamWaitEvent(st, h->ev_join, 0);
    }
    {
        PhaseTimer t(h, 3);
        sort_finish(h, src, isrc, st);
    }
    {
        // the passes' deposit, cell counts, births counters and chunk
        // counters start at zero (one launch for both species)
        PassReset r{};
        r.ng = h->ng;
        r.ncell = h->ncell;
        r.chunk_next = h->ds->chunk_next;
        for (int s = 0; s < (mv ? 2 : 1); ++s) {
            SpecDev &d = h->sp[s];
            r.N[s] = h->N[s];
            r.counts[s] = d.counts;
            r.nbirths[s] = d.d_nbirths[s == 1 ? idst : dst];
        }
        if (mv && h->K > 1) r.nb0 = h->sp[1].d_nb0;  // else always 0
        k_pass_reset<<<std::max(1, std::min(152 * 4, (std::max(h->ng, h->ncell) + 255) / 256)), 256, 0, st>>>(r);
        h->launches += 1;
        if (!mv) {
            // held ions: deposit, counts and births stay; this pass's
            // newborns are numbered from the births already there
            k_hold_ions<<<1, 1, 0, st>>>(h->sctl, h->sp[1].d_nb0, h->sp[1].d_nbirths[idst]);
            h->launches += 1;
        }
    }
    // the two species' passes are independent (what they share -- the other
    // species' births, deposit and counts -- takes atomics or reserved
    // slots): with a second branch the ion pass runs beside the electrons'
    const bool fork2 = sb && mv;
    if (fork2) {
        cudaEventRecord(h->ev_fork2, st);
        cudaStreamWaitEvent(sb, h->ev_fork2, 0);
    }
    for (int s = 0; s < (mv ? 2 : 1); ++s) {
        PhaseTimer t(h, 1 + s);
        StepArgs<T> a;
        if (s == 0)
            fill_step_args<T>(h, a, 0, src, dst, idst);
        else
            fill_step_args<T>(h, a, 1, isrc, idst, idst);
        // blocks walk the chunks of the count on the device; a small store
        // takes no more blocks than its capacity has chunks
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(h->step_grid, (h->sp[s].cap + 1023) / 1024));
        launch_step<T>(a, grid, h->variant[s], (fork2 && s == 1) ? sb : st);
        h->launches += 1;
        h->particle_launches += 1;
    }
    if (fork2) {
        cudaEventRecord(h->ev_join2, sb);
        cudaStreamWaitEvent(st, h->ev_join2, 0);
    }
    {
        PhaseTimer t(h, 4);
        launch_moments(h->N[0], h->N[1], h->V, h->phi, h->Ez, h->Er, h->m_acc[0], h->m_acc[1],
                       h->m_acc[2], h->m_acc[3], h->m_acc[4], h->ng, h->sctl, st);
        k_step_end<<<1, 1, 0, st>>>(h->sctl, h->ds, h->sp[0].d_nmain[dst], h->sp[0].d_nalive,
                                     mv ? h->sp[1].d_nmain[idst] : nullptr, mv ? h->sp[1].d_nalive : nullptr);
        h->launches += 2;
    }
    h->cur = dst;
    h->cur_i = idst;
}

// the capacity check of the last pass's sort alone (end of a call): the
// scans of the cell counts and the check.  Rank, births numbering and the
// sorted counts stay pending; the next step's graph runs them beside its
// solve, or complete_sort() before the state is read.  Scans and check are
// idempotent on unchanged counts, so running them again there is harmless.
void check_tail(pic_handle *h) {
    PhaseTimer t(h, 3);
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        launch_scan(d.counts, d.cursor, h->ncell, d.block_sums, d.d_ntotal, d.cap, h->ds, h->sctl, h->st);
    }
    launch_step_check(h->ds, h->sctl, h->st);
    h->launches += 7;
}

// the pending sort of the last pass (end of a call), on h->st
template <typename T>
void sort_tail(pic_handle *h) {
    PhaseTimer t(h, 3);
    sort_branch<T>(h, h->cur, h->cur_i, true, h->st);
    sort_finish(h, h->cur, h->cur_i, h->st);
}

void drop_graphs(pic_handle *h) {
    for (StepGraph &g : h->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = StepGraph();
    }
    for (StepGraph &g : h->sort_graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = StepGraph();
    }
    for (StepGraph &g : h->check_graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g = StepGraph();
    }
}

void destroy_streams(pic_handle *h) {
    drop_graphs(h);
    for (cudaEvent_t e : {h->ev_in, h->ev_out, h->ev_fork, h->ev_join, h->ev_fork2, h->ev_join2})
        if (e) cudaEventDestroy(e);
    if (h->gst) cudaStreamDestroy(h->gst);
    if (h->gst2) cudaStreamDestroy(h->gst2);
    h->ev_in = h->ev_out = h->ev_fork = h->ev_join = h->ev_fork2 = h->ev_join2 = nullptr;
    h->gst = h->gst2 = nullptr;
}

// capture one step (from the current parities) on the private stream
template <typename T>
void capture_step(pic_handle *h, StepGraph &g, bool mv) {
    const int cur = h->cur, cur_i = h->cur_i;
    const int64_t L0 = h->launches, P0 = h->particle_launches;
    cudaStream_t keep = h->st;
    h->st = h->gst;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        one_step<T>(h, h->gst2, mv);
        e = cudaStreamEndCapture(h->gst, &graph);
    }
    h->st = keep;
    h->cur = cur;
    h->cur_i = cur_i;
    g.launches = h->launches - L0;
    h->launches = L0;
    h->particle_launches = P0;
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !g.exec) {
        g.exec = nullptr;
        g.failed = true;
        cudaGetLastError();
    }
}

// capture the pending sort of the current parity (the end of a call), or
// its capacity check alone
template <typename T>
void capture_sort(pic_handle *h, StepGraph &g, bool check_only) {
    const int64_t L0 = h->launches;
    cudaStream_t keep = h->st;
    h->st = h->gst;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->gst, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        if (check_only)
            check_tail(h);
        else
            sort_tail<T>(h);
        e = cudaStreamEndCapture(h->gst, &graph);
    }
    h->st = keep;
    g.launches = h->launches - L0;
    h->launches = L0;
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !g.exec) {
        g.exec = nullptr;
        g.failed = true;
        cudaGetLastError();
    }
}

// enqueue the pending sort, or its capacity check alone, on stream `on`
// (private stream: as a graph)
void enqueue_sort_tail(pic_handle *h, cudaStream_t on, bool check_only = false) {
    StepGraph &g = (check_only ? h->check_graphs : h->sort_graphs)[h->cur + 2 * h->cur_i];
    if (on == h->gst && !g.exec && !g.failed) {
        if (h->mixed)
            capture_sort<float>(h, g, check_only);
        else
            capture_sort<double>(h, g, check_only);
    }
    if (on == h->gst && g.exec) {
        cudaGraphLaunch(g.exec, h->gst);
        h->launches += g.launches;
        return;
    }
    cudaStream_t keep = h->st;
    h->st = on;
    if (check_only)
        check_tail(h);
    else if (h->mixed)
        sort_tail<float>(h);
    else
        sort_tail<double>(h);
    h->st = keep;
}

// capture one step of every reactor of the batch as one fork-join graph
// One batch step as one graph.  Reactors without an external circuit share
// their field solves: each branch runs its step up to the solve's set-up, the
// branches join, the solves of all of them run in a few cooperative launches
// (one per precision and line chunk; every reactor's blocks synchronise among
// themselves only), and the branches fork again for the rest of the step.
// Reactors with a circuit (two solves per step) run their whole step in one
// branch.  Without the shared launches (they cannot be planned), every
// reactor's step runs in its own branch.
void capture_batch(pic_batch *b, pic_batch::Graph &g) {
    const size_t nh = b->hs.size();
    g.launches.assign(nh, 0);
    std::vector<SolveJob> jobs;
    std::vector<char> shared(nh, 0);
    for (size_t k = 0; k < nh; ++k) {
        pic_handle *h = b->hs[k];
        if (h->cfg.circuit_C > 0.0) continue;
        FieldDims fd{h->nz, h->nr, h->dz, h->dr, h->cfg.mesh.L, h->cfg.chi_face};
        SolveJob j;
        if (!solve_job(fd, h->mgf, h->phi, h->mixed, h->cfg.mg_tol, h->cfg.mg_max_cycles, h->sctl, false, j))
            continue;
        jobs.push_back(j);
        shared[k] = 1;
    }
    std::vector<std::pair<int, int>> plan;
    bool concurrent = false;
    if (!jobs.empty()) {
        plan = mg_multi_plan(jobs, concurrent);
        if (!g.jobs_d && cudaMalloc(&g.jobs_d, jobs.size() * sizeof(SolveJob)) != cudaSuccess) g.jobs_d = nullptr;
        if (!g.jobs_d ||
            cudaMemcpy(g.jobs_d, jobs.data(), jobs.size() * sizeof(SolveJob), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaGetLastError();
            std::fill(shared.begin(), shared.end(), 0);
            plan.clear();
        }
    }
    if (!b->ev_fork2) cudaEventCreateWithFlags(&b->ev_fork2, cudaEventDisableTiming);
    // one part of reactor k's step, on its branch
    auto run = [&](size_t k, int part) {
        pic_handle *h = b->hs[k];
        const int64_t L0 = h->launches, P0 = h->particle_launches;
        cudaStream_t keep = h->st;
        h->st = h->gst;
        h->in_batch = true;
        SolveJob unused;
        if (h->mixed)
            one_step<float>(h, nullptr, true, part, &unused);
        else
            one_step<double>(h, nullptr, true, part, &unused);
        h->in_batch = false;
        h->st = keep;
        g.launches[k] += h->launches - L0;
        h->launches = L0;
        h->particle_launches = P0;
    };
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        std::vector<int> cur(nh), cur_i(nh);
        for (size_t k = 0; k < nh; ++k) {
            cur[k] = b->hs[k]->cur;
            cur_i[k] = b->hs[k]->cur_i;
        }
        cudaEventRecord(b->ev_fork, b->origin);
        for (size_t k = 0; k < nh; ++k) {
            cudaStreamWaitEvent(b->hs[k]->gst, b->ev_fork, 0);
            // the reactors' branches run side by side; inside a branch the
            // step stays in order (its own second branch adds nodes, not speed)
            run(k, shared[k] ? 1 : 0);
            cudaEventRecord(b->ev_join[k], b->hs[k]->gst);
            cudaStreamWaitEvent(b->origin, b->ev_join[k], 0);
        }
        if (!plan.empty()) {
            // the kinds' launches side by side (their blocks fit the GPU
            // together), each on a branch of its own; a kind's further
            // launches follow its first on the same branch
            cudaEventRecord(b->ev_fork2, b->origin);
            std::vector<char> used(nh, 0);
            std::vector<std::pair<int, int>> kinds;  // (mixed, M) in order of appearance
            for (size_t r = 0; r < plan.size(); ++r) {
                const SolveJob &j = jobs[plan[r].first];
                size_t kind = 0;
                while (kind < kinds.size() && kinds[kind] != std::make_pair(j.mixed, j.M)) ++kind;
                if (kind == kinds.size()) kinds.push_back({j.mixed, j.M});
                const size_t br = concurrent ? kind % nh : 0;
                cudaStream_t bs = b->hs[br]->gst;
                if (!used[br]) {
                    cudaStreamWaitEvent(bs, b->ev_fork2, 0);
                    used[br] = 1;
                }
                mg_multi_launch(jobs, plan[r].first, plan[r].second, g.jobs_d, bs);
            }
            for (size_t k = 0; k < nh; ++k)
                if (used[k]) {
                    cudaEventRecord(b->ev_join[k], b->hs[k]->gst);
                    cudaStreamWaitEvent(b->origin, b->ev_join[k], 0);
                }
            cudaEventRecord(b->ev_fork2, b->origin);
            for (size_t k = 0; k < nh; ++k) {
                if (!shared[k]) continue;
                cudaStreamWaitEvent(b->hs[k]->gst, b->ev_fork2, 0);
                run(k, 2);
                cudaEventRecord(b->ev_join[k], b->hs[k]->gst);
                cudaStreamWaitEvent(b->origin, b->ev_join[k], 0);
            }
        }
        for (size_t k = 0; k < nh; ++k) {  // the replays flip them
            b->hs[k]->cur = cur[k];
            b->hs[k]->cur_i = cur_i[k];
        }
        e = cudaStreamEndCapture(b->origin, &graph);
    }
    if (e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess || !g.exec) {
        g.exec = nullptr;
        g.failed = true;
        cudaGetLastError();
    }
}

void release(pic_handle *h, void *p) {
    for (size_t k = 0; k < h->allocs.size(); ++k)
        if (h->allocs[k].first == p) {
            if (h->cfg.free)
                h->cfg.free(p, h->allocs[k].second, h->cfg.alloc_ctx, (void *)h->st);
            else if (!h->cfg.alloc)
                cudaFree(p);
            h->allocs.erase(h->allocs.begin() + k);
            return;
        }
}

template <typename T>
pic_status set_particles_t(pic_handle *h, int s, const pic_particles_view *v) {
    SpecDev &d = h->sp[s];
    const int64_t n = v->n;
    if (n > d.cap) return fail(h, PIC_ERR_CAPACITY, "more particles than the species capacity");
    uint64_t mx = 0;
    for (int64_t k = 0; k < n; ++k) mx = std::max<uint64_t>(mx, v->id[k] + 1);
    double *stage = n > 0 ? (double *)dalloc(h, (size_t)n * 8 * sizeof(double)) : nullptr;
    uint64_t *sid = n > 0 ? (uint64_t *)dalloc(h, (size_t)n * sizeof(uint64_t)) : nullptr;
    const double *srcs[8] = {v->r, v->z, v->vr, v->vt, v->vz, v->ar, v->az, v->w};
    for (int f = 0; f < 8 && n > 0; ++f)
        cudaMemcpyAsync(stage + (size_t)f * n, srcs[f], (size_t)n * sizeof(double),
                        cudaMemcpyHostToDevice, h->st);
    if (n > 0) cudaMemcpyAsync(sid, v->id, (size_t)n * sizeof(uint64_t), cudaMemcpyHostToDevice, h->st);
    double *sat = nullptr;
    if (n > 0 && v->at && h->cfg.pusher == PIC_PUSH_XYZ) {
        sat = (double *)dalloc(h, (size_t)n * sizeof(double));
        cudaMemcpyAsync(sat, v->at, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, h->st);
    }
    const int c = par_of(h, s);
    launch_from_abs<T>(view<T>(d.main[c]), n, stage, stage + n, stage + 2 * n, stage + 3 * n,
                       stage + 4 * n, stage + 5 * n, stage + 6 * n, stage + 7 * n, sid, sat, h->nz, h->nr,
                       h->dz, h->dr, h->st);
    const int32_t nn = (int32_t)n, zero = 0;
    cudaMemcpyAsync(d.d_nmain[c], &nn, 4, cudaMemcpyHostToDevice, h->st);
    cudaMemcpyAsync(d.d_nbirths[c], &zero, 4, cudaMemcpyHostToDevice, h->st);
    cudaMemsetAsync(d.d_nb0, 0, sizeof(int32_t), h->st);
    cudaMemsetAsync(d.counts, 0, (size_t)h->ncell * sizeof(int32_t), h->st);
    launch_hist<T>(view<T>(d.main[c]), d.d_nmain[c], d.counts, h->st);
    launch_scan(d.counts, d.cursor, h->ncell, d.block_sums, d.d_ntotal, d.cap, h->ds, nullptr, h->st);
    launch_rank<T>(view<T>(d.main[c]), d.d_nmain[c], view<T>(d.births[c]), d.d_nbirths[c],
                   d.cursor, d.perm, d.d_ntotal, d.cap, &h->ds->status, nullptr, h->ncell, h->st);
    cudaMemcpyAsync(d.d_nalive, d.d_ntotal, 4, cudaMemcpyDeviceToDevice, h->st);
    h->launches += 6;
    d.next_id = mx;
    deposit_current<T>(h);
    cudaStreamSynchronize(h->st);
    if (stage) release(h, stage);
    if (sid) release(h, sid);
    if (sat) release(h, sat);
    push_ctl(h);
    return cuda_check(h, "set_particles");
}

template <typename T>
pic_status get_particles_t(pic_handle *h, int s, pic_particles_view *v, int64_t capacity) {
    SpecDev &d = h->sp[s];
    int32_t n = 0;
    cudaMemcpyAsync(&n, d.d_nalive, 4, cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    const int64_t m = std::min<int64_t>(n, capacity);
    v->n = m;
    if (m <= 0) return PIC_OK;
    double *stage = (double *)dalloc(h, (size_t)n * 8 * sizeof(double));
    uint64_t *sid = (uint64_t *)dalloc(h, (size_t)n * sizeof(uint64_t));
    int32_t *scell = (int32_t *)dalloc(h, (size_t)n * sizeof(int32_t));
    double *sat = v->at ? (double *)dalloc(h, (size_t)n * sizeof(double)) : nullptr;
    const int c = par_of(h, s);
    launch_to_abs<T>(view<T>(d.main[c]), view<T>(d.births[c]), d.d_nmain[c], d.perm, n, stage + n,
                     stage, stage + 2 * n, stage + 3 * n, stage + 4 * n, stage + 5 * n,
                     stage + 6 * n, stage + 7 * n, sid, scell, sat, h->nz, h->dz, h->dr, h->st);
    if (sat) cudaMemcpyAsync(v->at, sat, (size_t)m * sizeof(double), cudaMemcpyDeviceToHost, h->st);
    h->launches += 1;
    double *dsts[8] = {v->z, v->r, v->vr, v->vt, v->vz, v->ar, v->az, v->w};
    for (int f = 0; f < 8; ++f)
        if (dsts[f])
            cudaMemcpyAsync(dsts[f], stage + (size_t)f * n, (size_t)m * sizeof(double),
                            cudaMemcpyDeviceToHost, h->st);
    if (v->id) cudaMemcpyAsync(v->id, sid, (size_t)m * sizeof(uint64_t), cudaMemcpyDeviceToHost, h->st);
    if (v->cell)
        cudaMemcpyAsync(v->cell, scell, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    release(h, stage);
    release(h, sid);
    release(h, scell);
    if (sat) release(h, sat);
    return cuda_check(h, "get_particles");
}

// After the steps of a call are enqueued: the one synchronisation of the
// call, then the step control and the status word decide the outcome; the
// host copies of the step number, ids and solve statistics are refreshed,
// and on a halt the state is left at the last completed step.
void *win_alloc(void *ctx, size_t bytes) { return dalloc((pic_handle *)ctx, bytes); }
void win_release(void *ctx, void *p) { release((pic_handle *)ctx, p); }

// the collisionless window from the handle's current (sorted) particles
template <typename T>
pic_status window_t(pic_handle *h, int32_t nsteps, int32_t ckpt, const double *w, double amp0,
                    const double *phi_zL, bool grad, double *J, double *dA, double *dphi) {
    WindowIn<T> in{};
    in.nz = h->nz;
    in.nr = h->nr;
    in.dz = h->dz;
    in.dr = h->dr;
    in.L = h->cfg.mesh.L;
    in.dt = h->cfg.dt;
    in.chi_face = h->cfg.chi_face;
    in.mixed = h->mixed;
    const int cur = h->cur;
    for (int s = 0; s < 2; ++s) {
        SpecDev &d = h->sp[s];
        in.q[s] = h->cfg.sp[s].q;
        in.m[s] = h->cfg.sp[s].m;
        int32_t na = 0, nm = 0;
        cudaMemcpyAsync(&na, d.d_nalive, 4, cudaMemcpyDeviceToHost, h->st);
        cudaMemcpyAsync(&nm, d.d_nmain[cur], 4, cudaMemcpyDeviceToHost, h->st);
        cudaStreamSynchronize(h->st);
        in.n[s] = na;
        in.nmain[s] = nm;
        in.main[s] = view<T>(d.main[cur]);
        in.births[s] = view<T>(d.births[cur]);
        in.perm[s] = d.perm;
        fill_step_args<T>(h, in.args[s], s, cur, 1 - cur, 1 - cur);
    }
    in.V = h->V;
    in.phi0 = h->phi;
    in.mgf = &h->mgf;
    in.tol = h->cfg.mg_tol;
    in.max_cycles = h->cfg.mg_max_cycles;
    in.nrf = h->cfg.rf.n;
    in.rf_amp = h->own_rf.data();
    in.rf_freq = h->own_rf.data() + h->cfg.rf.n;
    in.rf_phase = h->own_rf.data() + 2 * h->cfg.rf.n;
    in.step0 = h->step;
    in.st = h->st;
    in.alloc = win_alloc;
    in.release = win_release;
    in.actx = h;
    std::vector<double> pz((size_t)h->nr, 0.0);
    if (phi_zL)
        for (int j = 0; j < h->nr; ++j) pz[j] = phi_zL[j];
    std::string err;
    const int r = window_run<T>(in, nsteps, ckpt, w, amp0, pz.data(), grad, J, dA, dphi, err);
    if (r != PIC_OK) return fail(h, (pic_status)r, err.c_str());
    return cuda_check(h, "window");
}

// After a failed call with ion subcycling: the ions as the last completed
// step left them.  A dropped pass that held them had appended its newborn
// ions to their births (cut off again); a dropped pass that moved them had
// recounted their cells.  So the counts, the permutation and the count of
// ions are rebuilt from the state, and the deposit with them.
template <typename T>
void resync_ions(pic_handle *h, bool cut_births) {
    SpecDev &d = h->sp[1];
    const int c = h->cur_i;
    if (cut_births) cudaMemcpyAsync(d.d_nbirths[c], d.d_nb0, sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
    cudaMemsetAsync(d.d_nb0, 0, sizeof(int32_t), h->st);
    cudaMemsetAsync(d.counts, 0, (size_t)h->ncell * sizeof(int32_t), h->st);
    launch_hist<T>(view<T>(d.main[c]), d.d_nmain[c], d.counts, h->st);
    launch_hist<T>(view<T>(d.births[c]), d.d_nbirths[c], d.counts, h->st);
    launch_scan(d.counts, d.cursor, h->ncell, d.block_sums, d.d_ntotal, d.cap, h->ds, nullptr, h->st);
    launch_rank<T>(view<T>(d.main[c]), d.d_nmain[c], view<T>(d.births[c]), d.d_nbirths[c], d.cursor, d.perm,
                   d.d_ntotal, d.cap, &h->ds->status, nullptr, h->ncell, h->st);
    cudaMemcpyAsync(d.d_nalive, d.d_ntotal, sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
    h->launches += 6;
}

pic_status finish_call(pic_handle *h, int64_t step0, int cur0, int cur_i0, int32_t nsteps) {
    // the one synchronisation of a call: both words into pinned memory
    if (!h->host_ctl && cudaMallocHost((void **)&h->host_ctl, sizeof(*h->host_ctl)) != cudaSuccess) {
        h->host_ctl = nullptr;
        cudaGetLastError();
    }
    StepCtl local_c;
    int32_t local_status = 0;
    StepCtl *cp = h->host_ctl ? &h->host_ctl->c : &local_c;
    int32_t *sp = h->host_ctl ? &h->host_ctl->status : &local_status;
    cudaMemcpyAsync(cp, h->sctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, h->st);
    cudaMemcpyAsync(sp, &h->ds->status, sizeof(int32_t), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    const StepCtl c = *cp;
    const int32_t status = *sp;
    pic_status ce = cuda_check(h, "step");
    if (ce != PIC_OK) return ce;
    // a failed sort ends the call at the pass it sorts, before any later failure
    const int64_t done = c.sort_fail ? c.sort_fail_step - step0 : c.halt ? c.halt_step - step0 : (int64_t)nsteps;
    h->cur = (int)(cur0 ^ (int)(done & 1));
    h->cur_i = (int)(cur_i0 ^ (int)((ion_passes_before(h, step0 + done) - ion_passes_before(h, step0)) & 1));
    h->step = step0 + done;
    h->nsamples += done;
    h->steps_total += done;
    h->sp[0].next_id = c.next_id[0];
    h->sp[1].next_id = c.next_id[1];
    h->mg_cycles_total = (int64_t)c.mg_cycles;
    h->last_cycles = c.mg_last_cycles;
    h->last_res = c.mg_last_res;
    pic_status result = PIC_OK;
    if (c.mg_flags & 1) {
        result = PIC_ERR_NOT_CONVERGED;
        h->err = "multigrid stopped before the tolerance";
        const int32_t z = 0;
        cudaMemcpyAsync(&h->sctl->mg_flags, &z, sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
    }
    if (status & ST_NAN) {
        result = PIC_ERR_NUMERIC;
        h->err = "non-finite particle state (particles dropped)";
        cudaMemsetAsync(&h->ds->status, 0, 4, h->st);
    }
    if (c.halt || c.sort_fail) {
        // the state stays at the last completed step (sorted: its sort is
        // done, the failed pass's is dropped)
        const int32_t z[3] = {0, 0, 0};
        cudaMemcpyAsync(&h->sctl->halt, z, 2 * sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
        cudaMemcpyAsync(&h->sctl->sort_pending, z, 3 * sizeof(int32_t), cudaMemcpyHostToDevice, h->st);
        cudaMemsetAsync(&h->ds->status, 0, 4, h->st);
        const int why = c.sort_fail ? c.sort_fail_status : c.halt_status;
        if (h->K > 1) {
            const bool cut = c.sort_fail && !moves_ions(h, c.sort_fail_step);
            if (h->mixed)
                resync_ions<float>(h, cut);
            else
                resync_ions<double>(h, cut);
            if (!(why & (ST_CAPACITY | ST_BIRTH_OVERFLOW))) {
                if (h->mixed)
                    deposit_current<float>(h);
                else
                    deposit_current<double>(h);
            }
        }
        if (why & (ST_CAPACITY | ST_BIRTH_OVERFLOW)) {
            if (h->mixed)
                deposit_current<float>(h);
            else
                deposit_current<double>(h);
            cudaStreamSynchronize(h->st);
            return fail(h, PIC_ERR_CAPACITY, (why & ST_CAPACITY) ? "particle capacity exceeded"
                                                                 : "births capacity exceeded");
        }
        cudaStreamSynchronize(h->st);
        return fail(h, PIC_ERR_TIMEOUT, c.sort_fail ? "births numbering: grid barrier timed out"
                                                    : "multigrid grid barrier timed out");
    }
    cudaStreamSynchronize(h->st);
    return result;
}

// Finish the last pass's deferred sort (rank, births numbering, sorted
// counts) before the particle state is read or replaced.  A failure there
// (the numbering's grid barrier timing out) drops that pass, as in a call.
pic_status complete_sort(pic_handle *h) {
    if (!h->sort_deferred) return PIC_OK;
    h->sort_deferred = false;
    enqueue_sort_tail(h, h->st);
    return finish_call(h, h->step, h->cur, h->cur_i, 0);
}

}  // namespace

extern "C" {

const char *pic_status_string(pic_status s) {
    switch (s) {
    case PIC_OK: return "ok";
    case PIC_ERR_ARG: return "invalid argument";
    case PIC_ERR_CAPACITY: return "capacity exceeded";
    case PIC_ERR_CUDA: return "CUDA error";
    case PIC_ERR_NOT_CONVERGED: return "multigrid not converged";
    case PIC_ERR_NUMERIC: return "non-finite particle state";
    case PIC_ERR_TIMEOUT: return "device wait timed out";
    case PIC_ERR_STATE: return "invalid state";
    }
    return "unknown";
}

const char *pic_last_error(const pic_handle *h) { return h ? h->err.c_str() : "null handle"; }

pic_status pic_init(const pic_config *cfg, pic_handle **out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!cfg) return PIC_ERR_ARG;
    std::string why;
    if (validate(cfg, why) != PIC_OK) {
        fprintf(stderr, "pic_init: %s\n", why.c_str());
        return PIC_ERR_ARG;
    }
    pic_handle *h = new (std::nothrow) pic_handle();
    if (!h) return PIC_ERR_ARG;
    h->cfg = *cfg;
    h->st = (cudaStream_t)cfg->stream;
    h->user_st = h->st;
    // the step's main branch at the highest priority, the sort branch at the lowest
    int least = 0, greatest = 0;
    cudaDeviceGetStreamPriorityRange(&least, &greatest);
    if (cudaStreamCreateWithPriority(&h->gst, cudaStreamNonBlocking, greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&h->gst2, cudaStreamNonBlocking, least) != cudaSuccess) {
        if (h->gst) cudaStreamDestroy(h->gst);
        h->gst = h->gst2 = nullptr;
        cudaGetLastError();
    }
    for (cudaEvent_t *e : {&h->ev_in, &h->ev_out, &h->ev_fork, &h->ev_join, &h->ev_fork2, &h->ev_join2})
        cudaEventCreateWithFlags(e, cudaEventDisableTiming);
    for (int s = 0; s < 2; ++s) {
        const pic_xsec &x = cfg->xs[s];
        h->own_sigma[s].assign(x.sigma_m2, x.sigma_m2 + (size_t)x.n_ch * x.n_e);
        h->own_thr[s].assign(x.threshold_eV, x.threshold_eV + x.n_ch);
        h->own_kind[s].assign(x.kind, x.kind + x.n_ch);
        h->cfg.xs[s].sigma_m2 = h->own_sigma[s].data();
        h->cfg.xs[s].threshold_eV = h->own_thr[s].data();
        h->cfg.xs[s].kind = h->own_kind[s].data();
    }
    h->own_rf.resize(3 * (size_t)std::max(cfg->rf.n, 0));
    for (int k = 0; k < cfg->rf.n; ++k) {
        h->own_rf[k] = cfg->rf.amp_V[k];
        h->own_rf[cfg->rf.n + k] = cfg->rf.freq_Hz[k];
        h->own_rf[2 * cfg->rf.n + k] = cfg->rf.phase_rad[k];
    }
    h->has_phiL = cfg->phi_zL != nullptr;
    if (h->has_phiL) h->own_phiL.assign(cfg->phi_zL, cfg->phi_zL + cfg->mesh.nr);
    h->cfg.phi_zL = nullptr;
    h->cfg.rf.amp_V = h->cfg.rf.freq_Hz = h->cfg.rf.phase_rad = nullptr;
    h->nz = cfg->mesh.nz;
    h->nr = cfg->mesh.nr;
    h->ncz = h->nz - 1;
    h->ncr = h->nr - 1;
    h->ncell = h->ncz * h->ncr;
    h->ng = h->nz * h->nr;
    h->dz = cfg->mesh.L / h->ncz;
    h->dr = cfg->mesh.R / h->ncr;
    h->mixed = cfg->precision == PIC_MIXED;
    h->ngas = cfg->gas.p_Pa / (kKB * cfg->gas.T_K);
    h->K = cfg->ion_subcycle > 1 ? cfg->ion_subcycle : 1;
    for (int s = 0; s < 2; ++s) {
        h->nu_max[s] = nu_max_of(h, s);
        h->p_null[s] = 1.0 - exp(-h->nu_max[s] * dt_of(h, s));
        // candidate iff (x + 1/2) 2^-32 < P_null  <=>  x < ceil(P_null 2^32 - 1/2)
        const double c = ldexp(h->p_null[s], 32) - 0.5;
        h->t_null[s] = c <= 0.0 ? 0ull : (unsigned long long)ceil(c);
    }
    try {
        setup_device(h);
        pic_status s = h->mixed ? load_all<float>(h) : load_all<double>(h);
        if (s != PIC_OK) {
            fprintf(stderr, "pic_init: %s\n", h->err.c_str());
            free_all(h);
            destroy_streams(h);
            delete h;
            return s;
        }
    } catch (const std::bad_alloc &) {
        fprintf(stderr, "pic_init: device allocation failed\n");
        free_all(h);
        destroy_streams(h);
        delete h;
        return PIC_ERR_CUDA;
    }
    *out = h;
    return PIC_OK;
}

pic_status pic_step(pic_handle *h, int32_t nsteps) {
    if (!h) return PIC_ERR_ARG;
    if (nsteps < 0) return fail(h, PIC_ERR_ARG, "nsteps < 0");
    if (nsteps == 0) return PIC_OK;
    const int64_t step0 = h->step;
    const int cur0 = h->cur, cur_i0 = h->cur_i;
    // steps run as graph replays on the private stream, ordered after the
    // caller's stream and before it again; with profiling on they launch
    // one by one on the caller's stream (phase timers)
    bool on_gst = false;
    for (int k = 0; k < nsteps; ++k) {
        const bool mv = moves_ions(h, step0 + k);
        StepGraph &g = h->graphs[h->cur + 2 * h->cur_i + (mv ? 4 : 0)];
        if (!h->prof && h->gst && !g.exec && !g.failed) {
            if (h->mixed)
                capture_step<float>(h, g, mv);
            else
                capture_step<double>(h, g, mv);
        }
        if (!h->prof && g.exec) {
            if (!on_gst) {
                cudaEventRecord(h->ev_in, h->st);
                cudaStreamWaitEvent(h->gst, h->ev_in, 0);
                on_gst = true;
            }
            cudaGraphLaunch(g.exec, h->gst);
            h->launches += g.launches;
            h->particle_launches += mv ? 2 : 1;
            h->cur ^= 1;
            if (mv) h->cur_i ^= 1;
            continue;
        }
        if (on_gst) {
            cudaEventRecord(h->ev_out, h->gst);
            cudaStreamWaitEvent(h->st, h->ev_out, 0);
            on_gst = false;
        }
        if (h->mixed)
            one_step<float>(h, nullptr, mv);
        else
            one_step<double>(h, nullptr, mv);
    }
    // the last pass's sort: its capacity check now (a failure is this
    // call's); its rank and births numbering run beside the next step's
    // solve, or before the particle state is read (complete_sort)
    enqueue_sort_tail(h, on_gst ? h->gst : h->st, true);
    if (on_gst) {
        cudaEventRecord(h->ev_out, h->gst);
        cudaStreamWaitEvent(h->st, h->ev_out, 0);
    }
    const pic_status r = finish_call(h, step0, cur0, cur_i0, nsteps);
    // a failed step leaves the state at the last completed step, sorted
    h->sort_deferred = r == PIC_OK || r == PIC_ERR_NOT_CONVERGED || r == PIC_ERR_NUMERIC;
    return r;
}

pic_status pic_tune(pic_handle *h, int32_t steps_per_variant, int32_t *variants) {
    if (!h || steps_per_variant < 0) return PIC_ERR_ARG;
    if (steps_per_variant == 0) {
        if (!variants) return fail(h, PIC_ERR_ARG, "no variants given");
        for (int s = 0; s < 2; ++s)
            if (variants[s] < -1 || variants[s] >= kStepVariants) return fail(h, PIC_ERR_ARG, "bad variant");
        h->variant[0] = variants[0];
        h->variant[1] = variants[1];
        drop_graphs(h);  // the shape is part of the captured step
        return PIC_OK;
    }
    // time every shape on real steps of this reactor (the simulation advances)
    const bool prof = h->prof;
    double best[2] = {1e300, 1e300};
    int pick[2] = {-1, -1};
    double t[kNumTiming];
    int64_t pl = 0, al = 0;
    pic_timings(h, nullptr, nullptr, nullptr, 1);
    for (int v = 0; v < kStepVariants; ++v) {
        h->variant[0] = h->variant[1] = v;
        h->prof = true;
        pic_status st = pic_step(h, steps_per_variant);
        h->prof = prof;
        if (st != PIC_OK && st != PIC_ERR_NOT_CONVERGED) return st;
        pic_timings(h, t, &pl, &al, 1);
        for (int s = 0; s < 2; ++s)
            if (t[1 + s] < best[s]) {
                best[s] = t[1 + s];
                pick[s] = v;
            }
    }
    h->variant[0] = pick[0];
    h->variant[1] = pick[1];
    drop_graphs(h);
    if (variants) {
        variants[0] = pick[0];
        variants[1] = pick[1];
    }
    return PIC_OK;
}

pic_status pic_batch_init(pic_handle *const *handles, int32_t n, void *stream, pic_batch **out) {
    if (!out) return PIC_ERR_ARG;
    *out = nullptr;
    if (!handles || n < 1) return PIC_ERR_ARG;
    for (int k = 0; k < n; ++k) {
        if (!handles[k] || !handles[k]->gst) return PIC_ERR_ARG;
        if (handles[k]->K > 1) return fail(handles[k], PIC_ERR_ARG, "batched reactors move their ions every step");
        for (int q = 0; q < k; ++q)
            if (handles[q] == handles[k]) return PIC_ERR_ARG;
    }
    pic_batch *b = new (std::nothrow) pic_batch();
    if (!b) return PIC_ERR_ARG;
    b->hs.assign(handles, handles + n);
    b->st = (cudaStream_t)stream;
    bool ok = cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
    b->ev_join.assign(n, nullptr);
    for (int k = 0; k < n && ok; ++k)
        ok = cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pic_batch_destroy(b);
        return PIC_ERR_CUDA;
    }
    *out = b;
    return PIC_OK;
}

pic_status pic_batch_step(pic_batch *b, int32_t nsteps, pic_status *statuses) {
    if (!b || nsteps < 0) return PIC_ERR_ARG;
    const size_t nh = b->hs.size();
    for (pic_handle *h : b->hs)
        if (h->prof) return fail(h, PIC_ERR_ARG, "batched steps need profiling off");
    std::vector<int64_t> step0(nh);
    std::vector<int> cur0(nh);
    for (size_t k = 0; k < nh; ++k) {
        step0[k] = b->hs[k]->step;
        cur0[k] = b->hs[k]->cur;
        // the reactor's own work so far comes first
        cudaEventRecord(b->hs[k]->ev_in, b->hs[k]->st);
        cudaStreamWaitEvent(b->origin, b->hs[k]->ev_in, 0);
    }
    cudaEventRecord(b->ev_in, b->st);
    cudaStreamWaitEvent(b->origin, b->ev_in, 0);
    for (int s = 0; s < nsteps; ++s) {
        std::vector<char> key(nh);
        for (size_t k = 0; k < nh; ++k) key[k] = (char)b->hs[k]->cur;
        pic_batch::Graph &g = b->graphs[key];
        if (!g.exec && !g.failed) capture_batch(b, g);
        if (g.exec) {
            cudaGraphLaunch(g.exec, b->origin);
            for (size_t k = 0; k < nh; ++k) {
                b->hs[k]->cur ^= 1;
                b->hs[k]->cur_i ^= 1;
                b->hs[k]->particle_launches += 2;
                b->hs[k]->launches += g.launches[k];
            }
            continue;
        }
        // no graph: the reactors' steps one after another
        for (pic_handle *h : b->hs) {
            cudaStream_t keep = h->st;
            h->st = b->origin;
            h->in_batch = true;
            if (h->mixed)
                one_step<float>(h, nullptr, true);
            else
                one_step<double>(h, nullptr, true);
            h->in_batch = false;
            h->st = keep;
        }
    }
    if (nsteps > 0) {
        // every reactor's last sort, side by side on the reactors' streams
        for (pic_handle *h : b->hs) {
            StepGraph &g = h->sort_graphs[h->cur + 2 * h->cur_i];
            if (!g.exec && !g.failed) {
                if (h->mixed)
                    capture_sort<float>(h, g, false);
                else
                    capture_sort<double>(h, g, false);
            }
        }
        cudaEventRecord(b->ev_fork, b->origin);
        for (size_t k = 0; k < nh; ++k) {
            pic_handle *h = b->hs[k];
            cudaStreamWaitEvent(h->gst, b->ev_fork, 0);
            enqueue_sort_tail(h, h->gst);
            cudaEventRecord(b->ev_join[k], h->gst);
            cudaStreamWaitEvent(b->origin, b->ev_join[k], 0);
        }
    }
    cudaEventRecord(b->ev_out, b->origin);
    cudaStreamWaitEvent(b->st, b->ev_out, 0);
    for (pic_handle *h : b->hs) cudaStreamWaitEvent(h->st, b->ev_out, 0);
    cudaStreamSynchronize(b->st);
    pic_status first = PIC_OK;
    for (size_t k = 0; k < nh; ++k) {
        const pic_status r = nsteps > 0 ? finish_call(b->hs[k], step0[k], cur0[k], cur0[k], nsteps) : PIC_OK;
        if (nsteps > 0) b->hs[k]->sort_deferred = false;  // the batch ends with the whole sort
        if (statuses) statuses[k] = r;
        if (first == PIC_OK && r != PIC_OK) first = r;
    }
    return first;
}

void pic_batch_destroy(pic_batch *b) {
    if (!b) return;
    if (b->origin) cudaStreamSynchronize(b->origin);
    for (auto &kv : b->graphs) {
        if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
        if (kv.second.jobs_d) cudaFree(kv.second.jobs_d);
    }
    if (b->ev_fork2) cudaEventDestroy(b->ev_fork2);
    for (cudaEvent_t e : b->ev_join)
        if (e) cudaEventDestroy(e);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->ev_fork) cudaEventDestroy(b->ev_fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

pic_status pic_field_solve(pic_handle *h, const double *rho, const double *chi, double V,
                           double *phi, int32_t on_device, pic_solve_info *info) {
    if (!h || !rho || !chi || !phi) return fail(h, PIC_ERR_ARG, "null argument");
    const size_t gb = (size_t)h->ng * sizeof(double);
    const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    cudaMemcpyAsync(h->tmp_grid[0], rho, gb, kin, h->st);
    cudaMemcpyAsync(h->tmp_grid[1], chi, gb, kin, h->st);
    FieldDims fd{h->nz, h->nr, h->dz, h->dr, h->cfg.mesh.L, h->cfg.chi_face};
    int L = 0;
    double res = 0.0;
    const int r = mg_fast_solve(fd, h->mgf, h->tmp_grid[0], h->tmp_grid[1], V,
                                h->has_phiL ? h->phiL_d : nullptr, h->tmp_grid[2], false,
                                h->mixed, h->cfg.mg_tol, h->cfg.mg_max_cycles, &res, &L, nullptr, h->st);
    h->launches += L;
    if (r == kSolveTimeout) return fail(h, PIC_ERR_TIMEOUT, "multigrid grid barrier timed out");
    if (r == kSolveNoLaunch) return fail(h, PIC_ERR_CUDA, "multigrid solve could not be launched");
    cudaMemcpyAsync(phi, h->tmp_grid[2], gb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    if (info) {
        info->cycles = r >= 0 ? r : -r - 1;
        info->rel_residual = res;
    }
    pic_status ce = cuda_check(h, "field_solve");
    if (ce != PIC_OK) return ce;
    return r >= 0 ? PIC_OK : PIC_ERR_NOT_CONVERGED;
}

pic_status pic_moments(pic_handle *h, pic_moments_out *out, int32_t reset) {
    if (!h || !out) return fail(h, PIC_ERR_ARG, "null argument");
    const size_t gb = (size_t)h->ng * sizeof(double);
    const double f = h->nsamples > 0 ? 1.0 / (double)h->nsamples : 0.0;
    double *dst[5] = {out->ne, out->ni, out->phi, out->Ez, out->Er};
    // host buffers: scaled on the device into a staging area, then one
    // copy per output and one synchronisation for all
    const int nb = std::max(1, h->cfg.eedf_bins);
    if (!out->on_device && !h->mom_stage) {
        try {
            h->mom_stage = (double *)dalloc(h, (5 * (size_t)h->ng + (size_t)nb) * sizeof(double));
        } catch (const std::bad_alloc &) {
            return fail(h, PIC_ERR_CUDA, "moments: staging allocation failed");
        }
    }
    for (int k = 0; k < 5; ++k) {
        if (!dst[k]) continue;
        double *to = out->on_device ? dst[k] : h->mom_stage + (size_t)k * h->ng;
        k_scale<<<(h->ng + 255) / 256, 256, 0, h->st>>>(h->m_acc[k], to, h->ng, f);
        if (!out->on_device) cudaMemcpyAsync(dst[k], to, gb, cudaMemcpyDeviceToHost, h->st);
        h->launches += 1;
    }
    if (out->eedf && h->cfg.eedf_bins > 0) {
        double *to = out->on_device ? out->eedf : h->mom_stage + 5 * (size_t)h->ng;
        k_scale<<<(h->cfg.eedf_bins + 255) / 256, 256, 0, h->st>>>(h->eedf, to, h->cfg.eedf_bins, f);
        if (!out->on_device)
            cudaMemcpyAsync(out->eedf, to, (size_t)h->cfg.eedf_bins * sizeof(double), cudaMemcpyDeviceToHost, h->st);
        h->launches += 1;
    }
    DevScalars ds;
    cudaMemcpyAsync(&ds, h->ds, sizeof(ds), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    if (out->counters) {
        for (int k = 0; k < PIC_NCOUNT; ++k) out->counters[k] = (int64_t)ds.cnt[k];
        out->counters[PIC_C_MGCYC] = h->mg_cycles_total;
        out->counters[PIC_C_STEPS] = h->steps_total;
    }
    if (out->charge)
        for (int k = 0; k < 3; ++k) out->charge[k] = ds.qabs[k];
    out->nsamples = h->nsamples;
    if (reset) {
        for (int k = 0; k < 5; ++k) cudaMemsetAsync(h->m_acc[k], 0, gb, h->st);
        cudaMemsetAsync(h->eedf, 0, (size_t)std::max(1, h->cfg.eedf_bins) * 8, h->st);
        cudaMemsetAsync(h->ds->cnt, 0, sizeof(ds.cnt), h->st);
        cudaMemsetAsync(h->ds->qabs, 0, sizeof(ds.qabs), h->st);
        h->nsamples = 0;
        h->mg_cycles_total = 0;
        cudaMemsetAsync(&h->sctl->mg_cycles, 0, sizeof(unsigned long long), h->st);
        h->steps_total = 0;
        cudaStreamSynchronize(h->st);
    }
    return cuda_check(h, "moments");
}

pic_status pic_get_particles(pic_handle *h, int32_t s, pic_particles_view *view_, int64_t capacity) {
    if (!h || !view_ || s < 0 || s > 1) return fail(h, PIC_ERR_ARG, "bad argument");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    try {
        return h->mixed ? get_particles_t<float>(h, s, view_, capacity)
                        : get_particles_t<double>(h, s, view_, capacity);
    } catch (const std::bad_alloc &) {
        return fail(h, PIC_ERR_CUDA, "staging allocation failed");
    }
}

pic_status pic_set_particles(pic_handle *h, int32_t s, const pic_particles_view *v) {
    if (!h || !v || s < 0 || s > 1 || v->n < 0) return fail(h, PIC_ERR_ARG, "bad argument");
    if (v->n > 0 && (!v->r || !v->z || !v->vr || !v->vt || !v->vz || !v->ar || !v->az || !v->w || !v->id))
        return fail(h, PIC_ERR_ARG, "null particle array");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    try {
        pic_status st = h->mixed ? set_particles_t<float>(h, s, v) : set_particles_t<double>(h, s, v);
        return st;
    } catch (const std::bad_alloc &) {
        return fail(h, PIC_ERR_CUDA, "staging allocation failed");
    }
}

pic_status pic_set_step(pic_handle *h, int64_t step) {
    if (!h || step < 0) return fail(h, PIC_ERR_ARG, "bad step");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    h->step = step;
    push_ctl(h);
    return cuda_check(h, "set_step");
}

pic_status pic_set_boundary(pic_handle *h, const double *phi_zL, int32_t on_device) {
    if (!h) return PIC_ERR_ARG;
    if (!phi_zL) {
        if (h->has_phiL) drop_graphs(h);
        h->has_phiL = false;
        return PIC_OK;
    }
    if (!h->has_phiL) drop_graphs(h);
    cudaMemcpyAsync(h->phiL_d, phi_zL, (size_t)h->nr * sizeof(double),
                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st);
    h->has_phiL = true;
    if (!on_device) cudaStreamSynchronize(h->st);
    return cuda_check(h, "set_boundary");
}

// The deposit the next step's solve takes (Sec. 2.7: with the particles
// shared among processes each deposits its own and the sums are
// all-reduced, then every process solves the same field).
pic_status pic_get_deposit(pic_handle *h, double *Ne, double *Ni, double *q, int32_t on_device) {
    if (!h) return PIC_ERR_ARG;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t gb = (size_t)h->ng * sizeof(double);
    if (Ne) cudaMemcpyAsync(Ne, h->N[0], gb, k, h->st);
    if (Ni) cudaMemcpyAsync(Ni, h->N[1], gb, k, h->st);
    if (q) cudaMemcpyAsync(q, h->ds->qstep, 3 * sizeof(double), k, h->st);
    if (!on_device) cudaStreamSynchronize(h->st);
    return cuda_check(h, "get_deposit");
}

pic_status pic_set_deposit(pic_handle *h, const double *Ne, const double *Ni, const double *q,
                           int32_t on_device) {
    if (!h) return PIC_ERR_ARG;
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t gb = (size_t)h->ng * sizeof(double);
    if (Ne) cudaMemcpyAsync(h->N[0], Ne, gb, k, h->st);
    if (Ni) cudaMemcpyAsync(h->N[1], Ni, gb, k, h->st);
    if (q) cudaMemcpyAsync(h->ds->qstep, q, 3 * sizeof(double), k, h->st);
    // host sources are the caller's: they are read before the call returns
    if (!on_device) cudaStreamSynchronize(h->st);
    return cuda_check(h, "set_deposit");
}

pic_status pic_set_id_stride(pic_handle *h, const uint64_t *next_id, uint64_t stride) {
    if (!h || !next_id || stride < 1) return fail(h, PIC_ERR_ARG, "bad id stride");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    h->sp[0].next_id = next_id[0];
    h->sp[1].next_id = next_id[1];
    push_ctl(h);
    cudaMemcpyAsync(&h->sctl->id_stride, &stride, sizeof(stride), cudaMemcpyHostToDevice, h->st);
    cudaStreamSynchronize(h->st);
    return cuda_check(h, "set_id_stride");
}

pic_status pic_get_fields(pic_handle *h, double *rho, double *chi, double *phi, double *Ez,
                          double *Er, int32_t on_device) {
    if (!h) return PIC_ERR_ARG;
    // rho and chi as the next step's solve takes them
    launch_finalize(h->N[0], h->N[1], h->V, h->cfg.sp[0].q, h->cfg.sp[1].q, chi_coef(h, 0, true),
                    chi_coef(h, 1, moves_ions(h, h->step)), h->rho, h->chi, h->ng, nullptr, h->st);
    h->launches += 1;
    const size_t gb = (size_t)h->ng * sizeof(double);
    const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    double *src[5] = {h->rho, h->chi, h->phi, h->Ez, h->Er};
    double *dst[5] = {rho, chi, phi, Ez, Er};
    for (int q = 0; q < 5; ++q)
        if (dst[q]) cudaMemcpyAsync(dst[q], src[q], gb, k, h->st);
    cudaStreamSynchronize(h->st);
    return cuda_check(h, "get_fields");
}

pic_status pic_get_counts(pic_handle *h, int64_t *n_alive, int64_t *step, uint64_t *next_id) {
    if (!h) return PIC_ERR_ARG;
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    int32_t n[2] = {0, 0};
    for (int s = 0; s < 2; ++s) cudaMemcpyAsync(&n[s], h->sp[s].d_nalive, 4, cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    if (n_alive) {
        n_alive[0] = n[0];
        n_alive[1] = n[1];
    }
    if (step) *step = h->step;
    if (next_id) {
        next_id[0] = h->sp[0].next_id;
        next_id[1] = h->sp[1].next_id;
    }
    return cuda_check(h, "get_counts");
}

pic_status pic_get_circuit(pic_handle *h, double *out) {
    if (!h || !out) return PIC_ERR_ARG;
    StepCtl c;
    cudaMemcpyAsync(&c, h->sctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    out[0] = c.circ_V;
    out[1] = c.circ_Q;
    out[2] = c.circ_Qc;
    return cuda_check(h, "get_circuit");
}

pic_status pic_window(pic_handle *h, int32_t nsteps, int32_t ckpt, const double *w, double amp0,
                      const double *phi_zL, int32_t grad, double *J, double *dJ_damp, double *dJ_dphi_zL) {
    if (!h || !w || nsteps < 1 || ckpt < 1) return fail(h, PIC_ERR_ARG, "bad window arguments");
    if (h->cfg.rf.n < 1) return fail(h, PIC_ERR_ARG, "the window needs an rf component");
    if (h->cfg.pusher != PIC_PUSH_LOCAL) return fail(h, PIC_ERR_ARG, "the window takes the local pusher");
    if (h->K > 1) return fail(h, PIC_ERR_ARG, "the window moves the ions every step (no subcycling)");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    return h->mixed ? window_t<float>(h, nsteps, ckpt, w, amp0, phi_zL, grad != 0, J, dJ_damp, dJ_dphi_zL)
                    : window_t<double>(h, nsteps, ckpt, w, amp0, phi_zL, grad != 0, J, dJ_damp, dJ_dphi_zL);
}

pic_status pic_merge(pic_handle *h, int32_t s, double frac, double dv, int64_t *pairs, double *energy_J) {
    if (!h || s < 0 || s > 1 || !(frac > 0.0) || !std::isfinite(frac) || !(dv > 0.0) || !std::isfinite(dv))
        return fail(h, PIC_ERR_ARG, "merge: species 0 or 1, frac and dv positive");
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    SpecDev &d = h->sp[s];
    const int c = par_of(h, s);
    struct Out {
        unsigned long long pairs;
        double energy;
        int overflow;
    };
    Out *o = nullptr;
    try {
        o = (Out *)dalloc(h, sizeof(Out));
    } catch (const std::bad_alloc &) {
        return fail(h, PIC_ERR_CUDA, "merge: allocation failed");
    }
    cudaMemsetAsync(o, 0, sizeof(Out), h->st);
    // the cells' ends in the permutation of the sorted store: recount, scan
    // and rank (the same order the store already has)
    auto resort = [&](auto tag) {
        using T = decltype(tag);
        cudaMemsetAsync(d.counts, 0, (size_t)h->ncell * sizeof(int32_t), h->st);
        launch_hist<T>(view<T>(d.main[c]), d.d_nmain[c], d.counts, h->st);
        launch_hist<T>(view<T>(d.births[c]), d.d_nbirths[c], d.counts, h->st);
        launch_scan(d.counts, d.cursor, h->ncell, d.block_sums, d.d_ntotal, d.cap, h->ds, nullptr, h->st);
        launch_rank<T>(view<T>(d.main[c]), d.d_nmain[c], view<T>(d.births[c]), d.d_nbirths[c], d.cursor, d.perm,
                       d.d_ntotal, d.cap, &h->ds->status, nullptr, h->ncell, h->st);
        cudaMemcpyAsync(d.d_nalive, d.d_ntotal, sizeof(int32_t), cudaMemcpyDeviceToDevice, h->st);
        h->launches += 6;
    };
    auto run = [&](auto tag) {
        using T = decltype(tag);
        resort(tag);
        launch_merge<T>(view<T>(d.main[c]), view<T>(d.births[c]), d.d_nmain[c], d.perm, d.cursor, h->ncell, h->ncz,
                        h->dz, h->dr, (const T *)d.w_ref, frac, dv, h->cfg.sp[s].m,
                        h->cfg.pusher == PIC_PUSH_XYZ ? 1 : 0, &o->pairs, &o->energy, &o->overflow, h->st);
        h->launches += 1;
        resort(tag);  // drops the merged-away records
        deposit_current<T>(h);
    };
    if (h->mixed)
        run(0.0f);
    else
        run(0.0);
    Out out;
    cudaMemcpyAsync(&out, o, sizeof(Out), cudaMemcpyDeviceToHost, h->st);
    cudaStreamSynchronize(h->st);
    release(h, o);
    if (pairs) *pairs = (int64_t)out.pairs;
    if (energy_J) *energy_J = out.energy;
    const pic_status ce = cuda_check(h, "merge");
    if (ce != PIC_OK) return ce;
    if (out.overflow) return fail(h, PIC_ERR_CAPACITY, "merge: a cell held more light particles than one block takes");
    return PIC_OK;
}

static const uint64_t kCkptMagic = 0x50494352475a3032ull;  // "PICRGZ02"

pic_status pic_save(pic_handle *h, const char *path) {
    if (!h || !path) return PIC_ERR_ARG;
    const pic_status cs = complete_sort(h);
    if (cs != PIC_OK) return cs;
    FILE *f = fopen(path, "wb");
    if (!f) return fail(h, PIC_ERR_ARG, "cannot open checkpoint for writing");
    const int circuit = h->cfg.circuit_C > 0.0 ? 1 : 0;
    const int xyz = h->cfg.pusher == PIC_PUSH_XYZ ? 1 : 0;
    int64_t hdr[8] = {(int64_t)kCkptMagic, h->nz, h->nr, h->step, h->mixed ? 1 : 0, circuit, xyz,
                      h->K > 1 ? h->K : 0};
    uint64_t ids[2] = {h->sp[0].next_id, h->sp[1].next_id};
    fwrite(hdr, sizeof(hdr), 1, f);
    fwrite(ids, sizeof(ids), 1, f);
    std::vector<double> g((size_t)h->ng);
    for (double *src : {h->phi, h->phi_prev, h->N[0], h->N[1]}) {
        cudaMemcpy(g.data(), src, g.size() * 8, cudaMemcpyDeviceToHost);
        fwrite(g.data(), 8, g.size(), f);
    }
    pic_status st = PIC_OK;
    for (int s = 0; s < 2 && st == PIC_OK; ++s) {
        int64_t n = 0;
        int32_t n32 = 0;
        cudaMemcpy(&n32, h->sp[s].d_nalive, 4, cudaMemcpyDeviceToHost);
        n = n32;
        std::vector<double> a((size_t)std::max<int64_t>(n, 1) * 9);
        std::vector<uint64_t> id((size_t)std::max<int64_t>(n, 1));
        pic_particles_view v;
        v.n = n;
        v.r = a.data();
        v.z = a.data() + n;
        v.vr = a.data() + 2 * n;
        v.vt = a.data() + 3 * n;
        v.vz = a.data() + 4 * n;
        v.ar = a.data() + 5 * n;
        v.az = a.data() + 6 * n;
        v.w = a.data() + 7 * n;
        v.id = id.data();
        v.cell = nullptr;
        v.at = xyz ? a.data() + 8 * n : nullptr;
        st = pic_get_particles(h, s, &v, n);
        fwrite(&n, 8, 1, f);
        fwrite(a.data(), 8, (size_t)n * 8, f);
        fwrite(id.data(), 8, (size_t)n, f);
        if (xyz) fwrite(a.data() + 8 * n, 8, (size_t)n, f);
    }
    if (circuit && st == PIC_OK) {
        // circuit state, the charge collected since the last circuit solve,
        // and the two superposition parts (the next solves start from them)
        double cs[6];
        pic_get_circuit(h, cs);
        cudaMemcpy(cs + 3, h->ds->qstep, 3 * sizeof(double), cudaMemcpyDeviceToHost);
        fwrite(cs, 8, 6, f);
        for (double *src : {h->phi_P, h->phi_L}) {
            cudaMemcpy(g.data(), src, g.size() * 8, cudaMemcpyDeviceToHost);
            fwrite(g.data(), 8, g.size(), f);
        }
    }
    fclose(f);
    return st;
}

pic_status pic_load(pic_handle *h, const char *path) {
    if (!h || !path) return PIC_ERR_ARG;
    const pic_status pending = complete_sort(h);
    if (pending != PIC_OK) return pending;
    FILE *f = fopen(path, "rb");
    if (!f) return fail(h, PIC_ERR_ARG, "cannot open checkpoint");
    int64_t hdr[8];
    uint64_t ids[2];
    const int circuit = h->cfg.circuit_C > 0.0 ? 1 : 0;
    const int xyz = h->cfg.pusher == PIC_PUSH_XYZ ? 1 : 0;
    if (fread(hdr, sizeof(hdr), 1, f) != 1 || (uint64_t)hdr[0] != kCkptMagic || hdr[1] != h->nz ||
        hdr[2] != h->nr || hdr[5] != circuit || hdr[6] != xyz || hdr[7] != (h->K > 1 ? h->K : 0) ||
        fread(ids, sizeof(ids), 1, f) != 1) {
        fclose(f);
        return fail(h, PIC_ERR_ARG, "checkpoint does not match this handle");
    }
    std::vector<double> g((size_t)h->ng), gp((size_t)h->ng), N0((size_t)h->ng), N1((size_t)h->ng);
    bool ok = fread(g.data(), 8, g.size(), f) == g.size() && fread(gp.data(), 8, gp.size(), f) == gp.size() &&
              fread(N0.data(), 8, N0.size(), f) == N0.size() && fread(N1.data(), 8, N1.size(), f) == N1.size();
    pic_status st = ok ? PIC_OK : fail(h, PIC_ERR_ARG, "truncated checkpoint");
    for (int s = 0; s < 2 && st == PIC_OK; ++s) {
        int64_t n = 0;
        if (fread(&n, 8, 1, f) != 1 || n < 0 || n > h->sp[s].cap) {
            st = fail(h, PIC_ERR_ARG, "bad particle count in checkpoint");
            break;
        }
        std::vector<double> a((size_t)std::max<int64_t>(n, 1) * 9);
        std::vector<uint64_t> id((size_t)std::max<int64_t>(n, 1));
        if (fread(a.data(), 8, (size_t)n * 8, f) != (size_t)n * 8 || fread(id.data(), 8, (size_t)n, f) != (size_t)n ||
            (xyz && fread(a.data() + 8 * n, 8, (size_t)n, f) != (size_t)n)) {
            st = fail(h, PIC_ERR_ARG, "truncated checkpoint");
            break;
        }
        pic_particles_view v;
        v.n = n;
        v.r = a.data();
        v.z = a.data() + n;
        v.vr = a.data() + 2 * n;
        v.vt = a.data() + 3 * n;
        v.vz = a.data() + 4 * n;
        v.ar = a.data() + 5 * n;
        v.az = a.data() + 6 * n;
        v.w = a.data() + 7 * n;
        v.id = id.data();
        v.cell = nullptr;
        v.at = xyz ? a.data() + 8 * n : nullptr;
        st = pic_set_particles(h, s, &v);
    }
    double cs[6] = {0, 0, 0, 0, 0, 0};
    std::vector<double> gP, gL;
    if (circuit && st == PIC_OK) {
        gP.resize((size_t)h->ng);
        gL.resize((size_t)h->ng);
        if (fread(cs, 8, 6, f) != 6 || fread(gP.data(), 8, gP.size(), f) != gP.size() ||
            fread(gL.data(), 8, gL.size(), f) != gL.size())
            st = fail(h, PIC_ERR_ARG, "truncated checkpoint");
    }
    fclose(f);
    if (st != PIC_OK) return st;
    if (circuit) {
        StepCtl c;
        cudaMemcpy(&c, h->sctl, sizeof(StepCtl), cudaMemcpyDeviceToHost);
        c.circ_V = cs[0];
        c.circ_Q = cs[1];
        c.circ_Qc = cs[2];
        cudaMemcpy(h->sctl, &c, sizeof(StepCtl), cudaMemcpyHostToDevice);
        cudaMemcpy(h->ds->qstep, cs + 3, 3 * sizeof(double), cudaMemcpyHostToDevice);
        cudaMemcpy(h->phi_P, gP.data(), gP.size() * 8, cudaMemcpyHostToDevice);
        cudaMemcpy(h->phi_L, gL.data(), gL.size() * 8, cudaMemcpyHostToDevice);
    }
    h->step = hdr[3];
    h->sp[0].next_id = ids[0];
    h->sp[1].next_id = ids[1];
    push_ctl(h);
    cudaMemcpy(h->phi, g.data(), g.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(h->phi_prev, gp.data(), gp.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(h->N[0], N0.data(), N0.size() * 8, cudaMemcpyHostToDevice);
    cudaMemcpy(h->N[1], N1.data(), N1.size() * 8, cudaMemcpyHostToDevice);
    return cuda_check(h, "load");
}

pic_status pic_profile(pic_handle *h, int32_t on) {
    if (!h) return PIC_ERR_ARG;
    h->prof = on != 0;
    return PIC_OK;
}

pic_status pic_timings(pic_handle *h, double *ms, int64_t *particle_launches, int64_t *all_launches,
                       int32_t reset) {
    if (!h) return PIC_ERR_ARG;
    resolve_events(h);
    if (ms)
        for (int k = 0; k < kNumTiming; ++k) ms[k] = h->t_ms[k];
    if (particle_launches) *particle_launches = h->particle_launches;
    if (all_launches) *all_launches = h->launches;
    if (reset) {
        for (int k = 0; k < kNumTiming; ++k) h->t_ms[k] = 0.0;
        h->particle_launches = 0;
        h->launches = 0;
    }
    return PIC_OK;
}

pic_status pic_selftest_wait(int64_t polls, int32_t *gave_up) {
    if (!gave_up || polls < 256 || polls > kSpinLimit) return PIC_ERR_ARG;
    int g = 0;
    if (wait_selftest((long long)polls, &g) != 0) {
        cudaGetLastError();
        return PIC_ERR_CUDA;
    }
    *gave_up = g;
    return cudaGetLastError() == cudaSuccess ? PIC_OK : PIC_ERR_CUDA;
}

void pic_destroy(pic_handle *h) {
    if (!h) return;
    cudaStreamSynchronize(h->st);
    if (h->gst) cudaStreamSynchronize(h->gst);
    resolve_events(h);
    for (auto e : h->ev_pool) cudaEventDestroy(e);
    destroy_streams(h);
    free_all(h);
    if (h->host_ctl) cudaFreeHost(h->host_ctl);
    delete h;
}

}  // extern "C"
