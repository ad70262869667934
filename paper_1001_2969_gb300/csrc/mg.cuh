// mg.cuh -- workspace and control block of the multigrid solve in mg.cu.
#pragma once

#include <vector>

#include "pic_internal.cuh"

namespace pic {

// device-side control of one solve (the one-launch V-cycles)
struct MGCtl {
    unsigned long long b_bits;  // max |b| (first cycle), bits of a positive double
    unsigned long long rb[2];   // per-cycle max |r| (alternating)
    int converged, zero_rhs, cycles, timeout;
    double last_res, bnorm;
    // barrier counters of the one-launch solve (whole grid; the coarse
    // levels' group of blocks), each on its own cache line
    struct alignas(128) Line {
        unsigned int v;
        unsigned int pad[31];
    };
    Line bar_count;
    Line gbar_count;
};

// returned by mg_fast_solve when a bounded device wait gave up, and when
// the one-launch solve cannot be launched (shared memory, co-residency)
constexpr int kSolveTimeout = -1000000;
constexpr int kSolveNoLaunch = -1000001;

constexpr int kMaxLevels = 16;

struct MGFast;
struct MGFast {
    int nlev;
    int nz[kMaxLevels];
    double dz[kMaxLevels];
    double *chi[kMaxLevels], *cz[kMaxLevels], *cr[kMaxLevels];
    float *cz32[kMaxLevels], *cr32[kMaxLevels];
    // face geometry per level, by column j (filled once by mg_fast_geometry):
    // gz = pi (r_{j+1/2}^2 - r_{j-1/2}^2) / dz_l, gr = 2 pi r_{j+1/2} dz_l / dr;
    // ga = pi (r_{j+1/2}^2 - r_{j-1/2}^2) dz / eps0 (level 0's right-hand side)
    double *gz[kMaxLevels], *gr[kMaxLevels];
    double *ga;
    // V-cycle correction and right-hand side per level (level 0: the
    // correction of phi and the residual), FP64 path / FP32 (mixed) path
    double *u64[kMaxLevels], *f64[kMaxLevels];
    float *u32[kMaxLevels], *f32[kMaxLevels];
    double *fac64[kMaxLevels];                  // line factors, FP64 path
    float *fac32[kMaxLevels];                   // line factors, FP32 V-cycle
    double *facc;                               // coarsest level's line factors (FP64)
    float *facc32;                              // coarsest level's line factors, FP32 V-cycle
    double *fc64;                               // coarsest level's right-hand side
    double *f0;                                 // fine right-hand side
    double *dg0;                                // fine operator's diagonal
    double *phi2;                               // second copy of phi (the solve alternates)
    // flexible GCR(1) of the mixed path (null on the FP64 path): the FP64
    // residual, A z of the last correction z, the previous direction and
    // its A-image, and per-block partial dot products (4 per block)
    double *kr, *kw, *kzp, *kwp, *kpart;
    MGCtl *ctl;
    MGFast *self;  // device copy of this struct (kernels read it through a pointer)
};

// line-factor elements of one r-line of a mesh with nr nodes per row
// (the same count in FP32 and FP64)
size_t mg_line_factor_elems(int nr);

// copy the level table to the device (once: its pointers do not change)
void mg_fast_upload(MGFast &m, cudaStream_t st);
// host values of gz, gr (every level) and ga, laid out [gz_0 gr_0 gz_1 gr_1 ... ga]
// with nr entries each; the caller copies them to one device array
void mg_fast_geometry(const MGFast &m, int nr, double dr, std::vector<double> &out);

// Solve into phi.  Alone (sctl null): returns the cycles (>= 0, converged)
// or -cycles-1, after a host synchronisation.  Inside a timestep (sctl set):
// enqueues the work only, takes the voltage from sctl->V (v_from_ctl), skips everything
// once sctl->halt is set, reports cycles, residual and failures to sctl, and
// returns 0 (or kSolveNoLaunch).  at_solve (optional) is recorded on st just
// before the one-launch solve, after the set-up: work that waits for it runs
// beside the solve.  wide: two blocks per black line (a reactor alone on the
// GPU); else one (many reactors solving side by side).
int mg_fast_solve(const FieldDims &fd, MGFast &m, const double *rho, const double *chi, double V,
                  const double *phi_zL, double *phi, bool warm, bool mixed, double tol,
                  int max_cycles, double *rel_res, int *launches, StepCtl *sctl, cudaStream_t st,
                  bool v_from_ctl = true, bool setup = true, cudaEvent_t at_solve = nullptr,
                  bool wide = true);

}  // namespace pic
