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

// Shared-memory layout of the one-launch solve (byte offsets), set on the host.
struct SolveLayout {
    int offBuf;  // three line buffers (right-hand side in, solution out), M * 33 values of 8 bytes each
    int offW;    // the black line's two coupling coefficients, 32 M values of 8 bytes each
    int offF;    // factors of the two red lines and the black line; the residual tile lies over them
    int offC;    // factors of the coarsest row (FP64)
    int tw;      // columns per residual tile
};

// One reactor's one-launch solve, as the kernel takes it (a table of these
// drives the solves of several reactors in one cooperative launch), with its
// launch shape on the host.
struct SolveJob {
    const MGFast *mp;
    double *phi;
    int nr, first_cycle;
    SolveLayout lay;
    double tol;
    int max_cycles;
    const StepCtl *sctl;
    int block0, nblocks;  // this job's blocks in the launch
    // host side
    int M, mixed, minb;
    size_t smem;
    void *fn;
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
// defer (narrow solves of a batch): the set-up is enqueued, the solve itself
// is described in *defer and left to mg_multi_launch; its end (the report to
// sctl) is then mg_solve_done's.
// phi_prev (warm solves only, optional): the potential of the step before
// phi's; the V-cycles then start from 2 phi - phi_prev on the interior, and
// phi_prev takes phi's values (the starting value w_0 of Algorithm 1,
// extrapolated linearly in time).
int mg_fast_solve(const FieldDims &fd, MGFast &m, const double *rho, const double *chi, double V,
                  const double *phi_zL, double *phi, bool warm, bool mixed, double tol,
                  int max_cycles, double *rel_res, int *launches, StepCtl *sctl, cudaStream_t st,
                  bool v_from_ctl = true, bool setup = true, cudaEvent_t at_solve = nullptr,
                  bool wide = true, SolveJob *defer = nullptr, double *phi_prev = nullptr);

// the launch shape of one reactor's solve (host only); false: not launchable
bool solve_job(const FieldDims &fd, MGFast &m, double *phi, bool mixed, double tol, int max_cycles,
               const StepCtl *sctl, bool wide, SolveJob &job);

// Plan deferred solves for shared cooperative launches: jobs of one (precision,
// line chunk) kind share a launch; each kind gets SMs in proportion to the
// blocks its jobs would take alone, and each job's blocks are cut in
// proportion so that the launches of all kinds fit the GPU together (at
// least one block per job; a kind with more jobs than its share takes
// several launches).  concurrent (out): the kinds' launches fit side by side;
// else each takes the whole GPU and they run one after another.
// Returns the launches as [first job, end job) ranges of `jobs`, which it
// reorders by kind and fills with block0 / nblocks.  Host only.
std::vector<std::pair<int, int>> mg_multi_plan(std::vector<SolveJob> &jobs, bool &concurrent);
// launch the planned range [j0, j1) of the device copy of the table
int mg_multi_launch(const std::vector<SolveJob> &jobs, int j0, int j1, const SolveJob *jobs_dev,
                    cudaStream_t st);
// a deferred solve's report to its step control (k_solve_done)
void mg_solve_done(MGFast &m, StepCtl *sctl, bool first_of_step, cudaStream_t st);

}  // namespace pic
