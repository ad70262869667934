// mg.cuh -- workspace and control block of the multigrid solve in mg.cu.
#pragma once

#include "pic_internal.cuh"

namespace pic {

// device-side control of one solve: the residual kernel's last block fills
// it and raises `done`; the other kernels of a cycle return early once done
struct MGCtl {
    unsigned long long res_bits;  // max |r| of the current cycle (bits of a positive double)
    unsigned long long b_bits;    // max |b| (first cycle)
    unsigned long long rb[2];     // per-cycle max |r| of the one-launch solve (alternating)
    unsigned int blocks_in;
    int done, converged, zero_rhs, cycles, max_cycles, timeout;
    double tol, last_res, bnorm;
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
    MGCtl *ctl;
    MGFast *self;  // device copy of this struct (kernels read it through a pointer)
};

// line-factor elements of one r-line of a mesh with nr nodes per row
// (the same count in FP32 and FP64)
size_t mg_line_factor_elems(int nr);

// solve into phi; returns the cycles (>= 0, converged) or -cycles-1
int mg_fast_solve(const FieldDims &fd, MGFast &m, const double *rho, const double *chi, double V,
                  const double *phi_zL, double *phi, bool warm, bool mixed, double tol,
                  int max_cycles, double *rel_res, int *launches, cudaStream_t st);

}  // namespace pic
