// window.cuh -- the collisionless window of the timestep and its adjoint
// (window.cu): the state it works on and what it takes from a handle.
#pragma once

#include <string>

#include "pic_internal.cuh"

namespace pic {

struct MGFast;

// slot-stable particle state of one species (cell -1: left the domain)
template <typename T>
struct WinState {
    typename V4<T>::type *q0, *q1;
    int32_t *cell;
};

// adjoint of a species' state (FP64, per absolute coordinate), SoA
struct WinAdj {
    double *z, *r, *vr, *vt, *vz, *ar, *az;
};

template <typename T>
struct WindowIn {
    int nz, nr;
    double dz, dr, L, dt;
    int chi_face;
    bool mixed;
    double q[2], m[2];
    int n[2];                 // particles per species at the start
    PBuf<T> main[2], births[2];
    const int32_t *perm[2];   // the sorted store's permutation
    int nmain[2];
    StepArgs<T> args[2];      // the production pass's constants per species
    const double *V;          // node volumes
    const double *phi0;       // the first solve's start
    MGFast *mgf;
    double tol;
    int max_cycles;
    int nrf;
    const double *rf_amp, *rf_freq, *rf_phase;  // host
    int64_t step0;            // step index at the start
    cudaStream_t st;
    void *(*alloc)(void *ctx, size_t bytes);   // throws when out of memory
    void (*release)(void *ctx, void *p);
    void *actx;
};

// J over K steps from the handle's particles; with grad, dJ/d amp0 and
// dJ/d phi_zL (nr values) as well.  Returns a pic_status.
template <typename T>
int window_run(const WindowIn<T> &in, int K, int ckpt, const double *w_host, double amp0,
               const double *phizL_host, bool grad, double *J, double *dA, double *dphizL, std::string &err);

}  // namespace pic
