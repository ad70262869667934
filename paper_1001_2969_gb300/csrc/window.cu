// window.cu -- the collisionless window of the r-z timestep (Wang, Jiang &
// Wang, arXiv:1001.2969: Sec. 2.1 merged cycle with the Monte Carlo step
// off) and its hand-written adjoint: the gradient of
//   J = (1/K) sum_{n=1..K} sum_k w_k N_i^n(k)
// (the time average of the volume integral of w n_i, N_i^n the ion deposit
// after step n) with respect to the amplitude of the first rf component and
// the potentials of the z = L row.
//
// Forward: the production particle arithmetic (pmath.cuh) without collisions,
// births, splitting or sorting; particles keep their slot for the whole
// window (a particle that reaches a wall gets cell -1 and stays), so the
// adjoint of step n maps slot to slot.  Field: finalize, the one-launch
// multigrid solve, E.  The forward keeps a checkpoint of the particles every
// `ckpt` steps; the backward recomputes one segment at a time from its
// checkpoint, keeping the segment's states and fields, and runs the reverse
// of each step (each particle's Jacobian in the forward's precision, every
// adjoint stored and accumulated in FP64):
//   particles: deposit at x~^n, first push (rotation), final push (axis
//     reflection), gather of E at x~^{n-1}  ->  particle adjoints of step
//     n-1 and the adjoint of E on the mesh;
//   field: adjoint of E = -grad phi, the adjoint solve A(chi) lambda =
//     phi_bar on the interior (the finite-volume operator is symmetric, so
//     the same multigrid solves it), then rho_bar = lambda f'(rho),
//     chi_bar = -sum over faces (lambda_a - lambda_b)(phi_a - phi_b) G_f to
//     the face's max node, N_bar = (q rho_bar + c chi_bar)/V, and the
//     boundary rows' adjoints: phi_bar_B + sum c_IB lambda_I.
// Non-differentiable points take the conventions of the oracle's autograd
// reference: cells piecewise constant, |.| at the axis with sign(.), frozen
// particles drop out, max(chi_lo, chi_hi) passes to chi_lo iff chi_lo >
// chi_hi.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "mg.cuh"
#include "pmath.cuh"
#include "window.cuh"

namespace pic {

namespace {

constexpr int kWT = 256;

// z-face area of the control volume of radial node j
__device__ __forceinline__ double area_z(int j, double dr) {
    const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
    return kPi * (rp * rp - rm * rm);
}

template <typename T>
__device__ __forceinline__ void load_w(const WinState<T> &s, int k, PS<T> &p, int ncz, float inv_ncz, int &cell) {
    ld4(s.q0 + k, p.oz, p.orr, p.vr, p.vt);
    ld4(s.q1 + k, p.vz, p.ar, p.az, p.w);
    cell = s.cell[k];
    if (cell >= 0) decode_cell(cell, ncz, inv_ncz, p.i, p.j);
}

template <typename T>
__device__ __forceinline__ void store_w(const WinState<T> &s, int k, const PS<T> &p, int cell) {
    st4(s.q0 + k, p.oz, p.orr, p.vr, p.vt);
    st4(s.q1 + k, p.vz, p.ar, p.az, p.w);
    s.cell[k] = cell;
}

// shape factors and their derivatives per unit length (inv_dz = 1/dz,
// inv_dr = 1/dr)
template <typename A>
__device__ __forceinline__ void shapes(int weighting, int j, A oz, A orr, A inv_dz, A inv_dr, A sz[2], A sr[2],
                                       A dsz[2], A dsr[2]) {
    sz[1] = oz;
    sz[0] = (A)1 - oz;
    dsz[1] = inv_dz;
    dsz[0] = -inv_dz;
    if (weighting == PIC_WEIGHT_ZR) {
        sr[1] = orr;
        dsr[1] = inv_dr;
    } else {
        const A it = (A)1 / (A)(2 * j + 1);
        sr[1] = orr * ((A)(2 * j) + orr) * it;
        dsr[1] = ((A)(2 * j) + (A)2 * orr) * it * inv_dr;
    }
    sr[0] = (A)1 - sr[1];
    dsr[0] = -dsr[1];
}

// ---- the sorted store -> slot-stable window state ----
template <typename T>
__global__ void k_win_init(PBuf<T> main, PBuf<T> births, const int32_t *perm, int nmain, int n,
                           WinState<T> dst) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int pidx = perm[k];
    const PBuf<T> &src = pidx < nmain ? main : births;
    const int si = pidx < nmain ? pidx : pidx - nmain;
    dst.q0[k] = src.q0[si];
    dst.q1[k] = src.q1[si];
    dst.cell[k] = src.cell[si];
}

// deposit of a state (alive particles) into N (FP64)
template <typename T>
__global__ void k_win_deposit(WinState<T> s, int n, int ncz, float inv_ncz, int nr, int weighting, double *N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    PS<T> p;
    int cell;
    load_w(s, k, p, ncz, inv_ncz, cell);
    if (cell < 0) return;
    T s0, s1;
    shape_r(weighting, p.j, p.orr, s0, s1);
    const T z0 = (T)1 - p.oz, z1 = p.oz;
    double *g = N + (size_t)p.i * nr + p.j;
    atomicAdd(g, (double)(p.w * z0 * s0));
    atomicAdd(g + 1, (double)(p.w * z0 * s1));
    atomicAdd(g + nr, (double)(p.w * z1 * s0));
    atomicAdd(g + nr + 1, (double)(p.w * z1 * s1));
}

// ---- forward step of one species: the production pass without the Monte
// Carlo step (gather, final push, axis, walls, first push, walls, deposit)
template <typename T>
__global__ void k_win_push(StepArgs<T> a, WinState<T> in, WinState<T> out, int n, double *N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    PS<T> p;
    int cell;
    load_w(in, k, p, a.ncz, a.inv_ncz, cell);
    if (cell < 0) {
        store_w(out, k, p, -1);
        return;
    }
    const PS<T> p0 = p;
    T s0, s1;
    shape_r(a.weighting, p.j, p.orr, s0, s1);
    const T z0 = (T)1 - p.oz, z1 = p.oz;
    const auto *Ep = a.E + (size_t)p.i * a.nr + p.j;
    const auto e00 = Ep[0], e01 = Ep[1], e10 = Ep[a.nr], e11 = Ep[a.nr + 1];
    const T Ez = z0 * (s0 * e00.x + s1 * e01.x) + z1 * (s0 * e10.x + s1 * e11.x);
    const T Er = z0 * (s0 * e00.y + s1 * e01.y) + z1 * (s0 * e10.y + s1 * e11.y);
    p.oz += a.kz * Ez;
    carry(p.oz, p.i);
    const T ro = p.orr + a.kr * Er;
    const T fl = m_floor(ro);
    int jn = p.j + (int)fl;
    bool axis = false;
    if (jn < 0) {
        const T rr = -((T)p.j + ro);
        const T f2 = m_floor(rr);
        jn = (int)f2;
        p.orr = rr - f2;
        axis = true;
    } else {
        p.orr = ro - fl;
    }
    p.j = jn;
    p.vz += a.kv * Ez;
    p.vr += a.kv * Er;
    p.az = (T)0.5 * (a.ka * Ez + p.az);
    p.ar = (T)0.5 * (a.ka * Er + p.ar);
    if (axis) {
        p.vr = m_abs(p.vr);
        p.ar = m_abs(p.ar);
    }
    if (wall_of(p.i, p.oz, p.j, a.nz, a.nr) >= 0) {
        store_w(out, k, p0, -1);  // left: frozen
        return;
    }
    first_push(a, p);
    if (wall_of(p.i, p.oz, p.j, a.nz, a.nr) >= 0) {
        store_w(out, k, p0, -1);
        return;
    }
    const int oc = p.j * a.ncz + p.i;
    store_w(out, k, p, oc);
    T r0, r1;
    shape_r(a.weighting, p.j, p.orr, r0, r1);
    const T y0 = (T)1 - p.oz, y1 = p.oz;
    double *g = N + (size_t)p.i * a.nr + p.j;
    atomicAdd(g, (double)(p.w * y0 * r0));
    atomicAdd(g + 1, (double)(p.w * y0 * r1));
    atomicAdd(g + a.nr, (double)(p.w * y1 * r0));
    atomicAdd(g + a.nr + 1, (double)(p.w * y1 * r1));
}

// J += scale * sum_k w_k N_k (one block per 256 x 8 nodes)
__global__ void k_win_J(const double *N, const double *w, int ng, double scale, double *J) {
    __shared__ double red[kWT / 32];
    double v = 0.0;
    for (int k = blockIdx.x * blockDim.x * 8 + threadIdx.x; k < min(ng, (blockIdx.x + 1) * blockDim.x * 8);
         k += blockDim.x)
        v += w[k] * N[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int q = 0; q < kWT / 32; ++q) t += red[q];
        atomicAdd(J, scale * t);
    }
}

// ---- reverse of one step of one species ----
// prev: the state before the step (x~^{n-1}), cur: after it (x~^n);
// bin: adjoint of cur (read), bout: adjoint of prev (written);
// Nb: adjoint of this species' deposit N^n; Eb: adjoint of E^n (added to).
// The step's Jacobian is taken in the forward's precision T (the forward
// ran in it); the adjoints are stored and accumulated in FP64.
template <typename T>
__global__ void k_win_back(StepArgs<T> a, WinState<T> prev, WinState<T> cur, int n, const double *Nb,
                           WinAdj bin, WinAdj bout, double *Ebz, double *Ebr, T dr, T inv_dz, T inv_dr, T qm,
                           T dt) {
    using A = T;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    PS<T> p, q;
    int c0, c1;
    load_w(prev, k, p, a.ncz, a.inv_ncz, c0);
    load_w(cur, k, q, a.ncz, a.inv_ncz, c1);
    if (c0 < 0 || c1 < 0) {  // gone before or during the step: no part in J
        bout.z[k] = bout.r[k] = bout.vr[k] = bout.vt[k] = bout.vz[k] = bout.ar[k] = bout.az[k] = 0.0;
        return;
    }
    const int nr = a.nr;
    // adjoint of x~^n: the state's own plus its deposit
    A zb2 = (A)bin.z[k], rb2 = (A)bin.r[k];
    {
        A sz[2], sr[2], dsz[2], dsr[2];
        shapes<A>(a.weighting, q.j, q.oz, q.orr, inv_dz, inv_dr, sz, sr, dsz, dsr);
        const double *g = Nb + (size_t)q.i * nr + q.j;
        const A nb[2][2] = {{(A)g[0], (A)g[1]}, {(A)g[nr], (A)g[nr + 1]}};
        A az_ = 0, ar_ = 0;
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
            for (int v = 0; v < 2; ++v) {
                az_ += dsz[u] * sr[v] * nb[u][v];
                ar_ += sz[u] * dsr[v] * nb[u][v];
            }
        zb2 += q.w * az_;
        rb2 += q.w * ar_;
    }
    const A vrb2 = (A)bin.vr[k], vtb2 = (A)bin.vt[k], vzb2 = (A)bin.vz[k], arb2 = (A)bin.ar[k],
            azb2 = (A)bin.az[k];
    // the step's forward again, from x~^{n-1}
    A sz[2], sr[2], dsz[2], dsr[2];
    shapes<A>(a.weighting, p.j, p.oz, p.orr, inv_dz, inv_dr, sz, sr, dsz, dsr);
    const auto *Ep = a.E + (size_t)p.i * nr + p.j;
    const auto e00 = Ep[0], e01 = Ep[1], e10 = Ep[nr], e11 = Ep[nr + 1];
    const A ez[2][2] = {{e00.x, e01.x}, {e10.x, e11.x}};
    const A er[2][2] = {{e00.y, e01.y}, {e10.y, e11.y}};
    A Ez = 0, Er = 0;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            Ez += sz[u] * sr[v] * ez[u][v];
            Er += sz[u] * sr[v] * er[u][v];
        }
    const A r = ((A)p.j + p.orr) * dr;
    const A kz = (A)0.5 * qm * dt * dt, kv = (A)0.5 * qm * dt;
    const A rr = r + kz * Er;
    const bool flip = rr < (A)0;
    const A r1 = flip ? -rr : rr;
    const A vr1u = p.vr + kv * Er;
    const A ar1u = (A)0.5 * (qm * Er + p.ar);
    const A vr1 = flip ? m_abs(vr1u) : vr1u;
    const A ar1 = flip ? m_abs(ar1u) : ar1u;
    const A vt1 = p.vt;
    // first push
    const A vx = vr1 + (A)0.5 * ar1 * dt, vy = vt1;
    const A xr = r1 + vx * dt, yr = vy * dt;
    const A q2 = xr * xr + yr * yr;
    A c = 1, s = 0, ir2 = 0;
    if (q2 > (A)0) {
        ir2 = m_rsqrt(q2);
        c = xr * ir2;
        s = yr * ir2;
    }
    // reverse of the first push
    A vxb = vrb2 * c - vtb2 * s;
    A vyb = vrb2 * s + vtb2 * c;
    const A cb = vrb2 * vx + vtb2 * vy + arb2 * ar1;
    const A sb = vrb2 * vy - vtb2 * vx;
    A ar1b = arb2 * c;
    A xrb = 0, yrb = 0;
    if (q2 > (A)0) {
        xrb = rb2 * c + (cb * s * s - sb * c * s) * ir2;
        yrb = rb2 * s + (-cb * c * s + sb * c * c) * ir2;
    }
    const A r1b = xrb;
    vxb += dt * xrb;
    vyb += dt * yrb;
    const A z1b = zb2;
    const A vz2b = vzb2 + dt * zb2;
    const A vz1b = vz2b;
    const A az1b = azb2 + (A)0.5 * dt * vz2b;
    const A vr1b = vxb;
    ar1b += (A)0.5 * dt * vxb;
    const A vt1b = vyb;
    // reverse of the final push (and the axis reflection)
    const A rrb = flip ? -r1b : r1b;
    const A vr1ub = flip ? (vr1u < (A)0 ? -vr1b : (vr1u > (A)0 ? vr1b : (A)0)) : vr1b;
    const A ar1ub = flip ? (ar1u < (A)0 ? -ar1b : (ar1u > (A)0 ? ar1b : (A)0)) : ar1b;
    const A Ezb = kz * z1b + kv * vz1b + (A)0.5 * qm * az1b;
    const A Erb = kz * rrb + kv * vr1ub + (A)0.5 * qm * ar1ub;
    A zb = z1b, rb = rrb;
    // reverse of the gather: E's adjoint on the mesh, positions' share
    double *gz = Ebz + (size_t)p.i * nr + p.j, *gr = Ebr + (size_t)p.i * nr + p.j;
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const A wgt = sz[u] * sr[v];
            atomicAdd(gz + u * nr + v, (double)(wgt * Ezb));
            atomicAdd(gr + u * nr + v, (double)(wgt * Erb));
            const A f = ez[u][v] * Ezb + er[u][v] * Erb;
            zb += dsz[u] * sr[v] * f;
            rb += sz[u] * dsr[v] * f;
        }
    bout.z[k] = (double)zb;
    bout.r[k] = (double)rb;
    bout.vr[k] = (double)vr1ub;
    bout.vt[k] = (double)vt1b;
    bout.vz[k] = (double)vz1b;
    bout.ar[k] = (double)((A)0.5 * ar1ub);
    bout.az[k] = (double)((A)0.5 * az1b);
}

// adjoint of E = -grad phi (the stencils of k_efield) onto phi_bar
__global__ void k_efield_adj(const double *Ebz, const double *Ebr, double *phib, int nz, int nr, double dz,
                             double dr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    const double ez = Ebz[k], er = Ebr[k];
    if (ez != 0.0) {
        if (i == 0) {
            atomicAdd(phib + nr + j, -ez / dz);
            atomicAdd(phib + j, ez / dz);
        } else if (i == nz - 1) {
            atomicAdd(phib + k, -ez / dz);
            atomicAdd(phib + k - nr, ez / dz);
        } else {
            atomicAdd(phib + k + nr, -ez / (2.0 * dz));
            atomicAdd(phib + k - nr, ez / (2.0 * dz));
        }
    }
    if (er != 0.0 && j > 0) {
        if (j == nr - 1) {
            atomicAdd(phib + k, -er / dr);
            atomicAdd(phib + k - 1, er / dr);
        } else {
            atomicAdd(phib + k + 1, -er / (2.0 * dr));
            atomicAdd(phib + k - 1, er / (2.0 * dr));
        }
    }
}

// right-hand side of the adjoint solve in the solver's charge form: the
// solver's f = rho A_j dz / eps0 becomes phi_bar on the interior rows
__global__ void k_adj_rhs(const double *phib, double *rho, int nz, int nr, double dz, double dr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    rho[k] = (i > 0 && i < nz - 1 && j < nr - 1) ? phib[k] * kEps0 / (area_z(j, dr) * dz) : 0.0;
}

// chi_bar from the faces: dJ/dc_f = -(lam_a - lam_b)(phi_a - phi_b), c_f =
// (1 + chi_f) G_f, chi_f = max (or mean) of the two nodes' chi
__global__ void k_face_adj(const double *lam, const double *phi, const double *chi, double *chib, int nz,
                           int nr, double dz, double dr, int face_mean) {
    const int nzf = (nz - 1) * nr;  // z-faces (i, i+1) at column j, then r-faces (j, j+1) at row i
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nzf + nz * (nr - 1)) return;
    int a, b;
    double G;
    if (f < nzf) {
        a = f;
        b = f + nr;
        G = area_z(f % nr, dr) / dz;
    } else {
        const int g = f - nzf, i = g / (nr - 1), j = g % (nr - 1);
        a = i * nr + j;
        b = a + 1;
        G = 2.0 * kPi * ((j + 0.5) * dr) * dz / dr;
    }
    const double gf = -(lam[a] - lam[b]) * (phi[a] - phi[b]) * G;
    if (gf == 0.0) return;
    if (face_mean) {
        atomicAdd(chib + a, 0.5 * gf);
        atomicAdd(chib + b, 0.5 * gf);
    } else {
        atomicAdd(chib + (chi[a] > chi[b] ? a : b), gf);
    }
}

// per node: rho_bar, N_bar of both species (plus the functional's own term
// for the ions), and the Dirichlet rows' adjoints -> parameter gradients
__global__ void k_node_adj(const double *lam, const double *chi, const double *phib, const double *chib,
                           const double *V, const double *w, double *Nb0, double *Nb1, int nz, int nr,
                           double dz, double dr, int face_mean, double q0, double q1, double c0, double c1,
                           double jscale, double sin_t, double *Ab, double *phizLb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    const bool inner = i > 0 && i < nz - 1 && j < nr - 1;
    const double rhob = inner ? lam[k] * area_z(j, dr) * dz / kEps0 : 0.0;
    const double cb = chib[k];
    Nb0[k] = (q0 * rhob + c0 * cb) / V[k];
    Nb1[k] = (q1 * rhob + c1 * cb) / V[k] + jscale * w[k];
    auto face = [&](int lo, int hi) {
        return face_mean ? 0.5 * (chi[lo] + chi[hi]) : fmax(chi[lo], chi[hi]);
    };
    const double Gz = area_z(j, dr) / dz;
    if (i == 0 && j < nr - 1) {
        double b = phib[k];
        if (nz > 2) b += (1.0 + face(k, k + nr)) * Gz * lam[k + nr];
        atomicAdd(Ab, sin_t * b);
    } else if (i == nz - 1) {
        double b = phib[k];
        if (nz > 2 && j < nr - 1) b += (1.0 + face(k - nr, k)) * Gz * lam[k - nr];
        phizLb[j] += b;
    }
}

__global__ void k_set_J_term(double *Nb0, double *Nb1, const double *w, int ng, double jscale) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng) return;
    Nb0[k] = 0.0;
    Nb1[k] = jscale * w[k];
}

inline int blocks(long long n) { return (int)std::max(1LL, (n + kWT - 1) / kWT); }

}  // namespace

template <typename T>
int window_run(const WindowIn<T> &in, int K, int ckpt, const double *w_host, double amp0,
               const double *phizL_host, bool grad, double *J, double *dA, double *dphizL, std::string &err) {
    using V4T = typename V4<T>::type;
    using V2T = typename V2<T>::type;
    const int nz = in.nz, nr = in.nr, ng = nz * nr;
    cudaStream_t st = in.st;
    std::vector<void *> owned;
    auto take = [&](size_t bytes) {
        void *p = in.alloc(in.actx, bytes);
        owned.push_back(p);
        return p;
    };
    auto dgrid = [&]() { return (double *)take((size_t)ng * sizeof(double)); };
    int status = PIC_OK;
    try {
        const int nseg = (K + ckpt - 1) / ckpt;
        auto new_state = [&](int n) {
            WinState<T> s;
            s.q0 = (V4T *)take((size_t)std::max(n, 1) * sizeof(V4T));
            s.q1 = (V4T *)take((size_t)std::max(n, 1) * sizeof(V4T));
            s.cell = (int32_t *)take((size_t)std::max(n, 1) * sizeof(int32_t));
            return s;
        };
        auto new_adj = [&](int n) {
            WinAdj b;
            double **f[7] = {&b.z, &b.r, &b.vr, &b.vt, &b.vz, &b.ar, &b.az};
            for (auto q : f) *q = (double *)take((size_t)std::max(n, 1) * sizeof(double));
            return b;
        };
        // checkpoints [nseg + 1] per species; the segment's states [ckpt] per species
        std::vector<WinState<T>> ck[2], seg[2];
        for (int s = 0; s < 2; ++s) {
            for (int m = 0; m <= nseg; ++m) ck[s].push_back(new_state(in.n[s]));
            if (grad)
                for (int m = 0; m < ckpt; ++m) seg[s].push_back(new_state(in.n[s]));
        }
        // the potential of every step (the backward's recomputation takes it
        // instead of solving again: K grids, small beside the particles)
        std::vector<double *> phi_all(grad ? K + 1 : 0);
        for (auto &g : phi_all) g = dgrid();
        double *rho = dgrid(), *chi = dgrid(), *phi = dgrid(), *Ez = dgrid(), *Er = dgrid();
        double *N[2][2] = {{dgrid(), dgrid()}, {dgrid(), dgrid()}};  // [rolling][species]
        V2T *E2 = (V2T *)take((size_t)ng * sizeof(V2T));
        double *w_d = dgrid();
        double *pzl = (double *)take((size_t)nr * sizeof(double));
        double *acc = (double *)take((size_t)(2 + nr) * sizeof(double));  // J, A_bar, phi_zL_bar[nr]
        StepCtl *wctl = (StepCtl *)take(sizeof(StepCtl));
        cudaMemsetAsync(wctl, 0, sizeof(StepCtl), st);
        cudaMemsetAsync(acc, 0, (size_t)(2 + nr) * sizeof(double), st);
        cudaMemcpyAsync(w_d, w_host, (size_t)ng * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(pzl, phizL_host, (size_t)nr * sizeof(double), cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(phi, in.phi0, (size_t)ng * sizeof(double), cudaMemcpyDeviceToDevice, st);
        for (int s = 0; s < 2; ++s)
            if (in.n[s] > 0)
                k_win_init<T><<<blocks(in.n[s]), kWT, 0, st>>>(in.main[s], in.births[s], in.perm[s], in.nmain[s],
                                                                in.n[s], ck[s][0]);
        FieldDims fd{nz, nr, in.dz, in.dr, in.L, in.chi_face};
        StepArgs<T> a[2];
        for (int s = 0; s < 2; ++s) {
            a[s] = in.args[s];
            a[s].E = E2;
        }
        const double c_chi[2] = {0.5 * (in.q[0] / in.m[0]) * in.q[0] * in.dt * in.dt / kEps0,
                                 0.5 * (in.q[1] / in.m[1]) * in.q[1] * in.dt * in.dt / kEps0};
        auto voltage = [&](double t) {
            double v = amp0 * std::sin(2.0 * kPi * in.rf_freq[0] * t + in.rf_phase[0]);
            for (int q = 1; q < in.nrf; ++q) v += in.rf_amp[q] * std::sin(2.0 * kPi * in.rf_freq[q] * t + in.rf_phase[q]);
            return v;
        };
        auto deposit = [&](const WinState<T> *S, double **Nout) {
            for (int s = 0; s < 2; ++s) {
                cudaMemsetAsync(Nout[s], 0, (size_t)ng * sizeof(double), st);
                if (in.n[s] > 0)
                    k_win_deposit<T><<<blocks(in.n[s]), kWT, 0, st>>>(S[s], in.n[s], a[s].ncz, a[s].inv_ncz, nr,
                                                                       a[s].weighting, Nout[s]);
            }
        };
        int L = 0;
        // one forward step: field from Nin, push states in -> out, deposit into Nout
        // one forward step; `again`: the step's potential is the stored one
        auto fwd = [&](int n, const WinState<T> *Sin, const WinState<T> *Sout, double **Nin, double **Nout,
                       bool again) {
            launch_finalize(Nin[0], Nin[1], in.V, in.q[0], in.q[1], c_chi[0], c_chi[1], rho, chi, ng, nullptr, st);
            if (again) {
                cudaMemcpyAsync(phi, phi_all[n], (size_t)ng * sizeof(double), cudaMemcpyDeviceToDevice, st);
            } else {
                const double t = (double)(in.step0 + n) * in.dt;
                if (mg_fast_solve(fd, *in.mgf, rho, chi, voltage(t), pzl, phi, true, in.mixed, in.tol,
                                  in.max_cycles, nullptr, &L, wctl, st, false, true) == kSolveNoLaunch)
                    throw 1;
                if (grad) cudaMemcpyAsync(phi_all[n], phi, (size_t)ng * sizeof(double), cudaMemcpyDeviceToDevice, st);
            }
            launch_efield<T>(phi, Ez, Er, E2, nz, nr, in.dz, in.dr, nullptr, st);
            for (int s = 0; s < 2; ++s) {
                cudaMemsetAsync(Nout[s], 0, (size_t)ng * sizeof(double), st);
                if (in.n[s] > 0)
                    k_win_push<T><<<blocks(in.n[s]), kWT, 0, st>>>(a[s], Sin[s], Sout[s], in.n[s], Nout[s]);
            }
        };
        // ---- forward with checkpoints ----
        {
            WinState<T> cur[2] = {ck[0][0], ck[1][0]};
            double *Nc[2] = {N[0][0], N[0][1]}, *Nn[2] = {N[1][0], N[1][1]};
            deposit(cur, Nc);
            // two working states beyond the checkpoints: reuse the segment's (or
            // the next checkpoint slot when only the forward runs)
            for (int n = 1; n <= K; ++n) {
                const int m = (n - 1) / ckpt;
                WinState<T> nxt[2];
                for (int s = 0; s < 2; ++s) nxt[s] = (n % ckpt == 0 || n == K) ? ck[s][m + 1] : (grad ? seg[s][(n - 1) % ckpt] : ck[s][m + 1]);
                fwd(n, cur, nxt, Nc, Nn, false);
                k_win_J<<<(ng + kWT * 8 - 1) / (kWT * 8), kWT, 0, st>>>(Nn[1], w_d, ng, 1.0 / K, acc);
                for (int s = 0; s < 2; ++s) {
                    cur[s] = nxt[s];
                    std::swap(Nc[s], Nn[s]);
                }
            }
        }
        if (grad) {
            // per segment step: E and chi of the recomputed forward
            std::vector<V2T *> E2s(ckpt);
            std::vector<double *> chis(ckpt);
            for (int q = 0; q < ckpt; ++q) {
                E2s[q] = (V2T *)take((size_t)ng * sizeof(V2T));
                chis[q] = dgrid();
            }
            WinAdj b[2][2];
            for (int s = 0; s < 2; ++s) {
                b[0][s] = new_adj(in.n[s]);
                b[1][s] = new_adj(in.n[s]);
                for (double *f : {b[0][s].z, b[0][s].r, b[0][s].vr, b[0][s].vt, b[0][s].vz, b[0][s].ar, b[0][s].az})
                    cudaMemsetAsync(f, 0, (size_t)std::max(in.n[s], 1) * sizeof(double), st);
            }
            double *Nb[2] = {dgrid(), dgrid()};
            double *Ebz = dgrid(), *Ebr = dgrid(), *phib = dgrid(), *rhof = dgrid(), *lam = dgrid(), *chib = dgrid();
            cudaMemsetAsync(lam, 0, (size_t)ng * sizeof(double), st);
            k_set_J_term<<<blocks(ng), kWT, 0, st>>>(Nb[0], Nb[1], w_d, ng, 1.0 / K);
            int pb = 0;  // b[pb] holds the adjoint of the current state
            for (int m = nseg - 1; m >= 0; --m) {
                const int a0 = m * ckpt, b0 = std::min(a0 + ckpt, K);
                // recompute the segment: states S[a0..b0] (S[a0] the checkpoint)
                std::vector<WinState<T>> S[2];
                for (int s = 0; s < 2; ++s) {
                    S[s].push_back(ck[s][m]);
                    for (int q = 0; q < b0 - a0; ++q) S[s].push_back(seg[s][q]);
                }
                double *Nc[2] = {N[0][0], N[0][1]}, *Nn[2] = {N[1][0], N[1][1]};
                WinState<T> c0[2] = {S[0][0], S[1][0]};
                deposit(c0, Nc);
                for (int n = a0 + 1; n <= b0; ++n) {
                    const int q = n - a0;
                    WinState<T> si[2] = {S[0][q - 1], S[1][q - 1]}, so[2] = {S[0][q], S[1][q]};
                    fwd(n, si, so, Nc, Nn, true);
                    cudaMemcpyAsync(E2s[q - 1], E2, (size_t)ng * sizeof(V2T), cudaMemcpyDeviceToDevice, st);
                    cudaMemcpyAsync(chis[q - 1], chi, (size_t)ng * sizeof(double), cudaMemcpyDeviceToDevice, st);
                    for (int s = 0; s < 2; ++s) std::swap(Nc[s], Nn[s]);
                }
                // reverse of the segment's steps
                for (int n = b0; n > a0; --n) {
                    const int q = n - a0;
                    cudaMemsetAsync(Ebz, 0, (size_t)ng * sizeof(double), st);
                    cudaMemsetAsync(Ebr, 0, (size_t)ng * sizeof(double), st);
                    for (int s = 0; s < 2; ++s) {
                        if (in.n[s] == 0) continue;
                        StepArgs<T> as = a[s];
                        as.E = E2s[q - 1];
                        k_win_back<T><<<blocks(in.n[s]), kWT, 0, st>>>(
                            as, S[s][q - 1], S[s][q], in.n[s], Nb[s], b[pb][s], b[1 - pb][s], Ebz, Ebr, (T)in.dr,
                            (T)(1.0 / in.dz), (T)(1.0 / in.dr), (T)(in.q[s] / in.m[s]), (T)in.dt);
                    }
                    pb = 1 - pb;
                    cudaMemsetAsync(phib, 0, (size_t)ng * sizeof(double), st);
                    k_efield_adj<<<blocks(ng), kWT, 0, st>>>(Ebz, Ebr, phib, nz, nr, in.dz, in.dr);
                    k_adj_rhs<<<blocks(ng), kWT, 0, st>>>(phib, rhof, nz, nr, in.dz, in.dr);
                    // warm start from the previous step's lambda (zero at first):
                    // consecutive adjoint fields are close
                    if (mg_fast_solve(fd, *in.mgf, rhof, chis[q - 1], 0.0, nullptr, lam, true, in.mixed, in.tol,
                                      in.max_cycles, nullptr, &L, wctl, st, false, true) == kSolveNoLaunch)
                        throw 1;
                    cudaMemsetAsync(chib, 0, (size_t)ng * sizeof(double), st);
                    k_face_adj<<<blocks((long long)(nz - 1) * nr + (long long)nz * (nr - 1)), kWT, 0, st>>>(
                        lam, phi_all[n], chis[q - 1], chib, nz, nr, in.dz, in.dr, in.chi_face == PIC_CHI_MEAN);
                    const double t = (double)(in.step0 + n) * in.dt;
                    const double sin_t = std::sin(2.0 * kPi * in.rf_freq[0] * t + in.rf_phase[0]);
                    k_node_adj<<<blocks(ng), kWT, 0, st>>>(lam, chis[q - 1], phib, chib, in.V, w_d, Nb[0], Nb[1], nz,
                                                          nr, in.dz, in.dr, in.chi_face == PIC_CHI_MEAN, in.q[0],
                                                          in.q[1], c_chi[0], c_chi[1], n > 1 ? 1.0 / K : 0.0, sin_t,
                                                          acc + 1, acc + 2);
                }
            }
        }
        double hv[2];
        std::vector<double> pz((size_t)nr);
        StepCtl c;
        cudaMemcpyAsync(hv, acc, 2 * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(pz.data(), acc + 2, (size_t)nr * sizeof(double), cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(&c, wctl, sizeof(StepCtl), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (J) *J = hv[0];
        if (grad) {
            if (dA) *dA = hv[1];
            if (dphizL)
                for (int j = 0; j < nr; ++j) dphizL[j] = pz[j];
        }
        if (c.halt) {
            status = PIC_ERR_TIMEOUT;
            err = "window: multigrid grid barrier timed out";
        } else if (c.mg_flags & 1) {
            status = PIC_ERR_NOT_CONVERGED;
            err = "window: multigrid stopped before the tolerance";
        }
    } catch (...) {
        cudaStreamSynchronize(st);
        status = PIC_ERR_CUDA;
        err = "window: allocation or solver launch failed";
    }
    cudaStreamSynchronize(st);
    for (void *p : owned) in.release(in.actx, p);
    return status;
}

template int window_run<float>(const WindowIn<float> &, int, int, const double *, double, const double *, bool,
                               double *, double *, double *, std::string &);
template int window_run<double>(const WindowIn<double> &, int, int, const double *, double, const double *, bool,
                                double *, double *, double *, std::string &);

}  // namespace pic
