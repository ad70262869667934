// mg.cu -- the multigrid field solve of the timestep (Sec. 2.5, Algorithm 1),
// arranged for few launches and little FP64 work on GB300.
//
// Same method as the reference GPU multigrid in field.cu (and as the
// oracle): finite-volume operator, z-only coarsening, V(0,1) cycles with a
// red-black r-line sweep per level on the way up, [1/2 1 1/2] restriction
// of volume-integrated residuals, linear prolongation in z.  What changes is
// the arrangement:
//  - the parallel-cyclic-reduction elimination factors of every r-line of
//    every level are computed once per solve (the line matrices do not
//    change between cycles); a line sweep is then two FMAs per unknown and
//    step;
//  - one kernel computes the fine residual and runs the whole restriction
//    chain down one column per warp (restriction acts in z only);
//  - prolongation is folded into the red sweep: red (odd) rows are
//    recomputed whole by their line solve, so only the injection of the
//    coarse correction into the black (even) neighbour rows is ever used;
//  - convergence is decided on the device: the last block of the residual
//    kernel compares max|r| with tol max|b| and raises a done flag that
//    turns the remaining kernels of a batch into no-ops, so the host reads
//    back once per batch of cycles.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "mg.cuh"

namespace pic {

namespace {

// bit pattern of |x|: ordered like |x| for numbers, above them for a NaN
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *dst, double v) {
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

// ---- set-up ----

// nodal chi of every coarse level: full weighting in z, injection on the
// boundary rows; one warp per column, lanes over rows, levels in shared memory
__global__ void k_chi_levels(const MGFast *__restrict__ mp, int nr) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MGFast &m = *mp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nz0 = m.nz[0];
    const int j = blockIdx.x * (blockDim.x >> 5) + warp;
    if (j >= nr) return;
    double *src = reinterpret_cast<double *>(smem_raw) + (size_t)warp * 2 * nz0;
    double *dst = src + nz0;
    for (int i = lane; i < nz0; i += 32) src[i] = m.chi[0][(size_t)i * nr + j];
    __syncwarp();
    for (int l = 1; l < m.nlev; ++l) {
        const int nzc = m.nz[l];
        for (int I = lane; I < nzc; I += 32) {
            const double v = (I == 0 || I == nzc - 1)
                                 ? src[2 * I]
                                 : 0.25 * src[2 * I - 1] + 0.5 * src[2 * I] + 0.25 * src[2 * I + 1];
            dst[I] = v;
            m.chi[l][(size_t)I * nr + j] = v;
        }
        __syncwarp();
        double *t = src;
        src = dst;
        dst = t;
    }
}

// face coefficients of every level (flat index over all levels' nodes)
__global__ void k_coefs_levels(const MGFast *__restrict__ mp, int nr, double dr, int face_mean, int total) {
    const MGFast &m = *mp;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total) return;
    int l = 0, k = g;
    while (k >= m.nz[l] * nr) {
        k -= m.nz[l] * nr;
        ++l;
    }
    const int nz = m.nz[l], i = k / nr, j = k % nr;
    const double dz = m.dz[l];
    const double *chi = m.chi[l];
    const double c = chi[k];
    double vz = 0.0, vr = 0.0;
    if (i + 1 < nz) {
        const double cn = chi[k + nr];
        const double f = face_mean ? 0.5 * (c + cn) : fmax(c, cn);
        const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
        vz = (1.0 + f) * (kPi * (rp * rp - rm * rm)) / dz;
    }
    if (j + 1 < nr) {
        const double cn = chi[k + 1];
        const double f = face_mean ? 0.5 * (c + cn) : fmax(c, cn);
        vr = (1.0 + f) * 2.0 * kPi * ((j + 0.5) * dr) * dz / dr;
    }
    m.cz[l][k] = vz;
    m.cr[l][k] = vr;
    if (m.cz32[l]) {
        m.cz32[l][k] = (float)vz;
        m.cr32[l][k] = (float)vr;
    }
}

// 1/x: IEEE division in FP32; in FP64 a float reciprocal refined by two
// Newton-Raphson steps r <- r (2 - x r) (relative error ~1e-16 from ~6e-8)
__device__ __forceinline__ float recip(float x) { return 1.0f / x; }
__device__ __forceinline__ double recip(double x) {
    double r = (double)(1.0f / (float)x);
    r = fma(r, fma(-x, r, 1.0), r);
    r = fma(r, fma(-x, r, 1.0), r);
    return r;
}

// PCR elimination factors, one r-line per block, over the lines of levels
// [l0, l1).  Line system for row i: lower -d_j = -cr[i][j-1] (0 on the
// axis), diagonal a+c+d+e, upper -e_j = -cr[i][j] (0 on the last unknown).
// Step s = 2^k combines equation j with j -/+ s: alpha = -lo_j / diag_{j-s},
// gamma = -up_j / diag_{j+s}.  Stored per line: [k][alpha(n), gamma(n)] for
// k < K, then 1/diag (n).
template <typename Ts>
__global__ void k_factor_levels(const MGFast *__restrict__ mp, int l0, int l1, int nr, int K) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MGFast &m = *mp;
    const int n = nr - 1;
    int g = blockIdx.x, l = l0;
    while (l < l1 && g >= m.nz[l] - 2) {
        g -= m.nz[l] - 2;
        ++l;
    }
    if (l >= l1) return;
    const bool f64 = sizeof(Ts) == 8;
    const Ts *cz = f64 ? (const Ts *)m.cz[l] : (const Ts *)m.cz32[l];
    const Ts *cr = f64 ? (const Ts *)m.cr[l] : (const Ts *)m.cr32[l];
    Ts *fac = (l == m.nlev - 1) ? (Ts *)m.facc : (f64 ? (Ts *)m.fac64[l] : (Ts *)m.fac32[l]);
    Ts *A = reinterpret_cast<Ts *>(smem_raw);
    Ts *B = A + n, *C = B + n, *A2 = C + n, *B2 = A2 + n, *C2 = B2 + n, *IB = C2 + n;
    const int i = 1 + g;  // interior row
    const size_t rowk = (size_t)i * nr;
    Ts *f = fac + (size_t)g * (2 * K + 1) * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const size_t k = rowk + j;
        const Ts a = cz[k - nr], c = cz[k], e = cr[k];
        const Ts d = j > 0 ? cr[k - 1] : (Ts)0;
        A[j] = -d;
        B[j] = a + c + d + e;
        C[j] = j < n - 1 ? -e : (Ts)0;
    }
    __syncthreads();
    int step = 0;
    for (int s = 1; s < n; s <<= 1, ++step) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) IB[j] = recip(B[j]);
        __syncthreads();
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            const Ts a = A[j], c = C[j];
            Ts b = B[j], na = 0, nc = 0, al = 0, ga = 0;
            if (j - s >= 0) {
                al = -a * IB[j - s];
                na = al * A[j - s];
                b += al * C[j - s];
            }
            if (j + s < n) {
                ga = -c * IB[j + s];
                nc = ga * C[j + s];
                b += ga * A[j + s];
            }
            A2[j] = na;
            B2[j] = b;
            C2[j] = nc;
            f[(size_t)(2 * step) * n + j] = al;
            f[(size_t)(2 * step + 1) * n + j] = ga;
        }
        __syncthreads();
        Ts *t;
        t = A; A = A2; A2 = t;
        t = B; B = B2; B2 = t;
        t = C; C = C2; C2 = t;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) f[(size_t)(2 * K) * n + j] = recip(B[j]);
}

// right-hand side rho A_j dz / eps0 and the Dirichlet data of phi
__global__ void k_rhs_bc(const double *rho, double *f0, double *phi, const double *phi_zL,
                         double V, int nz, int nr, double dz, double dr, int cold) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    double v = 0.0;
    if (i > 0 && i < nz - 1 && j < nr - 1) {
        const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
        v = rho[k] * (kPi * (rp * rp - rm * rm)) * dz / kEps0;
    }
    f0[k] = v;
    if (i == 0)
        phi[k] = (j == nr - 1) ? 0.0 : V;
    else if (i == nz - 1)
        phi[k] = phi_zL ? phi_zL[j] : 0.0;
    else if (j == nr - 1)
        phi[k] = 0.0;
    else if (cold)
        phi[k] = 0.0;
}

// ---- the PCR line solve with precomputed factors (block per line) ----
// One unknown per thread (n <= blockDim <= 1024).  A thread first loads all
// its factors into registers -- independent loads, one memory round trip --
// so the K reduction steps touch only shared memory.
constexpr int kMaxK = 10;  // n <= 1024

template <typename Ts>
struct LineFac {
    Ts f[2 * kMaxK + 1];
};

template <typename Ts>
__device__ __forceinline__ LineFac<Ts> load_fac(const Ts *fac, int n, int K, int j) {
    LineFac<Ts> r;
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        r.f[2 * k] = (k < K && j < n) ? fac[(size_t)(2 * k) * n + j] : (Ts)0;
        r.f[2 * k + 1] = (k < K && j < n) ? fac[(size_t)(2 * k + 1) * n + j] : (Ts)0;
    }
    r.f[2 * kMaxK] = j < n ? fac[(size_t)(2 * K) * n + j] : (Ts)0;
    return r;
}

// d = this thread's right-hand side; returns the solution of unknown j
template <typename Ts>
__device__ __forceinline__ Ts pcr_solve(Ts d, Ts *D, Ts *D2, const LineFac<Ts> &fr, int n, int K) {
    const int j = threadIdx.x;
    if (j < n) D[j] = d;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kMaxK; ++k) {
        if (k < K) {
            const int s = 1 << k;
            if (j < n) {
                Ts v = D[j];
                if (j - s >= 0) v += fr.f[2 * k] * D[j - s];
                if (j + s < n) v += fr.f[2 * k + 1] * D[j + s];
                D2[j] = v;
                d = v;
            }
            __syncthreads();
            Ts *t = D;
            D = D2;
            D2 = t;
        }
    }
    return d * fr.f[2 * kMaxK];
}

// ---- per-cycle kernels ----

// r = f - A phi on the fine level (FP64, all SMs), its max norm, and on the
// first cycle max|b|; the mixed path also keeps r in FP32 as its level-0
// right-hand side.  The last block decides convergence.
__global__ void k_resid(const MGFast *__restrict__ mp, int nr, const double *phi, int first) {
    const MGFast &m = *mp;
    MGCtl *ctl = m.ctl;
    if (ctl->done) return;
    const int nz = m.nz[0], ng = nz * nr;
    const double *cz = m.cz[0], *cr = m.cr[0];
    double rmax = 0.0, bmax = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < ng; k += gridDim.x * blockDim.x) {
        const int i = k / nr, j = k % nr;
        double r = 0.0;
        if (i > 0 && i < nz - 1 && j < nr - 1) {
            const double a = cz[k - nr], c = cz[k], e = cr[k], d = j > 0 ? cr[k - 1] : 0.0;
            double Au = (a + c + d + e) * phi[k] - a * phi[k - nr] - c * phi[k + nr] - e * phi[k + 1];
            if (j > 0) Au -= d * phi[k - 1];
            r = m.f0[k] - Au;
            rmax = fmax(rmax, fabs(r));
            if (first) {
                double b = m.f0[k];
                if (i == 1) b += a * phi[k - nr];
                if (i == nz - 2) b += c * phi[k + nr];
                if (j == nr - 2) b += e * phi[k + 1];
                bmax = fmax(bmax, fabs(b));
            }
        }
        m.r[k] = r;
        if (m.f32[0]) m.f32[0][k] = (float)r;
    }
    for (int o = 16; o > 0; o >>= 1) {
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
        bmax = fmax(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
    }
    __shared__ double s_r[32], s_b[32];
    __shared__ bool s_last;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_r[warp] = rmax;
        s_b[warp] = bmax;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double r = 0.0, b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            r = fmax(r, s_r[w]);
            b = fmax(b, s_b[w]);
        }
        atomic_max_pos(&ctl->res_bits, r);
        if (first) atomic_max_pos(&ctl->b_bits, b);
        __threadfence();
        const unsigned prev = atomicAdd(&ctl->blocks_in, 1u);
        s_last = prev == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const double rn = __longlong_as_double((long long)atomicAdd(&ctl->res_bits, 0ull));
        const double bn = __longlong_as_double((long long)atomicAdd(&ctl->b_bits, 0ull));
        ctl->last_res = rn;
        ctl->bnorm = bn;
        bool done = false;
        if (bn == 0.0) {
            done = true;
            ctl->zero_rhs = 1;
        } else if (ctl->tol > 0.0 && rn <= ctl->tol * bn) {
            done = true;
            ctl->converged = 1;
        } else if (ctl->cycles >= ctl->max_cycles) {
            done = true;
            ctl->converged = ctl->tol > 0.0 ? 0 : 1;
        }
        ctl->res_bits = 0ull;
        ctl->blocks_in = 0u;
        if (done)
            ctl->done = 1;
        else
            ctl->cycles += 1;
    }
}

// restriction chain, one lane per column j < nr-1: level values go through
// shared memory laid out [row][lane]; each level is
// f_{l+1}[I] = f_l[2I-1]/2 + f_l[2I] + f_l[2I+1]/2 on interior rows
template <typename Tv>
__global__ void k_chain(const MGFast *__restrict__ mp, int nr) {
    const MGFast &m = *mp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (m.ctl->done) return;
    const int lane = threadIdx.x;
    const int j = blockIdx.x * 32 + lane;
    const int n1 = m.nz[1], nz0 = m.nz[0];
    double *col = reinterpret_cast<double *>(smem_raw);      // [nz0][32]
    Tv *bufA = reinterpret_cast<Tv *>(col + (size_t)nz0 * 32);  // [n1][32]
    Tv *bufB = bufA + (size_t)n1 * 32;
    const bool on = j < nr - 1;
    // the column of the fine residual: independent loads, then compute
    {
        const double *__restrict__ r = m.r;
        for (int i = 0; i < nz0; ++i) col[i * 32 + lane] = on ? r[(size_t)i * nr + j] : 0.0;
    }
    for (int I = 0; I < n1; ++I) {
        Tv v = 0;
        if (I > 0 && I < n1 - 1)
            v = (Tv)(0.5 * col[(2 * I - 1) * 32 + lane] + col[(2 * I) * 32 + lane] +
                     0.5 * col[(2 * I + 1) * 32 + lane]);
        bufA[I * 32 + lane] = v;
        if (on) {
            const size_t k = (size_t)I * nr + j;
            if (m.nlev == 2)
                m.fc64[k] = (double)v;
            else if (sizeof(Tv) == 8)
                m.f64[1][k] = (double)v;
            else
                m.f32[1][k] = (float)v;
        }
    }
    Tv *src = bufA, *dst = bufB;
    for (int l = 2; l < m.nlev; ++l) {
        const int nzc = m.nz[l];
        for (int I = 0; I < nzc; ++I) {
            Tv v = 0;
            if (I > 0 && I < nzc - 1)
                v = (Tv)0.5 * src[(2 * I - 1) * 32 + lane] + src[(2 * I) * 32 + lane] +
                    (Tv)0.5 * src[(2 * I + 1) * 32 + lane];
            dst[I * 32 + lane] = v;
            if (on) {
                const size_t k = (size_t)I * nr + j;
                if (l == m.nlev - 1)
                    m.fc64[k] = (double)v;
                else if (sizeof(Tv) == 8)
                    m.f64[l][k] = (double)v;
                else
                    m.f32[l][k] = (float)v;
            }
        }
        Tv *t = src;
        src = dst;
        dst = t;
    }
}

// coarsest level: one interior row, FP64 factors, result stored in the
// V-cycle's type
template <typename Tv>
__global__ void k_coarse(const MGFast *__restrict__ mp, int nr, int K) {
    const MGFast &m = *mp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (m.ctl->done) return;
    const int n = nr - 1, L = m.nlev - 1, j = threadIdx.x;
    double *D = reinterpret_cast<double *>(smem_raw);
    const LineFac<double> fr = load_fac(m.facc, n, K, j);
    const double rhs = j < n ? m.fc64[(size_t)nr + j] : 0.0;
    const double x = pcr_solve<double>(rhs, D, D + n, fr, n, K);
    Tv *u = sizeof(Tv) == 8 ? (Tv *)m.u64[L] : (Tv *)m.u32[L];
    if (j < n) u[(size_t)nr + j] = (Tv)x;
}

// Red sweep of level l with the prolongation folded in: row i (odd) solves
// with neighbours u_old[i-/+1] + injected coarse correction (even rows are
// coarse rows (i-/+1)/2).  Level 0 of the FP64 path works on phi itself
// (u_old = phi, Dirichlet values read from phi); every other level works on
// a correction that starts at zero with zero Dirichlet values.
template <typename Tv>
__global__ void k_red(const MGFast *__restrict__ mp, int l, int nr, int K, Tv *u, const Tv *uc, const Tv *f,
                      const Tv *cz, const Tv *cr, const Tv *fac, int on_phi) {
    const MGFast &m = *mp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (m.ctl->done) return;
    const int n = nr - 1, nz = m.nz[l], nzc = m.nz[l + 1], j = threadIdx.x;
    Tv *D = reinterpret_cast<Tv *>(smem_raw);
    const int i = 1 + 2 * blockIdx.x;
    const size_t rowk = (size_t)i * nr;
    const LineFac<Tv> fr = load_fac(fac + (size_t)(i - 1) * (2 * K + 1) * n, n, K, j);
    Tv rhs = 0;
    if (j < n) {
        const int Idn = (i - 1) / 2, Iup = (i + 1) / 2;
        const size_t k = rowk + j;
        Tv udn, uup;
        if (i - 1 == 0)
            udn = on_phi ? u[k - nr] : (Tv)0;
        else
            udn = (on_phi ? u[k - nr] : (Tv)0) + ((Idn > 0 && Idn < nzc - 1) ? uc[(size_t)Idn * nr + j] : (Tv)0);
        if (i + 1 == nz - 1)
            uup = on_phi ? u[k + nr] : (Tv)0;
        else
            uup = (on_phi ? u[k + nr] : (Tv)0) + ((Iup > 0 && Iup < nzc - 1) ? uc[(size_t)Iup * nr + j] : (Tv)0);
        rhs = f[k] + cz[k - nr] * udn + cz[k] * uup;
        if (j == n - 1 && on_phi) rhs += cr[k] * u[k + 1];
    }
    const Tv x = pcr_solve<Tv>(rhs, D, D + n, fr, n, K);
    if (j < n) u[rowk + j] = x;
}

// Black sweep: row i (even, interior) solves with the new red rows i-/+1.
template <typename Tv>
__global__ void k_black(const MGFast *__restrict__ mp, int l, int nr, int K, Tv *u, const Tv *f, const Tv *cz,
                        const Tv *cr, const Tv *fac, int on_phi) {
    const MGFast &m = *mp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (m.ctl->done) return;
    const int n = nr - 1, j = threadIdx.x;
    Tv *D = reinterpret_cast<Tv *>(smem_raw);
    const int i = 2 + 2 * blockIdx.x;
    const size_t rowk = (size_t)i * nr;
    const LineFac<Tv> fr = load_fac(fac + (size_t)(i - 1) * (2 * K + 1) * n, n, K, j);
    Tv rhs = 0;
    if (j < n) {
        const size_t k = rowk + j;
        rhs = f[k] + cz[k - nr] * u[k - nr] + cz[k] * u[k + nr];
        if (j == n - 1 && on_phi) rhs += cr[k] * u[k + 1];
    }
    const Tv x = pcr_solve<Tv>(rhs, D, D + n, fr, n, K);
    if (j < n) u[rowk + j] = x;
}

// mixed path: phi += delta on interior nodes
__global__ void k_correct(const MGFast *__restrict__ mp, double *phi, const float *du, int nz, int nr) {
    const MGFast &m = *mp;
    if (m.ctl->done) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    if (i == 0 || i == nz - 1 || j == nr - 1) return;
    phi[k] += (double)du[k];
}

// nz = 3: the one interior row of phi solved exactly with the fine right-hand side
__global__ void k_single_row(const MGFast *__restrict__ mp, double *phi, int nr, int K) {
    const MGFast &m = *mp;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (m.ctl->done) return;
    const int n = nr - 1, j = threadIdx.x;
    double *D = reinterpret_cast<double *>(smem_raw);
    const LineFac<double> fr = load_fac(m.facc, n, K, j);
    double rhs = 0.0;
    if (j < n) {
        const double *cz = m.cz[0], *cr = m.cr[0];
        const size_t k = (size_t)nr + j;
        rhs = m.f0[k] + cz[k - nr] * phi[k - nr] + cz[k] * phi[k + nr];
        if (j == n - 1) rhs += cr[k] * phi[k + 1];
    }
    const double x = pcr_solve<double>(rhs, D, D + n, fr, n, K);
    if (j < n) phi[(size_t)nr + j] = x;
}

// ---------------------------------------------------------------------------
// The whole solve in one cooperative launch.  Blocks are co-resident (the
// launch guarantees it), and phases are separated by a grid barrier whose
// spin is bounded: after kSpinLimit polls a block raises `timeout` and every
// block leaves.  The V-cycle works on the correction delta of phi in both
// precisions (FP32 delta and residual for the mixed path).  Per cycle:
//   1. residual of phi + delta, its norms and the restriction chain down to
//      the coarsest level, one tile of columns per block (coalesced rows);
//   2. convergence decision (every block reads the same maxima), then
//      phi += delta;
//   3. up the levels, one phase per level: the block owning black line
//      i = 2q + 2 solves the red lines 2q + 1 and 2q + 3 beside it (the two
//      halves of the block at once when they fit), keeps them in shared
//      memory and solves the black line.  A red line shared by two blocks is
//      computed by both from the same data, bit for bit, and stored by one.
//      So one barrier separates two levels instead of two.
// The coarsest row is solved by block 0 in the phase of level L-1, which
// block 0 sweeps alone.  Levels with at most kBarGroup black lines belong to
// the first kBarGroup blocks, separated by a barrier among those blocks only;
// the rest of the grid waits at the next full barrier.
// ---------------------------------------------------------------------------
constexpr long long kSpinLimit = 1LL << 26;

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void atom_add_release(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Barrier on a counter that only grows: thread 0 of each block adds 1 with
// release semantics and polls with acquire loads until the counter reaches
// the target of this barrier (its number of participants times the number
// of barriers of this kind the block has passed).  The block's writes before
// the barrier are visible to every participant after it.  The poll is
// bounded: after kSpinLimit tries (or once another block gave up) the block
// raises `timeout` and returns false.
constexpr int kBarGroup = 8;  // blocks that sweep the coarse levels alone

__device__ __forceinline__ bool count_barrier(unsigned *count, unsigned target, MGCtl *ctl) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        atom_add_release(count, 1u);
        long long it = 0;
        while ((int)(ld_acquire(count) - target) < 0) {
            if ((++it & 255) == 0 && (it > kSpinLimit || *(volatile int *)&ctl->timeout)) {
                atomicExch(&ctl->timeout, 1);
                ok = 0;
                break;
            }
        }
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Asynchronous copy of `bytes` (a multiple of the element size) from global
// to shared memory by threads t = 0..nt-1 of the block: 16-byte pieces when
// both ends and the length allow it, else 8- or 4-byte pieces.  The caller
// commits the group.
__device__ __forceinline__ void copy_async(void *dst, const void *src, int bytes, int t, int nt) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    const char *s = static_cast<const char *>(src);
    const unsigned long long a = (unsigned long long)s | d | (unsigned)bytes;
    if ((a & 15) == 0) {
        for (int o = t * 16; o < bytes; o += nt * 16)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d + o), "l"(s + o) : "memory");
    } else if ((a & 7) == 0) {
        for (int o = t * 8; o < bytes; o += nt * 8)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d + o), "l"(s + o) : "memory");
    } else {
        for (int o = t * 4; o < bytes; o += nt * 4)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d + o), "l"(s + o) : "memory");
    }
}
__device__ __forceinline__ void copy_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void copy_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// PCR reduction of one line whose factors F were requested with cp.async:
// unknown j of the line (active when act) with right-hand side d; returns
// its solution.  Every thread of the block calls it (the two halves of a
// block may reduce two lines at once).  keep_newest: the most recent copy
// group may still be in flight (it belongs to a later line).
template <typename Ts>
__device__ __forceinline__ Ts pcr_line(Ts d, Ts *D, Ts *D2, const Ts *F, int n, int K, int j, bool act,
                                       bool keep_newest) {
    if (keep_newest)
        asm volatile("cp.async.wait_group 1;" ::: "memory");
    else
        asm volatile("cp.async.wait_group 0;" ::: "memory");
    if (act) D[j] = d;
    __syncthreads();
    int k = 0;
    for (int s = 1; s < n; s <<= 1, ++k) {
        if (act) {
            Ts v = D[j];
            if (j - s >= 0) v += F[(size_t)(2 * k) * n + j] * D[j - s];
            if (j + s < n) v += F[(size_t)(2 * k + 1) * n + j] * D[j + s];
            D2[j] = v;
            d = v;
        }
        __syncthreads();
        Ts *t = D;
        D = D2;
        D2 = t;
    }
    const Ts x = act ? d * F[(size_t)(2 * K) * n + j] : (Ts)0;
    __syncthreads();  // F and D are reused by the next line
    return x;
}

// Shared-memory layout of the one-launch solve (byte offsets), set on the host.
struct SolveLayout {
    int offD;   // PCR scratch: per half 2n values of 8 bytes
    int offX;   // the two red lines' solutions, kept for the black line's right-hand side
    int offR0;  // factors of the first red line; the coarsest row's FP64 factors
    int offR1;  // factors of the second red line (== offR0: reds one after the other)
    int offB;   // factors of the black line (== offR0: requested after the reds)
    int offT;   // residual / restriction tile (== offR0: no early request of the coarsest factors)
    int tw;     // columns per residual tile
    int lt;     // threads per line (power of two >= n)
    int pair;   // the two halves of the block reduce the two red lines at once
};

// black lines of a level with nz rows (at least one unit of work: nz = 3 has
// a red line only)
__device__ __forceinline__ int units_of(int nz) { return max((nz - 3) / 2, 1); }

template <typename Tv>
__global__ void __launch_bounds__(1024) k_solve_persistent(const MGFast *__restrict__ mp, double *phi, int nr, int K,
                                   int first_cycle, SolveLayout lay) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MGFast &m = *mp;
    MGCtl *ctl = m.ctl;
    const int n = nr - 1, nz0 = m.nz[0], ng = nz0 * nr, L = m.nlev - 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    const bool mixed = sizeof(Tv) == 4;
    Tv *delta = mixed ? (Tv *)m.u32[0] : (Tv *)m.u64[0];  // level-0 correction (zero on the boundary)
    const bool cpre = lay.offT != lay.offR0;                // coarsest factors requested early
    const bool bsep = lay.offB != lay.offR0;
    const int FE = (2 * K + 1) * n;                         // factor elements of a line
    // levels whose work fits in G blocks are swept by the first G blocks only
    const int G = min(kBarGroup, (int)gridDim.x);
    int lb = L;
    while (lb > 0 && units_of(m.nz[lb - 1]) <= G) --lb;
    const bool in_group = (int)blockIdx.x < G;
    __shared__ unsigned long long s_r[32], s_b[32];
    __shared__ int s_decide;
    int first = first_cycle;
    unsigned ngrid = 0, ngroup = 0;  // barriers of each kind passed
    Tv *X = reinterpret_cast<Tv *>(smem_raw + lay.offX);
    Tv *R0 = reinterpret_cast<Tv *>(smem_raw + lay.offR0);
    Tv *R1 = reinterpret_cast<Tv *>(smem_raw + lay.offR1);
    Tv *FBk = reinterpret_cast<Tv *>(smem_raw + lay.offB);
    const int half = lay.pair ? (tid >= lay.lt) : 0;
    const int jl = lay.pair ? tid - half * lay.lt : tid;  // unknown of this thread's line
    Tv *Dh = reinterpret_cast<Tv *>(smem_raw + lay.offD + (size_t)half * 2 * n * sizeof(double));
    for (int cyc = 0;; ++cyc) {
        // ---- residual of phi + delta, its norms, and the restriction chain ----
        if (cpre && blockIdx.x == 0 && L > 0) copy_async(R0, m.facc, FE * 8, tid, nt);
        copy_commit();
        // maxima as bit patterns of |x| (ordered like the values; a NaN
        // compares above every number), so the reductions are integer work
        unsigned long long rmax = 0ull, bmax = 0ull;
        {
            const double *cz = m.cz[0], *cr = m.cr[0];
            const int tw = lay.tw;
            // the restriction chain runs in the V-cycle's type
            Tv *T0 = reinterpret_cast<Tv *>(smem_raw + lay.offT);
            Tv *T1 = T0 + (size_t)tw * nz0;
            Tv *f0v = mixed ? (Tv *)m.f32[0] : (Tv *)m.f64[0];
            const int ntile = (n + tw - 1) / tw;
            for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
                const int j0 = t * tw;
                // interior rows only: the chain never reads a level's boundary rows
                for (int e = tid; e < tw * (nz0 - 2); e += nt) {
                    const int c = e % tw, i = 1 + e / tw, j = j0 + c;
                    double r = 0.0;
                    if (j < n) {
                        const size_t k = (size_t)i * nr + j;
                        const double pc = phi[k] + (double)delta[k], ps = phi[k - nr] + (double)delta[k - nr];
                        const double pn = phi[k + nr] + (double)delta[k + nr], pe = phi[k + 1] + (double)delta[k + 1];
                        const double pw = j > 0 ? phi[k - 1] + (double)delta[k - 1] : 0.0;
                        const double a = cz[k - nr], cc = cz[k], ee = cr[k], d = j > 0 ? cr[k - 1] : 0.0;
                        double Au = (a + cc + d + ee) * pc - a * ps - cc * pn - ee * pe;
                        if (j > 0) Au -= d * pw;
                        const double f = m.f0[k];
                        r = f - Au;
                        rmax = max(rmax, abs_bits(r));
                        if (first) {
                            double bb = f;
                            if (i == 1) bb += a * phi[k - nr];
                            if (i == nz0 - 2) bb += cc * phi[k + nr];
                            if (j == nr - 2) bb += ee * phi[k + 1];
                            bmax = max(bmax, abs_bits(bb));
                        }
                        if (L > 0) f0v[k] = (Tv)r;
                    }
                    T0[(size_t)c * nz0 + i] = (Tv)r;
                }
                __syncthreads();
                Tv *src = T0, *dst = T1;
                int nzp = nz0;
                for (int l = 1; l <= L; ++l) {
                    const int nzc = m.nz[l];
                    Tv *fl = mixed ? (Tv *)m.f32[l] : (Tv *)m.f64[l];
                    for (int e = tid; e < tw * (nzc - 2); e += nt) {
                        const int c = e % tw, I = 1 + e / tw, j = j0 + c;
                        const Tv *s = src + (size_t)c * nzp;
                        const Tv v = (Tv)0.5 * s[2 * I - 1] + s[2 * I] + (Tv)0.5 * s[2 * I + 1];
                        dst[(size_t)c * nzc + I] = v;
                        if (j < n) {
                            const size_t k = (size_t)I * nr + j;
                            if (l == L)
                                m.fc64[k] = (double)v;
                            else
                                fl[k] = v;
                        }
                    }
                    __syncthreads();
                    Tv *tmp = src;
                    src = dst;
                    dst = tmp;
                    nzp = nzc;
                }
            }
            for (int o = 16; o > 0; o >>= 1) {
                rmax = max(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
                bmax = max(bmax, __shfl_xor_sync(0xffffffffu, bmax, o));
            }
            if (lane == 0) {
                s_r[warp] = rmax;
                s_b[warp] = bmax;
            }
            __syncthreads();
            if (tid < 32) {
                unsigned long long r = tid < (nt >> 5) ? s_r[tid] : 0ull;
                unsigned long long b = tid < (nt >> 5) ? s_b[tid] : 0ull;
                for (int o = 16; o > 0; o >>= 1) {
                    r = max(r, __shfl_xor_sync(0xffffffffu, r, o));
                    b = max(b, __shfl_xor_sync(0xffffffffu, b, o));
                }
                if (tid == 0) {
                    atomicMax(&ctl->rb[cyc & 1], r);
                    if (first) atomicMax(&ctl->b_bits, b);
                }
            }
        }
        if (!count_barrier(&ctl->bar_count.v, (++ngrid) * gridDim.x, ctl)) {
            copy_wait_all();
            return;
        }
        // ---- decision: every block reads the same maxima ----
        if (tid == 0) {
            const double rn = __longlong_as_double((long long)*(volatile unsigned long long *)&ctl->rb[cyc & 1]);
            const double bn = __longlong_as_double((long long)*(volatile unsigned long long *)&ctl->b_bits);
            int d = 0;  // 0 continue, 1 converged, 2 out of cycles, 3 zero right-hand side
            if (bn == 0.0)
                d = 3;
            else if (ctl->tol > 0.0 && rn <= ctl->tol * bn)
                d = 1;
            else if (cyc >= ctl->max_cycles)
                d = ctl->tol > 0.0 ? 2 : 1;
            s_decide = d;
            if (blockIdx.x == 0) {
                ctl->last_res = rn;
                ctl->bnorm = bn;
                ctl->cycles = cyc;
                ctl->rb[(cyc + 1) & 1] = 0ull;  // read by all blocks one cycle ago
                if (d == 1) ctl->converged = 1;
                if (d == 3) ctl->zero_rhs = 1;
            }
        }
        __syncthreads();
        const int decide = s_decide;
        first = 0;
        if (decide == 3) {
            for (int k = blockIdx.x * nt + tid; k < ng; k += gridDim.x * nt) {
                const int i = k / nr, j = k % nr;
                if (i > 0 && i < nz0 - 1 && j < nr - 1) phi[k] = 0.0;
            }
            copy_wait_all();
            return;
        }
        // the pending correction goes into phi (also on the way out); nothing
        // reads phi again before the next residual
        if (L > 0)
            for (int k = blockIdx.x * nt + tid; k < ng; k += gridDim.x * nt) {
                const int i = k / nr, j = k % nr;
                if (i > 0 && i < nz0 - 1 && j < nr - 1) phi[k] += (double)delta[k];
            }
        if (decide != 0) {
            copy_wait_all();
            return;
        }
        if (L == 0) {
            // nz = 3: the single interior row of phi, exactly
            if (blockIdx.x == 0) {
                double *D = reinterpret_cast<double *>(smem_raw + lay.offD);
                double *F = reinterpret_cast<double *>(smem_raw + lay.offR0);
                copy_async(F, m.facc, FE * 8, tid, nt);
                copy_commit();
                double rhs = 0.0;
                const bool act = tid < n;
                if (act) {
                    const double *cz = m.cz[0], *cr = m.cr[0];
                    const size_t k = (size_t)nr + tid;
                    rhs = m.f0[k] + cz[k - nr] * phi[k - nr] + cz[k] * phi[k + nr];
                    if (tid == n - 1) rhs += cr[k] * phi[k + 1];
                }
                const double x = pcr_line<double>(rhs, D, D + n, F, n, K, tid, act, false);
                if (act) phi[(size_t)nr + tid] = x;
            }
            if (!count_barrier(&ctl->bar_count.v, (++ngrid) * gridDim.x, ctl)) return;
            continue;
        }
        // level 0's sweeps rewrite delta: when they run in the group alone,
        // every block's update of phi has to be in first
        if (lb == 0)
            if (!count_barrier(&ctl->bar_count.v, (++ngrid) * gridDim.x, ctl)) {
                copy_wait_all();
                return;
            }
        // ---- up: per level, each black line with the two red lines beside it ----
        bool have = false;  // this block's first red factors of the level are requested
        for (int l = L - 1; l >= 0; --l) {
            const bool grp = l >= lb;
            const int P = grp ? G : (int)gridDim.x;
            const int nzl = m.nz[l], nzc = m.nz[l + 1];
            const int NB = (nzl - 3) / 2;  // black lines
            const int nq = units_of(nzl);
            Tv *u = mixed ? (Tv *)m.u32[l] : (Tv *)m.u64[l];
            const Tv *uc = mixed ? (const Tv *)m.u32[l + 1] : (const Tv *)m.u64[l + 1];
            const Tv *f = mixed ? (const Tv *)m.f32[l] : (const Tv *)m.f64[l];
            const Tv *cz = mixed ? (const Tv *)m.cz32[l] : (const Tv *)m.cz[l];
            const Tv *fac = mixed ? (const Tv *)m.fac32[l] : (const Tv *)m.fac64[l];
            if ((int)blockIdx.x < P) {
                if (l == L - 1 && blockIdx.x == 0) {
                    // the coarsest row (FP64 factors), then level L-1 in this block alone
                    double *D = reinterpret_cast<double *>(smem_raw + lay.offD);
                    double *F = reinterpret_cast<double *>(smem_raw + lay.offR0);
                    if (!cpre) copy_async(F, m.facc, FE * 8, tid, nt);
                    copy_commit();
                    const bool act = tid < n;
                    const double rhs = act ? m.fc64[(size_t)nr + tid] : 0.0;
                    const double x = pcr_line<double>(rhs, D, D + n, F, n, K, tid, act, false);
                    Tv *ucw = mixed ? (Tv *)m.u32[L] : (Tv *)m.u64[L];
                    if (act) ucw[(size_t)nr + tid] = (Tv)x;
                    __syncthreads();
                    have = false;
                }
                for (int q = blockIdx.x; q < nq; q += P) {
                    const int ra = 2 * q + 1, rb = 2 * q + 3, ib = 2 * q + 2;
                    const bool hasb = NB >= 1;
                    // factor requests: the reds (unless already in), then the black
                    if (!(have && q == (int)blockIdx.x)) {
                        if (lay.pair) {
                            copy_async(R0, fac + (size_t)(ra - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                            if (hasb) copy_async(R1, fac + (size_t)(rb - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                        } else {
                            copy_async(R0, fac + (size_t)(ra - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                        }
                    }
                    copy_commit();
                    if (hasb && bsep) copy_async(FBk, fac + (size_t)(ib - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                    copy_commit();
                    have = false;
                    // the black line's own inputs do not depend on the reds: load them first
                    Tv fb = 0, cb0 = 0, cb1 = 0;
                    if (hasb && tid < n) {
                        const size_t k = (size_t)ib * nr + tid;
                        fb = f[k];
                        cb0 = cz[k - nr];
                        cb1 = cz[k];
                    }
                    // red right-hand sides: f plus the coarse correction injected at rows i -/+ 1
                    auto red_rhs = [&](int i, int j) -> Tv {
                        const size_t k = (size_t)i * nr + j;
                        const int Idn = (i - 1) / 2, Iup = (i + 1) / 2;
                        const Tv udn = (Idn > 0 && Idn < nzc - 1) ? uc[(size_t)Idn * nr + j] : (Tv)0;
                        const Tv uup = (Iup > 0 && Iup < nzc - 1) ? uc[(size_t)Iup * nr + j] : (Tv)0;
                        return f[k] + cz[k - nr] * udn + cz[k] * uup;
                    };
                    if (lay.pair) {
                        const int i = half ? rb : ra;
                        const bool act = jl < n && (half == 0 || hasb);
                        const Tv rhs = act ? red_rhs(i, jl) : (Tv)0;
                        const Tv x = pcr_line<Tv>(rhs, Dh, Dh + n, half ? R1 : R0, n, K, jl, act, true);
                        if (act) {
                            X[half * n + jl] = x;
                            // red rb is also the next black's red ra: one block writes it
                            if (half == 0 || q == NB - 1) u[(size_t)i * nr + jl] = x;
                        }
                    } else {
                        const bool act = tid < n;
                        Tv rhs = act ? red_rhs(ra, tid) : (Tv)0;
                        Tv x = pcr_line<Tv>(rhs, Dh, Dh + n, R0, n, K, tid, act, true);
                        if (act) {
                            X[tid] = x;
                            u[(size_t)ra * nr + tid] = x;
                        }
                        if (hasb) {
                            copy_async(R0, fac + (size_t)(rb - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                            copy_commit();
                            rhs = act ? red_rhs(rb, tid) : (Tv)0;
                            x = pcr_line<Tv>(rhs, Dh, Dh + n, R0, n, K, tid, act, false);
                            if (act) {
                                X[n + tid] = x;
                                if (q == NB - 1) u[(size_t)rb * nr + tid] = x;
                            }
                        }
                    }
                    if (hasb) {
                        __syncthreads();  // X complete
                        Tv *F = FBk;
                        if (!bsep) {
                            copy_async(R0, fac + (size_t)(ib - 1) * FE, FE * (int)sizeof(Tv), tid, nt);
                            copy_commit();
                            F = R0;
                        }
                        const bool act = tid < n;
                        const Tv rhs = act ? fb + cb0 * X[tid] + cb1 * X[n + tid] : (Tv)0;
                        Tv *D = reinterpret_cast<Tv *>(smem_raw + lay.offD);
                        const Tv x = pcr_line<Tv>(rhs, D, D + n, F, n, K, tid, act, false);
                        if (act) u[(size_t)ib * nr + tid] = x;
                    }
                }
                // request the next level's first red factors of this block
                if (l > 0) {
                    const int ln = l - 1;
                    const int Pn = ln >= lb ? G : (int)gridDim.x;
                    const int nqn = units_of(m.nz[ln]);
                    if ((int)blockIdx.x < Pn && (int)blockIdx.x < nqn) {
                        const Tv *facn = mixed ? (const Tv *)m.fac32[ln] : (const Tv *)m.fac64[ln];
                        const int q = blockIdx.x;
                        copy_async(R0, facn + (size_t)(2 * q) * FE, FE * (int)sizeof(Tv), tid, nt);
                        if (lay.pair && (m.nz[ln] - 3) / 2 >= 1)
                            copy_async(R1, facn + (size_t)(2 * q + 2) * FE, FE * (int)sizeof(Tv), tid, nt);
                        have = true;
                    }
                    copy_commit();
                }
            }
            // levels in the group alone are separated by the group barrier;
            // every other level boundary is a grid barrier
            bool ok;
            if (l > 0 && grp && l - 1 >= lb)
                ok = in_group ? count_barrier(&ctl->gbar_count.v, (++ngroup) * G, ctl) : true;
            else
                ok = count_barrier(&ctl->bar_count.v, (++ngrid) * gridDim.x, ctl);
            if (!ok) {
                copy_wait_all();
                return;
            }
        }
    }
}

// kernels whose dynamic shared memory can pass 48 KB on the largest meshes
constexpr size_t kSolveSmemLimit = 220 * 1024;

void raise_smem_limits() {
    static bool done = false;
    if (done) return;
    const int lim = (int)kSolveSmemLimit;
    cudaFuncSetAttribute(k_factor_levels<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_factor_levels<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_chi_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_chain<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_chain<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_solve_persistent<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    cudaFuncSetAttribute(k_solve_persistent<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    done = true;
}

int line_threads(int n) {
    int t = 32;
    while (t < n && t < 1024) t <<= 1;
    return t;
}

int pcr_steps(int n) {
    int K = 0;
    for (int s = 1; s < n; s <<= 1) ++K;
    return K;
}

}  // namespace

size_t mg_fast_factor_elems(int nz, int nr, bool mixed, size_t *n32) {
    const int n = nr - 1, K = pcr_steps(n);
    size_t e64 = 0, e32 = 0;
    int nl = 0;
    for (int z = nz;; z = (z + 1) / 2) {
        const size_t lines = (size_t)(z - 2);
        const bool coarsest = (z == 3);
        const size_t e = lines * (2 * K + 1) * n;
        if (coarsest || !mixed)
            e64 += e;
        else
            e32 += e;
        ++nl;
        if (z == 3) break;
    }
    if (n32) *n32 = e32;
    return e64;
}

int mg_fast_solve(const FieldDims &fd, MGFast &m, const double *rho, const double *chi, double V,
                  const double *phi_zL, double *phi, bool warm, bool mixed, double tol,
                  int max_cycles, double *rel_res, int *launches, cudaStream_t st) {
    const int nz = fd.nz, nr = fd.nr, n = nr - 1, ng = nz * nr;
    const int K = pcr_steps(n);
    const int nlev = m.nlev;
    int L = 0;
    const int lt = line_threads(n);
    raise_smem_limits();
    MGFast *mp = m.self;
    cudaMemcpyAsync(mp, &m, sizeof(MGFast), cudaMemcpyHostToDevice, st);
    // set-up: levels' chi, coefficients, line factors, right-hand side and boundary data
    cudaMemcpyAsync(m.chi[0], chi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st);
    if (nlev > 1) {
        k_chi_levels<<<(nr + 7) / 8, 256, (size_t)8 * 2 * nz * sizeof(double), st>>>(mp, nr);
        ++L;
    }
    int total = 0;
    for (int l = 0; l < nlev; ++l) total += m.nz[l] * nr;
    k_coefs_levels<<<(total + 255) / 256, 256, 0, st>>>(mp, nr, fd.dr, fd.chi_face == PIC_CHI_MEAN,
                                                         total);
    ++L;
    {
        // line factors: FP64 for the FP64 path and for the coarsest level,
        // FP32 for the mixed path's other levels
        int lines_all = 0, lines_fine = 0;
        for (int l = 0; l < nlev; ++l) {
            lines_all += m.nz[l] - 2;
            if (l < nlev - 1) lines_fine += m.nz[l] - 2;
        }
        if (!mixed) {
            k_factor_levels<double><<<lines_all, lt, 7 * n * sizeof(double), st>>>(mp, 0, nlev, nr, K);
            ++L;
        } else {
            if (lines_fine > 0) {
                k_factor_levels<float><<<lines_fine, lt, 7 * n * sizeof(float), st>>>(mp, 0, nlev - 1, nr, K);
                ++L;
            }
            k_factor_levels<double><<<1, lt, 7 * n * sizeof(double), st>>>(mp, nlev - 1, nlev, nr, K);
            ++L;
        }
    }
    k_rhs_bc<<<(ng + 255) / 256, 256, 0, st>>>(rho, m.f0, phi, phi_zL, V, nz, nr, fd.dz, fd.dr,
                                               warm ? 0 : 1);
    ++L;
    // the level-0 correction starts at zero and stays zero on the boundary
    if (mixed)
        cudaMemsetAsync(m.u32[0], 0, sizeof(float) * ng, st);
    else
        cudaMemsetAsync(m.u64[0], 0, sizeof(double) * ng, st);
    MGCtl c0;
    memset(&c0, 0, sizeof(c0));
    c0.tol = tol;
    c0.max_cycles = max_cycles;
    cudaMemcpyAsync(m.ctl, &c0, sizeof(MGCtl), cudaMemcpyHostToDevice, st);
    // one cooperative launch for all cycles when the blocks fit on the GPU
    {
        int dev = 0, nsm = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t limit = std::min<size_t>((size_t)std::max(optin - 2048, 0), kSolveSmemLimit);
        SolveLayout lay{};
        size_t sp = 0;
        bool found = false;
        const size_t es = mixed ? sizeof(float) : sizeof(double);
        const size_t FE = (size_t)(2 * K + 1) * n;
        // richest layout first: both reds at once, black factors and the
        // residual tile in their own space; then less overlap, then one red
        // line at a time
        for (int v = 0; v < 6 && !found; ++v) {
            const int pair = v < 3;
            const int mode = v % 3;  // 0: separate B and T, 1: separate T, 2: T over R
            if (pair && 2 * lt > 1024) continue;
            size_t off = 0;
            auto take = [&](size_t b) {
                const size_t o = off;
                off += (b + 15) & ~(size_t)15;
                return (int)o;
            };
            lay.tw = 8;
            lay.lt = lt;
            lay.pair = pair;
            lay.offD = take((size_t)(pair ? 2 : 1) * 2 * n * sizeof(double));
            lay.offX = take((size_t)2 * n * es);
            const size_t Tb = (size_t)2 * lay.tw * nz * sizeof(double);
            size_t Rb = std::max((size_t)(pair ? 2 : 1) * FE * es, FE * sizeof(double));
            if (mode == 2) Rb = std::max(Rb, Tb);
            lay.offR0 = take(Rb);
            lay.offR1 = pair ? lay.offR0 + (int)(FE * es) : lay.offR0;
            lay.offB = mode == 0 ? take(FE * es) : lay.offR0;
            lay.offT = mode == 2 ? lay.offR0 : take(Tb);
            sp = off;
            found = sp <= limit;
        }
        const int threads = lay.pair ? 2 * lt : lt;
        int per_sm = 0;
        if (found) {
            if (mixed)
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_persistent<float>, threads, sp);
            else
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_persistent<double>, threads, sp);
        }
        const int grid = std::max(1, std::min(std::min(nsm, nsm * per_sm), (nz - 1) / 2));
        if (found && per_sm >= 1) {
            int first_cycle = 1;
            int Kv = K, nrv = nr;
            void *args[] = {(void *)&mp, (void *)&phi, (void *)&nrv, (void *)&Kv, (void *)&first_cycle,
                            (void *)&lay};
            cudaError_t e = mixed ? cudaLaunchCooperativeKernel((void *)k_solve_persistent<float>, grid, threads,
                                                                args, sp, st)
                                  : cudaLaunchCooperativeKernel((void *)k_solve_persistent<double>, grid, threads,
                                                                args, sp, st);
            ++L;
            if (e == cudaSuccess) {
                MGCtl ch;
                cudaMemcpyAsync(&ch, m.ctl, sizeof(MGCtl), cudaMemcpyDeviceToHost, st);
                cudaStreamSynchronize(st);
                if (launches) *launches += L;
                if (ch.timeout) {
                    if (rel_res) *rel_res = 0.0;
                    return kSolveTimeout;
                }
                if (ch.zero_rhs) {
                    if (rel_res) *rel_res = 0.0;
                    return 0;
                }
                if (rel_res) *rel_res = ch.bnorm > 0 ? ch.last_res / ch.bnorm : 0.0;
                return ch.converged ? ch.cycles : -ch.cycles - 1;
            }
            cudaGetLastError();  // fall back to one launch per phase
        }
    }
    const int gres = std::max(1, std::min((ng + 255) / 256, 152 * 2));
    const int gchain = (n + 31) / 32;
    const size_t schain = nlev > 1 ? (size_t)nz * 32 * sizeof(double) +
                                         (size_t)2 * m.nz[1] * 32 * (mixed ? sizeof(float) : sizeof(double))
                                   : 0;
    bool first = true;
    MGCtl ch;
    int batch = 4;
    for (;;) {
        for (int b = 0; b < batch; ++b) {
            k_resid<<<gres, 256, 0, st>>>(mp, nr, phi, first ? 1 : 0);
            ++L;
            first = false;
            if (nlev > 1) {
                if (mixed)
                    k_chain<float><<<gchain, 32, schain, st>>>(mp, nr);
                else
                    k_chain<double><<<gchain, 32, schain, st>>>(mp, nr);
                ++L;
            }
            if (nlev == 1) {
                k_single_row<<<1, lt, 2 * n * sizeof(double), st>>>(mp, phi, nr, K);
                ++L;
                continue;
            }
            if (mixed)
                k_coarse<float><<<1, lt, 2 * n * sizeof(double), st>>>(mp, nr, K);
            else
                k_coarse<double><<<1, lt, 2 * n * sizeof(double), st>>>(mp, nr, K);
            ++L;
            for (int l = nlev - 2; l >= 0; --l) {
                const int nzl = m.nz[l];
                const int nred = (nzl - 1) / 2, nblack = (nzl - 3) / 2;
                if (!mixed) {
                    double *u = l == 0 ? phi : m.u64[l];
                    const double *f = l == 0 ? m.f0 : m.f64[l];
                    k_red<double><<<nred, lt, 2 * n * sizeof(double), st>>>(
                        mp, l, nr, K, u, m.u64[l + 1], f, m.cz[l], m.cr[l], m.fac64[l], l == 0);
                    if (nblack > 0)
                        k_black<double><<<nblack, lt, 2 * n * sizeof(double), st>>>(
                            mp, l, nr, K, u, f, m.cz[l], m.cr[l], m.fac64[l], l == 0);
                } else {
                    k_red<float><<<nred, lt, 2 * n * sizeof(float), st>>>(
                        mp, l, nr, K, m.u32[l], m.u32[l + 1], m.f32[l], m.cz32[l], m.cr32[l],
                        m.fac32[l], 0);
                    if (nblack > 0)
                        k_black<float><<<nblack, lt, 2 * n * sizeof(float), st>>>(
                            mp, l, nr, K, m.u32[l], m.f32[l], m.cz32[l], m.cr32[l], m.fac32[l], 0);
                }
                L += nblack > 0 ? 2 : 1;
            }
            if (mixed) {
                k_correct<<<(ng + 255) / 256, 256, 0, st>>>(mp, phi, m.u32[0], nz, nr);
                ++L;
            }
        }
        cudaMemcpyAsync(&ch, m.ctl, sizeof(MGCtl), cudaMemcpyDeviceToHost, st);
        cudaStreamSynchronize(st);
        if (ch.done) break;
        // the residual falls by roughly a constant factor per cycle: size the
        // next batch by the cycles still needed
        batch = 2;
        if (ch.cycles >= 2 && ch.last_res > 0 && ch.tol > 0) {
            const double need = log(ch.tol * ch.bnorm / ch.last_res);
            const double per = log(0.12);
            const int est = (int)ceil(need / per);
            batch = std::max(1, std::min(est + 1, 6));
        }
    }
    if (ch.zero_rhs) {
        k_rhs_bc<<<(ng + 255) / 256, 256, 0, st>>>(rho, m.f0, phi, phi_zL, V, nz, nr, fd.dz, fd.dr, 1);
        ++L;
        if (rel_res) *rel_res = 0.0;
        if (launches) *launches += L;
        return 0;
    }
    if (rel_res) *rel_res = ch.bnorm > 0 ? ch.last_res / ch.bnorm : 0.0;
    if (launches) *launches += L;
    return ch.converged ? ch.cycles : -ch.cycles - 1;
}

}  // namespace pic
