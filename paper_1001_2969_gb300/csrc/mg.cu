// mg.cu -- the multigrid field solve of the timestep (Sec. 2.5, Algorithm 1),
// arranged for one launch and little FP64 work on GB300.
//
// Same method as the oracle and as the reference GPU multigrid in field.cu:
// finite-volume operator, z-only coarsening, V(0,1) cycles with a red-black
// r-line sweep per level on the way up, [1/2 1 1/2] restriction of
// volume-integrated residuals, linear prolongation in z.  What changes is the
// arrangement:
//  - every r-line of every level is factored once per solve (the line
//    matrices do not change between cycles) for a warp-level solver: Thomas
//    on a chunk of the line per lane, the chunks' interface unknowns by
//    parallel cyclic reduction over the lanes;
//  - the whole solve is one cooperative launch: the residual and the
//    restriction chain run over tiles of columns, convergence is decided on
//    the device, and a block sweeps one black line with the two red lines
//    beside it, so one barrier separates two levels;
//  - prolongation is folded into the red sweep: red (odd) rows are
//    recomputed whole by their line solve, so only the injection of the
//    coarse correction into the black (even) neighbour rows is ever used;
//  - the cycle works on the correction of phi; the mixed path keeps the
//    correction, the coarse right-hand sides and the line factors in FP32
//    and the residual in FP64 (iterative refinement).
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

// ---- set-up ----

// nodal chi of every coarse level: full weighting in z, injection on the
// boundary rows; one warp per column, lanes over rows, levels in shared memory
__global__ void k_chi_levels(const MGFast *__restrict__ mp, int nr, const StepCtl *ctl) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const MGFast &m = *mp;
    if (ctl && ctl->halt) return;
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
__global__ void k_coefs_levels(const MGFast *__restrict__ mp, int nr, int face_mean, int total, const StepCtl *ctl) {
    const MGFast &m = *mp;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= total || (ctl && ctl->halt)) return;
    int l = 0, k = g;
    while (k >= m.nz[l] * nr) {
        k -= m.nz[l] * nr;
        ++l;
    }
    const int nz = m.nz[l], i = k / nr, j = k % nr;
    const double *chi = m.chi[l];
    const double c = chi[k];
    double vz = 0.0, vr = 0.0;
    if (i + 1 < nz) {
        const double cn = chi[k + nr];
        const double f = face_mean ? 0.5 * (c + cn) : fmax(c, cn);
        vz = (1.0 + f) * m.gz[l][j];
    }
    if (j + 1 < nr) {
        const double cn = chi[k + 1];
        const double f = face_mean ? 0.5 * (c + cn) : fmax(c, cn);
        vr = (1.0 + f) * m.gr[l][j];
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

// ---- r-line factors for the warp line solve ----
//
// Line system of row i: lo_j x_{j-1} + dg_j x_j + up_j x_{j+1} = b_j with
// lo_j = -cr[i][j-1] (0 on the axis), dg_j = a + c + d + e, up_j = -cr[i][j]
// (0 on the last unknown).  One warp solves a line: lane p owns the chunk
// j = pM .. pM + M - 1 (unknowns past n are x = 0 rows).  The chunk's last
// unknown is its interface I_p; the M - 1 interior unknowns are
//     y = z + I_{p-1} v + I_p w,
// z the interior solution with zero neighbours (Thomas), v and w the
// responses to the two neighbouring interfaces.  Substituting into the
// interface equations leaves a tridiagonal system in I_0..I_31, which the
// warp reduces by parallel cyclic reduction over lanes (shuffles).  Only the
// right-hand side changes between cycles, so all of this except the
// right-hand-side sweeps is computed once per solve.  Per line the factors
// are, lane-minor ([arr][k][32]):
//   ell (forward multipliers), invd (1/pivot), cp (up * invd), v, w
//   (5 arrays of M), then loI, upI (interface couplings), the five PCR
//   steps' alpha and gamma, and 1/diagonal of the reduced system.
constexpr int kLine = 32;  // lanes per line

__host__ __device__ constexpr int line_factor_elems(int M) { return 5 * M * kLine + 2 * kLine + 10 * kLine + kLine; }

// chunk per lane: the least power of two M with 32 M >= n
inline int line_chunk(int n) {
    int M = 1;
    while (kLine * M < n) M <<= 1;
    return M;
}

// One warp per line over all lines of levels [l0, l1).  Computed in Ts.
template <typename Ts>
__global__ void k_factor_lines(const MGFast *__restrict__ mp, int l0, int l1, int nr, int M, int nlines,
                               const StepCtl *ctl) {
    const MGFast &m = *mp;
    if (ctl && ctl->halt) return;
    const int n = nr - 1;
    const int p = threadIdx.x & 31;
    int g = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (g >= nlines) return;
    int l = l0;
    while (l < l1 && g >= m.nz[l] - 2) {
        g -= m.nz[l] - 2;
        ++l;
    }
    if (l >= l1) return;
    const bool f64 = sizeof(Ts) == 8;
    const Ts *cz = f64 ? (const Ts *)m.cz[l] : (const Ts *)m.cz32[l];
    const Ts *cr = f64 ? (const Ts *)m.cr[l] : (const Ts *)m.cr32[l];
    Ts *fac = (l == m.nlev - 1) ? (f64 ? (Ts *)m.facc : (Ts *)m.facc32)
                                : (f64 ? (Ts *)m.fac64[l] : (Ts *)m.fac32[l]);
    Ts *F = fac + (size_t)g * line_factor_elems(M);
    const size_t rowk = (size_t)(1 + g) * nr;
    auto coef = [&](int k, Ts &lo, Ts &dg, Ts &up) {
        const int j = p * M + k;
        if (j >= n) {
            lo = 0;
            dg = 1;
            up = 0;
            return;
        }
        const size_t q = rowk + j;
        const Ts a = cz[q - nr], c = cz[q], e = cr[q];
        const Ts d = j > 0 ? cr[q - 1] : (Ts)0;
        lo = -d;
        dg = a + c + d + e;
        up = j < n - 1 ? -e : (Ts)0;
    };
    auto at = [&](int arr, int k) -> Ts & { return F[((size_t)arr * M + k) * kLine + p]; };
    const int MI = M - 1;
    Ts A, B, C;  // reduced (interface) equation of this lane
    Ts loI, dgI, upI;
    coef(M - 1, loI, dgI, upI);
    if (MI > 0) {
        // interior Thomas factors
        Ts lo, dg, up, upm = 0, invd = 0;
        for (int k = 0; k < MI; ++k) {
            coef(k, lo, dg, up);
            Ts ell = 0, d = dg;
            if (k > 0) {
                ell = lo * invd;
                d = dg - ell * upm;
            }
            invd = recip(d);
            at(0, k) = ell;
            at(1, k) = invd;
            at(2, k) = up * invd;
            upm = up;
        }
        // spikes: v answers -lo_0 at the first interior unknown, w answers
        // -up_{MI-1} at the last (forward sweep, then backward)
        Ts lo0, dg0, up0;
        coef(0, lo0, dg0, up0);
        Ts vp = -lo0;
        at(3, 0) = vp;
        for (int k = 1; k < MI; ++k) {
            vp = -at(0, k) * vp;
            at(3, k) = vp;
        }
        Ts loL, dgL, upL;
        coef(MI - 1, loL, dgL, upL);
        Ts vn = at(3, MI - 1) * at(1, MI - 1), wn = -upL * at(1, MI - 1);
        at(3, MI - 1) = vn;
        at(4, MI - 1) = wn;
        for (int k = MI - 2; k >= 0; --k) {
            vn = at(3, k) * at(1, k) - at(2, k) * vn;
            wn = -at(2, k) * wn;
            at(3, k) = vn;
            at(4, k) = wn;
        }
        const Ts v0n = __shfl_down_sync(0xffffffffu, at(3, 0), 1);
        const Ts w0n = __shfl_down_sync(0xffffffffu, at(4, 0), 1);
        const Ts vL = at(3, MI - 1), wL = at(4, MI - 1);
        A = loI * vL;
        B = dgI + loI * wL + (p < kLine - 1 ? upI * v0n : (Ts)0);
        C = p < kLine - 1 ? upI * w0n : (Ts)0;
    } else {
        A = loI;
        B = dgI;
        C = upI;
    }
    Ts *Gf = F + (size_t)5 * M * kLine;
    Gf[p] = loI;
    Gf[kLine + p] = upI;
    // parallel cyclic reduction of the interface system over the lanes
    for (int st = 0; st < 5; ++st) {
        const int s = 1 << st;
        const Ts Bm = __shfl_up_sync(0xffffffffu, B, s), Bp = __shfl_down_sync(0xffffffffu, B, s);
        const Ts Am = __shfl_up_sync(0xffffffffu, A, s), Ap = __shfl_down_sync(0xffffffffu, A, s);
        const Ts Cm = __shfl_up_sync(0xffffffffu, C, s), Cp = __shfl_down_sync(0xffffffffu, C, s);
        Ts al = 0, ga = 0;
        if (p >= s) al = -A * recip(Bm);
        if (p + s < kLine) ga = -C * recip(Bp);
        Gf[2 * kLine + st * kLine + p] = al;
        Gf[7 * kLine + st * kLine + p] = ga;
        const Ts nB = B + (p >= s ? al * Cm : (Ts)0) + (p + s < kLine ? ga * Ap : (Ts)0);
        A = p >= s ? al * Am : (Ts)0;
        C = p + s < kLine ? ga * Cp : (Ts)0;
        B = nB;
    }
    Gf[12 * kLine + p] = recip(B);
}

// Warp solve of one line with factors F (shared memory): right-hand side in
// Bs and solution out to the same place, both [k * 33 + p] (lane-minor with
// a pad against bank conflicts).  All 32 lanes take part.
constexpr int kRow = 33;

template <typename Ts, int M>
__device__ __forceinline__ void warp_line_solve(const Ts *__restrict__ F, Ts *Bs, int p) {
    constexpr int MI = M - 1;
    const Ts *Gf = F + 5 * M * kLine;
    Ts r;
    Ts z[MI > 0 ? MI : 1];
    if constexpr (MI > 0) {
        Ts zp = Bs[p];
        z[0] = zp;
#pragma unroll
        for (int k = 1; k < MI; ++k) {
            zp = Bs[k * kRow + p] - F[(0 * M + k) * kLine + p] * zp;
            z[k] = zp;
        }
        Ts zn = z[MI - 1] * F[(1 * M + MI - 1) * kLine + p];
        z[MI - 1] = zn;
#pragma unroll
        for (int k = MI - 2; k >= 0; --k) {
            zn = z[k] * F[(1 * M + k) * kLine + p] - F[(2 * M + k) * kLine + p] * zn;
            z[k] = zn;
        }
        const Ts z0n = __shfl_down_sync(0xffffffffu, z[0], 1);
        r = Bs[(M - 1) * kRow + p] - Gf[p] * z[MI - 1] - Gf[kLine + p] * (p < kLine - 1 ? z0n : (Ts)0);
    } else {
        r = Bs[p];
    }
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int s = 1 << st;
        const Ts rm = __shfl_up_sync(0xffffffffu, r, s), rp = __shfl_down_sync(0xffffffffu, r, s);
        r = r + Gf[(2 + st) * kLine + p] * rm + Gf[(7 + st) * kLine + p] * rp;
    }
    const Ts I = r * Gf[12 * kLine + p];
    if constexpr (MI > 0) {
        const Ts Ip = __shfl_up_sync(0xffffffffu, I, 1);  // lane 0: v is zero there
#pragma unroll
        for (int k = 0; k < MI; ++k) Bs[k * kRow + p] = z[k] + F[(3 * M + k) * kLine + p] * Ip + F[(4 * M + k) * kLine + p] * I;
    }
    Bs[(M - 1) * kRow + p] = I;
}

// right-hand side rho A_j dz / eps0 and the Dirichlet data of phi; with
// phi_prev (a warm solve) the interior starts from 2 phi - phi_prev, the
// linear extrapolation in time of the last two steps' potentials, and
// phi_prev takes the last step's
__global__ void k_rhs_bc(const MGFast *__restrict__ mp, const double *rho, double *phi, const double *phi_zL,
                         double V_arg, int nz, int nr, int cold, const StepCtl *ctl, int v_from_ctl,
                         double *phi_prev) {
    const MGFast &m = *mp;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr || (ctl && ctl->halt)) return;
    const double V = (ctl && v_from_ctl) ? ctl->V : V_arg;  // in a timestep the source voltage comes with the step
    const int i = k / nr, j = k % nr;
    double v = 0.0, dg = 0.0;
    if (i > 0 && i < nz - 1 && j < nr - 1) {
        v = rho[k] * m.ga[j];
        const double *cz = m.cz[0], *cr = m.cr[0];
        dg = cz[k - nr] + cz[k] + (j > 0 ? cr[k - 1] : 0.0) + cr[k];
    }
    m.f0[k] = v;
    m.dg0[k] = dg;
    double p;
    if (i == 0)
        p = (j == nr - 1) ? 0.0 : V;
    else if (i == nz - 1)
        p = phi_zL ? phi_zL[j] : 0.0;
    else if (j == nr - 1)
        p = 0.0;
    else if (cold)
        p = 0.0;
    else if (phi_prev) {
        const double t = phi[k];
        p = 2.0 * t - phi_prev[k];
        phi_prev[k] = t;
    } else
        p = phi[k];
    phi[k] = p;
    // the solve alternates between phi and a copy (both carry the boundary
    // values); the level-0 correction starts at zero (and stays zero on the
    // boundary); the solve's control block starts cleared
    m.phi2[k] = p;
    if (m.u32[0])
        m.u32[0][k] = 0.0f;
    else
        m.u64[0][k] = 0.0;
    for (int w = k; w < (int)(sizeof(MGCtl) / sizeof(unsigned)); w += nz * nr)
        reinterpret_cast<unsigned *>(m.ctl)[w] = 0u;
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
//      i = 2q + 2 solves the red lines 2q + 1 and 2q + 3 beside it (two
//      warps at once), keeps them in shared memory and solves the black
//      line.  A red line shared by two blocks is computed by both from the
//      same data, bit for bit, and stored by one.  So one barrier separates
//      two levels instead of two.
// The coarsest row is solved by block 0 in the phase of level L-1, which
// block 0 sweeps alone.  Levels with at most kBarGroup black lines belong to
// the first kBarGroup blocks, separated by a barrier among those blocks only;
// the rest of the grid waits at the next full barrier.
// ---------------------------------------------------------------------------
constexpr int kBarGroup = 8;  // blocks that sweep the coarse levels alone

// ---- factor lines into shared memory ----
// A line's factors move in one bulk copy that completes on the region's
// mbarrier (thread 0 issues it).  All threads of the block keep the same
// state: the parity of the next completion and whether a copy is pending.
struct Loader {
    unsigned mbar;
    unsigned phase;
    int pending;
};

__device__ __forceinline__ void ld_begin(Loader &q, unsigned bytes) {
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(q.mbar), "r"(bytes) : "memory");
    }
    q.pending = 1;
}

// sizes and addresses are multiples of 16 bytes
__device__ __forceinline__ void ld_copy(Loader &q, void *dst, const void *src, unsigned bytes) {
    if (threadIdx.x == 0)
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src), "r"(bytes), "r"(q.mbar)
                     : "memory");
}

// wait for the region's copy (every thread of the block calls it); false,
// for the whole block, when the bounded wait gave up
__device__ __forceinline__ bool ld_wait(Loader &q) {
    if (!q.pending) return true;
    bool ok = false;
    for (long long it = 0; it < kSpinLimit && !ok; ++it) {
        unsigned done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(done)
            : "r"(q.mbar), "r"(q.phase)
            : "memory");
        ok = done != 0;
    }
    ok = !__syncthreads_or(!ok);
    if (ok) {
        q.pending = 0;
        q.phase ^= 1u;
    }
    return ok;
}

// black lines of a level with nz rows (at least one unit of work: nz = 3 has
// a red line only)
__device__ __forceinline__ int units_of(int nz) { return max((nz - 3) / 2, 1); }

constexpr int kSolveThreads = 256;
constexpr int kU = 4;   // elements per thread and batch in the residual phase
constexpr int kUL = 4;  // unknowns per thread and batch of a level's right-hand sides

// MINB: blocks per SM the registers must allow.  One (the compiler then
// takes ~200 registers) is a little faster for a reactor's solve alone; two
// (127 registers, no spills) lets the solves of a batch of reactors share
// SMs, and the batch step runs ~28 % faster with it.
// One reactor's solve on nbk blocks (bid: this block's index among them).
template <typename Tv, int M>
__device__ __forceinline__ void solve_body(const MGFast *__restrict__ mp, double *phi, int nr, int first_cycle,
                                           const SolveLayout &lay, double tol, int max_cycles,
                                           const StepCtl *sctl, const int bid, const int nbk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if (sctl && sctl->halt) return;  // an earlier failure of this step
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nt = blockDim.x;
    // the level table in shared memory: every grid barrier's acquire drops
    // L1, and a table read from L2 before each level's loads would put an L2
    // round trip in front of every phase
    __shared__ __align__(16) MGFast s_m;
    {
        static_assert(sizeof(MGFast) % 8 == 0, "the level table is copied in 8-byte words");
        const unsigned long long *src = reinterpret_cast<const unsigned long long *>(mp);
        unsigned long long *dst = reinterpret_cast<unsigned long long *>(&s_m);
        for (int k = tid; k < (int)(sizeof(MGFast) / 8); k += nt) dst[k] = src[k];
        __syncthreads();
    }
    const MGFast &m = s_m;
    MGCtl *ctl = m.ctl;
    const int n = nr - 1, nz0 = m.nz[0], ng = nz0 * nr, L = m.nlev - 1;
    constexpr int NW = kLine * M;  // unknowns of a line with its padding
    const bool mixed = sizeof(Tv) == 4;
    Tv *delta = mixed ? (Tv *)m.u32[0] : (Tv *)m.u64[0];  // level-0 correction (zero on the boundary)
    constexpr int LFE = line_factor_elems(M);
    const unsigned FBv = (unsigned)(LFE * sizeof(Tv)), FBd = (unsigned)(LFE * sizeof(double));
    // levels whose work fits in G blocks are swept by the first G blocks only
    const int G = min(kBarGroup, nbk);
    int lb = L;
    while (lb > 0 && units_of(m.nz[lb - 1]) <= G) --lb;
    const bool in_group = bid < G;
    __shared__ unsigned long long s_r[32], s_b[32];
    __shared__ double s_dot[4][32];
    __shared__ double s_sum[4];
    __shared__ double s_ab[3];  // the GCR step's beta, alpha and |q|^2
    // the mixed path accelerates its refinement by flexible GCR(1) (the
    // Krylov vectors are allocated for it); the FP64 path runs the paper's
    // plain V(0,1) iteration
    const bool kry = mixed && m.kr != nullptr && L > 0;
    double kc = 0.0;  // |w|^2 of the previous direction's A-image
    __shared__ __align__(8) unsigned long long s_mbar[3];
    __shared__ int s_decide;
    if (tid == 0) {
        for (int b = 0; b < 3; ++b)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"((unsigned)__cvta_generic_to_shared(&s_mbar[b]))
                         : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // red factors; black factors; coarsest-row factors
    Loader qR{(unsigned)__cvta_generic_to_shared(&s_mbar[0]), 0u, 0};
    Loader qB{(unsigned)__cvta_generic_to_shared(&s_mbar[1]), 0u, 0};
    Loader qC{(unsigned)__cvta_generic_to_shared(&s_mbar[2]), 0u, 0};
    // leave with no copy in flight (bounded waits); fail: a wait gave up
    auto leave = [&](bool fail) {
        if (fail && tid == 0) atomicExch(&ctl->timeout, 1);
        ld_wait(qR);
        ld_wait(qB);
        ld_wait(qC);
    };
    int first = first_cycle;
    unsigned ngrid = 0, ngroup = 0;  // barriers of each kind passed
    // the iterate alternates between phi and its copy (L > 0): the residual
    // phase reads cur + delta and stores it as nxt, the next cycle's iterate
    const bool dbuf = L > 0;
    double *cur = phi, *nxt = m.phi2;
    // coarsest-row factors in the V-cycle's type (nz = 3: phi's own row, FP64)
    const Tv *facc_v = mixed ? (const Tv *)m.facc32 : (const Tv *)m.facc;
    const unsigned FBc = (unsigned)(LFE * sizeof(Tv));
    Tv *Bf0 = reinterpret_cast<Tv *>(smem_raw + lay.offBuf);
    Tv *Bf1 = reinterpret_cast<Tv *>(smem_raw + lay.offBuf + M * kRow * 8);
    Tv *Bf2 = reinterpret_cast<Tv *>(smem_raw + lay.offBuf + 2 * M * kRow * 8);
    double *BC = reinterpret_cast<double *>(smem_raw + lay.offBuf);
    Tv *W0 = reinterpret_cast<Tv *>(smem_raw + lay.offW);
    Tv *W1 = W0 + NW;
    Tv *R0 = reinterpret_cast<Tv *>(smem_raw + lay.offF);
    Tv *R1 = R0 + LFE;
    Tv *FBk = R1 + LFE;
    Tv *FC = reinterpret_cast<Tv *>(smem_raw + lay.offC);
    double *FC64 = reinterpret_cast<double *>(smem_raw + lay.offC);
    // position of unknown j in a line buffer
    auto at = [](int j) { return (j % M) * kRow + j / M; };
    for (int cyc = 0;; ++cyc) {
        // ---- residual of phi + delta, its norms, and the restriction chain ----
        if (bid == 0 && L > 0) {
            ld_begin(qC, FBc);
            ld_copy(qC, FC, facc_v, FBc);
        }
        // maxima as bit patterns of |x| (ordered like the values; a NaN
        // compares above every number), so the reductions are integer work
        unsigned long long rmax = 0ull, bmax = 0ull;
        {
            const double *cz = m.cz[0], *cr = m.cr[0];
            const int tw = lay.tw, sw = tw + 2;
            // phi + delta of the tile and its two neighbour columns, all rows
            double *S = reinterpret_cast<double *>(smem_raw + lay.offBuf);
            // the restriction chain runs in the V-cycle's type
            Tv *T0 = reinterpret_cast<Tv *>(smem_raw + lay.offF);
            Tv *T1 = T0 + (size_t)tw * nz0;
            Tv *f0v = mixed ? (Tv *)m.f32[0] : (Tv *)m.f64[0];
            const int ntile = (n + tw - 1) / tw;
            // the restriction chain of the residual tile T0 (columns j0 ..)
            // down to the coarsest level, in the V-cycle's type
            auto chain = [&](int j0) {
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
            };
            if (kry && cyc > 0) {
                // ---- flexible GCR(1) step (mixed path) ----
                // z: the V-cycle's correction of the last cycle; w = A z;
                // the direction is z less its projection on the previous
                // one (in the A-image), the step length minimises |r|_2
                double a[4] = {0.0, 0.0, 0.0, 0.0};  // r.w, w.w, w.wp, r.wp
                for (int t = bid; t < ntile; t += nbk) {
                    const int j0 = t * tw;
                    for (int e0 = tid; e0 < sw * nz0; e0 += kU * nt) {
                        Tv dv[kU];
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % sw - 1, i = e / sw, j = j0 + c;
                            dv[u] = (e < sw * nz0 && j >= 0 && j < nr) ? delta[(size_t)i * nr + j] : (Tv)0;
                        }
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % sw - 1, i = e / sw;
                            if (e < sw * nz0) S[(size_t)(c + 1) * nz0 + i] = (double)dv[u];
                        }
                    }
                    __syncthreads();
                    // batches of kU nodes per thread, loads first
                    for (int e0 = tid; e0 < tw * (nz0 - 2); e0 += kU * nt) {
                        double ca[kU], cb[kU], ce[kU], cd[kU], dgv[kU], rv[kU], wpv[kU];
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                            ca[u] = cb[u] = ce[u] = cd[u] = dgv[u] = rv[u] = wpv[u] = 0.0;
                            if (e < tw * (nz0 - 2) && j < n) {
                                const size_t k = (size_t)i * nr + j;
                                ca[u] = cz[k - nr];
                                cb[u] = cz[k];
                                ce[u] = cr[k];
                                cd[u] = j > 0 ? cr[k - 1] : 0.0;
                                dgv[u] = m.dg0[k];
                                rv[u] = m.kr[k];
                                wpv[u] = m.kwp[k];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                            if (e >= tw * (nz0 - 2) || j >= n) continue;
                            const size_t k = (size_t)i * nr + j;
                            const double *Sc = S + (size_t)(c + 1) * nz0 + i;
                            const double w = dgv[u] * Sc[0] - ca[u] * Sc[-1] - cb[u] * Sc[1] - ce[u] * Sc[nz0] -
                                             cd[u] * Sc[-nz0];
                            m.kw[k] = w;
                            a[0] += rv[u] * w;
                            a[1] += w * w;
                            a[2] += w * wpv[u];
                            a[3] += rv[u] * wpv[u];
                        }
                    }
                    __syncthreads();  // S is reused by the next tile
                }
                // the warp's four sums with few FP64 additions (the pipe is
                // narrow): halves of the warp trade the products they do not
                // keep (16 apart: 0, 1 stay low, 2, 3 high; 8 apart: one
                // product per quarter), then each quarter sums its own;
                // product 2 (lane >> 4) + ((lane >> 3) & 1) ends in the
                // quarter's lanes
                {
                    const bool hi = lane >= 16, q1 = (lane & 8) != 0;
                    const double s0 = __shfl_xor_sync(0xffffffffu, hi ? a[0] : a[2], 16);
                    const double s1 = __shfl_xor_sync(0xffffffffu, hi ? a[1] : a[3], 16);
                    const double b0 = (hi ? a[2] : a[0]) + s0, b1 = (hi ? a[3] : a[1]) + s1;
                    double c = (q1 ? b1 : b0) + __shfl_xor_sync(0xffffffffu, q1 ? b0 : b1, 8);
                    for (int o = 4; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
                    if ((lane & 7) == 0) s_dot[2 * (lane >> 4) + ((lane >> 3) & 1)][warp] = c;
                }
                __syncthreads();
                if (tid < 4) {
                    double v = 0.0;
                    for (int q = 0; q < (nt >> 5); ++q) v += s_dot[tid][q];
                    m.kpart[(size_t)bid * 4 + tid] = v;
                }
                if (!count_barrier(&ctl->bar_count.v, (++ngrid) * nbk, &ctl->timeout)) {
                    leave(false);
                    return;
                }
                // every block sums the partial products in the same fixed
                // order (the same step length everywhere), all its threads
                // loading at once: thread t takes entries t, t + nt, ... of
                // product t % 4 (nt is a multiple of 32)
                {
                    double v = 0.0;
#pragma unroll 4
                    for (int e = tid; e < 4 * nbk; e += nt) v += m.kpart[e];
                    for (int o = 4; o < 32; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
                    if (lane < 4) s_dot[lane][warp] = v;
                    __syncthreads();
                    if (tid < 4) {
                        double t = 0.0;
                        for (int q = 0; q < (nt >> 5); ++q) t += s_dot[tid][q];
                        s_sum[tid] = t;
                    }
                    __syncthreads();
                    // the step's scalars by one thread: GB300's FP64 pipe is
                    // narrow, and every thread dividing cost microseconds
                    if (tid == 0) {
                        const double beta = kc > 0.0 ? s_sum[2] / kc : 0.0;
                        const double den = s_sum[1] - beta * s_sum[2];
                        s_ab[0] = beta;
                        s_ab[1] = den > 0.0 ? (s_sum[0] - beta * s_sum[3]) / den : 1.0;
                        s_ab[2] = den > 0.0 ? den : 0.0;
                    }
                    __syncthreads();
                }
                const double beta = s_ab[0], alpha = s_ab[1];
                kc = s_ab[2];
                __syncthreads();  // s_sum and s_ab are rewritten by the next cycle
                for (int t = bid; t < ntile; t += nbk) {
                    const int j0 = t * tw;
                    for (int e0 = tid; e0 < tw * (nz0 - 2); e0 += kU * nt) {
                        double pz[kU], qw[kU], zp[kU], wpv[kU], xv[kU], rv[kU];
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                            pz[u] = qw[u] = zp[u] = wpv[u] = xv[u] = rv[u] = 0.0;
                            if (e < tw * (nz0 - 2) && j < n) {
                                const size_t k = (size_t)i * nr + j;
                                pz[u] = (double)delta[k];
                                qw[u] = m.kw[k];
                                if (beta != 0.0) {
                                    zp[u] = m.kzp[k];
                                    wpv[u] = m.kwp[k];
                                }
                                xv[u] = cur[k];
                                rv[u] = m.kr[k];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kU; ++u) {
                            const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                            if (e >= tw * (nz0 - 2)) break;
                            double rn = 0.0;
                            if (j < n) {
                                const size_t k = (size_t)i * nr + j;
                                const double p = pz[u] - beta * zp[u], q = qw[u] - beta * wpv[u];
                                nxt[k] = xv[u] + alpha * p;
                                rn = rv[u] - alpha * q;
                                m.kr[k] = rn;
                                m.kzp[k] = p;
                                m.kwp[k] = q;
                                rmax = max(rmax, abs_bits(rn));
                                f0v[k] = (Tv)rn;
                            }
                            T0[(size_t)c * nz0 + i] = (Tv)rn;
                        }
                    }
                    __syncthreads();
                    chain(j0);
                }
            } else
            for (int t = bid; t < ntile; t += nbk) {
                const int j0 = t * tw;
                // batches of kU elements per thread: all loads first (stores to
                // global memory would otherwise hold back the next loads)
                for (int e0 = tid; e0 < sw * nz0; e0 += kU * nt) {
                    double pv[kU];
                    Tv dv[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int e = e0 + u * nt, c = e % sw - 1, i = e / sw, j = j0 + c;
                        pv[u] = 0.0;
                        dv[u] = 0;
                        if (e < sw * nz0 && j >= 0 && j < nr) {
                            const size_t k = (size_t)i * nr + j;
                            pv[u] = cur[k];
                            dv[u] = delta[k];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int e = e0 + u * nt, c = e % sw - 1, i = e / sw, j = j0 + c;
                        if (e >= sw * nz0) break;
                        const double v = pv[u] + (double)dv[u];
                        // the iterate of the next cycle, stored by the tile that owns the node
                        if (dbuf && c >= 0 && c < tw && j < n && i > 0 && i < nz0 - 1) nxt[(size_t)i * nr + j] = v;
                        S[(size_t)(c + 1) * nz0 + i] = v;
                    }
                }
                __syncthreads();
                // interior rows only: the chain never reads a level's boundary rows
                for (int e0 = tid; e0 < tw * (nz0 - 2); e0 += kU * nt) {
                    double ca[kU], cb[kU], ce[kU], cd[kU], dgv[kU], fv[kU];
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                        const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                        ca[u] = cb[u] = ce[u] = cd[u] = dgv[u] = fv[u] = 0.0;
                        if (e < tw * (nz0 - 2) && j < n) {
                            const size_t k = (size_t)i * nr + j;
                            ca[u] = cz[k - nr];
                            cb[u] = cz[k];
                            ce[u] = cr[k];
                            cd[u] = j > 0 ? cr[k - 1] : 0.0;
                            dgv[u] = m.dg0[k];
                            fv[u] = m.f0[k];
                        }
                    }
#pragma unroll
                    for (int u = 0; u < kU; ++u) {
                    const int e = e0 + u * nt, c = e % tw, i = 1 + e / tw, j = j0 + c;
                    if (e >= tw * (nz0 - 2)) break;
                    double r = 0.0;
                    if (j < n) {
                        const size_t k = (size_t)i * nr + j;
                        const double *Sc = S + (size_t)(c + 1) * nz0 + i;
                        const double a = ca[u], cc = cb[u], ee = ce[u], d = cd[u];
                        const double Au = dgv[u] * Sc[0] - a * Sc[-1] - cc * Sc[1] - ee * Sc[nz0] - d * Sc[-nz0];
                        const double f = fv[u];
                        r = f - Au;
                        rmax = max(rmax, abs_bits(r));
                        if (first) {
                            double bb = f;
                            if (i == 1) bb += a * Sc[-1];
                            if (i == nz0 - 2) bb += cc * Sc[1];
                            if (j == nr - 2) bb += ee * Sc[nz0];
                            bmax = max(bmax, abs_bits(bb));
                        }
                        if (L > 0) f0v[k] = (Tv)r;
                        if (kry) m.kr[k] = r;
                    }
                    T0[(size_t)c * nz0 + i] = (Tv)r;
                    }
                }
                __syncthreads();
                chain(j0);
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
        if (!count_barrier(&ctl->bar_count.v, (++ngrid) * nbk, &ctl->timeout)) {
            leave(false);
            return;
        }
        // ---- decision: every block reads the same maxima ----
        if (tid == 0) {
            const double rn = __longlong_as_double((long long)*(volatile unsigned long long *)&ctl->rb[cyc & 1]);
            const double bn = __longlong_as_double((long long)*(volatile unsigned long long *)&ctl->b_bits);
            int d = 0;  // 0 continue, 1 converged, 2 out of cycles, 3 zero right-hand side
            if (bn == 0.0)
                d = 3;
            else if (tol > 0.0 && rn <= tol * bn)
                d = 1;
            else if (cyc >= max_cycles)
                d = tol > 0.0 ? 2 : 1;
            s_decide = d;
            if (bid == 0) {
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
            for (int k = bid * nt + tid; k < ng; k += nbk * nt) {
                const int i = k / nr, j = k % nr;
                if (i > 0 && i < nz0 - 1 && j < nr - 1) phi[k] = 0.0;
            }
            leave(false);
            return;
        }
        if (decide != 0) {
            // the answer is the iterate the residual phase just stored
            if (dbuf && nxt != phi)
                for (int k = bid * nt + tid; k < ng; k += nbk * nt) {
                    const int i = k / nr, j = k % nr;
                    if (i > 0 && i < nz0 - 1 && j < nr - 1) phi[k] = nxt[k];
                }
            leave(false);
            return;
        }
        if (dbuf) {
            double *t = cur;
            cur = nxt;
            nxt = t;
        }
        if (L == 0) {
            // nz = 3: the single interior row of phi, exactly
            if (bid == 0) {
                ld_begin(qC, FBd);
                ld_copy(qC, FC64, m.facc, FBd);
                const double *cz = m.cz[0], *cr = m.cr[0];
                for (int j = tid; j < NW; j += nt) {
                    double rhs = 0.0;
                    if (j < n) {
                        const size_t k = (size_t)nr + j;
                        rhs = m.f0[k] + cz[k - nr] * phi[k - nr] + cz[k] * phi[k + nr];
                        if (j == n - 1) rhs += cr[k] * phi[k + 1];
                    }
                    BC[at(j)] = rhs;
                }
                __syncthreads();
                if (!ld_wait(qC)) {
                    leave(true);
                    return;
                }
                if (warp == 0) warp_line_solve<double, M>(FC64, BC, lane);
                __syncthreads();
                for (int j = tid; j < n; j += nt) phi[(size_t)nr + j] = BC[at(j)];
            }
            if (!count_barrier(&ctl->bar_count.v, (++ngrid) * nbk, &ctl->timeout)) {
                leave(false);
                return;
            }
            continue;
        }
        // level 0's sweeps rewrite delta: when they run in the group alone,
        // every block's update of phi has to be in first
        if (lb == 0)
            if (!count_barrier(&ctl->bar_count.v, (++ngrid) * nbk, &ctl->timeout)) {
                leave(false);
                return;
            }
        // ---- up: per level, each black line with the two red lines beside it ----
        bool have = false;  // this block's first red factors of the level are requested
        for (int l = L - 1; l >= 0; --l) {
            const bool grp = l >= lb;
            const int P = grp ? G : nbk;
            const int nzl = m.nz[l], nzc = m.nz[l + 1];
            const int NB = (nzl - 3) / 2;  // black lines (>= 1: nzl >= 5 here)
            Tv *u = mixed ? (Tv *)m.u32[l] : (Tv *)m.u64[l];
            const Tv *uc = mixed ? (const Tv *)m.u32[l + 1] : (const Tv *)m.u64[l + 1];
            const Tv *f = mixed ? (const Tv *)m.f32[l] : (const Tv *)m.f64[l];
            const Tv *cz = mixed ? (const Tv *)m.cz32[l] : (const Tv *)m.cz[l];
            const Tv *fac = mixed ? (const Tv *)m.fac32[l] : (const Tv *)m.fac64[l];
            bool fail = false;
            if (bid < P) {
                if (l == L - 1 && bid == 0) {
                    // the coarsest row (FP64 factors, requested with the residual),
                    // then level L-1 in this block alone
                    for (int j = tid; j < NW; j += nt) Bf0[at(j)] = j < n ? (Tv)m.fc64[(size_t)nr + j] : (Tv)0;
                    __syncthreads();
                    if (!ld_wait(qC)) {
                        leave(true);
                        return;
                    }
                    if (warp == 0) warp_line_solve<Tv, M>(FC, Bf0, lane);
                    __syncthreads();
                    Tv *ucw = mixed ? (Tv *)m.u32[L] : (Tv *)m.u64[L];
                    for (int j = tid; j < n; j += nt) ucw[(size_t)nr + j] = Bf0[at(j)];
                    __syncthreads();
                    have = false;
                }
                for (int q = bid; q < NB; q += P) {
                    const int ra = 2 * q + 1, rb = 2 * q + 3, ib = 2 * q + 2;
                    // factor requests: the reds (unless already in), then the black
                    if (!(have && q == bid)) {
                        ld_begin(qR, 2 * FBv);
                        ld_copy(qR, R0, fac + (size_t)(ra - 1) * LFE, FBv);
                        ld_copy(qR, R1, fac + (size_t)(rb - 1) * LFE, FBv);
                    }
                    ld_begin(qB, FBv);
                    ld_copy(qB, FBk, fac + (size_t)(ib - 1) * LFE, FBv);
                    have = false;
                    // right-hand sides: reds get f plus the coarse correction
                    // injected at rows i -/+ 1; the black line keeps its own f
                    // and couplings for later
                    const int Ia = (ra - 1) / 2, Ib = (rb + 1) / 2;  // coarse rows below ra, above rb
                    const int Im = (ra + 1) / 2;                     // coarse row between (= row ib)
                    const bool va = Ia > 0 && Ia < nzc - 1, vm = Im > 0 && Im < nzc - 1, vb = Ib > 0 && Ib < nzc - 1;
                    for (int j0 = tid; j0 < NW; j0 += kUL * nt) {
                        // rows ra, ib = ra + 1, rb = ra + 2: cz[ib - 1] = cz[ra], cz[ib] = cz[rb - 1]
                        Tv ua[kUL], um[kUL], ub[kUL], fa[kUL], fbv[kUL], fk[kUL], z0[kUL], z1[kUL], z2[kUL], z3[kUL];
#pragma unroll
                        for (int u = 0; u < kUL; ++u) {
                            const int j = j0 + u * nt;
                            ua[u] = um[u] = ub[u] = fa[u] = fbv[u] = fk[u] = z0[u] = z1[u] = z2[u] = z3[u] = 0;
                            if (j < n) {
                                const size_t ka = (size_t)ra * nr + j;
                                if (va) ua[u] = uc[(size_t)Ia * nr + j];
                                if (vm) um[u] = uc[(size_t)Im * nr + j];
                                if (vb) ub[u] = uc[(size_t)Ib * nr + j];
                                fa[u] = f[ka];
                                fk[u] = f[ka + nr];
                                fbv[u] = f[ka + 2 * nr];
                                z0[u] = cz[ka - nr];
                                z1[u] = cz[ka];
                                z2[u] = cz[ka + nr];
                                z3[u] = cz[ka + 2 * nr];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < kUL; ++u) {
                            const int j = j0 + u * nt;
                            if (j >= NW) break;
                            const int pj = at(j);
                            Bf0[pj] = fa[u] + z0[u] * ua[u] + z1[u] * um[u];
                            Bf1[pj] = fbv[u] + z2[u] * um[u] + z3[u] * ub[u];
                            Bf2[pj] = fk[u];
                            W0[j] = z1[u];
                            W1[j] = z2[u];
                        }
                    }
                    __syncthreads();
                    if (!ld_wait(qR)) {
                        fail = true;
                        break;
                    }
                    if (warp == 0)
                        warp_line_solve<Tv, M>(R0, Bf0, lane);
                    else if (warp == 1)
                        warp_line_solve<Tv, M>(R1, Bf1, lane);
                    __syncthreads();
                    for (int j = tid; j < NW; j += nt) {
                        const int pj = at(j);
                        const Tv x0 = Bf0[pj], x1 = Bf1[pj];
                        if (j < n) {
                            u[(size_t)ra * nr + j] = x0;
                            // red rb is also the next black's red ra: one block stores it
                            if (q == NB - 1) u[(size_t)rb * nr + j] = x1;
                            Bf2[pj] = Bf2[pj] + W0[j] * x0 + W1[j] * x1;
                        }
                    }
                    __syncthreads();
                    if (!ld_wait(qB)) {
                        fail = true;
                        break;
                    }
                    if (warp == 0) warp_line_solve<Tv, M>(FBk, Bf2, lane);
                    __syncthreads();
                    for (int j = tid; j < n; j += nt) u[(size_t)ib * nr + j] = Bf2[at(j)];
                    __syncthreads();  // buffers and factor regions are reused
                }
                // request the next level's first red factors of this block
                if (!fail && l > 0) {
                    const int ln = l - 1;
                    const int Pn = ln >= lb ? G : nbk;
                    const int nbn = (m.nz[ln] - 3) / 2;
                    if (bid < Pn && bid < nbn) {
                        const Tv *facn = mixed ? (const Tv *)m.fac32[ln] : (const Tv *)m.fac64[ln];
                        const int q = bid;
                        ld_begin(qR, 2 * FBv);
                        ld_copy(qR, R0, facn + (size_t)(2 * q) * LFE, FBv);
                        ld_copy(qR, R1, facn + (size_t)(2 * q + 2) * LFE, FBv);
                        have = true;
                    }
                }
            }
            if (fail) {
                leave(true);
                return;
            }
            // levels in the group alone are separated by the group barrier;
            // every other level boundary is a grid barrier
            bool ok;
            if (l > 0 && grp && l - 1 >= lb)
                ok = in_group ? count_barrier(&ctl->gbar_count.v, (++ngroup) * G, &ctl->timeout) : true;
            else
                ok = count_barrier(&ctl->bar_count.v, (++ngrid) * nbk, &ctl->timeout);
            if (!ok) {
                leave(false);
                return;
            }
        }
    }
}

template <typename Tv, int M, int MINB>
__global__ void __launch_bounds__(kSolveThreads, MINB)
    k_solve_persistent(const MGFast *__restrict__ mp, double *phi, int nr, int first_cycle, SolveLayout lay,
                       double tol, int max_cycles, const StepCtl *sctl) {
    solve_body<Tv, M>(mp, phi, nr, first_cycle, lay, tol, max_cycles, sctl, blockIdx.x, gridDim.x);
}

// The solves of several reactors (one line chunk M, one precision) in one
// cooperative launch: job k takes blocks [block0, block0 + nblocks) and its
// barriers count its own blocks only, so the reactors proceed side by side.
template <typename Tv, int M, int MINB>
__global__ void __launch_bounds__(kSolveThreads, MINB) k_solve_multi(const SolveJob *__restrict__ jobs, int njobs) {
    int lo = 0, hi = njobs - 1;  // the job whose block range holds this block
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].block0 <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const SolveJob &j = jobs[lo];
    const int bid = (int)blockIdx.x - j.block0;
    if (bid >= j.nblocks) return;
    solve_body<Tv, M>(j.mp, j.phi, j.nr, j.first_cycle, j.lay, j.tol, j.max_cycles, j.sctl, bid, j.nblocks);
}

}  // namespace

size_t mg_line_factor_elems(int nr) { return (size_t)line_factor_elems(line_chunk(nr - 1)); }

int mg_line_chunk(int nr) { return line_chunk(nr - 1); }

namespace {

template <typename Tv, int M>
void *solve_fn(int minb) {
    return minb == 2 ? (void *)k_solve_persistent<Tv, M, 2> : (void *)k_solve_persistent<Tv, M, 1>;
}

template <typename Tv, int M>
void *multi_fn(int minb) {
    return minb == 2 ? (void *)k_solve_multi<Tv, M, 2> : (void *)k_solve_multi<Tv, M, 1>;
}

template <typename Tv>
void *multi_kernel(int M, int minb) {
    switch (M) {
        case 1: return multi_fn<Tv, 1>(minb);
        case 2: return multi_fn<Tv, 2>(minb);
        case 4: return multi_fn<Tv, 4>(minb);
        case 8: return multi_fn<Tv, 8>(minb);
        case 16: return multi_fn<Tv, 16>(minb);
        default: return multi_fn<Tv, 32>(minb);
    }
}

template <typename Tv>
void *solve_kernel(int M, int minb) {
    switch (M) {
        case 1: return solve_fn<Tv, 1>(minb);
        case 2: return solve_fn<Tv, 2>(minb);
        case 4: return solve_fn<Tv, 4>(minb);
        case 8: return solve_fn<Tv, 8>(minb);
        case 16: return solve_fn<Tv, 16>(minb);
        default: return solve_fn<Tv, 32>(minb);
    }
}

// kernels whose dynamic shared memory can pass 48 KB on the largest meshes
constexpr size_t kSolveSmemLimit = 220 * 1024;

void raise_smem_limits() {
    static bool done = false;
    if (done) return;
    const int lim = (int)kSolveSmemLimit;
    cudaFuncSetAttribute(k_chi_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    for (int M = 1; M <= 32; M <<= 1) {
        for (int minb = 1; minb <= 2; ++minb) {
            cudaFuncSetAttribute(solve_kernel<float>(M, minb), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            cudaFuncSetAttribute(solve_kernel<double>(M, minb), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            cudaFuncSetAttribute(multi_kernel<float>(M, minb), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
            cudaFuncSetAttribute(multi_kernel<double>(M, minb), cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
        }
    }
    done = true;
}

}  // namespace

namespace {

// a timestep's solve reports to the step control instead of the host: V-cycle
// count, residual, an unconverged flag, and a halt on a timed-out wait
// `cont`: a second solve with the previous one's operator (the external
// circuit's charge-free part) adds its cycles to the step's last report and
// keeps the larger residual
__global__ void k_solve_done(const MGCtl *c, StepCtl *s, int cont) {
    if (s->halt) return;
    if (c->timeout) {
        s->halt = 1;
        s->halt_status = ST_TIMEOUT;
        s->halt_step = s->step;
        return;
    }
    const int cyc = c->zero_rhs ? 0 : c->cycles;
    s->mg_cycles += (unsigned long long)cyc;
    const double res = (c->zero_rhs || !(c->bnorm > 0.0)) ? 0.0 : c->last_res / c->bnorm;
    if (cont) {
        s->mg_last_cycles += cyc;
        s->mg_last_res = fmax(s->mg_last_res, res);
    } else {
        s->mg_last_cycles = cyc;
        s->mg_last_res = res;
    }
    if (!c->zero_rhs && !c->converged) s->mg_flags |= 1;
}

}  // namespace

void mg_fast_geometry(const MGFast &m, int nr, double dr, std::vector<double> &out) {
    // FV face areas of the annuli (z faces) and cylinder sides (r faces)
    // over the node distances, Sec. 2.4: the set-up kernels only scale them
    // by 1 + chi of the face
    out.assign((size_t)(2 * m.nlev + 1) * nr, 0.0);
    for (int l = 0; l < m.nlev; ++l) {
        const double dz = m.dz[l];
        double *gz = out.data() + (size_t)2 * l * nr, *gr = gz + nr;
        for (int j = 0; j < nr; ++j) {
            const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
            gz[j] = (kPi * (rp * rp - rm * rm)) / dz;
            gr[j] = 2.0 * kPi * rp * dz / dr;
        }
    }
    double *ga = out.data() + (size_t)2 * m.nlev * nr;
    for (int j = 0; j < nr; ++j) {
        const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
        ga[j] = (kPi * (rp * rp - rm * rm)) * m.dz[0] / kEps0;
    }
}

void mg_fast_upload(MGFast &m, cudaStream_t st) {
    cudaMemcpyAsync(m.self, &m, sizeof(MGFast), cudaMemcpyHostToDevice, st);
    cudaStreamSynchronize(st);
}

// The launch shape of one reactor's one-launch solve (shared-memory layout,
// blocks, kernel); false when it cannot be launched.
bool solve_job(const FieldDims &fd, MGFast &m, double *phi, bool mixed, double tol, int max_cycles,
               const StepCtl *sctl, bool wide, SolveJob &job) {
    const int nz = fd.nz, nr = fd.nr, n = nr - 1;
    const int M = line_chunk(n);
    raise_smem_limits();
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t es = mixed ? sizeof(float) : sizeof(double);
    const size_t LFE = (size_t)line_factor_elems(M);
    SolveLayout lay{};
    // wide: residual tiles of 4 columns over two blocks per black line: the
    // residual phase (FP64 stencil, restriction chain) runs on twice the SMs
    // the line phases need; the remaining SMs stay free for the cell sort
    // that runs beside the solve in a timestep (measured on c2: 0.551 ->
    // 0.518 ms per solve; three blocks per line leave the sort too few SMs).
    // Narrow (one block per black line, tiles of 8): many reactors solving
    // side by side each take fewer SMs.
    lay.tw = wide ? 4 : 8;
    size_t off = 0;
    auto take = [&](size_t b) {
        const size_t o = off;
        off += (b + 127) & ~(size_t)127;
        return (int)o;
    };
    // line buffers and couplings; during the residual phase the same space
    // holds phi + delta of a tile of columns with its two neighbours
    const size_t bufw = (size_t)3 * M * kRow * sizeof(double) + (size_t)2 * kLine * M * sizeof(double);
    const size_t stage = (size_t)(lay.tw + 2) * nz * sizeof(double);
    lay.offBuf = take(std::max(bufw, stage) - (size_t)2 * kLine * M * sizeof(double));
    lay.offW = take((size_t)2 * kLine * M * sizeof(double));
    lay.offF = take(std::max((size_t)3 * LFE * es, (size_t)2 * lay.tw * nz * es));
    lay.offC = take(LFE * sizeof(double));
    const size_t sp = off;
    // a wide solve (one reactor alone) takes the one-block-per-SM build; a
    // narrow one (a reactor of a batch) the two-block build
    const int minb = wide ? 1 : 2;
    void *fn = mixed ? solve_kernel<float>(M, minb) : solve_kernel<double>(M, minb);
    int per_sm = 0;
    if (sp <= kSolveSmemLimit) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kSolveThreads, sp);
    if (per_sm < 1) return false;
    const int grid = std::max(1, std::min(nsm * per_sm, std::min(nsm, (wide ? 2 : 1) * ((nz - 1) / 2))));
    job.mp = m.self;
    job.phi = phi;
    job.nr = nr;
    job.first_cycle = 1;
    job.lay = lay;
    job.tol = tol;
    job.max_cycles = max_cycles;
    job.sctl = sctl;
    job.block0 = 0;
    job.nblocks = grid;
    job.M = M;
    job.mixed = mixed ? 1 : 0;
    job.minb = minb;
    job.smem = sp;
    job.fn = fn;
    return true;
}

int mg_fast_solve(const FieldDims &fd, MGFast &m, const double *rho, const double *chi, double V,
                  const double *phi_zL, double *phi, bool warm, bool mixed, double tol,
                  int max_cycles, double *rel_res, int *launches, StepCtl *sctl, cudaStream_t st,
                  bool v_from_ctl, bool setup, cudaEvent_t at_solve, bool wide, SolveJob *defer,
                  double *phi_prev) {
    const int nz = fd.nz, nr = fd.nr, n = nr - 1, ng = nz * nr;
    const int M = line_chunk(n);
    const int nlev = m.nlev;
    int L = 0;
    raise_smem_limits();
    MGFast *mp = m.self;  // uploaded once (mg_fast_upload)
    // set-up: levels' chi, coefficients, line factors (skipped when the
    // operator is the one of the previous solve), right-hand side and
    // boundary data
    if (setup) {
    cudaMemcpyAsync(m.chi[0], chi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st);
    if (nlev > 1) {
        k_chi_levels<<<(nr + 7) / 8, 256, (size_t)8 * 2 * nz * sizeof(double), st>>>(mp, nr, sctl);
        ++L;
    }
    int total = 0;
    for (int l = 0; l < nlev; ++l) total += m.nz[l] * nr;
    k_coefs_levels<<<(total + 255) / 256, 256, 0, st>>>(mp, nr, fd.chi_face == PIC_CHI_MEAN, total, sctl);
    ++L;
    {
        // line factors in the V-cycle's type; one warp per line
        int lines_all = 0;
        for (int l = 0; l < nlev; ++l) lines_all += m.nz[l] - 2;
        if (!mixed) {
            k_factor_lines<double><<<(lines_all + 7) / 8, 256, 0, st>>>(mp, 0, nlev, nr, M, lines_all, sctl);
            ++L;
        } else if (nlev > 1) {
            k_factor_lines<float><<<(lines_all + 7) / 8, 256, 0, st>>>(mp, 0, nlev, nr, M, lines_all, sctl);
            ++L;
        } else {
            // nz = 3: the single row is phi's own, solved in FP64
            k_factor_lines<double><<<1, 32, 0, st>>>(mp, 0, 1, nr, M, 1, sctl);
            ++L;
        }
    }
    }
    k_rhs_bc<<<(ng + 255) / 256, 256, 0, st>>>(mp, rho, phi, phi_zL, V, nz, nr, warm ? 0 : 1, sctl,
                                               v_from_ctl ? 1 : 0, warm ? phi_prev : nullptr);
    ++L;
    // (k_rhs_bc also copies phi to its alternate, clears the level-0
    // correction and the solve's control block)
    // all cycles in one cooperative launch
    SolveJob job;
    if (!solve_job(fd, m, phi, mixed, tol, max_cycles, sctl, wide, job)) {
        if (at_solve) cudaEventRecord(at_solve, st);
        if (launches) *launches += L;
        return kSolveNoLaunch;
    }
    if (defer) {
        // the caller launches it with other reactors' solves (mg_multi_launch)
        *defer = job;
        if (launches) *launches += L;
        return 0;
    }
    const SolveLayout lay = job.lay;
    const size_t sp = job.smem;
    void *fn = job.fn;
    const int grid = job.nblocks;
    int first_cycle = 1, nrv = nr, mc = max_cycles;
    double tv = tol;
    const StepCtl *sc = sctl;
    void *args[] = {(void *)&mp, (void *)&phi, (void *)&nrv, (void *)&first_cycle, (void *)&lay,
                    (void *)&tv, (void *)&mc, (void *)&sc};
    // the highest stream priority: when a step sorts beside the solve, the
    // solve's blocks take SMs as soon as the sort's short blocks retire
    static int prio = 1;
    if (prio > 0) {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        prio = greatest;
    }
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(grid);
    lc.blockDim = dim3(kSolveThreads);
    lc.dynamicSmemBytes = sp;
    lc.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    at[1].id = cudaLaunchAttributePriority;
    at[1].val.priority = prio;
    lc.attrs = at;
    lc.numAttrs = 2;
    if (at_solve) cudaEventRecord(at_solve, st);
    const cudaError_t e = cudaLaunchKernelExC(&lc, fn, args);
    ++L;
    if (e != cudaSuccess) {
        if (launches) *launches += L;
        return kSolveNoLaunch;
    }
    if (sctl) {
        // inside a timestep: the result stays on the device
        k_solve_done<<<1, 1, 0, st>>>(m.ctl, sctl, setup ? 0 : 1);
        ++L;
        if (launches) *launches += L;
        return 0;
    }
    if (launches) *launches += L;
    MGCtl ch;
    cudaMemcpyAsync(&ch, m.ctl, sizeof(MGCtl), cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
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

std::vector<std::pair<int, int>> mg_multi_plan(std::vector<SolveJob> &jobs, bool &concurrent) {
    std::stable_sort(jobs.begin(), jobs.end(), [](const SolveJob &a, const SolveJob &b) {
        return a.mixed != b.mixed ? a.mixed < b.mixed : a.M < b.M;
    });
    std::vector<std::pair<int, int>> out;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    // the kinds' ranges, their kernels and their share of the GPU: every
    // kind's launch gets SMs in proportion to the blocks its jobs would take
    // alone, so that the launches of all kinds fit the GPU together
    struct Kind {
        size_t a, b;
        void *fn;
        size_t smem;
        int want;
    };
    std::vector<Kind> kinds;
    int want_all = 0;
    for (size_t a = 0; a < jobs.size();) {
        size_t b = a;
        size_t smem = 0;
        int want = 0;
        while (b < jobs.size() && jobs[b].mixed == jobs[a].mixed && jobs[b].M == jobs[a].M) {
            smem = std::max(smem, jobs[b].smem);
            want += jobs[b].nblocks;
            ++b;
        }
        void *fn = jobs[a].mixed ? multi_kernel<float>(jobs[a].M, 2) : multi_kernel<double>(jobs[a].M, 2);
        kinds.push_back({a, b, fn, smem, want});
        want_all += want;
        a = b;
    }
    // side by side only while that leaves the jobs a fair part of their
    // blocks: with more than six times the GPU's co-resident blocks wanted
    // (64 c4 reactors), the kinds take the whole GPU one after another
    // (measured: 16 and 32 reactors 1.08 -> 1.35 and 1.21 -> 1.35e10
    // particle-steps/s side by side, 64 reactors 1.48 -> 1.32e10)
    int per_min = 1 << 30;
    for (const Kind &k : kinds) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, kSolveThreads, k.smem);
        per_min = std::min(per_min, std::max(per_sm, 1));
    }
    const bool side_by_side = want_all <= 6 * per_min * nsm;
    concurrent = side_by_side;
    for (const Kind &k : kinds) {
        int per_sm = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k.fn, kSolveThreads, k.smem);
        const int share = side_by_side ? std::max(1, (int)((double)nsm * k.want / std::max(want_all, 1))) : nsm;
        const int cap = std::max(1, per_sm * share);
        // launches of at most `cap` blocks and one block per job at least
        for (size_t a = k.a; a < k.b;) {
            const size_t e = std::min(k.b, a + (size_t)cap);
            int want = 0;
            for (size_t j = a; j < e; ++j) want += jobs[j].nblocks;
            const double scale = want > cap ? (double)cap / want : 1.0;
            int used = 0;
            for (size_t j = a; j < e; ++j) {
                jobs[j].nblocks = std::max(1, (int)(jobs[j].nblocks * scale));
                used += jobs[j].nblocks;
            }
            while (used > cap) {  // the one-block floors overshot: trim the largest
                size_t big = a;
                for (size_t j = a; j < e; ++j)
                    if (jobs[j].nblocks > jobs[big].nblocks) big = j;
                if (jobs[big].nblocks <= 1) break;
                --jobs[big].nblocks;
                --used;
            }
            used = 0;
            for (size_t j = a; j < e; ++j) {
                jobs[j].block0 = used;
                jobs[j].fn = k.fn;
                jobs[j].smem = k.smem;
                used += jobs[j].nblocks;
            }
            out.push_back({(int)a, (int)e});
            a = e;
        }
    }
    return out;
}

int mg_multi_launch(const std::vector<SolveJob> &jobs, int j0, int j1, const SolveJob *jobs_dev,
                    cudaStream_t st) {
    if (j1 <= j0) return 0;
    int blocks = 0;
    for (int k = j0; k < j1; ++k) blocks = std::max(blocks, jobs[k].block0 + jobs[k].nblocks);
    const SolveJob *tab = jobs_dev + j0;
    int nj = j1 - j0;
    void *args[] = {(void *)&tab, (void *)&nj};
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(blocks);
    lc.blockDim = dim3(kSolveThreads);
    lc.dynamicSmemBytes = jobs[j0].smem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    return cudaLaunchKernelExC(&lc, jobs[j0].fn, args) == cudaSuccess ? 0 : kSolveNoLaunch;
}

void mg_solve_done(MGFast &m, StepCtl *sctl, bool first_of_step, cudaStream_t st) {
    k_solve_done<<<1, 1, 0, st>>>(m.ctl, sctl, first_of_step ? 0 : 1);
}

}  // namespace pic
