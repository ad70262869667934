// field.cu -- grids of the r-z implicit PIC/MC timestep (arXiv:1001.2969):
// rho and chi from the deposit (Sec. 2.1, Eq. (10)), the z-semi-coarsening
// multigrid solve of div[(1+chi) grad phi] = -rho/eps0 (Sec. 2.5,
// Algorithm 1) with zebra r-line relaxation, E = -grad phi, and the running
// time averages.
//
// Discretisation: finite volumes on node-centred control volumes; z faces
// carry eps A_j / dz with A_j = pi (r_{j+1/2}^2 - r_{j-1/2}^2), r faces carry
// eps 2 pi r_{j+1/2} dz / dr, eps = 1 + chi_face (max or mean of the two
// nodes).  The right-hand side is rho A_j dz / eps0.
//
// Multigrid: levels nz, (nz+1)/2, ..., 3 with nr fixed; coarse operators
// rediscretised from the z-full-weighted nodal chi; restriction [1/2 1 1/2]
// in z of the volume-integrated residual; prolongation linear in z; V(0,1):
// restrict down with zero coarse guesses, exact solve of the single interior
// row of the coarsest level, then prolong-correct and one red-black line
// sweep (odd rows, then even rows) per level going up.  Each r-line is a
// tridiagonal system solved by parallel cyclic reduction in shared memory.
// The mixed variant runs the V-cycle in FP32 on the correction of an FP64
// residual (iterative refinement); its coarsest solve stays in FP64.
#include <math.h>
#include <string.h>

#include "pic_internal.cuh"

namespace pic {

__global__ void k_finalize(const double *Ne, const double *Ni, const double *V, double q0,
                           double q1, double c0, double c1, double *rho, double *chi, int ng,
                           const StepCtl *ctl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng || (ctl && ctl->halt)) return;
    const double ne = Ne[k] / V[k], ni = Ni[k] / V[k];
    rho[k] = q0 * ne + q1 * ni;
    // chi = dt^2/(2 eps0) sum_s q_s^2 n_s / m_s ; c_s = q_s^2 dt^2 / (2 eps0 m_s)
    chi[k] = c0 * ne + c1 * ni;
}

void launch_finalize(const double *Ne, const double *Ni, const double *V, double q0, double q1,
                     double c0, double c1, double *rho, double *chi, int ng, const StepCtl *ctl,
                     cudaStream_t st) {
    k_finalize<<<(ng + 255) / 256, 256, 0, st>>>(Ne, Ni, V, q0, q1, c0, c1, rho, chi, ng, ctl);
}

// ---- level set-up ----
__global__ void k_restrict_chi(const double *fine, double *coarse, int nzc, int nr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nzc * nr) return;
    const int I = k / nr, j = k % nr;
    double v;
    if (I == 0 || I == nzc - 1)
        v = fine[(size_t)(2 * I) * nr + j];
    else
        v = 0.25 * fine[(size_t)(2 * I - 1) * nr + j] + 0.5 * fine[(size_t)(2 * I) * nr + j] +
            0.25 * fine[(size_t)(2 * I + 1) * nr + j];
    coarse[k] = v;
}

// cz[i][j]: z face between rows i and i+1; cr[i][j]: r face between j and j+1
__global__ void k_coefs(const double *chi, double *cz, double *cr, float *cz32, float *cr32,
                        int nz, int nr, double dz, double dr, int face_mean) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
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
    cz[k] = vz;
    cr[k] = vr;
    if (cz32) {
        cz32[k] = (float)vz;
        cr32[k] = (float)vr;
    }
}

// right-hand side rho A_j dz / eps0 on interior nodes, 0 on Dirichlet nodes
__global__ void k_rhs(const double *rho, double *f, int nz, int nr, double dz, double dr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    double v = 0.0;
    if (i > 0 && i < nz - 1 && j < nr - 1) {
        const double rp = (j + 0.5) * dr, rm = j > 0 ? (j - 0.5) * dr : 0.0;
        v = rho[k] * (kPi * (rp * rp - rm * rm)) * dz / kEps0;
    }
    f[k] = v;
}

// Dirichlet data: z = 0 at V (r = R corner grounded), z = L at phi_zL or 0,
// r = R at 0; cold start zeroes the interior
__global__ void k_bc(double *phi, const double *phi_zL, double V, int nz, int nr, int cold) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    if (i == 0)
        phi[k] = (j == nr - 1) ? 0.0 : V;
    else if (i == nz - 1)
        phi[k] = phi_zL ? phi_zL[j] : 0.0;
    else if (j == nr - 1)
        phi[k] = 0.0;
    else if (cold)
        phi[k] = 0.0;
}

__device__ __forceinline__ void atomic_max_pos(unsigned long long *dst, double v) {
    atomicMax(dst, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v) {
    __shared__ double s_m[32];
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_m[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < (int)(blockDim.x >> 5) ? s_m[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    return v;
}

// max |b|, b = f with the boundary values moved to the right-hand side
__global__ void k_bnorm(const double *f, const double *phi, const double *cz, const double *cr,
                        int nz, int nr, unsigned long long *out) {
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz * nr; k += gridDim.x * blockDim.x) {
        const int i = k / nr, j = k % nr;
        if (i == 0 || i == nz - 1 || j == nr - 1) continue;
        double v = f[k];
        if (i == 1) v += cz[k - nr] * phi[k - nr];
        if (i == nz - 2) v += cz[k] * phi[k + nr];
        if (j == nr - 2) v += cr[k] * phi[k + 1];
        m = fmax(m, fabs(v));
    }
    m = block_max(m);
    if (threadIdx.x == 0) atomic_max_pos(out, m);
}

// r = f - A u (FP64), max |r|
__global__ void k_residual(const double *f, const double *u, const double *cz, const double *cr,
                           double *r, int nz, int nr, unsigned long long *out) {
    double m = 0.0;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nz * nr; k += gridDim.x * blockDim.x) {
        const int i = k / nr, j = k % nr;
        double v = 0.0;
        if (i > 0 && i < nz - 1 && j < nr - 1) {
            const double a = cz[k - nr], c = cz[k], e = cr[k], d = j > 0 ? cr[k - 1] : 0.0;
            double Au = (a + c + d + e) * u[k] - a * u[k - nr] - c * u[k + nr] - e * u[k + 1];
            if (j > 0) Au -= d * u[k - 1];
            v = f[k] - Au;
            m = fmax(m, fabs(v));
        }
        r[k] = v;
    }
    m = block_max(m);
    if (threadIdx.x == 0) atomic_max_pos(out, m);
}

// coarse f = [1/2 1 1/2] in z of the fine volume-integrated residual; coarse u = 0
template <typename Ti, typename To>
__global__ void k_restrict(const Ti *fine, To *fc, To *uc, int nzc, int nr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nzc * nr) return;
    const int I = k / nr, j = k % nr;
    To v = 0;
    if (I > 0 && I < nzc - 1 && j < nr - 1)
        v = (To)(0.5 * (double)fine[(size_t)(2 * I - 1) * nr + j] +
                 (double)fine[(size_t)(2 * I) * nr + j] +
                 0.5 * (double)fine[(size_t)(2 * I + 1) * nr + j]);
    fc[k] = v;
    uc[k] = 0;
}

// u_f += P u_c on interior rows, j <= nr-2
template <typename T>
__global__ void k_prolong(const T *uc, T *uf, int nzf, int nr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nzf * nr) return;
    const int i = k / nr, j = k % nr;
    if (i == 0 || i == nzf - 1 || j == nr - 1) return;
    T corr;
    if ((i & 1) == 0)
        corr = uc[(size_t)(i / 2) * nr + j];
    else
        corr = (T)0.5 * (uc[(size_t)(i / 2) * nr + j] + uc[(size_t)(i / 2 + 1) * nr + j]);
    uf[k] += corr;
}

// One r-line per block (Sec. 2.5, Eq. (12)): row i of the level,
//   -d u_{i,j-1} + b u_ij - e u_{i,j+1} = f_ij + a u_{i-1,j} + c u_{i+1,j}
// (+ e u_{i,nr-1} on the last unknown), solved by parallel cyclic
// reduction in shared memory.  Tc: coefficient type, Tu: u/f storage type,
// Ts: solve type.
template <typename Tc, typename Tu, typename Ts>
__global__ void k_line(const Tc *cz, const Tc *cr, const Tu *f, Tu *u, int nr, int row0,
                       int row_step) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = nr - 1;
    Ts *A = reinterpret_cast<Ts *>(smem_raw);
    Ts *B = A + n, *C = B + n, *D = C + n;
    Ts *A2 = D + n, *B2 = A2 + n, *C2 = B2 + n, *D2 = C2 + n;
    const int i = row0 + blockIdx.x * row_step;
    const size_t rowk = (size_t)i * nr;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const size_t k = rowk + j;
        const Ts a = (Ts)cz[k - nr], c = (Ts)cz[k], e = (Ts)cr[k];
        const Ts d = j > 0 ? (Ts)cr[k - 1] : (Ts)0;
        Ts rhs = (Ts)f[k] + a * (Ts)u[k - nr] + c * (Ts)u[k + nr];
        if (j == n - 1) rhs += e * (Ts)u[k + 1];
        A[j] = -d;
        B[j] = a + c + d + e;
        C[j] = j < n - 1 ? -e : (Ts)0;
        D[j] = rhs;
    }
    __syncthreads();
    for (int s = 1; s < n; s <<= 1) {
        for (int j = threadIdx.x; j < n; j += blockDim.x) {
            Ts a = A[j], b = B[j], c = C[j], d = D[j];
            Ts na = 0, nc = 0;
            if (j - s >= 0) {
                const Ts al = -a / B[j - s];
                na = al * A[j - s];
                b += al * C[j - s];
                d += al * D[j - s];
            }
            if (j + s < n) {
                const Ts ga = -c / B[j + s];
                nc = ga * C[j + s];
                b += ga * A[j + s];
                d += ga * D[j + s];
            }
            A2[j] = na;
            B2[j] = b;
            C2[j] = nc;
            D2[j] = d;
        }
        __syncthreads();
        Ts *t;
        t = A; A = A2; A2 = t;
        t = B; B = B2; B2 = t;
        t = C; C = C2; C2 = t;
        t = D; D = D2; D2 = t;
    }
    for (int j = threadIdx.x; j < n; j += blockDim.x) u[rowk + j] = (Tu)(D[j] / B[j]);
}

template <typename T>
__global__ void k_cast(const double *src, T *dst, int n) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) dst[k] = (T)src[k];
}

__global__ void k_add_correction(double *u, const float *du, int nz, int nr) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr) return;
    const int i = k / nr, j = k % nr;
    if (i == 0 || i == nz - 1 || j == nr - 1) return;
    u[k] += (double)du[k];
}

static inline int nblk(int n, int t = 256) { return (n + t - 1) / t; }

template <typename Tc, typename Tu, typename Ts>
static void line_rows(const Tc *cz, const Tc *cr, const Tu *f, Tu *u, int nz, int nr, int row0,
                      cudaStream_t st, int *launches) {
    if (nz - 2 - row0 < 0) return;
    const int nrows = (nz - 2 - row0) / 2 + 1;  // rows row0, row0+2, ... <= nz-2
    const int n = nr - 1;
    const size_t smem = 8 * (size_t)n * sizeof(Ts);
    int threads = 32;
    while (threads < n && threads < 1024) threads <<= 1;
    // the opt-in is a per-device attribute of the kernel: set it once for
    // every device this process launches on
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || !attr_set[dev])) {
        cudaFuncSetAttribute(k_line<Tc, Tu, Ts>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    k_line<Tc, Tu, Ts><<<nrows, threads, smem, st>>>(cz, cr, f, u, nr, row0, 2);
    ++*launches;
}

static double read_bits(DevScalars *ds, bool aux, cudaStream_t st) {
    unsigned long long v = 0;
    cudaMemcpyAsync(&v, aux ? &ds->mg_aux_bits : &ds->mg_res_bits, sizeof(v),
                    cudaMemcpyDeviceToHost, st);
    cudaStreamSynchronize(st);
    double d;
    memcpy(&d, &v, sizeof(d));
    return d;
}

int mg_solve(const FieldDims &fd, MGWork &mg, const double *rho, const double *chi, double V,
             const double *phi_zL, double *phi, bool warm, bool mixed, double tol, int max_cycles,
             double *rel_res, int *launches, cudaStream_t st) {
    const int nz = fd.nz, nr = fd.nr, ng = nz * nr;
    const int nlev = mg.nlev;
    int L = 0;
    // level chi and coefficients
    cudaMemcpyAsync(mg.lv[0].chi, chi, sizeof(double) * ng, cudaMemcpyDeviceToDevice, st);
    for (int l = 1; l < nlev; ++l) {
        const int nzc = mg.lv[l].nz;
        k_restrict_chi<<<nblk(nzc * nr), 256, 0, st>>>(mg.lv[l - 1].chi, mg.lv[l].chi, nzc, nr);
        ++L;
    }
    for (int l = 0; l < nlev; ++l) {
        const MGLevel &lv = mg.lv[l];
        k_coefs<<<nblk(lv.nz * nr), 256, 0, st>>>(lv.chi, lv.cz, lv.cr, mixed ? lv.cz32 : nullptr,
                                                   mixed ? lv.cr32 : nullptr, lv.nz, nr, lv.dz,
                                                   fd.dr, fd.chi_face == PIC_CHI_MEAN);
        ++L;
    }
    k_rhs<<<nblk(ng), 256, 0, st>>>(rho, mg.f0, nz, nr, fd.dz, fd.dr);
    k_bc<<<nblk(ng), 256, 0, st>>>(phi, phi_zL, V, nz, nr, warm ? 0 : 1);
    cudaMemsetAsync(&mg.ds->mg_aux_bits, 0, sizeof(unsigned long long), st);
    k_bnorm<<<nblk(ng), 256, 0, st>>>(mg.f0, phi, mg.lv[0].cz, mg.lv[0].cr, nz, nr,
                                      &mg.ds->mg_aux_bits);
    L += 3;
    const double bnorm = read_bits(mg.ds, true, st);
    int cyc = 0, status = 1;
    double rn = 0.0;
    const int gres = (ng + 255) / 256 < 152 * 4 ? (ng + 255) / 256 : 152 * 4;
    if (bnorm == 0.0) {
        k_bc<<<nblk(ng), 256, 0, st>>>(phi, phi_zL, V, nz, nr, 1);
        ++L;
        if (rel_res) *rel_res = 0.0;
        if (launches) *launches += L;
        return 0;
    }
    for (;;) {
        cudaMemsetAsync(&mg.ds->mg_res_bits, 0, sizeof(unsigned long long), st);
        k_residual<<<gres, 256, 0, st>>>(mg.f0, phi, mg.lv[0].cz, mg.lv[0].cr, mg.r, nz, nr,
                                         &mg.ds->mg_res_bits);
        ++L;
        rn = read_bits(mg.ds, false, st);
        if (tol > 0.0 && rn <= tol * bnorm) {
            status = 0;
            break;
        }
        if (cyc >= max_cycles) {
            status = tol > 0.0 ? 1 : 0;
            break;
        }
        if (nlev == 1) {
            // nz = 3: the single interior row is the whole problem; solve it exactly
            line_rows<double, double, double>(mg.lv[0].cz, mg.lv[0].cr, mg.f0, phi, nz, nr, 1, st, &L);
        } else if (!mixed) {
            // restrict the residual down; coarse levels start from zero
            for (int l = 1; l < nlev; ++l) {
                const MGLevel &c = mg.lv[l];
                const double *src = l == 1 ? mg.r : mg.lv[l - 1].f;
                k_restrict<double, double><<<nblk(c.nz * nr), 256, 0, st>>>(src, c.f, c.u, c.nz, nr);
                ++L;
            }
            const MGLevel &cl = mg.lv[nlev - 1];
            line_rows<double, double, double>(cl.cz, cl.cr, cl.f, cl.u, cl.nz, nr, 1, st, &L);
            for (int l = nlev - 2; l >= 0; --l) {
                const MGLevel &lv = mg.lv[l];
                double *u = l == 0 ? phi : lv.u;
                const double *f = l == 0 ? mg.f0 : lv.f;
                k_prolong<double><<<nblk(lv.nz * nr), 256, 0, st>>>(mg.lv[l + 1].u, u, lv.nz, nr);
                ++L;
                line_rows<double, double, double>(lv.cz, lv.cr, f, u, lv.nz, nr, 1, st, &L);
                line_rows<double, double, double>(lv.cz, lv.cr, f, u, lv.nz, nr, 2, st, &L);
            }
        } else {
            // FP32 V-cycle on the correction of the FP64 residual
            const MGLevel &f0 = mg.lv[0];
            k_restrict<double, float><<<nblk(mg.lv[1].nz * nr), 256, 0, st>>>(
                mg.r, mg.lv[1].f32, mg.lv[1].u32, mg.lv[1].nz, nr);
            k_cast<float><<<nblk(ng), 256, 0, st>>>(mg.r, f0.f32, ng);
            cudaMemsetAsync(f0.u32, 0, sizeof(float) * ng, st);
            L += 2;
            for (int l = 2; l < nlev; ++l) {
                const MGLevel &c = mg.lv[l];
                k_restrict<float, float><<<nblk(c.nz * nr), 256, 0, st>>>(mg.lv[l - 1].f32, c.f32,
                                                                           c.u32, c.nz, nr);
                ++L;
            }
            const MGLevel &cl = mg.lv[nlev - 1];
            line_rows<double, float, double>(cl.cz, cl.cr, cl.f32, cl.u32, cl.nz, nr, 1, st, &L);
            for (int l = nlev - 2; l >= 0; --l) {
                const MGLevel &lv = mg.lv[l];
                k_prolong<float><<<nblk(lv.nz * nr), 256, 0, st>>>(mg.lv[l + 1].u32, lv.u32, lv.nz,
                                                                    nr);
                ++L;
                line_rows<float, float, float>(lv.cz32, lv.cr32, lv.f32, lv.u32, lv.nz, nr, 1, st,
                                               &L);
                line_rows<float, float, float>(lv.cz32, lv.cr32, lv.f32, lv.u32, lv.nz, nr, 2, st,
                                               &L);
            }
            k_add_correction<<<nblk(ng), 256, 0, st>>>(phi, f0.u32, nz, nr);
            ++L;
        }
        ++cyc;
    }
    if (rel_res) *rel_res = rn / bnorm;
    if (launches) *launches += L;
    return status == 0 ? cyc : -cyc - 1;
}

// E = -grad phi: central inside, one-sided first order on the boundary rows
// and on r = R, E_r = 0 on the axis
template <typename T>
__global__ void k_efield(const double *phi, double *Ez, double *Er, typename V2<T>::type *E2,
                         int nz, int nr, double dz, double dr, const StepCtl *ctl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nz * nr || (ctl && ctl->halt)) return;
    const int i = k / nr, j = k % nr;
    double ez, er;
    if (i == 0)
        ez = -(phi[k + nr] - phi[k]) / dz;
    else if (i == nz - 1)
        ez = -(phi[k] - phi[k - nr]) / dz;
    else
        ez = -(phi[k + nr] - phi[k - nr]) / (2.0 * dz);
    if (j == 0)
        er = 0.0;
    else if (j == nr - 1)
        er = -(phi[k] - phi[k - 1]) / dr;
    else
        er = -(phi[k + 1] - phi[k - 1]) / (2.0 * dr);
    Ez[k] = ez;
    Er[k] = er;
    typename V2<T>::type e;
    e.x = (T)ez;
    e.y = (T)er;
    E2[k] = e;
}

template <typename T>
void launch_efield(const double *phi, double *Ez, double *Er, typename V2<T>::type *E2, int nz,
                   int nr, double dz, double dr, const StepCtl *ctl, cudaStream_t st) {
    k_efield<T><<<nblk(nz * nr), 256, 0, st>>>(phi, Ez, Er, E2, nz, nr, dz, dr, ctl);
}
template void launch_efield<float>(const double *, double *, double *, float2 *, int, int, double,
                                   double, const StepCtl *, cudaStream_t);
template void launch_efield<double>(const double *, double *, double *, double2 *, int, int,
                                    double, double, const StepCtl *, cudaStream_t);

__global__ void k_moments(const double *Ne, const double *Ni, const double *V, const double *phi,
                          const double *Ez, const double *Er, double *m_ne, double *m_ni,
                          double *m_phi, double *m_ez, double *m_er, int ng, const StepCtl *ctl) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= ng || (ctl && ctl->halt)) return;
    m_ne[k] += Ne[k] / V[k];
    m_ni[k] += Ni[k] / V[k];
    m_phi[k] += phi[k];
    m_ez[k] += Ez[k];
    m_er[k] += Er[k];
}

void launch_moments(const double *Ne, const double *Ni, const double *V, const double *phi,
                    const double *Ez, const double *Er, double *m_ne, double *m_ni, double *m_phi,
                    double *m_ez, double *m_er, int ng, const StepCtl *ctl, cudaStream_t st) {
    k_moments<<<nblk(ng), 256, 0, st>>>(Ne, Ni, V, phi, Ez, Er, m_ne, m_ni, m_phi, m_ez, m_er, ng, ctl);
}

}  // namespace pic
