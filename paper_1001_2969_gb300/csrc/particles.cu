// particles.cu -- particle kernels of the r-z implicit PIC/MC timestep
// (Wang, Jiang & Wang, arXiv:1001.2969): the load, the fused particle pass
// (gather -> final push -> axis/walls -> null-collision MC -> split -> first
// push -> deposit), the plain deposit, and the absolute-coordinate
// conversions.  Positions are stored as an integer cell plus in-cell offsets
// in [0, 1), so single precision keeps its resolution at large radius.
#include <math.h>

#include <algorithm>

#include "pmath.cuh"

namespace pic {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of
// (c0,c1,c2,c3) -> (hi(M1 c2)^c1^k0, lo(M1 c2), hi(M0 c0)^c3^k1, lo(M0 c0)),
// the key bumped by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// draws of particle `id` of species s at `step` on `stream`
__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint64_t id, uint32_t step,
                                      int stream, int s) {
    return philox10(make_uint4((uint32_t)id, (uint32_t)(id >> 32), step, (uint32_t)(stream * 2 + s)),
                    k0, k1);
}

// uniform on (0, 1) from one 32-bit word
template <typename T>
__device__ __forceinline__ T unif(uint32_t x);
template <>
__device__ __forceinline__ float unif<float>(uint32_t x) {
    return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f);
}
template <>
__device__ __forceinline__ double unif<double>(uint32_t x) {
    return ((double)x + 0.5) * (1.0 / 4294967296.0);
}

// all channels' sigma(E) at once from the interleaved table sig4[k] = {s0..s3}
template <typename T>
__device__ __forceinline__ void sigma_all(const Xs<T> &xs, T E, T s[4]) {
    T a0, a1, a2, a3;
    if (E >= xs.emax) {
        ld4(xs.sig4 + (xs.n_e - 1), a0, a1, a2, a3);
        const T f = m_div(xs.emax, E);
        s[0] = a0 * f;
        s[1] = a1 * f;
        s[2] = a2 * f;
        s[3] = a3 * f;
        return;
    }
    const T x = E * xs.inv_dE;
    int k = x >= (T)0 ? (int)m_floor(x) : 0;  // also keeps a NaN off the table
    if (k > xs.n_e - 2) k = xs.n_e - 2;
    const T f = x - (T)k;
    T b0, b1, b2, b3;
    ld4(xs.sig4 + k, a0, a1, a2, a3);
    ld4(xs.sig4 + k + 1, b0, b1, b2, b3);
    s[0] = a0 + f * (b0 - a0);
    s[1] = a1 + f * (b1 - a1);
    s[2] = a2 + f * (b2 - a2);
    s[3] = a3 + f * (b3 - a3);
}

template <typename T>
__device__ __forceinline__ T sigma_of(const Xs<T> &xs, int ch, T E) {
    const T *sg = xs.sigma + ch * xs.n_e;
    if (E >= xs.emax) return sg[xs.n_e - 1] * xs.emax / E;
    if (E <= (T)0) return sg[0];
    const T x = E * xs.inv_dE;
    int k = x >= (T)0 ? (int)m_floor(x) : 0;  // also keeps a NaN off the table
    if (k > xs.n_e - 2) k = xs.n_e - 2;
    const T f = x - (T)k;
    return sg[k] + f * (sg[k + 1] - sg[k]);
}

// Vahedi-Surendra scattering angle (isotropic below 1e-6 eV or on request)
template <typename T>
__device__ __forceinline__ T cos_chi(int scatter, T eps, T R) {
    T c;
    if (scatter == PIC_SCATTER_ISOTROPIC || eps < (T)1e-6)
        c = (T)1 - (T)2 * R;
    else
        c = m_div((T)2 + eps - (T)2 * m_powR((T)1 + eps, R), eps);
    return c > (T)1 ? (T)1 : (c < (T)-1 ? (T)-1 : c);
}

// new direction: cos(chi) u + sin(chi)[cos(phi) e1 + sin(phi) e2] with
// e1 = (u_y, -u_x, 0)/s, e2 = (u_x u_z, u_y u_z, -s^2)/s, s^2 = u_x^2 + u_y^2
template <typename T>
__device__ __forceinline__ void scatter_dir(T ux, T uy, T uz, T cc, T uphi, T &ox, T &oy,
                                            T &oz) {
    const T sc = m_sqrt(fmax((T)0, (T)1 - cc * cc));
    T sp, cp;
    m_sincos2pi(uphi, &sp, &cp);
    const T s2 = ux * ux + uy * uy;
    const T tiny = sizeof(T) == 8 ? (T)1e-24 : (T)1e-12;
    if (s2 < tiny) {
        ox = sc * cp;
        oy = sc * sp * uz;
        oz = cc * uz;
        return;
    }
    const T s = m_sqrt(s2);
    ox = cc * ux + sc * (cp * uy + sp * ux * uz) / s;
    oy = cc * uy + sc * (-cp * ux + sp * uy * uz) / s;
    oz = cc * uz + sc * (-sp * s2) / s;
}

template <typename T>
__device__ __forceinline__ void normals(uint32_t xa, uint32_t xb, T &n0, T &n1) {
    const T ua = unif<T>(xa), ub = unif<T>(xb);
    const T rad = m_sqrt((T)-2 * m_log(ua));
    T s, c;
    m_sincos2pi(ub, &s, &c);
    n0 = rad * c;
    n1 = rad * s;
}

// block-local tallies, flushed once per block
struct BlockTally {
    unsigned long long cnt[PIC_NCOUNT];
    double q[3];
};

// deposit one particle's weight with the shape factors at its cell
template <typename T>
__device__ __forceinline__ void deposit_global(double *N, int nr, int weighting, const PS<T> &p) {
    T s0, s1;
    shape_r(weighting, p.j, p.orr, s0, s1);
    const T z0 = (T)1 - p.oz, z1 = p.oz;
    double *g = N + (size_t)p.i * nr + p.j;
    atomicAdd(g, (double)(p.w * z0 * s0));
    atomicAdd(g + 1, (double)(p.w * z0 * s1));
    atomicAdd(g + nr, (double)(p.w * z1 * s0));
    atomicAdd(g + nr + 1, (double)(p.w * z1 * s1));
}

// newborn: first push, wall test, deposit, count, append with its order key
template <typename T>
__device__ void emit_birth(const StepArgs<T> &a, BlockTally *bt, int ts, int ps, uint64_t pid,
                           int k, PS<T> q) {
    atomicAdd(&bt->cnt[PIC_C_BIRTHS + ts], 1ull);
    if (a.xyz)
        first_push_xyz(a, q, a.bdt[ts], a.bdt_dz[ts]);
    else
        first_push(a, q, a.bdt[ts], a.bdt_dz[ts]);
    const int wall = wall_of(q.i, q.oz, q.j, a.nz, a.nr);
    if (wall >= 0) {
        atomicAdd(&bt->cnt[PIC_C_ABS + ts * 3 + wall], 1ull);
        atomicAdd(&bt->q[wall], (double)q.w * a.qch[ts]);
        return;
    }
    const int slot = atomicAdd(a.nb[ts], 1);
    if (slot >= a.bcap) {
        atomicOr(&a.ds->status, ST_BIRTH_OVERFLOW);
        return;
    }
    deposit_global(a.N[ts], a.nr, a.weighting, q);
    const int cell = q.j * a.ncz + q.i;
    atomicAdd(a.counts[ts] + cell, 1);
    store_p(a.births[ts], slot, q, cell, 0ull);
    if (a.xyz) a.births[ts].at[slot] = q.at;
    a.bkey[ts][slot] = ((uint64_t)ps << 63) | (pid << 16) | (uint64_t)k;
}

// Null-collision Monte Carlo (Sec. 2.6) on the post-final-push state, in
// three parts: the relative velocity against the target, the channel of a
// candidate, and the collision itself.
template <typename T>
struct Rel {
    T gx, gy, gz;     // velocity relative to the target
    T vnx, vny, vnz;  // the target atom's velocity (ions)
    T g, E;           // relative speed, collision energy
};

// electrons: the gas at rest; ions: an atom drawn from the gas Maxwellian
template <typename T>
__device__ __forceinline__ Rel<T> relative(const StepArgs<T> &a, uint64_t id, uint32_t step, const PS<T> &p) {
    Rel<T> r;
    r.gx = p.vr;
    r.gy = p.vt;
    r.gz = p.vz;
    r.vnx = r.vny = r.vnz = 0;
    if (a.s == 1) {
        const uint4 y = draw(a.key0, a.key1, id, step, 1, a.s);
        T n0, n1, n2, n3;
        normals(y.x, y.y, n0, n1);
        normals(y.z, y.w, n2, n3);
        r.vnx = a.v_gas * n0;
        r.vny = a.v_gas * n1;
        r.vnz = a.v_gas * n2;
        r.gx = p.vr - r.vnx;
        r.gy = p.vt - r.vny;
        r.gz = p.vz - r.vnz;
    }
    r.g = m_sqrt(r.gx * r.gx + r.gy * r.gy + r.gz * r.gz);
    r.E = a.half_m_e * r.g * r.g;
    return r;
}

// channel of a candidate whose stream-0 draw is x: -1 for a null collision
// (also an inelastic channel picked below its threshold); counts nu_max
// overruns and real collisions
template <typename T>
__device__ __forceinline__ int choose(const StepArgs<T> &a, BlockTally *bt, const uint4 x, const Rel<T> &r) {
    T nu[kMaxCh];
    sigma_all(a.xs, r.E, nu);
    T tot = 0;
    const T ngg = a.ng * r.g;
#pragma unroll
    for (int ch = 0; ch < kMaxCh; ++ch) {
        nu[ch] = ch < a.xs.n_ch ? ngg * nu[ch] : (T)0;
        tot += nu[ch];
    }
    if (tot > a.nu_max) atomicAdd(&bt->cnt[PIC_C_NUOVER + a.s], 1ull);
    const T sel = unif<T>(x.y) * a.nu_max;
    T cum = 0;
    int ch = -1;
#pragma unroll
    for (int k = 0; k < kMaxCh; ++k) {
        if (ch < 0 && k < a.xs.n_ch) {
            cum += nu[k];
            if (sel < cum) ch = k;
        }
    }
    if (ch < 0) return -1;
    const int kind = a.xs.kind[ch];
    if ((kind == PIC_XS_EXCITE || kind == PIC_XS_IONIZE) && r.E <= a.xs.thr[ch]) return -1;
    atomicAdd(&bt->cnt[PIC_C_COLL + a.s * 4 + ch], 1ull);
    return ch;
}

// the collision on channel ch (Vahedi-Surendra scattering, ionisation
// births, charge exchange)
template <typename T>
__device__ __forceinline__ void scatter(const StepArgs<T> &a, BlockTally *bt, uint64_t id, uint32_t step,
                                        const uint4 x, int ch, const Rel<T> &r, PS<T> &p) {
    const int kind = a.xs.kind[ch];
    const T thr = a.xs.thr[ch];
    const T g = r.g, E = r.E;
    if (kind == PIC_XS_CX) {
        p.vr = r.vnx;
        p.vt = r.vny;
        p.vz = r.vnz;
        return;
    }
    const T ux = r.gx / g, uy = r.gy / g, uz = r.gz / g;
    T dx, dy, dz;
    if (kind == PIC_XS_ELASTIC) {
        const T cc = cos_chi(a.scatter, E, unif<T>(x.z));
        scatter_dir(ux, uy, uz, cc, unif<T>(x.w), dx, dy, dz);
        const T gn = g * m_sqrt((T)1 - a.two_m_M * ((T)1 - cc));
        p.vr = gn * dx;
        p.vt = gn * dy;
        p.vz = gn * dz;
    } else if (kind == PIC_XS_EXCITE) {
        const T Ep = E - thr;
        const T cc = cos_chi(a.scatter, Ep, unif<T>(x.z));
        scatter_dir(ux, uy, uz, cc, unif<T>(x.w), dx, dy, dz);
        const T gn = m_sqrt(a.two_e_m * Ep);
        p.vr = gn * dx;
        p.vt = gn * dy;
        p.vz = gn * dz;
    } else {  // ionisation
        const uint4 y = draw(a.key0, a.key1, id, step, 1, a.s);
        const uint4 zz = draw(a.key0, a.key1, id, step, 2, a.s);
        const T Eej = a.xs.B * m_tan(unif<T>(y.x) * m_atan((E - thr) / ((T)2 * a.xs.B)));
        T Esc = E - thr - Eej;
        if (Esc < (T)0) Esc = (T)0;
        const T c1 = cos_chi(a.scatter, Esc, unif<T>(x.z));
        scatter_dir(ux, uy, uz, c1, unif<T>(x.w), dx, dy, dz);
        const T c2 = cos_chi(a.scatter, Eej, unif<T>(y.y));
        T ex, ey, ez;
        scatter_dir(ux, uy, uz, c2, unif<T>(y.z), ex, ey, ez);
        const T g1 = m_sqrt(a.two_e_m * Esc), g2 = m_sqrt(a.two_e_m * Eej);
        PS<T> e2 = p;
        e2.vr = g2 * ex;
        e2.vt = g2 * ey;
        e2.vz = g2 * ez;
        p.vr = g1 * dx;
        p.vt = g1 * dy;
        p.vz = g1 * dz;
        PS<T> ion = p;
        T n0, n1, n2, n3;
        normals(zz.x, zz.y, n0, n1);
        normals(zz.z, zz.w, n2, n3);
        ion.vr = a.v_gas * n0;
        ion.vt = a.v_gas * n1;
        ion.vz = a.v_gas * n2;
        ion.ar = p.ar * a.ion_acc;
        ion.az = p.az * a.ion_acc;
        ion.at = a.xyz ? p.at * a.ion_acc : (T)0;
        emit_birth(a, bt, 0, a.s, id, 0, e2);
        emit_birth(a, bt, 1, a.s, id, 1, ion);
    }
}

// the whole Monte Carlo step of one particle
template <typename T>
__device__ __forceinline__ void collide(const StepArgs<T> &a, BlockTally *bt, uint64_t id, uint32_t step,
                                        PS<T> &p) {
    const uint4 x = draw(a.key0, a.key1, id, step, 0, a.s);
    if ((unsigned long long)x.x >= a.t_null) return;
    atomicAdd(&bt->cnt[PIC_C_CAND + a.s], 1ull);
    const Rel<T> r = relative(a, id, step, p);
    const int ch = choose(a, bt, x, r);
    if (ch >= 0) scatter(a, bt, id, step, x, ch, r, p);
}

// cp.async of 4, 8 or 16 bytes (global -> shared; both ends aligned to the size)
__device__ __forceinline__ void cpa16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cpa4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

constexpr int kThreads = 256;
// the block's EEDF is kept in this many interleaved copies (lane % copies):
// electrons of a warp crowd into few low-energy bins, and same-address
// shared-memory atomics of a warp are serialised
constexpr int kEedfCopies = 8;

// The fused particle pass (Sec. 2.1 merged cycle).  Each warp works on
// units of 32 kPPT particles of the cell-sorted input, claimed from a counter.  Lanes of a warp hold
// consecutive particles, so their output cells come in runs; each run's
// deposit is summed across its lanes and its first lane adds it to the four
// nodes with global reductions (fire-and-forget, resolved in L2).  A
// shared-memory window of the chunk's nodes needs atomics that conflict
// between runs and warps and costs more instructions than it saves.
// PF: the unit's particles come into shared memory by cp.async a unit at
// a time, ahead of their use (for latency-bound passes)
// PPT: particles per thread in a unit (32 * PPT particles per warp)
// XYZ: the global X-Y-Z pusher (a_theta carried; a.xyz set)
template <typename T, bool PF, int kPPT, bool XYZ>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 4 : 2) k_step(StepArgs<T> a) {
    constexpr int kChunk = kThreads * kPPT;  // the block's staging slots
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using V = typename V4<T>::type;
    // the warps' current units' particles, fetched into shared memory ahead
    // of their use (PF): [kPPT][kThreads] of q0, q1, id, cell
    V *st_q0 = reinterpret_cast<V *>(smem_raw);
    V *st_q1 = st_q0 + kChunk;
    uint64_t *st_id = reinterpret_cast<uint64_t *>(st_q1 + kChunk);
    int32_t *st_cell = reinterpret_cast<int32_t *>(st_id + kChunk);
    T *st_at = reinterpret_cast<T *>(st_cell + kChunk);  // PF and XYZ
    T *s_eedf = PF ? (XYZ ? st_at + kChunk : reinterpret_cast<T *>(st_cell + kChunk))
                   : reinterpret_cast<T *>(smem_raw);
    __shared__ BlockTally bt;
    const int tid = threadIdx.x, lane = tid & 31;
    if (a.ctl->halt) return;  // an earlier failure of this step
    const uint32_t step = (uint32_t)a.ctl->step;  // Philox counter word
    const bool do_split = a.ctl->do_split != 0;
    for (int k = tid; k < PIC_NCOUNT; k += blockDim.x) bt.cnt[k] = 0;
    if (tid < 3) bt.q[tid] = 0.0;
    if (a.eedf)
        for (int k = tid; k < a.eedf_bins * kEedfCopies; k += blockDim.x) s_eedf[k] = (T)0;
    __syncthreads();  // tallies and EEDF cleared before any thread adds to them
    const int n = *a.n_alive;
    const int nmain = *a.n_main_src;
    // the prefetching shapes' copy of a particle (source index pidx) into
    // the staging slot, by cp.async
    auto fetch = [&](int pidx, int slot) {
        const bool from_main = pidx < nmain;
        const PBuf<T> &src = from_main ? a.src_main : a.src_births;
        const int si = from_main ? pidx : pidx - nmain;
        for (int h = 0; h < (int)(sizeof(V) / 16); ++h) {
            cpa16(reinterpret_cast<char *>(st_q0 + slot) + 16 * h,
                  reinterpret_cast<const char *>(src.q0 + si) + 16 * h);
            cpa16(reinterpret_cast<char *>(st_q1 + slot) + 16 * h,
                  reinterpret_cast<const char *>(src.q1 + si) + 16 * h);
        }
        cpa8(st_id + slot, src.id + si);
        cpa4(st_cell + slot, src.cell + si);
        if (XYZ) {
            if (sizeof(T) == 8)
                cpa8(st_at + slot, src.at + si);
            else
                cpa4(st_at + slot, src.at + si);
        }
    };
    // one particle of the pass: the state at sorted position k (read through
    // the permutation, or staged at slot by fetch), gathered, pushed,
    // collided, split, pushed again and deposited; every lane of the warp
    // calls it together (valid false: a lane past the end)
    auto process = [&](int k, bool valid, int slot) {
        int out_cell = -1;
        T c00 = 0, c01 = 0, c10 = 0, c11 = 0;
        if (valid) {
            PS<T> p;
            uint64_t id;
            if (PF) {
                ld4(st_q0 + slot, p.oz, p.orr, p.vr, p.vt);
                ld4(st_q1 + slot, p.vz, p.ar, p.az, p.w);
                decode_cell(st_cell[slot], a.ncz, a.inv_ncz, p.i, p.j);
                id = st_id[slot];
                if (XYZ) p.at = st_at[slot];
            } else {
                const int pidx = a.perm[k];
                const bool from_main = pidx < nmain;
                const PBuf<T> &src = from_main ? a.src_main : a.src_births;
                const int si = from_main ? pidx : pidx - nmain;
                p = load_p_fast(src, si, a.ncz, a.inv_ncz);
                id = src.id[si];
                if (XYZ) p.at = src.at[si];
            }
            // a stored cell outside the mesh (never written by a pass)
            // is reported and the record dropped, never followed
            const bool in_mesh = (unsigned)p.i < (unsigned)a.ncz && (unsigned)p.j < (unsigned)a.ncr;
            if (!in_mesh) p.i = p.j = 0;
            // gather E at x~ with the deposit's shape factors (Sec. 2.4)
            T s0, s1;
            shape_r(a.weighting, p.j, p.orr, s0, s1);
            const T z0 = (T)1 - p.oz, z1 = p.oz;
            const auto *Ep = a.E + (size_t)p.i * a.nr + p.j;
            const auto e00 = Ep[0], e01 = Ep[1], e10 = Ep[a.nr], e11 = Ep[a.nr + 1];
            const T Ez = z0 * (s0 * e00.x + s1 * e01.x) + z1 * (s0 * e10.x + s1 * e11.x);
            const T Er = z0 * (s0 * e00.y + s1 * e01.y) + z1 * (s0 * e10.y + s1 * e11.y);
            // final push (Sec. 2.1 finalpush, Sec. 2.3 in r-z)
            p.oz += a.kz * Ez;
            carry(p.oz, p.i);
            const T ro = p.orr + a.kr * Er;
            const T fl = m_floor(ro);
            int jn = p.j + (int)fl;
            bool axis = false;
            if (jn < 0) {  // through the axis: |r|, |v_r|, |a_r|
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
            if (XYZ) p.at = (T)0.5 * p.at;  // no E_theta
            if (axis) {
                if (XYZ) {  // through the axis to the opposite azimuth
                    p.vr = -p.vr;
                    p.ar = -p.ar;
                    p.vt = -p.vt;
                    p.at = -p.at;
                } else {  // |v_r|, |a_r| (Sec. 2.3)
                    p.vr = m_abs(p.vr);
                    p.ar = m_abs(p.ar);
                }
            }
            bool alive = true;
            // one test for all: a NaN or infinity anywhere makes the sum
            // non-finite (the values are far below overflow)
            if (!in_mesh || !m_finite(p.oz + p.orr + p.vr + p.vt + p.vz + p.w)) {
                atomicOr(&a.ds->status, ST_NAN);
                alive = false;
            }
            int wall = alive ? wall_of(p.i, p.oz, p.j, a.nz, a.nr) : -1;
            if (wall >= 0) {
                atomicAdd(&bt.cnt[PIC_C_ABS + a.s * 3 + wall], 1ull);
                atomicAdd(&bt.q[wall], (double)p.w * a.qch[a.s]);
                alive = false;
            }
            if (alive) {
                collide(a, &bt, id, step, p);
                if (a.eedf) {
                    const T Ek = a.half_m_e * (p.vr * p.vr + p.vt * p.vt + p.vz * p.vz);
                    const T x = Ek * a.eedf_scale;
                    if (x >= (T)0 && x < (T)a.eedf_bins)
                        atomicAdd(&s_eedf[(int)x * kEedfCopies + (lane & (kEedfCopies - 1))], p.w);
                }
                if (do_split) {  // weight-conserving split (Sec. 2.2)
                    const T wr_ = a.w_ref[p.j];
                    if (p.w > wr_) {
                        T Nf = m_floor(p.w / wr_);
                        if (Nf > (T)kSplitNMax) Nf = (T)kSplitNMax;
                        int Nc = (int)Nf;
                        T rem = p.w - Nf * wr_;
                        if (!(rem > (T)0)) {
                            Nc -= 1;
                            rem = p.w - (T)Nc * wr_;
                        }
                        if (Nc > 0) {
                            atomicAdd(&bt.cnt[PIC_C_SPLITS + a.s], 1ull);
                            PS<T> cp = p;
                            cp.w = wr_;
                            p.w = rem;
                            for (int c = 0; c < Nc; ++c) emit_birth(a, &bt, a.s, a.s, id, 2 + c, cp);
                        }
                    }
                }
                if (XYZ)
                    first_push_xyz(a, p);
                else
                    first_push(a, p);
                wall = wall_of(p.i, p.oz, p.j, a.nz, a.nr);
                if (wall >= 0) {
                    atomicAdd(&bt.cnt[PIC_C_ABS + a.s * 3 + wall], 1ull);
                    atomicAdd(&bt.q[wall], (double)p.w * a.qch[a.s]);
                    alive = false;
                }
            }
            if (alive) {
                out_cell = p.j * a.ncz + p.i;
                // deposit weights at the new x~ (Sec. 2.4)
                T r0, r1;
                shape_r(a.weighting, p.j, p.orr, r0, r1);
                const T y0 = (T)1 - p.oz, y1 = p.oz;
                c00 = p.w * y0 * r0;
                c01 = p.w * y0 * r1;
                c10 = p.w * y1 * r0;
                c11 = p.w * y1 * r1;
            }
            store_p(a.dst_main, k, p, out_cell, id);
            if (XYZ) a.dst_main.at[k] = p.at;
        }
        // runs of lanes with one output cell: sum each run into its first
        // lane, which makes the four deposit reductions and the histogram count
        const int cprev = __shfl_up_sync(0xffffffffu, out_cell, 1);
        const bool head = lane == 0 || cprev != out_cell;
        const unsigned heads = __ballot_sync(0xffffffffu, head);
        const unsigned above = heads & ~((2u << lane) - 1u);
        const int rend = above ? __ffs(above) - 1 : 32;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const T t00 = __shfl_down_sync(0xffffffffu, c00, d);
            const T t01 = __shfl_down_sync(0xffffffffu, c01, d);
            const T t10 = __shfl_down_sync(0xffffffffu, c10, d);
            const T t11 = __shfl_down_sync(0xffffffffu, c11, d);
            if (lane + d < rend) {
                c00 += t00;
                c01 += t01;
                c10 += t10;
                c11 += t11;
            }
        }
        if (head && out_cell >= 0) {
            atomicAdd(a.counts[a.s] + out_cell, rend - lane);
            int ci, cj;
            decode_cell(out_cell, a.ncz, a.inv_ncz, ci, cj);
            double *g = a.N[a.s] + (size_t)ci * a.nr + cj;
            atomicAdd(g, (double)c00);
            atomicAdd(g + 1, (double)c01);
            atomicAdd(g + a.nr, (double)c10);
            atomicAdd(g + a.nr + 1, (double)c11);
        }
    };
    // Work is claimed from a counter in slots of 32 consecutive particles.
    // The direct-load shapes, while the pass is far from its end, claim a
    // block's kPPT x kThreads particles at a time (its warps load
    // neighbouring particles together, whose sources lie together: faster
    // at 1e7 particles and more).  Otherwise each warp claims on its own,
    // up to kPPT slots, shrinking to one slot over the last 2 x (warps x
    // kPPT) slots (guided self-scheduling): no warp waits for another of its
    // block, and the pass ends within about one slot's time.  A unit's
    // width follows the latest claim its claimer knows of (the counter only
    // grows, so a width is never too small).  The next claim is made while
    // the current unit is worked on; the prefetching shapes claim two ahead
    // and read the next unit's perm entries early.
    const int nslots = (n + 31) >> 5;
    const int twice_warps = 2 * (int)gridDim.x * (kThreads / 32);
    constexpr int kBlockSlots = kPPT * (kThreads / 32);
    const int bulk_end = nslots - twice_warps * kPPT;  // block claims start before it
    auto width = [&](int at) { return max(1, min(kPPT, (nslots - at) / twice_warps)); };
    int pn[kPPT];  // this thread's perm entries of its next unit
    // the next unit's perm entries: a block unit's slot m is kThreads
    // particles on from its slot m-1, a warp unit's 32 (only its w slots)
    auto perm_ahead = [&](int c, int w, bool blk_unit) {
#pragma unroll
        for (int m = 0; m < kPPT; ++m) {
            const int k = c * 32 + (blk_unit ? m * kThreads + tid : m * 32 + lane);
            pn[m] = (blk_unit || m < w) && k < n ? a.perm[k] : 0;
        }
    };
    __shared__ int s_claim;
    bool blk = !PF && bulk_end > 0;  // block claims (block-uniform)
    int cl, cw, cn = 0, cnw = 0;
    // a warp's first claims (two for the prefetching shapes)
    auto warp_start = [&]() {
        int x = 0, y = 0;
        cw = cnw = width(max(bulk_end, 0));
        if (lane == 0) {
            x = atomicAdd(a.chunk_next, cw);
            if (PF) y = atomicAdd(a.chunk_next, cnw);
        }
        cl = __shfl_sync(0xffffffffu, x, 0);
        if (PF) cn = __shfl_sync(0xffffffffu, y, 0);
    };
    if (blk) {
        if (tid == 0) s_claim = atomicAdd(a.chunk_next, kBlockSlots);
        __syncthreads();
        cl = s_claim;
        cw = kBlockSlots;
    } else {
        warp_start();
    }
    if (PF) perm_ahead(cl, cw, blk);
    for (;;) {
        if (cl >= nslots) {
            if (!blk) break;
            blk = false;  // the block's last unit is done: the rest warp by warp
            warp_start();
            if (PF) perm_ahead(cl, cw, false);
            continue;
        }
        const int stride = blk ? kThreads : 32, off = blk ? tid : lane;
        const int base = cl * 32;
        const int nslot = blk ? kPPT : min(cw, nslots - cl);
        const int end = min(base + (blk ? kBlockSlots : nslot) * 32, n);
        int claim = 0, w;
        if (blk) {
            const bool more = cl + kBlockSlots < bulk_end;  // block-uniform
            __syncthreads();  // every thread has read s_claim
            if (tid == 0 && more) s_claim = atomicAdd(a.chunk_next, kBlockSlots);
            __syncthreads();
            claim = more ? s_claim : nslots;
            w = kBlockSlots;
        } else {
            w = width(PF ? cn + cnw : cl + cw);
            if (lane == 0) claim = atomicAdd(a.chunk_next, w);
        }
        // request the unit's particles, then read the next unit's perm
        // entries; a thread fills and reads only its own slots
        if (PF) {
#pragma unroll
            for (int m = 0; m < kPPT; ++m) {
                const int k = base + m * stride + off;
                if (k < end) fetch(pn[m], m * kThreads + tid);
            }
            asm volatile("cp.async.commit_group;" ::: "memory");
            if (blk)
                perm_ahead(claim, w, true);
            else
                perm_ahead(cn, cnw, false);
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
#pragma unroll 1
        for (int m = 0; m < nslot; ++m) {
            const int k = base + m * stride + off;
            process(k, k < end, m * kThreads + tid);
        }
        if (blk) {
            cl = claim;
        } else if (PF) {
            cl = cn;
            cw = cnw;
            cn = __shfl_sync(0xffffffffu, claim, 0);
            cnw = w;
        } else {
            cl = __shfl_sync(0xffffffffu, claim, 0);
            cw = w;
        }
    }
    __syncthreads();
    for (int k = tid; k < PIC_NCOUNT; k += blockDim.x)
        if (bt.cnt[k]) atomicAdd(&a.ds->cnt[k], bt.cnt[k]);
    if (tid < 3 && bt.q[tid] != 0.0) {
        atomicAdd(&a.ds->qabs[tid], bt.q[tid]);
        atomicAdd(&a.ds->qstep[tid], bt.q[tid]);
    }
    if (a.eedf)
        for (int k = tid; k < a.eedf_bins; k += blockDim.x) {
            double v = 0.0;
            for (int c = 0; c < kEedfCopies; ++c) v += (double)s_eedf[k * kEedfCopies + c];
            if (v != 0.0) atomicAdd(a.eedf + k, v);
        }
}

template <typename T, bool PF, int PPT, bool XYZ>
void launch_shape(const StepArgs<T> &a, int grid, cudaStream_t st) {
    const size_t stage =
        PF ? (size_t)kThreads * PPT *
                 (2 * sizeof(typename V4<T>::type) + sizeof(uint64_t) + sizeof(int32_t) + (XYZ ? sizeof(T) : 0))
           : 0;
    const size_t eedf = (size_t)(a.eedf ? a.eedf_bins : 0) * kEedfCopies * sizeof(T);
    const size_t smem = stage + eedf;
    // dynamic plus static shared memory above 48 KB needs the opt-in: set
    // it for every size (the static tallies come on top of `smem`)
    if (smem > 0)
        cudaFuncSetAttribute(k_step<T, PF, PPT, XYZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // blocks claim chunks until none is left: as many as are resident at once
    int per_sm = 0, dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step<T, PF, PPT, XYZ>, kThreads, smem);
    if (per_sm > 0 && nsm > 0) grid = std::min(grid, per_sm * nsm);
    k_step<T, PF, PPT, XYZ><<<grid, kThreads, smem, st>>>(a);
}

template <typename T, bool PF, int PPT>
void launch_variant(const StepArgs<T> &a, int grid, cudaStream_t st) {
    if (a.xyz)
        launch_shape<T, PF, PPT, true>(a, grid, st);
    else
        launch_shape<T, PF, PPT, false>(a, grid, st);
}

// variant: bit 0 = prefetch the chunk into shared memory, bit 1 = 8
// particles per thread (else 4); -1 = the default for the species, the
// faster shape on GB300 at 1e7 particles per species: ions prefetch 4 per
// thread (their pass is latency-bound), electrons load directly, 8 per
// thread (theirs is bound by issue)
template <typename T>
void launch_step(const StepArgs<T> &a, int grid, int variant, cudaStream_t st) {
    const int v = variant >= 0 ? (variant & 3) : (a.s == 1 ? 1 : 2);
    switch (v) {
        case 0: launch_variant<T, false, 4>(a, grid, st); break;
        case 1: launch_variant<T, true, 4>(a, grid, st); break;
        case 2: launch_variant<T, false, 8>(a, grid, st); break;
        default: launch_variant<T, true, 8>(a, grid, st); break;
    }
}

// ---------------------------------------------------------------------------
// load: uniform density n0, weights ~ cell volume (Sec. 2.2, Eq. (3))
// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_load(PBuf<T> dst, int64_t n, int s, int nz, int nr, double dz, double dr,
                       double n0, double T_eV, double m, uint32_t k0, uint32_t k1,
                       int64_t ncell) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    const int ncz = nz - 1;
    const int64_t base = n / ncell, rem = n % ncell;
    const int64_t c = p < rem * (base + 1) ? p / (base + 1) : rem + (p - rem * (base + 1)) / base;
    const int64_t ppc = base + (c < rem ? 1 : 0);
    const int i = (int)(c % ncz), j = (int)(c / ncz);
    const uint4 x = draw(k0, k1, (uint64_t)p, 0xFFFFFFFFu, 3, s);
    const uint4 y = draw(k0, k1, (uint64_t)p, 0xFFFFFFFFu, 4, s);
    const double oz = unif<double>(x.x);
    // uniform in r^2 inside the cell: offset = u(2j+1) / (sqrt(j^2 + u(2j+1)) + j)
    const double t = unif<double>(x.y) * (2.0 * j + 1.0);
    const double orr = t / (sqrt((double)j * j + t) + (double)j);
    double g0, g1, g2, g3;
    normals<double>(x.z, x.w, g0, g1);
    normals<double>(y.x, y.y, g2, g3);
    const double sig = sqrt(T_eV * kQe / m);
    const double r0 = j * dr, r1 = (j + 1) * dr;
    const double w = n0 * kPi * (r1 * r1 - r0 * r0) * dz / (double)ppc;
    PS<T> q;
    q.i = i;
    q.j = j;
    q.oz = (T)oz < (T)1 ? (T)oz : below_one<T>();
    q.orr = (T)orr < (T)1 ? (T)orr : below_one<T>();
    q.vr = (T)(sig * g0);
    q.vt = (T)(sig * g1);
    q.vz = (T)(sig * g2);
    q.ar = q.az = (T)0;
    q.w = (T)w;
    store_p(dst, (int)p, q, (int)c, (uint64_t)p);
    if (dst.at) dst.at[p] = (T)0;
}

template <typename T>
void launch_load(PBuf<T> dst, int64_t n, int s, int nz, int nr, double dz, double dr, double n0,
                 double T_eV, double m, uint32_t key0, uint32_t key1, int64_t ncell,
                 cudaStream_t st) {
    if (n <= 0) return;
    k_load<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, n, s, nz, nr, dz, dr, n0, T_eV, m,
                                                            key0, key1, ncell);
}

// plain deposit of entries [0, n) (used after a load or an upload)
template <typename T>
__global__ void k_deposit(PBuf<T> src, const int32_t *n_dev, int nz, int nr, int weighting,
                          double *N) {
    const int n = *n_dev;
    const int ncz = nz - 1;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        if (src.cell[k] < 0) continue;
        PS<T> p = load_p(src, k, ncz);
        deposit_global(N, nr, weighting, p);
    }
}

template <typename T>
void launch_deposit(PBuf<T> src, const int32_t *n_dev, int nz, int nr, int weighting, double *N,
                    cudaStream_t st) {
    k_deposit<T><<<152 * 8, 256, 0, st>>>(src, n_dev, nz, nr, weighting, N);
}

// absolute (r, z) -> cell + offsets
template <typename T>
__global__ void k_from_abs(PBuf<T> dst, int64_t n, const double *r, const double *z,
                           const double *vr, const double *vt, const double *vz, const double *ar,
                           const double *az, const double *w, const uint64_t *id, const double *at,
                           int nz, int nr, double dz, double dr) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double xz = z[k] / dz, xr = r[k] / dr;
    int i = (int)floor(xz), j = (int)floor(xr);
    i = i < 0 ? 0 : (i > nz - 2 ? nz - 2 : i);
    j = j < 0 ? 0 : (j > nr - 2 ? nr - 2 : j);
    PS<T> q;
    q.i = i;
    q.j = j;
    const T oz = (T)(xz - i), orr = (T)(xr - j);
    q.oz = oz < (T)1 ? (oz < (T)0 ? (T)0 : oz) : below_one<T>();
    q.orr = orr < (T)1 ? (orr < (T)0 ? (T)0 : orr) : below_one<T>();
    q.vr = (T)vr[k];
    q.vt = (T)vt[k];
    q.vz = (T)vz[k];
    q.ar = (T)ar[k];
    q.az = (T)az[k];
    q.w = (T)w[k];
    store_p(dst, (int)k, q, j * (nz - 1) + i, id[k]);
    if (dst.at) dst.at[k] = at ? (T)at[k] : (T)0;
}

template <typename T>
void launch_from_abs(PBuf<T> dst, int64_t n, const double *r, const double *z, const double *vr,
                     const double *vt, const double *vz, const double *ar, const double *az,
                     const double *w, const uint64_t *id, const double *at, int nz, int nr, double dz,
                     double dr, cudaStream_t st) {
    if (n <= 0) return;
    k_from_abs<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, n, r, z, vr, vt, vz, ar, az, w,
                                                                id, at, nz, nr, dz, dr);
}

// cell + offsets -> absolute, in perm order
template <typename T>
__global__ void k_to_abs(PBuf<T> sm, PBuf<T> sb, const int32_t *n_main_src, const int32_t *perm,
                         int64_t n, double *r, double *z, double *vr, double *vt, double *vz,
                         double *ar, double *az, double *w, uint64_t *id, int32_t *cell, double *at,
                         int nz, double dz, double dr) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int nmain = *n_main_src;
    const int p = perm[k];
    const PBuf<T> &src = p < nmain ? sm : sb;
    const int si = p < nmain ? p : p - nmain;
    PS<T> q = load_p(src, si, nz - 1);
    z[k] = ((double)q.i + (double)q.oz) * dz;
    r[k] = ((double)q.j + (double)q.orr) * dr;
    vr[k] = q.vr;
    vt[k] = q.vt;
    vz[k] = q.vz;
    ar[k] = q.ar;
    az[k] = q.az;
    w[k] = q.w;
    id[k] = src.id[si];
    cell[k] = src.cell[si];
    if (at) at[k] = src.at ? (double)src.at[si] : 0.0;
}

template <typename T>
void launch_to_abs(PBuf<T> sm, PBuf<T> sb, const int32_t *n_main_src, const int32_t *perm,
                   int64_t n, double *r, double *z, double *vr, double *vt, double *vz, double *ar,
                   double *az, double *w, uint64_t *id, int32_t *cell, double *at, int nz, double dz,
                   double dr, cudaStream_t st) {
    if (n <= 0) return;
    k_to_abs<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(sm, sb, n_main_src, perm, n, r, z, vr,
                                                              vt, vz, ar, az, w, id, cell, at, nz, dz,
                                                              dr);
}

// ---------------------------------------------------------------------------
// merging of light particles in pairs (Sec. 2.2 names the need, no
// algorithm): one block per cell of the sorted store.  The cell's particles
// lighter than frac * w_r(j) are collected in shared memory, sorted by
// (velocity bin, id), and consecutive ones of a bin are merged in pairs
// into the lower id: w, z, r^2, v_r, v_z, a_r, a_z as weighted means,
// v_theta (and a_theta) from the angular momentum at the merged radius.
// The other one of a pair is left as a dead record (cell -1), which the
// re-sort that follows drops.
// ---------------------------------------------------------------------------
constexpr int kMergeCap = 1024;  // light particles of one cell a block can take
constexpr int kMergeThreads = 256;

__device__ __forceinline__ uint64_t vbin_of(double v, double dv) {
    double b = floor(v / dv);
    b = fmin(fmax(b, -1048576.0), 1048575.0);
    return (uint64_t)((int64_t)b + 1048576);
}

__device__ __forceinline__ bool key_less(uint64_t ka, uint64_t ia, uint64_t kb, uint64_t ib) {
    return ka < kb || (ka == kb && ia < ib);
}

template <typename T>
__global__ void __launch_bounds__(kMergeThreads)
    k_merge(PBuf<T> mainb, PBuf<T> births, const int32_t *nmain_dev, const int32_t *perm, const int32_t *cursor,
            int ncell, int ncz, double dz, double dr, const T *w_ref, double frac, double dv, double mass, int xyz,
            unsigned long long *pairs_out, double *energy_out, int *overflow) {
    __shared__ uint64_t s_key[kMergeCap], s_id[kMergeCap];
    __shared__ int32_t s_loc[kMergeCap], s_first[kMergeCap / 2];
    __shared__ int s_n, s_np;
    __shared__ double s_red[kMergeThreads / 32];
    __shared__ unsigned long long s_cnt[kMergeThreads / 32];
    const int tid = threadIdx.x;
    const int nmain = *nmain_dev;
    double e_mine = 0.0;
    unsigned long long p_mine = 0;
    for (int c = blockIdx.x; c < ncell; c += gridDim.x) {
        // cursor holds each cell's end in the permutation (after the rank)
        const int start = c > 0 ? cursor[c - 1] : 0, end = cursor[c];
        if (end - start >= 2) {
            const int i = c % ncz, j = c / ncz;
            const double thr = frac * (double)w_ref[j];
            if (tid == 0) s_n = 0;
            __syncthreads();
            for (int q = start + tid; q < end; q += blockDim.x) {
                const int loc = perm[q];
                const bool in_main = loc < nmain;
                const PBuf<T> &b = in_main ? mainb : births;
                const int k = in_main ? loc : loc - nmain;
                const PS<T> p = load_p(b, k, ncz);
                if ((double)p.w < thr) {
                    const int slot = atomicAdd(&s_n, 1);
                    if (slot < kMergeCap) {
                        s_key[slot] = (vbin_of((double)p.vr, dv) << 42) | (vbin_of((double)p.vt, dv) << 21) |
                                      vbin_of((double)p.vz, dv);
                        s_id[slot] = b.id[k];
                        s_loc[slot] = loc;
                    }
                }
            }
            __syncthreads();
            const int n = s_n;
            if (n > kMergeCap) {
                if (tid == 0) atomicExch(overflow, 1);
            } else if (n >= 2) {
                int P = 2;
                while (P < n) P <<= 1;
                for (int t = n + tid; t < P; t += blockDim.x) {
                    s_key[t] = ~0ull;
                    s_id[t] = ~0ull;
                    s_loc[t] = -1;
                }
                __syncthreads();
                // bitonic sort by (bin, id)
                for (int kk = 2; kk <= P; kk <<= 1)
                    for (int jj = kk >> 1; jj > 0; jj >>= 1) {
                        for (int t = tid; t < P; t += blockDim.x) {
                            const int u = t ^ jj;
                            if (u > t) {
                                const bool up = (t & kk) == 0;
                                const bool gt = key_less(s_key[u], s_id[u], s_key[t], s_id[t]);
                                if (up == gt) {
                                    const uint64_t k0 = s_key[t], i0 = s_id[t];
                                    const int32_t l0 = s_loc[t];
                                    s_key[t] = s_key[u];
                                    s_id[t] = s_id[u];
                                    s_loc[t] = s_loc[u];
                                    s_key[u] = k0;
                                    s_id[u] = i0;
                                    s_loc[u] = l0;
                                }
                            }
                        }
                        __syncthreads();
                    }
                // pairs: consecutive entries of one bin, from the bin's first
                if (tid == 0) {
                    int np = 0;
                    for (int u = 0; u < n;) {
                        int e = u + 1;
                        while (e < n && s_key[e] == s_key[u]) ++e;
                        for (int v = u; v + 1 < e; v += 2) s_first[np++] = v;
                        u = e;
                    }
                    s_np = np;
                }
                __syncthreads();
                for (int q = tid; q < s_np; q += blockDim.x) {
                    const int u = s_first[q];
                    const int la = s_loc[u], lb = s_loc[u + 1];
                    const PBuf<T> &ba = la < nmain ? mainb : births;
                    const PBuf<T> &bb = lb < nmain ? mainb : births;
                    const int ka = la < nmain ? la : la - nmain, kb = lb < nmain ? lb : lb - nmain;
                    const PS<T> a = load_p(ba, ka, ncz), b = load_p(bb, kb, ncz);
                    const double wa = a.w, wb = b.w, W = wa + wb;
                    const double za = (i + (double)a.oz) * dz, zb = (i + (double)b.oz) * dz;
                    const double ra = (j + (double)a.orr) * dr, rb = (j + (double)b.orr) * dr;
                    const double r = sqrt((wa * ra * ra + wb * rb * rb) / W);
                    const double vr = (wa * a.vr + wb * b.vr) / W, vz = (wa * a.vz + wb * b.vz) / W;
                    const double vt = r > 0.0 ? (wa * ra * a.vt + wb * rb * b.vt) / (W * r) : (wa * a.vt + wb * b.vt) / W;
                    const double e0 = wa * ((double)a.vr * a.vr + (double)a.vt * a.vt + (double)a.vz * a.vz) +
                                      wb * ((double)b.vr * b.vr + (double)b.vt * b.vt + (double)b.vz * b.vz);
                    e_mine += 0.5 * mass * (e0 - W * (vr * vr + vt * vt + vz * vz));
                    double oz = ((wa * za + wb * zb) / W) / dz - i, orr = r / dr - j;
                    oz = fmin(fmax(oz, 0.0), (double)below_one<T>());
                    orr = fmin(fmax(orr, 0.0), (double)below_one<T>());
                    PS<T> m = a;
                    m.oz = (T)oz;
                    m.orr = (T)orr;
                    m.vr = (T)vr;
                    m.vt = (T)vt;
                    m.vz = (T)vz;
                    m.ar = (T)((wa * a.ar + wb * b.ar) / W);
                    m.az = (T)((wa * a.az + wb * b.az) / W);
                    m.w = (T)W;
                    store_p(ba, ka, m, c, s_id[u]);
                    if (xyz) {
                        const double ata = ba.at[ka], atb = bb.at[kb];
                        ba.at[ka] = (T)(r > 0.0 ? (wa * ra * ata + wb * rb * atb) / (W * r) : (wa * ata + wb * atb) / W);
                    }
                    bb.cell[kb] = -1;
                    ++p_mine;
                }
            }
        }
        __syncthreads();  // the cell's shared arrays are free again
    }
    // block sums of the energy lost and the pairs merged
    const int lane = tid & 31, warp = tid >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        e_mine += __shfl_down_sync(0xffffffffu, e_mine, o);
        p_mine += __shfl_down_sync(0xffffffffu, p_mine, o);
    }
    if (lane == 0) {
        s_red[warp] = e_mine;
        s_cnt[warp] = p_mine;
    }
    __syncthreads();
    if (tid == 0) {
        double e = 0.0;
        unsigned long long p = 0;
        for (int w = 0; w < kMergeThreads / 32; ++w) {
            e += s_red[w];
            p += s_cnt[w];
        }
        if (p) {
            atomicAdd(energy_out, e);
            atomicAdd(pairs_out, p);
        }
    }
}

template <typename T>
void launch_merge(PBuf<T> mainb, PBuf<T> births, const int32_t *nmain_dev, const int32_t *perm,
                  const int32_t *cursor, int ncell, int ncz, double dz, double dr, const T *w_ref, double frac,
                  double dv, double mass, int xyz, unsigned long long *pairs, double *energy, int *overflow,
                  cudaStream_t st) {
    const int grid = std::max(1, std::min(ncell, 152 * 4));
    k_merge<T><<<grid, kMergeThreads, 0, st>>>(mainb, births, nmain_dev, perm, cursor, ncell, ncz, dz, dr, w_ref,
                                                frac, dv, mass, xyz, pairs, energy, overflow);
}

#define PIC_INST(T)                                                                              \
    template void launch_step<T>(const StepArgs<T> &, int, int, cudaStream_t);                   \
    template void launch_merge<T>(PBuf<T>, PBuf<T>, const int32_t *, const int32_t *, const int32_t *, int, \
                                  int, double, double, const T *, double, double, double, int,             \
                                  unsigned long long *, double *, int *, cudaStream_t);                    \
    template void launch_load<T>(PBuf<T>, int64_t, int, int, int, double, double, double, double, \
                                 double, uint32_t, uint32_t, int64_t, cudaStream_t);              \
    template void launch_deposit<T>(PBuf<T>, const int32_t *, int, int, int, double *,           \
                                    cudaStream_t);                                               \
    template void launch_from_abs<T>(PBuf<T>, int64_t, const double *, const double *,          \
                                     const double *, const double *, const double *,            \
                                     const double *, const double *, const double *,            \
                                     const uint64_t *, const double *, int, int, double, double, \
                                     cudaStream_t);                                              \
    template void launch_to_abs<T>(PBuf<T>, PBuf<T>, const int32_t *, const int32_t *, int64_t,  \
                                   double *, double *, double *, double *, double *, double *,   \
                                   double *, double *, uint64_t *, int32_t *, double *, int,     \
                                   double, double, cudaStream_t);
PIC_INST(float)
PIC_INST(double)

}  // namespace pic
