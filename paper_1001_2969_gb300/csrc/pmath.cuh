// pmath.cuh -- per-particle arithmetic shared by the particle kernels
// (particles.cu) and the collisionless window with its adjoint (window.cu):
// type-generic math, 128-bit access to the particle record, the cell
// decode, shape factors, walls and the first push.
#pragma once

#include <math.h>

#include "pic_internal.cuh"

namespace pic {

// type-generic math
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_pow(float x, float y) { return powf(x, y); }
__device__ __forceinline__ double m_pow(double x, double y) { return pow(x, y); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
// x^R for x >= 1, R in (0, 1): FP32 through the hardware base-2 log/exp
__device__ __forceinline__ float m_powR(float x, float R) { return exp2f(R * __log2f(x)); }
__device__ __forceinline__ double m_powR(double x, double R) { return pow(x, R); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_tan(float x) { return tanf(x); }
__device__ __forceinline__ double m_tan(double x) { return tan(x); }
__device__ __forceinline__ float m_atan(float x) { return atanf(x); }
__device__ __forceinline__ double m_atan(double x) { return atan(x); }
__device__ __forceinline__ void m_sincos2pi(float u, float *s, float *c) { sincospif(2.0f * u, s, c); }
__device__ __forceinline__ void m_sincos2pi(double u, double *s, double *c) { sincospi(2.0 * u, s, c); }
__device__ __forceinline__ bool m_finite(float x) { return isfinite(x); }
__device__ __forceinline__ bool m_finite(double x) { return isfinite(x); }
// a / b: IEEE in FP64; in FP32 the approximate division (2 ulp), used only
// where the result feeds positions/weights (never a threshold test on its own)
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ float m_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double m_rsqrt(double x) { return 1.0 / sqrt(x); }

template <typename T>
__device__ __forceinline__ T below_one();
template <>
__device__ __forceinline__ float below_one<float>() { return 0.99999994f; }
template <>
__device__ __forceinline__ double below_one<double>() { return 0.99999999999999989; }

// 128-bit vector access
__device__ __forceinline__ void ld4(const float4 *p, float &a, float &b, float &c, float &d) {
    float4 v = *p;
    a = v.x;
    b = v.y;
    c = v.z;
    d = v.w;
}
__device__ __forceinline__ void ld4(const dbl4 *p, double &a, double &b, double &c, double &d) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
    double2 u = q[0], v = q[1];
    a = u.x;
    b = u.y;
    c = v.x;
    d = v.y;
}
__device__ __forceinline__ void st4(float4 *p, float a, float b, float c, float d) {
    *p = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(dbl4 *p, double a, double b, double c, double d) {
    double2 *q = reinterpret_cast<double2 *>(p);
    q[0] = make_double2(a, b);
    q[1] = make_double2(c, d);
}

// particle in registers
template <typename T>
struct PS {
    int i, j;
    T oz, orr, vr, vt, vz, ar, az, w;
    T at;  // a_theta: read and written by the X-Y-Z pusher only
};

// c = j ncz + i -> (i, j) without an integer division: (c + 1/2)/ncz lies
// strictly inside (j, j+1), far from its ends compared with FP32 rounding
// for c < 2^24; one correction step covers the rest
__device__ __forceinline__ void decode_cell(int c, int ncz, float inv_ncz, int &i, int &j) {
    int jj = __float2int_rz(((float)c + 0.5f) * inv_ncz);
    int ii = c - jj * ncz;
    if (ii < 0) {
        jj -= 1;
        ii += ncz;
    } else if (ii >= ncz) {
        jj += 1;
        ii -= ncz;
    }
    i = ii;
    j = jj;
}

template <typename T>
__device__ __forceinline__ PS<T> load_p_fast(const PBuf<T> &b, int idx, int ncz, float inv_ncz) {
    PS<T> p;
    ld4(b.q0 + idx, p.oz, p.orr, p.vr, p.vt);
    ld4(b.q1 + idx, p.vz, p.ar, p.az, p.w);
    decode_cell(b.cell[idx], ncz, inv_ncz, p.i, p.j);
    return p;
}

template <typename T>
__device__ __forceinline__ PS<T> load_p(const PBuf<T> &b, int idx, int ncz) {
    PS<T> p;
    ld4(b.q0 + idx, p.oz, p.orr, p.vr, p.vt);
    ld4(b.q1 + idx, p.vz, p.ar, p.az, p.w);
    int c = b.cell[idx];
    p.i = c % ncz;
    p.j = c / ncz;
    return p;
}

template <typename T>
__device__ __forceinline__ void store_p(const PBuf<T> &b, int idx, const PS<T> &p, int cell,
                                        uint64_t id) {
    st4(b.q0 + idx, p.oz, p.orr, p.vr, p.vt);
    st4(b.q1 + idx, p.vz, p.ar, p.az, p.w);
    b.cell[idx] = cell;
    b.id[idx] = id;
}

// radial shape factors of Eq. (9) (z-r^2) or Eq. (8) (z-r) in offset form:
// z-r^2: S_{j+1} = (r^2 - r_j^2)/(r_{j+1}^2 - r_j^2) = o (2j + o)/(2j + 1)
template <typename T>
__device__ __forceinline__ void shape_r(int weighting, int j, T o, T &s0, T &s1) {
    if (weighting == PIC_WEIGHT_ZR) {
        s1 = o;
        s0 = (T)1 - o;
    } else if (sizeof(T) == 4) {
        const T t = (T)(2 * j + 1);
        const T it = m_div((T)1, t);
        s1 = o * ((T)(2 * j) + o) * it;
        s0 = ((T)1 - o) * (t + o) * it;
    } else {
        const T t = (T)(2 * j + 1);
        s1 = m_div(o * ((T)(2 * j) + o), t);
        s0 = m_div(((T)1 - o) * (t + o), t);
    }
}

template <typename T>
__device__ __forceinline__ void carry(T &off, int &idx) {
    const T f = m_floor(off);
    idx += (int)f;
    off -= f;
}

// wall of a stored position (domain 0 < z < L, 0 <= r < R; z walls first)
template <typename T>
__device__ __forceinline__ int wall_of(int i, T oz, int j, int nz, int nr) {
    if (i < 0 || (i == 0 && oz == (T)0)) return 0;
    if (i >= nz - 1) return 1;
    if (j >= nr - 1) return 2;
    return -1;
}

// first push of Sec. 2.3 in the local X-Y frame, then the rotation by theta
// back to r-theta; a_theta = 0, so v_y' = v_theta and a_r' = a_r cos(theta).
// The radial step is formed without cancellation:
// r' - r = (2 r dx + dx^2 + dy^2) / (r' + r).
template <typename T>
__device__ __forceinline__ void first_push(const StepArgs<T> &a, PS<T> &p, const T dt, const T dt_dz) {
    const T vx = p.vr + (T)0.5 * p.ar * dt;
    const T vy = p.vt;
    const T vz = p.vz + (T)0.5 * p.az * dt;
    p.oz += vz * dt_dz;
    carry(p.oz, p.i);
    const T r = ((T)p.j + p.orr) * a.dr;
    const T dx = vx * dt, dy = vy * dt;
    const T xr = r + dx;
    const T q2 = xr * xr + dy * dy;
    T c = (T)1, sn = (T)0, rn = (T)0;
    if (q2 > (T)0) {
        if (sizeof(T) == 4) {
            const T inv = m_rsqrt(q2);
            rn = q2 * inv;
            c = xr * inv;
            sn = dy * inv;
        } else {
            rn = m_sqrt(q2);
            c = xr / rn;
            sn = dy / rn;
        }
    }
    const T den = rn + r;
    const T drr = den > (T)0 ? m_div((T)2 * r * dx + dx * dx + dy * dy, den) : (T)0;
    T ro = p.orr + drr * a.inv_dr;
    const T fl = m_floor(ro);
    int jn = p.j + (int)fl;
    ro -= fl;
    if (jn < 0) {
        jn = 0;
        ro = (T)0;
    }
    p.j = jn;
    p.orr = ro;
    p.vr = vx * c + vy * sn;
    p.vt = -vx * sn + vy * c;
    p.vz = vz;
    p.ar = p.ar * c;
}
// the species' own step (a newborn of another species passes that one's)
template <typename T>
__device__ __forceinline__ void first_push(const StepArgs<T> &a, PS<T> &p) {
    first_push(a, p, a.dt, a.dt_dz);
}

// the same in the global X-Y-Z form (Sec. 2.3, end) for a particle taken at
// azimuth 0 (the field is axisymmetric): v_y' = v_theta + a_theta dt / 2,
// and (a_r, a_theta) rotate onto the new local frame with (v_x, v_y)
template <typename T>
__device__ __forceinline__ void first_push_xyz(const StepArgs<T> &a, PS<T> &p, const T dt, const T dt_dz) {
    const T vx = p.vr + (T)0.5 * p.ar * dt;
    const T vy = p.vt + (T)0.5 * p.at * dt;
    const T vz = p.vz + (T)0.5 * p.az * dt;
    p.oz += vz * dt_dz;
    carry(p.oz, p.i);
    const T r = ((T)p.j + p.orr) * a.dr;
    const T dx = vx * dt, dy = vy * dt;
    const T xr = r + dx;
    const T q2 = xr * xr + dy * dy;
    T c = (T)1, sn = (T)0, rn = (T)0;
    if (q2 > (T)0) {
        if (sizeof(T) == 4) {
            const T inv = m_rsqrt(q2);
            rn = q2 * inv;
            c = xr * inv;
            sn = dy * inv;
        } else {
            rn = m_sqrt(q2);
            c = xr / rn;
            sn = dy / rn;
        }
    }
    const T den = rn + r;
    const T drr = den > (T)0 ? m_div((T)2 * r * dx + dx * dx + dy * dy, den) : (T)0;
    T ro = p.orr + drr * a.inv_dr;
    const T fl = m_floor(ro);
    int jn = p.j + (int)fl;
    ro -= fl;
    if (jn < 0) {
        jn = 0;
        ro = (T)0;
    }
    p.j = jn;
    p.orr = ro;
    p.vr = vx * c + vy * sn;
    p.vt = -vx * sn + vy * c;
    p.vz = vz;
    const T arn = p.ar * c + p.at * sn;
    p.at = -p.ar * sn + p.at * c;
    p.ar = arn;
}
// the species' own step (a newborn of another species passes that one's)
template <typename T>
__device__ __forceinline__ void first_push_xyz(const StepArgs<T> &a, PS<T> &p) {
    first_push_xyz(a, p, a.dt, a.dt_dz);
}

}  // namespace pic
