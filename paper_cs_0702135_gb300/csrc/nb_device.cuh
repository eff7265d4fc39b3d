// nb_device.cuh -- device arithmetic shared by every kernel that predicts,
// corrects or sums pair forces, so that the single-system step, the ensemble
// step and the reverse mode evaluate the same formulas bit for bit.
#pragma once

#include <cuda_runtime.h>

#include <cfloat>

#include "nb_internal.cuh"

namespace nbk {
namespace dev {

constexpr double kTick = 0x1p-40;  // one tick in N-body time units

__device__ __forceinline__ double ticks_to_time(long long d)
{
    return __dmul_rn(__ll2double_rn(d), kTick);
}

// 1/sqrt(x) on the SFU: the PTX approximate reciprocal square root with
// flush-to-zero (one MUFU instruction; relative error about 2^-23).  r^2 >=
// eps^2 is never subnormal, so the denormal handling of rsqrtf() would only
// cost issue slots here.
__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Knuth's TwoSum: hi + lo absorbs x, with the rounding error of hi + x in lo.
__device__ __forceinline__ void two_sum_acc(float &hi, float &lo, float x)
{
    float s = hi + x;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += e;
}

// Sum of two double-single values (h, l) += (h2, l2).
__device__ __forceinline__ void ds_add(float &h, float &l, float h2, float l2)
{
    float s = h + h2;
    float bb = s - h;
    float e = (h - (s - bb)) + (h2 - bb);
    h = s;
    l = (l + l2) + e;
}

// a / C rounded to nearest, for the constants C = 3, 12, 20 of the predictor
// and corrector, without an FP64 division (a long sequence on the GB300's
// narrow FP64 pipe): q0 = RN(a y) with y = RN(1/C) is within one ulp of a/C
// (1/C is rounded with relative error 2^-54 for these C), the residual
// r = a - C q0 is exact in one FMA, and RN(q0 + r y) is then RN(a/C) by
// Markstein's theorem (IBM J. Res. Dev. 34, 1990).  Operands outside
// 2^-900 < |a| < 2^1000 (zero with its sign, huge, not finite) take the plain
// division; the range test reads the exponent bits on the integer pipe.
template <int C>
__device__ __forceinline__ double div_by(double a)
{
    static_assert(C == 3 || C == 12 || C == 20, "reciprocal error checked for 3, 12, 20 only");
    const unsigned hi = (unsigned)__double2hiint(a) & 0x7FFFFFFFu;
    if (hi >= (123u << 20) && hi < (2023u << 20)) {
        constexpr double y = 1.0 / C;
        const double q0 = __dmul_rn(a, y);
        const double r = __fma_rn(-q0, (double)C, a);
        return __fma_rn(r, y, q0);
    }
    return __ddiv_rn(a, (double)C);
}

// Hermite predictor (Section 2), round-to-nearest in the formula's order:
//   x_p = x + (v + (dt/2)(a + (dt/3) k)) dt,   v_p = v + (a + (dt/2) k) dt.
// dt/2 is taken as dt * 0.5, the same number (halving is exact for every dt on
// the tick grid), which saves an FP64 division on the GB300's small FP64 pipe.
// With h = dt/2 and q = dt/3 given (one division per particle, not per axis):
__device__ __forceinline__ void predict1hq(double x, double v, double a, double k, double dt,
                                           double h, double q, double &xp, double &vp)
{
    xp = __dadd_rn(x, __dmul_rn(__dadd_rn(v, __dmul_rn(h, __dadd_rn(a, __dmul_rn(q, k)))), dt));
    vp = __dadd_rn(v, __dmul_rn(__dadd_rn(a, __dmul_rn(h, k)), dt));
}

__device__ __forceinline__ void predict1(double x, double v, double a, double k, double dt,
                                         double &xp, double &vp)
{
    predict1hq(x, v, a, k, dt, __dmul_rn(dt, 0.5), div_by<3>(dt), xp, vp);
}

// State loads: plain, or past L1 (CG) for state that other SMs may have
// written earlier in the same launch.
template <bool CG, typename T>
__device__ __forceinline__ T ldst(const T *p)
{
    if (CG) return __ldcg(p);
    return *p;
}

// All three axes of particle i of `s` (component-major, stride n).
template <bool CG = false>
__device__ __forceinline__ void predict3(const State &s, long long i, long long n, double dt,
                                         double xp[3], double vp[3])
{
    const double h = __dmul_rn(dt, 0.5), q = div_by<3>(dt);
#pragma unroll
    for (int c = 0; c < 3; ++c)
        predict1hq(ldst<CG>(&s.x[c * n + i]), ldst<CG>(&s.v[c * n + i]), ldst<CG>(&s.a[c * n + i]),
                   ldst<CG>(&s.k[c * n + i]), dt, h, q, xp[c], vp[c]);
}

// A predicted FP64 position split into double-single: x = hi + lo to 2^-48.
__device__ __forceinline__ void split_ds(double x, float &hi, float &lo)
{
    hi = __double2float_rn(x);
    lo = __double2float_rn(__dsub_rn(x, (double)hi));
}

__device__ __forceinline__ double norm3(double u0, double u1, double u2)
{
    return __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(u0, u0), __dmul_rn(u1, u1)), __dmul_rn(u2, u2)));
}

// Block level of a raw step: k of the largest 2^-k <= dt_raw, from the FP64
// exponent field (dt_raw >= 2^-40 is a normal number), clamped to k >= kmin.
// Returns false when dt_raw is not a number or below 2^-40.
__device__ __forceinline__ bool level_of(double dt_raw, int kmin, int &level)
{
    if (isnan(dt_raw) || dt_raw < 0x1p-40) return false;
    int k;
    if (isinf(dt_raw)) {
        k = kmin;
    } else {
        const long long bits = __double_as_longlong(dt_raw);
        k = 1023 - (int)((bits >> 52) & 0x7FF);
        if (k < kmin) k = kmin;
    }
    level = k;
    return true;
}

// Halve at once; double by one level only when the new time is a multiple of
// the doubled step; never above the largest step.
__device__ __forceinline__ int next_level(int k_old, int k_q, long long t_new, int kmin)
{
    if (k_q > k_old) return k_q;
    if (k_q < k_old && k_old > kmin) {
        const long long twice_old = 1LL << (kTickBits - k_old + 1);
        if (t_new % twice_old == 0) return k_old - 1;
    }
    return k_old;
}

// Start-up step eta_init |a| / |k|; +infinity when the jerk vanishes.
__device__ __forceinline__ double initial_dt(const double a[3], const double k[3], double eta_init)
{
    const double nk = norm3(k[0], k[1], k[2]);
    return nk == 0.0 ? (double)INFINITY : __ddiv_rn(__dmul_rn(eta_init, norm3(a[0], a[1], a[2])), nk);
}

// Hermite corrector and Aarseth step for particle i of `s` (Section 2).  In
// the paper's notation a, k are the old values (in s) and a_p, k_p the new:
//   a3 = 2 (a - a_p) + (k + k_p) dt,   a2 = -3 (a - a_p) - (2 k + k_p) dt,
//   x = x_p + (a2/12 + a3/20) dt^2,    v = v_p + (a2/3 + a3/4) dt.
// Snap s0 = 2 a2 / dt^2, crackle c = 6 a3 / dt^3, s1 = s0 + c dt, and
//   dt_new = sqrt(eta (|a_p| |s1| + |k_p|^2) / (|k_p| |c| + |s1|^2)),
// quantised by level_of and next_level (level_fixed > 0 keeps that level).
// x_p, v_p are recomputed with predict1, bit for bit the values the force
// saw.  Returns false when the new step fell below 2^-40.
template <bool CG = false>
__device__ __forceinline__ bool correct_particle(const State &s, long long i, long long stride,
                                                 long long tn, const double ap[3], const double kp[3],
                                                 double eta, int level_min, int level_fixed)
{
    const double dt = ticks_to_time(tn - ldst<CG>(&s.t[i]));
    const double h = __dmul_rn(dt, 0.5), q = div_by<3>(dt);
    double a2[3], a3[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const long long e = c * stride + i;
        const double x = ldst<CG>(&s.x[e]), v = ldst<CG>(&s.v[e]), a = ldst<CG>(&s.a[e]),
                     k = ldst<CG>(&s.k[e]);
        double xp, vp;
        predict1hq(x, v, a, k, dt, h, q, xp, vp);
        const double d = __dsub_rn(a, ap[c]);
        a3[c] = __dadd_rn(__dmul_rn(2.0, d), __dmul_rn(__dadd_rn(k, kp[c]), dt));
        a2[c] = __dsub_rn(__dmul_rn(-3.0, d), __dmul_rn(__dadd_rn(__dmul_rn(2.0, k), kp[c]), dt));
        s.x[e] = __dadd_rn(xp, __dmul_rn(__dadd_rn(div_by<12>(a2[c]), div_by<20>(a3[c])),
                                         __dmul_rn(dt, dt)));
        // a3 / 4 as a3 * 0.25: the same real number, so the same rounded result
        s.v[e] = __dadd_rn(vp, __dmul_rn(__dadd_rn(div_by<3>(a2[c]), __dmul_rn(a3[c], 0.25)), dt));
        s.a[e] = ap[c];
        s.k[e] = kp[c];
    }
    s.t[i] = tn;
    if (level_fixed > 0) {
        s.lev[i] = level_fixed;
        return true;
    }
    const double dt2 = __dmul_rn(dt, dt);
    const double dt3 = __dmul_rn(dt2, dt);
    // A block step is a power of two: dividing by dt^2 and dt^3 is then the
    // same real number as multiplying by their exact reciprocals (powers of
    // two, from the exponent field), so the rounded results are identical and
    // four FP64 divisions per axis leave the latency chain.
    const bool pow2 = (__double_as_longlong(dt) & 0x000FFFFFFFFFFFFFLL) == 0 && dt > 0x1p-100;
    const double r2 = pow2 ? __longlong_as_double((2046LL << 52) - (__double_as_longlong(dt2) & 0x7FF0000000000000LL)) : 0.0;
    const double r3 = pow2 ? __longlong_as_double((2046LL << 52) - (__double_as_longlong(dt3) & 0x7FF0000000000000LL)) : 0.0;
    double s1[3], cr[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double s0;
        if (pow2) {
            s0 = __dmul_rn(__dmul_rn(2.0, a2[c]), r2);
            cr[c] = __dmul_rn(__dmul_rn(6.0, a3[c]), r3);
        } else {
            s0 = __ddiv_rn(__dmul_rn(2.0, a2[c]), dt2);
            cr[c] = __ddiv_rn(__dmul_rn(6.0, a3[c]), dt3);
        }
        s1[c] = __dadd_rn(s0, __dmul_rn(cr[c], dt));
    }
    const double na = norm3(ap[0], ap[1], ap[2]);
    const double nk = norm3(kp[0], kp[1], kp[2]);
    const double ns = norm3(s1[0], s1[1], s1[2]);
    const double nc = norm3(cr[0], cr[1], cr[2]);
    const double num = __dadd_rn(__dmul_rn(na, ns), __dmul_rn(nk, nk));
    const double den = __dadd_rn(__dmul_rn(nk, nc), __dmul_rn(ns, ns));
    const double dt_raw = den == 0.0 ? (double)INFINITY : __dsqrt_rn(__ddiv_rn(__dmul_rn(eta, num), den));
    int kq;
    const bool ok = level_of(dt_raw, level_min, kq);
    if (!ok) kq = kTickBits;
    s.lev[i] = next_level(ldst<CG>(&s.lev[i]), kq, tn, level_min);
    return ok;
}

// ---------------------------------------------------------------------------
// Single-precision mirror of the FP64 state, for j records predicted with FP32
// Taylor increments: position as double-single (x_hi + mass, x_lo), velocity,
// acceleration and jerk in FP32, as five float4 arrays of the particle count.
struct Mirror {
    float4 *h, *l, *v, *a, *k;
};

// The mirror of particle i from its FP64 state (component-major, stride n).
template <bool CG = false>
__device__ __forceinline__ void write_mirror(const State &s, const Mirror &mr, long long i, long long n)
{
    float hi[3], lo[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) split_ds(ldst<CG>(&s.x[c * n + i]), hi[c], lo[c]);
    mr.h[i] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(ldst<CG>(&s.m[i])));
    mr.l[i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
    mr.v[i] = make_float4(__double2float_rn(ldst<CG>(&s.v[i])), __double2float_rn(ldst<CG>(&s.v[n + i])),
                          __double2float_rn(ldst<CG>(&s.v[2 * n + i])), 0.0f);
    mr.a[i] = make_float4(__double2float_rn(ldst<CG>(&s.a[i])), __double2float_rn(ldst<CG>(&s.a[n + i])),
                          __double2float_rn(ldst<CG>(&s.a[2 * n + i])), 0.0f);
    mr.k[i] = make_float4(__double2float_rn(ldst<CG>(&s.k[i])), __double2float_rn(ldst<CG>(&s.k[n + i])),
                          __double2float_rn(ldst<CG>(&s.k[2 * n + i])), 0.0f);
}

// (hi, lo) + d in double-single: TwoSum of hi and d, then renormalised.
__device__ __forceinline__ void ds_add_f(float hi, float lo, float d, float &ho, float &lout)
{
    const float s = hi + d;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (d - bb);
    const float l2 = lo + e;
    ho = s + l2;
    lout = l2 - (ho - s);
}

// j record of particle i, dt ticks after its own time, from the mirror: the
// predictor's Taylor increments (Section 2) in FP32,
//   dx = (v + (dt/2)(a + (dt/3) k)) dt,   v_p = v + (a + (dt/2) k) dt,
// and the position accumulated in double-single, x_p = (x_hi + x_lo) + dx.
template <bool CG = false>
__device__ __forceinline__ void predict_j32(const Mirror &mr, long long i, long long dt_ticks,
                                            float4 &ph, float4 &pl, float4 &pv)
{
    const float dt = (float)dt_ticks * 0x1p-40f;
    const float h = 0.5f * dt, q = dt * (1.0f / 3.0f);
    const float4 xh = ldst<CG>(&mr.h[i]), xl = ldst<CG>(&mr.l[i]), v = ldst<CG>(&mr.v[i]),
                 a = ldst<CG>(&mr.a[i]), k = ldst<CG>(&mr.k[i]);
    ds_add_f(xh.x, xl.x, fmaf(h, fmaf(q, k.x, a.x), v.x) * dt, ph.x, pl.x);
    ds_add_f(xh.y, xl.y, fmaf(h, fmaf(q, k.y, a.y), v.y) * dt, ph.y, pl.y);
    ds_add_f(xh.z, xl.z, fmaf(h, fmaf(q, k.z, a.z), v.z) * dt, ph.z, pl.z);
    pv.x = fmaf(fmaf(h, k.x, a.x), dt, v.x);
    pv.y = fmaf(fmaf(h, k.y, a.y), dt, v.y);
    pv.z = fmaf(fmaf(h, k.z, a.z), dt, v.z);
    ph.w = xh.w;
    pl.w = 0.0f;
    pv.w = 0.0f;
}

// correct_particle spread over the four lanes of a quad (lanes 4u .. 4u+3 of
// a warp), for blocks too small to fill the GPU: the corrector is a chain of
// FP64 operations, and on the GB300 an FP64 warp instruction occupies the SM's
// narrow FP64 pipe for many cycles however few of its lanes are active, so
// one particle's three axes on three lanes (and its four norms on four)
// issue about half the FP64 instructions of the one-thread form.  Each lane
// evaluates exactly the operations of correct_particle for its axis, in the
// same order, so the results are the same bits.
//
// Every lane of the warp must call this together (it shuffles over the whole
// warp).  Lane q = lane & 3 of a quad passes component q of the new
// acceleration and jerk (lane 3: any finite value, e.g. that of axis 2) and
// the same particle i as its quad; `active` false (the whole quad) computes
// on a valid i without storing.  Returns false (on every lane of an active
// quad) when the new step fell below 2^-40.
template <bool CG = false>
__device__ __forceinline__ bool correct_particle_quad(const State &s, long long i, long long stride,
                                                      long long tn, double apc, double kpc,
                                                      double eta, int level_min, int level_fixed,
                                                      bool active)
{
    const int lane = threadIdx.x & 31, q = lane & 3, base = lane & ~3;
    const int c = q < 3 ? q : 2;          // lane 3 shadows axis 2 without storing
    const bool own = active && q < 3;
    const double dt = ticks_to_time(tn - ldst<CG>(&s.t[i]));
    const double h = __dmul_rn(dt, 0.5), q3 = div_by<3>(dt);
    const long long e = c * stride + i;
    const double x = ldst<CG>(&s.x[e]), v = ldst<CG>(&s.v[e]), a = ldst<CG>(&s.a[e]),
                 k = ldst<CG>(&s.k[e]);
    const int lev_old = ldst<CG>(&s.lev[i]);
    double xp, vp;
    predict1hq(x, v, a, k, dt, h, q3, xp, vp);
    const double d = __dsub_rn(a, apc);
    const double a3 = __dadd_rn(__dmul_rn(2.0, d), __dmul_rn(__dadd_rn(k, kpc), dt));
    const double a2 = __dsub_rn(__dmul_rn(-3.0, d), __dmul_rn(__dadd_rn(__dmul_rn(2.0, k), kpc), dt));
    const double xn = __dadd_rn(xp, __dmul_rn(__dadd_rn(div_by<12>(a2), div_by<20>(a3)),
                                            __dmul_rn(dt, dt)));
    const double vn = __dadd_rn(vp, __dmul_rn(__dadd_rn(div_by<3>(a2), __dmul_rn(a3, 0.25)), dt));
    // every lane of the quad has read the old state before any lane stores
    __syncwarp();
    if (own) {
        s.x[e] = xn;
        s.v[e] = vn;
        s.a[e] = apc;
        s.k[e] = kpc;
    }
    if (level_fixed > 0) {
        if (active && q == 0) {
            s.t[i] = tn;
            s.lev[i] = level_fixed;
        }
        return true;
    }
    const double dt2 = __dmul_rn(dt, dt);
    const double dt3 = __dmul_rn(dt2, dt);
    const bool pow2 = (__double_as_longlong(dt) & 0x000FFFFFFFFFFFFFLL) == 0 && dt > 0x1p-100;
    const double r2 = pow2 ? __longlong_as_double((2046LL << 52) - (__double_as_longlong(dt2) & 0x7FF0000000000000LL)) : 0.0;
    const double r3 = pow2 ? __longlong_as_double((2046LL << 52) - (__double_as_longlong(dt3) & 0x7FF0000000000000LL)) : 0.0;
    double s0, cr;
    if (pow2) {
        s0 = __dmul_rn(__dmul_rn(2.0, a2), r2);
        cr = __dmul_rn(__dmul_rn(6.0, a3), r3);
    } else {
        s0 = __ddiv_rn(__dmul_rn(2.0, a2), dt2);
        cr = __ddiv_rn(__dmul_rn(6.0, a3), dt3);
    }
    const double s1 = __dadd_rn(s0, __dmul_rn(cr, dt));
    // |a_p|, |k_p|, |s1|, |c| on lanes 0..3 of the quad, each as norm3 forms it
    const double sq0 = __dmul_rn(apc, apc), sq1 = __dmul_rn(kpc, kpc);
    const double sq2 = __dmul_rn(s1, s1), sq3 = __dmul_rn(cr, cr);
    double w[3];
#pragma unroll
    for (int cc = 0; cc < 3; ++cc) {
        const double t0 = __shfl_sync(0xffffffffu, sq0, base + cc);
        const double t1 = __shfl_sync(0xffffffffu, sq1, base + cc);
        const double t2 = __shfl_sync(0xffffffffu, sq2, base + cc);
        const double t3 = __shfl_sync(0xffffffffu, sq3, base + cc);
        w[cc] = q == 0 ? t0 : (q == 1 ? t1 : (q == 2 ? t2 : t3));
    }
    const double nrm = __dsqrt_rn(__dadd_rn(__dadd_rn(w[0], w[1]), w[2]));
    const double na = __shfl_sync(0xffffffffu, nrm, base + 0);
    const double nk = __shfl_sync(0xffffffffu, nrm, base + 1);
    const double ns = __shfl_sync(0xffffffffu, nrm, base + 2);
    const double nc = __shfl_sync(0xffffffffu, nrm, base + 3);
    const double num = __dadd_rn(__dmul_rn(na, ns), __dmul_rn(nk, nk));
    const double den = __dadd_rn(__dmul_rn(nk, nc), __dmul_rn(ns, ns));
    const double dt_raw = den == 0.0 ? (double)INFINITY : __dsqrt_rn(__ddiv_rn(__dmul_rn(eta, num), den));
    int kq;
    const bool ok = level_of(dt_raw, level_min, kq);
    if (!ok) kq = kTickBits;
    if (active && q == 0) {
        s.t[i] = tn;
        s.lev[i] = next_level(lev_old, kq, tn, level_min);
    }
    return ok;
}

// FP32 pair terms of Eq. 1 (attractive sign; pair terms of the Appendix A
// kernel) from the separation dx = x_j - x_i and the velocity difference
// u = v_j - v_i.  SOFT = false drops pairs at r = 0; GUARD drops the pair
// j == i.
template <bool SOFT, bool GUARD>
__device__ __forceinline__ void pair_terms(float dx, float dy, float dz, float ux, float uy, float uz,
                                           float m, float eps2, float acc[3], float jk[3], float &pot,
                                           int j, int i)
{
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    const float rv = fmaf(dx, ux, fmaf(dy, uy, dz * uz));
    float rinv = rsqrt_sfu(r2);
    if (!SOFT) rinv = (r2 > 0.0f) ? rinv : 0.0f;
    if (GUARD) rinv = (j == i) ? 0.0f : rinv;
    const float rinv2 = rinv * rinv;
    const float mr = m * rinv;             // m_j / r
    const float mr3 = mr * rinv2;          // m_j / r^3
    const float b = -3.0f * rv * rinv2;    // -3 (dx . dv) / r^2
    acc[0] = fmaf(mr3, dx, acc[0]);
    acc[1] = fmaf(mr3, dy, acc[1]);
    acc[2] = fmaf(mr3, dz, acc[2]);
    const float qx = fmaf(b, dx, ux);
    const float qy = fmaf(b, dy, uy);
    const float qz = fmaf(b, dz, uz);
    jk[0] = fmaf(mr3, qx, jk[0]);
    jk[1] = fmaf(mr3, qy, jk[1]);
    jk[2] = fmaf(mr3, qz, jk[2]);
    pot -= mr;
}

// One FP32 pair interaction on double-single positions, dx = x_j - x_i formed
// as (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo).
template <bool SOFT, bool GUARD>
__device__ __forceinline__ void pair_ds(const float4 &p, const float4 &l, const float4 &w,
                                        const float xh[3], const float xl[3], const float vi[3],
                                        float eps2, float acc[3], float jk[3], float &pot,
                                        int j = 0, int i = 1)
{
    const float dx = (p.x - xh[0]) + (l.x - xl[0]);
    const float dy = (p.y - xh[1]) + (l.y - xl[1]);
    const float dz = (p.z - xh[2]) + (l.z - xl[2]);
    pair_terms<SOFT, GUARD>(dx, dy, dz, w.x - vi[0], w.y - vi[1], w.z - vi[2], p.w, eps2, acc, jk, pot,
                            j, i);
}

// The i side of a pair in the packed form below: the x and y components
// negated and paired, z kept as it is.
struct IDS {
    float2 nh, nl, nv;   // (-x_hi, -y_hi), (-x_lo, -y_lo), (-v_x, -v_y)
    float zh, zl, vz;
};

__device__ __forceinline__ IDS make_ids(const float4 &p, const float4 &l, const float4 &v)
{
    IDS I;
    I.nh = make_float2(-p.x, -p.y);
    I.nl = make_float2(-l.x, -l.y);
    I.nv = make_float2(-v.x, -v.y);
    I.zh = p.z; I.zl = l.z; I.vz = v.z;
    return I;
}

// pair_ds with the x and y components of the three differences taken by
// packed two-lane FP32 adds (add.f32x2): four instructions instead of eight,
// each lane rounded exactly as the scalar subtraction it replaces
// (RN(a + (-b)) = RN(a - b)), so the result is bit for bit that of pair_ds.
// The FMA pipe does the same work; the saving is issue slots.
template <bool SOFT, bool GUARD>
__device__ __forceinline__ void pair_ds_packed(const float4 &p, const float4 &l, const float4 &w,
                                               const IDS &I, float eps2, float acc[3], float jk[3],
                                               float &pot, int j = 0, int i = 1)
{
    const float2 dh = __fadd2_rn(make_float2(p.x, p.y), I.nh);
    const float2 dl = __fadd2_rn(make_float2(l.x, l.y), I.nl);
    const float2 d = __fadd2_rn(dh, dl);
    const float2 u = __fadd2_rn(make_float2(w.x, w.y), I.nv);
    const float dz = (p.z - I.zh) + (l.z - I.zl);
    pair_terms<SOFT, GUARD>(d.x, d.y, dz, u.x, u.y, w.z - I.vz, p.w, eps2, acc, jk, pot, j, i);
}

// Block size of a force launch: read on the device when the host does not know it.
__device__ __forceinline__ int read_na(const ForceArgs &fa)
{
    return fa.na_dev ? *fa.na_dev : fa.na_host;
}

// Index loads of padding lanes are clamped into [0, n).
__device__ __forceinline__ int clamp_index(int i, int n) { return min(max(i, 0), n - 1); }

// One particle's acc, jerk, pot into the public output layout.
__device__ __forceinline__ void store_result(const ForceOut &o, int a, const double r[kComp])
{
    if (o.acc) {
        o.acc[3 * (long long)a + 0] = r[0];
        o.acc[3 * (long long)a + 1] = r[1];
        o.acc[3 * (long long)a + 2] = r[2];
    }
    if (o.jerk) {
        o.jerk[3 * (long long)a + 0] = r[3];
        o.jerk[3 * (long long)a + 1] = r[4];
        o.jerk[3 * (long long)a + 2] = r[5];
    }
    if (o.pot) o.pot[a] = r[6];
}

// Component c (0-2 acc, 3-5 jerk, 6 pot) of output a.
__device__ __forceinline__ void write_combined(const ForceOut &o, int c, int a, double s)
{
    if (c < 3) {
        if (o.acc) o.acc[3 * (long long)a + c] = s;
    } else if (c < 6) {
        if (o.jerk) o.jerk[3 * (long long)a + (c - 3)] = s;
    } else if (o.pot) {
        o.pot[a] = s;
    }
}

// ---------------------------------------------------------------------------
// Summation variants (Section 6): single-precision pair terms with IEEE
// round-to-nearest operations in a fixed order, and the exact integer
// arithmetic of the GRAPE-style fixed-point sums.

// The seven single-precision terms of j on i, each scaled as stated above;
// false when r2 = 0 (the terms are then not numbers and must be skipped).
__device__ __forceinline__ bool pair_rn(const float4 &p, const float4 &l, const float4 &w,
                                        const float xh[3], const float xl[3], const float vi[3],
                                        float eps2, float sa, float sk, float sp, float t[7],
                                        float *key = nullptr)
{
    const float dx0 = __fadd_rn(__fsub_rn(p.x, xh[0]), __fsub_rn(l.x, xl[0]));
    const float dx1 = __fadd_rn(__fsub_rn(p.y, xh[1]), __fsub_rn(l.y, xl[1]));
    const float dx2 = __fadd_rn(__fsub_rn(p.z, xh[2]), __fsub_rn(l.z, xl[2]));
    const float u0 = __fsub_rn(w.x, vi[0]);
    const float u1 = __fsub_rn(w.y, vi[1]);
    const float u2 = __fsub_rn(w.z, vi[2]);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx0, dx0), __fmul_rn(dx1, dx1)), __fmul_rn(dx2, dx2));
    const float r2 = __fadd_rn(d2, eps2);
    const float rv = __fadd_rn(__fadd_rn(__fmul_rn(dx0, u0), __fmul_rn(dx1, u1)), __fmul_rn(dx2, u2));
    const float rinv = __frcp_rn(__fsqrt_rn(r2));
    const float rinv2 = __fmul_rn(rinv, rinv);
    const float mr = __fmul_rn(p.w, rinv);
    const float mr3 = __fmul_rn(mr, rinv2);
    const float b = __fmul_rn(__fmul_rn(-3.0f, rv), rinv2);
    const float fa = __fmul_rn(mr3, sa), fk = __fmul_rn(mr3, sk), fp = __fmul_rn(mr, sp);
    t[0] = __fmul_rn(fa, dx0);
    t[1] = __fmul_rn(fa, dx1);
    t[2] = __fmul_rn(fa, dx2);
    t[3] = __fmul_rn(fk, __fadd_rn(u0, __fmul_rn(b, dx0)));
    t[4] = __fmul_rn(fk, __fadd_rn(u1, __fmul_rn(b, dx1)));
    t[5] = __fmul_rn(fk, __fadd_rn(u2, __fmul_rn(b, dx2)));
    t[6] = -fp;
    if (key) *key = fminf(__fmul_rn(mr3, __fsqrt_rn(d2)), FLT_MAX);
    return r2 != 0.0f;
}

__device__ __forceinline__ void load_i(const JDS &J, int i, float xh[3], float xl[3], float vi[3])
{
    const float4 p = J.pos_hi[i], l = J.pos_lo[i], v = J.vel[i];
    xh[0] = p.x; xh[1] = p.y; xh[2] = p.z;
    xl[0] = l.x; xl[1] = l.y; xl[2] = l.z;
    vi[0] = v.x; vi[1] = v.y; vi[2] = v.z;
}

// ---------------------------------------------------------------------------
// Fixed point

struct Scale {
    float sc[3];    // 2^s: acc, jerk, pot
    double inv[3];  // 2^-s
};

__device__ __forceinline__ int exp_above(unsigned bits)
{
    const int be = (int)((bits >> 23) & 0xFF);
    return be == 0 ? -126 : be - 126;
}

__device__ __forceinline__ int floor_half(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

// Scales from the bounds.  With eps2 >= 2^F, every mass < 2^Em and every
// |vx| + |vy| + |vz| < 2^Ev (Em, Ev at least -64), the terms obey
//   |acc| <= mj / r^2 < 2^(Em - F),   |pot| = mj / r < 2^(Em - floor(F/2)),
//   |jerk| <= 4 mj |dv| / r^3 < 2^(3 + Em + Ev - floor(3F/2))
// up to single-precision rounding, which the factor 2 between 2^56 and 2^57
// absorbs; s = min(56 - e, 126).  False when eps2 is not a normal float or a
// scale falls below -126.
__device__ __forceinline__ bool fixed_scale(const unsigned *bounds, float eps2, Scale &S)
{
    const int be = (int)((__float_as_uint(eps2) >> 23) & 0xFF);
    if (be == 0 || be == 255) return false;
    const int F = be - 127;
    const int Em = max(exp_above(bounds[0]), -64), Ev = max(exp_above(bounds[1]), -64);
    const int e[3] = {Em - F, 3 + Em + Ev - floor_half(3 * F), Em - floor_half(F)};
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const int s = min(56 - e[q], 126);
        if (s < -126) return false;
        S.sc[q] = __int_as_float((s + 127) << 23);
        S.inv[q] = __longlong_as_double((long long)(1023 - s) << 52);
    }
    return true;
}

// Exact integer rounding of a term |t| < 2^57 - 2^34 on the FP32 pipe.  For
// C = 1.5 * 2^(23+g), s = fl(t + C) stays in C's binade while |t| < 2^(22+g),
// so s - C is t rounded to a multiple of 2^g and bits(s) - bits(C) is that
// multiple's count.  With g = 35, 13 and 0:
//   s1 = fl(t + C1),  r  = t - (s1 - C1)      |r|  <= 2^34, exact
//   s2 = fl(r + C2),  r2 = r - (s2 - C2)      |r2| <= 2^12, exact
//   s3 = fl(r2 + C3)                          r2 rounded half to even
// and round_half_even(t) = a1 2^35 + a2 2^13 + a3 with a_k = bits(s_k) -
// bits(C_k) (the first two parts are even, so the tie rule carries over).  A
// tile adds the raw bit patterns in 32 bits (mod 2^32) and subtracts the
// constants once: the true sums stay below 2^28 in magnitude.
constexpr float kC1 = 0x1.8p58f, kC2 = 0x1.8p36f, kC3 = 0x1.8p23f;

__device__ __forceinline__ void split_add(float t, unsigned &a1, unsigned &a2, unsigned &a3)
{
    const float s1 = __fadd_rn(t, kC1);
    const float r = __fsub_rn(t, __fsub_rn(s1, kC1));
    const float s2 = __fadd_rn(r, kC2);
    const float r2 = __fsub_rn(r, __fsub_rn(s2, kC2));
    const float s3 = __fadd_rn(r2, kC3);
    a1 += __float_as_uint(s1);
    a2 += __float_as_uint(s2);
    a3 += __float_as_uint(s3);
}

// The integer sum of a tile of `cnt` split terms.
__device__ __forceinline__ long long tile_sum(unsigned a1, unsigned a2, unsigned a3, unsigned cnt)
{
    const int q1 = (int)(a1 - cnt * __float_as_uint(kC1));
    const int q2 = (int)(a2 - cnt * __float_as_uint(kC2));
    const int q3 = (int)(a3 - cnt * __float_as_uint(kC3));
    return ((long long)q1 << 35) + ((long long)q2 << 13) + (long long)q3;
}

// (hi, lo) += x, a 128-bit two's-complement sum.
__device__ __forceinline__ void add128(long long &hi, unsigned long long &lo, long long x)
{
    const unsigned long long l2 = lo + (unsigned long long)x;
    hi += (x >> 63) + (l2 < lo ? 1 : 0);
    lo = l2;
}

// |Y| = H 2^64 + L  ->  fl64(fl64(H) 2^64 + fl64(L)), with Y's sign.
__device__ __forceinline__ double i128_to_double(long long hi, unsigned long long lo)
{
    const bool neg = hi < 0;
    if (neg) {
        lo = ~lo + 1ULL;
        hi = ~hi + (lo == 0ULL ? 1 : 0);
    }
    const double d = __dadd_rn(__dmul_rn(__ull2double_rn((unsigned long long)hi), 0x1p64),
                               __ull2double_rn(lo));
    return neg ? -d : d;
}

}  // namespace dev
}  // namespace nbk
