// k_adjoint.cu -- reverse-mode kernels: the vector-Jacobian product of the
// direct-summation force, and the transposes of the (linear) Hermite
// corrector and predictor for a fixed shared time step.  The paper has no
// gradients; these extend its method to a differentiable trajectory.
//
// Force VJP.  For every ordered pair (i, j), j != i, with d = x_j - x_i,
// w = v_j - v_i, r^2 = |d|^2 + eps^2, s = d.w and cotangents (abar_i, kbar_i)
// on acc_i and jerk_i, the derivatives of abar_i.acc_i + kbar_i.jerk_i are
//   g_d(abar, kbar) = m_j [ abar/r^3 - 3 (s kbar + (kbar.d) w)/r^5
//                           + (-3 (abar.d + kbar.w)/r^5 + 15 s (kbar.d)/r^7) d ]
//   g_w(kbar)       = m_j [ kbar/r^3 - 3 (kbar.d) d/r^5 ]
//   g_m             = abar.d/r^3 + kbar.(w/r^3 - 3 s d/r^5)        (w.r.t. m_j)
// with xbar_j += g_d, xbar_i -= g_d, vbar_j += g_w, vbar_i -= g_w.  Both g_d
// and g_w are even in (d, w) and linear in (abar, kbar), so for particle k
// the contributions as i (partner p as j, weight m_p) and as j (partner p as
// i, weight m_k) fold into one evaluation with
//   A = m_k abar_p - m_p abar_k,   K = m_k kbar_p - m_p kbar_k:
//   xbar_k += G(A, K),   vbar_k += H(K),
//   mbar_k += -(abar_p.d + kbar_p.w)/r^3 + 3 s (kbar_p.d)/r^5,
// with d = x_p - x_k.  One k-parallel sweep, no atomics; each thread owns
// kVKR particles k (one in the FP64 twin) and streams the partners through
// shared memory in tiles, like the forward i-parallel kernel (double-single
// positions, FP32 pair arithmetic, TwoSum-promoted tile partials).
#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

constexpr int kVNT = 128;  // threads per CTA = partners per tile
#ifndef NB_VJP_R
#define NB_VJP_R 2
#endif
#ifndef NB_VJP_UNROLL
#define NB_VJP_UNROLL 4
#endif
constexpr int kVKR = NB_VJP_R;          // DS: particles k per thread
constexpr int kVUnroll = NB_VJP_UNROLL; // DS: partner unrolling

// One particle's VJP record: (predicted) position and velocity, mass and the
// cotangents of its acc and jerk, in the layout of the context's precision.
__device__ __forceinline__ void write_vjp_record(int i, const double x[3], const double v[3], double m,
                                 const double ab[3], const double kb[3], int precision,
                                 VjpRecDS rec, VjpRec64 rec64)
{
    if (precision == NB_FP64) {
        rec64.x[i] = make_double4_32a(x[0], x[1], x[2], m);
        rec64.v[i] = make_double4_32a(v[0], v[1], v[2], 0.0);
        rec64.ab[i] = make_double4_32a(ab[0], ab[1], ab[2], 0.0);
        rec64.kb[i] = make_double4_32a(kb[0], kb[1], kb[2], 0.0);
    } else {
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) split_ds(x[c], hi[c], lo[c]);
        rec.ph[i] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(m));
        rec.pl[i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        rec.v[i] = make_float4(__double2float_rn(v[0]), __double2float_rn(v[1]),
                               __double2float_rn(v[2]), 0.0f);
        rec.ab[i] = make_float4(__double2float_rn(ab[0]), __double2float_rn(ab[1]),
                                __double2float_rn(ab[2]), 0.0f);
        rec.kb[i] = make_float4(__double2float_rn(kb[0]), __double2float_rn(kb[1]),
                                __double2float_rn(kb[2]), 0.0f);
    }
}


// One (k, p) pair in FP32 on double-single positions; acc[0..2] xbar,
// acc[3..5] vbar, acc[6] mbar.
template <bool SOFT, bool GUARD>
__device__ __forceinline__ void vjp_pair_ds(const VjpRec &P, const VjpRec &Kp, float eps2,
                                            float acc[7], int p = 0, int k = 1)
{
    const float dx = (P.ph.x - Kp.ph.x) + (P.pl.x - Kp.pl.x);
    const float dy = (P.ph.y - Kp.ph.y) + (P.pl.y - Kp.pl.y);
    const float dz = (P.ph.z - Kp.ph.z) + (P.pl.z - Kp.pl.z);
    const float wx = P.v.x - Kp.v.x, wy = P.v.y - Kp.v.y, wz = P.v.z - Kp.v.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
    float rinv = rsqrt_sfu(r2);
    if (!SOFT) rinv = (r2 > 0.0f) ? rinv : 0.0f;
    if (GUARD) rinv = (p == k) ? 0.0f : rinv;
    const float rinv2 = rinv * rinv;
    const float r3 = rinv * rinv2;
    const float r5 = r3 * rinv2;
    const float r7 = r5 * rinv2;
    const float s = fmaf(dx, wx, fmaf(dy, wy, dz * wz));
    const float mk = Kp.ph.w, mp = P.ph.w;
    const float Ax = fmaf(mk, P.ab.x, -mp * Kp.ab.x);
    const float Ay = fmaf(mk, P.ab.y, -mp * Kp.ab.y);
    const float Az = fmaf(mk, P.ab.z, -mp * Kp.ab.z);
    const float Kx = fmaf(mk, P.kb.x, -mp * Kp.kb.x);
    const float Ky = fmaf(mk, P.kb.y, -mp * Kp.kb.y);
    const float Kz = fmaf(mk, P.kb.z, -mp * Kp.kb.z);
    const float Ad = fmaf(Ax, dx, fmaf(Ay, dy, Az * dz));
    const float Kd = fmaf(Kx, dx, fmaf(Ky, dy, Kz * dz));
    const float Kw = fmaf(Kx, wx, fmaf(Ky, wy, Kz * wz));
    const float t5 = -3.0f * r5;
    const float cd = fmaf(t5, Ad + Kw, 15.0f * s * Kd * r7);   // coefficient of d in G
    const float cs = t5 * s;                                    // coefficient of K in G
    const float cw = t5 * Kd;                                   // coefficient of w in G, of d in H
    acc[0] += fmaf(r3, Ax, fmaf(cs, Kx, fmaf(cw, wx, cd * dx)));
    acc[1] += fmaf(r3, Ay, fmaf(cs, Ky, fmaf(cw, wy, cd * dy)));
    acc[2] += fmaf(r3, Az, fmaf(cs, Kz, fmaf(cw, wz, cd * dz)));
    acc[3] += fmaf(r3, Kx, cw * dx);
    acc[4] += fmaf(r3, Ky, cw * dy);
    acc[5] += fmaf(r3, Kz, cw * dz);
    const float apd = fmaf(P.ab.x, dx, fmaf(P.ab.y, dy, P.ab.z * dz));
    const float kpw = fmaf(P.kb.x, wx, fmaf(P.kb.y, wy, P.kb.z * wz));
    const float kpd = fmaf(P.kb.x, dx, fmaf(P.kb.y, dy, P.kb.z * dz));
    acc[6] += fmaf(-r3, apd + kpw, 3.0f * s * kpd * r5);
}

template <bool SOFT>
__global__ void __launch_bounds__(kVNT) k_force_vjp_ds(VjpArgs va)
{
    constexpr int R = kVKR;
    const Plan P = va.plan;
    __shared__ float4 s_ph[kVNT], s_pl[kVNT], s_v[kVNT], s_ab[kVNT], s_kb[kVNT];
    const float eps2 = (float)va.eps2;
    const int tid = threadIdx.x;
    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        const int ib = w % P.n_iblk, sl = w / P.n_iblk;
        const int j0 = sl * P.jslice;
        const int j1 = min(va.n, j0 + P.jslice);
        int kk[R], k[R];
        VjpRec K[R];
        float hi[R][7], lo[R][7];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            kk[r] = ib * kVNT * R + r * kVNT + tid;
            k[r] = clamp_index(kk[r], va.n);
            K[r].ph = va.rec.ph[k[r]]; K[r].pl = va.rec.pl[k[r]]; K[r].v = va.rec.v[k[r]];
            K[r].ab = va.rec.ab[k[r]]; K[r].kb = va.rec.kb[k[r]];
#pragma unroll
            for (int c = 0; c < 7; ++c) hi[r][c] = lo[r][c] = 0.0f;
        }
        for (int jt = j0; jt < j1; jt += kVNT) {
            __syncthreads();
            const int j = jt + tid;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            s_ph[tid] = j < j1 ? va.rec.ph[j] : z;
            s_pl[tid] = j < j1 ? va.rec.pl[j] : z;
            s_v[tid] = j < j1 ? va.rec.v[j] : z;
            s_ab[tid] = j < j1 ? va.rec.ab[j] : z;
            s_kb[tid] = j < j1 ? va.rec.kb[j] : z;
            __syncthreads();
            float t[R][7];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < 7; ++c) t[r][c] = 0.0f;
            bool mine = false;
#pragma unroll
            for (int r = 0; r < R; ++r) mine |= (unsigned)(k[r] - jt) < (unsigned)kVNT;
            if (__any_sync(0xffffffffu, mine)) {
                for (int jj = 0; jj < kVNT; ++jj) {
                    VjpRec Pq;
                    Pq.ph = s_ph[jj]; Pq.pl = s_pl[jj]; Pq.v = s_v[jj]; Pq.ab = s_ab[jj]; Pq.kb = s_kb[jj];
#pragma unroll
                    for (int r = 0; r < R; ++r) vjp_pair_ds<SOFT, true>(Pq, K[r], eps2, t[r], jt + jj, k[r]);
                }
            } else {
#pragma unroll (kVUnroll)
                for (int jj = 0; jj < kVNT; ++jj) {
                    VjpRec Pq;
                    Pq.ph = s_ph[jj]; Pq.pl = s_pl[jj]; Pq.v = s_v[jj]; Pq.ab = s_ab[jj]; Pq.kb = s_kb[jj];
#pragma unroll
                    for (int r = 0; r < R; ++r) vjp_pair_ds<SOFT, false>(Pq, K[r], eps2, t[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int c = 0; c < 7; ++c) two_sum_acc(hi[r][c], lo[r][c], t[r][c]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (kk[r] >= va.n) continue;
            double res[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) res[c] = (double)hi[r][c] + (double)lo[r][c];
            if (P.S == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    va.xbar[3 * (long long)k[r] + c] = res[c];
                    va.vbar[3 * (long long)k[r] + c] = res[3 + c];
                }
                va.mbar[k[r]] = res[6];
            } else {
#pragma unroll
                for (int c = 0; c < 7; ++c) va.part[((long long)sl * 7 + c) * va.n + k[r]] = res[c];
            }
        }
    }
}

// FP64 twin, one k per thread, partners through shared memory.
template <bool SOFT>
__global__ void __launch_bounds__(kVNT) k_force_vjp_f64(VjpArgs va)
{
    const Plan P = va.plan;
    __shared__ double4_32a s_x[kVNT], s_v[kVNT], s_a[kVNT], s_k[kVNT];
    const double eps2 = va.eps2;
    const int tid = threadIdx.x;
    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        const int ib = w % P.n_iblk, sl = w / P.n_iblk;
        const int j0 = sl * P.jslice;
        const int j1 = min(va.n, j0 + P.jslice);
        const int kk = ib * kVNT + tid;
        const int k = clamp_index(kk, va.n);
        const double4_32a Xk = va.rec64.x[k], Vk = va.rec64.v[k], Ak = va.rec64.ab[k],
                          Kk = va.rec64.kb[k];
        double acc[7] = {0., 0., 0., 0., 0., 0., 0.};
        for (int jt = j0; jt < j1; jt += kVNT) {
            __syncthreads();
            const int j = jt + tid;
            const double4_32a z = make_double4_32a(0., 0., 0., 0.);
            s_x[tid] = j < j1 ? va.rec64.x[j] : z;
            s_v[tid] = j < j1 ? va.rec64.v[j] : z;
            s_a[tid] = j < j1 ? va.rec64.ab[j] : z;
            s_k[tid] = j < j1 ? va.rec64.kb[j] : z;
            __syncthreads();
            for (int jj = 0; jj < kVNT; ++jj) {
                const double4_32a Xp = s_x[jj], Vp = s_v[jj], Ap = s_a[jj], Kp = s_k[jj];
                const double dx = Xp.x - Xk.x, dy = Xp.y - Xk.y, dz = Xp.z - Xk.z;
                const double wx = Vp.x - Vk.x, wy = Vp.y - Vk.y, wz = Vp.z - Vk.z;
                const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
                double rinv = rsqrt(r2);
                if (!SOFT) rinv = (r2 > 0.0) ? rinv : 0.0;
                rinv = (jt + jj == k) ? 0.0 : rinv;
                const double rinv2 = rinv * rinv, r3 = rinv * rinv2, r5 = r3 * rinv2, r7 = r5 * rinv2;
                const double s = fma(dx, wx, fma(dy, wy, dz * wz));
                const double mk = Xk.w, mp = Xp.w;
                const double Ax = mk * Ap.x - mp * Ak.x, Ay = mk * Ap.y - mp * Ak.y, Az = mk * Ap.z - mp * Ak.z;
                const double Kx = mk * Kp.x - mp * Kk.x, Ky = mk * Kp.y - mp * Kk.y, Kz = mk * Kp.z - mp * Kk.z;
                const double Ad = Ax * dx + Ay * dy + Az * dz;
                const double Kd = Kx * dx + Ky * dy + Kz * dz;
                const double Kw = Kx * wx + Ky * wy + Kz * wz;
                const double cd = -3.0 * r5 * (Ad + Kw) + 15.0 * s * Kd * r7;
                const double cs = -3.0 * r5 * s, cw = -3.0 * r5 * Kd;
                acc[0] += r3 * Ax + cs * Kx + cw * wx + cd * dx;
                acc[1] += r3 * Ay + cs * Ky + cw * wy + cd * dy;
                acc[2] += r3 * Az + cs * Kz + cw * wz + cd * dz;
                acc[3] += r3 * Kx + cw * dx;
                acc[4] += r3 * Ky + cw * dy;
                acc[5] += r3 * Kz + cw * dz;
                const double apd = Ap.x * dx + Ap.y * dy + Ap.z * dz;
                const double kpw = Kp.x * wx + Kp.y * wy + Kp.z * wz;
                const double kpd = Kp.x * dx + Kp.y * dy + Kp.z * dz;
                acc[6] += -r3 * (apd + kpw) + 3.0 * s * kpd * r5;
            }
        }
        if (kk < va.n) {
            if (P.S == 1) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    va.xbar[3 * (long long)k + c] = acc[c];
                    va.vbar[3 * (long long)k + c] = acc[3 + c];
                }
                va.mbar[k] = acc[6];
            } else {
#pragma unroll
                for (int c = 0; c < 7; ++c) va.part[((long long)sl * 7 + c) * va.n + k] = acc[c];
            }
        }
    }
}

__global__ void k_vjp_combine(VjpArgs va, int S)
{
    const long long total = 7LL * va.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / va.n), k = (int)(e % va.n);
        double s = 0.0;
        for (int q = 0; q < S; ++q) s += va.part[((long long)q * 7 + c) * va.n + k];
        if (c < 3) va.xbar[3 * (long long)k + c] = s;
        else if (c < 6) va.vbar[3 * (long long)k + (c - 3)] = s;
        else va.mbar[k] = s;
    }
}

// Backward step, first half: from the cotangents (xb, vb, ab, kb) of the state
// after a step that started at `st`, the cotangents of the new acc and jerk
// (through the corrector's D = a - a1, a3 and a2, and the new state's own
// acc and jerk) go into the force-VJP records, together with the predicted
// positions and velocities of the step; ab, kb become the corrector's part of
// the old acc and jerk cotangents.
//   a2b = xb dt^2/12 + vb dt/3,  a3b = xb dt^2/20 + vb dt/4,  Db = 2 a3b - 3 a2b
//   a1b = ab - Db,  k1b = kb + (a3b - a2b) dt,  ab <- Db,  kb <- (a3b - 2 a2b) dt
__global__ void k_adj_pre(State st, double dt, const double *xb, const double *vb, double *ab,
                          double *kb, int precision, VjpRecDS rec, VjpRec64 rec64)
{
    const int n = st.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double xp[3], vp[3], a1b[3], k1b[3];
        predict3(st, i, n, dt, xp, vp);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long q = 3LL * i + c;
            const double a2b = xb[q] * dt * dt / 12.0 + vb[q] * dt / 3.0;
            const double a3b = xb[q] * dt * dt / 20.0 + vb[q] * dt / 4.0;
            const double Db = 2.0 * a3b - 3.0 * a2b;
            a1b[c] = ab[q] - Db;
            k1b[c] = kb[q] + (a3b - a2b) * dt;
            ab[q] = Db;
            kb[q] = (a3b - 2.0 * a2b) * dt;
        }
        write_vjp_record(i, xp, vp, st.m[i], a1b, k1b, precision, rec, rec64);
    }
}

// Backward step, second half: add the force VJP to the cotangents of the
// predicted state and take them through the predictor's transpose:
//   xp = x + v dt + a h dt + k q h dt,   vp = v + a dt + k h dt.
__global__ void k_adj_post(int n, double dt, double *xb, double *vb, double *ab, double *kb,
                           double *mb, const double *xg, const double *vg, const double *mg)
{
    const double h = dt / 2.0, q = dt / 3.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const long long e = 3LL * i + c;
            const double xpb = xb[e] + xg[e], vpb = vb[e] + vg[e];
            xb[e] = xpb;
            vb[e] = xpb * dt + vpb;
            ab[e] += xpb * h * dt + vpb * dt;
            kb[e] += xpb * q * h * dt + vpb * h * dt;
        }
        mb[i] += mg[i];
    }
}

// Records for a VJP at the un-predicted state (the initial force), and the
// final accumulation of its result.
__global__ void k_adj_initial_rec(State st, const double *ab, const double *kb, int precision,
                                  VjpRecDS rec, VjpRec64 rec64)
{
    const int n = st.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double x[3], v[3], a[3], k[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = st.x[c * n + i];
            v[c] = st.v[c * n + i];
            a[c] = ab[3LL * i + c];
            k[c] = kb[3LL * i + c];
        }
        write_vjp_record(i, x, v, st.m[i], a, k, precision, rec, rec64);
    }
}

__global__ void k_add3(int n, double *dst, const double *src, double *dst2, const double *src2,
                       double *dstm, const double *srcm)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            dst[3LL * i + c] += src[3LL * i + c];
            dst2[3LL * i + c] += src2[3LL * i + c];
        }
        dstm[i] += srcm[i];
    }
}

// Acceleration and jerk of a full sweep (public layout) into the SoA state.
__global__ void k_set_ak(State st, const double *acc, const double *jerk)
{
    const int n = st.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            st.a[c * n + i] = acc[3LL * i + c];
            st.k[c * n + i] = jerk[3LL * i + c];
        }
}

// Copies of the FP64 state (checkpoints).
__global__ void k_copy_state(State dst, State src)
{
    const long long n3 = 3LL * src.n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n3;
         e += (long long)gridDim.x * blockDim.x) {
        dst.x[e] = src.x[e];
        dst.v[e] = src.v[e];
        dst.a[e] = src.a[e];
        dst.k[e] = src.k[e];
    }
}

int grid_for(long long n, int nt)
{
    long long g = (n + nt - 1) / nt;
    return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
}

}  // namespace

int vjp_slots(int precision, int sms)
{
    int b = 0;
    cudaError_t e = precision == NB_FP64
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_force_vjp_f64<true>, kVNT, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_force_vjp_ds<true>, kVNT, 0);
    return e == cudaSuccess ? sms * (b > 0 ? b : 1) : sms;
}

int vjp_tile() { return kVNT; }

int launch_force_vjp(const VjpArgs &va_in, int precision, bool softened, cudaStream_t st)
{
    VjpArgs va = va_in;
    // once, on the host; the DS kernel owns kVKR particles per thread
    va.plan = plan_ipar(va.n, va.n, kVNT * (precision == NB_FP64 ? 1 : kVKR), kVNT, va.slots, 0,
                        va.part_cap);
    const Plan P = va.plan;
    const int g = P.items < va.slots ? P.items : va.slots;
    if (precision == NB_FP64) {
        if (softened) k_force_vjp_f64<true><<<g, kVNT, 0, st>>>(va);
        else k_force_vjp_f64<false><<<g, kVNT, 0, st>>>(va);
    } else {
        if (softened) k_force_vjp_ds<true><<<g, kVNT, 0, st>>>(va);
        else k_force_vjp_ds<false><<<g, kVNT, 0, st>>>(va);
    }
    int launches = 1;
    if (P.S > 1) {
        k_vjp_combine<<<grid_for(7LL * va.n, 256), 256, 0, st>>>(va, P.S);
        ++launches;
    }
    return launches;
}

void launch_adj_pre(const State &s, double dt, const double *xb, const double *vb, double *ab,
                    double *kb, int precision, const VjpRecDS &rec, const VjpRec64 &rec64,
                    cudaStream_t st)
{
    k_adj_pre<<<grid_for(s.n, 128), 128, 0, st>>>(s, dt, xb, vb, ab, kb, precision, rec, rec64);
}

void launch_adj_post(int n, double dt, double *xb, double *vb, double *ab, double *kb, double *mb,
                     const double *xg, const double *vg, const double *mg, cudaStream_t st)
{
    k_adj_post<<<grid_for(n, 256), 256, 0, st>>>(n, dt, xb, vb, ab, kb, mb, xg, vg, mg);
}

void launch_adj_initial_rec(const State &s, const double *ab, const double *kb, int precision,
                            const VjpRecDS &rec, const VjpRec64 &rec64, cudaStream_t st)
{
    k_adj_initial_rec<<<grid_for(s.n, 256), 256, 0, st>>>(s, ab, kb, precision, rec, rec64);
}

void launch_add3(int n, double *dst, const double *src, double *dst2, const double *src2,
                 double *dstm, const double *srcm, cudaStream_t st)
{
    k_add3<<<grid_for(n, 256), 256, 0, st>>>(n, dst, src, dst2, src2, dstm, srcm);
}

void launch_set_ak(const State &s, const double *acc, const double *jerk, cudaStream_t st)
{
    k_set_ak<<<grid_for(s.n, 256), 256, 0, st>>>(s, acc, jerk);
}

void launch_copy_state(const State &dst, const State &src, cudaStream_t st)
{
    k_copy_state<<<grid_for(3LL * src.n, 256), 256, 0, st>>>(dst, src);
}

}  // namespace nbk
