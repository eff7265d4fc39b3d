// k_run.cu -- the block-step loop of nb_run (Section 2: select the block,
// predict, force, correct, repeat) in one persistent cooperative launch, for
// systems small enough that a step is mostly launch latency on the
// kernel-per-stage path.
//
// CTA r owns particles [r P, (r + 1) P).  One block step is three phases
// separated by grid barriers (a counter in global memory, added to with
// release and read with acquire semantics; each wait ends after about 2 s
// with NB_ETIMEOUT, and the cooperative launch keeps every CTA resident):
//   1. the CTA corrects its own particles of the previous block: a warp adds a
//      particle's partials over the CTAs (lanes over CTAs, then a fixed
//      shuffle tree), then the FP64 corrector and Aarseth step run (four
//      lanes per particle for up to 16 particles); the new end times
//      t_i + 2^-lev_i of its particles, kept in shared memory, give its
//      minimum and how many of its particles end then;
//   2. the block time t_next = min over the CTAs (the same in every CTA, so
//      every CTA takes the same decision to stop); a CTA has block particles
//      exactly when its own minimum is t_next, and writes them, in ascending
//      order, at its offset in the block list; its particles predicted (FP64)
//      into the double-single j records (fixed point: its largest mass and
//      |vx|+|vy|+|vz|);
//   3. force partials: every CTA sums every block particle's pair terms over
//      its own particles as j and writes them per (CTA, block particle).
// Since a particle is corrected by its owner, no CTA reads another CTA's
// state, and the correction needs no barrier of its own.
// Everything that other CTAs wrote in the same launch is read past L1
// (__ldcg).  Two summations: the compensated double-single sums
// (TwoSum-promoted FP32 partials, FP64 across CTAs) and the GRAPE-style
// fixed-point sums of k_sum.cu (exact, so the run is bit-identical to the
// kernel-per-stage path and to any IEEE evaluation of the same sums).
#include <climits>

#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

constexpr unsigned kFullR = 0xffffffffu;
constexpr long long kRunSpinCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ long long end_time_of(const State &s, int i)
{
    return __ldcg(&s.t[i]) + (1LL << (kTickBits - __ldcg(&s.lev[i])));
}

__device__ __forceinline__ void arrive_release(unsigned long long *p)
{
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(p) : "memory");
}

__device__ __forceinline__ unsigned long long load_acquire(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait (one thread): until *p >= target, read with acquire semantics;
// false after `limit` SM cycles.  Spins first, then sleeps between reads.
__device__ __forceinline__ bool wait_counter(const unsigned long long *p, unsigned long long target,
                                             long long limit)
{
    const long long t0 = clock64();
    int spins = 0;
    while (load_acquire(p) < target) {
        if (++spins > 256) {
            if (clock64() - t0 > limit) return false;
            __nanosleep(64);
        }
    }
    return true;
}

// Grid barrier: thread 0 of every CTA adds one arrival (release: the CTA's
// writes, ordered before it by __syncthreads, become visible first) and waits
// (acquire) until all CTAs' arrivals for this barrier are in.  False when the
// wait ran out (error NB_ETIMEOUT).
__device__ __forceinline__ bool grid_barrier(const RunArgs &ra, unsigned long long &target, int *s_ok)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        target += (unsigned long long)ra.ncta;
        arrive_release(ra.bar);
        const bool ok = wait_counter(ra.bar, target, kRunSpinCycles);
        if (!ok) atomicCAS(&ra.ctrl->err, 0, NB_ETIMEOUT);
        *s_ok = ok;
    }
    __syncthreads();
    return *s_ok != 0;
}

// The same wait on a counter that nothing increments, for nb_check_wait.
__global__ void k_check_wait(const unsigned long long *counter, long long limit, Ctrl *ctrl)
{
    if (!wait_counter(counter, 1ULL, limit)) atomicCAS(&ctrl->err, 0, NB_ETIMEOUT);
}

template <typename T, typename Op>
__device__ __forceinline__ T cta_reduce_r(T v, Op op, T *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = op(v, __shfl_xor_sync(kFullR, v, o));
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    T r = smem[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = op(r, smem[w]);
    __syncthreads();
    return r;
}

struct MinR {
    __device__ long long operator()(long long a, long long b) const { return a < b ? a : b; }
};
struct AddR {
    __device__ long long operator()(long long a, long long b) const { return a + b; }
};
struct MaxU {
    __device__ unsigned operator()(unsigned a, unsigned b) const { return a > b ? a : b; }
};

// Phase 4, compensated sums: block particles a in passes of NT / g, g lanes
// per particle splitting the CTA's j slice; FP32 partials promoted by TwoSum
// every 64 pairs per lane, the lane group reduced in double-single.
__device__ __forceinline__ void force_ds(const RunArgs &ra, int r, int na, int j0, int m,
                                         const float4 *s_p, const float4 *s_l, const float4 *s_v)
{
    const int tid = threadIdx.x;
    int g = 1;
    while (g < 32 && g * 2 * na <= kRunNT) g <<= 1;
    const int grp = tid / g, lig = tid % g;
    for (int a0 = 0; a0 < na; a0 += kRunNT / g) {
        const int a = a0 + grp;
        const bool valid = a < na;
        const int i = __ldcg(&ra.act[valid ? a : 0]);
        const float4 ip = __ldcg(&ra.j.pos_hi[i]), il = __ldcg(&ra.j.pos_lo[i]), iv = __ldcg(&ra.j.vel[i]);
        const IDS I = make_ids(ip, il, iv);
        float hi[7] = {0, 0, 0, 0, 0, 0, 0}, lo[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int jb = 0; jb < m; jb += 64 * g) {
            const int je = min(m, jb + 64 * g);
            float ta[3] = {0, 0, 0}, tk[3] = {0, 0, 0}, tp = 0.0f;
            for (int jj = jb + lig; jj < je; jj += g)
                pair_ds_packed<false, true>(s_p[jj], s_l[jj], s_v[jj], I, ra.eps2f, ta, tk, tp,
                                            j0 + jj, i);
            const float t7[7] = {ta[0], ta[1], ta[2], tk[0], tk[1], tk[2], tp};
#pragma unroll
            for (int c = 0; c < 7; ++c) two_sum_acc(hi[c], lo[c], t7[c]);
        }
        for (int sh = 1; sh < g; sh <<= 1) {
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const float h2 = __shfl_xor_sync(kFullR, hi[c], sh);
                const float l2 = __shfl_xor_sync(kFullR, lo[c], sh);
                ds_add(hi[c], lo[c], h2, l2);
            }
        }
        if (valid && lig == 0) {
            double *p = ra.part + ((long long)r * ra.n + a) * kComp;
#pragma unroll
            for (int c = 0; c < 7; ++c) p[c] = (double)hi[c] + (double)lo[c];
        }
    }
}

// Phase 4, fixed point: the same passes; every term rounded to an integer by
// the exact FP32 splits, tiles of at most 64 terms per lane summed in 32 bits
// and then in 128 bits, the lane group reduced in 128 bits.
__device__ __forceinline__ void force_fixed(const RunArgs &ra, int r, int na, int j0, int m,
                                            const float4 *s_p, const float4 *s_l, const float4 *s_v,
                                            const Scale &S)
{
    const int tid = threadIdx.x;
    int g = 1;
    while (g < 32 && g * 2 * na <= kRunNT) g <<= 1;
    const int grp = tid / g, lig = tid % g;
    long long *part = reinterpret_cast<long long *>(ra.part);
    for (int a0 = 0; a0 < na; a0 += kRunNT / g) {
        const int a = a0 + grp;
        const bool valid = a < na;
        const int i = __ldcg(&ra.act[valid ? a : 0]);
        const float4 ip = __ldcg(&ra.j.pos_hi[i]), il = __ldcg(&ra.j.pos_lo[i]), iv = __ldcg(&ra.j.vel[i]);
        const float xh[3] = {ip.x, ip.y, ip.z}, xl[3] = {il.x, il.y, il.z}, vi[3] = {iv.x, iv.y, iv.z};
        long long hi[7];
        unsigned long long lo[7];
#pragma unroll
        for (int c = 0; c < 7; ++c) hi[c] = 0, lo[c] = 0;
        for (int jb = 0; jb < m; jb += 64 * g) {
            const int je = min(m, jb + 64 * g);
            unsigned s1[7], s2[7], s3[7];
#pragma unroll
            for (int c = 0; c < 7; ++c) s1[c] = s2[c] = s3[c] = 0u;
            unsigned cnt = 0;
            for (int jj = jb + lig; jj < je; jj += g) {
                float t[7];
                pair_rn(s_p[jj], s_l[jj], s_v[jj], xh, xl, vi, ra.eps2f, S.sc[0], S.sc[1], S.sc[2], t);
                const bool self = j0 + jj == i;
#pragma unroll
                for (int c = 0; c < 7; ++c) split_add(self ? 0.0f : t[c], s1[c], s2[c], s3[c]);
                ++cnt;
            }
#pragma unroll
            for (int c = 0; c < 7; ++c) add128(hi[c], lo[c], tile_sum(s1[c], s2[c], s3[c], cnt));
        }
        for (int sh = 1; sh < g; sh <<= 1) {
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                const long long h2 = __shfl_xor_sync(kFullR, hi[c], sh);
                const unsigned long long l2 = __shfl_xor_sync(kFullR, lo[c], sh);
                const unsigned long long ls = lo[c] + l2;
                hi[c] += h2 + (ls < lo[c] ? 1 : 0);
                lo[c] = ls;
            }
        }
        if (valid && lig == 0) {
            long long *p = part + 2 * (((long long)r * ra.n + a) * kComp);
#pragma unroll
            for (int c = 0; c < 7; ++c) {
                p[2 * c] = hi[c];
                p[2 * c + 1] = (long long)lo[c];
            }
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kRunNT) k_run(RunArgs ra)
{
    __shared__ float4 s_p[kRunNT], s_l[kRunNT], s_v[kRunNT];
    __shared__ long long s_red[kRunNT / 32];
    __shared__ unsigned s_redu[kRunNT / 32];
    __shared__ int s_wtot[kRunNT / 32];
    __shared__ int s_ok, s_err;
    __shared__ double s_res[kRunNT][kComp];   // phase 5: combined force of this CTA's block particles
    __shared__ int s_idx[kRunNT];              // phase 5: their particle indices
    __shared__ long long s_et[kRunNT];         // end times t_i + 2^-lev_i of this CTA's particles
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, r = blockIdx.x;
    const State &S = ra.s;
    const int n = ra.n;
    const int i0 = r * ra.per, i1 = min(n, i0 + ra.per);
    const int m = max(0, i1 - i0);
    unsigned long long target = 0;
    long long steps = 0;

    // end times of this CTA's particles: read once here, then kept up to date
    // by this CTA's own corrections (phase 1a)
    if (tid < m) s_et[tid] = end_time_of(S, i0 + tid);
    __syncthreads();
    long long off_b = 0, cnt_b = 0, tn_b = 0;
    for (;;) {
        if (steps > 0) {
            // 1a. The previous block's particles that this CTA owns (block
            // positions off_b .. off_b + cnt_b - 1): partials in CTA order,
            // corrector, new steps, and their new end times into s_et.
            Scale Sc;
            bool scale_ok = true;
            if (MODE == NB_SUM_FIXED) {
                unsigned bm = 0, bv = 0;
                for (int q = tid; q < ra.ncta; q += kRunNT) {
                    bm = max(bm, __ldcg(&ra.maxs[2 * q]));
                    bv = max(bv, __ldcg(&ra.maxs[2 * q + 1]));
                }
                bm = cta_reduce_r(bm, MaxU(), s_redu);
                bv = cta_reduce_r(bv, MaxU(), s_redu);
                const unsigned bounds[2] = {bm, bv};
                scale_ok = fixed_scale(bounds, ra.eps2f, Sc);
            }
            // warp w adds the partials of particles k = w, w + 8, ... over the CTAs
            // (lane l takes CTAs l, l + 32, ... in order, then a fixed xor tree;
            // exact in fixed point), then the particles are corrected
            const long long cnt_r = cnt_b;
            for (long long k0 = 0; scale_ok && k0 < cnt_r; k0 += kRunNT) {
                const int kn = (int)min((long long)kRunNT, cnt_r - k0);
                for (int k = warp; k < kn; k += kRunNT / 32) {
                    const long long a = off_b + k0 + k;
                    if (lane == 0) s_idx[k] = __ldcg(&ra.act[a]);
                    // a CTA's seven partials of a particle are contiguous: a lane
                    // loads all seven of each of its CTAs at once, so the loads
                    // of every component are in flight together
                    if (MODE == NB_SUM_FIXED) {
                        const long long *part = reinterpret_cast<const long long *>(ra.part);
                        long long hi[7];
                        unsigned long long lo[7];
#pragma unroll
                        for (int c = 0; c < 7; ++c) hi[c] = 0, lo[c] = 0;
                        for (int q = lane; q < ra.ncta; q += 32) {
                            const long long *pp = part + 2 * (((long long)q * n + a) * kComp);
                            long long ph[7], pl[7];
#pragma unroll
                            for (int c = 0; c < 7; ++c) ph[c] = __ldcg(&pp[2 * c]), pl[c] = __ldcg(&pp[2 * c + 1]);
#pragma unroll
                            for (int c = 0; c < 7; ++c) {
                                const unsigned long long l2 = lo[c] + (unsigned long long)pl[c];
                                hi[c] += ph[c] + (l2 < lo[c] ? 1 : 0);
                                lo[c] = l2;
                            }
                        }
#pragma unroll
                        for (int c = 0; c < 7; ++c) {
#pragma unroll
                            for (int o = 16; o >= 1; o >>= 1) {
                                const long long h2 = __shfl_xor_sync(kFullR, hi[c], o);
                                const unsigned long long l2 = __shfl_xor_sync(kFullR, lo[c], o);
                                const unsigned long long ls = lo[c] + l2;
                                hi[c] += h2 + (ls < lo[c] ? 1 : 0);
                                lo[c] = ls;
                            }
                            if (lane == 0)
                                s_res[k][c] = __dmul_rn(i128_to_double(hi[c], lo[c]),
                                                        c < 3 ? Sc.inv[0] : (c < 6 ? Sc.inv[1] : Sc.inv[2]));
                        }
                    } else {
                        // per component the same order as before: CTAs lane,
                        // lane + 32, ... in turn, then the fixed xor tree
                        double sum[7] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
                        for (int q = lane; q < ra.ncta; q += 32) {
                            const double *pp = ra.part + ((long long)q * n + a) * kComp;
                            double v[7];
#pragma unroll
                            for (int c = 0; c < 7; ++c) v[c] = __ldcg(&pp[c]);
#pragma unroll
                            for (int c = 0; c < 7; ++c) sum[c] += v[c];
                        }
#pragma unroll
                        for (int c = 0; c < 7; ++c) {
                            double t = sum[c];
#pragma unroll
                            for (int o = 16; o >= 1; o >>= 1) t += __shfl_xor_sync(kFullR, t, o);
                            if (lane == 0) s_res[k][c] = t;
                        }
                    }
                }
                __syncthreads();
                if (kn <= kRunQuadMax) {
                    // few particles: four lanes each (the same FP64 operations,
                    // about half the FP64 instructions per particle)
                    if (warp * 8 < kn) {
                        const int kq = tid >> 2, qd = tid & 3;
                        const bool active = kq < kn;
                        const int kk = active ? kq : kn - 1;
                        const int c = qd < 3 ? qd : 2;
                        const int i = s_idx[kk];
                        const bool ok = correct_particle_quad<true>(S, i, n, tn_b, s_res[kk][c],
                                                                    s_res[kk][3 + c], ra.eta,
                                                                    ra.level_min, ra.level_fixed, active);
                        if (active && qd == 0) {
                            if (!ok) atomicCAS(&ra.ctrl->err, 0, NB_ESTEP);
                            // this lane stored the new level: read back in program order
                            s_et[i - i0] = tn_b + (1LL << (kTickBits - S.lev[i]));
                        }
                    }
                } else if (tid < kn) {
                    const double ap[3] = {s_res[tid][0], s_res[tid][1], s_res[tid][2]};
                    const double kp[3] = {s_res[tid][3], s_res[tid][4], s_res[tid][5]};
                    const int i = s_idx[tid];
                    if (!correct_particle<true>(S, i, n, tn_b, ap, kp, ra.eta, ra.level_min, ra.level_fixed))
                        atomicCAS(&ra.ctrl->err, 0, NB_ESTEP);
                    s_et[i - i0] = tn_b + (1LL << (kTickBits - S.lev[i]));
                }
                __syncthreads();
            }
            __syncthreads();
        }

        // 1b. own minimum end time (kept in s_et) and the particles that end then
        const long long et = tid < m ? s_et[tid] : LLONG_MAX;
        const long long mn = cta_reduce_r(et, MinR(), s_red);
        const bool at_min = tid < m && et == mn;
        const unsigned bal = __ballot_sync(kFullR, at_min);
        if (lane == 0) s_wtot[warp] = __popc(bal);
        __syncthreads();
        int woff = 0, cnt_min = 0;
        for (int w = 0; w < kRunNT / 32; ++w) {
            woff += w < warp ? s_wtot[w] : 0;
            cnt_min += s_wtot[w];
        }
        if (tid == 0) {
            ra.mins[r] = mn;
            ra.counts[r] = cnt_min;
        }
        if (!grid_barrier(ra, target, &s_ok)) return;

        // 2. block time, stop decision, offsets, block list, prediction.  The
        // state the prediction reads does not depend on the block time, and
        // each CTA's minimum and count are read once: all go out first.
        long long p_t = 0;
        double p_x[3], p_v[3], p_a[3], p_k[3];
        if (tid < m) {
            const int i = i0 + tid;
            p_t = __ldcg(&S.t[i]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                p_x[c] = __ldcg(&S.x[c * n + i]);
                p_v[c] = __ldcg(&S.v[c * n + i]);
                p_a[c] = __ldcg(&S.a[c * n + i]);
                p_k[c] = __ldcg(&S.k[c * n + i]);
            }
        }
        long long m_own = LLONG_MAX, c_own = 0;  // CTA tid's minimum and count
        if (tid < ra.ncta) {
            m_own = __ldcg(&ra.mins[tid]);
            c_own = __ldcg(&ra.counts[tid]);
        }
        long long tn = m_own;
        for (int q = tid + kRunNT; q < ra.ncta; q += kRunNT) tn = min(tn, __ldcg(&ra.mins[q]));
        tn = cta_reduce_r(tn, MinR(), s_red);
        if (tid == 0) s_err = *(volatile int *)&ra.ctrl->err;
        __syncthreads();
        if (s_err != 0 || tn > ra.t_end || steps >= ra.max_steps) {
            if (r == 0 && tid == 0 && s_err == 0 && tn > ra.t_end) {
                ra.ctrl->t_next = tn;  // as the per-stage scheduler leaves it
                ra.ctrl->n_active = 0;
            }
            return;
        }
        long long na = m_own == tn ? c_own : 0;
        long long off = tid < r ? na : 0;
        for (int q = tid + kRunNT; q < ra.ncta; q += kRunNT) {
            const long long cq = __ldcg(&ra.mins[q]) == tn ? (long long)__ldcg(&ra.counts[q]) : 0;
            na += cq;
            off += q < r ? cq : 0;
        }
        na = cta_reduce_r(na, AddR(), s_red);
        off = cta_reduce_r(off, AddR(), s_red);
        if (at_min && mn == tn) ra.act[off + woff + __popc(bal & ((1u << lane) - 1u))] = i0 + tid;
        off_b = off;                      // this CTA's block particles, corrected next iteration
        cnt_b = mn == tn ? cnt_min : 0;
        tn_b = tn;
        unsigned mb = 0, vb = 0;
        if (tid < m) {
            const int i = i0 + tid;
            // predict3's arithmetic on the state loaded above
            const double dt = ticks_to_time(tn - p_t);
            const double dt_h = __dmul_rn(dt, 0.5), dt_q = div_by<3>(dt);
            double xp[3], vp[3];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                predict1hq(p_x[c], p_v[c], p_a[c], p_k[c], dt, dt_h, dt_q, xp[c], vp[c]);
            float h[3], l[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) split_ds(xp[c], h[c], l[c]);
            const float mf = __double2float_rn(S.m[i]);
            const float4 v4 = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]),
                                          __double2float_rn(vp[2]), 0.0f);
            ra.j.pos_hi[i] = make_float4(h[0], h[1], h[2], mf);
            ra.j.pos_lo[i] = make_float4(l[0], l[1], l[2], 0.0f);
            ra.j.vel[i] = v4;
            if (MODE == NB_SUM_FIXED) {
                mb = __float_as_uint(mf);
                vb = __float_as_uint(__fadd_rn(__fadd_rn(fabsf(v4.x), fabsf(v4.y)), fabsf(v4.z)));
            }
        }
        if (MODE == NB_SUM_FIXED) {
            mb = cta_reduce_r(mb, MaxU(), s_redu);
            vb = cta_reduce_r(vb, MaxU(), s_redu);
            if (tid == 0) {
                ra.maxs[2 * r] = mb;
                ra.maxs[2 * r + 1] = vb;
            }
        }
        if (!grid_barrier(ra, target, &s_ok)) return;

        // 3. force partials of every block particle over this CTA's particles
        if (tid < m) {
            s_p[tid] = __ldcg(&ra.j.pos_hi[i0 + tid]);
            s_l[tid] = __ldcg(&ra.j.pos_lo[i0 + tid]);
            s_v[tid] = __ldcg(&ra.j.vel[i0 + tid]);
        }
        __syncthreads();
        if (MODE == NB_SUM_FIXED) {
            unsigned bm = 0, bv = 0;
            for (int q = tid; q < ra.ncta; q += kRunNT) {
                bm = max(bm, __ldcg(&ra.maxs[2 * q]));
                bv = max(bv, __ldcg(&ra.maxs[2 * q + 1]));
            }
            bm = cta_reduce_r(bm, MaxU(), s_redu);
            bv = cta_reduce_r(bv, MaxU(), s_redu);
            const unsigned bounds[2] = {bm, bv};
            Scale Sc;
            if (!fixed_scale(bounds, ra.eps2f, Sc)) {
                if (tid == 0) atomicCAS(&ra.ctrl->err, 0, kErrFixedScale);
                // keep the barriers in step; the next stop decision ends the run
            } else {
                force_fixed(ra, r, (int)na, i0, m, s_p, s_l, s_v, Sc);
            }
        } else {
            force_ds(ra, r, (int)na, i0, m, s_p, s_l, s_v);
        }
        if (!grid_barrier(ra, target, &s_ok)) return;

        ++steps;
        if (r == 0 && tid == 0) {
            ra.ctrl->t_next = tn;
            ra.ctrl->t_now = tn;
            ra.ctrl->n_active = (int)na;
            ra.ctrl->steps += 1;
            ra.ctrl->interactions += na * (long long)(n - 1);
        }
    }
}

}  // namespace

int run_layout(int n, int sms, int blocks_per_sm, int *ncta, int *per)
{
    // 32 particles per CTA up to 64 CTAs, then up to 64 particles per CTA
    // (64 CTAs at n = 4096), then one CTA per SM (measured on whole runs: more
    // CTAs share the force and the predictor but add to every barrier and to
    // the partials each block particle sums; above 4096 bodies the force
    // share wins)
    int p = (n + 63) / 64;
    if (p < 32) p = 32;
    if (p > 64) p = (n + sms - 1) / sms;
    if (p > kRunNT) return -1;
    const int c = (n + p - 1) / p;
    if (c > sms * blocks_per_sm) return -1;
    *ncta = c;
    *per = p;
    return 0;
}

int occupancy_run(int summation, int *blocks_per_sm)
{
    const cudaError_t e =
        summation == NB_SUM_FIXED
            ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_run<NB_SUM_FIXED>, kRunNT, 0)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_run<NB_SUM_COMPENSATED>, kRunNT, 0);
    return e == cudaSuccess ? 0 : -1;
}

cudaError_t launch_check_wait(const unsigned long long *counter, long long limit_cycles, Ctrl *ctrl,
                              cudaStream_t st)
{
    k_check_wait<<<1, 1, 0, st>>>(counter, limit_cycles, ctrl);
    return cudaGetLastError();
}

cudaError_t launch_run(const RunArgs &ra, int summation, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(ra.ncta);
    cfg.blockDim = dim3(kRunNT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (summation == NB_SUM_FIXED) return cudaLaunchKernelEx(&cfg, k_run<NB_SUM_FIXED>, ra);
    return cudaLaunchKernelEx(&cfg, k_run<NB_SUM_COMPENSATED>, ra);
}

}  // namespace nbk
