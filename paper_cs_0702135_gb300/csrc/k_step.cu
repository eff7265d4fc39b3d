// k_step.cu -- the O(N) kernels around the force: Hermite predictor, Hermite
// corrector with the block time step, block scheduler, energy reduction.
//
// All FP64 arithmetic of the predictor, corrector and time-step criterion
// (nb_device.cuh, shared with the ensemble and reverse-mode kernels) uses
// explicit round-to-nearest intrinsics (__dadd_rn, __dmul_rn, __ddiv_rn,
// __dsqrt_rn) in the order the formulas are written, so that no multiply-add
// is contracted and the same inputs give the same bits as any IEEE FP64
// evaluation of those formulas in that order.  This is what lets integer block
// levels be compared bit for bit with a CPU evaluation.
#include <algorithm>
#include <climits>

#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

__device__ __forceinline__ void raise_err(int *err, int code)
{
    atomicCAS(err, 0, code);
}

// ---------------------------------------------------------------------------

// Particle i predicted to tn, written as its j record of the force kernels.
__device__ __forceinline__ void predict_record(const State &s, int i, long long tn, int precision,
                                               const JDS &jds, const JF64 &jf)
{
    const double dt = ticks_to_time(tn - s.t[i]);
    double xp[3], vp[3];
    predict3(s, i, s.n, dt, xp, vp);
    const double m = s.m[i];
    if (precision == NB_FP64) {
        jf.pos[i] = make_double4_32a(xp[0], xp[1], xp[2], m);
        jf.vel[i] = make_double4_32a(vp[0], vp[1], vp[2], 0.0);
    } else {
        float hi[3], lo[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) split_ds(xp[c], hi[c], lo[c]);
        jds.pos_hi[i] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(m));
        jds.pos_lo[i] = make_float4(lo[0], lo[1], lo[2], 0.0f);
        jds.vel[i] = make_float4(__double2float_rn(vp[0]), __double2float_rn(vp[1]),
                                 __double2float_rn(vp[2]), 0.0f);
    }
}

__global__ void k_predict(State s, long long t_val, const long long *t_ptr, const int *gate,
                          int precision, JDS jds, JF64 jf)
{
    if (gate && *gate <= 0) return;
    const long long tn = t_ptr ? *t_ptr : t_val;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s.n; i += gridDim.x * blockDim.x)
        predict_record(s, i, tn, precision, jds, jf);
}

// Hermite corrector and Aarseth step for the block (Section 2); the
// arithmetic is correct_particle's.  One warp per CTA: blocks of at most
// quad_max particles take four lanes per particle (correct_particle_quad),
// eight particles per warp, so a small block spreads over many SMs' FP64
// pipes; larger blocks take one thread per particle.
__global__ void __launch_bounds__(32) k_correct(State s, const int *act, int na_host,
                                                const int *na_dev, long long t_val,
                                                const long long *t_ptr, const double *acc_new,
                                                const double *jerk_new, double eta, int level_min,
                                                int level_fixed, int quad_max, int *err)
{
    const int na = na_dev ? *na_dev : na_host;
    if (na <= 0) return;
    const long long tn = t_ptr ? *t_ptr : t_val;
    const int lane = threadIdx.x;
    if (na <= quad_max) {
        const int tasks = (na + 7) / 8;
        for (int w = blockIdx.x; w < tasks; w += gridDim.x) {
            const int b = w * 8 + (lane >> 2), q = lane & 3;
            const bool active = b < na;
            const long long bb = active ? b : na - 1;
            const int c = q < 3 ? q : 2;
            const bool ok = correct_particle_quad(s, act[bb], s.n, tn, acc_new[3 * bb + c],
                                                  jerk_new[3 * bb + c], eta, level_min, level_fixed,
                                                  active);
            if (active && q == 0 && !ok) raise_err(err, NB_ESTEP);
        }
        return;
    }
    for (int b = blockIdx.x * 32 + lane; b < na; b += gridDim.x * 32) {
        double ap[3], kp[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ap[c] = acc_new[3 * (long long)b + c];
            kp[c] = jerk_new[3 * (long long)b + c];
        }
        if (!correct_particle(s, act[b], s.n, tn, ap, kp, eta, level_min, level_fixed))
            raise_err(err, NB_ESTEP);
    }
}

// Start-up: acc and jerk from the t = 0 sweep (public layout) into the SoA
// state, t = 0, and the initial step eta_init |a| / |k|.
__global__ void k_initial(State s, const double *acc, const double *jerk, double eta_init,
                          int level_min, int level_fixed, int *err)
{
    const int n = s.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double a[3], k[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            a[c] = acc[3 * (long long)i + c];
            k[c] = jerk[3 * (long long)i + c];
            s.a[c * n + i] = a[c];
            s.k[c * n + i] = k[c];
        }
        s.t[i] = 0;
        if (level_fixed > 0) {
            s.lev[i] = level_fixed;
            continue;
        }
        int lv;
        if (!level_of(initial_dt(a, k, eta_init), level_min, lv)) {
            raise_err(err, NB_ESTEP);
            lv = kTickBits;
        }
        s.lev[i] = lv;
    }
}

// ---------------------------------------------------------------------------
// Block scheduler: t_next = min_i (t_i + 2^-lev_i) in ticks, then the block
// {i : t_i + 2^-lev_i = t_next} compacted in ascending order by warp ballot
// and prefix sums.  Two launches: per-chunk minimum and the count at it; then
// the global minimum, per-chunk offsets and scatter, in the same launch as the
// prediction of every particle to the new block time (Section 2's predictor
// step, which needs nothing but that time).

constexpr int kSchedNT = 256;
constexpr int kSchedChunk = kSchedNT * 8;

__device__ __forceinline__ long long end_time(const State &s, int i)
{
    return s.t[i] + (1LL << (kTickBits - s.lev[i]));
}

template <typename T, typename Op>
__device__ __forceinline__ T block_reduce(T v, Op op, T *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, off));
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    T r = smem[0];
    for (int w = 1; w < nw; ++w) r = op(r, smem[w]);
    return r;
}

struct MinOp {
    __device__ long long operator()(long long a, long long b) const { return a < b ? a : b; }
};
struct SumOp {
    template <typename T>
    __device__ T operator()(T a, T b) const { return a + b; }
};

// Per chunk its minimum end time and how many of its particles end then (a
// chunk's count matters only if its minimum is the block time).
__global__ void k_sched_min(State s, long long *blockmin, int *blockcnt)
{
    __shared__ long long sm[kSchedNT / 32];
    __shared__ int si[kSchedNT / 32];
    constexpr int kPer = kSchedChunk / kSchedNT;
    const int lo = blockIdx.x * kSchedChunk;
    const int hi = min(s.n, lo + kSchedChunk);
    long long et[kPer];
    long long m = LLONG_MAX;
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
        const int i = lo + q * kSchedNT + threadIdx.x;
        et[q] = i < hi ? end_time(s, i) : LLONG_MAX;
        m = min(m, et[q]);
    }
    m = block_reduce(m, MinOp(), sm);
    int cnt = 0;
#pragma unroll
    for (int q = 0; q < kPer; ++q) cnt += et[q] == m;
    cnt = block_reduce(cnt, SumOp(), si);
    if (threadIdx.x == 0) {
        blockmin[blockIdx.x] = m;
        blockcnt[blockIdx.x] = cnt;
    }
}

// Every CTA reduces the chunk minima to the block time; CTAs below nblocks
// scatter their chunk's block members into act (the last of them also writes
// n_active and the force plan), then every CTA predicts its share of the
// particles.
__global__ void k_sched_scatter(State s, Ctrl *ctrl, const long long *blockmin, const int *blockcnt,
                                int *act, int nblocks, ForceArgs fa, ForcePlan *plan_out,
                                int precision, JDS jds, JF64 jf)
{
    __shared__ long long sm[kSchedNT / 32];
    __shared__ int si[kSchedNT / 32];
    __shared__ int wtot[kSchedNT / 32];
    // the block time: the least chunk minimum (every CTA reduces the same values)
    long long tn = LLONG_MAX;
    for (int b = threadIdx.x; b < nblocks; b += kSchedNT) tn = min(tn, blockmin[b]);
    tn = block_reduce(tn, MinOp(), sm);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->t_next = tn;
    const bool done = tn > ctrl->t_end;
    const bool chunk = blockIdx.x < nblocks;   // CTAs past the chunks only predict
    int pre = 0;   // no block past the end time: nothing counted
    if (!done && chunk)
        for (int b = threadIdx.x; b < blockIdx.x; b += kSchedNT) pre += blockmin[b] == tn ? blockcnt[b] : 0;
    pre = block_reduce(pre, SumOp(), si);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int lo = blockIdx.x * kSchedChunk;
    const int hi = min(s.n, lo + kSchedChunk);
    int running = 0;
    if (!done && chunk) {
        for (int base = lo; base < hi; base += kSchedNT) {
            const int i = base + threadIdx.x;
            const bool f = i < hi && end_time(s, i) == tn;
            const unsigned bal = __ballot_sync(0xffffffffu, f);
            const int below = __popc(bal & ((1u << lane) - 1u));
            __syncthreads();
            if (lane == 0) wtot[warp] = __popc(bal);
            __syncthreads();
            int woff = 0, tot = 0;
            for (int w = 0; w < kSchedNT / 32; ++w) {
                if (w < warp) woff += wtot[w];
                tot += wtot[w];
            }
            if (f) act[pre + running + woff + below] = i;
            running += tot;
        }
    }
    if (blockIdx.x == nblocks - 1 && threadIdx.x == 0) {
        const int total = pre + running;
        ctrl->n_active = total;
        *plan_out = make_force_plan(fa, total);   // the force launches read it
        if (total > 0) {
            ctrl->t_now = tn;
            ctrl->steps += 1;
            ctrl->interactions += (long long)total * (long long)(s.n - 1);
        }
    }
    // every particle predicted to the block time (a block exists whenever tn
    // is not past the end time)
    if (!done)
        for (int i = blockIdx.x * kSchedNT + threadIdx.x; i < s.n; i += gridDim.x * kSchedNT)
            predict_record(s, i, tn, precision, jds, jf);
}

// ---------------------------------------------------------------------------
// Energy: T = 1/2 sum m v_p^2 with v predicted to the system time, and
// W = 1/2 sum m_i pot_i; per-block FP64 partials, then one block sums them in
// block order (deterministic).

constexpr int kEnNT = 256;

__global__ void k_energy_partial(State s, const long long *t_ptr, const double *pot, double *part)
{
    __shared__ double sm[kEnNT / 32];
    const long long tn = *t_ptr;
    const int n = s.n;
    double ke = 0.0, pe = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double dt = ticks_to_time(tn - s.t[i]);
        double xp[3], vp[3], v2 = 0.0;
        predict3(s, i, n, dt, xp, vp);
#pragma unroll
        for (int c = 0; c < 3; ++c) v2 += vp[c] * vp[c];
        ke += 0.5 * s.m[i] * v2;
        pe += 0.5 * s.m[i] * pot[i];
    }
    ke = block_reduce(ke, SumOp(), sm);
    pe = block_reduce(pe, SumOp(), sm);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = ke;
        part[2 * blockIdx.x + 1] = pe;
    }
}

__global__ void k_energy_final(const double *part, int nblocks, Ctrl *ctrl)
{
    __shared__ double sm[kEnNT / 32];
    double ke = 0.0, pe = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kEnNT) {
        ke += part[2 * b];
        pe += part[2 * b + 1];
    }
    ke = block_reduce(ke, SumOp(), sm);
    pe = block_reduce(pe, SumOp(), sm);
    if (threadIdx.x == 0) {
        ctrl->ekin = ke;
        ctrl->epot = pe;
    }
}

// ---------------------------------------------------------------------------

__global__ void k_validate(const int *idx, int na, int n, unsigned int *bitmap, int *err)
{
    for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < na; a += gridDim.x * blockDim.x) {
        const int i = idx[a];
        if (i < 0 || i >= n) {
            raise_err(err, NB_EINVAL);
            continue;
        }
        const unsigned bit = 1u << (i & 31);
        if (atomicOr(&bitmap[i >> 5], bit) & bit) raise_err(err, NB_EINVAL);
    }
}

__global__ void k_check_input(const double *p, long long cnt, bool nonneg, int *err)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < cnt;
         e += (long long)gridDim.x * blockDim.x) {
        const double q = p[e];
        if (!isfinite(q) || (nonneg && q < 0.0)) raise_err(err, kErrInput);
    }
}

__global__ void k_gather_state(State s, double *x, double *v, double *a, double *k)
{
    const int n = s.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (x) x[3 * (long long)i + c] = s.x[c * n + i];
            if (v) v[3 * (long long)i + c] = s.v[c * n + i];
            if (a) a[3 * (long long)i + c] = s.a[c * n + i];
            if (k) k[3 * (long long)i + c] = s.k[c * n + i];
        }
}

__global__ void k_scatter_state(State s, const double *x, const double *v, const double *a,
                                const double *k)
{
    const int n = s.n;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            if (x) s.x[c * n + i] = x[3 * (long long)i + c];
            if (v) s.v[c * n + i] = v[3 * (long long)i + c];
            if (a) s.a[c * n + i] = a[3 * (long long)i + c];
            if (k) s.k[c * n + i] = k[3 * (long long)i + c];
        }
}

__global__ void k_iota(int *p, int n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

int grid_for(long long n, int nt)
{
    long long g = (n + nt - 1) / nt;
    if (g < 1) g = 1;
    if (g > 8192) g = 8192;
    return (int)g;
}

}  // namespace

void launch_predict(const State &s, long long t_val, const long long *t_ptr, const int *gate,
                    int precision, JDS jds, JF64 jf, cudaStream_t st)
{
    k_predict<<<grid_for(s.n, 256), 256, 0, st>>>(s, t_val, t_ptr, gate, precision, jds, jf);
}

void launch_correct(const State &s, const int *act, int na_host, const int *na_dev, long long t_val,
                    const long long *t_ptr, const double *acc_new, const double *jerk_new,
                    double eta, int level_min, int level_fixed, int *err, int sms, cudaStream_t st)
{
    // quad_max: where eight particles per warp stop beating 32 (a warp per
    // SM of each form; measured on whole block-step runs)
    const int quad_max = kCorrectQuadPerSM * (sms > 0 ? sms : 1);
    const long long cap = na_dev ? (long long)s.n : (long long)na_host;
    const long long tasks = std::max((cap + 31) / 32, (std::min<long long>(cap, quad_max) + 7) / 8);
    const int g = (int)std::max(1LL, std::min(tasks, 8192LL));
    k_correct<<<g, 32, 0, st>>>(s, act, na_host, na_dev, t_val, t_ptr, acc_new, jerk_new, eta,
                                level_min, level_fixed, quad_max, err);
}

void launch_initial_steps(const State &s, const double *acc, const double *jerk, double eta_init,
                          int level_min, int level_fixed, int *err, cudaStream_t st)
{
    k_initial<<<grid_for(s.n, 256), 256, 0, st>>>(s, acc, jerk, eta_init, level_min, level_fixed, err);
}

int schedule_blocks(int n) { return cdiv(n, kSchedChunk); }

void launch_schedule(const State &s, Ctrl *ctrl, long long *blockmin, int *blockcnt, int *act,
                     int nblocks, const ForceArgs &fa, ForcePlan *plan_out, int precision,
                     const JDS &jds, const JF64 &jf, cudaStream_t st)
{
    k_sched_min<<<nblocks, kSchedNT, 0, st>>>(s, blockmin, blockcnt);
    const int g = std::max(nblocks, grid_for(s.n, kSchedNT));
    k_sched_scatter<<<g, kSchedNT, 0, st>>>(s, ctrl, blockmin, blockcnt, act, nblocks, fa, plan_out,
                                            precision, jds, jf);
}

int energy_blocks(int n)
{
    int g = cdiv(n, kEnNT * 8);
    return g < 1 ? 1 : (g > 1024 ? 1024 : g);
}

void launch_energy(const State &s, const long long *t_ptr, const double *pot, double *part,
                   Ctrl *ctrl, cudaStream_t st)
{
    const int nb = energy_blocks(s.n);
    k_energy_partial<<<nb, kEnNT, 0, st>>>(s, t_ptr, pot, part);
    k_energy_final<<<1, kEnNT, 0, st>>>(part, nb, ctrl);
}

void launch_validate(const int *idx, int na, int n, unsigned int *bitmap, int *err, cudaStream_t st)
{
    if (na <= 0) return;
    k_validate<<<grid_for(na, 256), 256, 0, st>>>(idx, na, n, bitmap, err);
}

void launch_gather_state(const State &s, double *x, double *v, double *a, double *k, cudaStream_t st)
{
    k_gather_state<<<grid_for(s.n, 256), 256, 0, st>>>(s, x, v, a, k);
}

void launch_scatter_state(const State &s, const double *x, const double *v, const double *a,
                          const double *k, cudaStream_t st)
{
    k_scatter_state<<<grid_for(s.n, 256), 256, 0, st>>>(s, x, v, a, k);
}

void launch_check_input(const double *p, long long cnt, bool nonneg, int *err, cudaStream_t st)
{
    if (cnt <= 0 || !p) return;
    k_check_input<<<grid_for(cnt, 256), 256, 0, st>>>(p, cnt, nonneg, err);
}

void launch_iota(int *p, int n, cudaStream_t st)
{
    k_iota<<<grid_for(n, 256), 256, 0, st>>>(p, n);
}

}  // namespace nbk
