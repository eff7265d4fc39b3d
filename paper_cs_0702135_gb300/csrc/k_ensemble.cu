// k_ensemble.cu -- many independent clusters advanced together: every
// ensemble block step advances every unfinished cluster by its own next block
// step (Section 2 step loop: select the block, predict, force, correct) in one
// persistent cooperative launch, replayed from a CUDA graph.  Its CTAs work in
// two phases:
//   A. clusters, largest first, from a work counter: block time t_next = min
//      over the cluster of t_i + dt_i, the block compacted in ascending order
//      (ballot + prefix sums), every particle predicted to t_next (FP64, the
//      single-system predictor's arithmetic) into global double-single j
//      records, and one work item per chunk of up to threads / gmax active
//      particles published to a queue (the item's cluster index is written
//      last and marks it ready).  A cluster above 512 particles is not
//      predicted here: its prediction goes to the queue as chunks of 512,
//      ahead of its force items, so several CTAs share the FP64 work;
//   B. once every cluster is claimed, queue items in order: prediction chunks;
//      force items (which first wait for their cluster's prediction): the j
//      records stream through shared-memory tiles, g consecutive lanes share one
//      active particle and split its j loop when the chunk is small (g = the
//      largest power of two with g * chunk <= threads, capped at gmax), FP32
//      pair arithmetic on double-single positions with TwoSum-promoted partials
//      and a shuffle reduction in the lane group; the group's first lane
//      corrects its particle (FP64 corrector and Aarseth step, the
//      single-system corrector's arithmetic).  The force reads only the j
//      records, so correcting while other items still sum is safe.
// An item waits only for its own cluster's phase A, so the large clusters'
// items run while small clusters are still being predicted.  A CTA waiting for
// an item spins with a time limit (error NB_ETIMEOUT past it); the cooperative
// launch keeps every CTA resident, and every cluster is claimed before any CTA
// waits, so the wait always ends.  Every item is computed by one CTA in a fixed
// order, so results do not depend on which CTA takes it.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

constexpr int kEnsMaxN = 4096;       // largest cluster
constexpr int kEnsPredChunk = 512;   // larger clusters are predicted in chunks by several CTAs

struct EnsArgs {
    int C;                    // clusters
    const long long *off;     // [C + 1] particle offsets
    const int *order;         // clusters in decreasing size
    State s;                  // all particles, SoA over the total count
    float eps2;
    double eta, eta_init;
    int level_min;
    long long t_end;
    int gmax;                 // largest lane group per active particle
    int chunk;                // active particles per work item (threads / gmax)
    int *work;                // phase A: cluster counter
    int *work_b;              // phase B: item counter
    int *qlen;                // queue length (items reserved in phase A)
    int *a_done;              // clusters whose phase A finished
    int *qc, *qk;             // queue: cluster (-1 = not ready); force chunk k >= 0 or
                              // prediction chunk -1 - k of each item
    int qcap;                 // queue capacity: P + C (at most n_c + 1 items per cluster)
    int *pred_left;           // [C] prediction chunks of the cluster not yet done
    float4 *jph, *jpl, *jv;   // [P] predicted double-single records
    Mirror mir;               // [P] single-precision mirror of the FP64 state for the j predictor
    int *act;                 // [P] active particles of each cluster (local indices)
    int *na;                  // [C] block sizes
    long long *tnext;         // [C] block times
    int *done;                // [C]
    long long *steps;         // [C]
    long long *inter;         // [C] sum of n_active (n - 1)
    int *err;
    double *out_acc, *out_jerk, *out_pot;  // force-only mode: [P][3], [P][3], [P]
};

template <typename T, typename Op>
__device__ __forceinline__ T cta_reduce(T v, Op op, T *smem)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v = op(v, __shfl_xor_sync(0xffffffffu, v, o));
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    T r = smem[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = op(r, smem[w]);
    __syncthreads();
    return r;
}

struct MinLL {
    __device__ long long operator()(long long a, long long b) const { return a < b ? a : b; }
};

enum EnsMode { kEnsStep = 0, kEnsForce = 1, kEnsInit = 2 };

// j record of particle gi at block time tn from the single-precision mirror
// (predict_j32: FP32 Taylor increments, double-single position add).  The FP64
// state itself is predicted in FP64 by the corrector.
__device__ __forceinline__ void ens_predict_j32(const EnsArgs &ea, long long gi, long long tn)
{
    float4 ph, pl, pv;
    predict_j32(ea.mir, gi, tn - ea.s.t[gi], ph, pl, pv);
    ea.jph[gi] = ph;
    ea.jpl[gi] = pl;
    ea.jv[gi] = pv;
}

__device__ __forceinline__ void ens_write_mirror(const EnsArgs &ea, long long gi)
{
    write_mirror(ea.s, ea.mir, gi, ea.s.n);
}

__global__ void k_ens_mirror(EnsArgs ea)
{
    for (long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x; gi < ea.s.n;
         gi += (long long)gridDim.x * blockDim.x)
        ens_write_mirror(ea, gi);
}

// Phase A for the cluster of rank q: schedule, predict, compact, publish.
template <int NT, int MODE>
__device__ __forceinline__ void ens_a_cluster(const EnsArgs &ea, int q, long long *s_red, int *s_wtot)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const State &S = ea.s;
    const long long P = S.n;
    const int c = ea.order[q];
    const long long o = ea.off[c];
    const int n = (int)(ea.off[c + 1] - o);
    if (MODE == kEnsStep && ea.done[c]) return;
    long long tn = 0;
    if (MODE == kEnsStep) {
        long long mn = LLONG_MAX;
        for (int i = tid; i < n; i += NT)
            mn = min(mn, S.t[o + i] + (1LL << (kTickBits - S.lev[o + i])));
        tn = cta_reduce(mn, MinLL(), s_red);
        if (tn > ea.t_end) {
            if (tid == 0) ea.done[c] = 1;
            return;
        }
    }
    const bool split = n > kEnsPredChunk;  // prediction left to queue items
    int running = 0;
    for (int base = 0; base < n; base += NT) {
        const int i = base + tid;
        bool f = false;
        if (i < n && !split) {
            const long long gi = o + i;
            if (MODE == kEnsStep) {
                ens_predict_j32(ea, gi, tn);
            } else {
                // start-up and force-only passes: the stored state itself (dt = 0)
                float hi[3], lo[3];
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) split_ds(S.x[cc * P + gi], hi[cc], lo[cc]);
                ea.jph[gi] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(S.m[gi]));
                ea.jpl[gi] = make_float4(lo[0], lo[1], lo[2], 0.0f);
                ea.jv[gi] = make_float4(__double2float_rn(S.v[gi]), __double2float_rn(S.v[P + gi]),
                                        __double2float_rn(S.v[2 * P + gi]), 0.0f);
            }
        }
        if (i < n) {
            const long long gi = o + i;
            f = MODE == kEnsStep ? (S.t[gi] + (1LL << (kTickBits - S.lev[gi])) == tn) : true;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, f);
        if (lane == 0) s_wtot[warp] = __popc(bal);
        __syncthreads();
        int woff = 0, tot = 0;
        for (int w = 0; w < NT / 32; ++w) {
            woff += w < warp ? s_wtot[w] : 0;
            tot += s_wtot[w];
        }
        if (f) ea.act[o + running + woff + __popc(bal & ((1u << lane) - 1u))] = i;
        running += tot;
        __syncthreads();
    }
    // every thread's records and active indices are written before tid 0 publishes
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const int na = running;
        ea.na[c] = na;
        ea.tnext[c] = tn;
        if (MODE == kEnsStep) {
            ea.steps[c] += 1;
            ea.inter[c] += (long long)na * (n - 1);
        }
        const int npred = split ? (n + kEnsPredChunk - 1) / kEnsPredChunk : 0;
        const int nforce = (na + ea.chunk - 1) / ea.chunk;
        ea.pred_left[c] = npred;
        const int base = atomicAdd(ea.qlen, npred + nforce);
        for (int k = 0; k < npred; ++k) ea.qk[base + k] = -1 - k;  // ahead of the force items
        for (int k = 0; k < nforce; ++k) ea.qk[base + npred + k] = k;
        __threadfence();
        for (int k = 0; k < npred + nforce; ++k) atomicExch(&ea.qc[base + k], c);
    }
}

// Queue item `it` for phase B: true with (c, k) once it is published; false
// when there is no such item (every cluster's phase A finished and the queue
// is shorter) or the wait ran past its limit (error NB_ETIMEOUT).  Consuming
// an item marks it not ready again for the next launch.
constexpr long long kEnsSpinCycles = 4000000000LL;  // about 2 s at 2 GHz

__device__ __forceinline__ bool ens_take_item(const EnsArgs &ea, int it, int &c, int &k)
{
    // Every CTA takes one index past the last item before it stops, so indices
    // run up to (items + CTAs - 1): those at or past the capacity hold no item.
    if (it >= ea.qcap) return false;
    volatile int *qc = ea.qc;
    volatile int *adone = ea.a_done;
    volatile int *qlen = ea.qlen;
    const long long t0 = clock64();
    for (;;) {
        const int cc = qc[it];
        if (cc >= 0) {
            __threadfence();
            c = cc;
            k = __ldcg(&ea.qk[it]);
            qc[it] = -1;
            return true;
        }
        if (*adone >= ea.C) {
            __threadfence();
            if (it >= *qlen) return false;
            continue;  // published before the last cluster finished: visible next read
        }
        if (clock64() - t0 > kEnsSpinCycles) {
            atomicCAS(ea.err, 0, NB_ETIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
}

// Phase B, prediction item: particles [512 p, 512 (p + 1)) of cluster c to its
// block time; the last CTA to finish a cluster's chunks releases its force items.
template <int NT, int MODE>
__device__ __forceinline__ void ens_predict_chunk(const EnsArgs &ea, int c, int p)
{
    const int tid = threadIdx.x;
    const State &S = ea.s;
    const long long P = S.n;
    const long long o = ea.off[c];
    const int n = (int)(ea.off[c + 1] - o);
    const long long tn = __ldcg(&ea.tnext[c]);
    const int i1 = min(n, (p + 1) * kEnsPredChunk);
    for (int i = p * kEnsPredChunk + tid; i < i1; i += NT) {
        const long long gi = o + i;
        if (MODE == kEnsStep) {
            ens_predict_j32(ea, gi, tn);
        } else {
            float hi[3], lo[3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) split_ds(S.x[cc * P + gi], hi[cc], lo[cc]);
            ea.jph[gi] = make_float4(hi[0], hi[1], hi[2], __double2float_rn(S.m[gi]));
            ea.jpl[gi] = make_float4(lo[0], lo[1], lo[2], 0.0f);
            ea.jv[gi] = make_float4(__double2float_rn(S.v[gi]), __double2float_rn(S.v[P + gi]),
                                    __double2float_rn(S.v[2 * P + gi]), 0.0f);
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) atomicSub(&ea.pred_left[c], 1);
}

// Waits (thread 0) until cluster c's prediction chunks are done; false past
// the time limit (error NB_ETIMEOUT).  The chunks precede the cluster's force
// items in the queue, so CTAs already hold them and finish them without waiting.
__device__ __forceinline__ bool ens_wait_predicted(const EnsArgs &ea, int c)
{
    volatile int *left = ea.pred_left;
    const long long t0 = clock64();
    while (left[c] > 0) {
        if (clock64() - t0 > kEnsSpinCycles) {
            atomicCAS(ea.err, 0, NB_ETIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// Phase B, force item (c, k): force on one chunk of the cluster's block, then the
// correction (or the start-up levels, or plain output).
template <int NT, int MODE>
__device__ __forceinline__ void ens_b_item(const EnsArgs &ea, int c, int k, float4 *s_ph, float4 *s_pl,
                                           float4 *s_v, int *s_ok)
{
    const int tid = threadIdx.x;
    const State &S = ea.s;
    const long long P = S.n;
    const long long o = ea.off[c];
    const int n = (int)(ea.off[c + 1] - o);
    if (tid == 0) *s_ok = ens_wait_predicted(ea, c);
    __syncthreads();
    if (!*s_ok) return;
    // Everything phase A wrote in this launch is read past L1 (__ldcg): L1 is
    // not coherent across SMs, and a line read earlier for a neighbouring
    // cluster could hold this cluster's records from before they were written.
    const int s0 = k * ea.chunk;
    const int cnt = min(ea.chunk, __ldcg(&ea.na[c]) - s0);
    int g = 1;
    while (g < ea.gmax && g * 2 * cnt <= NT) g <<= 1;
    const int grp = tid / g, lig = tid % g;
    const bool valid = grp < cnt;
    const int i = __ldcg(&ea.act[o + s0 + (valid ? grp : 0)]);
    const float4 ip = __ldcg(&ea.jph[o + i]), il = __ldcg(&ea.jpl[o + i]), iv = __ldcg(&ea.jv[o + i]);
    const IDS I = make_ids(ip, il, iv);
    float hi[7] = {0, 0, 0, 0, 0, 0, 0}, lo[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int jt = 0; jt < n; jt += NT) {
        __syncthreads();
        const int j = jt + tid;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        s_ph[tid] = j < n ? __ldcg(&ea.jph[o + j]) : z;
        s_pl[tid] = j < n ? __ldcg(&ea.jpl[o + j]) : z;
        s_v[tid] = j < n ? __ldcg(&ea.jv[o + j]) : z;
        __syncthreads();
        const int jc = min(NT, n - jt);
        // FP32 partials over at most 64 pairs per lane, then TwoSum promotion
        for (int jb = 0; jb < jc; jb += 64 * g) {
            const int je = min(jc, jb + 64 * g);
            float ta[3] = {0, 0, 0}, tk[3] = {0, 0, 0}, tp = 0.0f;
            for (int jj = jb + lig; jj < je; jj += g)
                pair_ds_packed<false, true>(s_ph[jj], s_pl[jj], s_v[jj], I, ea.eps2, ta, tk, tp,
                                            jt + jj, i);
            const float t7[7] = {ta[0], ta[1], ta[2], tk[0], tk[1], tk[2], tp};
#pragma unroll
            for (int cc = 0; cc < 7; ++cc) two_sum_acc(hi[cc], lo[cc], t7[cc]);
        }
    }
    for (int sh = 1; sh < g; sh <<= 1) {
#pragma unroll
        for (int cc = 0; cc < 7; ++cc) {
            const float h2 = __shfl_xor_sync(0xffffffffu, hi[cc], sh);
            const float l2 = __shfl_xor_sync(0xffffffffu, lo[cc], sh);
            ds_add(hi[cc], lo[cc], h2, l2);
        }
    }
    double res[7];
#pragma unroll
    for (int cc = 0; cc < 7; ++cc) res[cc] = (double)hi[cc] + (double)lo[cc];
    const long long gi = o + i;
    if (MODE == kEnsStep && g >= 4) {
        // every lane of the group holds the sums: its first four lanes correct
        // the particle together (the same FP64 operations as one lane would);
        // the CTA's other lanes run along inactive, as the quads need
        const int qd = lig & 3, cq = qd < 3 ? qd : 2;
        const bool active = valid && lig < 4;
        const bool ok = correct_particle_quad(S, gi, P, __ldcg(&ea.tnext[c]), res[cq], res[3 + cq],
                                              ea.eta, ea.level_min, 0, active);
        __syncwarp();
        if (active && qd == 0) {
            if (!ok) atomicCAS(ea.err, 0, NB_ESTEP);
            ens_write_mirror(ea, gi);
        }
        return;
    }
    if (!valid || lig != 0) return;
    if (MODE == kEnsForce) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            ea.out_acc[3 * gi + cc] = res[cc];
            ea.out_jerk[3 * gi + cc] = res[3 + cc];
        }
        ea.out_pot[gi] = res[6];
        return;
    }
    if (MODE == kEnsInit) {
#pragma unroll
        for (int cc = 0; cc < 3; ++cc) {
            S.a[cc * P + gi] = res[cc];
            S.k[cc * P + gi] = res[3 + cc];
        }
        S.t[gi] = 0;
        int lv;
        if (!level_of(initial_dt(res, res + 3, ea.eta_init), ea.level_min, lv)) {
            atomicCAS(ea.err, 0, NB_ESTEP);
            lv = kTickBits;
        }
        S.lev[gi] = lv;
        return;
    }
    // corrector and new step (the single-system corrector's arithmetic)
    const double ap[3] = {res[0], res[1], res[2]}, kp[3] = {res[3], res[4], res[5]};
    if (!correct_particle(S, gi, P, __ldcg(&ea.tnext[c]), ap, kp, ea.eta, ea.level_min, 0))
        atomicCAS(ea.err, 0, NB_ESTEP);
    ens_write_mirror(ea, gi);
}

// One ensemble block step (or start-up, or force-only pass): phase A over the
// clusters, then phase B over the queue.
template <int NT, int MODE>
__global__ void __launch_bounds__(NT) k_ens_step(EnsArgs ea)
{
    __shared__ long long s_red[NT / 32];
    __shared__ int s_wtot[NT / 32];
    __shared__ float4 s_ph[NT], s_pl[NT], s_v[NT];
    __shared__ int s_q, s_c, s_k, s_ok;
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) s_q = atomicAdd(ea.work, 1);
        __syncthreads();
        const int q = s_q;
        __syncthreads();
        if (q >= ea.C) break;
        ens_a_cluster<NT, MODE>(ea, q, s_red, s_wtot);
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            atomicAdd(ea.a_done, 1);
        }
    }
    for (;;) {
        if (tid == 0) {
            int c = -1, k = 0;
            const int it = atomicAdd(ea.work_b, 1);
            if (!ens_take_item(ea, it, c, k)) c = -1;
            s_c = c;
            s_k = k;
        }
        __syncthreads();
        const int c = s_c, k = s_k;
        __syncthreads();
        if (c < 0) break;
        if (k < 0)
            ens_predict_chunk<NT, MODE>(ea, c, -1 - k);
        else
            ens_b_item<NT, MODE>(ea, c, k, s_ph, s_pl, s_v, &s_ok);
    }
}

// Energy of every cluster at its particles' own times (exact when the cluster
// is synchronised): kinetic from FP64 velocities, potential as the FP64 pair
// sum -sum_{i<j} m_i m_j / sqrt(r^2 + eps^2), per cluster in a fixed order.
template <int NT>
__global__ void __launch_bounds__(NT) k_ens_energy(EnsArgs ea, double eps2, double *ekin, double *epot)
{
    __shared__ double s_red[NT / 32];
    const int tid = threadIdx.x;
    const State &S = ea.s;
    const long long P = S.n;
    for (int c = blockIdx.x; c < ea.C; c += gridDim.x) {
        const long long o = ea.off[c];
        const int n = (int)(ea.off[c + 1] - o);
        double ke = 0.0, pe = 0.0;
        for (int i = tid; i < n; i += NT) {
            const long long gi = o + i;
            const double vx = S.v[gi], vy = S.v[P + gi], vz = S.v[2 * P + gi];
            ke += 0.5 * S.m[gi] * (vx * vx + vy * vy + vz * vz);
            const double xi = S.x[gi], yi = S.x[P + gi], zi = S.x[2 * P + gi];
            double row = 0.0;
            for (int j = i + 1; j < n; ++j) {
                const long long gj = o + j;
                const double dx = S.x[gj] - xi, dy = S.x[P + gj] - yi, dz = S.x[2 * P + gj] - zi;
                row += S.m[gj] / sqrt(dx * dx + dy * dy + dz * dz + eps2);
            }
            pe -= S.m[gi] * row;
        }
        struct Add {
            __device__ double operator()(double a, double b) const { return a + b; }
        };
        ke = cta_reduce(ke, Add(), s_red);
        pe = cta_reduce(pe, Add(), s_red);
        if (tid == 0) {
            ekin[c] = ke;
            epot[c] = pe;
        }
    }
}

// host AoS [P][3] -> device SoA staging -> state arrays
__global__ void k_aos_to_soa(const double *aos, double *soa, long long P)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * P;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / 3, c = e % 3;
        soa[c * P + i] = aos[e];
    }
}

__global__ void k_soa_to_aos(const double *soa, double *aos, long long P)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < 3 * P;
         e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / 3, c = e % 3;
        aos[e] = soa[c * P + i];
    }
}

}  // namespace
}  // namespace nbk

using namespace nbk;

// ---------------------------------------------------------------------------
// Host side: the nb_ens context and its C ABI.

struct nb_ens {
    int C = 0;
    long long P = 0;
    double eps = 0.0;
    nb_opts o{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int sms = 0;
    State S{};
    long long *d_off = nullptr;
    int *d_order = nullptr;
    double *d_x = nullptr, *d_v = nullptr, *d_a = nullptr, *d_k = nullptr, *d_m = nullptr;
    long long *d_t = nullptr;
    int *d_lev = nullptr;
    int *d_work = nullptr, *d_done = nullptr, *d_err = nullptr;  // d_work: [4] counters A, B, queue, A done
    float4 *d_jph = nullptr, *d_jpl = nullptr, *d_jv = nullptr;
    float4 *d_mirror = nullptr;  // [5 P]: x_hi + m, x_lo, v, a, k in single precision
    int *d_act = nullptr, *d_na = nullptr, *d_qc = nullptr, *d_qk = nullptr, *d_pred = nullptr;
    long long *d_tnext = nullptr;
    long long qcap = 0;
    long long *d_steps = nullptr, *d_inter = nullptr;
    double *d_stage = nullptr;   // [7 P] host I/O staging
    double *d_backup = nullptr;  // state copy for tuning
    long long *d_tbak = nullptr;
    int *d_lbak = nullptr;
    int nt = 256, gmax = 8;      // threads per CTA and lane-group cap (tunable); items of nt / gmax
    long long t_end = LLONG_MAX;
    cudaGraphExec_t graph = nullptr;
    int graph_nt = 0, graph_gmax = 0;
    long long graph_tend = -1;
    long long launches = 0;
    std::string err;
};

namespace ens_impl {

thread_local std::string g_ens_init_err;

// An NVTX range over one entry point (no cost unless a tool is attached).
struct EnsRange {
    explicit EnsRange(const char *name) { nvtxRangePushA(name); }
    ~EnsRange() { nvtxRangePop(); }
};

int efail(nb_ens *e, int code, const char *fmt, ...)
{
    if (e) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        e->err = buf;
    }
    return code;
}

#define ECK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return efail(e, e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA,       \
                         "%s: %s", #call, cudaGetErrorString(e_));                        \
    } while (0)

EnsArgs ens_args(nb_ens *e)
{
    EnsArgs a{};
    a.C = e->C;
    a.off = e->d_off;
    a.order = e->d_order;
    a.s = e->S;
    a.eps2 = (float)(e->eps * e->eps);
    a.eta = e->o.eta;
    a.eta_init = e->o.eta_init;
    a.level_min = e->o.level_min;
    a.t_end = e->t_end;
    a.gmax = e->gmax;
    a.chunk = e->nt / e->gmax;  // every full item uses gmax lanes per particle
    a.work = e->d_work;
    a.work_b = e->d_work + 1;
    a.qlen = e->d_work + 2;
    a.a_done = e->d_work + 3;
    a.pred_left = e->d_pred;
    a.qc = e->d_qc;
    a.qcap = (int)(e->P + e->C);
    a.qk = e->d_qk;
    a.jph = e->d_jph;
    a.jpl = e->d_jpl;
    a.jv = e->d_jv;
    a.mir.h = e->d_mirror;
    a.mir.l = e->d_mirror + e->P;
    a.mir.v = e->d_mirror + 2 * e->P;
    a.mir.a = e->d_mirror + 3 * e->P;
    a.mir.k = e->d_mirror + 4 * e->P;
    a.act = e->d_act;
    a.na = e->d_na;
    a.tnext = e->d_tnext;
    a.done = e->d_done;
    a.steps = e->d_steps;
    a.inter = e->d_inter;
    a.err = e->d_err;
    return a;
}

// Resident CTAs per SM of the fused kernel for this configuration.
template <int NT, int MODE>
int ens_blocks_per_sm()
{
    static int bps = 0;
    if (bps == 0 &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_ens_step<NT, MODE>, NT, 0) != cudaSuccess)
        bps = 1;
    return bps > 0 ? bps : 1;
}

// One cooperative launch over all resident CTAs (CTAs wait on each other's
// phase A, so they must all be resident).
template <int NT, int MODE>
cudaError_t launch_step_t(nb_ens *e, const EnsArgs &a)
{
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.gridDim = dim3(e->sms * ens_blocks_per_sm<NT, MODE>());
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = e->st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_ens_step<NT, MODE>, a);
}

// One pass: counters zeroed, then the fused launch.
template <int MODE>
int enqueue_ens(nb_ens *e, const EnsArgs &a)
{
    ECK(cudaMemsetAsync(e->d_work, 0, 4 * sizeof(int), e->st));
    cudaError_t ce;
    switch (e->nt) {
    case 128: ce = launch_step_t<128, MODE>(e, a); break;
    case 512: ce = launch_step_t<512, MODE>(e, a); break;
    default: ce = launch_step_t<256, MODE>(e, a); break;
    }
    if (ce != cudaSuccess) return efail(e, NB_ECUDA, "ensemble launch: %s", cudaGetErrorString(ce));
    e->launches += 1;
    return NB_OK;
}

// One ensemble block step.
int enqueue_ens_step(nb_ens *e) { return enqueue_ens<kEnsStep>(e, ens_args(e)); }

// Refreshes the single-precision mirror after the FP64 state was set from outside a step.
int enqueue_mirror(nb_ens *e)
{
    k_ens_mirror<<<(int)std::min<long long>(8LL * e->sms, (e->P + 255) / 256), 256, 0, e->st>>>(
        ens_args(e));
    ECK(cudaGetLastError());
    e->launches += 1;
    return NB_OK;
}

int ens_sync(nb_ens *e)
{
    int h_err = 0;
    ECK(cudaMemcpyAsync(&h_err, e->d_err, sizeof(int), cudaMemcpyDeviceToHost, e->st));
    ECK(cudaStreamSynchronize(e->st));
    ECK(cudaGetLastError());
    if (h_err) {
        // an aborted launch may leave items unconsumed: mark every item not ready
        ECK(cudaMemsetAsync(e->d_qc, 0xff, sizeof(int) * (e->P + e->C), e->st));
        ECK(cudaMemsetAsync(e->d_err, 0, sizeof(int), e->st));
        ECK(cudaStreamSynchronize(e->st));
        if (h_err == NB_ETIMEOUT)
            return efail(e, NB_ETIMEOUT, "an ensemble launch waited too long for a cluster's block");
        return efail(e, h_err, "a new time step fell below 2^-40 in some cluster");
    }
    return NB_OK;
}

template <typename T>
int ealloc(nb_ens *e, T **p, long long count)
{
    if (count < 1) count = 1;
    if (cudaMalloc((void **)p, sizeof(T) * (size_t)count) != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return efail(e, NB_ENOMEM, "cudaMalloc of %lld bytes failed", (long long)(sizeof(T) * count));
    }
    return NB_OK;
}

void ens_release(nb_ens *e)
{
    if (e->st) cudaStreamSynchronize(e->st);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    void *ptrs[] = {e->d_off, e->d_order, e->d_x, e->d_v, e->d_a, e->d_k, e->d_m, e->d_t,
                    e->d_lev, e->d_work, e->d_done, e->d_err, e->d_steps, e->d_inter,
                    e->d_stage, e->d_backup, e->d_tbak, e->d_lbak, e->d_jph, e->d_jpl, e->d_jv,
                    e->d_mirror,
                    e->d_act, e->d_na, e->d_qc, e->d_qk, e->d_tnext, e->d_pred};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (e->own_stream && e->st) cudaStreamDestroy(e->st);
}

bool finite_all(const double *p, long long cnt)
{
    for (long long i = 0; i < cnt; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

int grid_of(long long n) { return (int)std::min<long long>(4096, std::max<long long>(1, (n + 255) / 256)); }

int ens_init_impl(nb_ens *e, int32_t C, const int64_t *off, const double *m, const double *x,
                  const double *v, double eps, const nb_opts *opts)
{
    nb_opts o;
    nb_default_opts(&o);
    if (opts) o = *opts;
    if (C < 1 || !off || !m || !x || !v) return efail(e, NB_EINVAL, "bad arguments");
    if (!std::isfinite(eps) || eps < 0.0) return efail(e, NB_EINVAL, "eps must be finite and >= 0");
    if (o.level_min < 0 || o.level_min > kTickBits || o.level_fixed != 0 || o.precision != NB_DS)
        return efail(e, NB_EINVAL, "ensembles use DS precision and individual block steps");
    if (o.summation != NB_SUM_COMPENSATED)
        return efail(e, NB_EINVAL, "ensembles use the compensated summation");
    if (!(o.eta > 0.0) || !(o.eta_init > 0.0)) return efail(e, NB_EINVAL, "eta must be positive");
    if (off[0] != 0) return efail(e, NB_EINVAL, "offsets must start at 0");
    std::vector<std::pair<long long, int>> sizes;
    for (int c = 0; c < C; ++c) {
        const long long nc = off[c + 1] - off[c];
        if (nc < 1 || nc > kEnsMaxN)
            return efail(e, NB_EINVAL, "cluster %d has %lld particles (1..%d allowed)", c, nc, kEnsMaxN);
        sizes.push_back({-nc, c});
    }
    const long long P = off[C];
    if (P > INT_MAX / 8) return efail(e, NB_EINVAL, "too many particles");
    if (!finite_all(m, P) || !finite_all(x, 3 * P) || !finite_all(v, 3 * P))
        return efail(e, NB_EINVAL, "non-finite input");
    for (long long i = 0; i < P; ++i)
        if (m[i] < 0.0) return efail(e, NB_EINVAL, "negative mass");
    std::stable_sort(sizes.begin(), sizes.end());
    std::vector<int> order(C);
    for (int q = 0; q < C; ++q) order[q] = sizes[q].second;

    e->C = C;
    e->P = P;
    e->eps = eps;
    e->o = o;
    if (o.stream) {
        e->st = (cudaStream_t)o.stream;
    } else {
        ECK(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking));
        e->own_stream = true;
    }
    int dev = 0;
    ECK(cudaGetDevice(&dev));
    ECK(cudaDeviceGetAttribute(&e->sms, cudaDevAttrMultiProcessorCount, dev));
    int rc;
    if ((rc = ealloc(e, &e->d_off, C + 1)) || (rc = ealloc(e, &e->d_order, C)) ||
        (rc = ealloc(e, &e->d_x, 3 * P)) || (rc = ealloc(e, &e->d_v, 3 * P)) ||
        (rc = ealloc(e, &e->d_a, 3 * P)) || (rc = ealloc(e, &e->d_k, 3 * P)) ||
        (rc = ealloc(e, &e->d_m, P)) || (rc = ealloc(e, &e->d_t, P)) || (rc = ealloc(e, &e->d_lev, P)) ||
        (rc = ealloc(e, &e->d_work, 4)) || (rc = ealloc(e, &e->d_done, C)) || (rc = ealloc(e, &e->d_err, 1)) ||
        (rc = ealloc(e, &e->d_steps, C)) || (rc = ealloc(e, &e->d_inter, C)) ||
        (rc = ealloc(e, &e->d_stage, 7 * P)) || (rc = ealloc(e, &e->d_jph, P)) ||
        (rc = ealloc(e, &e->d_jpl, P)) || (rc = ealloc(e, &e->d_jv, P)) ||
        (rc = ealloc(e, &e->d_act, P)) || (rc = ealloc(e, &e->d_na, C)) ||
        (rc = ealloc(e, &e->d_tnext, C)) || (rc = ealloc(e, &e->d_qc, P + C)) ||
        (rc = ealloc(e, &e->d_qk, P + C)) || (rc = ealloc(e, &e->d_pred, C)) ||
        (rc = ealloc(e, &e->d_mirror, 5 * P)))
        return rc;
    e->S.x = e->d_x;
    e->S.v = e->d_v;
    e->S.a = e->d_a;
    e->S.k = e->d_k;
    e->S.m = e->d_m;
    e->S.t = e->d_t;
    e->S.lev = e->d_lev;
    e->S.n = (int)P;
    ECK(cudaMemcpyAsync(e->d_off, off, sizeof(long long) * (C + 1), cudaMemcpyHostToDevice, e->st));
    ECK(cudaMemcpyAsync(e->d_order, order.data(), sizeof(int) * C, cudaMemcpyHostToDevice, e->st));
    ECK(cudaMemcpyAsync(e->d_m, m, sizeof(double) * P, cudaMemcpyHostToDevice, e->st));
    ECK(cudaMemcpyAsync(e->d_stage, x, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, e->st));
    k_aos_to_soa<<<grid_of(3 * P), 256, 0, e->st>>>(e->d_stage, e->d_x, P);
    ECK(cudaStreamSynchronize(e->st));
    ECK(cudaMemcpyAsync(e->d_stage, v, sizeof(double) * 3 * P, cudaMemcpyHostToDevice, e->st));
    k_aos_to_soa<<<grid_of(3 * P), 256, 0, e->st>>>(e->d_stage, e->d_v, P);
    ECK(cudaMemsetAsync(e->d_a, 0, sizeof(double) * 3 * P, e->st));
    ECK(cudaMemsetAsync(e->d_k, 0, sizeof(double) * 3 * P, e->st));
    ECK(cudaMemsetAsync(e->d_t, 0, sizeof(long long) * P, e->st));
    ECK(cudaMemsetAsync(e->d_done, 0, sizeof(int) * C, e->st));
    ECK(cudaMemsetAsync(e->d_err, 0, sizeof(int), e->st));
    ECK(cudaMemsetAsync(e->d_steps, 0, sizeof(long long) * C, e->st));
    ECK(cudaMemsetAsync(e->d_inter, 0, sizeof(long long) * C, e->st));
    ECK(cudaMemsetAsync(e->d_qc, 0xff, sizeof(int) * (P + C), e->st));  // no item ready
    ECK(cudaMemsetAsync(e->d_pred, 0, sizeof(int) * C, e->st));
    // start-up: force on every particle of every cluster, initial steps
    if ((rc = enqueue_ens<kEnsInit>(e, ens_args(e)))) return rc;
    ECK(cudaGetLastError());
    if ((rc = enqueue_mirror(e))) return rc;
    return ens_sync(e);
}

}  // namespace ens_impl

using namespace ens_impl;

extern "C" {

int nb_ens_init(nb_ens **ens, int32_t n_clusters, const int64_t *offsets, const double *m,
                const double *x, const double *v, double eps, const nb_opts *opts)
{
    const EnsRange range_("nb_ens_init");
    g_ens_init_err.clear();
    if (!ens) return NB_EINVAL;
    *ens = nullptr;
    nb_ens *e = new (std::nothrow) nb_ens();
    if (!e) return NB_ENOMEM;
    const int rc = ens_init_impl(e, n_clusters, offsets, m, x, v, eps, opts);
    if (rc != NB_OK) {
        g_ens_init_err = e->err;
        ens_release(e);
        delete e;
        return rc;
    }
    *ens = e;
    return NB_OK;
}

void nb_ens_free(nb_ens *e)
{
    if (!e) return;
    ens_release(e);
    delete e;
}

const char *nb_ens_last_error(const nb_ens *e)
{
    if (e) return e->err.c_str();
    return g_ens_init_err.empty() ? "null ensemble" : g_ens_init_err.c_str();
}

int nb_ens_configure(nb_ens *e, int threads, int gmax)
{
    if (!e) return NB_EINVAL;
    if ((threads != 128 && threads != 256 && threads != 512) ||
        (gmax != 1 && gmax != 2 && gmax != 4 && gmax != 8 && gmax != 16 && gmax != 32))
        return efail(e, NB_EINVAL, "threads in {128, 256, 512}, gmax a power of two <= 32");
    e->nt = threads;
    e->gmax = gmax;
    return NB_OK;
}

int nb_ens_run(nb_ens *e, double t_end, int64_t max_launches, int64_t *launches_out,
               int64_t *interactions_out)
{
    const EnsRange range_("nb_ens_run");
    if (!e) return NB_EINVAL;
    if (!std::isfinite(t_end) || t_end < 0.0 || t_end >= 0x1p22 || t_end * 0x1p40 != std::floor(t_end * 0x1p40))
        return efail(e, NB_EINVAL, "t_end is not on the 2^-40 grid");
    if (max_launches < 0) return efail(e, NB_EINVAL, "max_launches < 0");
    const long long te = (long long)(t_end * 0x1p40);
    if (te != e->t_end) {
        // a new end time re-opens finished clusters
        ECK(cudaMemsetAsync(e->d_done, 0, sizeof(int) * e->C, e->st));
        e->t_end = te;
    }
    // capture one ensemble step (memset + persistent launch) into a graph
    if (!e->graph || e->graph_nt != e->nt || e->graph_gmax != e->gmax || e->graph_tend != te) {
        if (e->graph) cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
        int rc0 = 0;
        // a first launch of this configuration outside capture (occupancy query)
        EnsArgs probe = ens_args(e);
        probe.C = 0;
        if ((rc0 = enqueue_ens<kEnsStep>(e, probe))) return rc0;
        ECK(cudaStreamSynchronize(e->st));
        cudaGraph_t g;
        ECK(cudaStreamBeginCapture(e->st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = e->launches;
        const int rc = enqueue_ens_step(e);
        e->launches = l0;
        cudaError_t ce = cudaStreamEndCapture(e->st, &g);
        if (rc) return rc;
        if (ce != cudaSuccess) return efail(e, NB_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&e->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            e->graph = nullptr;
            return efail(e, NB_ECUDA, "graph instantiate: %s", cudaGetErrorString(ce));
        }
        e->graph_nt = e->nt;
        e->graph_gmax = e->gmax;
        e->graph_tend = te;
    }
    std::vector<int> done(e->C);
    long long n = 0;
    std::vector<long long> inter0(e->C), inter1(e->C);
    ECK(cudaMemcpyAsync(inter0.data(), e->d_inter, sizeof(long long) * e->C, cudaMemcpyDeviceToHost, e->st));
    while (n < max_launches) {
        const long long k = std::min<long long>(32, max_launches - n);
        for (long long q = 0; q < k; ++q) ECK(cudaGraphLaunch(e->graph, e->st));
        n += k;
        e->launches += k;
        ECK(cudaMemcpyAsync(done.data(), e->d_done, sizeof(int) * e->C, cudaMemcpyDeviceToHost, e->st));
        int rc = ens_sync(e);
        if (rc) return rc;
        bool all = true;
        for (int c = 0; c < e->C && all; ++c) all = done[c] != 0;
        if (all) break;
    }
    ECK(cudaMemcpyAsync(inter1.data(), e->d_inter, sizeof(long long) * e->C, cudaMemcpyDeviceToHost, e->st));
    ECK(cudaStreamSynchronize(e->st));
    long long it = 0;
    for (int c = 0; c < e->C; ++c) it += inter1[c] - inter0[c];
    if (launches_out) *launches_out = n;
    if (interactions_out) *interactions_out = it;
    return NB_OK;
}

int nb_ens_tune(nb_ens *e, int launches_per_candidate, int *threads_out, int *gmax_out,
                double *ms_out)
{
    const EnsRange range_("nb_ens_tune");
    if (!e) return NB_EINVAL;
    if (launches_per_candidate < 1) return efail(e, NB_EINVAL, "launches_per_candidate < 1");
    const long long P = e->P, C = e->C;
    int rc;
    if (!e->d_backup && ((rc = ealloc(e, &e->d_backup, 12 * P + 2 * C)) ||
                         (rc = ealloc(e, &e->d_tbak, P)) || (rc = ealloc(e, &e->d_lbak, P + C))))
        return rc;
    // snapshot: x, v, a, k, times, levels, per-cluster counters and flags
    double *arrs[4] = {e->d_x, e->d_v, e->d_a, e->d_k};
    auto save = [&](bool restore) -> int {
        for (int q = 0; q < 4; ++q) {
            double *b = e->d_backup + q * 3 * P;
            ECK(cudaMemcpyAsync(restore ? arrs[q] : b, restore ? b : arrs[q], sizeof(double) * 3 * P,
                                cudaMemcpyDeviceToDevice, e->st));
        }
        long long *cb = (long long *)(e->d_backup + 12 * P);
        ECK(cudaMemcpyAsync(restore ? e->d_t : e->d_tbak, restore ? e->d_tbak : e->d_t,
                            sizeof(long long) * P, cudaMemcpyDeviceToDevice, e->st));
        ECK(cudaMemcpyAsync(restore ? e->d_lev : e->d_lbak, restore ? e->d_lbak : e->d_lev,
                            sizeof(int) * P, cudaMemcpyDeviceToDevice, e->st));
        ECK(cudaMemcpyAsync(restore ? e->d_done : e->d_lbak + P, restore ? e->d_lbak + P : e->d_done,
                            sizeof(int) * C, cudaMemcpyDeviceToDevice, e->st));
        ECK(cudaMemcpyAsync(restore ? e->d_steps : cb, restore ? cb : e->d_steps,
                            sizeof(long long) * C, cudaMemcpyDeviceToDevice, e->st));
        ECK(cudaMemcpyAsync(restore ? e->d_inter : cb + C, restore ? cb + C : e->d_inter,
                            sizeof(long long) * C, cudaMemcpyDeviceToDevice, e->st));
        return restore ? enqueue_mirror(e) : NB_OK;
    };
    if ((rc = save(false))) return rc;
    cudaEvent_t e0, e1;
    ECK(cudaEventCreate(&e0));
    ECK(cudaEventCreate(&e1));
    const int cand_nt[3] = {128, 256, 512};
    const int cand_g[6] = {1, 2, 4, 8, 16, 32};
    float best = 1e30f;
    int bnt = e->nt, bg = e->gmax;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 6; ++b) {
            e->nt = cand_nt[a];
            e->gmax = cand_g[b];
            if ((rc = save(true))) return rc;
            if ((rc = enqueue_ens_step(e))) return rc;  // warm-up (and shared-memory set-up)
            ECK(cudaEventRecord(e0, e->st));
            for (int q = 0; q < launches_per_candidate; ++q)
                if ((rc = enqueue_ens_step(e))) return rc;
            ECK(cudaEventRecord(e1, e->st));
            if ((rc = ens_sync(e))) return rc;
            float ms = 0.0f;
            ECK(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bnt = e->nt;
                bg = e->gmax;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if ((rc = save(true))) return rc;
    ECK(cudaStreamSynchronize(e->st));
    e->nt = bnt;
    e->gmax = bg;
    if (threads_out) *threads_out = bnt;
    if (gmax_out) *gmax_out = bg;
    if (ms_out) *ms_out = best / launches_per_candidate;
    return NB_OK;
}

int nb_ens_step(nb_ens *e)
{
    const EnsRange range_("nb_ens_step");
    if (!e) return NB_EINVAL;
    int rc = enqueue_ens_step(e);
    if (rc) return rc;
    return ens_sync(e);
}

int nb_ens_force(nb_ens *e, double *acc, double *jerk, double *pot)
{
    const EnsRange range_("nb_ens_force");
    if (!e) return NB_EINVAL;
    const long long P = e->P;
    EnsArgs a = ens_args(e);
    a.out_acc = e->d_stage;
    a.out_jerk = e->d_stage + 3 * P;
    a.out_pot = e->d_stage + 6 * P;
    int rc = enqueue_ens<kEnsForce>(e, a);
    if (rc) return rc;
    if (acc) ECK(cudaMemcpyAsync(acc, a.out_acc, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, e->st));
    if (jerk) ECK(cudaMemcpyAsync(jerk, a.out_jerk, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, e->st));
    if (pot) ECK(cudaMemcpyAsync(pot, a.out_pot, sizeof(double) * P, cudaMemcpyDeviceToHost, e->st));
    return ens_sync(e);
}

int nb_ens_energy(nb_ens *e, double *ekin, double *epot)
{
    const EnsRange range_("nb_ens_energy");
    if (!e) return NB_EINVAL;
    double *d = e->d_stage;
    k_ens_energy<256><<<std::max(1, std::min(e->C, 8 * e->sms)), 256, 0, e->st>>>(
        ens_args(e), e->eps * e->eps, d, d + e->C);
    e->launches += 1;
    if (ekin) ECK(cudaMemcpyAsync(ekin, d, sizeof(double) * e->C, cudaMemcpyDeviceToHost, e->st));
    if (epot) ECK(cudaMemcpyAsync(epot, d + e->C, sizeof(double) * e->C, cudaMemcpyDeviceToHost, e->st));
    return ens_sync(e);
}

int nb_ens_get_state(nb_ens *e, double *x, double *v, double *a, double *k, int64_t *t,
                     int32_t *level, int64_t *steps, int64_t *interactions)
{
    if (!e) return NB_EINVAL;
    const long long P = e->P;
    double *src[4] = {e->d_x, e->d_v, e->d_a, e->d_k};
    double *dst[4] = {x, v, a, k};
    for (int q = 0; q < 4; ++q) {
        if (!dst[q]) continue;
        k_soa_to_aos<<<grid_of(3 * P), 256, 0, e->st>>>(src[q], e->d_stage, P);
        ECK(cudaMemcpyAsync(dst[q], e->d_stage, sizeof(double) * 3 * P, cudaMemcpyDeviceToHost, e->st));
        ECK(cudaStreamSynchronize(e->st));
    }
    if (t) ECK(cudaMemcpyAsync(t, e->d_t, sizeof(long long) * P, cudaMemcpyDeviceToHost, e->st));
    if (level) ECK(cudaMemcpyAsync(level, e->d_lev, sizeof(int) * P, cudaMemcpyDeviceToHost, e->st));
    if (steps) ECK(cudaMemcpyAsync(steps, e->d_steps, sizeof(long long) * e->C, cudaMemcpyDeviceToHost, e->st));
    if (interactions)
        ECK(cudaMemcpyAsync(interactions, e->d_inter, sizeof(long long) * e->C, cudaMemcpyDeviceToHost, e->st));
    return ens_sync(e);
}

int nb_ens_set_state(nb_ens *e, const double *x, const double *v, const double *a, const double *k,
                     const int64_t *t, const int32_t *level)
{
    if (!e) return NB_EINVAL;
    if (!x || !v || !a || !k || !t || !level) return efail(e, NB_EINVAL, "all arrays are required");
    const long long P = e->P;
    if (!finite_all(x, 3 * P) || !finite_all(v, 3 * P) || !finite_all(a, 3 * P) || !finite_all(k, 3 * P))
        return efail(e, NB_EINVAL, "non-finite state");
    for (long long i = 0; i < P; ++i) {
        if (level[i] < e->o.level_min || level[i] > kTickBits) return efail(e, NB_EINVAL, "bad level");
        if (t[i] < 0 || t[i] % (1LL << (kTickBits - level[i])) != 0)
            return efail(e, NB_EINVAL, "time not a multiple of its step");
    }
    const double *src[4] = {x, v, a, k};
    double *dst[4] = {e->d_x, e->d_v, e->d_a, e->d_k};
    for (int q = 0; q < 4; ++q) {
        ECK(cudaMemcpyAsync(e->d_stage, src[q], sizeof(double) * 3 * P, cudaMemcpyHostToDevice, e->st));
        k_aos_to_soa<<<grid_of(3 * P), 256, 0, e->st>>>(e->d_stage, dst[q], P);
        ECK(cudaStreamSynchronize(e->st));
    }
    ECK(cudaMemcpyAsync(e->d_t, t, sizeof(long long) * P, cudaMemcpyHostToDevice, e->st));
    ECK(cudaMemcpyAsync(e->d_lev, level, sizeof(int) * P, cudaMemcpyHostToDevice, e->st));
    ECK(cudaMemsetAsync(e->d_done, 0, sizeof(int) * e->C, e->st));
    int rc = enqueue_mirror(e);
    if (rc) return rc;
    return ens_sync(e);
}

}  // extern "C"
