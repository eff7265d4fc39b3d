// nb_internal.cuh -- device data layout, control block and launchers shared by
// the CUDA translation units of the library (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nb.h"

namespace nbk {

constexpr int kTickBits = 40;

// Device-resident control block.  Every kernel of a block step reads its
// block time and block size from here, so a whole step can be replayed from a
// CUDA graph with no host round trip.
struct Ctrl {
    long long t_now;         // system time: block time of the last step (ticks)
    long long t_next;        // block time chosen by the scheduler (ticks)
    long long t_end;         // steps stop once the next block time would pass this
    long long steps;         // block steps taken
    long long interactions;  // sum over steps of n_active * (n - 1)
    double ekin, epot;       // last energy reduction
    int n_active;            // size of the current block; 0 = nothing to do
    int err;                 // first NB_* error raised by a kernel (0 = none)
    int err_where;           // which check raised it (for messages)
    int pad;
};

// FP64 master state, structure of arrays: x[c * n + i] for component c.
struct State {
    double *x, *v, *a, *k;   // position, velocity, acceleration, jerk
    const double *m;         // masses
    long long *t;            // particle times in ticks
    int *lev;                // block levels: dt_i = 2^-lev
    int n;
};

// j-particle records written by the predictor.
//  DS:   pos_hi = (x_hi, y_hi, z_hi, m), pos_lo = (x_lo, y_lo, z_lo, 0),
//        vel = (vx, vy, vz, 0) with x = x_hi + x_lo to 2^-48 relative.
//  FP64: pos = (x, y, z, m), vel = (vx, vy, vz, 0).
struct JDS {
    float4 *pos_hi, *pos_lo, *vel;
};
struct JF64 {
    double4_32a *pos, *vel;
};

// Force results in the public layout: acc[a][3], jerk[a][3], pot[a].
struct ForceOut {
    double *acc, *jerk, *pot;
};

// ---------------------------------------------------------------------------
// Work decomposition.  The same functions run on the host (to size buffers and
// grids) and on the device (where n_active is only known there).

#ifndef NB_IPAR_NT
#define NB_IPAR_NT 64
#endif
#ifndef NB_IPAR_R
#define NB_IPAR_R 4
#endif
#ifndef NB_IPAR_UNROLL
#define NB_IPAR_UNROLL 4
#endif

constexpr int kIparNT = NB_IPAR_NT;  // threads per CTA (= j per tile), i-parallel kernels
constexpr int kIparR = NB_IPAR_R;    // i per thread, DS i-parallel kernel
constexpr int kIparUnroll = NB_IPAR_UNROLL;  // j unrolling of the DS inner loop
#ifndef NB_IPAR_TILE_MULT
#define NB_IPAR_TILE_MULT 2
#endif
constexpr int kIparTileMult = NB_IPAR_TILE_MULT;  // DS i-parallel: j per tile = threads x this
constexpr int kIparR64 = 1;    // i per thread, FP64 i-parallel kernel
constexpr int kJparNT = 256;   // threads per CTA, j-parallel kernels
constexpr int kJparIC = 4;     // i per pass, j-parallel kernels
constexpr int kJparIC1Max = 2;  // DS j-parallel kernel: one i per pass up to this block size
constexpr int kJparMaxActive = 96;     // automatic mode, DS: j-parallel up to this block size
constexpr int kJparMaxActive64 = 32;   // automatic mode, FP64
constexpr int kIparSmallR = 1;      // i per thread of the small-block DS i-parallel kernel
constexpr int kSmallMaxActive = 1024;  // automatic mode: small-block kernel considered up to this size
constexpr int kComp = 7;       // acc xyz, jerk xyz, pot

struct Plan {
    int n_iblk;   // i-blocks (i-parallel) or i-chunks (j-parallel)
    int S;        // j slices of a sliced i-block
    int jslice;   // j per slice (multiple of the tile)
    int items;    // work items: n_whole + (n_iblk - n_whole) * S
    int n_whole;  // i-parallel: leading i-blocks taken whole (all j in one item, result
                  // written directly); the others are sliced.  0 for uniform plans.
    int a0;       // first block position of the sliced i-blocks (n_whole * i-block size)
};

__host__ __device__ inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// i-parallel: CTAs own iblk consecutive active particles and one j slice.
// The slice count S starts at s0 = 1, or, with fewer than two i-blocks per
// resident CTA, at the count that makes two; then among a few candidates
// (s0 .. s0 + 7 and the counts that fill 1 .. 8 waves of the slots resident
// CTAs exactly) the smallest whose last wave is at least 95% full is taken,
// else the one with the fullest last wave.  Slices keep at least two tiles and
// the partials fit in part_cap doubles.  Integer arithmetic only, computed
// once per force launch (host or scheduler, see ForcePlan).
// Every quotient in the slice search has operands below 2^31 (item counts are
// at most 8 slots + 8 i-blocks), so it uses 32-bit unsigned divisions, which
// cost a fraction of the 64-bit ones.
__host__ __device__ inline unsigned udiv(unsigned a, unsigned b) { return a / b; }
__host__ __device__ inline unsigned ucdiv(unsigned a, unsigned b) { return (a + b - 1) / b; }

__host__ __device__ inline bool better_fill(unsigned items_a, unsigned slots, unsigned items_b)
{
    // fill(x) = x / (ceil(x / slots) * slots); compare fill(a) > fill(b)
    const unsigned long long wa = ucdiv(items_a, slots), wb = ucdiv(items_b, slots);
    return items_a * wb > items_b * wa;
}

__host__ __device__ inline bool fill_ok(unsigned items, unsigned slots)
{
    const unsigned long long w = ucdiv(items, slots);
    return 20ULL * items >= 19ULL * w * slots;
}

// Cost of one plan shape in j per resident CTA: waves of `items` equal items
// of `len` j each on `slots` CTAs, with a per-item overhead worth
// kItemCostJ j (the i records, the tile start-up and the result stores).
constexpr unsigned kItemCostJ = 64;
__host__ __device__ inline unsigned long long wave_cost(unsigned items, unsigned slots, unsigned len)
{
    return (unsigned long long)ucdiv(items, slots) * (len + kItemCostJ);
}

__host__ __device__ inline unsigned slice_len(int n, int S, int tile)
{
    return (unsigned)cdiv(cdiv(n, S), tile) * (unsigned)tile;
}

__host__ __device__ inline unsigned ugcd(unsigned a, unsigned b)
{
    while (b) {
        const unsigned t = a % b;
        a = b;
        b = t;
    }
    return a;
}

__host__ __device__ inline Plan plan_ipar(int na, int n, int iblk, int tile, int slots,
                                          int split, long long part_cap, bool tail_split = false)
{
    Plan p;
    p.n_iblk = (int)ucdiv((unsigned)na, (unsigned)iblk);
    p.n_whole = 0;
    p.a0 = 0;
    const int smax_tiles = (int)ucdiv((unsigned)n, 2u * (unsigned)tile);
    const long long pmax = part_cap / ((long long)kComp * (na > 0 ? na : 1));
    int smax = smax_tiles < pmax ? smax_tiles : (int)pmax;
    if (smax < 1) smax = 1;
    int S;
    if (split > 0) {
        S = split < smax ? split : smax;
    } else {
        const unsigned nib = (unsigned)p.n_iblk, us = (unsigned)slots;
        int s0 = nib >= 2 * us ? 1 : (int)ucdiv(2 * us, nib);
        if (s0 > smax) s0 = smax;
        int best = s0, first_ok = fill_ok(nib * (unsigned)s0, us) ? s0 : 0;
#pragma unroll
        for (int q = 0; q < 24; ++q) {
            int s;
            if (q < 8) s = s0 + q;
            else if (q < 16) s = (int)udiv((unsigned)(q - 7) * us, nib);
            else s = (int)ucdiv((unsigned)(q - 15) * us, nib);
            if (s < s0 || s > smax) continue;
            const unsigned it = nib * (unsigned)s;
            if (fill_ok(it, us) && (first_ok == 0 || s < first_ok)) first_ok = s;
            if (better_fill(it, us, nib * (unsigned)best)) best = s;
        }
        S = first_ok ? first_ok : best;
        // With at least one full wave of i-blocks, the blocks of the full
        // waves may instead run whole and only the remainder be sliced, in a
        // slice count that fills its waves (multiples of slots / gcd(rem,
        // slots) fill them exactly): taken when its cost is lower.
        const unsigned rem = nib % us;
        if (tail_split && nib >= us && rem > 0) {
            const unsigned whole = nib - rem;
            const long long arem = (long long)na - (long long)whole * iblk;
            const long long pmax_t = part_cap / ((long long)kComp * arem);
            int smax_t = smax_tiles < pmax_t ? smax_tiles : (int)pmax_t;
            const unsigned long long c_uni = wave_cost(nib * (unsigned)S, us, slice_len(n, S, tile));
            const unsigned long long c_whole = wave_cost(whole, us, (unsigned)n);
            const unsigned per = us / ugcd(rem, us);
            int bt = 0;
            unsigned long long c_best = c_uni;
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                const int s = q < 4 ? (int)(per * (unsigned)(q + 1)) : (int)ucdiv((unsigned)(q - 3) * us, rem);
                if (s < 2 || s > smax_t) continue;
                const unsigned long long c =
                    c_whole + wave_cost(rem * (unsigned)s, us, slice_len(n, s, tile));
                if (c < c_best) {
                    c_best = c;
                    bt = s;
                }
            }
            if (bt > 0) {
                p.n_whole = (int)whole;
                p.a0 = (int)((long long)whole * iblk);
                S = bt;
            }
        }
    }
    p.jslice = (int)slice_len(n, S, tile);
    p.S = cdiv(n, p.jslice);
    p.items = p.n_whole + (p.n_iblk - p.n_whole) * p.S;
    return p;
}

// Work item w of an i-parallel plan: its i-block ib, j range [j0, j1) and
// slice sl (-1 for an i-block taken whole, whose result is final).
__host__ __device__ inline void ipar_item(int w, int n_iblk, int n_whole, int S, int jslice, int n,
                                          int &ib, int &sl, int &j0, int &j1)
{
    if (w < n_whole || S == 1) {
        ib = w;
        sl = -1;
        j0 = 0;
        j1 = n;
    } else {
        const int nb = n_iblk - n_whole, q = w - n_whole;
        ib = n_whole + q % nb;
        sl = q / nb;
        j0 = sl * jslice;
        j1 = n < j0 + jslice ? n : j0 + jslice;
    }
}

// j-parallel: CTAs own ic active particles and one j slice; each thread takes
// every nt-th j of the slice, at least eight per thread.  The slice count aims
// at two work items per resident CTA, else (slices too short) at one, so that
// the last wave is not a small remainder.
__host__ __device__ inline Plan plan_jpar(int na, int n, int nt, int ic, int slots,
                                          long long part_cap)
{
    Plan p;
    p.n_iblk = cdiv(na, ic);
    int S = cdiv(2LL * slots, p.n_iblk);
    const int smax = cdiv(n, 8LL * nt);
    if (S > smax) S = cdiv((long long)slots, p.n_iblk);
    if (S > smax) S = smax;
    long long pmax = part_cap / ((long long)kComp * ic * p.n_iblk);
    if (S > pmax) S = (int)pmax;
    if (S < 1) S = 1;
    p.jslice = cdiv(cdiv(n, S), nt) * nt;
    p.S = cdiv(n, p.jslice);
    p.items = p.n_iblk * p.S;
    p.n_whole = 0;
    p.a0 = 0;
    return p;
}

// Lanes per output of the slice combine: a power of two T <= 32, T <= S, with
// about 2^18 threads in all (T * 7 na), so that both small blocks with many
// slices and large blocks with few get enough loads in flight.
__host__ __device__ inline int combine_lanes(int na, int S)
{
    const long long want = (1LL << 18) / ((long long)kComp * (na > 0 ? na : 1));
    int T = 1;
    while (T < 32 && T < want && 2 * T <= S) T *= 2;
    return T;
}

// Which kernel serves a block of na particles: jpar for na <= jpar_max.
__host__ __device__ inline bool use_jpar(int na, int jpar_max) { return na <= jpar_max; }

// Force kernels by block size: j-parallel, small-block i-parallel (one i per
// thread, blocks of kIparNT i), i-parallel (kIparR i per thread, blocks of
// kIparNT * kIparR i).  The small-block kernel runs at about three quarters of
// the other's rate on full blocks, so it serves a block when its padded i
// count is at most 3/4 of the other's: up to 192, 257..384 and 513..576 active
// with 64-i and 256-i blocks (measured crossings on 2^16 and 2^20 bodies).
// small_max <= jpar_max disables it.
__host__ __device__ inline bool small_pays(int na)
{
    const long long s = (long long)cdiv(na, kIparNT) * kIparNT;
    const long long r = (long long)cdiv(na, kIparNT * kIparR) * (kIparNT * kIparR);
    return 4 * s <= 3 * r;
}

enum Regime { kRegJpar = 0, kRegSmall = 1, kRegIpar = 2 };
__host__ __device__ inline int regime_of(int na, int jpar_max, int small_max)
{
    if (na <= jpar_max) return kRegJpar;
    if (na <= small_max && small_pays(na)) return kRegSmall;
    return kRegIpar;
}

// The work decomposition of one force launch: the block size, the kernel
// that serves it and that kernel's plan.  It is computed once per launch, by
// make_force_plan on the host when the block size is known there, else by the
// scheduler's last thread next to the block size; kernels read it instead of
// planning in every CTA.
struct ForcePlan {
    Plan p;        // plan of the serving kernel (zero for the FP32 summation variants)
    int na;        // block size
    int regime;    // kRegJpar / kRegSmall / kRegIpar (summation variants: kRegIpar)
    int ic;        // j-parallel: i per pass
    int lanes;     // slice combine: lanes per output
};

// Everything a force launch needs.
struct ForceArgs {
    int n;                    // j count
    const int *act;           // active indices (device)
    const int *na_dev;        // device block size, or nullptr to use na_host
    int na_host;
    ForcePlan plan;           // the plan for na_host (na_dev == nullptr)
    const ForcePlan *plan_dev;  // the plan for *na_dev, written by the scheduler
    int precision;            // NB_DS or NB_FP64
    int summation;            // NB_SUM_*
    int slots_sum;            // resident CTAs of the summation variant's kernel
    int jpar_max;             // regime boundaries (see regime_of)
    int small_max;
    int split;                // forced slice count for i-parallel, 0 = auto
    int slots_ipar, slots_jpar, slots_small;
    long long part_cap;       // capacity of part in doubles
    double *part;             // slice partials: part[(s * 7 + c) * na + a]; the DS
                              // j-parallel kernel: part[(chunk * 7 ic + e) * S + s]
    int *jcnt;                // per-chunk slice arrival counters (zero between launches)
    ForceOut out;
    double eps2;
    int *err;                 // device error word
};

// Summation variants (k_sum.cu): the force with single-precision pair terms in
// IEEE round-to-nearest arithmetic, summed in 64-bit fixed point (GRAPE-style,
// independent of summation order), or in FP32 in index order, or in FP32
// smallest pair force first.
struct SumArgs {
    int mode;                       // NB_SUM_FIXED, NB_SUM_FP32 or NB_SUM_FP32_SORTED
    unsigned *bounds;               // [2] fixed point: largest fl32 mass, largest fl32 |vx|+|vy|+|vz| (bits)
    unsigned long long *scratch;    // sorted: 2 n keyed items per resident CTA
    int slots;                      // resident CTAs of the mode's force kernel
};
#ifndef NB_FIX_NT
#define NB_FIX_NT 64
#endif
#ifndef NB_FIX_R
#define NB_FIX_R 1
#endif
#ifndef NB_FIX_UNROLL
#define NB_FIX_UNROLL 4
#endif
constexpr int kFixNT = NB_FIX_NT;   // fixed point: threads per CTA (= j per tile)
constexpr int kFixR = NB_FIX_R;     // fixed point: i per thread
constexpr int kFixUnroll = NB_FIX_UNROLL;  // fixed point: j unrolling of the inner loop
constexpr int kSeqNT = 128;         // FP32 index order: threads per CTA, one i each
constexpr int kSortNT = 1024;       // FP32 sorted: one CTA per i
constexpr int kErrFixedScale = 64;  // device error word: fixed-point scales out of range
constexpr int kErrInput = 65;       // device error word: a non-finite value or a negative mass

__host__ __device__ inline ForcePlan make_force_plan(const ForceArgs &fa, int na)
{
    ForcePlan f{};
    f.na = na;
    f.regime = kRegIpar;
    if (na <= 0) return f;
    if (fa.summation == NB_SUM_FIXED) {
        f.p = plan_ipar(na, fa.n, kFixNT * kFixR, kFixNT, fa.slots_sum, fa.split, fa.part_cap / 2);
        return f;
    }
    if (fa.summation != NB_SUM_COMPENSATED) return f;   // no slices
    const bool f64 = fa.precision == NB_FP64;
    f.regime = f64 ? (use_jpar(na, fa.jpar_max) ? kRegJpar : kRegIpar)
                   : regime_of(na, fa.jpar_max, fa.small_max);
    if (f.regime == kRegJpar) {
        f.ic = !f64 && na <= kJparIC1Max ? 1 : kJparIC;
        f.p = plan_jpar(na, fa.n, kJparNT, f.ic, fa.slots_jpar, fa.part_cap);
    } else {
        const int r = f64 ? kIparR64 : (f.regime == kRegSmall ? kIparSmallR : kIparR);
        const int slots = f.regime == kRegSmall ? fa.slots_small : fa.slots_ipar;
        f.p = plan_ipar(na, fa.n, kIparNT * r, kIparNT * (f64 ? 1 : kIparTileMult), slots, fa.split,
                        fa.part_cap, true);
    }
    f.lanes = combine_lanes(na - f.p.a0, f.p.S);
    return f;
}

#ifdef __CUDACC__
// The plan of this launch (a uniform load for the device-sized launches).
__device__ __forceinline__ ForcePlan load_plan(const ForceArgs &fa)
{
    return fa.plan_dev ? *fa.plan_dev : fa.plan;
}
#endif

// Persistent block-step loop (k_run.cu): nb_run in one cooperative launch for
// systems of up to kRunMaxN particles, kRunNT threads per CTA, one CTA per
// `per` particles.
constexpr int kRunNT = 256;
// a CTA corrects up to this many particles of a step with four lanes each
constexpr int kRunQuadMax = 16;
constexpr int kRunMaxN = 16384;   // above it the per-stage graph, using every SM for the force, is faster
struct RunArgs {
    State s;
    JDS j;
    Ctrl *ctrl;
    int n, ncta, per;            // particles, CTAs, particles per CTA (<= kRunNT)
    float eps2f;                 // single-precision eps^2 of the pair terms
    double eta;
    int level_min, level_fixed;
    long long t_end, max_steps;  // stop before a block time past t_end, or after max_steps steps
    int *act;                    // [n] block list
    long long *mins;             // [ncta] per-CTA minimum end time
    int *counts;                 // [ncta] per-CTA block count
    unsigned *maxs;              // [2 ncta] fixed point: per-CTA mass and |v|_1 bounds (float bits)
    double *part;                // [ncta][n][7] partials (fixed point: pairs of int64)
    unsigned long long *bar;     // grid-barrier arrivals (zero at launch)
};

// Reverse mode (k_adjoint.cu).  Force-VJP records: DS (x_hi, y_hi, z_hi, m),
// (x_lo, y_lo, z_lo, 0), (vx, vy, vz, 0), (abar, 0), (kbar, 0); FP64 (x, y,
// z, m), (v, 0), (abar, 0), (kbar, 0).
struct VjpRec {
    float4 ph, pl, v, ab, kb;
};
struct VjpRecDS {
    float4 *ph, *pl, *v, *ab, *kb;
};
struct VjpRec64 {
    double4_32a *x, *v, *ab, *kb;
};
struct VjpArgs {
    int n;
    double eps2;
    int slots;
    long long part_cap;
    Plan plan;             // plan_ipar over all n particles (set by the launcher)
    double *part;          // slice partials part[(s * 7 + c) * n + k]
    VjpRecDS rec;
    VjpRec64 rec64;
    const double *m;
    double *xbar, *vbar, *mbar;  // outputs [n][3], [n][3], [n] (overwritten)
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files).

// k_force.cu
// Returns the number of kernels launched.
int launch_force_ds(const ForceArgs &fa, const JDS &j, bool softened, int grid_ipar, int grid_jpar,
                    int grid_small, cudaStream_t st);
void launch_force_f64(const ForceArgs &fa, const JF64 &j, bool softened, int grid_ipar,
                      int grid_jpar, cudaStream_t st);
int occupancy_force(int precision, int regime, int *blocks_per_sm);

// k_sum.cu
int occupancy_sum(int mode, int *blocks_per_sm);
int grid_summed(const ForceArgs &fa, const SumArgs &sa);
int launch_force_summed(const ForceArgs &fa, const JDS &j, const SumArgs &sa, int grid,
                        cudaStream_t st);

// k_run.cu
int run_layout(int n, int sms, int blocks_per_sm, int *ncta, int *per);
int occupancy_run(int summation, int *blocks_per_sm);
cudaError_t launch_run(const RunArgs &ra, int summation, cudaStream_t st);
cudaError_t launch_check_wait(const unsigned long long *counter, long long limit_cycles, Ctrl *ctrl,
                              cudaStream_t st);

// k_step.cu
void launch_predict(const State &s, long long t_val, const long long *t_ptr, const int *gate,
                    int precision, JDS jds, JF64 jf, cudaStream_t st);
// Blocks of at most kCorrectQuadPerSM x SMs particles are corrected with four
// lanes per particle (correct_particle_quad), larger ones one thread each.
constexpr int kCorrectQuadPerSM = 16;
void launch_correct(const State &s, const int *act, int na_host, const int *na_dev,
                    long long t_val, const long long *t_ptr, const double *acc_new,
                    const double *jerk_new, double eta, int level_min, int level_fixed,
                    int *err, int sms, cudaStream_t st);
void launch_initial_steps(const State &s, const double *acc, const double *jerk, double eta_init,
                          int level_min, int level_fixed, int *err, cudaStream_t st);
// Also writes the plan of the force on the new block (make_force_plan(fa, n_active))
// and predicts every particle to the block time into the j records (as
// launch_predict), unless no block is left before the end time.
void launch_schedule(const State &s, Ctrl *ctrl, long long *blockmin, int *blockcnt, int *act,
                     int nblocks, const ForceArgs &fa, ForcePlan *plan_out, int precision,
                     const JDS &jds, const JF64 &jf, cudaStream_t st);
int schedule_blocks(int n);
void launch_energy(const State &s, const long long *t_ptr, const double *pot, double *part,
                   Ctrl *ctrl, cudaStream_t st);
int energy_blocks(int n);
void launch_validate(const int *idx, int na, int n, unsigned int *bitmap, int *err,
                     cudaStream_t st);
void launch_gather_state(const State &s, double *x, double *v, double *a, double *k,
                         cudaStream_t st);
void launch_scatter_state(const State &s, const double *x, const double *v, const double *a,
                          const double *k, cudaStream_t st);
void launch_iota(int *p, int n, cudaStream_t st);
// Raises kErrInput unless every value of p[cnt] is finite (and, with
// nonneg, >= 0).
void launch_check_input(const double *p, long long cnt, bool nonneg, int *err, cudaStream_t st);

// k_adjoint.cu
int vjp_slots(int precision, int sms);
int vjp_tile();
int launch_force_vjp(const VjpArgs &va, int precision, bool softened, cudaStream_t st);
void launch_adj_pre(const State &s, double dt, const double *xb, const double *vb, double *ab,
                    double *kb, int precision, const VjpRecDS &rec, const VjpRec64 &rec64,
                    cudaStream_t st);
void launch_adj_post(int n, double dt, double *xb, double *vb, double *ab, double *kb, double *mb,
                     const double *xg, const double *vg, const double *mg, cudaStream_t st);
void launch_adj_initial_rec(const State &s, const double *ab, const double *kb, int precision,
                            const VjpRecDS &rec, const VjpRec64 &rec64, cudaStream_t st);
void launch_add3(int n, double *dst, const double *src, double *dst2, const double *src2,
                 double *dstm, const double *srcm, cudaStream_t st);
void launch_set_ak(const State &s, const double *acc, const double *jerk, cudaStream_t st);
void launch_copy_state(const State &dst, const State &src, cudaStream_t st);

}  // namespace nbk
