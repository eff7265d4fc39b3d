// k_sum.cu -- the force with the summation variants of Section 6.
//
// The paper contrasts GRAPE-6, which accumulates pair forces in 64-bit fixed
// point, with the GPU, which sums in single precision, and suggests sorting
// the forces and adding the smallest first.  These kernels evaluate the same
// single-precision pair terms on the double-single j records,
//
//   dx   = (xj_hi - xi_hi) + (xj_lo - xi_lo),   u = vj - vi        (per axis)
//   d2   = (dx0 dx0 + dx1 dx1) + dx2 dx2,        r2 = d2 + eps2
//   rv   = (dx0 u0 + dx1 u1) + dx2 u2
//   rinv = 1 / sqrt(r2),  rinv2 = rinv rinv,  mr = mj rinv,  mr3 = mr rinv2
//   b    = (-3 rv) rinv2
//   acc  = (mr3 Sa) dx,   jerk = (mr3 Sk) (u + b dx),   pot = -(mr Sp),
//
// every operation one IEEE single-precision operation rounded to nearest in
// that order (the __f*_rn intrinsics are never contracted into multiply-adds),
// so a CPU evaluating the same sequence gets the same bits.  The pair j = i
// and pairs with r2 = 0 contribute nothing.  Three summations:
//
//  NB_SUM_FIXED  Sa, Sk, Sp are powers of two chosen from bounds over all
//    particles so that every scaled term stays below 2^56; each term is
//    rounded to the nearest integer (ties to even) and the integers are summed
//    exactly in 128 bits.  Integer sums do not depend on their order, so the
//    result depends on neither the order of j, nor the j slices, nor which
//    CTA computes what.  (The rounding avoids float-to-int64 conversions, which
//    run on the FP64 pipe: three exact FP32 splits do it on the FP32 pipe.)
//  NB_SUM_FP32  one thread per i, an FP32 running sum over j = 0, 1, ... .
//  NB_SUM_FP32_SORTED  one CTA per i: the pair-force magnitudes |mj dx/r^3|
//    as keys, a stable radix sort of (key, j), then the FP32 running sum in
//    increasing key (ties in increasing j).
#include <cfloat>

#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

constexpr unsigned kFull = 0xffffffffu;

// The largest single-precision mass and |vx| + |vy| + |vz| over all j, as
// float bits (non-negative floats order like their bits); bounds[] must be
// zero on entry.
__global__ void k_fixed_bounds(JDS J, int n, unsigned *bounds)
{
    unsigned mb = 0, vb = 0;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const float4 v = J.vel[j];
        const float v1 = __fadd_rn(__fadd_rn(fabsf(v.x), fabsf(v.y)), fabsf(v.z));
        mb = max(mb, __float_as_uint(J.pos_hi[j].w));
        vb = max(vb, __float_as_uint(v1));
    }
    mb = __reduce_max_sync(kFull, mb);
    vb = __reduce_max_sync(kFull, vb);
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&bounds[0], mb);
        atomicMax(&bounds[1], vb);
    }
}

// One pair into the tile's split sums; the pair j = i adds zeros, so every
// tile adds exactly NT terms.
template <bool GUARD>
__device__ __forceinline__ void pair_fixed(const float4 &p, const float4 &l, const float4 &w,
                                           const float xh[3], const float xl[3], const float vi[3],
                                           float eps2, const Scale &S, unsigned a[3][7], int j = 0,
                                           int i = 1)
{
    float t[7];
    pair_rn(p, l, w, xh, xl, vi, eps2, S.sc[0], S.sc[1], S.sc[2], t);
#pragma unroll
    for (int q = 0; q < 7; ++q) split_add(GUARD && j == i ? 0.0f : t[q], a[0][q], a[1][q], a[2][q]);
}

// i-parallel like the DS kernel: a CTA owns R * NT active i and one j slice,
// tiles of NT j in shared memory; 64-bit tile sums, 128-bit totals; with
// several slices the totals go to the partial buffer as (hi, lo) pairs.
template <int NT, int R>
__global__ void __launch_bounds__(NT) k_force_fixed(ForceArgs fa, JDS J, SumArgs sa)
{
    const ForcePlan F = load_plan(fa);
    const int na = F.na;
    if (na <= 0) return;
    const float eps2 = (float)fa.eps2;
    Scale S;
    if (!fixed_scale(sa.bounds, eps2, S)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(fa.err, 0, kErrFixedScale);
        return;
    }
    const Plan P = F.p;
    long long *part = reinterpret_cast<long long *>(fa.part);
    __shared__ float4 s_p[NT], s_l[NT], s_v[NT];
    const int tid = threadIdx.x;

    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        const int ib = w % P.n_iblk;
        const int sl = w / P.n_iblk;
        const int j0 = sl * P.jslice;
        const int j1 = min(fa.n, j0 + P.jslice);

        float xh[R][3], xl[R][3], vi[R][3];
        int ia[R], ii[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int a = ib * NT * R + r * NT + tid;
            ia[r] = a < na ? a : -1;
            ii[r] = clamp_index(fa.act[a < na ? a : 0], fa.n);
            load_i(J, ii[r], xh[r], xl[r], vi[r]);
        }
        long long hi[R][7];
        unsigned long long lo[R][7];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int q = 0; q < 7; ++q) hi[r][q] = 0, lo[r][q] = 0;

        for (int jt = j0; jt < j1; jt += NT) {
            __syncthreads();
            const int j = jt + tid;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);  // mass 0: contributes 0
            s_p[tid] = j < j1 ? J.pos_hi[j] : z;
            s_l[tid] = j < j1 ? J.pos_lo[j] : z;
            s_v[tid] = j < j1 ? J.vel[j] : z;
            __syncthreads();
            unsigned ch[R][3][7];
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 7; ++q) ch[r][0][q] = ch[r][1][q] = ch[r][2][q] = 0u;
            bool mine = false;
#pragma unroll
            for (int r = 0; r < R; ++r) mine |= (unsigned)(ii[r] - jt) < (unsigned)NT;
            if (__any_sync(kFull, mine)) {
                for (int jj = 0; jj < NT; ++jj)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        pair_fixed<true>(s_p[jj], s_l[jj], s_v[jj], xh[r], xl[r], vi[r], eps2, S,
                                         ch[r], jt + jj, ii[r]);
            } else {
#pragma unroll (kFixUnroll)
                for (int jj = 0; jj < NT; ++jj)
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        pair_fixed<false>(s_p[jj], s_l[jj], s_v[jj], xh[r], xl[r], vi[r], eps2, S,
                                          ch[r]);
            }
#pragma unroll
            for (int r = 0; r < R; ++r)
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    add128(hi[r][q], lo[r][q], tile_sum(ch[r][0][q], ch[r][1][q], ch[r][2][q], NT));
        }

#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (ia[r] < 0) continue;
            if (P.S == 1) {
                double res[kComp];
#pragma unroll
                for (int q = 0; q < 7; ++q)
                    res[q] = __dmul_rn(i128_to_double(hi[r][q], lo[r][q]),
                                       S.inv[q < 3 ? 0 : (q < 6 ? 1 : 2)]);
                store_result(fa.out, ia[r], res);
            } else {
#pragma unroll
                for (int q = 0; q < 7; ++q) {
                    long long *pp = part + 2 * (((long long)sl * kComp + q) * na + ia[r]);
                    pp[0] = hi[r][q];
                    pp[1] = (long long)lo[r][q];
                }
            }
        }
    }
}

// Sum of the slices' 128-bit totals (exact, any order) and conversion.
__global__ void k_fixed_combine(ForceArgs fa, SumArgs sa)
{
    const ForcePlan F = load_plan(fa);
    const int na = F.na;
    if (na <= 0) return;
    const Plan P = F.p;
    if (P.S == 1) return;
    Scale S;
    if (!fixed_scale(sa.bounds, (float)fa.eps2, S)) return;
    const long long *part = reinterpret_cast<const long long *>(fa.part);
    const long long total = (long long)na * kComp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e / na), a = (int)(e % na);
        long long hi = 0;
        unsigned long long lo = 0;
        for (int q = 0; q < P.S; ++q) {
            const long long *pp = part + 2 * (((long long)q * kComp + c) * na + a);
            const unsigned long long l2 = lo + (unsigned long long)pp[1];
            hi += pp[0] + (l2 < lo ? 1 : 0);
            lo = l2;
        }
        const double inv = c < 3 ? S.inv[0] : (c < 6 ? S.inv[1] : S.inv[2]);
        write_combined(fa.out, c, a, __dmul_rn(i128_to_double(hi, lo), inv));
    }
}

// ---------------------------------------------------------------------------
// FP32 running sum in index order: one thread per i over all j, in order.

template <int NT>
__global__ void __launch_bounds__(NT) k_force_seq(ForceArgs fa, JDS J)
{
    const int na = read_na(fa);
    if (na <= 0) return;
    __shared__ float4 s_p[NT], s_l[NT], s_v[NT];
    const float eps2 = (float)fa.eps2;
    const int tid = threadIdx.x, n = fa.n;
    const int nblk = cdiv(na, NT);
    for (int ib = blockIdx.x; ib < nblk; ib += gridDim.x) {
        const int a = ib * NT + tid;
        const int i = clamp_index(fa.act[a < na ? a : 0], n);
        float xh[3], xl[3], vi[3];
        load_i(J, i, xh, xl, vi);
        float sum[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int jt = 0; jt < n; jt += NT) {
            __syncthreads();
            const int j = jt + tid;
            if (j < n) {
                s_p[tid] = J.pos_hi[j];
                s_l[tid] = J.pos_lo[j];
                s_v[tid] = J.vel[j];
            }
            __syncthreads();
            const int jc = min(NT, n - jt);
            for (int jj = 0; jj < jc; ++jj) {
                float t[7];
                const bool ok = pair_rn(s_p[jj], s_l[jj], s_v[jj], xh, xl, vi, eps2, 1.0f, 1.0f,
                                        1.0f, t);
                if (ok && jt + jj != i) {
#pragma unroll
                    for (int q = 0; q < 7; ++q) sum[q] = __fadd_rn(sum[q], t[q]);
                }
            }
        }
        if (a < na) {
            double res[kComp];
#pragma unroll
            for (int q = 0; q < 7; ++q) res[q] = (double)sum[q];
            store_result(fa.out, a, res);
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 running sum, smallest pair force first: one CTA per active i.
//  1. keyed items (key bits << 32 | j) for every j into the CTA's scratch, in
//     index order; j = i and r2 = 0 get the key 0xffffffff (sorted last).
//  2. stable LSD radix sort on the key, four passes of 8 bits: a histogram,
//     its exclusive scan, then tile by tile each item's rank among the equal
//     digits of its warp (match_any) plus the counts of the earlier warps and
//     tiles; stability keeps equal keys in index order.
//  3. tiles of NT sorted items: every thread computes one item's terms into
//     shared memory, then seven threads add them in order, one per component.

constexpr int kSortW = kSortNT / 32;

__global__ void __launch_bounds__(kSortNT) k_force_sorted(ForceArgs fa, JDS J, SumArgs sa)
{
    constexpr int NT = kSortNT;
    const int na = read_na(fa);
    if (na <= 0) return;
    __shared__ unsigned s_base[256], s_tot[256];
    __shared__ unsigned short s_wc[kSortW][256];
    __shared__ float s_t[7][NT];
    __shared__ float s_res[7];
    __shared__ int s_cnt;
    const int n = fa.n, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const float eps2 = (float)fa.eps2;
    unsigned long long *const A = sa.scratch + (size_t)blockIdx.x * 2 * (size_t)n;
    unsigned long long *const B = A + n;

    for (int a = blockIdx.x; a < na; a += gridDim.x) {
        const int i = clamp_index(fa.act[a], n);
        float xh[3], xl[3], vi[3];
        load_i(J, i, xh, xl, vi);
        if (tid == 0) s_cnt = 0;
        __syncthreads();

        int cnt = 0;
        for (int j = tid; j < n; j += NT) {
            float t[7], key;
            const bool ok = pair_rn(J.pos_hi[j], J.pos_lo[j], J.vel[j], xh, xl, vi, eps2, 1.0f, 1.0f,
                                    1.0f, t, &key) && j != i;
            const unsigned kb = ok ? __float_as_uint(key) : 0xffffffffu;
            A[j] = ((unsigned long long)kb << 32) | (unsigned)j;
            cnt += ok;
        }
        cnt = __reduce_add_sync(kFull, cnt);
        if (lane == 0) atomicAdd(&s_cnt, cnt);

        unsigned long long *src = A, *dst = B;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 32 + 8 * pass;
            if (tid < 256) s_base[tid] = 0;
            for (int e = tid; e < kSortW * 256; e += NT) (&s_wc[0][0])[e] = 0;
            __syncthreads();
            for (int t0 = 0; t0 < n; t0 += NT) {
                const int idx = t0 + tid;
                const bool valid = idx < n;
                const unsigned d = valid ? (unsigned)(src[idx] >> shift) & 255u : 256u;
                const unsigned peers = __match_any_sync(kFull, d);
                if (valid && (peers & lt) == 0) atomicAdd(&s_base[d], (unsigned)__popc(peers));
            }
            __syncthreads();
            unsigned incl = 0, cntd = 0;
            if (tid < 256) {
                cntd = s_base[tid];
                incl = cntd;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                s_tot[tid] = incl;
            }
            __syncthreads();
            if (tid < 256) {
                unsigned off = 0;
                for (int w = 0; w < warp; ++w) off += s_tot[w * 32 + 31];
                s_base[tid] = incl - cntd + off;
            }
            __syncthreads();
            for (int t0 = 0; t0 < n; t0 += NT) {
                const int idx = t0 + tid;
                const bool valid = idx < n;
                const unsigned long long item = valid ? src[idx] : 0ULL;
                const unsigned d = valid ? (unsigned)(item >> shift) & 255u : 256u;
                const unsigned peers = __match_any_sync(kFull, d);
                const int rank = __popc(peers & lt);
                if (valid && rank == 0) s_wc[warp][d] = (unsigned short)__popc(peers);
                __syncthreads();
                if (tid < 256) {
                    unsigned run = 0;
                    for (int w = 0; w < kSortW; ++w) {
                        const unsigned c = s_wc[w][tid];
                        s_wc[w][tid] = (unsigned short)run;
                        run += c;
                    }
                    s_tot[tid] = run;
                }
                __syncthreads();
                if (valid) dst[s_base[d] + s_wc[warp][d] + rank] = item;
                __syncthreads();
                if (tid < 256) s_base[tid] += s_tot[tid];
                for (int e = tid; e < kSortW * 256; e += NT) (&s_wc[0][0])[e] = 0;
                __syncthreads();
            }
            unsigned long long *tmp = src;
            src = dst;
            dst = tmp;
        }

        const int total = s_cnt;
        float run = 0.0f;
        for (int t0 = 0; t0 < total; t0 += NT) {
            const int k = t0 + tid;
            if (k < total) {
                const int j = (int)(unsigned)(src[k] & 0xffffffffULL);
                float t[7];
                pair_rn(J.pos_hi[j], J.pos_lo[j], J.vel[j], xh, xl, vi, eps2, 1.0f, 1.0f, 1.0f, t);
#pragma unroll
                for (int q = 0; q < 7; ++q) s_t[q][tid] = t[q];
            }
            __syncthreads();
            if (tid < 7) {
                const int m = min(NT, total - t0);
#pragma unroll 8
                for (int k2 = 0; k2 < m; ++k2) run = __fadd_rn(run, s_t[tid][k2]);
            }
            __syncthreads();
        }
        if (tid < 7) s_res[tid] = run;
        __syncthreads();
        if (tid == 0) {
            double res[kComp];
#pragma unroll
            for (int q = 0; q < 7; ++q) res[q] = (double)s_res[q];
            store_result(fa.out, a, res);
        }
        __syncthreads();
    }
}

}  // namespace

int occupancy_sum(int mode, int *blocks_per_sm)
{
    cudaError_t e;
    if (mode == NB_SUM_FIXED)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_force_fixed<kFixNT, kFixR>,
                                                          kFixNT, 0);
    else if (mode == NB_SUM_FP32)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_force_seq<kSeqNT>, kSeqNT, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_force_sorted, kSortNT, 0);
    return e == cudaSuccess ? 0 : -1;
}

int grid_summed(const ForceArgs &fa, const SumArgs &sa)
{
    if (fa.na_dev) return sa.slots;
    const int na = fa.na_host;
    if (na <= 0) return 0;
    long long items;
    if (sa.mode == NB_SUM_FIXED)
        items = fa.plan.p.items;
    else if (sa.mode == NB_SUM_FP32)
        items = cdiv(na, kSeqNT);
    else
        items = na;
    return (int)(items < sa.slots ? items : sa.slots);
}

int launch_force_summed(const ForceArgs &fa, const JDS &j, const SumArgs &sa, int grid,
                        cudaStream_t st)
{
    if (grid <= 0) return 0;
    if (sa.mode == NB_SUM_FIXED) {
        cudaMemsetAsync(sa.bounds, 0, 2 * sizeof(unsigned), st);
        const int gb = (int)(cdiv(fa.n, 256) < 1024 ? cdiv(fa.n, 256) : 1024);
        k_fixed_bounds<<<gb, 256, 0, st>>>(j, fa.n, sa.bounds);
        k_force_fixed<kFixNT, kFixR><<<grid, kFixNT, 0, st>>>(fa, j, sa);
        long long gc = fa.na_dev ? 1024 : cdiv((long long)fa.na_host * kComp, 256);
        if (gc > 4096) gc = 4096;
        k_fixed_combine<<<(int)gc, 256, 0, st>>>(fa, sa);
        return 3;
    }
    if (sa.mode == NB_SUM_FP32) {
        k_force_seq<kSeqNT><<<grid, kSeqNT, 0, st>>>(fa, j);
        return 1;
    }
    k_force_sorted<<<grid, kSortNT, 0, st>>>(fa, j, sa);
    return 1;
}

}  // namespace nbk
