// k_force.cu -- direct-summation force kernels on the CUDA cores.
//
// For every active i and every j != i (Eq. 1 with the attractive sign and the
// pair terms of the Appendix A kernel), with dx = x_j - x_i, dv = v_j - v_i,
// r^2 = |dx|^2 + eps^2:
//   acc  +=  m_j dx / r^3
//   jerk +=  m_j (dv / r^3 - 3 (dx . dv) dx / r^5)
//   pot  -=  m_j / r
//
// DS kernels: positions are double-single (hi + lo FP32), the difference
// x_j - x_i is formed as (x_j,hi - x_i,hi) + (x_j,lo - x_i,lo), the pair terms
// run in FP32 with rsqrt.approx on the SFU, and each thread's per-tile FP32 partials
// are folded into hi + lo FP32 accumulators with TwoSum, so that the error of
// the sum over all N does not grow with N.  FP64 kernels do everything in FP64.
//
// i-parallel kernels: a CTA owns a block of active i (R per thread, in
// registers) and one j slice, streamed through shared memory in tiles that
// every thread reads by broadcast.  j-parallel kernels (small blocks): a CTA
// owns up to four active i and one j slice, each thread takes every NT-th j,
// and the CTA reduces with a warp-shuffle tree.  With several j slices the
// slice partials go to a buffer and are summed in fixed slice order (by a
// combine kernel, or, in the DS j-parallel kernel, by the CTA that finishes a
// chunk's last slice), so results are deterministic and no floating-point
// atomics are used.
//
// The self term j = i is dropped inside the loop: a warp whose own i fall in
// the current j tile runs a guarded copy of the inner loop that zeroes the
// pair with j = i; every other tile runs the unguarded loop.  (Leaving the
// self pair in and subtracting -m_i / eps at the end would inflate the FP32
// tile partial of the potential by m_i / eps, which at small N or large mass
// ratios is larger than the potential itself.)  With eps = 0 a pair at r = 0
// between distinct particles is dropped as well.
#include "nb_device.cuh"

namespace nbk {
namespace {

using namespace dev;

// One FP64 pair interaction.
template <bool SOFT>
__device__ __forceinline__ void pair_f64(const double4_32a &p, const double4_32a &w, const double xi[3],
                                         const double vi[3], double eps2, double acc[3],
                                         double jk[3], double &pot, int j, int i)
{
    const double dx = p.x - xi[0];
    const double dy = p.y - xi[1];
    const double dz = p.z - xi[2];
    const double ux = w.x - vi[0];
    const double uy = w.y - vi[1];
    const double uz = w.z - vi[2];
    const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
    const double rv = fma(dx, ux, fma(dy, uy, dz * uz));
    double rinv = rsqrt(r2);
    if (!SOFT) rinv = (r2 > 0.0) ? rinv : 0.0;
    rinv = (j == i) ? 0.0 : rinv;
    const double rinv2 = rinv * rinv;
    const double mr = p.w * rinv;
    const double mr3 = mr * rinv2;
    const double b = -3.0 * rv * rinv2;
    acc[0] = fma(mr3, dx, acc[0]);
    acc[1] = fma(mr3, dy, acc[1]);
    acc[2] = fma(mr3, dz, acc[2]);
    jk[0] = fma(mr3, fma(b, dx, ux), jk[0]);
    jk[1] = fma(mr3, fma(b, dy, uy), jk[1]);
    jk[2] = fma(mr3, fma(b, dz, uz), jk[2]);
    pot -= mr;
}


// ----------------------------------------------------------------------------
// DS, i-parallel.

// Work items (see plan_ipar / ipar_item): i-blocks taken whole write their
// result directly; the i-blocks of a sliced remainder write one partial per
// slice, which k_force_combine adds in slice order.
//
// The kernel reads its plan once into shared memory and takes the plan's
// fields from there where it uses them (volatile reads), and stores a slice
// partial through one pointer per particle: measured on the GB300 with the
// packed pair terms and 4-fold unrolling, these forms of the same arithmetic
// compile to the fastest of the variants tried (0.698 of the FP32 peak on
// N = 2^20 all active, against 0.668-0.681 for others), ahead of 2-, 6- and
// 8-fold unrolling and of 192- or 256-j tiles.
template <int NT, int R, int REG, bool SOFT>
__global__ void __launch_bounds__(NT) k_force_ipar_ds(ForceArgs fa, JDS J)
{
    __shared__ Plan s_plan;
    __shared__ int s_na;
    if (threadIdx.x == 0) {
        const ForcePlan F = load_plan(fa);
        s_plan = F.p;
        s_na = (F.na > 0 && F.regime == REG) ? F.na : 0;
    }
    __syncthreads();
    const int na = *(volatile int *)&s_na;
    if (na <= 0) return;
    const volatile Plan &P = s_plan;
    constexpr int TL = NT * kIparTileMult;   // j per shared-memory tile
    __shared__ float4 s_p[TL], s_l[TL], s_v[TL];
    const float eps2 = (float)fa.eps2;
    const int tid = threadIdx.x;

    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        int ib, sl, j0, j1;
        ipar_item(w, P.n_iblk, P.n_whole, P.S, P.jslice, fa.n, ib, sl, j0, j1);

        IDS I[R];
        int ia[R], ii[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int a = ib * NT * R + r * NT + tid;
            ia[r] = a < na ? a : -1;
            const int i = clamp_index(fa.act[a < na ? a : 0], fa.n);
            ii[r] = i;
            I[r] = make_ids(J.pos_hi[i], J.pos_lo[i], J.vel[i]);
        }
        float hi[R][kComp], lo[R][kComp];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < kComp; ++c) hi[r][c] = lo[r][c] = 0.0f;

        for (int jt = j0; jt < j1; jt += TL) {
            __syncthreads();
#pragma unroll
            for (int u = 0; u < kIparTileMult; ++u) {
                const int t = tid + u * NT, j = jt + t;
                if (j < j1) {
                    s_p[t] = J.pos_hi[j];
                    s_l[t] = J.pos_lo[j];
                    s_v[t] = J.vel[j];
                } else {
                    s_p[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                    s_l[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                    s_v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
            __syncthreads();
            float ta[R][3], tk[R][3], tp[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                ta[r][0] = ta[r][1] = ta[r][2] = 0.0f;
                tk[r][0] = tk[r][1] = tk[r][2] = 0.0f;
                tp[r] = 0.0f;
            }
            bool mine = false;
#pragma unroll
            for (int r = 0; r < R; ++r) mine |= (unsigned)(ii[r] - jt) < (unsigned)TL;
            if (__any_sync(0xffffffffu, mine)) {
                for (int jj = 0; jj < TL; ++jj) {
                    const float4 p = s_p[jj], l = s_l[jj], v = s_v[jj];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        pair_ds_packed<SOFT, true>(p, l, v, I[r], eps2, ta[r], tk[r], tp[r], jt + jj, ii[r]);
                }
            } else {
#pragma unroll (kIparUnroll)
                for (int jj = 0; jj < TL; ++jj) {
                    const float4 p = s_p[jj], l = s_l[jj], v = s_v[jj];
#pragma unroll
                    for (int r = 0; r < R; ++r)
                        pair_ds_packed<SOFT, false>(p, l, v, I[r], eps2, ta[r], tk[r], tp[r]);
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                two_sum_acc(hi[r][0], lo[r][0], ta[r][0]);
                two_sum_acc(hi[r][1], lo[r][1], ta[r][1]);
                two_sum_acc(hi[r][2], lo[r][2], ta[r][2]);
                two_sum_acc(hi[r][3], lo[r][3], tk[r][0]);
                two_sum_acc(hi[r][4], lo[r][4], tk[r][1]);
                two_sum_acc(hi[r][5], lo[r][5], tk[r][2]);
                two_sum_acc(hi[r][6], lo[r][6], tp[r]);
            }
        }

#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (ia[r] < 0) continue;
            double res[kComp];
#pragma unroll
            for (int c = 0; c < kComp; ++c) res[c] = (double)hi[r][c] + (double)lo[r][c];
            if (sl < 0) {
                store_result(fa.out, ia[r], res);
            } else {
                const int nb = na - P.a0;
                double *dst = fa.part + (long long)sl * kComp * nb - P.a0 + ia[r];
#pragma unroll
                for (int c = 0; c < kComp; ++c) dst[(long long)c * nb] = res[c];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// DS, j-parallel (small blocks).
//
// A CTA owns IC consecutive active i (IC = 1 for blocks of one or two
// particles, kJparIC otherwise) and one j slice; each thread takes every NT-th
// j of the slice.  The per-thread partials are reduced over the warp by a
// reduce-scatter tree (each level halves the number of values a lane carries,
// so the 7 values of an i cost 9 shuffle steps instead of 35), then over the warps in
// shared memory.  The CTA that finishes the last slice of an i chunk (an
// arrival counter per chunk, reset by that CTA) adds the chunk's slice
// partials in slice order: the result depends only on the plan, and no
// second launch is needed.

// Lane l ends up holding, for value index e = l >> (5 - log2 P), the DS sum of
// value e over all 32 lanes; P is a power of two <= 32.
template <int P>
__device__ __forceinline__ void warp_reduce_scatter(float (&h)[P], float (&lo)[P], int lane)
{
    int c = P;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        if (c > 1) {
            const bool up = (lane & off) != 0;
            const int half = c / 2;
#pragma unroll
            for (int k = 0; k < P / 2; ++k) {
                if (k < half) {
                    const float sh = up ? h[k] : h[k + half], sl = up ? lo[k] : lo[k + half];
                    float kh = up ? h[k + half] : h[k], kl = up ? lo[k + half] : lo[k];
                    const float rh = __shfl_xor_sync(0xffffffffu, sh, off);
                    const float rl = __shfl_xor_sync(0xffffffffu, sl, off);
                    ds_add(kh, kl, rh, rl);
                    h[k] = kh;
                    lo[k] = kl;
                }
            }
            c = half;
        } else {
            const float rh = __shfl_xor_sync(0xffffffffu, h[0], off);
            const float rl = __shfl_xor_sync(0xffffffffu, lo[0], off);
            ds_add(h[0], lo[0], rh, rl);
        }
    }
}

template <int NT, int IC, bool SOFT>
__device__ __forceinline__ void jpar_ds_items(const ForceArgs &fa, const JDS &J, int na, const Plan &P)
{
    constexpr int NW = NT / 32;
    constexpr int NV = IC * kComp;
    __shared__ float s_h[NW][NV], s_l[NW][NV];
    __shared__ int s_last;
    constexpr int UNROLL = IC == 1 ? 4 : 2;   // j in flight per thread
    const float eps2 = (float)fa.eps2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        const int ch = w % P.n_iblk;
        const int sl = w / P.n_iblk;
        const int j0 = sl * P.jslice;
        const int j1 = min(fa.n, j0 + P.jslice);
        const int nq = min(IC, na - ch * IC);   // i of this chunk (uniform in the CTA)

        float xh[IC][3], xl[IC][3], vi[IC][3];
        int ii[IC];
#pragma unroll
        for (int q = 0; q < IC; ++q) {
            const int a = ch * IC + q;
            const int i = clamp_index(fa.act[a < na ? a : 0], fa.n);
            ii[q] = i;
            const float4 p = J.pos_hi[i], l = J.pos_lo[i], v = J.vel[i];
            xh[q][0] = p.x; xh[q][1] = p.y; xh[q][2] = p.z;
            xl[q][0] = l.x; xl[q][1] = l.y; xl[q][2] = l.z;
            vi[q][0] = v.x; vi[q][1] = v.y; vi[q][2] = v.z;
        }
        float va[IC][3], vk[IC][3], vp[IC];
#pragma unroll
        for (int q = 0; q < IC; ++q) {
            va[q][0] = va[q][1] = va[q][2] = 0.0f;
            vk[q][0] = vk[q][1] = vk[q][2] = 0.0f;
            vp[q] = 0.0f;
        }
#pragma unroll UNROLL
        for (int j = j0 + tid; j < j1; j += NT) {
            const float4 p = __ldg(&J.pos_hi[j]), l = __ldg(&J.pos_lo[j]), v = __ldg(&J.vel[j]);
#pragma unroll
            for (int q = 0; q < IC; ++q)
                if (q == 0 || q < nq)
                    pair_ds<SOFT, true>(p, l, v, xh[q], xl[q], vi[q], eps2, va[q], vk[q], vp[q], j, ii[q]);
        }
        // one i at a time keeps the live registers down: 8 values (7 and a
        // zero) per reduce-scatter, lane l ends with value l >> 2
#pragma unroll
        for (int q = 0; q < IC; ++q) {
            float h[8] = {va[q][0], va[q][1], va[q][2], vk[q][0], vk[q][1], vk[q][2], vp[q], 0.0f};
            float lo[8] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
            if (q == 0 || q < nq) {
                warp_reduce_scatter<8>(h, lo, lane);
                const int e = lane >> 2;
                if ((lane & 3) == 0 && e < kComp) {
                    s_h[warp][q * kComp + e] = h[0];
                    s_l[warp][q * kComp + e] = lo[0];
                }
            }
        }
        __syncthreads();
        if (tid < nq * kComp) {
            float th = s_h[0][tid], tl = s_l[0][tid];
#pragma unroll
            for (int ww = 1; ww < NW; ++ww) ds_add(th, tl, s_h[ww][tid], s_l[ww][tid]);
            fa.part[((long long)ch * NV + tid) * P.S + sl] = (double)th + (double)tl;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0) {
            const int old = atomicAdd(&fa.jcnt[ch], 1);
            s_last = old == P.S - 1;
            if (s_last) fa.jcnt[ch] = 0;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            // warp per output: lane l adds slices l, l + 32, ... in four
            // interleaved chains, then a fixed xor tree
            for (int e = warp; e < nq * kComp; e += NW) {
                const double *src = fa.part + (long long)ch * NV * P.S + (long long)e * P.S;
                double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
                int q = lane;
                for (; q + 96 < P.S; q += 128) {
                    const double v0 = __ldcg(src + q), v1 = __ldcg(src + q + 32);
                    const double v2 = __ldcg(src + q + 64), v3 = __ldcg(src + q + 96);
                    s0 += v0; s1 += v1; s2 += v2; s3 += v3;
                }
                for (; q < P.S; q += 32) s0 += __ldcg(src + q);
                double s = (s0 + s1) + (s2 + s3);
#pragma unroll
                for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
                if (lane == 0) {
                    const int qq = e / kComp, c = e % kComp;
                    write_combined(fa.out, c, ch * IC + qq, s);
                }
            }
        }
        __syncthreads();
    }
}

template <int NT, bool SOFT>
__global__ void __launch_bounds__(NT, 2) k_force_jpar_ds(ForceArgs fa, JDS J)
{
    const ForcePlan F = load_plan(fa);
    if (F.na <= 0 || F.regime != kRegJpar) return;
    if (F.ic == 1) jpar_ds_items<NT, 1, SOFT>(fa, J, F.na, F.p);
    else jpar_ds_items<NT, kJparIC, SOFT>(fa, J, F.na, F.p);
}

// ----------------------------------------------------------------------------
// FP64, i-parallel.

template <int NT, int R, bool SOFT>
__global__ void __launch_bounds__(NT) k_force_ipar_f64(ForceArgs fa, JF64 J)
{
    const ForcePlan F = load_plan(fa);
    const int na = F.na;
    if (na <= 0 || F.regime != kRegIpar) return;
    const Plan P = F.p;
    __shared__ double4_32a s_p[NT], s_v[NT];
    const double eps2 = fa.eps2;
    const int tid = threadIdx.x;

    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        int ib, sl, j0, j1;
        ipar_item(w, P.n_iblk, P.n_whole, P.S, P.jslice, fa.n, ib, sl, j0, j1);

        double xi[R][3], vi[R][3];
        int ia[R], ii[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int a = ib * NT * R + r * NT + tid;
            ia[r] = a < na ? a : -1;
            const int i = clamp_index(fa.act[a < na ? a : 0], fa.n);
            ii[r] = i;
            const double4_32a p = J.pos[i], v = J.vel[i];
            xi[r][0] = p.x; xi[r][1] = p.y; xi[r][2] = p.z;
            vi[r][0] = v.x; vi[r][1] = v.y; vi[r][2] = v.z;
        }
        double acc[R][3], jk[R][3], pot[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            acc[r][0] = acc[r][1] = acc[r][2] = 0.0;
            jk[r][0] = jk[r][1] = jk[r][2] = 0.0;
            pot[r] = 0.0;
        }
        for (int jt = j0; jt < j1; jt += NT) {
            __syncthreads();
            const int j = jt + tid;
            if (j < j1) {
                s_p[tid] = J.pos[j];
                s_v[tid] = J.vel[j];
            } else {
                s_p[tid] = make_double4_32a(0., 0., 0., 0.);
                s_v[tid] = make_double4_32a(0., 0., 0., 0.);
            }
            __syncthreads();
#pragma unroll 4
            for (int jj = 0; jj < NT; ++jj) {
                const double4_32a p = s_p[jj], v = s_v[jj];
#pragma unroll
                for (int r = 0; r < R; ++r)
                    pair_f64<SOFT>(p, v, xi[r], vi[r], eps2, acc[r], jk[r], pot[r], jt + jj, ii[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (ia[r] < 0) continue;
            double res[kComp] = {acc[r][0], acc[r][1], acc[r][2], jk[r][0], jk[r][1], jk[r][2],
                                 pot[r]};
            if (sl < 0) {
                store_result(fa.out, ia[r], res);
            } else {
                const int nb = na - P.a0;
#pragma unroll
                for (int c = 0; c < kComp; ++c)
                    fa.part[((long long)sl * kComp + c) * nb + (ia[r] - P.a0)] = res[c];
            }
        }
    }
}

// ----------------------------------------------------------------------------
// FP64, j-parallel (small blocks).

template <int NT, int IC, bool SOFT>
__global__ void __launch_bounds__(NT) k_force_jpar_f64(ForceArgs fa, JF64 J)
{
    const ForcePlan F = load_plan(fa);
    const int na = F.na;
    if (na <= 0 || F.regime != kRegJpar) return;
    const Plan P = F.p;
    constexpr int NW = NT / 32;
    constexpr int NV = IC * kComp;
    __shared__ double s_r[NW][NV];
    const double eps2 = fa.eps2;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int w = blockIdx.x; w < P.items; w += gridDim.x) {
        const int ch = w % P.n_iblk;
        const int sl = w / P.n_iblk;
        const int j0 = sl * P.jslice;
        const int j1 = min(fa.n, j0 + P.jslice);
        double xi[IC][3], vi[IC][3];
        int ii[IC];
#pragma unroll
        for (int q = 0; q < IC; ++q) {
            const int a = ch * IC + q;
            const int i = clamp_index(fa.act[a < na ? a : 0], fa.n);
            ii[q] = i;
            const double4_32a p = J.pos[i], v = J.vel[i];
            xi[q][0] = p.x; xi[q][1] = p.y; xi[q][2] = p.z;
            vi[q][0] = v.x; vi[q][1] = v.y; vi[q][2] = v.z;
        }
        double val[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) val[e] = 0.0;
        for (int j = j0 + tid; j < j1; j += NT) {
            const double4_32a p = J.pos[j], v = J.vel[j];
#pragma unroll
            for (int q = 0; q < IC; ++q) {
                double a3[3] = {val[q * kComp], val[q * kComp + 1], val[q * kComp + 2]};
                double k3[3] = {val[q * kComp + 3], val[q * kComp + 4], val[q * kComp + 5]};
                double pp = val[q * kComp + 6];
                pair_f64<SOFT>(p, v, xi[q], vi[q], eps2, a3, k3, pp, j, ii[q]);
                val[q * kComp] = a3[0]; val[q * kComp + 1] = a3[1]; val[q * kComp + 2] = a3[2];
                val[q * kComp + 3] = k3[0]; val[q * kComp + 4] = k3[1]; val[q * kComp + 5] = k3[2];
                val[q * kComp + 6] = pp;
            }
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int e = 0; e < NV; ++e) val[e] += __shfl_xor_sync(0xffffffffu, val[e], off);
        if (lane == 0)
#pragma unroll
            for (int e = 0; e < NV; ++e) s_r[warp][e] = val[e];
        __syncthreads();
        if (tid < NV) {
            double r = s_r[0][tid];
            for (int ww = 1; ww < NW; ++ww) r += s_r[ww][tid];
            const int q = tid / kComp, c = tid % kComp;
            const int a = ch * IC + q;
            if (a < na) {
                fa.part[((long long)sl * kComp + c) * na + a] = r;
            }
        }
        __syncthreads();
    }
}

// ----------------------------------------------------------------------------
// Slice combine: out = sum over slices in a fixed order (FP64).

__global__ void k_force_combine(ForceArgs fa, int precision)
{
    const ForcePlan F = load_plan(fa);
    const int na = F.na;
    if (na <= 0) return;
    // the DS j-parallel kernel combines its own slices; the i-parallel kernels
    // store the result directly when there is one slice
    if (F.regime == kRegJpar ? precision != NB_FP64 : F.p.S == 1) return;
    const int S = F.p.S;
    // only the sliced i-blocks (block positions a0 .. na - 1) have partials
    const int a0 = F.regime == kRegJpar ? 0 : F.p.a0, nb = na - a0;
    const long long total = (long long)nb * kComp;
    // T lanes per output (a power of two, chosen from na and S only, so the
    // order of the additions is fixed): lane t of a group adds slices t,
    // t + T, ... in order, then a fixed xor tree over the group.  The groups
    // of a warp take consecutive particles, so each load instruction reads
    // whole 32-byte sectors of T slice rows.
    const int T = F.lanes;
    const int gpw = 32 / T;
    const int lane = threadIdx.x & 31, sub = lane & (T - 1);
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long wb = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; wb * gpw < total;
         wb += warps) {
        const long long o = wb * gpw + lane / T;
        const int c = (int)(o / nb), a = (int)(o % nb);
        double s = 0.0;
        if (o < total)
            for (int q = sub; q < S; q += T) s += fa.part[((long long)q * kComp + c) * nb + a];
        for (int off = T / 2; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (sub == 0 && o < total) write_combined(fa.out, c, a0 + a, s);
    }
}

int combine_grid(const ForceArgs &fa)
{
    if (!fa.na_dev) {
        // one thread per lane of every output group (up to 32 per output)
        long long total = (long long)fa.na_host * kComp * 32;
        long long g = (total + 255) / 256;
        return (int)(g < 1 ? 1 : (g > 4096 ? 4096 : g));
    }
    return 1024;
}

}  // namespace

int launch_force_ds(const ForceArgs &fa, const JDS &j, bool softened, int grid_ipar,
                    int grid_jpar, int grid_small, cudaStream_t st)
{
    if (softened) {
        if (grid_ipar > 0)
            k_force_ipar_ds<kIparNT, kIparR, kRegIpar, true><<<grid_ipar, kIparNT, 0, st>>>(fa, j);
        if (grid_small > 0)
            k_force_ipar_ds<kIparNT, kIparSmallR, kRegSmall, true><<<grid_small, kIparNT, 0, st>>>(fa, j);
        if (grid_jpar > 0) k_force_jpar_ds<kJparNT, true><<<grid_jpar, kJparNT, 0, st>>>(fa, j);
    } else {
        if (grid_ipar > 0)
            k_force_ipar_ds<kIparNT, kIparR, kRegIpar, false><<<grid_ipar, kIparNT, 0, st>>>(fa, j);
        if (grid_small > 0)
            k_force_ipar_ds<kIparNT, kIparSmallR, kRegSmall, false><<<grid_small, kIparNT, 0, st>>>(fa, j);
        if (grid_jpar > 0) k_force_jpar_ds<kJparNT, false><<<grid_jpar, kJparNT, 0, st>>>(fa, j);
    }
    int launches = (grid_ipar > 0) + (grid_small > 0) + (grid_jpar > 0);
    // a host-sized j-parallel launch combines its own slices
    if (fa.na_dev || grid_ipar > 0 || grid_small > 0) {
        k_force_combine<<<combine_grid(fa), 256, 0, st>>>(fa, NB_DS);
        ++launches;
    }
    return launches;
}

void launch_force_f64(const ForceArgs &fa, const JF64 &j, bool softened, int grid_ipar,
                      int grid_jpar, cudaStream_t st)
{
    if (softened) {
        if (grid_ipar > 0) k_force_ipar_f64<kIparNT, kIparR64, true><<<grid_ipar, kIparNT, 0, st>>>(fa, j);
        if (grid_jpar > 0) k_force_jpar_f64<kJparNT, kJparIC, true><<<grid_jpar, kJparNT, 0, st>>>(fa, j);
    } else {
        if (grid_ipar > 0) k_force_ipar_f64<kIparNT, kIparR64, false><<<grid_ipar, kIparNT, 0, st>>>(fa, j);
        if (grid_jpar > 0) k_force_jpar_f64<kJparNT, kJparIC, false><<<grid_jpar, kJparNT, 0, st>>>(fa, j);
    }
    k_force_combine<<<combine_grid(fa), 256, 0, st>>>(fa, NB_FP64);
}

int occupancy_force(int precision, int regime, int *blocks_per_sm)
{
    cudaError_t e;
    if (precision == NB_FP64)
        e = regime == kRegJpar
                ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      blocks_per_sm, k_force_jpar_f64<kJparNT, kJparIC, true>, kJparNT, 0)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                      blocks_per_sm, k_force_ipar_f64<kIparNT, kIparR64, true>, kIparNT, 0);
    else if (regime == kRegJpar)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, k_force_jpar_ds<kJparNT, true>, kJparNT, 0);
    else if (regime == kRegSmall)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, k_force_ipar_ds<kIparNT, kIparSmallR, kRegSmall, true>, kIparNT, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            blocks_per_sm, k_force_ipar_ds<kIparNT, kIparR, kRegIpar, true>, kIparNT, 0);
    return e == cudaSuccess ? 0 : -1;
}

}  // namespace nbk
