// k_noalloc.cu -- force on a few particles with no device allocation at all.
//
// Some callers cannot allocate device memory when they need a force: a host
// application that hands this library a fixed slice of GPU memory and forbids
// later cudaMalloc calls, a real-time loop in which an allocation could block
// or fail, or a plug-in whose host owns the device allocator.  For them
// nb_force_few_noalloc evaluates the force on up to NB_NOALLOC_MAX_ACTIVE
// particles straight from the caller's FP64 arrays, with no context.  Its
// only working memory is the file-scope array below, which the runtime places
// on each GPU when the library's module is loaded there and keeps until the
// process exits.
//
// The kernels are a variant of the j-parallel force: each CTA takes up to four
// active particles and one slice of the j range, every thread takes every
// 256th j of the slice, positions are split into double-single form as they
// are read, the CTA reduces with a warp-shuffle tree in double-single, and the
// per-slice partial sums go to the scratch array; a second kernel sums the
// slices in slice order.  Each thread adds its pair terms in FP32 runs of at
// most eight and folds every run into double-single sums.  Every partial is
// written before it is read in the same call, so nothing in the scratch array
// needs clearing between calls.
#include <climits>
#include <cmath>
#include <mutex>

#include "nb.h"
#include <cuda_runtime.h>

namespace {

constexpr int kNT = 256;                    // threads per CTA
constexpr int kIC = 4;                      // active particles per CTA
constexpr int kComp = 7;                    // acc xyz, jerk xyz, pot
constexpr int kMaxSlices = 2048;            // j slices at most
constexpr int kRun = 8;                     // FP32 pair terms per thread between promotions
constexpr long long kScratchDoubles = (long long)kMaxSlices * kComp * NB_NOALLOC_MAX_ACTIVE;
constexpr int kMaxDevices = 64;

// Slice partials: part[(s * 7 + c) * n_active + a].  7 MiB per GPU.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

__device__ __forceinline__ float rsqrt_sfu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void ds_add(float &h, float &l, float h2, float l2)
{
    float s = h + h2;
    float bb = s - h;
    float e = (h - (s - bb)) + (h2 - bb);
    h = s;
    l = (l + l2) + e;
}

struct DSPoint {
    float xh[3], xl[3], v[3], m;
};

__device__ __forceinline__ DSPoint load_point(const double *m, const double *x, const double *v,
                                              long long j)
{
    DSPoint p;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double xc = x[3 * j + c];
        p.xh[c] = __double2float_rn(xc);
        p.xl[c] = __double2float_rn(__dsub_rn(xc, (double)p.xh[c]));
        p.v[c] = __double2float_rn(v[3 * j + c]);
    }
    p.m = __double2float_rn(m[j]);
    return p;
}

// FP32 pair terms (Eq. 1 with the pair terms of the Appendix A kernel) on
// double-single positions; the pair j = i and, with eps = 0, any pair at r = 0
// contribute nothing.
__device__ __forceinline__ void pair(const DSPoint &J, const DSPoint &I, float eps2, bool skip,
                                     float acc[3], float jk[3], float &pot)
{
    float d[3], u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        d[c] = (J.xh[c] - I.xh[c]) + (J.xl[c] - I.xl[c]);
        u[c] = J.v[c] - I.v[c];
    }
    const float r2 = fmaf(d[0], d[0], fmaf(d[1], d[1], fmaf(d[2], d[2], eps2)));
    const float rv = fmaf(d[0], u[0], fmaf(d[1], u[1], d[2] * u[2]));
    float rinv = rsqrt_sfu(r2);
    rinv = (skip || !(r2 > 0.0f)) ? 0.0f : rinv;
    const float rinv2 = rinv * rinv;
    const float mr = J.m * rinv;
    const float mr3 = mr * rinv2;
    const float b = -3.0f * rv * rinv2;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = fmaf(mr3, d[c], acc[c]);
        jk[c] = fmaf(mr3, fmaf(b, d[c], u[c]), jk[c]);
    }
    pot -= mr;
}

__global__ void __launch_bounds__(kNT) k_few_partials(long long n, const double *m, const double *x,
                                                      const double *v, float eps2, const int *act,
                                                      int na, int S, long long jslice,
                                                      double *part)
{
    constexpr int NW = kNT / 32;
    constexpr int NV = kIC * kComp;
    __shared__ float s_h[NW][NV], s_l[NW][NV];
    const int chunks = (na + kIC - 1) / kIC;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int w = blockIdx.x; w < chunks * S; w += gridDim.x) {
        const int ch = w % chunks, sl = w / chunks;
        const long long j0 = sl * jslice;
        const long long j1 = j0 + jslice < n ? j0 + jslice : n;
        DSPoint ip[kIC];
        long long ii[kIC];
#pragma unroll
        for (int q = 0; q < kIC; ++q) {
            const int a = ch * kIC + q;
            long long i = act[a < na ? a : 0];
            i = i < 0 ? 0 : (i >= n ? n - 1 : i);
            ii[q] = i;
            ip[q] = load_point(m, x, v, i);
        }
        // Plain FP32 runs of at most kRun pair terms per thread, each folded
        // into the double-single sums (h, lo) by TwoSum, so the rounding error
        // of a thread's sum does not grow with the slice length.
        float h[NV], lo[NV];
#pragma unroll
        for (int e = 0; e < NV; ++e) h[e] = lo[e] = 0.0f;
        for (long long jb = j0 + tid; jb < j1; jb += (long long)kNT * kRun) {
            float t[NV];
#pragma unroll
            for (int e = 0; e < NV; ++e) t[e] = 0.0f;
#pragma unroll 1
            for (int u = 0; u < kRun; ++u) {
                const long long j = jb + (long long)u * kNT;
                if (j >= j1) break;
                const DSPoint jp = load_point(m, x, v, j);
#pragma unroll
                for (int q = 0; q < kIC; ++q) {
                    float a3[3] = {t[q * kComp], t[q * kComp + 1], t[q * kComp + 2]};
                    float k3[3] = {t[q * kComp + 3], t[q * kComp + 4], t[q * kComp + 5]};
                    float pp = t[q * kComp + 6];
                    pair(jp, ip[q], eps2, j == ii[q], a3, k3, pp);
                    t[q * kComp] = a3[0]; t[q * kComp + 1] = a3[1]; t[q * kComp + 2] = a3[2];
                    t[q * kComp + 3] = k3[0]; t[q * kComp + 4] = k3[1]; t[q * kComp + 5] = k3[2];
                    t[q * kComp + 6] = pp;
                }
            }
#pragma unroll
            for (int e = 0; e < NV; ++e) ds_add(h[e], lo[e], t[e], 0.0f);
        }
#pragma unroll
        for (int off = 16; off >= 1; off >>= 1)
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                const float h2 = __shfl_xor_sync(0xffffffffu, h[e], off);
                const float l2 = __shfl_xor_sync(0xffffffffu, lo[e], off);
                ds_add(h[e], lo[e], h2, l2);
            }
        if (lane == 0)
#pragma unroll
            for (int e = 0; e < NV; ++e) {
                s_h[warp][e] = h[e];
                s_l[warp][e] = lo[e];
            }
        __syncthreads();
        if (tid < NV) {
            float th = s_h[0][tid], tl = s_l[0][tid];
            for (int ww = 1; ww < NW; ++ww) ds_add(th, tl, s_h[ww][tid], s_l[ww][tid]);
            const int q = tid / kComp, c = tid % kComp;
            const int a = ch * kIC + q;
            if (a < na) part[((long long)sl * kComp + c) * na + a] = (double)th + (double)tl;
        }
        __syncthreads();
    }
}

__global__ void k_few_combine(int na, int S, const double *part, double *acc, double *jerk,
                              double *pot)
{
    const int total = na * kComp;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int c = e / na, a = e % na;
        double s = 0.0;
        for (int q = 0; q < S; ++q) s += part[((long long)q * kComp + c) * na + a];
        if (c < 3) {
            if (acc) acc[3 * a + c] = s;
        } else if (c < 6) {
            if (jerk) jerk[3 * a + (c - 3)] = s;
        } else if (pot) {
            pot[a] = s;
        }
    }
}

// Per-device set-up: the device address of g_scratch (host code may not use
// the symbol itself, which on the host is only a stand-in) and the SM count.
struct DeviceSetup {
    double *scratch = nullptr;
    int sms = 0;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

int setup_current_device(DeviceSetup *out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NB_ECUDA;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &s = g_setup[dev];
    if (!s.scratch) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return NB_ECUDA;
        }
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            return NB_ECUDA;
        }
        s.sms = sms > 0 ? sms : 1;
        s.scratch = (double *)p;
    }
    *out = s;
    return NB_OK;
}

}  // namespace

extern "C" int nb_force_few_noalloc(int64_t n, const double *d_m, const double *d_x,
                                    const double *d_v, double eps, const int32_t *d_active_idx,
                                    int32_t n_active, double *d_acc, double *d_jerk, double *d_pot,
                                    void *stream)
{
    if (n < 1 || n > INT_MAX) return NB_EINVAL;
    if (n_active < 0 || n_active > NB_NOALLOC_MAX_ACTIVE) return NB_EINVAL;
    if (!std::isfinite(eps) || eps < 0.0) return NB_EINVAL;
    if (n_active == 0) return NB_OK;
    if (!d_m || !d_x || !d_v || !d_active_idx) return NB_EINVAL;
    // An error left pending by earlier work is not this call's: report it
    // without launching and without clearing it.
    if (cudaPeekAtLastError() != cudaSuccess) return NB_ECUDA;
    DeviceSetup s;
    const int rc = setup_current_device(&s);
    if (rc != NB_OK) return rc;

    // Slices: about two CTAs per SM in total, at least eight j per thread,
    // at most kMaxSlices (so the partials fit the scratch array).
    const int chunks = (n_active + kIC - 1) / kIC;
    long long S = (2LL * s.sms + chunks - 1) / chunks;
    const long long smax = (n + 8LL * kNT - 1) / (8LL * kNT);
    if (S > smax) S = smax;
    if (S > kMaxSlices) S = kMaxSlices;
    if (S < 1) S = 1;
    const long long jslice = ((n + S - 1) / S + kNT - 1) / kNT * kNT;
    S = (n + jslice - 1) / jslice;
    const long long items = (long long)chunks * S;
    const int grid = (int)(items < 4LL * s.sms ? items : 4LL * s.sms);

    cudaStream_t st = (cudaStream_t)stream;
    k_few_partials<<<grid, kNT, 0, st>>>(n, d_m, d_x, d_v, (float)(eps * eps), d_active_idx,
                                         n_active, (int)S, jslice, s.scratch);
    if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
    k_few_combine<<<(n_active * kComp + 255) / 256, 256, 0, st>>>(n_active, (int)S, s.scratch,
                                                                  d_acc, d_jerk, d_pot);
    return cudaGetLastError() == cudaSuccess ? NB_OK : NB_ECUDA;
}
