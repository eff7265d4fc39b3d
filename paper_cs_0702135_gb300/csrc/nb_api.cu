// nb_api.cu -- the C ABI declared in include/nb.h: context, argument checks,
// host-driven calls (nb_predict / nb_force / nb_correct) and the device-driven
// block step (nb_step / nb_run) replayed from a captured CUDA graph.
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "nb_internal.cuh"

using namespace nbk;

namespace {
// An NVTX range over one entry point (no cost unless a tool is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};
}  // namespace

struct nb_ctx {
    int n = 0;
    double eps = 0.0;
    nb_opts o{};
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int sms = 0;

    State S{};
    double *d_x = nullptr, *d_v = nullptr, *d_a = nullptr, *d_k = nullptr, *d_m = nullptr;
    long long *d_t = nullptr;
    int *d_lev = nullptr;
    JDS jds{};
    JF64 jf{};
    double *d_res = nullptr;        // force results: acc [n][3], jerk [n][3], pot [n]
    double *d_part = nullptr;       // slice partials
    ForcePlan *d_plan = nullptr;    // plan of the device-sized force (written by the scheduler)
    int *d_jcnt = nullptr;          // [n] slice arrival counters of the DS j-parallel kernel
    long long part_cap = 0;
    int *d_act = nullptr;           // block of the device-driven step
    int *d_idx = nullptr;           // indices passed by the host-driven calls
    int *d_all = nullptr;           // 0 .. n-1
    unsigned *d_bitmap = nullptr;   // index validation
    Ctrl *d_ctrl = nullptr;
    Ctrl *h_ctrl = nullptr;         // pinned mirror
    long long *d_blockmin = nullptr;
    int *d_blockcnt = nullptr;
    int nsched = 0;
    double *d_epart = nullptr;
    double *d_stage = nullptr;      // [7n] staging for host I/O

    int slots_ipar = 0, slots_jpar = 0, slots_small = 0, jpar_max = 0, small_max = 0;
    SumArgs sum{};                  // summation variant (NB_SUM_COMPENSATED: unused)
    // persistent nb_run (k_run.cu), allocated on first use
    double *d_run_part = nullptr;
    long long *d_run_mins = nullptr;
    int *d_run_counts = nullptr;
    unsigned *d_run_maxs = nullptr;
    unsigned long long *d_run_bar = nullptr;
    int run_ncta = 0, run_per = 0;
    unsigned *d_bounds = nullptr;   // fixed point: mass and velocity bounds
    unsigned long long *d_sort = nullptr;  // sorted: keyed items, 2n per resident CTA
    long long t_pred = 0;           // ticks of the last host-driven prediction
    bool force_valid = false;       // results in d_res usable by nb_correct
    int force_na = 0;
    long long force_t = 0;
    long long t_end_dev = -1;       // value of ctrl->t_end on the device
    cudaGraphExec_t step_exec = nullptr;
    long long step_nodes = 0;       // kernels in one captured step
    bool capturing = false;

    // differentiable trajectory (nb_traj_forward / nb_traj_backward)
    double *d_ck = nullptr;         // checkpoints, 12n doubles each: x, v, a, k (SoA)
    long long ck_slots = 0;
    double *d_seg = nullptr;        // step states of one segment, 12n doubles each
    long long seg_slots = 0;
    double *d_fin = nullptr;        // final state of the trajectory
    long long *d_tfin = nullptr;    // particle times at its end
    double *d_cot = nullptr;        // cotangents xb, vb, ab, kb [n][3], mb [n]; VJP xg, vg [n][3], mg [n]
    VjpRecDS vrec{};
    VjpRec64 vrec64{};
    int slots_vjp = 0;
    bool traj_valid = false;
    long long traj_steps = 0, traj_ckpt = 0;

    // measurement counters (nb_get_stats)
    long long launches = 0;
    bool profiling = false;
    std::vector<cudaEvent_t> ev_free, ev_pending;  // pending: start, stop, start, stop, ...
    long long force_launches = 0;
    double force_ms = 0.0;
    std::string err;
};

namespace {

const char *const kNoCtx = "null context";
thread_local std::string g_init_err;  // message of the last failed nb_init on this thread

int fail(nb_ctx *c, int code, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return code;
}

#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(c, e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA,        \
                        "%s: %s", #call, cudaGetErrorString(e_));                         \
    } while (0)

bool finite_all(const double *p, long long cnt)
{
    for (long long i = 0; i < cnt; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Converts a time to ticks of 2^-40; false if off the grid or out of range.
bool time_to_ticks(double t, long long *ticks)
{
    if (!std::isfinite(t) || t < 0.0 || t >= 0x1p22) return false;
    const double s = t * 0x1p40;
    if (s != std::floor(s)) return false;
    *ticks = (long long)s;
    return true;
}

int check_indices_host(nb_ctx *c, const int32_t *idx, int32_t na)
{
    if (na < 0 || na > c->n) return fail(c, NB_EINVAL, "n_active=%d outside [0, %d]", na, c->n);
    if (na > 0 && !idx) return fail(c, NB_EINVAL, "active_idx is NULL");
    std::vector<unsigned char> seen((size_t)c->n, 0);
    for (int32_t a = 0; a < na; ++a) {
        const int32_t i = idx[a];
        if (i < 0 || i >= c->n) return fail(c, NB_EINVAL, "active_idx[%d]=%d out of range", a, i);
        if (seen[(size_t)i]) return fail(c, NB_EINVAL, "active_idx[%d]=%d repeated", a, i);
        seen[(size_t)i] = 1;
    }
    return NB_OK;
}

// Pulls the control block to the host and turns a kernel-raised error into a
// return code (clearing it on the device).
int sync_ctrl(nb_ctx *c)
{
    CK(cudaMemcpyAsync(c->h_ctrl, c->d_ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    CK(cudaGetLastError());
    const int e = c->h_ctrl->err;
    if (e != 0) {
        CK(cudaMemsetAsync(&c->d_ctrl->err, 0, sizeof(int), c->st));
        CK(cudaStreamSynchronize(c->st));
        if (e == NB_ESTEP) return fail(c, NB_ESTEP, "a new time step fell below 2^-40");
        if (e == NB_EINVAL) return fail(c, NB_EINVAL, "invalid particle index (device check)");
        if (e == NB_ETIMEOUT)
            return fail(c, NB_ETIMEOUT, "a bounded device wait ran out");
        if (e == kErrInput)
            return fail(c, NB_EINVAL, "non-finite input or negative mass (device check)");
        if (e == kErrFixedScale)
            return fail(c, NB_EINVAL, "fixed-point summation: masses, velocities or eps put the "
                                      "fixed-point units outside the single-precision range");
        return fail(c, e, "device error %d", e);
    }
    return NB_OK;
}

ForceArgs force_args(nb_ctx *c, const int *act, int na_host, const int *na_dev, ForceOut out)
{
    ForceArgs fa{};
    fa.n = c->n;
    fa.act = act;
    fa.na_dev = na_dev;
    fa.na_host = na_host;
    fa.jpar_max = c->jpar_max;
    fa.small_max = c->small_max;
    fa.split = c->o.split_j;
    fa.slots_ipar = c->slots_ipar;
    fa.slots_jpar = c->slots_jpar;
    fa.slots_small = c->slots_small;
    fa.part_cap = c->part_cap;
    fa.part = c->d_part;
    fa.jcnt = c->d_jcnt;
    fa.out = out;
    fa.eps2 = c->eps * c->eps;
    fa.err = &c->d_ctrl->err;
    fa.precision = c->o.precision;
    fa.summation = c->o.summation;
    fa.slots_sum = c->sum.slots;
    if (na_dev) fa.plan_dev = c->d_plan;   // written by the scheduler with *na_dev
    else fa.plan = make_force_plan(fa, na_host);
    return fa;
}

ForceOut res_out(nb_ctx *c)
{
    ForceOut o;
    o.acc = c->d_res;
    o.jerk = c->d_res + 3LL * c->n;
    o.pot = c->d_res + 6LL * c->n;
    return o;
}

// Enqueues the force on `act`.  With na_dev the block size and the plan are
// read on the device (the scheduler wrote them): every force kernel of the
// precision is launched with a persistent grid and all but the one serving the
// block exit at once.  Otherwise the host plans, and only the kernel that
// serves na_host is launched, sized to its work.
void enqueue_force(nb_ctx *c, const int *act, int na_host, const int *na_dev, ForceOut out)
{
    const ForceArgs fa = force_args(c, act, na_host, na_dev, out);
    const bool f64 = c->o.precision == NB_FP64;
    int gi = c->slots_ipar, gj = c->slots_jpar, gs = f64 ? 0 : c->slots_small;
    if (!na_dev) {
        if (na_host <= 0) return;
        const Plan &p = fa.plan.p;
        gi = gj = gs = 0;
        if (fa.plan.regime == kRegJpar) gj = p.items < c->slots_jpar ? p.items : c->slots_jpar;
        else if (fa.plan.regime == kRegSmall) gs = p.items < c->slots_small ? p.items : c->slots_small;
        else gi = p.items < c->slots_ipar ? p.items : c->slots_ipar;
    }
    const bool summed = c->o.summation != NB_SUM_COMPENSATED;
    const int gsum = summed ? grid_summed(fa, c->sum) : 0;
    if (summed && gsum <= 0) return;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    const bool timed = c->profiling && !c->capturing;
    if (timed) {
        for (int q = 0; q < 2; ++q) {
            if (!c->ev_free.empty()) {
                ev[q] = c->ev_free.back();
                c->ev_free.pop_back();
            } else if (cudaEventCreate(&ev[q]) != cudaSuccess) {
                ev[q] = nullptr;
            }
        }
        if (ev[0] && ev[1]) cudaEventRecord(ev[0], c->st);
    }
    if (summed) {
        c->launches += launch_force_summed(fa, c->jds, c->sum, gsum, c->st);
    } else if (f64) {
        launch_force_f64(fa, c->jf, c->eps > 0.0, gi, gj, c->st);
        c->launches += (gi > 0) + (gj > 0) + 1;
    } else {
        c->launches += launch_force_ds(fa, c->jds, c->eps > 0.0, gi, gj, gs, c->st);
    }
    if (timed) {
        if (ev[0] && ev[1]) {
            cudaEventRecord(ev[1], c->st);
            c->ev_pending.push_back(ev[0]);
            c->ev_pending.push_back(ev[1]);
        } else {
            for (cudaEvent_t e : ev)
                if (e) c->ev_free.push_back(e);
        }
    }
}

// The device-driven block step: schedule, predict all, force, correct.
void enqueue_step(nb_ctx *c)
{
    launch_schedule(c->S, c->d_ctrl, c->d_blockmin, c->d_blockcnt, c->d_act, c->nsched,
                    force_args(c, c->d_act, 0, &c->d_ctrl->n_active, res_out(c)), c->d_plan,
                    c->o.precision, c->jds, c->jf, c->st);
    enqueue_force(c, c->d_act, 0, &c->d_ctrl->n_active, res_out(c));
    launch_correct(c->S, c->d_act, 0, &c->d_ctrl->n_active, 0, &c->d_ctrl->t_next, c->d_res,
                   c->d_res + 3LL * c->n, c->o.eta, c->o.level_min, c->o.level_fixed,
                   &c->d_ctrl->err, c->sms, c->st);
    c->launches += 2 + 1;  // scheduler with the predictor, corrector (force counted above)
}

int set_t_end(nb_ctx *c, long long t_end)
{
    if (c->t_end_dev == t_end) return NB_OK;
    CK(cudaStreamSynchronize(c->st));
    c->h_ctrl->t_end = t_end;
    CK(cudaMemcpyAsync(&c->d_ctrl->t_end, &c->h_ctrl->t_end, sizeof(long long),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->t_end_dev = t_end;
    return NB_OK;
}

template <typename T>
int dalloc(nb_ctx *c, T **p, long long count)
{
    if (count < 1) count = 1;
    cudaError_t e = cudaMalloc((void **)p, sizeof(T) * (size_t)count);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return fail(c, NB_ENOMEM, "cudaMalloc of %lld bytes failed: %s",
                    (long long)(sizeof(T) * count), cudaGetErrorString(e));
    }
    return NB_OK;
}

void release(nb_ctx *c)
{
    if (c->st) cudaStreamSynchronize(c->st);
    if (c->step_exec) cudaGraphExecDestroy(c->step_exec);
    void *ptrs[] = {c->d_x, c->d_v, c->d_a, c->d_k, c->d_m, c->d_t, c->d_lev, c->jds.pos_hi,
                    c->jds.pos_lo, c->jds.vel, c->jf.pos, c->jf.vel, c->d_res, c->d_part,
                    c->d_act, c->d_idx, c->d_all, c->d_bitmap, c->d_ctrl, c->d_blockmin,
                    c->d_blockcnt, c->d_epart, c->d_stage, c->d_ck, c->d_seg, c->d_fin, c->d_tfin,
                    c->d_jcnt, c->d_plan, c->d_cot, c->vrec.ph, c->vrec.pl, c->vrec.v, c->vrec.ab, c->vrec.kb,
                    c->vrec64.x, c->vrec64.v, c->vrec64.ab, c->vrec64.kb, c->d_bounds, c->d_sort,
                    c->d_run_part, c->d_run_mins, c->d_run_counts, c->d_run_maxs, c->d_run_bar};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_pending) cudaEventDestroy(e);
    if (c->h_ctrl) cudaFreeHost(c->h_ctrl);
    if (c->own_stream && c->st) cudaStreamDestroy(c->st);
}

// Full sweep on all particles into d_res (predicted state must be current).
void enqueue_full_sweep(nb_ctx *c) { enqueue_force(c, c->d_all, c->n, nullptr, res_out(c)); }

// A State view of 12n doubles laid out x, v, a, k (SoA), with the context's
// masses, times and levels.
State state_view(nb_ctx *c, double *base)
{
    State s = c->S;
    const long long n3 = 3LL * c->n;
    s.x = base;
    s.v = base + n3;
    s.a = base + 2 * n3;
    s.k = base + 3 * n3;
    return s;
}

// Buffers of the force VJP (records, cotangents, results), allocated on first use.
int vjp_alloc(nb_ctx *c)
{
    if (c->d_cot) return NB_OK;
    const long long N = c->n;
    int rc;
    if ((rc = dalloc(c, &c->d_cot, 20 * N))) return rc;
    if (c->o.precision == NB_FP64) {
        if ((rc = dalloc(c, &c->vrec64.x, N)) || (rc = dalloc(c, &c->vrec64.v, N)) ||
            (rc = dalloc(c, &c->vrec64.ab, N)) || (rc = dalloc(c, &c->vrec64.kb, N)))
            return rc;
    } else {
        if ((rc = dalloc(c, &c->vrec.ph, N)) || (rc = dalloc(c, &c->vrec.pl, N)) ||
            (rc = dalloc(c, &c->vrec.v, N)) || (rc = dalloc(c, &c->vrec.ab, N)) ||
            (rc = dalloc(c, &c->vrec.kb, N)))
            return rc;
    }
    c->slots_vjp = vjp_slots(c->o.precision, c->sms);
    return NB_OK;
}

double *cot(nb_ctx *c, int which)  // 0 xb, 1 vb, 2 ab, 3 kb, 4 mb, 5 xg, 6 vg, 7 mg
{
    const long long n3 = 3LL * c->n, N = c->n;
    const long long off[8] = {0, n3, 2 * n3, 3 * n3, 4 * n3, 4 * n3 + N, 5 * n3 + N, 6 * n3 + N};
    return c->d_cot + off[which];
}

// VJP of every particle's acc and jerk at the records in c->vrec / vrec64,
// results into xg, vg, mg.
void enqueue_vjp(nb_ctx *c)
{
    VjpArgs va{};
    va.n = c->n;
    va.eps2 = c->eps * c->eps;
    va.slots = c->slots_vjp;
    va.part_cap = c->part_cap;
    va.part = c->d_part;
    va.rec = c->vrec;
    va.rec64 = c->vrec64;
    va.m = c->d_m;
    va.xbar = cot(c, 5);
    va.vbar = cot(c, 6);
    va.mbar = cot(c, 7);
    c->launches += launch_force_vjp(va, c->o.precision, c->eps > 0.0, c->st);
}

int copy_results_out(nb_ctx *c, int na, double *acc, double *jerk, double *pot, cudaMemcpyKind k)
{
    if (na <= 0) return NB_OK;
    if (acc) CK(cudaMemcpyAsync(acc, c->d_res, sizeof(double) * 3 * (size_t)na, k, c->st));
    if (jerk)
        CK(cudaMemcpyAsync(jerk, c->d_res + 3LL * c->n, sizeof(double) * 3 * (size_t)na, k, c->st));
    if (pot) CK(cudaMemcpyAsync(pot, c->d_res + 6LL * c->n, sizeof(double) * (size_t)na, k, c->st));
    return NB_OK;
}

// nb_run in one persistent launch (k_run.cu) when the system is small enough:
// NB_OK or an error code, or kRunNotUsed when this context uses the
// per-stage graph instead.
constexpr int kRunNotUsed = 1;

int run_persistent(nb_ctx *c, long long te, long long max_steps)
{
    if (c->n > kRunMaxN || c->o.precision != NB_DS || (c->o.flags & NB_RUN_GRAPH) ||
        (c->o.summation != NB_SUM_COMPENSATED && c->o.summation != NB_SUM_FIXED))
        return kRunNotUsed;
    if (!c->d_run_bar) {
        int bps = 0;
        if (occupancy_run(c->o.summation, &bps) ||
            run_layout(c->n, c->sms, bps, &c->run_ncta, &c->run_per))
            return kRunNotUsed;
        const long long C = c->run_ncta, N = c->n;
        int rc;
        if ((rc = dalloc(c, &c->d_run_part, C * N * 2 * kComp)) || (rc = dalloc(c, &c->d_run_mins, C)) ||
            (rc = dalloc(c, &c->d_run_counts, C)) || (rc = dalloc(c, &c->d_run_maxs, 2 * C)) ||
            (rc = dalloc(c, &c->d_run_bar, 1))) {
            // all or nothing: a later call starts again from scratch
            void *ps[] = {c->d_run_part, c->d_run_mins, c->d_run_counts, c->d_run_maxs, c->d_run_bar};
            for (void *q : ps)
                if (q) cudaFree(q);
            c->d_run_part = nullptr;
            c->d_run_mins = nullptr;
            c->d_run_counts = nullptr;
            c->d_run_maxs = nullptr;
            c->d_run_bar = nullptr;
            return rc;
        }
    }
    RunArgs ra{};
    ra.s = c->S;
    ra.j = c->jds;
    ra.ctrl = c->d_ctrl;
    ra.n = c->n;
    ra.ncta = c->run_ncta;
    ra.per = c->run_per;
    ra.eps2f = (float)(c->eps * c->eps);
    ra.eta = c->o.eta;
    ra.level_min = c->o.level_min;
    ra.level_fixed = c->o.level_fixed;
    ra.t_end = te;
    ra.max_steps = max_steps;
    ra.act = c->d_act;
    ra.mins = c->d_run_mins;
    ra.counts = c->d_run_counts;
    ra.maxs = c->d_run_maxs;
    ra.part = c->d_run_part;
    ra.bar = c->d_run_bar;
    CK(cudaMemsetAsync(c->d_run_bar, 0, sizeof(unsigned long long), c->st));
    const cudaError_t e = launch_run(ra, c->o.summation, c->st);
    if (e == cudaErrorCooperativeLaunchTooLarge) {
        // not every CTA can be resident now (a shared GPU): use the graph
        cudaGetLastError();
        return kRunNotUsed;
    }
    if (e != cudaSuccess) return fail(c, NB_ECUDA, "persistent run launch: %s", cudaGetErrorString(e));
    c->launches += 1;
    return sync_ctrl(c);
}

}  // namespace

extern "C" {

void nb_default_opts(nb_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->eta = 0.01;
    o->eta_init = 0.01;
    o->level_min = 3;
    o->level_fixed = 0;
    o->precision = NB_DS;
    o->force_mode = NB_FORCE_AUTO;
    o->split_j = 0;
    o->flags = 0;
    o->summation = NB_SUM_COMPENSATED;
    o->stream = nullptr;
}

int64_t nb_num_particles(const nb_ctx *c) { return c ? c->n : -1; }

const char *nb_last_error(const nb_ctx *c)
{
    if (c) return c->err.c_str();
    return g_init_err.empty() ? kNoCtx : g_init_err.c_str();
}

void nb_free(nb_ctx *c)
{
    if (!c) return;
    release(c);
    delete c;
}

// dev: m, x, v are device arrays (checked on the device) instead of host arrays.
static int init_impl(nb_ctx *c, int64_t n, const double *m, const double *x, const double *v,
                     double eps, const nb_opts *opts, bool dev)
{
    nb_opts o;
    nb_default_opts(&o);
    if (opts) o = *opts;
    if (n < 1 || n > INT_MAX / 8) return fail(c, NB_EINVAL, "n=%lld out of range", (long long)n);
    if (!m || !x || !v) return fail(c, NB_EINVAL, "m, x and v are required");
    if (!std::isfinite(eps) || eps < 0.0) return fail(c, NB_EINVAL, "eps must be finite and >= 0");
    if (!(o.eta > 0.0) || !std::isfinite(o.eta) || !(o.eta_init > 0.0) || !std::isfinite(o.eta_init))
        return fail(c, NB_EINVAL, "eta and eta_init must be positive");
    if (o.level_min < 0 || o.level_min > kTickBits)
        return fail(c, NB_EINVAL, "level_min must lie in [0, 40]");
    if (o.level_fixed < 0 || o.level_fixed > kTickBits ||
        (o.level_fixed > 0 && o.level_fixed < o.level_min))
        return fail(c, NB_EINVAL, "level_fixed must be 0 or in [level_min, 40]");
    if (o.precision != NB_DS && o.precision != NB_FP64)
        return fail(c, NB_EINVAL, "precision must be NB_DS or NB_FP64");
    if (o.force_mode < NB_FORCE_AUTO || o.force_mode > NB_FORCE_JPAR)
        return fail(c, NB_EINVAL, "bad force_mode");
    if (o.split_j < 0 || (o.flags & ~(NB_INIT_NO_FORCE | NB_RUN_GRAPH)) != 0)
        return fail(c, NB_EINVAL, "bad split_j or flags");
    if (o.summation < NB_SUM_COMPENSATED || o.summation > NB_SUM_FP32_SORTED)
        return fail(c, NB_EINVAL, "bad summation");
    if (o.summation != NB_SUM_COMPENSATED && o.precision != NB_DS)
        return fail(c, NB_EINVAL, "summation variants need precision NB_DS");
    if (o.summation == NB_SUM_FIXED) {
        const float e2 = (float)(eps * eps);
        if (!(e2 >= 0x1p-126f) || std::isinf(e2))
            return fail(c, NB_EINVAL, "NB_SUM_FIXED needs eps^2 to be a normal single-precision number");
    }
    if (!dev) {
        if (!finite_all(m, n) || !finite_all(x, 3 * n) || !finite_all(v, 3 * n))
            return fail(c, NB_EINVAL, "non-finite input");
        for (int64_t i = 0; i < n; ++i)
            if (m[i] < 0.0) return fail(c, NB_EINVAL, "negative mass at %lld", (long long)i);
    }

    c->n = (int)n;
    c->eps = eps;
    c->o = o;
    if (o.stream) {
        c->st = (cudaStream_t)o.stream;
    } else {
        CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
        c->own_stream = true;
    }
    int device = 0;
    CK(cudaGetDevice(&device));
    CK(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device));
    const bool f64 = o.precision == NB_FP64;
    int bi = 0, bj = 0, bs = 0;
    if (occupancy_force(o.precision, kRegIpar, &bi) || occupancy_force(o.precision, kRegJpar, &bj) ||
        occupancy_force(o.precision, kRegSmall, &bs))
        return fail(c, NB_ECUDA, "occupancy query failed");
    c->slots_ipar = c->sms * (bi > 0 ? bi : 1);
    c->slots_jpar = c->sms * (bj > 0 ? bj : 1);
    c->slots_small = c->sms * (bs > 0 ? bs : 1);
    c->jpar_max = o.force_mode == NB_FORCE_IPAR ? 0
                  : o.force_mode == NB_FORCE_JPAR ? INT_MAX
                                                  : (f64 ? kJparMaxActive64 : kJparMaxActive);
    c->small_max = f64 || o.force_mode == NB_FORCE_JPAR ? 0 : kSmallMaxActive;
    if (o.summation != NB_SUM_COMPENSATED) {
        int bsum = 0;
        if (occupancy_sum(o.summation, &bsum)) return fail(c, NB_ECUDA, "occupancy query failed");
        c->sum.mode = o.summation;
        c->sum.slots = c->sms * (bsum > 0 ? bsum : 1);
        if (o.summation == NB_SUM_FP32_SORTED) {
            // keyed items: 16 n bytes per resident CTA, at most 4 GiB in all
            const long long per = 16LL * n, cap = (4LL << 30) / per;
            if (cap < c->sum.slots) c->sum.slots = (int)(cap > 0 ? cap : 1);
        }
    }
    const long long iblk = kIparNT * (f64 ? kIparR64 : kIparR);
    // Partials: up to 16 slots' worth of i-blocks, and four slices of all n.
    long long cap = 16LL * c->slots_ipar * iblk;
    if (cap < 4LL * n) cap = 4LL * n;
    const long long cap_j = 8LL * c->slots_jpar * kJparIC;
    c->part_cap = (long long)kComp * (cap > cap_j ? cap : cap_j);
    c->nsched = schedule_blocks(c->n);

    int rc;
    const long long N = c->n;
    if ((rc = dalloc(c, &c->d_x, 3 * N)) || (rc = dalloc(c, &c->d_v, 3 * N)) ||
        (rc = dalloc(c, &c->d_a, 3 * N)) || (rc = dalloc(c, &c->d_k, 3 * N)) ||
        (rc = dalloc(c, &c->d_m, N)) || (rc = dalloc(c, &c->d_t, N)) ||
        (rc = dalloc(c, &c->d_lev, N)) || (rc = dalloc(c, &c->d_res, 7 * N)) ||
        (rc = dalloc(c, &c->d_part, c->part_cap)) || (rc = dalloc(c, &c->d_act, N)) ||
        (rc = dalloc(c, &c->d_idx, N)) || (rc = dalloc(c, &c->d_all, N)) ||
        (rc = dalloc(c, &c->d_bitmap, (N + 31) / 32)) || (rc = dalloc(c, &c->d_ctrl, 1)) ||
        (rc = dalloc(c, &c->d_blockmin, c->nsched)) || (rc = dalloc(c, &c->d_blockcnt, c->nsched)) ||
        (rc = dalloc(c, &c->d_epart, 2LL * energy_blocks(c->n))) ||
        (rc = dalloc(c, &c->d_stage, 7 * N)) || (rc = dalloc(c, &c->d_jcnt, N)) ||
        (rc = dalloc(c, &c->d_plan, 1)))
        return rc;
    if (o.summation == NB_SUM_FIXED) {
        if ((rc = dalloc(c, &c->d_bounds, 2))) return rc;
        c->sum.bounds = c->d_bounds;
    } else if (o.summation == NB_SUM_FP32_SORTED) {
        if ((rc = dalloc(c, &c->d_sort, 2LL * N * c->sum.slots))) return rc;
        c->sum.scratch = c->d_sort;
    }
    if (f64) {
        if ((rc = dalloc(c, &c->jf.pos, N)) || (rc = dalloc(c, &c->jf.vel, N))) return rc;
    } else {
        if ((rc = dalloc(c, &c->jds.pos_hi, N)) || (rc = dalloc(c, &c->jds.pos_lo, N)) ||
            (rc = dalloc(c, &c->jds.vel, N)))
            return rc;
    }
    cudaError_t he = cudaMallocHost((void **)&c->h_ctrl, sizeof(Ctrl));
    if (he != cudaSuccess) {
        c->h_ctrl = nullptr;
        return fail(c, NB_ENOMEM, "cudaMallocHost failed: %s", cudaGetErrorString(he));
    }
    std::memset(c->h_ctrl, 0, sizeof(Ctrl));
    c->h_ctrl->t_end = LLONG_MAX;
    c->t_end_dev = LLONG_MAX;

    c->S.x = c->d_x;
    c->S.v = c->d_v;
    c->S.a = c->d_a;
    c->S.k = c->d_k;
    c->S.m = c->d_m;
    c->S.t = c->d_t;
    c->S.lev = c->d_lev;
    c->S.n = c->n;

    CK(cudaMemcpyAsync(c->d_ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st));
    CK(cudaMemsetAsync(c->d_a, 0, sizeof(double) * 3 * N, c->st));
    CK(cudaMemsetAsync(c->d_k, 0, sizeof(double) * 3 * N, c->st));
    CK(cudaMemsetAsync(c->d_t, 0, sizeof(long long) * N, c->st));
    CK(cudaMemsetAsync(c->d_jcnt, 0, sizeof(int) * N, c->st));
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(c->d_m, m, sizeof(double) * N, kind, c->st));
    CK(cudaMemcpyAsync(c->d_stage, x, sizeof(double) * 3 * N, kind, c->st));
    CK(cudaMemcpyAsync(c->d_stage + 3 * N, v, sizeof(double) * 3 * N, kind, c->st));
    if (dev) {
        // the host checks of nb_init, on the device; reported by the final sync
        launch_check_input(c->d_m, N, true, &c->d_ctrl->err, c->st);
        launch_check_input(c->d_stage, 6 * N, false, &c->d_ctrl->err, c->st);
        c->launches += 2;
    }
    launch_scatter_state(c->S, c->d_stage, c->d_stage + 3 * N, nullptr, nullptr, c->st);
    launch_iota(c->d_all, c->n, c->st);
    launch_predict(c->S, 0, nullptr, nullptr, o.precision, c->jds, c->jf, c->st);
    if (o.flags & NB_INIT_NO_FORCE)
        CK(cudaMemsetAsync(c->d_res, 0, sizeof(double) * 6 * N, c->st));  // a = k = 0
    else
        enqueue_full_sweep(c);
    launch_initial_steps(c->S, c->d_res, c->d_res + 3 * N, o.eta_init, o.level_min, o.level_fixed,
                         &c->d_ctrl->err, c->st);
    c->launches += 4;
    CK(cudaGetLastError());
    c->t_pred = 0;
    c->force_valid = false;
    return sync_ctrl(c);
}

int nb_init(nb_ctx **ctx, int64_t n, const double *m, const double *x, const double *v,
            double eps, const nb_opts *opts)
{
    const Range range_("nb_init");
    g_init_err.clear();
    if (!ctx) {
        g_init_err = "ctx is NULL";
        return NB_EINVAL;
    }
    *ctx = nullptr;
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) {
        g_init_err = "out of host memory";
        return NB_ENOMEM;
    }
    const int rc = init_impl(c, n, m, x, v, eps, opts, false);
    if (rc != NB_OK) {
        g_init_err = c->err;  // readable through nb_last_error(NULL)
        nb_free(c);
        return rc;
    }
    *ctx = c;
    return NB_OK;
}

int nb_init_dev(nb_ctx **ctx, int64_t n, const double *d_m, const double *d_x, const double *d_v,
                double eps, const nb_opts *opts)
{
    const Range range_("nb_init_dev");
    g_init_err.clear();
    if (!ctx) {
        g_init_err = "ctx is NULL";
        return NB_EINVAL;
    }
    *ctx = nullptr;
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) {
        g_init_err = "out of host memory";
        return NB_ENOMEM;
    }
    const int rc = init_impl(c, n, d_m, d_x, d_v, eps, opts, true);
    if (rc != NB_OK) {
        g_init_err = c->err;
        nb_free(c);
        return rc;
    }
    *ctx = c;
    return NB_OK;
}

int nb_predict(nb_ctx *c, double t)
{
    const Range range_("nb_predict");
    if (!c) return NB_EINVAL;
    long long ticks;
    if (!time_to_ticks(t, &ticks)) return fail(c, NB_EINVAL, "t=%.17g is not on the 2^-40 grid", t);
    launch_predict(c->S, ticks, nullptr, nullptr, c->o.precision, c->jds, c->jf, c->st);
    CK(cudaGetLastError());
    c->launches += 1;
    c->t_pred = ticks;
    c->force_valid = false;
    return NB_OK;
}

int nb_force(nb_ctx *c, const int32_t *idx, int32_t na, double *acc, double *jerk, double *pot)
{
    const Range range_("nb_force");
    if (!c) return NB_EINVAL;
    int rc = check_indices_host(c, idx, na);
    if (rc) return rc;
    if (na > 0) {
        CK(cudaMemcpyAsync(c->d_idx, idx, sizeof(int) * (size_t)na, cudaMemcpyHostToDevice, c->st));
        enqueue_force(c, c->d_idx, na, nullptr, res_out(c));
        CK(cudaGetLastError());
        if ((rc = copy_results_out(c, na, acc, jerk, pot, cudaMemcpyDeviceToHost))) return rc;
    }
    if ((rc = sync_ctrl(c))) return rc;
    c->force_valid = true;
    c->force_na = na;
    c->force_t = c->t_pred;
    return NB_OK;
}

int nb_force_dev(nb_ctx *c, const int32_t *d_idx, int32_t na, double *d_acc, double *d_jerk,
                 double *d_pot)
{
    const Range range_("nb_force_dev");
    if (!c) return NB_EINVAL;
    if (na < 0 || na > c->n) return fail(c, NB_EINVAL, "n_active=%d outside [0, %d]", na, c->n);
    if (na > 0 && !d_idx) return fail(c, NB_EINVAL, "active_idx is NULL");
    if (na > 0) {
        // Validation and force (on the caller's indices) go out together, and
        // the one synchronisation follows the force: the force kernels clamp every
        // index into [0, n), so a bad index costs only wasted work, and the
        // caller's outputs are written only once the indices proved valid.
        CK(cudaMemsetAsync(c->d_bitmap, 0, sizeof(unsigned) * (size_t)((c->n + 31) / 32), c->st));
        launch_validate(d_idx, na, c->n, c->d_bitmap, &c->d_ctrl->err, c->st);
        c->launches += 1;
        enqueue_force(c, d_idx, na, nullptr, res_out(c));
        CK(cudaGetLastError());
        int rc = sync_ctrl(c);
        if (rc) return rc;
        if ((rc = copy_results_out(c, na, d_acc, d_jerk, d_pot, cudaMemcpyDeviceToDevice))) return rc;
    }
    c->force_valid = true;
    c->force_na = na;
    c->force_t = c->t_pred;
    return NB_OK;
}

int nb_correct(nb_ctx *c, const int32_t *idx, int32_t na, double t, const double *acc,
               const double *jerk)
{
    const Range range_("nb_correct");
    if (!c) return NB_EINVAL;
    long long ticks;
    if (!time_to_ticks(t, &ticks)) return fail(c, NB_EINVAL, "t=%.17g is not on the 2^-40 grid", t);
    int rc = check_indices_host(c, idx, na);
    if (rc) return rc;
    if ((acc == nullptr) != (jerk == nullptr))
        return fail(c, NB_EINVAL, "acc and jerk must be given together");
    if (!acc && (!c->force_valid || c->force_na != na || c->force_t != ticks))
        return fail(c, NB_ESTATE, "nb_correct needs a preceding nb_force on %d particles at t", na);
    if (na == 0) return NB_OK;
    const long long N = c->n;
    const double *an = c->d_res, *kn = c->d_res + 3 * N;
    if (acc) {
        if (!finite_all(acc, 3LL * na) || !finite_all(jerk, 3LL * na))
            return fail(c, NB_EINVAL, "non-finite acc or jerk");
        CK(cudaMemcpyAsync(c->d_stage, acc, sizeof(double) * 3 * (size_t)na, cudaMemcpyHostToDevice,
                           c->st));
        CK(cudaMemcpyAsync(c->d_stage + 3 * N, jerk, sizeof(double) * 3 * (size_t)na,
                           cudaMemcpyHostToDevice, c->st));
        an = c->d_stage;
        kn = c->d_stage + 3 * N;
    }
    CK(cudaMemcpyAsync(c->d_idx, idx, sizeof(int) * (size_t)na, cudaMemcpyHostToDevice, c->st));
    launch_correct(c->S, c->d_idx, na, nullptr, ticks, nullptr, an, kn, c->o.eta, c->o.level_min,
                   c->o.level_fixed, &c->d_ctrl->err, c->sms, c->st);
    CK(cudaGetLastError());
    c->launches += 1;
    c->force_valid = false;
    if ((rc = sync_ctrl(c))) return rc;
    if (ticks > c->h_ctrl->t_now) {
        // the system time follows the latest corrected block
        c->h_ctrl->t_now = ticks;
        CK(cudaMemcpyAsync(&c->d_ctrl->t_now, &c->h_ctrl->t_now, sizeof(long long),
                           cudaMemcpyHostToDevice, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return NB_OK;
}

int nb_step(nb_ctx *c, double *t_out, int32_t *na_out)
{
    const Range range_("nb_step");
    if (!c) return NB_EINVAL;
    int rc = set_t_end(c, LLONG_MAX);
    if (rc) return rc;
    enqueue_step(c);
    CK(cudaGetLastError());
    c->force_valid = false;
    if (t_out || na_out) {
        if ((rc = sync_ctrl(c))) return rc;
        if (t_out) *t_out = (double)c->h_ctrl->t_now * 0x1p-40;
        if (na_out) *na_out = c->h_ctrl->n_active;
    }
    return NB_OK;
}

int nb_run(nb_ctx *c, double t_end, int64_t max_steps, int64_t *steps_out, int64_t *inter_out)
{
    const Range range_("nb_run");
    if (!c) return NB_EINVAL;
    long long te;
    if (!time_to_ticks(t_end, &te)) return fail(c, NB_EINVAL, "t_end is not on the 2^-40 grid");
    if (max_steps < 0) return fail(c, NB_EINVAL, "max_steps < 0");
    int rc = set_t_end(c, te);
    if (rc) return rc;
    if ((rc = sync_ctrl(c))) return rc;
    const long long steps0 = c->h_ctrl->steps, inter0 = c->h_ctrl->interactions;
    c->force_valid = false;
    rc = run_persistent(c, te, max_steps);
    if (rc != kRunNotUsed) {
        if (rc) return rc;
        if (steps_out) *steps_out = c->h_ctrl->steps - steps0;
        if (inter_out) *inter_out = c->h_ctrl->interactions - inter0;
        return set_t_end(c, LLONG_MAX);
    }
    if (!c->step_exec) {
        cudaGraph_t g;
        CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
        const long long l0 = c->launches;
        c->capturing = true;
        enqueue_step(c);
        c->capturing = false;
        c->step_nodes = c->launches - l0;
        c->launches = l0;
        cudaError_t ce = cudaStreamEndCapture(c->st, &g);
        if (ce != cudaSuccess) return fail(c, NB_ECUDA, "graph capture: %s", cudaGetErrorString(ce));
        const cudaError_t e = cudaGraphInstantiate(&c->step_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->step_exec = nullptr;
            return fail(c, NB_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    c->force_valid = false;
    long long done = 0;
    const int batch = 32;
    while (done < max_steps) {
        const long long k = (max_steps - done) < batch ? (max_steps - done) : batch;
        for (long long s = 0; s < k; ++s) {
            CK(cudaGraphLaunch(c->step_exec, c->st));
            c->launches += c->step_nodes;
        }
        if ((rc = sync_ctrl(c))) return rc;
        done = c->h_ctrl->steps - steps0;
        if (c->h_ctrl->n_active == 0) break;
    }
    if (steps_out) *steps_out = c->h_ctrl->steps - steps0;
    if (inter_out) *inter_out = c->h_ctrl->interactions - inter0;
    return set_t_end(c, LLONG_MAX);
}

int nb_check_wait(nb_ctx *c, int32_t ms)
{
    if (!c) return NB_EINVAL;
    const Range range_("nb_check_wait");
    if (ms < 1 || ms > 2000) return fail(c, NB_EINVAL, "ms=%d outside [1, 2000]", ms);
    int dev = 0, khz = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
    unsigned long long *counter = nullptr;
    int rc;
    if ((rc = dalloc(c, &counter, 1))) return rc;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), c->st);
    if (e == cudaSuccess) e = launch_check_wait(counter, (long long)ms * (khz > 0 ? khz : 2000000), c->d_ctrl, c->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->st);
    cudaFree(counter);
    if (e != cudaSuccess) return fail(c, NB_ECUDA, "wait check: %s", cudaGetErrorString(e));
    c->launches += 1;
    return sync_ctrl(c);
}

int nb_energy(nb_ctx *c, double *ekin, double *epot)
{
    const Range range_("nb_energy");
    if (!c) return NB_EINVAL;
    launch_predict(c->S, 0, &c->d_ctrl->t_now, nullptr, c->o.precision, c->jds, c->jf, c->st);
    enqueue_full_sweep(c);
    launch_energy(c->S, &c->d_ctrl->t_now, c->d_res + 6LL * c->n, c->d_epart, c->d_ctrl, c->st);
    CK(cudaGetLastError());
    c->launches += 1 + 2;
    c->force_valid = false;
    const int rc = sync_ctrl(c);
    if (rc) return rc;
    if (ekin) *ekin = c->h_ctrl->ekin;
    if (epot) *epot = c->h_ctrl->epot;
    return NB_OK;
}

int nb_get_state(nb_ctx *c, double *x, double *v, double *a, double *k, int64_t *t, int32_t *lev)
{
    const Range range_("nb_get_state");
    if (!c) return NB_EINVAL;
    const long long N = c->n;
    launch_gather_state(c->S, c->d_stage, c->d_stage + 3 * N, nullptr, nullptr, c->st);
    CK(cudaGetLastError());
    if (x) CK(cudaMemcpyAsync(x, c->d_stage, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->st));
    if (v)
        CK(cudaMemcpyAsync(v, c->d_stage + 3 * N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (a || k) {
        launch_gather_state(c->S, nullptr, nullptr, c->d_stage, c->d_stage + 3 * N, c->st);
        CK(cudaGetLastError());
        if (a) CK(cudaMemcpyAsync(a, c->d_stage, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->st));
        if (k)
            CK(cudaMemcpyAsync(k, c->d_stage + 3 * N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost,
                               c->st));
    }
    if (t) CK(cudaMemcpyAsync(t, c->d_t, sizeof(long long) * N, cudaMemcpyDeviceToHost, c->st));
    if (lev) CK(cudaMemcpyAsync(lev, c->d_lev, sizeof(int) * N, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NB_OK;
}

int nb_get_state_dev(nb_ctx *c, double *d_x, double *d_v, double *d_a, double *d_k, int64_t *d_t,
                     int32_t *d_lev)
{
    const Range range_("nb_get_state_dev");
    if (!c) return NB_EINVAL;
    const long long N = c->n;
    if (d_x || d_v || d_a || d_k) {
        launch_gather_state(c->S, d_x, d_v, d_a, d_k, c->st);
        c->launches += 1;
    }
    if (d_t) CK(cudaMemcpyAsync(d_t, c->d_t, sizeof(long long) * N, cudaMemcpyDeviceToDevice, c->st));
    if (d_lev) CK(cudaMemcpyAsync(d_lev, c->d_lev, sizeof(int) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaGetLastError());
    return NB_OK;
}

int nb_set_state(nb_ctx *c, const double *x, const double *v, const double *a, const double *k,
                 const int64_t *t, const int32_t *lev)
{
    const Range range_("nb_set_state");
    if (!c) return NB_EINVAL;
    if (!x || !v || !a || !k || !t || !lev) return fail(c, NB_EINVAL, "all state arrays are required");
    const long long N = c->n;
    if (!finite_all(x, 3 * N) || !finite_all(v, 3 * N) || !finite_all(a, 3 * N) ||
        !finite_all(k, 3 * N))
        return fail(c, NB_EINVAL, "non-finite state");
    long long t_max = 0;
    for (long long i = 0; i < N; ++i) {
        if (lev[i] < c->o.level_min || lev[i] > kTickBits)
            return fail(c, NB_EINVAL, "level[%lld]=%d outside [%d, 40]", i, lev[i], c->o.level_min);
        const long long dt = 1LL << (kTickBits - lev[i]);
        if (t[i] < 0 || t[i] % dt != 0 || t[i] > (1LL << 62))
            return fail(c, NB_EINVAL, "t_ticks[%lld] is not a multiple of its step", i);
        if (t[i] > t_max) t_max = t[i];
    }
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpyAsync(c->d_stage, x, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_stage + 3 * N, v, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    launch_scatter_state(c->S, c->d_stage, c->d_stage + 3 * N, nullptr, nullptr, c->st);
    CK(cudaStreamSynchronize(c->st));
    CK(cudaMemcpyAsync(c->d_stage, a, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_stage + 3 * N, k, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    launch_scatter_state(c->S, nullptr, nullptr, c->d_stage, c->d_stage + 3 * N, c->st);
    CK(cudaMemcpyAsync(c->d_t, t, sizeof(long long) * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(c->d_lev, lev, sizeof(int) * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->h_ctrl->t_now = t_max;
    CK(cudaMemcpyAsync(&c->d_ctrl->t_now, &c->h_ctrl->t_now, sizeof(long long),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(c->st));
    c->force_valid = false;
    return NB_OK;
}

int nb_get_active(nb_ctx *c, int32_t *idx, int32_t cap, int32_t *na, int64_t *t_ticks)
{
    if (!c) return NB_EINVAL;
    int rc = sync_ctrl(c);
    if (rc) return rc;
    const int n_act = c->h_ctrl->n_active;
    if (na) *na = n_act;
    if (t_ticks) *t_ticks = c->h_ctrl->t_now;
    const int cnt = n_act < cap ? n_act : cap;
    if (idx && cnt > 0) {
        CK(cudaMemcpyAsync(idx, c->d_act, sizeof(int) * (size_t)cnt, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
    }
    return NB_OK;
}

int nb_force_vjp(nb_ctx *c, const double *abar, const double *kbar, double *xbar, double *vbar,
                 double *mbar)
{
    const Range range_("nb_force_vjp");
    if (!c) return NB_EINVAL;
    if (!abar || !kbar) return fail(c, NB_EINVAL, "abar and kbar are required");
    const long long N = c->n;
    if (!finite_all(abar, 3 * N) || !finite_all(kbar, 3 * N))
        return fail(c, NB_EINVAL, "non-finite cotangent");
    int rc = vjp_alloc(c);
    if (rc) return rc;
    CK(cudaMemcpyAsync(cot(c, 2), abar, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpyAsync(cot(c, 3), kbar, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, c->st));
    launch_adj_initial_rec(c->S, cot(c, 2), cot(c, 3), c->o.precision, c->vrec, c->vrec64, c->st);
    c->launches += 1;
    enqueue_vjp(c);
    CK(cudaGetLastError());
    if (xbar) CK(cudaMemcpyAsync(xbar, cot(c, 5), sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->st));
    if (vbar) CK(cudaMemcpyAsync(vbar, cot(c, 6), sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->st));
    if (mbar) CK(cudaMemcpyAsync(mbar, cot(c, 7), sizeof(double) * N, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return NB_OK;
}

int nb_traj_forward(nb_ctx *c, int64_t steps, int64_t checkpoint_every)
{
    const Range range_("nb_traj_forward");
    if (!c) return NB_EINVAL;
    if (c->o.level_fixed <= 0)
        return fail(c, NB_ESTATE, "a trajectory needs the shared step (opts.level_fixed > 0)");
    if (steps < 1 || checkpoint_every < 1 || checkpoint_every > steps || steps > (1LL << 30))
        return fail(c, NB_EINVAL, "need 1 <= checkpoint_every <= steps");
    int rc = vjp_alloc(c);
    if (rc) return rc;
    const long long N = c->n, per = 12 * N;
    const long long nck = (steps + checkpoint_every - 1) / checkpoint_every;
    if (c->ck_slots < nck) {
        if (c->d_ck) cudaFree(c->d_ck);
        c->d_ck = nullptr;
        c->ck_slots = 0;
        if ((rc = dalloc(c, &c->d_ck, nck * per))) return rc;
        c->ck_slots = nck;
    }
    if (c->seg_slots < checkpoint_every) {
        if (c->d_seg) cudaFree(c->d_seg);
        c->d_seg = nullptr;
        c->seg_slots = 0;
        if ((rc = dalloc(c, &c->d_seg, checkpoint_every * per))) return rc;
        c->seg_slots = checkpoint_every;
    }
    if (!c->d_fin && ((rc = dalloc(c, &c->d_fin, per)) || (rc = dalloc(c, &c->d_tfin, N)))) return rc;
    if ((rc = set_t_end(c, LLONG_MAX))) return rc;
    // the initial acceleration and jerk are the force of the initial state
    launch_predict(c->S, 0, &c->d_ctrl->t_now, nullptr, c->o.precision, c->jds, c->jf, c->st);
    enqueue_full_sweep(c);
    launch_set_ak(c->S, c->d_res, c->d_res + 3 * N, c->st);
    c->launches += 2;
    for (long long s = 0; s < steps; ++s) {
        if (s % checkpoint_every == 0) {
            launch_copy_state(state_view(c, c->d_ck + (s / checkpoint_every) * per), c->S, c->st);
            c->launches += 1;
        }
        enqueue_step(c);
    }
    launch_copy_state(state_view(c, c->d_fin), c->S, c->st);
    c->launches += 1;
    CK(cudaMemcpyAsync(c->d_tfin, c->d_t, sizeof(long long) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaGetLastError());
    c->force_valid = false;
    if ((rc = sync_ctrl(c))) return rc;
    c->traj_valid = true;
    c->traj_steps = steps;
    c->traj_ckpt = checkpoint_every;
    return NB_OK;
}

// dev: the cotangents and the gradients are device arrays.
static int traj_backward_impl(nb_ctx *c, const double *xbar_T, const double *vbar_T, double *xbar0,
                              double *vbar0, double *mbar, bool dev)
{
    if (!c) return NB_EINVAL;
    if (!c->traj_valid) return fail(c, NB_ESTATE, "nb_traj_backward needs nb_traj_forward first");
    if (!xbar_T) return fail(c, NB_EINVAL, "xbar_T is required");
    const long long N = c->n, per = 12 * N;
    if (!dev && (!finite_all(xbar_T, 3 * N) || (vbar_T && !finite_all(vbar_T, 3 * N))))
        return fail(c, NB_EINVAL, "non-finite cotangent");
    int rc = sync_ctrl(c);
    if (rc) return rc;
    const Ctrl saved = *c->h_ctrl;
    const double dt = ldexp(1.0, -c->o.level_fixed);
    const cudaMemcpyKind kin = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind kout = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    CK(cudaMemcpyAsync(cot(c, 0), xbar_T, sizeof(double) * 3 * N, kin, c->st));
    if (vbar_T)
        CK(cudaMemcpyAsync(cot(c, 1), vbar_T, sizeof(double) * 3 * N, kin, c->st));
    else
        CK(cudaMemsetAsync(cot(c, 1), 0, sizeof(double) * 3 * N, c->st));
    if (dev) {
        launch_check_input(cot(c, 0), 6 * N, false, &c->d_ctrl->err, c->st);
        c->launches += 1;
    }
    CK(cudaMemsetAsync(cot(c, 2), 0, sizeof(double) * (6 * N + N), c->st));  // ab, kb, mb
    const long long steps = c->traj_steps, ck = c->traj_ckpt;
    const long long nseg = (steps + ck - 1) / ck;
    for (long long seg = nseg - 1; seg >= 0; --seg) {
        const long long s0 = seg * ck, len = (s0 + ck < steps ? ck : steps - s0);
        // recompute the segment's step states from its checkpoint
        launch_copy_state(c->S, state_view(c, c->d_ck + seg * per), c->st);
        c->launches += 1;
        for (long long q = 0; q < len; ++q) {
            launch_copy_state(state_view(c, c->d_seg + q * per), c->S, c->st);
            c->launches += 1;
            enqueue_step(c);
        }
        for (long long q = len - 1; q >= 0; --q) {
            launch_adj_pre(state_view(c, c->d_seg + q * per), dt, cot(c, 0), cot(c, 1), cot(c, 2),
                           cot(c, 3), c->o.precision, c->vrec, c->vrec64, c->st);
            enqueue_vjp(c);
            launch_adj_post(c->n, dt, cot(c, 0), cot(c, 1), cot(c, 2), cot(c, 3), cot(c, 4),
                            cot(c, 5), cot(c, 6), cot(c, 7), c->st);
            c->launches += 2;
        }
    }
    // the initial acceleration and jerk were the force of the initial state
    launch_adj_initial_rec(state_view(c, c->d_ck), cot(c, 2), cot(c, 3), c->o.precision, c->vrec,
                           c->vrec64, c->st);
    enqueue_vjp(c);
    launch_add3(c->n, cot(c, 0), cot(c, 5), cot(c, 1), cot(c, 6), cot(c, 4), cot(c, 7), c->st);
    c->launches += 2;
    CK(cudaGetLastError());
    if (xbar0) CK(cudaMemcpyAsync(xbar0, cot(c, 0), sizeof(double) * 3 * N, kout, c->st));
    if (vbar0) CK(cudaMemcpyAsync(vbar0, cot(c, 1), sizeof(double) * 3 * N, kout, c->st));
    if (mbar) CK(cudaMemcpyAsync(mbar, cot(c, 4), sizeof(double) * N, kout, c->st));
    // leave the context at the end of the trajectory, as after nb_traj_forward
    launch_copy_state(c->S, state_view(c, c->d_fin), c->st);
    CK(cudaMemcpyAsync(c->d_t, c->d_tfin, sizeof(long long) * N, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    if ((rc = sync_ctrl(c))) return rc;  // errors raised during the recomputation
    c->h_ctrl->t_now = saved.t_now;
    c->h_ctrl->steps = saved.steps;
    c->h_ctrl->interactions = saved.interactions;
    CK(cudaMemcpyAsync(c->d_ctrl, c->h_ctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, c->st));
    c->force_valid = false;
    return sync_ctrl(c);
}

int nb_traj_backward(nb_ctx *c, const double *xbar_T, const double *vbar_T, double *xbar0,
                     double *vbar0, double *mbar)
{
    const Range range_("nb_traj_backward");
    return traj_backward_impl(c, xbar_T, vbar_T, xbar0, vbar0, mbar, false);
}

int nb_traj_backward_dev(nb_ctx *c, const double *d_xbar_T, const double *d_vbar_T, double *d_xbar0,
                         double *d_vbar0, double *d_mbar)
{
    const Range range_("nb_traj_backward_dev");
    return traj_backward_impl(c, d_xbar_T, d_vbar_T, d_xbar0, d_vbar0, d_mbar, true);
}

int nb_set_profiling(nb_ctx *c, int enable)
{
    if (!c) return NB_EINVAL;
    c->profiling = enable != 0;
    return NB_OK;
}

int nb_get_stats(nb_ctx *c, nb_stats *out, int reset)
{
    if (!c) return NB_EINVAL;
    int rc = sync_ctrl(c);
    if (rc) return rc;
    for (size_t q = 0; q + 1 < c->ev_pending.size(); q += 2) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, c->ev_pending[q], c->ev_pending[q + 1]));
        c->force_ms += ms;
        c->force_launches += 1;
    }
    for (cudaEvent_t e : c->ev_pending) c->ev_free.push_back(e);
    c->ev_pending.clear();
    if (out) {
        out->steps = c->h_ctrl->steps;
        out->interactions = c->h_ctrl->interactions;
        out->kernel_launches = c->launches;
        out->force_launches = c->force_launches;
        out->force_ms = c->force_ms;
    }
    if (reset) {
        c->launches = 0;
        c->force_launches = 0;
        c->force_ms = 0.0;
    }
    return NB_OK;
}

}  // extern "C"
