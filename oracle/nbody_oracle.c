/*
 * nbody_oracle.c -- plain FP64 CPU oracle of the direct N-body Hermite
 * block-time-step method (Portegies Zwart, Belleman & Geldof, "High
 * Performance Direct Gravitational N-body Simulations on Graphics Processing
 * Units", Section 2 and Appendix A).
 *
 * TEST INFRASTRUCTURE, NOT THE PRODUCT.  This file is the slow, obviously
 * correct reference that the CUDA path is checked against.  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product library never does, and the two share no code.
 *
 * Every routine is the plain definition or the paper's steps in the paper's
 * order: double loops, no blocking, no reordering.  Compile with
 *   -O2 -ffp-contract=off -fno-fast-math
 * so that every double operation is one IEEE round-to-nearest operation in
 * source order (no fused multiply-add), which is what lets integer block
 * levels be compared bit for bit with the GPU path.
 *
 * Readings of points the paper leaves open (all pinned by tests):
 *  - Eq. 1 prints (r_i - r_j) with a plus sign, which is repulsive; the
 *    Appendix A kernel uses dx = x_j - x_i, which is attractive.  The kernel's
 *    sign is taken.
 *  - Softening: r^2 = |dx|^2 + eps^2 (Plummer softening, Appendix A kernel).
 *  - The self term j = i is excluded, as Eq. 1's sum states.
 *  - The time-step criterion is not printed (the abstract only says "the same
 *    time step criterion"); the standard Aarseth criterion with eta = 0.01 is
 *    used, with the snap and crackle that the corrector's a2 and a3 define.
 *  - Times are integer ticks of 2^-40; time steps are 2^-k with
 *    k_min <= k <= 40 (k_min = 3 gives the paper's dt_max = 0.125).
 *  - Initial step: eta_init * |a| / |k| quantised like every other step.
 *  - A step may halve as often as needed, but double only once per step and
 *    only when the new time is a multiple of the doubled step.
 *
 * The end of the file adds the summation variants of Section 6 (GRAPE-6's
 * 64-bit fixed-point sums; FP32 sums in index order and smallest force
 * first).  They are defined on single-precision pair terms, whose every
 * operation is spelled out there, so that a GPU evaluating the same IEEE
 * operations gives the same bits; the integrator takes the summation as an
 * argument (0 = the FP64 definition above).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TICK_BITS 40
#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ESTEP (-4)

static void orc_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Ticks -> time units: exact, because tick counts stay below 2^53. */
static double orc_ticks_to_time(int64_t ticks)
{
    return ldexp((double)ticks, -ORC_TICK_BITS);
}

/*
 * Direct summation (Eq. 1; pair terms as in the Appendix A kernel):
 *   acc_i  =  sum_{j != i} m_j dx / r^3
 *   jerk_i =  sum_{j != i} m_j ( dv / r^3 - 3 (dx . dv) dx / r^5 )
 *   pot_i  = -sum_{j != i} m_j / r
 * with dx = x_j - x_i, dv = v_j - v_i, r = sqrt(|dx|^2 + eps^2), G = 1.
 * x, v are [n][3]; idx lists the active i; outputs are [n_act][3] and [n_act].
 */
void orc_force(int64_t n, const double *m, const double *x, const double *v,
               double eps, int64_t n_act, const int32_t *idx,
               double *acc, double *jerk, double *pot, int nthreads)
{
    orc_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t a = 0; a < n_act; a++) {
        int64_t i = idx[a];
        double ai[3] = {0.0, 0.0, 0.0};
        double ki[3] = {0.0, 0.0, 0.0};
        double pi = 0.0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double dx[3], dv[3];
            for (int c = 0; c < 3; c++) {
                dx[c] = x[3 * j + c] - x[3 * i + c];
                dv[c] = v[3 * j + c] - v[3 * i + c];
            }
            double r2 = dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2] + eps * eps;
            double r = sqrt(r2);
            double r3 = r2 * r;
            double r5 = r3 * r2;
            double xv = dx[0] * dv[0] + dx[1] * dv[1] + dx[2] * dv[2];
            for (int c = 0; c < 3; c++) {
                ai[c] += m[j] * dx[c] / r3;
                ki[c] += m[j] * (dv[c] / r3 - 3.0 * xv * dx[c] / r5);
            }
            pi -= m[j] / r;
        }
        for (int c = 0; c < 3; c++) {
            acc[3 * a + c] = ai[c];
            jerk[3 * a + c] = ki[c];
        }
        pot[a] = pi;
    }
}

/*
 * Total energy E = T + W with T = 1/2 sum m v^2 and the softened potential
 * energy W = -sum_{i<j} m_i m_j / sqrt(|x_i - x_j|^2 + eps^2), the energy whose
 * conservation the paper reports (Section 6).
 */
void orc_energy(int64_t n, const double *m, const double *x, const double *v,
                double eps, double *ekin, double *epot, int nthreads)
{
    double *wrow = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double t = 0.0, w = 0.0;
    for (int64_t i = 0; i < n; i++)
        t += 0.5 * m[i] * (v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] + v[3 * i + 2] * v[3 * i + 2]);
    orc_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int64_t j = i + 1; j < n; j++) {
            double d0 = x[3 * i] - x[3 * j];
            double d1 = x[3 * i + 1] - x[3 * j + 1];
            double d2 = x[3 * i + 2] - x[3 * j + 2];
            s -= m[i] * m[j] / sqrt(d0 * d0 + d1 * d1 + d2 * d2 + eps * eps);
        }
        wrow[i] = s;
    }
    for (int64_t i = 0; i < n; i++) w += wrow[i];
    free(wrow);
    *ekin = t;
    *epot = w;
}

/*
 * Hermite predictor (Section 2):
 *   x_p = x + (v + (dt/2) (a + (dt/3) k)) dt
 *   v_p = v + (a + (dt/2) k) dt
 */
void orc_predict_one(const double *x, const double *v, const double *a, const double *k,
                     double dt, double *xp, double *vp)
{
    for (int c = 0; c < 3; c++) {
        xp[c] = x[c] + (v[c] + (dt / 2.0) * (a[c] + (dt / 3.0) * k[c])) * dt;
        vp[c] = v[c] + (a[c] + (dt / 2.0) * k[c]) * dt;
    }
}

/*
 * Hermite corrector (Section 2).  In the paper's notation a, k are the values
 * at the start of the step and a_p, k_p those recomputed at the predicted point:
 *   a3 = 2 (a - a_p) + (k + k_p) dt
 *   a2 = -3 (a - a_p) - (2 k + k_p) dt
 *   x  = x_p + (a2/12 + a3/20) dt^2
 *   v  = v_p + (a2/3 + a3/4) dt
 */
void orc_correct_one(const double *xp, const double *vp, const double *a, const double *k,
                     const double *ap, const double *kp, double dt,
                     double *x, double *v, double *a2, double *a3)
{
    for (int c = 0; c < 3; c++) {
        a3[c] = 2.0 * (a[c] - ap[c]) + (k[c] + kp[c]) * dt;
        a2[c] = -3.0 * (a[c] - ap[c]) - (2.0 * k[c] + kp[c]) * dt;
        x[c] = xp[c] + (a2[c] / 12.0 + a3[c] / 20.0) * (dt * dt);
        v[c] = vp[c] + (a2[c] / 3.0 + a3[c] / 4.0) * dt;
    }
}

static double orc_norm3(const double *u)
{
    return sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
}

/*
 * Aarseth time-step criterion at the end of a step of length dt.  The
 * corrector's a2 = (dk/dt) dt^2 / 2 and a3 = (d2k/dt2) dt^3 / 6 (Section 2)
 * give the snap at the start, s0 = 2 a2 / dt^2, the crackle c = 6 a3 / dt^3,
 * and the snap at the end, s1 = s0 + c dt.  With a1, k1 the new acceleration
 * and jerk:
 *   dt_new = sqrt( eta (|a1| |s1| + |k1|^2) / (|k1| |c| + |s1|^2) ).
 * A zero denominator gives +infinity (no constraint).
 */
double orc_aarseth_dt(const double *a1, const double *k1, const double *a2, const double *a3,
                      double dt, double eta)
{
    double dt2 = dt * dt;
    double dt3 = dt2 * dt;
    double s0[3], cr[3], s1[3];
    for (int c = 0; c < 3; c++) {
        s0[c] = 2.0 * a2[c] / dt2;
        cr[c] = 6.0 * a3[c] / dt3;
        s1[c] = s0[c] + cr[c] * dt;
    }
    double na = orc_norm3(a1), nk = orc_norm3(k1), ns = orc_norm3(s1), nc = orc_norm3(cr);
    double num = na * ns + nk * nk;
    double den = nk * nc + ns * ns;
    if (den == 0.0) return INFINITY;
    return sqrt(eta * num / den);
}

/* Initial step eta_init |a| / |k|; +infinity when the jerk vanishes. */
double orc_initial_dt(const double *a, const double *k, double eta_init)
{
    double nk = orc_norm3(k);
    if (nk == 0.0) return INFINITY;
    return eta_init * orc_norm3(a) / nk;
}

/*
 * Block level of a raw step: the k of the largest 2^-k <= dt_raw, clamped to
 * k >= kmin.  frexp gives dt_raw = f 2^e with 1/2 <= f < 1, so that power of
 * two is 2^(e-1) and k = 1 - e, exactly.  Returns ORC_ESTEP when dt_raw is
 * not a number or below 2^-40.
 */
int orc_level_of(double dt_raw, int kmin, int *level)
{
    if (isnan(dt_raw) || dt_raw < ldexp(1.0, -ORC_TICK_BITS)) return ORC_ESTEP;
    int k;
    if (isinf(dt_raw)) {
        k = kmin;
    } else {
        int e;
        (void)frexp(dt_raw, &e);
        k = 1 - e;
        if (k < kmin) k = kmin;
    }
    *level = k;
    return ORC_OK;
}

/*
 * New block level after a step that ends at t_new (ticks), from the old level
 * and the quantised criterion (see the readings in the header).
 */
int orc_next_level(int k_old, int k_q, int64_t t_new, int kmin)
{
    if (k_q > k_old) return k_q;
    if (k_q < k_old && k_old > kmin) {
        int64_t twice_old = (int64_t)1 << (ORC_TICK_BITS - k_old + 1);
        if (t_new % twice_old == 0) return k_old - 1;
    }
    return k_old;
}

/* Force with the summation the integrator was asked for (see the summation
 * variants at the end of this file); mode 0 is orc_force itself. */
static void orc_force_mode(int mode, int64_t n, const double *m, const double *x, const double *v,
                           double eps, int64_t n_act, const int32_t *idx, double *acc,
                           double *jerk, double *pot, int nthreads);

/*
 * Start-up: full force at t = 0 on every particle, then the initial step.
 * With kfix > 0 every particle gets the shared level kfix instead.  sum_mode
 * selects the force's summation (0: FP64, otherwise a summation variant).
 * Arrays are [n][3] (x, v, a, k), [n] ticks t and levels lev.
 */
int orc_init(int64_t n, const double *m, const double *x, const double *v, double eps,
             double eta_init, int kmin, int kfix, double *a, double *k, double *pot,
             int64_t *t, int32_t *lev, int nthreads, int sum_mode)
{
    if (n < 1 || eps < 0.0 || kmin < 0 || kmin > ORC_TICK_BITS) return ORC_EINVAL;
    if (sum_mode < 0 || sum_mode > 3) return ORC_EINVAL;
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!all) return ORC_ENOMEM;
    for (int64_t i = 0; i < n; i++) all[i] = (int32_t)i;
    orc_force_mode(sum_mode, n, m, x, v, eps, n, all, a, k, pot, nthreads);
    free(all);
    int rc = ORC_OK;
    for (int64_t i = 0; i < n; i++) {
        t[i] = 0;
        if (kfix > 0) {
            lev[i] = kfix;
            continue;
        }
        int level;
        if (orc_level_of(orc_initial_dt(a + 3 * i, k + 3 * i, eta_init), kmin, &level) != ORC_OK) {
            rc = ORC_ESTEP;
            level = ORC_TICK_BITS;
        }
        lev[i] = level;
    }
    return rc;
}

/* Earliest end time t_i + 2^-k_i over all particles, in ticks. */
int64_t orc_next_time(int64_t n, const int64_t *t, const int32_t *lev)
{
    int64_t best = INT64_MAX;
    for (int64_t i = 0; i < n; i++) {
        int64_t e = t[i] + ((int64_t)1 << (ORC_TICK_BITS - lev[i]));
        if (e < best) best = e;
    }
    return best;
}

/*
 * One block step (Section 2's step loop): select the block (the particles
 * with the smallest t_i + dt_i), predict all particles to that time, recompute
 * acceleration and jerk on the block from the predicted state, correct the
 * block and give it new steps.  No step is taken when the block time would
 * exceed t_end (ticks); the return value is then 0.  Otherwise it is the block
 * size (active indices in act[], ascending, and the block time in *t_next),
 * or ORC_ESTEP if some new step fell below 2^-40.  pot_out[] (length n) gets
 * the block's potentials at the predicted state, indexed by particle.
 */
int64_t orc_step(int64_t n, const double *m, double eps, double eta, int kmin, int kfix,
                 int64_t t_end, double *x, double *v, double *a, double *k,
                 int64_t *t, int32_t *lev, int32_t *act, int64_t *t_next_out,
                 double *pot_out, int nthreads, int sum_mode)
{
    int64_t tn = orc_next_time(n, t, lev);
    *t_next_out = tn;
    if (tn > t_end) return 0;

    int64_t na = 0;
    for (int64_t i = 0; i < n; i++)
        if (t[i] + ((int64_t)1 << (ORC_TICK_BITS - lev[i])) == tn) act[na++] = (int32_t)i;

    double *xp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *vp = (double *)malloc(sizeof(double) * 3 * (size_t)n);
    double *anew = (double *)malloc(sizeof(double) * 3 * (size_t)na);
    double *knew = (double *)malloc(sizeof(double) * 3 * (size_t)na);
    double *pnew = (double *)malloc(sizeof(double) * (size_t)na);
    if (!xp || !vp || !anew || !knew || !pnew) {
        free(xp); free(vp); free(anew); free(knew); free(pnew);
        return ORC_ENOMEM;
    }
    for (int64_t j = 0; j < n; j++)
        orc_predict_one(x + 3 * j, v + 3 * j, a + 3 * j, k + 3 * j,
                        orc_ticks_to_time(tn - t[j]), xp + 3 * j, vp + 3 * j);

    orc_force_mode(sum_mode, n, m, xp, vp, eps, na, act, anew, knew, pnew, nthreads);

    int64_t rc = na;
    for (int64_t s = 0; s < na; s++) {
        int64_t i = act[s];
        double dt = orc_ticks_to_time(tn - t[i]);
        double a2[3], a3[3];
        orc_correct_one(xp + 3 * i, vp + 3 * i, a + 3 * i, k + 3 * i, anew + 3 * s, knew + 3 * s,
                        dt, x + 3 * i, v + 3 * i, a2, a3);
        for (int c = 0; c < 3; c++) {
            a[3 * i + c] = anew[3 * s + c];
            k[3 * i + c] = knew[3 * s + c];
        }
        if (pot_out) pot_out[i] = pnew[s];
        t[i] = tn;
        if (kfix > 0) continue;
        int kq;
        if (orc_level_of(orc_aarseth_dt(a + 3 * i, k + 3 * i, a2, a3, dt, eta), kmin, &kq) != ORC_OK) {
            rc = ORC_ESTEP;
            kq = ORC_TICK_BITS;
        }
        lev[i] = orc_next_level(lev[i], kq, tn, kmin);
    }
    free(xp); free(vp); free(anew); free(knew); free(pnew);
    return rc;
}

/*
 * Runs block steps until every particle has reached t_end (ticks) or
 * max_steps steps were taken.  Optional outputs: hist_nact[s] = block size of
 * step s (up to max_steps entries), *interactions = sum of n_active (n - 1).
 * Returns the number of steps, or a negative error.
 */
int64_t orc_run(int64_t n, const double *m, double eps, double eta, int kmin, int kfix,
                int64_t t_end, int64_t max_steps, double *x, double *v, double *a, double *k,
                int64_t *t, int32_t *lev, int32_t *hist_nact, int64_t *interactions, int nthreads,
                int sum_mode)
{
    int32_t *act = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!act) return ORC_ENOMEM;
    int64_t steps = 0, inter = 0;
    while (steps < max_steps) {
        int64_t tn;
        int64_t na = orc_step(n, m, eps, eta, kmin, kfix, t_end, x, v, a, k, t, lev, act, &tn,
                              NULL, nthreads, sum_mode);
        if (na < 0) { free(act); return na; }
        if (na == 0) break;
        if (hist_nact) hist_nact[steps] = (int32_t)na;
        inter += na * (n - 1);
        steps++;
    }
    free(act);
    if (interactions) *interactions = inter;
    return steps;
}

/* ------------------------------------------------------------------------
 * Differentiation (no counterpart in the paper, which has no gradients).
 *
 * Vector-Jacobian product of the direct-summation acceleration and jerk of
 * every particle with respect to all positions, velocities and masses: given
 * cotangents abar_i, kbar_i on acc_i, jerk_i, accumulate xbar, vbar, mbar.
 * Written as the pair loop of the definition: for every ordered pair (i, j),
 * j != i, with d = x_j - x_i, w = v_j - v_i, r^2 = |d|^2 + eps^2, s = d.w,
 *   acc_i  += m_j d / r^3
 *   jerk_i += m_j (w / r^3 - 3 s d / r^5)
 * differentiate abar_i . acc_i + kbar_i . jerk_i with respect to d, w, m_j:
 *   g_d = m_j [ abar/r^3 - 3 (abar.d) d/r^5 - 3 (kbar.w) d/r^5
 *               - 3 (kbar.d) w/r^5 - 3 s kbar/r^5 + 15 s (kbar.d) d/r^7 ]
 *   g_w = m_j [ kbar/r^3 - 3 (kbar.d) d/r^5 ]
 *   g_m = abar.d/r^3 + kbar.(w/r^3 - 3 s d/r^5)
 * and since d, w are x_j - x_i, v_j - v_i: xbar_j += g_d, xbar_i -= g_d,
 * vbar_j += g_w, vbar_i -= g_w, mbar_j += g_m.  Outputs are overwritten.
 */
void orc_force_vjp(int64_t n, const double *m, const double *x, const double *v, double eps,
                   const double *abar, const double *kbar, double *xbar, double *vbar,
                   double *mbar)
{
    for (int64_t q = 0; q < 3 * n; q++) xbar[q] = vbar[q] = 0.0;
    for (int64_t q = 0; q < n; q++) mbar[q] = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double *ab = abar + 3 * i, *kb = kbar + 3 * i;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            double d[3], w[3];
            for (int c = 0; c < 3; c++) {
                d[c] = x[3 * j + c] - x[3 * i + c];
                w[c] = v[3 * j + c] - v[3 * i + c];
            }
            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] + eps * eps;
            double r = sqrt(r2);
            double r3 = r2 * r, r5 = r3 * r2, r7 = r5 * r2;
            double s = d[0] * w[0] + d[1] * w[1] + d[2] * w[2];
            double ad = ab[0] * d[0] + ab[1] * d[1] + ab[2] * d[2];
            double kd = kb[0] * d[0] + kb[1] * d[1] + kb[2] * d[2];
            double kw = kb[0] * w[0] + kb[1] * w[1] + kb[2] * w[2];
            for (int c = 0; c < 3; c++) {
                double gd = m[j] * (ab[c] / r3 - 3.0 * ad * d[c] / r5 - 3.0 * kw * d[c] / r5
                                    - 3.0 * kd * w[c] / r5 - 3.0 * s * kb[c] / r5
                                    + 15.0 * s * kd * d[c] / r7);
                double gw = m[j] * (kb[c] / r3 - 3.0 * kd * d[c] / r5);
                xbar[3 * j + c] += gd;
                xbar[3 * i + c] -= gd;
                vbar[3 * j + c] += gw;
                vbar[3 * i + c] -= gw;
            }
            mbar[j] += ad / r3 + kw / r3 - 3.0 * s * kd / r5;
        }
    }
}

/*
 * Fixed shared-step Hermite trajectory and its gradient.  With every
 * particle on the same step dt, one step is (Section 2): predict every
 * particle, recompute acc and jerk of every particle at the predicted state,
 * correct every particle.  The initial acc and jerk are the force of the
 * initial state.  Given the cotangents xbar_T, vbar_T of the final positions
 * and velocities, the gradient with respect to the initial x, v and the
 * masses is accumulated by running the steps backwards, each through the
 * transposes of the (linear) corrector and predictor and the force VJP above.
 * All intermediate states are stored (plain reverse mode, no checkpointing).
 * On return x, v hold the final state; xbar, vbar are overwritten with the
 * gradient with respect to the initial state, mbar with that w.r.t. masses.
 */
int orc_traj_vjp(int64_t n, const double *m, double *x, double *v, double eps, double dt,
                 int64_t steps, const double *xbar_T, const double *vbar_T, double *xbar,
                 double *vbar, double *mbar)
{
    size_t n3 = 3 * (size_t)n;
    size_t per = 4 * n3; /* x, v, a, k */
    double *st = (double *)malloc(sizeof(double) * per * (size_t)(steps + 1));
    double *xp = (double *)malloc(sizeof(double) * n3), *vp = (double *)malloc(sizeof(double) * n3);
    double *a1 = (double *)malloc(sizeof(double) * n3), *k1 = (double *)malloc(sizeof(double) * n3);
    double *pot = (double *)malloc(sizeof(double) * (size_t)n);
    double *ab = (double *)malloc(sizeof(double) * n3), *kb = (double *)malloc(sizeof(double) * n3);
    double *a1b = (double *)malloc(sizeof(double) * n3), *k1b = (double *)malloc(sizeof(double) * n3);
    double *xg = (double *)malloc(sizeof(double) * n3), *vg = (double *)malloc(sizeof(double) * n3);
    double *mg = (double *)malloc(sizeof(double) * (size_t)n);
    int32_t *all = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    if (!st || !xp || !vp || !a1 || !k1 || !pot || !ab || !kb || !a1b || !k1b || !xg || !vg ||
        !mg || !all) {
        free(st); free(xp); free(vp); free(a1); free(k1); free(pot); free(ab); free(kb);
        free(a1b); free(k1b); free(xg); free(vg); free(mg); free(all);
        return ORC_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++) all[i] = (int32_t)i;
    const double h = dt / 2.0, q = dt / 3.0;

    /* forward */
    double *s0 = st;
    memcpy(s0, x, sizeof(double) * n3);
    memcpy(s0 + n3, v, sizeof(double) * n3);
    orc_force(n, m, x, v, eps, n, all, s0 + 2 * n3, s0 + 3 * n3, pot, 1);
    for (int64_t s = 0; s < steps; s++) {
        double *cur = st + per * (size_t)s, *nxt = st + per * (size_t)(s + 1);
        for (int64_t i = 0; i < n; i++)
            orc_predict_one(cur + 3 * i, cur + n3 + 3 * i, cur + 2 * n3 + 3 * i,
                            cur + 3 * n3 + 3 * i, dt, xp + 3 * i, vp + 3 * i);
        orc_force(n, m, xp, vp, eps, n, all, a1, k1, pot, 1);
        for (int64_t i = 0; i < n; i++) {
            double a2[3], a3[3];
            orc_correct_one(xp + 3 * i, vp + 3 * i, cur + 2 * n3 + 3 * i, cur + 3 * n3 + 3 * i,
                            a1 + 3 * i, k1 + 3 * i, dt, nxt + 3 * i, nxt + n3 + 3 * i, a2, a3);
        }
        memcpy(nxt + 2 * n3, a1, sizeof(double) * n3);
        memcpy(nxt + 3 * n3, k1, sizeof(double) * n3);
    }
    memcpy(x, st + per * (size_t)steps, sizeof(double) * n3);
    memcpy(v, st + per * (size_t)steps + n3, sizeof(double) * n3);

    /* backward: cotangents of the state (x, v, a, k) after step s */
    for (size_t c = 0; c < n3; c++) {
        xbar[c] = xbar_T[c];
        vbar[c] = vbar_T[c];
        ab[c] = 0.0;
        kb[c] = 0.0;
    }
    for (int64_t i = 0; i < n; i++) mbar[i] = 0.0;
    for (int64_t s = steps - 1; s >= 0; s--) {
        double *cur = st + per * (size_t)s;
        /* corrector: x' = xp + (a2/12 + a3/20) dt^2, v' = vp + (a2/3 + a3/4) dt with
           a3 = 2 D + (k + k1) dt, a2 = -3 D - (2 k + k1) dt, D = a - a1;
           the new state's acc and jerk are a1, k1 (cotangents ab, kb on entry) */
        for (size_t c = 0; c < n3; c++) {
            double a2b = xbar[c] * dt * dt / 12.0 + vbar[c] * dt / 3.0;
            double a3b = xbar[c] * dt * dt / 20.0 + vbar[c] * dt / 4.0;
            double Db = 2.0 * a3b - 3.0 * a2b;
            a1b[c] = ab[c] - Db;                        /* through D and the new acc */
            k1b[c] = kb[c] + a3b * dt - a2b * dt;       /* through a3, a2 and the new jerk */
            ab[c] = Db;                                 /* old acc, through D */
            kb[c] = a3b * dt - 2.0 * a2b * dt;          /* old jerk */
        }
        /* xbar, vbar now hold the cotangents of xp, vp (the corrector adds them) */
        for (int64_t i = 0; i < n; i++)
            orc_predict_one(cur + 3 * i, cur + n3 + 3 * i, cur + 2 * n3 + 3 * i,
                            cur + 3 * n3 + 3 * i, dt, xp + 3 * i, vp + 3 * i);
        orc_force_vjp(n, m, xp, vp, eps, a1b, k1b, xg, vg, mg);
        for (int64_t i = 0; i < n; i++) mbar[i] += mg[i];
        for (size_t c = 0; c < n3; c++) {
            double xpb = xbar[c] + xg[c], vpb = vbar[c] + vg[c];
            /* predictor: xp = x + v dt + a h dt + k q h dt, vp = v + a dt + k h dt */
            xbar[c] = xpb;
            vbar[c] = xpb * dt + vpb;
            ab[c] += xpb * h * dt + vpb * dt;
            kb[c] += xpb * q * h * dt + vpb * h * dt;
        }
    }
    /* initial acc and jerk are the force of the initial state */
    orc_force_vjp(n, m, st, st + n3, eps, ab, kb, xg, vg, mg);
    for (int64_t i = 0; i < n; i++) mbar[i] += mg[i];
    for (size_t c = 0; c < n3; c++) {
        xbar[c] += xg[c];
        vbar[c] += vg[c];
    }
    free(st); free(xp); free(vp); free(a1); free(k1); free(pot); free(ab); free(kb);
    free(a1b); free(k1b); free(xg); free(vg); free(mg); free(all);
    return ORC_OK;
}

/* ------------------------------------------------------------------------
 * Summation variants (Section 6 on accuracy).  The paper notes that the
 * GRAPE-6 accumulates the pair forces in 64-bit fixed point while the GPU
 * sums in single precision, and that summing the smallest forces first would
 * make the GPU's sums more accurate.  Three summations of the same
 * single-precision pair terms are defined here:
 *   ORC_SUM_FIXED       every term rounded to 64-bit fixed point and summed
 *                       exactly (GRAPE-style; independent of the order of j);
 *   ORC_SUM_FP32        FP32 running sum in increasing j;
 *   ORC_SUM_FP32_SORTED FP32 running sum, smallest pair force first.
 *
 * The terms are those of the Appendix A kernel evaluated on the single-
 * precision record of every particle: position as hi = fl32(x),
 * lo = fl32(x - hi); velocity fl32(v); mass fl32(m); softening
 * eps2 = fl32(eps * eps).  Each operation below is one IEEE single-precision
 * operation rounded to nearest, in the order written (this file is compiled
 * without contraction), so any IEEE implementation of the same sequence gives
 * the same bits:
 *   dx   = (xj_hi - xi_hi) + (xj_lo - xi_lo),   u = vj - vi       (per axis)
 *   d2   = (dx0 dx0 + dx1 dx1) + dx2 dx2,        r2 = d2 + eps2
 *   rv   = (dx0 u0 + dx1 u1) + dx2 u2
 *   rinv = 1 / sqrt(r2),  rinv2 = rinv rinv,  mr = mj rinv,  mr3 = mr rinv2
 *   b    = (-3 rv) rinv2
 *   acc  = (mr3 Sa) dx,   jerk = (mr3 Sk) (u + b dx),   pot = -(mr Sp)
 *   key  = min(mr3 sqrt(d2), FLT_MAX)        (the pair force |m_j dx / r^3|)
 * with Sa = Sk = Sp = 1 for the FP32 sums and powers of two for fixed point.
 * A pair contributes nothing when j = i or r2 = 0 (eps = 0 and coincident
 * particles).
 */
#include <float.h>

#define ORC_SUM_FP64 0
#define ORC_SUM_FIXED 1
#define ORC_SUM_FP32 2
#define ORC_SUM_FP32_SORTED 3

typedef struct {
    float hi[3], lo[3], v[3], m;
} orc_rec32;

static void orc_rec32_of(const double *x, const double *v, double m, orc_rec32 *r)
{
    for (int c = 0; c < 3; c++) {
        r->hi[c] = (float)x[c];
        r->lo[c] = (float)(x[c] - (double)r->hi[c]);
        r->v[c] = (float)v[c];
    }
    r->m = (float)m;
}

/* The pair terms t[0..6] (acc xyz, jerk xyz, pot) of j on i and the pair's
 * key; returns 0 for a pair that contributes nothing (r2 = 0). */
static int orc_pair32(const orc_rec32 *pi, const orc_rec32 *pj, float eps2, const float sc[3],
                      float t[7], float *key)
{
    float dx[3], u[3];
    for (int c = 0; c < 3; c++) {
        dx[c] = (pj->hi[c] - pi->hi[c]) + (pj->lo[c] - pi->lo[c]);
        u[c] = pj->v[c] - pi->v[c];
    }
    float d2 = (dx[0] * dx[0] + dx[1] * dx[1]) + dx[2] * dx[2];
    float r2 = d2 + eps2;
    if (r2 == 0.0f) return 0;
    float rv = (dx[0] * u[0] + dx[1] * u[1]) + dx[2] * u[2];
    float rinv = 1.0f / sqrtf(r2);
    float rinv2 = rinv * rinv;
    float mr = pj->m * rinv;
    float mr3 = mr * rinv2;
    float b = (-3.0f * rv) * rinv2;
    float fa = mr3 * sc[0], fk = mr3 * sc[1], fp = mr * sc[2];
    for (int c = 0; c < 3; c++) {
        t[c] = fa * dx[c];
        t[3 + c] = fk * (u[c] + b * dx[c]);
    }
    t[6] = -fp;
    if (key) *key = fminf(mr3 * sqrtf(d2), FLT_MAX);
    return 1;
}

/* Smallest e with x < 2^e for a float x >= 0, read from its exponent field
 * (-126 for zero and subnormals). */
static int orc_exp_above(float x)
{
    uint32_t b;
    memcpy(&b, &x, sizeof b);
    int be = (int)((b >> 23) & 0xFF);
    return be == 0 ? -126 : be - 126;
}

static int orc_floor_half(int a) { return a >= 0 ? a / 2 : -((1 - a) / 2); }

/*
 * Fixed-point scales 2^s (s[0] acc, s[1] jerk, s[2] pot) for the system
 * m[n], v[n][3], eps.  Every term must stay below 2^56 in fixed-point units,
 * so that 64 of them sum without overflow in 64 bits.  With
 *   eps2 >= 2^F (F from eps2's exponent field; eps2 must be a normal float),
 *   m_j < 2^Em, |vx| + |vy| + |vz| < 2^Ev for every particle (fl32 values;
 *   Em, Ev at least -64),
 * the terms obey |acc| <= m_j / r^2 < 2^(Em - F), |pot| = m_j / r <
 * 2^(Em - floor(F/2)) and |jerk| <= 4 m_j |dv| / r^3 < 2^(3 + Em + Ev -
 * floor(3F/2)) (|dv| <= 2 max |v|, r >= eps), up to single-precision
 * rounding, which the factor 2 between 2^56 and 2^57 absorbs.  Then
 * s = 56 - e, at most 126.  Returns ORC_EINVAL when eps2 is zero, subnormal
 * or infinite, or a scale falls below -126.
 */
int orc_fixed_scales(int64_t n, const double *m, const double *v, double eps, int s[3])
{
    float eps2 = (float)(eps * eps);
    uint32_t eb;
    memcpy(&eb, &eps2, sizeof eb);
    int be = (int)((eb >> 23) & 0xFF);
    if (be == 0 || be == 255) return ORC_EINVAL;
    int F = be - 127;
    float mmax = 0.0f, vmax = 0.0f;
    for (int64_t j = 0; j < n; j++) {
        float mf = (float)m[j];
        float v1 = (fabsf((float)v[3 * j]) + fabsf((float)v[3 * j + 1])) + fabsf((float)v[3 * j + 2]);
        if (mf > mmax) mmax = mf;
        if (v1 > vmax) vmax = v1;
    }
    int Em = orc_exp_above(mmax), Ev = orc_exp_above(vmax);
    if (Em < -64) Em = -64;
    if (Ev < -64) Ev = -64;
    int e[3] = {Em - F, 3 + Em + Ev - orc_floor_half(3 * F), Em - orc_floor_half(F)};
    for (int q = 0; q < 3; q++) {
        s[q] = 56 - e[q];
        if (s[q] > 126) s[q] = 126;
        if (s[q] < -126) return ORC_EINVAL;
    }
    return ORC_OK;
}

/* An exact integer as a double: |y| = H 2^64 + L, then fl64(fl64(H) 2^64 +
 * fl64(L)) with y's sign.  (gcc's 128-bit integers hold the exact sums.) */
static double orc_i128_to_double(__int128 y)
{
    int neg = y < 0;
    unsigned __int128 u = neg ? -(unsigned __int128)y : (unsigned __int128)y;
    uint64_t H = (uint64_t)(u >> 64), L = (uint64_t)u;
    double d = (double)H * 0x1p64 + (double)L;
    return neg ? -d : d;
}

typedef struct {
    uint32_t key;  /* bits of the non-negative key: their order is the keys' order */
    int32_t j;
} orc_keyed;

static int orc_keyed_cmp(const void *pa, const void *pb)
{
    const orc_keyed *a = (const orc_keyed *)pa, *b = (const orc_keyed *)pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return a->j < b->j ? -1 : (a->j > b->j);
}

/*
 * acc, jerk, pot on the listed i with one of the summation variants above
 * (mode ORC_SUM_FIXED, ORC_SUM_FP32 or ORC_SUM_FP32_SORTED).
 *   fixed:  Y_q = sum_j round_half_even(t_q,j) exactly, with the scales of
 *           orc_fixed_scales over all n particles; result Y_q 2^-s_q.
 *   fp32:   S = 0; S = fl32(S + t_j) for j = 0, 1, ..., n - 1.
 *   sorted: the same running sum over j in increasing key, ties in
 *           increasing j.
 * Returns ORC_EINVAL for a bad mode or (fixed) unusable scales.
 */
int orc_force_summed(int mode, int64_t n, const double *m, const double *x, const double *v,
                     double eps, int64_t n_act, const int32_t *idx, double *acc, double *jerk,
                     double *pot, int nthreads)
{
    if (mode != ORC_SUM_FIXED && mode != ORC_SUM_FP32 && mode != ORC_SUM_FP32_SORTED)
        return ORC_EINVAL;
    int s[3] = {0, 0, 0};
    if (mode == ORC_SUM_FIXED && orc_fixed_scales(n, m, v, eps, s) != ORC_OK) return ORC_EINVAL;
    float sc[3] = {1.0f, 1.0f, 1.0f};
    for (int q = 0; q < 3; q++) sc[q] = ldexpf(1.0f, s[q]);
    const float eps2 = (float)(eps * eps);
    orc_rec32 *rec = (orc_rec32 *)malloc(sizeof(orc_rec32) * (size_t)(n > 0 ? n : 1));
    if (!rec) return ORC_ENOMEM;
    for (int64_t j = 0; j < n; j++) orc_rec32_of(x + 3 * j, v + 3 * j, m[j], &rec[j]);
    int failed = 0;
    orc_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t a = 0; a < n_act; a++) {
        int64_t i = idx[a];
        float t[7];
        double out[7];
        if (mode == ORC_SUM_FIXED) {
            __int128 Y[7] = {0, 0, 0, 0, 0, 0, 0};
            for (int64_t j = 0; j < n; j++) {
                if (j == i || !orc_pair32(&rec[i], &rec[j], eps2, sc, t, NULL)) continue;
                for (int q = 0; q < 7; q++) Y[q] += (__int128)llrintf(t[q]);
            }
            for (int q = 0; q < 7; q++)
                out[q] = orc_i128_to_double(Y[q]) * ldexp(1.0, -s[q < 3 ? 0 : (q < 6 ? 1 : 2)]);
        } else {
            float S[7] = {0, 0, 0, 0, 0, 0, 0};
            if (mode == ORC_SUM_FP32) {
                for (int64_t j = 0; j < n; j++) {
                    if (j == i || !orc_pair32(&rec[i], &rec[j], eps2, sc, t, NULL)) continue;
                    for (int q = 0; q < 7; q++) S[q] = S[q] + t[q];
                }
            } else {
                orc_keyed *ord = (orc_keyed *)malloc(sizeof(orc_keyed) * (size_t)(n > 0 ? n : 1));
                if (!ord) {
#pragma omp atomic write
                    failed = 1;
                    continue;
                }
                int64_t cnt = 0;
                for (int64_t j = 0; j < n; j++) {
                    float key;
                    if (j == i || !orc_pair32(&rec[i], &rec[j], eps2, sc, t, &key)) continue;
                    memcpy(&ord[cnt].key, &key, sizeof key);
                    ord[cnt].j = (int32_t)j;
                    cnt++;
                }
                qsort(ord, (size_t)cnt, sizeof(orc_keyed), orc_keyed_cmp);
                for (int64_t q2 = 0; q2 < cnt; q2++) {
                    orc_pair32(&rec[i], &rec[ord[q2].j], eps2, sc, t, NULL);
                    for (int q = 0; q < 7; q++) S[q] = S[q] + t[q];
                }
                free(ord);
            }
            for (int q = 0; q < 7; q++) out[q] = (double)S[q];
        }
        for (int c = 0; c < 3; c++) {
            acc[3 * a + c] = out[c];
            jerk[3 * a + c] = out[3 + c];
        }
        pot[a] = out[6];
    }
    free(rec);
    return failed ? ORC_ENOMEM : ORC_OK;
}

/* The pair terms (scaled as the fixed-point sum scales them when `scaled`)
 * and keys of every j on particle i: t[n][7], key[n], ok[n] (0 for j = i and
 * pairs that contribute nothing).  Exposed so that tests can redo the
 * summations independently. */
int orc_pair_terms32(int64_t n, const double *m, const double *x, const double *v, double eps,
                     int64_t i, int scaled, float *t, float *key, int32_t *ok)
{
    int s[3] = {0, 0, 0};
    if (scaled && orc_fixed_scales(n, m, v, eps, s) != ORC_OK) return ORC_EINVAL;
    float sc[3];
    for (int q = 0; q < 3; q++) sc[q] = ldexpf(1.0f, s[q]);
    const float eps2 = (float)(eps * eps);
    orc_rec32 ri, rj;
    orc_rec32_of(x + 3 * i, v + 3 * i, m[i], &ri);
    for (int64_t j = 0; j < n; j++) {
        orc_rec32_of(x + 3 * j, v + 3 * j, m[j], &rj);
        ok[j] = j != i && orc_pair32(&ri, &rj, eps2, sc, t + 7 * j, key + j);
        if (!ok[j]) {
            for (int q = 0; q < 7; q++) t[7 * j + q] = 0.0f;
            key[j] = 0.0f;
        }
    }
    return ORC_OK;
}

static void orc_force_mode(int mode, int64_t n, const double *m, const double *x, const double *v,
                           double eps, int64_t n_act, const int32_t *idx, double *acc,
                           double *jerk, double *pot, int nthreads)
{
    if (mode == ORC_SUM_FP64) {
        orc_force(n, m, x, v, eps, n_act, idx, acc, jerk, pot, nthreads);
    } else if (orc_force_summed(mode, n, m, x, v, eps, n_act, idx, acc, jerk, pot, nthreads) != ORC_OK) {
        for (int64_t a = 0; a < n_act; a++) {  /* unusable input: NaN results */
            for (int c = 0; c < 3; c++) acc[3 * a + c] = jerk[3 * a + c] = NAN;
            pot[a] = NAN;
        }
    }
}
