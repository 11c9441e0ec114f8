/*
 * rrg_oracle.c -- plain, sequential FP64 CPU oracle for the scenario-based
 * robust reference governor (RG) of Ossareh, Shayne & Chevalier,
 * "CPU- and GPU-Based Parallelization of the Robust Reference Governor"
 * (arXiv 2510.08288).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library.  Only the test suite, the smoke check of the build entry point and
 * the CPU-baseline / reference legs of the benchmark may load or call it.  It
 * shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function states the passage of the paper it follows.  Floating point
 * is IEEE binary64, round-to-nearest, compiled with -ffp-contract=off so that
 * no multiply-add is fused behind the reader's back.
 *
 * Parity status (see the tests under tests/ for the pins):
 *   philox4x64_10      pinned: bit-equal to numpy.random.Philox raw output.
 *   rk4 step           pinned: equals the degree-4 Taylor closed form on a
 *                      linear system; global error slope 4 vs expm.
 *   fc3 rhs / output   pinned only through invariants (equilibrium residual,
 *                      conservation identities, derivative signs).  The
 *                      paper prints no model equations and no trajectory, so
 *                      the FC3 values themselves are "parity unpinned".
 *   equilibrium        pinned: residual of the full right-hand side at the
 *                      returned point, and RK4 rollouts stay on it.
 *   searches           pinned: brute-force dyadic grid vs bisection,
 *                      Alg. 1 == Alg. 2 with d = 0 and N = 1, scenario
 *                      monotonicity, early-exit invariance.
 *   param multipliers  pinned: range, moments and mask of the draws, words
 *                      from the numpy-pinned Philox stream 2, and scenario
 *                      k's rollout equal to the nominal rollout of theta m^k.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* FC3: third-order fuel-cell air-path closed loop (the build's stand-in for
 * the model of Sec. IV-A; the paper names the states [p_ca, w_cp, p_sm], the
 * 381 cells, the 300 A limit and the OER >= 1.9 output constraint but gives
 * no equations).  Parameter vector layout: */
enum {
    O_P_ATM, O_T_ATM, O_T_ST, O_R_A, O_V_SM, O_V_CA, O_K_SM, O_K_CA,
    O_N_CELL, O_FARADAY, O_M_O2, O_X_O2, O_GAMMA, O_C_P, O_ETA_CP, O_J_CP,
    O_ETA_CM, O_K_T, O_K_V, O_R_CM, O_A_W, O_A_P, O_LAM_REF, O_K_P,
    O_C0, O_C1, O_C2, O_NPARAM
};

int orc_nparam(void) { return O_NPARAM; }

/* O2 mass flow consumed by the stack at current I (Faraday's law). */
static double o2_consumed(const double *p, double I)
{
    return p[O_M_O2] * p[O_N_CELL] * I / (4.0 * p[O_FARADAY]);
}

/* Right-hand side dx/dt = f_c(x, I) of the continuous-time closed loop.
 * x = [p_ca, w_cp, p_sm]; the setpoint v is the stack current I (Sec. IV-A). */
void orc_fc3_rhs(const double *p, const double *x, double I, double *dx)
{
    double p_ca = x[0], w = x[1], p_sm = x[2];
    double W_cp = p[O_A_W] * w - p[O_A_P] * (p_sm - p[O_P_ATM]);
    double W_sm = p[O_K_SM] * (p_sm - p_ca);
    double W_ca = p[O_K_CA] * (p_ca - p[O_P_ATM]);
    double W_o2 = o2_consumed(p, I);
    double e = (p[O_GAMMA] - 1.0) / p[O_GAMMA];
    double Pi = p_sm / p[O_P_ATM];
    double tau_cp = p[O_C_P] * p[O_T_ATM] / p[O_ETA_CP] * (pow(Pi, e) - 1.0) * W_cp / w;
    double W_ref = p[O_LAM_REF] * W_o2 / p[O_X_O2];
    double v_cm = p[O_C0] + p[O_C1] * I + p[O_C2] * I * I + p[O_K_P] * (W_ref - W_cp);
    double tau_cm = p[O_ETA_CM] * p[O_K_T] * (v_cm - p[O_K_V] * w) / p[O_R_CM];
    double RT = p[O_R_A] * p[O_T_ST];
    dx[0] = RT / p[O_V_CA] * (W_sm - W_ca - W_o2);
    dx[1] = (tau_cm - tau_cp) / p[O_J_CP];
    dx[2] = RT / p[O_V_SM] * (W_cp - W_sm);
}

/* Constrained output y = h(x, v): the oxygen excess ratio (Sec. IV-A). */
double orc_fc3_output(const double *p, const double *x, double I)
{
    double W_sm = p[O_K_SM] * (x[2] - x[0]);
    return p[O_X_O2] * W_sm / o2_consumed(p, I);
}

/* One classical fourth-order Runge-Kutta step of size dt (Sec. IV-A, fixed
 * step 0.01 s): the discrete map f(x, v) of Eq. 1. */
void orc_rk4_step(const double *p, const double *x, double I, double dt, double *xn)
{
    double k1[3], k2[3], k3[3], k4[3], t[3];
    int i;
    orc_fc3_rhs(p, x, I, k1);
    for (i = 0; i < 3; i++) t[i] = x[i] + 0.5 * dt * k1[i];
    orc_fc3_rhs(p, t, I, k2);
    for (i = 0; i < 3; i++) t[i] = x[i] + 0.5 * dt * k2[i];
    orc_fc3_rhs(p, t, I, k3);
    for (i = 0; i < 3; i++) t[i] = x[i] + dt * k3[i];
    orc_fc3_rhs(p, t, I, k4);
    for (i = 0; i < 3; i++)
        xn[i] = x[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* Generic RK4 step for a linear system dx/dt = A x + B u (n <= 8), used only
 * by the RK4 pin against the Taylor closed form and the matrix exponential. */
void orc_rk4_linear(int n, const double *A, const double *B, double u,
                    const double *x, double dt, double *xn)
{
    double k[4][8], t[8];
    int s, i, j;
    for (s = 0; s < 4; s++) {
        double c = (s == 0) ? 0.0 : (s == 3 ? dt : 0.5 * dt);
        for (i = 0; i < n; i++) t[i] = (s == 0) ? x[i] : x[i] + c * k[s - 1][i];
        for (i = 0; i < n; i++) {
            double acc = B[i] * u;
            for (j = 0; j < n; j++) acc += A[i * n + j] * t[j];
            k[s][i] = acc;
        }
    }
    for (i = 0; i < n; i++)
        xn[i] = x[i] + (dt / 6.0) * (k[0][i] + 2.0 * k[1][i] + 2.0 * k[2][i] + k[3][i]);
}

/* ------------------------------------------------------------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
 * easy as 1, 2, 3", SC'11): ten rounds of two 64x64->128 multiplies with a
 * Weyl-sequence key schedule.  Scenario sampling (Sec. II-C, Alg. 3 draws
 * N_sim sequences d_j^k every RG step) is defined on top of it below. */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo)
{
    unsigned __int128 prod = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(prod >> 64);
    *lo = (uint64_t)prod;
}

void orc_philox4x64_10(const uint64_t *ctr, const uint64_t *key, uint64_t *out)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    int r;
    for (r = 0; r < 10; r++) {
        uint64_t hi0, lo0, hi1, lo1;
        if (r > 0) { k0 += W0; k1 += W1; }
        mulhilo64(M0, c0, &hi0, &lo0);
        mulhilo64(M1, c2, &hi1, &lo1);
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Counter streams: word 3 of the counter selects what is drawn. */
enum { STREAM_SCENARIO = 0, STREAM_PLANT = 1, STREAM_PARAM = 2 };

/* Uniform on [-a, a): top 53 bits of a Philox word as u in [0, 1). */
static double uniform_sym(uint64_t w, double a)
{
    double u = (double)(w >> 11) * 0x1.0p-53;
    return a * (2.0 * u - 1.0);
}

/* d_j^k for scenario k, step j of RG update t, components in state order
 * [p_ca, w_cp, p_sm], each i.i.d. uniform on [-a_i, a_i] (Sec. IV-A gives
 * +-50, +-10, +-50).  Output layout d[(i*H + j)*N + k]. */
void orc_sample_disturbances(uint64_t seed, uint64_t update, int64_t N, int64_t H,
                             const double *amp, double *d)
{
    int64_t j, k;
    uint64_t key[2] = { seed, 0 };
    for (j = 0; j < H; j++) {
        for (k = 0; k < N; k++) {
            uint64_t ctr[4] = { (uint64_t)j, (uint64_t)k, update, STREAM_SCENARIO };
            uint64_t w[4];
            int i;
            orc_philox4x64_10(ctr, key, w);
            for (i = 0; i < 3; i++) d[((int64_t)i * H + j) * N + k] = uniform_sym(w[i], amp[i]);
        }
    }
}

/* Parametric uncertainty: scenario k of update t sees the model parameters
 * theta_p m_p^k, m_p^k = 1 + rho (2u - 1) uniform on [1 - rho, 1 + rho] for
 * every parameter p set in `mask` (bit p) and 1 otherwise; u from word p % 4
 * of Philox4x64-10(counter = (p / 4, k, t, 2), key = (seed, 0)).
 * Output m[k * nparam + p]. */
void orc_sample_param_multipliers(uint64_t seed, uint64_t update, int64_t N, double rho,
                                  uint32_t mask, double *m)
{
    uint64_t key[2] = { seed, 0 };
    int64_t k;
    int p;
    for (k = 0; k < N; k++) {
        for (p = 0; p < O_NPARAM; p++) {
            double mult = 1.0;
            if (mask & (1u << p)) {
                uint64_t ctr[4] = { (uint64_t)(p / 4), (uint64_t)k, update, STREAM_PARAM };
                uint64_t w[4];
                orc_philox4x64_10(ctr, key, w);
                mult = 1.0 + uniform_sym(w[p % 4], rho);
            }
            m[k * O_NPARAM + p] = mult;
        }
    }
}

/* Multipliers the evaluations below apply to scenario k's parameters
 * (NULL: every scenario sees the nominal parameters).  The steady-state check
 * always uses the nominal parameters. */
static const double *g_param_mult = NULL;

void orc_set_param_multipliers(const double *m) { g_param_mult = m; }

/* Disturbance acting on the simulated plant at closed-loop step t (Eq. 4). */
void orc_plant_disturbance(uint64_t seed, uint64_t t, const double *amp, double *d3)
{
    uint64_t key[2] = { seed, 0 };
    uint64_t ctr[4] = { 0, 0, t, STREAM_PLANT };
    uint64_t w[4];
    int i;
    orc_philox4x64_10(ctr, key, w);
    for (i = 0; i < 3; i++) d3[i] = uniform_sym(w[i], amp[i]);
}

/* ------------------------------------------------------------------------- */
/* Steady state y_ss(v) (Sec. II-A: the equilibrium manifold is assumed known).
 * At an equilibrium of FC3 the three mass/torque balances reduce to one
 * equation in the air flow W = W_cp = W_sm: the cathode balance fixes p_ca,
 * the orifice fixes p_sm, the compressor map fixes w_cp, and the remaining
 * torque balance g(W) = tau_cm - tau_cp = 0 is solved by plain bisection. */
static void state_from_flow(const double *p, double I, double W, double *x)
{
    double p_ca = p[O_P_ATM] + (W - o2_consumed(p, I)) / p[O_K_CA];
    double p_sm = p_ca + W / p[O_K_SM];
    double w = (W + p[O_A_P] * (p_sm - p[O_P_ATM])) / p[O_A_W];
    x[0] = p_ca; x[1] = w; x[2] = p_sm;
}

static double torque_balance(const double *p, double I, double W)
{
    double x[3], dx[3];
    state_from_flow(p, I, W, x);
    orc_fc3_rhs(p, x, I, dx);
    return dx[1];
}

int orc_equilibrium(const double *p, double I, double *x_eq)
{
    double lo, hi, glo, ghi;
    int it;
    if (!(I > 0.0) || !isfinite(I)) return -1;
    lo = o2_consumed(p, I);
    hi = 2.0 * p[O_LAM_REF] * lo / p[O_X_O2];
    glo = torque_balance(p, I, lo);
    ghi = torque_balance(p, I, hi);
    for (it = 0; it < 60 && ghi > 0.0; it++) { hi *= 2.0; ghi = torque_balance(p, I, hi); }
    if (!(glo > 0.0) || !(ghi < 0.0)) return -2;
    for (it = 0; it < 400; it++) {
        double mid = 0.5 * (lo + hi), g;
        if (mid <= lo || mid >= hi) break;
        g = torque_balance(p, I, mid);
        if (g > 0.0) lo = mid; else hi = mid;
    }
    state_from_flow(p, I, 0.5 * (lo + hi), x_eq);
    return 0;
}

/* Configuration of one RG problem (the parameters the paper lists: j*, dt,
 * the constraint set, epsilon; Sec. II, Sec. IV). */
typedef struct {
    double dt;        /* RK4 step (Sec. IV-A: 0.01 s) */
    int64_t H;        /* horizon j*: outputs checked at j = 0..H */
    int64_t N;        /* N_sim scenarios */
    double y_min;     /* Y = { y >= y_min } (Sec. IV-A: 1.9) */
    int ss_check;     /* 1: enforce y_ss(v) in the tightened set */
    double eps_ss;    /* epsilon of (1 - eps) Y */
    double y_c;       /* centre of Y used to tighten a one-sided set */
    int early_exit;   /* stop a rollout at its first violation (Sec. III-B/C) */
} orc_cfg;

/* Steady-state condition y_ss(v) in (1 - eps) Y (Eq. 3).  Y = {y >= y_min}
 * does not contain 0, so (1 - eps) Y is read as shrinking Y towards the
 * nominal output y_c: y_ss >= y_min + eps (y_c - y_min). */
int orc_ss_ok(const double *p, const orc_cfg *c, double I)
{
    double x[3], y;
    if (!c->ss_check) return 1;
    if (orc_equilibrium(p, I, x) != 0) return 0;
    y = orc_fc3_output(p, x, I);
    return y >= c->y_min + c->eps_ss * (c->y_c - c->y_min);
}

/* One scenario rollout (Alg. 3 parallel steps 2-3; Eq. 4): x_0 = x_t,
 * x_{j+1} = RK4(x_j, v) + d_j^k; slack s_j = h(x_j, v) - y_min at
 * j = 0..H.  Returns min_j s_j, -inf if any state or output is not finite.
 * d == NULL means the disturbance-free model of Eq. 1. */
double orc_rollout(const double *p_nominal, const orc_cfg *c, const double *x0, double I,
                   const double *d, int64_t k, int64_t *steps_out)
{
    double x[3] = { x0[0], x0[1], x0[2] }, xn[3];
    double smin = INFINITY;
    int64_t j, steps = 0;
    double pk[O_NPARAM];
    const double *p = p_nominal;
    if (g_param_mult) {
        int i;
        for (i = 0; i < O_NPARAM; i++) pk[i] = p_nominal[i] * g_param_mult[k * O_NPARAM + i];
        p = pk;
    }
    for (j = 0; j <= c->H; j++) {
        double s = orc_fc3_output(p, x, I) - c->y_min;
        int i;
        if (!isfinite(s) || !isfinite(x[0]) || !isfinite(x[1]) || !isfinite(x[2])) s = -INFINITY;
        if (s < smin) smin = s;
        if (c->early_exit && s < 0.0) break;
        if (j == c->H) break;
        orc_rk4_step(p, x, I, c->dt, xn);
        for (i = 0; i < 3; i++)
            x[i] = xn[i] + (d ? d[((int64_t)i * c->H + j) * c->N + k] : 0.0);
        steps++;
    }
    if (steps_out) *steps_out = steps;
    return smin;
}

/* Governed reference of Eq. 2. */
double orc_governed(double v_prev, double r, double kappa)
{
    return v_prev + kappa * (r - v_prev);
}

/* ---- candidate evaluation (Alg. 3 parallel steps 1-3 and Eq. 5's P) ----- */
typedef struct {
    const double *p; const orc_cfg *c; const double *x_t;
    const double *v; const int *ss; int m; const double *d;
    double *slack; int64_t *steps; int64_t begin, end;
} lane_job;

static void *lane_worker(void *arg)
{
    lane_job *J = (lane_job *)arg;
    int64_t q;
    for (q = J->begin; q < J->end; q++) {
        int64_t i = q / J->c->N, k = q % J->c->N;
        int64_t st = 0;
        J->slack[q] = orc_rollout(J->p, J->c, J->x_t, J->v[i], J->d, k, &st);
        J->steps[q] = st;
    }
    return NULL;
}

/* Evaluates m candidate kappas against all N scenarios.
 *   adm[i]       = ss_i AND (min_j s_j^k >= 0 for every k)      (Eq. 5 row)
 *   min_slack[i] = min over k, j of s_j^k (computed even when ss fails)
 *   P[i*N + k]   = ss_i AND min_j s_j^k >= 0   (optional, may be NULL)
 * Lanes are split over nthreads threads in contiguous i-major chunks, so for
 * m >= nthreads each thread owns a subset of the kappa values and all their
 * scenarios, the CPU scheme of Sec. III-B.  Returns executed RK4 steps. */
int64_t orc_eval_candidates(const double *p, const orc_cfg *c, const double *x_t,
                            double v_prev, double r, const double *kappas, int m,
                            const double *d, uint8_t *adm, double *min_slack,
                            uint8_t *P, int nthreads)
{
    int64_t L = (int64_t)m * c->N, q, total = 0;
    double *v = (double *)malloc(sizeof(double) * (size_t)m);
    int *ss = (int *)malloc(sizeof(int) * (size_t)m);
    double *slack = (double *)malloc(sizeof(double) * (size_t)(L > 0 ? L : 1));
    int64_t *steps = (int64_t *)malloc(sizeof(int64_t) * (size_t)(L > 0 ? L : 1));
    int i, t;
    if (nthreads < 1) nthreads = 1;
    for (i = 0; i < m; i++) {
        v[i] = orc_governed(v_prev, r, kappas[i]);
        ss[i] = orc_ss_ok(p, c, v[i]);
    }
    if (nthreads == 1 || L < 2) {
        lane_job J = { p, c, x_t, v, ss, m, d, slack, steps, 0, L };
        lane_worker(&J);
    } else {
        pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
        lane_job *jobs = (lane_job *)malloc(sizeof(lane_job) * (size_t)nthreads);
        for (t = 0; t < nthreads; t++) {
            lane_job J = { p, c, x_t, v, ss, m, d, slack, steps,
                           L * t / nthreads, L * (t + 1) / nthreads };
            jobs[t] = J;
            pthread_create(&th[t], NULL, lane_worker, &jobs[t]);
        }
        for (t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
        free(th); free(jobs);
    }
    for (i = 0; i < m; i++) {
        int all = ss[i];
        double s = INFINITY;
        int64_t k;
        for (k = 0; k < c->N; k++) {
            q = (int64_t)i * c->N + k;
            if (slack[q] < s) s = slack[q];
            if (!(slack[q] >= 0.0)) all = 0;
            if (P) P[q] = (uint8_t)(ss[i] && slack[q] >= 0.0);
            total += steps[q];
        }
        adm[i] = (uint8_t)all;
        if (min_slack) min_slack[i] = s;
    }
    free(v); free(ss); free(slack); free(steps);
    return total;
}

/* Joint predicate of the robust problem: candidate admissible for every
 * scenario (d != NULL) or for the disturbance-free model (d == NULL). */
static int predicate(const double *p, const orc_cfg *c, const double *x_t,
                     double v_prev, double r, double kappa, const double *d,
                     int nthreads)
{
    uint8_t a;
    if (d == NULL) {
        double v = orc_governed(v_prev, r, kappa);
        if (!orc_ss_ok(p, c, v)) return 0;
        return orc_rollout(p, c, x_t, v, NULL, 0, NULL) >= 0.0;
    }
    orc_eval_candidates(p, c, x_t, v_prev, r, &kappa, 1, d, &a, NULL, NULL, nthreads);
    return a;
}

/* Bisection of Alg. 1 on a given predicate: start at kappa = 1; a feasible
 * kappa raises the lower end (and ends the search when kappa = 1), an
 * infeasible one lowers the upper end; N_kappa iterations.  *flags bit 0 is
 * set when no tested kappa was feasible (kappa_opt stays 0: hold v_prev). */
typedef int (*pred_fn)(void *ctx, double kappa);

static double bisection(pred_fn f, void *ctx, int n_kappa, int *flags)
{
    double lo = 0.0, hi = 1.0, kappa = 1.0, kopt = 0.0;
    int it, any = 0;
    for (it = 1; it <= n_kappa; it++) {
        if (f(ctx, kappa)) {
            kopt = kappa;
            any = 1;
            if (kappa == 1.0) break;
            lo = kappa;
            kappa = (lo + hi) / 2.0;
        } else {
            hi = kappa;
            kappa = (lo + hi) / 2.0;
        }
    }
    if (flags) *flags = any ? 0 : 1;
    return kopt;
}

typedef struct {
    const double *p; const orc_cfg *c; const double *x_t; double v_prev, r;
    const double *d; int64_t k; int nthreads;
} pred_ctx;

static int pred_joint(void *vctx, double kappa)
{
    pred_ctx *q = (pred_ctx *)vctx;
    return predicate(q->p, q->c, q->x_t, q->v_prev, q->r, kappa, q->d, q->nthreads);
}

static int pred_single(void *vctx, double kappa)
{
    pred_ctx *q = (pred_ctx *)vctx;
    double v = orc_governed(q->v_prev, q->r, kappa);
    if (!orc_ss_ok(q->p, q->c, v)) return 0;
    return orc_rollout(q->p, q->c, q->x_t, v, q->d, q->k, NULL) >= 0.0;
}

/* Alg. 1: nominal (non-robust) RG, disturbance-free predictions. */
double orc_alg1(const double *p, const orc_cfg *c, const double *x_t, double v_prev,
                double r, int n_kappa, int *flags)
{
    pred_ctx q = { p, c, x_t, v_prev, r, NULL, 0, 1 };
    return bisection(pred_joint, &q, n_kappa, flags);
}

/* Alg. 2: robust RG as the minimum over scenarios of per-scenario Alg. 1. */
double orc_alg2(const double *p, const orc_cfg *c, const double *x_t, double v_prev,
                double r, int n_kappa, const double *d, int *flags)
{
    double kopt = 1.0;
    int64_t k;
    int fl = 0;
    for (k = 0; k < c->N; k++) {
        pred_ctx q = { p, c, x_t, v_prev, r, d, k, 1 };
        int f = 0;
        double kk = bisection(pred_single, &q, n_kappa, &f);
        if (kk < kopt) kopt = kk;
        if (f) fl = 1;
    }
    if (flags) *flags = fl;
    return kopt;
}

/* Joint bisection: Alg. 1 run on "admissible for all N_sim scenarios". */
double orc_bisect_joint(const double *p, const orc_cfg *c, const double *x_t,
                        double v_prev, double r, int n_kappa, const double *d,
                        int *flags, int nthreads)
{
    pred_ctx q = { p, c, x_t, v_prev, r, d, 0, nthreads };
    return bisection(pred_joint, &q, n_kappa, flags);
}

/* Alg. 3 / Eq. 5: grid kappa_i = (i-1)/(M-1), i* = max{i : P_ik = 1 for all k}. */
double orc_alg3(const double *p, const orc_cfg *c, const double *x_t, double v_prev,
                double r, int M, const double *d, int *flags, int nthreads)
{
    double *kap = (double *)malloc(sizeof(double) * (size_t)M);
    uint8_t *adm = (uint8_t *)malloc((size_t)M);
    double kopt = 0.0;
    int i, best = -1;
    for (i = 1; i <= M; i++) kap[i - 1] = (double)(i - 1) / (double)(M - 1);
    orc_eval_candidates(p, c, x_t, v_prev, r, kap, M, d, adm, NULL, NULL, nthreads);
    for (i = 1; i <= M; i++) if (adm[i - 1]) best = i;
    if (best > 0) kopt = (double)(best - 1) / (double)(M - 1);
    if (flags) *flags = (best > 0) ? 0 : 1;
    free(kap); free(adm);
    return kopt;
}

/* Parallel k-section: round 1 is the grid of Alg. 3; every further round puts
 * M equispaced points strictly inside (kappa_{i*}, kappa_{i*+1}),
 * kappa_m = lo + ((hi - lo) * m) / (M + 1), m = 1..M, and again keeps the
 * largest all-admissible point (the literal max of Eq. 5 in each round). */
double orc_ksection(const double *p, const orc_cfg *c, const double *x_t, double v_prev,
                    double r, int M, int rounds, const double *d, int *flags, int nthreads)
{
    double *kap = (double *)malloc(sizeof(double) * (size_t)M);
    uint8_t *adm = (uint8_t *)malloc((size_t)M);
    double lo, hi, kopt;
    int i, best, rd;
    for (i = 0; i < M; i++) kap[i] = (double)i / (double)(M - 1);
    orc_eval_candidates(p, c, x_t, v_prev, r, kap, M, d, adm, NULL, NULL, nthreads);
    best = -1;
    for (i = 0; i < M; i++) if (adm[i]) best = i;
    if (best < 0) {
        if (flags) *flags = 1;
        free(kap); free(adm);
        return 0.0;
    }
    if (flags) *flags = 0;
    kopt = kap[best];
    if (best == M - 1) { free(kap); free(adm); return kopt; }
    lo = kap[best]; hi = kap[best + 1];
    for (rd = 1; rd < rounds; rd++) {
        for (i = 0; i < M; i++) kap[i] = lo + ((hi - lo) * (double)(i + 1)) / (double)(M + 1);
        orc_eval_candidates(p, c, x_t, v_prev, r, kap, M, d, adm, NULL, NULL, nthreads);
        best = -1;
        for (i = 0; i < M; i++) if (adm[i]) best = i;
        if (best < 0) { hi = kap[0]; continue; }
        kopt = kap[best];
        lo = kap[best];
        if (best < M - 1) hi = kap[best + 1];
    }
    free(kap); free(adm);
    return kopt;
}

/* ------------------------------------------------------------------------- */
/* Closed loop of Fig. 1 driven by the robust RG: at each step t the scenarios
 * are redrawn (Sec. II-C), the RG picks kappa by joint bisection (search 0),
 * the grid of Alg. 3 (search 1) or k-section (search 2), and the plant moves
 * one RK4 step under v_t plus its own disturbance (Eq. 4).
 * Outputs per step: v[t], kappa[t], flags[t], x[(t+1)*3 ..] (x[0..2] = x0). */
int64_t orc_closed_loop(const double *p, const orc_cfg *c, const double *x0, double v0,
                        const double *r_seq, int T, uint64_t seed, uint64_t t0,
                        const double *amp, const double *plant_amp, int search,
                        int n_kappa, int M, int rounds, int nthreads, double param_unc_rel,
                        uint32_t param_unc_mask,
                        double *v_out, double *kappa_out, int *flags_out, double *x_out)
{
    double *d = (double *)malloc(sizeof(double) * (size_t)(3 * c->H * c->N));
    double *m = param_unc_rel > 0.0 ? (double *)malloc(sizeof(double) * (size_t)(c->N * O_NPARAM))
                                    : NULL;
    double x[3] = { x0[0], x0[1], x0[2] }, v = v0;
    int t, i;
    memcpy(x_out, x0, sizeof(double) * 3);
    for (t = 0; t < T; t++) {
        double kap, xn[3], dp[3];
        int fl = 0;
        orc_sample_disturbances(seed, t0 + (uint64_t)t, c->N, c->H, amp, d);
        /* scenario k of this update also draws its parameter multipliers;
         * the plant below runs the nominal model */
        if (m) {
            orc_sample_param_multipliers(seed, t0 + (uint64_t)t, c->N, param_unc_rel,
                                         param_unc_mask, m);
            orc_set_param_multipliers(m);
        }
        if (search == 0) kap = orc_bisect_joint(p, c, x, v, r_seq[t], n_kappa, d, &fl, nthreads);
        else if (search == 1) kap = orc_alg3(p, c, x, v, r_seq[t], M, d, &fl, nthreads);
        else kap = orc_ksection(p, c, x, v, r_seq[t], M, rounds, d, &fl, nthreads);
        if (m) orc_set_param_multipliers(NULL);
        v = orc_governed(v, r_seq[t], kap);
        v_out[t] = v; kappa_out[t] = kap; flags_out[t] = fl;
        orc_rk4_step(p, x, v, c->dt, xn);
        orc_plant_disturbance(seed, t0 + (uint64_t)t, plant_amp, dp);
        for (i = 0; i < 3; i++) x[i] = xn[i] + dp[i];
        memcpy(x_out + 3 * (t + 1), x, sizeof(double) * 3);
    }
    free(d);
    free(m);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Gradient of the robust objective g(kappa) = min over scenarios k and steps
 * j of the slack s_j^k (the quantity the admissibility test thresholds at 0),
 * at its argmin (k*, j*), with respect to kappa, x_t and every model
 * parameter.  The oracle computes it by the complex-step method (Squire &
 * Trapp, SIAM Review 40, 1998; Martins, Sturdza & Alonso, ACM TOMS 29, 2003):
 * f'(a) = Im f(a + i h) / h for analytic f, with no subtraction error, so it is
 * an independent check of the CUDA path's hand-written discrete adjoint. */
#include <complex.h>

typedef double complex cplx;

static void fc3_rhs_cs(const cplx *p, const cplx *x, cplx cur, cplx *dx)
{
    cplx p_ca = x[0], w = x[1], p_sm = x[2];
    cplx W_cp = p[O_A_W] * w - p[O_A_P] * (p_sm - p[O_P_ATM]);
    cplx W_sm = p[O_K_SM] * (p_sm - p_ca);
    cplx W_ca = p[O_K_CA] * (p_ca - p[O_P_ATM]);
    cplx W_o2 = p[O_M_O2] * p[O_N_CELL] * cur / (4.0 * p[O_FARADAY]);
    cplx e = (p[O_GAMMA] - 1.0) / p[O_GAMMA];
    cplx Pi = p_sm / p[O_P_ATM];
    cplx tau_cp = p[O_C_P] * p[O_T_ATM] / p[O_ETA_CP] * (cpow(Pi, e) - 1.0) * W_cp / w;
    cplx W_ref = p[O_LAM_REF] * W_o2 / p[O_X_O2];
    cplx v_cm = p[O_C0] + p[O_C1] * cur + p[O_C2] * cur * cur + p[O_K_P] * (W_ref - W_cp);
    cplx tau_cm = p[O_ETA_CM] * p[O_K_T] * (v_cm - p[O_K_V] * w) / p[O_R_CM];
    cplx RT = p[O_R_A] * p[O_T_ST];
    dx[0] = RT / p[O_V_CA] * (W_sm - W_ca - W_o2);
    dx[1] = (tau_cm - tau_cp) / p[O_J_CP];
    dx[2] = RT / p[O_V_SM] * (W_cp - W_sm);
}

static cplx fc3_output_cs(const cplx *p, const cplx *x, cplx cur)
{
    cplx W_sm = p[O_K_SM] * (x[2] - x[0]);
    return p[O_X_O2] * W_sm / (p[O_M_O2] * p[O_N_CELL] * cur / (4.0 * p[O_FARADAY]));
}

static void rk4_step_cs(const cplx *p, const cplx *x, cplx cur, double dt, cplx *xn)
{
    cplx k1[3], k2[3], k3[3], k4[3], t[3];
    int i;
    fc3_rhs_cs(p, x, cur, k1);
    for (i = 0; i < 3; i++) t[i] = x[i] + 0.5 * dt * k1[i];
    fc3_rhs_cs(p, t, cur, k2);
    for (i = 0; i < 3; i++) t[i] = x[i] + 0.5 * dt * k2[i];
    fc3_rhs_cs(p, t, cur, k3);
    for (i = 0; i < 3; i++) t[i] = x[i] + dt * k3[i];
    fc3_rhs_cs(p, t, cur, k4);
    for (i = 0; i < 3; i++)
        xn[i] = x[i] + (dt / 6.0) * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* s_jstar of scenario k with every input allowed to carry an imaginary part. */
static cplx slack_cs(const cplx *p, const orc_cfg *c, const cplx *x0, cplx cur, const double *d,
                     int64_t k, int64_t jstar)
{
    cplx x[3] = { x0[0], x0[1], x0[2] }, xn[3], pk[O_NPARAM];
    int64_t j;
    int i;
    if (g_param_mult) {
        /* scenario k's parameters theta m^k (the derivative stays the one
         * with respect to the nominal theta) */
        for (i = 0; i < O_NPARAM; i++) pk[i] = p[i] * g_param_mult[k * O_NPARAM + i];
        p = pk;
    }
    for (j = 0; j < jstar; j++) {
        rk4_step_cs(p, x, cur, c->dt, xn);
        for (i = 0; i < 3; i++)
            x[i] = xn[i] + (d ? d[((int64_t)i * c->H + j) * c->N + k] : 0.0);
    }
    return fc3_output_cs(p, x, cur) - c->y_min;
}

/* min over k, j of s_j^k over the full horizon (no early exit); the argmin is
 * the first (k, then j) attaining it.  Returns the min. */
double orc_min_slack_argmin(const double *p, const orc_cfg *c, const double *x0, double cur,
                            const double *d, int64_t *k_out, int64_t *j_out)
{
    double best = INFINITY;
    int64_t kb = -1, jb = -1, k, j;
    const double *p_nominal = p;
    double pk[O_NPARAM];
    for (k = 0; k < c->N; k++) {
        double x[3] = { x0[0], x0[1], x0[2] }, xn[3];
        if (g_param_mult) {
            int i;
            for (i = 0; i < O_NPARAM; i++) pk[i] = p_nominal[i] * g_param_mult[k * O_NPARAM + i];
            p = pk;
        }
        for (j = 0; j <= c->H; j++) {
            double s = orc_fc3_output(p, x, cur) - c->y_min;
            int i;
            if (s < best) { best = s; kb = k; jb = j; }
            if (j == c->H) break;
            orc_rk4_step(p, x, cur, c->dt, xn);
            for (i = 0; i < 3; i++) x[i] = xn[i] + (d ? d[((int64_t)i * c->H + j) * c->N + k] : 0.0);
        }
    }
    if (k_out) *k_out = kb;
    if (j_out) *j_out = jb;
    return best;
}

/* grad[0] = ds/dkappa, grad[1..3] = ds/dx_t, grad[4..4+NPARAM) = ds/dtheta
 * for s = s_jstar^k at kappa (v = v_prev + kappa (r - v_prev)).  Complex
 * step of size 1e-30 per direction. */
void orc_slack_grad(const double *p, const orc_cfg *c, const double *x_t, double v_prev, double r,
                    double kappa, const double *d, int64_t k, int64_t jstar, double *grad,
                    double *s_out)
{
    const double h = 1e-30;
    cplx pc[O_NPARAM], xc[3];
    int dir, i;
    for (dir = 0; dir < 4 + O_NPARAM; dir++) {
        cplx kap = kappa, s;
        for (i = 0; i < O_NPARAM; i++) pc[i] = p[i];
        for (i = 0; i < 3; i++) xc[i] = x_t[i];
        if (dir == 0) kap += _Complex_I * h;
        else if (dir < 4) xc[dir - 1] += _Complex_I * h;
        else pc[dir - 4] += _Complex_I * h;
        s = slack_cs(pc, c, xc, v_prev + kap * (r - v_prev), d, k, jstar);
        grad[dir] = cimag(s) / h;
        if (dir == 0 && s_out) *s_out = creal(s);
    }
}
