/*
 * rrg.h -- C ABI of librrg, a single-GPU (sm_103a) implementation of the
 * scenario-based robust reference governor (RG) of Ossareh, Shayne &
 * Chevalier, "CPU- and GPU-Based Parallelization of the Robust Reference
 * Governor" (arXiv 2510.08288).
 *
 * What one RG update computes (Sec. II-III):
 *   given the measured state x_t, the previous governed reference v_{t-1} and
 *   the desired reference r_t, find the largest kappa in [0, 1] such that the
 *   governed reference v = v_{t-1} + kappa (r_t - v_{t-1})            (Eq. 2)
 *   keeps the predicted output y_j = h(x_j, v) in Y = { y >= y_min } for
 *   j = 0..j* along x_{j+1} = f(x_j, v) + d_j^k for every one of N_sim
 *   sampled disturbance sequences d^k                          (Eq. 3, Eq. 4)
 *   and keeps the steady-state output in the tightened set      (Eq. 3),
 *   by bisection (Alg. 1 / Alg. 2) or by the parallel grid of Alg. 3 (Eq. 5).
 *
 * Model: FC3, the library's third-order fuel-cell air-path closed loop with
 * states x = [p_ca (Pa), w_cp (rad/s), p_sm (Pa)] and setpoint v = stack
 * current (A) (the paper's Sec. IV-A names these states and the OER >= 1.9
 * output constraint; its own equations are not published in the paper).
 * f is one classical RK4 step of size dt (Sec. IV-A: 0.01 s).
 *
 * Conventions for every entry point:
 *   - Return value: RRG_OK (0) or one of the RRG_E* codes below.  On error,
 *     rrg_last_error(h) returns a message owned by the handle (valid until
 *     the next call on that handle); for a failed rrg_create, rrg_last_error
 *     (NULL) returns the calling thread's last creation error.
 *   - A handle is not thread-safe: use one handle per host thread / stream.
 *   - Host pointers ("host") are owned by the caller and are read or written
 *     synchronously before the call returns.  Device pointers ("device", the
 *     *_dev entry points) must point to memory of the handle's device; those
 *     calls only enqueue work on the handle's stream and return at once.
 *   - Scenario arrays use the layout d[(i*H + j)*N + k]: component i in
 *     state order, step j = 0..H-1, scenario k = 0..N-1 (k fastest).
 *   - No entry point falls back to a CPU implementation.
 */
#ifndef RRG_H
#define RRG_H

#include <stdint.h>

/* Entry points are exported; everything else in the library is hidden. */
#if defined(__GNUC__)
#define RRG_API __attribute__((visibility("default")))
#else
#define RRG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------- */
#define RRG_OK        0
#define RRG_EINVAL    1   /* an argument is out of range or not finite   */
#define RRG_ENOMEM    2   /* device or host allocation failed            */
#define RRG_ECUDA     3   /* a CUDA runtime call failed                  */
#define RRG_ETIMEOUT  4   /* a bounded device-side wait gave up          */
#define RRG_ENOTIMPL  5   /* the requested option is not implemented     */

/* ---- search strategies (rrg_config.search) --------------------------- */
#define RRG_SEARCH_BISECT      0  /* Alg. 1 on the joint all-scenario predicate:
                                     one candidate per round, n_bisect rounds */
#define RRG_SEARCH_GRID        1  /* Alg. 3 / Eq. 5: M = max_candidates points */
#define RRG_SEARCH_KSECTION    2  /* repeated grid: round 1 is Alg. 3, later
                                     rounds put M points strictly inside the
                                     bracket (kappa_i*, kappa_i*+1); n_rounds */
#define RRG_SEARCH_SPEC_BISECT 3  /* same result as RRG_SEARCH_BISECT: each
                                     round evaluates every node of the next
                                     levels of Alg. 1's bisection tree that
                                     fit in max_candidates, then follows
                                     Alg. 1's path through their outcomes */

/* ---- arithmetic of the rollouts (rrg_config.precision) --------------- */
#define RRG_FP64          0  /* all rollouts in binary64                    */
#define RRG_FP32          1  /* all rollouts in binary32                    */
#define RRG_FP32_RECHECK  2  /* binary32 rollouts; any trajectory whose FP32
                                min slack lies within recheck_eps_rel * y_min
                                of zero is rolled out again in binary64 and
                                the binary64 decision replaces it            */

/* ---- early termination (rrg_config.early_exit) ----------------------- */
#define RRG_EXIT_NONE       0  /* every trajectory runs all H steps          */
#define RRG_EXIT_LANE       1  /* a trajectory stops at its first violation
                                  (Sec. III-B/C)                             */
#define RRG_EXIT_CANDIDATE  2  /* additionally, all trajectories of a
                                  candidate stop once one of them violates   */

#define RRG_NPARAM 27         /* length of the FC3 parameter vector          */
#define RRG_MAX_CANDIDATES 1024

/* FC3 parameter vector layout (SI units):
 *  0 p_atm   1 T_atm   2 T_st    3 R_a     4 V_sm    5 V_ca    6 k_sm
 *  7 k_ca    8 n_cell  9 faraday 10 M_O2   11 x_O2   12 gamma  13 c_p
 * 14 eta_cp 15 J_cp   16 eta_cm 17 k_t    18 k_v    19 R_cm   20 a_w
 * 21 a_p    22 lam_ref 23 K_p   24 c0     25 c1     26 c2                   */

typedef struct {
    double  dt;              /* RK4 step, s (> 0)                             */
    int32_t horizon;         /* H = j*: outputs checked at j = 0..H (>= 1)    */
    int32_t n_scenarios;     /* N_sim (>= 1)                                  */
    int32_t max_candidates;  /* candidates per round, 1..RRG_MAX_CANDIDATES;
                                the grid size M for GRID and KSECTION         */
    int32_t n_bisect;        /* N_kappa of Alg. 1 (>= 1)                      */
    int32_t n_rounds;        /* KSECTION rounds (>= 1)                        */
    int32_t search;          /* RRG_SEARCH_*                                  */
    int32_t precision;       /* RRG_FP64 / RRG_FP32 / RRG_FP32_RECHECK        */
    int32_t early_exit;      /* RRG_EXIT_*                                    */
    int32_t ss_check;        /* 1: require y_ss(v) >= y_min + eps_ss (y_c -
                                y_min) (Eq. 3, steady-state tightening)       */
    double  y_min;           /* output constraint y >= y_min (Sec. IV-A: 1.9) */
    double  eps_ss;          /* epsilon of (1 - eps) Y, in [0, 1)             */
    double  y_c;             /* nominal output the tightening shrinks towards */
    double  recheck_eps_rel; /* FP64 recheck band, relative to y_min          */
    double  dist_amp[3];     /* scenario disturbance half-ranges (Sec. IV-A:
                                50 Pa, 10 rad/s, 50 Pa)                       */
    int32_t probe_steps;     /* RRG_SEARCH_SPEC_BISECT only; > 0 pipelines its
                                first two rounds: round 1 runs its first
                                probe_steps steps, round 2's tree is built from
                                those provisional outcomes and runs while round
                                1 finishes; round 1 is then re-walked with its
                                final outcomes and, if any decision changed,
                                round 2 is redone (counted in rrg_stats.repairs).
                                The result is always Alg. 1's.  0 = off;
                                ignored when >= horizon                       */
    double  param_unc_rel;   /* parametric uncertainty (the sampled model
                                uncertainties of Sec. I next to the
                                disturbances of Eq. 4); 0 = off, else in
                                (0, 1): scenario k of an update sees every
                                parameter p set in param_unc_mask scaled by
                                m_p^k = 1 + rho (2u - 1), rho = param_unc_rel,
                                u = (w >> 11) 2^-53 with w word p % 4 of
                                Philox4x64-10(counter = (p / 4, k,
                                update_index, 2), key = (seed, 0)); drawn with
                                the disturbances by rrg_sample_scenarios.  The
                                rollouts, rechecks and the adjoint use theta_p
                                m_p^k (pressures measured from scenario k's
                                p_atm); the steady-state check (Eq. 3) and the
                                simulated plant keep the nominal theta.       */
    uint32_t param_unc_mask; /* bit p: parameter p is uncertain (bits below
                                RRG_NPARAM only)                             */
    int32_t scenarios_in_register; /* 1: the rollouts draw each step's
                                disturbances from its Philox counters inside
                                the trajectory loop instead of reading the
                                stored array (rrg_sample_scenarios then writes
                                no array); same values, same results.  0
                                (default): stored array.  Single-problem
                                handles only; rrg_set_scenarios is then
                                RRG_EINVAL.                                   */
    int64_t scenario_base;   /* global index of the handle's scenario 0, in
                                [0, 2^62]: scenario k of the handle draws its
                                disturbances (and parameter multipliers) from
                                the Philox counters of global scenario
                                scenario_base + k.  Handles with bases 0, n_1,
                                n_1 + n_2, ... then hold consecutive shards of
                                one scenario set (Sec. II-C's N_sim scenarios
                                are independent), and the AND of their
                                admissibility flags (the min of their min
                                slacks) is the unsharded handle's; see
                                rrg_bisect_plan.  Default 0.  Single-problem
                                handles only (the batched handles and the
                                allocation-free call ignore or reject it).    */
} rrg_config;

/* FC3 parameters perturbed by default: k_ca, eta_cp, J_cp, eta_cm, R_cm,
 * a_w, a_p (the air path's dynamics; k_sm, which also scales the OER output
 * map, stays nominal). */
#define RRG_PARAM_UNC_MASK_FC3 0x0039c080u

typedef struct rrg_ctx *rrg_handle;

/* Counters kept by a handle since creation or the last rrg_reset_stats.
 * Under closed-loop graph replay the launch, rollout and round counts are
 * those of the kernels that ran: a conditional node's body is counted on the
 * replays that executed it (by the device, read back here). */
typedef struct {
    uint64_t launches;          /* kernels this handle launched               */
    uint64_t rollout_launches;  /* of which rollout kernels                   */
    uint64_t lane_steps;        /* RK4 steps executed over all trajectories   */
    uint64_t lane_steps_fp64;   /* of which in binary64                       */
    uint64_t rechecked;         /* trajectories re-run in binary64            */
    uint64_t rounds;            /* search rounds run                          */
    double   rollout_ms;        /* summed device time of rollout launches
                                   (only while profiling is on)               */
    double   recheck_ms;        /* same for recheck launches                  */
    uint64_t timed_rollouts;    /* rollout launches covered by rollout_ms     */
    uint64_t repairs;           /* pipelined rounds redone after a provisional
                                   outcome turned out wrong                   */
    uint64_t graph_conditional; /* 1: the cached closed-loop graph holds the
                                   rounds after a pipelined pair in a
                                   conditional node (run only when needed)    */
    uint64_t lane_steps_paired; /* of lane_steps, those run two trajectories
                                   per thread (rrg_set_pairing)               */
    uint64_t wait_timeouts;     /* bounded device waits that gave up (a TMA
                                   copy that never landed); each makes the
                                   lanes it served report a violation, so a
                                   result is never admissible on missing
                                   data.  0 in every correct run.             */
    uint64_t lane_steps_tma;    /* of lane_steps, those whose disturbances came
                                   through the TMA ring (rrg_set_tma)         */
} rrg_stats;

/* Fills *cfg with the defaults of the paper's fuel-cell experiment: dt 0.01,
 * H 500, N 32, M 32, N_kappa 12, 3 rounds, SPEC_BISECT, FP32_RECHECK,
 * EXIT_CANDIDATE, ss_check 1, y_min 1.9, eps_ss 0.05, y_c 2.2, recheck band
 * 1e-6, amplitudes (50, 10, 50), probe_steps 128, no parametric
 * uncertainty (param_unc_rel 0, param_unc_mask RRG_PARAM_UNC_MASK_FC3).
 * Never fails. */
RRG_API void rrg_config_default(rrg_config *cfg);

/* Creates a governor on the current CUDA device.
 *   model_params  host, n_params doubles in the FC3 layout above; copied.
 *   cfg           host; copied.  Validated: RRG_EINVAL on a bad field.
 *   cuda_stream   a cudaStream_t of the current device; all work of the
 *                 handle goes there.  NULL: the handle creates (and later
 *                 destroys) a private non-blocking stream of its own.
 *   out           host; receives the handle.
 * Allocates all device memory the handle needs (about 36 H N bytes of
 * scenarios, 24 H N with scenarios_in_register, plus O(max_candidates * N)
 * bytes of per-candidate and recheck buffers).  RRG_ENOMEM / RRG_ECUDA on failure (nothing leaks). */
RRG_API int rrg_create(const double *model_params, int n_params, const rrg_config *cfg,
               void *cuda_stream, rrg_handle *out);

/* Releases every resource of h (after synchronising its stream).  NULL is
 * accepted.  Returns RRG_ECUDA if the stream reported an error. */
RRG_API int rrg_destroy(rrg_handle h);

RRG_API const char *rrg_last_error(rrg_handle h);

/* Draws the N scenario sequences of one RG update on the device (Sec. II-C:
 * scenarios are redrawn at every RG time step; Alg. 3 step 2):
 * d_j^k[i] = a_i (2u - 1), u = (w_i >> 11) 2^-53 with (w_0, w_1, w_2, w_3) =
 * Philox4x64-10(counter = (j, k, update_index, 0), key = (seed, 0)).
 * With precision RRG_FP32 or RRG_FP32_RECHECK only the binary32 copy used by
 * the binary32 rollouts is drawn, from the top 24 bits of the same words:
 * RN32((w_i >> 40) - 2^23) a_i 2^-23) (within a_i 2^-23 plus one rounding of
 * the binary64 value); the binary64 values are regenerated from the same
 * counters wherever they are needed (recheck, rrg_get_scenarios).
 * Asynchronous on the handle's stream. */
RRG_API int rrg_sample_scenarios(rrg_handle h, uint64_t seed, uint64_t update_index);

/* Copies the per-scenario parameter multipliers of the current scenarios,
 * m[k * RRG_NPARAM + p], to host m (N * RRG_NPARAM doubles; all 1 when
 * param_unc_rel = 0 or before the first draw).  Synchronous. */
RRG_API int rrg_get_param_multipliers(rrg_handle h, double *m);

/* Loads explicit multipliers m[k * RRG_NPARAM + p] (host, N * RRG_NPARAM
 * doubles, each finite and > 0; parameters outside param_unc_mask are used
 * as given too).  RRG_EINVAL unless the handle was created with
 * param_unc_rel > 0.  The next rrg_sample_scenarios overwrites them.
 * Synchronous. */
RRG_API int rrg_set_param_multipliers(rrg_handle h, const double *m);

/* Loads explicit scenarios instead: d host, 3*H*N doubles (layout above).
 * The binary32 copy is the round-to-nearest of each value.  Synchronous. */
RRG_API int rrg_set_scenarios(rrg_handle h, const double *d);

/* Copies the current scenarios (binary64, layout above, 3*H*N doubles) to the
 * host buffer d.  Synchronous. */
RRG_API int rrg_get_scenarios(rrg_handle h, double *d);

/* Evaluates m candidate kappas on the current scenarios (Alg. 3 parallel
 * steps 1-3 for given kappas, Eq. 5's P).  Host buffers:
 *   x_t[3], v_prev, r_t   the RG inputs (finite; v values must be > 0)
 *   kappas[m]             each in [0, 1]; 1 <= m <= max_candidates
 *   admissible[m]  out    1 iff the steady-state check passes and every
 *                         scenario's trajectory keeps y >= y_min at j=0..H
 *   min_slack[m]   out    (optional, NULL) min over scenarios and steps of
 *                         y_j - y_min; NaN when the steady-state check fails
 *                         (no rollout is run); with early exit on, for an
 *                         inadmissible candidate it is only an upper bound
 *   P[m*N]         out    (optional, NULL) P[i*N + k] = 1 iff candidate i is
 *                         admissible for scenario k; when P is requested the
 *                         candidate-level early exit is not used
 * Synchronous. */
RRG_API int rrg_eval_candidates(rrg_handle h, const double *x_t, double v_prev, double r_t,
                        const double *kappas, int m, uint8_t *admissible,
                        double *min_slack, uint8_t *P);

/* Error of the binary32 rollouts against binary64, per trajectory and per
 * step: the quantity behind the FP32 + FP64-recheck rule (the paper reports
 * no visible effect of single precision in Sec. III-C and leaves its accuracy
 * open in Sec. V).  For each of the m candidate kappas (host, each in [0, 1])
 * and each scenario k of the current scenarios, the trajectory from x_t is
 * integrated over the full horizon, without early exit, twice: exactly as the
 * binary32 rollouts integrate it (stored binary32 disturbances, the same
 * constants and right-hand side) and exactly as the binary64 rollouts and the
 * recheck do (binary64 disturbances, regenerated from their Philox counters
 * unless rrg_set_scenarios stored them).  Host outputs, each m * N values at
 * [i * N + k]:
 *   err[]     max over j = 0..H of |s32_j - s64_j| (+inf where exactly one
 *             side is non-finite at some step, 0 at steps where both are)
 *   j_err[]   (optional) the first step attaining it
 *   smin32[]  (optional) min over j of s32_j (as binary64); equals the
 *             binary32 rollout's min slack of that trajectory bit for bit
 *   smin64[]  (optional) min over j of s64_j
 *   unsafe[]  (optional) number of steps at which the recheck rule with the
 *             absolute band `band` decides wrongly: s32_j >= band but
 *             s64_j < 0, or s32_j < -band but s64_j >= 0.  The handle's
 *             band is recheck_eps_rel * |y_min|.
 *   ratio[]   (optional) max over j of |s32_j - s64_j| / max(band, |s64_j|):
 *             below 1, no step of the trajectory can be decided wrongly by
 *             the band rule (1 / ratio is the margin)
 * The handle must use RRG_FP32 or RRG_FP32_RECHECK (RRG_EINVAL otherwise);
 * 1 <= m <= max_candidates; band finite and >= 0.  Allocates 40 m N bytes of
 * device scratch on first use (grown on demand).  Synchronous.  RRG_EINVAL,
 * RRG_ECUDA. */
RRG_API int rrg_slack_error(rrg_handle h, const double *x_t, double v_prev, double r_t,
                    const double *kappas, int m, double band, double *err, int32_t *j_err,
                    double *smin32, double *smin64, int32_t *unsafe, double *ratio);

/* One robust RG update with the configured search on the current scenarios.
 * Host in: x_t[3], r_t, v_prev.  Host out: *v_t (Eq. 2 applied to the chosen
 * kappa, evaluated as v_prev + kappa * (r_t - v_prev) without fused
 * multiply-add), *kappa, *flags (bit 0: no evaluated candidate was admissible,
 * so kappa = 0 and v_t = v_prev; bit 1: inputs were rejected on the device).
 * Synchronous. */
RRG_API int rrg_step(rrg_handle h, const double *x_t, double r_t, double v_prev,
             double *v_t, double *kappa, int32_t *flags);

/* Same as rrg_step with device pointers: d_x_t[3], *d_r_t, *d_v_prev in;
 * *d_v_t, *d_kappa, *d_flags out.  Asynchronous; nothing is copied to or from
 * the host, so it can be enqueued back to back or captured in a CUDA graph. */
RRG_API int rrg_step_dev(rrg_handle h, const double *d_x_t, const double *d_r_t,
                 const double *d_v_prev, double *d_v_t, double *d_kappa,
                 int32_t *d_flags);

/* Equilibrium of FC3 at constant setpoint v (Sec. II-A's equilibrium
 * manifold) and its output y_ss(v), in binary64 on the device.  Host out.
 * RRG_EINVAL if v is not positive and finite or no equilibrium is found. */
RRG_API int rrg_equilibrium(rrg_handle h, double v, double *x_eq, double *y_ss);

/* Closed loop of Fig. 1 with a simulated plant, T updates, all on the device:
 * for t = 0..T-1: sample scenarios (seed, t0 + t); RG update with r_seq[t];
 * plant step x_{t+1} = RK4(x_t, v_t) + d_plant, d_plant drawn like the
 * scenarios from Philox4x64-10(counter = (0, 0, t0 + t, 1), key = (seed, 0))
 * with half-ranges plant_amp[3].
 *   host in:  x0[3], v0, r_seq[T], plant_amp[3]
 *   host out: v_out[T], kappa_out[T], flags_out[T], x_out[3*(T+1)] (x_out[0..2]
 *             = x0).  Any output pointer may be NULL.
 *   use_graph: 1 replays one captured CUDA graph per update, 0 launches the
 *             kernels of each update directly.
 * Synchronous. */
RRG_API int rrg_closed_loop(rrg_handle h, const double *x0, double v0, const double *r_seq,
                    int T, uint64_t seed, uint64_t t0, const double *plant_amp,
                    int use_graph, double *v_out, double *kappa_out,
                    int32_t *flags_out, double *x_out);

/* Device-pointer form of rrg_closed_loop: d_r_seq[T] in; d_v_out[T],
 * d_kappa_out[T], d_flags_out[T], d_x_out[3*(T+1)] out (d_x_out[0..2] is
 * written with x0).  x0, v0 and plant_amp are host values.  Asynchronous.
 * x0 == NULL continues the loop where the previous call on this handle left
 * it: state, v_{t-1} and the update counter t carry over, r_seq and the
 * outputs are indexed by that running t (so they must cover every update of
 * the run), and the scenarios of update t use update index t0 + t. */
RRG_API int rrg_closed_loop_dev(rrg_handle h, const double *x0, double v0, const double *d_r_seq,
                        int T, uint64_t seed, uint64_t t0, const double *plant_amp,
                        int use_graph, double *d_v_out, double *d_kappa_out,
                        int32_t *d_flags_out, double *d_x_out);

/* One plant step of the closed loop above with host buffers: x_next =
 * RK4(x_t, v_t) + d_plant(seed, t).  Synchronous. */
RRG_API int rrg_plant_step(rrg_handle h, const double *x_t, double v_t, uint64_t seed, uint64_t t,
                   const double *plant_amp, double *x_next);

/* Shape of RRG_SEARCH_SPEC_BISECT: m tree nodes per round (1 .. max_candidates)
 * and the probe length that pipelines its first two rounds (0, or any value
 * when the handle was created with probe_steps > 0).  The result is Alg. 1's
 * for every shape; only the time per update changes.  rrg_set_tuning waits
 * for the handle's stream; RRG_EINVAL for other searches or values. */
RRG_API int rrg_set_tuning(rrg_handle h, int m, int probe_steps);
RRG_API int rrg_get_tuning(rrg_handle h, int32_t *m, int32_t *probe_steps);

/* Autotuner of RRG_SEARCH_SPEC_BISECT: on the current scenarios and the host
 * inputs x_t[3], r_t, v_prev, times 1 + repeats updates (CUDA events on the
 * handle's stream) for each tree width m in {4, 8, ..., max_candidates} and
 * probe length in {0, 32, 128, 512} (below the horizon; 0 only unless the
 * handle has probe storage), keeps the fastest and returns it in *m_out,
 * *probe_out and its mean device time per update in *ms_out (each may be
 * NULL).  Synchronous; the cached closed-loop graph is discarded. */
RRG_API int rrg_autotune(rrg_handle h, const double *x_t, double r_t, double v_prev, int repeats,
                 int32_t *m_out, int32_t *probe_out, double *ms_out);

/* Trajectories per thread of the binary32 rollouts that read the stored
 * scenario array (RRG_FP32, RRG_FP32_RECHECK; scenarios_in_register = 0):
 * RRG_PAIR_NEVER, one trajectory per thread; RRG_PAIR_FILLED, two candidates
 * of one scenario per thread (one load of each disturbance, two independent
 * step chains) in register-ring launches large enough that the paired grid
 * fills the SMs at least six times over, one elsewhere (launches that take
 * the TMA ring, rrg_set_tma, stay single: the TMA ring measured faster than
 * either pairing);
 * RRG_PAIR_ALWAYS, two in every launch whose rows are full-horizon segments,
 * on whichever ring the launch takes (the probe and continuation launches of
 * a pipelined search never pair).
 * The same arithmetic in every mode: every admissible flag, every search
 * result and the min slack of every admissible candidate are identical; only
 * the time changes.  Both calls wait for the handle's stream; setting the mode
 * discards the cached closed-loop graph.  RRG_EINVAL for a null handle or
 * pointer or a mode outside 0..2.  New handles start at RRG_PAIR_FILLED. */
#define RRG_PAIR_NEVER 0
#define RRG_PAIR_FILLED 1
#define RRG_PAIR_ALWAYS 2
RRG_API int rrg_set_pairing(rrg_handle h, int mode);
RRG_API int rrg_get_pairing(rrg_handle h, int32_t *mode);

/* How the binary32 rollouts on the stored scenario array bring in their
 * disturbances.  The TMA ring: one tensor copy per warp of a 32-scenario x
 * 16-step x 3-component box into shared memory, completion on an mbarrier, so
 * a step reads its values with three shared loads.  Otherwise: per-lane
 * 4-byte asynchronous copies into a shared-memory ring (launches of at most
 * 16 warps per SM, 64 under parametric uncertainty) or register prefetch
 * (larger launches, optionally two candidates per thread, rrg_set_pairing).
 * RRG_TMA_NEVER: never the TMA; RRG_TMA_AUTO (the default where available):
 * the TMA for launches of at least 24 warps per SM, where warps compete for
 * issue and the saved load instructions pay, ahead of pairing (which it beat
 * where both apply); below, where a warp running alone would pay the
 * chunk's wait and warp votes on its dependency chain, the per-lane forms;
 * RRG_TMA_ALWAYS: the TMA for every such launch.  The results are identical;
 * only the time changes.  The TMA needs stored binary32 scenarios with
 * n_scenarios a multiple of 4 (the tensor map's row stride must be a multiple
 * of 16 bytes) and a driver that encodes the map: without it rrg_get_tma
 * reports RRG_TMA_NEVER and setting another mode returns RRG_EINVAL.  Setting
 * waits for the handle's stream and discards the cached closed-loop graph;
 * RRG_EINVAL for a mode outside 0..2. */
#define RRG_TMA_NEVER 0
#define RRG_TMA_AUTO 1
#define RRG_TMA_ALWAYS 2
RRG_API int rrg_set_tma(rrg_handle h, int mode);
RRG_API int rrg_get_tma(rrg_handle h, int32_t *mode);

/* Test support for the device-side failure handling (0, the default, in
 * normal use).  RRG_INJECT_TMA_NO_COPY: the TMA ring issues no copies, so each
 * warp's first chunk wait runs out (after at most 0.1 s): the warp counts one
 * timeout in rrg_stats.wait_timeouts, its running lanes report a violation
 * (no candidate is admissible on data that did not arrive), the kernel
 * returns and the handle stays usable.  Waits for the stream and discards the
 * cached closed-loop graph; RRG_EINVAL for unknown flags. */
#define RRG_INJECT_TMA_NO_COPY 1
RRG_API int rrg_set_injection(rrg_handle h, int flags);

/* Times 1 + repeats updates of the handle's search (rrg_autotune's
 * protocol: current scenarios, host inputs x_t[3], r_t, v_prev, CUDA events
 * on the handle's stream) in each pairing mode, keeps the fastest and returns
 * it in *mode_out and the mean device time per update of each mode in
 * ms_out[3] (each may be NULL).  Synchronous; the cached closed-loop graph is
 * discarded.  RRG_EINVAL for invalid inputs, RRG_ECUDA if an update fails
 * (the mode is then left unchanged). */
RRG_API int rrg_autotune_pairing(rrg_handle h, const double *x_t, double r_t, double v_prev, int repeats,
                         int32_t *mode_out, double *ms_out);

/* Gradient of the robust objective g(kappa) = min over scenarios k and steps
 * j = 0..H of s_j^k = h(x_j^k, v) - y_min on the current scenarios, with
 * v = v_prev + kappa (r_t - v_prev) (Eq. 2) and x_{j+1} = RK4(x_j, v) + d_j^k
 * over the full horizon (Eq. 4; Alg. 3's admissibility test is g >= 0 plus
 * the steady-state check).  The derivative is taken at the argmin (k*, j*)
 * (first k, then first j, attaining the min; a subgradient where the argmin
 * is not unique) by the discrete adjoint of the RK4 recursion: the forward
 * pass saves every trajectory's state every `checkpoint` steps, the reverse
 * pass recomputes trajectory k*'s segments before j* in parallel and then
 * sweeps them backwards; the handle keeps N * (H / checkpoint + 1) * 3 and
 * (H + 1) * 12 doubles of device scratch for them, allocated on first use.
 * Errors: RRG_EINVAL for a null handle or an argument outside its range,
 * RRG_ECUDA (message in rrg_last_error) from the allocation or the
 * launches.  Host in: x_t[3]
 * (finite), v_prev, r_t (> 0), kappa in [0, 1], checkpoint in [1, 65536], precision
 * RRG_FP64 or RRG_FP32 (arithmetic of both passes).  Host out (each may be
 * NULL): *g, grad[31] = (dg/dkappa, dg/dx_t[3], dg/dtheta[27] in the FC3
 * parameter layout), *k_star, *j_star.  Under parametric uncertainty
 * scenario k runs with theta_p m_p^k and dg/dtheta is with respect to the
 * nominal theta.  rrg_slack_gradients with m = 1.  Synchronous. */
RRG_API int rrg_slack_gradient(rrg_handle h, const double *x_t, double v_prev, double r_t, double kappa,
                       int checkpoint, int precision, double *g, double *grad, int64_t *k_star,
                       int64_t *j_star);

/* The same for m kappas at once (host kappas[m], 1 <= m <= max_candidates,
 * each in [0, 1]): one forward pass over the m x N trajectories, one argmin
 * and one reverse sweep per kappa, all in one launch each.  With 4,096
 * scenarios the forward pass of one kappa occupies one warp per SM, so a few
 * kappas cost about as much as one.  The forward pass integrates with the
 * rollouts' arithmetic (deviation coordinates about each candidate's
 * equilibrium; the binary32 gradient reads the stored binary32 disturbances
 * when the handle draws them); the reverse sweep recomputes the segments
 * before j* from the saved states in the gauge form of the model.  Host out,
 * each may be NULL: g[m], grad[m * 31] (kappa i's 31 values at 31 i),
 * k_star[m], j_star[m], ss_ok[m] (1: the steady-state check of Eq. 3 passed
 * at kappa i; always 1 with ss_check off).  Device scratch as above, times m
 * (allocated on first use, grown on demand).  Synchronous.  RRG_EINVAL,
 * RRG_ECUDA. */
RRG_API int rrg_slack_gradients(rrg_handle h, const double *x_t, double v_prev, double r_t,
                        const double *kappas, int m, int checkpoint, int precision, double *g,
                        double *grad, int64_t *k_star, int64_t *j_star, uint8_t *ss_ok);

/* Adjoint-driven search for the largest admissible kappa on the current
 * scenarios; only the handle's own evaluation (rrg_eval_candidates) decides,
 * the gradients steer:
 *   A. one forward pass (no reverse sweep) at kappa = j / G, j = 0..G (G = 8,
 *      or the largest power of two with G + 1 <= max_candidates): g and the
 *      steady-state outcome at each point.  kappa = 1 (Alg. 1's first test)
 *      is evaluated by the handle unless its g is below -1e-4 or its
 *      steady-state check failed (then it is inadmissible in binary64 too);
 *      admissible: done.  Alg. 1's path below kappa = 1 through the grid's
 *      outcomes (steady-state check and g >= 0, in the gradient's precision)
 *      gives a bracket of width 1 / G;
 *   B. the reverse sweep of the bracket's upper (violating) end on the
 *      saved states, and a Newton step from there as the first estimate (the
 *      secant through both ends' values when it leaves the bracket);
 *   C. Newton steps on g(kappa) = 0, one gradient each, kept inside the
 *      bracket the outcomes narrow, until the step, or the next iterate's
 *      error predicted from the curvature of the last two slopes, is below
 *      tol / 4, or max_iter gradients have been computed;
 *   D. the handle evaluates [k - tol/2, k + tol/2] around the last iterate;
 *      if it does not judge the lower end admissible and the upper one not,
 *      exact rounds of max_candidates points equispaced inside the judged
 *      bracket (Alg. 3's rule) shrink it to at most tol.
 * Host out: *kappa = the judged bracket's admissible end (0 if none), *flags
 * (bit 0: no evaluated kappa was admissible), *iterations (gradient
 * evaluations, each kappa of a multi-kappa call counted).  Under a monotone
 * predicate the result is within tol + 2^(1 - N) of Alg. 1's with N
 * iterations.  Needs max_candidates >= 3.  Synchronous.  RRG_EINVAL,
 * RRG_ECUDA. */
RRG_API int rrg_newton_search(rrg_handle h, const double *x_t, double r_t, double v_prev, double tol,
                      int max_iter, int checkpoint, int precision, double *kappa, int32_t *flags,
                      int32_t *iterations);

/* Profiling: while on, every rollout and recheck launch is bracketed by CUDA
 * events on the handle's stream and their durations are summed into
 * rrg_stats.rollout_ms / recheck_ms.  The forward pass of rrg_slack_gradient
 * (every scenario over the full horizon) counts as a rollout launch. */
RRG_API int rrg_set_profiling(rrg_handle h, int on);

/* Reads the counters (synchronises the handle's stream).  Host out. */
RRG_API int rrg_get_stats(rrg_handle h, rrg_stats *out);
RRG_API int rrg_reset_stats(rrg_handle h);

/* ---- Alg. 1 rounds for evaluations the caller runs --------------------
 * The searches of rrg_step run on the device without a host round trip.  A
 * caller that evaluates candidates itself -- typically one handle per shard
 * of the scenarios (rrg_config.scenario_base), one per GPU or several on one,
 * combined per round by an AND of their admissible flags -- splits each round
 * of the speculative bisection into plan -> evaluate -> combine -> decide:
 *   rrg_bisect_init(&s, n_bisect);
 *   while (!s.done) {
 *     rrg_bisect_plan(&s, m_max, kappas, &m);          (m >= 1 while !done)
 *     for each shard: rrg_eval_candidates(shard, x_t, v_prev, r_t, kappas, m,
 *                                         adm_shard, NULL, NULL);
 *     adm[i] = AND over shards of adm_shard[i];         (the exchange)
 *     rrg_bisect_decide(&s, adm, m);
 *   }
 *   kappa = s.kappa_opt; flags bit 0 = !s.any; v_t = v_prev + kappa (r_t - v_prev)
 * The result is Alg. 1's (Sec. II-B, the joint predicate over all scenarios
 * of all shards): each round evaluates every node of the next levels of
 * Alg. 1's bisection tree that fit in m_max (2^d - 1 nodes, or 2^(d-1) from
 * a kappa = 1 root, whose admissible outcome ends the search), and decide
 * walks Alg. 1's path through their outcomes -- the same tree and walk as
 * RRG_SEARCH_SPEC_BISECT without pipelining.  Host only: no device work, no
 * handle.  Nodes are listed breadth-first: node 0 is the state's kappa; node
 * n's children follow "not admissible" (upper bracket end <- its kappa)
 * before "admissible" (lower end <- its kappa); children's kappas are the
 * bracket midpoints (lo + hi) / 2.  Errors (RRG_EINVAL): null pointers,
 * n_bisect outside [1, 62], m_max < 1, decide on a finished state or with an
 * m that is not the size of the planned round. */
typedef struct {
    double  lo, hi;        /* Alg. 1's bracket                              */
    double  kappa;         /* the kappa Alg. 1 tests next                   */
    double  kappa_opt;     /* largest admissible kappa found (0: none yet)  */
    int32_t iter;          /* iterations of Alg. 1 done (of n_bisect)       */
    int32_t n_bisect;      /* N_kappa                                       */
    int32_t any;           /* 1: some tested kappa was admissible           */
    int32_t done;          /* 1: kappa_opt is Alg. 1's result               */
} rrg_bisect_state;

RRG_API int rrg_bisect_init(rrg_bisect_state *s, int n_bisect);
/* kappas: host, room for m_max doubles; *m receives the round's node count
 * (0 once the search is done). */
RRG_API int rrg_bisect_plan(const rrg_bisect_state *s, int m_max, double *kappas, int32_t *m);
/* admissible: host, the m combined outcomes of the planned kappas. */
RRG_API int rrg_bisect_decide(rrg_bisect_state *s, const uint8_t *admissible, int m);

/* ---- allocation-free candidate evaluation ---------------------------
 * The paper has no counterpart of this entry point.  It is for callers that
 * must not allocate device memory once they run: a fixed-rate control task
 * (the governor's natural home) where an allocation can block for an
 * unbounded time or fail once device memory is fragmented, or a host program
 * that hands all device memory out from its own pool and does not allow a
 * library to call cudaMalloc.  Such a caller cannot create a handle
 * (rrg_create allocates), so this call needs none.
 *
 * It computes what rrg_eval_candidates computes (without P) for m kappas on
 * scenarios the caller already holds on the device:
 *   model_params   host, RRG_NPARAM doubles; cfg host (validated like
 *                  rrg_create; search and n_rounds are ignored)
 *   cuda_stream    stream to enqueue on (NULL: the legacy default stream)
 *   d_scen64       device, 3*H*N doubles (layout above); needed unless
 *                  cfg->precision == RRG_FP32
 *   d_scen32       device, 3*H*N floats, the binary32 copy; needed unless
 *                  cfg->precision == RRG_FP64
 *   d_x_t          device, 3 doubles; v_prev, r_t by value (finite, > 0)
 *   d_kappas       device, m doubles, each in [0, 1] (not checked: device data)
 *   d_admissible   device out, m bytes; d_min_slack device out, m doubles or
 *                  NULL (same meaning as in rrg_eval_candidates)
 * Its only working memory is one file-scope device array of
 * RRG_STATIC_SCRATCH_BYTES bytes, which every GPU that loads the library
 * holds until the process exits.  Limits: 1 <= m <= RRG_STATIC_MAX_CANDIDATES
 * (and <= cfg->max_candidates) and m * n_scenarios <= RRG_STATIC_MAX_LANES;
 * beyond them the call returns RRG_EINVAL and rrg_last_error(NULL) says which
 * limit was hit.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.  It only enqueues work (asynchronous).
 *
 * The first call on each device looks up the scratch's device address
 * (cudaGetSymbolAddress) with that device current, and looks it up again
 * whenever the device's current context has changed since (after a
 * cudaDeviceReset, for example, the module and its array are loaded anew);
 * make the first call on a device, and the first after such a change, before
 * any stream capture begins.  The binary64 rollouts evaluate x^e - 1 by the
 * same series as a handle's, so results equal rrg_eval_candidates's on the
 * same scenarios bit for bit.  Every call uses the same scratch, which
 * keeps the last call's contents; each call re-initialises everything it
 * reads, but calls that may overlap on the GPU (on different streams, or from
 * host threads without ordering between them) race on the scratch and their
 * results are undefined.  Parametric uncertainty is not available here
 * (param_unc_rel != 0: RRG_ENOTIMPL).  Errors: RRG_EINVAL, RRG_ENOTIMPL,
 * RRG_ECUDA. */
#define RRG_STATIC_MAX_CANDIDATES 64
#define RRG_STATIC_MAX_LANES 131072
#define RRG_STATIC_SCRATCH_BYTES (2u << 20)
RRG_API int rrg_eval_candidates_static(const double *model_params, int n_params, const rrg_config *cfg,
                               void *cuda_stream, const double *d_scen64, const float *d_scen32,
                               const double *d_x_t, double v_prev, double r_t,
                               const double *d_kappas, int m, uint8_t *d_admissible,
                               double *d_min_slack);

/* Measured throughput of the arithmetic units the rollouts use, on the current
 * device (about 10 ms): binary32 FMA and binary64 FMA in TFLOP/s (an FMA
 * counted as 2 flops) and MUFU exp2 in Top/s; each output may be NULL.
 * Synchronous on the legacy default stream.  RRG_ECUDA / RRG_ENOMEM. */
RRG_API int rrg_alu_peaks(double *fp32_tflops, double *fp64_tflops, double *mufu_tops);

/* Latency of one binary32 trajectory step on the current device: one warp
 * integrates `steps` RK4 steps of the rollout (the handle's model, setpoint v,
 * from the equilibrium of v, no disturbance, the slack test of every step)
 * and the SM clock times it; *cycles_per_step receives the least of three
 * runs.  The bound of a launch whose lanes each run alone on a warp
 * scheduler (the closed loop's long rollouts).  Synchronous on the handle's
 * stream.  RRG_EINVAL: v not finite or <= 0, steps < 1, no equilibrium. */
RRG_API int rrg_step_latency(rrg_handle h, double v, int steps, double *cycles_per_step);

/* ------------------------------------------------------------------------ */
/* Batched instances: S independent robust RG problems (instance s with its
 * own N_s scenarios and horizon H_s) that share the model, dt, the search and
 * its settings, advanced together by one fixed launch sequence per update.
 * The trajectories of all instances' candidates are tiles (instance,
 * candidate, block of scenarios) of one persistent rollout launch per search
 * round, taken from a queue in longest-horizon-first order.  Instance s draws
 * its scenarios exactly as rrg_sample_scenarios with seed + s (mod 2^64), and
 * its simulated plant disturbance as rrg_plant_step with seed + s.  Search:
 * RRG_SEARCH_GRID (Alg. 3) or RRG_SEARCH_KSECTION with max_candidates per
 * instance and round, or RRG_SEARCH_SPEC_BISECT (Alg. 1's result, trees of a
 * tunable width, see rrg_batch_set_width; no pipelined probe); precision
 * RRG_FP32_RECHECK; no parametric uncertainty (otherwise RRG_ENOTIMPL).  Each
 * instance's result equals rrg_step's for the same inputs and scenarios. */
#define RRG_BATCH_MAX_INSTANCES 1024
#define RRG_BATCH_VARIANTS 10  /* rollout variants: lanes per tile {64, 128,
                                  256} x disturbance prefetch depth {8, 16},
                                  then warp tiles (32 lanes, each warp takes its
                                  own) x {8, 16}, then warp tiles of two
                                  candidates per thread (prefetch 8), then warp
                                  tiles of 16 scenarios at two lanes per
                                  trajectory (prefetch 8; tile_lanes reports
                                  16) */
typedef struct rrg_batch_ctx *rrg_batch_handle;

/* cfg as for rrg_create (n_scenarios and horizon are ignored); n_scenarios
 * and horizons: host arrays of n_instances values >= 1; sum over instances of
 * max_candidates * N_s must be below 2^31.  Allocates 12 sum(H_s N_s) bytes of
 * scenarios plus O(sum M N_s) bytes of recheck list. */
RRG_API int rrg_batch_create(const double *model_params, int n_params, const rrg_config *cfg,
                     int n_instances, const int32_t *n_scenarios, const int32_t *horizons,
                     void *cuda_stream, rrg_batch_handle *out);
RRG_API int rrg_batch_destroy(rrg_batch_handle h);
RRG_API const char *rrg_batch_last_error(rrg_batch_handle h);

/* One update of every instance from device inputs: d_x[3 S] (instance s at
 * 3 s), d_r[S], d_v_prev[S]; draws the scenarios of update_index, searches,
 * and writes d_v_t[S], d_kappa[S], d_flags[S] (each may be NULL; flags as
 * rrg_step).  An instance with non-finite or non-positive inputs holds
 * (kappa 0, flag bit 1).  Asynchronous on the handle's stream. */
RRG_API int rrg_batch_step_dev(rrg_batch_handle h, const double *d_x, const double *d_r,
                       const double *d_v_prev, uint64_t seed, uint64_t update_index,
                       double *d_v_t, double *d_kappa, int32_t *d_flags);

/* T closed-loop updates of every instance on the device (as
 * rrg_closed_loop_dev per instance): d_x0[3 S], d_v0[S] start the loop (NULL
 * d_x0: continue the previous call's loop), d_r_seq[t S + s] (t counted from
 * the loop start), plant_amp host[3]; outputs at [t S + s] (d_x_out at
 * [((t + 1) S + s) 3], the start at t = 0), each may be NULL.  use_graph: one
 * update is captured once and replayed (the graph is kept while pointers,
 * seed, t0 and the rollout variant stay the same).  Asynchronous. */
RRG_API int rrg_batch_closed_loop_dev(rrg_batch_handle h, const double *d_x0, const double *d_v0,
                              const double *d_r_seq, int T, uint64_t seed, uint64_t t0,
                              const double *plant_amp, int use_graph, double *d_v_out,
                              double *d_kappa_out, int32_t *d_flags_out, double *d_x_out);

/* Autotuner: runs 1 + repeats updates on the given inputs with each rollout
 * variant, times the rollout launches (CUDA events), keeps the fastest and
 * returns it in *variant_out; ms_out (optional, RRG_BATCH_VARIANTS doubles)
 * receives each variant's mean rollout time per update.  Results do not
 * depend on the variant.  Synchronous. */
RRG_API int rrg_batch_autotune(rrg_batch_handle h, const double *d_x, const double *d_r,
                       const double *d_v_prev, uint64_t seed, uint64_t update_index, int repeats,
                       int *variant_out, double *ms_out);
RRG_API int rrg_batch_set_variant(rrg_batch_handle h, int variant);
RRG_API int rrg_batch_get_variant(rrg_batch_handle h, int *variant, int *tile_lanes, int *prefetch);
/* Width of RRG_SEARCH_SPEC_BISECT batches: the tree nodes each instance
 * evaluates per round, 1..max_candidates (default max_candidates).  Every
 * instance's result is Alg. 1's for every width (the same tree and walk as
 * rrg_bisect_plan / rrg_bisect_decide); the width sets the number of rounds
 * (1 + ceil((n_bisect - d0) / d1) for trees of d0 levels from the kappa = 1
 * root and d1 below it) against the work per round.  RRG_EINVAL for the grid
 * searches, whose candidate count is their grid size.  set_width waits for
 * the handle's stream; the cached closed-loop graph is rebuilt on its next
 * use. */
#define RRG_BATCH_MAX_WIDTHS 24
RRG_API int rrg_batch_set_width(rrg_batch_handle h, int width);
RRG_API int rrg_batch_get_width(rrg_batch_handle h, int *width);
/* Autotuner of the width: times 1 + repeats whole updates (CUDA events on the
 * handle's stream around sample and search) on the given inputs for each tree
 * size 1, 2, 3, 4, 7, 8, 15, 16, ... up to max_candidates (at most
 * RRG_BATCH_MAX_WIDTHS of them), keeps the fastest and returns it in
 * *width_out; widths[] / ms_out[] (each may be NULL, room for
 * RRG_BATCH_MAX_WIDTHS) receive the widths tried and their mean ms per
 * update, *n_out how many.  Results do not depend on the width.  Synchronous. */
RRG_API int rrg_batch_autotune_width(rrg_batch_handle h, const double *d_x, const double *d_r,
                             const double *d_v_prev, uint64_t seed, uint64_t update_index, int repeats,
                             int *width_out, int32_t *widths, double *ms_out, int *n_out);
RRG_API int rrg_batch_set_profiling(rrg_batch_handle h, int on);
RRG_API int rrg_batch_get_stats(rrg_batch_handle h, rrg_stats *out);
RRG_API int rrg_batch_reset_stats(rrg_batch_handle h);

#ifdef __cplusplus
}
#endif

#endif /* RRG_H */
