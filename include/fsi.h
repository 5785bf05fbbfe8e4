/*
 * fsi.h -- C ABI of libfsi, the B300 (sm_103a) hot path of the fourth-order forward
 * symplectic integrator (FSI) with hierarchical Hamiltonian splitting (HHS) of
 * BIFROST (Rantala et al. 2022, arXiv 2210.02472).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - All array arguments are DEVICE pointers owned by the caller, unless a comment
 *    says "host".  Floating point is IEEE double.  Positions, velocities and
 *    accelerations are structure-of-arrays "3 x N": the x components of all N
 *    particles, then all y, then all z, each row contiguous.
 *  - Index lists are int32 global particle ids in [0, N).  A NULL list means all N
 *    particles in order (the fast path: no gather).  Per-set outputs are 3 x n
 *    (row stride n) in the order of the list.
 *  - `stream` is a cudaStream_t passed as void*; NULL is the legacy default stream.
 *    Every call only enqueues work on `stream` and returns; results are ready when
 *    the stream is.  Calls never synchronise the device, except fsi_sync_status, the
 *    calls documented as "synchronous", and workspace growth (see fsi_reserve).
 *  - The library never allocates per call except to grow the context's workspace;
 *    call fsi_reserve first to keep a call sequence free of allocations (required
 *    under CUDA graph capture).
 *  - Return value: FSI_OK (0) or a negative FSI_ERR_* code for errors detected on the
 *    host (bad arguments, CUDA launch errors).  Errors detected on the device
 *    (coincident particles, a non-finite result, a timed-out wait) are latched in a
 *    per-context device word (the first error wins) and reported by fsi_sync_status.
 *    A pass whose result is non-finite scans its sources once for a partner at
 *    exactly the same position and latches FSI_ERR_COINCIDENT if it finds one,
 *    FSI_ERR_NONFINITE otherwise.  fsi_last_error() returns a thread-local text
 *    message for the last host-side error.
 *  - Self-interaction is excluded by global particle id, never by position.
 *  - G = 1 (N-body units).
 *
 * Precision (fsi_params.precision)
 * --------------------------------
 *  FSI_FP64:  every pair term in FP64; agrees with an FP64 direct sum to ~1e-13
 *             relative (summation order differs).
 *  FSI_MIXED: positions are split into FP32 hi + lo parts so that each pair
 *             difference is accurate to FP32 precision relative to the separation;
 *             the pair arithmetic (r^-3, gradient terms) is FP32 with one residual
 *             correction of the hardware rsqrt; a receiver's FP32 partial sums run over
 *             at most 32 sources and are accumulated as float-float pairs (TwoSum).
 *             Sets of >= 196608 particles take the pairs inside each i-block (each
 *             particle's nearest neighbours in Morton order) in float-float arithmetic
 *             in their acceleration passes.  Relative acceleration error |da_i| / |a_i|
 *             at N = 2^20: median 2e-8, 99.9th percentile 1e-7 (larger where the pair
 *             terms cancel, |a_i| << sum_j m_j / r_ij^2).  Valid for separations > ~1e-7
 *             (FP32 range of r^-5).
 */
#ifndef LIBFSI_FSI_H
#define LIBFSI_FSI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define FSI_OK 0
#define FSI_ERR_ARG (-1)          /* invalid argument (sizes, NULL, overlapping sets) */
#define FSI_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define FSI_ERR_NONFINITE (-3)    /* a result was inf/NaN for a reason other than
                                     coincident particles (FP32 overflow of r^-3 in the
                                     mixed path at separations below ~1e-13, a non-finite
                                     input) */
#define FSI_ERR_COINCIDENT (-4)   /* two distinct particles at exactly the same position
                                     with eps2 = 0, where the pair terms of Sect. 2.1 are
                                     undefined (and, for the time steps of Sect. 3.4 and
                                     the PN1.0 kick, which are unsoftened, at any eps2);
                                     latched by the acceleration, gradient, time-step,
                                     energy and PN passes */
#define FSI_ERR_TIMEOUT (-5)      /* a bounded device wait ran out */
#define FSI_ERR_MAXLEVEL (-6)     /* HHS: a particle wanted a level deeper than max_level */
#define FSI_ERR_UNSUPPORTED (-7)
#define FSI_ERR_NOMEM (-8)        /* workspace allocation failed */

#define FSI_FP64 0
#define FSI_MIXED 1

/* ---- context ----------------------------------------------------------------- */
typedef struct fsi_ctx fsi_ctx;

typedef struct fsi_params {
    int precision;        /* FSI_FP64 or FSI_MIXED */
    double eps2;          /* Plummer softening squared (0 = none), used by step/HHS */
    double eta_ff;        /* free-fall time-step parameter (Sect. 3.4), e.g. 0.2 */
    double eta_fb;        /* fly-by time-step parameter, e.g. 0.2 */
    double eta_jerk;      /* jerk time-step parameter, e.g. 0.1 */
    int max_level;        /* deepest HHS level (pivot tau / 2^max_level), e.g. 40 */
    double c;             /* speed of light in N-body units; 0 switches PN1.0 off */
    int split;            /* source-split factor override (0 = automatic) */
    long long timeout_ns; /* budget of every bounded device wait (0 = 2e9 ns) */
    int symmetric;        /* 1 (default): a set's self-interaction (pair sums and time
                             steps), and the two directions of a large cross-level pass,
                             evaluate every unordered pair once and add it to both
                             particles (Newton's third law); 0: every ordered pair is
                             evaluated by its receiving particle */
    int hhs_small_max;    /* HHS: a fast set of at most this many particles (0 = 256; the
                             maximum is 512) runs its whole recursion inside one CTA; -1 =
                             always walk the levels from the host */
    int order_min;        /* mixed + symmetric with a far-tile kernel variant selected (see
                             fsi_autotune): fsi_step puts a set of at least this many
                             particles in Morton order for the duration of the call (0 =
                             32768; -1 = never); fsi_hhs_interval (mixed + symmetric) puts
                             the level-0 list of N >= order_min in Morton order, and its
                             bipartite cross-level passes whose smaller set has at least
                             min(16384, order_min) particles take the far-tile arithmetic for
                             that set's sub-tiles.  The order only changes which pairs take
                             the far-tile arithmetic and the summation order. */
    double eta_grad;      /* gradient time-step parameter eta_nabla (Sect. 3.4, Eqs. dt-nabla1
                             and dt-nabla2): eps = eta (|v_i| / |g'_i|)^{1/3} and
                             eps = eta (|a_i| / |g'_i|)^{1/2}, g'_i = G_i / 24 from the
                             set's own accelerations (one extra acc + grad pass per
                             time-step assignment); 0 (default) = off */
    double eta_va;        /* velocity-per-acceleration time-step parameter (Sect. 3.4, Eq.
                             vel-acc-crit): eps = eta |v_i| / |a_i|; 0 (default) = off */
    int wide_ctas;        /* a pair pass (acc or grad, unmasked) whose tiled form would run
                             fewer CTAs than this takes the wide form instead: up to 32
                             lanes per receiver splitting its sources (0 = 32; -1 =
                             never).  Only the summation order differs. */
    int hhs_grid_max;     /* HHS: a fast set of more than hhs_small_max and at
                             most this many particles (0 = 4096; -1 = never) runs its whole
                             recursion in one cooperative launch over the GPU, and an
                             interval of N <= hhs_grid_max particles is that one launch
                             (no host synchronisation, so it can be captured in a CUDA
                             graph; see fsi_hhs_interval).  Only summation orders differ
                             from the host walk.  Raising it to N makes any interval
                             capturable; its large levels then run the launch's
                             one-sided passes (an N = 65536 interval: ~2x the time). */
    int hhs_grid_ctas;    /* CTAs of that cooperative launch (0 = one per SM, the most that
                             are co-resident; otherwise clamped to [2, that maximum]). */
} fsi_params;

/* Fill *p with the defaults (FP64, eps2 0, eta 0.2/0.2/0.1, max_level 40, PN off,
 * symmetric self-interaction). */
void fsi_default_params(fsi_params *p);

/* Create a context on the current CUDA device.  *ctx receives the handle.
 * The context owns a device workspace (grown on demand) and a device error word. */
int fsi_create(fsi_ctx **ctx, const fsi_params *p);

/* Free the workspace and the handle.  Synchronises the device first. */
int fsi_destroy(fsi_ctx *ctx);

/* Change precision / parameters of an existing context (host only, no sync). */
int fsi_set_params(fsi_ctx *ctx, const fsi_params *p);

/* Grow the workspace so that calls on sets of up to n particles (out of N total)
 * allocate nothing; with n == N also an HHS interval of the N particles (so that an
 * interval captured in a CUDA graph right after it allocates nothing).  Synchronous. */
int fsi_reserve(fsi_ctx *ctx, int N, int n);

/* Thread-local text of the last host-side error (never NULL). */
const char *fsi_last_error(void);

/* Synchronise `stream`, then return and clear the latched device error word
 * (FSI_OK if none).  Synchronous. */
int fsi_sync_status(fsi_ctx *ctx, void *stream);

/* ---- pair sums ------------------------------------------------------------------- */

/* Newtonian acceleration, Sect. 2.1 Eq. (new-newton-acc), of the active set A from the
 * source set B:  acc_out[:, k] = sum_{j in B, j != A[k]} m_j (r_j - r_i) /
 *                                  (|r_j - r_i|^2 + eps2)^{3/2},  i = A[k].
 * pos: 3 x N, mass: N, A: nA ids (NULL = all), B: nB ids (NULL = all),
 * acc_out: 3 x nA (row stride nA).  A and B may overlap arbitrarily.  When A points into
 * B's memory (A = B + k with k + nA <= nB, a rank's slice of a sharded pass), the self
 * pairs are found by the index offset k and only the tiles around them are checked. */
int fsi_accel(fsi_ctx *ctx, int N, const double *pos, const double *mass,
              const int *A, int nA, const int *B, int nB, double eps2,
              double *acc_out, void *stream);

/* Gradient sum of the FSI gradient kick, Sect. 2.1 Eq. (new-grad-acc):
 *   grad_out[:, k] = sum_{j in B, j != i} m_j / r^5 ( r^2 a_ji - 3 (a_ji . r_ji) r_ji ),
 *   r_ji = r_j - r_i, r^2 = |r_ji|^2 + eps2, a_ji = a_j - a_i, i = A[k],
 * WITHOUT the factor eps^2/24 (the gradient acceleration is a + (eps^2/24) grad).
 * accg: 3 x N accelerations indexed by global id (only the entries of A and B are
 * read).  A and B may overlap arbitrarily (A a slice of B's memory: as in fsi_accel). */
int fsi_grad(fsi_ctx *ctx, int N, const double *pos, const double *mass,
             const double *accg, const int *A, int nA, const int *B, int nB,
             double eps2, double *grad_out, void *stream);

/* Share `part` (0 <= part < nparts) of the same-set pass acc(A <- A) (Sect. 2.1, Eq.
 * new-newton-acc) or G(A <- A) (Eq. new-grad-acc, accg as for fsi_grad): the pair sums
 * of a subset of the set's unordered pairs, for all nA receivers (out: 3 x nA, device,
 * in the order of A; overwritten).  The nparts shares add up to fsi_accel / fsi_grad of
 * the set (up to the order of the additions): one rank's part of a pass split over ranks
 * by pairs, each pair evaluated once on one rank for both of its particles (Newton's
 * third law), then summed over the ranks.  With fsi_params.symmetric = 1 and a set large
 * enough for the tiled symmetric kernel (not the wide form of small passes), share k is a
 * contiguous range of the kernel's blocks of receivers with about 1/nparts of its work;
 * otherwise share 0 is the whole pass and the other shares are zero.  All shares of a pass
 * must come from contexts with the same fsi_params and tuning on the same set and inputs
 * (the split depends on the kernel variant and on the set's spatial order).  FSI_ERR_ARG
 * for a bad share.  Asynchronous. */
int fsi_accel_part(fsi_ctx *ctx, int N, const double *pos, const double *mass, const int *A,
                   int nA, int part, int nparts, double eps2, double *acc_out, void *stream);
int fsi_grad_part(fsi_ctx *ctx, int N, const double *pos, const double *mass,
                  const double *accg, const int *A, int nA, int part, int nparts, double eps2,
                  double *grad_out, void *stream);

/* acc(A <- B) and the gradient sum G(A <- B) of one splitting term:
 *  - A and B the same list (same pointer, or both NULL): the set's self-interaction
 *    (Sect. 2.1); the a_j inside G are acc(A <- A).
 *  - A and B disjoint: the slow-fast inter-level term (Sect. 2.2); a_i = acc(A <- B),
 *    a_j = acc(B <- A).
 * Partial overlap is an error (latched on the device as FSI_ERR_ARG).
 * vel may be NULL.  acc_out, grad_out: 3 x nA. */
int fsi_accel_grad(fsi_ctx *ctx, int N, const double *pos, const double *vel,
                   const double *mass, const int *A, int nA, const int *B, int nB,
                   double eps2, double *acc_out, double *grad_out, void *stream);

/* PN1.0 pair acceleration (Sect. 3.9): for i = A[k], the sum over j in B, j != i, of
 * the two-body 1PN Einstein-Infeld-Hoffmann acceleration of i due to j, restricted to
 * pairs with at least one black hole (is_bh: N bytes, nonzero = black hole).
 * With n = (x_i - x_j)/r:
 *   a_i = m_j/(c^2 r^2) { n [ -v_i^2 - 2 v_j^2 + 4 v_i.v_j + 3/2 (n.v_j)^2
 *                              + 5 m_i/r + 4 m_j/r ] + (v_i - v_j) [4 n.v_i - 3 n.v_j] }.
 * out: 3 x nA.  Unsoftened.  Evaluated through black-hole sublists of A and B (cost
 * O((nA + nB) x black holes)); more than 1024 black holes in a list latch
 * FSI_ERR_UNSUPPORTED. */
int fsi_pn_accel(fsi_ctx *ctx, int N, const double *pos, const double *vel,
                 const double *mass, const unsigned char *is_bh, double c,
                 const int *A, int nA, const int *B, int nB, double *out, void *stream);

/* ---- integrator steps -------------------------------------------------------------- */

/* nsteps FSI cycles of step h (Sect. 2.1, Eq. fsi-cycle) of the set idx (n ids, NULL =
 * all N) interacting with itself only, in place on pos/vel (3 x N):
 *   kick h/6 (a), drift h/2, kick 2h/3 (a + h^2/24 G), drift h/2, kick h/6 (a).
 * Consecutive cycles share the acceleration between the closing and the next opening
 * kick (three pair passes per cycle).  With fsi_params.c > 0, PN1.0 half-kicks of h/2
 * wrap every cycle (Sect. 3.9) for pairs with a black hole (is_bh, N bytes; may be
 * NULL when c == 0).  eps2 comes from fsi_params. */
int fsi_step(fsi_ctx *ctx, int N, double *pos, double *vel, const double *mass,
             const unsigned char *is_bh, const int *idx, int n, double h, int nsteps,
             void *stream);

/* Kick then drift of the set idx with given accelerations (the kinetic and potential
 * factors of Sect. 2.1, Eq. fsi-cycle, applied on their own): for k < n, i = idx[k]
 * (idx NULL: i = k and n <= N),
 *   vel[:, i] += c_kick * acc[:, k],   then   pos[:, i] += c_drift * vel[:, i],
 * every operation an FP64 FMA.  pos, vel: 3 x N device arrays, updated in place; acc:
 * 3 x n compact device rows (NULL: drift only); idx: n device ids in [0, N) without
 * repeats (not checked: a repeated id races).  HBM-bound: 120 B per particle moved
 * (124 B with idx).  Asynchronous on `stream`; FSI_ERR_ARG for a NULL state array or a
 * bad n. */
int fsi_kick_drift(fsi_ctx *ctx, int N, double *pos, double *vel, const double *acc,
                   const int *idx, int n, double c_kick, double c_drift, void *stream);

/* One FSI cycle (PN off) of the set idx exactly as fsi_step with nsteps = 1 (the set kept
 * in its own order), also writing the cycle's intermediates for fsi_step_vjp_rec: a0 =
 * a(x0), a1 = a(x1) and g1 = G(x1) (Sect. 2.1, Eq. fsi-cycle; x1 = the positions after the
 * first drift), each 3 x n compact device rows in the order of idx.  FSI_ERR_UNSUPPORTED
 * when fsi_params.c > 0. */
int fsi_step_record(fsi_ctx *ctx, int N, double *pos, double *vel, const double *mass,
                    const int *idx, int n, double h, double *a0, double *a1, double *g1,
                    void *stream);

/* Adjoint of one fsi_step cycle (PN off): given the input state (pos0, vel0; 3 x N) of
 * a cycle of step h on the set idx (n ids, NULL = all) and the cotangents gx_out, gv_out
 * (3 x N) of its output state, writes the cotangents of the input state into gx_in,
 * gv_in (3 x N; entries outside the set are copied from gx_out / gv_out) and ADDS the
 * mass cotangent into gm (N) so that multi-step products can accumulate.  The cycle's
 * intermediates are recomputed (context precision); the adjoint pair sums run in FP64:
 *   VJP of a with cotangent u:   rbar_k = sum_j T(d)(m_k u_j - m_j u_k),
 *                                mbar_k = -sum_j (u_j . d)/s^3,
 *   VJP of G (a fixed), cotangent w: rbar_k = sum_j Q(d, a_j - a_k)(m_k w_j - m_j w_k),
 *                                mbar_k = -sum_j w_j . T(d)(a_j - a_k),
 * with d = r_j - r_k, s^2 = |d|^2 + eps2, T(d) = I/s^3 - 3 d d^T/s^5 and
 * Q(d, b) = d(T(d) b)/dd, chained backwards through kick h/6, drift h/2, gradient kick
 * 2h/3 (Sect. 2.1, Eq. fsi-cycle), drift h/2, kick h/6.  gx_in may alias gx_out and
 * gv_in may alias gv_out.  Returns FSI_ERR_UNSUPPORTED when fsi_params.c > 0. */
int fsi_step_vjp(fsi_ctx *ctx, int N, const double *pos0, const double *vel0,
                 const double *mass, const int *idx, int n, double h,
                 const double *gx_out, const double *gv_out, double *gx_in, double *gv_in,
                 double *gm, void *stream);

/* fsi_step_vjp given the cycle's intermediates a0, a1, g1 as written by fsi_step_record
 * for the same input state, instead of recomputing them (three pair passes fewer). */
int fsi_step_vjp_rec(fsi_ctx *ctx, int N, const double *pos0, const double *vel0,
                     const double *mass, const int *idx, int n, double h, const double *a0,
                     const double *a1, const double *g1, const double *gx_out,
                     const double *gv_out, double *gx_in, double *gv_in, double *gm,
                     void *stream);

/* nsteps FSI cycles of the set idx (NULL = all N, then n == N) with binary subsystems
 * (Sect. 2.3, Algorithm 1), in place: kick eps/6, subsystems eps/2, drift of the single
 * particles eps/2, gradient kick 2 eps/3 (a + eps^2/24 G), subsystems eps/2, drift eps/2,
 * kick eps/6, where every acceleration and gradient sum ignores the pair inside a
 * subsystem.  pairs: device int array of 2 x n_pairs global ids, binary s =
 * (pairs[2s], pairs[2s+1]); both members must be in the set and in no other binary
 * (else FSI_ERR_ARG is latched on the device).  A binary's subsystem flow is its exact
 * two-body motion over eps/2 (Kepler's equation, FP64); an unbound pair latches
 * FSI_ERR_UNSUPPORTED (regularised and secular subsystem integrators are not part of
 * this library).  Newtonian only: FSI_ERR_UNSUPPORTED when fsi_params.c > 0.  Masked
 * passes take the one-sided pair kernel in the context's precision. */
int fsi_step_sub(fsi_ctx *ctx, int N, double *pos, double *vel, const double *mass,
                 const int *idx, int n, const int *pairs, int n_pairs, double h, int nsteps,
                 void *stream);

/* Time steps of the set P against itself (Sect. 3.4): min of the free-fall
 * eta_ff min_j (r^3/(m_i+m_j))^{1/2}, fly-by eta_fb min_j r/|v_ij| and jerk
 * eta_jerk |a_i|/|j_i| criteria (eta's and eps2 from fsi_params), and, when
 * fsi_params.eta_grad / eta_va are > 0, the gradient criteria (Eqs. dt-nabla1, dt-nabla2)
 * and the velocity-per-acceleration criterion (Eq. vel-acc-crit) from the set's own
 * accelerations and force-gradient sums (one extra acc + grad pass).  step_out: n.
 * FSI_FP64: FP64 throughout; with fsi_params.symmetric = 1 and n >= 2048 every unordered
 * pair is evaluated once (the a and j sums of the jerk criterion then add in another
 * order, the free-fall and fly-by minima are the same).  FSI_MIXED: FP32 pair arithmetic
 * (hi/lo separations, minima of squared ratios), ~1e-6 relative. */
int fsi_timesteps(fsi_ctx *ctx, int N, const double *pos, const double *vel,
                  const double *mass, const int *P, int n, double *step_out, void *stream);

/* Time steps of the entries P[lo, hi) of the set against the whole set P (Sect. 3.4: the
 * free-fall, fly-by and jerk criteria of fsi_timesteps; one receiver slice of an i-sharded
 * time-step pass).  step_out: hi - lo, device, in the order of P[lo, hi).  Asynchronous.
 * FSI_ERR_ARG for a bad range; FSI_ERR_UNSUPPORTED when eta_grad or eta_va > 0 (those
 * criteria need the whole set's own accelerations). */
int fsi_timesteps_sub(fsi_ctx *ctx, int N, const double *pos, const double *vel,
                      const double *mass, const int *P, int n, int lo, int hi, double *step_out,
                      void *stream);

/* Kinetic and potential energy of the set P (Sect. 2.1 Hamiltonian), FP64:
 * out[0] = sum 1/2 m v^2, out[1] = -sum_{i<j} m_i m_j / (r^2 + eps2)^{1/2}.
 * out: 2 doubles, device. */
int fsi_energy(fsi_ctx *ctx, int N, const double *pos, const double *vel,
               const double *mass, const int *P, int n, double *out, void *stream);

/* One HHS interval of length tau over all N particles (Sect. 2.2, Eq. hhsfsi-cycle):
 * per level, time steps against the level set (level 0 against all N; deeper levels
 * take min with the level-0 step), the split S = {eps >= tau}, F = {eps < tau}, then
 * U_SF(tau/6) FSI(S, tau/2) HHS(F, tau/2) U~_SF(2 tau/3) HHS(F, tau/2) FSI(S, tau/2)
 * U_SF(tau/6).  In place on pos/vel.
 * How the levels run: the host walks the large levels (one device->host read of the
 * split counts per level visit, so the call is synchronous); a fast set of
 * more than hhs_small_max and at most hhs_grid_max particles runs its whole recursion in
 * one cooperative launch over the GPU, and a fast set of at most hhs_small_max in one CTA.
 * When N <= hhs_grid_max the whole interval is that one launch: the call then
 * does not synchronise with the host and may be captured in a CUDA graph (stream
 * capture; reserve the workspace first with fsi_reserve(ctx, N, N) or one uncaptured
 * interval); a replay repeats the interval bit for bit on the captured buffers.  Under
 * capture the level statistics stay on the device (fsi_level_stats reads those of the
 * last replay) and a depth-cap hit is latched as FSI_ERR_MAXLEVEL in the error word
 * (fsi_sync_status) instead of being returned.  An interval that needs the host walk
 * returns FSI_ERR_UNSUPPORTED when its stream is capturing.  PN (c > 0): at most 1024
 * black holes per level set (FSI_ERR_UNSUPPORTED latched otherwise).  Device waits are
 * bounded by fsi_params.timeout_ns (FSI_ERR_TIMEOUT latched on expiry). */
int fsi_hhs_interval(fsi_ctx *ctx, int N, double *pos, double *vel, const double *mass,
                     const unsigned char *is_bh, double tau, void *stream);

/* One HHS interval with adaptive energy-error restarts (Sect. 3.12): the state is saved
 * (device copies in the context workspace) and E = T + W (fsi_energy) taken; after the
 * interval, if |Delta E / E| > eta_restart, the saved state is restored and the interval
 * re-run with eta_ff, eta_fb, eta_jerk, eta_grad and eta_va all lowered by 50 % per
 * consecutive restart.  An attempt is accepted when its error is within eta_restart, when
 * it is larger than the previous attempt's (the current result is kept), or after
 * max_restarts restarts; the context's parameters are unchanged afterwards.  *restarts
 * (host, may be NULL) receives the number of restarts, *rel_err (host, may be NULL) the
 * accepted attempt's |Delta E / E|; fsi_level_stats reports the accepted attempt's
 * levels.  Synchronous.  Returns like fsi_hhs_interval; FSI_ERR_ARG for eta_restart < 0
 * or max_restarts < 0. */
int fsi_hhs_interval_restart(fsi_ctx *ctx, int N, double *pos, double *vel,
                             const double *mass, const unsigned char *is_bh, double tau,
                             double eta_restart, int max_restarts, int *restarts,
                             double *rel_err, void *stream);

/* ---- batched ensembles ---------------------------------------------------------- */
typedef struct fsi_batch fsi_batch;

/* Plan the FSI cycles of K independent clusters whose particles are concatenated in one
 * SoA set: cluster k is [offsets[k], offsets[k+1]) (offsets: host array of K+1 values,
 * offsets[0] = 0, non-decreasing).  The plan holds the work-item tables (clusters by
 * decreasing size) and the records of the concatenated set, sized for up to max_steps
 * cycles per fsi_batch_step (0 = 16).  Synchronous; allocates. */
int fsi_batch_create(fsi_ctx *ctx, int K, const long long *offsets, int max_steps,
                     fsi_batch **batch);
int fsi_batch_destroy(fsi_batch *batch);

/* nsteps FSI cycles of step h (Sect. 2.1, Eq. fsi-cycle) of every cluster on itself, in
 * place on pos/vel (3 x Ntot, Ntot = offsets[K]), mass (Ntot), in ONE persistent kernel
 * launch: work items (phase, cluster, block of active particles) are handed out by an
 * atomic counter and each waits (bounded, fsi_params.timeout_ns) for its cluster's
 * previous phase.  Consecutive cycles share the closing/opening acceleration pass.
 * Asynchronous, allocation-free and capturable in a CUDA graph.  Newtonian only
 * (FSI_ERR_UNSUPPORTED when fsi_params.c > 0); eps2 from fsi_params. */
int fsi_batch_step(fsi_ctx *ctx, fsi_batch *batch, double *pos, double *vel,
                   const double *mass, double h, int nsteps, void *stream);

/* Tuning of the batched kernel: active particles per thread -- 1 or 2 (one-sided form,
 * every ordered pair by its receiver), 4, 6 or 8 (symmetric form, every unordered pair
 * once, mixed precision only; blocks of 1024 / 1536 / 2048 particles, 2 / 2 / 1 resident
 * CTAs per SM) -- and resident CTAs per SM (0 = occupancy maximum). */
int fsi_batch_set_tuning(fsi_ctx *ctx, fsi_batch *batch, int ipt, int ctas_per_sm);
int fsi_batch_get_tuning(fsi_batch *batch, int *ipt, int *ctas_per_sm);

/* Idle accounting of the batch's persistent launches since the last reset (load balance
 * across clusters of uneven size): *wait_ns = time the CTAs spent waiting for other CTAs'
 * phases, *life_ns = summed CTA lifetimes (start to leaving the work loop), *ctas = CTAs
 * of the last launch.  With the launches' summed elapsed time T, the idle fraction is
 * 1 - (life_ns - wait_ns) / (ctas T): waits inside CTAs plus CTAs out of work before the
 * launch ends.  Synchronises the device; reset != 0 zeroes the counters after reading. */
int fsi_batch_stats(fsi_batch *batch, long long *wait_ns, long long *life_ns, int *ctas,
                    int reset);

/* Instrumentation of the ensemble launch (Sect. 2.1 FSI cycles of every cluster): busy
 * time of the symmetric persistent launches' work items by kind since the last reset: ns[0] / items[0] the sum items of a block with itself (its own pairs), [1] the
 * sum items of two blocks, [2] pack and apply items (thread 0 of the CTA, from the end of
 * the item's phase wait to its completion signal).  ns, items: host long long[3].
 * Synchronises the device; reset != 0 zeroes these counters after reading. */
int fsi_batch_item_stats(fsi_batch *batch, long long *ns, long long *items, int reset);

/* Test hook: during the next fsi_batch_step the items of `cluster` wait for a phase
 * count that is never reached, so their bounded waits run out and the launch ends with
 * FSI_ERR_TIMEOUT latched (read by fsi_sync_status) instead of hanging.  The next step
 * after that runs normally.  That call synchronises the stream. */
int fsi_batch_inject_stall(fsi_batch *batch, int cluster);

/* Per-level slow-set sizes summed over the visits of the last fsi_hhs_interval (of its
 * last replay, when that interval was captured in a CUDA graph; the call then
 * synchronises the device).  counts: host array of `max` entries.  Returns the number of
 * levels used. */
int fsi_level_stats(fsi_ctx *ctx, long long *counts, int max);

/* ---- tuning ----------------------------------------------------------------------- */

/* Autotuner: times every built variant of the acceleration and gradient pair kernels
 * (context precision; the symmetric kernels when fsi_params.symmetric, else the
 * one-sided ones) on the first n particles of pos/mass as one self-interacting set,
 * `reps` timed launches each after one warm-up, and keeps the fastest in the context.
 * Symmetric variants are kept per set-size class (n < 32768, 32768 <= n < 196608,
 * n >= 196608: small sets are latency-bound and favour few particles per thread); each
 * class that n reaches is tuned on the first min(n, 8192), min(n, 65536) and n particles.
 * A variant is the number of active particles each thread holds in registers (low 4
 * bits, 1-6); one-sided mixed kernels add 16 to carry their per-tile partial sums as
 * float-float pairs instead of FP64; symmetric mixed kernels add 32 for the second form
 * (FP64 sums in shared memory, select-free source reduce-scatter) and 96 for the second
 * form with the far-tile path: for a warp of 32 I consecutive particles and a 32-record
 * source sub-tile of centre C and radius R whose gap is at least 4 R, the separation is
 * formed as (C - x_i) + (x_j - C) from FP32 values relative to C (3 additions instead of
 * 9; relative error of d at most about 3 u (1 + 1/3), u = 2^-24).  When n >= the order
 * threshold (fsi_params.order_min), the set is timed in Morton order, as fsi_step runs
 * it.  Synchronous.  (The source-split factor of one-sided passes is chosen per launch
 * from the wave count, or fixed by fsi_params.split.) */
int fsi_autotune(fsi_ctx *ctx, int N, const double *pos, const double *mass, int n, int reps,
                 void *stream);

/* Read / set the pair-kernel variants (acc, grad) of the context precision and mode
 * (symmetric or one-sided).  fsi_get_tuning reads the largest size class,
 * fsi_get_tuning_for the class of a set of n particles; fsi_set_tuning sets every class
 * and rejects variants the library was not built with (FSI_ERR_ARG). */
int fsi_get_tuning(fsi_ctx *ctx, int *ipt_acc, int *ipt_grad);
int fsi_get_tuning_for(fsi_ctx *ctx, int n, int *ipt_acc, int *ipt_grad);
int fsi_set_tuning(fsi_ctx *ctx, int ipt_acc, int ipt_grad);

/* ---- context-free, allocation-free variant ------------------------------------------- */

/* The paper has no counterpart: this entry point exists for callers that cannot allocate
 * device memory -- code under a host framework that owns every device allocation, or
 * code that must not allocate inside a region that will be captured into a CUDA graph.
 * It computes the same Newtonian accelerations as fsi_accel with an FP64 context for the
 * self-interaction of all N particles (A = B = all):
 *   acc_out[:, i] = sum_{j != i} m_j (r_j - r_i) / (|r_j - r_i|^2 + eps2)^{3/2},
 * pos: 3 x N, mass: N, acc_out: 3 x N, all device pointers owned by the caller.
 * It calls no allocating routine.  Its scratch (packed source records and split partial
 * sums) is a fixed array in the library's device image, 4 MiB on every GPU that loads the
 * library, held until the process exits.  Limit: N <= 32768; larger N returns FSI_ERR_ARG
 * with a message in fsi_last_error, and nothing is launched.  All calls share the array:
 * each call rewrites every scratch byte it reads (nothing needs clearing), and calls that
 * overlap on the GPU (unordered streams) race on it.  The first call on a device looks
 * the array's device address up (cudaGetSymbolAddress) and caches it; make that first
 * call before any stream capture.  Device-side errors are not latched anywhere (there is
 * no context and so no error word): a non-finite result (coincident particles with
 * eps2 = 0 included) stays in acc_out, and a bounded wait of the pair kernel that runs
 * out (a bulk copy that never lands) makes the affected CTA write quiet NaN into its
 * rows, so every device-side failure shows up as non-finite entries of acc_out: check
 * them.  Asynchronous on `stream`. */
int fsi_accel_noalloc(int N, const double *pos, const double *mass, double eps2,
                      double *acc_out, void *stream);

/* ---- instrumentation ------------------------------------------------------------ */

/* Start (enable = 1) or stop (0) recording a CUDA event pair around every pair-kernel
 * launch of this context, on the stream the kernel is launched on.  Recording costs two
 * event records per launch and no synchronisation. */
int fsi_profile(fsi_ctx *ctx, int enable);

/* Synchronise the recorded events and return, per kernel kind (0 = acceleration pass,
 * 1 = gradient pass, 2 = split-finalize), the number of launches and their summed device
 * milliseconds, then clear the record.  launches: host long long[3], ms: host double[3]. */
int fsi_profile_read(fsi_ctx *ctx, long long *launches, double *ms);

/* Phase profile of the HHS recursions (Sect. 2.2) run in one cooperative launch
 * (recorded while fsi_profile is on): per phase kind (0 time steps, 1 split (empty: every CTA splits on
 * its own without a barrier, and that time counts toward the next phase), 2 inter-level
 * kick (incl. the FSI passes that share one), 3 FSI pass of the slow set, 4 one-CTA
 * recursion of a small fast set, 5 gradient time-step criteria, 6 set-up, 7 PN1.0 kick
 * phases), the wall-clock nanoseconds from the end of the previous phase to the end of
 * this one as seen by CTA 0 (the work and the grid barrier after it), and the number of
 * phases.  ns, phases: host long long[8].  reset != 0 clears after reading.  Synchronises
 * `stream`. */
int fsi_grid_stats(fsi_ctx *ctx, long long *ns, long long *phases, int reset, void *stream);

/* Pair-sum work issued by this context: ordered (receiver, source) pairs of the
 * acceleration passes and of the gradient passes (a symmetric pass counts both
 * directions), since creation or the last reset (reset != 0 clears after reading). */
int fsi_work_stats(fsi_ctx *ctx, long long *acc_pairs, long long *grad_pairs, int reset);

/* Far-tile statistics of the symmetric mixed kernel (variants >= 96): (warp, 32-record
 * source sub-tile) visits that took the far-tile separation and that took the hi/lo
 * separation, since creation or the last reset (reset != 0 clears after reading).
 * Synchronises `stream`. */
int fsi_far_stats(fsi_ctx *ctx, long long *far_visits, long long *near_visits, int reset,
                  void *stream);

/* Number of kernels this library has launched in this process (all contexts). */
long long fsi_launch_count(void);

/* FP32 (fp64 = 0), FP64 (fp64 = 1) or packed FP32x2 (fp64 = 2, fma.rn.f32x2) fused
 * multiply-add throughput probe: launches `blocks` CTAs of 256 threads, each thread
 * running 8 independent FMA chains for `iters` iterations, writing one value per thread
 * to sink (device, blocks*256 entries of the probe's scalar type: float for 0 and 2).
 * *flops receives the nominal flop count (2 per FMA, 4 per packed FMA).  Time it with
 * CUDA events on `stream`.  The paper has no counterpart: it measures the pipe peaks
 * that the pair kernels' roofline fractions are quoted against. */
int fsi_fma_probe(int fp64, int blocks, int iters, void *sink, double *flops, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LIBFSI_FSI_H */
