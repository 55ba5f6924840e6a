/*
 * gqaoa.h - C ABI of the GB300 (sm_103a) Grover-QAOA statevector library.
 *
 * Method: Grover-mixer QAOA on random 3-SAT, arXiv:2402.02585
 * ("Grover-QAOA for 3-SAT: Quadratic Speedup, Fair-Sampling, and Parameter
 * Clustering", Zhang et al.). Section and equation numbers below refer to it.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Status: every function returns an int, GQAOA_OK (0) on success or a
 *    negative GQAOA_E* code. No C++ exception and no abort crosses the ABI.
 *    gqaoa_strerror() names a code.
 *  - Ownership: the caller allocates and owns every buffer. The library never
 *    allocates device memory; entry points that need scratch take a workspace
 *    pointer and its size, and a *_workspace_size() function reports the
 *    minimum. A workspace smaller than that is rejected with GQAOA_ENOMEM.
 *  - Memory spaces: each pointer argument says "host" or "device". Device
 *    pointers must be addresses in the current CUDA device's memory.
 *  - Streams: `stream` is a cudaStream_t (NULL = legacy default stream). All
 *    work is enqueued asynchronously on it; results written to device memory
 *    are valid once the stream reaches that point. No entry point
 *    synchronises, allocates or copies from the host after argument checks
 *    (except gqaoa_build_cost, which passes the clause masks by value in the
 *    kernel launch), so every call can be captured into a CUDA graph.
 *  - Errors found by argument checks are returned before anything is
 *    enqueued. A CUDA launch error is returned as GQAOA_ECUDA; the CUDA error
 *    itself can be read with cudaGetLastError().
 *  - Assignment index: z in [0, 2^n); bit j of z is Boolean variable x_j, and
 *    bit value 1 means "true" (Appendix B: tau(x) = 1 satisfies literal x).
 *  - Literals: DIMACS integers, +(v+1) for x_v and -(v+1) for NOT x_v.
 *  - Complex state: complex64, interleaved (float re, float im), 8 bytes per
 *    amplitude, index z. Alignment: 16 bytes.
 *  - Sizes: 1 <= n <= GQAOA_MAX_N, 0 <= m <= GQAOA_MAX_M, 1 <= p.
 *  - Per-device state: the library caches, per device ordinal, the SM count,
 *    the occupancy of its clustered passes and (gqaoa_evolve_noalloc) the
 *    device address of its static scratch. cudaDeviceReset destroys the
 *    context those belong to, so a process must not call the library on a
 *    device after resetting it.
 */
#ifndef GQAOA_H
#define GQAOA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define GQAOA_OK 0
#define GQAOA_EINVAL (-1)   /* null pointer, bad literal, misaligned buffer */
#define GQAOA_ERANGE (-2)   /* n, m, p or a count outside the supported range */
#define GQAOA_ECUDA (-3)    /* a CUDA runtime call or kernel launch failed */
#define GQAOA_ETIMEOUT (-4) /* reserved: the asynchronous calls report a bounded
                               device-side wait that gave up as NaN results */
#define GQAOA_ENOMEM (-5)   /* the caller's workspace is smaller than required */

#define GQAOA_MAX_N 34   /* 2^34 complex64 amplitudes = 128 GiB */
#define GQAOA_MAX_M 255  /* the cost C(z) is stored in one byte */

/* gqaoa_evolve flags */
#define GQAOA_STATE_IN 1u /* `state` holds the initial state psi_0 on entry */
/* out[0] becomes the probability of cost value c (0..255) instead of C = 0;
 * with c the lowest non-empty class it is the Max-SAT probability D of an
 * unsatisfiable instance (Fig. 1(b)). Not combined with a trace (EINVAL). */
#define GQAOA_READOUT_CLASS(c) (((unsigned)(c) & 0xFFu) << 8)

/* gqaoa_grad objectives */
#define GQAOA_OBJ_P0 0     /* P(C=0) = sum_{z: C(z)=0} |psi_p(z)|^2 */
#define GQAOA_OBJ_ENERGY 1 /* <H_P> = sum_z C(z) |psi_p(z)|^2 (Eq. 4) */
/* the probability of cost value c (0..255): sum_{z: C(z)=c} |psi_p(z)|^2;
 * GQAOA_OBJ_CLASS(0) is GQAOA_OBJ_P0 */
#define GQAOA_OBJ_CLASS(c) (256 + ((int)(c) & 0xFF))
/* OR-ed into the objective of gqaoa_grad / gqaoa_grad_batched: take the
 * streaming passes (one launch per round and direction; for n <= 11 the
 * one-CTA forward and adjoint kernels) also where the cluster-resident
 * adjoint would run (10 <= n <= 16); they agree to the rounding of their
 * sums. */
#define GQAOA_GRAD_STREAMING (1 << 16)

/* Human-readable name of a status code (static storage, never NULL). */
const char *gqaoa_strerror(int status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int gqaoa_version(void);

/*
 * Cost table and energy-manifold histogram (Section II.A, Eq. 1; Appendix B;
 * Appendix C's "counting the states in each distinct energy manifold").
 *
 *   C(z) = number of clauses that assignment z leaves unsatisfied
 *        = <z| H_P |z>,  H_P = sum_i H_C^(i)               (Eq. 1)
 *   h[c] = #{ z : C(z) = c },  c = 0..m
 *
 * lits  host   int32 [m][3]  DIMACS literals; each |lit| in 1..n.
 * n, m         1 <= n <= 34, 0 <= m <= 255.
 * cost  device uint8 [2^n]   written: C(z).
 * hist  device uint64 [m+1]  written: h[c]; may be NULL.
 * Errors: GQAOA_EINVAL (NULL lits/cost, literal 0 or |lit| > n),
 *         GQAOA_ERANGE (n, m out of range), GQAOA_ECUDA.
 * The result is exact (integer arithmetic).
 */
int gqaoa_build_cost(const int32_t *lits, int n, int m, uint8_t *cost, uint64_t *hist,
                     void *stream);

/*
 * Workspace bytes for gqaoa_evolve(n, p, ...). Writes *bytes.
 * Errors: GQAOA_EINVAL (bytes NULL), GQAOA_ERANGE.
 */
int gqaoa_evolve_workspace_size(int n, int p, size_t *bytes);

/*
 * G-QAOA evolution (Section II.B, Eqs. 2-3):
 *
 *   psi_p = e^{-i beta_p H_M} e^{-i gamma_p H_P} ... e^{-i beta_1 H_M} e^{-i gamma_1 H_P} psi_0
 *
 * with H_M = |+><+| (Eq. 2), so each round is the diagonal phase
 * chi(z) = e^{-i gamma_k C(z)} psi(z) followed by the rank-1 Grover mixer
 * psi = chi + (e^{-i beta_k} - 1) <+|chi> |+>, whose coefficient needs a
 * reduction over all 2^n amplitudes. psi_0 = |+> (uniform) unless
 * flags & GQAOA_STATE_IN. The single-angle-pair protocol (Eq. 5) is the case
 * gamma_k = gamma, beta_k = beta for all k.
 *
 * cost    device uint8 [2^n]     C(z) from gqaoa_build_cost; values <= m.
 * n, m                           sizes as for gqaoa_build_cost.
 * gammas  device double [p]      gamma_1..gamma_p (radians).
 * betas   device double [p]      beta_1..beta_p (radians).
 * p                              number of rounds, 1 <= p <= 2^20.
 * state   device complex64 [2^n] written: psi_p. Read first as psi_0 when
 *                                flags & GQAOA_STATE_IN. 16-byte aligned.
 * out     device double [3]      written: P(C=0) (or the probability of the
 *                                class named by GQAOA_READOUT_CLASS), <H_P>,
 *                                sum |psi_p|^2 of the final state; may be NULL.
 * trace   device double [p]      written: P(C=0) after each round; may be NULL.
 * ws, ws_bytes  device workspace, at least gqaoa_evolve_workspace_size(n, p).
 * flags                          0, GQAOA_STATE_IN, or-ed with
 *                                GQAOA_READOUT_CLASS(c) (then trace must be NULL).
 * Precision: complex64 state, phase factors e^{-i gamma c} evaluated in FP64
 * and rounded to FP32; the mixer sum <+|chi> and every readout are FP64.
 * Errors: GQAOA_EINVAL, GQAOA_ERANGE, GQAOA_ENOMEM, GQAOA_ECUDA.
 */
int gqaoa_evolve(const uint8_t *cost, int n, int m, const double *gammas, const double *betas,
                 int p, void *state, double *out, double *trace, void *ws, size_t ws_bytes,
                 unsigned flags, void *stream);

/* Workspace bytes for gqaoa_prob(n, ...). */
int gqaoa_prob_workspace_size(int n, size_t *bytes);

/*
 * Readout of a state (Eq. 4; Appendix B's solution probability):
 *   out[0] = P(C=0) = sum_{z: C(z)=0} |psi(z)|^2
 *   out[1] = <H_P>  = sum_z C(z) |psi(z)|^2
 *   out[2] = sum_z |psi(z)|^2
 * state device complex64 [2^n], cost device uint8 [2^n], out device double [3].
 * Sums are FP64.
 */
int gqaoa_prob(const void *state, const uint8_t *cost, int n, double *out, void *ws,
               size_t ws_bytes, void *stream);

/* Workspace bytes for gqaoa_sample(n, shots, ...). */
int gqaoa_sample_workspace_size(int n, int64_t shots, size_t *bytes);

/*
 * Fair sampling of measurement shots (Section IV, "sample all solutions";
 * Section II.B: the Grover mixer weights every solution equally):
 *   shot s = smallest z with CDF(z) > u_s * CDF(2^n - 1),
 *   CDF(z) = sum_{y <= z} |psi(y)|^2, each |psi(y)|^2 formed from the
 *            complex64 parts as a double-float pair (relative error below
 *            2^-46), sums of 16 consecutive weights and their prefixes within
 *            a tile of 4096 amplitudes in double-float (rounded to FP64), and
 *            prefixes of the tile totals in FP64 pairs rounded to FP64: every
 *            CDF value lies within a few FP64 rounding units of the total of
 *            the exact prefix sum,
 *   u_s    = uniform double in [0,1) from Philox4x32-10 (Salmon et al.,
 *            SC 2011) with counter (s mod 2^32, s >> 32, 0, 0) and key
 *            (seed mod 2^32, seed >> 32); the top 53 bits of the 64-bit word
 *            (out1 << 32 | out0) scaled by 2^-53.
 * state   device complex64 [2^n]; must have nonzero norm.
 * seed    the Philox key.
 * shots   0 <= shots < 2^32 (shot numbers and per-tile shot offsets are
 *         32-bit).
 * out_idx device uint64 [shots] written: z of each shot, in shot order.
 * ws      device workspace of gqaoa_sample_workspace_size(n, shots) bytes.
 */
int gqaoa_sample(const void *state, int n, uint64_t seed, int64_t shots, uint64_t *out_idx,
                 void *ws, size_t ws_bytes, void *stream);

/*
 * gqaoa_evolve followed by gqaoa_sample, as one call (Eqs. 2-3, then
 * Section IV's shots), for callers that want the readouts and the shots of
 * psi_p but not psi_p itself. The evolution's last mixer step adds the same
 * a_p (e^{-i beta_p} - 1) <+|chi_p> to every amplitude; instead of writing
 * psi_p = chi_p + a_p back (one more read and write of the whole state), the
 * readout pass and the sampler add a_p as they read chi_p, with the same
 * FP32 addition, so `out`, `trace` and the shots are those that gqaoa_evolve
 * followed by gqaoa_sample on the same workspace sizes returns.
 * Arguments as for gqaoa_evolve (one instance) and gqaoa_sample, except:
 * state   device complex64 [2^n]: the evolution's working state (psi_0 on
 *         entry if GQAOA_STATE_IN); on return it holds psi_p - a_p, not psi_p,
 *         whenever the fused path is taken (2^n >= 4096 and at most 64 shots per
 *         4096 amplitudes on average); otherwise psi_p.
 * ws      device workspace of gqaoa_evolve_sample_workspace_size(n, p, shots)
 *         bytes (16-byte aligned).
 * Errors: those of gqaoa_evolve and gqaoa_sample.
 */
int gqaoa_evolve_sample_workspace_size(int n, int p, int64_t shots, size_t *bytes);
int gqaoa_evolve_sample(const uint8_t *cost, int n, int m, const double *gammas,
                        const double *betas, int p, void *state, double *out, double *trace,
                        uint64_t seed, int64_t shots, uint64_t *out_idx, void *ws,
                        size_t ws_bytes, unsigned flags, void *stream);

/* Workspace bytes for gqaoa_grad(n, p, ...): the per-round checkpoints of the
 * state (p * 2^n * 8 bytes) plus reduction scratch. */
int gqaoa_grad_workspace_size(int n, int p, size_t *bytes);

/*
 * Objective and adjoint gradient with respect to every angle of Eq. 3
 * (Appendix C optimises the angles with a gradient method, L-BFGS-B):
 *   objective GQAOA_OBJ_P0:       L = P(C=0)
 *   objective GQAOA_OBJ_ENERGY:   L = <H_P>  (Eq. 4)
 *   objective GQAOA_OBJ_CLASS(c): L = probability of cost value c (the
 *                                 Max-SAT probability D for the lowest
 *                                 non-empty class; Fig. 1(b))
 * Forward: the rounds of gqaoa_evolve from |+>, storing each round's phased
 * state chi_k = e^{-i gamma_k C} psi_{k-1} in the workspace (checkpoints).
 * Backward, lambda_p = O psi_p and for k = p..1:
 *   dL/dbeta_k   = 2 Re[-i e^{-i beta_k} (S_k / 2^n) conj(sum_z lambda_k)], S_k = sum_z chi_k
 *   mu_k         = lambda_k + (e^{i beta_k} - 1) mean(lambda_k)
 *   dL/dgamma_k  = 2 Re[ sum_z conj(mu_k) (-i C) chi_k ]
 *   lambda_{k-1} = e^{+i gamma_k C} mu_k
 * cost device uint8 [2^n]; gammas, betas device double [p];
 * value  device double [1] written: L;
 * dgamma, dbeta device double [p] written.
 * Paths: for 10 <= n <= 16 one CTA (64 or 128 threads, n = 10, 11) or one
 * thread-block cluster of 2^n / 4096 CTAs of 256 threads (n = 12..16, two
 * CTAs per SM) per instance holds the state on chip for all rounds, forward
 * and backward, in one launch (16 amplitudes per thread; the checkpoints
 * still go to the workspace); otherwise, or with
 * GQAOA_GRAD_STREAMING, one CTA per instance for n <= 11 (forward and
 * adjoint kernels) and streaming passes over HBM above.
 * The clusters exchange each round's partial sums through mbarrier waits
 * bounded at 2 s; the call is asynchronous, so a wait that gives up (which
 * no correct launch does) is reported in the results: every value and
 * derivative of the call is then NaN.
 */
int gqaoa_grad(const uint8_t *cost, int n, int m, const double *gammas, const double *betas,
               int p, int objective, double *value, double *dgamma, double *dbeta, void *ws,
               size_t ws_bytes, void *stream);

/*
 * Batched evolution of `batch` instances of equal n (Eq. 3 per instance).
 * cost        device uint8: instance b's table at cost + b * cost_stride;
 *             cost_stride = 2^n for one table per instance, 0 for one table
 *             shared by every instance (e.g. many angle sets of one formula);
 *             a multiple of 16 when n >= 12.
 * gammas, betas device double [batch][p].
 * state       device complex64 [batch][2^n] (in: psi_0 if GQAOA_STATE_IN; out: psi_p).
 * out         device double [batch][3] or NULL; trace device double [batch][p] or NULL.
 * ws          device workspace of gqaoa_evolve_batched_workspace_size(n, batch, p).
 * Other arguments and errors as for gqaoa_evolve, plus GQAOA_ERANGE when
 * batch < 1 or batch * p > 2^32.
 */
int gqaoa_evolve_batched_workspace_size(int n, int batch, int p, size_t *bytes);
int gqaoa_evolve_batched(const uint8_t *cost, int64_t cost_stride, int n, int m, int batch,
                         const double *gammas, const double *betas, int p, void *state,
                         double *out, double *trace, void *ws, size_t ws_bytes, unsigned flags,
                         void *stream);

/*
 * Batched objective and adjoint gradient of `batch` instances of equal n
 * (same definitions as gqaoa_grad, per instance). cost and cost_stride as for
 * gqaoa_evolve_batched; gammas, betas, dgamma, dbeta device double [batch][p];
 * value device double [batch]. The workspace
 * (gqaoa_grad_batched_workspace_size) holds p * batch * 2^n * 8 bytes of
 * checkpoints.
 */
int gqaoa_grad_batched_workspace_size(int n, int batch, int p, size_t *bytes);
int gqaoa_grad_batched(const uint8_t *cost, int64_t cost_stride, int n, int m, int batch,
                       const double *gammas, const double *betas, int p, int objective,
                       double *value, double *dgamma, double *dbeta, void *ws, size_t ws_bytes,
                       void *stream);

/*
 * Launch geometry of the streaming passes of gqaoa_evolve_batched and
 * gqaoa_grad_batched (adjoint = 0: forward rounds; 1: adjoint rounds) for
 * `batch` instances of 2^n amplitudes on the current device: the CTAs that
 * share one instance and the per-round reduction records each instance's
 * mixer sum <+|chi_k> (Eq. 2) is combined from. batch = 1 is the geometry
 * of gqaoa_evolve and gqaoa_grad. A query only: nothing is launched.
 * Errors: GQAOA_EINVAL (NULL outputs), GQAOA_ERANGE (n, batch).
 */
int gqaoa_batched_geometry(int n, int batch, int adjoint, int *ctas_per_instance,
                           int *records_per_instance);

/*
 * Single-angle-pair sweep (Eq. 5; Appendix C's grid scan): `batch` instances
 * of equal n times `angles` angle points, each evolved p rounds from |+> with
 * gamma_k = gammas[a], beta_k = betas[a], and P(C=0) read out after each
 * round count listed in `rounds`. One persistent launch; each work item
 * (instance, angle point) is owned by one CTA or thread-block cluster.
 * cost    device uint8 [batch][2^n] (16-byte aligned).
 * gammas, betas  device double [angles].
 * rounds  host int32 [nrounds], strictly ascending, each in 1..p; nrounds <= 16.
 * out     device double [batch][angles][nrounds] written.
 * ws      device workspace of gqaoa_sweep_workspace_size(n, angles,
 *         amps_per_thread) bytes (16-byte aligned), caller-owned.
 * amps_per_thread  selects where the state lives:
 *   16  a thread holds 16 amplitudes in registers (n in 9..18);
 *   32  16 in registers and 16 in shared memory (n in 10..19);
 *   GQAOA_SWEEP_L2  cluster-resident: one 16-CTA cluster per item keeps
 *       540672 amplitudes on chip (147456 in registers, 393216 in shared
 *       memory: 52 % of an n = 20 state) and streams the rest through its
 *       slot of the workspace (16 slots of 2^n * 8 bytes), which stays in L2
 *       while the items in flight fit there (n = 20: 3.75 MiB touched per
 *       item, at most 16 items); n in GQAOA_SWEEP_L2_MIN_N..
 *       GQAOA_SWEEP_L2_MAX_N;
 *   0   16 for n <= 18, 32 for n = 19, GQAOA_SWEEP_L2 for n >= 20.
 *   Other values: GQAOA_EINVAL; n outside the selected range: GQAOA_ERANGE.
 * Precision: complex64 state; the mixer sum is FP32 within a warp
 * (GQAOA_SWEEP_L2: double-float within a thread, then FP32 across the warp)
 * and double-float above that; P is formed in FP64.
 * The CTAs of a cluster exchange each round's partial sums through mbarrier
 * waits bounded at 2 s; the call is asynchronous, so a wait that gives up
 * (which no correct launch does) shows in the results: the P values that
 * depend on a missing partial are NaN.
 */
#define GQAOA_SWEEP_MIN_N 9
#define GQAOA_SWEEP_MAX_N 19
#define GQAOA_SWEEP_L2 1
#define GQAOA_SWEEP_L2_MIN_N 20
#define GQAOA_SWEEP_L2_MAX_N 24
int gqaoa_sweep_workspace_size(int n, int angles, int amps_per_thread, size_t *bytes);
int gqaoa_sweep(const uint8_t *cost, int n, int m, int batch, const double *gammas,
                const double *betas, int angles, int p, const int32_t *rounds, int nrounds,
                int amps_per_thread, double *out, void *ws, size_t ws_bytes, void *stream);

/*
 * Cost-class (reduced) model of single-angle-pair G-QAOA (Appendix C): from
 * |+> the state stays a function of the cost value, psi_k(z) = f_k(C(z)), so
 * a round (Eq. 3) acts on the class amplitudes f(c), c < hist_stride,
 * weighted by the manifold sizes h[c]. This is the paper's own simulation
 * method and the fast path of its angle grid searches; the statevector
 * entry points above remain the evolution itself.
 * For every instance b < batch and angle point a < angles it evolves p
 * rounds with gamma_k = gammas[a], beta_k = betas[a] from |+> and writes,
 * after every round k (0-based), round-major (the angle points of one round
 * and readout contiguous),
 *   out[((b * p + k) * 3 + 0) * angles + a] = P(C=0),
 *   out[((b * p + k) * 3 + 1) * angles + a] = <H_P> (Eq. 4),
 *   out[((b * p + k) * 3 + 2) * angles + a] = D, the probability of the
 *        lowest non-empty cost class (a Max-SAT assignment; D = P for a
 *        satisfiable instance).
 * hist   device uint64 [batch][hist_stride] (8-byte aligned): h[b][c], the
 *        number of assignments with cost c; each row sums to 2^n.
 *        hist_stride in 1..256 (m + 1 for m clauses).
 * gammas, betas  device double [angles].
 * out    device float [batch][p][3][angles] (4-byte aligned), written.
 * best   optional device int32 [batch][p]: the angle point with the smallest
 *        written <H_P> after round k (the smallest index among equal values;
 *        -1 where every value is NaN). NULL skips it.
 * ws     device workspace of gqaoa_reduced_sweep_workspace_size(hist_stride,
 *        batch, angles, p) bytes (16-byte aligned, caller-owned): the phase
 *        tables (hist_stride rounded up to 32 entries per angle point), the
 *        FP32 class weights and the per-warp minima behind `best`.
 * The kernel's work grows with hist_stride (8 to 16 classes per lane, 1 to 16
 * lanes per item): a caller that knows its last non-empty class can pass the
 * histogram cut after it (classes past the stride are empty).
 * Precision: complex64 class amplitudes and phases rounded to complex64 (as
 * the statevector path); the class sums and the readouts are FP32.
 * Errors: GQAOA_ERANGE for n outside 1..GQAOA_MAX_N, hist_stride outside
 * 1..256, batch < 1, angles outside 1..2^24, p outside 1..2^20, batch * angles
 * above 2^40 or batch * p of 2^31 or more; GQAOA_EINVAL for NULL or
 * misaligned pointers; GQAOA_ENOMEM for a short workspace. All are checked
 * before any launch; the workspace query checks the same shape limits.
 */
int gqaoa_reduced_sweep_workspace_size(int hist_stride, int batch, int angles, int p,
                                       size_t *bytes);
int gqaoa_reduced_sweep(const uint64_t *hist, int hist_stride, int n, int batch,
                        const double *gammas, const double *betas, int angles, int p,
                        float *out, int32_t *best, void *ws, size_t ws_bytes, void *stream);

/*
 * Fair-sampling metrics of Section IV (Table I): how evenly the shots of
 * gqaoa_sample cover the solutions (or any target cost class, e.g. the
 * lowest non-empty class for Max-SAT). For each of `runs` independent runs
 * (run r takes the shots r, r + runs, r + 2 runs, ... in that order, so
 * `shots` holds runs * shots_per_run outcomes from one sampler call):
 *   to_all[r]    = 1-based index (within the run) of the shot that completes
 *                  the set of target assignments, 0 if the run never does;
 *   to_reject[r] = the number of target draws d at which a chi-square test
 *                  of uniform sampling over the M target assignments first
 *                  rejects, 0 if it never does. The test runs after every
 *                  draw with d >= min_draws and rejects when
 *                  double(M sum_j O_j^2 - d^2) > chi2_crit * double(d), i.e.
 *                  Pearson's X^2 = sum_j (O_j - d/M)^2 / (d/M) > chi2_crit
 *                  with the exact integer numerator (O_j: draws of target j;
 *                  chi2_crit: the caller's (1 - alpha) quantile of the
 *                  chi-square law with M - 1 degrees of freedom).
 * The paper reports the mean of to_all over runs and the median of
 * to_reject over trials.
 * shots   device uint64 [shots_per_run][runs] (8-byte aligned); outcomes
 *         >= 2^n count as non-target.
 * cost    device uint8 [2^n] (gqaoa_build_cost).
 * target  the cost class counted (0 = solutions); targets: its size M, i.e.
 *         h[target] of gqaoa_build_cost. If the table has a different
 *         number of assignments of that cost, every output is -1.
 * to_all, to_reject  device int64 [runs], written.
 * ws      gqaoa_fairness_workspace_size(n, runs, targets) bytes (16-byte
 *         aligned, caller-owned): labels of the 2^n assignments and
 *         runs * M counters.
 * Errors: GQAOA_ERANGE for n outside 1..30, runs outside 1..2^32, target
 * outside 0..255, targets outside 1..2^n, min_draws < 1, or
 * targets * shots_per_run^2 beyond 4e18; GQAOA_EINVAL for NULL or
 * misaligned pointers; GQAOA_ENOMEM for a short workspace.
 */
int gqaoa_fairness_workspace_size(int n, int64_t runs, int targets, size_t *bytes);
int gqaoa_fairness(const uint64_t *shots, int64_t runs, int64_t shots_per_run,
                   const uint8_t *cost, int n, int target, int targets, double chi2_crit,
                   int64_t min_draws, int64_t *to_all, int64_t *to_reject, void *ws,
                   size_t ws_bytes, void *stream);

/* ------------------------------------------------------------------------
 * Learned angle proposer (K9). The paper observes that optimal angles
 * cluster with the instance size and clause count (Section III.B, Fig. 2;
 * Appendix D) and proposes deriving angles from statistics of the density of
 * states (Section V). The proposer is an MLP on the normalised cost
 * histogram:
 *   x = [h[c]/2^n for c = 0..d_in-3 (zero-padded), n/32, m/128]
 *   z1 = W1 x + b1, h1 = GELU(z1); z2 = W2 h1 + b2, h2 = GELU(z2);
 *   o = W3 h2 + b3; angles = 2 pi sigmoid(o) (d_out = 2p: p gammas, p betas)
 *   loss = mean over batch and outputs of 2 (1 - cos(angles - labels))
 *          (angles are 2 pi periodic; equal to the squared error for small
 *          differences)
 * GELU(x) = x Phi(x), exact normal CDF. FP32 throughout (loss in FP64).
 * params: device float, one flat vector [W1 (d_h x d_in), b1, W2 (d_h x d_h),
 * b2, W3 (d_out x d_h), b3], row-major. x: device float [batch][d_in].
 * ------------------------------------------------------------------------ */
int gqaoa_mlp_param_count(int d_in, int d_h, int d_out, size_t *count);
/* Activation workspace for a batch (both forward and backward). */
int gqaoa_mlp_workspace_size(int batch, int d_in, int d_h, int d_out, size_t *bytes);
/* angles: device float [batch][d_out] written. */
int gqaoa_mlp_forward(const float *params, int d_in, int d_h, int d_out, const float *x,
                      int batch, float *angles, void *ws, size_t ws_bytes, void *stream);
/* Forward + backward of the periodic loss against labels (device float
 * [batch][d_out]); grads: device float [param_count] written; loss: device
 * double [1] written. */
int gqaoa_mlp_backward(const float *params, int d_in, int d_h, int d_out, const float *x,
                       const float *labels, int batch, float *grads, double *loss, void *ws,
                       size_t ws_bytes, void *stream);
/* Features from histograms: hist device int64 [batch][hist_stride] (h[c] for
 * c <= m_b), ns, ms device int32 [batch]; x device float [batch][d_in]. */
int gqaoa_mlp_features(const int64_t *hist, int hist_stride, const int32_t *ns, const int32_t *ms,
                       int batch, int d_in, float *x, void *stream);

/*
 * Adam (Kingma and Ba, 2015) on `count` device values, in place:
 *   g' = grad_scale * g; m = b1 m + (1-b1) g'; v = b2 v + (1-b2) g'^2;
 *   p -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps)
 * step >= 1 is the 1-based update count. grad_scale = -1 maximises.
 * Used for the proposer's weights (f32) and for G-QAOA angles (f64).
 */
int gqaoa_adam_f32(float *params, const float *grads, float *m, float *v, int64_t count,
                   double lr, double beta1, double beta2, double eps, int step, double grad_scale,
                   void *stream);
int gqaoa_adam_f64(double *params, const double *grads, double *m, double *v, int64_t count,
                   double lr, double beta1, double beta2, double eps, int step, double grad_scale,
                   void *stream);

/*
 * gqaoa_evolve without a workspace, for callers that cannot allocate device
 * memory or pass scratch: a plugin behind a fixed interface that hands over
 * only inputs and outputs, code inside a framework that owns all device
 * memory, or code issuing work while a stream is captured in the global
 * capture mode (where cudaMalloc is refused). The paper has no counterpart;
 * this is a calling convention of this library only.
 *
 * Same arguments, results and errors as gqaoa_evolve, minus ws/ws_bytes.
 * Scratch: one file-scope device array of GQAOA_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits. p is limited
 * to 1..GQAOA_NOALLOC_MAX_P (GQAOA_ERANGE beyond). The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) with
 * that device current; make it before any stream capture. The address is
 * kept for the life of the process, so the entry point must not be called on
 * a device after cudaDeviceReset. All calls on a device share the array:
 * calls whose GPU work overlaps race and must be serialised by the caller. No
 * scratch word needs to start at zero; the contents left by a previous call
 * are overwritten before use.
 */
#define GQAOA_NOALLOC_MAX_P 256
#define GQAOA_NOALLOC_SCRATCH_BYTES (1u << 20) /* 1 MiB */
int gqaoa_evolve_noalloc(const uint8_t *cost, int n, int m, const double *gammas,
                         const double *betas, int p, void *state, double *out, double *trace,
                         unsigned flags, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GQAOA_H */
