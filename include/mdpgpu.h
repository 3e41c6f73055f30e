/*
 * mdpgpu.h - C ABI of the GB300 (sm_103a) library for inexact GMRES policy iteration
 * (iGMRES-PI) on finite discounted-cost Markov decision processes.
 *
 * Problem (paper Sec. 2): a finite MDP {S, A, P, g, gamma} with states 0..S-1 and actions
 * 0..A-1 (the paper counts from 1), transition rows p_{ss'}(a) that sum to one, bounded
 * stage costs g(s, a), discount gamma in (0, 1) and nonempty allowed-action sets A(s).
 *
 * Conventions shared by every entry point:
 *   - Return value: MDP_OK (0) on success, a negative MDP_E* code on failure;
 *     mdp_last_error() then returns a message (thread-local, valid until the next call on
 *     the same thread).  MDP_ENOCONV still writes the last iterate, policy and stats.
 *   - Plain entry points take HOST pointers: inputs are copied to the device, outputs are
 *     copied back before the call returns (the call synchronises the handle's stream).
 *     The *_dev entry points take DEVICE pointers, enqueue on the handle's stream and
 *     return without a host-side wait except where a scalar decides control flow.
 *   - Layouts are row-major C arrays: P[a][s][s'], col/val[a][s][j], g[a][s], mask[s][a].
 *   - A handle owns device copies of P, g and mask plus all solver workspace; the caller
 *     keeps ownership of every pointer it passes.  One handle serves one stream at a time;
 *     distinct handles may be used from distinct threads.
 *   - Every device wait inside the library is bounded; nothing here spins without limit.
 */
#ifndef MDPGPU_H
#define MDPGPU_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mdp_s* mdp_t;

enum mdp_status {
  MDP_OK = 0,
  MDP_EINVAL = -1,    /* bad argument or malformed MDP (see mdp_last_error) */
  MDP_ENOMEM = -2,    /* device allocation failed */
  MDP_ENOCONV = -3,   /* iteration cap reached before the stopping rule held */
  MDP_EDEVICE = -4,   /* CUDA runtime error */
  MDP_ETIMEOUT = -5,  /* a bounded device wait ran out */
  MDP_EBREAKDOWN_INFO = 1 /* informational success, returned by policy_eval_gmres when the
                           * target was met and its last inner GMRES solve ended by a lucky
                           * breakdown (the result is exact in the Krylov space); the solvers
                           * count breakdowns in mdp_stats.breakdowns and return MDP_OK */
};

enum mdp_dtype { MDP_F32 = 0, MDP_F64 = 1 };

/* Arithmetic of the solvers.
 *   MDP_PREC_FP64  : every vector and sum in FP64 (needs P stored in FP64 for full accuracy;
 *                    FP32-stored P is widened exactly on the fly).
 *   MDP_PREC_MIXED : P (FP32) and the Krylov vectors in FP32 with FP32 accumulation; the
 *                    value vector, the Bellman sweep that gives ||T(v)-v||_inf and the final
 *                    polish sweep in double-float (two-FP32) arithmetic, accurate to about
 *                    2^-48 relative; the Hessenberg least-squares (Givens) in FP64. */
enum mdp_precision { MDP_PREC_FP64 = 0, MDP_PREC_MIXED = 1 };

/* ---------------------------------------------------------------------------- handles */

/* Dense MDP (Sec. 2).  P: A*S*S values of type p_dtype, P[a][s][s'] = p_{ss'}(a); every
 * row must be nonnegative, finite and sum to 1 within 1e-5 absolute (either dtype, so FP32
 * rows widened to FP64 are accepted as the same MDP).
 * g: A*S finite FP64 costs, g[a][s] = g(s, a).  gamma in (0, 1).  mask: NULL (all actions
 * allowed) or S*A bytes, nonzero = allowed, with at least one allowed action per state.
 * On success *out holds a new handle.  Errors: MDP_EINVAL (bad sizes/values; nothing is
 * allocated), MDP_ENOMEM, MDP_EDEVICE. */
int mdp_create_dense(int64_t S, int32_t A, const void* P, int p_dtype, const double* g,
                     double gamma, const uint8_t* mask, mdp_t* out);

/* ELL-sparse MDP: row (a, s) lists k pairs (col[a][s][j], val[a][s][j]); p_{ss'}(a) is the
 * sum of val over the j with col = s'.  1 <= k <= S, 0 <= col < S, val as P above.
 * The handle may keep each row's pairs in another order: for banded data (every column within
 * 1792 states of its row) the pairs are placed to spread the windowed sweep's shared-memory
 * gathers over the banks.  Only the rounding of each row's sum can change; every solve, batch
 * and server holding the same MDP uses the same order. */
int mdp_create_ell(int64_t S, int32_t A, int32_t k, const int32_t* col, const void* val,
                   int val_dtype, const double* g, double gamma, const uint8_t* mask,
                   mdp_t* out);

/* Same as the two above with DEVICE input pointers (copied device-to-device).  Inputs are
 * validated on the device; no host copy of P is made. */
int mdp_create_dense_dev(int64_t S, int32_t A, const void* P, int p_dtype, const double* g,
                         double gamma, const uint8_t* mask, mdp_t* out);
int mdp_create_ell_dev(int64_t S, int32_t A, int32_t k, const int32_t* col, const void* val,
                       int val_dtype, const double* g, double gamma, const uint8_t* mask,
                       mdp_t* out);

/* Replace the transition data and costs of an existing handle with new HOST arrays of the
 * same shape and dtype (no allocation; validation as at creation).  This is the per-request
 * upload path of a client that reuses one handle for a stream of same-shaped MDPs. */
int mdp_load_dense(mdp_t h, const void* P, const double* g);
int mdp_load_ell(mdp_t h, const int32_t* col, const void* val, const double* g);
/* The same loads, enqueued on the handle's stream without waiting: the copies (asynchronous
 * from pinned host memory), the layout change and the device validation run in stream order,
 * and the host arrays must stay valid until the next call on this handle returns.  That next
 * call (a solve, bellman_apply, policy_eval_gmres, another load, mdp_set_stream, a batch over
 * the handle) first waits for this handle's stream and returns the validation result
 * (MDP_EINVAL for invalid data, nothing else done).  With two handles a client uploads the
 * next MDP while the current one solves. */
int mdp_load_dense_async(mdp_t h, const void* P, const double* g);
int mdp_load_ell_async(mdp_t h, const int32_t* col, const void* val, const double* g);

void mdp_destroy(mdp_t h);

/* Run the handle's work on a caller-provided cudaStream_t (passed as void*); NULL selects
 * the handle's own stream. */
int mdp_set_stream(mdp_t h, void* cuda_stream);

/* Shape query: any pointer may be NULL. kind: 0 dense, 1 ELL. */
int mdp_info(mdp_t h, int64_t* S, int32_t* A, int32_t* k, int32_t* kind, int32_t* dtype,
             double* gamma);

/* Device bytes held by the handle (transition data, costs, workspace). */
int64_t mdp_device_bytes(mdp_t h);

/* ---------------------------------------------------------------------------- options */

typedef struct {
  double alpha;        /* forcing term of the inner stopping rule (Sec. 3, Eq. stopping_rule) */
  double tol;          /* outer stop: ||T(v) - v||_inf <= tol */
  int32_t restart;     /* GMRES restart length W (1..64) */
  int32_t max_outer;   /* cap K on outer iterations (Alg. 2) */
  int32_t max_inner;   /* cap on Arnoldi steps per outer iteration */
  int32_t precision;   /* enum mdp_precision */
  int32_t opi_W;       /* OPI: applications of T^pi per outer step (Sec. 2.1) */
  int32_t pi_inner_tol_exp; /* PI: relative GMRES tolerance 10^-x for "exact" evaluation */
  int32_t flags;       /* MDP_FLAG_* bits */
  const double* v0;    /* initial V_0 (host for host calls, device for *_dev); NULL = 0 */
  double forcing_c;    /* forcing sequence of the inner stopping rule (Sec. 3): 0 = constant
                        * alpha (Alg. 2); c > 0: alpha_k = min(alpha, c ||Phi_k||_inf), which
                        * tends to 0 (locally Q-superlinear, Sec. 3 theorem), with the inner
                        * threshold alpha_k ||Phi_k||_inf kept >= tol / 10 */
  int32_t precond_block; /* ipi_solve on ELL data: 0 = plain GMRES (Alg. 2); b = 2^j in
                        * [4, 2^20] = right-preconditioned inner GMRES with the two-level
                        * preconditioner M^{-1} q = q + Pr J_c^{-1} R q, where R averages over
                        * blocks of b consecutive states, Pr copies a block value back and
                        * J_c = R J^pi Pr (preconditioning is the extension named in Sec. 5).
                        * Needs at most 8192 blocks and transitions that stay within 31 blocks
                        * of their state (MDP_EINVAL otherwise).  Other solvers reject it. */
} mdp_opts;

/* ipi_solve runs each inner GMRES solve as one CUDA-graph launch with a device-side loop.
 * MDP_FLAG_HOST_LOOP enqueues the same kernels step by step from the host instead (one
 * host wait per Arnoldi step), for tools that cannot follow conditional graph nodes. */
#define MDP_FLAG_HOST_LOOP 1
/* ELL data whose columns all lie within 1792 states of their row's state (banded P, measured
 * when the data is validated) is swept, and multiplied in the Arnoldi steps, by kernels that
 * keep a window of the vector in shared memory; MDP_FLAG_NO_WINDOW makes the solvers use the
 * global-gather kernels instead (same values; for comparison and profiling).  mdp_set_geometry
 * with sweep_blocks > 0 (matvec_blocks > 0) also selects the global-gather sweep (matvec). */
#define MDP_FLAG_NO_WINDOW 2
/* With precond_block > 0, ipi_solve builds the coarse factorization of the two-level
 * preconditioner for the first policy and rebuilds it only when more than 1 in 1000 states have
 * changed their action since it was built (a preconditioner built for a nearby policy is still a
 * valid right preconditioner: the iterate uses the same M^{-1} as the Arnoldi process, so only
 * the number of steps can change, never the result).  MDP_FLAG_PC_REBUILD rebuilds it for every
 * policy. */
#define MDP_FLAG_PC_REBUILD 4

/* alpha 0.1, tol 1e-8, restart 30, max_outer 100, max_inner 3000, precision MIXED,
 * opi_W 50, pi_inner_tol_exp 13, flags 0, v0 NULL, forcing_c 0, precond_block 0. */
mdp_opts mdp_opts_default(void);

typedef struct {
  int32_t outer;        /* outer iterations done */
  int32_t inner;        /* Arnoldi steps (all outer iterations) */
  int32_t restarts;     /* GMRES restarts */
  int32_t sweeps;       /* Bellman sweeps (full, all actions) */
  int32_t matvecs;      /* P^pi matrix-vector products (incl. T^pi applications) */
  int32_t status;       /* enum mdp_status of the solve */
  double residual_inf;  /* ||T(V_K) - V_K||_inf of the returned iterate */
  double seconds;       /* wall time of the call */
  double bytes;         /* algorithmic HBM bytes moved by the solve's kernels */
  double sweep_ms;      /* summed device time of the Bellman sweep launches (timing on) */
  double matvec_ms;     /* summed device time of the P^pi matvec launches (timing on) */
  int32_t timed_sweeps; /* sweep launches covered by sweep_ms */
  int32_t timed_matvecs;/* matvec launches covered by matvec_ms */
  int32_t launches;     /* kernels launched by the call */
  int32_t breakdowns;   /* inner GMRES solves that ended by a lucky breakdown (Alg. 2's
                         * "||q||_2 = 0" branch: the Krylov space is invariant, so the least-
                         * squares iterate solves the inner system exactly) */
} mdp_stats;

/* Kernel shape for ELL data: lanes that share one row in the Bellman sweep and in the P^pi
 * matvec (1, 2, 4 or 8; 0 = the library's choice).  Results do not depend on it beyond the
 * order of floating-point additions.  Returns MDP_EINVAL for other values. */
int mdp_set_tuning(mdp_t h, int32_t ell_lanes_sweep, int32_t ell_lanes_matvec);

/* Block geometry of the ELL kernels: blocks of the Bellman sweep, of the P^pi matvec and of
 * the Krylov vector kernels (0 = library choice, else 1..2048).  Norms and dot products are
 * summed per block first, so the geometry fixes the order of floating-point additions; a
 * batch reports each instance's geometry (mdp_batch_geometry) so that a single solve can
 * reproduce that instance's results bit for bit.  ELL handles only, else MDP_EINVAL. */
int mdp_set_geometry(mdp_t h, int32_t sweep_blocks, int32_t matvec_blocks,
                     int32_t krylov_blocks);

/* When on (nonzero), every Bellman-sweep and matvec launch is bracketed by CUDA events on
 * the handle's stream and its device time is added to mdp_stats.sweep_ms / matvec_ms. */
int mdp_set_timing(mdp_t h, int on);

/* ---------------------------------------------------------------------------- operators */

/* One Bellman sweep (Sec. 2; Alg. 2 lines "pi_k <- GreedyPolicy(V_k)" and "Phi_k"):
 *   Q(s,a) = g(s,a) + gamma * sum_s' p_{ss'}(a) v(s'),  pi(s) = argmin_{a in A(s)} Q(s,a)
 *   (lowest index among exact minima), Tv(s) = Q(s, pi(s)), res_inf = ||Tv - v||_inf.
 * Host pointers v[S] (in), Tv[S], pi[S] (out, may be NULL), res_inf (out, may be NULL).
 * precision selects FP64 or double-float accumulation (see enum mdp_precision). */
int bellman_apply(mdp_t h, const double* v, double* Tv, int32_t* pi, double* res_inf,
                  int32_t precision);

/* Device-pointer form; margin[S] (may be NULL) receives Q2(s) - Q1(s), the gap between the
 * two smallest Q values (+inf with one allowed action).  *res_inf is a HOST pointer and the
 * call waits for it when it is not NULL. */
int bellman_apply_dev(mdp_t h, const double* v, double* Tv, int32_t* pi, double* margin,
                      double* res_inf, int32_t precision);

/* Largest S that bellman_apply_ell_noalloc_dev accepts. */
#define MDP_NOALLOC_MAX_STATES (1 << 20)

/* One Bellman sweep that allocates nothing, for callers that may not allocate memory while
 * they run: a server or control loop that gave the whole device to its own pooling allocator
 * at start-up (another allocator's cudaMalloc would fail or fragment that pool), or
 * latency-critical code in which cudaMalloc/cudaFree, which can synchronise the device, would
 * stall other streams.  The paper has no counterpart; it is a convenience of this library.
 *   Inputs, all DEVICE pointers in the caller's layout, FP64 values: col[a][s][j] and
 *   val[a][s][j] (A*S*k), g[a][s] (A*S), v[s] (S); every action is allowed.
 *   Outputs (DEVICE): Tv[S], pi[S] (lowest index among exact minima) and res_inf[1] =
 *   ||Tv - v||_inf, or NaN when some col lies outside [0, S) (that entry is skipped).
 * Its only scratch is a fixed array in the library's device image (33 KiB, held by every GPU
 * that loads the library until the process exits); no cudaMalloc, cudaFree or other
 * allocating call is made.  S > MDP_NOALLOC_MAX_STATES is rejected with MDP_EINVAL before any
 * work.  Errors are reported by the return code only (MDP_EINVAL for bad sizes or null
 * pointers, MDP_EDEVICE for CUDA errors); mdp_last_error is not updated, since storing a
 * message could allocate host memory.  The first call on a device looks the scratch address
 * up (cudaGetSymbolAddress), so make that first call before any stream capture.  The address
 * is cached per device for the life of the process: cudaDeviceReset (or anything else that
 * destroys the primary context) unloads the device image it points into, so after such a reset
 * this entry point must not be called again in that process.  All calls
 * share the scratch, which keeps the last call's contents; each call clears the counters it
 * needs on its own stream first, and calls whose work overlaps on the GPU (unordered streams)
 * race on it.  Work is enqueued on `stream` (a cudaStream_t; NULL = legacy default stream)
 * and the call returns without waiting. */
int bellman_apply_ell_noalloc_dev(int64_t S, int32_t A, int32_t k, const int32_t* col,
                                  const double* val, const double* g, double gamma,
                                  const double* v, double* Tv, int32_t* pi, double* res_inf,
                                  void* stream);

/* Inexact policy evaluation (Alg. 2 inner loop for a fixed pi): restarted GMRES(W) on
 * (I - gamma P^pi) V = g^pi from v0 (NULL = 0) until ||g^pi - (I - gamma P^pi) V||_inf <=
 * target_inf or opts->max_inner steps.  Host pointers pi[S], v0[S], v_out[S]. */
int policy_eval_gmres(mdp_t h, const int32_t* pi, const double* v0, double target_inf,
                      const mdp_opts* opts, double* v_out, mdp_stats* stats);
int policy_eval_gmres_dev(mdp_t h, const int32_t* pi, const double* v0, double target_inf,
                          const mdp_opts* opts, double* v_out, mdp_stats* stats);

/* ---------------------------------------------------------------------------- solvers */

/* iGMRES-PI, Alg. 2: for k < max_outer: pi_k = GreedyPolicy(V_k), Phi_k = T(V_k) - V_k;
 * stop when ||Phi_k||_inf <= tol; otherwise GMRES(W) on (I - gamma P^{pi_k}) V = g^{pi_k}
 * from V_k while ||g^{pi_k} - (I - gamma P^{pi_k}) V_{k+1}||_inf > alpha ||Phi_k||_inf.
 * Returns v = T(V_K), pi = GreedyPolicy(V_K) and ||Phi_K||_inf in stats.  Host pointers. */
int ipi_solve(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
              mdp_stats* stats);
int ipi_solve_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
                  mdp_stats* stats);

/* VI (Sec. 2.1, Eq. VI_optimalcost): V <- T V until ||T V - V||_inf <= tol. */
int vi_solve(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out, mdp_stats* stats);
int vi_solve_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
                 mdp_stats* stats);

/* PI (Sec. 2.1): policy evaluation by GMRES to a relative residual 10^-pi_inner_tol_exp,
 * then improvement, until ||T V - V||_inf <= tol or the policy repeats. */
int pi_solve(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out, mdp_stats* stats);
int pi_solve_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
                 mdp_stats* stats);

/* OPI (Sec. 2.1): per outer step, W = opts->opi_W applications of T^{pi_k}, the first being
 * the T V_k of the greedy sweep. */
int opi_solve(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
              mdp_stats* stats);
int opi_solve_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
                  mdp_stats* stats);

/* Inexact policy iteration with VI as the inner solver (Alg. 1; Sec. 3 notes it is OPI whose
 * number of inner steps is set by the stopping rule): per outer step, V <- T^{pi_k} V from
 * T V_k while ||g^{pi_k} - J^{pi_k} V||_inf > alpha_k ||Phi_k||_inf (alpha_k as in ipi_solve,
 * at most max_inner steps).  stats.inner counts the applications of T^{pi_k}. */
int ipi_vi_solve(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out, mdp_stats* stats);
int ipi_vi_solve_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,
                     mdp_stats* stats);

/* ---------------------------------------------------------------------------- batches */
/* A batch solves n independent MDPs with iGMRES-PI (Alg. 2, mixed precision) in one
 * CUDA-graph launch: each instance runs the outer loop as a device-side state machine, and
 * one loop iteration serves every instance with one launch per kernel family (Bellman sweep,
 * P^pi matvec, CGS2, estimate, ...), each launch walking only the instances whose step is
 * due.  Every instance's results equal those of ipi_solve on that handle alone with the
 * batch's kernel shape (mdp_batch_geometry -> mdp_set_tuning + mdp_set_geometry).
 *
 * hs: n ELL handles with FP32 transition data on the current device; the batch reads their
 * device data, so they must outlive it.  opts: shared options (NULL = defaults); precision
 * must be MDP_PREC_MIXED, v0 NULL (every instance starts from V_0 = 0), 0 < alpha < 1.
 * The batch allocates its workspace in one block at creation (mdp_batch_device_bytes).
 * Errors: MDP_EINVAL (bad arguments), MDP_ENOMEM, MDP_EDEVICE. */
typedef struct mdp_batch_s* mdp_batch_t;
int mdp_batch_create(const mdp_t* hs, int32_t n, const mdp_opts* opts, mdp_batch_t* out);
void mdp_batch_destroy(mdp_batch_t b);
/* Stream for the batch's launches (a cudaStream_t; NULL = the batch's own stream). */
int mdp_batch_set_stream(mdp_batch_t b, void* stream);
/* Autotuner: for each ELL row length present, times the batched Bellman sweep and the
 * batched matvec with 1, 2, 4 and 8 lanes per row (warp shape) and keeps the fastest, then, with
 * that shape, times row tiles of 1/2, 1, 2 and 4 times the library's states per virtual block
 * (about 512 KB of P per sweep block and 256 KB per matvec block) and keeps the fastest; tiles
 * whose matvec partial sums would not fit the instance's workspace are skipped.  Both change
 * only the order of floating-point additions (mdp_batch_geometry reports the choice, so a single
 * solve can reproduce an instance bit for bit).  Runs kernels on the batch's stream; synchronous. */
int mdp_batch_tune(mdp_batch_t b);
/* Kernel shape of instance i (any output may be NULL). */
int mdp_batch_geometry(mdp_batch_t b, int32_t i, int32_t* lanes_sweep, int32_t* lanes_matvec,
                       int32_t* sweep_blocks, int32_t* matvec_blocks, int32_t* krylov_blocks);
int64_t mdp_batch_device_bytes(mdp_batch_t b);
/* Solve every instance.  v_out[i]: S_i doubles = T(V_K); pi_out[i]: S_i ints = pi_K;
 * stats[i] (stats may be NULL; launches counts the whole batch's kernels).  The pointer
 * arrays are host arrays; the buffers they point to are host memory (mdp_batch_solve) or
 * device memory (mdp_batch_solve_dev).  Synchronous.  Returns MDP_OK when every instance
 * converged, MDP_ENOCONV when some reached max_outer (stats[i].status says which; their
 * best v and pi are still written), MDP_ETIMEOUT when the loop guard ended the launch. */
int mdp_batch_solve(mdp_batch_t b, double* const* v_out, int32_t* const* pi_out,
                    mdp_stats* stats);
int mdp_batch_solve_dev(mdp_batch_t b, double* const* v_out, int32_t* const* pi_out,
                        mdp_stats* stats);
/* One Bellman sweep (Sec. 2, the operator T) of every instance at its current V, in one
 * launch per lane class: after a solve V = V_K, so this recomputes T V_K, GreedyPolicy(V_K)
 * and ||T V_K - V_K||_inf inside the batch's workspace.  res_inf: n host doubles, or NULL
 * to return without waiting (the launches are then only enqueued on the batch's stream). */
int mdp_batch_bellman(mdp_batch_t b, double* res_inf);
/* opts->flags & MDP_FLAG_HOST_LOOP makes mdp_batch_solve enqueue the loop iterations from the
 * host (one host wait per iteration) instead of launching one graph: same kernels, same
 * results, visible to profilers that cannot follow conditional graph nodes. */
/* One-shot form: create a batch of hs[0..n-1], solve into host buffers, destroy. */
int ipi_solve_batch(const mdp_t* hs, int32_t n, const mdp_opts* opts, double* const* v_out,
                    int32_t* const* pi_out, mdp_stats* stats);

/* ---------------------------------------------------------------------------- serving */
/* A server solves a stream of requests with continuous batching: each request is an ELL MDP
 * with FP32 transition data, solved by iGMRES-PI (Alg. 2, mixed precision) from V_0 = 0.
 * Admitted requests keep P, g, V, pi and the Krylov basis resident on the device; the
 * device runs the batch engine's loop (see mdp_batch_*) over every active slot, in launches
 * of iters_per_launch iterations, and between launches the host retires finished requests
 * and activates newly uploaded ones, so requests that arrive while others are solving join
 * the running mix.  A request is admitted (in arrival order) when a slot is free and its
 * device bytes fit in the HBM budget together with every other admitted request.  Each
 * result equals that of the same MDP solved alone (ipi_solve with the batch engine's kernel
 * shape, see mdp_batch_geometry): the slots never exchange data.
 * A server is used by one host thread at a time; it never blocks on the device except in
 * mdp_server_drain. */
typedef struct mdp_server_s* mdp_server_t;
typedef struct {
  int64_t hbm_budget_bytes; /* device bytes of all admitted requests together (default 120 GiB) */
  int32_t max_slots;        /* requests on the device at once (1..4096, default 256) */
  int32_t iters_per_launch; /* loop iterations per device launch (default 4) */
  mdp_opts solver;          /* shared solver options: precision MIXED, v0 NULL, 0 < alpha < 1 */
} mdp_server_opts;
mdp_server_opts mdp_server_opts_default(void);
int mdp_server_create(const mdp_server_opts* opts, mdp_server_t* out);
void mdp_server_destroy(mdp_server_t s);  /* waits for the device, drops unfinished requests */
/* Queue one request.  col / val [A][S][k] (int32 / FP32), g [A][S] (FP64): host arrays
 * (pinned memory keeps the upload asynchronous).  v_out (S doubles) and pi_out (S ints):
 * host or device buffers that receive T(V_K) and pi_K.  Every array must stay valid until
 * the request is reported done.  *request_id (may be NULL) identifies it in poll results.
 * Invalid data (found on the device) completes the request with status MDP_EINVAL; a request
 * larger than the whole budget completes with MDP_ENOMEM. */
int mdp_server_submit(mdp_server_t s, int64_t S, int32_t A, int32_t k, const int32_t* col,
                      const float* val, const double* g, double gamma, double* v_out,
                      int32_t* pi_out, int64_t* request_id);
/* Advance the server without waiting (retire, admit, activate, launch) and report up to
 * max_done completed requests: ids[i] and stats[i] (status, outer/inner counts, residual,
 * seconds = submit-to-completion latency).  ids / stats may be NULL. */
int mdp_server_poll(mdp_server_t s, int64_t* ids, mdp_stats* stats, int32_t max_done,
                    int32_t* n_done);
/* Run until every submitted request has completed (results stay queued for poll). */
int mdp_server_drain(mdp_server_t s);
/* Requests holding a slot, requests waiting, device bytes admitted, loop launches so far. */
int mdp_server_info(mdp_server_t s, int32_t* active, int32_t* pending, int64_t* bytes_in_use,
                    int64_t* launches);

/* ------------------------------------------------------------ row-sharded solve (multi-GPU)
 * One MDP whose states are split by rows over several processes, one GPU each: the parallel /
 * distributed iGMRES-PI the paper names as future work (Sec. 5).  Rank r owns the contiguous
 * global rows [row_begin[r], row_begin[r+1]) of every P_a and g_a, and the same rows of V, T V,
 * Phi, pi and of every Krylov vector.  Alg. 2 then needs three exchanges, which the caller
 * supplies as HOST collectives (any transport: torch.distributed, MPI, NCCL behind a staging
 * copy): an all-gather of the rows of a vector (V before each Bellman sweep, the Arnoldi vector
 * before each P^pi matvec, a candidate iterate before its true residual), an allreduce-max
 * (||Phi||_inf, the true residual's inf-norm, the agreement on each accept / restart decision)
 * and an allreduce-sum (||Phi||_2^2, the two CGS2 projections Q^T w, ||w||_2^2).  The Hessenberg
 * least squares and its Givens rotations are replicated on every rank in FP64. */
typedef struct mdp_shard_s* mdp_shard_t;

/* allgather: local holds this rank's rows (rows * bytes_per_row bytes, host), global receives
 * every rank's rows in row order (S * bytes_per_row bytes, host).  allreduce: vals[n] (host) is
 * replaced in place by the sum (op 0) or the maximum (op 1) over ranks; every rank must receive
 * the same values.  Both return 0 on success; a nonzero return ends the solve with MDP_EDEVICE.
 * Every rank calls them in the same order with the same sizes. */
typedef int (*mdp_allgather_fn)(void* ctx, const void* local, void* global, int64_t bytes_per_row);
typedef int (*mdp_allreduce_fn)(void* ctx, double* vals, int32_t n, int32_t op);
typedef struct {
  void* ctx;                  /* passed to the callbacks */
  int32_t rank, world;        /* this rank, number of ranks */
  const int64_t* row_begin;   /* [world + 1]: row_begin[0] = 0, row_begin[world] = S */
  mdp_allgather_fn allgather;
  mdp_allreduce_fn allreduce;
} mdp_comm;

/* This rank's rows of an ELL MDP with S states in all: rows [row0, row0 + rows), arrays in the
 * layout of mdp_create_ell restricted to those rows: col / val [A][rows][k] (int32 global
 * column indices in [0, S); FP32 or FP64 values), g [A][rows] (FP64), host pointers, copied.
 * Every action is allowed.  Validation on the host: sizes, 0 <= col < S, values finite and
 * >= 0, row sums within 1e-5 of 1, g finite, 0 < gamma < 1 (MDP_EINVAL otherwise). */
int mdp_shard_create(int64_t S, int64_t row0, int64_t rows, int32_t A, int32_t k, const int32_t* col,
                     const void* val, int val_dtype, const double* g, double gamma,
                     mdp_shard_t* out);
void mdp_shard_destroy(mdp_shard_t h);

/* iGMRES-PI (Alg. 2) on the sharded MDP, called by every rank with its own shard and the same
 * options: the stopping rules of ipi_solve (outer ||T V - V||_inf <= tol; inner true residual
 * ||g^pi - J^pi V||_inf <= alpha_k ||Phi_k||_inf, formed once the Givens estimate comes within
 * sqrt(S) of it, at the end of each restart cycle, at a lucky breakdown and at max_inner), in
 * FP64 arithmetic (opts->precision is ignored; precond_block must be 0).  Outputs are this rank's
 * rows: v_out[rows] = T(V_K), pi_out[rows] = GreedyPolicy(V_K) (host or device pointers, pi_out
 * may be NULL).  opts->v0 (rows entries) warm-starts V.  Returns MDP_OK, MDP_ENOCONV at
 * max_outer, MDP_EINVAL when the communicator's partition does not match the shard, MDP_EDEVICE
 * on a CUDA or callback failure. */
int ipi_solve_sharded(mdp_shard_t h, const mdp_comm* comm, const mdp_opts* opts, double* v_out,
                      int32_t* pi_out, mdp_stats* stats);

/* Inspection of the two-level preconditioner (the preconditioned policy evaluation that
 * ipi_solve runs with mdp_opts.precond_block; preconditioning is named as future work in
 * Sec. 5).  For the policy pi[S] (host or device pointer, every entry an allowed action) and
 * aggregation blocks of `block` states (a power of two in [2, S]), builds the Galerkin coarse
 * operator J_c = R (I - gamma P^pi) Pr, factors it and forms J_c^{-1} in FP32 exactly as the
 * solver does once per policy, and copies J_c^{-1} row-major into inv_out[nc * nc] (host;
 * NULL = size query only).  *nc_out = number of coarse blocks ceil(S / block), *bw_out = the
 * band half-width of J_c in blocks (either may be NULL).  ELL handles only.  Returns MDP_EINVAL
 * for dense data, a bad block, a policy entry out of range, more than 8192 blocks or a band
 * wider than 31 blocks; the handle's solver workspace is reused. */
int mdp_precond_coarse_inverse(mdp_t h, const int32_t* pi, int32_t block, float* inv_out,
                               int64_t* nc_out, int32_t* bw_out);

/* Arithmetic-rate probe (no counterpart in the paper; it states the peak against which the
 * plain FP64 form's sweep is measured, since on this GPU that form can be bound by FP64
 * arithmetic rather than by HBM).  Runs eight independent FMA chains per thread over a grid of
 * 8 blocks per SM on the current device, in the given dtype (MDP_F64 or MDP_F32), and writes
 * the best of three timed launches to *tflops (2 flops per FMA).  Allocates a small scratch
 * buffer and a private stream for the duration of the call and synchronises on it; about 0.1 s
 * for FP64.  Returns MDP_EINVAL for another dtype or a NULL output, MDP_EDEVICE/ENOMEM on CUDA
 * failures. */
int mdp_probe_alu(int32_t dtype, double* tflops);

/* Self-test of the bounded device waits (no counterpart in the paper).  Every spin-wait in the
 * library's kernels (the mbarrier waits of the bulk-copy pipelines) gives up after about a
 * second of SM clock cycles, raises an error flag that the host reads back as MDP_ETIMEOUT, and
 * leaves the context usable.  This call runs that same wait helper in a one-thread kernel on the
 * current device, on an mbarrier that expects one arrival, with the given limit in clock cycles
 * (1 .. 2^31): with arrive = 0 nothing arrives, so the wait runs out and the call returns
 * MDP_ETIMEOUT; with arrive = 1 the thread arrives first and the call returns MDP_OK.  No copy
 * is in flight while it waits.  Synchronous; allocates 4 bytes for the flag. */
int mdp_selftest_wait(int64_t limit_cycles, int32_t arrive);

/* Message for the last nonzero return on this thread ("" if none). */
const char* mdp_last_error(void);

/* Library version string. */
const char* mdp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MDPGPU_H */
