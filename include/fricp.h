/*
 * fricp.h -- C ABI of a GB300 (sm_103a) implementation of the per-iteration hot
 * path of "Fast and Robust Iterative Closest Point" (J. Zhang, Y. Yao, B. Deng;
 * IEEE TPAMI 2021, arXiv 2007.07627).
 *
 * The problem (Sec. 3, Eq. 1): find a rigid motion (R, t) taking the source set
 * P = {p_i} (M points) onto the target set Q = {q_j} (N points, optionally with
 * unit normals n_j). Three solvers are provided:
 *   FRICP_P2P_AA          point-to-point ICP with Anderson acceleration on the
 *                         se(3) parameterisation and the energy safeguard
 *                         (Sec. 4.2, "Fast ICP"): Algorithm 1 with psi(x) = x^2,
 *                         unit weights and a single stage;
 *   FRICP_P2P_WELSCH_AA   Welsch-robust point-to-point ICP (Sec. 4.3, Alg. 1);
 *   FRICP_P2PL_WELSCH_AA  Welsch-robust point-to-plane ICP (Sec. 5, Alg. 2);
 *   FRICP_P2PL_AA         plain point-to-plane ICP (Sec. 5, Eq. 15) with the
 *                         Gauss-Newton / Anderson / line-search scheme of
 *                         Alg. 2 and psi(x) = x^2.
 * Points in the plane (the paper states the problem in R^d, Sec. 3) are
 * registered as 3-D points with z = 0: the result is then a rotation about z
 * and a translation in the plane (see the 2-D tests).
 *
 * Conventions for every call:
 *   - Point arrays are contiguous float32 [n][3] (x, y, z); normals likewise.
 *     `on_device` != 0 means the pointer is CUDA device memory of the current
 *     device, otherwise host memory. The library never keeps a caller pointer
 *     past the call: inputs are copied into library-owned device buffers.
 *   - Transforms are double [16], row-major 4x4 homogeneous matrices
 *     [[R, t], [0, 1]] in the caller's coordinates, x -> R x + t.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream). All device work
 *     of a call is issued on it; calls that return results to the host wait for
 *     that stream only.
 *   - No call aborts, traps or exits. Every call returns a fricp_status; on any
 *     status other than FRICP_OK, fricp_last_error() returns a message
 *     (thread-local, valid until the next call on the same thread).
 *   - All calls are thread-compatible: distinct handles may be used from
 *     distinct threads; one handle must not be used by two threads at once.
 */
#ifndef FRICP_H
#define FRICP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FRICP_OK = 0,
    FRICP_EINVAL = 1,       /* bad argument: null pointer, size, NaN/Inf input, non-unit normal */
    FRICP_ENOMEM = 2,       /* device or host allocation failed */
    FRICP_ECUDA = 3,        /* a CUDA runtime call failed (message has the CUDA error string) */
    FRICP_ETIMEOUT = 4,     /* the registration did not finish within params.timeout_s or the step budget */
    FRICP_EDEGENERATE = 5,  /* all Welsch weights vanished (sum w = 0) or the 6x6 point-to-plane
                               system is not positive definite; the last valid iterate is returned */
    FRICP_EUNSUPPORTED = 6, /* variant needs something the target lacks (normals) */
    FRICP_EBUSY = 7,        /* the server's request queue is full; step it and submit again */
    FRICP_EOVERFLOW = 8     /* a bounded internal work buffer (a search stack, a candidate or tile
                               list) overflowed; not expected on finite input */
} fricp_status;

typedef enum {
    FRICP_P2P_AA = 0,
    FRICP_P2P_WELSCH_AA = 1,
    FRICP_P2PL_WELSCH_AA = 2,
    FRICP_P2PL_AA = 3,       /* plain point-to-plane ICP (Eq. 15) solved like Alg. 2 with psi(x) = x^2:
                                weights 1, energy sum H_i^2, one stage capped by max_iters */
    FRICP_SYM_WELSCH_AA = 4  /* Welsch-robust symmetric objective, the extension Sec. 7 proposes: Alg. 2
                                on H_i = (R p_i + t - q_i) . (R np_i + nq_i), the two surfaces' normals
                                summed at each pair (needs source normals: fricp_register_symmetric) */
} fricp_variant;

/* Arithmetic of the correspondence search and the per-point terms. The sums,
 * the 3x3 / 6x6 solves and the Anderson least squares are FP64 in every mode.
 *   FRICP_PREC_FP64          the reference: candidates screened in float and
 *                            re-ranked in double-float, so the winner is the FP64
 *                            argmin (ties to the lowest original index); residuals,
 *                            weights and products in FP64;
 *   FRICP_PREC_FP32          transform, distances, residuals, weights and products in
 *                            float (ties among equal float distances to the lowest
 *                            original index), widened to FP64 for the sums;
 *   FRICP_PREC_FP16_STORAGE  as FP32, on target coordinates stored as 16-bit offsets
 *                            in their bucket's bounding box (8 B per point instead of
 *                            16; built once per target on first use); ties to the
 *                            lowest position in bucket order.
 * FP32 and FP16 results differ from the FP64 oracle by their rounding (closest
 * points within float resolution, weights to ~1e-7); registrations, not passes,
 * are what they are meant for. */
typedef enum {
    FRICP_PREC_FP64 = 0,
    FRICP_PREC_FP32 = 1,
    FRICP_PREC_FP16_STORAGE = 2
} fricp_precision;

/* How the exact closest-point search (Eq. 3) of fricp_register is laid out on
 * the GPU; the result is the same exact argmin either way, only the time
 * differs.
 *   FRICP_SEARCH_TILE   a warp takes 8 Morton-adjacent queries (four lanes
 *                       each), walks the tree once for all eight, pruning each
 *                       node by every query's own bound, and streams the
 *                       buckets kept through shared memory with asynchronous
 *                       copies; a query without a warm start is searched by
 *                       the whole warp alone. Fewer instructions per query,
 *                       but one registration's slowest tiles bound the pass;
 *   FRICP_SEARCH_QUERY  every query is searched by a whole warp (two per warp
 *                       where the Welsch cap is off): the default, faster on a
 *                       single registration.
 * The batched and served engines choose between the two per size class by
 * timing them (fricp_batch_last_shape). */
typedef enum {
    FRICP_SEARCH_TILE = 0,
    FRICP_SEARCH_QUERY = 1
} fricp_search;

/* Solver parameters. fricp_params_default fills the paper's defaults. */
typedef struct {
    int32_t variant;            /* fricp_variant */
    int32_t anderson_m;         /* m, previous iterates used by AA: 5 (Sec. 4.2). 0..8; 0 = plain MM */
    int32_t max_iters;          /* I_nu for point-to-point: 1000 (Sec. 4.3). >= 1 */
    int32_t p2pl_iters_first;   /* I_nu at nu_max for point-to-plane: 6 (Sec. 5) */
    int32_t p2pl_iters_cap;     /* +1 per nu stage, at most 10 (Sec. 5) */
    int32_t max_line_search;    /* l_max of Alg. 2; the paper gives no value: 10 */
    double  eps;                /* epsilon_nu, convergence threshold: 1e-5 (Sec. 4.3, Sec. 5) */
    double  nu_max;             /* <= 0: 3 x median initial distance (Sec. 4.3) / plane distance (Sec. 5) */
    double  nu_min;             /* <= 0: E_Q / (3 sqrt 3) (Sec. 4.3) / H_Q / 6 (Sec. 5) */
    double  nu_min_floor;       /* lower clamp of nu_min (normalised units): 1e-6 */
    int32_t steps_per_sync;     /* device steps replayed between two host polls of the done flag: 16 */
    int32_t use_graph;          /* 1: replay the steps as a captured CUDA graph; 0: plain launches */
    int32_t time_passes;        /* 1: bracket every step launch with CUDA events (implies use_graph = 0) */
    int32_t max_steps;          /* hard cap on device steps (correspondence passes): 100000 */
    double  timeout_s;          /* host wait limit for one registration: 600 */
    int32_t precision;          /* fricp_precision: FRICP_PREC_FP64 */
    int32_t search;             /* fricp_search: FRICP_SEARCH_QUERY */
} fricp_params;

/* Result of one registration. All transforms in the caller's coordinates. */
typedef struct {
    double  R[9];               /* row-major rotation */
    double  t[3];               /* translation */
    int32_t status;             /* FRICP_OK, FRICP_EDEGENERATE or FRICP_EOVERFLOW */
    int32_t iterations;         /* inner-loop bodies run over all nu stages (Alg. 1 / Alg. 2) */
    int32_t corr_passes;        /* correspondence computations the algorithm needed */
    int32_t aa_accepted;        /* Anderson iterates that passed the energy check */
    int32_t reverts;            /* energy checks that failed (revert in Alg. 1, line search in Alg. 2) */
    int32_t line_search_trials; /* Alg. 2 line-search evaluations */
    int32_t stages;             /* nu stages run */
    int32_t device_steps;       /* fused step kernels that did work (>= corr_passes) */
    int32_t trace_len;          /* energies written to the caller's trace buffer */
    int32_t pad0;
    double  nu_max, nu_min;     /* in normalised units (bounding-box diagonal of P u Q = 1) */
    double  final_energy;       /* last accepted energy E_prev */
    double  scale;              /* s of the normalisation x -> s (x - c) */
    double  center[3];          /* c, the centroid of Q */
    double  pass_ms;            /* summed device time of step launches when params.time_passes */
    double  wall_ms;            /* host wall time of the call */
    double  search_ms;          /* part of pass_ms spent in the closest-point search kernel */
} fricp_result;

typedef struct fricp_target fricp_target;

/* Fill `out` with the paper's defaults for `variant` (see fricp_params).
 * Errors: EINVAL for an unknown variant or out == NULL. */
fricp_status fricp_params_default(int32_t variant, fricp_params *out);

/* Build the target set Q once (Sec. 3: Q is fixed over all iterations): copies
 * q_xyz (and q_normals if not NULL; they must be unit length within 1e-3) to
 * the device, builds the exact nearest-neighbour index (Morton-ordered buckets
 * under a complete bounding-box tree, each bucket also bounded by an oriented
 * box along its points' principal axes) and the centroid used by the
 * normalisation. n >= 1. The handle owns all its device memory until
 * fricp_target_destroy. Errors: EINVAL (bad pointer/size/NaN/non-unit normal),
 * ENOMEM, ECUDA. */
fricp_status fricp_target_create(const float *q_xyz, const float *q_normals, int64_t n,
                                 int32_t on_device, void *stream, fricp_target **out);

/* Unit normals of a point set whose surface is unknown, as the paper
 * estimates them for real scans (Sec. 6: from the 30 nearest neighbours;
 * k = 30 reproduces that). The neighbourhood of q_i is its k nearest points
 * of the set, q_i included, ordered by (FP64 squared distance, index); the
 * normal is the unit eigenvector of the smallest eigenvalue of the
 * neighbourhood's covariance about its centroid, turned so that
 * n . (viewpoint - q_i) >= 0 (viewpoint: double[3], NULL = the origin).
 * q_xyz and normals_out: float32 [n][3], both host or both device memory (per
 * on_device). 3 <= k <= 32 (k is capped at n). The result can be passed as
 * q_normals to fricp_target_create. Blocks until the normals are written.
 * Errors: EINVAL (bad pointer/size/k/NaN), ENOMEM, ECUDA. */
fricp_status fricp_estimate_normals(const float *q_xyz, int64_t n, int32_t k, int32_t on_device,
                                    const double *viewpoint, float *normals_out, void *stream);

/* Release a target (NULL is accepted). Waits for work queued on the target's
 * creation stream. */
fricp_status fricp_target_destroy(fricp_target *target);

/* Number of points / whether normals are present. */
int64_t fricp_target_size(const fricp_target *target);
int32_t fricp_target_has_normals(const fricp_target *target);

/* Register source P onto the target (Alg. 1 or Alg. 2 of the paper, after the
 * Sec. 6 normalisation of both sets by one similarity). m >= 1 source points.
 * T0: initial transform (NULL = identity). trace: optional host buffer receiving
 * the accepted energy of every inner iteration (Fig. 2), up to trace_capacity
 * values. Blocks until the result is on the host. Errors: EINVAL, EUNSUPPORTED
 * (point-to-plane without normals), ENOMEM, ECUDA, ETIMEOUT; EDEGENERATE is
 * returned in out->status with FRICP_OK as the call status. */
fricp_status fricp_register(const fricp_target *target, const float *p_xyz, int64_t m,
                            int32_t on_device, const double *T0, const fricp_params *params,
                            void *stream, fricp_result *out, double *trace,
                            int32_t trace_capacity);

/* One correspondence pass of a registration and the decision that followed
 * it, as recorded by fricp_register_recorded (Alg. 1 / Alg. 2; the initial
 * pass that yields nu_max is not recorded). Normalised coordinates. */
typedef struct {
    int32_t step;          /* device step index of the pass (0-based, counting the initial pass) */
    int32_t phase;         /* the pass: 1 stage start (alignment from T^(k-1) with the new nu), 2 energy
                              check at the head of an inner iteration, 3 the pass at T' after a revert
                              (Alg. 1), 4 energy check of the iterate carried out of a stage on the
                              iteration cap, 5 line-search trial (Alg. 2) */
    int32_t revert;        /* 1: the energy check of this pass failed (E >= E_prev): Alg. 1 reverts to
                              T', Alg. 2 starts its line search */
    int32_t accepted;      /* 1: an Anderson iterate passed the energy check */
    int32_t stage;         /* nu stages started so far */
    int32_t done;          /* 1: the registration ended after this pass */
    double  nu;            /* nu of the pass (unused by the non-robust variants) */
    double  E;             /* energy of the pass (Eq. 1, Eq. 9 or Eq. 15) */
    double  E_prev;        /* the accepted energy the pass was compared with (+inf where none) */
    double  T[12];         /* the transform evaluated: R row-major, then t */
    double  xi[6];         /* point-to-plane: the parameter vector evaluated, T = exp(xi); else 0 */
    double  result[12];    /* at this pass: T' of the alignment step (Eq. 4 / Eq. 12; 12 values), or
                              xi* = G_ppl(xi) of the Gauss-Newton step (Eq. 19; 6 values) */
} fricp_step_record;

/* fricp_register that also records every correspondence pass (for checking
 * a registration step by step against a reference). steps: host buffer of
 * steps_capacity records; *steps_len receives the number of passes recorded
 * (at most steps_capacity; later passes are not recorded). Recording adds one
 * alignment solve per pass to the device work. Errors: as fricp_register, and
 * EINVAL for a NULL steps buffer with steps_capacity > 0. */
fricp_status fricp_register_recorded(const fricp_target *target, const float *p_xyz, int64_t m,
                                     int32_t on_device, const double *T0, const fricp_params *params,
                                     void *stream, fricp_result *out, double *trace,
                                     int32_t trace_capacity, fricp_step_record *steps,
                                     int32_t steps_capacity, int32_t *steps_len);

/* The Welsch-robust symmetric objective, the extension the paper proposes in
 * Sec. 7 (replacing symmetric ICP's l2 target with a robust metric): Alg. 2
 * (Gauss-Newton on the App. D parameterisation, Anderson step, line search,
 * nu stages) on the residual H_i = (R p_i + t - q_i) . (R np_i + nq_i) of each
 * source point and its closest target point, where np_i is the source point's
 * unit normal (moved with the source) and nq_i the target's. Welsch weights and
 * energy on H_i; nu_max = 3 x median |H_i| at T0, nu_min = H_Q / 6 as for
 * point-to-plane (Sec. 5). params->variant must be FRICP_SYM_WELSCH_AA; the
 * target needs normals. p_normals: float32 [m][3] in p_xyz's memory space,
 * each a unit normal (within 1e-3) or zero for a point without a normal, whose
 * residual is then the point-to-plane one (with every np_i zero the
 * registration is FRICP_P2PL_WELSCH_AA's, bit for bit). Other arguments as
 * fricp_register_recorded (steps may be NULL with steps_capacity 0). The
 * batched and served engines do not run this variant.
 * Errors: as fricp_register; EINVAL for a source normal neither zero nor unit. */
fricp_status fricp_register_symmetric(const fricp_target *target, const float *p_xyz, const float *p_normals,
                                      int64_t m, int32_t on_device, const double *T0,
                                      const fricp_params *params, void *stream, fricp_result *out,
                                      double *trace, int32_t trace_capacity, fricp_step_record *steps,
                                      int32_t steps_capacity, int32_t *steps_len);

/* Batched registration (no counterpart in the paper, which registers one pair
 * at a time): npairs independent registrations -- pair i registers p_xyz[i]
 * (m[i] points, host or device per on_device) onto targets[i] with params[i]
 * (variants may differ) from T0[16*i .. 16*i+15] (T0 == NULL: identity for
 * all) -- advance together, one device step for all unfinished pairs per set of
 * launches (plan, search, accumulate/solve), replayed from a CUDA graph of
 * params[0].steps_per_sync steps. Each pair's result equals, bit for bit, what
 * fricp_register returns for it alone. The launch shape of the search (queries
 * per work ticket, blocks per SM) is chosen by timing candidates on the batch's
 * first pass and remembered per size class (see fricp_batch_last_shape).
 * Loop controls (use_graph, steps_per_sync, max_steps, timeout_s) come from
 * params[0]; time_passes is ignored. out: npairs results (wall_ms is the whole
 * call's). trace: NULL or npairs * trace_capacity doubles, pair i's energies at
 * trace[i * trace_capacity]. 1 <= npairs <= 4096. Blocks until every result is
 * on the host. Errors: as fricp_register, with the failing pair named in the
 * message; per-pair EDEGENERATE is returned in out[i].status. */
fricp_status fricp_batch_register(int32_t npairs, const fricp_target *const *targets,
                                  const float *const *p_xyz, const int64_t *m, int32_t on_device,
                                  const double *T0, const fricp_params *params, void *stream,
                                  fricp_result *out, double *trace, int32_t trace_capacity);

/* Fix the launch shape of later batched and served runs on every thread
 * instead of autotuning it: chunk queries per search ticket (a divisor of 256),
 * search blocks per SM (clamped to the kernel's occupancy) and the ticket
 * order: 0 = from an atomic counter, one query per warp; 1 = dealt in a fixed
 * stride, one query per warp; 2 = query tiles (tickets of 8 Morton-adjacent
 * queries searched together by a warp, see FRICP_SEARCH_TILE; chunk is then
 * 8). chunk = 0 returns to autotuning. The results do not depend on the shape,
 * only the time. Errors: EINVAL. */
fricp_status fricp_batch_set_shape(int32_t chunk, int32_t search_blocks_per_sm, int32_t static_order);

/* Launch shape the autotuner chose for the last batched or served run on any
 * thread: queries per search ticket, search blocks per SM, accumulate blocks
 * per SM, and the ticket order (0 counter, 1 fixed stride, 2 query tiles, as
 * in fricp_batch_set_shape). Any pointer may be NULL. Never fails. */
void fricp_batch_last_shape(int32_t *chunk, int32_t *search_blocks_per_sm,
                            int32_t *accumulate_blocks_per_sm, int32_t *static_order);

/* Serving loop with continuous batching (no counterpart in the paper).
 * Registrations are submitted at any time; fricp_server_step admits queued
 * requests in FIFO order while a slot is free and their device buffers fit in
 * the server's HBM budget, keeps each admitted request's state, correspondences
 * and packed source resident on the device, and advances all of them together
 * with the batched step of fricp_batch_register (one CUDA graph of
 * steps_per_sync steps per replay). Admission work (staging, Morton sort,
 * nu statistics) runs on a second stream while the step graph replays. Each
 * served result equals, bit for bit, what fricp_register returns for the same
 * request alone. A handle is used by one thread at a time (calls are also
 * serialised internally). */
typedef struct fricp_server fricp_server;

/* hbm_budget: bytes of device memory the requests in flight may hold (0 = half
 * of the free device memory): a request's own buffers (28 B per source point,
 * 224 B per 256 points and one solver state of a few KB) and the index of its
 * target (16 B per point, 16 more with normals, 128 B per bucket of 16 for its
 * axis-aligned and oriented boxes, 8 B per point of FP16 storage), a target
 * counted once however many requests in
 * flight share it. Requests are admitted in FIFO order while a slot is free
 * and the budget holds them. max_slots: requests in flight at most
 * (1..4096). steps_per_sync: device steps per graph replay. max_queue:
 * requests waiting for admission at most. stream: submits of device sources
 * are ordered after the work queued on it. Errors: EINVAL, ENOMEM, ECUDA. */
fricp_status fricp_server_create(size_t hbm_budget, int32_t max_slots, int32_t steps_per_sync,
                                 int32_t max_queue, void *stream, fricp_server **out);

/* Queue a registration (arguments as fricp_register, without the trace). The
 * source is copied (host memory to a host buffer; device memory to a library
 * device buffer, ordered after the server's stream), so the caller may reuse
 * p_xyz at once; the target must stay alive until the request's result has
 * been polled. Never blocks on the GPU. *ticket identifies the request.
 * Errors: EINVAL (as fricp_register, or a request that with its target is
 * larger than the budget),
 * EUNSUPPORTED, ENOMEM, ECUDA; EBUSY when max_queue requests are waiting. */
fricp_status fricp_server_submit(fricp_server *server, const fricp_target *target, const float *p_xyz,
                                 int64_t m, int32_t on_device, const double *T0,
                                 const fricp_params *params, uint64_t *ticket);

/* Run about nsteps device steps (rounded up to whole graph replays) for every
 * request in flight, admit what fits from the queue (overlapping the steps),
 * and collect the requests that finished. Blocks until the steps are done.
 * in_flight / queued (may be NULL): counts after the call. A request whose
 * admission fails (bad data found on the device, out of memory) finishes with
 * that status in its result; the server carries on. Errors: EINVAL, ECUDA,
 * ETIMEOUT. */
fricp_status fricp_server_step(fricp_server *server, int32_t nsteps, int32_t *in_flight, int32_t *queued);

/* *done = 1 and *out filled (once) when the request has finished, else
 * *done = 0. Errors: EINVAL (NULL or a ticket never issued). */
fricp_status fricp_server_poll(fricp_server *server, uint64_t ticket, fricp_result *out, int32_t *done);

/* Wait for the server's work, free everything it holds (NULL is accepted). */
fricp_status fricp_server_destroy(fricp_server *server);

/* The correspondence step alone (Sec. 3, Eq. 3): for every x_i = R p_i + t
 * (T: double[16] row-major, NULL = identity; p_xyz device float32 [m][3]),
 * the index of its closest target point (original order of Q; ties to the
 * lowest index) and the squared distance, recomputed in FP64. idx_out and
 * d2_out are device arrays of m entries. Asynchronous on `stream`.
 * Errors: EINVAL, ECUDA. */
fricp_status fricp_closest_points(const fricp_target *target, const float *p_xyz, int64_t m,
                                  const double *T, int64_t *idx_out, double *d2_out,
                                  void *stream);

/* One fused correspondence pass at a fixed transform, reduced on the device and
 * returned to the host: the quantities one iteration of Alg. 1 / Alg. 2 consumes.
 *   variant P2P_AA / P2P_WELSCH_AA: out[0] = E (sum D_i^2, resp. sum psi_nu(D_i),
 *     Eq. 1 / Eq. 9), out[1..9] = R' row-major and out[10..12] = t' of the
 *     alignment step (Eq. 4 / Eq. 12).
 *   variant P2PL_WELSCH_AA: out[0] = E~ (sum psi_nu(H_i), Eq. 15),
 *     out[1..6] = xi* = G_ppl(xi) (Eq. 19) for xi = log(T) = [delta; u].
 *   variant P2PL_AA: as P2PL_WELSCH_AA with weights 1 and out[0] = sum H_i^2.
 *   out[16..43]: the reduced FP64 sums of the pass. Point-to-point (17 values):
 *     sum w, sum w p~ (3), sum w q~ (3), sum w p~ q~^T (9, row-major), E, with
 *     p~ = p - center, q~ = q - center in the caller's units. Point-to-plane
 *     (28 values): the upper triangle of sum g z z^T row by row (21), sum g z B
 *     (6), E, with z = [R p_n x n; n] in normalised units (App. D: J = K z).
 * T_normalized (double[16], row-major), nu and every output are in the
 * normalised coordinates x -> scale (x - center); pass scale = 1 and center =
 * NULL for the caller's coordinates. p_xyz: float32 [m][3] (host or device per
 * on_device). Blocks until `out` (48 doubles) is filled. Errors: EINVAL,
 * EUNSUPPORTED, EDEGENERATE, ENOMEM, ECUDA. */
fricp_status fricp_eval_pass(const fricp_target *target, const float *p_xyz, int64_t m,
                             int32_t on_device, int32_t variant, const double *T_normalized,
                             double nu, double scale, const double *center, void *stream,
                             double *out);

/* No counterpart in the paper: fricp_eval_pass for callers that cannot
 * allocate device memory -- a caller that has already handed the whole device
 * to another allocator (a framework's caching allocator), a latency-critical
 * loop in which cudaMalloc / cudaFree would synchronize the device, or a
 * real-time or certified deployment that forbids allocation after start-up.
 * Same arguments and the same 48 outputs as fricp_eval_pass, except:
 *   - p_xyz_dev is device memory (float32 [m][3]) and 1 <= m <= 32768; a larger
 *     m returns FRICP_EINVAL with a message saying so;
 *   - the pass takes the source points in the caller's order (no Morton sort),
 *     so FP64 sums may differ from fricp_eval_pass in the last bits;
 *   - its scratch (solver state, tile records, correspondences, packed points)
 *     is one static device array of about 0.7 MB that every GPU which loads the
 *     library keeps until the process exits. The call makes no cudaMalloc,
 *     cudaFree or other allocating call.
 * The first call on a device looks up the array's device address (set-up, once
 * per device, with that device current; the cached address does not survive
 * cudaDeviceReset). Every call copies its inputs from host memory and waits for
 * its stream, so no call can be captured into a CUDA graph. All calls share
 * the one array and it keeps the last call's
 * contents; each call rewrites everything it reads, but calls that overlap on
 * the GPU (different streams or threads) race on it: issue them one after
 * another. Blocks until `out` is filled. Errors: EINVAL, EUNSUPPORTED,
 * EDEGENERATE, ECUDA. */
fricp_status fricp_eval_pass_static(const fricp_target *target, const float *p_xyz_dev, int64_t m,
                                    int32_t variant, const double *T_normalized, double nu,
                                    double scale, const double *center, void *stream, double *out);

/* The nu rules alone, in normalised units for the given scale (Sec. 4.3, Sec. 5,
 * App. C): nu_min from the six nearest neighbours of every target point. */
fricp_status fricp_target_nu_min(const fricp_target *target, int32_t variant, double scale,
                                 void *stream, double *nu_min_out);

/* Accounting of the calls made on this thread since the last reset: kernel
 * launches issued by libfricp (each replayed graph node counts once, and each
 * radix sort counts the launches it issues) and bytes copied host->device and
 * device->host. Any pointer may be NULL. reset != 0 zeroes the counters after
 * reading them. Never fails. */
void fricp_counters(int64_t *kernel_launches, int64_t *h2d_bytes, int64_t *d2h_bytes, int32_t reset);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char *fricp_last_error(void);

/* ABI version: (major << 16) | minor. */
int32_t fricp_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FRICP_H */
