/*
 * libpradmm -- C ABI of a GB300 (sm_103a) implementation of PRADMM, the
 * parallelizable Riemannian ADMM for non-convex pose graph optimization
 * (Chen, Cui, Han, Qi, arXiv 2601.15684).
 *
 * The problem (Section 2, Eq. (1)): a directed graph of n poses
 * (q_i unit quaternion, t_i in R^3) and m relative measurements
 * (q_ij, t_ij) on edges (i, j); minimise
 *   F = sum_{(i,j)} omega_e |t~_j - t~_i - q_i t~_ij q_i^*|^2
 *                 + kappa_e |q_j^* q_i q_ij - 1|^2 ,  q_i in U (unit sphere),
 * where t~ = [0, t] and Sigma_1 = omega_e I_4, Sigma_2 = kappa_e I_4 are
 * per-edge scalar weights.  The solver runs the PRADMM iteration of
 * Section 3.2 Eq. (3a)-(3f) / Algorithm 1 on the split model (2): closed-form
 * per-vertex updates of the rotation copy p (projection onto S^3), the
 * quaternion copy q, the translations t and s (Appendix B), the relaxed
 * multiplier updates with step tau in (0,2), and the residual e^k of
 * Appendix E.1 with the stopping test e^k < tol.
 *
 * Conventions
 *  - Quaternions are scalar first, [q0, q1, q2, q3] (Appendix A.2).
 *  - Arrays are row major and C contiguous: an "n x 4" array holds
 *    q_0[0..3], q_1[0..3], ...
 *  - Vertex indices are int32 in [0, n); self-loops are rejected; repeated
 *    edges are allowed and summed.
 *  - Unless a name ends in _device, pointers are HOST memory.  The library
 *    copies every input it is given and owns all device memory it allocates;
 *    callers own their buffers.
 *  - All GPU work of a handle runs on the CUDA stream given to create (NULL:
 *    the library makes a private non-blocking stream).  Calls on one handle
 *    are not thread safe; distinct handles are independent.
 *  - No function aborts or prints.  Each returns a status; after a failure
 *    pradmm_last_error() gives a one-line message for the calling thread.
 *  - Precision: PRADMM_FP64 runs everything in double.  PRADMM_FP32 keeps the
 *    pose state and bulk arithmetic in float, and does the residual, the
 *    stopping test, the objective and the fallback of the p-update in double.
 *
 * Readings of passages the paper leaves open (also used by the test oracle):
 *  - the in-edge matrix of the p-subproblem is W(q_li) W(q_l) D (Appendix B.1
 *    prints it without D, which would make noise-free ground truth not a
 *    fixed point);
 *  - c_e = Im(q_tail t~_e p_tail^*) for an edge e = (tail, head)
 *    (Appendix B.3 prints garbled indices);
 *  - proximal anchors x^{k+1/2} of Appendix B are x^k, or with a nonzero
 *    pradmm_params.inertia theta the extrapolated x^k + theta (x^k - x^{k-1})
 *    (the inertial variant; the paper gives no rule for x^{k+1/2});
 *  - e^{k+1} = |dlambda|^2/beta1 + |dz|^2/beta2 + beta1 |dq|^2 + beta2 |dt|^2
 *    (Appendix E.1 uses a single beta);
 *  - lambda^0 = z^0 = 0, p^0 = q^0, s^0 = t^0;
 *  - if |u_i| = 0 in the p-update (p = u/|u| = -b_1/|b_1|, Section 3.3) the
 *    vertex keeps p_i^k.
 */
#ifndef PRADMM_H
#define PRADMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pradmm_s* pradmm_t;

typedef enum {
    PRADMM_OK = 0,
    PRADMM_ERR_ARG = 1,            /* null pointer, bad size or bad parameter   */
    PRADMM_ERR_INDEX = 2,          /* edge endpoint outside [0, n)              */
    PRADMM_ERR_SELFLOOP = 3,       /* edge (i, i)                               */
    PRADMM_ERR_NONFINITE = 4,      /* NaN/Inf in an input or in the iteration  */
    PRADMM_ERR_NOMEM = 5,          /* host or device allocation failed          */
    PRADMM_ERR_CUDA = 6,           /* a CUDA runtime call failed                */
    PRADMM_ERR_TIMEOUT = 7,        /* reserved: no call returns it (the library
                                      has no device-side waits)                */
    PRADMM_ERR_NOT_CONVERGED = 8,  /* solve hit max_iter with e >= tol (state valid) */
    PRADMM_ERR_QUATERNION = 9,     /* |q_meas| differs from 1 by more than 1e-6 */
    PRADMM_ERR_STATE = 10          /* operation needs a state that was never set */
} pradmm_status;

enum { PRADMM_FP64 = 0, PRADMM_FP32 = 1 };

typedef struct {
    double beta1;        /* penalty beta_1 of the p = q constraint (Section 3.2)   */
    double beta2;        /* penalty beta_2 of the t = s constraint                 */
    double relax;        /* relaxed dual step tau in (0, 2), Eq. (3e)-(3f)         */
    double gamma[4];     /* proximal weights: H_s = gamma[s-1] I, s = 1..4         */
    double tol;          /* stop when e^k < tol (Appendix E.1)                     */
    int32_t max_iter;    /* iteration cap of pradmm_solve                          */
    int32_t precision;   /* PRADMM_FP64 or PRADMM_FP32                             */
    double fallback_eps; /* FP32: recompute u_i in FP64 when |u_i| < eps (beta1+gamma1) */
    int32_t use_graph;   /* 1: loop inside a CUDA graph with a device-side while node;
                            0: plain stream launches                               */
    int32_t block;       /* threads per CTA of the sweeps: a multiple of 32 in
                            [32, 256], or 0: 256, halved (to 32 at least) while
                            n / block is below half the number of SMs         */
    int32_t l2_window;   /* 1: the sweep launches mark the vertex arrays they
                            gather (t, s, q, both p buffers; one contiguous block)
                            as persisting in L2, and the library sets aside that
                            much L2 for the process while a handle using it
                            lives (restored when the last one is destroyed);
                            0: plain caching                                       */
    int32_t reserved;    /* 0 */
    double inertia;      /* theta in [0, 1) of the inertial variant: the proximal
                            anchors of p, q, t, s are x^k + theta (x^k - x^{k-1})
                            (the paper's x^{k+1/2}, Appendix B; the extrapolation
                            rule is this library's reading); 0 (default) is plain
                            PRADMM.  A nonzero theta works with scalar and
                            general weights (pradmm_set_sigma), in the batched
                            form (each pradmm_batch_solve starts the
                            extrapolation afresh) and in the reverse mode
                            (scalar weights; the recording starts afresh);
                            setting a state or the weights restarts the
                            extrapolation (x^{k-1} := x^k). */
} pradmm_params;

/* Defaults: beta1 = beta2 = 1, relax = 1.5, gamma = {1, 1e-3, 1e-3, 1e-3},
 * tol = 1e-4, max_iter = 300 (Section 5 settings; beta is not given in the
 * paper and is fixed here by a sweep on the 128-pose walk), FP32,
 * fallback_eps = 1e-6, use_graph = 1, block = 0, l2_window = 1. */
void pradmm_default_params(pradmm_params* prm);

/* Builds a solver for one pose graph (Section 2): uploads the arrays on
 * `cuda_stream` (a cudaStream_t or NULL), validates the edges on the device
 * before anything indexes with them (ERR_INDEX, ERR_SELFLOOP, ERR_NONFINITE for
 * non-finite measurements or weights, ERR_ARG for weights <= 0,
 * ERR_QUATERNION; the error names the first failing edge in input order),
 * renormalises q_meas, sorts the edges by tail and by head, finds the
 * spanning forest of pradmm_init_odometry (from the endpoints, while the
 * measurements upload on a second stream) and packs structure-of-arrays
 * device buffers.
 *   src, dst     m int32 edge endpoints (tail i, head j)
 *   q_meas       m x 4 relative rotations q_ij
 *   t_meas       m x 3 relative translations t_ij
 *   kappa, omega m per-edge weights (> 0); NULL means all ones
 * n >= 1, m >= 0.  The state is unset until pradmm_set_state* or
 * pradmm_init_odometry.  On failure *out is NULL. */
pradmm_status pradmm_create(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                            const double* q_meas, const double* t_meas, const double* kappa,
                            const double* omega, const pradmm_params* prm, void* cuda_stream,
                            pradmm_t* out);

/* Same as pradmm_create with every array in device memory (e.g. torch
 * tensors): `cuda_stream` (NULL: the legacy default stream) is synchronised
 * first, so work queued there that writes the arrays is finished; they are
 * then copied device to device on the handle's stream and validated there,
 * all before return. */
pradmm_status pradmm_create_device(int64_t n, int64_t m, const int32_t* src_d, const int32_t* dst_d,
                                   const double* q_meas_d, const double* t_meas_d,
                                   const double* kappa_d, const double* omega_d,
                                   const pradmm_params* prm, void* cuda_stream, pradmm_t* out);

/* Initial point of Algorithm 1 from poses (q: n x 4, t: n x 3):
 * p = q, s = t, lambda = z = 0 (reading of the unspecified initial multipliers). */
pradmm_status pradmm_set_state(pradmm_t h, const double* q, const double* t);

/* Full ADMM state (checkpoint/resume): p, q, lam n x 4; t, s, z n x 3. */
pradmm_status pradmm_set_state_full(pradmm_t h, const double* p, const double* q, const double* t,
                                    const double* s, const double* lam, const double* z);

/* pradmm_set_state_full from device arrays (double, same shapes; lam and z
 * may be NULL for zero multipliers).  The arrays are read on the handle's
 * stream, so the caller's writes must be complete or ordered before the
 * call; they are copied, not kept.  Finiteness is not checked on the host: a
 * non-finite entry surfaces as PRADMM_ERR_NONFINITE from the next iteration.
 * Like every state set, it restarts the inertial extrapolation. */
pradmm_status pradmm_set_state_full_device(pradmm_t h, const double* p_d, const double* q_d, const double* t_d,
                                           const double* s_d, const double* lam_d, const double* z_d);

/* Initial poses by odometry composition along a spanning forest: edges are
 * taken in input order, an edge joins the forest when it links two
 * components, the lowest vertex of each component gets the identity, and the
 * others follow q_j = q_i q_ij, t_j = t_i + R(q_i) t_ij (Section 2).  Then as
 * pradmm_set_state.  (The paper starts from a chordal initialisation it does
 * not define.)  The forest is found by pradmm_create; this call composes the
 * poses along it on the device, in FP64. */
pradmm_status pradmm_init_odometry(pradmm_t h);

/* The spanning forest of pradmm_init_odometry, copied to host arrays of n
 * int32 each: parent[v] is v's forest parent (-1 for the root of a
 * component, its lowest vertex); pedge[v] the forest edge e joining v to it,
 * coded e when v is the edge's head (dst[e] == v) and -(e + 2) when v is its
 * tail (src[e] == v), -1 for a root.  Edge indices are input order.  NULL
 * arguments are ERR_ARG.  Synchronises the handle's stream. */
pradmm_status pradmm_odometry_forest(pradmm_t h, int32_t* parent, int32_t* pedge);

/* Schedule search: times `iters` >= 1 iterations from the current state at
 * each CTA size of the sweeps (32, 64, 128 and 256 threads; a thread per
 * vertex), keeps the fastest and restores the state as
 * pradmm_set_state_full would (the iteration count and the inertial
 * extrapolation restart).  The iterates do not depend on the CTA size (each
 * vertex sums its edges in the same order); the residual's reduction tree
 * does, in its last bits.  block_out (nullable) receives the choice.
 * PRADMM_ERR_STATE before a state is set. */
pradmm_status pradmm_autotune(pradmm_t h, int32_t iters, int32_t* block_out);

/* Runs `iters` >= 0 iterations of Algorithm 1 (no stopping test).
 * e_last (nullable) receives e^k of the last iteration. */
pradmm_status pradmm_step(pradmm_t h, int32_t iters, double* e_last);

/* Runs Algorithm 1 until e^k < prm.tol or prm.max_iter iterations of this call.
 * Returns PRADMM_OK on convergence, PRADMM_ERR_NOT_CONVERGED otherwise (the
 * state stays valid).  iters_done, e_final are nullable. */
pradmm_status pradmm_solve(pradmm_t h, int32_t* iters_done, double* e_final);

/* F of Eq. (1) at (p, t) in double precision (Appendix E.1 reports p, since
 * |q_i| != 1 during the iteration). */
pradmm_status pradmm_objective(pradmm_t h, double* F);

/* Copies the state to host arrays (any pointer may be NULL):
 * p, q, lam n x 4; t, s, z n x 3. */
pradmm_status pradmm_get_state(pradmm_t h, double* p, double* q, double* t, double* s, double* lam,
                               double* z);

/* Same with device destination arrays (double, same shapes). */
pradmm_status pradmm_get_state_device(pradmm_t h, double* p, double* q, double* t, double* s,
                                      double* lam, double* z);

/* Output of Algorithm 1: rotations p (n x 4, unit) and translations t (n x 3). */
pradmm_status pradmm_get_poses(pradmm_t h, double* q_out, double* t_out);

/* Iterations run since the state was last set. */
int64_t pradmm_iterations(pradmm_t h);

/* Index-checked builds (libpradmm_debug.so, compiled with
 * PRADMM_DEBUG_CHECKS): every neighbour index and CSR row bound the plain
 * sweeps read is range-checked on the device; an out-of-range value is
 * counted, replaced by 0 so the access stays in bounds, and the run returns
 * PRADMM_ERR_INDEX.  No counterpart in the paper: a test hook that writes
 * `value` (in [0, n], where n itself is out of range) into out-edge slot
 * `slot` of the device CSR, to check that the checks fire.  The release
 * library returns PRADMM_ERR_STATE.  PRADMM_ERR_ARG for a slot outside [0, m)
 * or a value outside [0, n]. */
pradmm_status pradmm_debug_set_neighbour(pradmm_t h, int64_t slot, int32_t value);

/* Per-iteration residual trace (Appendix E.1's e^k in FP64, the value the
 * stopping test of Algorithm 1 reads).  capacity > 0: from now on every
 * iteration the handle runs (step, solve, the reverse mode's recording)
 * writes its e^k into a device ring of `capacity` doubles, entry
 * (k - 1) % capacity for iteration k, with no host round trip; capacity 0
 * turns the trace off and frees the ring.  The handle owns the ring.  Setting
 * the state restarts the count.  Errors: PRADMM_ERR_ARG (capacity < 0),
 * PRADMM_ERR_NOMEM. */
pradmm_status pradmm_set_trace(pradmm_t h, int32_t capacity);

/* The traced residuals, oldest first: *count = min(iterations since the trace
 * started or the state was set, capacity) values into host e_out (room for
 * `capacity` doubles), *first_iter (nullable) = the iteration number k of
 * e_out[0] (iterations are numbered from 1 after a state set).
 * PRADMM_ERR_STATE if no trace is on. */
pradmm_status pradmm_get_trace(pradmm_t h, double* e_out, int64_t* first_iter, int32_t* count);

/* Counters: [0] p-updates recomputed in FP64, [1] p-updates with |u| = 0
 * that kept p^k, [2] iterations, [3] stop flag.  out has 4 entries. */
pradmm_status pradmm_counters(pradmm_t h, int64_t* out);

/* Algorithmic bytes of one iteration and of each sweep kernel under the
 * byte model of the library's roofline report (FP32 words of every array a
 * sweep needs, counted once per sweep):
 *   out[0] total, out[1] q/lambda sweep, out[2] t sweep, out[3] s/z + next p sweep. */
pradmm_status pradmm_bytes_per_iteration(pradmm_t h, double* out);

/* L2 persistence of the handle (params.l2_window): out[0] window bytes (0 if
 * off), out[1] its hit ratio, out[2] the process's current L2 set-aside bytes. */
pradmm_status pradmm_l2_window_info(pradmm_t h, double* out);

/* Times `iters` iterations launched kernel by kernel on the handle's stream
 * with CUDA events around each sweep kernel; ms_out[0..2] receive the mean
 * duration (ms) of the q/lambda, t and s/z+p kernels, ms_out[3] the mean
 * iteration time.  The state advances by `iters` iterations. */
pradmm_status pradmm_profile_sweeps(pradmm_t h, int32_t iters, double* ms_out);

/* The same launches, every iteration's durations kept: per_iter_ms (host,
 * 4 x iters, row k for the k-th profiled iteration) receives the q/lambda,
 * t and s/z+p kernel times and the iteration time (ms).  The state advances
 * by `iters` iterations. */
pradmm_status pradmm_profile_iterations(pradmm_t h, int32_t iters, double* per_iter_ms);

/* General weight matrices (Lemma 1, Algorithm 1's branch for non-scalar
 * Sigma): edge e weighs its translation residual with omega_e Sigma1 and its
 * rotation residual with kappa_e Sigma2, Sigma1 and Sigma2 symmetric positive
 * definite 4x4 (row-major, 16 doubles each, copied).  The p-update then solves
 * min_{|p|=1} 1/2 p^T A_1 p + b_1^T p per vertex through the eigen-
 * decomposition of A_1 and the secular equation of Lemma 1 (hard case
 * included: of the two minimisers the one closer to p^k is kept); FP32
 * handles repeat that solve in FP64 when the eigen-gap or the component of
 * b_1 on the bottom eigenvector is tiny (counted in pradmm_counters out[0]).
 * The q, t and s blocks solve 4x4 / 3x3 systems.  Both NULL returns to the
 * scalar model (Sigma = I).  PRADMM_ERR_ARG if only one is given or one is
 * not symmetric positive definite, PRADMM_ERR_NONFINITE for non-finite
 * entries.  Keeps the state (the next iteration recomputes p^{k+1}) and,
 * with a nonzero inertia, restarts the extrapolation; the reverse mode and
 * pradmm_profile_sweeps need the scalar model. */
pradmm_status pradmm_set_sigma(pradmm_t h, const double* Sigma1, const double* Sigma2);

/* ---- reverse mode -------------------------------------------------------------
 * Gradients of a loss L(p^K, t^K) of the poses after K iterations of
 * Algorithm 1 with respect to the measurements q_e, t_e and the weights
 * kappa_e, omega_e of Eq. (1), through the unrolled iterations (3a)-(3f)
 * with the closed forms of Appendix B.  The starting state x^0 is held fixed
 * (its own dependence on the measurements, e.g. through odometry, is not
 * differentiated); its adjoint is available as an output.  q_e is treated as
 * a point of R^4: the gradient is not projected onto the tangent space of
 * the unit sphere.  Where a p-update met |u_i| = 0 and kept p_i^k, the
 * adjoint of p_i^{k+1} passes to p_i^k.  Derivatives of A_2 with respect to
 * p are dropped: they point along p and the sphere projection removes them.
 *
 * pradmm_adjoint_record runs `iters` iterations from the current state x^0
 * (like pradmm_step) and keeps a checkpoint of the full state every
 * `ckpt_every` iterations (device memory for ceil(iters/ckpt_every)+1
 * checkpoints plus ckpt_every-1 recompute slots, 28 n reals each).
 * ckpt_every = 0 chooses the spacing from the device memory: the smallest
 * one whose tape fits in half of the free memory (1 where it fits: every
 * iterate is kept and the reverse pass recomputes nothing); negative values
 * return PRADMM_ERR_ARG.  With a nonzero inertia the recording restarts the
 * extrapolation (x^{-1} := x^0, whose adjoint then holds both shares); with
 * a spacing above 1 each slot also keeps x^{k-1} (q, t, s and p: 44 n reals
 * a slot), with spacing 1 the previous slot holds it.  The tape stays valid until the state changes
 * (set_state, init_odometry, step, solve, another record). */
pradmm_status pradmm_adjoint_record(pradmm_t h, int32_t iters, int32_t ckpt_every);

/* The checkpoint spacing and the tape's device bytes of the current
 * recording (PRADMM_ERR_STATE if there is none).  Either pointer may be
 * NULL. */
pradmm_status pradmm_adjoint_tape_info(pradmm_t h, int32_t* ckpt_every, double* tape_bytes);

/* Runs the reverse sweeps over the recorded iterations for the cotangent
 * (p_bar = dL/dp^K, n x 4; t_bar = dL/dt^K, n x 3; NULL means zero) and
 * writes, in the caller's edge order, dL/dq_meas (m x 4), dL/dt_meas (m x 3),
 * dL/dkappa (m), dL/domega (m), and, if x0_bar is not NULL, the adjoint of
 * x^0 as 21 n doubles: p (n x 4), q (n x 4), t (n x 3), s (n x 3),
 * lam (n x 4), z (n x 3).  Any output pointer may be NULL.  Segments between
 * checkpoints are recomputed with the forward sweep kernels, bitwise as
 * recorded.  The tape stays valid, so several cotangents may be run. */
pradmm_status pradmm_adjoint(pradmm_t h, const double* p_bar, const double* t_bar, double* q_meas_bar,
                             double* t_meas_bar, double* kappa_bar, double* omega_bar, double* x0_bar);

/* Same with every array in device memory (double).  The work runs on the
 * handle's stream and has finished when the call returns. */
pradmm_status pradmm_adjoint_device(pradmm_t h, const double* p_bar_d, const double* t_bar_d,
                                    double* q_meas_bar_d, double* t_meas_bar_d, double* kappa_bar_d,
                                    double* omega_bar_d, double* x0_bar_d);

/* F of Eq. (1) for poses already in device memory, written to the device
 * double *F_d, without allocating any memory.  There is no counterpart in the
 * paper: it serves callers that cannot allocate device memory when they need
 * the objective (for example a real-time process that reserves all of its GPU
 * memory at start-up and forbids allocation afterwards, since an allocation
 * can synchronise the device and stall the loop), and that therefore cannot
 * create a handle.
 *   src_d, dst_d     m int32 edge endpoints in [0, n); an edge with an
 *                    endpoint outside [0, n) reads no pose and makes *F_d NaN
 *   q_meas_d         m x 4 relative rotations (used as given, not renormalised)
 *   t_meas_d         m x 3 relative translations
 *   kappa_d, omega_d m weights, or NULL for all ones
 *   q_d, t_d         n x 4 rotations and n x 3 translations to evaluate
 *   F_d              one double, written on `cuda_stream`
 * All pointers are device memory; the call is asynchronous on cuda_stream.
 * Scratch: one FP64 partial per chunk of 1024 edges and a counter live in a
 * 32 KiB static device array, part of the library's device code; m above
 * 4,194,304 is rejected with PRADMM_ERR_ARG.  A GPU receives that array when
 * the library's device code is loaded onto it and keeps it until process
 * exit.  Under CUDA's lazy module loading (the default) that load happens at
 * the first call on the GPU, and loading allocates device memory and may
 * synchronise: make the first call on each GPU at start-up, before any
 * stream capture (it also looks up the array's device address with the
 * device current).  Later calls allocate nothing.  Every call on
 * a device shares that device's array and leaves its contents behind, so
 * calls that may overlap on the same GPU (for example on different streams)
 * race: serialise them.  Each call clears the counter before its kernel
 * runs and rewrites every partial it reads. */
pradmm_status pradmm_objective_noalloc(int64_t n, int64_t m, const int32_t* src_d, const int32_t* dst_d,
                                       const double* q_meas_d, const double* t_meas_d,
                                       const double* kappa_d, const double* omega_d, const double* q_d,
                                       const double* t_d, double* F_d, void* cuda_stream);

/* Frees every resource of the handle (NULL is a no-op). */
void pradmm_destroy(pradmm_t h);

const char* pradmm_status_string(pradmm_status st);

/* Message of the last failure on the calling thread ("" if none). */
const char* pradmm_last_error(void);

/* ---- batched solver ---------------------------------------------------------
 * Many independent pose graphs (each a problem of the form of Eq. (1)) solved
 * by Algorithm 1 in one persistent launch captured in a CUDA graph.  The batch
 * is stored as one disjoint-union graph; a work queue ordered largest first
 * gives each large graph a whole CTA and packs small graphs one per warp.
 * Each graph stops on its own: when e^k <= rel_tol * e^1 (the ratio of its
 * Appendix E.1 residual to the first iteration's), when e^k is not finite,
 * or after max_iter iterations.  A graph's results agree with the plain
 * solver run for the same number of iterations to rounding (the same
 * per-vertex updates, compiled into a different kernel), and a repeated
 * solve is bitwise identical. */
typedef struct pradmm_batch_s* pradmm_batch_t;

/* G graphs; graph g has n_g[g] >= 1 vertices and m_g[g] >= 0 edges.  Edge
 * arrays are concatenated in graph order with GRAPH-LOCAL endpoints in
 * [0, n_g[g]); layouts and validation as pradmm_create.  The schedule starts
 * at block 256, warp_max_n 256, no clusters.  prm->inertia applies to every
 * graph (the inertial variant; each solve starts with x^{-1} = x^0). */
pradmm_status pradmm_batch_create(int32_t G, const int64_t* n_g, const int64_t* m_g, const int32_t* src,
                                  const int32_t* dst, const double* q_meas, const double* t_meas,
                                  const double* kappa, const double* omega, const pradmm_params* prm,
                                  void* cuda_stream, pradmm_batch_t* out);

/* Schedule: `block` threads per CTA of the persistent kernel (64, 128, 256,
 * 512); graphs with at most warp_max_n vertices are solved one per warp,
 * larger ones one per CTA.  With `cluster` = 2, 4 or 8, graphs with more than
 * cluster_min_n vertices are solved by a thread-block cluster of that many
 * CTAs (the hardware co-schedules them; the sweeps of an iteration are
 * separated by cluster barriers and the residual parts are exchanged through
 * distributed shared memory); cluster = 1 uses no clusters.  PRADMM_ERR_ARG
 * if a value is out of range or no cluster of that shape fits the GPU. */
pradmm_status pradmm_batch_set_schedule(pradmm_batch_t b, int32_t block, int32_t warp_max_n, int32_t cluster,
                                        int32_t cluster_min_n);
pradmm_status pradmm_batch_get_schedule(pradmm_batch_t b, int32_t* block, int32_t* warp_max_n, int32_t* cluster,
                                        int32_t* cluster_min_n);

/* Runs `iters` iterations of candidate schedules from the current state in
 * two stages -- block 128/256/512 x warp_max_n 0/64/256/1024 without clusters,
 * then clusters (cluster, cluster_min_n) = (4, 2048), (8, 2048), (8, 8192),
 * (4, 8192) at the best CTA shape -- scores each by the batch's time plus 4x
 * the largest graph's own duration (a solve to a relative residual runs its
 * slowest graphs several times the mean iteration count, so that graph's
 * group sets the makespan), keeps the best and restores the state.  Outputs
 * are nullable. */
pradmm_status pradmm_batch_autotune(pradmm_batch_t b, int32_t iters, int32_t* block_out,
                                    int32_t* warp_max_n_out, int32_t* cluster_out, int32_t* cluster_min_n_out);

/* Schedule search with the iteration profile of the last pradmm_batch_solve
 * (PRADMM_ERR_STATE if there is none): every candidate is timed on a probe in
 * which graph g runs ceil(work_fraction x its iterations in that solve)
 * iterations from the current state, so the probe has the solve's mix of work
 * (a fixed-iteration probe weighs the small graphs far above their share) and
 * its time is the score.  Candidates: block 128/256/512 x warp_max_n
 * 0/64/256/1024 without clusters, then at 256 and 512 threads (with the best
 * warp_max_n of that size) clusters of 2/4/8 above 2048/4096/8192 vertices.
 * work_fraction in (0, 1].  Keeps the best schedule and restores the state;
 * the per-graph outputs of the profiled solve are overwritten by the probes.
 * Outputs are nullable.  The paper has no counterpart. */
pradmm_status pradmm_batch_autotune_profiled(pradmm_batch_t b, double work_fraction, int32_t* block_out,
                                             int32_t* warp_max_n_out, int32_t* cluster_out,
                                             int32_t* cluster_min_n_out);

/* Initial states, all graphs at once (q: N x 4, t: N x 3 with N = sum n_g, in
 * graph order): odometry composition per graph, or given poses. */
/* General weight matrices for every graph of the batch (as pradmm_set_sigma;
 * both NULL returns to scalar weights).  Each graph's iteration then runs the
 * four general-weight sweeps; an FP32 p-update that needs the FP64 re-solve
 * does it in the same thread (counted in the handle's FP64 re-solves), and
 * pradmm_batch_objectives uses the Sigma-weighted norms.  The schedule's grid
 * is re-sized for the other kernel; a cluster shape that no longer fits
 * falls back to the start schedule. */
pradmm_status pradmm_batch_set_sigma(pradmm_batch_t b, const double* Sigma1, const double* Sigma2);

pradmm_status pradmm_batch_init_odometry(pradmm_batch_t b);
pradmm_status pradmm_batch_set_state(pradmm_batch_t b, const double* q, const double* t);

/* Runs every graph from the current state until its stopping rule.  Per-graph
 * outputs (G entries each, nullable): iterations, e^1, last e^k, and the
 * outcome (PRADMM_OK converged, PRADMM_ERR_NOT_CONVERGED max_iter reached,
 * PRADMM_ERR_NONFINITE).  Returns PRADMM_OK when every graph converged. */
pradmm_status pradmm_batch_solve(pradmm_batch_t b, double rel_tol, int32_t max_iter, int32_t* iters,
                                 double* e_first, double* e_last, int32_t* status);

/* F of Eq. (1) of each graph at its (p, t), double precision: F has G entries. */
pradmm_status pradmm_batch_objectives(pradmm_batch_t b, double* F);

/* Tracing: for each graph g of the last pradmm_batch_solve (or autotune
 * trial), the device time at which the work item that solves g started and
 * finished, in nanoseconds of the GPU's global timer (the same clock for all
 * graphs of one solve; differences are durations).  spans is 2 G uint64,
 * (start, end) per graph, host memory.  The paper has no counterpart: it is
 * for finding the graphs on a batch's critical path. */
pradmm_status pradmm_batch_spans(pradmm_batch_t b, uint64_t* spans);

/* State of all graphs (N rows each, graph order); any pointer may be NULL. */
pradmm_status pradmm_batch_get_state(pradmm_batch_t b, double* p, double* q, double* t, double* s,
                                     double* lam, double* z);

void pradmm_batch_destroy(pradmm_batch_t b);

#ifdef __cplusplus
}
#endif

#endif /* PRADMM_H */
