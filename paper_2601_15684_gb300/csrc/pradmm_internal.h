// Internal declarations shared by the host side and the sweep kernels of
// libpradmm.  Not part of the public ABI (include/pradmm.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pradmm {

// Device-resident control block of one handle.  The last CTA of every
// s/z + p sweep reduces the residual partials, advances `iter` and decides
// whether the next iteration runs (`halt`), so a whole solve needs no
// host round trip.
struct Ctrl {
    long long iter;        // completed iterations k (state is x^k)
    long long target;      // halt once iter reaches target
    double e_last;         // e^k (Appendix E.1, reading R6)
    double parts[4];       // |dlam|^2, |dz|^2, |dq|^2, |dt|^2 of the last iteration
    double tol;            // stopping tolerance when use_tol
    unsigned int ticket;   // CTA arrival counter of the last-block reduction
    int halt;              // 1: sweep kernels return at once
    int stop;              // 1: e^k < tol was met
    int use_tol;           // 1: solve (stopping test on), 0: step
    int nonfinite;         // 1: e^k was NaN or Inf
    unsigned long long fallbacks;  // p-updates recomputed in FP64
    unsigned long long zero_u;     // p-updates with |u| == 0 (kept p^k)
};

// Residual partial slots (double part[4 * pstride]).
enum { SLOT_DLAM = 0, SLOT_DZ = 1, SLOT_DQ = 2, SLOT_DT = 3 };

// Graph in CSR form over internal vertex ids (internal vertex i is user
// vertex perm[i]; see launch_pack4).  The out-edges of i are slots
// [out_ptr[i], out_ptr[i+1]) in input order, its in-edges [in_ptr[i],
// in_ptr[i+1]).  Consecutive vertices' edge ranges are adjacent, so the 32
// lanes of a warp walk one dense block of edge records.
template <typename R>
struct GraphDev {
    int64_t n, m;
    const int32_t* out_ptr;  // n+1
    const int32_t* in_ptr;   // n+1
    const int32_t* out_idx;  // m: head j (internal id) of each out-edge
    const R* out_te;         // 4m: (t_e x, y, z, omega_e)
    const R* out_qk;         // 4m: kappa_e q_e
    const int32_t* in_idx;   // m: tail l (internal id) of each in-edge
    const R* in_te;          // 4m: (t_e x, y, z, omega_e)
    const R* in_qk;          // 4m: kappa_e q_e
    // index-checked builds (PRADMM_DEBUG_CHECKS): [0] indices found out of
    // range, [1] the last such value (device memory; unused otherwise)
    unsigned int* dbg = nullptr;
};

// Pose / multiplier state in internal vertex order.  p is double buffered:
// p[k & 1] holds p^k and p[(k+1) & 1] the p^{k+1} that the s/z sweep of
// iteration k-1 (or the first p sweep) computed ahead.  3-vectors are padded
// to 4; the padding carries the iteration-invariant inverse block matrices
// (Appendix B with scalar Sigma): s.w = 1/A_2, t.w = 1/A_3, z.w = 1/A_4.
template <typename R>
struct StateDev {
    R* p[2];
    R* q;
    R* lam;
    R* t;
    R* s;
    R* z;
    // inertial variant only (else NULL): the previous iterates q^{k-1},
    // t^{k-1}, s^{k-1} of the extrapolated proximal anchors
    R* qprev = nullptr;
    R* tprev = nullptr;
    R* sprev = nullptr;
};

template <typename R>
struct Coef {
    R beta1, beta2;      // penalties
    R tb1, tb2;          // tau * beta1, tau * beta2
    R g1, g2, g3, g4;    // proximal weights
    double b1d, b2d;     // penalties in double (residual)
    double fb_thresh;    // FP64 recompute of the p-update below this |u|
    R theta = R(0);      // inertial extrapolation of the proximal anchors (0: plain)
};

struct TapeRec;

struct Launch {
    int grid_p, grid_q, grid_t, grid_sp;  // CTAs of each sweep (fixed per handle)
    int pstride;              // partial slot stride (>= every grid)
    int block;                // threads per CTA (multiple of 32)
    cudaStream_t stream;
    Ctrl* ctrl;
    double* part;             // 4 * pstride doubles
    cudaGraphConditionalHandle cond;
    int has_cond;
    cudaAccessPolicyWindow window;  // L2 persistence of the gathered vertex arrays
    int has_window;
    double* trace = nullptr;        // optional ring of e^k: iteration k writes trace[(k - 1) % trace_cap]
    long long trace_cap = 0;
    // reverse-mode recording with scalar weights: the s/z + p sweep also
    // writes each vertex's state into the tape slot of its iteration
    const TapeRec* tape = nullptr;
};

template <typename R>
cudaError_t launch_p(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L);
template <typename R>
cudaError_t launch_q(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L);
template <typename R>
cudaError_t launch_t(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L);
template <typename R>
cudaError_t launch_sp(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L);

// Resident CTAs per SM of the sweep kernels at `block` threads:
// bps[0] first p sweep, bps[1] q sweep, bps[2] t sweep, bps[3] s/z + p sweep.
cudaError_t sweep_occupancy(int is_double, int block, int* bps);

// Set-up on the device (pradmm_setup.cu).  build_csr_device: CSR of the edges
// by `key` (input order inside a row): ptr (n+1), slot_edge (slot -> edge),
// idx (slot -> other endpoint), edge_slot (edge -> slot, nullable); fill (n)
// and sums ((n + 1023) / 1024) are scratch.
cudaError_t build_csr_device(const int32_t* key, const int32_t* other, int64_t n, int64_t m, int32_t* ptr,
                             int32_t* slot_edge, int32_t* idx, int32_t* edge_slot, int32_t* fill, int32_t* sums,
                             cudaStream_t st);
// The per-edge checks of pradmm_create on the uploaded arrays (ka, om may be
// NULL: unit weights); *first_bad, set to m beforehand, receives the lowest
// failing edge.
cudaError_t launch_validate(const int32_t* src, const int32_t* dst, const double* q, const double* t, const double* ka,
                            const double* om, int64_t n, int64_t m, int32_t* first_bad, cudaStream_t st);
// The endpoint checks of launch_validate on their own (endpoints in [0, n),
// no self-loop), lowering *first_bad; endpoints outside [0, n) are replaced
// by 0 in place so that kernels indexing with them stay in bounds.
cudaError_t launch_check_ends(int32_t* src, int32_t* dst, int64_t n, int64_t m, int32_t* first_bad, cudaStream_t st);
// Inclusive scan of a[0, len) in place; sums holds (len + 1023) / 1024 ints.
cudaError_t inclusive_scan_i32(int32_t* a, int64_t len, int32_t* sums, cudaStream_t st);
// The odometry start's spanning forest (Kruskal by edge order, found by
// Boruvka's rounds) rooted at each component's lowest vertex
// (pradmm_forest.cu), from the out-edge CSR (out_ptr, out_idx: heads,
// out_edge: input edge per slot): par[v] the parent (-1 for a root), pedge[v]
// the tree edge e to it coded as for launch_odometry.  scratch:
// forest_scratch_ints(n, m) ints.  Synchronises the stream (host reads of
// the round counts).  pradmm_create runs it once per handle.
size_t forest_scratch_ints(int64_t n, int64_t m);
cudaError_t launch_forest(const int32_t* out_ptr, const int32_t* out_idx, const int32_t* out_edge, int64_t n,
                          int64_t m, int32_t* scratch, int32_t* par, int32_t* pedge, cudaStream_t st);
cudaError_t launch_block_inv(const int32_t* out_ptr, const int32_t* out_edge, const int32_t* in_ptr,
                             const int32_t* in_edge, int64_t n, const double* t, const double* ka, const double* om,
                             double a2_0, double a3_0, double a4_0, double* inv2, double* inv3, double* inv4,
                             cudaStream_t st);
cudaError_t launch_iota(int32_t* a, int64_t n, cudaStream_t st);
cudaError_t launch_slot_owner(const int32_t* ptr, int64_t n, int32_t* owner, cudaStream_t st);
// Odometry poses from the spanning forest: pedge[v] = e when v is the head of
// its tree edge e, -(e + 2) when v is its tail, -1 for a root; par[v] the
// parent (-1 for a root).  The poses end in q (4n), t (3n); q_tmp, t_tmp and
// `scratch` (odometry_scratch_bytes(n), 8-byte aligned) are work space.  No
// host synchronisation: every pointer-jumping loop runs enough rounds for
// any tree of n vertices.
size_t odometry_scratch_bytes(int64_t n);
cudaError_t launch_odometry(const int32_t* pedge, const int32_t* par, const int32_t* edge_slot, const double* qe64,
                            const double* te64, int64_t n, void* scratch, double* q, double* t, double* q_tmp,
                            double* t_tmp, cudaStream_t st);

// Device-side parameters of a tape recording (reverse mode): after the
// iteration that brings ctrl->iter to k0 + d, with d a multiple of C or
// d = K, the whole state block (slot_bytes, a multiple of 16) is copied to
// tape slot ceil(d / C) at base + slot * slot_bytes.
struct TapeRec {
    char* base;
    long long k0, K, C, slot_bytes;
    // the states inside the last segment (iterations d_last + j, 0 < j,
    // below K) also go to slots slot_last + j - 1: the recompute slots the
    // reverse pass reads for that segment, which it then need not recompute
    long long d_last, slot_last;
};

// Inertial recording: copies p[ctrl->iter & 1] (p^k, before the s/z + next-p
// sweep overwrites it) to dst (n 4-real rows).
template <typename R>
cudaError_t launch_keep_pk(const Ctrl* ctrl, const R* p0, const R* p1, R* dst, int64_t n, int grid, cudaStream_t st);
// Fills *rec with k0 = ctrl->iter (read on the device) and the arguments.
cudaError_t launch_tape_rec_arm(TapeRec* rec, const Ctrl* ctrl, void* base, long long K, long long C,
                                long long slot_bytes, long long d_last, long long slot_last, cudaStream_t st);
// The checkpoint copy that follows each recorded iteration (a no-op between
// checkpoints); grid-stride 16-byte copies from the state block `src`.
cudaError_t launch_tape_copy(const TapeRec* rec, const Ctrl* ctrl, const void* src, int grid, cudaStream_t st);

// Sets target = iter + iters, halt = (iters <= 0), stop = 0, use_tol, tol.
cudaError_t launch_arm(Ctrl* ctrl, long long iters, int use_tol, double tol, cudaStream_t st);

// F of Eq. (1) at (p^k, t^k) in double: per-CTA partials, then the last CTA
// sums them in a fixed order into *F_dev.  qe64, te64, ka64, om64 are the
// measurements in out-edge order.
template <typename R>
cudaError_t launch_objective(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64,
                             const double* te64, const double* kappa64, const double* omega64,
                             Ctrl* ctrl, double* part, unsigned int* ticket, double* F_dev, int grid,
                             int block, cudaStream_t st);

// Layout conversion between caller arrays (double, user vertex order, n x 4 /
// n x 3) and the padded internal arrays: internal vertex i is user vertex
// perm[i]; `inv` (internal order) supplies the padding of a 3-vector.
// Per-slot edge records of one CSR order (slot k holds input edge edge[k]),
// packed from the caller's measurements in device memory: te_out (t_e,
// omega_e) and qk_out kappa_e q_e/|q_e| in R; for the out order also the FP64
// copies qe64 (normalised), te64, ka64, om64 (NULL for the in order).  ka, om
// NULL mean all ones.  Asynchronous on st.
template <typename R>
cudaError_t launch_pack_slots(const int32_t* edge, int64_t slots, const double* q, const double* t, const double* ka,
                              const double* om, R* te_out, R* qk_out, double* qe64, double* te64, double* ka64,
                              double* om64, cudaStream_t st);
// In-order records (te_out, qk_out per in-slot; ie: in-slot -> input edge)
// gathered from the out-order FP64 copies that launch_pack_slots wrote.
template <typename R>
cudaError_t launch_pack_in(const int32_t* ie, const int32_t* edge_slot, int64_t slots, const double* qe64,
                           const double* te64, const double* ka64, const double* om64, R* te_out, R* qk_out,
                           cudaStream_t st);

template <typename R>
cudaError_t launch_pack4(const double* src, const int32_t* perm, R* dst, int64_t n, cudaStream_t st);
template <typename R>
cudaError_t launch_pack3(const double* src, const int32_t* perm, const double* inv, R* dst, int64_t n,
                         cudaStream_t st);
template <typename R>
cudaError_t launch_unpack4(const R* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st);
template <typename R>
cudaError_t launch_unpack3(const R* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st);

// ---- general weight matrices (Sigma_1, Sigma_2 not scalar) ------------------------

// Passed by value as a kernel parameter.  S1, S2 row-major 4x4; U (row-major
// 3x3, columns the eigenvectors) and mu the eigen-decomposition of the
// translation block Sigma1_hat = S1[1..3][1..3].
// One queued FP64 re-solve: vertex, FP32 A_1 (upper triangle, row by row),
// b_1 and p^k.
struct FbRec {
    int32_t i;
    float a[10];
    float b[4];
    float pk[4];
    float pad;
};

template <typename R>
struct SigmaDev {
    R S1[16];
    R S2[16];
    R U[9];
    R mu[3];
    // sandwich maps: X(a)^T S X(a) (upper triangle, 10 entries) as a linear
    // map of a a^T (10 entries), row-major 10 x 10.  LM1D: X = M, S = Sigma_1,
    // D-conjugated (p-block out-edges); LW2D: X = W, S = Sigma_2,
    // D-conjugated (p-block in-edges); LW1: X = W, S = Sigma_1 (q-block G3).
    R LM1D[100];
    R LW2D[100];
    R LW1[100];
    // FP32 handles: p-updates whose sphere-constrained quadratic needs the FP64
    // re-solve are queued by the p sweep (their FP32 A_1, b_1, p^k) and solved
    // together by the next kernel, full warps of FP64 work instead of one lane
    // per warp.  fb_n[k & 1] counts iteration k's entries.
    FbRec* fb_q = nullptr;   // n records
    unsigned int* fb_n = nullptr;  // 2 counters
};

// One iteration with general Sigma: p, q, t sweeps and the s/z sweep with the
// residual and stop state (the same partial slots and control block as the
// scalar sweeps).
template <typename R>
cudaError_t launch_sigma_iteration(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c,
                                   const SigmaDev<R>& sg, const Launch& L);
template <typename R>
cudaError_t launch_objective_sigma(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64,
                                   const double* te64, const double* ka64, const double* om64, const double* S1,
                                   const double* S2, Ctrl* ctrl, double* part, unsigned int* ticket, double* F_dev,
                                   int grid, int block, cudaStream_t st);

// ---- batched solver ------------------------------------------------------------

// Per-graph outcome codes (the pradmm_status values of the same meaning).
enum { PRADMM_BATCH_CONVERGED = 0, PRADMM_BATCH_NONFINITE = 4, PRADMM_BATCH_MAXITER = 8 };

// Device view of a batch: graph g owns internal vertices [gv[g], gv[g+1]) of
// the union graph.  Work items (order positions, count): count < 0 is one
// graph solved by a whole CTA, count > 0 a pack of that many small graphs
// solved by one warp each.  `next` is the queue counter.
struct BatchDev {
    const int64_t* gv;    // G + 1
    const int32_t* order; // graphs by size, largest first
    const int2* items;    // n_items
    int n_items;
    int* next;
    int n_big;            // cluster items: order positions [0, n_big) (k_batch_cl)
    int* next_big;
    int32_t* iters;       // G outputs
    double* e_first;
    double* e_last;
    int32_t* status;
    unsigned long long* t_span;  // 2 G: device clock (ns) at each graph's start and end
    double rel_tol, abs_tol;
    int max_iter;
    const int32_t* iter_cap = nullptr;  // G per-graph iteration limits (NULL: max_iter for all)
};

// cluster > 1: the cluster kernel (grid a multiple of cluster); 1: k_batch.
// INERT: the inertial variant (S.qprev, S.tprev, S.sprev set; c.theta != 0).
template <typename R, bool INERT>
cudaError_t launch_batch(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const BatchDev& b,
                         Ctrl* ctrl, int grid, int block, int cluster, cudaStream_t st);
template <typename R, bool INERT>
cudaError_t batch_occupancy(int block, int* bps);
template <typename R, bool INERT>
cudaError_t batch_cluster_occupancy(int block, int cluster, int* clusters);
// The batched form with general weights (pradmm_batch_sigma.cu).
template <typename R, bool INERT>
cudaError_t launch_batch_sigma(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const SigmaDev<R>& sg,
                               const BatchDev& b, Ctrl* ctrl, int grid, int block, int cluster, cudaStream_t st);
template <typename R, bool INERT>
cudaError_t batch_sigma_occupancy(int block, int* bps);
template <typename R, bool INERT>
cudaError_t batch_sigma_cluster_occupancy(int block, int cluster, int* clusters);
// S1, S2: Sigma_1, Sigma_2 on the device (16 doubles each), or NULL for scalar weights.
template <typename R>
cudaError_t launch_batch_objective(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64,
                                   const double* te64, const double* ka64, const double* om64, const double* S1,
                                   const double* S2, const BatchDev& b, double* F, int G, cudaStream_t st);

// ---- reverse mode (adjoint) ------------------------------------------------------

// Per-vertex adjoint arrays (internal vertex order, 4 reals per vertex unless
// noted) and the per-out-slot measurement gradients.
template <typename R>
struct AdjDev {
    R* gs;   // (gs, A_4bar): adjoint of the s-block numerator / A_4, and of A_4
    R* gs_w; // where step A writes the next (earlier) iteration's gs: the other
             // of two buffers by iteration parity, so that the gradient sweep of
             // iteration k can still read its gs while step A of k - 1 runs
    R* gt;   // (gt, A_3bar)
    R* gq;   // gq = qbar / A_2
    R* a2b;  // n: A_2bar
    R* pb;   // adjoint of p^{k+1} (accumulating)
    R* qb;   // adjoint of q^{k+1}
    R* tb;   // adjoint of t^{k+1}
    R* ub;   // adjoint of u (sphere projection)
    R *op, *oq, *ot, *os, *ol, *oz;  // adjoint of x^k (p, q, t, s, lam, z)
    // inertial variant (else NULL): the share of x^{k-1}'s adjoint that
    // iteration k's anchors x^k + theta (x^k - x^{k-1}) produce (p, q, t, s)
    R *vp = nullptr, *vq = nullptr, *vt = nullptr, *vs = nullptr;
    const R* eq;     // 4m: q_e per out-slot (unscaled)
    const R* ek;     // m: kappa_e per out-slot
    double* g_te;    // 4m: (dL/dt_e, dL/domega_e) per out-slot
    double* g_qe;    // 4m: dL/dq_e
    double* g_ka;    // m: dL/dkappa_e
};

// State of one unrolled iteration k -> k+1 (tape slots; pads as in StateDev).
template <typename R>
struct AdjStep {
    const R* pc;   // p^k
    const R* pn;   // p^{k+1}
    const R *q, *lam, *t, *s, *z;  // x^k
    const R *qn, *tn;              // q^{k+1}, t^{k+1}
    const R* pp = nullptr;         // p^{k-1} (inertial variant)
};

template <typename R>
cudaError_t launch_adj_seed(const GraphDev<R>& g, const AdjDev<R>& A, const Coef<R>& c, const R* s_K, const R* z_K,
                            int block, cudaStream_t st);
// The reverse sweeps of iteration k (out_src: tail of each out-slot); `more`
// = 1 starts iteration k-1.  With `side` (and the events fork, join) the
// per-edge gradient sweep runs on that stream beside the sweep that starts
// iteration k-1 (they share no written array: A.gs_w != A.gs), joined
// before return; else everything runs on st in order.
template <typename R>
cudaError_t launch_adj_iteration(const GraphDev<R>& g, const AdjDev<R>& A, const AdjStep<R>& X, const Coef<R>& c,
                                 const int32_t* out_src, int more, int block, cudaStream_t st,
                                 cudaStream_t side = nullptr, cudaEvent_t fork = nullptr, cudaEvent_t join = nullptr);
template <typename R>
cudaError_t launch_adj_edges(const double* qe64, const double* ka64, int64_t m, R* eq, R* ek, cudaStream_t st);
cudaError_t launch_adj_scatter(const double* g_qe, const double* g_te, const double* g_ka, const int32_t* eidx,
                               int64_t m, double* qe_bar, double* te_bar, double* ka_bar, double* om_bar,
                               cudaStream_t st);
// Sets a tape control block to iteration `iter` with no halt and no target.
cudaError_t launch_tape_arm(Ctrl* ctrl, long long iter, cudaStream_t st);

// Records the message pradmm_last_error() returns on the calling thread.
void set_last_error(const char* msg);

}  // namespace pradmm
