// Batched PRADMM with general weight matrices Sigma_1, Sigma_2: the persistent
// kernels of pradmm_batch.cuh with a policy that runs each graph's iteration
// as the four sweeps of the general-weight path (pradmm_sigma.cuh), separated
// by the group's barriers:
//   p-block (3a): the p-update of Lemma 1 per vertex, an FP32 update that asks
//                 for the FP64 re-solve doing it in the same thread (the
//                 stand-alone path queues it for a separate kernel; both run
//                 fb_solve on the same FP32 data)
//   q-block (3b) + lambda, t-block (3c), s-block (3d) + z
// then the group's residual e^k (Appendix E.1) and the batch's stopping rule,
// as in the plain batched iteration.
#include "pradmm_batch.cuh"
#include "pradmm_sigma.cuh"

namespace pradmm {
namespace {

using namespace dev;

template <typename R, bool INERT, typename G>
__device__ void solve_graph_sigma(const G& grp, const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                                  const SigmaDev<R>& sg, const BatchDev& b, int gid, Ctrl* ctrl) {
    const int64_t v0 = b.gv[gid], v1 = b.gv[gid + 1];
    const int r = grp.rank(), nt = grp.size();
    if (r == 0) b.t_span[2 * gid] = clock_ns();
    if (INERT) {
        // x^{-1} := x^0 (p^{-1} in the buffer the first p-block overwrites)
        for (int64_t i = v0 + r; i < v1; i += nt) {
            const R4<R> p0 = IO<R>::ld(S.p[0], i), q0 = IO<R>::ld(S.q, i);
            const R4<R> t0 = IO<R>::ld(S.t, i), s0 = IO<R>::ld(S.s, i);
            IO<R>::st(S.p[1], i, p0.a, p0.b, p0.c, p0.d);
            IO<R>::st(S.qprev, i, q0.a, q0.b, q0.c, q0.d);
            IO<R>::st(S.tprev, i, t0.a, t0.b, t0.c, t0.d);
            IO<R>::st(S.sprev, i, s0.a, s0.b, s0.c, s0.d);
        }
        grp.sync();
    }
    int k = 0, status = PRADMM_BATCH_MAXITER;
    double e1 = 0.0, e = 0.0;
    unsigned long long resolves = 0;
    const int cap = b.iter_cap ? b.iter_cap[gid] : b.max_iter;
    while (k < cap) {
        const R* pc = S.p[k & 1];
        R* pn = S.p[(k + 1) & 1];
        for (int64_t i = v0 + r; i < v1; i += nt) {
            FbRec rec;
            if (p_sig_vertex<R, INERT>(g, S, c, sg, pc, pn, i, rec)) {
                double xd[4];
                fb_solve(rec, xd);
                IO<R>::st(pn, i, R(xd[0]), R(xd[1]), R(xd[2]), R(xd[3]));
                ++resolves;
            }
        }
        grp.sync();
        Acc<R> adq, adl, adt, adz;
        for (int64_t i = v0 + r; i < v1; i += nt) q_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adq, adl);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) t_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adt);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) s_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adz);
        double d4[4] = {adl.get(), adz.get(), adq.get(), adt.get()};
        e = grp.residual(d4, c.b1d, c.b2d);
        ++k;
        if (k == 1) e1 = e;
        grp.sync_after_sum();
        if (!isfinite(e)) {
            status = PRADMM_BATCH_NONFINITE;
            break;
        }
        if (e <= b.rel_tol * e1 || e < b.abs_tol) {
            status = PRADMM_BATCH_CONVERGED;
            break;
        }
    }
    if (resolves) atomicAdd(&ctrl->fallbacks, resolves);
    // p^k is in buffer k & 1; keep the graph's result in buffer 0
    if (k & 1) {
        for (int64_t i = v0 + r; i < v1; i += nt) {
            const R4<R> v = IO<R>::ld(S.p[1], i);
            IO<R>::st(S.p[0], i, v.a, v.b, v.c, v.d);
        }
    }
    grp.sync();
    if (r == 0) {
        b.iters[gid] = k;
        b.e_first[gid] = e1;
        b.e_last[gid] = e;
        b.status[gid] = status;
        b.t_span[2 * gid + 1] = clock_ns();
    }
}

// The general-weight iteration as a batch policy.
template <typename R, bool INERT>
struct SigmaSolve {
    GraphDev<R> g;
    StateDev<R> S;
    Coef<R> c;
    SigmaDev<R> sg;
    template <typename G>
    __device__ __forceinline__ void operator()(const G& grp, const BatchDev& b, int gid, Ctrl* ctrl) const {
        solve_graph_sigma<R, INERT>(grp, g, S, c, sg, b, gid, ctrl);
    }
};

}  // namespace

template <typename R, bool INERT>
cudaError_t launch_batch_sigma(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const SigmaDev<R>& sg,
                               const BatchDev& b, Ctrl* ctrl, int grid, int block, int cluster, cudaStream_t st) {
    return launch_persistent(SigmaSolve<R, INERT>{g, s, c, sg}, b, ctrl, grid, block, cluster, st);
}

template <typename R, bool INERT>
cudaError_t batch_sigma_occupancy(int block, int* bps) {
    return persistent_occupancy<SigmaSolve<R, INERT>>(block, bps);
}

template <typename R, bool INERT>
cudaError_t batch_sigma_cluster_occupancy(int block, int cluster, int* clusters) {
    return persistent_cluster_occupancy<SigmaSolve<R, INERT>>(block, cluster, clusters);
}

#define PRADMM_BATCH_SIGMA_INST(R, I)                                                                          \
    template cudaError_t launch_batch_sigma<R, I>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&,       \
                                                  const SigmaDev<R>&, const BatchDev&, Ctrl*, int, int, int,    \
                                                  cudaStream_t);                                                \
    template cudaError_t batch_sigma_occupancy<R, I>(int, int*);                                                \
    template cudaError_t batch_sigma_cluster_occupancy<R, I>(int, int, int*);

// The build compiles this file once per precision and INERT flag (the four
// instances are the slowest code of the library to compile); without the
// macros it instantiates all four.
#if defined(PRADMM_BATCH_SIGMA_R)
PRADMM_BATCH_SIGMA_INST(PRADMM_BATCH_SIGMA_R, PRADMM_BATCH_SIGMA_INERT)
#else
PRADMM_BATCH_SIGMA_INST(float, false)
PRADMM_BATCH_SIGMA_INST(double, false)
PRADMM_BATCH_SIGMA_INST(float, true)
PRADMM_BATCH_SIGMA_INST(double, true)
#endif

}  // namespace pradmm
