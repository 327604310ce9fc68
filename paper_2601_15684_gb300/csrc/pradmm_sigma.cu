// PRADMM sweeps with general weight matrices Sigma_1, Sigma_2 for sm_103a:
// one launch per block of Eq. (3a)-(3f), each a grid-stride loop over
// vertices running the per-vertex updates of pradmm_sigma.cuh.
//   k_p_sig     p-block (3a); FP32 p-updates that need an FP64 re-solve are
//               queued (one atomic slot each)
//   k_p_sig_fb  the queued FP64 re-solves, full warps spread over the SMs
//   k_q_sig     q-block (3b) + lambda
//   k_t_sig     t-block (3c)
//   k_s_sig     s-block (3d) + z, residual and stop (last CTA)
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_sigma.cuh"

namespace pradmm {
namespace {

using namespace dev;

// ---- kernels --------------------------------------------------------------------

template <typename R, bool INERT>
__global__ void __launch_bounds__(256) k_p_sig(GraphDev<R> g, StateDev<R> S, Coef<R> c, SigmaDev<R> sg, Ctrl* ctrl) {
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pc = S.p[k & 1];
    R* pn = S.p[(k + 1) & 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        FbRec rec;
        if (p_sig_vertex<R, INERT>(g, S, c, sg, pc, pn, i, rec)) {
            // queued for k_p_sig_fb, which writes p_i
            const unsigned slot = atomicAdd(&sg.fb_n[k & 1], 1u);
            sg.fb_q[slot] = rec;
            atomicAdd(&ctrl->fallbacks, 1ull);
        }
    }
}

// The FP64 re-solves queued by k_p_sig in iteration k (FP32 handles only):
// entry kFbLanes w + l goes to lane l of global warp w, and consecutive warps
// go to different CTAs, so the few warps of FP64 work spread over the SMs.
// Clears iteration k+1's counter (its last use was iteration k-1, finished).
__global__ void __launch_bounds__(128) k_p_sig_fb(SigmaDev<float> sg, StateDev<float> S, const Ctrl* ctrl) {
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    float* pn = S.p[(k + 1) & 1];
    const unsigned cnt = sg.fb_n[k & 1];
    const unsigned lane = threadIdx.x & 31, wib = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const unsigned nw = gridDim.x * wpb;
    for (unsigned w = blockIdx.x + gridDim.x * wib; kFbLanes * w < cnt; w += nw) {
        const unsigned e = kFbLanes * w + lane;
        if (lane >= kFbLanes || e >= cnt) continue;
        const FbRec& q = sg.fb_q[e];
        double xd[4];
        fb_solve(q, xd);
        IO<float>::st(pn, q.i, float(xd[0]), float(xd[1]), float(xd[2]), float(xd[3]));
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sg.fb_n[(k + 1) & 1] = 0u;
}

template <typename R, bool INERT>
__global__ void __launch_bounds__(256) k_q_sig(GraphDev<R> g, StateDev<R> S, Coef<R> c, SigmaDev<R> sg, Ctrl* ctrl,
                                               double* part, int pstride) {
    __shared__ double sh[32];
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    Acc<R> adq, adl;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        q_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adq, adl);
    const double sq = block_sum(adq.get(), sh);
    const double sl = block_sum(adl.get(), sh);
    if (threadIdx.x == 0) {
        part[SLOT_DQ * pstride + blockIdx.x] = sq;
        part[SLOT_DLAM * pstride + blockIdx.x] = sl;
    }
}

template <typename R, bool INERT>
__global__ void __launch_bounds__(256) k_t_sig(GraphDev<R> g, StateDev<R> S, Coef<R> c, SigmaDev<R> sg, Ctrl* ctrl,
                                               double* part, int pstride) {
    __shared__ double sh[32];
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    Acc<R> adt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        t_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adt);
    const double st = block_sum(adt.get(), sh);
    if (threadIdx.x == 0) part[SLOT_DT * pstride + blockIdx.x] = st;
}

template <typename R, bool INERT>
__global__ void __launch_bounds__(256) k_s_sig(GraphDev<R> g, StateDev<R> S, Coef<R> c, SigmaDev<R> sg, Launch L) {
    __shared__ double sh[32];
    Ctrl* ctrl = L.ctrl;
    if (ctrl->halt) {
        if (L.has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(L.cond, 0u);
        return;
    }
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    Acc<R> adz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        s_sig_vertex<R, INERT>(g, S, c, sg, pn, i, adz);
    const double sd = block_sum(adz.get(), sh);
    if (threadIdx.x == 0) L.part[SLOT_DZ * L.pstride + blockIdx.x] = sd;
    finish_iteration(ctrl, L, c.b1d, c.b2d);
}

// F of Eq. (1) with Sigma-weighted norms at (p^k, t^k), in double.
template <typename R>
__global__ void __launch_bounds__(256) k_objective_sig(GraphDev<R> g, StateDev<R> S, const double* __restrict__ qe,
                                                       const double* __restrict__ te, const double* __restrict__ ka,
                                                       const double* __restrict__ om, const double* __restrict__ S1,
                                                       const double* __restrict__ S2, Ctrl* ctrl, double* part,
                                                       unsigned int* ticket, double* F) {
    __shared__ double sh[32];
    __shared__ bool last;
    const R* pc = S.p[ctrl->iter & 1];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        acc += objective_sig_vertex<R>(g, pc, S.t, qe, te, ka, om, S1, S2, i);
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = bs;
    __threadfence();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(part + b);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *F = tot;
        *ticket = 0u;
    }
}

}  // namespace

template <typename R>
cudaError_t launch_sigma_iteration(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c,
                                   const SigmaDev<R>& sg, const Launch& L) {
    if (c.theta != R(0)) {
        k_p_sig<R, true><<<L.grid_p, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl);
        if constexpr (sizeof(R) == sizeof(float)) k_p_sig_fb<<<152, 128, 0, L.stream>>>(sg, s, L.ctrl);
        k_q_sig<R, true><<<L.grid_q, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl, L.part, L.pstride);
        k_t_sig<R, true><<<L.grid_t, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl, L.part, L.pstride);
        k_s_sig<R, true><<<L.grid_sp, L.block, 0, L.stream>>>(g, s, c, sg, L);
    } else {
        k_p_sig<R, false><<<L.grid_p, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl);
        if constexpr (sizeof(R) == sizeof(float)) k_p_sig_fb<<<152, 128, 0, L.stream>>>(sg, s, L.ctrl);
        k_q_sig<R, false><<<L.grid_q, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl, L.part, L.pstride);
        k_t_sig<R, false><<<L.grid_t, L.block, 0, L.stream>>>(g, s, c, sg, L.ctrl, L.part, L.pstride);
        k_s_sig<R, false><<<L.grid_sp, L.block, 0, L.stream>>>(g, s, c, sg, L);
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_objective_sigma(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64,
                                   const double* te64, const double* ka64, const double* om64, const double* S1,
                                   const double* S2, Ctrl* ctrl, double* part, unsigned int* ticket, double* F_dev,
                                   int grid, int block, cudaStream_t st) {
    k_objective_sig<R><<<grid, block, 0, st>>>(g, s, qe64, te64, ka64, om64, S1, S2, ctrl, part, ticket, F_dev);
    return cudaGetLastError();
}

#define PRADMM_SIGMA_INST(R)                                                                                      \
    template cudaError_t launch_sigma_iteration<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&,         \
                                                   const SigmaDev<R>&, const Launch&);                            \
    template cudaError_t launch_objective_sigma<R>(const GraphDev<R>&, const StateDev<R>&, const double*,         \
                                                   const double*, const double*, const double*, const double*,    \
                                                   const double*, Ctrl*, double*, unsigned int*, double*, int, int, \
                                                   cudaStream_t);

PRADMM_SIGMA_INST(float)
PRADMM_SIGMA_INST(double)

}  // namespace pradmm
