// Sweep kernels of one PRADMM iteration (Section 3.2 Eq. (3a)-(3f),
// Algorithm 1, closed forms of Appendix B with scalar Sigma_1 = omega_e I,
// Sigma_2 = kappa_e I) for sm_103a.
//
// One iteration k -> k+1 is three launches in stream order:
//   k_q   q-block (3b) + relaxed lambda update (3e) + |dq|^2, |dlam|^2 partials
//   k_t   t-block (3c) + |dt|^2 partial
//   k_sp  s-block (3d) + relaxed z update (3f) + |dz|^2 partial, then the
//         p-block (3a) of iteration k+1 for the same vertex, then the last CTA
//         reduces the residual e^{k+1} (Appendix E.1) and sets the stop state.
// The p-block of iteration k+1 only needs the vertex's own s^{k+1}, while its
// gathers (t^{k+1}_j over out-edges, q^{k+1}_l over in-edges) were finished by
// earlier launches, so it fuses into the s-sweep and shares its pass over the
// out-edges.  p is double buffered so the p^{k+2} computed ahead never
// overwrites the p^{k+1} the same launch reads.
//
// Work decomposition.  Every block of the iteration is Jacobi over vertices,
// so one thread owns one vertex and loops over that vertex's CSR edges in
// input order: every sum has a fixed order and results are deterministic.
// The 32 vertices of a warp are consecutive, so their edge ranges form one
// dense block of 16-byte records that L1 serves across the loop steps; each
// step issues two edges' loads and neighbour gathers before using any of
// them.  Edge records and neighbour gathers go through the read-only path
// with normal caching (the records are invariant and no plain sweep writes
// an array it gathers); the gathered vertex arrays stay in L2 through the
// launches' access-policy window.
// Residual partials are per-thread compensated FP32 sums (FP32 has the
// throughput; FP64 on this part does not), then a fixed-order FP64 tree across
// threads and CTAs.
#include <cuda_runtime.h>

#include <cstdint>
#include <utility>

#include "pradmm_device.cuh"
#include "pradmm_internal.h"

// Resident 256-thread CTAs per SM requested from the register allocator.
#ifndef PRADMM_MINB_SP
#define PRADMM_MINB_SP 3
#endif
#ifndef PRADMM_MINB_Q
#define PRADMM_MINB_Q 3
#endif
#ifndef PRADMM_MINB_T
#define PRADMM_MINB_T 0
#endif
// pipelined edge loops (for_edges2) in the q and s/z + p sweeps; the t sweep
// always pipelines (it has registers to spare)
#ifndef PRADMM_PIPE_Q
#define PRADMM_PIPE_Q 0
#endif
#ifndef PRADMM_PIPE_SP
#define PRADMM_PIPE_SP 0
#endif
// 1: neighbour gathers on the read-only (non-coherent) path: each plain sweep
// writes none of the arrays it gathers (the batched kernel, which runs all
// sweeps in one launch, keeps coherent loads)
#ifndef PRADMM_NC
#define PRADMM_NC 1
#endif
#if PRADMM_MINB_T > 0
#define PRADMM_BOUNDS_T __launch_bounds__(256, PRADMM_MINB_T)
#else
#define PRADMM_BOUNDS_T __launch_bounds__(256)
#endif

namespace pradmm {
namespace {

using namespace dev;

template <typename R, bool INERT = false>
__global__ void __launch_bounds__(256, PRADMM_MINB_Q) k_q(GraphDev<R> g, StateDev<R> S, Coef<R> c, Ctrl* ctrl, double* part,
                                           int pstride) {
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    Acc<R> adq, adl;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        q_vertex<R, PRADMM_PIPE_Q != 0, PRADMM_NC != 0, INERT>(g, S, c, pn, i, adq, adl);
    __shared__ double sh2[2 * 32];
    double v[2] = {adq.get(), adl.get()};
    block_sum_n<2>(v, sh2);  // both CTA totals in one reduction
    const double sq = v[0], sl = v[1];
    if (threadIdx.x == 0) {
        part[SLOT_DQ * pstride + blockIdx.x] = sq;
        part[SLOT_DLAM * pstride + blockIdx.x] = sl;
    }
}

template <typename R, bool INERT = false>
__global__ void PRADMM_BOUNDS_T k_t(GraphDev<R> g, StateDev<R> S, Coef<R> c, Ctrl* ctrl, double* part,
                                           int pstride) {
    __shared__ double sh[32];
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    Acc<R> adt;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        t_vertex<R, true, PRADMM_NC != 0, INERT>(g, S, c, pn, i, adt);
    const double st = block_sum(adt.get(), sh);
    if (threadIdx.x == 0) part[SLOT_DT * pstride + blockIdx.x] = st;
}

// REC (scalar-weight recording, WITH_S): the state after this iteration
// goes to the tape slot of its iteration, if it has one (checkpoints and the
// last segment's iterates), each thread writing its own vertex's rows.
template <typename R, bool WITH_S, bool INERT = false, bool REC = false>
__global__ void __launch_bounds__(256, PRADMM_MINB_SP) k_sp(GraphDev<R> g, StateDev<R> S, Coef<R> c, Launch L) {
    __shared__ double sh[32];
    Ctrl* ctrl = L.ctrl;
    if (WITH_S && ctrl->halt) {
        // a halted while-loop body must still end the loop
        if (L.has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(L.cond, 0u);
        return;
    }
    const long long k = ctrl->iter;
    const R* pc = WITH_S ? S.p[(k + 1) & 1] : S.p[k & 1];  // p used by this sweep
    R* pn = WITH_S ? S.p[k & 1] : S.p[(k + 1) & 1];        // p computed ahead
    R* tape = nullptr;
    if (REC) {
        const TapeRec* T = L.tape;
        const long long d = k + 1 - T->k0;
        long long slot = -1;
        if (d > 0 && d <= T->K) {
            if (d % T->C == 0 || d == T->K) slot = (d + T->C - 1) / T->C;  // a checkpoint
            else if (d > T->d_last) slot = T->slot_last + (d - T->d_last) - 1;  // inside the last segment
        }
        if (slot >= 0) tape = reinterpret_cast<R*>(T->base + slot * T->slot_bytes);
    }
    Acc<R> adz;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        sp_vertex<R, WITH_S, PRADMM_PIPE_SP != 0, PRADMM_NC != 0, INERT, REC>(g, S, c, pc, pn, i, adz, ctrl, tape);
    if (WITH_S) {
        const double sd = block_sum(adz.get(), sh);
        if (threadIdx.x == 0) L.part[SLOT_DZ * L.pstride + blockIdx.x] = sd;
        finish_iteration(ctrl, L, c.b1d, c.b2d);
    }
}

__global__ void k_arm(Ctrl* ctrl, long long iters, int use_tol, double tol) {
    ctrl->target = ctrl->iter + iters;
    ctrl->halt = iters <= 0 ? 1 : 0;
    ctrl->stop = 0;
    ctrl->use_tol = use_tol;
    ctrl->tol = tol;
    ctrl->nonfinite = 0;
    ctrl->ticket = 0u;
}

// ---- objective F of Eq. (1) at (p^k, t^k), double precision ------------------
template <typename R>
__global__ void __launch_bounds__(256) k_objective(GraphDev<R> g, StateDev<R> S, const double* __restrict__ qe,
                                                   const double* __restrict__ te, const double* __restrict__ ka,
                                                   const double* __restrict__ om, Ctrl* ctrl, double* part,
                                                   unsigned int* ticket, double* F) {
    __shared__ double sh[32];
    __shared__ bool last;
    const long long k = ctrl->iter;
    const R* pc = S.p[k & 1];
    double acc = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x)
        acc += objective_vertex<R>(g, pc, S.t, qe, te, ka, om, i);
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

// ---- layout conversion (internal vertex i <-> user vertex perm[i]) -------------
template <typename R>
__global__ void k_pack4(const double* __restrict__ src, const int32_t* __restrict__ perm, R* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = perm[i];
        IO<R>::st(dst, i, R(src[4 * u]), R(src[4 * u + 1]), R(src[4 * u + 2]), R(src[4 * u + 3]));
    }
}
template <typename R>
__global__ void k_pack3(const double* __restrict__ src, const int32_t* __restrict__ perm,
                        const double* __restrict__ inv, R* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = perm[i];
        IO<R>::st(dst, i, R(src[3 * u]), R(src[3 * u + 1]), R(src[3 * u + 2]), R(inv[i]));
    }
}
template <typename R>
__global__ void k_unpack4(const R* src, const int32_t* __restrict__ perm, double* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = IO<R>::ld(src, i);
        const int64_t u = perm[i];
        dst[4 * u] = v.a;
        dst[4 * u + 1] = v.b;
        dst[4 * u + 2] = v.c;
        dst[4 * u + 3] = v.d;
    }
}
template <typename R>
__global__ void k_unpack3(const R* src, const int32_t* __restrict__ perm, double* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = IO<R>::ld(src, i);
        const int64_t u = perm[i];
        dst[3 * u] = v.a;
        dst[3 * u + 1] = v.b;
        dst[3 * u + 2] = v.c;
    }
}

inline int conv_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

// Sweep launch with the handle's L2 access-policy window as a launch
// attribute (captured into the CUDA graph with the kernel node).
template <typename... P, typename... A>
cudaError_t launch_sweep(const Launch& L, int grid, void (*kern)(P...), A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)L.block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = L.stream;
    cudaLaunchAttribute at[1];
    if (L.has_window) {
        at[0].id = cudaLaunchAttributeAccessPolicyWindow;
        at[0].val.accessPolicyWindow = L.window;
        cfg.attrs = at;
        cfg.numAttrs = 1;
    }
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}


template <typename R>
cudaError_t launch_p(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    return launch_sweep(L, L.grid_p, k_sp<R, false>, g, s, c, L);
}
template <typename R>
cudaError_t launch_q(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    // the inertial variant (theta != 0) runs its own instances of the sweeps
    if (c.theta != R(0)) return launch_sweep(L, L.grid_q, k_q<R, true>, g, s, c, L.ctrl, L.part, L.pstride);
    return launch_sweep(L, L.grid_q, k_q<R>, g, s, c, L.ctrl, L.part, L.pstride);
}
template <typename R>
cudaError_t launch_t(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    if (c.theta != R(0)) return launch_sweep(L, L.grid_t, k_t<R, true>, g, s, c, L.ctrl, L.part, L.pstride);
    return launch_sweep(L, L.grid_t, k_t<R>, g, s, c, L.ctrl, L.part, L.pstride);
}
template <typename R>
cudaError_t launch_sp(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    if (c.theta != R(0)) return launch_sweep(L, L.grid_sp, k_sp<R, true, true>, g, s, c, L);
    if (L.tape) return launch_sweep(L, L.grid_sp, k_sp<R, true, false, true>, g, s, c, L);
    return launch_sweep(L, L.grid_sp, k_sp<R, true>, g, s, c, L);
}

template <typename R>
cudaError_t occupancy_r(int block, int* bps) {
    cudaError_t e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[0], k_sp<R, false>, block, 0))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[1], k_q<R>, block, 0))) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[2], k_t<R>, block, 0))) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps[3], k_sp<R, true>, block, 0);
}

cudaError_t sweep_occupancy(int is_double, int block, int* bps) {
    return is_double ? occupancy_r<double>(block, bps) : occupancy_r<float>(block, bps);
}

cudaError_t launch_arm(Ctrl* ctrl, long long iters, int use_tol, double tol, cudaStream_t st) {
    k_arm<<<1, 1, 0, st>>>(ctrl, iters, use_tol, tol);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_objective(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64, const double* te64,
                             const double* kappa64, const double* omega64, Ctrl* ctrl, double* part,
                             unsigned int* ticket, double* F_dev, int grid, int block, cudaStream_t st) {
    k_objective<R><<<grid, block, 0, st>>>(g, s, qe64, te64, kappa64, omega64, ctrl, part, ticket, F_dev);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pack4(const double* src, const int32_t* perm, R* dst, int64_t n, cudaStream_t st) {
    k_pack4<R><<<conv_grid(n), 256, 0, st>>>(src, perm, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_pack3(const double* src, const int32_t* perm, const double* inv, R* dst, int64_t n,
                         cudaStream_t st) {
    k_pack3<R><<<conv_grid(n), 256, 0, st>>>(src, perm, inv, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_unpack4(const R* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st) {
    k_unpack4<R><<<conv_grid(n), 256, 0, st>>>(src, perm, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_unpack3(const R* src, const int32_t* perm, double* dst, int64_t n, cudaStream_t st) {
    k_unpack3<R><<<conv_grid(n), 256, 0, st>>>(src, perm, dst, n);
    return cudaGetLastError();
}

#define PRADMM_INST(R)                                                                                        \
    template cudaError_t launch_p<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_q<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_t<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_sp<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&); \
    template cudaError_t launch_objective<R>(const GraphDev<R>&, const StateDev<R>&, const double*,           \
                                             const double*, const double*, const double*, Ctrl*, double*,     \
                                             unsigned int*, double*, int, int, cudaStream_t);                 \
    template cudaError_t launch_pack4<R>(const double*, const int32_t*, R*, int64_t, cudaStream_t);           \
    template cudaError_t launch_pack3<R>(const double*, const int32_t*, const double*, R*, int64_t,           \
                                         cudaStream_t);                                                       \
    template cudaError_t launch_unpack4<R>(const R*, const int32_t*, double*, int64_t, cudaStream_t);         \
    template cudaError_t launch_unpack3<R>(const R*, const int32_t*, double*, int64_t, cudaStream_t);

PRADMM_INST(float)
PRADMM_INST(double)

}  // namespace pradmm
