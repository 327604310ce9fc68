// Batched PRADMM: many independent pose graphs solved in one persistent
// launch.  The batch is one disjoint-union graph (each graph's vertices are a
// contiguous internal range), so the per-vertex updates are exactly those of
// the plain sweeps (pradmm_device.cuh).  Each CTA of the persistent kernel
// repeatedly takes the next work item from a queue ordered largest first:
//   - a graph item: the whole CTA runs Algorithm 1 on one graph, the three
//     sweeps of an iteration separated by CTA barriers;
//   - a pack item: each warp of the CTA runs Algorithm 1 on its own small
//     graph, sweeps separated by warp barriers.
// A graph's residual e^k (Appendix E.1) is reduced inside its group, and the
// group stops when e^k <= rel_tol * e^1 (the batch's relative stopping rule),
// e^k < abs_tol, the residual is not finite, or max_iter is reached.  No CTA
// ever waits for another CTA.
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_device.cuh"
#include "pradmm_internal.h"

namespace pradmm {
namespace {

using namespace dev;

// Thread group that owns one graph: the whole CTA or one warp.
struct CtaGroup {
    double* sh;  // 32 doubles of shared scratch for the reductions
    __device__ int rank() const { return threadIdx.x; }
    __device__ int size() const { return blockDim.x; }
    __device__ void sync() const { __syncthreads(); }
    // FP64 sum over the group, returned to every thread (fixed tree)
    __device__ double sum(double v) const {
        const double r = block_sum(v, sh);
        if (threadIdx.x == 0) sh[0] = r;
        __syncthreads();
        const double out = sh[0];
        __syncthreads();
        return out;
    }
};

struct WarpGroup {
    __device__ int rank() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ void sync() const { __syncwarp(); }
    __device__ double sum(double v) const {
        v = warp_sum(v);
        return __shfl_sync(0xffffffffu, v, 0);
    }
};

template <typename R, typename G>
__device__ void solve_graph(const G& grp, const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                            const BatchDev& b, int gid, Ctrl* ctrl) {
    const int64_t v0 = b.gv[gid], v1 = b.gv[gid + 1];
    const int r = grp.rank(), nt = grp.size();
    Acc<R> unused;
    // first p-block: p^1 from x^0 (p^0 in buffer 0)
    for (int64_t i = v0 + r; i < v1; i += nt) sp_vertex<R, false>(g, S, c, S.p[0], S.p[1], i, unused, ctrl);
    grp.sync();
    int k = 0, status = PRADMM_BATCH_MAXITER;
    double e1 = 0.0, e = 0.0;
    while (k < b.max_iter) {
        const R* pcur = S.p[(k + 1) & 1];  // p^{k+1}
        Acc<R> adq, adl, adt, adz;
        for (int64_t i = v0 + r; i < v1; i += nt) q_vertex<R>(g, S, c, pcur, i, adq, adl);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) t_vertex<R>(g, S, c, pcur, i, adt);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) sp_vertex<R, true>(g, S, c, pcur, S.p[k & 1], i, adz, ctrl);
        const double dl = grp.sum(adl.get()), dz = grp.sum(adz.get());
        const double dq = grp.sum(adq.get()), dt = grp.sum(adt.get());
        e = dl / c.b1d + dz / c.b2d + c.b1d * dq + c.b2d * dt;
        ++k;
        if (k == 1) e1 = e;
        grp.sync();
        if (!isfinite(e)) {
            status = PRADMM_BATCH_NONFINITE;
            break;
        }
        if (e <= b.rel_tol * e1 || e < b.abs_tol) {
            status = PRADMM_BATCH_CONVERGED;
            break;
        }
    }
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
    }
}

// Persistent solver: every CTA takes items until the queue is empty.
template <typename R, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch(GraphDev<R> g, StateDev<R> S, Coef<R> c, BatchDev b, Ctrl* ctrl) {
    __shared__ double sh[32];
    __shared__ int s_item;
    const CtaGroup cta{sh};
    const WarpGroup warp;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.next, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= b.n_items) break;
        const int2 item = b.items[it];  // (first position in order, graphs; < 0: one graph for the CTA)
        if (item.y < 0) {
            solve_graph<R>(cta, g, S, c, b, b.order[item.x], ctrl);
        } else {
            const int w = threadIdx.x >> 5;
            if (w < item.y) solve_graph<R>(warp, g, S, c, b, b.order[item.x + w], ctrl);
            __syncthreads();
        }
    }
}

// F of Eq. (1) per graph at (p, t) in double, one CTA per graph (fixed order).
template <typename R>
__global__ void __launch_bounds__(256) k_batch_objective(GraphDev<R> g, StateDev<R> S, const double* __restrict__ qe,
                                                         const double* __restrict__ te, const double* __restrict__ ka,
                                                         const double* __restrict__ om, BatchDev b, double* F) {
    __shared__ double sh[32];
    const int gid = blockIdx.x;
    const int64_t v0 = b.gv[gid], v1 = b.gv[gid + 1];
    double acc = 0.0;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x) acc += objective_vertex<R>(g, S.p[0], S.t, qe, te, ka, om, i);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) F[gid] = tot;
}

}  // namespace

template <typename R>
cudaError_t launch_batch(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const BatchDev& b, Ctrl* ctrl,
                         int grid, int block, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.next, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    switch (block) {
        case 64: k_batch<R, 2><<<grid, 64, 0, st>>>(g, s, c, b, ctrl); break;
        case 128: k_batch<R, 4><<<grid, 128, 0, st>>>(g, s, c, b, ctrl); break;
        case 512: k_batch<R, 16><<<grid, 512, 0, st>>>(g, s, c, b, ctrl); break;
        default: k_batch<R, 8><<<grid, 256, 0, st>>>(g, s, c, b, ctrl); break;
    }
    return cudaGetLastError();
}

template <typename R>
cudaError_t batch_occupancy(int block, int* bps) {
    switch (block) {
        case 64: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<R, 2>, 64, 0);
        case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<R, 4>, 128, 0);
        case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<R, 16>, 512, 0);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<R, 8>, 256, 0);
    }
}

template <typename R>
cudaError_t launch_batch_objective(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64, const double* te64,
                                   const double* ka64, const double* om64, const BatchDev& b, double* F, int G,
                                   cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    k_batch_objective<R><<<G, 256, 0, st>>>(g, s, qe64, te64, ka64, om64, b, F);
    return cudaGetLastError();
}

#define PRADMM_BATCH_INST(R)                                                                                   \
    template cudaError_t launch_batch<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const BatchDev&, \
                                         Ctrl*, int, int, cudaStream_t);                                        \
    template cudaError_t batch_occupancy<R>(int, int*);                                                         \
    template cudaError_t launch_batch_objective<R>(const GraphDev<R>&, const StateDev<R>&, const double*,       \
                                                   const double*, const double*, const double*, const BatchDev&, \
                                                   double*, int, cudaStream_t);

PRADMM_BATCH_INST(float)
PRADMM_BATCH_INST(double)

}  // namespace pradmm
