// Batched PRADMM: many independent pose graphs solved in one persistent
// launch.  The batch is one disjoint-union graph (each graph's vertices are a
// contiguous internal range), so the per-vertex updates are exactly those of
// the plain sweeps (pradmm_device.cuh).  Each CTA of the persistent kernel
// repeatedly takes the next work item from a queue ordered largest first:
//   - a graph item: the whole CTA runs Algorithm 1 on one graph, the three
//     sweeps of an iteration separated by CTA barriers;
//   - a pack item: each warp of the CTA runs Algorithm 1 on its own small
//     graph, sweeps separated by warp barriers.
//   - a cluster item (k_batch_cl only): the CTAs of one thread-block cluster
//     run Algorithm 1 on one large graph together, sweeps separated by
//     cluster barriers (the hardware co-schedules a cluster's CTAs).
// A graph's residual e^k (Appendix E.1) is reduced inside its group, and the
// group stops when e^k <= rel_tol * e^1 (the batch's relative stopping rule),
// e^k < abs_tol, the residual is not finite, or max_iter is reached.  Apart
// from the barriers of its own cluster, no CTA ever waits for another CTA.
//
// This header holds the persistent kernels, templated on a policy that solves
// one graph with a group (the plain iteration here, general weights in
// pradmm_batch_sigma.cu), and the plain iteration's launchers as templates on
// INERT (the inertial variant: proximal anchors x^k + theta (x^k - x^{k-1}),
// the previous iterates in S.qprev, S.tprev, S.sprev, each solve starting
// afresh with x^{-1} = x^0).  pradmm_batch.cu instantiates the plain form and
// pradmm_batch_inert.cu the inertial one, so they compile in parallel.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_device.cuh"
#include "pradmm_internal.h"

namespace pradmm {
namespace {

using namespace dev;

// Sums of four values over a warp by reduce-scatter, in FP64 with a fixed
// tree: the first butterfly step splits the values between the half warps,
// the second between quarter... (lanes 0-7 keep value 0, 8-15 value 1, 16-23
// value 2, 24-31 value 3), the last three steps are a butterfly on the one
// value a lane keeps: 6 FP64 additions per lane instead of 20 for four
// separate trees.  Lane 0 ends with all four totals in v.
__device__ __forceinline__ void warp_sum4(double* v) {
    constexpr unsigned kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool hi = lane >= 16, odd = (lane & 8) != 0;
    // step 16: keep (0, 1) in the low half, (2, 3) in the high half
    const double s0 = hi ? v[0] : v[2], s1 = hi ? v[1] : v[3];
    const double r0 = __shfl_xor_sync(kAll, s0, 16), r1 = __shfl_xor_sync(kAll, s1, 16);
    const double k0 = (hi ? v[2] : v[0]) + r0, k1 = (hi ? v[3] : v[1]) + r1;
    // step 8: keep the first of the pair in lanes with bit 3 clear, else the second
    const double s = odd ? k0 : k1;
    double x = (odd ? k1 : k0) + __shfl_xor_sync(kAll, s, 8);
    x += __shfl_xor_sync(kAll, x, 4);
    x += __shfl_xor_sync(kAll, x, 2);
    x += __shfl_xor_sync(kAll, x, 1);
    // lanes 0, 8, 16, 24 hold the totals of values 0..3
    const double t1 = __shfl_sync(kAll, x, 8), t2 = __shfl_sync(kAll, x, 16), t3 = __shfl_sync(kAll, x, 24);
    v[0] = x;
    v[1] = t1;
    v[2] = t2;
    v[3] = t3;
}

// Four CTA totals (thread 0 gets them) from warp_sum4 in every warp and
// again over the warp totals; sh holds 4 x 32 doubles.
__device__ __forceinline__ void block_sum4_rs(double* v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    warp_sum4(v);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 4; ++k) sh[32 * k + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = lane < nw ? sh[32 * k + lane] : 0.0;
        warp_sum4(v);
    }
    __syncthreads();
}

// Thread group that owns one graph: the whole CTA or one warp.
struct CtaGroup {
    double* sh;  // 4 x 32 doubles of shared scratch for the reductions
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
    // e^k from the four residual parts (dlam, dz, dq, dt): one CTA reduction
    // (each part with sum()'s tree), e formed by thread 0 and broadcast
    __device__ double residual(double* v, double b1, double b2) const {
        block_sum4_rs(v, sh);
        if (threadIdx.x == 0) sh[0] = v[0] / b1 + v[1] / b2 + b1 * v[2] + b2 * v[3];
        __syncthreads();
        const double e = sh[0];
        __syncthreads();
        return e;
    }
    // after residual(): its barriers already follow every write of the iteration
    __device__ void sync_after_sum() const {}
};

struct WarpGroup {
    __device__ int rank() const { return threadIdx.x & 31; }
    __device__ int size() const { return 32; }
    __device__ void sync() const { __syncwarp(); }
    __device__ double sum(double v) const {
        v = warp_sum(v);
        return __shfl_sync(0xffffffffu, v, 0);
    }
    // e^k from the four residual parts: lane 0 holds the totals, forms e and
    // broadcasts it
    __device__ double residual(double* v, double b1, double b2) const {
        warp_sum4(v);
        double e = 0.0;
        if ((threadIdx.x & 31) == 0) e = v[0] / b1 + v[1] / b2 + b1 * v[2] + b2 * v[3];
        return __shfl_sync(0xffffffffu, e, 0);
    }
    // shuffles do not order memory: a warp barrier after the sums
    __device__ void sync_after_sum() const { __syncwarp(); }
};

// The CTAs of one thread-block cluster.  A sum is each CTA's fixed-tree total
// written into slot [cta rank] of every CTA's shared array (distributed shared
// memory), then added in rank order after a cluster barrier: every thread gets
// the same double.  Slots alternate between two banks, so a bank is rewritten
// only after the barrier of the next sum has passed.
constexpr int kMaxCluster = 16;
struct ClusterGroup {
    double* sh;       // 4 x 32 doubles of shared scratch (CTA reductions)
    double* slots;    // 2 * kMaxCluster * 4 doubles in this CTA's shared memory
    int* bank;        // this CTA's bank toggle (shared)
    __device__ int rank() const {
        return (int)cooperative_groups::this_cluster().block_rank() * blockDim.x + threadIdx.x;
    }
    __device__ int size() const { return (int)cooperative_groups::this_cluster().num_blocks() * blockDim.x; }
    __device__ void sync() const { cooperative_groups::this_cluster().sync(); }
    // e^k from the four residual parts with one exchange: thread 0 of every
    // CTA adds the CTA totals in rank order, forms e and broadcasts it
    __device__ double residual(double* v, double b1, double b2) const {
        auto cl = cooperative_groups::this_cluster();
        double cta[4] = {v[0], v[1], v[2], v[3]};
        block_sum4_rs(cta, sh);  // thread 0 holds the CTA totals
        const int b = *bank;
        const unsigned me = cl.block_rank(), nb = cl.num_blocks();
        if (threadIdx.x == 0)
            for (unsigned r = 0; r < nb; ++r) {
                double* dst = cl.map_shared_rank(slots, r) + (b * kMaxCluster + me) * 4;
                for (int k = 0; k < 4; ++k) dst[k] = cta[k];
            }
        cl.sync();
        if (threadIdx.x == 0) {
            double tot[4];
            for (int k = 0; k < 4; ++k) {
                tot[k] = 0.0;
                for (unsigned r = 0; r < nb; ++r) tot[k] += slots[(b * kMaxCluster + r) * 4 + k];
            }
            sh[0] = tot[0] / b1 + tot[1] / b2 + b1 * tot[2] + b2 * tot[3];
            *bank = b ^ 1;
        }
        __syncthreads();
        const double e = sh[0];
        __syncthreads();
        return e;
    }
    // after residual(): its cluster barrier already follows every write of the iteration
    __device__ void sync_after_sum() const {}
};

__device__ __forceinline__ unsigned long long clock_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename R, bool INERT, typename G>
__device__ void solve_graph(const G& grp, const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                            const BatchDev& b, int gid, Ctrl* ctrl) {
    const int64_t v0 = b.gv[gid], v1 = b.gv[gid + 1];
    const int r = grp.rank(), nt = grp.size();
    if (r == 0) b.t_span[2 * gid] = clock_ns();
    Acc<R> unused;
    // first p-block: p^1 from x^0 (p^0 in buffer 0); INERT: x^{-1} := x^0
    for (int64_t i = v0 + r; i < v1; i += nt) {
        sp_vertex<R, false>(g, S, c, S.p[0], S.p[1], i, unused, ctrl);
        if (INERT) {
            const R4<R> q0 = IO<R>::ld(S.q, i), t0 = IO<R>::ld(S.t, i), s0 = IO<R>::ld(S.s, i);
            IO<R>::st(S.qprev, i, q0.a, q0.b, q0.c, q0.d);
            IO<R>::st(S.tprev, i, t0.a, t0.b, t0.c, t0.d);
            IO<R>::st(S.sprev, i, s0.a, s0.b, s0.c, s0.d);
        }
    }
    grp.sync();
    int k = 0, status = PRADMM_BATCH_MAXITER;
    double e1 = 0.0, e = 0.0;
    const int cap = b.iter_cap ? b.iter_cap[gid] : b.max_iter;
    while (k < cap) {
        const R* pcur = S.p[(k + 1) & 1];  // p^{k+1}
        Acc<R> adq, adl, adt, adz;
        for (int64_t i = v0 + r; i < v1; i += nt) q_vertex<R, false, false, INERT>(g, S, c, pcur, i, adq, adl);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) t_vertex<R, false, false, INERT>(g, S, c, pcur, i, adt);
        grp.sync();
        for (int64_t i = v0 + r; i < v1; i += nt) sp_vertex<R, true, false, false, INERT>(g, S, c, pcur, S.p[k & 1], i, adz, ctrl);
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

// The plain iteration as a batch policy: solves graph gid with group grp.
template <typename R, bool INERT>
struct PlainSolve {
    GraphDev<R> g;
    StateDev<R> S;
    Coef<R> c;
    template <typename G>
    __device__ __forceinline__ void operator()(const G& grp, const BatchDev& b, int gid, Ctrl* ctrl) const {
        solve_graph<R, INERT>(grp, g, S, c, b, gid, ctrl);
    }
};

// Persistent solver: every CTA takes items until the queue is empty.  Policy
// P solves one graph with a group (PlainSolve here; general weights in
// pradmm_batch_sigma.cu).
template <typename P, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch(P solve, BatchDev b, Ctrl* ctrl) {
    __shared__ double sh[4 * 32];
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
            solve(cta, b, b.order[item.x], ctrl);
        } else {
            const int w = threadIdx.x >> 5;
            if (w < item.y) solve(warp, b, b.order[item.x + w], ctrl);
            __syncthreads();
        }
    }
}

// Persistent solver with clusters: each cluster first takes cluster items
// (graphs too large for one CTA) from their queue, largest first; once that
// queue is empty every CTA takes the CTA and warp-pack items as k_batch does.
template <typename P, int WPB>
__global__ void __launch_bounds__(WPB * 32) k_batch_cl(P solve, BatchDev b, Ctrl* ctrl) {
    __shared__ double sh[4 * 32];
    __shared__ double slots[2 * kMaxCluster * 4];
    __shared__ int s_item, s_bank;
    auto cl = cooperative_groups::this_cluster();
    if (threadIdx.x == 0) s_bank = 0;
    const ClusterGroup cgp{sh, slots, &s_bank};
    for (;;) {
        if (cl.block_rank() == 0 && threadIdx.x == 0) s_item = atomicAdd(b.next_big, 1);
        cl.sync();
        const int it = *cl.map_shared_rank(&s_item, 0);
        cl.sync();  // every CTA has read the item before rank 0 fetches the next
        if (it >= b.n_big) break;
        solve(cgp, b, b.order[it], ctrl);
    }
    const CtaGroup cta{sh};
    const WarpGroup warp;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.next, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();
        if (it >= b.n_items) break;
        const int2 item = b.items[it];
        if (item.y < 0) {
            solve(cta, b, b.order[item.x], ctrl);
        } else {
            const int w = threadIdx.x >> 5;
            if (w < item.y) solve(warp, b, b.order[item.x + w], ctrl);
            __syncthreads();
        }
    }
    cl.sync();  // no CTA leaves while a peer could still address its shared memory
}

template <typename P, int WPB>
cudaError_t launch_cl(const P& solve, const BatchDev& b, Ctrl* ctrl, int grid, int cluster, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(WPB * 32);
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_batch_cl<P, WPB>, solve, b, ctrl);
}

template <typename P, int WPB>
cudaError_t occupancy_cl(int cluster, int* clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3(WPB * 32);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cluster;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, k_batch_cl<P, WPB>, &cfg);
}

// One persistent launch of policy P: cluster > 1 the cluster kernel (grid a
// multiple of cluster), else k_batch; block 64, 128, 256 or 512.
template <typename P>
cudaError_t launch_persistent(const P& solve, const BatchDev& b, Ctrl* ctrl, int grid, int block, int cluster,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(b.next, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (cluster > 1) {
        if ((e = cudaMemsetAsync(b.next_big, 0, sizeof(int), st)) != cudaSuccess) return e;
        switch (block) {
            case 64: return launch_cl<P, 2>(solve, b, ctrl, grid, cluster, st);
            case 128: return launch_cl<P, 4>(solve, b, ctrl, grid, cluster, st);
            case 512: return launch_cl<P, 16>(solve, b, ctrl, grid, cluster, st);
            default: return launch_cl<P, 8>(solve, b, ctrl, grid, cluster, st);
        }
    }
    switch (block) {
        case 64: k_batch<P, 2><<<grid, 64, 0, st>>>(solve, b, ctrl); break;
        case 128: k_batch<P, 4><<<grid, 128, 0, st>>>(solve, b, ctrl); break;
        case 512: k_batch<P, 16><<<grid, 512, 0, st>>>(solve, b, ctrl); break;
        default: k_batch<P, 8><<<grid, 256, 0, st>>>(solve, b, ctrl); break;
    }
    return cudaGetLastError();
}

template <typename P>
cudaError_t persistent_occupancy(int block, int* bps) {
    switch (block) {
        case 64: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<P, 2>, 64, 0);
        case 128: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<P, 4>, 128, 0);
        case 512: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<P, 16>, 512, 0);
        default: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, k_batch<P, 8>, 256, 0);
    }
}

template <typename P>
cudaError_t persistent_cluster_occupancy(int block, int cluster, int* clusters) {
    switch (block) {
        case 64: return occupancy_cl<P, 2>(cluster, clusters);
        case 128: return occupancy_cl<P, 4>(cluster, clusters);
        case 512: return occupancy_cl<P, 16>(cluster, clusters);
        default: return occupancy_cl<P, 8>(cluster, clusters);
    }
}

}  // namespace

template <typename R, bool INERT>
cudaError_t launch_batch(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const BatchDev& b, Ctrl* ctrl,
                         int grid, int block, int cluster, cudaStream_t st) {
    return launch_persistent(PlainSolve<R, INERT>{g, s, c}, b, ctrl, grid, block, cluster, st);
}

template <typename R, bool INERT>
cudaError_t batch_occupancy(int block, int* bps) {
    return persistent_occupancy<PlainSolve<R, INERT>>(block, bps);
}

template <typename R, bool INERT>
cudaError_t batch_cluster_occupancy(int block, int cluster, int* clusters) {
    return persistent_cluster_occupancy<PlainSolve<R, INERT>>(block, cluster, clusters);
}

}  // namespace pradmm
