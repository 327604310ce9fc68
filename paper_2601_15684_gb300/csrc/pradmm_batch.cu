// Batched PRADMM, plain form: the persistent kernels of pradmm_batch.cuh
// instantiated without the inertial anchors, and the per-graph objective.
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_batch.cuh"
#include "pradmm_sigma.cuh"

namespace pradmm {
namespace {

using namespace dev;

// F of Eq. (1) per graph at (p, t) in double, one CTA per graph (fixed order);
// with S1, S2 (device, 16 doubles each) the Sigma-weighted norms.
template <typename R>
__global__ void __launch_bounds__(256) k_batch_objective(GraphDev<R> g, StateDev<R> S, const double* __restrict__ qe,
                                                         const double* __restrict__ te, const double* __restrict__ ka,
                                                         const double* __restrict__ om, const double* __restrict__ S1,
                                                         const double* __restrict__ S2, BatchDev b, double* F) {
    __shared__ double sh[32];
    const int gid = blockIdx.x;
    const int64_t v0 = b.gv[gid], v1 = b.gv[gid + 1];
    double acc = 0.0;
    for (int64_t i = v0 + threadIdx.x; i < v1; i += blockDim.x)
        acc += S1 ? objective_sig_vertex<R>(g, S.p[0], S.t, qe, te, ka, om, S1, S2, i)
                  : objective_vertex<R>(g, S.p[0], S.t, qe, te, ka, om, i);
    const double tot = block_sum(acc, sh);
    if (threadIdx.x == 0) F[gid] = tot;
}

}  // namespace

template <typename R>
cudaError_t launch_batch_objective(const GraphDev<R>& g, const StateDev<R>& s, const double* qe64, const double* te64,
                                   const double* ka64, const double* om64, const double* S1, const double* S2,
                                   const BatchDev& b, double* F, int G, cudaStream_t st) {
    if (G <= 0) return cudaSuccess;
    k_batch_objective<R><<<G, 256, 0, st>>>(g, s, qe64, te64, ka64, om64, S1, S2, b, F);
    return cudaGetLastError();
}

#define PRADMM_BATCH_INST(R)                                                                                   \
    template cudaError_t launch_batch<R, false>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&,          \
                                                const BatchDev&, Ctrl*, int, int, int, cudaStream_t);            \
    template cudaError_t batch_occupancy<R, false>(int, int*);                                                  \
    template cudaError_t batch_cluster_occupancy<R, false>(int, int, int*);                                     \
    template cudaError_t launch_batch_objective<R>(const GraphDev<R>&, const StateDev<R>&, const double*,       \
                                                   const double*, const double*, const double*, const double*,   \
                                                   const double*, const BatchDev&, double*, int, cudaStream_t);

PRADMM_BATCH_INST(float)
PRADMM_BATCH_INST(double)

}  // namespace pradmm
