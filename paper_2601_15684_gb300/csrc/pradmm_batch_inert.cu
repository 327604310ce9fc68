// Batched PRADMM, inertial form (proximal anchors x^k + theta (x^k - x^{k-1})):
// the persistent kernels of pradmm_batch.cuh instantiated with INERT = true.
#include "pradmm_batch.cuh"

namespace pradmm {

#define PRADMM_BATCH_INERT_INST(R)                                                                             \
    template cudaError_t launch_batch<R, true>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&,           \
                                               const BatchDev&, Ctrl*, int, int, int, cudaStream_t);             \
    template cudaError_t batch_occupancy<R, true>(int, int*);                                                   \
    template cudaError_t batch_cluster_occupancy<R, true>(int, int, int*);

PRADMM_BATCH_INERT_INST(float)
PRADMM_BATCH_INERT_INST(double)

}  // namespace pradmm
