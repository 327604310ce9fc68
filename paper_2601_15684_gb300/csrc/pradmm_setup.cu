// Set-up kernels of pradmm_create: the per-slot edge records of both CSR
// orders, packed on the device from the caller's measurement arrays (one
// upload of the raw arrays instead of packing and uploading every record
// array from host memory).
//
// A slot k of an edge order holds input edge e = edge[k]:
//   te_out[k] = (t_e, omega_e)            in the state precision
//   qk_out[k] = kappa_e q_e / |q_e|       in the state precision
// and, for the out order, the FP64 measurements of the objective:
//   qe64[k] = q_e / |q_e|, te64[k] = t_e, ka64[k] = kappa_e, om64[k] = omega_e.
// |q_e| is the same sum of squares in the same order as the host's validation,
// so the normalised quaternion is the host's.
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_internal.h"

namespace pradmm {
namespace {

template <typename R>
__global__ void __launch_bounds__(256) k_pack_slots(const int32_t* __restrict__ edge, int64_t slots,
                                                    const double* __restrict__ q, const double* __restrict__ t,
                                                    const double* __restrict__ ka, const double* __restrict__ om,
                                                    R* __restrict__ te_out, R* __restrict__ qk_out,
                                                    double* __restrict__ qe64, double* __restrict__ te64,
                                                    double* __restrict__ ka64, double* __restrict__ om64) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < slots; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = edge[k];
        const double k_e = ka ? ka[e] : 1.0, w_e = om ? om[e] : 1.0;
        double qv[4], nn = 0.0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            qv[c] = q[4 * e + c];
            nn = __dadd_rn(nn, __dmul_rn(qv[c], qv[c]));
        }
        nn = sqrt(nn);
#pragma unroll
        for (int c = 0; c < 4; ++c) qv[c] = qv[c] / nn;
        const double tv[3] = {t[3 * e], t[3 * e + 1], t[3 * e + 2]};
        te_out[4 * k] = R(tv[0]);
        te_out[4 * k + 1] = R(tv[1]);
        te_out[4 * k + 2] = R(tv[2]);
        te_out[4 * k + 3] = R(w_e);
#pragma unroll
        for (int c = 0; c < 4; ++c) qk_out[4 * k + c] = R(k_e * qv[c]);
        if (qe64) {
#pragma unroll
            for (int c = 0; c < 4; ++c) qe64[4 * k + c] = qv[c];
#pragma unroll
            for (int c = 0; c < 3; ++c) te64[3 * k + c] = tv[c];
            ka64[k] = k_e;
            om64[k] = w_e;
        }
    }
}

}  // namespace

template <typename R>
cudaError_t launch_pack_slots(const int32_t* edge, int64_t slots, const double* q, const double* t, const double* ka,
                              const double* om, R* te_out, R* qk_out, double* qe64, double* te64, double* ka64,
                              double* om64, cudaStream_t st) {
    if (slots <= 0) return cudaSuccess;
    const int64_t want = (slots + 255) / 256;
    const int grid = (int)(want < 152 * 8 ? want : 152 * 8);
    k_pack_slots<R><<<grid, 256, 0, st>>>(edge, slots, q, t, ka, om, te_out, qk_out, qe64, te64, ka64, om64);
    return cudaGetLastError();
}

#define PRADMM_SETUP_INST(R)                                                                                     \
    template cudaError_t launch_pack_slots<R>(const int32_t*, int64_t, const double*, const double*,             \
                                              const double*, const double*, R*, R*, double*, double*, double*,  \
                                              double*, cudaStream_t);
PRADMM_SETUP_INST(float)
PRADMM_SETUP_INST(double)

}  // namespace pradmm
