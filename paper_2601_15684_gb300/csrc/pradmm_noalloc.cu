// pradmm_objective_noalloc: the objective F of Eq. (1) for poses and
// measurements that already live in device memory, computed without
// allocating any memory.
//
// Some callers cannot allocate device memory at the time they need the
// objective: a real-time or safety-constrained process that reserves all of
// its GPU memory at start-up and forbids allocation afterwards (a cudaMalloc
// can synchronise the device and stall a control loop), or an application
// whose memory pool already owns the whole device.  The regular path
// (pradmm_objective) needs a handle, and a handle allocates.  This entry
// point takes the caller's device arrays and writes F to a caller-provided
// device double; the only scratch it needs -- one FP64 partial sum per chunk
// of kChunkEdges edges and an arrival counter -- lives in the file-scope array
// g_objective_scratch below.  The array belongs to the library's device code:
// a GPU receives it when that code is loaded onto it (under CUDA's lazy
// module loading, at the first launch or symbol lookup on that GPU, which
// itself allocates and may synchronise) and keeps it until process exit.
// The first call on each GPU therefore belongs to the caller's start-up;
// later calls allocate nothing.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <mutex>

#include "pradmm.h"
#include "pradmm_internal.h"

namespace {

constexpr int kChunkEdges = 1024;    // edges summed into one partial
constexpr int kMaxChunks = 4096;     // partials the scratch holds
constexpr int kThreads = 256;
constexpr int64_t kMaxEdges = (int64_t)kChunkEdges * kMaxChunks;  // 4,194,304 edges per call
constexpr size_t kTicketOffset = sizeof(double) * kMaxChunks;     // byte offset of the counter
constexpr size_t kScratchBytes = kTicketOffset + 256;             // 32 KiB + 256 B

static __device__ __align__(256) unsigned char g_objective_scratch[kScratchBytes];

void fail_msg(const char* msg) { pradmm::set_last_error(msg); }

// Device address of g_objective_scratch, looked up once per device (with
// that device current).  In host code the symbol's name is only a host-side
// stand-in, so the kernel must be given this address, never the name.
std::mutex g_mu;
void* g_scratch_ptr[64] = {};

pradmm_status scratch_for_current_device(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    char buf[160];
    if (e != cudaSuccess) {
        std::snprintf(buf, sizeof(buf), "cudaGetDevice: %s", cudaGetErrorString(e));
        fail_msg(buf);
        return PRADMM_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) {
        std::snprintf(buf, sizeof(buf), "device %d is beyond the 64 devices this entry point tracks", dev);
        fail_msg(buf);
        return PRADMM_ERR_ARG;
    }
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_objective_scratch);
        if (e != cudaSuccess || !p) {
            std::snprintf(buf, sizeof(buf), "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
            fail_msg(buf);
            return PRADMM_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    return PRADMM_OK;
}

struct Qd {
    double w, x, y, z;
};

__device__ __forceinline__ Qd qmul(const Qd& a, const Qd& b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z, a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x, a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    }
    __syncthreads();
    return r;
}

// CTA c sums the terms of edges [c*kChunkEdges, (c+1)*kChunkEdges) into
// partial[c]; the last CTA to finish adds the partials in chunk order, so
// the result does not depend on scheduling.
//   F += w_e |t~_j - t~_i - q_i t~_e q_i^*|^2 + k_e |q_j^* q_i q_e - 1|^2
// An edge whose endpoint lies outside [0, n) is skipped (no pose is read for
// it) and its chunk's partial becomes NaN, so F comes back NaN.
__global__ void __launch_bounds__(kThreads) k_objective_noalloc(int64_t n, int64_t m, const int32_t* __restrict__ src,
                                                                const int32_t* __restrict__ dst,
                                                                const double* __restrict__ qe,
                                                                const double* __restrict__ te,
                                                                const double* __restrict__ ka,
                                                                const double* __restrict__ om,
                                                                const double* __restrict__ q,
                                                                const double* __restrict__ t, double* F,
                                                                unsigned char* scratch) {
    __shared__ double sh[32];
    __shared__ bool last;
    double* partial = reinterpret_cast<double*>(scratch);
    unsigned int* ticket = reinterpret_cast<unsigned int*>(scratch + kTicketOffset);
    const int64_t e0 = (int64_t)blockIdx.x * kChunkEdges;
    const int64_t e1 = e0 + kChunkEdges < m ? e0 + kChunkEdges : m;
    double acc = 0.0;
    bool bad = false;
    for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int64_t i = src[e], j = dst[e];
        if (i < 0 || i >= n || j < 0 || j >= n) {
            bad = true;
            continue;
        }
        const Qd qi = {q[4 * i], q[4 * i + 1], q[4 * i + 2], q[4 * i + 3]};
        const Qd qj = {q[4 * j], q[4 * j + 1], q[4 * j + 2], q[4 * j + 3]};
        const Qd tp = {0.0, te[3 * e], te[3 * e + 1], te[3 * e + 2]};
        const Qd qic = {qi.w, -qi.x, -qi.y, -qi.z};
        const Qd rot = qmul(qmul(qi, tp), qic);
        const double r0 = -rot.w;
        const double r1 = t[3 * j] - t[3 * i] - rot.x;
        const double r2 = t[3 * j + 1] - t[3 * i + 1] - rot.y;
        const double r3 = t[3 * j + 2] - t[3 * i + 2] - rot.z;
        acc += (om ? om[e] : 1.0) * (r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
        const Qd qq = {qe[4 * e], qe[4 * e + 1], qe[4 * e + 2], qe[4 * e + 3]};
        const Qd qjc = {qj.w, -qj.x, -qj.y, -qj.z};
        Qd h = qmul(qmul(qjc, qi), qq);
        h.w -= 1.0;
        acc += (ka ? ka[e] : 1.0) * (h.w * h.w + h.x * h.x + h.y * h.y + h.z * h.z);
    }
    if (bad) acc = __longlong_as_double(0x7ff8000000000000ll);  // quiet NaN
    const double bs = block_sum(acc, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
    __threadfence();
    if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double v = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(partial + b);
    const double tot = block_sum(v, sh);
    if (threadIdx.x == 0) {
        *F = tot;
        *ticket = 0u;
    }
}

}  // namespace

extern "C" pradmm_status pradmm_objective_noalloc(int64_t n, int64_t m, const int32_t* src_d, const int32_t* dst_d,
                                                  const double* q_meas_d, const double* t_meas_d,
                                                  const double* kappa_d, const double* omega_d, const double* q_d,
                                                  const double* t_d, double* F_d, void* cuda_stream) {
    char buf[160];
    if (n < 1 || m < 0 || n > INT32_MAX - 1) {
        fail_msg("need 1 <= n < 2^31 - 1 and m >= 0");
        return PRADMM_ERR_ARG;
    }
    if (m > kMaxEdges) {
        std::snprintf(buf, sizeof(buf), "m = %lld exceeds the %lld edges the static scratch of this entry point holds",
                      (long long)m, (long long)kMaxEdges);
        fail_msg(buf);
        return PRADMM_ERR_ARG;
    }
    if (!q_d || !t_d || !F_d || (m > 0 && (!src_d || !dst_d || !q_meas_d || !t_meas_d))) {
        fail_msg("NULL device pointer");
        return PRADMM_ERR_ARG;
    }
    unsigned char* scratch = nullptr;
    pradmm_status st = scratch_for_current_device(&scratch);
    if (st != PRADMM_OK) return st;
    cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
    // the arrival counter must start at zero; the partials are all rewritten
    cudaError_t e = cudaMemsetAsync(scratch + kTicketOffset, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) {
        const int chunks = m > 0 ? (int)((m + kChunkEdges - 1) / kChunkEdges) : 1;
        k_objective_noalloc<<<chunks, kThreads, 0, stream>>>(n, m, src_d, dst_d, q_meas_d, t_meas_d, kappa_d, omega_d,
                                                              q_d, t_d, F_d, scratch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        std::snprintf(buf, sizeof(buf), "launch: %s", cudaGetErrorString(e));
        fail_msg(buf);
        return PRADMM_ERR_CUDA;
    }
    return PRADMM_OK;
}
