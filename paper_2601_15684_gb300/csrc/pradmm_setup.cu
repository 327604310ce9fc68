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

// In-order records from the out-order FP64 copies: in-slot k holds input edge
// ie[k], whose out-slot is edge_slot[ie[k]]; the values are those k_pack_slots
// formed there (the normalised q_e among them), so both orders hold the same
// bits without a second normalisation.
template <typename R>
__global__ void __launch_bounds__(256) k_pack_in(const int32_t* __restrict__ ie, const int32_t* __restrict__ edge_slot,
                                                 int64_t slots, const double* __restrict__ qe64,
                                                 const double* __restrict__ te64, const double* __restrict__ ka64,
                                                 const double* __restrict__ om64, R* __restrict__ te_out,
                                                 R* __restrict__ qk_out) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < slots; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = edge_slot[ie[k]];
        const double k_e = ka64[o];
        te_out[4 * k] = R(te64[3 * o]);
        te_out[4 * k + 1] = R(te64[3 * o + 1]);
        te_out[4 * k + 2] = R(te64[3 * o + 2]);
        te_out[4 * k + 3] = R(om64[o]);
#pragma unroll
        for (int c = 0; c < 4; ++c) qk_out[4 * k + c] = R(k_e * qe64[4 * o + c]);
    }
}

// ---- CSR of one edge order on the device ------------------------------------
// ptr[k + 1] counts the edges with key k; an inclusive scan of ptr[1 .. n]
// turns the counts into row offsets; each edge takes a slot of its row by an
// atomic ticket, and each row is then sorted by edge id, so a vertex's slots
// hold its edges in input order (the order every per-vertex sum uses).
__global__ void __launch_bounds__(256) k_degree(const int32_t* __restrict__ key, int64_t m, int32_t* cnt1) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(cnt1 + key[e], 1);
}

constexpr int kScanBlock = 1024;  // elements per CTA of the scan (256 threads x 4)

__device__ __forceinline__ int32_t warp_incl(int32_t v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

// Inclusive scan of a[0, len) within blocks of kScanBlock; block totals to sums.
__global__ void __launch_bounds__(256) k_scan_blocks(int32_t* a, int64_t len, int32_t* sums) {
    __shared__ int32_t wsum[8];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + 4 * (int64_t)threadIdx.x;
    int32_t v[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) v[j] = base + j < len ? a[base + j] : 0;
    v[1] += v[0];
    v[2] += v[1];
    v[3] += v[2];
    const int32_t tot = v[3];
    int32_t inc = warp_incl(tot);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 31) wsum[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int32_t w = lane < 8 ? wsum[lane] : 0;
        w = warp_incl(w);
        if (lane < 8) wsum[lane] = w;
    }
    __syncthreads();
    const int32_t off = inc - tot + (wid > 0 ? wsum[wid - 1] : 0);
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (base + j < len) a[base + j] = v[j] + off;
    if (threadIdx.x == 0) sums[blockIdx.x] = wsum[7];
}

// One CTA: inclusive scan of the block totals, in chunks of 256.
__global__ void __launch_bounds__(256) k_scan_sums(int32_t* sums, int64_t nb) {
    __shared__ int32_t wsum[8];
    __shared__ int32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t c0 = 0; c0 < nb; c0 += 256) {
        const int64_t i = c0 + threadIdx.x;
        const int32_t x = i < nb ? sums[i] : 0;
        const int32_t inc = warp_incl(x);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        if (lane == 31) wsum[wid] = inc;
        __syncthreads();
        if (wid == 0) {
            int32_t w = lane < 8 ? wsum[lane] : 0;
            w = warp_incl(w);
            if (lane < 8) wsum[lane] = w;
        }
        __syncthreads();
        const int32_t val = inc + (wid > 0 ? wsum[wid - 1] : 0) + carry;
        if (i < nb) sums[i] = val;
        __syncthreads();
        if (threadIdx.x == 255) carry = val;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_scan_add(int32_t* a, int64_t len, const int32_t* __restrict__ sums) {
    const int64_t b = blockIdx.x;
    if (b == 0) return;
    const int32_t off = sums[b - 1];
    const int64_t base = b * kScanBlock;
    for (int j = threadIdx.x; j < kScanBlock; j += blockDim.x)
        if (base + j < len) a[base + j] += off;
}

__global__ void __launch_bounds__(256) k_place(const int32_t* __restrict__ key, int64_t m,
                                               const int32_t* __restrict__ ptr, int32_t* fill, int32_t* slot_edge) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = key[e];
        slot_edge[ptr[k] + atomicAdd(fill + k, 1)] = (int32_t)e;
    }
}

// Each row sorted by edge id (insertion sort: rows are short; a hub's row
// costs its degree squared in one thread).
__global__ void __launch_bounds__(256) k_sort_rows(const int32_t* __restrict__ ptr, int64_t n, int32_t* slot_edge) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = ptr[v], b = ptr[v + 1];
        for (int32_t i = a + 1; i < b; ++i) {
            const int32_t x = slot_edge[i];
            int32_t j = i - 1;
            while (j >= a && slot_edge[j] > x) {
                slot_edge[j + 1] = slot_edge[j];
                --j;
            }
            slot_edge[j + 1] = x;
        }
    }
}

__global__ void __launch_bounds__(256) k_slot_other(const int32_t* __restrict__ slot_edge, int64_t m,
                                                    const int32_t* __restrict__ other, int32_t* idx,
                                                    int32_t* edge_slot) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t e = slot_edge[k];
        idx[k] = other[e];
        if (edge_slot) edge_slot[e] = (int32_t)k;
    }
}

// 1/A_2, 1/A_3, 1/A_4 of every vertex (Appendix B with scalar Sigma), summed
// over its slots in input order with unfused FP64 operations (the same
// rounding as a host loop without contraction).
__global__ void __launch_bounds__(256) k_block_inv(const int32_t* __restrict__ out_ptr, const int32_t* __restrict__ out_edge,
                                                   const int32_t* __restrict__ in_ptr, const int32_t* __restrict__ in_edge,
                                                   int64_t n, const double* __restrict__ t, const double* __restrict__ ka,
                                                   const double* __restrict__ om, double a2_0, double a3_0, double a4_0,
                                                   double* inv2, double* inv3, double* inv4) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double A2 = a2_0, A3 = a3_0, A4 = a4_0;
        for (int32_t k = out_ptr[i]; k < out_ptr[i + 1]; ++k) {
            const int64_t e = out_edge[k];
            const double w = om ? om[e] : 1.0, kk = ka ? ka[e] : 1.0;
            const double x = t[3 * e], y = t[3 * e + 1], z = t[3 * e + 2];
            const double tn2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
            A2 = __dadd_rn(A2, __dmul_rn(2.0, __dadd_rn(__dmul_rn(w, tn2), kk)));
            A4 = __dadd_rn(A4, __dmul_rn(2.0, w));
        }
        for (int32_t k = in_ptr[i]; k < in_ptr[i + 1]; ++k) {
            const int64_t e = in_edge[k];
            A3 = __dadd_rn(A3, __dmul_rn(2.0, om ? om[e] : 1.0));
        }
        inv2[i] = 1.0 / A2;
        inv3[i] = 1.0 / A3;
        inv4[i] = 1.0 / A4;
    }
}

__global__ void __launch_bounds__(256) k_iota(int32_t* a, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = (int32_t)i;
}

__global__ void __launch_bounds__(256) k_slot_owner(const int32_t* __restrict__ ptr, int64_t n, int32_t* owner) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        for (int32_t k = ptr[i]; k < ptr[i + 1]; ++k) owner[k] = (int32_t)i;
}

// ---- validation of the caller's edges ----------------------------------------
// The checks of pradmm_create, edge by edge: endpoints in [0, n) and distinct,
// weights finite and > 0, measurements finite, |q_e| within 1e-6 of 1 (the
// squared norm summed in component order with separate roundings, as a host
// loop without contraction forms it, then the correctly rounded square root);
// *first_bad = the lowest failing edge (m when none fails).
__global__ void __launch_bounds__(256) k_validate(const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                                                  const double* __restrict__ q, const double* __restrict__ t,
                                                  const double* __restrict__ ka, const double* __restrict__ om,
                                                  int64_t n, int64_t m, int32_t* first_bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        bool ok = a >= 0 && a < n && b >= 0 && b < n && a != b;
        const double k_e = ka ? ka[e] : 1.0, w_e = om ? om[e] : 1.0;
        ok = ok && isfinite(k_e) && isfinite(w_e) && k_e > 0.0 && w_e > 0.0;
        double nn = 0.0;
        for (int c = 0; c < 4; ++c) nn = __dadd_rn(nn, __dmul_rn(q[4 * e + c], q[4 * e + c]));
        ok = ok && isfinite(nn) && isfinite(t[3 * e]) && isfinite(t[3 * e + 1]) && isfinite(t[3 * e + 2]);
        ok = ok && fabs(__dadd_rn(__dsqrt_rn(nn), -1.0)) <= 1e-6;
        if (!ok) atomicMin(first_bad, (int32_t)e);
    }
}

// The endpoint checks alone, before the measurements have arrived: an edge
// with an endpoint outside [0, n) or a self-loop lowers *first_bad, and an
// endpoint outside [0, n) is replaced by 0, so the structure kernels that
// follow (CSR, spanning forest) stay in bounds whatever the caller passed;
// the handle is discarded when *first_bad < m after the full checks.
__global__ void __launch_bounds__(256) k_check_ends(int32_t* src, int32_t* dst, int64_t n, int64_t m,
                                                    int32_t* first_bad) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t a = src[e], b = dst[e];
        const bool ia = a >= 0 && a < n, ib = b >= 0 && b < n;
        if (!(ia && ib && a != b)) {
            atomicMin(first_bad, (int32_t)e);
            if (!ia) src[e] = 0;
            if (!ib) dst[e] = 0;
        }
    }
}

// ---- odometry composition on the device -----------------------------------
// The spanning forest (pradmm_forest.cu) gives every vertex its parent and the tree edge
// to it; the pose of a vertex is the composition of the SE(3) steps along the
// tree path from its component's root, T_v = T_parent o T_step with
// (q_a, t_a) o (q_b, t_b) = (q_a q_b, t_a + R(q_a) t_b), composed by pointer
// jumping in segments of tree levels (below).
__device__ __forceinline__ void hq_mul(const double* a, const double* b, double* o) {
    const double w = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    const double x = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    const double y = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    const double z = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
    o[0] = w;
    o[1] = x;
    o[2] = y;
    o[3] = z;
}

// R(q) v through the rotation matrix of a unit quaternion
__device__ __forceinline__ void hq_rot(const double* q, const double* v, double* o) {
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    const double r00 = 1 - 2 * (y * y + z * z), r01 = 2 * (x * y - w * z), r02 = 2 * (x * z + w * y);
    const double r10 = 2 * (x * y + w * z), r11 = 1 - 2 * (x * x + z * z), r12 = 2 * (y * z - w * x);
    const double r20 = 2 * (x * z - w * y), r21 = 2 * (y * z + w * x), r22 = 1 - 2 * (x * x + y * y);
    o[0] = r00 * v[0] + r01 * v[1] + r02 * v[2];
    o[1] = r10 * v[0] + r11 * v[1] + r12 * v[2];
    o[2] = r20 * v[0] + r21 * v[1] + r22 * v[2];
}

// Step of every vertex from its parent: the edge (parent, v) gives (q_e, t_e);
// the edge (v, parent) gives its inverse (q_e^*, -R(q_e^*) t_e).  pedge[v]:
// e for (parent, v), -(e + 2) for (v, parent), -1 for a root.
__global__ void __launch_bounds__(256) k_odo_steps(const int32_t* __restrict__ pedge, const int32_t* __restrict__ edge_slot,
                                                   const double* __restrict__ qe64, const double* __restrict__ te64,
                                                   int64_t n, double* q, double* t) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t code = pedge[v];
        double qv[4] = {1.0, 0.0, 0.0, 0.0}, tv[3] = {0.0, 0.0, 0.0};
        if (code != -1) {
            const bool tail = code < -1;
            const int64_t s = edge_slot[tail ? -(int64_t)code - 2 : code];
            const double* qq = qe64 + 4 * s;
            const double* tt = te64 + 3 * s;
            if (tail) {  // the inverse step
                qv[0] = qq[0];
                qv[1] = -qq[1];
                qv[2] = -qq[2];
                qv[3] = -qq[3];
                double r[3];
                hq_rot(qv, tt, r);
                tv[0] = -r[0];
                tv[1] = -r[1];
                tv[2] = -r[2];
            } else {
                for (int c = 0; c < 4; ++c) qv[c] = qq[c];
                for (int c = 0; c < 3; ++c) tv[c] = tt[c];
            }
        }
        for (int c = 0; c < 4; ++c) q[4 * v + c] = qv[c];
        for (int c = 0; c < 3; ++c) t[3 * v + c] = tv[c];
    }
}

// (q_a, t_a) o (q_b, t_b) into (qo, to)
__device__ __forceinline__ void se3_compose(const double* qa, const double* ta, const double* qb, const double* tb,
                                            double* qo, double* to) {
    double r[3];
    hq_mul(qa, qb, qo);
    hq_rot(qa, tb, r);
    for (int c = 0; c < 3; ++c) to[c] = ta[c] + r[c];
}

__device__ __forceinline__ void ld_pose(const double* q, const double* t, int64_t v, double* qv, double* tv) {
    for (int c = 0; c < 4; ++c) qv[c] = q[4 * v + c];
    for (int c = 0; c < 3; ++c) tv[c] = t[3 * v + c];
}

__device__ __forceinline__ void st_pose(double* q, double* t, int64_t v, const double* qv, const double* tv) {
    for (int c = 0; c < 4; ++c) q[4 * v + c] = qv[c];
    for (int c = 0; c < 3; ++c) t[3 * v + c] = tv[c];
}

// The poses are composed in segments of kSeg tree levels.  A vertex whose
// depth is a multiple of kSeg (every root) heads a segment; every other
// vertex v composes the steps below its segment head sigma(v) by pointer
// jumping that stops at heads (log2 kSeg rounds), the heads, packed into a
// dense list (one vertex in kSeg on a deep tree, so that their FP64 work
// fills whole warps), compose their head-to-head chains by pointer jumping
// among themselves, and each vertex then takes pose(sigma(v)) o C(v).
// About log2(kSeg) + 1 compositions per vertex instead of log2(depth).
constexpr int kSeg = 16;

// depth by pointer jumping: d = number of steps to the current pointer
__global__ void __launch_bounds__(256) k_depth_init(const int32_t* __restrict__ par, int64_t n, int32_t* p_out,
                                                    int32_t* d_out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = par[v];
        p_out[v] = p;
        d_out[v] = p >= 0 ? 1 : 0;
    }
}

__global__ void __launch_bounds__(256) k_depth_jump(const int32_t* __restrict__ p_in, const int32_t* __restrict__ d_in,
                                                    int64_t n, int32_t* p_out, int32_t* d_out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = p_in[v];
        if (p >= 0) {
            d_out[v] = d_in[v] + d_in[p];
            p_out[v] = p_in[p];
        } else {
            d_out[v] = d_in[v];
            p_out[v] = p;
        }
    }
}

__device__ __forceinline__ bool seg_head(const int32_t* depth, int64_t v) { return depth[v] % kSeg == 0; }

// segment pointers (a head's is -1: it does not jump; every other vertex's
// its parent) and the head flags
__global__ void __launch_bounds__(256) k_seg_init(const int32_t* __restrict__ par, const int32_t* __restrict__ depth,
                                                  int64_t n, int32_t* p_out, int32_t* head_flag) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const bool h = seg_head(depth, v);
        p_out[v] = h ? -1 : par[v];
        head_flag[v] = h ? 1 : 0;
    }
}

// one round inside the segments: (P(v), v] grows to (P(P(v)), v] unless P(v) is a head
__global__ void __launch_bounds__(256) k_seg_jump(const int32_t* __restrict__ p_in, const double* __restrict__ q_in,
                                                  const double* __restrict__ t_in, const int32_t* __restrict__ depth,
                                                  int64_t n, int32_t* p_out, double* q_out, double* t_out) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = p_in[v];
        double qv[4], tv[3];
        ld_pose(q_in, t_in, v, qv, tv);
        if (p >= 0 && !seg_head(depth, p)) {
            double qp[4], tp[3], qn[4], tn[3];
            ld_pose(q_in, t_in, p, qp, tp);
            se3_compose(qp, tp, qv, tv, qn, tn);
            st_pose(q_out, t_out, v, qn, tn);
            p_out[v] = p_in[p];
        } else {
            st_pose(q_out, t_out, v, qv, tv);
            p_out[v] = p;
        }
    }
}

// The dense head list: hv[hpos[v] - 1] = v for every head v (hpos the
// inclusive scan of the head flags).
__global__ void __launch_bounds__(256) k_head_list(const int32_t* __restrict__ depth, const int32_t* __restrict__ hpos,
                                                   int64_t n, int32_t* hv) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x)
        if (seg_head(depth, v)) hv[hpos[v] - 1] = (int32_t)v;
}

// Head k of the dense list (vertex hv[k]): the ordinal of the head above
// (-1 for a root) and the pose step from it, C(par(s)) o step(s) (just
// step(s) when the parent is a head itself; the identity for a root).  One
// thread per head, so the FP64 work fills whole warps.
__global__ void __launch_bounds__(256) k_head_init(const int32_t* __restrict__ par, const int32_t* __restrict__ seg_p,
                                                   const int32_t* __restrict__ depth, const int32_t* __restrict__ hpos,
                                                   const int32_t* __restrict__ hv, const int32_t* __restrict__ count,
                                                   const double* __restrict__ q, const double* __restrict__ t,
                                                   int32_t* hp, double* hq, double* ht) {
    const int64_t H = *count;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < H; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = hv[k];
        const int32_t p = par[v];
        double qv[4], tv[3];
        ld_pose(q, t, v, qv, tv);
        if (p < 0) {
            hp[k] = -1;
        } else if (seg_head(depth, p)) {
            hp[k] = hpos[p] - 1;
        } else {
            double qp[4], tp[3], qn[4], tn[3];
            ld_pose(q, t, p, qp, tp);
            se3_compose(qp, tp, qv, tv, qn, tn);
            for (int c = 0; c < 4; ++c) qv[c] = qn[c];
            for (int c = 0; c < 3; ++c) tv[c] = tn[c];
            hp[k] = hpos[seg_p[p]] - 1;
        }
        st_pose(hq, ht, k, qv, tv);
    }
}

// pointer jumping over the dense head list (its length read on the device)
__global__ void __launch_bounds__(256) k_head_jump(const int32_t* __restrict__ p_in, const double* __restrict__ q_in,
                                                   const double* __restrict__ t_in, const int32_t* __restrict__ count,
                                                   int32_t* p_out, double* q_out, double* t_out) {
    const int64_t H = *count;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < H; k += (int64_t)gridDim.x * blockDim.x) {
        const int32_t p = p_in[k];
        double qv[4], tv[3];
        ld_pose(q_in, t_in, k, qv, tv);
        if (p >= 0) {
            double qp[4], tp[3], qn[4], tn[3];
            ld_pose(q_in, t_in, p, qp, tp);
            se3_compose(qp, tp, qv, tv, qn, tn);
            st_pose(q_out, t_out, k, qn, tn);
            p_out[k] = p_in[p];
        } else {
            st_pose(q_out, t_out, k, qv, tv);
            p_out[k] = p;
        }
    }
}

// pose(v) = pose(sigma(v)) o C(v); a head's pose is its chain's; in place in q, t
__global__ void __launch_bounds__(256) k_seg_apply(const int32_t* __restrict__ seg_p, const int32_t* __restrict__ depth,
                                                   const int32_t* __restrict__ hpos, const double* __restrict__ hq,
                                                   const double* __restrict__ ht, int64_t n, double* q, double* t) {
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        double qn[4], tn[3];
        if (seg_head(depth, v)) {
            ld_pose(hq, ht, hpos[v] - 1, qn, tn);
        } else {
            double qs[4], ts[3], qv[4], tv[3];
            ld_pose(hq, ht, hpos[seg_p[v]] - 1, qs, ts);
            ld_pose(q, t, v, qv, tv);
            se3_compose(qs, ts, qv, tv, qn, tn);
        }
        st_pose(q, t, v, qn, tn);
    }
}

inline int grid_of(int64_t work) {
    const int64_t want = (work + 255) / 256;
    return (int)(want < 152 * 8 ? (want > 0 ? want : 1) : 152 * 8);
}

}  // namespace

cudaError_t launch_validate(const int32_t* src, const int32_t* dst, const double* q, const double* t, const double* ka,
                            const double* om, int64_t n, int64_t m, int32_t* first_bad, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_validate<<<grid_of(m), 256, 0, st>>>(src, dst, q, t, ka, om, n, m, first_bad);
    return cudaGetLastError();
}

cudaError_t launch_check_ends(int32_t* src, int32_t* dst, int64_t n, int64_t m, int32_t* first_bad, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_check_ends<<<grid_of(m), 256, 0, st>>>(src, dst, n, m, first_bad);
    return cudaGetLastError();
}

cudaError_t inclusive_scan_i32(int32_t* a, int64_t len, int32_t* sums, cudaStream_t st) {
    if (len <= 0) return cudaSuccess;
    const int64_t nb = (len + kScanBlock - 1) / kScanBlock;
    k_scan_blocks<<<(unsigned)nb, 256, 0, st>>>(a, len, sums);
    k_scan_sums<<<1, 256, 0, st>>>(sums, nb);
    k_scan_add<<<(unsigned)nb, 256, 0, st>>>(a, len, sums);
    return cudaGetLastError();
}

cudaError_t build_csr_device(const int32_t* key, const int32_t* other, int64_t n, int64_t m, int32_t* ptr,
                             int32_t* slot_edge, int32_t* idx, int32_t* edge_slot, int32_t* fill, int32_t* sums,
                             cudaStream_t st) {
    cudaError_t e;
    if ((e = cudaMemsetAsync(ptr, 0, sizeof(int32_t) * (n + 1), st))) return e;
    if ((e = cudaMemsetAsync(fill, 0, sizeof(int32_t) * n, st))) return e;
    if (m > 0) k_degree<<<grid_of(m), 256, 0, st>>>(key, m, ptr + 1);
    if ((e = inclusive_scan_i32(ptr + 1, n, sums, st))) return e;
    if (m > 0) {
        k_place<<<grid_of(m), 256, 0, st>>>(key, m, ptr, fill, slot_edge);
        k_sort_rows<<<grid_of(n), 256, 0, st>>>(ptr, n, slot_edge);
        k_slot_other<<<grid_of(m), 256, 0, st>>>(slot_edge, m, other, idx, edge_slot);
    }
    return cudaGetLastError();
}

cudaError_t launch_block_inv(const int32_t* out_ptr, const int32_t* out_edge, const int32_t* in_ptr,
                             const int32_t* in_edge, int64_t n, const double* t, const double* ka, const double* om,
                             double a2_0, double a3_0, double a4_0, double* inv2, double* inv3, double* inv4,
                             cudaStream_t st) {
    k_block_inv<<<grid_of(n), 256, 0, st>>>(out_ptr, out_edge, in_ptr, in_edge, n, t, ka, om, a2_0, a3_0, a4_0, inv2,
                                            inv3, inv4);
    return cudaGetLastError();
}

cudaError_t launch_iota(int32_t* a, int64_t n, cudaStream_t st) {
    k_iota<<<grid_of(n), 256, 0, st>>>(a, n);
    return cudaGetLastError();
}

cudaError_t launch_slot_owner(const int32_t* ptr, int64_t n, int32_t* owner, cudaStream_t st) {
    k_slot_owner<<<grid_of(n), 256, 0, st>>>(ptr, n, owner);
    return cudaGetLastError();
}

size_t odometry_scratch_bytes(int64_t n) {
    return (size_t)n * (9 * sizeof(int32_t) + 14 * sizeof(double)) + (size_t)((n + 1023) / 1024 + 8) * sizeof(int32_t) +
           256;
}

cudaError_t launch_odometry(const int32_t* pedge, const int32_t* par, const int32_t* edge_slot, const double* qe64,
                            const double* te64, int64_t n, void* scratch, double* q, double* t, double* q_tmp,
                            double* t_tmp, cudaStream_t st) {
    cudaError_t e;
    double* hq[2] = {static_cast<double*>(scratch), static_cast<double*>(scratch) + 7 * n};
    double* ht[2] = {hq[0] + 4 * n, hq[1] + 4 * n};
    int32_t* ib = reinterpret_cast<int32_t*>(hq[1] + 7 * n);
    int32_t* pp[2] = {ib, ib + n};  // depth pointers, then segment pointers
    int32_t* dd[2] = {ib + 2 * n, ib + 3 * n};
    int32_t* hp[2] = {ib + 4 * n, ib + 5 * n};
    int32_t* hpos = ib + 6 * n;      // head flags, then their inclusive scan
    int32_t* hv = ib + 7 * n;        // the dense head list
    int32_t* sums = ib + 8 * n;
    const int g = grid_of(n);
    // smallest even r with 2^r >= x
    auto even_rounds = [](int64_t x) {
        int r = 0;
        while (((int64_t)1 << r) < x) ++r;
        return r + (r & 1);
    };
    // depth of every vertex (integer pointer jumping, enough rounds for any depth < n)
    k_depth_init<<<g, 256, 0, st>>>(par, n, pp[0], dd[0]);
    const int rd = even_rounds(n);
    for (int r = 0; r < rd; ++r)
        k_depth_jump<<<g, 256, 0, st>>>(pp[r & 1], dd[r & 1], n, pp[(r + 1) & 1], dd[(r + 1) & 1]);
    const int32_t* depth = dd[0];
    // the steps, then the compositions inside the segments: a vertex is at
    // most kSeg - 1 steps below its head (ends in q, t)
    k_odo_steps<<<g, 256, 0, st>>>(pedge, edge_slot, qe64, te64, n, q, t);
    k_seg_init<<<g, 256, 0, st>>>(par, depth, n, pp[0], hpos);
    double* qb[2] = {q, q_tmp};
    double* tb[2] = {t, t_tmp};
    const int rs = even_rounds(kSeg - 1);
    for (int r = 0; r < rs; ++r)
        k_seg_jump<<<g, 256, 0, st>>>(pp[r & 1], qb[r & 1], tb[r & 1], depth, n, pp[(r + 1) & 1], qb[(r + 1) & 1],
                                      tb[(r + 1) & 1]);
    const int32_t* seg_p = pp[0];
    // the heads, packed: their chains by pointer jumping, then every vertex's pose
    if ((e = inclusive_scan_i32(hpos, n, sums, st))) return e;
    const int32_t* count = hpos + n - 1;
    k_head_list<<<g, 256, 0, st>>>(depth, hpos, n, hv);
    k_head_init<<<grid_of(n / kSeg + 1), 256, 0, st>>>(par, seg_p, depth, hpos, hv, count, q, t, hp[0], hq[0], ht[0]);
    const int rh = even_rounds(n / kSeg + 2);
    for (int r = 0; r < rh; ++r)
        k_head_jump<<<grid_of(n / kSeg + 1), 256, 0, st>>>(hp[r & 1], hq[r & 1], ht[r & 1], count, hp[(r + 1) & 1],
                                                            hq[(r + 1) & 1], ht[(r + 1) & 1]);
    k_seg_apply<<<g, 256, 0, st>>>(seg_p, depth, hpos, hq[0], ht[0], n, q, t);
    return cudaGetLastError();
}

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

template <typename R>
cudaError_t launch_pack_in(const int32_t* ie, const int32_t* edge_slot, int64_t slots, const double* qe64,
                           const double* te64, const double* ka64, const double* om64, R* te_out, R* qk_out,
                           cudaStream_t st) {
    if (slots <= 0) return cudaSuccess;
    k_pack_in<R><<<grid_of(slots), 256, 0, st>>>(ie, edge_slot, slots, qe64, te64, ka64, om64, te_out, qk_out);
    return cudaGetLastError();
}

#define PRADMM_SETUP_INST(R)                                                                                     \
    template cudaError_t launch_pack_in<R>(const int32_t*, const int32_t*, int64_t, const double*, const double*, \
                                           const double*, const double*, R*, R*, cudaStream_t);                  \
    template cudaError_t launch_pack_slots<R>(const int32_t*, int64_t, const double*, const double*,             \
                                              const double*, const double*, R*, R*, double*, double*, double*,  \
                                              double*, cudaStream_t);
PRADMM_SETUP_INST(float)
PRADMM_SETUP_INST(double)

}  // namespace pradmm
