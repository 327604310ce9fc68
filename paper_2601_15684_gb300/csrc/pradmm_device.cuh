// Device-side building blocks of the PRADMM sweeps, shared by the plain
// sweep kernels (pradmm_kernels.cu) and the batched solver (pradmm_batch.cu):
// quaternion algebra, vector I/O, residual accumulators, and the per-vertex
// closed-form updates of Eq. (3a)-(3f) (Appendix B, scalar Sigma).  Both
// callers run exactly these functions, so their arithmetic is identical.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_internal.h"

namespace pradmm {
namespace dev {


template <typename R>
struct Q {
    R w, x, y, z;
};

template <typename R>
struct R4 {
    R a, b, c, d;
};

template <typename R>
struct IO;

template <>
struct IO<float> {
    static __device__ __forceinline__ R4<float> ld(const float* p, int64_t i) {
        float4 v = reinterpret_cast<const float4*>(p)[i];
        return {v.x, v.y, v.z, v.w};
    }
    // edge records (invariant while any sweep runs) on the read-only path with
    // normal caching: the 32 lanes of a warp walk one dense block of records,
    // and a line fetched for one lane serves its neighbours in later loop
    // steps, so L1 must keep it (an evict-first hint cost 16 % per iteration)
    static __device__ __forceinline__ R4<float> ldr(const float* __restrict__ p, int64_t i) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
        return {v.x, v.y, v.z, v.w};
    }
    static __device__ __forceinline__ void st(float* p, int64_t i, float a, float b, float c, float d) {
        reinterpret_cast<float4*>(p)[i] = make_float4(a, b, c, d);
    }
    // read-only (non-coherent) path: only for arrays no thread writes during the launch
    static __device__ __forceinline__ R4<float> ldg(const float* __restrict__ p, int64_t i) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
        return {v.x, v.y, v.z, v.w};
    }
};

template <>
struct IO<double> {
    static __device__ __forceinline__ R4<double> ld(const double* p, int64_t i) {
        const double2* v = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 u = v[0], w = v[1];
        return {u.x, u.y, w.x, w.y};
    }
    static __device__ __forceinline__ R4<double> ldr(const double* __restrict__ p, int64_t i) {
        const double2* v = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 u = __ldg(v), w = __ldg(v + 1);
        return {u.x, u.y, w.x, w.y};
    }
    static __device__ __forceinline__ void st(double* p, int64_t i, double a, double b, double c, double d) {
        double2* v = reinterpret_cast<double2*>(p) + 2 * i;
        v[0] = make_double2(a, b);
        v[1] = make_double2(c, d);
    }
    static __device__ __forceinline__ R4<double> ldg(const double* __restrict__ p, int64_t i) {
        const double2* v = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 u = __ldg(v), w = __ldg(v + 1);
        return {u.x, u.y, w.x, w.y};
    }
};

// Neighbour gather: the read-only path when NC (the launch writes none of the
// gathered arrays), else a coherent load.
template <typename R, bool NC>
__device__ __forceinline__ R4<R> gat(const R* p, int64_t i) {
    if constexpr (NC) return IO<R>::ldg(p, i);
    else return IO<R>::ld(p, i);
}

// Index-checked builds (-DPRADMM_DEBUG_CHECKS=1): a neighbour index outside
// [0, n) or a CSR row bound outside [0, m] read by a sweep is recorded in
// g.dbg (count and value) and replaced by 0, so the access that follows stays
// in bounds and the host reports the count as an error after the run.  No
// trap: the kernel completes.  Release builds compile the check away.
#ifndef PRADMM_DEBUG_CHECKS
#define PRADMM_DEBUG_CHECKS 0
#endif
template <typename G>
__device__ __forceinline__ int32_t chk(const G& g, int32_t v, int64_t bound) {
#if PRADMM_DEBUG_CHECKS
    if (v < 0 || (int64_t)v >= bound) {
        atomicAdd(g.dbg, 1u);
        atomicExch(g.dbg + 1, (unsigned int)v);
        return 0;
    }
#endif
    (void)g;
    (void)bound;
    return v;
}

template <typename A, typename R>
__device__ __forceinline__ Q<A> asq(const R4<R>& v) {
    return {A(v.a), A(v.b), A(v.c), A(v.d)};
}

// ---- quaternion algebra (Appendix A.2): pq = [p0 q0 - p.q, p0 q + q0 p + p x q]

template <typename A>
__device__ __forceinline__ Q<A> qmul(const Q<A>& a, const Q<A>& b) {
    return {a.w * b.w - a.x * b.x - a.y * b.y - a.z * b.z,
            a.w * b.x + a.x * b.w + a.y * b.z - a.z * b.y,
            a.w * b.y - a.x * b.z + a.y * b.w + a.z * b.x,
            a.w * b.z + a.x * b.y - a.y * b.x + a.z * b.w};
}

// a b^*
template <typename A>
__device__ __forceinline__ Q<A> qmul_c(const Q<A>& a, const Q<A>& b) {
    return {a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z,
            -a.w * b.x + a.x * b.w - a.y * b.z + a.z * b.y,
            -a.w * b.y + a.x * b.z + a.y * b.w - a.z * b.x,
            -a.w * b.z - a.x * b.y + a.y * b.x + a.z * b.w};
}

// [0, v] b
template <typename A>
__device__ __forceinline__ Q<A> qmul_pl(A vx, A vy, A vz, const Q<A>& b) {
    return {-vx * b.x - vy * b.y - vz * b.z,
            vx * b.w + vy * b.z - vz * b.y,
            -vx * b.z + vy * b.w + vz * b.x,
            vx * b.y - vy * b.x + vz * b.w};
}

// a [0, v]
template <typename A>
__device__ __forceinline__ Q<A> qmul_pr(const Q<A>& a, A vx, A vy, A vz) {
    return {-a.x * vx - a.y * vy - a.z * vz,
            a.w * vx + a.y * vz - a.z * vy,
            a.w * vy - a.x * vz + a.z * vx,
            a.w * vz + a.x * vy - a.y * vx};
}

// Im(a [0, v] b^*): the rotated-translation term c_e = Im(q t~_e p^*).
template <typename A>
__device__ __forceinline__ void im_rot(const Q<A>& a, A vx, A vy, A vz, const Q<A>& b, A& cx, A& cy, A& cz) {
    const Q<A> h = qmul_pr(a, vx, vy, vz);
    cx = -h.w * b.x + h.x * b.w - h.y * b.z + h.z * b.y;
    cy = -h.w * b.y + h.x * b.z + h.y * b.w - h.z * b.x;
    cz = -h.w * b.z - h.x * b.y + h.y * b.x + h.z * b.w;
}

template <typename A>
__device__ __forceinline__ void axpy(Q<A>& y, A a, const Q<A>& x) {
    y.w += a * x.w;
    y.x += a * x.x;
    y.y += a * x.y;
    y.z += a * x.z;
}

// ---- residual accumulation ----------------------------------------------------
// Per-thread partial of a sum of squares: compensated (Kahan) in FP32, plain
// in FP64.  The cross-thread and cross-CTA sums are FP64 with a fixed tree.
template <typename R>
struct Acc;
template <>
struct Acc<float> {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double get() const { return double(s) - double(c); }
};
template <>
struct Acc<double> {
    double s = 0.0;
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double get() const { return s; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// CTA total in thread 0 (other threads: unspecified); fixed shuffle tree.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < nw ? sh[lane] : 0.0;
        r = warp_sum(r);
    }
    __syncthreads();
    return r;
}

// N CTA totals at once (thread 0 gets them), each with block_sum's tree, so
// each equals a block_sum of its own: sh holds N x 32 doubles.
template <int N>
__device__ __forceinline__ void block_sum_n(double* v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < N; ++k) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) sh[32 * k + wid] = v[k];
    __syncthreads();
    if (wid == 0)
#pragma unroll
        for (int k = 0; k < N; ++k) v[k] = warp_sum(lane < nw ? sh[32 * k + lane] : 0.0);
    __syncthreads();
}

// ---- residual e^{k+1} and stop decision (last CTA of the s/z + p sweep) ---------
// Called by every CTA of the last sweep of an iteration after writing its
// partials; the last CTA to arrive forms e^{k+1}, advances the iteration and
// sets the stop state and the while-node condition.
__device__ __forceinline__ void finish_iteration(Ctrl* ctrl, const Launch& L, double b1, double b2) {
    __shared__ bool last;
    // thread 0 wrote the CTA's partial: it publishes it before taking a ticket
    if (threadIdx.x == 0) {
        __threadfence();
        last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    const int cnt[4] = {L.grid_q, L.grid_sp, L.grid_q, L.grid_t};  // slots DLAM, DZ, DQ, DT
    double tot[4];
    // the four slots in one pass (each slot's terms in the same order and
    // tree as a pass of its own)
    {
        __shared__ double sh4[4 * 32];
        const int most = max(max(cnt[0], cnt[1]), max(cnt[2], cnt[3]));
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int b = threadIdx.x; b < most; b += blockDim.x)
#pragma unroll
            for (int sl = 0; sl < 4; ++sl)
                if (b < cnt[sl]) v[sl] += __ldcg(L.part + sl * L.pstride + b);
        block_sum_n<4>(v, sh4);
#pragma unroll
        for (int sl = 0; sl < 4; ++sl) tot[sl] = v[sl];
    }
    if (threadIdx.x == 0) {
        const double dl = tot[SLOT_DLAM], dz = tot[SLOT_DZ], dq = tot[SLOT_DQ], dt = tot[SLOT_DT];
        const double e = dl / b1 + dz / b2 + b1 * dq + b2 * dt;
        ctrl->parts[0] = dl;
        ctrl->parts[1] = dz;
        ctrl->parts[2] = dq;
        ctrl->parts[3] = dt;
        ctrl->e_last = e;
        const long long it = ctrl->iter + 1;
        ctrl->iter = it;
        if (L.trace) L.trace[(it - 1) % L.trace_cap] = e;
        int halt = 0;
        if (!isfinite(e)) {
            ctrl->nonfinite = 1;
            halt = 1;
        }
        if (ctrl->use_tol && e < ctrl->tol) {
            ctrl->stop = 1;
            halt = 1;
        }
        if (it >= ctrl->target) halt = 1;
        ctrl->halt = halt;
        ctrl->ticket = 0u;
        __threadfence();
        if (L.has_cond) cudaGraphSetConditional(L.cond, halt ? 0u : 1u);
    }
}

// ---- p-block, serial form (FP64 recompute of a tiny |u|) ---------------------
// u_i = sum_{e=(i,j)} 2 w_e (t~_j - s~_i)^* q_i t~_e + sum_{e=(l,i)} 2 k_e q_l q_e
//       + beta1 q_i + lam_i + gamma1 p_i ,      p_i^{new} = u_i / |u_i|
// (Eq. (3a) / Appendix B.1: A_1 is scalar by Lemma MW(c), and the minimiser of
// the linear term on S^3 is -b_1/|b_1| = u/|u|.)  t~_j - s~_i is pure, so its
// conjugate is its negative: the out-edge term is -2 w_e r~ q_i t~_e, r = t_j - s_i.
template <typename R, typename A>
__device__ __noinline__ Q<A> p_rhs_serial(const GraphDev<R>& g, const R* t, const R* q, int64_t i, const Q<A>& qi,
                                          const Q<A>& li, const Q<A>& pi, A sx, A sy, A sz, const Coef<R>& c) {
    const A b1 = A(c.beta1), g1 = A(c.g1);
    Q<A> u = {b1 * qi.w + li.w + g1 * pi.w, b1 * qi.x + li.x + g1 * pi.x, b1 * qi.y + li.y + g1 * pi.y,
              b1 * qi.z + li.z + g1 * pi.z};
    for (int e = chk(g, g.out_ptr[i], g.m + 1), e1 = chk(g, g.out_ptr[i + 1], g.m + 1); e < e1; ++e) {
        const R4<R> te = IO<R>::ld(g.out_te, e);
        const R4<R> tj = IO<R>::ld(t, chk(g, g.out_idx[e], g.n));
        const A rx = A(tj.a) - sx, ry = A(tj.b) - sy, rz = A(tj.c) - sz;
        axpy(u, A(-2) * A(te.d), qmul_pr(qmul_pl(rx, ry, rz, qi), A(te.a), A(te.b), A(te.c)));
    }
    for (int e = chk(g, g.in_ptr[i], g.m + 1), e1 = chk(g, g.in_ptr[i + 1], g.m + 1); e < e1; ++e)
        axpy(u, A(2), qmul(asq<A>(IO<R>::ld(q, chk(g, g.in_idx[e], g.n))), asq<A>(IO<R>::ld(g.in_qk, e))));
    return u;
}

// p-update finish for vertex i: normalise u; in FP32 a tiny |u| is recomputed in
// FP64 from the same inputs; |u| == 0 keeps p^k (sphere minimiser not unique).
// pa: the proximal anchor of the p-block (p^k, or its inertial extrapolation).
template <typename R>
__device__ __forceinline__ void p_normalise(const GraphDev<R>& g, const StateDev<R>& S, int64_t i, const Q<R>& u,
                                            const R4<R>& qr, const R4<R>& lr, const R4<R>& pr, const R4<R>& pa,
                                            R sx, R sy, R sz, const Coef<R>& c, R* p_out, Ctrl* ctrl) {
    const R nn = u.w * u.w + u.x * u.x + u.y * u.y + u.z * u.z;
    const R nrm = sqrt(nn);
    if (sizeof(R) == sizeof(float) && nrm < R(c.fb_thresh)) {
        const Q<double> ud = p_rhs_serial<R, double>(g, S.t, S.q, i, asq<double>(qr), asq<double>(lr), asq<double>(pa),
                                                     double(sx), double(sy), double(sz), c);
        const double nd = sqrt(ud.w * ud.w + ud.x * ud.x + ud.y * ud.y + ud.z * ud.z);
        atomicAdd(&ctrl->fallbacks, 1ull);
        if (nd > 0.0) {
            IO<R>::st(p_out, i, R(ud.w / nd), R(ud.x / nd), R(ud.y / nd), R(ud.z / nd));
        } else {
            atomicAdd(&ctrl->zero_u, 1ull);
            IO<R>::st(p_out, i, pr.a, pr.b, pr.c, pr.d);
        }
        return;
    }
    if (nn > R(0)) {
        const R inv = R(1) / nrm;
        IO<R>::st(p_out, i, u.w * inv, u.x * inv, u.y * inv, u.z * inv);
    } else {
        atomicAdd(&ctrl->zero_u, 1ull);
        IO<R>::st(p_out, i, pr.a, pr.b, pr.c, pr.d);
    }
}

// Visits edges [e0, e1) kUnroll at a time: load(e, buffer) issues the loads
// of one edge, use(buffer) consumes them; the group's loads are all in
// flight before the first use.  Uses run in edge order.
#ifndef PRADMM_UNROLL
#define PRADMM_UNROLL 2
#endif
constexpr int kUnroll = PRADMM_UNROLL;

template <typename T, typename LoadF, typename UseF>
__device__ __forceinline__ void for_edges(int e0, int e1, LoadF load, UseF use) {
    int e = e0;
    for (; e + kUnroll <= e1; e += kUnroll) {
        T b[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) load(e + u, b[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) use(b[u]);
    }
    for (; e < e1; ++e) {
        T b0;
        load(e, b0);
        use(b0);
    }
}

// As for_edges with each edge's loads split in two: load_a(e, buffer) the
// loads that need only e (the neighbour index and the edge records),
// load_b(buffer) the gathers that need the index.  PIPE overlaps a group's
// gathers with the next group's index and record loads (one dependent load
// level per group instead of two) at the cost of registers: it pays where the
// kernel has registers to spare (measured: the plain t sweep).  Uses run in
// edge order either way; rounding can differ where the compiler contracts
// multiply-adds differently.
template <typename T, bool PIPE, typename LoadA, typename LoadB, typename UseF>
__device__ __forceinline__ void for_edges2(int e0, int e1, LoadA load_a, LoadB load_b, UseF use) {
    if (!PIPE) {
        for_edges<T>(
            e0, e1,
            [&](int e, T& x) {
                load_a(e, x);
                load_b(x);
            },
            use);
        return;
    }
    if (e0 >= e1) return;
    T a[kUnroll];
    int cnt = e1 - e0 < kUnroll ? e1 - e0 : kUnroll;
#pragma unroll
    for (int u = 0; u < kUnroll; ++u)
        if (u < cnt) load_a(e0 + u, a[u]);
    int e = e0;
    for (;;) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (u < cnt) load_b(a[u]);
        const int en = e + cnt;
        const int cn = e1 - en < kUnroll ? e1 - en : kUnroll;
        T nx[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (u < cn) load_a(en + u, nx[u]);
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
            if (u < cnt) use(a[u]);
        if (cn <= 0) break;
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) a[u] = nx[u];
        e = en;
        cnt = cn;
    }
}

// ---- q-block (3b) / Appendix B.2 + lambda (3e) --------------------------------
// q_i = [sum_{e=(i,j)} 2 (w_e r~ p_i t~_e^* + k_e p_j q_e^*) + beta1 p_i - lam_i + gamma2 q_i] / A_2,
// r = t_j - s_i (t^k, s^k), p = p^{k+1};  lam_i -= tau beta1 (p_i - q_i^{new}).
template <typename R>
struct QEdge {
    int j;
    R4<R> te, qk, tj, pj;
};

// One vertex of the q-block + lambda update; adds |dq_i|^2, |dlam_i|^2.
// INERT: the proximal anchor is q^k + theta (q^k - q^{k-1}) (inertial variant;
// S.qprev holds q^{k-1} and receives q^k).
template <typename R, bool PIPE = false, bool NC = false, bool INERT = false>
__device__ __forceinline__ void q_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c, const R* pn,
                                         int64_t i, Acc<R>& adq, Acc<R>& adl) {
    const Q<R> pi = asq<R>(IO<R>::ld(pn, i));
    const Q<R> qi = asq<R>(IO<R>::ld(S.q, i));
    const Q<R> li = asq<R>(IO<R>::ld(S.lam, i));
    const R4<R> sr = IO<R>::ld(S.s, i);  // (s_i, 1/A_2)
    Q<R> qa = qi;
    if (INERT) {
        const Q<R> qp = asq<R>(IO<R>::ld(S.qprev, i));
        qa = {qi.w + c.theta * (qi.w - qp.w), qi.x + c.theta * (qi.x - qp.x), qi.y + c.theta * (qi.y - qp.y),
              qi.z + c.theta * (qi.z - qp.z)};
    }
    Q<R> b = {c.beta1 * pi.w - li.w + c.g2 * qa.w, c.beta1 * pi.x - li.x + c.g2 * qa.x,
              c.beta1 * pi.y - li.y + c.g2 * qa.y, c.beta1 * pi.z - li.z + c.g2 * qa.z};
    for_edges2<QEdge<R>, PIPE>(
        chk(g, g.out_ptr[i], g.m + 1), chk(g, g.out_ptr[i + 1], g.m + 1),
        [&](int e, QEdge<R>& x) {
            x.j = chk(g, __ldg(g.out_idx + e), g.n);
            x.te = IO<R>::ldr(g.out_te, e);
            x.qk = IO<R>::ldr(g.out_qk, e);
        },
        [&](QEdge<R>& x) {
            x.tj = gat<R, NC>(S.t, x.j);
            x.pj = gat<R, NC>(pn, x.j);
        },
        [&](const QEdge<R>& x) {
            const R rx = x.tj.a - sr.a, ry = x.tj.b - sr.b, rz = x.tj.c - sr.c;
            // 2 w r~ p t~^* = -2 w r~ p t~ (t~ pure);  2 k p_j q_e^* = 2 p_j (k q_e)^*
            axpy(b, R(-2) * x.te.d, qmul_pr(qmul_pl(rx, ry, rz, pi), x.te.a, x.te.b, x.te.c));
            axpy(b, R(2), qmul_c(asq<R>(x.pj), asq<R>(x.qk)));
        });
    const R inv = sr.d;
    const R qw = b.w * inv, qx = b.x * inv, qy = b.y * inv, qz = b.z * inv;
    const R lw = li.w - c.tb1 * (pi.w - qw), lx = li.x - c.tb1 * (pi.x - qx);
    const R ly = li.y - c.tb1 * (pi.y - qy), lz = li.z - c.tb1 * (pi.z - qz);
    IO<R>::st(S.q, i, qw, qx, qy, qz);
    IO<R>::st(S.lam, i, lw, lx, ly, lz);
    if (INERT) IO<R>::st(S.qprev, i, qi.w, qi.x, qi.y, qi.z);
    R d0 = qw - qi.w, d1 = qx - qi.x, d2 = qy - qi.y, d3 = qz - qi.z;
    adq.add(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3);
    d0 = lw - li.w; d1 = lx - li.x; d2 = ly - li.y; d3 = lz - li.z;
    adl.add(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3);
}

// ---- t-block (3c) / Appendix B.3 ------------------------------------------------
// t_i = [sum_{e=(l,i)} 2 w_e (s_l + c_e) + beta2 s_i + z_i + gamma3 t_i] / A_3,
// c_e = Im(q_l t~_e p_l^*) with q = q^{k+1}, p = p^{k+1} (tail of e), s = s^k.
// c_e is recomputed from the gathered tail state rather than stored.
template <typename R>
struct TEdge {
    int l;
    R4<R> te, sl, ql, pl;
};

// One vertex of the t-block; adds |dt_i|^2.  PIPE: see for_edges2.
// INERT: the proximal anchor is t^k + theta (t^k - t^{k-1}) (S.tprev).
template <typename R, bool PIPE = false, bool NC = false, bool INERT = false>
__device__ __forceinline__ void t_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c, const R* pn,
                                         int64_t i, Acc<R>& adt) {
    const R4<R> tr = IO<R>::ld(S.t, i);  // (t_i, 1/A_3)
    const R4<R> sr = IO<R>::ld(S.s, i);
    const R4<R> zr = IO<R>::ld(S.z, i);
    R tax = tr.a, tay = tr.b, taz = tr.c;
    if (INERT) {
        const R4<R> tp = IO<R>::ld(S.tprev, i);
        tax += c.theta * (tr.a - tp.a);
        tay += c.theta * (tr.b - tp.b);
        taz += c.theta * (tr.c - tp.c);
    }
    R ax = c.beta2 * sr.a + zr.a + c.g3 * tax;
    R ay = c.beta2 * sr.b + zr.b + c.g3 * tay;
    R az = c.beta2 * sr.c + zr.c + c.g3 * taz;
    for_edges2<TEdge<R>, PIPE>(
        chk(g, g.in_ptr[i], g.m + 1), chk(g, g.in_ptr[i + 1], g.m + 1),
        [&](int e, TEdge<R>& x) {
            x.l = chk(g, __ldg(g.in_idx + e), g.n);
            x.te = IO<R>::ldr(g.in_te, e);
        },
        [&](TEdge<R>& x) {
            x.sl = gat<R, NC>(S.s, x.l);
            x.ql = gat<R, NC>(S.q, x.l);
            x.pl = gat<R, NC>(pn, x.l);
        },
        [&](const TEdge<R>& x) {
            R cx, cy, cz;
            im_rot(asq<R>(x.ql), x.te.a, x.te.b, x.te.c, asq<R>(x.pl), cx, cy, cz);
            const R w2 = R(2) * x.te.d;
            ax += w2 * (x.sl.a + cx);
            ay += w2 * (x.sl.b + cy);
            az += w2 * (x.sl.c + cz);
        });
    const R inv = tr.d;
    const R nx = ax * inv, ny = ay * inv, nz = az * inv;
    IO<R>::st(S.t, i, nx, ny, nz, inv);
    if (INERT) IO<R>::st(S.tprev, i, tr.a, tr.b, tr.c, tr.d);
    const R d0 = nx - tr.a, d1 = ny - tr.b, d2 = nz - tr.c;
    adt.add(d0 * d0 + d1 * d1 + d2 * d2);
}

// ---- s-block (3d) / Appendix B.4 + z (3f), then p-block (3a) of the next iteration ----
// WITH_S = true  (k_sp): s_i = [sum_{e=(i,j)} 2 w_e (t_j - c_e) + beta2 t_i - z_i + gamma4 s_i] / A_4
//   with t = t^{k+1}, c_e = Im(q_i t~_e p_i^*) (q^{k+1}, p^{k+1}), s = s^k, z = z^k;
//   z_i -= tau beta2 (t_i - s_i^{new}); then p^{k+2} from (q, lam, p, s, t)^{k+1}.
// WITH_S = false (k_p, the first p-block of a run): p^{k+1} from x^k.
// The p-block's out-edge term needs s_i^{new}, known only after the whole
// out-edge sum of the s-block; by bilinearity
//   sum_e -2 w_e (t~_j - s~^{new}) q t~_e
//     = sum_e -2 w_e (t~_j - s~^{old}) q t~_e  -  (s~^{old} - s~^{new}) q (sum_e 2 w_e t~_e),
// so one pass over the out-edges serves both blocks.  Both parts stay well
// conditioned: t_j - s^{old} is a short edge-length vector and s^{old} - s^{new}
// is the step of s, not a difference of absolute positions.
template <typename R>
struct SEdge {
    int j;
    R4<R> te, tj;
};
template <typename R>
struct PEdge {
    int l;
    R4<R> qk, ql;
};

// One vertex of the s-block + z update (WITH_S; adds |dz_i|^2) followed by
// the p-block of the next iteration, which reads p from pc and writes pn.
// INERT (with the s-block): the proximal anchors are s^k + theta (s^k - s^{k-1})
// (S.sprev) and, for the next p-block, p^{k+1} + theta (p^{k+1} - p^k), p^k being
// the vertex's value in pn before it is overwritten.
// REC with tape != nullptr: vertex i's rows of the state after this
// iteration (t, s, q, both p buffers, lam, z) also go to `tape`, a copy of
// the state block's layout.
template <typename R, bool WITH_S, bool PIPE = false, bool NC = false, bool INERT = false, bool REC = false>
__device__ __forceinline__ void sp_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c, const R* pc,
                                          R* pn, int64_t i, Acc<R>& adz, Ctrl* ctrl, R* tape = nullptr) {
    const R4<R> sr = IO<R>::ld(S.s, i);  // (s_i, 1/A_2)
    const R4<R> qr = IO<R>::ld(S.q, i);
    const R4<R> pr = IO<R>::ld(pc, i);
    const R4<R> lr = IO<R>::ld(S.lam, i);
    const Q<R> qi = asq<R>(qr), pi = asq<R>(pr);
    // out-edge pass: s-block sum (WITH_S), p-block term at s^{old}, sum 2 w t_e
    R ax = R(0), ay = R(0), az = R(0);
    R wx = R(0), wy = R(0), wz = R(0);
    Q<R> u = {R(0), R(0), R(0), R(0)};
    for_edges2<SEdge<R>, PIPE>(
        chk(g, g.out_ptr[i], g.m + 1), chk(g, g.out_ptr[i + 1], g.m + 1),
        [&](int e, SEdge<R>& x) {
            x.j = chk(g, __ldg(g.out_idx + e), g.n);
            x.te = IO<R>::ldr(g.out_te, e);
        },
        [&](SEdge<R>& x) { x.tj = gat<R, NC>(S.t, x.j); },
        [&](const SEdge<R>& x) {
            const R w2 = R(2) * x.te.d;
            if (WITH_S) {
                ax += w2 * x.tj.a;
                ay += w2 * x.tj.b;
                az += w2 * x.tj.c;
                wx += w2 * x.te.a;
                wy += w2 * x.te.b;
                wz += w2 * x.te.c;
            }
            const R rx = x.tj.a - sr.a, ry = x.tj.b - sr.b, rz = x.tj.c - sr.c;
            axpy(u, -w2, qmul_pr(qmul_pl(rx, ry, rz, qi), x.te.a, x.te.b, x.te.c));
        });
    R sx = sr.a, sy = sr.b, sz = sr.c;
    if (WITH_S) {
        // sum_e 2 w_e c_e = Im(q_i (sum_e 2 w_e t~_e) p_i^*): c_e is linear in t_e,
        // so the s-block's c_e terms are formed once, not edge by edge
        R cx, cy, cz;
        im_rot(qi, wx, wy, wz, pi, cx, cy, cz);
        ax -= cx;
        ay -= cy;
        az -= cz;
        const R4<R> tr = IO<R>::ld(S.t, i);
        const R4<R> zr = IO<R>::ld(S.z, i);  // (z_i, 1/A_4)
        const R inv = zr.d;
        R sax = sr.a, say = sr.b, saz = sr.c;
        if (INERT) {
            const R4<R> sp = IO<R>::ld(S.sprev, i);
            sax += c.theta * (sr.a - sp.a);
            say += c.theta * (sr.b - sp.b);
            saz += c.theta * (sr.c - sp.c);
        }
        sx = (ax + c.beta2 * tr.a - zr.a + c.g4 * sax) * inv;
        sy = (ay + c.beta2 * tr.b - zr.b + c.g4 * say) * inv;
        sz = (az + c.beta2 * tr.c - zr.c + c.g4 * saz) * inv;
        const R zx = zr.a - c.tb2 * (tr.a - sx), zy = zr.b - c.tb2 * (tr.b - sy), zz = zr.c - c.tb2 * (tr.c - sz);
        IO<R>::st(S.s, i, sx, sy, sz, sr.d);
        IO<R>::st(S.z, i, zx, zy, zz, inv);
        if (INERT) IO<R>::st(S.sprev, i, sr.a, sr.b, sr.c, sr.d);
        if (REC && tape) {
            IO<R>::st(tape, i, tr.a, tr.b, tr.c, tr.d);  // t: the block's first array
            IO<R>::st(tape + (S.s - S.t), i, sx, sy, sz, sr.d);
            IO<R>::st(tape + (S.z - S.t), i, zx, zy, zz, inv);
        }
        const R d0 = zx - zr.a, d1 = zy - zr.b, d2 = zz - zr.c;
        adz.add(d0 * d0 + d1 * d1 + d2 * d2);
        // move the p-block's out-edge term from s^{old} to s^{new}
        axpy(u, R(-1), qmul_pr(qmul_pl(sr.a - sx, sr.b - sy, sr.c - sz, qi), wx, wy, wz));
    }
    // own terms beta1 q_i + lam_i + gamma1 p_i, then in-edge terms 2 q_l (k_e q_e)
    R4<R> pa = pr;  // the p-block's proximal anchor
    if (INERT && WITH_S) {
        const R4<R> po = IO<R>::ld(pn, i);  // p^k, about to be replaced by p^{k+2}
        pa = {pr.a + c.theta * (pr.a - po.a), pr.b + c.theta * (pr.b - po.b), pr.c + c.theta * (pr.c - po.c),
              pr.d + c.theta * (pr.d - po.d)};
    }
    Q<R> v = {c.beta1 * qr.a + lr.a + c.g1 * pa.a, c.beta1 * qr.b + lr.b + c.g1 * pa.b,
              c.beta1 * qr.c + lr.c + c.g1 * pa.c, c.beta1 * qr.d + lr.d + c.g1 * pa.d};
    axpy(v, R(1), u);
    for_edges2<PEdge<R>, PIPE>(
        chk(g, g.in_ptr[i], g.m + 1), chk(g, g.in_ptr[i + 1], g.m + 1),
        [&](int e, PEdge<R>& x) {
            x.l = chk(g, __ldg(g.in_idx + e), g.n);
            x.qk = IO<R>::ldr(g.in_qk, e);
        },
        [&](PEdge<R>& x) { x.ql = gat<R, NC>(S.q, x.l); },
        [&](const PEdge<R>& x) { axpy(v, R(2), qmul(asq<R>(x.ql), asq<R>(x.qk))); });
    p_normalise<R>(g, S, i, v, qr, lr, pr, pa, sx, sy, sz, c, pn, ctrl);
    if (REC && tape) {
        const R4<R> pv = IO<R>::ld(pn, i);  // this thread's own store
        IO<R>::st(tape + (S.q - S.t), i, qr.a, qr.b, qr.c, qr.d);
        IO<R>::st(tape + (S.lam - S.t), i, lr.a, lr.b, lr.c, lr.d);
        IO<R>::st(tape + (pc - S.t), i, pr.a, pr.b, pr.c, pr.d);
        IO<R>::st(tape + (pn - S.t), i, pv.a, pv.b, pv.c, pv.d);
    }
}

// Out-edge terms of vertex i in F of Eq. (1) at (p, t), in double:
//   sum_{e=(i,j)} w_e |t~_j - t~_i - p_i t~_e p_i^*|^2 + k_e |p_j^* p_i q_e - 1|^2
// with the FP64 measurements of the out-edge order.
template <typename R>
__device__ __forceinline__ double objective_vertex(const GraphDev<R>& g, const R* pc, const R* t,
                                                   const double* __restrict__ qe, const double* __restrict__ te,
                                                   const double* __restrict__ ka, const double* __restrict__ om,
                                                   int64_t i) {
    double acc = 0.0;
    const Q<double> pi = asq<double>(IO<R>::ld(pc, i));
    const R4<R> ti = IO<R>::ld(t, i);
    for (int e = g.out_ptr[i]; e < g.out_ptr[i + 1]; ++e) {
        const int j = g.out_idx[e];
        const Q<double> pj = asq<double>(IO<R>::ld(pc, j));
        const R4<R> tj = IO<R>::ld(t, j);
        // t~_j - t~_i - p_i t~_e p_i^*
        const Q<double> rot = qmul_c(qmul_pr(pi, te[3 * e], te[3 * e + 1], te[3 * e + 2]), pi);
        const double r0 = -rot.w;
        const double r1 = double(tj.a) - double(ti.a) - rot.x;
        const double r2 = double(tj.b) - double(ti.b) - rot.y;
        const double r3 = double(tj.c) - double(ti.c) - rot.z;
        acc += om[e] * (r0 * r0 + r1 * r1 + r2 * r2 + r3 * r3);
        // p_j^* p_i q_e - 1
        const Q<double> qq = {qe[4 * e], qe[4 * e + 1], qe[4 * e + 2], qe[4 * e + 3]};
        const Q<double> pjc = {pj.w, -pj.x, -pj.y, -pj.z};
        Q<double> h = qmul(qmul(pjc, pi), qq);
        h.w -= 1.0;
        acc += ka[e] * (h.w * h.w + h.x * h.x + h.y * h.y + h.z * h.z);
    }
    return acc;
}

}  // namespace dev
}  // namespace pradmm
