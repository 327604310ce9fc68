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
// earlier launches, so it fuses into the s-sweep: the three sweeps share one
// pass over the vertex and its out-edges.  p is double buffered so the p^{k+2}
// computed ahead never overwrites the p^{k+1} the same launch reads.
//
// Every block is Jacobi over vertices (each vertex reads pre-block values of
// its neighbours), so one thread owns one vertex and loops over its CSR
// edges in a fixed order: results are deterministic and the residual
// reductions use a fixed tree (per-CTA partials in double, summed by the last
// CTA in CTA order).
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_internal.h"

namespace pradmm {
namespace {

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
    static __device__ __forceinline__ R4<float> ldro(const float* __restrict__ p, int64_t i) {
        float4 v = __ldg(reinterpret_cast<const float4*>(p) + i);
        return {v.x, v.y, v.z, v.w};
    }
    static __device__ __forceinline__ void st(float* p, int64_t i, float a, float b, float c, float d) {
        reinterpret_cast<float4*>(p)[i] = make_float4(a, b, c, d);
    }
};

template <>
struct IO<double> {
    static __device__ __forceinline__ R4<double> ld(const double* p, int64_t i) {
        const double2* v = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 u = v[0], w = v[1];
        return {u.x, u.y, w.x, w.y};
    }
    static __device__ __forceinline__ R4<double> ldro(const double* __restrict__ p, int64_t i) {
        const double2* v = reinterpret_cast<const double2*>(p) + 2 * i;
        double2 u = __ldg(v), w = __ldg(v + 1);
        return {u.x, u.y, w.x, w.y};
    }
    static __device__ __forceinline__ void st(double* p, int64_t i, double a, double b, double c, double d) {
        double2* v = reinterpret_cast<double2*>(p) + 2 * i;
        v[0] = make_double2(a, b);
        v[1] = make_double2(c, d);
    }
};

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

template <typename A>
__device__ __forceinline__ void axpy(Q<A>& y, A a, const Q<A>& x) {
    y.w += a * x.w;
    y.x += a * x.x;
    y.y += a * x.y;
    y.z += a * x.z;
}

// ---- deterministic CTA reduction of doubles (fixed shuffle tree) ----------

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Returns the CTA total in thread 0 (other threads: unspecified).
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

// ---- p-block, Eq. (3a) / Appendix B.1 ---------------------------------------
// u_i = sum_{e=(i,j)} 2 w_e (t~_j - s~_i)^* q_i t~_e + sum_{e=(l,i)} 2 k_e q_l q_e
//       + beta1 q_i + lam_i + gamma1 p_i ,      p_i^{new} = u_i / |u_i|
// (A_1 is scalar by Lemma MW(c), and the minimiser of its linear term on S^3
// is -b_1/|b_1| = u/|u|.)  Since t~_j - s~_i is pure, its conjugate is its
// negative: the out-edge term is -2 w_e r~ q_i t~_e with r = t_j - s_i.
template <typename R, typename A>
__device__ __forceinline__ Q<A> p_rhs(const GraphDev<R>& g, const R* __restrict__ t, const R* __restrict__ q,
                                      int64_t i, const Q<A>& qi, const Q<A>& li, const Q<A>& pi, A sx, A sy,
                                      A sz, const Coef<R>& c) {
    const A b1 = A(c.beta1), g1 = A(c.g1);
    Q<A> u = {b1 * qi.w + li.w + g1 * pi.w, b1 * qi.x + li.x + g1 * pi.x, b1 * qi.y + li.y + g1 * pi.y,
              b1 * qi.z + li.z + g1 * pi.z};
    const int e0 = g.out_ptr[i], e1 = g.out_ptr[i + 1];
    for (int e = e0; e < e1; ++e) {
        const int j = g.out_dst[e];
        const R4<R> te = IO<R>::ldro(g.out_te, e);
        const R4<R> tj = IO<R>::ld(t, j);
        const A rx = A(tj.a) - sx, ry = A(tj.b) - sy, rz = A(tj.c) - sz;
        const Q<A> v = qmul_pr(qmul_pl(rx, ry, rz, qi), A(te.a), A(te.b), A(te.c));
        axpy(u, A(-2) * A(te.d), v);
    }
    const int f0 = g.in_ptr[i], f1 = g.in_ptr[i + 1];
    for (int e = f0; e < f1; ++e) {
        const int l = g.in_src[e];
        const Q<A> qk = asq<A>(IO<R>::ldro(g.in_qk, e));
        const Q<A> ql = asq<A>(IO<R>::ld(q, l));
        axpy(u, A(2), qmul(ql, qk));
    }
    return u;
}

// Normalises u (computed in R); in FP32, a tiny |u| is recomputed in FP64
// from the same inputs; |u| == 0 keeps p^k (the sphere minimiser is not
// unique then).  Writes p_out[i].
template <typename R>
__device__ __forceinline__ void p_finish(const GraphDev<R>& g, const R* t, const R* q, int64_t i,
                                         const R4<R>& qr, const R4<R>& lr, const R4<R>& pr, R sx, R sy,
                                         R sz, const Coef<R>& c, R* p_out, Ctrl* ctrl) {
    const Q<R> qi = asq<R>(qr), li = asq<R>(lr), pi = asq<R>(pr);
    Q<R> u = p_rhs<R, R>(g, t, q, i, qi, li, pi, sx, sy, sz, c);
    const R nn = u.w * u.w + u.x * u.x + u.y * u.y + u.z * u.z;
    if (sizeof(R) == sizeof(float) && double(sqrt(nn)) < c.fb_thresh) {
        const Q<double> qd = asq<double>(qr), ld = asq<double>(lr), pd = asq<double>(pr);
        const Q<double> ud = p_rhs<R, double>(g, t, q, i, qd, ld, pd, double(sx), double(sy), double(sz), c);
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
        const R inv = R(1) / sqrt(nn);
        IO<R>::st(p_out, i, u.w * inv, u.x * inv, u.y * inv, u.z * inv);
    } else {
        atomicAdd(&ctrl->zero_u, 1ull);
        IO<R>::st(p_out, i, pr.a, pr.b, pr.c, pr.d);
    }
}

// First p-block of a run (when no p^{k+1} was computed ahead).
template <typename R>
__global__ void __launch_bounds__(256) k_p(GraphDev<R> g, StateDev<R> S, Coef<R> c, Ctrl* ctrl) {
    const long long k = ctrl->iter;
    const R* pc = S.p[k & 1];
    R* pn = S.p[(k + 1) & 1];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> qr = IO<R>::ld(S.q, i), lr = IO<R>::ld(S.lam, i), pr = IO<R>::ld(pc, i);
        const R4<R> sr = IO<R>::ld(S.s, i);
        p_finish<R>(g, S.t, S.q, i, qr, lr, pr, sr.a, sr.b, sr.c, c, pn, ctrl);
    }
}

// ---- q-block (3b) / Appendix B.2 + lambda (3e) ----------------------------
// q_i = [sum_{e=(i,j)} 2 (w_e r~ p_i t~_e^* + k_e p_j q_e^*) + beta1 p_i - lam_i + gamma2 q_i] / A_2,
// r = t_j - s_i (t^k, s^k), p = p^{k+1};  lam_i -= tau beta1 (p_i - q_i^{new}).
template <typename R>
__global__ void __launch_bounds__(256) k_q(GraphDev<R> g, StateDev<R> S, Coef<R> c, Ctrl* ctrl, double* part) {
    __shared__ double sh[32];
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    double acc_dq = 0.0, acc_dl = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const Q<R> pi = asq<R>(IO<R>::ld(pn, i));
        const Q<R> qi = asq<R>(IO<R>::ld(S.q, i));
        const Q<R> li = asq<R>(IO<R>::ld(S.lam, i));
        const R4<R> sr = IO<R>::ld(S.s, i);  // (s_i, 1/A_2)
        Q<R> b = {c.beta1 * pi.w - li.w + c.g2 * qi.w, c.beta1 * pi.x - li.x + c.g2 * qi.x,
                  c.beta1 * pi.y - li.y + c.g2 * qi.y, c.beta1 * pi.z - li.z + c.g2 * qi.z};
        const int e0 = g.out_ptr[i], e1 = g.out_ptr[i + 1];
        for (int e = e0; e < e1; ++e) {
            const int j = g.out_dst[e];
            const R4<R> te = IO<R>::ldro(g.out_te, e);
            const Q<R> qk = asq<R>(IO<R>::ldro(g.out_qk, e));
            const R4<R> tj = IO<R>::ld(S.t, j);
            const Q<R> pj = asq<R>(IO<R>::ld(pn, j));
            const R rx = tj.a - sr.a, ry = tj.b - sr.b, rz = tj.c - sr.c;
            // 2 w r~ p t~^* = -2 w r~ p t~ (t~ pure)
            axpy(b, R(-2) * te.d, qmul_pr(qmul_pl(rx, ry, rz, pi), te.a, te.b, te.c));
            // 2 k p_j q_e^* = 2 p_j (k q_e)^*
            axpy(b, R(2), qmul_c(pj, qk));
        }
        const R inv = sr.d;
        const R qw = b.w * inv, qx = b.x * inv, qy = b.y * inv, qz = b.z * inv;
        const R lw = li.w - c.tb1 * (pi.w - qw), lx = li.x - c.tb1 * (pi.x - qx);
        const R ly = li.y - c.tb1 * (pi.y - qy), lz = li.z - c.tb1 * (pi.z - qz);
        IO<R>::st(S.q, i, qw, qx, qy, qz);
        IO<R>::st(S.lam, i, lw, lx, ly, lz);
        double d0 = double(qw) - double(qi.w), d1 = double(qx) - double(qi.x);
        double d2 = double(qy) - double(qi.y), d3 = double(qz) - double(qi.z);
        acc_dq += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
        d0 = double(lw) - double(li.w); d1 = double(lx) - double(li.x);
        d2 = double(ly) - double(li.y); d3 = double(lz) - double(li.z);
        acc_dl += d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3;
    }
    const double sq = block_sum(acc_dq, sh);
    const double sl = block_sum(acc_dl, sh);
    if (threadIdx.x == 0) {
        part[SLOT_DQ * gridDim.x + blockIdx.x] = sq;
        part[SLOT_DLAM * gridDim.x + blockIdx.x] = sl;
    }
}

// ---- t-block (3c) / Appendix B.3 ------------------------------------------
// t_i = [sum_{e=(l,i)} 2 w_e (s_l + c_e) + beta2 s_i + z_i + gamma3 t_i] / A_3,
// c_e = Im(q_l t~_e p_l^*) with q = q^{k+1}, p = p^{k+1} (reading R3), s = s^k.
// c_e is recomputed from the gathered tail state rather than stored.
template <typename R>
__global__ void __launch_bounds__(256) k_t(GraphDev<R> g, StateDev<R> S, Coef<R> c, Ctrl* ctrl, double* part) {
    __shared__ double sh[32];
    if (ctrl->halt) return;
    const long long k = ctrl->iter;
    const R* pn = S.p[(k + 1) & 1];
    double acc_dt = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> tr = IO<R>::ld(S.t, i);  // (t_i, 1/A_3)
        const R4<R> sr = IO<R>::ld(S.s, i);
        const R4<R> zr = IO<R>::ld(S.z, i);
        R ax = c.beta2 * sr.a + zr.a + c.g3 * tr.a;
        R ay = c.beta2 * sr.b + zr.b + c.g3 * tr.b;
        R az = c.beta2 * sr.c + zr.c + c.g3 * tr.c;
        const int f0 = g.in_ptr[i], f1 = g.in_ptr[i + 1];
        for (int e = f0; e < f1; ++e) {
            const int l = g.in_src[e];
            const R4<R> te = IO<R>::ldro(g.in_te, e);
            const R4<R> sl = IO<R>::ld(S.s, l);
            const Q<R> ql = asq<R>(IO<R>::ld(S.q, l));
            const Q<R> pl = asq<R>(IO<R>::ld(pn, l));
            const Q<R> ce = qmul_c(qmul_pr(ql, te.a, te.b, te.c), pl);
            const R w2 = R(2) * te.d;
            ax += w2 * (sl.a + ce.x);
            ay += w2 * (sl.b + ce.y);
            az += w2 * (sl.c + ce.z);
        }
        const R inv = tr.d;
        const R nx = ax * inv, ny = ay * inv, nz = az * inv;
        IO<R>::st(S.t, i, nx, ny, nz, inv);
        const double d0 = double(nx) - double(tr.a), d1 = double(ny) - double(tr.b), d2 = double(nz) - double(tr.c);
        acc_dt += d0 * d0 + d1 * d1 + d2 * d2;
    }
    const double st = block_sum(acc_dt, sh);
    if (threadIdx.x == 0) part[SLOT_DT * gridDim.x + blockIdx.x] = st;
}

// ---- residual e^{k+1} and stop decision (last CTA) --------------------------
__device__ __forceinline__ void finish_iteration(Ctrl* ctrl, const double* part, const Launch& L,
                                                 double b1, double b2, double* sh) {
    __shared__ bool last;
    __threadfence();
    if (threadIdx.x == 0) last = (atomicAdd(&ctrl->ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!last) return;
    __threadfence();
    double tot[4];
#pragma unroll
    for (int sl = 0; sl < 4; ++sl) {
        double v = 0.0;
        for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) v += __ldcg(part + sl * gridDim.x + b);
        tot[sl] = block_sum(v, sh);
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

// ---- s-block (3d) / Appendix B.4 + z (3f), then p-block of iteration k+1 ----
// s_i = [sum_{e=(i,j)} 2 w_e (t_j - c_e) + beta2 t_i - z_i + gamma4 s_i] / A_4 with
// t = t^{k+1}, c_e = Im(q_i t~_e p_i^*) (q^{k+1}, p^{k+1}), s = s^k, z = z^k;
// z_i -= tau beta2 (t_i - s_i^{new}).
template <typename R>
__global__ void __launch_bounds__(256) k_sp(GraphDev<R> g, StateDev<R> S, Coef<R> c, Launch L) {
    __shared__ double sh[32];
    Ctrl* ctrl = L.ctrl;
    if (ctrl->halt) {
        // a halted while-loop body must still end the loop
        if (L.has_cond && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(L.cond, 0u);
        return;
    }
    const long long k = ctrl->iter;
    const R* pc = S.p[(k + 1) & 1];  // p^{k+1}
    R* pn = S.p[k & 1];              // p^{k+2}, computed ahead
    double acc_dz = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> tr = IO<R>::ld(S.t, i);
        const R4<R> sr = IO<R>::ld(S.s, i);  // (s_i, 1/A_2)
        const R4<R> zr = IO<R>::ld(S.z, i);  // (z_i, 1/A_4)
        const R4<R> qr = IO<R>::ld(S.q, i);
        const R4<R> pr = IO<R>::ld(pc, i);
        const Q<R> qi = asq<R>(qr), pi = asq<R>(pr);
        R ax = c.beta2 * tr.a - zr.a + c.g4 * sr.a;
        R ay = c.beta2 * tr.b - zr.b + c.g4 * sr.b;
        R az = c.beta2 * tr.c - zr.c + c.g4 * sr.c;
        const int e0 = g.out_ptr[i], e1 = g.out_ptr[i + 1];
        for (int e = e0; e < e1; ++e) {
            const int j = g.out_dst[e];
            const R4<R> te = IO<R>::ldro(g.out_te, e);
            const R4<R> tj = IO<R>::ld(S.t, j);
            const Q<R> ce = qmul_c(qmul_pr(qi, te.a, te.b, te.c), pi);
            const R w2 = R(2) * te.d;
            ax += w2 * (tj.a - ce.x);
            ay += w2 * (tj.b - ce.y);
            az += w2 * (tj.c - ce.z);
        }
        const R inv = zr.d;
        const R sx = ax * inv, sy = ay * inv, sz = az * inv;
        const R zx = zr.a - c.tb2 * (tr.a - sx), zy = zr.b - c.tb2 * (tr.b - sy), zz = zr.c - c.tb2 * (tr.c - sz);
        IO<R>::st(S.s, i, sx, sy, sz, sr.d);
        IO<R>::st(S.z, i, zx, zy, zz, inv);
        const double d0 = double(zx) - double(zr.a), d1 = double(zy) - double(zr.b), d2 = double(zz) - double(zr.c);
        acc_dz += d0 * d0 + d1 * d1 + d2 * d2;
        // p-block of iteration k+1 (uses q^{k+1}, lam^{k+1}, p^{k+1}, s^{k+1}, t^{k+1})
        const R4<R> lr = IO<R>::ld(S.lam, i);
        p_finish<R>(g, S.t, S.q, i, qr, lr, pr, sx, sy, sz, c, pn, ctrl);
    }
    const double sd = block_sum(acc_dz, sh);
    if (threadIdx.x == 0) L.part[SLOT_DZ * gridDim.x + blockIdx.x] = sd;
    finish_iteration(ctrl, L.part, L, c.b1d, c.b2d, sh);
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
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < g.n; i += (int64_t)gridDim.x * blockDim.x) {
        const Q<double> pi = asq<double>(IO<R>::ld(pc, i));
        const R4<R> ti = IO<R>::ld(S.t, i);
        const int e0 = g.out_ptr[i], e1 = g.out_ptr[i + 1];
        for (int e = e0; e < e1; ++e) {
            const int j = g.out_dst[e];
            const Q<double> pj = asq<double>(IO<R>::ld(pc, j));
            const R4<R> tj = IO<R>::ld(S.t, j);
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
    }
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

// ---- layout conversion ---------------------------------------------------------
template <typename R>
__global__ void k_pack4(const double* __restrict__ src, R* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        IO<R>::st(dst, i, R(src[4 * i]), R(src[4 * i + 1]), R(src[4 * i + 2]), R(src[4 * i + 3]));
}
template <typename R>
__global__ void k_pack3(const double* __restrict__ src, const double* __restrict__ inv, R* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        IO<R>::st(dst, i, R(src[3 * i]), R(src[3 * i + 1]), R(src[3 * i + 2]), R(inv[i]));
}
template <typename R>
__global__ void k_unpack4(const R* src, double* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = IO<R>::ld(src, i);
        dst[4 * i] = v.a;
        dst[4 * i + 1] = v.b;
        dst[4 * i + 2] = v.c;
        dst[4 * i + 3] = v.d;
    }
}
template <typename R>
__global__ void k_unpack3(const R* src, double* dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = IO<R>::ld(src, i);
        dst[3 * i] = v.a;
        dst[3 * i + 1] = v.b;
        dst[3 * i + 2] = v.c;
    }
}

inline int conv_grid(int64_t n) {
    int64_t g = (n + 255) / 256;
    if (g > 4096) g = 4096;
    if (g < 1) g = 1;
    return (int)g;
}

}  // namespace

template <typename R>
cudaError_t launch_p(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    k_p<R><<<L.grid, L.block, 0, L.stream>>>(g, s, c, L.ctrl);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_q(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    k_q<R><<<L.grid, L.block, 0, L.stream>>>(g, s, c, L.ctrl, L.part);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_t(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    k_t<R><<<L.grid, L.block, 0, L.stream>>>(g, s, c, L.ctrl, L.part);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_sp(const GraphDev<R>& g, const StateDev<R>& s, const Coef<R>& c, const Launch& L) {
    k_sp<R><<<L.grid, L.block, 0, L.stream>>>(g, s, c, L);
    return cudaGetLastError();
}

cudaError_t sweep_occupancy(int is_double, int block, int* blocks_per_sm) {
    int a = 0, b = 0, c = 0, d = 0;
    cudaError_t err;
    if (is_double) {
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_q<double>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t<double>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_sp<double>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_p<double>, block, 0))) return err;
    } else {
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_q<float>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t<float>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_sp<float>, block, 0))) return err;
        if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&d, k_p<float>, block, 0))) return err;
    }
    int m = a < b ? a : b;
    m = m < c ? m : c;
    m = m < d ? m : d;
    *blocks_per_sm = m;
    return cudaSuccess;
}

cudaError_t launch_arm(Ctrl* ctrl, long long iters, int use_tol, double tol, cudaStream_t st) {
    k_arm<<<1, 1, 0, st>>>(ctrl, iters, use_tol, tol);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_objective(const GraphDev<R>& g, const StateDev<R>& s, const int32_t*, const int32_t*,
                             const double* qe64, const double* te64, const double* kappa64,
                             const double* omega64, Ctrl* ctrl, double* part, unsigned int* ticket, double* F_dev,
                             int grid, int block, cudaStream_t st) {
    k_objective<R><<<grid, block, 0, st>>>(g, s, qe64, te64, kappa64, omega64, ctrl, part, ticket, F_dev);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pack4(const double* src, R* dst, int64_t n, cudaStream_t st) {
    k_pack4<R><<<conv_grid(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_pack3(const double* src, const double* inv, R* dst, int64_t n, cudaStream_t st) {
    k_pack3<R><<<conv_grid(n), 256, 0, st>>>(src, inv, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_unpack4(const R* src, double* dst, int64_t n, cudaStream_t st) {
    k_unpack4<R><<<conv_grid(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_unpack3(const R* src, double* dst, int64_t n, cudaStream_t st) {
    k_unpack3<R><<<conv_grid(n), 256, 0, st>>>(src, dst, n);
    return cudaGetLastError();
}

#define PRADMM_INST(R)                                                                                        \
    template cudaError_t launch_p<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_q<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_t<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&);  \
    template cudaError_t launch_sp<R>(const GraphDev<R>&, const StateDev<R>&, const Coef<R>&, const Launch&); \
    template cudaError_t launch_objective<R>(const GraphDev<R>&, const StateDev<R>&, const int32_t*,           \
                                             const int32_t*, const double*, const double*, const double*,     \
                                             const double*, Ctrl*, double*, unsigned int*, double*, int, int,  \
                                             cudaStream_t);                                                   \
    template cudaError_t launch_pack4<R>(const double*, R*, int64_t, cudaStream_t);                           \
    template cudaError_t launch_pack3<R>(const double*, const double*, R*, int64_t, cudaStream_t);            \
    template cudaError_t launch_unpack4<R>(const R*, double*, int64_t, cudaStream_t);                         \
    template cudaError_t launch_unpack3<R>(const R*, double*, int64_t, cudaStream_t);

PRADMM_INST(float)
PRADMM_INST(double)

}  // namespace pradmm
