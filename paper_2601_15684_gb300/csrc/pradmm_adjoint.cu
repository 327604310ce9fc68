// Reverse mode (adjoint) of the unrolled PRADMM iteration for sm_103a.
//
// Given the adjoint xbar^{k+1} of the state after iteration k (the map
// x^k -> x^{k+1} of Eq. (3a)-(3f), Appendix B closed forms with scalar
// Sigma), the sweeps below produce xbar^k and add iteration k's share of
// dL/dq_e, dL/dt_e, dL/dkappa_e, dL/domega_e.  The forward blocks run
// p -> q -> t -> s -> (lambda, z); their adjoints run in the opposite order:
//
//   (step A, per vertex) duals (3e, 3f), then the s-block (3d): s = sn / A_4
//   k_adj_t   t-block (3c): gathers the s-block adjoint over in-edges
//   k_adj_q   c_e = Im(q_i t~_e p_i^*) and the q-block (3b): out-edges
//   k_adj_p   p-block (3a) with the sphere projection p = u / |u|, whose
//             adjoint is ubar = (I - p p^T) pbar / |u|: out- and in-edges
//   k_adj_grad the measurement gradients of every block (one thread per edge)
//   k_adj_v   the p-block's edge terms of the state adjoints, and step A of
//             the next (earlier) iteration
//
// Inertial variant (Coef::theta != 0): the proximal terms of iteration k are
// gamma (x^k + theta (x^k - x^{k-1})), so each gamma term's adjoint goes
// (1 + theta) to x^k and -theta to x^{k-1}.  The latter is held in A.vp ..
// A.vs until step A of iteration k-2 starts xbar^{k-1} with it; after the
// first iteration it joins xbar^0 (x^{-1} = x^0).  The p-block's recomputed
// u takes p^{k-1} from the step (X.pp).
//
// For a quaternion product V = a x b the adjoint of x is a^* Vbar b^*
// (Lemma MW: M(a)^T = M(a^*), W(b)^T = W(b^*)), and a conjugated operand
// takes the conjugate of its adjoint.  Every sum a vertex needs is a gather
// over its own CSR edges (the transpose of a scatter along out-edges is a
// gather along in-edges), so each output has exactly one writer: no atomics,
// fixed summation order, deterministic results.
//
// A_2 uses |p_i| = |p_j| = 1 (as the forward does); its derivative with
// respect to p points along p and is removed by the sphere projection.  The
// per-edge gradients accumulate in double over all iterations.
#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_device.cuh"
#include "pradmm_internal.h"

namespace pradmm {
namespace {

using namespace dev;

template <typename R>
struct V3 {
    R x, y, z;
};

template <typename R>
__device__ __forceinline__ Q<R> qconj(const Q<R>& a) {
    return {a.w, -a.x, -a.y, -a.z};
}
template <typename R>
__device__ __forceinline__ R qdot(const Q<R>& a, const Q<R>& b) {
    return a.w * b.w + a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R>
__device__ __forceinline__ R vdot(const V3<R>& a, const V3<R>& b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <typename R>
__device__ __forceinline__ V3<R> im(const Q<R>& a) {
    return {a.x, a.y, a.z};
}
template <typename R>
__device__ __forceinline__ V3<R> v3(const R4<R>& a) {
    return {a.a, a.b, a.c};
}
template <typename R>
__device__ __forceinline__ void vaxpy(V3<R>& y, R a, const V3<R>& x) {
    y.x += a * x.x;
    y.y += a * x.y;
    y.z += a * x.z;
}
template <typename R>
__device__ __forceinline__ Q<R> ldq(const R* p, int64_t i) {
    return asq<R>(IO<R>::ld(p, i));
}
template <typename R>
__device__ __forceinline__ void stq(R* p, int64_t i, const Q<R>& v) {
    IO<R>::st(p, i, v.w, v.x, v.y, v.z);
}
template <typename R>
__device__ __forceinline__ void stv(R* p, int64_t i, const V3<R>& v, R pad) {
    IO<R>::st(p, i, v.x, v.y, v.z, pad);
}
// [0, v] a  and  a [0, v]
template <typename R>
__device__ __forceinline__ Q<R> pl(const V3<R>& v, const Q<R>& a) {
    return qmul_pl(v.x, v.y, v.z, a);
}
template <typename R>
__device__ __forceinline__ Q<R> pr(const Q<R>& a, const V3<R>& v) {
    return qmul_pr(a, v.x, v.y, v.z);
}

// Step A: from xbar^{k+1} (pb1 .. zb1) of vertex i, the adjoints of the dual
// updates (3e, 3f) and of the s-block (3d), s^{k+1} = sn / A_4.  Starts the
// accumulators of iteration k: pbar, qbar, tbar of the block outputs
// p^{k+1}, q^{k+1}, t^{k+1}, and the six parts of xbar^k.
// Inertial variant: xbar^k starts from the shares that iteration k+1's anchors
// left in A.vp .. A.vs (none for the last iteration, `first`), and A.vs
// receives iteration k's own s share of xbar^{k-1}.
template <typename R>
__device__ __forceinline__ void step_a(const AdjDev<R>& A, const Coef<R>& c, int64_t i, const Q<R>& pb1,
                                       const Q<R>& qb1, const V3<R>& tb1, const V3<R>& sb1, const Q<R>& lb1,
                                       const V3<R>& zb1, const V3<R>& s_next, R inv4, bool first) {
    const Q<R> PB = {pb1.w - c.tb1 * lb1.w, pb1.x - c.tb1 * lb1.x, pb1.y - c.tb1 * lb1.y, pb1.z - c.tb1 * lb1.z};
    const Q<R> QB = {qb1.w + c.tb1 * lb1.w, qb1.x + c.tb1 * lb1.x, qb1.y + c.tb1 * lb1.y, qb1.z + c.tb1 * lb1.z};
    const V3<R> gs = {(sb1.x + c.tb2 * zb1.x) * inv4, (sb1.y + c.tb2 * zb1.y) * inv4, (sb1.z + c.tb2 * zb1.z) * inv4};
    const R a4b = -vdot(gs, s_next);
    const V3<R> TB = {tb1.x - c.tb2 * zb1.x + c.beta2 * gs.x, tb1.y - c.tb2 * zb1.y + c.beta2 * gs.y,
                      tb1.z - c.tb2 * zb1.z + c.beta2 * gs.z};
    const V3<R> oz = {zb1.x - gs.x, zb1.y - gs.y, zb1.z - gs.z};
    stv(A.gs_w, i, gs, a4b);
    stq(A.pb, i, PB);
    stq(A.qb, i, QB);
    stv(A.tb, i, TB, R(0));
    stq(A.ol, i, lb1);
    stv(A.oz, i, oz, R(0));
    if (c.theta != R(0)) {
        const R g4c = c.g4 * (R(1) + c.theta), g4p = -c.g4 * c.theta;
        R4<R> hp = {R(0), R(0), R(0), R(0)}, hq = hp, ht = hp, hs = hp;
        if (!first) {
            hp = IO<R>::ld(A.vp, i);
            hq = IO<R>::ld(A.vq, i);
            ht = IO<R>::ld(A.vt, i);
            hs = IO<R>::ld(A.vs, i);
        }
        const V3<R> os = {g4c * gs.x + hs.a, g4c * gs.y + hs.b, g4c * gs.z + hs.c};
        stv(A.os, i, os, R(0));
        IO<R>::st(A.vs, i, g4p * gs.x, g4p * gs.y, g4p * gs.z, R(0));
        IO<R>::st(A.op, i, hp.a, hp.b, hp.c, hp.d);
        IO<R>::st(A.oq, i, hq.a, hq.b, hq.c, hq.d);
        IO<R>::st(A.ot, i, ht.a, ht.b, ht.c, R(0));
        return;
    }
    const V3<R> os = {c.g4 * gs.x, c.g4 * gs.y, c.g4 * gs.z};
    stv(A.os, i, os, R(0));
    IO<R>::st(A.op, i, R(0), R(0), R(0), R(0));
    IO<R>::st(A.oq, i, R(0), R(0), R(0), R(0));
    IO<R>::st(A.ot, i, R(0), R(0), R(0), R(0));
}

#define VERTEX_LOOP(n) \
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < (n); i += (int64_t)gridDim.x * blockDim.x)

// Seed for the last iteration: xbar^K = (pbar in op, 0, tbar in ot, 0, 0, 0).
template <typename R>
__global__ void __launch_bounds__(256) k_adj_seed(GraphDev<R> g, AdjDev<R> A, Coef<R> c, const R* s_K, const R* z_K) {
    VERTEX_LOOP(g.n) {
        const Q<R> pb1 = ldq(A.op, i);
        const V3<R> tb1 = v3(IO<R>::ld(A.ot, i));
        const Q<R> zq = {R(0), R(0), R(0), R(0)};
        const V3<R> zv = {R(0), R(0), R(0)};
        step_a<R>(A, c, i, pb1, zq, tb1, zv, zq, zv, v3(IO<R>::ld(s_K, i)), IO<R>::ld(z_K, i).d, true);
    }
}

// t-block adjoint: tbar_i += sum_{e=(l,i)} 2 w_e gs_l, then t^{k+1} = tn / A_3.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_t(GraphDev<R> g, AdjDev<R> A, AdjStep<R> X, Coef<R> c) {
    VERTEX_LOOP(g.n) {
        V3<R> TB = v3(IO<R>::ld(A.tb, i));
        struct E {
            R w;
            R4<R> gsl;
        };
        for_edges<E>(
            g.in_ptr[i], g.in_ptr[i + 1],
            [&](int e, E& x) {
                x.w = IO<R>::ld(g.in_te, e).d;
                x.gsl = IO<R>::ld(A.gs, g.in_idx[e]);
            },
            [&](const E& x) { vaxpy(TB, R(2) * x.w, v3(x.gsl)); });
        const R inv3 = IO<R>::ld(X.t, i).d;
        const V3<R> gt = {TB.x * inv3, TB.y * inv3, TB.z * inv3};
        const R a3b = -vdot(gt, v3(IO<R>::ld(X.tn, i)));
        stv(A.gt, i, gt, a3b);
        V3<R> os = v3(IO<R>::ld(A.os, i)), oz = v3(IO<R>::ld(A.oz, i)), ot = v3(IO<R>::ld(A.ot, i));
        vaxpy(os, c.beta2, gt);
        vaxpy(oz, R(1), gt);
        if (c.theta != R(0)) {
            vaxpy(ot, c.g3 * (R(1) + c.theta), gt);
            const R g3p = -c.g3 * c.theta;
            IO<R>::st(A.vt, i, g3p * gt.x, g3p * gt.y, g3p * gt.z, R(0));
        } else {
            vaxpy(ot, c.g3, gt);
        }
        stv(A.os, i, os, R(0));
        stv(A.oz, i, oz, R(0));
        stv(A.ot, i, ot, R(0));
    }
}

// c_e and q-block adjoint over out-edges e = (i, j):
//   cbar_e = 2 w_e (gt_j - gs_i);  h = [0, cbar_e]
//   qbar_i += h p_i t~_e^*,  pbar_i += h^* q_i t~_e   (q = q^{k+1}, p = p^{k+1})
//   sbar_i += 2 w_e gt_j  (the t-block reads s_i^k through in-edges of j)
// then q^{k+1} = qn / A_2: gq = qbar / A_2, A_2bar = -gq . q^{k+1}.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_q(GraphDev<R> g, AdjDev<R> A, AdjStep<R> X, Coef<R> c) {
    VERTEX_LOOP(g.n) {
        Q<R> QB = ldq(A.qb, i), PB = ldq(A.pb, i);
        const V3<R> gs = v3(IO<R>::ld(A.gs, i));
        const Q<R> P = ldq(X.pn, i), Qn = ldq(X.qn, i);
        V3<R> os = v3(IO<R>::ld(A.os, i));
        struct E {
            R4<R> te, gt;
        };
        for_edges<E>(
            g.out_ptr[i], g.out_ptr[i + 1],
            [&](int e, E& x) {
                x.te = IO<R>::ld(g.out_te, e);
                x.gt = IO<R>::ld(A.gt, g.out_idx[e]);
            },
            [&](const E& x) {
                const V3<R> tv = {x.te.a, x.te.b, x.te.c};
                const V3<R> gt = v3(x.gt);
                const R w2 = R(2) * x.te.d;
                const V3<R> cb = {w2 * (gt.x - gs.x), w2 * (gt.y - gs.y), w2 * (gt.z - gs.z)};
                // h p t~^* = -(h p) t~ and h^* q t~ = -(h q) t~ for pure h, t~
                axpy(QB, R(-1), pr(pl(cb, P), tv));
                axpy(PB, R(-1), pr(pl(cb, Qn), tv));
                vaxpy(os, w2, gt);
            });
        const R inv2 = IO<R>::ld(X.s, i).d;
        const Q<R> gq = {QB.w * inv2, QB.x * inv2, QB.y * inv2, QB.z * inv2};
        const R a2b = -qdot(gq, Qn);
        axpy(PB, c.beta1, gq);
        Q<R> ol = ldq(A.ol, i), oq = ldq(A.oq, i);
        axpy(ol, R(-1), gq);
        if (c.theta != R(0)) {
            axpy(oq, c.g2 * (R(1) + c.theta), gq);
            const R g2p = -c.g2 * c.theta;
            IO<R>::st(A.vq, i, g2p * gq.w, g2p * gq.x, g2p * gq.y, g2p * gq.z);
        } else {
            axpy(oq, c.g2, gq);
        }
        stq(A.gq, i, gq);
        A.a2b[i] = a2b;
        stq(A.pb, i, PB);
        stq(A.ol, i, ol);
        stq(A.oq, i, oq);
        stv(A.os, i, os, R(0));
    }
}

// p-block adjoint.  u_i = beta1 q_i + lam_i + gamma1 p_i
//   + sum_{e=(i,j)} 2 w_e r~^* q_i t~_e + sum_{e=(l,i)} 2 k_e q_l q_e  (x^k, r = t_j - s_i)
// is recomputed; the q-block edge terms that reach p^{k+1} and t^k finish here:
//   pbar_i += sum_{e=(i,j)} 2 w_e r~^* gq_i t~_e + sum_{e=(l,i)} 2 k_e gq_l q_e
//   sbar_i -= sum_{e=(i,j)} 2 w_e Im(gq_i t~_e p_i^*)
//   tbar_i += sum_{e=(l,i)} 2 w_e Im(gq_l t~_e p_l^*)
// then ubar = (I - p p^T) pbar / |u| (|u| = 0: p^{k+1} = p^k, pbar passes on).
template <typename R>
__global__ void __launch_bounds__(256) k_adj_p(GraphDev<R> g, AdjDev<R> A, AdjStep<R> X, Coef<R> c) {
    VERTEX_LOOP(g.n) {
        const Q<R> qi = ldq(X.q, i), li = ldq(X.lam, i), pk = ldq(X.pc, i);
        const V3<R> si = v3(IO<R>::ld(X.s, i));
        const Q<R> P = ldq(X.pn, i), gq = ldq(A.gq, i);
        Q<R> PB = ldq(A.pb, i);
        V3<R> os = v3(IO<R>::ld(A.os, i)), ot = v3(IO<R>::ld(A.ot, i));
        Q<R> pa = pk;  // the proximal anchor, formed as the forward forms it
        if (c.theta != R(0)) {
            const Q<R> po = ldq(X.pp, i);
            pa = {pk.w + c.theta * (pk.w - po.w), pk.x + c.theta * (pk.x - po.x), pk.y + c.theta * (pk.y - po.y),
                  pk.z + c.theta * (pk.z - po.z)};
        }
        Q<R> u = {c.beta1 * qi.w + li.w + c.g1 * pa.w, c.beta1 * qi.x + li.x + c.g1 * pa.x,
                  c.beta1 * qi.y + li.y + c.g1 * pa.y, c.beta1 * qi.z + li.z + c.g1 * pa.z};
        struct EO {
            R4<R> te, tj;
        };
        for_edges<EO>(
            g.out_ptr[i], g.out_ptr[i + 1],
            [&](int e, EO& x) {
                x.te = IO<R>::ld(g.out_te, e);
                x.tj = IO<R>::ld(X.t, g.out_idx[e]);
            },
            [&](const EO& x) {
                const V3<R> tv = {x.te.a, x.te.b, x.te.c};
                const V3<R> r = {x.tj.a - si.x, x.tj.b - si.y, x.tj.c - si.z};
                const R w2 = R(2) * x.te.d;
                // r~^* = -r~ (pure)
                axpy(u, -w2, pr(pl(r, qi), tv));
                axpy(PB, -w2, pr(pl(r, gq), tv));
                R cx, cy, cz;
                im_rot(gq, x.te.a, x.te.b, x.te.c, P, cx, cy, cz);
                os.x -= w2 * cx;
                os.y -= w2 * cy;
                os.z -= w2 * cz;
            });
        struct EI {
            R4<R> qk, te, ql, gql, pl;
        };
        for_edges<EI>(
            g.in_ptr[i], g.in_ptr[i + 1],
            [&](int e, EI& x) {
                const int l = g.in_idx[e];
                x.qk = IO<R>::ld(g.in_qk, e);
                x.te = IO<R>::ld(g.in_te, e);
                x.ql = IO<R>::ld(X.q, l);
                x.gql = IO<R>::ld(A.gq, l);
                x.pl = IO<R>::ld(X.pn, l);
            },
            [&](const EI& x) {
                const Q<R> qk = asq<R>(x.qk), gql = asq<R>(x.gql);
                axpy(u, R(2), qmul(asq<R>(x.ql), qk));
                axpy(PB, R(2), qmul(gql, qk));
                R cx, cy, cz;
                im_rot(gql, x.te.a, x.te.b, x.te.c, asq<R>(x.pl), cx, cy, cz);
                const R w2 = R(2) * x.te.d;
                ot.x += w2 * cx;
                ot.y += w2 * cy;
                ot.z += w2 * cz;
            });
        const R nu = sqrt(qdot(u, u));
        Q<R> op = ldq(A.op, i), oq = ldq(A.oq, i), ol = ldq(A.ol, i);
        Q<R> ub = {R(0), R(0), R(0), R(0)};
        if (nu > R(0)) {
            const R pp = qdot(P, PB);
            const R inv = R(1) / nu;
            ub = {(PB.w - P.w * pp) * inv, (PB.x - P.x * pp) * inv, (PB.y - P.y * pp) * inv,
                  (PB.z - P.z * pp) * inv};
        } else {
            axpy(op, R(1), PB);
        }
        axpy(oq, c.beta1, ub);
        axpy(ol, R(1), ub);
        if (c.theta != R(0)) {
            axpy(op, c.g1 * (R(1) + c.theta), ub);
            const R g1p = -c.g1 * c.theta;
            IO<R>::st(A.vp, i, g1p * ub.w, g1p * ub.x, g1p * ub.y, g1p * ub.z);
        } else {
            axpy(op, c.g1, ub);
        }
        stq(A.ub, i, ub);
        stq(A.op, i, op);
        stq(A.oq, i, oq);
        stq(A.ol, i, ol);
        stv(A.os, i, os, R(0));
        stv(A.ot, i, ot, R(0));
    }
}

// Measurement gradients of iteration k, one thread per out-slot e = (i, j)
// (r = t_j^k - s_i^k, c_e = Im(q_i^{k+1} t~_e p_i^{k+1*}), h = [0, 2 w_e (gt_j - gs_i)]):
//   dL/dw_e += 2 (t_j^{k+1} - c_e).gs_i + 2 A_4bar_i + 2 (s_i + c_e).gt_j + 2 A_3bar_j
//              + 2 gq_i.(r~ p_i t~_e^*) + 2 |t_e|^2 A_2bar_i + 2 ub_i.(r~^* q_i t~_e)
//   dL/dk_e += 2 gq_i.(p_j q_e^*) + 2 |q_e|^2 A_2bar_i + 2 ub_j.(q_i q_e)
//   dL/dt_e += Im(q_i^{k+1*} h p_i) + 2 w_e Im(gq_i^* r~ p_i) + 4 w_e A_2bar_i t_e
//              + 2 w_e Im(q_i^* r~ ub_i)
//   dL/dq_e += 2 k_e gq_i^* p_j + 4 k_e A_2bar_i q_e + 2 k_e q_i^* ub_j
// Each slot has one writer; the sums over iterations are FP64.
template <typename R>
__global__ void __launch_bounds__(256) k_adj_grad(GraphDev<R> g, AdjDev<R> A, AdjStep<R> X, const int32_t* __restrict__ out_src) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < g.m; e += (int64_t)gridDim.x * blockDim.x) {
        const int i = out_src[e], j = g.out_idx[e];
        const R4<R> te = IO<R>::ld(g.out_te, e);
        const V3<R> tv = {te.a, te.b, te.c};
        const R w = te.d, w2 = R(2) * te.d;
        const Q<R> qe = ldq(A.eq, e);
        const R ka = A.ek[e];
        const Q<R> qi = ldq(X.q, i), P = ldq(X.pn, i), Qn = ldq(X.qn, i), gq = ldq(A.gq, i), ub = ldq(A.ub, i);
        const V3<R> si = v3(IO<R>::ld(X.s, i));
        const R4<R> gsr = IO<R>::ld(A.gs, i);
        const V3<R> gs = v3(gsr);
        const R a4b = gsr.d, a2b = A.a2b[i];
        const V3<R> tj = v3(IO<R>::ld(X.t, j));
        const V3<R> tnj = v3(IO<R>::ld(X.tn, j));
        const Q<R> Pj = ldq(X.pn, j), ubj = ldq(A.ub, j);
        const R4<R> gtr = IO<R>::ld(A.gt, j);
        const V3<R> gt = v3(gtr);
        const V3<R> r = {tj.x - si.x, tj.y - si.y, tj.z - si.z};
        R cx, cy, cz;
        im_rot(Qn, te.a, te.b, te.c, P, cx, cy, cz);
        const V3<R> ce = {cx, cy, cz};
        const V3<R> h = {w2 * (gt.x - gs.x), w2 * (gt.y - gs.y), w2 * (gt.z - gs.z)};
        const Q<R> rpt = pr(pl(r, P), tv);   // r~ p t~ = -(r~ p t~^*)
        const Q<R> rqt = pr(pl(r, qi), tv);  // r~ q t~ = -(r~^* q t~)
        const V3<R> tmc = {tnj.x - ce.x, tnj.y - ce.y, tnj.z - ce.z};
        const V3<R> spc = {si.x + ce.x, si.y + ce.y, si.z + ce.z};
        const R tn2 = vdot(tv, tv), qn2 = qdot(qe, qe);
        const R dw = R(2) * vdot(tmc, gs) + R(2) * a4b + R(2) * vdot(spc, gt) + R(2) * gtr.d -
                     R(2) * qdot(gq, rpt) + R(2) * tn2 * a2b - R(2) * qdot(ub, rqt);
        const R dk = R(2) * qdot(gq, qmul_c(Pj, qe)) + R(2) * qn2 * a2b + R(2) * qdot(ubj, qmul(qi, qe));
        const V3<R> t1 = im(qmul(qconj(Qn), pl(h, P)));
        const V3<R> t2 = im(qmul(qconj(gq), pl(r, P)));
        const V3<R> t3 = im(qmul(qconj(qi), pl(r, ub)));
        const R f2 = R(4) * w * a2b;
        const Q<R> m1 = qmul(qconj(gq), Pj), m3 = qmul(qconj(qi), ubj);
        const R k2 = R(2) * ka, f4 = R(4) * ka * a2b;
        double* gte = A.g_te + 4 * e;
        double* gqe = A.g_qe + 4 * e;
        gte[0] += double(t1.x + w2 * (t2.x + t3.x) + f2 * tv.x);
        gte[1] += double(t1.y + w2 * (t2.y + t3.y) + f2 * tv.y);
        gte[2] += double(t1.z + w2 * (t2.z + t3.z) + f2 * tv.z);
        gte[3] += double(dw);
        gqe[0] += double(k2 * (m1.w + m3.w) + f4 * qe.w);
        gqe[1] += double(k2 * (m1.x + m3.x) + f4 * qe.x);
        gqe[2] += double(k2 * (m1.y + m3.y) + f4 * qe.y);
        gqe[3] += double(k2 * (m1.z + m3.z) + f4 * qe.z);
        A.g_ka[e] += double(dk);
    }
}

// p-block edge terms of the state adjoints, then step A of iteration k-1.
// Out-edges e = (i, j), r = t_j^k - s_i^k:
//   qbar_i += 2 k_e ub_j q_e^* + 2 w_e r~ ub_i t~_e^*,  sbar_i += 2 w_e Im(ub_i (q_i t~_e)^*)
// In-edges e = (l, i): tbar_i -= 2 w_e Im(ub_l (q_l t~_e)^*).
template <typename R>
__global__ void __launch_bounds__(256) k_adj_v(GraphDev<R> g, AdjDev<R> A, AdjStep<R> X, Coef<R> c, int more) {
    VERTEX_LOOP(g.n) {
        const Q<R> qi = ldq(X.q, i), ub = ldq(A.ub, i);
        const V3<R> si = v3(IO<R>::ld(X.s, i));
        Q<R> oq = ldq(A.oq, i);
        V3<R> os = v3(IO<R>::ld(A.os, i)), ot = v3(IO<R>::ld(A.ot, i));
        struct EO {
            R ek;
            R4<R> te, tj, ubj, eq;
        };
        for_edges<EO>(
            g.out_ptr[i], g.out_ptr[i + 1],
            [&](int e, EO& x) {
                const int j = g.out_idx[e];
                x.te = IO<R>::ld(g.out_te, e);
                x.eq = IO<R>::ld(A.eq, e);
                x.ek = A.ek[e];
                x.tj = IO<R>::ld(X.t, j);
                x.ubj = IO<R>::ld(A.ub, j);
            },
            [&](const EO& x) {
                const V3<R> tv = {x.te.a, x.te.b, x.te.c};
                const R w2 = R(2) * x.te.d;
                const V3<R> r = {x.tj.a - si.x, x.tj.b - si.y, x.tj.c - si.z};
                axpy(oq, R(2) * x.ek, qmul_c(asq<R>(x.ubj), asq<R>(x.eq)));
                axpy(oq, -w2, pr(pl(r, ub), tv));  // r~ ub t~^* = -r~ ub t~
                vaxpy(os, w2, im(qmul_c(ub, pr(qi, tv))));
            });
        struct EI {
            R4<R> te, ubl, ql;
        };
        for_edges<EI>(
            g.in_ptr[i], g.in_ptr[i + 1],
            [&](int e, EI& x) {
                const int l = g.in_idx[e];
                x.te = IO<R>::ld(g.in_te, e);
                x.ubl = IO<R>::ld(A.ub, l);
                x.ql = IO<R>::ld(X.q, l);
            },
            [&](const EI& x) {
                const V3<R> tv = {x.te.a, x.te.b, x.te.c};
                vaxpy(ot, R(-2) * x.te.d, im(qmul_c(asq<R>(x.ubl), pr(asq<R>(x.ql), tv))));
            });
        if (more) {
            // xbar^k is the xbar^{k+1} of iteration k-1, whose s^{k+1} is s^k here
            step_a<R>(A, c, i, ldq(A.op, i), oq, ot, os, ldq(A.ol, i), v3(IO<R>::ld(A.oz, i)), si,
                      IO<R>::ld(X.z, i).d, false);
        } else {
            if (c.theta != R(0)) {
                // the first iteration's anchor shares belong to x^{-1} = x^0
                Q<R> op = ldq(A.op, i);
                axpy(op, R(1), ldq(A.vp, i));
                axpy(oq, R(1), ldq(A.vq, i));
                vaxpy(ot, R(1), v3(IO<R>::ld(A.vt, i)));
                vaxpy(os, R(1), v3(IO<R>::ld(A.vs, i)));
                stq(A.op, i, op);
            }
            stq(A.oq, i, oq);
            stv(A.os, i, os, R(0));
            stv(A.ot, i, ot, R(0));
        }
    }
}

// Out-slot gradients -> caller's edge order: slot k holds input edge eidx[k].
__global__ void k_adj_scatter(const double* __restrict__ g_qe, const double* __restrict__ g_te,
                              const double* __restrict__ g_ka, const int32_t* __restrict__ eidx, int64_t m,
                              double* qe_bar, double* te_bar, double* ka_bar, double* om_bar) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t e = eidx[k];
        if (qe_bar)
            for (int c = 0; c < 4; ++c) qe_bar[4 * e + c] = g_qe[4 * k + c];
        if (te_bar)
            for (int c = 0; c < 3; ++c) te_bar[3 * e + c] = g_te[4 * k + c];
        if (om_bar) om_bar[e] = g_te[4 * k + 3];
        if (ka_bar) ka_bar[e] = g_ka[k];
    }
}

// Per-slot unscaled q_e and kappa_e in the state precision.
template <typename R>
__global__ void k_adj_edges(const double* __restrict__ qe64, const double* __restrict__ ka64, int64_t m, R* eq, R* ek) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += (int64_t)gridDim.x * blockDim.x) {
        IO<R>::st(eq, k, R(qe64[4 * k]), R(qe64[4 * k + 1]), R(qe64[4 * k + 2]), R(qe64[4 * k + 3]));
        ek[k] = R(ka64[k]);
    }
}

// Tape control block: iteration counter k (picks the p buffers), never halts.
__global__ void k_tape_arm(Ctrl* ctrl, long long iter) {
    ctrl->iter = iter;
    ctrl->target = 0x3fffffffffffffffLL;
    ctrl->halt = 0;
    ctrl->stop = 0;
    ctrl->use_tol = 0;
    ctrl->tol = 0.0;
    ctrl->nonfinite = 0;
    ctrl->ticket = 0u;
}

__global__ void k_tape_rec_arm(TapeRec* rec, const Ctrl* ctrl, void* base, long long K, long long C,
                               long long slot_bytes, long long d_last, long long slot_last) {
    rec->base = static_cast<char*>(base);
    rec->k0 = ctrl->iter;
    rec->K = K;
    rec->C = C;
    rec->slot_bytes = slot_bytes;
    rec->d_last = d_last;
    rec->slot_last = slot_last;
}

__global__ void __launch_bounds__(256) k_tape_copy(const TapeRec* __restrict__ rec, const Ctrl* __restrict__ ctrl,
                                                   const float4* __restrict__ src) {
    const long long d = ctrl->iter - rec->k0;
    if (d <= 0 || d > rec->K) return;
    long long slot;
    if (d % rec->C == 0 || d == rec->K) slot = (d + rec->C - 1) / rec->C;  // a checkpoint
    else if (d > rec->d_last) slot = rec->slot_last + (d - rec->d_last) - 1;  // inside the last segment
    else return;
    float4* dst = reinterpret_cast<float4*>(rec->base + slot * rec->slot_bytes);
    const long long nv = rec->slot_bytes / 16;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// Inertial recording: before the s/z + next-p sweep of iteration k overwrites
// p^k, keep it in the state block's p^{k-1} area, so the checkpoint copied
// after the iteration (x^{k+1}) carries its p^{(k+1)-1}.
template <typename R>
__global__ void __launch_bounds__(256) k_keep_pk(const Ctrl* __restrict__ ctrl, const R* p0, const R* p1, R* dst,
                                                 int64_t n) {
    if (ctrl->halt) return;
    const R* src = (ctrl->iter & 1) ? p1 : p0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const R4<R> v = IO<R>::ld(src, i);
        IO<R>::st(dst, i, v.a, v.b, v.c, v.d);
    }
}

int grid_for(int64_t n, int block) {
    const int64_t gmax = 152 * 16;
    int64_t gb = (n + block - 1) / block;
    return (int)(gb < 1 ? 1 : (gb > gmax ? gmax : gb));
}

}  // namespace

template <typename R>
cudaError_t launch_adj_seed(const GraphDev<R>& g, const AdjDev<R>& A, const Coef<R>& c, const R* s_K, const R* z_K,
                            int block, cudaStream_t st) {
    k_adj_seed<R><<<grid_for(g.n, block), block, 0, st>>>(g, A, c, s_K, z_K);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adj_iteration(const GraphDev<R>& g, const AdjDev<R>& A, const AdjStep<R>& X, const Coef<R>& c,
                                 const int32_t* out_src, int more, int block, cudaStream_t st, cudaStream_t side,
                                 cudaEvent_t fork, cudaEvent_t join) {
    cudaError_t e;
    const int grid = grid_for(g.n, block);
    k_adj_t<R><<<grid, block, 0, st>>>(g, A, X, c);
    k_adj_q<R><<<grid, block, 0, st>>>(g, A, X, c);
    k_adj_p<R><<<grid, block, 0, st>>>(g, A, X, c);
    const bool split = side && g.m > 0 && A.gs_w != A.gs;
    if (split) {
        if ((e = cudaEventRecord(fork, st))) return e;
        if ((e = cudaStreamWaitEvent(side, fork, 0))) return e;
    }
    if (g.m > 0) k_adj_grad<R><<<grid_for(g.m, 256), 256, 0, split ? side : st>>>(g, A, X, out_src);
    if (split && (e = cudaEventRecord(join, side))) return e;
    k_adj_v<R><<<grid, block, 0, st>>>(g, A, X, c, more);
    if (split && (e = cudaStreamWaitEvent(st, join, 0))) return e;
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_keep_pk(const Ctrl* ctrl, const R* p0, const R* p1, R* dst, int64_t n, int grid, cudaStream_t st) {
    k_keep_pk<R><<<grid, 256, 0, st>>>(ctrl, p0, p1, dst, n);
    return cudaGetLastError();
}

template <typename R>
cudaError_t launch_adj_edges(const double* qe64, const double* ka64, int64_t m, R* eq, R* ek, cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_adj_edges<R><<<grid_for(m, 256), 256, 0, st>>>(qe64, ka64, m, eq, ek);
    return cudaGetLastError();
}

cudaError_t launch_adj_scatter(const double* g_qe, const double* g_te, const double* g_ka, const int32_t* eidx,
                               int64_t m, double* qe_bar, double* te_bar, double* ka_bar, double* om_bar,
                               cudaStream_t st) {
    if (m <= 0) return cudaSuccess;
    k_adj_scatter<<<grid_for(m, 256), 256, 0, st>>>(g_qe, g_te, g_ka, eidx, m, qe_bar, te_bar, ka_bar, om_bar);
    return cudaGetLastError();
}

cudaError_t launch_tape_rec_arm(TapeRec* rec, const Ctrl* ctrl, void* base, long long K, long long C,
                                long long slot_bytes, long long d_last, long long slot_last, cudaStream_t st) {
    k_tape_rec_arm<<<1, 1, 0, st>>>(rec, ctrl, base, K, C, slot_bytes, d_last, slot_last);
    return cudaGetLastError();
}

cudaError_t launch_tape_copy(const TapeRec* rec, const Ctrl* ctrl, const void* src, int grid, cudaStream_t st) {
    k_tape_copy<<<grid, 256, 0, st>>>(rec, ctrl, static_cast<const float4*>(src));
    return cudaGetLastError();
}

cudaError_t launch_tape_arm(Ctrl* ctrl, long long iter, cudaStream_t st) {
    k_tape_arm<<<1, 1, 0, st>>>(ctrl, iter);
    return cudaGetLastError();
}

#define PRADMM_ADJ_INST(R)                                                                                           \
    template cudaError_t launch_adj_seed<R>(const GraphDev<R>&, const AdjDev<R>&, const Coef<R>&, const R*, const R*, \
                                            int, cudaStream_t);                                                    \
    template cudaError_t launch_adj_iteration<R>(const GraphDev<R>&, const AdjDev<R>&, const AdjStep<R>&,             \
                                                 const Coef<R>&, const int32_t*, int, int, cudaStream_t,           \
                                                 cudaStream_t, cudaEvent_t, cudaEvent_t);                          \
    template cudaError_t launch_adj_edges<R>(const double*, const double*, int64_t, R*, R*, cudaStream_t);        \
    template cudaError_t launch_keep_pk<R>(const Ctrl*, const R*, const R*, R*, int64_t, int, cudaStream_t);

PRADMM_ADJ_INST(float)
PRADMM_ADJ_INST(double)

}  // namespace pradmm
