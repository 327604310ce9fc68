// Per-vertex updates of the PRADMM sweeps with general weight matrices
// Sigma_1, Sigma_2 (sm_103a), shared by the stand-alone sweep kernels
// (pradmm_sigma.cu) and the batched form (pradmm_batch_sigma.cu).
//
// Edge e = (i, j) weighs the translation residual with omega_e Sigma_1 and
// the rotation residual with kappa_e Sigma_2 (symmetric positive definite
// 4x4, shared by all edges).  The block matrices of Appendix B are then no
// longer scalar:
//   p_sig_vertex  p-block (3a): A_1, b_1 assembled per vertex, then the
//            sphere-constrained quadratic min_{|p|=1} 1/2 p^T A_1 p + b_1^T p
//            of Lemma 1, solved through the eigen-decomposition of A_1
//            (cyclic Jacobi) and the secular equation sum_k g_k^2 /
//            (a_k + lambda)^2 = 1 for lambda > -a_min (the characterisation of
//            the Appendix C lemma), with its hard case; FP32 asks for an FP64
//            re-solve (fb_solve) when the eigen-gap or the component of b_1 on
//            the bottom eigenvector is tiny
//   q_sig_vertex  q-block (3b) + lambda: A_2 (4x4) by Cholesky
//   t_sig_vertex  t-block (3c): A_3 = a Sigma1_hat + (beta2 + gamma3) I, solved
//            in the eigenbasis of Sigma1_hat (the translation block of Sigma_1)
//   s_sig_vertex  s-block (3d) + z
// With
//   G1 = M(q_i t~_e) D,  G2 = W(q_l q_e) D,  G3 = W(t~_e p_i^*),  G4 = M(p_j^*) W(q_e),
//   c~_e = q_i t~_e p_i^* (whole quaternion; its real part couples to the
//   translation through Sigma_1's off-diagonal entries).
// INERT (inertial variant): the proximal anchors are x^k + theta (x^k - x^{k-1})
// instead of x^k.  p^{k-1} is the vertex's value in the p buffer about to
// receive p^{k+1}; q^{k-1}, t^{k-1}, s^{k-1} are in S.qprev, S.tprev, S.sprev,
// which each update overwrites with x^k after its own stores.
// Each vertex sums over its CSR edges in edge order: deterministic.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "pradmm_device.cuh"
#include "pradmm_internal.h"

namespace pradmm {
namespace {

using namespace dev;

template <typename T>
struct Tol;
template <>
struct Tol<float> {
    static __device__ __forceinline__ float jac() { return 1e-7f; }
    static __device__ __forceinline__ float newton() { return 2e-7f; }
};
template <>
struct Tol<double> {
    static __device__ __forceinline__ double jac() { return 1e-15; }
    static __device__ __forceinline__ double newton() { return 1e-15; }
};

// 4x4 matrices of quaternion multiplication (Appendix A.2): M(a) b = a b, W(b) a = a b.
template <typename T>
__device__ __forceinline__ void mat_M(const Q<T>& a, T m[4][4]) {
    m[0][0] = a.w; m[0][1] = -a.x; m[0][2] = -a.y; m[0][3] = -a.z;
    m[1][0] = a.x; m[1][1] = a.w;  m[1][2] = -a.z; m[1][3] = a.y;
    m[2][0] = a.y; m[2][1] = a.z;  m[2][2] = a.w;  m[2][3] = -a.x;
    m[3][0] = a.z; m[3][1] = -a.y; m[3][2] = a.x;  m[3][3] = a.w;
}
template <typename T>
__device__ __forceinline__ void mat_W(const Q<T>& a, T m[4][4]) {
    m[0][0] = a.w; m[0][1] = -a.x; m[0][2] = -a.y; m[0][3] = -a.z;
    m[1][0] = a.x; m[1][1] = a.w;  m[1][2] = a.z;  m[1][3] = -a.y;
    m[2][0] = a.y; m[2][1] = -a.z; m[2][2] = a.w;  m[2][3] = a.x;
    m[3][0] = a.z; m[3][1] = a.y;  m[3][2] = -a.x; m[3][3] = a.w;
}

// A += w G^T S G (upper triangle of A is all that is read later, but the
// full matrix is kept for the Jacobi sweeps)
template <typename T, typename R>
__device__ __forceinline__ void add_sandwich(T A[4][4], const T G[4][4], const R* S, T w) {
    T X[4][4];  // S G
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            T v = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) v += T(S[4 * r + k]) * G[k][c];
            X[r][c] = v;
        }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = r; c < 4; ++c) {
            T v = T(0);
#pragma unroll
            for (int k = 0; k < 4; ++k) v += G[k][r] * X[k][c];
            A[r][c] += w * v;
            if (c != r) A[c][r] += w * v;
        }
}

// y += w G^T (S v)
template <typename T, typename R>
__device__ __forceinline__ void add_gts(T y[4], const T G[4][4], const R* S, const T v[4], T w) {
    T sv[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) sv[r] = T(S[4 * r]) * v[0] + T(S[4 * r + 1]) * v[1] + T(S[4 * r + 2]) * v[2] + T(S[4 * r + 3]) * v[3];
#pragma unroll
    for (int c = 0; c < 4; ++c) y[c] += w * (G[0][c] * sv[0] + G[1][c] * sv[1] + G[2][c] * sv[2] + G[3][c] * sv[3]);
}

// P += w a a^T (upper triangle, row by row: 10 entries)
template <typename T>
__device__ __forceinline__ void add_outer(T P[10], const Q<T>& a, T w) {
    const T v[4] = {a.w, a.x, a.y, a.z};
    int t = 0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const T wm = w * v[m];
#pragma unroll
        for (int n = m; n < 4; ++n) P[t++] += wm * v[n];
    }
}

// A += L(P): the 10 x 10 sandwich map (SigmaDev) applied to the accumulated
// outer products, written to both triangles
template <typename T, typename R>
__device__ __forceinline__ void apply_map(T A[4][4], const R* L, const T P[10]) {
    int o = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = r; c < 4; ++c, ++o) {
            T v = T(0);
#pragma unroll
            for (int q = 0; q < 10; ++q) v += T(L[10 * o + q]) * P[q];
            A[r][c] += v;
            if (c != r) A[c][r] += v;
        }
}

#ifndef PRADMM_SIG_MONO
#define PRADMM_SIG_MONO 1
#endif

// D X D with D = diag(1, -1, -1, -1)
template <typename T>
__device__ __forceinline__ T dsign(int r) {
    return r == 0 ? T(1) : T(-1);
}

// ---- Lemma 1: min_{|x| = 1} 1/2 x^T A x + b^T x ------------------------------

// One Jacobi rotation zeroing a[p][q], in Rutishauser's formulation of the
// cyclic Jacobi eigenvalue method (H. Rutishauser, "The Jacobi method for
// real symmetric matrices", Numer. Math. 9, 1966; the form textbooks give:
// theta = (a_qq - a_pp) / (2 a_pq), t = sgn(theta) / (|theta| + sqrt(theta^2 + 1)),
// c = 1 / sqrt(t^2 + 1), s = t c, and updates through tau = s / (1 + c)).
// A rotation only has to be orthogonal,
// not the exact one, so the FP32 instance (PRADMM_FAST_ROT) takes its
// parameters from the fast reciprocal square root and division intrinsics
// (cs^2 + sn^2 = 1 to a few ulp; the sweeps still drive the off-diagonal part
// to the FP32 tolerance).  The FP64 instance is exact.
#ifndef PRADMM_FAST_ROT
#define PRADMM_FAST_ROT 1
#endif
template <typename T>
__device__ __forceinline__ void jacobi_rotate(T a[4][4], T v[4][4], int p, int q) {
    const T apq = a[p][q];
    if (apq == T(0)) return;
    T t, cs;
    if constexpr (sizeof(T) == sizeof(float) && PRADMM_FAST_ROT) {
        const float theta = __fdividef(a[q][q] - a[p][p], 2.0f * apq);
        const float at = fabsf(theta);
        const float h = theta * theta + 1.0f;
        t = at > 1e15f ? __fdividef(0.5f, theta) : __fdividef(theta >= 0.0f ? 1.0f : -1.0f, at + h * rsqrtf(h));
        cs = rsqrtf(t * t + 1.0f);
    } else {
        const T theta = (a[q][q] - a[p][p]) / (T(2) * apq);
        const T at = fabs(theta);
        t = at > T(1e15) ? T(0.5) / theta : (theta >= T(0) ? T(1) : T(-1)) / (at + sqrt(theta * theta + T(1)));
        cs = T(1) / sqrt(t * t + T(1));
    }
    const T sn = t * cs;
    // the rotation zeroes a[p][q]: the diagonal pair moves by t a[p][q], and
    // only rows / columns p and q change elsewhere (tau = sn / (1 + cs))
    T tau;
    if constexpr (sizeof(T) == sizeof(float) && PRADMM_FAST_ROT) tau = __fdividef(sn, 1.0f + cs);
    else tau = sn / (T(1) + cs);
    a[p][p] -= t * apq;
    a[q][q] += t * apq;
    a[p][q] = a[q][p] = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (r == p || r == q) continue;
        const T arp = a[r][p], arq = a[r][q];
        a[r][p] = a[p][r] = arp - sn * (arq + tau * arp);
        a[r][q] = a[q][r] = arq + sn * (arp - tau * arq);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const T vrp = v[r][p], vrq = v[r][q];
        v[r][p] = vrp - sn * (vrq + tau * vrp);
        v[r][q] = vrq + sn * (vrp - tau * vrq);
    }
}

// Cyclic Jacobi: a -> diag (eigenvalues), v columns the eigenvectors, sorted ascending.
template <typename T>
__device__ void eig4(T a[4][4], T ev[4], T v[4][4]) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) v[r][c] = r == c ? T(1) : T(0);
    for (int sweep = 0; sweep < 12; ++sweep) {
        T off = T(0), dg = T(0);
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            dg += a[r][r] * a[r][r];
#pragma unroll
            for (int c = r + 1; c < 4; ++c) off += a[r][c] * a[r][c];
        }
        if (off <= Tol<T>::jac() * Tol<T>::jac() * dg) break;
        jacobi_rotate(a, v, 0, 1);
        jacobi_rotate(a, v, 0, 2);
        jacobi_rotate(a, v, 0, 3);
        jacobi_rotate(a, v, 1, 2);
        jacobi_rotate(a, v, 1, 3);
        jacobi_rotate(a, v, 2, 3);
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) ev[k] = a[k][k];
    // sort ascending with the columns (selection, 4 elements)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int mn = i;
#pragma unroll
        for (int j = i + 1; j < 4; ++j)
            if (ev[j] < ev[mn]) mn = j;
        if (mn != i) {
            const T e = ev[i];
            ev[i] = ev[mn];
            ev[mn] = e;
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const T x = v[r][i];
                v[r][i] = v[r][mn];
                v[r][mn] = x;
            }
        }
    }
}

// Returns 1 if the solve should be repeated in FP64 (FP32 only: tiny eigen-gap or
// a near-hard case), else writes x (unit) and returns 0.  hard_eps: relative
// size below which b's component on the bottom eigenvector counts as zero --
// the accuracy of the data A and b, not of the arithmetic (FP32 data re-solved
// in FP64 keeps the FP32 threshold, so the hard case and its sign rule apply
// as they would to exact data).
// lam_init: a starting point for the secular Newton iteration (e.g. the root
// found in lower precision), used when it lies inside the bracket; Newton on
// the concave increasing 1/|x(lambda)| - 1 lands left of the root after one
// step from either side and then rises monotonically.  lam_out, v_out
// (optional): the root (NaN in the hard case) and the eigenvectors.
template <typename T>
__device__ int trs4(const T A0[4][4], const T b[4], const T pk[4], T x[4], bool want_fallback, T hard_eps,
                    T lam_init = T(-1), T* lam_out = nullptr, T (*v_out)[4] = nullptr) {
    T a[4][4], v[4][4], ev[4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) a[r][c] = A0[r][c];
    eig4(a, ev, v);
    if (v_out) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) v_out[r][c] = v[r][c];
    }
    if (lam_out) *lam_out = T(NAN);
    T g[4], gn2 = T(0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        g[k] = v[0][k] * b[0] + v[1][k] * b[1] + v[2][k] * b[2] + v[3][k] * b[3];
        gn2 += g[k] * g[k];
    }
    const T scale = fmax(fmax(fabs(ev[0]), fabs(ev[3])), T(1e-30));
    const T gn = sqrt(gn2);
    if (want_fallback && ((ev[1] - ev[0]) < T(1e-3) * scale || fabs(g[0]) < T(1e-3) * gn)) return 1;
    T y[4];
    // hard case: no component of b on the bottom eigenvector, and the rest of
    // the secular sum at lambda = -a_min is below 1
    bool hard = fabs(g[0]) <= hard_eps * fmax(gn, scale);
    if (hard) {
        T rest = T(0);
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const T d = ev[k] - ev[0];
            if (d > T(64) * Tol<T>::jac() * scale) rest += g[k] * g[k] / (d * d);
            else if (fabs(g[k]) > hard_eps * fmax(gn, scale)) rest = T(2);  // degenerate, not hard
        }
        hard = rest < T(1);
        if (hard) {
            y[0] = T(0);
#pragma unroll
            for (int k = 1; k < 4; ++k) {
                const T d = ev[k] - ev[0];
                y[k] = d > T(64) * Tol<T>::jac() * scale ? -g[k] / d : T(0);
            }
            const T alpha = sqrt(fmax(T(0), T(1) - (y[1] * y[1] + y[2] * y[2] + y[3] * y[3])));
            // of the two signs keep the one closer to p^k: sign of v0 . (p^k - x_particular)
            T xp[4], dot = T(0);
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                xp[r] = v[r][1] * y[1] + v[r][2] * y[2] + v[r][3] * y[3];
                dot += v[r][0] * (pk[r] - xp[r]);
            }
            const T sg = dot < T(0) ? T(-1) : T(1);
#pragma unroll
            for (int r = 0; r < 4; ++r) x[r] = xp[r] + sg * alpha * v[r][0];
            return 0;
        }
    }
    // secular equation phi(lambda) = sum g_k^2 / (a_k + lambda)^2 = 1 on
    // [-a_min + |g_0|, -a_min + |g|], Newton on 1/|x(lambda)| from the left
    // (monotone), clamped to the bracket
    // (a lower end strictly above -a_min keeps every 1/(a_k + lambda) finite)
    const T lo = -ev[0] + fmax(fabs(g[0]), T(64) * Tol<T>::jac() * scale), hi = fmax(-ev[0] + gn, lo);
    T lam = (lam_init > lo && lam_init < hi) ? lam_init : lo;
    for (int it = 0; it < 60; ++it) {
        T phi = T(0), w2 = T(0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const T d = T(1) / (ev[k] + lam);
            const T gd = g[k] * d;
            phi += gd * gd;
            w2 += gd * gd * d;
        }
        const T nx = sqrt(phi);
        if (fabs(nx - T(1)) <= Tol<T>::newton() || w2 <= T(0)) break;
        T nl = lam + (nx - T(1)) * phi / w2;
        nl = fmin(fmax(nl, lo), hi);
        if (nl == lam) break;
        lam = nl;
    }
    if (lam_out) *lam_out = lam;
#pragma unroll
    for (int k = 0; k < 4; ++k) y[k] = -g[k] / (ev[k] + lam);
    T nn = T(0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        x[r] = v[r][0] * y[0] + v[r][1] * y[1] + v[r][2] * y[2] + v[r][3] * y[3];
        nn += x[r] * x[r];
    }
    const T inv = T(1) / sqrt(nn);
#pragma unroll
    for (int r = 0; r < 4; ++r) x[r] *= inv;
    return 0;
}

// 4x4 SPD solve by Cholesky (A = L L^T)
template <typename T>
__device__ __forceinline__ void chol_solve4(T A[4][4], T b[4], T x[4]) {
    T L[4][4] = {};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        T d = A[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        const T ljj = sqrt(d);
        L[j][j] = ljj;
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            T v = A[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = v / ljj;
        }
    }
    T y[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        T v = b[i];
#pragma unroll
        for (int k = 0; k < i; ++k) v -= L[i][k] * y[k];
        y[i] = v / L[i][i];
    }
#pragma unroll
    for (int i = 3; i >= 0; --i) {
        T v = y[i];
#pragma unroll
        for (int k = i + 1; k < 4; ++k) v -= L[k][i] * x[k];
        x[i] = v / L[i][i];
    }
}

// E^T S1 w for a 4-vector w (rows 1..3 of S1)
template <typename R>
__device__ __forceinline__ void et_s1(const SigmaDev<R>& sg, const R w[4], R out[3]) {
#pragma unroll
    for (int r = 0; r < 3; ++r)
        out[r] = sg.S1[4 * (r + 1)] * w[0] + sg.S1[4 * (r + 1) + 1] * w[1] + sg.S1[4 * (r + 1) + 2] * w[2] +
                 sg.S1[4 * (r + 1) + 3] * w[3];
}

// (a Sigma1_hat + c I)^{-1} v through Sigma1_hat = U diag(mu) U^T
template <typename R>
__device__ __forceinline__ void solve_hat(const SigmaDev<R>& sg, R a, R cI, const R v[3], R x[3]) {
    R y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k)
        y[k] = (sg.U[k] * v[0] + sg.U[3 + k] * v[1] + sg.U[6 + k] * v[2]) / (a * sg.mu[k] + cI);
#pragma unroll
    for (int r = 0; r < 3; ++r) x[r] = sg.U[3 * r] * y[0] + sg.U[3 * r + 1] * y[1] + sg.U[3 * r + 2] * y[2];
}

// ---- per-vertex updates ------------------------------------------------------

// p-block of vertex i: reads p^k from pc, writes p^{k+1} to pn and returns
// false; or (FP32 only) fills q with the FP32 A_1, b_1, p^k for the FP64
// re-solve of fb_solve and returns true without writing p_i.
template <typename R, bool INERT>
__device__ __forceinline__ bool p_sig_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                                             const SigmaDev<R>& sg, const R* pc, R* pn, int64_t i, FbRec& q) {
        const Q<R> qi = asq<R>(IO<R>::ld(S.q, i)), li = asq<R>(IO<R>::ld(S.lam, i)), pk = asq<R>(IO<R>::ld(pc, i));
        const R4<R> sr = IO<R>::ld(S.s, i);
        Q<R> pa = pk;  // the proximal anchor
        if (INERT) {
            const Q<R> po = asq<R>(IO<R>::ld(pn, i));  // p^{k-1}
            pa = {pk.w + c.theta * (pk.w - po.w), pk.x + c.theta * (pk.x - po.x), pk.y + c.theta * (pk.y - po.y),
                  pk.z + c.theta * (pk.z - po.z)};
        }
        R A[4][4], b[4] = {-c.beta1 * qi.w - li.w - c.g1 * pa.w, -c.beta1 * qi.x - li.x - c.g1 * pa.x,
                           -c.beta1 * qi.y - li.y - c.g1 * pa.y, -c.beta1 * qi.z - li.z - c.g1 * pa.z};
    #pragma unroll
        for (int r = 0; r < 4; ++r)
    #pragma unroll
            for (int cc = 0; cc < 4; ++cc) A[r][cc] = r == cc ? c.beta1 + c.g1 : R(0);
        R G[4][4], bo[4] = {R(0), R(0), R(0), R(0)};
        R P1[10] = {}, P2[10] = {};
        // out-edges: G1 = M(q_i t~_e) D (the D is applied once at the end)
        for (int e = g.out_ptr[i]; e < g.out_ptr[i + 1]; ++e) {
            const R4<R> te = IO<R>::ld(g.out_te, e);
            const R4<R> tj = IO<R>::ld(S.t, g.out_idx[e]);
            const Q<R> a = qmul_pr(qi, te.a, te.b, te.c);
            mat_M(a, G);
            const R r4[4] = {R(0), tj.a - sr.a, tj.b - sr.b, tj.c - sr.c};
            if (PRADMM_SIG_MONO) {
                add_outer(P1, a, R(2) * te.d);
            } else {
                R Ao[4][4] = {};
                add_sandwich(Ao, G, sg.S1, R(2) * te.d);
    #pragma unroll
                for (int r = 0; r < 4; ++r)
    #pragma unroll
                    for (int cc = 0; cc < 4; ++cc) A[r][cc] += dsign<R>(r) * dsign<R>(cc) * Ao[r][cc];
            }
            add_gts(bo, G, sg.S1, r4, R(-2) * te.d);
        }
        // in-edges: G2 = W(q_l q_e) D; the stored record is k_e q_e, so
        // k_e G2^T S2 G2 = (1/k_e) W(h)^T S2 W(h) D-conjugated with h = q_l (k_e q_e),
        // and -2 k_e G2^T S2 1~ = -2 D (sigma2 h^*) with sigma2 the first column of S2
        Q<R> hs = {R(0), R(0), R(0), R(0)};
        for (int e = g.in_ptr[i]; e < g.in_ptr[i + 1]; ++e) {
            const Q<R> qk = asq<R>(IO<R>::ld(g.in_qk, e));
            const R kap = sqrt(qk.w * qk.w + qk.x * qk.x + qk.y * qk.y + qk.z * qk.z);
            const Q<R> h = qmul(asq<R>(IO<R>::ld(S.q, g.in_idx[e])), qk);
            if (PRADMM_SIG_MONO) {
                add_outer(P2, h, R(2) / kap);
            } else {
                mat_W(h, G);
                R Ai[4][4] = {};
                add_sandwich(Ai, G, sg.S2, R(2) / kap);
    #pragma unroll
                for (int r = 0; r < 4; ++r)
    #pragma unroll
                    for (int cc = 0; cc < 4; ++cc) A[r][cc] += dsign<R>(r) * dsign<R>(cc) * Ai[r][cc];
            }
            hs.w += h.w;
            hs.x += h.x;
            hs.y += h.y;
            hs.z += h.z;
        }
        if (PRADMM_SIG_MONO) {
            apply_map(A, sg.LM1D, P1);
            apply_map(A, sg.LW2D, P2);
        }
        // b_1 = own - 2 D (sum G1-part) - 2 D (sigma2 (sum h)^*)
        const Q<R> s2 = {sg.S2[0], sg.S2[4], sg.S2[8], sg.S2[12]};
        const Q<R> sh = qmul_c(s2, hs);
        const R bi[4] = {sh.w, sh.x, sh.y, sh.z};
    #pragma unroll
        for (int r = 0; r < 4; ++r) b[r] += dsign<R>(r) * bo[r] - R(2) * dsign<R>(r) * bi[r];
        const R pkv[4] = {pk.w, pk.x, pk.y, pk.z};
        R x[4];
        if (trs4<R>(A, b, pkv, x, sizeof(R) == sizeof(float), R(64) * Tol<R>::jac())) {
            // for the FP64 re-solve, which writes p_i
            q.i = (int32_t)i;
            int t = 0;
    #pragma unroll
            for (int r = 0; r < 4; ++r)
    #pragma unroll
                for (int cc = r; cc < 4; ++cc) q.a[t++] = float(A[r][cc]);
    #pragma unroll
            for (int r = 0; r < 4; ++r) {
                q.b[r] = float(b[r]);
                q.pk[r] = float(pkv[r]);
            }
            return true;
        }
        IO<R>::st(pn, i, x[0], x[1], x[2], x[3]);
        return false;
}

// The FP64 re-solves queued by k_p_sig in iteration k (FP32 handles only):
// entry kFbLanes w + l goes to lane l of global warp w, and consecutive warps
// go to different CTAs, so the few warps of FP64 work spread over the SMs.
// Warm start: the FP32 eigenvectors of A_1, orthonormalised in FP64, rotate
// the problem (A' = V^T A V, b' = V^T b, p' = V^T p^k; the constraint |x| = 1
// and the hard-case tests are invariant), so the FP64 Jacobi sweeps start
// from a nearly diagonal matrix; x = V x'.  Clears iteration k+1's counter
// (its last use was iteration k-1, finished).
#ifndef PRADMM_FB_LANES
#define PRADMM_FB_LANES 32
#endif
#ifndef PRADMM_FB_WARM
#define PRADMM_FB_WARM 1
#endif
#ifndef PRADMM_FB_LAM
#define PRADMM_FB_LAM 1
#endif
constexpr unsigned kFbLanes = PRADMM_FB_LANES;

// The FP64 re-solve of one p-update from its FP32 data (A_1 upper triangle,
// b_1, p^k): xd is p^{k+1}.
__device__ __forceinline__ void fb_solve(const FbRec& q, double xd[4]) {
    double Ad[4][4], bd[4], pd[4];
    float Af[4][4];
    int t = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = r; cc < 4; ++cc) {
            Ad[r][cc] = Ad[cc][r] = double(q.a[t]);
            Af[r][cc] = Af[cc][r] = q.a[t];
            ++t;
        }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        bd[r] = double(q.b[r]);
        pd[r] = double(q.pk[r]);
    }
    if (PRADMM_FB_WARM) {
        // FP32 eigenvectors and secular root (no fallback test)
        float vf[4][4], bf[4], pf[4], xf[4], lamf;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            bf[r] = q.b[r];
            pf[r] = q.pk[r];
        }
        trs4<float>(Af, bf, pf, xf, false, 64.0f * Tol<float>::jac(), -1.0f, &lamf, vf);
        double V[4][4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) V[r][cc] = double(vf[r][cc]);
        // modified Gram-Schmidt on the columns
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int i2 = 0; i2 < j; ++i2) {
                const double d = V[0][i2] * V[0][j] + V[1][i2] * V[1][j] + V[2][i2] * V[2][j] + V[3][i2] * V[3][j];
#pragma unroll
                for (int r = 0; r < 4; ++r) V[r][j] -= d * V[r][i2];
            }
            const double nv = 1.0 / sqrt(V[0][j] * V[0][j] + V[1][j] * V[1][j] + V[2][j] * V[2][j] + V[3][j] * V[3][j]);
#pragma unroll
            for (int r = 0; r < 4; ++r) V[r][j] *= nv;
        }
        double X[4][4], Ap[4][4], bp[4], pp[4], xp[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc)
                X[r][cc] = Ad[r][0] * V[0][cc] + Ad[r][1] * V[1][cc] + Ad[r][2] * V[2][cc] + Ad[r][3] * V[3][cc];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
#pragma unroll
            for (int cc = r; cc < 4; ++cc)
                Ap[r][cc] = Ap[cc][r] = V[0][r] * X[0][cc] + V[1][r] * X[1][cc] + V[2][r] * X[2][cc] + V[3][r] * X[3][cc];
            bp[r] = V[0][r] * bd[0] + V[1][r] * bd[1] + V[2][r] * bd[2] + V[3][r] * bd[3];
            pp[r] = V[0][r] * pd[0] + V[1][r] * pd[1] + V[2][r] * pd[2] + V[3][r] * pd[3];
        }
        // lamf is NaN in the hard case: the bracket test then fails and Newton starts at lo
        trs4<double>(Ap, bp, pp, xp, false, 1e-5, PRADMM_FB_LAM ? double(lamf) : -1.0);  // FP32 data
#pragma unroll
        for (int r = 0; r < 4; ++r) xd[r] = V[r][0] * xp[0] + V[r][1] * xp[1] + V[r][2] * xp[2] + V[r][3] * xp[3];
    } else {
        trs4<double>(Ad, bd, pd, xd, false, 1e-5);  // FP32 data
    }
}

// q-block (3b) and lambda (3e) of vertex i; adds |dq|^2 and |dlam|^2.
template <typename R, bool INERT>
__device__ __forceinline__ void q_sig_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                                             const SigmaDev<R>& sg, const R* pn, int64_t i, Acc<R>& adq,
                                             Acc<R>& adl) {
        const Q<R> P = asq<R>(IO<R>::ld(pn, i)), qi = asq<R>(IO<R>::ld(S.q, i)), li = asq<R>(IO<R>::ld(S.lam, i));
        const R4<R> sr = IO<R>::ld(S.s, i);
        Q<R> qa = qi;  // the proximal anchor
        if (INERT) {
            const Q<R> qp = asq<R>(IO<R>::ld(S.qprev, i));
            qa = {qi.w + c.theta * (qi.w - qp.w), qi.x + c.theta * (qi.x - qp.x), qi.y + c.theta * (qi.y - qp.y),
                  qi.z + c.theta * (qi.z - qp.z)};
        }
        R A[4][4], b[4] = {c.beta1 * P.w - li.w + c.g2 * qa.w, c.beta1 * P.x - li.x + c.g2 * qa.x,
                           c.beta1 * P.y - li.y + c.g2 * qa.y, c.beta1 * P.z - li.z + c.g2 * qa.z};
    #pragma unroll
        for (int r = 0; r < 4; ++r)
    #pragma unroll
            for (int cc = 0; cc < 4; ++cc) A[r][cc] = r == cc ? c.beta1 + c.g2 : R(0);
        const Q<R> Pc = {P.w, -P.x, -P.y, -P.z};
        const Q<R> s2 = {sg.S2[0], sg.S2[4], sg.S2[8], sg.S2[12]};
        R P3[10] = {};
        for (int e = g.out_ptr[i]; e < g.out_ptr[i + 1]; ++e) {
            const int j = g.out_idx[e];
            const R4<R> te = IO<R>::ld(g.out_te, e);
            const R4<R> tj = IO<R>::ld(S.t, j);
            const Q<R> Pj = asq<R>(IO<R>::ld(pn, j));
            const Q<R> qk = asq<R>(IO<R>::ld(g.out_qk, e));  // k_e q_e
            const R kap = sqrt(qk.w * qk.w + qk.x * qk.x + qk.y * qk.y + qk.z * qk.z);
            // G3 = W(t~_e p_i^*)
            R G[4][4];
            const Q<R> a3 = qmul_pl(te.a, te.b, te.c, Pc);
            mat_W(a3, G);
            if (PRADMM_SIG_MONO) add_outer(P3, a3, R(2) * te.d);
            else add_sandwich(A, G, sg.S1, R(2) * te.d);
            const R r4[4] = {R(0), tj.a - sr.a, tj.b - sr.b, tj.c - sr.c};
            add_gts(b, G, sg.S1, r4, R(2) * te.d);
            // G4' = M(p_j^*) W(k_e q_e) = k_e G4: k_e G4^T S2 G4 = (1/k_e) G4'^T S2 G4',
            // 2 k_e G4^T S2 1~ = 2 G4'^T sigma2 = 2 (p_j sigma2) (k_e q_e)^*
            R Mp[4][4], Wq[4][4];
            mat_M(Q<R>{Pj.w, -Pj.x, -Pj.y, -Pj.z}, Mp);
            mat_W(qk, Wq);
    #pragma unroll
            for (int r = 0; r < 4; ++r)
    #pragma unroll
                for (int cc = 0; cc < 4; ++cc)
                    G[r][cc] = Mp[r][0] * Wq[0][cc] + Mp[r][1] * Wq[1][cc] + Mp[r][2] * Wq[2][cc] + Mp[r][3] * Wq[3][cc];
            add_sandwich(A, G, sg.S2, R(2) / kap);
            const Q<R> v = qmul_c(qmul(Pj, s2), qk);
            b[0] += R(2) * v.w;
            b[1] += R(2) * v.x;
            b[2] += R(2) * v.y;
            b[3] += R(2) * v.z;
        }
        if (PRADMM_SIG_MONO) apply_map(A, sg.LW1, P3);
        R x[4];
        chol_solve4(A, b, x);
        const R lw = li.w - c.tb1 * (P.w - x[0]), lx = li.x - c.tb1 * (P.x - x[1]);
        const R ly = li.y - c.tb1 * (P.y - x[2]), lz = li.z - c.tb1 * (P.z - x[3]);
        IO<R>::st(S.q, i, x[0], x[1], x[2], x[3]);
        IO<R>::st(S.lam, i, lw, lx, ly, lz);
        if (INERT) IO<R>::st(S.qprev, i, qi.w, qi.x, qi.y, qi.z);
        R d0 = x[0] - qi.w, d1 = x[1] - qi.x, d2 = x[2] - qi.y, d3 = x[3] - qi.z;
        adq.add(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3);
        d0 = lw - li.w; d1 = lx - li.x; d2 = ly - li.y; d3 = lz - li.z;
        adl.add(d0 * d0 + d1 * d1 + d2 * d2 + d3 * d3);
}

// t-block (3c) of vertex i; adds |dt|^2.
template <typename R, bool INERT>
__device__ __forceinline__ void t_sig_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                                             const SigmaDev<R>& sg, const R* pn, int64_t i, Acc<R>& adt) {
        const R4<R> tr = IO<R>::ld(S.t, i), sr = IO<R>::ld(S.s, i), zr = IO<R>::ld(S.z, i);
        R4<R> ta = tr;  // the proximal anchor
        if (INERT) {
            const R4<R> tp = IO<R>::ld(S.tprev, i);
            ta = {tr.a + c.theta * (tr.a - tp.a), tr.b + c.theta * (tr.b - tp.b), tr.c + c.theta * (tr.c - tp.c), tr.d};
        }
        R bv[3] = {c.beta2 * sr.a + zr.a + c.g3 * ta.a, c.beta2 * sr.b + zr.b + c.g3 * ta.b,
                   c.beta2 * sr.c + zr.c + c.g3 * ta.c};
        R a = R(0);
        for (int e = g.in_ptr[i]; e < g.in_ptr[i + 1]; ++e) {
            const int l = g.in_idx[e];
            const R4<R> te = IO<R>::ld(g.in_te, e);
            const R4<R> sl = IO<R>::ld(S.s, l);
            const Q<R> cq = qmul_c(qmul_pr(asq<R>(IO<R>::ld(S.q, l)), te.a, te.b, te.c), asq<R>(IO<R>::ld(pn, l)));
            const R w[4] = {cq.w, sl.a + cq.x, sl.b + cq.y, sl.c + cq.z};
            R o[3];
            et_s1(sg, w, o);
            const R w2 = R(2) * te.d;
            bv[0] += w2 * o[0];
            bv[1] += w2 * o[1];
            bv[2] += w2 * o[2];
            a += w2;
        }
        R x[3];
        solve_hat(sg, a, c.beta2 + c.g3, bv, x);
        IO<R>::st(S.t, i, x[0], x[1], x[2], tr.d);
        if (INERT) IO<R>::st(S.tprev, i, tr.a, tr.b, tr.c, tr.d);
        const R d0 = x[0] - tr.a, d1 = x[1] - tr.b, d2 = x[2] - tr.c;
        adt.add(d0 * d0 + d1 * d1 + d2 * d2);
}

// s-block (3d) and z (3f) of vertex i; adds |dz|^2.
template <typename R, bool INERT>
__device__ __forceinline__ void s_sig_vertex(const GraphDev<R>& g, const StateDev<R>& S, const Coef<R>& c,
                                             const SigmaDev<R>& sg, const R* pn, int64_t i, Acc<R>& adz) {
        const R4<R> tr = IO<R>::ld(S.t, i), sr = IO<R>::ld(S.s, i), zr = IO<R>::ld(S.z, i);
        const Q<R> qi = asq<R>(IO<R>::ld(S.q, i)), P = asq<R>(IO<R>::ld(pn, i));
        R4<R> sa = sr;  // the proximal anchor
        if (INERT) {
            const R4<R> sp = IO<R>::ld(S.sprev, i);
            sa = {sr.a + c.theta * (sr.a - sp.a), sr.b + c.theta * (sr.b - sp.b), sr.c + c.theta * (sr.c - sp.c), sr.d};
        }
        R bv[3] = {c.beta2 * tr.a - zr.a + c.g4 * sa.a, c.beta2 * tr.b - zr.b + c.g4 * sa.b,
                   c.beta2 * tr.c - zr.c + c.g4 * sa.c};
        R a = R(0);
        for (int e = g.out_ptr[i]; e < g.out_ptr[i + 1]; ++e) {
            const R4<R> te = IO<R>::ld(g.out_te, e);
            const R4<R> tj = IO<R>::ld(S.t, g.out_idx[e]);
            const Q<R> cq = qmul_c(qmul_pr(qi, te.a, te.b, te.c), P);
            const R w[4] = {-cq.w, tj.a - cq.x, tj.b - cq.y, tj.c - cq.z};
            R o[3];
            et_s1(sg, w, o);
            const R w2 = R(2) * te.d;
            bv[0] += w2 * o[0];
            bv[1] += w2 * o[1];
            bv[2] += w2 * o[2];
            a += w2;
        }
        R x[3];
        solve_hat(sg, a, c.beta2 + c.g4, bv, x);
        const R zx = zr.a - c.tb2 * (tr.a - x[0]), zy = zr.b - c.tb2 * (tr.b - x[1]), zz = zr.c - c.tb2 * (tr.c - x[2]);
        IO<R>::st(S.s, i, x[0], x[1], x[2], sr.d);
        IO<R>::st(S.z, i, zx, zy, zz, zr.d);
        if (INERT) IO<R>::st(S.sprev, i, sr.a, sr.b, sr.c, sr.d);
        const R d0 = zx - zr.a, d1 = zy - zr.b, d2 = zz - zr.c;
        adz.add(d0 * d0 + d1 * d1 + d2 * d2);
}

// Vertex i's share of F (Eq. (1) with Sigma-weighted norms) at (p, t) in
// double: its out-edges' terms.
template <typename R>
__device__ __forceinline__ double objective_sig_vertex(const GraphDev<R>& g, const R* pc, const R* t,
                                                       const double* __restrict__ qe, const double* __restrict__ te,
                                                       const double* __restrict__ ka, const double* __restrict__ om,
                                                       const double* __restrict__ S1, const double* __restrict__ S2,
                                                       int64_t i) {
    double acc = 0.0;
    const Q<double> pi = asq<double>(IO<R>::ld(pc, i));
    const R4<R> ti = IO<R>::ld(t, i);
    for (int e = g.out_ptr[i]; e < g.out_ptr[i + 1]; ++e) {
        const int j = g.out_idx[e];
        const Q<double> pj = asq<double>(IO<R>::ld(pc, j));
        const R4<R> tj = IO<R>::ld(t, j);
        const Q<double> rot = qmul_c(qmul_pr(pi, te[3 * e], te[3 * e + 1], te[3 * e + 2]), pi);
        const double rho[4] = {-rot.w, double(tj.a) - double(ti.a) - rot.x, double(tj.b) - double(ti.b) - rot.y,
                               double(tj.c) - double(ti.c) - rot.z};
        const Q<double> qq = {qe[4 * e], qe[4 * e + 1], qe[4 * e + 2], qe[4 * e + 3]};
        Q<double> h = qmul(qmul(Q<double>{pj.w, -pj.x, -pj.y, -pj.z}, pi), qq);
        const double eta[4] = {h.w - 1.0, h.x, h.y, h.z};
        double f1 = 0.0, f2 = 0.0;
        for (int r = 0; r < 4; ++r)
            for (int cc = 0; cc < 4; ++cc) {
                f1 += rho[r] * S1[4 * r + cc] * rho[cc];
                f2 += eta[r] * S2[4 * r + cc] * eta[cc];
            }
        acc += om[e] * f1 + ka[e] * f2;
    }
    return acc;
}

}  // namespace
}  // namespace pradmm
