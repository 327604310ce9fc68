/*
 * PRADMM oracle -- plain, slow, FP64 CPU implementation of one PRADMM
 * iteration (Chen, Cui, Han, Qi, "Parallelizable Riemannian ADMM for
 * Non-convex Pose Graph Optimization", arXiv 2601.15684).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA library is
 * compared against.  Only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg may load it.  It shares no code, header, table or helper
 * with the CUDA library, and the library never calls it.
 *
 * Everything is double precision, single threaded, with loops written in the
 * order the paper states the steps:
 *   - quaternion algebra .................. Appendix A.2
 *   - model (1) objective F ............... Section 2, Eq. (1)
 *   - split model (2), f and g ............ Section 3.1, Eq. (2)
 *   - augmented Lagrangian L_beta ......... Section 3.2
 *   - one iteration (3a)-(3f) ............. Section 3.2 Eq. (3), Algorithm 1,
 *                                           closed forms of Appendix B
 *   - residual e^{k+1} and stopping ....... Appendix E.1
 *   - reverse mode of the unrolled ........ derivative of Eq. (3a)-(3f) with
 *     iteration (adjoint)                   respect to the measurements and x^0
 *
 * Readings of passages that are garbled or silent (the same readings the CUDA
 * path follows):
 *   R1  the in-edge matrix of the p-block is W(q_li) W(q_l) D (the printed
 *       form drops D); in product form its transpose times 1~ is q_l q_li.
 *   R2  x = A^{-1} b with b as printed for the q, t, s blocks; p = -b1/|b1|.
 *   R3  c_e = Im(q_tail t~_e p_tail^*) for e = (tail, head).
 *   R4  proximal anchors x^{k+1/2} are read as x^k (plain PRADMM).
 *   R27 the inertial variant (named once, rule not given) extrapolates the
 *       anchors: x^{k+1/2} = x^k + theta (x^k - x^{k-1}) for p, q, t, s.
 *   R5  z lives in R^{3n}.
 *   R6  e^{k+1} uses beta1 for the lambda / q terms and beta2 for z / t.
 *   R8  lambda^0 = z^0 = 0, p^0 = q^0, s^0 = t^0 (set by the caller).
 *   R9  Sigma_1 = omega_e I_4 and Sigma_2 = kappa_e I_4 per edge.
 *   R11 if |u_i| == 0 the p-block keeps p_i^k.
 *   R13 Jacobi inside a block: every vertex reads pre-block values.
 *   R21 the adjoint differentiates the unrolled map x^0 -> x^K with x^0 held
 *       fixed; q_e is a point of R^4 (no renormalisation inside the map);
 *       where |u_i| == 0 (R11) the adjoint of p_i^{k+1} passes to p_i^k.
 *
 * Quaternions are scalar first, [q0, q1, q2, q3] (Appendix A.2).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    double beta1, beta2; /* penalties beta_1, beta_2 (Section 3.2) */
    double tau;          /* relaxed dual step tau in (0,2), Eq. (3e,f) */
    double gamma[4];     /* H_{s,i} = gamma_s I (Section 3.2) */
} orc_params;

/* ---- quaternion algebra, Appendix A.2 -------------------------------- */

/* p q = [p0 q0 - p.q, p0 q + q0 p + p x q] */
static void qmul(const double* a, const double* b, double* o) {
    double r0 = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    double r1 = a[0] * b[1] + b[0] * a[1] + (a[2] * b[3] - a[3] * b[2]);
    double r2 = a[0] * b[2] + b[0] * a[2] + (a[3] * b[1] - a[1] * b[3]);
    double r3 = a[0] * b[3] + b[0] * a[3] + (a[1] * b[2] - a[2] * b[1]);
    o[0] = r0; o[1] = r1; o[2] = r2; o[3] = r3;
}

/* q^* = [q0, -q] */
static void qconj(const double* a, double* o) {
    o[0] = a[0]; o[1] = -a[1]; o[2] = -a[2]; o[3] = -a[3];
}

/* pure quaternion t~ = [0, t] (Section 2) */
static void qpure(const double* t3, double* o) {
    o[0] = 0.0; o[1] = t3[0]; o[2] = t3[1]; o[3] = t3[2];
}

static double dot4(const double* a, const double* b) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2] + a[3] * b[3];
}

/* [0, R(q) t] = q [0, t] q^*  (Appendix A.2) */
static void qrotate(const double* q, const double* t3, double* out3) {
    double tp[4], a[4], qc[4], r[4];
    qpure(t3, tp);
    qmul(q, tp, a);
    qconj(q, qc);
    qmul(a, qc, r);
    out3[0] = r[1]; out3[1] = r[2]; out3[2] = r[3];
}

/* Exported for the oracle's own unit tests (Lemma MW, R(q) identities). */
void orc_qmul(const double* a, const double* b, double* o) { qmul(a, b, o); }
void orc_qrotate(const double* q, const double* t3, double* o) { qrotate(q, t3, o); }

/* ---- odometry initialisation --------------------------------------------
 * The paper starts every method from a chordal initialisation that it does
 * not define (Section 5).  The initial point used here is odometry
 * composition along a spanning forest: edges are taken in input order and an
 * edge joins the forest when it links two components (Kruskal by edge
 * index).  The lowest vertex of each component gets the identity pose, and
 * every other vertex is composed from its forest parent with the generative
 * relation of Section 2, q_j = q_i q_ij and t_j = t_i + R_i t_ij.
 */
static int64_t uf_find(int64_t* par, int64_t x) {
    while (par[x] != x) { par[x] = par[par[x]]; x = par[x]; }
    return x;
}

/* The walk of orc_init_odometry; with q == NULL no pose is composed.  par,
 * pedge (optional): each vertex's forest parent (-1 for a root) and the tree
 * edge e to it, coded e when the vertex is the edge's head and -(e + 2) when
 * it is its tail (-1 for a root). */
static int odometry_walk(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                         const double* te, double* q, double* t, int32_t* parent, int32_t* pedge) {
    int64_t* par = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t* deg = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
    int64_t* tree = (int64_t*)malloc(sizeof(int64_t) * (size_t)(m > 0 ? m : 1));
    if (!par || !deg || !tree) { free(par); free(deg); free(tree); return -1; }
    for (int64_t i = 0; i < n; ++i) par[i] = i;
    int64_t nt = 0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t a = uf_find(par, src[e]), b = uf_find(par, dst[e]);
        if (a == b) continue;
        if (a < b) par[b] = a; else par[a] = b;
        tree[nt++] = e;
    }
    /* adjacency of the forest (CSR over both endpoints) */
    for (int64_t k = 0; k < nt; ++k) { deg[src[tree[k]] + 1]++; deg[dst[tree[k]] + 1]++; }
    for (int64_t i = 0; i < n; ++i) deg[i + 1] += deg[i];
    int64_t* adj = (int64_t*)malloc(sizeof(int64_t) * (size_t)(2 * nt + 1));
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    char* done = (char*)calloc((size_t)n + 1, 1);
    int64_t* queue = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!adj || !fill || !done || !queue) {
        free(par); free(deg); free(tree); free(adj); free(fill); free(done); free(queue);
        return -1;
    }
    for (int64_t i = 0; i < n; ++i) fill[i] = deg[i];
    for (int64_t k = 0; k < nt; ++k) {
        int64_t e = tree[k];
        adj[fill[src[e]]++] = e;
        adj[fill[dst[e]]++] = e;
    }
    for (int64_t r = 0; r < n; ++r) {
        if (done[r]) continue;
        /* r is the lowest vertex of a component not yet reached */
        if (q) {
            q[4 * r] = 1.0; q[4 * r + 1] = q[4 * r + 2] = q[4 * r + 3] = 0.0;
            t[3 * r] = t[3 * r + 1] = t[3 * r + 2] = 0.0;
        }
        if (parent) { parent[r] = -1; pedge[r] = -1; }
        done[r] = 1;
        int64_t head = 0, tail = 0;
        queue[tail++] = r;
        while (head < tail) {
            int64_t v = queue[head++];
            for (int64_t k = deg[v]; k < deg[v + 1]; ++k) {
                int64_t e = adj[k];
                int64_t a = src[e], b = dst[e];
                if (a == v && !done[b]) {
                    /* q_b = q_a q_e ; t_b = t_a + R(q_a) t_e */
                    if (q) {
                        double rt[3];
                        qmul(&q[4 * a], &qe[4 * e], &q[4 * b]);
                        qrotate(&q[4 * a], &te[3 * e], rt);
                        for (int c = 0; c < 3; ++c) t[3 * b + c] = t[3 * a + c] + rt[c];
                    }
                    if (parent) { parent[b] = (int32_t)a; pedge[b] = (int32_t)e; }
                    done[b] = 1;
                    queue[tail++] = b;
                } else if (b == v && !done[a]) {
                    /* q_a = q_b q_e^* ; t_a = t_b - R(q_a) t_e */
                    if (q) {
                        double qc[4], rt[3];
                        qconj(&qe[4 * e], qc);
                        qmul(&q[4 * b], qc, &q[4 * a]);
                        qrotate(&q[4 * a], &te[3 * e], rt);
                        for (int c = 0; c < 3; ++c) t[3 * a + c] = t[3 * b + c] - rt[c];
                    }
                    if (parent) { parent[a] = (int32_t)b; pedge[a] = (int32_t)(-(e + 2)); }
                    done[a] = 1;
                    queue[tail++] = a;
                }
            }
        }
    }
    free(par); free(deg); free(tree); free(adj); free(fill); free(done); free(queue);
    return 0;
}

int orc_init_odometry(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      const double* qe, const double* te, double* q, double* t) {
    return odometry_walk(n, m, src, dst, qe, te, q, t, NULL, NULL);
}

/* The forest of orc_init_odometry itself: parent and tree-edge code of every
 * vertex (see odometry_walk). */
int orc_odometry_forest(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, int32_t* parent,
                        int32_t* pedge) {
    return odometry_walk(n, m, src, dst, NULL, NULL, NULL, NULL, parent, pedge);
}

/* ---- objectives --------------------------------------------------------- */

/* Model (1), Eq. (1), at (q, t) with Sigma_1 = omega_e I_4, Sigma_2 = kappa_e I_4:
 * F = sum_e omega_e |t~_j - t~_i - q_i t~_ij q_i^*|^2 + kappa_e |q_j^* q_i q_ij - 1|^2 */
double orc_objective(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                     const double* qe, const double* te, const double* kappa,
                     const double* omega, const double* q, const double* t) {
    (void)n;
    double F = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double tp[4], a[4], qc[4], rot[4], r[4];
        qpure(&te[3 * e], tp);
        qmul(&q[4 * i], tp, a);
        qconj(&q[4 * i], qc);
        qmul(a, qc, rot);
        r[0] = -rot[0];
        for (int c = 0; c < 3; ++c) r[c + 1] = t[3 * j + c] - t[3 * i + c] - rot[c + 1];
        double w = omega ? omega[e] : 1.0;
        F += w * dot4(r, r);
        double qjc[4], b[4], g[4];
        qconj(&q[4 * j], qjc);
        qmul(qjc, &q[4 * i], b);
        qmul(b, &qe[4 * e], g);
        g[0] -= 1.0;
        double k = kappa ? kappa[e] : 1.0;
        F += k * dot4(g, g);
    }
    return F;
}

/* Split model (2): f = sum_e omega_e |t~_j - s~_i - q_i t~_ij p_i^*|^2,
 * g = sum_e kappa_e |p_j^* q_i q_ij - 1|^2.  Writes f and g. */
void orc_split_objective(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                         const double* qe, const double* te, const double* kappa,
                         const double* omega, const double* p, const double* q,
                         const double* t, const double* s, double* f_out, double* g_out) {
    (void)n;
    double f = 0.0, g = 0.0;
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double tp[4], a[4], pc[4], c[4], r[4];
        qpure(&te[3 * e], tp);
        qmul(&q[4 * i], tp, a);
        qconj(&p[4 * i], pc);
        qmul(a, pc, c);
        r[0] = -c[0];
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k] - c[k + 1];
        f += (omega ? omega[e] : 1.0) * dot4(r, r);
        double pjc[4], b[4], h[4];
        qconj(&p[4 * j], pjc);
        qmul(pjc, &q[4 * i], b);
        qmul(b, &qe[4 * e], h);
        h[0] -= 1.0;
        g += (kappa ? kappa[e] : 1.0) * dot4(h, h);
    }
    *f_out = f;
    *g_out = g;
}

/* Augmented Lagrangian L_beta of Section 3.2. */
double orc_lagrangian(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                      const double* qe, const double* te, const double* kappa,
                      const double* omega, const orc_params* prm, const double* p,
                      const double* q, const double* t, const double* s,
                      const double* lam, const double* z) {
    double f, g;
    orc_split_objective(n, m, src, dst, qe, te, kappa, omega, p, q, t, s, &f, &g);
    double L = f + g;
    for (int64_t i = 0; i < n; ++i) {
        double d2 = 0.0, ld = 0.0;
        for (int c = 0; c < 4; ++c) {
            double d = p[4 * i + c] - q[4 * i + c];
            ld += lam[4 * i + c] * d;
            d2 += d * d;
        }
        L += -ld + 0.5 * prm->beta1 * d2;
        double e2 = 0.0, zd = 0.0;
        for (int c = 0; c < 3; ++c) {
            double d = t[3 * i + c] - s[3 * i + c];
            zd += z[3 * i + c] * d;
            e2 += d * d;
        }
        L += -zd + 0.5 * prm->beta2 * e2;
    }
    return L;
}

/* ---- one PRADMM iteration, Eq. (3a)-(3f) / Algorithm 1 --------------------
 * The blocks below update (p, q, t, s, lam, z) in place from x^k to x^{k+1}
 * when called in the order of Algorithm 1: p, q, c, t, s, duals.  Each
 * block reads only what Eq. (3) gives it; ap .. as are the proximal anchors.
 * u, qn, tn, sn (4n, 4n, 3n, 3n) and a (n) are scratch; c (3m) carries c_e
 * from block_c to the t- and s-blocks. */

/* (3a) p-block, Appendix B.1.  With scalar Sigma the quadratic form A_1 is
 * a multiple of I_4 (Lemma MW(c)) and the minimiser of the linear term on
 * the unit sphere is p = -b_1/|b_1| = u/|u|, where
 *   u_i = sum_{out} 2 w_e G1^T r_e + sum_{in} 2 k_e G2^T 1~ + b1 q_i + lam_i + g1 p_i,
 * G1^T r = r^* q_i t~_e  (G1 = M(q_i) M(t~_e) D),
 * G2^T 1~ = q_l q_e      (G2 = W(q_e) W(q_l) D, reading R1),
 * r_e = t~_j - s~_i.  Returns the vertices whose |u_i| == 0 (R11). */
static int64_t block_p(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                       const double* te, const double* kappa, const double* omega, const orc_params* prm,
                       double* p, const double* q, const double* t, const double* s, const double* lam,
                       const double* ap, double* u) {
    const double b1 = prm->beta1, g1 = prm->gamma[0];
    int64_t nzero = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k)
            u[4 * i + k] = b1 * q[4 * i + k] + lam[4 * i + k] + g1 * ap[4 * i + k];
    for (int64_t e = 0; e < m; ++e) { /* out-edge sums: e = (i, j) */
        int64_t i = src[e], j = dst[e];
        double r[4], rc[4], tp[4], a[4], v[4];
        r[0] = 0.0;
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
        qconj(r, rc);
        qpure(&te[3 * e], tp);
        qmul(rc, &q[4 * i], a);
        qmul(a, tp, v);
        double w = 2.0 * (omega ? omega[e] : 1.0);
        for (int k = 0; k < 4; ++k) u[4 * i + k] += w * v[k];
    }
    for (int64_t e = 0; e < m; ++e) { /* in-edge sums: e = (l, i) */
        int64_t l = src[e], i = dst[e];
        double v[4];
        qmul(&q[4 * l], &qe[4 * e], v);
        double w = 2.0 * (kappa ? kappa[e] : 1.0);
        for (int k = 0; k < 4; ++k) u[4 * i + k] += w * v[k];
    }
    for (int64_t i = 0; i < n; ++i) {
        double nu = sqrt(dot4(&u[4 * i], &u[4 * i]));
        if (nu > 0.0) {
            for (int k = 0; k < 4; ++k) p[4 * i + k] = u[4 * i + k] / nu;
        } else {
            nzero++; /* R11: keep p_i^k */
        }
    }
    return nzero;
}

/* (3b) q-block, Appendix B.2: q_i = b_2 / A_2 with
 *   A_2 = sum_{out} 2 (w_e |p_i|^2 |t_e|^2 + k_e |p_j|^2 |q_e|^2) + b1 + g2,
 *   b_2 = sum_{out} 2 (w_e G3^T r_e + k_e G4^T 1~) + b1 p_i - lam_i + g2 q_i,
 * G3^T r = r p_i t~_e^*   (G3 = W(p_i)^T W(t~_e)),
 * G4^T 1~ = p_j q_e^*     (G4 = W(q_e) M(p_j)^T).                        */
static void block_q(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                    const double* te, const double* kappa, const double* omega, const orc_params* prm,
                    const double* p, double* q, const double* t, const double* s, const double* lam,
                    const double* aq, double* qn, double* a2) {
    const double b1 = prm->beta1, g2 = prm->gamma[1];
    for (int64_t i = 0; i < n; ++i) {
        a2[i] = b1 + g2;
        for (int k = 0; k < 4; ++k) qn[4 * i + k] = b1 * p[4 * i + k] - lam[4 * i + k] + g2 * aq[4 * i + k];
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = omega ? omega[e] : 1.0, kk = kappa ? kappa[e] : 1.0;
        double r[4], tp[4], tc[4], a[4], v[4], qc[4], h[4];
        r[0] = 0.0;
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
        qpure(&te[3 * e], tp);
        qconj(tp, tc);
        qmul(r, &p[4 * i], a);
        qmul(a, tc, v);
        qconj(&qe[4 * e], qc);
        qmul(&p[4 * j], qc, h);
        double tn2 = dot4(tp, tp);
        a2[i] += 2.0 * (w * dot4(&p[4 * i], &p[4 * i]) * tn2 +
                        kk * dot4(&p[4 * j], &p[4 * j]) * dot4(&qe[4 * e], &qe[4 * e]));
        for (int k = 0; k < 4; ++k) qn[4 * i + k] += 2.0 * (w * v[k] + kk * h[k]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k) q[4 * i + k] = qn[4 * i + k] / a2[i];
}

/* c_e = Im(q_i^{k+1} t~_e (p_i^{k+1})^*) for e = (i, j) (reading R3) */
static void block_c(int64_t m, const int32_t* src, const double* te, const double* p, const double* q, double* c) {
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e];
        double tp[4], a[4], pc[4], v[4];
        qpure(&te[3 * e], tp);
        qmul(&q[4 * i], tp, a);
        qconj(&p[4 * i], pc);
        qmul(a, pc, v);
        c[3 * e] = v[1]; c[3 * e + 1] = v[2]; c[3 * e + 2] = v[3];
    }
}

/* (3c) t-block, Appendix B.3 with hat-Sigma_1 = w_e I_3:
 *   t_i = [sum_{in} 2 w_e (s_l + c_e) + b2 s_i + z_i + g3 t_i] / [sum_{in} 2 w_e + b2 + g3] */
static void block_t(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* omega,
                    const orc_params* prm, double* t, const double* s, const double* z, const double* at,
                    const double* c, double* tn, double* a3) {
    const double b2 = prm->beta2, g3 = prm->gamma[2];
    for (int64_t i = 0; i < n; ++i) {
        a3[i] = b2 + g3;
        for (int k = 0; k < 3; ++k) tn[3 * i + k] = b2 * s[3 * i + k] + z[3 * i + k] + g3 * at[3 * i + k];
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t l = src[e], i = dst[e];
        double w = omega ? omega[e] : 1.0;
        a3[i] += 2.0 * w;
        for (int k = 0; k < 3; ++k) tn[3 * i + k] += 2.0 * w * (s[3 * l + k] + c[3 * e + k]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) t[3 * i + k] = tn[3 * i + k] / a3[i];
}

/* (3d) s-block, Appendix B.4 (the section's variable is s_i):
 *   s_i = [sum_{out} 2 w_e (t_j - c_e) + b2 t_i - z_i + g4 s_i] / [sum_{out} 2 w_e + b2 + g4] */
static void block_s(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* omega,
                    const orc_params* prm, const double* t, double* s, const double* z, const double* as,
                    const double* c, double* sn, double* a4) {
    const double b2 = prm->beta2, g4 = prm->gamma[3];
    for (int64_t i = 0; i < n; ++i) {
        a4[i] = b2 + g4;
        for (int k = 0; k < 3; ++k) sn[3 * i + k] = b2 * t[3 * i + k] - z[3 * i + k] + g4 * as[3 * i + k];
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = omega ? omega[e] : 1.0;
        a4[i] += 2.0 * w;
        for (int k = 0; k < 3; ++k) sn[3 * i + k] += 2.0 * w * (t[3 * j + k] - c[3 * e + k]);
    }
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 3; ++k) s[3 * i + k] = sn[3 * i + k] / a4[i];
}

/* (3e), (3f) relaxed dual updates */
static void block_duals(int64_t n, const orc_params* prm, const double* p, const double* q, const double* t,
                        const double* s, double* lam, double* z) {
    const double b1 = prm->beta1, b2 = prm->beta2, tau = prm->tau;
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 4; ++k) lam[4 * i + k] -= tau * b1 * (p[4 * i + k] - q[4 * i + k]);
        for (int k = 0; k < 3; ++k) z[3 * i + k] -= tau * b2 * (t[3 * i + k] - s[3 * i + k]);
    }
}

/* One iteration x^k -> x^{k+1} (in place).  res_out (nullable) receives 5
 * numbers: e^{k+1} (Appendix E.1, reading R6), then |dlam|^2, |dz|^2, |dq|^2,
 * |dt|^2.  Returns the number of vertices whose p-block hit |u_i| == 0 (R11),
 * or -1 if out of memory. */
static int64_t iterate_anchored(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                const double* qe, const double* te, const double* kappa,
                                const double* omega, const orc_params* prm, double* p, double* q,
                                double* t, double* s, double* lam, double* z, const double* ap,
                                const double* aq, const double* at, const double* as, double* res_out) {
    const double b1 = prm->beta1, b2 = prm->beta2;
    double* u = (double*)calloc((size_t)(4 * n + 1), sizeof(double));
    double* qn = (double*)calloc((size_t)(4 * n + 1), sizeof(double));
    double* a2 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* tn = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    double* a3 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* sn = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    double* a4 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* c = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
    double* qold = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* told = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* lold = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* zold = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    int64_t nzero = 0;
    if (!u || !qn || !a2 || !tn || !a3 || !sn || !a4 || !c || !qold || !told || !lold || !zold) {
        nzero = -1;
        goto out;
    }
    memcpy(qold, q, sizeof(double) * (size_t)(4 * n));
    memcpy(told, t, sizeof(double) * (size_t)(3 * n));
    memcpy(lold, lam, sizeof(double) * (size_t)(4 * n));
    memcpy(zold, z, sizeof(double) * (size_t)(3 * n));

    nzero = block_p(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, ap, u);
    block_q(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, aq, qn, a2);
    block_c(m, src, te, p, q, c);
    block_t(n, m, src, dst, omega, prm, t, s, z, at, c, tn, a3);
    block_s(n, m, src, dst, omega, prm, t, s, z, as, c, sn, a4);
    block_duals(n, prm, p, q, t, s, lam, z);

    /* residual of Appendix E.1 (reading R6) */
    if (res_out) {
        double dl = 0.0, dz = 0.0, dq = 0.0, dt = 0.0;
        for (int64_t k = 0; k < 4 * n; ++k) {
            double a = lam[k] - lold[k], b = q[k] - qold[k];
            dl += a * a;
            dq += b * b;
        }
        for (int64_t k = 0; k < 3 * n; ++k) {
            double a = z[k] - zold[k], b = t[k] - told[k];
            dz += a * a;
            dt += b * b;
        }
        res_out[0] = dl / b1 + dz / b2 + b1 * dq + b2 * dt;
        res_out[1] = dl; res_out[2] = dz; res_out[3] = dq; res_out[4] = dt;
    }
out:
    free(u); free(qn); free(a2); free(tn); free(a3); free(sn); free(a4); free(c);
    free(qold); free(told); free(lold); free(zold);
    return nzero;
}

/* One block of plain PRADMM (anchors x^k), for callers that run the blocks
 * of Algorithm 1 one at a time (the vertex-partitioned iteration exchanges
 * halo values between them): which = 0 p, 1 q, 2 c_e, 3 t, 4 s, 5 duals.
 * c (3m) carries c_e from block 2 to blocks 3 and 4.  Returns the p-block's
 * |u| == 0 count (block 0), 0 for the others, -1 if out of memory or
 * `which` is unknown. */
int64_t orc_block(int which, int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                  const double* te, const double* kappa, const double* omega, const orc_params* prm, double* p,
                  double* q, double* t, double* s, double* lam, double* z, double* c) {
    int64_t r = 0;
    double* w4 = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* w1 = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    double* anc = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    if (!w4 || !w1 || !anc) {
        r = -1;
        goto out;
    }
    switch (which) {
        case 0:
            memcpy(anc, p, sizeof(double) * (size_t)(4 * n));
            r = block_p(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, anc, w4);
            break;
        case 1:
            memcpy(anc, q, sizeof(double) * (size_t)(4 * n));
            block_q(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, anc, w4, w1);
            break;
        case 2: block_c(m, src, te, p, q, c); break;
        case 3:
            memcpy(anc, t, sizeof(double) * (size_t)(3 * n));
            block_t(n, m, src, dst, omega, prm, t, s, z, anc, c, w4, w1);
            break;
        case 4:
            memcpy(anc, s, sizeof(double) * (size_t)(3 * n));
            block_s(n, m, src, dst, omega, prm, t, s, z, anc, c, w4, w1);
            break;
        case 5: block_duals(n, prm, p, q, t, s, lam, z); break;
        default: r = -1;
    }
out:
    free(w4);
    free(w1);
    free(anc);
    return r;
}

/* The proximal anchors of the four primal blocks (the points the terms
 * 1/2 |x - x^{k+1/2}|^2_{H} of Appendix B pull towards) are ap, aq, at, as;
 * every term that reads them does so before its block overwrites the iterate,
 * so passing the iterate itself gives the anchors x^{k+1/2} = x^k (reading
 * R4) of plain PRADMM. */
int64_t orc_iterate(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                    const double* qe, const double* te, const double* kappa,
                    const double* omega, const orc_params* prm, double* p, double* q,
                    double* t, double* s, double* lam, double* z, double* res_out) {
    return iterate_anchored(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, z, p, q, t, s, res_out);
}

/* Inertial PRADMM (reading R27): the anchors are the extrapolated points
 *   x^{k+1/2} = x^k + theta (x^k - x^{k-1})     for x = p, q, t, s,
 * with x^{k-1} in pp, qp, tp, sp (equal to x^0 before the first iteration);
 * theta = 0 is plain PRADMM.  On return pp .. sp hold x^k, the previous
 * iterate of the next call.  Returns as orc_iterate, or -1 if out of memory. */
int64_t orc_iterate_inertial(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                             const double* qe, const double* te, const double* kappa,
                             const double* omega, const orc_params* prm, double theta, double* p,
                             double* q, double* t, double* s, double* lam, double* z, double* pp,
                             double* qp, double* tp, double* sp, double* res_out) {
    double* ap = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* aq = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* at = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* as = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    int64_t r = -1;
    if (ap && aq && at && as) {
        for (int64_t k = 0; k < 4 * n; ++k) {
            ap[k] = p[k] + theta * (p[k] - pp[k]);
            aq[k] = q[k] + theta * (q[k] - qp[k]);
        }
        for (int64_t k = 0; k < 3 * n; ++k) {
            at[k] = t[k] + theta * (t[k] - tp[k]);
            as[k] = s[k] + theta * (s[k] - sp[k]);
        }
        memcpy(pp, p, sizeof(double) * (size_t)(4 * n));
        memcpy(qp, q, sizeof(double) * (size_t)(4 * n));
        memcpy(tp, t, sizeof(double) * (size_t)(3 * n));
        memcpy(sp, s, sizeof(double) * (size_t)(3 * n));
        r = iterate_anchored(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, z, ap, aq, at, as, res_out);
    }
    free(ap); free(aq); free(at); free(as);
    return r;
}

/* Algorithm 1 with the stopping rule of Appendix E.1: iterate until
 * e^{k+1} < tol or max_iter iterations.  Returns the iterations done;
 * e_out receives the last residual, trace (nullable, max_iter entries)
 * every residual. */
int64_t orc_solve(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                  const double* qe, const double* te, const double* kappa,
                  const double* omega, const orc_params* prm, int64_t max_iter, double tol,
                  double* p, double* q, double* t, double* s, double* lam, double* z,
                  double* e_out, double* trace) {
    double res[5] = {0, 0, 0, 0, 0};
    int64_t k = 0;
    while (k < max_iter) {
        orc_iterate(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, z, res);
        if (trace) trace[k] = res[0];
        ++k;
        if (res[0] < tol) break;
    }
    if (e_out) *e_out = res[0];
    return k;
}

/* ---- reverse mode of one iteration ------------------------------------------
 * Vector-Jacobian product of the map x^k -> x^{k+1} of orc_iterate (Eq. (3a)-
 * (3f) with the Appendix B closed forms), written by hand step by step in
 * reverse order.  For a quaternion product V = a x b the adjoint of x is
 * a^* V_bar b^* (Lemma MW: left/right multiplication matrices are orthogonal
 * up to scale, M(a)^T = M(a^*), W(b)^T = W(b^*)); a conjugate x^* = D x
 * contributes the conjugate of that adjoint; the normalisation p = u/|u| has
 * adjoint u_bar = (I - p p^T) p_bar / |u|.
 *
 * in:  x^k (p, q, t, s, lam, z) and the adjoints of x^{k+1} (pb1 .. zb1)
 * out: adjoints of x^k (pb .. zb, overwritten) and of the measurements,
 *      ACCUMULATED: qeb (m x 4), teb (m x 3), kab (m), omb (m).
 * Returns 0, or -1 on allocation failure.
 */
static void qadd(double* a, const double* b, double s) {
    for (int k = 0; k < 4; ++k) a[k] += s * b[k];
}

/* The reverse mode of one iteration as above, with proximal anchors ap, aq,
 * at, as in place of x^k (the forward is iterate_anchored), formed as x^k + theta (x^k - x^{k-1}) (reading R27):
 * each gamma term's adjoint goes (1 + theta) to x^k and -theta to x^{k-1},
 * the latter written to ppb, qpb, tpb, spb (overwritten; NULL when theta is
 * 0, where the anchors are x^k and this is orc_iterate_adjoint). */
static int iterate_adjoint_anchored(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                                    const double* te, const double* kappa, const double* omega,
                                    const orc_params* prm, const double* p, const double* q, const double* t,
                                    const double* s, const double* lam, const double* z, const double* ap,
                                    const double* aq, const double* at, const double* as, double theta,
                                    const double* pb1, const double* qb1, const double* tb1, const double* sb1,
                                    const double* lb1, const double* zb1, double* pb, double* qb, double* tb,
                                    double* sb, double* lb, double* zb, double* ppb, double* qpb, double* tpb,
                                    double* spb, double* qeb, double* teb, double* kab, double* omb) {
    const double b1 = prm->beta1, b2 = prm->beta2, tau = prm->tau;
    const double g1 = prm->gamma[0], g2 = prm->gamma[1], g3 = prm->gamma[2], g4 = prm->gamma[3];
    const double cur = 1.0 + theta, prv = -theta; /* d anchor / d x^k, d anchor / d x^{k-1} */
    /* forward intermediates, recomputed exactly as the forward does */
    double* P = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* Qn = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* Tn = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* Sn = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* L = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    double* Z = (double*)malloc(sizeof(double) * (size_t)(3 * n + 1));
    double* u = (double*)calloc((size_t)(4 * n + 1), sizeof(double));
    double* nu = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* a2 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* a3 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* a4 = (double*)calloc((size_t)(n + 1), sizeof(double));
    double* c = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
    /* adjoint accumulators */
    double* pba = (double*)calloc((size_t)(4 * n + 1), sizeof(double)); /* of p^{k+1} */
    double* qba = (double*)calloc((size_t)(4 * n + 1), sizeof(double)); /* of q^{k+1} */
    double* tba = (double*)calloc((size_t)(3 * n + 1), sizeof(double)); /* of t^{k+1} */
    double* sba = (double*)calloc((size_t)(3 * n + 1), sizeof(double)); /* of s^{k+1} */
    double* cb = (double*)calloc((size_t)(3 * m + 1), sizeof(double));
    double* gs = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    double* gt = (double*)calloc((size_t)(3 * n + 1), sizeof(double));
    double* gq = (double*)calloc((size_t)(4 * n + 1), sizeof(double));
    double* ub = (double*)calloc((size_t)(4 * n + 1), sizeof(double));
    int rc = 0;
    if (!P || !Qn || !Tn || !Sn || !L || !Z || !u || !nu || !a2 || !a3 || !a4 || !c || !pba || !qba || !tba ||
        !sba || !cb || !gs || !gt || !gq || !ub) {
        rc = -1;
        goto out;
    }
    memcpy(P, p, sizeof(double) * (size_t)(4 * n));
    memcpy(Qn, q, sizeof(double) * (size_t)(4 * n));
    memcpy(Tn, t, sizeof(double) * (size_t)(3 * n));
    memcpy(Sn, s, sizeof(double) * (size_t)(3 * n));
    memcpy(L, lam, sizeof(double) * (size_t)(4 * n));
    memcpy(Z, z, sizeof(double) * (size_t)(3 * n));
    if (iterate_anchored(n, m, src, dst, qe, te, kappa, omega, prm, P, Qn, Tn, Sn, L, Z, ap, aq, at, as, NULL) < 0) {
        rc = -1;
        goto out;
    }
    /* u and |u| of the p-block (same order of operations as the forward) */
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 4; ++k) u[4 * i + k] = b1 * q[4 * i + k] + lam[4 * i + k] + g1 * ap[4 * i + k];
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double r[4], rc_[4], tp[4], a[4], v[4];
        r[0] = 0.0;
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
        qconj(r, rc_);
        qpure(&te[3 * e], tp);
        qmul(rc_, &q[4 * i], a);
        qmul(a, tp, v);
        qadd(&u[4 * i], v, 2.0 * (omega ? omega[e] : 1.0));
    }
    for (int64_t e = 0; e < m; ++e) {
        double v[4];
        qmul(&q[4 * src[e]], &qe[4 * e], v);
        qadd(&u[4 * dst[e]], v, 2.0 * (kappa ? kappa[e] : 1.0));
    }
    for (int64_t i = 0; i < n; ++i) nu[i] = sqrt(dot4(&u[4 * i], &u[4 * i]));
    for (int64_t i = 0; i < n; ++i) {
        a2[i] = b1 + g2;
        a3[i] = b2 + g3;
        a4[i] = b2 + g4;
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = omega ? omega[e] : 1.0, kk = kappa ? kappa[e] : 1.0, tp[4];
        qpure(&te[3 * e], tp);
        a2[i] += 2.0 * (w * dot4(&P[4 * i], &P[4 * i]) * dot4(tp, tp) + kk * dot4(&P[4 * j], &P[4 * j]) * dot4(&qe[4 * e], &qe[4 * e]));
        a3[j] += 2.0 * w;
        a4[i] += 2.0 * w;
        double a[4], pc[4], v[4];
        qmul(&Qn[4 * i], tp, a);
        qconj(&P[4 * i], pc);
        qmul(a, pc, v);
        c[3 * e] = v[1]; c[3 * e + 1] = v[2]; c[3 * e + 2] = v[3];
    }
    memset(pb, 0, sizeof(double) * (size_t)(4 * n));
    memset(qb, 0, sizeof(double) * (size_t)(4 * n));
    memset(tb, 0, sizeof(double) * (size_t)(3 * n));
    memset(sb, 0, sizeof(double) * (size_t)(3 * n));
    memset(lb, 0, sizeof(double) * (size_t)(4 * n));
    memset(zb, 0, sizeof(double) * (size_t)(3 * n));
    /* (3e), (3f) */
    for (int64_t i = 0; i < n; ++i) {
        for (int k = 0; k < 4; ++k) {
            lb[4 * i + k] += lb1[4 * i + k];
            pba[4 * i + k] = pb1[4 * i + k] - tau * b1 * lb1[4 * i + k];
            qba[4 * i + k] = qb1[4 * i + k] + tau * b1 * lb1[4 * i + k];
        }
        for (int k = 0; k < 3; ++k) {
            zb[3 * i + k] += zb1[3 * i + k];
            tba[3 * i + k] = tb1[3 * i + k] - tau * b2 * zb1[3 * i + k];
            sba[3 * i + k] = sb1[3 * i + k] + tau * b2 * zb1[3 * i + k];
        }
    }
    /* (3d) s = sn / a4 */
    for (int64_t i = 0; i < n; ++i) {
        double a4b = 0.0;
        for (int k = 0; k < 3; ++k) {
            gs[3 * i + k] = sba[3 * i + k] / a4[i];
            a4b -= gs[3 * i + k] * Sn[3 * i + k];
            tba[3 * i + k] += b2 * gs[3 * i + k];
            zb[3 * i + k] -= gs[3 * i + k];
            sb[3 * i + k] += cur * g4 * gs[3 * i + k];
            if (spb) spb[3 * i + k] = prv * g4 * gs[3 * i + k];
        }
        a4[i] = a4b; /* reuse: adjoint of A_4 */
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = omega ? omega[e] : 1.0, dot = 0.0;
        for (int k = 0; k < 3; ++k) {
            tba[3 * j + k] += 2.0 * w * gs[3 * i + k];
            cb[3 * e + k] -= 2.0 * w * gs[3 * i + k];
            dot += (Tn[3 * j + k] - c[3 * e + k]) * gs[3 * i + k];
        }
        omb[e] += 2.0 * dot + 2.0 * a4[i];
    }
    /* (3c) t = tn / a3 */
    for (int64_t i = 0; i < n; ++i) {
        double a3b = 0.0;
        for (int k = 0; k < 3; ++k) {
            gt[3 * i + k] = tba[3 * i + k] / a3[i];
            a3b -= gt[3 * i + k] * Tn[3 * i + k];
            sb[3 * i + k] += b2 * gt[3 * i + k];
            zb[3 * i + k] += gt[3 * i + k];
            tb[3 * i + k] += cur * g3 * gt[3 * i + k];
            if (tpb) tpb[3 * i + k] = prv * g3 * gt[3 * i + k];
        }
        a3[i] = a3b;
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t l = src[e], i = dst[e];
        double w = omega ? omega[e] : 1.0, dot = 0.0;
        for (int k = 0; k < 3; ++k) {
            sb[3 * l + k] += 2.0 * w * gt[3 * i + k];
            cb[3 * e + k] += 2.0 * w * gt[3 * i + k];
            dot += (s[3 * l + k] + c[3 * e + k]) * gt[3 * i + k];
        }
        omb[e] += 2.0 * dot + 2.0 * a3[i];
    }
    /* c_e = Im(q'_i t~_e p'_i^*) */
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e];
        double hb[4] = {0.0, cb[3 * e], cb[3 * e + 1], cb[3 * e + 2]}, tp[4], tc[4], a[4], v[4], qc[4];
        qpure(&te[3 * e], tp);
        qconj(tp, tc);
        /* q' adjoint: hb (t~ p'^*)^* = hb p' t~^* */
        qmul(hb, &P[4 * i], a);
        qmul(a, tc, v);
        qadd(&qba[4 * i], v, 1.0);
        /* p' adjoint: hb^* (q' t~) */
        double hc[4];
        qconj(hb, hc);
        qmul(&Qn[4 * i], tp, a);
        qmul(hc, a, v);
        qadd(&pba[4 * i], v, 1.0);
        /* t~ adjoint: q'^* hb p' */
        qconj(&Qn[4 * i], qc);
        qmul(qc, hb, a);
        qmul(a, &P[4 * i], v);
        for (int k = 0; k < 3; ++k) teb[3 * e + k] += v[k + 1];
    }
    /* (3b) q = qn / a2 */
    for (int64_t i = 0; i < n; ++i) {
        double a2b = 0.0;
        for (int k = 0; k < 4; ++k) {
            gq[4 * i + k] = qba[4 * i + k] / a2[i];
            a2b -= gq[4 * i + k] * Qn[4 * i + k];
            pba[4 * i + k] += b1 * gq[4 * i + k];
            lb[4 * i + k] -= gq[4 * i + k];
            qb[4 * i + k] += cur * g2 * gq[4 * i + k];
            if (qpb) qpb[4 * i + k] = prv * g2 * gq[4 * i + k];
        }
        a2[i] = a2b;
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = omega ? omega[e] : 1.0, kk = kappa ? kappa[e] : 1.0;
        double r[4], tp[4], tc[4], a[4], v[4], g[4];
        r[0] = 0.0;
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
        qpure(&te[3 * e], tp);
        qconj(tp, tc);
        memcpy(g, &gq[4 * i], sizeof(g));
        /* term 2 w r p'_i t~^* */
        qmul(g, tp, a); /* g t~ */
        double pc[4];
        qconj(&P[4 * i], pc);
        qmul(a, pc, v); /* g t~ p'^*  = adjoint of r (times 2w) */
        for (int k = 0; k < 3; ++k) {
            tb[3 * j + k] += 2.0 * w * v[k + 1];
            sb[3 * i + k] -= 2.0 * w * v[k + 1];
        }
        double rcj[4];
        qconj(r, rcj);
        qmul(rcj, g, a); /* r^* g */
        qmul(a, tp, v);  /* r^* g t~ = (r)^* g (t~^*)^* */
        qadd(&pba[4 * i], v, 2.0 * w);
        double gc[4], rp[4];
        qconj(g, gc);
        qmul(r, &P[4 * i], rp);
        qmul(gc, rp, v); /* g^* (r p') */
        for (int k = 0; k < 3; ++k) teb[3 * e + k] += 2.0 * w * v[k + 1];
        double tv[4];
        qmul(rp, tc, tv);
        omb[e] += 2.0 * dot4(g, tv);
        /* term 2 k p'_j q_e^* */
        qmul(g, &qe[4 * e], v); /* g (q_e^*)^* */
        qadd(&pba[4 * j], v, 2.0 * kk);
        qmul(gc, &P[4 * j], v); /* g^* p'_j */
        qadd(&qeb[4 * e], v, 2.0 * kk);
        double qc[4];
        qconj(&qe[4 * e], qc);
        qmul(&P[4 * j], qc, v);
        kab[e] += 2.0 * dot4(g, v);
        /* A_2 = ... + 2 (w |p'_i|^2 |t_e|^2 + k |p'_j|^2 |q_e|^2) */
        double pn2 = dot4(&P[4 * i], &P[4 * i]), pj2 = dot4(&P[4 * j], &P[4 * j]);
        double tn2 = dot4(tp, tp), qn2 = dot4(&qe[4 * e], &qe[4 * e]);
        omb[e] += 2.0 * pn2 * tn2 * a2[i];
        kab[e] += 2.0 * pj2 * qn2 * a2[i];
        for (int k = 0; k < 3; ++k) teb[3 * e + k] += 4.0 * w * pn2 * te[3 * e + k] * a2[i];
        qadd(&qeb[4 * e], &qe[4 * e], 4.0 * kk * pj2 * a2[i]);
        qadd(&pba[4 * i], &P[4 * i], 4.0 * w * tn2 * a2[i]);
        qadd(&pba[4 * j], &P[4 * j], 4.0 * kk * qn2 * a2[i]);
    }
    /* (3a) p = u / |u|  (|u| = 0 keeps p^k: p' = p) */
    for (int64_t i = 0; i < n; ++i) {
        if (nu[i] > 0.0) {
            double pp = dot4(&P[4 * i], &pba[4 * i]);
            for (int k = 0; k < 4; ++k) ub[4 * i + k] = (pba[4 * i + k] - P[4 * i + k] * pp) / nu[i];
        } else {
            for (int k = 0; k < 4; ++k) pb[4 * i + k] += pba[4 * i + k];
        }
        for (int k = 0; k < 4; ++k) {
            qb[4 * i + k] += b1 * ub[4 * i + k];
            lb[4 * i + k] += ub[4 * i + k];
            pb[4 * i + k] += cur * g1 * ub[4 * i + k];
            if (ppb) ppb[4 * i + k] = prv * g1 * ub[4 * i + k];
        }
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e], j = dst[e];
        double w = 2.0 * (omega ? omega[e] : 1.0);
        double r[4], rcj[4], tp[4], tc[4], qt[4], a[4], v[4], g[4];
        r[0] = 0.0;
        for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
        qconj(r, rcj);
        qpure(&te[3 * e], tp);
        qconj(tp, tc);
        memcpy(g, &ub[4 * i], sizeof(g));
        /* V = w r^* q_i t~ : adjoint of r^* is w g (q_i t~)^*, of r its conjugate */
        qmul(&q[4 * i], tp, qt);
        double qtc[4];
        qconj(qt, qtc);
        qmul(g, qtc, a);
        for (int k = 0; k < 3; ++k) {
            tb[3 * j + k] -= w * a[k + 1];
            sb[3 * i + k] += w * a[k + 1];
        }
        /* q_i: (w r^*)^* g t~^* = w r g t~^* */
        qmul(r, g, a);
        qmul(a, tc, v);
        qadd(&qb[4 * i], v, w);
        /* t~: (w r^* q_i)^* g */
        double rq[4], rqc[4];
        qmul(rcj, &q[4 * i], rq);
        qconj(rq, rqc);
        qmul(rqc, g, v);
        for (int k = 0; k < 3; ++k) teb[3 * e + k] += w * v[k + 1];
        qmul(rq, tp, v);
        omb[e] += 2.0 * dot4(g, v);
    }
    for (int64_t e = 0; e < m; ++e) {
        int64_t l = src[e], i = dst[e];
        double kk = 2.0 * (kappa ? kappa[e] : 1.0), g[4], qc[4], ql[4], v[4];
        memcpy(g, &ub[4 * i], sizeof(g));
        qconj(&qe[4 * e], qc);
        qmul(g, qc, v); /* g q_e^* */
        qadd(&qb[4 * l], v, kk);
        qconj(&q[4 * l], ql);
        qmul(ql, g, v); /* q_l^* g */
        qadd(&qeb[4 * e], v, kk);
        qmul(&q[4 * l], &qe[4 * e], v);
        kab[e] += 2.0 * dot4(g, v);
    }
out:
    free(P); free(Qn); free(Tn); free(Sn); free(L); free(Z); free(u); free(nu); free(a2); free(a3); free(a4);
    free(c); free(pba); free(qba); free(tba); free(sba); free(cb); free(gs); free(gt); free(gq); free(ub);
    return rc;
}

int orc_iterate_adjoint(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                        const double* te, const double* kappa, const double* omega, const orc_params* prm,
                        const double* p, const double* q, const double* t, const double* s, const double* lam,
                        const double* z, const double* pb1, const double* qb1, const double* tb1,
                        const double* sb1, const double* lb1, const double* zb1, double* pb, double* qb,
                        double* tb, double* sb, double* lb, double* zb, double* qeb, double* teb, double* kab,
                        double* omb) {
    return iterate_adjoint_anchored(n, m, src, dst, qe, te, kappa, omega, prm, p, q, t, s, lam, z, p, q, t, s, 0.0,
                                    pb1, qb1, tb1, sb1, lb1, zb1, pb, qb, tb, sb, lb, zb, NULL, NULL, NULL, NULL,
                                    qeb, teb, kab, omb);
}

/* Gradient of a terminal loss through `iters` iterations of Algorithm 1 from
 * a fixed x^0 (reverse mode: every state x^0 .. x^{iters} is kept, then
 * orc_iterate_adjoint runs from the last iteration back to the first).
 * pbK, tbK: dL/dp^K (n x 4) and dL/dt^K (n x 3); the loss depends on no
 * other part of x^K.  Outputs dL/dq_e (m x 4), dL/dt_e (m x 3), dL/dkappa_e,
 * dL/domega_e (each overwritten), x^K's p and t (nullable), and the adjoint
 * of x^0 packed as (p, q, t, s, lam, z), 21 n values (nullable).
 * Returns 0, or -1 on allocation failure. */
int orc_adjoint(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe, const double* te,
                const double* kappa, const double* omega, const orc_params* prm, int64_t iters, const double* p0,
                const double* q0, const double* t0, const double* s0, const double* lam0, const double* z0,
                const double* pbK, const double* tbK, double* pK, double* tK, double* qeb, double* teb,
                double* kab, double* omb, double* x0b) {
    const int64_t W = 21 * n; /* one state: p 4n, q 4n, t 3n, s 3n, lam 4n, z 3n */
    const int64_t off[6] = {0, 4 * n, 8 * n, 11 * n, 14 * n, 18 * n};
    double* tape = (double*)malloc(sizeof(double) * (size_t)(W * (iters + 1) + 1));
    double* bar = (double*)calloc((size_t)(2 * W + 1), sizeof(double));
    int rc = 0;
    if (!tape || !bar) {
        rc = -1;
        goto out;
    }
    memcpy(tape + off[0], p0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[1], q0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[2], t0, sizeof(double) * (size_t)(3 * n));
    memcpy(tape + off[3], s0, sizeof(double) * (size_t)(3 * n));
    memcpy(tape + off[4], lam0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[5], z0, sizeof(double) * (size_t)(3 * n));
    for (int64_t k = 0; k < iters; ++k) {
        double* x = tape + W * (k + 1);
        memcpy(x, tape + W * k, sizeof(double) * (size_t)W);
        if (orc_iterate(n, m, src, dst, qe, te, kappa, omega, prm, x + off[0], x + off[1], x + off[2], x + off[3],
                        x + off[4], x + off[5], NULL) < 0) {
            rc = -1;
            goto out;
        }
    }
    if (pK) memcpy(pK, tape + W * iters + off[0], sizeof(double) * (size_t)(4 * n));
    if (tK) memcpy(tK, tape + W * iters + off[2], sizeof(double) * (size_t)(3 * n));
    memset(qeb, 0, sizeof(double) * (size_t)(4 * m));
    memset(teb, 0, sizeof(double) * (size_t)(3 * m));
    memset(kab, 0, sizeof(double) * (size_t)m);
    memset(omb, 0, sizeof(double) * (size_t)m);
    /* bar[0 .. W) holds the adjoint of x^{k+1}, bar[W .. 2W) receives that of x^k */
    memcpy(bar + off[0], pbK, sizeof(double) * (size_t)(4 * n));
    memcpy(bar + off[2], tbK, sizeof(double) * (size_t)(3 * n));
    for (int64_t k = iters - 1; k >= 0; --k) {
        const double* x = tape + W * k;
        double *a1 = bar, *a0 = bar + W;
        if (orc_iterate_adjoint(n, m, src, dst, qe, te, kappa, omega, prm, x + off[0], x + off[1], x + off[2],
                                x + off[3], x + off[4], x + off[5], a1 + off[0], a1 + off[1], a1 + off[2],
                                a1 + off[3], a1 + off[4], a1 + off[5], a0 + off[0], a0 + off[1], a0 + off[2],
                                a0 + off[3], a0 + off[4], a0 + off[5], qeb, teb, kab, omb) < 0) {
            rc = -1;
            goto out;
        }
        memcpy(a1, a0, sizeof(double) * (size_t)W);
    }
    if (x0b) memcpy(x0b, bar, sizeof(double) * (size_t)W);
out:
    free(tape);
    free(bar);
    return rc;
}

/* orc_adjoint for the inertial iteration (orc_iterate_inertial, reading R27)
 * started with x^{-1} = x^0.  Iteration k reads x^k and x^{k-1} (through
 * its anchors), so the reverse pass carries, besides the adjoint of x^{k+1},
 * the share of x^k's adjoint that iteration k+1 produced through its anchors
 * (p, q, t, s); x^{-1} is x^0, so the last such share joins x0b.  Arguments
 * and outputs as orc_adjoint, plus theta. */
int orc_adjoint_inertial(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                         const double* te, const double* kappa, const double* omega, const orc_params* prm,
                         double theta, int64_t iters, const double* p0, const double* q0, const double* t0,
                         const double* s0, const double* lam0, const double* z0, const double* pbK,
                         const double* tbK, double* pK, double* tK, double* qeb, double* teb, double* kab,
                         double* omb, double* x0b) {
    const int64_t W = 21 * n;
    const int64_t off[6] = {0, 4 * n, 8 * n, 11 * n, 14 * n, 18 * n};
    double* tape = (double*)malloc(sizeof(double) * (size_t)(W * (iters + 1) + 1));
    double* bar = (double*)calloc((size_t)(2 * W + 1), sizeof(double));
    double* pend = (double*)calloc((size_t)(W + 1), sizeof(double)); /* p, q, t, s parts used */
    double* prev = (double*)calloc((size_t)(W + 1), sizeof(double));
    double* anc = (double*)malloc(sizeof(double) * (size_t)(W + 1));
    int rc = 0;
    if (!tape || !bar || !pend || !prev || !anc) {
        rc = -1;
        goto out;
    }
    memcpy(tape + off[0], p0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[1], q0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[2], t0, sizeof(double) * (size_t)(3 * n));
    memcpy(tape + off[3], s0, sizeof(double) * (size_t)(3 * n));
    memcpy(tape + off[4], lam0, sizeof(double) * (size_t)(4 * n));
    memcpy(tape + off[5], z0, sizeof(double) * (size_t)(3 * n));
    memcpy(prev, tape, sizeof(double) * (size_t)W); /* x^{-1} = x^0 */
    for (int64_t k = 0; k < iters; ++k) {
        double* x = tape + W * (k + 1);
        memcpy(x, tape + W * k, sizeof(double) * (size_t)W);
        if (orc_iterate_inertial(n, m, src, dst, qe, te, kappa, omega, prm, theta, x + off[0], x + off[1],
                                 x + off[2], x + off[3], x + off[4], x + off[5], prev + off[0], prev + off[1],
                                 prev + off[2], prev + off[3], NULL) < 0) {
            rc = -1;
            goto out;
        }
    }
    if (pK) memcpy(pK, tape + W * iters + off[0], sizeof(double) * (size_t)(4 * n));
    if (tK) memcpy(tK, tape + W * iters + off[2], sizeof(double) * (size_t)(3 * n));
    memset(qeb, 0, sizeof(double) * (size_t)(4 * m));
    memset(teb, 0, sizeof(double) * (size_t)(3 * m));
    memset(kab, 0, sizeof(double) * (size_t)m);
    memset(omb, 0, sizeof(double) * (size_t)m);
    memcpy(bar + off[0], pbK, sizeof(double) * (size_t)(4 * n));
    memcpy(bar + off[2], tbK, sizeof(double) * (size_t)(3 * n));
    for (int64_t k = iters - 1; k >= 0; --k) {
        const double* x = tape + W * k;
        const double* xp = tape + W * (k > 0 ? k - 1 : 0);
        /* the anchors of iteration k, formed as the forward forms them */
        for (int64_t j = 0; j < 4 * n; ++j) {
            anc[off[0] + j] = x[off[0] + j] + theta * (x[off[0] + j] - xp[off[0] + j]);
            anc[off[1] + j] = x[off[1] + j] + theta * (x[off[1] + j] - xp[off[1] + j]);
        }
        for (int64_t j = 0; j < 3 * n; ++j) {
            anc[off[2] + j] = x[off[2] + j] + theta * (x[off[2] + j] - xp[off[2] + j]);
            anc[off[3] + j] = x[off[3] + j] + theta * (x[off[3] + j] - xp[off[3] + j]);
        }
        double *a1 = bar, *a0 = bar + W;
        if (iterate_adjoint_anchored(n, m, src, dst, qe, te, kappa, omega, prm, x + off[0], x + off[1], x + off[2],
                                     x + off[3], x + off[4], x + off[5], anc + off[0], anc + off[1], anc + off[2],
                                     anc + off[3], theta, a1 + off[0], a1 + off[1], a1 + off[2], a1 + off[3],
                                     a1 + off[4], a1 + off[5], a0 + off[0], a0 + off[1], a0 + off[2], a0 + off[3],
                                     a0 + off[4], a0 + off[5], prev + off[0], prev + off[1], prev + off[2],
                                     prev + off[3], qeb, teb, kab, omb) < 0) {
            rc = -1;
            goto out;
        }
        /* adjoint of x^k: this iteration's share plus iteration k+1's anchor share */
        for (int64_t j = 0; j < 14 * n; ++j) a0[j] += pend[j];
        memcpy(pend, prev, sizeof(double) * (size_t)(14 * n));
        memcpy(a1, a0, sizeof(double) * (size_t)W);
    }
    /* x^{-1} is x^0 */
    for (int64_t j = 0; j < 14 * n; ++j) bar[j] += pend[j];
    if (x0b) memcpy(x0b, bar, sizeof(double) * (size_t)W);
out:
    free(tape);
    free(bar);
    free(pend);
    free(prev);
    free(anc);
    return rc;
}

#ifdef ORC_OPENMP
/* ---- OpenMP timing build (compiled only with -DORC_OPENMP -fopenmp) ---------
 * A CPU baseline, not the checker: the same iteration as orc_iterate with
 * every block's loop running over vertices in parallel.  The sweeps of
 * Eq. (3a)-(3d) are Jacobi over vertices (every vertex of a block reads only
 * values from before the block), so a vertex can sum its own edges.  The
 * caller passes each vertex's out-edges (tail i) and in-edges (head i) in
 * input order -- out_eid[out_ptr[i] .. out_ptr[i+1]) and likewise for in --
 * so every per-vertex sum adds the same terms in the same order as the
 * sequential edge loops above, and the state comes out bitwise equal to
 * orc_iterate's.  Only the residual's four sums are reduced in another
 * order.  Plain PRADMM (anchors x^k), scalar weights. */
#include <omp.h>

int orc_omp_threads(void) { return omp_get_max_threads(); }

int64_t orc_iterate_omp(int64_t n, int64_t m, const int32_t* src, const int32_t* dst, const double* qe,
                        const double* te, const double* kappa, const double* omega, const orc_params* prm,
                        const int64_t* out_ptr, const int32_t* out_eid, const int64_t* in_ptr,
                        const int32_t* in_eid, double* p, double* q, double* t, double* s, double* lam, double* z,
                        double* res_out) {
    const double b1 = prm->beta1, b2 = prm->beta2, tau = prm->tau;
    const double g1 = prm->gamma[0], g2 = prm->gamma[1], g3 = prm->gamma[2], g4 = prm->gamma[3];
    double* c = (double*)malloc(sizeof(double) * (size_t)(3 * m + 1));
    double* lold = (double*)malloc(sizeof(double) * (size_t)(4 * n + 1));
    if (!c || !lold) {
        free(c);
        free(lold);
        return -1;
    }
    int64_t nzero = 0;
    double dl = 0.0, dz = 0.0, dq = 0.0, dt = 0.0;
    (void)dst;
    /* (3a) p-block */
#pragma omp parallel for schedule(static) reduction(+ : nzero)
    for (int64_t i = 0; i < n; ++i) {
        double u[4];
        for (int k = 0; k < 4; ++k) u[k] = b1 * q[4 * i + k] + lam[4 * i + k] + g1 * p[4 * i + k];
        for (int64_t x = out_ptr[i]; x < out_ptr[i + 1]; ++x) {
            const int64_t e = out_eid[x], j = dst[e];
            double r[4], rc[4], tp[4], a[4], v[4];
            r[0] = 0.0;
            for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
            qconj(r, rc);
            qpure(&te[3 * e], tp);
            qmul(rc, &q[4 * i], a);
            qmul(a, tp, v);
            double w = 2.0 * (omega ? omega[e] : 1.0);
            for (int k = 0; k < 4; ++k) u[k] += w * v[k];
        }
        for (int64_t x = in_ptr[i]; x < in_ptr[i + 1]; ++x) {
            const int64_t e = in_eid[x], l = src[e];
            double v[4];
            qmul(&q[4 * l], &qe[4 * e], v);
            double w = 2.0 * (kappa ? kappa[e] : 1.0);
            for (int k = 0; k < 4; ++k) u[k] += w * v[k];
        }
        double nu = sqrt(dot4(u, u));
        if (nu > 0.0) {
            for (int k = 0; k < 4; ++k) p[4 * i + k] = u[k] / nu;
        } else {
            nzero++;
        }
    }
    /* (3b) q-block; the old lambda is kept for the residual */
#pragma omp parallel for schedule(static) reduction(+ : dq)
    for (int64_t i = 0; i < n; ++i) {
        double a2 = b1 + g2, qn[4];
        for (int k = 0; k < 4; ++k) qn[k] = b1 * p[4 * i + k] - lam[4 * i + k] + g2 * q[4 * i + k];
        for (int64_t x = out_ptr[i]; x < out_ptr[i + 1]; ++x) {
            const int64_t e = out_eid[x], j = dst[e];
            double w = omega ? omega[e] : 1.0, kk = kappa ? kappa[e] : 1.0;
            double r[4], tp[4], tc[4], a[4], v[4], qc[4], h[4];
            r[0] = 0.0;
            for (int k = 0; k < 3; ++k) r[k + 1] = t[3 * j + k] - s[3 * i + k];
            qpure(&te[3 * e], tp);
            qconj(tp, tc);
            qmul(r, &p[4 * i], a);
            qmul(a, tc, v);
            qconj(&qe[4 * e], qc);
            qmul(&p[4 * j], qc, h);
            double tn2 = dot4(tp, tp);
            a2 += 2.0 * (w * dot4(&p[4 * i], &p[4 * i]) * tn2 +
                         kk * dot4(&p[4 * j], &p[4 * j]) * dot4(&qe[4 * e], &qe[4 * e]));
            for (int k = 0; k < 4; ++k) qn[k] += 2.0 * (w * v[k] + kk * h[k]);
        }
        for (int k = 0; k < 4; ++k) {
            const double qk = qn[k] / a2, d = qk - q[4 * i + k];
            dq += d * d;
            q[4 * i + k] = qk;
            lold[4 * i + k] = lam[4 * i + k];
        }
    }
    /* c_e = Im(q_i^{k+1} t~_e (p_i^{k+1})^*) */
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < m; ++e) {
        int64_t i = src[e];
        double tp[4], a[4], pc[4], v[4];
        qpure(&te[3 * e], tp);
        qmul(&q[4 * i], tp, a);
        qconj(&p[4 * i], pc);
        qmul(a, pc, v);
        c[3 * e] = v[1]; c[3 * e + 1] = v[2]; c[3 * e + 2] = v[3];
    }
    /* (3c) t-block: a vertex reads only its own t here, so t is written in place */
#pragma omp parallel for schedule(static) reduction(+ : dt)
    for (int64_t i = 0; i < n; ++i) {
        double a3 = b2 + g3, tn[3];
        for (int k = 0; k < 3; ++k) tn[k] = b2 * s[3 * i + k] + z[3 * i + k] + g3 * t[3 * i + k];
        for (int64_t x = in_ptr[i]; x < in_ptr[i + 1]; ++x) {
            const int64_t e = in_eid[x], l = src[e];
            double w = omega ? omega[e] : 1.0;
            a3 += 2.0 * w;
            for (int k = 0; k < 3; ++k) tn[k] += 2.0 * w * (s[3 * l + k] + c[3 * e + k]);
        }
        for (int k = 0; k < 3; ++k) {
            const double tk = tn[k] / a3, d = tk - t[3 * i + k];
            dt += d * d;
            t[3 * i + k] = tk;
        }
    }
    /* (3d) s-block, then the relaxed duals (3e), (3f) of the same vertex */
#pragma omp parallel for schedule(static) reduction(+ : dl, dz)
    for (int64_t i = 0; i < n; ++i) {
        double a4 = b2 + g4, sn[3];
        for (int k = 0; k < 3; ++k) sn[k] = b2 * t[3 * i + k] - z[3 * i + k] + g4 * s[3 * i + k];
        for (int64_t x = out_ptr[i]; x < out_ptr[i + 1]; ++x) {
            const int64_t e = out_eid[x], j = dst[e];
            double w = omega ? omega[e] : 1.0;
            a4 += 2.0 * w;
            for (int k = 0; k < 3; ++k) sn[k] += 2.0 * w * (t[3 * j + k] - c[3 * e + k]);
        }
        for (int k = 0; k < 3; ++k) s[3 * i + k] = sn[k] / a4;
        for (int k = 0; k < 4; ++k) {
            lam[4 * i + k] -= tau * b1 * (p[4 * i + k] - q[4 * i + k]);
            const double d = lam[4 * i + k] - lold[4 * i + k];
            dl += d * d;
        }
        for (int k = 0; k < 3; ++k) {
            const double zo = z[3 * i + k];
            z[3 * i + k] -= tau * b2 * (t[3 * i + k] - s[3 * i + k]);
            const double d = z[3 * i + k] - zo;
            dz += d * d;
        }
    }
    if (res_out) {
        res_out[0] = dl / b1 + dz / b2 + b1 * dq + b2 * dt;
        res_out[1] = dl; res_out[2] = dz; res_out[3] = dq; res_out[4] = dt;
    }
    free(c);
    free(lold);
    return nzero;
}
#endif /* ORC_OPENMP */
