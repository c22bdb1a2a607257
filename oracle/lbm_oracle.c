/*
 * FP64 CPU oracle for the Cole-Hopf fourth-order MRT-LB method
 * (Chen, Liu, Chai & Shi, "A Cole-Hopf transformation based fourth-order
 * multiple-relaxation-time lattice Boltzmann model for the coupled Burgers'
 * equations", arXiv:2309.02825).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA library is checked against.  Only the tests, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, header, table or constant
 * with the CUDA library.
 *
 * Everything is IEEE double, built without fast-math and without FP
 * contraction.  The update is written the plain way: dense q x q matrices
 * built from the paper's definitions, one node at a time, collide then
 * stream (push), storing the pre-collision distribution f(x, t).
 *
 * Layout: node index = x0 + N0*(x1 + N1*(x2 + N2*x3)) (x0 fastest);
 * distributions f[i*nodes + node]; vector fields g[a*nodes + node].
 * The domain is periodic with nodes at x_a = j*dx, j = 0..N_a-1.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXD 4
#define ORC_MAXQ (1 + 2 * ORC_MAXD * ORC_MAXD)

/* ------------------------------------------------------------------ */
/* Lattice DdQ(1+2d^2): Eqs. (d1q3), (d2q9), (d3q19), (ddqq).          */
/* ------------------------------------------------------------------ */

int orc_q(int d) { return 1 + 2 * d * d; }

/*
 * Host threads.  The node loops below are split across OpenMP threads when
 * the library is built with OpenMP; each node's values are computed exactly
 * as in the serial loop and every sum over nodes is taken serially in node
 * order, so the results do not depend on the thread count.
 */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
int orc_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/*
 * Discrete velocities in lattice units e_i = c_i / c, written to
 * e[i*d + a].  Order: the rest velocity; +e_p for p = 1..d; -e_p for
 * p = 1..d (the Q_p block of Eq. (ddqq)); then, for each coordinate pair
 * (i < j) in lexicographic order, the four velocities whose (i, j)
 * components are (J1[k], J2[k]), k = 0..3, with J1 = (1,-1,-1,1) and
 * J2 = (1,1,-1,-1).  For d = 1, 2, 3 this reproduces the printed lists of
 * Eqs. (d1q3), (d2q9) and (d3q19) element for element.
 */
void orc_lattice(int d, int *e)
{
    static const int J1[4] = {1, -1, -1, 1};
    static const int J2[4] = {1, 1, -1, -1};
    int q = orc_q(d);
    memset(e, 0, sizeof(int) * (size_t)q * (size_t)d);
    int n = 1;
    for (int p = 0; p < d; ++p) e[(1 + p) * d + p] = 1;
    for (int p = 0; p < d; ++p) e[(1 + d + p) * d + p] = -1;
    n = 1 + 2 * d;
    for (int i = 0; i < d; ++i)
        for (int j = i + 1; j < d; ++j)
            for (int k = 0; k < 4; ++k) {
                e[n * d + i] = J1[k];
                e[n * d + j] = J2[k];
                ++n;
            }
}

/* product over a of e_a^{p_a} for one velocity */
static double mono(int d, const int *ei, const int *p)
{
    double v = 1.0;
    for (int a = 0; a < d; ++a)
        for (int k = 0; k < p[a]; ++k) v *= (double)ei[a];
    return v;
}

/*
 * Natural-moment transformation matrix M (Eqs. (d1q3)-(ddqq)) in lattice
 * units, row-major M[r*q + i].  Rows in order: 1; e_a (a = 1..d); e_a^2;
 * e_a e_b (a < b); e_a e_b^2 (a < b); e_a^2 e_b (a < b); e_a^2 e_b^2 (a < b).
 * Writing M with powers of e instead of c scales each row by a power of c;
 * since S is diagonal, M^-1 S M is unchanged.  The d = 3 print lists the
 * third-order rows pair by pair instead of family by family; they all
 * relax with rate 1, so the order is immaterial.
 * Also returns, in kind[r], the family of row r:
 * 0 conserved, 1 first order, 2 e_a^2, 3 e_a e_b, 4 third order, 5 fourth order.
 */
void orc_moment_matrix(int d, const int *e, double *M, int *kind)
{
    int q = orc_q(d);
    int r = 0;
    int p[ORC_MAXD];
#define ORC_ROW(KIND)                                              \
    do {                                                           \
        for (int i = 0; i < q; ++i) M[r * q + i] = mono(d, e + i * d, p); \
        kind[r] = (KIND);                                          \
        ++r;                                                       \
    } while (0)
    memset(p, 0, sizeof p);
    ORC_ROW(0);
    for (int a = 0; a < d; ++a) { memset(p, 0, sizeof p); p[a] = 1; ORC_ROW(1); }
    for (int a = 0; a < d; ++a) { memset(p, 0, sizeof p); p[a] = 2; ORC_ROW(2); }
    for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) { memset(p, 0, sizeof p); p[a] = 1; p[b] = 1; ORC_ROW(3); }
    for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) { memset(p, 0, sizeof p); p[a] = 1; p[b] = 2; ORC_ROW(4); }
    for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) { memset(p, 0, sizeof p); p[a] = 2; p[b] = 1; ORC_ROW(4); }
    for (int a = 0; a < d; ++a)
        for (int b = a + 1; b < d; ++b) { memset(p, 0, sizeof p); p[a] = 2; p[b] = 2; ORC_ROW(5); }
#undef ORC_ROW
}

/* Gauss-Jordan inverse with partial pivoting; returns 0 on success. */
int orc_invert(int n, const double *A, double *Ainv)
{
    double W[ORC_MAXQ * 2 * ORC_MAXQ];
    int w2 = 2 * n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < w2; ++j)
            W[i * w2 + j] = (j < n) ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
    for (int col = 0; col < n; ++col) {
        int piv = col;
        for (int i = col + 1; i < n; ++i)
            if (fabs(W[i * w2 + col]) > fabs(W[piv * w2 + col])) piv = i;
        if (fabs(W[piv * w2 + col]) < 1e-300) return -1;
        if (piv != col)
            for (int j = 0; j < w2; ++j) {
                double t = W[col * w2 + j];
                W[col * w2 + j] = W[piv * w2 + j];
                W[piv * w2 + j] = t;
            }
        double inv = 1.0 / W[col * w2 + col];
        for (int j = 0; j < w2; ++j) W[col * w2 + j] *= inv;
        for (int i = 0; i < n; ++i) {
            if (i == col) continue;
            double fac = W[i * w2 + col];
            if (fac == 0.0) continue;
            for (int j = 0; j < w2; ++j) W[i * w2 + j] -= fac * W[col * w2 + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * w2 + n + j];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Theorem 2, Eq. (Bur-Sol): the fourth-order relaxation set.          */
/* eps = nu*dt/dx^2.  For d = 1, s2x is s_2; for d > 1 it is s_21.     */
/* ------------------------------------------------------------------ */
void orc_paper_set(int d, double eps, double *s1, double *s2x, double *s22,
                   double *w1, double *wd)
{
    double a = 6.0 * eps + 1.0;
    *s1 = 2.0 / a;
    *s2x = 24.0 * eps / (a * a);
    if (d == 1) {
        *s22 = 1.0; /* no such moment for d = 1 */
        *w1 = 1.0 / 6.0;
        *wd = 0.0;
    } else {
        *s22 = 4.0 / (6.0 * eps + 3.0);
        *w1 = 1.0 / 6.0 - (d - 1) * eps / 3.0;
        *wd = eps / 6.0;
    }
}

/*
 * Weights of Eq. (d1-3-weight): w_0 = 1 - 2d w_1 - 2d(d-1) w_{1+2d}; the
 * 2d axis velocities carry w_1 and the 2d(d-1) diagonal ones w_{1+2d}.
 */
void orc_weights(int d, double w1, double wd, double *w)
{
    int q = orc_q(d);
    w[0] = 1.0 - 2.0 * d * w1 - 2.0 * d * (d - 1) * wd;
    for (int i = 1; i <= 2 * d; ++i) w[i] = w1;
    for (int i = 2 * d + 1; i < q; ++i) w[i] = wd;
}

/* ------------------------------------------------------------------ */
/* Model: lattice, M, M^-1, S, weights, and the two q x q operators.    */
/* ------------------------------------------------------------------ */
typedef struct {
    int d, q;
    long N[ORC_MAXD];
    long nodes;
    double nu, dx, dt, c, eps, cs2;
    double s0, s1, s2x, s22, w0, w1, wd;
    int e[ORC_MAXQ * ORC_MAXD];
    int kind[ORC_MAXQ];
    double M[ORC_MAXQ * ORC_MAXQ];
    double Minv[ORC_MAXQ * ORC_MAXQ];
    double sdiag[ORC_MAXQ];
    double w[ORC_MAXQ];
    double Ccol[ORC_MAXQ * ORC_MAXQ];  /* M^-1 S M       (collision, Eq. (distribution-f)) */
    double Cinv[ORC_MAXQ * ORC_MAXQ];  /* M^-1 S^-1 M    (Lambda^-1 of Eq. (f-expression)) */
} orc_model;

static void matmul(int n, const double *A, const double *B, double *C)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += A[i * n + k] * B[k * n + j];
            C[i * n + j] = s;
        }
}

/*
 * Build a model.  paper_set != 0: s1, s2x, s22, w1, wd from Eq. (Bur-Sol)
 * with eps = nu*dt/dx^2.  Otherwise rs = {s1, s2x, s22, w1, wd}.  s0 is
 * irrelevant (the conserved moment equals its equilibrium) and set to 1.
 * Returns NULL on invalid input.
 */
orc_model *orc_create(int d, const long *N, double nu, double dx, double dt,
                      int paper_set, const double *rs)
{
    if (d < 1 || d > ORC_MAXD || !(nu > 0) || !(dx > 0) || !(dt > 0)) return NULL;
    orc_model *m = (orc_model *)calloc(1, sizeof(orc_model));
    if (!m) return NULL;
    m->d = d;
    m->q = orc_q(d);
    m->nodes = 1;
    for (int a = 0; a < d; ++a) {
        if (N[a] < 1) { free(m); return NULL; }
        m->N[a] = N[a];
        m->nodes *= N[a];
    }
    m->nu = nu;
    m->dx = dx;
    m->dt = dt;
    m->c = dx / dt;
    m->eps = nu * dt / (dx * dx);
    if (paper_set) {
        orc_paper_set(d, m->eps, &m->s1, &m->s2x, &m->s22, &m->w1, &m->wd);
    } else {
        m->s1 = rs[0]; m->s2x = rs[1]; m->s22 = rs[2]; m->w1 = rs[3]; m->wd = rs[4];
        if (d == 1) m->wd = 0.0;
    }
    m->s0 = 1.0;
    orc_lattice(d, m->e);
    orc_moment_matrix(d, m->e, m->M, m->kind);
    if (orc_invert(m->q, m->M, m->Minv) != 0) { free(m); return NULL; }
    orc_weights(d, m->w1, m->wd, m->w);
    m->w0 = m->w[0];
    /* c_s^2 = [2 w_1 + 4(d-1) w_{1+2d}] c^2 (text after Eq. (conseved-moment)) */
    m->cs2 = (2.0 * m->w1 + 4.0 * (d - 1) * m->wd) * m->c * m->c;
    /* S = diag(s0, s1 I_d, s21 I_d, s22 I_{d(d-1)/2}, 1 ...): Eqs. (d1q3)-(ddqq) */
    for (int r = 0; r < m->q; ++r) {
        switch (m->kind[r]) {
        case 0: m->sdiag[r] = m->s0; break;
        case 1: m->sdiag[r] = m->s1; break;
        case 2: m->sdiag[r] = m->s2x; break;
        case 3: m->sdiag[r] = m->s22; break;
        default: m->sdiag[r] = 1.0; break;
        }
    }
    double SM[ORC_MAXQ * ORC_MAXQ], SinvM[ORC_MAXQ * ORC_MAXQ];
    int q = m->q;
    for (int r = 0; r < q; ++r)
        for (int i = 0; i < q; ++i) {
            SM[r * q + i] = m->sdiag[r] * m->M[r * q + i];
            SinvM[r * q + i] = m->M[r * q + i] / m->sdiag[r];
        }
    matmul(q, m->Minv, SM, m->Ccol);
    matmul(q, m->Minv, SinvM, m->Cinv);
    return m;
}

void orc_free(orc_model *m) { free(m); }

/* Accessors for the tests. */
void orc_get_params(const orc_model *m, double *out /* 12 */)
{
    out[0] = m->eps; out[1] = m->c; out[2] = m->cs2;
    out[3] = m->s0; out[4] = m->s1; out[5] = m->s2x; out[6] = m->s22;
    out[7] = m->w0; out[8] = m->w1; out[9] = m->wd;
    out[10] = (double)m->q; out[11] = (double)m->nodes;
}
void orc_get_matrices(const orc_model *m, double *M, double *Minv, double *sdiag,
                      double *w, double *Ccol, double *Cinv, int *e)
{
    int q = m->q;
    memcpy(M, m->M, sizeof(double) * q * q);
    memcpy(Minv, m->Minv, sizeof(double) * q * q);
    memcpy(sdiag, m->sdiag, sizeof(double) * q);
    memcpy(w, m->w, sizeof(double) * q);
    memcpy(Ccol, m->Ccol, sizeof(double) * q * q);
    memcpy(Cinv, m->Cinv, sizeof(double) * q * q);
    memcpy(e, m->e, sizeof(int) * q * m->d);
}

/* ------------------------------------------------------------------ */
/* Index helpers (periodic).                                            */
/* ------------------------------------------------------------------ */
static void node_coords(const orc_model *m, long node, long *x)
{
    for (int a = 0; a < m->d; ++a) {
        x[a] = node % m->N[a];
        node /= m->N[a];
    }
}
static long coords_node(const orc_model *m, const long *x)
{
    long node = 0;
    for (int a = m->d - 1; a >= 0; --a) {
        long v = x[a] % m->N[a];
        if (v < 0) v += m->N[a];
        node = node * m->N[a] + v;
    }
    return node;
}

/*
 * Fourth-order central difference of theta along axis a (periodic),
 * used when no analytic initial gradient is supplied:
 * (-t(x+2) + 8 t(x+1) - 8 t(x-1) + t(x-2)) / (12 dx).
 */
void orc_fd4_gradient(const orc_model *m, const double *theta, double *grad)
{
#pragma omp parallel for schedule(static)
    for (long n = 0; n < m->nodes; ++n) {
        long x[ORC_MAXD], y[ORC_MAXD];
        node_coords(m, n, x);
        for (int a = 0; a < m->d; ++a) {
            double acc = 0.0;
            static const int off[4] = {2, 1, -1, -2};
            static const double cof[4] = {-1.0, 8.0, -8.0, 1.0};
            for (int k = 0; k < 4; ++k) {
                memcpy(y, x, sizeof(long) * m->d);
                y[a] += off[k];
                acc += cof[k] * theta[coords_node(m, y)];
            }
            grad[a * m->nodes + n] = acc / (12.0 * m->dx);
        }
    }
}

/*
 * Initialisation with the first two terms of Eq. (f-feq-o5) (Sec. IV):
 *   f = f^eq - eta dx^2 Lambda^-1 Dbar f^eq,  eta dx^2 = dt,
 *   f^eq_i = w_i theta0 (Eq. (feq)),  Dbar = diag(c_i . grad),
 * with Lambda^-1 read as the velocity-space inverse collision matrix
 * M^-1 S^-1 M (the reading under which the first moment of f^ne carries
 * the factor 1/s1 stated below Eq. (f-feq-o5)).
 * grad0 == NULL: the fourth-order central difference above is used.
 * Output: pre-collision f(x, 0).
 */
void orc_initialize(const orc_model *m, const double *theta0, const double *grad0, double *f)
{
    int q = m->q, d = m->d;
    long nodes = m->nodes;
    double *gbuf = NULL;
    if (!grad0) {
        gbuf = (double *)malloc(sizeof(double) * d * nodes);
        orc_fd4_gradient(m, theta0, gbuf);
        grad0 = gbuf;
    }
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nodes; ++n) {
        double g[ORC_MAXQ];
        for (int k = 0; k < q; ++k) {
            double cdotgrad = 0.0;
            for (int a = 0; a < d; ++a) cdotgrad += m->c * m->e[k * d + a] * grad0[a * nodes + n];
            g[k] = m->w[k] * cdotgrad; /* [Dbar f^eq]_k = w_k (c_k . grad theta) */
        }
        for (int i = 0; i < q; ++i) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += m->Cinv[i * q + k] * g[k];
            f[i * nodes + n] = m->w[i] * theta0[n] - m->dt * s;
        }
    }
    free(gbuf);
}

/*
 * One time step of Eq. (distribution-f):
 *   f_i(x + c_i dt, t + dt) = f_i(x,t) - (M^-1 S M)_{ik} [f_k - f_k^eq](x,t),
 * with f^eq = w theta and theta = sum_i f_i (Eqs. (feq), (conseved-moment)).
 * Collide at every node, then push each post-collision value to the
 * neighbour x + e_i (periodic wrap).  f_in and f_out must not alias.
 */
void orc_step(const orc_model *m, const double *f_in, double *f_out)
{
    int q = m->q, d = m->d;
    long nodes = m->nodes;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nodes; ++n) {
        long x[ORC_MAXD], y[ORC_MAXD];
        double fl[ORC_MAXQ], fne[ORC_MAXQ];
        double theta = 0.0;
        for (int i = 0; i < q; ++i) {
            fl[i] = f_in[i * nodes + n];
            theta += fl[i];
        }
        for (int k = 0; k < q; ++k) fne[k] = fl[k] - m->w[k] * theta;
        node_coords(m, n, x);
        for (int i = 0; i < q; ++i) {
            double s = 0.0;
            for (int k = 0; k < q; ++k) s += m->Ccol[i * q + k] * fne[k];
            double fstar = fl[i] - s;
            for (int a = 0; a < d; ++a) y[a] = x[a] + m->e[i * d + a];
            f_out[i * nodes + coords_node(m, y)] = fstar;
        }
    }
}

/* nsteps time steps; f holds f(x,t) on entry and f(x, t + nsteps*dt) on exit. */
int orc_run(const orc_model *m, double *f, long nsteps)
{
    size_t bytes = sizeof(double) * (size_t)m->q * (size_t)m->nodes;
    double *tmp = (double *)malloc(bytes);
    if (!tmp) return -1;
    for (long s = 0; s < nsteps; ++s) {
        orc_step(m, f, tmp);
        memcpy(f, tmp, bytes);
    }
    free(tmp);
    return 0;
}

/*
 * Macroscopic recovery from the pre-collision f(x, t) (Sec. III.C):
 *   theta = sum_k f_k                                   (Eq. (conseved-moment))
 *   f^ne  = f - w theta
 *   grad theta = - s1 sum_k c_k f^ne_k / (dt c_s^2)     (Eq. (nabla-theta), with
 *                the division that the identity before it implies)
 *   u_a   = (2 - s1) sum_k c_ka f^ne_k / sum_k f_k      (Eq. (ui-compute))
 * grad and u may be NULL.
 */
void orc_recover(const orc_model *m, const double *f, double *theta, double *grad, double *u)
{
    int q = m->q, d = m->d;
    long nodes = m->nodes;
#pragma omp parallel for schedule(static)
    for (long n = 0; n < nodes; ++n) {
        double th = 0.0;
        for (int k = 0; k < q; ++k) th += f[k * nodes + n];
        if (theta) theta[n] = th;
        for (int a = 0; a < d; ++a) {
            double j = 0.0;
            for (int k = 0; k < q; ++k) {
                double fne = f[k * nodes + n] - m->w[k] * th;
                j += m->c * m->e[k * d + a] * fne;
            }
            if (grad) grad[a * nodes + n] = -m->s1 * j / (m->dt * m->cs2);
            if (u) u[a * nodes + n] = (2.0 - m->s1) * j / th;
        }
    }
}

/* Sum over all nodes and populations of f (= sum_x theta(x)). */
double orc_total(const orc_model *m, const double *f)
{
    double s = 0.0;
    long total = (long)m->q * m->nodes;
    for (long k = 0; k < total; ++k) s += f[k];
    return s;
}

/* ------------------------------------------------------------------ */
/* Discrete adjoint of the whole forward map (reference gradient).     */
/*                                                                     */
/* Forward: f_0 = Init(theta0, G theta0) (first two terms of Eq.       */
/* (f-feq-o5), G the fourth-order central difference), T steps of Eq.  */
/* (distribution-f), u from Eq. (ui-compute) at t = T dt, and          */
/* L = 1/2 sum_x sum_a (u_a - utarget_a)^2.  The adjoint runs the      */
/* same operations transposed, in reverse order, with every forward    */
/* state kept in memory (small grids only).  eps = nu dt / dx^2 enters */
/* through the relaxation set of Eq. (Bur-Sol); its derivatives are    */
/* those of the closed forms of Theorem 2.                             */
/* ------------------------------------------------------------------ */

/* d/d eps of the Eq. (Bur-Sol) quantities: s1, s2x, s22, w1, wd. */
static void paper_set_deriv(int d, double eps, double *ds1, double *ds2x, double *ds22, double *dw1,
                            double *dwd)
{
    double a = 6.0 * eps + 1.0;
    *ds1 = -12.0 / (a * a);
    *ds2x = 24.0 / (a * a) - 24.0 * eps * 12.0 / (a * a * a);
    if (d == 1) {
        *ds22 = 0.0;
        *dw1 = 0.0;
        *dwd = 0.0;
    } else {
        double b = 6.0 * eps + 3.0;
        *ds22 = -24.0 / (b * b);
        *dw1 = -(d - 1) / 3.0;
        *dwd = 1.0 / 6.0;
    }
}

/*
 * Compensated (Neumaier) summation: the running sum plus a correction that
 * collects the low-order bits each addition drops, so the error of a sum of
 * n terms stays near one rounding of the result instead of growing with n.
 * dL/deps sums T * nodes * q terms of both signs (about 5e9 at 512^2,
 * T = 2000), far too many for a plain running sum to hold 1e-12.
 */
typedef struct {
    double s, c;
} orc_ksum;
static void ksum_add(orc_ksum *k, double x)
{
    double t = k->s + x;
    if (fabs(k->s) >= fabs(x))
        k->c += (k->s - t) + x;
    else
        k->c += (x - t) + k->s;
    k->s = t;
}
static double ksum_value(const orc_ksum *k) { return k->s + k->c; }

/*
 * L and its gradients with respect to theta0 (nodes values) and eps, for
 *   L = 1/2 sum_x sum_a (u_a(x,T) - utarget_a(x))^2
 *       [+ 1/2 sum_x (theta(x,T) - ttarget(x))^2   when ttarget != NULL].
 * Requires a model built with the paper's relaxation set.
 * C = 0 keeps every forward state f_0..f_T in memory.  C > 0 keeps f_n only
 * at n = 0, C, 2C, ... and recomputes the states of one segment of C steps
 * at a time, by the same steps, as the reverse pass reaches it; the states,
 * and so the results, are the same bit for bit.
 * Every sum over nodes is taken serially in node order (per-node terms are
 * formed first, in parallel), so the results do not depend on the thread
 * count; L and dL/deps are compensated sums (orc_ksum).  Returns L, or NAN on
 * allocation failure or invalid C.
 */
double orc_adjoint(const orc_model *m, const double *theta0, const double *utarget, const double *ttarget,
                   long T, long C, double *dL_dtheta0, double *dL_deps)
{
    int q = m->q, d = m->d;
    long nodes = m->nodes;
    size_t fs = (size_t)q * (size_t)nodes;
    if (T < 0 || C < 0 || C > (T > 0 ? T : 1)) return NAN;
    /* kept states: all T + 1 (C = 0), or ceil(T/C) checkpoints, f_T and one segment */
    long nck = (C == 0) ? T + 1 : (T + C - 1) / C;
    size_t kept = (C == 0) ? (size_t)(T + 1) : (size_t)nck + 1 + (size_t)C;
    double *F = (double *)malloc(sizeof(double) * fs * kept);
    double *grad = (double *)malloc(sizeof(double) * d * nodes);
    double *phi = (double *)malloc(sizeof(double) * fs);
    double *phin = (double *)malloc(sizeof(double) * fs);
    double *h = (double *)malloc(sizeof(double) * d * nodes);
    double *terms = (double *)malloc(sizeof(double) * (size_t)nodes * (size_t)(q > d + 1 ? q : d + 1) * 2);
    if (!F || !grad || !phi || !phin || !h || !terms) {
        free(F); free(grad); free(phi); free(phin); free(h); free(terms);
        return NAN;
    }
    /* forward.  C = 0: F holds f_n at F + fs n.  C > 0: checkpoint k (f_kC)
     * at F + fs k, f_T at F + fs nck, the segment buffer after it. */
    orc_fd4_gradient(m, theta0, grad);
    orc_initialize(m, theta0, grad, F);
    double *fT;
    double *seg = NULL;
    if (C == 0) {
        for (long n = 0; n < T; ++n) orc_step(m, F + fs * n, F + fs * (n + 1));
        fT = F + fs * T;
    } else {
        fT = F + fs * nck;
        seg = fT + fs;
        memcpy(seg, F, sizeof(double) * fs);
        double *cur = seg, *nxt = seg + fs; /* two scratch states of the segment buffer (C >= 1: room for 1) */
        if (C == 1) nxt = fT;               /* C = 1: every state is a checkpoint; use f_T's slot as scratch */
        for (long n = 0; n < T; ++n) {
            orc_step(m, cur, nxt);
            double *t = cur;
            cur = nxt;
            nxt = t;
            if ((n + 1) % C == 0 && (n + 1) / C < nck) memcpy(F + fs * ((n + 1) / C), cur, sizeof(double) * fs);
        }
        if (cur != fT) memcpy(fT, cur, sizeof(double) * fs);
    }

    /* derivatives of the parameters with respect to eps */
    double ds1, ds2x, ds22, dw1, dwd;
    paper_set_deriv(d, m->eps, &ds1, &ds2x, &ds22, &dw1, &dwd);
    double dw[ORC_MAXQ], dS[ORC_MAXQ];
    dw[0] = -2.0 * d * dw1 - 2.0 * d * (d - 1) * dwd;
    for (int i = 1; i <= 2 * d; ++i) dw[i] = dw1;
    for (int i = 2 * d + 1; i < q; ++i) dw[i] = dwd;
    for (int r = 0; r < q; ++r) {
        switch (m->kind[r]) {
        case 1: dS[r] = ds1; break;
        case 2: dS[r] = ds2x; break;
        case 3: dS[r] = ds22; break;
        default: dS[r] = 0.0; break;
        }
    }
    /* K = I - C (I - w 1^T) with C = M^-1 S M; dK = -C'(I - w 1^T) + C w' 1^T */
    double K[ORC_MAXQ * ORC_MAXQ], dK[ORC_MAXQ * ORC_MAXQ], dC[ORC_MAXQ * ORC_MAXQ];
    double dSM[ORC_MAXQ * ORC_MAXQ], dCinv[ORC_MAXQ * ORC_MAXQ], dSinvM[ORC_MAXQ * ORC_MAXQ];
    for (int r = 0; r < q; ++r)
        for (int i = 0; i < q; ++i) {
            dSM[r * q + i] = dS[r] * m->M[r * q + i];
            dSinvM[r * q + i] = -dS[r] / (m->sdiag[r] * m->sdiag[r]) * m->M[r * q + i];
        }
    matmul(q, m->Minv, dSM, dC);
    matmul(q, m->Minv, dSinvM, dCinv);
    for (int i = 0; i < q; ++i)
        for (int j = 0; j < q; ++j) {
            double k = (i == j) ? 1.0 : 0.0, dk = 0.0;
            for (int l = 0; l < q; ++l) {
                double proj = ((l == j) ? 1.0 : 0.0) - m->w[l];
                k -= m->Ccol[i * q + l] * proj;
                dk -= dC[i * q + l] * proj;
                dk += m->Ccol[i * q + l] * dw[l];
            }
            K[i * q + j] = k;
            dK[i * q + j] = dk;
        }

    /* recovery at T and the seed phi_T = dL/df_T.  Per node x: the loss
     * terms of u_0..u_{d-1} (and theta) in terms[2(d+1)x + ...], their eps
     * terms after them; summed below in node order. */
    orc_ksum L = {0.0, 0.0}, deps = {0.0, 0.0};
    const int ns = d + 1;
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nodes; ++x) {
        double *tl = terms + (size_t)2 * ns * x, *te = tl + ns;
        double th = 0.0;
        for (int k = 0; k < q; ++k) th += fT[k * nodes + x];
        for (int k = 0; k < q; ++k) phi[k * nodes + x] = 0.0;
        for (int a = 0; a < d; ++a) {
            double j = 0.0, sew = 0.0, dsew = 0.0;
            for (int k = 0; k < q; ++k) {
                j += m->c * m->e[k * d + a] * (fT[k * nodes + x] - m->w[k] * th);
                sew += m->c * m->e[k * d + a] * m->w[k];
                dsew += m->c * m->e[k * d + a] * dw[k];
            }
            double u = (2.0 - m->s1) * j / th;
            double r = u - utarget[a * nodes + x];
            tl[a] = 0.5 * r * r;
            for (int k = 0; k < q; ++k) {
                double djdf = m->c * m->e[k * d + a] - sew;
                phi[k * nodes + x] += r * (2.0 - m->s1) * (djdf * th - j) / (th * th);
            }
            /* explicit eps dependence of u: through s1 and through w in f^ne */
            te[a] = r * (-ds1 * j / th + (2.0 - m->s1) * (-dsew * th) / th);
        }
        if (ttarget) {
            /* theta = sum_k f_k: d theta / d f_k = 1, no explicit eps dependence */
            double rt = th - ttarget[x];
            tl[d] = 0.5 * rt * rt;
            for (int k = 0; k < q; ++k) phi[k * nodes + x] += rt;
        }
    }
    for (long x = 0; x < nodes; ++x) {
        const double *tl = terms + (size_t)2 * ns * x, *te = tl + ns;
        for (int a = 0; a < d; ++a) {
            ksum_add(&L, tl[a]);
            ksum_add(&deps, te[a]);
        }
        if (ttarget) ksum_add(&L, tl[d]);
    }

    /* reverse steps: f_{n+1}(x + e_i)_i = (K f_n(x))_i */
    long curseg = -1;
    for (long n = T - 1; n >= 0; --n) {
        const double *fn;
        if (C == 0) {
            fn = F + fs * n;
        } else {
            long k = n / C;
            if (k != curseg) {
                /* recompute the states kC .. min(kC + C, T) - 1 from checkpoint k */
                long len = (k + 1) * C <= T ? C : T - k * C;
                memcpy(seg, F + fs * k, sizeof(double) * fs);
                for (long j = 1; j < len; ++j) orc_step(m, seg + fs * (j - 1), seg + fs * j);
                curseg = k;
            }
            fn = seg + fs * (n - k * C);
        }
#pragma omp parallel for schedule(static)
        for (long x = 0; x < nodes; ++x) {
            long xc[ORC_MAXD], yc[ORC_MAXD];
            double mu[ORC_MAXQ];
            double *tx = terms + (size_t)q * x;
            node_coords(m, x, xc);
            for (int i = 0; i < q; ++i) {
                for (int a = 0; a < d; ++a) yc[a] = xc[a] + m->e[i * d + a];
                mu[i] = phi[i * nodes + coords_node(m, yc)];
            }
            for (int j = 0; j < q; ++j) {
                double s = 0.0;
                for (int i = 0; i < q; ++i) s += K[i * q + j] * mu[i];
                phin[j * nodes + x] = s;
            }
            for (int i = 0; i < q; ++i) {
                double s = 0.0;
                for (int j = 0; j < q; ++j) s += dK[i * q + j] * fn[j * nodes + x];
                tx[i] = mu[i] * s;
            }
        }
        for (size_t k = 0; k < fs; ++k) ksum_add(&deps, terms[k]);
        double *t = phi;
        phi = phin;
        phin = t;
    }

    /* initialisation: f_0 = w theta0 - dt Cinv (w o (c e . g)), g = G theta0 */
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nodes; ++x) {
        double *tx = terms + (size_t)q * x;
        double s = 0.0;
        for (int i = 0; i < q; ++i) s += m->w[i] * phi[i * nodes + x];
        dL_dtheta0[x] = s;
        for (int a = 0; a < d; ++a) {
            double acc = 0.0;
            for (int i = 0; i < q; ++i) {
                double cw = 0.0;
                for (int k = 0; k < q; ++k) cw += m->Cinv[i * q + k] * m->w[k] * m->c * m->e[k * d + a];
                acc += phi[i * nodes + x] * cw;
            }
            h[a * nodes + x] = -m->dt * acc;
        }
        /* eps dependence of the initialisation */
        for (int i = 0; i < q; ++i) {
            double v = dw[i] * theta0[x];
            for (int k = 0; k < q; ++k) {
                double cg = 0.0;
                for (int a = 0; a < d; ++a) cg += m->c * m->e[k * d + a] * grad[a * nodes + x];
                v -= m->dt * (dCinv[i * q + k] * m->w[k] + m->Cinv[i * q + k] * dw[k]) * cg;
            }
            tx[i] = phi[i * nodes + x] * v;
        }
    }
    for (size_t k = 0; k < fs; ++k) ksum_add(&deps, terms[k]);
    /* transpose of the fourth-order difference: (G^T h)(x) = sum_k cof_k h(x - off_k e_a) / (12 dx) */
    static const int off[4] = {2, 1, -1, -2};
    static const double cof[4] = {-1.0, 8.0, -8.0, 1.0};
#pragma omp parallel for schedule(static)
    for (long x = 0; x < nodes; ++x) {
        long xc[ORC_MAXD], yc[ORC_MAXD];
        node_coords(m, x, xc);
        double s = 0.0;
        for (int a = 0; a < d; ++a)
            for (int k = 0; k < 4; ++k) {
                memcpy(yc, xc, sizeof(long) * d);
                yc[a] -= off[k];
                s += cof[k] * h[a * nodes + coords_node(m, yc)];
            }
        dL_dtheta0[x] += s / (12.0 * m->dx);
    }
    *dL_deps = ksum_value(&deps);
    free(F); free(grad); free(phi); free(phin); free(h); free(terms);
    return ksum_value(&L);
}

/* L only (the same forward as orc_adjoint), for finite-difference checks. */
double orc_loss(const orc_model *m, const double *theta0, const double *utarget, long T)
{
    size_t fs = (size_t)m->q * (size_t)m->nodes;
    double *f = (double *)malloc(sizeof(double) * fs);
    double *grad = (double *)malloc(sizeof(double) * m->d * m->nodes);
    double *u = (double *)malloc(sizeof(double) * m->d * m->nodes);
    if (!f || !grad || !u) {
        free(f); free(grad); free(u);
        return NAN;
    }
    orc_fd4_gradient(m, theta0, grad);
    orc_initialize(m, theta0, grad, f);
    orc_run(m, f, T);
    orc_recover(m, f, NULL, NULL, u);
    double L = 0.0;
    for (long k = 0; k < (long)m->d * m->nodes; ++k) {
        double r = u[k] - utarget[k];
        L += 0.5 * r * r;
    }
    free(f); free(grad); free(u);
    return L;
}
