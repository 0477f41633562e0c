/*
 * softsim oracle -- plain, slow, single-threaded FP64 reference of the
 * simulator's hot path.  TEST INFRASTRUCTURE ONLY: it exists to check the
 * CUDA library, and only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header or table with the CUDA
 * path.
 *
 * What it computes (Rojas, Sifakis, Kavan, "Differentiable Implicit
 * Soft-Body Physics", arXiv 2102.05791):
 *   - the potential energy E(x, a) of a triangle / tet mesh: neo-Hookean
 *     elasticity (Eq. neohookean-psi, Sec. 2; its 3D form uses I1 - 3), a
 *     per-element muscle term (k/2) a |F f|^2, gravity, and a one-sided
 *     ground penalty (Eq. energy-collision, Sec. 4.2, here with a free power);
 *   - its gradient, i.e. minus the force (Eq. f-as-grad, Sec. 3);
 *   - the Hessian-vector product that the paper obtains by back-propagating
 *     <f, v> (Eq. matrix-free-dfdx, Sec. 3.1), written out analytically;
 *   - the parameter VJP -lambda^T d2E/dx da (Eq. dLda-re-ordered, Sec. 3);
 *   - the backward-Euler incremental potential (Eq. opt-be, Sec. 4), with
 *     the optional ground friction k_f |v_horizontal|^2 ReLU(eps - y0) of
 *     Sec. 4.2 evaluated at v = (x - x0)/h;
 *   - the energy minimisation of Eq. x1-quasistatic-argmin by Newton-CG with
 *     backtracking, and a CG solve for the adjoint system (Sec. 3).
 *
 * Readings where the paper is silent: the quadratic stand-in for log J is
 * the second-order Taylor polynomial q(J) = (J-1) - (J-1)^2/2 (Sec. 2 names
 * a quadratic approximation without giving it).  Two muscle models, both
 * integrated over the element like Psi: the contractile term (k/2) a |F f|^2,
 * and the paper's active spring (Eq. active-spring-potential) with the
 * fiber's stretch |F f| = l / l0 (f a unit rest fiber), (k/2)(|F f|/a - 1)^2.
 *
 * Everything is a direct element loop with "+=" into vertex arrays.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int d;                      /* 2 or 3 */
    long nv, ne;
    const int *T;               /* [ne][d+1] */
    const double *Dminv;        /* [ne][d][d] inverse rest edge matrix */
    const double *W;            /* [ne] rest area / volume */
    const double *fiber;        /* [ne][d] unit fiber */
    const double *mass;         /* [nv] lumped mass (may be NULL: no gravity/inertia) */
    const unsigned char *fixed; /* [nv] or NULL: no Dirichlet mask */
    double mu, lam, k_muscle, gravity, k_contact;
    int contact_power;          /* 2 or 3 */
    int log_mode;               /* 0 exact log J, 1 quadratic q(J) */
    double h;                   /* time step; 0 = quasistatic */
    const double *xhat;         /* [nv][d] inertial target x0 + h v0 (dynamics only) */
    int muscle_model;           /* 0: contractile (k/2) a |F f|^2; 1: active spring (k/2)(|F f|/a - 1)^2 */
    double k_friction;          /* ground friction stiffness (dynamics only; 0 = off) */
    double eps_friction;        /* contact tolerance of the friction weight */
    const double *x0;           /* [nv][d] previous positions (dynamics only) */
} or_model;

typedef struct {
    int newton_iters, cg_iters_total, ls_halvings, status;
    double res0, res_final, min_J;
} or_stats;

enum { OR_OK = 0, OR_EINVERTED = -3, OR_ENOTCONVERGED = -4, OR_ELINESEARCH = -5 };

/* ---------------------------------------------------------------- small dense */

static double det_d(int d, const double A[3][3])
{
    if (d == 2) return A[0][0] * A[1][1] - A[0][1] * A[1][0];
    return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
         - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
         + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

/* 2 x 2 minor of A without row i and column j (3 x 3 A). */
static double minor3(const double A[3][3], int i, int j)
{
    int r0 = i == 0 ? 1 : 0, r1 = i == 2 ? 1 : 2;
    int c0 = j == 0 ? 1 : 0, c1 = j == 2 ? 1 : 2;
    return A[r0][c0] * A[r1][c1] - A[r0][c1] * A[r1][c0];
}

/* Directional derivative of minor3 along dA (product rule on the 2 x 2 det). */
static double dminor3(const double A[3][3], const double dA[3][3], int i, int j)
{
    int r0 = i == 0 ? 1 : 0, r1 = i == 2 ? 1 : 2;
    int c0 = j == 0 ? 1 : 0, c1 = j == 2 ? 1 : 2;
    return dA[r0][c0] * A[r1][c1] + A[r0][c0] * dA[r1][c1] - dA[r0][c1] * A[r1][c0] - A[r0][c1] * dA[r1][c0];
}

/* Cofactor matrix cof(A)_ij = (-1)^(i+j) M_ij (signed minors), so that
 * d det(A) / dA = cof(A) and A^-T = cof(A)/det A. */
static void cof_d(int d, const double A[3][3], double C[3][3])
{
    memset(C, 0, sizeof(double) * 9);
    if (d == 2) {
        C[0][0] = A[1][1];  C[0][1] = -A[1][0];
        C[1][0] = -A[0][1]; C[1][1] = A[0][0];
        return;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[i][j] = ((i + j) % 2 ? -1.0 : 1.0) * minor3(A, i, j);
}

/* Directional derivative of cof(A) along dA. */
static void dcof_d(int d, const double A[3][3], const double dA[3][3], double dC[3][3])
{
    memset(dC, 0, sizeof(double) * 9);
    if (d == 2) {
        dC[0][0] = dA[1][1];  dC[0][1] = -dA[1][0];
        dC[1][0] = -dA[0][1]; dC[1][1] = dA[0][0];
        return;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) dC[i][j] = ((i + j) % 2 ? -1.0 : 1.0) * dminor3(A, dA, i, j);
}

static void inv_d(int d, const double A[3][3], double Ai[3][3])
{
    double C[3][3];
    cof_d(d, A, C);
    double det = det_d(d, A);
    memset(Ai, 0, sizeof(double) * 9);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Ai[i][j] = C[j][i] / det; /* A^-1 = cof(A)^T / det */
}

static void mul_d(int d, const double A[3][3], const double B[3][3], double C[3][3])
{
    double R[3][3] = {{0}};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
            for (int k = 0; k < d; ++k) R[i][j] += A[i][k] * B[k][j];
    memcpy(C, R, sizeof(R));
}

static void transpose_d(int d, const double A[3][3], double B[3][3])
{
    double R[3][3] = {{0}};
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) R[i][j] = A[j][i];
    memcpy(B, R, sizeof(R));
}

static double ddot_d(int d, const double A[3][3], const double B[3][3])
{
    double s = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) s += A[i][j] * B[i][j];
    return s;
}

static void load_Dminv(const or_model *M, long e, double B[3][3])
{
    int d = M->d;
    memset(B, 0, sizeof(double) * 9);
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) B[i][j] = M->Dminv[(e * d + i) * d + j];
}

/* Edge matrix [y_1 - y_0, ..., y_d - y_0] of element e for a vertex field y. */
static void edge_matrix(const or_model *M, long e, const double *y, double D[3][3])
{
    int d = M->d;
    const int *t = M->T + e * (d + 1);
    memset(D, 0, sizeof(double) * 9);
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) D[i][j] = y[(long)t[j + 1] * d + i] - y[(long)t[0] * d + i];
}

/* Scatter the d x d matrix G = dE_e/dDs into vertex vector out:
 * column j goes to vertex j+1 and minus the sum of the columns to vertex 0. */
static void scatter(const or_model *M, long e, const double G[3][3], double *out)
{
    int d = M->d;
    const int *t = M->T + e * (d + 1);
    for (int j = 0; j < d; ++j)
        for (int i = 0; i < d; ++i) {
            out[(long)t[j + 1] * d + i] += G[i][j];
            out[(long)t[0] * d + i] -= G[i][j];
        }
}

/* ---------------------------------------------------------------- rest data */

/* Dm^-1 and W = det(Dm)/d! per element.  Returns OR_EINVERTED if an element
 * has det(Dm) <= 0. */
int or_rest(int d, long nv, long ne, const double *X, const int *T, double *Dminv, double *W)
{
    (void)nv;
    or_model M;
    memset(&M, 0, sizeof(M));
    M.d = d; M.ne = ne; M.T = T;
    for (long e = 0; e < ne; ++e) {
        double Dm[3][3], Bi[3][3];
        edge_matrix(&M, e, X, Dm);
        double det = det_d(d, Dm);
        if (!(det > 0.0)) return OR_EINVERTED;
        inv_d(d, Dm, Bi);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) Dminv[(e * d + i) * d + j] = Bi[i][j];
        W[e] = det / (d == 2 ? 2.0 : 6.0);
    }
    return OR_OK;
}

/* Lumped mass: each element gives rho * W / (d+1) to each of its vertices. */
void or_mass(int d, long nv, long ne, const int *T, const double *W, double rho, double *m)
{
    for (long i = 0; i < nv; ++i) m[i] = 0.0;
    for (long e = 0; e < ne; ++e)
        for (int k = 0; k <= d; ++k) m[T[e * (d + 1) + k]] += rho * W[e] / (d + 1);
}

/* ---------------------------------------------------------------- muscle */

/* Muscle energy density of one element as a function of q = F f. */
static double muscle_psi(const or_model *M, double a, const double *q)
{
    int d = M->d;
    double q2 = 0.0;
    for (int i = 0; i < d; ++i) q2 += q[i] * q[i];
    if (M->muscle_model == 0) return 0.5 * M->k_muscle * a * q2;
    double r = sqrt(q2) / a - 1.0;
    return 0.5 * M->k_muscle * r * r;
}

/* d psi / d q. */
static void muscle_dpsi(const or_model *M, double a, const double *q, double *out)
{
    int d = M->d;
    if (M->muscle_model == 0) {
        for (int i = 0; i < d; ++i) out[i] = M->k_muscle * a * q[i];
        return;
    }
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += q[i] * q[i];
    s = sqrt(s);
    double r = s / a - 1.0;
    /* k r dr/dq, dr/dq = q / (a s) */
    for (int i = 0; i < d; ++i) out[i] = M->k_muscle * r * q[i] / (a * s);
}

/* (d^2 psi / dq^2) dq: the spring's Hessian is k/(a^2 s^2) q q^T (the
 * squared slope of r) plus k r times the Hessian of s/a,
 * (I/s - q q^T/s^3)/a. */
static void muscle_d2psi(const or_model *M, double a, const double *q, const double *dq, double *out)
{
    int d = M->d;
    if (M->muscle_model == 0) {
        for (int i = 0; i < d; ++i) out[i] = M->k_muscle * a * dq[i];
        return;
    }
    double s2 = 0.0, qdq = 0.0;
    for (int i = 0; i < d; ++i) {
        s2 += q[i] * q[i];
        qdq += q[i] * dq[i];
    }
    double s = sqrt(s2);
    double r = s / a - 1.0;
    double k = M->k_muscle;
    for (int i = 0; i < d; ++i)
        out[i] = k / (a * a * s2) * qdq * q[i] + k * r / a * (dq[i] / s - qdq * q[i] / (s2 * s));
}

/* d^2 psi / dq da. */
static void muscle_dpsi_da(const or_model *M, double a, const double *q, double *out)
{
    int d = M->d;
    if (M->muscle_model == 0) {
        for (int i = 0; i < d; ++i) out[i] = M->k_muscle * q[i];
        return;
    }
    double s = 0.0;
    for (int i = 0; i < d; ++i) s += q[i] * q[i];
    s = sqrt(s);
    /* d/da of k (s/a - 1) q / (a s) = k q / s * d/da (s/a^2 - 1/a) */
    for (int i = 0; i < d; ++i) out[i] = M->k_muscle * q[i] / s * (-2.0 * s / (a * a * a) + 1.0 / (a * a));
}

/* ---------------------------------------------------------------- energy */

/* Ground friction (Sec. 4.2, Eq. energy-friction): with the velocity
 * v(x) = (x - x0)/h of backward Euler (Eq. v-of-x-vec), each vertex adds
 * k_f |v_horizontal(x)|^2 ReLU(eps - y0), horizontal meaning every axis but
 * y (x in 2D; x and z in 3D).  Weight of vertex i: */
static double friction_w(const or_model *M, long i)
{
    if (!(M->h > 0.0) || !M->x0 || M->k_friction == 0.0) return 0.0;
    double r = M->eps_friction - M->x0[i * M->d + 1];
    return r > 0.0 ? M->k_friction * r : 0.0;
}

/* Per-vertex ground penalty k_c * max(0, -y)^p and its first two derivatives. */
static double contact_e(const or_model *M, double y)
{
    double pen = y < 0.0 ? -y : 0.0;
    return M->k_contact * pow(pen, M->contact_power);
}
static double contact_de(const or_model *M, double y)
{
    double pen = y < 0.0 ? -y : 0.0;
    if (pen == 0.0) return 0.0;
    return -M->contact_power * M->k_contact * pow(pen, M->contact_power - 1);
}
static double contact_d2e(const or_model *M, double y)
{
    double pen = y < 0.0 ? -y : 0.0;
    if (pen == 0.0) return 0.0;
    int p = M->contact_power;
    return p * (p - 1) * M->k_contact * pow(pen, p - 2);
}

/* Potential energy E(x, a) (quasistatic) or the incremental potential
 * 1/2 |x - xhat|_M^2 + h^2 E(x, a) (h > 0).  Returns +inf if an element has
 * J <= 0 under the exact log.  *abs_sum receives the sum of the magnitudes of
 * all the terms added (a scale for the round-off of the total). */
double or_energy(const or_model *M, const double *x, const double *a, double *abs_sum,
                 double *min_J)
{
    int d = M->d;
    double E = 0.0, S = 0.0, mj = INFINITY;
    for (long e = 0; e < M->ne; ++e) {
        double Ds[3][3], B[3][3], F[3][3];
        edge_matrix(M, e, x, Ds);
        load_Dminv(M, e, B);
        mul_d(d, Ds, B, F);
        double J = det_d(d, F);
        if (J < mj) mj = J;
        double I1 = ddot_d(d, F, F);
        double l;
        if (M->log_mode == 0) {
            if (!(J > 0.0)) {
                if (abs_sum) *abs_sum = INFINITY;
                if (min_J) *min_J = mj;
                return INFINITY;
            }
            l = log(J);
        } else {
            l = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
        }
        double psi = 0.5 * M->mu * (I1 - d) - M->mu * l + 0.5 * M->lam * l * l;
        const double *f = M->fiber + e * d;
        double q[3] = {0, 0, 0};
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) q[i] += F[i][j] * f[j];
        double psim = muscle_psi(M, a[e], q);
        double w = M->W[e] * (psi + psim);
        E += w;
        S += fabs(w);
    }
    for (long i = 0; i < M->nv; ++i) {
        double y = x[i * d + 1];
        double m = M->mass ? M->mass[i] : 0.0;
        double t = m * M->gravity * y + contact_e(M, y);
        double w = friction_w(M, i);
        if (w != 0.0)
            for (int c = 0; c < d; ++c) {
                if (c == 1) continue;
                double vc = (x[i * d + c] - M->x0[i * d + c]) / M->h;
                t += w * vc * vc;
            }
        E += t;
        S += fabs(t);
    }
    if (M->h > 0.0) {
        double h2 = M->h * M->h, I = 0.0;
        for (long i = 0; i < M->nv; ++i)
            for (int c = 0; c < d; ++c) {
                double r = x[i * d + c] - M->xhat[i * d + c];
                I += 0.5 * M->mass[i] * r * r;
            }
        E = I + h2 * E;
        S = I + h2 * S;
    }
    if (abs_sum) *abs_sum = S;
    if (min_J) *min_J = mj;
    return E;
}

/* ---------------------------------------------------------------- gradient */

/* First Piola-Kirchhoff stress of the elastic part. */
static void pk1(const or_model *M, const double F[3][3], double P[3][3])
{
    int d = M->d;
    double J = det_d(d, F);
    memset(P, 0, sizeof(double) * 9);
    if (M->log_mode == 0) {
        /* P = mu (F - F^-T) + lambda log(J) F^-T */
        double Fi[3][3], FiT[3][3];
        inv_d(d, F, Fi);
        transpose_d(d, Fi, FiT);
        double l = log(J);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) P[i][j] = M->mu * (F[i][j] - FiT[i][j]) + M->lam * l * FiT[i][j];
    } else {
        /* Psi = mu/2 (I1 - d) - mu q + lambda/2 q^2, dJ/dF = cof(F):
         * P = mu F + (lambda q - mu) q' cof(F) */
        double C[3][3];
        cof_d(d, F, C);
        double q = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
        double qp = 1.0 - (J - 1.0);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) P[i][j] = M->mu * F[i][j] + (M->lam * q - M->mu) * qp * C[i][j];
    }
}

/* Gradient of or_energy w.r.t. x (= -force).  Entries of pinned vertices are
 * zeroed when M->fixed is given.  If abs_scale is non-NULL it receives, per
 * entry, the sum of the magnitudes of the element contributions (a scale for
 * cancellation in the vertex sums). */
void or_grad(const or_model *M, const double *x, const double *a, double *g, double *abs_scale)
{
    int d = M->d;
    long n = M->nv * d;
    for (long i = 0; i < n; ++i) g[i] = 0.0;
    if (abs_scale)
        for (long i = 0; i < n; ++i) abs_scale[i] = 0.0;
    for (long e = 0; e < M->ne; ++e) {
        double Ds[3][3], B[3][3], F[3][3], P[3][3], BT[3][3], G[3][3];
        edge_matrix(M, e, x, Ds);
        load_Dminv(M, e, B);
        mul_d(d, Ds, B, F);
        pk1(M, F, P);
        const double *f = M->fiber + e * d;
        double Ff[3] = {0, 0, 0}, dpsi[3];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) Ff[i] += F[i][j] * f[j];
        muscle_dpsi(M, a[e], Ff, dpsi);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) P[i][j] += dpsi[i] * f[j];
        transpose_d(d, B, BT);
        mul_d(d, P, BT, G);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) G[i][j] *= M->W[e];
        scatter(M, e, G, g);
        if (abs_scale) {
            const int *t = M->T + e * (d + 1);
            for (int i = 0; i < d; ++i) {
                double s0 = 0.0;
                for (int j = 0; j < d; ++j) {
                    abs_scale[(long)t[j + 1] * d + i] += fabs(G[i][j]);
                    s0 += G[i][j];
                }
                abs_scale[(long)t[0] * d + i] += fabs(s0);
            }
        }
    }
    for (long i = 0; i < M->nv; ++i) {
        double y = x[i * d + 1];
        double m = M->mass ? M->mass[i] : 0.0;
        g[i * d + 1] += m * M->gravity + contact_de(M, y);
        if (abs_scale) abs_scale[i * d + 1] += fabs(m * M->gravity) + fabs(contact_de(M, y));
        double w = friction_w(M, i);
        if (w != 0.0)
            for (int c = 0; c < d; ++c) {
                if (c == 1) continue;
                double gf = 2.0 * w * (x[i * d + c] - M->x0[i * d + c]) / (M->h * M->h);
                g[i * d + c] += gf;
                if (abs_scale) abs_scale[i * d + c] += fabs(gf);
            }
    }
    if (M->h > 0.0) {
        double h2 = M->h * M->h;
        for (long i = 0; i < M->nv; ++i)
            for (int c = 0; c < d; ++c) {
                long k = i * d + c;
                double in = M->mass[i] * (x[k] - M->xhat[k]);
                g[k] = in + h2 * g[k];
                if (abs_scale) abs_scale[k] = fabs(in) + h2 * abs_scale[k];
            }
    }
    if (M->fixed)
        for (long i = 0; i < M->nv; ++i)
            if (M->fixed[i])
                for (int c = 0; c < d; ++c) g[i * d + c] = 0.0;
}

/* ---------------------------------------------------------------- HVP */

/* Differential of the elastic P along dF. */
static void dpk1(const or_model *M, const double F[3][3], const double dF[3][3], double dP[3][3])
{
    int d = M->d;
    double J = det_d(d, F);
    memset(dP, 0, sizeof(double) * 9);
    if (M->log_mode == 0) {
        /* dP = mu dF + (mu - lambda log J) F^-T dF^T F^-T + lambda tr(F^-1 dF) F^-T */
        double Fi[3][3], FiT[3][3], dFT[3][3], T1[3][3], T2[3][3], FidF[3][3];
        inv_d(d, F, Fi);
        transpose_d(d, Fi, FiT);
        transpose_d(d, dF, dFT);
        mul_d(d, FiT, dFT, T1);
        mul_d(d, T1, FiT, T2);
        mul_d(d, Fi, dF, FidF);
        double tr = 0.0;
        for (int i = 0; i < d; ++i) tr += FidF[i][i];
        double l = log(J);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                dP[i][j] = M->mu * dF[i][j] + (M->mu - M->lam * l) * T2[i][j] + M->lam * tr * FiT[i][j];
    } else {
        /* P = mu F + c(J) cof(F), c = (lambda q - mu) q'
         * dP = mu dF + c'(J) (cof(F):dF) cof(F) + c(J) dcof(F)[dF] */
        double C[3][3], dC[3][3];
        cof_d(d, F, C);
        dcof_d(d, F, dF, dC);
        double q = (J - 1.0) - 0.5 * (J - 1.0) * (J - 1.0);
        double qp = 1.0 - (J - 1.0);
        double qpp = -1.0;
        double c = (M->lam * q - M->mu) * qp;
        double cp = M->lam * qp * qp + (M->lam * q - M->mu) * qpp;
        double dJ = ddot_d(d, C, dF);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) dP[i][j] = M->mu * dF[i][j] + cp * dJ * C[i][j] + c * dC[i][j];
    }
}

/* Hv = (d^2 g / dx^2) v, with the same masking as or_grad (pinned rows and
 * pinned entries of v both dropped, i.e. the Hessian of the constrained
 * problem restricted to free entries). */
void or_hvp(const or_model *M, const double *x, const double *a, const double *v, double *Hv)
{
    int d = M->d;
    long n = M->nv * d;
    double *vm = NULL;
    if (M->fixed) {
        vm = (double *)malloc(sizeof(double) * n);
        for (long i = 0; i < M->nv; ++i)
            for (int c = 0; c < d; ++c) vm[i * d + c] = M->fixed[i] ? 0.0 : v[i * d + c];
        v = vm;
    }
    for (long i = 0; i < n; ++i) Hv[i] = 0.0;
    for (long e = 0; e < M->ne; ++e) {
        double Ds[3][3], dDs[3][3], B[3][3], F[3][3], dF[3][3], dP[3][3], BT[3][3], G[3][3];
        edge_matrix(M, e, x, Ds);
        edge_matrix(M, e, v, dDs);
        load_Dminv(M, e, B);
        mul_d(d, Ds, B, F);
        mul_d(d, dDs, B, dF);
        dpk1(M, F, dF, dP);
        const double *f = M->fiber + e * d;
        double Ff[3] = {0, 0, 0}, dFf[3] = {0, 0, 0}, d2[3];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                Ff[i] += F[i][j] * f[j];
                dFf[i] += dF[i][j] * f[j];
            }
        muscle_d2psi(M, a[e], Ff, dFf, d2);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) dP[i][j] += d2[i] * f[j];
        transpose_d(d, B, BT);
        mul_d(d, dP, BT, G);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) G[i][j] *= M->W[e];
        scatter(M, e, G, Hv);
    }
    for (long i = 0; i < M->nv; ++i) {
        Hv[i * d + 1] += contact_d2e(M, x[i * d + 1]) * v[i * d + 1];
        double w = friction_w(M, i);
        if (w != 0.0)
            for (int c = 0; c < d; ++c)
                if (c != 1) Hv[i * d + c] += 2.0 * w / (M->h * M->h) * v[i * d + c];
    }
    if (M->h > 0.0) {
        double h2 = M->h * M->h;
        for (long i = 0; i < M->nv; ++i)
            for (int c = 0; c < d; ++c) Hv[i * d + c] = M->mass[i] * v[i * d + c] + h2 * Hv[i * d + c];
    }
    if (M->fixed)
        for (long i = 0; i < M->nv; ++i)
            if (M->fixed[i])
                for (int c = 0; c < d; ++c) Hv[i * d + c] = 0.0;
    free(vm);
}

/* ---------------------------------------------------------------- param VJP */

/* dL/da_e = -lambda^T d(grad E)/da_e = -s W_e (d^2 psi/dq da) . (dF(lambda) f)
 * with q = F f (for the contractile term k (F f) . (dF(lambda) f)), where
 * s = h^2 for the incremental potential and 1 otherwise (Eq. dLda-re-ordered
 * with the muscle term as the only a-dependent energy). */
void or_param_vjp(const or_model *M, const double *x, const double *a, const double *lam, double *dLda)
{
    int d = M->d;
    double s = M->h > 0.0 ? M->h * M->h : 1.0;
    for (long e = 0; e < M->ne; ++e) {
        double Ds[3][3], dDs[3][3], B[3][3], F[3][3], dF[3][3];
        edge_matrix(M, e, x, Ds);
        edge_matrix(M, e, lam, dDs);
        load_Dminv(M, e, B);
        mul_d(d, Ds, B, F);
        mul_d(d, dDs, B, dF);
        const double *f = M->fiber + e * d;
        double Ff[3] = {0, 0, 0}, dFf[3] = {0, 0, 0}, mix[3];
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                Ff[i] += F[i][j] * f[j];
                dFf[i] += dF[i][j] * f[j];
            }
        muscle_dpsi_da(M, a[e], Ff, mix);
        double dot = 0.0;
        for (int i = 0; i < d; ++i) dot += mix[i] * dFf[i];
        dLda[e] = -s * M->W[e] * dot;
    }
}

/* ---------------------------------------------------------------- material VJP */

/* dL/dtheta_e = -s lambda^T d(grad E)/dtheta_e for theta = mu, lambda and the
 * muscle stiffness k of element e (Eq. dLda-re-ordered with theta in place
 * of a).  P is linear in (mu, lambda) and the muscle force linear in k, so
 * each derivative of P is P itself evaluated with that parameter set to 1
 * and the others to 0.  Any output may be NULL. */
void or_material_vjp(const or_model *M, const double *x, const double *a, const double *lam, double *dmu,
                     double *dlam, double *dk)
{
    int d = M->d;
    double s = M->h > 0.0 ? M->h * M->h : 1.0;
    or_model Mmu = *M, Mlam = *M, Mk = *M;
    Mmu.mu = 1.0;
    Mmu.lam = 0.0;
    Mlam.mu = 0.0;
    Mlam.lam = 1.0;
    Mk.k_muscle = 1.0;
    for (long e = 0; e < M->ne; ++e) {
        double Ds[3][3], dDs[3][3], B[3][3], F[3][3], dF[3][3], P[3][3];
        edge_matrix(M, e, x, Ds);
        edge_matrix(M, e, lam, dDs);
        load_Dminv(M, e, B);
        mul_d(d, Ds, B, F);
        mul_d(d, dDs, B, dF);
        if (dmu) {
            pk1(&Mmu, F, P);
            dmu[e] = -s * M->W[e] * ddot_d(d, P, dF);
        }
        if (dlam) {
            pk1(&Mlam, F, P);
            dlam[e] = -s * M->W[e] * ddot_d(d, P, dF);
        }
        if (dk) {
            const double *f = M->fiber + e * d;
            double q[3] = {0, 0, 0}, dq[3] = {0, 0, 0}, dpsi[3], t = 0.0;
            for (int i = 0; i < d; ++i)
                for (int j = 0; j < d; ++j) {
                    q[i] += F[i][j] * f[j];
                    dq[i] += dF[i][j] * f[j];
                }
            muscle_dpsi(&Mk, a[e], q, dpsi);
            for (int i = 0; i < d; ++i) t += dpsi[i] * dq[i];
            dk[e] = -s * M->W[e] * t;
        }
    }
}

/* ---------------------------------------------------------------- solvers */

static double vdot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

/* Conjugate gradients for H(x) sol = b, starting from sol = 0, stopped when
 * |r| <= rtol |b|, after max_iter iterations, or at non-positive curvature
 * (then sol keeps the last iterate, or the first search direction if that
 * happens on the first iteration).  Returns the iteration count. */
int or_cg(const or_model *M, const double *x, const double *a, const double *b, double *sol,
          double rtol, int max_iter, int *neg_curv)
{
    long n = M->nv * M->d;
    double *r = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    double *Ap = (double *)malloc(sizeof(double) * n);
    for (long i = 0; i < n; ++i) {
        sol[i] = 0.0;
        r[i] = b[i];
        p[i] = b[i];
    }
    double rr = vdot(n, r, r);
    double tol = rtol * sqrt(rr);
    int k = 0;
    if (neg_curv) *neg_curv = 0;
    for (; k < max_iter; ++k) {
        if (sqrt(rr) <= tol) break;
        or_hvp(M, x, a, p, Ap);
        double pAp = vdot(n, p, Ap);
        if (!(pAp > 0.0)) {
            if (neg_curv) *neg_curv = 1;
            if (k == 0)
                for (long i = 0; i < n; ++i) sol[i] = p[i];
            break;
        }
        double alpha = rr / pAp;
        for (long i = 0; i < n; ++i) {
            sol[i] += alpha * p[i];
            r[i] -= alpha * Ap[i];
        }
        double rr_new = vdot(n, r, r);
        double beta = rr_new / rr;
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
        rr = rr_new;
    }
    free(r);
    free(p);
    free(Ap);
    return k;
}

/* Newton-CG minimisation of or_energy from the initial x (overwritten with the
 * result).  Each step solves H d = -g by CG to the forcing tolerance
 * eta = min(0.5, sqrt(|g|/|g0|)) (falling back to -g when CG does not give a
 * descent direction), then backtracks t = 1, 1/2, ... until the Armijo
 * condition E(x + t d) <= E(x) + 1e-4 t g.d holds (allowing for round-off of
 * the energy sum, and rejecting steps that invert an element).  Stops when
 * |g| <= rtol |g0|. */
int or_newton(const or_model *M, const double *a, double *x, double rtol, int max_newton, int max_cg,
              int max_ls, or_stats *st)
{
    int d = M->d;
    long n = M->nv * d;
    double *g = (double *)malloc(sizeof(double) * n);
    double *mg = (double *)malloc(sizeof(double) * n);
    double *dir = (double *)malloc(sizeof(double) * n);
    double *xt = (double *)malloc(sizeof(double) * n);
    or_stats s;
    memset(&s, 0, sizeof(s));
    s.status = OR_ENOTCONVERGED;
    or_grad(M, x, a, g, NULL);
    double gn = sqrt(vdot(n, g, g));
    s.res0 = gn;
    double g0 = gn;
    double Sabs, mJ;
    double E = or_energy(M, x, a, &Sabs, &mJ);
    int it = 0;
    for (;; ++it) {
        if (gn <= rtol * g0) {
            s.status = OR_OK;
            break;
        }
        if (it >= max_newton) break;
        double eta = sqrt(gn / g0);
        if (eta > 0.5) eta = 0.5;
        for (long i = 0; i < n; ++i) mg[i] = -g[i];
        int neg = 0;
        s.cg_iters_total += or_cg(M, x, a, mg, dir, eta, max_cg, &neg);
        double gd = vdot(n, g, dir);
        if (!(gd < 0.0)) {
            for (long i = 0; i < n; ++i) dir[i] = -g[i];
            gd = -gn * gn;
        }
        double t = 1.0, Et = INFINITY, St = 0.0;
        int ok = 0;
        for (int ls = 0; ls < max_ls; ++ls) {
            for (long i = 0; i < n; ++i) xt[i] = x[i] + t * dir[i];
            Et = or_energy(M, xt, a, &St, NULL);
            double slack = 64.0 * 2.220446049250313e-16 * (Sabs > St ? Sabs : St);
            if (isfinite(Et) && Et <= E + 1e-4 * t * gd + slack) {
                ok = 1;
                break;
            }
            t *= 0.5;
            s.ls_halvings += 1;
        }
        if (!ok) {
            s.status = OR_ELINESEARCH;
            break;
        }
        memcpy(x, xt, sizeof(double) * n);
        E = Et;
        Sabs = St;
        or_grad(M, x, a, g, NULL);
        gn = sqrt(vdot(n, g, g));
    }
    s.newton_iters = it;
    s.res_final = gn;
    or_energy(M, x, a, NULL, &mJ);
    s.min_J = mJ;
    if (st) *st = s;
    free(g);
    free(mg);
    free(dir);
    free(xt);
    return s.status;
}
