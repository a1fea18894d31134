/*
 * Plain FP64 CPU oracle for high-order TMOP (Dobrev, Knupp, Kolev, Mittal,
 * Tomov, "The Target-Matrix Optimization Paradigm for High-Order Meshes").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, obviously-correct statement
 * of what the GPU library computes. Only the test suite, the smoke check and
 * the CPU-baseline leg of the benchmark load it. It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls it.
 *
 * Deliberately naive:
 *   - basis gradients are evaluated at every quadrature point from the 1D
 *     Lagrange product formula (no sum factorisation, O(n^d) per point);
 *   - A, T, mu and its derivatives are formed point by point in the order of
 *     the paper's formulas;
 *   - F is accumulated with Neumaier compensated summation in element order;
 *   - nodal vectors are accumulated in element order.
 *
 * Parity status of each function (pins live in tests/test_oracle_pins.py):
 *   quadrature, Lagrange basis, geometry (A), mu1/mu2/mu7/mu14/mu9/mu77/mu302/mu303
 *   values, first and second derivatives, energy, gradient, Hessian action,
 *   MINRES, CG, Newton: all pinned (closed forms, invariants, finite
 *   differences, textbook stiffness, library routines, brute force).
 *   mu302 is not in the paper; its definition |T|^2 |T^-1|^2 / 9 - 1 is pinned
 *   only by mu(I)=0, rotation/scale invariance and finite differences.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846
#define ORC_MAXD 3
#define ORC_MAXN 8  /* 1D nodes (order <= 7) */
#define ORC_MAXQ 12 /* 1D quadrature points */

enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_INVERTED = 3, ORC_ERR_LINESEARCH = 4, ORC_ERR_NOT_CONVERGED = 5 };
enum { ORC_GL = 0, ORC_GLL = 1 };
enum { ORC_W_IDENTITY = 0, ORC_W_CONST = 1, ORC_W_PER_QP = 2 };

/* Problem description, mirrored by a ctypes Structure in oracle/__init__.py. */
typedef struct {
  int dim, order, nelem, nnode;
  const int32_t* elem_nodes;   /* [nelem][(order+1)^dim], local lexicographic, x fastest */
  const uint8_t* fixed;        /* [dim][nnode], 1 = fixed dof; NULL = none fixed */
  int quad_kind, nq;           /* ORC_GL / ORC_GLL, points per direction */
  int metric;                  /* 1, 2, 7, 9, 14, 77 (2D); 1, 14, 302, 303 (3D) */
  int wkind;                   /* ORC_W_* */
  const double* W;             /* CONST: [d][d] row-major; PER_QP: [nelem][Q][d][d] */
  /* optional second term of a composite metric (Section 4.2, eq. (4.1)):
   * mu = mu_metric(A W^-1) + eta_q mu_metric2(A W2^-1); metric2 = 0: none */
  int metric2;
  const double* W2;            /* [d][d] constant target of the second term */
  const double* eta2;          /* [nelem][Q] weights of the second term, or NULL for 1 */
  /* restricted node movement (Section 4.3.1, eq. (4.2)): adds
   * sum_E int_{E_t} delta |x - x_init|^2 dx_t; delta = 0: none */
  double delta;
  const double* x_init;        /* [dim][nnode] */
} orc_problem;

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and quadrature (Section 3.3: GL or GLL tensor rules) */

/* P_m(t) and P_m'(t) by the three-term recurrence. */
static void legendre(int m, double t, double* P, double* dP) {
  double p0 = 1.0, p1 = t;
  if (m == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int j = 2; j <= m; ++j) {
    double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
    p0 = p1; p1 = p2;
  }
  *P = p1;
  /* (t^2 - 1) P_m' = m (t P_m - P_{m-1}); only used away from t = +-1 */
  *dP = m * (t * p1 - p0) / (t * t - 1.0);
}

/* Gauss-Legendre rule with q points mapped to [0,1] (weights sum to 1). */
int orc_gauss_legendre(int q, double* pts, double* wts) {
  if (q < 1 || q > ORC_MAXQ) return ORC_ERR_ARG;
  for (int i = 0; i < q; ++i) {
    double t = cos(ORC_PI * (i + 0.75) / (q + 0.5)), P, dP;
    for (int it = 0; it < 100; ++it) {
      legendre(q, t, &P, &dP);
      double dt = P / dP;
      t -= dt;
      if (fabs(dt) < 1e-16) break;
    }
    legendre(q, t, &P, &dP);
    /* ascending order on [0,1] */
    pts[q - 1 - i] = 0.5 * (t + 1.0);
    wts[q - 1 - i] = 0.5 * 2.0 / ((1.0 - t * t) * dP * dP);
  }
  return ORC_OK;
}

/* Gauss-Lobatto-Legendre rule with q >= 2 points mapped to [0,1]. The
 * interior points are the roots of P'_{q-1}. */
int orc_gauss_lobatto(int q, double* pts, double* wts) {
  if (q < 2 || q > ORC_MAXQ) return ORC_ERR_ARG;
  int m = q - 1;
  for (int j = 0; j <= m; ++j) {
    double t;
    if (j == 0) t = -1.0;
    else if (j == m) t = 1.0;
    else {
      t = -cos(ORC_PI * j / m);
      for (int it = 0; it < 100; ++it) {
        double P, dP;
        legendre(m, t, &P, &dP);
        double d2P = (2.0 * t * dP - m * (m + 1.0) * P) / (1.0 - t * t);
        double dt = dP / d2P;
        t -= dt;
        if (fabs(dt) < 1e-16) break;
      }
    }
    double P, dP;
    legendre(m, t, &P, &dP);
    if (j == 0 || j == m) P = (j == 0 && (m % 2)) ? -1.0 : 1.0;
    pts[j] = 0.5 * (t + 1.0);
    wts[j] = 0.5 * 2.0 / (m * (m + 1.0) * P * P);
  }
  return ORC_OK;
}

/* 1D Lagrange basis on the given nodes, value and derivative at xi, by the
 * product formula (nodal basis of Q_k, eq. (2.1)). */
void orc_lagrange(int n, const double* nodes, double xi, double* phi, double* dphi) {
  for (int i = 0; i < n; ++i) {
    double v = 1.0, d = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double den = nodes[i] - nodes[j];
      /* d(prod) by the product rule: d <- d*f + v*f' */
      d = d * (xi - nodes[j]) / den + v / den;
      v = v * (xi - nodes[j]) / den;
    }
    phi[i] = v;
    dphi[i] = d;
  }
}

/* ------------------------------------------------------------------------ */
/* Small dense matrix helpers (row-major d x d) */

static double det_d(int d, const double* M) {
  if (d == 2) return M[0] * M[3] - M[1] * M[2];
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* Cofactor matrix: C_ij = (-1)^(i+j) minor_ij, so that d(det)/dM = C. */
static void cof_d(int d, const double* M, double* C) {
  if (d == 2) {
    C[0] = M[3]; C[1] = -M[2]; C[2] = -M[1]; C[3] = M[0];
    return;
  }
  C[0] = M[4] * M[8] - M[5] * M[7];
  C[1] = -(M[3] * M[8] - M[5] * M[6]);
  C[2] = M[3] * M[7] - M[4] * M[6];
  C[3] = -(M[1] * M[8] - M[2] * M[7]);
  C[4] = M[0] * M[8] - M[2] * M[6];
  C[5] = -(M[0] * M[7] - M[1] * M[6]);
  C[6] = M[1] * M[5] - M[2] * M[4];
  C[7] = -(M[0] * M[5] - M[2] * M[3]);
  C[8] = M[0] * M[4] - M[1] * M[3];
}

/* Directional derivative of the cofactor matrix, by the product rule applied
 * to each 2x2 minor (in 2D the cofactor is linear in M). */
static void dcof_d(int d, const double* M, const double* E, double* dC) {
  if (d == 2) { cof_d(2, E, dC); return; }
#define PR(a, b, c, e) (E[a] * M[b] + M[a] * E[b] - E[c] * M[e] - M[c] * E[e])
  dC[0] = PR(4, 8, 5, 7);
  dC[1] = -PR(3, 8, 5, 6);
  dC[2] = PR(3, 7, 4, 6);
  dC[3] = -PR(1, 8, 2, 7);
  dC[4] = PR(0, 8, 2, 6);
  dC[5] = -PR(0, 7, 1, 6);
  dC[6] = PR(1, 5, 2, 4);
  dC[7] = -PR(0, 5, 2, 3);
  dC[8] = PR(0, 4, 1, 3);
#undef PR
}

static double ddot_m(int d, const double* X, const double* Y) {
  double s = 0.0;
  for (int i = 0; i < d * d; ++i) s += X[i] * Y[i];
  return s;
}

static void matmul_d(int d, const double* X, const double* Y, double* Z) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) {
      double s = 0.0;
      for (int k = 0; k < d; ++k) s += X[i * d + k] * Y[k * d + j];
      Z[i * d + j] = s;
    }
}

static void transpose_d(int d, const double* X, double* Y) {
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Y[j * d + i] = X[i * d + j];
}

static int inverse_d(int d, const double* M, double* Minv) {
  double C[9], det = det_d(d, M);
  if (!(det != 0.0)) return ORC_ERR_ARG;
  cof_d(d, M, C);
  /* M^{-1} = C^T / det */
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) Minv[i * d + j] = C[j * d + i] / det;
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Quality metrics (Section 3.2, Table 3.1) with first derivative P = dmu/dT
 * and second directional derivative dP = d^2mu/dT^2 : dT (Section 3.4: the
 * Hessian needs the second derivatives of mu; they are written here in the
 * invariants I1 = |T|^2, tau = det T, C = cof T, d tau = C : dT).
 *
 * Returns 0, or ORC_ERR_INVERTED if the metric is a barrier metric and
 * tau <= 0 (mu undefined; the caller treats F as +inf). P and dP may be NULL.
 */
int orc_metric(int id, int d, const double* T, const double* dT, double* mu, double* P, double* dP) {
  const int dd = d * d;
  int ok2 = (id == 2 || id == 7 || id == 9 || id == 77), ok3 = (id == 302 || id == 303);
  if (!(id == 1 || id == 14 || id == 98 || (d == 2 && ok2) || (d == 3 && ok3))) return ORC_ERR_ARG;
  double tau = det_d(d, T);
  double C[9], dC[9];
  double I1 = ddot_m(d, T, T);
  cof_d(d, T, C);
  double dtau = 0.0, dI1 = 0.0;
  if (dP) {
    dcof_d(d, T, dT, dC);
    dtau = ddot_m(d, C, dT);
    dI1 = 2.0 * ddot_m(d, T, dT);
  }
  switch (id) {
    case 1: /* mu1 = |T|^2 */
      *mu = I1;
      if (P) for (int i = 0; i < dd; ++i) P[i] = 2.0 * T[i];
      if (dP) for (int i = 0; i < dd; ++i) dP[i] = 2.0 * dT[i];
      return ORC_OK;
    case 14: { /* mu14 = |T - I|^2 */
      double s = 0.0;
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          double e = T[i * d + j] - (i == j ? 1.0 : 0.0);
          s += e * e;
          if (P) P[i * d + j] = 2.0 * e;
        }
      *mu = s;
      if (dP) for (int i = 0; i < dd; ++i) dP[i] = 2.0 * dT[i];
      return ORC_OK;
    }
    default: break;
  }
  if (!(tau > 0.0)) { *mu = INFINITY; return ORC_ERR_INVERTED; }
  switch (id) {
    case 98: { /* mu98 = |T - I|^2 / tau, the replication barrier metric (Section 4.3.2), any d */
      double E[9], s = 0.0;
      for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
          E[i * d + j] = T[i * d + j] - (i == j ? 1.0 : 0.0);
          s += E[i * d + j] * E[i * d + j];
        }
      *mu = s / tau;
      /* P = (2 (T - I) - mu C) / tau */
      double Pl[9];
      for (int i = 0; i < dd; ++i) Pl[i] = (2.0 * E[i] - *mu * C[i]) / tau;
      if (P) for (int i = 0; i < dd; ++i) P[i] = Pl[i];
      if (dP) {
        /* dP = (2 dT - dmu C - mu dC - P dtau) / tau, dmu = P : dT */
        double dmu = ddot_m(d, Pl, dT);
        for (int i = 0; i < dd; ++i) dP[i] = (2.0 * dT[i] - dmu * C[i] - *mu * dC[i] - Pl[i] * dtau) / tau;
      }
      return ORC_OK;
    }
    case 2: { /* mu2 = |T|^2 / (2 tau) - 1, 2D shape */
      if (d != 2) return ORC_ERR_ARG;
      *mu = I1 / (2.0 * tau) - 1.0;
      double a = 1.0 / tau, b = I1 / (2.0 * tau * tau);
      if (P) for (int i = 0; i < dd; ++i) P[i] = a * T[i] - b * C[i];
      if (dP) {
        double da = -dtau / (tau * tau);
        double db = dI1 / (2.0 * tau * tau) - I1 * dtau / (tau * tau * tau);
        for (int i = 0; i < dd; ++i) dP[i] = a * dT[i] + da * T[i] - db * C[i] - b * dC[i];
      }
      return ORC_OK;
    }
    case 7: { /* mu7 = |T - T^{-t}|^2 = I1 (1 + tau^-2) - 4 in 2D (|T^-1|^2 = I1/tau^2) */
      if (d != 2) return ORC_ERR_ARG;
      double it2 = 1.0 / (tau * tau);
      *mu = I1 * (1.0 + it2) - 4.0;
      double a = 2.0 * (1.0 + it2), b = 2.0 * I1 * it2 / tau;
      if (P) for (int i = 0; i < dd; ++i) P[i] = a * T[i] - b * C[i];
      if (dP) {
        double da = -4.0 * dtau * it2 / tau;
        double db = 2.0 * dI1 * it2 / tau - 6.0 * I1 * dtau * it2 * it2;
        for (int i = 0; i < dd; ++i) dP[i] = a * dT[i] + da * T[i] - db * C[i] - b * dC[i];
      }
      return ORC_OK;
    }
    case 9: { /* mu9 = tau |T - T^{-t}|^2 = tau I1 + I1/tau - 4 tau in 2D */
      if (d != 2) return ORC_ERR_ARG;
      *mu = tau * I1 + I1 / tau - 4.0 * tau;
      /* P = (2 tau + 2/tau) T + (I1 - I1/tau^2 - 4) C */
      double a = 2.0 * tau + 2.0 / tau, b = I1 - I1 / (tau * tau) - 4.0;
      if (P) for (int i = 0; i < dd; ++i) P[i] = a * T[i] + b * C[i];
      if (dP) {
        double da = 2.0 * dtau - 2.0 * dtau / (tau * tau);
        double db = dI1 - dI1 / (tau * tau) + 2.0 * I1 * dtau / (tau * tau * tau);
        for (int i = 0; i < dd; ++i) dP[i] = a * dT[i] + da * T[i] + b * dC[i] + db * C[i];
      }
      return ORC_OK;
    }
    case 77: { /* mu77 = (tau - 1/tau)^2 / 2, 2D size */
      if (d != 2) return ORC_ERR_ARG;
      double s = tau - 1.0 / tau, ds = 1.0 + 1.0 / (tau * tau);
      *mu = 0.5 * s * s;
      /* P = s ds C */
      if (P) for (int i = 0; i < dd; ++i) P[i] = s * ds * C[i];
      if (dP) {
        double dsds = (ds * ds - s * 2.0 / (tau * tau * tau)) * dtau; /* d(s ds) */
        for (int i = 0; i < dd; ++i) dP[i] = dsds * C[i] + s * ds * dC[i];
      }
      return ORC_OK;
    }
    case 303: { /* mu303 = |T|^2 / (3 tau^{2/3}) - 1, 3D shape */
      if (d != 3) return ORC_ERR_ARG;
      double t23 = pow(tau, -2.0 / 3.0); /* tau^{-2/3} */
      double t53 = t23 / tau;            /* tau^{-5/3} */
      *mu = I1 * t23 / 3.0 - 1.0;
      double a = 2.0 * t23 / 3.0, b = 2.0 * I1 * t53 / 9.0;
      if (P) for (int i = 0; i < dd; ++i) P[i] = a * T[i] - b * C[i];
      if (dP) {
        double da = -4.0 * t53 * dtau / 9.0;
        double db = 2.0 * dI1 * t53 / 9.0 - 10.0 * I1 * t53 * dtau / (27.0 * tau);
        for (int i = 0; i < dd; ++i) dP[i] = a * dT[i] + da * T[i] - db * C[i] - b * dC[i];
      }
      return ORC_OK;
    }
    case 302: { /* mu302 = |T|^2 |T^-1|^2 / 9 - 1 = I1 K / (9 tau^2) - 1, K = |cof T|^2 */
      if (d != 3) return ORC_ERR_ARG;
      double K = ddot_m(3, C, C);
      double TtT[9], Tt[9], TTtT[9], Kp[9];
      transpose_d(3, T, Tt);
      matmul_d(3, Tt, T, TtT);
      matmul_d(3, T, TtT, TTtT);
      /* dK/dT = 2 (I1 T - T T^t T) */
      for (int i = 0; i < 9; ++i) Kp[i] = 2.0 * (I1 * T[i] - TTtT[i]);
      double a = 1.0 / (9.0 * tau * tau);
      *mu = a * I1 * K - 1.0;
      double c = 2.0 * a * I1 * K / tau;
      if (P) for (int i = 0; i < 9; ++i) P[i] = a * (I1 * Kp[i] + 2.0 * K * T[i]) - c * C[i];
      if (dP) {
        double dK = ddot_m(3, Kp, dT);
        double da = -2.0 * a * dtau / tau;
        /* d(T T^t T) = dT T^t T + T dT^t T + T T^t dT */
        double dTt[9], X1[9], X2[9], X3[9], tmp[9];
        transpose_d(3, dT, dTt);
        matmul_d(3, dT, TtT, X1);
        matmul_d(3, dTt, T, tmp);
        matmul_d(3, T, tmp, X2);
        matmul_d(3, Tt, dT, tmp);
        matmul_d(3, T, tmp, X3);
        double dc = 2.0 * (da * I1 * K + a * dI1 * K + a * I1 * dK) / tau - c * dtau / tau;
        for (int i = 0; i < 9; ++i) {
          double dKp = 2.0 * (dI1 * T[i] + I1 * dT[i] - X1[i] - X2[i] - X3[i]);
          dP[i] = da * (I1 * Kp[i] + 2.0 * K * T[i]) +
                  a * (dI1 * Kp[i] + I1 * dKp + 2.0 * dK * T[i] + 2.0 * K * dT[i]) - dc * C[i] - c * dC[i];
        }
      }
      return ORC_OK;
    }
    default:
      return ORC_ERR_ARG;
  }
}

/* ------------------------------------------------------------------------ */
/* Per-problem tables: quadrature, GLL nodal basis, gradients at every point */

typedef struct {
  int d, n, nq, ndof_e, Q;
  double qp[ORC_MAXQ], qw[ORC_MAXQ];
  double gll[ORC_MAXN];
  double* w;      /* [Q] tensor weights */
  double* gradphi; /* [Q][ndof_e][d]: reference gradient of every local basis function */
  double* phi;     /* [Q][ndof_e]: value of every local basis function */
} orc_tables;

static int ipow(int b, int e) { int r = 1; while (e--) r *= b; return r; }

static int tables_init(const orc_problem* p, orc_tables* t) {
  memset(t, 0, sizeof(*t));
  if (p->dim < 2 || p->dim > 3 || p->order < 1 || p->order + 1 > ORC_MAXN) return ORC_ERR_ARG;
  t->d = p->dim;
  t->n = p->order + 1;
  t->nq = p->nq;
  double dummy[ORC_MAXN];
  /* Lagrange nodes: Gauss-Lobatto points of the element, ascending on [0,1] */
  if (orc_gauss_lobatto(t->n, t->gll, dummy) != ORC_OK) return ORC_ERR_ARG;
  int rc = (p->quad_kind == ORC_GLL) ? orc_gauss_lobatto(p->nq, t->qp, t->qw) : orc_gauss_legendre(p->nq, t->qp, t->qw);
  if (rc != ORC_OK) return rc;
  t->ndof_e = ipow(t->n, t->d);
  t->Q = ipow(t->nq, t->d);
  t->w = (double*)malloc(sizeof(double) * t->Q);
  t->gradphi = (double*)malloc(sizeof(double) * t->Q * t->ndof_e * t->d);
  t->phi = (double*)malloc(sizeof(double) * t->Q * t->ndof_e);
  double phi[ORC_MAXQ][ORC_MAXN], dphi[ORC_MAXQ][ORC_MAXN];
  for (int a = 0; a < t->nq; ++a) orc_lagrange(t->n, t->gll, t->qp[a], phi[a], dphi[a]);
  for (int q = 0; q < t->Q; ++q) {
    int qi[3] = {q % t->nq, (q / t->nq) % t->nq, q / (t->nq * t->nq)};
    double wq = 1.0;
    for (int c = 0; c < t->d; ++c) wq *= t->qw[qi[c]];
    t->w[q] = wq;
    for (int i = 0; i < t->ndof_e; ++i) {
      int ii[3] = {i % t->n, (i / t->n) % t->n, i / (t->n * t->n)};
      double v = 1.0;
      for (int c = 0; c < t->d; ++c) v *= phi[qi[c]][ii[c]];
      t->phi[(size_t)q * t->ndof_e + i] = v;
      for (int b = 0; b < t->d; ++b) {
        /* d phi_i / d xi_b = phi'(xi_b) * prod_{c != b} phi(xi_c) */
        double g = 1.0;
        for (int c = 0; c < t->d; ++c) g *= (c == b) ? dphi[qi[c]][ii[c]] : phi[qi[c]][ii[c]];
        t->gradphi[((size_t)q * t->ndof_e + i) * t->d + b] = g;
      }
    }
  }
  return ORC_OK;
}

static void tables_free(orc_tables* t) { free(t->w); free(t->gradphi); free(t->phi); }

/* Target at (element, qp): W^{-1} and det W (Section 3.1; det W > 0 required). */
static int target_at(const orc_problem* p, int e, int q, int Q, double* Winv, double* detW) {
  int d = p->dim;
  if (p->wkind == ORC_W_IDENTITY) {
    for (int i = 0; i < d * d; ++i) Winv[i] = 0.0;
    for (int i = 0; i < d; ++i) Winv[i * d + i] = 1.0;
    *detW = 1.0;
    return ORC_OK;
  }
  const double* W = (p->wkind == ORC_W_CONST) ? p->W : p->W + ((size_t)e * Q + q) * d * d;
  *detW = det_d(d, W);
  if (!(*detW > 0.0)) return ORC_ERR_ARG;
  return inverse_d(d, W, Winv);
}

/* Jacobian A_ab = sum_i x_{i,a} d phi_i / d xi_b at quadrature point q of element e (eq. (2.2)). */
static void jacobian_at(const orc_problem* p, const orc_tables* t, const double* x, int e, int q, double* A) {
  int d = t->d;
  for (int i = 0; i < d * d; ++i) A[i] = 0.0;
  const int32_t* en = p->elem_nodes + (size_t)e * t->ndof_e;
  for (int i = 0; i < t->ndof_e; ++i) {
    const double* gp = t->gradphi + ((size_t)q * t->ndof_e + i) * d;
    for (int a = 0; a < d; ++a) {
      double xa = x[(size_t)a * p->nnode + en[i]];
      for (int b = 0; b < d; ++b) A[a * d + b] += xa * gp[b];
    }
  }
}

/* Neumaier compensated sum */
typedef struct { double s, c; } ksum;
static void kadd(ksum* k, double v) {
  double t = k->s + v;
  if (fabs(k->s) >= fabs(v)) k->c += (k->s - t) + v;
  else k->c += (v - t) + k->s;
  k->s = t;
}

/* Every A at every quadrature point: out [nelem][Q][d][d]. */
int orc_jacobians(const orc_problem* p, const double* x, double* out) {
  orc_tables t;
  int rc = tables_init(p, &t);
  if (rc) return rc;
  int dd = t.d * t.d;
  for (int e = 0; e < p->nelem; ++e)
    for (int q = 0; q < t.Q; ++q) jacobian_at(p, &t, x, e, q, out + ((size_t)e * t.Q + q) * dd);
  tables_free(&t);
  return ORC_OK;
}

/* Tensor quadrature weights and basis gradients used by the oracle, for tests. */
int orc_tables_dump(const orc_problem* p, double* w_out, double* gradphi_out) {
  orc_tables t;
  int rc = tables_init(p, &t);
  if (rc) return rc;
  if (w_out) memcpy(w_out, t.w, sizeof(double) * t.Q);
  if (gradphi_out) memcpy(gradphi_out, t.gradphi, sizeof(double) * t.Q * t.ndof_e * t.d);
  tables_free(&t);
  return ORC_OK;
}

/* Variational objective F_V = sum_E sum_q w_q det W mu(T), T = A W^{-1} (eq. (2.4)).
 * elems: optional list of element ids (NULL = all). Any det A <= 0 makes
 * F = +inf when the metric is a barrier (Section 3.4: "big value"); min det A
 * over the visited points is always returned. Returns ORC_ERR_INVERTED when
 * some det A <= 0. */
int orc_energy(const orc_problem* p, const double* x, const int32_t* elems, int nelems, double* F, double* min_detA) {
  orc_tables t;
  int rc = tables_init(p, &t);
  if (rc) return rc;
  int d = t.d, ne = elems ? nelems : p->nelem;
  ksum acc = {0.0, 0.0};
  double mdet = INFINITY;
  int inverted = 0, barrier_hit = 0;
  for (int k = 0; k < ne; ++k) {
    int e = elems ? elems[k] : k;
    for (int q = 0; q < t.Q; ++q) {
      double A[9], Winv[9], T[9], detW, mu;
      jacobian_at(p, &t, x, e, q, A);
      if (target_at(p, e, q, t.Q, Winv, &detW)) { tables_free(&t); return ORC_ERR_ARG; }
      double dA = det_d(d, A);
      if (dA < mdet) mdet = dA;
      if (!(dA > 0.0)) inverted = 1;
      matmul_d(d, A, Winv, T);
      int mrc = orc_metric(p->metric, d, T, NULL, &mu, NULL, NULL);
      if (mrc == ORC_ERR_ARG) { tables_free(&t); return ORC_ERR_ARG; }
      if (mrc == ORC_ERR_INVERTED) { barrier_hit = 1; continue; }
      kadd(&acc, t.w[q] * detW * mu);
      if (p->metric2) {  /* eq. (4.1): second term with its own target and weight */
        double W2inv[9], detW2, T2[9], mu2;
        if (inverse_d(d, p->W2, W2inv) != ORC_OK) { tables_free(&t); return ORC_ERR_ARG; }
        detW2 = det_d(d, p->W2);
        matmul_d(d, A, W2inv, T2);
        int m2 = orc_metric(p->metric2, d, T2, NULL, &mu2, NULL, NULL);
        if (m2 == ORC_ERR_ARG) { tables_free(&t); return ORC_ERR_ARG; }
        if (m2 == ORC_ERR_INVERTED) { barrier_hit = 1; continue; }
        const double eta = p->eta2 ? p->eta2[(size_t)e * t.Q + q] : 1.0;
        kadd(&acc, t.w[q] * detW2 * eta * mu2);
      }
      if (p->delta != 0.0) {  /* eq. (4.2): delta |x - x_init|^2 at the point */
        const int32_t* en = p->elem_nodes + (size_t)e * t.ndof_e;
        double u2 = 0.0;
        for (int a = 0; a < d; ++a) {
          double u = 0.0;
          for (int i = 0; i < t.ndof_e; ++i) {
            const size_t dof = (size_t)a * p->nnode + en[i];
            u += (x[dof] - p->x_init[dof]) * t.phi[(size_t)q * t.ndof_e + i];
          }
          u2 += u * u;
        }
        kadd(&acc, t.w[q] * detW * p->delta * u2);
      }
    }
  }
  *F = barrier_hit ? INFINITY : acc.s + acc.c;
  *min_detA = mdet;
  tables_free(&t);
  return inverted ? ORC_ERR_INVERTED : ORC_OK;
}

/* Shared driver of the gradient (Section 3.4) and the Hessian action:
 *   g_{i,a} = sum_E sum_q w_q det W sum_c P_ac (W^{-t} grad phi_i)_c
 *   y_{i,a} = sum_E sum_q w_q det W sum_c dP_ac (W^{-t} grad phi_i)_c,
 * with dP = d^2mu/dT^2 : dT and dT = (sum_i v_i (x) grad phi_i) W^{-1}.
 * Fixed dofs of the output are zero; for the Hessian action v is masked first. */
static int nodal_op(const orc_problem* p, const double* x, const double* v, const int32_t* elems, int nelems, double* out) {
  orc_tables t;
  int rc = tables_init(p, &t);
  if (rc) return rc;
  int d = t.d, ne = elems ? nelems : p->nelem, status = ORC_OK;
  size_t ndof = (size_t)d * p->nnode;
  for (size_t i = 0; i < ndof; ++i) out[i] = 0.0;
  for (int k = 0; k < ne; ++k) {
    int e = elems ? elems[k] : k;
    const int32_t* en = p->elem_nodes + (size_t)e * t.ndof_e;
    for (int q = 0; q < t.Q; ++q) {
      double A[9], Winv[9], T[9], detW, mu, P[9], dA[9], dT[9], dP[9], G[9];
      jacobian_at(p, &t, x, e, q, A);
      if (target_at(p, e, q, t.Q, Winv, &detW)) { tables_free(&t); return ORC_ERR_ARG; }
      matmul_d(d, A, Winv, T);
      if (v) {
        for (int i = 0; i < d * d; ++i) dA[i] = 0.0;
        for (int i = 0; i < t.ndof_e; ++i) {
          const double* gp = t.gradphi + ((size_t)q * t.ndof_e + i) * d;
          for (int a = 0; a < d; ++a) {
            size_t dof = (size_t)a * p->nnode + en[i];
            double va = (p->fixed && p->fixed[dof]) ? 0.0 : v[dof];
            for (int b = 0; b < d; ++b) dA[a * d + b] += va * gp[b];
          }
        }
        matmul_d(d, dA, Winv, dT);
      }
      int mrc = orc_metric(p->metric, d, T, v ? dT : NULL, &mu, v ? NULL : P, v ? dP : NULL);
      if (mrc == ORC_ERR_ARG) { tables_free(&t); return ORC_ERR_ARG; }
      if (mrc == ORC_ERR_INVERTED) { status = ORC_ERR_INVERTED; continue; }
      const double* S = v ? dP : P;
      double wdet = t.w[q] * detW;
      /* G = S W^{-t}: then (S W^{-t} grad phi_i)_a = sum_b G_ab grad phi_i_b */
      double WinvT[9];
      transpose_d(d, Winv, WinvT);
      matmul_d(d, S, WinvT, G);
      for (int i = 0; i < t.ndof_e; ++i) {
        const double* gp = t.gradphi + ((size_t)q * t.ndof_e + i) * d;
        for (int a = 0; a < d; ++a) {
          double s = 0.0;
          for (int b = 0; b < d; ++b) s += G[a * d + b] * gp[b];
          out[(size_t)a * p->nnode + en[i]] += wdet * s;
        }
      }
      if (p->metric2) {  /* eq. (4.1): the second term, same formulas with W2 and eta */
        double W2inv[9], W2invT[9], T2[9], dT2[9], P2[9], dP2[9], G2[9], mu2;
        if (inverse_d(d, p->W2, W2inv) != ORC_OK) { tables_free(&t); return ORC_ERR_ARG; }
        const double detW2 = det_d(d, p->W2);
        matmul_d(d, A, W2inv, T2);
        if (v) matmul_d(d, dA, W2inv, dT2);
        int m2 = orc_metric(p->metric2, d, T2, v ? dT2 : NULL, &mu2, v ? NULL : P2, v ? dP2 : NULL);
        if (m2 == ORC_ERR_ARG) { tables_free(&t); return ORC_ERR_ARG; }
        if (m2 == ORC_ERR_INVERTED) { status = ORC_ERR_INVERTED; continue; }
        const double eta = p->eta2 ? p->eta2[(size_t)e * t.Q + q] : 1.0;
        transpose_d(d, W2inv, W2invT);
        matmul_d(d, v ? dP2 : P2, W2invT, G2);
        const double wdet2 = t.w[q] * detW2 * eta;
        for (int i = 0; i < t.ndof_e; ++i) {
          const double* gp = t.gradphi + ((size_t)q * t.ndof_e + i) * d;
          for (int a = 0; a < d; ++a) {
            double s = 0.0;
            for (int b = 0; b < d; ++b) s += G2[a * d + b] * gp[b];
            out[(size_t)a * p->nnode + en[i]] += wdet2 * s;
          }
        }
      }
      if (p->delta != 0.0) {
        /* eq. (4.2): gradient 2 delta (x - x_init)(x_q) phi_i, Hessian action
         * 2 delta v(x_q) phi_i (a mass matrix) */
        const double* ph = t.phi + (size_t)q * t.ndof_e;
        for (int a = 0; a < d; ++a) {
          double u = 0.0;
          for (int i = 0; i < t.ndof_e; ++i) {
            const size_t dof = (size_t)a * p->nnode + en[i];
            if (v) u += ((p->fixed && p->fixed[dof]) ? 0.0 : v[dof]) * ph[i];
            else u += (x[dof] - p->x_init[dof]) * ph[i];
          }
          const double c = 2.0 * p->delta * wdet * u;
          for (int i = 0; i < t.ndof_e; ++i) out[(size_t)a * p->nnode + en[i]] += c * ph[i];
        }
      }
    }
  }
  if (p->fixed)
    for (size_t i = 0; i < ndof; ++i)
      if (p->fixed[i]) out[i] = 0.0;
  tables_free(&t);
  return status;
}

int orc_gradient(const orc_problem* p, const double* x, const int32_t* elems, int nelems, double* g) {
  return nodal_op(p, x, NULL, elems, nelems, g);
}

int orc_hess_apply(const orc_problem* p, const double* x, const double* v, const int32_t* elems, int nelems, double* y) {
  return nodal_op(p, x, v, elems, nelems, y);
}

/* ------------------------------------------------------------------------ */
/* Newton with MINRES inner solves and the det(A) > 0 line search (Section 3.4,
 * Section 5: MINRES, relative tolerance 1e-12). */

static double vdot(size_t n, const double* a, const double* b) {
  double s = 0.0;
  for (size_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* MINRES for H p = b (H symmetric, possibly indefinite), zero initial guess:
 * Lanczos tridiagonalisation of H with the residual minimised through Givens
 * rotations (Paige and Saunders). Stops when the residual estimate falls to
 * rtol * |b|. Returns iterations used (negative if maxit was reached). */
int orc_minres(const orc_problem* p, const double* x, const double* b, double rtol, int maxit, double* sol) {
  size_t n = (size_t)p->dim * p->nnode;
  double* v_prev = calloc(n, sizeof(double));
  double* v = malloc(n * sizeof(double));
  double* Av = malloc(n * sizeof(double));
  double* w_prev = calloc(n, sizeof(double));
  double* w = calloc(n, sizeof(double));
  for (size_t i = 0; i < n; ++i) sol[i] = 0.0;
  double beta1 = sqrt(vdot(n, b, b));
  int it = 0, done = 0;
  if (beta1 == 0.0) done = 1;
  for (size_t i = 0; i < n; ++i) v[i] = done ? 0.0 : b[i] / beta1;
  double beta = beta1, eta = beta1;
  /* Givens state: the last two rotations */
  double c_old = 1.0, s_old = 0.0, c = 1.0, s = 0.0;
  while (!done && it < maxit) {
    ++it;
    orc_hess_apply(p, x, v, NULL, 0, Av);
    double alpha = vdot(n, v, Av);
    /* Lanczos: beta_next v_next = H v - alpha v - beta v_prev */
    for (size_t i = 0; i < n; ++i) Av[i] -= alpha * v[i] + beta * v_prev[i];
    double beta_next = sqrt(vdot(n, Av, Av));
    /* apply the two previous rotations to the new column (beta, alpha, beta_next) */
    double r1 = s_old * beta;            /* entry two above the diagonal */
    double tmp = c_old * beta;
    double r2 = c * tmp + s * alpha;     /* entry one above the diagonal */
    double r3 = -s * tmp + c * alpha;    /* diagonal before the new rotation */
    double rho = sqrt(r3 * r3 + beta_next * beta_next);
    double c_new = rho > 0.0 ? r3 / rho : 1.0, s_new = rho > 0.0 ? beta_next / rho : 0.0;
    /* w = (v - r1 w_prev2' - r2 w_prev') / rho with the running direction vectors */
    for (size_t i = 0; i < n; ++i) {
      double wn = (v[i] - r1 * w_prev[i] - r2 * w[i]) / rho;
      w_prev[i] = w[i];
      w[i] = wn;
      sol[i] += c_new * eta * wn;
    }
    eta = -s_new * eta;
    c_old = c; s_old = s; c = c_new; s = s_new;
    if (fabs(eta) <= rtol * beta1 || beta_next == 0.0) { done = 1; break; }
    for (size_t i = 0; i < n; ++i) {
      v_prev[i] = v[i];
      v[i] = Av[i] / beta_next;
    }
    beta = beta_next;
  }
  free(v_prev); free(v); free(Av); free(w_prev); free(w);
  return done ? it : -it;
}

/* Conjugate gradients for H p = b, zero initial guess (valid when H is SPD). */
int orc_cg(const orc_problem* p, const double* x, const double* b, double rtol, int maxit, double* sol) {
  size_t n = (size_t)p->dim * p->nnode;
  double* r = malloc(n * sizeof(double));
  double* d = malloc(n * sizeof(double));
  double* Hd = malloc(n * sizeof(double));
  for (size_t i = 0; i < n; ++i) { sol[i] = 0.0; r[i] = b[i]; d[i] = b[i]; }
  double rr = vdot(n, r, r), r0 = sqrt(rr);
  int it = 0, done = (r0 == 0.0);
  while (!done && it < maxit) {
    ++it;
    orc_hess_apply(p, x, d, NULL, 0, Hd);
    double dHd = vdot(n, d, Hd);
    if (!(dHd > 0.0)) break;
    double a = rr / dHd;
    for (size_t i = 0; i < n; ++i) { sol[i] += a * d[i]; r[i] -= a * Hd[i]; }
    double rr_new = vdot(n, r, r);
    if (sqrt(rr_new) <= rtol * r0) { done = 1; break; }
    for (size_t i = 0; i < n; ++i) d[i] = r[i] + (rr_new / rr) * d[i];
    rr = rr_new;
  }
  free(r); free(d); free(Hd);
  return done ? it : -it;
}

typedef struct {
  int max_newton;      /* Newton iteration cap */
  double rtol;         /* stop when |g| <= rtol |g0| (Section 5: 1e-12) */
  int krylov;          /* 0 = MINRES, 1 = CG */
  double krylov_rtol;  /* inner relative residual */
  int krylov_maxit;
  double alpha_shrink; /* step reduction factor */
  int max_halvings;
  double f_factor;     /* accept if F_new < f_factor F (Section 3.4: 1.2) */
  double g_factor;     /* accept if |g_new| < g_factor |g| (Section 3.4: 1.2) */
} orc_newton_opts;

/* history: [max_newton + 1][5] = F, |g|, min det A, alpha, krylov iterations */
int orc_newton(const orc_problem* p, double* x, const orc_newton_opts* o, double* history, int* iters_out) {
  size_t n = (size_t)p->dim * p->nnode;
  double* g = malloc(n * sizeof(double));
  double* pdir = malloc(n * sizeof(double));
  double* xt = malloc(n * sizeof(double));
  double* gt = malloc(n * sizeof(double));
  double F, mdet, Ft, mdett;
  int status = ORC_OK, it = 0;
  int rc = orc_energy(p, x, NULL, 0, &F, &mdet);
  if (rc == ORC_ERR_ARG || rc == ORC_ERR_INVERTED) { status = rc; goto out; }
  orc_gradient(p, x, NULL, 0, g);
  double ng = sqrt(vdot(n, g, g)), ng0 = ng;
  history[0] = F; history[1] = ng; history[2] = mdet; history[3] = 0.0; history[4] = 0.0;
  status = ORC_ERR_NOT_CONVERGED;
  for (it = 0; it < o->max_newton; ++it) {
    if (ng <= o->rtol * ng0) { status = ORC_OK; break; }
    int kit = (o->krylov == 1) ? orc_cg(p, x, g, o->krylov_rtol, o->krylov_maxit, pdir)
                               : orc_minres(p, x, g, o->krylov_rtol, o->krylov_maxit, pdir);
    double alpha = 1.0;
    int accepted = 0;
    for (int h = 0; h <= o->max_halvings; ++h, alpha *= o->alpha_shrink) {
      for (size_t i = 0; i < n; ++i) xt[i] = x[i] - alpha * pdir[i];
      orc_energy(p, xt, NULL, 0, &Ft, &mdett);
      if (!(mdett > 0.0) || !(Ft < o->f_factor * F)) continue;
      orc_gradient(p, xt, NULL, 0, gt);
      double ngt = sqrt(vdot(n, gt, gt));
      if (!(ngt < o->g_factor * ng)) continue;
      memcpy(x, xt, n * sizeof(double));
      memcpy(g, gt, n * sizeof(double));
      F = Ft; mdet = mdett; ng = ngt;
      accepted = 1;
      break;
    }
    double* hrow = history + (size_t)(it + 1) * 5;
    hrow[0] = F; hrow[1] = ng; hrow[2] = mdet; hrow[3] = accepted ? alpha : 0.0; hrow[4] = (double)kit;
    if (!accepted) { status = ORC_ERR_LINESEARCH; ++it; break; }
  }
  if (status == ORC_ERR_NOT_CONVERGED && ng <= o->rtol * ng0) status = ORC_OK;
out:
  *iters_out = it;
  free(g); free(pdir); free(xt); free(gt);
  return status;
}
