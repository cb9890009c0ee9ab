/*
 * Plain FP64 CPU oracle for the matrix-free DG operators of Kronbichler &
 * Kormann, "Fast matrix-free evaluation of discontinuous Galerkin finite
 * element operators" (arXiv:1711.03590).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or constant with the CUDA library.
 *
 * What it evaluates, with no sum factorization, blocking or fusion:
 *   - the symmetric interior penalty (SIPG) Laplacian, Sec. 2, Eq. (poisson_sip),
 *     with the average/jump definitions and the Dirichlet mirror principle
 *     of Sec. 2 (u+ = -u- + 2g, g = 0);
 *   - the upwind advection operator, Sec. 2, Eq. (advection), with the
 *     boundary flux |c.n| u- of Algorithm 1 step (iv)(c);
 *   - numerical integration on the tensor Gauss rule with the Jacobian of
 *     the reference-to-real map, Eq. (integral_advection).
 * Every basis function is evaluated directly as the product of three 1D
 * Lagrange polynomials at each 3D quadrature point.
 *
 * Two routes to y = A u (Eq. matvec):
 *   R1 (or_assemble): assembled sparse matrix, cell loop plus a loop over
 *       unique faces that fills the four (-,-),(-,+),(+,-),(+,+) blocks;
 *   R2 (or_apply_cells): unassembled, cell by cell: the cell integral and
 *       the six faces of the cell tested on this cell only.
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - tau_F = (p+1)^2 * max(A_F/|K-|, A_F/|K+|) (interior),
 *     (p+1)^2 * A_F/|K| (boundary), times penalty_scale; the paper only
 *     asks for "sufficiently large" tau (Sec. 2, after Eq. poisson_sip).
 *   - the coefficient kappa(x) = 1 + 0.5 sin(2 pi x_0) multiplies the cell
 *     integrand, the face average and the penalty;
 *   - at Dirichlet faces grad u+ = grad u- (the mirror is applied to values).
 *   - basis: Lagrange on the k Gauss-Lobatto points, quadrature: k Gauss
 *     points per direction on cells, k x k on faces.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXK 12
#define OR_PI 3.14159265358979323846264338327950288

typedef struct {
  int n[3];         /* cells per direction */
  int periodic;     /* 1: periodic in all directions, 0: Dirichlet on all of the boundary */
  int mapping;      /* 0: identity, 1: x_i = X_i + a sin(pi X) sin(pi Y) sin(pi Z),
                       2: affine, x_i = X_i + a X_{(i+1) mod 3} */
  double amplitude; /* a */
  int cell_jacobian; /* 0: analytic J of the mapping; 1: variant G2 of Sec. 5, the
                        cell term's J is the collocation derivative of the
                        positions of the cell's Gauss points */
  int basis;         /* 0: Lagrange on the Gauss-Lobatto points; 1: Hermite-like (degree >= 3,
                        see herm_value) */
} or_mesh;

typedef struct {
  int op;               /* 0: SIPG Laplacian, 1: upwind advection */
  int coeff;            /* 0: kappa = 1, 1: kappa = 1 + 0.5 sin(2 pi x_0) */
  double velocity[3];   /* advection speed c (constant) */
  double penalty_scale; /* multiplies tau */
} or_form;

/* ------------------------------------------------------------------ */
/* 1D rules (Sec. 2.1: tensor product of 1D Gauss formulas; GL nodes)  */
/* ------------------------------------------------------------------ */

/* Legendre polynomial P_n and its derivative at t in (-1,1), by the
 * three-term recurrence (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}. */
static void legendre_pd(int n, long double t, long double *p, long double *dp) {
  long double pm = 1.0L, pc = t;
  if (n == 0) { *p = 1.0L; *dp = 0.0L; return; }
  for (int m = 1; m < n; ++m) {
    long double pn = ((2.0L * m + 1.0L) * t * pc - (long double)m * pm) / (m + 1.0L);
    pm = pc;
    pc = pn;
  }
  *p = pc;
  /* (t^2 - 1) P_n' = n (t P_n - P_{n-1}) */
  *dp = (long double)n * (t * pc - pm) / (t * t - 1.0L);
}

/* k-point Gauss-Legendre rule mapped to [0,1], nodes ascending. */
int or_gauss(int k, double *x, double *w) {
  if (k < 1 || k > 64) return -1;
  for (int i = 0; i < k; ++i) {
    long double t = -cosl((long double)OR_PI * (i + 0.75L) / (k + 0.5L));
    long double p, dp;
    for (int it = 0; it < 100; ++it) {
      legendre_pd(k, t, &p, &dp);
      long double dt = p / dp;
      t -= dt;
      if (fabsl(dt) < 1e-30L) break;
    }
    legendre_pd(k, t, &p, &dp);
    x[i] = (double)(0.5L * (1.0L + t));
    w[i] = (double)(1.0L / ((1.0L - t * t) * dp * dp));  /* 2/((1-t^2)P'^2) / 2 */
  }
  return 0;
}

/* k-point Gauss-Lobatto rule on [0,1]: endpoints and the roots of P'_{k-1};
 * weights 2/(n(n+1) P_n(t)^2) / 2 with n = k-1. */
int or_gauss_lobatto(int k, double *x, double *w) {
  if (k < 2 || k > 64) return -1;
  int n = k - 1;
  for (int i = 0; i < k; ++i) {
    long double t;
    if (i == 0) t = -1.0L;
    else if (i == k - 1) t = 1.0L;
    else {
      t = -cosl((long double)OR_PI * i / (long double)n);
      for (int it = 0; it < 100; ++it) {
        long double p, dp;
        legendre_pd(n, t, &p, &dp);
        /* P_n'' from Legendre's equation: (1-t^2) P'' = 2 t P' - n(n+1) P */
        long double d2p = (2.0L * t * dp - (long double)n * (n + 1.0L) * p) / (1.0L - t * t);
        long double dt = dp / d2p;
        t -= dt;
        if (fabsl(dt) < 1e-30L) break;
      }
    }
    long double p;
    if (i == 0) p = (n % 2 == 0) ? 1.0L : -1.0L;
    else if (i == k - 1) p = 1.0L;
    else { long double dp; legendre_pd(n, t, &p, &dp); }
    x[i] = (double)(0.5L * (1.0L + t));
    w[i] = (double)(1.0L / ((long double)n * (n + 1.0L) * p * p));
  }
  x[0] = 0.0;
  x[k - 1] = 1.0;
  return 0;
}

/* Lagrange polynomial j on the given nodes, by the product formula. */
double or_lagrange(int k, const double *nodes, int j, double t) {
  double v = 1.0;
  for (int m = 0; m < k; ++m)
    if (m != j) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
  return v;
}

/* Its derivative: sum over the dropped factor l of the remaining product. */
double or_lagrange_deriv(int k, const double *nodes, int j, double t) {
  double s = 0.0;
  for (int l = 0; l < k; ++l) {
    if (l == j) continue;
    double v = 1.0 / (nodes[j] - nodes[l]);
    for (int m = 0; m < k; ++m)
      if (m != j && m != l) v *= (t - nodes[m]) / (nodes[j] - nodes[m]);
    s += v;
  }
  return s;
}

/* ------------------------------------------------------------------ */
/* Mesh, mapping and geometry (Sec. 2, reference-to-real map)          */
/* ------------------------------------------------------------------ */

static int64_t n_cells(const or_mesh *m) { return (int64_t)m->n[0] * m->n[1] * m->n[2]; }

static void cell_ijk(const or_mesh *m, int64_t c, int ijk[3]) {
  ijk[0] = (int)(c % m->n[0]);
  ijk[1] = (int)((c / m->n[0]) % m->n[1]);
  ijk[2] = (int)(c / ((int64_t)m->n[0] * m->n[1]));
}

static int64_t cell_id(const or_mesh *m, const int ijk[3]) {
  return ijk[0] + (int64_t)m->n[0] * (ijk[1] + (int64_t)m->n[1] * ijk[2]);
}

/* Neighbour across face (d, side s) of cell c; -1 at a Dirichlet boundary. */
static int64_t neighbour(const or_mesh *m, int64_t c, int d, int s) {
  int ijk[3];
  cell_ijk(m, c, ijk);
  ijk[d] += s ? 1 : -1;
  if (ijk[d] < 0 || ijk[d] >= m->n[d]) {
    if (!m->periodic) return -1;
    ijk[d] = (ijk[d] + m->n[d]) % m->n[d];
  }
  return cell_id(m, ijk);
}

/* Physical point x and Jacobian J = dx/dxi of cell c at reference point xi.
 * Cartesian point X_d = (i_d + xi_d)/n_d; mapping 1 shifts every coordinate
 * by a*s(X) with s = sin(pi X) sin(pi Y) sin(pi Z); mapping 2 is the linear
 * shear x_i = X_i + a X_{(i+1) mod 3} (constant J per cell, det = (1 + a^3)
 * / (n0 n1 n2)). */
static void cell_map(const or_mesh *m, int64_t c, const double xi[3], double x[3], double J[3][3]) {
  int ijk[3];
  cell_ijk(m, c, ijk);
  double X[3], h[3];
  for (int d = 0; d < 3; ++d) {
    h[d] = 1.0 / m->n[d];
    X[d] = (ijk[d] + xi[d]) * h[d];
  }
  double s = 0.0, gs[3] = {0.0, 0.0, 0.0};
  if (m->mapping == 1) {
    double sn[3], cs[3];
    for (int d = 0; d < 3; ++d) { sn[d] = sin(OR_PI * X[d]); cs[d] = cos(OR_PI * X[d]); }
    s = sn[0] * sn[1] * sn[2];
    gs[0] = OR_PI * cs[0] * sn[1] * sn[2];
    gs[1] = OR_PI * sn[0] * cs[1] * sn[2];
    gs[2] = OR_PI * sn[0] * sn[1] * cs[2];
  }
  if (m->mapping == 2) {
    double a = m->amplitude;
    for (int i = 0; i < 3; ++i) {
      int i1 = (i + 1) % 3;
      x[i] = X[i] + a * X[i1];
      for (int j = 0; j < 3; ++j) J[i][j] = ((i == j ? 1.0 : 0.0) + (j == i1 ? a : 0.0)) * h[j];
    }
    return;
  }
  double a = (m->mapping == 1) ? m->amplitude : 0.0;
  for (int i = 0; i < 3; ++i) {
    x[i] = X[i] + a * s;
    for (int j = 0; j < 3; ++j) J[i][j] = ((i == j ? 1.0 : 0.0) + a * gs[j]) * h[j];
  }
}

static double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

static void inv3(const double A[3][3], double det, double B[3][3]) {
  B[0][0] = (A[1][1] * A[2][2] - A[1][2] * A[2][1]) / det;
  B[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) / det;
  B[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) / det;
  B[1][0] = (A[1][2] * A[2][0] - A[1][0] * A[2][2]) / det;
  B[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) / det;
  B[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) / det;
  B[2][0] = (A[1][0] * A[2][1] - A[1][1] * A[2][0]) / det;
  B[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) / det;
  B[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) / det;
}

static double kappa_at(const or_form *f, const double x[3]) {
  return f->coeff == 1 ? 1.0 + 0.5 * sin(2.0 * OR_PI * x[0]) : 1.0;
}

/* ------------------------------------------------------------------ */
/* Basis tables for one degree                                          */
/* ------------------------------------------------------------------ */

typedef struct {
  int k;
  int kind;                    /* 0 Gauss-Lobatto Lagrange, 1 Hermite-like */
  double gl[OR_MAXK];          /* GL nodes (basis support of the Lagrange basis) */
  double gq[OR_MAXK], gw[OR_MAXK]; /* Gauss points/weights (quadrature) */
} basis1d;

static int basis_init(basis1d *b, int degree, int kind) {
  int k = degree + 1;
  if (degree < 1 || k > OR_MAXK) return -1;
  if (kind == 1 && degree < 3) return -1;
  b->k = k;
  b->kind = kind;
  double wl[OR_MAXK];
  if (or_gauss_lobatto(k, b->gl, wl)) return -1;
  if (or_gauss(k, b->gq, b->gw)) return -1;
  return 0;
}

/* Hermite-like basis of degree p >= 3 (the paper's Laplacian basis, Sec.
 * 3.1 and the table of tensor-product kernels, is characterized there only
 * by its face property: at most two nonzero entries in S_f and in D_f).
 * Reading, with x_0 = 0 < x_1 < ... < x_p = 1 the Gauss-Lobatto points and
 * w(t) = prod_{i=2}^{p-2} (t - x_i):
 *   phi_0 = (1 - t)^2 (1 + c t) w(t) / w(0), c = 2 - w'(0) / w(0),
 *   phi_1 = t (1 - t)^2 w(t) / (x_1 (1 - x_1)^2 w(x_1)),
 *   phi_j = t^2 (1 - t)^2 l_j(t) / (x_j^2 (1 - x_j)^2), 2 <= j <= p-2,
 *           l_j the Lagrange polynomial on x_2 .. x_{p-2},
 *   phi_{p-1}(t) = phi_1(1 - t), phi_p(t) = phi_0(1 - t).
 * They span P_p; only phi_0 is nonzero at t = 0 (value 1) and only phi_1
 * has a nonzero derivative there (phi_0'(0) = 0 by the choice of c), and
 * mirror-symmetrically at t = 1.  Every function but phi_0 and phi_p is 1 at
 * its own node x_j and 0 at the other interior nodes x_2 .. x_{p-2}, which
 * keeps the basis close to the Lagrange one (the change of basis at the
 * Gauss-Lobatto points has condition number 2.5-3.7 for p = 3..8).  deriv
 * != 0: the derivative. */
static void herm_w(const basis1d *b, double t, double *w, double *dw) {
  int p = b->k - 1;
  double v = 1.0, d = 0.0;
  for (int i = 2; i <= p - 2; ++i) {
    d = d * (t - b->gl[i]) + v;
    v *= t - b->gl[i];
  }
  *w = v;
  *dw = d;
}

static double herm_left(const basis1d *b, int j, double t, int deriv) {
  /* phi_0 (j = 0) or phi_1 (j = 1) */
  double w, dw, w0, dw0;
  herm_w(b, t, &w, &dw);
  herm_w(b, 0.0, &w0, &dw0);
  double u = 1.0 - t;
  if (j == 0) {
    double c = 2.0 - dw0 / w0;
    double A = u * u, dA = -2.0 * u, B = 1.0 + c * t, dB = c;
    return deriv ? (dA * B * w + A * dB * w + A * B * dw) / w0 : A * B * w / w0;
  }
  double x1 = b->gl[1], w1, dw1;
  herm_w(b, x1, &w1, &dw1);
  double sc = 1.0 / (x1 * (1.0 - x1) * (1.0 - x1) * w1);
  double g = t * u * u, dg = u * u - 2.0 * t * u;
  return sc * (deriv ? dg * w + g * dw : g * w);
}

static double herm_value(const basis1d *b, int j, double t, int deriv) {
  int p = b->k - 1;
  if (j <= 1) return herm_left(b, j, t, deriv);
  if (j >= p - 1) return deriv ? -herm_left(b, p - j, 1.0 - t, 1) : herm_left(b, p - j, 1.0 - t, 0);
  double u = 1.0 - t, xj = b->gl[j];
  double g = t * t * u * u, dg = 2.0 * t * u * u - 2.0 * t * t * u;
  double l = or_lagrange(p - 3, b->gl + 2, j - 2, t), dl = or_lagrange_deriv(p - 3, b->gl + 2, j - 2, t);
  double sc = 1.0 / (xj * xj * (1.0 - xj) * (1.0 - xj));
  return sc * (deriv ? dg * l + g * dl : g * l);
}

/* 1D basis function j of the basis at t (or its derivative). */
static double basis1(const basis1d *b, int j, double t, int deriv) {
  if (b->kind == 1) return herm_value(b, j, t, deriv);
  return deriv ? or_lagrange_deriv(b->k, b->gl, j, t) : or_lagrange(b->k, b->gl, j, t);
}

/* Point x and the Jacobian used by the cell integral at the Gauss point
 * (q0, q1, q2) of cell c.  Analytic (cell_map), or for variant G2 (Sec. 5:
 * positions of the quadrature points stored, the Jacobian computed by a
 * collocation derivative): column d of J is the derivative along xi_d of
 * the polynomial interpolating the physical positions of the k Gauss points
 * on the line through the point, J[i][d] = sum_j l_j'(g_{q_d}) x_i(.., g_j,
 * ..), with l_j the Lagrange polynomials on the Gauss points. */
static void cell_point(const or_mesh *m, const basis1d *b, int64_t c, const int q[3], double x[3], double J[3][3]) {
  double xi[3] = {b->gq[q[0]], b->gq[q[1]], b->gq[q[2]]};
  cell_map(m, c, xi, x, J);
  if (m->cell_jacobian != 1) return;
  int k = b->k;
  for (int d = 0; d < 3; ++d) {
    double col[3] = {0.0, 0.0, 0.0};
    for (int j = 0; j < k; ++j) {
      double xj[3] = {xi[0], xi[1], xi[2]}, pj[3], Jj[3][3];
      xj[d] = b->gq[j];
      cell_map(m, c, xj, pj, Jj);
      double dl = or_lagrange_deriv(k, b->gq, j, xi[d]);
      for (int i = 0; i < 3; ++i) col[i] += dl * pj[i];
    }
    for (int i = 0; i < 3; ++i) J[i][d] = col[i];
  }
}

/* Values and reference gradients of all k^3 tensor basis functions
 * phi_{i0 i1 i2}(xi) = l_{i0}(xi_0) l_{i1}(xi_1) l_{i2}(xi_2) at xi. */
static void basis_at(const basis1d *b, const double xi[3], double *val, double (*grad)[3]) {
  int k = b->k;
  double l[3][OR_MAXK], dl[3][OR_MAXK];
  for (int d = 0; d < 3; ++d)
    for (int j = 0; j < k; ++j) {
      l[d][j] = basis1(b, j, xi[d], 0);
      dl[d][j] = basis1(b, j, xi[d], 1);
    }
  for (int i2 = 0; i2 < k; ++i2)
    for (int i1 = 0; i1 < k; ++i1)
      for (int i0 = 0; i0 < k; ++i0) {
        int i = i0 + k * (i1 + k * i2);
        val[i] = l[0][i0] * l[1][i1] * l[2][i2];
        grad[i][0] = dl[0][i0] * l[1][i1] * l[2][i2];
        grad[i][1] = l[0][i0] * dl[1][i1] * l[2][i2];
        grad[i][2] = l[0][i0] * l[1][i1] * dl[2][i2];
      }
}

/* Physical gradients grad_x phi = J^{-T} grad_xi phi. */
static void to_physical(int nb, const double Jinv[3][3], double (*gref)[3], double (*gx)[3]) {
  for (int i = 0; i < nb; ++i)
    for (int a = 0; a < 3; ++a)
      gx[i][a] = Jinv[0][a] * gref[i][0] + Jinv[1][a] * gref[i][1] + Jinv[2][a] * gref[i][2];
}

/* |K| by the cell's k-point Gauss rule of det J. */
double or_cell_volume(const or_mesh *m, int degree, int64_t c) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1.0;
  int k = b.k;
  double vol = 0.0;
  for (int q2 = 0; q2 < k; ++q2)
    for (int q1 = 0; q1 < k; ++q1)
      for (int q0 = 0; q0 < k; ++q0) {
        double xi[3] = {b.gq[q0], b.gq[q1], b.gq[q2]}, x[3], J[3][3];
        cell_map(m, c, xi, x, J);
        vol += det3(J) * b.gw[q0] * b.gw[q1] * b.gw[q2];
      }
  return vol;
}

/* Face quadrature point (a,b) on face (d, side s) of cell c: tangential
 * directions t1 < t2 carry the Gauss points, xi_d = s. Returns the physical
 * point, J^{-1}, the outward unit normal n and the weighted area element
 * da*w = det J |J^{-T} nhat| w_a w_b (Nanson's formula). */
typedef struct {
  double x[3], Jinv[3][3], n[3], daw, detJ;
  double xi[3];
} facepoint;

static void face_point(const or_mesh *m, const basis1d *b, int64_t c, int d, int s, int qa, int qb,
                       facepoint *fp) {
  int t1 = (d == 0) ? 1 : 0, t2 = (d == 2) ? 1 : 2;
  fp->xi[d] = s ? 1.0 : 0.0;
  fp->xi[t1] = b->gq[qa];
  fp->xi[t2] = b->gq[qb];
  double J[3][3];
  cell_map(m, c, fp->xi, fp->x, J);
  fp->detJ = det3(J);
  inv3(J, fp->detJ, fp->Jinv);
  double sg = s ? 1.0 : -1.0, v[3], nv = 0.0;
  for (int a = 0; a < 3; ++a) {  /* (J^{-T} nhat)_a = sum_b Jinv[b][a] nhat_b */
    v[a] = sg * fp->Jinv[d][a];
    nv += v[a] * v[a];
  }
  nv = sqrt(nv);
  for (int a = 0; a < 3; ++a) fp->n[a] = v[a] / nv;
  fp->daw = fabs(fp->detJ) * nv * b->gw[qa] * b->gw[qb];
}

/* A_F by the k x k Gauss rule on face (d, s) of cell c. */
static double face_area(const or_mesh *m, const basis1d *b, int64_t c, int d, int s) {
  double A = 0.0;
  for (int qb = 0; qb < b->k; ++qb)
    for (int qa = 0; qa < b->k; ++qa) {
      facepoint fp;
      face_point(m, b, c, d, s, qa, qb, &fp);
      A += fp.daw;
    }
  return A;
}

/* Penalty of face (d, s) of cell c; the area is always taken from the cell
 * on the lower side of the face so both sides see the same number. */
static double face_penalty(const or_mesh *m, const basis1d *b, const or_form *f, int64_t c, int d, int s) {
  int p = b->k - 1;
  double scale = (double)(p + 1) * (p + 1) * f->penalty_scale;
  int64_t nb = neighbour(m, c, d, s);
  if (nb < 0) {
    return scale * face_area(m, b, c, d, s) / or_cell_volume(m, p, c);
  }
  int64_t lo = s ? c : nb, hi = s ? nb : c;
  double A = face_area(m, b, lo, d, 1);
  double r1 = A / or_cell_volume(m, p, lo), r2 = A / or_cell_volume(m, p, hi);
  return scale * (r1 > r2 ? r1 : r2);
}

/* ------------------------------------------------------------------ */
/* R2: unassembled apply, cell by cell                                  */
/* ------------------------------------------------------------------ */

/* Contributions tested on cell c only: the cell integral plus the six face
 * integrals with the test function restricted to c (Algorithm 1 steps (ii)-(iv)
 * regrouped by test cell).  y[c k^3 + i] is set. */
static void apply_one_cell(const or_mesh *m, const basis1d *b, const or_form *f, const double *u,
                           double *y, int64_t c, double *val, double (*gref)[3], double (*gx)[3],
                           double *val2, double (*gx2)[3]) {
  int k = b->k, nb3 = k * k * k;
  double yl[OR_MAXK * OR_MAXK * OR_MAXK];
  memset(yl, 0, sizeof(double) * nb3);
  const double *uc = u + c * nb3;

  /* cell integral (steps (ii)(a)-(e)) */
  for (int q2 = 0; q2 < k; ++q2)
    for (int q1 = 0; q1 < k; ++q1)
      for (int q0 = 0; q0 < k; ++q0) {
        double xi[3] = {b->gq[q0], b->gq[q1], b->gq[q2]}, x[3], J[3][3], Ji[3][3];
        int q[3] = {q0, q1, q2};
        cell_point(m, b, c, q, x, J);
        double detJ = det3(J);
        inv3(J, detJ, Ji);
        double jxw = detJ * b->gw[q0] * b->gw[q1] * b->gw[q2];
        basis_at(b, xi, val, gref);
        to_physical(nb3, Ji, gref, gx);
        if (f->op == 0) {
          double g[3] = {0, 0, 0};
          for (int j = 0; j < nb3; ++j)
            for (int a = 0; a < 3; ++a) g[a] += uc[j] * gx[j][a];
          double kap = kappa_at(f, x) * jxw;
          for (int i = 0; i < nb3; ++i)
            yl[i] += kap * (gx[i][0] * g[0] + gx[i][1] * g[1] + gx[i][2] * g[2]);
        } else {
          double uq = 0.0;
          for (int j = 0; j < nb3; ++j) uq += uc[j] * val[j];
          const double *cv = f->velocity;
          for (int i = 0; i < nb3; ++i)
            yl[i] -= jxw * uq * (gx[i][0] * cv[0] + gx[i][1] * cv[1] + gx[i][2] * cv[2]);
        }
      }

  /* face integrals of the six faces, test function on this cell */
  for (int d = 0; d < 3; ++d)
    for (int s = 0; s < 2; ++s) {
      int64_t nbc = neighbour(m, c, d, s);
      double tau = (f->op == 0) ? face_penalty(m, b, f, c, d, s) : 0.0;
      const double *un = (nbc >= 0) ? u + nbc * nb3 : NULL;
      for (int qb = 0; qb < k; ++qb)
        for (int qa = 0; qa < k; ++qa) {
          facepoint fo, fn;
          face_point(m, b, c, d, s, qa, qb, &fo);
          basis_at(b, fo.xi, val, gref);
          to_physical(nb3, fo.Jinv, gref, gx);
          double um = 0.0, dnm = 0.0;
          for (int j = 0; j < nb3; ++j) {
            um += uc[j] * val[j];
            dnm += uc[j] * (gx[j][0] * fo.n[0] + gx[j][1] * fo.n[1] + gx[j][2] * fo.n[2]);
          }
          double up = 0.0, dnp = 0.0;
          if (un) {
            face_point(m, b, nbc, d, 1 - s, qa, qb, &fn);
            basis_at(b, fn.xi, val2, gref);
            to_physical(nb3, fn.Jinv, gref, gx2);
            for (int j = 0; j < nb3; ++j) {
              up += un[j] * val2[j];
              dnp += un[j] * (gx2[j][0] * fo.n[0] + gx2[j][1] * fo.n[1] + gx2[j][2] * fo.n[2]);
            }
          }
          double tv, tg;
          if (f->op == 0) {
            double kw = kappa_at(f, fo.x) * fo.daw;
            if (un) {
              double jump = um - up, avg = 0.5 * (dnm + dnp);
              tv = kw * (tau * jump - avg);
              tg = -0.5 * kw * jump;
            } else {
              tv = kw * (2.0 * tau * um - dnm);
              tg = -kw * um;
            }
          } else {
            const double *cv = f->velocity;
            double cn = cv[0] * fo.n[0] + cv[1] * fo.n[1] + cv[2] * fo.n[2];
            if (un) tv = fo.daw * (0.5 * cn * (um + up) + 0.5 * fabs(cn) * (um - up));
            else tv = fo.daw * fabs(cn) * um;
            tg = 0.0;
          }
          for (int i = 0; i < nb3; ++i) {
            double dni = gx[i][0] * fo.n[0] + gx[i][1] * fo.n[1] + gx[i][2] * fo.n[2];
            yl[i] += tv * val[i] + tg * dni;
          }
        }
    }
  for (int i = 0; i < nb3; ++i) y[c * nb3 + i] = yl[i];
}

/* y = A u restricted to the rows of the listed cells (all cells if cells is
 * NULL).  Returns 0 on success. */
int or_apply_cells(const or_mesh *m, int degree, const or_form *f, const double *u, double *y,
                   const int64_t *cells, int64_t ncells) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1;
  int64_t nc = cells ? ncells : n_cells(m);
  int nb3 = b.k * b.k * b.k;
  int err = 0;
#pragma omp parallel
  {
    double *val = (double *)malloc(sizeof(double) * nb3 * 2);
    double(*gref)[3] = malloc(sizeof(double) * 3 * nb3);
    double(*gx)[3] = malloc(sizeof(double) * 3 * nb3);
    double(*gx2)[3] = malloc(sizeof(double) * 3 * nb3);
    if (!val || !gref || !gx || !gx2) {
#pragma omp atomic write
      err = 1;
    } else {
#pragma omp for schedule(dynamic, 4)
      for (int64_t i = 0; i < nc; ++i) {
        int64_t c = cells ? cells[i] : i;
        apply_one_cell(m, &b, f, u, y, c, val, gref, gx, val + nb3, gx2);
      }
    }
    free(val); free(gref); free(gx); free(gx2);
  }
  return err ? -2 : 0;
}

/* ------------------------------------------------------------------ */
/* R1: assembled matrix (cell loop + loop over unique faces)            */
/* ------------------------------------------------------------------ */

typedef struct {
  int64_t cells[7];
  int nblk;
} blockrow;

static double *block_of(blockrow *br, double *blocks, int64_t row_cell, int64_t col_cell, int nb3) {
  blockrow *r = &br[row_cell];
  for (int i = 0; i < r->nblk; ++i)
    if (r->cells[i] == col_cell) return blocks + ((row_cell * 7 + i) * (int64_t)nb3 * nb3);
  return NULL;
}

/* Number of stored entries of the assembled matrix. */
int64_t or_assemble_nnz(const or_mesh *m, int degree) {
  int k = degree + 1;
  int64_t nb3 = (int64_t)k * k * k, tot = 0;
  for (int64_t c = 0; c < n_cells(m); ++c) {
    int64_t list[7];
    int n = 0;
    list[n++] = c;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int64_t nb = neighbour(m, c, d, s);
        if (nb < 0) continue;
        int dup = 0;
        for (int i = 0; i < n; ++i) dup |= (list[i] == nb);
        if (!dup) list[n++] = nb;
      }
    tot += n * nb3 * nb3;
  }
  return tot;
}

/* Assemble A into CSR (rowptr[n+1], col[nnz], val[nnz]); column indices of
 * each row ascending.  Returns nnz, or a negative value on error. */
int64_t or_assemble(const or_mesh *m, int degree, const or_form *f, int64_t *rowptr, int32_t *col,
                    double *valout) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1;
  int k = b.k, nb3 = k * k * k;
  int64_t nc = n_cells(m);
  blockrow *br = (blockrow *)calloc(nc, sizeof(blockrow));
  double *blocks = (double *)calloc((size_t)nc * 7 * nb3 * nb3, sizeof(double));
  if (!br || !blocks) { free(br); free(blocks); return -2; }
  for (int64_t c = 0; c < nc; ++c) {
    blockrow *r = &br[c];
    r->cells[r->nblk++] = c;
    for (int d = 0; d < 3; ++d)
      for (int s = 0; s < 2; ++s) {
        int64_t nb = neighbour(m, c, d, s);
        if (nb < 0) continue;
        int dup = 0;
        for (int i = 0; i < r->nblk; ++i) dup |= (r->cells[i] == nb);
        if (!dup) r->cells[r->nblk++] = nb;
      }
    /* ascending cell order so that the CSR columns come out sorted */
    for (int i = 1; i < r->nblk; ++i)
      for (int j = i; j > 0 && r->cells[j - 1] > r->cells[j]; --j) {
        int64_t t = r->cells[j]; r->cells[j] = r->cells[j - 1]; r->cells[j - 1] = t;
      }
  }

  /* cell integrals */
#pragma omp parallel
  {
    double *val = malloc(sizeof(double) * nb3);
    double(*gref)[3] = malloc(sizeof(double) * 3 * nb3);
    double(*gx)[3] = malloc(sizeof(double) * 3 * nb3);
#pragma omp for schedule(dynamic, 1)
    for (int64_t c = 0; c < nc; ++c) {
      double *B = block_of(br, blocks, c, c, nb3);
      for (int q2 = 0; q2 < k; ++q2)
        for (int q1 = 0; q1 < k; ++q1)
          for (int q0 = 0; q0 < k; ++q0) {
            double xi[3] = {b.gq[q0], b.gq[q1], b.gq[q2]}, x[3], J[3][3], Ji[3][3];
            int q[3] = {q0, q1, q2};
            cell_point(m, &b, c, q, x, J);
            double detJ = det3(J);
            inv3(J, detJ, Ji);
            double jxw = detJ * b.gw[q0] * b.gw[q1] * b.gw[q2];
            basis_at(&b, xi, val, gref);
            to_physical(nb3, Ji, gref, gx);
            double kap = kappa_at(f, x) * jxw;
            const double *cv = f->velocity;
            for (int i = 0; i < nb3; ++i)
              for (int j = 0; j < nb3; ++j) {
                double e;
                if (f->op == 0)
                  e = kap * (gx[i][0] * gx[j][0] + gx[i][1] * gx[j][1] + gx[i][2] * gx[j][2]);
                else
                  e = -jxw * val[j] * (gx[i][0] * cv[0] + gx[i][1] * cv[1] + gx[i][2] * cv[2]);
                B[(int64_t)i * nb3 + j] += e;
              }
          }
    }
    free(val); free(gref); free(gx);
  }

  /* unique faces: for direction d, the face at the upper side of cell c;
   * plus the Dirichlet faces at the lower domain end.  Serial over faces
   * because blocks of neighbouring faces overlap. */
  double *vm = malloc(sizeof(double) * nb3), *vp = malloc(sizeof(double) * nb3);
  double(*gr)[3] = malloc(sizeof(double) * 3 * nb3);
  double(*gm)[3] = malloc(sizeof(double) * 3 * nb3), (*gp)[3] = malloc(sizeof(double) * 3 * nb3);
  double *dnm = malloc(sizeof(double) * nb3), *dnp = malloc(sizeof(double) * nb3);
  for (int64_t c = 0; c < nc; ++c)
    for (int d = 0; d < 3; ++d)
      for (int side = 0; side < 2; ++side) {
        int ijk[3];
        cell_ijk(m, c, ijk);
        int64_t nb = neighbour(m, c, d, side);
        if (side == 0 && nb >= 0) continue;  /* interior faces visited from the lower cell */
        int interior = nb >= 0;
        double tau = (f->op == 0) ? face_penalty(m, &b, f, c, d, side) : 0.0;
        for (int qb = 0; qb < k; ++qb)
          for (int qa = 0; qa < k; ++qa) {
            facepoint fo, fn;
            face_point(m, &b, c, d, side, qa, qb, &fo);
            basis_at(&b, fo.xi, vm, gr);
            to_physical(nb3, fo.Jinv, gr, gm);
            for (int i = 0; i < nb3; ++i)
              dnm[i] = gm[i][0] * fo.n[0] + gm[i][1] * fo.n[1] + gm[i][2] * fo.n[2];
            if (!interior) {
              double *B = block_of(br, blocks, c, c, nb3);
              for (int i = 0; i < nb3; ++i)
                for (int j = 0; j < nb3; ++j) {
                  double e;
                  if (f->op == 0) {
                    double kw = kappa_at(f, fo.x) * fo.daw;
                    e = kw * (-dnm[i] * vm[j] - vm[i] * dnm[j] + 2.0 * tau * vm[i] * vm[j]);
                  } else {
                    const double *cv = f->velocity;
                    double cn = cv[0] * fo.n[0] + cv[1] * fo.n[1] + cv[2] * fo.n[2];
                    e = fo.daw * fabs(cn) * vm[i] * vm[j];
                  }
                  B[(int64_t)i * nb3 + j] += e;
                }
              continue;
            }
            face_point(m, &b, nb, d, 0, qa, qb, &fn);
            basis_at(&b, fn.xi, vp, gr);
            to_physical(nb3, fn.Jinv, gr, gp);
            for (int i = 0; i < nb3; ++i)  /* n = n^- (outward normal of the lower cell) */
              dnp[i] = gp[i][0] * fo.n[0] + gp[i][1] * fo.n[1] + gp[i][2] * fo.n[2];
            /* blocks (row side, column side); sigma = +1 on the - side, -1 on the + side */
            for (int rs = 0; rs < 2; ++rs)
              for (int cs = 0; cs < 2; ++cs) {
                int64_t rc = rs ? nb : c, cc = cs ? nb : c;
                double *B = block_of(br, blocks, rc, cc, nb3);
                double si = rs ? -1.0 : 1.0, sj = cs ? -1.0 : 1.0;
                const double *vi = rs ? vp : vm, *vj = cs ? vp : vm;
                const double *di = rs ? dnp : dnm, *dj = cs ? dnp : dnm;
                for (int i = 0; i < nb3; ++i)
                  for (int j = 0; j < nb3; ++j) {
                    double e;
                    if (f->op == 0) {
                      double kw = kappa_at(f, fo.x) * fo.daw;
                      e = kw * (-0.5 * di[i] * sj * vj[j] - si * vi[i] * 0.5 * dj[j] +
                                tau * si * sj * vi[i] * vj[j]);
                    } else {
                      const double *cv = f->velocity;
                      double cn = cv[0] * fo.n[0] + cv[1] * fo.n[1] + cv[2] * fo.n[2];
                      e = fo.daw * si * vi[i] * vj[j] * 0.5 * (cn + sj * fabs(cn));
                    }
                    B[(int64_t)i * nb3 + j] += e;
                  }
              }
          }
      }
  free(vm); free(vp); free(gr); free(gm); free(gp); free(dnm); free(dnp);

  /* CSR */
  int64_t pos = 0;
  for (int64_t c = 0; c < nc; ++c) {
    blockrow *r = &br[c];
    for (int i = 0; i < nb3; ++i) {
      rowptr[c * nb3 + i] = pos;
      for (int bl = 0; bl < r->nblk; ++bl) {
        const double *B = blocks + ((c * 7 + bl) * (int64_t)nb3 * nb3);
        for (int j = 0; j < nb3; ++j) {
          col[pos] = (int32_t)(r->cells[bl] * nb3 + j);
          valout[pos] = B[(int64_t)i * nb3 + j];
          ++pos;
        }
      }
    }
  }
  rowptr[nc * nb3] = pos;
  free(br);
  free(blocks);
  return pos;
}

/* y = A x for a CSR matrix, fixed summation order. */
void or_spmv(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, const double *x,
             double *y) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t p = rowptr[i]; p < rowptr[i + 1]; ++p) s += val[p] * x[col[p]];
    y[i] = s;
  }
}

/* Conjugate gradients on a CSR matrix; x holds the initial guess. */
int or_cg_csr(int64_t n, const int64_t *rowptr, const int32_t *col, const double *val, const double *rhs,
              double *x, double rtol, int maxit, int *iters, double *relres) {
  double *r = malloc(sizeof(double) * n), *p = malloc(sizeof(double) * n), *ap = malloc(sizeof(double) * n);
  if (!r || !p || !ap) { free(r); free(p); free(ap); return -2; }
  or_spmv(n, rowptr, col, val, x, ap);
  double bb = 0.0, rr = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    r[i] = rhs[i] - ap[i];
    p[i] = r[i];
    bb += rhs[i] * rhs[i];
    rr += r[i] * r[i];
  }
  double bn = sqrt(bb > 0 ? bb : 1.0);
  int it = 0;
  while (it < maxit && sqrt(rr) > rtol * bn) {
    or_spmv(n, rowptr, col, val, p, ap);
    double pap = 0.0;
    for (int64_t i = 0; i < n; ++i) pap += p[i] * ap[i];
    double alpha = rr / pap, rr_new = 0.0;
    for (int64_t i = 0; i < n; ++i) {
      x[i] += alpha * p[i];
      r[i] -= alpha * ap[i];
      rr_new += r[i] * r[i];
    }
    double beta = rr_new / rr;
    rr = rr_new;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    ++it;
  }
  *iters = it;
  *relres = sqrt(rr) / bn;
  free(r); free(p); free(ap);
  return sqrt(rr) <= rtol * bn ? 0 : 1;
}

/* ------------------------------------------------------------------ */
/* Mass matrix, right-hand side, L2 error, dof points                   */
/* ------------------------------------------------------------------ */

/* y = M u with M_ij = (phi_i, phi_j) by the k-point Gauss rule (the
 * interpolate / JxW / integrate sequence of Sec. 3.1, evaluated directly). */
int or_mass_apply(const or_mesh *m, int degree, const double *u, double *y) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1;
  int k = b.k, nb3 = k * k * k;
  int64_t nc = n_cells(m);
#pragma omp parallel
  {
    double *val = malloc(sizeof(double) * nb3);
    double(*gref)[3] = malloc(sizeof(double) * 3 * nb3);
#pragma omp for
    for (int64_t c = 0; c < nc; ++c) {
      double yl[OR_MAXK * OR_MAXK * OR_MAXK];
      memset(yl, 0, sizeof(double) * nb3);
      for (int q2 = 0; q2 < k; ++q2)
        for (int q1 = 0; q1 < k; ++q1)
          for (int q0 = 0; q0 < k; ++q0) {
            double xi[3] = {b.gq[q0], b.gq[q1], b.gq[q2]}, x[3], J[3][3];
            cell_map(m, c, xi, x, J);
            double jxw = det3(J) * b.gw[q0] * b.gw[q1] * b.gw[q2];
            basis_at(&b, xi, val, gref);
            double uq = 0.0;
            for (int j = 0; j < nb3; ++j) uq += u[c * nb3 + j] * val[j];
            for (int i = 0; i < nb3; ++i) yl[i] += jxw * uq * val[i];
          }
      for (int i = 0; i < nb3; ++i) y[c * nb3 + i] = yl[i];
    }
    free(val); free(gref);
  }
  return 0;
}

/* Manufactured data: u = sin(pi x) sin(pi y) sin(pi z).
 * which = 0: f = -Lap u = 3 pi^2 u;  which = 1: f = -div(kappa grad u) with
 * kappa = 1 + 0.5 sin(2 pi x_0). */
static double exact_u(const double x[3]) {
  return sin(OR_PI * x[0]) * sin(OR_PI * x[1]) * sin(OR_PI * x[2]);
}
static double rhs_f(int which, const double x[3]) {
  double s = exact_u(x);
  if (which == 0) return 3.0 * OR_PI * OR_PI * s;
  double kap = 1.0 + 0.5 * sin(2.0 * OR_PI * x[0]);
  double dkap = OR_PI * cos(2.0 * OR_PI * x[0]);
  double dux = OR_PI * cos(OR_PI * x[0]) * sin(OR_PI * x[1]) * sin(OR_PI * x[2]);
  return 3.0 * OR_PI * OR_PI * kap * s - dkap * dux;
}

/* rhs_i = (phi_i, f) with the (k+2)-point Gauss rule per direction. */
int or_rhs(const or_mesh *m, int degree, int which, double *rhs) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1;
  int k = b.k, nb3 = k * k * k, kq = k + 2;
  double gq[OR_MAXK + 2], gw[OR_MAXK + 2];
  or_gauss(kq, gq, gw);
  int64_t nc = n_cells(m);
#pragma omp parallel
  {
    double *val = malloc(sizeof(double) * nb3);
    double(*gref)[3] = malloc(sizeof(double) * 3 * nb3);
#pragma omp for
    for (int64_t c = 0; c < nc; ++c) {
      double yl[OR_MAXK * OR_MAXK * OR_MAXK];
      memset(yl, 0, sizeof(double) * nb3);
      for (int q2 = 0; q2 < kq; ++q2)
        for (int q1 = 0; q1 < kq; ++q1)
          for (int q0 = 0; q0 < kq; ++q0) {
            double xi[3] = {gq[q0], gq[q1], gq[q2]}, x[3], J[3][3];
            cell_map(m, c, xi, x, J);
            double jxw = det3(J) * gw[q0] * gw[q1] * gw[q2];
            basis_at(&b, xi, val, gref);
            double fv = rhs_f(which, x) * jxw;
            for (int i = 0; i < nb3; ++i) yl[i] += fv * val[i];
          }
      for (int i = 0; i < nb3; ++i) rhs[c * nb3 + i] = yl[i];
    }
    free(val); free(gref);
  }
  return 0;
}

/* ||u_h - u||_{L2} with the (k+2)-point Gauss rule. */
double or_l2_error(const or_mesh *m, int degree, const double *u) {
  basis1d b;
  if (basis_init(&b, degree, m->basis)) return -1.0;
  int k = b.k, nb3 = k * k * k, kq = k + 2;
  double gq[OR_MAXK + 2], gw[OR_MAXK + 2];
  or_gauss(kq, gq, gw);
  int64_t nc = n_cells(m);
  double err = 0.0;
#pragma omp parallel reduction(+ : err)
  {
    double *val = malloc(sizeof(double) * nb3);
    double(*gref)[3] = malloc(sizeof(double) * 3 * nb3);
#pragma omp for
    for (int64_t c = 0; c < nc; ++c)
      for (int q2 = 0; q2 < kq; ++q2)
        for (int q1 = 0; q1 < kq; ++q1)
          for (int q0 = 0; q0 < kq; ++q0) {
            double xi[3] = {gq[q0], gq[q1], gq[q2]}, x[3], J[3][3];
            cell_map(m, c, xi, x, J);
            double jxw = det3(J) * gw[q0] * gw[q1] * gw[q2];
            basis_at(&b, xi, val, gref);
            double uh = 0.0;
            for (int j = 0; j < nb3; ++j) uh += u[c * nb3 + j] * val[j];
            double e = uh - exact_u(x);
            err += e * e * jxw;
          }
    free(val); free(gref);
  }
  return sqrt(err);
}

/* Value (deriv = 0) or derivative (deriv = 1) of 1D basis function j of the
 * given kind (0 Gauss-Lobatto Lagrange, 1 Hermite-like) and degree at t;
 * NaN for an invalid degree. */
double or_basis_value(int kind, int degree, int j, double t, int deriv) {
  basis1d b;
  if (basis_init(&b, degree, kind) || j < 0 || j > degree) return NAN;
  return basis1(&b, j, t, deriv);
}

/* Physical coordinates of every dof (images of the GL nodes), xyz[3 i + d]. */
int or_dof_points(const or_mesh *m, int degree, double *xyz) {
  basis1d b;
  if (m->basis != 0) return -1;  /* the Hermite-like basis is not nodal */
  if (basis_init(&b, degree, m->basis)) return -1;
  int k = b.k, nb3 = k * k * k;
  int64_t nc = n_cells(m);
  for (int64_t c = 0; c < nc; ++c)
    for (int i2 = 0; i2 < k; ++i2)
      for (int i1 = 0; i1 < k; ++i1)
        for (int i0 = 0; i0 < k; ++i0) {
          double xi[3] = {b.gl[i0], b.gl[i1], b.gl[i2]}, x[3], J[3][3];
          cell_map(m, c, xi, x, J);
          int64_t i = c * nb3 + i0 + k * (i1 + k * i2);
          for (int d = 0; d < 3; ++d) xyz[3 * i + d] = x[d];
        }
  return 0;
}

/* Number of OpenMP threads the oracle runs on. */
int or_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
