// C-ABI entry points of the GB300 DG operator library (declared in
// include/dg.h): operator set-up (1D tables, geometry), apply dispatch,
// right-hand side, and the conjugate-gradient solver with fused vector
// updates.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/dg.h"
#include "dg_df64.cuh"
#include "dg_internal.cuh"

using dg::df64;
using dg::kMaxK;

// ---------------------------------------------------------------------------
// 1D tables.  Gauss points from the eigenvalues of the Legendre Jacobi matrix
// (Golub-Welsch), interior Gauss-Lobatto points from the Jacobi matrix of the
// Jacobi polynomials P^{(1,1)}_{k-2}; Lagrange values and derivatives by the
// barycentric formulas.  (Sec. 2: tensor Gauss quadrature, nodal basis on
// the Gauss-Lobatto points; Sec. 3.1: S, D^co, S_f, D_f.)
// ---------------------------------------------------------------------------
namespace {

// Eigen-decomposition of a symmetric tridiagonal matrix (diagonal a, off-diagonal
// b) by cyclic Jacobi rotations on the dense matrix; returns eigenvalues and
// the first component of each normalized eigenvector.
void sym_tridiag_eig(int n, const double* a, const double* b, double* lam, double* v0) {
  std::vector<double> A(n * n, 0.0), V(n * n, 0.0);
  for (int i = 0; i < n; ++i) {
    A[i * n + i] = a[i];
    V[i * n + i] = 1.0;
    if (i + 1 < n) A[i * n + i + 1] = A[(i + 1) * n + i] = b[i];
  }
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[p * n + q] * A[p * n + q];
    if (off < 1e-34) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[p * n + q];
        if (std::fabs(apq) < 1e-300) continue;
        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {
          double akp = A[k * n + p], akq = A[k * n + q];
          A[k * n + p] = c * akp - s * akq;
          A[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          double apk = A[p * n + k], aqk = A[q * n + k];
          A[p * n + k] = c * apk - s * aqk;
          A[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) {
    lam[i] = A[i * n + i];
    v0[i] = V[0 * n + i];
  }
  // sort ascending
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && lam[j - 1] > lam[j]; --j) {
      std::swap(lam[j - 1], lam[j]);
      std::swap(v0[j - 1], v0[j]);
    }
}

// Polish a root of the Legendre-type polynomial given by its recurrence with
// Newton steps in long double.  f(t) evaluates the polynomial and derivative.
template <typename F>
double polish(double t0, F f) {
  long double t = t0;
  for (int it = 0; it < 6; ++it) {
    long double p, dp;
    f(t, p, dp);
    if (dp == 0) break;
    t -= p / dp;
  }
  return (double)t;
}

// Legendre P_n and P_n' by the three-term recurrence (long double).
void legendre_eval(int n, long double t, long double& p, long double& dp) {
  long double p0 = 1.0L, p1 = t, d0 = 0.0L, d1 = 1.0L;
  if (n == 0) { p = 1.0L; dp = 0.0L; return; }
  for (int j = 2; j <= n; ++j) {
    long double p2 = ((2 * j - 1) * t * p1 - (j - 1) * p0) / j;
    long double d2 = d0 + (2 * j - 1) * p1;  // P'_j = P'_{j-2} + (2j-1) P_{j-1}
    p0 = p1; p1 = p2; d0 = d1; d1 = d2;
  }
  p = p1;
  dp = d1;
}

void gauss_rule(int k, double* x, double* w) {
  std::vector<double> a(k, 0.0), b(k, 0.0), lam(k), v0(k);
  for (int j = 1; j < k; ++j) b[j - 1] = j / std::sqrt(4.0 * j * j - 1.0);
  sym_tridiag_eig(k, a.data(), b.data(), lam.data(), v0.data());
  for (int i = 0; i < k; ++i) {
    double t = polish(lam[i], [k](long double tt, long double& p, long double& dp) { legendre_eval(k, tt, p, dp); });
    long double p, dp;
    legendre_eval(k, t, p, dp);
    x[i] = 0.5 * (t + 1.0);
    w[i] = (double)(1.0L / ((1.0L - (long double)t * t) * dp * dp));  // 2/((1-t^2)P'^2) on [-1,1], halved
  }
}

void lobatto_nodes(int k, double* x) {
  x[0] = 0.0;
  x[k - 1] = 1.0;
  int n = k - 2;
  if (n <= 0) return;
  std::vector<double> a(n, 0.0), b(n, 0.0), lam(n), v0(n);
  for (int j = 1; j < n; ++j) b[j - 1] = std::sqrt((double)j * (j + 2) / ((2.0 * j + 1.0) * (2.0 * j + 3.0)));
  sym_tridiag_eig(n, a.data(), b.data(), lam.data(), v0.data());
  for (int i = 0; i < n; ++i) {
    // interior GL nodes are the roots of P'_{k-1}; polish with P'' from Legendre's equation
    double t = polish(lam[i], [k](long double tt, long double& p, long double& dp) {
      long double q, dq;
      legendre_eval(k - 1, tt, q, dq);
      p = dq;
      dp = (2.0L * tt * dq - (long double)(k - 1) * k * q) / (1.0L - tt * tt);
    });
    x[i + 1] = 0.5 * (t + 1.0);
  }
}

void bary_weights(int k, const double* x, double* lam) {
  for (int j = 0; j < k; ++j) {
    double p = 1.0;
    for (int m = 0; m < k; ++m)
      if (m != j) p *= (x[j] - x[m]);
    lam[j] = 1.0 / p;
  }
}

// values l_j(t) of the Lagrange polynomials on nodes x (second barycentric form)
void bary_values(int k, const double* x, const double* lam, double t, double* out) {
  for (int j = 0; j < k; ++j)
    if (t == x[j]) {
      for (int m = 0; m < k; ++m) out[m] = (m == j) ? 1.0 : 0.0;
      return;
    }
  double den = 0.0;
  for (int j = 0; j < k; ++j) den += lam[j] / (t - x[j]);
  for (int j = 0; j < k; ++j) out[j] = lam[j] / (t - x[j]) / den;
}

// differentiation matrix on the nodes: Dm[i][j] = l_j'(x_i)
void bary_diff_matrix(int k, const double* x, const double* lam, double* Dm) {
  for (int i = 0; i < k; ++i) {
    double diag = 0.0;
    for (int j = 0; j < k; ++j) {
      if (j == i) continue;
      double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      Dm[i * k + j] = v;
      diag -= v;
    }
    Dm[i * k + i] = diag;
  }
}

struct Tables64 {
  int basis;  // DG_BASIS_LAGRANGE or DG_BASIS_HERMITE
  double gq[kMaxK], gw[kMaxK], gl[kMaxK];
  double S[kMaxK * kMaxK], D[kMaxK * kMaxK], DS[kMaxK * kMaxK], E[2][kMaxK], DF[2][kMaxK];
  // the basis values at t = 0 and t = 1 are the unit vectors e_0 and e_p
  // (the face value is the end layer's coefficient: the face loop's forward
  // launch relies on it for the x faces)
  bool end_nodal;
};

// Hermite-like basis of degree p = k - 1 >= 3 on the Gauss-Lobatto points
// g_0 = 0 < g_1 < ... < g_p = 1, with w(t) = prod_{j=2}^{p-2} (t - g_j):
// f_0 = (1-t)^2 (1 + c t) w(t) / w(0) with c such that f_0'(0) = 0;
// f_1 = t (1-t)^2 w(t), scaled to f_1(g_1) = 1; f_j, 2 <= j <= p-2, =
// t^2 (1-t)^2 times the Lagrange polynomial on g_2 .. g_{p-2} that is 1 at
// g_j, scaled to f_j(g_j) = 1; f_{p-1}(t) = f_1(1-t), f_p(t) = f_0(1-t).
// Only f_0 is nonzero at t = 0 and only f_1 has a nonzero derivative there
// (mirror-symmetric at t = 1), so a face value and a face-normal derivative
// each come from one coefficient per face point (the Hermite-type property
// of Sec. 3.1); the interior nodes keep the basis close to the Lagrange one.
// val[j], der[j] at t.
void hermite_values(int k, const double* g, double t, double* val, double* der) {
  const int p = k - 1;
  // w and w' at t, 0 and g_1 (product rule over the factors)
  auto wfun = [&](double x, double& w, double& dw) {
    w = 1.0;
    dw = 0.0;
    for (int j = 2; j <= p - 2; ++j) {
      dw = dw * (x - g[j]) + w;
      w *= x - g[j];
    }
  };
  // f_0 and f_1 at x (value, derivative)
  auto left = [&](int which, double x, double& v, double& d) {
    double w, dw, w0, dw0;
    wfun(x, w, dw);
    wfun(0.0, w0, dw0);
    const double u = 1.0 - x;
    if (which == 0) {
      const double c = 2.0 - dw0 / w0;
      const double a = u * u / w0, da = -2.0 * u / w0, b = 1.0 + c * x;
      v = a * b * w;
      d = da * b * w + a * c * w + a * b * dw;
    } else {
      double w1, dw1;
      wfun(g[1], w1, dw1);
      const double sc = 1.0 / (g[1] * (1.0 - g[1]) * (1.0 - g[1]) * w1);
      const double h = x * u * u, dh = u * (u - 2.0 * x);
      v = sc * h * w;
      d = sc * (dh * w + h * dw);
    }
  };
  left(0, t, val[0], der[0]);
  left(1, t, val[1], der[1]);
  double v, d;
  left(1, 1.0 - t, v, d);
  val[p - 1] = v;
  der[p - 1] = -d;
  left(0, 1.0 - t, v, d);
  val[p] = v;
  der[p] = -d;
  const double u = 1.0 - t, b = t * t * u * u, db = 2.0 * t * u * (u - t);
  for (int j = 2; j <= p - 2; ++j) {
    double l = 1.0, dl = 0.0;
    for (int m = 2; m <= p - 2; ++m) {
      if (m == j) continue;
      const double f = 1.0 / (g[j] - g[m]);
      dl = dl * (t - g[m]) * f + l * f;
      l *= (t - g[m]) * f;
    }
    const double sc = 1.0 / (g[j] * g[j] * (1.0 - g[j]) * (1.0 - g[j]));
    val[j] = sc * b * l;
    der[j] = sc * (db * l + b * dl);
  }
}

// values of the k basis functions at t (and derivatives, if der)
void basis_values(const Tables64& t, int k, double x, double* val, double* der) {
  if (t.basis == DG_BASIS_HERMITE) {
    double d[kMaxK];
    hermite_values(k, t.gl, x, val, der ? der : d);
    return;
  }
  double ll[kMaxK];
  bary_weights(k, t.gl, ll);
  bary_values(k, t.gl, ll, x, val);
  if (der) {
    double DL[kMaxK * kMaxK];
    bary_diff_matrix(k, t.gl, ll, DL);
    // derivative at x of the interpolant: sum over the nodes of l_m(x) D_L[m][j]
    for (int j = 0; j < k; ++j) {
      double s = 0.0;
      for (int m = 0; m < k; ++m) s += val[m] * DL[m * k + j];
      der[j] = s;
    }
  }
}

void build_tables(int k, Tables64& t, int basis) {
  t.basis = basis;
  gauss_rule(k, t.gq, t.gw);
  lobatto_nodes(k, t.gl);
  double lg[kMaxK], ll[kMaxK];
  bary_weights(k, t.gq, lg);
  bary_weights(k, t.gl, ll);
  for (int q = 0; q < k; ++q) basis_values(t, k, t.gq[q], t.S + q * k, nullptr);
  bary_diff_matrix(k, t.gq, lg, t.D);
  // derivative of the GL basis at the Gauss points: the Gauss-collocation
  // derivative of its (exact) Gauss-point interpolant
  for (int q = 0; q < k; ++q)
    for (int i = 0; i < k; ++i) {
      double s = 0.0;
      for (int j = 0; j < k; ++j) s += t.D[q * k + j] * t.S[j * k + i];
      t.DS[q * k + i] = s;
    }
  bary_values(k, t.gq, lg, 0.0, t.E[0]);
  bary_values(k, t.gq, lg, 1.0, t.E[1]);
  double v0[kMaxK], v1[kMaxK];
  basis_values(t, k, 0.0, v0, t.DF[0]);
  basis_values(t, k, 1.0, v1, t.DF[1]);
  t.end_nodal = true;
  for (int i = 0; i < k; ++i)
    t.end_nodal = t.end_nodal && std::fabs(v0[i] - (i == 0 ? 1.0 : 0.0)) <= 1e-13 &&
                  std::fabs(v1[i] - (i == k - 1 ? 1.0 : 0.0)) <= 1e-13;
  (void)ll;
}

template <typename T>
dg::Tables<T> cast_tables(int k, const Tables64& t) {
  dg::Tables<T> o;
  memset(&o, 0, sizeof(o));
  for (int i = 0; i < k * k; ++i) {
    o.S[i] = (T)t.S[i];
    o.D[i] = (T)t.D[i];
    o.DS[i] = (T)t.DS[i];
  }
  for (int s = 0; s < 2; ++s)
    for (int i = 0; i < k; ++i) {
      o.E[s][i] = (T)t.E[s][i];
      o.DF[s][i] = (T)t.DF[s][i];
    }
  for (int i = 0; i < k; ++i) o.W[i] = (T)t.gw[i];
  o.slim = t.basis == DG_BASIS_HERMITE ? 1 : 0;
  // even-odd halves, from the FP64 tables
  const int h = k / 2, h2 = (k + 1) / 2;
  for (int m = 0; m < 5; ++m) {
    auto M = [&](int q, int i) {
      return m == dg::EO_S    ? t.S[q * k + i]
             : m == dg::EO_ST ? t.S[i * k + q]
             : m == dg::EO_D  ? t.D[q * k + i]
             : m == dg::EO_DT ? t.D[i * k + q]
                              : t.DS[q * k + i];
    };
    for (int q = 0; q < h2; ++q) {
      for (int i = 0; i < h; ++i) {
        o.EO[m][0][q * dg::kHalf + i] = (T)(0.5 * (M(q, i) + M(q, k - 1 - i)));
        o.EO[m][1][q * dg::kHalf + i] = (T)(0.5 * (M(q, i) - M(q, k - 1 - i)));
      }
      if (k % 2) o.EO[m][0][q * dg::kHalf + h] = (T)M(q, h);
    }
  }
  return o;
}

}  // namespace

// ---------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------
// slabs of the pipelined host-buffer apply
constexpr int kHostSlabs = 8;

struct dg_handle {
  dg_mesh mesh;
  dg_opts opts;
  int degree, k, geom, prec, op;
  int cpb;  // cells per block of the apply kernel
  int64_t n_cells, n_dofs;
  cudaStream_t stream;
  Tables64 t64;
  dg::Tables<double> tabd;
  dg::Tables<float> tabf;
  dg::Tables<df64> tabdf;
  dg::Geometry<double> geod;
  dg::Geometry<float> geof;
  dg::Geometry<df64> geodf;
  void* cell_geo;         // device: per-quadrature-point cell arrays
  void* face_geo[3];      // device: per-face-point arrays
  void* face_tau[3];      // device: penalty per face
  void* kappa_tab;        // device: Cartesian kappa tables
  int64_t cell_bytes, face_bytes;
  // CG work vectors (FP64) and reduction scratch
  double *r, *p, *ap;
  double* partial;        // per-block partials
  int64_t partial_len;
  double* scal;           // device scalars
  double* scal_host;      // host copy of the solver scalars (points into scal_buf)
  double scal_buf[16];
  cudaStream_t cg_stream;  // solver stream (non-blocking, capturable) and ordering event
  cudaEvent_t cg_event;
  double* xw;             // extra work vectors (inner solution and right-hand side of
  double* bw;             // the mixed-precision solve), allocated on first use
  // host-buffer apply staging, and the copy streams and events of its slab
  // pipeline (created on first use)
  void *stage_src, *stage_dst;
  // face evaluation of the binary64 / double-float apply (dg_set_face_mode)
  int face_mode;
  dg::SplitArrays split;
  const double* skip;     // device flag handed to the apply launches (null: never skip)
  cudaStream_t h2d_stream, d2h_stream, cmp_stream, bwd_stream[2];
  cudaEvent_t pipe_ev[3 * kHostSlabs + 2];
  std::string err;
};

namespace {

thread_local std::string g_setup_error;

dg_status fail(dg_handle* h, dg_status s, const std::string& msg) {
  if (h) h->err = msg;
  else g_setup_error = msg;
  return s;
}

dg_status cuda_fail(dg_handle* h, cudaError_t e, const char* what) {
  return fail(h, DG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Kernel geometry variant of a public dg_geom value.
int kernel_geo(int geom) {
  return geom == DG_GEOM_CARTESIAN  ? dg::GEO_CART
         : geom == DG_GEOM_FULL_JAC ? dg::GEO_FULL
         : geom == DG_GEOM_POSITIONS ? dg::GEO_POS
                                     : dg::GEO_MERGED;
}

#define DG_CUDA(h, call)                                   \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

// Device memory comes from the stream-ordered allocator (cudaMallocAsync on
// the handle's stream): unlike cudaMalloc/cudaFree it does not synchronize the
// device, so operators set up and torn down in one thread do not stall work
// running on other streams.
dg_status dev_alloc(dg_handle* h, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) return DG_OK;
  cudaError_t e = cudaMallocAsync(p, bytes, h->stream);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    *p = nullptr;
    return fail(h, DG_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "cudaMallocAsync");
  return DG_OK;
}

void dev_free(dg_handle* h, void* p) {
  if (p) cudaFreeAsync(p, h->stream);
}

// ---------------------------------------------------------------------------
// Geometry set-up kernels (FP64 arithmetic, stored as T)
// ---------------------------------------------------------------------------
struct SetupParams {
  int n[3];
  int periodic;
  int mapping;
  double amp;
  int k;
  int P[3];
  double gq[kMaxK], gw[kMaxK];
  int op, coeff, geom;
  double vel[3];
  double penalty;  // penalty_scale (p+1)^2
  int cblk;        // cell arrays: 0 = structure of arrays, else cell-blocked with this width
  int ncomp;       // number of cell arrays
  int fold;        // full Jacobians, SIPG, binary64 storage: sqrt(kappa JxW) folded into J^{-1}
  int face_minor;  // face arrays: 0 = [array][face][point]; 1 = blocks of kFaceBlock faces,
                   // [face block][array][point][face in block], faces numbered like cells
                   // (x fastest; the face position replaces the index along d)
  int nfa;         // number of face arrays
  int face_pair;   // binary32 SIPG: both sides' J^{-T} n (else one vector, see setup_face_geometry)
};

// Position of array m, face f (numbered pos + P_d (i_t1 + n_t1 i_t2)) and
// point q in the face arrays of direction d, for the layout selected by
// S.face_minor (nfq = faces x points, the array stride of the plain layout).
__device__ int64_t face_slot(const SetupParams& S, int d, int m, int64_t f, int q, int64_t nfq) {
  const int k2 = S.k * S.k;
  if (!S.face_minor) return m * nfq + f * k2 + q;
  const int64_t fm = dg::face_minor_id(S.n, S.P, d, f);
  constexpr int B = dg::kFaceBlock;
  return ((fm / B) * S.nfa * k2 + (int64_t)m * k2 + q) * B + fm % B;
}

// mapping 1: x = X + a s(X)(1,1,1), s = sin(pi X) sin(pi Y) sin(pi Z);
// mapping 2: the shear x_i = X_i + a X_{(i+1) mod 3}; J = dx/dxi includes 1/n_d
__device__ void map_point(const SetupParams& S, const int ijk[3], const double xi[3], double x[3], double J[9]) {
  double X[3];
  for (int d = 0; d < 3; ++d) X[d] = (ijk[d] + xi[d]) / S.n[d];
  if (S.mapping == 2) {
    for (int i = 0; i < 3; ++i) {
      const int i1 = (i + 1) % 3;
      x[i] = X[i] + S.amp * X[i1];
      for (int j = 0; j < 3; ++j) J[i * 3 + j] = ((i == j) + (j == i1 ? S.amp : 0.0)) / S.n[j];
    }
    return;
  }
  double grad[3] = {0.0, 0.0, 0.0}, sv = 0.0;
  if (S.mapping == 1) {
    double sn[3], cs[3];
    for (int d = 0; d < 3; ++d) sincospi(X[d], &sn[d], &cs[d]);
    sv = sn[0] * sn[1] * sn[2];
    grad[0] = M_PI * cs[0] * sn[1] * sn[2];
    grad[1] = M_PI * sn[0] * cs[1] * sn[2];
    grad[2] = M_PI * sn[0] * sn[1] * cs[2];
  }
  const double a = S.mapping == 1 ? S.amp : 0.0;
  for (int i = 0; i < 3; ++i) {
    x[i] = X[i] + a * sv;
    for (int j = 0; j < 3; ++j) J[i * 3 + j] = ((i == j) + a * grad[j]) / S.n[j];
  }
}

// inverse through the adjugate; returns det
__device__ double invert3(const double J[9], double Ji[9]) {
  const double c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
  const double det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  const double r = 1.0 / det;
  Ji[0] = c00 * r;
  Ji[3] = c01 * r;
  Ji[6] = c02 * r;
  Ji[1] = (J[2] * J[7] - J[1] * J[8]) * r;
  Ji[4] = (J[0] * J[8] - J[2] * J[6]) * r;
  Ji[7] = (J[1] * J[6] - J[0] * J[7]) * r;
  Ji[2] = (J[1] * J[5] - J[2] * J[4]) * r;
  Ji[5] = (J[2] * J[3] - J[0] * J[5]) * r;
  Ji[8] = (J[0] * J[4] - J[1] * J[3]) * r;
  return det;
}

__device__ double kappa_of(const SetupParams& S, const double x[3]) {
  return S.coeff == 1 ? 1.0 + 0.5 * sinpi(2.0 * x[0]) : 1.0;
}

__device__ void cell_of(const SetupParams& S, int64_t c, int ijk[3]) {
  ijk[0] = (int)(c % S.n[0]);
  ijk[1] = (int)((c / S.n[0]) % S.n[1]);
  ijk[2] = (int)(c / ((int64_t)S.n[0] * S.n[1]));
}

template <typename T>
__global__ void setup_cell_geometry(const SetupParams S, int64_t n_cells, T* out, int64_t ncq, double* vol_part,
                                    int* bad) {
  const int k = S.k, k3 = k * k * k;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_cells * k3;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = idx / k3;
    const int q = (int)(idx - c * k3);
    const int q0 = q % k, q1 = (q / k) % k, q2 = q / (k * k);
    int ijk[3];
    cell_of(S, c, ijk);
    const double xi[3] = {S.gq[q0], S.gq[q1], S.gq[q2]};
    double x[3], J[9], Ji[9];
    map_point(S, ijk, xi, x, J);
    const double det = invert3(J, Ji);
    if (!(det > 0.0)) atomicOr(bad, 1);
    const double jxw = det * S.gw[q0] * S.gw[q1] * S.gw[q2];
    vol_part[idx] = jxw;
    if (!out) continue;
    // element index of array m at this point
    auto at = [&](int m) -> int64_t {
      return S.cblk ? (((c / S.cblk) * S.ncomp + m) * (int64_t)k3 + q) * S.cblk + c % S.cblk : m * ncq + idx;
    };
    if (S.geom == dg::GEO_POS) {
      // G2: the point's position (the kernel differentiates them), and kappa
      for (int m = 0; m < 3; ++m) out[at(m)] = (T)x[m];
      if (S.op == dg::OP_SIPG) out[at(3)] = (T)kappa_of(S, x);
    } else if (S.geom == dg::GEO_FULL && S.fold) {
      // kappa JxW J^{-1} J^{-T} = (s J^{-1}) (s J^{-1})^T with s = sqrt(kappa JxW)
      const double sw = sqrt(kappa_of(S, x) * jxw);
      for (int m = 0; m < 9; ++m) out[at(m)] = (T)(sw * Ji[m]);
    } else if (S.geom == dg::GEO_FULL) {
      for (int m = 0; m < 9; ++m) out[at(m)] = (T)Ji[m];
      out[at(9)] = (T)(S.op == dg::OP_SIPG ? kappa_of(S, x) * jxw : jxw);
    } else if (S.op == dg::OP_SIPG) {
      const double kw = kappa_of(S, x) * jxw;
      const int ia[6] = {0, 0, 0, 1, 1, 2}, ib[6] = {0, 1, 2, 1, 2, 2};
      for (int m = 0; m < 6; ++m) {
        double g = 0.0;
        for (int c2 = 0; c2 < 3; ++c2) g += Ji[ia[m] * 3 + c2] * Ji[ib[m] * 3 + c2];
        out[at(m)] = (T)(kw * g);
      }
    } else {
      for (int a = 0; a < 3; ++a)
        out[at(a)] = (T)(-jxw * (Ji[a * 3 + 0] * S.vel[0] + Ji[a * 3 + 1] * S.vel[1] + Ji[a * 3 + 2] * S.vel[2]));
    }
  }
}

// per-cell volume from the per-point det J w values (fixed order)
__global__ void sum_cells(const double* part, int k3, int64_t n_cells, double* vol) {
  for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < n_cells; c += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < k3; ++q) s += part[c * k3 + q];
    vol[c] = s;
  }
}

// face (direction d) geometry: slot 0 = lower cell (its xi_d = 1), slot 1 = upper cell (xi_d = 0)
template <typename T>
__global__ void setup_face_geometry(const SetupParams S, int d, int64_t n_faces, T* out, int64_t nfq, double* daw_out,
                                    int* bad) {
  const int k = S.k, k2 = k * k;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < n_faces * k2;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t f = idx / k2;
    const int q = (int)(idx - f * k2);
    const int qa = q % k, qb = q / k;
    const int pos = (int)(f % S.P[d]);
    const int64_t rest = f / S.P[d];
    const int it1 = (int)(rest % S.n[t1]), it2 = (int)(rest / S.n[t1]);
    bool has[2];
    has[0] = S.periodic || pos >= 1;
    has[1] = S.periodic || pos < S.n[d];
    double jn[2][3] = {{0, 0, 0}, {0, 0, 0}}, nrm[2][3] = {{0, 0, 0}, {0, 0, 0}};
    double daw = 0.0, kap = 1.0;
    bool first = true;
    for (int slot = 0; slot < 2; ++slot) {
      if (!has[slot]) continue;
      int ijk[3];
      ijk[t1] = it1;
      ijk[t2] = it2;
      ijk[d] = slot == 0 ? (pos - 1 + S.n[d]) % S.n[d] : pos % S.n[d];
      double xi[3];
      xi[d] = slot == 0 ? 1.0 : 0.0;
      xi[t1] = S.gq[qa];
      xi[t2] = S.gq[qb];
      double x[3], J[9], Ji[9];
      map_point(S, ijk, xi, x, J);
      const double det = invert3(J, Ji);
      if (!(det > 0.0)) atomicOr(bad, 1);
      const double sg = slot == 0 ? 1.0 : -1.0;
      double v[3], len = 0.0;
      for (int a = 0; a < 3; ++a) {
        v[a] = sg * Ji[d * 3 + a];  // J^{-T} nhat
        len += v[a] * v[a];
      }
      len = sqrt(len);
      for (int a = 0; a < 3; ++a) nrm[slot][a] = v[a] / len;
      for (int a = 0; a < 3; ++a)
        jn[slot][a] = Ji[a * 3 + 0] * nrm[slot][0] + Ji[a * 3 + 1] * nrm[slot][1] + Ji[a * 3 + 2] * nrm[slot][2];
      if (first) {
        daw = det * len * S.gw[qa] * S.gw[qb];
        kap = kappa_of(S, x);
        first = false;
      }
    }
    daw_out[idx] = daw;
    auto at = [&](int m) { return face_slot(S, d, m, f, q, nfq); };
    if (S.op == dg::OP_SIPG && S.face_minor && !S.face_pair) {
      // one vector per face point: J^{-T} n for n = +e_d.  Inside the
      // domain the mapping is smooth, so both sides evaluate the same J at
      // the face and their vectors differ only in the normal's sign (slot 1
      // = -slot 0).  (Not across a periodic boundary of a deformed mesh,
      // where the sine mapping's derivative changes sign: face_pair.)
      for (int a = 0; a < 3; ++a) out[at(a)] = (T)(has[0] ? jn[0][a] : -jn[1][a]);
      out[at(3)] = (T)(kap * daw);
    } else if (S.op == dg::OP_SIPG) {
      // both sides' j_n and w = kappa da w; in binary64 storage the weight
      // is folded in: w j_n per side, and w, which setup_face_tau turns into
      // w tau (binary32 face_pair storage keeps j_n and w)
      const double w = kap * daw;
      const double sc = S.face_minor ? 1.0 : w;
      for (int slot = 0; slot < 2; ++slot)
        for (int a = 0; a < 3; ++a) out[at(slot * 3 + a)] = (T)(sc * jn[slot][a]);
      out[at(6)] = (T)w;
    } else {
      // c.n da w with n the normal pointing to +d (outward normal of the lower side)
      double n[3];
      for (int a = 0; a < 3; ++a) n[a] = has[0] ? nrm[0][a] : -nrm[1][a];
      out[at(0)] = (T)((S.vel[0] * n[0] + S.vel[1] * n[1] + S.vel[2] * n[2]) * daw);
    }
  }
}

__device__ inline double dg_to_double(double v) { return v; }
__device__ inline double dg_to_double(float v) { return v; }
__device__ inline double dg_to_double(df64 v) { return dg::dfp::df_to_double(v); }

// Penalty per face; binary64 storage: also w tau per face point (the face
// array 6 holds w = kappa da w on entry).
template <typename T>
__global__ void setup_face_tau(const SetupParams S, int d, int64_t n_faces, const double* daw, const double* vol,
                               T* tau, T* face, int64_t nfq) {
  const int k2 = S.k * S.k;
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < n_faces; f += (int64_t)gridDim.x * blockDim.x) {
    double A = 0.0;
    for (int q = 0; q < k2; ++q) A += daw[f * k2 + q];
    const int pos = (int)(f % S.P[d]);
    const int64_t rest = f / S.P[d];
    const int it1 = (int)(rest % S.n[t1]), it2 = (int)(rest / S.n[t1]);
    double r = 0.0;
    for (int slot = 0; slot < 2; ++slot) {
      const bool has = slot == 0 ? (S.periodic || pos >= 1) : (S.periodic || pos < S.n[d]);
      if (!has) continue;
      int ijk[3];
      ijk[t1] = it1;
      ijk[t2] = it2;
      ijk[d] = slot == 0 ? (pos - 1 + S.n[d]) % S.n[d] : pos % S.n[d];
      const int64_t c = ijk[0] + (int64_t)S.n[0] * (ijk[1] + (int64_t)S.n[1] * ijk[2]);
      r = fmax(r, A / vol[c]);
    }
    const double t = S.penalty * r;
    tau[S.face_minor ? dg::face_minor_id(S.n, S.P, d, f) : f] = (T)t;
    if (!S.face_minor)
      for (int q = 0; q < k2; ++q) {
        T& wq = face[6 * nfq + f * k2 + q];
        wq = (T)(t * dg_to_double(wq));
      }
  }
}

// ---------------------------------------------------------------------------
// Right-hand side (phi_i, f), (k+2)-point Gauss rule, one block per cell
// ---------------------------------------------------------------------------
struct RhsParams {
  SetupParams S;
  int which;
  int kq;
  double xq[kMaxK + 2], wq[kMaxK + 2];
  double phi[(kMaxK + 2) * kMaxK];  // phi[q*k + i] = basis function i at xq[q]
};

__global__ void rhs_kernel(const __grid_constant__ RhsParams R, int64_t n_cells, double* rhs) {
  extern __shared__ double fq[];
  const int k = R.S.k, kq = R.kq, nq = kq * kq * kq, k3 = k * k * k;
  for (int64_t c = blockIdx.x; c < n_cells; c += gridDim.x) {
    int ijk[3];
    cell_of(R.S, c, ijk);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const int q0 = q % kq, q1 = (q / kq) % kq, q2 = q / (kq * kq);
      const double xi[3] = {R.xq[q0], R.xq[q1], R.xq[q2]};
      double x[3], J[9], Ji[9];
      map_point(R.S, ijk, xi, x, J);
      const double det = invert3(J, Ji);
      double sx, cx, sy, sz, cy, cz;
      sincospi(x[0], &sx, &cx);
      sincospi(x[1], &sy, &cy);
      sincospi(x[2], &sz, &cz);
      const double u = sx * sy * sz;
      double f = 3.0 * M_PI * M_PI * u;
      if (R.which == 1) {
        const double kap = 1.0 + 0.5 * sinpi(2.0 * x[0]);
        const double dkap = M_PI * cospi(2.0 * x[0]);
        f = 3.0 * M_PI * M_PI * kap * u - dkap * M_PI * cx * sy * sz;
      }
      fq[q] = f * det * R.wq[q0] * R.wq[q1] * R.wq[q2];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < k3; i += blockDim.x) {
      const int i0 = i % k, i1 = (i / k) % k, i2 = i / (k * k);
      double s = 0.0;
      for (int q = 0; q < nq; ++q) {
        const int q0 = q % kq, q1 = (q / kq) % kq, q2 = q / (kq * kq);
        s += fq[q] * R.phi[q0 * k + i0] * R.phi[q1 * k + i1] * R.phi[q2 * k + i2];
      }
      rhs[c * k3 + i] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// L2 error against the manufactured solution u = sin(pi x) sin(pi y) sin(pi z),
// (k+2)-point Gauss rule, one block per cell, one partial per block
// ---------------------------------------------------------------------------
__global__ void l2_error_kernel(const __grid_constant__ RhsParams R, int64_t n_cells, const double* x,
                                double* part) {
  extern __shared__ double xs[];  // the cell's k^3 coefficients
  __shared__ double red[128];
  const int k = R.S.k, kq = R.kq, nq = kq * kq * kq, k3 = k * k * k;
  double acc = 0.0;
  for (int64_t c = blockIdx.x; c < n_cells; c += gridDim.x) {
    for (int i = threadIdx.x; i < k3; i += blockDim.x) xs[i] = x[c * k3 + i];
    __syncthreads();
    int ijk[3];
    cell_of(R.S, c, ijk);
    for (int q = threadIdx.x; q < nq; q += blockDim.x) {
      const int q0 = q % kq, q1 = (q / kq) % kq, q2 = q / (kq * kq);
      const double xi[3] = {R.xq[q0], R.xq[q1], R.xq[q2]};
      double xp[3], J[9], Ji[9];
      map_point(R.S, ijk, xi, xp, J);
      const double det = invert3(J, Ji);
      double uh = 0.0;
      for (int i2 = 0; i2 < k; ++i2)
        for (int i1 = 0; i1 < k; ++i1) {
          const double f12 = R.phi[q1 * k + i1] * R.phi[q2 * k + i2];
          for (int i0 = 0; i0 < k; ++i0) uh += xs[i0 + k * (i1 + k * i2)] * R.phi[q0 * k + i0] * f12;
        }
      const double e = uh - sinpi(xp[0]) * sinpi(xp[1]) * sinpi(xp[2]);
      acc += e * e * det * R.wq[q0] * R.wq[q1] * R.wq[q2];
    }
    __syncthreads();
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 64; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// CG vector kernels.  Reductions: per-block partials in a fixed order, then a
// single-block fixed-order pass, so every sum is reproducible bit for bit.
// ---------------------------------------------------------------------------
constexpr int kRedThreads = 256;
constexpr int kRedBlocks = 1024;

// device scalars: 0 rr, 1 bb, 2 pAp, 3 alpha, 4 beta, 5 rr_new, 6 breakdown flag,
// 7 stop flag (converged, breakdown or max_it), 8 iterations done,
// 9 (rtol |b|)^2, 10 max_it, 11 converged flag; the mixed-precision solver's
// residual replacement adds 12 the largest r.r since the last replacement,
// 13 delta^2, 14 replacement requested, 15 keep p (iterations frozen after a
// request leave the search direction alone)
enum {
  S_RR = 0, S_BB, S_PAP, S_ALPHA, S_BETA, S_RRNEW, S_FLAG, S_STOP, S_ITER, S_TOL2, S_MAXIT, S_DONE,
  // residual replacement of the mixed-precision solver
  S_MAXRR, S_DELTA2, S_RU, S_KEEP,
  S_COUNT
};

__device__ void block_store_sum(double v, double* out) {
  __shared__ double red[kRedThreads];
  red[threadIdx.x] = v;
  __syncthreads();
  for (int s = kRedThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

// r = b - ap (ap may be null: r = b), p = r; partials of r.r and b.b (FP64)
template <typename T>
__global__ void cg_init(int64_t n, const T* b, const T* ap, T* r, T* p, double* part) {
  double rr = 0.0, bb = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = ap ? b[i] - ap[i] : b[i];
    r[i] = ri;
    p[i] = ri;
    rr += (double)ri * (double)ri;
    bb += (double)b[i] * (double)b[i];
  }
  block_store_sum(rr, part + blockIdx.x);
  block_store_sum(bb, part + kRedBlocks + blockIdx.x);
}

// single block: sum the first n partials of part (fixed order), call fn
__device__ double reduce_partials(const double* part, int64_t n) {
  __shared__ double red[kRedThreads];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += kRedThreads) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kRedThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// Scalars of the CG iteration, kept on the device so that iterations need no
// host round trip.  Once converged (r.r <= (rtol |b|)^2), broken down or at
// max_it, alpha and beta are forced to zero: later iterations leave x and r
// unchanged, so the host may check only every few iterations.
__global__ void cg_scalars_init(const double* part, int64_t nparts, double* scal, double rtol, double max_it) {
  const double rr = reduce_partials(part, nparts);
  const double bb = reduce_partials(part + kRedBlocks, nparts);
  if (threadIdx.x == 0) {
    scal[S_RR] = rr;
    scal[S_BB] = bb;
    scal[S_FLAG] = 0.0;
    scal[S_ITER] = 0.0;
    scal[S_MAXIT] = max_it;
    const double tol2 = rtol * rtol * (bb > 0.0 ? bb : 1.0);
    scal[S_TOL2] = tol2;
    scal[S_DONE] = rr <= tol2 ? 1.0 : 0.0;
    scal[S_STOP] = (rr <= tol2 || max_it <= 0.0) ? 1.0 : 0.0;
  }
}

__global__ void cg_scalars_alpha(const double* part, int64_t nparts, double* scal) {
  const double pap = reduce_partials(part, nparts);
  if (threadIdx.x == 0) {
    scal[S_PAP] = pap;
    if (scal[S_STOP] != 0.0) {
      scal[S_ALPHA] = 0.0;
      return;
    }
    const double a = scal[S_RR] / pap;
    if (!(pap > 0.0) || !isfinite(a)) {
      scal[S_FLAG] = 1.0;
      scal[S_STOP] = 1.0;
      scal[S_ALPHA] = 0.0;
    } else {
      scal[S_ALPHA] = a;
    }
  }
}

// x += alpha p, r -= alpha ap; partials of r.r (FP64)
template <typename T>
__global__ void cg_update(int64_t n, const double* scal, T* x, T* r, const T* p, const T* ap, double* part) {
  const T a = (T)scal[S_ALPHA];
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    x[i] = fma(a, p[i], x[i]);
    const T ri = fma(-a, ap[i], r[i]);
    r[i] = ri;
    rr += (double)ri * (double)ri;
  }
  block_store_sum(rr, part + blockIdx.x);
}

__global__ void cg_scalars_beta(const double* part, int64_t nparts, double* scal) {
  const double rr = reduce_partials(part, nparts);
  if (threadIdx.x == 0) {
    scal[S_RRNEW] = rr;
    if (scal[S_STOP] != 0.0) {
      scal[S_BETA] = 0.0;
      return;
    }
    const double b = rr / scal[S_RR];
    scal[S_BETA] = isfinite(b) ? b : 0.0;
    scal[S_RR] = rr;
    scal[S_ITER] += 1.0;
    if (!isfinite(rr)) {
      scal[S_FLAG] = 1.0;
      scal[S_STOP] = 1.0;
    } else if (rr <= scal[S_TOL2]) {
      scal[S_DONE] = 1.0;
      scal[S_STOP] = 1.0;
    } else if (scal[S_ITER] >= scal[S_MAXIT]) {
      scal[S_STOP] = 1.0;
    }
  }
}

// p = r + beta p
template <typename T>
__global__ void cg_direction(int64_t n, const double* scal, const T* r, T* p) {
  const T b = (T)scal[S_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], r[i]);
}

// defect correction: r64 = b - ap64 with partials of r.r; r32 = r64 * scale;
// x += scale * d32
__global__ void mp_residual(int64_t n, const double* b, const double* ap, double* r, double* part) {
  double rr = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - ap[i];
    r[i] = ri;
    rr += ri * ri;
  }
  block_store_sum(rr, part + blockIdx.x);
}

template <typename T>
__global__ void mp_correct(int64_t n, double scale, const T* d, double* x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = fma(scale, (double)d[i], x[i]);
}

// Residual replacement ("reliable updates": Sleijpen & van der Vorst 1996,
// Clark et al. 2010) of the mixed-precision solver.  The binary32 iteration
// works on the scaled system A d = sigma r64 (sigma = 1 / |r64| at the last
// replacement): d accumulates in xl32, r32 is its recursive residual and p32
// the search direction.  A replacement is requested once r.r <= delta^2
// max r.r, r.r <= the scaled target, or after max_it iterations: that
// iteration stops before its direction update and later ones are frozen.
// The host then adds xl32 / sigma to the FP64 solution, recomputes the FP64
// residual r64, and continues the CG recursion with it in place of the
// recursive residual: beta = |r64|^2 / |r_old|^2 (r_old the residual at the
// start of the replacing iteration, S_RR) and p = r64 + beta p, so the
// search directions built so far are kept.
__global__ void ru_scalars_beta(const double* part, int64_t nparts, double* scal) {
  const double rr = reduce_partials(part, nparts);
  if (threadIdx.x == 0) {
    scal[S_RRNEW] = rr;
    if (scal[S_STOP] != 0.0) {
      scal[S_BETA] = 0.0;
      scal[S_KEEP] = 1.0;
      return;
    }
    scal[S_ITER] += 1.0;
    if (rr > scal[S_MAXRR]) scal[S_MAXRR] = rr;
    if (!isfinite(rr)) {
      scal[S_FLAG] = 1.0;
      scal[S_STOP] = 1.0;
      scal[S_KEEP] = 1.0;
    } else if (rr <= scal[S_TOL2] || rr <= scal[S_DELTA2] * scal[S_MAXRR] || scal[S_ITER] >= scal[S_MAXIT]) {
      // replacement: S_RR keeps |r_old|^2 for the host's beta
      scal[S_RU] = 1.0;
      scal[S_STOP] = 1.0;
      scal[S_KEEP] = 1.0;
    } else {
      const double b = rr / scal[S_RR];
      scal[S_BETA] = isfinite(b) ? b : 0.0;
      scal[S_RR] = rr;
    }
  }
}

// p = r + beta p, except in iterations frozen after a replacement request
template <typename T>
__global__ void ru_direction(int64_t n, const double* scal, const T* r, T* p) {
  if (scal[S_KEEP] != 0.0) return;
  const T b = (T)scal[S_BETA];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = fma(b, p[i], r[i]);
}

// Restart of the recursion from the FP64 residual: r32 = sigma r64 and
// p32 = r32 + bscaled p32 (bscaled = beta sigma_new / sigma_old; 0 on the
// first start), xl32 = 0; partials of r32.r32 (FP64).
template <typename T>
__global__ void ru_restart(int64_t n, const double* r64, double sigma, double bscaled, T* r32, T* p32, T* xl32,
                           double* part) {
  double rr = 0.0;
  const T fb = (T)bscaled;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T ri = (T)(r64[i] * sigma);
    r32[i] = ri;
    p32[i] = bscaled != 0.0 ? fma(fb, p32[i], ri) : ri;
    xl32[i] = T(0);
    rr += (double)ri * (double)ri;
  }
  block_store_sum(rr, part + blockIdx.x);
}

__global__ void ru_scalars_reset(const double* part, int64_t nparts, double* scal, double tol2, double delta2,
                                 double max_it) {
  const double rr = reduce_partials(part, nparts);
  if (threadIdx.x == 0) {
    scal[S_RR] = rr;
    scal[S_MAXRR] = rr;
    scal[S_TOL2] = tol2;
    scal[S_DELTA2] = delta2;
    scal[S_MAXIT] = max_it;
    scal[S_ITER] = 0.0;
    scal[S_STOP] = 0.0;
    scal[S_RU] = 0.0;
    scal[S_KEEP] = 0.0;
    scal[S_FLAG] = 0.0;
    scal[S_DONE] = 0.0;
    scal[S_ALPHA] = 0.0;
    scal[S_BETA] = 0.0;
  }
}

__global__ void sum_to_scalar(const double* part, int64_t nparts, double* out) {
  const double v = reduce_partials(part, nparts);
  if (threadIdx.x == 0) *out = v;
}

// Valid cells-per-block values of an operator's apply kernel, ascending:
// the binary32 kernel's two compiled tile shapes, else the autotuner's
// candidates up to the largest block.
std::vector<int> tile_choices(const dg_handle* h) {
  if (h->prec == DG_FP32) return {dg::f32_tile_small(h->k), dg::f32_geometry_block(h->k)};
  static const int cands[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 14, 16, 20, 24, 28, 32, 40, 48, 56, 64};
  std::vector<int> out;
  for (int c : cands)
    if (c <= dg::cells_per_block(h->k)) out.push_back(c);
  return out;
}

int64_t apply_blocks(const dg_handle* h) {
  const int C = h->cpb;
  return (h->n_cells + C - 1) / C;
}

dg_status launch_apply_range(dg_handle* h, const void* src, void* dst, double* dot_partial, int64_t cell_begin,
                             int64_t cell_end, cudaStream_t stream, int split_stage = 0) {
  dg::ApplyLaunch L;
  L.k = h->k;
  L.prec = h->prec;
  L.geo = kernel_geo(h->geom);
  L.op = h->op;
  L.src = src;
  L.dst = dst;
  L.tables = h->prec == DG_FP64 ? (const void*)&h->tabd
             : h->prec == DG_FP32 ? (const void*)&h->tabf
                                  : (const void*)&h->tabdf;
  L.geometry = h->prec == DG_FP64 ? (const void*)&h->geod
               : h->prec == DG_FP32 ? (const void*)&h->geof
                                    : (const void*)&h->geodf;
  L.dot_partial = dot_partial;
  L.skip = h->skip;
  L.stream = stream;
  L.cpb = h->cpb;
  L.cell_begin = cell_begin;
  L.cell_end = cell_end;
  L.face_mode = h->face_mode;
  L.split_stage = split_stage;
  L.split = &h->split;
  cudaError_t e;
  switch (h->k) {
    case 2: e = dg::launch_apply_k2(L, h->n_cells); break;
    case 3: e = dg::launch_apply_k3(L, h->n_cells); break;
    case 4: e = dg::launch_apply_k4(L, h->n_cells); break;
    case 5: e = dg::launch_apply_k5(L, h->n_cells); break;
    case 6: e = dg::launch_apply_k6(L, h->n_cells); break;
    case 7: e = dg::launch_apply_k7(L, h->n_cells); break;
    case 8: e = dg::launch_apply_k8(L, h->n_cells); break;
    case 9: e = dg::launch_apply_k9(L, h->n_cells); break;
    default: return fail(h, DG_ERR_ARG, "degree out of range");
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "apply kernel launch");
  return DG_OK;
}

dg_status launch_apply(dg_handle* h, const void* src, void* dst, double* dot_partial) {
  return launch_apply_range(h, src, dst, dot_partial, 0, h->n_cells, h->stream);
}

template <typename T>
void fill_geometry(dg_handle* h, dg::Geometry<T>& g) {
  memset(&g, 0, sizeof(g));
  for (int d = 0; d < 3; ++d) {
    g.n[d] = h->mesh.n[d];
    g.P[d] = h->mesh.periodic ? h->mesh.n[d] : h->mesh.n[d] + 1;
  }
  g.periodic = h->mesh.periodic;
  g.n_cells = h->n_cells;
  g.ncq = h->n_cells * h->k * h->k * h->k;
  g.cell = static_cast<const T*>(h->cell_geo);
  const int k2 = h->k * h->k;
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int64_t nf = (int64_t)g.P[d] * h->mesh.n[t1] * h->mesh.n[t2];
    g.nfq[d] = nf * k2;
    g.nfc[d] = (int)nf;
    g.face_pair = h->mesh.periodic && h->mesh.mapping != 0;
    g.face[d] = static_cast<const T*>(h->face_geo[d]);
    g.tau[d] = static_cast<const T*>(h->face_tau[d]);
  }
  const double ps = (h->opts.penalty_scale > 0 ? h->opts.penalty_scale : 1.0) * (h->k) * (h->k);
  g.cart_detj = (T)(1.0 / ((double)h->mesh.n[0] * h->mesh.n[1] * h->mesh.n[2]));
  for (int d = 0; d < 3; ++d) {
    g.cart_jinv[d] = (T)h->mesh.n[d];
    g.cart_tau[d] = (T)(ps * h->mesh.n[d]);
    g.vel[d] = (T)h->opts.velocity[d];
  }
  if (h->kappa_tab) {
    g.kq = static_cast<const T*>(h->kappa_tab);
    g.kf = g.kq + (int64_t)h->mesh.n[0] * h->k;
  }
}

template <typename T>
dg_status setup_geometry(dg_handle* h) {
  const int k = h->k, k2 = k * k, k3 = k2 * k;
  const int64_t ncq = h->n_cells * k3;
  SetupParams S;
  memset(&S, 0, sizeof(S));
  for (int d = 0; d < 3; ++d) {
    S.n[d] = h->mesh.n[d];
    S.P[d] = h->mesh.periodic ? h->mesh.n[d] : h->mesh.n[d] + 1;
    S.vel[d] = h->opts.velocity[d];
  }
  S.periodic = h->mesh.periodic;
  S.mapping = h->mesh.mapping;
  S.amp = h->mesh.amplitude;
  S.k = k;
  for (int i = 0; i < k; ++i) {
    S.gq[i] = h->t64.gq[i];
    S.gw[i] = h->t64.gw[i];
  }
  S.op = h->op;
  S.coeff = h->op == DG_OP_SIPG ? h->opts.coeff : 0;
  S.geom = kernel_geo(h->geom);
  S.penalty = (h->opts.penalty_scale > 0 ? h->opts.penalty_scale : 1.0) * k * k;

  int* bad = nullptr;
  double *part = nullptr, *vol = nullptr;
  dg_status st;
  if ((st = dev_alloc(h, (void**)&bad, sizeof(int))) != DG_OK) return st;
  DG_CUDA(h, cudaMemsetAsync(bad, 0, sizeof(int), h->stream));
  if ((st = dev_alloc(h, (void**)&part, sizeof(double) * ncq)) != DG_OK) { dev_free(h, bad); return st; }
  if ((st = dev_alloc(h, (void**)&vol, sizeof(double) * h->n_cells)) != DG_OK) {
    dev_free(h, bad);
    dev_free(h, part);
    return st;
  }

  const bool cart = h->geom == DG_GEOM_CARTESIAN;
  int ncell_arrays = 0;
  // full Jacobians for SIPG in binary64 storage (FP64 and double-float
  // operators): sqrt(kappa JxW) J^{-1}, 9 arrays; otherwise J^{-1} and the
  // weight, 10 arrays (the binary32 kernel keeps the weight separate)
  S.fold = h->geom == DG_GEOM_FULL_JAC && h->op == DG_OP_SIPG && h->prec != DG_FP32;
  if (!cart) {
    if (h->geom == DG_GEOM_FULL_JAC) ncell_arrays = S.fold ? 9 : 10;
    else if (h->geom == DG_GEOM_POSITIONS) ncell_arrays = h->op == DG_OP_SIPG ? 4 : 3;  // x, y, z (+ kappa)
    else ncell_arrays = h->op == DG_OP_SIPG ? 6 : 3;
  }
  // binary32: cell-blocked layout padded to whole blocks (zero padding)
  S.ncomp = ncell_arrays;
  S.cblk = h->prec == DG_FP32 ? dg::f32_geometry_block(k) : 0;
  S.face_minor = h->prec == DG_FP32 ? 1 : 0;
  S.face_pair = S.face_minor && h->mesh.periodic && h->mesh.mapping != 0;
  const int64_t ncell_alloc = S.cblk ? (h->n_cells + S.cblk - 1) / S.cblk * S.cblk : h->n_cells;
  h->cell_bytes = (int64_t)ncell_arrays * ncell_alloc * k3 * sizeof(T);
  st = dev_alloc(h, &h->cell_geo, (size_t)h->cell_bytes);
  if (st == DG_OK && h->cell_bytes > 0 && ncell_alloc != h->n_cells) {
    cudaError_t e = cudaMemsetAsync(h->cell_geo, 0, (size_t)h->cell_bytes, h->stream);
    if (e != cudaSuccess) st = cuda_fail(h, e, "cell geometry padding");
  }
  if (st == DG_OK) {
    const int threads = 256;
    const int64_t blocks = std::min<int64_t>((ncq + threads - 1) / threads, 152 * 64);
    setup_cell_geometry<T><<<(unsigned)blocks, threads, 0, h->stream>>>(S, h->n_cells, static_cast<T*>(h->cell_geo),
                                                                         ncq, part, bad);
    sum_cells<<<(unsigned)std::min<int64_t>((h->n_cells + 255) / 256, 4096), 256, 0, h->stream>>>(part, k3, h->n_cells,
                                                                                                 vol);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_fail(h, e, "cell geometry kernel");
  }
  h->face_bytes = 0;
  for (int d = 0; d < 3 && st == DG_OK && !cart; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int64_t nf = (int64_t)S.P[d] * h->mesh.n[t1] * h->mesh.n[t2];
    const int64_t nfq = nf * k2;
    const int nfa = h->op == DG_OP_SIPG ? (S.face_minor && !S.face_pair ? 4 : 7) : 1;
    S.nfa = nfa;
    // the blocked binary32 layout is padded to whole face blocks (zeros)
    const int64_t nf_alloc = S.face_minor ? (nf + dg::kFaceBlock - 1) / dg::kFaceBlock * dg::kFaceBlock : nf;
    const int64_t fbytes = (int64_t)sizeof(T) * nfa * nf_alloc * k2;
    double* daw = nullptr;
    if ((st = dev_alloc(h, &h->face_geo[d], fbytes)) != DG_OK) break;
    if (nf_alloc != nf) {
      cudaError_t e = cudaMemsetAsync(h->face_geo[d], 0, fbytes, h->stream);
      if (e != cudaSuccess) {
        st = cuda_fail(h, e, "face geometry padding");
        break;
      }
    }
    if (h->op == DG_OP_SIPG && (st = dev_alloc(h, &h->face_tau[d], sizeof(T) * nf)) != DG_OK) break;
    if ((st = dev_alloc(h, (void**)&daw, sizeof(double) * nfq)) != DG_OK) break;
    h->face_bytes += fbytes + (h->op == DG_OP_SIPG ? (int64_t)sizeof(T) * nf : 0);
    const int threads = 256;
    setup_face_geometry<T><<<(unsigned)std::min<int64_t>((nfq + threads - 1) / threads, 152 * 64), threads, 0,
                             h->stream>>>(S, d, nf, static_cast<T*>(h->face_geo[d]), nfq, daw, bad);
    if (h->op == DG_OP_SIPG)
      setup_face_tau<T><<<(unsigned)std::min<int64_t>((nf + threads - 1) / threads, 4096), threads, 0, h->stream>>>(
          S, d, nf, daw, vol, static_cast<T*>(h->face_tau[d]), static_cast<T*>(h->face_geo[d]), nfq);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    dev_free(h, daw);
    if (e != cudaSuccess) st = cuda_fail(h, e, "face geometry kernels");
  }
  if (st == DG_OK) {
    int hbad = 0;
    cudaError_t e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) st = cuda_fail(h, e, "geometry set-up");
    else if (hbad) st = fail(h, DG_ERR_ARG, "mapping has a non-positive Jacobian determinant");
  }
  dev_free(h, bad);
  dev_free(h, part);
  dev_free(h, vol);
  return st;
}

// kappa tables for the Cartesian geometry: kappa at (ix + g_q)/n0 and at ix/n0
template <typename T>
dg_status setup_kappa_table(dg_handle* h) {
  if (!(h->geom == DG_GEOM_CARTESIAN && h->op == DG_OP_SIPG && h->opts.coeff == 1)) return DG_OK;
  const int n0 = h->mesh.n[0], k = h->k;
  std::vector<T> tab((size_t)n0 * k + n0 + 1);
  for (int i = 0; i < n0; ++i)
    for (int q = 0; q < k; ++q) tab[(size_t)i * k + q] = (T)(1.0 + 0.5 * std::sin(2.0 * M_PI * (i + h->t64.gq[q]) / n0));
  for (int i = 0; i <= n0; ++i) tab[(size_t)n0 * k + i] = (T)(1.0 + 0.5 * std::sin(2.0 * M_PI * i / n0));
  dg_status st = dev_alloc(h, &h->kappa_tab, sizeof(T) * tab.size());
  if (st != DG_OK) return st;
  DG_CUDA(h, cudaMemcpyAsync(h->kappa_tab, tab.data(), sizeof(T) * tab.size(), cudaMemcpyHostToDevice, h->stream));
  DG_CUDA(h, cudaStreamSynchronize(h->stream));
  return DG_OK;
}

void free_handle(dg_handle* h) {
  if (!h) return;
  dev_free(h, h->cell_geo);
  for (int d = 0; d < 3; ++d) {
    dev_free(h, h->face_geo[d]);
    dev_free(h, h->face_tau[d]);
  }
  dev_free(h, h->kappa_tab);
  dev_free(h, h->r);
  dev_free(h, h->p);
  dev_free(h, h->ap);
  dev_free(h, h->partial);
  dev_free(h, h->scal);
  dev_free(h, h->stage_src);
  dev_free(h, h->stage_dst);
  dev_free(h, h->xw);
  dev_free(h, h->bw);
  for (int d = 0; d < 3; ++d) {
    dev_free(h, h->split.tr[d]);
  }
  dev_free(h, h->split.tq);
  if (h->cg_stream) cudaStreamDestroy(h->cg_stream);
  if (h->h2d_stream) cudaStreamDestroy(h->h2d_stream);
  if (h->d2h_stream) cudaStreamDestroy(h->d2h_stream);
  if (h->cmp_stream) cudaStreamDestroy(h->cmp_stream);
  for (cudaStream_t bs : h->bwd_stream)
    if (bs) cudaStreamDestroy(bs);
  for (auto e : h->pipe_ev)
    if (e) cudaEventDestroy(e);
  if (h->cg_event) cudaEventDestroy(h->cg_event);
  delete h;
}

}  // namespace

// CG work vectors (n doubles each, used as T* for the handle's precision),
// partial-sum buffer [vector partials | apply partials] and scalars.
dg_status ensure_cg_work(dg_handle* h, bool with_extra) {
  const int64_t n = h->n_dofs;
  dg_status st;
  if (!h->r) {
    if ((st = dev_alloc(h, (void**)&h->r, sizeof(double) * n)) != DG_OK) return st;
    if ((st = dev_alloc(h, (void**)&h->p, sizeof(double) * n)) != DG_OK) return st;
    if ((st = dev_alloc(h, (void**)&h->ap, sizeof(double) * n)) != DG_OK) return st;
    h->partial_len = 2 * kRedBlocks + h->n_cells;  // apply partials for any block size
    if ((st = dev_alloc(h, (void**)&h->partial, sizeof(double) * h->partial_len)) != DG_OK) return st;
    if ((st = dev_alloc(h, (void**)&h->scal, sizeof(double) * S_COUNT)) != DG_OK) return st;
  }
  if (with_extra && !h->xw) {
    if ((st = dev_alloc(h, (void**)&h->xw, sizeof(double) * n)) != DG_OK) return st;
    if ((st = dev_alloc(h, (void**)&h->bw, sizeof(double) * n)) != DG_OK) return st;
  }
  // Scalars are read back into handle memory (a small pageable copy after a
  // stream synchronization anyway); no page-locked allocation, which would
  // synchronize the whole device and disturb solves captured as graphs in
  // other threads.
  h->scal_host = h->scal_buf;
  // the work vectors are used on other streams (the solver's); make the
  // stream-ordered allocations complete first
  DG_CUDA(h, cudaStreamSynchronize(h->stream));
  return DG_OK;
}

// Conjugate gradients for A x = b in the handle's precision T (vectors of T,
// every reduction in FP64, fixed order).  x holds the initial guess, or is
// set to zero when x_zero.  Stops when |r| <= rtol |b| or after max_it
// iterations (DG_ERR_NOT_CONVERGED).  Each iteration: the apply with p.Ap in
// its epilogue, the fused update x += alpha p, r -= alpha Ap with r.r, and
// p = r + beta p; the scalars are read back once per iteration.
template <typename T>
dg_status run_cg(dg_handle* h, const T* b, T* x, bool x_zero, double rtol, int max_it, int* iters, double* rel_out,
                 double* bnorm_out) {
  const int64_t n = h->n_dofs;
  const int vb = (int)std::min<int64_t>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads);
  const int64_t nblk = apply_blocks(h);
  double* part_vec = h->partial;
  double* part_apply = h->partial + 2 * kRedBlocks;
  T* r = reinterpret_cast<T*>(h->r);
  T* p = reinterpret_cast<T*>(h->p);
  T* ap = reinterpret_cast<T*>(h->ap);
  // run on a handle-owned stream (capturable), ordered after the caller's
  cudaStream_t user = h->stream;
  if (!h->cg_stream) DG_CUDA(h, cudaStreamCreateWithFlags(&h->cg_stream, cudaStreamNonBlocking));
  if (!h->cg_event) DG_CUDA(h, cudaEventCreateWithFlags(&h->cg_event, cudaEventDisableTiming));
  DG_CUDA(h, cudaEventRecord(h->cg_event, user));
  DG_CUDA(h, cudaStreamWaitEvent(h->cg_stream, h->cg_event, 0));
  cudaStream_t s = h->cg_stream;
  h->stream = s;
  dg_status st = DG_OK;
  cudaGraphExec_t exec = nullptr;
  int it = 0;
  double rel = 0.0, bnorm = 1.0;
  do {
    if (x_zero) {
      DG_CUDA(h, cudaMemsetAsync(x, 0, sizeof(T) * n, s));
      cg_init<T><<<vb, kRedThreads, 0, s>>>(n, b, nullptr, r, p, part_vec);
    } else {
      if ((st = launch_apply(h, x, ap, nullptr)) != DG_OK) break;
      cg_init<T><<<vb, kRedThreads, 0, s>>>(n, b, ap, r, p, part_vec);
    }
    cg_scalars_init<<<1, kRedThreads, 0, s>>>(part_vec, vb, h->scal, rtol, (double)max_it);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      st = cuda_fail(h, e, "CG set-up");
      break;
    }
    // a block of kIterBlock iterations: apply with p.Ap fused into its
    // epilogue, fused x/r update with r.r, direction update; captured once
    // as a CUDA graph when the solve may be long.  Iterations after
    // convergence skip their applies (the flag was set by cg_scalars_init).
    h->skip = h->scal + S_STOP;
    const int kIterBlock = 8;
    auto enqueue_block = [&]() -> dg_status {
      for (int j = 0; j < kIterBlock; ++j) {
        dg_status s2 = launch_apply(h, p, ap, part_apply);
        if (s2 != DG_OK) return s2;
        cg_scalars_alpha<<<1, kRedThreads, 0, s>>>(part_apply, nblk, h->scal);
        cg_update<T><<<vb, kRedThreads, 0, s>>>(n, h->scal, x, r, p, ap, part_vec);
        cg_scalars_beta<<<1, kRedThreads, 0, s>>>(part_vec, vb, h->scal);
        cg_direction<T><<<vb, kRedThreads, 0, s>>>(n, h->scal, r, p);
      }
      return DG_OK;
    };
    if (max_it >= 4 * kIterBlock) {
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        dg_status s2 = enqueue_block();
        cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (s2 == DG_OK && ec == cudaSuccess && graph) {
          if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();  // a failed capture falls back to direct launches
    }
    while (true) {
      DG_CUDA(h, cudaMemcpyAsync(h->scal_host, h->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s));
      DG_CUDA(h, cudaStreamSynchronize(s));
      if (it == 0 && rel == 0.0) bnorm = std::sqrt(h->scal_host[S_BB] > 0 ? h->scal_host[S_BB] : 1.0);
      it = (int)h->scal_host[S_ITER];
      rel = std::sqrt(h->scal_host[S_RR]) / bnorm;
      if (h->scal_host[S_FLAG] != 0.0) {
        st = fail(h, DG_ERR_BREAKDOWN, "CG breakdown: p.Ap <= 0 or non-finite scalar");
        break;
      }
      if (h->scal_host[S_DONE] != 0.0) break;
      if (h->scal_host[S_STOP] != 0.0 || it >= max_it) {
        st = fail(h, DG_ERR_NOT_CONVERGED, "CG reached max_it");
        break;
      }
      if (exec) {
        cudaError_t e2 = cudaGraphLaunch(exec, s);
        if (e2 != cudaSuccess) {
          st = cuda_fail(h, e2, "CG graph launch");
          break;
        }
      } else if ((st = enqueue_block()) != DG_OK) {
        break;
      }
    }
  } while (false);
  if (exec) cudaGraphExecDestroy(exec);
  h->skip = nullptr;
  cudaEventRecord(h->cg_event, s);
  cudaStreamWaitEvent(user, h->cg_event, 0);
  h->stream = user;
  *iters = it;
  *rel_out = rel;
  *bnorm_out = bnorm;
  return st;
}

// Used by dg_noalloc.cu: the apply launch with caller-provided per-block
// partials of src . dst, after the same argument checks as dg_apply.
cudaError_t dg_internal_noalloc_preload();  // dg_noalloc.cu

dg_status dg_internal_apply_with_partials(dg_handle* h, const void* src, void* dst, double* partials,
                                          int64_t* n_blocks, cudaStream_t* stream) {
  if (!src || !dst) return fail(h, DG_ERR_ARG, "src or dst is NULL");
  const int64_t bytes = h->n_dofs * (h->prec == DG_FP32 ? 4 : 8);
  const char* a = static_cast<const char*>(src);
  const char* b = static_cast<const char*>(dst);
  if (a < b + bytes && b < a + bytes) return fail(h, DG_ERR_ARG, "src and dst overlap");
  if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15)
    return fail(h, DG_ERR_ARG, "src and dst must be 16-byte aligned");
  *n_blocks = apply_blocks(h);
  *stream = h->stream;
  return launch_apply(h, src, dst, partials);
}

dg_status dg_internal_fail(dg_handle* h, dg_status s, const char* msg) { return fail(h, s, msg); }

// Used by dg_batch.cu: the batched-launch description of one operator
// (key: degree k, arithmetic, geometry variant, weak form, face mode, tile
// shape), its tables, and the per-degree batched launch.
dg_status dg_internal_batch_desc(dg_handle* h, const void* src, void* dst, dg::BatchOp* op, int key[6],
                                 const void** tables) {
  if (!h || !op || !key || !tables) return DG_ERR_ARG;
  op->geometry = h->prec == DG_FP64 ? (const void*)&h->geod
                 : h->prec == DG_FP32 ? (const void*)&h->geof
                                      : (const void*)&h->geodf;
  op->src = src;
  op->dst = dst;
  op->split = (h->prec != DG_FP32 && h->face_mode == DG_FACE_LOOP) ? (const void*)&h->split : nullptr;
  op->n_cells = h->n_cells;
  key[0] = h->k;
  key[1] = h->prec;
  key[2] = kernel_geo(h->geom);
  key[3] = h->op;
  key[4] = h->prec != DG_FP32 ? h->face_mode : 0;
  key[5] = h->cpb;
  *tables = h->prec == DG_FP64 ? (const void*)&h->tabd
            : h->prec == DG_FP32 ? (const void*)&h->tabf
                                 : (const void*)&h->tabdf;
  return DG_OK;
}

cudaError_t dg_internal_batch_launch(const dg::BatchLaunch& L) {
  switch (L.k) {
    case 2: return dg::launch_batch_k2(L);
    case 3: return dg::launch_batch_k3(L);
    case 4: return dg::launch_batch_k4(L);
    case 5: return dg::launch_batch_k5(L);
    case 6: return dg::launch_batch_k6(L);
    case 7: return dg::launch_batch_k7(L);
    case 8: return dg::launch_batch_k8(L);
    case 9: return dg::launch_batch_k9(L);
    default: return cudaErrorInvalidValue;
  }
}
// Used by dg_batch.cu: dg_apply on a given stream (for graph capture).
dg_status dg_internal_apply_on_stream(dg_handle* h, const void* src, void* dst, void* stream) {
  if (!h) return DG_ERR_ARG;
  cudaStream_t saved = h->stream;
  h->stream = static_cast<cudaStream_t>(stream);
  dg_status st = dg_apply(h, src, dst);
  h->stream = saved;
  return st;
}


// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

dg_status dg_setup(const dg_mesh* mesh, int degree, int geom, const dg_opts* opts, void* stream, dg_handle** out) {
  if (!out) return fail(nullptr, DG_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!mesh || !opts) return fail(nullptr, DG_ERR_ARG, "mesh or opts is NULL");
  if (degree < 1 || degree > kMaxK - 1) return fail(nullptr, DG_ERR_ARG, "degree must be in 1..8");
  for (int d = 0; d < 3; ++d)
    if (mesh->n[d] < 1 || mesh->n[d] > (1 << 20)) return fail(nullptr, DG_ERR_ARG, "cells per direction must be >= 1");
  if (mesh->mapping < 0 || mesh->mapping > 2) return fail(nullptr, DG_ERR_ARG, "mapping must be 0, 1 or 2");
  if (mesh->mapping == 2 && mesh->periodic && opts->op == DG_OP_SIPG && opts->coeff == 1)
    return fail(nullptr, DG_ERR_ARG,
                "kappa = 1 + 0.5 sin(2 pi x) is not periodic on the sheared mesh (x shifts across the y/z wrap)");
  if (opts->op != DG_OP_SIPG && opts->op != DG_OP_ADVECTION) return fail(nullptr, DG_ERR_ARG, "unknown operator");
  if (opts->prec != DG_FP64 && opts->prec != DG_FP32 && opts->prec != DG_FP64_EMU)
    return fail(nullptr, DG_ERR_ARG, "unknown precision");
  if (opts->coeff != 0 && opts->coeff != 1) return fail(nullptr, DG_ERR_ARG, "coeff must be 0 or 1");
  if (opts->basis != DG_BASIS_LAGRANGE && opts->basis != DG_BASIS_HERMITE)
    return fail(nullptr, DG_ERR_ARG, "unknown basis");
  if (opts->basis == DG_BASIS_HERMITE && degree < 3)
    return fail(nullptr, DG_ERR_ARG, "the Hermite-like basis needs degree >= 3");
  if (geom != DG_GEOM_CARTESIAN && geom != DG_GEOM_FULL_JAC && geom != DG_GEOM_MERGED && geom != DG_GEOM_POSITIONS)
    return fail(nullptr, DG_ERR_ARG, "unknown geometry variant");
  if (geom == DG_GEOM_CARTESIAN && mesh->mapping != 0)
    return fail(nullptr, DG_ERR_ARG, "Cartesian geometry needs the identity mapping");
  const int64_t nc = (int64_t)mesh->n[0] * mesh->n[1] * mesh->n[2];
  const int k = degree + 1;
  if (nc >= ((int64_t)1 << 31) || nc * k * k * k > (int64_t)1 << 40)
    return fail(nullptr, DG_ERR_ARG, "mesh too large (at most 2^31 - 1 cells)");
  {
    // face ids of each direction are 32-bit in the kernels
    for (int d = 0; d < 3; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      if ((int64_t)(mesh->n[d] + 1) * mesh->n[t1] * mesh->n[t2] >= ((int64_t)1 << 31))
        return fail(nullptr, DG_ERR_ARG, "mesh too large (faces per direction must stay below 2^31)");
    }
  }

  dg_handle* h = new (std::nothrow) dg_handle();
  if (!h) return fail(nullptr, DG_ERR_OOM, "host allocation failed");
  h->mesh = *mesh;
  h->opts = *opts;
  h->degree = degree;
  h->k = k;
  h->geom = geom;
  h->prec = opts->prec;
  h->op = opts->op;
  h->n_cells = nc;
  h->n_dofs = nc * k * k * k;
  h->cpb = h->prec == DG_FP32 ? dg::f32_tile_default(k) : dg::element_cells_per_block(k, h->prec);
  h->stream = static_cast<cudaStream_t>(stream);
  build_tables(k, h->t64, opts->basis);
  h->tabd = cast_tables<double>(k, h->t64);
  h->tabf = cast_tables<float>(k, h->t64);
  h->tabdf = cast_tables<df64>(k, h->t64);

  dg_status st = h->prec == DG_FP64   ? setup_geometry<double>(h)
                 : h->prec == DG_FP32 ? setup_geometry<float>(h)
                                      : setup_geometry<df64>(h);
  if (st == DG_OK)
    st = h->prec == DG_FP64   ? setup_kappa_table<double>(h)
         : h->prec == DG_FP32 ? setup_kappa_table<float>(h)
                              : setup_kappa_table<df64>(h);
  if (st != DG_OK) {
    g_setup_error = h->err;
    free_handle(h);
    return st;
  }
  {
    // load the allocation-free entry point's module now, while allocating is allowed
    const cudaError_t e = dg_internal_noalloc_preload();
    if (e != cudaSuccess) {
      cuda_fail(h, e, "loading the allocation-free scratch module");
      g_setup_error = h->err;
      free_handle(h);
      return DG_ERR_CUDA;
    }
  }
  fill_geometry<double>(h, h->geod);
  fill_geometry<float>(h, h->geof);
  fill_geometry<df64>(h, h->geodf);
  if (geom == DG_GEOM_POSITIONS && h->prec != DG_FP32) {
    // G2 in binary64 / double-float: the face loop (its forward kernel stages the positions)
    st = dg_set_face_mode(h, DG_FACE_LOOP);
    if (st != DG_OK) {
      g_setup_error = h->err;
      free_handle(h);
      return st;
    }
  }
  *out = h;
  return DG_OK;
}

dg_status dg_n_dofs(const dg_handle* h, int64_t* n) {
  if (!h || !n) return DG_ERR_ARG;
  *n = h->n_dofs;
  return DG_OK;
}

dg_status dg_info(const dg_handle* h, dg_info_t* info) {
  if (!h || !info) return DG_ERR_ARG;
  info->n_dofs = h->n_dofs;
  info->n_cells = h->n_cells;
  info->degree = h->degree;
  info->prec = h->prec;
  info->geom = h->geom;
  info->op = h->op;
  info->cell_geometry_bytes = h->cell_bytes;
  info->face_geometry_bytes = h->face_bytes;
  info->cells_per_block = h->cpb;
  info->threads_per_block = h->cpb * h->k * h->k;
  info->shared_bytes_per_block = h->prec == DG_FP32 ? dg::f32_smem_bytes(h->k, h->op, h->cpb, kernel_geo(h->geom))
                                 : h->face_mode == DG_FACE_LOOP ? dg::split_smem_backward(h->k, h->op, h->cpb)
                                                                : dg::smem_bytes_per_block(h->k, h->op, 8, h->cpb);
  info->blocks = apply_blocks(h);
  const std::vector<int> tc = tile_choices(h);
  for (int i = 0; i < 24; ++i) info->tile_choices[i] = i < (int)tc.size() ? tc[i] : 0;
  info->face_mode = h->face_mode;
  return DG_OK;
}

dg_status dg_set_stream(dg_handle* h, void* stream) {
  if (!h) return DG_ERR_ARG;
  h->stream = static_cast<cudaStream_t>(stream);
  return DG_OK;
}

dg_status dg_apply(dg_handle* h, const void* src, void* dst) {
  if (!h) return DG_ERR_ARG;
  if (!src || !dst) return fail(h, DG_ERR_ARG, "src or dst is NULL");
  const int64_t bytes = h->n_dofs * (h->prec == DG_FP32 ? 4 : 8);
  const char* a = static_cast<const char*>(src);
  const char* b = static_cast<const char*>(dst);
  if (a < b + bytes && b < a + bytes) return fail(h, DG_ERR_ARG, "src and dst overlap");
  if ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15)
    return fail(h, DG_ERR_ARG, "src and dst must be 16-byte aligned");
  return launch_apply(h, src, dst, nullptr);
}

// dst = A src with host buffers, pipelined over slabs of whole z-planes of
// cells (contiguous cell ranges): all host-to-device copies are queued on one
// copy stream; slab s is applied (on the handle's stream and a second
// compute stream, alternately) as soon as slab s+1 (its upper z-neighbours)
// has arrived; its result is copied back on a second copy stream while later
// slabs are computed.  Results are the same as one
// dg_apply (every cell's arithmetic is independent of the launch range).
// The face loop runs its forward launch per slab as the slabs arrive and
// slab s's backward launch once slab s+1's forward launch is done.
// Periodic meshes in z (the first slab needs the last) and meshes whose
// z-planes do not align with the kernels' cell blocks use a single slab.
dg_status dg_apply_host(dg_handle* h, const void* src_host, void* dst_host) {
  if (!h) return DG_ERR_ARG;
  if (!src_host || !dst_host) return fail(h, DG_ERR_ARG, "src or dst is NULL");
  const size_t scal = h->prec == DG_FP32 ? 4 : 8;
  const size_t bytes = (size_t)h->n_dofs * scal;
  dg_status st;
  if (!h->stage_src && (st = dev_alloc(h, &h->stage_src, bytes)) != DG_OK) return st;
  if (!h->stage_dst && (st = dev_alloc(h, &h->stage_dst, bytes)) != DG_OK) return st;
  if (!h->h2d_stream) {
    DG_CUDA(h, cudaStreamCreateWithFlags(&h->h2d_stream, cudaStreamNonBlocking));
    DG_CUDA(h, cudaStreamCreateWithFlags(&h->d2h_stream, cudaStreamNonBlocking));
    DG_CUDA(h, cudaStreamCreateWithFlags(&h->cmp_stream, cudaStreamNonBlocking));
    for (cudaStream_t& bs : h->bwd_stream) DG_CUDA(h, cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    for (auto& e : h->pipe_ev) DG_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int64_t plane = (int64_t)h->mesh.n[0] * h->mesh.n[1];
  const int nz = h->mesh.n[2];
  int slabs = (!h->mesh.periodic && plane % 64 == 0 && nz >= 4) ? std::min(kHostSlabs, nz / 2) : 1;
  const int64_t k3 = (int64_t)h->k * h->k * h->k;
  // slab boundaries in z-planes: one-plane first and last slabs (the
  // pipeline's fill -- the first copy in -- and drain -- the last slab's
  // compute and copy out -- are short), the planes between split evenly
  auto plane_of_slab = [&](int s) -> int64_t {
    if (slabs < 4) return (int64_t)nz * s / slabs;
    if (s == 0) return 0;
    if (s == slabs) return nz;
    if (s == slabs - 1) return nz - 1;
    return 1 + (int64_t)(nz - 2) * (s - 1) / (slabs - 2);
  };
  auto cell_of_slab = [&](int s) { return plane * plane_of_slab(s); };
  cudaEvent_t* ev_in = h->pipe_ev;              // slab s on the device
  cudaEvent_t* ev_out = h->pipe_ev + kHostSlabs;  // slab s computed
  cudaEvent_t ev_start = h->pipe_ev[2 * kHostSlabs], ev_cmp = h->pipe_ev[2 * kHostSlabs + 1];
  // the copies follow earlier work on the handle's stream (staging reuse)
  DG_CUDA(h, cudaEventRecord(ev_start, h->stream));
  DG_CUDA(h, cudaStreamWaitEvent(h->h2d_stream, ev_start, 0));
  DG_CUDA(h, cudaStreamWaitEvent(h->d2h_stream, ev_start, 0));
  DG_CUDA(h, cudaStreamWaitEvent(h->cmp_stream, ev_start, 0));
  for (cudaStream_t bs : h->bwd_stream) DG_CUDA(h, cudaStreamWaitEvent(bs, ev_start, 0));
  for (int s = 0; s < slabs; ++s) {
    const int64_t c0 = cell_of_slab(s), c1 = cell_of_slab(s + 1);
    const size_t off = (size_t)(c0 * k3) * scal, len = (size_t)((c1 - c0) * k3) * scal;
    DG_CUDA(h, cudaMemcpyAsync(static_cast<char*>(h->stage_src) + off, static_cast<const char*>(src_host) + off, len,
                               cudaMemcpyHostToDevice, h->h2d_stream));
    DG_CUDA(h, cudaEventRecord(ev_in[s], h->h2d_stream));
  }
  if (h->face_mode == DG_FACE_LOOP) {
    // face loop: the forward launch of slab s as soon as it has arrived, the
    // backward launch of slab s once the forward launches of slabs s - 1, s
    // and s + 1 (which write the traces of its z-neighbours) are done.
    // Forward launches alternate between two streams and backward launches
    // between two more, so that consecutive slabs overlap: a slab of few
    // planes does not fill the GPU, and the pipeline's fill (the first
    // slab's forward launch) and drain (the last slab's backward launch)
    // then run beside their neighbours' launches instead of alone.
    cudaEvent_t* ev_fwd = h->pipe_ev + 2 * kHostSlabs + 2;
    cudaStream_t fs[2] = {h->stream, h->cmp_stream};
    for (int s = 0; s < slabs; ++s) {
      cudaStream_t f = fs[s % 2];
      DG_CUDA(h, cudaStreamWaitEvent(f, ev_in[s], 0));
      if ((st = launch_apply_range(h, h->stage_src, h->stage_dst, nullptr, cell_of_slab(s), cell_of_slab(s + 1), f,
                                   1)) != DG_OK)
        return st;
      DG_CUDA(h, cudaEventRecord(ev_fwd[s], f));
    }
    for (int s = 0; s < slabs; ++s) {
      const int64_t c0 = cell_of_slab(s), c1 = cell_of_slab(s + 1);
      cudaStream_t bs = h->bwd_stream[s % 2];
      for (int n = std::max(s - 1, 0); n <= std::min(s + 1, slabs - 1); ++n)
        DG_CUDA(h, cudaStreamWaitEvent(bs, ev_fwd[n], 0));
      if ((st = launch_apply_range(h, h->stage_src, h->stage_dst, nullptr, c0, c1, bs, 2)) != DG_OK) return st;
      DG_CUDA(h, cudaEventRecord(ev_out[s], bs));
      DG_CUDA(h, cudaStreamWaitEvent(h->d2h_stream, ev_out[s], 0));
      const size_t off = (size_t)(c0 * k3) * scal, len = (size_t)((c1 - c0) * k3) * scal;
      DG_CUDA(h, cudaMemcpyAsync(static_cast<char*>(dst_host) + off, static_cast<const char*>(h->stage_dst) + off,
                                 len, cudaMemcpyDeviceToHost, h->d2h_stream));
    }
    // join the compute streams into the handle's stream (later work and the
    // next call's staging reuse follow it)
    for (cudaStream_t js : {h->cmp_stream, h->bwd_stream[0], h->bwd_stream[1]}) {
      DG_CUDA(h, cudaEventRecord(ev_cmp, js));
      DG_CUDA(h, cudaStreamWaitEvent(h->stream, ev_cmp, 0));
    }
    DG_CUDA(h, cudaStreamSynchronize(h->d2h_stream));
    DG_CUDA(h, cudaStreamSynchronize(h->stream));
    return DG_OK;
  }
  for (int s = 0; s < slabs; ++s) {
    const int64_t c0 = cell_of_slab(s), c1 = cell_of_slab(s + 1);
    // slabs alternate between two compute streams so that one slab's last
    // blocks overlap the next slab's first ones
    cudaStream_t cs = (s % 2) ? h->cmp_stream : h->stream;
    DG_CUDA(h, cudaStreamWaitEvent(cs, ev_in[std::min(s + 1, slabs - 1)], 0));
    if ((st = launch_apply_range(h, h->stage_src, h->stage_dst, nullptr, c0, c1, cs)) != DG_OK) return st;
    DG_CUDA(h, cudaEventRecord(ev_out[s], cs));
    DG_CUDA(h, cudaStreamWaitEvent(h->d2h_stream, ev_out[s], 0));
    const size_t off = (size_t)(c0 * k3) * scal, len = (size_t)((c1 - c0) * k3) * scal;
    DG_CUDA(h, cudaMemcpyAsync(static_cast<char*>(dst_host) + off, static_cast<const char*>(h->stage_dst) + off, len,
                               cudaMemcpyDeviceToHost, h->d2h_stream));
  }
  DG_CUDA(h, cudaEventRecord(ev_cmp, h->cmp_stream));
  DG_CUDA(h, cudaStreamWaitEvent(h->stream, ev_cmp, 0));
  DG_CUDA(h, cudaStreamSynchronize(h->d2h_stream));
  DG_CUDA(h, cudaStreamSynchronize(h->stream));
  return DG_OK;
}

static void fill_rhs_params(const dg_handle* h, int which_f, RhsParams& R) {
  memset(&R, 0, sizeof(R));
  for (int d = 0; d < 3; ++d) R.S.n[d] = h->mesh.n[d];
  R.S.periodic = h->mesh.periodic;
  R.S.mapping = h->mesh.mapping;
  R.S.amp = h->mesh.amplitude;
  R.S.k = h->k;
  R.which = which_f;
  R.kq = h->k + 2;
  double xq[kMaxK + 2], wq[kMaxK + 2];
  gauss_rule(R.kq, xq, wq);
  for (int q = 0; q < R.kq; ++q) {
    R.xq[q] = xq[q];
    R.wq[q] = wq[q];
    basis_values(h->t64, h->k, xq[q], R.phi + q * h->k, nullptr);
  }
}

dg_status dg_l2_error(dg_handle* h, const double* x, double* err) {
  if (!h) return DG_ERR_ARG;
  if (!x || !err) return fail(h, DG_ERR_ARG, "x or err is NULL");
  RhsParams R;
  fill_rhs_params(h, 0, R);
  const int nblk = (int)std::min<int64_t>(h->n_cells, 152 * 16);
  double* part = nullptr;
  dg_status st = dev_alloc(h, (void**)&part, sizeof(double) * nblk);
  if (st != DG_OK) return st;
  l2_error_kernel<<<nblk, 128, sizeof(double) * h->k * h->k * h->k, h->stream>>>(R, h->n_cells, x, part);
  std::vector<double> hp(nblk);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), part, sizeof(double) * nblk, cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  dev_free(h, part);
  if (e != cudaSuccess) return cuda_fail(h, e, "L2 error kernel");
  double sum = 0.0;
  for (double v : hp) sum += v;
  *err = std::sqrt(sum);
  return DG_OK;
}

dg_status dg_rhs(dg_handle* h, int which_f, double* rhs) {
  if (!h) return DG_ERR_ARG;
  if (!rhs) return fail(h, DG_ERR_ARG, "rhs is NULL");
  if (which_f != 0 && which_f != 1) return fail(h, DG_ERR_ARG, "which_f must be 0 or 1");
  RhsParams R;
  fill_rhs_params(h, which_f, R);
  const int nq = R.kq * R.kq * R.kq;
  rhs_kernel<<<(unsigned)std::min<int64_t>(h->n_cells, 152 * 16), 128, sizeof(double) * nq, h->stream>>>(R, h->n_cells,
                                                                                                         rhs);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "rhs kernel");
  return DG_OK;
}

dg_status dg_cg_solve(dg_handle* h, const double* rhs, double* x, double rtol, int max_it, int* iters,
                      double* final_rel_res) {
  if (!h) return DG_ERR_ARG;
  if (h->op != DG_OP_SIPG) return fail(h, DG_ERR_UNSUPPORTED, "CG needs the symmetric SIPG operator");
  if (h->prec == DG_FP32) return fail(h, DG_ERR_UNSUPPORTED, "CG runs on FP64 handles (see dg_cg_solve_mixed)");
  if (!rhs || !x) return fail(h, DG_ERR_ARG, "rhs or x is NULL");
  if (!(rtol > 0.0) || max_it < 0) return fail(h, DG_ERR_ARG, "rtol must be > 0 and max_it >= 0");
  dg_status st = ensure_cg_work(h, false);
  if (st != DG_OK) return st;
  double rel = 0.0, bn = 0.0;
  int it = 0;
  st = run_cg<double>(h, rhs, x, false, rtol, max_it, &it, &rel, &bn);
  if (iters) *iters = it;
  if (final_rel_res) *final_rel_res = rel;
  return st;
}

}  // extern "C"

namespace {

// Result of one run of the mixed-precision iteration.
struct MixedOut {
  int outer = 0;        // residual replacements (FP64 residuals after the first)
  int inner = 0;        // iterations of the low-precision recursion
  double rel = 0.0;     // |b - A x| / |b| (FP64) at return
  double rel0 = 0.0;    // the same at entry
  bool converged = false;
  bool slow = false;    // probe: the recursion was found too slow (see mixed_run)
};

// Conjugate gradients in the inner handle's arithmetic T (binary32 vectors
// for a DG_FP32 handle, binary64 vectors with double-float applies for a
// DG_FP64_EMU handle) with residual replacement by the FP64 residual of h64
// (the kernels above): every replacement adds the inner solution to x in
// FP64, recomputes b - A x with the FP64 operator and continues the CG
// recursion from it.  probe > 0: at most 16 inner iterations per phase, and
// at every replacement the iterations still needed at the rate observed
// since entry are estimated; once they are at most `few` the run goes on
// normally, but after `probe` inner iterations without that it returns with
// mo.slow set (x holds the solution so far).  x holds the initial guess.
template <typename T>
dg_status mixed_run(dg_handle* h64, dg_handle* hl, const double* rhs, double* x, double rtol, int max_outer,
                    double delta, int max_inner, int probe, double few, MixedOut& mo) {
  dg_status st = ensure_cg_work(h64, false);
  if (st == DG_OK) st = ensure_cg_work(hl, true);
  if (st != DG_OK) return st;
  // the whole solve runs on the inner handle's solver stream (capturable),
  // ordered after the caller's stream and before its later work
  cudaStream_t user = h64->stream;
  if (!hl->cg_stream) DG_CUDA(h64, cudaStreamCreateWithFlags(&hl->cg_stream, cudaStreamNonBlocking));
  if (!hl->cg_event) DG_CUDA(h64, cudaEventCreateWithFlags(&hl->cg_event, cudaEventDisableTiming));
  DG_CUDA(h64, cudaEventRecord(hl->cg_event, user));
  DG_CUDA(h64, cudaStreamWaitEvent(hl->cg_stream, hl->cg_event, 0));
  cudaStream_t s = hl->cg_stream;
  cudaStream_t savedl = hl->stream;
  h64->stream = s;
  hl->stream = s;
  const int64_t n = h64->n_dofs;
  const int vb = (int)std::min<int64_t>(kRedBlocks, (n + kRedThreads - 1) / kRedThreads);
  const int64_t nblkl = apply_blocks(hl);
  T* r32 = reinterpret_cast<T*>(hl->r);
  T* p32 = reinterpret_cast<T*>(hl->p);
  T* ap32 = reinterpret_cast<T*>(hl->ap);
  T* xl32 = reinterpret_cast<T*>(hl->xw);
  double* part32 = hl->partial;
  double* part_apply32 = hl->partial + 2 * kRedBlocks;
  const double delta2 = delta * delta;
  cudaGraphExec_t exec = nullptr;
  int outer = 0, inner_total = 0;
  double rel = 0.0, bnorm = 1.0, sigma = 1.0;
  int phase_max = probe > 0 ? std::min(16, max_inner) : max_inner;
  bool probing = probe > 0;
  // FP64 residual r64 = b - A x into h64->r and its r.r into h64->scal[S_RR]
  auto fp64_residual = [&](double* rr_out) -> dg_status {
    dg_status s2 = launch_apply(h64, x, h64->ap, nullptr);
    if (s2 != DG_OK) return s2;
    mp_residual<<<vb, kRedThreads, 0, s>>>(n, rhs, h64->ap, h64->r, h64->partial);
    sum_to_scalar<<<1, kRedThreads, 0, s>>>(h64->partial, vb, h64->scal + S_RR);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(h64->scal_host, h64->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h64, e, "mixed-precision FP64 residual");
    *rr_out = h64->scal_host[S_RR];
    return DG_OK;
  };
  // restart the inner recursion from the FP64 residual (norm^2 rr64);
  // rr_old: |r_old|^2 of the replacing iteration in the old scaling
  auto restart = [&](double rr64, bool first, double rr_old) -> dg_status {
    const double sig = 1.0 / std::sqrt(rr64);
    // beta = |r64|^2 / |r_old / sigma|^2, times sigma_new / sigma_old for the
    // rescaling of p
    const double bscaled = first ? 0.0 : (rr64 * sigma * sigma / rr_old) * (sig / sigma);
    if (!first && !(std::isfinite(bscaled) && bscaled > 0.0))
      return fail(h64, DG_ERR_BREAKDOWN, "mixed-precision CG: invalid beta at a residual replacement");
    ru_restart<T><<<vb, kRedThreads, 0, s>>>(n, h64->r, sig, bscaled, r32, p32, xl32, part32);
    sigma = sig;
    const double tol = rtol * bnorm * sigma;
    ru_scalars_reset<<<1, kRedThreads, 0, s>>>(part32, vb, hl->scal, tol * tol, delta2, (double)phase_max);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DG_OK : cuda_fail(h64, e, "mixed-precision restart");
  };
  // a block of inner iterations; the applies skip themselves once the
  // iteration is frozen (replacement requested or breakdown)
  const int kIterBlock = 8;
  auto enqueue_block = [&]() -> dg_status {
    for (int j = 0; j < kIterBlock; ++j) {
      dg_status s2 = launch_apply(hl, p32, ap32, part_apply32);
      if (s2 != DG_OK) return s2;
      cg_scalars_alpha<<<1, kRedThreads, 0, s>>>(part_apply32, nblkl, hl->scal);
      cg_update<T><<<vb, kRedThreads, 0, s>>>(n, hl->scal, xl32, r32, p32, ap32, part32);
      ru_scalars_beta<<<1, kRedThreads, 0, s>>>(part32, vb, hl->scal);
      ru_direction<T><<<vb, kRedThreads, 0, s>>>(n, hl->scal, r32, p32);
    }
    return DG_OK;
  };
  hl->skip = hl->scal + S_STOP;
  do {
    // |b| and the initial residual
    cg_init<double><<<vb, kRedThreads, 0, s>>>(n, rhs, nullptr, h64->r, h64->p, h64->partial);
    sum_to_scalar<<<1, kRedThreads, 0, s>>>(h64->partial + kRedBlocks, vb, h64->scal + S_BB);
    double rr64 = 0.0;
    if ((st = fp64_residual(&rr64)) != DG_OK) break;
    bnorm = std::sqrt(h64->scal_host[S_BB] > 0 ? h64->scal_host[S_BB] : 1.0);
    rel = std::sqrt(rr64) / bnorm;
    mo.rel0 = rel;
    if (!std::isfinite(rel)) {
      st = fail(h64, DG_ERR_BREAKDOWN, "mixed-precision CG: non-finite residual");
      break;
    }
    if (rel <= rtol) break;
    if (rr64 <= 0.0) break;
    if (max_outer <= 0) {
      st = fail(h64, DG_ERR_NOT_CONVERGED, "mixed-precision CG reached max_outer");
      break;
    }
    if ((st = restart(rr64, true, 0.0)) != DG_OK) break;
    {
      cudaGraph_t graph = nullptr;
      if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
        dg_status s2 = enqueue_block();
        cudaError_t ec = cudaStreamEndCapture(s, &graph);
        if (s2 == DG_OK && ec == cudaSuccess && graph) {
          if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) exec = nullptr;
        }
        if (graph) cudaGraphDestroy(graph);
      }
      cudaGetLastError();  // a failed capture falls back to direct launches
    }
    int last_it = 0, stalled = 0;
    double best_rel = rel;
    while (true) {
      if (exec) {
        cudaError_t e2 = cudaGraphLaunch(exec, s);
        if (e2 != cudaSuccess) {
          st = cuda_fail(h64, e2, "mixed-precision graph launch");
          break;
        }
      } else if ((st = enqueue_block()) != DG_OK) {
        break;
      }
      cudaError_t e = cudaMemcpyAsync(hl->scal_host, hl->scal, sizeof(double) * S_COUNT, cudaMemcpyDeviceToHost, s);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) {
        st = cuda_fail(h64, e, "mixed-precision scalars");
        break;
      }
      const int it = (int)hl->scal_host[S_ITER];
      inner_total += it - last_it;
      last_it = it;
      if (hl->scal_host[S_FLAG] != 0.0) {
        st = fail(h64, DG_ERR_BREAKDOWN, "mixed-precision CG breakdown: p.Ap <= 0 or non-finite scalar");
        break;
      }
      if (hl->scal_host[S_RU] == 0.0) continue;
      // residual replacement: x += xl / sigma, FP64 residual, restart
      mp_correct<T><<<vb, kRedThreads, 0, s>>>(n, 1.0 / sigma, xl32, x);
      if ((st = fp64_residual(&rr64)) != DG_OK) break;
      ++outer;
      rel = std::sqrt(rr64) / bnorm;
      if (!std::isfinite(rel)) {
        st = fail(h64, DG_ERR_BREAKDOWN, "mixed-precision CG: non-finite residual");
        break;
      }
      if (rel <= rtol || rr64 <= 0.0) break;
      if (probing) {
        double need = 1e30;
        if (rel > 0.0 && mo.rel0 > rel && inner_total > 0)
          need = inner_total * std::log(rel / rtol) / std::log(mo.rel0 / rel);
        if (need <= few) {
          probing = false;
          phase_max = max_inner;
        } else if (inner_total >= probe) {
          mo.slow = true;
          break;
        }
      }
      if (outer >= max_outer) {
        st = fail(h64, DG_ERR_NOT_CONVERGED, "mixed-precision CG reached max_outer residual replacements");
        break;
      }
      // stagnation: the outer residual's attainable floor (e.g. a
      // double-float outer operator near 1e-10) is reached when four
      // replacements in a row bring no halving of the best residual so far
      if (rel < 0.5 * best_rel) {
        best_rel = rel;
        stalled = 0;
      } else if (++stalled >= 4) {
        st = fail(h64, DG_ERR_NOT_CONVERGED, "mixed-precision CG stagnated: the outer residual no longer decreases");
        break;
      }
      if ((st = restart(rr64, false, hl->scal_host[S_RR])) != DG_OK) break;
      last_it = 0;
    }
  } while (false);
  hl->skip = nullptr;
  if (exec) cudaGraphExecDestroy(exec);
  cudaEventRecord(hl->cg_event, s);
  cudaStreamWaitEvent(user, hl->cg_event, 0);
  h64->stream = user;
  hl->stream = savedl;
  mo.outer += outer;
  mo.inner += inner_total;
  mo.rel = rel;
  mo.converged = st == DG_OK && rel <= rtol;
  return st;
}

dg_status check_mixed_pair(dg_handle* h64, dg_handle* hl) {
  if (h64->op != DG_OP_SIPG || hl->op != DG_OP_SIPG)
    return fail(h64, DG_ERR_UNSUPPORTED, "mixed-precision CG needs the symmetric SIPG operator");
  if (memcmp(&h64->mesh, &hl->mesh, sizeof(dg_mesh)) != 0 || h64->degree != hl->degree ||
      h64->geom != hl->geom || h64->opts.coeff != hl->opts.coeff || h64->opts.basis != hl->opts.basis ||
      h64->opts.penalty_scale != hl->opts.penalty_scale)
    return fail(h64, DG_ERR_ARG, "the handles of the mixed-precision solve describe different operators");
  return DG_OK;
}

}  // namespace

extern "C" {

dg_status dg_cg_solve_mixed(dg_handle* h64, dg_handle* h32, const double* rhs, double* x, double rtol, int max_outer,
                            double inner_rtol, int max_inner, int* outer_iters, int* inner_iters,
                            double* final_rel_res) {
  if (!h64 || !h32) return DG_ERR_ARG;
  if (h64->prec == DG_FP32 || (h32->prec != DG_FP32 && h32->prec != DG_FP64_EMU))
    return fail(h64, DG_ERR_ARG, "mixed-precision CG needs an FP64 (or emulated FP64) handle and an FP32 or "
                                 "emulated-FP64 inner handle");
  dg_status st = check_mixed_pair(h64, h32);
  if (st != DG_OK) return st;
  if (!rhs || !x) return fail(h64, DG_ERR_ARG, "rhs or x is NULL");
  if (!(rtol > 0.0) || !(inner_rtol > 0.0) || inner_rtol >= 1.0 || max_outer < 0 || max_inner < 1)
    return fail(h64, DG_ERR_ARG, "need rtol > 0, 0 < inner_rtol < 1, max_outer >= 0, max_inner >= 1");
  MixedOut mo;
  st = h32->prec == DG_FP32 ? mixed_run<float>(h64, h32, rhs, x, rtol, max_outer, inner_rtol, max_inner, 0, 0.0, mo)
                            : mixed_run<double>(h64, h32, rhs, x, rtol, max_outer, inner_rtol, max_inner, 0, 0.0, mo);
  if (outer_iters) *outer_iters = mo.outer;
  if (inner_iters) *inner_iters = mo.inner;
  if (final_rel_res) *final_rel_res = mo.rel;
  return st;
}

dg_status dg_cg_solve_mixed_auto(dg_handle* h64, dg_handle* hemu, dg_handle* h32, const double* rhs, double* x,
                                 double rtol, int max_outer, double inner_rtol, int max_inner, int* outer_iters,
                                 int* inner_iters, double* final_rel_res, int* inner_prec) {
  if (!h64 || !hemu || !h32) return DG_ERR_ARG;
  if (h64->prec == DG_FP32 || hemu->prec != DG_FP64_EMU || h32->prec != DG_FP32)
    return fail(h64, DG_ERR_ARG, "need an FP64 handle, an emulated-FP64 handle and an FP32 handle");
  dg_status st = check_mixed_pair(h64, hemu);
  if (st == DG_OK) st = check_mixed_pair(h64, h32);
  if (st != DG_OK) return st;
  if (!rhs || !x) return fail(h64, DG_ERR_ARG, "rhs or x is NULL");
  if (!(rtol > 0.0) || !(inner_rtol > 0.0) || inner_rtol >= 1.0 || max_outer < 1 || max_inner < 1)
    return fail(h64, DG_ERR_ARG, "need rtol > 0, 0 < inner_rtol < 1, max_outer >= 1, max_inner >= 1");
  // the double-float recursion first, as a probe: it goes on if the
  // iterations still needed at the observed rate are few (a binary32
  // recursion would add rounding noise across the whole spectrum, which CG
  // then has to remove again), otherwise after kProbe iterations the
  // binary32 recursion, several times cheaper per iteration, takes over
  constexpr int kProbe = 48;
  constexpr double kFewIterations = 200.0;
  MixedOut mo;
  int kind = DG_FP64_EMU;
  st = mixed_run<double>(h64, hemu, rhs, x, rtol, max_outer, inner_rtol, max_inner, kProbe, kFewIterations, mo);
  if (st == DG_OK && mo.slow) {
    kind = DG_FP32;
    const int left = std::max(1, max_outer - mo.outer);
    mo.slow = false;
    st = mixed_run<float>(h64, h32, rhs, x, rtol, left, inner_rtol, max_inner, 0, 0.0, mo);
  }
  if (outer_iters) *outer_iters = mo.outer;
  if (inner_iters) *inner_iters = mo.inner;
  if (final_rel_res) *final_rel_res = mo.rel;
  if (inner_prec) *inner_prec = kind;
  return st;
}

dg_status dg_set_face_mode(dg_handle* h, int mode) {
  if (!h) return DG_ERR_ARG;
  if (mode != DG_FACE_ELEMENT && mode != DG_FACE_LOOP) return fail(h, DG_ERR_ARG, "unknown face mode");
  if (mode == DG_FACE_LOOP && h->prec == DG_FP32)
    return fail(h, DG_ERR_UNSUPPORTED, "the face-loop apply is implemented for DG_FP64 and DG_FP64_EMU");
  if (mode == DG_FACE_LOOP && !h->t64.end_nodal)
    return fail(h, DG_ERR_UNSUPPORTED, "the face-loop apply needs a basis whose face values are its end layers");
  if (mode == DG_FACE_ELEMENT && h->geom == DG_GEOM_POSITIONS && h->prec != DG_FP32)
    return fail(h, DG_ERR_UNSUPPORTED, "G2 (positions) binary64 and double-float operators run the face loop only");
  if (mode == DG_FACE_LOOP && !h->split.tq) {
    // traces per face and slot, gradient-test fields per point
    const int k2 = h->k * h->k;
    const int nf = h->op == DG_OP_SIPG ? 4 : 1;
    dg_status st = DG_OK;
    for (int d = 0; d < 3 && st == DG_OK; ++d) {
      const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
      const int64_t faces = (int64_t)(h->mesh.periodic ? h->mesh.n[d] : h->mesh.n[d] + 1) * h->mesh.n[t1] *
                            h->mesh.n[t2];
      const size_t bytes = sizeof(double) * faces * 2 * nf * k2;
      st = dev_alloc(h, (void**)&h->split.tr[d], bytes);
    }
    if (st == DG_OK) st = dev_alloc(h, (void**)&h->split.tq, sizeof(double) * 3 * h->n_dofs);
    if (st != DG_OK) {  // nothing half-allocated stays behind; the mode is unchanged
      for (auto& p : h->split.tr) {
        dev_free(h, p);
        p = nullptr;
      }
      dev_free(h, h->split.tq);
      h->split.tq = nullptr;
      return st;
    }
    DG_CUDA(h, cudaStreamSynchronize(h->stream));
  }
  // an unchanged default tile shape follows the mode's default
  const int def_old = h->face_mode == DG_FACE_LOOP ? dg::split_cells_per_block(h->k, h->prec)
                                                    : dg::element_cells_per_block(h->k, h->prec);
  if (h->prec != DG_FP32 && h->cpb == def_old)
    h->cpb = mode == DG_FACE_LOOP ? dg::split_cells_per_block(h->k, h->prec)
                                  : dg::element_cells_per_block(h->k, h->prec);
  h->face_mode = mode;
  return DG_OK;
}

dg_status dg_set_cells_per_block(dg_handle* h, int cpb) {
  if (!h) return DG_ERR_ARG;
  if (h->prec == DG_FP32) {
    // the binary32 kernel is compiled for two tile shapes
    if (cpb == 0) cpb = dg::f32_tile_default(h->k);
    if (cpb != dg::f32_tile_small(h->k) && cpb != dg::f32_geometry_block(h->k))
      return fail(h, DG_ERR_ARG, "binary32 cells per block must be " + std::to_string(dg::f32_tile_small(h->k)) +
                                     " or " + std::to_string(dg::f32_geometry_block(h->k)));
    h->cpb = cpb;
    return DG_OK;
  }
  if (cpb == 0)
    cpb = h->face_mode == DG_FACE_LOOP ? dg::split_cells_per_block(h->k, h->prec)
                                       : dg::element_cells_per_block(h->k, h->prec);
  if (cpb < 1 || cpb > dg::cells_per_block(h->k))
    return fail(h, DG_ERR_ARG, "cells per block must be in 1.." + std::to_string(dg::cells_per_block(h->k)));
  h->cpb = cpb;
  return DG_OK;
}

dg_status dg_autotune(dg_handle* h, int* best_cpb, double* best_ms) {
  if (!h) return DG_ERR_ARG;
  const size_t bytes = (size_t)h->n_dofs * (h->prec == DG_FP32 ? 4 : 8);
  dg_status st;
  if (!h->stage_src && (st = dev_alloc(h, &h->stage_src, bytes)) != DG_OK) return st;
  if (!h->stage_dst && (st = dev_alloc(h, &h->stage_dst, bytes)) != DG_OK) return st;
  DG_CUDA(h, cudaMemsetAsync(h->stage_src, 0, bytes, h->stream));
  cudaEvent_t e0, e1;
  DG_CUDA(h, cudaEventCreate(&e0));
  DG_CUDA(h, cudaEventCreate(&e1));
  const int saved = h->cpb;
  int best = saved;
  float best_t = 1e30f;
  st = DG_OK;
  for (int c : tile_choices(h)) {
    h->cpb = c;
    for (int w = 0; w < 2 && st == DG_OK; ++w) st = launch_apply(h, h->stage_src, h->stage_dst, nullptr);
    if (st != DG_OK) break;
    cudaEventRecord(e0, h->stream);
    const int reps = 5;
    for (int r = 0; r < reps && st == DG_OK; ++r) st = launch_apply(h, h->stage_src, h->stage_dst, nullptr);
    cudaEventRecord(e1, h->stream);
    if (st != DG_OK) break;
    cudaError_t e = cudaEventSynchronize(e1);
    if (e != cudaSuccess) {
      st = cuda_fail(h, e, "autotune timing");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (ms < best_t) {
      best_t = ms;
      best = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->cpb = st == DG_OK ? best : saved;
  if (best_cpb) *best_cpb = h->cpb;
  if (best_ms) *best_ms = best_t;
  return st;
}

dg_status dg_destroy(dg_handle* h) {
  if (!h) return DG_OK;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
  return DG_OK;
}

const char* dg_last_error(const dg_handle* h) {
  if (!h) return g_setup_error.c_str();
  return h->err.c_str();
}

}  // extern "C"
