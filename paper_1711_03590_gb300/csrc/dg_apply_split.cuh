// Face-loop variant of the binary64 apply: the neighbour's traces are read,
// not recomputed.
//
// The fused kernel (dg_apply.cuh) is element-centric: each cell evaluates
// its six faces and re-interpolates the neighbour's traces from its
// Gauss-Lobatto dofs (S_f, D_f and the in-face sweeps of Eq. face_integral).
// On GB300 the binary64 apply is bound by the FP64 pipe (1/64 of the binary32
// rate) while HBM is nearly idle, so this variant trades memory traffic for
// arithmetic, in the spirit of the paper's separate cell and face loops
// (Algorithm 1 steps (ii)-(iv)), without atomics, in two launches:
//
//   1. cell kernel: gather, S (x) S (x) S and D^co sweeps; the cell's own
//      traces on its six faces (u and the reference gradient, by the
//      Gauss-collocation extrapolation E_s) are written per face and slot
//      (slot 0: the cell below the face along its direction, slot 1: the
//      cell above); the q-point operation (Sec. 5 geometry) writes the
//      gradient-test fields at the Gauss points;
//   2. cell kernel: for each face point of its six faces, the numerical
//      flux (Eq. poisson_sip / advection) from both slots' traces and the
//      face geometry, tested on this cell's side (value and reference
//      gradient, Algorithm 1 step (iii)(c)); the gradient-test fields and
//      the faces' test coefficients are injected (transpose of E_s) and
//      integrated (D^co^T, S^T (x) S^T (x) S^T); dst is set.
//
// Each side's flux evaluation is its own (the paper's face loop evaluates
// once and adds into both sides; here each side writes only its own cell).
// Work arrays (per operator, allocated when the mode is selected): traces
// [face][slot][field][k^2] per direction and three gradient-test fields
// [field][cell][k^3].  A launch covers a range of cells; the backward launch
// of a range needs the forward launch of the range and of its neighbours.
// The results equal the fused kernel's up to rounding (same method, other
// operation order).
#pragma once

#include <cstdint>
#include <type_traits>

namespace dg {

template <int OP>
struct SplitFields {
  static constexpr int NTR = OP == OP_SIPG ? 4 : 1;  // u (+ reference gradient)
  static constexpr int NFT = OP == OP_SIPG ? 4 : 1;  // value test (+ gradient test)
};

// Face id (pos + P_d (i_t1 + n_t1 i_t2)) of side s (0: lower face, 1: upper
// face) of cell ijk in direction d.
__device__ __forceinline__ int split_face_id(const int ijk[3], int d, int s, const int n[3], const int P[3],
                                             int periodic) {
  const int id = d == 0 ? ijk[0] : d == 1 ? ijk[1] : ijk[2];
  const int it1 = d == 0 ? ijk[1] : ijk[0], it2 = d == 2 ? ijk[1] : ijk[2];
  const int nd = d == 0 ? n[0] : d == 1 ? n[1] : n[2];
  const int nt1 = d == 0 ? n[1] : n[0];
  const int Pd = d == 0 ? P[0] : d == 1 ? P[1] : P[2];
  int pos = id + s;
  if (periodic && pos == nd) pos = 0;
  return pos + Pd * (it1 + nt1 * it2);
}

// Shared tables of the double-float kernels (rolled loops read their
// matrices from shared memory): E_0, E_1, W, S, D.
template <int K>
__host__ __device__ constexpr int split_table_scalars() {
  return 3 * K + 2 * K * K;
}

// Step 1: sweeps, own traces, q-point operation.  T: double (binary64) or
// df64 (double-float on the FP32 pipe; vectors, traces and gradient-test
// fields are stored as 8-byte values either way).
template <int K, typename T, int GEO, int OP, typename PP>
__device__ __forceinline__ void split_forward_body(const Tables<T>& tb, const PP& P, const SplitArrays& SA,
                                                   const int blk) {
  using A = Arith<T>;
  constexpr int K2 = K * K, K3 = K2 * K;
  constexpr int NTR = SplitFields<OP>::NTR;
  constexpr bool kCompact = std::is_same<T, df64>::value;
  constexpr bool kEO = !kCompact && K >= 5;
  constexpr int kUq = kCompact ? 1 : K;  // unroll of the sweep output loops
  constexpr int kUz = kCompact ? 1 : K;  // unroll of the q-point loop
  constexpr int kUd = kCompact ? 1 : 3;  // unroll of the trace-direction loop
  const int C = P.C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // [C][K3]
  T* G = U + C * K3;                      // [3][C][K3]
  T* sE = G + 3 * C * K3;                 // [2][K] (double-float only)
  T* sW = sE + 2 * K;                     // [K]
  T* sS = sW + K;                         // [K][K]
  T* sD = sS + K2;                        // [K][K]
  T* XP = sD + K2;                        // [3][C][K3] Gauss-point positions (G2 only)
  T* const tr_out[3] = {reinterpret_cast<T*>(SA.tr[0]), reinterpret_cast<T*>(SA.tr[1]),
                        reinterpret_cast<T*>(SA.tr[2])};
  T* const tq_out = reinterpret_cast<T*>(SA.tq);
  const Geometry<T>& gm = P.geo;
  const int tid = threadIdx.x;
  const int lc = tid / K2;
  const int ln = tid - lc * K2;
  const int la = ln % K, lb = ln / K;
  const int64_t cell0 = P.cell_begin + (int64_t)blk * C;
  const int64_t cell = cell0 + lc;
  const bool active = cell < P.cell_end;
  const int nloc = (int)min((int64_t)C, P.cell_end - cell0);
  T* Uc = U + lc * K3;
  T* G0 = G + lc * K3;
  T* G1 = G + (C + lc) * K3;
  T* G2 = G + (2 * C + lc) * K3;
  int ijk[3];
  {
    const unsigned c = (unsigned)(active ? cell : cell0);
    const unsigned q = c / (unsigned)gm.n[0];
    ijk[0] = (int)(c - q * (unsigned)gm.n[0]);
    ijk[1] = (int)(q % (unsigned)gm.n[1]);
    ijk[2] = (int)(q / (unsigned)gm.n[1]);
  }
  for (int i = tid; i < nloc * K3; i += blockDim.x) U[i] = A::load(P.src + cell0 * K3 + i);
  if constexpr (GEO == GEO_POS) {
    for (int i = tid; i < nloc * K3; i += blockDim.x) {
      const int64_t q = cell0 * K3 + i;
      XP[i] = gm.cell[q];
      XP[C * K3 + i] = gm.cell[gm.ncq + q];
      XP[2 * C * K3 + i] = gm.cell[2 * gm.ncq + q];
    }
  }
  if constexpr (kCompact) {
    if (tid < 2 * K) sE[tid] = tb.E[tid / K][tid % K];
    if (tid < K) sW[tid] = tb.W[tid];
    for (int i = tid; i < K2; i += blockDim.x) {
      sS[i] = tb.S[i];
      sD[i] = tb.D[i];
    }
  }
  __syncthreads();
  const T* mS = kCompact ? sS : tb.S;
  const T* mD = kCompact ? sD : tb.D;
  const T* mE0 = kCompact ? sE : tb.E[0];
  const T* mE1 = kCompact ? sE + K : tb.E[1];
  const T* mW = kCompact ? sW : tb.W;
  auto sweep_S = [&](int base, int stride) {
    if constexpr (kEO) eo_apply<K, EO_S>(tb, Uc, base, stride);
    else line_apply<K, false, kUq>(mS, Uc, base, stride);
  };
  auto sweep_D = [&](int base, int stride, T* out) {
    if constexpr (kEO) eo_derivative_to<K>(tb, Uc, base, stride, out, base, stride);
    else line_apply_to<K, kUq>(mD, Uc, base, stride, out, base, stride);
  };
  // S along z, y, then x: before the x sweep the x-line (y = la, z = lb)
  // holds the coefficients along x at the Gauss points in y and z, and its
  // end layers are the cell's x-face traces of u at face point (la, lb)
  // (both bases take the face value from the end layer alone: Lagrange on
  // Gauss-Lobatto points, and the Hermite-like basis by construction)
  T xu[2] = {T(0), T(0)};
  if (active) sweep_S(la + K * lb, K2);
  __syncthreads();
  if (active) sweep_S(la + K2 * lb, K);
  __syncthreads();
  if (active) {
    xu[0] = Uc[K * (la + K * lb)];
    xu[1] = Uc[K * (la + K * lb) + K - 1];
    sweep_S(K * (la + K * lb), 1);
  }
  __syncthreads();
  if (OP == OP_SIPG) {
    if (active) {
      sweep_D(K * (la + K * lb), 1, G0);
      sweep_D(la + K2 * lb, K, G1);
      sweep_D(la + K * lb, K2, G2);
    }
    __syncthreads();
  }
  if (!active) return;

  // own traces on the six faces: this cell is slot 1 of its lower face
  // (s = 0) and slot 0 of its upper face (s = 1)
#pragma unroll(kUd)
  for (int d = 0; d < 3; ++d) {
    const int base = line_base<K>(d, la, lb);
    const int strd = d == 0 ? 1 : d == 1 ? K : K2;
    T lu[K], lg[3][K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      lu[j] = Uc[base + j * strd];
      if (OP == OP_SIPG) {
        lg[0][j] = G0[base + j * strd];
        lg[1][j] = G1[base + j * strd];
        lg[2][j] = G2[base + j * strd];
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T v[NTR];
#pragma unroll
      for (int f = 0; f < NTR; ++f) v[f] = T(0);
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const T e = s ? mE1[j] : mE0[j];
        if (d != 0) v[0] = fma(e, lu[j], v[0]);
        if (OP == OP_SIPG) {
#pragma unroll
          for (int c = 0; c < 3; ++c) v[1 + c] = fma(e, lg[c][j], v[1 + c]);
        }
      }
      if (d == 0) v[0] = xu[s];
      const int fid = split_face_id(ijk, d, s, gm.n, gm.P, gm.periodic);
      T* out = (d == 0 ? tr_out[0] : d == 1 ? tr_out[1] : tr_out[2]) + ((int64_t)(fid * 2 + (1 - s)) * NTR) * K2 + ln;
#pragma unroll
      for (int f = 0; f < NTR; ++f) out[f * K2] = v[f];
    }
  }

  // q-point operation: the gradient-test fields t_c at the Gauss points
  const T wa = mW[la], wb = mW[lb];
#pragma unroll(kUz)
  for (int z = 0; z < K; ++z) {
    const int pt = la + K * (lb + K * z);
    const int64_t qi = cell * K3 + pt;
    T t0, t1, t2;
    if (OP == OP_SIPG) {
      const T g0 = G0[pt], g1 = G1[pt], g2 = G2[pt];
      if (GEO == GEO_CART) {
        T w = wa * wb * mW[z] * gm.cart_detj;
        if (gm.kq) w *= gm.kq[ijk[0] * K + la];
        t0 = w * gm.cart_jinv[0] * gm.cart_jinv[0] * g0;
        t1 = w * gm.cart_jinv[1] * gm.cart_jinv[1] * g1;
        t2 = w * gm.cart_jinv[2] * gm.cart_jinv[2] * g2;
      } else if (GEO == GEO_FULL) {
        // stored: s J^{-1} with s = sqrt(kappa JxW), so t = (sJ^{-1}) (sJ^{-1})^T grad_xi u
        const T* cp = gm.cell + qi;
        const int64_t n = gm.ncq;
        T J[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) J[m] = cp[m * n];
        const T x0 = J[0] * g0 + J[3] * g1 + J[6] * g2;
        const T x1 = J[1] * g0 + J[4] * g1 + J[7] * g2;
        const T x2 = J[2] * g0 + J[5] * g1 + J[8] * g2;
        t0 = J[0] * x0 + J[1] * x1 + J[2] * x2;
        t1 = J[3] * x0 + J[4] * x1 + J[5] * x2;
        t2 = J[6] * x0 + J[7] * x1 + J[8] * x2;
      } else if (GEO == GEO_POS) {
        // G2: J from the positions; kappa stored per point (array 3)
        T Ji[9];
        const T det = g2_inverse_jacobian<K, T>(mD, XP + lc * K3, XP + (C + lc) * K3, XP + (2 * C + lc) * K3, la,
                                                lb, z, Ji);
        const T kw = gm.cell[3 * gm.ncq + qi] * det * (wa * wb * mW[z]);
        const T x0 = kw * (Ji[0] * g0 + Ji[3] * g1 + Ji[6] * g2);
        const T x1 = kw * (Ji[1] * g0 + Ji[4] * g1 + Ji[7] * g2);
        const T x2 = kw * (Ji[2] * g0 + Ji[5] * g1 + Ji[8] * g2);
        t0 = Ji[0] * x0 + Ji[1] * x1 + Ji[2] * x2;
        t1 = Ji[3] * x0 + Ji[4] * x1 + Ji[5] * x2;
        t2 = Ji[6] * x0 + Ji[7] * x1 + Ji[8] * x2;
      } else {
        const T* cp = gm.cell + qi;
        const int64_t n = gm.ncq;
        const T a00 = cp[0], a01 = cp[n], a02 = cp[2 * n], a11 = cp[3 * n], a12 = cp[4 * n], a22 = cp[5 * n];
        t0 = a00 * g0 + a01 * g1 + a02 * g2;
        t1 = a01 * g0 + a11 * g1 + a12 * g2;
        t2 = a02 * g0 + a12 * g1 + a22 * g2;
      }
    } else {
      const T uq = Uc[pt];
      T b0, b1, b2;
      if (GEO == GEO_CART) {
        const T w = -(wa * wb * mW[z] * gm.cart_detj);
        b0 = w * gm.cart_jinv[0] * gm.vel[0];
        b1 = w * gm.cart_jinv[1] * gm.vel[1];
        b2 = w * gm.cart_jinv[2] * gm.vel[2];
      } else if (GEO == GEO_FULL) {
        const T* cp = gm.cell + qi;
        const int64_t n = gm.ncq;
        T J[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) J[m] = cp[m * n];
        const T jw = -cp[9 * n];
        b0 = jw * (J[0] * gm.vel[0] + J[1] * gm.vel[1] + J[2] * gm.vel[2]);
        b1 = jw * (J[3] * gm.vel[0] + J[4] * gm.vel[1] + J[5] * gm.vel[2]);
        b2 = jw * (J[6] * gm.vel[0] + J[7] * gm.vel[1] + J[8] * gm.vel[2]);
      } else if (GEO == GEO_POS) {
        T Ji[9];
        const T det = g2_inverse_jacobian<K, T>(mD, XP + lc * K3, XP + (C + lc) * K3, XP + (2 * C + lc) * K3, la,
                                                lb, z, Ji);
        const T jw = -(det * (wa * wb * mW[z]));
        b0 = jw * (Ji[0] * gm.vel[0] + Ji[1] * gm.vel[1] + Ji[2] * gm.vel[2]);
        b1 = jw * (Ji[3] * gm.vel[0] + Ji[4] * gm.vel[1] + Ji[5] * gm.vel[2]);
        b2 = jw * (Ji[6] * gm.vel[0] + Ji[7] * gm.vel[1] + Ji[8] * gm.vel[2]);
      } else {
        const T* cp = gm.cell + qi;
        const int64_t n = gm.ncq;
        b0 = cp[0];
        b1 = cp[n];
        b2 = cp[2 * n];
      }
      t0 = b0 * uq;
      t1 = b1 * uq;
      t2 = b2 * uq;
    }
    tq_out[qi] = t0;
    tq_out[gm.ncq + qi] = t1;
    tq_out[2 * gm.ncq + qi] = t2;
  }
}

// Numerical flux at face point fp (qa = fp mod K along t1, qb along t2) of
// face fid of direction d, tested on slot so (Eq. poisson_sip / advection,
// Algorithm 1 step (iii)(c)): u, g are both slots' traces (value and
// reference gradient; the other slot's are read only if `interior`).  Writes
// the value test and (SIPG) the reference-gradient test of slot so to
// ft[0], ft[fs], ft[2 fs], ft[3 fs].
template <int K, typename T, int GEO, int OP>
__device__ __forceinline__ void split_slot_flux(const T* W, const Geometry<T>& gm, int d, int64_t fid, int pos,
                                                int it1, int fp, int so, bool interior, const T (&u)[2],
                                                const T (&g)[2][3], T* ft, int fs) {
  constexpr int K2 = K * K;
  const int la = fp % K, lb = fp / K;
  const int sn = 1 - so;
  const T cjd = gm.cart_jinv[d];
  if (OP == OP_SIPG) {
    // j_n per slot (each side's own outward normal: +d for slot 0); with
    // per-point geometry stored as w j_n and w tau (w = kappa da w), so
    // that dno and dnn carry the weight
    T jo[3], jn[3], w, wtau;
    if (GEO == GEO_CART) {
      const T j = so == 0 ? cjd : -cjd;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        jo[c] = c == d ? j : T(0);
        jn[c] = -jo[c];
      }
      T kap = T(1);
      if (gm.kq) kap = d == 0 ? gm.kf[pos] : gm.kq[it1 * K + la];
      w = kap * W[la] * W[lb] * gm.cart_detj * cjd;
      wtau = w * gm.cart_tau[d];
    } else {
      const T* f = gm.face[d] + fid * K2 + fp;
      const int64_t nfq = gm.nfq[d];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        jo[c] = f[(so * 3 + c) * nfq];
        jn[c] = f[(sn * 3 + c) * nfq];
      }
      wtau = f[6 * nfq];
    }
    const T dno = jo[0] * g[so][0] + jo[1] * g[so][1] + jo[2] * g[so][2];
    T tv, tg;
    if (GEO == GEO_CART) {
      if (interior) {
        const T dnn = -(jn[0] * g[sn][0] + jn[1] * g[sn][1] + jn[2] * g[sn][2]);
        const T jump = u[so] - u[sn];
        tv = w * (gm.cart_tau[d] * jump - T(0.5) * (dno + dnn));
        tg = T(-0.5) * w * jump;
      } else {
        tv = w * (T(2) * gm.cart_tau[d] * u[so] - dno);
        tg = -w * u[so];
      }
    } else if (interior) {
      // the neighbour's derivative along this side's outward normal
      const T dnn = -(jn[0] * g[sn][0] + jn[1] * g[sn][1] + jn[2] * g[sn][2]);
      const T jump = u[so] - u[sn];
      tv = wtau * jump - T(0.5) * (dno + dnn);
      tg = T(-0.5) * jump;
    } else {
      tv = T(2) * wtau * u[so] - dno;
      tg = -u[so];
    }
    ft[0] = tv;
#pragma unroll
    for (int c = 0; c < 3; ++c) ft[(1 + c) * fs] = tg * jo[c];
  } else {
    T cn;
    if (GEO == GEO_CART) cn = gm.vel[d] * W[la] * W[lb] * gm.cart_detj * cjd;
    else cn = gm.face[d][fid * K2 + fp];
    const T cno = so == 0 ? cn : -cn;  // c.n da w with n this side's outward normal
    ft[0] = interior ? T(0.5) * cno * (u[so] + u[sn]) + T(0.5) * fabs(cno) * (u[so] - u[sn]) : fabs(cno) * u[so];
  }
}

// Step 2: the numerical flux of this cell's slot on its six faces from both
// slots' traces, injection of the test coefficients, integration, dst.
template <int K, typename T, int GEO, int OP, typename PP>
__device__ __forceinline__ void split_backward_body(const Tables<T>& tb, const PP& P, const SplitArrays& SA,
                                                    const int blk) {
  using A = Arith<T>;
  constexpr int K2 = K * K, K3 = K2 * K;
  constexpr int NTR = SplitFields<OP>::NTR, NFT = SplitFields<OP>::NFT;
  constexpr bool kCompact = std::is_same<T, df64>::value;
  constexpr bool kEO = !kCompact && K >= 5;
  constexpr int kUq = kCompact ? 1 : K;  // unroll of the sweep output loops
  constexpr int kUz = kCompact ? 1 : K;  // unroll of the injection loop
  constexpr int kUd = kCompact ? 1 : 3;  // unroll of the face-direction loop
  const int C = P.C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // [C][K3]
  T* G = U + C * K3;                      // [3][C][K3]
  T* FT = G + 3 * C * K3;                 // [C][3][2][NFT][K2]: test coefficients of the six faces
  T* sE = FT + C * 6 * NFT * K2;          // [2][K] (double-float only)
  T* sW = sE + 2 * K;                     // [K]
  T* sS = sW + K;                         // [K][K]
  T* sD = sS + K2;                        // [K][K]
  const T* const tr_in[3] = {reinterpret_cast<const T*>(SA.tr[0]), reinterpret_cast<const T*>(SA.tr[1]),
                             reinterpret_cast<const T*>(SA.tr[2])};
  const T* const tq_in = reinterpret_cast<const T*>(SA.tq);
  const Geometry<T>& gm = P.geo;
  const int tid = threadIdx.x;
  const int lc = tid / K2;
  const int ln = tid - lc * K2;
  const int la = ln % K, lb = ln / K;
  const int64_t cell0 = P.cell_begin + (int64_t)blk * C;
  const int64_t cell = cell0 + lc;
  const bool active = cell < P.cell_end;
  const int nloc = (int)min((int64_t)C, P.cell_end - cell0);
  T* Uc = U + lc * K3;
  T* G0 = G + lc * K3;
  T* G1 = G + (C + lc) * K3;
  T* G2 = G + (2 * C + lc) * K3;
  for (int i = tid; i < nloc * K3; i += blockDim.x) {
    const int64_t q = cell0 * K3 + i;
    G[i] = tq_in[q];
    G[C * K3 + i] = tq_in[gm.ncq + q];
    G[2 * C * K3 + i] = tq_in[2 * gm.ncq + q];
  }
  if constexpr (kCompact) {
    if (tid < 2 * K) sE[tid] = tb.E[tid / K][tid % K];
    if (tid < K) sW[tid] = tb.W[tid];
    for (int i = tid; i < K2; i += blockDim.x) {
      sS[i] = tb.S[i];
      sD[i] = tb.D[i];
    }
  }
  const T* mS = kCompact ? sS : tb.S;
  const T* mD = kCompact ? sD : tb.D;
  const T* mE0 = kCompact ? sE : tb.E[0];
  const T* mE1 = kCompact ? sE + K : tb.E[1];
  const T* mW = kCompact ? sW : tb.W;
  if constexpr (kCompact) __syncthreads();  // the shared tables are read below
  if (active) {
    int ijk[3];
    const unsigned c = (unsigned)cell;
    const unsigned q = c / (unsigned)gm.n[0];
    ijk[0] = (int)(c - q * (unsigned)gm.n[0]);
    ijk[1] = (int)(q % (unsigned)gm.n[1]);
    ijk[2] = (int)(q / (unsigned)gm.n[1]);
    // this cell's slot of face (d, s) is 1 - s
#pragma unroll(kUd)
    for (int d = 0; d < 3; ++d) {
#pragma unroll(kUd == 1 ? 1 : 2)
      for (int s = 0; s < 2; ++s) {
        const int fid = split_face_id(ijk, d, s, gm.n, gm.P, gm.periodic);
        T* dst = FT + (((lc * 3 + d) * 2 + s) * NFT) * K2 + ln;
        const int id = ijk[d], nd = gm.n[d];
        const bool interior = gm.periodic || (s ? id + 1 < nd : id >= 1);
        int pos = id + s;
        if (gm.periodic && pos == nd) pos = 0;
        const int it1 = d == 0 ? ijk[1] : ijk[0];
        T u[2] = {T(0), T(0)}, g[2][3] = {{T(0), T(0), T(0)}, {T(0), T(0), T(0)}};
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
          if (sl == s && !interior) continue;  // slot s is the neighbour's
          const T* tr = (d == 0 ? tr_in[0] : d == 1 ? tr_in[1] : tr_in[2]) + ((int64_t)fid * 2 + sl) * NTR * K2 + ln;
          u[sl] = tr[0];
          if (OP == OP_SIPG) {
#pragma unroll
            for (int c = 0; c < 3; ++c) g[sl][c] = tr[(1 + c) * K2];
          }
        }
        split_slot_flux<K, T, GEO, OP>(mW, gm, d, fid, pos, it1, ln, 1 - s, interior, u, g, dst, K2);
      }
    }
  }
  __syncthreads();
  if (active) {
    const T e0a = mE0[la], e1a = mE1[la], e0b = mE0[lb], e1b = mE1[lb];
    const T* ftc = FT + lc * 6 * NFT * K2;
#pragma unroll(kUz)
    for (int z = 0; z < K; ++z) {
      const int pt = la + K * (lb + K * z);
      // x faces at (y=lb, z), y faces at (x=la, z), z faces at (x=la, y=lb)
      const T* fx0 = ftc + (0 * 2 + 0) * NFT * K2 + lb + K * z;
      const T* fx1 = ftc + (0 * 2 + 1) * NFT * K2 + lb + K * z;
      const T* fy0 = ftc + (1 * 2 + 0) * NFT * K2 + la + K * z;
      const T* fy1 = ftc + (1 * 2 + 1) * NFT * K2 + la + K * z;
      const T* fz0 = ftc + (2 * 2 + 0) * NFT * K2 + la + K * lb;
      const T* fz1 = ftc + (2 * 2 + 1) * NFT * K2 + la + K * lb;
      const T ez0 = mE0[z], ez1 = mE1[z];
      // the six faces' coefficients of field f extrapolated to the point
      // (E_s along each direction), accumulated onto a
      auto inj = [&](int f, T a) {
        a = fma(e0a, fx0[f * K2], a);
        a = fma(e1a, fx1[f * K2], a);
        a = fma(e0b, fy0[f * K2], a);
        a = fma(e1b, fy1[f * K2], a);
        a = fma(ez0, fz0[f * K2], a);
        return fma(ez1, fz1[f * K2], a);
      };
      {
        T a = e0a * fx0[0];
        a = fma(e1a, fx1[0], a);
        a = fma(e0b, fy0[0], a);
        a = fma(e1b, fy1[0], a);
        a = fma(ez0, fz0[0], a);
        Uc[pt] = fma(ez1, fz1[0], a);
      }
      if (OP == OP_SIPG) {
        G0[pt] = inj(1, G0[pt]);
        G1[pt] = inj(2, G1[pt]);
        G2[pt] = inj(3, G2[pt]);
      }
    }
  }
  __syncthreads();
  auto sweep_DT = [&](const T* t, int base, int stride) {
    if constexpr (kEO) eo_add_derivative_transposed<K>(tb, t, Uc, base, stride);
    else line_add_transposed<K, kUq>(mD, t, Uc, base, stride);
  };
  auto sweep_ST = [&](int base, int stride) {
    if constexpr (kEO) eo_apply<K, EO_ST>(tb, Uc, base, stride);
    else line_apply<K, true, kUq>(mS, Uc, base, stride);
  };
  if (active) sweep_DT(G0, K * (la + K * lb), 1);
  __syncthreads();
  if (active) sweep_DT(G1, la + K2 * lb, K);
  __syncthreads();
  if (active) {
    sweep_DT(G2, la + K * lb, K2);
    sweep_ST(la + K * lb, K2);
  }
  __syncthreads();
  if (active) sweep_ST(la + K2 * lb, K);
  __syncthreads();
  if (active) sweep_ST(K * (la + K * lb), 1);
  __syncthreads();
  {
    double* o = P.dst + cell0 * K3;
    const double* s = P.src + cell0 * K3;
    double acc = 0.0;
    const bool dot = P.dot_partial != nullptr;
    for (int i = tid; i < nloc * K3; i += blockDim.x) {
      A::store(o + i, U[i]);
      if (dot) acc += A::to_double(U[i]) * s[i];
    }
    if (dot) {
      double* red = reinterpret_cast<double*>(G);  // free now
      red[tid] = acc;
      __syncthreads();
      if (tid == 0) {
        double t = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) t += red[i];
        P.dot_partial[blk] = t;
      }
    }
  }
}

template <int K, typename T, int GEO, int OP>
__global__ void __launch_bounds__(Shape<K>::max_threads)
    split_cell_forward(const __grid_constant__ ApplyParams<T> P, const __grid_constant__ SplitArrays SA) {
  if (P.skip != nullptr && *P.skip != 0.0) return;
  split_forward_body<K, T, GEO, OP>(P.tab, P, SA, (int)blockIdx.x);
}
template <int K, typename T, int GEO, int OP>
__global__ void __launch_bounds__(Shape<K>::max_threads)
    split_cell_backward(const __grid_constant__ ApplyParams<T> P, const __grid_constant__ SplitArrays SA) {
  if (P.skip != nullptr && *P.skip != 0.0) return;
  split_backward_body<K, T, GEO, OP>(P.tab, P, SA, (int)blockIdx.x);
}
// The same over the blocks of several operators (one batched launch each)
template <int K, typename T, int GEO, int OP>
__global__ void __launch_bounds__(Shape<K>::max_threads)
    split_forward_batch(const __grid_constant__ BatchParams<T> B) {
  const int i = batch_op(B, (int)blockIdx.x);
  split_forward_body<K, T, GEO, OP>(B.tab, B.op[i], B.op[i].split, (int)blockIdx.x - B.block_start[i]);
}
template <int K, typename T, int GEO, int OP>
__global__ void __launch_bounds__(Shape<K>::max_threads)
    split_backward_batch(const __grid_constant__ BatchParams<T> B) {
  const int i = batch_op(B, (int)blockIdx.x);
  split_backward_body<K, T, GEO, OP>(B.tab, B.op[i], B.op[i].split, (int)blockIdx.x - B.block_start[i]);
}

template <int K, typename T, int GEO, int OP>
cudaError_t launch_split(const ApplyLaunch& L) {
  static_assert(sizeof(T) == 8, "traces and gradient-test fields are 8-byte scalars");
  ApplyParams<T> P;
  P.tab = *static_cast<const Tables<T>*>(L.tables);
  P.geo = *static_cast<const Geometry<T>*>(L.geometry);
  P.src = static_cast<const double*>(L.src);
  P.dst = static_cast<double*>(L.dst);
  P.dot_partial = L.dot_partial;
  P.skip = L.skip;
  const int C = (L.cpb >= 1 && L.cpb <= cells_per_block(K)) ? L.cpb : cells_per_block(K);
  P.C = C;
  P.cell_begin = L.cell_begin;
  P.cell_end = L.cell_end;
  const SplitArrays SA = *static_cast<const SplitArrays*>(L.split);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(split_cell_forward<K, T, GEO, OP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         split_smem_forward(K, cells_per_block(K), GEO));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(split_cell_backward<K, T, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               split_smem_backward(K, OP, cells_per_block(K)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int64_t grid = (L.cell_end - L.cell_begin + C - 1) / C;
  if (grid <= 0) return cudaSuccess;
  if (L.split_stage != 2)
    split_cell_forward<K, T, GEO, OP><<<(unsigned)grid, C * K * K, split_smem_forward(K, C, GEO), L.stream>>>(P, SA);
  if (L.split_stage != 1)
    split_cell_backward<K, T, GEO, OP>
        <<<(unsigned)grid, C * K * K, split_smem_backward(K, OP, C), L.stream>>>(P, SA);
  return cudaGetLastError();
}

template <int K, typename T>
cudaError_t launch_apply_split_t(const ApplyLaunch& L) {
  if (L.op == OP_SIPG) {
    if (L.geo == GEO_CART) return launch_split<K, T, GEO_CART, OP_SIPG>(L);
    if (L.geo == GEO_FULL) return launch_split<K, T, GEO_FULL, OP_SIPG>(L);
    if (L.geo == GEO_POS) return launch_split<K, T, GEO_POS, OP_SIPG>(L);
    return launch_split<K, T, GEO_MERGED, OP_SIPG>(L);
  }
  if (L.geo == GEO_CART) return launch_split<K, T, GEO_CART, OP_ADV>(L);
  if (L.geo == GEO_FULL) return launch_split<K, T, GEO_FULL, OP_ADV>(L);
  if (L.geo == GEO_POS) return launch_split<K, T, GEO_POS, OP_ADV>(L);
  return launch_split<K, T, GEO_MERGED, OP_ADV>(L);
}

// Binary64 (prec 0) and double-float (prec 2) face loops.
template <int K>
cudaError_t launch_apply_split(const ApplyLaunch& L) {
  return L.prec == 0 ? launch_apply_split_t<K, double>(L) : launch_apply_split_t<K, df64>(L);
}

}  // namespace dg
