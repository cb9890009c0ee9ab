// Fused element-centric DG apply kernel for the binary64 and double-float
// operators (one launch per operator evaluation; the binary32 operator has
// its own kernel in dg_apply_f32.cuh).
//
// Each CUDA block owns C consecutive cells (C k^2 threads; thread (a,b) of a
// cell owns one line of k points in whichever direction a phase sweeps).
// For every cell the block computes, in shared memory:
//   1. gather the cell's k^3 contiguous dofs (Algorithm 1 step (ii)(a));
//   2. basis change S (x) S (x) S to the Gauss points and the collocation
//      derivative D^co along x, y, z (Eq. tensor_to_collocation);
//   3. for the six faces, one direction at a time: the neighbour's traces
//      from its Gauss-Lobatto dofs through S_f / D_f and the in-face S (x) S
//      and derivative steps of Eq. (face_integral); the own traces by
//      extrapolating the Gauss-point fields to xi = 0 / 1; the numerical flux
//      of Eq. (poisson_sip) or Eq. (advection) at each face point (Algorithm 1
//      steps (iii)(c), (iv)(c)); the test coefficients of this cell's side;
//   4. the quadrature-point operation with the stored geometry (Sec. 5: G3
//      J^{-1} and det J w, G4 merged coefficient, or Cartesian constants) and
//      the injection of the face test coefficients into the Gauss-point fields;
//   5. the transposed derivative and basis change (integration), and a set
//      (not add) of the cell's dst entries (the remark after Algorithm 1).
// Every face is evaluated once from each side; each cell's result is written
// exactly once, with no atomics and a fixed summation order.
//
// All 1D matrices are read with compile-time indices from the kernel
// parameters (constant bank operands); the few values indexed by thread
// position (E, W) are copied to shared memory first.
#pragma once

#include <cstring>
#include <type_traits>

#include "dg_df64.cuh"
#include "dg_internal.cuh"

namespace dg {

// Vector storage type and conversions for each arithmetic type: float and
// double vectors are used as they are; the double-float arithmetic reads and
// writes binary64 vectors.
template <typename T>
struct Arith {
  using V = T;
  static __device__ __forceinline__ T load(const V* p) { return *p; }
  static __device__ __forceinline__ void store(V* p, T v) { *p = v; }
  static __device__ __forceinline__ double to_double(T v) { return (double)v; }
};
template <>
struct Arith<df64> {
  using V = double;
  static __device__ __forceinline__ df64 load(const double* p) { return dfp::df_from_double(*p); }
  static __device__ __forceinline__ void store(double* p, df64 v) { *p = dfp::df_to_double(v); }
  static __device__ __forceinline__ double to_double(df64 v) { return dfp::df_to_double(v); }
};

// Dot-product accumulation: a chain of FMAs, or for double-float a
// compensated sum renormalized once.
template <typename T>
struct Acc {
  T v;
  __device__ __forceinline__ void init() { v = T(0); }
  __device__ __forceinline__ void init(T c) { v = c; }
  __device__ __forceinline__ void add(T a, T b) { v = fma(a, b, v); }
  __device__ __forceinline__ T get() const { return v; }
};
template <>
struct Acc<df64> : DfAcc {};

// 1 / x in the kernel arithmetic (binary64 division; double-float Newton step)
template <typename T>
__device__ __forceinline__ T recip_of(T x) {
  return T(1) / x;
}
template <>
__device__ __forceinline__ df64 recip_of<df64>(df64 x) {
  return dfp::df_recip(x);
}

// Geometry variant G2 (Sec. 5): the Jacobian at Gauss point (a, b, c) of a
// cell whose k^3 Gauss-point positions X[i][k^3] (component i, x fastest)
// are in shared memory, by the collocation derivative D^co along the three
// lines through the point (J[i][d] = dx_i / dxi_d); J^{-1} by the adjugate
// (Ji[r*3 + s] = (J^{-1})_{rs}).  Returns det J.
template <int K, typename T>
__device__ __forceinline__ T g2_inverse_jacobian(const T* __restrict__ D, const T* X0, const T* X1, const T* X2,
                                                 int a, int b, int c, T (&Ji)[9]) {
  T J[9];
  const T* X[3] = {X0, X1, X2};
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Acc<T> s0, s1, s2;
    s0.init();
    s1.init();
    s2.init();
#pragma unroll
    for (int j = 0; j < K; ++j) {
      s0.add(D[a * K + j], X[i][j + K * (b + K * c)]);
      s1.add(D[b * K + j], X[i][a + K * (j + K * c)]);
      s2.add(D[c * K + j], X[i][a + K * (b + K * j)]);
    }
    J[i * 3 + 0] = s0.get();
    J[i * 3 + 1] = s1.get();
    J[i * 3 + 2] = s2.get();
  }
  const T c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
  const T det = J[0] * c00 + J[1] * c01 + J[2] * c02;
  const T r = recip_of(det);
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

template <typename T>
struct ApplyParams {
  Tables<T> tab;
  Geometry<T> geo;
  const typename Arith<T>::V* src;
  typename Arith<T>::V* dst;
  double* dot_partial;
  const double* skip;  // optional device flag: the launch does nothing while *skip != 0
  int C;  // cells per block
  int64_t cell_begin, cell_end;  // cells of this launch
};

// Per-operator part of the launch parameters (all but the 1D tables), for
// the batched launches that cover the blocks of several operators of one
// degree, arithmetic, geometry variant, weak form and tile shape.
template <typename T>
struct OpParams {
  Geometry<T> geo;
  const typename Arith<T>::V* src;
  typename Arith<T>::V* dst;
  double* dot_partial;
  const double* skip;
  int C;
  int64_t cell_begin, cell_end;
  SplitArrays split;  // face-loop work arrays (face-loop operators only)
};

// Parameters of a batched launch: the shared tables and up to kBatchOps
// operators; block b of the launch is block b - block_start[i] of operator i
// (block_start ascending, block_start[nops] = the grid size).
template <typename T>
struct BatchParams {
  Tables<T> tab;
  int nops;
  int block_start[kBatchOps + 1];
  OpParams<T> op[kBatchOps];
};
static_assert(sizeof(BatchParams<double>) <= 32000, "batched launch parameters exceed the kernel parameter space");

// operator of block b: the last i with block_start[i] <= b (binary search)
template <typename T>
__device__ __forceinline__ int batch_op(const BatchParams<T>& B, int b) {
  int lo = 0, hi = B.nops - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.block_start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <int K>
struct Shape {
  static constexpr int max_threads = cells_per_block(K) * K * K;
};

template <int K, int OP>
struct Smem {
  static constexpr int NBA = OP == OP_SIPG ? 2 : 1;  // value and normal derivative of the neighbour
  static constexpr int NBB = OP == OP_SIPG ? 3 : 1;  // after the first in-face sweep: value, d_n, d_t1
                                                     // (FP64 per-point variant uses the first NBA)
  static constexpr int FTF = OP == OP_SIPG ? 4 : 1;  // face test fields per face
  static constexpr int per_cell = smem_scalars_per_cell(K, OP);
};

// The outer (output) loops of the line helpers unroll UQ times: fully for
// binary64 (matrix entries become constant-bank operands), not at
// all for double-float, whose 12-instruction products would otherwise
// overflow the instruction cache (its matrices are then read from shared
// memory).

// v[base + q stride] = sum_i M[q][i] v[base + i stride]   (TR: M[i][q])
template <int K, bool TR, int UQ, typename T>
__device__ __forceinline__ void line_apply(const T* __restrict__ M, T* v, int base, int stride) {
  T in[K];
#pragma unroll
  for (int i = 0; i < K; ++i) in[i] = v[base + i * stride];
#pragma unroll(UQ)
  for (int q = 0; q < K; ++q) {
    Acc<T> s;
    s.init();
#pragma unroll
    for (int i = 0; i < K; ++i) s.add(TR ? M[i * K + q] : M[q * K + i], in[i]);
    v[base + q * stride] = s.get();
  }
}

// out[ob + q os] = sum_i M[q][i] in[ib + i is]
template <int K, int UQ, typename T>
__device__ __forceinline__ void line_apply_to(const T* __restrict__ M, const T* in, int ib, int is, T* out, int ob,
                                              int os) {
  T x[K];
#pragma unroll
  for (int i = 0; i < K; ++i) x[i] = in[ib + i * is];
#pragma unroll(UQ)
  for (int q = 0; q < K; ++q) {
    Acc<T> s;
    s.init();
#pragma unroll
    for (int i = 0; i < K; ++i) s.add(M[q * K + i], x[i]);
    out[ob + q * os] = s.get();
  }
}

// v[base + j stride] += sum_q M[q][j] t[base + q stride]
template <int K, int UQ, typename T>
__device__ __forceinline__ void line_add_transposed(const T* __restrict__ M, const T* t, T* v, int base,
                                                    int stride) {
  T x[K];
#pragma unroll
  for (int q = 0; q < K; ++q) x[q] = t[base + q * stride];
#pragma unroll(UQ)
  for (int j = 0; j < K; ++j) {
    Acc<T> s;
    s.init(v[base + j * stride]);
#pragma unroll
    for (int q = 0; q < K; ++q) s.add(M[q * K + j], x[q]);
    v[base + j * stride] = s.get();
  }
}

// Even-odd form of a 1D kernel (Sec. 4.1): out = M in for a
// centrosymmetric (ANTI = false: S, S^T) or anti-centrosymmetric (ANTI =
// true: D, D^T) k x k matrix from its even and odd halves ME, MO (see
// Tables::EO): about k^2/2 + 2k operations instead of k^2.
// Even-odd split of a line (Sec. 4.1): e_i = u_i + u_{k-1-i}, o_i = u_i -
// u_{k-1-i} for i < k/2, and e_{k/2} = u_{k/2} for odd k.
template <int K, typename T>
__device__ __forceinline__ void eo_split(const T (&in)[K], T (&e)[(K + 1) / 2], T (&o)[K / 2]) {
  constexpr int h = K / 2;
#pragma unroll
  for (int i = 0; i < h; ++i) {
    e[i] = in[i] + in[K - 1 - i];
    o[i] = in[i] - in[K - 1 - i];
  }
  if (K % 2) e[h] = in[h];
}

// out = M in from the split line, M centrosymmetric (ANTI false) or
// anti-centrosymmetric (ANTI true) with even-odd halves ME, MO.
template <int K, bool ANTI, typename T>
__device__ __forceinline__ void eo_combine(const T* __restrict__ ME, const T* __restrict__ MO,
                                           const T (&e)[(K + 1) / 2], const T (&o)[K / 2], T (&out)[K]) {
  constexpr int h = K / 2, H2 = (K + 1) / 2;
#pragma unroll
  for (int q = 0; q < h; ++q) {
    T ev = ME[q * kHalf] * e[0];
#pragma unroll
    for (int i = 1; i < H2; ++i) ev = fma(ME[q * kHalf + i], e[i], ev);
    T od = MO[q * kHalf] * o[0];
#pragma unroll
    for (int i = 1; i < h; ++i) od = fma(MO[q * kHalf + i], o[i], od);
    out[q] = ev + od;
    out[K - 1 - q] = ANTI ? od - ev : ev - od;
  }
  if (K % 2) {
    T mid;
    if (!ANTI) {
      mid = ME[h * kHalf] * e[0];
#pragma unroll
      for (int i = 1; i < H2; ++i) mid = fma(ME[h * kHalf + i], e[i], mid);
    } else {
      mid = MO[h * kHalf] * o[0];
#pragma unroll
      for (int i = 1; i < h; ++i) mid = fma(MO[h * kHalf + i], o[i], mid);
    }
    out[h] = mid;
  }
}

template <int K, bool ANTI, typename T>
__device__ __forceinline__ void eo_line(const T* __restrict__ ME, const T* __restrict__ MO, const T (&in)[K],
                                        T (&out)[K]) {
  T e[(K + 1) / 2], o[K / 2];
  eo_split<K>(in, e, o);
  eo_combine<K, ANTI>(ME, MO, e, o, out);
}

// The sweeps of the binary64 kernel in even-odd form (k >= 5, where it saves
// operations): S or S^T in place on a line, D from a line to a line, and
// v += D^T t along a line.
template <int K, int WHICH, typename T>
__device__ __forceinline__ void eo_apply(const Tables<T>& tb, T* v, int base, int stride) {
  T in[K], out[K];
#pragma unroll
  for (int i = 0; i < K; ++i) in[i] = v[base + i * stride];
  eo_line<K, false>(tb.EO[WHICH][0], tb.EO[WHICH][1], in, out);
#pragma unroll
  for (int i = 0; i < K; ++i) v[base + i * stride] = out[i];
}
template <int K, typename T>
__device__ __forceinline__ void eo_derivative_to(const Tables<T>& tb, const T* in, int ib, int is, T* out_, int ob,
                                                 int os) {
  T x[K], out[K];
#pragma unroll
  for (int i = 0; i < K; ++i) x[i] = in[ib + i * is];
  eo_line<K, true>(tb.EO[EO_D][0], tb.EO[EO_D][1], x, out);
#pragma unroll
  for (int i = 0; i < K; ++i) out_[ob + i * os] = out[i];
}
template <int K, typename T>
__device__ __forceinline__ void eo_add_derivative_transposed(const Tables<T>& tb, const T* t, T* v, int base,
                                                             int stride) {
  T x[K], out[K];
#pragma unroll
  for (int i = 0; i < K; ++i) x[i] = t[base + i * stride];
  eo_line<K, true>(tb.EO[EO_DT][0], tb.EO[EO_DT][1], x, out);
#pragma unroll
  for (int i = 0; i < K; ++i) v[base + i * stride] += out[i];
}

// start of the line along direction d through tangential indices (a, b)
template <int K>
__device__ __forceinline__ int line_base(int d, int a, int b) {
  return d == 0 ? K * (a + K * b) : d == 1 ? a + K * K * b : a + K * b;
}

__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.L2 [%0];" ::"l"(p));
}

// The element-centric apply of one block (blk) of an operator: the body of
// apply_kernel (one operator) and apply_kernel_batch (several).
template <int K, typename T, int GEO, int OP, typename PP>
__device__ __forceinline__ void apply_body(const Tables<T>& tb, const PP& P, const int blk) {
  constexpr int K2 = K * K, K3 = K2 * K;
  const int C = P.C;
  constexpr int NBA = Smem<K, OP>::NBA, NBB = Smem<K, OP>::NBB, FTF = Smem<K, OP>::FTF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* U = reinterpret_cast<T*>(smem_raw);  // [C][K3] u -> u at Gauss points -> test value field
  T* G = U + C * K3;                      // [3][C][K3] gradients -> test gradient fields
  T* NBa = G + 3 * C * K3;                // [C][2][NBA][K2] neighbour traces
  T* NBb = NBa + C * 2 * NBA * K2;        // [C][2][NBB][K2]
  T* FT = NBb + C * 2 * NBB * K2;         // [C][3][2][FTF][K2] face test coefficients
  T* sE = FT + C * 6 * FTF * K2;          // [2][K]
  T* sW = sE + 2 * K;                     // [K]
  T* sS = sW + K;                         // [K][K] (rows indexed by thread position)
  T* sD = sS + K2;                        // [K][K]
  constexpr bool kCompact = std::is_same<T, df64>::value;
  constexpr int kUq = kCompact ? 1 : K;     // unroll of the sweep output loops
  constexpr int kUd = kCompact ? 1 : 3;     // unroll of the face-direction loop
  using A = Arith<T>;

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

  // 0. start the HBM fetch of this block's cell geometry into L2; it is read
  // in phase 4, after the sweeps and face work
  if (GEO != GEO_CART) {
    constexpr int NA = GEO == GEO_FULL ? (OP == OP_SIPG ? 9 : 10) : (OP == OP_SIPG ? 6 : 3);
    const char* base = reinterpret_cast<const char*>(gm.cell + cell0 * K3);
    const int64_t bytes = (int64_t)nloc * K3 * (int64_t)sizeof(T);
    const int lines = (int)((bytes + 127) / 128) + 1;
    for (int t = tid; t < NA * lines; t += blockDim.x) {
      const int a = t / lines, l = t - a * lines;
      const char* p = base + a * gm.ncq * (int64_t)sizeof(T) + (int64_t)l * 128;
      if (p < base + a * gm.ncq * (int64_t)sizeof(T) + bytes) prefetch_l2(p);
    }
  }

  int ijk[3];
  {
    // cell counts stay below 2^31 (checked at set-up): 32-bit division
    const unsigned c = (unsigned)(active ? cell : cell0);
    const unsigned q = c / (unsigned)gm.n[0];
    ijk[0] = (int)(c - q * (unsigned)gm.n[0]);
    ijk[1] = (int)(q % (unsigned)gm.n[1]);
    ijk[2] = (int)(q / (unsigned)gm.n[1]);
  }
  // ... and of the six faces' geometry of each cell (read in phase 3)
  if (GEO != GEO_CART && active) {
    constexpr int NFA = OP == OP_SIPG ? 7 : 1;
    constexpr int LPS = (K2 * (int)sizeof(T) + 127) / 128 + 1;  // lines per face segment
    for (int t = ln; t < 6 * NFA * LPS; t += K2) {
      const int face = t / (NFA * LPS), a = (t / LPS) % NFA, l = t % LPS;
      const int d = face >> 1, sd = face & 1;
      // selects instead of indexing ijk / n by d keep everything in registers
      const int id = d == 0 ? ijk[0] : d == 1 ? ijk[1] : ijk[2];
      const int it1 = d == 0 ? ijk[1] : ijk[0], it2 = d == 2 ? ijk[1] : ijk[2];
      const int nd = d == 0 ? gm.n[0] : d == 1 ? gm.n[1] : gm.n[2];
      const int nt1 = d == 0 ? gm.n[1] : gm.n[0];
      const int Pd = d == 0 ? gm.P[0] : d == 1 ? gm.P[1] : gm.P[2];
      const T* fbase = d == 0 ? gm.face[0] : d == 1 ? gm.face[1] : gm.face[2];
      const int64_t nfqd = d == 0 ? gm.nfq[0] : d == 1 ? gm.nfq[1] : gm.nfq[2];
      int pos = id + sd;
      if (gm.periodic && pos == nd) pos = 0;
      const int64_t fidp = (int64_t)(pos + Pd * (it1 + nt1 * it2));
      const char* seg = reinterpret_cast<const char*>(fbase + a * nfqd + fidp * K2);
      const char* p = seg + l * 128;
      if (p < seg + K2 * (int)sizeof(T)) prefetch_l2(p);
    }
  }

  if (tid < 2 * K) sE[tid] = tb.E[tid / K][tid % K];
  if (tid < K) sW[tid] = tb.W[tid];
  for (int i = tid; i < K2; i += blockDim.x) {
    sS[i] = tb.S[i];
    sD[i] = tb.D[i];
  }

  // 1. gather (coalesced over the block's contiguous range)
  {
    const typename A::V* s = P.src + cell0 * K3;
    for (int i = tid; i < nloc * K3; i += blockDim.x) U[i] = A::load(s + i);
  }
  __syncthreads();

  // 2. basis change to the Gauss points, x then y then z; collocation derivatives
  const T* mS = kCompact ? sS : tb.S;
  const T* mD = kCompact ? sD : tb.D;
  // binary64 sweeps in even-odd form where that saves operations (k >= 5)
  constexpr bool kEO = !kCompact && K >= 5;
  auto sweep_S = [&](int base, int stride) {
    if constexpr (kEO) eo_apply<K, EO_S>(tb, Uc, base, stride);
    else line_apply<K, false, kUq>(mS, Uc, base, stride);
  };
  auto sweep_D = [&](int base, int stride, T* out) {
    if constexpr (kEO) eo_derivative_to<K>(tb, Uc, base, stride, out, base, stride);
    else line_apply_to<K, kUq>(mD, Uc, base, stride, out, base, stride);
  };
  if (active) sweep_S(K * (la + K * lb), 1);
  __syncthreads();
  if (active) sweep_S(la + K2 * lb, K);
  __syncthreads();
  if (active) sweep_S(la + K * lb, K2);
  __syncthreads();
  if (OP == OP_SIPG) {
    if (active) {
      sweep_D(K * (la + K * lb), 1, G0);
      sweep_D(la + K2 * lb, K, G1);
      sweep_D(la + K * lb, K2, G2);
    }
    __syncthreads();
  }

  // 3. faces, one direction at a time.  The loop is unrolled (d constant)
  // except for double-float; direction-dependent values are selects, so the
  // body is valid for a runtime d.
#pragma unroll(kUd)
  for (int d = 0; d < 3; ++d) {
    const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
    const int strd = d == 0 ? 1 : d == 1 ? K : K2;
    const int id = d == 0 ? ijk[0] : d == 1 ? ijk[1] : ijk[2];
    const int it1 = d == 0 ? ijk[1] : ijk[0], it2 = d == 2 ? ijk[1] : ijk[2];
    const int nd = d == 0 ? gm.n[0] : d == 1 ? gm.n[1] : gm.n[2];
    const int nt1 = d == 0 ? gm.n[1] : gm.n[0];
    const int Pd = d == 0 ? gm.P[0] : d == 1 ? gm.P[1] : gm.P[2];
    const T* fgeo = d == 0 ? gm.face[0] : d == 1 ? gm.face[1] : gm.face[2];
    const int64_t nfqd = d == 0 ? gm.nfq[0] : d == 1 ? gm.nfq[1] : gm.nfq[2];
    const T cjd = d == 0 ? gm.cart_jinv[0] : d == 1 ? gm.cart_jinv[1] : gm.cart_jinv[2];
    const T ctaud = d == 0 ? gm.cart_tau[0] : d == 1 ? gm.cart_tau[1] : gm.cart_tau[2];
    const T veld = d == 0 ? gm.vel[0] : d == 1 ? gm.vel[1] : gm.vel[2];
    int64_t nbc[2];
    int64_t fid[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      int jd = id + (s ? 1 : -1);
      int pos = id + s;
      bool inside = jd >= 0 && jd < nd;
      if (!inside && gm.periodic) {
        jd = jd < 0 ? nd - 1 : 0;
        inside = true;
      }
      if (gm.periodic && pos == nd) pos = 0;
      const int j0 = d == 0 ? jd : ijk[0], j1 = d == 1 ? jd : ijk[1], j2 = d == 2 ? jd : ijk[2];
      nbc[s] = inside ? (int64_t)(j0 + gm.n[0] * (j1 + gm.n[1] * j2)) : -1;
      fid[s] = (int64_t)(pos + Pd * (it1 + nt1 * it2));
    }
    T* nba = NBa + lc * 2 * NBA * K2;  // [2][NBA][K2]
    T* nbb = NBb + lc * 2 * NBB * K2;  // [2][NBB][K2]
    // 3a. neighbour's face-normal interpolation from its Gauss-Lobatto dofs:
    // the value is the layer on the shared face, the normal derivative uses D_f
    if (active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (nbc[s] < 0) continue;
        const typename A::V* un = P.src + nbc[s] * K3 + line_base<K>(d, la, lb);
        T v[K];
#pragma unroll
        for (int l = 0; l < K; ++l) v[l] = A::load(un + l * strd);
        nba[(s * NBA) * K2 + ln] = s ? v[0] : v[K - 1];
        if (OP == OP_SIPG) {
          Acc<T> dv;
          dv.init();
#pragma unroll
          for (int l = 0; l < K; ++l) dv.add(tb.DF[1 - s][l], v[l]);
          nba[(s * NBA + 1) * K2 + ln] = dv.get();
        }
      }
    }
    __syncthreads();
    // 3b. in-face interpolation of the neighbour's traces to the face Gauss
    // points, one thread per face point so that every lane works (the FP64
    // pipe is charged per warp instruction).
    // along t1 (output point (qa = la, j = lb)), then along t2 (point (i = la, qb = lb))
    if (active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (nbc[s] < 0) continue;
#pragma unroll
        for (int f = 0; f < NBA; ++f) {
          const T* in = nba + (s * NBA + f) * K2;
          Acc<T> acc;
          acc.init();
#pragma unroll
          for (int i = 0; i < K; ++i) acc.add(sS[la * K + i], in[i + K * lb]);
          nbb[(s * NBB + f) * K2 + ln] = acc.get();
        }
      }
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (nbc[s] < 0) continue;
#pragma unroll
        for (int f = 0; f < NBA; ++f) {
          const T* in = nbb + (s * NBB + f) * K2;
          Acc<T> acc;
          acc.init();
#pragma unroll
          for (int j = 0; j < K; ++j) acc.add(sS[lb * K + j], in[la + K * j]);
          nba[(s * NBA + f) * K2 + ln] = acc.get();
        }
      }
    }
    __syncthreads();
    // neighbour derivative along this cell's outward normal at point (la, lb)
    T dnn[2] = {T(0), T(0)};
    if (OP == OP_SIPG && active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        if (nbc[s] < 0) continue;
        const T* nbt = nba + s * NBA * K2;
        if (GEO == GEO_CART) {
          dnn[s] = (s ? T(1) : T(-1)) * cjd * nbt[K2 + ln];
        } else {
          Acc<T> a1, a2;
          a1.init();
          a2.init();
#pragma unroll
          for (int i = 0; i < K; ++i) {
            a1.add(sD[la * K + i], nbt[i + K * lb]);
            a2.add(sD[lb * K + i], nbt[la + K * i]);
          }
          // reference-axis components: d carries the normal derivative,
          // t1 < t2 the two tangential ones
          const T gdn = nbt[K2 + ln], ga1 = a1.get(), ga2 = a2.get();
          const T gx = d == 0 ? gdn : ga1;
          const T gy = d == 1 ? gdn : (d == 0 ? ga1 : ga2);
          const T gz = d == 2 ? gdn : ga2;
          const T* fp = fgeo + fid[s] * K2 + ln;
          dnn[s] = -(fp[(s * 3 + 0) * nfqd] * gx + fp[(s * 3 + 1) * nfqd] * gy + fp[(s * 3 + 2) * nfqd] * gz);
        }
      }
    }
    if (OP == OP_SIPG) {
      __syncthreads();  // every read of the d_n field is done before it is overwritten
      if (active) {
#pragma unroll
        for (int s = 0; s < 2; ++s)
          if (nbc[s] >= 0) nba[(s * NBA + 1) * K2 + ln] = dnn[s];
      }
    }
    __syncthreads();
    // 3c. numerical flux at face point (la, lb) of both faces of direction d
    if (active) {
      const int base = line_base<K>(d, la, lb);
      T lu[K], lg0[K], lg1[K], lg2[K];
#pragma unroll
      for (int j = 0; j < K; ++j) {
        lu[j] = Uc[base + j * strd];
        if (OP == OP_SIPG) {
          lg0[j] = G0[base + j * strd];
          lg1[j] = G1[base + j * strd];
          lg2[j] = G2[base + j * strd];
        }
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const bool interior = nbc[s] >= 0;
        const T sg = s ? T(1) : T(-1);
        Acc<T> au;
        au.init();
#pragma unroll
        for (int j = 0; j < K; ++j) au.add(tb.E[s][j], lu[j]);
        const T u = au.get();
        const T* nbt = nba + s * NBA * K2;
        const T un = interior ? nbt[ln] : T(0);
        T* ft = FT + (((lc * 3 + d) * 2 + s) * FTF) * K2 + ln;
        if (OP == OP_SIPG) {
          Acc<T> ag0, ag1, ag2;
          ag0.init();
          ag1.init();
          ag2.init();
#pragma unroll
          for (int j = 0; j < K; ++j) {
            const T e = tb.E[s][j];
            ag0.add(e, lg0[j]);
            ag1.add(e, lg1[j]);
            ag2.add(e, lg2[j]);
          }
          T g[3] = {ag0.get(), ag1.get(), ag2.get()};
          const T dnn = interior ? nbt[K2 + ln] : T(0);
          T jo[3], dno, tv, tg;
          if (GEO == GEO_CART) {
            const T jn = sg * cjd;
            jo[0] = d == 0 ? jn : T(0);
            jo[1] = d == 1 ? jn : T(0);
            jo[2] = d == 2 ? jn : T(0);
            dno = jn * (d == 0 ? g[0] : d == 1 ? g[1] : g[2]);
            T kap = T(1);
            if (gm.kq) kap = d == 0 ? gm.kf[ijk[0] + s] : gm.kq[ijk[0] * K + la];
            const T fjxw = kap * sW[la] * sW[lb] * gm.cart_detj * cjd, tau = ctaud;
            if (interior) {
              const T jump = u - un;
              tv = fjxw * (tau * jump - T(0.5) * (dno + dnn));
              tg = T(-0.5) * fjxw * jump;
            } else {
              tv = fjxw * (T(2) * tau * u - dno);
              tg = -fjxw * u;
            }
          } else {
            // stored with the weight w = kappa da w folded in: w j_n per side
            // (so dno and dnn carry w) and w tau
            const T* fp = fgeo + fid[s] * K2 + ln;
            const int so = 1 - s;  // own slot: the lower side of the face is slot 0
            jo[0] = fp[(so * 3 + 0) * nfqd];
            jo[1] = fp[(so * 3 + 1) * nfqd];
            jo[2] = fp[(so * 3 + 2) * nfqd];
            dno = jo[0] * g[0] + jo[1] * g[1] + jo[2] * g[2];
            const T wtau = fp[6 * nfqd];
            if (interior) {
              const T jump = u - un;
              tv = wtau * jump - T(0.5) * (dno + dnn);
              tg = T(-0.5) * jump;
            } else {
              tv = T(2) * wtau * u - dno;
              tg = -u;
            }
          }
          ft[0] = tv;
          ft[K2] = tg * jo[0];
          ft[2 * K2] = tg * jo[1];
          ft[3 * K2] = tg * jo[2];
        } else {
          T cn;
          if (GEO == GEO_CART) {
            cn = veld * sW[la] * sW[lb] * gm.cart_detj * cjd;
          } else {
            cn = fgeo[fid[s] * K2 + ln];
          }
          const T cno = s ? cn : -cn;  // c.n da w with n the own outward normal
          ft[0] = interior ? T(0.5) * cno * (u + un) + T(0.5) * fabs(cno) * (u - un) : fabs(cno) * u;
        }
      }
    }
    __syncthreads();
  }

  // 4. quadrature-point operation and injection of the face test coefficients
  if (active) {
    const T e0a = sE[la], e1a = sE[K + la], e0b = sE[lb], e1b = sE[K + lb];
    const T* ftc = FT + lc * 6 * FTF * K2;
#pragma unroll(kCompact ? 1 : K)
    for (int z = 0; z < K; ++z) {
      const int pt = la + K * (lb + K * z);
      T fv, fg0 = T(0), fg1 = T(0), fg2 = T(0);
      {
        // x faces: along = la, proj = lb + K z; y faces: along = lb, proj = la + K z;
        // z faces: along = z, proj = la + K lb
        const T* fx0 = ftc + (0 * 2 + 0) * FTF * K2 + lb + K * z;
        const T* fx1 = ftc + (0 * 2 + 1) * FTF * K2 + lb + K * z;
        const T* fy0 = ftc + (1 * 2 + 0) * FTF * K2 + la + K * z;
        const T* fy1 = ftc + (1 * 2 + 1) * FTF * K2 + la + K * z;
        const T* fz0 = ftc + (2 * 2 + 0) * FTF * K2 + la + K * lb;
        const T* fz1 = ftc + (2 * 2 + 1) * FTF * K2 + la + K * lb;
        const T ez0 = kCompact ? sE[z] : tb.E[0][z], ez1 = kCompact ? sE[K + z] : tb.E[1][z];
        auto inj = [&](int f) {
          Acc<T> a;
          a.init();
          a.add(e0a, fx0[f * K2]);
          a.add(e1a, fx1[f * K2]);
          a.add(e0b, fy0[f * K2]);
          a.add(e1b, fy1[f * K2]);
          a.add(ez0, fz0[f * K2]);
          a.add(ez1, fz1[f * K2]);
          return a.get();
        };
        fv = inj(0);
        if (OP == OP_SIPG) {
          fg0 = inj(1);
          fg1 = inj(2);
          fg2 = inj(3);
        }
      }
      T t0, t1, t2;
      const int64_t qi = cell * K3 + pt;
      if (OP == OP_SIPG) {
        const T g0 = G0[pt], g1 = G1[pt], g2 = G2[pt];
        if (GEO == GEO_CART) {
          T w = sW[la] * sW[lb] * (kCompact ? sW[z] : tb.W[z]) * gm.cart_detj;
          if (gm.kq) w *= gm.kq[ijk[0] * K + la];
          t0 = w * gm.cart_jinv[0] * gm.cart_jinv[0] * g0;
          t1 = w * gm.cart_jinv[1] * gm.cart_jinv[1] * g1;
          t2 = w * gm.cart_jinv[2] * gm.cart_jinv[2] * g2;
        } else if (GEO == GEO_FULL) {
          // stored: s J^{-1} with s = sqrt(kappa JxW); grad_x u = J^{-T}
          // grad_xi u, flux = kappa JxW grad_x u, t = J^{-1} flux = (sJ^{-1}) (sJ^{-1})^T grad_xi u
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
          const T w = -sW[la] * sW[lb] * (kCompact ? sW[z] : tb.W[z]) * gm.cart_detj;
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
      G0[pt] = t0 + fg0;
      G1[pt] = t1 + fg1;
      G2[pt] = t2 + fg2;
      Uc[pt] = fv;
    }
  }
  __syncthreads();

  // 5. integration: V += D^T T_x, D^T T_y, D^T T_z, then S^T along z, y, x
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

  // write (set) the block's contiguous range; optional src . dst partial
  {
    typename A::V* o = P.dst + cell0 * K3;
    double acc = 0.0;
    const typename A::V* s = P.src + cell0 * K3;
    const bool dot = P.dot_partial != nullptr;
    for (int i = tid; i < nloc * K3; i += blockDim.x) {
      const T v = U[i];
      A::store(o + i, v);
      if (dot) acc += A::to_double(v) * (double)s[i];
    }
    if (dot) {
      // the gradient region is free now; its start (rounded up to 8 bytes)
      // holds blockDim doubles
      double* red = reinterpret_cast<double*>(
          smem_raw + ((size_t)C * K3 * sizeof(T) + 7) / 8 * 8);
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
__global__ void __launch_bounds__(Shape<K>::max_threads) apply_kernel(const __grid_constant__ ApplyParams<T> P) {
  if (P.skip != nullptr && *P.skip != 0.0) return;
  apply_body<K, T, GEO, OP>(P.tab, P, (int)blockIdx.x);
}

template <int K, typename T, int GEO, int OP>
__global__ void __launch_bounds__(Shape<K>::max_threads) apply_kernel_batch(const __grid_constant__ BatchParams<T> B) {
  const int i = batch_op(B, (int)blockIdx.x);
  apply_body<K, T, GEO, OP>(B.tab, B.op[i], (int)blockIdx.x - B.block_start[i]);
}

template <int K, typename T, int GEO, int OP>
cudaError_t launch_one(const ApplyLaunch& L, int64_t n_cells) {
  ApplyParams<T> P;
  P.tab = *static_cast<const Tables<T>*>(L.tables);
  P.geo = *static_cast<const Geometry<T>*>(L.geometry);
  P.src = static_cast<const typename Arith<T>::V*>(L.src);
  P.dst = static_cast<typename Arith<T>::V*>(L.dst);
  P.dot_partial = L.dot_partial;
  P.skip = L.skip;
  const int C = (L.cpb >= 1 && L.cpb <= cells_per_block(K)) ? L.cpb : cells_per_block(K);
  P.C = C;
  P.cell_begin = L.cell_begin;
  P.cell_end = L.cell_end;
  const int smem = smem_bytes_per_block(K, OP, (int)sizeof(T), C);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(apply_kernel<K, T, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes_per_block(K, OP, (int)sizeof(T), cells_per_block(K)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  (void)n_cells;
  const int64_t grid = (L.cell_end - L.cell_begin + C - 1) / C;
  if (grid <= 0) return cudaSuccess;
  apply_kernel<K, T, GEO, OP><<<(unsigned)grid, C * K * K, smem, L.stream>>>(P);
  return cudaGetLastError();
}

template <int K, typename T>
cudaError_t launch_prec(const ApplyLaunch& L, int64_t n_cells) {
  if (L.geo == GEO_POS) return cudaErrorInvalidValue;  // G2 runs the face loop (binary64, double-float)
  if (L.op == OP_SIPG) {
    if (L.geo == GEO_CART) return launch_one<K, T, GEO_CART, OP_SIPG>(L, n_cells);
    if (L.geo == GEO_FULL) return launch_one<K, T, GEO_FULL, OP_SIPG>(L, n_cells);
    return launch_one<K, T, GEO_MERGED, OP_SIPG>(L, n_cells);
  }
  if (L.geo == GEO_CART) return launch_one<K, T, GEO_CART, OP_ADV>(L, n_cells);
  if (L.geo == GEO_FULL) return launch_one<K, T, GEO_FULL, OP_ADV>(L, n_cells);
  return launch_one<K, T, GEO_MERGED, OP_ADV>(L, n_cells);
}

}  // namespace dg

#include "dg_apply_f32.cuh"
#include "dg_apply_split.cuh"

namespace dg {

template <int K>
cudaError_t launch_apply(const ApplyLaunch& L, int64_t n_cells) {
  if (L.prec != 1 && L.face_mode != 0) return launch_apply_split<K>(L);
  if (L.prec == 0) return launch_prec<K, double>(L, n_cells);
  if (L.prec == 1) return launch_apply_f32<K>(L, n_cells);
  return launch_prec<K, df64>(L, n_cells);
}

// ---- batched launches: the blocks of several operators in one grid ----

// Kernel parameters of a batched launch with tile shape C; returns the grid
// size (blocks of all operators, largest-first order as given).
template <typename T>
int fill_batch(BatchParams<T>& B, const BatchLaunch& L, int C) {
  B.tab = *static_cast<const Tables<T>*>(L.tables);
  B.nops = L.nops;
  int start = 0;
  for (int i = 0; i < L.nops; ++i) {
    const BatchOp& o = L.ops[i];
    OpParams<T>& q = B.op[i];
    q.geo = *static_cast<const Geometry<T>*>(o.geometry);
    q.src = static_cast<const typename Arith<T>::V*>(o.src);
    q.dst = static_cast<typename Arith<T>::V*>(o.dst);
    q.dot_partial = nullptr;
    q.skip = nullptr;
    q.C = C;
    q.cell_begin = 0;
    q.cell_end = o.n_cells;
    if (o.split) q.split = *static_cast<const SplitArrays*>(o.split);
    else memset(&q.split, 0, sizeof(q.split));
    B.block_start[i] = start;
    start += (int)((o.n_cells + C - 1) / C);
  }
  B.block_start[L.nops] = start;
  return start;
}

template <int K, typename T, int GEO, int OP>
cudaError_t launch_batch_one(const BatchLaunch& L) {
  const int C = (L.cpb >= 1 && L.cpb <= cells_per_block(K)) ? L.cpb : cells_per_block(K);
  static thread_local BatchParams<T> B;  // large (kernel parameter space): not on the stack
  const int grid = fill_batch<T>(B, L, C);
  if (grid <= 0) return cudaSuccess;
  if (L.face_mode != 0) {
    static bool configured = false;
    if (!configured) {
      cudaError_t e = cudaFuncSetAttribute(split_forward_batch<K, T, GEO, OP>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           split_smem_forward(K, cells_per_block(K), GEO));
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(split_backward_batch<K, T, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 split_smem_backward(K, OP, cells_per_block(K)));
      if (e != cudaSuccess) return e;
      configured = true;
    }
    split_forward_batch<K, T, GEO, OP><<<grid, C * K * K, split_smem_forward(K, C, GEO), L.stream>>>(B);
    split_backward_batch<K, T, GEO, OP><<<grid, C * K * K, split_smem_backward(K, OP, C), L.stream>>>(B);
    return cudaGetLastError();
  }
  if constexpr (GEO == GEO_POS) {
    return cudaErrorInvalidValue;  // G2 binary64 / double-float operators run the face loop only
  } else {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(apply_kernel_batch<K, T, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem_bytes_per_block(K, OP, (int)sizeof(T), cells_per_block(K)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  apply_kernel_batch<K, T, GEO, OP>
      <<<grid, C * K * K, smem_bytes_per_block(K, OP, (int)sizeof(T), C), L.stream>>>(B);
  return cudaGetLastError();
  }
}

template <int K, int C, int GEO, int OP>
cudaError_t launch_batch_f32_one(const BatchLaunch& L) {
  static thread_local BatchParams<float> B;
  const int grid = fill_batch<float>(B, L, C);
  if (grid <= 0) return cudaSuccess;
  const int smem = f32_smem_bytes(K, OP, C, GEO);
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(apply_f32_batch<K, C, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int want = f32_min_blocks(K, C, OP) * (smem + 1024);
    const int pct = want >= 228 * 1024 ? 100 : (want * 100 + 228 * 1024 - 1) / (228 * 1024);
    e = cudaFuncSetAttribute(apply_f32_batch<K, C, GEO, OP>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  apply_f32_batch<K, C, GEO, OP><<<grid, C * K * K, smem, L.stream>>>(B);
  return cudaGetLastError();
}

template <int K, int C>
cudaError_t launch_batch_f32_tile(const BatchLaunch& L) {
  if (L.op == OP_SIPG) {
    if (L.geo == GEO_CART) return launch_batch_f32_one<K, C, GEO_CART, OP_SIPG>(L);
    if (L.geo == GEO_FULL) return launch_batch_f32_one<K, C, GEO_FULL, OP_SIPG>(L);
    if (L.geo == GEO_POS) return launch_batch_f32_one<K, C, GEO_POS, OP_SIPG>(L);
    return launch_batch_f32_one<K, C, GEO_MERGED, OP_SIPG>(L);
  }
  if (L.geo == GEO_CART) return launch_batch_f32_one<K, C, GEO_CART, OP_ADV>(L);
  if (L.geo == GEO_FULL) return launch_batch_f32_one<K, C, GEO_FULL, OP_ADV>(L);
  if (L.geo == GEO_POS) return launch_batch_f32_one<K, C, GEO_POS, OP_ADV>(L);
  return launch_batch_f32_one<K, C, GEO_MERGED, OP_ADV>(L);
}

template <int K, typename T>
cudaError_t launch_batch_prec(const BatchLaunch& L) {
  if (L.op == OP_SIPG) {
    if (L.geo == GEO_CART) return launch_batch_one<K, T, GEO_CART, OP_SIPG>(L);
    if (L.geo == GEO_FULL) return launch_batch_one<K, T, GEO_FULL, OP_SIPG>(L);
    if (L.geo == GEO_POS) return launch_batch_one<K, T, GEO_POS, OP_SIPG>(L);
    return launch_batch_one<K, T, GEO_MERGED, OP_SIPG>(L);
  }
  if (L.geo == GEO_CART) return launch_batch_one<K, T, GEO_CART, OP_ADV>(L);
  if (L.geo == GEO_FULL) return launch_batch_one<K, T, GEO_FULL, OP_ADV>(L);
  if (L.geo == GEO_POS) return launch_batch_one<K, T, GEO_POS, OP_ADV>(L);
  return launch_batch_one<K, T, GEO_MERGED, OP_ADV>(L);
}

template <int K>
cudaError_t launch_batch(const BatchLaunch& L) {
  if (L.nops < 1 || L.nops > kBatchOps) return cudaErrorInvalidValue;
  if (L.prec == 0) return launch_batch_prec<K, double>(L);
  if (L.prec == 2) return launch_batch_prec<K, df64>(L);
  if (L.cpb == F32Tiles<K>::large) return launch_batch_f32_tile<K, F32Tiles<K>::large>(L);
  if (L.cpb == F32Tiles<K>::small) return launch_batch_f32_tile<K, F32Tiles<K>::small>(L);
  return cudaErrorInvalidValue;
}

}  // namespace dg

#define DG_DEFINE_APPLY_LAUNCHER(KK)                                              \
  namespace dg {                                                                  \
  cudaError_t launch_apply_k##KK(const ApplyLaunch& L, int64_t n_cells) {         \
    return launch_apply<KK>(L, n_cells);                                          \
  }                                                                               \
  cudaError_t launch_batch_k##KK(const BatchLaunch& L) { return launch_batch<KK>(L); } \
  }
