// Internal declarations shared by the apply kernels and the C-ABI layer.
//
// Notation (Kronbichler & Kormann, arXiv:1711.03590):
//   k = p+1 points per direction; S = values of the k Gauss-Lobatto Lagrange
//   polynomials at the k Gauss points (basis change, Eq. tensor_to_collocation);
//   D = collocation derivative D^co on the Gauss points; the face kernels use
//   S_f / D_f of Eq. (face_integral) for the Gauss-Lobatto basis and the
//   extrapolation E_s of the Gauss-collocation basis to the faces xi = s.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dg {

constexpr int kMaxK = 9;  // degree 8
constexpr int kHalf = (kMaxK + 1) / 2;

// Geometry variants of the kernels (Sec. 5): Cartesian compression, G3 (full
// per-point Jacobians), G4 (merged coefficients), G2 (per-point positions;
// the Jacobian by a collocation derivative in the kernel)
enum Geo { GEO_CART = 0, GEO_FULL = 2, GEO_MERGED = 3, GEO_POS = 4 };
enum Op { OP_SIPG = 0, OP_ADV = 1 };

// 1D tables, passed by value as kernel parameters (constant bank).
template <typename T>
struct Tables {
  T S[kMaxK * kMaxK];   // S[q*k+i]  = l^GL_i(g_q)
  T D[kMaxK * kMaxK];   // D[q*k+j]  = (l^G_j)'(g_q), Gauss-collocation derivative
  T DS[kMaxK * kMaxK];  // DS[q*k+i] = (l^GL_i)'(g_q) = (D S)[q][i], GL derivative at the Gauss points
  T E[2][kMaxK];        // E[s][j]   = l^G_j(s), Gauss-collocation value at xi = s
  T DF[2][kMaxK];       // DF[s][i]  = (l^GL_i)'(s), GL derivative at xi = s
  T W[kMaxK];           // Gauss weights on [0,1]
  // Even-odd halves of S, S^T, D, D^T and DS (index EO_S, EO_ST, EO_D,
  // EO_DT, EO_DS) for the 1D kernels of Sec. 4.1: S is centrosymmetric
  // (M[q][i] = M[k-1-q][k-1-i]) and D and DS anti-centrosymmetric
  // (M[q][i] = -M[k-1-q][k-1-i]),
  // so with h = k/2, rows q < (k+1)/2 and e_i = u_i + u_{k-1-i},
  // o_i = u_i - u_{k-1-i} (i < h; e_h = u_h for odd k):
  //   ME[q][i] = (M[q][i] + M[q][k-1-i]) / 2 (i < h), ME[q][h] = M[q][h],
  //   MO[q][i] = (M[q][i] - M[q][k-1-i]) / 2 (i < h),
  // stored with row stride kHalf.
  T EO[5][2][kHalf * kHalf];
  // 1 for a basis with one nonzero in S_f and in D_f per end (the
  // Hermite-like basis: value from layer 0, normal derivative from layer 1,
  // mirrored at xi = 1): kernels may then read only those two layers of a
  // neighbour (the "slim" face access of Sec. 3.1)
  int slim;
};
enum { EO_S = 0, EO_ST = 1, EO_D = 2, EO_DT = 3, EO_DS = 4 };

// Device geometry and mesh description used by the apply kernel.
template <typename T>
struct Geometry {
  int n[3];
  int periodic;
  int64_t n_cells;
  // faces of direction d: positions P_d = periodic ? n_d : n_d + 1,
  // face id = pos + P_d (i_t1 + n_t1 i_t2), t1 < t2 the other directions
  int P[3];
  // FULL / MERGED cell arrays: structure of arrays, stride ncq = n_cells k^3
  // (binary64 and double-float); binary32: cell-blocked, see f32_geometry_block
  const T* __restrict__ cell;  // FULL SIPG: 9 sqrt(kappa JxW) J^{-1} (binary32: 9 J^{-1} + 1 kappa JxW);
                               // FULL ADV: 9 J^{-1} + 1 JxW;
                               // MERGED SIPG: 6; MERGED ADV: 3
  int64_t ncq;
  // face arrays per direction (stride nfq[d] = nfaces_d k^2)
  const T* __restrict__ face[3];  // SIPG: 6 w j_n (slot0 xyz, slot1 xyz) + 1 w tau, w = kappa da w;
                                  // ADV: 1 c.n da w (binary32 SIPG: j_n unscaled + w, and unless
                                  // face_pair only slot 0's 3 j_n + w)
  const T* __restrict__ tau[3];   // SIPG: penalty per face
  int64_t nfq[3];
  int nfc[3];  // faces per direction
  int face_pair;  // binary32 SIPG face arrays: 1 = both sides' j_n (7 arrays), 0 = one (4)
  // Cartesian compression
  T cart_jinv[3];       // n_d
  T cart_detj;          // 1 / (n0 n1 n2)
  T cart_tau[3];        // (p+1)^2 n_d penalty_scale
  const T* __restrict__ kq;  // kappa at cell Gauss x-positions [n0 k] (or null: kappa = 1)
  const T* __restrict__ kf;  // kappa at x-face positions [n0 + 1]
  T vel[3];             // advection velocity
};

// Work arrays of the face-loop variant of the binary64 apply (device
// pointers; dg_apply_split.cuh).
struct SplitArrays {
  double* tr[3];  // own traces per face of direction d: [face][slot][NTR][k^2]
  double* tq;     // gradient-test fields at the Gauss points: [3][n_cells k^3]
};

// Host-side description of one apply launch.
struct ApplyLaunch {
  int k;
  int prec;  // 0 double, 1 float
  int geo;
  int op;
  const void* src;
  void* dst;
  const void* tables;    // Tables<T>*
  const void* geometry;  // Geometry<T>*
  double* dot_partial;   // optional: per-block partial of src . dst (FP64)
  const double* skip;    // optional device flag: every block returns at once while *skip != 0
                         // (frozen iterations of the device-driven solvers)
  cudaStream_t stream;
  int cpb;               // cells per block (1 .. cells_per_block(k))
  int64_t cell_begin;    // the launch covers cells cell_begin .. cell_end - 1 (neighbours anywhere);
  int64_t cell_end;      // binary32: cell_begin a multiple of f32_geometry_block(k)
  int face_mode;         // binary64: 0 element-centric (fused kernel), 1 face loop (two launches)
  int split_stage;       // face loop: 0 the whole apply, 1 the cell-forward launch only, 2 the
                         // backward launch only (cell ranges: the forward launch of every
                         // neighbour of the range must have run)
  const void* split;     // SplitArrays* of the face loop
};

// Host description of one operator in a batched launch (one launch covering
// the blocks of several operators of the same degree, arithmetic, geometry
// variant, weak form, face mode and tile shape; dg_batch.cu).
constexpr int kBatchOps = 64;  // operators per batched launch (kernel parameter space)
struct BatchOp {
  const void* geometry;  // Geometry<T>*
  const void* src;
  void* dst;
  const void* split;     // SplitArrays* of a face-loop operator, else null
  int64_t n_cells;
};
struct BatchLaunch {
  int k, prec, geo, op, face_mode, cpb;
  const void* tables;    // Tables<T>* (the same for every operator of the launch)
  int nops;              // 1 .. kBatchOps
  const BatchOp* ops;
  cudaStream_t stream;
};

// Largest number of cells per block of the apply kernel for k points per
// direction (about 256 threads, k^2 per cell); also the default.  The block
// size is a launch parameter: any value 1 .. cells_per_block(k) is valid and
// the autotuner picks one per operator by timing.
__host__ __device__ constexpr int cells_per_block(int k) {
  return k == 2 ? 64 : k == 3 ? 28 : k == 4 ? 16 : k == 5 ? 10 : k == 6 ? 7 : k == 7 ? 5 : k == 8 ? 4 : 3;
}

// Default cells per block of the element-centric kernel and of the
// face-loop kernels (binary64, prec 0; double-float, prec 2), from sweeps of
// 1 .. cells_per_block(k) on the 32^3 deformed mesh (G3 SIPG) on GB300; any
// value 1 .. cells_per_block(k) is valid, and dg_autotune picks per operator.
__host__ __device__ constexpr int element_cells_per_block(int k, int prec) {
  return prec == 0 ? (k == 2 ? 8 : k == 3 ? 7 : k == 4 ? 8 : k == 5 ? 5 : k == 6 ? 6 : k == 7 ? 3 : k == 8 ? 2 : 3)
                   : (k == 2 ? 16 : k == 3 ? 7 : k == 4 ? 8 : k == 5 ? 5 : k == 6 ? 6 : k == 7 ? 3 : k == 8 ? 2 : 3);
}
__host__ __device__ constexpr int split_cells_per_block(int k, int prec) {
  return prec == 0 ? (k <= 3 ? 24 : k == 4 ? 8 : k == 5 ? 5 : k == 6 ? 7 : k == 7 ? 5 : 3)
                   : (k == 2 ? 24 : k == 3 ? 7 : k == 4 ? 4 : k == 5 ? 5 : k == 6 ? 7 : k == 7 ? 5 : 1);
}

// Shared-memory bytes of the face-loop kernels (C cells per block; 8-byte
// scalars, plus the double-float kernels' tables).
__host__ __device__ constexpr int split_smem_forward(int k, int C, int geo = 0) {
  return (4 * C * k * k * k + 3 * k + 2 * k * k + (geo == GEO_POS ? 3 * C * k * k * k : 0)) * 8;
}
__host__ __device__ constexpr int split_smem_backward(int k, int op, int C) {
  return (4 * C * k * k * k + C * 6 * (op == OP_SIPG ? 4 : 1) * k * k + 3 * k + 2 * k * k) * 8;
}

// Cell-block width of the binary32 kernel's cell geometry layout (the largest
// of its compiled tile shapes, which all divide it).
__host__ __device__ constexpr int f32_geometry_block(int k) {
  return k == 2 ? 32 : k == 3 ? 16 : 8;
}
// Compiled tile shapes (cells per block) of the binary32 kernel, and the
// default: the faster of the two on the 32^3 deformed G3 SIPG apply (GB300).
__host__ __device__ constexpr int f32_tile_small(int k) { return f32_geometry_block(k) / 2; }
__host__ __device__ constexpr int f32_tile_default(int k) {
  return k == 2 ? 32 : k == 3 ? 16 : k <= 6 ? 8 : 4;
}

// Faces per block of the binary32 face layout [face block][array][point]
// [face in block]: one block row is a 32-byte sector, and the faces of up to
// 8 consecutive cells are one contiguous chunk per direction and side.
constexpr int kFaceBlock = 8;

// Binary32 face numbering: faces of direction d numbered like cells, x
// fastest, with the face position pos in [0, P_d) in place of the index
// along d, so that the faces of consecutive cells are consecutive.  f is the
// face id pos + P_d (i_t1 + n_t1 i_t2).
__host__ __device__ inline int64_t face_minor_id(const int n[3], const int P[3], int d, int64_t f) {
  const int t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
  const int pos = (int)(f % P[d]);
  const int64_t rest = f / P[d];
  const int it1 = (int)(rest % n[t1]), it2 = (int)(rest / n[t1]);
  int c[3];
  c[d] = pos;
  c[t1] = it1;
  c[t2] = it2;
  const int e0 = d == 0 ? P[0] : n[0], e1 = d == 1 ? P[1] : n[1];
  return c[0] + (int64_t)e0 * (c[1] + (int64_t)e1 * c[2]);
}

// Face buffers of the binary32 kernel: odd row pitch, and per-face padding
// (in scalars, for nf fields per face) chosen so that the line tasks of the
// in-face sweeps, C cells per block, touch every shared-memory bank once.
__host__ __device__ constexpr int f32_face_pitch(int k) { return k % 2 ? k : k + 1; }
__host__ __device__ constexpr int f32_face_pad(int k, int C, int nf) {
  return nf == 2 ? (k == 3 ? (C == 32 ? 0 : 1) : k == 4 && C == 4 ? 4 : k == 5 ? (C == 16 ? 1 : 3) : k == 6 ? 2
                    : k == 7 ? (C == 4 ? 5 : 1) : k == 9 ? (C == 4 ? 7 : 3) : 0)
         : nf == 3 ? (k == 5 && C == 8 ? 2 : k == 7 && C == 4 ? 4 : k == 9 ? (C == 4 ? 6 : 2) : 0)
                   : 0;
}

// Shared-memory bytes of the binary32 kernel for k points and C cells: four
// padded point fields (seven with the G2 positions), the neighbour face data (6 faces x 2 fields), the
// in-face sweep buffer (6 faces x 3 fields) and two face tables (6 ints each).
__host__ __device__ constexpr int f32_smem_bytes(int k, int op, int C, int geo = 0) {
  return 4 * ((geo == GEO_POS ? 7 : 4) * (k * (k % 2 == 0 ? k + 1 : k) * k) * C +
              6 * ((op == OP_SIPG ? 2 : 1) * k * f32_face_pitch(k) + f32_face_pad(k, C, op == OP_SIPG ? 2 : 1)) * C +
              6 * ((op == OP_SIPG ? 3 : 1) * k * f32_face_pitch(k) + f32_face_pad(k, C, op == OP_SIPG ? 3 : 1)) * C +
              12 * C);
}

// Shared-memory scalars per cell: u, three gradient fields, the two
// neighbour trace buffers (2 faces x NBA / NBB fields x k^2) and the face test
// coefficients (6 faces x FTF fields x k^2): NBA = 2, NBB = 3, FTF = 4 for
// SIPG, 1, 1, 1 for advection.  Plus 3k + 2k^2 scalars of tables per block.
__host__ __device__ constexpr int smem_scalars_per_cell(int k, int op) {
  return 4 * k * k * k + 2 * ((op == OP_SIPG ? 2 : 1) + (op == OP_SIPG ? 3 : 1)) * k * k +
         6 * (op == OP_SIPG ? 4 : 1) * k * k;
}
__host__ __device__ constexpr int smem_bytes_per_block(int k, int op, int scalar_bytes, int cpb) {
  return (cpb * smem_scalars_per_cell(k, op) + 3 * k + 2 * k * k) * scalar_bytes;
}

// Implemented per degree in dg_apply_k<K>.cu.
cudaError_t launch_apply_k2(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k3(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k4(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k5(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k6(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k7(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k8(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_apply_k9(const ApplyLaunch&, int64_t n_cells);
cudaError_t launch_batch_k2(const BatchLaunch&);
cudaError_t launch_batch_k3(const BatchLaunch&);
cudaError_t launch_batch_k4(const BatchLaunch&);
cudaError_t launch_batch_k5(const BatchLaunch&);
cudaError_t launch_batch_k6(const BatchLaunch&);
cudaError_t launch_batch_k7(const BatchLaunch&);
cudaError_t launch_batch_k8(const BatchLaunch&);
cudaError_t launch_batch_k9(const BatchLaunch&);

}  // namespace dg
