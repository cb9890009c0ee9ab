// Binary32 DG apply kernel, laid out for shared-memory and instruction
// economy (one launch per operator evaluation).
//
// Same method and face treatment as the FP64 kernel (element-centric: every
// interior face is evaluated from both sides, each cell's result is set
// exactly once, no atomics), reorganized because in binary32 the arithmetic
// is cheap and the kernel is limited by shared-memory traffic, integer work
// and latency:
//
//  * C cells per block (a compile-time tile shape), k^2 threads per cell;
//    thread (a, b) of a cell owns the x-line (y=a, z=b), the y-line (x=a,
//    z=b) and the z-line (x=a, y=b) in the phases that sweep in x, y and z,
//    and face point (a, b) of the faces of every direction.
//  * Shared memory is cell-minor: the value at point p of cell c sits at
//    p C + c and thread t works on cell t mod C, so the 32 lanes of a warp
//    address 32/C consecutive line positions of C cells; rows are padded to
//    an odd length so that no line direction has bank conflicts, and the face
//    buffers are padded per face for the in-face line tasks.
//  * The block's source cells and their x-neighbours are staged with
//    coalesced loads (asynchronous copies from k = 5 on); the y/z
//    neighbours' lines through the thread's face points are loaded before
//    the first barrier, or (k = 5, 6 with per-point geometry) the four
//    neighbouring blocks of C cells are staged whole with coalesced
//    asynchronous copies.
//  * The 1D sweeps keep their line in registers (k loads, k^2 FMAs, k
//    stores); the z-line owner computes the z-derivative from registers.
//  * The in-face sum factorization of the neighbours' traces (Eq.
//    face_integral: S (x) S and the tangential derivatives of the face-normal
//    data S_f u, D_f u) runs as line tasks spread over all threads of the
//    block; the results land at the face point of the thread that forms the
//    flux.
//  * Face test functions are injected by the line owners in the phase where
//    they integrate (apply D^T along their direction), so the only shared
//    traffic for faces is the tangential gradient-test components pulled
//    across directions.
//  * Cell geometry is stored in a cell-blocked layout [block][array][point]
//    [cell in block] and face geometry in blocks of 8 faces, so that their
//    loads are whole sectors; bulk L2 prefetches of both start after the
//    first barrier.  Boundary and tail handling are selects on clamped
//    indices (no divergent branches).
//
// Phases (barrier-separated): staging, face tables | neighbour face data,
// S_z | S_y, first in-face sweep | S_x, D_x, second in-face sweep with the
// neighbour's normal flux | D_y, D_z | own x/y face traces (extrapolation of
// the Gauss-point fields, E_s) and numerical fluxes (Eq. poisson_sip /
// advection), and for k <= 6 the z-line's traces, fluxes and q-point
// operation (Sec. 5 geometry variants) | z: (k >= 7: the same, point by
// point) z-face injection, pulled components, D_z^T | y: D_y^T | x: D_x^T,
// S_x^T | y: S_y^T | z: S_z^T and the store (set) of dst.  A launch covers a
// range of cells (the whole mesh, or a slab of the pipelined host apply).
#pragma once

#include <cstdint>
#include <type_traits>

#include "dg_internal.cuh"

namespace dg {

template <int K, int C>
struct F32Shape {
  static constexpr int K2 = K * K, K3 = K2 * K;
  static constexpr int XS = (K % 2 == 0) ? K + 1 : K;  // odd row pitch
  static constexpr int YS = XS * K;
  static constexpr int NP = YS * K;  // padded points per cell
  static constexpr int NT = C * K2;  // threads per block
};

__device__ __forceinline__ void f32_prefetch_bulk_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// Asynchronous 4-byte global-to-shared copies (staging without a register
// round trip); completed by f32_cp_async_wait before the next barrier.
__device__ __forceinline__ void f32_cp_async4(float* s, const float* g) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(s);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(g) : "memory");
}
__device__ __forceinline__ void f32_cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// One 1D sweep of a line in binary32, out = M in with M = S, D or S^T
// (WHICH = EO_S, EO_D, EO_ST): from k = 5 on in the even-odd form of Sec.
// 4.1 (k = 5: 21 instead of 25 operations; the kernel is bound by its
// instruction count), below it directly.
template <int K, int WHICH>
__device__ __forceinline__ void f32_line(const Tables<float>& tb, const float (&in)[K], float (&out)[K]) {
  if constexpr (K >= 5) {
    eo_line<K, WHICH == EO_D>(tb.EO[WHICH][0], tb.EO[WHICH][1], in, out);
  } else {
#pragma unroll
    for (int q = 0; q < K; ++q) {
      float acc = 0.f;
#pragma unroll
      for (int j = 0; j < K; ++j) {
        const float m = WHICH == EO_S ? tb.S[q * K + j] : WHICH == EO_D ? tb.D[q * K + j] : tb.S[j * K + q];
        acc = fmaf(m, in[j], acc);
      }
      out[q] = acc;
    }
  }
}

// Resident blocks per SM the register allocation is sized for: about 900
// threads per SM up to k = 8 (72-80 registers without spills; at k = 7, 8
// 7-13% faster than the 700 that the longer lines of k = 9 keep, which
// spill otherwise); 1000 for advection, whose smaller kernel fits 56
// registers without spilling (k = 5: five blocks of 200 threads, 5% faster
// than four); the shared memory of that many blocks fits as well.
__host__ __device__ constexpr int f32_min_blocks(int k, int C, int op) {
  return (op == OP_ADV ? 1000 : k <= 8 ? 900 : 700) / (C * k * k) > 0
             ? (op == OP_ADV ? 1000 : k <= 8 ? 900 : 700) / (C * k * k)
             : 1;
}

// One block (blk) of the binary32 apply: the body of apply_f32_kernel (one
// operator) and apply_f32_batch (several).
template <int K, int C, int GEO, int OP, typename PP>
__device__ __forceinline__ void f32_body(const Tables<float>& tb, const PP& P, const int blk) {
  using Sh = F32Shape<K, C>;
  constexpr int K2 = Sh::K2, K3 = Sh::K3, XS = Sh::XS, YS = Sh::YS, NP = Sh::NP, NT = Sh::NT;
  constexpr int CBL = f32_geometry_block(K);
  constexpr bool SIPG = OP == OP_SIPG;
  constexpr bool CART = GEO == GEO_CART;
  constexpr bool TANG = SIPG && !CART;        // tangential gradients on faces
  constexpr int NBF = SIPG ? 2 : 1;           // neighbour face fields (value, normal derivative)
  constexpr int NBB = SIPG ? (CART ? 2 : 3) : 1;  // after the first in-face sweep
  constexpr bool POS = GEO == GEO_POS;  // G2: positions (+ kappa) per point, J in the kernel
  constexpr int NA = GEO == GEO_FULL ? 10 : POS ? (SIPG ? 4 : 3) : (SIPG ? 6 : 3);
  static_assert(C == 4 || C == 8 || C == 16 || C == 32 || C == 64, "cells per block");
  static_assert(CBL % C == 0, "geometry block width");

  extern __shared__ __align__(16) float sm[];
  float* U = sm;             // [NP][C]: u -> u at Gauss points -> integrated field
  float* G0 = U + NP * C;    // gradients, then test fields
  float* G1 = G0 + NP * C;
  float* G2 = G1 + NP * C;
  // face buffers: face point (a, b) at a + KP b (odd row pitch KP), fields
  // KK apart, faces FSA / FSB apart (padded so that the line tasks of the
  // in-face sweeps are free of bank conflicts)
  constexpr int KP = f32_face_pitch(K), KK = K * KP;
  constexpr int FSA = NBF * KK + f32_face_pad(K, C, NBF), FSB = NBB * KK + f32_face_pad(K, C, NBB);
  float* FA = G2 + NP * C;   // [6 faces][NBF][K KP][C]: neighbour data at GL face points,
                             // then (u+, w+) at the face Gauss points; last: dot reduction
  float* FB = FA + 6 * FSA * C;  // [6][NBB][K KP][C]: after the first in-face sweep;
                                 // then the pulled face test components [2][2][2][K KP][C]
  int* NBC = reinterpret_cast<int*>(FB + 6 * FSB * C);  // [6][C] neighbour cell or -1
  int* FID = NBC + 6 * C;                                    // [6][C] face id
  float* XP = reinterpret_cast<float*>(FID + 6 * C);          // G2: [3][NP][C] Gauss-point positions
  constexpr int RS = K3;  // cell stride of the staged source
  static_assert((C + 2) * RS <= 2 * NP * C, "staged source fits in G1/G2");

  const Geometry<float>& gm = P.geo;
  // face arrays: blocks of FBW faces, [face block][array][point][face in
  // block]; element (m, fp) of face f at face_at(d, f)[(m K2 + fp) FBW]
  constexpr int FBW = kFaceBlock;
  const int NFA = SIPG ? (gm.face_pair ? 7 : 4) : 1;
  auto face_at = [&](int d, int f) -> const float* {
    return gm.face[d] + (size_t)(f / FBW) * (NFA * K2 * FBW) + f % FBW;
  };
  const int tid = threadIdx.x;
  const int lc = tid % C;
  const int ln = tid / C;
  const int a = ln % K, b = ln / K;
  const int fpt = a + f32_face_pitch(K) * b;  // face point (a, b) in the face buffers
  const int ncell = (int)gm.n_cells;
  const int cell0 = (int)P.cell_begin + blk * C;  // this block's first cell
  const int cell_end = (int)P.cell_end;                         // end of this launch's cells
  const int cell_raw = cell0 + lc;
  const bool valid = cell_raw < cell_end;
  const int cell = valid ? cell_raw : cell_end - 1;
  int i0, i1, i2;
  {
    const unsigned q = (unsigned)cell / (unsigned)gm.n[0];
    i0 = cell - (int)(q * (unsigned)gm.n[0]);
    i1 = (int)(q % (unsigned)gm.n[1]);
    i2 = (int)(q / (unsigned)gm.n[1]);
  }

  // y and z neighbours.  SIPG with per-point geometry, k = 5, 6: the four
  // blocks of C cells at offsets -n0, +n0, -n0 n1, +n0 n1 from the block's
  // first cell are contiguous in memory and are staged into shared memory
  // with coalesced asynchronous copies (chunk 0 in G0, chunks 1-3 in FB, both
  // free until phase 2); cells whose neighbour is not at that offset
  // (periodic wrap) read it from global memory, boundary sides read the own
  // cell (their data is not used).  Otherwise the lines through the thread's
  // face points are loaded into registers before the first barrier
  // (advection: only the face layer), so that their latency overlaps the
  // staging below.  (Measured against the register path: +9% at k = 6, +-0
  // at k = 5; slower for k <= 4 and for the arithmetic-bound Cartesian
  // kernel.)
  constexpr bool EARLY = K <= 6;
  constexpr bool STAGE_YZ = EARLY && K >= 5 && TANG && 3 * K3 <= 6 * FSB;
  // the source staging below also uses asynchronous copies from k = 5 on
  // (+1-4% at k = 7, 8; slower for k <= 4)
  constexpr bool ASYNC_R = K >= 5;
  auto yz_chunk = [&](int j) -> float* { return j == 0 ? G0 : FB + (j - 1) * C * K3; };
  float wyz[EARLY && !STAGE_YZ ? 4 : 1][EARLY && !STAGE_YZ ? K : 1];
  // slim face access (a basis whose face value and normal derivative each
  // come from one layer, Sec. 3.1): only layers edge and edge +- 1 of a
  // neighbour's normal line are read; the others have zero weight in D_f
  const bool slim = tb.slim != 0;
  auto need = [&](int l, int s) -> bool {
    return SIPG ? (!slim || l == (s ? 0 : K - 1) || l == (s ? 1 : K - 2)) : l == (s ? 0 : K - 1);
  };
  if (STAGE_YZ && !slim) {
    const int n0 = gm.n[0], n01 = gm.n[0] * gm.n[1];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int off = j == 0 ? -n0 : j == 1 ? n0 : j == 2 ? -n01 : n01;
      const int cb = cell0 + off;  // first cell of the chunk
      const int lo = cb < 0 ? -cb * K3 : 0;
      const int64_t rem = ((int64_t)ncell - cb) * K3;  // elements from the chunk start to the end
      const int hi = rem < C * K3 ? (int)rem : C * K3;
      float* dstc = yz_chunk(j);
      const float* srcc = P.src + (int64_t)cb * K3;
      static_assert((C * K3) % NT == 0, "chunk staging rounds");
      if (lo == 0 && hi == C * K3) {  // whole chunk inside the mesh (block-uniform)
#pragma unroll
        for (int r = 0; r < C * K3 / NT; ++r) f32_cp_async4(dstc + tid + r * NT, srcc + tid + r * NT);
      } else {
#pragma unroll
        for (int r = 0; r < C * K3 / NT; ++r) {
          const int e = tid + r * NT;
          if (e >= lo && e < hi) f32_cp_async4(dstc + e, srcc + e);
        }
      }
    }
  } else if constexpr (EARLY) {
    const int n0 = gm.n[0], n01 = gm.n[0] * gm.n[1];
    const int per = gm.periodic;
    const int ny[2] = {i1 > 0 ? cell - n0 : per ? cell + (gm.n[1] - 1) * n0 : cell,
                       i1 < gm.n[1] - 1 ? cell + n0 : per ? cell - (gm.n[1] - 1) * n0 : cell};
    const int nz[2] = {i2 > 0 ? cell - n01 : per ? cell + (gm.n[2] - 1) * n01 : cell,
                       i2 < gm.n[2] - 1 ? cell + n01 : per ? cell - (gm.n[2] - 1) * n01 : cell};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const float* py = P.src + (size_t)ny[s] * K3 + a + K2 * b;
      const float* pz = P.src + (size_t)nz[s] * K3 + a + K * b;
#pragma unroll
      for (int l = 0; l < K; ++l) {
        if (need(l, s)) {
          wyz[s][l] = py[l * K];
          wyz[2 + s][l] = pz[l * K2];
        } else {
          wyz[s][l] = wyz[2 + s][l] = 0.f;
        }
      }
    }
  }

  // the source of the block's cells and their two x-neighbours
  // (cells cell0 - 1 .. cell0 + C, contiguous in memory) staged in shared
  // memory with coalesced loads (cell-major, stride k^3); it occupies the
  // G1/G2 region until phase 4
  float* R = G1;
  const int cfirst = cell0 - 1;
  {
    const int64_t base = (int64_t)cfirst * K3;
    constexpr int NR = (C + 2) * K3;
    const unsigned lo = cfirst < 0 ? K3 : 0u;  // cell -1 does not exist
    const int rem = ncell - cfirst;            // cells from cfirst to the end of the mesh
    const unsigned hi = (unsigned)(rem < C + 2 ? rem : C + 2) * K3;
    if (lo == 0 && hi == (unsigned)NR) {  // whole range inside the mesh (block-uniform)
#pragma unroll
      for (int r = 0; r < NR / NT; ++r) {
        const unsigned e = tid + r * NT;
        if constexpr (ASYNC_R) f32_cp_async4(R + e, P.src + base + e);
        else R[e] = P.src[base + e];
      }
      if (NR % NT != 0 && tid < NR % NT) {
        const unsigned e = tid + (NR / NT) * NT;
        if constexpr (ASYNC_R) f32_cp_async4(R + e, P.src + base + e);
        else R[e] = P.src[base + e];
      }
    } else {
#pragma unroll
      for (int r = 0; r < (NR + NT - 1) / NT; ++r) {
        const unsigned e = tid + r * NT;
        if (e >= lo && e < hi) {
          if constexpr (ASYNC_R) f32_cp_async4(R + e, P.src + base + e);
          else R[e] = P.src[base + e];
        }
      }
    }
  }
  // neighbour cells and face ids of the six faces (d, s), one thread each;
  // faces are numbered like cells with the face position along d
  for (int t = ln; t < 6; t += K2) {
    const int d = t >> 1, s = t & 1;
    const int id = d == 0 ? i0 : d == 1 ? i1 : i2;
    const int nd = gm.n[d];
    int jd = id + (s ? 1 : -1);
    bool inside = jd >= 0 && jd < nd;
    if (!inside && gm.periodic) {
      jd = jd < 0 ? nd - 1 : 0;
      inside = true;
    }
    int pos = id + s;
    if (gm.periodic && pos == nd) pos = 0;
    const int j0 = d == 0 ? jd : i0, j1 = d == 1 ? jd : i1, j2 = d == 2 ? jd : i2;
    NBC[t * C + lc] = inside ? j0 + gm.n[0] * (j1 + gm.n[1] * j2) : -1;
    const int f0 = d == 0 ? pos : i0, f1 = d == 1 ? pos : i1, f2 = d == 2 ? pos : i2;
    const int e0 = d == 0 ? gm.P[0] : gm.n[0], e1 = d == 1 ? gm.P[1] : gm.n[1];
    FID[t * C + lc] = f0 + e0 * (f1 + e1 * f2);
  }
  if constexpr (POS) {
    // G2: the block's Gauss-point positions (cell-blocked arrays 0..2) into
    // the padded cell-minor layout of the point fields
    const float* gb = gm.cell + ((size_t)(cell0 / CBL) * NA * K3) * CBL + (cell0 % CBL);
    constexpr int NE = 3 * K3 * C;
#pragma unroll 1
    for (int e = tid; e < NE; e += NT) {
      const int c = e % C, q = (e / C) % K3, m = e / (C * K3);
      const int x = q % K, y = (q / K) % K, z = q / K2;
      f32_cp_async4(XP + (m * NP + x + XS * y + YS * z) * C + c, gb + (m * K3 + q) * CBL + c);
    }
  }
  if constexpr (ASYNC_R || STAGE_YZ || POS) f32_cp_async_wait();
  __syncthreads();

  // start the HBM fetch of this block's cell geometry (read in phase 6)
  // and face geometry (phases 3, 5, 6) into L2: bulk prefetches of the
  // geometry block and of the face blocks of the first and last cell of
  // every face direction and side
  if constexpr (!CART) {
    constexpr unsigned BYTES = NA * K3 * CBL * 4, NPF = 8;
    constexpr unsigned CH = (BYTES / NPF + 15) / 16 * 16;
    if (tid < (int)NPF) {
      const char* g = reinterpret_cast<const char*>(gm.cell + ((size_t)(cell0 / CBL) * NA * K3) * CBL);
      const unsigned off = tid * CH;
      if (off < BYTES) {
        const unsigned sz = BYTES - off < CH ? BYTES - off : CH;
        f32_prefetch_bulk_l2(g + off, sz);
      }
    } else if (tid < (int)NPF + 12) {
      const int i = tid - NPF, t = i >> 1, d = t >> 1;
      const int fb = FID[t * C + ((i & 1) ? C - 1 : 0)] / FBW;
      if (!(i & 1) || fb != FID[t * C] / FBW)
        f32_prefetch_bulk_l2(gm.face[d] + (size_t)fb * (NFA * K2 * FBW), NFA * K2 * FBW * 4);
    }
  }

  // 1. neighbours' face data at GL face point (a, b): the layer on the shared
  // face and (SIPG) the normal derivative D_f of the line through it; x
  // neighbours from the staged source where they are staged
  float v[K];
#pragma unroll
  for (int j = 0; j < K; ++j) v[j] = R[(lc + 1) * RS + a + K * b + K2 * j];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    const int d = t >> 1, s = t & 1;
    const int nb = NBC[t * C + lc];
    const int off = d == 0 ? K * (a + K * b) : d == 1 ? a + K2 * b : a + K * b;
    const int str = d == 0 ? 1 : d == 1 ? K : K2;
    float w[K];
    if (d == 0) {
      const int r = (nb >= 0 ? nb : cell) - cfirst;
      if (r >= 0 && r < C + 2) {
#pragma unroll
        for (int l = 0; l < K; ++l) w[l] = need(l, s) ? R[r * RS + off + l] : 0.f;
      } else {
        const float* p = P.src + (size_t)nb * K3 + off;
#pragma unroll
        for (int l = 0; l < K; ++l) w[l] = need(l, s) ? p[l] : 0.f;
      }
    } else if constexpr (STAGE_YZ) {
      const int nstep = d == 1 ? gm.n[0] : gm.n[0] * gm.n[1];
      if (!slim && nb == cell + (s ? nstep : -nstep)) {
        const float* p = yz_chunk(t - 2) + lc * K3 + off;
#pragma unroll
        for (int l = 0; l < K; ++l) w[l] = p[l * str];
      } else if (nb >= 0) {
        const float* p = P.src + (size_t)nb * K3 + off;
#pragma unroll
        for (int l = 0; l < K; ++l) w[l] = need(l, s) ? p[l * str] : 0.f;
      } else {
#pragma unroll
        for (int l = 0; l < K; ++l) w[l] = need(l, s) ? R[(lc + 1) * RS + off + l * str] : 0.f;
      }
    } else if constexpr (EARLY) {
#pragma unroll
      for (int l = 0; l < K; ++l) w[l] = wyz[t - 2][l];
    } else {
      const float* p = P.src + (size_t)(nb >= 0 ? nb : cell) * K3 + off;
#pragma unroll
      for (int l = 0; l < K; ++l) w[l] = need(l, s) ? p[l * str] : 0.f;
    }
    FA[(t * FSA + fpt) * C + lc] = s ? w[0] : w[K - 1];
    if (SIPG) {
      float dn = 0.f;
#pragma unroll
      for (int l = 0; l < K; ++l) dn = fmaf(tb.DF[1 - s][l], w[l], dn);
      FA[(t * FSA + KK + fpt) * C + lc] = dn;
    }
    // long lines: keep at most two of them in flight (register budget)
    if (K >= 7 && s == 1) __syncwarp();
  }
  // S along z
  {
    float o[K];
    f32_line<K, EO_S>(tb, v, o);
#pragma unroll
    for (int q = 0; q < K; ++q) U[(a + XS * b + YS * q) * C + lc] = o[q];
  }
  __syncthreads();

  // 2. S along y; first in-face sweep (along t1) of the neighbour data
  {
    float w[K], o[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = U[(a + XS * j + YS * b) * C + lc];
    f32_line<K, EO_S>(tb, w, o);
#pragma unroll
    for (int q = 0; q < K; ++q) U[(a + XS * q + YS * b) * C + lc] = o[q];
  }
  {
    constexpr int NTASK = 6 * K * C, ROUNDS = (NTASK + NT - 1) / NT;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
      const int task = tid + r * NT;
      if (NTASK % NT == 0 || task < NTASK) {
        const int tc = task % C, rest = task / C;
        const int bb = rest % K, t = rest / K;
        const float* in = FA + (t * FSA + KP * bb) * C + tc;  // row (i, bb)
        float* out = FB + (t * FSB + KP * bb) * C + tc;
        float xv[K], xn[K];
#pragma unroll
        for (int i = 0; i < K; ++i) {
          xv[i] = in[i * C];
          if (SIPG) xn[i] = in[(KK + i) * C];
        }
        if constexpr (K >= 5) {
          // even-odd form, the split of xv shared by S and DS
          float e[(K + 1) / 2], o[K / 2], s0[K], s1[K], s2[K];
          eo_split<K>(xv, e, o);
          eo_combine<K, false>(tb.EO[EO_S][0], tb.EO[EO_S][1], e, o, s0);
          if (TANG) eo_combine<K, true>(tb.EO[EO_DS][0], tb.EO[EO_DS][1], e, o, s1);
          if (SIPG) eo_line<K, false>(tb.EO[EO_S][0], tb.EO[EO_S][1], xn, s2);
#pragma unroll
          for (int qa = 0; qa < K; ++qa) {
            out[qa * C] = s0[qa];
            if (TANG) out[(KK + qa) * C] = s1[qa];
            if (SIPG) out[((NBB - 1) * KK + qa) * C] = s2[qa];
          }
        } else {
#pragma unroll
          for (int qa = 0; qa < K; ++qa) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
            for (int i = 0; i < K; ++i) {
              s0 = fmaf(tb.S[qa * K + i], xv[i], s0);
              if (TANG) s1 = fmaf(tb.DS[qa * K + i], xv[i], s1);
              if (SIPG) s2 = fmaf(tb.S[qa * K + i], xn[i], s2);
            }
            out[qa * C] = s0;
            if (TANG) out[(KK + qa) * C] = s1;
            if (SIPG) out[((NBB - 1) * KK + qa) * C] = s2;
          }
        }
      }
    }
  }
  __syncthreads();

  // 3. S along x -> u at the Gauss points; D along x; second in-face sweep
  // (along t2) giving the neighbour's value u+ and normal flux w+ = (its
  // derivative along this cell's outward normal) at face Gauss point (qa, qb)
  {
    float ux[K];
    float w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = U[(j + XS * a + YS * b) * C + lc];
    f32_line<K, EO_S>(tb, w, ux);
#pragma unroll
    for (int q = 0; q < K; ++q) U[(q + XS * a + YS * b) * C + lc] = ux[q];
    if (SIPG) {
      f32_line<K, EO_D>(tb, ux, w);
#pragma unroll
      for (int q = 0; q < K; ++q) G0[(q + XS * a + YS * b) * C + lc] = w[q];
    }
  }
  {
    constexpr int NTASK = 6 * K * C, ROUNDS = (NTASK + NT - 1) / NT;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
      const int task = tid + r * NT;
      if (NTASK % NT == 0 || task < NTASK) {
        const int tc = task % C, rest = task / C;
        const int qa = rest % K, t = rest / K;
        const int d = t >> 1, s = t & 1;
        const float* in = FB + (t * FSB + qa) * C + tc;  // row (qa, j): stride KP C
        float* out = FA + (t * FSA + qa) * C + tc;
        float sv[K], dsv[K], sn[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
          sv[j] = in[j * KP * C];
          if (TANG) dsv[j] = in[(KK + j * KP) * C];
          if (SIPG) sn[j] = in[((NBB - 1) * KK + j * KP) * C];
        }
        const float* fg = nullptr;
        if (TANG) fg = face_at(d, FID[t * C + tc]) + qa * FBW;
        const float cj = CART && SIPG ? (s ? 1.f : -1.f) * gm.cart_jinv[d] : 0.f;
        // u, dt2 = (S, DS) sv, dt1 = S dsv, dn = S sn at the K points qb
        float uo[K], d2o[K], d1o[K], dno[K];
        if constexpr (K >= 5) {
          float e[(K + 1) / 2], o[K / 2];
          eo_split<K>(sv, e, o);
          eo_combine<K, false>(tb.EO[EO_S][0], tb.EO[EO_S][1], e, o, uo);
          if (TANG) {
            eo_combine<K, true>(tb.EO[EO_DS][0], tb.EO[EO_DS][1], e, o, d2o);
            eo_line<K, false>(tb.EO[EO_S][0], tb.EO[EO_S][1], dsv, d1o);
          }
          if (SIPG) eo_line<K, false>(tb.EO[EO_S][0], tb.EO[EO_S][1], sn, dno);
        } else {
#pragma unroll
          for (int qb = 0; qb < K; ++qb) {
            float u = 0.f, dt2 = 0.f, dt1 = 0.f, dn = 0.f;
#pragma unroll
            for (int j = 0; j < K; ++j) {
              u = fmaf(tb.S[qb * K + j], sv[j], u);
              if (TANG) {
                dt2 = fmaf(tb.DS[qb * K + j], sv[j], dt2);
                dt1 = fmaf(tb.S[qb * K + j], dsv[j], dt1);
              }
              if (SIPG) dn = fmaf(tb.S[qb * K + j], sn[j], dn);
            }
            uo[qb] = u;
            d2o[qb] = dt2;
            d1o[qb] = dt1;
            dno[qb] = dn;
          }
        }
#pragma unroll
        for (int qb = 0; qb < K; ++qb) {
          const float u = uo[qb], dt2 = TANG ? d2o[qb] : 0.f, dt1 = TANG ? d1o[qb] : 0.f,
                      dn = SIPG ? dno[qb] : 0.f;
          out[qb * KP * C] = u;
          if (SIPG) {
            float wn;
            if (CART) {
              wn = cj * dn;
            } else {
              // reference-axis components: d carries the normal derivative,
              // t1 < t2 the tangential ones; the neighbour is slot s
              const float gx = d == 0 ? dn : dt1;
              const float gy = d == 1 ? dn : (d == 0 ? dt1 : dt2);
              const float gz = d == 2 ? dn : dt2;
              // face vector j_f = J^{-T} e_d; the neighbour (slot s) has
              // (s ? -j_f : j_f) (face_pair: both stored), and its
              // derivative along this cell's outward normal is minus that
              const float* f = fg + qb * K * FBW + (gm.face_pair ? s * 3 * K2 * FBW : 0);
              const float jd = f[0] * gx + f[K2 * FBW] * gy + f[2 * K2 * FBW] * gz;
              wn = (s && !gm.face_pair) ? jd : -jd;
            }
            out[(KK + qb * KP) * C] = wn;
          }
        }
      }
    }
  }
  __syncthreads();

  // 4. D along y and z
  if (SIPG) {
    float uy[K], uz[K], s1[K], s2[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      uy[j] = U[(a + XS * j + YS * b) * C + lc];
      uz[j] = U[(a + XS * b + YS * j) * C + lc];
    }
    f32_line<K, EO_D>(tb, uy, s1);
    f32_line<K, EO_D>(tb, uz, s2);
#pragma unroll
    for (int q = 0; q < K; ++q) {
      G1[(a + XS * q + YS * b) * C + lc] = s1[q];
      G2[(a + XS * b + YS * q) * C + lc] = s2[q];
    }
    __syncthreads();
  }

  // 5. own traces at face point (a, b) of the x and y faces (extrapolation
  // E_s of the Gauss-point fields along the owned line) and the numerical
  // flux; test coefficients: value tv, gradient tg * j_o.  The own-direction
  // coefficients replace (u+, w+) in this thread's own slots of FA; the
  // tangential ones consumed by other line owners go to FT.  (The z faces
  // follow in phase 6, where the z-line owner holds the fields anyway.)
  const float ea0 = tb.E[0][a], ea1 = tb.E[1][a], eb0 = tb.E[0][b], eb1 = tb.E[1][b];
  const float wa = tb.W[a], wb = tb.W[b];
  float* FT = FB;  // [face direction x, y][side][component slot][K2][C]
  // trace and flux of face (d, s) at this thread's face point
  // numerical flux of face (d, s) at this thread's face point from the own
  // traces uf (value) and gf (reference gradient; the components other than
  // d are needed on non-Cartesian meshes only)
  auto face_flux = [&](auto dc, int s, float uf, const float(&gf)[3], float& tvv, float(&tgo)[3]) {
    constexpr int d = decltype(dc)::value;
    const int t = 2 * d + s;
    const bool interior = NBC[t * C + lc] >= 0;
    const int fid = FID[t * C + lc];
    const float* slot = FA + (t * FSA + fpt) * C + lc;  // this thread's (u+, w+) of face t
    const float un = slot[0];
    tgo[0] = tgo[1] = tgo[2] = 0.f;
    if (SIPG) {
      const float wn = slot[KK * C];
      float jo[3], fjxw, tau;
      if (CART) {
        const float jn = (s ? 1.f : -1.f) * gm.cart_jinv[d];
        jo[0] = d == 0 ? jn : 0.f;
        jo[1] = d == 1 ? jn : 0.f;
        jo[2] = d == 2 ? jn : 0.f;
        float kap = 1.f;
        if (gm.kq) kap = d == 0 ? gm.kf[i0 + s] : gm.kq[i0 * K + a];
        fjxw = kap * wa * wb * gm.cart_detj * gm.cart_jinv[d];
        tau = gm.cart_tau[d];
      } else {
        const float* fp = face_at(d, fid) + ln * FBW;
        // own slot 1 - s: the lower side (slot 0) has j_f, the upper -j_f
        // (or both stored: face_pair)
        const float* jp = fp + (gm.face_pair ? (1 - s) * 3 * K2 * FBW : 0);
        const float sg = (s || gm.face_pair) ? 1.f : -1.f;
        jo[0] = sg * jp[0];
        jo[1] = sg * jp[K2 * FBW];
        jo[2] = sg * jp[2 * K2 * FBW];
        fjxw = fp[(gm.face_pair ? 6 : 3) * K2 * FBW];
        tau = gm.tau[d][fid];
      }
      const float dno = CART ? jo[d] * gf[d] : jo[0] * gf[0] + jo[1] * gf[1] + jo[2] * gf[2];
      const float jump = interior ? uf - un : 2.f * uf;
      tvv = interior ? fjxw * (tau * jump - 0.5f * (dno + wn)) : fjxw * (tau * jump - dno);
      const float tg = -0.5f * fjxw * jump;
#pragma unroll
      for (int c = 0; c < 3; ++c) tgo[c] = tg * jo[c];
    } else {
      float cn;
      if (CART) {
        cn = gm.vel[d] * wa * wb * gm.cart_detj * gm.cart_jinv[d];
      } else {
        cn = face_at(d, fid)[ln * FBW];
      }
      const float cno = s ? cn : -cn;  // c.n da w with n the own outward normal
      tvv = interior ? 0.5f * cno * (uf + un) + 0.5f * fabsf(cno) * (uf - un) : fabsf(cno) * uf;
    }
  };
  // the same from the fields along the owned d-line (extrapolation E_s)
  auto own_flux = [&](auto dc, int s, const float(&lu)[K], const float(&lg)[3][K], float& tvv, float(&tgo)[3]) {
    constexpr int d = decltype(dc)::value;
    float uf = 0.f, gf[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float e = tb.E[s][j];
      uf = fmaf(e, lu[j], uf);
      if (SIPG) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
          if (c == d || TANG) gf[c] = fmaf(e, lg[c][j], gf[c]);
      }
    }
    face_flux(dc, s, uf, gf, tvv, tgo);
  };
  auto xy_faces = [&](auto dc) {
    constexpr int d = decltype(dc)::value;
    float lu[K], lg[3][K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int pidx = (d == 0 ? (j + XS * a + YS * b) : (a + XS * j + YS * b)) * C + lc;
      lu[j] = U[pidx];
      if (SIPG) {
        lg[0][j] = (d == 0 || TANG) ? G0[pidx] : 0.f;
        lg[1][j] = (d == 1 || TANG) ? G1[pidx] : 0.f;
        lg[2][j] = TANG ? G2[pidx] : 0.f;
      }
    }
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float tvv, tgo[3];
      own_flux(dc, s, lu, lg, tvv, tgo);
      float* slot = FA + ((2 * d + s) * FSA + fpt) * C + lc;
      slot[0] = tvv;
      if (SIPG) slot[KK * C] = tgo[d];
      if (TANG) {
        // x faces give components 1 and 2, y faces 0 and 2
        FT[(((d * 2 + s) * 2 + 0) * KK + fpt) * C + lc] = tgo[d == 0 ? 1 : 0];
        FT[(((d * 2 + s) * 2 + 1) * KK + fpt) * C + lc] = tgo[2];
      }
    }
  };
  // z-line owner: z-face traces and fluxes, q-point operation at (a, b, j)
  // (Sec. 5 geometry), z-face injection; results: the reference
  // gradient-test fields along the line (tz0..tz2) and the z faces' value
  // tests tvz.
  // It reads only fields that are complete after phase 4 and its own face
  // slots, so for short lines it runs before the barrier below, and its
  // geometry loads overlap the x and y face work; the stores of tz0, tz1 into
  // G0, G1 (read by the x and y traces) follow the barrier.
  float tz0[K], tz1[K], tz2[K], tvz[2];
  // cell-blocked geometry: array m, point q of cell c at
  // ((c / CBL) NA + m) K3 + q) CBL + c mod CBL (padded to whole blocks, so
  // the unclamped index of tail threads stays inside the allocation)
  size_t gofs = 0;
  if constexpr (!CART) gofs = ((size_t)(cell_raw / CBL) * NA * K3) * CBL + (cell_raw % CBL);
  constexpr int MS = K3 * CBL;  // array stride
  float kx = 1.f;
  if (CART && SIPG && gm.kq) kx = gm.kq[i0 * K + a];
  // G2 (Sec. 5): J at (a, b, j) by the collocation derivative D^co of the
  // staged positions along the three lines through the point; J^{-1} by the
  // adjugate (Ji[r*3 + s] = (J^{-1})_{rs}); returns det J
  auto g2_jinv = [&](int j, float(&Ji)[9]) -> float {
    float J[9];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float* X = XP + i * NP * C + lc;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
      for (int m = 0; m < K; ++m) {
        s0 = fmaf(tb.D[a * K + m], X[(m + XS * b + YS * j) * C], s0);
        s1 = fmaf(tb.D[b * K + m], X[(a + XS * m + YS * j) * C], s1);
        s2 = fmaf(tb.D[j * K + m], X[(a + XS * b + YS * m) * C], s2);
      }
      J[i * 3 + 0] = s0;
      J[i * 3 + 1] = s1;
      J[i * 3 + 2] = s2;
    }
    const float c00 = J[4] * J[8] - J[5] * J[7], c01 = J[5] * J[6] - J[3] * J[8], c02 = J[3] * J[7] - J[4] * J[6];
    const float det = J[0] * c00 + J[1] * c01 + J[2] * c02;
    const float r = 1.f / det;
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
  };
  // q-point operation at (a, b, j) and the z faces' gradient-test injection
  // (tgz: the z faces' coefficients, [component][side])
  auto qpoint = [&](int j, float g0, float g1, float g2, float uq, const float(&tgz)[3][2], float& t0, float& t1,
                    float& t2) {
    const int q = a + K * b + K2 * j;
    const float* cp = CART ? gm.cell : gm.cell + gofs + (size_t)q * CBL;
    if (SIPG) {
      if (CART) {
        const float w = wa * wb * tb.W[j] * gm.cart_detj * kx;
        t0 = w * gm.cart_jinv[0] * gm.cart_jinv[0] * g0;
        t1 = w * gm.cart_jinv[1] * gm.cart_jinv[1] * g1;
        t2 = w * gm.cart_jinv[2] * gm.cart_jinv[2] * g2;
      } else if (GEO == GEO_FULL) {
        float J[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) J[m] = cp[m * MS];
        const float jw = cp[9 * MS];
        // grad_x u = J^{-T} grad_xi u, flux = kappa JxW grad_x u, t = J^{-1} flux
        const float x0 = jw * (J[0] * g0 + J[3] * g1 + J[6] * g2);
        const float x1 = jw * (J[1] * g0 + J[4] * g1 + J[7] * g2);
        const float x2 = jw * (J[2] * g0 + J[5] * g1 + J[8] * g2);
        t0 = J[0] * x0 + J[1] * x1 + J[2] * x2;
        t1 = J[3] * x0 + J[4] * x1 + J[5] * x2;
        t2 = J[6] * x0 + J[7] * x1 + J[8] * x2;
      } else if (POS) {
        float Ji[9];
        const float det = g2_jinv(j, Ji);
        const float kw = cp[3 * MS] * det * (wa * wb * tb.W[j]);
        const float x0 = kw * (Ji[0] * g0 + Ji[3] * g1 + Ji[6] * g2);
        const float x1 = kw * (Ji[1] * g0 + Ji[4] * g1 + Ji[7] * g2);
        const float x2 = kw * (Ji[2] * g0 + Ji[5] * g1 + Ji[8] * g2);
        t0 = Ji[0] * x0 + Ji[1] * x1 + Ji[2] * x2;
        t1 = Ji[3] * x0 + Ji[4] * x1 + Ji[5] * x2;
        t2 = Ji[6] * x0 + Ji[7] * x1 + Ji[8] * x2;
      } else {
        const float a00 = cp[0], a01 = cp[MS], a02 = cp[2 * MS], a11 = cp[3 * MS], a12 = cp[4 * MS],
                    a22 = cp[5 * MS];
        t0 = a00 * g0 + a01 * g1 + a02 * g2;
        t1 = a01 * g0 + a11 * g1 + a12 * g2;
        t2 = a02 * g0 + a12 * g1 + a22 * g2;
      }
      // z faces: gradient test along the line
      const float e0 = tb.E[0][j], e1 = tb.E[1][j];
      if (TANG) {
        t0 = fmaf(e0, tgz[0][0], fmaf(e1, tgz[0][1], t0));
        t1 = fmaf(e0, tgz[1][0], fmaf(e1, tgz[1][1], t1));
      }
      t2 = fmaf(e0, tgz[2][0], fmaf(e1, tgz[2][1], t2));
    } else {
      float b0, b1, b2;
      if (CART) {
        const float w = -wa * wb * tb.W[j] * gm.cart_detj;
        b0 = w * gm.cart_jinv[0] * gm.vel[0];
        b1 = w * gm.cart_jinv[1] * gm.vel[1];
        b2 = w * gm.cart_jinv[2] * gm.vel[2];
      } else if (GEO == GEO_FULL) {
        float J[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) J[m] = cp[m * MS];
        const float jw = -cp[9 * MS];
        b0 = jw * (J[0] * gm.vel[0] + J[1] * gm.vel[1] + J[2] * gm.vel[2]);
        b1 = jw * (J[3] * gm.vel[0] + J[4] * gm.vel[1] + J[5] * gm.vel[2]);
        b2 = jw * (J[6] * gm.vel[0] + J[7] * gm.vel[1] + J[8] * gm.vel[2]);
      } else if (POS) {
        float Ji[9];
        const float jw = -(g2_jinv(j, Ji) * (wa * wb * tb.W[j]));
        b0 = jw * (Ji[0] * gm.vel[0] + Ji[1] * gm.vel[1] + Ji[2] * gm.vel[2]);
        b1 = jw * (Ji[3] * gm.vel[0] + Ji[4] * gm.vel[1] + Ji[5] * gm.vel[2]);
        b2 = jw * (Ji[6] * gm.vel[0] + Ji[7] * gm.vel[1] + Ji[8] * gm.vel[2]);
      } else {
        b0 = cp[0];
        b1 = cp[MS];
        b2 = cp[2 * MS];
      }
      t0 = b0 * uq;
      t1 = b1 * uq;
      t2 = b2 * uq;
    }
  };
  auto z_line = [&]() {
    float lu[K], lg[3][K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int pidx = (a + XS * b + YS * j) * C + lc;
      lu[j] = U[pidx];
      if (SIPG) {
        lg[0][j] = G0[pidx];
        lg[1][j] = G1[pidx];
        lg[2][j] = G2[pidx];
      }
    }
    float tgz[3][2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float tvv, tgo[3];
      own_flux(std::integral_constant<int, 2>{}, s, lu, lg, tvv, tgo);
      tvz[s] = tvv;
#pragma unroll
      for (int c = 0; c < 3; ++c) tgz[c][s] = tgo[c];
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      qpoint(j, SIPG ? lg[0][j] : 0.f, SIPG ? lg[1][j] : 0.f, SIPG ? lg[2][j] : 0.f, lu[j], tgz, tz0[j], tz1[j],
             tz2[j]);
    }
  };
  if constexpr (EARLY) z_line();
  xy_faces(std::integral_constant<int, 0>{});
  xy_faces(std::integral_constant<int, 1>{});
  __syncthreads();

  // 6. z-line owner: the pulled z components of the x- and y-face gradient
  // tests, then D_z^T.  Long lines (k >= 7) do the z-line work here, point
  // by point through shared memory (register budget).
  if constexpr (EARLY) {
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int pidx = (a + XS * b + YS * j) * C + lc;
      G0[pidx] = tz0[j];
      G1[pidx] = tz1[j];
      if (TANG) {
        // x faces at (y=b, z=j), y faces at (x=a, z=j)
        float acc = tz2[j];
        acc = fmaf(ea0, FT[(((0 * 2 + 0) * 2 + 1) * KK + b + KP * j) * C + lc], acc);
        acc = fmaf(ea1, FT[(((0 * 2 + 1) * 2 + 1) * KK + b + KP * j) * C + lc], acc);
        acc = fmaf(eb0, FT[(((1 * 2 + 0) * 2 + 1) * KK + a + KP * j) * C + lc], acc);
        tz2[j] = fmaf(eb1, FT[(((1 * 2 + 1) * 2 + 1) * KK + a + KP * j) * C + lc], acc);
      }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      float acc = fmaf(tb.E[0][i], tvz[0], tb.E[1][i] * tvz[1]);
#pragma unroll
      for (int j = 0; j < K; ++j) acc = fmaf(tb.D[j * K + i], tz2[j], acc);
      U[(a + XS * b + YS * i) * C + lc] = acc;
    }
  } else {
    // z traces: extrapolate the fields along the line
    float uf[2] = {0.f, 0.f}, gf[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
      const int pidx = (a + XS * b + YS * j) * C + lc;
      const float u = U[pidx];
      float g[3] = {0.f, 0.f, 0.f};
      if (SIPG) {
        g[2] = G2[pidx];
        if (TANG) {
          g[0] = G0[pidx];
          g[1] = G1[pidx];
        }
      }
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const float e = tb.E[s][j];
        uf[s] = fmaf(e, u, uf[s]);
#pragma unroll
        for (int c = 0; c < 3; ++c) gf[s][c] = fmaf(e, g[c], gf[s][c]);
      }
    }
    float tgz[3][2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      float tvv, tgo[3];
      face_flux(std::integral_constant<int, 2>{}, s, uf[s], gf[s], tvv, tgo);
      tvz[s] = tvv;
#pragma unroll
      for (int c = 0; c < 3; ++c) tgz[c][s] = tgo[c];
    }
    // q-point operation, injection and pulled components, point by point;
    // the gradient-test fields go to G0..G2
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
      const int pidx = (a + XS * b + YS * j) * C + lc;
      float t0, t1, t2;
      qpoint(j, SIPG ? G0[pidx] : 0.f, SIPG ? G1[pidx] : 0.f, SIPG ? G2[pidx] : 0.f, U[pidx], tgz, t0, t1, t2);
      if (TANG) {
        t2 = fmaf(ea0, FT[(((0 * 2 + 0) * 2 + 1) * KK + b + KP * j) * C + lc], t2);
        t2 = fmaf(ea1, FT[(((0 * 2 + 1) * 2 + 1) * KK + b + KP * j) * C + lc], t2);
        t2 = fmaf(eb0, FT[(((1 * 2 + 0) * 2 + 1) * KK + a + KP * j) * C + lc], t2);
        t2 = fmaf(eb1, FT[(((1 * 2 + 1) * 2 + 1) * KK + a + KP * j) * C + lc], t2);
      }
      G0[pidx] = t0;
      G1[pidx] = t1;
      G2[pidx] = t2;
    }
    float t2l[K];
#pragma unroll
    for (int j = 0; j < K; ++j) t2l[j] = G2[(a + XS * b + YS * j) * C + lc];
#pragma unroll
    for (int i = 0; i < K; ++i) {
      float acc = fmaf(tb.E[0][i], tvz[0], tb.E[1][i] * tvz[1]);
#pragma unroll
      for (int j = 0; j < K; ++j) acc = fmaf(tb.D[j * K + i], t2l[j], acc);
      U[(a + XS * b + YS * i) * C + lc] = acc;
    }
  }
  __syncthreads();

  // 7. y-line owner (x=a, z=b): x-face and own y-face y components, D_y^T
  {
    const float* own = FA + (2 * FSA + fpt) * C + lc;  // faces (1, s): tv, t_y part
    const float tv0 = own[0], tv1 = own[FSA * C];
    float tg0 = 0.f, tg1 = 0.f;
    if (SIPG) {
      tg0 = own[KK * C];
      tg1 = own[(FSA + KK) * C];
    }
    float t1[K], w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int pidx = (a + XS * j + YS * b) * C + lc;
      t1[j] = G1[pidx];
      w[j] = U[pidx];
      if (SIPG) t1[j] = fmaf(tb.E[0][j], tg0, fmaf(tb.E[1][j], tg1, t1[j]));
      if (TANG)
        t1[j] = fmaf(ea0, FT[(((0 * 2 + 0) * 2 + 0) * KK + j + KP * b) * C + lc],
                     fmaf(ea1, FT[(((0 * 2 + 1) * 2 + 0) * KK + j + KP * b) * C + lc], t1[j]));
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      float acc = fmaf(tb.E[0][i], tv0, fmaf(tb.E[1][i], tv1, w[i]));
#pragma unroll
      for (int j = 0; j < K; ++j) acc = fmaf(tb.D[j * K + i], t1[j], acc);
      U[(a + XS * i + YS * b) * C + lc] = acc;
    }
  }
  __syncthreads();

  // 8. x-line owner (y=a, z=b): y-face and own x-face x components, D_x^T,
  // then S_x^T (the integrated field is complete along x here)
  {
    const float* own = FA + fpt * C + lc;  // faces (0, s): tv, t_x part
    const float tv0 = own[0], tv1 = own[FSA * C];
    float tg0 = 0.f, tg1 = 0.f;
    if (SIPG) {
      tg0 = own[KK * C];
      tg1 = own[(FSA + KK) * C];
    }
    float t0[K], w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int pidx = (j + XS * a + YS * b) * C + lc;
      t0[j] = G0[pidx];
      w[j] = U[pidx];
      if (SIPG) t0[j] = fmaf(tb.E[0][j], tg0, fmaf(tb.E[1][j], tg1, t0[j]));
      if (TANG)
        t0[j] = fmaf(ea0, FT[(((1 * 2 + 0) * 2 + 0) * KK + j + KP * b) * C + lc],
                     fmaf(ea1, FT[(((1 * 2 + 1) * 2 + 0) * KK + j + KP * b) * C + lc], t0[j]));
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
      float acc = fmaf(tb.E[0][i], tv0, fmaf(tb.E[1][i], tv1, w[i]));
#pragma unroll
      for (int j = 0; j < K; ++j) acc = fmaf(tb.D[j * K + i], t0[j], acc);
      w[i] = acc;
    }
    float o[K];
    f32_line<K, EO_ST>(tb, w, o);
#pragma unroll
    for (int i = 0; i < K; ++i) U[(i + XS * a + YS * b) * C + lc] = o[i];
  }
  __syncthreads();

  // 9. S_y^T
  {
    float w[K], o[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = U[(a + XS * j + YS * b) * C + lc];
    f32_line<K, EO_ST>(tb, w, o);
#pragma unroll
    for (int i = 0; i < K; ++i) U[(a + XS * i + YS * b) * C + lc] = o[i];
  }
  __syncthreads();

  // 10. S_z^T and the store (set) of the cell's dst z-line; optional src.dst
  {
    float w[K];
#pragma unroll
    for (int j = 0; j < K; ++j) w[j] = U[(a + XS * b + YS * j) * C + lc];
    float* o = P.dst + (size_t)cell * K3 + a + K * b;
    const float* s = P.src + (size_t)cell * K3 + a + K * b;
    float r[K];
    f32_line<K, EO_ST>(tb, w, r);
#pragma unroll
    for (int i = 0; i < K; ++i)
      if (valid) o[K2 * i] = r[i];
    if (P.dot_partial) {
      double acc = 0.0;
#pragma unroll
      for (int i = 0; i < K; ++i) acc += (double)r[i] * (double)s[K2 * i];
      // fixed-order block reduction (FA is free since phase 5)
      double* red = reinterpret_cast<double*>(FA);
      red[tid] = valid ? acc : 0.0;
      __syncthreads();
      if (tid < 32) {
        double t = 0.0;
        for (int i = tid; i < NT; i += 32) t += red[i];
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (tid == 0) P.dot_partial[blk] = t;
      }
    }
  }
}

template <int K, int C, int GEO, int OP>
__global__ void __launch_bounds__(C * K * K, f32_min_blocks(K, C, OP))
    apply_f32_kernel(const __grid_constant__ ApplyParams<float> P) {
  if (P.skip != nullptr && *P.skip != 0.0) return;
  f32_body<K, C, GEO, OP>(P.tab, P, (int)blockIdx.x);
}

template <int K, int C, int GEO, int OP>
__global__ void __launch_bounds__(C * K * K, f32_min_blocks(K, C, OP))
    apply_f32_batch(const __grid_constant__ BatchParams<float> B) {
  const int i = batch_op(B, (int)blockIdx.x);
  f32_body<K, C, GEO, OP>(B.tab, B.op[i], (int)blockIdx.x - B.block_start[i]);
}

// Compiled tile shapes (cells per block) of the binary32 kernel.
template <int K>
struct F32Tiles {
  static constexpr int small = f32_tile_small(K);
  static constexpr int large = f32_geometry_block(K);
};

template <int K, int C, int GEO, int OP>
cudaError_t launch_f32_one(const ApplyLaunch& L, int64_t n_cells) {
  ApplyParams<float> P;
  P.tab = *static_cast<const Tables<float>*>(L.tables);
  P.geo = *static_cast<const Geometry<float>*>(L.geometry);
  P.src = static_cast<const float*>(L.src);
  P.dst = static_cast<float*>(L.dst);
  P.dot_partial = L.dot_partial;
  P.skip = L.skip;
  P.C = C;
  P.cell_begin = L.cell_begin;
  P.cell_end = L.cell_end;
  const int smem = f32_smem_bytes(K, OP, C, GEO);
  static bool configured = false;
  if (!configured) {
    cudaError_t e =
        cudaFuncSetAttribute(apply_f32_kernel<K, C, GEO, OP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // shared-memory carveout for the intended resident blocks (percent of
    // the 228 KB maximum); the rest of the unified cache stays L1
    const int want = f32_min_blocks(K, C, OP) * (smem + 1024);
    const int pct = want >= 228 * 1024 ? 100 : (want * 100 + 228 * 1024 - 1) / (228 * 1024);
    e = cudaFuncSetAttribute(apply_f32_kernel<K, C, GEO, OP>, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  (void)n_cells;
  const int64_t grid = (L.cell_end - L.cell_begin + C - 1) / C;
  if (grid <= 0) return cudaSuccess;
  apply_f32_kernel<K, C, GEO, OP><<<(unsigned)grid, C * K * K, smem, L.stream>>>(P);
  return cudaGetLastError();
}

template <int K, int C>
cudaError_t launch_f32_tile(const ApplyLaunch& L, int64_t n_cells) {
  if (L.op == OP_SIPG) {
    if (L.geo == GEO_CART) return launch_f32_one<K, C, GEO_CART, OP_SIPG>(L, n_cells);
    if (L.geo == GEO_FULL) return launch_f32_one<K, C, GEO_FULL, OP_SIPG>(L, n_cells);
    if (L.geo == GEO_POS) return launch_f32_one<K, C, GEO_POS, OP_SIPG>(L, n_cells);
    return launch_f32_one<K, C, GEO_MERGED, OP_SIPG>(L, n_cells);
  }
  if (L.geo == GEO_CART) return launch_f32_one<K, C, GEO_CART, OP_ADV>(L, n_cells);
  if (L.geo == GEO_FULL) return launch_f32_one<K, C, GEO_FULL, OP_ADV>(L, n_cells);
  if (L.geo == GEO_POS) return launch_f32_one<K, C, GEO_POS, OP_ADV>(L, n_cells);
  return launch_f32_one<K, C, GEO_MERGED, OP_ADV>(L, n_cells);
}

template <int K>
cudaError_t launch_apply_f32(const ApplyLaunch& L, int64_t n_cells) {
  if (L.cpb == F32Tiles<K>::large) return launch_f32_tile<K, F32Tiles<K>::large>(L, n_cells);
  if (L.cpb == F32Tiles<K>::small) return launch_f32_tile<K, F32Tiles<K>::small>(L, n_cells);
  return cudaErrorInvalidValue;
}

}  // namespace dg
