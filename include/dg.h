/*
 * dg.h -- C ABI of the GB300 (sm_103a) matrix-free discontinuous Galerkin
 * operator library.
 *
 * The library evaluates y = A u (Kronbichler & Kormann, arXiv:1711.03590,
 * Sec. 2, Eq. (matvec)) for two weak forms on hexahedral meshes of the unit
 * cube with a tensor-product Lagrange basis on the k = p+1 Gauss-Lobatto
 * points and k Gauss points per direction:
 *   - the symmetric interior penalty Laplacian, Eq. (poisson_sip), with the
 *     average/jump definitions and the Dirichlet mirror principle of Sec. 2;
 *   - the upwind advection operator, Eq. (advection), with the boundary flux
 *     |c.n| u- of Algorithm 1 step (iv)(c).
 * Cell integrals use the sum-factorized basis change and collocation
 * derivative of Eq. (tensor_to_collocation); face integrals interpolate both
 * sides' traces as in Eq. (face_integral); the geometry is stored per
 * quadrature point (variants G3/G4 of Sec. 5) or compressed (Cartesian).
 *
 * Degrees of freedom.  Cell c = ix + n0 (iy + n1 iz) owns the contiguous
 * range [c k^3, (c+1) k^3); its dof (i0, i1, i2) sits at c k^3 + i0 +
 * k (i1 + k i2) (x fastest), the Lagrange node at the Gauss-Lobatto points.
 * Cell c maps the reference cube [0,1]^3 onto its box of the unit cube and,
 * for mapping 1, shifts every coordinate by a sin(pi X) sin(pi Y) sin(pi Z)
 * (mapping 2: the linear shear x_i = X_i + a X_{(i+1) mod 3}).
 *
 * Conventions for every call:
 *   - Device pointers are CUDA device addresses of the current device with
 *     n_dofs contiguous scalars of the handle's precision (double for
 *     DG_FP64 and DG_FP64_EMU, float for DG_FP32), 16-byte aligned.  The
 *     caller owns them.
 *   - Calls are stream-ordered on the handle's stream and asynchronous,
 *     unless stated otherwise.
 *   - Errors are returned as dg_status codes, never by aborting; a message is
 *     kept in the handle (dg_last_error).  DG_ERR_CUDA means a CUDA call
 *     failed; the handle should then be destroyed.
 *   - A handle is not thread-safe: use one handle per host thread.
 */
#ifndef DG_GB300_H
#define DG_GB300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,            /* invalid argument (null, size, aliasing, degree, geometry) */
  DG_ERR_OOM = 2,            /* device or host allocation failed */
  DG_ERR_CUDA = 3,           /* a CUDA runtime call or kernel launch failed */
  DG_ERR_UNSUPPORTED = 4,    /* valid but unsupported combination */
  DG_ERR_NOT_CONVERGED = 5,  /* CG reached max_it; x holds the last iterate */
  DG_ERR_BREAKDOWN = 6,      /* CG found p.Ap <= 0 or a non-finite scalar */
  DG_ERR_TIMEOUT = 7         /* reserved for bounded device waits */
} dg_status;

typedef enum { DG_OP_SIPG = 0, DG_OP_ADVECTION = 1 } dg_op;

/* Geometry storage (Sec. 5).
 *  CARTESIAN: identity mapping only; constant J^{-1} and det J per mesh,
 *             no per-point arrays (the kappa coefficient, when enabled, is a
 *             table over x positions).
 *  (Value 1 is not a geometry variant: a per-cell compressed storage for
 *  affine cells is not offered; affine (sheared, mapping 2) meshes take
 *  FULL_JAC, MERGED or POSITIONS, and dg_setup answers 1 with DG_ERR_ARG.)
 *  FULL_JAC:  variant G3: per cell quadrature point J^{-1} (9 values) and
 *             det J * w (* kappa for SIPG) (1 value) -- for SIPG in binary64
 *             and double-float storage the weight is folded in as
 *             sqrt(kappa det J w) J^{-1} (9 values); per face quadrature
 *             point and side n.J^{-T} (3 values each, Design Choice
 *             "normal times inverse Jacobian") and kappa*da*w (1 value), and
 *             one penalty per face -- in binary64 and double-float storage
 *             the vectors are stored times kappa*da*w and the weight times
 *             the penalty.  Advection stores c.n da w (1 value) per face
 *             point instead.
 *  MERGED:    variant G4: per cell quadrature point the merged coefficient
 *             kappa det J w J^{-1} J^{-T} (6 values, SIPG) or
 *             -det J w J^{-1} c (3 values, advection); faces as FULL_JAC.
 *  POSITIONS: variant G2: per cell quadrature point its physical position
 *             (3 values) and, for SIPG, kappa (1 value); the kernels compute
 *             J at each point by the collocation derivative of the positions
 *             along the three lines through it (the derivative of the degree-p
 *             interpolant of the map through the Gauss points), then det J
 *             and J^{-1}; faces as FULL_JAC (face data is stored separately,
 *             as Sec. 5 notes for Gauss rules).  Binary64 and double-float
 *             operators run the face loop (dg_setup selects DG_FACE_LOOP and
 *             allocates its work arrays; DG_FACE_ELEMENT is refused). */
typedef enum {
  DG_GEOM_CARTESIAN = 0,
  DG_GEOM_FULL_JAC = 2,
  DG_GEOM_MERGED = 3,
  DG_GEOM_POSITIONS = 4
} dg_geom;

/* Arithmetic of the apply.
 *  DG_FP64:     IEEE binary64 vectors and arithmetic (the FP64 pipe).
 *  DG_FP32:     binary32 vectors and arithmetic.
 *  DG_FP64_EMU: binary64 vectors; arithmetic in double-float (pairs of
 *               binary32 numbers, ~48-bit significand) on the FP32 pipe, which
 *               GB300 runs 64x faster than its FP64 pipe.  Accuracy is held to
 *               the same 1e-12 relative tolerance as DG_FP64; values keep full
 *               accuracy for magnitudes in about [1e-30, 1e38]. */
typedef enum { DG_FP64 = 0, DG_FP32 = 1, DG_FP64_EMU = 2 } dg_prec;

typedef struct {
  int n[3];         /* cells per direction, each >= 1 */
  int periodic;     /* 1: periodic in every direction; 0: Dirichlet (g = 0) on all of the boundary */
  int mapping;      /* 0: identity; 1: x_i = X_i + amplitude sin(pi X) sin(pi Y) sin(pi Z);
                       2: the shear x_i = X_i + amplitude X_{(i+1) mod 3} (constant J per cell;
                       with periodic boundaries only kappa = 1, since x_0 shifts across the wrap) */
  double amplitude; /* used by mappings 1 and 2; det J must stay positive */
} dg_mesh;

typedef struct {
  int op;               /* dg_op */
  int prec;             /* dg_prec: arithmetic and storage precision of apply */
  double velocity[3];   /* advection speed c (constant vector) */
  int coeff;            /* SIPG coefficient: 0 kappa = 1; 1 kappa = 1 + 0.5 sin(2 pi x_0) */
  double penalty_scale; /* tau = penalty_scale (p+1)^2 max(A_F/|K-|, A_F/|K+|); <= 0 means 1 */
  int basis;            /* dg_basis: DG_BASIS_LAGRANGE (the workloads' basis) or DG_BASIS_HERMITE */
} dg_opts;

/* Polynomial basis of each direction (the dof layout is the same: index i
 * of direction d is basis function i).
 *  LAGRANGE: Lagrange polynomials on the k Gauss-Lobatto points.
 *  HERMITE:  the Hermite-like basis (degree >= 3) with the face property of
 *            Sec. 3.1: at xi = 0 only function 0 is nonzero (value 1) and
 *            only function 1 has a nonzero derivative, mirror-symmetric at
 *            xi = 1 (functions p and p-1).  With the Gauss-Lobatto points
 *            g_0 = 0 < g_1 < ... < g_p = 1 and w(t) = prod_{j=2}^{p-2}
 *            (t - g_j): f_0 = (1-t)^2 (1 + c t) w(t) / w(0) with c such
 *            that f_0'(0) = 0; f_1 = t (1-t)^2 w(t) scaled to f_1(g_1) = 1;
 *            f_j (2 <= j <= p-2) = t^2 (1-t)^2 times the Lagrange
 *            polynomial on g_2 .. g_{p-2} that is 1 at g_j, scaled to
 *            f_j(g_j) = 1; f_{p-1}(t) = f_1(1-t), f_p(t) = f_0(1-t) (nodal at
 *            the interior points, for conditioning).  Same operator as
 *            LAGRANGE in another basis of the same space. */
typedef enum { DG_BASIS_LAGRANGE = 0, DG_BASIS_HERMITE = 1 } dg_basis;

typedef struct dg_handle dg_handle;
typedef struct dg_server dg_server;

/* Static sizes of a set-up operator, for bandwidth accounting. */
typedef struct {
  int64_t n_dofs;
  int64_t n_cells;
  int degree;
  int prec;
  int geom;
  int op;
  int64_t cell_geometry_bytes;  /* per-quadrature-point cell arrays read by one apply */
  int64_t face_geometry_bytes;  /* per-face arrays read by one apply */
  int cells_per_block;          /* cells processed by one CUDA block of the apply kernel */
  int threads_per_block;
  int shared_bytes_per_block;
  int64_t blocks;               /* blocks of one apply launch */
  int tile_choices[24];         /* valid cells_per_block values, ascending, 0-terminated */
  int face_mode;                /* DG_FACE_ELEMENT or DG_FACE_LOOP (dg_set_face_mode) */
} dg_info_t;

/* Build an operator: 1D tables, geometry arrays and work buffers on the
 * current CUDA device, computed in FP64 and stored in opts->prec.
 *   mesh    mesh description (copied).
 *   degree  polynomial degree p, 1..8.
 *   geom    dg_geom storage variant.
 *   opts    operator options (copied).
 *   stream  cudaStream_t used by every later call (NULL = legacy default stream).
 *   out     receives the handle; on error *out is NULL.
 * Returns DG_ERR_ARG for invalid sizes, degree, geometry/mapping mismatch
 * (CARTESIAN needs mapping 0) or a non-positive det J; DG_ERR_OOM if device
 * memory runs out.  Blocks until set-up is complete.
 * Cite: Sec. 5 (G2, G3, G4, compressed Cartesian), Design Choice on j_n. */
dg_status dg_setup(const dg_mesh *mesh, int degree, int geom, const dg_opts *opts, void *stream,
                   dg_handle **out);

/* Number of degrees of freedom n = n0 n1 n2 (p+1)^3 (the dimension of the
 * DG space of Sec. 2: (p+1)^3 Lagrange coefficients per cell).  Synchronous. */
dg_status dg_n_dofs(const dg_handle *h, int64_t *n);

/* Sizes of the operator's data (see dg_info_t).  Synchronous. */
dg_status dg_info(const dg_handle *h, dg_info_t *info);

/* Change the stream used by later calls. */
dg_status dg_set_stream(dg_handle *h, void *stream);

/* Tile shape of the apply kernel: cells per CUDA block (k^2 threads each).
 * Valid values are listed in dg_info_t.tile_choices: for DG_FP64 and
 * DG_FP64_EMU any value 1 .. floor(256 / k^2) (the autotuner tries a subset),
 * for DG_FP32 one of the two compiled shapes.  0 restores the default
 * (which for DG_FACE_LOOP is its own per-degree default).  Results do not
 * depend on it (each cell's arithmetic is the same); an invalid value
 * returns DG_ERR_ARG.  Synchronous. */
dg_status dg_set_cells_per_block(dg_handle *h, int cells_per_block);

/* Face evaluation of the DG_FP64 / DG_FP64_EMU apply.  DG_FACE_ELEMENT (default): one
 * fused kernel, every cell evaluates its six faces (the neighbour's traces
 * re-interpolated from its dofs).  DG_FACE_LOOP: two launches -- cells write
 * their own face traces (u and the reference gradient, per face and side) and
 * q-point fields; then cells read both sides' traces of their six faces, form
 * the flux tested on their own side, inject and integrate (the paper's
 * separate cell and face work, Algorithm 1 steps (ii)-(iv), without atomics)
 * -- trading memory traffic for FP64 arithmetic.  Same results up to
 * rounding.  DG_FACE_LOOP allocates its work arrays here (on first use; they
 * stay with the handle until dg_destroy): 24/k + 3 doubles per dof for SIPG
 * (62 bytes per dof at p = 4), 6/k + 3 for advection.  DG_ERR_OOM if they do
 * not fit (the mode is then unchanged).
 * DG_FP64 and DG_FP64_EMU handles; DG_FP32: DG_ERR_UNSUPPORTED.  The face
 * loop takes the x faces' values from the end layers of the x lines, so it
 * needs a basis whose value at each end of the interval is its end
 * coefficient (both bases here are; another basis: DG_ERR_UNSUPPORTED).  A tile
 * shape equal to the previous mode's default moves to the new mode's
 * default; any other stays.  Synchronous. */
typedef enum { DG_FACE_ELEMENT = 0, DG_FACE_LOOP = 1 } dg_face_mode;
dg_status dg_set_face_mode(dg_handle *h, int mode);

/* Autotuner: times the apply for every value in tile_choices on
 * the handle's stream (CUDA events, warm-up first) and keeps the fastest.
 * Uses handle-owned staging buffers (allocated on first use).  best_cpb and
 * best_ms (may be NULL) receive the choice and its time per apply.
 * Synchronous. */
dg_status dg_autotune(dg_handle *h, int *best_cpb, double *best_ms);

/* dst = A src on the device (Algorithm 1 steps (ii)-(iv); one kernel launch,
 * two with DG_FACE_LOOP: each cell computes its cell integral and its six
 * face integrals tested on itself and sets its dst entries).  src and dst: device pointers to n_dofs
 * scalars of the handle's precision; src == dst, or overlapping ranges, give
 * DG_ERR_ARG.  Asynchronous. */
dg_status dg_apply(dg_handle *h, const void *src, void *dst);

/* The same operator with HOST buffers: copies src to the device, applies,
 * copies the result back, and waits for the stream.  Pinned host memory
 * makes the copies asynchronous DMA; on non-periodic meshes whose z-planes
 * hold a multiple of 64 cells the work is pipelined over up to 8 slabs of
 * z-planes (copies in, applies and copies out overlap; with DG_FACE_LOOP a
 * slab's second launch follows the next slab's first; the result is the
 * same bits as dg_apply).  Device staging buffers, two copy streams, a
 * second compute stream and their events are created on the first call and
 * kept by the handle. */
dg_status dg_apply_host(dg_handle *h, const void *src_host, void *dst_host);

/* rhs_i = (phi_i, f) for the manufactured solution u = sin(pi x) sin(pi y)
 * sin(pi z) (Dirichlet g = 0), by the (k+2)-point Gauss rule per direction,
 * in FP64 regardless of the handle's precision.
 *   which_f 0: f = 3 pi^2 u (-Laplace u);  1: f = -div(kappa grad u) with
 *   kappa = 1 + 0.5 sin(2 pi x_0).
 * rhs: device pointer to n_dofs doubles.  Asynchronous.
 * No counterpart in the paper (it reports operator evaluations, not solves);
 * the load vector is the right-hand side of the weak form of Sec. 2. */
dg_status dg_rhs(dg_handle *h, int which_f, double *rhs);

/* err = || u_h - u ||_{L2(Omega)} for the coefficient vector x (device, n_dofs
 * doubles) against the manufactured u = sin(pi x) sin(pi y) sin(pi z), by the
 * (k+2)-point Gauss rule per direction on the mapped cells.  Synchronous.
 * (Evaluation aid for the solvers; the paper reports no solves.) */
dg_status dg_l2_error(dg_handle *h, const double *x, double *err);

/* Conjugate gradients for A x = rhs (SIPG only; DG_ERR_UNSUPPORTED for
 * advection, which is not symmetric).  rhs, x: device pointers to n_dofs
 * doubles; x holds the initial guess on entry and the last iterate on exit.
 * Each iteration: one apply with p.Ap fused into the apply epilogue, then
 * one fused vector update x += alpha p, r -= alpha Ap with r.r, then
 * p = r + beta p.  All reductions are two-stage in a fixed order, so results
 * are bitwise reproducible on a given device and size.  An FP32 handle
 * returns DG_ERR_UNSUPPORTED (see dg_cg_solve_mixed); DG_FP64_EMU handles
 * run the same CG with their emulated-FP64 apply.
 * Stops when |r| <= rtol |rhs|.  Returns DG_ERR_NOT_CONVERGED after max_it
 * iterations and DG_ERR_BREAKDOWN on p.Ap <= 0 or non-finite scalars.
 * iters and final_rel_res (may be NULL) receive the count and |r|/|rhs|.
 * Synchronous.  No counterpart in the paper: it evaluates the operator for
 * iterative solvers (Sec. 1 and the conclusions) without giving one; this is
 * textbook CG on the SPD operator of Eq. (poisson_sip). */
dg_status dg_cg_solve(dg_handle *h, const double *rhs, double *x, double rtol, int max_it, int *iters,
                      double *final_rel_res);

/* Mixed-precision solve of A x = rhs (SIPG): conjugate gradients in a
 * cheaper arithmetic with residual replacement ("reliable updates") by the
 * FP64 residual.  h64 and h32 describe the same operator (mesh, degree,
 * geometry, coefficient, penalty); h64 is DG_FP64 (or DG_FP64_EMU), h32 the
 * inner handle: DG_FP32 (binary32 vectors and applies) or DG_FP64_EMU
 * (binary64 vectors, double-float applies).  The inner CG works on the
 * system scaled by 1 / |r| (every inner product accumulated in FP64); once
 * its recursive residual has dropped by inner_rtol against the largest since
 * the last replacement (or reached the scaled target, or after max_inner
 * iterations), its solution is added to x in FP64, r = rhs - A x is
 * recomputed with h64, and the recursion continues from the new r with
 * beta = |r|^2 / |r_old|^2 and p = r + beta p, so the search directions
 * built so far are kept (Sleijpen & van der Vorst 1996; Clark et al. 2010).
 * Stops when |r| <= rtol |rhs| with the FP64 residual.  rhs, x: device
 * pointers to n_dofs doubles; x is the initial guess on entry.  Work vectors
 * are allocated on first use.  Ordered on h64's stream.  Returns
 * DG_ERR_NOT_CONVERGED after max_outer replacements or when four
 * replacements in a row do not halve the best residual (the attainable
 * floor of an emulated-FP64 h64, about 2e-10 relative at p = 5);
 * DG_ERR_BREAKDOWN on a non-finite residual or an inner breakdown.
 * outer_iters (replacements), inner_iters (inner iterations), final_rel_res
 * may be NULL.  Synchronous.  (Beyond the paper, whose solvers are only
 * referred to in Sec. 1 and Sec. 6.) */
dg_status dg_cg_solve_mixed(dg_handle *h64, dg_handle *h32, const double *rhs, double *x, double rtol,
                            int max_outer, double inner_rtol, int max_inner, int *outer_iters, int *inner_iters,
                            double *final_rel_res);

/* The same with the inner arithmetic chosen by measurement: double-float
 * iterations (hemu, DG_FP64_EMU) in chunks of 16, at most 48, measure the
 * convergence rate; as soon as at that rate the remaining iterations are few
 * (<= 200) the double-float recursion continues (a binary32 recursion would
 * add rounding noise across the whole spectrum, which CG must then remove:
 * on smooth, fast-converging problems that costs far more iterations than it
 * saves per iteration); after 48 without that, the binary32 recursion (h32,
 * DG_FP32) takes over from the current x.  h64,
 * hemu and h32 describe the same operator.  inner_prec (may be NULL)
 * receives the inner arithmetic used after the probe (DG_FP64_EMU or
 * DG_FP32); the counts include the probe.  Other arguments and results as
 * dg_cg_solve_mixed.  Synchronous. */
dg_status dg_cg_solve_mixed_auto(dg_handle *h64, dg_handle *hemu, dg_handle *h32, const double *rhs, double *x,
                                 double rtol, int max_outer, double inner_rtol, int max_inner, int *outer_iters,
                                 int *inner_iters, double *final_rel_res, int *inner_prec);

/* Batched evaluation (beyond the paper, which evaluates one operator
 * at a time).  A batch applies count set-up operators -- any mix of meshes,
 * degrees, geometries, precisions and face modes -- with one CUDA graph
 * launch.  Operators sharing a kernel (degree, precision, geometry variant,
 * weak form, face mode) form a group that runs as fused launches: one grid
 * holds the blocks of up to 64 operators (larger operators first), each
 * block finding its operator in a prefix table of block counts, so small
 * meshes fill the SMs together instead of one launch each; face-loop groups
 * take two such launches.  The groups' launches are dealt to branches of the
 * graph, largest groups first, so groups of different degrees overlap.
 * handles[i], srcs[i], dsts[i]: operator i and its device vectors (as for
 * dg_apply; two operators may not share a dst); the pointers are fixed at
 * creation.  autotune != 0: each group's tile shape (cells per block) is
 * chosen by timing the group's fused launch for every valid tile shape
 * (dg_info_t.tile_choices); otherwise the group takes its first (largest)
 * operator's.  Every member's tile shape is set to its group's
 * (dg_set_cells_per_block).  branches (1..32): graph branches.  stream: the
 * cudaStream_t dg_batch_launch launches on.  Creation performs one plain
 * apply per operator, tunes, captures the graph and blocks until done.  The
 * handles must outlive the batch and must not change tile shape or face mode
 * afterwards.  Results equal the single applies bit for bit. */
typedef struct dg_batch dg_batch;
dg_status dg_batch_create(dg_handle *const *handles, const void *const *srcs, void *const *dsts, int count,
                          int autotune, int branches, void *stream, dg_batch **out);
/* Number of kernel groups and of kernel launches per dg_batch_launch. */
dg_status dg_batch_info(const dg_batch *b, int *groups, int *launches);
/* All applies of the batch, asynchronously on the batch's stream. */
dg_status dg_batch_launch(dg_batch *b);
dg_status dg_batch_destroy(dg_batch *b);
/* Message of the last batch error of the calling thread. */
const char *dg_batch_last_error(void);

/* Solve server (beyond the paper: serving with continuous batching).
 * A request is a Poisson problem -div(kappa grad u) = f with the
 * manufactured u = sin(pi x) sin(pi y) sin(pi z), Dirichlet boundary,
 * solved by dg_cg_solve_mixed (binary32 inner CG) on its own FP64 and FP32
 * operators.  Requests are
 * queued in arrival order; `slots` worker threads (one CUDA stream each)
 * admit a queued request (the oldest, or by dg_server_set_policy) as soon as
 * a slot is free and its estimated device memory (dg_request_device_bytes)
 * fits into the remaining budget, so the work of all admitted requests
 * overlaps on the device.  A result does
 * not depend on the other requests (fixed-order reductions): it is the same
 * alone and in the mix, bit for bit.  Device memory comes from the
 * stream-ordered pool, which keeps freed memory for later requests. */
typedef struct {
  int n[3];            /* cells per direction */
  int periodic;        /* 0 (Dirichlet) for the manufactured problem */
  int mapping;         /* 0 identity, 1 sine map */
  double amplitude;
  int degree;          /* 1..8 */
  int geom;            /* dg_geom (CARTESIAN needs mapping 0) */
  int coeff;           /* kappa variant, as dg_opts.coeff */
  int which_f;         /* right-hand side, as dg_rhs: 0 for coeff 0, 1 for coeff 1 */
  double rtol;         /* outer relative residual */
  double inner_rtol;   /* FP32 inner reduction per correction */
  int max_outer, max_inner;
  double *x_host;      /* optional: receives the n_dofs solution values (host memory) */
} dg_request;

typedef struct {
  int status;          /* dg_status of the solve */
  int outer_iters, inner_iters;
  double rel_res;
  int64_t n_dofs;
  int64_t device_bytes;        /* the admission estimate */
  double t_submit, t_admit, t_done;  /* seconds since the server was created */
  char message[160];           /* error message when status != DG_OK */
} dg_result;

/* Device memory, in bytes, that the server budgets for a request: the
 * geometry of its FP64 and FP32 operators, the solver's vectors and set-up
 * scratch (per dof, from the degree and the geometry storage), plus 64 MiB.
 * -1 for an invalid request (NULL, degree outside 1..8, or a mesh extent
 * below 1).  Host arithmetic only; no device work.  No counterpart in the
 * paper. */
int64_t dg_request_device_bytes(const dg_request *r);
dg_status dg_server_create(int device, int64_t budget_bytes, int slots, dg_server **out);
/* Admission policy: which queued request a free slot takes.  policy 0
 * (default): FIFO, the oldest request once it fits into the remaining
 * budget.  policy 1: shortest job first with aging -- a request queued
 * longer than max_age_s seconds goes first (oldest first); otherwise the
 * smallest estimated work (dofs x (p+1)) among the requests that fit.
 * Applies to later admissions. */
dg_status dg_server_set_policy(dg_server *s, int policy, double max_age_s);
dg_status dg_server_submit(dg_server *s, const dg_request *r, int64_t *ticket);
/* Blocks until the request is done; each ticket can be waited for once. */
dg_status dg_server_wait(dg_server *s, int64_t ticket, dg_result *out);
/* Finishes every submitted request, then stops the workers. */
dg_status dg_server_destroy(dg_server *s);
const char *dg_server_last_error(void);

/* No counterpart in the paper: an allocation-free variant of the apply with
 * the FP64 product src . dst that the CG iteration fuses into the apply.
 *
 * For callers that cannot call cudaMalloc once they are running: code inside
 * a device-memory pool owned by another framework, a real-time loop that
 * must not enter the allocator, or a process whose device memory is already
 * fully handed out.  The per-block partial sums of the product, which
 * dg_cg_solve keeps in memory it allocates, live here in a fixed static
 * device array of the library (65,536 partials, about 512 KiB, held by
 * every GPU that loads the library until the process exits).
 *   src, dst  device pointers as for dg_apply (dst = A src, same kernel).
 *   dot       device pointer to one double; receives sum_i src_i dst_i,
 *             reduced in a fixed order (bitwise reproducible).
 * Operators whose apply needs more than 65,536 CUDA blocks (see
 * dg_info_t.blocks) are rejected with DG_ERR_ARG.  No call allocates or
 * frees memory: dg_setup, which allocates anyway, loads the library module
 * that holds the array (with lazy module loading the array's memory is
 * allocated at that load) and looks up its device address
 * (cudaGetSymbolAddress) with the handle's device current, once per device.
 * The first dg_setup on a device must therefore come before any stream
 * capture that records this call.  All calls share the array: calls that
 * overlap on the GPU race on it and must be ordered by the caller.
 * Asynchronous on the handle's stream. */
dg_status dg_apply_dot_noalloc(dg_handle *h, const void *src, void *dst, double *dot);

/* Measurement aid, no counterpart in the paper: the FMA throughput of the
 * current device, measured by a kernel of independent fused multiply-add
 * chains (a whole number of resident blocks per SM; best of four timed
 * launches after a warm-up, CUDA events; the best of a few shapes of chains
 * per thread and threads per block).
 *   kind    0: binary64 FMA (the FP64 pipe), 1: binary32 FMA.
 *   tflops  receives 2 x FMAs per second / 1e12.
 * Allocates and frees a small device buffer; synchronous (legacy default
 * stream).  DG_ERR_ARG for another kind or a NULL tflops. */
dg_status dg_peak_probe(int kind, double *tflops);

/* Free everything the handle owns.  NULL is accepted.  No counterpart in the
 * paper (resource management of this library). */
dg_status dg_destroy(dg_handle *h);

/* Message of the last error on this handle ("" if none); for errors before a
 * handle exists, dg_last_error(NULL) returns the last set-up message of the
 * calling thread. */
const char *dg_last_error(const dg_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* DG_GB300_H */
