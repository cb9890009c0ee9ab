"""FP64 CPU oracle for the matrix-free DG operators (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library: its arithmetic lives in ``dg_oracle.c`` (brute-force quadrature, no
sum factorization), and this module only marshals numpy arrays through
ctypes.

Mesh and form descriptions are plain dicts:
    mesh = {"n": (nx, ny, nz), "periodic": bool, "mapping": 0|1|2, "amplitude": a,
            "cell_jacobian": "analytic"|"g2"}
    (mapping 2: the affine shear x_i = X_i + a X_{(i+1) mod 3}; cell_jacobian
    "g2": the cell term's Jacobian is the collocation derivative of the Gauss
    points' positions, geometry variant G2 of Sec. 5; faces, penalty, rhs
    and errors keep the analytic map; "basis": "lagrange" (default, on the
    Gauss-Lobatto points) or "hermite" (the Hermite-like basis of degree
    >= 3 defined in dg_oracle.c, whose face values and normal derivatives
    each come from one coefficient per face point; Sec. 3.1))
    form = {"op": "sipg"|"advection", "coeff": 0|1,
            "velocity": (c0, c1, c2), "penalty_scale": 1.0}

Functions and the passages of Kronbichler & Kormann (arXiv:1711.03590) they
follow:
    gauss, gauss_lobatto     Sec. 2 (tensor Gauss quadrature; GL nodal basis)
    assemble                 Eq. (matvec) with Eq. (poisson_sip) / Eq. (advection)
                             assembled (route R1)
    apply                    the same operator applied cell by cell (route R2),
                             Algorithm 1 regrouped by test cell
    mass_apply               Sec. 3.1 mass evaluation (interpolate, JxW, integrate)
    rhs, l2_error            manufactured solution u = sin(pi x) sin(pi y) sin(pi z)
    cg                       conjugate gradients on the assembled matrix
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


class _Mesh(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int),
                ("mapping", ctypes.c_int), ("amplitude", ctypes.c_double),
                ("cell_jacobian", ctypes.c_int), ("basis", ctypes.c_int)]


class _Form(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("coeff", ctypes.c_int),
                ("velocity", ctypes.c_double * 3), ("penalty_scale", ctypes.c_double)]


_P = ctypes.POINTER
_d = ctypes.c_double
_i64 = ctypes.c_int64


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.or_gauss.argtypes = [ctypes.c_int, _P(_d), _P(_d)]
        L.or_gauss_lobatto.argtypes = [ctypes.c_int, _P(_d), _P(_d)]
        L.or_lagrange.argtypes = [ctypes.c_int, _P(_d), ctypes.c_int, _d]
        L.or_lagrange.restype = _d
        L.or_lagrange_deriv.argtypes = [ctypes.c_int, _P(_d), ctypes.c_int, _d]
        L.or_lagrange_deriv.restype = _d
        L.or_basis_value.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _d, ctypes.c_int]
        L.or_basis_value.restype = _d
        L.or_cell_volume.argtypes = [_P(_Mesh), ctypes.c_int, _i64]
        L.or_cell_volume.restype = _d
        L.or_apply_cells.argtypes = [_P(_Mesh), ctypes.c_int, _P(_Form), _P(_d), _P(_d),
                                     _P(_i64), _i64]
        L.or_assemble_nnz.argtypes = [_P(_Mesh), ctypes.c_int]
        L.or_assemble_nnz.restype = _i64
        L.or_assemble.argtypes = [_P(_Mesh), ctypes.c_int, _P(_Form), _P(_i64),
                                  _P(ctypes.c_int32), _P(_d)]
        L.or_assemble.restype = _i64
        L.or_spmv.argtypes = [_i64, _P(_i64), _P(ctypes.c_int32), _P(_d), _P(_d), _P(_d)]
        L.or_cg_csr.argtypes = [_i64, _P(_i64), _P(ctypes.c_int32), _P(_d), _P(_d), _P(_d),
                                _d, ctypes.c_int, _P(ctypes.c_int), _P(_d)]
        L.or_mass_apply.argtypes = [_P(_Mesh), ctypes.c_int, _P(_d), _P(_d)]
        L.or_rhs.argtypes = [_P(_Mesh), ctypes.c_int, ctypes.c_int, _P(_d)]
        L.or_l2_error.argtypes = [_P(_Mesh), ctypes.c_int, _P(_d)]
        L.or_l2_error.restype = _d
        L.or_dof_points.argtypes = [_P(_Mesh), ctypes.c_int, _P(_d)]
        L.or_num_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a, t=_d):
    return a.ctypes.data_as(_P(t))


def _mesh(m):
    n = m["n"]
    if isinstance(n, int):
        n = (n, n, n)
    cj = m.get("cell_jacobian", 0)
    cj = {"analytic": 0, "g2": 1}.get(cj, cj)
    bs = m.get("basis", 0)
    bs = {"lagrange": 0, "gl": 0, "hermite": 1}.get(bs, bs)
    return _Mesh((ctypes.c_int * 3)(*n), int(bool(m.get("periodic", False))),
                 int(m.get("mapping", 0)), float(m.get("amplitude", 0.0)), int(cj), int(bs))


def _form(f):
    op = f.get("op", "sipg")
    op = {"sipg": 0, "advection": 1}.get(op, op)
    v = f.get("velocity", (1.0, 0.5, 0.25))
    return _Form(int(op), int(f.get("coeff", 0)), (_d * 3)(*v),
                 float(f.get("penalty_scale", 1.0)))


def n_cells(mesh):
    n = mesh["n"]
    if isinstance(n, int):
        return n ** 3
    return int(n[0]) * int(n[1]) * int(n[2])


def n_dofs(mesh, degree):
    return n_cells(mesh) * (degree + 1) ** 3


def num_threads():
    return lib().or_num_threads()


def gauss(k):
    x = np.zeros(k)
    w = np.zeros(k)
    if lib().or_gauss(k, _ptr(x), _ptr(w)):
        raise ValueError("bad k")
    return x, w


def gauss_lobatto(k):
    x = np.zeros(k)
    w = np.zeros(k)
    if lib().or_gauss_lobatto(k, _ptr(x), _ptr(w)):
        raise ValueError("bad k")
    return x, w


def lagrange(nodes, j, t, deriv=False):
    nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    fn = lib().or_lagrange_deriv if deriv else lib().or_lagrange
    return fn(len(nodes), _ptr(nodes), j, float(t))


def basis_value(kind, degree, j, t, deriv=False):
    """1D basis function j (kind "lagrange" or "hermite") at t, or its derivative."""
    kind = {"lagrange": 0, "gl": 0, "hermite": 1}.get(kind, kind)
    return lib().or_basis_value(int(kind), int(degree), int(j), float(t), int(bool(deriv)))


def cell_volume(mesh, degree, cell):
    return lib().or_cell_volume(ctypes.byref(_mesh(mesh)), degree, cell)


def apply(mesh, degree, form, u, cells=None):
    """y = A u (route R2).  With ``cells`` only those cells' rows are
    computed; the other entries of the returned vector are NaN."""
    u = np.ascontiguousarray(u, dtype=np.float64)
    n = n_dofs(mesh, degree)
    if u.shape != (n,):
        raise ValueError("u has shape %s, expected (%d,)" % (u.shape, n))
    y = np.full(n, np.nan)
    if cells is None:
        cp, nc = None, 0
    else:
        cells = np.ascontiguousarray(cells, dtype=np.int64)
        cp, nc = _ptr(cells, _i64), len(cells)
    rc = lib().or_apply_cells(ctypes.byref(_mesh(mesh)), degree, ctypes.byref(_form(form)),
                              _ptr(u), _ptr(y), cp, nc)
    if rc:
        raise RuntimeError("or_apply_cells failed: %d" % rc)
    return y


def assemble(mesh, degree, form):
    """Assembled sparse matrix (route R1) as a scipy CSR matrix."""
    import scipy.sparse as sp
    m = _mesh(mesh)
    n = n_dofs(mesh, degree)
    nnz = lib().or_assemble_nnz(ctypes.byref(m), degree)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    got = lib().or_assemble(ctypes.byref(m), degree, ctypes.byref(_form(form)),
                            _ptr(rowptr, _i64), _ptr(col, ctypes.c_int32), _ptr(val))
    if got != nnz:
        raise RuntimeError("or_assemble returned %d, expected %d" % (got, nnz))
    return sp.csr_matrix((val, col, rowptr), shape=(n, n))


def spmv(A, x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.zeros(A.shape[0])
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    lib().or_spmv(A.shape[0], _ptr(indptr, _i64), _ptr(indices, ctypes.c_int32), _ptr(data),
                  _ptr(x), _ptr(y))
    return y


def cg(A, b, x0=None, rtol=1e-10, maxit=10000):
    """CG on the assembled matrix; returns (x, iterations, relative residual)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    indptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
    indices = np.ascontiguousarray(A.indices, dtype=np.int32)
    data = np.ascontiguousarray(A.data, dtype=np.float64)
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0)
    lib().or_cg_csr(A.shape[0], _ptr(indptr, _i64), _ptr(indices, ctypes.c_int32), _ptr(data),
                    _ptr(b), _ptr(x), rtol, maxit, ctypes.byref(it), ctypes.byref(rr))
    return x, it.value, rr.value


def mass_apply(mesh, degree, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    y = np.zeros_like(u)
    lib().or_mass_apply(ctypes.byref(_mesh(mesh)), degree, _ptr(u), _ptr(y))
    return y


def rhs(mesh, degree, which=0):
    """(phi_i, f) for f = 3 pi^2 u (which=0) or -div(kappa grad u) (which=1)."""
    y = np.zeros(n_dofs(mesh, degree))
    lib().or_rhs(ctypes.byref(_mesh(mesh)), degree, which, _ptr(y))
    return y


def l2_error(mesh, degree, u):
    u = np.ascontiguousarray(u, dtype=np.float64)
    return lib().or_l2_error(ctypes.byref(_mesh(mesh)), degree, _ptr(u))


def dof_points(mesh, degree):
    xyz = np.zeros((n_dofs(mesh, degree), 3))
    lib().or_dof_points(ctypes.byref(_mesh(mesh)), degree, _ptr(xyz))
    return xyz
