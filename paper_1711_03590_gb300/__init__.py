"""GB300 (sm_103a) matrix-free DG operators: Python binding of the C ABI.

Thin ctypes marshalling over ``_build/libdg_gb300.so`` (declared in
``include/dg.h``).  The functions keep the C names (``dg_setup``,
``dg_apply``, ...); every step of an operator evaluation runs in the CUDA
kernels of the library.  There is no CPU fallback: if the library is
missing, importing the bindings raises ``DGLibraryMissing``; call
``build()`` first (``__graft_entry__.build()`` does).

PyTorch is used only to hand device memory and streams to the library:
tensors must be CUDA, contiguous, of the handle's dtype (float64 for FP64,
float32 for FP32) and hold n_dofs entries.

Reference: Kronbichler & Kormann, arXiv:1711.03590 -- Sec. 2 (weak forms,
Algorithm 1), Sec. 3.1 (sum factorization), Sec. 5 (geometry variants).
"""
import ctypes
import os

from .build import LIB, build  # noqa: F401

DG_OK = 0
DG_ERR_ARG = 1
DG_ERR_OOM = 2
DG_ERR_CUDA = 3
DG_ERR_UNSUPPORTED = 4
DG_ERR_NOT_CONVERGED = 5
DG_ERR_BREAKDOWN = 6
DG_ERR_TIMEOUT = 7
STATUS_NAMES = {0: "DG_OK", 1: "DG_ERR_ARG", 2: "DG_ERR_OOM", 3: "DG_ERR_CUDA", 4: "DG_ERR_UNSUPPORTED",
                5: "DG_ERR_NOT_CONVERGED", 6: "DG_ERR_BREAKDOWN", 7: "DG_ERR_TIMEOUT"}

DG_OP_SIPG = 0
DG_OP_ADVECTION = 1
DG_GEOM_CARTESIAN = 0
DG_GEOM_FULL_JAC = 2
DG_GEOM_MERGED = 3
DG_GEOM_POSITIONS = 4
DG_FACE_ELEMENT = 0
DG_FACE_LOOP = 1
DG_FP64 = 0
DG_FP32 = 1
DG_FP64_EMU = 2

GEOMS = {"cartesian": DG_GEOM_CARTESIAN, "full": DG_GEOM_FULL_JAC,
         "merged": DG_GEOM_MERGED, "positions": DG_GEOM_POSITIONS}
OPS = {"sipg": DG_OP_SIPG, "advection": DG_OP_ADVECTION}
PRECS = {"fp64": DG_FP64, "fp32": DG_FP32, "fp64emu": DG_FP64_EMU}
DG_BASIS_LAGRANGE = 0
DG_BASIS_HERMITE = 1
BASES = {"lagrange": DG_BASIS_LAGRANGE, "hermite": DG_BASIS_HERMITE}

EXPORTED = ["dg_setup", "dg_n_dofs", "dg_info", "dg_set_stream", "dg_apply", "dg_apply_host", "dg_rhs",
            "dg_cg_solve", "dg_cg_solve_mixed", "dg_destroy", "dg_last_error", "dg_apply_dot_noalloc",
            "dg_set_cells_per_block", "dg_autotune", "dg_batch_create", "dg_batch_launch", "dg_batch_destroy",
            "dg_batch_last_error", "dg_request_device_bytes", "dg_server_create", "dg_server_submit",
            "dg_server_wait", "dg_server_destroy", "dg_server_last_error", "dg_l2_error", "dg_set_face_mode",
            "dg_peak_probe", "dg_batch_info", "dg_server_set_policy", "dg_cg_solve_mixed_auto"]


class DGLibraryMissing(RuntimeError):
    pass


class DGError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))


class dg_mesh(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int), ("mapping", ctypes.c_int),
                ("amplitude", ctypes.c_double)]


class dg_opts(ctypes.Structure):
    _fields_ = [("op", ctypes.c_int), ("prec", ctypes.c_int), ("velocity", ctypes.c_double * 3),
                ("coeff", ctypes.c_int), ("penalty_scale", ctypes.c_double), ("basis", ctypes.c_int)]


class dg_info_t(ctypes.Structure):
    _fields_ = [("n_dofs", ctypes.c_int64), ("n_cells", ctypes.c_int64), ("degree", ctypes.c_int),
                ("prec", ctypes.c_int), ("geom", ctypes.c_int), ("op", ctypes.c_int),
                ("cell_geometry_bytes", ctypes.c_int64), ("face_geometry_bytes", ctypes.c_int64),
                ("cells_per_block", ctypes.c_int), ("threads_per_block", ctypes.c_int),
                ("shared_bytes_per_block", ctypes.c_int), ("blocks", ctypes.c_int64),
                ("tile_choices", ctypes.c_int * 24), ("face_mode", ctypes.c_int)]


class dg_request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int * 3), ("periodic", ctypes.c_int), ("mapping", ctypes.c_int),
                ("amplitude", ctypes.c_double), ("degree", ctypes.c_int), ("geom", ctypes.c_int),
                ("coeff", ctypes.c_int), ("which_f", ctypes.c_int), ("rtol", ctypes.c_double),
                ("inner_rtol", ctypes.c_double), ("max_outer", ctypes.c_int), ("max_inner", ctypes.c_int),
                ("x_host", ctypes.c_void_p)]


class dg_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("n_dofs", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("message", ctypes.c_char * 160)]


_lib = None
_vp = ctypes.c_void_p


def load_library(path=None):
    """Load the CUDA library (raises DGLibraryMissing if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise DGLibraryMissing("CUDA library %s is missing; run paper_1711_03590_gb300.build()" % path)
    L = ctypes.CDLL(path)
    L.dg_setup.argtypes = [ctypes.POINTER(dg_mesh), ctypes.c_int, ctypes.c_int, ctypes.POINTER(dg_opts), _vp,
                           ctypes.POINTER(_vp)]
    L.dg_n_dofs.argtypes = [_vp, ctypes.POINTER(ctypes.c_int64)]
    L.dg_info.argtypes = [_vp, ctypes.POINTER(dg_info_t)]
    L.dg_set_stream.argtypes = [_vp, _vp]
    L.dg_apply.argtypes = [_vp, _vp, _vp]
    L.dg_apply_host.argtypes = [_vp, _vp, _vp]
    L.dg_rhs.argtypes = [_vp, ctypes.c_int, _vp]
    L.dg_cg_solve.argtypes = [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                              ctypes.POINTER(ctypes.c_double)]
    L.dg_apply_dot_noalloc.argtypes = [_vp, _vp, _vp, _vp]
    L.dg_set_cells_per_block.argtypes = [_vp, ctypes.c_int]
    L.dg_set_face_mode.argtypes = [_vp, ctypes.c_int]
    L.dg_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int,
                                  ctypes.c_int, ctypes.c_int, _vp, ctypes.POINTER(_vp)]
    L.dg_batch_launch.argtypes = [_vp]
    L.dg_batch_info.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.dg_batch_destroy.argtypes = [_vp]
    L.dg_batch_last_error.argtypes = []
    L.dg_request_device_bytes.argtypes = [ctypes.POINTER(dg_request)]
    L.dg_l2_error.argtypes = [_vp, _vp, ctypes.POINTER(ctypes.c_double)]
    L.dg_server_create.argtypes = [ctypes.c_int, ctypes.c_int64, ctypes.c_int, ctypes.POINTER(_vp)]
    L.dg_server_submit.argtypes = [_vp, ctypes.POINTER(dg_request), ctypes.POINTER(ctypes.c_int64)]
    L.dg_server_set_policy.argtypes = [_vp, ctypes.c_int, ctypes.c_double]
    L.dg_server_wait.argtypes = [_vp, ctypes.c_int64, ctypes.POINTER(dg_result)]
    L.dg_server_destroy.argtypes = [_vp]
    L.dg_server_last_error.argtypes = []
    L.dg_autotune.argtypes = [_vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]
    L.dg_cg_solve_mixed.argtypes = [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                    ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                    ctypes.POINTER(ctypes.c_double)]
    L.dg_peak_probe.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.dg_cg_solve_mixed_auto.argtypes = [_vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.dg_destroy.argtypes = [_vp]
    L.dg_last_error.argtypes = [_vp]
    L.dg_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        getattr(L, name).restype = ctypes.c_char_p if name.endswith("last_error") else ctypes.c_int
    L.dg_request_device_bytes.restype = ctypes.c_int64
    _lib = L
    return L


def _check(status, handle):
    if status != DG_OK:
        msg = load_library().dg_last_error(handle)
        raise DGError(status, msg.decode() if msg else "")
    return status


def make_mesh(n, periodic=False, mapping=0, amplitude=0.1):
    if isinstance(n, int):
        n = (n, n, n)
    return dg_mesh((ctypes.c_int * 3)(*n), int(bool(periodic)), int(mapping), float(amplitude))


def make_opts(op="sipg", prec="fp64", velocity=(1.0, 0.5, 0.25), coeff=0, penalty_scale=1.0, basis="lagrange"):
    return dg_opts(OPS.get(op, op), PRECS.get(prec, prec), (ctypes.c_double * 3)(*velocity), int(coeff),
                   float(penalty_scale), BASES.get(basis, basis))


# ---- C-ABI functions with the same names ---------------------------------

def dg_setup(mesh, degree, geom, opts, stream=None):
    """Returns the opaque handle (an int).  ``stream`` is a cudaStream_t value
    (e.g. ``torch.cuda.current_stream().cuda_stream``) or None."""
    L = load_library()
    h = _vp()
    st = L.dg_setup(ctypes.byref(mesh), int(degree), GEOMS.get(geom, geom), ctypes.byref(opts),
                    _vp(stream or 0), ctypes.byref(h))
    _check(st, None)
    return h.value


def dg_n_dofs(handle):
    n = ctypes.c_int64()
    _check(load_library().dg_n_dofs(_vp(handle), ctypes.byref(n)), handle)
    return n.value


def dg_info(handle):
    info = dg_info_t()
    _check(load_library().dg_info(_vp(handle), ctypes.byref(info)), handle)
    out = {f: getattr(info, f) for f, _ in dg_info_t._fields_}
    out["tile_choices"] = [c for c in info.tile_choices if c > 0]
    return out


def dg_set_stream(handle, stream):
    _check(load_library().dg_set_stream(_vp(handle), _vp(stream or 0)), handle)


def dg_apply(handle, src_ptr, dst_ptr):
    _check(load_library().dg_apply(_vp(handle), _vp(src_ptr), _vp(dst_ptr)), handle)


def dg_apply_host(handle, src_ptr, dst_ptr):
    _check(load_library().dg_apply_host(_vp(handle), _vp(src_ptr), _vp(dst_ptr)), handle)


def dg_apply_dot_noalloc(handle, src_ptr, dst_ptr, dot_ptr):
    """dst = A src and *dot = src . dst without any device allocation (the
    partial sums live in a fixed static device array of the library)."""
    _check(load_library().dg_apply_dot_noalloc(_vp(handle), _vp(src_ptr), _vp(dst_ptr), _vp(dot_ptr)), handle)


def dg_l2_error(handle, x_ptr):
    e = ctypes.c_double(0.0)
    _check(load_library().dg_l2_error(_vp(handle), _vp(x_ptr), ctypes.byref(e)), handle)
    return e.value


def dg_rhs(handle, which_f, rhs_ptr):
    _check(load_library().dg_rhs(_vp(handle), int(which_f), _vp(rhs_ptr)), handle)


def dg_cg_solve(handle, rhs_ptr, x_ptr, rtol, max_it, raise_on_error=True):
    """Returns (status, iterations, final relative residual)."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load_library().dg_cg_solve(_vp(handle), _vp(rhs_ptr), _vp(x_ptr), float(rtol), int(max_it),
                                    ctypes.byref(it), ctypes.byref(rr))
    if raise_on_error:
        _check(st, handle)
    return st, it.value, rr.value


def dg_cg_solve_mixed(h64, h32, rhs_ptr, x_ptr, rtol, max_outer=50, inner_rtol=1e-3, max_inner=10000,
                      raise_on_error=True):
    """Returns (status, outer corrections, total FP32 iterations, final relative residual)."""
    oi = ctypes.c_int(0)
    ii = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    st = load_library().dg_cg_solve_mixed(_vp(h64), _vp(h32), _vp(rhs_ptr), _vp(x_ptr), float(rtol), int(max_outer),
                                          float(inner_rtol), int(max_inner), ctypes.byref(oi), ctypes.byref(ii),
                                          ctypes.byref(rr))
    if raise_on_error:
        _check(st, h64)
    return st, oi.value, ii.value, rr.value


def dg_cg_solve_mixed_auto(h64, hemu, h32, rhs_ptr, x_ptr, rtol, max_outer=50, inner_rtol=1e-2, max_inner=20000,
                           raise_on_error=True):
    """Returns (status, replacements, inner iterations, final relative
    residual, inner precision used: "fp64emu" or "fp32")."""
    oi, ii, kind = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(-1)
    rr = ctypes.c_double(0.0)
    st = load_library().dg_cg_solve_mixed_auto(_vp(h64), _vp(hemu), _vp(h32), _vp(rhs_ptr), _vp(x_ptr), float(rtol),
                                               int(max_outer), float(inner_rtol), int(max_inner), ctypes.byref(oi),
                                               ctypes.byref(ii), ctypes.byref(rr), ctypes.byref(kind))
    if raise_on_error:
        _check(st, h64)
    return st, oi.value, ii.value, rr.value, {DG_FP32: "fp32", DG_FP64_EMU: "fp64emu"}.get(kind.value)


def dg_set_cells_per_block(handle, cells_per_block):
    _check(load_library().dg_set_cells_per_block(_vp(handle), int(cells_per_block)), handle)


def dg_set_face_mode(handle, mode):
    _check(load_library().dg_set_face_mode(_vp(handle), int(mode)), handle)


def dg_autotune(handle):
    """Returns (cells per block chosen, ms per apply)."""
    c = ctypes.c_int(0)
    ms = ctypes.c_double(0.0)
    _check(load_library().dg_autotune(_vp(handle), ctypes.byref(c), ctypes.byref(ms)), handle)
    return c.value, ms.value


def dg_batch_create(handles, src_ptrs, dst_ptrs, autotune=True, branches=8, stream=None):
    """Capture the applies of several operators into one CUDA graph; returns
    the batch handle (an int)."""
    L = load_library()
    n = len(handles)
    H = (_vp * n)(*handles)
    S = (_vp * n)(*src_ptrs)
    D = (_vp * n)(*dst_ptrs)
    b = _vp()
    st = L.dg_batch_create(H, S, D, n, int(bool(autotune)), int(branches), _vp(stream or 0), ctypes.byref(b))
    if st != DG_OK:
        raise DGError(st, L.dg_batch_last_error().decode())
    return b.value


def dg_batch_info(batch):
    """Returns (kernel groups, kernel launches per dg_batch_launch)."""
    L = load_library()
    g, n = ctypes.c_int(0), ctypes.c_int(0)
    st = L.dg_batch_info(_vp(batch), ctypes.byref(g), ctypes.byref(n))
    if st != DG_OK:
        raise DGError(st, L.dg_batch_last_error().decode())
    return g.value, n.value


def dg_batch_launch(batch):
    L = load_library()
    st = L.dg_batch_launch(_vp(batch))
    if st != DG_OK:
        raise DGError(st, L.dg_batch_last_error().decode())


def dg_batch_destroy(batch):
    if batch:
        load_library().dg_batch_destroy(_vp(batch))


def make_request(n, degree, mapping=1, geom=None, coeff=None, rtol=1e-8, inner_rtol=1e-3, max_outer=50,
                 max_inner=20000, x_host_ptr=None, amplitude=0.1):
    """A manufactured Poisson solve request: deformed meshes use G3 geometry
    and kappa = 1 + 0.5 sin(2 pi x), Cartesian meshes kappa = 1."""
    if isinstance(n, int):
        n = (n, n, n)
    if geom is None:
        geom = "full" if mapping else "cartesian"
    if coeff is None:
        coeff = 1 if mapping else 0
    return dg_request((ctypes.c_int * 3)(*n), 0, int(mapping), float(amplitude), int(degree), GEOMS.get(geom, geom),
                      int(coeff), int(coeff), float(rtol), float(inner_rtol), int(max_outer), int(max_inner),
                      _vp(x_host_ptr or 0))


def dg_request_device_bytes(req):
    return load_library().dg_request_device_bytes(ctypes.byref(req))


def dg_server_create(budget_bytes, slots, device=0):
    L = load_library()
    s = _vp()
    st = L.dg_server_create(int(device), int(budget_bytes), int(slots), ctypes.byref(s))
    if st != DG_OK:
        raise DGError(st, L.dg_server_last_error().decode())
    return s.value


def dg_server_set_policy(server, policy, max_age_s=0.0):
    """policy 0: FIFO; 1: shortest job first with aging (max_age_s)."""
    L = load_library()
    st = L.dg_server_set_policy(_vp(server), int(policy), float(max_age_s))
    if st != DG_OK:
        raise DGError(st, L.dg_server_last_error().decode())


def dg_server_submit(server, req):
    L = load_library()
    t = ctypes.c_int64(0)
    st = L.dg_server_submit(_vp(server), ctypes.byref(req), ctypes.byref(t))
    if st != DG_OK:
        raise DGError(st, L.dg_server_last_error().decode())
    return t.value


def dg_server_wait(server, ticket):
    L = load_library()
    r = dg_result()
    st = L.dg_server_wait(_vp(server), int(ticket), ctypes.byref(r))
    if st != DG_OK:
        raise DGError(st, L.dg_server_last_error().decode())
    out = {f: getattr(r, f) for f, _ in dg_result._fields_}
    out["message"] = out["message"].decode(errors="replace")
    return out


def dg_server_destroy(server):
    if server:
        load_library().dg_server_destroy(_vp(server))


def serve_arrivals(requests, arrivals, budget_bytes, slots, policy=0, max_age_s=0.0):
    """Submit requests at the given arrival times (seconds from now, sorted)
    to a fresh server (admission policy as dg_server_set_policy) and wait for
    all; returns the result dicts in request order (latency = t_done -
    t_submit)."""
    import time
    server = dg_server_create(budget_bytes, slots)
    try:
        if policy:
            dg_server_set_policy(server, policy, max_age_s)
        tickets = []
        start = time.perf_counter()
        for req, t in zip(requests, arrivals):
            delay = start + t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets.append(dg_server_submit(server, req))
        return [dg_server_wait(server, t) for t in tickets]
    finally:
        dg_server_destroy(server)


def dg_peak_probe(kind):
    """Measured FMA throughput of the current device in TFLOP/s: kind 0
    binary64, 1 binary32 (2 flops per FMA)."""
    t = ctypes.c_double(0.0)
    _check(load_library().dg_peak_probe(int(kind), ctypes.byref(t)), None)
    return t.value


def dg_destroy(handle):
    if handle:
        load_library().dg_destroy(_vp(handle))


def dg_last_error(handle=None):
    msg = load_library().dg_last_error(_vp(handle or 0))
    return msg.decode() if msg else ""


# ---- convenience wrapper over torch tensors -------------------------------

class Operator:
    """One set-up DG operator on the current CUDA device.

    Operator(n=32, degree=4, geom="full", op="sipg", prec="fp64",
             periodic=False, mapping=1, amplitude=0.1, coeff=1)
    """

    def __init__(self, n, degree, geom="full", op="sipg", prec="fp64", periodic=False, mapping=0,
                 amplitude=0.1, coeff=0, velocity=(1.0, 0.5, 0.25), penalty_scale=1.0, stream=None,
                 basis="lagrange"):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.mesh = make_mesh(n, periodic, mapping, amplitude)
        self.opts = make_opts(op, prec, velocity, coeff, penalty_scale, basis)
        self.degree = degree
        self.dtype = torch.float32 if PRECS.get(prec, prec) == DG_FP32 else torch.float64
        self.handle = None
        self.handle = dg_setup(self.mesh, degree, geom, self.opts, stream)
        self.n_dofs = dg_n_dofs(self.handle)

    def _check_tensor(self, t, dtype=None):
        dtype = dtype or self.dtype
        if not t.is_cuda or t.dtype != dtype or not t.is_contiguous() or t.numel() != self.n_dofs:
            raise ValueError("expected a contiguous CUDA %s tensor with %d entries" % (dtype, self.n_dofs))

    def apply(self, src, dst=None):
        import torch
        self._check_tensor(src)
        if dst is None:
            dst = torch.empty_like(src)
        self._check_tensor(dst)
        dg_apply(self.handle, src.data_ptr(), dst.data_ptr())
        return dst

    def apply_host(self, src_host, dst_host):
        if src_host.is_cuda or dst_host.is_cuda:
            raise ValueError("apply_host takes CPU tensors")
        dg_apply_host(self.handle, src_host.data_ptr(), dst_host.data_ptr())
        return dst_host

    def rhs(self, which=0):
        import torch
        out = torch.empty(self.n_dofs, dtype=torch.float64, device="cuda")
        dg_rhs(self.handle, which, out.data_ptr())
        return out

    def cg(self, rhs, x=None, rtol=1e-10, max_it=5000, raise_on_error=True):
        import torch
        self._check_tensor(rhs, torch.float64)
        if x is None:
            x = torch.zeros_like(rhs)
        self._check_tensor(x, torch.float64)
        st, it, rr = dg_cg_solve(self.handle, rhs.data_ptr(), x.data_ptr(), rtol, max_it, raise_on_error)
        return x, it, rr, st

    def info(self):
        return dg_info(self.handle)

    def l2_error(self, x):
        import torch
        self._check_tensor(x, torch.float64)
        return dg_l2_error(self.handle, x.data_ptr())

    def set_cells_per_block(self, cpb):
        dg_set_cells_per_block(self.handle, cpb)

    def set_face_mode(self, mode):
        """"element" (fused kernel, default) or "loop" (two launches, the
        neighbours' traces read from memory; FP64 and emulated FP64)."""
        dg_set_face_mode(self.handle, {"element": DG_FACE_ELEMENT, "loop": DG_FACE_LOOP}.get(mode, mode))

    def autotune(self):
        return dg_autotune(self.handle)

    def close(self):
        if self.handle:
            dg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
