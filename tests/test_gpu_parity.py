"""Parity of the CUDA apply (through the C ABI) with the FP64 oracle.

Tolerances (norm-wise relative, |y_gpu - y_ref|_2 / |y_ref|_2): 1e-12 for
FP64 arithmetic, 1e-5 for FP32 arithmetic.  Small meshes compare every
entry with the oracle's cell-by-cell route; the 32^3 deformed workload
compares sampled cells (boundary corners and a seeded sample) at full size,
in the launch configurations the benchmark times (FP64 and emulated FP64 in
both face modes, FP32).
"""
import numpy as np
import pytest

import dg_inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402

TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp64emu": 1e-12, "fp64-loop": 1e-12, "fp64emu-loop": 1e-12}


@pytest.fixture(scope="module", autouse=True)
def _built():
    dgp.build()
    dgp.load_library()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _gpu_apply(mesh, p, geom, form, prec, u):
    """The GPU apply; prec "<p>-loop" is the operator of arithmetic <p> in
    face-loop mode."""
    loop = prec.endswith("-loop")
    prec = prec[:-len("-loop")] if loop else prec
    op = dgp.Operator(mesh["n"], p, geom=geom, op=form.get("op", "sipg"), prec=prec,
                      periodic=mesh.get("periodic", False), mapping=mesh.get("mapping", 0),
                      amplitude=mesh.get("amplitude", 0.1), coeff=form.get("coeff", 0),
                      velocity=form.get("velocity", dg_inputs.VELOCITY),
                      penalty_scale=form.get("penalty_scale", 1.0))
    if loop:
        op.set_face_mode("loop")
    src = torch.tensor(u, dtype=op.dtype, device="cuda")
    dst = op.apply(src)
    torch.cuda.synchronize()
    out = dst.double().cpu().numpy()
    op.close()
    return out


DEF = dict(mapping=1, amplitude=0.1)
# meshes span several blocks with a ragged last block for every degree
SMALL = [
    (dict(n=(4, 4, 4), periodic=True), "cartesian"),
    (dict(n=(1, 1, 1), periodic=True, **DEF), "full"),
    (dict(n=(2, 2, 2), periodic=True, **DEF), "full"),
    (dict(n=(3, 4, 5), periodic=False, **DEF), "full"),
    (dict(n=(5, 3, 2), periodic=False), "cartesian"),
    (dict(n=(3, 2, 4), periodic=True, **DEF), "merged"),
    (dict(n=(4, 3, 3), periodic=False, **DEF), "merged"),
]


def test_config1_cartesian_periodic_p2_vs_assembled():
    """1728-dof workload: GPU apply equals the oracle's assembled sparse
    matrix times the seeded vector (route R1)."""
    w = dg_inputs.workload("cartesian_periodic_4x4x4_p2")
    mesh, p = w["mesh"], w["degree"]
    form = dict(op="sipg", coeff=0)
    A = oracle.assemble(mesh, p, form)
    u = dg_inputs.src_vector(A.shape[0], seed=1)
    ref = A @ u
    for geom in ("cartesian", "full", "merged"):
        got = _gpu_apply(mesh, p, geom, form, "fp64", u)
        assert _rel(got, ref) < TOL["fp64"], geom
        gote = _gpu_apply(mesh, p, geom, form, "fp64emu", u)
        assert _rel(gote, ref) < TOL["fp64emu"], geom
        got32 = _gpu_apply(mesh, p, geom, form, "fp32", u)
        assert _rel(got32, ref) < TOL["fp32"], geom


@pytest.mark.parametrize("p", range(1, 9))
@pytest.mark.parametrize("case", range(len(SMALL)))
@pytest.mark.parametrize("op", ["sipg", "advection"])
def test_small_meshes_all_degrees(p, case, op):
    mesh, geom = SMALL[case]
    n = oracle.n_dofs(mesh, p)
    if n * (p + 1) ** 3 > 6e7:
        mesh = dict(mesh, n=tuple(min(v, 3) for v in mesh["n"]))
        n = oracle.n_dofs(mesh, p)
    form = dict(op=op, coeff=1 if (op == "sipg" and case % 2 == 1) else 0, velocity=dg_inputs.VELOCITY)
    u = dg_inputs.src_vector(n, seed=100 + p)
    ref = oracle.apply(mesh, p, form, u)
    for prec in ("fp64", "fp32", "fp64emu", "fp64-loop", "fp64emu-loop"):
        got = _gpu_apply(mesh, p, geom, form, prec, u)
        assert _rel(got, ref) < TOL[prec], (prec, _rel(got, ref))


@pytest.mark.parametrize("p", [1, 2, 4, 8])
@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp64emu", "fp64-loop", "fp64emu-loop"])
def test_full_size_deformed_sampled(p, prec):
    """32^3 deformed mesh, full per-point Jacobians, kappa variable,
    Dirichlet: full-size GPU apply, compared on sampled cells (all eight
    corner cells plus a seeded sample) with the oracle's cell-wise route."""
    w = dg_inputs.workload("deformed_dirichlet_32^3_p%d" % p)
    mesh = w["mesh"]
    nc = oracle.n_cells(mesh)
    n = oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=7)
    N = mesh["n"][0]
    corners = [i + N * (j + N * k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]
    cells = dg_inputs.sample_cells(nc, 24 if p >= 6 else 56, seed=p, must=corners)
    for op in ("sipg", "advection"):
        form = dict(op=op, coeff=w["coeff"] if op == "sipg" else 0, velocity=dg_inputs.VELOCITY)
        ref = oracle.apply(mesh, p, form, u, cells=cells)
        got = _gpu_apply(mesh, p, "full", form, prec, u)
        k3 = (p + 1) ** 3
        idx = (cells[:, None] * k3 + np.arange(k3)[None, :]).ravel()
        assert _rel(got[idx], ref[idx]) < TOL[prec], (op, _rel(got[idx], ref[idx]))
        assert np.all(np.isfinite(got))


@pytest.mark.parametrize("geom", ["full", "merged"])
def test_constants_in_kernel_periodic_deformed(geom):
    """A 1 = 0 for SIPG with periodic boundaries on the deformed mesh."""
    op = dgp.Operator((5, 3, 4), 3, geom=geom, periodic=True, mapping=1, coeff=1)
    one = torch.ones(op.n_dofs, dtype=torch.float64, device="cuda")
    y = op.apply(one)
    scale = op.apply(torch.tensor(dg_inputs.src_vector(op.n_dofs), device="cuda")).abs().max()
    assert float(y.abs().max()) < 1e-12 * float(scale)


def test_symmetry_on_gpu():
    """u^T A v = v^T A u from two GPU applies (deformed, Dirichlet, kappa)."""
    op = dgp.Operator((6, 5, 4), 4, geom="full", mapping=1, coeff=1)
    u = torch.tensor(dg_inputs.src_vector(op.n_dofs, 1), device="cuda")
    v = torch.tensor(dg_inputs.src_vector(op.n_dofs, 2), device="cuda")
    a = float(torch.dot(u, op.apply(v)))
    b = float(torch.dot(v, op.apply(u)))
    assert abs(a - b) < 1e-12 * abs(a)


def test_apply_is_deterministic_and_host_path_matches():
    op = dgp.Operator(8, 3, geom="full", mapping=1, coeff=1)
    u = torch.tensor(dg_inputs.src_vector(op.n_dofs, 3), device="cuda")
    y1 = op.apply(u)
    y2 = op.apply(u)
    assert torch.equal(y1, y2)
    hu = u.cpu().pin_memory()
    hy = torch.empty_like(hu).pin_memory()
    op.apply_host(hu, hy)
    assert torch.equal(hy, y1.cpu())


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp64emu"])
@pytest.mark.parametrize("mesh,geom,op_name", [
    (dict(n=(8, 8, 9), periodic=False, mapping=1), "full", "sipg"),    # 4 slabs of z-planes
    (dict(n=(16, 4, 6), periodic=False, mapping=0), "cartesian", "advection"),  # 3 slabs
    (dict(n=(8, 8, 8), periodic=True, mapping=1), "full", "sipg"),     # periodic: one slab
    (dict(n=(5, 5, 8), periodic=False, mapping=1), "merged", "sipg"),  # planes of 25 cells: one slab
])
def test_pipelined_host_apply_matches_device_apply(prec, mesh, geom, op_name):
    """dg_apply_host overlaps copies and applies over slabs of z-planes; every
    slab boundary must give the same bits as one device apply."""
    op = dgp.Operator(mesh["n"], 3, geom=geom, op=op_name, prec=prec, periodic=mesh["periodic"],
                      mapping=mesh["mapping"], amplitude=0.1, coeff=1 if op_name == "sipg" else 0)
    u = torch.tensor(dg_inputs.src_vector(op.n_dofs, 7), dtype=op.dtype, device="cuda")
    y = op.apply(u).cpu()
    hu = u.cpu().pin_memory()
    hy = torch.full_like(hu, float("nan")).pin_memory()
    for _ in range(2):
        op.apply_host(hu, hy)
        assert torch.equal(hy, y), (prec, mesh, geom)
    op.close()


def test_rhs_matches_oracle():
    for mesh, geom, which in ((dict(n=(3, 4, 2), mapping=1, amplitude=0.1), "full", 1),
                              (dict(n=(4, 4, 4)), "cartesian", 0)):
        p = 3
        op = dgp.Operator(mesh["n"], p, geom=geom, mapping=mesh.get("mapping", 0), coeff=which)
        got = op.rhs(which).cpu().numpy()
        ref = oracle.rhs(mesh, p, which)
        assert _rel(got, ref) < 1e-12


def test_cg_solution_matches_oracle():
    """Dirichlet SIPG on the deformed mesh: the GPU CG solution agrees with
    the oracle's CG solution, and its oracle residual is small."""
    mesh = dict(n=(4, 4, 4), periodic=False, mapping=1, amplitude=0.1)
    p = 2
    A = oracle.assemble(mesh, p, dict(op="sipg", coeff=1))
    b = oracle.rhs(mesh, p, 1)
    x_ref, it_ref, _ = oracle.cg(A, b, rtol=1e-12)
    op = dgp.Operator(mesh["n"], p, geom="full", mapping=1, coeff=1)
    rhs = torch.tensor(b, device="cuda")
    x, it, rr, st = op.cg(rhs, rtol=1e-12, max_it=5000)
    xs = x.cpu().numpy()
    assert st == dgp.DG_OK and rr <= 1e-12
    assert np.linalg.norm(b - A @ xs) <= 2e-12 * np.linalg.norm(b)
    assert _rel(xs, x_ref) < 1e-9
    assert abs(oracle.l2_error(mesh, p, xs) - oracle.l2_error(mesh, p, x_ref)) < 1e-10
    # bitwise reproducible
    x2, it2, rr2, _ = op.cg(rhs, rtol=1e-12, max_it=5000)
    assert it2 == it and torch.equal(x2, x)


def test_error_paths():
    op = dgp.Operator(3, 2, geom="full", mapping=1)
    u = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_apply(op.handle, u.data_ptr(), u.data_ptr())
    assert e.value.status == dgp.DG_ERR_ARG
    b = op.rhs(0)
    x, it, rr, st = op.cg(b, rtol=1e-14, max_it=2, raise_on_error=False)
    assert st == dgp.DG_ERR_NOT_CONVERGED and it == 2
    adv = dgp.Operator(3, 2, geom="full", op="advection", mapping=1)
    with pytest.raises(dgp.DGError) as e:
        adv.cg(b)
    assert e.value.status == dgp.DG_ERR_UNSUPPORTED
    with pytest.raises(dgp.DGError) as e:
        dgp.Operator(2, 2, geom="full", mapping=1, amplitude=0.9)  # det J < 0 somewhere
    assert e.value.status == dgp.DG_ERR_ARG


@pytest.mark.parametrize("p", [1, 4, 8])
def test_tile_shape_does_not_change_results(p):
    """Cells per block is a launch parameter only: every value gives the same
    bits; the autotuner keeps one of them."""
    for prec in ("fp64", "fp32", "fp64emu"):
        op = dgp.Operator((5, 4, 3), p, geom="full", prec=prec, mapping=1, coeff=1)
        u = torch.tensor(dg_inputs.src_vector(op.n_dofs, 5), dtype=op.dtype, device="cuda")
        ref = op.apply(u).clone()
        choices = op.info()["tile_choices"]
        assert choices == sorted(choices) and op.info()["cells_per_block"] in choices
        cmax = choices[-1]
        for c in sorted({choices[0], choices[min(1, len(choices) - 1)], choices[len(choices) // 2], cmax}):
            op.set_cells_per_block(c)
            assert op.info()["cells_per_block"] == c
            assert op.info()["threads_per_block"] == c * (p + 1) ** 2
            assert torch.equal(op.apply(u), ref), (prec, c)
        c, ms = op.autotune()
        assert c in choices and ms > 0
        assert torch.equal(op.apply(u), ref)
        with pytest.raises(dgp.DGError):
            op.set_cells_per_block(cmax + 1)
        op.close()


def test_emulated_fp64_range_and_special_values():
    """Double-float loads: zeros, tiny and large magnitudes and mixed signs
    in the input vector keep the FP64 tolerance against the FP64 apply."""
    for scale in (1e-20, 1.0, 1e20):
        op = dgp.Operator((3, 3, 3), 3, geom="full", prec="fp64emu", mapping=1, coeff=1)
        o64 = dgp.Operator((3, 3, 3), 3, geom="full", prec="fp64", mapping=1, coeff=1)
        u = dg_inputs.src_vector(op.n_dofs, 9) * scale
        u[::7] = 0.0
        src = torch.tensor(u, device="cuda")
        ye, y64 = op.apply(src), o64.apply(src)
        rel = float((ye - y64).norm() / y64.norm())
        assert rel < 1e-12, (scale, rel)
        op.close()
        o64.close()


def test_emulated_fp64_cg_matches_fp64_cg():
    mesh = dict(n=(4, 4, 4), periodic=False, mapping=1, amplitude=0.1)
    p = 3
    b = oracle.rhs(mesh, p, 1)
    A = oracle.assemble(mesh, p, dict(op="sipg", coeff=1))
    rhs = torch.tensor(b, device="cuda")
    oe = dgp.Operator(mesh["n"], p, geom="full", prec="fp64emu", mapping=1, coeff=1)
    xe, ite, rre, st = oe.cg(rhs, rtol=1e-11, max_it=20000)
    assert st == dgp.DG_OK
    assert np.linalg.norm(b - A @ xe.cpu().numpy()) <= 3e-11 * np.linalg.norm(b)


def _componentwise(got, ref, A, u):
    """max_i |y_gpu - y_ref|_i / (|A| |u|)_i: the error of each entry against
    the magnitude of the terms summed into it (cancellation-aware)."""
    scale = abs(A) @ np.abs(u)
    return float(np.max(np.abs(got - ref) / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("p", [1, 3, 5, 8])
@pytest.mark.parametrize("case", [1, 3, 6])
@pytest.mark.parametrize("op", ["sipg", "advection"])
def test_componentwise_error_against_abs_a_abs_u(p, case, op):
    """The componentwise diagnostic: every entry of the GPU apply within the
    stated tolerance of (|A| |u|)_i, A the oracle's assembled matrix."""
    mesh, geom = SMALL[case]
    if oracle.n_cells(mesh) * (p + 1) ** 6 > 3e7:
        mesh = dict(mesh, n=tuple(min(v, 2) for v in mesh["n"]))
    form = dict(op=op, coeff=1 if op == "sipg" else 0, velocity=dg_inputs.VELOCITY)
    A = oracle.assemble(mesh, p, form)
    u = dg_inputs.src_vector(A.shape[0], seed=300 + p)
    ref = A @ u
    for prec in ("fp64", "fp32", "fp64emu", "fp64-loop", "fp64emu-loop"):
        got = _gpu_apply(mesh, p, geom, form, prec, u)
        cw = _componentwise(got, ref, A, u)
        assert cw < TOL[prec], (prec, cw)
