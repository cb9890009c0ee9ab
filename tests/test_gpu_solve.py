"""Solvers through the C ABI: plain FP64 CG and mixed-precision defect
correction (FP32 CG inside, FP64 residual/update/inner products), checked
against the FP64 oracle's assembled matrix and against each other."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402


def _ops(n, p, geom="full", mapping=1, coeff=1):
    o64 = dgp.Operator(n, p, geom=geom, prec="fp64", mapping=mapping, coeff=coeff)
    o32 = dgp.Operator(n, p, geom=geom, prec="fp32", mapping=mapping, coeff=coeff)
    return o64, o32


@pytest.mark.parametrize("n,p", [((5, 4, 6), 3), ((4, 4, 4), 5)])
def test_mixed_precision_reaches_fp64_accuracy(n, p):
    dgp.build()
    mesh = dict(n=n, periodic=False, mapping=1, amplitude=0.1)
    A = oracle.assemble(mesh, p, dict(op="sipg", coeff=1))
    b = oracle.rhs(mesh, p, 1)
    o64, o32 = _ops(n, p)
    rhs = torch.tensor(b, device="cuda")
    x64, it64, rr64, st = o64.cg(rhs, rtol=1e-10, max_it=20000)
    assert st == dgp.DG_OK
    xm = torch.zeros_like(rhs)
    st, outer, inner, rrm = dgp.dg_cg_solve_mixed(o64.handle, o32.handle, rhs.data_ptr(), xm.data_ptr(), 1e-10)
    assert st == dgp.DG_OK and rrm <= 1e-10 and outer >= 2
    xs = xm.cpu().numpy()
    # residual of the mixed solution measured with the oracle's FP64 matrix
    assert np.linalg.norm(b - A @ xs) <= 3e-10 * np.linalg.norm(b)
    x64n = x64.cpu().numpy()
    assert np.linalg.norm(xs - x64n) <= 1e-7 * np.linalg.norm(x64n)
    e_m, e_64 = oracle.l2_error(mesh, p, xs), oracle.l2_error(mesh, p, x64n)
    assert abs(e_m - e_64) <= 1e-6 * e_64
    # reproducible bit for bit
    xm2 = torch.zeros_like(rhs)
    st2, outer2, inner2, _ = dgp.dg_cg_solve_mixed(o64.handle, o32.handle, rhs.data_ptr(), xm2.data_ptr(), 1e-10)
    assert (outer2, inner2) == (outer, inner) and torch.equal(xm, xm2)


def test_mixed_precision_argument_checks():
    dgp.build()
    o64, o32 = _ops((3, 3, 3), 2)
    other = dgp.Operator((3, 3, 4), 2, geom="full", prec="fp32", mapping=1, coeff=1)
    rhs = o64.rhs(1)
    x = torch.zeros_like(rhs)
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_cg_solve_mixed(o64.handle, other.handle, rhs.data_ptr(), x.data_ptr(), 1e-10)
    assert e.value.status == dgp.DG_ERR_ARG
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_cg_solve_mixed(o32.handle, o64.handle, rhs.data_ptr(), x.data_ptr(), 1e-10)
    assert e.value.status == dgp.DG_ERR_ARG
    st, outer, inner, rr = dgp.dg_cg_solve_mixed(o64.handle, o32.handle, rhs.data_ptr(), x.data_ptr(), 1e-12,
                                                 max_outer=1, raise_on_error=False)
    assert st == dgp.DG_ERR_NOT_CONVERGED and outer == 1


@pytest.mark.parametrize("p", [1, 2, 4, 6])
@pytest.mark.parametrize("tile", [0, -1])
def test_fp32_dot_epilogue_every_tile_shape(p, tile):
    """The binary32 apply's src.dst epilogue (a block reduction in FP64 in
    shared memory) for both compiled tile shapes and a cell count that leaves
    a partial last block.  Checked through the allocation-free dot entry
    point and the mixed solve on a Cartesian mesh."""
    dgp.build()
    o32 = dgp.Operator((3, 3, 7), p, geom="cartesian", prec="fp32")
    o64 = dgp.Operator((3, 3, 7), p, geom="cartesian", prec="fp64")
    cpb = o32.info()["tile_choices"][tile]
    o32.set_cells_per_block(cpb)
    assert 63 % cpb != 0
    src = torch.tensor(np.random.default_rng(p).uniform(-1, 1, o32.n_dofs), dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    dgp.dg_apply_dot_noalloc(o32.handle, src.data_ptr(), dst.data_ptr(), dot.data_ptr())
    torch.cuda.synchronize()
    want = float(torch.dot(src.double(), dst.double()))
    assert abs(float(dot.item()) - want) <= 1e-5 * float(src.double().norm() * dst.double().norm())
    rhs = o64.rhs(0)
    x = torch.zeros_like(rhs)
    st, outer, inner, rr = dgp.dg_cg_solve_mixed(o64.handle, o32.handle, rhs.data_ptr(), x.data_ptr(), 1e-8)
    assert st == dgp.DG_OK and rr <= 1e-8
    o32.close()
    o64.close()


def test_l2_error_matches_oracle():
    dgp.build()
    for mesh, p in ((dict(n=(3, 4, 2), periodic=False, mapping=1, amplitude=0.1), 3),
                    (dict(n=(4, 4, 4), periodic=False, mapping=0, amplitude=0.1), 5)):
        op = dgp.Operator(mesh["n"], p, geom="full" if mesh["mapping"] else "cartesian", mapping=mesh["mapping"],
                          coeff=mesh["mapping"])
        x = np.random.default_rng(2).uniform(-1, 1, op.n_dofs) * 0.1
        pts = oracle.dof_points(mesh, p)
        x += np.sin(np.pi * pts[:, 0]) * np.sin(np.pi * pts[:, 1]) * np.sin(np.pi * pts[:, 2])
        got = op.l2_error(torch.tensor(x, device="cuda"))
        ref = oracle.l2_error(mesh, p, x)
        assert abs(got - ref) <= 1e-12 * ref
        op.close()


def test_mixed_with_double_float_inner_against_the_oracle():
    """The inner recursion in double-float arithmetic (DG_FP64_EMU handle,
    binary64 vectors) with FP64 residual replacement: the oracle's residual
    of the solution."""
    dgp.build()
    mesh = dict(n=(4, 3, 5), periodic=False, mapping=1, amplitude=0.1)
    p = 3
    A = oracle.assemble(mesh, p, dict(op="sipg", coeff=1))
    b = oracle.rhs(mesh, p, 1)
    o64 = dgp.Operator(mesh["n"], p, geom="full", prec="fp64", mapping=1, coeff=1)
    oe = dgp.Operator(mesh["n"], p, geom="full", prec="fp64emu", mapping=1, coeff=1)
    oe.set_face_mode("loop")
    rhs = torch.tensor(b, device="cuda")
    x = torch.zeros_like(rhs)
    st, outer, inner, rr = dgp.dg_cg_solve_mixed(o64.handle, oe.handle, rhs.data_ptr(), x.data_ptr(), 1e-10)
    assert st == dgp.DG_OK and rr <= 1e-10 and outer >= 1
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 3e-10 * np.linalg.norm(b)
    o64.close()
    oe.close()


@pytest.mark.parametrize("n,mapping,expect", [((12, 12, 12), 0, "fp64emu"), ((16, 16, 16), 1, "fp32")])
def test_mixed_auto_picks_the_inner_arithmetic(n, mapping, expect):
    """Cartesian manufactured problem: FP64 CG converges in a few dozen
    iterations, so the probe keeps the double-float recursion; deformed mesh
    with variable kappa: hundreds of iterations, so binary32 takes over.
    Either way the FP64 residual meets the target and the solution matches
    plain FP64 CG."""
    dgp.build()
    p = 3
    kw = dict(geom="full" if mapping else "cartesian", mapping=mapping, coeff=mapping)
    o64 = dgp.Operator(n, p, prec="fp64", **kw)
    oe = dgp.Operator(n, p, prec="fp64emu", **kw)
    o32 = dgp.Operator(n, p, prec="fp32", **kw)
    rhs = o64.rhs(mapping)
    xr, it, rr, st = o64.cg(rhs, rtol=1e-10, max_it=20000)
    x = torch.zeros_like(rhs)
    st, outer, inner, rel, kind = dgp.dg_cg_solve_mixed_auto(o64.handle, oe.handle, o32.handle, rhs.data_ptr(),
                                                             x.data_ptr(), 1e-10)
    assert st == dgp.DG_OK and rel <= 1e-10
    assert kind == expect, (kind, it)
    assert float((x - xr).norm() / xr.norm()) <= 1e-7
    for o in (o64, oe, o32):
        o.close()


@pytest.mark.parametrize("geom,basis", [("positions", "lagrange"), ("full", "hermite")])
def test_mixed_solvers_with_g2_and_hermite(geom, basis):
    """The automatic mixed solver on G2 storage and on the Hermite-like basis
    (the three operators of the solve share geometry and basis): FP64
    residual below the target, solution equal to plain FP64 CG's."""
    dgp.build()
    n, p = (6, 5, 6), 3
    kw = dict(geom=geom, mapping=1, coeff=1, basis=basis)
    o64 = dgp.Operator(n, p, prec="fp64", **kw)
    oe = dgp.Operator(n, p, prec="fp64emu", **kw)
    o32 = dgp.Operator(n, p, prec="fp32", **kw)
    rhs = o64.rhs(1)
    xr, it, rr, st = o64.cg(rhs, rtol=1e-10, max_it=50000)
    assert st == dgp.DG_OK
    x = torch.zeros_like(rhs)
    st, outer, inner, rel, kind = dgp.dg_cg_solve_mixed_auto(o64.handle, oe.handle, o32.handle, rhs.data_ptr(),
                                                             x.data_ptr(), 1e-10)
    assert st == dgp.DG_OK and rel <= 1e-10
    assert float((x - xr).norm() / xr.norm()) <= 1e-6
    other = dgp.Operator(n, p, prec="fp32", geom=geom, mapping=1, coeff=1,
                         basis="hermite" if basis == "lagrange" else "lagrange")
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_cg_solve_mixed(o64.handle, other.handle, rhs.data_ptr(), x.data_ptr(), 1e-10)
    assert e.value.status == dgp.DG_ERR_ARG
    for o in (o64, oe, o32, other):
        o.close()
