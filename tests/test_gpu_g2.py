"""Geometry variant G2 (Sec. 5: quadrature-point positions stored, the
Jacobian computed in the kernel by a collocation derivative) and the sheared
(affine) mapping, through the C ABI against the FP64 oracle.

The G2 operator differs from the analytic-J operator on curved meshes (its
Jacobian is the derivative of the degree-p interpolant of the map through the
Gauss points), so the reference is the oracle's own G2 route; on linear maps
the two coincide, which the oracle pins check.  Tolerances as everywhere:
1e-12 relative for FP64 and emulated FP64, 1e-5 for FP32."""
import numpy as np
import pytest

import dg_inputs
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402

TOL = {"fp64": 1e-12, "fp64emu": 1e-12, "fp32": 1e-5}
MESHES = [
    dict(n=(3, 4, 2), periodic=False, mapping=1, amplitude=0.1),
    dict(n=(2, 3, 3), periodic=True, mapping=1, amplitude=0.1),
    dict(n=(3, 2, 4), periodic=False, mapping=2, amplitude=0.1),
    dict(n=(2, 2, 3), periodic=True, mapping=2, amplitude=0.1),
]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _gpu(mesh, p, geom, form, prec, u):
    op = dgp.Operator(mesh["n"], p, geom=geom, op=form["op"], prec=prec, periodic=mesh["periodic"],
                      mapping=mesh["mapping"], amplitude=mesh["amplitude"], coeff=form["coeff"],
                      velocity=dg_inputs.VELOCITY)
    src = torch.tensor(u, dtype=op.dtype, device="cuda")
    out = op.apply(src).double().cpu().numpy()
    info = op.info()
    op.close()
    return out, info


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 8])
@pytest.mark.parametrize("case", range(len(MESHES)))
@pytest.mark.parametrize("opname", ["sipg", "advection"])
def test_g2_apply_matches_the_oracle_g2_route(p, case, opname):
    mesh = MESHES[case]
    coeff = 1 if (opname == "sipg" and not (mesh["periodic"] and mesh["mapping"] == 2)) else 0
    form = dict(op=opname, coeff=coeff, velocity=dg_inputs.VELOCITY)
    n = oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=700 + p)
    ref = oracle.apply(dict(mesh, cell_jacobian="g2"), p, form, u)
    for prec in ("fp64", "fp64emu", "fp32"):
        got, info = _gpu(mesh, p, "positions", form, prec, u)
        assert _rel(got, ref) < TOL[prec], (prec, _rel(got, ref))
        if prec != "fp32":
            assert info["face_mode"] == dgp.DG_FACE_LOOP


@pytest.mark.parametrize("p", [1, 3, 5])
def test_sheared_mapping_with_stored_jacobians(p):
    """The affine shear through the G3 and G4 storage against the oracle's
    analytic route (the GPU set-up evaluates the mapping on its own)."""
    mesh = MESHES[2]
    form = dict(op="sipg", coeff=1)
    n = oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=710 + p)
    ref = oracle.apply(mesh, p, form, u)
    for geom in ("full", "merged"):
        for prec in ("fp64", "fp32"):
            got, _ = _gpu(mesh, p, geom, form, prec, u)
            assert _rel(got, ref) < TOL[prec], (geom, prec, _rel(got, ref))


def test_g2_cg_solution_against_the_oracle():
    """CG on the G2 operator (face loop) solves the oracle's G2 system."""
    dgp.build()
    mesh = dict(n=(3, 3, 4), periodic=False, mapping=1, amplitude=0.1)
    p = 3
    A = oracle.assemble(dict(mesh, cell_jacobian="g2"), p, dict(op="sipg", coeff=1))
    b = oracle.rhs(mesh, p, 1)
    op = dgp.Operator(mesh["n"], p, geom="positions", prec="fp64", mapping=1, coeff=1)
    x, it, rr, st = op.cg(torch.tensor(b, device="cuda"), rtol=1e-10, max_it=5000)
    assert st == dgp.DG_OK
    xs = x.cpu().numpy()
    assert np.linalg.norm(b - A @ xs) <= 3e-10 * np.linalg.norm(b)
    op.close()


def test_g2_argument_rules():
    dgp.build()
    op = dgp.Operator((2, 2, 2), 2, geom="positions", prec="fp64", mapping=1)
    with pytest.raises(dgp.DGError) as e:
        op.set_face_mode("element")
    assert e.value.status == dgp.DG_ERR_UNSUPPORTED
    op.close()
    with pytest.raises(dgp.DGError) as e:
        dgp.Operator((2, 2, 2), 2, geom="full", prec="fp64", periodic=True, mapping=2, coeff=1)
    assert e.value.status == dgp.DG_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_g2_full_size_sampled(prec):
    """The 32^3 deformed p = 4 workload with G2 storage at full size (the
    bench's launch configuration), compared on the corner cells and a seeded
    sample with the oracle's G2 route."""
    dgp.build()
    w = dg_inputs.workload("deformed_dirichlet_32^3_p4")
    mesh, p = w["mesh"], 4
    nc, n = oracle.n_cells(mesh), oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=17)
    N = mesh["n"][0]
    corners = [i + N * (j + N * k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]
    cells = dg_inputs.sample_cells(nc, 40, seed=4, must=corners)
    form = dict(op="sipg", coeff=w["coeff"])
    ref = oracle.apply(dict(mesh, cell_jacobian="g2"), p, form, u, cells=cells)
    op = dgp.Operator(mesh["n"], p, geom="positions", prec=prec, mapping=1, amplitude=0.1, coeff=w["coeff"])
    got = op.apply(torch.tensor(u, dtype=op.dtype, device="cuda")).double().cpu().numpy()
    op.close()
    k3 = (p + 1) ** 3
    idx = (cells[:, None] * k3 + np.arange(k3)[None, :]).ravel()
    assert _rel(got[idx], ref[idx]) < TOL[prec]
    assert np.all(np.isfinite(got))
