"""The Hermite-like basis (Sec. 3.1: face values and face-normal derivatives
from one coefficient per face point) through the C ABI against the FP64
oracle's Hermite route: every arithmetic and face mode, both operators,
Cartesian, G3, G4 and G2 storage, periodic and Dirichlet meshes; CG on the
Hermite operator.  Tolerances: 1e-12 relative (FP64, emulated FP64), 1e-5
(FP32)."""
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
CASES = [
    (dict(n=(3, 2, 4), periodic=True, mapping=1, amplitude=0.1), "full"),
    (dict(n=(2, 3, 3), periodic=False, mapping=1, amplitude=0.1), "merged"),
    (dict(n=(3, 3, 2), periodic=False, mapping=0, amplitude=0.1), "cartesian"),
    (dict(n=(2, 2, 3), periodic=False, mapping=1, amplitude=0.1), "positions"),
]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("p", [3, 4, 5, 6, 8])
@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("opname", ["sipg", "advection"])
def test_hermite_apply_matches_the_oracle(p, case, opname):
    dgp.build()
    mesh, geom = CASES[case]
    coeff = 1 if (opname == "sipg" and mesh["mapping"] == 1) else 0
    form = dict(op=opname, coeff=coeff, velocity=dg_inputs.VELOCITY)
    omesh = dict(mesh, basis="hermite", cell_jacobian="g2" if geom == "positions" else "analytic")
    u = dg_inputs.src_vector(oracle.n_dofs(mesh, p), seed=900 + p)
    ref = oracle.apply(omesh, p, form, u)
    for prec, mode in (("fp64", "element"), ("fp64", "loop"), ("fp64emu", "loop"), ("fp32", "element")):
        if geom == "positions" and mode == "element" and prec != "fp32":
            continue  # G2 runs the face loop in binary64 / double-float
        op = dgp.Operator(mesh["n"], p, geom=geom, op=opname, prec=prec, periodic=mesh["periodic"],
                          mapping=mesh["mapping"], amplitude=mesh["amplitude"], coeff=coeff, basis="hermite",
                          velocity=dg_inputs.VELOCITY)
        if prec != "fp32":
            op.set_face_mode(mode)
        got = op.apply(torch.tensor(u, dtype=op.dtype, device="cuda")).double().cpu().numpy()
        op.close()
        assert _rel(got, ref) < TOL[prec], (prec, mode, _rel(got, ref))


def test_hermite_cg_against_the_oracle():
    dgp.build()
    mesh = dict(n=(3, 4, 3), periodic=False, mapping=1, amplitude=0.1)
    p = 4
    hm = dict(mesh, basis="hermite")
    A = oracle.assemble(hm, p, dict(op="sipg", coeff=1))
    b = oracle.rhs(hm, p, 1)
    op = dgp.Operator(mesh["n"], p, geom="full", prec="fp64", mapping=1, coeff=1, basis="hermite")
    rhs = op.rhs(1)
    assert _rel(rhs.cpu().numpy(), b) < 1e-12
    # (CG needs more iterations than with the Lagrange basis: 1780 against
    # 338 with the oracle's CSR CG on this problem)
    x, it, rr, st = op.cg(rhs, rtol=1e-10, max_it=20000)
    assert st == dgp.DG_OK
    assert np.linalg.norm(b - A @ x.cpu().numpy()) <= 3e-10 * np.linalg.norm(b)
    # the discrete solution is the same function as with the Lagrange basis
    assert abs(op.l2_error(x) - oracle.l2_error(hm, p, x.cpu().numpy())) <= 1e-12 * oracle.l2_error(hm, p,
                                                                                                   x.cpu().numpy())
    op.close()


def test_hermite_needs_degree_three():
    dgp.build()
    with pytest.raises(dgp.DGError) as e:
        dgp.Operator((2, 2, 2), 2, geom="full", mapping=1, basis="hermite")
    assert e.value.status == dgp.DG_ERR_ARG


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_hermite_full_size_sampled(prec):
    """The 32^3 deformed p = 4 workload in the Hermite-like basis at full
    size (binary32 with the slim neighbour access), on the corner cells and
    a seeded sample, against the oracle's Hermite route."""
    dgp.build()
    w = dg_inputs.workload("deformed_dirichlet_32^3_p4")
    mesh, p = w["mesh"], 4
    nc, n = oracle.n_cells(mesh), oracle.n_dofs(mesh, p)
    u = dg_inputs.src_vector(n, seed=19)
    N = mesh["n"][0]
    corners = [i + N * (j + N * k) for i in (0, N - 1) for j in (0, N - 1) for k in (0, N - 1)]
    cells = dg_inputs.sample_cells(nc, 40, seed=5, must=corners)
    form = dict(op="sipg", coeff=w["coeff"])
    ref = oracle.apply(dict(mesh, basis="hermite"), p, form, u, cells=cells)
    op = dgp.Operator(mesh["n"], p, geom="full", prec=prec, mapping=1, amplitude=0.1, coeff=w["coeff"],
                      basis="hermite")
    if prec == "fp64":
        op.set_face_mode("loop")
    got = op.apply(torch.tensor(u, dtype=op.dtype, device="cuda")).double().cpu().numpy()
    op.close()
    k3 = (p + 1) ** 3
    idx = (cells[:, None] * k3 + np.arange(k3)[None, :]).ravel()
    assert _rel(got[idx], ref[idx]) < TOL[prec]
