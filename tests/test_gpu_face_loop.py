"""The face-loop variant of the FP64 and emulated-FP64 applies
(dg_set_face_mode): two launches, the neighbours' traces read instead of
recomputed.  It must give the fused kernel's
results up to rounding on every geometry, operator, degree and boundary
treatment, match the oracle, and serve the solvers."""
import numpy as np
import pytest
import torch

import dg_inputs
import oracle
import paper_1711_03590_gb300 as dgp

pytestmark = pytest.mark.gpu

DEF = dict(mapping=1, amplitude=0.1)
MESHES = [
    (dict(n=(3, 4, 5), periodic=False, **DEF), "full"),
    (dict(n=(2, 3, 2), periodic=True, **DEF), "full"),
    (dict(n=(4, 3, 3), periodic=False, **DEF), "merged"),
    (dict(n=(5, 3, 2), periodic=False, mapping=0), "cartesian"),
    (dict(n=(3, 3, 3), periodic=True, mapping=0), "cartesian"),
    (dict(n=(1, 1, 1), periodic=True, **DEF), "full"),
]


def _op(mesh, p, geom, op_name, mode, prec="fp64"):
    o = dgp.Operator(mesh["n"], p, geom=geom, op=op_name, prec=prec, periodic=mesh["periodic"],
                     mapping=mesh["mapping"], amplitude=mesh.get("amplitude", 0.0),
                     coeff=1 if op_name == "sipg" else 0)
    o.set_face_mode(mode)
    assert o.info()["face_mode"] == (dgp.DG_FACE_LOOP if mode == "loop" else dgp.DG_FACE_ELEMENT)
    return o


@pytest.mark.parametrize("p", [1, 2, 4, 5, 8])
@pytest.mark.parametrize("case", range(len(MESHES)))
@pytest.mark.parametrize("op_name", ["sipg", "advection"])
@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
def test_face_loop_equals_fused_kernel(p, case, op_name, prec):
    mesh, geom = MESHES[case]
    fused = _op(mesh, p, geom, op_name, "element", prec)
    loop = _op(mesh, p, geom, op_name, "loop", prec)
    u = torch.tensor(dg_inputs.src_vector(fused.n_dofs, 11 + p), device="cuda")
    a = fused.apply(u)
    b = loop.apply(u)
    rel = float((a - b).norm() / a.norm())
    # binary64: rounding of two operation orders; double-float (48-bit
    # significands): both within 1e-12 of the exact result
    assert rel < (1e-13 if prec == "fp64" else 1e-12), (p, case, op_name, rel)
    assert torch.equal(loop.apply(u), b)  # deterministic
    fused.close()
    loop.close()


@pytest.mark.parametrize("op_name", ["sipg", "advection"])
@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
def test_face_loop_matches_oracle(op_name, prec):
    mesh = dict(n=(3, 2, 4), periodic=False, mapping=1, amplitude=0.1)
    p = 3
    o = _op(mesh, p, "full", op_name, "loop", prec)
    u = dg_inputs.src_vector(o.n_dofs, 5)
    form = dict(op=op_name, coeff=1) if op_name == "sipg" else dict(op=op_name, coeff=0, velocity=dg_inputs.VELOCITY)
    ref = oracle.apply(mesh, p, form, u)
    got = o.apply(torch.tensor(u, device="cuda")).cpu().numpy()
    assert np.linalg.norm(got - ref) < 1e-12 * np.linalg.norm(ref)
    o.close()


def test_face_loop_in_solvers_and_errors():
    mesh = dict(n=(6, 6, 6), periodic=False, mapping=1, amplitude=0.1)
    o = _op(mesh, 3, "full", "sipg", "loop")
    ref = _op(mesh, 3, "full", "sipg", "element")
    b = o.rhs(1)
    x1, it1, rr1, _ = o.cg(b, torch.zeros_like(b), rtol=1e-10, max_it=5000)
    x2, it2, rr2, _ = ref.cg(b, torch.zeros_like(b), rtol=1e-10, max_it=5000)
    assert rr1 <= 1e-10 and abs(it1 - it2) <= 2
    assert float((x1 - x2).norm() / x2.norm()) < 1e-9
    # src.dst partial of the last kernel: the allocation-free dot entry point
    u = torch.tensor(dg_inputs.src_vector(o.n_dofs, 3), device="cuda")
    y = torch.empty_like(u)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    dgp.dg_apply_dot_noalloc(o.handle, u.data_ptr(), y.data_ptr(), dot.data_ptr())
    torch.cuda.synchronize()
    assert abs(float(dot.item()) - float(torch.dot(u, y))) <= 1e-12 * float(u.norm() * y.norm())
    # host buffers (6 z-planes of 36 cells: one slab)
    hu = u.cpu().pin_memory()
    hy = torch.empty_like(hu).pin_memory()
    o.apply_host(hu, hy)
    assert torch.equal(hy, y.cpu())
    o.close()
    ref.close()
    op = dgp.Operator((2, 2, 2), 2, prec="fp32")
    with pytest.raises(dgp.DGError) as e:
        op.set_face_mode("loop")
    assert e.value.status == dgp.DG_ERR_UNSUPPORTED
    op.close()
    with pytest.raises(dgp.DGError):
        dgp.Operator((2, 2, 2), 2).set_face_mode(7)


@pytest.mark.parametrize("p", [2, 4, 7])
@pytest.mark.parametrize("op_name", ["sipg", "advection"])
@pytest.mark.parametrize("prec", ["fp64", "fp64emu"])
def test_face_loop_pipelined_host_apply(p, op_name, prec):
    """Host buffers on a mesh that the host apply splits into slabs of
    z-planes: each slab's backward launch follows the next slab's forward
    launch; the result is bitwise the device apply's."""
    mesh = dict(n=(8, 8, 9), periodic=False, mapping=1, amplitude=0.1)
    o = _op(mesh, p, "full", op_name, "loop", prec)
    u = torch.tensor(dg_inputs.src_vector(o.n_dofs, 21), device="cuda")
    y = o.apply(u)
    hu = u.cpu().pin_memory()
    hy = torch.full_like(hu, float("nan")).pin_memory()
    o.apply_host(hu, hy)
    assert torch.equal(hy, y.cpu())
    o.close()


def test_emulated_face_loop_cg():
    """CG with the emulated-FP64 face loop reaches the FP64 solution."""
    mesh = dict(n=(6, 6, 6), periodic=False, mapping=1, amplitude=0.1)
    o = _op(mesh, 3, "full", "sipg", "loop", "fp64emu")
    ref = _op(mesh, 3, "full", "sipg", "loop")
    b = ref.rhs(1)
    x1, it1, rr1, _ = o.cg(b, torch.zeros_like(b), rtol=1e-9, max_it=5000)
    x2, it2, rr2, _ = ref.cg(b, torch.zeros_like(b), rtol=1e-9, max_it=5000)
    assert rr1 <= 1e-9 and abs(it1 - it2) <= 3
    assert float((x1 - x2).norm() / x2.norm()) < 1e-8
    o.close()
    ref.close()


def test_face_mode_tile_defaults():
    """Selecting a face mode moves an unchanged default tile shape to that
    mode's default and back; an explicitly chosen one stays."""
    for prec in ("fp64", "fp64emu"):
        o = dgp.Operator((4, 4, 4), 1, prec=prec)  # k = 2: the two defaults differ
        elem = o.info()["cells_per_block"]
        o.set_face_mode("loop")
        loop = o.info()["cells_per_block"]
        assert loop != elem and loop in o.info()["tile_choices"]
        o.set_face_mode("element")
        assert o.info()["cells_per_block"] == elem
        o.set_cells_per_block(3)
        o.set_face_mode("loop")
        assert o.info()["cells_per_block"] == 3
        o.set_cells_per_block(0)  # the mode's default
        assert o.info()["cells_per_block"] == loop
        o.close()
