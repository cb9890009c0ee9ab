"""Batched evaluation: one CUDA graph launch applying operators of different
meshes, degrees, geometries and precisions gives exactly the bits of the
individual applies (each apply's arithmetic does not depend on the batch)."""
import pytest

import dg_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402

CASES = [
    dict(n=(6, 6, 6), p=1, geom="cartesian", prec="fp64", periodic=True, mapping=0, coeff=0, op="sipg"),
    dict(n=(5, 4, 3), p=3, geom="full", prec="fp32", periodic=False, mapping=1, coeff=1, op="sipg"),
    dict(n=(3, 3, 3), p=7, geom="full", prec="fp64emu", periodic=False, mapping=1, coeff=1, op="sipg"),
    dict(n=(4, 4, 4), p=2, geom="merged", prec="fp64", periodic=True, mapping=1, coeff=0, op="advection"),
    dict(n=(4, 4, 4), p=5, geom="full", prec="fp32", periodic=True, mapping=1, coeff=1, op="sipg"),
    dict(n=(6, 6, 6), p=4, geom="full", prec="fp64", periodic=False, mapping=1, coeff=1, op="sipg"),
    # face-loop operators (two launches each, work arrays per handle)
    dict(n=(5, 6, 4), p=3, geom="full", prec="fp64", periodic=False, mapping=1, coeff=1, op="sipg", face="loop"),
    dict(n=(4, 4, 4), p=5, geom="merged", prec="fp64emu", periodic=True, mapping=1, coeff=0, op="advection",
         face="loop"),
    # G2 (positions; binary64 runs the face loop), the sheared mapping, the Hermite-like basis
    dict(n=(4, 3, 5), p=3, geom="positions", prec="fp64", periodic=False, mapping=1, coeff=1, op="sipg"),
    dict(n=(3, 3, 3), p=4, geom="positions", prec="fp32", periodic=True, mapping=1, coeff=1, op="sipg"),
    dict(n=(3, 4, 3), p=5, geom="full", prec="fp64", periodic=False, mapping=2, coeff=1, op="sipg", basis="hermite"),
    dict(n=(3, 3, 4), p=3, geom="merged", prec="fp32", periodic=False, mapping=1, coeff=0, op="advection",
         basis="hermite"),
]


@pytest.mark.parametrize("branches,autotune", [(1, False), (3, True)])
def test_batch_equals_individual_applies(branches, autotune):
    dgp.build()
    ops, srcs, dsts, refs = [], [], [], []
    for i, c in enumerate(CASES):
        op = dgp.Operator(c["n"], c["p"], geom=c["geom"], op=c["op"], prec=c["prec"], periodic=c["periodic"],
                          mapping=c["mapping"], coeff=c["coeff"], basis=c.get("basis", "lagrange"))
        if c.get("face"):
            op.set_face_mode(c["face"])
        src = torch.tensor(dg_inputs.src_vector(op.n_dofs, 40 + i), dtype=op.dtype, device="cuda")
        refs.append(op.apply(src).clone())
        ops.append(op)
        srcs.append(src)
        dsts.append(torch.zeros_like(src))
    b = dgp.dg_batch_create([o.handle for o in ops], [s.data_ptr() for s in srcs], [d.data_ptr() for d in dsts],
                            autotune=autotune, branches=branches)
    for _ in range(2):
        for d in dsts:
            d.zero_()
        dgp.dg_batch_launch(b)
        torch.cuda.synchronize()
        for d, r in zip(dsts, refs):
            assert torch.equal(d, r)
    dgp.dg_batch_destroy(b)
    for o in ops:
        o.close()


def test_batch_argument_errors():
    dgp.build()
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_batch_create([], [], [])
    assert e.value.status == dgp.DG_ERR_ARG
    op = dgp.Operator(3, 2, geom="full", mapping=1)
    u = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    with pytest.raises(dgp.DGError) as e:  # src == dst is refused by the first plain apply
        dgp.dg_batch_create([op.handle], [u.data_ptr()], [u.data_ptr()])
    assert e.value.status == dgp.DG_ERR_ARG
    op.close()


def test_batch_against_the_oracle():
    """A batched mix of degrees, meshes, geometries and arithmetics (several
    operators per fused launch, and one kernel group of 70 operators, more
    than one launch holds) against the FP64 oracle's cell-wise route,
    element by element: 1e-12 for FP64 and emulated FP64, 1e-5 for FP32."""
    import numpy as np
    import oracle
    dgp.build()
    tol = {"fp64": 1e-12, "fp64emu": 1e-12, "fp32": 1e-5}
    cases = []
    for i, (n, p) in enumerate([((3, 2, 4), 1), ((2, 3, 3), 2), ((4, 3, 2), 3), ((3, 3, 2), 4), ((2, 2, 3), 5)]):
        for prec, face in (("fp64", None), ("fp64", "loop"), ("fp32", None), ("fp64emu", "loop")):
            cases.append(dict(n=n, p=p, prec=prec, face=face, periodic=(i % 2 == 1), mapping=1, geom="full",
                              coeff=1, op="sipg" if (i + len(cases)) % 3 else "advection"))
    # one kernel group larger than a fused launch holds (64 operators)
    for j in range(70):
        cases.append(dict(n=(1 + j % 3, 2, 1 + j % 2), p=1, prec="fp32", face=None, periodic=False, mapping=1,
                          geom="full", coeff=1, op="sipg"))
    ops, srcs, dsts, refs = [], [], [], []
    for i, c in enumerate(cases):
        mesh = dict(n=c["n"], periodic=c["periodic"], mapping=c["mapping"], amplitude=0.1)
        form = dict(op=c["op"], coeff=c["coeff"] if c["op"] == "sipg" else 0, velocity=dg_inputs.VELOCITY)
        op = dgp.Operator(c["n"], c["p"], geom=c["geom"], op=c["op"], prec=c["prec"], periodic=c["periodic"],
                          mapping=c["mapping"], coeff=form["coeff"])
        if c["face"]:
            op.set_face_mode(c["face"])
        u = dg_inputs.src_vector(op.n_dofs, 500 + i)
        refs.append(oracle.apply(mesh, c["p"], form, u))
        srcs.append(torch.tensor(u, dtype=op.dtype, device="cuda"))
        dsts.append(torch.full_like(srcs[-1], float("nan")))
        ops.append(op)
    b = dgp.dg_batch_create([o.handle for o in ops], [s.data_ptr() for s in srcs], [d.data_ptr() for d in dsts],
                            autotune=True, branches=4)
    groups, launches = dgp.dg_batch_info(b)
    assert groups < len(ops) and launches < len(ops)
    dgp.dg_batch_launch(b)
    torch.cuda.synchronize()
    for c, d, r in zip(cases, dsts, refs):
        got = d.double().cpu().numpy()
        rel = float(np.linalg.norm(got - r) / np.linalg.norm(r))
        assert rel < tol[c["prec"]], (c, rel)
    dgp.dg_batch_destroy(b)
    for o in ops:
        o.close()
