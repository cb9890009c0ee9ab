"""Solve server: admission under a memory budget, overlap of concurrent
requests, and results that are the same alone and in the mix."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402


def _req(n, p, mapping, out=None, rtol=1e-8):
    return dgp.make_request(n, p, mapping=mapping, rtol=rtol, x_host_ptr=out.ctypes.data if out is not None else None)


def test_result_same_alone_and_in_the_mix():
    dgp.build()
    n, p = (5, 4, 6), 3
    ndofs = 5 * 4 * 6 * (p + 1) ** 3
    alone = np.full(ndofs, np.nan)
    res = dgp.serve_arrivals([_req(n, p, 1, alone)], [0.0], 8 << 30, 1)[0]
    assert res["status"] == dgp.DG_OK and res["rel_res"] <= 1e-8
    # the same request among others of different sizes, degrees and meshes,
    # several running at once
    mixed = np.full(ndofs, np.nan)
    others = [((8, 8, 8), 2, 0), ((6, 6, 6), 4, 1), ((10, 9, 8), 2, 1), ((4, 4, 4), 6, 0), ((7, 7, 7), 3, 1)]
    reqs = [_req(nn, pp, mm) for nn, pp, mm in others[:2]] + [_req(n, p, 1, mixed)] + \
           [_req(nn, pp, mm) for nn, pp, mm in others[2:]]
    results = dgp.serve_arrivals(reqs, [0.0] * len(reqs), 32 << 30, 4)
    assert all(r["status"] == dgp.DG_OK for r in results), [(r["status"], r["message"]) for r in results]
    assert np.array_equal(alone, mixed)
    # several requests overlapped in time
    spans = sorted((r["t_admit"], r["t_done"]) for r in results)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))


def test_solution_matches_plain_fp64_cg():
    dgp.build()
    n, p = (6, 5, 4), 4
    x = np.zeros(6 * 5 * 4 * (p + 1) ** 3)
    res = dgp.serve_arrivals([_req(n, p, 1, x, rtol=1e-10)], [0.0], 8 << 30, 2)[0]
    assert res["status"] == dgp.DG_OK
    op = dgp.Operator(n, p, geom="full", mapping=1, coeff=1)
    xr, it, rr, st = op.cg(op.rhs(1), rtol=1e-10, max_it=20000)
    xr = xr.cpu().numpy()
    assert np.linalg.norm(x - xr) <= 1e-7 * np.linalg.norm(xr)


def test_admission_respects_the_budget():
    dgp.build()
    reqs = [_req((6, 6, 6), 3, 1) for _ in range(4)]
    one = dgp.dg_request_device_bytes(reqs[0])
    # room for one request at a time: admissions are serialized
    results = dgp.serve_arrivals(reqs, [0.0] * 4, int(one * 1.5), 4)
    spans = sorted((r["t_admit"], r["t_done"]) for r in results)
    for a, b in zip(spans, spans[1:]):
        assert b[0] >= a[1] - 1e-6
    server = dgp.dg_server_create(one // 2, 1)
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_server_submit(server, reqs[0])
    assert e.value.status == dgp.DG_ERR_ARG
    dgp.dg_server_destroy(server)


def test_served_solutions_against_the_oracle():
    """Each served solution of a small mixed set (degrees 2-4, Cartesian and
    deformed meshes, run together) against the FP64 oracle: its residual with
    the oracle's assembled matrix and its distance to the oracle's own CG
    solution."""
    import oracle
    dgp.build()
    cases = [((3, 4, 3), 2, 1), ((4, 3, 3), 3, 0), ((3, 3, 3), 4, 1), ((2, 3, 4), 3, 1)]
    rtol = 1e-10
    outs = [np.full(n[0] * n[1] * n[2] * (p + 1) ** 3, np.nan) for n, p, _ in cases]
    reqs = [_req(n, p, m, x, rtol=rtol) for (n, p, m), x in zip(cases, outs)]
    results = dgp.serve_arrivals(reqs, [0.0] * len(reqs), 8 << 30, 3)
    for (n, p, m), x, r in zip(cases, outs, results):
        assert r["status"] == dgp.DG_OK and r["rel_res"] <= rtol, (n, p, m, r["message"])
        mesh = dict(n=n, periodic=False, mapping=m, amplitude=0.1)
        A = oracle.assemble(mesh, p, dict(op="sipg", coeff=m))
        b = oracle.rhs(mesh, p, m)
        assert np.linalg.norm(b - A @ x) <= 3 * rtol * np.linalg.norm(b), (n, p, m)
        xo, _, rro = oracle.cg(A, b, rtol=1e-13, maxit=20000)
        assert np.linalg.norm(x - xo) <= 1e-7 * np.linalg.norm(xo), (n, p, m)


@pytest.mark.parametrize("policy", [0, 1])
def test_admission_policy_order(policy):
    """One slot: a running request, then a large and two small ones queued
    behind it.  FIFO admits the large one first; shortest job first (no
    aging within the test) admits the small ones first.  Results are the same
    either way (each solve is independent of the mix)."""
    dgp.build()
    blocker = _req((8, 8, 8), 3, 1)
    large = _req((10, 10, 10), 4, 1)
    small = [_req((3, 3, 3), 2, 0), _req((4, 3, 3), 2, 1)]
    server = dgp.dg_server_create(32 << 30, 1)
    try:
        if policy:
            dgp.dg_server_set_policy(server, 1, 100.0)
        tickets = [dgp.dg_server_submit(server, r) for r in [blocker, large] + small]
        res = [dgp.dg_server_wait(server, t) for t in tickets]
    finally:
        dgp.dg_server_destroy(server)
    assert all(r["status"] == dgp.DG_OK for r in res)
    t_large, t_small = res[1]["t_admit"], min(r["t_admit"] for r in res[2:])
    if policy == 0:
        assert t_large < t_small
    else:
        assert t_small < t_large


def test_policy_rejects_bad_arguments():
    dgp.build()
    server = dgp.dg_server_create(1 << 30, 1)
    try:
        with pytest.raises(dgp.DGError):
            dgp.dg_server_set_policy(server, 2, 0.0)
        with pytest.raises(dgp.DGError):
            dgp.dg_server_set_policy(server, 1, -1.0)
    finally:
        dgp.dg_server_destroy(server)
