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
