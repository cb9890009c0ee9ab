"""The allocation-free apply (dg_apply_dot_noalloc) against the allocating
entry point.

dg_apply_dot_noalloc serves callers that cannot allocate device memory while
they run (a memory pool owned by another framework, a real-time loop, a
device budget already handed out): its scratch is a fixed static device
array.  Its dst must equal dg_apply's dst, and its dot must equal the FP64
product src . dst, on two calls in a row (the second call must not see the
first call's leftovers).  This file is collected last so a failure here
comes after every other test has run.
"""
import numpy as np
import pytest

import dg_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1711_03590_gb300 as dgp  # noqa: E402


CASES = [("fp64", "element", 1e-12), ("fp32", "element", 1e-5), ("fp64", "loop", 1e-12),
         ("fp64emu", "element", 1e-12), ("fp64emu", "loop", 1e-12)]


@pytest.mark.parametrize("prec,mode,tol", CASES)
def test_noalloc_apply_dot_matches_allocating_path(prec, mode, tol):
    """Both face modes (the face loop writes the partials in its second
    launch) and all three arithmetics, two calls in a row."""
    dgp.build()
    op = dgp.Operator((6, 5, 7), 3, geom="full", prec=prec, mapping=1, coeff=1)
    if mode != "element":
        op.set_face_mode(mode)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    for call, seed in enumerate((21, 22)):
        src = torch.tensor(dg_inputs.src_vector(op.n_dofs, seed), dtype=op.dtype, device="cuda")
        ref = op.apply(src)
        dst = torch.full_like(src, float("nan"))
        dgp.dg_apply_dot_noalloc(op.handle, src.data_ptr(), dst.data_ptr(), dot.data_ptr())
        torch.cuda.synchronize()
        rel = float((dst.double() - ref.double()).norm() / ref.double().norm())
        assert rel <= tol, (call, rel)
        want = float(torch.dot(src.double(), ref.double()))
        got = float(dot.item())
        assert abs(got - want) <= tol * float(src.double().norm() * ref.double().norm()), (call, got, want)
    op.close()


def test_noalloc_leaves_free_device_memory_unchanged():
    """The defining property: once the operator is set up, calls change the
    device's free memory by nothing (no allocation, no lazy module load)."""
    dgp.build()
    op = dgp.Operator((5, 6, 4), 2, geom="full", prec="fp64", mapping=1, coeff=1)
    src = torch.tensor(dg_inputs.src_vector(op.n_dofs, 5), dtype=op.dtype, device="cuda")
    dst = torch.empty_like(src)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    dgp.dg_apply_dot_noalloc(op.handle, src.data_ptr(), dst.data_ptr(), dot.data_ptr())  # warm-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        dgp.dg_apply_dot_noalloc(op.handle, src.data_ptr(), dst.data_ptr(), dot.data_ptr())
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    op.close()


def test_noalloc_rejects_too_many_blocks():
    dgp.build()
    # one cell per block: 65537 cells need more than 65536 blocks
    op = dgp.Operator((65537, 1, 1), 1, geom="cartesian", prec="fp64")
    op.set_cells_per_block(1)
    assert op.info()["blocks"] > 65536
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    src = torch.zeros(op.n_dofs, dtype=torch.float64, device="cuda")
    dst = torch.zeros_like(src)
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_apply_dot_noalloc(op.handle, src.data_ptr(), dst.data_ptr(), dot.data_ptr())
    assert e.value.status == dgp.DG_ERR_ARG
    assert "65536" in str(e.value)
    op.close()
