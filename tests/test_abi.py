"""The C-ABI library: built, loadable, exporting every symbol of include/dg.h
(no compute calls: these run without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("dg_setup", "dg_apply", "dg_cg_solve", "dg_destroy", "dg_last_error", "dg_rhs", "dg_n_dofs"):
        assert n in names


def test_library_exports_every_declared_symbol():
    import ctypes
    import paper_1711_03590_gb300 as dgp
    path = dgp.build()
    lib = ctypes.CDLL(path)
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(dgp.EXPORTED) == _declared()


def test_bindings_fail_loudly_without_library(tmp_path):
    import paper_1711_03590_gb300 as dgp
    with pytest.raises(dgp.DGLibraryMissing):
        dgp._lib_backup = dgp._lib
        try:
            dgp._lib = None
            dgp.load_library(str(tmp_path / "missing.so"))
        finally:
            dgp._lib = dgp._lib_backup


def test_setup_errors_without_gpu_are_status_codes():
    """Argument checks happen before any device work and return codes."""
    import paper_1711_03590_gb300 as dgp
    dgp.build()
    m = dgp.make_mesh(4, periodic=True, mapping=1)
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_setup(m, 2, "cartesian", dgp.make_opts())
    assert e.value.status == dgp.DG_ERR_ARG
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_setup(m, 9, "full", dgp.make_opts())
    assert e.value.status == dgp.DG_ERR_ARG
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_setup(m, 2, 1, dgp.make_opts())  # 1: no geometry variant (no per-cell affine storage)
    assert e.value.status == dgp.DG_ERR_ARG


@pytest.mark.parametrize("case", [
    dict(n=(0, 4, 4)),                    # no cells along x
    dict(n=(4, 4, -1)),                   # negative extent
    dict(n=(1 << 21, 1, 1)),              # beyond 2^20 cells per direction
    dict(n=(1 << 20, 1 << 20, 1)),        # more than 2^31 - 1 cells
    dict(degree=0),
    dict(degree=-3),
    dict(mapping=3),
    dict(op=5),
    dict(prec=7),
    dict(coeff=2),
    dict(basis=3),
    dict(basis="hermite", degree=2),      # the Hermite-like basis needs degree >= 3
    dict(geom=9),
    dict(geom="cartesian", mapping=1),    # Cartesian storage on a curved mesh
    dict(mapping=2, periodic=True, coeff=1),  # kappa(x) not periodic on the sheared mesh
])
def test_degenerate_and_out_of_range_setup_arguments(case):
    """Empty meshes, out-of-range sizes and degrees and unknown enum values
    are rejected with DG_ERR_ARG before any device work (no GPU needed)."""
    import paper_1711_03590_gb300 as dgp
    dgp.build()
    m = dgp.make_mesh(case.get("n", (4, 4, 4)), periodic=case.get("periodic", False),
                      mapping=case.get("mapping", 1))
    o = dgp.make_opts(op=case.get("op", "sipg"), prec=case.get("prec", "fp64"), coeff=case.get("coeff", 0),
                      basis=case.get("basis", "lagrange"))
    with pytest.raises(dgp.DGError) as e:
        dgp.dg_setup(m, case.get("degree", 2), case.get("geom", "full"), o)
    assert e.value.status == dgp.DG_ERR_ARG


def test_request_memory_estimate_is_host_arithmetic():
    """The server's admission estimate (no device work, so no GPU needed):
    invalid requests give -1; the estimate grows with the mesh, in
    proportion to the dofs once the fixed 64 MiB is taken off, and orders
    the geometry storages by their per-point arrays (G3 > G4 > Cartesian)."""
    import paper_1711_03590_gb300 as dgp
    dgp.build()
    est = dgp.dg_request_device_bytes
    assert est(dgp.make_request(8, 0)) == -1
    assert est(dgp.make_request(8, 9)) == -1
    assert est(dgp.make_request((0, 8, 8), 3)) == -1
    fixed = 64 << 20
    small, large = est(dgp.make_request(16, 4)), est(dgp.make_request(32, 4))
    assert fixed < small < large
    assert abs((large - fixed) / (small - fixed) - 8.0) < 1e-6
    g3 = est(dgp.make_request(16, 4, geom="full"))
    g4 = est(dgp.make_request(16, 4, geom="merged"))
    g2 = est(dgp.make_request(16, 4, geom="positions"))
    cart = est(dgp.make_request(16, 4, mapping=0))
    assert g3 > g4 > g2 > cart > fixed
    # 32^3 cells at p = 4 with G3 storage: 4,096,000 dofs at
    # (10 + 21/5) x (8 + 4) geometry bytes and 88 vector bytes per dof
    assert large == int(4096000 * ((10 + 21 / 5) * 12 + 88)) + fixed
