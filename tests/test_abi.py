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
