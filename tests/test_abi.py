"""The C-ABI library builds, loads and exports every entry point that
include/lbm.h declares (no compute call: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1903_01111_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("lbm_create_lattice", "lbm_destroy", "lbm_set_geometry", "lbm_init_equilibrium", "lbm_step",
                     "lbm_moments", "lbm_force", "lbm_get_distributions", "lbm_set_distributions",
                     "lbm_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_wraps_every_declared_symbol(lib):
    from paper_1903_01111_gb300 import lbm

    assert sorted(lbm.EXPORTED) == _declared()


def test_last_error_is_empty_string_initially(lib):
    lib.lbm_last_error.restype = ctypes.c_char_p
    assert lib.lbm_last_error() == b""


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # argument checks run before any CUDA call
    from paper_1903_01111_gb300 import lbm

    assert lib.lbm_create_lattice(None, None) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_step(None, ctypes.c_int64(1)) == lbm.LBM_ERR_INVALID_ARG
    assert lib.lbm_destroy(None) == lbm.LBM_OK


def test_config_layouts_agree_with_the_oracle():
    """The oracle and the library read the same test inputs; their config
    structs share the leading fields in the same order."""
    import oracle as O
    from paper_1903_01111_gb300 import lbm

    ofields = [f[0] for f in O.OracleConfig._fields_]
    lfields = [f[0] for f in lbm.lbm_config._fields_]
    assert lfields[: len(ofields)] == ofields
    assert O.LINK_DTYPE == lbm.LINK_DTYPE


def test_noalloc_binding_rejects_host_tensors_before_the_call():
    """lbm_force_noalloc's binding checks its tensor arguments (device,
    dtype, size) before it calls into the library; a host tensor is refused
    without touching a GPU."""
    torch = pytest.importorskip("torch")
    from paper_1903_01111_gb300 import lbm

    cfg = lbm.make_config(stencil=0, nx=8, ny=8, nz=1, tau=0.8)
    f = torch.zeros(9 * 64, dtype=torch.float64)
    solid = torch.zeros(64, dtype=torch.uint8)
    links = torch.zeros(lbm.LINK_DTYPE.itemsize, dtype=torch.uint8)
    F = torch.zeros(3, dtype=torch.float64)
    with pytest.raises(ValueError, match="f_post"):
        lbm.lbm_force_noalloc(cfg, f, solid, links, 1, 0, F)
