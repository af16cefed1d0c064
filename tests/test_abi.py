"""The C-ABI library builds, loads without a GPU and exports every function
include/stokes.h declares."""
import pathlib
import re

import pytest

ROOT = pathlib.Path(__file__).resolve().parent.parent


def _declared():
    text = (ROOT / "include" / "stokes.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(stokes_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    b = __graft_entry__._build_module()
    if not b.LIB.exists():
        b.build()
    import paper_1609_04484_gb300 as S
    return S


def test_header_declares_the_boundary():
    names = _declared()
    for want in ("stokes_geometry_create", "stokes_matvec", "stokes_precond_setup",
                 "stokes_gmres_solve", "stokes_eval_velocity", "stokes_last_error"):
        assert want in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib.lib, name), name
        assert hasattr(lib, name), f"binding lacks {name}"


def test_null_handle_is_rejected_without_gpu(lib):
    assert lib.lib.stokes_geometry_num_nodes(None) == -1
    assert lib.lib.stokes_precond_setup(None, 1, None) == lib.STOKES_EINVAL
    assert "null handle" in lib.stokes_last_error()
    assert lib.lib.stokes_geometry_destroy(None) == lib.STOKES_OK


def test_noalloc_binding_checks_array_lengths_without_gpu(lib):
    """The binding rejects offsets or centres that do not match n_comp
    before the library would read past their ends."""
    import numpy as np
    z = np.zeros(16)
    with pytest.raises(ValueError):
        lib.stokes_matvec_noalloc(z, z, z, z, np.array([0, 8], dtype=np.int64), 2, 0, np.zeros(4), z, z)
    with pytest.raises(ValueError):
        lib.stokes_matvec_noalloc(z, z, z, z, np.array([0, 8, 16], dtype=np.int64), 2, 0, np.zeros(2), z, z)
