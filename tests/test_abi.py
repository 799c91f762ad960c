"""The C-ABI library builds, loads, and exports every entry point the header declares."""
import os
import re

import pytest

from paper_1408_5535_gb300 import native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "phsvds.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(phsvds_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(native.LIB_PATH):
        import __graft_entry__
        __graft_entry__.build()
    return native.lib()


def test_header_declares_the_boundary():
    d = _declared()
    for name in ("phsvds_create", "phsvds_solve", "phsvds_destroy", "phsvds_ata_spmm_f64"):
        assert name in d


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name
    assert sorted(native.EXPORTED) == _declared()


def test_default_opts_and_status_strings(lib):
    o = native.default_opts()
    assert (o.block_size, o.max_basis, o.min_restart, o.max_restarts) == (1, 35, 21, 10000)
    assert lib.phsvds_status_string(0) == b"ok"
    assert lib.phsvds_status_string(2) == b"not converged"


def test_create_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.PhsvdsError):
        native.Handle(0)


def test_static_scratch_capacity_matches_header():
    """The binding's capacity of the allocation-free SpMM scratch is the header's."""
    txt = open(os.path.join(ROOT, "include", "phsvds.h")).read()
    assert int(re.search(r"#define\s+PHSVDS_STATIC_Z_MAX\s+(\d+)", txt).group(1)) == native.STATIC_Z_MAX
