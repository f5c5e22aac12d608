"""The C-ABI library builds, loads and exports every symbol include/pmat.h
declares; argument checks answer without a GPU (no compute calls here)."""
import ctypes as C

import pytest

from paper_1905_04356_gb300 import build as pbuild
from paper_1905_04356_gb300 import pmat


@pytest.fixture(scope="module")
def L():
    pbuild.build()
    return pmat.lib()


def test_header_declares_the_boundary():
    names = pmat.header_functions()
    for n in ("pm_create", "pm_destroy", "pm_set_option", "pm_sync", "pm_last_error", "pmat_mul",
              "pmat_mul_trunc", "pmat_middle_product", "pmat_mul_batched", "pm_basis", "bivariate_resultant"):
        assert n in names


def test_library_exports_every_declared_symbol(L):
    for n in pmat.header_functions():
        assert hasattr(L, n), n


def test_null_context_is_rejected(L):
    assert L.pm_destroy(None) == pmat.PM_EINVAL
    assert L.pm_sync(None) == pmat.PM_EINVAL
    assert L.pm_set_option(None, 1, 0) == pmat.PM_EINVAL
    assert L.pmat_mul(None, 97, 4, 1, 1, 1, None, 1, None, 1, None) == pmat.PM_EINVAL
    assert L.pmat_mul_trunc(None, 97, 4, 1, 1, 1, None, 1, None, 1, 1, None) == pmat.PM_EINVAL
    assert L.pmat_middle_product(None, 97, 4, 1, 1, 1, None, 1, None, 1, 0, 1, None) == pmat.PM_EINVAL
    assert L.pmat_mul_batched(None, 0, None) == pmat.PM_EINVAL
    assert L.pm_basis(None, 97, 2, 1, None, 1, 1, None, None, None) == pmat.PM_EINVAL
    assert L.bivariate_resultant(None, 1, None, 1, 1, None, 1, 1, None, None) == pmat.PM_EINVAL
    assert L.pm_last_error(None) == b"null context"


def test_create_on_missing_device_is_rejected(L):
    h = C.c_void_p()
    assert L.pm_create(C.byref(h), 1 << 20, None) == pmat.PM_EINVAL
    assert not h.value
