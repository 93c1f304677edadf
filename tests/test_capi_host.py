"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function include/pcms.h declares, and rejects invalid arguments before enqueuing work."""
import ctypes
import os

import pytest

from tests._helpers import header_functions


@pytest.fixture(scope="module")
def lib():
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    return pcms.lib()


def test_header_declares_the_boundary():
    fns = header_functions()
    for name in ["pcms_create_map", "pcms_apply_map", "pcms_locate_interp", "pcms_mls_transfer",
                 "pcms_mesh_create", "pcms_map_export", "pcms_last_error"]:
        assert name in fns


def test_library_exports_every_declared_symbol(lib):
    from paper_2510_18838_gb300 import pcms
    for name in header_functions():
        assert hasattr(lib, name), name
        assert name in pcms.SIGNATURES, f"binding lacks {name}"


def test_version_and_defaults(lib):
    from paper_2510_18838_gb300 import pcms
    assert lib.pcms_version() >= 10000
    o = pcms.MapOpts()
    lib.pcms_map_opts_default(ctypes.byref(o))
    assert o.precision == pcms.FP64 and o.weight == 0 and o.lambda_ == 0.0
    assert o.min_neighbors == 0 and o.domain_known == 0 and o.growth == 0


@pytest.mark.parametrize("dim,deg,radius,ns,nt", [
    (6, 1, 0.1, 10, 10), (1, 1, 0.1, 10, 10), (2, 3, 0.1, 10, 10), (2, -1, 0.1, 10, 10),
    (2, 1, 0.0, 10, 10), (2, 1, -1.0, 10, 10), (2, 1, float("nan"), 10, 10),
    (2, 1, float("inf"), 10, 10), (2, 1, 0.1, -1, 10), (2, 1, 0.1, 10, -5),
    (2, 1, 0.1, 1 << 31, 10),
])
def test_create_map_rejects_bad_arguments(lib, dim, deg, radius, ns, nt):
    from paper_2510_18838_gb300 import pcms
    h = ctypes.c_void_p(123)
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation fails first
    st = lib.pcms_create_map(dim, fake, ns, fake, nt, deg, radius, None, None, ctypes.byref(h))
    assert st == pcms.INVALID_ARG
    assert h.value is None
    assert b"pcms_create_map" in lib.pcms_last_error()


def test_dimensions_above_three_are_fp64_only(lib):
    from paper_2510_18838_gb300 import pcms
    h = ctypes.c_void_p()
    fake = ctypes.c_void_p(0x1000)
    o = pcms.MapOpts()
    lib.pcms_map_opts_default(ctypes.byref(o))
    for dim in (4, 5):
        bad = pcms.MapOpts.from_buffer_copy(o)
        bad.precision = pcms.MIXED
        assert lib.pcms_create_map(dim, fake, 5, fake, 5, 1, 0.1, ctypes.byref(bad), None,
                                   ctypes.byref(h)) == pcms.INVALID_ARG
        bad = pcms.MapOpts.from_buffer_copy(o)
        bad.domain_known = 1
        assert lib.pcms_create_map(dim, fake, 5, fake, 5, 1, 0.1, ctypes.byref(bad), None,
                                   ctypes.byref(h)) == pcms.INVALID_ARG
    assert lib.pcms_create_map(6, fake, 5, fake, 5, 1, 0.1, None, None,
                               ctypes.byref(h)) == pcms.INVALID_ARG


def test_null_pointers_and_bad_opts_rejected(lib):
    from paper_2510_18838_gb300 import pcms
    h = ctypes.c_void_p()
    assert lib.pcms_create_map(2, None, 5, None, 5, 1, 0.1, None, None, ctypes.byref(h)) == pcms.INVALID_ARG
    assert lib.pcms_create_map(2, None, 0, None, 0, 1, 0.1, None, None, None) == pcms.INVALID_ARG
    o = pcms.MapOpts()
    lib.pcms_map_opts_default(ctypes.byref(o))
    fake = ctypes.c_void_p(0x1000)
    for field, val in [("precision", 7), ("weight", 42), ("lambda_", -1.0), ("min_neighbors", -3),
                       ("growth", 2), ("growth", -1)]:
        bad = pcms.MapOpts.from_buffer_copy(o)
        setattr(bad, field, val)
        assert lib.pcms_create_map(2, fake, 5, fake, 5, 1, 0.1, ctypes.byref(bad), None,
                                   ctypes.byref(h)) == pcms.INVALID_ARG, field
    bad = pcms.MapOpts.from_buffer_copy(o)
    bad.domain_known = 1
    bad.lo[0], bad.hi[0] = 1.0, 0.0
    assert lib.pcms_create_map(2, fake, 5, fake, 5, 1, 0.1, ctypes.byref(bad), None,
                               ctypes.byref(h)) == pcms.INVALID_ARG


def test_apply_transfer_mesh_argument_checks(lib):
    from paper_2510_18838_gb300 import pcms
    fake = ctypes.c_void_p(0x1000)
    assert lib.pcms_apply_map(None, fake, 1, fake, None) == pcms.INVALID_ARG
    for nf in (0, 17, -1):
        assert lib.pcms_mls_transfer(2, fake, 5, fake, 5, 1, 0.1, None, fake, nf, fake, None,
                                     None) == pcms.INVALID_ARG
    h = ctypes.c_void_p()
    assert lib.pcms_mesh_create(None, 4, fake, 2, None, ctypes.byref(h)) == pcms.INVALID_ARG
    assert lib.pcms_mesh_create(fake, -1, fake, 2, None, ctypes.byref(h)) == pcms.INVALID_ARG
    assert lib.pcms_locate_interp(None, fake, 3, None, fake, None, None, None) == pcms.INVALID_ARG
    lib.pcms_map_destroy(None, None)     # no-ops
    lib.pcms_mesh_destroy(None, None)


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2510_18838_gb300 import pcms
    monkeypatch.setattr(pcms, "_lib", None)
    monkeypatch.setattr(pcms, "LIB_PATH", os.path.join(str(tmp_path), "missing.so"))
    with pytest.raises(ImportError):
        pcms.lib()


def test_tune_table_is_validated_and_replaced_whole():
    """pcms_tune_set takes a whole table or nothing: an invalid entry (lanes other than 8 or
    32, a cell divisor out of [1, 8], an apply bucket beyond 16 fields) is refused and the
    table stays as it was. No GPU is needed."""
    from paper_2510_18838_gb300 import build, pcms
    build.build()
    good = [{"dim": 2, "degree": 2, "precision": "mixed", "mode": pcms.TUNE_MAP, "bucket": 5,
             "lanes": 8, "cell_div": 4.0},
            {"dim": 3, "degree": 2, "precision": "mixed", "mode": pcms.TUNE_APPLY, "bucket": 16,
             "apply_form": 1}]
    pcms.tune_set(good)
    assert len(pcms.tune_get()) == 2
    for bad in (dict(good[0], lanes=16), dict(good[0], cell_div=0.5), dict(good[0], dim=4),
                dict(good[1], bucket=17), dict(good[0], mode=7)):
        with pytest.raises(pcms.PcmsError):
            pcms.tune_set([good[0], bad])
        assert pcms.tune_get() == [dict(good[0], apply_form=0),
                                   dict(good[1], lanes=0, cell_div=0.0)]
    pcms.tune_set([])
    assert pcms.tune_get() == []
