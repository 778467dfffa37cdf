"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/flash.h declares (no GPU needed: nothing is called but the symbols'
lookup and the pure host helpers)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flash.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(flash_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def libflash():
    import paper_1709_01190_gb300 as fl
    path = fl.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path():
    names = declared_functions()
    for n in ("flash_hash", "flash_keys", "flash_build", "flash_query", "flash_knn_graph", "flash_index_free",
              "flash_strerror", "flash_index_export", "flash_set_scratch_budget"):
        assert n in names


def test_every_declared_symbol_is_exported(libflash):
    missing = [n for n in declared_functions() if not hasattr(libflash, n)]
    assert not missing, missing


def test_host_only_helpers(libflash):
    libflash.flash_strerror.restype = ctypes.c_char_p
    assert libflash.flash_strerror(0) == b"ok"
    assert b"invalid" in libflash.flash_strerror(1)
    libflash.flash_version.restype = ctypes.c_char_p
    assert b"sm_103a" in libflash.flash_version()
    import paper_1709_01190_gb300 as fl
    p = fl.FlashParams(4, 64, 64, 18, 1)
    need = fl.flash_knn_graph_scratch_bytes(p, 350_000)
    assert need >= 5 * 4 * 64 * 350_000  # keys, sorted keys, sort ping-pong, ids
    assert fl.flash_knn_graph_scratch_bytes(fl.FlashParams(0, 1, 1, 1, 1), 10) == 0
    assert fl.flash_knn_graph_scratch_bytes(fl.FlashParams(4, 64, 64, 18, 1, densify=1), 10) > 0
    assert fl.flash_knn_graph_scratch_bytes(fl.FlashParams(4, 64, 64, 18, 1, densify=2), 10) == 0
    old = fl.flash_set_scratch_budget(123)
    assert fl.flash_set_scratch_budget(old) == 123


def test_product_path_fails_loudly_without_a_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    import paper_1709_01190_gb300 as fl
    with pytest.raises(Exception):
        fl.hash_rows(fl.FlashParams(2, 2, 2, 4, 1), None)


def test_tuning_knobs_roundtrip_and_validation(libflash):
    from paper_1709_01190_gb300 import FlashError, tuning
    try:
        t = tuning.Tuning(query_warp_table=256, doph_rows_per_grab=8, doph_order=1)
        tuning.set_tuning(t)
        assert tuning.get_tuning() == t
        for bad in (tuning.Tuning(query_warp_table=100), tuning.Tuning(query_warp_table=32),
                    tuning.Tuning(doph_order=2), tuning.Tuning(doph_rows_per_grab=5000)):
            with pytest.raises(FlashError):
                tuning.set_tuning(bad)
        assert tuning.get_tuning() == t      # a rejected setting changes nothing
    finally:
        tuning.set_tuning(None)
    assert tuning.get_tuning() == tuning.Tuning()
