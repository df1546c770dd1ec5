"""The C-ABI library builds, loads and exports every symbol include/sft.h
declares; argument errors are reported without touching a GPU."""
import ctypes as C

import pytest

from paper_2501_06377_gb300 import build as B
from paper_2501_06377_gb300 import sft


@pytest.fixture(scope="module")
def lib():
    B.build()
    return sft.load()


def test_every_header_function_is_exported(lib):
    names = sft.header_functions()
    assert len(names) >= 20
    raw = C.CDLL(sft.LIB_PATH)
    missing = [n for n in names if not hasattr(raw, n)]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    assert set(sft.header_functions()) == set(sft._SIGS)


def test_abi_version(lib):
    assert lib.sft_abi_version() == 7


def test_create_rejects_bad_arguments_before_any_cuda_call(lib):
    h = C.c_void_p()
    assert lib.sft_create_grid(None, 0, 0, 0, None, C.byref(h)) == sft.SFT_ERR_ARG
    shp = (sft.sft_shape * 1)(sft.sft_shape(4, 64))   # ntheta < 5
    assert lib.sft_create_grid(shp, 1, 0, 0, None, C.byref(h)) == sft.SFT_ERR_ARG
    assert b"shape" in lib.sft_last_error(None)
    shp = (sft.sft_shape * 1)(sft.sft_shape(16, 64))
    assert lib.sft_create_grid(shp, 1, 7, 0, None, C.byref(h)) == sft.SFT_ERR_ARG
    assert lib.sft_step(None, 1.0, 0, None) == sft.SFT_ERR_ARG


def test_noalloc_rejects_oversized_maps_before_any_cuda_call(lib):
    """The size check of sft_flux_diagnostics_noalloc comes before any CUDA
    call, so it is checked here without a GPU (no map is ever read)."""
    out = sft.sft_diag()
    fake = C.c_void_p(256)   # never dereferenced: the call must stop at the size check
    big = 1 << 20            # tables alone need 32 MiB >> the 4 MiB scratch
    assert lib.sft_flux_diagnostics_noalloc(fake, big, big, 0, 60.0, None, C.byref(out)) == sft.SFT_ERR_ARG
    assert b"scratch" in lib.sft_last_error(None)
    assert lib.sft_flux_diagnostics_noalloc(fake, 64, 7, 0, 60.0, None, C.byref(out)) == sft.SFT_ERR_ARG
    assert lib.sft_flux_diagnostics_noalloc(None, 64, 128, 0, 60.0, None, C.byref(out)) == sft.SFT_ERR_ARG


def test_surrogate_header_exported_and_bound(lib):
    from paper_2501_06377_gb300 import surrogate
    names = sft.header_functions(sft.HEADER.replace("sft.h", "sfs.h"), prefix="sfs_")
    assert len(names) >= 10
    raw = C.CDLL(sft.LIB_PATH)
    assert all(hasattr(raw, n) for n in names)
    assert set(names) == set(surrogate._SIGS)


def test_debug_entry_points_without_a_gpu(lib):
    """The release library reports that it has no device checks, and the
    allocation-failure injector validates its argument (no CUDA call)."""
    assert lib.sft_debug_checks(None, None, 0) == sft.SFT_ERR_STATE
    assert b"SFT_DEBUG" in lib.sft_last_error(None)
    assert lib.sft_debug_probe(1, 5, 0, 10) == sft.SFT_ERR_STATE
    assert lib.sft_debug_fail_alloc(-1) == sft.SFT_ERR_ARG
    assert lib.sft_debug_fail_alloc(0) == sft.SFT_OK


def test_debug_library_builds_and_exports_the_header():
    path = B.build(debug=True)
    raw = C.CDLL(path)
    missing = [n for n in sft.header_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_every_declaration_is_documented():
    """Each C-ABI entry point has its own comment block right above it
    (argument meaning, layout, ownership and errors are stated there)."""
    import os
    import re
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    for name in ("sft.h", "sfs.h"):
        text = open(os.path.join(root, "include", name)).read()
        decls = list(re.finditer(r"^(?:sft_status|int32_t|int64_t|const char\*|void|double)\s+"
                                 r"((?:sft|sfs)_[a-z0-9_]+)\s*\(", text, flags=re.M))
        assert len(decls) >= 8
        bare = [m.group(1) for m in decls if not text[:m.start()].rstrip().endswith("*/")]
        assert not bare, (name, bare)
