"""The C ABI library on a machine without a GPU: it loads, exports every
function include/crac.h declares, and its host-side registry logic (no CUDA
call involved) behaves as documented."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def C():
    import __graft_entry__
    __graft_entry__._load_builder().build()
    import paper_2008_10596_gb300 as mod
    return mod


def _declared():
    txt = open(os.path.join(ROOT, "include", "crac.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"CRAC_API[^;(]*?\b(crac_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(C):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(C.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(C.EXPORTED) == names


def test_boundary_calls_present(C):
    for n in ("crac_register_alloc", "crac_free", "crac_checkpoint", "crac_restart"):
        assert n in _declared()


def test_status_strings(C):
    assert C.crac_status_str(0) == "CRAC_OK"
    assert C.crac_status_str(-6) == "CRAC_ERR_IMAGE_MISMATCH"
    assert C.crac_status_str(-99) == "CRAC_ERR_UNKNOWN"


def test_config_validation(C):
    for bad in (dict(chunk_bytes=3000), dict(chunk_bytes=8), dict(chunk_bytes=1 << 25),
                dict(image_residency=7), dict(launch_mode=9), dict(threads=128),
                dict(warps_per_chunk=3), dict(chunks_per_tile=1000), dict(pass_kernel=5),
                dict(pass_kernel=C.CRAC_PASS_TMA, chunk_bytes=512),
                dict(pass_kernel=C.CRAC_PASS_TMA, chunk_bytes=128 << 10),
                dict(pass_kernel=C.CRAC_PASS_SPARSE),         # needs device-resident images
                dict(flags=32),
                dict(pass_kernel=C.CRAC_PASS_SPARSE, image_residency=C.CRAC_RESIDENCY_DEVICE,
                     flags=C.CRAC_FLAG_COMPRESS)):       # the sparse payload is not compacted
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_create(C.crac_config_default(**bad))
        assert e.value.code == C.CRAC_ERR_INVALID_ARG
    for ok in (dict(pass_kernel=C.CRAC_PASS_TMA, chunk_bytes=1024),
               dict(pass_kernel=C.CRAC_PASS_TMA, chunk_bytes=64 << 10),
               dict(pass_kernel=C.CRAC_PASS_SPARSE, image_residency=C.CRAC_RESIDENCY_DEVICE),
               dict(flags=C.CRAC_FLAG_COMPRESS | C.CRAC_FLAG_DIRECT_DRAIN),
               dict(flags=C.CRAC_FLAG_WAIT_PASS),
               dict(pass_kernel=C.CRAC_PASS_TMA, chunk_bytes=4096, flags=C.CRAC_FLAG_COMPRESS)):
        C.crac_ctx_destroy(C.crac_ctx_create(C.crac_config_default(**ok)))


def test_registry_host_logic(C):
    ctx = C.crac_ctx_create(C.crac_config_default(chunk_bytes=4096))
    base = 1 << 40
    C.crac_ctx_register_alloc(ctx, base, 100)
    C.crac_ctx_register_alloc(ctx, base + 112, 16, C.CRAC_KIND_MANAGED)   # adjacent
    cases = [((base + 64, 10), C.CRAC_ERR_OVERLAP), ((base + 8, 8), C.CRAC_ERR_INVALID_ARG),
             ((base + 4096, 0), C.CRAC_ERR_INVALID_ARG), ((0, 16), C.CRAC_ERR_INVALID_ARG)]
    for (p, n), code in cases:
        with pytest.raises(C.CracError) as e:
            C.crac_ctx_register_alloc(ctx, p, n)
        assert e.value.code == code
    with pytest.raises(C.CracError) as e:
        C.crac_ctx_register_alloc(ctx, base + 4096, 16, 5)
    assert e.value.code == C.CRAC_ERR_INVALID_ARG
    with pytest.raises(C.CracError) as e:
        C.crac_ctx_register_alloc(ctx, base + 4096, 16, 3)
    assert e.value.code == C.CRAC_ERR_INVALID_ARG
    C.crac_ctx_register_alloc(ctx, base + 4096, 16, C.CRAC_KIND_HOST)   # page-locked host memory
    C.crac_ctx_free(ctx, base + 4096)
    with pytest.raises(C.CracError) as e:
        C.crac_ctx_free(ctx, base + 4096)
    assert e.value.code == C.CRAC_ERR_UNKNOWN_PTR
    C.crac_ctx_free(ctx, base)
    C.crac_ctx_register_alloc(ctx, base, 100)      # free makes the range available again
    C.crac_ctx_invalidate(ctx)
    C.crac_ctx_destroy(ctx)


def test_null_handles(C):
    lib = ctypes.CDLL(C.LIB_PATH)
    lib.crac_image_release.argtypes = [ctypes.c_void_p]
    assert lib.crac_image_release(None) == C.CRAC_ERR_INVALID_ARG
    lib.crac_ctx_destroy.argtypes = [ctypes.c_void_p]
    assert lib.crac_ctx_destroy(None) == C.CRAC_ERR_INVALID_ARG
    lib.crac_image_deserialize.argtypes = [ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    out = ctypes.c_void_p()
    assert lib.crac_image_deserialize(b"CRACIMG0" + bytes(72), 80, ctypes.byref(out)) == C.CRAC_ERR_CORRUPT
