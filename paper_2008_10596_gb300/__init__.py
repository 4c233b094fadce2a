"""Python binding of libcrac (include/crac.h): argument marshalling only.

Every function here forwards to the C function of the same name in the
in-tree shared library paper_2008_10596_gb300/_lib/libcrac.so.  There is no
fallback: importing this package without the built library raises
ImportError.  Streams may be given as torch.cuda.Stream objects, raw
cudaStream_t integers, or None (the NULL stream: device-wide sync first).
Pointers are integers (e.g. tensor.data_ptr()).
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libcrac.so")
TESTKIT_PATH = os.path.join(_HERE, "_lib", "libcrac_testkit.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libcrac.so is not built ({LIB_PATH}); run "
                      "python -c 'import __graft_entry__ as g; g.build()'")

_lib = ctypes.CDLL(LIB_PATH)

CRAC_OK = 0
CRAC_ERR_INVALID_ARG = -1
CRAC_ERR_UNKNOWN_PTR = -2
CRAC_ERR_OVERLAP = -3
CRAC_ERR_CUDA = -4
CRAC_ERR_OOM = -5
CRAC_ERR_IMAGE_MISMATCH = -6
CRAC_ERR_TIMEOUT = -7
CRAC_ERR_BUSY = -8
CRAC_ERR_UNSUPPORTED = -9
CRAC_ERR_CORRUPT = -10

CRAC_KIND_DEVICE = 0
CRAC_KIND_MANAGED = 1
CRAC_KIND_HOST = 2
CRAC_RESIDENCY_HOST = 0
CRAC_RESIDENCY_DEVICE = 1
CRAC_LAUNCH_BATCHED = 0
CRAC_LAUNCH_PER_ALLOC = 1
CRAC_IMAGE_FULL = 1
CRAC_IMAGE_CODED = 2
CRAC_PASS_AUTO = 0
CRAC_PASS_LDG = 1
CRAC_PASS_TMA = 2
CRAC_PASS_SPLIT = 3
CRAC_PASS_SPARSE = 4
CRAC_FLAG_STAGED_RESTORE = 1
CRAC_FLAG_INCREMENTAL_RESTORE = 2
CRAC_FLAG_DIRECT_DRAIN = 4
CRAC_FLAG_COMPRESS = 8
CRAC_FLAG_WAIT_PASS = 16

CRAC_FAULT_NONE = 0
CRAC_FAULT_PASS = 1
CRAC_FAULT_DRAIN = 2
CRAC_FAULT_H2D = 3
CRAC_FAULT_ALLOC = 4
CRAC_FAULT_DEVICE_WAIT = 5
CRAC_FAULT_ENCODE_WAIT = 6

EXPORTED = [
    "crac_config_default", "crac_ctx_create", "crac_ctx_destroy", "crac_ctx_register_alloc",
    "crac_ctx_free", "crac_ctx_checkpoint", "crac_ctx_restart", "crac_ctx_invalidate", "crac_ctx_drop_history",
    "crac_ctx_last_pass", "crac_register_alloc", "crac_free", "crac_checkpoint", "crac_restart",
    "crac_image_wait", "crac_image_info", "crac_image_serialize", "crac_image_read", "crac_image_deserialize",
    "crac_image_release", "crac_status_str", "crac_last_cuda_error", "crac_kernel_launches",
    "crac_alloc_managed", "crac_free_managed", "crac_debug_inject_fault", "crac_pass_noalloc",
    "crac_ctx_tune_observe", "crac_ctx_tune_apply", "crac_ctx_last_restart", "crac_time_now", "crac_server_create",
    "crac_server_destroy", "crac_server_submit", "crac_server_wait", "crac_server_stats", "crac_memory_stats",
]
CRAC_NOALLOC_MAX_TILES = 32768


class CracConfig(ctypes.Structure):
    _fields_ = [
        ("struct_size", ctypes.c_uint32), ("chunk_bytes", ctypes.c_uint32),
        ("staging_bytes", ctypes.c_uint64), ("lineage", ctypes.c_uint64),
        ("image_residency", ctypes.c_uint32), ("launch_mode", ctypes.c_uint32),
        ("threads", ctypes.c_uint32), ("chunks_per_tile", ctypes.c_uint32),
        ("ctas_per_sm", ctypes.c_uint32), ("warps_per_chunk", ctypes.c_uint32),
        ("timeout_ns", ctypes.c_uint64), ("device", ctypes.c_int32), ("pad0", ctypes.c_uint32),
        ("reserve_host_bytes", ctypes.c_uint64), ("reserve_device_bytes", ctypes.c_uint64),
        ("pass_kernel", ctypes.c_uint32), ("flags", ctypes.c_uint32),
    ]


class CracImageInfo(ctypes.Structure):
    _fields_ = [
        ("lineage", ctypes.c_uint64), ("epoch", ctypes.c_uint64), ("parent_epoch", ctypes.c_uint64),
        ("flags", ctypes.c_uint32), ("chunk_bytes", ctypes.c_uint32), ("n_allocs", ctypes.c_uint64),
        ("n_chunks", ctypes.c_uint64), ("k", ctypes.c_uint64), ("payload_bytes", ctypes.c_uint64),
        ("serialized_bytes", ctypes.c_uint64), ("residency", ctypes.c_uint32),
        ("complete", ctypes.c_uint32), ("raw_bytes", ctypes.c_uint64),
        ("drain_ms", ctypes.c_float), ("reserved", ctypes.c_uint32),
    ]


class CracPassInfo(ctypes.Structure):
    _fields_ = [
        ("tracked_bytes", ctypes.c_uint64), ("n_chunks", ctypes.c_uint64), ("k", ctypes.c_uint64),
        ("payload_bytes", ctypes.c_uint64), ("segments", ctypes.c_uint32),
        ("kernel_launches", ctypes.c_uint32), ("device_ms", ctypes.c_float),
        ("prefetch_ms", ctypes.c_float), ("grid", ctypes.c_uint32),
        ("chunks_per_tile", ctypes.c_uint32), ("warps_per_chunk", ctypes.c_uint32),
        ("hash_ms", ctypes.c_float), ("finalize_ms", ctypes.c_float), ("gather_ms", ctypes.c_float),
        ("pass_kernel", ctypes.c_uint32), ("codec_ms", ctypes.c_float), ("stored_bytes", ctypes.c_uint64),
        ("in_place", ctypes.c_uint64),
    ]


CRAC_TUNE_MAX = 8


class CracRestartInfo(ctypes.Structure):
    _fields_ = [("chain_length", ctypes.c_uint32), ("images_used", ctypes.c_uint32),
                ("restored_bytes", ctypes.c_uint64), ("entries_scanned", ctypes.c_uint64),
                ("h2d_bytes", ctypes.c_uint64), ("scatter_launches", ctypes.c_uint32),
                ("device_ms", ctypes.c_float), ("chunks_rewritten", ctypes.c_uint64),
                ("reserved", ctypes.c_uint32 * 2)]


class CracTuneResult(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_uint32), ("rounds", ctypes.c_uint32), ("chosen_chunk_bytes", ctypes.c_uint32),
        ("chosen_pass_kernel", ctypes.c_uint32), ("chunk_bytes", ctypes.c_uint32 * CRAC_TUNE_MAX),
        ("last_pass_ms", ctypes.c_float * CRAC_TUNE_MAX), ("last_dirty_bytes", ctypes.c_uint64 * CRAC_TUNE_MAX),
        ("mean_pass_ms", ctypes.c_float * CRAC_TUNE_MAX), ("mean_dirty_bytes", ctypes.c_double * CRAC_TUNE_MAX),
        ("cost_ms", ctypes.c_float * CRAC_TUNE_MAX), ("variant_ms", ctypes.c_float * 8),
        ("chosen_chunks_per_tile", ctypes.c_uint32), ("ldg_tiles", ctypes.c_uint32 * 3),
        ("ldg_tile_ms", ctypes.c_float * 3), ("pad0", ctypes.c_uint32),
    ]

    def to_dict(self) -> dict:
        n = self.n
        return {"rounds": self.rounds, "chosen_chunk_bytes": self.chosen_chunk_bytes,
                "chosen_pass_kernel": self.chosen_pass_kernel, "chunk_bytes": list(self.chunk_bytes[:n]),
                "last_pass_ms": list(self.last_pass_ms[:n]), "last_dirty_bytes": list(self.last_dirty_bytes[:n]),
                "mean_pass_ms": list(self.mean_pass_ms[:n]), "mean_dirty_bytes": list(self.mean_dirty_bytes[:n]),
                "cost_ms": list(self.cost_ms[:n]), "variant_ms": list(self.variant_ms[:5]),
                "chosen_chunks_per_tile": self.chosen_chunks_per_tile,
                "ldg_tiles": [t for t in self.ldg_tiles if t],
                "ldg_tile_ms": [m for t, m in zip(self.ldg_tiles, self.ldg_tile_ms) if t]}


class CracServerConfig(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("workers", ctypes.c_uint32),
                ("staging_budget", ctypes.c_uint64), ("max_lease", ctypes.c_uint64),
                ("device", ctypes.c_int32), ("reserved", ctypes.c_uint32 * 5)]


class CracRequestResult(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("status", ctypes.c_int32), ("type", ctypes.c_uint32),
                ("image", ctypes.c_void_p), ("t_arrival", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("tracked_bytes", ctypes.c_uint64),
                ("payload_bytes", ctypes.c_uint64), ("lease_bytes", ctypes.c_uint64),
                ("t_op", ctypes.c_double), ("t_op_end", ctypes.c_double)]


class CracServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("queued", ctypes.c_uint32),
                ("in_flight", ctypes.c_uint32), ("max_in_flight", ctypes.c_uint32), ("pad", ctypes.c_uint32),
                ("staging_used", ctypes.c_uint64), ("staging_high_water", ctypes.c_uint64),
                ("staging_budget", ctypes.c_uint64)]


class CracMemoryStats(ctypes.Structure):
    _fields_ = [("host_region_bytes", ctypes.c_uint64), ("host_used_bytes", ctypes.c_uint64),
                ("device_region_bytes", ctypes.c_uint64), ("device_used_bytes", ctypes.c_uint64),
                ("host_regions", ctypes.c_uint32), ("device_regions", ctypes.c_uint32),
                ("host_grow_events", ctypes.c_uint32), ("device_grow_events", ctypes.c_uint32),
                ("scratch_grow_events", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


CRAC_REQ_CHECKPOINT = 0
CRAC_REQ_RESTART = 1
PREPARE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_vp = ctypes.c_void_p
_st = ctypes.c_int
_sigs = {
    "crac_config_default": (None, [ctypes.POINTER(CracConfig)]),
    "crac_ctx_create": (_st, [ctypes.POINTER(CracConfig), ctypes.POINTER(_vp)]),
    "crac_ctx_destroy": (_st, [_vp]),
    "crac_ctx_register_alloc": (_st, [_vp, _vp, ctypes.c_size_t, ctypes.c_int]),
    "crac_ctx_free": (_st, [_vp, _vp]),
    "crac_ctx_checkpoint": (_st, [_vp, _vp, ctypes.POINTER(_vp)]),
    "crac_ctx_restart": (_st, [_vp, _vp, _vp]),
    "crac_ctx_invalidate": (_st, [_vp]),
    "crac_ctx_drop_history": (_st, [_vp]),
    "crac_ctx_last_pass": (_st, [_vp, ctypes.POINTER(CracPassInfo)]),
    "crac_register_alloc": (_st, [_vp, ctypes.c_size_t, ctypes.c_int]),
    "crac_free": (_st, [_vp]),
    "crac_checkpoint": (_st, [_vp, ctypes.POINTER(_vp)]),
    "crac_restart": (_st, [_vp, _vp]),
    "crac_image_wait": (_st, [_vp, ctypes.c_uint64]),
    "crac_image_info": (_st, [_vp, ctypes.POINTER(CracImageInfo)]),
    "crac_image_serialize": (_st, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "crac_image_read": (_st, [_vp, ctypes.c_uint64, _vp, ctypes.c_size_t]),
    "crac_image_deserialize": (_st, [_vp, ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "crac_image_release": (_st, [_vp]),
    "crac_status_str": (ctypes.c_char_p, [_st]),
    "crac_last_cuda_error": (ctypes.c_int, []),
    "crac_kernel_launches": (ctypes.c_uint64, []),
    "crac_alloc_managed": (_st, [ctypes.c_size_t, ctypes.POINTER(_vp)]),
    "crac_free_managed": (_st, [_vp]),
    "crac_debug_inject_fault": (None, [ctypes.c_int, ctypes.c_int]),
    "crac_ctx_tune_observe": (_st, [_vp, _vp, ctypes.POINTER(ctypes.c_uint32), ctypes.c_uint32,
                                    ctypes.POINTER(CracTuneResult)]),
    "crac_ctx_tune_apply": (_st, [_vp, _vp, ctypes.c_double, ctypes.POINTER(CracTuneResult)]),
    "crac_ctx_last_restart": (_st, [_vp, ctypes.POINTER(CracRestartInfo)]),
    "crac_time_now": (ctypes.c_double, []),
    "crac_memory_stats": (_st, [ctypes.POINTER(CracMemoryStats)]),
    "crac_server_create": (_st, [ctypes.POINTER(CracServerConfig), ctypes.POINTER(_vp)]),
    "crac_server_destroy": (_st, [_vp]),
    "crac_server_submit": (_st, [_vp, _vp, ctypes.c_uint32, _vp, _vp, PREPARE_FN, _vp, ctypes.c_double,
                                 ctypes.POINTER(ctypes.c_uint64)]),
    "crac_server_wait": (_st, [_vp, ctypes.c_uint64, ctypes.c_uint64, ctypes.POINTER(CracRequestResult)]),
    "crac_server_stats": (_st, [_vp, ctypes.POINTER(CracServerStats)]),
    "crac_pass_noalloc": (_st, [_vp, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32, _vp, _vp, _vp, _vp,
                                ctypes.c_uint64, _vp, ctypes.c_uint64, _vp, _vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class CracError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.crac_status_str(code).decode()
        if code == CRAC_ERR_CUDA:
            msg += f" (cudaError {_lib.crac_last_cuda_error()})"
        super().__init__(f"{where}: {msg}")


def _check(st: int, where: str) -> None:
    if st != CRAC_OK:
        raise CracError(st, where)


def _stream(s) -> int | None:
    if s is None:
        return None
    if hasattr(s, "cuda_stream"):
        return s.cuda_stream or None
    return int(s) or None


def _ptr(p) -> int:
    return p.data_ptr() if hasattr(p, "data_ptr") else int(p)


# ---- configuration and contexts --------------------------------------------

def crac_config_default(**overrides) -> CracConfig:
    cfg = CracConfig()
    _lib.crac_config_default(ctypes.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def crac_ctx_create(cfg: CracConfig | None = None) -> int:
    h = _vp()
    _check(_lib.crac_ctx_create(ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
           "crac_ctx_create")
    return h.value


def crac_ctx_destroy(ctx: int) -> None:
    _check(_lib.crac_ctx_destroy(ctx), "crac_ctx_destroy")


def crac_ctx_register_alloc(ctx: int, ptr, nbytes: int, kind: int = CRAC_KIND_DEVICE) -> None:
    _check(_lib.crac_ctx_register_alloc(ctx, _ptr(ptr), nbytes, kind), "crac_ctx_register_alloc")


def crac_ctx_free(ctx: int, ptr) -> None:
    _check(_lib.crac_ctx_free(ctx, _ptr(ptr)), "crac_ctx_free")


def crac_ctx_checkpoint(ctx: int, stream=None) -> int:
    h = _vp()
    _check(_lib.crac_ctx_checkpoint(ctx, _stream(stream), ctypes.byref(h)), "crac_ctx_checkpoint")
    return h.value


def crac_ctx_restart(ctx: int, image: int, stream=None) -> None:
    _check(_lib.crac_ctx_restart(ctx, image, _stream(stream)), "crac_ctx_restart")


def crac_ctx_tune_observe(ctx: int, chunk_sizes, stream=None) -> dict:
    arr = (ctypes.c_uint32 * len(chunk_sizes))(*chunk_sizes)
    out = CracTuneResult()
    _check(_lib.crac_ctx_tune_observe(ctx, _stream(stream), arr, len(chunk_sizes), ctypes.byref(out)),
           "crac_ctx_tune_observe")
    return out.to_dict()


def crac_ctx_tune_apply(ctx: int, link_gbs: float = 0.0, stream=None) -> dict:
    out = CracTuneResult()
    _check(_lib.crac_ctx_tune_apply(ctx, _stream(stream), link_gbs, ctypes.byref(out)), "crac_ctx_tune_apply")
    return out.to_dict()


def crac_ctx_last_restart(ctx: int, out: "CracRestartInfo | None" = None):
    """The last restart's statistics as a dict; given `out`, fills it and
    returns it unconverted."""
    info = CracRestartInfo() if out is None else out
    _check(_lib.crac_ctx_last_restart(ctx, ctypes.byref(info)), "crac_ctx_last_restart")
    return info if out is not None else restart_info_dict(info)


def restart_info_dict(info: "CracRestartInfo") -> dict:
    return {f: getattr(info, f) for f, _ in CracRestartInfo._fields_ if f != "reserved"}


def crac_memory_stats() -> dict:
    st = CracMemoryStats()
    _check(_lib.crac_memory_stats(ctypes.byref(st)), "crac_memory_stats")
    return {f: getattr(st, f) for f, _ in CracMemoryStats._fields_}


def crac_time_now() -> float:
    return _lib.crac_time_now()


def crac_server_create(workers: int = 0, staging_budget: int = 0, max_lease: int = 0, device: int = -1) -> int:
    cfg = CracServerConfig(ctypes.sizeof(CracServerConfig), workers, staging_budget, max_lease, device)
    h = _vp()
    _check(_lib.crac_server_create(ctypes.byref(cfg), ctypes.byref(h)), "crac_server_create")
    return h.value


def crac_server_destroy(server: int) -> None:
    _check(_lib.crac_server_destroy(server), "crac_server_destroy")


_NO_PREPARE = PREPARE_FN()


def crac_server_submit(server: int, ctx: int, type_: int, image: int | None = None, stream=None,
                       prepare=None, prepare_arg: int | None = None, t_arrival: float = 0.0) -> int:
    """prepare: a PREPARE_FN instance (keep it alive until the request completes)."""
    t = ctypes.c_uint64()
    _check(_lib.crac_server_submit(server, ctx, type_, image, _stream(stream),
                                   prepare if prepare is not None else _NO_PREPARE, prepare_arg,
                                   t_arrival, ctypes.byref(t)), "crac_server_submit")
    return t.value


def crac_server_wait(server: int, ticket: int, timeout_ns: int = 0) -> dict:
    r = CracRequestResult()
    _check(_lib.crac_server_wait(server, ticket, timeout_ns, ctypes.byref(r)), "crac_server_wait")
    return {f: getattr(r, f) for f, _ in CracRequestResult._fields_}


def crac_server_stats(server: int) -> dict:
    st = CracServerStats()
    _check(_lib.crac_server_stats(server, ctypes.byref(st)), "crac_server_stats")
    return {f: getattr(st, f) for f, _ in CracServerStats._fields_ if f != "pad"}


def crac_ctx_invalidate(ctx: int) -> None:
    _check(_lib.crac_ctx_invalidate(ctx), "crac_ctx_invalidate")


def crac_ctx_drop_history(ctx: int) -> None:
    _check(_lib.crac_ctx_drop_history(ctx), "crac_ctx_drop_history")


def crac_ctx_last_pass(ctx: int, out: "CracPassInfo | None" = None):
    """The last pass's statistics as a dict; given `out` (a CracPassInfo), fills
    it and returns it unconverted (no per-field Python work, for timed loops)."""
    info = CracPassInfo() if out is None else out
    _check(_lib.crac_ctx_last_pass(ctx, ctypes.byref(info)), "crac_ctx_last_pass")
    return info if out is not None else pass_info_dict(info)


def pass_info_dict(info: "CracPassInfo") -> dict:
    return {f: getattr(info, f) for f, _ in CracPassInfo._fields_ if f != "reserved"}


# ---- default-context forms ---------------------------------------------------

def crac_register_alloc(ptr, nbytes: int, kind: int = CRAC_KIND_DEVICE) -> None:
    _check(_lib.crac_register_alloc(_ptr(ptr), nbytes, kind), "crac_register_alloc")


def crac_free(ptr) -> None:
    _check(_lib.crac_free(_ptr(ptr)), "crac_free")


def crac_checkpoint(stream=None) -> int:
    h = _vp()
    _check(_lib.crac_checkpoint(_stream(stream), ctypes.byref(h)), "crac_checkpoint")
    return h.value


def crac_restart(image: int, stream=None) -> None:
    _check(_lib.crac_restart(image, _stream(stream)), "crac_restart")


# ---- images -----------------------------------------------------------------

def crac_image_wait(image: int, timeout_ns: int = 0) -> None:
    _check(_lib.crac_image_wait(image, timeout_ns), "crac_image_wait")


def crac_image_info(image: int) -> dict:
    info = CracImageInfo()
    _check(_lib.crac_image_info(image, ctypes.byref(info)), "crac_image_info")
    return {f: getattr(info, f) for f, _ in CracImageInfo._fields_}


def crac_image_serialize(image: int) -> bytes:
    need = ctypes.c_size_t()
    _check(_lib.crac_image_serialize(image, None, 0, ctypes.byref(need)), "crac_image_serialize")
    buf = ctypes.create_string_buffer(need.value)
    _check(_lib.crac_image_serialize(image, buf, need.value, ctypes.byref(need)), "crac_image_serialize")
    return buf.raw


def crac_image_read(image: int, offset: int, n: int, out=None):
    """Bytes [offset, offset + n) of the serialized image.  With `out` (a
    writable buffer of n bytes: bytearray, numpy array) fills it and returns
    it; else returns bytes."""
    if out is None:
        buf = ctypes.create_string_buffer(max(n, 1))
        _check(_lib.crac_image_read(image, offset, buf, n), "crac_image_read")
        return buf.raw[:n]
    mv = memoryview(out).cast("B")
    if mv.nbytes != n or mv.readonly:
        raise ValueError("out must be a writable buffer of n bytes")
    addr = ctypes.addressof(ctypes.c_char.from_buffer(mv)) if n else None
    _check(_lib.crac_image_read(image, offset, addr, n), "crac_image_read")
    return out


def crac_image_deserialize(data: bytes) -> int:
    h = _vp()
    b = ctypes.create_string_buffer(bytes(data), len(data))
    _check(_lib.crac_image_deserialize(b, len(data), ctypes.byref(h)), "crac_image_deserialize")
    return h.value


def crac_image_release(image: int) -> None:
    _check(_lib.crac_image_release(image), "crac_image_release")


# ---- diagnostics ---------------------------------------------------------------

def crac_status_str(code: int) -> str:
    return _lib.crac_status_str(code).decode()


def crac_last_cuda_error() -> int:
    return _lib.crac_last_cuda_error()


def crac_kernel_launches() -> int:
    return _lib.crac_kernel_launches()


def crac_alloc_managed(nbytes: int) -> int:
    h = _vp()
    _check(_lib.crac_alloc_managed(nbytes, ctypes.byref(h)), "crac_alloc_managed")
    return h.value


def crac_free_managed(ptr: int) -> None:
    _check(_lib.crac_free_managed(ptr), "crac_free_managed")


def crac_debug_inject_fault(step: int, count: int = 1) -> None:
    _lib.crac_debug_inject_fault(step, count)


def crac_pass_noalloc(regions_dev, n_regions: int, n_chunks: int, chunk_bytes: int, fp_old_dev,
                      fp_new_dev, idx_dev, off_dev, idx_cap: int, staging_dev, staging_cap: int,
                      totals_dev, stream=None) -> None:
    """The checkpoint pass over caller-owned device buffers, allocating nothing.

    For callers that cannot allocate device memory at the moment they need a
    checkpoint (inside an interposed cudaMalloc/cudaFree or allocator hook, at
    preemption time, or when the allocator is exhausted).  regions_dev holds
    n_regions x {u64 ptr, u64 bytes, u64 first_chunk, u64 base_first}; results
    go to the output buffers and totals_dev = {u32 0, u32 err, u64 k, u64 bytes}.
    Calls share one fixed scratch area, so calls that overlap on the GPU race.
    """
    _check(_lib.crac_pass_noalloc(_ptr(regions_dev), n_regions, n_chunks, chunk_bytes,
                                  _ptr(fp_old_dev) if fp_old_dev is not None else None, _ptr(fp_new_dev),
                                  _ptr(idx_dev), _ptr(off_dev), idx_cap,
                                  _ptr(staging_dev) if staging_dev is not None else None, staging_cap,
                                  _ptr(totals_dev), _stream(stream)), "crac_pass_noalloc")
