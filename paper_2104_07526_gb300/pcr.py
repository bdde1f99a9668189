"""Python binding of libpcr.so (include/pcr.h).

Argument marshalling only: every function here has the name of a C entry
point, turns tensors into device pointers, calls the library and raises
PcrError on a non-zero status.  All rendering work runs in the library's CUDA
kernels; there is no Python or CPU fallback.  If the library has not been
built, loading it raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libpcr.so")

PCR_OK, PCR_ERR_ARG, PCR_ERR_CUDA, PCR_ERR_WORKSPACE, PCR_ERR_TIMEOUT, PCR_ERR_UNSUPPORTED = 0, -1, -2, -3, -4, -5
PCR_ERR_BUSY = -6
PCR_SERVE_ARRIVAL, PCR_SERVE_LARGEST_GROUP = 0, 1

PCR_VARIANT_ATOMICMIN = 0
PCR_VARIANT_EARLYZ = 1
PCR_VARIANT_DEDUP = 2
PCR_VARIANT_DEDUP_EARLYZ = 3
PCR_VARIANT_REDUCE = 4
PCR_VARIANT_REDUCE_EARLYZ = 5
PCR_VARIANT_JUST_SET = 6
PCR_VARIANT_BUSY_LOOP = 7
EXACT_VARIANTS = (0, 1, 2, 3, 4, 5)
VARIANT_NAMES = {0: "atomicMin", 1: "early-z", 2: "dedup", 3: "dedup+early-z", 4: "reduce",
                 5: "reduce+early-z", 6: "just-set", 7: "busy-loop"}

PCR_RESOLVE_BASIC = 0
PCR_RESOLVE_HQ = 1
PCR_RESOLVE_HQ1R = 2
PCR_RESOLVE_RGB = 3

PCR_CLEAR_KEYS = 1
PCR_CLEAR_HQ = 2

PCR_BATCH_BASIC = 1
PCR_BATCH_HQ = 2
PCR_BATCH_MAX_CLOUDS = 256
PCR_BATCH_MAX_VIEWS = 256

PCR_ORDER_MORTON = 0
PCR_ORDER_MORTON_SHUFFLE128 = 1
PCR_ORDER_SHUFFLE = 2
PCR_ORDER_MORTON63 = 3
PCR_ORDER_MORTON63_SHUFFLE128 = 4

PCR_DEVICE_ERROR_KEY_RANGE = 1
PCR_DEVICE_ERROR_WAIT_TIMEOUT = 2
PCR_DEVICE_ERROR_BOUNDS = 4


class PcrBatchCloud(C.Structure):
    """pcr_batch_cloud"""
    _fields_ = [("points", C.c_void_p), ("n", C.c_uint64)]


class PcrBatchView(C.Structure):
    """pcr_batch_view"""
    _fields_ = [("matrix", C.c_float * 16), ("width", C.c_int32), ("height", C.c_int32), ("cloud", C.c_uint32),
                ("flags", C.c_uint32), ("keys", C.c_void_p), ("image", C.c_void_p), ("hq_depth", C.c_void_p),
                ("hq_rg", C.c_void_p), ("hq_ba", C.c_void_p), ("hq_image", C.c_void_p)]


class PcrBatchTuning(C.Structure):
    """pcr_batch_tuning"""
    _fields_ = [("l2_budget_mb", C.c_uint32), ("config", C.c_int32), ("threads", C.c_uint32),
                ("unroll1", C.c_uint32), ("unroll2", C.c_uint32), ("from_cache", C.c_uint32), ("tried", C.c_uint32),
                ("single_colors", C.c_uint32), ("best_ms", C.c_double), ("default_ms", C.c_double)]


class PcrServerConfig(C.Structure):
    """pcr_server_config"""
    _fields_ = [("dev_arena", C.c_void_p), ("arena_bytes", C.c_uint64), ("max_width", C.c_uint32),
                ("max_height", C.c_uint32), ("num_slots", C.c_uint32), ("max_batch_views", C.c_uint32),
                ("max_inflight", C.c_uint32), ("streams", C.c_uint32), ("max_batch_clouds", C.c_uint32),
                ("batch_config", C.c_int32), ("depth_factor", C.c_float), ("background_rgba", C.c_uint32),
                ("max_queue", C.c_uint32), ("deadline_us", C.c_uint32), ("policy", C.c_uint32),
                ("l2_budget_mb", C.c_uint32)]


class PcrRequest(C.Structure):
    """pcr_request"""
    _fields_ = [("cloud_id", C.c_uint32), ("matrix", C.c_float * 16), ("width", C.c_int32), ("height", C.c_int32),
                ("flags", C.c_uint32)]


class PcrServerResult(C.Structure):
    """pcr_server_result"""
    _fields_ = [("width", C.c_int32), ("height", C.c_int32), ("flags", C.c_uint32), ("pad", C.c_uint32),
                ("keys", C.c_void_p), ("image", C.c_void_p), ("hq_depth", C.c_void_p), ("hq_rg", C.c_void_p),
                ("hq_ba", C.c_void_p), ("hq_image", C.c_void_p), ("submit_us", C.c_double),
                ("launch_us", C.c_double), ("done_us", C.c_double), ("points", C.c_uint64)]


class PcrServerStats(C.Structure):
    """pcr_server_stats"""
    _fields_ = [(k, C.c_uint64) for k in ("submitted", "completed", "batches", "views_launched", "uploads",
                                          "evictions", "bytes_uploaded", "points_rendered", "peak_queue", "queued",
                                          "resident_clouds", "resident_bytes", "rejected", "expired",
                                          "cancelled")]


PCR_REQUEST_QUEUED, PCR_REQUEST_RUNNING, PCR_REQUEST_DONE, PCR_REQUEST_EXPIRED, PCR_REQUEST_CANCELLED = 0, 1, 2, 3, 4


class PcrError(RuntimeError):
    def __init__(self, status: int, call: str):
        self.status = status
        super().__init__(f"{call} failed: {pcr_status_string(status)} ({status})")


_lock = threading.Lock()
_lib = None

_VP, _U64, _U32, _INT, _FLT = C.c_void_p, C.c_uint64, C.c_uint32, C.c_int, C.c_float
_SIGS = {
    "pcr_create": [C.POINTER(_VP), _INT],
    "pcr_destroy": [_VP],
    "pcr_set_stream": [_VP, _VP],
    "pcr_upload_points": [_VP, _VP, _U64],
    "pcr_upload_points_from_host": [_VP, _VP, _VP, _U64],
    "pcr_upload_points_mapped": [_VP, _VP, _U64],
    "pcr_set_matrix": [_VP, C.POINTER(_FLT)],
    "pcr_set_viewport": [_VP, _INT, _INT],
    "pcr_set_framebuffer": [_VP, _VP, _VP, _VP, _VP],
    "pcr_clear": [_VP, _INT],
    "pcr_render_basic": [_VP, _INT, _INT],
    "pcr_render_rgb": [_VP, _INT, _INT],
    "pcr_set_lock_buffer": [_VP, _VP, _U32],
    "pcr_render_hq": [_VP, _FLT, _INT, _INT],
    "pcr_resolve": [_VP, _INT, _VP, _U32],
    "pcr_set_hq1r_buffer": [_VP, _VP],
    "pcr_render_hq1r": [_VP, _FLT, _INT, _INT],
    "pcr_download": [_VP, _VP, _VP, _U64],
    "pcr_synchronize": [_VP],
    "pcr_reorder_workspace_size": [_U64, C.POINTER(_U64)],
    "pcr_reorder_morton_shuffle128": [_VP, _VP, _U64, _U64, _INT, _VP, _U64, _VP],
    "pcr_reorder_morton_shuffle128_noalloc": [_VP, _VP, _U64, _U64, _INT, _VP],
    "pcr_last_device_error": [_VP, C.POINTER(_U32)],
    "pcr_check_division": [_VP, _U32, _U32, _VP, _U32, _U32, _U32, _FLT, C.POINTER(_U64)],
    "pcr_debug_counters": [_VP, C.POINTER(_U64)],
    "pcr_batch_workspace_size": [C.POINTER(_U64)],
    "pcr_batch_num_configs": [C.POINTER(_INT)],
    "pcr_batch_prepare": [_VP, C.POINTER(PcrBatchCloud), _U32, C.POINTER(PcrBatchView), _U32, _FLT, _U32, _VP, _U64],
    "pcr_batch_launch": [_VP, _VP, _INT],
    "pcr_batch_autotune": [_VP, _VP, C.POINTER(_INT)],
    "pcr_batch_tune": [_VP, C.POINTER(PcrBatchCloud), _U32, C.POINTER(PcrBatchView), _U32, _FLT, _U32, _VP, _U64,
                       C.c_char_p, C.POINTER(PcrBatchTuning)],
    "pcr_batch_capture": [_VP, _VP, _INT, C.POINTER(_VP)],
    "pcr_batch_launch_count": [_VP, _VP, _INT, C.POINTER(_INT)],
    "pcr_capture_begin": [_VP],
    "pcr_capture_end": [_VP, C.POINTER(_VP)],
    "pcr_graph_launch": [_VP, _VP],
    "pcr_graph_destroy": [_VP],
    "pcr_server_create": [_VP, C.POINTER(PcrServerConfig), C.POINTER(_VP)],
    "pcr_server_destroy": [_VP],
    "pcr_server_add_cloud": [_VP, _U32, _VP, _U64],
    "pcr_server_add_device_cloud": [_VP, _U32, _VP, _U64],
    "pcr_server_submit": [_VP, C.POINTER(PcrRequest), C.POINTER(_U64)],
    "pcr_server_step": [_VP, C.POINTER(_U32)],
    "pcr_server_state": [_VP, _U64, C.POINTER(_INT)],
    "pcr_server_get_result": [_VP, _U64, C.POINTER(PcrServerResult)],
    "pcr_server_release": [_VP, _U64],
    "pcr_server_poll_completed": [_VP, C.POINTER(_U64), _U32, C.POINTER(_U32)],
    "pcr_server_stats_get": [_VP, C.POINTER(PcrServerStats)],
    "pcr_server_cancel": [_VP, _U64],
}


DEBUG_LIB_PATH = os.path.join(HERE, "libpcr_debug.so")


def load_library(path: str) -> C.CDLL:
    """Load a build of the library (libpcr.so or libpcr_debug.so) with the
    C signatures set; raises if it has not been built."""
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2104_07526_gb300.build.build()")
    L = C.CDLL(path)
    for name, args in _SIGS.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = _INT
    L.pcr_status_string.argtypes = [_INT]
    L.pcr_status_string.restype = C.c_char_p
    return L


def lib() -> C.CDLL:
    """Load libpcr.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(LIB_PATH)
    return _lib


def _check(status: int, call: str):
    if status != PCR_OK:
        raise PcrError(status, call)


def _dptr(t, what: str) -> int | None:
    """Device address of a CUDA tensor (None passes NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    return t.data_ptr()


def _hptr(a, what: str) -> int:
    """Host address of a CPU tensor or numpy array."""
    if hasattr(a, "data_ptr"):
        if a.is_cuda:
            raise ValueError(f"{what} must be in host memory")
        if not a.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        return a.data_ptr()
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError(f"{what} must be contiguous")
    return a.ctypes.data


def _nbytes(t) -> int:
    return t.numel() * t.element_size() if hasattr(t, "element_size") else t.nbytes


def pcr_status_string(status: int) -> str:
    return lib().pcr_status_string(status).decode()


def pcr_create(device: int = 0) -> int:
    h = _VP()
    _check(lib().pcr_create(C.byref(h), device), "pcr_create")
    return h.value


def pcr_destroy(ctx: int):
    _check(lib().pcr_destroy(ctx), "pcr_destroy")


def pcr_set_stream(ctx: int, stream=None):
    """stream: a torch.cuda.Stream, a raw cudaStream_t address, or None."""
    handle = getattr(stream, "cuda_stream", stream)
    _check(lib().pcr_set_stream(ctx, handle), "pcr_set_stream")


def pcr_upload_points(ctx: int, points, n: int | None = None):
    if n is None:
        n = _nbytes(points) // 16
    _check(lib().pcr_upload_points(ctx, _dptr(points, "points"), n), "pcr_upload_points")


def pcr_upload_points_from_host(ctx: int, dev_points, host_points, n: int | None = None):
    if n is None:
        n = _nbytes(host_points) // 16
    _check(lib().pcr_upload_points_from_host(ctx, _dptr(dev_points, "dev_points"),
                                             _hptr(host_points, "host_points"), n), "pcr_upload_points_from_host")


def pcr_upload_points_mapped(ctx: int, host_points, n: int | None = None):
    """host_points: a pinned CPU tensor (e.g. torch.empty(..., pin_memory=True))."""
    if n is None:
        n = _nbytes(host_points) // 16
    _check(lib().pcr_upload_points_mapped(ctx, _hptr(host_points, "host_points"), n), "pcr_upload_points_mapped")


def pcr_set_matrix(ctx: int, m):
    vals = [float(v) for v in (m.reshape(-1).tolist() if hasattr(m, "reshape") else m)]
    if len(vals) != 16:
        raise ValueError("matrix must have 16 entries")
    arr = (_FLT * 16)(*vals)
    _check(lib().pcr_set_matrix(ctx, arr), "pcr_set_matrix")


def pcr_set_viewport(ctx: int, width: int, height: int):
    _check(lib().pcr_set_viewport(ctx, width, height), "pcr_set_viewport")


def pcr_set_framebuffer(ctx: int, keys=None, hq_depth=None, hq_rg=None, hq_ba=None):
    _check(lib().pcr_set_framebuffer(ctx, _dptr(keys, "keys"), _dptr(hq_depth, "hq_depth"), _dptr(hq_rg, "hq_rg"),
                                     _dptr(hq_ba, "hq_ba")), "pcr_set_framebuffer")


def pcr_clear(ctx: int, what: int = PCR_CLEAR_KEYS):
    _check(lib().pcr_clear(ctx, what), "pcr_clear")


def pcr_render_basic(ctx: int, variant: int = PCR_VARIANT_DEDUP_EARLYZ, clear: bool = True):
    _check(lib().pcr_render_basic(ctx, variant, int(bool(clear))), "pcr_render_basic")


def pcr_render_hq(ctx: int, depth_factor: float = 1.01, variant: int = PCR_VARIANT_DEDUP_EARLYZ, clear: bool = True):
    _check(lib().pcr_render_hq(ctx, depth_factor, variant, int(bool(clear))), "pcr_render_hq")


def pcr_render_rgb(ctx: int, variant: int = PCR_VARIANT_DEDUP_EARLYZ, clear: bool = True):
    _check(lib().pcr_render_rgb(ctx, variant, int(bool(clear))), "pcr_render_rgb")


def pcr_set_lock_buffer(ctx: int, locks=None, wait_limit_us: int = 0):
    _check(lib().pcr_set_lock_buffer(ctx, _dptr(locks, "locks"), wait_limit_us), "pcr_set_lock_buffer")


def pcr_set_hq1r_buffer(ctx: int, primary=None):
    _check(lib().pcr_set_hq1r_buffer(ctx, _dptr(primary, "primary")), "pcr_set_hq1r_buffer")


def pcr_render_hq1r(ctx: int, depth_factor: float = 1.01, variant: int = PCR_VARIANT_DEDUP_EARLYZ,
                    clear: bool = True):
    _check(lib().pcr_render_hq1r(ctx, depth_factor, variant, int(bool(clear))), "pcr_render_hq1r")


def pcr_resolve(ctx: int, mode: int, out, background_rgba: int = 0):
    _check(lib().pcr_resolve(ctx, mode, _dptr(out, "out"), background_rgba & 0xFFFFFFFF), "pcr_resolve")


def pcr_download(ctx: int, host_dst, dev_src, nbytes: int | None = None):
    if nbytes is None:
        nbytes = _nbytes(dev_src)
    _check(lib().pcr_download(ctx, _hptr(host_dst, "host_dst"), _dptr(dev_src, "dev_src"), nbytes), "pcr_download")


def pcr_synchronize(ctx: int):
    _check(lib().pcr_synchronize(ctx), "pcr_synchronize")


def pcr_reorder_workspace_size(n: int) -> int:
    out = _U64()
    _check(lib().pcr_reorder_workspace_size(n, C.byref(out)), "pcr_reorder_workspace_size")
    return out.value


def pcr_reorder_morton_shuffle128(ctx: int, points, n: int, seed: int, mode: int, workspace, perm_out=None):
    _check(lib().pcr_reorder_morton_shuffle128(ctx, _dptr(points, "points"), n, seed & ((1 << 64) - 1), mode,
                                               _dptr(workspace, "workspace"),
                                               _nbytes(workspace) if workspace is not None else 0,
                                               _dptr(perm_out, "perm_out")), "pcr_reorder_morton_shuffle128")


PCR_REORDER_NOALLOC_MAX_POINTS = 262144


def pcr_reorder_morton_shuffle128_noalloc(ctx: int, points, n: int, seed: int, mode: int, perm_out=None):
    """Reorder without a workspace (the library's fixed scratch array; at
    most PCR_REORDER_NOALLOC_MAX_POINTS points; calls on one device must not
    overlap on the GPU)."""
    _check(lib().pcr_reorder_morton_shuffle128_noalloc(ctx, _dptr(points, "points"), n, seed & ((1 << 64) - 1), mode,
                                                       _dptr(perm_out, "perm_out")),
           "pcr_reorder_morton_shuffle128_noalloc")


def batch_cloud(points, n: int | None = None) -> PcrBatchCloud:
    """pcr_batch_cloud for a CUDA tensor of 16-byte records (None: empty)."""
    if points is None:
        return PcrBatchCloud(None, 0)
    return PcrBatchCloud(_dptr(points, "points"), n if n is not None else _nbytes(points) // 16)


def batch_view(matrix, width: int, height: int, cloud: int, flags: int, keys=None, image=None, hq_depth=None,
               hq_rg=None, hq_ba=None, hq_image=None) -> PcrBatchView:
    vals = [float(v) for v in (matrix.reshape(-1).tolist() if hasattr(matrix, "reshape") else matrix)]
    return PcrBatchView((C.c_float * 16)(*vals), width, height, cloud, flags, _dptr(keys, "keys"),
                        _dptr(image, "image"), _dptr(hq_depth, "hq_depth"), _dptr(hq_rg, "hq_rg"),
                        _dptr(hq_ba, "hq_ba"), _dptr(hq_image, "hq_image"))


def pcr_batch_workspace_size() -> int:
    out = _U64()
    _check(lib().pcr_batch_workspace_size(C.byref(out)), "pcr_batch_workspace_size")
    return out.value


def pcr_batch_num_configs() -> int:
    out = _INT()
    _check(lib().pcr_batch_num_configs(C.byref(out)), "pcr_batch_num_configs")
    return out.value


def pcr_batch_prepare(ctx: int, clouds, views, depth_factor: float, background_rgba: int, workspace):
    ca = (PcrBatchCloud * len(clouds))(*clouds)
    va = (PcrBatchView * len(views))(*views)
    _check(lib().pcr_batch_prepare(ctx, ca, len(clouds), va, len(views), depth_factor, background_rgba & 0xFFFFFFFF,
                                   _dptr(workspace, "workspace"), _nbytes(workspace) if workspace is not None else 0),
           "pcr_batch_prepare")


def pcr_batch_launch(ctx: int, workspace, config: int = 0):
    _check(lib().pcr_batch_launch(ctx, _dptr(workspace, "workspace"), config), "pcr_batch_launch")


def pcr_batch_autotune(ctx: int, workspace) -> int:
    out = _INT()
    _check(lib().pcr_batch_autotune(ctx, _dptr(workspace, "workspace"), C.byref(out)), "pcr_batch_autotune")
    return out.value


def pcr_batch_tune(ctx: int, clouds, views, depth_factor: float, background_rgba: int, workspace,
                   cache_path: str | None = None) -> dict:
    """Prepare the batch with its tuned L2 budget and pick its launch
    configuration (see pcr.h); returns the pcr_batch_tuning fields."""
    ca = (PcrBatchCloud * len(clouds))(*clouds)
    va = (PcrBatchView * len(views))(*views)
    out = PcrBatchTuning()
    _check(lib().pcr_batch_tune(ctx, ca, len(clouds), va, len(views), depth_factor, background_rgba & 0xFFFFFFFF,
                                _dptr(workspace, "workspace"), _nbytes(workspace) if workspace is not None else 0,
                                cache_path.encode() if cache_path else None, C.byref(out)), "pcr_batch_tune")
    return {k: getattr(out, k) for k, _ in PcrBatchTuning._fields_}


def pcr_batch_launch_count(ctx: int, workspace, config: int) -> int:
    out = _INT()
    _check(lib().pcr_batch_launch_count(ctx, _dptr(workspace, "workspace"), config, C.byref(out)),
           "pcr_batch_launch_count")
    return out.value


def pcr_batch_capture(ctx: int, workspace, config: int) -> int:
    out = _VP()
    _check(lib().pcr_batch_capture(ctx, _dptr(workspace, "workspace"), config, C.byref(out)), "pcr_batch_capture")
    return out.value


def pcr_capture_begin(ctx: int):
    _check(lib().pcr_capture_begin(ctx), "pcr_capture_begin")


def pcr_capture_end(ctx: int) -> int:
    out = _VP()
    _check(lib().pcr_capture_end(ctx, C.byref(out)), "pcr_capture_end")
    return out.value


def pcr_graph_launch(ctx: int, graph_exec: int):
    _check(lib().pcr_graph_launch(ctx, graph_exec), "pcr_graph_launch")


def pcr_graph_destroy(graph_exec: int):
    _check(lib().pcr_graph_destroy(graph_exec), "pcr_graph_destroy")


def pcr_server_create(ctx: int, arena, max_width: int, max_height: int, num_slots: int, max_batch_views: int = 64,
                      max_inflight: int = 2, streams: int = 0, max_batch_clouds: int = 0, batch_config: int = 0,
                      depth_factor: float = 1.01, background_rgba: int = 0, max_queue: int = 0,
                      deadline_us: int = 0, policy: int = PCR_SERVE_ARRIVAL, l2_budget_mb: int = 0) -> int:
    """arena: CUDA uint8 tensor (the server's device memory)."""
    cfg = PcrServerConfig(_dptr(arena, "arena"), _nbytes(arena), max_width, max_height, num_slots, max_batch_views,
                          max_inflight, streams, max_batch_clouds, batch_config, depth_factor,
                          background_rgba & 0xFFFFFFFF, max_queue, deadline_us, policy, l2_budget_mb)
    out = _VP()
    _check(lib().pcr_server_create(ctx, C.byref(cfg), C.byref(out)), "pcr_server_create")
    return out.value


def pcr_server_destroy(srv: int):
    _check(lib().pcr_server_destroy(srv), "pcr_server_destroy")


def pcr_server_add_cloud(srv: int, cloud_id: int, host_points, n: int | None = None):
    """host_points must stay alive as long as the server."""
    if n is None:
        n = _nbytes(host_points) // 16
    _check(lib().pcr_server_add_cloud(srv, cloud_id, _hptr(host_points, "host_points") if n else None, n),
           "pcr_server_add_cloud")


def pcr_server_add_device_cloud(srv: int, cloud_id: int, dev_points, n: int | None = None):
    if n is None:
        n = _nbytes(dev_points) // 16
    _check(lib().pcr_server_add_device_cloud(srv, cloud_id, _dptr(dev_points, "dev_points") if n else None, n),
           "pcr_server_add_device_cloud")


def pcr_server_submit(srv: int, cloud_id: int, matrix, width: int, height: int, flags: int) -> int:
    """Ticket of the queued request; raises PcrError (status PCR_ERR_BUSY)
    when admission control refuses it."""
    vals = [float(v) for v in (matrix.reshape(-1).tolist() if hasattr(matrix, "reshape") else matrix)]
    req = PcrRequest(cloud_id, (C.c_float * 16)(*vals), width, height, flags)
    t = _U64()
    _check(lib().pcr_server_submit(srv, C.byref(req), C.byref(t)), "pcr_server_submit")
    return t.value


def pcr_server_step(srv: int) -> int:
    done = _U32()
    _check(lib().pcr_server_step(srv, C.byref(done)), "pcr_server_step")
    return done.value


def pcr_server_state(srv: int, ticket: int) -> int:
    st = _INT()
    _check(lib().pcr_server_state(srv, ticket, C.byref(st)), "pcr_server_state")
    return st.value


def pcr_server_get_result(srv: int, ticket: int) -> PcrServerResult:
    out = PcrServerResult()
    _check(lib().pcr_server_get_result(srv, ticket, C.byref(out)), "pcr_server_get_result")
    return out


def pcr_server_poll_completed(srv: int, capacity: int = 256) -> list[int]:
    buf = (_U64 * capacity)()
    count = _U32()
    _check(lib().pcr_server_poll_completed(srv, buf, capacity, C.byref(count)), "pcr_server_poll_completed")
    return list(buf[:count.value])


def pcr_server_release(srv: int, ticket: int):
    _check(lib().pcr_server_release(srv, ticket), "pcr_server_release")


def pcr_server_cancel(srv: int, ticket: int):
    _check(lib().pcr_server_cancel(srv, ticket), "pcr_server_cancel")


def pcr_server_stats_get(srv: int) -> dict:
    out = PcrServerStats()
    _check(lib().pcr_server_stats_get(srv, C.byref(out)), "pcr_server_stats_get")
    return {k: getattr(out, k) for k, _ in PcrServerStats._fields_}


def pcr_last_device_error(ctx: int) -> int:
    code = _U32()
    _check(lib().pcr_last_device_error(ctx, C.byref(code)), "pcr_last_device_error")
    return code.value


def pcr_check_division(ctx: int, w_first: int, w_count: int, c_bits=None, c_first: int = 0, c_count: int = 0,
                       c_step: int = 1, size: float = 1920.0) -> dict:
    """Device check of the projection's screen division (synchronous).
    c_bits: optional CUDA tensor of float32 bit patterns (int32 storage)."""
    out = (_U64 * 5)()
    if c_bits is not None:
        c_count = int(c_bits.numel())
    _check(lib().pcr_check_division(ctx, w_first, w_count, _dptr(c_bits, "c_bits"), c_first, c_count, c_step, size,
                                    out), "pcr_check_division")
    return {"reciprocal_mismatches": out[0], "quotient_mismatches": out[1], "screen_mismatches": out[2],
            "quotient_pairs": out[3], "pairs": out[4]}


# ---------------------------------------------------------------------------
# Small conveniences for callers that hold their buffers in torch tensors.
# ---------------------------------------------------------------------------

def alloc_framebuffer(width: int, height: int, device="cuda", hq: bool = True) -> dict:
    """Device tensors for one viewport: keys (int64 storage of uint64),
    hq_depth (int32 storage of uint32), hq_rg, hq_ba, the HQS1R primary
    words, the busy-loop lock words (zeroed) and the rgba image."""
    import torch
    npx = width * height
    fb = {"keys": torch.empty(npx, dtype=torch.int64, device=device),
          "image": torch.empty(npx, dtype=torch.int32, device=device)}
    if hq:
        fb["hq_depth"] = torch.empty(npx, dtype=torch.int32, device=device)
        fb["hq_rg"] = torch.empty(npx, dtype=torch.int64, device=device)
        fb["hq_ba"] = torch.empty(npx, dtype=torch.int64, device=device)
        fb["hq1r_primary"] = torch.empty(npx, dtype=torch.int64, device=device)
    fb["locks"] = torch.zeros(npx, dtype=torch.int32, device=device)
    return fb


class Context:
    """Owns one pcr_ctx; `with Context(0) as c:` destroys it on exit."""

    def __init__(self, device: int = 0, stream=None):
        self.handle = pcr_create(device)
        if stream is not None:
            pcr_set_stream(self.handle, stream)

    def close(self):
        if self.handle:
            pcr_destroy(self.handle)
            self.handle = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
