"""Thin Python binding of libfastatlas (include/fastatlas.h).

Functions named ``fa_*`` mirror the C ABI one to one and only marshal arguments:
torch CUDA tensors are passed as raw device pointers and
``torch.cuda.current_stream().cuda_stream`` as the stream.  Every step of the
atlasing path runs in the library's CUDA kernels; there is no CPU fallback, and
loading fails loudly when the library has not been built.

The small classes at the bottom (``Context``, ``Mesh``, ``FrameBuffers``) own the
torch tensors the calls write into, so that they stay alive while kernels run.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfastatlas.so")

FA_OK = 0
FA_E_INVALID_ARG = 1
FA_E_OUT_OF_MEMORY = 2
FA_E_CAPACITY = 3
FA_E_PACK_FAILED = 4
FA_E_TIMEOUT = 5
FA_E_CUDA = 6
FA_CHARTS_EDGE = 0
FA_CHARTS_VERTEX = 1
FA_SELECT_EFFECTIVE = 0
FA_SELECT_LARGEST_K = 1
FA_BOX_FRUSTUM_CLIP = 1
FA_VIS_CONSERVATIVE = 2
FA_FRAME_PERSISTENT = 1 << 12


def FA_LOWRES(d):
    """Frame flags field: the packing also serves the atlas scaled by 2^-d (Sec. 7)."""
    return (int(d) & 7) << 8

EXPORTS = ["fa_version", "fa_status_string", "fa_create", "fa_destroy", "fa_mesh_register",
           "fa_mesh_release", "fa_visibility", "fa_chartify", "fa_parameterize", "fa_pack", "fa_uv",
           "fa_atlas_frame", "fa_last_device_status", "fa_launch_count", "fa_profile_enable",
           "fa_profile_read", "fa_pack_noalloc", "fa_atlas_frame_dev_matrix", "fa_batch_create",
           "fa_batch_destroy", "fa_batch_mesh_register", "fa_batch_set_schedule", "fa_batch_get_schedule",
           "fa_atlas_batch", "fa_batch_tune", "fa_batch_launch_count", "fa_server_create", "fa_server_destroy",
           "fa_server_session_open", "fa_server_session_close", "fa_server_submit", "fa_server_poll",
           "fa_server_stats", "fa_server_now_ms", "fa_frame_stats_read", "fa_set_wait_limits",
           "fa_batch_plan_create", "fa_batch_plan_launch", "fa_batch_plan_get_schedule",
           "fa_batch_plan_set_schedule", "fa_batch_plan_tune", "fa_batch_plan_destroy", "fa_set_raster_schedule",
           "fa_set_chart_pack_schedule", "fa_get_kernel_schedule", "fa_batch_get_kernel_schedule"]
FA_RASTER_MID_OFF = 16
FA_RASTER_MID_MAX = 256
FA_RASTER_HIZ = 1
FA_DEFAULT_LOOP_CAP = 1 << 24
FA_DEFAULT_WAIT_NS = 1_000_000_000

FA_BATCH_ROUND_ROBIN, FA_BATCH_LONGEST_FIRST = 0, 1


class fa_config(ctypes.Structure):
    _fields_ = [("max_tris", ctypes.c_uint32), ("max_verts", ctypes.c_uint32),
                ("max_charts", ctypes.c_uint32), ("max_width", ctypes.c_uint32),
                ("max_height", ctypes.c_uint32), ("max_atlas_log2", ctypes.c_uint32),
                ("min_box", ctypes.c_uint32), ("gutter", ctypes.c_uint32), ("device", ctypes.c_int32)]


class fa_charts(ctypes.Structure):
    _fields_ = [("root", ctypes.c_void_p), ("bbox", ctypes.c_void_p), ("fa", ctypes.c_void_p),
                ("fb", ctypes.c_void_p), ("rot", ctypes.c_void_p), ("count", ctypes.c_void_p)]


class fa_placement(ctypes.Structure):
    _fields_ = [("x", ctypes.c_int32), ("y", ctypes.c_int32), ("w", ctypes.c_int32), ("h", ctypes.c_int32)]


class fa_pack_result(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("omega", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("count", ctypes.c_uint32)]


class fa_frame_params(ctypes.Structure):
    _fields_ = [("view_proj", ctypes.c_float * 16), ("width", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("ratio", ctypes.c_float), ("atlas_log2", ctypes.c_uint32), ("chart_mode", ctypes.c_uint32),
                ("n_scales", ctypes.c_uint32), ("select_mode", ctypes.c_uint32), ("flags", ctypes.c_uint32)]


class fa_frame_out(ctypes.Structure):
    _fields_ = [("vt", ctypes.c_void_p), ("tri_chart", ctypes.c_void_p), ("vert_chart", ctypes.c_void_p),
                ("charts", fa_charts), ("order", ctypes.c_void_p), ("place", ctypes.c_void_p),
                ("result", ctypes.c_void_p), ("uv", ctypes.c_void_p), ("affine", ctypes.c_void_p),
                ("partial", ctypes.c_void_p)]


class fa_frame_stats(ctypes.Structure):
    _fields_ = [("survivors", ctypes.c_uint32), ("clipped", ctypes.c_uint32), ("clip_records", ctypes.c_uint32),
                ("big_entries", ctypes.c_uint32), ("big_tiles", ctypes.c_uint64), ("visible", ctypes.c_uint32),
                ("charts", ctypes.c_uint32), ("visible_tiles", ctypes.c_uint32)]


class fa_plan_schedule(ctypes.Structure):
    _fields_ = [("lanes", ctypes.c_uint32), ("policy", ctypes.c_uint32), ("worker_pct", ctypes.c_uint32),
                ("mid_max_pix", ctypes.c_uint32), ("raster_flags", ctypes.c_uint32)]


class fa_kernel_schedule(ctypes.Structure):
    _fields_ = [("mid_max_pix", ctypes.c_uint32), ("raster_flags", ctypes.c_uint32),
                ("uf_threads", ctypes.c_uint32), ("push_threads", ctypes.c_uint32)]

    def as_dict(self):
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


class fa_server_done(ctypes.Structure):
    _fields_ = [("ticket", ctypes.c_uint64), ("session", ctypes.c_uint32), ("slot", ctypes.c_uint32),
                ("submit_ms", ctypes.c_double), ("dispatch_ms", ctypes.c_double), ("done_ms", ctypes.c_double)]


_lib = None


def load(path: str = LIB_PATH):
    """Load libfastatlas.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libfastatlas is not built ({path} missing); run "
                           "python -m paper_2502_17712_gb300.build")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    u32 = ctypes.c_uint32
    f32 = ctypes.c_float
    st = ctypes.c_int
    lib.fa_version.restype = u32
    lib.fa_status_string.argtypes = [st]
    lib.fa_status_string.restype = ctypes.c_char_p
    lib.fa_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(fa_config)]
    lib.fa_create.restype = st
    lib.fa_destroy.argtypes = [P]
    lib.fa_destroy.restype = None
    lib.fa_mesh_register.argtypes = [P, P, u32, P, u32, ctypes.POINTER(P), P]
    lib.fa_mesh_register.restype = st
    lib.fa_mesh_release.argtypes = [P]
    lib.fa_mesh_release.restype = None
    lib.fa_visibility.argtypes = [P, P, P, u32, u32, u32, P, P]
    lib.fa_visibility.restype = st
    lib.fa_chartify.argtypes = [P, P, P, u32, P, P, ctypes.POINTER(fa_charts), P]
    lib.fa_chartify.restype = st
    lib.fa_parameterize.argtypes = [P, P, P, u32, u32, f32, P, ctypes.POINTER(fa_charts), u32, P, P]
    lib.fa_parameterize.restype = st
    lib.fa_pack.argtypes = [P, P, P, P, u32, u32, u32, P, P, P, u32, P]
    lib.fa_pack.restype = st
    lib.fa_uv.argtypes = [P, P, P, u32, u32, f32, P, ctypes.POINTER(fa_charts), P, P, u32, u32, P, P, P]
    lib.fa_uv.restype = st
    lib.fa_atlas_frame.argtypes = [P, P, ctypes.POINTER(fa_frame_params), ctypes.POINTER(fa_frame_out), P]
    lib.fa_atlas_frame.restype = st
    lib.fa_atlas_frame_dev_matrix.argtypes = [P, P, ctypes.POINTER(fa_frame_params), P,
                                              ctypes.POINTER(fa_frame_out), P]
    lib.fa_atlas_frame_dev_matrix.restype = st
    lib.fa_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(fa_config), u32]
    lib.fa_batch_create.restype = st
    lib.fa_batch_destroy.argtypes = [P]
    lib.fa_batch_destroy.restype = None
    lib.fa_batch_mesh_register.argtypes = [P, P, u32, P, u32, ctypes.POINTER(P), P]
    lib.fa_batch_mesh_register.restype = st
    lib.fa_batch_set_schedule.argtypes = [P, u32, u32]
    lib.fa_batch_set_schedule.restype = st
    lib.fa_batch_get_schedule.argtypes = [P, ctypes.POINTER(u32), ctypes.POINTER(u32)]
    lib.fa_batch_get_schedule.restype = st
    lib.fa_atlas_batch.argtypes = [P, u32, ctypes.POINTER(P), ctypes.POINTER(fa_frame_params),
                                   ctypes.POINTER(fa_frame_out), P]
    lib.fa_atlas_batch.restype = st
    lib.fa_batch_tune.argtypes = [P, u32, ctypes.POINTER(P), ctypes.POINTER(fa_frame_params),
                                  ctypes.POINTER(fa_frame_out), u32, ctypes.POINTER(f32)]
    lib.fa_batch_tune.restype = st
    lib.fa_batch_plan_create.argtypes = [P, u32, ctypes.POINTER(P), ctypes.POINTER(fa_frame_params),
                                         ctypes.POINTER(P), ctypes.POINTER(fa_frame_out), ctypes.POINTER(P)]
    lib.fa_batch_plan_create.restype = st
    lib.fa_batch_plan_launch.argtypes = [P, P]
    lib.fa_batch_plan_launch.restype = st
    lib.fa_batch_plan_get_schedule.argtypes = [P, ctypes.POINTER(fa_plan_schedule)]
    lib.fa_batch_plan_get_schedule.restype = st
    lib.fa_batch_plan_set_schedule.argtypes = [P, ctypes.POINTER(fa_plan_schedule)]
    lib.fa_batch_plan_set_schedule.restype = st
    lib.fa_batch_plan_tune.argtypes = [P, u32, ctypes.POINTER(f32)]
    lib.fa_batch_plan_tune.restype = st
    lib.fa_batch_plan_destroy.argtypes = [P]
    lib.fa_batch_plan_destroy.restype = None
    lib.fa_batch_launch_count.argtypes = [P]
    lib.fa_batch_launch_count.restype = ctypes.c_uint64
    lib.fa_server_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(fa_config), u32, ctypes.c_uint64,
                                     ctypes.POINTER(u32)]
    lib.fa_server_create.restype = st
    lib.fa_server_destroy.argtypes = [P]
    lib.fa_server_destroy.restype = None
    lib.fa_server_session_open.argtypes = [P, P, u32, P, u32, ctypes.POINTER(fa_frame_out), ctypes.POINTER(u32)]
    lib.fa_server_session_open.restype = st
    lib.fa_server_session_close.argtypes = [P, u32]
    lib.fa_server_session_close.restype = st
    lib.fa_server_submit.argtypes = [P, u32, ctypes.POINTER(fa_frame_params), ctypes.POINTER(fa_frame_out),
                                     ctypes.POINTER(ctypes.c_uint64)]
    lib.fa_server_submit.restype = st
    lib.fa_server_poll.argtypes = [P, ctypes.POINTER(fa_server_done), u32, ctypes.POINTER(u32)]
    lib.fa_server_poll.restype = st
    lib.fa_server_stats.argtypes = [P, ctypes.POINTER(u32), ctypes.POINTER(u32), ctypes.POINTER(u32),
                                    ctypes.POINTER(ctypes.c_uint64)]
    lib.fa_server_stats.restype = st
    lib.fa_server_now_ms.argtypes = [P]
    lib.fa_server_now_ms.restype = ctypes.c_double
    lib.fa_last_device_status.argtypes = [P, P, ctypes.POINTER(ctypes.c_int32)]
    lib.fa_last_device_status.restype = st
    lib.fa_launch_count.argtypes = [P]
    lib.fa_launch_count.restype = ctypes.c_uint64
    lib.fa_set_raster_schedule.argtypes = [P, u32, u32]
    lib.fa_set_raster_schedule.restype = st
    lib.fa_set_chart_pack_schedule.argtypes = [P, u32, u32]
    lib.fa_set_chart_pack_schedule.restype = st
    lib.fa_get_kernel_schedule.argtypes = [P, ctypes.POINTER(fa_kernel_schedule)]
    lib.fa_get_kernel_schedule.restype = st
    lib.fa_batch_get_kernel_schedule.argtypes = [P, ctypes.POINTER(fa_kernel_schedule)]
    lib.fa_batch_get_kernel_schedule.restype = st
    lib.fa_set_wait_limits.argtypes = [P, u32, ctypes.c_uint64]
    lib.fa_set_wait_limits.restype = st
    lib.fa_frame_stats_read.argtypes = [P, P, ctypes.POINTER(fa_frame_stats)]
    lib.fa_frame_stats_read.restype = st
    lib.fa_profile_enable.argtypes = [P, ctypes.c_int]
    lib.fa_profile_enable.restype = st
    lib.fa_profile_read.argtypes = [P, ctypes.c_int, ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int)]
    lib.fa_profile_read.restype = st
    lib.fa_pack_noalloc.argtypes = [P, P, u32, u32, u32, u32, u32, u32, P, P, P, P]
    lib.fa_pack_noalloc.restype = st
    _lib = lib
    return lib


class FastAtlasError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        name = load().fa_status_string(status).decode() if _lib is not None else str(status)
        super().__init__(f"{where}: {name}")


def _check(status: int, where: str):
    if status != FA_OK:
        raise FastAtlasError(status, where)


def _ptr(t) -> int | None:
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return t.data_ptr()


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _mat(M):
    return (ctypes.c_float * 16)(*np.ascontiguousarray(M, np.float32).ravel().tolist())


# ------------------------------------------------------------------ C ABI mirrors

def fa_version() -> int:
    return load().fa_version()


def fa_create(cfg: fa_config) -> int:
    h = ctypes.c_void_p()
    _check(load().fa_create(ctypes.byref(h), ctypes.byref(cfg)), "fa_create")
    return h.value


def fa_destroy(ctx: int):
    load().fa_destroy(ctx)


def fa_mesh_register(ctx, pos, idx, stream=None) -> int:
    m = ctypes.c_void_p()
    _check(load().fa_mesh_register(ctx, _ptr(pos), pos.shape[0], _ptr(idx), idx.shape[0], ctypes.byref(m),
                                   _stream(stream)), "fa_mesh_register")
    return m.value


def fa_mesh_release(mesh: int):
    load().fa_mesh_release(mesh)


def fa_visibility(ctx, mesh, M, width, height, vt, stream=None, flags=0):
    _check(load().fa_visibility(ctx, mesh, _mat(M), width, height, int(flags), _ptr(vt), _stream(stream)),
           "fa_visibility")


def fa_chartify(ctx, mesh, vt, mode, tri_chart, vert_chart, charts: fa_charts, stream=None):
    _check(load().fa_chartify(ctx, mesh, _ptr(vt), mode, _ptr(tri_chart), _ptr(vert_chart),
                              ctypes.byref(charts), _stream(stream)), "fa_chartify")


def fa_parameterize(ctx, mesh, M, width, height, ratio, tri_chart, charts: fa_charts, flags=0, partial=None,
                    stream=None):
    _check(load().fa_parameterize(ctx, mesh, _mat(M), width, height, float(ratio), _ptr(tri_chart),
                                  ctypes.byref(charts), int(flags), _ptr(partial), _stream(stream)),
           "fa_parameterize")


def fa_pack(ctx, fa, fb, count, atlas_log2, n_scales, select_mode, order, place, res, stream=None,
            lowres_log2=0):
    _check(load().fa_pack(ctx, _ptr(fa), _ptr(fb), _ptr(count), atlas_log2, n_scales, select_mode, _ptr(order),
                          _ptr(place), _ptr(res), int(lowres_log2), _stream(stream)), "fa_pack")


def fa_pack_noalloc(fa, fb, n, atlas_log2, n_scales, select_mode, min_box, gutter, order, place, res,
                    stream=None):
    """fa_pack without a context or any allocation (scratch is a static device array
    inside the library, at most 4096 boxes); for callers that may not allocate."""
    _check(load().fa_pack_noalloc(_ptr(fa), _ptr(fb), n, atlas_log2, n_scales, select_mode, min_box, gutter,
                                  _ptr(order), _ptr(place), _ptr(res), _stream(stream)), "fa_pack_noalloc")


def fa_uv(ctx, mesh, M, width, height, ratio, tri_chart, charts: fa_charts, place, res, atlas_log2, n_scales,
          uv, affine, stream=None):
    _check(load().fa_uv(ctx, mesh, _mat(M), width, height, float(ratio), _ptr(tri_chart), ctypes.byref(charts),
                        _ptr(place), _ptr(res), atlas_log2, n_scales, _ptr(uv), _ptr(affine), _stream(stream)),
           "fa_uv")


def fa_atlas_frame(ctx, mesh, params: fa_frame_params, out: fa_frame_out, stream=None):
    _check(load().fa_atlas_frame(ctx, mesh, ctypes.byref(params), ctypes.byref(out), _stream(stream)),
           "fa_atlas_frame")


def fa_atlas_frame_dev_matrix(ctx, mesh, params: fa_frame_params, d_view_proj, out: fa_frame_out,
                              stream=None):
    _check(load().fa_atlas_frame_dev_matrix(ctx, mesh, ctypes.byref(params), _ptr(d_view_proj), ctypes.byref(out),
                                            _stream(stream)), "fa_atlas_frame_dev_matrix")


def fa_last_device_status(ctx, stream=None) -> int:
    v = ctypes.c_int32()
    _check(load().fa_last_device_status(ctx, _stream(stream), ctypes.byref(v)), "fa_last_device_status")
    return v.value


def fa_launch_count(ctx) -> int:
    return load().fa_launch_count(ctx)


def fa_set_wait_limits(ctx, loop_cap=FA_DEFAULT_LOOP_CAP, wait_ns=FA_DEFAULT_WAIT_NS):
    _check(load().fa_set_wait_limits(ctx, int(loop_cap), int(wait_ns)), "fa_set_wait_limits")


def fa_frame_stats_read(ctx, stream=None) -> dict:
    """Work counts of the last frame on the context (synchronizes the stream)."""
    r = fa_frame_stats()
    _check(load().fa_frame_stats_read(ctx, _stream(stream), ctypes.byref(r)), "fa_frame_stats_read")
    return {f: int(getattr(r, f)) for f, _ in fa_frame_stats._fields_}


def fa_profile_enable(ctx, enable: bool):
    _check(load().fa_profile_enable(ctx, 1 if enable else 0), "fa_profile_enable")


def fa_profile_read(ctx, max_n: int = 64):
    """[(kernel name, ms)] of the last traced call (waits for it to finish)."""
    ms = (ctypes.c_float * max_n)()
    names = (ctypes.c_char_p * max_n)()
    n = ctypes.c_int()
    _check(load().fa_profile_read(ctx, max_n, ms, names, ctypes.byref(n)), "fa_profile_read")
    return [(names[i].decode(), float(ms[i])) for i in range(min(n.value, max_n))]


# ------------------------------------------------------------------ owners of device buffers

class Context:
    """An fa_ctx plus its configuration."""

    def __init__(self, max_tris, max_verts, max_charts=1 << 16, max_width=1920, max_height=1080,
                 max_atlas_log2=12, min_box=2, gutter=0, device=0):
        self.cfg = fa_config(max_tris, max_verts, max_charts, max_width, max_height, max_atlas_log2,
                             min_box, gutter, device)
        self.handle = fa_create(self.cfg)

    def close(self):
        if self.handle:
            fa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_status(self, stream=None) -> int:
        return fa_last_device_status(self.handle, stream)

    def set_wait_limits(self, loop_cap=FA_DEFAULT_LOOP_CAP, wait_ns=FA_DEFAULT_WAIT_NS):
        fa_set_wait_limits(self.handle, loop_cap, wait_ns)

    def set_raster_schedule(self, mid_max_pix=FA_RASTER_MID_OFF, flags=0):
        _check(load().fa_set_raster_schedule(self.handle, int(mid_max_pix), int(flags)), "fa_set_raster_schedule")

    def set_chart_pack_schedule(self, uf_threads=1024, push_threads=512):
        _check(load().fa_set_chart_pack_schedule(self.handle, int(uf_threads), int(push_threads)),
               "fa_set_chart_pack_schedule")

    def kernel_schedule(self) -> dict:
        out = fa_kernel_schedule()
        _check(load().fa_get_kernel_schedule(self.handle, ctypes.byref(out)), "fa_get_kernel_schedule")
        return out.as_dict()

    @property
    def launches(self) -> int:
        return fa_launch_count(self.handle)

    def frame_stats(self, stream=None) -> dict:
        return fa_frame_stats_read(self.handle, stream)


class Mesh:
    """A registered mesh; keeps its position / index tensors alive."""

    def __init__(self, ctx: Context, pos, idx, stream=None):
        import torch
        self.ctx = ctx
        self.pos = pos if torch.is_tensor(pos) else torch.as_tensor(np.ascontiguousarray(pos, np.float32)).cuda()
        idx_np = idx if torch.is_tensor(idx) else np.ascontiguousarray(idx, np.uint32).view(np.int32)
        self.idx = idx_np if torch.is_tensor(idx_np) else torch.as_tensor(idx_np).cuda()
        self.T = int(self.idx.shape[0])
        self.V = int(self.pos.shape[0])
        self.handle = fa_mesh_register(ctx.handle, self.pos, self.idx, stream)

    def close(self):
        if self.handle:
            fa_mesh_release(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class FrameBuffers:
    """Device outputs of one frame (torch tensors) and their C views."""
    vt: object
    tri_chart: object
    vert_chart: object
    root: object
    bbox: object
    fa: object
    fb: object
    rot: object
    count: object
    order: object
    place: object
    result: object
    uv: object
    affine: object
    partial: object = None

    @staticmethod
    def allocate(T, V, max_charts, uv=True, vert_chart=False, partial=False, device="cuda"):
        import torch
        i32, u8, f32 = torch.int32, torch.uint8, torch.float32
        z = lambda *s, dt=i32: torch.zeros(*s, dtype=dt, device=device)
        return FrameBuffers(
            vt=z((T + 31) // 32), tri_chart=z(T), vert_chart=z(V) if vert_chart else None,
            root=z(max_charts), bbox=z(max_charts, 4, dt=f32), fa=z(max_charts), fb=z(max_charts),
            rot=z(max_charts, dt=u8), count=z(1), order=z(max_charts), place=z(max_charts, 4),
            result=z(5), uv=torch.full((T, 3, 2), float("nan"), dtype=f32, device=device) if uv else None,
            affine=z(max_charts, 6, dt=f32), partial=z((T + 31) // 32) if partial else None)

    def charts(self) -> fa_charts:
        return fa_charts(_ptr(self.root), _ptr(self.bbox), _ptr(self.fa), _ptr(self.fb), _ptr(self.rot),
                         _ptr(self.count))

    def c_out(self) -> fa_frame_out:
        return fa_frame_out(_ptr(self.vt), _ptr(self.tri_chart), _ptr(self.vert_chart), self.charts(),
                            _ptr(self.order), _ptr(self.place), _ptr(self.result), _ptr(self.uv),
                            _ptr(self.affine), _ptr(self.partial))


def frame_params(M, width, height, ratio, atlas_log2, chart_mode=FA_CHARTS_EDGE, n_scales=64,
                 select_mode=FA_SELECT_EFFECTIVE, flags=0) -> fa_frame_params:
    return fa_frame_params(_mat(M), width, height, float(ratio), atlas_log2, chart_mode, n_scales, select_mode,
                           flags)


def atlas_frame(ctx: Context, mesh: Mesh, bufs: FrameBuffers, M, width, height, ratio, atlas_log2,
                chart_mode=FA_CHARTS_EDGE, n_scales=64, select_mode=FA_SELECT_EFFECTIVE, stream=None, flags=0):
    """Enqueue the whole per-frame path (fa_atlas_frame); results land in ``bufs``."""
    p = frame_params(M, width, height, ratio, atlas_log2, chart_mode, n_scales, select_mode, flags)
    fa_atlas_frame(ctx.handle, mesh.handle, p, bufs.c_out(), stream)


def atlas_frame_dev_matrix(ctx: Context, mesh: Mesh, bufs: FrameBuffers, d_view_proj, width, height, ratio,
                           atlas_log2, chart_mode=FA_CHARTS_EDGE, n_scales=64, select_mode=FA_SELECT_EFFECTIVE,
                           stream=None, flags=0):
    """fa_atlas_frame_dev_matrix: the matrix is the device tensor ``d_view_proj``
    (16 float32, row-major), read when the kernels run."""
    p = frame_params(np.eye(4, dtype=np.float32), width, height, ratio, atlas_log2, chart_mode, n_scales,
                     select_mode, flags)
    fa_atlas_frame_dev_matrix(ctx.handle, mesh.handle, p, d_view_proj, bufs.c_out(), stream)


# ------------------------------------------------------------------ batches

class Batch:
    """An fa_batch: n_lanes contexts of one configuration, each with its own stream."""

    def __init__(self, n_lanes, max_tris, max_verts, max_charts=1 << 16, max_width=1920, max_height=1080,
                 max_atlas_log2=12, min_box=2, gutter=0, device=0):
        self.cfg = fa_config(max_tris, max_verts, max_charts, max_width, max_height, max_atlas_log2,
                             min_box, gutter, device)
        h = ctypes.c_void_p()
        _check(load().fa_batch_create(ctypes.byref(h), ctypes.byref(self.cfg), n_lanes), "fa_batch_create")
        self.handle = h.value
        self.n_lanes = n_lanes

    def close(self):
        if self.handle:
            load().fa_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_schedule(self, lanes, policy=FA_BATCH_ROUND_ROBIN):
        _check(load().fa_batch_set_schedule(self.handle, lanes, policy), "fa_batch_set_schedule")

    def schedule(self):
        lanes, pol = ctypes.c_uint32(), ctypes.c_uint32()
        _check(load().fa_batch_get_schedule(self.handle, ctypes.byref(lanes), ctypes.byref(pol)),
               "fa_batch_get_schedule")
        return lanes.value, pol.value

    def kernel_schedule(self) -> dict:
        out = fa_kernel_schedule()
        _check(load().fa_batch_get_kernel_schedule(self.handle, ctypes.byref(out)), "fa_batch_get_kernel_schedule")
        return out.as_dict()

    @property
    def launches(self) -> int:
        return int(load().fa_batch_launch_count(self.handle))


class BatchMesh(Mesh):
    """A mesh registered with a batch (any lane may atlas it)."""

    def __init__(self, batch: Batch, pos, idx, stream=None):
        import torch
        self.ctx = batch
        self.pos = pos if torch.is_tensor(pos) else torch.as_tensor(np.ascontiguousarray(pos, np.float32)).cuda()
        idx_np = idx if torch.is_tensor(idx) else np.ascontiguousarray(idx, np.uint32).view(np.int32)
        self.idx = idx_np if torch.is_tensor(idx_np) else torch.as_tensor(idx_np).cuda()
        self.T = int(self.idx.shape[0])
        self.V = int(self.pos.shape[0])
        h = ctypes.c_void_p()
        _check(load().fa_batch_mesh_register(batch.handle, _ptr(self.pos), self.V, _ptr(self.idx), self.T,
                                             ctypes.byref(h), _stream(stream)), "fa_batch_mesh_register")
        self.handle = h.value


def _batch_arrays(meshes, params, bufs):
    n = len(meshes)
    mh = (ctypes.c_void_p * n)(*[m.handle for m in meshes])
    pa = (fa_frame_params * n)(*params)
    oa = (fa_frame_out * n)(*[b.c_out() for b in bufs])
    return n, mh, pa, oa


def atlas_batch(batch: Batch, meshes, params, bufs, stream=None):
    """Enqueue fa_atlas_batch: view i = meshes[i] with params[i] (fa_frame_params,
    see frame_params) into bufs[i]."""
    n, mh, pa, oa = _batch_arrays(meshes, params, bufs)
    _check(load().fa_atlas_batch(batch.handle, n, mh, pa, oa, _stream(stream)), "fa_atlas_batch")


def batch_tune(batch: Batch, meshes, params, bufs, reps=3):
    """fa_batch_tune; returns (lanes, policy, best_ms)."""
    n, mh, pa, oa = _batch_arrays(meshes, params, bufs)
    ms = ctypes.c_float()
    _check(load().fa_batch_tune(batch.handle, n, mh, pa, oa, reps, ctypes.byref(ms)), "fa_batch_tune")
    lanes, pol = batch.schedule()
    return lanes, pol, ms.value


class BatchPlan:
    """An fa_batch_plan: the views of a batch atlased by one launch of the persistent
    frame kernel.  ``d_view_proj`` (optional) is a list of device tensors of 16
    float32 each, read when the kernel runs (the views' params matrices are then
    ignored)."""

    def __init__(self, batch: Batch, meshes, params, bufs, d_view_proj=None):
        n, mh, pa, oa = _batch_arrays(meshes, params, bufs)
        dm = None
        if d_view_proj is not None:
            dm = (ctypes.c_void_p * n)(*[_ptr(t) for t in d_view_proj])
        h = ctypes.c_void_p()
        _check(load().fa_batch_plan_create(batch.handle, n, mh, pa, dm, oa, ctypes.byref(h)),
               "fa_batch_plan_create")
        self.handle = h.value
        self._keep = (batch, meshes, bufs, d_view_proj, mh, pa, oa)

    def launch(self, stream=None):
        _check(load().fa_batch_plan_launch(self.handle, _stream(stream)), "fa_batch_plan_launch")

    def schedule(self):
        s = fa_plan_schedule()
        _check(load().fa_batch_plan_get_schedule(self.handle, ctypes.byref(s)), "fa_batch_plan_get_schedule")
        return s.lanes, s.policy, s.worker_pct, s.mid_max_pix, s.raster_flags

    def set_schedule(self, lanes, policy=FA_BATCH_LONGEST_FIRST, worker_pct=100, mid_max_pix=FA_RASTER_MID_OFF,
                     raster_flags=0):
        s = fa_plan_schedule(lanes, policy, worker_pct, mid_max_pix, raster_flags)
        _check(load().fa_batch_plan_set_schedule(self.handle, ctypes.byref(s)), "fa_batch_plan_set_schedule")

    def tune(self, reps=3):
        """fa_batch_plan_tune; returns (lanes, policy, worker_pct, mid_max_pix, raster_flags, best_ms)."""
        ms = ctypes.c_float()
        _check(load().fa_batch_plan_tune(self.handle, reps, ctypes.byref(ms)), "fa_batch_plan_tune")
        return (*self.schedule(), ms.value)

    def close(self):
        if self.handle:
            load().fa_batch_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ serving

class Server:
    """An fa_server: slots (context + stream) admitted by a device-memory budget,
    sessions with device-resident meshes, continuous batching of view requests."""

    def __init__(self, max_slots, budget_bytes, max_tris, max_verts, max_charts=1 << 16, max_width=1920,
                 max_height=1080, max_atlas_log2=12, min_box=2, gutter=0, device=0):
        self.cfg = fa_config(max_tris, max_verts, max_charts, max_width, max_height, max_atlas_log2,
                             min_box, gutter, device)
        h, n = ctypes.c_void_p(), ctypes.c_uint32()
        _check(load().fa_server_create(ctypes.byref(h), ctypes.byref(self.cfg), max_slots, int(budget_bytes),
                                       ctypes.byref(n)), "fa_server_create")
        self.handle = h.value
        self.n_slots = n.value
        self._keep = {}

    def close(self):
        if self.handle:
            load().fa_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def open_session(self, pos, idx, bufs: "FrameBuffers | None" = None) -> int:
        import torch
        pos = pos if torch.is_tensor(pos) else torch.as_tensor(np.ascontiguousarray(pos, np.float32)).cuda()
        idx = idx if torch.is_tensor(idx) else torch.as_tensor(
            np.ascontiguousarray(idx, np.uint32).view(np.int32)).cuda()
        sid = ctypes.c_uint32()
        out = ctypes.byref(bufs.c_out()) if bufs is not None else None
        _check(load().fa_server_session_open(self.handle, _ptr(pos), int(pos.shape[0]), _ptr(idx),
                                             int(idx.shape[0]), out, ctypes.byref(sid)), "fa_server_session_open")
        self._keep[sid.value] = (pos, idx, bufs)
        return sid.value

    def close_session(self, sid: int):
        _check(load().fa_server_session_close(self.handle, sid), "fa_server_session_close")
        self._keep.pop(sid, None)

    def submit(self, sid: int, params: fa_frame_params, bufs: "FrameBuffers | None" = None) -> int:
        t = ctypes.c_uint64()
        out = ctypes.byref(bufs.c_out()) if bufs is not None else None
        _check(load().fa_server_submit(self.handle, sid, ctypes.byref(params), out, ctypes.byref(t)),
               "fa_server_submit")
        return t.value

    def poll(self, max_done=64):
        arr = (fa_server_done * max_done)()
        n = ctypes.c_uint32()
        _check(load().fa_server_poll(self.handle, arr, max_done, ctypes.byref(n)), "fa_server_poll")
        return [dict(ticket=d.ticket, session=d.session, slot=d.slot, submit_ms=d.submit_ms,
                     dispatch_ms=d.dispatch_ms, done_ms=d.done_ms) for d in arr[:n.value]]

    def stats(self):
        q, r, m, b = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint64()
        _check(load().fa_server_stats(self.handle, ctypes.byref(q), ctypes.byref(r), ctypes.byref(m),
                                      ctypes.byref(b)), "fa_server_stats")
        return dict(queued=q.value, running=r.value, max_running=m.value, used_bytes=b.value)

    def now_ms(self) -> float:
        return float(load().fa_server_now_ms(self.handle))
