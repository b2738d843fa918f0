"""Plain CPU oracle for the FastAtlas per-frame atlasing path.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the product path never does.  The oracle is a
single-threaded C++17 library (``fa_oracle.cpp``) compiled with
``-ffp-contract=off`` so every fp32 expression rounds once per operation in the
order written; this wrapper only marshals numpy arrays.

Each function follows one step of the paper (FastAtlas, Vining et al. 2025):

=================  =====================================================
``visibility``     Sec. 5.1 + App. A (depth pre-pass, "<=" marking pass)
``chartify``       Sec. 5.1 + App. A / Alg. 1 (connected components)
``parameterize``   Sec. 5.2 (near clip + Blinn box) and Sec. 4.1 (rotate tall)
``order``          Sec. 4.1 (height descending, root ascending)
``pack``           Sec. 4.2 (scale search) and Sec. 4.3 (fold + push)
``uv``             Sec. 3 / App. A (projection into the chart's atlas box)
=================  =====================================================
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fa_oracle.cpp")
_LIB = os.path.join(_HERE, "_build", "libfa_oracle.so")
_lib = None

CXXFLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (seconds); rebuilt when the source is newer."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *CXXFLAGS, _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class PackResult(ctypes.Structure):
    _fields_ = [("k", ctypes.c_uint32), ("omega", ctypes.c_uint32), ("height", ctypes.c_uint32),
                ("status", ctypes.c_int32), ("count", ctypes.c_uint32)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i = ctypes.c_int
        f = ctypes.c_float
        lib.or_transform.argtypes = [P, P, i, P]
        lib.or_raster_triangle.argtypes = [P, P, P, P, i, i, P, P, i]
        lib.or_visibility.argtypes = [P, P, P, i, i, i, P, P, i]
        lib.or_chartify.argtypes = [P, i, i, P, i, P, P, i, P]
        lib.or_chartify.restype = i
        lib.or_parameterize.argtypes = [P, P, P, i, i, i, f, P, i, P, P, P, P, ctypes.c_uint32, P]
        lib.or_order.argtypes = [P, i, P]
        lib.or_pack_candidate.argtypes = [P, P, P, i, i, i, i, i, i, P, P, P, P, P, P, P]
        lib.or_pack.argtypes = [P, P, i, i, i, i, i, i, P, ctypes.POINTER(PackResult), P, P, P, i]
        lib.or_uv.argtypes = [P, P, P, i, i, i, f, P, i, P, P, P, ctypes.POINTER(PackResult),
                              i, i, i, P, P]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def transform(M, pos):
    pos = _f32(pos)
    out = np.empty((pos.shape[0], 4), np.float32)
    _load().or_transform(_p(_f32(M)), _p(pos), pos.shape[0], _p(out))
    return out


def raster_triangle(M, p0, p1, p2, width, height, conservative=False):
    """Coverage mask and min depth key of one triangle (row py from the bottom):
    sample coverage, or the marking pass's conservative coverage."""
    cover = np.empty((height, width), np.uint8)
    key = np.empty((height, width), np.uint32)
    _load().or_raster_triangle(_p(_f32(M)), _p(_f32(p0)), _p(_f32(p1)), _p(_f32(p2)),
                               width, height, _p(cover), _p(key), int(bool(conservative)))
    return cover.astype(bool), key


VIS_CONSERVATIVE = 2  # flags bit: conservative coverage in the marking pass (App. A)


def LOWRES(d):
    """flags field: the packing also serves the atlas scaled by 2^-d (Sec. 7)."""
    return (int(d) & 7) << 8


def visibility(M, pos, idx, width, height, return_zbuf=False, conservative=False):
    """VT bitmask (uint32[ceil(T/32)]) and optionally the depth-key buffer [H][W]."""
    pos, idx = _f32(pos), _u32(idx)
    T = idx.shape[0]
    vt = np.zeros((T + 31) // 32, np.uint32)
    zb = np.empty((height, width), np.uint32)
    _load().or_visibility(_p(_f32(M)), _p(pos), _p(idx), T, width, height, _p(vt), _p(zb),
                          int(bool(conservative)))
    return (vt, zb) if return_zbuf else vt


def vt_to_bool(vt, T):
    bits = np.unpackbits(vt.view(np.uint8), bitorder="little")[:T]
    return bits.astype(bool)


def bool_to_vt(vis):
    vis = np.asarray(vis, bool)
    T = vis.shape[0]
    pad = np.zeros(((T + 31) // 32) * 32, bool)
    pad[:T] = vis
    return np.packbits(pad, bitorder="little").view(np.uint32).copy()


@dataclass
class Charts:
    tri_chart: np.ndarray  # int32 [T]
    roots: np.ndarray      # uint32 [C]
    vert_chart: np.ndarray  # int32 [V]

    @property
    def C(self):
        return int(self.roots.shape[0])


def chartify(idx, V, vt, mode=0, max_charts=1 << 24):
    idx = _u32(idx)
    T = idx.shape[0]
    tc = np.empty(T, np.int32)
    roots = np.empty(min(max_charts, max(T, 1)), np.uint32)
    vc = np.empty(V, np.int32)
    C = _load().or_chartify(_p(idx), T, V, _p(_u32(vt)), mode, _p(tc), _p(roots),
                            min(max_charts, max(T, 1)), _p(vc))
    if C < 0:
        raise OverflowError("chart count exceeds max_charts")
    return Charts(tc, roots[:C].copy(), vc)


@dataclass
class Footprints:
    bbox: np.ndarray     # float32 [C, 4] xmin, ymin, xmax, ymax (NDC)
    fa: np.ndarray       # uint32 [C] (1/256 texel), fa <= fb
    fb: np.ndarray
    rot: np.ndarray      # uint8 [C]
    partial: np.ndarray  # uint32 [ceil(T/32)] partial-visibility bits of the visible triangles


BOX_FRUSTUM_CLIP = 1  # flags bit: best single frustum plane clip for the boxes (Sec. 5.2)


def parameterize(M, pos, idx, width, height, ratio, tri_chart, C, flags=0):
    pos, idx = _f32(pos), _u32(idx)
    bbox = np.empty((C, 4), np.float32)
    fa = np.empty(C, np.uint32)
    fb = np.empty(C, np.uint32)
    rot = np.empty(C, np.uint8)
    partial = np.empty((idx.shape[0] + 31) // 32, np.uint32)
    _load().or_parameterize(_p(_f32(M)), _p(pos), _p(idx), idx.shape[0], width, height,
                            float(ratio), _p(np.ascontiguousarray(tri_chart, np.int32)), C,
                            _p(bbox), _p(fa), _p(fb), _p(rot), int(flags), _p(partial))
    return Footprints(bbox, fa, fb, rot, partial)


def order(fb):
    fb = _u32(fb)
    out = np.empty(fb.shape[0], np.uint32)
    _load().or_order(_p(fb), fb.shape[0], _p(out))
    return out


def pack_candidate(fa, fb, order_, atlas_log2, k, n_scales=64, min_box=2, gutter=0):
    fa, fb, order_ = _u32(fa), _u32(fb), _u32(order_)
    C = fa.shape[0]
    x, y, w, h = (np.empty(C, np.uint32) for _ in range(4))
    om = ctypes.c_uint64()
    H = ctypes.c_uint64()
    ok = ctypes.c_int()
    _load().or_pack_candidate(_p(fa), _p(fb), _p(order_), C, atlas_log2, k, n_scales, min_box,
                              gutter, _p(x), _p(y), _p(w), _p(h), ctypes.byref(om),
                              ctypes.byref(H), ctypes.byref(ok))
    return dict(x=x, y=y, w=w, h=h, omega=om.value, height=H.value, accepted=bool(ok.value))


@dataclass
class Packing:
    place: np.ndarray   # int32 [C, 4] x, y, w, h (chart order, virtual grid)
    k: int
    omega: int          # virtual side Omega of the chosen candidate
    height: int
    status: int
    cand_omega: np.ndarray
    cand_height: np.ndarray
    cand_ok: np.ndarray
    raw: PackResult


def pack(fa, fb, atlas_log2, n_scales=64, min_box=2, gutter=0, select_mode=0, lowres_log2=0):
    fa, fb = _u32(fa), _u32(fb)
    C = fa.shape[0]
    place = np.zeros((C, 4), np.int32)
    res = PackResult()
    co = np.empty(n_scales, np.uint64)
    ch = np.empty(n_scales, np.uint64)
    ck = np.empty(n_scales, np.int32)
    _load().or_pack(_p(fa), _p(fb), C, atlas_log2, n_scales, min_box, gutter, select_mode,
                    _p(place), ctypes.byref(res), _p(co), _p(ch), _p(ck), int(lowres_log2))
    return Packing(place, res.k, res.omega, res.height, res.status, co, ch, ck.astype(bool), res)


def uv(M, pos, idx, width, height, ratio, tri_chart, fp: Footprints, pk: Packing, atlas_log2,
       n_scales=64, gutter=0):
    """fp64 per-corner UVs [T, 3, 2] (NaN for invisible / w<=0) and affines [C, 6]."""
    pos, idx = _f32(pos), _u32(idx)
    T = idx.shape[0]
    C = fp.fa.shape[0]
    out = np.full((T, 3, 2), np.nan, np.float64)
    aff = np.zeros((C, 6), np.float64)
    _load().or_uv(_p(_f32(M)), _p(pos), _p(idx), T, width, height, float(ratio),
                  _p(np.ascontiguousarray(tri_chart, np.int32)), C,
                  _p(np.ascontiguousarray(fp.bbox, np.float32)), _p(np.ascontiguousarray(fp.rot, np.uint8)),
                  _p(np.ascontiguousarray(pk.place, np.int32)), ctypes.byref(pk.raw),
                  atlas_log2, n_scales, gutter, _p(out), _p(aff))
    return out, aff


@dataclass
class Frame:
    vt: np.ndarray
    charts: Charts
    fp: Footprints
    order: np.ndarray
    pk: Packing
    uv: np.ndarray
    affine: np.ndarray


def atlas_frame(M, pos, idx, width, height, ratio, atlas_log2, mode=0, n_scales=64,
                min_box=2, gutter=0, select_mode=0, vt=None, flags=0):
    """The whole per-frame path, step by step."""
    if vt is None:
        vt = visibility(M, pos, idx, width, height, conservative=bool(flags & VIS_CONSERVATIVE))
    ch = chartify(idx, pos.shape[0], vt, mode)
    fp = parameterize(M, pos, idx, width, height, ratio, ch.tri_chart, ch.C, flags)
    od = order(fp.fb)
    pk = pack(fp.fa, fp.fb, atlas_log2, n_scales, min_box, gutter, select_mode, (flags >> 8) & 7)
    u, aff = uv(M, pos, idx, width, height, ratio, ch.tri_chart, fp, pk, atlas_log2, n_scales, gutter)
    return Frame(vt, ch, fp, od, pk, u, aff)
