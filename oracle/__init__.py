"""CPU oracle for the ray-traced sphere-splat image warping (Zellmann 2020, arXiv 2006.14726).

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's CPU-baseline leg
are the only callers.  The CUDA library and its Python binding never import this package.

The arithmetic lives in ``oracle.c`` (plain C, binary64 for continuous quantities, binary32 for
every discrete decision as the written spec fixes it).  This module compiles it with gcc and
marshals numpy arrays through ctypes.  Functions and the paper passage each one follows:

* :func:`primary_ray` -- the ray ``r = o + d t`` of a pixel (Eq. 1, spec S1).
* :func:`raycast` -- the server's volume ray marcher with the first-hit depth heuristic
  (§4.1, §4.2, Fig. 2; the heuristic itself is cited from earlier work, §2) and the readings of
  the other heuristics of §2 and §5 (max contribution, accumulated opacity, max gradient; S2a).
* :func:`unproject` -- object-space samples ``p = o + d t_i`` (Eq. 1), footprint radius (§4.1),
  zero-radius compaction (§4.1).
* :func:`unproject_interval` -- samples smeared along their viewing ray over the depth interval
  of growing opacity, as chains of touching spheres (future work, §6; reading: spec S3b).
* :func:`append_frame`, :func:`accumulate` -- splats of several server frames in one set, the
  accumulation over frames named as future work in §6 (reading: spec S3a).
* :func:`point_splat` -- the earlier warping the paper compares against (§2, §5, Fig. 3): each
  sample drawn as a fixed-size pixel square with one depth per point (reading: spec S10).
* :func:`psnr` -- the image-quality measure used to restate Fig. 3 numerically (spec S10).
* :func:`encode`, :func:`decode` -- the 64-bit quantised position + radius word and the 32-bit
  colour the server sends (§4.1, §6; bit layout: reading of spec S11).
* :func:`trace` -- first-hit / multi-hit ray tracing of the samples as semi-transparent spheres
  with constant colour (Fig. 2 caption, §4), front-to-back compositing (spec S6).
* :func:`trace64` -- the same trace with every decision in binary64, and which pixels are ties
  (a move of at most 1e-6 can change their hit list): the exclusion list of the parity budget.
* :func:`trace_backward` -- the adjoint of that compositing (spec S7; not in the paper).
* :func:`lbvh` -- Morton codes, sorted order and the binary radix tree of the LBVH (§4.1, §4.2).

Every function here is pinned by ``tests/test_oracle_*.py`` against closed forms, invariants and
brute force, never against the CUDA path.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

CFLAGS = ["-O2", "-fPIC", "-shared", "-pthread", "-std=gnu11", "-ffp-contract=off",
          "-frounding-math", "-fno-fast-math"]

RADIUS_FOOTPRINT = 0
RADIUS_VOXEL = 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, no GPU needed)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Cam(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3),
                ("tan_half_fovy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class _Scene(ctypes.Structure):
    _fields_ = [("pos_r", ctypes.c_void_p), ("rgba", ctypes.c_void_p), ("id", ctypes.c_void_p),
                ("n", ctypes.c_int64), ("scale", ctypes.c_void_p), ("global_scale", ctypes.c_float),
                ("opacity", ctypes.c_void_p), ("max_hits", ctypes.c_int32),
                ("t_stop", ctypes.c_double), ("beta", ctypes.c_double)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.orc_primary_ray.argtypes = [ctypes.POINTER(_Cam), ctypes.c_int, ctypes.c_int, P, P]
        lib.orc_raycast.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, P,
                                    ctypes.POINTER(_Cam), ctypes.c_float, ctypes.c_float, P,
                                    ctypes.c_int64, P, P, ctypes.c_int]
        lib.orc_raycast_heuristic.argtypes = [P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              P, ctypes.POINTER(_Cam), ctypes.c_float, ctypes.c_int,
                                              ctypes.c_float, P, ctypes.c_int64, P, P, ctypes.c_int]
        lib.orc_unproject.argtypes = [P, P, ctypes.POINTER(_Cam), ctypes.c_int, ctypes.c_float,
                                      P, P, P, ctypes.c_int64]
        lib.orc_unproject.restype = ctypes.c_int64
        lib.orc_bvh_build.argtypes = [P, P, ctypes.c_float, ctypes.c_int64, ctypes.c_int]
        lib.orc_bvh_build.restype = P
        lib.orc_bvh_free.argtypes = [P]
        lib.orc_trace.argtypes = [ctypes.POINTER(_Scene), P, ctypes.POINTER(_Cam), P,
                                  ctypes.c_int64, P, P, P, P, P, P, ctypes.c_int]
        lib.orc_primary_ray64.argtypes = [ctypes.POINTER(_Cam), ctypes.c_int, ctypes.c_int, P, P]
        lib.orc_trace64.argtypes = [ctypes.POINTER(_Scene), P, ctypes.POINTER(_Cam), P,
                                    ctypes.c_int64, ctypes.c_double, P, P, P, P, P, ctypes.c_int]
        lib.orc_trace_backward.argtypes = [ctypes.POINTER(_Scene), P, ctypes.POINTER(_Cam), P, P,
                                           P, P, ctypes.c_int]
        lib.orc_lbvh.argtypes = [P, P, ctypes.c_float, ctypes.c_int64, ctypes.c_int32, P, P, P, P,
                                 P, P]
        lib.orc_point_splat.argtypes = [P, P, ctypes.c_int64, ctypes.POINTER(_Cam), ctypes.c_int, P, P]
        lib.orc_unproject_interval.argtypes = [P, P, P, ctypes.POINTER(_Cam), ctypes.c_int,
                                               ctypes.c_float, ctypes.c_int, P, P, P, ctypes.c_int64]
        lib.orc_unproject_interval.restype = ctypes.c_int64
        lib.orc_encode.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_float, P, P]
        lib.orc_decode.argtypes = [P, P, ctypes.c_int64, P, P, ctypes.c_float, P, P]
        lib.orc_default_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def default_threads() -> int:
    return int(_load().orc_default_threads())


def _cam(cam) -> _Cam:
    c = _Cam()
    for f in ("eye", "right", "up", "fwd"):
        v = np.asarray(getattr(cam, f), dtype=np.float32)
        getattr(c, f)[:] = [float(x) for x in v]
    c.tan_half_fovy = float(np.float32(cam.tan_half_fovy))
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data


def _c(a, dtype) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=dtype)


def primary_ray(cam, x: int, y: int):
    """Spec S1 ray of pixel (x, y): returns (o, d) as float32[3] arrays."""
    o = np.zeros(3, np.float32)
    d = np.zeros(3, np.float32)
    _load().orc_primary_ray(ctypes.byref(_cam(cam)), int(x), int(y), o.ctypes.data, d.ctypes.data)
    return o, d


DEPTH_FIRST_HIT = 0
DEPTH_MAX_CONTRIBUTION = 1
DEPTH_ACCUMULATED = 2
DEPTH_MAX_GRADIENT = 3


def raycast(vol: np.ndarray, tf: np.ndarray, cam, step_vox: float = 0.5, tau: float = 0.1,
            pixels: Optional[np.ndarray] = None, threads: int = 0, heuristic: int = DEPTH_FIRST_HIT,
            param: Optional[float] = None):
    """Server volume ray caster + depth heuristic (spec S2; other heuristics: S2a).

    vol: [nz, ny, nx] float32 in [0,1] or uint8.  ``param``: tau of the first-hit heuristic
    (default ``tau``), theta of the accumulated-opacity heuristic (default 0.5), unused otherwise.
    Returns (rgba float64 [npix,4] premultiplied, depth float32 [npix]) for ``pixels`` (flat
    indices y*W+x), or images [H,W,4] / [H,W] if None.
    """
    lib = _load()
    if vol.dtype == np.uint8:
        dtype = 1
    else:
        dtype = 0
        vol = _c(vol, np.float32)
    vol = np.ascontiguousarray(vol)
    nz, ny, nx = vol.shape
    tf = _c(tf, np.float32)
    assert tf.shape == (256, 4)
    if param is None:
        param = 0.5 if heuristic == DEPTH_ACCUMULATED else tau
    if pixels is None:
        npix = cam.width * cam.height
        pix = None
    else:
        pix = _c(pixels, np.int32)
        npix = pix.size
    rgba = np.zeros((npix, 4), np.float64)
    depth = np.zeros(npix, np.float32)
    rc = lib.orc_raycast_heuristic(vol.ctypes.data, dtype, nx, ny, nz, tf.ctypes.data,
                                   ctypes.byref(_cam(cam)), float(step_vox), int(heuristic),
                                   float(param), _ptr(pix), int(npix), rgba.ctypes.data,
                                   depth.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("orc_raycast_heuristic: bad arguments")
    if pixels is None:
        return rgba.reshape(cam.height, cam.width, 4), depth.reshape(cam.height, cam.width)
    return rgba, depth


@dataclass
class Splats:
    """Compacted splats in server-pixel order: pos_r [N,4] (x,y,z,r0), rgba [N,4], id [N]."""
    pos_r: np.ndarray
    rgba: np.ndarray
    id: np.ndarray

    @property
    def n(self) -> int:
        return int(self.id.shape[0])


def unproject(rgba: np.ndarray, depth: np.ndarray, cam, mode: int = RADIUS_FOOTPRINT,
              voxel_diag: float = 0.0) -> Splats:
    """Eq. 1 unprojection with footprint / voxel radius and stable compaction (spec S3)."""
    rgba = _c(rgba, np.float32).reshape(-1, 4)
    depth = _c(depth, np.float32).reshape(-1)
    cap = depth.size
    pos_r = np.zeros((cap, 4), np.float32)
    out = np.zeros((cap, 4), np.float32)
    ids = np.zeros(cap, np.uint32)
    n = _load().orc_unproject(rgba.ctypes.data, depth.ctypes.data, ctypes.byref(_cam(cam)), int(mode),
                              float(voxel_diag), pos_r.ctypes.data, out.ctypes.data, ids.ctypes.data,
                              cap)
    if n < 0:
        raise ValueError(f"orc_unproject failed ({n})")
    return Splats(pos_r[:n].copy(), out[:n].copy(), ids[:n].copy())


def unproject_interval(rgba: np.ndarray, depth_lo: np.ndarray, depth_hi: np.ndarray, cam,
                       mode: int = RADIUS_FOOTPRINT, voxel_diag: float = 0.0,
                       max_chain: int = 8) -> Splats:
    """Each kept pixel as a chain of spheres along its server ray over [depth_lo, depth_hi]
    (spec S3b); ids = pixel * max_chain + position in the chain."""
    rgba = _c(rgba, np.float32).reshape(-1, 4)
    lo = _c(depth_lo, np.float32).reshape(-1)
    hi = _c(depth_hi, np.float32).reshape(-1)
    cap = lo.size * int(max_chain)
    pos_r = np.zeros((cap, 4), np.float32)
    out = np.zeros((cap, 4), np.float32)
    ids = np.zeros(cap, np.uint32)
    n = _load().orc_unproject_interval(rgba.ctypes.data, lo.ctypes.data, hi.ctypes.data,
                                       ctypes.byref(_cam(cam)), int(mode), float(voxel_diag),
                                       int(max_chain), pos_r.ctypes.data, out.ctypes.data,
                                       ids.ctypes.data, cap)
    if n < 0:
        raise ValueError(f"orc_unproject_interval failed ({n})")
    return Splats(pos_r[:n].copy(), out[:n].copy(), ids[:n].copy())


STATUS_SPLAT_OVERFLOW = 8
AMB_STOP64 = 4  # trace()["amb"] bit: a binary64 transmittance would stop at another hit


def append_frame(acc: Optional[Splats], rgba: np.ndarray, depth: np.ndarray, cam, weight: float = 1.0,
                 id_base: int = 0, capacity: Optional[int] = None, mode: int = RADIUS_FOOTPRINT,
                 voxel_diag: float = 0.0):
    """Append one server frame's splats to ``acc`` (spec S3a; accumulation over frames, §6).

    Steps in the reading's order: the frame's kept pixels by the unprojection rule (S3); ids
    shifted by ``id_base``; colours scaled by ``weight`` in binary32; appended after the current
    records; records beyond ``capacity`` dropped.  Returns ``(splats, overflow)``."""
    new = unproject(rgba, depth, cam, mode, voxel_diag)
    w = np.float32(weight)
    col = new.rgba if w == np.float32(1.0) else (new.rgba * w).astype(np.float32)
    ids = new.id.astype(np.uint64) + np.uint64(id_base)
    if ids.size and int(ids.max()) >= 2**32:
        raise ValueError("id_base + pixel index exceeds 32 bits")
    if acc is None:
        acc = Splats(np.zeros((0, 4), np.float32), np.zeros((0, 4), np.float32), np.zeros(0, np.uint32))
    pos_r = np.concatenate([acc.pos_r, new.pos_r])
    col = np.concatenate([acc.rgba, col])
    ids = np.concatenate([acc.id, ids.astype(np.uint32)])
    overflow = capacity is not None and ids.shape[0] > capacity
    if overflow:
        pos_r, col, ids = pos_r[:capacity], col[:capacity], ids[:capacity]
    return Splats(pos_r.copy(), col.copy(), ids.copy()), overflow


def window_weights(frames: int, decay: float = 1.0) -> np.ndarray:
    """Weight of the frame of age g (0 = newest): decay^g by repeated binary32 multiplication."""
    w = np.ones(frames, np.float32)
    for g in range(1, frames):
        w[g] = np.float32(w[g - 1] * np.float32(decay))
    return w


def accumulate(frames, decay: float = 1.0, mode: int = RADIUS_FOOTPRINT,
               voxel_diag: float = 0.0) -> Splats:
    """The splat set of a window of server frames (spec S3a).  ``frames`` = [(rgba, depth, cam)]
    ordered newest first; the frame of age g is appended with weight decay^g and ids offset by
    g * Ws * Hs, so that newer frames come first and win ties of equal hit distance."""
    acc = None
    w = window_weights(len(frames), decay)
    for g, (rgba, depth, cam) in enumerate(frames):
        npix = int(np.asarray(depth).size)
        acc, _ = append_frame(acc, rgba, depth, cam, float(w[g]), g * npix, None, mode, voxel_diag)
    return acc


def point_splat(splats: Splats, cam, size: int = 1):
    """Point-splat warping of the splats into the client camera (spec S10): returns (rgba float32
    [H, W, 4], index int64 [H, W] of the point each pixel shows, -1 where none)."""
    pos_r = _c(splats.pos_r, np.float32)
    rgba = _c(splats.rgba, np.float32)
    out = np.zeros((cam.height, cam.width, 4), np.float32)
    idx = np.zeros((cam.height, cam.width), np.int64)
    rc = _load().orc_point_splat(pos_r.ctypes.data, rgba.ctypes.data, splats.n, ctypes.byref(_cam(cam)),
                                 int(size), out.ctypes.data, idx.ctypes.data)
    if rc != 0:
        raise ValueError(f"orc_point_splat failed ({rc})")
    return out, idx


def psnr(img: np.ndarray, ref: np.ndarray) -> float:
    """10 log10(1 / MSE) over all channels of images with values in [0, 1] (binary64)."""
    mse = float(np.mean((np.asarray(img, np.float64) - np.asarray(ref, np.float64)) ** 2))
    return float("inf") if mse == 0.0 else 10.0 * np.log10(1.0 / mse)


def encode(splats: Splats, lo, hi, r_max: float):
    """Quantise splats into 64-bit position + radius words and 32-bit colours (spec S11).
    Returns (word uint64 [N], color uint32 [N])."""
    pos_r = _c(splats.pos_r, np.float32)
    rgba = _c(splats.rgba, np.float32)
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    word = np.zeros(splats.n, np.uint64)
    color = np.zeros(splats.n, np.uint32)
    if _load().orc_encode(pos_r.ctypes.data, rgba.ctypes.data, splats.n, lo.ctypes.data, hi.ctypes.data,
                          float(r_max), word.ctypes.data, color.ctypes.data) != 0:
        raise ValueError("orc_encode: bad box or radius bound")
    return word, color


def decode(word: np.ndarray, color: np.ndarray, lo, hi, r_max: float) -> Splats:
    """Splats from the words and colours of :func:`encode` (spec S11); id = stream index."""
    word = _c(word, np.uint64)
    color = _c(color, np.uint32)
    lo = _c(lo, np.float32)
    hi = _c(hi, np.float32)
    n = word.size
    pos_r = np.zeros((n, 4), np.float32)
    rgba = np.zeros((n, 4), np.float32)
    if _load().orc_decode(word.ctypes.data, color.ctypes.data, n, lo.ctypes.data, hi.ctypes.data,
                          float(r_max), pos_r.ctypes.data, rgba.ctypes.data) != 0:
        raise ValueError("orc_decode failed")
    return Splats(pos_r, rgba, np.arange(n, dtype=np.uint32))


@dataclass
class Scene:
    """Everything the compositing reads: splats + per-splat parameters + compositing settings."""
    splats: Splats
    scale: Optional[np.ndarray] = None    # per-splat radius scale (compacted order) or None
    global_scale: float = 1.0
    opacity: Optional[np.ndarray] = None  # per-splat opacity or None (= 1)
    max_hits: int = 0                     # H: 1 = first hit (the paper), 0 = all hits
    t_stop: float = 1e-5
    beta: float = 0.0                     # soft-edge width (0 = hard spheres)

    def _c(self):
        self._keep = [_c(self.splats.pos_r, np.float32), _c(self.splats.rgba, np.float32),
                      _c(self.splats.id, np.uint32),
                      None if self.scale is None else _c(self.scale, np.float32),
                      None if self.opacity is None else _c(self.opacity, np.float32)]
        k = self._keep
        return _Scene(_ptr(k[0]), _ptr(k[1]), _ptr(k[2]), self.splats.n, _ptr(k[3]),
                      float(self.global_scale), _ptr(k[4]), int(self.max_hits), float(self.t_stop),
                      float(self.beta))


class BVH:
    """The oracle's own top-down median-split BVH (an accelerator only: images equal brute force)."""

    def __init__(self, scene: Scene, leaf: int = 4):
        self._keep = [_c(scene.splats.pos_r, np.float32),
                      None if scene.scale is None else _c(scene.scale, np.float32)]
        self.h = _load().orc_bvh_build(_ptr(self._keep[0]), _ptr(self._keep[1]),
                                       float(scene.global_scale), scene.splats.n, int(leaf))

    def __del__(self):
        if getattr(self, "h", None):
            _load().orc_bvh_free(self.h)
            self.h = None


def trace(scene: Scene, cam, pixels: Optional[np.ndarray] = None, bvh="auto", threads: int = 0):
    """Trace the client camera's rays through the spheres (spec S5, S6).

    Returns dict: rgba float64 [npix,4] (premultiplied), T [npix], nused [npix] (hits composited),
    nhits [npix] (all hits), amb [npix] (bit 1: a binary64 hit test would disagree, bit 2: a binary64
    key would reorder the hits, bit 4: the binary64 transmittance would stop at another hit than
    the binary32 one the decision uses -- diagnostics of the binary32 reading, not exclusions;
    a bit-4 pixel's image moves by about T_stop at most, the adjoint of its alpha by the later
    hit's full weight), hash [npix] (FNV-1a of the ids of the composited hits, in order).
    ``bvh``: "auto" builds the oracle BVH, None = brute force, or a :class:`BVH`.
    """
    lib = _load()
    if isinstance(bvh, str):
        bvh = BVH(scene) if scene.splats.n > 0 else None
    if pixels is None:
        npix = cam.width * cam.height
        pix = None
    else:
        pix = _c(pixels, np.int32)
        npix = pix.size
    rgba = np.zeros((npix, 4), np.float64)
    T = np.zeros(npix, np.float64)
    nused = np.zeros(npix, np.int32)
    nhits = np.zeros(npix, np.int32)
    amb = np.zeros(npix, np.uint8)
    hsh = np.zeros(npix, np.uint64)
    sc = scene._c()
    rc = lib.orc_trace(ctypes.byref(sc), None if bvh is None else bvh.h, ctypes.byref(_cam(cam)),
                       _ptr(pix), int(npix), rgba.ctypes.data, T.ctypes.data, nused.ctypes.data,
                       nhits.ctypes.data, amb.ctypes.data, hsh.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("orc_trace failed")
    return {"rgba": rgba, "T": T, "nused": nused, "nhits": nhits, "amb": amb, "hash": hsh}


TIE = 1e-6  # decision margin (scene units: the volume is the unit cube) below which a pixel is a tie


def primary_ray64(cam, x: int, y: int):
    """The ray of pixel (x, y) evaluated in binary64 from the camera's fields (spec S1):
    returns (o, d) as float64[3] arrays."""
    o = np.zeros(3, np.float64)
    d = np.zeros(3, np.float64)
    _load().orc_primary_ray64(ctypes.byref(_cam(cam)), int(x), int(y), o.ctypes.data, d.ctypes.data)
    return o, d


def trace64(scene: Scene, cam, pixels: Optional[np.ndarray] = None, bvh="auto", tie: float = TIE,
            threads: int = 0):
    """:func:`trace` with every decision in binary64: the primary ray, hit or miss, entry
    distance and hit order (Fig. 2 caption, §4; spec S5, S6 evaluated in double).

    Returns dict: rgba float64 [npix,4], T, nused, nhits as :func:`trace`, ``tie_kind`` [npix]
    uint8 and ``tie`` [npix] bool (= tie_kind != 0).  A pixel is a tie when moving the ray or a
    sphere by at most ``tie`` (scene units; the volume is the unit cube) can change which
    spheres it composites or their order: bit 1 a composited sphere can be missed, bit 2 two
    entry distances can swap (one of them among the composited hits), bit 4 a missed sphere can
    be hit in front of the point where compositing stopped.  Only tie pixels can differ between
    this image and one whose decisions are taken in another precision.
    """
    lib = _load()
    if isinstance(bvh, str):
        bvh = BVH(scene) if scene.splats.n > 0 else None
    if pixels is None:
        npix = cam.width * cam.height
        pix = None
    else:
        pix = _c(pixels, np.int32)
        npix = pix.size
    rgba = np.zeros((npix, 4), np.float64)
    T = np.zeros(npix, np.float64)
    nused = np.zeros(npix, np.int32)
    nhits = np.zeros(npix, np.int32)
    kind = np.zeros(npix, np.uint8)
    sc = scene._c()
    rc = lib.orc_trace64(ctypes.byref(sc), None if bvh is None else bvh.h, ctypes.byref(_cam(cam)),
                         _ptr(pix), int(npix), float(tie), rgba.ctypes.data, T.ctypes.data,
                         nused.ctypes.data, nhits.ctypes.data, kind.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("orc_trace64 failed")
    return {"rgba": rgba, "T": T, "nused": nused, "nhits": nhits, "tie_kind": kind, "tie": kind != 0}


def trace_backward(scene: Scene, cam, dL_dimg: np.ndarray, bvh="auto", threads: int = 0):
    """Adjoint of :func:`trace` (spec S7): returns (g_rgba [N,4], g_opacity [N], g_scale [N])
    in compacted splat order, for the upstream gradient dL_dimg [H*W,4] (float64)."""
    lib = _load()
    if isinstance(bvh, str):
        bvh = BVH(scene) if scene.splats.n > 0 else None
    n = scene.splats.n
    g = _c(dL_dimg, np.float64).reshape(-1, 4)
    assert g.shape[0] == cam.width * cam.height
    gr = np.zeros((max(n, 1), 4), np.float64)
    go = np.zeros(max(n, 1), np.float64)
    gs = np.zeros(max(n, 1), np.float64)
    sc = scene._c()
    rc = lib.orc_trace_backward(ctypes.byref(sc), None if bvh is None else bvh.h,
                                ctypes.byref(_cam(cam)), g.ctypes.data, gr.ctypes.data,
                                go.ctypes.data, gs.ctypes.data, int(threads))
    if rc != 0:
        raise ValueError("orc_trace_backward failed")
    return gr[:n], go[:n], gs[:n]


def lbvh(pos_r: np.ndarray, scale: Optional[np.ndarray] = None, global_scale: float = 1.0,
         leaf: int = 1):
    """LBVH reference (spec S8): Morton codes, stable order, radix-tree children, child boxes.

    Returns dict: codes (sorted, uint32 [N]), order (uint32 [N], sorted -> compacted index),
    child (int32 [M-1, 2], bit 31 set = leaf index), boxes (float32 [M-1, 2, 6]: child lo xyz, hi xyz),
    root (int32), cbounds (float32 [6]).
    """
    pos_r = _c(pos_r, np.float32)
    n = pos_r.shape[0]
    M = (n + leaf - 1) // leaf
    codes = np.zeros(n, np.uint32)
    order = np.zeros(n, np.uint32)
    child = np.zeros((max(M - 1, 1), 2), np.int32)
    boxes = np.zeros((max(M - 1, 1), 2, 6), np.float32)
    root = np.zeros(1, np.int32)
    cb = np.zeros(6, np.float32)
    sc = None if scale is None else _c(scale, np.float32)
    rc = _load().orc_lbvh(pos_r.ctypes.data, _ptr(sc), float(global_scale), n, int(leaf),
                          codes.ctypes.data, order.ctypes.data, child.ctypes.data, boxes.ctypes.data,
                          root.ctypes.data, cb.ctypes.data)
    if rc != 0:
        raise ValueError("orc_lbvh failed")
    return {"codes": codes, "order": order, "child": child[:M - 1], "boxes": boxes[:M - 1],
            "root": int(root[0]), "cbounds": cb}
