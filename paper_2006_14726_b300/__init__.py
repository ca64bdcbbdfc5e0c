"""Python binding of libwrs: ray-traced sphere-splat image warping on B300 (sm_103a).

Zellmann, "Augmenting Image Warping-Based Remote Volume Rendering with Ray Tracing" (2020):
each pixel of a server-rendered colour + depth image becomes an object-space sphere (Eq. 1,
§4.1), an LBVH is built over the spheres (§4.1, §4.2), and every client frame ray-traces them
from the newer camera, compositing the hits front to back (Fig. 2 caption, §4).

This module only marshals arguments: every step runs in the CUDA kernels of ``libwrs.so``
(built from ``csrc/`` by ``python paper_2006_14726_b300/_build.py``).  PyTorch provides device
memory and streams.  There is no CPU fallback: importing this package without the built library
raises ImportError, and every call needs CUDA tensors.

Entry points (same names as the C ABI in ``include/wrs.h``): :func:`raycast_volume`,
:func:`unproject`, :func:`build_lbvh`, :func:`trace`, :func:`trace_count`, :func:`trace_batched`,
:func:`trace_backward`, plus :class:`TraceFunction` (torch.autograd) and :mod:`.autotune`.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import List, Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libwrs.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2006_14726_b300/_build.py` "
                      "(there is no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

WRS_OK = 0
WRS_ERR_ARG = -1
WRS_ERR_CUDA = -2
WRS_ERR_CAPACITY = -3
WRS_ERR_SCRATCH = -4
WRS_ERR_DEVICE = -5
STATUS_STACK_OVERFLOW = 1
STATUS_CHUNK_OVERFLOW = 2
STATUS_MALFORMED_TREE = 4
STATUS_SPLAT_OVERFLOW = 8
F32 = 0
U8 = 1
RADIUS_FOOTPRINT = 0
RADIUS_VOXEL = 1
SCHEDULE_PER_PIXEL = 0
SCHEDULE_PERSISTENT = 1
SCHEDULE_PACKET = 2
SCHEDULE_PER_SESSION = 3  # trace_batched only: each session's own schedule (Batch(schedules=...))
LBVH_FULL = 0  # tree layouts: binary records and 4-wide nodes (any traversal)
LBVH_WIDE = 1  # the 4-wide nodes only (width 4 or the packet schedule); a faster build
DEPTH_FIRST_HIT = 0
DEPTH_MAX_CONTRIBUTION = 1
DEPTH_ACCUMULATED = 2
DEPTH_MAX_GRADIENT = 3


class WrsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"[{code}] {msg}")
        self.code = code


class Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("right", ctypes.c_float * 3),
                ("up", ctypes.c_float * 3), ("fwd", ctypes.c_float * 3),
                ("tan_half_fovy", ctypes.c_float), ("width", ctypes.c_int32),
                ("height", ctypes.c_int32)]


class _Splats(ctypes.Structure):
    _fields_ = [("pos_r", ctypes.c_void_p), ("rgba", ctypes.c_void_p), ("id", ctypes.c_void_p),
                ("src", ctypes.c_void_p), ("n", ctypes.c_void_p), ("capacity", ctypes.c_uint32)]


class _Lbvh(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("capacity", ctypes.c_uint32),
                ("leaf_size", ctypes.c_uint32), ("layout", ctypes.c_uint32)]


class _Params(ctypes.Structure):
    _fields_ = [("max_hits", ctypes.c_int32), ("t_stop", ctypes.c_float),
                ("edge_softness", ctypes.c_float), ("opacity", ctypes.c_void_p),
                ("k_chunk", ctypes.c_int32), ("block", ctypes.c_int32),
                ("schedule", ctypes.c_int32), ("width", ctypes.c_int32)]


class Codec(ctypes.Structure):
    """wrs_codec: quantisation box and radius bound of the 64-bit splat word."""
    _fields_ = [("lo", ctypes.c_float * 3), ("hi", ctypes.c_float * 3), ("r_max", ctypes.c_float)]


def make_codec(lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), r_max: float = 0.01) -> Codec:
    c = Codec()
    c.lo[:] = [float(x) for x in lo]
    c.hi[:] = [float(x) for x in hi]
    c.r_max = float(r_max)
    return c


class Session(ctypes.Structure):
    _fields_ = [("nodes", ctypes.c_void_p), ("pos_r", ctypes.c_void_p), ("rgba", ctypes.c_void_p),
                ("id", ctypes.c_void_p), ("src", ctypes.c_void_p), ("opacity", ctypes.c_void_p),
                ("rgba_out", ctypes.c_void_p), ("cam", Camera), ("tile_begin", ctypes.c_uint32),
                ("schedule", ctypes.c_uint32)]


def _sig(name, res, *args):
    if not hasattr(_lib, name):
        raise ImportError(f"{LIB_PATH} lacks {name}: it is out of date; rebuild it with "
                          "`python paper_2006_14726_b300/_build.py`")
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = list(args)
    return f


_P = ctypes.c_void_p
_I = ctypes.c_int32
_U = ctypes.c_uint32
_F = ctypes.c_float
_Z = ctypes.c_size_t
_sig("wrs_version", ctypes.c_char_p)
_sig("wrs_last_error", ctypes.c_char_p)
_sig("wrs_session_size", _Z)
_sig("wrs_camera_size", _Z)
_sig("wrs_check_status", _I, _P, _P)
_sig("wrs_window_weight", _F, _F, _U)
_sig("wrs_raycast_volume", _I, _P, _I, _I, _I, _I, _P, ctypes.POINTER(Camera), _F, _F, _P, _P, _P)
_sig("wrs_raycast_volume_heuristic", _I, _P, _I, _I, _I, _I, _P, ctypes.POINTER(Camera), _F, _I, _F,
     _P, _P, _P)
_sig("wrs_unproject_scratch_bytes", _Z, _I, _I)
_sig("wrs_unproject", _I, _P, _P, ctypes.POINTER(Camera), _I, _F, ctypes.POINTER(_Splats), _P, _Z, _P)
_sig("wrs_unproject_append", _I, _P, _P, ctypes.POINTER(Camera), _I, _F, _F, _U,
     ctypes.POINTER(_Splats), _P, _Z, _P, _P)
_sig("wrs_unproject_encode", _I, _P, _P, ctypes.POINTER(Camera), _I, _F, ctypes.POINTER(Codec), _P, _P,
     _P, _U, _P, _Z, _P)
_sig("wrs_encode_splats", _I, ctypes.POINTER(_Splats), ctypes.POINTER(Codec), _P, _P, _P, _P)
_sig("wrs_decode_splats", _I, _P, _P, _P, _U, ctypes.POINTER(Codec), ctypes.POINTER(_Splats), _P)
_sig("wrs_point_splat_scratch_bytes", _Z, _I, _I)
_sig("wrs_point_splat", _I, ctypes.POINTER(_Splats), ctypes.POINTER(Camera), _I, _P, _P, _P, _Z, _P)
_sig("wrs_unproject_interval", _I, _P, _P, _P, ctypes.POINTER(Camera), _I, _F, _I,
     ctypes.POINTER(_Splats), _P, _Z, _P, _P)
_sig("wrs_unproject_static", _I, _P, _P, ctypes.POINTER(Camera), _I, _F, ctypes.POINTER(_Splats), _P)
_sig("wrs_lbvh_bytes", _Z, _U, _U)
_sig("wrs_lbvh_scratch_bytes", _Z, _U, _U)
_sig("wrs_build_lbvh", _I, ctypes.POINTER(_Splats), _P, _F, ctypes.POINTER(_Lbvh),
     ctypes.POINTER(_Splats), _P, _Z, _P)
_sig("wrs_refit_lbvh", _I, ctypes.POINTER(_Splats), _P, _F, ctypes.POINTER(_Lbvh),
     ctypes.POINTER(_Splats), _P, _Z, _P)
_sig("wrs_trace", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats), ctypes.POINTER(Camera),
     ctypes.POINTER(_Params), _P, _P, _P)
_sig("wrs_trace_count", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats), ctypes.POINTER(Camera),
     ctypes.POINTER(_Params), _P, _P, _P)
_sig("wrs_fma_peak", _I, _P, _I, _I, _P)
_sig("wrs_stream_copy", _I, _P, _P, _Z, _I, _I, _P)
_sig("wrs_trace_views", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats), ctypes.POINTER(Camera),
     _I, ctypes.POINTER(_Params), _P, _P, _P)
_sig("wrs_trace_backward_views", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats),
     ctypes.POINTER(Camera), _I, ctypes.POINTER(_Params), _P, _F, _P, _P, _P, _P, _I, _P, _P)
_sig("wrs_trace_views_record", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats),
     ctypes.POINTER(Camera), _I, ctypes.POINTER(_Params), _P, _P, _P, _U, _P, _P)
_sig("wrs_trace_backward_views_recorded", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats),
     ctypes.POINTER(Camera), _I, ctypes.POINTER(_Params), _P, _F, _P, _P, _U, _P, _P, _P, _P, _I,
     _P, _P)
_sig("wrs_session_tiles", _U, _I, _I)
_sig("wrs_trace_batched", _I, _P, _I, _U, ctypes.POINTER(_Params), _P, _P, _P)
_sig("wrs_trace_backward", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats), ctypes.POINTER(Camera),
     ctypes.POINTER(_Params), _P, _F, _P, _P, _P, _P, _P, _P)
_sig("wrs_trace_backward_accumulate", _I, ctypes.POINTER(_Lbvh), ctypes.POINTER(_Splats),
     ctypes.POINTER(Camera), ctypes.POINTER(_Params), _P, _F, _P, _P, _P, _P, _P, _P)

lib = _lib
assert _lib.wrs_session_size() == ctypes.sizeof(Session), "wrs_session layout mismatch"
assert _lib.wrs_camera_size() == ctypes.sizeof(Camera), "wrs_camera layout mismatch"


def version() -> str:
    return _lib.wrs_version().decode()


def last_error() -> str:
    return _lib.wrs_last_error().decode()


def _check(rc: int, fn: str):
    if rc != WRS_OK:
        raise WrsError(rc, f"{fn}: {last_error()}")


_raw_stream = getattr(torch._C, "_cuda_getCurrentRawStream", None)
_cur_device = getattr(torch._C, "_cuda_getDevice", None)


def _stream(stream) -> Optional[int]:
    """The cudaStream_t handle: ``stream`` (a torch.cuda.Stream or a raw handle), else torch's
    current stream of the current device (read without building a Stream object: the lookup is
    on every call of every entry point)."""
    if stream is None:
        if _raw_stream is not None and _cur_device is not None:
            return _raw_stream(_cur_device())
        stream = torch.cuda.current_stream()
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libwrs takes CUDA tensors only (there is no CPU path)")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _buf(t: Optional[torch.Tensor], numel: int, dtype, what: str) -> Optional[torch.Tensor]:
    """A caller-provided output/input buffer the kernels index by the camera's size: it must be a
    contiguous CUDA tensor of the given dtype with at least ``numel`` elements (the C ABI takes a
    raw pointer and cannot check this)."""
    if t is None:
        return None
    if t.dtype != dtype:
        raise ValueError(f"{what}: dtype {t.dtype}, expected {dtype}")
    if t.numel() < numel:
        raise ValueError(f"{what}: {t.numel()} elements, at least {numel} needed")
    _ptr(t)
    return t


def make_camera(cam) -> Camera:
    """Any object with eye/right/up/fwd/tan_half_fovy/width/height -> the C struct."""
    c = Camera()
    for f in ("eye", "right", "up", "fwd"):
        getattr(c, f)[:] = [float(x) for x in getattr(cam, f)]
    c.tan_half_fovy = float(cam.tan_half_fovy)
    c.width = int(cam.width)
    c.height = int(cam.height)
    return c


def _cam(cam) -> Camera:
    return cam if isinstance(cam, Camera) else make_camera(cam)


# ----------------------------------------------------------------------------------------------
# buffers
# ----------------------------------------------------------------------------------------------
class SplatBuffers:
    """Device splat set (see wrs_splats): pos_r [cap,4], rgba [cap,4], id [cap], src [cap], n [1].

    ``id`` and ``src`` are int32 tensors holding uint32 values (< 2^31)."""

    def __init__(self, capacity: int, device=None, sorted: bool = False, _fill: bool = True):
        device = device or torch.device("cuda")
        cap = max(int(capacity), 1)
        self.capacity = int(capacity)
        # zero-filled (count 0) unless a producer writes count and rows before any reader runs
        new = torch.zeros if _fill else torch.empty
        self.pos_r = new(cap, 4, dtype=torch.float32, device=device)
        self.rgba = new(cap, 4, dtype=torch.float32, device=device)
        self.id = new(cap, dtype=torch.int32, device=device)
        self.src = new(cap, dtype=torch.int32, device=device) if sorted else None
        self.n = new(1, dtype=torch.int32, device=device)

    def c(self) -> _Splats:
        return _Splats(_ptr(self.pos_r), _ptr(self.rgba), _ptr(self.id), _ptr(self.src),
                       _ptr(self.n), self.capacity)

    def count(self) -> int:
        return int(self.n.item())

    def view(self):
        """(pos_r, rgba, id[, src]) trimmed to the current count (synchronises)."""
        k = self.count()
        out = [self.pos_r[:k], self.rgba[:k], self.id[:k]]
        if self.src is not None:
            out.append(self.src[:k])
        return tuple(out)


class LBVH:
    """Device LBVH buffer (see wrs_lbvh).  ``layout``: :data:`LBVH_FULL` (binary records and
    4-wide nodes) or :data:`LBVH_WIDE` (4-wide nodes only: traced with width 4 or the packet
    schedule; the build skips most binary records)."""

    def __init__(self, capacity: int, leaf_size: int = 1, device=None, _fill: bool = True,
                 layout: int = LBVH_FULL):
        device = device or torch.device("cuda")
        nbytes = _lib.wrs_lbvh_bytes(int(capacity), int(leaf_size))
        if nbytes == 0:
            raise ValueError(f"leaf_size {leaf_size} not in 1..16")
        self.capacity = int(capacity)
        self.leaf_size = int(leaf_size)
        self.layout = int(layout)
        # zero-filled (an empty tree) unless a build writes the header before any reader runs
        self.nodes = (torch.zeros if _fill else torch.empty)(nbytes, dtype=torch.uint8, device=device)

    def c(self) -> _Lbvh:
        return _Lbvh(_ptr(self.nodes), self.capacity, self.leaf_size, self.layout)

    def header(self) -> dict:
        h = self.nodes[:64].cpu()
        u = h.view(torch.int32)
        f = h.view(torch.float32)
        return {"n": int(u[0]), "m": int(u[1]), "leaf": int(u[2]), "root": int(u[3]),
                "cmin": f[4:7].tolist(), "cmax": f[7:10].tolist(), "maxabs": float(f[10]),
                "rmax": float(f[11]), "layout": int(u[13])}

    def node_table(self) -> Tuple[torch.Tensor, torch.Tensor]:
        """(boxes [M-1, 2, 6] float32, child refs [M-1, 2] int32) of the internal nodes."""
        m = self.header()["m"]
        k = max(m - 1, 0)
        raw = self.nodes[64:64 + 64 * k].view(torch.float32).view(k, 16)
        boxes = raw[:, :12].reshape(k, 2, 6)
        refs = raw[:, 12:14].contiguous().view(torch.int32)
        return boxes, refs

    def wide_table(self) -> Tuple[torch.Tensor, torch.Tensor]:
        """(boxes [M-1, 4, 6] float32 as lo xyz, hi xyz; refs [M-1, 4] int32) of the 4-wide nodes
        (unused entries have reference -1)."""
        m = self.header()["m"]
        k = max(m - 1, 0)
        start = 64 + 64 * int(self.nodes[48:52].view(torch.int32).item())
        raw = self.nodes[start:start + 128 * k].view(torch.float32).view(k, 8, 4)
        boxes = raw[:, :6, :].permute(0, 2, 1).contiguous()  # [k, entry, coord]
        refs = raw[:, 6, :].contiguous().view(torch.int32)
        return boxes, refs


def _scratch(nbytes: int, device=None) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device or torch.device("cuda"))


# ----------------------------------------------------------------------------------------------
# entry points
# ----------------------------------------------------------------------------------------------
def raycast_volume(vol: torch.Tensor, tf: torch.Tensor, cam, step_vox: float = 0.5,
                   tau: float = 0.1, rgba_out: Optional[torch.Tensor] = None,
                   depth_out: Optional[torch.Tensor] = None, stream=None,
                   heuristic: int = 0, param: Optional[float] = None):
    """Server volume ray caster + depth heuristic (DEPTH_*; default first hit with ``tau``).
    vol: CUDA [nz,ny,nx] float32 or uint8; tf: CUDA [256,4] float32.  ``param``: theta of
    DEPTH_ACCUMULATED (default 0.5), tau of DEPTH_FIRST_HIT (default ``tau``).  Returns
    (rgba [H,W,4], depth [H,W])."""
    c = _cam(cam)
    if vol.dtype == torch.uint8:
        dt = U8
    elif vol.dtype == torch.float32:
        dt = F32
    else:
        raise TypeError("volume must be float32 or uint8")
    nz, ny, nx = vol.shape
    if rgba_out is None:
        rgba_out = torch.empty(c.height, c.width, 4, dtype=torch.float32, device=vol.device)
    if depth_out is None:
        depth_out = torch.empty(c.height, c.width, dtype=torch.float32, device=vol.device)
    _buf(rgba_out, c.height * c.width * 4, torch.float32, "rgba_out")
    _buf(depth_out, c.height * c.width, torch.float32, "depth_out")
    if param is None:
        param = 0.5 if heuristic == DEPTH_ACCUMULATED else tau
    _check(_lib.wrs_raycast_volume_heuristic(_ptr(vol), dt, nx, ny, nz, _ptr(tf), ctypes.byref(c),
                                             float(step_vox), int(heuristic), float(param),
                                             _ptr(rgba_out), _ptr(depth_out), _stream(stream)),
           "wrs_raycast_volume")
    return rgba_out, depth_out


def unproject_scratch_bytes(width: int, height: int) -> int:
    return int(_lib.wrs_unproject_scratch_bytes(int(width), int(height)))


def unproject(rgba: torch.Tensor, depth: torch.Tensor, cam, radius_mode: int = RADIUS_FOOTPRINT,
              voxel_diag: float = 0.0, out: Optional[SplatBuffers] = None,
              scratch: Optional[torch.Tensor] = None, stream=None) -> SplatBuffers:
    """Eq. 1 unprojection + radius + stable compaction of a server image into splats."""
    c = _cam(cam)
    if out is None:
        out = SplatBuffers(c.width * c.height, device=rgba.device)
    need = unproject_scratch_bytes(c.width, c.height)
    if scratch is None:
        scratch = _scratch(need, rgba.device)
    sp = out.c()
    _check(_lib.wrs_unproject(_ptr(rgba), _ptr(depth), ctypes.byref(c), int(radius_mode),
                              float(voxel_diag), ctypes.byref(sp), _ptr(scratch), scratch.numel(),
                              _stream(stream)), "wrs_unproject")
    return out


def window_weight(decay: float, age: int) -> float:
    """Colour weight of the server frame of age ``age`` in an accumulated window
    (wrs_window_weight: decay^age in binary32)."""
    w = float(_lib.wrs_window_weight(float(decay), int(age)))
    if w != w:
        raise ValueError("decay must lie in (0, 1]")
    return w


def unproject_append(rgba: torch.Tensor, depth: torch.Tensor, cam, out: SplatBuffers,
                     weight: float = 1.0, id_base: int = 0, radius_mode: int = RADIUS_FOOTPRINT,
                     voxel_diag: float = 0.0, status: Optional[torch.Tensor] = None,
                     scratch: Optional[torch.Tensor] = None, stream=None) -> SplatBuffers:
    """Append one more server frame's splats to ``out`` (accumulation over frames; see
    wrs_unproject_append): ids offset by ``id_base``, colours scaled by ``weight``.  Splats beyond
    the capacity are dropped and flag STATUS_SPLAT_OVERFLOW in ``status``."""
    c = _cam(cam)
    if int(id_base) + c.width * c.height > 2**31:
        raise ValueError("id_base + pixels must stay below 2^31 (ids are held in int32 tensors)")
    need = unproject_scratch_bytes(c.width, c.height)
    if scratch is None:
        scratch = _scratch(need, rgba.device)
    sp = out.c()
    _check(_lib.wrs_unproject_append(_ptr(rgba), _ptr(depth), ctypes.byref(c), int(radius_mode),
                                     float(voxel_diag), float(weight), int(id_base),
                                     ctypes.byref(sp), _ptr(scratch), scratch.numel(), _ptr(status),
                                     _stream(stream)), "wrs_unproject_append")
    return out


class EncodedSplats:
    """The server's stream of a splat set (see wrs_codec): word uint64 [cap] (held in an int64
    tensor), color uint32 [cap] (held in an int32 tensor), n [1] on the device, 12 bytes a splat."""

    def __init__(self, capacity: int, device=None):
        device = device or torch.device("cuda")
        cap = max(int(capacity), 1)
        self.capacity = int(capacity)
        self.word = torch.zeros(cap, dtype=torch.int64, device=device)
        self.color = torch.zeros(cap, dtype=torch.int32, device=device)
        self.n = torch.zeros(1, dtype=torch.int32, device=device)

    def count(self) -> int:
        return int(self.n.item())

    def nbytes(self) -> int:
        """Bytes of the valid records (what the server sends; synchronises)."""
        return 12 * self.count()


def unproject_encode(rgba: torch.Tensor, depth: torch.Tensor, cam, codec: Codec,
                     radius_mode: int = RADIUS_FOOTPRINT, voxel_diag: float = 0.0,
                     out: Optional[EncodedSplats] = None, scratch: Optional[torch.Tensor] = None,
                     stream=None) -> EncodedSplats:
    """Unprojection (Eq. 1, §4.1) writing the 64-bit word + 32-bit colour stream (§4.1, §6)."""
    c = _cam(cam)
    if out is None:
        out = EncodedSplats(c.width * c.height, device=rgba.device)
    if scratch is None:
        scratch = _scratch(unproject_scratch_bytes(c.width, c.height), rgba.device)
    _check(_lib.wrs_unproject_encode(_ptr(rgba), _ptr(depth), ctypes.byref(c), int(radius_mode),
                                     float(voxel_diag), ctypes.byref(codec), _ptr(out.word),
                                     _ptr(out.color), _ptr(out.n), out.capacity, _ptr(scratch),
                                     scratch.numel(), _stream(stream)), "wrs_unproject_encode")
    return out


def encode_splats(splats: SplatBuffers, codec: Codec, out: Optional[EncodedSplats] = None,
                  stream=None) -> EncodedSplats:
    """Encode a float splat set into the 12-byte stream (the count is written on the device)."""
    if out is None:
        out = EncodedSplats(splats.capacity, device=splats.pos_r.device)
    sp = splats.c()
    _check(_lib.wrs_encode_splats(ctypes.byref(sp), ctypes.byref(codec), _ptr(out.word),
                                  _ptr(out.color), _ptr(out.n), _stream(stream)), "wrs_encode_splats")
    return out


def decode_splats(enc: EncodedSplats, codec: Codec, out: Optional[SplatBuffers] = None,
                  stream=None) -> SplatBuffers:
    """Decode the stream into float splats (id = stream index) for wrs_build_lbvh."""
    if out is None:
        out = SplatBuffers(enc.capacity, device=enc.word.device)
    sp = out.c()
    _check(_lib.wrs_decode_splats(_ptr(enc.word), _ptr(enc.color), _ptr(enc.n), enc.capacity,
                                  ctypes.byref(codec), ctypes.byref(sp), _stream(stream)),
           "wrs_decode_splats")
    return out


def unproject_interval(rgba: torch.Tensor, depth_lo: torch.Tensor, depth_hi: torch.Tensor, cam,
                       max_chain: int = 8, radius_mode: int = RADIUS_FOOTPRINT,
                       voxel_diag: float = 0.0, out: Optional[SplatBuffers] = None,
                       status: Optional[torch.Tensor] = None, scratch: Optional[torch.Tensor] = None,
                       stream=None) -> SplatBuffers:
    """Each kept pixel as a chain of spheres along its server ray over [depth_lo, depth_hi], the
    depth interval of growing opacity (depth uncertainty; see wrs_unproject_interval).  The default
    output holds width * height * max_chain records."""
    c = _cam(cam)
    if out is None:
        out = SplatBuffers(c.width * c.height * int(max_chain), device=rgba.device)
    if scratch is None:
        scratch = _scratch(unproject_scratch_bytes(c.width, c.height), rgba.device)
    sp = out.c()
    _check(_lib.wrs_unproject_interval(_ptr(rgba), _ptr(depth_lo), _ptr(depth_hi), ctypes.byref(c),
                                       int(radius_mode), float(voxel_diag), int(max_chain),
                                       ctypes.byref(sp), _ptr(scratch), scratch.numel(),
                                       _ptr(status), _stream(stream)), "wrs_unproject_interval")
    return out


def point_splat_scratch_bytes(width: int, height: int) -> int:
    return int(_lib.wrs_point_splat_scratch_bytes(int(width), int(height)))


def point_splat(splats: SplatBuffers, cam, point_size: int = 1, out: Optional[torch.Tensor] = None,
                index: Optional[torch.Tensor] = None, scratch: Optional[torch.Tensor] = None,
                stream=None) -> torch.Tensor:
    """The earlier warping the paper compares against (§2, §5, Fig. 3): each splat drawn as a
    point_size x point_size pixel square with one depth per point, nearest kept (wrs_point_splat).
    Returns premultiplied RGBA [H,W,4]; ``index`` (int32 [H,W], optional) receives the winner."""
    c = _cam(cam)
    dev = splats.pos_r.device
    if out is None:
        out = torch.empty(c.height, c.width, 4, dtype=torch.float32, device=dev)
    _buf(out, c.height * c.width * 4, torch.float32, "point_splat out")
    _buf(index, c.height * c.width, torch.int32, "point_splat index")
    if scratch is None:
        scratch = _scratch(point_splat_scratch_bytes(c.width, c.height), dev)
    sp = splats.c()
    _check(_lib.wrs_point_splat(ctypes.byref(sp), ctypes.byref(c), int(point_size), _ptr(out),
                                _ptr(index), _ptr(scratch), scratch.numel(), _stream(stream)),
           "wrs_point_splat")
    return out


def lbvh_scratch_bytes(capacity: int, leaf_size: int) -> int:
    return int(_lib.wrs_lbvh_scratch_bytes(int(capacity), int(leaf_size)))


def build_lbvh(splats: SplatBuffers, leaf_size: int = 1, radius_scale: Optional[torch.Tensor] = None,
               global_scale: float = 1.0, bvh: Optional[LBVH] = None,
               sorted: Optional[SplatBuffers] = None, scratch: Optional[torch.Tensor] = None,
               stream=None, layout: int = LBVH_FULL) -> Tuple[LBVH, SplatBuffers]:
    """LBVH over the splats; returns (bvh, sorted splats with baked effective radius).  A new
    ``bvh`` gets ``layout``; a given one keeps its own."""
    dev = splats.pos_r.device
    # buffers made here are returned only after the build wrote the header, the count and every
    # node and row that a traversal can reach, so they need no zero fill
    if bvh is None:
        bvh = LBVH(splats.capacity, leaf_size, device=dev, _fill=False, layout=layout)
    if sorted is None:
        sorted = SplatBuffers(splats.capacity, device=dev, sorted=True, _fill=False)
    need = lbvh_scratch_bytes(splats.capacity, bvh.leaf_size)
    if scratch is None:
        scratch = _scratch(need, dev)
    a, b, o = splats.c(), bvh.c(), sorted.c()
    _check(_lib.wrs_build_lbvh(ctypes.byref(a), _ptr(radius_scale), float(global_scale), ctypes.byref(b),
                               ctypes.byref(o), _ptr(scratch), scratch.numel(), _stream(stream)),
           "wrs_build_lbvh")
    return bvh, sorted


def refit_lbvh(splats: SplatBuffers, bvh: LBVH, sorted: SplatBuffers, scratch: torch.Tensor,
               radius_scale: Optional[torch.Tensor] = None, global_scale: float = 1.0,
               stream=None) -> Tuple[LBVH, SplatBuffers]:
    """wrs_refit_lbvh: the tree that :func:`build_lbvh` built into ``bvh``/``sorted`` with
    ``scratch`` over the same splat centres, with new radius scales (bitwise the tree a new build
    would give; no Morton codes, sort or radix tree).  The splat centres, their count and the
    scratch must be unchanged since that build."""
    _buf(scratch, lbvh_scratch_bytes(splats.capacity, bvh.leaf_size), torch.uint8, "scratch")
    a, b, o = splats.c(), bvh.c(), sorted.c()
    _check(_lib.wrs_refit_lbvh(ctypes.byref(a), _ptr(radius_scale), float(global_scale), ctypes.byref(b),
                               ctypes.byref(o), _ptr(scratch), scratch.numel(), _stream(stream)),
           "wrs_refit_lbvh")
    return bvh, sorted


class RefitTree:
    """An LBVH over splats whose centres stay fixed while their radius scales change (a radius
    fit): the first :meth:`update` builds it (wrs_build_lbvh), later ones refit it
    (wrs_refit_lbvh) in the same buffers.  The buffers are reused: a tree handed to a traversal
    must have been used before the next update (an autograd step's backward runs before the next
    step's forward)."""

    def __init__(self, splats: SplatBuffers, leaf_size: int = 1, layout: int = LBVH_FULL):
        dev = splats.pos_r.device
        self.splats = splats
        self.leaf_size = int(leaf_size)
        self.bvh = LBVH(splats.capacity, leaf_size, device=dev, _fill=False, layout=layout)
        self.sorted = SplatBuffers(splats.capacity, device=dev, sorted=True, _fill=False)
        self.scratch = _scratch(lbvh_scratch_bytes(splats.capacity, leaf_size), dev)
        self.built = False

    def update(self, radius_scale: Optional[torch.Tensor] = None, global_scale: float = 1.0,
               stream=None) -> Tuple[LBVH, SplatBuffers]:
        if self.built:
            return refit_lbvh(self.splats, self.bvh, self.sorted, self.scratch, radius_scale,
                              global_scale, stream)
        build_lbvh(self.splats, self.leaf_size, radius_scale, global_scale, bvh=self.bvh,
                   sorted=self.sorted, scratch=self.scratch, stream=stream)
        self.built = True
        return self.bvh, self.sorted


@dataclass
class TraceParams:
    max_hits: int = 0            # 1 = first hit (the paper), 0 = all hits
    t_stop: float = 1e-5
    edge_softness: float = 0.0
    k_chunk: int = 8
    block: int = 128
    schedule: int = 0            # 0 = one thread per pixel, 1 = persistent with lane refill,
                                 # 2 = one warp-shared traversal per 8x4 tile (wrs_trace only)
    width: int = 4               # 4 = 4-wide nodes (faster in every measured case), 2 = binary

    def c(self, opacity: Optional[torch.Tensor] = None) -> _Params:
        return _Params(int(self.max_hits), float(self.t_stop), float(self.edge_softness),
                       _ptr(opacity), int(self.k_chunk), int(self.block), int(self.schedule),
                       int(self.width))


def tree_layout(params: TraceParams) -> int:
    """The LBVH layout that traces with ``params`` need: LBVH_WIDE (the 4-wide nodes only, a
    faster build) unless they walk the binary nodes (width 2 under a schedule other than the
    packet one)."""
    return LBVH_WIDE if (params.width == 4 or params.schedule == SCHEDULE_PACKET) else LBVH_FULL


def trace(bvh: LBVH, sorted: SplatBuffers, cam, params: TraceParams = TraceParams(),
          opacity: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
          status: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Trace the client camera through the spheres; returns premultiplied RGBA [H,W,4]."""
    c = _cam(cam)
    if out is None:
        out = torch.empty(c.height, c.width, 4, dtype=torch.float32, device=sorted.pos_r.device)
    _buf(out, c.height * c.width * 4, torch.float32, "trace out")
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace(ctypes.byref(b), ctypes.byref(s), ctypes.byref(c), ctypes.byref(p),
                          _ptr(out), _ptr(status), _stream(stream)), "wrs_trace")
    return out


def _cams(cams) -> Tuple[ctypes.Array, int, int]:
    arr = (Camera * len(cams))(*[_cam(c) for c in cams])
    return arr, arr[0].width, arr[0].height


def trace_views(bvh: LBVH, sorted: SplatBuffers, cams: Sequence, params: TraceParams = TraceParams(),
                opacity: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                status: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Several same-size client views in one launch (wrs_trace_views); returns [V,H,W,4], view v
    bitwise equal to ``trace(bvh, sorted, cams[v], ...)``."""
    arr, w, h = _cams(cams)
    if out is None:
        out = torch.empty(len(cams), h, w, 4, dtype=torch.float32, device=sorted.pos_r.device)
    _buf(out, len(cams) * h * w * 4, torch.float32, "trace_views out")
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace_views(ctypes.byref(b), ctypes.byref(s), arr, len(cams), ctypes.byref(p),
                                _ptr(out), _ptr(status), _stream(stream)), "wrs_trace_views")
    return out


class HitLists:
    """The composited hits of every ray of a multi-view trace (wrs_trace_views_record): ``hits``
    [rays, capacity] sorted-splat indices in compositing order, ``count`` [rays] their number
    (capacity + 1: more than fit, the adjoint traces that ray again); ray = view * H * W + pixel."""

    MAX_CAPACITY = 32

    def __init__(self, rays: int, capacity: int = 16, device=None):
        if not 1 <= capacity <= self.MAX_CAPACITY:
            raise ValueError(f"hit capacity {capacity} not in 1..{self.MAX_CAPACITY}")
        device = device or torch.device("cuda")
        self.rays, self.capacity = int(rays), int(capacity)
        self.hits = torch.empty(self.rays, self.capacity, dtype=torch.int32, device=device)
        self.count = torch.empty(self.rays, dtype=torch.int32, device=device)

    @staticmethod
    def nbytes(rays: int, capacity: int) -> int:
        return 4 * int(rays) * (int(capacity) + 1)


def trace_views_record(bvh: LBVH, sorted: SplatBuffers, cams: Sequence,
                       params: TraceParams = TraceParams(), hit_capacity: int = 16,
                       opacity: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                       lists: Optional[HitLists] = None, status: Optional[torch.Tensor] = None,
                       stream=None) -> Tuple[torch.Tensor, HitLists]:
    """trace_views that also records every ray's composited hits (wrs_trace_views_record) for
    :func:`trace_backward_views_recorded`; returns (images [V,H,W,4], HitLists)."""
    arr, w, h = _cams(cams)
    dev = sorted.pos_r.device
    if out is None:
        out = torch.empty(len(cams), h, w, 4, dtype=torch.float32, device=dev)
    _buf(out, len(cams) * h * w * 4, torch.float32, "trace_views_record out")
    rays = len(cams) * h * w
    if lists is None:
        lists = HitLists(rays, hit_capacity, dev)
    if lists.rays != rays:
        raise ValueError(f"hit lists for {lists.rays} rays, the views have {rays}")
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace_views_record(ctypes.byref(b), ctypes.byref(s), arr, len(cams),
                                       ctypes.byref(p), _ptr(out), _ptr(lists.hits),
                                       _ptr(lists.count), lists.capacity, _ptr(status),
                                       _stream(stream)), "wrs_trace_views_record")
    return out, lists


COUNTER_NAMES = ("nodes", "boxes", "spheres", "gathered", "composited", "passes")


def trace_count(bvh: LBVH, sorted: SplatBuffers, cam, params: TraceParams = TraceParams(),
                opacity: Optional[torch.Tensor] = None, status: Optional[torch.Tensor] = None,
                stream=None) -> dict:
    """Traversal statistics over all rays (synchronises)."""
    c = _cam(cam)
    cnt = torch.zeros(6, dtype=torch.int64, device=sorted.pos_r.device)
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace_count(ctypes.byref(b), ctypes.byref(s), ctypes.byref(c), ctypes.byref(p),
                                _ptr(cnt), _ptr(status), _stream(stream)), "wrs_trace_count")
    return dict(zip(COUNTER_NAMES, [int(v) for v in cnt.cpu()]))


def session_tiles(width: int, height: int) -> int:
    return int(_lib.wrs_session_tiles(int(width), int(height)))


# client pixels per splat from which a session of a multi-session launch takes the warp-shared
# traversal by default (SCHEDULE_PER_SESSION): on the 64-session workload the per-pixel traversal
# wins below it
SPARSE_PIXELS_PER_SPLAT = 8.0


def sparse_schedules(sessions: Sequence[Tuple[LBVH, SplatBuffers, object]],
                     ratio: float = SPARSE_PIXELS_PER_SPLAT) -> List[int]:
    """Per-session schedules for SCHEDULE_PER_SESSION: the warp-shared traversal where the client
    image has at least ``ratio`` pixels per splat (neighbouring rays then hit the same splats),
    one thread per pixel elsewhere.  The splat counts are read back from the device once (one
    synchronisation), so a server image with a large empty background counts as sparse."""
    counts = [sp.count() for _, sp, _ in sessions]
    out = []
    for (_, _, cam), n in zip(sessions, counts):
        c = _cam(cam)
        out.append(SCHEDULE_PACKET if c.width * c.height >= ratio * max(n, 1)
                   else SCHEDULE_PER_PIXEL)
    return out


class Batch:
    """Descriptors of many client sessions for :func:`trace_batched` (device array + outputs)."""

    def __init__(self, sessions: Sequence[Tuple[LBVH, SplatBuffers, object]],
                 opacity: Optional[Sequence[Optional[torch.Tensor]]] = None, device=None,
                 schedules: Optional[Sequence[int]] = None):
        """``schedules``: per session SCHEDULE_PER_PIXEL or SCHEDULE_PACKET, used by launches with
        ``schedule=SCHEDULE_PER_SESSION`` (default: the packet traversal for sessions with at
        least SPARSE_PIXELS_PER_SPLAT client pixels per splat, see :func:`sparse_schedules`)."""
        device = device or torch.device("cuda")
        n = len(sessions)
        if schedules is None:
            schedules = sparse_schedules(sessions)
        if len(schedules) != n:
            raise ValueError("one schedule per session")
        arr = (Session * n)()
        self.outputs: List[torch.Tensor] = []
        self._keep = []
        tile = 0
        for i, (bvh, sp, cam) in enumerate(sessions):
            c = _cam(cam)
            out = torch.empty(c.height, c.width, 4, dtype=torch.float32, device=device)
            op = opacity[i] if opacity is not None else None
            arr[i] = Session(_ptr(bvh.nodes), _ptr(sp.pos_r), _ptr(sp.rgba), _ptr(sp.id),
                             _ptr(sp.src), _ptr(op), _ptr(out), c, tile, int(schedules[i]))
            self.outputs.append(out)
            self._keep.append((bvh, sp, op))
            tile += session_tiles(c.width, c.height)
        self.total_tiles = tile
        self.n_sessions = n
        self.schedules = [int(v) for v in schedules]
        raw = bytes(memoryview(arr).cast("B"))
        self.desc = torch.frombuffer(bytearray(raw), dtype=torch.uint8).to(device)
        self.work = torch.zeros(1, dtype=torch.int32, device=device)


def trace_batched(batch: Batch, params: TraceParams = TraceParams(),
                  status: Optional[torch.Tensor] = None, stream=None) -> List[torch.Tensor]:
    """All sessions of ``batch`` in one launch (params.schedule: per-pixel warps, persistent, or
    one warp-shared traversal per tile); returns the per-session images."""
    p = params.c(None)
    _check(_lib.wrs_trace_batched(_ptr(batch.desc), batch.n_sessions, batch.total_tiles,
                                  ctypes.byref(p), _ptr(batch.work), _ptr(status), _stream(stream)),
           "wrs_trace_batched")
    return batch.outputs


def trace_backward(bvh: LBVH, sorted: SplatBuffers, cam, dL_drgba: torch.Tensor,
                   params: TraceParams = TraceParams(), opacity: Optional[torch.Tensor] = None,
                   radius_scale: Optional[torch.Tensor] = None, global_scale: float = 1.0,
                   want_opacity: bool = True, want_scale: bool = True,
                   status: Optional[torch.Tensor] = None, stream=None, accumulate_into=None):
    """Adjoint of :func:`trace`: returns (g_rgba [cap,4], g_opacity [cap] | None, g_scale [cap] | None)
    in compacted splat order.  ``accumulate_into=(g_rgba, g_opacity, g_scale)`` adds this view's
    gradients to those buffers instead (wrs_trace_backward_accumulate) and returns them."""
    c = _cam(cam)
    dev = sorted.pos_r.device
    cap = max(sorted.capacity, 1)
    _buf(dL_drgba.contiguous(), c.height * c.width * 4, torch.float32, "dL_drgba")
    if accumulate_into is not None:
        g_rgba, g_op, g_sc = accumulate_into
        _buf(g_rgba, sorted.capacity * 4, torch.float32, "g_rgba")
        _buf(g_op, sorted.capacity, torch.float32, "g_opacity")
        _buf(g_sc, sorted.capacity, torch.float32, "g_scale")
        fn, name = _lib.wrs_trace_backward_accumulate, "wrs_trace_backward_accumulate"
    else:
        g_rgba = torch.empty(cap, 4, dtype=torch.float32, device=dev)
        g_op = torch.empty(cap, dtype=torch.float32, device=dev) if want_opacity else None
        g_sc = torch.empty(cap, dtype=torch.float32, device=dev) if want_scale else None
        fn, name = _lib.wrs_trace_backward, "wrs_trace_backward"
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(fn(ctypes.byref(b), ctypes.byref(s), ctypes.byref(c), ctypes.byref(p),
              _ptr(radius_scale), float(global_scale), _ptr(dL_drgba.contiguous()), _ptr(g_rgba),
              _ptr(g_op), _ptr(g_sc), _ptr(status), _stream(stream)), name)
    return g_rgba, g_op, g_sc


def trace_backward_views(bvh: LBVH, sorted: SplatBuffers, cams: Sequence, dL_drgba: torch.Tensor,
                         params: TraceParams = TraceParams(), opacity: Optional[torch.Tensor] = None,
                         radius_scale: Optional[torch.Tensor] = None, global_scale: float = 1.0,
                         want_opacity: bool = True, want_scale: bool = True,
                         status: Optional[torch.Tensor] = None, stream=None, accumulate_into=None):
    """Adjoint of :func:`trace_views` (dL_drgba [V,H,W,4]): the sum over the views of their
    :func:`trace_backward` gradients, in one launch.  ``accumulate_into`` as for trace_backward."""
    arr, w, h = _cams(cams)
    dev = sorted.pos_r.device
    cap = max(sorted.capacity, 1)
    _buf(dL_drgba.contiguous(), len(cams) * h * w * 4, torch.float32, "dL_drgba")
    if accumulate_into is not None:
        g_rgba, g_op, g_sc = accumulate_into
        _buf(g_rgba, sorted.capacity * 4, torch.float32, "g_rgba")
        _buf(g_op, sorted.capacity, torch.float32, "g_opacity")
        _buf(g_sc, sorted.capacity, torch.float32, "g_scale")
    else:
        g_rgba = torch.empty(cap, 4, dtype=torch.float32, device=dev)
        g_op = torch.empty(cap, dtype=torch.float32, device=dev) if want_opacity else None
        g_sc = torch.empty(cap, dtype=torch.float32, device=dev) if want_scale else None
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace_backward_views(
        ctypes.byref(b), ctypes.byref(s), arr, len(cams), ctypes.byref(p), _ptr(radius_scale),
        float(global_scale), _ptr(dL_drgba.contiguous()), _ptr(g_rgba), _ptr(g_op), _ptr(g_sc),
        1 if accumulate_into is not None else 0, _ptr(status), _stream(stream)),
        "wrs_trace_backward_views")
    return g_rgba, g_op, g_sc


def trace_backward_views_recorded(bvh: LBVH, sorted: SplatBuffers, cams: Sequence, lists: HitLists,
                                  dL_drgba: torch.Tensor, params: TraceParams = TraceParams(),
                                  opacity: Optional[torch.Tensor] = None,
                                  radius_scale: Optional[torch.Tensor] = None,
                                  global_scale: float = 1.0, want_opacity: bool = True,
                                  want_scale: bool = True, status: Optional[torch.Tensor] = None,
                                  stream=None, accumulate_into=None):
    """:func:`trace_backward_views` from the hit lists of :func:`trace_views_record` (same scene,
    cameras and parameters): no traversal for the rays whose list is complete."""
    arr, w, h = _cams(cams)
    dev = sorted.pos_r.device
    cap = max(sorted.capacity, 1)
    if lists.rays != len(cams) * h * w:
        raise ValueError("hit lists do not belong to these views")
    _buf(dL_drgba.contiguous(), len(cams) * h * w * 4, torch.float32, "dL_drgba")
    if accumulate_into is not None:
        g_rgba, g_op, g_sc = accumulate_into
        _buf(g_rgba, sorted.capacity * 4, torch.float32, "g_rgba")
        _buf(g_op, sorted.capacity, torch.float32, "g_opacity")
        _buf(g_sc, sorted.capacity, torch.float32, "g_scale")
    else:
        g_rgba = torch.empty(cap, 4, dtype=torch.float32, device=dev)
        g_op = torch.empty(cap, dtype=torch.float32, device=dev) if want_opacity else None
        g_sc = torch.empty(cap, dtype=torch.float32, device=dev) if want_scale else None
    b, s, p = bvh.c(), sorted.c(), params.c(opacity)
    _check(_lib.wrs_trace_backward_views_recorded(
        ctypes.byref(b), ctypes.byref(s), arr, len(cams), ctypes.byref(p), _ptr(radius_scale),
        float(global_scale), _ptr(lists.hits), _ptr(lists.count), lists.capacity,
        _ptr(dL_drgba.contiguous()), _ptr(g_rgba), _ptr(g_op), _ptr(g_sc),
        1 if accumulate_into is not None else 0, _ptr(status), _stream(stream)),
        "wrs_trace_backward_views_recorded")
    return g_rgba, g_op, g_sc


def fma_peak(blocks: int, iters: int, stream=None, out: Optional[torch.Tensor] = None):
    """Launch the FP32 FMA throughput kernel (blocks x 256 threads x iters x 128 FMAs); the caller
    times it.  Returns the flop count of the launch."""
    if out is None or out.numel() < blocks:
        out = torch.empty(blocks, dtype=torch.float32, device="cuda")
    _check(_lib.wrs_fma_peak(_ptr(out), int(blocks), int(iters), _stream(stream)), "wrs_fma_peak")
    return 2.0 * blocks * 256 * iters * 128


def stream_copy(dst: torch.Tensor, src: torch.Tensor, blocks: int, reps: int = 1, stream=None):
    """Copy src into dst (same byte size, device) ``reps`` times with the streaming copy kernel;
    the caller times it."""
    nb = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nb:
        raise ValueError("stream_copy: buffers of different sizes")
    _check(_lib.wrs_stream_copy(_ptr(dst), _ptr(src), nb, int(blocks), int(reps), _stream(stream)),
           "wrs_stream_copy")


def check_status(status: torch.Tensor, stream=None):
    """Raise WrsError if a kernel reported an error in the status word (synchronises)."""
    _check(_lib.wrs_check_status(_ptr(status), _stream(stream)), "wrs_check_status")


def new_status(device=None) -> torch.Tensor:
    return torch.zeros(1, dtype=torch.int32, device=device or torch.device("cuda"))


from .autograd import MultiViewTraceFunction, TraceFunction, render, render_views  # noqa: E402,F401
from .accumulate import FrameWindow  # noqa: E402,F401
