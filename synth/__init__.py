"""Seeded synthetic inputs for the sphere-splat warping workloads.

This module is shared by the tests, the benchmark and the smoke check.  It holds none of the
method's arithmetic (no ray generation, no unprojection, no intersection, no compositing): it only
draws volumes, a transfer function, camera poses and stand-in 2.5D images from fixed seeds
(numpy PCG64).  The paper's own data set is unnamed and not available; these inputs stand in for
it with the sizes of its workload (a 1024^2 view with about 0.6 M splats, Table 1) and the larger
sizes of the benchmark.

Volume layout: ``vol[z, y, x]`` (x fastest), occupying the unit cube.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, replace
from typing import List, Tuple

import numpy as np


@dataclass(frozen=True)
class Camera:
    """Pinhole camera: eye, orthonormal basis (right, up, fwd), tan(fovy/2), image size.

    The vectors are float32 exactly as the libraries read them."""
    eye: Tuple[float, float, float]
    right: Tuple[float, float, float]
    up: Tuple[float, float, float]
    fwd: Tuple[float, float, float]
    tan_half_fovy: float
    width: int
    height: int

    def with_size(self, width: int, height: int) -> "Camera":
        return replace(self, width=int(width), height=int(height))


def _f32(v) -> Tuple[float, float, float]:
    a = np.asarray(v, dtype=np.float64).astype(np.float32)
    return tuple(float(x) for x in a)


def look_at(eye, target, up_hint, fovy_deg: float, width: int, height: int) -> Camera:
    eye = np.asarray(eye, np.float64)
    fwd = np.asarray(target, np.float64) - eye
    fwd /= np.linalg.norm(fwd)
    right = np.cross(fwd, np.asarray(up_hint, np.float64))
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(_f32(eye), _f32(right), _f32(up), _f32(fwd),
                  float(np.float32(math.tan(math.radians(fovy_deg) / 2))), int(width), int(height))


CENTER = np.array([0.5, 0.5, 0.5])


def server_camera(distance: float, fovy_deg: float, width: int, height: int) -> Camera:
    """Camera on the +z side of the cube centre looking at it, +y up."""
    return look_at(CENTER + np.array([0.0, 0.0, distance]), CENTER, (0.0, 1.0, 0.0), fovy_deg,
                   width, height)


def _rotate(v: np.ndarray, axis: np.ndarray, ang: float) -> np.ndarray:
    axis = axis / np.linalg.norm(axis)
    return (v * math.cos(ang) + np.cross(axis, v) * math.sin(ang)
            + axis * np.dot(axis, v) * (1 - math.cos(ang)))


def orbit(cam: Camera, axis, angle_deg: float, width: int = None, height: int = None) -> Camera:
    """Rotate the camera's eye and basis about the cube centre by angle_deg around ``axis``."""
    ang = math.radians(angle_deg)
    axis = np.asarray(axis, np.float64)
    eye = _rotate(np.asarray(cam.eye, np.float64) - CENTER, axis, ang) + CENTER
    up = _rotate(np.asarray(cam.up, np.float64), axis, ang)
    fovy = 2 * math.degrees(math.atan(cam.tan_half_fovy))
    return look_at(eye, CENTER, up, fovy, width or cam.width, height or cam.height)


def poses_in_cap(cam: Camera, n: int, max_deg: float, seed: int, width: int = None,
                 height: int = None) -> List[Camera]:
    """n poses whose view axis is uniform over the spherical cap of half-angle max_deg around the
    given camera's view axis (rotation about a random axis perpendicular to the view direction)."""
    rng = np.random.default_rng(seed)
    fwd = np.asarray(cam.fwd, np.float64)
    right = np.asarray(cam.right, np.float64)
    up = np.asarray(cam.up, np.float64)
    out = []
    cmin = math.cos(math.radians(max_deg))
    for _ in range(n):
        ang = math.degrees(math.acos(rng.uniform(cmin, 1.0)))
        az = rng.uniform(0, 2 * math.pi)
        axis = math.cos(az) * right + math.sin(az) * up
        out.append(orbit(cam, axis, ang, width, height))
    return out


def tf_ramp() -> np.ndarray:
    """256-entry RGBA transfer function, x = i/255: (x, 1-|2x-1|, 1-x, x)."""
    x = np.arange(256, dtype=np.float64) / 255.0
    return np.stack([x, 1 - np.abs(2 * x - 1), 1 - x, x], axis=1).astype(np.float32)


def tf_iso(lo: float = 0.45, hi: float = 0.55, alpha: float = 0.9) -> np.ndarray:
    """256-entry transfer function for iso-surface-like renderings (a narrow band of values mapped
    to high opacity, the kind of transfer function the warping works best with, §2): colour as
    tf_ramp, alpha = ``alpha`` for x in [lo, hi] and 0 elsewhere."""
    t = tf_ramp()
    x = np.arange(256, dtype=np.float64) / 255.0
    t[:, 3] = np.where((x >= lo) & (x <= hi), alpha, 0.0).astype(np.float32)
    return t


def gaussian_volume(n: int, nblobs: int, seed: int) -> np.ndarray:
    """Sum of isotropic Gaussian blobs at the voxel centres, divided by its maximum, float32."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(nblobs, 3))
    sig = rng.uniform(0.08, 0.15, size=nblobs)
    amp = rng.uniform(0.5, 1.0, size=nblobs)
    g = (np.arange(n) + 0.5) / n
    vol = np.zeros((n, n, n), np.float64)
    for b in range(nblobs):
        ex = np.exp(-((g - c[b, 0]) ** 2) / (2 * sig[b] ** 2))
        ey = np.exp(-((g - c[b, 1]) ** 2) / (2 * sig[b] ** 2))
        ez = np.exp(-((g - c[b, 2]) ** 2) / (2 * sig[b] ** 2))
        vol += amp[b] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    vol /= vol.max()
    return vol.astype(np.float32)


def fourier_volume(n: int, nmodes: int, kmax: int, seed: int) -> np.ndarray:
    """Sum of random Fourier modes |k|^(-5/3) cos(2 pi k.x + phi), integer k with 1 <= |k| <= kmax,
    min-max normalised and rounded to uint8.  Evaluated slice by slice as a rank-nmodes product of
    per-axis complex exponentials."""
    rng = np.random.default_rng(seed)
    ks = []
    while len(ks) < nmodes:
        k = rng.integers(-kmax, kmax + 1, size=3)
        m = float(np.linalg.norm(k))
        if 1 <= m <= kmax:
            ks.append(k)
    ks = np.array(ks, np.float64)
    amp = np.linalg.norm(ks, axis=1) ** (-5.0 / 3.0)
    phi = rng.uniform(0, 2 * math.pi, size=nmodes)
    g = (np.arange(n) + 0.5) / n
    X = np.exp(2j * math.pi * g[:, None] * ks[None, :, 0])   # [n, m]
    Y = np.exp(2j * math.pi * g[:, None] * ks[None, :, 1])
    Z = np.exp(2j * math.pi * g[:, None] * ks[None, :, 2])
    a = amp * np.exp(1j * phi)
    vol = np.empty((n, n, n), np.float32)
    for z in range(n):
        w = a * Z[z]                                            # [m]
        vol[z] = ((Y * w[None, :]) @ X.T).real                  # [y, x]
    lo, hi = float(vol.min()), float(vol.max())
    q = np.empty((n, n, n), np.uint8)
    for z in range(n):
        q[z] = np.clip(np.rint((vol[z].astype(np.float64) - lo) * (255.0 / (hi - lo))), 0, 255)
    return q


def synthetic_server_image(width: int, height: int, seed: int, hole_frac: float = 0.05,
                           depth_range=(1.0, 1.4)):
    """A stand-in 2.5D colour + depth image (premultiplied RGBA float32 [H,W,4], depth float32 [H,W])
    with the structure of a volume rendering's depth image: a smooth depth field with a few depth
    discontinuities, mostly opaque pixels with translucent regions, and holes (depth = +inf)."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.linspace(0, 1, height), np.linspace(0, 1, width), indexing="ij")
    field = np.zeros((height, width))
    for _ in range(12):
        fx, fy = rng.uniform(0.5, 6, size=2)
        ph = rng.uniform(0, 2 * math.pi, size=2)
        field += rng.uniform(0.2, 1) * np.sin(2 * math.pi * fx * xx + ph[0]) * np.sin(2 * math.pi * fy * yy + ph[1])
    field = (field - field.min()) / (np.ptp(field) + 1e-12)
    steps = np.zeros((height, width))
    for _ in range(4):  # a few depth discontinuities (half-planes)
        a, b, c = rng.normal(size=3)
        steps += ((a * (xx - 0.5) + b * (yy - 0.5) + 0.2 * c) > 0) * rng.uniform(0.02, 0.08)
    lo, hi = depth_range
    depth = (lo + (hi - lo) * 0.8 * field + steps).astype(np.float32)
    alpha = np.where(rng.uniform(size=(height, width)) < 0.75, 1.0,
                     rng.uniform(0.05, 1.0, size=(height, width)))
    alpha = np.clip(alpha * (0.6 + 0.4 * field + 0.4), 0, 1)
    rgb = rng.uniform(0, 1, size=(height, width, 3)) * 0.3 + 0.7 * np.stack(
        [field, 1 - field, 0.5 + 0.5 * np.sin(6 * field)], axis=-1)
    rgba = np.concatenate([rgb * alpha[..., None], alpha[..., None]], axis=-1).astype(np.float32)
    holes = rng.uniform(size=(height, width)) < hole_frac
    depth[holes] = np.inf
    rgba[holes] = 0
    return rgba, depth


# ------------------------------------------------------------------------------------------------
# The five workloads.  Each returns plain parameters; the volumes are generated lazily.
# ------------------------------------------------------------------------------------------------
@dataclass(frozen=True)
class Workload:
    name: str
    vol_kind: str          # "gauss" | "fourier"
    vol_n: int
    vol_param: int         # blobs or modes
    server_w: int
    server_h: int
    client_w: int
    client_h: int
    eye_dist: float
    fovy: float
    n_poses: int
    cap_deg: float
    seed: int

    def volume(self, seed_offset: int = 0) -> np.ndarray:
        if self.vol_kind == "gauss":
            return gaussian_volume(self.vol_n, self.vol_param, self.seed + seed_offset)
        return fourier_volume(self.vol_n, self.vol_param, 32, self.seed + seed_offset)

    def server_cam(self, w: int = None, h: int = None) -> Camera:
        return server_camera(self.eye_dist, self.fovy, w or self.server_w, h or self.server_h)

    def client_poses(self, n: int = None, seed_offset: int = 0) -> List[Camera]:
        return poses_in_cap(self.server_cam(), n or self.n_poses, self.cap_deg,
                            self.seed + 500 + seed_offset, self.client_w, self.client_h)

    @property
    def voxel_diag(self) -> float:
        return float(np.float32(math.sqrt(3.0) / self.vol_n))


TINY = Workload("tiny: 32^3 f32 4 blobs, server 128^2, client 128^2 rotated 5 deg",
                "gauss", 32, 4, 128, 128, 128, 128, 2.0, 45.0, 1, 5.0, 1000)
MID = Workload("mid: 256^3 f32 64 blobs, server 512^2, client 1024^2, 30 poses within 15 deg",
               "gauss", 256, 64, 512, 512, 1024, 1024, 1.4, 30.0, 30, 15.0, 2000)
LARGE = Workload("large: 512^3 u8 256 Fourier modes, server 1920x1080, client 1920x1080, "
                 "60 poses within 20 deg, rebuild every 4 frames",
                 "fourier", 512, 256, 1920, 1080, 1920, 1080, 1.4, 30.0, 60, 20.0, 3000)
BATCHED = Workload("batched: 64 sessions of the mid volume, server sizes in {256,384,512,768,1024}^2, "
                   "client 1024^2, offsets within 15 deg",
                   "gauss", 256, 64, 512, 512, 1024, 1024, 1.4, 30.0, 64, 15.0, 4000)
DIFF = Workload("diff: 256^3 f32, server 512^2, 8 novel views within 10 deg at 512^2",
                "gauss", 256, 64, 512, 512, 512, 512, 1.4, 30.0, 8, 10.0, 5000)

BATCHED_SERVER_SIZES = (256, 384, 512, 768, 1024)


def tiny_client_camera() -> Camera:
    """The tiny workload's client: the server camera rotated 5 degrees about +y around the centre."""
    return orbit(TINY.server_cam(), (0.0, 1.0, 0.0), 5.0)


def batched_sessions(n: int = 64, seed: int = 4000):
    """Per-session (server size, client camera) for the batched workload."""
    rng = np.random.default_rng(seed)
    sizes = rng.choice(BATCHED_SERVER_SIZES, size=n)
    out = []
    for s in range(n):
        srv = BATCHED.server_cam(int(sizes[s]), int(sizes[s]))
        cli = poses_in_cap(srv, 1, BATCHED.cap_deg, seed + 100 + s, BATCHED.client_w,
                           BATCHED.client_h)[0]
        out.append((int(sizes[s]), srv, cli))
    return out


def gaussian_volume_device(n: int, nblobs: int, seed: int, device="cuda"):
    """The same Gaussian-blob law as :func:`gaussian_volume` (same seed -> same blobs), evaluated
    with torch on ``device`` in float64 and stored as float32.  Used where many large volumes are
    needed quickly (the batched workload); values may differ from the numpy version in the last
    bit of float32."""
    import torch
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(nblobs, 3))
    sig = rng.uniform(0.08, 0.15, size=nblobs)
    amp = rng.uniform(0.5, 1.0, size=nblobs)
    g = (torch.arange(n, dtype=torch.float64, device=device) + 0.5) / n
    vol = torch.zeros((n, n, n), dtype=torch.float64, device=device)
    for b in range(nblobs):
        ex = torch.exp(-((g - c[b, 0]) ** 2) / (2 * sig[b] ** 2))
        ey = torch.exp(-((g - c[b, 1]) ** 2) / (2 * sig[b] ** 2))
        ez = torch.exp(-((g - c[b, 2]) ** 2) / (2 * sig[b] ** 2))
        vol += amp[b] * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    vol /= vol.max()
    return vol.to(torch.float32)
