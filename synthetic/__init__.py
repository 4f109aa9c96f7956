"""Seeded synthetic cameras and Gaussian scenes.

This module only draws inputs: random numbers, camera intrinsics and poses.
It holds none of the rendering arithmetic (no ray generation, no footprint,
no response, no compositing), so both the FP64 oracle and the CUDA path can
take their inputs from it without sharing any of the method's code.

The paper evaluates on real captures (ScanNet++, Zip-NeRF fisheye, Mip-NeRF
360 pinhole; Sec. 5 "Datasets"), which are not available here.  The scenes
below stand in for them: Gaussian counts, resolutions and value
distributions follow the five benchmark workloads (C1..C5) listed in the
design notes.

Conventions (shared by every consumer of these inputs):
  * camera frame is OpenCV (x right, y down, z forward);
  * ``cam_to_world`` is a 3x4 row-major matrix [R | o]: R maps camera-frame
    directions to world, o is the optical centre;
  * pixel (i, j) covers [i, i+1) x [j, j+1); its centre is (i+0.5, j+0.5);
  * quaternions are (w, x, y, z);
  * SH coefficients are [n, (deg+1)^2, 3] in the (l, m = -l..l) order.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Iterator, List, Optional

import numpy as np

PINHOLE = 0
KB_FISHEYE = 1

SH_C0 = 0.28209479177387814  # 1 / (2 sqrt(pi)), the l=0 real SH constant


@dataclasses.dataclass
class Camera:
    model: int
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    k: np.ndarray = dataclasses.field(default_factory=lambda: np.zeros(4, np.float32))
    cam_to_world: np.ndarray = dataclasses.field(
        default_factory=lambda: np.concatenate([np.eye(3), np.zeros((3, 1))], 1).astype(np.float32))
    theta_lim: float = 0.0  # KB valid half field of view (rad); unused for pinhole

    def __post_init__(self):
        # Every parameter is stored exactly as an FP32 value; both sides read these.
        self.fx, self.fy = float(np.float32(self.fx)), float(np.float32(self.fy))
        self.cx, self.cy = float(np.float32(self.cx)), float(np.float32(self.cy))
        self.theta_lim = float(np.float32(self.theta_lim))
        self.k = np.asarray(self.k, np.float32).reshape(4)
        self.cam_to_world = np.asarray(self.cam_to_world, np.float32).reshape(3, 4)

    @property
    def intrinsics(self) -> np.ndarray:
        return np.array([self.fx, self.fy, self.cx, self.cy], np.float32)

    @property
    def n_pixels(self) -> int:
        return self.width * self.height

    def scaled(self, s: float) -> "Camera":
        """Same pose and model, calibration scaled with the resolution (Sec. 5 scale convention)."""
        w, h = max(1, int(round(self.width * s))), max(1, int(round(self.height * s)))
        return Camera(self.model, w, h, self.fx * s, self.fy * s, self.cx * s, self.cy * s,
                      self.k.copy(), self.cam_to_world.copy(), self.theta_lim)


@dataclasses.dataclass
class Scene:
    means: np.ndarray        # [n,3] f32
    log_scales: np.ndarray   # [n,3] f32
    quats: np.ndarray        # [n,4] f32 (w,x,y,z)
    opacity_logits: np.ndarray  # [n] f32
    sh: np.ndarray           # [n,(deg+1)^2,3] f32
    sh_degree: int
    rho2: np.ndarray         # [n] f32 (training-frequency floor; zeros = no floor)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def subset(self, idx) -> "Scene":
        idx = np.asarray(idx)
        return Scene(self.means[idx].copy(), self.log_scales[idx].copy(), self.quats[idx].copy(),
                     self.opacity_logits[idx].copy(), self.sh[idx].copy(), self.sh_degree,
                     self.rho2[idx].copy())

    def with_rho2(self, rho2) -> "Scene":
        return dataclasses.replace(self, rho2=np.asarray(rho2, np.float32).reshape(self.n))


# ----------------------------------------------------------------------------- cameras

def pinhole(width: int, height: int, f: float, cx: Optional[float] = None, cy: Optional[float] = None,
            cam_to_world=None) -> Camera:
    cam = Camera(PINHOLE, width, height, f, f,
                 width / 2.0 if cx is None else cx, height / 2.0 if cy is None else cy)
    if cam_to_world is not None:
        cam.cam_to_world = np.asarray(cam_to_world, np.float32).reshape(3, 4)
    return cam


def kb_limit(k: np.ndarray, theta_max: float = math.radians(95.0), min_slope: float = 0.25) -> float:
    """Valid half-FOV of a Kannala-Brandt camera: the largest theta <= theta_max
    below which d(theta_d)/d(theta) stays >= min_slope (so that the mapping
    is monotone and pixel footprints stay bounded near the edge)."""
    k = np.asarray(k, np.float64)
    th = np.linspace(0.0, theta_max, 200001)
    t2 = th * th
    slope = 1 + 3 * k[0] * t2 + 5 * k[1] * t2 ** 2 + 7 * k[2] * t2 ** 3 + 9 * k[3] * t2 ** 4
    bad = np.nonzero(slope < min_slope)[0]
    return float(th[bad[0] - 1]) if bad.size else float(theta_max)


def kb_theta_d(theta: float, k: np.ndarray) -> float:
    t2 = theta * theta
    k = np.asarray(k, np.float64)
    return theta * (1 + k[0] * t2 + k[1] * t2 ** 2 + k[2] * t2 ** 3 + k[3] * t2 ** 4)


def kb_fisheye(width: int, height: int, k, radius_px: Optional[float] = None, zoom: float = 1.0,
               cam_to_world=None) -> Camera:
    """KB equidistant fisheye with distortion k; the focal length puts the valid
    circle (radius theta_d(theta_lim) * f) at ``radius_px`` (default min(W,H)/2)."""
    k = np.asarray(k, np.float32)
    th_lim = float(np.float32(kb_limit(k)))
    rad = min(width, height) / 2.0 if radius_px is None else radius_px
    f = zoom * rad / kb_theta_d(th_lim, k)
    cam = Camera(KB_FISHEYE, width, height, f, f, width / 2.0, height / 2.0, k, theta_lim=th_lim)
    if cam_to_world is not None:
        cam.cam_to_world = np.asarray(cam_to_world, np.float32).reshape(3, 4)
    return cam


def look_at(eye, target) -> np.ndarray:
    """cam_to_world for an OpenCV camera at ``eye`` looking at ``target`` (world y is 'down')."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    x = np.cross(np.array([0.0, 1.0, 0.0]), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.concatenate([np.stack([x, y, z], 1), eye[:, None]], 1).astype(np.float32)


# ----------------------------------------------------------------------------- scenes

def _random_quats(rng, n) -> np.ndarray:
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def uniform_box_scene(n: int = 1000, seed: int = 0, log_scale_mean: float = -3.0,
                      log_scale_std: float = 0.5, sh_degree: int = 0) -> Scene:
    """C1 distribution: means U([-1,1]^2 x [2,6]), log-scales N(-3,0.5)^3, random unit
    quaternions, opacity logit N(0,1), RGB U[0,1] stored as the DC SH term."""
    rng = np.random.default_rng(seed)
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(2, 6, n)], 1)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _random_quats(rng, n)
    logits = rng.standard_normal(n)
    rgb = rng.uniform(0, 1, (n, 3))
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rgb - 0.5) / SH_C0
    if k > 1:
        sh[:, 1:, :] = rng.normal(0, 0.3, (n, k - 1, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats,
                 logits.astype(np.float32), sh.astype(np.float32), sh_degree, np.zeros(n, np.float32))


def blob_scene(n: int = 500_000, seed: int = 0, cam: Optional[Camera] = None, n_blobs: int = 64,
               blob_frac: float = 0.8, shell=(20.0, 25.0), log_scale_mean: float = -4.5,
               log_scale_std: float = 0.8, sh_degree: int = 3, target=None) -> Scene:
    """C2 distribution: ``blob_frac`` of the Gaussians in ``n_blobs`` isotropic clusters whose
    centres are uniform over the image of ``cam`` at z-depth U[3,12] (std 0.03 * depth), the
    rest uniform in volume in a spherical shell around the camera centre; log-scales
    N(-4.5,0.8)^3, SH degree 3 with coefficients N(0,0.3), opacity logit N(0,1)."""
    rng = np.random.default_rng(seed)
    cam = cam if cam is not None else pinhole(1280, 720, 1200.0)
    R = cam.cam_to_world[:, :3].astype(np.float64)
    o = cam.cam_to_world[:, 3].astype(np.float64)
    n_blob = int(round(n * blob_frac))
    n_shell = n - n_blob
    # blob centres, drawn in the camera frame of ``cam``
    px = rng.uniform(0, cam.width, n_blobs)
    py = rng.uniform(0, cam.height, n_blobs)
    z = rng.uniform(3.0, 12.0, n_blobs)
    centres_c = np.stack([(px - cam.cx) / cam.fx * z, (py - cam.cy) / cam.fy * z, z], 1)
    centres = centres_c @ R.T + o
    which = np.arange(n_blob) % n_blobs
    means_blob = centres[which] + rng.standard_normal((n_blob, 3)) * (0.03 * z[which])[:, None]
    # shell: direction uniform on the sphere, radius uniform in volume
    dirs = rng.standard_normal((n_shell, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    r = np.cbrt(rng.uniform(shell[0] ** 3, shell[1] ** 3, n_shell))
    means_shell = o + dirs * r[:, None]
    means = np.concatenate([means_blob, means_shell], 0)
    log_scales = rng.normal(log_scale_mean, log_scale_std, (n, 3))
    quats = _random_quats(rng, n)
    logits = rng.standard_normal(n)
    k = (sh_degree + 1) ** 2
    sh = rng.normal(0, 0.3, (n, k, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats,
                 logits.astype(np.float32), sh.astype(np.float32), sh_degree, np.zeros(n, np.float32))


def _quat_from_matrix(R: np.ndarray) -> np.ndarray:
    """(w, x, y, z) of rotation matrices R [n,3,3] (columns: the local axes in world)."""
    n = R.shape[0]
    q = np.zeros((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    for i in range(n):
        m = R[i]
        if tr[i] > 0:
            s = 2.0 * math.sqrt(1.0 + tr[i])
            q[i] = (0.25 * s, (m[2, 1] - m[1, 2]) / s, (m[0, 2] - m[2, 0]) / s, (m[1, 0] - m[0, 1]) / s)
        else:
            k = int(np.argmax([m[0, 0], m[1, 1], m[2, 2]]))
            a, b = (k + 1) % 3, (k + 2) % 3
            s = 2.0 * math.sqrt(1.0 + m[k, k] - m[a, a] - m[b, b])
            v = np.zeros(3)
            v[k] = 0.25 * s
            v[a] = (m[a, k] + m[k, a]) / s
            v[b] = (m[b, k] + m[k, b]) / s
            q[i] = ((m[b, a] - m[a, b]) / s, *v)
    return q


def flat_scene(n: int, seed: int = 0, ratio: float = 1e3, tilt_deg=(0.0, 30.0), cam: Optional[Camera] = None,
               fov_deg: float = 80.0, depth=(2.0, 6.0), log_scale_mean: float = -2.6, sh_degree: int = 1) -> Scene:
    """Near-degenerate flat Gaussians (disks): two scales exp(N(log_scale_mean, 0.3)), the
    third smaller than the larger of them by ``ratio`` x U(1.02, 1.3); the thin axis is
    tilted by U(tilt_deg) from the direction of the optical centre (0: seen face-on;
    near 90: edge-on, at a grazing angle).  Means: directions within ``fov_deg`` of the
    camera's optical axis, distance U(depth).  Opacity logit N(1, 0.5)."""
    rng = np.random.default_rng(seed)
    cam = cam if cam is not None else pinhole(96, 72, 90.0)
    Rc = cam.cam_to_world[:, :3].astype(np.float64)
    o = cam.cam_to_world[:, 3].astype(np.float64)
    ct = rng.uniform(math.cos(math.radians(fov_deg)), 1.0, n)
    ph = rng.uniform(0.0, 2.0 * math.pi, n)
    st = np.sqrt(1.0 - ct * ct)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], 1) @ Rc.T
    means = o + dirs * rng.uniform(depth[0], depth[1], n)[:, None]
    tilt = np.radians(rng.uniform(tilt_deg[0], tilt_deg[1], n))
    perp = np.cross(dirs, rng.standard_normal((n, 3)))
    perp /= np.linalg.norm(perp, axis=1, keepdims=True)
    thin = np.cos(tilt)[:, None] * dirs + np.sin(tilt)[:, None] * perp
    e1 = np.cross(thin, rng.standard_normal((n, 3)))
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(thin, e1)
    R = np.stack([e1, e2, thin], 2)
    big = rng.normal(log_scale_mean, 0.3, (n, 2))
    small = big.max(1) - np.log(ratio * rng.uniform(1.02, 1.3, n))
    log_scales = np.concatenate([big, small[:, None]], 1)
    quats = _quat_from_matrix(R)
    logits = rng.normal(1.0, 0.5, n)
    k = (sh_degree + 1) ** 2
    sh = np.zeros((n, k, 3))
    sh[:, 0, :] = (rng.uniform(0, 1, (n, 3)) - 0.5) / SH_C0
    if k > 1:
        sh[:, 1:, :] = rng.normal(0, 0.3, (n, k - 1, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats.astype(np.float32),
                 logits.astype(np.float32), sh.astype(np.float32), sh_degree, np.zeros(n, np.float32))


def _round_bf16(a: np.ndarray) -> np.ndarray:
    """FP32 values rounded to the nearest BF16 value (ties to even), as FP32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def quantized(scene: Scene, kind: str) -> Scene:
    """The scene with SH coefficients and opacity logits rounded to the half
    precision they are stored in ("bf16" or "f16"), kept as FP32 values."""
    if kind == "bf16":
        q = _round_bf16
    elif kind == "f16":
        q = lambda a: np.asarray(a, np.float32).astype(np.float16).astype(np.float32)
    else:
        raise ValueError(kind)
    return dataclasses.replace(scene, sh=q(scene.sh), opacity_logits=q(scene.opacity_logits))


def perturbed(scene: Scene, seed: int = 1) -> Scene:
    """The C3 target scene: mu + N(0,0.01), log s + N(0,0.05), DC + N(0,0.05), logit + N(0,0.1)."""
    rng = np.random.default_rng(seed)
    n = scene.n
    sh = scene.sh.copy()
    means = scene.means + rng.normal(0, 0.01, (n, 3)).astype(np.float32)
    log_scales = scene.log_scales + rng.normal(0, 0.05, (n, 3)).astype(np.float32)
    sh[:, 0, :] += rng.normal(0, 0.05, (n, 3)).astype(np.float32)
    logits = scene.opacity_logits + rng.normal(0, 0.1, n).astype(np.float32)
    return Scene(means, log_scales, scene.quats.copy(), logits, sh, scene.sh_degree, scene.rho2.copy())


# ----------------------------------------------------------------------------- workloads

def c1():
    """Plain forward, pinhole 64x48 (f=60, centred principal point), 1000 Gaussians, seed 0."""
    return pinhole(64, 48, 60.0), uniform_box_scene(1000, seed=0)


def c2_cameras() -> List[Camera]:
    """Pinhole 1280x720 (f=1200, same 56 deg HFOV as C1) and the same camera at 1/8 (160x90)."""
    full = pinhole(1280, 720, 1200.0)
    return [full, full.scaled(1.0 / 8.0)]


def c2_scene(n: int = 500_000, seed: int = 0) -> Scene:
    return blob_scene(n, seed=seed, cam=c2_cameras()[0])


def c3_camera(width: int = 1024, height: int = 1024, seed: int = 0) -> Camera:
    """KB equidistant fisheye, 190 deg FOV, k1..k4 ~ U(-0.05,0.05) (seed 0)."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(-0.05, 0.05, 4)
    return kb_fisheye(width, height, k)


def c3_scene(n: int = 1_000_000, seed: int = 0) -> Scene:
    return uniform_box_scene(n, seed=seed)


def c4_rig(scale_list=(1.0, 0.5, 0.25, 0.125), base=(1920, 1080), seed: int = 3) -> List[Camera]:
    """8 cameras on a circle of radius 0.5 in z=0 looking at (0,0,4): 4 pinhole (f=1800 s)
    and 4 KB fisheye (k seed 3, valid circle radius 540 s) at s in ``scale_list``."""
    rng = np.random.default_rng(seed)
    k = rng.uniform(-0.05, 0.05, 4)
    cams = []
    for i in range(8):
        ang = 2 * math.pi * i / 8
        pose = look_at((0.5 * math.cos(ang), 0.5 * math.sin(ang), 0.0), (0.0, 0.0, 4.0))
        s = scale_list[i % 4]
        w, h = int(round(base[0] * s)), int(round(base[1] * s))
        if i < 4:
            cams.append(pinhole(w, h, 1800.0 * s, cam_to_world=pose))
        else:
            cams.append(kb_fisheye(w, h, k, radius_px=540.0 * s, cam_to_world=pose))
    return cams


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    camera: Camera


def c5_requests(n_requests: int, rate_hz: float = 200.0, seed: int = 0) -> Iterator[Request]:
    """Poisson request stream: model Bernoulli(1/2); u ~ U(0,1), W = round(160*24^u),
    H = round(120*18^u); zoom 8^U(-1,1) multiplies the base focal length
    (pinhole f0 = W*60/64, KB f0 from its valid circle); pose uniform among the 8 C4 poses."""
    rng = np.random.default_rng(seed)
    rig = c4_rig()
    kb_k = rig[4].k
    t = 0.0
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        model = int(rng.integers(0, 2))
        u = rng.uniform(0, 1)
        w, h = int(round(160 * 24 ** u)), int(round(120 * 18 ** u))
        zoom = 8.0 ** rng.uniform(-1, 1)
        pose = rig[int(rng.integers(0, 8))].cam_to_world
        if model == PINHOLE:
            cam = pinhole(w, h, w * 60.0 / 64.0 * zoom, cam_to_world=pose)
        else:
            cam = kb_fisheye(w, h, kb_k, zoom=zoom, cam_to_world=pose)
        yield Request(rid, t, cam)
