"""Seeded synthetic scenes, cameras and target images.

This module only draws inputs: random Gaussian parameters, look-at cameras and
target images, with the shapes and value distributions of the workloads the
method is measured on (4K outdoor scenes with millions of Gaussians). It holds
none of the rasterizer's arithmetic, so both the CUDA path and the CPU oracle
can be fed from it.

Workloads (seed = 2412135470 + index, NumPy PCG64, independent sub-streams for
scene, cameras and targets):

* ``small``  -- 128x128, 2,000 Gaussians uniform in [-1,1]^3, log-scales
  N(-3, 0.3), uniform unit quaternions, opacity logits N(0, 1.5), SH degree 0
  whose DC coefficient is drawn so that the colour is U[0,1]; target U[0,1].
* ``hd``     -- 1920x1080, 1M Gaussians: 90% from 64 anisotropic clusters, 10%
  on a background shell of radius 3; log-scales N(-4, 0.5); SH degree 3 (DC
  drawn for a U[0,1] colour, higher bands N(0, 0.05)).
* ``uhd``    -- 3840x2160, 3M Gaussians, same distribution.
* ``batch``  -- 8 views of mixed resolution (2 x 1920x1080, 3 x 2560x1440,
  3 x 3840x2160) at radius 2.6, random azimuth U[0, 360) and elevation
  U[0, 60] degrees, around 2M Gaussians of the same distribution of which 20%
  are packed into a ball at the origin whose image covers about 5% of a 4K
  frame (a heavy-tailed tile load).

Cameras look at the origin from radius 4 (small) or 2.6 (inside the background
shell, outside the cluster cube's circumsphere) with a 60 degree horizontal
field of view and square pixels; pixel centres sit at integer coordinates, so
the principal point is ((W-1)/2, (H-1)/2).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

BASE_SEED = 2412135470

# DC coefficient range that maps to colours in [0, 1] at SH degree 0: the
# degree-0 basis function is the constant 1/(2 sqrt(pi)) and the colour adds 0.5.
_DC_HALF_RANGE = math.sqrt(math.pi)


@dataclass
class Cam:
    """World-to-camera rotation R (3x3, rows = right, down, forward), translation T."""
    R: np.ndarray
    T: np.ndarray
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    z_near: float = 0.2


@dataclass
class Scene:
    means: np.ndarray          # (n, 3) float32
    log_scales: np.ndarray     # (n, 3) float32
    quats: np.ndarray          # (n, 4) float32, (w, x, y, z), not normalised
    opacity_logits: np.ndarray  # (n,)  float32
    sh: np.ndarray             # (n, (deg+1)^2, 3) float32
    sh_degree: int
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def as_dict(self) -> dict:
        return dict(means=self.means, log_scales=self.log_scales, quats=self.quats,
                    opacity_logits=self.opacity_logits, sh=self.sh)


def streams(index: int):
    """Independent generators for (scene, cameras, targets) of workload ``index``."""
    ss = np.random.SeedSequence(BASE_SEED + index)
    return [np.random.Generator(np.random.PCG64(s)) for s in ss.spawn(3)]


def look_at(eye, target=(0.0, 0.0, 0.0), up=(0.0, 0.0, 1.0), width=128, height=128,
            fov_x_deg=60.0, z_near=0.2) -> Cam:
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, np.float64))
    if np.linalg.norm(r) < 1e-9:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    dn = np.cross(f, r)
    R = np.stack([r, dn, f]).astype(np.float32).astype(np.float64)
    T = (-R @ eye).astype(np.float32).astype(np.float64)
    fx = float(np.float32(0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)))
    return Cam(R=R, T=T, fx=fx, fy=fx, cx=(width - 1) / 2.0, cy=(height - 1) / 2.0,
               width=int(width), height=int(height), z_near=z_near)


def orbit_eye(radius: float, azimuth_deg: float, elevation_deg: float):
    az, el = math.radians(azimuth_deg), math.radians(elevation_deg)
    return (radius * math.cos(el) * math.cos(az), radius * math.cos(el) * math.sin(az),
            radius * math.sin(el))


def _unit_quats(rng, n):
    return rng.standard_normal((n, 4)).astype(np.float32)


def _sh(rng, n, deg, high_sd=0.05):
    k = (deg + 1) ** 2
    sh = np.empty((n, k, 3), np.float32)
    sh[:, 0, :] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (n, 3))
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, high_sd, (n, k - 1, 3))
    return sh


def small_scene(n=2000, index=0, sh_degree=0, log_scale_mean=-3.0) -> Scene:
    rng, _, _ = streams(index)
    return Scene(
        means=rng.uniform(-1.0, 1.0, (n, 3)).astype(np.float32),
        log_scales=rng.normal(log_scale_mean, 0.3, (n, 3)).astype(np.float32),
        quats=_unit_quats(rng, n),
        opacity_logits=rng.normal(0.0, 1.5, n).astype(np.float32),
        sh=_sh(rng, n, sh_degree),
        sh_degree=sh_degree, name="small")


def _random_rotations(rng, k):
    """k random orthonormal frames (QR of Gaussian matrices, signs fixed)."""
    out = np.empty((k, 3, 3))
    for i in range(k):
        q, r = np.linalg.qr(rng.standard_normal((3, 3)))
        out[i] = q * np.sign(np.diag(r))
    return out


def cluster_scene(n: int, index: int, sh_degree=3, n_clusters=64, shell_frac=0.1,
                  shell_radius=3.0, log_scale_mean=-4.0, log_scale_sd=0.5,
                  packed_frac=0.0, packed_radius=0.0) -> Scene:
    """Clustered scene: anisotropic clusters in [-1,1]^3 plus a background shell;
    optionally a fraction packed into a small ball at the origin (heavy-tailed
    tile load)."""
    rng, _, _ = streams(index)
    n_shell = int(round(n * shell_frac))
    n_packed = int(round(n * packed_frac))
    n_clu = n - n_shell - n_packed
    centres = rng.uniform(-1.0, 1.0, (n_clusters, 3))
    rots = _random_rotations(rng, n_clusters)
    sds = np.exp(rng.uniform(math.log(0.05), math.log(0.3), (n_clusters, 3)))
    weights = rng.dirichlet(np.ones(n_clusters))
    counts = rng.multinomial(n_clu, weights)
    parts = []
    for c in range(n_clusters):
        if counts[c] == 0:
            continue
        z = rng.standard_normal((counts[c], 3)) * sds[c]
        parts.append(centres[c] + z @ rots[c].T)
    means = [np.concatenate(parts, 0)] if parts else []
    if n_shell:
        d = rng.standard_normal((n_shell, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        means.append(d * (shell_radius + rng.normal(0.0, 0.02, (n_shell, 1))))
    if n_packed:
        d = rng.standard_normal((n_packed, 3))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        means.append(d * packed_radius * np.cbrt(rng.uniform(0.0, 1.0, (n_packed, 1))))
    means = np.concatenate(means, 0).astype(np.float32)
    perm = rng.permutation(n)
    means = means[perm]
    return Scene(
        means=np.ascontiguousarray(means),
        log_scales=rng.normal(log_scale_mean, log_scale_sd, (n, 3)).astype(np.float32),
        quats=_unit_quats(rng, n),
        opacity_logits=rng.normal(0.0, 1.5, n).astype(np.float32),
        sh=_sh(rng, n, sh_degree),
        sh_degree=sh_degree, name="clusters")


def target_image(width: int, height: int, index: int, seed_offset: int = 0) -> np.ndarray:
    """U[0,1] target, height x width x 3 float32."""
    _, _, rng = streams(index)
    if seed_offset:
        rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([BASE_SEED + index, seed_offset])))
    return rng.uniform(0.0, 1.0, (height, width, 3)).astype(np.float32)


def quantize_u8(img: np.ndarray) -> np.ndarray:
    """An image in [0, 1] as 8-bit values (round to nearest), the form photographs
    are stored in and the kernels accept as targets (GS_TARGET_U8)."""
    return np.clip(np.rint(np.asarray(img, np.float64) * 255.0), 0, 255).astype(np.uint8)


def u8_values(img8: np.ndarray) -> np.ndarray:
    """The FP32 values the kernels read for an 8-bit target: t * (1/255), 1/255
    rounded to FP32 and the product rounded to FP32."""
    return np.asarray(img8, np.uint8).astype(np.float32) * np.float32(1.0 / 255.0)


# ----------------------------------------------------------------------------
# Named workloads
# ----------------------------------------------------------------------------

def workload_small():
    """128x128 view, 2k Gaussians, SH degree 0, camera at radius 4."""
    scene = small_scene(2000, index=0)
    cam = look_at(orbit_eye(4.0, 30.0, 20.0), width=128, height=128)
    return scene, cam, target_image(128, 128, 0)


def workload_hd(n=1_000_000):
    """1920x1080 view, 1M clustered Gaussians, SH degree 3, camera at radius 2.6."""
    scene = cluster_scene(n, index=1)
    cam = look_at(orbit_eye(2.6, 30.0, 20.0), width=1920, height=1080)
    return scene, cam, target_image(1920, 1080, 1)


def workload_uhd(n=3_000_000):
    """3840x2160 view, 3M clustered Gaussians, SH degree 3, camera at radius 2.6."""
    scene = cluster_scene(n, index=2)
    cam = look_at(orbit_eye(2.6, 30.0, 20.0), width=3840, height=2160)
    return scene, cam, target_image(3840, 2160, 2)


BATCH_RESOLUTIONS = ((1920, 1080),) * 2 + ((2560, 1440),) * 3 + ((3840, 2160),) * 3


def packed_ball_radius(frac_of_frame=0.05, width=3840, height=2160, distance=2.6, fov_x_deg=60.0):
    """World radius of a ball at the origin whose image disc covers the given
    fraction of a frame seen from ``distance``."""
    f = 0.5 * width / math.tan(math.radians(fov_x_deg) / 2.0)
    r_px = math.sqrt(frac_of_frame * width * height / math.pi)
    return r_px * distance / f


def workload_batch(n=2_000_000, resolutions=BATCH_RESOLUTIONS, with_targets=True):
    """Mixed-resolution views of one clustered 2M-Gaussian scene with 20%
    of the Gaussians packed into a ball covering ~5% of a 4K frame."""
    scene = cluster_scene(n, index=3, packed_frac=0.2, packed_radius=packed_ball_radius())
    _, rng, _ = streams(3)
    cams = []
    for w, h in resolutions:
        az, el = rng.uniform(0.0, 360.0), rng.uniform(0.0, 60.0)
        cams.append(look_at(orbit_eye(2.6, az, el), width=w, height=h))
    targets = [target_image(c.width, c.height, 3, seed_offset=i + 1) for i, c in enumerate(cams)] \
        if with_targets else None
    return scene, cams, targets


def fit_workload(n_gt=2_000_000, n_init=100_000, n_train=200, n_eval=10, width=3840, height=2160, index=4):
    """A scene to fit: a clustered SH-3 ground truth (the hd distribution),
    training and held-out cameras on a jittered ring/hemisphere (radius
    2.6 +- U(0.1), elevation U[0, 60] degrees, look-at jitter N(0, 0.02)), and
    an initialisation of n_init points drawn from the ground-truth means with
    N(0, 0.02) noise, log-scale -4.5, random rotations, opacity 0.1 and the DC
    colour of the Gaussian each point was drawn from plus N(0, 0.05) noise."""
    gt = cluster_scene(n_gt, index=index)
    _, rng_cam, rng_init = streams(index)
    cams = []
    for _ in range(n_train + n_eval):
        r = 2.6 + rng_cam.uniform(-0.1, 0.1)
        eye = orbit_eye(r, rng_cam.uniform(0.0, 360.0), rng_cam.uniform(0.0, 60.0))
        cams.append(look_at(eye, target=tuple(rng_cam.normal(0.0, 0.02, 3)), width=width, height=height))
    src = rng_init.integers(0, n_gt, n_init)
    k = gt.sh.shape[1]
    sh = np.zeros((n_init, k, 3), np.float32)
    sh[:, 0, :] = gt.sh[src, 0, :] + rng_init.normal(0.0, 0.05, (n_init, 3))
    init = dict(means=(gt.means[src] + rng_init.normal(0.0, 0.02, (n_init, 3))).astype(np.float32),
                log_scales=np.full((n_init, 3), -4.5, np.float32),
                quats=_unit_quats(rng_init, n_init),
                opacity_logits=np.full(n_init, math.log(0.1 / 0.9), np.float32),
                sh=sh)
    return gt, init, cams[:n_train], cams[n_train:]


def rotating_offset(step: int, d: int):
    """Seeded rotation through the d*d offsets: step -> (ox, oy)."""
    k = step % (d * d)
    return k % d, k // d
