"""Seeded synthetic inputs for the textured 2D-Gaussian rasterizer.

This module only draws random inputs and builds cameras; it holds none of the
rasterizer's arithmetic, so both the CUDA path and the FP64 oracle can consume
the very same arrays.  The workloads stand in for the paper's image-fitting,
NeRF360 and face-capture scenes (Sec. 4), none of which ships with the paper:

* ``cube``      - centres uniform in a cube, random frames (1k-splat case,
                  the splat budget of the paper's Fig. 4 overfit).
* ``planes``    - 80 % of the splats on 6 random planes with normal-aligned
                  frames, 20 % uniform clutter in a 10^3 box (100k / 1M / 3M
                  splat cases, the primitive budgets of Fig. 1, Fig. 6 and Sec. 4.2).
* ``fit_*``     - the image-fitting setup of Sec. 4.1: seeded synthetic target
                  images at the paper's three resolutions, a camera facing the
                  image plane and raw splat parameters in that plane.
* ``with_texel_sh`` - per-texel SH coefficients (Sec. 4.2) for a scene's grids.

Parameters are returned activated (linear scales, opacity in (0, 1)); the
log-scale / logit draws are turned into those values here.  Texture and SH
values that are stored in FP16 or BF16 are rounded here (round to nearest
even), so every consumer reads exactly the stored values.

A scene is a dict of float32 numpy arrays:
  means [K,3], quats [K,4] (w,x,y,z), scales [K,2], opacities [K],
  sh [K,(D+1)^2,3], textures [K,N,N,3] (C[i_u][i_v][rgb]),
and the ints / strings sh_degree, tex_n, sh_dtype, tex_dtype, sigma.
A camera is a dict: width, height, fx, fy, cx, cy (float32), R [3,3] and
t [3] (world-to-camera, OpenCV axes: x right, y down, z forward), near.
"""
from __future__ import annotations

import math

import numpy as np

SIGMA_DEFAULT = 0.5


# --------------------------------------------------------------------------
# storage rounding
# --------------------------------------------------------------------------

def round_to(x: np.ndarray, dtype: str) -> np.ndarray:
    """Rounds float32 values to the given storage type and back (RNE)."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    if dtype == "f32":
        return x.copy()
    if dtype == "f16":
        return x.astype(np.float16).astype(np.float32)
    if dtype == "bf16":
        # round to nearest even on the upper 16 bits; finite inputs stay below 2^32
        u = x.view(np.uint32).copy()
        lsb = (u >> 16) & 1
        u += np.uint32(0x7FFF)
        u += lsb
        u &= np.uint32(0xFFFF0000)
        return u.view(np.float32)
    raise ValueError(f"unknown storage dtype {dtype!r}")


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at(eye, target, width: int, height: int, fov_x_deg: float = 60.0,
            near: float = 0.01) -> dict:
    """Pinhole camera at ``eye`` looking at ``target``; world up is +y.

    Axes are OpenCV's: z_c = normalize(target - eye), x_c = normalize(z_c x up)
    (up = +x when the view is nearly vertical), y_c = z_c x x_c.  The field of
    view is horizontal, fx = fy = (W/2) / tan(fov/2), principal point (W/2, H/2).
    """
    eye = np.asarray(eye, np.float64)
    f = np.asarray(target, np.float64) - eye
    f /= np.linalg.norm(f)
    up = np.array([0.0, 1.0, 0.0])
    if abs(f @ up) > 0.999:
        up = np.array([1.0, 0.0, 0.0])
    x = np.cross(f, up)
    x /= np.linalg.norm(x)
    y = np.cross(f, x)
    R = np.stack([x, y, f])
    t = -R @ eye
    foc = (width / 2.0) / math.tan(math.radians(fov_x_deg) / 2.0)
    return {
        "width": int(width), "height": int(height),
        "fx": np.float32(foc), "fy": np.float32(foc),
        "cx": np.float32(width / 2.0), "cy": np.float32(height / 2.0),
        "R": R.astype(np.float32), "t": t.astype(np.float32), "near": np.float32(near),
    }


def fibonacci_dirs(n: int) -> np.ndarray:
    """n near-uniform unit directions on the sphere (golden-angle spiral)."""
    i = np.arange(n) + 0.5
    z = 1.0 - 2.0 * i / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = np.arange(n) * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def random_sphere_eye(rng: np.random.Generator, radius: float) -> np.ndarray:
    d = rng.standard_normal(3)
    return radius * d / np.linalg.norm(d)


# --------------------------------------------------------------------------
# splats
# --------------------------------------------------------------------------

def _unit_quats(rng, K):
    q = rng.standard_normal((K, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _quat_mul(a, b):
    aw, ax, ay, az = a.T
    bw, bx, by, bz = b.T
    return np.stack([
        aw * bw - ax * bx - ay * by - az * bz,
        aw * bx + ax * bw + ay * bz - az * by,
        aw * by - ax * bz + ay * bw + az * bx,
        aw * bz + ax * by - ay * bx + az * bw,
    ], axis=1)


def _normal_aligned_quats(rng, normals):
    """Quaternions whose frame has its third axis along ``normals``.

    Shortest-arc rotation from +z to n, composed with a random spin about z.
    """
    K = normals.shape[0]
    n = normals / np.linalg.norm(normals, axis=1, keepdims=True)
    ez = np.array([0.0, 0.0, 1.0])
    w = 1.0 + n @ ez
    xyz = np.cross(np.broadcast_to(ez, n.shape), n)
    qa = np.concatenate([w[:, None], xyz], axis=1)
    flip = w < 1e-6
    qa[flip] = np.array([0.0, 1.0, 0.0, 0.0])
    qa /= np.linalg.norm(qa, axis=1, keepdims=True)
    ang = rng.uniform(0.0, 2.0 * math.pi, K)
    qs = np.stack([np.cos(ang / 2), np.zeros(K), np.zeros(K), np.sin(ang / 2)], axis=1)
    return _quat_mul(qa, qs)


def _sigmoid(x):
    return 1.0 / (1.0 + np.exp(-x))


def _finish(rng, means, quats, log_scales, K, sh_degree, tex_n, sh_dtype, tex_dtype,
            sh_std=None, sh0_colour=False, sigma=SIGMA_DEFAULT) -> dict:
    M = (sh_degree + 1) ** 2
    opac = _sigmoid(rng.standard_normal(K))
    if sh0_colour:
        # "SH degree 0 colour ~ U[0,1]": colour = k00 * Y00, Y00 = 1 / (2 sqrt(pi))
        col = rng.uniform(0.0, 1.0, (K, 3))
        sh = np.zeros((K, M, 3))
        sh[:, 0, :] = col * (2.0 * math.sqrt(math.pi))
    else:
        sh = rng.normal(0.0, sh_std, (K, M, 3))
    tex = rng.uniform(0.0, 1.0, (K, tex_n, tex_n, 3))
    return {
        "means": np.ascontiguousarray(means, np.float32),
        "quats": np.ascontiguousarray(quats, np.float32),
        "scales": np.ascontiguousarray(np.exp(log_scales), np.float32),
        "opacities": np.ascontiguousarray(opac, np.float32),
        "sh": round_to(sh, sh_dtype),
        "textures": round_to(tex, tex_dtype),
        "sh_degree": int(sh_degree), "tex_n": int(tex_n),
        "sh_dtype": sh_dtype, "tex_dtype": tex_dtype, "sigma": float(sigma),
    }


def cube_scene(seed: int, K: int = 1000, half: float = 1.0, log_scale=(-3.0, 0.5),
               sh_degree: int = 0, tex_n: int = 4, sh_dtype: str = "f32",
               tex_dtype: str = "f32", sigma: float = SIGMA_DEFAULT) -> dict:
    """Centres U[-half, half]^3, uniform random frames, log-scales ~ N(mu, sd)."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-half, half, (K, 3))
    quats = _unit_quats(rng, K)
    ls = rng.normal(log_scale[0], log_scale[1], (K, 2))
    return _finish(rng, means, quats, ls, K, sh_degree, tex_n, sh_dtype, tex_dtype,
                   sh_std=0.1, sh0_colour=(sh_degree == 0), sigma=sigma)


def planes_scene(seed: int, K: int, half: float = 5.0, log_scale=(-4.0, 0.7),
                 sh_degree: int = 3, tex_n: int = 8, sh_dtype: str = "f32",
                 tex_dtype: str = "f32", n_planes: int = 6, clutter: float = 0.2,
                 sigma: float = SIGMA_DEFAULT) -> dict:
    """80 % of splats on random planes (normal-aligned frames), 20 % clutter."""
    rng = np.random.default_rng(seed)
    n_clutter = int(round(clutter * K))
    n_plane = K - n_clutter
    pts = rng.uniform(-half, half, (n_planes, 3))
    nrm = rng.standard_normal((n_planes, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    which = rng.integers(0, n_planes, n_plane)
    # orthonormal in-plane basis per plane
    ref = np.where(np.abs(nrm[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    e1 = np.cross(nrm, ref)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(nrm, e1)
    ab = rng.uniform(-half, half, (n_plane, 2))
    m_plane = pts[which] + ab[:, :1] * e1[which] + ab[:, 1:] * e2[which]
    q_plane = _normal_aligned_quats(rng, nrm[which])
    m_cl = rng.uniform(-half, half, (n_clutter, 3))
    q_cl = _unit_quats(rng, n_clutter)
    means = np.concatenate([m_plane, m_cl])
    quats = np.concatenate([q_plane, q_cl])
    ls = rng.normal(log_scale[0], log_scale[1], (K, 2))
    return _finish(rng, means, quats, ls, K, sh_degree, tex_n, sh_dtype, tex_dtype,
                   sh_std=0.1, sigma=sigma)


def subset(scene: dict, idx) -> dict:
    """The splats ``idx`` of a scene (arrays copied, metadata kept)."""
    out = dict(scene)
    for k in ("means", "quats", "scales", "opacities", "sh", "textures"):
        out[k] = np.ascontiguousarray(scene[k][idx])
    return out


def image_grads(seed: int, cams, channels: int = 3) -> list:
    """dL/d(image) ~ N(0, 1) per pixel and channel, one array per camera."""
    rng = np.random.default_rng(seed + 7919)
    return [rng.standard_normal((c["height"], c["width"], channels)).astype(np.float32) for c in cams]


# --------------------------------------------------------------------------
# the five workloads
# --------------------------------------------------------------------------

def workload(name: str, seed: int = 0, tex_n: int | None = None) -> dict:
    """Returns {"scenes": [...], "cams": [...], "cam_scene": [...], "d_rgb": [...]}.

    plain_1k       1,000 splats in [-1,1]^3, SH degree 0 colour, 4x4 FP32 textures,
                   one 128x128 camera (60 deg) at distance 4 looking at the origin.
    plain_100k     100,000 planar+clutter splats, SH degree 3 FP32, 8x8 FP32
                   textures, one 1280x720 camera on the radius-6 sphere.
    batched_1m     1,000,000 splats (same generator), FP16 SH and textures
                   (tex_n 4 or 8), 16 cameras on Fibonacci directions of the
                   radius-6 sphere at 960x540 / 1280x720 / 1920x1080 by i mod 3.
    train_3m       3,000,000 splats, BF16 SH degree 3 and 8x8 BF16 textures,
                   8 cameras at 1600x1067.
    multi_scene    12 scenes, splat counts log-uniform in [1e4, 2e6], texture
                   sizes cycling 2/4/8, FP16 storage, 1-4 cameras each.
    """
    if name == "plain_1k":
        sc = cube_scene(seed, K=1000, tex_n=tex_n or 4)
        cams = [look_at([0.0, 0.0, -4.0], [0, 0, 0], 128, 128)]
        return _pack([sc], cams, [0], seed)
    if name == "plain_100k":
        sc = planes_scene(seed, K=100_000, tex_n=tex_n or 8)
        rng = np.random.default_rng(seed + 1)
        cams = [look_at(random_sphere_eye(rng, 6.0), [0, 0, 0], 1280, 720)]
        return _pack([sc], cams, [0], seed)
    if name == "batched_1m":
        sc = planes_scene(seed, K=1_000_000, tex_n=tex_n or 4, sh_dtype="f16", tex_dtype="f16")
        res = [(960, 540), (1280, 720), (1920, 1080)]
        cams = [look_at(6.0 * d, [0, 0, 0], *res[i % 3]) for i, d in enumerate(fibonacci_dirs(16))]
        return _pack([sc], cams, [0] * 16, seed)
    if name == "train_3m":
        sc = planes_scene(seed, K=3_000_000, tex_n=tex_n or 8, sh_dtype="bf16", tex_dtype="bf16")
        cams = [look_at(6.0 * d, [0, 0, 0], 1600, 1067) for d in fibonacci_dirs(8)]
        return _pack([sc], cams, [0] * 8, seed)
    if name == "multi_scene":
        rng = np.random.default_rng(seed)
        res = [(512, 512), (960, 540), (1024, 768), (1280, 720), (1600, 900), (1920, 1080)]
        scenes, cams, cam_scene = [], [], []
        for s in range(12):
            K = int(round(math.exp(rng.uniform(math.log(1e4), math.log(2e6)))))
            scenes.append(planes_scene(100 + s, K=K, tex_n=[2, 4, 8][s % 3],
                                       sh_dtype="f16", tex_dtype="f16"))
            for _ in range(int(rng.integers(1, 5))):
                w, h = res[int(rng.integers(0, len(res)))]
                cams.append(look_at(random_sphere_eye(rng, 6.0), [0, 0, 0], w, h))
                cam_scene.append(s)
        return _pack(scenes, cams, cam_scene, seed)
    raise ValueError(f"unknown workload {name!r}")


def _pack(scenes, cams, cam_scene, seed):
    return {"scenes": scenes, "cams": cams, "cam_scene": list(cam_scene),
            "d_rgb": image_grads(seed, cams)}


# --------------------------------------------------------------------------
# tiny scenes for finite-difference and parity tests
# --------------------------------------------------------------------------

def tiny_camera(width: int = 16, height: int = 16, focal: float = 30.0,
                eye=(0.0, 0.0, -4.0)) -> dict:
    """Narrow-field camera so that a few splats cover a small image."""
    cam = look_at(eye, [0.0, 0.0, 0.0], width, height)
    cam["fx"] = np.float32(focal)
    cam["fy"] = np.float32(focal)
    return cam


def tiny_scene(seed: int, K: int = 5, tex_n: int = 4, sh_degree: int = 3,
               scale_range=(0.3, 0.8), spread: float = 0.5, sh_dtype: str = "f32",
               tex_dtype: str = "f32", sigma: float = SIGMA_DEFAULT) -> dict:
    """A handful of large, overlapping, randomly oriented splats near the origin."""
    rng = np.random.default_rng(seed)
    means = rng.uniform(-spread, spread, (K, 3))
    quats = _unit_quats(rng, K)
    ls = rng.uniform(math.log(scale_range[0]), math.log(scale_range[1]), (K, 2))
    out = _finish(rng, means, quats, ls, K, sh_degree, tex_n, sh_dtype, tex_dtype,
                  sh_std=0.2, sigma=sigma)
    out["opacities"] = rng.uniform(0.3, 0.95, K).astype(np.float32)
    return out


# --------------------------------------------------------------------------
# 2D image fitting (Sec. 4.1): synthetic targets, a camera facing the image
# plane and raw (pre-activation) splat parameters in that plane
# --------------------------------------------------------------------------

# the three target resolutions of the paper's image-fitting ablations
FIT_TARGETS = {"wide": (1920, 871), "landscape": (2016, 1512), "portrait": (1833, 2000)}


def fit_target(name_or_size, seed: int = 0) -> np.ndarray:
    """Seeded synthetic target image [H, W, 3] in [0, 1] (float32).

    ``name_or_size`` is a key of FIT_TARGETS or a (width, height) pair.  The
    image mixes a smooth colour field (random low-frequency cosines), 60
    soft-edged ellipses of random colour, size and orientation and two
    striped regions, so that it holds edges, gradients and texture at
    several scales; it stands in for the paper's photographs, none of which
    is reproduced."""
    W, H = FIT_TARGETS[name_or_size] if isinstance(name_or_size, str) else name_or_size
    rng = np.random.default_rng(seed + 7919)
    y, x = np.mgrid[0:H, 0:W].astype(np.float32)
    xn, yn = x / W, y / H
    img = np.zeros((H, W, 3), np.float32)
    for _ in range(8):
        kx, ky = rng.uniform(0.5, 4.0, 2)
        ph = rng.uniform(0, 2 * math.pi)
        amp = rng.uniform(0.05, 0.15, 3).astype(np.float32)
        img += amp * np.cos(2 * math.pi * (kx * xn + ky * yn) + ph)[..., None]
    img += 0.45
    for _ in range(60):
        cx, cy = rng.uniform(0, 1, 2)
        a, b = rng.uniform(0.01, 0.15, 2)
        th = rng.uniform(0, math.pi)
        c, s = math.cos(th), math.sin(th)
        col = rng.uniform(0, 1, 3).astype(np.float32)
        # window of the ellipse (1.5 x its larger semi-axis, in x-normalised units)
        r = 1.5 * max(a, b)
        x0, x1 = max(int((cx - r) * W), 0), min(int((cx + r) * W) + 1, W)
        y0, y1 = max(int((cy - r * W / H) * H), 0), min(int((cy + r * W / H) * H) + 1, H)
        if x0 >= x1 or y0 >= y1:
            continue
        xs, ys = xn[y0:y1, x0:x1], yn[y0:y1, x0:x1]
        u = ((xs - cx) * c + (ys - cy) * s * H / W) / a
        v = (-(xs - cx) * s + (ys - cy) * c * H / W) / b
        m = (1.0 / (1.0 + np.exp(np.clip(12.0 * (u * u + v * v - 1.0), -30, 30))))[..., None]
        img[y0:y1, x0:x1] = img[y0:y1, x0:x1] * (1 - 0.8 * m) + 0.8 * m * col
    for _ in range(2):
        x0, y0 = rng.uniform(0, 0.7, 2)
        w, h = rng.uniform(0.1, 0.3, 2)
        f = rng.uniform(20, 60)
        th = rng.uniform(0, math.pi)
        inside = (xn > x0) & (xn < x0 + w) & (yn > y0) & (yn < y0 + h)
        stripes = 0.5 + 0.5 * np.sin(2 * math.pi * f * (xn * math.cos(th) + yn * math.sin(th)))
        img = np.where(inside[..., None], 0.5 * img + 0.5 * stripes[..., None], img)
    return np.ascontiguousarray(np.clip(img, 0.0, 1.0), np.float32)


def fit_camera(width: int, height: int) -> dict:
    """Camera at the origin looking down +z with camera axes = world axes and
    focal length = width: the plane z = 1 spans x in [-1/2, 1/2]."""
    return {"width": int(width), "height": int(height), "fx": np.float32(width), "fy": np.float32(width),
            "cx": np.float32(width / 2), "cy": np.float32(height / 2), "R": np.eye(3, dtype=np.float32),
            "t": np.zeros(3, np.float32), "near": np.float32(0.01)}


def fit_init(K: int, width: int, height: int, seed: int = 0, tex_n: int = 4) -> dict:
    """Raw parameters of K splats for fitting a width x height image (Sec. 4.1):
    random position in the image plane z = 1 (plus a depth offset below 1e-3
    that fixes a strict order), random rotation angle about the view axis,
    random size (log-normal around the spacing of a K-splat grid over the
    image), random opacity logit and a random colour, held by the colour grid
    (constant per splat) with a zero SH term (degree 0).

    Returns float32 arrays: theta [K], xy [K,2], z [K], log_scales [K,2],
    logit_opacities [K], sh [K,1,3], textures [K,N,N,3]; plus tex_n and sigma.
    """
    rng = np.random.default_rng(seed + 104729)
    half_w, half_h = 0.5, 0.5 * height / width
    xy = np.stack([rng.uniform(-half_w, half_w, K), rng.uniform(-half_h, half_h, K)], 1)
    spacing = math.sqrt(4.0 * half_w * half_h / K)
    log_s = np.log(spacing * 0.5) + rng.normal(0.0, 0.3, (K, 2))
    col = rng.uniform(0.0, 1.0, (K, 1, 1, 3))
    return {
        "theta": rng.uniform(0.0, math.pi, K).astype(np.float32),
        "xy": xy.astype(np.float32),
        "z": (1.0 + 1e-3 * rng.permutation(K) / max(K, 1)).astype(np.float32),
        "log_scales": log_s.astype(np.float32),
        "logit_opacities": rng.normal(0.0, 1.0, K).astype(np.float32),
        "sh": np.zeros((K, 1, 3), np.float32),
        "textures": np.ascontiguousarray(np.broadcast_to(col, (K, tex_n, tex_n, 3)), np.float32),
        "tex_n": int(tex_n), "sigma": SIGMA_DEFAULT,
    }


def with_texel_sh(scene: dict, degree: int, seed: int = 0, std: float = 0.1) -> dict:
    """The scene with per-texel spherical harmonics of the given degree
    (Sec. 4.2): textures [K, N, N, (degree+1)^2, 3] whose degree-0 term keeps
    the texel's colour (k00 = colour 2 sqrt(pi)) and whose higher terms are
    N(0, std), rounded to the scene's texture storage type."""
    rng = np.random.default_rng(seed + 65537)
    K, N = scene["textures"].shape[:2]
    M = (degree + 1) ** 2
    k = rng.normal(0.0, std, (K, N, N, M, 3))
    k[:, :, :, 0, :] = scene["textures"].astype(np.float64) * (2.0 * math.sqrt(math.pi))
    out = dict(scene)
    out["textures"] = round_to(k, scene.get("tex_dtype", "f32"))
    out["tex_sh_degree"] = int(degree)
    return out


def with_splat_tex_n(scene: dict, sizes, seed: int = 0, fill: float = 7.0) -> dict:
    """The scene with a per-splat grid size: splat k gets n_k drawn from
    ``sizes`` (each <= the scene's tex_n) and keeps the texels in rows and
    columns 0..n_k-1 of its tex_n x tex_n block; the texels outside are set to
    ``fill`` (a renderer must never read them)."""
    rng = np.random.default_rng(seed)
    N = int(scene["tex_n"])
    K = int(scene["means"].shape[0])
    n = rng.choice(np.asarray(sizes, np.int32), K).astype(np.int32)
    assert n.min() >= 1 and n.max() <= N
    tex = np.array(scene["textures"], np.float32, copy=True)
    ii = np.arange(N)
    outside = (ii[None, :, None] >= n[:, None, None]) | (ii[None, None, :] >= n[:, None, None])
    tex[outside] = round_to(np.float32(fill), scene.get("tex_dtype", "f32"))
    return dict(scene, textures=tex, splat_tex_n=n)
