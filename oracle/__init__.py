"""FP64 CPU oracle for the Gaussian Billboards rasterizer (arXiv 2412.12734).

TEST INFRASTRUCTURE ONLY.  The test-suite, the smoke check and the CPU-baseline
leg of the bench are the only callers.  The product library never imports,
links or runs anything in this directory, and this directory imports nothing
from the product package: the two sides see the same seeded input arrays and
nothing else.

The arithmetic lives in ``gbill_oracle.cpp`` (plain C++17, FP64, brute force
over every splat at every pixel with an explicit depth sort).  This module
only marshals numpy arrays through ctypes, plus two steps that are plain
library primitives: turning FP32 pixel rectangles into tile keys and sorting
them (numpy's stable argsort).

Sections cited: Sec. 3.1 Eq. 2-4 (compositing, 2DGS plane, uv Gaussian),
Sec. 3.2 Eq. 5 (bilinear colour grid), Sec. 4.2 (SH added to the grid colour),
Alg. 1 (rasterize fwd/bwd), Alg. 2 (bilinear / adj-bilinear), Sec. 4.1 and
Fig. 4 f, g (colour grid box-filtered to a coarser mip level at render time).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gbill_oracle.cpp")
_SO = os.path.join(_HERE, "libgbill_oracle.so")
_lock = threading.Lock()
_lib = None

GXX_FLAGS = ["-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread"]


def build(force: bool = False) -> str:
    """Compiles the oracle with g++ if the shared object is missing or stale."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", *GXX_FLAGS, "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


class _Scene(C.Structure):
    _fields_ = [
        ("num_splats", C.c_int64),
        ("means", C.c_void_p), ("quats", C.c_void_p), ("scales", C.c_void_p),
        ("opacities", C.c_void_p), ("sh", C.c_void_p), ("textures", C.c_void_p),
        ("sh_degree", C.c_int32), ("tex_n", C.c_int32), ("sigma", C.c_double),
        ("splat_n", C.c_void_p),
    ]


class _Camera(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32),
        ("fx", C.c_double), ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
        ("w2c", C.c_double * 12), ("near_plane", C.c_double),
    ]


class _Window(C.Structure):
    _fields_ = [("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32), ("h", C.c_int32)]


class _FwdOut(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("rgb", "depth", "alpha", "t_final", "n_contrib", "margin_fwd", "margin_grad", "n_pairs")]


class _Grads(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in
                ("d_means", "d_quats", "d_scales", "d_opacities", "d_sh", "d_textures")]


def load(path: str) -> C.CDLL:
    """Opens a compiled oracle (this directory's, or a test's variant of it)."""
    L = C.CDLL(path)
    for name in ("orc_render_forward", "orc_render_backward", "orc_keys32", "orc_project",
                 "orc_eval_pairs", "orc_sh_basis", "orc_bilinear", "orc_adj_bilinear",
                 "orc_num_threads", "orc_pixel_trace"):
        getattr(L, name).restype = C.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = load(_SO)
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def mip_grid(textures, level: int):
    """Colour grids box-filtered to mip level ``level`` (Sec. 4.1, Fig. 4 f, g):
    texel (i, j) of the (N/2^l) x (N/2^l) grid is the mean of the 2^l x 2^l
    block of texels (2^l i + a, 2^l j + b), a, b < 2^l.  Level 0 is the grid
    itself."""
    t = _f64(textures)
    K, N = t.shape[0], t.shape[1]
    f = 1 << int(level)
    if N % f:
        raise ValueError(f"mip level {level} needs N divisible by {f}")
    return np.ascontiguousarray(t.reshape(K, N // f, f, N // f, f, 3).mean(axis=(2, 4)))


def mip_grid_adjoint(d_coarse, level: int):
    """Adjoint of mip_grid: every fine texel of a block receives 1/4^l of the
    block's coarse gradient."""
    f = 1 << int(level)
    return np.repeat(np.repeat(_f64(d_coarse), f, axis=1), f, axis=2) / float(f * f)


class _SceneRef:
    """Holds FP64 copies (exact upcasts of the stored values) alive for a call.
    A scene with ``mip_level`` l > 0 is rendered with its grids box-filtered
    to N / 2^l (mip_grid).  A scene with ``splat_tex_n`` [K] renders splat k
    with the n_k x n_k grid in rows and columns 0..n_k-1 of its N x N block
    (Alg. 2 with n_k)."""

    def __init__(self, scene: dict):
        self.splat_n = None
        if scene.get("splat_tex_n") is not None:
            if int(scene.get("mip_level", 0)) or int(scene.get("tex_sh_degree", 0)):
                raise ValueError("per-splat grid sizes take no mip level and no per-texel SH")
            self.splat_n = np.ascontiguousarray(np.asarray(scene["splat_tex_n"]).astype(np.int32))
            assert self.splat_n.min() >= 1 and self.splat_n.max() <= int(scene["tex_n"])
        self.arrays = {k: _f64(scene[k]) for k in
                       ("means", "quats", "scales", "opacities", "sh", "textures")}
        self.K = int(self.arrays["means"].shape[0])
        self.D = int(scene["sh_degree"])
        self.mip = int(scene.get("mip_level", 0))
        self.N_src = int(scene["tex_n"])
        if self.mip:
            self.arrays["textures"] = mip_grid(self.arrays["textures"], self.mip)
        self.N = self.N_src >> self.mip
        s = _Scene()
        s.num_splats = self.K
        for k, a in self.arrays.items():
            setattr(s, k, _p(a))
        s.sh_degree = self.D
        s.tex_n = self.N
        s.sigma = float(scene.get("sigma", 0.5))
        s.splat_n = _p(self.splat_n) if self.splat_n is not None else None
        self.struct = s


def _camera(cam: dict) -> _Camera:
    c = _Camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(cam[k])) for k in ("fx", "fy", "cx", "cy"))
    R = np.asarray(cam["R"], dtype=np.float32).astype(np.float64)
    t = np.asarray(cam["t"], dtype=np.float32).astype(np.float64)
    w2c = np.concatenate([R, t[:, None]], axis=1).reshape(-1)
    for i in range(12):
        c.w2c[i] = float(w2c[i])
    c.near_plane = float(np.float32(cam.get("near", 0.01)))
    return c


def _window(cam: dict, window):
    if window is None:
        window = (0, 0, int(cam["width"]), int(cam["height"]))
    w = _Window()
    w.x0, w.y0, w.w, w.h = (int(v) for v in window)
    return w


def num_threads() -> int:
    return int(lib().orc_num_threads())


def _campos(cam: dict) -> np.ndarray:
    R = np.asarray(cam["R"], dtype=np.float32).astype(np.float64)
    t = np.asarray(cam["t"], dtype=np.float32).astype(np.float64)
    return -R.T @ t


def tex_sh_grids(scene: dict, cam: dict):
    """Per-texel spherical harmonics (Sec. 4.2: M coefficient triples per texel
    instead of one RGB colour): the colour grid each splat shows to ``cam``,
    texel colour = sum_lm k_texel,lm Y_lm(d) with d = (p - camera centre) /
    |p - camera centre|, the splat's view direction.  ``scene["textures"]`` is
    [K, N, N, (Dt+1)^2, 3] with Dt = scene["tex_sh_degree"] >= 1.

    Returns (grids [K,N,N,3], Y [K,M], dY/dd [K,M,3], d [K,3], |p - c| [K],
    coefficients [K,N,N,M,3])."""
    Dt = int(scene["tex_sh_degree"])
    M = (Dt + 1) ** 2
    K, N = int(np.shape(scene["means"])[0]), int(scene["tex_n"])
    p = _f64(scene["means"])
    v = p - _campos(cam)[None, :]
    dist = np.sqrt(np.sum(v * v, axis=1))
    d = v / dist[:, None]
    Y, dY = sh_basis(Dt, d)
    k = _f64(scene["textures"]).reshape(K, N, N, M, 3)
    return np.einsum("km,kijmc->kijc", Y, k), Y, dY, d, dist, k


def _view_scene(scene: dict, cam: dict):
    """The scene with plain RGB grids that ``cam`` sees (per-texel SH evaluated)."""
    if int(scene.get("tex_sh_degree", 0)) <= 0:
        return scene, None
    if int(scene.get("mip_level", 0)):
        raise ValueError("per-texel SH takes no mip level")
    ev = tex_sh_grids(scene, cam)
    return dict(scene, textures=ev[0], tex_sh_degree=0), ev


def render(scene: dict, cam: dict, window=None, bg=None, prefilter: bool = False) -> dict:
    """Brute-force FP64 forward of one view (Alg. 1 fwd, Eq. 2, Eq. 5).

    Returns rgb [h,w,3], depth, alpha, t_final, n_contrib, margin_fwd,
    margin_grad (each [h,w]) and the number of (pixel, splat) pairs
    evaluated.
    """
    scene, _ = _view_scene(scene, cam)
    S = _SceneRef(scene)
    cm = _camera(cam)
    win = _window(cam, window)
    h, w = win.h, win.w
    out = {
        "rgb": np.zeros((h, w, 3)), "depth": np.zeros((h, w)), "alpha": np.zeros((h, w)),
        "t_final": np.zeros((h, w)), "n_contrib": np.zeros((h, w), np.int32),
        "margin_fwd": np.zeros((h, w)), "margin_grad": np.zeros((h, w)),
        "n_pairs": np.zeros(1, np.int64),
    }
    fo = _FwdOut()
    for k, a in out.items():
        setattr(fo, k, _p(a))
    bgv = _f64(bg) if bg is not None else None
    rc = lib().orc_render_forward(C.byref(S.struct), C.byref(cm), C.byref(win),
                                  _p(bgv) if bgv is not None else None, int(prefilter), C.byref(fo))
    assert rc == 0
    out["n_pairs"] = int(out["n_pairs"][0])
    return out


def backward(scene: dict, cam: dict, dL_drgb, dL_ddepth=None, dL_dalpha=None, window=None,
             bg=None, prefilter: bool = False, grads: dict | None = None) -> dict:
    """FP64 analytic backward of one view (Alg. 1 bwd, Alg. 2 adj-bilinear).

    Gradients are ACCUMULATED into ``grads`` when given (sum over views).
    """
    if int(scene.get("tex_sh_degree", 0)) > 0:
        return _backward_tex_sh(scene, cam, dL_drgb, dL_ddepth, dL_dalpha, window, bg, prefilter, grads)
    S = _SceneRef(scene)
    cm = _camera(cam)
    win = _window(cam, window)
    K, D, N = S.K, S.D, S.N_src
    if grads is None:
        grads = {
            "means": np.zeros((K, 3)), "quats": np.zeros((K, 4)), "scales": np.zeros((K, 2)),
            "opacities": np.zeros(K), "sh": np.zeros((K, (D + 1) ** 2, 3)),
            "textures": np.zeros((K, N, N, 3)),
        }
    g = _Grads()
    for k in ("means", "quats", "scales", "opacities", "sh", "textures"):
        assert grads[k].dtype == np.float64 and grads[k].flags.c_contiguous
        setattr(g, "d_" + k, _p(grads[k]))
    d_coarse = None
    if S.mip:
        # the C oracle differentiates the box-filtered grid; mip_grid_adjoint maps back
        d_coarse = np.zeros((K, S.N, S.N, 3))
        g.d_textures = _p(d_coarse)
    drgb = _f64(dL_drgb).reshape(win.h, win.w, 3)
    ddep = _f64(dL_ddepth).reshape(win.h, win.w) if dL_ddepth is not None else None
    dalp = _f64(dL_dalpha).reshape(win.h, win.w) if dL_dalpha is not None else None
    bgv = _f64(bg) if bg is not None else None
    rc = lib().orc_render_backward(C.byref(S.struct), C.byref(cm), C.byref(win),
                                   _p(bgv) if bgv is not None else None, int(prefilter), _p(drgb),
                                   _p(ddep) if ddep is not None else None,
                                   _p(dalp) if dalp is not None else None, C.byref(g))
    assert rc == 0
    if d_coarse is not None:
        grads["textures"] += mip_grid_adjoint(d_coarse, S.mip)
    return grads


def _backward_tex_sh(scene, cam, dL_drgb, dL_ddepth, dL_dalpha, window, bg, prefilter, grads):
    """Backward with per-texel SH: the view's grid gradient C^ gives the
    coefficient gradients Y_lm(d) C^ and, through d, a term of the centre
    gradient: sum C^ . k dY/dd, projected by (I - d d^T) / |p - c|."""
    view, (grid, Y, dY, d, dist, k) = _view_scene(scene, cam)
    K, N = k.shape[0], k.shape[1]
    M = Y.shape[1]
    if grads is None:
        D = int(scene["sh_degree"])
        grads = {
            "means": np.zeros((K, 3)), "quats": np.zeros((K, 4)), "scales": np.zeros((K, 2)),
            "opacities": np.zeros(K), "sh": np.zeros((K, (D + 1) ** 2, 3)),
            "textures": np.zeros((K, N, N, M, 3)),
        }
    g = backward(view, cam, dL_drgb, dL_ddepth, dL_dalpha, window=window, bg=bg, prefilter=prefilter)
    for key in ("means", "quats", "scales", "opacities", "sh"):
        grads[key] += g[key]
    ch = g["textures"]  # [K, N, N, 3]
    grads["textures"] += np.einsum("km,kijc->kijmc", Y, ch).reshape(grads["textures"].shape)
    g_dir = np.einsum("kijc,kijmc,kmx->kx", ch, k, dY)
    dd = np.sum(g_dir * d, axis=1)
    grads["means"] += (g_dir - d * dd[:, None]) / dist[:, None]
    return grads


def keys32(scene: dict, cam: dict):
    """FP32 culling decision, depth and inclusive pixel rectangle per splat (R14-R16)."""
    S = _SceneRef(scene)
    cm = _camera(cam)
    valid = np.zeros(S.K, np.int32)
    depth = np.zeros(S.K, np.float32)
    prect = np.zeros((S.K, 4), np.int32)
    rc = lib().orc_keys32(C.byref(S.struct), C.byref(cm), _p(valid), _p(depth), _p(prect))
    assert rc == 0
    return valid.astype(bool), depth, prect


def tile_keys(scene: dict, cam: dict, tile: int, tile_offset: int = 0):
    """Sorted (key, splat id) list of one view.

    key = (global tile id << 32) | bits(FP32 depth); instances are emitted in
    splat order and sorted stably, so equal keys keep ascending splat ids.
    """
    valid, depth, prect = keys32(scene, cam)
    tiles_x = (int(cam["width"]) + tile - 1) // tile
    keys, ids = [], []
    dbits = depth.view(np.uint32).astype(np.uint64)
    for k in np.nonzero(valid)[0]:
        x0, y0, x1, y1 = (int(v) for v in prect[k])
        tx = np.arange(x0 // tile, x1 // tile + 1)
        ty = np.arange(y0 // tile, y1 // tile + 1)
        t = (tile_offset + ty[:, None] * tiles_x + tx[None, :]).reshape(-1).astype(np.uint64)
        keys.append((t << np.uint64(32)) | dbits[k])
        ids.append(np.full(t.shape, k, np.int64))
    if not keys:
        return np.zeros(0, np.uint64), np.zeros(0, np.int64)
    keys = np.concatenate(keys)
    ids = np.concatenate(ids)
    order = np.argsort(keys, kind="stable")
    return keys[order], ids[order]


def project(scene: dict, cam: dict) -> dict:
    """FP64 homography T, adj(T), projected centre, SH colour and FP64 bbox per splat."""
    S = _SceneRef(scene)
    cm = _camera(cam)
    K = S.K
    out = {"T": np.zeros((K, 3, 3)), "adj": np.zeros((K, 3, 3)), "centre": np.zeros((K, 2)),
           "rgb_sh": np.zeros((K, 3)), "bbox": np.zeros((K, 4))}
    rc = lib().orc_project(C.byref(S.struct), C.byref(cm), _p(out["T"]), _p(out["adj"]),
                           _p(out["centre"]), _p(out["rgb_sh"]), _p(out["bbox"]))
    assert rc == 0
    return out


def eval_pairs(scene: dict, cam: dict, k: int, xy) -> dict:
    """u, v, alpha and branch of splat k at the given pixel-centre coordinates."""
    S = _SceneRef(scene)
    cm = _camera(cam)
    xy = _f64(xy).reshape(-1, 2)
    n = xy.shape[0]
    u, v, a = np.zeros(n), np.zeros(n), np.zeros(n)
    br = np.zeros(n, np.int32)
    rc = lib().orc_eval_pairs(C.byref(S.struct), C.byref(cm), C.c_int64(k), _p(xy), C.c_int64(n),
                              _p(u), _p(v), _p(a), _p(br))
    assert rc == 0
    return {"u": u, "v": v, "alpha": a, "uv_branch": br}


def sh_basis(D: int, dirs):
    """Y[n, (D+1)^2] and dY/dd[n, (D+1)^2, 3] of the oracle's SH basis."""
    dirs = _f64(dirs).reshape(-1, 3)
    n = dirs.shape[0]
    M = (D + 1) ** 2
    Y = np.zeros((n, M))
    dY = np.zeros((n, M, 3))
    rc = lib().orc_sh_basis(C.c_int32(D), _p(dirs), C.c_int64(n), _p(Y), _p(dY))
    assert rc == 0
    return Y, dY


def bilinear(uv, N: int, sigma: float, grid):
    """Alg. 2 bilinear at each (u, v) row of ``uv`` on grid [N, N, 3]."""
    uv = _f64(uv).reshape(-1, 2)
    grid = _f64(grid).reshape(N, N, 3)
    out = np.zeros((uv.shape[0], 3))
    rc = lib().orc_bilinear(_p(uv), C.c_int64(uv.shape[0]), C.c_int32(N), C.c_double(sigma),
                            _p(grid), _p(out))
    assert rc == 0
    return out


def adj_bilinear(uv, N: int, sigma: float, grid, chat):
    """Alg. 2 adj-bilinear: grid adjoint (summed over rows) and per-row uv adjoint."""
    uv = _f64(uv).reshape(-1, 2)
    grid = _f64(grid).reshape(N, N, 3)
    chat = _f64(chat).reshape(-1, 3)
    Chat = np.zeros((N, N, 3))
    uvh = np.zeros((uv.shape[0], 2))
    rc = lib().orc_adj_bilinear(_p(uv), C.c_int64(uv.shape[0]), C.c_int32(N), C.c_double(sigma),
                                _p(grid), _p(chat), _p(Chat), _p(uvh))
    assert rc == 0
    return Chat, uvh


def pixel_trace(scene: dict, cam: dict, px: int, py: int, cap: int = 4096) -> dict:
    """Blended splats of one pixel in order: ids, alpha, transmittance before each."""
    S = _SceneRef(scene)
    cm = _camera(cam)
    ids = np.zeros(cap, np.int64)
    a = np.zeros(cap)
    tr = np.zeros(cap)
    tf = np.zeros(1)
    n = lib().orc_pixel_trace(C.byref(S.struct), C.byref(cm), C.c_int32(px), C.c_int32(py),
                              C.c_int32(cap), _p(ids), _p(a), _p(tr), _p(tf))
    n = min(n, cap)
    return {"ids": ids[:n], "alpha": a[:n], "trans": tr[:n], "t_final": float(tf[0])}


def adam_step(param, grad, m, v, step: int, lr: float, beta1: float, beta2: float, eps: float):
    """Adam (Kingma & Ba, Algorithm 1; the optimiser of Sec. 3.3) in FP64.

    Returns the new (param, m, v); inputs are not modified."""
    p = np.asarray(param, np.float64)
    g = np.asarray(grad, np.float64)
    m = beta1 * np.asarray(m, np.float64) + (1.0 - beta1) * g
    v = beta2 * np.asarray(v, np.float64) + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


# --------------------------------------------------------------------------
# image fitting (Sec. 4.1): a camera looking down +z, splats turning about
# the view axis only, MSE loss; FP64 numpy
# --------------------------------------------------------------------------

def fit_params(raw: dict) -> dict:
    """Activated splat parameters of raw image-fitting parameters:
    q = (cos(theta/2), 0, 0, sin(theta/2)) (a turn by theta about z),
    p = (x, y, z), s = exp(log_s), o = 1 / (1 + exp(-logit))."""
    th = _f64(raw["theta"])
    K = th.shape[0]
    q = np.zeros((K, 4))
    q[:, 0] = np.cos(th / 2)
    q[:, 3] = np.sin(th / 2)
    means = np.concatenate([_f64(raw["xy"]), _f64(raw["z"])[:, None]], axis=1)
    return {"quats": q, "means": means, "scales": np.exp(_f64(raw["log_scales"])),
            "opacities": 1.0 / (1.0 + np.exp(-_f64(raw["logit_opacities"])))}


def fit_params_backward(raw: dict, g: dict) -> dict:
    """Chain rule through fit_params (the depth z is held fixed)."""
    th = _f64(raw["theta"])
    dq = _f64(g["quats"])
    o = 1.0 / (1.0 + np.exp(-_f64(raw["logit_opacities"])))
    return {"theta": 0.5 * (np.cos(th / 2) * dq[:, 3] - np.sin(th / 2) * dq[:, 0]),
            "xy": _f64(g["means"])[:, :2].copy(),
            "log_scales": _f64(g["scales"]) * np.exp(_f64(raw["log_scales"])),
            "logit_opacities": _f64(g["opacities"]) * o * (1.0 - o)}


def mse_loss(rgb, target):
    """Mean squared error over all values and its gradient 2 (rgb - target) / n."""
    r = _f64(rgb) - _f64(target)
    return float(np.mean(r * r)), 2.0 * r / r.size


def fit_scene(raw: dict, sh_degree: int = 0) -> dict:
    """The renderer's scene for raw image-fitting parameters (FP64 activation
    of the stored raw values)."""
    sc = fit_params(raw)
    sc.update({"sh": raw["sh"], "textures": raw["textures"], "sh_degree": int(sh_degree),
               "tex_n": int(raw["tex_n"]), "sigma": float(raw.get("sigma", 0.5))})
    return sc


def fit_step(raw: dict, target, cam: dict, mask=None) -> dict:
    """One image-fitting evaluation: render, MSE against ``target`` and the
    gradients of the raw parameters (and of sh, textures).  ``mask``
    (optional [H,W]) multiplies the loss gradient per pixel (test use: zero
    at pixels whose decisions sit within the margin)."""
    sc = fit_scene(raw)
    ref = render(sc, cam)
    loss, d = mse_loss(ref["rgb"], target)
    if mask is not None:
        d = d * mask[..., None]
    g = backward(sc, cam, d)
    out = fit_params_backward(raw, g)
    out.update({"sh": g["sh"], "textures": g["textures"], "loss": loss, "render": ref, "d_rgb": d})
    return out
