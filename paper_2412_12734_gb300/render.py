"""PyTorch front end of the GB300 textured 2D-Gaussian rasterizer.

``Rasterizer`` owns a C-ABI context and converts torch CUDA tensors and camera
dicts into the structs of include/gbill.h; ``render`` is the differentiable
``torch.autograd.Function`` whose backward recomputes per-pixel
transmittance from the saved final T and last-contributor index (no per-splat
alphas are stored).  PyTorch provides device memory and streams only; every
step of the forward and backward runs in ``libgbill.so``.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

DTYPES = {torch.float32: L.GB_F32, torch.float16: L.GB_F16, torch.bfloat16: L.GB_BF16}
STORAGE = {"f32": torch.float32, "f16": torch.float16, "bf16": torch.bfloat16}
PARAMS = ("means", "quats", "scales", "opacities", "sh", "textures")


def camera_struct(cam: dict, scene: int = 0) -> L.gb_camera:
    c = L.gb_camera()
    c.width, c.height = int(cam["width"]), int(cam["height"])
    c.fx, c.fy, c.cx, c.cy = (float(cam[k]) for k in ("fx", "fy", "cx", "cy"))
    R = np.asarray(cam["R"], np.float32)
    t = np.asarray(cam["t"], np.float32)
    w2c = np.concatenate([R, t[:, None]], axis=1).reshape(-1)
    for i in range(12):
        c.world_to_cam[i] = float(w2c[i])
    c.near_plane = float(cam.get("near", 0.01))
    c.scene = int(scene)
    return c


def scene_to_device(scene: dict, device="cuda") -> dict:
    """Copies a generator scene (numpy) to torch tensors in its storage types."""
    out = {}
    for k in ("means", "quats", "scales", "opacities"):
        out[k] = torch.as_tensor(np.ascontiguousarray(scene[k]), dtype=torch.float32, device=device)
    out["sh"] = torch.as_tensor(scene["sh"], device=device).to(STORAGE[scene.get("sh_dtype", "f32")]).contiguous()
    out["textures"] = torch.as_tensor(scene["textures"], device=device).to(
        STORAGE[scene.get("tex_dtype", "f32")]).contiguous()
    out["sh_degree"] = int(scene["sh_degree"])
    out["tex_n"] = int(scene["tex_n"])
    out["sigma"] = float(scene.get("sigma", 0.5))
    out["mip_level"] = int(scene.get("mip_level", 0))
    out["tex_sh_degree"] = int(scene.get("tex_sh_degree", 0))
    if scene.get("splat_tex_n") is not None:
        out["splat_tex_n"] = torch.as_tensor(np.asarray(scene["splat_tex_n"]).astype(np.uint8), device=device)
    return out


def _check_tensor(t: torch.Tensor, name: str, shape_tail, dtypes=(torch.float32,)):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype not in dtypes:
        raise ValueError(f"{name}: dtype {t.dtype} not in {dtypes}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if tuple(t.shape[1:]) != tuple(shape_tail):
        raise ValueError(f"{name}: shape {tuple(t.shape)} does not end in {shape_tail}")


def _check_buffer(t: torch.Tensor, name: str, numel: int):
    """A buffer the library reads or writes through a plain pointer (an
    output, an upstream gradient or a gradient output): CUDA, float32,
    contiguous and exactly ``numel`` elements, which the C ABI cannot check."""
    if not isinstance(t, torch.Tensor) or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor")
    if t.numel() != numel:
        raise ValueError(f"{name}: {t.numel()} elements, expected {numel}")
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")


def grad_shapes(K: int, D: int, N: int, Mt: int) -> dict:
    """Shape of each gradient output of a scene of K splats, SH degree D,
    N x N grids and Mt SH coefficients per texel (0: RGB texels)."""
    return {"means": (K, 3), "quats": (K, 4), "scales": (K, 2), "opacities": (K,), "sh": (K, (D + 1) ** 2, 3),
            "textures": (K, N, N, 3) if Mt == 0 else (K, N, N, Mt, 3)}


def scene_struct(sc: dict) -> L.gb_scene:
    K = int(sc["means"].shape[0])
    D, N = int(sc["sh_degree"]), int(sc["tex_n"])
    _check_tensor(sc["means"], "means", (3,))
    _check_tensor(sc["quats"], "quats", (4,))
    _check_tensor(sc["scales"], "scales", (2,))
    _check_tensor(sc["opacities"], "opacities", ())
    _check_tensor(sc["sh"], "sh", ((D + 1) ** 2, 3), tuple(DTYPES))
    Dt = int(sc.get("tex_sh_degree", 0))
    _check_tensor(sc["textures"], "textures", (N, N, 3) if Dt == 0 else (N, N, (Dt + 1) ** 2, 3), tuple(DTYPES))
    for k in PARAMS:
        if sc[k].shape[0] != K:
            raise ValueError(f"{k}: first dimension {sc[k].shape[0]} != {K}")
    s = L.gb_scene()
    s.num_splats = K
    s.means, s.quats, s.scales = sc["means"].data_ptr(), sc["quats"].data_ptr(), sc["scales"].data_ptr()
    s.opacities, s.sh, s.textures = sc["opacities"].data_ptr(), sc["sh"].data_ptr(), sc["textures"].data_ptr()
    s.sh_degree, s.sh_dtype = D, DTYPES[sc["sh"].dtype]
    s.tex_n, s.tex_dtype = N, DTYPES[sc["textures"].dtype]
    s.sigma = float(sc.get("sigma", 0.5))
    s.mip_level = int(sc.get("mip_level", 0))
    s.tex_sh_degree = Dt
    s.reserved = 0
    sn = sc.get("splat_tex_n")
    if sn is not None:
        _check_tensor(sn, "splat_tex_n", (), (torch.uint8,))
        if sn.shape[0] != K:
            raise ValueError(f"splat_tex_n: first dimension {sn.shape[0]} != {K}")
        s.splat_tex_n = sn.data_ptr()
    return s


class Saved:
    """Owns one gb_saved handle (state kept between a forward and its backward)."""

    def __init__(self, rast: "Rasterizer"):
        self.rast = rast
        h = C.c_void_p()
        L.check(L.load().gb_saved_create(rast.ctx, C.byref(h)), rast.ctx)
        self.handle = h
        self.n_scenes = 0
        self.shapes = []
        self.n_pix = None

    def reserve(self, records: int, instances: int, pixels: int, tiles: int):
        L.check(L.load().gb_saved_reserve(self.handle, records, instances, pixels, tiles), self.rast.ctx)

    def stats(self) -> dict:
        st = L.gb_stats()
        L.check(L.load().gb_saved_stats(self.handle, C.byref(st)), self.rast.ctx)
        return {f: getattr(st, f) for f, _ in L.gb_stats._fields_}

    def check(self):
        L.check(L.load().gb_saved_check(self.handle), self.rast.ctx)

    def phase_times(self) -> dict:
        """Milliseconds per phase of the last forward/backward run with GB_FLAG_TIMING."""
        arr = (C.c_float * len(L.PHASES))()
        L.check(L.load().gb_saved_phase_times(self.handle, arr, len(L.PHASES)), self.rast.ctx)
        return dict(zip(L.PHASES, (float(x) for x in arr)))

    def export_records(self, lo: bool = False):
        """(records [R,16] float32, visible [R] bool) of the last forward, and
        with ``lo`` the low parts [R,12] of the flagged records as a third item."""
        n = C.c_int64()
        L.check(L.load().gb_saved_export_records(self.handle, None, None, None, 0, C.byref(n)), self.rast.ctx)
        rec = np.zeros((n.value, 16), np.float32)
        rlo = np.zeros((n.value, 12), np.float32)
        vis = np.zeros(n.value, np.uint8)
        if n.value:
            L.check(L.load().gb_saved_export_records(self.handle, rec.ctypes.data, rlo.ctypes.data, vis.ctypes.data,
                                                     n.value, C.byref(n)), self.rast.ctx)
        return (rec, vis.astype(bool), rlo) if lo else (rec, vis.astype(bool))

    def export_keys(self):
        """Sorted (key, splat id, camera) instance list of the last forward."""
        n = C.c_int64()
        L.check(L.load().gb_saved_export_keys(self.handle, None, None, None, 0, C.byref(n)), self.rast.ctx)
        cnt = n.value
        keys = np.zeros(cnt, np.uint64)
        ids = np.zeros(cnt, np.int64)
        cams = np.zeros(cnt, np.int32)
        if cnt:
            L.check(L.load().gb_saved_export_keys(self.handle, keys.ctypes.data, ids.ctypes.data,
                                                  cams.ctypes.data, cnt, C.byref(n)), self.rast.ctx)
        return keys, ids, cams

    def __del__(self):
        try:
            if self.handle:
                L.load().gb_saved_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


class Rasterizer:
    """A C-ABI context on one CUDA device."""

    def __init__(self, device: int | None = None):
        lib = L.load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = C.c_void_p()
        st = lib.gb_context_create(self.device, C.byref(h))
        if st != L.GB_OK:
            raise L.GbillError(st, f"cannot create a context on CUDA device {self.device}")
        self.ctx = h

    def __del__(self):
        try:
            if self.ctx:
                L.load().gb_context_destroy(self.ctx)
                self.ctx = None
        except Exception:
            pass

    @staticmethod
    def pixel_count(cams) -> int:
        return sum(int(c["width"]) * int(c["height"]) for c in cams)

    def forward(self, scenes: list, cams: list, cam_scene=None, saved: Saved | None = None,
                tile: int = 16, batch: int = 0, flags: int = 0, background=None, stream=None,
                out=None, ppt: int = 0, batch_fwd: int = 0, bwd_kernel: int = 0):
        """Renders every camera; returns (rgb [P,3], depth [P], alpha [P], saved).

        batch is the backward's batch depth (and the forward's unless
        batch_fwd is given); 0 picks each pass's automatic depth."""
        lib = L.load()
        n_s, n_c = len(scenes), len(cams)
        cam_scene = list(cam_scene) if cam_scene is not None else [0] * n_c
        sarr = (L.gb_scene * n_s)(*[scene_struct(s) for s in scenes])
        carr = (L.gb_camera * n_c)(*[camera_struct(c, cam_scene[i]) for i, c in enumerate(cams)])
        opt = L.gb_options()
        opt.tile_size, opt.batch_depth, opt.flags, opt.pixels_per_thread = tile, batch, flags, ppt
        opt.batch_depth_fwd = batch_fwd
        opt.bwd_kernel = bwd_kernel
        if background is not None:
            for i in range(3):
                opt.background[i] = float(background[i])
        P = self.pixel_count(cams)
        dev = scenes[0]["means"].device
        if out is None:
            rgb = torch.empty((P, 3), device=dev)
            depth = torch.empty(P, device=dev)
            alpha = torch.empty(P, device=dev)
        else:
            rgb, depth, alpha = out
            _check_buffer(rgb, "rgb", 3 * P)
            if depth is not None:
                _check_buffer(depth, "depth", P)
            if alpha is not None:
                _check_buffer(alpha, "alpha", P)
        if saved is None:
            saved = Saved(self)
        saved.n_pix = P
        saved.n_scenes = n_s
        saved.shapes = [(int(s["means"].shape[0]), int(s["sh_degree"]), int(s["tex_n"]),
                         (int(s.get("tex_sh_degree", 0)) + 1) ** 2 if int(s.get("tex_sh_degree", 0)) else 0)
                        for s in scenes]
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        st = lib.gb_render_forward(self.ctx, saved.handle, sarr, n_s, carr, n_c, C.byref(opt),
                                   rgb.data_ptr(), depth.data_ptr() if depth is not None else None,
                                   alpha.data_ptr() if alpha is not None else None, C.c_void_p(s.cuda_stream))
        L.check(st, self.ctx)
        return rgb, depth, alpha, saved

    def backward(self, saved: Saved, d_rgb: torch.Tensor, d_depth=None, d_alpha=None, grads=None,
                 stream=None):
        """Gradients of every scene (list of dicts), summed over its cameras."""
        lib = L.load()
        dev = d_rgb.device
        if grads is None:
            grads = [{k: torch.empty(shape, device=dev) for k, shape in grad_shapes(*sh).items()}
                     for sh in saved.shapes]
        if len(grads) != saved.n_scenes:
            raise ValueError(f"grads: {len(grads)} entries for {saved.n_scenes} scenes")
        garr = (L.gb_grads * len(grads))()
        for i, g in enumerate(grads):
            want = grad_shapes(*saved.shapes[i])
            for k in PARAMS:
                t = g.get(k)
                if t is not None:
                    _check_buffer(t, f"grads[{i}][{k!r}]", int(np.prod(want[k])))
                setattr(garr[i], "d_" + k, t.data_ptr() if t is not None else None)
        n_pix = saved.n_pix
        for t, name, m in ((d_rgb, "d_rgb", 3), (d_depth, "d_depth", 1), (d_alpha, "d_alpha", 1)):
            if t is not None:
                if n_pix is not None:
                    _check_buffer(t, name, m * n_pix)
                elif not t.is_contiguous() or t.dtype != torch.float32:
                    raise ValueError(f"{name} must be contiguous float32")
        s = stream if stream is not None else torch.cuda.current_stream(dev)
        st = lib.gb_render_backward(self.ctx, saved.handle, d_rgb.data_ptr(),
                                    d_depth.data_ptr() if d_depth is not None else None,
                                    d_alpha.data_ptr() if d_alpha is not None else None,
                                    garr, len(grads), C.c_void_p(s.cuda_stream))
        L.check(st, self.ctx)
        return grads


    def autotune(self, scenes: list, cams: list, cam_scene=None, reps: int = 3, saved: Saved | None = None,
                 cache: str | None = None) -> dict:
        """Picks (tile, batch_depth, pixels per thread) with the library's
        autotuner; results are cached in a JSON file keyed by every scene's
        grid size, mip level, per-texel SH degree, storage types and SH
        degree, the splat count and pixel count (rounded to powers of two)
        and the number of cameras."""
        import json
        import os
        key = "|".join(str(x) for x in (
            [(int(s["tex_n"]), int(s.get("mip_level", 0)), int(s.get("tex_sh_degree", 0)), str(s["textures"].dtype),
              str(s["sh"].dtype), int(s["sh_degree"])) for s in scenes],
            sum(int(s["means"].shape[0]) for s in scenes).bit_length(),
            self.pixel_count(cams).bit_length(), len(cams)))
        path = cache or os.path.join(os.path.expanduser("~"), ".cache", "gbill", "autotune.json")
        table = {}
        if os.path.exists(path):
            try:
                table = json.load(open(path))
            except (OSError, ValueError):
                table = {}
        if key in table:
            return table[key]
        lib = L.load()
        n_s, n_c = len(scenes), len(cams)
        cam_scene = list(cam_scene) if cam_scene is not None else [0] * n_c
        sarr = (L.gb_scene * n_s)(*[scene_struct(s) for s in scenes])
        carr = (L.gb_camera * n_c)(*[camera_struct(c, cam_scene[i]) for i, c in enumerate(cams)])
        best = L.gb_options()
        ms = (C.c_float * 128)()
        tiles = (C.c_int32 * 128)()
        batches = (C.c_int32 * 128)()
        ppts = (C.c_int32 * 128)()
        n = C.c_int32()
        saved = saved or Saved(self)
        L.check(lib.gb_autotune(self.ctx, saved.handle, sarr, n_s, carr, n_c, None, reps, C.byref(best),
                                C.addressof(ms), C.addressof(tiles), C.addressof(batches), C.addressof(ppts), 128,
                                C.byref(n)), self.ctx)
        # candidates with ppt 0 time the forward alone at batch depth "batch"; ppt 3
        # marks the splat-parallel backward
        res = {"tile": best.tile_size, "batch": best.batch_depth, "ppt": best.pixels_per_thread,
               "batch_fwd": best.batch_depth_fwd, "bwd_kernel": best.bwd_kernel,
               "candidates": [{"tile": tiles[i], "batch": batches[i], "ppt": ppts[i], "ms": ms[i]}
                              for i in range(min(n.value, 128))]}
        table[key] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            json.dump(table, open(path, "w"), indent=1)
        except OSError:
            pass
        return res


_default = {}


def default_rasterizer() -> Rasterizer:
    dev = torch.cuda.current_device()
    if dev not in _default:
        _default[dev] = Rasterizer(dev)
    return _default[dev]


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacities, sh, textures, meta):
        rast, cams, sh_degree, tex_n, sigma, background, mip_level, tex_sh_degree = meta
        sc = {"means": means.contiguous(), "quats": quats.contiguous(), "scales": scales.contiguous(),
              "opacities": opacities.contiguous(), "sh": sh.contiguous(), "textures": textures.contiguous(),
              "sh_degree": sh_degree, "tex_n": tex_n, "sigma": sigma, "mip_level": mip_level,
              "tex_sh_degree": tex_sh_degree}
        rgb, depth, alpha, saved = rast.forward([sc], cams, background=background)
        ctx.saved_handle = saved
        ctx.rast = rast
        ctx.keep = sc  # parameters must stay alive and unchanged until backward
        ctx.dtypes = (sh.dtype, textures.dtype)
        ctx.n_pix = rgb.shape[0]
        return rgb, depth, alpha

    @staticmethod
    def backward(ctx, d_rgb, d_depth, d_alpha):
        d_rgb = d_rgb.contiguous().float() if d_rgb is not None else None
        if d_rgb is None:  # only without materialised gradients: the library needs [P, 3]
            d_rgb = torch.zeros((ctx.n_pix, 3), device=ctx.keep["means"].device)
        d_depth = d_depth.contiguous().float() if d_depth is not None else None
        d_alpha = d_alpha.contiguous().float() if d_alpha is not None else None
        g = ctx.rast.backward(ctx.saved_handle, d_rgb, d_depth, d_alpha)[0]
        return (g["means"], g["quats"], g["scales"], g["opacities"], g["sh"].to(ctx.dtypes[0]),
                g["textures"].to(ctx.dtypes[1]), None)


def render(means, quats, scales, opacities, sh, textures, cams, sh_degree: int, tex_n: int,
           sigma: float = 0.5, background=None, rasterizer: Rasterizer | None = None, mip_level: int = 0,
           tex_sh_degree: int = 0):
    """Differentiable render of one scene into all ``cams``.

    Returns (rgb [P,3], depth [P], alpha [P]) with the cameras' pixels packed
    one after another (row-major per camera).  mip_level l > 0 renders the
    colour grids box-filtered to N / 2^l (Sec. 4.1, Fig. 4 f, g);
    tex_sh_degree Dt > 0 takes textures [K, N, N, (Dt+1)^2, 3] of per-texel SH
    coefficients (Sec. 4.2).
    """
    rast = rasterizer or default_rasterizer()
    meta = (rast, list(cams), int(sh_degree), int(tex_n), float(sigma), background, int(mip_level),
            int(tex_sh_degree))
    return _RenderFn.apply(means, quats, scales, opacities, sh, textures, meta)


def _adam_tensors(params: list, grads: list, ms: list, vs: list, shadows=None):
    n = len(params)
    arr = (L.gb_adam_tensor * n)()
    for i in range(n):
        p, g, m, v = params[i], grads[i], ms[i], vs[i]
        for t in (p, g, m, v):
            if t.dtype != torch.float32 or not t.is_contiguous() or t.numel() != p.numel():
                raise ValueError("adam tensors must be contiguous float32 of equal size")
        arr[i].param, arr[i].grad, arr[i].m, arr[i].v = p.data_ptr(), g.data_ptr(), m.data_ptr(), v.data_ptr()
        sh = shadows[i] if shadows is not None else None
        arr[i].shadow = sh.data_ptr() if sh is not None else None
        arr[i].shadow_dtype = DTYPES[sh.dtype] if sh is not None else 0
        arr[i].reserved = 0
        arr[i].n = p.numel()
    return arr, n


def adam_step(rast: Rasterizer, params: list, grads: list, ms: list, vs: list, step: int, lr: float = 1e-3,
              betas=(0.9, 0.999), eps: float = 1e-15, shadows=None, stream=None):
    """Fused Adam over up to 16 FP32 tensors in one launch (gb_adam_step).

    shadows[i] (optional) receives the updated params[i] in its own dtype
    (e.g. the BF16 textures the renderer reads)."""
    arr, n = _adam_tensors(params, grads, ms, vs, shadows)
    cfg = L.gb_adam_config(float(lr), float(betas[0]), float(betas[1]), float(eps), int(step), 0)
    s = stream if stream is not None else torch.cuda.current_stream()
    L.check(L.load().gb_adam_step(rast.ctx, arr, n, C.byref(cfg), C.c_void_p(s.cuda_stream)), rast.ctx)


class AdamStep:
    """gb_adam_step over a fixed set of tensors with its argument arrays built
    once, for training loops whose host time matters; the tensors must stay
    allocated (and in place) while the object is used."""

    def __init__(self, rast: Rasterizer, params: list, grads: list, ms: list, vs: list, lr: float = 1e-3,
                 betas=(0.9, 0.999), eps: float = 1e-15, shadows=None):
        self.rast = rast
        self.arr, self.n = _adam_tensors(params, grads, ms, vs, shadows)
        self.cfg = L.gb_adam_config(float(lr), float(betas[0]), float(betas[1]), float(eps), 1, 0)
        self.keep = (list(params), list(grads), list(ms), list(vs), shadows)

    def __call__(self, step: int, stream=None):
        self.cfg.step = int(step)
        s = stream if stream is not None else torch.cuda.current_stream()
        L.check(L.load().gb_adam_step(self.rast.ctx, self.arr, self.n, C.byref(self.cfg),
                                      C.c_void_p(s.cuda_stream)), self.rast.ctx)


class BatchedRenderer:
    """Forward and backward of one fixed frame (scenes, cameras, options)
    replayed from CUDA graphs.

    The constructor renders once with a host sync to size the saved state,
    reserves ``headroom`` times that instance count, allocates the outputs
    (rgb, depth, alpha), the upstream-gradient buffer ``d_rgb`` [P, 3] and
    the gradients (one dict per scene), and runs one no-sync forward and
    backward.  ``forward()`` and ``backward()`` then replay a graph each
    (captured on first use).  The scenes' tensors are read where they are:
    parameters updated in place between steps (an optimiser step) are
    rendered by the next replay, whatever their visible set and instance
    count.  A replay never waits for the host and never allocates; ``check()``
    reports an instance list that outgrew the reservation and
    ``ensure_capacity()`` grows it and captures again.  With
    ``flags=GB_FLAG_PERSISTENT`` the views and scenes of each render group
    (grid size and storage type) share one persistent launch per pass, whose
    blocks take tiles from a device counter, longest tiles first.
    """

    def __init__(self, rast: Rasterizer, scenes: list, cams: list, cam_scene=None, tile: int = 16,
                 batch: int = 0, batch_fwd: int = 0, ppt: int = 0, flags: int = 0, background=None,
                 headroom: float = 1.25, bwd_kernel: int = 0):
        self.rast = rast
        self.scenes, self.cams = list(scenes), list(cams)
        self.cam_scene = list(cam_scene) if cam_scene is not None else [0] * len(self.cams)
        self.opts = {"tile": tile, "batch": batch, "batch_fwd": batch_fwd, "ppt": ppt, "background": background,
                     "bwd_kernel": bwd_kernel}
        self.flags = int(flags) & ~(L.GB_FLAG_NO_SYNC | L.GB_FLAG_TIMING)
        self.P = rast.pixel_count(self.cams)
        self.saved = Saved(rast)
        rgb, depth, alpha, _ = rast.forward(self.scenes, self.cams, cam_scene=self.cam_scene, saved=self.saved,
                                            flags=self.flags, **self.opts)
        self.out = (rgb, depth, alpha)
        st = self.saved.stats()
        self.saved.reserve(st["records"], int(st["instances"] * headroom) + 4096, self.P, st["tiles"])
        self.d_rgb = torch.zeros((self.P, 3), device=rgb.device)
        self.grads = rast.backward(self.saved, self.d_rgb)
        self._graphs = None
        self._forward()
        self._backward()
        torch.cuda.synchronize(rgb.device)
        self.saved.check()

    def _forward(self):
        self.rast.forward(self.scenes, self.cams, cam_scene=self.cam_scene, saved=self.saved, out=self.out,
                          flags=self.flags | L.GB_FLAG_NO_SYNC, **self.opts)

    def _backward(self):
        self.rast.backward(self.saved, self.d_rgb, grads=self.grads)

    def capture(self):
        """Records the forward and the backward as one graph each."""
        graphs = []
        for run in (self._forward, self._backward):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                run()
            graphs.append(g)
        self._graphs = graphs

    def forward(self):
        """Renders every camera into self.out = (rgb [P,3], depth [P], alpha [P])."""
        if self._graphs is None:
            self.capture()
        self._graphs[0].replay()
        return self.out

    def backward(self, d_rgb: torch.Tensor | None = None):
        """Gradients of the last forward's splats from dL/drgb: ``d_rgb`` (a
        [P, 3] float32 device tensor) is copied into self.d_rgb first; without
        it self.d_rgb is used as it stands (write it in place).  Returns the
        gradient dicts (overwritten by every call)."""
        if d_rgb is not None:
            self.d_rgb.copy_(d_rgb.reshape(self.P, 3))
        if self._graphs is None:
            self.capture()
        self._graphs[1].replay()
        return self.grads

    def check(self):
        """Raises if a replayed forward outgrew the reservation (synchronizes)."""
        self.saved.check()

    def ensure_capacity(self, headroom: float = 0.7):
        """Checks the last forward and doubles the instance capacity once it is
        more than ``headroom`` full; the graphs are captured again on next use
        (the saved state's buffers moved).  Synchronizes."""
        self.check()
        st = self.saved.stats()
        if st["instances"] > headroom * st["capacity"]:
            self.saved.reserve(st["records"], 2 * st["capacity"], self.P, st["tiles"])
            self._graphs = None
