"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Nothing here compares the oracle with itself: every expected value is a closed
form, a library routine (scipy's spherical harmonics), a brute-force identity
or a statement printed in the paper (tests/golden/).  Sections: Sec. 3.1 Eq. 2-4,
Sec. 3.2 Eq. 5 and Fig. 2, Sec. 4.2 (SH colour), Alg. 1, Alg. 2.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2412_12734_gb300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- SH basis --

def _real_sh_scipy(l, m, dirs):
    """Real SH from scipy's complex Y_l^m (Condon-Shortley phase included).

    The oracle's basis is sqrt(2) Re Y_l^m (m > 0), Y_l^0, sqrt(2) Im Y_l^|m|
    (m < 0): the usual real basis times (-1)^m.
    """
    from scipy.special import sph_harm_y
    x, y, z = dirs.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    Y = sph_harm_y(l, abs(m), theta, phi)
    if m > 0:
        return math.sqrt(2) * Y.real
    if m < 0:
        return math.sqrt(2) * Y.imag
    return Y.real


def test_sh_basis_matches_scipy():
    rng = np.random.default_rng(1)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y, _ = oracle.sh_basis(3, d)
    i = 0
    for l in range(4):
        for m in range(-l, l + 1):
            np.testing.assert_allclose(Y[:, i], _real_sh_scipy(l, m, d), atol=1e-13, rtol=0)
            i += 1


def test_sh_gradient_finite_difference():
    rng = np.random.default_rng(2)
    d = rng.standard_normal((20, 3))
    _, dY = oracle.sh_basis(3, d)
    h = 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        Yp, _ = oracle.sh_basis(3, d + e)
        Ym, _ = oracle.sh_basis(3, d - e)
        np.testing.assert_allclose(dY[:, :, j], (Yp - Ym) / (2 * h), atol=1e-7)


# ---------------------------------------------------------------- bilinear --

@pytest.mark.parametrize("N", [2, 4, 8, 16])
@pytest.mark.parametrize("sigma", [0.5, 2.0])
def test_bilinear_reproduces_texels(N, sigma):
    """Corner-aligned grid: texel (i, j) sits at u = -sigma + 2 sigma i / (N-1)."""
    rng = np.random.default_rng(N)
    grid = rng.uniform(0, 1, (N, N, 3))
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    u = -sigma + 2 * sigma * ii / (N - 1)
    v = -sigma + 2 * sigma * jj / (N - 1)
    out = oracle.bilinear(np.stack([u.ravel(), v.ravel()], 1), N, sigma, grid)
    np.testing.assert_allclose(out, grid.reshape(-1, 3), atol=1e-14)


@pytest.mark.parametrize("N", [2, 3, 4, 8, 16])
def test_bilinear_affine_grid_is_exact_and_oriented(N):
    """Grid C[i_u][i_v] = a i_u + b i_v + c interpolates to a u' + b v' + c.

    a != b, so a transposed index order fails.  Outside [-sigma, sigma] the
    lookup is border clamped (Fig. 2 text, Alg. 2 clamp).
    """
    sigma = 0.5
    a, b, c = np.array([0.25, -0.125, 0.0625]), np.array([-0.125, 0.375, 0.1875]), np.array([0.125, 0.25, 0.3125])
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    grid = ii[..., None] * a + jj[..., None] * b + c
    rng = np.random.default_rng(0)
    uv = rng.uniform(-1.5 * sigma, 1.5 * sigma, (500, 2))
    out = oracle.bilinear(uv, N, sigma, grid)
    up = np.clip((N - 1) * (uv[:, 0] + sigma) / (2 * sigma), 0, N - 1)
    vp = np.clip((N - 1) * (uv[:, 1] + sigma) / (2 * sigma), 0, N - 1)
    np.testing.assert_allclose(out, up[:, None] * a + vp[:, None] * b + c, atol=1e-13)


def test_bilinear_partition_of_unity_and_n1():
    rng = np.random.default_rng(3)
    uv = rng.uniform(-1, 1, (300, 2))
    for N in (2, 4, 8):
        out = oracle.bilinear(uv, N, 0.5, np.ones((N, N, 3)))
        np.testing.assert_allclose(out, 1.0, atol=1e-14)
    col = np.array([0.25, 0.5, 0.75])
    out = oracle.bilinear(uv, 1, 0.5, col.reshape(1, 1, 3))
    assert np.all(out == col)


@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_adj_bilinear_matches_finite_differences(N):
    """Alg. 2 adj-bilinear: grid adjoint = interpolation weights, uv adjoint =
    derivative of the interpolant inside (-sigma, sigma), zero outside."""
    sigma = 0.5
    rng = np.random.default_rng(10 + N)
    grid = rng.uniform(0, 1, (N, N, 3))
    uv = rng.uniform(-0.8, 0.8, (200, 2))
    k = (N - 1) / (2 * sigma)
    # keep away from cell boundaries and from the clamp border
    cell = lambda t: (N - 1) * (t + sigma) / (2 * sigma)
    ok = np.ones(len(uv), bool)
    for j in range(2):
        cp = cell(uv[:, j])
        ok &= np.abs(cp - np.round(cp)) > 1e-4
        ok &= np.abs(np.abs(uv[:, j]) - sigma) > 1e-4
    uv = uv[ok]
    chat = rng.standard_normal((len(uv), 3))
    Chat, uvh = oracle.adj_bilinear(uv, N, sigma, grid, chat)
    h = 1e-6
    for j in range(2):
        e = np.zeros(2)
        e[j] = h
        fp = oracle.bilinear(uv + e, N, sigma, grid)
        fm = oracle.bilinear(uv - e, N, sigma, grid)
        fd = ((fp - fm) / (2 * h) * chat).sum(1)
        np.testing.assert_allclose(uvh[:, j], fd, atol=1e-7)
        inside = np.abs(uv[:, j]) < sigma
        assert np.all(uvh[~inside, j] == 0)
        assert np.any(uvh[inside, j] != 0)
    # grid adjoint: d(sum chat . bilinear)/dC by linearity = weights
    Chat_fd = np.zeros_like(grid)
    for idx in np.ndindex(N, N, 3):
        g2 = grid.copy()
        g2[idx] += 1.0
        Chat_fd[idx] = ((oracle.bilinear(uv, N, sigma, g2) - oracle.bilinear(uv, N, sigma, grid)) * chat).sum()
    np.testing.assert_allclose(Chat, Chat_fd, atol=1e-11)
    assert k > 0


def test_fig2_isoline_facts():
    """Fig. 2 / Sec. 3.2: sigma = 0.5 puts the grid border near the 0.8 isoline,
    sigma = 2 near the 0.1 isoline.  Checked on the oracle's alpha of a
    fronto-parallel splat of opacity 0.98 at pixels with u = sigma, v = 0 and
    at the grid corner u = v = sigma."""
    rows = [l.split() for l in open(os.path.join(GOLDEN, "fig2_isolines.txt"))
            if l.strip() and not l.startswith("#")]
    for sig, iso in ((float(a), float(b)) for a, b in rows):
        sc, cam = _fronto_scene(s=(1.0, 1.0), o=0.98, z=4.0, sigma=sig)
        f = float(cam["fx"])
        cx = float(cam["cx"]) + 0.5
        cy = float(cam["cy"]) + 0.5
        # centre at (cx, cy); u = (x - cx) d / (f s)  (camera axes = world axes here)
        px = cx + sig * f / 4.0
        py = cy + sig * f / 4.0
        r = oracle.eval_pairs(sc, cam, 0, [[px, cy], [px, py]])
        np.testing.assert_allclose(r["u"], [sig, sig], rtol=1e-8)  # FP32-rounded centre
        G_axis, G_corner = r["alpha"] / 0.98
        assert G_axis >= iso >= G_corner


# --------------------------------------------------------- closed-form scenes --

def _identity_camera(W=64, H=48, f=64.0):
    """Camera at the origin looking down +z with camera axes = world axes."""
    return {"width": W, "height": H, "fx": np.float32(f), "fy": np.float32(f),
            "cx": np.float32(W / 2), "cy": np.float32(H / 2),
            "R": np.eye(3, dtype=np.float32), "t": np.zeros(3, np.float32), "near": np.float32(0.01)}


def _fronto_scene(s=(0.5, 0.5), o=0.7, z=4.0, N=4, grid=None, colour=(0.1, 0.2, 0.3), sigma=0.5,
                  offset_px=(0.5, 0.5), f=64.0, W=64, H=48):
    """One splat parallel to the image plane whose centre projects onto the
    pixel centre (W/2 + offset, H/2 + offset); t_u = +x, t_v = +y."""
    cam = _identity_camera(W, H, f)
    px = offset_px[0] * z / f
    py = offset_px[1] * z / f
    if grid is None:
        grid = np.random.default_rng(5).uniform(0, 1, (N, N, 3))
    sc = {
        "means": np.array([[px, py, z]], np.float32),
        "quats": np.array([[1, 0, 0, 0]], np.float32),
        "scales": np.array([s], np.float32),
        "opacities": np.array([o], np.float32),
        "sh": (np.array(colour, np.float32) * 2 * math.sqrt(math.pi)).reshape(1, 1, 3),
        "textures": np.asarray(grid, np.float32).reshape(1, N, N, 3),
        "sh_degree": 0, "tex_n": N, "sigma": sigma, "sh_dtype": "f32", "tex_dtype": "f32",
    }
    return sc, cam


@pytest.mark.parametrize("N", [1, 2, 4, 8, 16])
@pytest.mark.parametrize("o", [0.01, 0.6, 0.995])
def test_single_splat_at_pixel_centre(N, o):
    """u = v = 0 at the centre pixel: alpha = min(0.99, o) (Eq. 4, alpha clamp)
    and colour = bilinear(C, 0, 0) + SH colour (Eq. 5, Sec. 4.2).  For even N
    bilinear(C, 0, 0) is the mean of the four central texels."""
    grid = np.random.default_rng(N).uniform(0, 1, (N, N, 3)).astype(np.float32).astype(np.float64)
    colour = np.array([0.1, 0.2, 0.3], np.float32).astype(np.float64)
    sc, cam = _fronto_scene(o=o, N=N, grid=grid, colour=colour)
    sc["sh"] = sc["sh"].astype(np.float32)
    Y00 = 0.5 / math.sqrt(math.pi)
    col = sc["sh"][0, 0].astype(np.float64) * Y00
    if N == 1:
        centre = grid[0, 0]
    elif N % 2 == 0:
        c = N // 2
        centre = grid[c - 1:c + 1, c - 1:c + 1].mean(axis=(0, 1))
    else:
        centre = grid[N // 2, N // 2]
    r = oracle.render(sc, cam)
    x, y = 32, 24
    alpha = min(0.99, float(np.float32(o)))
    np.testing.assert_allclose(r["alpha"][y, x], alpha, rtol=1e-12)
    np.testing.assert_allclose(r["rgb"][y, x], alpha * (centre + col), rtol=1e-12)
    np.testing.assert_allclose(r["depth"][y, x], alpha * 4.0, rtol=1e-6)


def test_faint_splat_below_the_alpha_cutoff_is_culled():
    """o = 0.003 < 1/255: alpha <= o < 1/255 everywhere, so the splat is culled
    (R14) and draws nothing, even at its centre; o = 0.004 >= 1/255 draws
    alpha = o there."""
    sc, cam = _fronto_scene(o=0.003)
    assert not oracle.keys32(sc, cam)[0][0]
    r = oracle.render(sc, cam)
    assert np.all(r["alpha"] == 0.0) and np.all(r["rgb"] == 0.0)
    sc, cam = _fronto_scene(o=0.004)
    assert oracle.keys32(sc, cam)[0][0]
    np.testing.assert_allclose(oracle.render(sc, cam)["alpha"][24, 32], float(np.float32(0.004)), rtol=1e-12)


def test_empty_and_behind_camera_scenes_render_the_background():
    """No splat in front of the camera (K = 0, or every centre behind it):
    every pixel keeps T = 1, so the image is the background (Alg. 1 with an
    empty list), alpha and depth are zero, and every gradient is zero."""
    cam = scenes.tiny_camera(24, 16)
    bg = np.array([0.2, 0.5, 0.7])
    empty = scenes.subset(scenes.tiny_scene(1, K=3), np.arange(0))
    behind = scenes.tiny_scene(2, K=4)
    behind["means"][:, 2] = -6.0  # the camera sits at z = -4 looking along +z
    rng = np.random.default_rng(3)
    for sc in (empty, behind):
        r = oracle.render(sc, cam, bg=bg)
        assert np.array_equal(r["rgb"], np.broadcast_to(bg, r["rgb"].shape))
        assert np.all(r["alpha"] == 0.0) and np.all(r["depth"] == 0.0)
        assert np.all(r["t_final"] == 1.0) and np.all(r["n_contrib"] == 0)
        g = oracle.backward(sc, cam, rng.standard_normal((16, 24, 3)), bg=bg)
        for k, v in g.items():
            assert v.shape[0] == sc["means"].shape[0] and np.all(v == 0.0), k


def test_fronto_parallel_uv_and_colour_closed_form():
    """Fronto-parallel splat: u = (x_c - c_x) d / (f s_u), v likewise; alpha =
    o exp(-(u^2+v^2)/2) on the uv branch; colour from an affine grid."""
    N, sigma = 4, 0.5
    a, b, c = np.array([0.25, -0.125, 0.0625]), np.array([-0.125, 0.375, 0.1875]), np.array([0.125, 0.25, 0.3125])
    ii, jj = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
    grid = ii[..., None] * a + jj[..., None] * b + c
    s, z, f, o = (0.6, 0.4), 5.0, 64.0, 0.8
    sc, cam = _fronto_scene(s=s, o=o, z=z, N=N, grid=grid, colour=(0, 0, 0), f=f)
    r = oracle.render(sc, cam)
    xs, ys = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    cxp, cyp = 32.5, 24.5
    s32 = np.asarray(s, np.float32).astype(np.float64)  # the stored scales
    u = (xs - cxp) * z / (f * s32[0])
    v = (ys - cyp) * z / (f * s32[1])
    rho_uv = u * u + v * v
    rho_lp = 2 * ((xs - cxp) ** 2 + (ys - cyp) ** 2)
    rho = np.minimum(rho_uv, rho_lp)
    alpha = np.minimum(0.99, np.float32(o) * np.exp(-rho / 2))
    up = np.clip((N - 1) * (u + sigma) / (2 * sigma), 0, N - 1)
    vp = np.clip((N - 1) * (v + sigma) / (2 * sigma), 0, N - 1)
    col = up[..., None] * a + vp[..., None] * b + c
    assert np.array_equal(np.asarray(grid, np.float32), grid)  # dyadic: exact in FP32
    expect = np.where((alpha >= 1 / 255)[..., None], alpha[..., None] * col, 0.0)
    np.testing.assert_allclose(r["rgb"], expect, atol=1e-12)
    zmap = np.where(alpha >= 1 / 255, alpha * z, 0.0)
    np.testing.assert_allclose(r["depth"], zmap, atol=1e-9)


def test_rotated_thin_fronto_splat_closed_form():
    """A thin splat parallel to the image plane and turned by theta about the
    optical axis (the ray/plane hit of Sec. 3.1 in closed form): u = (dx cos +
    dy sin) z / (f s_u), v = (-dx sin + dy cos) z / (f s_v), alpha = min(0.99,
    o exp(-min(u^2 + v^2, 2 |d|^2) / 2)) where it reaches 1/255.  Pixels along
    the long axis, far from the centre, are where an FP32 evaluation about the
    centre loses most digits."""
    th = math.radians(30.0)
    sc, cam = _fronto_scene(s=(0.01, 0.6), o=0.8, z=5.0, N=4, sigma=1.0)
    sc["quats"] = np.array([[math.cos(th / 2), 0, 0, math.sin(th / 2)]], np.float32)
    r = oracle.render(sc, cam)
    q = sc["quats"][0].astype(np.float64)
    q /= np.linalg.norm(q)
    th = 2 * math.atan2(q[3], q[0])
    p = sc["means"][0].astype(np.float64)
    f, z = 64.0, p[2]
    c = (f * p[0] / z + 32, f * p[1] / z + 24)
    s32 = sc["scales"][0].astype(np.float64)
    xs, ys = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    dx, dy = xs - c[0], ys - c[1]
    co, si = math.cos(th), math.sin(th)
    u = (dx * co + dy * si) * z / (f * s32[0])
    v = (-dx * si + dy * co) * z / (f * s32[1])
    rho_uv, rho_lp = u * u + v * v, 2 * (dx * dx + dy * dy)
    alpha = np.minimum(0.99, np.float32(0.8) * np.exp(-np.minimum(rho_uv, rho_lp) / 2))
    expect = np.where(alpha >= 1 / 255, alpha, 0.0)
    assert (expect > 0).sum() > 40 and np.abs(dx[expect > 0]).max() > 10  # a long footprint
    np.testing.assert_allclose(r["alpha"], expect, rtol=0, atol=1e-12)


def test_lowpass_branch_closed_form():
    """A splat far smaller than a pixel is drawn by the screen-space low-pass
    disk: alpha = o exp(-|x - c|^2) (rho = 2 |x - c|^2)."""
    sc, cam = _fronto_scene(s=(0.002, 0.002), o=0.9, z=4.0, N=2, offset_px=(0.3, -0.2))
    r = oracle.render(sc, cam)
    xs, ys = np.meshgrid(np.arange(64) + 0.5, np.arange(48) + 0.5)
    c = (32 + 0.3, 24 - 0.2)
    # the FP32 centre is the FP32-rounded world point projected in FP64
    p = sc["means"][0].astype(np.float64)
    c = (64.0 * p[0] / p[2] + 32, 64.0 * p[1] / p[2] + 24)
    alpha = np.minimum(0.99, np.float32(0.9) * np.exp(-((xs - c[0]) ** 2 + (ys - c[1]) ** 2)))
    alpha = np.where(alpha >= 1 / 255, alpha, 0)
    np.testing.assert_allclose(r["alpha"], alpha, atol=1e-12)


def test_tilted_splat_ray_plane_intersection():
    """R9: u, v of a pixel equal the ray/plane hit expressed in the splat frame,
    computed here independently: ray through the pixel centre, plane through p
    with normal t_u x t_v, u = (P - p).t_u / s_u.  The uv-branch depth is the
    hit's camera z."""
    sc = scenes.tiny_scene(4, K=3, tex_n=4, sh_degree=0)
    cam = scenes.tiny_camera(24, 20)
    R = cam["R"].astype(np.float64)
    t = cam["t"].astype(np.float64)
    f = float(cam["fx"])
    rng = np.random.default_rng(0)
    xy = rng.uniform(0, 20, (100, 2))
    for k in range(3):
        q = sc["quats"][k].astype(np.float64)
        q /= np.linalg.norm(q)
        w, x, y, z = q
        tu = np.array([1 - 2 * (y * y + z * z), 2 * (x * y + w * z), 2 * (x * z - w * y)])
        tv = np.array([2 * (x * y - w * z), 1 - 2 * (x * x + z * z), 2 * (y * z + w * x)])
        p = sc["means"][k].astype(np.float64)
        s = sc["scales"][k].astype(np.float64)
        # camera-space frame
        pc, tuc, tvc = R @ p + t, R @ tu, R @ tv
        n = np.cross(tuc, tvc)
        dirs = np.stack([(xy[:, 0] - float(cam["cx"])) / f, (xy[:, 1] - float(cam["cy"])) / f,
                         np.ones(len(xy))], 1)
        lam = (pc @ n) / (dirs @ n)
        P = dirs * lam[:, None]
        u = (P - pc) @ tuc / s[0]
        v = (P - pc) @ tvc / s[1]
        r = oracle.eval_pairs(sc, cam, k, xy)
        np.testing.assert_allclose(r["u"], u, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(r["v"], v, rtol=1e-9, atol=1e-9)


def test_two_splats_composite():
    """Eq. 2: C = c1 a1 + c2 a2 (1 - a1) for two co-centred fronto-parallel splats."""
    g1 = np.full((2, 2, 3), 0.2)
    g2 = np.full((2, 2, 3), 0.7)
    s1, cam = _fronto_scene(o=0.6, z=3.0, N=2, grid=g1, colour=(0, 0, 0))
    s2, _ = _fronto_scene(o=0.5, z=5.0, N=2, grid=g2, colour=(0, 0, 0))
    sc = {k: (np.concatenate([s1[k], s2[k]]) if isinstance(s1[k], np.ndarray) else s1[k]) for k in s1}
    r = oracle.render(sc, cam)
    a1, a2 = float(np.float32(0.6)), float(np.float32(0.5))
    c1, c2 = float(np.float32(0.2)), float(np.float32(0.7))
    x, y = 32, 24
    np.testing.assert_allclose(r["rgb"][y, x], c1 * a1 + c2 * a2 * (1 - a1), rtol=1e-12)
    np.testing.assert_allclose(r["alpha"][y, x], 1 - (1 - a1) * (1 - a2), rtol=1e-12)
    np.testing.assert_allclose(r["depth"][y, x], 3.0 * a1 + 5.0 * a2 * (1 - a1), rtol=1e-6)
    tr = oracle.pixel_trace(sc, cam, x, y)
    assert list(tr["ids"]) == [0, 1]


def test_transmittance_cutoff_stops_the_stack():
    """Alg. 1 fwd stops before a splat that would take T below 1e-4: eight
    co-centred fronto-parallel splats of alpha a = 0.8 at depths 3, 3.5, ...
    leave T = 0.2^j after j of them (3.2e-4 after five, 6.4e-5 after six),
    so exactly the first five blend (Eq. 2 over them)."""
    parts = []
    for j in range(8):
        g = np.full((2, 2, 3), (j + 1) / 8.0)
        s, cam = _fronto_scene(o=0.8, z=3.0 + 0.5 * j, N=2, grid=g, colour=(0, 0, 0))
        parts.append(s)
    sc = {k: (np.concatenate([p[k] for p in parts]) if isinstance(parts[0][k], np.ndarray) else parts[0][k])
          for k in parts[0]}
    a = float(np.float32(0.8))
    w = [a * (1 - a) ** j for j in range(5)]
    x, y = 32, 24
    r = oracle.render(sc, cam)
    np.testing.assert_allclose(r["alpha"][y, x], 1 - (1 - a) ** 5, rtol=1e-12)
    np.testing.assert_allclose(r["rgb"][y, x], sum(wj * (j + 1) / 8.0 for j, wj in enumerate(w)), rtol=1e-12)
    np.testing.assert_allclose(r["depth"][y, x], sum(wj * (3.0 + 0.5 * j) for j, wj in enumerate(w)), rtol=1e-6)
    assert list(oracle.pixel_trace(sc, cam, x, y)["ids"]) == [0, 1, 2, 3, 4]


@pytest.mark.parametrize("seed", [2, 7, 12])
def test_input_order_does_not_matter(seed):
    """Alg. 1 blends in depth order: permuting the splat arrays leaves the
    image unchanged and permutes the gradients with them (distinct depths,
    so no tie is broken by the splat id)."""
    sc = scenes.tiny_scene(seed, K=8, tex_n=4, sh_degree=2)
    cam = scenes.tiny_camera(32, 24)
    perm = np.random.default_rng(seed).permutation(8)
    sp = dict(sc)
    for k in ("means", "quats", "scales", "opacities", "sh", "textures"):
        sp[k] = np.ascontiguousarray(np.asarray(sc[k])[perm])
    _, z, _ = oracle.keys32(sc, cam)
    assert len(set(z.view(np.uint32).tolist())) == 8
    a, b = oracle.render(sc, cam), oracle.render(sp, cam)
    for k in ("rgb", "depth", "alpha"):
        np.testing.assert_allclose(b[k], a[k], rtol=0, atol=1e-14)
    d = np.random.default_rng(seed + 1).standard_normal((24, 32, 3))
    ga, gb = oracle.backward(sc, cam, d), oracle.backward(sp, cam, d)
    for k in ("means", "quats", "scales", "opacities", "sh", "textures"):
        np.testing.assert_allclose(gb[k], ga[k][perm], rtol=1e-12, atol=1e-14)


def test_constant_grid_equals_plain_2dgs():
    """N = 1 is plain 2DGS (Sec. 4.1); a constant N x N grid must give the same
    image up to rounding, and its texel gradients must sum to the N = 1 gradient
    while every other gradient is unchanged."""
    base = scenes.tiny_scene(7, K=5, tex_n=1, sh_degree=3)
    cam = scenes.tiny_camera(20, 16)
    for N in (2, 4, 8):
        sc = dict(base)
        sc["tex_n"] = N
        sc["textures"] = np.ascontiguousarray(np.broadcast_to(base["textures"], (5, N, N, 3)))
        r1 = oracle.render(base, cam)
        rN = oracle.render(sc, cam)
        for k in ("rgb", "depth", "alpha"):
            np.testing.assert_allclose(rN[k], r1[k], rtol=1e-14, atol=1e-15, err_msg=k)
        dL = np.random.default_rng(1).standard_normal((16, 20, 3))
        g1 = oracle.backward(base, cam, dL)
        gN = oracle.backward(sc, cam, dL)
        np.testing.assert_allclose(gN["textures"].sum(axis=(1, 2)), g1["textures"][:, 0, 0], rtol=1e-10, atol=1e-12)
        for k in ("means", "quats", "scales", "opacities", "sh"):
            np.testing.assert_allclose(gN[k], g1[k], rtol=1e-9, atol=1e-11)


# ------------------------------------------------------------------ invariants --

def test_invariants_plain_1k():
    """alpha + T_final = 1; T_final >= 1e-4 (cutoff); weights sum to alpha <= 1;
    transmittance is monotone along each pixel's list (T_{i+1} = T_i (1 - a_i));
    depth / alpha lies within the depth range of the splats."""
    w = scenes.workload("plain_1k")
    sc, cam = w["scenes"][0], w["cams"][0]
    r = oracle.render(sc, cam)
    np.testing.assert_allclose(r["alpha"] + r["t_final"], 1.0, atol=1e-15)
    assert np.all(r["t_final"] >= 1e-4) and np.all(r["t_final"] <= 1.0)
    valid, z32, _ = oracle.keys32(sc, cam)
    # plane hits lie within sqrt(rho_max) * max scale of the centre depth
    ext = math.sqrt(2 * math.log(255)) * float(sc["scales"].max())
    zmin, zmax = z32[valid].min() - ext, z32[valid].max() + ext
    assert np.all(r["depth"] <= zmax * r["alpha"] + 1e-12)
    assert np.all(r["depth"] >= zmin * r["alpha"] - 1e-12)
    ys, xs = np.nonzero(r["n_contrib"] >= 3)
    for y, x in list(zip(ys, xs))[:40]:
        tr = oracle.pixel_trace(sc, cam, int(x), int(y))
        T = np.concatenate([tr["trans"], [tr["t_final"]]])
        assert T[0] == 1.0
        assert np.all(np.diff(T) <= 0)
        np.testing.assert_allclose(T[1:], T[:-1] * (1 - tr["alpha"]), rtol=1e-14)
        assert np.all(tr["alpha"] >= 1 / 255) and np.all(tr["alpha"] <= 0.99)
        # depth order: FP32 depth keys ascending
        assert np.all(np.diff(z32[tr["ids"]]) >= 0)


def test_prefilter_equals_brute_force():
    """The bbox-prefiltered mode skips only pairs whose alpha is below 1/255."""
    for sc, cam in [
        (scenes.workload("plain_1k")["scenes"][0], scenes.workload("plain_1k")["cams"][0]),
        (scenes.planes_scene(3, K=3000, tex_n=4), scenes.look_at([0, 0, -7], [0, 0, 0], 96, 64)),
    ]:
        a = oracle.render(sc, cam, prefilter=False)
        b = oracle.render(sc, cam, prefilter=True)
        assert b["n_pairs"] < a["n_pairs"]
        for k in ("rgb", "depth", "alpha", "n_contrib"):
            assert np.array_equal(a[k], b[k]), k


def test_fp32_rectangles_are_conservative():
    """Every (pixel, splat) pair with FP64 alpha >= 1/255 lies in the splat's
    FP32 pixel rectangle (R15): the tiled path can skip the rest."""
    for sc, cam in [
        (scenes.workload("plain_1k")["scenes"][0], scenes.workload("plain_1k")["cams"][0]),
        (scenes.planes_scene(4, K=400, tex_n=4, log_scale=(-2.5, 0.7)),
         scenes.look_at([0, 0, -9], [0, 0, 0], 96, 64)),
        (scenes.tiny_scene(9, K=8), scenes.tiny_camera(40, 30)),
    ]:
        valid, _, prect = oracle.keys32(sc, cam)
        W, H = cam["width"], cam["height"]
        xs, ys = np.meshgrid(np.arange(W) + 0.5, np.arange(H) + 0.5)
        xy = np.stack([xs.ravel(), ys.ravel()], 1)
        for k in np.nonzero(valid)[0]:
            r = oracle.eval_pairs(sc, cam, int(k), xy)
            x0, y0, x1, y1 = prect[k]
            px, py = xy[:, 0] - 0.5, xy[:, 1] - 0.5
            outside = (px < x0) | (px > x1) | (py < y0) | (py > y1)
            assert np.all(r["alpha"][outside] < 1 / 255 * (1 - 1e-5))


@pytest.mark.parametrize("s,z,f", [((0.5, 0.3), 4.0, 64.0), ((0.2, 0.45), 6.0, 40.0), ((0.01, 0.02), 5.0, 64.0)])
def test_fp32_rectangle_of_a_fronto_splat_is_tight(s, z, f):
    """R15 in closed form: for a splat parallel to the image plane the box of
    the rho_max ellipse has half-widths sqrt(rho_max) f s / z about the
    projected centre; united with the low-pass disk of radius sqrt(ln 255)
    its pixels are [ceil(c - h - 1/2), floor(c + h - 1/2)], clamped to the
    view (the last case is a sub-pixel splat: the disk decides)."""
    sc, cam = _fronto_scene(s=s, z=z, f=f)
    valid, _, prect = oracle.keys32(sc, cam)
    assert valid[0]
    rho, r_lp = 2 * math.log(255), math.sqrt(math.log(255))
    s32 = np.asarray(s, np.float32).astype(np.float64)
    cx, cy = 32.5, 24.5
    hx = max(math.sqrt(rho) * f * s32[0] / z, r_lp)
    hy = max(math.sqrt(rho) * f * s32[1] / z, r_lp)
    for b in (cx - hx - 0.5, cx + hx - 0.5, cy - hy - 0.5, cy + hy - 0.5):
        assert abs(b - round(b)) > 1e-3  # no bound within FP32 rounding of an integer
    expect = [max(math.ceil(cx - hx - 0.5), 0), max(math.ceil(cy - hy - 0.5), 0),
              min(math.floor(cx + hx - 0.5), 63), min(math.floor(cy + hy - 0.5), 47)]
    assert [int(v) for v in prect[0]] == expect


def test_fp32_keys_against_fp64_projection():
    """FP32 depth = FP64 camera depth to FP32 rounding; culled splats have no
    pixel with alpha >= 1/255; keys sort by tile, then depth, then splat id."""
    w = scenes.workload("plain_1k")
    sc, cam = w["scenes"][0], w["cams"][0]
    valid, z32, prect = oracle.keys32(sc, cam)
    pr = oracle.project(sc, cam)
    z64 = pr["T"][:, 2, 2]
    np.testing.assert_allclose(z32[valid], z64[valid], rtol=3e-7)
    keys, ids = oracle.tile_keys(sc, cam, 16)
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    same = keys[1:] == keys[:-1]
    assert np.all(ids[1:][same] > ids[:-1][same])
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    counts = np.bincount(ids, minlength=len(valid))
    nx = (prect[:, 2] // 16 - prect[:, 0] // 16 + 1)
    ny = (prect[:, 3] // 16 - prect[:, 1] // 16 + 1)
    assert np.array_equal(counts[valid], (nx * ny)[valid])
    assert tiles.max() < 64


@pytest.mark.parametrize("tile", [8, 16])
def test_tile_keys_by_brute_force(tile):
    """Each splat's keys name exactly the tiles its FP32 pixel rectangle
    touches (every tile of a non-square view tested against the rectangle),
    offset by the view's first tile id, with the FP32 depth's bits below."""
    sc = scenes.planes_scene(4, K=300, tex_n=4, log_scale=(-2.5, 0.7))
    cam = scenes.look_at([0, 0, -9], [0, 0, 0], 100, 52)
    off = 1000
    valid, z32, prect = oracle.keys32(sc, cam)
    keys, ids = oracle.tile_keys(sc, cam, tile, tile_offset=off)
    tx_n, ty_n = -(-100 // tile), -(-52 // tile)
    got = {}
    for key, k in zip(keys.tolist(), ids.tolist()):
        got.setdefault(k, set()).add((key >> 32) - off)
        assert key & 0xFFFFFFFF == int(z32[k:k + 1].view(np.uint32)[0])
    assert set(got) == set(np.nonzero(valid)[0].tolist())
    for k, tiles in got.items():
        x0, y0, x1, y1 = prect[k]
        expect = {ty * tx_n + tx for ty in range(ty_n) for tx in range(tx_n)
                  if tx * tile <= x1 and x0 < (tx + 1) * tile and ty * tile <= y1 and y0 < (ty + 1) * tile}
        assert tiles == expect, k

