"""Planted mistakes: every pin set must notice a plausible error in the oracle.

Each mutant below is one small edit of ``oracle/gbill_oracle.cpp``:
- a dropped term, a flipped sign, a wrong constant, swapped texels or a wrong index;
- arithmetic only, so that no mutant can read or write out of bounds.

The edited source is compiled into a temporary library. The oracle module is pointed at it,
and the fast pins of ``test_oracle_pins.py`` and ``test_oracle_fd.py`` run in turn. The test
passes when at least one pin fails for every mutant. Mistakes that the forward and the
backward make consistently, such as a wrong SH sign or a wrong rotation entry, are left to
the closed-form pins. Mistakes that split them, such as a missing adjoint term, are left to
the finite differences.
"""
import concurrent.futures as cf
import os
import subprocess
import types

import pytest

import oracle
from tests import test_adam as adam
from tests import test_oracle_fd as fd
from tests import test_oracle_fit2d as fit
from tests import test_oracle_mip as mip
from tests import test_oracle_pins as pins
from tests import test_oracle_texsh as texsh
from tests import test_oracle_varn as varn

SRC = os.path.join(os.path.dirname(oracle.__file__), "gbill_oracle.cpp")

# name: (original text, planted text)
MUTANTS = {
    # forward (Eq. 2-5, Alg. 1 fwd)
    "low-pass factor 1 instead of 2": ("static const double kLowPass = 2.0;", "static const double kLowPass = 1.0;"),
    "alpha clamp 0.999": ("static const double kAlphaMax = 0.99;", "static const double kAlphaMax = 0.999;"),
    "alpha cutoff 1/128": ("static const double kAlphaMin = 1.0 / 255.0;",
                           "static const double kAlphaMin = 1.0 / 128.0;"),
    "transmittance cutoff 1e-3": ("static const double kTMin = 1e-4;", "static const double kTMin = 1e-3;"),
    "Gaussian exp(-rho)": ("e.G = std::exp(-0.5 * e.rho);", "e.G = std::exp(-e.rho);"),
    "splats blended in input order": ("return a.first < b.first;", "return false;"),
    "splats blended back to front": ("return a.first < b.first;", "return a.first > b.first;"),
    "texels transposed": ("const double *c10 = C + ((b.iu + 1) * stride + b.iv) * 3;\n"
                          "    const double *c01 = C + ((b.iu) * stride + b.iv + 1) * 3;",
                          "const double *c10 = C + ((b.iu) * stride + b.iv + 1) * 3;\n"
                          "    const double *c01 = C + ((b.iu + 1) * stride + b.iv) * 3;"),
    "per-splat grid size ignored": ("bilinear(e.u, e.v, sc.splat_n ? sc.splat_n[k] : N, sg,",
                                    "bilinear(e.u, e.v, N, sg,"),
    "per-splat grid read at its own width": ("sc.textures + k * N * N * 3, cb.col, N);",
                                             "sc.textures + k * N * N * 3, cb.col);"),
    "blend weight with the next T": ("const double w = e.alpha * T;", "const double w = e.alpha * tT;"),
    "depth without the tilt terms": ("cb.zi = e.uv_branch ? (pr.T[6] * e.u + pr.T[7] * e.v + pr.T[8]) : pr.T[8];",
                                     "cb.zi = pr.T[8];"),
    "background dropped": ("rgb[c] = C[c] + T * cx.bg[c];", "rgb[c] = C[c];"),
    "SH basis sign (l = 1, m = -1)": ("put(-c1 * y, 0, -c1, 0);", "put(c1 * y, 0, c1, 0);"),
    "rotation entry sign": ("R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);"),
    "adjugate cofactor sign": ("A[i * 3 + j] = T[r1 * 3 + c1] * T[r2 * 3 + c2] - T[r1 * 3 + c2] * T[r2 * 3 + c1];",
                               "A[i * 3 + j] = T[r1 * 3 + c1] * T[r2 * 3 + c2] + T[r1 * 3 + c2] * T[r2 * 3 + c1];"),
    "low-pass branch comparison reversed": ("e.uv_branch = e.rho_uv <= e.rho_lp;", "e.uv_branch = e.rho_uv >= e.rho_lp;"),
    "uv-to-texel scale N instead of N - 1": ("double up = (N - 1) * (u + sigma) / (2.0 * sigma);",
                                             "double up = N * (u + sigma) / (2.0 * sigma);"),
    "SH basis gradient component dropped": ("put(c1 * z, 0, 0, c1);", "put(c1 * z, 0, 0, 0);"),
    # backward (Alg. 1 bwd, Alg. 2 adj-bilinear) and the chain to the parameters
    "adj-bilinear u difference reversed": ("fu_hat += chat[c] * ((C[i10 + c] - C[i00 + c])",
                                           "fu_hat += chat[c] * ((C[i00 + c] - C[i10 + c])"),
    "adj-bilinear missing the +-sigma mask": ("uv_hat[0] = (u > -sigma && u < sigma) ? k * fu_hat : 0.0;",
                                              "uv_hat[0] = k * fu_hat;"),
    "low-pass centre gradient sign": ("A.c_hat[0] += rho_hat * kLowPass * -2.0 * e.dx;",
                                      "A.c_hat[0] += rho_hat * kLowPass * 2.0 * e.dx;"),
    "back-to-front sum weighted by T": ("for (int ch = 0; ch < 3; ++ch) S[ch] += c.col[ch] * w;",
                                        "for (int ch = 0; ch < 3; ++ch) S[ch] += c.col[ch] * T;"),
    "1 / (1 + alpha) in the alpha adjoint": ("const double inv1ma = 1.0 / (1.0 - a);",
                                             "const double inv1ma = 1.0 / (1.0 + a);"),
    "ray-intersection adjoint sign": ("-(u_hat * e.u + v_hat * e.v) * iz", "(u_hat * e.u + v_hat * e.v) * iz"),
    "low-pass centre gradient y from dx": ("A.c_hat[1] += rho_hat * kLowPass * -2.0 * e.dy;",
                                           "A.c_hat[1] += rho_hat * kLowPass * -2.0 * e.dx;"),
    "depth uv adjoint from the wrong column": ("u_hat += zi_hat * pr.T[6];", "u_hat += zi_hat * pr.T[7];"),
    "principal point cy dropped from the chain": (
        "colhat[j][2] = cam.cx * That[0 * 3 + j] + cam.cy * That[1 * 3 + j] + That[2 * 3 + j];",
        "colhat[j][2] = cam.cx * That[0 * 3 + j] + That[2 * 3 + j];"),
    "scale adjoint against the other tangent": ("sv_hat += world_hat[1][i] * pr.tv[i];",
                                                "sv_hat += world_hat[1][i] * pr.tu[i];"),
    "tangent adjoint with the other scale": ("tu_hat[i] = s[0] * world_hat[0][i];", "tu_hat[i] = s[1] * world_hat[0][i];"),
    "SH coefficient gradient without the basis": ("g->d_sh[(k * M + m) * 3 + c] += Y[m] * A.rgb_hat[c];",
                                                  "g->d_sh[(k * M + m) * 3 + c] += A.rgb_hat[c];"),
    "background adjoint dropped": ("a_hat += (dA - bgdot) * t_final * inv1ma;", "a_hat += dA * t_final * inv1ma;"),
    "gradient through a clamped alpha": ("if (!e.clamped) {", "if (true) {"),
    "depth adjoint index": ("A.T_hat[7] += zi_hat * e.v;", "A.T_hat[7] += zi_hat * e.u;"),
    "centre adjoint sign": ("That[8] -= (A.c_hat[0] * T[2] + A.c_hat[1] * T[5]) / (T[8] * T[8]);",
                            "That[8] += (A.c_hat[0] * T[2] + A.c_hat[1] * T[5]) / (T[8] * T[8]);"),
    "quaternion normalisation adjoint dropped": ("(qh[i] - pr.qn[i] * qd) / pr.qnorm", "qh[i] / pr.qnorm"),
    "SH direction adjoint not projected": ("p_hat[i] += (dir_hat[i] - pr.dir[i] * dd) / pr.dist;",
                                           "p_hat[i] += dir_hat[i] / pr.dist;"),
    # FP32 tile rectangles (keys)
    "key depth from the wrong coordinate": ("*z_out = P2;", "*z_out = P0;"),
    "opacity cull threshold 1/64": ("if (!(o >= 1.0f / 255.0f)) return 0;", "if (!(o >= 1.0f / 64.0f)) return 0;"),
    "near-plane cull dropped": ("if (!(P2 > near_plane)) return 0;", "if (false) return 0;"),
    "rectangle radius too small": ("static const float kRhoMaxF = 11.0825270903f;",
                                   "static const float kRhoMaxF = 9.0f;"),
    "rectangle low bound rounded down": ("const float fx0 = std::fmax(std::ceil(lox - 0.5f), 0.0f);",
                                         "const float fx0 = std::fmax(std::floor(lox - 0.5f), 0.0f);"),
    "low-pass disk left out of the rectangle": (
        "const float lox = std::fmin(elx, cx - kLowPassRadiusF), hix = std::fmax(ehx, cx + kLowPassRadiusF);",
        "const float lox = elx, hix = ehx;"),
}

# fast pins, cheapest first
PINS = [
    (pins.test_sh_basis_matches_scipy, {}),
    (pins.test_bilinear_reproduces_texels, {"N": 4, "sigma": 0.5}),
    (pins.test_bilinear_affine_grid_is_exact_and_oriented, {"N": 4}),
    (pins.test_bilinear_partition_of_unity_and_n1, {}),
    (pins.test_adj_bilinear_matches_finite_differences, {"N": 4}),
    (pins.test_single_splat_at_pixel_centre, {"N": 4, "o": 0.6}),
    (pins.test_single_splat_at_pixel_centre, {"N": 4, "o": 0.995}),
    (pins.test_single_splat_at_pixel_centre, {"N": 4, "o": 0.01}),
    (pins.test_faint_splat_below_the_alpha_cutoff_is_culled, {}),
    (pins.test_empty_and_behind_camera_scenes_render_the_background, {}),
    (pins.test_fronto_parallel_uv_and_colour_closed_form, {}),
    (pins.test_lowpass_branch_closed_form, {}),
    (pins.test_tilted_splat_ray_plane_intersection, {}),
    (pins.test_two_splats_composite, {}),
    (pins.test_transmittance_cutoff_stops_the_stack, {}),
    (pins.test_constant_grid_equals_plain_2dgs, {}),
    (pins.test_fig2_isoline_facts, {}),
    (pins.test_invariants_plain_1k, {}),
    (pins.test_fp32_rectangles_are_conservative, {}),
    (pins.test_fp32_rectangle_of_a_fronto_splat_is_tight, {"s": (0.5, 0.3), "z": 4.0, "f": 64.0}),
    (pins.test_fp32_rectangle_of_a_fronto_splat_is_tight, {"s": (0.01, 0.02), "z": 5.0, "f": 64.0}),
    (pins.test_sh_gradient_finite_difference, {}),
    (fd.test_fd_clamped_opacity_and_lowpass, {}),
    (fd.test_fd_through_clamped_alpha, {}),
    (fd.test_fd_with_background_and_ragged_view, {}),
    (fd.test_fd_all_gradients, {"N": 4, "D": 3}),
    (fd.test_fd_texture_only_heavy_grid, {}),
    (varn.test_embedded_grids_equal_the_uniform_scene, {}),
]


def _compile(src_text: str, out: str) -> str:
    cpp = out[:-3] + ".cpp"
    with open(cpp, "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", *oracle.GXX_FLAGS, "-o", out, cpp])
    return out


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(SRC).read()
    d = tmp_path_factory.mktemp("mutants")
    jobs = {}
    for i, (name, (old, new)) in enumerate(MUTANTS.items()):
        assert src.count(old) == 1, f"mutation site of {name!r} not found once in the oracle"
        jobs[name] = (src.replace(old, new), str(d / f"m{i}.so"))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_compile, text, path) for name, (text, path) in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_mistake_fails_a_pin(name, mutant_libs, monkeypatch):
    monkeypatch.setattr(oracle, "_lib", oracle.load(mutant_libs[name]))
    for pin, kw in PINS:
        try:
            pin(**kw)
        except Exception as e:  # an assertion, or a check that raised on a malformed result
            print(f"{name}: caught by {pin.__name__}{kw or ''} ({type(e).__name__})")
            return
    pytest.fail(f"no pin notices the planted mistake: {name}")


# --- the oracle's numpy steps (mip filter, per-texel SH, tile keys, Adam,
# the image-fitting map and loss): planted in a copy of the module source,
# whose functions replace the module's for the test

PY_SRC = os.path.join(os.path.dirname(oracle.__file__), "__init__.py")

PY_MUTANTS = {
    "mip block summed, not averaged": (".mean(axis=(2, 4)))", ".sum(axis=(2, 4)))"),
    "mip adjoint divided by 2^l": ("/ float(f * f)", "/ float(f)"),
    "texel SH grid transposed": ('"km,kijmc->kijc"', '"km,kjimc->kijc"'),
    "texel SH view direction reversed": ("v = p - _campos(cam)[None, :]", "v = _campos(cam)[None, :] - p"),
    "tile id with x and y swapped": ("t = (tile_offset + ty[:, None] * tiles_x + tx[None, :])",
                                     "t = (tile_offset + ty[:, None] + tx[None, :] * tiles_x)"),
    "tile offset dropped": ("t = (tile_offset + ty[:, None] * tiles_x + tx[None, :])",
                            "t = (ty[:, None] * tiles_x + tx[None, :])"),
    "Adam without bias correction": ("m_hat = m / (1.0 - beta1 ** step)", "m_hat = m"),
    "Adam second moment of g, not g^2": ("(1.0 - beta2) * g * g", "(1.0 - beta2) * g"),
    "fit quaternion with the full angle": ("q[:, 3] = np.sin(th / 2)", "q[:, 3] = np.sin(th)"),
    "fit angle adjoint sign": ("0.5 * (np.cos(th / 2) * dq[:, 3] - np.sin(th / 2) * dq[:, 0])",
                               "0.5 * (np.cos(th / 2) * dq[:, 3] + np.sin(th / 2) * dq[:, 0])"),
    "fit logit adjoint without 1 - o": ("_f64(g[\"opacities\"]) * o * (1.0 - o)", "_f64(g[\"opacities\"]) * o"),
    "MSE gradient without the factor 2": ("2.0 * r / r.size", "r / r.size"),
}

PY_PINS = [
    (mip.test_mip_grid_matches_loops, {}),
    (mip.test_mip_adjoint_is_the_transpose, {}),
    (mip.test_top_level_is_the_mean_colour, {"N": 4}),
    (mip.test_constant_grid_renders_the_same_at_every_level, {}),
    (mip.test_texture_gradient_at_a_mip_level_by_central_differences, {"lvl": 1}),
    (texsh.test_degree_zero_coefficient_is_the_colour, {}),
    (texsh.test_identical_texel_sh_equals_splat_sh, {"Dt": 2}),
    (texsh.test_texel_sh_gradients_by_central_differences, {"name": "means"}),
    (texsh.test_texel_sh_gradients_by_central_differences, {"name": "textures"}),
    (pins.test_tile_keys_by_brute_force, {"tile": 16}),
    (pins.test_fp32_keys_against_fp64_projection, {}),
    (adam.test_oracle_adam_constant_gradient_closed_form, {}),
    (adam.test_oracle_adam_zero_gradient_keeps_parameters, {}),
    (fit.test_fit_params_closed_forms, {}),
    (fit.test_mse_closed_form_and_gradient, {}),
    (fit.test_fit_gradients_by_central_differences, {"name": "theta"}),
    (fit.test_fit_gradients_by_central_differences, {"name": "logit_opacities"}),
]


@pytest.mark.filterwarnings("ignore::RuntimeWarning")  # a mutant may take sqrt of a negative moment
@pytest.mark.parametrize("name", list(PY_MUTANTS))
def test_planted_numpy_mistake_fails_a_pin(name, monkeypatch):
    old, new = PY_MUTANTS[name]
    src = open(PY_SRC).read()
    assert src.count(old) == 1, f"mutation site of {name!r} not found once in the oracle module"
    mod = types.ModuleType("oracle_mutant")
    mod.__file__ = oracle.__file__
    exec(compile(src.replace(old, new), PY_SRC, "exec"), mod.__dict__)
    for attr, val in vars(mod).items():
        if callable(val) and getattr(val, "__module__", None) == "oracle_mutant":
            monkeypatch.setattr(oracle, attr, val)
    for pin, kw in PY_PINS:
        try:
            pin(**kw)
        except Exception as e:  # an assertion, or a check that raised on a malformed result
            print(f"{name}: caught by {pin.__name__}{kw or ''} ({type(e).__name__})")
            return
    pytest.fail(f"no pin notices the planted mistake: {name}")

