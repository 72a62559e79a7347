"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle (an exact substring
replacement: a dropped term, a wrong sign, a swapped operand, a misread
constant) and runs every pin of the oracle's pin file against the copy: at
least one must fail.  A copy without any change must pass them all, so the
harness itself cannot be what fails.  The renderer's oracle
(``oracle/wsr_oracle.c``) is copied, built with the oracle's own compiler
flags and loaded in place of the real library; the training-step oracle
(``oracle/train.py``) is copied and imported as a separate module in place
of the real one.  The oracle's own files are never modified.
"""
import importlib.util
import inspect
import os
import subprocess

import pytest

import oracle

SRC = os.path.join(os.path.dirname(oracle.__file__), "wsr_oracle.c")
TRAIN_SRC = os.path.join(os.path.dirname(oracle.__file__), "train.py")

# name -> (text in the oracle, planted replacement); each text occurs exactly once
MUTANTS = {
    # projection and footprint (Eqs. 3, 5; 3DGS pre-processing)
    "no_dilation": ("#define ORC_DILATION 0.3", "#define ORC_DILATION 0.0"),
    "rotation_sign": ("R[1] = 2 * (x * y - w * z);", "R[1] = 2 * (x * y + w * z);"),
    "fx_fy_swapped_in_jacobian": (
        "const double J[6] = {cam->fx / tz, 0, -cam->fx * rxc / tz, 0, cam->fy / tz, -cam->fy * ryc / tz};",
        "const double J[6] = {cam->fy / tz, 0, -cam->fy * rxc / tz, 0, cam->fx / tz, -cam->fx * ryc / tz};"),
    "y_clamped_with_x_limit": ("const double ryc = clampd(ty / tz, -ORC_CLAMP * tany, ORC_CLAMP * tany);",
                               "const double ryc = clampd(ty / tz, -ORC_CLAMP * tanx, ORC_CLAMP * tanx);"),
    "no_near_plane": ("if (!(o->t[2] > cam->znear))", "if (!(o->t[2] > 0.0))"),
    "scale_not_exponentiated": (
        "s[k] = exp(S->log_scales[3 * i + k]);\n    for (int r = 0; r < 3; ++r)\n        for (int c = 0; c < 3; ++c) M",
        "s[k] = S->log_scales[3 * i + k];\n    for (int r = 0; r < 3; ++r)\n        for (int c = 0; c < 3; ++c) M"),
    # colour and opacity (Eqs. 4, 11)
    "no_condon_shortley_phase": ("pref = Kl * sqrt(2.0) * ipow(-1.0, am);", "pref = Kl * sqrt(2.0);"),
    "no_colour_offset": ("o->color[ch] = r + 0.5 > 0 ? r + 0.5 : 0.0;", "o->color[ch] = r > 0 ? r : 0.0;"),
    "sigmoid_sign": ("o->u = 1.0 / (1.0 + exp(-S->opac[i]));", "o->u = 1.0 / (1.0 + exp(S->opac[i]));"),
    # weights (Eqs. 8-10) and the weighted sum (Eq. 7)
    "depth_as_distance": ("o->d = o->t[2];",
                          "o->d = sqrt(o->t[0] * o->t[0] + o->t[1] * o->t[1] + o->t[2] * o->t[2]);"),
    "lc_not_clamped": ("o->w = (lin > 0 ? lin : 0.0) * S->lc_v[i];", "o->w = lin * S->lc_v[i];"),
    "exp_weight_sign": ("o->w = exp(-wt->sigma * pow(d, wt->beta));", "o->w = exp(wt->sigma * pow(d, wt->beta));"),
    "gaussian_without_half": ("const double a = o->u * o->w * g;            /* alpha_i w(d_i) */",
                              "const double a = o->u * o->w * g * g;            /* alpha_i w(d_i) */"),
    "no_background_colour": ("out_rgb[3 * p + ch] = (wt.c_bg[ch] * wt.w_bg + num[3 * p + ch]) / D;",
                             "out_rgb[3 * p + ch] = num[3 * p + ch] / D;"),
    "cutoff_misread": ("#define ORC_CUTOFF 9.0", "#define ORC_CUTOFF 8.0"),
    # gradient
    "beta_derivative_without_log": ("gbeta += dL_dw * (-wt->sigma * db * log(d)) * o->w;",
                                    "gbeta += dL_dw * (-wt->sigma * db) * o->w;"),
    "conic_offdiagonal_counted_once": ("t[3] = dLdq * 2.0 * dx * dy;", "t[3] = dLdq * dx * dy;"),
    "mean_gradient_sign": ("t[1] = dLdq * (-2.0) * (o->conic[1] * dx + o->conic[2] * dy);",
                           "t[1] = dLdq * (2.0) * (o->conic[1] * dx + o->conic[2] * dy);"),
    "projection_depth_term_sign": (
        "g_t[2] += -g2[0] * cam->fx * tx / (tz * tz) - g2[1] * cam->fy * ty / (tz * tz);",
        "g_t[2] += -g2[0] * cam->fx * tx / (tz * tz) + g2[1] * cam->fy * ty / (tz * tz);"),
    "background_weight_gradient_sign": ("g_wpar[2] += grad_rgb[3 * p + ch] * (wt.c_bg[ch] - rgb[3 * p + ch]) / D;",
                                        "g_wpar[2] += grad_rgb[3 * p + ch] * (rgb[3 * p + ch] - wt.c_bg[ch]) / D;"),
    "covariance_chain_factor": ("for (int e = 0; e < 6; ++e) GT[e] *= 2.0;", "for (int e = 0; e < 6; ++e) GT[e] *= 1.0;"),
    "sigmoid_derivative": ("out->opac[0] = dL_du * o->u * (1.0 - o->u);", "out->opac[0] = dL_du * o->u;"),
    "quaternion_not_projected": ("out->quats[k] = (gqn[k] - q[k] * dot) / qn;",
                                 "out->quats[k] = gqn[k] / qn;"),
    "legendre_normalisation_inverted": ("const double norm = sqrt(fact(l - am) / fact(l + am));",
                                        "const double norm = sqrt(fact(l + am) / fact(l - am));"),
    "sh_index_order": ("const int idx = l * l + l + m;", "const int idx = l * l + l - m;"),
    "rotation_derivative_entry": ("{0, 0, -4 * y, -4 * z},", "{0, 0, -4 * y, 4 * z},"),
    "direction_gradient_not_tangential": ("g_p[e] += (g_dir[e] - o->dir[e] * dd) / o->vnorm;",
                                          "g_p[e] += g_dir[e] / o->vnorm;"),
    "lc_sigma_derivative_sign": ("gsig += dL_dw * v * d / (wt->sigma * wt->sigma);",
                                 "gsig -= dL_dw * v * d / (wt->sigma * wt->sigma);"),
    "clamped_x_moves_with_t": ("const int freex = (tx / tz >= -limx && tx / tz <= limx);", "const int freex = 1;"),
    "camera_centre_from_rows": (
        "f[k] = -(cam->R[k] * cam->T[0] + cam->R[3 + k] * cam->T[1] + cam->R[6 + k] * cam->T[2]);",
        "f[k] = -(cam->R[3 * k] * cam->T[0] + cam->R[3 * k + 1] * cam->T[1] + cam->R[3 * k + 2] * cam->T[2]);"),
    "principal_point_swapped": ("o->mean2d[0] = cam->fx * tx / tz + cam->cx;", "o->mean2d[0] = cam->fx * tx / tz + cam->cy;"),
    "colour_gradient_without_opacity": ("t[6 + ch] = c->G[3 * p + ch] * a / D;                   /* dL/dc */",
                                        "t[6 + ch] = c->G[3 * p + ch] * g / D;                   /* dL/dc */"),
    "exp_depth_derivative_power": ("dL_dd = dL_dw * (-wt->sigma * wt->beta * pow(d, wt->beta - 1.0)) * o->w;",
                                   "dL_dd = dL_dw * (-wt->sigma * wt->beta * pow(d, wt->beta)) * o->w;"),
    "opacity_sh_gradient_basis": ("gHa[k] = dL_du * Y[k];", "gHa[k] = dL_du;"),
    "footprint_extent_two_sigma": ("o->rx = 3.0 * sqrt(a);", "o->rx = 2.0 * sqrt(a);"),
    "jacobian_clamp_misread": ("#define ORC_CLAMP 1.3", "#define ORC_CLAMP 1.2"),
    # (the +1 is slack only: 3 sqrt(a) is the exact x-extent of q <= 9, so the range one column
    # short of the exact bound is the smallest mistake a pin can see)
    "pixel_range_one_column_short": ("*x1 = (int)ceil(o->mean2d[0] + rx - 0.5) + 1;",
                                     "*x1 = (int)ceil(o->mean2d[0] + rx - 0.5) - 2;"),
    "row_bands_overlap": ("jobs[t].lo = n * t / nthreads;", "jobs[t].lo = n * t / nthreads - (t > 0);"),
    "pixel_list_bound_too_tight": ("if (fabs(dx) > o->rx + 1.0 || fabs(dy) > o->ry + 1.0) continue;",
                                   "if (fabs(dx) > 0.5 * o->rx || fabs(dy) > 0.5 * o->ry) continue;"),
    "background_colour_gradient": ("g_wpar[3 + ch] += grad_rgb[3 * p + ch] * wt.w_bg / D;",
                                   "g_wpar[3 + ch] += grad_rgb[3 * p + ch] / D;"),
    # cutoff ties: the FP32 rounding model behind the windows, and the bounds built on them
    "tie_model_without_the_mean": ("const double t_mean = 2.0 * (fabs(vx) * m->ex + fabs(vy) * m->ey);",
                                   "const double t_mean = 0.0;"),
    "tie_model_without_the_rows": ("const double t_rows = 2.0 * sqrt(tv2 * ev2);", "const double t_rows = 0.0;"),
    "tie_model_without_the_evaluation": ("return 2.0 * (t_mean + t_rows + t_sums + t_rec + t_cut + t_eval);",
                                         "return 2.0 * (t_mean + t_rows + t_sums + t_rec + t_cut);"),
    "tie_window_a_twentieth": ("return 2.0 * (t_mean + t_rows + t_sums + t_rec + t_cut + t_eval);",
                               "return 0.1 * (t_mean + t_rows + t_sums + t_rec + t_cut + t_eval);"),
    "tie_allowance_over_the_unmoved_denominator": (
        "if (amb[p] > 0) amb[p] = dlo > 0 ? amb[p] / dlo : HUGE_VAL;",
        "if (amb[p] > 0) amb[p] = amb[p] / fabs(out_den[p]);"),
    "tie_bound_ignores_the_colour_shift": ("dla += Gc * (c->amb[p] + e * c->mass[p] / fabs(D)) / dlo;",
                                           "dla += Gc * (e * c->mass[p] / fabs(D)) / dlo;"),
    "tie_bound_chain_with_signs": ("out[k] = s > 0 ? out[k] + s * fabs(x[k]) : x[k];",
                                   "out[k] = s > 0 ? out[k] + s * x[k] : x[k];"),
    "tie_bound_background_weight_ignores_the_colour_shift": (
        "b_wpar[2] += dlo > 0 ? Gc * (amb[p] + fabs(wt.c_bg[ch] - rgb[3 * p + ch]) * mass[p] / fabs(D)) / dlo",
        "b_wpar[2] += dlo > 0 ? Gc * (fabs(wt.c_bg[ch] - rgb[3 * p + ch]) * mass[p] / fabs(D)) / dlo"),
    "tie_bound_conic_terms_halved": ("const double sq = fabs(uw) * 0.5 * g * dla;",
                                     "const double sq = fabs(uw) * 0.25 * g * dla;"),
}


def _build(text: str, path) -> str:
    # the flags of oracle.build(): portable, no FMA contraction
    src = path / "mutant.c"
    src.write_text(text)
    so = path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    str(src), "-o", str(so), "-lm", "-lpthread"], check=True)
    return str(so)


def _run_pins(P=None, first=False):
    """Every pin of a pin module (test_oracle_pins.py by default) with each
    of its parameter sets; returns the (pin, parameters) that failed (with
    ``first``, stops at the first failure)."""
    if P is None:
        from tests import test_oracle_pins as P
    failed = []
    for name, fn in inspect.getmembers(P, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != P.__name__:
            continue
        combos = [{}]
        for m in reversed(getattr(fn, "pytestmark", [])):
            if m.name != "parametrize":
                continue
            names = [s.strip() for s in m.args[0].split(",")]
            combos = [{**c, **dict(zip(names, v if len(names) > 1 else (v,)))} for c in combos for v in m.args[1]]
        for kw in combos:
            try:
                fn(**kw)
            except Exception:       # an assertion, or a non-finite result caught by numpy
                failed.append((name, kw))
                if first:
                    return failed
    return failed


def _with_library(monkeypatch, so):
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: so)


def test_an_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    _with_library(monkeypatch, _build(open(SRC).read(), tmp_path))
    assert _run_pins() == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_a_planted_mistake_fails_a_pin(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, "the planted text must name one place in the oracle"
    _with_library(monkeypatch, _build(text.replace(old, new), tmp_path))
    assert _run_pins(first=True), f"no pin fails with the mistake '{name}' planted"


# the training-step oracle (Sec. 4.4 loss, Adam): name -> (text, planted replacement)
TRAIN_MUTANTS = {
    "ssim_c1_misread": ("SSIM_C1 = 0.01 ** 2", "SSIM_C1 = 0.03 ** 2"),
    "ssim_c2_misread": ("SSIM_C2 = 0.03 ** 2", "SSIM_C2 = 0.01 ** 2"),
    "window_sigma_misread": ("SSIM_SIGMA = 1.5", "SSIM_SIGMA = 1.0"),
    "window_not_normalised": ("    g /= g.sum()\n    return np.outer(g, g)", "    return np.outer(g, g)"),
    "filter_is_a_convolution": ("out += win[a, b] * pad[a:a + H, b:b + W]",
                                "out += win[-1 - a, -1 - b] * pad[a:a + H, b:b + W]"),
    "adjoint_with_transposed_window": ("acc[a:a + H, b:b + W] += win[a, b] * g", "acc[a:a + H, b:b + W] += win[b, a] * g"),
    "ssim_mean_gradient_sign": ("/ (b1 * b2) - s * (2.0 * mx / b1 - 2.0 * mx / b2)",
                                "/ (b1 * b2) + s * (2.0 * mx / b1 - 2.0 * mx / b2)"),
    "ssim_second_moment_gradient_sign": ("d_exx = -s / b2", "d_exx = s / b2"),
    "ssim_cross_moment_gradient_factor": ("d_exy = 2.0 * a1 / (b1 * b2)", "d_exy = a1 / (b1 * b2)"),
    "dssim_gradient_sign": ("gs = np.full(a.shape[:2], -lam / count)", "gs = np.full(a.shape[:2], lam / count)"),
    "l1_gradient_sign": ("ga += (1.0 - lam) * np.sign(a - b) / count", "ga += (1.0 - lam) * np.sign(b - a) / count"),
    "lambda_on_the_wrong_term": ("loss=(1.0 - lam) * l1 + lam * (1.0 - ssim)", "loss=lam * l1 + (1.0 - lam) * (1.0 - ssim)"),
    "adam_v_not_bias_corrected": ("v_hat = v / (1.0 - beta2 ** t)", "v_hat = v"),
    "adam_m_corrected_with_beta2": ("m_hat = m / (1.0 - beta1 ** t)", "m_hat = m / (1.0 - beta2 ** t)"),
    "adam_eps_inside_the_root": ("(np.sqrt(v_hat) + eps)", "np.sqrt(v_hat + eps)"),
    "adam_second_moment_of_g": ("(1.0 - beta2) * g * g", "(1.0 - beta2) * np.abs(g)"),
}


def _with_train_module(monkeypatch, text, path):
    src = path / "train_mutant.py"
    src.write_text(text)
    spec = importlib.util.spec_from_file_location("oracle_train_mutant", str(src))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    from tests import test_train_oracle_pins as P
    monkeypatch.setattr(P, "T", mod)
    return P


def test_an_unchanged_copy_of_the_training_oracle_passes_every_pin(tmp_path, monkeypatch):
    P = _with_train_module(monkeypatch, open(TRAIN_SRC).read(), tmp_path)
    assert _run_pins(P) == []


@pytest.mark.parametrize("name", sorted(TRAIN_MUTANTS))
def test_a_planted_mistake_in_the_training_oracle_fails_a_pin(name, tmp_path, monkeypatch):
    old, new = TRAIN_MUTANTS[name]
    text = open(TRAIN_SRC).read()
    assert text.count(old) == 1, "the planted text must name one place in the oracle"
    P = _with_train_module(monkeypatch, text.replace(old, new), tmp_path)
    assert _run_pins(P, first=True), f"no pin fails with the mistake '{name}' planted"
