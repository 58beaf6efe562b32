"""Planted mistakes in the oracle.

Each entry below writes one plausible mistake into a scratch copy of the oracle's C source:
a dropped term, a wrong sign, index or factor, a transposed operand, a missing
projection. The copy is compiled, and the oracle's pins then run against it. Every
mistake must make at least one pin fail. A pin set that lets a mistake through does not
pin the oracle.

Groups:
- model: forward model, derivatives, prior, CG and LM loop (Eq. (1), (2), (5)-(9));
- options: the safeguard of Alg. 2, the geometry priors of Eq. (6), α continuation,
  gradient projection and the linear bound of Sec. 2.2;
- depth: the depth factors of Eq. (5).

The mistake is planted on the CPU only, in a temporary directory; the committed oracle
is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "pget_oracle.c")

PIN_FILES = ["test_oracle_forward.py", "test_oracle_derivatives.py", "test_oracle_solver.py",
             "test_oracle_accel.py", "test_oracle_geo.py", "test_oracle_sgp.py", "test_oracle_linear.py",
             "test_oracle_depth.py"]
FIRST = {"model": PIN_FILES[:3], "options": PIN_FILES[3:7], "depth": PIN_FILES[7:]}

# (name, group, text in the oracle source, text replacing its first occurrence)
MUTATIONS = [
    ('half_self_term_dropped', 'model', 'double E = h * (S + 0.5 * m);', 'double E = h * S;'),
    ('attenuation_accumulated_away_from_detector', 'model', 'for (int j = o->T - 1; j >= 0; --j) {', 'for (int j = 0; j < o->T; ++j) {'),
    ('jvp_attenuation_sign', 'model', '(a - l * c * dE);', '(a + l * c * dE);'),
    ('vjp_half_self_term_dropped', 'model', 'double Q = P + 0.5 * c * term;', 'double Q = P;'),
    ('bilinear_weights_transposed', 'model', 'double ws[4] = {(1 - ax) * (1 - ay), ax * (1 - ay), (1 - ax) * ay, ax * ay};', 'double ws[4] = {(1 - ax) * (1 - ay), ay * (1 - ax), (1 - ay) * ax, ax * ay};'),
    ('ray_normal_sign', 'model', 'double x1 = -ry->s * ry->st + t * ry->ct;', 'double x1 = ry->s * ry->st + t * ry->ct;'),
    ('box_subray_weights', 'model', 'w[k] = 1.0 - fabs(u[k]) / o->p;', 'w[k] = 1.0;'),
    ('second_bank_not_interleaved', 'model', '? 0.5 : 0.0;', '? 0.0 : 0.0;'),
    ('divergence_sign', 'model', 'if (ix > 0) v += gx[i - 1];', 'if (ix > 0) v -= gx[i - 1];'),
    ('tv_weight_without_sqrt', 'model', '1.0 / sqrt(gx[i] * gx[i] + gy[i] * gy[i] + eps * eps)', '1.0 / (gx[i] * gx[i] + gy[i] * gy[i] + eps * eps)'),
    ('cg_beta_inverted', 'model', 'double beta = rr_new / rr;', 'double beta = rr / rr_new;'),
    ('lm_model_decrease_factor', 'model', '- 0.5 * og_dot(m, Js, Js) - 0.5 * sHs;', '- og_dot(m, Js, Js) - 0.5 * sHs;'),
    ('lm_damping_raised_on_success', 'model', 'nu *= pr->nu_up;', 'nu *= pr->nu_down;'),
    ('lm_step_not_projected', 'model', 'ut[i] = lam[i] + delta[i];\n            ut[np + i] = mu[i] + delta[np + i];\n            og_project_px(pr, &ut[i], &ut[np + i]);', 'ut[i] = lam[i] + delta[i];\n            ut[np + i] = mu[i] + delta[np + i];'),
    ('sgp_no_cap', 'options', '        if (lstep > 1.0) lstep = 1.0;\n', ''),
    ('sgp_wrong_bound', 'options', 'pm = og_clamp(*m, 0.0, pr->mu_max);', 'pm = og_clamp(*m, 0.0, pr->lambda_max);'),
    ('sgp_no_grad_update', 'options', '            gq[i] += lstep * Ad[i];\n', ''),
    ('sgp_sign', 'options', 'double zl = lam[i] + x[i] - alpha * gq[i], zm = mu[i] + x[np + i] - alpha * gq[np + i];', 'double zl = lam[i] + x[i] + alpha * gq[i], zm = mu[i] + x[np + i] + alpha * gq[np + i];'),
    ('geo_grad_no2', 'options', '        grad[i] += 2.0 * pr->geo_alpha_lambda * om2 * lam[i];', '        grad[i] += pr->geo_alpha_lambda * om2 * lam[i];'),
    ('geo_no_hess', 'options', '    og_geo_hess_add(n, pr, v, out);\n}', '}'),
    ('geo_no_water', 'options', '        grad[np + i] += 2.0 * pr->geo_alpha_mu * om2 * (mu[i] - pr->geo_mu_water);', '        grad[np + i] += 2.0 * pr->geo_alpha_mu * om2 * mu[i];'),
    ('geo_no_quad_model', 'options', '    sHs += og_geo_quad(n, pr, s);\n    return -og_dot', '    return -og_dot'),
    ('geo_om_not_squared', 'options', '        double om2 = (1.0 - pr->geo_mask[i]) * (1.0 - pr->geo_mask[i]);\n        out[i]', '        double om2 = (1.0 - pr->geo_mask[i]);\n        out[i]'),
    ('cont_no_f_refresh', 'options', '            f = og_objective(g, &prk, lam, mu, y, r);\n            og_gradient', '            og_gradient'),
    ('cont_no_grad_refresh', 'options', '            og_gradient(g, &prk, lam, mu, r, Wl, Wm, grad, tmp);\n        }\n        pr = &prk;', '        }\n        pr = &prk;'),
    ('cont_off_by_one', 'options', '        int e = k < pr->alpha_decay_iters ? k : pr->alpha_decay_iters;', '        int e = k + 1 < pr->alpha_decay_iters ? k + 1 : pr->alpha_decay_iters;'),
    ('cont_no_halt', 'options', '        int e = k < pr->alpha_decay_iters ? k : pr->alpha_decay_iters;', '        int e = k;'),
    ('flip_compare', 'options', 'out->accept = rho > pr->eta && pred_p >= pred_s;', 'out->accept = rho > pr->eta && pred_p <= pred_s;'),
    ('no_half_JsJs', 'options', 'return -og_dot(2 * np, s, grad) - 0.5 * og_dot(m, Js, Js) - 0.5 * sHs;', 'return -og_dot(2 * np, s, grad) - og_dot(m, Js, Js) - 0.5 * sHs;'),
    ('no_projection', 'options', '        ut[i] = pl[i];\n        ut[np + i] = pm[i];\n        og_project_px(pr, &ut[i], &ut[np + i]);', '        ut[i] = pl[i];\n        ut[np + i] = pm[i];'),
    ('rho_with_step_pred', 'options', 'double rho = (pred_p > 0.0 && isfinite(fp)) ? ared / pred_p : -INFINITY;', 'double rho = (pred_s > 0.0 && isfinite(fp)) ? ared / pred_s : -INFINITY;'),
    ('nu_swap', 'options', 'out->nu_next = rho < pr->rho_lo ? nu * pr->nu_up : (rho > pr->rho_hi ? nu * pr->nu_down : nu);', 'out->nu_next = rho < pr->rho_lo ? nu * pr->nu_down : (rho > pr->rho_hi ? nu * pr->nu_up : nu);'),
    ('sHs_sign', 'options', '    return -og_dot(2 * np, s, grad) - 0.5 * og_dot(m, Js, Js) - 0.5 * sHs;', '    return -og_dot(2 * np, s, grad) - 0.5 * og_dot(m, Js, Js) + 0.5 * sHs;'),
    ('rho_ge_eta', 'options', 'out->accept = rho > pr->eta && pred_p >= pred_s;', 'out->accept = rho >= 0 && pred_p >= pred_s;'),
    ('no_denominator', 'options', 'double t = ((*l - b) * k + *m) / (k * k + 1.0);', 'double t = ((*l - b) * k + *m);'),
    ('no_t_hi', 'options', '        if (k > 0.0 && (pr->lambda_max - b) / k < t_hi) t_hi = (pr->lambda_max - b) / k;\n', ''),
    ('offset_sign', 'options', 'if (pr->lin_constraint && pl - pr->lin_slope * pm > pr->lin_offset) {', 'if (pr->lin_constraint && pl - pr->lin_slope * pm > -pr->lin_offset) {'),
    ('project_box_point', 'options', 'double t = ((*l - b) * k + *m) / (k * k + 1.0);', 'double t = ((pl - b) * k + pm) / (k * k + 1.0);'),
    ('foot_sign', 'options', 'double t = ((*l - b) * k + *m) / (k * k + 1.0);', 'double t = ((*l + b) * k + *m) / (k * k + 1.0);'),
    ('swap_lm', 'options', '        pl = k * t + b;\n        pm = t;', '        pm = k * t + b;\n        pl = t;'),
    ('sgp_unit_pg_unprojected', 'options', '            double z1l = lam[i] + x[i] - gq[i], z1m = mu[i] + x[np + i] - gq[np + i];\n            og_project_px(pr, &z1l, &z1m);', '            double z1l = lam[i] + x[i] - gq[i], z1m = mu[i] + x[np + i] - gq[np + i];'),
    ('lm_start_unprojected', 'options', '    og_project(pr, np, lam, mu);\n    double f = og_objective', '    double f = og_objective'),
    ('step_box_only', 'options', '        ut[i] = lam[i] + delta[i];\n            ut[np + i] = mu[i] + delta[np + i];\n            og_project_px(pr, &ut[i], &ut[np + i]);', '        ut[i] = lam[i] + delta[i] < 0 ? 0 : (lam[i] + delta[i] > pr->lambda_max ? pr->lambda_max : lam[i] + delta[i]);\n            ut[np + i] = mu[i] + delta[np + i] < 0 ? 0 : (mu[i] + delta[np + i] > pr->mu_max ? pr->mu_max : mu[i] + delta[np + i]);'),
    ('w_reversed', 'depth', 'static double og_dw(const og_ctx* o, int j) { return o->g.depth_w ? o->g.depth_w[j] : 1.0; }', 'static double og_dw(const og_ctx* o, int j) { return o->g.depth_w ? o->g.depth_w[o->T - 1 - j] : 1.0; }'),
    ('c_reversed', 'depth', 'static double og_dc(const og_ctx* o, int j) { return o->g.depth_c ? o->g.depth_c[j] : 1.0; }', 'static double og_dc(const og_ctx* o, int j) { return o->g.depth_c ? o->g.depth_c[o->T - 1 - j] : 1.0; }'),
    ('c_off_by_one', 'depth', 'static double og_dc(const og_ctx* o, int j) { return o->g.depth_c ? o->g.depth_c[j] : 1.0; }', 'static double og_dc(const og_ctx* o, int j) { return o->g.depth_c ? o->g.depth_c[j > 0 ? j - 1 : 0] : 1.0; }'),
    ('jvp_no_c_dE', 'depth', '(a - l * c * dE)', '(a - l * dE)'),
    ('jvp_no_c_exp', 'depth', 'q += h * og_dw(o, j) * exp(-c * E) * (a - l * c * dE);', 'q += h * og_dw(o, j) * exp(-E) * (a - l * c * dE);'),
    ('vjp_prefix_no_c', 'depth', '        P += c * term;', '        P += term;'),
    ('vjp_half_no_c', 'depth', 'double Q = P + 0.5 * c * term;', 'double Q = P + 0.5 * term;'),
    ('vjp_no_w', 'depth', 'ex[j] = og_dw(o, j) * exp(-og_dc(o, j) * h * (S + 0.5 * m));', 'ex[j] = exp(-og_dc(o, j) * h * (S + 0.5 * m));'),
    ('fwd_w_in_exp', 'depth', 'q += h * og_dw(o, j) * l * exp(-og_dc(o, j) * E);', 'q += h * l * exp(-og_dc(o, j) * og_dw(o, j) * E);'),
]


@pytest.fixture(scope="module")
def scratch(tmp_path_factory):
    """A copy of the oracle, the tests and the package's Python modules (the synthetic
    inputs), without built libraries."""
    d = tmp_path_factory.mktemp("planted")
    skip = shutil.ignore_patterns("*.so", "*.so.*", "__pycache__", "csrc", "*.tmp")
    for sub in ("oracle", "tests", "paper_2604_26745_gb300"):
        shutil.copytree(os.path.join(ROOT, sub), os.path.join(d, sub), ignore=skip)
    shutil.copy(os.path.join(ROOT, "pytest.ini"), d)
    return str(d)


def test_every_pattern_is_in_the_source():
    src = open(SRC).read()
    names = [m[0] for m in MUTATIONS]
    assert len(set(names)) == len(names) == 52
    for name, group, old, new in MUTATIONS:
        assert group in FIRST and old != new, name
        assert old in src, name


def _run_pins(scratch, source, files):
    with open(os.path.join(scratch, "oracle", "pget_oracle.c"), "w") as fh:
        fh.write(source)
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    # the source must compile: a build error is not a caught mistake
    b = subprocess.run([sys.executable, "-c", "from oracle import oracle as O; O.build(force=True)"],
                       cwd=scratch, env=env, capture_output=True, text=True, timeout=300)
    assert b.returncode == 0, b.stderr[-2000:]
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu"]
                          + [os.path.join("tests", f) for f in files],
                          cwd=scratch, env=env, capture_output=True, text=True, timeout=900)


@pytest.mark.slow
def test_unmodified_copy_passes_every_pin(scratch):
    """The control: the scratch copy itself is sound, so a failure below is the mistake's."""
    t = _run_pins(scratch, open(SRC).read(), PIN_FILES)
    assert t.returncode == 0, t.stdout[-2000:]


@pytest.mark.slow
@pytest.mark.parametrize("name", [m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(scratch, name):
    _, group, old, new = next(m for m in MUTATIONS if m[0] == name)
    files = FIRST[group] + [f for f in PIN_FILES if f not in FIRST[group]]
    t = _run_pins(scratch, open(SRC).read().replace(old, new, 1), files)
    assert t.returncode == 1, f"{name}: not caught (pytest exit {t.returncode})\n{t.stdout[-1500:]}"
