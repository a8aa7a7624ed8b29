"""Planted mistakes in the oracle must fail one of its pins.

Each case copies the oracle, the input generators and one pin file into a
temporary directory, plants one plausible mistake in the copy of the oracle
(a dropped term, a wrong sign, index or factor, a transposed operand) and
runs that pin file there: it has to report a failing test. The repository's
own oracle is never modified.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

FWI = [
    ("taper_prev", "a_next = g * (2.0 * a + w * lap) - g * g * a_prev",
     "a_next = g * (2.0 * a + w * lap) - g * a_prev"),
    ("centre_coefficient", "out = 2.0 * C8[0] * u", "out = C8[0] * u"),
    ("source_scale", "geom.f0, geom.t0) / geom.dx ** 2", "geom.f0, geom.t0) / geom.dx"),
    ("adjoint_w_outside", "lk = 2.0 * g * lam1 + laplacian(w * g * lam1, geom.dx)",
     "lk = 2.0 * g * lam1 + w * g * laplacian(lam1, geom.dx)"),
    ("gradient_factor", "gpad1 = 2.0 * vpad * geom.dt ** 2 * acc1",
     "gpad1 = vpad * geom.dt ** 2 * acc1"),
    ("fold_shift", "iz = np.clip(np.arange(geom.NZ) - nb, 0, geom.nz - 1)",
     "iz = np.clip(np.arange(geom.NZ) - nb + 1, 0, geom.nz - 1)"),
    ("record_early", "traces[:, n] = a_next[rz, rx]", "traces[:, n] = a[rz, rx]"),
    ("ricker", "return (1.0 - 2.0 * a) * np.exp(-a)", "return (1.0 - a) * np.exp(-a)"),
    ("taper_profile", "into = np.maximum(np.maximum(nb - i, i - (N - 1 - nb)), 0)",
     "into = np.maximum(np.maximum(nb - i - 1, i - (N - 1 - nb)), 0)"),
    ("adjoint_taper", "- g * g * lam2 + rho", "- g * lam2 + rho"),
    ("imaging_taper", "term = g * lam[n + 1] * src_term", "term = lam[n + 1] * src_term"),
    ("magnitude_abs", "accm += np.abs(term)", "accm += term"),
]
SVGD = [
    ("bandwidth_log", "return med / (2.0 * np.log(n + 1.0))", "return med / (2.0 * np.log(n))"),
    ("rbf_factor", "return np.exp(-D2 / (2.0 * h2))", "return np.exp(-D2 / h2)"),
    ("repulsion_sign", "(K[i][:, None] * (X[i][None, :] - X)).sum(axis=0) / h2",
     "(K[i][:, None] * (X - X[i][None, :])).sum(axis=0) / h2"),
    ("mean", "return (attract + repulse) / n, h2, K", "return (attract + repulse), h2, K"),
    ("log_jacobian", "* (b - a) * s * (1.0 - s) + (1.0 - 2.0 * s)", "* (b - a) * s * (1.0 - s)"),
    ("inverse_transform", "return a + (b - a) / (1.0 + np.exp(-theta))",
     "return a + (b - a) / (1.0 + np.exp(theta))"),
]
SSVGD_NOISE = ("noise = np.sqrt(2.0 * eps / n) * (L @ np.asarray(xi, dtype=np.float64))\n"
               "    return clip(X + eps * phi + noise, lo, hi), h2u, tau")
SVGD += [
    ("rows_noise_transposed", "np.stack([L[i] @ xi for i in rows])",
     "np.stack([L[:, i] @ xi for i in rows])"),
    ("rows_attraction_shift", "attract = K[i] @ G ", "attract = K[i][:-1] @ G[1:] "),
    ("noise_scale", SSVGD_NOISE, SSVGD_NOISE.replace("np.sqrt(2.0 * eps / n)", "np.sqrt(eps / n)")),
    ("noise_transposed", SSVGD_NOISE, SSVGD_NOISE.replace("(L @", "(L.T @")),
]
ADVI = [
    ("entropy", "grad_omega = (g * eta * np.exp(omega)[None, :]).mean(axis=0) + 1.0",
     "grad_omega = (g * eta * np.exp(omega)[None, :]).mean(axis=0)"),
    ("omega_chain", "grad_omega = (g * eta * np.exp(omega)[None, :]).mean(axis=0) + 1.0",
     "grad_omega = (g * eta).mean(axis=0) + 1.0"),
    ("log_jacobian", "g = gm * (b - a)[None, :] * s * (1.0 - s) + (1.0 - 2.0 * s)",
     "g = gm * (b - a)[None, :] * s * (1.0 - s)"),
    ("adam_bias", "mhat = m1 / (1.0 - BETA1 ** t)", "mhat = m1"),
    ("adam_sign", "return p + lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m1, m2",
     "return p - lr * mhat / (np.sqrt(vhat) + ADAM_EPS), m1, m2"),
    ("adadelta_eps", "dx = np.sqrt(edx2 + ADADELTA_EPS) / np.sqrt(eg2 + ADADELTA_EPS) * grad",
     "dx = np.sqrt(edx2 + ADADELTA_EPS) / np.sqrt(eg2) * grad"),
    ("adagrad_square", "acc = acc + grad * grad", "acc = acc + np.abs(grad)"),
    ("lowrank_B_entropy", "grad_B = g.T @ eps / S + Sinv @ B", "grad_B = g.T @ eps / S"),
]
TOMO = [
    ("two_sided_root", "np.sqrt(2.0 * f * f - (hi - lo) ** 2)",
     "np.sqrt(f * f - (hi - lo) ** 2 + 1e-300)"),
    ("one_sided_branch", "if hi - lo >= f:", "if True:"),
    ("ray_axes_swapped", "g = np.array([_bilinear(gy, *p), _bilinear(gx, *p)])",
     "g = np.array([_bilinear(gx, *p), _bilinear(gy, *p)])"),
    ("gradient_sign", "grad = -h * Ksum / (v * v)", "grad = h * Ksum / (v * v)"),
    ("gradient_power", "grad = -h * Ksum / (v * v)", "grad = -h * Ksum / v"),
    ("bilinear_weight", "K[i0, j0 + 1] += L * (1 - fy) * fx", "K[i0, j0 + 1] += L * fy * (1 - fx)"),
    ("ray_uphill", "q = p - ds * g / n", "q = p + ds * g / n"),
    ("pair_index", "return s * ns - s * (s + 1) // 2 + (r - s - 1)",
     "return s * ns - s * (s - 1) // 2 + (r - s - 1)"),
]

CASES = ([("fwi.py", "test_oracle_fwi.py") + m for m in FWI] +
         [("svgd.py", "test_oracle_svgd.py") + m for m in SVGD] +
         [("advi.py", "test_oracle_advi.py") + m for m in ADVI] +
         [("tomo.py", "test_oracle_tomo.py") + m for m in TOMO])


def _run_pins(tmp_path, pins, module=None, old=None, new=None):
    """Run one pin file against a copy of the oracle (optionally with one
    line replaced); returns pytest's exit code and the end of its output."""
    shutil.copytree(os.path.join(ROOT, "oracle"), tmp_path / "oracle",
                    ignore=shutil.ignore_patterns("__pycache__", "_build"))
    shutil.copytree(os.path.join(ROOT, "synth"), tmp_path / "synth",
                    ignore=shutil.ignore_patterns("__pycache__"))
    (tmp_path / "tests").mkdir()
    for f in ("conftest.py", pins):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    if module is not None:
        target = tmp_path / "oracle" / module
        src = target.read_text()
        assert src.count(old) >= 1, "the planted line is no longer in the oracle"
        target.write_text(src.replace(old, new, 1))
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    env.pop("PYTHONPATH", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join("tests", pins)], cwd=tmp_path, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


@pytest.mark.parametrize("module,pins,name,old,new", CASES,
                         ids=["%s-%s" % (c[0][:-3], c[2]) for c in CASES])
def test_planted_mistake_fails_a_pin(tmp_path, module, pins, name, old, new):
    code, out = _run_pins(tmp_path, pins, module, old, new)
    # exit code 1: tests ran and at least one failed (not a collection error)
    assert code == 1, (name, code, out)


@pytest.mark.parametrize("pins", ["test_oracle_fwi.py", "test_oracle_svgd.py",
                                  "test_oracle_advi.py", "test_oracle_tomo.py"])
def test_unmodified_copy_passes(tmp_path, pins):
    # the control: the same harness on an untouched copy reports success
    code, out = _run_pins(tmp_path, pins)
    assert code == 0, out
