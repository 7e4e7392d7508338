"""The oracle's pins catch plausible mistakes.  Each case plants one mistake
(a dropped term, a wrong sign, factor, index order or rounding) in a copy of
the oracle, on the CPU, and runs the pins that cover that function against the
copy: at least one of them must fail.  The oracle itself is never modified."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what goes wrong, text in oracle/uot_oracle.py, the planted text, pins that cover it)
PLANTS = [
    ("KL row exponent", "U = (F.lam / (F.lam + eps)) * ubar", "U = (F.lam / (F.lam + 2 * eps)) * ubar",
     "prox_rows_brute_force or one_point_kl"),
    ("TV clamp", "U = np.clip(ubar, -F.lam, F.lam)", "U = np.clip(ubar, -2 * F.lam, F.lam)",
     "prox_rows_brute_force or one_point_piecewise"),
    ("sign of S in the update", "eps * np.where(p_zero, 0.0, logp) - S_f", "eps * np.where(p_zero, 0.0, logp) + S_f",
     "prox_rows_brute_force"),
    ("Gibbs weights dropped", "L = V / eps + np.asarray(logw, dtype=np.float64)", "L = V / eps",
     "gibbs_operator_matches_definition"),
    ("barycenter weight normalisation", "(lse(Z, axis=0) - math.log(np.sum(alpha)))", "(lse(Z, axis=0))",
     "barycenter"),
    ("WF cost: cos not squared", "np.log(np.cos(np.minimum(d, math.pi / 2)) ** 2)",
     "np.log(np.cos(np.minimum(d, math.pi / 2)))", "wf_cost_closed_forms"),
    ("growth: per-species T", "Ttot = eps * lse(T / eps, axis=0)", "Ttot = T[0]",
     "growth_prox_two_species"),
    ("growth: lam dropped", "-lam * Ttot / (lam + eps))", "-Ttot / (lam + eps))", "growth_prox"),
    ("bins: round for floor", "k = np.floor(P[:, a] * np.float32(n))", "k = np.round(P[:, a] * np.float32(n))",
     "bin_index or color_histogram"),
    ("mass: U - S", "np.asarray(logdx) + (U + S) / eps", "np.asarray(logdx) + (U - S) / eps", "mass_update"),
    ("mass: dx dropped", "np.asarray(logdx) + (U + S) / eps", "0.0 + (U + S) / eps", "mass_update"),
    ("eps stages: one too many in the ratio", "rho = (eps_start / eps_final) ** (1.0 / stages)",
     "rho = (eps_start / eps_final) ** (1.0 / (stages + 1))", "eps_schedule"),
    ("grid points column-major", 'indexing="ij"', 'indexing="xy"', "grid_axes"),
    ("bin centres", "(np.arange(n, dtype=np.float64) + 0.5) / n", "(np.arange(n, dtype=np.float64) + 0.5) / (n + 1)",
     "grid_axes"),
    ("growth: tau alpha for 2 tau alpha", "c = 1.0 - 2.0 * tau * alpha / lam", "c = 1.0 - tau * alpha / lam",
     "growth_c"),
    ("streamed operator: weights dropped",
     "L = np.asarray(V, dtype=np.float64) / eps + np.asarray(logw, dtype=np.float64)",
     "L = np.asarray(V, dtype=np.float64) / eps", "streamed"),
    ("violation relative to the current marginal", "den = np.sum(w * np.exp(lt))", "den = np.sum(w * np.exp(lr))",
     "violation_measure"),
    ("Algorithm 4: Z dropped from the a-update", "Sz = np.where(np.isneginf(S), NEG_INF, S + Z)", "Sz = S",
     "alg4"),
    ("Algorithm 4: Z dropped from the b-update", "Tz = np.where(np.isneginf(T), NEG_INF, T + Z)", "Tz = T",
     "alg4"),
    ("next density per species", "return R2 / np.maximum(c, np.sum(R2, axis=0))", "return R2 / np.maximum(c, R2)",
     "growth_next_density"),
    ("next log density per species", "tot = np.sum(np.exp(logR2), axis=0)", "tot = np.exp(logR2)",
     "growth_next or wf_step"),
    ("WF step: U for V in r2", "logr2 = np.where(np.isneginf(T), NEG_INF, (V + T) / eps)",
     "logr2 = np.where(np.isneginf(T), NEG_INF, (U + T) / eps)", "wf_step"),
    ("colour: dy weights dropped", "w = np.ravel(np.asarray(dy, dtype=np.float64))",
     "w = np.ones(np.size(dy))", "barycentric_projection"),
    ("colour: empty rows sent to 0", "return np.where(den[:, None] > 0, T, X)",
     "return np.where(den[:, None] > 0, T, 0.0)", "barycentric_projection"),
    ("translation: sign of the shift", "return U + c, V - c", "return U - c, V + c", "translation"),
    ("translation: one-sided lambda weight", "F1.lam * F2.lam / (F1.lam + F2.lam) * (la - lb)",
     "0.5 * F1.lam * (la - lb)", "translation"),
    ("translation: dx weights dropped", "ta = np.ravel(logdx + logp)", "ta = np.ravel(0.0 * logdx + logp)",
     "translation"),
]


# The same for the warm-start network's reference (oracle/net_oracle.py) and
# its pins (tests/test_net_oracle.py): brute-force convolution, closed-form and
# finite-difference gradients.
NET_PLANTS = [
    ("conv: taps flipped", "sl = xp[:, :, kh * dil:kh * dil + H, kw * dil:kw * dil + W]",
     "sl = xp[:, :, (2 - kh) * dil:(2 - kh) * dil + H, (2 - kw) * dil:(2 - kw) * dil + W]",
     "brute_force"),
    ("conv: leak slope", "LEAK = 0.1", "LEAK = 0.2", "brute_force"),
    ("conv: bias dropped", "y = np.zeros((N, Cout, H, W)) + np.asarray(b, dtype=np.float64)[None, :, None, None]",
     "y = np.zeros((N, Cout, H, W))", "brute_force or closed_form"),
    ("conv: padding of one for every dilation", "    pad = dil\n    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad))\n"
     "    xp[:, :, pad:pad + H, pad:pad + W] = x\n    y = ",
     "    pad = 1\n    xp = np.zeros((N, Cin, H + 2 * pad, W + 2 * pad))\n"
     "    xp[:, :, pad:pad + H, pad:pad + W] = x\n    y = ", "brute_force"),
    ("data gradient: gradient not shifted back",
     "gs = gp[:, :, (2 - kh) * dil:(2 - kh) * dil + H, (2 - kw) * dil:(2 - kw) * dil + W]",
     "gs = gp[:, :, kh * dil:kh * dil + H, kw * dil:kw * dil + W]", "conv2d_grads"),
    ("weight gradient: tap flipped", 'dw[:, :, kh, kw] = np.einsum("nohw,nchw->oc", g, xs)',
     'dw[:, :, 2 - kh, 2 - kw] = np.einsum("nohw,nchw->oc", g, xs)', "conv2d_grads"),
    ("bias gradient over the channels", "return dx, dw, g.sum(axis=(0, 2, 3))",
     "return dx, dw, g.sum(axis=(1, 2, 3))[: g.shape[1]]", "conv2d_grads"),
    ("finite difference: one-sided step", "return (lp - lm) / (2 * h)", "return (lp - lm) / h", "closed_form"),
]


def _copy_tree(dst):
    """The oracle, its pins and the seeded input generator, nothing else."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    os.makedirs(os.path.join(dst, "paper_1607_05816_gb300"))
    for rel in ("pytest.ini", os.path.join("tests", "conftest.py"), os.path.join("tests", "test_oracle_pins.py"),
                os.path.join("tests", "test_net_oracle.py"),
                os.path.join("paper_1607_05816_gb300", "__init__.py"),
                os.path.join("paper_1607_05816_gb300", "synth.py")):
        shutil.copy(os.path.join(ROOT, rel), os.path.join(dst, rel))


@pytest.mark.parametrize("what,orig,planted,pins", PLANTS, ids=[p[0] for p in PLANTS])
def test_planted_mistake_is_caught(tmp_path, what, orig, planted, pins):
    _copy_tree(str(tmp_path))
    path = os.path.join(str(tmp_path), "oracle", "uot_oracle.py")
    src = open(path).read()
    assert src.count(orig) >= 1, f"the oracle no longer contains the text of plant '{what}'"
    open(path, "w").write(src.replace(orig, planted, 1))
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-x", "-k", pins],
                         cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    # exit code 1: tests ran and at least one failed (2-5 would be usage, import or collection errors)
    assert out.returncode == 1, f"plant '{what}' not caught:\n{out.stdout[-1500:]}{out.stderr[-1500:]}"


def test_unplanted_copy_passes_the_same_pins(tmp_path):
    """Control: the copy without a plant passes every pin the cases select,
    so each failure above is the plant's."""
    _copy_tree(str(tmp_path))
    sel = " or ".join(sorted({p[3] for p in PLANTS}))
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "-q", "-k", sel],
                         cwd=str(tmp_path), capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]


@pytest.mark.parametrize("what,orig,planted,pins", NET_PLANTS, ids=[p[0] for p in NET_PLANTS])
def test_planted_network_mistake_is_caught(tmp_path, what, orig, planted, pins):
    _copy_tree(str(tmp_path))
    path = os.path.join(str(tmp_path), "oracle", "net_oracle.py")
    src = open(path).read()
    assert src.count(orig) >= 1, f"the network oracle no longer contains the text of plant '{what}'"
    open(path, "w").write(src.replace(orig, planted, 1))
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_net_oracle.py", "-q", "-x", "-k", pins],
                         cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert out.returncode == 1, f"plant '{what}' not caught:\n{out.stdout[-1500:]}{out.stderr[-1500:]}"


def test_unplanted_network_copy_passes_the_same_pins(tmp_path):
    _copy_tree(str(tmp_path))
    sel = " or ".join(sorted({p[3] for p in NET_PLANTS}))
    out = subprocess.run([sys.executable, "-m", "pytest", "tests/test_net_oracle.py", "-q", "-k", sel],
                         cwd=str(tmp_path), capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-2000:]
