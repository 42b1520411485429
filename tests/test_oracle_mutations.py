"""Mistakes planted in a copy of the oracle, on the CPU: every one must fail a pin
(tests/test_oracle_pins.py for the lattice Boltzmann oracle, tests/test_mlp_oracle.py for
the FP64 network), so that the pins would catch it in the oracle itself.

Each case copies oracle/, workloads/ and the pins into a scratch directory, changes
one line of the source (the change must apply exactly once), rebuilds the copy and
runs the pins against it in a separate process.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("wall gradient of the wetting ghosts with the wrong sign (Sec. 2.2)",
     "out[jy][jx] = raw[1 - dy][1] - 2.0 * h;", "out[jy][jx] = raw[1 - dy][1] + 2.0 * h;"),
    ("xy weights of Eq. (equilibrium) on the wrong diagonals",
     "static const double WXY[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.25, 0.25, -0.25, -0.25};",
     "static const double WXY[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.25, -0.25, 0.25, -0.25};"),
    ("lambda term of Eq. (equilibrium) without its u . grad rho trace",
     "lambda * (u[a] * dr[b] + u[b] * dr[a] + (a == b ? udr : 0.0))", "lambda * (u[a] * dr[b] + u[b] * dr[a])"),
    ("binary pressure without -kappa phi lap phi (Sec. 3.1)",
     "const double P0 = p0 - p->kappa * ph * s->plap[k];", "const double P0 = p0;"),
    ("g^eq with M mu instead of 2 M mu (App. A)", "double s = 2.0 * Mob * mu;", "double s = Mob * mu;"),
    ("no rest rule at boundary nodes (Sec. 2.2)", "if (s->bnd[k]) rest_node(s->ft + 9 * (size_t)k);", "(void)0;"),
    ("a wrong row of M (App. A)", "{0, 1, -1, 0, 0, 1, -1, -1, 1},", "{0, 1, -1, 0, 0, 1, -1, 1, -1},"),
    ("Eq. (nu) interpolated in the square of (phi + 1)/2 (right only at phi = +-1)",
     "double c = 0.5 * (phi + 1.0);", "double c = 0.25 * (phi + 1.0) * (phi + 1.0);"),
    ("liquid-gas l(t) threshold at rho_l / 2 instead of (rho_l + rho_g) / 2 (Sec. 1)",
     "const double thr = p->model == 0 ? 0.5 * (p->rho_l + p->rho_g) : 0.0;",
     "const double thr = p->model == 0 ? 0.5 * p->rho_l : 0.0;"),
    ("liquid-gas liquid fraction measured from rho_l instead of rho_g",
     "vol += p->model == 0 ? (q - p->rho_g) / (p->rho_l - p->rho_g) : 0.5 * (q + 1.0);",
     "vol += p->model == 0 ? (p->rho_l - q) / (p->rho_l - p->rho_g) : 0.5 * (q + 1.0);"),
]


def run_pins(tmp_path, mutate=None, source="lb_oracle.c", pins="test_oracle_pins.py"):
    """Copy the oracle and its pins to tmp_path, apply mutate to one oracle source, run the pins."""
    for d in ("oracle", "workloads"):
        shutil.copytree(os.path.join(ROOT, d), tmp_path / d,
                        ignore=shutil.ignore_patterns("*.so", "*.tmp", "__pycache__"))
    (tmp_path / "tests").mkdir()
    for f in (pins, "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    if mutate:
        src = tmp_path / "oracle" / source
        src.write_text(mutate(src.read_text()))
    return subprocess.run([sys.executable, "-m", "pytest", "tests/" + pins, "-x", "-q", "-p",
                           "no:cacheprovider"], cwd=tmp_path, capture_output=True, text=True, timeout=900,
                          env={**os.environ, "PYTHONPATH": str(tmp_path)})


def test_unchanged_copy_passes_the_pins(tmp_path):
    """The control: the scratch copy itself passes, so a failure below is the mistake's."""
    r = run_pins(tmp_path)
    assert r.returncode == 0, r.stdout[-800:]


@pytest.mark.parametrize("what,old,new", MUTATIONS, ids=[m[0][:40] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, what, old, new):
    def mutate(text):
        assert text.count(old) == 1, f"mutation no longer applies: {what}"
        return text.replace(old, new)
    r = run_pins(tmp_path, mutate)
    assert r.returncode != 0 and " failed" in r.stdout, f"no pin caught: {what}\n{r.stdout[-800:]}"


MLP_MUTATIONS = [
    ("tanh derivative without the square", "dz2 = (dy @ W3) * (1.0 - h2 * h2)", "dz2 = (dy @ W3) * (1.0 - h2)"),
    ("loss gradient without its factor 2", "dy = 2.0 * d / (n * nout)", "dy = d / (n * nout)"),
    ("transposed W2 in the backward pass", "dz1 = (dz2 @ W2) * (1.0 - h1 * h1)", "dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)"),
    ("output-bias gradient averaged over rows", "gb3 = dy.sum(0)", "gb3 = dy.mean(0)"),
    ("first-layer gradient from the wrong activations", "gW1 = dz1.T @ x", "gW1 = dz1.T @ np.tanh(x)"),
]


@pytest.mark.parametrize("what,old,new", MLP_MUTATIONS, ids=[m[0][:40] for m in MLP_MUTATIONS])
def test_planted_mistake_in_the_network_reference_fails_a_pin(tmp_path, what, old, new):
    def mutate(text):
        assert text.count(old) == 1, f"mutation no longer applies: {what}"
        return text.replace(old, new)
    r = run_pins(tmp_path, mutate, source="mlp.py", pins="test_mlp_oracle.py")
    assert r.returncode != 0 and " failed" in r.stdout, f"no pin caught: {what}\n{r.stdout[-800:]}"
