"""The oracle's pins have teeth: each plausible slip in the FP64 C oracle
(a transposed index, a dropped factor, a flipped sign, an off-by-one window,
the wrong rounding, a missed state update) is planted in a copy of
esim_oracle.c on the CPU, the copy is compiled, and the pins of
test_oracle_pins.py run against it in a child process through
ESIM_ORACLE_LIB.  Every mutant must make them fail; the unmutated copy built
the same way must pass them, so a failure means the mutation, not the
mechanism.  Nothing here touches a GPU or the library.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

# (what the slip is, the text it replaces, the slipped text); each original
# text occurs exactly once in esim_oracle.c
MUTANTS = [
    ("luminance weights on the wrong channels",
     "0.7152 * radiance[n + p]", "0.7152 * radiance[2 * n + p]"),
    ("log epsilon dropped",
     "y[p] = log(Y + c->log_eps);", "y[p] = log(Y);"),
    ("Gaussian exponent without the 1/2 (Eq. 5)",
     "double w = exp(-0.5 * u);", "double w = exp(-u);"),
    ("feature difference with the sign flipped",
     "d[2 + j] = ring_x(s, tau, j, q) - xcen[j];", "d[2 + j] = xcen[j] - ring_x(s, tau, j, q);"),
    ("coordinate offset not divided by r",
     "d[0] = (qx - cx) / unit;", "d[0] = (qx - cx);"),
    ("dy regressor built from the x offset",
     "d[1] = (qy - cy) / unit;", "d[1] = (qx - cx) / unit;"),
    ("feature bandwidths ignored",
     "hb[2 + j] = c->h * c->bandwidth[j];", "hb[2 + j] = c->h;"),
    ("temporal window one frame too long",
     "int32_t tau0 = t - c->frames + 1;", "int32_t tau0 = t - c->frames;"),
    ("ridge not scaled by the weight sum W",
     "double sr = sqrt(c->ridge * W);", "double sr = sqrt(c->ridge);"),
    ("ridge applied to the intercept too",
     "for (int k = 1; k < NP; ++k) {\n            for (int q = 0; q < NP; ++q) a[rows * NP + q]",
     "for (int k = 0; k < NP; ++k) {\n            for (int q = 0; q < NP; ++q) a[rows * NP + q]"),
    ("residual R not normalised by W (Eq. 7)",
     "*R_out = R / W;", "*R_out = R;"),
    ("Proposition 1 reads the wrong slopes",
     "st += s->beta[p * ND + 2 + j] * (s->xc[p * NF + j] - xnow[j]);",
     "st += s->beta[p * ND + 1 + j] * (s->xc[p * NF + j] - xnow[j]);"),
    ("crossings rounded instead of floored (Eq. 1)",
     "double k = floor(fabs(dl) / C);", "double k = round(fabs(dl) / C);"),
    ("brightness reference reset to alpha instead of moved by p n C",
     "s->l_last[p] += pol * k * C;", "s->l_last[p] = theta[0];"),
    ("model not replaced at an event",
     "                for (int j = 0; j < ND; ++j) s->beta[p * ND + j] = theta[1 + j];\n"
     "                for (int j = 0; j < NF; ++j) s->xc[p * NF + j] = xnow[j];\n            }\n        }",
     "            }\n        }"),
    ("model replaced at every regression, not only at events",
     "            if (k >= 1.0) {\n                int32_t pol",
     "            for (int j = 0; j < ND; ++j) s->beta[p * ND + j] = theta[1 + j];\n"
     "            for (int j = 0; j < NF; ++j) s->xc[p * NF + j] = xnow[j];\n"
     "            if (k >= 1.0) {\n                int32_t pol"),
    ("Proposition 1 compares the stored feature with itself",
     "(s->xc[p * NF + j] - xnow[j])", "(s->xc[p * NF + j] - s->xc[p * NF + j])"),
    ("event polarity inverted",
     "int32_t pol = dl > 0 ? 1 : -1;", "int32_t pol = dl > 0 ? -1 : 1;"),
    ("event x and y swapped",
     "push_event(s, t, (int32_t)(p % W), (int32_t)(p / W), pol)",
     "push_event(s, t, (int32_t)(p / W), (int32_t)(p % W), pol)"),
    ("Householder reflection with factor 1 instead of 2",
     "double f = 2.0 * dot / vtv;\n            for (int64_t i = k; i < m; ++i) a[i * NP + c]",
     "double f = dot / vtv;\n            for (int64_t i = k; i < m; ++i) a[i * NP + c]"),
]


def _build(tmp, source, name):
    d = tmp / name
    d.mkdir()
    shutil.copy(os.path.join(ORACLE, "esim_oracle.h"), d / "esim_oracle.h")
    (d / "esim_oracle.c").write_text(source)
    lib = d / "liboracle.so"
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", str(lib),
                           str(d / "esim_oracle.c"), "-lm"])
    return str(lib)


def _pins(lib):
    env = dict(os.environ, ESIM_ORACLE_LIB=lib, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr).strip().splitlines()[-1:]


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(ORACLE, "esim_oracle.c")) as f:
        return f.read()


def test_unmutated_copy_passes_the_pins(tmp_path, source):
    rc, tail = _pins(_build(tmp_path, source, "original"))
    assert rc == 0, tail


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(tmp_path, source, what, old, new):
    assert source.count(old) == 1, f"mutation site not unique or missing: {what}"
    rc, tail = _pins(_build(tmp_path, source.replace(old, new), "mutant"))
    assert rc != 0, f"the pins did not catch: {what}"
