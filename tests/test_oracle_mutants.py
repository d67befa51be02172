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




# ---------------------------------------------------------------- numpy oracles
# The second-order, evaluation and renderer oracles and the differentiation
# form's FP64 reference are Python modules: a mutated copy replaces the module
# in a child pytest run (a plugin loads it under the module's name before the
# pins are collected).

PY_MUTANTS = {
    "render": ("test_render_pins.py", [
        ("geometry term without 1/pi",
         "g = ((cs * cl) * area) / (f32(3.14159274) * d2)", "g = ((cs * cl) * area) / d2"),
        ("geometry term without the light's cosine",
         "g = ((cs * cl) * area) / (f32(3.14159274) * d2)", "g = (cs * area) / (f32(3.14159274) * d2)"),
        ("light sampled on the floor plane",
         "np.full(n_pix, f32(sc.box[1]), f32)", "np.full(n_pix, f32(-sc.box[1]), f32)"),
        ("image rows flipped",
         "syp = (f32(1.0) - ((py + _unit(jit[1])) / f32(H)) * f32(2.0)) * tany",
         "syp = (((py + _unit(jit[1])) / f32(H)) * f32(2.0) - f32(1.0)) * tany"),
        ("variance of the mean divided by n^2 instead of n (n - 1)",
         "/ (nf * (nf - f32(1.0)))", "/ (nf * nf)"),
        ("path throughput not attenuated by the albedo",
         "thr = [thr[c] * a[c] for c in range(3)]", "thr = [thr[c] for c in range(3)]"),
        ("floor and ceiling normals swapped",
         "nwy = [0, 0, 1, -1, 0]", "nwy = [0, 0, -1, 1, 0]"),
        ("directly seen emitter at half radiance",
         "L[c] = np.where(alive & light, L[c] + Le[c], L[c])",
         "L[c] = np.where(alive & light, L[c] + f32(0.5) * Le[c], L[c])"),
        ("bounce radius uz instead of sqrt(uz)",
         "rr = np.sqrt(uz)", "rr = uz"),
        ("bounce directions uniform in solid angle instead of cosine-weighted",
         "rr = np.sqrt(uz)\n    lz = np.sqrt(np.maximum(f32(1.0) - uz, f32(0.0)))",
         "rr = np.sqrt(np.maximum(f32(1.0) - (f32(1.0) - uz) * (f32(1.0) - uz), f32(0.0)))\n"
         "    lz = f32(1.0) - uz"),
        ("tangent basis with the wrong sign",
         "aa = f32(-1.0) / (sg + n[2])", "aa = f32(1.0) / (sg + n[2])"),
    ]),
    "wlr_reference": ("test_adjoint_pins.py", [
        ("sqrt(w) with the Gaussian's full exponent",
         "sw = torch.exp(-0.25 * (((d / hb.view(9, 1, 1)) ** 2).sum(0))) * valid[sl]",
         "sw = torch.exp(-0.5 * (((d / hb.view(9, 1, 1)) ** 2).sum(0))) * valid[sl]"),
        ("coordinate offset not divided by r",
         "d[0] = ox / r", "d[0] = ox"),
        ("normal-equation ridge not scaled by W",
         "+ ridge * wv.sum(-1)[..., None, None] * P", "+ ridge * P"),
        ("least-squares ridge rows not scaled by W",
         "torch.sqrt(ridge * Wsum)[..., None, None]", "torch.sqrt(ridge + 0 * Wsum)[..., None, None]"),
        ("temporal window one frame too long",
         "for tau in range(max(0, t - T + 1), t + 1):", "for tau in range(max(0, t - T), t + 1):"),
        ("clipped offsets not masked",
         "** 2).sum(0))) * valid[sl]", "** 2).sum(0)))"),
        ("loss summed instead of averaged",
         "return ((alpha - log_luminance(clean, eps)) ** 2).mean()",
         "return ((alpha - log_luminance(clean, eps)) ** 2).sum()"),
        ("Rec.709 weights on the wrong channels",
         "REC709 = (0.2126, 0.7152, 0.0722)", "REC709 = (0.0722, 0.7152, 0.2126)"),
    ]),
    "wlr2": ("test_wlr2_pins.py", [
        ("squares d_a^2 left out of the quadratic terms",
         "PAIRS = [(a, b) for a in range(ND) for b in range(a, ND)]",
         "PAIRS = [(a, b) for a in range(ND) for b in range(a + 1, ND)]"),
        ("linear terms left out of the design row",
         "np.ones(d.shape[:-1] + (1,)), d, quad", "np.ones(d.shape[:-1] + (1,)), 0 * d, quad"),
        ("Gaussian exponent without the 1/2 (Eq. 5)",
         "w = np.exp(-0.5 * np.sum((d / hb) ** 2, axis=-1)) * valid",
         "w = np.exp(-np.sum((d / hb) ** 2, axis=-1)) * valid"),
        ("clipped neighbours not masked out",
         "w = np.exp(-0.5 * np.sum((d / hb) ** 2, axis=-1)) * valid",
         "w = np.exp(-0.5 * np.sum((d / hb) ** 2, axis=-1))"),
        ("temporal window one frame too long",
         "taus = np.arange(t - frames + 1, t + 1)", "taus = np.arange(t - frames, t + 1)"),
        ("coordinate offset not divided by r",
         "d[..., 0] = (qx - cx[:, None]) / radius", "d[..., 0] = (qx - cx[:, None])"),
        ("dy regressor built from the x offset",
         "d[..., 1] = (qy - cy[:, None]) / radius", "d[..., 1] = (qx - cx[:, None]) / radius"),
        ("ridge not scaled by the weight sum W",
         "np.sqrt(ridge * W)[:, None]", "np.sqrt(ridge)"),
        ("ridge on the intercept instead of the last coefficient",
         "ridge_rows[:, np.arange(NZ - 1), np.arange(1, NZ)]",
         "ridge_rows[:, np.arange(NZ - 1), np.arange(0, NZ - 1)]"),
        ("luminance weights on the wrong channels",
         "LUMA = np.array([0.2126, 0.7152, 0.0722])", "LUMA = np.array([0.2126, 0.0722, 0.7152])"),
        ("log epsilon dropped",
         "return np.log(Y + log_eps)", "return np.log(Y)"),
        ("feature bandwidths ignored",
         "hb = np.array([h, h] + [h * float(b) for b in bandwidth])", "hb = np.array([h, h] + [h for b in bandwidth])"),
        ("back substitution against the wrong column",
         "R[:NZ, :NZ], R[:NZ, NZ])", "R[:NZ, :NZ], R[:NZ, NZ - 1])"),
        ("listed centres read as (t, x, y)",
         "cen[k, 2], cen[k, 1], radius, frames)", "cen[k, 1], cen[k, 2], radius, frames)"),
    ]),
    "quality": ("test_quality_pins.py", [
        ("events matched against the opposite polarity",
         "r, _ = event_points(ref_counts, p)", "r, _ = event_points(ref_counts, -p)"),
        ("time axis not normalised by F",
         "pts = np.stack([x / W, y / H, t / F], axis=1)", "pts = np.stack([x / W, y / H, t], axis=1)"),
        ("x and y normalised by the wrong sides",
         "pts = np.stack([x / W, y / H, t / F], axis=1)", "pts = np.stack([x / H, y / W, t / F], axis=1)"),
        ("ESIM crossings rounded instead of floored",
         "n = np.floor(np.abs(dl) / C).astype(np.int64)", "n = np.round(np.abs(dl) / C).astype(np.int64)"),
        ("ESIM reference reset to the frame instead of moved by p n C",
         "return counts, l_last + counts * C", "return counts, y.copy()"),
        ("event multiplicities ignored",
         "return pts, np.abs(counts[sel]).astype(np.int64)", "return pts, np.ones(len(pts), np.int64)"),
        ("F-score without the factor 2",
         "Fs.append(2 * p * r / (p + r) if p + r > 0 else 0.0)", "Fs.append(p * r / (p + r) if p + r > 0 else 0.0)"),
        ("chamfer distance not squared",
         "cd = (float((wg * dg ** 2).sum()) / ng", "cd = (float((wg * dg).sum()) / ng"),
        ("recall normalised by the generated count",
         "r = float(wr[dr < tau].sum()) / nr if nr else 0.0", "r = float(wr[dr < tau].sum()) / ng if ng else 0.0"),
        ("Rec.709 weights on the wrong channels",
         "REC709 = (0.2126, 0.7152, 0.0722)", "REC709 = (0.7152, 0.2126, 0.0722)"),
    ]),
}

_PLUGIN = '''import importlib, importlib.util, os, sys


def pytest_configure(config):
    name = os.environ["ESIM_MUTANT_MODULE"]
    pkg = importlib.import_module(name.rsplit(".", 1)[0]) if "." in name else None
    spec = importlib.util.spec_from_file_location(name, os.environ["ESIM_MUTANT_FILE"])
    mod = importlib.util.module_from_spec(spec)
    sys.modules[name] = mod
    spec.loader.exec_module(mod)
    if pkg is not None:
        setattr(pkg, name.rsplit(".", 1)[1], mod)
'''


# the differentiation form's FP64 autograd reference is a test module, not
# part of oracle/
TOP_LEVEL = {"wlr_reference": os.path.join(ROOT, "tests", "wlr_reference.py")}


def _py_pins(tmp, module, pins, source):
    (tmp / "esim_mutant_plugin.py").write_text(_PLUGIN)
    path = tmp / f"{module}_copy.py"
    path.write_text(source)
    name = module if module in TOP_LEVEL else f"oracle.{module}"
    env = dict(os.environ, ESIM_MUTANT_MODULE=name, ESIM_MUTANT_FILE=str(path),
               PYTHONPATH=os.pathsep.join([str(tmp)] + [p for p in [os.environ.get("PYTHONPATH")] if p]),
               OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-p", "esim_mutant_plugin",
                        os.path.join(ROOT, "tests", pins), "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, (r.stdout + r.stderr).strip().splitlines()[-1:]


# ---------------------------------------------------------------- the runs
# Every case (each unmutated copy and each mutant) is one child process.  Run
# serially (no xdist worker), the module's first test starts them all, up to
# eight at a time, and each test then reads its own outcome.

def _source(module):
    path = os.path.join(ORACLE, "esim_oracle.c") if module == "c" else \
        TOP_LEVEL.get(module, os.path.join(ORACLE, f"{module}.py"))
    with open(path) as f:
        return f.read()


def _cases():
    out = {("c", None): ("c", _source("c"))}
    for what, old, new in MUTANTS:
        out[("c", what)] = ("c", _source("c").replace(old, new))
    for m, (_, muts) in PY_MUTANTS.items():
        out[(m, None)] = (m, _source(m))
        for what, old, new in muts:
            out[(m, what)] = (m, _source(m).replace(old, new))
    return out


def _run(tmp, module, text):
    if module == "c":
        return _pins(_build(tmp, text, "copy"))
    return _py_pins(tmp, module, PY_MUTANTS[module][0], text)


@pytest.fixture(scope="module")
def outcome(tmp_path_factory):
    cases = _cases()
    done = {}
    if not os.environ.get("PYTEST_XDIST_WORKER"):
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(max_workers=max(2, min(8, os.cpu_count() or 2))) as ex:
            futs = {k: ex.submit(_run, tmp_path_factory.mktemp("case"), *v) for k, v in cases.items()}
            done = {k: f.result() for k, f in futs.items()}

    def get(module, what=None):
        key = (module, what)
        if key not in done:
            done[key] = _run(tmp_path_factory.mktemp("case"), *cases[key])
        return done[key]
    return get


def test_unmutated_copy_passes_the_pins(outcome):
    rc, tail = outcome("c")
    assert rc == 0, tail


@pytest.mark.parametrize("what,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_the_mutant(outcome, what, old, new):
    assert _source("c").count(old) == 1, f"mutation site not unique or missing: {what}"
    rc, tail = outcome("c", what)
    assert rc != 0, f"the pins did not catch: {what}"


@pytest.mark.parametrize("module", sorted(PY_MUTANTS))
def test_unmutated_python_oracle_copy_passes_the_pins(outcome, module):
    rc, tail = outcome(module)
    assert rc == 0, tail


_PY_CASES = [(m, w, o, n) for m in sorted(PY_MUTANTS) for (w, o, n) in PY_MUTANTS[m][1]]


@pytest.mark.parametrize("module,what,old,new", _PY_CASES, ids=[f"{c[0]}: {c[1]}" for c in _PY_CASES])
def test_python_oracle_pins_catch_the_mutant(outcome, module, what, old, new):
    assert _source(module).count(old) == 1, f"mutation site not unique or missing: {what}"
    rc, tail = outcome(module, what)
    assert rc != 0, f"the pins did not catch: {what}"
