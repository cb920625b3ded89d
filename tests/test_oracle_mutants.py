"""Sensitivity of the oracle's pins: copies of the oracle, each with one plausible
mistake planted in its C source (a wrong cost, sign, index, weight or tie-break)
or in one of its Python functions, are built on the CPU, and for every copy at
least one pin of the stage it touches must fail. The C copies live in a temporary
directory; each copy is loaded in place of the oracle only for one check."""
import ctypes  # noqa: F401  (the oracle wrapper loads the copies through ctypes)
import inspect
import itertools
import os
import subprocess
import tempfile

import pytest

import oracle
import test_oracle_cross
import test_oracle_degraf
import test_oracle_epic
import test_oracle_fb
import test_oracle_gm
import test_oracle_pyramid
import test_oracle_rlof

SRC = os.path.join(os.path.dirname(oracle.__file__), "degraf_oracle.c")

# name: (text in the oracle source, its replacement, pin modules that must catch it)
MUTANTS = {
    "detection swaps the negative centroid's coordinates": (
        "double cx = use_neg ? (double)Xn / (double)Sn : (double)X / (double)S;",
        "double cx = use_neg ? (double)Yn / (double)Sn : (double)X / (double)S;", [test_oracle_degraf]),
    "pyramid mean weighs one pixel twice": (
        "I[(long)y * Wl + x] = ((a + b) + (c + d)) * 0.25;", "I[(long)y * Wl + x] = ((a + a) + (c + d)) * 0.25;",
        [test_oracle_pyramid]),
    "pyramid y-gradient uses the x kernel": (
        "gy += sobel_x[dx + 1][dy + 1] * v; /* transposed kernel */",
        "gy += sobel_x[dy + 1][dx + 1] * v; /* transposed kernel */", [test_oracle_pyramid]),
    "tracking keeps points with too little gradient": (
        "if (lam_min / n_keep < R(prm->min_eig)) { status = OR_SMALL_EIG; break; }",
        "if (lam_min / n_keep < R(-prm->min_eig)) { status = OR_SMALL_EIG; break; }", [test_oracle_rlof]),
    "tracking residual adds the offset": (
        "res = J - (1 + m) * T[s] - c;", "res = J - (1 + m) * T[s] + c;", [test_oracle_rlof]),
    "Hampel drops the clipping between its first two knots": (
        "if (ar <= b) return a * s;", "if (ar <= b) return r;", [test_oracle_rlof]),
    "Hampel's descending part spans the wrong interval": (
        "if (ar <= c) return a * s * (c - ar) / (c - b);", "if (ar <= c) return a * s * (c - ar) / (c - a);",
        [test_oracle_rlof]),
    "tracking template sampled half a pixel off in y": (
        "T[s] = bilinear(A->I, A->W, A->H, plx + kx, ply + ky);",
        "T[s] = bilinear(A->I, A->W, A->H, plx + kx, ply + ky + R(0.5));", [test_oracle_rlof]),
    "DeGraF tie picks the negative centroid": (
        "int use_neg = Sn > S;\n            double cx = use_neg ? (double)Xn",
        "int use_neg = Sn >= S;\n            double cx = use_neg ? (double)Xn", [test_oracle_degraf]),
    "pyramid level sizes rounded up": (
        "for (int k = 0; k < l; ++k) { w /= 2; h /= 2; }", "for (int k = 0; k < l; ++k) { w = (w + 1) / 2; h = (h + 1) / 2; }",
        [test_oracle_pyramid]),
    "cross rows measured from the centre pixel": (
        "while (lf < r && fabs(PIX(cx - lf - 1, cy + ky) - va) <= tau) ++lf;",
        "while (lf < r && fabs(PIX(cx - lf - 1, cy + ky) - vc) <= tau) ++lf;", [test_oracle_cross]),
    "global-motion weights lose their square": (
        "const double u = 1.0 - (e / ck) * (e / ck);", "const double u = 1.0 - (e / ck);", [test_oracle_gm]),
    "global-motion fit transposes an operand": (
        "bx[r] += w * v[r] * qx;", "bx[r] += w * v[r] * qy;", [test_oracle_gm]),
    "EPIC step cost counts one end only": (
        "const ep_item c = {it.d + C[it.v] + C[o], it.s, (int32_t)o};",
        "const ep_item c = {it.d + 2 * C[o], it.s, (int32_t)o};", [test_oracle_epic]),
    "EPIC tie keeps the higher seed index": (
        "(c.d == D[o] && c.s < S[o])", "(c.d == D[o] && c.s > S[o])", [test_oracle_epic]),
    "EPIC link weight drops a cost": (
        "const int64_t w = D[o] + C[o] + C[nb[q]] + D[nb[q]];",
        "const int64_t w = D[o] + C[nb[q]] + D[nb[q]];", [test_oracle_epic]),
    "EPIC kernel loses its factor 2": (
        "exp(-p->a * (double)it.d / (2.0 * p->cost_base))", "exp(-p->a * (double)it.d / p->cost_base)",
        [test_oracle_epic]),
    "EPIC fit offsets flip sign in x": (
        "const double v[3] = {pts[2 * t] - xs, pts[2 * t + 1] - ys, 1.0};",
        "const double v[3] = {xs - pts[2 * t], pts[2 * t + 1] - ys, 1.0};", [test_oracle_epic]),
    "EPIC edges from a Prewitt instead of a Sobel operator": (
        "const int wc = dy == 0 ? 2 : 1, wr = dx == 0 ? 2 : 1;", "const int wc = 1, wr = 1;", [test_oracle_epic]),
}


# Mistakes in the oracle's Python functions: name: (function, text, replacement, pin modules)
PY_MUTANTS = {
    "round-trip error subtracts the backward flow": (
        "rlof_track_fb", "np.hypot(*(f + b).T)", "np.hypot(*(f - b).T)", [test_oracle_fb]),
    "backward pass starts from the start points": (
        "rlof_track_fb", "rlof_track(I2, I1, pts + f, params, nthreads,", "rlof_track(I2, I1, pts, params, nthreads,",
        [test_oracle_fb]),
    "the filter also rejects points the forward pass lost": (
        "rlof_track_fb", "status[fwd & (err > fb_max)] = FB_REJECTED", "status[err > fb_max] = FB_REJECTED",
        [test_oracle_fb]),
    "global-motion prior forgets to subtract the point": (
        "gm_prior_flow", "a[0] * x + a[1] * y + a[2] - x", "a[0] * x + a[1] * y + a[2]", [test_oracle_gm]),
}


def module_fixtures(module):
    """The module's argument-free fixtures, as plain functions."""
    out = {}
    for name, obj in vars(module).items():
        fn = None
        if hasattr(obj, "_get_wrapped_function"):  # pytest >= 8.4
            fn = obj._get_wrapped_function()
        elif hasattr(obj, "__pytest_wrapped__"):
            fn = obj.__pytest_wrapped__.obj
        if fn is not None and not inspect.signature(fn).parameters:
            out[name] = fn
    return out


def pin_calls(module):
    """(name, callable) for every pin of a module: parametrized pins expanded and the
    module's own fixtures supplied."""
    fixtures = module_fixtures(module)
    for name, fn in inspect.getmembers(module, inspect.isfunction):
        if not name.startswith("test_") or fn.__module__ != module.__name__:
            continue
        marks = [m for m in getattr(fn, "pytestmark", []) if m.name == "parametrize"]
        params = list(inspect.signature(fn).parameters)
        fx = {p: fixtures[p] for p in params if p in fixtures}
        if not marks:
            if set(fx) == set(params):
                yield name, (lambda f=fn, x=fx: f(**{k: v() for k, v in x.items()}))
            continue
        grids = []
        for m in marks:
            names = [n.strip() for n in m.args[0].split(",")] if isinstance(m.args[0], str) else list(m.args[0])
            values = [v if len(names) > 1 else (v,) for v in m.args[1]]
            grids.append([dict(zip(names, v)) for v in values])
        for combo in itertools.product(*grids):
            kw = {}
            for d in combo:
                kw.update(d)
            if set(kw) | set(fx) == set(params):
                yield f"{name}{kw}", (lambda f=fn, k=kw, x=fx: f(**k, **{n: v() for n, v in x.items()}))


def build_copy(source: str, directory: str) -> str:
    c = os.path.join(directory, "mutant.c")
    so = os.path.join(directory, "libmutant.so")
    with open(c, "w") as f:
        f.write(source)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
                    "-o", so, c, "-lm"], check=True, capture_output=True)
    return so


@pytest.mark.parametrize("name", list(MUTANTS))
def test_every_planted_mistake_fails_a_pin(name, monkeypatch):
    old, new, modules = MUTANTS[name]
    source = open(SRC).read()
    assert source.count(old) == 1, f"mutation site not unique: {old}"
    with tempfile.TemporaryDirectory() as tmp:
        so = build_copy(source.replace(old, new), tmp)
        monkeypatch.setattr(oracle, "_libs", {})
        monkeypatch.setattr(oracle, "build", lambda force=False, precision="f64": so)
        failed = []
        for module in modules:
            for pin, call in pin_calls(module):
                try:
                    call()
                except Exception:  # a failed assertion, or an error the mistake provokes
                    failed.append(pin)
        monkeypatch.setattr(oracle, "_libs", {})  # the real oracle is loaded again on next use
    print(f"{name}: caught by {failed[:3]}{' ...' if len(failed) > 3 else ''}")
    assert failed, f"no pin catches: {name}"


@pytest.mark.parametrize("name", list(PY_MUTANTS))
def test_every_planted_python_mistake_fails_a_pin(name, monkeypatch):
    fn_name, old, new, modules = PY_MUTANTS[name]
    source = inspect.getsource(getattr(oracle, fn_name))
    assert source.count(old) == 1, f"mutation site not unique: {old}"
    namespace = dict(vars(oracle))
    exec(compile(source.replace(old, new), f"<mutant of oracle.{fn_name}>", "exec"), namespace)
    monkeypatch.setattr(oracle, fn_name, namespace[fn_name])
    failed = []
    for module in modules:
        for pin, call in pin_calls(module):
            try:
                call()
            except Exception:  # a failed assertion, or an error the mistake provokes
                failed.append(pin)
    print(f"{name}: caught by {failed[:3]}{' ...' if len(failed) > 3 else ''}")
    assert failed, f"no pin catches: {name}"
