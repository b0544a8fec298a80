"""The pins are strong enough to catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of `oracle/` (on the CPU: a source line
replaced, the C part rebuilt in the copy) and runs the pins of that part
against the copy in a fresh interpreter; the pins must fail.  A replacement
string must occur exactly once in the current source, so that an edit of the
oracle that moves a line fails here rather than leaving a case that plants
nothing.  Mutants that are equivalent to the oracle (same outputs on every
input) are not listed."""
import concurrent.futures
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C = "l1line_oracle.c"
FIT_PINS = ["tests/test_oracle_pins.py"]
PATH_PINS = ["tests/test_path_oracle_pins.py"]
MUTANTS = {
    # Algorithm 1 and Lemma 1 (C)
    "fit": (FIT_PINS, [
        (C, "scratch[cnt].w = (double)ABS(bi);", "scratch[cnt].w = (double)ABS(a[i * sa]);"),
        (C, "scratch[cnt].w = lambda;", "scratch[cnt].w = 0.0;"),
        (C, "scratch[cnt].w = lambda;", "scratch[cnt].w = 2.0 * lambda;"),
        (C, "nsum_add(&z, pen);", ""),
        (C, "v[k] = (k == jh) ? (T)1 :", "v[k] = (k == jh) ? (T)0 :"),
        (C, "double term = fabs((double)X[i * m + k] - prod);",
         "double term = fabs((double)X[i * m + k] + prod);"),
        (C, "if (kacc_sign(&D) > 0) return", "if (kacc_sign(&D) >= 0) return"),
        (C, "if (best < 0 || zj < zbest) {", "if (best < 0 || zj <= zbest) {"),
        (C, "            kacc_add(&D, list[p].w, 0);\n            kacc_add(&D, list[p].w, 0);\n",
         "            kacc_add(&D, list[p].w, 0);\n"),
    ]),
    # Algorithm 2 (C)
    "path": (PATH_PINS, [
        (C, "if (r < 0.0) kacc_neg(&x);", "if (r > 0.0) kacc_neg(&x);"),
        (C, "            kacc_add(&lam, w, 1);", "            kacc_add(&lam, w, 0);"),
        (C, "            kacc_add(&top, w, 0);", "            kacc_add(&top, w, 1);"),
        (C, "    return (x < y) - (x > y);", "    return (x > y) - (x < y);"),
        (C, "if (k == 0 || out[p].v != out[k - 1].v) out[k++] = out[p];", "out[k++] = out[p];"),
        (C, "if (tv > lmax) lmax = tv;", "if (tv < lmax) lmax = tv;"),
        (C, "        kacc_add(&before, w, 0);", "        if (r != 0.0) kacc_add(&before, w, 0);"),
        (C, "    out[e].v = v0;", "    out[e].v = 0.0;"),
    ]),
    # Algorithm 3 (Python, exact rationals)
    "solution_path": (["tests/test_solution_path_pins.py"], [
        ("solution_path.py", "Z.append(r + lo * S[jh])", "Z.append(r)"),
        ("solution_path.py", "beta_l = max(bl) if bl else None", "beta_l = min(bl) if bl else None"),
        ("solution_path.py", "beta_u = min(bu) if bu else None", "beta_u = max(bu) if bu else None"),
        ("solution_path.py", "(Z[h] == Z[j] and h < j)", "(Z[h] == Z[j] and h > j)"),
        ("solution_path.py", 'side="right")) - 1', 'side="left")) - 1'),
        ("solution_path.py", "S = [sum(abs(x) for x in V[jh]) for jh in range(m)]",
         "S = [sum(x for x in V[jh]) for jh in range(m)]"),
        ("solution_path.py", "            out[-1] = e\n", "            pass\n"),
    ]),
    # successive components (Python)
    "components": (["tests/test_components_pins.py"], [
        ("components.py", "return (X - prod).astype(X.dtype)", "return (X + prod).astype(X.dtype)"),
        ("components.py", "X = deflate(X, j, v)", "X = deflate(X, 0, v)"),
        ("components.py", "        X = deflate(X, j, v)\n        mats.append(X)",
         "        mats.append(X)\n        X = deflate(X, j, v)"),
    ]),
    # the proposer's float64 reference (Python)
    "proposer": (["tests/test_proposer_ref_pins.py"], [
        ("proposer_ref.py", "(n - 1) // 2", "n // 2"),
        ("proposer_ref.py", "sd = np.sqrt(((F - mu) ** 2).mean(axis=0))",
         "sd = np.sqrt(((F - mu) ** 2).sum(axis=0) / (F.shape[0] - 1))"),
        ("proposer_ref.py", "g2 = np.outer(ds, w3) * (a2 > 0)", "g2 = np.outer(ds, w3) * (a2 >= 0)"),
        ("proposer_ref.py", "g1 = (g2 @ W2) * (a1 > 0)", "g1 = (g2 @ W2)"),
        ("proposer_ref.py", "dW2 = g2.T @ h1", "dW2 = h1.T @ g2"),
        ("proposer_ref.py", "ds[r0:r1] = (p - q) / nb", "ds[r0:r1] = (p - q)"),
        ("proposer_ref.py", "mh = m1 / (1.0 - beta1 ** step)", "mh = m1"),
        ("proposer_ref.py", "np.sqrt(vh) + eps", "np.sqrt(vh + eps)"),
        ("proposer_ref.py", "pack(r(W1), b1, r(W2), b2, r(w3), b3)",
         "pack(r(W1), r(b1), r(W2), r(b2), r(w3), b3)"),
        ("proposer_ref.py", "order = np.lexsort((np.arange(s.size), -key, nanmask))",
         "order = np.lexsort((-np.arange(s.size), -key, nanmask))"),
        ("proposer_ref.py", "return -(z - zs[0]) / (temperature * span)",
         "return -(z - zs[0]) / span"),
        ("proposer_ref.py", "loss += -(q * s[r0:r1]).sum() + lse",
         "loss += -(p * s[r0:r1]).sum() + lse"),
    ]),
}

# exit 3: the copy could not be set up (not a caught mistake)
RUNNER = """
import sys
sys.path.insert(0, {tmp!r})
try:
    import oracle
    assert oracle.__file__.startswith({tmp!r}), oracle.__file__
    oracle.build(force=True)
except Exception as e:
    print("setup failed:", e)
    sys.exit(3)
import pytest
sys.exit(pytest.main(["-q", "-x", "-p", "no:cacheprovider", *{pins!r}]))
"""


def _plant(tmp, fname, old, new):
    dst = os.path.join(tmp, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("*.so", "__pycache__", "*.tmp*"))
    path = os.path.join(dst, fname)
    src = open(path).read()
    assert src.count(old) == 1, f"{fname}: the planted line no longer occurs once: {old!r}"
    open(path, "w").write(src.replace(old, new))


def _pins_fail(tmp, pins) -> bool:
    """True when the pins fail on the copy (pytest exit 1); a copy that could
    not be set up or a run that did not test anything raises."""
    r = subprocess.run([sys.executable, "-c", RUNNER.format(tmp=tmp, pins=pins)], cwd=ROOT,
                       capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, OMP_NUM_THREADS="2"))
    if r.returncode not in (0, 1):
        raise RuntimeError(f"pins did not run on {tmp} (exit {r.returncode}):\n"
                           + r.stdout[-1500:] + r.stderr[-1500:])
    return r.returncode == 1


@pytest.mark.parametrize("part", sorted(MUTANTS))
def test_pins_catch_planted_mistakes(part, tmp_path):
    pins, cases = MUTANTS[part]
    dirs = []
    for i, (fname, old, new) in enumerate(cases):
        d = str(tmp_path / f"m{i}")
        os.makedirs(d)
        _plant(d, fname, old, new)
        dirs.append(d)
    workers = max(1, min(4, (os.cpu_count() or 2) // 2))
    with concurrent.futures.ThreadPoolExecutor(workers) as ex:
        caught = list(ex.map(lambda d: _pins_fail(d, pins), dirs))
    missed = [f"{c[0]}: {c[1].strip()!r} -> {c[2].strip()!r}"
              for c, ok in zip(cases, caught) if not ok]
    assert not missed, "pins passed with a planted mistake:\n" + "\n".join(missed)
