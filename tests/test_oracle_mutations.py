"""The oracle's pins must catch plausible mistakes in the oracle itself.

Each mutant is a copy of oracle/fic_oracle.c with one planted mistake (a
dropped term, a wrong sign, a swapped index or order, an off-by-one, a
wrong rounding), compiled on the CPU into a temporary library; the pin
suite (tests/test_oracle_pins.py) then runs against it, named by the
explicit --oracle-lib option of the pytest process, and must fail.  A control copy with no change must pass, so
a failure means the mistake was seen and not that the harness broke.
Nothing here touches the CUDA path."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "fic_oracle.c")

# name -> [(exact text in the oracle, replacement), ...]
MUTANTS = {
    # Sec. 2 isometries
    "rotation counter-clockwise": [
        ("out[i * B + j] = in[(B - 1 - j) * B + i];", "out[i * B + j] = in[j * B + (B - 1 - i)];")],
    "mirror about the horizontal axis": [
        ("out[i * B + j] = in[i * B + (B - 1 - j)];", "out[i * B + j] = in[(B - 1 - i) * B + j];")],
    "mirror before rotation": [
        ("    memcpy(a, in, sizeof(int32_t) * n);\n    for (int r = 0; r < (k & 3); ++r) {",
         "    memcpy(a, in, sizeof(int32_t) * n);\n"
         "    if (k >= 4) { mirror(a, B, b); memcpy(a, b, sizeof(int32_t) * n); k -= 4; }\n"
         "    for (int r = 0; r < (k & 3); ++r) {")],
    # Sec. 2 decimation: one pixel of the 2x2 counted twice
    "decimation drops a pixel": [
        ("img[(yy + 1) * N + xx] + img[(yy + 1) * N + xx + 1];",
         "img[(yy + 1) * N + xx] + img[(yy + 1) * N + xx];")],
    # Eq. 5-6 entropy
    "entropy in nats": [("h -= p * log2(p);", "h -= p * log(p);")],
    "entropy normalised by 4n + 1": [
        ("double total = (double)size * (double)size;", "double total = (double)size * (double)size + 1.0;")],
    # Eq. 1-3 score
    "cross term sign": [("- 8 * p * q * crd + p * p * vd;", "+ 8 * p * q * crd + p * p * vd;")],
    "domain variance term dropped": [("- 8 * p * q * crd + p * p * vd;", "- 8 * p * q * crd;")],
    "range variance without the mean": [("int64_t vr = n * sr2 - sr * sr;", "int64_t vr = n * sr2;")],
    "covariance with the wrong sum": [("int64_t crd = n * srd - sr * sd;", "int64_t crd = n * srd - sr * sr;")],
    "domain variance transposed sums": [("int64_t vd = n * sd2 - sd * sd;", "int64_t vd = n * sd2 - sd * sd2;")],
    # search and tie-break
    "ties to the last candidate": [("if (sc < best.score) {", "if (sc <= best.score) {")],
    "last pool domain skipped": [
        ("for (int64_t c = 0; c < pl->dn; ++c) {\n        const int32_t* d = pl->dsum",
         "for (int64_t c = 0; c < pl->dn - 1; ++c) {\n        const int32_t* d = pl->dsum")],
    "last S value skipped": [("for (int s = 0; s < ss->n_s; ++s) {\n                int64_t sc",
                              "for (int s = 0; s < ss->n_s - 1; ++s) {\n                int64_t sc")],
    "range block read transposed": [("r[i * B + j] = img[(y + i) * N + x + j];",
                                     "r[i * B + j] = img[(y + j) * N + x + i];")],
    "isometries 0-6 only": [("for (int k = 0; k < 8; ++k) {\n            or_isometry(d, B, k, t);",
                             "for (int k = 0; k < 7; ++k) {\n            or_isometry(d, B, k, t);")],
    # Sec. 3 pool
    "entropy threshold not strict": [("admit[i] = h > thr;", "admit[i] = h >= thr;")],
    "pool in column order": [
        ("pl->x[pl->dn] = (int32_t)(i % per) * L;\n            pl->y[pl->dn] = (int32_t)(i / per) * L;",
         "pl->x[pl->dn] = (int32_t)(i / per) * L;\n            pl->y[pl->dn] = (int32_t)(i % per) * L;")],
    "top-DN entropies rounded down": [("hx[i] = h * OR_HQ_SCALE + 0.5;", "hx[i] = h * OR_HQ_SCALE;")],
    "top-DN ties in reverse raster order": [
        ("return (u->i > v->i) - (u->i < v->i);", "return (u->i < v->i) - (u->i > v->i);")],
    "positions per axis off by one": [("return (N - 2 * B) / L + 1;", "return (N - 2 * B) / L;")],
    # Sec. 2 quadtree
    "split threshold with n instead of n^2": [
        ("16 * q * q * n * n * (int64_t)e->e16 * e->e16", "16 * q * q * n * (int64_t)e->e16 * e->e16")],
    "children TR and BL swapped": [
        ("if (encode_block(e, x + h, y, level + 1, out)) return -1;     /* TR */",
         "if (encode_block(e, x, y + h, level + 1, out)) return -1;     /* TR */"),
        ("if (encode_block(e, x, y + h, level + 1, out)) return -1;     /* BL */",
         "if (encode_block(e, x + h, y, level + 1, out)) return -1;     /* BL */")],
    "tolerance truncated to 1/16": [("(int)lround(16.0 * tol)", "(int)(16.0 * tol)")],
    "8-bit range mean": [("int64_t oq = sr / (2 * n);", "int64_t oq = sr / n;")],
    # decoder and eq. 4
    "decoder truncates": [("+ p * (n * t[i * B + j] - sd) + den / 2;", "+ p * (n * t[i * B + j] - sd);")],
    "decoder offset without the half step": [
        ("(2 * (int64_t)c->o_q + 1) * den", "(2 * (int64_t)c->o_q) * den")],
    "decoder reads the new iterate": [
        ("apply_code(&codes[i], ss, cur, N, nxt);", "apply_code(&codes[i], ss, nxt, N, nxt);")],
    "PSNR peak 256": [("return 10.0 * log10(255.0 * 255.0 / (se / (double)npx));",
                       "return 10.0 * log10(256.0 * 256.0 / (se / (double)npx));")],
    # eq. 8 address width
    "address bits off by one": [("while (((int64_t)1 << x) < dn) ++x;", "while (((int64_t)1 << x) <= dn) ++x;")],
}


def _build(src_text, d, name):
    c = os.path.join(d, name + ".c")
    so = os.path.join(d, name + ".so")
    with open(c, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", c, "-o", so, "-lm"],
                   check=True, capture_output=True)
    return so


def _pins(so):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        "--oracle-lib", so, os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _mutate(text, reps):
    for old, new in reps:
        assert text.count(old) == 1, f"mutation site not unique or missing: {old!r}"
        text = text.replace(old, new)
    return text


@pytest.fixture(scope="module")
def results():
    text = open(SRC).read()
    d = tempfile.mkdtemp(prefix="fic_mut_")
    jobs = {"control": text}
    for i, (name, reps) in enumerate(MUTANTS.items()):
        jobs[name] = _mutate(text, reps)
    libs = {name: _build(t, d, f"m{i}") for i, (name, t) in enumerate(jobs.items())}
    workers = max(1, min(8, (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_pins, so) for name, so in libs.items()}
        return {name: f.result() for name, f in futs.items()}


def test_control_copy_passes_the_pins(results):
    rc, out = results["control"]
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_pins_catch_the_mutant(results, name):
    rc, out = results[name]
    assert rc == 1, f"pins did not catch '{name}' (exit {rc}):\n{out}"
