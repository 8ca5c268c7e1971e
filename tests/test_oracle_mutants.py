"""The oracle's pins catch plausible mistakes.

Each case below copies oracle.c, plants one mistake of the kind a careful
reader could still make (a dropped term, a wrong sign, index or constant, a
transposed operand, an inverse permutation), builds the copy with the oracle's
own flags and runs the pin tests (test_oracle_pins.py) against it through
ORACLE_LIB; at least one pin must fail.  The unmodified copy runs the same way
first and must pass, so that a broken harness cannot pass for a caught
mistake.  oracle.c itself is never changed.

Left out on purpose, because they change no result that any test could see
(equivalent mutants): keeping the imaginary part of the Nyquist bin in the
inverse real transform (it contributes only to the imaginary part of the
output, which is discarded) and skipping the mean removal of the TK95 series
(X_0 = 0 already makes the mean zero up to rounding)."""
import concurrent.futures as cf
import os
import subprocess
import sys

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (what the mistake is, text in oracle.c, text put in its place)
MUTANTS = [
    ("Philox Weyl constant", "#define PHILOX_W1 0xBB67AE85u", "#define PHILOX_W1 0xBB67AE86u"),
    ("Philox word routing", "        c1 = lo1;\n", "        c1 = lo0;\n"),
    ("u01 without the half-step offset", "(double)(2 * u + 1) * 0x1p-53", "(double)(2 * u) * 0x1p-53"),
    ("exp Taylor coefficient", "p = fma(p, r, 1.0 / 5040.0);", "p = fma(p, r, 1.0 / 5041.0);"),
    ("exp reduction without the low part of ln2", "    r = fma(-k, OR_LN2_LO, r);\n", "\n"),
    ("log series coefficient", "q = fma(q, z, 1.0 / 3.0);", "q = fma(q, z, 1.0 / 3.1);"),
    ("log1p without the rounding correction", "return or_spec_log(w) + t;", "return or_spec_log(w);"),
    ("ERDF upper mass divided by the lower slope", "M2 = (e2 - 1.0) / c2;", "M2 = (e2 - 1.0) / c1;"),
    ("ERDF lower branch sign", "u = ub + t / c1;", "u = ub - t / c1;"),
    ("ERDF linear-space slope shift dropped in the inverse",
     "    if (linear_space) { a1 = a1 + 1.0; a2 = a2 + 1.0; }\n    double c1 = a1 * OR_LN10, c2 = a2 * OR_LN10;\n"
     "    double e1", "    double c1 = a1 * OR_LN10, c2 = a2 * OR_LN10;\n    double e1"),
    ("ERDF upper clamp dropped", "    if (lam > hi) lam = hi;\n", "\n"),
    ("log-normal exponent factor", "double e = -0.5 * t * t;", "double e = -t * t;"),
    ("log-normal linear-space term sign", "if (linear_space) e = e + OR_LN10 * d;",
     "if (linear_space) e = e - OR_LN10 * d;"),
    ("Eq. 1 smooth form sign", "return 1.0 / (or_spec_exp(-c1 * d) + or_spec_exp(-c2 * d));",
     "return 1.0 / (or_spec_exp(c1 * d) + or_spec_exp(-c2 * d));"),
    ("Simpson weight", "+ 4.0 * or_erdf_density", "+ 2.0 * or_erdf_density"),
    ("tabulated inverse without interpolation", "double u = (umin + (double)lo * h) + t * h;",
     "double u = (umin + (double)lo * h);"),
    ("draws not rounded to float", "out[k] = prec == 0 ? (double)(float)lam : lam;", "out[k] = lam;"),
    ("Eq. 3 slopes", "return 1.0 / (pow(y, a_low) + pow(y, a_high));",
     "return 1.0 / (pow(y, a_low) + pow(y, a_low));"),
    ("Eq. 3 break frequency", "double y = f / f_br;", "double y = f * f_br;"),
    ("TK95 power not split over Re and Im", "double a = coeffs == 1 ? sqrt(P) : sqrt(P / 2.0);",
     "double a = coeffs == 1 ? sqrt(P) : sqrt(P);"),
    ("Fourier frequency", "double f = (double)j / ((double)n * dt);", "double f = (double)j / (double)n * dt;"),
    ("Box-Muller radius", "sqrt(-2.0 * log(U1))", "sqrt(-log(U1))"),
    ("Box-Muller pair correlated", "g_im = rad * sin(two_pi * U2);", "g_im = rad * cos(two_pi * U2);"),
    ("TK95 Nyquist power", "X[2 * j] = coeffs == 1 ? (g_re < 0.0 ? -sqrt(P) : sqrt(P)) : sqrt(P) * g_re;",
     "X[2 * j] = coeffs == 1 ? (g_re < 0.0 ? -sqrt(P) : sqrt(P)) : sqrt(P / 2.0) * g_re;"),
    ("fixed-amplitude radius", "double rad = coeffs == 1 ? 1.0 :", "double rad = coeffs == 1 ? 2.0 :"),
    ("direct DFT index", "size_t t = (j * k) % n;", "size_t t = (j * (k + 1)) % n;"),
    ("FFT butterfly sign", "cplx t = {o.re * c - o.im * s, o.re * s + o.im * c};",
     "cplx t = {o.re * c + o.im * s, o.re * s + o.im * c};"),
    ("FFT twiddle angle", "double ang = (double)sign * two_pi * (double)k / (double)n;",
     "double ang = (double)sign * two_pi * (double)k / (double)h;"),
    ("forward transform sign", "or_fft(n, buf, spec, -1);", "or_fft(n, buf, spec, +1);"),
    ("inverse real transform without the conjugate", "buf[2 * (n - j) + 1] = -Y[2 * j + 1];",
     "buf[2 * (n - j) + 1] = Y[2 * j + 1];"),
    ("sample instead of population variance", "    var /= (double)n;\n", "    var /= (double)(n - 1);\n"),
    ("amplitudes not scaled by sigma", "A[j] = hypot(X[2 * j], X[2 * j + 1]) / sigma;",
     "A[j] = hypot(X[2 * j], X[2 * j + 1]);"),
    ("PSD variance with a doubled Nyquist bin", "sp += j < nh ? 2.0 * P : P;", "sp += 2.0 * P;"),
    ("descending sort", "    if (a->v < b->v) return -1;\n    if (a->v > b->v) return 1;\n",
     "    if (a->v < b->v) return 1;\n    if (a->v > b->v) return -1;\n"),
    ("ties in reverse index order", "return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);",
     "return a->i < b->i ? 1 : (a->i > b->i ? -1 : 0);"),
    ("phase taken from the real part twice", "X[2 * j + 1] = A[j] * (im / mag);", "X[2 * j + 1] = A[j] * (re / mag);"),
    ("Nyquist sign not kept", "X[2 * nh] = X[2 * nh] < 0.0 ? -A[nh] : A[nh];", "X[2 * nh] = A[nh];"),
    ("DC bin not replaced by A_0", "X[0] = A[0]; X[1] = 0.0;", "X[0] = 1.0; X[1] = 0.0;"),
    ("inverse permutation in the rank step", "for (size_t r = 0; r < n; ++r) x[perm[r]] = s[r];",
     "for (size_t r = 0; r < n; ++r) x[r] = s[perm[r]];"),
    ("draws not sorted", "    or_sort(n, s);\n", "\n"),
    ("Eq. 4 with the natural log", "double t = log10(x_new[k] / x_old[k]);", "double t = log(x_new[k] / x_old[k]);"),
    ("Eq. 4 without the root", "return sqrt(acc / (double)n);", "return acc / (double)n;"),
    ("convergence threshold inclusive", "if (d < thr) break;", "if (d <= thr) break;"),
    ("convergence distance against the wrong iterate", "        double d = or_delta(n, xp, x);\n",
     "        double d = or_delta(n, x, x);\n"),
    ("Eq. A2 factor", "2.0 * p2 / (nd * nd)", "p2 / (nd * nd)"),
    ("Eq. A4 mean squared", "2.0 * dt * p2 / (mu * mu * nd)", "2.0 * dt * p2 / (mu * nd)"),
    ("Eq. A6 pair count", "sf2[l] = acc / (double)(n - tau);", "sf2[l] = acc / (double)n;"),
    ("Eq. A6 lag", "double d = x[i] - x[i + tau];", "double d = x[i] - x[i + tau - 1];"),
    ("batch offsets from the first length", "offsets[c + 1] = offsets[c] + ((size_t)1 << log2n[c]);",
     "offsets[c + 1] = offsets[c] + ((size_t)1 << log2n[0]);"),
]


PHILOX_PIN = os.path.join("tests", "test_oracle_pins.py") + "::test_philox_matches_independent_implementation"


def _run_pins(src_text, workdir, philox=True):
    """Build src_text as the oracle library and run the pins against it:
    (exit code, the pytest summary lines).  philox=False leaves out the
    comparison with an independent Philox (a few seconds in Triton's
    interpreter), which checks nothing but the generator."""
    src = os.path.join(workdir, "oracle.c")
    so = os.path.join(workdir, "liboracle.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *oracle.CFLAGS, "-o", so, src, "-lm"], check=True)
    env = dict(os.environ, ORACLE_LIB=so)
    cmd = [sys.executable, "-m", "pytest", os.path.join("tests", "test_oracle_pins.py"), "-x", "-q",
           "-m", "not gpu", "-p", "no:cacheprovider"]
    if not philox:
        cmd += ["--deselect", PHILOX_PIN]
    r = subprocess.run(cmd,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return r.returncode, [ln for ln in r.stdout.splitlines() if ln.startswith(("FAILED", "ERROR"))]


def test_every_planted_mistake_fails_a_pin(tmp_path):
    with open(os.path.join(ROOT, "oracle", "oracle.c")) as f:
        src = f.read()
    for name, old, _ in MUTANTS:
        assert src.count(old) == 1, f"{name}: the text to replace must occur exactly once"
    control = tmp_path / "control"
    control.mkdir()
    rc, lines = _run_pins(src, str(control))
    assert rc == 0, ("the unmodified copy must pass the pins", lines)

    def one(k):
        name, old, new = MUTANTS[k]
        d = tmp_path / f"m{k}"
        d.mkdir()
        rc, lines = _run_pins(src.replace(old, new), str(d), philox=name.startswith("Philox"))
        return name, rc, lines

    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        results = list(ex.map(one, range(len(MUTANTS))))
    survived = [name for name, rc, _ in results if rc == 0]
    errored = [(name, lines) for name, rc, lines in results if rc != 0 and not any(ln.startswith("FAILED") for ln in lines)]
    assert not survived, f"planted mistakes that no pin catches: {survived}"
    assert not errored, f"mistakes that broke the harness instead of failing a pin: {errored}"
