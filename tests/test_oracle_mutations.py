"""The oracle's pins catch plausible mistakes.  Each case plants one mistake in a copy of
`oracle/cme_oracle.c` (a conjugate on the wrong factor, a dropped conjugate or factor, a wrong
index or sign, a dropped or wrong Runge-Kutta term, the pump on the wrong mode, a wrong
normalisation, a wrong mode band, a wrong step in the adjoint), compiles it with the oracle's
own flags, and runs the committed pin suites (test_oracle_pins, test_oracle_adjoint,
test_oracle_tangent, test_oracle_padding, test_oracle_kerr) in a child process whose oracle calls all go to the modified build.  The
same is done for the oracle's numpy Eq. 4 engine (`oracle/fft_engine.py`) through a copy of the
package.  The unmodified sources must pass the pins; every mutant must fail at least one.
CPU only."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cme_oracle.c")
PIN_SUITES = ["tests/test_oracle_pins.py", "tests/test_oracle_adjoint.py",
              "tests/test_oracle_tangent.py", "tests/test_oracle_padding.py",
              "tests/test_oracle_kerr.py"]

# name: (text in cme_oracle.c, replacement); the text occurs exactly once.
MUTATIONS = {
    # four-wave-mixing sum (Eq. 2 / Eq. 3)
    "FWM: conjugate on alpha": ("s += D[ia] * cb * D[gamma + h];",
                                "s += conj(D[ia]) * cb * D[gamma + h];"),
    "FWM: conjugate dropped on beta": ("const cplx cb = conj(D[beta + h]);",
                                       "const cplx cb = D[beta + h];"),
    "FWM: wrong index relation": ("long alpha = (long)mu + beta - gamma;\n                int ia;\n                if (linear)",
                                  "long alpha = (long)mu - beta + gamma;\n                int ia;\n                if (linear)"),
    "FWM: wrapped index off by one": ("long i = (mu + N / 2) % N;",
                                      "long i = (mu + N / 2 + 1) % N;"),
    # right-hand side and linear operator
    "detuning sign": ("m->omega[i] - omega0 - m->sigma", "m->omega[i] - omega0 + m->sigma"),
    "loss sign": ("return -0.5 * m->kappa[i] + I", "return 0.5 * m->kappa[i] + I"),
    "Kerr coefficient not imaginary": ("out[i] *= I * kerr_coef(m, i);",
                                       "out[i] *= kerr_coef(m, i);"),
    "per-mode Kerr coefficient ignored": ("return m->g0mu ? m->g0mu[i] : m->g0;",
                                          "return m->g0;"),
    "per-mode Kerr coefficient of the mirrored mode": (
        "return m->g0mu ? m->g0mu[i] : m->g0;",
        "return m->g0mu ? m->g0mu[m->N - 1 - i] : m->g0;"),
    "pump on the wrong mode": ("out[m->N / 2] += sqrt", "out[m->N / 2 + 1] += sqrt"),
    "pump without sqrt(kappa_ext)": ("out[m->N / 2] += sqrt(m->kappa_ext) * m->A_in;",
                                     "out[m->N / 2] += m->kappa_ext * m->A_in;"),
    # RK4IP
    "RK4IP: dropped k4 term": ("2.0 * k3[i])) + h / 6.0 * k4[i];", "2.0 * k3[i]));"),
    "RK4IP: wrong stage coefficient": ("x[i] = AI[i] + 0.5 * h * k1[i];",
                                       "x[i] = AI[i] + h * k1[i];"),
    "RK4IP: missing propagator on the last stage": ("x[i] = E[i] * (AI[i] + h * k3[i]);",
                                                    "x[i] = AI[i] + h * k3[i];"),
    "RK4IP: full-step propagator": ("E[i] = cexp(lin_coef(m, i) * (0.5 * h));\n    for (int i = 0; i < N; ++i)\n        AI[i]",
                                    "E[i] = cexp(lin_coef(m, i) * h);\n    for (int i = 0; i < N; ++i)\n        AI[i]"),
    # plain RK4
    "RK4: wrong last stage": ("x[i] = D[i] + h * k3[i];", "x[i] = D[i] + 0.5 * h * k3[i];"),
    # split step and transforms (Eq. 4)
    "Strang: Kerr phase sign": ("cexp(I * (m->g0 * p2 * h))", "cexp(-I * (m->g0 * p2 * h))"),
    "Strang: missing 1/N": ("? D[i] / (double)N : 0.0", "? D[i] : 0.0"),
    "Strang: pump term of the linear flow": ("D[i] += (e - 1.0) / L * p;", "D[i] += e / L * p;"),
    "DFT: wrong sign of the forward transform": ("s += a[j] * cexp(-I * (2.0 * M_PI",
                                                 "s += a[j] * cexp(I * (2.0 * M_PI"),
    # padding (physical band)
    "padding: band one mode too wide": ("return i >= first && i < first + M;",
                                        "return i >= first && i <= first + M;"),
    # Eq. 1 in the laboratory frame
    "Eq. 1: phase sign of mu": ("+ m->omega[gamma + hN]\n                                  - m->omega[mu + hN];",
                                "+ m->omega[gamma + hN]\n                                  + m->omega[mu + hN];"),
    # invariants
    "Hamiltonian: quartic factor": ("out[1] = quad + 0.5 * g0 * creal(quart);",
                                    "out[1] = quad + g0 * creal(quart);"),
    # adjoint
    "VJP: factor 2 dropped": ("s += 2.0 * w * D[beta + h] * conj(D[i]);",
                              "s += w * D[beta + h] * conj(D[i]);"),
    "VJP: conjugate dropped on the cotangent": ("s += conj(w) * D[i] * D[gamma + h];",
                                                "s += w * D[i] * D[gamma + h];"),
    "adjoint: Kerr coefficient not conjugated": ("tmp[i] = conj(I * kerr_coef(m, i)) * ybar[i];",
                                                 "tmp[i] = (I * kerr_coef(m, i)) * ybar[i];"),
    "adjoint: k3 cotangent": ("kb[i] = h / 3.0 * wb[i] + h * vb[i];",
                              "kb[i] = h / 3.0 * wb[i] + 0.5 * h * vb[i];"),
    "adjoint: log10 derivative": ("2.0 * r / ((P + eps) * log(10.0));", "2.0 * r / (P + eps);"),
    "adjoint: propagator cotangent": ("const cplx Lb = conj(0.5 * h * E[i]) * Eb[i];",
                                      "const cplx Lb = conj(h * E[i]) * Eb[i];"),
    "adjoint: pump cotangent conjugated": ("*pbar += ybar[N / 2];", "*pbar += conj(ybar[N / 2]);"),
    "adjoint: propagator cotangent of k1 = E y1 dropped": (
        "            Eb[i] += conj(y1[i]) * kb[i];\n", ""),
    "adjoint: propagator cotangent of the last stage dropped": (
        "            Eb[i] += conj(v[i]) * xb[i];\n", ""),
    "adjoint: k1 cotangent weight": ("kb[i] = h / 6.0 * wb[i] + 0.5 * h * xb[i]; /* k1bar */",
                                     "kb[i] = h / 3.0 * wb[i] + 0.5 * h * xb[i]; /* k1bar */"),
    # adjoint of the Strang split step
    "Strang adjoint: phase factor not conjugated": (
        "ab[j] = conj(u[j]) * (1.0 - I * gam * p2) * bb[j] +",
        "ab[j] = u[j] * (1.0 - I * gam * p2) * bb[j] +"),
    "Strang adjoint: sign of the |a|^2 term": ("(1.0 - I * gam * p2) * bb[j]",
                                               "(1.0 + I * gam * p2) * bb[j]"),
    "Strang adjoint: conjugate cotangent term": ("I * gam * a[j] * a[j] * u[j] * conj(bb[j]);",
                                                 "I * gam * a[j] * a[j] * u[j] * bb[j];"),
    "Strang adjoint: missing 1/N": ("bb[j] /= (double)N;", "bb[j] /= 1.0;"),
    "Strang adjoint: pump cotangent of the second half flow": ("cbar += Db[c0];",
                                                               "cbar += 0.0;"),
    "Strang adjoint: derivative of the pump increment": ("(dt * e[c0] - phi) / L0",
                                                         "(e[c0] - phi) / L0"),
    "Strang adjoint: propagator cotangent over h": ("cplx Lb = conj(dt * e[i]) * Eb[i];",
                                                    "cplx Lb = conj(h * e[i]) * Eb[i];"),
    "Strang adjoint: log10 derivative": ("2.0 * r / (log(10.0) * (P + eps));",
                                         "2.0 * r / (P + eps);"),
    "Strang adjoint: padding modes in the Kerr cotangent": (
        "tmp[i] = physical(i, N, M) ? Db[i] : 0.0;", "tmp[i] = Db[i];"),
}


def compile_oracle(text, tmp_path):
    src = tmp_path / "cme_oracle.c"
    src.write_text(text)
    lib = tmp_path / "libcme_oracle.so"
    subprocess.run(["gcc", "-std=gnu11", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC",
                    "-shared", "-o", str(lib), str(src), "-lm"], check=True)
    return str(lib)


def run_pins(lib):
    """Exit code of the pin suites with every oracle call going to `lib` (0: all passed,
    1: some failed)."""
    code = ("import sys, pytest, oracle; oracle.use_library(sys.argv[1]); "
            "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu'] "
            "+ sys.argv[2:]))")
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", code, lib, *PIN_SUITES], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def test_unmodified_oracle_passes_the_pins(tmp_path):
    rc, out = run_pins(compile_oracle(open(SRC).read(), tmp_path))
    assert rc == 0, out


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTATIONS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, name
    rc, out = run_pins(compile_oracle(text.replace(old, new), tmp_path))
    assert rc == 1, f"{name}: pins exit {rc}\n{out}"


# The oracle's numpy Eq. 4 engine (fft_engine.py), pinned to the direct engine: the same
# planted-mistake check through a copy of the oracle package with one edit in fft_engine.py.
ENGINE_MUTATIONS = {
    "Eq. 4: missing 1/N": ("return _to_centred(np.fft.fft(np.abs(a) ** 2 * a, axis=-1) / N)",
                           "return _to_centred(np.fft.fft(np.abs(a) ** 2 * a, axis=-1))"),
    "Eq. 4: padding modes keep their FWM term": ("        out = np.where(self.mask, out, 0.0)\n",
                                                 ""),
    "engine: detuning sign": ("1j * (self.omega - om0 - self.sigma)",
                              "1j * (self.omega - om0 + self.sigma)"),
    "engine RK4IP: missing propagator on the last stage": (
        "k4 = batch.F(E * (AI + h * k3), linear)", "k4 = batch.F(AI + h * k3, linear)"),
    "engine Strang: half the Kerr phase": (
        "a = a * np.exp(1j * batch.g0[:, :1] * np.abs(a) ** 2 * h)",
        "a = a * np.exp(1j * batch.g0[:, :1] * np.abs(a) ** 2 * 0.5 * h)"),
    "engine: per-mode Kerr coefficient of the mirrored mode": (
        "else np.asarray(i.g0_mu, dtype=np.float64) for i in instances])",
        "else np.asarray(i.g0_mu, dtype=np.float64)[::-1] for i in instances])"),
    "engine Strang: pump increment": ("(e[:, N // 2] - 1.0) / np.where", "e[:, N // 2] / np.where"),
}


def run_pins_with_oracle_copy(tmp_path, edit=None):
    """Exit code of the pin suites with `import oracle` resolving to a copy of the package in
    tmp_path (its C library built there), fft_engine.py edited by `edit` = (old, new)."""
    import shutil
    dst = tmp_path / "oracle"
    shutil.copytree(os.path.join(ROOT, "oracle"), dst,
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    if edit:
        p = dst / "fft_engine.py"
        text = p.read_text()
        assert text.count(edit[0]) == 1, edit[0]
        p.write_text(text.replace(edit[0], edit[1]))
    code = ("import sys, pytest, oracle; "
            "assert oracle.__file__.startswith(sys.argv[1]), oracle.__file__; "
            "sys.exit(pytest.main(['-x', '-q', '-p', 'no:cacheprovider', '-m', 'not gpu', "
            "'--rootdir', sys.argv[2]] + sys.argv[3:]))")
    env = dict(os.environ, PYTHONPATH=str(tmp_path) + os.pathsep + ROOT)
    suites = [os.path.join(ROOT, s) for s in PIN_SUITES]
    r = subprocess.run([sys.executable, "-c", code, str(tmp_path), ROOT, *suites],
                       cwd=str(tmp_path), env=env, capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:] + r.stderr[-1000:]


def test_unmodified_engine_copy_passes_the_pins(tmp_path):
    rc, out = run_pins_with_oracle_copy(tmp_path)
    assert rc == 0, out


@pytest.mark.parametrize("name", list(ENGINE_MUTATIONS))
def test_planted_mistake_in_the_eq4_engine_is_caught(tmp_path, name):
    rc, out = run_pins_with_oracle_copy(tmp_path, ENGINE_MUTATIONS[name])
    assert rc == 1, f"{name}: pins exit {rc}\n{out}"
