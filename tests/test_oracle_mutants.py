"""The oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of oracle/hq_oracle.c (a transposed operand, a wrong bit or
index order, a dropped term, a wrong sign, a missing conjugate), compiles it
on the CPU, and runs tests/test_oracle_pins.py against it: the pin suite has
to fail."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hq_oracle.c")

MUTANTS = {
    "transposed_matrix": ("acc += M[r * K + c] * v[c];", "acc += M[c * K + r] * v[c];"),
    "qubit_bit_order": ("return (int64_t)1 << (n - 1 - q);", "return (int64_t)1 << q;"),
    "local_index_order": ("if ((r >> (k - 1 - j)) & 1) off[r] += qubit_bit(n, qubits[j]);",
                          "if ((r >> j) & 1) off[r] += qubit_bit(n, qubits[j]);"),
    "dropped_hamiltonian_term": ("        e += coeff[t] * creal(inner(dim, psi, tmp));",
                                 "        if (t > 0) e += coeff[t] * creal(inner(dim, psi, tmp));"),
    "derivative_sign": ("for (int i = 0; i < 4; ++i) m[i] = -0.5 * I * c * P[i];",
                        "for (int i = 0; i < 4; ++i) m[i] = 0.5 * I * c * P[i];"),
    "pauli_y_sign": ("static const cplx Y[4] = {0, -I, I, 0};", "static const cplx Y[4] = {0, I, -I, 0};"),
    "minus_token_sign": ("else if (t == '-') f = bit ? -s : s;", "else if (t == '-') f = s;"),
    "missing_conjugate": ("for (int64_t x = 0; x < dim; ++x) s += conj(a[x]) * b[x];",
                          "for (int64_t x = 0; x < dim; ++x) s += a[x] * b[x];"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mutant = tmp_path / "mutant.c"
    mutant.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O1", "-std=gnu99", "-fopenmp", "-fPIC", "-shared", "-o", str(lib), str(mutant),
                           "-lm"])
    env = dict(os.environ, HQ_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode != 0, f"the pins did not catch the planted mistake {name}:\n{r.stdout[-2000:]}"
