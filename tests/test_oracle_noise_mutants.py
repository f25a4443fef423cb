"""The noise oracle's pins must catch plausible mistakes.  Each case plants one
mistake in a copy of oracle/noise.py (a swapped row/column order, a missing
dagger or square root, a wrong channel weight or operator, a wrong inverse
permutation, a transposed partial trace, a conjugated Pauli), places the copy
in a scratch tree beside the unchanged oracle and input modules, and runs
tests/test_oracle_noise_pins.py there: the pin suite has to fail."""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "noise.py")

MUTANTS = {
    "superop_row_column_swap": (
        "order = list(qubits) + [n + q for q in qubits] + rest + [n + q for q in rest]",
        "order = [n + q for q in qubits] + list(qubits) + rest + [n + q for q in rest]"),
    "map_missing_dagger": ("out += s[i][j] * (li @ rho @ rj.conj().T)", "out += s[i][j] * (li @ rho @ rj.T)"),
    "depolarizing_identity_weight": ("w = (1 - p + p / 4 ** k) if", "w = (1 - p) if"),
    "amplitude_damping_transposed": (
        "K1 = np.array([[0, np.sqrt(gamma)], [0, 0]], dtype=np.complex128)",
        "K1 = np.array([[0, 0], [np.sqrt(gamma), 0]], dtype=np.complex128)"),
    "embed_wrong_inverse": ("    inv = np.argsort(order)\n    t = t.transpose(list(inv) + [n + i for i in inv])",
                            "    inv = order\n    t = t.transpose(list(inv) + [n + i for i in inv])"),
    "trajectory_missing_sqrt": ("return i, outs[i] / np.sqrt(p[i])", "return i, outs[i] / p[i]"),
    "partial_trace_transposed": ('red = np.einsum("aiaj->ij", t)', 'red = np.einsum("aiaj->ji", t)'),
    "expectation_conjugated_pauli": ("np.trace(rho @ pauli_matrix(n, term))",
                                     "np.trace(rho @ pauli_matrix(n, term).conj())"),
}


def _scratch_tree(dst):
    """The pins' imports (oracle, oracle.noise, circuits) in a tree of their own."""
    os.makedirs(os.path.join(dst, "tests"))
    for f in ("conftest.py", "test_oracle_noise_pins.py"):
        shutil.copy2(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    os.makedirs(os.path.join(dst, "oracle"))
    for f in ("__init__.py", "hq_oracle.c", "noise.py"):
        shutil.copy2(os.path.join(ROOT, "oracle", f), os.path.join(dst, "oracle", f))
    os.makedirs(os.path.join(dst, "paper_2111_06868_gb300"))
    for f in ("__init__.py", "circuits.py"):
        shutil.copy2(os.path.join(ROOT, "paper_2111_06868_gb300", f), os.path.join(dst, "paper_2111_06868_gb300", f))


@pytest.fixture(scope="module")
def oracle_lib():
    import oracle

    return oracle.build()


def _run_pins(tree, lib):
    env = dict(os.environ, HQ_ORACLE_LIB=lib)
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(tree, "tests", "test_oracle_noise_pins.py")],
                          cwd=tree, env=env, capture_output=True, text=True, timeout=300)


def test_unmutated_copy_passes(tmp_path, oracle_lib):
    """The scratch tree itself is sound: the unchanged copy passes its pins."""
    _scratch_tree(str(tmp_path))
    r = _run_pins(str(tmp_path), oracle_lib)
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, tmp_path, oracle_lib):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    _scratch_tree(str(tmp_path))
    with open(os.path.join(str(tmp_path), "oracle", "noise.py"), "w") as f:
        f.write(src.replace(old, new))
    r = _run_pins(str(tmp_path), oracle_lib)
    assert r.returncode != 0, f"the pins did not catch the planted mistake {name}:\n{r.stdout[-2000:]}"
