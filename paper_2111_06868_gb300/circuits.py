"""Seeded synthetic inputs: gate definitions, grid layouts and random circuits.

This module only *describes* circuits. It holds none of the simulation
arithmetic (no gate application, no fusion, no reductions): both the CUDA path
and the CPU oracle consume the gate lists it emits, each with its own code.

Conventions (HybridQ, arXiv 2111.06868):
  * A gate is a dense 2^k x 2^k complex matrix on k named qubits (``MatrixGate``,
    Sec. 2 "Gates").  Its local basis index is r = sum_j r_j 2^(k-1-j), i.e.
    ``qubits[0]`` is the most significant local bit (the Kronecker order of the
    qubit list).
  * Qubit q of an n-qubit state is axis q of the C-order ``(2,)*n`` tensor, so it
    is bit n-1-q of the flat amplitude index (pinned by the Grover example of
    Sec. 2.2, where a flip of |00> on qubits 1,2 negates entries 000 and 100).

Random numbers come from SplitMix64 (Steele, Lea, Flood 2014; the constants are
the published ones), so the gate lists do not depend on the numpy version.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Iterable, Sequence

import numpy as np

_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (published definition: golden-gamma increment,
    two xor-shift-multiply mixing rounds)."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform in [lo, hi] (inclusive); modulo bias < 2^-58."""
        return lo + self.next_u64() % (hi - lo + 1)


# ----------------------------------------------------------------------------
# Gate matrices (inputs).  R_P(theta) = exp(-i theta P / 2).
# ----------------------------------------------------------------------------
_S2 = 1.0 / math.sqrt(2.0)
PAULI = {
    "I": np.array([[1, 0], [0, 1]], dtype=np.complex128),
    "X": np.array([[0, 1], [1, 0]], dtype=np.complex128),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=np.complex128),
    "Z": np.array([[1, 0], [0, -1]], dtype=np.complex128),
}


def sqrt_x() -> np.ndarray:
    """sqrt(X) = R_X(pi/2) = (I - iX)/sqrt(2)."""
    return _S2 * np.array([[1, -1j], [-1j, 1]], dtype=np.complex128)


def sqrt_y() -> np.ndarray:
    """sqrt(Y) = R_Y(pi/2) = (I - iY)/sqrt(2)."""
    return _S2 * np.array([[1, -1], [1, 1]], dtype=np.complex128)


def sqrt_w() -> np.ndarray:
    """sqrt(W) = R_W(pi/2), W = (X + Y)/sqrt(2)."""
    return _S2 * np.array(
        [[1, np.exp(-0.75j * math.pi)], [np.exp(-0.25j * math.pi), 1]], dtype=np.complex128
    )


def hadamard() -> np.ndarray:
    return _S2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)


def rot(axis: str, theta: float) -> np.ndarray:
    """R_P(theta) = cos(theta/2) I - i sin(theta/2) P."""
    return math.cos(theta / 2) * PAULI["I"] - 1j * math.sin(theta / 2) * PAULI[axis]


def cz() -> np.ndarray:
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def cnot() -> np.ndarray:
    """Controlled-X with control qubits[0] (local MSB) and target qubits[1]."""
    m = np.eye(4, dtype=np.complex128)
    m[2:, 2:] = PAULI["X"]
    return m


def cphase(phi: float) -> np.ndarray:
    """diag(1, 1, 1, e^{i phi})."""
    return np.diag([1, 1, 1, np.exp(1j * phi)]).astype(np.complex128)


def swap() -> np.ndarray:
    m = np.zeros((4, 4), dtype=np.complex128)
    m[0, 0] = m[1, 2] = m[2, 1] = m[3, 3] = 1
    return m


def fsim(theta: float, phi: float) -> np.ndarray:
    """fSim(theta, phi) on |q_a q_b>, q_a the local MSB."""
    c, s = math.cos(theta), math.sin(theta)
    return np.array(
        [[1, 0, 0, 0], [0, c, -1j * s, 0], [0, -1j * s, c, 0], [0, 0, 0, np.exp(-1j * phi)]],
        dtype=np.complex128,
    )


def random_unitary(k: int, rng: SplitMix64) -> np.ndarray:
    """Haar-ish random 2^k x 2^k unitary: QR of a Gaussian matrix built from
    Box-Muller draws of the seeded generator (phase-fixed R diagonal)."""
    d = 1 << k
    vals = np.empty(2 * d * d)
    for i in range(0, 2 * d * d, 2):
        u1 = max(rng.uniform(), 1e-300)
        u2 = rng.uniform()
        r = math.sqrt(-2.0 * math.log(u1))
        vals[i] = r * math.cos(2 * math.pi * u2)
        vals[i + 1] = r * math.sin(2 * math.pi * u2)
    z = (vals[0::2] + 1j * vals[1::2]).reshape(d, d)
    q, r = np.linalg.qr(z)
    ph = np.diagonal(r) / np.abs(np.diagonal(r))
    return q * ph[None, :]


# ----------------------------------------------------------------------------
# Circuit containers
# ----------------------------------------------------------------------------
@dataclass
class Gate:
    """One gate.  Either a fixed matrix (``matrix`` set) or a rotation
    exp(-i theta P/2) about ``axis`` with theta = params[``param``]."""

    name: str
    qubits: tuple
    matrix: np.ndarray | None = None
    axis: str | None = None
    param: int = -1

    @property
    def k(self) -> int:
        return len(self.qubits)

    def matrix_at(self, params: Sequence[float] | None = None) -> np.ndarray:
        if self.matrix is not None:
            return self.matrix
        return rot(self.axis, float(params[self.param]))


@dataclass
class Circuit:
    n: int
    gates: list = field(default_factory=list)
    n_params: int = 0

    def __len__(self) -> int:
        return len(self.gates)

    def inverse(self) -> "Circuit":
        """The adjoint circuit (reversed order, conjugate-transposed matrices).
        Only fixed-matrix circuits."""
        gs = []
        for g in reversed(self.gates):
            if g.matrix is None:
                raise ValueError("inverse() needs fixed-matrix gates")
            gs.append(Gate(g.name + "^+", g.qubits, np.ascontiguousarray(g.matrix.conj().T)))
        return Circuit(self.n, gs, 0)

    def bound(self, params: Sequence[float]) -> "Circuit":
        """Fixed-matrix copy with rotation angles substituted."""
        return Circuit(self.n, [Gate(g.name, g.qubits, g.matrix_at(params)) for g in self.gates], 0)

    def packed(self):
        """Flat arrays for the C boundaries: k (G,), qubits (G,6, -1 padded),
        kind (G,: 0 matrix, 1 rotation), axis (G,: 0 or ord('X'/'Y'/'Z')),
        param (G,), matrices (concatenated row-major complex128), offsets (G,)
        in complex elements (-1 for rotations)."""
        G = len(self.gates)
        ks = np.zeros(G, np.int32)
        qs = np.full((G, 6), -1, np.int32)
        kind = np.zeros(G, np.int32)
        axis = np.zeros(G, np.int32)
        param = np.full(G, -1, np.int32)
        offs = np.full(G, -1, np.int64)
        mats = []
        off = 0
        for i, g in enumerate(self.gates):
            ks[i] = g.k
            qs[i, : g.k] = g.qubits
            if g.matrix is not None:
                m = np.ascontiguousarray(g.matrix, dtype=np.complex128).ravel()
                mats.append(m)
                offs[i] = off
                off += m.size
            else:
                kind[i] = 1
                axis[i] = ord(g.axis)
                param[i] = g.param
        mat = np.concatenate(mats) if mats else np.zeros(0, np.complex128)
        return dict(k=ks, qubits=qs, kind=kind, axis=axis, param=param, matrices=mat, offsets=offs)


# Pauli sums: list of (coeff, ((qubit, 'X'|'Y'|'Z'), ...)).
PauliSum = list


# ----------------------------------------------------------------------------
# Grid layouts and the four cycling nearest-neighbour edge patterns
# ----------------------------------------------------------------------------
@dataclass
class Layout:
    rows: int
    cols: int
    sites: list  # kept (r, c), row-major; qubit index = position in this list

    @property
    def n(self) -> int:
        return len(self.sites)

    def qubit(self, r: int, c: int) -> int | None:
        try:
            return self._index[(r, c)]
        except KeyError:
            return None

    def __post_init__(self):
        self._index = {s: i for i, s in enumerate(self.sites)}

    def pattern(self, which: int) -> list:
        """Edges of pattern A (0): horizontal, even column; B (1): horizontal,
        odd column; C (2): vertical, even row; D (3): vertical, odd row.  Edges
        touching a removed site are dropped.  Returned as (qubit_a, qubit_b)."""
        edges = []
        for (r, c) in self.sites:
            if which in (0, 1):
                if c % 2 != which:
                    continue
                other = (r, c + 1)
            else:
                if r % 2 != which - 2:
                    continue
                other = (r + 1, c)
            qa, qb = self.qubit(r, c), self.qubit(*other)
            if qa is not None and qb is not None:
                edges.append((qa, qb))
        return edges


def grid(rows: int, cols: int, removed: Iterable = (), first: int | None = None) -> Layout:
    removed = set(tuple(x) for x in removed)
    sites = [(r, c) for r in range(rows) for c in range(cols) if (r, c) not in removed]
    if first is not None:
        sites = sites[:first]
    return Layout(rows, cols, sites)


def layout_for(n: int) -> Layout:
    """R = floor(sqrt(n)), C = ceil(n / R), first n sites row-major."""
    R = max(1, int(math.isqrt(n)))
    C = -(-n // R)
    return grid(R, C, first=n)


ONE_QUBIT_SET = (("sqrtX", sqrt_x), ("sqrtY", sqrt_y), ("sqrtW", sqrt_w))


def random_circuit(layout: Layout, depth: int, seed: int, two_qubit: str = "cz") -> Circuit:
    """Random circuit on a grid: each layer applies to every qubit (ascending)
    a gate drawn from {sqrt(X), sqrt(Y), sqrt(W)} (uniform over 3 in layer 0,
    then uniform over the 2 that differ from the qubit's previous gate), then a
    two-qubit gate (CZ or fSim(pi/2, pi/6)) on every edge of pattern
    (layer mod 4)."""
    rng = SplitMix64(seed)
    n = layout.n
    mats = [f() for _, f in ONE_QUBIT_SET]
    names = [nm for nm, _ in ONE_QUBIT_SET]
    if two_qubit == "cz":
        m2, nm2 = cz(), "CZ"
    elif two_qubit == "fsim":
        m2, nm2 = fsim(math.pi / 2, math.pi / 6), "fSim"
    else:
        raise ValueError(two_qubit)
    prev = [-1] * n
    gates = []
    patterns = [layout.pattern(p) for p in range(4)]
    for layer in range(depth):
        for q in range(n):
            if prev[q] < 0:
                choice = rng.randint(0, 2)
            else:
                others = [i for i in range(3) if i != prev[q]]
                choice = others[rng.randint(0, 1)]
            prev[q] = choice
            gates.append(Gate(names[choice], (q,), mats[choice]))
        for (a, b) in patterns[layer % 4]:
            gates.append(Gate(nm2, (a, b), m2))
    return Circuit(n, gates)


def random_dense_circuit(n: int, n_gates: int, seed: int, kmax: int = 3) -> Circuit:
    """Random Haar-ish k-qubit gates (k uniform in 1..kmax) on random distinct
    qubits; exercises every bit-position class."""
    rng = SplitMix64(seed)
    gates = []
    for _ in range(n_gates):
        k = rng.randint(1, min(kmax, n))
        qs = []
        while len(qs) < k:
            q = rng.randint(0, n - 1)
            if q not in qs:
                qs.append(q)
        gates.append(Gate(f"U{k}", tuple(qs), random_unitary(k, rng)))
    return Circuit(n, gates)


# ----------------------------------------------------------------------------
# The five workloads
# ----------------------------------------------------------------------------
def config_small(seed: int = 0) -> Circuit:
    """n=12 on a 3x4 grid, depth 10, CZ entanglers (120 + 43 gates)."""
    return random_circuit(grid(3, 4), 10, seed, "cz")


def config_n30(seed: int = 0) -> Circuit:
    """n=30 on a 5x6 grid, depth 20, fSim(pi/2, pi/6) entanglers (600 + 245 gates)."""
    return random_circuit(grid(5, 6), 20, seed, "fsim")


SITES_33 = dict(rows=6, cols=6, removed=((0, 5), (5, 0), (5, 5)))


def config_n33(seed: int = 0, first: int | None = None) -> Circuit:
    """n=33 on a 6x6 grid minus corners (0,5),(5,0),(5,5), depth 24, fSim
    (792 + 324 gates).  ``first=28`` gives the 28-qubit subset (first 28 kept
    sites row-major, induced edges, same generator)."""
    return random_circuit(grid(first=first, **SITES_33), 24, seed, "fsim")


def ansatz(n: int = 20, layers: int = 8) -> Circuit:
    """Variational ansatz: per layer RY(theta) then RZ(phi) on every qubit,
    then CZ(i, i+1) for i = 0..n-2.  Parameter index (layer*n + q)*2 + {0: RY,
    1: RZ}."""
    gates = []
    for layer in range(layers):
        for q in range(n):
            base = (layer * n + q) * 2
            gates.append(Gate("RY", (q,), None, "Y", base))
            gates.append(Gate("RZ", (q,), None, "Z", base + 1))
        for q in range(n - 1):
            gates.append(Gate("CZ", (q, q + 1), cz()))
    return Circuit(n, gates, layers * n * 2)


def ansatz_hamiltonian(n: int = 20) -> PauliSum:
    """H = sum_{i=0}^{n-2} Z_i Z_{i+1} + 0.5 sum_{i=0}^{n-1} X_i (open chain)."""
    h = [(1.0, ((i, "Z"), (i + 1, "Z"))) for i in range(n - 1)]
    h += [(0.5, ((i, "X"),)) for i in range(n)]
    return h


def ansatz_params(n_params: int, batch: int, seed: int) -> np.ndarray:
    """(batch, n_params) angles uniform in [0, 2 pi)."""
    rng = SplitMix64(seed)
    out = np.empty((batch, n_params), np.float64)
    for b in range(batch):
        for p in range(n_params):
            out[b, p] = 2 * math.pi * rng.uniform()
    return out


def config_batch(count: int = 512, seed: int = 0, n_range=(10, 24), depth_range=(8, 32)) -> list:
    """Serving-style load: ``count`` circuits, n ~ U{10..24}, depth ~ U{8..32},
    sqrt(X/Y/W) + CZ gate set on the R x C layout of ``layout_for(n)``."""
    rng = SplitMix64(seed)
    out = []
    for i in range(count):
        n = rng.randint(*n_range)
        d = rng.randint(*depth_range)
        out.append(random_circuit(layout_for(n), d, seed * 1_000_003 + i, "cz"))
    return out


def ghz_circuit(n: int) -> Circuit:
    gates = [Gate("H", (0,), hadamard())]
    gates += [Gate("CNOT", (i, i + 1), cnot()) for i in range(n - 1)]
    return Circuit(n, gates)


def qft_circuit(n: int) -> Circuit:
    """Textbook QFT with qubit 0 as the most significant bit: H and controlled
    phases 2 pi / 2^(m-j+1), then the bit-reversal swaps."""
    gates = []
    for j in range(n):
        gates.append(Gate("H", (j,), hadamard()))
        for m in range(j + 1, n):
            gates.append(Gate("CPHASE", (m, j), cphase(2 * math.pi / (1 << (m - j + 1)))))
    for j in range(n // 2):
        gates.append(Gate("SWAP", (j, n - 1 - j), swap()))
    return Circuit(n, gates)


def basis_prep(n: int, x: int) -> Circuit:
    """X gates that take |0..0> to |x> (qubit q carries bit n-1-q of x)."""
    return Circuit(n, [Gate("X", (q,), PAULI["X"].copy()) for q in range(n) if (x >> (n - 1 - q)) & 1])


def pauli_string(n: int, term) -> str:
    s = ["I"] * n
    for q, p in term:
        s[q] = p
    return "".join(s)


# ----------------------------------------------------------------------------
# Noise channels (Sec. 2.1 "Noisy gates") as Kraus operator lists, and noisy
# circuits as operation lists ("gate", qubits, matrix) / ("kraus", qubits, Ks)
# ----------------------------------------------------------------------------
def depolarizing(p: float, k: int = 1) -> list:
    """rho -> (1 - p) rho + p I / 2^k on k qubits, as Kraus operators: every
    k-fold Pauli product P with weight p / 4^k, plus 1 - p on the identity."""
    out = []
    paulis = [""]
    for _ in range(k):
        paulis = [s + c for s in paulis for c in "IXYZ"]
    for s in paulis:
        m = np.ones((1, 1), dtype=np.complex128)
        for c in s:
            m = np.kron(m, PAULI[c])
        weight = p / 4 ** k + (1.0 - p if s == "I" * k else 0.0)
        out.append(math.sqrt(weight) * m)
    return out


def dephasing(p: float, sigma: str = "Z") -> list:
    """rho -> (1 - p) rho + p sigma rho sigma."""
    return [math.sqrt(1.0 - p) * PAULI["I"], math.sqrt(p) * PAULI[sigma]]


def amplitude_damping(gamma: float, excitation: float = 0.0) -> list:
    """Decay |1> -> |0> at rate gamma, and |0> -> |1> at the excitation rate."""
    ops = [np.diag([math.sqrt(1.0 - excitation), math.sqrt(1.0 - gamma)]).astype(np.complex128),
           math.sqrt(gamma) * np.array([[0, 1], [0, 0]], dtype=np.complex128)]
    if excitation > 0:
        ops.append(math.sqrt(excitation) * np.array([[0, 0], [1, 0]], dtype=np.complex128))
    return ops


def noisy_ops(circuit: Circuit, p1: float = 0.0, p2: float = 0.0, gamma: float = 0.0) -> list:
    """The circuit's gates with a depolarizing channel after each one (p1 for
    one-qubit, p2 for two-qubit gates) and amplitude damping (gamma) on the
    qubit of every one-qubit gate."""
    ops = []
    for g in circuit.gates:
        ops.append(("gate", tuple(g.qubits), g.matrix))
        p = p1 if g.k == 1 else p2
        if p > 0 and g.k <= 2:
            ops.append(("kraus", tuple(g.qubits), depolarizing(p, g.k)))
        if gamma > 0 and g.k == 1:
            ops.append(("kraus", tuple(g.qubits), amplitude_damping(gamma)))
    return ops
