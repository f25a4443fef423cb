"""The named channels the package offers as inputs (circuits.py) equal the
noise oracle's pinned definitions, and the noise entry points validate
their arguments on the host."""
import numpy as np
import pytest

from oracle import noise as N
from paper_2111_06868_gb300 import circuits as C


def test_channels_equal_oracle_definitions():
    pairs = [(C.depolarizing(0.3, 1), N.depolarizing_kraus(0.3, 1)), (C.depolarizing(0.2, 2), N.depolarizing_kraus(0.2, 2)),
             (C.dephasing(0.1, "Y"), N.dephasing_kraus(0.1, "Y")),
             (C.amplitude_damping(0.4), N.amplitude_damping_kraus(0.4)),
             (C.amplitude_damping(0.4, 0.1), N.amplitude_damping_kraus(0.4, 0.1))]
    for a, b in pairs:
        assert len(a) == len(b)
        for x, y in zip(a, b):
            np.testing.assert_allclose(x, y, atol=1e-16)


def test_noisy_ops_layout():
    circ = C.random_circuit(C.grid(2, 3), 3, seed=1, two_qubit="cz")
    ops = C.noisy_ops(circ, p1=0.01, p2=0.02, gamma=0.03)
    gates = [o for o in ops if o[0] == "gate"]
    assert len(gates) == len(circ.gates)
    n1 = sum(1 for g in circ.gates if g.k == 1)
    assert sum(1 for o in ops if o[0] == "kraus") == n1 * 2 + (len(circ.gates) - n1)


def test_noise_entry_points_validate_on_the_host():
    from paper_2111_06868_gb300 import build
    from paper_2111_06868_gb300 import hq

    build.build()
    lib = hq.load()
    fake = hq.ctypes.c_void_p(1 << 20)
    q = (hq.ctypes.c_int * 3)(0, 1, 2)
    out = np.zeros(32)
    ptr = out.ctypes.data_as(hq.ctypes.c_void_p)
    assert lib.hq_reduced_density_matrix(fake, 4, 0, q, 3, ptr, None) == -4  # k > 2
    assert lib.hq_reduced_density_matrix(fake, 4, 0, q, 0, ptr, None) == -4
    assert lib.hq_reduced_density_matrix(fake, 4, 0, (hq.ctypes.c_int * 1)(4), 1, ptr, None) == -2
    assert lib.hq_reduced_density_matrix(fake, 4, 0, q, 1, None, None) == -1
    ks = np.ascontiguousarray(np.stack(C.amplitude_damping(0.1)), np.complex128)
    kp = ks.ctypes.data_as(hq.ctypes.c_void_p)
    assert lib.hq_apply_kraus_sampled(fake, 4, 0, q, 1, 2, kp, hq.ctypes.c_double(1.0), None, None) == -12
    assert lib.hq_apply_kraus_sampled(fake, 4, 0, q, 1, 0, kp, hq.ctypes.c_double(0.5), None, None) == -12
    assert lib.hq_apply_kraus_sampled(fake, 4, 0, q, 1, 2, None, hq.ctypes.c_double(0.5), None, None) == -1
    assert lib.hq_run_trajectory(fake, 4, 0, None, 1, None, None, None, None) == -1
    assert lib.hq_run_trajectory(fake, 4, 0, None, -1, None, None, None, None) == -12
