"""OpenQASM 2.0 front end and the ring u3/cz generator, on the CPU: gate
matrices against their textbook definitions and identities, the qubit
convention against a dense simulation, parse/dump round trips, error
handling, and the generator's mirrored peak."""
import math

import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from paper_2607_07816_b300 import qasm
from tests.dense import dense_run


def _close(a, b, tol=1e-12):
    return np.max(np.abs(np.asarray(a) - np.asarray(b))) <= tol


def test_single_qubit_identities():
    pi = math.pi
    assert _close(qasm.op_matrix("u3", (pi, 0, pi)), C.mat_x())
    assert _close(qasm.op_matrix("u2", (0, pi)), C.mat_h())
    for th in (0.3, 1.7, -2.2):
        # rx, ry as u3 up to no global phase (the u3 definition has none here)
        assert _close(qasm.op_matrix("ry", (th,)), qasm.op_matrix("u3", (th, 0, 0)))
        assert _close(qasm.op_matrix("rx", (th,)), qasm.op_matrix("u3", (th, -pi / 2, pi / 2)))
        # u1 = p = diag(1, e^{i l}); rz differs by a global phase
        assert _close(qasm.op_matrix("u1", (th,)), np.diag([1, np.exp(1j * th)]))
        rz = qasm.op_matrix("rz", (th,))
        assert _close(rz * np.exp(1j * th / 2), qasm.op_matrix("p", (th,)))
    s, t = qasm.op_matrix("s", ()), qasm.op_matrix("t", ())
    assert _close(t @ t, s)
    assert _close(s @ s, qasm.op_matrix("z", ()))
    sx = qasm.op_matrix("sx", ())
    assert _close(sx @ sx, C.mat_x())
    assert _close(sx @ qasm.op_matrix("sxdg", ()), np.eye(2))
    assert _close(s @ qasm.op_matrix("sdg", ()), np.eye(2))


def test_u3_inverse_rule():
    rng = np.random.default_rng(3)
    for _ in range(20):
        p = tuple(rng.uniform(-4, 4, size=3))
        u = qasm.op_matrix("u3", p)
        ui = qasm.op_matrix("u3", qasm.u3_inverse(p))
        assert _close(ui @ u, np.eye(2))


def test_every_gate_is_unitary():
    for name, ar in qasm.ARITY.items():
        params = tuple(0.37 * (i + 1) for i in range(qasm.NPARAMS.get(name, 0)))
        u = qasm.op_matrix(name, params)
        assert u.shape == (1 << ar, 1 << ar)
        assert _close(u.conj().T @ u, np.eye(1 << ar))


def test_controls_first_convention_on_dense_states():
    # Bell pair from h; cx (control q0, target q1): keys 0 and 3
    n, ops = qasm.parse("OPENQASM 2.0; qreg q[2]; h q[0]; cx q[0],q[1];")
    psi = dense_run(n, qasm.to_gates(ops))
    assert _close(np.abs(psi) ** 2, [0.5, 0, 0, 0.5])
    # x on q1 then cx q1 -> q0: key 0b11
    n, ops = qasm.parse("qreg q[2]; x q[1]; cx q[1],q[0];")
    assert _close(np.abs(dense_run(n, qasm.to_gates(ops))), [0, 0, 0, 1])
    # ccx with both controls set flips the target; with one control it does not
    n, ops = qasm.parse("qreg q[3]; x q[0]; x q[2]; ccx q[0],q[2],q[1];")
    psi = dense_run(n, qasm.to_gates(ops))
    assert abs(psi[0b111]) == pytest.approx(1.0)
    n, ops = qasm.parse("qreg q[3]; x q[0]; ccx q[0],q[2],q[1];")
    assert abs(dense_run(n, qasm.to_gates(ops))[0b001]) == pytest.approx(1.0)
    # cz and cp are symmetric in their qubits
    for g in ("cz q[0],q[1]", "cp(0.7) q[0],q[1]"):
        a = qasm.parse(f"qreg q[2]; h q[0]; h q[1]; {g};")
        b = qasm.parse(f"qreg q[2]; h q[0]; h q[1]; {g.replace('q[0],q[1]', 'q[1],q[0]')};")
        assert _close(dense_run(2, qasm.to_gates(a[1])), dense_run(2, qasm.to_gates(b[1])))


def test_parse_registers_expressions_and_comments():
    text = """OPENQASM 2.0;
include "qelib1.inc";
// two registers laid out one after the other
qreg a[2];
qreg b[3];
creg c[5];
u3(pi/2, -pi/4, 2*pi/3) a[1];   // comment
rz(-(pi - 0.5)/2) b[0];
barrier a[0], b[2];
cx a[0], b[2];
measure a[0] -> c[0];
"""
    n, ops = qasm.parse(text)
    assert n == 5
    assert [o.name for o in ops] == ["u3", "rz", "cx"]
    assert ops[0].qubits == (1,) and ops[1].qubits == (2,) and ops[2].qubits == (0, 4)
    assert ops[0].params == pytest.approx((math.pi / 2, -math.pi / 4, 2 * math.pi / 3))
    assert ops[1].params == pytest.approx((-(math.pi - 0.5) / 2,))


@pytest.mark.parametrize("bad", [
    "qreg q[2]; foo q[0];",              # unknown gate
    "qreg q[2]; cx q[0];",               # arity
    "qreg q[2]; cx q[0],q[0];",          # repeated qubit
    "qreg q[2]; h q[2];",                # out of range
    "qreg q[2]; h r[0];",                # unknown register
    "qreg q[2]; u3(1,2) q[0];",          # parameter count
    "qreg q[2]; rz(__import__) q[0];",   # not an arithmetic expression
    "qreg q[2]; reset q[0];",            # not supported
])
def test_parse_errors(bad):
    with pytest.raises(ValueError):
        qasm.parse(bad)


def test_dump_parse_round_trip():
    ops, _ = qasm.sharp_peak_like(n=12, blocks=30, seed=5)
    text = qasm.dumps(12, ops)
    n, back = qasm.parse(text)
    assert n == 12 and len(back) == len(ops)
    for a, b in zip(ops, back):
        assert a.name == b.name and a.qubits == b.qubits
        assert a.params == pytest.approx(b.params, abs=0, rel=0)


def test_sharp_peak_shape_and_exact_mirror():
    ops, hidden = qasm.sharp_peak_like()
    assert 560 <= len(ops) <= 620
    assert {o.name for o in ops} <= {"u3", "cz", "x"}
    pairs = {tuple(sorted(o.qubits)) for o in ops if o.name == "cz"}
    assert (0, 43) in pairs and (0, 1) in pairs and (42, 43) in pairs
    # the unperturbed mirror returns exactly the hidden string (dense, small ring)
    ops, hidden = qasm.sharp_peak_like(n=10, blocks=25, seed=7, sigma=0.0)
    psi = dense_run(10, qasm.to_gates(ops))
    assert abs(psi[hidden]) ** 2 == pytest.approx(1.0, abs=1e-12)


def test_sharp_peak_perturbed_is_peaked_at_hidden():
    ops, hidden = qasm.sharp_peak_like(n=10, blocks=25, seed=8, sigma=0.05)
    probs = np.abs(dense_run(10, qasm.to_gates(ops))) ** 2
    assert int(np.argmax(probs)) == hidden and probs[hidden] > 0.5
