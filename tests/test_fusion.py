"""Gate reordering and fusion front end, on the CPU: the circuit's result is
unchanged (dense simulation), dependencies are respected, blocks stay within
the qubit limit, and new qubits are postponed."""
import numpy as np
import pytest

from paper_2607_07816_b300 import circuits as C
from paper_2607_07816_b300 import fusion, qasm
from tests.dense import dense_run


def _random_gates(n, count, rng):
    out = []
    for _ in range(count):
        m = int(rng.integers(1, 4))
        out.append(C.random_gate(n, m, rng, "haar"))
    return out


def _per_qubit_sequences(gates):
    seq = {}
    for j, (q, u) in enumerate(gates):
        for x in q:
            seq.setdefault(x, []).append(id(u))
    return seq


@pytest.mark.parametrize("seed", range(4))
def test_reorder_keeps_dependencies_and_result(seed):
    rng = np.random.default_rng(seed)
    n = 9
    gates = _random_gates(n, 40, rng)
    re = fusion.reorder(gates)
    assert sorted(map(id, (u for _, u in re))) == sorted(map(id, (u for _, u in gates)))
    assert _per_qubit_sequences(re) == _per_qubit_sequences(gates)
    assert np.max(np.abs(dense_run(n, re) - dense_run(n, gates))) <= 1e-12


def test_reorder_postpones_new_qubits():
    h = C.mat_h()
    cz = C.mat_cz()
    # q2 and q3 are brought in by the second gate; the later gates on q0, q1
    # do not depend on them and move ahead
    gates = [((0, 1), cz), ((2, 3), cz), ((0,), h), ((1,), h), ((0, 1), cz)]
    re = fusion.reorder([((0,), h)] + gates)
    names = [q for q, _ in re]
    assert names.index((2, 3)) == len(names) - 1
    prof = fusion.active_profile(re)
    assert prof[-2] == 2 and prof[-1] == 4


@pytest.mark.parametrize("maxq", [1, 2, 3, 4])
def test_fuse_keeps_result_and_limit(maxq):
    rng = np.random.default_rng(10 + maxq)
    n = 8
    gates = [g for g in _random_gates(n, 50, rng) if len(g[0]) <= maxq]
    fused = fusion.fuse(gates, maxq)
    assert all(len(q) <= maxq for q, _ in fused)
    assert all(list(q) == sorted(q) for q, _ in fused)
    assert len(fused) <= len(gates)
    for q, u in fused:
        d = 1 << len(q)
        assert np.max(np.abs(u.conj().T @ u - np.eye(d))) <= 1e-12
    assert np.max(np.abs(dense_run(n, fused) - dense_run(n, gates))) <= 1e-12


def test_fuse_rejects_wide_gates():
    with pytest.raises(ValueError):
        fusion.fuse([((0, 1, 2), np.eye(8))], 2)
    with pytest.raises(ValueError):
        fusion.fuse([], 5)


def test_embed_matches_dense_on_block():
    rng = np.random.default_rng(4)
    u = C.haar_unitary(4, rng)
    block = (1, 3, 6)
    E = fusion.embed((6, 1), u, block)
    # apply both ways on a random 3-qubit state laid out on qubits 1, 3, 6 of 7
    n = 7
    psi0 = np.zeros(1 << n, dtype=np.complex128)
    v = rng.standard_normal(8) + 1j * rng.standard_normal(8)
    for r in range(8):
        key = sum(((r >> k) & 1) << block[k] for k in range(3))
        psi0[key] = v[r]
    from tests.dense import dense_apply
    a = dense_apply(psi0, n, (6, 1), u)
    b = dense_apply(psi0, n, block, E)
    assert np.max(np.abs(a - b)) <= 1e-13


def test_ring_circuit_fuses_into_pair_blocks():
    ops, hidden = qasm.sharp_peak_like(n=12, blocks=30, seed=3)
    gates = qasm.to_gates(ops)
    fused = fusion.fuse(gates, 2)
    xs = sum(1 for o in ops if o.name == "x")
    # one block per (u3, u3, cz); the X layer fuses pairwise-adjacent single gates
    assert len([1 for q, _ in fused if len(q) == 2]) >= 2 * 30 - 2
    assert len(fused) <= 2 * 30 + xs
    full = fusion.prepare(gates, 2)
    assert np.max(np.abs(dense_run(12, full) - dense_run(12, gates))) <= 1e-11
    probs = np.abs(dense_run(12, full)) ** 2
    assert int(np.argmax(probs)) == hidden
