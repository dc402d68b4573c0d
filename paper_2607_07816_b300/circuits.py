"""Seeded synthetic circuit generators (inputs only).

This module produces the gate lists that both the CUDA path and the CPU
oracle consume.  It holds none of the simulation arithmetic: it only draws
unitaries and lays out gate sequences.  Every gate is a pair
``(qubits, U)`` where ``qubits`` is a tuple of m distinct qubit indices and
``U`` is a complex128 ``(2**m, 2**m)`` numpy array acting on the local index
``r = sum_t bit(key, qubits[t]) << t`` (so ``qubits[0]`` is the least
significant bit of ``r``), row-major ``U[r_out, r_in]``.  This is the
2^m x 2^m generalisation of the single-qubit rule of Eq. (3) (Sec. I and
Sec. IV-A of the paper).  Controlled gates list their controls first and the
target last.

The workload shapes follow the paper's application (Sec. VI): peaked
circuits built from random-looking layers followed by layers that undo them
and mark a hidden bit string.  The paper's own circuits are not available, so
mirrored circuits with a known peak stand in for them.
"""
from __future__ import annotations

import dataclasses
from typing import List, Sequence, Tuple

import numpy as np

Gate = Tuple[Tuple[int, ...], np.ndarray]

SQRT1_2 = 0.7071067811865476  # correctly rounded 1/sqrt(2)


@dataclasses.dataclass
class Circuit:
    """A gate list on ``n`` qubits with the hidden string it peaks on."""

    n: int
    gates: List[Gate]
    hidden: int = 0          # bit i = s_i (qubit i <-> key bit i)
    K: int = 1 << 62
    p: float = 1.0
    name: str = ""

    @property
    def num_gates(self) -> int:
        return len(self.gates)


def splitmix64(x: int) -> int:
    """SplitMix64 finaliser (Steele et al.), used to derive per-item seeds."""
    x = (x + 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF
    z = x
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & 0xFFFFFFFFFFFFFFFF
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & 0xFFFFFFFFFFFFFFFF
    return z ^ (z >> 31)


# ---------------------------------------------------------------- matrices
def haar_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed U(d) via QR of a complex Ginibre matrix with the
    phases of R's diagonal divided out (Mezzadri's construction)."""
    z = (rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))) / np.sqrt(2.0)
    q, r = np.linalg.qr(z)
    ph = np.diag(r) / np.abs(np.diag(r))
    return q * ph[None, :]


def haar_special_unitary(d: int, rng: np.random.Generator) -> np.ndarray:
    u = haar_unitary(d, rng)
    det = np.linalg.det(u)
    return u / det ** (1.0 / d)


def random_hermitian_unit(d: int, rng: np.random.Generator) -> np.ndarray:
    a = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    g = (a + a.conj().T) / 2.0
    return g / np.linalg.norm(g)


def expm_hermitian(g: np.ndarray, theta: float) -> np.ndarray:
    """exp(-i theta G) for Hermitian G through its eigendecomposition."""
    w, v = np.linalg.eigh(g)
    return (v * np.exp(-1j * theta * w)[None, :]) @ v.conj().T


def perturbed_inverse(u: np.ndarray, rng: np.random.Generator, sigma: float) -> np.ndarray:
    """U^dagger . exp(-i theta G), theta ~ N(0, sigma), G unit-norm Hermitian.
    With sigma == 0 this is the exact inverse."""
    if sigma == 0.0:
        return u.conj().T.copy()
    g = random_hermitian_unit(u.shape[0], rng)
    theta = rng.normal(0.0, sigma)
    return u.conj().T @ expm_hermitian(g, theta)


def mat_x() -> np.ndarray:
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def mat_h() -> np.ndarray:
    return np.array([[SQRT1_2, SQRT1_2], [SQRT1_2, -SQRT1_2]], dtype=np.complex128)


def mat_rz(theta: float) -> np.ndarray:
    return np.diag([np.exp(-0.5j * theta), np.exp(0.5j * theta)]).astype(np.complex128)


def mat_cz() -> np.ndarray:
    return np.diag([1, 1, 1, -1]).astype(np.complex128)


def mat_mcx(m: int) -> np.ndarray:
    """Multi-controlled X on m qubits: controls are local bits 0..m-2, the
    target is local bit m-1 (CNOT for m=2, Toffoli for m=3, C3X for m=4)."""
    d = 1 << m
    u = np.zeros((d, d), dtype=np.complex128)
    ctrl = (1 << (m - 1)) - 1
    tbit = 1 << (m - 1)
    for r in range(d):
        r2 = r ^ tbit if (r & ctrl) == ctrl else r
        u[r2, r] = 1.0
    return u


def mat_swap() -> np.ndarray:
    u = np.zeros((4, 4), dtype=np.complex128)
    for r in range(4):
        u[((r & 1) << 1) | (r >> 1), r] = 1.0
    return u


# ---------------------------------------------------------------- layouts
def brickwork_pairs(n: int, layer: int) -> List[Tuple[int, int]]:
    start = layer % 2
    return [(i, i + 1) for i in range(start, n - 1, 2)]


def mirror(gates: Sequence[Gate], rng: np.random.Generator, sigma: float) -> List[Gate]:
    """Reversed gate order, each gate replaced by its (perturbed) inverse."""
    return [(q, perturbed_inverse(u, rng, sigma)) for (q, u) in reversed(list(gates))]


def x_layer(hidden: int, n: int) -> List[Gate]:
    return [((i,), mat_x()) for i in range(n) if (hidden >> i) & 1]


def draw_hidden(n: int, rng: np.random.Generator) -> int:
    bits = rng.integers(0, 2, size=n)
    return int(sum(int(b) << i for i, b in enumerate(bits)))


def brickwork_circuit(n: int, layers: int, seed: int, sigma: float, K: int, p: float,
                      name: str = "") -> Circuit:
    """Brickwork of Haar SU(4) gates, then the (perturbed) mirror, then X on
    the hidden string's one-bits."""
    rng = np.random.default_rng(seed)
    hidden = draw_hidden(n, rng)
    fwd: List[Gate] = []
    for layer in range(layers):
        for (a, b) in brickwork_pairs(n, layer):
            fwd.append(((a, b), haar_special_unitary(4, rng)))
    gates = fwd + mirror(fwd, rng, sigma) + x_layer(hidden, n)
    return Circuit(n=n, gates=gates, hidden=hidden, K=K, p=p, name=name)


def exact_mirror_n12(seed: int = 1001) -> Circuit:
    """n=12, 3 brickwork layers of Haar SU(4), the exact inverse, X^s;
    K=4096, p=1 (no truncation).  The output is |s> with probability 1."""
    return brickwork_circuit(12, 3, seed, 0.0, K=4096, p=1.0, name="n12_exact_mirror")


def brickwork_n40(seed: int = 1002, layers: int = 8, K: int = 1 << 24, p: float = 1.0) -> Circuit:
    """n=40, 8 brickwork layers of Haar SU(4), perturbed mirror
    (theta ~ N(0, 0.05)), X^s; top-K truncation after every gate."""
    return brickwork_circuit(40, layers, seed, 0.05, K=K, p=p, name="n40_brickwork")


def random_mix_circuit(n: int, num_gates: int, seed: int, sigma: float, K: int, p: float,
                       name: str = "") -> Circuit:
    """Gates drawn uniformly from {H, CNOT, CZ, RZ, Toffoli, C3X, Haar U(8)}
    on uniformly drawn distinct qubits (controls first), then the perturbed
    mirror and X^s."""
    rng = np.random.default_rng(seed)
    hidden = draw_hidden(n, rng)
    kinds = ["h", "cnot", "cz", "rz", "toffoli", "c3x", "haar3"]
    fwd: List[Gate] = []
    for _ in range(num_gates):
        kind = kinds[int(rng.integers(0, len(kinds)))]
        if kind == "h":
            m, u = 1, mat_h()
        elif kind == "rz":
            m, u = 1, mat_rz(float(rng.uniform(0.0, 2.0 * np.pi)))
        elif kind == "cnot":
            m, u = 2, mat_mcx(2)
        elif kind == "cz":
            m, u = 2, mat_cz()
        elif kind == "toffoli":
            m, u = 3, mat_mcx(3)
        elif kind == "c3x":
            m, u = 4, mat_mcx(4)
        else:
            m, u = 3, haar_unitary(8, rng)
        qs = tuple(int(q) for q in rng.choice(n, size=m, replace=False))
        fwd.append((qs, u))
    gates = fwd + mirror(fwd, rng, sigma) + x_layer(hidden, n)
    return Circuit(n=n, gates=gates, hidden=hidden, K=K, p=p, name=name)


def mix_n60(seed: int = 1003, num_gates: int = 400, K: int = 1 << 26, p: float = 0.9999) -> Circuit:
    return random_mix_circuit(60, num_gates, seed, 0.05, K=K, p=p, name="n60_mix")


def batch_circuits(count: int = 512, seed: int = 1004, n_range=(16, 48), depth_range=(2, 10),
                   k_range=(10, 20)) -> List[Circuit]:
    """Mirrored brickwork peaked circuits of uneven n, depth and K."""
    out = []
    for j in range(count):
        s = splitmix64(seed ^ j)
        rng = np.random.default_rng(s)
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        c = brickwork_circuit(n, depth, int(s & 0x7FFFFFFF), 0.05, K=1 << k, p=1.0,
                              name=f"batch_{j}")
        out.append(c)
    return out


def serving_request(j: int, seed: int = 1005, large_frac: float = 0.02, large=(56, 12, 25),
                    n_range=(16, 48), depth_range=(2, 10), k_range=(10, 20)) -> Circuit:
    """Request j of the serving stream: a mirrored brickwork peaked circuit
    drawn like batch_circuits, except that a large_frac share are large
    ones of (n, forward depth, log2 K) = large."""
    s = splitmix64(seed ^ (j * 0x9E3779B97F4A7C15 & 0xFFFFFFFFFFFFFFFF))
    rng = np.random.default_rng(s)
    if rng.random() < large_frac:
        n, depth, k = large
        name = f"serve_{j}_large"
    else:
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        depth = int(rng.integers(depth_range[0], depth_range[1] + 1))
        k = int(rng.integers(k_range[0], k_range[1] + 1))
        name = f"serve_{j}"
    return brickwork_circuit(n, depth, int(s & 0x7FFFFFFF), 0.05, K=1 << k, p=1.0, name=name)


def random_gate(n: int, m: int, rng: np.random.Generator, kind: str = "haar") -> Gate:
    """One gate on m distinct random qubits (parity fuzzing)."""
    qs = tuple(int(q) for q in rng.choice(n, size=m, replace=False))
    if kind == "haar":
        u = haar_unitary(1 << m, rng)
    elif kind == "mcx":
        u = mat_mcx(m) if m >= 2 else mat_x()
    elif kind == "h":
        qs = qs[:1]
        u = mat_h()
    else:
        raise ValueError(kind)
    return (qs, u)


def random_state(n: int, count: int, rng: np.random.Generator, dist: str = "gauss",
                 ties: bool = False):
    """Distinct random keys below 2**n with complex amplitudes, normalised.
    With ``ties`` some magnitudes are duplicated exactly (forced equal
    probabilities)."""
    count = min(count, 1 << n)
    if n <= 20:
        keys = rng.choice(1 << n, size=count, replace=False).astype(np.uint64)
    else:
        keys = np.unique(rng.integers(0, 1 << n, size=int(count * 1.1) + 8, dtype=np.uint64))
        rng.shuffle(keys)
        keys = keys[:count]
    if dist == "gauss":
        amps = (rng.standard_normal(count) + 1j * rng.standard_normal(count)) / np.sqrt(2.0)
    else:
        amps = np.exp(2j * np.pi * rng.random(count)) * rng.random(count)
    if ties and count > 4:
        idx = rng.choice(count, size=count // 3, replace=False)
        src = rng.choice(count, size=count // 3, replace=True)
        amps[idx] = amps[src]
    amps = amps / np.sqrt(np.sum(np.abs(amps) ** 2))
    return keys, amps.astype(np.complex128)
