"""The gate fuser's planning on the host (no GPU): the fused blocks, applied
one after another by the FP64 oracle, give the same state as the original
gates applied one by one (Sec. II, gate fusion), every block has at most
max_k qubits, and fusing cuts the number of passes."""
import numpy as np
import pytest

import oracle
from paper_1604_06460_gb300 import build as B
from paper_1604_06460_gb300 import inputs as I
from paper_1604_06460_gb300 import qe


@pytest.fixture(scope="module")
def lib():
    B.build()
    return qe.load()


def apply_all(psi, ops):
    for q, U in ops:
        psi = oracle.apply_gate(psi, list(q), U)
    return psi


@pytest.mark.parametrize("max_k", [1, 2, 3, 4, 5])
def test_blocks_reproduce_the_circuit(lib, max_k):
    n = 9
    gates = I.random_circuit(n, 6, seed=max_k)
    blocks = qe.plan_fusion(n, gates, max_k)
    # max_k = 1: no fusion, every gate is its own block (CNOTs keep 2 qubits)
    assert all(1 <= len(q) <= max(max_k, 2) for q, _ in blocks)
    if max_k > 1:
        assert all(len(q) <= max_k for q, _ in blocks)
    psi = I.random_state(n, 3)
    want = apply_all(psi, [(g.qubits, g.matrix) for g in gates])
    got = apply_all(psi, blocks)
    assert np.max(np.abs(got - want)) < 1e-12
    if max_k == 1:
        assert len(blocks) == len(gates)
    else:
        assert len(blocks) < len(gates) / max_k * 1.5


def test_blocks_are_unitary_and_ordered_on_shared_qubits(lib):
    # gates that overlap in a chain force closing and reopening of blocks
    n = 7
    rng = np.random.default_rng(4)
    gates = []
    for t in range(40):
        a = int(rng.integers(0, n - 1))
        gates.append(I.Gate([a, a + 1], np.kron(I.haar_u2(rng), I.haar_u2(rng))))
    for max_k in (2, 3, 5):
        blocks = qe.plan_fusion(n, gates, max_k)
        for q, U in blocks:
            assert np.allclose(U.conj().T @ U, np.eye(len(U)), atol=1e-12)
        psi = I.random_state(n, 9)
        want = apply_all(psi, [(g.qubits, g.matrix) for g in gates])
        assert np.max(np.abs(apply_all(psi, blocks) - want)) < 1e-12


@pytest.mark.parametrize("max_k", [2, 3, 4, 5])
def test_mixed_width_gates(lib, max_k):
    # gates of 1..5 qubits; those wider than max_k stay passes of their own
    # and the blocks around them keep the order on their shared qubits
    n = 8
    rng = np.random.default_rng(40 + max_k)
    gates = []
    for _ in range(60):
        w = int(rng.integers(1, 6))
        qs = [int(v) for v in rng.permutation(n)[:w]]
        z = rng.standard_normal((1 << w, 1 << w)) + 1j * rng.standard_normal((1 << w, 1 << w))
        U, _ = np.linalg.qr(z)
        gates.append(I.Gate(tuple(qs), U))
    blocks = qe.plan_fusion(n, gates, max_k)
    for q, U in blocks:
        assert len(q) <= max(max_k, max(len(g.qubits) for g in gates))
        assert np.allclose(U.conj().T @ U, np.eye(len(U)), atol=1e-12)
    assert len(blocks) <= len(gates)
    psi = I.random_state(n, 5)
    want = apply_all(psi, [(g.qubits, g.matrix) for g in gates])
    assert np.max(np.abs(apply_all(psi, blocks) - want)) < 1e-12


def test_frontier_blocks_on_the_benchmark_circuits(lib):
    # each pass takes the qubit set that absorbs the most front gates (from
    # 30 qubits on ranked with a one-block look-ahead): on the depth-20,
    # 30-qubit random circuit 71 blocks of at most 5 qubits (86 with the
    # earlier greedy open-block planner), 114 on the depth-30, 32-qubit one
    for n, depth, seed, most in ((30, 20, 0, 71), (32, 30, 5, 114)):
        gates = I.random_circuit(n, depth, seed=seed)
        blocks = qe.plan_fusion(n, gates, 5)
        assert len(blocks) <= most
        assert all(len(q) <= 5 for q, _ in blocks)
        for q, U in blocks[:6]:
            assert np.allclose(U.conj().T @ U, np.eye(len(U)), atol=1e-12)


def test_empty_and_invalid(lib):
    assert qe.plan_fusion(4, [], 5) == []
    with pytest.raises(qe.QEError):
        qe.plan_fusion(4, [I.Gate([4], np.eye(2))], 5)      # qubit out of range
    with pytest.raises(qe.QEError):
        qe.plan_fusion(4, [I.Gate([1, 1], np.eye(4))], 5)   # repeated qubit
    with pytest.raises(qe.QEError):
        qe.plan_fusion(4, [I.Gate([0], np.eye(2))], 6)      # max_k out of range
