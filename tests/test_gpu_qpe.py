"""Phase estimation by emulation (Sec. III-C) through the C ABI: the dense
matrix of a circuit built on the GPU, FP64 matrix products, and the emulated
phase estimation against the oracle's gate-by-gate circuit."""
import numpy as np
import pytest

import oracle
from paper_1604_06460_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qe():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1604_06460_gb300 import build as B
    B.build()
    from paper_1604_06460_gb300 import qe as Q
    Q.load()
    return Q


def tfim_step(n):
    return I.tfim_trotter_step(n)


def dense_on_gpu(qe, nsys, gates, arith=None):
    st = qe.State(2 * nsys, "c128")
    if arith is not None:
        st.set_arith(arith)
    st.set_policy(qe.POLICY_AUTO, 0)
    st.init_identity(nsys)
    for g in gates:
        st.apply(g)
    st.flush()
    return st


def as_matrix(st, nsys):
    return st.get().reshape(1 << nsys, 1 << nsys).T     # column-major storage


@pytest.mark.parametrize("nsys", [3, 5, 6, 8])
def test_dense_unitary_built_from_the_identity(qe, nsys):
    gates = tfim_step(nsys) + I.random_circuit(nsys, 2, seed=nsys)
    with dense_on_gpu(qe, nsys, gates) as st:
        U = as_matrix(st, nsys)
    ref = oracle.dense_unitary(nsys, gates)
    assert len(tfim_step(nsys)) == 4 * nsys - 3
    assert np.max(np.abs(U - ref)) < 1e-12


@pytest.mark.parametrize("k", [4, 6, 7])
def test_matmul_vs_numpy(qe, k):
    ga = I.random_circuit(k, 2, seed=1)
    gb = I.random_circuit(k, 2, seed=2)
    with dense_on_gpu(qe, k, ga) as sa, dense_on_gpu(qe, k, gb) as sb, qe.State(2 * k, "c128") as sc:
        sc.matmul(sa, sb)
        A, B, C = as_matrix(sa, k), as_matrix(sb, k), as_matrix(sc, k)
    assert np.max(np.abs(C - A @ B)) < 1e-13 * (1 << k)
    with pytest.raises(qe.QEError):
        with qe.State(2 * k, "c128") as x:
            x.matmul(x, x)


@pytest.mark.parametrize("nsys,b", [(2, 3), (3, 4), (4, 5)])
def test_qpe_emulated_vs_oracle_circuit(qe, nsys, b):
    gates = tfim_step(nsys)
    psi = I.random_state(nsys, 7 + nsys)
    ref = oracle.qpe_circuit(psi, nsys, b, gates)
    n = nsys + b
    with dense_on_gpu(qe, nsys, gates) as u, qe.State(n, "c128") as st:
        full = np.zeros(1 << n, complex)
        full[: 1 << nsys] = psi
        st.set(full)
        st.qpe_emulate(nsys, b, u)
        got = st.get()
    assert np.max(np.abs(got - ref)) < 1e-12
    assert oracle.fidelity(ref, got) > 1 - 1e-10


def test_qpe_reads_exact_eigenphases(qe):
    # U diagonal with eigenvalue exp(2 pi i (3 x0 + 5 x1 + 9 x2) / 64) on |x>:
    # b = 6 ancillas read k exactly, with the system register unchanged
    nsys, b = 3, 6
    def phase(q, k):
        return I.Gate((q,), np.diag([1.0, np.exp(2j * np.pi * k / 64)]), (), "p")
    gates = [phase(0, 3), phase(1, 5), phase(2, 9)]
    with dense_on_gpu(qe, nsys, gates) as u:
        for x in range(8):
            with qe.State(nsys + b, "c128") as st:
                st.init_basis(x)
                st.qpe_emulate(nsys, b, u)
                p = np.abs(st.get()) ** 2
            k = (3 * (x & 1) + 5 * ((x >> 1) & 1) + 9 * (x >> 2)) % 64
            assert abs(p[(k << nsys) | x] - 1) < 1e-12
