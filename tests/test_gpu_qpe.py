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


# ------------------------------------------- tensor-core matrix products
def matrix_state(qe, k, M):
    st = qe.State(2 * k, "c128")
    st.set(np.ascontiguousarray(M.T).reshape(-1))     # column-major storage
    return st


def product(qe, k, A, B, fp64=False):
    import os
    if fp64:
        os.environ["QE_GEMM_F64"] = "1"
    try:
        with matrix_state(qe, k, A) as sa, matrix_state(qe, k, B) as sb, qe.State(2 * k, "c128") as sc:
            sc.profile(True)
            sc.matmul(sa, sb)
            prof = sc.profile_read()
            C = as_matrix(sc, k)
    finally:
        os.environ.pop("QE_GEMM_F64", None)
    return C, prof


def long_double_rows(A, B, rows):
    a = A[rows].astype(np.clongdouble)
    return a @ B.astype(np.clongdouble)


@pytest.mark.parametrize("k", [6, 7, 8, 9])
def test_matmul_tensor_cores_vs_long_double(qe, k):
    # Gaussian complex matrices: every element of the tensor-core product
    # within K rowmax(A) colmax(B) 2^-51 of the long-double product (the
    # 56-bit splitting bound), and the path must be the tensor cores
    D = 1 << k
    rng = np.random.default_rng(10 + k)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    B = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    C, prof = product(qe, k, A, B)
    assert "oz_zgemm" in prof and "zgemm" not in prof, prof
    C64, prof64 = product(qe, k, A, B, fp64=True)
    assert "zgemm" in prof64 and "oz_zgemm" not in prof64
    rows = np.arange(D) if k <= 8 else rng.choice(D, 48, replace=False)
    ref = long_double_rows(A, B, rows)
    rowmax = np.max(np.maximum(np.abs(A.real), np.abs(A.imag)), axis=1)[rows][:, None]
    colmax = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)[None, :]
    bound = D * rowmax * colmax * 2.0 ** -51
    err = np.abs(C[rows].astype(np.clongdouble) - ref).astype(float)
    assert np.all(err <= bound)
    err64 = np.abs(C64[rows].astype(np.clongdouble) - ref).astype(float)
    # typical errors of both products are rounding-level
    assert np.max(err / (rowmax * colmax)) < 64 * 2.0 ** -52
    assert np.max(err64 / (rowmax * colmax)) < D * 2.0 ** -52


def test_matmul_tensor_cores_scales_and_exact_cases(qe):
    # rows of A and columns of B scaled by 2^-300 .. 2^300: each element keeps
    # its relative accuracy; identity and permutation products are exact;
    # a zero row and a zero column give zeros
    k = 7
    D = 1 << k
    rng = np.random.default_rng(3)
    A = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    B = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
    er = rng.integers(-300, 300, D)
    fc = rng.integers(-300, 300, D)
    As = A * np.ldexp(1.0, er)[:, None]
    Bs = B * np.ldexp(1.0, fc)[None, :]
    As[5] = 0
    Bs[:, 9] = 0
    C, _ = product(qe, k, As, Bs)
    ref = long_double_rows(A, B, np.arange(D))
    got = (C * np.ldexp(1.0, -er)[:, None] * np.ldexp(1.0, -fc)[None, :]).astype(np.clongdouble)
    rowmax = np.max(np.maximum(np.abs(A.real), np.abs(A.imag)), axis=1)[:, None]
    colmax = np.max(np.maximum(np.abs(B.real), np.abs(B.imag)), axis=0)[None, :]
    mask = np.ones((D, D), bool)
    mask[5, :] = False
    mask[:, 9] = False
    err = np.abs(got - ref).astype(float)
    assert np.all(err[mask] <= (D * rowmax * colmax * 2.0 ** -51)[mask])
    assert np.all(C[5, :] == 0) and np.all(C[:, 9] == 0)
    # a permutation (identity) times B: each element is one product, within
    # colmax(B) 2^-51 of its value (the 56-bit splitting of B's column and one
    # rounding of Y, each at most 2^(E+F-57))
    perm = rng.permutation(D)
    P = np.eye(D)[perm].astype(complex)
    for Pm, want in ((np.eye(D, dtype=complex), B), (P, B[perm])):
        Cp, _ = product(qe, k, Pm, B)
        assert np.all(np.abs(Cp - want) <= colmax * 2.0 ** -51)


@pytest.mark.parametrize("nsys,b", [(6, 3), (7, 2)])
def test_qpe_tensor_core_squaring_vs_oracle(qe, nsys, b):
    # nsys >= 6: the powers U^(2^j) come from the tensor-core product
    gates = tfim_step(nsys)
    psi = I.random_state(nsys, 70 + nsys)
    ref = oracle.qpe_circuit(psi, nsys, b, gates)
    n = nsys + b
    with dense_on_gpu(qe, nsys, gates) as u, qe.State(n, "c128") as st:
        full = np.zeros(1 << n, complex)
        full[: 1 << nsys] = psi
        st.set(full)
        st.profile(True)
        st.qpe_emulate(nsys, b, u)
        prof = st.profile_read()
        got = st.get()
    assert "oz_zgemm" in prof
    assert np.max(np.abs(got - ref)) < 1e-12
    assert oracle.fidelity(ref, got) > 1 - 1e-10


def test_qpe_tensor_core_controlled_powers_vs_oracle(qe):
    # 2^7 = 128 rows per controlled power (nsys = 6, b = 8): the controlled
    # products run on the tensor cores too
    nsys, b = 6, 8
    gates = tfim_step(nsys)
    psi = I.random_state(nsys, 91)
    ref = oracle.qpe_circuit(psi, nsys, b, gates)
    n = nsys + b
    with dense_on_gpu(qe, nsys, gates) as u, qe.State(n, "c128") as st:
        full = np.zeros(1 << n, complex)
        full[: 1 << nsys] = psi
        st.set(full)
        st.profile(True)
        st.qpe_emulate(nsys, b, u)
        prof = st.profile_read()
        got = st.get()
    assert prof["oz_zgemm"][0] == 2 * b - 1 and "zgemm_controlled" not in prof, prof
    assert np.max(np.abs(got - ref)) < 1e-12
    assert oracle.fidelity(ref, got) > 1 - 1e-10
