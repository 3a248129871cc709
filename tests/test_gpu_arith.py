"""Emulated multiplication and division (Sec. III-A) through the C ABI
against the oracle's index maps: bit-exact, every layout of the registers,
both plane paths (shared memory, scratch batches), both state types, and the
multiplication's gate circuit on the GPU."""
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


def layout(kind, N, n):
    if kind == "paper":      # c in the low qubits, then b, then a (the paper's i = a b c)
        return list(range(2 * N, 3 * N)), list(range(N, 2 * N)), list(range(N))
    if kind == "offset":     # registers above two spectator qubits
        return list(range(2 + 2 * N, 2 + 3 * N)), list(range(2 + N, 2 + 2 * N)), list(range(2, 2 + N))
    rng = np.random.default_rng(N * 7 + n)   # scattered, unsorted qubits
    q = [int(v) for v in rng.permutation(n)[:3 * N]]
    return q[:N], q[N:2 * N], q[2 * N:]


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N,n,kind", [(1, 3, "paper"), (2, 8, "offset"), (3, 9, "paper"), (4, 14, "mixed"),
                                      (5, 15, "paper"), (6, 20, "offset"), (4, 16, "mixed")])
def test_mul_emulated_bit_exact(qe, dtype, N, n, kind):
    qa, qb, qc = layout(kind, N, n)
    psi = I.random_state(n, 100 + N)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    with qe.State(n, dtype) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.set(psi)
        st.mul(qa, qb, qc)
        got = st.get()
    want = oracle.mul(psi.astype(np.complex128), qa, qb, qc)
    assert np.array_equal(got, want.astype(got.dtype))


@pytest.mark.parametrize("N,n,kind", [(2, 7, "paper"), (3, 12, "mixed"), (4, 15, "offset")])
def test_mul_simulated_circuit_bit_exact(qe, N, n, kind):
    qa, qb, qc = layout(kind, N, n)
    psi = I.random_state(n, 200 + N)
    with qe.State(n, "c128") as st:
        st.set_policy(qe.POLICY_SIMULATE, 1)
        st.set(psi)
        st.reset_stats()
        st.mul(qa, qb, qc)
        got = st.get()
        gates = st.stats()["gates_applied"]
    assert np.array_equal(got, oracle.mul(psi, qa, qb, qc))
    assert gates == sum(N - i - j for i in range(N) for j in range(N - i))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("N,n,kind", [(1, 4, "paper"), (2, 6, "paper"), (3, 11, "mixed"), (4, 14, "offset"),
                                      (6, 18, "paper"), (7, 21, "paper"), (7, 23, "mixed")])
def test_div_emulated_bit_exact(qe, dtype, N, n, kind):
    # N <= 6 (complex128) / 6 (complex64): planes of 2^(2N) in shared memory;
    # N = 7: planes of 256 KB (128 KB) through the scratch buffer
    qa, qb, qc = layout(kind, N, n)
    psi = I.random_state(n, 300 + N)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    with qe.State(n, dtype) as st:
        st.set(psi)
        st.div(qa, qb, qc)
        got = st.get()
    want = oracle.div(psi.astype(np.complex128), qa, qb, qc)
    assert np.array_equal(got, want.astype(got.dtype))


def test_div_scratch_batches_bit_exact(qe):
    # n = 27, N = 8: 2048 planes of 1 MiB, two scratch batches of 1 GiB
    N, n = 8, 27
    qc, qb, qa = list(range(3, 11)), list(range(11, 19)), list(range(19, 27))
    with qe.State(n, "c128") as st:
        st.init_random(17)
        psi = st.get()
        st.div(qa, qb, qc)
        got = st.get()
    assert np.array_equal(got, oracle.div(psi, qa, qb, qc))


def test_div_on_zero_quotient_register_is_divmod(qe):
    # the paper's map (a, b, 0) -> (a mod b, b, a div b) on basis states
    N, n = 5, 15
    qc, qb, qa = list(range(5)), list(range(5, 10)), list(range(10, 15))
    with qe.State(n, "c128") as st:
        for a, b in ((29, 3), (31, 31), (7, 9), (0, 5), (17, 0), (30, 1)):
            st.init_basis((a << 10) | (b << 5))
            st.div(qa, qb, qc)
            got = st.get()
            idx = int(np.nonzero(got)[0][0])
            q, r = divmod(a, b) if b else (0, a)
            assert idx == (r << 10) | (b << 5) | q and got[idx] == 1


def test_mul_then_inverse_power_is_identity(qe):
    # c + 2^N a b = c (mod 2^N): 2^N multiplications restore the state
    N, n = 3, 11
    qa, qb, qc = [8, 9, 10], [5, 6, 7], [1, 2, 3]
    psi = I.random_state(n, 9)
    with qe.State(n, "c128") as st:
        st.set(psi)
        for _ in range(1 << N):
            st.mul(qa, qb, qc)
        assert np.array_equal(st.get(), psi)


def test_arith_rejects_bad_registers(qe):
    n = 9
    psi = I.random_state(n, 1)
    with qe.State(n, "c128") as st:
        st.set(psi)
        for bad in [lambda: st.mul([0, 1], [1, 2], [3, 4]), lambda: st.mul([0], [1], [9]),
                    lambda: st.div([0, 0], [1, 2], [3, 4]), lambda: st.mul([0, 1, 2, 3], [4, 5, 6, 7], [8, 0, 1, 2])]:
            with pytest.raises(qe.QEError) as ei:
                bad()
            assert ei.value.status == -1
        st.set_policy(qe.POLICY_SIMULATE, 1)
        with pytest.raises(qe.QEError) as ei:
            st.div([0, 1, 2], [3, 4, 5], [6, 7, 8])
        assert ei.value.status == -6
        assert np.array_equal(st.get(), psi)
