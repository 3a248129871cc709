"""Measurement (Sec. II) through the C ABI: inverse-CDF sampling with given
uniforms and the collapse onto an outcome, against the oracle.  Sampling
decides integers from FP64 sums taken in different orders on the two sides,
so every GPU outcome is checked to be a valid inverse-CDF outcome (its
cumulative interval contains the target up to rounding) and nearly all are
checked to equal the oracle's."""
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


def check_valid(out, u, P, rel=1e-12):
    """Every outcome r satisfies cdf(r-1) <= u total < cdf(r) up to rounding,
    with P(r) > 0."""
    cdf = np.cumsum(P)
    total = cdf[-1]
    t = np.asarray(u) * total
    r = np.asarray(out, dtype=np.int64)
    lo = np.where(r > 0, cdf[np.maximum(r - 1, 0)], 0.0)
    assert np.all(P[r] > 0)
    assert np.all(lo <= t + rel * total) and np.all(cdf[r] > t - rel * total)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n", [6, 14, 20])
def test_sample_all_qubits_vs_oracle(qe, dtype, n):
    # n <= 16: one distribution of 2^n bins; n = 20: blocks of 2^12 amplitudes
    psi = I.random_state(n, 40 + n)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    u = np.random.default_rng(n).random(3000)
    u[:3] = [0.0, np.nextafter(1.0, 0.0), 0.5]
    with qe.State(n, dtype) as st:
        st.set(psi)
        got = st.sample(u)
        assert np.array_equal(st.get(), psi)          # sampling leaves the state alone
    ref = oracle.sample(psi.astype(np.complex128), list(range(n)), u)
    P = np.abs(psi.astype(np.complex128)) ** 2
    check_valid(got, u, P)
    assert np.mean(got == ref) > 0.999


@pytest.mark.parametrize("qubits", [[0], [5, 1, 9], [11, 0, 3, 7, 2, 9, 4, 13, 6, 1]])
def test_sample_marginal_vs_oracle(qe, qubits):
    n = 14
    psi = I.random_state(n, 7)
    u = np.random.default_rng(3).random(2000)
    with qe.State(n, "c128") as st:
        st.set(psi)
        got = st.sample(u, qubits)
    ref = oracle.sample(psi, qubits, u)
    check_valid(got, u, oracle.probs(psi, qubits))
    assert np.mean(got == ref) > 0.999


def test_sample_never_picks_zero_probability_states(qe):
    # GHZ: only |0..0> and |1..1> carry probability 1/2 each
    n = 18
    u = np.concatenate([np.linspace(0, 1, 101)[:-1], [np.nextafter(0.5, 0), 0.5, np.nextafter(1.0, 0)]])
    with qe.State(n, "c128") as st:
        for g in I.ghz_circuit(n):
            st.apply(g)
        got = st.sample(u)
    want = np.where(u < 0.5, 0, (1 << n) - 1)
    assert np.array_equal(got.astype(np.int64), want)


def test_sample_full_size_blocks(qe):
    # n = 26: 2^14 blocks, targets spread over the whole distribution
    n = 26
    u = np.random.default_rng(11).random(4000)
    with qe.State(n, "c128") as st:
        st.init_random(5)
        psi = st.get()
        got = st.sample(u)
    check_valid(got, u, np.abs(psi) ** 2)


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-12), ("c64", 2e-6)])
@pytest.mark.parametrize("qubits,outcome", [([3], 1), ([0, 7], 2), ([12, 1, 5, 9], 11), (list(range(13)), 4321)])
def test_collapse_vs_oracle(qe, dtype, tol, qubits, outcome):
    n = 13
    psi = I.random_state(n, 9)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    with qe.State(n, dtype) as st:
        st.set(psi)
        p = st.collapse(qubits, outcome)
        got = st.get().astype(np.complex128)
    ref, p_ref = oracle.collapse(psi.astype(np.complex128), qubits, outcome)
    assert abs(p - p_ref) < tol * max(p_ref, 1e-3)
    assert np.max(np.abs(got - ref)) < tol * max(1.0, float(np.max(np.abs(ref))))


def test_collapse_ghz_and_errors(qe):
    n = 12
    with qe.State(n, "c128") as st:
        for g in I.ghz_circuit(n):
            st.apply(g)
        before = st.get()
        for bad in [lambda: st.collapse([0, 1], 2),          # probability zero for GHZ
                    lambda: st.collapse([0], 2),             # outcome beyond one bit
                    lambda: st.collapse([0, 0], 0), lambda: st.collapse([12], 0),
                    lambda: st.sample([1.0]), lambda: st.sample([-0.1]), lambda: st.sample([0.5], [0, 0])]:
            with pytest.raises(qe.QEError) as ei:
                bad()
            assert ei.value.status == -1
        assert np.array_equal(st.get(), before)
        p = st.collapse([5], 1)
        got = st.get()
    want = np.zeros(1 << n, complex)
    want[-1] = 1
    assert abs(p - 0.5) < 1e-15 and np.max(np.abs(got - want)) < 1e-15
