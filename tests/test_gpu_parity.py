"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every input comes from ``inputs`` (seeded); the oracle computes the expected
values; the GPU result is compared element by element.

Tolerances (complex128, FP64 mode and double-float mode alike):
  max |gpu - oracle| <= 1e-12 and fidelity >= 1 - 1e-10 (the FP64 bar);
  the FP64 mode is also checked against extended-precision references at the
  level of FP64 rounding (see the accuracy tests at the end);
  permutations (CNOT/MCX/SWAP, add-constant, bit reversal) are bit-exact.
complex64: FP32 arithmetic, max-abs <= 2e-6 per operation sequence used here
(about 2^-24 per gate times the few dozen gates of each test), stated per test.
"""
import numpy as np
import pytest

import oracle
from paper_1604_06460_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-12
FID = 1 - 1e-10


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


def close(got, ref, tol=TOL, fid=FID):
    err = float(np.max(np.abs(got - ref)))
    f = oracle.fidelity(ref, got)
    assert err <= tol, f"max-abs {err:.3e} > {tol}"
    assert f >= fid, f"fidelity {f!r}"
    return err


# complex128 arithmetic: "fp64" (default: FP64 mode, dense blocks on the
# tensor cores), "df64" (the double-float mode), "f64" (FP64 mode without
# tensor cores: native FP64 kernels only)
ARITHS = ["fp64", "df64", "f64"]


def make(qe, n, dtype="c128", psi=None, max_k=1, native=False, tile=False, arith=None):
    import os
    if native:
        arith = "f64"
    if arith and arith != "fp64":
        os.environ["QE_C128_ARITH"] = arith
    if tile:
        os.environ["QE_DENSE_TILE"] = "1"
    try:
        st = qe.State(n, dtype)
    finally:
        os.environ.pop("QE_C128_ARITH", None)
        os.environ.pop("QE_DENSE_TILE", None)
    st.set_policy(qe.POLICY_AUTO, max_k)
    if psi is not None:
        st.set(psi)
    return st


def rand_unitary(d, rng):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


# ------------------------------------------------------------------ init
def test_init_basis_exact(qe):
    with make(qe, 9) as st:
        st.init_basis(300)
        got = st.get()
    want = np.zeros(512, complex)
    want[300] = 1
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n", [5, 12, 17])
def test_init_random_matches_oracle_generator(qe, n):
    with make(qe, n) as st:
        st.init_random(1234 + n)
        got = st.get()
    ref = oracle.gaussian_state(n, 1234 + n)
    # same Philox words; libm vs CUDA log/sin/cos differ in the last ulp
    close(got, ref, tol=1e-14)


def test_init_random_c64(qe):
    with make(qe, 12, "c64") as st:
        st.init_random(7)
        got = st.get().astype(np.complex128)
    ref = oracle.gaussian_state(12, 7)
    assert np.max(np.abs(got - ref)) < 1e-7


# ------------------------------------------------------- single gates
@pytest.mark.parametrize("arith,tile", [("fp64", False), ("f64", False), ("df64", False), ("f64", True),
                                        ("df64", True)])
@pytest.mark.parametrize("q", [0, 1, 3, 4, 5, 9, 10, 13])
def test_1q_dense_every_position(qe, q, arith, tile):
    n = 14
    psi = I.random_state(n, q)
    U = I.haar_u2(np.random.default_rng(q))
    with make(qe, n, psi=psi, arith=arith, tile=tile) as st:
        st.apply_gate([q], U)
        got = st.get()
    close(got, oracle.apply_gate(psi, [q], U))


@pytest.mark.parametrize("arith", ARITHS)
@pytest.mark.parametrize("tile", [False, True])
@pytest.mark.parametrize("qubits", [[0, 1], [1, 0], [4, 11], [12, 2, 7], [0, 5, 10, 13],
                                    [3, 4, 5, 6, 7], [13, 0, 9, 1, 6], [10, 11, 12, 13]])
def test_kq_dense(qe, qubits, tile, arith):
    n = 14
    rng = np.random.default_rng(len(qubits) * 100 + qubits[0])
    U = rand_unitary(1 << len(qubits), rng)
    psi = I.random_state(n, 3)
    with make(qe, n, psi=psi, max_k=5, tile=tile, arith=arith) as st:
        st.apply_gate(qubits, U)
        got = st.get()
    close(got, oracle.apply_gate(psi, qubits, U))


def test_kq_dense_small_state(qe):
    # n below the tile size: one tile covers the whole state
    n = 6
    U = rand_unitary(8, np.random.default_rng(2))
    psi = I.random_state(n, 4)
    with make(qe, n, psi=psi, max_k=5) as st:
        st.apply_gate([5, 0, 3], U)
        got = st.get()
    close(got, oracle.apply_gate(psi, [5, 0, 3], U))


@pytest.mark.parametrize("arith", ARITHS)
def test_structured_gates(qe, arith):
    n = 13
    psi = I.random_state(n, 8)
    ref = psi.copy()
    gates = [I.cnot(3, 0), I.cnot(0, 12), I.cz(2, 9), I.cr(5, 1, 0.3), I.cr(0, 11, -1.7),
             I.single(7, I.mat_rz(0.4)), I.single(0, I.mat_t()), I.single(4, I.mat_s()),
             I.single(6, I.mat_x()), I.single(8, I.mat_y()), I.single(10, I.mat_z()),
             I.Gate((4, 9), np.eye(4)[[0, 2, 1, 3]].astype(complex), (), "swap")]
    with make(qe, n, psi=psi, arith=arith) as st:
        for g in gates:
            st.apply(g)
            ref = oracle.apply_gate(ref, g.qubits, g.matrix)
        got = st.get()
    close(got, ref)


def test_permutation_gates_bit_exact(qe):
    n = 12
    psi = I.random_state(n, 9)
    ref = psi.copy()
    gates = [I.cnot(0, 1), I.cnot(11, 3), I.single(5, I.mat_x()), I.mcx([0, 2, 7], 11),
             I.mcx([1, 3, 4, 5, 6, 8, 9, 10], 0)]
    with make(qe, n, psi=psi) as st:
        for g in gates:
            st.apply(g)
            if g.controls:
                ref = oracle.apply_mcx(ref, list(g.controls), g.qubits[0])
            else:
                ref = oracle.apply_gate(ref, g.qubits, g.matrix)
        got = st.get()
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("controls,targets", [([3], [0]), ([0, 9], [4]), ([2], [5, 11]), ([1, 4, 7], [0, 12])])
def test_controlled_dense(qe, controls, targets, arith):
    n = 13
    U = rand_unitary(1 << len(targets), np.random.default_rng(len(controls)))
    psi = I.random_state(n, 10)
    with make(qe, n, psi=psi, arith=arith) as st:
        st.apply_controlled(controls, targets, U)
        got = st.get()
    close(got, oracle.apply_controlled(psi, controls, targets, U))


# ------------------------------------------------------------ circuits
# The fusion planner keeps controlled gates as passes of their own and lets
# blocks on other qubits move past them: a fused random circuit with
# controlled-U and multi-controlled-X gates interleaved must match the
# oracle applied gate by gate.
@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_fused_circuit_with_controlled_gates(qe, dtype):
    n = 14
    rng = np.random.default_rng(31)
    gates = []
    for _ in range(6):
        for q in range(n):
            gates.append(I.single(q, I.haar_u2(rng)))
        perm = rng.permutation(n)
        for j in range(0, n - 1, 2):
            gates.append(I.cnot(int(perm[j]), int(perm[j + 1])))
        qs = [int(v) for v in rng.permutation(n)[:4]]
        gates.append(I.Gate((qs[0],), rand_unitary(2, rng), (qs[1], qs[2]), "cu"))
        gates.append(I.mcx([qs[3], qs[0]], qs[1]))
    psi = I.random_state(n, 17)
    ref = psi.copy()
    for g in gates:
        if g.controls:
            ref = oracle.apply_controlled(ref, list(g.controls), list(g.qubits), g.matrix)
        else:
            ref = oracle.apply_gate(ref, list(g.qubits), g.matrix)
    with make(qe, n, dtype, psi=psi, max_k=5) as st:
        st.reset_stats()
        for g in gates:
            st.apply(g)
        got = st.get().astype(np.complex128)
        passes = st.stats()["passes"]
    assert passes < len(gates) / 4
    if dtype == "c128":
        close(got, ref)
    else:
        assert np.max(np.abs(got - ref)) < 2e-5
        assert oracle.fidelity(ref, got) > 1 - 1e-8


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("max_k,tile", [(1, False), (2, False), (3, False), (4, False), (5, False),
                                        (2, True)])
def test_random_circuit_fused_vs_oracle(qe, max_k, tile, arith):
    n = 14
    gates = I.random_circuit(n, 10, seed=11)
    ref = oracle.zero_state(n)
    for g in gates:
        ref = oracle.apply_gate(ref, g.qubits, g.matrix)
    with make(qe, n, max_k=max_k, tile=tile, arith=arith) as st:
        for g in gates:
            st.apply(g)
        got = st.get()
        stats = st.stats()
    close(got, ref)
    assert stats["gates_applied"] == len(gates)


def test_ghz_closed_form(qe):
    n = 16
    with make(qe, n) as st:
        for g in I.ghz_circuit(n):
            st.apply(g)
        got = st.get()
    want = np.zeros(1 << n, complex)
    want[0] = want[-1] = 1 / np.sqrt(2)
    assert np.max(np.abs(got - want)) < 1e-15


def test_random_circuit_c64(qe):
    n = 14
    gates = I.random_circuit(n, 6, seed=5)
    ref = oracle.zero_state(n)
    for g in gates:
        ref = oracle.apply_gate(ref, g.qubits, g.matrix)
    for max_k in (1, 4):
        with make(qe, n, "c64", max_k=max_k) as st:
            for g in gates:
                st.apply(g)
            got = st.get().astype(np.complex128)
        # FP32: ~2^-24 per operation on amplitudes of size ~2^-7
        assert np.max(np.abs(got - ref)) < 2e-6
        assert oracle.fidelity(ref, got) > 1 - 1e-9


# ----------------------------------------------------------------- QFT
@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("n,lo,m", [(8, 0, 8), (10, 2, 5), (12, 0, 12), (14, 0, 14), (15, 1, 13), (13, 6, 7),
                                    # tensor-core digit passes (digits of 4, 3 and 5 qubits), the
                                    # digit reversal in shared-memory tiles and in chunk swaps
                                    (14, 2, 12), (18, 6, 12), (13, 0, 9), (16, 0, 5), (14, 3, 8),
                                    (12, 1, 10)])
@pytest.mark.parametrize("inverse", [False, True])
def test_qft_emulated_vs_dft(qe, n, lo, m, inverse, arith):
    psi = I.random_state(n, n + lo + m)
    with make(qe, n, psi=psi, arith=arith) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.apply_qft(lo, m, inverse)
        got = st.get()
    close(got, oracle.qft_dft(psi, lo, m, inverse))


@pytest.mark.parametrize("n,lo,m", [(9, 0, 9), (12, 3, 6)])
def test_qft_simulated_vs_dft(qe, n, lo, m):
    psi = I.random_state(n, 40 + m)
    with make(qe, n, psi=psi) as st:
        st.set_policy(qe.POLICY_SIMULATE, 1)
        st.apply_qft(lo, m)
        got = st.get()
    close(got, oracle.qft_dft(psi, lo, m))


def test_qft_basis_state_closed_form(qe):
    n, x = 13, 1234
    with make(qe, n) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.init_basis(x)
        st.apply_qft(0, n)
        got = st.get()
    l = np.arange(1 << n)
    want = np.exp(2j * np.pi * ((x * l) % (1 << n)) / (1 << n)) / np.sqrt(1 << n)
    assert np.max(np.abs(got - want)) < 1e-15


@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_qft_many_passes_sampled(qe, arith):
    # 24 register qubits: three FFT passes plus the bit reversal
    n, lo, m = 25, 1, 24
    with make(qe, n, arith=arith) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.init_random(3)
        psi = st.get()
        st.apply_qft(lo, m)
        rng = np.random.default_rng(0)
        idx = [0, 1, (1 << n) - 1] + list(rng.integers(0, 1 << n, size=3))
        for i in idx:
            want = oracle.qft_amplitude(psi, lo, m, int(i))
            got = st.get(int(i), 1)[0]
            assert abs(got - want) < 1e-12
        st.apply_qft(lo, m, inverse=True)
        back = st.get()
    close(back, psi)


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("n,lo,m", [(15, 0, 15), (17, 1, 15), (20, 0, 20), (21, 4, 16)])
def test_qft_tensor_core_digits_sampled(qe, n, lo, m, arith):
    # registers too large for the direct DFT: sampled outputs from the
    # oracle's one-amplitude definition, then the inverse restores the input
    with make(qe, n, arith=arith) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.init_random(3 + m)
        psi = st.get()
        st.profile(True)
        st.apply_qft(lo, m)
        prof = st.profile_read()
        st.profile(False)
        rng = np.random.default_rng(m)
        for i in [0, 1, (1 << n) - 1] + [int(v) for v in rng.integers(0, 1 << n, size=5)]:
            want = oracle.qft_amplitude(psi, lo, m, i)
            assert abs(st.get(i, 1)[0] - want) < 1e-12
        st.apply_qft(lo, m, inverse=True)
        back = st.get()
    if arith == "fp64":
        assert "digitrev" in prof and "fft_pass" not in prof
    close(back, psi)


def test_qft_c64(qe):
    n, lo, m = 14, 0, 14
    psi = I.random_state(n, 77)
    with make(qe, n, "c64", psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.apply_qft(lo, m)
        got = st.get().astype(np.complex128)
    ref = oracle.qft_dft(psi, lo, m)
    assert np.max(np.abs(got - ref)) < 1e-6


# --------------------------------------------------------- add constant
@pytest.mark.parametrize("n,qubits,c", [
    (12, list(range(0, 8)), 77),          # chunks of 2^8-amplitude slices in shared memory
    (12, list(range(2, 12)), 1000),       # slice of 2^12 (bulk copies)
    (18, list(range(0, 16)), 40503),      # cluster of 8 CTAs
    (17, list(range(1, 16)), 12345),      # cluster, lo = 1
    (14, list(range(6, 14)), 201),        # walk, coalesced columns
    (14, list(range(5, 14)), 256),        # walk with gcd > 1
    (13, [1, 5, 3, 12], 11),              # non-contiguous register
    (10, list(range(10)), 1023),          # whole state
])
def test_add_const_bit_exact(qe, n, qubits, c):
    psi = I.random_state(n, c)
    with make(qe, n, psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.add_const(qubits, c)
        got = st.get()
    assert np.array_equal(got, oracle.add_const(psi, qubits, c))


@pytest.mark.parametrize("n,qubits,c", [
    (12, list(range(0, 8)), 77),          # odd shift: 8-byte runs, shared-memory slice
    (14, list(range(0, 12)), 78),         # even shift: bulk copies, one CTA
    (18, list(range(0, 17)), 4097),       # odd shift, cluster through shared memory
    (18, list(range(0, 17)), 4098),       # even shift, bulk copies, cluster of eight
    (15, list(range(1, 13)), 5),          # lo = 1: the shift 10 is even
])
def test_add_const_c64_paths_bit_exact(qe, n, qubits, c):
    psi = I.random_state(n, c).astype(np.complex64)
    with make(qe, n, "c64", psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.add_const(qubits, c)
        got = st.get()
    want = oracle.add_const(psi.astype(np.complex128), qubits, c).astype(np.complex64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("n,qubits,c", [
    (14, [0], 1),                         # 2-amplitude slices, whole chunks of them
    (14, [0, 1, 2, 3], 5),                # 16-amplitude slices
    (14, [2, 3, 4], 5),                   # lo = 2: 32-amplitude slices, shift 20
    (15, list(range(0, 10)), 1001),       # 2^10 slices (below the bulk threshold)
    (11, [0, 1, 2, 3], 9),                # one chunk is the whole state (complex128)
    (9, [0, 1], 3),                       # the state is smaller than a chunk
])
def test_add_const_small_slices_in_chunks(qe, dtype, n, qubits, c):
    # registers at the bottom whose slices are far below a CTA's shared
    # memory: many whole slices per chunk, bit-exact, on the chunked kernel
    psi = I.random_state(n, 31 + c)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    with make(qe, n, dtype, psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.profile(True)
        st.add_const(qubits, c)
        prof = st.profile_read()
        got = st.get()
    assert set(prof) & {"add_slice", "add_bulk"} == {"add_slice"}, prof
    want = oracle.add_const(psi.astype(np.complex128), qubits, c)
    if dtype == "c64":
        want = want.astype(np.complex64)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("n,qubits", [(14, list(range(0, 12))), (18, list(range(0, 16)))])
def test_add_const_bulk_copy_wait_times_out(qe, monkeypatch, n, qubits):
    # one CTA (2^12-amplitude slices) and clusters of eight (2^16): block 0
    # announces its part but copies none; QE_ERR_TIMEOUT, then a fresh state
    # on the same context adds bit-exactly
    from paper_1604_06460_gb300.qe import QEError
    psi = I.random_state(n, 97)
    c = 1234
    with make(qe, n, psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        monkeypatch.setenv("QE_TEST_STALL_ADD", "1")
        with pytest.raises(QEError) as err:
            st.add_const(qubits, c)
            st.flush()
        assert err.value.status == -4 and "QE_ERR_TIMEOUT" in str(err.value)
        monkeypatch.delenv("QE_TEST_STALL_ADD")
        st.set(psi)
        st.profile(True)
        st.add_const(qubits, c)
        prof = st.profile_read()
        got = st.get()
    assert "add_bulk" in prof or "add_bulk_cluster" in prof, prof
    assert np.array_equal(got, oracle.add_const(psi, qubits, c))


def test_add_const_simulated_bit_exact(qe):
    n, qubits, c = 12, list(range(2, 10)), 173
    psi = I.random_state(n, 5)
    with make(qe, n, psi=psi) as st:
        st.set_policy(qe.POLICY_SIMULATE, 1)
        st.add_const(qubits, c)
        got = st.get()
    assert np.array_equal(got, oracle.add_const(psi, qubits, c))


def test_add_const_c64_and_roundtrip(qe):
    n, qubits, c = 16, list(range(0, 16)), 999
    psi = I.random_state(n, 6).astype(np.complex64)
    with make(qe, n, "c64", psi=psi) as st:
        st.add_const(qubits, c)
        got = st.get()
        st.add_const(qubits, (1 << 16) - c)
        back = st.get()
    want = oracle.add_const(psi.astype(np.complex128), qubits, c).astype(np.complex64)
    assert np.array_equal(got, want)
    assert np.array_equal(back, psi)


# ----------------------------------------------- expectation and probs
@pytest.mark.parametrize("dtype,arith", [("c128", "fp64"), ("c128", "df64"), ("c64", None)])
def test_tfim_expectation(qe, dtype, arith):
    n = 12
    psi = I.random_state(n, 21)
    xm, zm, cf = I.tfim_terms(n)
    with make(qe, n, dtype, psi=psi, arith=arith) as st:
        e = st.expectation(xm, zm, cf)
    ref = oracle.expectation(psi, xm, zm, cf)
    assert abs(e - ref) < (1e-12 if dtype == "c128" else 1e-5)


def _rounds_terms(n, seed, nweights=1):
    """Terms the register-round kernel takes: X/Y bits below qubit 12 inside
    one of the triples {0,1,2} .. {9,10,11} (every 3-bit pattern), one to
    three high X/Y bits, Z parts inside the triple, elsewhere in the tile and
    outside it; Z-only masks in several weight groups, some entirely outside
    the tile."""
    rng = np.random.default_rng(seed)
    xm, zm, cf = [], [], []
    wx = [0.35, -1.25][:nweights]
    for r in range(4):
        for pat in range(1, 8):
            xm.append(pat << (3 * r))
            zm.append(int(rng.integers(0, 1 << n)) if pat % 2 else 0)
            cf.append(wx[(r + pat) % nweights])
    for q in range(12, n):
        xm.append(1 << q); zm.append(0); cf.append(wx[q % nweights])
    high = [q for q in range(12, n)]
    for _ in range(6 if high else 0):
        k = int(rng.integers(1, 4))
        qs = rng.choice(high, size=k, replace=False)
        xm.append(int(sum(1 << int(q) for q in qs)))
        zm.append(int(rng.integers(0, 1 << n)))
        cf.append(wx[0])
    for i in range(n - 1):
        xm.append(0); zm.append((1 << i) | (1 << (i + 1))); cf.append(1.0)
    for _ in range(10):
        xm.append(0); zm.append(int(rng.integers(1, 1 << n))); cf.append(-0.5)
    if n > 12:
        xm.append(0); zm.append(((1 << (n - 12)) - 1) << 12); cf.append(0.25)   # outside the 12-qubit tile only
    xm.append(0); zm.append(0b101); cf.append(2.0)                            # triple 0 only
    return np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64), np.array(cf)


@pytest.mark.parametrize("dtype,arith,tol", [("c128", "fp64", 1e-12), ("c128", "df64", 1e-12), ("c64", None, 2e-5)])
@pytest.mark.parametrize("n,nweights", [(12, 1), (15, 2), (20, 1)])
def test_expectation_register_rounds(qe, dtype, arith, tol, n, nweights):
    # the register-round kernel forced on (QE_EXPECT_TILE=2) and off (=1):
    # both against the oracle, and the forced run must have used it
    import os
    xm, zm, cf = _rounds_terms(n, 60 + n, nweights)
    psi = I.random_state(n, 70 + n)
    ref = oracle.expectation(psi, xm, zm, cf)
    got = {}
    for sw in ("2", "1"):
        os.environ["QE_EXPECT_TILE"] = sw
        try:
            with make(qe, n, dtype, psi=psi, arith=arith) as st:
                st.profile(True)
                got[sw] = st.expectation(xm, zm, cf)
                prof = st.profile_read()
        finally:
            os.environ.pop("QE_EXPECT_TILE", None)
        tag = "expect_fx" if dtype == "c128" else "expect_rounds"
        assert (tag in prof) == (sw == "2"), prof
    bound = tol if dtype == "c128" else tol * float(np.sum(np.abs(cf)))
    for sw, e in got.items():
        assert abs(e - ref) < bound, (sw, e, ref)


@pytest.mark.parametrize("dtype,arith", [("c128", "fp64"), ("c128", "df64"), ("c64", None)])
def test_expectation_rounds_chosen_for_tfim(qe, dtype, arith):
    # TFIM at n = 24: 3 launches of the register-round kernel (qubits
    # [0, 12), then two layouts of six high qubits) instead of 4 tile ones,
    # in fixed point for complex128 in both modes; closed forms on |0..0>
    # and |+..+>
    n = 24
    xm, zm, cf = I.tfim_terms(n)
    with make(qe, n, dtype, arith=arith) as st:
        st.profile(True)
        e0 = st.expectation(xm, zm, cf)
        prof = st.profile_read()
        tag = "expect_fx" if dtype == "c128" else "expect_rounds"
        assert prof[tag][0] == 3 and "expect_tile" not in prof, prof
        for q in range(n):
            st.apply_gate([q], I.mat_h())
        e1 = st.expectation(xm, zm, cf)
    tol = 1e-12 if dtype == "c128" else 1e-5 * n
    assert abs(e0 - (n - 1)) < tol
    assert abs(e1 - 0.7 * n) < 10 * tol


def test_expectation_rounds_not_chosen_when_terms_do_not_fit(qe):
    # an X/Y mask across two triples (qubits 2 and 3) goes to the tile kernel
    n = 14
    xm, zm, cf = I.tfim_terms(n)
    xm = np.append(xm, np.uint64(0b1100)); zm = np.append(zm, np.uint64(0)); cf = np.append(cf, 0.3)
    psi = I.random_state(n, 3)
    with make(qe, n, psi=psi) as st:
        st.profile(True)
        e = st.expectation(xm, zm, cf)
        prof = st.profile_read()
    assert "expect_rounds" not in prof and "expect_fx" not in prof and "expect_tile" in prof
    assert abs(e - oracle.expectation(psi, xm, zm, cf)) < 1e-12


def _scaled_blocks(psi, seed, lo=-60):
    # every block of 256 amplitudes scaled by 2^k, k uniform in [lo, 0]; one
    # block in eight zero: tiles whose components span many binades
    rng = np.random.default_rng(seed)
    out = psi.copy().reshape(-1, 256)
    k = rng.integers(lo, 1, size=out.shape[0])
    out *= (2.0 ** k.astype(np.float64))[:, None]
    out[rng.random(out.shape[0]) < 0.125] = 0
    return out.reshape(-1)


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("scale", [0, 400, -400])
def test_expectation_fixed_point_dynamic_range(qe, arith, scale):
    # complex128 expectation in fixed point (the tile's largest component
    # keeps its 53 bits, the others share its grid): states whose tiles span
    # 60 binades and zero tiles, scaled by 2^scale (results by 2^(2 scale));
    # against the oracle within 1e-13 of sum |c_t| ||psi||^2
    n = 16
    xm, zm, cf = _rounds_terms(n, 91, 2)
    psi = _scaled_blocks(I.random_state(n, 92), 93) * 2.0 ** scale
    ref = oracle.expectation(psi, xm, zm, cf)
    with make(qe, n, "c128", psi=psi, arith=arith) as st:
        st.profile(True)
        e = st.expectation(xm, zm, cf)
        prof = st.profile_read()
    assert "expect_fx" in prof and "expect_tile" not in prof, prof
    bound = 1e-13 * float(np.sum(np.abs(cf))) * float(np.vdot(psi, psi).real)
    assert abs(e - ref) <= bound, (e, ref, bound)


def test_expectation_fixed_point_unbiased(qe):
    # the limbs are rounded to the nearest grid point: an energy dominated by
    # |a|^2 weights (sum_i Z_i) plus X terms stays within 1e-15 of the oracle
    # at n = 22 (truncated limbs shrink every |a|^2 alike: ~2e-15 here)
    n = 22
    xm = [1 << q for q in range(n)] + [0] * n
    zm = [0] * n + [1 << q for q in range(n)]
    cf = [0.7] * n + [1.0] * n
    xm, zm, cf = np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64), np.array(cf)
    psi = I.random_state(n, 95)
    ref = oracle.expectation(psi, xm, zm, cf)
    with make(qe, n, "c128", psi=psi) as st:
        e = st.expectation(xm, zm, cf)
    assert abs(e - ref) < 1e-15, (e, ref, e - ref)


def test_expectation_fixed_point_copy_wait_times_out(qe, monkeypatch):
    # block 0's first tile is announced but never copied: its bounded wait
    # runs out, the launch reports QE_ERR_TIMEOUT, and the state still works
    from paper_1604_06460_gb300.qe import QEError
    n = 16
    xm, zm, cf = I.tfim_terms(n)
    psi = I.random_state(n, 96)
    ref = oracle.expectation(psi, xm, zm, cf)
    with make(qe, n, "c128", psi=psi) as st:
        monkeypatch.setenv("QE_TEST_STALL_EXPECT", "1")
        with pytest.raises(QEError) as err:
            st.expectation(xm, zm, cf)
        assert err.value.status == -4 and "QE_ERR_TIMEOUT" in str(err.value)
        monkeypatch.delenv("QE_TEST_STALL_EXPECT")
        assert abs(st.expectation(xm, zm, cf) - ref) < 1e-12


def test_expectation_fixed_point_underflow(qe):
    # components below 2^-959: their products underflow FP64 and the fixed
    # point takes such tiles as zero; tiles of ordinary size beside them are
    # exact
    n = 14
    xm, zm, cf = I.tfim_terms(n)
    psi = I.random_state(n, 94)
    tiny = psi.copy()
    tiny[: 1 << 12] *= 2.0 ** -1000
    with make(qe, n, "c128", psi=tiny) as st:
        e = st.expectation(xm, zm, cf)
    ref = oracle.expectation(tiny, xm, zm, cf)
    assert abs(e - ref) < 1e-13, (e, ref)
    with make(qe, n, "c128", psi=psi * 2.0 ** -1000) as st:
        assert st.expectation(xm, zm, cf) == 0.0


def test_tfim_closed_forms(qe):
    n = 11
    xm, zm, cf = I.tfim_terms(n)
    with make(qe, n) as st:
        assert abs(st.expectation(xm, zm, cf) - (n - 1)) < 1e-13
        for q in range(n):
            st.apply_gate([q], I.mat_h())
        assert abs(st.expectation(xm, zm, cf) - 0.7 * n) < 1e-12


@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_general_pauli_terms(qe, arith):
    n = 10
    rng = np.random.default_rng(5)
    xm = rng.integers(0, 1 << n, size=13).astype(np.uint64)
    zm = rng.integers(0, 1 << n, size=13).astype(np.uint64)
    cf = rng.standard_normal(13)
    psi = I.random_state(n, 31)
    with make(qe, n, psi=psi, arith=arith) as st:
        e = st.expectation(xm, zm, cf)
    assert abs(e - oracle.expectation(psi, xm, zm, cf)) < 1e-12


@pytest.mark.parametrize("dtype,tol,arith", [("c128", 1e-12, "fp64"), ("c128", 1e-12, "df64"), ("c64", 1e-5, None)])
def test_expectation_parities_outside_the_tile(qe, dtype, tol, arith):
    # n = 16 > the 11/12-qubit tile: nearest-neighbour ZZ masks inside,
    # straddling and entirely outside the tile; Z strings on high qubits only;
    # X/Y terms whose Z parts lie inside, outside, or both
    n = 16
    xm, zm, cf = [], [], []
    for i in range(n - 1):
        xm.append(0); zm.append((1 << i) | (1 << (i + 1))); cf.append(1.0)
    for mask in (1 << 15, (1 << 13) | (1 << 15), (1 << 2) | (1 << 12) | (1 << 14), 0b111 << 11):
        xm.append(0); zm.append(mask); cf.append(-0.3)
    for q, z in ((0, 1 << 14), (3, (1 << 4) | (1 << 15)), (5, 1 << 5), (12, 1 << 1), (15, (1 << 3) | (1 << 13))):
        xm.append(1 << q); zm.append(z); cf.append(0.45)
    for q in range(n):
        xm.append(1 << q); zm.append(0); cf.append(0.7)
    xm, zm, cf = (np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64), np.array(cf))
    psi = I.random_state(n, 44)
    with make(qe, n, dtype, psi=psi, arith=arith) as st:
        e = st.expectation(xm, zm, cf)
    assert abs(e - oracle.expectation(psi, xm, zm, cf)) < tol


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("qubits", [[0], [3, 0], [11, 2, 6], [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11]])
def test_probs(qe, qubits, arith):
    n = 12
    psi = I.random_state(n, 17)
    with make(qe, n, psi=psi, arith=arith) as st:
        p = st.probs(qubits)
        nrm = st.norm2()
    ref = oracle.probs(psi, qubits)
    # FP64 sums, or double-float partials of about 44 significant bits
    assert np.max(np.abs(p - ref)) < 1e-13
    assert abs(nrm - 1) < 1e-13


@pytest.mark.parametrize("dtype,arith", [("c128", "fp64"), ("c128", "df64"), ("c64", None)])
@pytest.mark.parametrize("qubits", [[0], [0, 1, 2], [7, 0, 3], list(range(8)), [2, 9]])
def test_probs_low_qubits_contiguous_reads(qe, dtype, arith, qubits):
    # qubits all below 8 at n = 16: the kernel whose threads each own one bin
    # (contiguous reads); a register reaching qubit 9 keeps the bin-major one
    n = 16
    psi = I.random_state(n, 18)
    if dtype == "c64":
        psi = psi.astype(np.complex64)
    with make(qe, n, dtype, psi=psi, arith=arith) as st:
        st.profile(True)
        p = st.probs(qubits)
        prof = st.profile_read()
    assert ("probs_low" in prof) == (max(qubits) < 8), prof
    ref = oracle.probs(psi.astype(np.complex128), qubits)
    assert np.max(np.abs(p - ref)) < (1e-13 if dtype == "c128" else 1e-6)


def test_probs_ghz(qe):
    n = 9
    with make(qe, n) as st:
        for g in I.ghz_circuit(n):
            st.apply(g)
        p = st.probs([0, 8])
    assert np.allclose(p, [0.5, 0, 0, 0.5], atol=1e-15)


# --------------------------------------------------------- error paths
def test_invalid_arguments_leave_state_untouched(qe):
    n = 6
    psi = I.random_state(n, 1)
    with make(qe, n, psi=psi) as st:
        for bad in [lambda: st.apply_gate([0, 0], np.eye(4)), lambda: st.apply_gate([6], np.eye(2)),
                    lambda: st.apply_qft(3, 4), lambda: st.add_const([7], 1),
                    lambda: st.probs([0, 0]), lambda: st.apply_gate([1], np.full((2, 2), np.nan)),
                    lambda: st.apply_qft(-1, 2), lambda: st.init_basis(1 << n),
                    lambda: st.set(np.zeros(10), offset=60), lambda: st.get(offset=60, count=10),
                    lambda: st.apply_controlled([1], [1], I.mat_x()),
                    lambda: st.apply_controlled([0], [1, 2, 3], np.eye(8)),
                    lambda: st.expectation([1 << n], [0], [1.0]),
                    lambda: st.expectation([0], [1], [np.inf])]:
            with pytest.raises(qe.QEError) as ei:
                bad()
            assert ei.value.status == -1
        assert np.array_equal(st.get(), psi)


# ------------------------------------------- tensor cores (complex64, k = 4, 5)
@pytest.mark.parametrize("qubits", [[0, 1, 2, 3, 4], [10, 11, 12, 13, 14], [4, 0, 15, 7, 12],
                                    [2, 9, 5, 14], [15, 14, 13, 12]])
def test_tensor_core_blocks_c64(qe, qubits):
    # 3xTF32 products accumulated in FP32: about FP32 accuracy
    n = 16
    U = rand_unitary(1 << len(qubits), np.random.default_rng(sum(qubits)))
    psi = I.random_state(n, 12).astype(np.complex64)
    with make(qe, n, "c64", psi=psi, max_k=5) as st:
        st.reset_stats()
        st.apply_gate(qubits, U)
        got = st.get().astype(np.complex128)
        launches = st.stats()["launches"]
    ref = oracle.apply_gate(psi.astype(np.complex128), qubits, U)
    assert launches == 1
    assert np.max(np.abs(got - ref)) < 2e-6
    assert oracle.fidelity(ref, got) > 1 - 1e-10


def test_tensor_core_fused_circuit_c64(qe):
    n = 14
    gates = I.random_circuit(n, 8, seed=21)
    ref = oracle.zero_state(n)
    for g in gates:
        ref = oracle.apply_gate(ref, g.qubits, g.matrix)
    with make(qe, n, "c64", max_k=5) as st:
        for g in gates:
            st.apply(g)
        got = st.get().astype(np.complex128)
    assert np.max(np.abs(got - ref)) < 2e-5
    assert oracle.fidelity(ref, got) > 1 - 1e-8


# The complex64 kernel's bounded waits: the splitters withhold the first
# operand arrival, the MMA thread's wait runs out, every role leaves through
# the abort flag; QE_ERR_TIMEOUT, then the same context computes correctly.
def test_tensor_core_c64_wait_timeout_reports_and_recovers(qe, monkeypatch):
    from paper_1604_06460_gb300.qe import QEError
    n, qubits = 14, [1, 4, 6, 9, 13]
    U = rand_unitary(32, np.random.default_rng(78))
    psi = I.random_state(n, 22)
    with make(qe, n, "c64", psi=psi, max_k=5) as st:
        monkeypatch.setenv("QE_TEST_STALL_TC64", "1")
        with pytest.raises(QEError) as err:
            st.apply_gate(qubits, U)
            st.flush()
        assert err.value.status == -4 and "QE_ERR_TIMEOUT" in str(err.value)
        monkeypatch.delenv("QE_TEST_STALL_TC64")
        st.set(psi)
        st.apply_gate(qubits, U)
        got = st.get().astype(np.complex128)
    ref = oracle.apply_gate(psi, qubits, U)
    assert np.max(np.abs(got - ref)) < 2e-5
    assert oracle.fidelity(ref, got) > 1 - 1e-8


# ------------------------------------------ tensor cores (complex128, k = 1..5)
# Exact integer-digit products on the FP16 tensor pipe: inputs and matrix
# entries are rounded to 2^-56 (FP64 mode, seven digits) or 2^-48 (double-
# float mode, six digits) of their row scale, so the FP64 bar holds.
TC128 = {"fp64": "gate_tc_k5_c128", "df64": "gate_tc_k5_c128_df"}


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("qubits", [[0, 1, 2, 3, 4], [10, 11, 12, 13, 14], [4, 0, 15, 7, 12],
                                    [2, 9, 5, 14], [15, 14, 13, 12], [6, 3, 11, 1, 8],
                                    [2, 9, 13], [0, 1, 2]])
def test_tensor_core_blocks_c128(qe, qubits, arith):
    n = 16
    U = rand_unitary(1 << len(qubits), np.random.default_rng(100 + sum(qubits)))
    psi = I.random_state(n, 13)
    with make(qe, n, "c128", psi=psi, max_k=5, arith=arith) as st:
        st.reset_stats()
        st.profile(True)
        st.apply_gate(qubits, U)
        got = st.get()
        prof = st.profile_read()
        st.profile(False)
        launches = st.stats()["launches"]
    ref = oracle.apply_gate(psi, qubits, U)
    assert launches == 1
    assert prof.get(TC128[arith], (0,))[0] == 1
    close(got, ref)


# A bounded wait that runs out: the load warps withhold one stage arrival
# (a flag nothing else sets), the splitters give up after a short limit, every
# role leaves through the abort flag and tensor memory is freed; the host
# reports QE_ERR_TIMEOUT and the same context then runs the block correctly.
@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_tensor_core_c128_wait_timeout_reports_and_recovers(qe, monkeypatch, arith):
    from paper_1604_06460_gb300.qe import QEError
    n, qubits = 14, [0, 3, 6, 9, 12]
    U = rand_unitary(32, np.random.default_rng(77))
    psi = I.random_state(n, 21)
    with make(qe, n, "c128", psi=psi, max_k=5, arith=arith) as st:
        monkeypatch.setenv("QE_TEST_STALL_TC128", "1")
        with pytest.raises(QEError) as err:
            st.apply_gate(qubits, U)
            st.flush()
        assert err.value.status == -4 and "QE_ERR_TIMEOUT" in str(err.value)
        monkeypatch.delenv("QE_TEST_STALL_TC128")
        st.set(psi)
        st.apply_gate(qubits, U)
        got = st.get()
    close(got, oracle.apply_gate(psi, qubits, U))


@pytest.mark.parametrize("arith", ["fp64", "df64"])
@pytest.mark.parametrize("n,qubits", [(12, [0, 4, 7, 9, 11]), (12, [11, 10, 9, 8, 7]), (13, [12, 0, 6, 3, 9]),
                                      (13, [12, 11, 1])])
def test_tensor_core_c128_smallest_states(qe, n, qubits, arith):
    # n = 12: one tile holds the whole state (a single CTA); n = 13: two tiles;
    # the highest qubits as gate qubits
    U = rand_unitary(1 << len(qubits), np.random.default_rng(n * 31 + len(qubits)))
    psi = I.random_state(n, 5)
    with make(qe, n, "c128", psi=psi, max_k=5, arith=arith) as st:
        st.profile(True)
        st.apply_gate(qubits, U)
        got = st.get()
        prof = st.profile_read()
        st.profile(False)
    assert prof.get(TC128[arith], (0,))[0] == 1
    close(got, oracle.apply_gate(psi, qubits, U))


@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_tensor_core_c128_special_values(qe, arith):
    # a basis state (all but one amplitude zero), amplitudes that are powers of
    # two (the splitting's binade edges), +-1 entries, and rows below the flush
    # threshold next to ordinary ones
    n = 14
    qubits = [1, 3, 5, 7, 9]
    U = rand_unitary(32, np.random.default_rng(5))
    for case in range(3):
        if case == 0:
            psi = np.zeros(1 << n, dtype=np.complex128)
            psi[12345] = 1.0
        elif case == 1:
            rng = np.random.default_rng(8)
            psi = (np.exp2(-rng.integers(1, 30, 1 << n)) * rng.choice([-1, 1], 1 << n)
                   + 1j * np.exp2(-rng.integers(1, 30, 1 << n)) * rng.choice([-1, 1], 1 << n))
            psi[::97] = 1.0 - 1.0j
        else:
            psi = I.random_state(n, 21)
            psi[: 1 << 10] *= 1e-290         # groups far below the flush threshold
            psi[1 << 10: 1 << 11] *= 1e-200  # small but kept
        with make(qe, n, "c128", psi=psi, max_k=5, arith=arith) as st:
            st.apply_gate(qubits, U)
            got = st.get()
        ref = oracle.apply_gate(psi, qubits, U)
        scale = max(1.0, float(np.max(np.abs(psi))))
        assert np.max(np.abs(got - ref)) <= 1e-12 * scale, case
        if case == 2:
            # the kept small groups keep their relative accuracy
            blk = slice(1 << 10, 1 << 11)
            rel = np.max(np.abs(got[blk] - ref[blk])) / np.max(np.abs(ref[blk]))
            assert rel < 1e-12


@pytest.mark.parametrize("arith", ["fp64", "df64"])
def test_tensor_core_fused_circuit_c128(qe, arith):
    n = 14
    gates = I.random_circuit(n, 8, seed=22)
    ref = oracle.zero_state(n)
    for g in gates:
        ref = oracle.apply_gate(ref, g.qubits, g.matrix)
    with make(qe, n, "c128", max_k=5, arith=arith) as st:
        st.profile(True)
        for g in gates:
            st.apply(g)
        got = st.get()
        prof = st.profile_read()
        st.profile(False)
    assert prof.get(TC128[arith], (0,))[0] > 0
    close(got, ref)


@pytest.mark.parametrize("dtype,tol,arith", [("c128", 1e-12, "fp64"), ("c128", 1e-12, "df64"), ("c64", 1e-5, None)])
def test_many_pauli_terms_all_layouts(qe, dtype, tol, arith):
    # Z-only terms in several weight groups (more than fit one launch), X/Y
    # terms inside the low tile, with high qubits, and wider than one tile
    n = 15
    rng = np.random.default_rng(77)
    xm, zm, cf = [], [], []
    for t in range(90):                      # Z-only, 6 distinct weights
        xm.append(0)
        zm.append(int(rng.integers(0, 1 << n)))
        cf.append([1.0, -0.5, 0.25, 2.0, 0.7, -1.3][t % 6])
    for t in range(20):                      # low X/Y terms
        xm.append(int(rng.integers(1, 1 << 8)))
        zm.append(int(rng.integers(0, 1 << n)))
        cf.append(float(rng.standard_normal()))
    for q in range(n):                       # single high X
        xm.append(1 << q)
        zm.append(0)
        cf.append(0.7)
    for t in range(6):                       # wide X/Y strings
        xm.append(int(rng.integers(1 << 10, 1 << n)) | 0x7F00)
        zm.append(int(rng.integers(0, 1 << n)))
        cf.append(float(rng.standard_normal()))
    xm, zm, cf = (np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64), np.array(cf))
    psi = I.random_state(n, 5)
    with make(qe, n, dtype, psi=psi, arith=arith) as st:
        e = st.expectation(xm, zm, cf)
    assert abs(e - oracle.expectation(psi, xm, zm, cf)) < tol


# --------------------------------------------- FP64-mode accuracy (53 bits)
# The FP64 mode must be as accurate as FP64 arithmetic, not merely within the
# 1e-12 bar.  References here are the plain definitions evaluated in extended
# precision (numpy longdouble: 64-bit significands on x86, 113 on AArch64), so
# FP64 rounding of the reference itself does not mask the kernel's error.
def _ld_apply(psi, qubits, U):
    """Dense k-qubit gate on a state, the sum over the group evaluated in
    long double (matrix bit j <-> qubits[j], as the oracle)."""
    n = int(np.log2(psi.size))
    k = len(qubits)
    x = np.arange(psi.size)
    groups = x[(x & sum(1 << q for q in qubits)) == 0]
    dep = np.array([sum(((c >> j) & 1) << qubits[j] for j in range(k)) for c in range(1 << k)])
    idx = groups[:, None] + dep[None, :]                 # (groups, 2^k)
    A = psi[idx].astype(np.clongdouble)
    Ul = np.asarray(U, dtype=np.clongdouble)
    out = np.zeros_like(A)
    for c in range(1 << k):                              # out[g, r] = sum_c U[r, c] A[g, c]
        out += A[:, c:c + 1] * Ul[None, :, c]
    res = np.empty(psi.size, dtype=np.clongdouble)
    res[idx] = out
    return res, idx


def _rel_group_error(got, ref_ld, idx):
    err = np.abs(got.astype(np.clongdouble) - ref_ld)[idx]
    scale = np.sqrt(np.sum(np.abs(ref_ld[idx]) ** 2, axis=1))
    return float(np.max(np.max(err, axis=1) / scale))


@pytest.mark.parametrize("qubits", [[1, 4, 7, 10, 13], [0, 1, 2, 3, 4], [15, 3, 8, 0], [6, 12, 2], [2, 11], [9]])
def test_fp64_mode_blocks_at_fp64_rounding(qe, qubits):
    # 3-5-qubit blocks: inputs rounded to 2^-56 of the group scale, exact
    # digit products, one rounding of each output; 1-2-qubit blocks: native
    # FP64.  Either way the error relative to the group's norm is a few units
    # of 2^-53 at most (FP64 dot products of the same terms carry the same
    # order), where the 48-bit double-float splitting leaves ~1e-14
    n = 16
    rng = np.random.default_rng(900 + len(qubits))
    U = rand_unitary(1 << len(qubits), rng)
    psi = I.random_state(n, 29)
    ref, idx = _ld_apply(psi, qubits, U)
    with make(qe, n, "c128", psi=psi, max_k=5) as st:
        st.apply_gate(qubits, U)
        got = st.get()
    rel = _rel_group_error(got, ref, idx)
    assert rel < 4 * 2.0 ** -53, f"relative group error {rel:.3e}"


def test_fp64_mode_fft_at_fp64_rounding(qe):
    # the QFT definition (Sec. III-B) in long double for a 10-qubit register
    # inside a 12-qubit state; native FP64 butterflies and FP64 twiddles keep
    # the error within a few units of 2^-53 per radix-2 stage
    n, lo, m = 12, 1, 10
    psi = I.random_state(n, 61)
    N = 1 << m
    pi = np.longdouble("3.14159265358979323846264338327950288")
    k = np.arange(N)
    W = np.exp(np.clongdouble(2j) * pi * ((k[:, None] * k[None, :]) % N).astype(np.longdouble) / N)
    W /= np.sqrt(np.longdouble(N))
    x = np.arange(psi.size)
    reg = (x >> lo) & (N - 1)
    rest = x & ~((N - 1) << lo)
    ref = np.empty(psi.size, dtype=np.clongdouble)
    for r in np.unique(rest):
        sel = np.nonzero(rest == r)[0]
        order = sel[np.argsort(reg[sel])]
        ref[order] = W @ psi[order].astype(np.clongdouble)
    with make(qe, n, "c128", psi=psi) as st:
        st.set_policy(qe.POLICY_EMULATE, 1)
        st.apply_qft(lo, m)
        got = st.get()
    err = float(np.max(np.abs(got.astype(np.clongdouble) - ref)))
    rms = float(np.sqrt(np.mean(np.abs(ref) ** 2)))
    assert err / rms < m * 4 * 2.0 ** -53, f"relative error {err / rms:.3e}"


def test_fp64_mode_reductions_at_fp64_rounding(qe):
    # TFIM energy and marginals against long-double sums of the oracle's terms
    n = 14
    psi = I.random_state(n, 73)
    xm, zm, cf = I.tfim_terms(n)
    p = np.abs(psi.astype(np.clongdouble)) ** 2
    x = np.arange(psi.size)
    e_ref = np.longdouble(0)
    for i in range(n - 1):
        s = 1 - 2 * (((x >> i) ^ (x >> (i + 1))) & 1)
        e_ref += np.sum(p * s)
    for i in range(n):
        y = x ^ (1 << i)
        e_ref += np.longdouble(0.7) * np.sum((np.conj(psi[y].astype(np.clongdouble)) * psi.astype(np.clongdouble)).real)
    probs_ref = np.zeros(8, dtype=np.longdouble)
    for r in range(8):
        probs_ref[r] = np.sum(p[((x >> 3) & 7) == r])
    with make(qe, n, "c128", psi=psi) as st:
        e = st.expectation(xm, zm, cf)
        pr = st.probs([3, 4, 5])
    assert abs(np.longdouble(e) - e_ref) < 64 * 2.0 ** -53 * n
    assert float(np.max(np.abs(pr.astype(np.longdouble) - probs_ref))) < 16 * 2.0 ** -53
