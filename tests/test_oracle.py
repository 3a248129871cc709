"""Pins for the FP64 oracle against facts the paper and mathematics fix.

None of these compares the oracle with itself: each check uses a closed
form, a library routine the definition reduces to (numpy.kron, tensordot,
numpy.fft), an invariant, a printed example or brute force on tiny inputs.
The matrices are deliberately non-symmetric so that a transposed operand,
a wrong sign or a dropped term fails at least one test.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1604_06460_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def kron_list(ms):
    out = np.array([[1.0 + 0j]])
    for m in ms:
        out = np.kron(out, m)
    return out


def dense_1q(n, q, U):
    """Sec. II construction: Kronecker product of n 2x2 factors, identity
    except at qubit q; the leftmost factor is the highest qubit."""
    return kron_list([U if j == q else np.eye(2) for j in reversed(range(n))])


def tensordot_apply(psi, n, qubits, U):
    """Apply U by numpy.tensordot on the (2,)*n tensor; axis n-1-q is qubit q
    and the matrix index bit j is qubits[j] (so the reshaped U has its
    most significant axis first, i.e. qubits in reverse order)."""
    k = len(qubits)
    T = psi.reshape((2,) * n)
    Ut = U.reshape((2,) * (2 * k))
    axes_in = [n - 1 - q for q in reversed(qubits)]
    out = np.tensordot(Ut, T, axes=(list(range(k, 2 * k)), axes_in))
    # tensordot puts the k output axes first (in reversed-qubit order)
    out = np.moveaxis(out, list(range(k)), axes_in)
    return out.reshape(-1)


def rand_unitary(d, rng):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


# --- Philox: the published known-answer vectors ---------------------------
def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = oracle.philox4x32_10(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


# --- Sec. II: qubit order, Kronecker construction ----------------------------
def test_kron_example_is_not_on_qubit_1():
    rows = [l.split() for l in open(os.path.join(GOLD, "kron_not_example.txt"))
            if l.strip() and not l.startswith("#")]
    M = np.array(rows, dtype=float)
    cols = []
    for b in range(4):
        e = np.zeros(4, complex)
        e[b] = 1
        cols.append(oracle.apply_gate(e, [1], I.mat_x()))
    assert np.array_equal(np.array(cols).T.real, M)


def test_x_on_qubit0_maps_zero_to_index1():
    out = oracle.apply_gate(oracle.zero_state(3), [0], I.mat_x())
    assert out[1] == 1 and np.count_nonzero(out) == 1


@pytest.mark.parametrize("n,q", [(1, 0), (3, 0), (3, 2), (5, 3)])
def test_1q_gate_vs_kron(n, q):
    rng = np.random.default_rng(n * 10 + q)
    U = I.haar_u2(rng)
    psi = I.random_state(n, 7 + q)
    ref = dense_1q(n, q, U) @ psi
    got = oracle.apply_gate(psi, [q], U)
    assert np.max(np.abs(got - ref)) < 1e-14


def test_adjacent_2q_gate_vs_kron():
    # a 2-qubit gate on (q, q+1): matrix index bit 0 <-> q, bit 1 <-> q+1, so
    # in Kronecker order the gate's 4x4 block sits at factor position of q+1,q.
    n, q = 5, 1
    rng = np.random.default_rng(3)
    U = rand_unitary(4, rng)
    psi = I.random_state(n, 11)
    dense = kron_list([np.eye(2)] * (n - q - 2) + [U] + [np.eye(2)] * q)
    got = oracle.apply_gate(psi, [q, q + 1], U)
    assert np.max(np.abs(got - dense @ psi)) < 1e-14


@pytest.mark.parametrize("qubits", [[0], [4], [2, 0], [1, 5], [5, 1, 3], [0, 6, 2, 4], [6, 0, 3, 1, 5]])
def test_kq_gate_vs_tensordot(qubits):
    n = 7
    rng = np.random.default_rng(sum(qubits) + len(qubits))
    U = rand_unitary(1 << len(qubits), rng)
    psi = I.random_state(n, 5)
    ref = tensordot_apply(psi, n, qubits, U)
    got = oracle.apply_gate(psi, qubits, U)
    assert np.max(np.abs(got - ref)) < 1e-13


def test_cnot_truth_table_table1():
    # Table I CNOT: control is the matrix's high bit; cnot(c, t) flips t iff c.
    n = 3
    for b in range(8):
        e = np.zeros(8, complex)
        e[b] = 1
        g = I.cnot(2, 0)
        out = oracle.apply_gate(e, g.qubits, g.matrix)
        want = b ^ 1 if (b >> 2) & 1 else b
        assert out[want] == 1


def test_controlled_vs_projector_sum():
    # C-U = |0><0| (x) 1 + |1><1| (x) U on (control 2, target 0), n = 3
    rng = np.random.default_rng(1)
    U = I.haar_u2(rng)
    P0 = np.diag([1, 0]).astype(complex)
    P1 = np.diag([0, 1]).astype(complex)
    dense = kron_list([P0, np.eye(2), np.eye(2)]) + kron_list([P1, np.eye(2), U])
    psi = I.random_state(3, 2)
    got = oracle.apply_controlled(psi, [2], [0], U)
    assert np.max(np.abs(got - dense @ psi)) < 1e-14


def test_mcx_truth_table():
    n = 5
    for b in range(32):
        e = np.zeros(32, complex)
        e[b] = 1
        out = oracle.apply_mcx(e, [0, 3, 4], 2)
        want = b ^ 4 if (b & 0b11001) == 0b11001 else b
        assert out[want] == 1


def test_ghz_closed_form():
    n = 6
    psi = oracle.zero_state(n)
    for g in I.ghz_circuit(n):
        psi = oracle.apply_gate(psi, g.qubits, g.matrix)
    want = np.zeros(1 << n, complex)
    want[0] = want[-1] = 1 / np.sqrt(2)
    assert np.max(np.abs(psi - want)) < 1e-15


def test_random_circuit_norm_and_inverse():
    n = 8
    gates = I.random_circuit(n, 4, seed=9)
    psi = oracle.zero_state(n)
    for g in gates:
        psi = oracle.apply_gate(psi, g.qubits, g.matrix)
    assert abs(oracle.norm2(psi) - 1) < 1e-13
    for g in reversed(gates):
        psi = oracle.apply_gate(psi, g.qubits, g.matrix.conj().T)
    assert abs(psi[0] - 1) < 1e-13 and np.max(np.abs(psi[1:])) < 1e-13


def test_dense_brute_force_circuit_n6():
    # whole circuit as the product of dense Kronecker matrices (Sec. II)
    n = 6
    rng = np.random.default_rng(4)
    ops = []
    psi = I.random_state(n, 3)
    ref = psi.copy()
    for _ in range(10):
        q = int(rng.integers(n))
        U = I.haar_u2(rng)
        ops.append((q, U))
    for q, U in ops:
        ref = dense_1q(n, q, U) @ ref
        psi = oracle.apply_gate(psi, [q], U)
    assert np.max(np.abs(psi - ref)) < 1e-14


# --- Sec. III-B: QFT -------------------------------------------------------
@pytest.mark.parametrize("m", [1, 2, 3, 6])
def test_qft_dft_equals_numpy_ifft(m):
    # alpha_l -> 2^{-m/2} sum_k alpha_k e^{+2 pi i k l / 2^m} is numpy's
    # inverse FFT (sign +, scale 1/N) times sqrt(N).
    psi = I.random_state(m, m)
    ref = np.fft.ifft(psi) * np.sqrt(1 << m)
    assert np.max(np.abs(oracle.qft_dft(psi, 0, m) - ref)) < 1e-14
    ref_inv = np.fft.fft(psi) / np.sqrt(1 << m)
    assert np.max(np.abs(oracle.qft_dft(psi, 0, m, inverse=True) - ref_inv)) < 1e-14


def test_qft_subregister_batched_vs_numpy():
    # QFT on qubits [2, 6) of n = 8: independent transforms along axis of stride 4
    n, lo, m = 8, 2, 4
    psi = I.random_state(n, 21)
    T = psi.reshape(1 << (n - lo - m), 1 << m, 1 << lo)
    ref = (np.fft.ifft(T, axis=1) * np.sqrt(1 << m)).reshape(-1)
    assert np.max(np.abs(oracle.qft_dft(psi, lo, m) - ref)) < 1e-14


@pytest.mark.parametrize("x", [0, 1, 5, 13])
def test_qft_basis_state_closed_form(x):
    m = 4
    e = np.zeros(1 << m, complex)
    e[x] = 1
    out = oracle.qft_dft(e, 0, m)
    l = np.arange(1 << m)
    want = np.exp(2j * np.pi * ((x * l) % (1 << m)) / (1 << m)) / np.sqrt(1 << m)
    assert np.max(np.abs(out - want)) < 1e-15


@pytest.mark.parametrize("lo,m,inv", [(0, 5, False), (1, 4, False), (2, 3, True), (0, 6, True)])
def test_qft_circuit_equals_definition(lo, m, inv):
    n = 7
    psi = I.random_state(n, lo * 10 + m)
    a = oracle.qft_dft(psi, lo, m, inverse=inv)
    b = oracle.qft_circuit(psi, lo, m, inverse=inv)
    assert np.max(np.abs(a - b)) < 1e-13


def test_qft_parseval_square_and_inverse():
    m = 7
    psi = I.random_state(m, 77)
    f = oracle.qft_dft(psi, 0, m)
    assert abs(oracle.norm2(f) - 1) < 1e-14
    ff = oracle.qft_dft(f, 0, m)
    idx = (-np.arange(1 << m)) % (1 << m)   # QFT^2 maps k -> -k mod 2^m
    assert np.max(np.abs(ff - psi[idx])) < 1e-14
    back = oracle.qft_dft(f, 0, m, inverse=True)
    assert np.max(np.abs(back - psi)) < 1e-14


def test_qft_single_amplitude_matches_dft():
    n, lo, m = 9, 1, 6
    psi = I.random_state(n, 8)
    full = oracle.qft_dft(psi, lo, m)
    for idx in [0, 3, 77, 300, 511]:
        v = oracle.qft_amplitude(psi, lo, m, idx)
        assert abs(v - full[idx]) < 1e-15
        vi = oracle.qft_amplitude(psi, lo, m, idx, inverse=True)
        assert abs(vi - oracle.qft_dft(psi, lo, m, inverse=True)[idx]) < 1e-15


# --- Sec. III-A: addition as a permutation ----------------------------------
def test_add_const_exhaustive_basis_states():
    n, qubits = 6, [1, 2, 3, 4]
    m = len(qubits)
    for c in [0, 1, 7, 15, 9]:
        for x in range(1 << n):
            e = np.zeros(1 << n, complex)
            e[x] = 1
            out = oracle.add_const(e, qubits, c)
            r = sum(((x >> q) & 1) << j for j, q in enumerate(qubits))
            r2 = (r + c) % (1 << m)
            x2 = x & ~sum(1 << q for q in qubits)
            x2 |= sum(((r2 >> j) & 1) << q for j, q in enumerate(qubits))
            assert out[x2] == 1 and np.count_nonzero(out) == 1


def test_add_const_permuted_register_order():
    # register bits listed out of order: bit j of r is qubits[j]
    n, qubits, c = 5, [3, 0, 4], 5
    for x in range(32):
        e = np.zeros(32, complex)
        e[x] = 1
        out = oracle.add_const(e, qubits, c)
        r = ((x >> 3) & 1) | (((x >> 0) & 1) << 1) | (((x >> 4) & 1) << 2)
        r2 = (r + c) % 8
        x2 = (x & ~0b11001) | ((r2 & 1) << 3) | (((r2 >> 1) & 1) << 0) | (((r2 >> 2) & 1) << 4)
        assert out[x2] == 1


@pytest.mark.parametrize("qubits,c", [([0, 1, 2, 3, 4], 13), ([2, 3, 4, 5], 11), ([5, 1, 3], 6), ([0, 1, 2, 3, 4, 5, 6], 100)])
def test_add_const_circuit_equals_permutation_bit_exact(qubits, c):
    psi = I.random_state(7, c)
    a = oracle.add_const(psi, qubits, c)
    b = oracle.add_const_circuit(psi, qubits, c)
    assert np.array_equal(a, b)


def test_add_const_roundtrip_identity():
    psi = I.random_state(8, 3)
    q = [0, 1, 2, 3, 4, 5]
    c = 37
    out = oracle.add_const(oracle.add_const(psi, q, c), q, (1 << 6) - c)
    assert np.array_equal(out, psi)


# --- Sec. III-D: expectation values and probabilities ----------------------
def dense_pauli(n, xm, zm):
    X, Y, Z = I.mat_x(), I.mat_y(), I.mat_z()
    fs = []
    for q in reversed(range(n)):
        xb, zb = (xm >> q) & 1, (zm >> q) & 1
        fs.append(Y if xb and zb else X if xb else Z if zb else np.eye(2))
    return kron_list(fs)


def test_tfim_closed_forms():
    n = 6
    xm, zm, cf = I.tfim_terms(n)
    assert abs(oracle.expectation(oracle.zero_state(n), xm, zm, cf) - (n - 1)) < 1e-14
    plus = np.full(1 << n, 1 / np.sqrt(1 << n), complex)
    assert abs(oracle.expectation(plus, xm, zm, cf) - 0.7 * n) < 1e-13


@pytest.mark.parametrize("n,seed", [(2, 4), (7, 5)])
def test_one_layer_ansatz_tfim_energy_closed_form(n, seed):
    # RY(theta) then RZ(phi) on |0> gives <Z> = cos theta, <X> = sin theta
    # cos phi; the CZ ladder commutes with every Z_i Z_{i+1} and turns X_i
    # into Z_{i-1} X_i Z_{i+1}, whose mean factorises over the product state.
    psi = oracle.zero_state(n)
    for g in I.ansatz_circuit(n, 1, seed):
        psi = oracle.apply_gate(psi, g.qubits, g.matrix)
    th, ph = I.ansatz_angles(n, 1, seed)[0].T
    zz = sum(np.cos(th[i]) * np.cos(th[i + 1]) for i in range(n - 1))
    x = sum(np.sin(th[i]) * np.cos(ph[i]) * np.prod([np.cos(th[j]) for j in (i - 1, i + 1) if 0 <= j < n])
            for i in range(n))
    xm, zm, cf = I.tfim_terms(n)
    assert abs(oracle.expectation(psi, xm, zm, cf) - (zz + 0.7 * x)) < 1e-13


def test_expectation_dense_brute_force():
    n = 6
    rng = np.random.default_rng(12)
    xm = rng.integers(0, 1 << n, size=6).astype(np.uint64)
    zm = rng.integers(0, 1 << n, size=6).astype(np.uint64)
    cf = rng.standard_normal(6)
    psi = I.random_state(n, 13)
    H = sum(c * dense_pauli(n, int(x), int(z)) for x, z, c in zip(xm, zm, cf))
    ref = np.vdot(psi, H @ psi).real
    assert abs(oracle.expectation(psi, xm, zm, cf) - ref) < 1e-13


def test_y_eigenstate():
    # |+i> = (|0> + i|1>)/sqrt 2 is the +1 eigenstate of Y
    psi = np.array([1, 1j]) / np.sqrt(2)
    assert abs(oracle.expectation(psi, [1], [1], [1.0]) - 1) < 1e-15


def test_probs_ghz_and_product_state():
    n = 5
    psi = oracle.zero_state(n)
    for g in I.ghz_circuit(n):
        psi = oracle.apply_gate(psi, g.qubits, g.matrix)
    p = oracle.probs(psi, [0, 3])
    assert np.allclose(p, [0.5, 0, 0, 0.5], atol=1e-15)
    # product state RY(a) (x) RY(b): P(bit=1) = sin^2(theta/2)
    a, b = 0.3, 1.1
    st = np.kron(I.mat_ry(b) @ [1, 0], I.mat_ry(a) @ [1, 0])
    p = oracle.probs(st, [0, 1])
    pa, pb = np.sin(a / 2) ** 2, np.sin(b / 2) ** 2
    assert np.allclose(p, [(1 - pa) * (1 - pb), pa * (1 - pb), (1 - pa) * pb, pa * pb], atol=1e-15)


def test_probs_sum_to_norm_and_order():
    psi = I.random_state(7, 31)
    p = oracle.probs(psi, [6, 2, 0])
    assert abs(p.sum() - 1) < 1e-14
    # out[r], bit j of r <-> qubits[j]
    x = 0b1000100  # qubits 6 and 2 set -> r = 0b011
    e = np.zeros(128, complex)
    e[x] = 1
    assert oracle.probs(e, [6, 2, 0])[3] == 1


# --- the seeded random state ----------------------------------------------
def test_gaussian_state_normalised_and_slices():
    n = 12
    psi = oracle.gaussian_state(n, 1234)
    assert abs(oracle.norm2(psi) - 1) < 1e-14
    raw = oracle.gaussian_slice(1234, 0, 1 << n)
    scale = np.sqrt(np.vdot(raw, raw).real)
    assert np.max(np.abs(raw / scale - psi)) < 1e-15
    # standard complex Gaussian: E re^2 = E im^2 = 1, mean 0
    big = oracle.gaussian_slice(99, 1 << 40, 1 << 16)
    assert abs(np.mean(big.real ** 2) - 1) < 0.03 and abs(np.mean(big.imag ** 2) - 1) < 0.03
    assert abs(np.mean(big.real)) < 0.02 and abs(np.mean(big.imag)) < 0.02
    # re and im independent: zero correlation, |z|^2 exponential with mean 2
    assert abs(np.mean(big.real * big.imag)) < 0.02
    assert abs(np.mean(np.abs(big) ** 2) - 2) < 0.05


def test_gaussian_amplitude_by_hand_from_the_first_known_answer():
    # Amplitude 0 of seed 0 uses counter (0, 0, 0, 0) and key (0, 0): the first
    # published Philox4x32-10 vector.  Its words give, by the stated recipe,
    # u1 = ((w1:w0 >> 11) + 1) 2^-53 in (0, 1], u2 = (w3:w2 >> 11) 2^-53 in
    # [0, 1), re + i im = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2).  A
    # swapped word order, a lost "+ 1", u1/u2 exchanged or one phase for both
    # parts each change this value.
    import math
    row = [l.split() for l in open(os.path.join(GOLD, "philox4x32_10_kat.txt"))
           if l.strip() and not l.startswith("#")][0]
    v = [int(x, 16) for x in row]
    assert v[0:6] == [0] * 6
    w0, w1, w2, w3 = v[6:10]
    a = (w1 << 32) | w0
    b = (w3 << 32) | w2
    u1 = ((a >> 11) + 1) / 2.0 ** 53
    u2 = (b >> 11) / 2.0 ** 53
    r = math.sqrt(-2.0 * math.log(u1))
    want = complex(r * math.cos(2 * math.pi * u2), r * math.sin(2 * math.pi * u2))
    got = complex(oracle.gaussian_slice(0, 0, 1)[0])
    assert abs(got - want) < 1e-15 * max(1.0, abs(want))
    # the raw words: 0xe169c58d6627e8d5 and 0x9b00dbd8bc57ac4c
    assert a == 0xE169C58D6627E8D5 and b == 0x9B00DBD8BC57AC4C


# --- the cost model's network: pinned by finite differences -------------------
def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    d, h1, h2, n = 5, 7, 4, 9
    npar = oracle.mlp_param_count(d, h1, h2)
    assert npar == h1 * d + h1 + h2 * h1 + h2 + h2 + 1
    p = rng.standard_normal(npar) * 0.5
    X = rng.standard_normal((n, d))
    t = rng.standard_normal(n)
    loss, g = oracle.mlp_grad(p, X, t, h1, h2)
    y = oracle.mlp_forward(p, X, h1, h2)
    assert abs(loss - np.mean((y - t) ** 2)) < 1e-14
    eps = 1e-6
    fd = np.empty(npar)
    for k in range(npar):
        pp, pm = p.copy(), p.copy()
        pp[k] += eps
        pm[k] -= eps
        fd[k] = (np.mean((oracle.mlp_forward(pp, X, h1, h2) - t) ** 2)
                 - np.mean((oracle.mlp_forward(pm, X, h1, h2) - t) ** 2)) / (2 * eps)
    assert np.max(np.abs(fd - g)) < 1e-8


def test_mlp_forward_closed_form():
    # one hidden unit per layer, identity-like weights: y = w3 tanh(w2 tanh(w1 x + b1) + b2) + b3
    d, h1, h2 = 1, 1, 1
    p = np.array([0.3, -0.2, 1.5, 0.1, -2.0, 0.25])
    x = np.array([[0.7]])
    want = -2.0 * np.tanh(1.5 * np.tanh(0.3 * 0.7 - 0.2) + 0.1) + 0.25
    assert abs(oracle.mlp_forward(p, x, h1, h2)[0] - want) < 1e-15


def test_threaded_gate_loops_are_bit_identical():
    # the OpenMP gate loops split the independent groups among threads; every
    # group is computed by the same loop, so the state is bit-identical
    n = 12
    gates = I.random_circuit(n, 3, seed=4)
    out = []
    for t in (1, max(2, oracle.max_threads())):
        oracle.set_threads(t)
        psi = oracle.gaussian_state(n, 9)
        for g in gates:
            oracle.apply_gate(psi, g.qubits, g.matrix, inplace=True)
        oracle.apply_controlled(psi, [1, 5], [3], I.haar_u2(np.random.default_rng(2)), inplace=True)
        oracle.apply_mcx(psi, [0, 7], 11, inplace=True)
        out.append(psi)
    oracle.set_threads(oracle.max_threads())
    assert np.array_equal(out[0], out[1])


# --- Sec. III-A multiplication and division permutations ----------------------
def _reg_value(x, qs):
    return sum(((x >> q) & 1) << j for j, q in enumerate(qs))


def _basis_images(fn, n, qa, qb, qc):
    """Image index of every basis state under the oracle map fn."""
    out = []
    for x in range(1 << n):
        e = np.zeros(1 << n, complex)
        e[x] = 1
        y = fn(e, qa, qb, qc)
        nz = np.nonzero(y)[0]
        assert nz.size == 1 and y[nz[0]] == 1
        out.append(int(nz[0]))
    return out


@pytest.mark.parametrize("N,order", [(1, "abc"), (2, "abc"), (3, "abc"), (2, "mixed")])
def test_mul_is_the_paper_map_on_c0_and_a_permutation(N, order):
    # (a, b, 0) -> (a, b, ab mod 2^N), Python's integer product as reference;
    # every basis state goes to a distinct basis state
    if order == "abc":   # paper's layout: c in the low qubits, then b, then a
        qc, qb, qa = list(range(N)), list(range(N, 2 * N)), list(range(2 * N, 3 * N))
    else:
        qa, qb, qc = [4, 0], [2, 5], [1, 3]
    n = 3 * N
    img = _basis_images(oracle.mul, n, qa, qb, qc)
    assert sorted(img) == list(range(1 << n))
    for x in range(1 << n):
        a, b, c = _reg_value(x, qa), _reg_value(x, qb), _reg_value(x, qc)
        y = img[x]
        assert _reg_value(y, qa) == a and _reg_value(y, qb) == b
        if c == 0:
            assert _reg_value(y, qc) == (a * b) % (1 << N)


@pytest.mark.parametrize("N,order", [(1, "abc"), (2, "abc"), (3, "abc"), (3, "mixed")])
def test_div_is_the_paper_map_on_c0_and_a_permutation(N, order):
    # (a, b, 0) -> (a mod b, b, a div b) for b != 0 (Python's divmod), the
    # identity for b = 0; a permutation of all basis states
    if order == "abc":
        qc, qb, qa = list(range(N)), list(range(N, 2 * N)), list(range(2 * N, 3 * N))
    else:
        qa, qb, qc = [8, 1, 4], [0, 6, 2], [5, 3, 7]
    n = 3 * N
    img = _basis_images(oracle.div, n, qa, qb, qc)
    assert sorted(img) == list(range(1 << n))
    for x in range(1 << n):
        a, b, c = _reg_value(x, qa), _reg_value(x, qb), _reg_value(x, qc)
        y = img[x]
        assert _reg_value(y, qb) == b
        if c == 0:
            q, r = divmod(a, b) if b else (0, a)
            assert (_reg_value(y, qa), _reg_value(y, qc)) == (r, q)


@pytest.mark.parametrize("N", [1, 2, 3, 4])
def test_mul_circuit_equals_permutation_bit_exact(N):
    qc, qb, qa = list(range(N)), list(range(N, 2 * N)), list(range(2 * N, 3 * N))
    psi = oracle.gaussian_state(3 * N, 50 + N)
    assert np.array_equal(oracle.mul_circuit(psi, qa, qb, qc), oracle.mul(psi, qa, qb, qc))


def test_mul_applied_2_to_the_N_times_is_the_identity():
    # c -> c + 2^N ab = c (mod 2^N)
    N = 3
    qc, qb, qa = [0, 1, 2], [3, 4, 5], [6, 7, 8]
    psi = oracle.gaussian_state(9, 4)
    x = psi.copy()
    for _ in range(1 << N):
        x = oracle.mul(x, qa, qb, qc)
    assert np.array_equal(x, psi)


# --- Sec. II measurement: sampling and collapse -------------------------------
def _exact_state():
    # probabilities 1/4, 1/4, 1/4, 1/16 x 4, 0: exact in binary
    return np.array([0.5, 0.5j, -0.5, 0.25, -0.25j, 0.25, 0.25, 0.0], dtype=complex)


def test_sample_inverse_cdf_closed_form():
    psi = _exact_state()
    # cumulative: 0.25 0.5 0.75 0.8125 0.875 0.9375 1 1
    u = [0.0, 0.2499, 0.25, 0.5, 0.8125, 0.9, 0.9375, 0.99999]
    got = oracle.sample(psi, [0, 1, 2], u)
    assert list(got) == [0, 0, 1, 2, 4, 5, 6, 6]    # index 7 (probability 0) never
    # marginal of qubit 2: P(0) = 13/16 (x = 0..3), P(1) = 3/16; qubits (2, 0): r = b2 + 2 b0
    assert list(oracle.sample(psi, [2], [0.7, 0.8125, 0.9])) == [0, 1, 1]
    # P(r) for (q2, q0): r=0: x in {0,2}: 1/2; r=1: {4,6}: 1/8; r=2: {1,3}: 5/16; r=3: {5,7}: 1/16
    assert list(oracle.sample(psi, [2, 0], [0.49, 0.5, 0.62, 0.63, 0.95])) == [0, 1, 1, 2, 3]


def test_sample_frequencies_match_probabilities():
    # a statistical property: frequencies of 40000 samples within 5 sigma
    psi = I.random_state(6, 3)
    p = np.abs(psi) ** 2
    u = np.random.default_rng(1).random(40000)
    s = oracle.sample(psi, list(range(6)), u)
    f = np.bincount(s.astype(np.int64), minlength=64) / u.size
    sigma = np.sqrt(p * (1 - p) / u.size)
    assert np.all(np.abs(f - p) < 5 * sigma + 1e-12)


def test_collapse_closed_forms():
    n = 5
    ghz = np.zeros(1 << n, complex)
    ghz[0] = ghz[-1] = 2 ** -0.5
    post, p = oracle.collapse(ghz, [3], 1)
    want = np.zeros(1 << n, complex)
    want[-1] = 1
    assert abs(p - 0.5) < 1e-15 and np.allclose(post, want, atol=1e-15, rtol=0)
    # product state |+>|0>|1> (qubits 0, 1, 2): measuring qubit 0 as 1 leaves |1>|0>|1>
    plus = np.array([1, 1]) / np.sqrt(2)
    prod = np.kron(np.array([0, 1]), np.kron(np.array([1, 0]), plus)).astype(complex)
    post, p = oracle.collapse(prod, [0], 1)
    assert abs(p - 0.5) < 1e-15
    e = np.zeros(8, complex)
    e[0b101] = 1
    assert np.allclose(post, e, atol=1e-15, rtol=0)
    # an outcome of probability zero leaves the state unchanged
    post, p = oracle.collapse(prod, [1], 1)
    assert p == 0 and np.array_equal(post, prod)


def test_collapse_renormalises_and_fixes_the_measured_bits():
    psi = I.random_state(7, 8)
    post, p = oracle.collapse(psi, [5, 1], 2)        # qubit 5 = 0, qubit 1 = 1
    assert abs(p - oracle.probs(psi, [5, 1])[2]) < 1e-15
    assert abs(oracle.norm2(post) - 1) < 1e-14
    pr = oracle.probs(post, [5, 1])
    assert abs(pr[2] - 1) < 1e-14 and abs(pr.sum() - 1) < 1e-14


# --- Sec. III-C phase estimation ----------------------------------------------
def test_dense_unitary_matches_kronecker_products():
    # single-qubit gates on distinct qubits: U = kron of the factors (numpy),
    # qubit 0 the rightmost factor (little-endian)
    rng = np.random.default_rng(5)
    A, B2 = I.haar_u2(rng), I.haar_u2(rng)
    gates = [I.single(0, A), I.single(2, B2)]
    U = oracle.dense_unitary(3, gates)
    want = np.kron(B2, np.kron(np.eye(2), A))
    assert np.max(np.abs(U - want)) < 1e-15
    # a CNOT then: the product of the two matrices (numpy's matmul)
    cx = oracle.dense_unitary(3, [I.cnot(0, 1)])
    U2 = oracle.dense_unitary(3, gates + [I.cnot(0, 1)])
    assert np.max(np.abs(U2 - cx @ U)) < 1e-15


def test_qpe_circuit_reads_exact_phases():
    # U diagonal with eigenvalues exp(2 pi i k / 2^b) on basis states: the
    # ancilla register ends exactly in |k> (closed form of phase estimation)
    n, b = 2, 4
    # phase of basis state x: 2 pi (3 x0 + 5 x1) / 16 via two RZ-like diagonal gates
    def phase_gate(q, k):
        return I.Gate((q,), np.diag([1.0, np.exp(2j * np.pi * k / 16)]), (), "p")
    gates = [phase_gate(0, 3), phase_gate(1, 5)]
    for x in range(4):
        e = np.zeros(4, complex)
        e[x] = 1
        out = oracle.qpe_circuit(e, n, b, gates)
        k = (3 * (x & 1) + 5 * (x >> 1)) % 16
        assert abs(abs(out[(k << n) | x]) - 1) < 1e-12
