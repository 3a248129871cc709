"""The batch of ansatz circuits (one persistent launch in a CUDA graph)
against the oracle: every circuit's TFIM energy, for circuits that run whole
in shared memory and for circuits whose state lives in HBM (forced by small
tile sizes)."""
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


def oracle_energy(n, layers, seed, hx):
    psi = oracle.zero_state(n)
    for g in I.ansatz_circuit(n, layers, seed):
        oracle.apply_gate(psi, g.qubits, g.matrix, inplace=True)
    xm, zm, cf = I.tfim_terms(n, hx)
    return oracle.expectation(psi, xm, zm, cf)


def batch_inputs(ns, layers, seed0):
    return [I.ansatz_angles(int(n), layers, seed0 + i) for i, n in enumerate(ns)]


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 2e-4)])
@pytest.mark.parametrize("plan", [None, (6, 1, 128), (7, 3, 256), (8, 16, 128)])
def test_batch_energies_vs_oracle(qe, dtype, tol, plan):
    layers, hx = 3, 0.7
    ns = [1, 2, 3, 5, 7, 9, 11, 4, 6, 8, 10, 7, 3]
    angles = batch_inputs(ns, layers, 100)
    with qe.Batch(ns, angles, hx, dtype) as b:
        if plan is not None:
            b.set_plan(*plan)
        e1 = b.run()
        e2 = b.run()   # graph replay gives the same answer
    ref = np.array([oracle_energy(n, layers, 100 + i, hx) for i, n in enumerate(ns)])
    assert np.max(np.abs(e1 - ref)) < tol
    assert np.array_equal(e1, e2)


def test_batch_large_states_and_tuning(qe):
    layers, hx = 2, 0.7
    ns = [13, 14, 12, 15]
    angles = batch_inputs(ns, layers, 7)
    with qe.Batch(ns, angles, hx, "c128") as b:
        plan = b.tune(reps=1)
        e = b.run()
        info = b.info()
    ref = np.array([oracle_energy(n, layers, 7 + i, hx) for i, n in enumerate(ns)])
    assert np.max(np.abs(e - ref)) < 1e-11
    assert plan["tile_bits"] in (11, 12) and info["items"] > len(ns)


def test_batch_rejects_bad_input(qe):
    with pytest.raises(qe.QEError):
        qe.Batch([24], [np.zeros((1, 24, 2))], 0.7, "c128")
    with pytest.raises(qe.QEError):
        qe.Batch([3], [np.full((1, 3, 2), np.nan)], 0.7, "c128")


@pytest.mark.parametrize("dtype,tol", [("c128", 1e-11), ("c64", 5e-4)])
def test_batch_hbm_circuits_at_benchmark_sizes(qe, dtype, tol):
    # the benchmark's workload shape (8 layers, n drawn from 10..22) at the
    # default plan: circuits of 16-22 qubits live in HBM and take the
    # multi-CTA passes; sampled ones are checked against the oracle
    layers, hx, seed = 8, 0.7, 3
    ns = list(I.batch_sizes(48, 10, 22, seed)) + [16, 19, 22]
    angles = [I.ansatz_angles(int(n), layers, seed * 100000 + i) for i, n in enumerate(ns)]
    with qe.Batch(ns, angles, hx, dtype) as b:
        e = b.run()
    picks = [len(ns) - 3, len(ns) - 2, len(ns) - 1] + [i for i, n in enumerate(ns) if 16 <= n <= 21][:2]
    for i in picks:
        psi = oracle.zero_state(int(ns[i]))
        for g in I.ansatz_circuit(int(ns[i]), layers, seed * 100000 + i):
            oracle.apply_gate(psi, g.qubits, g.matrix, inplace=True)
        xm, zm, cf = I.tfim_terms(int(ns[i]), hx)
        ref = oracle.expectation(psi, xm, zm, cf)
        assert abs(e[i] - ref) < tol * max(1.0, abs(ref)), (i, ns[i], e[i], ref)


@pytest.mark.parametrize("plan", [None, (8, 3, 256), (9, 16, 128)])
def test_batch_fp64_energies_vs_oracle(qe, plan):
    # native FP64 gates and FP64 energy sums: shared-memory circuits and
    # circuits forced into HBM by small tiles, at FP64 rounding against the
    # oracle; switching back to double-float rebuilds the queue and agrees
    layers, hx = 3, 0.7
    ns = [1, 2, 3, 5, 7, 9, 11, 4, 6, 8, 10, 13, 14]
    angles = batch_inputs(ns, layers, 300)
    with qe.Batch(ns, angles, hx, "c128") as b:
        if plan is not None:
            b.set_plan(*plan)
        b.set_arith(qe.ARITH_FP64)
        e64 = b.run()
        b.set_arith(qe.ARITH_DF64)
        edf = b.run()
        with pytest.raises(qe.QEError):
            b.set_arith(7)
    ref = np.array([oracle_energy(n, layers, 300 + i, hx) for i, n in enumerate(ns)])
    assert np.max(np.abs(e64 - ref)) < 64 * n_terms_bound(ns)
    assert np.max(np.abs(edf - ref)) < 1e-11


def n_terms_bound(ns):
    # FP64 rounding: a few units of 2^-53 per term of the energy
    return 2.0 ** -53 * 2 * max(ns)
