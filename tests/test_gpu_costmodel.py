"""The learned cost model: its GPU forward/backward kernels against the FP64
oracle network, training, and what it gains over the analytic rule when it
chooses the fusion width (results are identical whichever width it picks)."""
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


def test_gradient_and_forward_match_oracle(qe):
    h1, h2, n = 24, 16, 200
    rng = np.random.default_rng(0)
    m = qe.CostModel(h1, h2, seed=3)
    p = (rng.standard_normal(m.param_count()) * 0.3).astype(np.float32)
    m.set_params(p)
    X = rng.standard_normal((n, qe.N_FEATURES)).astype(np.float32)
    t = rng.standard_normal(n).astype(np.float32)
    loss, g = m.gradient(X, t)
    ref_loss, ref_g = oracle.mlp_grad(p.astype(np.float64), X.astype(np.float64),
                                      t.astype(np.float64), h1, h2)
    # FP32 kernels vs FP64 oracle: relative to the gradient's scale
    assert abs(loss - ref_loss) < 1e-5 * max(1.0, ref_loss)
    assert np.max(np.abs(g - ref_g)) < 1e-4 * max(1.0, np.max(np.abs(ref_g)))
    y = m.predict(X)
    yref = oracle.mlp_forward(p.astype(np.float64), X.astype(np.float64), h1, h2)
    assert np.max(np.abs(y - yref)) < 1e-5
    m.close()


def test_training_fits_a_smooth_target(qe):
    rng = np.random.default_rng(1)
    X = rng.uniform(0, 1, (300, qe.N_FEATURES)).astype(np.float32)
    t = (np.sin(3 * X[:, 0]) + X[:, 1] * X[:, 2] - 0.5 * X[:, 5]).astype(np.float32)
    m = qe.CostModel(32, 32, seed=1)
    before, _ = m.gradient(X, t)
    after = m.train(X, t, epochs=1500, lr=3e-3)
    assert after < 0.05 * before
    m.close()


def test_learned_fusion_width_beats_analytic_rule(qe, monkeypatch):
    """With the tensor cores switched off (QE_TENSOR_CORES=0), complex128
    passes are ALU-bound in double-float arithmetic for wide blocks, so the
    memory-only analytic rule (fewest passes = widest blocks) is slow; a model
    trained on the emulator's own timings picks a narrower width.  Both
    produce the same state.  (With the tensor cores on, 5-qubit blocks are the
    fastest and both choose them.)"""
    monkeypatch.setenv("QE_TENSOR_CORES", "0")
    from paper_1604_06460_gb300 import costmodel
    X, y = costmodel.sweep_gate_passes([22, 23, 24], dtypes=("c128",), seed=0)
    model, loss = costmodel.train(X, y, epochs=3000, lr=3e-3, seed=0)
    assert loss < 0.05
    n = 24
    gates = I.random_circuit(n, 6, seed=2)
    import torch
    times, states = {}, {}
    for label in ("analytic", "learned"):
        with qe.State(n, "c128") as st:
            st.set_policy(qe.POLICY_AUTO, 5)
            if label == "learned":
                st.set_cost_model(model)
            for g in gates:
                st.apply(g)
            k = st.planned_fusion_width()
            st.flush()
            ts = []
            for _ in range(3):
                st.init_basis(0)
                for g in gates:
                    st.apply(g)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st.stream)
                st.flush()
                e1.record(st.stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            times[label] = (k, float(np.median(ts)))
            states[label] = st.get()
    assert times["analytic"][0] == 5
    assert times["learned"][0] < 5
    assert times["learned"][1] < times["analytic"][1]
    assert np.max(np.abs(states["learned"] - states["analytic"])) < 1e-12
    print("fusion width / ms:", times)
    model.close()


def test_learned_subroutine_choice_is_emulation(qe):
    from paper_1604_06460_gb300 import costmodel
    X, y = costmodel.sweep_subroutines([16, 18], dtypes=("c128",), seed=0, ms=(1, 2, 3, 5, 8, 12, 16, 18))
    model, loss = costmodel.train(X, y, epochs=3000, lr=3e-3, seed=1)
    n = 18
    psi = I.random_state(n, 4)
    with qe.State(n, "c128") as st:
        st.set(psi)
        st.set_cost_model(model)
        st.set_policy(qe.POLICY_AUTO, 2)
        st.reset_stats()
        st.apply_qft(0, n)
        launches = st.stats()["launches"]
        got = st.get()
    # emulation: a few FFT or digit passes instead of n + n(n-1)/2 gate passes
    assert launches < 20
    # the result equals the transform computed by the other path
    with qe.State(n, "c128") as st2:
        st2.set(psi)
        st2.set_policy(qe.POLICY_SIMULATE, 1)
        st2.apply_qft(0, n)
        sim = st2.get()
    assert np.max(np.abs(got - sim)) < 1e-12
    model.close()


def test_learned_subroutine_choices_beat_analytic_rule(qe):
    """Tensor cores on, FP64 mode (the defaults).  The analytic rule prices a
    path by its memory traffic and FP64 arithmetic (Sec. III-B's models on one
    GPU) but not by how fast each kernel moves its bytes; the learned model,
    trained on the emulator's own timings of other state sizes, knows both.
    On a held-out size the two pick the emulated or the simulated path for
    QFTs and additions (constants of every shape, registers at both ends);
    the learned picks must cost less in total, measured on the GPU, and both
    paths give the same state (the parity tests of either path)."""
    from paper_1604_06460_gb300 import costmodel
    X, y = costmodel.sweep_subroutines([22, 24], dtypes=("c128",), seed=0)
    model, loss = costmodel.train(X, y, epochs=4000, lr=3e-3, seed=0)
    assert loss < 0.05
    cases = costmodel.decision_cases(25)
    res, regret = costmodel.evaluate_decisions(25, cases, model)
    for r in res:
        print(r)
    print("regret:", regret)
    # measured: the analytic rule emulates every addition, also those whose
    # constant has only high bits set (one or two multi-controlled-NOT passes
    # beat the register rotation) and those on registers of a few low qubits
    # (tiny shared-memory slices); the learned model simulates those
    assert regret["learned"] < 0.5 * regret["analytic"]
    model.close()
