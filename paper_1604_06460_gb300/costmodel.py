"""Timing sweeps that train the learned cost model, through the public API.

The emulator measures itself: each sample is one operation (a fused gate pass
of width k, an emulated or simulated QFT, an emulated or simulated addition)
timed with CUDA events on the state's stream, paired with the operation's
features (``qe.cost_features``).  ``train`` fits ``qe.CostModel`` to
log-milliseconds with the library's GPU kernels; ``save`` / ``load`` keep the
parameters in a small ``.npz`` file.
"""
from __future__ import annotations

import numpy as np

from . import qe


def _time(fn, stream, reps=3):
    import torch
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        fn()
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    return float(np.median(ts))


def _unitary(d, rng):
    z = rng.standard_normal((d, d)) + 1j * rng.standard_normal((d, d))
    q, r = np.linalg.qr(z)
    return q * (np.diag(r) / np.abs(np.diag(r)))[None, :]


def sweep_gate_passes(ns, dtypes=("c128", "c64"), ks=(1, 2, 3, 4, 5), seed=0):
    """One dense k-qubit pass per (n, dtype, k, placement): low qubits [0, k),
    high qubits [n-k, n) and a spread set."""
    rng = np.random.default_rng(seed)
    X, y = [], []
    for dtype in dtypes:
        for n in ns:
            with qe.State(n, dtype) as st:
                st.init_basis(0)
                for k in ks:
                    st.set_policy(qe.POLICY_ANALYTIC, k)
                    U = _unitary(1 << k, rng)
                    for qubits in (list(range(k)), list(range(n - k, n)),
                                   sorted(rng.choice(n, size=k, replace=False).tolist())):
                        ms = _time(lambda: (st.apply_gate(qubits, U), st.flush()), st.stream)
                        X.append(qe.cost_features(qe.OP_GATE, n, dtype, k, min(qubits), max(qubits)))
                        y.append(np.log(ms))
    return np.array(X, dtype=np.float32), np.array(y, dtype=np.float32)


def _constants(m, rng):
    """Added constants of different shapes: random, a single low bit, a
    single high bit and the two high bits."""
    cs = [int(rng.integers(1, 1 << m)), 1, 1 << (m - 1)]
    if m >= 2:
        cs.append(3 << (m - 2))
    return sorted(set(cs))


def sweep_subroutines(ns, dtypes=("c128",), seed=0, ms=(1, 2, 3, 5, 8, 12)):
    """Emulated and simulated QFTs and additions on registers of several
    sizes at the low end, the middle and the top of the state, with added
    constants of several shapes (the simulated adder's cost follows the set
    bits of the constant)."""
    rng = np.random.default_rng(seed)
    X, y = [], []
    for dtype in dtypes:
        for n in ns:
            with qe.State(n, dtype) as st:
                st.init_random(1)
                for m in ms:
                    if m > n:
                        continue
                    for lo in sorted({0, (n - m) // 2, n - m}):
                        for op, pol in ((qe.OP_QFT_EMULATE, qe.POLICY_EMULATE), (qe.OP_QFT_SIMULATE, qe.POLICY_SIMULATE)):
                            st.set_policy(pol, 1)
                            ms_ = _time(lambda: st.apply_qft(lo, m), st.stream, reps=2)
                            X.append(qe.cost_features(op, n, dtype, 0, lo, lo + m - 1, m, 0))
                            y.append(np.log(ms_))
                        reg = list(range(lo, lo + m))
                        for c in _constants(m, rng):
                            for op, pol in ((qe.OP_ADD_EMULATE, qe.POLICY_EMULATE),
                                            (qe.OP_ADD_SIMULATE, qe.POLICY_SIMULATE)):
                                st.set_policy(pol, 1)
                                ms_ = _time(lambda: st.add_const(reg, c), st.stream, reps=2)
                                X.append(qe.cost_features(op, n, dtype, 0, lo, lo + m - 1, m, c))
                                y.append(np.log(ms_))
    return np.array(X, dtype=np.float32), np.array(y, dtype=np.float32)


def decision_cases(n, seed=1):
    """Emulate-or-simulate decisions to score a policy on: QFTs of small and
    medium registers and additions of constants of every shape, at both ends
    of the state."""
    rng = np.random.default_rng(seed)
    cases = []
    for m in (1, 2, 3, 4, 6, 10):
        for lo in (0, n - m):
            cases.append(("qft", lo, m, 0))
    for m in (4, 8, 12, 16):
        for lo in (0, n - m):
            for c in _constants(m, rng):
                cases.append(("add", lo, m, c))
    return cases


# kernels that only the emulated QFT and addition launch (the simulated paths
# run elementwise 1-2-qubit gates, controlled phases and permutations)
_EMULATED = {"fft_pass", "fft_twiddle", "digitrev", "gate_tc_k5_c128", "gate_tc_k5_c128_df",
             "add_slice", "add_cluster", "add_walk", "add_bulk", "add_bulk_cluster"}


def _path(prof):
    """'emulated' or 'simulated' from the kernels a call launched."""
    return "emulated" if set(prof) & _EMULATED else "simulated"


def evaluate_decisions(n, cases, model, dtype="c128", reps=2):
    """For every case the measured time of both paths (CUDA events) and the
    path the analytic rule and the learned model choose; returns the cases
    and, per policy, the regret sum(chosen) / sum(best) - 1."""
    out = []
    with qe.State(n, dtype) as st:
        st.init_random(1)

        def run(kind, lo, m, c):
            if kind == "qft":
                st.apply_qft(lo, m)
            else:
                st.add_const(list(range(lo, lo + m)), c)

        for kind, lo, m, c in cases:
            t = {}
            for label, pol in (("emulated", qe.POLICY_EMULATE), ("simulated", qe.POLICY_SIMULATE)):
                st.set_policy(pol, 1)
                t[label] = _time(lambda: run(kind, lo, m, c), st.stream, reps=reps)
            choice = {}
            for label, pol, mdl in (("analytic", qe.POLICY_ANALYTIC, None), ("learned", qe.POLICY_AUTO, model)):
                st.set_cost_model(mdl)
                st.set_policy(pol, 1)
                st.profile(True)
                run(kind, lo, m, c)
                choice[label] = _path(st.profile_read())
                st.profile(False)
            st.set_cost_model(None)
            out.append({"op": kind, "lo": lo, "m": m, "c": c, "emulated_ms": t["emulated"],
                        "simulated_ms": t["simulated"], "best": min(t, key=t.get),
                        "analytic": choice["analytic"], "learned": choice["learned"]})
    best = sum(min(r["emulated_ms"], r["simulated_ms"]) for r in out)
    regret = {p: sum(r[r[p] + "_ms"] for r in out) / best - 1.0 for p in ("analytic", "learned")}
    return out, regret


def train(X, y, epochs=3000, lr=3e-3, seed=0, hidden=(32, 32)):
    model = qe.CostModel(hidden[0], hidden[1], seed)
    loss = model.train(X, y, epochs, lr)
    return model, loss


def save(model, path):
    np.savez(path, params=model.params(), hidden=np.array(model.hidden))


def load(path):
    d = np.load(path)
    model = qe.CostModel(int(d["hidden"][0]), int(d["hidden"][1]))
    model.set_params(d["params"])
    return model
