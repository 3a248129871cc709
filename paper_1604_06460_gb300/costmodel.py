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


def sweep_subroutines(ns, dtypes=("c128", "c64"), seed=0):
    """Emulated and simulated QFTs and additions on registers of several sizes."""
    rng = np.random.default_rng(seed)
    X, y = [], []
    for dtype in dtypes:
        for n in ns:
            with qe.State(n, dtype) as st:
                st.init_random(1)
                for m in sorted({2, 4, n // 2, n - 2, n}):
                    if m < 1 or m > n:
                        continue
                    lo = n - m if m < n else 0
                    for op, pol in ((qe.OP_QFT_EMULATE, qe.POLICY_EMULATE), (qe.OP_QFT_SIMULATE, qe.POLICY_SIMULATE)):
                        st.set_policy(pol, 1)
                        ms = _time(lambda: st.apply_qft(lo, m), st.stream, reps=2)
                        X.append(qe.cost_features(op, n, dtype, 0, lo, lo + m - 1, m, 0))
                        y.append(np.log(ms))
                    reg = list(range(lo, lo + m))
                    c = int(rng.integers(1, 1 << m))
                    for op, pol in ((qe.OP_ADD_EMULATE, qe.POLICY_EMULATE), (qe.OP_ADD_SIMULATE, qe.POLICY_SIMULATE)):
                        st.set_policy(pol, 1)
                        ms = _time(lambda: st.add_const(reg, c), st.stream, reps=2)
                        X.append(qe.cost_features(op, n, dtype, 0, lo, lo + m - 1, m, c))
                        y.append(np.log(ms))
    return np.array(X, dtype=np.float32), np.array(y, dtype=np.float32)


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
