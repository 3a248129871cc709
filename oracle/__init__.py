"""FP64 CPU oracle for the state-vector path (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``oracle.c`` (plain C, FP64,
compiled with gcc) through ctypes; it imports nothing from the CUDA package
and the CUDA package imports nothing from it.

Every function takes and returns numpy arrays; states are ``complex128``
arrays of length 2**n, qubit q <-> bit q of the index.  The paper passage each
function follows is cited in ``oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "oracle.c"
_LIB_DIR = _HERE / "_build"
_LIB = _LIB_DIR / "liboracle.so"
_lib = None


def build(force: bool = False) -> Path:
    """Compile ``oracle.c`` into ``oracle/_build/liboracle.so`` with gcc."""
    _LIB_DIR.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB_DIR / f"liboracle.{os.getpid()}.so"
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(tmp), str(_SRC)]
        # OpenMP for the gate loops when the compiler has it; otherwise one thread
        if subprocess.run(base + ["-fopenmp", "-lm"], capture_output=True).returncode != 0:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(str(_LIB))
        dp = C.c_void_p
        i, u64, d = C.c_int, C.c_uint64, C.c_double
        sig = {
            "or_philox4x32_10": (None, [dp, dp, dp]),
            "or_set_threads": (None, [i]),
            "or_max_threads": (i, []),
            "or_norm2": (d, [dp, i]),
            "or_init_zero": (None, [dp, i]),
            "or_init_gaussian": (None, [dp, i, u64]),
            "or_gaussian_slice": (None, [dp, u64, u64, u64]),
            "or_apply_gate": (None, [dp, i, i, dp, dp]),
            "or_apply_controlled": (None, [dp, i, i, dp, i, dp, dp]),
            "or_apply_mcx": (None, [dp, i, i, dp, i]),
            "or_qft_dft": (None, [dp, i, i, i, i]),
            "or_qft_amplitude": (None, [dp, i, i, i, i, u64, dp, dp]),
            "or_qft_circuit": (None, [dp, i, i, i, i]),
            "or_add_const": (None, [dp, i, i, dp, u64]),
            "or_add_const_circuit": (None, [dp, i, i, dp, u64]),
            "or_mul": (None, [dp, i, i, dp, dp, dp]),
            "or_div": (None, [dp, i, i, dp, dp, dp]),
            "or_mul_circuit": (None, [dp, i, i, dp, dp, dp]),
            "or_expectation": (d, [dp, i, i, dp, dp, dp]),
            "or_probs": (None, [dp, i, i, dp, dp]),
            "or_sample": (None, [dp, i, i, dp, i, dp, dp]),
            "or_collapse": (d, [dp, i, i, dp, u64]),
            "or_mlp_param_count": (i, [i, i, i]),
            "or_mlp_forward": (None, [dp, i, i, i, dp, i, dp]),
            "or_mlp_grad": (d, [dp, i, i, i, dp, dp, i, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _state(psi):
    a = np.ascontiguousarray(psi, dtype=np.complex128)
    n = int(a.size).bit_length() - 1
    if a.ndim != 1 or a.size != (1 << n):
        raise ValueError("state must be a 1-D array of length 2**n")
    return a, n


def _ints(xs):
    return np.ascontiguousarray(np.asarray(xs, dtype=np.int32))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def set_threads(t):
    """Host threads for the gate loops (OpenMP; no effect without it)."""
    _load().or_set_threads(int(t))


def max_threads():
    """Threads the gate loops use (1 when the oracle was built without OpenMP)."""
    return int(_load().or_max_threads())


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32))
    out = np.zeros(4, dtype=np.uint32)
    _load().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def zero_state(n):
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().or_init_zero(_ptr(psi), n)
    return psi


def gaussian_state(n, seed):
    psi = np.empty(1 << n, dtype=np.complex128)
    _load().or_init_gaussian(_ptr(psi), n, seed)
    return psi


def gaussian_slice(seed, i0, count):
    out = np.empty(count, dtype=np.complex128)
    _load().or_gaussian_slice(_ptr(out), seed, i0, count)
    return out


def norm2(psi):
    a, n = _state(psi)
    return _load().or_norm2(_ptr(a), n)


def apply_gate(psi, qubits, matrix, inplace=False):
    """The gate applied to a copy of psi (to psi itself, a C-contiguous
    complex128 array, with inplace=True)."""
    a, n = _state(psi)
    if not inplace:
        a = a.copy()
    elif a is not psi:
        raise ValueError("inplace needs a C-contiguous complex128 array")
    q = _ints(qubits)
    U = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    if U.shape != (1 << q.size, 1 << q.size):
        raise ValueError("matrix shape does not match the number of qubits")
    _load().or_apply_gate(_ptr(a), n, q.size, _ptr(q), _ptr(U))
    return a


def apply_controlled(psi, controls, targets, matrix, inplace=False):
    a, n = _state(psi)
    if not inplace:
        a = a.copy()
    elif a is not psi:
        raise ValueError("inplace needs a C-contiguous complex128 array")
    c = _ints(controls)
    t = _ints(targets)
    U = np.ascontiguousarray(np.asarray(matrix, dtype=np.complex128))
    _load().or_apply_controlled(_ptr(a), n, c.size, _ptr(c), t.size, _ptr(t), _ptr(U))
    return a


def apply_mcx(psi, controls, target, inplace=False):
    a, n = _state(psi)
    if not inplace:
        a = a.copy()
    elif a is not psi:
        raise ValueError("inplace needs a C-contiguous complex128 array")
    c = _ints(controls)
    _load().or_apply_mcx(_ptr(a), n, c.size, _ptr(c), int(target))
    return a


def qft_dft(psi, lo, m, inverse=False):
    a, n = _state(psi)
    a = a.copy()
    _load().or_qft_dft(_ptr(a), n, lo, m, int(bool(inverse)))
    return a


def qft_amplitude(psi, lo, m, index, inverse=False):
    a, n = _state(psi)
    re, im = C.c_double(), C.c_double()
    _load().or_qft_amplitude(_ptr(a), n, lo, m, int(bool(inverse)), int(index),
                             C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def qft_circuit(psi, lo, m, inverse=False):
    a, n = _state(psi)
    a = a.copy()
    _load().or_qft_circuit(_ptr(a), n, lo, m, int(bool(inverse)))
    return a


def add_const(psi, qubits, c):
    a, n = _state(psi)
    a = a.copy()
    q = _ints(qubits)
    _load().or_add_const(_ptr(a), n, q.size, _ptr(q), int(c) & ((1 << 64) - 1))
    return a


def add_const_circuit(psi, qubits, c):
    a, n = _state(psi)
    a = a.copy()
    q = _ints(qubits)
    _load().or_add_const_circuit(_ptr(a), n, q.size, _ptr(q), int(c) & ((1 << 64) - 1))
    return a


def _regs(qa, qb, qc):
    a, b, c = _ints(qa), _ints(qb), _ints(qc)
    if not (a.size == b.size == c.size):
        raise ValueError("registers a, b, c need the same width")
    return a, b, c


def mul(psi, qa, qb, qc):
    """c -> (c + a b) mod 2^N on every basis state (Sec. III-A multiplication)."""
    s, n = _state(psi)
    s = s.copy()
    a, b, c = _regs(qa, qb, qc)
    _load().or_mul(_ptr(s), n, a.size, _ptr(a), _ptr(b), _ptr(c))
    return s


def div(psi, qa, qb, qc):
    """The restoring division (a, b, 0) -> (a mod b, b, a div b) on every
    basis state (Sec. III-A division; see oracle.c for c != 0)."""
    s, n = _state(psi)
    s = s.copy()
    a, b, c = _regs(qa, qb, qc)
    _load().or_div(_ptr(s), n, a.size, _ptr(a), _ptr(b), _ptr(c))
    return s


def mul_circuit(psi, qa, qb, qc):
    """The multiplication as multi-controlled NOTs (repeated add and shift)."""
    s, n = _state(psi)
    s = s.copy()
    a, b, c = _regs(qa, qb, qc)
    _load().or_mul_circuit(_ptr(s), n, a.size, _ptr(a), _ptr(b), _ptr(c))
    return s


def expectation(psi, xmask, zmask, coeff):
    a, n = _state(psi)
    xm = np.ascontiguousarray(np.asarray(xmask, dtype=np.uint64))
    zm = np.ascontiguousarray(np.asarray(zmask, dtype=np.uint64))
    cf = np.ascontiguousarray(np.asarray(coeff, dtype=np.float64))
    return _load().or_expectation(_ptr(a), n, xm.size, _ptr(xm), _ptr(zm), _ptr(cf))


def probs(psi, qubits):
    a, n = _state(psi)
    q = _ints(qubits)
    out = np.empty(1 << q.size, dtype=np.float64)
    _load().or_probs(_ptr(a), n, q.size, _ptr(q), _ptr(out))
    return out


def sample(psi, qubits, uniforms):
    """Inverse-CDF samples of measuring qubits[] (all qubits: range(n)), one
    per uniform in [0, 1) (Sec. II measurement)."""
    a, n = _state(psi)
    q = _ints(qubits)
    u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64))
    out = np.empty(u.size, dtype=np.uint64)
    _load().or_sample(_ptr(a), n, q.size, _ptr(q), u.size, _ptr(u), _ptr(out))
    return out


def collapse(psi, qubits, outcome):
    """(state after the outcome, its probability) (Sec. II collapse)."""
    a, n = _state(psi)
    a = a.copy()
    q = _ints(qubits)
    p = _load().or_collapse(_ptr(a), n, q.size, _ptr(q), int(outcome))
    return a, p


def dense_unitary(n, gates):
    """The 2^n x 2^n matrix of a circuit on n qubits (Sec. III-C): column j is
    the circuit applied, gate by gate, to the basis state |j>."""
    U = np.zeros((1 << n, 1 << n), dtype=np.complex128)
    for j in range(1 << n):
        e = np.zeros(1 << n, dtype=np.complex128)
        e[j] = 1.0
        for g in gates:
            if getattr(g, "controls", ()):
                e = apply_controlled(e, list(g.controls), list(g.qubits), g.matrix)
            else:
                e = apply_gate(e, list(g.qubits), g.matrix)
        U[:, j] = e
    return U


def qpe_circuit(psi_sys, n, b, gates):
    """Coherent phase estimation simulated gate by gate (Sec. III-C): b
    ancillas at qubits [n, n+b) start in |0>, get Hadamards, ancilla j
    controls U^(2^j) (the circuit repeated 2^j times, every gate controlled by
    it), then the inverse QFT on the ancillas.  Returns the (n+b)-qubit
    state; with an eigenvector of eigenvalue exp(2 pi i k / 2^b) the ancilla
    register ends in |k>."""
    psi = np.zeros(1 << (n + b), dtype=np.complex128)
    psi[: 1 << n] = psi_sys
    h = np.array([[1, 1], [1, -1]], dtype=np.complex128) / np.sqrt(2)
    for j in range(b):
        psi = apply_gate(psi, [n + j], h)
    for j in range(b):
        for _ in range(1 << j):
            for g in gates:
                ctl = [n + j] + list(getattr(g, "controls", ()))
                psi = apply_controlled(psi, ctl, list(g.qubits), g.matrix)
    return qft_dft(psi, n, b, inverse=True)


def fidelity(ref, got):
    """|<ref|got>|^2 / (<ref|ref><got|got>) in FP64 (max-abs and fidelity are
    the two error measures every parity test reports)."""
    r = np.asarray(ref, dtype=np.complex128)
    g = np.asarray(got, dtype=np.complex128)
    ov = np.vdot(r, g)
    return float(abs(ov) ** 2 / (np.vdot(r, r).real * np.vdot(g, g).real))


# --- cost-model network -------------------------------------------------
def mlp_param_count(d, h1, h2):
    return _load().or_mlp_param_count(d, h1, h2)


def mlp_forward(params, X, h1, h2):
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    n, d = X.shape
    y = np.empty(n)
    _load().or_mlp_forward(_ptr(p), d, h1, h2, _ptr(X), n, _ptr(y))
    return y


def mlp_grad(params, X, t, h1, h2):
    """(loss, gradient) of the mean squared error by backpropagation."""
    X = np.ascontiguousarray(np.asarray(X, dtype=np.float64))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float64))
    n, d = X.shape
    g = np.empty_like(p)
    loss = _load().or_mlp_grad(_ptr(p), d, h1, h2, _ptr(X), _ptr(t), n, _ptr(g))
    return loss, g
