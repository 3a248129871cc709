"""Python binding of the C ABI in ``include/qe.h`` (argument marshalling only).

Every operation runs in the CUDA kernels of ``libqe.so``; this module only
converts Python/numpy arguments to the C types, allocates the state's device
memory through PyTorch (so that torch's caching allocator and streams are
used) and turns error codes into exceptions.  There is no CPU fallback: if
the library is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

_LIB_PATH = Path(__file__).resolve().parent / "_build" / "libqe.so"
_lib = None

C64, C128 = 0, 1
POLICY_AUTO, POLICY_ANALYTIC, POLICY_EMULATE, POLICY_SIMULATE = 0, 1, 2, 3
ARITH_FP64, ARITH_DF64 = 0, 1

STATUS = {0: "QE_OK", -1: "QE_ERR_ARG", -2: "QE_ERR_OOM", -3: "QE_ERR_CUDA",
          -4: "QE_ERR_TIMEOUT", -5: "QE_ERR_STATE", -6: "QE_ERR_UNSUPPORTED"}

# name -> (restype, argtypes); exactly the entry points declared in include/qe.h
_vp, _i, _u64, _sz, _dp = C.c_void_p, C.c_int, C.c_uint64, C.c_size_t, C.c_void_p


class Stats(C.Structure):
    _fields_ = [("launches", C.c_uint64), ("passes", C.c_uint64),
                ("algorithmic_bytes", C.c_double), ("gates_applied", C.c_uint64),
                ("fused_blocks", C.c_uint64)]


class KernelProfile(C.Structure):
    _fields_ = [("name", C.c_char * 48), ("launches", C.c_uint64), ("total_ms", C.c_double),
                ("bytes", C.c_double)]


SIGNATURES = {
    "qe_alloc_state": (_i, [_i, _i, _vp, _sz, _vp, C.POINTER(_vp)]),
    "qe_free_state": (_i, [_vp]),
    "qe_state_info": (_i, [_vp, C.POINTER(_i), C.POINTER(_i), C.POINTER(_vp)]),
    "qe_init_basis": (_i, [_vp, _u64]),
    "qe_init_random": (_i, [_vp, _u64]),
    "qe_set_amplitudes": (_i, [_vp, _vp, _u64, _u64]),
    "qe_get_amplitudes": (_i, [_vp, _vp, _u64, _u64]),
    "qe_apply_gate": (_i, [_vp, _i, _vp, _vp]),
    "qe_apply_controlled": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "qe_apply_qft": (_i, [_vp, _i, _i, _i]),
    "qe_apply_add_const": (_i, [_vp, _i, _vp, _u64]),
    "qe_apply_mul": (_i, [_vp, _i, _vp, _vp, _vp]),
    "qe_apply_div": (_i, [_vp, _i, _vp, _vp, _vp]),
    "qe_expectation": (_i, [_vp, _i, _vp, _vp, _vp, _vp]),
    "qe_probs": (_i, [_vp, _i, _vp, _vp]),
    "qe_norm2": (_i, [_vp, _vp]),
    "qe_sample": (_i, [_vp, _i, _vp, _i, _vp, _vp]),
    "qe_init_identity": (_i, [_vp, _i]),
    "qe_matmul": (_i, [_vp, _vp, _vp]),
    "qe_qpe_emulate": (_i, [_vp, _i, _i, _vp]),
    "qe_collapse": (_i, [_vp, _i, _vp, _u64, _vp]),
    "qe_flush": (_i, [_vp]),
    "qe_sync": (_i, [_vp]),
    "qe_set_policy": (_i, [_vp, _i, _i]),
    "qe_set_arith": (_i, [_vp, _i]),
    "qe_get_arith": (_i, [_vp, C.POINTER(_i)]),
    "qe_get_stats": (_i, [_vp, C.POINTER(Stats)]),
    "qe_reset_stats": (_i, [_vp]),
    "qe_profile_enable": (_i, [_vp, _i]),
    "qe_profile_read": (_i, [_vp, C.POINTER(KernelProfile), _i, C.POINTER(_i)]),
    "qe_probs_noalloc": (_i, [_vp, _i, _i, _i, _vp, _vp, _vp]),
    "qe_batch_create": (_i, [_i, _vp, _i, _vp, C.c_double, _i, _vp, C.POINTER(_vp)]),
    "qe_batch_run": (_i, [_vp, _vp]),
    "qe_batch_tune": (_i, [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)]),
    "qe_batch_set_plan": (_i, [_vp, _i, _i, _i]),
    "qe_batch_set_arith": (_i, [_vp, _i]),
    "qe_batch_info": (_i, [_vp, C.POINTER(C.c_double), C.POINTER(_i)]),
    "qe_batch_free": (_i, [_vp]),
    "qe_cost_model_create": (_i, [_i, _i, _u64, C.POINTER(_vp)]),
    "qe_cost_model_param_count": (_i, [_vp, C.POINTER(_i)]),
    "qe_cost_model_get_params": (_i, [_vp, _vp, _i]),
    "qe_cost_model_set_params": (_i, [_vp, _vp, _i]),
    "qe_cost_model_gradient": (_i, [_vp, _vp, _vp, _i, _vp, C.POINTER(C.c_float)]),
    "qe_cost_model_train": (_i, [_vp, _vp, _vp, _i, _i, C.c_float, C.POINTER(C.c_float)]),
    "qe_cost_model_predict": (_i, [_vp, _vp, _i, _vp]),
    "qe_cost_model_free": (_i, [_vp]),
    "qe_cost_features": (_i, [_i, _i, _i, _i, _i, _i, _i, _u64, _vp]),
    "qe_set_cost_model": (_i, [_vp, _vp]),
    "qe_planned_fusion_width": (_i, [_vp, C.POINTER(_i)]),
    "qe_plan_fusion": (_i, [_i, _i, _vp, _vp, _vp, _vp, _i, _i, C.POINTER(_i), _vp, _vp, _vp]),
    "qe_last_error": (C.c_char_p, []),
}


class QEError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def library_path() -> Path:
    return _LIB_PATH


def load(path: str | Path | None = None):
    """Load libqe.so (built by ``paper_1604_06460_gb300.build``); raises if absent."""
    global _lib
    if _lib is None or path is not None:
        p = Path(path) if path else _LIB_PATH
        if not p.exists():
            raise RuntimeError(f"CUDA library {p} is missing: run the package build first")
        lib = C.CDLL(str(p))
        for name, (res, args) in SIGNATURES.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _check(status):
    if status != 0:
        raise QEError(status, load().qe_last_error().decode())


def _i32(xs):
    return np.ascontiguousarray(np.asarray(xs, dtype=np.int32).reshape(-1))


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def _mat(U, k):
    M = np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    if M.shape != (1 << k, 1 << k):
        raise ValueError(f"matrix must be {1 << k}x{1 << k}")
    return M


class State:
    """One state vector of 2**n amplitudes on the current CUDA device.

    ``dtype`` is ``"c128"`` or ``"c64"``.  Memory comes from a torch tensor
    (kept alive by this object); work is enqueued on ``stream`` (a
    ``torch.cuda.Stream``; default: torch's current stream).
    """

    def __init__(self, n: int, dtype: str = "c128", stream=None, tensor=None):
        import torch

        lib = load()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the emulator has no CPU fallback")
        self.n = int(n)
        self.dtype = dtype
        self._dt = C128 if dtype == "c128" else C64
        if dtype not in ("c128", "c64"):
            raise ValueError("dtype must be 'c128' or 'c64'")
        real = torch.float64 if self._dt == C128 else torch.float32
        if tensor is None:
            tensor = torch.empty(2 << self.n, dtype=real, device="cuda")
        self.tensor = tensor
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.qe_alloc_state(self.n, self._dt, C.c_void_p(tensor.data_ptr()),
                                  tensor.numel() * tensor.element_size(),
                                  C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    # -- lifetime --------------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            _check(load().qe_free_state(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- initialisation and data movement -------------------------------------
    def init_basis(self, index=0):
        _check(load().qe_init_basis(self._h, int(index)))

    def init_random(self, seed):
        _check(load().qe_init_random(self._h, int(seed)))

    def set(self, psi, offset=0):
        a = np.ascontiguousarray(psi, dtype=np.complex128 if self._dt == C128 else np.complex64)
        _check(load().qe_set_amplitudes(self._h, _ptr(a), int(offset), a.size))

    def get(self, offset=0, count=None, out=None):
        """Copy amplitudes to host memory (into ``out`` when given, e.g. a view
        of pinned memory)."""
        count = (1 << self.n) - offset if count is None else count
        dt = np.complex128 if self._dt == C128 else np.complex64
        a = np.empty(count, dtype=dt) if out is None else out
        if a.dtype != dt or a.size != count or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("out has the wrong dtype, size or layout")
        _check(load().qe_get_amplitudes(self._h, _ptr(a), int(offset), int(count)))
        return a

    # -- operations ---------------------------------------------------------
    def apply_gate(self, qubits, U):
        q = _i32(qubits)
        M = _mat(U, q.size)
        _check(load().qe_apply_gate(self._h, q.size, _ptr(q), _ptr(M)))

    def apply_controlled(self, controls, targets, U):
        c, t = _i32(controls), _i32(targets)
        M = _mat(U, t.size)
        _check(load().qe_apply_controlled(self._h, c.size, _ptr(c), t.size, _ptr(t), _ptr(M)))

    def apply(self, gate):
        """Apply an ``inputs.Gate`` (dense, or controlled when it has controls)."""
        if gate.controls:
            self.apply_controlled(gate.controls, gate.qubits, gate.matrix)
        else:
            self.apply_gate(gate.qubits, gate.matrix)

    def apply_qft(self, lo, m, inverse=False):
        _check(load().qe_apply_qft(self._h, int(lo), int(m), int(bool(inverse))))

    def add_const(self, qubits, c):
        q = _i32(qubits)
        _check(load().qe_apply_add_const(self._h, q.size, _ptr(q), int(c) & ((1 << 64) - 1)))

    def _regs(self, qa, qb, qc):
        a, b, c = _i32(qa), _i32(qb), _i32(qc)
        if not (a.size == b.size == c.size):
            raise ValueError("registers a, b, c need the same width")
        return a, b, c

    def mul(self, qa, qb, qc):
        """c -> (c + a b) mod 2^N (qe_apply_mul)."""
        a, b, c = self._regs(qa, qb, qc)
        _check(load().qe_apply_mul(self._h, a.size, _ptr(a), _ptr(b), _ptr(c)))

    def div(self, qa, qb, qc):
        """The restoring division (a, b, 0) -> (a mod b, b, a div b) (qe_apply_div)."""
        a, b, c = self._regs(qa, qb, qc)
        _check(load().qe_apply_div(self._h, a.size, _ptr(a), _ptr(b), _ptr(c)))

    def expectation(self, xmask, zmask, coeff):
        xm = np.ascontiguousarray(np.asarray(xmask, dtype=np.uint64))
        zm = np.ascontiguousarray(np.asarray(zmask, dtype=np.uint64))
        cf = np.ascontiguousarray(np.asarray(coeff, dtype=np.float64))
        out = C.c_double()
        _check(load().qe_expectation(self._h, xm.size, _ptr(xm), _ptr(zm), _ptr(cf), C.byref(out)))
        return out.value

    def probs(self, qubits):
        q = _i32(qubits)
        out = np.empty(1 << q.size, dtype=np.float64)
        _check(load().qe_probs(self._h, q.size, _ptr(q), _ptr(out)))
        return out

    def sample(self, uniforms, qubits=None):
        """Outcomes for the given uniforms in [0, 1): basis indices (qubits
        None: all qubits) or the measured qubits' values (qe_sample)."""
        u = np.ascontiguousarray(np.asarray(uniforms, dtype=np.float64).reshape(-1))
        out = np.empty(u.size, dtype=np.uint64)
        if qubits is None:
            _check(load().qe_sample(self._h, 0, None, u.size, _ptr(u), _ptr(out)))
        else:
            q = _i32(qubits)
            _check(load().qe_sample(self._h, q.size, _ptr(q), u.size, _ptr(u), _ptr(out)))
        return out

    def init_identity(self, nsys):
        """The identity matrix of 2^nsys x 2^nsys, column-major (qe_init_identity)."""
        _check(load().qe_init_identity(self._h, int(nsys)))

    def matmul(self, a, b):
        """self = a b for matrix states (qe_matmul)."""
        _check(load().qe_matmul(self._h, a._h, b._h))

    def qpe_emulate(self, nsys, b, u):
        """Phase estimation with b ancillas above the nsys system qubits, U
        held in the matrix state u (qe_qpe_emulate)."""
        _check(load().qe_qpe_emulate(self._h, int(nsys), int(b), u._h))

    def collapse(self, qubits, outcome):
        """Collapse onto the outcome of measuring qubits; returns its probability."""
        q = _i32(qubits)
        p = C.c_double()
        _check(load().qe_collapse(self._h, q.size, _ptr(q), int(outcome) & ((1 << 64) - 1), C.byref(p)))
        return p.value

    def norm2(self):
        out = C.c_double()
        _check(load().qe_norm2(self._h, C.byref(out)))
        return out.value

    def flush(self):
        _check(load().qe_flush(self._h))

    def sync(self):
        _check(load().qe_sync(self._h))

    def set_policy(self, policy=POLICY_AUTO, max_k=None):
        """max_k None (0): the library's default fusion width."""
        _check(load().qe_set_policy(self._h, int(policy), int(max_k or 0)))

    def set_arith(self, arith):
        """ARITH_FP64 (default for complex128) or ARITH_DF64 (the fast
        double-float mode); see qe_set_arith."""
        _check(load().qe_set_arith(self._h, int(arith)))

    def arith(self):
        a = C.c_int()
        _check(load().qe_get_arith(self._h, C.byref(a)))
        return a.value

    def set_cost_model(self, model):
        """Attach a CostModel (or None): QE_POLICY_AUTO then lets it choose."""
        _check(load().qe_set_cost_model(self._h, model._h if model is not None else None))
        self._model = model

    def planned_fusion_width(self):
        k = C.c_int()
        _check(load().qe_planned_fusion_width(self._h, C.byref(k)))
        return k.value

    def stats(self):
        st = Stats()
        _check(load().qe_get_stats(self._h, C.byref(st)))
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def reset_stats(self):
        _check(load().qe_reset_stats(self._h))

    def profile(self, enable=True):
        _check(load().qe_profile_enable(self._h, int(bool(enable))))

    def profile_read(self):
        """{kernel name: (launches, total_ms, algorithmic bytes)}; synchronises."""
        buf = (KernelProfile * 64)()
        cnt = C.c_int()
        _check(load().qe_profile_read(self._h, buf, 64, C.byref(cnt)))
        return {buf[i].name.decode(): (buf[i].launches, buf[i].total_ms, buf[i].bytes)
                for i in range(min(cnt.value, 64))}


class Batch:
    """Many hardware-efficient-ansatz circuits run by one persistent kernel
    replayed as a CUDA graph; ``run()`` returns each circuit's TFIM energy.

    ``nqubits``: qubit count per circuit; ``angles``: per circuit an array of
    shape (layers, n, 2) holding (theta_RY, phi_RZ); ``hx``: transverse field.
    """

    def __init__(self, nqubits, angles, hx=0.7, dtype="c128", stream=None):
        import torch

        lib = load()
        nq = np.ascontiguousarray(np.asarray(nqubits, dtype=np.int32))
        layers = {int(np.asarray(a).shape[0]) for a in angles}
        if len(layers) != 1:
            raise ValueError("all circuits need the same number of layers")
        self.layers = layers.pop()
        flat = np.ascontiguousarray(np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1)
                                                    for a in angles]))
        self.count = nq.size
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = C.c_void_p()
        _check(lib.qe_batch_create(nq.size, _ptr(nq), self.layers, _ptr(flat), float(hx),
                                   C128 if dtype == "c128" else C64,
                                   C.c_void_p(self.stream.cuda_stream), C.byref(h)))
        self._h = h

    def run(self):
        out = np.empty(self.count, dtype=np.float64)
        _check(load().qe_batch_run(self._h, _ptr(out)))
        return out

    def tune(self, reps=2):
        t, p, th = C.c_int(), C.c_int(), C.c_int()
        _check(load().qe_batch_tune(self._h, int(reps), C.byref(t), C.byref(p), C.byref(th)))
        return {"tile_bits": t.value, "tiles_per_item": p.value, "threads": th.value}

    def set_plan(self, tile_bits, tiles_per_item, threads):
        _check(load().qe_batch_set_plan(self._h, int(tile_bits), int(tiles_per_item), int(threads)))

    def set_arith(self, arith):
        """ARITH_DF64 (default) or ARITH_FP64 for complex128 batches."""
        _check(load().qe_batch_set_arith(self._h, int(arith)))

    def info(self):
        b, i = C.c_double(), C.c_int()
        _check(load().qe_batch_info(self._h, C.byref(b), C.byref(i)))
        return {"hbm_bytes": b.value, "items": i.value}

    def close(self):
        if getattr(self, "_h", None):
            _check(load().qe_batch_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


OP_GATE, OP_QFT_EMULATE, OP_QFT_SIMULATE, OP_ADD_EMULATE, OP_ADD_SIMULATE = range(5)
N_FEATURES = 16


def cost_features(op, n, dtype, k=0, lo=0, hi=0, m=0, c=0):
    f = np.empty(N_FEATURES, dtype=np.float32)
    _check(load().qe_cost_features(int(op), int(n), C128 if dtype == "c128" else C64, int(k),
                                   int(lo), int(hi), int(m), int(c) & ((1 << 64) - 1), _ptr(f)))
    return f


def plan_fusion(n, gates, max_k):
    """Host-only: the fused blocks (qubits, matrix) the flush would apply for
    `gates` (objects with .qubits and .matrix, uncontrolled), in order."""
    k = np.array([len(g.qubits) for g in gates], dtype=np.int32)
    qb = np.full((max(len(gates), 1), 5), -1, dtype=np.int32)
    mats, offs, off = [], [], 0
    for i, g in enumerate(gates):
        qb[i, :len(g.qubits)] = g.qubits
        m = np.ascontiguousarray(np.asarray(g.matrix, dtype=np.complex128)).view(np.float64).ravel()
        mats.append(m)
        offs.append(off)
        off += m.size
    mat = np.concatenate(mats) if mats else np.zeros(1)
    offs = np.array(offs or [0], dtype=np.int64)
    cap = max(len(gates), 1)
    nb = C.c_int(0)
    bk = np.zeros(cap, dtype=np.int32)
    bq = np.zeros((cap, 5), dtype=np.int32)
    bm = np.zeros((cap, 2048), dtype=np.float64)
    p = lambda a: a.ctypes.data_as(C.c_void_p)
    _check(load().qe_plan_fusion(n, len(gates), p(k), p(qb), p(mat), p(offs), max_k, cap, C.byref(nb),
                                 p(bk), p(bq), p(bm)))
    out = []
    for b in range(nb.value):
        kb = int(bk[b])
        D = 1 << kb
        U = bm[b, :2 * D * D].view(np.complex128).reshape(D, D).copy()
        out.append((list(bq[b, :kb]), U))
    return out


class CostModel:
    """The learned cost model (log-milliseconds from 16 features), trained and
    evaluated by the library's own GPU kernels."""

    def __init__(self, hidden1=32, hidden2=32, seed=0):
        h = C.c_void_p()
        _check(load().qe_cost_model_create(int(hidden1), int(hidden2), int(seed), C.byref(h)))
        self._h = h
        self.hidden = (hidden1, hidden2)

    def param_count(self):
        c = C.c_int()
        _check(load().qe_cost_model_param_count(self._h, C.byref(c)))
        return c.value

    def params(self):
        p = np.empty(self.param_count(), dtype=np.float32)
        _check(load().qe_cost_model_get_params(self._h, _ptr(p), p.size))
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        _check(load().qe_cost_model_set_params(self._h, _ptr(p), p.size))

    def gradient(self, X, t):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
        g = np.empty(self.param_count(), dtype=np.float32)
        loss = C.c_float()
        _check(load().qe_cost_model_gradient(self._h, _ptr(X), _ptr(t), t.size, _ptr(g), C.byref(loss)))
        return loss.value, g

    def train(self, X, t, epochs=2000, lr=3e-3):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        t = np.ascontiguousarray(np.asarray(t, dtype=np.float32))
        loss = C.c_float()
        _check(load().qe_cost_model_train(self._h, _ptr(X), _ptr(t), t.size, int(epochs), float(lr),
                                          C.byref(loss)))
        return loss.value

    def predict(self, X):
        X = np.ascontiguousarray(np.asarray(X, dtype=np.float32))
        y = np.empty(X.shape[0], dtype=np.float32)
        _check(load().qe_cost_model_predict(self._h, _ptr(X), X.shape[0], _ptr(y)))
        return y

    def close(self):
        if getattr(self, "_h", None):
            _check(load().qe_cost_model_free(self._h))
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
