"""qe_probs_noalloc, the allocation-free probability entry point.

It serves callers that cannot allocate device memory (code running while
another component captures a CUDA graph, processes whose GPU memory belongs to
another allocator, hosts that forbid allocation after start-up).  Its answer
must equal what qe_probs returns, within the probability tolerance of the
other tests (1e-13), for consecutive calls that share its static scratch.
This file sorts last so that, when it fails, every other test has already run.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-13   # same bar as the qe_probs parity tests


def _setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1604_06460_gb300 import build as B
    from paper_1604_06460_gb300 import qe
    B.build()
    return torch, qe, qe.load()


def _noalloc(lib, st, qubits, out):
    q = np.ascontiguousarray(np.asarray(qubits, dtype=np.int32))
    return lib.qe_probs_noalloc(C.c_void_p(st.tensor.data_ptr()), st.n, st._dt, q.size,
                                q.ctypes.data_as(C.c_void_p), C.c_void_p(out.data_ptr()),
                                C.c_void_p(st.stream.cuda_stream))


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_noalloc_probs_equal_qe_probs_on_consecutive_calls(dtype):
    torch, qe, lib = _setup()
    with qe.State(15, dtype) as st:
        st.init_random(2024)
        for qubits in ([0, 6, 14], [3, 11], [2, 9, 4, 0, 13, 7]):   # calls in a row
            ref = st.probs(qubits)
            out = torch.full((1 << len(qubits),), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(lib, st, qubits, out) == 0
            st.stream.synchronize()
            got = out.cpu().numpy()
            assert np.max(np.abs(got - ref)) < TOL


def test_noalloc_rejects_bad_arguments_without_launching():
    torch, qe, lib = _setup()
    with qe.State(6, "c128") as st:
        out = torch.zeros(1 << 17, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, st, [0, 0], out) == -1            # repeated qubit
        assert _noalloc(lib, st, [6], out) == -1               # qubit >= n
        assert _noalloc(lib, st, list(range(7)), out) == -1    # m > n
