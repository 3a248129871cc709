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


@pytest.mark.parametrize("dtype", ["c128", "c64"])
@pytest.mark.parametrize("qubits", [[0], [21, 3], list(range(16))])
def test_noalloc_many_chunks_per_bin_and_all_bins(dtype, qubits):
    # n = 22: one or two measured qubits spread each bin over many blocks
    # (several partials per bin, summed in order by the second kernel); 16
    # qubits fill 65536 bins
    torch, qe, lib = _setup()
    with qe.State(22, dtype) as st:
        st.init_random(77)
        ref = st.probs(qubits)
        for _ in range(2):
            out = torch.full((1 << len(qubits),), -1.0, dtype=torch.float64, device="cuda")
            assert _noalloc(lib, st, qubits, out) == 0
            st.stream.synchronize()
            assert np.max(np.abs(out.cpu().numpy() - ref)) < TOL


def test_noalloc_rejects_bad_arguments_and_leaves_out_untouched():
    torch, qe, lib = _setup()
    with qe.State(17, "c128") as st:
        out = torch.full((1 << 17,), -2.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, st, [0, 0], out) == -1            # repeated qubit
        assert _noalloc(lib, st, [17], out) == -1              # qubit >= n
        assert _noalloc(lib, st, list(range(17)), out) == -1   # m > 16
        q = np.array([0, 1], dtype=np.int32)
        qp = q.ctypes.data_as(C.c_void_p)
        dp, sp = C.c_void_p(st.tensor.data_ptr()), C.c_void_p(st.stream.cuda_stream)
        assert lib.qe_probs_noalloc(dp, st.n, 99, 2, qp, C.c_void_p(out.data_ptr()), sp) == -1      # dtype
        assert lib.qe_probs_noalloc(None, st.n, st._dt, 2, qp, C.c_void_p(out.data_ptr()), sp) == -1  # state
        assert lib.qe_probs_noalloc(dp, st.n, st._dt, 2, qp, None, sp) == -1                         # out
        assert lib.qe_probs_noalloc(dp, st.n, st._dt, 2, None, C.c_void_p(out.data_ptr()), sp) == -1  # qubits
        assert lib.qe_probs_noalloc(dp, 35, st._dt, 2, qp, C.c_void_p(out.data_ptr()), sp) == -1      # n
        st.stream.synchronize()
        assert bool(torch.all(out == -2.0))
    with qe.State(6, "c128") as st:
        out = torch.full((1 << 7,), -2.0, dtype=torch.float64, device="cuda")
        assert _noalloc(lib, st, list(range(7)), out) == -1    # m > n
        st.stream.synchronize()
        assert bool(torch.all(out == -2.0))
