"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only DRAWS inputs: gate matrices of Table I, Haar-random U(2)
gates, random circuits, the hardware-efficient ansatz, the transverse-field
Ising Hamiltonian as Pauli masks and small random states.  It performs none of
the state-vector arithmetic, imports nothing from the rest of the package and
nothing from the oracle, so both sides receive the very same inputs.

Conventions: a gate is ``Gate(qubits, matrix, controls)``; ``matrix`` is
2^k x 2^k complex128 with row/column bit j <-> ``qubits[j]`` and acts only
where every qubit in ``controls`` is 1.  Qubit q is bit q of the state index.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SQ2 = 1.0 / np.sqrt(2.0)


@dataclass(frozen=True)
class Gate:
    qubits: tuple
    matrix: np.ndarray
    controls: tuple = field(default=())
    name: str = ""


# --- Table I of the paper (little-endian: first listed qubit = bit 0) -------
def mat_x():
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def mat_y():
    return np.array([[0, -1j], [1j, 0]], dtype=np.complex128)


def mat_z():
    return np.array([[1, 0], [0, -1]], dtype=np.complex128)


def mat_h():
    return SQ2 * np.array([[1, 1], [1, -1]], dtype=np.complex128)


def mat_s():
    return np.array([[1, 0], [0, 1j]], dtype=np.complex128)


def mat_t():
    return np.array([[1, 0], [0, np.exp(1j * np.pi / 4)]], dtype=np.complex128)


def mat_rz(theta):
    return np.array([[np.exp(-0.5j * theta), 0], [0, np.exp(0.5j * theta)]],
                    dtype=np.complex128)


def mat_ry(theta):
    c, s = np.cos(0.5 * theta), np.sin(0.5 * theta)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def mat_cnot():
    """CNOT on qubits (target, control): flips bit 0 where bit 1 is set."""
    return np.array([[1, 0, 0, 0], [0, 1, 0, 0], [0, 0, 0, 1], [0, 0, 1, 0]],
                    dtype=np.complex128)


def mat_cr(theta):
    return np.diag([1, 1, 1, np.exp(1j * theta)]).astype(np.complex128)


def cnot(control, target):
    return Gate((target, control), mat_cnot(), (), "cnot")


def cz(a, b):
    return Gate((a, b), mat_cr(np.pi), (), "cz")


def cr(control, target, theta):
    return Gate((target, control), mat_cr(theta), (), "cr")


def single(q, m, name=""):
    return Gate((q,), np.asarray(m, dtype=np.complex128), (), name)


def mcx(controls, target):
    return Gate((target,), mat_x(), tuple(controls), "mcx")


# --- Haar-random U(2) ------------------------------------------------------
def haar_u2(rng):
    """QR of a complex Ginibre matrix with the phases of R's diagonal moved
    into Q (Mezzadri, Notices AMS 2007), which makes Q Haar-distributed."""
    z = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) * SQ2
    q, r = np.linalg.qr(z)
    d = np.diag(r)
    return (q * (d / np.abs(d))[None, :]).astype(np.complex128)


def random_circuit(n, depth, seed):
    """``depth`` layers; each is a Haar U(2) on every qubit 0..n-1, then CNOTs
    on floor(n/2) disjoint pairs from a seeded shuffle (control = first)."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(depth):
        for q in range(n):
            gates.append(single(q, haar_u2(rng), "u2"))
        perm = rng.permutation(n)
        for j in range(n // 2):
            gates.append(cnot(int(perm[2 * j]), int(perm[2 * j + 1])))
    return gates


def ghz_circuit(n):
    """Sec. IV-E entangling operation: H on the first qubit, then CNOTs from
    it to every other qubit."""
    return [single(0, mat_h(), "h")] + [cnot(0, t) for t in range(1, n)]


def ansatz_circuit(n, layers, seed):
    """Hardware-efficient ansatz: ``layers`` times (RY then RZ on every qubit,
    angles uniform in [0, 2 pi), then a CZ ladder (q, q+1))."""
    rng = np.random.default_rng(seed)
    gates = []
    for _ in range(layers):
        for q in range(n):
            gates.append(single(q, mat_ry(rng.uniform(0, 2 * np.pi)), "ry"))
            gates.append(single(q, mat_rz(rng.uniform(0, 2 * np.pi)), "rz"))
        for q in range(n - 1):
            gates.append(cz(q, q + 1))
    return gates


def ansatz_angles(n, layers, seed):
    """The angles ansatz_circuit draws, as an array (layers, n, 2)."""
    rng = np.random.default_rng(seed)
    out = np.empty((layers, n, 2))
    for l in range(layers):
        for q in range(n):
            out[l, q, 0] = rng.uniform(0, 2 * np.pi)
            out[l, q, 1] = rng.uniform(0, 2 * np.pi)
    return out


def batch_sizes(count, lo, hi, seed):
    """Qubit counts drawn uniformly from [lo, hi]."""
    return np.random.default_rng(seed).integers(lo, hi + 1, size=count)


def tfim_terms(n, h=0.7):
    """sum_{i=0}^{n-2} Z_i Z_{i+1} + h sum_{i=0}^{n-1} X_i (open chain) as
    Pauli masks: (xmask, zmask, coeff); (x,z) bits (1,0)=X, (0,1)=Z, (1,1)=Y."""
    xm, zm, cf = [], [], []
    for i in range(n - 1):
        xm.append(0)
        zm.append((1 << i) | (1 << (i + 1)))
        cf.append(1.0)
    for i in range(n):
        xm.append(1 << i)
        zm.append(0)
        cf.append(h)
    return (np.array(xm, dtype=np.uint64), np.array(zm, dtype=np.uint64),
            np.array(cf, dtype=np.float64))


def random_state(n, seed):
    """Small normalised complex Gaussian state drawn on the host (numpy PCG64)."""
    rng = np.random.default_rng(seed)
    a = rng.standard_normal(1 << n) + 1j * rng.standard_normal(1 << n)
    return (a / np.linalg.norm(a)).astype(np.complex128)


def random_constant(m, seed):
    return int(np.random.default_rng(seed).integers(0, 1 << m))


def tfim_trotter_step(n, dt=0.1, J=1.0, h=0.7):
    """One Trotter step of the 1-D transverse-field Ising time evolution as
    G = 4n - 3 gates: for every bond (i, i+1) a CNOT, RZ(2 J dt) on i+1 and
    the CNOT again, then RX(2 h dt) on every qubit (the operator of the
    phase-estimation timings, with G = 29 .. 53 for n = 8 .. 14)."""
    gates = []
    for i in range(n - 1):
        gates += [cnot(i, i + 1), single(i + 1, mat_rz(2 * J * dt), "rz"), cnot(i, i + 1)]
    c, sn = np.cos(h * dt), np.sin(h * dt)
    rx = np.array([[c, -1j * sn], [-1j * sn, c]])
    gates += [single(q, rx, "rx") for q in range(n)]
    return gates
