"""CPU oracle for the Pauli-frame sampler -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import, call or link anything under ``oracle/``. The product path
(``paper_2504_05611_gb300``) never does, and the oracle imports nothing from
it except the op-list generator ``paper_2504_05611_gb300.circuits`` (an input
generator with no sampling arithmetic).

Contents:
  * ``frame_oracle.c`` (via this module): one-shot-at-a-time Pauli-frame
    sampler implementing the sampling specification (Philox4x32-10 noise
    streams, geometric gaps from the gap table T), the gap table, Philox
    itself, and a 64-lane noiseless propagator for fault injection and
    gauge-randomised determinism audits.
  * ``statevector``: brute-force state-vector simulator for tiny circuits.
  * ``tableau``: CHP stabilizer tableau (Aaronson & Gottesman 2004) for the
    noiseless reference measurement record.
  * ``dem``: exhaustive single-fault detector-error-model enumeration, exact
    detector/observable flip marginals, brute-force circuit distance.

Parity: every function is pinned by ``tests/test_oracle_*.py`` against
values fixed by the paper or by mathematics (see each test's docstring).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence, Tuple

import numpy as np

from . import build as _build

# The oracle's own opcode numbering (by op name).
_CODES = {
    "R": 0, "RX": 1, "H": 2, "S": 3, "CX": 4, "M": 5, "MX": 6,
    "X_ERROR": 7, "Z_ERROR": 8, "DEPOLARIZE1": 9, "DEPOLARIZE2": 10,
    "XFEED": 11, "ZFEED": 12, "DETECTOR": 13, "OBSERVABLE": 14, "TICK": 15,
    "PAULI_CHANNEL_1": 16,
}

_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        U64 = ctypes.c_uint64
        L.oracle_philox4x32_10.argtypes = [P, P, P]
        L.oracle_philox4x32_10.restype = None
        L.oracle_gap_table.argtypes = [ctypes.c_double, P]
        L.oracle_gap_table.restype = None
        L.oracle_pauli_channel.argtypes = [ctypes.c_double] * 3 + [P, P, P]
        L.oracle_pauli_channel.restype = ctypes.c_int
        L.oracle_sample.argtypes = [I64, P, P, P, P, P, P, I64, I64, I64, I64, U64, U64, U64, P, P, ctypes.c_int]
        L.oracle_sample.restype = ctypes.c_int
        L.oracle_sample_measurements.argtypes = [I64, P, P, P, P, P, P, I64, I64, I64, I64, P, U64, U64, U64, P,
                                                 ctypes.c_int]
        L.oracle_sample_measurements.restype = ctypes.c_int
        L.oracle_propagate64.argtypes = [I64, P, P, P, P, P, P, I64, I64, I64, I64, I64, P, P, P, P, U64, P, P]
        L.oracle_propagate64.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class Marshalled:
    """Flat arrays of an op list in the oracle's own encoding."""

    def __init__(self, circuit):
        ops = circuit.ops
        self.n_ops = len(ops)
        self.codes = np.array([_CODES[o.name] for o in ops], dtype=np.int32)
        self.ps = np.array([o.p for o in ops], dtype=np.float64)
        self.args = np.array([o.arg for o in ops], dtype=np.uint32)
        self.args2 = np.zeros(self.n_ops, dtype=np.uint32)
        # PAULI_CHANNEL_1: the oracle derives the event probability and the
        # X/Y/Z thresholds from (px, py, pz) itself; the generator's copies
        # (op.p, op.arg, op.arg2) are not read
        for i, o in enumerate(ops):
            if o.name == "PAULI_CHANNEL_1":
                self.ps[i], self.args[i], self.args2[i] = pauli_channel(*o.channel)
        lens = np.array([o.targets.size for o in ops], dtype=np.int64)
        self.toff = np.zeros(self.n_ops + 1, dtype=np.int64)
        np.cumsum(lens, out=self.toff[1:])
        self.targets = (np.concatenate([o.targets for o in ops]).astype(np.uint32)
                        if self.n_ops else np.zeros(1, np.uint32))
        if self.targets.size == 0:
            self.targets = np.zeros(1, np.uint32)
        self.n_qubits = circuit.n_qubits
        self.n_meas = circuit.n_meas
        self.n_det = circuit.n_det
        self.n_obs = circuit.n_obs

    def head(self):
        return (self.n_ops, _ptr(self.codes), _ptr(self.ps), _ptr(self.args), _ptr(self.args2), _ptr(self.toff),
                _ptr(self.targets), self.n_qubits, self.n_meas, self.n_det, self.n_obs)


def philox4x32_10(ctr: Sequence[int], key: Sequence[int]) -> Tuple[int, int, int, int]:
    c = np.array(ctr, dtype=np.uint32)
    k = np.array(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return tuple(int(v) for v in out)


def pauli_channel(px: float, py: float, pz: float) -> Tuple[float, int, int]:
    """PAULI_CHANNEL_1(px, py, pz) as (p, t1, t2): event probability and the
    Pauli-word thresholds of X and Y (``oracle_pauli_channel``)."""
    p = np.zeros(1, dtype=np.float64)
    t = np.zeros(2, dtype=np.uint32)
    rc = lib().oracle_pauli_channel(float(px), float(py), float(pz), _ptr(p), _ptr(t), _ptr(t[1:]))
    if rc != 0:
        raise ValueError(f"PAULI_CHANNEL_1({px}, {py}, {pz}): invalid probabilities")
    return float(p[0]), int(t[0]), int(t[1])


def gap_table(p: float) -> np.ndarray:
    """T[1..4096] = floor(2^32 (1-p)^g) for noise probability p in (0, 1]."""
    t = np.zeros(4096, dtype=np.uint32)
    lib().oracle_gap_table(float(p), _ptr(t))
    return t


def sample(circuit, shots: int, seed: int, first_chunk: int = 0, threads: int = 1,
           marshalled: Optional[Marshalled] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Detector and observable flips, detector-major bit-packed:
    det[n_det][ceil(shots/64)], obs[n_obs][ceil(shots/64)] uint64; bit l of
    column c is shot 64c + l; pad bits are zero."""
    m = marshalled or Marshalled(circuit)
    cols = (shots + 63) // 64
    det = np.zeros((max(m.n_det, 1), max(cols, 1)), dtype=np.uint64)
    obs = np.zeros((max(m.n_obs, 1), max(cols, 1)), dtype=np.uint64)
    rc = lib().oracle_sample(*m.head(), seed & 0xFFFFFFFFFFFFFFFF, first_chunk, shots,
                             _ptr(det), _ptr(obs), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_sample failed with {rc}")
    return det[:m.n_det, :cols], obs[:m.n_obs, :cols]


def sample_measurements(circuit, shots: int, seed: int, first_chunk: int = 0, threads: int = 1,
                        reference: Optional[np.ndarray] = None) -> np.ndarray:
    """Raw measurement records, [n_meas][ceil(shots/64)] uint64 (bit l of
    column c = shot 64c + l): reference XOR flip with gauge-randomised
    frames, so random outcomes are fair coins. The reference record comes
    from the oracle tableau unless given."""
    m = Marshalled(circuit)
    if reference is None:
        from .tableau import reference_sample
        reference = reference_sample(circuit)["rec"]
    ref = np.ascontiguousarray(np.asarray(reference, dtype=np.uint8))
    if ref.size == 0:
        ref = np.zeros(1, np.uint8)
    cols = (shots + 63) // 64
    meas = np.zeros((max(m.n_meas, 1), max(cols, 1)), dtype=np.uint64)
    rc = lib().oracle_sample_measurements(*m.head(), _ptr(ref), seed & 0xFFFFFFFFFFFFFFFF, first_chunk, shots,
                                          _ptr(meas), int(threads))
    if rc != 0:
        raise ValueError(f"oracle_sample_measurements failed with {rc}")
    return meas[:m.n_meas, :cols]


def propagate64(circuit, inj_op, inj_target, inj_pauli, inj_lane, gauge_seed: int = 0,
                marshalled: Optional[Marshalled] = None) -> Tuple[np.ndarray, np.ndarray]:
    """Noiseless 64-lane propagation with injected Paulis (applied right after
    op ``inj_op``); returns per-detector and per-observable 64-bit lane words."""
    m = marshalled or Marshalled(circuit)
    order = np.argsort(np.asarray(inj_op, dtype=np.int64), kind="stable")
    io = np.ascontiguousarray(np.asarray(inj_op, dtype=np.int64)[order])
    it = np.ascontiguousarray(np.asarray(inj_target, dtype=np.uint32)[order])
    ip = np.ascontiguousarray(np.asarray(inj_pauli, dtype=np.uint32)[order])
    il = np.ascontiguousarray(np.asarray(inj_lane, dtype=np.uint32)[order])
    if io.size == 0:
        io, it, ip, il = (np.zeros(1, np.int64), np.zeros(1, np.uint32),
                          np.zeros(1, np.uint32), np.zeros(1, np.uint32))
        n_inj = 0
    else:
        n_inj = io.size
    det = np.zeros(max(m.n_det, 1), dtype=np.uint64)
    obs = np.zeros(max(m.n_obs, 1), dtype=np.uint64)
    rc = lib().oracle_propagate64(*m.head(), n_inj, _ptr(io), _ptr(it), _ptr(ip), _ptr(il),
                                  gauge_seed, _ptr(det), _ptr(obs))
    if rc != 0:
        raise ValueError(f"oracle_propagate64 failed with {rc}")
    return det[:m.n_det], obs[:m.n_obs]


def gauge_audit(circuit, seed: int = 12345, rounds: int = 2) -> Tuple[np.ndarray, np.ndarray]:
    """Indices of detectors and observables that are NOT deterministic in the
    noiseless circuit: under random gauge Paulis after every reset and
    measurement, a deterministic parity stays 0 in all 64*rounds lanes."""
    m = Marshalled(circuit)
    bad_d = np.zeros(m.n_det, dtype=bool)
    bad_o = np.zeros(m.n_obs, dtype=bool)
    for r in range(rounds):
        d, o = propagate64(circuit, [], [], [], [], gauge_seed=seed + 7919 * r + 1, marshalled=m)
        bad_d |= d != 0
        bad_o |= o != 0
    return np.nonzero(bad_d)[0], np.nonzero(bad_o)[0]


def unpack_bits(words: np.ndarray, shots: int) -> np.ndarray:
    """[rows][cols] uint64 -> [rows][shots] uint8 (shot-major per row)."""
    w = np.ascontiguousarray(words, dtype=np.uint64)
    b = np.unpackbits(w.view(np.uint8).reshape(w.shape[0], -1), axis=1, bitorder="little")
    return b[:, :shots]
