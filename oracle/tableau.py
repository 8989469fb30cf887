"""CHP stabilizer tableau -- TEST INFRASTRUCTURE.

Computes the noiseless reference measurement record of an op list with the
tableau algorithm of Aaronson & Gottesman, "Improved simulation of
stabilizer circuits", PRA 70, 052328 (2004): 2n generator rows
(destabilizers 0..n-1, stabilizers n..2n-1) of symplectic (x | z) bits plus
a sign bit, updated by conjugation for H, S and CX, with the paper's rowsum
phase rule for measurement.

A random measurement outcome is resolved to 0 (the reference-sample
convention of the sampler's C ABI); resets measure and then flip to |0>
(R) or additionally apply H (RX); MX is H, M, H. Noise ops are ignored.
"""
from __future__ import annotations

from typing import Dict, List

import numpy as np


class Tableau:
    def __init__(self, n: int):
        self.n = n
        self.x = np.zeros((2 * n, n), dtype=np.uint8)
        self.z = np.zeros((2 * n, n), dtype=np.uint8)
        self.r = np.zeros(2 * n, dtype=np.uint8)
        for i in range(n):
            self.x[i, i] = 1          # destabilizer X_i
            self.z[n + i, i] = 1      # stabilizer Z_i

    # -- Clifford conjugation (all rows at once) ----------------------------
    def h(self, a: int) -> None:
        self.r ^= self.x[:, a] & self.z[:, a]
        xa = self.x[:, a].copy()
        self.x[:, a] = self.z[:, a]
        self.z[:, a] = xa

    def s(self, a: int) -> None:
        self.r ^= self.x[:, a] & self.z[:, a]
        self.z[:, a] ^= self.x[:, a]

    def cx(self, a: int, b: int) -> None:
        self.r ^= self.x[:, a] & self.z[:, b] & (self.x[:, b] ^ self.z[:, a] ^ 1)
        self.x[:, b] ^= self.x[:, a]
        self.z[:, a] ^= self.z[:, b]

    def pauli_x(self, a: int) -> None:
        self.r ^= self.z[:, a]

    def pauli_z(self, a: int) -> None:
        self.r ^= self.x[:, a]

    # -- rowsum -------------------------------------------------------------
    @staticmethod
    def _g(x1, z1, x2, z2) -> np.ndarray:
        """Exponent of i picked up when multiplying Pauli (x1,z1) by (x2,z2)."""
        x1 = x1.astype(np.int64); z1 = z1.astype(np.int64)
        x2 = x2.astype(np.int64); z2 = z2.astype(np.int64)
        return np.where((x1 == 1) & (z1 == 1), z2 - x2,
               np.where((x1 == 1) & (z1 == 0), z2 * (2 * x2 - 1),
               np.where((x1 == 0) & (z1 == 1), x2 * (1 - 2 * z2), 0)))

    def _rowsum_into(self, hx, hz, hr, ix, iz, ir):
        """(hx,hz,hr) <- (ix,iz,ir) * (hx,hz,hr); rows broadcast."""
        tot = 2 * hr.astype(np.int64) + 2 * ir.astype(np.int64) + self._g(ix, iz, hx, hz).sum(axis=-1)
        tot %= 4
        return hx ^ ix, hz ^ iz, (tot // 2).astype(np.uint8)

    def measure(self, a: int) -> int:
        n = self.n
        stab_x = self.x[n:, a]
        hits = np.nonzero(stab_x)[0]
        if hits.size:
            p = n + int(hits[0])
            rows = [i for i in np.nonzero(self.x[:, a])[0] if i != p]
            if rows:
                rows = np.array(rows)
                nx, nz, nr = self._rowsum_into(self.x[rows], self.z[rows], self.r[rows],
                                               self.x[p][None, :], self.z[p][None, :], self.r[p][None])
                self.x[rows], self.z[rows], self.r[rows] = nx, nz, nr
            self.x[p - n] = self.x[p]
            self.z[p - n] = self.z[p]
            self.r[p - n] = self.r[p]
            self.x[p] = 0
            self.z[p] = 0
            self.z[p, a] = 1
            self.r[p] = 0  # random outcome resolved to 0
            return 0
        sx = np.zeros(n, dtype=np.uint8)
        sz = np.zeros(n, dtype=np.uint8)
        sr = np.zeros(1, dtype=np.uint8)
        for i in np.nonzero(self.x[:n, a])[0]:
            sx, sz, sr = self._rowsum_into(sx[None, :], sz[None, :], sr, self.x[n + i][None, :],
                                           self.z[n + i][None, :], self.r[n + i][None])
            sx, sz = sx[0], sz[0]
        return int(sr[0])


def reference_sample(circuit) -> Dict[str, np.ndarray]:
    """Noiseless reference record (random outcomes -> 0), detector and
    observable parities of ``circuit``."""
    t = Tableau(circuit.n_qubits)
    rec: List[int] = []
    det: List[int] = []
    obs = np.zeros(circuit.n_obs, dtype=np.uint8)
    for op in circuit.ops:
        tg = [int(v) for v in op.targets]
        nm = op.name
        if nm == "R":
            for q in tg:
                if t.measure(q):
                    t.pauli_x(q)
        elif nm == "RX":
            for q in tg:
                if t.measure(q):
                    t.pauli_x(q)
                t.h(q)
        elif nm == "H":
            for q in tg:
                t.h(q)
        elif nm == "S":
            for q in tg:
                t.s(q)
        elif nm == "CX":
            for a in range(0, len(tg), 2):
                t.cx(tg[a], tg[a + 1])
        elif nm == "M":
            for q in tg:
                rec.append(t.measure(q))
        elif nm == "MX":
            for q in tg:
                t.h(q)
                rec.append(t.measure(q))
                t.h(q)
        elif nm == "XFEED":
            for a in range(0, len(tg), 2):
                if rec[tg[a]]:
                    t.pauli_x(tg[a + 1])
        elif nm == "ZFEED":
            for a in range(0, len(tg), 2):
                if rec[tg[a]]:
                    t.pauli_z(tg[a + 1])
        elif nm == "DETECTOR":
            v = 0
            for rr in tg:
                v ^= rec[rr]
            det.append(v)
        elif nm == "OBSERVABLE":
            v = 0
            for rr in tg:
                v ^= rec[rr]
            obs[op.arg] ^= v
    return {"rec": np.array(rec, dtype=np.uint8), "det": np.array(det, dtype=np.uint8), "obs": obs}
