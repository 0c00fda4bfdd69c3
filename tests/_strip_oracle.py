"""A strip of the FP64 oracle with the interface of paper_1811_01604_gb300.strips.GpuStrip
(test support: lets the strip driver run on the CPU, in one process or over gloo ranks).

The strip's block holds its own rows and one row of each neighbouring strip, sliced from
the whole grid's initial state (Eq. 1 and Algorithm 2 step 2.2 by the oracle).  Each
half-sweep is the oracle's Algorithm 1 on the strip's own gap sites of one colour
(orc_sweep_rows: the whole grid's colours and Philox site indices); the strip's partial
totals are the Eq. 2 energy of its bonds after the sweep and its acceptance count, and the
control step is the oracle's Algorithm 2 step 5 (orc_relax_step) on the totals of all
strips.  Equilibrium sums add the back-transformed angles after every sweep, as
orc_predict does.
"""
import numpy as np
import torch

import oracle.oracle as orc
from paper_1811_01604_gb300 import strips


class OracleStrip:
    def __init__(self, phi0, z, mask, y0, y1, prm, chain=0):
        H, W = phi0.shape
        self.row0, self.Hb = strips.block(y0, y1, H)
        self.H, self.W = H, W
        rows = slice(self.row0, self.row0 + self.Hb)
        self.phi = np.ascontiguousarray(phi0[rows], np.float64)
        self.z = np.asarray(z[rows], np.float32)
        self.mask = np.asarray(mask[rows], np.uint8)
        self.own = (y0 - self.row0, y1 - self.row0)
        self.frozen = self.mask.copy()          # the neighbouring strips' rows are never updated here
        self.frozen[:self.own[0]] = 1
        self.frozen[self.own[1]:] = 1
        self.prm, self.chain = prm, chain
        self.ngp = W * (H - 1) + H * (W - 1)
        self.sweep = 0
        self.nacc = 0
        self.in_rows = [torch.zeros(W, dtype=torch.float64) for _ in range(2)]

    def extremes(self):
        z = self.z[self.own[0]:self.own[1]].astype(np.float64)
        s = self.mask[self.own[0]:self.own[1]] != 0
        return (float(z[s].min()), float(z[s].max()), int(s.sum())) if s.any() else (np.inf, -np.inf, 0)

    def init(self, zmin, zmax):
        self.zmin, self.zmax = zmin, zmax

    def set_temperature(self, T):
        self.T = T

    def energy(self):
        return orc.energy_rows(self.phi, self.own[0], self.own[1], self.prm.q)

    def gaps(self):
        return int((self.frozen == 0).sum())

    def begin(self, phase, H_total=0.0, P_total=0.0):
        self.P = int(P_total)
        if phase == 0:
            self.relax = orc.Relax(self.prm, H_total / self.ngp)
        else:
            self.sums = np.zeros_like(self.phi)

    def half_sweep(self, color, phase):
        self.phase = phase
        a = self.relax.s.a if phase == 0 else self.prm.a_eq
        n = orc.sweep_rows(self.phi, self.frozen, self.row0, self.own[0], self.own[1], color, a, self.T,
                           self.prm.q, self.prm.seed, self.chain, self.sweep, self.prm.or_mode)
        self.nacc = n if color == 0 else self.nacc + n

    def vec(self, values):
        return np.array([float(v) for v in values], dtype=np.float64)

    def partials(self):
        E = self.energy() if self.phase == 0 else 0.0
        return np.array([E, float(self.nacc)])

    def control(self, totals, phase):
        totals = np.asarray(totals, np.float64)
        self.sweep += 1
        if phase == 0:
            return not self.relax.step(int(totals[1]), self.P, float(totals[0]) / self.ngp)
        gap = self.frozen == 0
        self.sums[gap] += self.zmin + self.phi[gap] * (self.zmax - self.zmin) / (2 * np.pi)
        return False

    def first_row(self):
        return torch.from_numpy(self.phi[self.own[0]].copy())

    def last_row(self):
        return torch.from_numpy(self.phi[self.own[1] - 1].copy())

    def recv_buffers(self):
        return self.in_rows

    def set_above(self, buf):
        self.phi[0] = np.asarray(buf, np.float64)

    def set_below(self, buf):
        self.phi[-1] = np.asarray(buf, np.float64)

    def predict(self, M):
        out = np.where(self.frozen == 0, self.sums / M, self.z.astype(np.float64))
        return out[self.own[0]:self.own[1]]

    def state(self):
        return self.phi[self.own[0]:self.own[1]]
