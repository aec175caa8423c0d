"""Shared test helpers: hand-made Time Frames and helix truth (no tracker arithmetic)."""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np

VDRIFT = 2.58
BZ = 0.5


def float_tf(sector, row, y, z, bz=BZ, vdrift=VDRIFT):
    sector = np.ascontiguousarray(sector, np.uint8)
    return SimpleNamespace(n=len(sector), fmt=0, sector=sector, row=np.ascontiguousarray(row, np.uint8),
                           y=np.ascontiguousarray(y, np.float32), z=np.ascontiguousarray(z, np.float32),
                           packed=None, bz=bz, vdrift=vdrift)


def row_x(r):
    return 85.0 + r * 160.0 / 151.0


def npads(r):
    return int(math.floor(2.0 * row_x(r) * math.tan(math.radians(10.0)) / 0.4))


def sector_alpha(s):
    return math.radians((s % 18) * 20.0 + 10.0)


class Helix:
    """A particle from (0, 0, zv) at time t0: global circle through the
    origin.  Independent closed form used to pin the oracle's transport."""

    def __init__(self, pt, eta, phi0, q, zv=0.0, t0=0.0, bz=BZ):
        self.pt, self.eta, self.phi0, self.q, self.zv, self.t0 = pt, eta, phi0, q, zv, t0
        self.R = pt / (0.00299792458 * abs(bz))
        self.h = -q if bz > 0 else q
        self.tanl = math.sinh(eta)
        self.cx = -self.h * self.R * math.sin(phi0)
        self.cy = self.h * self.R * math.cos(phi0)

    def at_local_x(self, alpha, x):
        """(y, sin phi_local, arc length, z) at local x in the frame alpha,
        first crossing with 0 < s <= pi R; None if not crossed."""
        ca, sa = math.cos(alpha), math.sin(alpha)
        xc = self.cx * ca + self.cy * sa
        yc = -self.cx * sa + self.cy * ca
        v = (x - xc) / (self.h * self.R)
        if abs(v) > 1:
            return None
        best = None
        for ph in (math.asin(v), math.pi - math.asin(v)):
            s = self.h * self.R * (ph - (self.phi0 - alpha))
            per = 2 * math.pi * self.R
            s = math.fmod(s, per)
            if s < 0:
                s += per
            if 0 < s <= math.pi * self.R and (best is None or s < best[0]):
                best = (s, ph)
        if best is None:
            return None
        s, ph = best
        y = yc - self.h * self.R * math.cos(ph)
        return y, math.sin(ph), s, self.zv + s * self.tanl


class Line:
    """A particle from (0, 0, zv) at time t0 in a field-free TPC (Bz = 0): a
    straight line at azimuth phi0.  Independent closed form for the pulls
    of the field-free fit."""

    def __init__(self, eta, phi0, zv=0.0, t0=0.0):
        self.eta, self.phi0, self.zv, self.t0 = eta, phi0, zv, t0
        self.tanl = math.sinh(eta)

    def at_local_x(self, alpha, x):
        """(y, sin phi_local, arc length, z) at local x in the frame alpha;
        None if the line runs away from that x."""
        ph = self.phi0 - alpha
        c = math.cos(ph)
        if c <= 0:
            return None
        s = x / c
        return x * math.tan(ph), math.sin(ph), s, self.zv + s * self.tanl
