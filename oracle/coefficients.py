"""Time profiles of the Langevin coefficients and their deterministic integrals.

The Langevin SPDE (Eq. spde with b = c = beta = 0) reads
    du = (a(t)/2 d_vv + kappa v d_x) u dt + sigma(t) d_v u dW.
The paper fixes a, sigma constant (Eq. coeffsLangevinConst).  For the
time-dependent benchmark this project uses
    a(t)     = a0 + a1 sin(2 pi t)
    sigma(t) = s0 (1 + s1 cos(2 pi t))
and alpha(t) = a(t)/2 is the weight of the unit operator D^vv (x) I.

All deterministic integrals below are closed forms of these profiles.
"""
from __future__ import annotations

import math

from workloads import COEF_CONST, COEF_TRIG

TWO_PI = 2.0 * math.pi


class Coefficients:
    def __init__(self, kind: int, a0: float, a1: float, s0: float, s1: float):
        if kind not in (COEF_CONST, COEF_TRIG):
            raise ValueError("unknown coefficient kind")
        self.kind = kind
        self.a0, self.s0 = float(a0), float(s0)
        self.a1 = float(a1) if kind == COEF_TRIG else 0.0
        self.s1 = float(s1) if kind == COEF_TRIG else 0.0

    @classmethod
    def of(cls, w) -> "Coefficients":
        return cls(w.kind, w.a0, w.a1, w.s0, w.s1)

    # pointwise profiles -------------------------------------------------
    def a(self, t):
        import numpy as np
        return self.a0 + self.a1 * np.sin(TWO_PI * np.asarray(t, dtype=float))

    def alpha(self, t):
        return 0.5 * self.a(t)

    def sigma(self, t):
        import numpy as np
        return self.s0 * (1.0 + self.s1 * np.cos(TWO_PI * np.asarray(t, dtype=float)))

    # integrals over [t0, t0 + s] -----------------------------------------
    def alpha_bar(self, t0, s):
        """int_{t0}^{t0+s} alpha(r) dr."""
        import numpy as np
        t0 = np.asarray(t0, dtype=float)
        s = np.asarray(s, dtype=float)
        return 0.5 * (self.a0 * s + self.a1 * (np.cos(TWO_PI * t0) - np.cos(TWO_PI * (t0 + s))) / TWO_PI)

    def sigma_sq_integral(self, t0, h):
        """int_{t0}^{t0+h} sigma(r)^2 dr."""
        t1 = t0 + h
        s0, s1 = self.s0, self.s1
        return s0 * s0 * (h + 2.0 * s1 * (math.sin(TWO_PI * t1) - math.sin(TWO_PI * t0)) / TWO_PI
                          + s1 * s1 * (0.5 * h + (math.sin(2 * TWO_PI * t1) - math.sin(2 * TWO_PI * t0))
                                       / (4.0 * TWO_PI)))

    def s_alpha_integral(self, t0, h):
        """int_0^h s alpha(t0 + s) ds."""
        t1 = t0 + h
        c = TWO_PI
        # int_0^h s sin(c (t0 + s)) ds = -h cos(c t1)/c + (sin(c t1) - sin(c t0))/c^2
        trig = -h * math.cos(c * t1) / c + (math.sin(c * t1) - math.sin(c * t0)) / (c * c)
        return 0.5 * (self.a0 * h * h / 2.0 + self.a1 * trig)

    def g3(self, t0, h):
        """int_0^h (s alpha(t0+s) - alpha_bar(t0, s)) ds = 2 int s alpha - h alpha_bar(h)."""
        return 2.0 * self.s_alpha_integral(t0, h) - h * float(self.alpha_bar(t0, h))
