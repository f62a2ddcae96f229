"""Luo-Rudy phase-1 (1991) ventricular membrane model (oracle).

Test infrastructure only (see the package docstring).

Sec. 2, "Luo-Rudy model (LR91)": 8 states (v, m, h, j, d, f, X, [Ca]_i); the
gates obey dk/dt = alpha_k(v)(1 - k) - beta_k(v) k (Eq. (2.9)) and the calcium
concentration dc/dt = S(v, w, c) (Eq. (2.10)).  The paper prints neither the
currents nor the rate functions; it cites Luo & Rudy, Circ. Res. 68 (1991)
1501-1526 and uses its parameter set, except in the experiments of Sec. 4
where G_si = 0.02, G_Na = 4.0 and G_K = 0.423 ("paper" parameter set).  The
functions below are written from that publication: I_ion = I_Na + I_si + I_K +
I_K1 + I_Kp + I_b (the paper's list omits I_K but describes it).

Removable singularities (alpha_m at v = -47.13 mV, the X-gate factor X_i at
v = -77 mV) are written through exprel(z) = (e^z - 1)/z.  The h and j rates
switch at v = -40 mV; the v >= -40 branch is used at equality.

State order: V, m, h, j, d, f, X, Cai.

Parity of these formulas with the 1991 publication is only partly pinned:
the paper prints no cell traces.  Pins used: rest state near the published
-84 mV, biomarker ranges of Sec. 4 (conduction velocity with the paper's
parameter set), finite-difference Jacobian, every gate's rate relaxation
form, non-negative rates, bounds and direction.
"""
from __future__ import annotations

import numpy as np

from .cell import CellModel, exprel

# physical constants as in the 1991 model: R in mJ/(mol K), F in C/mol
R_GAS = 8314.0
T_K = 310.0
F_C = 96484.6
RTF = R_GAS * T_K / F_C          # mV

NA_O, NA_I = 140.0, 18.0
K_O, K_I = 5.4, 145.0
PR_NAK = 0.01833

ORIGINAL = dict(g_na=23.0, g_si=0.09, g_k=0.282)
PAPER = dict(g_na=4.0, g_si=0.02, g_k=0.423)


class LR91(CellModel):
    ns = 8
    names = ("V", "m", "h", "j", "d", "f", "X", "Cai")
    gate_rows = (1, 2, 3, 4, 5, 6)

    def __init__(self, params=None):
        p = dict(ORIGINAL)
        if params:
            p.update(params)
        self.g_na = p["g_na"]
        self.g_si = p["g_si"]
        self.g_k = p["g_k"] * np.sqrt(K_O / 5.4)
        self.g_k1 = 0.6047 * np.sqrt(K_O / 5.4)
        self.e_na = RTF * np.log(NA_O / NA_I)
        self.e_k = RTF * np.log((K_O + PR_NAK * NA_O) / (K_I + PR_NAK * NA_I))
        self.e_k1 = RTF * np.log(K_O / K_I)

    def initial(self):
        return np.array([-84.3801107371, 0.00171338077730188, 0.982660523699656,
                         0.989108212766685, 0.00302126301779861, 0.999967936476325,
                         0.0417603108167287, 0.00017948816388306])

    # -- rate functions of v (Luo & Rudy 1991, Table/appendix) --------------
    @staticmethod
    def rates(V):
        """alpha, beta for m, h, j, d, f, X as arrays (same shape as V)."""
        am = 3.2 / exprel(-0.1 * (V + 47.13))
        bm = 0.08 * np.exp(-V / 11.0)
        hi = V.real >= -40.0
        ah = np.where(hi, 0.0, 0.135 * np.exp((80.0 + V) / -6.8))
        bh = np.where(hi, 1.0 / (0.13 * (1.0 + np.exp((V + 10.66) / -11.1))),
                      3.56 * np.exp(0.079 * V) + 3.1e5 * np.exp(0.35 * V))
        aj = np.where(hi, 0.0,
                      (-1.2714e5 * np.exp(0.2444 * V) - 3.474e-5 * np.exp(-0.04391 * V))
                      * (V + 37.78) / (1.0 + np.exp(0.311 * (V + 79.23))))
        bj = np.where(hi, 0.3 * np.exp(-2.535e-7 * V) / (1.0 + np.exp(-0.1 * (V + 32.0))),
                      0.1212 * np.exp(-0.01052 * V) / (1.0 + np.exp(-0.1378 * (V + 40.14))))
        ad = 0.095 * np.exp(-0.01 * (V - 5.0)) / (1.0 + np.exp(-0.072 * (V - 5.0)))
        bd = 0.07 * np.exp(-0.017 * (V + 44.0)) / (1.0 + np.exp(0.05 * (V + 44.0)))
        af = 0.012 * np.exp(-0.008 * (V + 28.0)) / (1.0 + np.exp(0.15 * (V + 28.0)))
        bf = 0.0065 * np.exp(-0.02 * (V + 30.0)) / (1.0 + np.exp(-0.2 * (V + 30.0)))
        ax = 0.0005 * np.exp(0.083 * (V + 50.0)) / (1.0 + np.exp(0.057 * (V + 50.0)))
        bx = 0.0013 * np.exp(-0.06 * (V + 20.0)) / (1.0 + np.exp(-0.04 * (V + 20.0)))
        return (am, bm), (ah, bh), (aj, bj), (ad, bd), (af, bf), (ax, bx)

    def currents(self, X, i_stim):
        V, m, h, j, d, f, x, cai = X
        i_na = self.g_na * m ** 3 * h * j * (V - self.e_na)
        e_si = 7.7 - 13.0287 * np.log(cai)
        i_si = self.g_si * d * f * (V - e_si)
        xi = np.where(V.real > -100.0,
                      0.11348 * exprel(0.04 * (V + 77.0)) * np.exp(-0.04 * (V + 35.0)), 1.0)
        i_k = self.g_k * x * xi * (V - self.e_k)
        ak1 = 1.02 / (1.0 + np.exp(0.2385 * (V - self.e_k1 - 59.215)))
        bk1 = (0.49124 * np.exp(0.08032 * (V - self.e_k1 + 5.476))
               + np.exp(0.06175 * (V - self.e_k1 - 594.31))) \
            / (1.0 + np.exp(-0.5143 * (V - self.e_k1 + 4.753)))
        i_k1 = self.g_k1 * ak1 / (ak1 + bk1) * (V - self.e_k1)
        kp = 1.0 / (1.0 + np.exp((7.488 - V) / 5.98))
        i_kp = 0.0183 * kp * (V - self.e_k1)
        i_b = 0.03921 * (V + 59.87)
        I_ion = i_na + i_si + i_k + i_k1 + i_kp + i_b

        (am, bm), (ah, bh), (aj, bj), (ad, bd), (af, bf), (ax, bx) = self.rates(V)
        g = np.empty((7,) + np.shape(V), dtype=np.result_type(X, am))
        g[0] = am * (1.0 - m) - bm * m
        g[1] = ah * (1.0 - h) - bh * h
        g[2] = aj * (1.0 - j) - bj * j
        g[3] = ad * (1.0 - d) - bd * d
        g[4] = af * (1.0 - f) - bf * f
        g[5] = ax * (1.0 - x) - bx * x
        g[6] = -1e-4 * i_si + 0.07 * (1e-4 - cai)
        return I_ion, g


def model(paper_params: bool = False) -> LR91:
    return LR91(PAPER if paper_params else None)
