"""ten Tusscher-Panfilov 2006 human ventricular model, epicardial (oracle).

Test infrastructure only (see the package docstring).

Sec. 2, "Ten Tusscher model (TP06)": 19 states, 12 membrane currents (fast
Na, L-type Ca, rapid/slow delayed rectifier, inward rectifier, transient
outward, plateau K, Na-Ca exchanger, Na-K pump, sarcolemmal Ca pump,
background Na and Ca), epicardial parameter set.  The paper prints none of
the equations; it cites ten Tusscher & Panfilov, Am. J. Physiol. Heart Circ.
Physiol. 291 (2006) H1088-H1100.  The functions below are written from that
publication with these readings:
  * calcium buffering in the rapid-buffering differential form (factor
    1/(1 + B K/(c + K)^2)) instead of the publication's discrete quadratic
    update, because a Rosenbrock method needs the vector field itself;
  * the stimulus current enters dK_i/dt (as in the original formulation);
  * tau_f2 = 562 exp(-(V+27)^2/240) + 31/(1+exp((25-V)/10)) + 80/(1+exp((V+30)/10))
    as printed in the 2006 article;
  * the L-type current's removable singularity at V = 15 mV is written
    through exprel;
  * h and j switch at V = -40 mV, the V >= -40 branch taken at equality.

Units: V in mV, concentrations in mM, currents in pA/pF.  With the tissue
C_m = 1 uF/cm^2 a current in pA/pF equals one in uA/cm^2.

State order (gates first, then the coupled calcium/concentration block):
  V, m, h, j, d, f, f2, s, r, Xr1, Xr2, Xs, fCass, Rbar, Ki, Nai, Cai, CaSR, CaSS

Parity with the 2006 publication is only partly pinned (the paper prints no
traces): finite-difference Jacobian, the fast gates' steady states at the
published end-diastolic state, every gate's relaxation form, bounds and
direction, the current balance and the biomarker ranges of Sec. 4 (APD90 of
about 354 ms) are the pins.
"""
from __future__ import annotations

import numpy as np

from .cell import CellModel, exprel

R_GAS = 8314.472
T_K = 310.0
F_C = 96485.3415
RTF = R_GAS * T_K / F_C     # mV
FRT = 1.0 / RTF

CAP = 0.185          # cell capacitance, uF
V_C = 0.016404       # uL
V_SR = 0.001094
V_SS = 0.00005468
K_O, NA_O, CA_O = 5.4, 140.0, 2.0
P_KNA = 0.03
G_K1, G_KR, G_KS, G_NA, G_BNA = 5.405, 0.153, 0.392, 14.838, 0.00029
G_CAL, G_BCA, G_TO = 0.0000398, 0.000592, 0.294
P_NAK, K_MK, K_MNA = 2.724, 1.0, 40.0
K_NACA, GAMMA, ALPHA, KM_NAI, KM_CA, K_SAT = 1000.0, 0.35, 2.5, 87.5, 1.38, 0.1
G_PCA, K_PCA, G_PK = 0.1238, 0.0005, 0.0146
K1P, K2P, K3, K4, EC, MAX_SR, MIN_SR = 0.15, 0.045, 0.06, 0.005, 1.5, 2.5, 1.0
V_REL, V_XFER, K_UP, V_LEAK, VMAX_UP = 0.102, 0.0038, 0.00025, 0.00036, 0.006375
BUF_C, K_BUF_C, BUF_SR, K_BUF_SR, BUF_SS, K_BUF_SS = 0.2, 0.001, 10.0, 0.3, 0.4, 0.00025


class TP06(CellModel):
    ns = 19
    names = ("V", "m", "h", "j", "d", "f", "f2", "s", "r", "Xr1", "Xr2", "Xs",
             "fCass", "Rbar", "Ki", "Nai", "Cai", "CaSR", "CaSS")
    gate_rows = (1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12)

    def initial(self):
        # published initial values of the epicardial cell
        return np.array([-85.23, 0.00172, 0.7444, 0.7045, 3.373e-5, 0.7888, 0.9755,
                         0.999998, 2.42e-8, 0.00621, 0.4712, 0.0095, 0.9953, 0.9073,
                         136.89, 8.604, 0.000126, 3.64, 0.00036])

    @staticmethod
    def gate_inf_tau(V, cass):
        """(x_inf, tau_x) for m, h, j, d, f, f2, s, r, Xr1, Xr2, Xs, fCass."""
        e = np.exp
        m_inf = 1.0 / (1.0 + e((-56.86 - V) / 9.03)) ** 2
        am = 1.0 / (1.0 + e((-60.0 - V) / 5.0))
        bm = 0.1 / (1.0 + e((V + 35.0) / 5.0)) + 0.1 / (1.0 + e((V - 50.0) / 200.0))
        tau_m = am * bm
        h_inf = 1.0 / (1.0 + e((V + 71.55) / 7.43)) ** 2
        hi = V.real >= -40.0
        ah = np.where(hi, 0.0, 0.057 * e(-(V + 80.0) / 6.8))
        bh = np.where(hi, 0.77 / (0.13 * (1.0 + e(-(V + 10.66) / 11.1))),
                      2.7 * e(0.079 * V) + 3.1e5 * e(0.3485 * V))
        tau_h = 1.0 / (ah + bh)
        aj = np.where(hi, 0.0,
                      (-2.5428e4 * e(0.2444 * V) - 6.948e-6 * e(-0.04391 * V))
                      * (V + 37.78) / (1.0 + e(0.311 * (V + 79.23))))
        bj = np.where(hi, 0.6 * e(0.057 * V) / (1.0 + e(-0.1 * (V + 32.0))),
                      0.02424 * e(-0.01052 * V) / (1.0 + e(-0.1378 * (V + 40.14))))
        tau_j = 1.0 / (aj + bj)
        j_inf = h_inf
        d_inf = 1.0 / (1.0 + e((-8.0 - V) / 7.5))
        ad = 1.4 / (1.0 + e((-35.0 - V) / 13.0)) + 0.25
        bd = 1.4 / (1.0 + e((V + 5.0) / 5.0))
        cd = 1.0 / (1.0 + e((50.0 - V) / 20.0))
        tau_d = ad * bd + cd
        f_inf = 1.0 / (1.0 + e((V + 20.0) / 7.0))
        tau_f = (1102.5 * e(-(V + 27.0) ** 2 / 225.0) + 200.0 / (1.0 + e((13.0 - V) / 10.0))
                 + 180.0 / (1.0 + e((V + 30.0) / 10.0)) + 20.0)
        f2_inf = 0.67 / (1.0 + e((V + 35.0) / 7.0)) + 0.33
        tau_f2 = (562.0 * e(-(V + 27.0) ** 2 / 240.0) + 31.0 / (1.0 + e((25.0 - V) / 10.0))
                  + 80.0 / (1.0 + e((V + 30.0) / 10.0)))
        s_inf = 1.0 / (1.0 + e((V + 20.0) / 5.0))
        tau_s = (85.0 * e(-(V + 45.0) ** 2 / 320.0) + 5.0 / (1.0 + e((V - 20.0) / 5.0)) + 3.0)
        r_inf = 1.0 / (1.0 + e((20.0 - V) / 6.0))
        tau_r = 9.5 * e(-(V + 40.0) ** 2 / 1800.0) + 0.8
        xr1_inf = 1.0 / (1.0 + e((-26.0 - V) / 7.0))
        tau_xr1 = (450.0 / (1.0 + e((-45.0 - V) / 10.0))) * (6.0 / (1.0 + e((V + 30.0) / 11.5)))
        xr2_inf = 1.0 / (1.0 + e((V + 88.0) / 24.0))
        tau_xr2 = (3.0 / (1.0 + e((-60.0 - V) / 20.0))) * (1.12 / (1.0 + e((V - 60.0) / 20.0)))
        xs_inf = 1.0 / (1.0 + e((-5.0 - V) / 14.0))
        tau_xs = (1400.0 / np.sqrt(1.0 + e((5.0 - V) / 6.0))) * (1.0 / (1.0 + e((V - 35.0) / 15.0))) + 80.0
        q = (cass / 0.05) ** 2
        fcass_inf = 0.6 / (1.0 + q) + 0.4
        tau_fcass = 80.0 / (1.0 + q) + 2.0
        return ((m_inf, tau_m), (h_inf, tau_h), (j_inf, tau_j), (d_inf, tau_d),
                (f_inf, tau_f), (f2_inf, tau_f2), (s_inf, tau_s), (r_inf, tau_r),
                (xr1_inf, tau_xr1), (xr2_inf, tau_xr2), (xs_inf, tau_xs),
                (fcass_inf, tau_fcass))

    def currents(self, X, i_stim):
        (V, m, h, j, d, f, f2, s, r, xr1, xr2, xs, fcass, rbar,
         ki, nai, cai, casr, cass) = X
        e = np.exp
        e_na = RTF * np.log(NA_O / nai)
        e_k = RTF * np.log(K_O / ki)
        e_ks = RTF * np.log((K_O + P_KNA * NA_O) / (ki + P_KNA * nai))
        e_ca = 0.5 * RTF * np.log(CA_O / cai)
        ak1 = 0.1 / (1.0 + e(0.06 * (V - e_k - 200.0)))
        bk1 = (3.0 * e(0.0002 * (V - e_k + 100.0)) + e(0.1 * (V - e_k - 10.0))) \
            / (1.0 + e(-0.5 * (V - e_k)))
        i_k1 = G_K1 * np.sqrt(K_O / 5.4) * ak1 / (ak1 + bk1) * (V - e_k)
        i_to = G_TO * r * s * (V - e_k)
        i_kr = G_KR * np.sqrt(K_O / 5.4) * xr1 * xr2 * (V - e_k)
        i_ks = G_KS * xs ** 2 * (V - e_ks)
        z = 2.0 * (V - 15.0) * FRT
        i_cal = G_CAL * d * f * f2 * fcass * 2.0 * F_C * (0.25 * cass * e(z) - CA_O) / exprel(z)
        i_na = G_NA * m ** 3 * h * j * (V - e_na)
        i_bna = G_BNA * (V - e_na)
        i_bca = G_BCA * (V - e_ca)
        i_nak = (P_NAK * K_O / (K_O + K_MK) * nai / (nai + K_MNA)
                 / (1.0 + 0.1245 * e(-0.1 * V * FRT) + 0.0353 * e(-V * FRT)))
        i_naca = (K_NACA * (e(GAMMA * V * FRT) * nai ** 3 * CA_O
                            - e((GAMMA - 1.0) * V * FRT) * NA_O ** 3 * cai * ALPHA)
                  / ((KM_NAI ** 3 + NA_O ** 3) * (KM_CA + CA_O)
                     * (1.0 + K_SAT * e((GAMMA - 1.0) * V * FRT))))
        i_pca = G_PCA * cai / (cai + K_PCA)
        i_pk = G_PK * (V - e_k) / (1.0 + e((25.0 - V) / 5.98))
        I_ion = (i_k1 + i_to + i_kr + i_ks + i_cal + i_na + i_bna + i_bca
                 + i_nak + i_naca + i_pca + i_pk)

        # sarcoplasmic reticulum and subspace fluxes
        kcasr = MAX_SR - (MAX_SR - MIN_SR) / (1.0 + (EC / casr) ** 2)
        k1 = K1P / kcasr
        k2 = K2P * kcasr
        o = k1 * cass ** 2 * rbar / (K3 + k1 * cass ** 2)
        i_rel = V_REL * o * (casr - cass)
        i_up = VMAX_UP / (1.0 + K_UP ** 2 / cai ** 2)
        i_leak = V_LEAK * (casr - cai)
        i_xfer = V_XFER * (cass - cai)

        gates = (m, h, j, d, f, f2, s, r, xr1, xr2, xs, fcass)
        it = self.gate_inf_tau(V, cass)
        g = np.empty((18,) + np.shape(V), dtype=np.result_type(X, I_ion))
        for k, (x, (xinf, tau)) in enumerate(zip(gates, it)):
            g[k] = (xinf - x) / tau
        g[12] = -k2 * cass * rbar + K4 * (1.0 - rbar)
        g[13] = -(i_k1 + i_to + i_kr + i_ks + i_pk - 2.0 * i_nak - i_stim) * CAP / (V_C * F_C)
        g[14] = -(i_na + i_bna + 3.0 * i_nak + 3.0 * i_naca) * CAP / (V_C * F_C)
        b_c = 1.0 / (1.0 + BUF_C * K_BUF_C / (cai + K_BUF_C) ** 2)
        g[15] = b_c * ((i_leak - i_up) * V_SR / V_C + i_xfer
                       - (i_bca + i_pca - 2.0 * i_naca) * CAP / (2.0 * V_C * F_C))
        b_sr = 1.0 / (1.0 + BUF_SR * K_BUF_SR / (casr + K_BUF_SR) ** 2)
        g[16] = b_sr * (i_up - (i_rel + i_leak))
        b_ss = 1.0 / (1.0 + BUF_SS * K_BUF_SS / (cass + K_BUF_SS) ** 2)
        g[17] = b_ss * (-i_cal * CAP / (2.0 * V_SS * F_C) + i_rel * V_SR / V_SS
                        - i_xfer * V_C / V_SS)
        return I_ion, g


def model() -> TP06:
    return TP06()
