// models.cuh -- LR91 and TP06 membrane models for one mesh node, written
// over the compile-time sparse dual type of sd.cuh.
//
// Sec. 2 of the paper ("Ionic models") couples the bidomain equations to
// the Luo-Rudy 1991 model (8 states) and the ten Tusscher-Panfilov 2006
// epicardial model (19 states).  Neither model's equations are printed in
// the paper; they are written here from the original publications (Luo &
// Rudy, Circ. Res. 68, 1991; ten Tusscher & Panfilov, Am. J. Physiol. 291,
// 2006).  Readings shared with the test oracle and stated in the design
// notes: TP06 calcium buffering in rapid-buffer differential form, the
// stimulus current in dK_i/dt, tau_f2 as printed in the 2006 article, the
// v >= -40 mV branch at the switch of the h/j rates, removable 0/0 points
// written through exprel(z) = (e^z - 1)/z.
//
// Each model exposes
//   NS      number of states (state 0 is the transmembrane voltage V)
//   NG      number of "diagonal" gating states 1..NG: their rows depend only
//           on V and on themselves
//   NB      number of the remaining states NG+1..NS-1 (a small coupled block)
//   ROWMASK compile-time sparsity pattern of the node Jacobian: bit c of
//           ROWMASK[r] is set iff df_r/dX_c can be nonzero (the CTSM block
//           of Sec. 3.3.2)
//   eval(x, istim, inv_cm, sink)  evaluates f_0 = -(I_ion - I_stim)/C_m and
//           f_r = g_r (r >= 1) as SD values and hands each row to
//           sink.put<r>(value); put<r> statically checks that the row's
//           computed sparsity lies inside ROWMASK[r].
#pragma once
#include <cmath>
#include "sd.cuh"

namespace bd {

// ---- precision-dispatched elementary functions ----------------------------
BD_HD double fexp(double x) { return exp(x); }
BD_HD double flog(double x) { return log(x); }
BD_HD double fsqrt(double x) { return sqrt(x); }
BD_HD float fexp(float x) {
#ifdef __CUDA_ARCH__
  return __expf(x);
#else
  return expf(x);
#endif
}
BD_HD float flog(float x) {
#ifdef __CUDA_ARCH__
  return __logf(x);
#else
  return logf(x);
#endif
}
BD_HD float fsqrt(float x) { return sqrtf(x); }

// (e^z - 1)/z and its derivative, series near 0
BD_HD void exprel_vd(double z, double& f, double& df) {
  if (fabs(z) < 1e-2) {
    f = 1.0 + z * (1.0 / 2 + z * (1.0 / 6 + z * (1.0 / 24 + z * (1.0 / 120 + z * (1.0 / 720)))));
    df = 1.0 / 2 + z * (1.0 / 3 + z * (1.0 / 8 + z * (1.0 / 30 + z * (1.0 / 144 + z * (1.0 / 840)))));
  } else {
    const double em1 = expm1(z);
    f = em1 / z;
    df = ((em1 + 1.0) * z - em1) / (z * z);
  }
}
BD_HD void exprel_vd(float z, float& f, float& df) {
  if (fabsf(z) < 0.1f) {
    f = 1.f + z * (1.f / 2 + z * (1.f / 6 + z * (1.f / 24 + z * (1.f / 120))));
    df = 1.f / 2 + z * (1.f / 3 + z * (1.f / 8 + z * (1.f / 30)));
  } else {
    const float e = fexp(z);
    f = (e - 1.f) / z;
    df = (e * z - (e - 1.f)) / (z * z);
  }
}

template <class T, uint32_t A> BD_HD SD<T, A> sexp(const SD<T, A>& a) { const T e = fexp(a.v); return chain(a, e, e); }
template <class T, uint32_t A> BD_HD SD<T, A> slog(const SD<T, A>& a) { return chain(a, flog(a.v), T(1) / a.v); }
template <class T, uint32_t A> BD_HD SD<T, A> ssqrt(const SD<T, A>& a) { const T s = fsqrt(a.v); return chain(a, s, T(0.5) / s); }
template <class T, uint32_t A> BD_HD SD<T, A> sexprel(const SD<T, A>& a) { T f, df; exprel_vd(a.v, f, df); return chain(a, f, df); }
template <class T, uint32_t A> BD_HD SD<T, A> zero_like() { SD<T, A> r; r.v = T(0); for (int k = 0; k < SD<T, A>::nnz; ++k) r.d[k] = T(0); return r; }

constexpr uint32_t B(int k) { return 1u << k; }

// ===========================================================================
// Luo-Rudy 1991.  State order: V, m, h, j, d, f, X, Cai.
// ===========================================================================
template <class T>
struct LR91 {
  static constexpr int NS = 8, NG = 6, NB = 1;
  static constexpr uint32_t ROWMASK[NS] = {
      0xFFu,                                   // V: all currents
      B(0) | B(1), B(0) | B(2), B(0) | B(3),   // m, h, j
      B(0) | B(4), B(0) | B(5), B(0) | B(6),   // d, f, X
      B(0) | B(4) | B(5) | B(7)};              // Cai: -1e-4 I_si + 0.07 (1e-4 - Cai)

  T g_na, g_si, g_k, g_k1, e_na, e_k, e_k1;

  // parameters: paper_mod selects G_si = 0.02, G_Na = 4.0, G_K = 0.423 (Sec. 4)
  static LR91 make(bool paper_mod) {
    const double rtf = 8314.0 * 310.0 / 96484.6;
    const double nao = 140.0, nai = 18.0, ko = 5.4, ki = 145.0, pr = 0.01833;
    LR91 p;
    p.g_na = T(paper_mod ? 4.0 : 23.0);
    p.g_si = T(paper_mod ? 0.02 : 0.09);
    p.g_k = T((paper_mod ? 0.423 : 0.282) * std::sqrt(ko / 5.4));
    p.g_k1 = T(0.6047 * std::sqrt(ko / 5.4));
    p.e_na = T(rtf * std::log(nao / nai));
    p.e_k = T(rtf * std::log((ko + pr * nao) / (ki + pr * nai)));
    p.e_k1 = T(rtf * std::log(ko / ki));
    return p;
  }

  template <class Sink>
  BD_HD void eval(const T* x, T istim, T inv_cm, Sink& out) const {
    const auto V = var<0>(x[0]);
    const bool hi = x[0] >= T(-40);
    {  // m
      const auto m = var<1>(x[1]);
      const auto am = T(3.2) / sexprel(T(-0.1) * (V + T(47.13)));
      const auto bm = T(0.08) * sexp(V * T(-1.0 / 11.0));
      out.template put<1>(am * (T(1) - m) - bm * m);
    }
    {  // h
      const auto h = var<2>(x[2]);
      SD<T, 1u> ah, bh;
      if (hi) {
        ah = zero_like<T, 1u>();
        bh = T(1) / (T(0.13) * (T(1) + sexp((V + T(10.66)) * T(-1.0 / 11.1))));
      } else {
        ah = T(0.135) * sexp((V + T(80)) * T(-1.0 / 6.8));
        bh = T(3.56) * sexp(T(0.079) * V) + T(3.1e5) * sexp(T(0.35) * V);
      }
      out.template put<2>(ah * (T(1) - h) - bh * h);
    }
    {  // j
      const auto jg = var<3>(x[3]);
      SD<T, 1u> aj, bj;
      if (hi) {
        aj = zero_like<T, 1u>();
        bj = T(0.3) * sexp(T(-2.535e-7) * V) / (T(1) + sexp(T(-0.1) * (V + T(32))));
      } else {
        aj = (T(-1.2714e5) * sexp(T(0.2444) * V) - T(3.474e-5) * sexp(T(-0.04391) * V)) * (V + T(37.78))
             / (T(1) + sexp(T(0.311) * (V + T(79.23))));
        bj = T(0.1212) * sexp(T(-0.01052) * V) / (T(1) + sexp(T(-0.1378) * (V + T(40.14))));
      }
      out.template put<3>(aj * (T(1) - jg) - bj * jg);
    }
    {  // d
      const auto d = var<4>(x[4]);
      const auto ad = T(0.095) * sexp(T(-0.01) * (V - T(5))) / (T(1) + sexp(T(-0.072) * (V - T(5))));
      const auto bd = T(0.07) * sexp(T(-0.017) * (V + T(44))) / (T(1) + sexp(T(0.05) * (V + T(44))));
      out.template put<4>(ad * (T(1) - d) - bd * d);
    }
    {  // f
      const auto f = var<5>(x[5]);
      const auto af = T(0.012) * sexp(T(-0.008) * (V + T(28))) / (T(1) + sexp(T(0.15) * (V + T(28))));
      const auto bf = T(0.0065) * sexp(T(-0.02) * (V + T(30))) / (T(1) + sexp(T(-0.2) * (V + T(30))));
      out.template put<5>(af * (T(1) - f) - bf * f);
    }
    {  // X
      const auto X = var<6>(x[6]);
      const auto ax = T(0.0005) * sexp(T(0.083) * (V + T(50))) / (T(1) + sexp(T(0.057) * (V + T(50))));
      const auto bx = T(0.0013) * sexp(T(-0.06) * (V + T(20))) / (T(1) + sexp(T(-0.04) * (V + T(20))));
      out.template put<6>(ax * (T(1) - X) - bx * X);
    }
    // currents
    const auto m = var<1>(x[1]);
    const auto h = var<2>(x[2]);
    const auto jg = var<3>(x[3]);
    const auto d = var<4>(x[4]);
    const auto f = var<5>(x[5]);
    const auto X = var<6>(x[6]);
    const auto ca = var<7>(x[7]);
    const auto i_na = g_na * (m * m * m) * h * jg * (V - e_na);
    const auto e_si = T(7.7) - T(13.0287) * slog(ca);
    const auto i_si = g_si * d * f * (V - e_si);
    SD<T, 1u> xi;
    if (x[0] > T(-100)) xi = T(0.11348) * sexprel(T(0.04) * (V + T(77))) * sexp(T(-0.04) * (V + T(35)));
    else { xi = zero_like<T, 1u>(); xi.v = T(1); }
    const auto i_k = g_k * X * xi * (V - e_k);
    const auto dv1 = V - e_k1;
    const auto ak1 = T(1.02) / (T(1) + sexp(T(0.2385) * (dv1 - T(59.215))));
    const auto bk1 = (T(0.49124) * sexp(T(0.08032) * (dv1 + T(5.476))) + sexp(T(0.06175) * (dv1 - T(594.31))))
                     / (T(1) + sexp(T(-0.5143) * (dv1 + T(4.753))));
    const auto i_k1 = g_k1 * (ak1 / (ak1 + bk1)) * dv1;
    const auto kp = T(1) / (T(1) + sexp((T(7.488) - V) * T(1.0 / 5.98)));
    const auto i_kp = T(0.0183) * kp * dv1;
    const auto i_b = T(0.03921) * (V + T(59.87));
    const auto I = i_na + i_si + i_k + i_k1 + i_kp + i_b;
    out.template put<0>((I - istim) * (-inv_cm));
    out.template put<7>(T(-1e-4) * i_si + T(0.07) * (T(1e-4) - ca));
  }

  static void initial(double* x) {
    const double v[8] = {-84.3801107371, 0.00171338077730188, 0.982660523699656, 0.989108212766685,
                         0.00302126301779861, 0.999967936476325, 0.0417603108167287, 0.00017948816388306};
    for (int k = 0; k < 8; ++k) x[k] = v[k];
  }
};

// ===========================================================================
// ten Tusscher-Panfilov 2006, epicardial.  State order:
//  0 V, 1 m, 2 h, 3 j, 4 d, 5 f, 6 f2, 7 s, 8 r, 9 Xr1, 10 Xr2, 11 Xs,
// 12 fCass, 13 Rbar, 14 Ki, 15 Nai, 16 Cai, 17 CaSR, 18 CaSS
// ===========================================================================
template <class T>
struct TP06 {
  static constexpr int NS = 19, NG = 11, NB = 7;
  enum { V_ = 0, M_, H_, J_, D_, F_, F2_, S_, R_, XR1_, XR2_, XS_, FCASS_, RBAR_, KI_, NAI_, CAI_, CASR_, CASS_ };
  static constexpr uint32_t GATE(int k) { return B(0) | B(k); }
  static constexpr uint32_t ROWMASK[NS] = {
      0x7FFFFu & ~B(13) & ~B(17),                           // V: every current (not Rbar, CaSR)
      GATE(1), GATE(2), GATE(3), GATE(4), GATE(5), GATE(6),
      GATE(7), GATE(8), GATE(9), GATE(10), GATE(11),
      B(12) | B(18),                                        // fCass: fCass, CaSS
      B(13) | B(17) | B(18),                                // Rbar: k2(CaSR) CaSS Rbar
      B(0) | B(7) | B(8) | B(9) | B(10) | B(11) | B(14) | B(15),   // Ki
      B(0) | B(1) | B(2) | B(3) | B(15) | B(16),            // Nai
      B(0) | B(15) | B(16) | B(17) | B(18),                 // Cai
      B(13) | B(16) | B(17) | B(18),                        // CaSR
      B(0) | B(4) | B(5) | B(6) | B(12) | B(13) | B(16) | B(17) | B(18)};  // CaSS

  // constants of the 2006 publication (epicardial cell)
  static constexpr double R_GAS = 8314.472, T_K = 310.0, F_C = 96485.3415;
  static constexpr double CAP = 0.185, V_C = 0.016404, V_SR = 0.001094, V_SS = 0.00005468;
  static constexpr double K_O = 5.4, NA_O = 140.0, CA_O = 2.0, P_KNA = 0.03;
  static constexpr double G_K1 = 5.405, G_KR = 0.153, G_KS = 0.392, G_NA = 14.838, G_BNA = 0.00029;
  static constexpr double G_CAL = 0.0000398, G_BCA = 0.000592, G_TO = 0.294;
  static constexpr double P_NAK = 2.724, K_MK = 1.0, K_MNA = 40.0;
  static constexpr double K_NACA = 1000.0, GAM = 0.35, ALPH = 2.5, KM_NAI = 87.5, KM_CA = 1.38, K_SAT = 0.1;
  static constexpr double G_PCA = 0.1238, K_PCA = 0.0005, G_PK = 0.0146;
  static constexpr double K1P = 0.15, K2P = 0.045, K3 = 0.06, K4 = 0.005, EC = 1.5, MAX_SR = 2.5, MIN_SR = 1.0;
  static constexpr double V_REL = 0.102, V_XFER = 0.0038, K_UP = 0.00025, V_LEAK = 0.00036, VMAX_UP = 0.006375;
  static constexpr double BUF_C = 0.2, K_BUF_C = 0.001, BUF_SR = 10.0, K_BUF_SR = 0.3, BUF_SS = 0.4, K_BUF_SS = 0.00025;

  T rtf, frt, log_nao, log_ko, log_cao, sq_ko;   // derived, set by make()

  static TP06 make() {
    TP06 p;
    const double rtf = R_GAS * T_K / F_C;
    p.rtf = T(rtf);
    p.frt = T(1.0 / rtf);
    p.log_nao = T(std::log(NA_O));
    p.log_ko = T(std::log(K_O));
    p.log_cao = T(std::log(CA_O));
    p.sq_ko = T(std::sqrt(K_O / 5.4));
    return p;
  }

  template <int K, class Sink, class XINF, class TAU>
  BD_HD static void gate(const T* x, const XINF& xinf, const TAU& tau, Sink& out) {
    const auto g = var<K>(x[K]);
    out.template put<K>((xinf - g) / tau);
  }

  template <class Sink>
  BD_HD void eval(const T* x, T istim, T inv_cm, Sink& out) const {
    const auto V = var<0>(x[0]);
    const bool hi = x[0] >= T(-40);
    // ---- gates (rows 1..11) -------------------------------------------------
    {
      const auto e1 = T(1) + sexp((T(-56.86) - V) * T(1.0 / 9.03));
      const auto m_inf = T(1) / (e1 * e1);
      const auto am = T(1) / (T(1) + sexp((T(-60) - V) * T(0.2)));
      const auto bm = T(0.1) / (T(1) + sexp((V + T(35)) * T(0.2))) + T(0.1) / (T(1) + sexp((V - T(50)) * T(1.0 / 200)));
      gate<1>(x, m_inf, am * bm, out);
    }
    const auto e_h = T(1) + sexp((V + T(71.55)) * T(1.0 / 7.43));
    const auto hj_inf = T(1) / (e_h * e_h);
    {
      SD<T, 1u> ah, bh;
      if (hi) {
        ah = zero_like<T, 1u>();
        bh = T(0.77) / (T(0.13) * (T(1) + sexp((V + T(10.66)) * T(-1.0 / 11.1))));
      } else {
        ah = T(0.057) * sexp((V + T(80)) * T(-1.0 / 6.8));
        bh = T(2.7) * sexp(T(0.079) * V) + T(3.1e5) * sexp(T(0.3485) * V);
      }
      gate<2>(x, hj_inf, T(1) / (ah + bh), out);
    }
    {
      SD<T, 1u> aj, bj;
      if (hi) {
        aj = zero_like<T, 1u>();
        bj = T(0.6) * sexp(T(0.057) * V) / (T(1) + sexp(T(-0.1) * (V + T(32))));
      } else {
        aj = (T(-2.5428e4) * sexp(T(0.2444) * V) - T(6.948e-6) * sexp(T(-0.04391) * V)) * (V + T(37.78))
             / (T(1) + sexp(T(0.311) * (V + T(79.23))));
        bj = T(0.02424) * sexp(T(-0.01052) * V) / (T(1) + sexp(T(-0.1378) * (V + T(40.14))));
      }
      gate<3>(x, hj_inf, T(1) / (aj + bj), out);
    }
    {
      const auto d_inf = T(1) / (T(1) + sexp((T(-8) - V) * T(1.0 / 7.5)));
      const auto ad = T(1.4) / (T(1) + sexp((T(-35) - V) * T(1.0 / 13))) + T(0.25);
      const auto bd = T(1.4) / (T(1) + sexp((V + T(5)) * T(0.2)));
      const auto cd = T(1) / (T(1) + sexp((T(50) - V) * T(0.05)));
      gate<4>(x, d_inf, ad * bd + cd, out);
    }
    {
      const auto f_inf = T(1) / (T(1) + sexp((V + T(20)) * T(1.0 / 7)));
      const auto w = V + T(27);
      const auto tau_f = T(1102.5) * sexp(w * w * T(-1.0 / 225)) + T(200) / (T(1) + sexp((T(13) - V) * T(0.1)))
                         + T(180) / (T(1) + sexp((V + T(30)) * T(0.1))) + T(20);
      gate<5>(x, f_inf, tau_f, out);
      const auto f2_inf = T(0.67) / (T(1) + sexp((V + T(35)) * T(1.0 / 7))) + T(0.33);
      const auto tau_f2 = T(562) * sexp(w * w * T(-1.0 / 240)) + T(31) / (T(1) + sexp((T(25) - V) * T(0.1)))
                          + T(80) / (T(1) + sexp((V + T(30)) * T(0.1)));
      gate<6>(x, f2_inf, tau_f2, out);
    }
    {
      const auto s_inf = T(1) / (T(1) + sexp((V + T(20)) * T(0.2)));
      const auto w = V + T(45);
      const auto tau_s = T(85) * sexp(w * w * T(-1.0 / 320)) + T(5) / (T(1) + sexp((V - T(20)) * T(0.2))) + T(3);
      gate<7>(x, s_inf, tau_s, out);
      const auto r_inf = T(1) / (T(1) + sexp((T(20) - V) * T(1.0 / 6)));
      const auto w2 = V + T(40);
      const auto tau_r = T(9.5) * sexp(w2 * w2 * T(-1.0 / 1800)) + T(0.8);
      gate<8>(x, r_inf, tau_r, out);
    }
    {
      const auto xr1_inf = T(1) / (T(1) + sexp((T(-26) - V) * T(1.0 / 7)));
      const auto tau_xr1 = (T(450) / (T(1) + sexp((T(-45) - V) * T(0.1)))) * (T(6) / (T(1) + sexp((V + T(30)) * T(1.0 / 11.5))));
      gate<9>(x, xr1_inf, tau_xr1, out);
      const auto xr2_inf = T(1) / (T(1) + sexp((V + T(88)) * T(1.0 / 24)));
      const auto tau_xr2 = (T(3) / (T(1) + sexp((T(-60) - V) * T(0.05)))) * (T(1.12) / (T(1) + sexp((V - T(60)) * T(0.05))));
      gate<10>(x, xr2_inf, tau_xr2, out);
      const auto xs_inf = T(1) / (T(1) + sexp((T(-5) - V) * T(1.0 / 14)));
      const auto tau_xs = (T(1400) / ssqrt(T(1) + sexp((T(5) - V) * T(1.0 / 6)))) * (T(1) / (T(1) + sexp((V - T(35)) * T(1.0 / 15)))) + T(80);
      gate<11>(x, xs_inf, tau_xs, out);
    }
    // ---- currents ------------------------------------------------------------
    const auto m = var<1>(x[1]);
    const auto h = var<2>(x[2]);
    const auto jg = var<3>(x[3]);
    const auto d = var<4>(x[4]);
    const auto f = var<5>(x[5]);
    const auto f2 = var<6>(x[6]);
    const auto s = var<7>(x[7]);
    const auto r = var<8>(x[8]);
    const auto xr1 = var<9>(x[9]);
    const auto xr2 = var<10>(x[10]);
    const auto xs = var<11>(x[11]);
    const auto fcass = var<12>(x[12]);
    const auto rbar = var<13>(x[13]);
    const auto ki = var<14>(x[14]);
    const auto nai = var<15>(x[15]);
    const auto cai = var<16>(x[16]);
    const auto casr = var<17>(x[17]);
    const auto cass = var<18>(x[18]);

    const auto e_na = rtf * (log_nao - slog(nai));
    const auto e_k = rtf * (log_ko - slog(ki));
    const auto e_ks = rtf * slog((T(K_O + P_KNA * NA_O)) / (ki + T(P_KNA) * nai));
    const auto e_ca = T(0.5) * rtf * (log_cao - slog(cai));
    const auto vk = V - e_k;
    const auto ak1 = T(0.1) / (T(1) + sexp(T(0.06) * (vk - T(200))));
    const auto bk1 = (T(3) * sexp(T(0.0002) * (vk + T(100))) + sexp(T(0.1) * (vk - T(10)))) / (T(1) + sexp(T(-0.5) * vk));
    const auto i_k1 = T(G_K1) * sq_ko * (ak1 / (ak1 + bk1)) * vk;
    const auto i_to = T(G_TO) * r * s * vk;
    const auto i_kr = T(G_KR) * sq_ko * xr1 * xr2 * vk;
    const auto i_ks = T(G_KS) * (xs * xs) * (V - e_ks);
    const auto z = T(2) * frt * (V - T(15));
    const auto i_cal = T(G_CAL * 2.0 * F_C) * d * f * f2 * fcass * (T(0.25) * cass * sexp(z) - T(CA_O)) / sexprel(z);
    const auto i_na = T(G_NA) * (m * m * m) * h * jg * (V - e_na);
    const auto i_bna = T(G_BNA) * (V - e_na);
    const auto i_bca = T(G_BCA) * (V - e_ca);
    const auto i_nak = T(P_NAK * K_O / (K_O + K_MK)) * nai / (nai + T(K_MNA))
                       / (T(1) + T(0.1245) * sexp(T(-0.1) * frt * V) + T(0.0353) * sexp(-frt * V));
    const auto eg = sexp(T(GAM) * frt * V);
    const auto eg1 = sexp(T(GAM - 1.0) * frt * V);
    const auto i_naca = T(K_NACA / ((KM_NAI * KM_NAI * KM_NAI + NA_O * NA_O * NA_O) * (KM_CA + CA_O)))
                        * (eg * (nai * nai * nai) * T(CA_O) - eg1 * T(NA_O * NA_O * NA_O * ALPH) * cai)
                        / (T(1) + T(K_SAT) * eg1);
    const auto i_pca = T(G_PCA) * cai / (cai + T(K_PCA));
    const auto i_pk = T(G_PK) * vk / (T(1) + sexp((T(25) - V) * T(1.0 / 5.98)));
    const auto I = i_k1 + i_to + i_kr + i_ks + i_cal + i_na + i_bna + i_bca + i_nak + i_naca + i_pca + i_pk;
    out.template put<0>((I - istim) * (-inv_cm));

    // ---- fCass, Rbar and the concentrations ------------------------------------
    {
      const auto q = (cass * T(20)) * (cass * T(20));
      const auto fcass_inf = T(0.6) / (T(1) + q) + T(0.4);
      const auto tau_fcass = T(80) / (T(1) + q) + T(2);
      out.template put<12>((fcass_inf - fcass) / tau_fcass);
    }
    const auto ecs = T(EC) / casr;
    const auto kcasr = T(MAX_SR) - T(MAX_SR - MIN_SR) / (T(1) + ecs * ecs);
    const auto k1 = T(K1P) / kcasr;
    const auto k2 = T(K2P) * kcasr;
    out.template put<13>(-(k2 * cass * rbar) + T(K4) * (T(1) - rbar));
    const auto cs2 = cass * cass;
    const auto o = k1 * cs2 * rbar / (T(K3) + k1 * cs2);
    const auto i_rel = T(V_REL) * o * (casr - cass);
    const auto kc = T(K_UP) / cai;
    const auto i_up = T(VMAX_UP) / (T(1) + kc * kc);
    const auto i_leak = T(V_LEAK) * (casr - cai);
    const auto i_xfer = T(V_XFER) * (cass - cai);
    const T cvf = T(CAP / (V_C * F_C));
    out.template put<14>((i_k1 + i_to + i_kr + i_ks + i_pk - T(2) * i_nak - istim) * (-cvf));
    out.template put<15>((i_na + i_bna + T(3) * i_nak + T(3) * i_naca) * (-cvf));
    {
      const auto bc = cai + T(K_BUF_C);
      const auto b_c = T(1) / (T(1) + T(BUF_C * K_BUF_C) / (bc * bc));
      out.template put<16>(b_c * ((i_leak - i_up) * T(V_SR / V_C) + i_xfer
                                  - (i_bca + i_pca - T(2) * i_naca) * T(CAP / (2.0 * V_C * F_C))));
    }
    {
      const auto bs = casr + T(K_BUF_SR);
      const auto b_sr = T(1) / (T(1) + T(BUF_SR * K_BUF_SR) / (bs * bs));
      out.template put<17>(b_sr * (i_up - (i_rel + i_leak)));
    }
    {
      const auto bs = cass + T(K_BUF_SS);
      const auto b_ss = T(1) / (T(1) + T(BUF_SS * K_BUF_SS) / (bs * bs));
      out.template put<18>(b_ss * (i_cal * T(-CAP / (2.0 * V_SS * F_C)) + i_rel * T(V_SR / V_SS)
                                   - i_xfer * T(V_C / V_SS)));
    }
  }

  static void initial(double* x) {
    const double v[19] = {-85.23, 0.00172, 0.7444, 0.7045, 3.373e-5, 0.7888, 0.9755, 0.999998, 2.42e-8,
                          0.00621, 0.4712, 0.0095, 0.9953, 0.9073, 136.89, 8.604, 0.000126, 3.64, 0.00036};
    for (int k = 0; k < 19; ++k) x[k] = v[k];
  }
};

// ---- sinks -------------------------------------------------------------------

// Collects the node field and the Jacobian entries the condensation needs,
// touching only entries of the declared pattern.
template <class T, class Model>
struct JacSink {
  static constexpr int NS = Model::NS, NG = Model::NG, NB = Model::NB;
  T f[NS];
  T jv[NS];          // d f_0 / dX_c
  T jgd[NG + 1];     // gate diagonals d g_k / d x_k   (index 1..NG)
  T jgv[NG + 1];     // gate d g_k / dV
  T jb[NB][NS];      // block rows: d f_{NG+1+r} / dX_c

  template <int ROW, uint32_t M>
  BD_HD void put(const SD<T, M>& a) {
    static_assert((M & ~Model::ROWMASK[ROW]) == 0u, "row sparsity exceeds its declared pattern");
    f[ROW] = a.v;
    if constexpr (ROW == 0) {
      for_bits<Model::ROWMASK[0]>([&](auto b) { constexpr int c = decltype(b)::value; jv[c] = a.template der<c>(); });
    } else if constexpr (ROW <= NG) {
      static_assert((Model::ROWMASK[ROW] & ~(1u | (1u << ROW))) == 0u, "gate rows may depend on V and themselves only");
      jgd[ROW] = a.template der<ROW>();
      jgv[ROW] = a.template der<0>();
    } else {
      constexpr int r = ROW - 1 - NG;
      for_bits<Model::ROWMASK[ROW]>([&](auto b) { constexpr int c = decltype(b)::value; jb[r][c] = a.template der<c>(); });
    }
  }
};

// Values only (derivative arithmetic is dead code and removed by the compiler).
template <class T, class Model>
struct ValSink {
  T f[Model::NS];
  template <int ROW, uint32_t M>
  BD_HD void put(const SD<T, M>& a) { f[ROW] = a.v; }
};

// Dense Jacobian (tests and the host rest-state Newton).
template <class T, class Model>
struct DenseSink {
  T f[Model::NS];
  T J[Model::NS][Model::NS];
  BD_HD DenseSink() {
    for (int r = 0; r < Model::NS; ++r)
      for (int c = 0; c < Model::NS; ++c) J[r][c] = T(0);
  }
  template <int ROW, uint32_t M>
  BD_HD void put(const SD<T, M>& a) {
    static_assert((M & ~Model::ROWMASK[ROW]) == 0u, "row sparsity exceeds its declared pattern");
    f[ROW] = a.v;
    for_bits<M>([&](auto b) { constexpr int c = decltype(b)::value; J[ROW][c] = a.template der<c>(); });
  }
};

// ---- condensation onto v ------------------------------------------------------
//
// The node block of (alpha Mt - W) couples v to the remaining states y through
// A = alpha I - j_yy.  With rho the y right-hand side, the block elimination
//   k_y = z + w k_v,   z = A^{-1} rho,   w = A^{-1} j_yv
// leaves for v the Schur diagonal s = -j_vv - j_vy . w and the right-hand-side
// correction corr = j_vy . z.  A is block lower triangular (diagonal gates,
// then the NB x NB block that may depend on the gates), so the solve is a
// diagonal scaling followed by one small dense elimination.
template <class T, class Model>
BD_HD void condense(const JacSink<T, Model>& e, T alpha, const T* rho, T& s, T& corr, T* z, T* w) {
  constexpr int NG = Model::NG, NB = Model::NB;
  constexpr uint32_t GATES = ((1u << (NG + 1)) - 1u) & ~1u;
#pragma unroll
  for (int g = 1; g <= NG; ++g) {
    const T inv = T(1) / (alpha - e.jgd[g]);
    z[g - 1] = rho[g - 1] * inv;
    w[g - 1] = e.jgv[g] * inv;
  }
  T Bm[NB][NB];
  T rz[NB], rw[NB];
  auto fill = [&](auto rr) {
    constexpr int r = decltype(rr)::value;
    constexpr uint32_t RM = Model::ROWMASK[NG + 1 + r];
    rz[r] = rho[NG + r];
    if constexpr ((RM & 1u) != 0u) rw[r] = e.jb[r][0];
    else rw[r] = T(0);
    for_bits<RM & GATES>([&](auto b) {
      constexpr int c = decltype(b)::value;
      rz[r] += e.jb[r][c] * z[c - 1];
      rw[r] += e.jb[r][c] * w[c - 1];
    });
#pragma unroll
    for (int c = 0; c < NB; ++c) Bm[r][c] = (r == c) ? alpha : T(0);
    for_bits<(RM >> (NG + 1))>([&](auto b) {
      constexpr int c = decltype(b)::value;
      Bm[r][c] -= e.jb[r][NG + 1 + c];
    });
  };
  [&]<int... R>(std::integer_sequence<int, R...>) { (fill(std::integral_constant<int, R>{}), ...); }
  (std::make_integer_sequence<int, NB>{});
  // in-register LU without pivoting (A = alpha I - j_yy is dominated by alpha I)
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const T piv = T(1) / Bm[k][k];
#pragma unroll
    for (int i = k + 1; i < NB; ++i) {
      const T l = Bm[i][k] * piv;
#pragma unroll
      for (int c = k + 1; c < NB; ++c) Bm[i][c] -= l * Bm[k][c];
      rz[i] -= l * rz[k];
      rw[i] -= l * rw[k];
    }
  }
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
#pragma unroll
    for (int c = i + 1; c < NB; ++c) {
      rz[i] -= Bm[i][c] * rz[c];
      rw[i] -= Bm[i][c] * rw[c];
    }
    const T inv = T(1) / Bm[i][i];
    rz[i] *= inv;
    rw[i] *= inv;
    z[NG + i] = rz[i];
    w[NG + i] = rw[i];
  }
  s = -e.jv[0];
  corr = T(0);
  for_bits<Model::ROWMASK[0] & ~1u>([&](auto b) {
    constexpr int c = decltype(b)::value;
    s -= e.jv[c] * w[c - 1];
    corr += e.jv[c] * z[c - 1];
  });
}

// The node field and Jacobian (every entry of the declared pattern), stored
// by one membrane kernel and loaded by another that needs them at the same
// state (with the same or another shift).  Slots per node (strided by the
// node count; Jacobian entries outside the pattern are neither written nor
// read):
//   [0, NS)                 d f_0 / d X_c
//   [NS, NS + NG)           gate diagonals d g_k / d x_k, k = 1..NG
//   [NS + NG, NS + 2 NG)    gate d g_k / dV
//   then NB rows of NS      d f_{NG+1+r} / d X_c
//   then NS                 the field f
template <class Model>
constexpr int jac_pack_size() {
  return Model::NS + 2 * Model::NG + Model::NB * Model::NS + Model::NS;
}

template <class T, class Model, bool WITH_F = true>
BD_HD void jac_store(const JacSink<T, Model>& e, T* pk, int64_t stride) {
  constexpr int NS = Model::NS, NG = Model::NG, NB = Model::NB;
  for_bits<Model::ROWMASK[0]>([&](auto b) {
    constexpr int c = decltype(b)::value;
    pk[c * stride] = e.jv[c];
  });
#pragma unroll
  for (int g = 1; g <= NG; ++g) {
    pk[(NS + g - 1) * stride] = e.jgd[g];
    pk[(NS + NG + g - 1) * stride] = e.jgv[g];
  }
  auto row = [&](auto rr) {
    constexpr int r = decltype(rr)::value;
    for_bits<Model::ROWMASK[NG + 1 + r]>([&](auto b) {
      constexpr int c = decltype(b)::value;
      pk[(NS + 2 * NG + r * NS + c) * stride] = e.jb[r][c];
    });
  };
  [&]<int... R>(std::integer_sequence<int, R...>) { (row(std::integral_constant<int, R>{}), ...); }
  (std::make_integer_sequence<int, NB>{});
  if constexpr (WITH_F) {
#pragma unroll
    for (int k = 0; k < NS; ++k) pk[(NS + 2 * NG + NB * NS + k) * stride] = e.f[k];
  }
}

template <class T, class Model>
BD_HD void jac_load(JacSink<T, Model>& e, const T* pk, int64_t stride) {
  constexpr int NS = Model::NS, NG = Model::NG, NB = Model::NB;
  for_bits<Model::ROWMASK[0]>([&](auto b) {
    constexpr int c = decltype(b)::value;
    e.jv[c] = pk[c * stride];
  });
#pragma unroll
  for (int g = 1; g <= NG; ++g) {
    e.jgd[g] = pk[(NS + g - 1) * stride];
    e.jgv[g] = pk[(NS + NG + g - 1) * stride];
  }
  auto row = [&](auto rr) {
    constexpr int r = decltype(rr)::value;
    for_bits<Model::ROWMASK[NG + 1 + r]>([&](auto b) {
      constexpr int c = decltype(b)::value;
      e.jb[r][c] = pk[(NS + 2 * NG + r * NS + c) * stride];
    });
  };
  [&]<int... R>(std::integer_sequence<int, R...>) { (row(std::integral_constant<int, R>{}), ...); }
  (std::make_integer_sequence<int, NB>{});
#pragma unroll
  for (int k = 0; k < NS; ++k) e.f[k] = pk[(NS + 2 * NG + NB * NS + k) * stride];
}

// What stage 2 of a ROS2 step needs of stage 1's condensation (same node
// Jacobian, same shift alpha): stage 1 stores it, stage 2 then solves
// A z = rho for its new rho without evaluating the Jacobian again.  Layout per
// node, PACK values (strided by the node count):
//   [0, NG)             1 / (alpha - d g_k / d x_k), gates k = 1..NG
//   [NG, NG + NB NG)    d f_{NG+1+r} / d x_k, block row r, gate k (pattern entries)
//   next NB NB          the block matrix alpha I - J_yy restricted to the block
//   next NS             d f_0 / d X_c (pattern entries)
template <class Model>
constexpr int cond_pack_size() {
  return Model::NG + Model::NB * Model::NG + Model::NB * Model::NB + Model::NS;
}

template <class T, class Model>
BD_HD void cond_store(const JacSink<T, Model>& e, T alpha, T* pk, int64_t stride) {
  constexpr int NG = Model::NG, NB = Model::NB;
  constexpr uint32_t GATES = ((1u << (NG + 1)) - 1u) & ~1u;
#pragma unroll
  for (int g = 1; g <= NG; ++g) pk[(g - 1) * stride] = T(1) / (alpha - e.jgd[g]);
  auto row = [&](auto rr) {
    constexpr int r = decltype(rr)::value;
    constexpr uint32_t RM = Model::ROWMASK[NG + 1 + r];
    for_bits<RM & GATES>([&](auto b) {
      constexpr int c = decltype(b)::value;
      pk[(NG + r * NG + (c - 1)) * stride] = e.jb[r][c];
    });
#pragma unroll
    for (int c = 0; c < NB; ++c) pk[(NG + NB * NG + r * NB + c) * stride] = (r == c) ? alpha : T(0);
    for_bits<(RM >> (NG + 1))>([&](auto b) {
      constexpr int c = decltype(b)::value;
      pk[(NG + NB * NG + r * NB + c) * stride] = ((r == c) ? alpha : T(0)) - e.jb[r][NG + 1 + c];
    });
  };
  [&]<int... R>(std::integer_sequence<int, R...>) { (row(std::integral_constant<int, R>{}), ...); }
  (std::make_integer_sequence<int, NB>{});
  for_bits<Model::ROWMASK[0] & ~1u>([&](auto b) {
    constexpr int c = decltype(b)::value;
    pk[(NG + NB * NG + NB * NB + c) * stride] = e.jv[c];
  });
}

// z = A^-1 rho and corr = sum_c j_vc z_c from a stored pack: the arithmetic of
// condense() for z and corr, operation for operation
template <class T, class Model>
BD_HD void cond_solve(const T* pk, int64_t stride, const T* rho, T& corr, T* z) {
  constexpr int NG = Model::NG, NB = Model::NB;
  constexpr uint32_t GATES = ((1u << (NG + 1)) - 1u) & ~1u;
#pragma unroll
  for (int g = 1; g <= NG; ++g) z[g - 1] = rho[g - 1] * pk[(g - 1) * stride];
  T Bm[NB][NB];
  T rz[NB];
  auto fill = [&](auto rr) {
    constexpr int r = decltype(rr)::value;
    constexpr uint32_t RM = Model::ROWMASK[NG + 1 + r];
    rz[r] = rho[NG + r];
    for_bits<RM & GATES>([&](auto b) {
      constexpr int c = decltype(b)::value;
      rz[r] += pk[(NG + r * NG + (c - 1)) * stride] * z[c - 1];
    });
#pragma unroll
    for (int c = 0; c < NB; ++c) Bm[r][c] = pk[(NG + NB * NG + r * NB + c) * stride];
  };
  [&]<int... R>(std::integer_sequence<int, R...>) { (fill(std::integral_constant<int, R>{}), ...); }
  (std::make_integer_sequence<int, NB>{});
#pragma unroll
  for (int k = 0; k < NB; ++k) {
    const T piv = T(1) / Bm[k][k];
#pragma unroll
    for (int i = k + 1; i < NB; ++i) {
      const T l = Bm[i][k] * piv;
#pragma unroll
      for (int c = k + 1; c < NB; ++c) Bm[i][c] -= l * Bm[k][c];
      rz[i] -= l * rz[k];
    }
  }
#pragma unroll
  for (int i = NB - 1; i >= 0; --i) {
#pragma unroll
    for (int c = i + 1; c < NB; ++c) rz[i] -= Bm[i][c] * rz[c];
    const T inv = T(1) / Bm[i][i];
    rz[i] *= inv;
    z[NG + i] = rz[i];
  }
  corr = T(0);
  for_bits<Model::ROWMASK[0] & ~1u>([&](auto b) {
    constexpr int c = decltype(b)::value;
    corr += pk[(NG + NB * NG + NB * NB + c) * stride] * z[c - 1];
  });
}

}  // namespace bd
