// sd.cuh -- compile-time sparse forward-mode derivatives.
//
// The paper stores the local Jacobian block of every node as a compile-time
// sparse matrix (CTSM, Sec. 3.3.2).  Here the same idea is applied to the
// evaluation itself: SD<T, MASK> carries a value and the partial derivatives
// with respect to the node's state variables whose bits are set in MASK.
// MASK is a template parameter, so the sparsity of every intermediate is
// known to the compiler: an operation touches only the union of its
// operands' masks and never multiplies by a structural zero.  The model code
// reads like the plain formulas of the cell model and yields the exact
// Jacobian ("exact derivatives", Sec. 3.3.2) as a by-product.
#pragma once
#include <cstdint>
#include <type_traits>

#ifndef BD_HD
#define BD_HD __host__ __device__ __forceinline__
#endif

namespace bd {

namespace sdm {
constexpr int popc(uint32_t m) { int c = 0; while (m) { c += int(m & 1u); m >>= 1; } return c; }
constexpr int ctz(uint32_t m) { int c = 0; while (m && !(m & 1u)) { m >>= 1; ++c; } return c; }
constexpr int pos(uint32_t m, int bit) { return popc(m & ((1u << bit) - 1u)); }
constexpr bool has(uint32_t m, int bit) { return ((m >> bit) & 1u) != 0u; }
}  // namespace sdm

// Call f(integral_constant<int, b>) for every set bit b of M, in increasing order.
template <uint32_t M, class F>
BD_HD void for_bits(F&& f) {
  if constexpr (M != 0u) {
    f(std::integral_constant<int, sdm::ctz(M)>{});
    for_bits<M & (M - 1u)>(f);
  }
}

template <class T, uint32_t MASK>
struct SD {
  static constexpr uint32_t mask = MASK;
  static constexpr int nnz = sdm::popc(MASK);
  T v;
  T d[nnz > 0 ? nnz : 1];

  // partial derivative with respect to state variable BIT (0 if structurally zero)
  template <int BIT>
  BD_HD T der() const {
    if constexpr (sdm::has(MASK, BIT)) return d[sdm::pos(MASK, BIT)];
    else return T(0);
  }
};

template <class T> using SC = SD<T, 0u>;   // constant

// independent variable number BIT with value x
template <int BIT, class T>
BD_HD SD<T, (1u << BIT)> var(T x) {
  SD<T, (1u << BIT)> r;
  r.v = x;
  r.d[0] = T(1);
  return r;
}

template <class T>
BD_HD SC<T> cst(T x) { SC<T> r; r.v = x; return r; }

// r = f(a) with f'(a) = df  (chain rule)
template <class T, uint32_t A>
BD_HD SD<T, A> chain(const SD<T, A>& a, T f, T df) {
  SD<T, A> r;
  r.v = f;
  for_bits<A>([&](auto b) { constexpr int k = sdm::pos(A, decltype(b)::value); r.d[k] = df * a.d[k]; });
  return r;
}

// ---- binary arithmetic ----------------------------------------------------
template <class T, uint32_t A, uint32_t B>
BD_HD SD<T, A | B> operator+(const SD<T, A>& a, const SD<T, B>& b) {
  constexpr uint32_t C = A | B;
  SD<T, C> r;
  r.v = a.v + b.v;
  for_bits<C>([&](auto bb) {
    constexpr int bit = decltype(bb)::value;
    constexpr int k = sdm::pos(C, bit);
    if constexpr (sdm::has(A, bit) && sdm::has(B, bit)) r.d[k] = a.d[sdm::pos(A, bit)] + b.d[sdm::pos(B, bit)];
    else if constexpr (sdm::has(A, bit)) r.d[k] = a.d[sdm::pos(A, bit)];
    else r.d[k] = b.d[sdm::pos(B, bit)];
  });
  return r;
}

template <class T, uint32_t A>
BD_HD SD<T, A> operator-(const SD<T, A>& a) {
  SD<T, A> r;
  r.v = -a.v;
  for_bits<A>([&](auto b) { constexpr int k = sdm::pos(A, decltype(b)::value); r.d[k] = -a.d[k]; });
  return r;
}

template <class T, uint32_t A, uint32_t B>
BD_HD SD<T, A | B> operator-(const SD<T, A>& a, const SD<T, B>& b) {
  constexpr uint32_t C = A | B;
  SD<T, C> r;
  r.v = a.v - b.v;
  for_bits<C>([&](auto bb) {
    constexpr int bit = decltype(bb)::value;
    constexpr int k = sdm::pos(C, bit);
    if constexpr (sdm::has(A, bit) && sdm::has(B, bit)) r.d[k] = a.d[sdm::pos(A, bit)] - b.d[sdm::pos(B, bit)];
    else if constexpr (sdm::has(A, bit)) r.d[k] = a.d[sdm::pos(A, bit)];
    else r.d[k] = -b.d[sdm::pos(B, bit)];
  });
  return r;
}

template <class T, uint32_t A, uint32_t B>
BD_HD SD<T, A | B> operator*(const SD<T, A>& a, const SD<T, B>& b) {
  constexpr uint32_t C = A | B;
  SD<T, C> r;
  r.v = a.v * b.v;
  for_bits<C>([&](auto bb) {
    constexpr int bit = decltype(bb)::value;
    constexpr int k = sdm::pos(C, bit);
    if constexpr (sdm::has(A, bit) && sdm::has(B, bit))
      r.d[k] = a.d[sdm::pos(A, bit)] * b.v + a.v * b.d[sdm::pos(B, bit)];
    else if constexpr (sdm::has(A, bit)) r.d[k] = a.d[sdm::pos(A, bit)] * b.v;
    else r.d[k] = a.v * b.d[sdm::pos(B, bit)];
  });
  return r;
}

template <class T, uint32_t A, uint32_t B>
BD_HD SD<T, A | B> operator/(const SD<T, A>& a, const SD<T, B>& b) {
  constexpr uint32_t C = A | B;
  SD<T, C> r;
  const T inv = T(1) / b.v;
  r.v = a.v * inv;
  for_bits<C>([&](auto bb) {
    constexpr int bit = decltype(bb)::value;
    constexpr int k = sdm::pos(C, bit);
    if constexpr (sdm::has(A, bit) && sdm::has(B, bit))
      r.d[k] = (a.d[sdm::pos(A, bit)] - r.v * b.d[sdm::pos(B, bit)]) * inv;
    else if constexpr (sdm::has(A, bit)) r.d[k] = a.d[sdm::pos(A, bit)] * inv;
    else r.d[k] = -r.v * b.d[sdm::pos(B, bit)] * inv;
  });
  return r;
}

// ---- mixed with plain scalars -------------------------------------------
template <class T, uint32_t A> BD_HD SD<T, A> operator+(const SD<T, A>& a, T c) { SD<T, A> r = a; r.v += c; return r; }
template <class T, uint32_t A> BD_HD SD<T, A> operator+(T c, const SD<T, A>& a) { SD<T, A> r = a; r.v += c; return r; }
template <class T, uint32_t A> BD_HD SD<T, A> operator-(const SD<T, A>& a, T c) { SD<T, A> r = a; r.v -= c; return r; }
template <class T, uint32_t A> BD_HD SD<T, A> operator-(T c, const SD<T, A>& a) {
  SD<T, A> r = -a; r.v += c; return r;
}
template <class T, uint32_t A> BD_HD SD<T, A> operator*(const SD<T, A>& a, T c) {
  SD<T, A> r;
  r.v = a.v * c;
  for_bits<A>([&](auto b) { constexpr int k = sdm::pos(A, decltype(b)::value); r.d[k] = a.d[k] * c; });
  return r;
}
template <class T, uint32_t A> BD_HD SD<T, A> operator*(T c, const SD<T, A>& a) { return a * c; }
template <class T, uint32_t A> BD_HD SD<T, A> operator/(const SD<T, A>& a, T c) { return a * (T(1) / c); }
template <class T, uint32_t A> BD_HD SD<T, A> operator/(T c, const SD<T, A>& a) {
  const T inv = T(1) / a.v;
  const T f = c * inv;
  return chain(a, f, -f * inv);
}

}  // namespace bd
