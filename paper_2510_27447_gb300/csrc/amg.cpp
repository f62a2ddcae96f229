// amg.cpp -- host setup of an aggregation algebraic multigrid hierarchy for the
// elliptic operator A_ie.
//
// The paper preconditions the elliptic solve with an algebraic multigrid
// method built by a greedy aggregation heuristic on the strength of
// connection (Sec. 3.3.2, "AMG preconditioner ... greedy heuristic algorithm
// based on the strength of connection").  This is the smoothed-aggregation
// variant (Vanek, Mandel & Brezina, Computing 56, 1996):
//   strength   j is a strong neighbour of i if |a_ij| >= theta_l sqrt(a_ii a_jj),
//              theta_l = theta 2^-l on level l
//   aggregates greedy: (1) a node whose strong neighbours are all free starts
//              an aggregate with them; (2) remaining nodes join the aggregate
//              of their strongest aggregated neighbour; (3) leftovers start
//              aggregates with their free strong neighbours
//   prolongator P = (I - omega D^-1 A) T, T the aggregate indicator,
//              omega = 4 / (3 rho(D^-1 A)) (rho by power iteration)
//   coarse op  A_c = P^T A P
// until the operator has at most `coarse_max` rows; that last operator is
// singular (A 1 = 0 is preserved: T 1 = 1 and A 1 = 0), so its solve uses the
// dense inverse of A_c + c 1 1^T, which returns the zero-mean solution for any
// right-hand side orthogonal to 1.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <string>
#include <thread>
#include <vector>

#include "bd_internal.h"

namespace bd {

namespace {

template <class F>
void par_rows(int64_t n, F&& fn) {
  const unsigned nt = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  if (n < 4096 || nt == 1) {
    fn(int64_t(0), n);
    return;
  }
  std::vector<std::thread> th;
  const int64_t chunk = (n + nt - 1) / nt;
  for (unsigned t = 0; t < nt; ++t) {
    const int64_t lo = t * chunk, hi = std::min(n, lo + chunk);
    if (lo >= hi) break;
    th.emplace_back([&, lo, hi] { fn(lo, hi); });
  }
  for (auto& x : th) x.join();
}

// C = A * B (row-wise, dense marker accumulator per thread).  Each thread
// writes its rows contiguously into its own arrays (no per-row heap
// blocks); the row pieces are then stitched by row pointer.
HCsr spgemm(const HCsr& A, const HCsr& B) {
  HCsr C;
  C.n = A.n;
  C.m = B.m;
  struct Piece {
    int64_t lo = 0, hi = 0;
    std::vector<int64_t> len;
    std::vector<int32_t> ci;
    std::vector<double> v;
  };
  std::vector<Piece> pieces;
  std::mutex mu;
  par_rows(A.n, [&](int64_t lo, int64_t hi) {
    Piece pc;
    pc.lo = lo;
    pc.hi = hi;
    pc.len.resize(hi - lo);
    std::vector<int64_t> mark(B.m, -1);
    std::vector<double> acc(B.m, 0.0);
    std::vector<int32_t> cols;
    for (int64_t i = lo; i < hi; ++i) {
      cols.clear();
      for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
        const int32_t k = A.ci[p];
        const double a = A.v[p];
        for (int64_t q = B.rp[k]; q < B.rp[k + 1]; ++q) {
          const int32_t j = B.ci[q];
          if (mark[j] != i) {
            mark[j] = i;
            acc[j] = 0.0;
            cols.push_back(j);
          }
          acc[j] += a * B.v[q];
        }
      }
      std::sort(cols.begin(), cols.end());
      pc.len[i - lo] = int64_t(cols.size());
      for (int32_t j : cols) {
        pc.ci.push_back(j);
        pc.v.push_back(acc[j]);
      }
    }
    std::lock_guard<std::mutex> g(mu);
    pieces.push_back(std::move(pc));
  });
  C.rp.assign(A.n + 1, 0);
  for (const Piece& pc : pieces)
    for (int64_t i = pc.lo; i < pc.hi; ++i) C.rp[i + 1] = pc.len[i - pc.lo];
  for (int64_t i = 0; i < A.n; ++i) C.rp[i + 1] += C.rp[i];
  C.ci.resize(C.rp[A.n]);
  C.v.resize(C.rp[A.n]);
  for (const Piece& pc : pieces) {
    std::copy(pc.ci.begin(), pc.ci.end(), C.ci.begin() + C.rp[pc.lo]);
    std::copy(pc.v.begin(), pc.v.end(), C.v.begin() + C.rp[pc.lo]);
  }
  return C;
}

HCsr transpose(const HCsr& A) {
  HCsr T;
  T.n = A.m;
  T.m = A.n;
  T.rp.assign(T.n + 1, 0);
  for (int32_t j : A.ci) T.rp[j + 1]++;
  for (int64_t i = 0; i < T.n; ++i) T.rp[i + 1] += T.rp[i];
  T.ci.resize(A.ci.size());
  T.v.resize(A.v.size());
  std::vector<int64_t> fill(T.rp.begin(), T.rp.end() - 1);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int64_t q = fill[A.ci[p]]++;
      T.ci[q] = int32_t(i);
      T.v[q] = A.v[p];
    }
  return T;
}

std::vector<double> diagonal(const HCsr& A) {
  std::vector<double> d(A.n, 0.0);
  for (int64_t i = 0; i < A.n; ++i)
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (A.ci[p] == i) d[i] = A.v[p];
  return d;
}

// spectral radius of D^-1 A by power iteration (deterministic start vector)
double rho_dinv_a(const HCsr& A, const std::vector<double>& d, int iters) {
  std::vector<double> x(A.n), y(A.n);
  for (int64_t i = 0; i < A.n; ++i) x[i] = 1.0 + 0.37 * std::sin(1.3 * double(i) + 0.2) + ((i & 1) ? 0.5 : -0.5);
  double lam = 0.0;
  for (int it = 0; it < iters; ++it) {
    double nrm = 0.0;
    for (int64_t i = 0; i < A.n; ++i) nrm += x[i] * x[i];
    nrm = std::sqrt(nrm);
    if (!(nrm > 0)) break;
    for (auto& v : x) v /= nrm;
    par_rows(A.n, [&](int64_t lo, int64_t hi) {   // rows are independent; the sums below stay serial
      for (int64_t i = lo; i < hi; ++i) {
        double s = 0.0;
        for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) s += A.v[p] * x[A.ci[p]];
        y[i] = s / d[i];
      }
    });
    double num = 0.0;
    for (int64_t i = 0; i < A.n; ++i) num += x[i] * y[i];
    lam = num;
    x.swap(y);
  }
  // Rayleigh quotients approach rho from below; a small margin keeps the
  // smoother and the prolongator damping on the safe side
  return 1.05 * lam;
}

std::vector<int32_t> aggregate(const HCsr& A, const std::vector<double>& d, double theta, int64_t* n_agg) {
  const int64_t n = A.n;
  std::vector<uint8_t> strong(A.ci.size(), 0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      const int64_t j = A.ci[p];
      if (j != i && std::fabs(A.v[p]) >= theta * std::sqrt(std::fabs(d[i] * d[j]))) strong[p] = 1;
    }
  std::vector<int32_t> agg(n, -1);
  int32_t na = 0;
  // pass 1: nodes whose strong neighbourhood is entirely free
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    bool free_nb = true, any = false;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (strong[p]) {
        any = true;
        if (agg[A.ci[p]] >= 0) {
          free_nb = false;
          break;
        }
      }
    if (!free_nb || !any) continue;
    agg[i] = na;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (strong[p]) agg[A.ci[p]] = na;
    ++na;
  }
  // pass 2: join the strongest aggregated neighbour (decided from pass-1 state)
  std::vector<int32_t> agg1 = agg;
  for (int64_t i = 0; i < n; ++i) {
    if (agg1[i] >= 0) continue;
    double best = -1.0;
    int32_t b = -1;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (strong[p] && agg1[A.ci[p]] >= 0 && std::fabs(A.v[p]) > best) {
        best = std::fabs(A.v[p]);
        b = agg1[A.ci[p]];
      }
    if (b >= 0) agg[i] = b;
  }
  // pass 3: leftovers form aggregates with their free strong neighbours
  for (int64_t i = 0; i < n; ++i) {
    if (agg[i] >= 0) continue;
    agg[i] = na;
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p)
      if (strong[p] && agg[A.ci[p]] < 0) agg[A.ci[p]] = na;
    ++na;
  }
  *n_agg = na;
  return agg;
}

// dense Cholesky of an SPD matrix and its explicit inverse (row-major n x n)
bool dense_spd_inverse(std::vector<double>& a, int64_t n, std::vector<double>* inv) {
  for (int64_t j = 0; j < n; ++j) {
    double s = a[j * n + j];
    for (int64_t k = 0; k < j; ++k) s -= a[j * n + k] * a[j * n + k];
    if (!(s > 0)) return false;
    const double l = std::sqrt(s);
    a[j * n + j] = l;
    for (int64_t i = j + 1; i < n; ++i) {
      double t = a[i * n + j];
      for (int64_t k = 0; k < j; ++k) t -= a[i * n + k] * a[j * n + k];
      a[i * n + j] = t / l;
    }
  }
  // column c of the inverse: L y = e_c (y_i = 0 for i < c), then L^T x = y.
  // L^T is stored row-major so that the backward substitution reads rows;
  // columns are independent and split over threads.
  std::vector<double> lt(size_t(n * n), 0.0);
  for (int64_t i = 0; i < n; ++i)
    for (int64_t k = 0; k <= i; ++k) lt[k * n + i] = a[i * n + k];
  inv->assign(size_t(n * n), 0.0);
  auto columns = [&](int64_t t0, int64_t step) {
    std::vector<double> y(n, 0.0), x(n);
    for (int64_t c = t0; c < n; c += step) {
      for (int64_t i = c; i < n; ++i) {
        double t = (i == c) ? 1.0 : 0.0;
        for (int64_t k = c; k < i; ++k) t -= a[i * n + k] * y[k];
        y[i] = t / a[i * n + i];
      }
      for (int64_t i = n - 1; i >= 0; --i) {
        double t = i >= c ? y[i] : 0.0;
        for (int64_t k = i + 1; k < n; ++k) t -= lt[i * n + k] * x[k];
        x[i] = t / a[i * n + i];
      }
      for (int64_t i = 0; i < n; ++i) (*inv)[i * n + c] = x[i];
    }
  };
  const int64_t nt = std::max<int64_t>(1, std::min<int64_t>({32, int64_t(std::thread::hardware_concurrency()), n / 64}));
  std::vector<std::thread> th;
  // columns dealt round-robin (the forward pass of column c costs (n - c)^2 / 2)
  for (int64_t t = 0; t < nt; ++t) th.emplace_back(columns, t, nt);
  for (auto& x : th) x.join();
  return true;
}

}  // namespace

int amg_build(const HCsr& A0, const AmgParams& prm, AmgHost* out, std::string* err) {
  out->lev.clear();
  HCsr A = A0;
  while (A.n > prm.coarse_max && int(out->lev.size()) < prm.max_levels) {
    AmgHostLevel L;
    const std::vector<double> d = diagonal(A);
    for (int64_t i = 0; i < A.n; ++i)
      if (!(d[i] > 0)) {
        *err = "AMG: non-positive diagonal";
        return BD_ERR_ARG;
      }
    const double rho = rho_dinv_a(A, d, 30);
    int64_t nc = 0;
    // the strength threshold halves per level (Vanek, Mandel & Brezina): the
    // smoothed coarse operators spread their weight over many small entries,
    // and a fixed threshold leaves ~2 strong neighbours per row there --
    // aggregates of two and an exploding operator complexity
    const double theta = prm.theta * std::ldexp(1.0, -int(out->lev.size()));
    const std::vector<int32_t> agg = aggregate(A, d, theta, &nc);
    if (nc >= A.n) break;   // no coarsening possible
    // P = (I - w D^-1 A) T
    const double w = 4.0 / (3.0 * rho);
    HCsr P;
    P.n = A.n;
    P.m = nc;
    P.rp.assign(A.n + 1, 0);
    {
      // rows built per thread into contiguous pieces, then stitched
      struct Piece {
        int64_t lo = 0, hi = 0;
        std::vector<int64_t> len;
        std::vector<int32_t> ci;
        std::vector<double> v;
      };
      std::vector<Piece> pieces;
      std::mutex mu;
      par_rows(A.n, [&](int64_t lo, int64_t hi) {
        Piece pc;
        pc.lo = lo;
        pc.hi = hi;
        pc.len.resize(hi - lo);
        std::vector<int32_t> cols;
        std::vector<double> vals;
        std::vector<size_t> ord;
        for (int64_t i = lo; i < hi; ++i) {
          cols.clear();
          vals.clear();
          auto add = [&](int32_t c, double v) {
            for (size_t t = 0; t < cols.size(); ++t)
              if (cols[t] == c) {
                vals[t] += v;
                return;
              }
            cols.push_back(c);
            vals.push_back(v);
          };
          add(agg[i], 1.0);
          for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) add(agg[A.ci[p]], -w * A.v[p] / d[i]);
          ord.resize(cols.size());
          std::iota(ord.begin(), ord.end(), 0);
          std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return cols[x] < cols[y]; });
          pc.len[i - lo] = int64_t(cols.size());
          for (size_t t : ord) {
            pc.ci.push_back(cols[t]);
            pc.v.push_back(vals[t]);
          }
        }
        std::lock_guard<std::mutex> g(mu);
        pieces.push_back(std::move(pc));
      });
      for (const Piece& pc : pieces)
        for (int64_t i = pc.lo; i < pc.hi; ++i) P.rp[i + 1] = pc.len[i - pc.lo];
      for (int64_t i = 0; i < A.n; ++i) P.rp[i + 1] += P.rp[i];
      P.ci.resize(P.rp[A.n]);
      P.v.resize(P.rp[A.n]);
      for (const Piece& pc : pieces) {
        std::copy(pc.ci.begin(), pc.ci.end(), P.ci.begin() + P.rp[pc.lo]);
        std::copy(pc.v.begin(), pc.v.end(), P.v.begin() + P.rp[pc.lo]);
      }
    }
    HCsr R = transpose(P);
    HCsr Ac = spgemm(R, spgemm(A, P));
    L.invdiag.resize(A.n);
    for (int64_t i = 0; i < A.n; ++i) L.invdiag[i] = 1.0 / d[i];
    L.omega = 4.0 / (3.0 * rho);
    L.A = std::move(A);
    L.P = std::move(P);
    L.R = std::move(R);
    out->lev.push_back(std::move(L));
    A = std::move(Ac);
  }
  // coarsest operator: dense inverse of A_c + c 1 1^T
  const int64_t n = A.n;
  if (n > 4096) {
    *err = "AMG: coarsest level too large for a dense solve";
    return BD_ERR_ARG;
  }
  std::vector<double> dense(n * n, 0.0);
  double dmean = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t p = A.rp[i]; p < A.rp[i + 1]; ++p) {
      dense[i * n + A.ci[p]] += A.v[p];
      if (A.ci[p] == i) dmean += A.v[p];
    }
  dmean /= double(std::max<int64_t>(n, 1));
  const double c = dmean / double(std::max<int64_t>(n, 1));
  for (auto& x : dense) x += c;
  if (!dense_spd_inverse(dense, n, &out->cinv)) {
    *err = "AMG: coarsest operator is not positive definite";
    return BD_ERR_ARG;
  }
  out->nc = n;
  return BD_OK;
}

}  // namespace bd

namespace bd {

SellHost sell_from_csr(const HCsr& A, int wide) {
  SellHost S;
  S.n = A.n;
  int64_t maxw = 0;
  for (int64_t i = 0; i < A.n; ++i) maxw = std::max(maxw, A.rp[i + 1] - A.rp[i]);
  bool sell_wide = false;
  if (maxw > 32 && wide > 0) {
    // rows longer than 32 stay SELL-32 (thread per row, loads coalesced
    // across the slice) when padding every slice to its longest row stores
    // at most half again the entries and (wide == 1) the operator has many
    // moderate rows -- measured on the 3-D slab: R_0 (210k rows of 49
    // entries) and A_1 (210k rows of 74) run 1.4-1.8x faster than as CSR,
    // while operators of 14k rows of 230 entries run 5-25x slower (too few
    // threads, long chains)
    int64_t padded = 0;
    for (int64_t sl = 0; sl * 32 < A.n; ++sl) {
      int64_t w = 0;
      for (int64_t i = sl * 32; i < std::min<int64_t>(A.n, sl * 32 + 32); ++i) w = std::max(w, A.rp[i + 1] - A.rp[i]);
      padded += 32 * w;
    }
    const int64_t nnz = A.rp[A.n];
    sell_wide = 2 * padded <= 3 * nnz && (wide == 2 || (nnz <= 96 * A.n && A.n >= (int64_t(1) << 17)));
  }
  if (maxw > 32 && !sell_wide) {
    // long rows (coarse operators, restrictions in 3-D): CSR, one warp per row
    S.rp = A.rp;
    S.col.assign(A.ci.begin(), A.ci.end());
    S.val = A.v;
    S.wmax = -1;
    return S;
  }
  const int64_t nsl = (A.n + 31) / 32;
  S.sptr.resize(nsl);
  S.sw.resize(nsl);
  int64_t off = 0;
  for (int64_t sl = 0; sl < nsl; ++sl) {
    int w = 0;
    for (int64_t i = sl * 32; i < std::min<int64_t>(A.n, sl * 32 + 32); ++i)
      w = std::max<int>(w, int(A.rp[i + 1] - A.rp[i]));
    S.sw[sl] = w;
    S.sptr[sl] = off;
    off += 32 * int64_t(w);
  }
  S.col.assign(off, 0);
  S.val.assign(off, 0.0);
  for (int64_t i = 0; i < A.n; ++i) {
    const int64_t base = S.sptr[i / 32] + (i % 32);
    for (int64_t k = 0; k < A.rp[i + 1] - A.rp[i]; ++k) {
      S.col[base + 32 * k] = A.ci[A.rp[i] + k];
      S.val[base + 32 * k] = A.v[A.rp[i] + k];
    }
  }
  S.wmax = maxw <= 8 ? 8 : maxw <= 16 ? 16 : maxw <= 32 ? 32 : 0;   // 0: wide (streaming kernels only)
  return S;
}

}  // namespace bd
