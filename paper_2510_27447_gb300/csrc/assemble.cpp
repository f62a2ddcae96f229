// assemble.cpp -- host P1 assembly of the bidomain operators (runs once per
// handle, before the device path).
//
// Sec. 3.2, Eqs. (3.6)-(3.9): stiffness matrices
//   A_i = ((sigma_i grad w_a, grad w_b)),  A_ie = (((sigma_i + sigma_e) grad w_a, grad w_b)),
// and mass M = ((w_a, w_b)) for piecewise linear w on triangles (2-D) or
// tetrahedra (3-D).  The conductivity of an element is the transversely
// isotropic tensor sigma = s_t I + (s_l - s_t) f f^T of its fibre f.  Both
// stiffness matrices are divided by chi*C_m (the parabolic equation is
// written per unit membrane capacitance).  All three share one CSR pattern:
// the node graph of the mesh.
//
// Bidomain-bath coupling: a bath element contributes sigma_b I to A_ie only
// (no intracellular space, no membrane), so A_i, M and M_L vanish on the bath
// nodes and u is continuous across the interface with the normal currents in
// balance (the natural interface conditions of the weak form).
//
// Rows are assembled independently from a node -> element adjacency, so
// threads own disjoint rows and need no atomics.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "bd_internal.h"

namespace bd {

namespace {

struct ElemGeom {
  double meas;           // area / volume
  double g[4][3];        // gradients of the barycentric functions
};

bool elem_geom(int dim, const double* xyz, const int32_t* e, ElemGeom* out) {
  const int k = dim + 1;
  double Bm[3][3] = {{0}};
  for (int c = 0; c < dim; ++c)
    for (int r = 0; r < dim; ++r) Bm[r][c] = xyz[int64_t(e[c + 1]) * dim + r] - xyz[int64_t(e[0]) * dim + r];
  double inv[3][3];
  double det;
  if (dim == 2) {
    det = Bm[0][0] * Bm[1][1] - Bm[0][1] * Bm[1][0];
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = Bm[1][1] / det;  inv[0][1] = -Bm[0][1] / det;
    inv[1][0] = -Bm[1][0] / det; inv[1][1] = Bm[0][0] / det;
    out->meas = std::fabs(det) / 2.0;
  } else {
    det = Bm[0][0] * (Bm[1][1] * Bm[2][2] - Bm[1][2] * Bm[2][1]) -
          Bm[0][1] * (Bm[1][0] * Bm[2][2] - Bm[1][2] * Bm[2][0]) +
          Bm[0][2] * (Bm[1][0] * Bm[2][1] - Bm[1][1] * Bm[2][0]);
    if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) return false;
    inv[0][0] = (Bm[1][1] * Bm[2][2] - Bm[1][2] * Bm[2][1]) / det;
    inv[0][1] = (Bm[0][2] * Bm[2][1] - Bm[0][1] * Bm[2][2]) / det;
    inv[0][2] = (Bm[0][1] * Bm[1][2] - Bm[0][2] * Bm[1][1]) / det;
    inv[1][0] = (Bm[1][2] * Bm[2][0] - Bm[1][0] * Bm[2][2]) / det;
    inv[1][1] = (Bm[0][0] * Bm[2][2] - Bm[0][2] * Bm[2][0]) / det;
    inv[1][2] = (Bm[0][2] * Bm[1][0] - Bm[0][0] * Bm[1][2]) / det;
    inv[2][0] = (Bm[1][0] * Bm[2][1] - Bm[1][1] * Bm[2][0]) / det;
    inv[2][1] = (Bm[0][1] * Bm[2][0] - Bm[0][0] * Bm[2][1]) / det;
    inv[2][2] = (Bm[0][0] * Bm[1][1] - Bm[0][1] * Bm[1][0]) / det;
    out->meas = std::fabs(det) / 6.0;
  }
  // row a of inv is grad(lambda_{a+1}); lambda_0 = 1 - sum
  for (int d = 0; d < dim; ++d) {
    double s = 0.0;
    for (int a = 0; a < dim; ++a) {
      out->g[a + 1][d] = inv[a][d];
      s += inv[a][d];
    }
    out->g[0][d] = -s;
  }
  (void)k;
  return true;
}

}  // namespace

int assemble_host(const bd_mesh_t* mesh, const bd_cond_t* cond, HostOps* out, std::string* err) {
  const int dim = mesh->dim;
  const int64_t N = mesh->n_nodes, E = mesh->n_elems;
  const int k = dim + 1;
  if (N > int64_t(0x7fffffff) - 1) {
    *err = "mesh too large for 32-bit indices";
    return BD_ERR_ARG;
  }
  for (int64_t i = 0; i < N * dim; ++i)
    if (!std::isfinite(mesh->xyz[i])) {
      *err = "non-finite node coordinate";
      return BD_ERR_ARG;
    }
  for (int64_t e = 0; e < E * k; ++e)
    if (mesh->elems[e] < 0 || mesh->elems[e] >= N) {
      *err = "element node index out of range";
      return BD_ERR_ARG;
    }
  // node -> element adjacency
  std::vector<int64_t> nep(N + 1, 0);
  for (int64_t e = 0; e < E * k; ++e) nep[mesh->elems[e] + 1]++;
  for (int64_t i = 0; i < N; ++i) nep[i + 1] += nep[i];
  std::vector<int64_t> nel(nep[N]);
  {
    std::vector<int64_t> fill(nep.begin(), nep.end() - 1);
    for (int64_t e = 0; e < E; ++e)
      for (int a = 0; a < k; ++a) nel[fill[mesh->elems[e * k + a]]++] = e;
  }
  // element geometry and conductivity tensors are recomputed wherever an
  // element is used (once per node of it) instead of being stored: for meshes
  // of tens of millions of elements the stored form would need ~250 bytes per
  // element of host memory.  A first pass only validates.
  const double scale = 1.0 / (cond->chi * cond->cm);
  const uint8_t* bath = mesh->elem_bath;
  // tissue nodes: the nodes of the tissue elements, numbered first
  out->n_tissue = N;
  if (bath) {
    if (!(cond->sbath > 0.0) || !std::isfinite(cond->sbath)) {
      *err = "a mesh with bath elements needs sbath > 0";
      return BD_ERR_ARG;
    }
    std::vector<uint8_t> tis(N, 0);
    for (int64_t e = 0; e < E; ++e)
      if (!bath[e])
        for (int a = 0; a < k; ++a) tis[mesh->elems[e * k + a]] = 1;
    int64_t nt = 0;
    while (nt < N && tis[nt]) ++nt;
    for (int64_t i = nt; i < N; ++i)
      if (tis[i]) {
        *err = "tissue nodes must be numbered before bath nodes";
        return BD_ERR_ARG;
      }
    if (nt < 1) {
      *err = "the mesh has no tissue element";
      return BD_ERR_ARG;
    }
    out->n_tissue = nt;
  }
  unsigned nthreads = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<int> bad(nthreads, 0);
  auto par = [&](int64_t total, auto&& fn) {
    std::vector<std::thread> th;
    const int64_t chunk = (total + nthreads - 1) / nthreads;
    for (unsigned t = 0; t < nthreads; ++t) {
      const int64_t lo = t * chunk, hi = std::min(total, lo + chunk);
      if (lo >= hi) break;
      th.emplace_back([&, lo, hi, t] { fn(lo, hi, t); });
    }
    for (auto& x : th) x.join();
  };
  // geometry and the intra- / total conductivity tensors of element e;
  // returns 0, 1 (degenerate element) or 2 (bad fibre)
  auto element = [&](int64_t e, ElemGeom* G, double* Si, double* Sie) -> int {
    if (!elem_geom(dim, mesh->xyz, mesh->elems + e * k, G)) return 1;
    double f[3] = {1.0, 0.0, 0.0};
    if (mesh->fiber) {
      double nrm = 0.0;
      for (int d = 0; d < dim; ++d) {
        f[d] = mesh->fiber[e * dim + d];
        nrm += f[d] * f[d];
      }
      nrm = std::sqrt(nrm);
      if (!(nrm > 0.0) || !std::isfinite(nrm)) return 2;
      for (int d = 0; d < dim; ++d) f[d] /= nrm;
    }
    const bool b = bath && bath[e];
    for (int r = 0; r < dim; ++r)
      for (int c = 0; c < dim; ++c) {
        const double ff = f[r] * f[c], id = (r == c) ? 1.0 : 0.0;
        Si[r * 3 + c] = b ? 0.0 : cond->sit * id + (cond->sil - cond->sit) * ff;
        Sie[r * 3 + c] = b ? cond->sbath * id
                           : (cond->sit + cond->set) * id + ((cond->sil + cond->sel) - (cond->sit + cond->set)) * ff;
      }
    return 0;
  };
  par(E, [&](int64_t lo, int64_t hi, unsigned t) {
    ElemGeom G;
    double Si[9], Sie[9];
    for (int64_t e = lo; e < hi && !bad[t]; ++e) bad[t] = element(e, &G, Si, Sie);
  });
  for (int b : bad)
    if (b) {
      *err = b == 1 ? "degenerate element (zero or non-finite measure)" : "zero or non-finite fibre vector";
      return BD_ERR_ARG;
    }
  // CSR pattern: sorted union of the element neighbours of each node
  out->n = N;
  out->rowptr.assign(N + 1, 0);
  // each thread writes its rows' columns contiguously into its own piece
  // (no per-row heap blocks), the pieces are stitched by row pointer
  std::vector<std::vector<int32_t>> piece(nthreads);
  std::vector<int64_t> piece_lo(nthreads, 0);
  par(N, [&](int64_t lo, int64_t hi, unsigned t) {
    std::vector<int32_t> tmp;
    std::vector<int32_t>& pc = piece[t];
    piece_lo[t] = lo;
    for (int64_t i = lo; i < hi; ++i) {
      tmp.clear();
      for (int64_t q = nep[i]; q < nep[i + 1]; ++q)
        for (int a = 0; a < k; ++a) tmp.push_back(mesh->elems[nel[q] * k + a]);
      std::sort(tmp.begin(), tmp.end());
      tmp.erase(std::unique(tmp.begin(), tmp.end()), tmp.end());
      out->rowptr[i + 1] = int32_t(tmp.size());
      pc.insert(pc.end(), tmp.begin(), tmp.end());
    }
  });
  for (int64_t i = 0; i < N; ++i) out->rowptr[i + 1] += out->rowptr[i];
  const int64_t nnz = out->rowptr[N];
  out->col.resize(nnz);
  for (unsigned t = 0; t < nthreads; ++t)
    if (!piece[t].empty()) std::copy(piece[t].begin(), piece[t].end(), out->col.begin() + out->rowptr[piece_lo[t]]);
  piece.clear();
  out->Ai.assign(nnz, 0.0);
  out->Aie.assign(nnz, 0.0);
  out->M.assign(nnz, 0.0);
  out->ML.assign(N, 0.0);
  out->diagpos.assign(N, 0);
  const double mdiag = dim == 2 ? 2.0 / 12.0 : 2.0 / 20.0;
  const double moff = dim == 2 ? 1.0 / 12.0 : 1.0 / 20.0;
  par(N, [&](int64_t lo, int64_t hi, unsigned) {
    for (int64_t i = lo; i < hi; ++i) {
      const int64_t r0 = out->rowptr[i];
      const int32_t* const cb = out->col.data() + r0;
      const int32_t* const ce = out->col.data() + out->rowptr[i + 1];
      out->diagpos[i] = int32_t(r0 + (std::lower_bound(cb, ce, int32_t(i)) - cb));
      ElemGeom G;
      double Si[9], Sie[9];
      for (int64_t q = nep[i]; q < nep[i + 1]; ++q) {
        const int64_t e = nel[q];
        const int32_t* en = mesh->elems + e * k;
        int la = 0;
        while (en[la] != i) ++la;
        element(e, &G, Si, Sie);
        for (int b = 0; b < k; ++b) {
          const int64_t p = r0 + (std::lower_bound(cb, ce, en[b]) - cb);
          double si = 0.0, sie = 0.0;
          for (int r = 0; r < dim; ++r)
            for (int c = 0; c < dim; ++c) {
              const double gg = G.g[la][r] * G.g[b][c];
              si += gg * Si[r * 3 + c];
              sie += gg * Sie[r * 3 + c];
            }
          out->Ai[p] += G.meas * si * scale;
          out->Aie[p] += G.meas * sie * scale;
          if (!(bath && bath[e])) out->M[p] += G.meas * (la == b ? mdiag : moff);
        }
      }
      double ml = 0.0;
      for (int64_t p = r0; p < out->rowptr[i + 1]; ++p) ml += out->M[p];
      out->ML[i] = ml;
    }
  });
  return BD_OK;
}

}  // namespace bd
