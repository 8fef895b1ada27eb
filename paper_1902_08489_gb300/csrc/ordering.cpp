// Fiedler ordering of the orbitals (host).
//
// Sec. 3.2 sorts the molecular orbitals of the MPS calculations along a
// Fiedler vector, which narrows the band of the Hamiltonian matrix (the
// spectral ordering of orbitals known from DMRG): orbitals are vertices
// of a weighted graph, the eigenvector of the graph Laplacian with the
// second smallest eigenvalue (the Fiedler vector) embeds them on a line,
// and sorting by it places strongly coupled orbitals next to each other --
// which keeps the MPO and the entanglement across each bond small.
// Weights: W_ij = |h_ij| + |(ij|ji)| (one-electron coupling plus exchange
// integral) for i != j.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "internal.hpp"

namespace tdmps {

namespace {

// Cyclic Jacobi eigenvalue iteration for a symmetric n x n matrix (row-major,
// overwritten); returns eigenvalues, eigenvectors in the columns of V.
void jacobi_eigen(std::vector<double>& A, int n, std::vector<double>& w, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = 0; q < n; ++q) {
        double a = A[(size_t)p * n + q] * A[(size_t)p * n + q];
        tot += a;
        if (p != q) off += a;
      }
    if (off <= 1e-30 * std::max(tot, 1e-300)) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        // rotation angle that zeroes A[p][q]: tan(2 theta) = 2 apq / (aqq - app)
        const double theta = 0.5 * std::atan2(2.0 * apq, aqq - app);
        const double c = std::cos(theta), s = std::sin(theta);
        for (int k = 0; k < n; ++k) {   // A <- A J (columns p, q)
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {   // A <- J^T A (rows p, q)
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {   // V <- V J
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(n);
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
}

}  // namespace

void fiedler_order(const double* h, const double* eri, int L, int* perm) {
  if (L < 1 || L > 64) throw Error(TDMPS_ERR_INVALID_ARG, "L must be in [1, 64]");
  if (L < 3) {
    for (int i = 0; i < L; ++i) perm[i] = i;
    return;
  }
  const size_t L2 = (size_t)L * L;
  std::vector<double> Lap(L2, 0.0);
  for (int i = 0; i < L; ++i)
    for (int j = 0; j < L; ++j) {
      if (i == j) continue;
      const double hij = h[(size_t)i * L + j];
      const double kij = eri[(((size_t)i * L + j) * L + j) * L + i];   // (ij|ji)
      if (!std::isfinite(hij) || !std::isfinite(kij))
        throw Error(TDMPS_ERR_NONFINITE, "integrals contain NaN/Inf");
      const double w = 0.5 * (std::fabs(hij) + std::fabs(kij)) +
                       0.5 * (std::fabs(h[(size_t)j * L + i]) +
                              std::fabs(eri[(((size_t)j * L + i) * L + i) * L + j]));
      Lap[(size_t)i * L + j] = -w;
      Lap[(size_t)i * L + i] += w;
    }
  std::vector<double> w, V;
  jacobi_eigen(Lap, L, w, V);
  std::vector<int> idx(L);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return w[a] < w[b]; });
  const int f = idx[1];   // second smallest eigenvalue
  std::vector<double> fv(L);
  double corr = 0.0;
  for (int i = 0; i < L; ++i) {
    fv[i] = V[(size_t)i * L + f];
    corr += (i - 0.5 * (L - 1)) * fv[i];
  }
  if (corr < 0.0)   // orientation: keep the original order's direction
    for (auto& x : fv) x = -x;
  std::vector<int> ord(L);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return fv[a] < fv[b]; });
  for (int k = 0; k < L; ++k) perm[k] = ord[k];
}

}  // namespace tdmps
