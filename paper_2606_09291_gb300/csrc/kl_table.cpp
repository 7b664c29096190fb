// kl_table.cpp - host construction of the KL mode table (row a2's data).
//
// The random coefficient is exp of a truncated Karhunen-Loeve sum (Sec. 5
// field model).  This workload tensorises the 1D exponential covariance
// C(x, x') = exp(-|x - x'| / l_c) on [0, 1].  With t = x - 1/2 and c = 1/l_c,
// the eigenfunctions are cos(w t) (w tan(w/2) = c) and sin(w t)
// (tan(w/2) = -w / c), eigenvalue 2c / (w^2 + c^2); 1D mode n has w in
// (n pi, (n+1) pi), cosine for even n, sine for odd n.  The K largest products
// lambda_i lambda_j lambda_k are kept; the product is formed from the sorted
// factors so that permutations tie exactly, and ties are broken by (i, j, k)
// ascending.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kl_table.h"

namespace mlsgd {

static double bisect_root(int n, double c) {
  // s = w/2 in (n pi/2, (n+1) pi/2); even: 2 s sin s - c cos s = 0, odd: c sin s + 2 s cos s = 0
  auto f = [&](double s) { return (n % 2 == 0) ? 2.0 * s * std::sin(s) - c * std::cos(s) : c * std::sin(s) + 2.0 * s * std::cos(s); };
  double lo = n * M_PI / 2.0, hi = (n + 1) * M_PI / 2.0;
  double flo = f(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    const double fm = f(mid);
    if (fm == 0.0) return 2.0 * mid;
    if ((fm < 0.0) == (flo < 0.0)) { lo = mid; flo = fm; } else { hi = mid; }
  }
  return 2.0 * 0.5 * (lo + hi);
}

void kl_modes_1d(double corr_len, int n, std::vector<double>& omega, std::vector<double>& lam,
                 std::vector<double>& norm) {
  const double c = 1.0 / corr_len;
  omega.resize(n); lam.resize(n); norm.resize(n);
  for (int m = 0; m < n; ++m) {
    const double w = bisect_root(m, c);
    omega[m] = w;
    lam[m] = 2.0 * c / (w * w + c * c);
    const double sw = std::sin(w) / (2.0 * w);
    norm[m] = 1.0 / std::sqrt(m % 2 == 0 ? 0.5 + sw : 0.5 - sw);
  }
}

double kl_eval_1d(int m, double omega, double norm, double x) {
  const double t = x - 0.5;
  return norm * (m % 2 == 0 ? std::cos(omega * t) : std::sin(omega * t));
}

struct Cand { double key; int i, j, k; };

KLTable build_kl_table(double corr_len, int K) {
  KLTable T;
  int n1d = 4;
  for (;;) {
    kl_modes_1d(corr_len, n1d, T.omega, T.lam1, T.norm);
    std::vector<Cand> cand;
    cand.reserve((size_t)n1d * n1d * n1d);
    for (int i = 0; i < n1d; ++i)
      for (int j = 0; j < n1d; ++j)
        for (int k = 0; k < n1d; ++k) {
          double f[3] = {T.lam1[i], T.lam1[j], T.lam1[k]};
          std::sort(f, f + 3);
          cand.push_back(Cand{(f[0] * f[1]) * f[2], i, j, k});
        }
    std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
      if (a.key != b.key) return a.key > b.key;
      if (a.i != b.i) return a.i < b.i;
      if (a.j != b.j) return a.j < b.j;
      return a.k < b.k;
    });
    int used = 0;
    for (int t = 0; t < K; ++t) used = std::max(used, std::max(cand[t].i, std::max(cand[t].j, cand[t].k)));
    if (used < n1d - 1) {
      T.ix.resize(K); T.iy.resize(K); T.iz.resize(K); T.lam3.resize(K);
      for (int t = 0; t < K; ++t) {
        T.ix[t] = cand[t].i; T.iy[t] = cand[t].j; T.iz[t] = cand[t].k; T.lam3[t] = cand[t].key;
      }
      T.n1d = used + 1;
      T.omega.resize(T.n1d); T.lam1.resize(T.n1d); T.norm.resize(T.n1d);
      return T;
    }
    ++n1d;
  }
}

KLTable build_paper_table(double rho, int m) {
  KLTable T;
  T.model = 1;
  T.n1d = m;
  for (int j = 1; j <= m; ++j)
    for (int k = 1; k <= m; ++k)
      for (int l = 1; l <= m; ++l) {
        // phi_jkl(x) = cos(j pi x2) cos(k pi x3) cos(l pi x1): x-index l, y-index j, z-index k
        T.ix.push_back(l - 1);
        T.iy.push_back(j - 1);
        T.iz.push_back(k - 1);
        T.lam3.push_back(std::exp(-M_PI * (double)(j + k + l) * rho));
      }
  return T;
}

std::vector<double> kl_cell_table(const KLTable& T, int N) {
  std::vector<double> phi((size_t)T.n1d * N);
  for (int m = 0; m < T.n1d; ++m)
    for (int x = 0; x < N; ++x) {
      const double xc = (x + 0.5) / N;
      phi[(size_t)m * N + x] = T.model == 1 ? std::cos((m + 1) * M_PI * xc) : kl_eval_1d(m, T.omega[m], T.norm[m], xc);
    }
  return phi;
}

}  // namespace mlsgd
