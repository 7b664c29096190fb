// kl_table.h - host KL mode table of the exponential covariance (see kl_table.cpp).
#pragma once
#include <vector>

namespace mlsgd {

struct KLTable {
  int model = 0;                     // 0 = exponential covariance, 1 = the paper's cos-product field
  int n1d = 0;                       // 1D modes used (max index + 1)
  std::vector<double> omega, lam1, norm;  // 1D eigenpairs
  std::vector<int> ix, iy, iz;       // [K] 1D indices of each selected 3D mode
  std::vector<double> lam3;          // [K] lambda_i lambda_j lambda_k (descending)
};

KLTable build_kl_table(double corr_len, int K);
// the paper's Sec. 5 field: m^3 modes cos(j pi y) cos(k pi z) cos(l pi x), lambda = exp(-pi (j+k+l) rho)
KLTable build_paper_table(double rho, int m);
// phi_m((x + 1/2) / N) for m < n1d, x < N: [n1d][N]
std::vector<double> kl_cell_table(const KLTable& T, int N);

}  // namespace mlsgd
