// Rotational (rigid-body) primal constraints of an interface class: the
// near-null space of elasticity taken into the BDDC primal space (Section 4).
// Host code only.
#pragma once
#include <cmath>
#include <vector>

namespace cbddc {

// Principal moments below this fraction of the largest give no constraint
// (the axis of a straight edge: rotating about it moves no node of the edge).
constexpr double kRigidDrop = 1e-8;

// Eigen-decomposition of a symmetric 3x3 matrix by cyclic Jacobi rotations:
// on return lam[k] is an eigenvalue and column k of V its unit eigenvector.
inline void sym3_eigen(const double A[3][3], double lam[3], double V[3][3]) {
  double M[3][3], W[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      M[i][j] = A[i][j];
      V[i][j] = i == j ? 1.0 : 0.0;
    }
  static const int PQ[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 64; ++sweep) {
    const double off = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
    const double dia = M[0][0] * M[0][0] + M[1][1] * M[1][1] + M[2][2] * M[2][2];
    if (off == 0.0 || off <= 1e-34 * dia) break;
    for (const auto& pq : PQ) {
      const int p = pq[0], q = pq[1];
      if (M[p][q] == 0.0) continue;
      // J = identity except J_pp = J_qq = c, J_pq = s, J_qp = -s; the
      // (p, q) entry of J^T M J is (c^2 - s^2) M_pq + c s (M_pp - M_qq),
      // zero for t = s / c the smaller root of t^2 + 2 theta t - 1 = 0
      const double theta = (M[q][q] - M[p][p]) / (2.0 * M[p][q]);
      const double t = (theta >= 0.0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
      const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
      double J[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      J[p][p] = c; J[q][q] = c; J[p][q] = s; J[q][p] = -s;
      for (int i = 0; i < 3; ++i)          // W = M J
        for (int j = 0; j < 3; ++j) W[i][j] = M[i][0] * J[0][j] + M[i][1] * J[1][j] + M[i][2] * J[2][j];
      for (int i = 0; i < 3; ++i)          // M = J^T W
        for (int j = 0; j < 3; ++j) M[i][j] = J[0][i] * W[0][j] + J[1][i] * W[1][j] + J[2][i] * W[2][j];
      M[p][q] = M[q][p] = 0.0;
      for (int i = 0; i < 3; ++i) {        // V = V J
        const double vp = V[i][p], vq = V[i][q];
        V[i][p] = c * vp - s * vq;
        V[i][q] = s * vp + c * vq;
      }
    }
  }
  for (int k = 0; k < 3; ++k) lam[k] = M[k][k];
}

// Rotational constraints of the class with the given nodes (coordinates X,
// 3 per node): the rotations y -> v x y about the class centroid (y = x -
// xbar) along the principal axes v of the class, i.e. the eigenvectors of
// its inertia tensor M = sum_a (|y_a|^2 I - y_a y_a^T).  Since
// sum_a |v x y_a|^2 = v^T M v, each row is divided by the square root of its
// principal moment and has unit length; rows of different axes are
// orthogonal, and every row has zero component sums (orthogonal to the
// three averages).  Rows (3m weights each, node-major, xyz per node, in the
// order of `nodes`) are appended to w, largest moment first; the count is
// returned.
inline int class_rotations(const std::vector<double>& X, const std::vector<int>& nodes,
                           std::vector<double>& w) {
  const int m = (int)nodes.size();
  if (m < 2) return 0;
  double c[3] = {0, 0, 0};
  for (int v : nodes)
    for (int k = 0; k < 3; ++k) c[k] += X[3 * (size_t)v + k];
  for (int k = 0; k < 3; ++k) c[k] /= m;
  double M[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  for (int v : nodes) {
    double y[3];
    for (int k = 0; k < 3; ++k) y[k] = X[3 * (size_t)v + k] - c[k];
    const double yy = y[0] * y[0] + y[1] * y[1] + y[2] * y[2];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) M[i][j] += (i == j ? yy : 0.0) - y[i] * y[j];
  }
  double lam[3], V[3][3];
  sym3_eigen(M, lam, V);
  int order[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[order[j]] > lam[order[i]]) { const int t = order[i]; order[i] = order[j]; order[j] = t; }
  const double lmax = lam[order[0]];
  if (!(lmax > 0.0)) return 0;
  int n = 0;
  for (int r = 0; r < 3; ++r) {
    const int k = order[r];
    if (lam[k] < kRigidDrop * lmax) continue;
    const double ax[3] = {V[0][k], V[1][k], V[2][k]};
    const double inv = 1.0 / std::sqrt(lam[k]);
    for (int v : nodes) {
      double y[3];
      for (int q = 0; q < 3; ++q) y[q] = X[3 * (size_t)v + q] - c[q];
      w.push_back((ax[1] * y[2] - ax[2] * y[1]) * inv);
      w.push_back((ax[2] * y[0] - ax[0] * y[2]) * inv);
      w.push_back((ax[0] * y[1] - ax[1] * y[0]) * inv);
    }
    ++n;
  }
  return n;
}

}  // namespace cbddc
