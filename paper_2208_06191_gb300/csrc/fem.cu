// Element-batched residual and tangent assembly (FP64) and BSR SpMV.
//
// Section 2 of the paper: P = P_pas + P_act with the Guccione energy
//   Psi = C/2 (e^Q - 1) + B/2 (J - 1) log J,
//   Q = sum_ab w_ab E_ab^2 in the fibre frame {f, s, n},
// active stress gamma (F f)(x) f / |F f|, and the follower pressure
// p J F^{-T} N on the loaded faces (Eq. bc endo), here integrated through
// Nanson's relation J F^{-T} N dA = (dx/ds x dx/dt) ds dt on the deformed
// face.  The tangent is the exact derivative (Eq. tangent problem).
//
// Layout: one CTA per element; element matrices are written as 3x3 blocks
// [e][a][b][i][k] into a contribution buffer, and deterministic gather
// kernels (precomputed slot lists) sum them into the global BSR matrix and
// into the subdomain matrices.
#include <cmath>

#include "common.h"
#include "fem.h"

namespace cbddc {

// 1-D Lagrange basis on equispaced nodes and Gauss rule, per order (1, 2):
// c_L[o][q][i] = L_i(x_q), c_dL = L_i'(x_q), c_w = Gauss weight.
__constant__ double c_L[2][3][3];
__constant__ double c_dL[2][3][3];
__constant__ double c_w[2][3];
__constant__ double c_x[2][3];

// Tetrahedra (index o = order - 1): volume rule points q, shape values
// c_tN[o][q][a] and reference gradients c_tdN[o][q][a][j]; triangle faces:
// values c_fN[o][q][a] and parametric derivatives c_fds / c_fdt.
__constant__ double c_tN[3][8][10];
__constant__ double c_tdN[3][8][10][3];
__constant__ double c_tw[3][8];
__constant__ double c_fN[2][3][6];
__constant__ double c_fds[2][3][6];
__constant__ double c_fdt[2][3][6];
__constant__ double c_fw[2][3];

namespace {

// P1/P2 shape functions of the reference tetrahedron at xi (barycentric
// L0 = 1 - x - y - z, L1..3 = x, y, z; P2 vertices L(2L - 1), edge
// midpoints 4 L_a L_b on edges (0,1), (1,2), (0,2), (0,3), (1,3), (2,3)).
void tet_shape_host(int k, const double xi[3], double* N, double (*dN)[3]) {
  const double L[4] = {1.0 - xi[0] - xi[1] - xi[2], xi[0], xi[1], xi[2]};
  const double dL[4][3] = {{-1, -1, -1}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  if (k == 1) {
    for (int a = 0; a < 4; ++a) {
      N[a] = L[a];
      for (int j = 0; j < 3; ++j) dN[a][j] = dL[a][j];
    }
    return;
  }
  static const int ed[6][2] = {{0, 1}, {1, 2}, {0, 2}, {0, 3}, {1, 3}, {2, 3}};
  for (int a = 0; a < 4; ++a) {
    N[a] = L[a] * (2.0 * L[a] - 1.0);
    for (int j = 0; j < 3; ++j) dN[a][j] = (4.0 * L[a] - 1.0) * dL[a][j];
  }
  for (int m = 0; m < 6; ++m) {
    const int a = ed[m][0], b = ed[m][1];
    N[4 + m] = 4.0 * L[a] * L[b];
    for (int j = 0; j < 3; ++j) dN[4 + m][j] = 4.0 * (L[b] * dL[a][j] + L[a] * dL[b][j]);
  }
}

// P1/P2 shape functions of the reference triangle in the face parameters
// (s, t): vertices (0,0), (1,0), (0,1), then midpoints of (0,1), (1,2), (0,2).
void tri_shape_host(int k, double s, double t, double* N, double* ds, double* dt) {
  const double L[3] = {1.0 - s - t, s, t};
  const double dLs[3] = {-1, 1, 0}, dLt[3] = {-1, 0, 1};
  if (k == 1) {
    for (int a = 0; a < 3; ++a) { N[a] = L[a]; ds[a] = dLs[a]; dt[a] = dLt[a]; }
    return;
  }
  static const int ed[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  for (int a = 0; a < 3; ++a) {
    N[a] = L[a] * (2.0 * L[a] - 1.0);
    ds[a] = (4.0 * L[a] - 1.0) * dLs[a];
    dt[a] = (4.0 * L[a] - 1.0) * dLt[a];
  }
  for (int m = 0; m < 3; ++m) {
    const int a = ed[m][0], b = ed[m][1];
    N[3 + m] = 4.0 * L[a] * L[b];
    ds[3 + m] = 4.0 * (L[b] * dLs[a] + L[a] * dLs[b]);
    dt[3 + m] = 4.0 * (L[b] * dLt[a] + L[a] * dLt[b]);
  }
}

void init_tet_tables() {
  double tN[3][8][10] = {}, tdN[3][8][10][3] = {}, tw[3][8] = {};
  double fN[2][3][6] = {}, fds[2][3][6] = {}, fdt[2][3][6] = {}, fw[2][3] = {};
  // P1: centroid, weight 1/6 (volume of the reference tetrahedron)
  {
    const double xi[3] = {0.25, 0.25, 0.25};
    tet_shape_host(1, xi, tN[0][0], tdN[0][0]);
    tw[0][0] = 1.0 / 6.0;
  }
  // P2: symmetric 4-point rule of degree 2, barycentric (a, b, b, b)
  {
    const double a = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, b = (5.0 - std::sqrt(5.0)) / 20.0;
    for (int q = 0; q < 4; ++q) {
      double bary[4] = {b, b, b, b};
      bary[q] = a;
      const double xi[3] = {bary[1], bary[2], bary[3]};
      tet_shape_host(2, xi, tN[1][q], tdN[1][q]);
      tw[1][q] = 1.0 / 24.0;
    }
  }
  // table 2: the trilinear hexahedron at its 2 x 2 x 2 Gauss points (for the
  // quadrature-point-parallel kernel), point qx + 2 (qy + 2 qz), node
  // ax + 2 (ay + 2 az) at (-1 + 2 ax, -1 + 2 ay, -1 + 2 az)
  {
    const double g = 1.0 / std::sqrt(3.0);
    for (int q = 0; q < 8; ++q) {
      const double x[3] = {(q & 1) ? g : -g, (q & 2) ? g : -g, (q & 4) ? g : -g};
      for (int a = 0; a < 8; ++a) {
        const double s[3] = {(a & 1) ? 1.0 : -1.0, (a & 2) ? 1.0 : -1.0, (a & 4) ? 1.0 : -1.0};
        const double l[3] = {0.5 * (1.0 + s[0] * x[0]), 0.5 * (1.0 + s[1] * x[1]), 0.5 * (1.0 + s[2] * x[2])};
        tN[2][q][a] = l[0] * l[1] * l[2];
        tdN[2][q][a][0] = 0.5 * s[0] * l[1] * l[2];
        tdN[2][q][a][1] = 0.5 * s[1] * l[0] * l[2];
        tdN[2][q][a][2] = 0.5 * s[2] * l[0] * l[1];
      }
      tw[2][q] = 1.0;
    }
  }
  // triangle rules: centroid (weight 1/2) and the 3-point rule of degree 2
  tri_shape_host(1, 1.0 / 3.0, 1.0 / 3.0, fN[0][0], fds[0][0], fdt[0][0]);
  fw[0][0] = 0.5;
  const double st[3][2] = {{1.0 / 6.0, 1.0 / 6.0}, {2.0 / 3.0, 1.0 / 6.0}, {1.0 / 6.0, 2.0 / 3.0}};
  for (int q = 0; q < 3; ++q) {
    tri_shape_host(2, st[q][0], st[q][1], fN[1][q], fds[1][q], fdt[1][q]);
    fw[1][q] = 1.0 / 6.0;
  }
  CB_CUDA(cudaMemcpyToSymbol(c_tN, tN, sizeof(tN)));
  CB_CUDA(cudaMemcpyToSymbol(c_tdN, tdN, sizeof(tdN)));
  CB_CUDA(cudaMemcpyToSymbol(c_tw, tw, sizeof(tw)));
  CB_CUDA(cudaMemcpyToSymbol(c_fN, fN, sizeof(fN)));
  CB_CUDA(cudaMemcpyToSymbol(c_fds, fds, sizeof(fds)));
  CB_CUDA(cudaMemcpyToSymbol(c_fdt, fdt, sizeof(fdt)));
  CB_CUDA(cudaMemcpyToSymbol(c_fw, fw, sizeof(fw)));
}

}  // namespace

void init_shape_tables(int /*order*/) {
  init_tet_tables();
  double L[2][3][3] = {}, dL[2][3][3] = {}, w[2][3] = {}, x[2][3] = {};
  for (int o = 1; o <= 2; ++o) {
    const int m = o + 1;
    double gx[3], gw[3];
    if (o == 1) {
      gx[0] = -1.0 / std::sqrt(3.0); gx[1] = -gx[0]; gw[0] = gw[1] = 1.0;
    } else {
      gx[0] = -std::sqrt(0.6); gx[1] = 0.0; gx[2] = std::sqrt(0.6);
      gw[0] = gw[2] = 5.0 / 9.0; gw[1] = 8.0 / 9.0;
    }
    double nodes[3];
    for (int i = 0; i < m; ++i) nodes[i] = -1.0 + 2.0 * i / o;
    for (int q = 0; q < m; ++q) {
      x[o - 1][q] = gx[q];
      w[o - 1][q] = gw[q];
      for (int i = 0; i < m; ++i) {
        double v = 1.0, dv = 0.0;
        for (int j = 0; j < m; ++j) {
          if (j == i) continue;
          double fac = (gx[q] - nodes[j]) / (nodes[i] - nodes[j]);
          // product rule: d/dx prod = sum_j (1/(n_i-n_j)) prod_{l!=j}
          dv = dv * fac + v / (nodes[i] - nodes[j]);
          v *= fac;
        }
        L[o - 1][q][i] = v;
        dL[o - 1][q][i] = dv;
      }
    }
  }
  CB_CUDA(cudaMemcpyToSymbol(c_L, L, sizeof(L)));
  CB_CUDA(cudaMemcpyToSymbol(c_dL, dL, sizeof(dL)));
  CB_CUDA(cudaMemcpyToSymbol(c_w, w, sizeof(w)));
  CB_CUDA(cudaMemcpyToSymbol(c_x, x, sizeof(x)));
}

struct MatParams {
  double C, W[3][3], B;
  double fz0, fz1, fa0, fa1;  // slab helix fibre field
  double gamma, pressure;
  int nodal;                  // fibres from interpolated nodal (f, n)
  double rho_dt2;             // rho / dt^2 of the inertia term (0: off)
};

__device__ inline double det3(const double A[3][3]) {
  return A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) -
         A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
         A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
}

// inverse via the adjugate; returns the determinant
__device__ inline double inv3(const double A[3][3], double Ai[3][3]) {
  double c00 = A[1][1] * A[2][2] - A[1][2] * A[2][1];
  double c01 = A[1][2] * A[2][0] - A[1][0] * A[2][2];
  double c02 = A[1][0] * A[2][1] - A[1][1] * A[2][0];
  double det = A[0][0] * c00 + A[0][1] * c01 + A[0][2] * c02;
  double id = 1.0 / det;
  Ai[0][0] = c00 * id;
  Ai[1][0] = c01 * id;
  Ai[2][0] = c02 * id;
  Ai[0][1] = (A[0][2] * A[2][1] - A[0][1] * A[2][2]) * id;
  Ai[1][1] = (A[0][0] * A[2][2] - A[0][2] * A[2][0]) * id;
  Ai[2][1] = (A[0][1] * A[2][0] - A[0][0] * A[2][1]) * id;
  Ai[0][2] = (A[0][1] * A[1][2] - A[0][2] * A[1][1]) * id;
  Ai[1][2] = (A[0][2] * A[1][0] - A[0][0] * A[1][2]) * id;
  Ai[2][2] = (A[0][0] * A[1][1] - A[0][1] * A[1][0]) * id;
  return det;
}

// Fibre frame R = [f | s | n] (columns) at reference point X.
__device__ inline void fibre_frame(const MatParams& m, const double X[3], double R[3][3]) {
  double t = (X[2] - m.fz0) / (m.fz1 - m.fz0);
  double a = m.fa0 + (m.fa1 - m.fa0) * t;
  double c = cos(a), s = sin(a);
  R[0][0] = c;   R[0][1] = -s;  R[0][2] = 0.0;
  R[1][0] = s;   R[1][1] = c;   R[1][2] = 0.0;
  R[2][0] = 0.0; R[2][1] = 0.0; R[2][2] = 1.0;
}

// Fibre frame from interpolated nodal directions: f normalised, n made
// orthogonal to f and normalised, s = n x f; columns (f, s, n).
__device__ inline void frame_from_fn(const double fv[3], const double nv[3], double R[3][3]) {
  const double fl = 1.0 / sqrt(fv[0] * fv[0] + fv[1] * fv[1] + fv[2] * fv[2]);
  const double f[3] = {fv[0] * fl, fv[1] * fl, fv[2] * fl};
  const double nf = nv[0] * f[0] + nv[1] * f[1] + nv[2] * f[2];
  double n[3] = {nv[0] - nf * f[0], nv[1] - nf * f[1], nv[2] - nf * f[2]};
  const double nl = 1.0 / sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  n[0] *= nl; n[1] *= nl; n[2] *= nl;
  const double sv[3] = {n[1] * f[2] - n[2] * f[1], n[2] * f[0] - n[0] * f[2], n[0] * f[1] - n[1] * f[0]};
  for (int i = 0; i < 3; ++i) { R[i][0] = f[i]; R[i][1] = sv[i]; R[i][2] = n[i]; }
}

// Stress P (row-major 3x3) and, if A != nullptr, the tangent
// A[((i*3+J)*3+k)*3+L] = dP_iJ/dF_kL, at one quadrature point.
// Returns false if J <= 0.
__device__ bool material_point(const MatParams& m, const double F[3][3], const double R[3][3],
                               double* P, double* A) {
  double Fi[3][3];
  double J = inv3(F, Fi);
  if (!(J > 0.0)) return false;
  // E = (F^T F - I)/2 and its fibre-frame components E' = R^T E R
  double E[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double c = 0.0;
      for (int i = 0; i < 3; ++i) c += F[i][a] * F[i][b];
      E[a][b] = 0.5 * (c - (a == b ? 1.0 : 0.0));
    }
  double ER[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double c = 0.0;
      for (int j = 0; j < 3; ++j) c += E[a][j] * R[j][b];
      ER[a][b] = c;
    }
  double Ep[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      double c = 0.0;
      for (int i = 0; i < 3; ++i) c += R[i][a] * ER[i][b];
      Ep[a][b] = c;
    }
  double Q = 0.0;
  double WE[3][3];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) {
      WE[a][b] = m.W[a][b] * Ep[a][b];
      Q += WE[a][b] * Ep[a][b];
    }
  // Shat = R (W o E') R^T, S = C e^Q Shat
  double Sh[3][3], tmp[3][3];
  for (int i = 0; i < 3; ++i)
    for (int b = 0; b < 3; ++b) {
      double c = 0.0;
      for (int a = 0; a < 3; ++a) c += R[i][a] * WE[a][b];
      tmp[i][b] = c;
    }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double c = 0.0;
      for (int b = 0; b < 3; ++b) c += tmp[i][b] * R[j][b];
      Sh[i][j] = c;
    }
  const double eQ = m.C * exp(Q);
  const double lJ = log(J);
  const double kap = 0.5 * m.B * (J * lJ + J - 1.0);
  const double dkap = 0.5 * m.B * (lJ + 2.0);
  double FS[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double c = 0.0;
      for (int l = 0; l < 3; ++l) c += F[i][l] * Sh[l][j];
      FS[i][j] = c;
    }
  // active part: u = F f, m = u/|u|
  double u[3], un = 0.0;
  for (int i = 0; i < 3; ++i) {
    u[i] = F[i][0] * R[0][0] + F[i][1] * R[1][0] + F[i][2] * R[2][0];
    un += u[i] * u[i];
  }
  un = sqrt(un);
  double mv[3] = {u[0] / un, u[1] / un, u[2] / un};
  double f[3] = {R[0][0], R[1][0], R[2][0]};
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      P[i * 3 + j] = eQ * FS[i][j] + kap * Fi[j][i] + m.gamma * mv[i] * f[j];
  if (A == nullptr) return true;
  // pushed frame g_a = F r_a
  double g[3][3];  // g[a][i]
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i < 3; ++i) g[a][i] = F[i][0] * R[0][a] + F[i][1] * R[1][a] + F[i][2] * R[2][a];
  const double ga = m.gamma / un;
  // The anisotropic second-derivative term
  //   lin_iJkL = sum_ab W_ab g_ai R_Jb (g_ak R_Lb + g_bk R_La)
  // is factored as sum_a g_ai g_ak X_a(J,L) + sum_a (g_ai R_La) V_a(k,J) with
  //   X_a(J,L) = sum_b W_ab R_Jb R_Lb,   V_a(k,J) = sum_b W_ab g_bk R_Jb,
  // and A is major-symmetric (A_iJkL = A_kLiJ: the energy depends on F
  // only), so 45 entries are formed and mirrored (FP64 issue is the
  // bottleneck of this kernel).
  double X[3][3][3], V[3][3][3];  // X[a][J][L] (symmetric in J, L), V[a][k][J]
#pragma unroll
  for (int a = 0; a < 3; ++a) {
#pragma unroll
    for (int Jx = 0; Jx < 3; ++Jx)
#pragma unroll
      for (int L = Jx; L < 3; ++L) {
        const double v = m.W[a][0] * R[Jx][0] * R[L][0] + m.W[a][1] * R[Jx][1] * R[L][1] +
                         m.W[a][2] * R[Jx][2] * R[L][2];
        X[a][Jx][L] = v;
        X[a][L][Jx] = v;
      }
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
      for (int Jx = 0; Jx < 3; ++Jx)
        V[a][k][Jx] = m.W[a][0] * g[0][k] * R[Jx][0] + m.W[a][1] * g[1][k] * R[Jx][1] +
                      m.W[a][2] * g[2][k] * R[Jx][2];
  }
#pragma unroll
  for (int pq = 0; pq < 9; ++pq) {
    const int i = pq / 3, Jx = pq % 3;
#pragma unroll
    for (int qq = pq; qq < 9; ++qq) {
      const int k = qq / 3, L = qq % 3;
      double lin = 0.0;
      for (int a = 0; a < 3; ++a)
        lin += g[a][i] * (g[a][k] * X[a][Jx][L] + R[L][a] * V[a][k][Jx]);
      double v = eQ * (2.0 * FS[i][Jx] * FS[k][L] + 0.5 * lin);
      if (i == k) v += eQ * Sh[L][Jx];
      v += J * dkap * Fi[Jx][i] * Fi[L][k] - kap * Fi[Jx][k] * Fi[L][i];
      v += ga * ((i == k ? 1.0 : 0.0) - mv[i] * mv[k]) * f[Jx] * f[L];
      A[pq * 9 + qq] = v;
      A[qq * 9 + pq] = v;
    }
  }
  return true;
}

__global__ void scatter_free_kernel(const double* __restrict__ d, const int* __restrict__ free_nodes,
                                    int64_t n_free_nodes, double* __restrict__ d_full) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * n_free_nodes) return;
  int64_t node = free_nodes[i / 3];
  d_full[node * 3 + i % 3] = d[i];
}

// One CTA per element.  Order K hexahedron: M = K+1 points per direction,
// NEN = M^3 nodes and NQ = M^3 Gauss points.
template <int K, int THREADS>
__global__ void __launch_bounds__(THREADS)
element_kernel(MatParams mp, const double* __restrict__ coords, const int* __restrict__ elems,
               const double* __restrict__ fib, const double* __restrict__ d_full,
               const double* __restrict__ acc_full, double* __restrict__ rcontrib,
               double* __restrict__ contrib, int* __restrict__ status, int want_tangent) {
  constexpr int M = K + 1, NEN = M * M * M, NQ = NEN;
  constexpr int O = K - 1;
  __shared__ double X[NEN][3], U[NEN][3];
  __shared__ double G[NQ][NEN][3];
  __shared__ double Wd[NQ];
  __shared__ double Pq[NQ][9];
  __shared__ double Aq[NQ][81];
  __shared__ double T[NEN * 27];
  __shared__ double Nq[NQ][NEN], Aq3[NQ][3];  // shape values; d - 2d' + d'' at the points
  __shared__ int bad;
  const bool inertia = mp.rho_dt2 > 0.0;
  const int e = blockIdx.x;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int t = tid; t < NEN * 3; t += THREADS) {
    int a = t / 3, c = t % 3;
    int node = elems[(int64_t)e * NEN + a];
    X[a][c] = coords[(int64_t)node * 3 + c];
    U[a][c] = d_full[(int64_t)node * 3 + c];
  }
  __syncthreads();
  // geometry and constitutive update at each Gauss point
  for (int q = tid; q < NQ; q += THREADS) {
    const int qx = q % M, qy = (q / M) % M, qz = q / (M * M);
    double J0[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double Xq[3] = {0, 0, 0}, fq[3] = {0, 0, 0}, nq[3] = {0, 0, 0};
    for (int a = 0; a < NEN; ++a) {
      const int ax = a % M, ay = (a / M) % M, az = a / (M * M);
      const double lx = c_L[O][qx][ax], ly = c_L[O][qy][ay], lz = c_L[O][qz][az];
      const double dn[3] = {c_dL[O][qx][ax] * ly * lz, lx * c_dL[O][qy][ay] * lz,
                            lx * ly * c_dL[O][qz][az]};
      const double n = lx * ly * lz;
      Nq[q][a] = n;
      for (int i = 0; i < 3; ++i) {
        Xq[i] += n * X[a][i];
        for (int j = 0; j < 3; ++j) J0[i][j] += X[a][i] * dn[j];
      }
      if (mp.nodal) {
        const double* fa = fib + (int64_t)elems[(int64_t)e * NEN + a] * 6;
        for (int i = 0; i < 3; ++i) { fq[i] += n * fa[i]; nq[i] += n * fa[3 + i]; }
      }
      G[q][a][0] = dn[0];
      G[q][a][1] = dn[1];
      G[q][a][2] = dn[2];
    }
    if (inertia) {
      double aq[3] = {0, 0, 0};
      for (int a = 0; a < NEN; ++a) {
        const double* va = acc_full + (int64_t)elems[(int64_t)e * NEN + a] * 3;
        for (int i = 0; i < 3; ++i) aq[i] += Nq[q][a] * va[i];
      }
      for (int i = 0; i < 3; ++i) Aq3[q][i] = aq[i];
    }
    double J0i[3][3];
    const double det0 = inv3(J0, J0i);
    Wd[q] = c_w[O][qx] * c_w[O][qy] * c_w[O][qz] * det0;
    double F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int a = 0; a < NEN; ++a) {
      double dn[3] = {G[q][a][0], G[q][a][1], G[q][a][2]};
      double gx[3];
      for (int i = 0; i < 3; ++i) gx[i] = dn[0] * J0i[0][i] + dn[1] * J0i[1][i] + dn[2] * J0i[2][i];
      G[q][a][0] = gx[0];
      G[q][a][1] = gx[1];
      G[q][a][2] = gx[2];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) F[i][j] += U[a][i] * gx[j];
    }
    double R[3][3];
    if (mp.nodal) frame_from_fn(fq, nq, R);
    else fibre_frame(mp, Xq, R);
    if (!(det0 > 0.0) || !material_point(mp, F, R, Pq[q], want_tangent ? Aq[q] : nullptr)) {
      bad = 1;
      for (int i = 0; i < 9; ++i) Pq[q][i] = 0.0;
      if (want_tangent)
        for (int i = 0; i < 81; ++i) Aq[q][i] = 0.0;
    }
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(status, DEV_INVERTED);
  // residual r_a,i = sum_q w detJ0 P_iJ dN_a/dX_J
  for (int t = tid; t < NEN * 3; t += THREADS) {
    const int a = t / 3, i = t % 3;
    double r = 0.0;
    for (int q = 0; q < NQ; ++q)
      r += Wd[q] * (Pq[q][i * 3 + 0] * G[q][a][0] + Pq[q][i * 3 + 1] * G[q][a][1] +
                    Pq[q][i * 3 + 2] * G[q][a][2]);
    if (inertia)
      for (int q = 0; q < NQ; ++q) r += mp.rho_dt2 * Wd[q] * Nq[q][a] * Aq3[q][i];
    rcontrib[((int64_t)e * NEN + a) * 3 + i] = r;
  }
  if (!want_tangent) return;
  // K[a][b][i][k] = sum_q w detJ0 sum_JL dN_a/dX_J A_iJkL dN_b/dX_L
  constexpr int NE = NEN * NEN * 9;
  constexpr int PER = (NE + THREADS - 1) / THREADS;
  double acc[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) acc[j] = 0.0;
  for (int q = 0; q < NQ; ++q) {
    __syncthreads();
    // T[a][i][k][L] = w detJ0 sum_J dN_a/dX_J A_iJkL
    for (int t = tid; t < NEN * 27; t += THREADS) {
      const int a = t / 27, r = t % 27, i = r / 9, k = (r / 3) % 3, L = r % 3;
      const double* Aqq = Aq[q];
      T[t] = Wd[q] * (G[q][a][0] * Aqq[((i * 3 + 0) * 3 + k) * 3 + L] +
                      G[q][a][1] * Aqq[((i * 3 + 1) * 3 + k) * 3 + L] +
                      G[q][a][2] * Aqq[((i * 3 + 2) * 3 + k) * 3 + L]);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int t = tid + j * THREADS;
      if (t < NE) {
        const int a = t / (NEN * 9), b = (t / 9) % NEN, i = (t % 9) / 3, k = t % 3;
        const double* Ta = &T[a * 27 + i * 9 + k * 3];
        acc[j] += Ta[0] * G[q][b][0] + Ta[1] * G[q][b][1] + Ta[2] * G[q][b][2];
      }
    }
  }
  if (inertia) {
    // consistent mass rho/dt^2 sum_q w detJ0 N_a N_b on the diagonal i = k
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int t = tid + j * THREADS;
      if (t < NE) {
        const int a = t / (NEN * 9), b = (t / 9) % NEN, i = (t % 9) / 3, k = t % 3;
        if (i == k) {
          double m = 0.0;
          for (int q = 0; q < NQ; ++q) m += Wd[q] * Nq[q][a] * Nq[q][b];
          acc[j] += mp.rho_dt2 * m;
        }
      }
    }
  }
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int t = tid + j * THREADS;
    if (t < NE) contrib[(int64_t)e * NE + t] = acc[j];
  }
}


// Quadrature-point-parallel element kernel for elements with few points
// (P1: 1, P2: 4, Q1: 8; shape table O = 0, 1, 2), TET_THREADS material
// points per CTA (EPB = TET_THREADS / NQ elements), so that every lane of
// the FP64 material evaluation has work.  Phase 1: one thread per quadrature point computes the
// geometry, F, the fibre frame and the material point, and stores
// w detJ0 P and w detJ0 dP/dF in shared memory (stride 81 per point keeps
// the 8-byte accesses conflict-free).  Phase 2: one thread per residual
// entry (e, a, i).  Phase 3: one thread per (e, a, i, k) row of the element
// matrix, K[a][b][i][k] = sum_q sum_L (sum_J G_aJ A_iJkL) G_bL for all b.
constexpr int TET_THREADS = 32;

template <int NEN, int NQ, int O>
__global__ void __launch_bounds__(TET_THREADS)
qp_element_kernel(MatParams mp, const double* __restrict__ coords, const int* __restrict__ elems,
                  const double* __restrict__ fib, const double* __restrict__ d_full,
                  const double* __restrict__ acc_full, double* __restrict__ rcontrib,
                  double* __restrict__ contrib, int* __restrict__ status, int want_tangent, int n_el) {
  constexpr int EPB = TET_THREADS / NQ;
  static_assert(EPB * NQ == TET_THREADS, "whole elements per CTA");
  __shared__ double As[TET_THREADS * 81];
  __shared__ double Ps[TET_THREADS * 9];
  __shared__ double Gs[TET_THREADS][NEN][3];
  __shared__ double Xs[EPB][NEN][3], Us[EPB][NEN][3];
  __shared__ double Wq[TET_THREADS], Aq3[TET_THREADS][3];  // w detJ0 and the point's d - 2d' + d''
  const bool inertia = mp.rho_dt2 > 0.0;
  __shared__ int Ns[EPB][NEN];
  __shared__ int bad;
  const int tid = threadIdx.x;
  const int64_t e0 = (int64_t)blockIdx.x * EPB;
  const int ne_here = (int)min((int64_t)EPB, (int64_t)n_el - e0);
  if (tid == 0) bad = 0;
  for (int t = tid; t < ne_here * NEN; t += TET_THREADS) Ns[t / NEN][t % NEN] = elems[e0 * NEN + t];
  __syncthreads();
  for (int t = tid; t < ne_here * NEN * 3; t += TET_THREADS) {
    const int el = t / (NEN * 3), a = (t / 3) % NEN, c = t % 3;
    const int node = Ns[el][a];
    Xs[el][a][c] = coords[(int64_t)node * 3 + c];
    Us[el][a][c] = d_full[(int64_t)node * 3 + c];
  }
  __syncthreads();
  {
    const int p = tid, el = p / NQ, q = p % NQ;
    double* A = &As[p * 81];
    double* P = &Ps[p * 9];
    bool ok = el < ne_here;
    if (ok) {
      double J0[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
      double fq[3] = {0, 0, 0}, nq[3] = {0, 0, 0}, Xq[3] = {0, 0, 0};
      for (int a = 0; a < NEN; ++a) {
        const double n = c_tN[O][q][a];
        for (int i = 0; i < 3; ++i) {
          Xq[i] += n * Xs[el][a][i];
          for (int j = 0; j < 3; ++j) J0[i][j] += Xs[el][a][i] * c_tdN[O][q][a][j];
        }
        if (mp.nodal) {
          const double* fa = fib + (int64_t)Ns[el][a] * 6;
          for (int i = 0; i < 3; ++i) { fq[i] += n * fa[i]; nq[i] += n * fa[3 + i]; }
        }
      }
      double J0i[3][3];
      const double det0 = inv3(J0, J0i);
      double F[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
      for (int a = 0; a < NEN; ++a) {
        double gx[3];
        for (int i = 0; i < 3; ++i)
          gx[i] = c_tdN[O][q][a][0] * J0i[0][i] + c_tdN[O][q][a][1] * J0i[1][i] +
                  c_tdN[O][q][a][2] * J0i[2][i];
        for (int i = 0; i < 3; ++i) {
          Gs[p][a][i] = gx[i];
          for (int j = 0; j < 3; ++j) F[i][j] += Us[el][a][i] * gx[j];
        }
      }
      double R[3][3];
      if (mp.nodal) frame_from_fn(fq, nq, R);
      else fibre_frame(mp, Xq, R);
      ok = det0 > 0.0 && material_point(mp, F, R, P, want_tangent ? A : nullptr);
      if (inertia) {
        double aq[3] = {0, 0, 0};
        for (int a = 0; a < NEN; ++a)
          for (int i = 0; i < 3; ++i) aq[i] += c_tN[O][q][a] * acc_full[(int64_t)Ns[el][a] * 3 + i];
        for (int i = 0; i < 3; ++i) Aq3[p][i] = aq[i];
      }
      Wq[p] = c_tw[O][q] * det0;
      if (ok) {
        const double wd = c_tw[O][q] * det0;
        for (int i = 0; i < 9; ++i) P[i] *= wd;
        if (want_tangent)
          for (int i = 0; i < 81; ++i) A[i] *= wd;
      } else {
        bad = 1;
      }
    }
    if (!ok) {
      Wq[p] = 0.0;
      Aq3[p][0] = Aq3[p][1] = Aq3[p][2] = 0.0;
      for (int i = 0; i < 9; ++i) P[i] = 0.0;
      for (int i = 0; i < 81; ++i) A[i] = 0.0;
      for (int a = 0; a < NEN; ++a) Gs[p][a][0] = Gs[p][a][1] = Gs[p][a][2] = 0.0;
    }
  }
  __syncthreads();
  if (tid == 0 && bad) atomicOr(status, DEV_INVERTED);
  for (int t = tid; t < ne_here * NEN * 3; t += TET_THREADS) {
    const int el = t / (NEN * 3), a = (t / 3) % NEN, i = t % 3;
    double r = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int p = el * NQ + q;
      r += Ps[p * 9 + i * 3 + 0] * Gs[p][a][0] + Ps[p * 9 + i * 3 + 1] * Gs[p][a][1] +
           Ps[p * 9 + i * 3 + 2] * Gs[p][a][2];
      if (inertia) r += mp.rho_dt2 * Wq[p] * c_tN[O][q][a] * Aq3[p][i];
    }
    rcontrib[((e0 + el) * NEN + a) * 3 + i] = r;
  }
  if (!want_tangent) return;
  for (int t = tid; t < ne_here * NEN * 9; t += TET_THREADS) {
    const int el = t / (NEN * 9), a = (t / 9) % NEN, i = (t % 9) / 3, k = t % 3;
    double acc[NEN];
#pragma unroll
    for (int b = 0; b < NEN; ++b) acc[b] = 0.0;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int p = el * NQ + q;
      const double* A = &As[p * 81 + i * 27 + k * 3];
      const double g0 = Gs[p][a][0], g1 = Gs[p][a][1], g2 = Gs[p][a][2];
      const double T0 = g0 * A[0] + g1 * A[9] + g2 * A[18];
      const double T1 = g0 * A[1] + g1 * A[10] + g2 * A[19];
      const double T2 = g0 * A[2] + g1 * A[11] + g2 * A[20];
#pragma unroll
      for (int b = 0; b < NEN; ++b) acc[b] += T0 * Gs[p][b][0] + T1 * Gs[p][b][1] + T2 * Gs[p][b][2];
      if (inertia && i == k) {
        const double wa = mp.rho_dt2 * Wq[p] * c_tN[O][q][a];
#pragma unroll
        for (int b = 0; b < NEN; ++b) acc[b] += wa * c_tN[O][q][b];
      }
    }
    double* out = contrib + ((e0 + el) * NEN * NEN + (int64_t)a * NEN) * 9 + i * 3 + k;
#pragma unroll
    for (int b = 0; b < NEN; ++b) out[b * 9] = acc[b];
  }
}

// Follower pressure on one triangular face per CTA (same integrand as the
// quadrilateral faces, with the triangle rules).
template <int K, int THREADS>
__global__ void __launch_bounds__(THREADS)
tri_face_kernel(double pressure, const double* __restrict__ coords, const int* __restrict__ face_nodes,
                const double* __restrict__ d_full, double* __restrict__ rcontrib,
                double* __restrict__ contrib, int want_tangent) {
  constexpr int NFN = K == 1 ? 3 : 6, NQ = K == 1 ? 1 : 3, O = K - 1;
  __shared__ double x[NFN][3];
  __shared__ double xs[NQ][3], xt[NQ][3];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  for (int t = tid; t < NFN * 3; t += THREADS) {
    int a = t / 3, c = t % 3;
    int node = face_nodes[(int64_t)f * NFN + a];
    x[a][c] = coords[(int64_t)node * 3 + c] + d_full[(int64_t)node * 3 + c];
  }
  __syncthreads();
  for (int q = tid; q < NQ; q += THREADS) {
    double s[3] = {0, 0, 0}, t3[3] = {0, 0, 0};
    for (int a = 0; a < NFN; ++a)
      for (int i = 0; i < 3; ++i) { s[i] += c_fds[O][q][a] * x[a][i]; t3[i] += c_fdt[O][q][a] * x[a][i]; }
    for (int i = 0; i < 3; ++i) { xs[q][i] = s[i]; xt[q][i] = t3[i]; }
  }
  __syncthreads();
  for (int t = tid; t < NFN * 3; t += THREADS) {
    const int a = t / 3, i = t % 3;
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    double r = 0.0;
    for (int q = 0; q < NQ; ++q)
      r += c_fw[O][q] * c_fN[O][q][a] * (xs[q][i1] * xt[q][i2] - xs[q][i2] * xt[q][i1]);
    rcontrib[((int64_t)f * NFN + a) * 3 + i] = pressure * r;
  }
  if (!want_tangent) return;
  constexpr int NE = NFN * NFN * 9;
  for (int t = tid; t < NE; t += THREADS) {
    const int a = t / (NFN * 9), b = (t / 9) % NFN, i = (t % 9) / 3, k = t % 3;
    double v = 0.0;
    if (i != k) {
      const int l = 3 - i - k;
      const double eps = ((k - i + 3) % 3 == 1) ? 1.0 : -1.0;  // eps_ikl
      for (int q = 0; q < NQ; ++q)
        v += c_fw[O][q] * c_fN[O][q][a] * (c_fds[O][q][b] * eps * xt[q][l] - c_fdt[O][q][b] * eps * xs[q][l]);
    }
    contrib[(int64_t)f * NE + t] = pressure * v;
  }
}


// Generalized Robin condition of Eq. (bc epi) on one face per CTA: traction
// g = (N x N)(K_perp u + C_perp v) + (I - N x N)(K_par u + C_par v) with the
// reference unit normal N, u the displacement and v = (d - d_prev)/dt at the
// face points (v = 0 without a time state); residual N_a g dS and tangent
// N_a N_b [(N x N) k_perp + (I - N x N) k_par] dS, k = K + C / dt.  TRI
// selects the triangle rules (tetrahedra) or the tensor rules (hexahedra).
struct RobinParams {
  double par[2][4];  // K_perp, K_par, C_perp, C_par per set
  double inv_dt;     // 1/dt, 0 without a time state
};

template <bool TRI, int K, int THREADS>
__global__ void __launch_bounds__(THREADS)
robin_face_kernel(RobinParams rp, const double* __restrict__ coords, const int* __restrict__ face_nodes,
                  const int* __restrict__ robin_set, const double* __restrict__ d_full,
                  const double* __restrict__ vel_full, double* __restrict__ rcontrib,
                  double* __restrict__ contrib, int want_tangent) {
  constexpr int M = K + 1;
  constexpr int NFN = TRI ? (K == 1 ? 3 : 6) : M * M;
  constexpr int NQ = TRI ? (K == 1 ? 1 : 3) : M * M;
  constexpr int O = K - 1;
  __shared__ double X[NFN][3], U[NFN][3], Vv[NFN][3];
  __shared__ double Nn[NQ][3], wa[NQ], gq[NQ][3];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  // face shape value / derivatives at point q for node a
  auto shp = [&](int q, int a, double& n, double& ds, double& dt) {
    if constexpr (TRI) {
      n = c_fN[O][q][a]; ds = c_fds[O][q][a]; dt = c_fdt[O][q][a];
    } else {
      const int qs = q % M, qt = q / M, as = a % M, at = a / M;
      n = c_L[O][qs][as] * c_L[O][qt][at];
      ds = c_dL[O][qs][as] * c_L[O][qt][at];
      dt = c_L[O][qs][as] * c_dL[O][qt][at];
    }
  };
  auto wq = [&](int q) -> double {
    if constexpr (TRI) return c_fw[O][q];
    else return c_w[O][q % M] * c_w[O][q / M];
  };
  const double* par = rp.par[robin_set[f]];
  const double kp = par[0], kt = par[1], cp = par[2], ct = par[3];
  for (int t = tid; t < NFN * 3; t += THREADS) {
    const int a = t / 3, c = t % 3;
    const int node = face_nodes[(int64_t)f * NFN + a];
    X[a][c] = coords[(int64_t)node * 3 + c];
    U[a][c] = d_full[(int64_t)node * 3 + c];
    Vv[a][c] = vel_full ? vel_full[(int64_t)node * 3 + c] : 0.0;
  }
  __syncthreads();
  for (int q = tid; q < NQ; q += THREADS) {
    double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0}, u[3] = {0, 0, 0}, v[3] = {0, 0, 0};
    for (int a = 0; a < NFN; ++a) {
      double n, ds, dt;
      shp(q, a, n, ds, dt);
      for (int i = 0; i < 3; ++i) {
        xs[i] += ds * X[a][i];
        xt[i] += dt * X[a][i];
        u[i] += n * U[a][i];
        v[i] += n * Vv[a][i];
      }
    }
    const double A[3] = {xs[1] * xt[2] - xs[2] * xt[1], xs[2] * xt[0] - xs[0] * xt[2],
                         xs[0] * xt[1] - xs[1] * xt[0]};
    const double area = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    const double N[3] = {A[0] / area, A[1] / area, A[2] / area};
    const double un = N[0] * u[0] + N[1] * u[1] + N[2] * u[2];
    const double vn = N[0] * v[0] + N[1] * v[1] + N[2] * v[2];
    for (int i = 0; i < 3; ++i) {
      Nn[q][i] = N[i];
      gq[q][i] = kp * un * N[i] + kt * (u[i] - un * N[i]) + cp * vn * N[i] + ct * (v[i] - vn * N[i]);
    }
    wa[q] = wq(q) * area;
  }
  __syncthreads();
  for (int t = tid; t < NFN * 3; t += THREADS) {
    const int a = t / 3, i = t % 3;
    double r = 0.0;
    for (int q = 0; q < NQ; ++q) {
      double n, ds, dt;
      shp(q, a, n, ds, dt);
      r += wa[q] * n * gq[q][i];
    }
    rcontrib[((int64_t)f * NFN + a) * 3 + i] = r;
  }
  if (!want_tangent) return;
  const double kpe = kp + cp * rp.inv_dt, kte = kt + ct * rp.inv_dt;
  constexpr int NE = NFN * NFN * 9;
  for (int t = tid; t < NE; t += THREADS) {
    const int a = t / (NFN * 9), b = (t / 9) % NFN, i = (t % 9) / 3, k = t % 3;
    double v = 0.0;
    for (int q = 0; q < NQ; ++q) {
      double na, nb, ds, dt;
      shp(q, a, na, ds, dt);
      shp(q, b, nb, ds, dt);
      const double nn = Nn[q][i] * Nn[q][k];
      v += wa[q] * na * nb * (kpe * nn + kte * ((i == k ? 1.0 : 0.0) - nn));
    }
    contrib[(int64_t)f * NE + t] = v;
  }
}

// d_full-style node arrays of the time state: acc = d - 2 d_prev + d_prev2
// and vel = (d - d_prev)/dt at the free nodes (Dirichlet nodes stay zero).
__global__ void time_vectors_kernel(const double* __restrict__ d, const double* __restrict__ dp,
                                    const double* __restrict__ dpp, const int* __restrict__ free_nodes,
                                    int64_t n_free_nodes, double inv_dt, double* __restrict__ acc,
                                    double* __restrict__ vel) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= 3 * n_free_nodes) return;
  const int64_t j = (int64_t)free_nodes[i / 3] * 3 + i % 3;
  acc[j] = d[i] - 2.0 * dp[i] + dpp[i];
  vel[j] = (d[i] - dp[i]) * inv_dt;
}

// Follower pressure on one face per CTA: residual p (x_s x x_t) N_a and its
// derivative p N_a [dN_b/ds (e_k x x_t) + dN_b/dt (x_s x e_k)].
template <int K, int THREADS>
__global__ void __launch_bounds__(THREADS)
face_kernel(double pressure, const double* __restrict__ coords, const int* __restrict__ face_nodes,
            const double* __restrict__ d_full, double* __restrict__ rcontrib,
            double* __restrict__ contrib, int want_tangent) {
  constexpr int M = K + 1, NFN = M * M, NQ = M * M;
  constexpr int O = K - 1;
  __shared__ double x[NFN][3];
  __shared__ double xs[NQ][3], xt[NQ][3];
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  for (int t = tid; t < NFN * 3; t += THREADS) {
    int a = t / 3, c = t % 3;
    int node = face_nodes[(int64_t)f * NFN + a];
    x[a][c] = coords[(int64_t)node * 3 + c] + d_full[(int64_t)node * 3 + c];
  }
  __syncthreads();
  for (int q = tid; q < NQ; q += THREADS) {
    const int qs = q % M, qt = q / M;
    double s[3] = {0, 0, 0}, t3[3] = {0, 0, 0};
    for (int a = 0; a < NFN; ++a) {
      const int as = a % M, at = a / M;
      const double ds = c_dL[O][qs][as] * c_L[O][qt][at];
      const double dt = c_L[O][qs][as] * c_dL[O][qt][at];
      for (int i = 0; i < 3; ++i) { s[i] += ds * x[a][i]; t3[i] += dt * x[a][i]; }
    }
    for (int i = 0; i < 3; ++i) { xs[q][i] = s[i]; xt[q][i] = t3[i]; }
  }
  __syncthreads();
  for (int t = tid; t < NFN * 3; t += THREADS) {
    const int a = t / 3, i = t % 3;
    const int as = a % M, at = a / M;
    double r = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const int qs = q % M, qt = q / M;
      const double wN = c_w[O][qs] * c_w[O][qt] * c_L[O][qs][as] * c_L[O][qt][at];
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      r += wN * (xs[q][i1] * xt[q][i2] - xs[q][i2] * xt[q][i1]);
    }
    rcontrib[((int64_t)f * NFN + a) * 3 + i] = pressure * r;
  }
  if (!want_tangent) return;
  constexpr int NE = NFN * NFN * 9;
  for (int t = tid; t < NE; t += THREADS) {
    const int a = t / (NFN * 9), b = (t / 9) % NFN, i = (t % 9) / 3, k = t % 3;
    const int as = a % M, at = a / M, bs = b % M, bt = b / M;
    double v = 0.0;
    for (int q = 0; q < NQ; ++q) {
      const int qs = q % M, qt = q / M;
      const double wN = c_w[O][qs] * c_w[O][qt] * c_L[O][qs][as] * c_L[O][qt][at];
      const double dbs = c_dL[O][qs][bs] * c_L[O][qt][bt];
      const double dbt = c_L[O][qs][bs] * c_dL[O][qt][bt];
      // (e_k x v)_i = eps_ikl v_l ; (v x e_k)_i = eps_ijk v_j
      double ek_x_t = 0.0, s_x_ek = 0.0;
      if (i != k) {
        const int l = 3 - i - k;
        const double eps = ((k - i + 3) % 3 == 1) ? 1.0 : -1.0;  // eps_ikl
        ek_x_t = eps * xt[q][l];
        s_x_ek = -eps * xs[q][l];  // eps_ilk = -eps_ikl
      }
      v += wN * (dbs * ek_x_t + dbt * s_x_ek);
    }
    contrib[(int64_t)f * NE + t] = pressure * v;
  }
}

// Sum of listed 3x3 blocks into each BSR slot (one thread per entry).
__global__ void gather_blocks_kernel(const int* __restrict__ ptr, const int* __restrict__ src,
                                     const double* __restrict__ contrib, int64_t nslots,
                                     double* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslots * 9) return;
  int64_t s = t / 9;
  int c = (int)(t % 9);
  double v = 0.0;
  for (int j = ptr[s]; j < ptr[s + 1]; ++j) v += contrib[(int64_t)src[j] * 9 + c];
  out[t] = v;
}

__global__ void gather_vec_kernel(const int* __restrict__ ptr, const int* __restrict__ src,
                                  const double* __restrict__ rcontrib, int64_t nrows,
                                  double* __restrict__ out) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrows * 3) return;
  int64_t s = t / 3;
  int c = (int)(t % 3);
  double v = 0.0;
  for (int j = ptr[s]; j < ptr[s + 1]; ++j) v += rcontrib[(int64_t)src[j] * 3 + c];
  out[t] = v;
}

MatParams make_params(const fem_problem* P, double lam) {
  MatParams m;
  m.C = P->mat[0];
  const double bff = P->mat[1], bss = P->mat[2], bnn = P->mat[3], bfs = P->mat[4], bfn = P->mat[5],
               bsn = P->mat[6];
  m.W[0][0] = bff; m.W[0][1] = bfs; m.W[0][2] = bfn;
  m.W[1][0] = bfs; m.W[1][1] = bss; m.W[1][2] = bsn;
  m.W[2][0] = bfn; m.W[2][1] = bsn; m.W[2][2] = bnn;
  m.B = P->mat[7];
  m.fz0 = P->fiber[0]; m.fz1 = P->fiber[1]; m.fa0 = P->fiber[2]; m.fa1 = P->fiber[3];
  m.gamma = lam * P->gamma;
  m.pressure = lam * P->pressure;
  m.nodal = P->fiber_kind == CBDDC_FIBER_NODAL ? 1 : 0;
  m.rho_dt2 = (P->dt > 0.0 && P->rho > 0.0) ? P->rho / (P->dt * P->dt) : 0.0;
  return m;
}

void assemble(fem_problem* P, const double* d, double lam, double* residual, bool want_tangent,
              cudaStream_t s) {
  MatParams mp = make_params(P, lam);
  const int64_t nf = P->n_free_nodes;
  scatter_free_kernel<<<cdiv(3 * nf, 256), 256, 0, s>>>(d, P->free_nodes.p, nf, P->d_full.p);
  CB_LAUNCH();
  // time state: d - 2 d_prev + d_prev2 and (d - d_prev)/dt as node arrays
  const bool timed = P->dt > 0.0;
  if (timed) {
    if (!P->acc_full.p) {
      P->acc_full.alloc((size_t)P->n_nodes * 3);
      P->vel_full.alloc((size_t)P->n_nodes * 3);
      CB_CUDA(cudaMemsetAsync(P->acc_full.p, 0, P->acc_full.bytes(), s));
      CB_CUDA(cudaMemsetAsync(P->vel_full.p, 0, P->vel_full.bytes(), s));
    }
    time_vectors_kernel<<<cdiv(3 * nf, 256), 256, 0, s>>>(d, P->d_prev, P->d_prev2, P->free_nodes.p, nf,
                                                          1.0 / P->dt, P->acc_full.p, P->vel_full.p);
    CB_LAUNCH();
  }
  const double* accf = timed ? P->acc_full.p : nullptr;
  double* fc = P->contrib.p + P->n_elem_blocks * 9;
  double* fr = P->rcontrib.p + P->n_elem_vec * 3;
  const int wt = want_tangent ? 1 : 0;
  timer_begin(CBDDC_TIMER_ELEMENT, s);
  const double* fib = P->fib_nodal.p;
  if (P->tet || P->order == 1) {
    const int epb = TET_THREADS / P->n_qp;
    const int grid = (int)cdiv(P->n_el, epb);
    if (P->tet && P->order == 1)
      qp_element_kernel<4, 1, 0><<<grid, TET_THREADS, 0, s>>>(mp, P->coords.p, P->elems.p, fib, P->d_full.p,
                                                              accf, P->rcontrib.p, P->contrib.p, P->status.p, wt,
                                                              P->n_el);
    else if (P->tet)
      qp_element_kernel<10, 4, 1><<<grid, TET_THREADS, 0, s>>>(mp, P->coords.p, P->elems.p, fib, P->d_full.p,
                                                               accf, P->rcontrib.p, P->contrib.p, P->status.p, wt,
                                                               P->n_el);
    else
      qp_element_kernel<8, 8, 2><<<grid, TET_THREADS, 0, s>>>(mp, P->coords.p, P->elems.p, fib, P->d_full.p,
                                                              accf, P->rcontrib.p, P->contrib.p, P->status.p, wt,
                                                              P->n_el);
  } else {
    element_kernel<2, 256><<<P->n_el, 256, 0, s>>>(mp, P->coords.p, P->elems.p, fib, P->d_full.p,
                                                    accf, P->rcontrib.p, P->contrib.p, P->status.p, wt);
  }
  CB_LAUNCH();
  {
    // algorithmic work of the element kernel: the two-stage contraction
    // (n_qp * n_en * 81 + n_qp * n_en^2 * 27 FMA per element) and the bytes
    // of the element matrices and residuals it writes
    const double nq = P->n_qp, ne = P->n_en;
    const double fl = want_tangent ? 2.0 * P->n_el * (nq * ne * 81.0 + nq * ne * ne * 27.0) : 0.0;
    const double by = 8.0 * P->n_el * (want_tangent ? ne * ne * 9.0 : 0.0) + 8.0 * P->n_el * ne * 3.0;
    timer_end(CBDDC_TIMER_ELEMENT, s, fl, by);
  }
  if (P->n_faces && P->tet) {
    if (P->order == 1)
      tri_face_kernel<1, 32><<<P->n_faces, 32, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                       P->d_full.p, fr, fc, wt);
    else
      tri_face_kernel<2, 64><<<P->n_faces, 64, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                       P->d_full.p, fr, fc, wt);
    CB_LAUNCH();
  } else if (P->n_faces) {
    if (P->order == 1)
      face_kernel<1, 64><<<P->n_faces, 64, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                    P->d_full.p, fr, fc, wt);
    else
      face_kernel<2, 128><<<P->n_faces, 128, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                      P->d_full.p, fr, fc, wt);
    CB_LAUNCH();
  }
  if (P->n_robin) {
    RobinParams rp;
    for (int q = 0; q < 2; ++q)
      for (int c = 0; c < 4; ++c) rp.par[q][c] = P->robin_par[q][c];
    rp.inv_dt = timed ? 1.0 / P->dt : 0.0;
    const int nfn = P->n_fn;
    const int* rfn = P->face_nodes.p + (int64_t)P->n_faces * nfn;
    double* rr = fr + (int64_t)P->n_faces * nfn * 3;
    double* rc = fc + (int64_t)P->n_faces * nfn * nfn * 9;
    const double* vel = timed ? P->vel_full.p : nullptr;
    if (P->tet && P->order == 1)
      robin_face_kernel<true, 1, 32><<<P->n_robin, 32, 0, s>>>(rp, P->coords.p, rfn, P->robin_set.p, P->d_full.p,
                                                               vel, rr, rc, wt);
    else if (P->tet)
      robin_face_kernel<true, 2, 64><<<P->n_robin, 64, 0, s>>>(rp, P->coords.p, rfn, P->robin_set.p, P->d_full.p,
                                                               vel, rr, rc, wt);
    else if (P->order == 1)
      robin_face_kernel<false, 1, 64><<<P->n_robin, 64, 0, s>>>(rp, P->coords.p, rfn, P->robin_set.p,
                                                                P->d_full.p, vel, rr, rc, wt);
    else
      robin_face_kernel<false, 2, 128><<<P->n_robin, 128, 0, s>>>(rp, P->coords.p, rfn, P->robin_set.p,
                                                                  P->d_full.p, vel, rr, rc, wt);
    CB_LAUNCH();
  }
  if (residual) {
    gather_vec_kernel<<<cdiv(3 * nf, 256), 256, 0, s>>>(P->res_ptr.p, P->res_src.p, P->rcontrib.p,
                                                        nf, residual);
    CB_LAUNCH();
  }
  if (want_tangent) {
    gather_blocks_kernel<<<cdiv(9 * P->nnzb, 256), 256, 0, s>>>(
        P->slot_ptr.p, P->slot_src.p, P->contrib.p, P->nnzb, P->bsr_vals.p);
    CB_LAUNCH();
    P->has_tangent = true;
  }
}

// y = K x, three threads per block row: thread 3 i + r forms row r of the
// block row i, walking the row's blocks in order with one FMA per block
// entry of that row (three independent chains) and no reduction between
// threads.  FP64 FMA issue is the roof here (GB300 runs about two FP64 FMAs
// per SM and clock), so all 32 lanes of a warp carry useful FMAs except for
// the length differences of the about eleven block rows a warp holds; the
// 72-byte blocks of those rows are read 24 bytes per thread, and the
// sectors a thread leaves are the ones its row reads next (kept in L1).
__global__ void __launch_bounds__(256)
bsr_spmv_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col, const double* __restrict__ vals,
                const double* __restrict__ x, double* __restrict__ y, int nrows) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 3 * (int64_t)nrows) return;
  const int row = (int)(t / 3), r = (int)(t - 3 * (int64_t)row);
  const int b0 = __ldg(row_ptr + row), b1 = __ldg(row_ptr + row + 1);
  const double* v = vals + (int64_t)b0 * 9 + 3 * r;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0;
#pragma unroll 4
  for (int b = b0; b < b1; ++b, v += 9) {
    const double* xc = x + (int64_t)__ldg(col + b) * 3;
    a0 = fma(__ldg(v), __ldg(xc), a0);
    a1 = fma(__ldg(v + 1), __ldg(xc + 1), a1);
    a2 = fma(__ldg(v + 2), __ldg(xc + 2), a2);
  }
  y[t] = a0 + a1 + a2;
}

void bsr_spmv(const fem_problem* P, const double* x, double* y, cudaStream_t s) {
  const int64_t rows = P->n_free_nodes;
  timer_begin(CBDDC_TIMER_SPMV, s);
  bsr_spmv_kernel<<<cdiv(rows * 3, 256), 256, 0, s>>>(P->bsr_row_ptr.p, P->bsr_col.p,
                                                      P->bsr_vals.p, x, y, (int)rows);
  CB_LAUNCH();
  // bytes: 9 values + 1 column index per block, x read and y written once
  timer_end(CBDDC_TIMER_SPMV, s, 18.0 * P->nnzb, 76.0 * P->nnzb + 16.0 * 3 * rows);
}

}  // namespace cbddc
