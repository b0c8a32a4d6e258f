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

void init_shape_tables(int /*order*/) {
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
  for (int i = 0; i < 3; ++i)
    for (int Jx = 0; Jx < 3; ++Jx)
      for (int k = 0; k < 3; ++k)
        for (int L = 0; L < 3; ++L) {
          double lin = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              lin += m.W[a][b] * g[a][i] * R[Jx][b] * (g[a][k] * R[L][b] + g[b][k] * R[L][a]);
          double v = eQ * (2.0 * FS[i][Jx] * FS[k][L] + 0.5 * lin);
          if (i == k) v += eQ * Sh[L][Jx];
          v += J * dkap * Fi[Jx][i] * Fi[L][k] - kap * Fi[Jx][k] * Fi[L][i];
          v += ga * ((i == k ? 1.0 : 0.0) - mv[i] * mv[k]) * f[Jx] * f[L];
          A[((i * 3 + Jx) * 3 + k) * 3 + L] = v;
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
               const double* __restrict__ d_full, double* __restrict__ rcontrib,
               double* __restrict__ contrib, int* __restrict__ status, int want_tangent) {
  constexpr int M = K + 1, NEN = M * M * M, NQ = NEN;
  constexpr int O = K - 1;
  __shared__ double X[NEN][3], U[NEN][3];
  __shared__ double G[NQ][NEN][3];
  __shared__ double Wd[NQ];
  __shared__ double Pq[NQ][9];
  __shared__ double Aq[NQ][81];
  __shared__ double T[NEN * 27];
  __shared__ int bad;
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
    double Xq[3] = {0, 0, 0};
    for (int a = 0; a < NEN; ++a) {
      const int ax = a % M, ay = (a / M) % M, az = a / (M * M);
      const double lx = c_L[O][qx][ax], ly = c_L[O][qy][ay], lz = c_L[O][qz][az];
      const double dn[3] = {c_dL[O][qx][ax] * ly * lz, lx * c_dL[O][qy][ay] * lz,
                            lx * ly * c_dL[O][qz][az]};
      const double n = lx * ly * lz;
      for (int i = 0; i < 3; ++i) {
        Xq[i] += n * X[a][i];
        for (int j = 0; j < 3; ++j) J0[i][j] += X[a][i] * dn[j];
      }
      G[q][a][0] = dn[0];
      G[q][a][1] = dn[1];
      G[q][a][2] = dn[2];
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
    fibre_frame(mp, Xq, R);
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
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int t = tid + j * THREADS;
    if (t < NE) contrib[(int64_t)e * NE + t] = acc[j];
  }
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
  return m;
}

void assemble(fem_problem* P, const double* d, double lam, double* residual, bool want_tangent,
              cudaStream_t s) {
  MatParams mp = make_params(P, lam);
  const int64_t nf = P->n_free_nodes;
  scatter_free_kernel<<<cdiv(3 * nf, 256), 256, 0, s>>>(d, P->free_nodes.p, nf, P->d_full.p);
  CB_LAUNCH();
  double* fc = P->contrib.p + P->n_elem_blocks * 9;
  double* fr = P->rcontrib.p + P->n_elem_vec * 3;
  const int wt = want_tangent ? 1 : 0;
  timer_begin(CBDDC_TIMER_ELEMENT, s);
  if (P->order == 1)
    element_kernel<1, 64><<<P->n_el, 64, 0, s>>>(mp, P->coords.p, P->elems.p, P->d_full.p,
                                                  P->rcontrib.p, P->contrib.p, P->status.p, wt);
  else
    element_kernel<2, 256><<<P->n_el, 256, 0, s>>>(mp, P->coords.p, P->elems.p, P->d_full.p,
                                                    P->rcontrib.p, P->contrib.p, P->status.p, wt);
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
  if (P->n_faces) {
    if (P->order == 1)
      face_kernel<1, 64><<<P->n_faces, 64, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                    P->d_full.p, fr, fc, wt);
    else
      face_kernel<2, 128><<<P->n_faces, 128, 0, s>>>(mp.pressure, P->coords.p, P->face_nodes.p,
                                                      P->d_full.p, fr, fc, wt);
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

// y = K x, 3x3 BSR, one warp per block row.  Lane L < 24 owns row
// r = L % 3 of the blocks k, k + 8, k + 16, ... (k = L / 3): each value costs
// one FP64 FMA (FP64 issue is the scarce resource here), loads stay within
// the row's contiguous value segment, and three shuffle steps (12, 6, 3)
// sum the eight partial rows.
__global__ void bsr_spmv_kernel(const int* __restrict__ row_ptr, const int* __restrict__ col,
                                const double* __restrict__ vals, const double* __restrict__ x,
                                double* __restrict__ y, int nrows) {
  const int row = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nrows) return;
  const int b0 = row_ptr[row], nb = row_ptr[row + 1] - b0;
  const int r = lane % 3, k = lane / 3;
  double acc = 0.0;
  if (lane < 24) {
    const double* v = vals + (int64_t)b0 * 9 + r * 3;
    const int* c = col + b0;
#pragma unroll 4
    for (int b = k; b < nb; b += 8) {
      const double* vb = v + (int64_t)b * 9;
      const double* xb = x + (int64_t)__ldg(c + b) * 3;
      acc = fma(__ldcs(vb + 0), __ldg(xb + 0), acc);
      acc = fma(__ldcs(vb + 1), __ldg(xb + 1), acc);
      acc = fma(__ldcs(vb + 2), __ldg(xb + 2), acc);
    }
  }
  acc += __shfl_down_sync(0xffffffffu, acc, 12);
  acc += __shfl_down_sync(0xffffffffu, acc, 6);
  acc += __shfl_down_sync(0xffffffffu, acc, 3);
  if (lane < 3) y[(int64_t)row * 3 + lane] = acc;
}

void bsr_spmv(const fem_problem* P, const double* x, double* y, cudaStream_t s) {
  const int64_t rows = P->n_free_nodes;
  timer_begin(CBDDC_TIMER_SPMV, s);
  bsr_spmv_kernel<<<cdiv(rows * 32, 256), 256, 0, s>>>(P->bsr_row_ptr.p, P->bsr_col.p,
                                                       P->bsr_vals.p, x, y, (int)rows);
  CB_LAUNCH();
  // bytes: 9 values + 1 column index per block, x read and y written once
  timer_end(CBDDC_TIMER_SPMV, s, 18.0 * P->nnzb, 76.0 * P->nnzb + 16.0 * 3 * rows);
}

}  // namespace cbddc
