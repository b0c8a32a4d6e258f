// Batched dense kernels for the BDDC setup: a grouped GEMM (every batch
// item has its own sizes, offsets and leading dimensions) and the blocked
// Gauss-Jordan "sweep" over a leading range of pivots.
//
// Sweeping the pivots of the leading block A of [[A, B], [C, D]] yields
//   [[A^-1, A^-1 B], [-C A^-1, D - C A^-1 B]]
// in place.  With A = A_II this gives the Dirichlet inverse, the harmonic
// extension, the restriction operator and the Schur complement of
// Section 3.2 in one pass; sweeping a whole matrix inverts it.
//
// Pivot block k (rows/cols kk of width kb <= NB) is processed as
//   P = A_kk^-1 (one CTA per matrix, FP64 Gauss-Jordan in shared memory),
//   X = A[:, kk] with X[kk] = -I,   Y = P A[kk, :] with Y[:, kk] = P,
//   A[kk, :] = 0, A[:, kk] = 0,     A -= X Y   (grouped GEMM, K = kb),
// which is the rank-kb form of the sweep.  No pivoting: a pivot below
// tol * max|diag| (or non-finite) sets DEV_PIVOT in the status word.
#pragma once
#include "common.h"

namespace cbddc {

struct GemmProb {
  int M, N, K;
  int lda, ldb, ldc;
  int64_t a, b, c;  // element offsets from the kernel's base pointers
};

template <typename T> struct GemmCfg;
template <> struct GemmCfg<float> { static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8; };
template <> struct GemmCfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };

// C = alpha op(A) op(B) + beta C for every problem; grid (tilesN, tilesM, nprob).
// Row-major storage; op(A) = A^T reads A as K x M, op(B) = B^T reads B as N x K.
// A problem with K == 0 leaves C untouched (callers use beta = 1 there).
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__((GemmCfg<T>::BM / GemmCfg<T>::TM) * (GemmCfg<T>::BN / GemmCfg<T>::TN))
gemm_grouped_kernel(const GemmProb* __restrict__ probs, const T* __restrict__ A,
                    const T* __restrict__ B, T* __restrict__ C, T alpha, T beta) {
  constexpr int BM = GemmCfg<T>::BM, BN = GemmCfg<T>::BN, BK = GemmCfg<T>::BK;
  constexpr int TM = GemmCfg<T>::TM, TN = GemmCfg<T>::TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  const GemmProb p = probs[blockIdx.z];
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= p.M || n0 >= p.N || p.K <= 0) return;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  const T* Ab = A + p.a;
  const T* Bb = B + p.b;
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);
  for (int k0 = 0; k0 < p.K; k0 += BK) {
    // A tile (BM x BK) -> As[k][m]
#pragma unroll
    for (int t = tid; t < BM * BK; t += NT) {
      int m, k;
      if (TA) { k = t / BM; m = t % BM; } else { m = t / BK; k = t % BK; }
      const int gm = m0 + m, gk = k0 + k;
      T v = T(0);
      if (gm < p.M && gk < p.K) v = TA ? Ab[(int64_t)gk * p.lda + gm] : Ab[(int64_t)gm * p.lda + gk];
      As[k][m] = v;
    }
    // B tile (BK x BN) -> Bs[k][n]
#pragma unroll
    for (int t = tid; t < BN * BK; t += NT) {
      int n, k;
      if (TB) { n = t / BK; k = t % BK; } else { k = t / BN; n = t % BN; }
      const int gn = n0 + n, gk = k0 + k;
      T v = T(0);
      if (gn < p.N && gk < p.K) v = TB ? Bb[(int64_t)gn * p.ldb + gk] : Bb[(int64_t)gk * p.ldb + gn];
      Bs[k][n] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[k][ty * TM + i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[k][tx * TN + j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  T* Cb = C + p.c;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty * TM + i;
    if (gm >= p.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx * TN + j;
      if (gn >= p.N) continue;
      T* cp = Cb + (int64_t)gm * p.ldc + gn;
      *cp = (beta == T(0)) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * *cp;
    }
  }
}

template <typename T, bool TA, bool TB>
void launch_gemm(const GemmProb* probs, int nprob, int maxM, int maxN, const T* A, const T* B, T* C,
                 T alpha, T beta, cudaStream_t s) {
  if (nprob == 0 || maxM <= 0 || maxN <= 0) return;
  constexpr int BM = GemmCfg<T>::BM, BN = GemmCfg<T>::BN;
  constexpr int NT = (BM / GemmCfg<T>::TM) * (BN / GemmCfg<T>::TN);
  dim3 grid(cdiv(maxN, BN), cdiv(maxM, BM), nprob);
  gemm_grouped_kernel<T, TA, TB><<<grid, NT, 0, s>>>(probs, A, B, C, alpha, beta);
  CB_LAUNCH();
}

// --------------------------------------------------------------- sweeps
constexpr int SWEEP_NB = 64;

struct SweepDesc {
  int rows, cols, ld, p;  // matrix shape, leading dimension, pivots to sweep
  int64_t off;            // matrix offset
  int64_t offX;           // X panel offset (rows x NB, ld NB)
  int64_t offY;           // Y panel offset (NB x cols, ld ld)
  int64_t offP;           // diagonal inverse (NB x NB)
};

// P = inverse of the kb x kb diagonal block of pivot step k (FP64 in smem).
template <typename T>
__global__ void __launch_bounds__(256)
sweep_diag_kernel(const SweepDesc* __restrict__ desc, int k, T* __restrict__ mat, T* __restrict__ Pbuf,
                  int* __restrict__ status, double tol) {
  constexpr int NB = SWEEP_NB;
  __shared__ double a[NB][NB + 1];
  __shared__ double fcol[NB];
  __shared__ double piv_scale;
  __shared__ int bad;
  const SweepDesc d = desc[blockIdx.x];
  const int k0 = k * NB;
  if (k0 >= d.p) return;
  const int kb = min(NB, d.p - k0);
  const int tid = threadIdx.x;
  const T* A = mat + d.off;
  for (int t = tid; t < kb * kb; t += blockDim.x) {
    int i = t / kb, j = t % kb;
    a[i][j] = (double)A[(int64_t)(k0 + i) * d.ld + k0 + j];
  }
  if (tid == 0) { bad = 0; piv_scale = 0.0; }
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int i = 0; i < kb; ++i) s = fmax(s, fabs(a[i][i]));
    piv_scale = s;
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    const double pv = a[j][j];
    if (tid == 0 && (!(fabs(pv) > tol * piv_scale) || !isfinite(pv))) bad = 1;
    const double inv = 1.0 / pv;
    if (tid < kb) fcol[tid] = a[tid][j];
    __syncthreads();
    // scale row j (in-place Gauss-Jordan inverse)
    for (int c = tid; c < kb; c += blockDim.x) a[j][c] = (c == j) ? inv : a[j][c] * inv;
    __syncthreads();
    for (int t = tid; t < kb * kb; t += blockDim.x) {
      int i = t / kb, c = t % kb;
      if (i == j) continue;
      const double f = fcol[i];
      if (c == j) a[i][c] = -f * inv;
      else a[i][c] -= f * a[j][c];
    }
    __syncthreads();
  }
  T* P = Pbuf + d.offP;
  for (int t = tid; t < kb * kb; t += blockDim.x) {
    int i = t / kb, j = t % kb;
    P[i * NB + j] = (T)a[i][j];
  }
  if (tid == 0 && bad) atomicOr(status, DEV_PIVOT);
}

// Builds X and Y panels and zeroes the pivot rows/columns, for indices
// [blockIdx.x*64, +64) of each matrix (as columns for Y, as rows for X).
// Reads and writes of different CTAs touch disjoint entries: the Y part
// reads pivot rows outside the pivot columns, the X part reads pivot
// columns outside the pivot rows.
template <typename T>
__global__ void __launch_bounds__(256)
sweep_panel_kernel(const SweepDesc* __restrict__ desc, int k, T* __restrict__ mat,
                   const T* __restrict__ Pbuf, T* __restrict__ Xbuf, T* __restrict__ Ybuf) {
  constexpr int NB = SWEEP_NB, CH = 64;
  __shared__ T Ps[NB][NB + 1];
  __shared__ T col[NB][CH + 1];
  const SweepDesc d = desc[blockIdx.y];
  const int k0 = k * NB;
  if (k0 >= d.p) return;
  const int kb = min(NB, d.p - k0);
  const int c0 = blockIdx.x * CH;
  if (c0 >= d.rows && c0 >= d.cols) return;
  const int cn = c0 < d.cols ? min(CH, d.cols - c0) : 0;   // columns in this chunk
  const int rn = c0 < d.rows ? min(CH, d.rows - c0) : 0;   // rows in this chunk
  const int tid = threadIdx.x;
  T* A = mat + d.off;
  const T* P = Pbuf + d.offP;
  T* X = Xbuf + d.offX;
  T* Y = Ybuf + d.offY;
  for (int t = tid; t < kb * kb; t += blockDim.x) Ps[t / kb][t % kb] = P[(t / kb) * NB + t % kb];
  // pivot rows restricted to this column chunk
  for (int t = tid; t < kb * cn; t += blockDim.x) {
    int r = t / cn, c = t % cn;
    col[r][c] = A[(int64_t)(k0 + r) * d.ld + c0 + c];
  }
  __syncthreads();
  // Y[r, j] = sum_t P[r][t] A[k0+t, j]  (j outside kk),  Y[:, kk] = P
  for (int t = tid; t < kb * cn; t += blockDim.x) {
    int r = t / cn, c = t % cn;
    const int j = c0 + c;
    T v;
    if (j >= k0 && j < k0 + kb) {
      v = Ps[r][j - k0];
    } else {
      T s = T(0);
      for (int q = 0; q < kb; ++q) s = fma(Ps[r][q], col[q][c], s);
      v = s;
    }
    Y[(int64_t)r * d.ld + j] = v;
    A[(int64_t)(k0 + r) * d.ld + j] = T(0);
  }
  // X[i, :] = A[i, kk] (i outside kk), X[kk] = -I ; then A[i, kk] = 0
  for (int t = tid; t < rn * kb; t += blockDim.x) {
    int r = t / kb, q = t % kb;
    const int i = c0 + r;
    T v;
    if (i >= k0 && i < k0 + kb) {
      v = (i - k0 == q) ? T(-1) : T(0);
    } else {
      v = A[(int64_t)i * d.ld + k0 + q];
    }
    X[(int64_t)i * NB + q] = v;
    A[(int64_t)i * d.ld + k0 + q] = T(0);
  }
}

}  // namespace cbddc
