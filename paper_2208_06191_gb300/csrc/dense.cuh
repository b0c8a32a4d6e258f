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
#include <algorithm>
#include <vector>

#include "common.h"
#include "tc_gemm.cuh"

namespace cbddc {

struct GemmProb {
  int M, N, K;
  int lda, ldb, ldc;
  int64_t a, b, c;  // element offsets from the kernel's base pointers
};

// FP32 setup GEMMs run on the tensor cores (tcgen05, split TF32) unless
// this is cleared (cbddc_set_tensor_cores); the FP64 path always uses the
// SIMT kernels.  tc_parts(sweep) is the number of TF32 parts per operand
// (2 or 3) for sweep updates and for the other products, read when a
// context is created.
bool tensor_cores_enabled();
bool tensor_cores_for(bool sweep);  // per kind of list (sweep updates / other products)
bool tc_sweep_ks1();                 // sweep updates accumulate one K-step per TMEM slice
bool tc_other_ks1();                 // the other products too
int tc_parts(bool sweep);

template <typename T> struct GemmCfg;
template <> struct GemmCfg<float> { static constexpr int BM = 128, BN = 128, BK = 16, TM = 8, TN = 8; };
template <> struct GemmCfg<double> { static constexpr int BM = 64, BN = 64, BK = 16, TM = 4, TN = 4; };

// C = alpha op(A) op(B) + beta C for every problem; one CTA per output
// tile, the tiles listed as {problem, tile row, tile column} (only tiles
// that exist, so problems of uneven size launch no empty CTAs).
// Row-major storage; op(A) = A^T reads A as K x M, op(B) = B^T reads B as N x K.
// A problem with K == 0 has no tiles and leaves C untouched (callers use
// beta = 1 there).
template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__((GemmCfg<T>::BM / GemmCfg<T>::TM) * (GemmCfg<T>::BN / GemmCfg<T>::TN))
gemm_grouped_kernel(const int4* __restrict__ tiles, const GemmProb* __restrict__ probs, const T* __restrict__ A,
                    const T* __restrict__ B, T* __restrict__ C, T alpha, T beta) {
  constexpr int BM = GemmCfg<T>::BM, BN = GemmCfg<T>::BN, BK = GemmCfg<T>::BK;
  constexpr int TM = GemmCfg<T>::TM, TN = GemmCfg<T>::TN;
  constexpr int NT = (BM / TM) * (BN / TN);
  const int4 tl = tiles[blockIdx.x];
  const GemmProb p = probs[tl.x];
  const int m0 = tl.y * BM, n0 = tl.z * BN;
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

// Fast path for C = alpha A B + beta C (both operands row-major, not
// transposed): tiles of (32 VEC) x (32 VEC) with VEC = 16 / sizeof(T) (128 x
// 128 for FP32, 64 x 64 for FP64), 256 threads, a 2 VEC x 2 VEC split
// micro-tile per thread.  K slices of 16 go global -> shared with 16-byte
// asynchronous copies (cp.async) through a 3-stage ring, so two slices are
// in flight while one is multiplied, with one barrier per slice.  Operands
// must start on 16-byte boundaries with leading dimensions that are
// multiples of VEC (checked on the host); copies past M, N or K read nothing
// and zero-fill.
template <typename T> struct VecT;
template <> struct VecT<float> { using V = float4; static constexpr int W = 4; };
template <> struct VecT<double> { using V = double2; static constexpr int W = 2; };

template <typename T>
__device__ inline void vstore4(T* dst, const typename VecT<T>::V& v);
template <>
__device__ inline void vstore4<float>(float* d, const float4& v) { d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w; }
template <>
__device__ inline void vstore4<double>(double* d, const double2& v) { d[0] = v.x; d[1] = v.y; }

template <typename T>
__device__ inline typename VecT<T>::V vmask(typename VecT<T>::V v, int valid);
template <>
__device__ inline float4 vmask<float>(float4 v, int valid) {
  if (valid < 4) v.w = 0.f;
  if (valid < 3) v.z = 0.f;
  if (valid < 2) v.y = 0.f;
  if (valid < 1) v.x = 0.f;
  return v;
}
template <>
__device__ inline double2 vmask<double>(double2 v, int valid) {
  if (valid < 2) v.y = 0.0;
  if (valid < 1) v.x = 0.0;
  return v;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T>
__global__ void __launch_bounds__(256, 2)
gemm_nn_kernel(const int4* __restrict__ tiles, const GemmProb* __restrict__ probs, const T* __restrict__ A,
               const T* __restrict__ B, T* __restrict__ C, T alpha, T beta) {
  using V = typename VecT<T>::V;
  constexpr int W = VecT<T>::W;
  constexpr int BM = 32 * W, BN = 32 * W, BK = 16, STAGES = 3;
  constexpr int HALF = BM / 2;
  constexpr int ACH = BK / W;            // 16-byte chunks per A row slice
  static_assert(BM * BK / W == 2 * 256 && BK * BN / W == 2 * 256, "two chunks of A and of B per thread");
  const int4 tl = tiles[blockIdx.x];
  const GemmProb p = probs[tl.x];
  const int m0 = tl.y * BM, n0 = tl.z * BN;
  if (m0 >= p.M || n0 >= p.N || p.K <= 0) return;
  __shared__ __align__(16) T As[STAGES][BM][BK + 4];   // [m][k]
  __shared__ __align__(16) T Bs[STAGES][BK][BN + 4];   // [k][n]
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const T* Ab = A + p.a;
  const T* Bb = B + p.b;
  // issue the copies of K slice kt into stage st (zero-fill outside M, N, K)
  auto load_slice = [&](int kt, int st) {
    const int k0 = kt * BK;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + 256 * h;
      const int row = c / ACH, kq = (c % ACH) * W;
      const int gm = m0 + row, gk = k0 + kq;
      const int valid = (gm < p.M) ? max(0, min(W, p.K - gk)) : 0;
      const T* src = valid > 0 ? Ab + (int64_t)gm * p.lda + gk : Ab;
      cp_async16(&As[st][row][kq], src, valid * (int)sizeof(T));
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int c = tid + 256 * h;
      const int kr = c / (BN / W), nq = (c % (BN / W)) * W;
      const int gk = k0 + kr, gn = n0 + nq;
      const int valid = (gk < p.K) ? max(0, min(W, p.N - gn)) : 0;
      const T* src = valid > 0 ? Bb + (int64_t)gk * p.ldb + gn : Bb;
      cp_async16(&Bs[st][kr][nq], src, valid * (int)sizeof(T));
    }
  };
  const int kTiles = (p.K + BK - 1) / BK;
#pragma unroll
  for (int st = 0; st < STAGES - 1; ++st) {
    if (st < kTiles) load_slice(st, st);
    cp_async_commit();
  }
  // The C tile is prefetched into L2 now, so that the epilogue's reads of
  // C (beta != 0) do not wait on DRAM.
  T* Cb = C + p.c;
  const bool cvec = ((p.c % W) == 0) && ((p.ldc % W) == 0);
  if (beta != T(0)) {
#pragma unroll
    for (int i = 0; i < 2 * W; ++i) {
      const int gm = m0 + (i < W ? ty * W + i : HALF + ty * W + (i - W));
      if (gm < p.M && (tx & 7) == 0) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int gn0 = n0 + h * HALF + tx * W;
          if (gn0 < p.N)
            asm volatile("prefetch.global.L2 [%0];" ::"l"(Cb + (int64_t)gm * p.ldc + gn0));
        }
      }
    }
  }
  T acc[2 * W][2 * W];
#pragma unroll
  for (int i = 0; i < 2 * W; ++i)
#pragma unroll
    for (int j = 0; j < 2 * W; ++j) acc[i][j] = T(0);
  for (int kt = 0; kt < kTiles; ++kt) {
    cp_async_wait<STAGES - 2>();   // slice kt has landed (this thread's copies)
    __syncthreads();               // ... and everyone's; stage (kt-1)%S is free
    if (kt + STAGES - 1 < kTiles) load_slice(kt + STAGES - 1, (kt + STAGES - 1) % STAGES);
    cp_async_commit();
    const int st = kt % STAGES;
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[2 * W], b[2 * W];
#pragma unroll
      for (int i = 0; i < W; ++i) {
        a[i] = As[st][ty * W + i][k];
        a[W + i] = As[st][HALF + ty * W + i][k];
      }
      vstore4<T>(b, *reinterpret_cast<const V*>(&Bs[st][k][tx * W]));
      vstore4<T>(b + W, *reinterpret_cast<const V*>(&Bs[st][k][HALF + tx * W]));
#pragma unroll
      for (int i = 0; i < 2 * W; ++i)
#pragma unroll
        for (int j = 0; j < 2 * W; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
  }
  cp_async_wait<0>();
#pragma unroll
  for (int i = 0; i < 2 * W; ++i) {
    const int gm = m0 + (i < W ? ty * W + i : HALF + ty * W + (i - W));
    if (gm >= p.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gn0 = n0 + h * HALF + tx * W;
      T* cp = Cb + (int64_t)gm * p.ldc + gn0;
      if (cvec && gn0 + W <= p.N) {
        T v[W];
        if (beta != T(0)) vstore4<T>(v, *reinterpret_cast<const V*>(cp));
#pragma unroll
        for (int j = 0; j < W; ++j) v[j] = (beta == T(0)) ? alpha * acc[i][h * W + j] : alpha * acc[i][h * W + j] + beta * v[j];
        V o;
        if constexpr (W == 4) o = V{v[0], v[1], v[2], v[3]};
        else o = V{v[0], v[1]};
        *reinterpret_cast<V*>(cp) = o;
      } else {
#pragma unroll
        for (int j = 0; j < W; ++j) {
          if (gn0 + j >= p.N) break;
          const T v = alpha * acc[i][h * W + j];
          cp[j] = (beta == T(0)) ? v : v + beta * cp[j];
        }
      }
    }
  }
}

// Output tile edge of both GEMM kernels: 128 for FP32, 64 for FP64.
inline int gemm_tile(size_t esize) { return esize == 4 ? 128 : 64; }
static_assert(GemmCfg<float>::BM == 128 && GemmCfg<float>::BN == 128 && 32 * VecT<float>::W == 128, "tile");
static_assert(GemmCfg<double>::BM == 64 && GemmCfg<double>::BN == 64 && 32 * VecT<double>::W == 64, "tile");

// A list of grouped GEMM problems with its output tiles and host-side totals.
// FP32 lists also carry the plan of the tensor-core path: every problem's
// first row in the split operand arrays (op(A): M rows, op(B)^T: N rows, K
// padded to Kp), and, once bound to a scratch buffer, the four TMA maps.
struct GemmList {
  DVec<GemmProb> d;
  DVec<int4> tiles;  // {problem, tile row, tile column, 0}
  int n = 0, ntiles = 0;
  double flops = 0.0, bytes = 0.0;
  bool fast = true;  // every problem meets the vector-load alignment
  // tensor-core plan (FP32 only)
  bool tc_planned = false, tc_bound = false, presplit = false;
  int Kp = 0, maxM = 0, maxN = 0;
  int64_t rowsA = 0, rowsB = 0;
  DVec<tc::TcProb> tcp;
  DVec<tc::SplitProb> spa, spb;
  float* tc_base = nullptr;
  int* tc_status = nullptr;
  int np = 2;  // TF32 parts per operand
  tc::TcMaps maps;
  std::vector<GemmProb> h;  // host copy of the problems
  // order 1: tiles of the largest problems (M N K) first, so that with
  // uneven subdomains the long tile runs of a persistent kernel start early
  void set(const std::vector<GemmProb>& v, size_t esize, bool ta = false, int order = 0) {
    h = v;
    n = (int)v.size();
    flops = bytes = 0.0;
    const int w = (int)(16 / esize);
    const int tile = gemm_tile(esize);
    fast = !ta;
    std::vector<int4> t;
    for (int i = 0; i < n; ++i) {
      const GemmProb& q = v[i];
      if (q.M <= 0 || q.N <= 0 || q.K <= 0) continue;
      flops += 2.0 * q.M * q.N * q.K;
      bytes += (double)esize * (2.0 * q.M * q.N + (double)q.K * (q.M + q.N));
      if (q.a % w || q.b % w || q.lda % w || q.ldb % w) fast = false;
      for (int tm = 0; tm < (int)cdiv(q.M, tile); ++tm)
        for (int tn = 0; tn < (int)cdiv(q.N, tile); ++tn) t.push_back(make_int4(i, tm, tn, 0));
    }
    if (order == 1) {
      auto work = [&](const int4& a) { return (double)v[a.x].M * v[a.x].N * v[a.x].K; };
      std::stable_sort(t.begin(), t.end(), [&](const int4& a, const int4& b) { return work(a) > work(b); });
    }
    ntiles = (int)t.size();
    d.upload(v);
    tiles.upload(t);
    tc_planned = tc_bound = false;
    if (esize == 4 && ntiles > 0 && n <= 65535) plan_tc(v);
  }
  void plan_tc(const std::vector<GemmProb>& v) {
    std::vector<tc::TcProb> tp(n);
    std::vector<tc::SplitProb> sa(n), sb(n);
    int kmax = 0;
    rowsA = rowsB = 0;
    maxM = maxN = 0;
    for (int i = 0; i < n; ++i) {
      const GemmProb& q = v[i];
      const int M = std::max(q.M, 0), N = std::max(q.N, 0), K = std::max(q.K, 0);
      tp[i] = tc::TcProb{M, N, K, q.ldc, q.c, (int)rowsA, (int)rowsB};
      sa[i] = tc::SplitProb{K > 0 ? M : 0, K, q.lda, q.a, (int)rowsA};
      sb[i] = tc::SplitProb{K > 0 ? N : 0, K, q.ldb, q.b, (int)rowsB};
      rowsA += M;
      rowsB += N;
      kmax = std::max(kmax, K);
      maxM = std::max(maxM, M);
      maxN = std::max(maxN, N);
    }
    if (rowsA >= INT32_MAX || rowsB >= INT32_MAX) return;
    Kp = (int)round_up(std::max(kmax, 1), tc::BKC);
    tcp.upload(tp);
    spa.upload(sa);
    spb.upload(sb);
    tc_planned = true;
  }
  // floats of split operands this list needs
  int64_t tc_floats(int parts) const { return tc_planned ? parts * (rowsA + rowsB) * (int64_t)Kp : 0; }
  // Sweep updates whose operands the panel kernel writes already split:
  // op(A) = X at rows a / nb of the [rowsA][nb] hi/lo arrays, op(B)^T =
  // Y^T at rows b / nb of the [rowsB][nb] ones (panel offsets are multiples
  // of nb).
  void bind_presplit(int nb, int parts, float* const* Ap, int64_t rA, float* const* Bp, int64_t rB,
                     int* status) {
    if (ntiles == 0 || n > 65535) return;
    const std::vector<GemmProb>& v = h;
    std::vector<tc::TcProb> tp(n);
    for (int i = 0; i < n; ++i) {
      const GemmProb& q = v[i];
      tp[i] = tc::TcProb{std::max(q.M, 0), std::max(q.N, 0), std::max(q.K, 0), q.ldc, q.c, (int)(q.a / nb),
                         (int)(q.b / nb)};
    }
    tcp.upload(tp);
    Kp = nb;
    rowsA = rA;
    rowsB = rB;
    tc_status = status;
    np = parts;
    for (int q = 0; q < np; ++q) {
      maps.a[q] = tc::encode_kmajor(Ap[q], rA, nb);
      maps.b[q] = tc::encode_kmajor(Bp[q], rB, nb);
    }
    tc_planned = false;  // no split arrays in the shared scratch
    tc_bound = presplit = true;
  }
  // split arrays in the scratch: the parts of op(A) ([rowsA][Kp] each),
  // then those of op(B)^T ([rowsB][Kp] each)
  void bind_tc(float* base, int parts, int* status) {
    if (!tc_planned) return;
    tc_base = base;
    tc_status = status;
    np = parts;
    for (int q = 0; q < np; ++q) {
      maps.a[q] = tc::encode_kmajor(base + q * rowsA * Kp, rowsA, Kp);
      maps.b[q] = tc::encode_kmajor(base + np * rowsA * Kp + q * rowsB * Kp, rowsB, Kp);
    }
    tc_bound = true;
  }
};

// C = alpha op(A) op(B) + beta C for a bound FP32 list on the tensor cores:
// split both operands into the list's K-major hi/lo arrays, then one
// tcgen05 CTA per output tile.
template <bool TA, bool TB>
void launch_tc(const GemmList& g, const float* A, const float* B, float* C, float alpha, float beta,
               cudaStream_t s) {
  if (!g.presplit) {
    float* Ap = g.tc_base;
    float* Bp = Ap + g.np * g.rowsA * g.Kp;
    const dim3 ga(cdiv(g.maxM, 32) * (unsigned)(g.Kp / 32), g.n), gb(cdiv(g.maxN, 32) * (unsigned)(g.Kp / 32), g.n);
    // op(A) rows are A's rows unless TA; op(B)^T rows are B's rows when TB
    if (g.np == 3) {
      tc::tc_split_kernel<!TA, 3><<<ga, 256, 0, s>>>(g.spa.p, g.Kp, A, Ap, g.rowsA * g.Kp);
      CB_LAUNCH();
      tc::tc_split_kernel<TB, 3><<<gb, 256, 0, s>>>(g.spb.p, g.Kp, B, Bp, g.rowsB * g.Kp);
    } else {
      tc::tc_split_kernel<!TA, 2><<<ga, 256, 0, s>>>(g.spa.p, g.Kp, A, Ap, g.rowsA * g.Kp);
      CB_LAUNCH();
      tc::tc_split_kernel<TB, 2><<<gb, 256, 0, s>>>(g.spb.p, g.Kp, B, Bp, g.rowsB * g.Kp);
    }
    CB_LAUNCH();
  }
  tc::set_smem_attr();
  // rank-64 sweep updates (two K chunks) are bound by C's traffic: one
  // operand stage and two C buffers; longer K: two stages and one C buffer
  // (three-part operands: one stage and two C buffers always)
  const int grid = tc::tc_grid(g.ntiles);
  // one K-step per TMEM slice (else a 32-wide K block per slice)
  const bool ks1 = g.presplit ? tc_sweep_ks1() : tc_other_ks1();
#define CB_TC_LAUNCH(NST, NCB, NP, KS)                                                              \
  tc::tc_gemm_kernel<NST, NCB, NP, KS><<<grid, tc::TC_THREADS, tc::TcSmem<NST, NCB, NP>::bytes, s>>>( \
      g.tiles.p, g.ntiles, g.tcp.p, g.maps, C, alpha, beta, g.tc_status)
  if (g.np == 3) {
    if (ks1) CB_TC_LAUNCH(1, 2, 3, 1);
    else CB_TC_LAUNCH(1, 2, 3, 4);
  } else if (g.Kp <= 2 * tc::BKC) {
    if (ks1) CB_TC_LAUNCH(1, 2, 2, 1);
    else CB_TC_LAUNCH(1, 2, 2, 4);
  } else {
    if (ks1) CB_TC_LAUNCH(2, 1, 2, 1);
    else CB_TC_LAUNCH(2, 1, 2, 4);
  }
#undef CB_TC_LAUNCH
  CB_LAUNCH();
}

template <typename T, bool TA, bool TB>
void launch_gemm(const int4* tiles, int ntiles, const GemmProb* probs, const T* A, const T* B, T* C,
                 T alpha, T beta, cudaStream_t s, bool fast = false) {
  if (ntiles == 0) return;
  if (!TA && !TB && fast) {
    gemm_nn_kernel<T><<<ntiles, 256, 0, s>>>(tiles, probs, A, B, C, alpha, beta);
    CB_LAUNCH();
    return;
  }
  constexpr int BM = GemmCfg<T>::BM, BN = GemmCfg<T>::BN;
  constexpr int NT = (BM / GemmCfg<T>::TM) * (BN / GemmCfg<T>::TN);
  gemm_grouped_kernel<T, TA, TB><<<ntiles, NT, 0, s>>>(tiles, probs, A, B, C, alpha, beta);
  CB_LAUNCH();
}

// Launch of a whole list (timed as a setup GEMM when the timer follows
// them: FP32 lists in class SETUP_GEMM, FP64 ones in SETUP_GEMM_F64).
template <typename T, bool TA, bool TB>
void launch_list(const GemmList& g, const T* A, const T* B, T* C, T alpha, T beta, cudaStream_t s) {
  if (g.ntiles == 0) return;
  const int cls = sizeof(T) == 4 ? CBDDC_TIMER_SWEEP_GEMM : CBDDC_TIMER_SETUP_GEMM_F64;
  timer_begin(cls, s);
  if constexpr (sizeof(T) == 4) {
    if (g.tc_bound && tensor_cores_for(g.presplit)) {
      launch_tc<TA, TB>(g, A, B, C, alpha, beta, s);
      timer_end(cls, s, g.flops, g.bytes);
      return;
    }
  }
  launch_gemm<T, TA, TB>(g.tiles.p, g.ntiles, g.d.p, A, B, C, alpha, beta, s, g.fast);
  timer_end(cls, s, g.flops, g.bytes);
}

// --------------------------------------------------------------- sweeps
// Pivot block width of the sweeps: 64 (FP64 operators, and the FP32 default)
// or 128 (FP32; half the passes over each matrix for the same flops).
constexpr int SWEEP_NB = 64;
constexpr int SWEEP_NB_MAX = 128;

struct SweepDesc {
  int rows, cols, ld, p;  // matrix shape, leading dimension, pivots to sweep
  int64_t off;            // matrix offset
  int64_t offX;           // X panel offset (rows x NB, ld NB)
  int64_t offY;           // Y panel offset (NB x cols, ld ld)
  int64_t offP;           // diagonal inverse (NB x NB)
};

// P = inverse of the kb x kb diagonal block of pivot step k, by Gauss-Jordan
// in the operator precision T.  Thread (c, g) = (tid % NB, tid / NB) keeps
// RG rows of column c in registers (16 of 256 threads for NB = 64, 32 of
// 512 for NB = 128), so all four SM sub-partitions stay busy (the FP64
// coarse matrix needs every FP64 unit).  At pivot j every thread reads
// the old pivot column and pivot row from a double-buffered shared copy,
// updates its entries
//   a[j][c] <- a[j][c] / p,  a[i][c] <- a[i][c] - a[i][j] a[j][c] / p (c != j),
//   a[i][j] <- -a[i][j] / p, a[j][j] <- 1 / p,
// and the owners of column j + 1 and row j + 1 publish them into the other
// buffer, so one barrier per pivot suffices.
// Threads of the diagonal-block kernel: 256 for NB = 64 (16 rows of one
// column per thread), 512 for NB = 128 (32 rows per thread).
template <int NB>
struct DiagThreads { static constexpr int value = NB <= 64 ? 256 : 512; };
constexpr int DIAG_THREADS = 256;
template <typename T, int NB>
__global__ void __launch_bounds__(DiagThreads<NB>::value)
sweep_diag_kernel(const SweepDesc* __restrict__ desc, int k, T* __restrict__ mat, T* __restrict__ Pbuf,
                  int* __restrict__ status, double tol) {
  constexpr int NT = DiagThreads<NB>::value;
  constexpr int RG = NB / (NT / NB);  // rows per thread
  __shared__ T colb[2][NB], rowb[2][NB];
  __shared__ double piv_scale;
  __shared__ int bad;
  const SweepDesc d = desc[blockIdx.x];
  const int k0 = k * NB;
  if (k0 >= d.p) return;
  const int kb = min(NB, d.p - k0);
  const int tid = threadIdx.x;
  const int c = tid % NB, r0 = (tid / NB) * RG;
  const T* A = mat + d.off + (int64_t)k0 * d.ld + k0;
  if (tid == 0) bad = 0;
  T a[RG];
#pragma unroll
  for (int q = 0; q < RG; ++q)
    a[q] = (r0 + q < kb && c < kb) ? A[(int64_t)(r0 + q) * d.ld + c] : T(0);
  if (c == 0) {
#pragma unroll
    for (int q = 0; q < RG; ++q) colb[0][r0 + q] = a[q];
  }
  if (r0 == 0) rowb[0][c] = a[0];
  // scale of the pivots: largest |diagonal| of the block
  if (tid < 32) {
    double dv = 0.0;
    for (int i = tid; i < kb; i += 32) dv = fmax(dv, fabs((double)A[(int64_t)i * d.ld + i]));
    for (int o = 16; o > 0; o >>= 1) dv = fmax(dv, __shfl_xor_sync(0xffffffffu, dv, o));
    if (tid == 0) piv_scale = dv;
  }
  __syncthreads();
  const double scale = piv_scale;
  for (int j = 0; j < kb; ++j) {
    const int b = j & 1, nb = b ^ 1;
    const T pv = rowb[b][j];
    const T rj = rowb[b][c];
    const T inv = T(1) / pv;
    if (c < kb) {
      if (c == j) {
#pragma unroll
        for (int q = 0; q < RG; ++q) a[q] = (r0 + q == j) ? inv : -colb[b][r0 + q] * inv;
      } else {
        const T t = rj * inv;
#pragma unroll
        for (int q = 0; q < RG; ++q) a[q] = (r0 + q == j) ? t : a[q] - colb[b][r0 + q] * t;
      }
    }
    if (j + 1 < kb) {
      if (c == j + 1) {
#pragma unroll
        for (int q = 0; q < RG; ++q) colb[nb][r0 + q] = a[q];
      }
      const int jr = j + 1 - r0;
      if (jr >= 0 && jr < RG) {
        T v = T(0);
#pragma unroll
        for (int q = 0; q < RG; ++q)
          if (q == jr) v = a[q];
        rowb[nb][c] = v;
      }
    }
    if (tid == 0 && (!(fabs((double)pv) > tol * scale) || !isfinite((double)pv))) bad = 1;
    __syncthreads();
  }
  T* P = Pbuf + d.offP;
  if (c < kb) {
#pragma unroll
    for (int q = 0; q < RG; ++q)
      if (r0 + q < kb) P[(r0 + q) * NB + c] = a[q];
  }
  if (tid == 0 && bad) atomicOr(status, DEV_PIVOT);
}

// Builds X and Y panels and zeroes the pivot rows/columns, for indices
// [blockIdx.x*PANEL_CH, +PANEL_CH) of each matrix (as columns for Y, as rows
// for X).  Reads and writes of different CTAs touch disjoint entries: the Y
// part reads pivot rows outside the pivot columns, the X part reads pivot
// columns outside the pivot rows (the pivot block itself is read only into
// Y entries that are replaced by P).  Narrow chunks keep many CTAs in flight
// (a single coarse matrix still spreads over the GPU); each thread forms
// NB / 16 rows of one Y column and gathers its NB / 16 X entries before
// storing.  Shared memory (dynamic): P (NB x NB+1) and the chunk of pivot
// rows (NB x CH+1).
constexpr int PANEL_CH = 16;
template <typename T, int NB>
constexpr size_t panel_smem_bytes() {
  return sizeof(T) * ((size_t)NB * (NB + 1) + (size_t)NB * (PANEL_CH + 1));
}

//
// NP > 0 (FP32 operators on the tensor cores): the panels are written as the
// K-major TF32 parts of the update GEMM's operands instead, X parts (rows x
// NB) at Xbuf, Xlo (, Xlo2) and Y^T parts (columns x NB) at Ybuf, Ylo (,
// Ylo2), with zeros beyond the kb pivots of a partial last block, so the
// update needs no separate split pass.
template <typename T, int NB, int NP>
__global__ void __launch_bounds__(256)
sweep_panel_kernel(const SweepDesc* __restrict__ desc, int k, T* __restrict__ mat,
                   const T* __restrict__ Pbuf, T* __restrict__ Xbuf, T* __restrict__ Ybuf,
                   T* __restrict__ Xlo, T* __restrict__ Ylo, T* __restrict__ Xlo2, T* __restrict__ Ylo2) {
  constexpr bool SPLIT = NP > 0;
  constexpr int CH = PANEL_CH, PER = NB * CH / 256, RY = NB / 16;
  static_assert(CH == 16 && NB % 16 == 0, "NB / 16 rows of one column per thread");
  extern __shared__ __align__(16) unsigned char panel_smem[];
  T (*Ps)[NB + 1] = reinterpret_cast<T (*)[NB + 1]>(panel_smem);
  T (*col)[CH + 1] = reinterpret_cast<T (*)[CH + 1]>(panel_smem + sizeof(T) * NB * (NB + 1));
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
  if (cn > 0) {
    for (int t = tid; t < NB * NB; t += 256) {
      const int r = t / NB, q = t % NB;
      Ps[r][q] = (r < kb && q < kb) ? P[r * NB + q] : T(0);
    }
    // pivot rows restricted to this column chunk (zero outside kb x cn)
    for (int t = tid; t < NB * CH; t += 256) {
      const int r = t / CH, cc = t % CH;
      col[r][cc] = (r < kb && cc < cn) ? A[(int64_t)(k0 + r) * d.ld + c0 + cc] : T(0);
    }
  }
  // X[i, :] = A[i, kk] (i outside kk), X[kk] = -I ; then A[i, kk] = 0
  if (rn > 0) {
    T xv[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int t = tid + 256 * u, r = t / NB, q = t % NB, i = c0 + r;
      xv[u] = (r < rn && q < kb && !(i >= k0 && i < k0 + kb)) ? A[(int64_t)i * d.ld + k0 + q] : T(0);
    }
#pragma unroll
    for (int u = 0; u < PER; ++u) {
      const int t = tid + 256 * u, r = t / NB, q = t % NB, i = c0 + r;
      if (SPLIT) {
        if (r < rn) {
          const bool piv = i >= k0 && i < k0 + kb;
          const T x = q < kb ? (piv ? ((i - k0 == q) ? T(-1) : T(0)) : xv[u]) : T(0);
          float parts[3];
          tc::split_tf32<NP == 3 ? 3 : 2>((float)x, parts);
          X[(int64_t)i * NB + q] = parts[0];
          Xlo[d.offX + (int64_t)i * NB + q] = parts[1];
          if (NP == 3) Xlo2[d.offX + (int64_t)i * NB + q] = parts[2];
          if (q < kb) A[(int64_t)i * d.ld + k0 + q] = T(0);
        }
      } else if (r < rn && q < kb) {
        const bool piv = i >= k0 && i < k0 + kb;
        X[(int64_t)i * NB + q] = piv ? ((i - k0 == q) ? T(-1) : T(0)) : xv[u];
        A[(int64_t)i * d.ld + k0 + q] = T(0);
      }
    }
  }
  if (cn == 0) return;
  __syncthreads();
  // Y[r, j] = sum_q P[r][q] A[k0+q, j]  (j outside kk),  Y[:, kk] = P
  const int ty = tid / CH, c = tid % CH;   // rows RY ty .. RY ty + RY - 1 of column c
  T acc[RY];
#pragma unroll
  for (int i = 0; i < RY; ++i) acc[i] = T(0);
  for (int q = 0; q < kb; ++q) {
    const T cq = col[q][c];
#pragma unroll
    for (int i = 0; i < RY; ++i) acc[i] = fma(Ps[RY * ty + i][q], cq, acc[i]);
  }
  if (c >= cn) return;
  const int jg = c0 + c;
  const bool pivc = jg >= k0 && jg < k0 + kb;
#pragma unroll
  for (int i = 0; i < RY; ++i) {
    const int r = RY * ty + i;
    if (SPLIT) {
      // Y^T row jg, K index r (zero beyond kb)
      const T y = r < kb ? (pivc ? Ps[r][jg - k0] : acc[i]) : T(0);
      float parts[3];
      tc::split_tf32<NP == 3 ? 3 : 2>((float)y, parts);
      Y[(int64_t)jg * NB + r] = parts[0];
      Ylo[d.offY + (int64_t)jg * NB + r] = parts[1];
      if (NP == 3) Ylo2[d.offY + (int64_t)jg * NB + r] = parts[2];
      if (r < kb) A[(int64_t)(k0 + r) * d.ld + jg] = T(0);
      continue;
    }
    if (r >= kb) continue;
    Y[(int64_t)r * d.ld + jg] = pivc ? Ps[r][jg - k0] : acc[i];
    A[(int64_t)(k0 + r) * d.ld + jg] = T(0);
  }
}

}  // namespace cbddc
