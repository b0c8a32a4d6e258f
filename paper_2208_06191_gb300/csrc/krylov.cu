// Flexible GMRES (FP64) preconditioned by BDDC, and the Newton iteration of
// Eq. (tangent problem): d^{n,k} = d^{n,k-1} + delta, DF(d) delta = -F(d).
//
// GMRES: Arnoldi basis V (column j contiguous), preconditioned vectors
// Z_j = M^-1 v_j, classical Gram-Schmidt applied twice (two passes of
// h = V^T w, w -= V h), Givens rotations and the least-squares residual
// |g_{j+1}| kept on the device; restart after m steps with the true
// residual recomputed.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "bddc.h"
#include "fem.h"
#include "krylov.h"

namespace cbddc {

namespace cg = cooperative_groups;

namespace {

constexpr int DOT_THREADS = 256;
constexpr int64_t kCoopMaxN = 1000000;  // longest vector for the cooperative orthogonalisation
constexpr int MAXV = 128;       // Krylov vectors of the cooperative orthogonalisation
constexpr int MAXR = 1024;      // Krylov vectors per cycle (restart <= MAXR - 1)

__device__ inline double wsum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block dot products with a last-block reduction.  Each CTA owns a tile of
// 256 * RPT consecutive rows: it first forms its rows of w (optionally
// w -= V hin, which fuses the update of one Gram-Schmidt pass with the dots
// of the next), keeps them in shared memory, then every warp takes whole
// columns of V and reads the tile's rows of that column with all 32 lanes
// (coalesced, 8 * RPT independent loads per lane), so the reduction costs
// one warp sum per column and CTA.  The CTA that finishes last (atomic
// ticket) sums the per-CTA partials in CTA order, so results do not depend
// on scheduling.
struct DotArgs {
  const double* V;      // nvec columns of length n, stride ldv
  int64_t ldv;
  int nvec;
  double* w;            // [n]
  int64_t n;
  const double* hin;    // if non-null: w -= V hin before the dots
  int self_norm;        // dots of w with itself instead of with V
  double* partial;      // [gridDim.x][pstride]
  int pstride;          // row stride of partial (>= nvec)
  unsigned* ticket;     // zero on entry, reset by the last CTA
  double* out;          // [nvec] (or [1] for the norm)
  const int* done;      // skip everything once GMRES has converged
  const int* gate;      // if non-null: skip unless *gate != 0
  int also_norm;        // dots with V plus out[nvec] = ||w||^2 (before any update)
};

__device__ inline void last_block_sum(const DotArgs& a, int nout) {
  __shared__ bool last;
  __shared__ double half[MAXV];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  // two threads per output: CTAs [0, G/2) and [G/2, G), four accumulators
  // each in a fixed order, then the halves added in a fixed order; outputs
  // in chunks of 128
  const int jl = threadIdx.x & (MAXV - 1), side = threadIdx.x >> 7;
  const unsigned G = gridDim.x, mid = G / 2;
  const unsigned c0 = side ? mid : 0u, c1 = side ? G : mid;
  for (int j0 = 0; j0 < nout; j0 += MAXV) {
    const int j = j0 + jl;
    double s4[4] = {0.0, 0.0, 0.0, 0.0};
    if (j < nout) {
      unsigned c = c0;
      for (; c + 4 <= c1; c += 4) {
#pragma unroll
        for (int q = 0; q < 4; ++q) s4[q] += __ldcg(a.partial + (int64_t)(c + q) * a.pstride + j);
      }
      for (; c < c1; ++c) s4[0] += __ldcg(a.partial + (int64_t)c * a.pstride + j);
    }
    const double sum = (s4[0] + s4[1]) + (s4[2] + s4[3]);
    if (side == 1 && j < nout) half[jl] = sum;
    __syncthreads();
    if (side == 0 && j < nout) a.out[j] = sum + half[jl];
    __syncthreads();
  }
  if (threadIdx.x == 0) *a.ticket = 0u;
  __threadfence();
}

template <int RPT>
__global__ void __launch_bounds__(DOT_THREADS) fused_dots_kernel(DotArgs a) {
  if (a.done && *a.done) return;
  if (a.gate && !*a.gate) return;
  constexpr int TILE = DOT_THREADS * RPT;
  __shared__ double ws[TILE];
  __shared__ double hs[MAXR];
  __shared__ double red[DOT_THREADS / 32];
  const int64_t r0 = (int64_t)blockIdx.x * TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int rows = (int)min((int64_t)TILE, a.n - r0);
  // rows of w (updated when hin is given)
  double x[RPT];
#pragma unroll
  for (int t = 0; t < RPT; ++t) {
    const int q = tid + DOT_THREADS * t;
    x[t] = q < rows ? a.w[r0 + q] : 0.0;
  }
  if (a.hin) {
    for (int j = tid; j < a.nvec; j += DOT_THREADS) hs[j] = a.hin[j];
    __syncthreads();
    for (int j = 0; j < a.nvec; ++j) {
      const double hj = hs[j];
      const double* Vj = a.V + (int64_t)j * a.ldv + r0;
#pragma unroll
      for (int t = 0; t < RPT; ++t) {
        const int q = tid + DOT_THREADS * t;
        if (q < rows) x[t] -= Vj[q] * hj;
      }
    }
#pragma unroll
    for (int t = 0; t < RPT; ++t) {
      const int q = tid + DOT_THREADS * t;
      if (q < rows) a.w[r0 + q] = x[t];
    }
  }
  const int nout = a.self_norm ? 1 : a.nvec + (a.also_norm ? 1 : 0);
  if (a.also_norm && !a.self_norm) {
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < RPT; ++t) acc += x[t] * x[t];
    acc = wsum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double sm = 0.0;
      for (int q = 0; q < DOT_THREADS / 32; ++q) sm += red[q];
      a.partial[(int64_t)blockIdx.x * a.pstride + a.nvec] = sm;
    }
  }
  if (a.self_norm) {
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < RPT; ++t) acc += x[t] * x[t];
    acc = wsum(acc);
    if (lane == 0) red[warp] = acc;
    __syncthreads();
    if (tid == 0) {
      double sm = 0.0;
      for (int q = 0; q < DOT_THREADS / 32; ++q) sm += red[q];
      a.partial[(int64_t)blockIdx.x * a.pstride] = sm;
    }
  } else {
#pragma unroll
    for (int t = 0; t < RPT; ++t) ws[tid + DOT_THREADS * t] = x[t];
    __syncthreads();
    for (int j = warp; j < a.nvec; j += DOT_THREADS / 32) {
      const double* Vj = a.V + (int64_t)j * a.ldv + r0;
      double acc = 0.0;
#pragma unroll 8
      for (int q = lane; q < TILE; q += 32)
        if (q < rows) acc += Vj[q] * ws[q];
      acc = wsum(acc);
      if (lane == 0) a.partial[(int64_t)blockIdx.x * a.pstride + j] = acc;
    }
  }
  last_block_sum(a, nout);
}

// Column j of the Hessenberg matrix from h1 + h2 (the two CGS passes) and
// ||w||^2, previous rotations, the new rotation and the residual estimate.
// scal[0] = |g_{j+1}| / ||b||, scal[1] = 1 / h_{j+1,j}, scal[2] = ||b||.
__device__ void givens_update(int j, int m, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, const double* h1,
                              const double* h2, double wn2, double* __restrict__ scal, double rtol,
                              int* __restrict__ done, int* __restrict__ iters) {
  double* col = H + (int64_t)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h2 ? h1[i] + h2[i] : h1[i];
  const double hn = sqrt(fmax(wn2, 0.0));
  col[j + 1] = hn;
  scal[1] = hn > 0.0 ? 1.0 / hn : 0.0;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  cs[j] = den > 0.0 ? col[j] / den : 1.0;
  sn[j] = den > 0.0 ? col[j + 1] / den : 0.0;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  const double res = fabs(g[j + 1]) / scal[2];
  scal[0] = res;
  *iters += 1;
  if (res <= rtol || hn == 0.0) *done = 1;
}

__global__ void givens_kernel(int j, int m, double* __restrict__ H, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g,
                              const double* __restrict__ h1, const double* __restrict__ h2,
                              const double* __restrict__ wn2, double* __restrict__ scal, double rtol,
                              int* __restrict__ done, int* __restrict__ iters) {
  if (*done) return;
  givens_update(j, m, H, cs, sn, g, h1, h2, wn2[0], scal, rtol, done, iters);
}

// The whole orthogonalisation of one Arnoldi step in one cooperative launch
// (all CTAs resident, grid-wide barriers): h1 = V^T w; w -= V h1, h2 = V^T w;
// w -= V h2, ||w||^2; the Givens update (CTA 0) and v_{j+1} = w / ||w||.
// Row tiles of 256 go to the CTAs round-robin; each warp keeps partial dot
// products of its columns in registers across tiles, every CTA writes its
// partials, and after each barrier every CTA sums all CTAs' partials in CTA
// order (identical on every CTA, independent of scheduling).  This replaces
// five launches and their tails, which dominate at small n.
struct CgsArgs {
  const double* V;   // nvec columns of length n (stride n)
  int64_t n;
  int nvec;          // j + 1
  double* w;
  double* vnext;     // column j + 1
  double* part;      // [3][gridDim.x][MAXV]
  int j, m;
  double *H, *cs, *sn, *g, *scal;
  double rtol;
  int *done, *iters;
};

__device__ void cgs_phase(const CgsArgs& a, const double* hin, bool norm, double* ws, double* part) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int CPW = MAXV / (DOT_THREADS / 32);  // columns per warp
  double acc[CPW];
#pragma unroll
  for (int q = 0; q < CPW; ++q) acc[q] = 0.0;
  double nacc = 0.0;
  const int64_t ntiles = (a.n + DOT_THREADS - 1) / DOT_THREADS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r0 = t * DOT_THREADS;
    const int rows = (int)min((int64_t)DOT_THREADS, a.n - r0);
    double x = tid < rows ? a.w[r0 + tid] : 0.0;
    if (hin && tid < rows) {
      for (int j = 0; j < a.nvec; ++j) x -= a.V[(int64_t)j * a.n + r0 + tid] * hin[j];
      a.w[r0 + tid] = x;
    }
    if (norm) {
      nacc += x * x;
    } else {
      __syncthreads();   // the previous tile's readers of ws are done
      ws[tid] = x;
      __syncthreads();
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        const int j = warp + (DOT_THREADS / 32) * q;
        if (j < a.nvec) {
          const double* Vj = a.V + (int64_t)j * a.n + r0;
          for (int rr = lane; rr < rows; rr += 32) acc[q] += Vj[rr] * ws[rr];
        }
      }
    }
  }
  __shared__ double red[DOT_THREADS / 32];
  if (norm) {
    nacc = wsum(nacc);
    if (lane == 0) red[warp] = nacc;
    __syncthreads();
    if (tid == 0) {
      double sm = 0.0;
      for (int q = 0; q < DOT_THREADS / 32; ++q) sm += red[q];
      part[(int64_t)blockIdx.x * MAXV] = sm;
    }
  } else {
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int j = warp + (DOT_THREADS / 32) * q;
      const double v = wsum(acc[q]);
      if (lane == 0 && j < a.nvec) part[(int64_t)blockIdx.x * MAXV + j] = v;
    }
  }
}

// sums of every CTA's partials into out[0:nout] (shared memory): 4 threads
// per output, each over every 4th CTA, combined in a fixed order (identical
// on every CTA, independent of scheduling)
__device__ void cgs_reduce(const double* part, int nout, double* out) {
  __shared__ double red4[4][64];
  const int jl = threadIdx.x & 63, grp = threadIdx.x >> 6;
  for (int j0 = 0; j0 < nout; j0 += 64) {
    const int j = j0 + jl;
    double sacc = 0.0;
    if (j < nout)
      for (unsigned c = grp; c < gridDim.x; c += 4) sacc += __ldcg(part + (int64_t)c * MAXV + j);
    red4[grp][jl] = sacc;
    __syncthreads();
    if (grp == 0 && j < nout) out[j] = (red4[0][jl] + red4[1][jl]) + (red4[2][jl] + red4[3][jl]);
    __syncthreads();
  }
}

__global__ void __launch_bounds__(DOT_THREADS) cgs2_coop_kernel(CgsArgs a) {
  cg::grid_group grid = cg::this_grid();
  if (*a.done) return;  // read by every CTA before any barrier: uniform
  __shared__ double ws[DOT_THREADS];
  __shared__ double h1[MAXV], h2[MAXV], wn2s[1];
  const int64_t stride = (int64_t)gridDim.x * MAXV;
  cgs_phase(a, nullptr, false, ws, a.part);
  grid.sync();
  cgs_reduce(a.part, a.nvec, h1);
  cgs_phase(a, h1, false, ws, a.part + stride);
  grid.sync();
  cgs_reduce(a.part + stride, a.nvec, h2);
  cgs_phase(a, h2, true, ws, a.part + 2 * stride);
  grid.sync();
  cgs_reduce(a.part + 2 * stride, 1, wn2s);
  if (blockIdx.x == 0 && threadIdx.x == 0)
    givens_update(a.j, a.m, a.H, a.cs, a.sn, a.g, h1, h2, wn2s[0], a.scal, a.rtol, a.done, a.iters);
  // v_{j+1} = w / ||w|| (the same value on every CTA)
  const double hn = sqrt(fmax(wn2s[0], 0.0));
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  const int64_t ntiles = (a.n + DOT_THREADS - 1) / DOT_THREADS;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int64_t r = t * DOT_THREADS + threadIdx.x;
    if (r < a.n) a.vnext[r] = a.w[r] * inv;
  }
}

// The Arnoldi step for long vectors or long bases in one cooperative
// launch, by modified Gram-Schmidt (backward stable for GMRES without a
// second pass, and the oracle's orthogonalisation): each thread keeps
// RPT rows of w in registers (32-row slices of its warp's segment); for
// i = 0..j: h_i = v_i . w (block sums, one grid-wide barrier, every CTA
// adds the CTA partials in CTA order), w -= h_i v_i; then ||w||, the
// Givens update (CTA 0) and v_{j+1} = w / ||w||.  V is read once per step
// (the update re-reads the rows of v_i that the thread has just read), and
// every FP64 FMA of the step is one of the 2 (j + 1) n of MGS.
constexpr int MGS_THREADS = 640;
struct MgsArgs {
  const double* V;   // j + 1 columns of length n (stride n)
  int64_t n;
  double* w;
  double* vnext;
  double* part;      // [2][gridDim.x]
  double* hcol;      // [m + 1]: this step's Hessenberg column
  int j, m;
  double *H, *cs, *sn, *g, *scal;
  double rtol;
  int *done, *iters;
};

template <int RPT>
__global__ void __launch_bounds__(MGS_THREADS, 1) mgs_coop_kernel(MgsArgs a) {
  cg::grid_group grid = cg::this_grid();
  if (*a.done) return;  // read by every CTA before any barrier: uniform
  __shared__ double red[MGS_THREADS / 32];
  __shared__ double hsh;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G = gridDim.x;
  // warp-contiguous rows: the warp's segment of 32 RPT rows, lane + 32 k
  // (coalesced, and the offsets of the k loop are constants)
  const int64_t base = ((int64_t)blockIdx.x * (MGS_THREADS / 32) + warp) * (32 * RPT) + lane;
  const int64_t lim = a.n - base;  // row k exists iff 32 k < lim
  double x[RPT];
  {
    const double* wp = a.w + base;
#pragma unroll
    for (int k = 0; k < RPT; ++k) x[k] = 32 * k < lim ? wp[32 * k] : 0.0;
  }
  // grid-wide sum of one value per thread (deterministic), into hsh
  auto grid_sum = [&](double v, int buf) -> double {
    v = wsum(v);
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int q = 0; q < MGS_THREADS / 32; ++q) t += red[q];
      a.part[(int64_t)buf * G + blockIdx.x] = t;
    }
    grid.sync();
    if (warp == 0) {
      double t = 0.0;
      for (int b = lane; b < G; b += 32) t += __ldcg(a.part + (int64_t)buf * G + b);
      t = wsum(t);
      if (lane == 0) hsh = t;
    }
    __syncthreads();
    const double out = hsh;
    __syncthreads();
    return out;
  };
  for (int i = 0; i <= a.j; ++i) {
    const double* vp = a.V + (int64_t)i * a.n + base;
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
      if (32 * k < lim) acc = fma(vp[32 * k], x[k], acc);
    const double h = grid_sum(acc, i & 1);
    if (blockIdx.x == 0 && threadIdx.x == 0) a.hcol[i] = h;
#pragma unroll
    for (int k = 0; k < RPT; ++k)
      if (32 * k < lim) x[k] = fma(-h, vp[32 * k], x[k]);
  }
  double nacc = 0.0;
#pragma unroll
  for (int k = 0; k < RPT; ++k) nacc = fma(x[k], x[k], nacc);
  const double wn2 = grid_sum(nacc, (a.j + 1) & 1);
  if (blockIdx.x == 0 && threadIdx.x == 0)
    givens_update(a.j, a.m, a.H, a.cs, a.sn, a.g, a.hcol, nullptr, wn2, a.scal, a.rtol, a.done, a.iters);
  const double hn = sqrt(fmax(wn2, 0.0));
  const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
  double* op = a.vnext + base;
#pragma unroll
  for (int k = 0; k < RPT; ++k)
    if (32 * k < lim) op[32 * k] = x[k] * inv;
}

__global__ void scale_kernel(const double* __restrict__ w, double* __restrict__ v, int64_t n,
                             const double* __restrict__ scal, int idx, const int* __restrict__ done) {
  if (done && *done) return;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) v[i] = w[i] * scal[idx];
}

// y = R^-1 g (upper triangular, k columns), one CTA: column-oriented back
// substitution, y_i = s_i / R_ii and then s_r -= R_ri y_i for all r < i in
// parallel (one barrier per column)
__global__ void __launch_bounds__(256)
backsolve_kernel(const double* __restrict__ H, int m, const int* __restrict__ kp,
                 const double* __restrict__ g, double* __restrict__ y) {
  __shared__ double sv[MAXR];
  __shared__ double yi;
  const int k = *kp;
  for (int i = threadIdx.x; i < k; i += blockDim.x) sv[i] = g[i];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    const double* col = H + (int64_t)i * (m + 1);
    if (threadIdx.x == 0) {
      yi = sv[i] / col[i];
      y[i] = yi;
    }
    __syncthreads();
    const double v = yi;
    for (int r = threadIdx.x; r < i; r += blockDim.x) sv[r] -= col[r] * v;
    __syncthreads();
  }
}

// Second Gram-Schmidt pass needed?  reorth = (||w - V h1||^2 < ||w||^2 / 2)
// with ||w||^2 in h1[nvec]; without it h2 = 0.  count[0] counts the passes.
__global__ void dgks_kernel(const double* __restrict__ h1, int nvec, const double* __restrict__ wn2,
                            double* __restrict__ h2, int* __restrict__ reorth, int* __restrict__ count,
                            const int* __restrict__ done) {
  if (*done) return;
  const bool again = !(wn2[0] >= 0.5 * h1[nvec]);
  if (!again)
    for (int i = threadIdx.x; i < nvec; i += blockDim.x) h2[i] = 0.0;
  if (threadIdx.x == 0) {
    *reorth = again ? 1 : 0;
    if (again) *count += 1;
  }
}

// x += Z y  (k = number of columns)
__global__ void combine_kernel(const double* __restrict__ Z, int64_t ldz, const int* __restrict__ kp,
                               const double* __restrict__ y, double* __restrict__ x, int64_t n) {
  __shared__ double ys[MAXR];
  const int k = *kp;
  for (int j = threadIdx.x; j < k; j += blockDim.x) ys[j] = y[j];
  __syncthreads();
  const int64_t row = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (row >= n) return;
  double acc = x[row];
  for (int j = 0; j < k; ++j) acc += Z[(int64_t)j * ldz + row] * ys[j];
  x[row] = acc;
}

__global__ void axpby_kernel(double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                             double* __restrict__ out, int64_t n) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = a * x[i] + b * y[i];
}

// start of a cycle: beta = ||r|| -> g = (beta, 0, ...), scal[1] = 1/beta;
// the first cycle also records ||b||.
__global__ void cycle_start_kernel(const double* __restrict__ rn2, double* __restrict__ g, int m,
                                   double* __restrict__ scal, int first, double rtol,
                                   int* __restrict__ done, int* __restrict__ kcount) {
  const double beta = sqrt(fmax(rn2[0], 0.0));
  if (first) scal[2] = beta;
  for (int i = 0; i <= m; ++i) g[i] = 0.0;
  g[0] = beta;
  scal[1] = beta > 0.0 ? 1.0 / beta : 0.0;
  scal[0] = scal[2] > 0.0 ? beta / scal[2] : 0.0;
  *kcount = 0;
  *done = (beta <= rtol * scal[2]) ? 1 : 0;
}

}  // namespace

void Gmres::ensure_small(int64_t n_) {
  if (partial.p && nchunks == (int)cdiv(n_, DOT_THREADS)) return;
  nchunks = (int)cdiv(n_, DOT_THREADS);   // CTAs at one row per thread (the most)
  pstride = MAXV;
  partial.alloc((size_t)nchunks * pstride);
  ticket.alloc(1);
  CB_CUDA(cudaMemset(ticket.p, 0, sizeof(unsigned)));
  hstride = MAXV;
  h.alloc(3 * hstride);
  scal.alloc(8);
  flags.alloc(4);
  CB_CUDA(cudaMemset(flags.p, 0, 4 * sizeof(int)));
  if (!host_scal) CB_CUDA(cudaMallocHost(&host_scal, 64));
  if (!host_flags) CB_CUDA(cudaMallocHost(&host_flags, 16));
}

void Gmres::ensure(int64_t n_, int m_) {
  ensure_small(n_);
  if (n == n_ && m == m_) return;
  // cooperative orthogonalisation: at most two CTAs per SM, about four row
  // tiles per CTA; 0 when the device cannot launch cooperatively
  {
    int dev = 0, coop = 0, sms = 0, per_sm = 0;
    CB_CUDA(cudaGetDevice(&dev));
    CB_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    CB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cgs2_coop_kernel, DOT_THREADS, 0));
    const int64_t tiles = cdiv(n_, DOT_THREADS);
    // a few row tiles per CTA, so that the cross-CTA sums stay short; long
    // vectors (n > 1M, bandwidth-bound) keep the multi-launch path with its
    // larger row tiles
    coop_grid = (coop && n_ <= kCoopMaxN) ? (int)std::min<int64_t>(std::min(per_sm, 2) * (int64_t)sms,
                                                                   std::max<int64_t>(1, tiles / 4))
                                          : 0;
    if (coop_grid > 0) cpart.alloc((size_t)3 * coop_grid * MAXV);
    // MGS cooperative launch: one CTA of MGS_THREADS per SM, rows per
    // thread rounded up to 8, 16, 24 or 32 (n up to 3.1M on 152 SMs; 0:
    // the multi-launch path)
    mgs_grid = 0;
    mgs_rpt = 0;
    if (coop) {
      const int64_t T = (int64_t)sms * MGS_THREADS;
      const int64_t need = (n_ + T - 1) / T;
      const int rpt = need <= 8 ? 8 : need <= 16 ? 16 : need <= 24 ? 24 : need <= 32 ? 32 : 0;
      int per = 0;
      if (rpt == 8) CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_coop_kernel<8>, MGS_THREADS, 0));
      if (rpt == 16) CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_coop_kernel<16>, MGS_THREADS, 0));
      if (rpt == 24) CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_coop_kernel<24>, MGS_THREADS, 0));
      if (rpt == 32) CB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_coop_kernel<32>, MGS_THREADS, 0));
      if (rpt > 0 && per >= 1) {
        mgs_grid = sms;
        mgs_rpt = rpt;
        mpart.alloc((size_t)2 * sms);
      }
    }
  }
  CB_CHECK(m_ >= 1 && m_ < MAXR, CBDDC_EINVAL, "restart must be in [1, 1023]");
  n = n_;
  m = m_;
  // partial sums and Hessenberg columns for up to m + 1 Krylov vectors
  if (m + 1 > pstride) {
    pstride = (int)round_up(m + 1, 32);
    partial.alloc((size_t)nchunks * pstride);
  }
  if (m + 1 > hstride) {
    hstride = (int)round_up(m + 1, 32);
    h.alloc(3 * (size_t)hstride);
  }
  V.alloc((size_t)(m + 1) * n);
  Zb.alloc((size_t)m * n);
  w.alloc(n);
  r.alloc(n);
  H.alloc((size_t)(m + 1) * m);
  cs.alloc(m);
  sn.alloc(m);
  g.alloc(m + 1);
  y.alloc(m);
}

Gmres::~Gmres() {
  if (host_scal) cudaFreeHost(host_scal);
  if (host_flags) cudaFreeHost(host_flags);
}

// out = V^T w over nvec columns (stride ldv), optionally after w -= V hin,
// or out[0] = ||w||^2 with self_norm; one launch with a last-block reduction.
static void fused_dots(Gmres& G, const double* V, int64_t ldv, int nvec, double* w, int64_t n,
                       const double* hin, int self_norm, double* out, const int* done, cudaStream_t s,
                       const int* gate = nullptr, int also_norm = 0) {
  DotArgs a{V, ldv, nvec, w, n, hin, self_norm, G.partial.p, G.pstride, G.ticket.p, out, done, gate, also_norm};
  // rows per thread: the largest of 16, 8, 4, 2, 1 that still gives two
  // CTAs per SM (fewer CTAs also shorten the last CTA's reduction)
  const int64_t sms2 = 2 * 152;
  if (n >= 16 * DOT_THREADS * sms2) {
    fused_dots_kernel<16><<<(unsigned)cdiv(n, 16 * DOT_THREADS), DOT_THREADS, 0, s>>>(a);
  } else if (n >= 8 * DOT_THREADS * sms2) {
    fused_dots_kernel<8><<<(unsigned)cdiv(n, 8 * DOT_THREADS), DOT_THREADS, 0, s>>>(a);
  } else if (n >= 4 * DOT_THREADS * sms2) {
    fused_dots_kernel<4><<<(unsigned)cdiv(n, 4 * DOT_THREADS), DOT_THREADS, 0, s>>>(a);
  } else if (n >= 2 * DOT_THREADS * sms2) {
    fused_dots_kernel<2><<<(unsigned)cdiv(n, 2 * DOT_THREADS), DOT_THREADS, 0, s>>>(a);
  } else {
    fused_dots_kernel<1><<<(unsigned)cdiv(n, DOT_THREADS), DOT_THREADS, 0, s>>>(a);
  }
  CB_LAUNCH();
}

int gmres_run(fem_problem* P, bddc_ctx* C, Gmres& G, const double* b, double* x, int restart,
              int max_iters, double rtol, int* iters_out, double* relres_out, cudaStream_t s) {
  const int64_t n = P->n_free;
  G.ensure(n, restart);
  const int m = restart;
  const unsigned nb = cdiv(n, 256);
  int* done = G.flags.p;
  int* kcount = G.flags.p + 1;
  CB_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double), s));
  int total = 0;
  bool first = true;
  int* hflags = G.host_flags;
  CB_CUDA(cudaMemsetAsync(G.flags.p + 3, 0, sizeof(int), s));  // second Gram-Schmidt passes
  bool converged = false;
  while (true) {
    // r = b - K x
    if (first) {
      CB_CUDA(cudaMemcpyAsync(G.r.p, b, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
    } else {
      bsr_spmv(P, x, G.w.p, s);
      axpby_kernel<<<nb, 256, 0, s>>>(1.0, b, -1.0, G.w.p, G.r.p, n);
      CB_LAUNCH();
    }
    fused_dots(G, G.r.p, n, 1, G.r.p, n, nullptr, 1, G.h.p, nullptr, s);
    cycle_start_kernel<<<1, 1, 0, s>>>(G.h.p, G.g.p, m, G.scal.p, first ? 1 : 0, rtol, done, kcount);
    CB_LAUNCH();
    scale_kernel<<<nb, 256, 0, s>>>(G.r.p, G.V.p, n, G.scal.p, 1, nullptr);
    CB_LAUNCH();
    CB_CUDA(cudaMemcpyAsync(G.host_scal, G.scal.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaMemcpyAsync(hflags, done, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
    CB_CUDA(cudaStreamSynchronize(s));
    first = false;
    *relres_out = G.host_scal[0];
    if (hflags[0]) { converged = true; break; }
    if (total >= max_iters) break;
    int j = 0;
    for (; j < m && total < max_iters; ++j) {
      double* vj = G.V.p + (int64_t)j * n;
      double* zj = G.Zb.p + (int64_t)j * n;
      bddc_run_apply(C, vj, zj, s);
      bsr_spmv(P, zj, G.w.p, s);
      // classical Gram-Schmidt, twice: h1 = V^T w; w -= V h1 and h2 = V^T w;
      // w -= V h2 and ||w||^2 (three launches)
      double* h1 = G.h.p;
      double* h2 = G.h.p + G.hstride;
      double* wn2 = G.h.p + 2 * G.hstride;
      timer_begin(CBDDC_TIMER_ORTH, s);
      if (G.coop_grid > 0 && j + 1 <= MAXV) {
        // short vectors and bases: CGS2 in one cooperative launch
        CgsArgs ca{G.V.p, n, j + 1, G.w.p, G.V.p + (int64_t)(j + 1) * n, G.cpart.p, j, m,
                   G.H.p, G.cs.p, G.sn.p, G.g.p, G.scal.p, rtol, done, kcount};
        void* args[] = {&ca};
        CB_CUDA(cudaLaunchCooperativeKernel((const void*)cgs2_coop_kernel, dim3(G.coop_grid),
                                            dim3(DOT_THREADS), args, 0, s));
        CB_LAUNCH();
      } else if (G.mgs_grid > 0) {
        MgsArgs ma{G.V.p, n, G.w.p, G.V.p + (int64_t)(j + 1) * n, G.mpart.p, G.h.p, j, m,
                   G.H.p, G.cs.p, G.sn.p, G.g.p, G.scal.p, rtol, done, kcount};
        void* args[] = {&ma};
        const void* fn = G.mgs_rpt == 8    ? (const void*)mgs_coop_kernel<8>
                         : G.mgs_rpt == 16 ? (const void*)mgs_coop_kernel<16>
                         : G.mgs_rpt == 24 ? (const void*)mgs_coop_kernel<24>
                                           : (const void*)mgs_coop_kernel<32>;
        CB_CUDA(cudaLaunchCooperativeKernel(fn, dim3(G.mgs_grid), dim3(MGS_THREADS), args, 0, s));
        CB_LAUNCH();
      } else {
        // classical Gram-Schmidt with a second pass only where the first
        // one lost more than half of ||w||^2 (Daniel-Gragg-Kaufman-Stewart
        // criterion, eta = 1/sqrt(2)): h1 = V^T w with ||w||^2; w -= V h1
        // with the new ||w||^2; then, gated on the device, h2 = V^T w and
        // w -= V h2 with its norm
        int* reorth = G.flags.p + 2;
        fused_dots(G, G.V.p, n, j + 1, G.w.p, n, nullptr, 0, h1, done, s, nullptr, 1);
        fused_dots(G, G.V.p, n, j + 1, G.w.p, n, h1, 1, wn2, done, s);
        dgks_kernel<<<1, 256, 0, s>>>(h1, j + 1, wn2, h2, reorth, G.flags.p + 3, done);
        CB_LAUNCH();
        fused_dots(G, G.V.p, n, j + 1, G.w.p, n, nullptr, 0, h2, done, s, reorth);
        fused_dots(G, G.V.p, n, j + 1, G.w.p, n, h2, 1, wn2, done, s, reorth);
        givens_kernel<<<1, 1, 0, s>>>(j, m, G.H.p, G.cs.p, G.sn.p, G.g.p, h1, h2, wn2, G.scal.p, rtol,
                                      done, kcount);
        CB_LAUNCH();
        scale_kernel<<<nb, 256, 0, s>>>(G.w.p, G.V.p + (int64_t)(j + 1) * n, n, G.scal.p, 1, done);
        CB_LAUNCH();
      }
      // algorithmic traffic of one Gram-Schmidt pass (the second pass, when
      // taken, is not counted): V read twice (dots, update), w read twice
      // and written once, v_{j+1} written
      timer_end(CBDDC_TIMER_ORTH, s, 4.0 * (j + 1) * (double)n, 8.0 * (double)n * (2.0 * (j + 1) + 4.0));
      CB_CUDA(cudaMemcpyAsync(hflags, done, 4 * sizeof(int), cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      ++total;
      if (hflags[0]) { ++j; break; }
    }
    // x += Z y over the columns built in this cycle
    backsolve_kernel<<<1, 256, 0, s>>>(G.H.p, m, kcount, G.g.p, G.y.p);
    CB_LAUNCH();
    combine_kernel<<<nb, 256, 0, s>>>(G.Zb.p, n, kcount, G.y.p, x, n);
    CB_LAUNCH();
    if (total >= max_iters && !hflags[0]) {
      // final true residual
      bsr_spmv(P, x, G.w.p, s);
      axpby_kernel<<<nb, 256, 0, s>>>(1.0, b, -1.0, G.w.p, G.r.p, n);
      CB_LAUNCH();
      fused_dots(G, G.r.p, n, 1, G.r.p, n, nullptr, 1, G.h.p, nullptr, s);
      CB_CUDA(cudaMemcpyAsync(G.host_scal + 4, G.h.p, sizeof(double), cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaMemcpyAsync(G.host_scal, G.scal.p, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
      CB_CUDA(cudaStreamSynchronize(s));
      *relres_out = G.host_scal[2] > 0 ? std::sqrt(G.host_scal[4]) / G.host_scal[2] : 0.0;
      break;
    }
    // next cycle (or final check) recomputes the true residual
  }
  *iters_out = total;
  G.reorth = hflags[3];
  return converged ? CBDDC_OK : CBDDC_ENOCONV;
}

double device_norm(fem_problem* P, Gmres& G, const double* v, cudaStream_t s) {
  G.ensure_small(P->n_free);
  fused_dots(G, v, P->n_free, 1, const_cast<double*>(v), P->n_free, nullptr, 1, G.h.p, nullptr, s);
  CB_CUDA(cudaMemcpyAsync(G.host_scal + 4, G.h.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  CB_CUDA(cudaStreamSynchronize(s));
  return std::sqrt(G.host_scal[4]);
}

void axpby(double a, const double* x, double b, const double* y, double* out, int64_t n, cudaStream_t s) {
  axpby_kernel<<<cdiv(n, 256), 256, 0, s>>>(a, x, b, y, out, n);
  CB_LAUNCH();
}

}  // namespace cbddc
