// Two-level BDDC (Section 3.2 of the paper) on dense per-subdomain
// operators, for the whole tangent system through the exact interior /
// interface block factorisation.
//
// Setup (per subdomain i, all subdomains batched in each launch):
//   A^(i) (ordered [I | Gamma_r | Gamma_v]) from the element matrices;
//   sweep over I  -> [[A_II^-1, A_II^-1 A_IG], [-A_GI A_II^-1, S_i]];
//   sweep of a copy of S_i over Gamma_r
//                 -> [[S_rr^-1, S_rr^-1 S_rv], [., S_vv - S_vr S_rr^-1 S_rv]];
//   averages C (edge/face means per component) on Gamma_r:
//     Y = S_rr^-1 C^T, Z = C [S_rr^-1 | S_rr^-1 S_rv], G = C Y, W = G^-1 Z,
//     T_rr = S_rr^-1 - Y W_r        (constrained Neumann solve, zero primal
//                                    values: the local problem of Sec. 3.2),
//     Phi_r = [-(S_rr^-1 S_rv - Y W_v) | Y G^-1],  Phi_v = [I | 0]
//                                   (minimum-energy coarse basis);
//   S_PiPi = sum_i R_Pi^T Phi_i^T S_i Phi_i R_Pi, inverted in FP64.
// Apply z = M^-1 r (10 launches, all batched):
//   u0 = A_II^-1 r_I and h = A_GI A_II^-1 r_I       (one GEMV on [A_II^-1; -H])
//   g = r_G - sum_i R_i^T h_i ;  g_i = D_i R_i g
//   w_i = T_i g_i ;  c = sum_i R_Pi^T Phi_i^T g_i ;  u_c = S_PiPi^-1 c
//   z_G = sum_i R_i^T D_i (w_i + Phi_i R_Pi u_c)
//   z_I = u0 - A_II^-1 A_IG z_G
// The local operators are FP64 or FP32 (FP32 accumulation); vectors, the
// coarse restriction/prolongation sums and the coarse solve are FP64.
#include <algorithm>
#include <map>
#include <mutex>
#include <string>

#include "bddc.h"
#include "fem.h"
#include "rigid.h"
#include "sell.h"

namespace cbddc {

namespace {

__host__ __device__ inline int64_t round_up_dev(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

constexpr int64_t kAlign = 64;  // element alignment of every packed block

template <typename T> struct Vec2;
template <> struct Vec2<float> { using type = float4; static constexpr int W = 4; };
template <> struct Vec2<double> { using type = double2; static constexpr int W = 2; };

template <typename T>
__device__ inline T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ inline float vdot2(float4 a, float4 b) { return a.x * b.x + a.y * b.y + a.z * b.z + a.w * b.w; }
__device__ inline double vdot2(double2 a, double2 b) { return a.x * b.x + a.y * b.y; }

// Dot products of two rows (16-byte aligned) with a shared-memory vector,
// one warp: the rows go in chunks of 32 x U 16-byte vectors, and every lane
// issues all its loads of a chunk (2 x U, predicated at the row's end)
// before using them, so short rows (a few hundred entries) are one round of
// loads; no barriers.
template <typename T>
__device__ __forceinline__ void warp_dot2(const T* __restrict__ ra, const T* __restrict__ rb, bool has_b,
                                          const T* __restrict__ xs, int n, int lane, T& oa, T& ob) {
  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::W;
  constexpr int U = 4;
  const int nv = n / W;
  const V* va = reinterpret_cast<const V*>(ra);
  const V* vb = reinterpret_cast<const V*>(rb);
  const V* xv = reinterpret_cast<const V*>(xs);
  T acc_a = T(0), acc_b = T(0);
  for (int i0 = lane; i0 < nv; i0 += 32 * U) {
    V la[U], lb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + 32 * u;
      la[u] = i < nv ? __ldcs(va + i) : V{};
      lb[u] = (has_b && i < nv) ? __ldcs(vb + i) : V{};
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = i0 + 32 * u;
      if (i < nv) {
        const V x = xv[i];
        acc_a += vdot2(la[u], x);
        if (has_b) acc_b += vdot2(lb[u], x);
      }
    }
  }
  for (int c = nv * W + lane; c < n; c += 32) {
    acc_a += ra[c] * xs[c];
    if (has_b) acc_b += rb[c] * xs[c];
  }
  oa = warp_sum(acc_a);
  ob = has_b ? warp_sum(acc_b) : T(0);
}

// Row-block GEMV driver: rows [rb, re) of a matrix with leading dimension
// ld, 8 warps x two rows at a time; f(row, value) stores each result.
template <typename T, typename F>
__device__ __forceinline__ void gemv_rows(const T* __restrict__ A, int64_t ld, int rb, int re,
                                          const T* __restrict__ xs, int n, F f) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int r = rb + 2 * warp; r < re; r += 16) {
    const bool hb = (r + 1) < re;
    T va, vb;
    warp_dot2<T>(A + (int64_t)r * ld, A + (int64_t)(hb ? r + 1 : r) * ld, hb, xs, n, lane, va, vb);
    if (lane == 0) {
      f(r, va);
      if (hb) f(r + 1, vb);
    }
  }
}

constexpr int GROWS = 16;   // rows per group of the row-block GEMVs
constexpr int GGROUPS = 4;  // groups per CTA (64 rows share one x load)

// xs[0:n] = (T) x[0:n] from a packed FP64 vector (coalesced).
template <typename T>
__device__ __forceinline__ void load_x(T* __restrict__ xs, const double* __restrict__ x, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) xs[j] = (T)x[j];
  __syncthreads();
}

// ------------------------------------------------------------ setup kernels

template <typename T>
__global__ void densify_kernel(const int* __restrict__ lsub, const int* __restrict__ lrow,
                               const int* __restrict__ lcol, const int* __restrict__ lptr,
                               const int* __restrict__ lsrc, const double* __restrict__ contrib,
                               int64_t nslots, const int* __restrict__ perm,
                               const int64_t* __restrict__ offN, const int64_t* __restrict__ offA,
                               const int* __restrict__ ldA, const int* __restrict__ nI,
                               T* __restrict__ Aloc) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslots * 9) return;
  const int64_t sl = t / 9;
  const int e = (int)(t % 9), i = e / 3, k = e % 3;
  const int s = lsub[sl];
  const int pr = perm[offN[s] + lrow[sl]], pc = perm[offN[s] + lcol[sl]];
  double v = 0.0;
  for (int j = lptr[sl]; j < lptr[sl + 1]; ++j) v += contrib[(int64_t)lsrc[j] * 9 + e];
  const int row = 3 * pr + i;
  int col = 3 * pc + k;
  const int ni = nI[s];
  if (col >= ni) col += (int)(round_up_dev(ni, 4) - ni);
  Aloc[offA[s] + (int64_t)row * ldA[s] + col] = (T)v;
}

// Row copies between packed per-subdomain blocks: row i (< rows) of
// dst (ld_dst) <- row i of src (ld_src), n entries per row.  One warp per
// row, 8 rows per CTA, grid (row blocks, subdomains); 64-bit index
// arithmetic only per row.
template <typename T>
__device__ __forceinline__ void copy_rows(T* __restrict__ dst, int64_t ldd, const T* __restrict__ src, int64_t lds,
                                          int rows, int n) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= rows) return;
  const T* sr = src + (int64_t)i * lds;
  T* dr = dst + (int64_t)i * ldd;
  for (int j = lane; j < n; j += 32) dr[j] = sr[j];
}

// Sw <- S (the GG block of Aloc after the interior sweep), n_G x n_G.
template <typename T>
__global__ void __launch_bounds__(256)
copy_schur_kernel(const int* __restrict__ nI, const int* __restrict__ nG, const int64_t* __restrict__ offA,
                  const int* __restrict__ ldA, const int64_t* __restrict__ offS, const int* __restrict__ ldS,
                  const T* __restrict__ Aloc, T* __restrict__ Sw) {
  const int s = blockIdx.y;
  const int ng = nG[s], ni = nI[s];
  const int cI = (int)round_up_dev(ni, 4);
  copy_rows(Sw + offS[s], ldS[s], Aloc + offA[s] + (int64_t)ni * ldA[s] + cI, ldA[s], ng, ng);
}

// A_IG block <- E (the harmonic-extension operator A_II^-1 A_IG), n_I x n_G.
template <typename T>
__global__ void __launch_bounds__(256)
copy_e_kernel(const int* __restrict__ nI, const int* __restrict__ nG, const int64_t* __restrict__ offA,
              const int* __restrict__ ldA, const int64_t* __restrict__ offE, const int* __restrict__ ldE,
              const T* __restrict__ Et, T* __restrict__ Aloc) {
  const int s = blockIdx.y;
  const int ng = nG[s], ni = nI[s];
  const int cI = (int)round_up_dev(ni, 4);
  copy_rows(Aloc + offA[s] + cI, ldA[s], Et + offE[s], ldE[s], ni, ng);
}

// S_rr += alpha sum_q c_q c_q^T / |c_q|^2 over the constraint rows c_q
// (alpha = largest |S_ii| of the subdomain).  Since C w = 0 for every
// admissible w, the constrained solution operator and the coarse basis are
// unchanged, while S_rr becomes invertible for floating subdomains whose
// primal space has no vertices.  One CTA per subdomain; constraints are
// added one after the other.
template <typename T>
__global__ void __launch_bounds__(256)
augment_kernel(const int* __restrict__ nr, const int* __restrict__ na,
               const int64_t* __restrict__ offCon, const int* __restrict__ cptr,
               const int* __restrict__ cidx, const double* __restrict__ cw,
               const int64_t* __restrict__ offS, const int* __restrict__ ldS, T* __restrict__ Sw) {
  __shared__ double red[256];
  const int s = blockIdx.x;
  const int n = nr[s];
  if (na[s] == 0 || n == 0) return;
  T* S0 = Sw + offS[s];
  const int ld = ldS[s];
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs((double)S0[(int64_t)i * ld + i]));
  red[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + o]);
    __syncthreads();
  }
  const double alpha = red[0];
  for (int q = 0; q < na[s]; ++q) {
    const int64_t gq = offCon[s] + q;
    const int b = cptr[gq], cnt = cptr[gq + 1] - b;
    double nrm2 = 0.0;
    for (int j = 0; j < cnt; ++j) nrm2 += cw[b + j] * cw[b + j];
    const double scale = alpha / nrm2;  // alpha c c^T / |c|^2
    for (int t = threadIdx.x; t < cnt * cnt; t += blockDim.x) {
      const int a = b + t / cnt, e = b + t % cnt;
      S0[(int64_t)cidx[a] * ld + cidx[e]] += (T)(scale * cw[a] * cw[e]);
    }
    __syncthreads();  // the rotations of a class share members with its averages
  }
}

// Y[row][q] = sum_{j in q} w_j Sw[row][j], one warp per row (row < n_r),
// accumulated in the operator precision.
template <typename T>
__global__ void cons_y_kernel(const int* __restrict__ nr, const int* __restrict__ na,
                              const int64_t* __restrict__ offCon, const int* __restrict__ cptr,
                              const int* __restrict__ cidx, const double* __restrict__ cw,
                              const int64_t* __restrict__ offS, const int* __restrict__ ldS,
                              const int64_t* __restrict__ offY, const int* __restrict__ ldY,
                              const T* __restrict__ Sw, T* __restrict__ Y) {
  const int s = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * (blockDim.x >> 5) + warp;
  if (row >= nr[s]) return;
  const T* Srow = Sw + offS[s] + (int64_t)row * ldS[s];
  // one lane per constraint (classes have few members): no reductions,
  // and the row's Y entries are written together
  for (int q = lane; q < na[s]; q += 32) {
    const int64_t gq = offCon[s] + q;
    T acc = T(0);
    for (int j = cptr[gq]; j < cptr[gq + 1]; ++j) acc += Srow[cidx[j]] * (T)cw[j];
    Y[offY[s] + (int64_t)row * ldY[s] + q] = acc;
  }
}

// Zf[q][col] = sum_{j in q} w_j Sw[j][col] for all n_G columns (operator
// precision).
template <typename T>
__global__ void cons_z_kernel(const int* __restrict__ nG, const int* __restrict__ na,
                              const int64_t* __restrict__ offCon, const int* __restrict__ cptr,
                              const int* __restrict__ cidx, const double* __restrict__ cw,
                              const int64_t* __restrict__ offS, const int* __restrict__ ldS,
                              const int64_t* __restrict__ offZ, const T* __restrict__ Sw,
                              T* __restrict__ Zf) {
  const int s = blockIdx.y;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nG[s]) return;
  const T* S0 = Sw + offS[s];
  const int ld = ldS[s];
  for (int q = 0; q < na[s]; ++q) {
    const int64_t gq = offCon[s] + q;
    T acc = T(0);
    for (int j = cptr[gq]; j < cptr[gq + 1]; ++j) acc += S0[(int64_t)cidx[j] * ld + col] * (T)cw[j];
    Zf[offZ[s] + (int64_t)q * ld + col] = acc;
  }
}

// G[q][q2] = sum_{j in q} w_j Y[j][q2]
template <typename T>
__global__ void cons_g_kernel(const int* __restrict__ na, const int64_t* __restrict__ offCon,
                              const int* __restrict__ cptr, const int* __restrict__ cidx,
                              const double* __restrict__ cw, const int64_t* __restrict__ offY,
                              const int* __restrict__ ldY, const int64_t* __restrict__ offG,
                              const int* __restrict__ ldG, const T* __restrict__ Y, T* __restrict__ G) {
  const int s = blockIdx.y;
  const int n = na[s];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * n) return;
  const int q = t / n, q2 = t % n;
  const int64_t gq = offCon[s] + q;
  double acc = 0.0;
  for (int j = cptr[gq]; j < cptr[gq + 1]; ++j)
    acc += (double)Y[offY[s] + (int64_t)cidx[j] * ldY[s] + q2] * cw[j];
  G[offG[s] + (int64_t)q * ldG[s] + q2] = (T)acc;
}

// ------------------------------------------------- deluxe scaling (setup)
// S_b = the class block of block b's subdomain Schur complement S = A_GG -
// A_GI A_II^-1 A_IG (the GG block of Aloc), rows and columns at the class
// DoFs' interface positions.  Block b = blockIdx.x; its n^2 entries are
// spread over the gridDim.y CTAs of the block.
template <typename T>
__global__ void __launch_bounds__(256)
deluxe_gather_kernel(const int* __restrict__ bn, const int* __restrict__ bsub, const int* __restrict__ bld,
                     const int64_t* __restrict__ poff, const int* __restrict__ pos,
                     const int64_t* __restrict__ boff, const int* __restrict__ nI,
                     const int64_t* __restrict__ offA, const int* __restrict__ ldA,
                     const T* __restrict__ Aloc, T* __restrict__ Sb) {
  const int b = blockIdx.x;
  const int n = bn[b], s = bsub[b], ld = bld[b];
  const int ni = nI[s], lda = ldA[s];
  const T* S = Aloc + offA[s] + (int64_t)ni * lda + round_up_dev(ni, 4);
  const int* p = pos + poff[b];
  T* out = Sb + boff[b];
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < n * n; t += gridDim.y * blockDim.x) {
    const int i = t / n, j = t % n;
    out[(int64_t)i * ld + j] = S[(int64_t)p[i] * lda + p[j]];
  }
}

// Shat_K = sum of the class's blocks S_b, in block order.  Class k =
// blockIdx.x, its entries spread over gridDim.y CTAs.
template <typename T>
__global__ void __launch_bounds__(256)
deluxe_sum_kernel(const int* __restrict__ cptr, const int* __restrict__ cblk, const int* __restrict__ bn,
                  const int* __restrict__ bld, const int64_t* __restrict__ boff,
                  const int64_t* __restrict__ coff, const T* __restrict__ Sb, T* __restrict__ Sh) {
  const int k = blockIdx.x;
  const int b0 = cptr[k], b1 = cptr[k + 1];
  const int n = bn[cblk[b0]], ld = bld[cblk[b0]];
  T* out = Sh + coff[k];
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < n * n; t += gridDim.y * blockDim.x) {
    const int i = t / n, j = t % n;
    T v = T(0);
    for (int q = b0; q < b1; ++q) v += Sb[boff[cblk[q]] + (int64_t)i * ld + j];
    out[(int64_t)i * ld + j] = v;
  }
}

// E_b = D_b^T.  Block b = blockIdx.x, its entries spread over gridDim.y CTAs.
template <typename T>
__global__ void __launch_bounds__(256)
deluxe_transpose_kernel(const int* __restrict__ bn, const int* __restrict__ bld,
                        const int64_t* __restrict__ boff, const T* __restrict__ D, T* __restrict__ E) {
  const int b = blockIdx.x;
  const int n = bn[b], ld = bld[b];
  const T* d = D + boff[b];
  T* e = E + boff[b];
  for (int t = blockIdx.y * blockDim.x + threadIdx.x; t < n * n; t += gridDim.y * blockDim.x) {
    const int i = t / n, j = t % n;
    e[(int64_t)j * ld + i] = d[(int64_t)i * ld + j];
  }
}

// Phi[0:nr, 0:nv] = -Sw[0:nr, nr:nG] ; Phi[nr:nG, :] = [I 0]
template <typename T>
__global__ void phi_vertex_kernel(const int* __restrict__ nG, const int* __restrict__ nr,
                                  const int* __restrict__ nv, const int* __restrict__ nc,
                                  const int64_t* __restrict__ offS, const int* __restrict__ ldS,
                                  const int64_t* __restrict__ offPhi, const int* __restrict__ ldPhi,
                                  const T* __restrict__ Sw, T* __restrict__ Phi) {
  const int s = blockIdx.y;
  const int ncs = nc[s], ng = nG[s], nrs = nr[s], nvs = nv[s];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ng * ncs) return;
  const int row = (int)(t / ncs), c = (int)(t % ncs);
  T* dst = Phi + offPhi[s] + (int64_t)row * ldPhi[s] + c;
  if (row < nrs) {
    if (c < nvs) *dst = -Sw[offS[s] + (int64_t)row * ldS[s] + nrs + c];
  } else {
    *dst = (c == row - nrs) ? T(1) : T(0);
  }
}

// Left coarse basis of the Petrov coarse space, apart from the vertex
// columns of the r rows (a GEMM writes -(S_vr T)^T there):
// Psi[0:nr, nv:nc] = Wf[:, 0:nr]^T = (G^-1 C M_rr^-1)^T, the constraint
// columns of the constrained problem for S^T; Psi[nr:nG, :] = [I 0].
template <typename T>
__global__ void psi_fill_kernel(const int* __restrict__ nG, const int* __restrict__ nr,
                                const int* __restrict__ nv, const int* __restrict__ nc,
                                const int64_t* __restrict__ offZ, const int* __restrict__ ldS,
                                const int64_t* __restrict__ offPhi, const int* __restrict__ ldPhi,
                                const T* __restrict__ Wf, T* __restrict__ Psi) {
  const int s = blockIdx.y;
  const int ncs = nc[s], ng = nG[s], nrs = nr[s], nvs = nv[s];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ng * ncs) return;
  const int row = (int)(t / ncs), c = (int)(t % ncs);
  T* dst = Psi + offPhi[s] + (int64_t)row * ldPhi[s] + c;
  if (row < nrs) {
    if (c >= nvs) *dst = Wf[offZ[s] + (int64_t)(c - nvs) * ldS[s] + row];
  } else {
    *dst = (c == row - nrs) ? T(1) : T(0);
  }
}

__global__ void coarse_assemble_kernel_f(const int* __restrict__ key, const int* __restrict__ ptr,
                                         const int* __restrict__ src, int64_t n,
                                         const float* __restrict__ Kc, double* __restrict__ S) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v = 0.0;
  for (int j = ptr[t]; j < ptr[t + 1]; ++j) v += (double)Kc[src[j]];
  S[key[t]] = v;
}
__global__ void coarse_assemble_kernel_d(const int* __restrict__ key, const int* __restrict__ ptr,
                                         const int* __restrict__ src, int64_t n,
                                         const double* __restrict__ Kc, double* __restrict__ S) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  double v = 0.0;
  for (int j = ptr[t]; j < ptr[t + 1]; ++j) v += Kc[src[j]];
  S[key[t]] = v;
}

// ------------------------------------------------------------ apply kernels
constexpr int AROWS = 128;  // rows per CTA of the prolongation (8 warps x 4 rows, 4 passes)
constexpr int PHIT_ROWS = 128;  // interface rows per CTA of the coarse restriction
constexpr int NC_MAX = 512;  // primal constraints per subdomain

// xI = r[gdof of the interior DoFs], packed per subdomain.
__global__ void gather_kernel(const int* __restrict__ idx, int64_t n, const double* __restrict__ x,
                              double* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) out[i] = x[idx[i]];
}

// A_II^-1 x_I (rows of the A_II^-1 block), 64 rows per CTA: into the packed
// interior vector u0, or (SCATTER) into the interior entries of the global
// vector z.
template <typename T, bool SCATTER>
__global__ void __launch_bounds__(256)
apply_interior_kernel(const int2* __restrict__ items, const int* __restrict__ nI,
                      const int64_t* __restrict__ offA, const int* __restrict__ ldA,
                      const int64_t* __restrict__ offI, const int* __restrict__ gdofI,
                      const T* __restrict__ Aloc, const double* __restrict__ xI, double* __restrict__ u0,
                      T* __restrict__ uq) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const int ni = nI[s];
  const int rb = it.y * GROWS * GGROUPS;
  if (rb >= ni) return;
  const int64_t oi = offI[s];
  load_x<T>(xs, xI + oi, ni);
  gemv_rows<T>(Aloc + offA[s], ldA[s], rb, min(ni, rb + GROWS * GGROUPS), xs, ni, [&](int row, T v) {
    if (SCATTER) {
      u0[gdofI[oi + row]] = (double)v;
    } else {
      u0[oi + row] = (double)v;
      // node-packed copy for the coupling product (packed interior DoFs
      // are node-major, 3 per node)
      if (uq) uq[(oi + row) / 3 * 4 + (oi + row) % 3] = v;
    }
  });
}

// Sparse interior-interface coupling of the assembled matrix, in sliced
// ELL form: slice q holds 32 block rows (node rows, sorted by length inside
// windows of 8 slices), step k of lane l is block k of row rowmap[32 q + l]
// (column 0 and zero values past the row's end).  Values are stored
// [step][entry][lane] and column indices [step][lane], so each load of a
// warp reads 128 consecutive bytes; x comes node-packed as (x, y, z, pad).
// out[3 i + r] = r_in[rdof[3 i + r]] - (row r of block row i) x.  Used
// twice per apply: g_Gamma = r_Gamma - K_Gamma,I u0 (rows: assembled
// interface nodes, x: the packed interior solution) and t_I = r_I -
// K_I,Gamma z (rows: packed interior nodes, x: z on the interface nodes).
// One lane per block row, all nine products in the operator precision.
template <typename T> struct Q4;
template <> struct Q4<float> { using type = float4; };
template <> struct Q4<double> { using type = double4_32a; };

template <typename T>
__global__ void __launch_bounds__(256)
coupling_kernel(const int* __restrict__ off, const int* __restrict__ len, const int* __restrict__ rowmap,
                const int* __restrict__ col, const T* __restrict__ val,
                const typename Q4<T>::type* __restrict__ xq, const int* __restrict__ rdof,
                const double* __restrict__ r, double* __restrict__ out, int nslices) {
  const int q = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= nslices) return;
  const int row = rowmap[32 * q + lane];
  const int L = len[q];
  const int64_t base = off[q];
  T a0 = T(0), a1 = T(0), a2 = T(0);
#pragma unroll 2
  for (int k = 0; k < L; ++k) {
    const typename Q4<T>::type x = xq[__ldg(col + (base + k) * 32 + lane)];
    const T* v = val + (base + k) * 288 + lane;
    a0 = fma(__ldcs(v + 0), x.x, fma(__ldcs(v + 32), x.y, fma(__ldcs(v + 64), x.z, a0)));
    a1 = fma(__ldcs(v + 96), x.x, fma(__ldcs(v + 128), x.y, fma(__ldcs(v + 160), x.z, a1)));
    a2 = fma(__ldcs(v + 192), x.x, fma(__ldcs(v + 224), x.y, fma(__ldcs(v + 256), x.z, a2)));
  }
  if (row >= 0) {
    out[3 * (int64_t)row + 0] = r[rdof[3 * row + 0]] - (double)a0;
    out[3 * (int64_t)row + 1] = r[rdof[3 * row + 1]] - (double)a1;
    out[3 * (int64_t)row + 2] = r[rdof[3 * row + 2]] - (double)a2;
  }
}

// Values of the sliced coupling blocks from the assembled tangent, in the
// operator precision (once per setup): val[(step 9 + e) 32 + lane] = entry
// e of BSR block src[step 32 + lane] (zero where src < 0).
template <typename T>
__global__ void coupling_values_kernel(const int* __restrict__ src, int64_t steps,
                                       const double* __restrict__ bsr_vals, T* __restrict__ val) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= steps * 288) return;
  const int64_t step = t / 288;
  const int rem = (int)(t - step * 288), e = rem >> 5, lane = rem & 31;
  const int b = src[step * 32 + lane];
  val[t] = b >= 0 ? (T)bsr_vals[(int64_t)b * 9 + e] : T(0);
}

// hG = -A_GI u0 (the interface part of the interior correction).
template <typename T>
__global__ void __launch_bounds__(256)
apply_gi_kernel(const int2* __restrict__ items, const int* __restrict__ nI, const int* __restrict__ nG,
                const int64_t* __restrict__ offA, const int* __restrict__ ldA,
                const int64_t* __restrict__ offI, const int64_t* __restrict__ offGam,
                const T* __restrict__ Aloc, const double* __restrict__ u0, double* __restrict__ hG) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const int ni = nI[s], ng = nG[s];
  const int rb = it.y * GROWS * GGROUPS;
  if (rb >= ng) return;
  const int re = min(ng, rb + GROWS * GGROUPS);
  double* out = hG + offGam[s];
  if (ni == 0) {
    for (int row = rb + threadIdx.x; row < re; row += blockDim.x) out[row] = 0.0;
    return;
  }
  load_x<T>(xs, u0 + offI[s], ni);
  const int ld = ldA[s];
  gemv_rows<T>(Aloc + offA[s] + (int64_t)ni * ld, ld, rb, re, xs, ni,
               [&](int row, T v) { out[row] = -(double)v; });
}

__global__ void assemble_g_kernel(const int* __restrict__ if_dof, const int* __restrict__ if_ptr,
                                  const int* __restrict__ if_src, int n_if, const double* __restrict__ r,
                                  const double* __restrict__ hG, double* __restrict__ gI) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_if) return;
  double g = r[if_dof[m]];
  for (int j = if_ptr[m]; j < if_ptr[m + 1]; ++j) g += hG[if_src[j]];
  gI[m] = g;
}

__global__ void restrict_kernel(const int* __restrict__ gam_if, const double* __restrict__ Dg, int64_t n,
                                const double* __restrict__ gI, double* __restrict__ gl) {
  const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= n) return;
  gl[q] = Dg[q] * gI[gam_if[q]];
}

template <typename T>
__global__ void __launch_bounds__(256)
apply_local_kernel(const int2* __restrict__ items, const int* __restrict__ nG, const int* __restrict__ nr,
                   const int64_t* __restrict__ offS, const int* __restrict__ ldS,
                   const int64_t* __restrict__ offGam, const T* __restrict__ Sw,
                   const double* __restrict__ gl, double* __restrict__ wG) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const int ng = nG[s], nrs = nr[s];
  const int rb = it.y * GROWS * GGROUPS;
  if (rb >= ng) return;
  const int64_t og = offGam[s];
  const int re = min(ng, rb + GROWS * GGROUPS);
  double* out = wG + og;
  // vertex rows: the local solution vanishes there
  for (int row = max(rb, nrs) + threadIdx.x; row < re; row += blockDim.x) out[row] = 0.0;
  if (rb >= nrs) return;
  load_x<T>(xs, gl + og, nrs);
  gemv_rows<T>(Sw + offS[s], ldS[s], rb, min(nrs, re), xs, nrs, [&](int row, T v) { out[row] = (double)v; });
}

// Partial coarse restriction Phi^T g_i over one chunk of PHIT_ROWS interface
// rows: clp[(offC[s] + c) * nchunk + chunk] (FP64 accumulation), columns in
// blocks of 128.  Only the subdomain's own chunks exist (work items); the
// coarse gather sums each entry's chunks in order.
template <typename T>
__global__ void __launch_bounds__(256)
apply_phit_kernel(const int2* __restrict__ items, const int* __restrict__ nG, const int* __restrict__ nc,
                  const int64_t* __restrict__ offPhi, const int* __restrict__ ldPhi,
                  const int64_t* __restrict__ offGam, const int64_t* __restrict__ offC,
                  const T* __restrict__ Phi, const double* __restrict__ gl, double* __restrict__ clp,
                  int nchunk) {
  __shared__ double red[8][128];
  const int2 it = items[blockIdx.x];
  const int s = it.x, chunk = it.y;
  const int ng = nG[s], ncs = nc[s];
  if (ncs == 0) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const T* P0 = Phi + offPhi[s];
  const int ld = ldPhi[s];
  const int64_t og = offGam[s];
  const int r0 = chunk * PHIT_ROWS, r1 = min(ng, r0 + PHIT_ROWS);
  for (int cb = 0; cb < ncs; cb += 128) {
    // products and the chunk's partial sums in the operator precision (FP64
    // issue is the scarce resource on this part); chunks are summed in FP64
    T acc[4] = {T(0), T(0), T(0), T(0)};
    if (sizeof(T) == 4) {
      // FP32: lane owns columns 4 lane .. 4 lane + 3 of the block, one
      // 16-byte load per row (rows are 16-byte aligned and ld is a multiple
      // of 4, so the load stays inside the row; columns past nc are padding
      // whose sums are not stored)
      const bool in = cb + 4 * lane < ld;
#pragma unroll 4
      for (int j = r0 + warp; j < r1; j += 8) {
        const T gj = (T)gl[og + j];
        if (in) {
          const float4 v = __ldcs(reinterpret_cast<const float4*>(P0 + (int64_t)j * ld + cb) + lane);
          acc[0] += (T)v.x * gj;
          acc[1] += (T)v.y * gj;
          acc[2] += (T)v.z * gj;
          acc[3] += (T)v.w * gj;
        }
      }
    } else {
#pragma unroll 4
      for (int j = r0 + warp; j < r1; j += 8) {
        const T gj = (T)gl[og + j];
        const T* row = P0 + (int64_t)j * ld + cb;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const int c = lane + 32 * t;
          if (cb + c < ncs) acc[t] += row[c] * gj;
        }
      }
    }
    __syncthreads();  // red is reused across column blocks
#pragma unroll
    for (int t = 0; t < 4; ++t) red[warp][sizeof(T) == 4 ? 4 * lane + t : lane + 32 * t] = (double)acc[t];
    __syncthreads();
    for (int c = threadIdx.x; c < 128 && cb + c < ncs; c += blockDim.x) {
      double v = 0.0;
      for (int w = 0; w < 8; ++w) v += red[w][c];
      clp[(offC[s] + cb + c) * nchunk + chunk] = v;
    }
  }
}

// rc[p] = sum over the listed local primal entries of all their chunks
// (cnch[q]: chunks of the subdomain that owns local entry q).
__global__ void coarse_rhs_kernel(const int* __restrict__ ptr, const int* __restrict__ src, int n,
                                  const double* __restrict__ clp, int nchunk,
                                  const int* __restrict__ cnch, double* __restrict__ rc) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n) return;
  double v = 0.0;
  for (int j = ptr[m]; j < ptr[m + 1]; ++j) {
    const double* q = clp + (int64_t)src[j] * nchunk;
    const int nc = cnch[src[j]];
    for (int c = 0; c < nc; ++c) v += q[c];
  }
  rc[m] = v;
}

__global__ void dense_gemv_kernel(const double* __restrict__ A, int n, const double* __restrict__ x,
                                  double* __restrict__ y) {
  const int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double* a = A + (int64_t)row * n;
  double acc = 0.0;
  for (int j = lane; j < n; j += 32) acc += a[j] * __ldg(&x[j]);
  acc = warp_sum(acc);
  if (lane == 0) y[row] = acc;
}

// Deluxe blocks of the apply: out[og + pos_j] = sum_i M_b[i][j] x_i for the
// class DoFs of block b (og: the subdomain's first interface position).
// Restriction: x_i = gI[gam_if[og + pos_i]] (assembled interface values),
// M_b = D_b, so g_i gets D_b^T g on the class.  Extension: x_i = yG[og +
// pos_i], M_b = E_b = D_b^T, so the class part of y_i becomes D_b y_i.
// Inputs and outputs are different vectors, so the 64-column slices of a
// block (blockIdx.y) run independently.  Thread (g, c) sums rows i = g mod
// 4 of column c (a warp reads 32 consecutive entries of a row), and the
// four partial sums are added in a fixed order.
constexpr int DLX_COLS = 64, DLX_RG = 4;
template <typename T, bool GATHER>
__global__ void __launch_bounds__(DLX_COLS * DLX_RG)
deluxe_apply_kernel(const int* __restrict__ bn, const int* __restrict__ bsub, const int* __restrict__ bld,
                    const int64_t* __restrict__ poff, const int* __restrict__ pos,
                    const int64_t* __restrict__ boff, const int64_t* __restrict__ offGam,
                    const int* __restrict__ gam_if, const T* __restrict__ M,
                    const double* __restrict__ in, double* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  __shared__ T part[DLX_RG][DLX_COLS];
  const int b = blockIdx.x;
  const int n = bn[b];
  const int j0 = blockIdx.y * DLX_COLS;
  if (j0 >= n) return;  // whole CTA
  const int64_t og = offGam[bsub[b]];
  const int* p = pos + poff[b];
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t q = og + p[i];
    xs[i] = (T)(GATHER ? in[gam_if[q]] : in[q]);
  }
  __syncthreads();
  const int c = threadIdx.x % DLX_COLS, g = threadIdx.x / DLX_COLS;
  const int j = j0 + c;
  T acc = T(0);
  if (j < n) {
    const T* Mb = M + boff[b] + j;
    const int64_t ld = bld[b];
#pragma unroll 4
    for (int i = g; i < n; i += DLX_RG) acc = fma(Mb[i * ld], xs[i], acc);
  }
  part[g][c] = acc;
  __syncthreads();
  if (g == 0 && j < n) {
    T v = part[0][c];
#pragma unroll
    for (int q = 1; q < DLX_RG; ++q) v += part[q][c];
    out[og + p[j]] = (double)v;
  }
}

// y_i = D_i (w_i + Phi_i R_Pi u_c); 8 lanes per interface row.
template <typename T>
__global__ void __launch_bounds__(256)
apply_prolong_kernel(const int2* __restrict__ items, const int* __restrict__ nG, const int* __restrict__ nc,
                     const int64_t* __restrict__ offPhi, const int* __restrict__ ldPhi,
                     const int64_t* __restrict__ offGam, const int64_t* __restrict__ offC,
                     const int* __restrict__ gprim, const T* __restrict__ Phi,
                     const double* __restrict__ uc, const double* __restrict__ wG,
                     const double* __restrict__ Dg, double* __restrict__ yG) {
  using V = typename Vec2<T>::type;
  constexpr int W = Vec2<T>::W;
  __shared__ __align__(16) T ucl[NC_MAX];
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const int ng = nG[s], ncs = nc[s];
  const int r0 = it.y * AROWS;
  if (r0 >= ng) return;
  for (int c = threadIdx.x; c < ncs; c += blockDim.x) ucl[c] = (T)uc[gprim[offC[s] + c]];
  __syncthreads();
  const int sub = threadIdx.x & 7, grp = threadIdx.x >> 3;  // 32 groups of 8 lanes
  // the CTA's rows in passes of 32 (uniform trip count: the shuffles below
  // need every lane of the warp)
  for (int pass = 0; pass < AROWS / 32; ++pass) {
    const int row = r0 + grp + 32 * pass;
    T acc = T(0);  // operator precision, as in the other local products
    if (row < ng) {
      // rows start 16-byte aligned (block offsets are multiples of 64
      // elements, leading dimensions of 4): 8 lanes read 8 consecutive
      // 16-byte chunks
      const T* pr = Phi + offPhi[s] + (int64_t)row * ldPhi[s];
      const V* pv = reinterpret_cast<const V*>(pr);
      const V* uv = reinterpret_cast<const V*>(ucl);
      const int nv = ncs / W;
#pragma unroll 2
      for (int c = sub; c < nv; c += 8) acc += vdot2(__ldcs(pv + c), uv[c]);
      for (int c = nv * W + sub; c < ncs; c += 8) acc += pr[c] * ucl[c];
    }
    acc += __shfl_xor_sync(0xffffffffu, acc, 4);
    acc += __shfl_xor_sync(0xffffffffu, acc, 2);
    acc += __shfl_xor_sync(0xffffffffu, acc, 1);
    if (row < ng && sub == 0) {
      const int64_t og = offGam[s];
      yG[og + row] = Dg[og + row] * (wG[og + row] + (double)acc);
    }
  }
}

// z_G = sum over sharing subdomains of yG; also written to every packed
// local interface position (zl), the input of the harmonic extension, and,
// if zq is given, node-packed in the operator precision (the coupling
// product's input; interface DoFs are node-major, 3 per node).
template <typename T>
__global__ void average_kernel(const int* __restrict__ if_dof, const int* __restrict__ if_ptr,
                               const int* __restrict__ if_src, int n_if, const double* __restrict__ yG,
                               double* __restrict__ z, double* __restrict__ zl, T* __restrict__ zq) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= n_if) return;
  double v = 0.0;
  for (int j = if_ptr[m]; j < if_ptr[m + 1]; ++j) v += yG[if_src[j]];
  z[if_dof[m]] = v;
  for (int j = if_ptr[m]; j < if_ptr[m + 1]; ++j) zl[if_src[j]] = v;
  if (zq) zq[m / 3 * 4 + m % 3] = (T)v;
}

template <typename T>
__global__ void __launch_bounds__(256)
apply_extend_kernel(const int2* __restrict__ items, const int* __restrict__ nI, const int* __restrict__ nG,
                    const int64_t* __restrict__ offA, const int* __restrict__ ldA,
                    const int64_t* __restrict__ offI, const int64_t* __restrict__ offGam,
                    const int* __restrict__ gdofI, const T* __restrict__ Aloc,
                    const double* __restrict__ zl, const double* __restrict__ u0, double* __restrict__ z) {
  extern __shared__ __align__(16) unsigned char smraw[];
  T* xs = reinterpret_cast<T*>(smraw);
  const int2 it = items[blockIdx.x];
  const int s = it.x;
  const int ni = nI[s], ng = nG[s];
  const int rb = it.y * GROWS * GGROUPS;
  if (rb >= ni) return;
  const int re = min(ni, rb + GROWS * GGROUPS);
  const int64_t oi = offI[s];
  if (ng == 0) {
    for (int row = rb + threadIdx.x; row < re; row += blockDim.x) z[gdofI[oi + row]] = u0[oi + row];
    return;
  }
  load_x<T>(xs, zl + offGam[s], ng);
  const int cI = (ni + 3) / 4 * 4;
  gemv_rows<T>(Aloc + offA[s] + cI, ldA[s], rb, re, xs, ng,
               [&](int row, T v) { z[gdofI[oi + row]] = u0[oi + row] - (double)v; });
}

// Local coarse matrix of subdomain s (n_c x n_c, node-major: 3 DoFs per
// coarse node) -> 3x3 contribution blocks of the coarse problem, block
// (a, b) at cbase[s] + a * (n_c / 3) + b.
template <typename T>
__global__ void kc_to_blocks_kernel(const int* __restrict__ nc, const int64_t* __restrict__ offKc,
                                    const int* __restrict__ ldPhi, const int64_t* __restrict__ cbase,
                                    const T* __restrict__ Kc, double* __restrict__ blocks) {
  const int s = blockIdx.y;
  const int n = nc[s];
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * n) return;
  const int i = (int)(t / n), j = (int)(t % n);
  const int k = n / 3;
  const int a = i / 3, b = j / 3;
  blocks[(cbase[s] + (int64_t)a * k + b) * 9 + (i % 3) * 3 + (j % 3)] =
      (double)Kc[offKc[s] + (int64_t)i * ldPhi[s] + j];
}

__global__ void or_status_kernel(const int* __restrict__ from, int* __restrict__ to) {
  if (*from) atomicOr(to, *from);
}

}  // namespace

// ------------------------------------------------------------------ create
// The coarse problem of C as an unassembled matrix (Section 3.2, multilevel
// BDDC): nodes are the coarse nodes (3 consecutive primal DoFs each), the
// elements are the subdomains of C with their local coarse matrices, and
// C->part2 groups them into the level-2 subdomains.  No node is clamped.
static void build_coarse_problem(bddc_ctx* C, fem_problem* CP) {
  const int nsub = C->nsub;
  const int nn = C->n_pi / 3;
  CP->elem_type = 0;
  CP->n_nodes = nn;
  CP->n_el = nsub;
  CP->n_parts = C->n_parts2;
  CP->n_free_nodes = nn;
  CP->n_free = 3 * (int64_t)nn;
  CP->node_to_free.resize(nn);
  for (int v = 0; v < nn; ++v) CP->node_to_free[v] = v;
  std::vector<int> eptr{0}, eidx;
  std::vector<int64_t> cbase;
  int64_t nb = 0;
  for (int s = 0; s < nsub; ++s) {
    const int k = C->nc[s] / 3;
    for (int q = 0; q < k; ++q) eidx.push_back(C->gprim_h[C->offC[s] + 3 * q] / 3);
    eptr.push_back((int)eidx.size());
    cbase.push_back(nb);
    nb += (int64_t)k * k;
  }
  std::vector<std::vector<int>> members(nn);
  for (int s = 0; s < nsub; ++s)
    for (int q = eptr[s]; q < eptr[s + 1]; ++q) members[eidx[q]].push_back(C->part2[s]);
  CP->share_count.assign(nn, 0);
  for (int v = 0; v < nn; ++v) {
    auto& mv = members[v];
    std::sort(mv.begin(), mv.end());
    mv.erase(std::unique(mv.begin(), mv.end()), mv.end());
    CP->share_count[v] = (int)mv.size();
  }
  CP->subs.assign(CP->n_parts, SubHost{});
  for (int v = 0; v < nn; ++v)
    for (int g : members[v]) {
      CP->subs[g].nodes.push_back(v);
      CP->subs[g].iface.push_back(CP->share_count[v] >= 2 ? 1 : 0);
    }
  for (int g = 0; g < CP->n_parts; ++g)
    CB_CHECK(!CP->subs[g].nodes.empty(), CBDDC_EINVAL, "level-2 subdomain without coarse nodes");
  classify_interface(nn, members, CP->share_count, eptr, eidx, nullptr, CP->vertices, CP->edges,
                     CP->faces);
  build_local_slots(CP, eptr, eidx, C->part2, cbase);
  CP->n_elem_blocks = nb;
  CP->contrib.alloc((size_t)std::max<int64_t>(nb, 1) * 9);
  CP->status.alloc(4);
  CB_CUDA(cudaMemset(CP->status.p, 0, CP->status.bytes()));
  CP->has_tangent = true;
  C->d_cbase.upload(cbase);
}

void bddc_create(fem_problem* P, const bddc_options* opt, bddc_ctx* C) {
  CB_CHECK(opt != nullptr, CBDDC_EINVAL, "null options");
  CB_CHECK(opt->precision == CBDDC_FP64 || opt->precision == CBDDC_FP32, CBDDC_EINVAL, "bad precision");
  C->P = P;
  C->precision = opt->precision;
  C->primal = opt->primal;
  C->pivot_tol = opt->pivot_tol > 0 ? opt->pivot_tol : 1e-13;
  C->levels = opt->levels >= 3 ? 3 : 2;
  CB_CHECK(opt->levels <= 3, CBDDC_EINVAL, "at most three levels are supported");
  if (C->levels == 3) {
    CB_CHECK(opt->part2 != nullptr && opt->n_parts2 >= 1, CBDDC_EINVAL, "multilevel BDDC needs part2");
    C->n_parts2 = opt->n_parts2;
    C->primal2 = opt->primal2 ? opt->primal2 : (CBDDC_PRIMAL_V | CBDDC_PRIMAL_E | CBDDC_PRIMAL_F);
    CB_CHECK(opt->precision2 == CBDDC_FP64 || opt->precision2 == CBDDC_FP32, CBDDC_EINVAL,
             "bad precision2");
    C->precision2 = opt->precision2;
    C->part2.assign(opt->part2, opt->part2 + P->n_parts);
    for (int g : C->part2) CB_CHECK(g >= 0 && g < C->n_parts2, CBDDC_EINVAL, "part2 out of range");
  }
  C->esize = opt->precision == CBDDC_FP32 ? 4 : 8;
  CB_CHECK(opt->sweep_block == 0 || opt->sweep_block == 64 ||
               (opt->sweep_block == 128 && opt->precision == CBDDC_FP32),
           CBDDC_EINVAL, "sweep_block must be 0, 64, or 128 with FP32 operators");
  C->nb = opt->sweep_block == 128 ? 128 : SWEEP_NB;
  CB_CHECK(opt->tile_order == 0 || opt->tile_order == 1, CBDDC_EINVAL, "tile_order must be 0 or 1");
  C->tile_order = opt->tile_order;
  const int nsub = P->n_parts;
  C->nsub = nsub;
  const bool useV = opt->primal & CBDDC_PRIMAL_V;
  const bool useE = opt->primal & CBDDC_PRIMAL_E;
  const bool useF = opt->primal & CBDDC_PRIMAL_F;
  const bool useR = opt->primal & CBDDC_PRIMAL_R;
  const int nn = P->n_nodes;
  CB_CHECK(!useR || (C->levels == 2 && P->coords_h.size() == (size_t)nn * 3), CBDDC_EINVAL,
           "rotational primal constraints need the two-level method on the fine level");
  CB_CHECK(C->levels == 2 || !(C->primal2 & CBDDC_PRIMAL_R), CBDDC_EINVAL,
           "rotational primal constraints are not available on level 2");
  CB_CHECK(opt->scaling == CBDDC_SCALING_COUNTING || opt->scaling == CBDDC_SCALING_DELUXE, CBDDC_EINVAL,
           "bad scaling");
  C->scaling = opt->scaling;
  const bool deluxe = opt->scaling == CBDDC_SCALING_DELUXE;
  CB_CHECK(opt->coarse == CBDDC_COARSE_GALERKIN || opt->coarse == CBDDC_COARSE_PETROV, CBDDC_EINVAL,
           "bad coarse space");
  C->coarse = opt->coarse;
  // deluxe classes: every edge and face (vertex nodes keep counting)
  std::vector<const std::vector<int>*> dcls;
  std::vector<int> node_dcls(nn, -1);
  if (deluxe) {
    for (auto& e : P->edges) dcls.push_back(&e);
    for (auto& f : P->faces) dcls.push_back(&f);
    CB_CHECK(dcls.size() <= 65535, CBDDC_EINVAL, "deluxe scaling allows at most 65535 interface classes");
    for (size_t k = 0; k < dcls.size(); ++k) {
      CB_CHECK(!dcls[k]->empty() && dcls[k]->size() <= 1024, CBDDC_EINVAL,
               "deluxe scaling allows classes of 1 to 1024 nodes");
      for (int v : *dcls[k]) node_dcls[v] = (int)k;
    }
  }
  // deluxe blocks (class, subdomain) and the class DoFs' interface positions
  std::vector<int> dlx_cls, dlx_sub_h;
  std::vector<std::vector<int>> dlx_pos_h;
  std::vector<int> vert_pos(nn, -1);
  int n_vert = 0;
  if (useV)
    for (int v : P->vertices) vert_pos[v] = n_vert++;
  std::vector<const std::vector<int>*> avg;
  if (useE) for (auto& e : P->edges) avg.push_back(&e);
  if (useF) for (auto& f : P->faces) avg.push_back(&f);
  std::vector<int> node_cls(nn, -1);
  for (size_t j = 0; j < avg.size(); ++j)
    for (int v : *avg[j]) node_cls[v] = (int)j;
  // per class: 3 averages, then its rotations (rows of 3 * |class| weights
  // at rot_w[rot_off[j]]); global primal numbering: vertex DoFs, then the
  // constraints of each class at apos[j]
  std::vector<int> nrot(avg.size(), 0);
  std::vector<int64_t> rot_off(avg.size(), 0);
  std::vector<double> rot_w;
  std::vector<int> apos(avg.size(), 0);
  int n_pi = 3 * n_vert;
  for (size_t j = 0; j < avg.size(); ++j) {
    rot_off[j] = (int64_t)rot_w.size();
    if (useR) nrot[j] = class_rotations(P->coords_h, *avg[j], rot_w);
    apos[j] = n_pi;
    n_pi += 3 + nrot[j];
  }
  C->n_pi = n_pi;

  C->nI.assign(nsub, 0); C->nG = C->nr = C->nv = C->na = C->nc = C->ns = C->nI;
  std::vector<int> perm_h;
  std::vector<int64_t> offN(nsub + 1, 0);
  std::vector<int> gdofI, gdofG, gprim;
  std::vector<double> Dg;
  std::vector<int> cptr{0}, cidx;
  std::vector<double> cw;
  C->offI.assign(nsub + 1, 0);
  C->offGam.assign(nsub + 1, 0);
  C->offC.assign(nsub + 1, 0);
  C->offCon.assign(nsub + 1, 0);
  const std::vector<int>& n2f = P->node_to_free;
  for (int s = 0; s < nsub; ++s) {
    const auto& sub = P->subs[s];
    const int nl = (int)sub.nodes.size();
    std::vector<int> I, Gr, Gv;
    for (int l = 0; l < nl; ++l) {
      if (!sub.iface[l]) I.push_back(l);
      else if (vert_pos[sub.nodes[l]] >= 0) Gv.push_back(l);
      else Gr.push_back(l);
    }
    std::vector<int> perm(nl);
    int pos = 0;
    for (int l : I) perm[l] = pos++;
    std::vector<int> rpos(nl, -1);
    for (int l : Gr) { rpos[l] = pos - (int)I.size(); perm[l] = pos++; }
    for (int l : Gv) perm[l] = pos++;
    perm_h.insert(perm_h.end(), perm.begin(), perm.end());
    offN[s + 1] = offN[s] + nl;
    C->nI[s] = 3 * (int)I.size();
    C->nr[s] = 3 * (int)Gr.size();
    C->nv[s] = 3 * (int)Gv.size();
    C->nG[s] = C->nr[s] + C->nv[s];
    C->ns[s] = C->nI[s] + C->nG[s];
    for (int l : I)
      for (int c = 0; c < 3; ++c) gdofI.push_back(3 * n2f[sub.nodes[l]] + c);
    for (const std::vector<int>* lst : {&Gr, &Gv})
      for (int l : *lst)
        for (int c = 0; c < 3; ++c) {
          gdofG.push_back(3 * n2f[sub.nodes[l]] + c);
          Dg.push_back(node_dcls[sub.nodes[l]] >= 0 ? 1.0 : 1.0 / P->share_count[sub.nodes[l]]);
        }
    if (deluxe) {
      std::vector<int> dk;
      for (int l : Gr)
        if (node_dcls[sub.nodes[l]] >= 0) dk.push_back(node_dcls[sub.nodes[l]]);
      std::sort(dk.begin(), dk.end());
      dk.erase(std::unique(dk.begin(), dk.end()), dk.end());
      for (int k : dk) {
        std::vector<int> ps;
        for (int v : *dcls[k]) {
          auto it = std::lower_bound(sub.nodes.begin(), sub.nodes.end(), v);
          CB_CHECK(it != sub.nodes.end() && *it == v, CBDDC_EINVAL, "class node not in subdomain");
          const int l = (int)(it - sub.nodes.begin());
          CB_CHECK(rpos[l] >= 0, CBDDC_EINVAL, "class node is not a dual interface node");
          for (int c = 0; c < 3; ++c) ps.push_back(3 * rpos[l] + c);
        }
        dlx_cls.push_back(k);
        dlx_sub_h.push_back(s);
        dlx_pos_h.push_back(std::move(ps));
      }
    }
    // average constraints of classes touching this subdomain
    std::vector<int> cls;
    for (int l : Gr)
      if (node_cls[sub.nodes[l]] >= 0) cls.push_back(node_cls[sub.nodes[l]]);
    std::sort(cls.begin(), cls.end());
    cls.erase(std::unique(cls.begin(), cls.end()), cls.end());
    const size_t con0 = cptr.size();
    for (int j : cls) {
      const std::vector<int>& cn = *avg[j];
      std::vector<int> rl(cn.size());  // r-block position of each class node
      for (size_t a = 0; a < cn.size(); ++a) {
        auto it = std::lower_bound(sub.nodes.begin(), sub.nodes.end(), cn[a]);
        CB_CHECK(it != sub.nodes.end() && *it == cn[a], CBDDC_EINVAL, "class node not in subdomain");
        const int l = (int)(it - sub.nodes.begin());
        CB_CHECK(rpos[l] >= 0, CBDDC_EINVAL, "class node is not a dual interface node");
        rl[a] = rpos[l];
      }
      for (int c = 0; c < 3; ++c) {  // averages: weight 1 / |class| per member
        for (int r : rl) {
          cidx.push_back(3 * r + c);
          cw.push_back(1.0 / (double)cn.size());
        }
        cptr.push_back((int)cidx.size());
      }
      for (int k = 0; k < nrot[j]; ++k) {  // rotations: all 3 components
        const double* wk = rot_w.data() + rot_off[j] + (int64_t)k * 3 * (int64_t)cn.size();
        for (size_t a = 0; a < cn.size(); ++a)
          for (int c = 0; c < 3; ++c) {
            cidx.push_back(3 * rl[a] + c);
            cw.push_back(wk[3 * a + c]);
          }
        cptr.push_back((int)cidx.size());
      }
    }
    C->na[s] = (int)(cptr.size() - con0);
    C->nc[s] = C->nv[s] + C->na[s];
    CB_CHECK(C->nc[s] <= NC_MAX, CBDDC_EINVAL, "more than 512 primal constraints in one subdomain");
    for (int l : Gv)
      for (int c = 0; c < 3; ++c) gprim.push_back(3 * vert_pos[sub.nodes[l]] + c);
    for (int j : cls)
      for (int c = 0; c < 3 + nrot[j]; ++c) gprim.push_back(apos[j] + c);
    C->offI[s + 1] = C->offI[s] + C->nI[s];
    C->offGam[s + 1] = C->offGam[s] + C->nG[s];
    C->offC[s + 1] = C->offC[s] + C->nc[s];
    C->offCon[s + 1] = C->offCon[s] + C->na[s];
  }
  C->totI = C->offI[nsub];
  C->totG = C->offGam[nsub];
  C->totC = C->offC[nsub];

  // interface DoFs: global list and gather lists from packed Gamma positions
  std::vector<int> node_if(nn, -1);
  std::vector<int> if_dof;
  for (int v = 0; v < nn; ++v)
    if (n2f[v] >= 0 && P->share_count[v] >= 2) {
      node_if[v] = (int)(if_dof.size() / 3);
      for (int c = 0; c < 3; ++c) if_dof.push_back(3 * n2f[v] + c);
    }
  C->n_if = (int)if_dof.size();
  std::vector<int> gam_if(C->totG);
  std::vector<std::pair<int64_t, int>> ikv;
  {
    // map free DoF -> interface index
    std::vector<int> dof_if(P->n_free, -1);
    for (int m = 0; m < C->n_if; ++m) dof_if[if_dof[m]] = m;
    for (int64_t q = 0; q < C->totG; ++q) {
      const int m = dof_if[gdofG[q]];
      CB_CHECK(m >= 0, CBDDC_EINVAL, "interface DoF without interface index");
      gam_if[q] = m;
      ikv.push_back({m, (int)q});
    }
  }
  std::vector<int> if_ptr(C->n_if + 1, 0), if_src(ikv.size());
  for (auto& e : ikv) if_ptr[e.first + 1]++;
  for (int m = 0; m < C->n_if; ++m) if_ptr[m + 1] += if_ptr[m];
  {
    std::vector<int> fill(if_ptr.begin(), if_ptr.end() - 1);
    for (auto& e : ikv) if_src[fill[e.first]++] = e.second;
  }
  // coarse rhs gather
  std::vector<int> cg_ptr(C->n_pi + 1, 0), cg_src(C->totC);
  for (int64_t q = 0; q < C->totC; ++q) cg_ptr[gprim[q] + 1]++;
  for (int p = 0; p < C->n_pi; ++p) cg_ptr[p + 1] += cg_ptr[p];
  {
    std::vector<int> fill(cg_ptr.begin(), cg_ptr.end() - 1);
    for (int64_t q = 0; q < C->totC; ++q) cg_src[fill[gprim[q]]++] = (int)q;
  }

  // packed storage layout
  const int NB = C->nb;
  C->ldA.assign(nsub, 0); C->ldS = C->ldPhi = C->ldY = C->ldG = C->ldA;
  C->offA.assign(nsub + 1, 0); C->offS = C->offPhi = C->offY = C->offZ = C->offG = C->offSPhi =
      C->offKc = C->offX = C->offYp = C->offP = C->offE = C->offA;
  for (int s = 0; s < nsub; ++s) {
    const int cI = (int)round_up(C->nI[s], 4);
    C->ldA[s] = (int)round_up(cI + C->nG[s], 8);
    C->ldS[s] = (int)round_up(std::max(C->nG[s], 1), 8);
    C->ldPhi[s] = (int)round_up(std::max(C->nc[s], 1), 4);
    C->ldY[s] = (int)round_up(std::max(C->na[s], 1), 4);
    C->ldG[s] = C->ldY[s];
    C->offA[s + 1] = C->offA[s] + round_up((int64_t)C->ns[s] * C->ldA[s], kAlign);
    C->offS[s + 1] = C->offS[s] + round_up((int64_t)C->nG[s] * C->ldS[s], kAlign);
    C->offPhi[s + 1] = C->offPhi[s] + round_up((int64_t)C->nG[s] * C->ldPhi[s], kAlign);
    C->offSPhi[s + 1] = C->offPhi[s + 1];
    C->offY[s + 1] = C->offY[s] + round_up((int64_t)C->nr[s] * C->ldY[s], kAlign);
    C->offZ[s + 1] = C->offZ[s] + round_up((int64_t)C->na[s] * C->ldS[s], kAlign);
    C->offG[s + 1] = C->offG[s] + round_up((int64_t)C->na[s] * C->ldG[s], kAlign);
    C->offKc[s + 1] = C->offKc[s] + round_up((int64_t)C->nc[s] * C->ldPhi[s], kAlign);
    C->offX[s + 1] = C->offX[s] + round_up((int64_t)C->ns[s] * NB, kAlign);
    C->offYp[s + 1] = C->offYp[s] + round_up((int64_t)NB * C->ldA[s], kAlign);
    C->offP[s + 1] = C->offP[s] + NB * NB;
    C->offE[s + 1] = C->offE[s] + round_up((int64_t)C->nI[s] * C->ldS[s], kAlign);
    C->maxI = std::max(C->maxI, C->nI[s]);
    C->maxG = std::max(C->maxG, C->nG[s]);
    C->maxR = std::max(C->maxR, C->nr[s]);
    C->maxNs = std::max(C->maxNs, C->ns[s]);
    C->maxC = std::max(C->maxC, C->nc[s]);
    C->maxA = std::max(C->maxA, C->na[s]);
  }
  // every operand buffer gets kAlign elements of slack for masked vector loads
  const size_t es = C->esize;
  auto sized = [&](int64_t n) { return (size_t)(std::max<int64_t>(n, 1) + kAlign) * es; };
  C->Aloc.alloc(sized(C->offA[nsub]));
  C->Sw.alloc(sized(C->offS[nsub]));
  C->Phi.alloc(sized(C->offPhi[nsub]));
  C->SPhi.alloc(sized(C->offPhi[nsub]));
  C->Y.alloc(sized(C->offY[nsub]));
  C->Zf.alloc(sized(C->offZ[nsub]));
  C->Wf.alloc(sized(C->offZ[nsub]));
  C->G.alloc(sized(C->offG[nsub]));
  C->Kc.alloc(sized(C->offKc[nsub]));
  C->Xp.alloc(sized(C->offX[nsub]));
  C->Yp.alloc(sized(C->offYp[nsub]));
  C->Pd.alloc(sized(C->offP[nsub]));
  C->Et.alloc(sized(C->offE[nsub]));

  // sweep descriptors and GEMM problem lists.
  // Interior elimination: sweep of the A_II block alone (A_II^-1 in place),
  // then E = A_II^-1 A_IG and S = A_GG - A_GI E as two large-K GEMMs; E is
  // copied over A_IG afterwards (A_IG is not needed once S is formed).
  // The constraint matrix G = C S_rr^-1 C^T (n_a x n_a) is inverted by a
  // third sweep; its panels fit the same X / Y buffers (n_a <= n_s rows,
  // ld_G <= ld_A columns).
  std::vector<SweepDesc> sw1(nsub), sw2(nsub), swg(nsub);
  for (int s = 0; s < nsub; ++s) {
    sw1[s] = SweepDesc{C->nI[s], C->nI[s], C->ldA[s], C->nI[s], C->offA[s], C->offX[s], C->offYp[s],
                       C->offP[s]};
    sw2[s] = SweepDesc{C->nG[s], C->nG[s], C->ldS[s], C->nr[s], C->offS[s], C->offX[s], C->offYp[s],
                       C->offP[s]};
    swg[s] = SweepDesc{C->na[s], C->na[s], C->ldG[s], C->na[s], C->offG[s], C->offX[s], C->offYp[s],
                       C->offP[s]};
    C->steps1 = std::max(C->steps1, (int)cdiv(C->nI[s], NB));
    C->steps2 = std::max(C->steps2, (int)cdiv(C->nr[s], NB));
    C->stepsg = std::max(C->stepsg, (int)cdiv(C->na[s], NB));
  }
  C->sw1.upload(sw1);
  C->sw2.upload(sw2);
  C->swg.upload(swg);
  const int to_sw = C->tile_order;
  auto sweep_gemms = [NB, es, to_sw](const std::vector<SweepDesc>& sw, int steps, std::vector<GemmList>& out) {
    const int to = to_sw;
    const int nmat = (int)sw.size();
    out.clear();
    out.resize(steps);
    for (int k = 0; k < steps; ++k) {
      std::vector<GemmProb> g;
      for (int s = 0; s < nmat; ++s) {
        const SweepDesc& d = sw[s];
        const int kb = std::max(0, std::min(NB, d.p - k * NB));
        g.push_back(GemmProb{d.rows, d.cols, kb, NB, d.ld, d.ld, d.offX, d.offY, d.off});
      }
      out[k].set(g, es, false, to);
    }
  };
  sweep_gemms(sw1, C->steps1, C->gl_sw1);
  sweep_gemms(sw2, C->steps2, C->gl_sw2);
  sweep_gemms(swg, C->stepsg, C->gl_swg);
  double dlx_flops = 0.0;   // deluxe setup: class inverses and D_b products
  int64_t dlx_bytes = 0;    // deluxe blocks read per apply (D_b and E_b)
  if (deluxe && !dlx_cls.empty()) {
    // blocks in (class, subdomain) order; S_b, D_b, E_b at the same offsets
    const int nb = (int)dlx_cls.size(), nk = (int)dcls.size();
    std::vector<int> order(nb);
    for (int b = 0; b < nb; ++b) order[b] = b;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
      return dlx_cls[a] != dlx_cls[b] ? dlx_cls[a] < dlx_cls[b] : dlx_sub_h[a] < dlx_sub_h[b];
    });
    std::vector<int> bn(nb), bsub(nb), bld(nb), bpos, cptr(nk + 1, 0), cblk(nb);
    std::vector<int64_t> bpoff(nb), boff(nb + 1, 0);
    for (int q = 0; q < nb; ++q) {
      const int b = order[q];
      bn[q] = (int)dlx_pos_h[b].size();
      bsub[q] = dlx_sub_h[b];
      bld[q] = (int)round_up(bn[q], 8);
      bpoff[q] = (int64_t)bpos.size();
      bpos.insert(bpos.end(), dlx_pos_h[b].begin(), dlx_pos_h[b].end());
      boff[q + 1] = boff[q] + round_up((int64_t)bn[q] * bld[q], kAlign);
      cptr[dlx_cls[b] + 1]++;
      cblk[q] = q;
      C->maxDn = std::max(C->maxDn, bn[q]);
    }
    for (int k = 0; k < nk; ++k) cptr[k + 1] += cptr[k];
    CB_CHECK(cptr[nk] == nb, CBDDC_EINVAL, "deluxe block lists are inconsistent");
    // class matrices Shat_K (inverted in place by a sweep) and sweep panels
    std::vector<int64_t> coff(nk + 1, 0);
    std::vector<SweepDesc> swd(nk);
    int64_t xo = 0, yo = 0;
    for (int k = 0; k < nk; ++k) {
      CB_CHECK(cptr[k + 1] > cptr[k], CBDDC_EINVAL, "interface class without subdomains");
      const int q0 = cptr[k];
      const int n = bn[q0], ld = bld[q0];
      for (int q = q0; q < cptr[k + 1]; ++q) {
        CB_CHECK(bn[q] == n, CBDDC_EINVAL, "deluxe blocks of one class differ in size");
        dlx_flops += 2.0 * n * (double)n * n;
        dlx_bytes += 2 * (int64_t)n * n * (int64_t)es;
      }
      dlx_flops += 2.0 * n * (double)n * n;
      coff[k + 1] = coff[k] + round_up((int64_t)n * ld, kAlign);
      swd[k] = SweepDesc{n, n, ld, n, coff[k], xo, yo, (int64_t)k * NB * NB};
      xo += round_up((int64_t)n * NB, kAlign);
      yo += round_up((int64_t)NB * ld, kAlign);
      C->stepsd = std::max(C->stepsd, (int)cdiv(n, NB));
    }
    C->n_dlx = nb;
    C->n_dcls = nk;
    C->dlx_n.upload(bn); C->dlx_sub.upload(bsub); C->dlx_ld.upload(bld); C->dlx_pos.upload(bpos);
    C->dlx_poff.upload(bpoff); C->dlx_off.upload(boff); C->dcls_ptr.upload(cptr); C->dcls_blk.upload(cblk);
    C->dcls_off.upload(coff);
    C->swd.upload(swd);
    sweep_gemms(swd, C->stepsd, C->gl_swd);
    std::vector<GemmProb> gd(nb);
    for (int k = 0; k < nk; ++k)
      for (int q = cptr[k]; q < cptr[k + 1]; ++q)
        gd[q] = GemmProb{bn[q], bn[q], bn[q], bld[q], bld[q], bld[q], coff[k], boff[q], boff[q]};
    C->gl_dlx.set(gd, es, false, C->tile_order);
    auto sz = [&](int64_t n) { return (size_t)(std::max<int64_t>(n, 1) + kAlign) * es; };
    C->Dsb.alloc(sz(boff[nb]));
    C->Ddb.alloc(sz(boff[nb]));
    C->Deb.alloc(sz(boff[nb]));
    C->Dsh.alloc(sz(coff[nk]));
    C->DX.alloc(sz(xo));
    C->DY.alloc(sz(yo));
    C->DP.alloc(sz((int64_t)nk * NB * NB));
    C->yD.alloc(std::max<int64_t>(C->totG, 1));
  }
  std::vector<GemmProb> gE, gS, gW, gT, gPA, gSP, gKc;
  for (int s = 0; s < nsub; ++s) {
    const int cI = (int)round_up(C->nI[s], 4);
    const int64_t aII = C->offA[s], aIG = C->offA[s] + cI;
    const int64_t aGI = C->offA[s] + (int64_t)C->nI[s] * C->ldA[s], aGG = aGI + cI;
    gE.push_back(GemmProb{C->nI[s], C->nG[s], C->nI[s], C->ldA[s], C->ldA[s], C->ldS[s], aII, aIG,
                          C->offE[s]});
    gS.push_back(GemmProb{C->nG[s], C->nG[s], C->nI[s], C->ldA[s], C->ldS[s], C->ldA[s], aGI, C->offE[s],
                          aGG});
    gW.push_back(GemmProb{C->na[s], C->nG[s], C->na[s], C->ldG[s], C->ldS[s], C->ldS[s], C->offG[s],
                          C->offZ[s], C->offZ[s]});
    gT.push_back(GemmProb{C->nr[s], C->nG[s], C->na[s], C->ldY[s], C->ldS[s], C->ldS[s], C->offY[s],
                          C->offZ[s], C->offS[s]});
    gPA.push_back(GemmProb{C->nr[s], C->na[s], C->na[s], C->ldY[s], C->ldG[s], C->ldPhi[s], C->offY[s],
                           C->offG[s], C->offPhi[s] + C->nv[s]});
    gSP.push_back(GemmProb{C->nG[s], C->nc[s], C->nG[s], C->ldA[s], C->ldPhi[s], C->ldPhi[s], aGG,
                           C->offPhi[s], C->offPhi[s]});
    gKc.push_back(GemmProb{C->nc[s], C->nc[s], C->nG[s], C->ldPhi[s], C->ldPhi[s], C->ldPhi[s],
                           C->offPhi[s], C->offPhi[s], C->offKc[s]});
  }
  const int to = C->tile_order;
  C->gl_E.set(gE, es, false, to);
  C->gl_S.set(gS, es, false, to);
  C->gl_W.set(gW, es, false, to);
  C->gl_T.set(gT, es, false, to);
  C->gl_PhiA.set(gPA, es, false, to);
  C->gl_SPhi.set(gSP, es, false, to);
  C->gl_Kc.set(gKc, es, true, to);
  if (C->coarse == CBDDC_COARSE_PETROV) {
    // Psi[0:nr, 0:nv] = -T^T S_vr^T (T: constrained inverse in Sw's rr
    // block; S_vr: vertex rows, r columns of the Schur complement in Aloc)
    std::vector<GemmProb> gPV;
    for (int s = 0; s < nsub; ++s) {
      const int cI = (int)round_up(C->nI[s], 4);
      const int64_t aGG = C->offA[s] + (int64_t)C->nI[s] * C->ldA[s] + cI;
      gPV.push_back(GemmProb{C->nr[s], C->nv[s], C->nr[s], C->ldS[s], C->ldA[s], C->ldPhi[s], C->offS[s],
                             aGG + (int64_t)C->nr[s] * C->ldA[s], C->offPhi[s]});
    }
    C->gl_PsiV.set(gPV, es, true, C->tile_order);
    C->Psi.alloc(sized(C->offPhi[nsub]));
  }

  C->gprim_h = gprim;
  // coarse matrix entries (two-level: dense FP64 coarse inverse)
  if (C->n_pi > 0 && C->levels == 2) {
    std::vector<std::pair<int64_t, int>> ckv;
    for (int s = 0; s < nsub; ++s)
      for (int i = 0; i < C->nc[s]; ++i)
        for (int j = 0; j < C->nc[s]; ++j)
          ckv.push_back({(int64_t)gprim[C->offC[s] + i] * C->n_pi + gprim[C->offC[s] + j],
                         (int)(C->offKc[s] + (int64_t)i * C->ldPhi[s] + j)});
    std::sort(ckv.begin(), ckv.end());
    std::vector<int> key, ptr{0}, src;
    for (size_t i = 0; i < ckv.size();) {
      size_t j = i;
      while (j < ckv.size() && ckv[j].first == ckv[i].first) ++j;
      key.push_back((int)ckv[i].first);
      for (size_t q = i; q < j; ++q) src.push_back(ckv[q].second);
      ptr.push_back((int)src.size());
      i = j;
    }
    CB_CHECK((int64_t)C->n_pi * C->n_pi < INT32_MAX, CBDDC_EINVAL, "coarse space too large");
    C->n_ce = (int64_t)key.size();
    C->ce_key.upload(key);
    C->ce_ptr.upload(ptr);
    C->ce_src.upload(src);
    C->Sc.alloc((size_t)C->n_pi * C->n_pi);
    const int NBc = SWEEP_NB;  // the FP64 coarse inverse keeps 64-wide pivot blocks
    C->ScX.alloc((size_t)C->n_pi * NBc);
    C->ScY.alloc((size_t)C->n_pi * NBc);
    C->ScP.alloc((size_t)NBc * NBc);
    std::vector<SweepDesc> swc{SweepDesc{C->n_pi, C->n_pi, C->n_pi, C->n_pi, 0, 0, 0, 0}};
    C->swc.upload(swc);
    C->stepsc = (int)cdiv(C->n_pi, NBc);
    {
      // the coarse matrix is FP64 whatever the local precision
      const int nmat = 1;
      C->gl_swc.clear();
      C->gl_swc.resize(C->stepsc);
      for (int k = 0; k < C->stepsc; ++k) {
        const SweepDesc& d = swc[0];
        const int kb = std::max(0, std::min(NBc, d.p - k * NBc));
        std::vector<GemmProb> g{GemmProb{d.rows, d.cols, kb, NBc, d.ld, d.ld, d.offX, d.offY, d.off}};
        C->gl_swc[k].set(g, 8);
        (void)nmat;
      }
    }
  }

  // work items (subdomain, row block) of the batched apply kernels: only
  // blocks that exist, so many small subdomains of uneven size cost no
  // empty CTAs
  {
    std::vector<int2> iI, iG, iP, iR;
    std::vector<int> cn(std::max<int64_t>(C->totC, 1), 0);
    for (int s = 0; s < nsub; ++s) {
      for (int b = 0; b < (int)cdiv(C->nI[s], GROWS * GGROUPS); ++b) iI.push_back(make_int2(s, b));
      for (int b = 0; b < (int)cdiv(C->nG[s], GROWS * GGROUPS); ++b) iG.push_back(make_int2(s, b));
      for (int b = 0; b < (int)cdiv(C->nG[s], AROWS); ++b) iR.push_back(make_int2(s, b));
      if (C->nc[s] > 0) {
        const int nch_s = (int)cdiv(C->nG[s], PHIT_ROWS);
        for (int b = 0; b < nch_s; ++b) iP.push_back(make_int2(s, b));
        for (int c = 0; c < C->nc[s]; ++c) cn[C->offC[s] + c] = nch_s;
      }
    }
    C->n_itI = (int)iI.size(); C->n_itG = (int)iG.size();
    C->n_itP = (int)iP.size(); C->n_itR = (int)iR.size();
    C->itI.upload(iI); C->itG.upload(iG); C->itP.upload(iP); C->itR.upload(iR);
    C->cnch.upload(cn);
  }

  // device copies of sizes and maps
  C->d_nI.upload(C->nI); C->d_nG.upload(C->nG); C->d_nr.upload(C->nr); C->d_nv.upload(C->nv);
  C->d_na.upload(C->na); C->d_nc.upload(C->nc); C->d_ns.upload(C->ns);
  C->d_ldA.upload(C->ldA); C->d_ldS.upload(C->ldS); C->d_ldPhi.upload(C->ldPhi);
  C->d_ldY.upload(C->ldY); C->d_ldG.upload(C->ldG);
  C->d_offA.upload(C->offA); C->d_offS.upload(C->offS); C->d_offPhi.upload(C->offPhi);
  C->d_offY.upload(C->offY); C->d_offZ.upload(C->offZ); C->d_offG.upload(C->offG);
  C->d_offSPhi.upload(C->offSPhi); C->d_offKc.upload(C->offKc); C->d_offE.upload(C->offE);
  C->d_offI.upload(C->offI); C->d_offGam.upload(C->offGam); C->d_offC.upload(C->offC);
  C->d_offCon.upload(C->offCon); C->d_offN.upload(offN);
  C->perm.upload(perm_h);
  C->gdofI.upload(gdofI); C->gdofG.upload(gdofG); C->Dg.upload(Dg);
  C->gam_if.upload(gam_if); C->if_dof.upload(if_dof); C->if_ptr.upload(if_ptr); C->if_src.upload(if_src);
  C->cons_ptr.upload(cptr); C->cons_idx.upload(cidx); C->cons_w.upload(cw);
  C->gprim.upload(gprim); C->cg_ptr.upload(cg_ptr); C->cg_src.upload(cg_src);
  C->u0.alloc(std::max<int64_t>(C->totI, 1));
  C->xI.alloc(std::max<int64_t>(C->totI, 1));
  C->zl.alloc(std::max<int64_t>(C->totG, 1));
  C->hG.alloc(std::max<int64_t>(C->totG, 1));
  C->wG.alloc(std::max<int64_t>(C->totG, 1));
  C->yG.alloc(std::max<int64_t>(C->totG, 1));
  C->gI.alloc(std::max(C->n_if, 1));
  C->cl.alloc(std::max<int64_t>(C->totC * (int64_t)cdiv(std::max(C->maxG, 1), PHIT_ROWS), 1));
  C->rc.alloc(std::max(C->n_pi, 1));
  C->uc.alloc(std::max(C->n_pi, 1));
  C->gl.alloc(std::max<int64_t>(C->totG, 1));
  // Sparse interior-interface coupling.  Every element holding an interior
  // DoF of a subdomain belongs to that subdomain, so sum_i R_i^T A_Gamma,I^(i)
  // u0_i is the assembled block K_Gamma,I times the interior solution, and
  // A_I,Gamma^(i) z_Gamma,i is K_I,Gamma z.  Problems that carry the global
  // BSR matrix (every problem built from a mesh) read these blocks there:
  // about 9 values per coupled node pair instead of the dense n_I x n_Gamma
  // blocks, and the harmonic extension becomes A_II^-1 (r_I - K_I,Gamma z)
  // instead of u0 - E z_Gamma (n_I^2 values instead of n_I n_Gamma).
  C->sparse_cpl = P->nnzb > 0 && P->bsr_vals.p != nullptr && C->totI > 0 && C->n_if > 0;
  if (C->sparse_cpl) {
    const int64_t nfn = P->n_free_nodes;
    std::vector<int> rp(nfn + 1), bc(P->nnzb);
    CB_CUDA(cudaMemcpy(rp.data(), P->bsr_row_ptr.p, rp.size() * sizeof(int), cudaMemcpyDeviceToHost));
    CB_CUDA(cudaMemcpy(bc.data(), P->bsr_col.p, bc.size() * sizeof(int), cudaMemcpyDeviceToHost));
    std::vector<int> int_of(nfn, -1);  // free node -> packed interior node
    std::vector<int> if_of(nfn, -1);   // free node -> interface node
    for (int64_t q = 0; q < C->totI; q += 3) int_of[gdofI[q] / 3] = (int)(q / 3);
    for (int m = 0; m < C->n_if; m += 3) if_of[if_dof[m] / 3] = m / 3;
    std::vector<int> gptr{0}, gcol, gsrc, iptr{0}, icol, isrc;
    for (int m = 0; m < C->n_if; m += 3) {
      const int f = if_dof[m] / 3;
      for (int b = rp[f]; b < rp[f + 1]; ++b)
        if (int_of[bc[b]] >= 0) { gcol.push_back(int_of[bc[b]]); gsrc.push_back(b); }
      gptr.push_back((int)gcol.size());
    }
    for (int64_t q = 0; q < C->totI; q += 3) {
      const int f = gdofI[q] / 3;
      for (int b = rp[f]; b < rp[f + 1]; ++b)
        if (if_of[bc[b]] >= 0) { icol.push_back(if_of[bc[b]]); isrc.push_back(b); }
      iptr.push_back((int)icol.size());
    }
    C->n_cpl_blocks = (int64_t)gcol.size() + (int64_t)icol.size();
    const SellHost gi = build_sell(gptr, gcol, gsrc), ig = build_sell(iptr, icol, isrc);
    C->n_sgi = (int)gi.len.size();
    C->n_sig = (int)ig.len.size();
    C->steps_gi = gi.steps;
    C->steps_ig = ig.steps;
    C->sgi_off.upload(gi.off); C->sgi_len.upload(gi.len); C->sgi_row.upload(gi.row);
    C->sgi_col.upload(gi.col); C->sgi_src.upload(gi.src);
    C->sig_off.upload(ig.off); C->sig_len.upload(ig.len); C->sig_row.upload(ig.row);
    C->sig_col.upload(ig.col); C->sig_src.upload(ig.src);
    C->sgi_val.alloc((size_t)std::max<int64_t>(gi.steps, 1) * 288 * C->esize);
    C->sig_val.alloc((size_t)std::max<int64_t>(ig.steps, 1) * 288 * C->esize);
    C->uq.alloc((size_t)(C->totI / 3) * 4 * C->esize);
    C->zq.alloc((size_t)(C->n_if / 3) * 4 * C->esize);
    CB_CUDA(cudaMemset(C->uq.p, 0, C->uq.bytes()));
    CB_CUDA(cudaMemset(C->zq.p, 0, C->zq.bytes()));
  }
  // flops of one setup and bytes of local operators read per apply
  double fl = 0.0;
  int64_t lb = 0;
  for (int s = 0; s < nsub; ++s) {
    const double n = C->ns[s], ni = C->nI[s], ng = C->nG[s], nr = C->nr[s], na = C->na[s], nc = C->nc[s];
    (void)n;
    fl += 2.0 * ni * ni * ni + 2.0 * ni * ni * ng + 2.0 * ng * ng * ni + 2.0 * ng * ng * nr +
          2.0 * na * na * ng + 2.0 * nr * na * ng + 2.0 * nr * na * na + 2.0 * ng * ng * nc +
          2.0 * nc * nc * ng;
    if (C->sparse_cpl) lb += (int64_t)((2.0 * ni * ni + nr * nr + 2.0 * ng * nc) * C->esize);
    else lb += (int64_t)((ni * ni + 2.0 * ni * ng + nr * nr + 2.0 * ng * nc) * C->esize);
  }
  // coupling blocks: 9 values and one column index each (padding of the
  // sliced layout not counted)
  if (C->sparse_cpl) lb += C->n_cpl_blocks * (int64_t)(9 * C->esize + 4);
  fl += dlx_flops;
  lb += dlx_bytes;
  // multilevel: coarse problem and its BDDC context
  if (C->levels == 3 && C->n_pi > 0) {
    C->coarse_prob.reset(new fem_problem);
    build_coarse_problem(C, C->coarse_prob.get());
    bddc_options o2{};
    // level-2 local operators in precision2; the coarsest problem (level
    // 2's own coarse matrix) is always FP64
    o2.precision = C->precision2;
    o2.primal = C->primal2;
    o2.pivot_tol = C->pivot_tol;
    o2.levels = 2;
    o2.coarse = C->coarse;
    C->next.reset(new bddc_ctx);
    bddc_create(C->coarse_prob.get(), &o2, C->next.get());
    fl += C->next->setup_flops;
    lb += C->next->local_bytes;
  } else {
    fl += 2.0 * (double)C->n_pi * C->n_pi * C->n_pi;
    lb += (int64_t)C->n_pi * C->n_pi * 8;
  }
  C->setup_flops = fl;
  C->local_bytes = lb;
  C->apply_flops = (double)lb / (double)C->esize * 2.0;
  // FP32 contexts: one scratch buffer for the split operands of the
  // tensor-core GEMMs, shared by every list (they run one after another on
  // the setup stream)
  if (C->esize == 4) {
    // sweep updates: operands written split by the panel kernel into
    // Xp/Xlo ([rows][nb]) and Yp/Ylo ([columns][nb])
    const int nb = C->nb;
    const int ps = tc_parts(true), po = tc_parts(false);
    C->tc_parts_sweep = ps;
    C->tc_parts_other = po;
    C->Xlo.alloc(std::max<size_t>(C->Xp.bytes() / 4, 1));
    C->Ylo.alloc(std::max<size_t>(C->Yp.bytes() / 4, 1));
    if (ps == 3) {
      C->Xlo2.alloc(std::max<size_t>(C->Xp.bytes() / 4, 1));
      C->Ylo2.alloc(std::max<size_t>(C->Yp.bytes() / 4, 1));
    }
    float* xs[3] = {reinterpret_cast<float*>(C->Xp.p), C->Xlo.p, C->Xlo2.p};
    float* ys[3] = {reinterpret_cast<float*>(C->Yp.p), C->Ylo.p, C->Ylo2.p};
    const int64_t rx = (int64_t)(C->Xp.bytes() / 4) / nb, ry = (int64_t)(C->Yp.bytes() / 4) / nb;
    for (auto* v : {&C->gl_sw1, &C->gl_sw2, &C->gl_swg})
      for (auto& g : *v)
        if (rx > 0 && ry > 0) g.bind_presplit(nb, ps, xs, rx, ys, ry, P->status.p);
    if (C->DX.bytes() > 0) {
      C->DXlo.alloc(C->DX.bytes() / 4);
      C->DYlo.alloc(C->DY.bytes() / 4);
      if (ps == 3) {
        C->DXlo2.alloc(C->DX.bytes() / 4);
        C->DYlo2.alloc(C->DY.bytes() / 4);
      }
      float* dxs[3] = {reinterpret_cast<float*>(C->DX.p), C->DXlo.p, C->DXlo2.p};
      float* dys[3] = {reinterpret_cast<float*>(C->DY.p), C->DYlo.p, C->DYlo2.p};
      const int64_t dx = (int64_t)(C->DX.bytes() / 4) / nb, dy = (int64_t)(C->DY.bytes() / 4) / nb;
      for (auto& g : C->gl_swd)
        if (dx > 0 && dy > 0) g.bind_presplit(nb, ps, dxs, dx, dys, dy, P->status.p);
    }
    std::vector<GemmList*> lists{&C->gl_E, &C->gl_S, &C->gl_W, &C->gl_T, &C->gl_PhiA, &C->gl_SPhi, &C->gl_Kc,
                                 &C->gl_PsiV, &C->gl_dlx};
    for (auto* v : {&C->gl_sw1, &C->gl_sw2, &C->gl_swg, &C->gl_swd})
      for (auto& g : *v) lists.push_back(&g);
    int64_t need = 0;
    for (auto* g : lists) need = std::max(need, g->tc_floats(po));
    if (need > 0) {
      C->tc_scratch.alloc((size_t)need);
      for (auto* g : lists) g->bind_tc(C->tc_scratch.p, po, P->status.p);
    }
  }
}

// ------------------------------------------------------------------- setup
template <typename T, int NB, int NP>
static void panel_launch(dim3 grid, cudaStream_t s, const SweepDesc* desc, int k, T* mat, const T* Pbuf, T* X,
                         T* Y, T* const* lo) {
  constexpr size_t smem = panel_smem_bytes<T, NB>();
  static bool attr = false;
  if (!attr) {
    CB_CUDA(cudaFuncSetAttribute(sweep_panel_kernel<T, NB, NP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem));
    attr = true;
  }
  sweep_panel_kernel<T, NB, NP><<<grid, 256, smem, s>>>(desc, k, mat, Pbuf, X, Y, lo[0], lo[1], lo[2], lo[3]);
  CB_LAUNCH();
}

// One sweep: per pivot block the diagonal inverse, the panels and the
// rank-NB update.  FP32 lists bound to the tensor cores get their panels as
// split TF32 operands (X, Xlo, Y^T, Ylo) and skip the split pass.
// lo: the further TF32 parts of the panels {Xlo, Ylo, Xlo2, Ylo2} (FP32
// tensor-core lists; the list's part count selects how many are written).
template <typename T, int NB>
static void run_sweep_nb(const DVec<SweepDesc>& desc, int nmat, const std::vector<GemmList>& lists,
                         int maxRows, int maxCols, T* mat, T* X, T* Y, T* Pbuf, int* status, double tol,
                         cudaStream_t s, T* const* lo) {
  T* const none[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < (int)lists.size(); ++k) {
    sweep_diag_kernel<T, NB><<<nmat, DiagThreads<NB>::value, 0, s>>>(desc.p, k, mat, Pbuf, status, tol);
    CB_LAUNCH();
    dim3 grid(cdiv(std::max(maxRows, maxCols), PANEL_CH), nmat);
    const bool split = sizeof(T) == 4 && lists[k].presplit && lists[k].tc_bound && tensor_cores_for(true);
    if (split && lists[k].np == 3)
      panel_launch<T, NB, 3>(grid, s, desc.p, k, mat, Pbuf, X, Y, lo);
    else if (split)
      panel_launch<T, NB, 2>(grid, s, desc.p, k, mat, Pbuf, X, Y, lo);
    else
      panel_launch<T, NB, 0>(grid, s, desc.p, k, mat, Pbuf, X, Y, none);
    launch_list<T, false, false>(lists[k], X, Y, mat, T(-1), T(1), s);
  }
}

// Sweep with pivot blocks of nb (64, or 128 for FP32 operators).
template <typename T>
static void run_sweep(const DVec<SweepDesc>& desc, int nmat, const std::vector<GemmList>& lists,
                      int maxRows, int maxCols, T* mat, T* X, T* Y, T* Pbuf, int* status, double tol,
                      cudaStream_t s, int nb = SWEEP_NB, T* const* lo = nullptr) {
  T* const none[4] = {nullptr, nullptr, nullptr, nullptr};
  if (!lo) lo = none;
  if constexpr (sizeof(T) == 4) {
    if (nb == SWEEP_NB_MAX) {
      run_sweep_nb<T, SWEEP_NB_MAX>(desc, nmat, lists, maxRows, maxCols, mat, X, Y, Pbuf, status, tol, s, lo);
      return;
    }
  }
  run_sweep_nb<T, SWEEP_NB>(desc, nmat, lists, maxRows, maxCols, mat, X, Y, Pbuf, status, tol, s, lo);
}

template <typename T>
static void setup_impl(bddc_ctx* C, cudaStream_t s) {
  fem_problem* P = C->P;
  const int nsub = C->nsub;
  T* Aloc = reinterpret_cast<T*>(C->Aloc.p);
  T* Sw = reinterpret_cast<T*>(C->Sw.p);
  T* Phi = reinterpret_cast<T*>(C->Phi.p);
  T* SPhi = reinterpret_cast<T*>(C->SPhi.p);
  T* Y = reinterpret_cast<T*>(C->Y.p);
  T* Zf = reinterpret_cast<T*>(C->Zf.p);
  T* Wf = reinterpret_cast<T*>(C->Wf.p);
  T* G = reinterpret_cast<T*>(C->G.p);
  T* Kc = reinterpret_cast<T*>(C->Kc.p);
  T* Xp = reinterpret_cast<T*>(C->Xp.p);
  T* Yp = reinterpret_cast<T*>(C->Yp.p);
  T* Pd = reinterpret_cast<T*>(C->Pd.p);
  T* Et = reinterpret_cast<T*>(C->Et.p);
  int* status = P->status.p;
  const double tol = C->pivot_tol;
  // 1. subdomain matrices
  CB_CUDA(cudaMemsetAsync(C->Aloc.p, 0, C->Aloc.bytes(), s));
  densify_kernel<T><<<cdiv(P->n_lslots * 9, 256), 256, 0, s>>>(
      P->lslot_sub.p, P->lslot_row.p, P->lslot_col.p, P->lslot_ptr.p, P->lslot_src.p, P->contrib.p,
      P->n_lslots, C->perm.p, C->d_offN.p, C->d_offA.p, C->d_ldA.p, C->d_nI.p, Aloc);
  CB_LAUNCH();
  // 2. interior elimination: A_II^-1 by a sweep of the II block, then
  //    E = A_II^-1 A_IG and S = A_GG - A_GI E, and E stored over A_IG
  T* const lo[4] = {reinterpret_cast<T*>(C->Xlo.p), reinterpret_cast<T*>(C->Ylo.p),
                    reinterpret_cast<T*>(C->Xlo2.p), reinterpret_cast<T*>(C->Ylo2.p)};
  run_sweep<T>(C->sw1, nsub, C->gl_sw1, C->maxI, C->maxI, Aloc, Xp, Yp, Pd, status, tol, s, C->nb, lo);
  if (C->maxG == 0) return;  // one subdomain: no interface
  launch_list<T, false, false>(C->gl_E, Aloc, Aloc, Et, T(1), T(0), s);
  launch_list<T, false, false>(C->gl_S, Aloc, Et, Aloc, T(-1), T(1), s);
  if (C->sparse_cpl) {  // the apply reads the coupling blocks, not E
    if (C->steps_gi > 0) {
      coupling_values_kernel<T><<<cdiv(288 * C->steps_gi, 256), 256, 0, s>>>(
          C->sgi_src.p, C->steps_gi, P->bsr_vals.p, reinterpret_cast<T*>(C->sgi_val.p));
      CB_LAUNCH();
    }
    if (C->steps_ig > 0) {
      coupling_values_kernel<T><<<cdiv(288 * C->steps_ig, 256), 256, 0, s>>>(
          C->sig_src.p, C->steps_ig, P->bsr_vals.p, reinterpret_cast<T*>(C->sig_val.p));
      CB_LAUNCH();
    }
  } else if (C->maxI > 0) {
    copy_e_kernel<T><<<dim3(cdiv(C->maxI, 8), nsub), 256, 0, s>>>(
        C->d_nI.p, C->d_nG.p, C->d_offA.p, C->d_ldA.p, C->d_offE.p, C->d_ldS.p, Et, Aloc);
    CB_LAUNCH();
  }
  // 2b. deluxe scaling from the class blocks of the Schur complements:
  //     Shat_K = sum_b S_b inverted by a sweep, D_b = Shat_K^-1 S_b, E_b = D_b^T
  if (C->n_dlx > 0) {
    T* Dsb = reinterpret_cast<T*>(C->Dsb.p);
    T* Ddb = reinterpret_cast<T*>(C->Ddb.p);
    T* Dsh = reinterpret_cast<T*>(C->Dsh.p);
    const dim3 gb(C->n_dlx, std::min<unsigned>(cdiv((int64_t)C->maxDn * C->maxDn, 256), 64));
    const dim3 gk(C->n_dcls, gb.y);
    deluxe_gather_kernel<T><<<gb, 256, 0, s>>>(C->dlx_n.p, C->dlx_sub.p, C->dlx_ld.p, C->dlx_poff.p,
                                                     C->dlx_pos.p, C->dlx_off.p, C->d_nI.p, C->d_offA.p,
                                                     C->d_ldA.p, Aloc, Dsb);
    CB_LAUNCH();
    deluxe_sum_kernel<T><<<gk, 256, 0, s>>>(C->dcls_ptr.p, C->dcls_blk.p, C->dlx_n.p, C->dlx_ld.p,
                                                   C->dlx_off.p, C->dcls_off.p, Dsb, Dsh);
    CB_LAUNCH();
    T* const dlo[4] = {reinterpret_cast<T*>(C->DXlo.p), reinterpret_cast<T*>(C->DYlo.p),
                       reinterpret_cast<T*>(C->DXlo2.p), reinterpret_cast<T*>(C->DYlo2.p)};
    run_sweep<T>(C->swd, C->n_dcls, C->gl_swd, C->maxDn, C->maxDn, Dsh, reinterpret_cast<T*>(C->DX.p),
                 reinterpret_cast<T*>(C->DY.p), reinterpret_cast<T*>(C->DP.p), status, tol, s, C->nb, dlo);
    launch_list<T, false, false>(C->gl_dlx, Dsh, Dsb, Ddb, T(1), T(0), s);
    deluxe_transpose_kernel<T><<<gb, 256, 0, s>>>(C->dlx_n.p, C->dlx_ld.p, C->dlx_off.p, Ddb,
                                                        reinterpret_cast<T*>(C->Deb.p));
    CB_LAUNCH();
  }
  // 3. Schur complement copy, augmentation and sweep over Gamma_r
  copy_schur_kernel<T><<<dim3(cdiv(C->maxG, 8), nsub), 256, 0, s>>>(
      C->d_nI.p, C->d_nG.p, C->d_offA.p, C->d_ldA.p, C->d_offS.p, C->d_ldS.p, Aloc, Sw);
  CB_LAUNCH();
  if (C->maxA > 0) {
    augment_kernel<T><<<nsub, 256, 0, s>>>(C->d_nr.p, C->d_na.p, C->d_offCon.p, C->cons_ptr.p,
                                          C->cons_idx.p, C->cons_w.p, C->d_offS.p, C->d_ldS.p, Sw);
    CB_LAUNCH();
  }
  run_sweep<T>(C->sw2, nsub, C->gl_sw2, C->maxG, C->maxG, Sw, Xp, Yp, Pd, status, tol, s, C->nb, lo);
  // 4. average constraints
  if (C->maxA > 0) {
    cons_y_kernel<T><<<dim3(cdiv(C->maxR, 8), nsub), 256, 0, s>>>(
        C->d_nr.p, C->d_na.p, C->d_offCon.p, C->cons_ptr.p, C->cons_idx.p, C->cons_w.p, C->d_offS.p,
        C->d_ldS.p, C->d_offY.p, C->d_ldY.p, Sw, Y);
    CB_LAUNCH();
    cons_z_kernel<T><<<dim3(cdiv(C->maxG, 128), nsub), 128, 0, s>>>(
        C->d_nG.p, C->d_na.p, C->d_offCon.p, C->cons_ptr.p, C->cons_idx.p, C->cons_w.p, C->d_offS.p,
        C->d_ldS.p, C->d_offZ.p, Sw, Zf);
    CB_LAUNCH();
    cons_g_kernel<T><<<dim3(cdiv(C->maxA * C->maxA, 256), nsub), 256, 0, s>>>(
        C->d_na.p, C->d_offCon.p, C->cons_ptr.p, C->cons_idx.p, C->cons_w.p, C->d_offY.p, C->d_ldY.p,
        C->d_offG.p, C->d_ldG.p, Y, G);
    CB_LAUNCH();
    run_sweep<T>(C->swg, nsub, C->gl_swg, C->maxA, C->maxA, G, Xp, Yp, Pd, status, tol, s, C->nb, lo);
    launch_list<T, false, false>(C->gl_W, G, Zf, Wf, T(1), T(0), s);
    launch_list<T, false, false>(C->gl_T, Y, Wf, Sw, T(-1), T(1), s);
    launch_list<T, false, false>(C->gl_PhiA, Y, G, Phi, T(1), T(0), s);
  }
  // 5. vertex columns of Phi and the identity block (no primal constraint
  //    anywhere: Phi has no columns)
  if (C->maxC > 0) {
    phi_vertex_kernel<T><<<dim3(cdiv((int64_t)C->maxG * C->maxC, 256), nsub), 256, 0, s>>>(
        C->d_nG.p, C->d_nr.p, C->d_nv.p, C->d_nc.p, C->d_offS.p, C->d_ldS.p, C->d_offPhi.p, C->d_ldPhi.p,
        Sw, Phi);
    CB_LAUNCH();
  }
  // 5b. Petrov coarse space: the left basis Psi
  T* Psi = reinterpret_cast<T*>(C->Psi.p);
  if (C->coarse == CBDDC_COARSE_PETROV && C->maxC > 0) {
    psi_fill_kernel<T><<<dim3(cdiv((int64_t)C->maxG * C->maxC, 256), nsub), 256, 0, s>>>(
        C->d_nG.p, C->d_nr.p, C->d_nv.p, C->d_nc.p, C->d_offZ.p, C->d_ldS.p, C->d_offPhi.p, C->d_ldPhi.p,
        Wf, Psi);
    CB_LAUNCH();
    launch_list<T, true, true>(C->gl_PsiV, Sw, Aloc, Psi, T(-1), T(0), s);
  }
  // 6. local coarse matrices Psi^T S Phi (Psi = Phi: Galerkin) and the FP64
  //    coarse inverse
  if (C->n_pi > 0) {
    launch_list<T, false, false>(C->gl_SPhi, Aloc, Phi, SPhi, T(1), T(0), s);
    launch_list<T, true, false>(C->gl_Kc, C->coarse == CBDDC_COARSE_PETROV ? Psi : Phi, SPhi, Kc, T(1),
                                T(0), s);
    if (C->next) {
      // multilevel: the local coarse matrices become the element matrices of
      // the coarse problem, which the level-2 BDDC sets up in FP64
      fem_problem* CP = C->coarse_prob.get();
      kc_to_blocks_kernel<T><<<dim3(cdiv((int64_t)C->maxC * C->maxC, 256), nsub), 256, 0, s>>>(
          C->d_nc.p, C->d_offKc.p, C->d_ldPhi.p, C->d_cbase.p, Kc, CP->contrib.p);
      CB_LAUNCH();
      timer_begin(CBDDC_TIMER_LEVEL2_SETUP, s);
      bddc_run_setup(C->next.get(), s);
      timer_end(CBDDC_TIMER_LEVEL2_SETUP, s, C->next->setup_flops, 0.0);
      or_status_kernel<<<1, 1, 0, s>>>(CP->status.p, status);
      CB_LAUNCH();
      return;
    }
    timer_begin(CBDDC_TIMER_COARSE_SETUP, s);
    CB_CUDA(cudaMemsetAsync(C->Sc.p, 0, C->Sc.bytes(), s));
    if (sizeof(T) == 4)
      coarse_assemble_kernel_f<<<cdiv(C->n_ce, 256), 256, 0, s>>>(
          C->ce_key.p, C->ce_ptr.p, C->ce_src.p, C->n_ce, reinterpret_cast<const float*>(Kc), C->Sc.p);
    else
      coarse_assemble_kernel_d<<<cdiv(C->n_ce, 256), 256, 0, s>>>(
          C->ce_key.p, C->ce_ptr.p, C->ce_src.p, C->n_ce, reinterpret_cast<const double*>(Kc), C->Sc.p);
    CB_LAUNCH();
    run_sweep<double>(C->swc, 1, C->gl_swc, C->n_pi, C->n_pi, C->Sc.p, C->ScX.p, C->ScY.p, C->ScP.p,
                      status, tol, s);
    timer_end(CBDDC_TIMER_COARSE_SETUP, s, 2.0 * (double)C->n_pi * C->n_pi * C->n_pi, 0.0);
  }
}

void bddc_run_setup(bddc_ctx* C, cudaStream_t s) {
  timer_begin(CBDDC_TIMER_SETUP, s);
  if (C->precision == CBDDC_FP32) setup_impl<float>(C, s);
  else setup_impl<double>(C, s);
  timer_end(CBDDC_TIMER_SETUP, s, C->setup_flops, 0.0);
}

// ------------------------------------------------------------------- apply
namespace {

struct ApplyWork {
  double *u0, *hG, *gI, *gl, *wG, *cl, *rc, *uc, *yG, *xI, *zl, *yD;
  void *uq, *zq;  // node-packed coupling inputs (operator precision)
};

void apply_untimed(bddc_ctx* C, const double* r, double* z, cudaStream_t s);

// z = M^-1 r with caller-chosen work vectors (the context's own, or the
// static array of bddc_apply_noalloc).
template <typename T>
void apply_with_work(bddc_ctx* C, const double* r, double* z, const ApplyWork& w, cudaStream_t s) {
  const T* Aloc = reinterpret_cast<const T*>(C->Aloc.p);
  const T* Sw = reinterpret_cast<const T*>(C->Sw.p);
  const T* Phi = reinterpret_cast<const T*>(C->Phi.p);
  const T* Psi = reinterpret_cast<const T*>(C->Psi.p);
  const size_t smI = (size_t)round_up(std::max(C->maxI, 4), 4) * sizeof(T);
  const size_t smD = (size_t)round_up(std::max(C->maxDn, 4), 4) * sizeof(T);
  gather_kernel<<<cdiv(std::max<int64_t>(C->totI, 1), 256), 256, 0, s>>>(C->gdofI.p, C->totI, r, w.xI);
  CB_LAUNCH();
  if (C->n_itI > 0) {
    apply_interior_kernel<T, false><<<C->n_itI, 256, smI, s>>>(
        C->itI.p, C->d_nI.p, C->d_offA.p, C->d_ldA.p, C->d_offI.p, C->gdofI.p, Aloc, w.xI, w.u0,
        C->sparse_cpl ? static_cast<T*>(w.uq) : nullptr);
    CB_LAUNCH();
  }
  if (C->maxG > 0 && !C->sparse_cpl) {
    if (C->n_itG > 0) {
      apply_gi_kernel<T><<<C->n_itG, 256, smI, s>>>(
          C->itG.p, C->d_nI.p, C->d_nG.p, C->d_offA.p, C->d_ldA.p, C->d_offI.p, C->d_offGam.p, Aloc, w.u0, w.hG);
      CB_LAUNCH();
    }
  }
  if (C->n_if > 0) {
    if (C->sparse_cpl) {  // g = r_Gamma - K_Gamma,I u0
      coupling_kernel<T><<<cdiv((int64_t)C->n_sgi * 32, 256), 256, 0, s>>>(
          C->sgi_off.p, C->sgi_len.p, C->sgi_row.p, C->sgi_col.p, reinterpret_cast<const T*>(C->sgi_val.p),
          static_cast<const typename Q4<T>::type*>(w.uq), C->if_dof.p, r, w.gI, C->n_sgi);
    } else {
      assemble_g_kernel<<<cdiv(C->n_if, 256), 256, 0, s>>>(C->if_dof.p, C->if_ptr.p, C->if_src.p, C->n_if,
                                                          r, w.hG, w.gI);
    }
    CB_LAUNCH();
    restrict_kernel<<<cdiv(C->totG, 256), 256, 0, s>>>(C->gam_if.p, C->Dg.p, C->totG, w.gI, w.gl);
    CB_LAUNCH();
    if (C->n_dlx > 0) {  // deluxe: g_i = D_b^T g on each class
      deluxe_apply_kernel<T, true><<<dim3(C->n_dlx, cdiv(C->maxDn, DLX_COLS)), DLX_COLS * DLX_RG, smD, s>>>(
          C->dlx_n.p, C->dlx_sub.p, C->dlx_ld.p, C->dlx_poff.p, C->dlx_pos.p, C->dlx_off.p, C->d_offGam.p,
          C->gam_if.p, reinterpret_cast<const T*>(C->Ddb.p), w.gI, w.gl);
      CB_LAUNCH();
    }
    if (C->n_itG > 0) {
      apply_local_kernel<T><<<C->n_itG, 256,
                              (size_t)round_up(std::max(C->maxR, 4), 4) * sizeof(T), s>>>(
          C->itG.p, C->d_nG.p, C->d_nr.p, C->d_offS.p, C->d_ldS.p, C->d_offGam.p, Sw, w.gl, w.wG);
      CB_LAUNCH();
    }
    if (C->n_pi > 0) {
      const int nch = (int)cdiv(C->maxG, PHIT_ROWS);
      if (C->n_itP > 0) {
        apply_phit_kernel<T><<<C->n_itP, 256, 0, s>>>(C->itP.p, C->d_nG.p, C->d_nc.p, C->d_offPhi.p,
                                                            C->d_ldPhi.p, C->d_offGam.p, C->d_offC.p,
                                                            C->coarse == CBDDC_COARSE_PETROV ? Psi : Phi,
                                                            w.gl, w.cl, nch);
        CB_LAUNCH();
      }
      coarse_rhs_kernel<<<cdiv(C->n_pi, 256), 256, 0, s>>>(C->cg_ptr.p, C->cg_src.p, C->n_pi, w.cl, nch,
                                                           C->cnch.p, w.rc);
      CB_LAUNCH();
      if (C->next) {
        // the level-2 context uses its own work vectors, allocated at setup;
        // its apply is not timed on its own (an enclosing bddc_run_apply
        // times the whole recursion, and bddc_apply_noalloc times nothing)
        timer_begin(CBDDC_TIMER_LEVEL2_APPLY, s);
        apply_untimed(C->next.get(), w.rc, w.uc, s);
        timer_end(CBDDC_TIMER_LEVEL2_APPLY, s, C->next->apply_flops, (double)C->next->local_bytes);
      } else {
        timer_begin(CBDDC_TIMER_COARSE_APPLY, s);
        dense_gemv_kernel<<<cdiv((int64_t)C->n_pi * 32, 256), 256, 0, s>>>(C->Sc.p, C->n_pi, w.rc, w.uc);
        CB_LAUNCH();
        timer_end(CBDDC_TIMER_COARSE_APPLY, s, 2.0 * (double)C->n_pi * C->n_pi,
                  8.0 * (double)C->n_pi * C->n_pi);
      }
    }
    if (C->n_itR > 0) {
      apply_prolong_kernel<T><<<C->n_itR, 256, 0, s>>>(
          C->itR.p, C->d_nG.p, C->d_nc.p, C->d_offPhi.p, C->d_ldPhi.p, C->d_offGam.p, C->d_offC.p, C->gprim.p, Phi,
          w.uc, w.wG, C->Dg.p, w.yG);
      CB_LAUNCH();
    }
    const double* yavg = w.yG;
    if (C->n_dlx > 0) {  // deluxe: the class part of y_i becomes D_b y_i
      CB_CUDA(cudaMemcpyAsync(w.yD, w.yG, (size_t)C->totG * sizeof(double), cudaMemcpyDeviceToDevice, s));
      deluxe_apply_kernel<T, false><<<dim3(C->n_dlx, cdiv(C->maxDn, DLX_COLS)), DLX_COLS * DLX_RG, smD, s>>>(
          C->dlx_n.p, C->dlx_sub.p, C->dlx_ld.p, C->dlx_poff.p, C->dlx_pos.p, C->dlx_off.p, C->d_offGam.p,
          C->gam_if.p, reinterpret_cast<const T*>(C->Deb.p), w.yG, w.yD);
      CB_LAUNCH();
      yavg = w.yD;
    }
    average_kernel<T><<<cdiv(C->n_if, 256), 256, 0, s>>>(C->if_dof.p, C->if_ptr.p, C->if_src.p, C->n_if,
                                                        yavg, z, w.zl,
                                                        C->sparse_cpl ? static_cast<T*>(w.zq) : nullptr);
    CB_LAUNCH();
  }
  if (C->sparse_cpl) {
    // z_I = A_II^-1 (r_I - K_I,Gamma z): the coupling overwrites the
    // gathered r_I (no longer needed) with its right-hand side
    coupling_kernel<T><<<cdiv((int64_t)C->n_sig * 32, 256), 256, 0, s>>>(
        C->sig_off.p, C->sig_len.p, C->sig_row.p, C->sig_col.p, reinterpret_cast<const T*>(C->sig_val.p),
        static_cast<const typename Q4<T>::type*>(w.zq), C->gdofI.p, r, w.xI, C->n_sig);
    CB_LAUNCH();
    apply_interior_kernel<T, true><<<C->n_itI, 256, smI, s>>>(
        C->itI.p, C->d_nI.p, C->d_offA.p, C->d_ldA.p, C->d_offI.p, C->gdofI.p, Aloc, w.xI, z, nullptr);
    CB_LAUNCH();
  } else if (C->n_itI > 0) {
    apply_extend_kernel<T><<<C->n_itI, 256,
                             (size_t)round_up(std::max(C->maxG, 4), 4) * sizeof(T), s>>>(
        C->itI.p, C->d_nI.p, C->d_nG.p, C->d_offA.p, C->d_ldA.p, C->d_offI.p, C->d_offGam.p, C->gdofI.p,
        Aloc, w.zl, w.u0, z);
    CB_LAUNCH();
  }
}

template <typename T>
void apply_impl(bddc_ctx* C, const double* r, double* z, cudaStream_t s) {
  ApplyWork w{C->u0.p, C->hG.p, C->gI.p, C->gl.p, C->wG.p, C->cl.p, C->rc.p,
              C->uc.p, C->yG.p, C->xI.p, C->zl.p, C->yD.p, C->uq.p, C->zq.p};
  apply_with_work<T>(C, r, z, w, s);
}

// The apply with the context's own work vectors, outside the kernel timer.
void apply_untimed(bddc_ctx* C, const double* r, double* z, cudaStream_t s) {
  if (C->precision == CBDDC_FP32) apply_impl<float>(C, r, z, s);
  else apply_impl<double>(C, r, z, s);
}

}  // namespace

void bddc_run_apply(bddc_ctx* C, const double* r, double* z, cudaStream_t s) {
  timer_begin(CBDDC_TIMER_APPLY, s);
  apply_untimed(C, r, z, s);
  timer_end(CBDDC_TIMER_APPLY, s, C->apply_flops, (double)C->local_bytes);
}

// ------------------------------------------------ apply without allocation
// Work vectors of bddc_apply_noalloc.  They live in one file-scope device
// array that every device loading the library holds until the process
// exits, so that the call itself never needs cudaMalloc.  4 MiB holds the
// per-apply vectors of problems up to roughly 10^5 DoFs split into up to a
// few hundred subdomains (the 48x48x12 slab needs about 3.1 MiB).
constexpr int64_t kNoAllocScratchDoubles = 524288;  // 4 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the array's name is only a host-side stand-in, so kernels must get
// this address instead.
double* noalloc_scratch_address() {
  static std::mutex mu;
  static std::map<int, double*> cache;
  int dev = -1;
  CB_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  void* ptr = nullptr;
  CB_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
  CB_CHECK(ptr != nullptr, CBDDC_ECUDA, "cudaGetSymbolAddress returned a null address");
  cache[dev] = static_cast<double*>(ptr);
  return static_cast<double*>(ptr);
}

}  // namespace

int64_t bddc_noalloc_scratch_needed(const bddc_ctx* C) {
  auto pad = [](int64_t n) { return round_up(std::max<int64_t>(n, 1), 32); };
  const int64_t nch = cdiv(std::max(C->maxG, 1), PHIT_ROWS);
  // node-packed coupling inputs: 4 values of esize bytes per node
  const int64_t q = C->sparse_cpl ? pad((C->totI / 3) * 4 * (int64_t)C->esize / 8) +
                                        pad((C->n_if / 3) * 4 * (int64_t)C->esize / 8)
                                  : 0;
  return 2 * pad(C->totI) + (C->n_dlx > 0 ? 6 : 5) * pad(C->totG) + pad(C->n_if) + pad(C->totC * nch) +
         2 * pad(C->n_pi) + q;
}

int64_t bddc_noalloc_scratch_capacity() { return kNoAllocScratchDoubles; }

void bddc_run_apply_noalloc(bddc_ctx* C, const double* r, double* z, cudaStream_t s) {
  const int64_t need = bddc_noalloc_scratch_needed(C);
  CB_CHECK(need <= kNoAllocScratchDoubles, CBDDC_EINVAL,
           "bddc_apply_noalloc: this context needs " + std::to_string(need) +
               " doubles of work space, the static buffer holds " +
               std::to_string(kNoAllocScratchDoubles) + "; use bddc_apply");
  double* base = noalloc_scratch_address();
  auto pad = [](int64_t n) { return round_up(std::max<int64_t>(n, 1), 32); };
  ApplyWork w;
  double* p = base;
  w.u0 = p; p += pad(C->totI);
  w.xI = p; p += pad(C->totI);
  w.zl = p; p += pad(C->totG);
  w.hG = p; p += pad(C->totG);
  w.gl = p; p += pad(C->totG);
  w.wG = p; p += pad(C->totG);
  w.yG = p; p += pad(C->totG);
  w.gI = p; p += pad(C->n_if);
  w.cl = p; p += pad(C->totC * (int64_t)cdiv(std::max(C->maxG, 1), PHIT_ROWS));
  w.rc = p; p += pad(C->n_pi);
  w.uc = p; p += pad(C->n_pi);
  w.yD = nullptr;
  if (C->n_dlx > 0) { w.yD = p; p += pad(C->totG); }
  w.uq = w.zq = nullptr;
  if (C->sparse_cpl) {
    w.uq = p; p += pad((C->totI / 3) * 4 * (int64_t)C->esize / 8);
    w.zq = p; p += pad((C->n_if / 3) * 4 * (int64_t)C->esize / 8);
  }
  if (C->precision == CBDDC_FP32) apply_with_work<float>(C, r, z, w, s);
  else apply_with_work<double>(C, r, z, w, s);
}

}  // namespace cbddc

int64_t bddc_ctx::device_bytes() const {
  return (int64_t)(Aloc.bytes() + Sw.bytes() + Phi.bytes() + Y.bytes() + Zf.bytes() + Wf.bytes() +
                   G.bytes() + SPhi.bytes() + Kc.bytes() + Xp.bytes() + Yp.bytes() + Pd.bytes() + Et.bytes() +
                   Sc.bytes() + ScX.bytes() + ScY.bytes() + ScP.bytes() + u0.bytes() + hG.bytes() +
                   gI.bytes() + wG.bytes() + cl.bytes() + rc.bytes() + uc.bytes() + yG.bytes() + gl.bytes() + xI.bytes() + zl.bytes() +
                   Dsb.bytes() + Ddb.bytes() + Deb.bytes() + Dsh.bytes() + DX.bytes() + DY.bytes() + DP.bytes() +
                   yD.bytes() + Psi.bytes() + sgi_off.bytes() + sgi_len.bytes() + sgi_row.bytes() +
                   sgi_col.bytes() + sgi_src.bytes() + sgi_val.bytes() + sig_off.bytes() + sig_len.bytes() +
                   sig_row.bytes() + sig_col.bytes() + sig_src.bytes() + sig_val.bytes() + uq.bytes() +
                   zq.bytes()) +
         (next ? next->device_bytes() + coarse_prob->device_bytes() : 0);
}
