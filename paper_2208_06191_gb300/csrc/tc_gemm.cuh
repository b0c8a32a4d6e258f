// Grouped FP32 GEMM on the fifth-generation tensor cores (tcgen05,
// kind::tf32), for the dense contractions of the BDDC setup (the Gauss-Jordan
// sweep updates, E = A_II^-1 A_IG, S = A_GG - A_GI E, the constraint and
// coarse-basis products of Section 3.2).
//
// Precision: a TF32 operand keeps 10 mantissa bits, too few for explicit
// inverses of local matrices whose condition numbers reach 1e4.  Every
// operand x is therefore split into TF32 parts and the product accumulated
// in FP32 over the significant part products:
//   NP = 2: x = x1 + x2 + O(2^-22 x), x1 = tf32(x), x2 = tf32(x - x1);
//           A B ~ A1 B1 + A1 B2 + A2 B1 (three passes, about 2^-21 relative);
//   NP = 3: x = x1 + x2 + x3 exactly (x3 = x - x1 - x2 has at most a few
//           significant bits); A B ~ A1 B1 + A1 B2 + A2 B1 + A1 B3 + A3 B1
//           + A2 B2 (six passes; the dropped products are 2^-33 relative,
//           FP32-level results).
// The Gauss-Jordan sweeps need NP = 3 to keep the FP32 path's GMRES
// iterations within two of the FP64 path's.
//
// Data flow of C = alpha op(A) op(B) + beta C for a list of problems:
//   1. split kernels write op(A) (M x K) and op(B)^T (N x K) as K-major
//      hi/lo arrays into a scratch buffer, one row range per problem, K
//      zero-padded to a multiple of 32;
//   2. one CTA per 128 x 128 output tile: a TMA producer thread streams
//      K chunks of 32 (one 128-byte swizzled row per tile row; A_hi, A_lo,
//      B_hi, B_lo = 64 KB per stage, 2 stages) into shared memory; one
//      thread issues 3 x 4 tcgen05.mma (M = N = 128, K = 8) per chunk into a
//      128-column TMEM accumulator and frees the stage with tcgen05.commit;
//      meanwhile (beta != 0) the four warps copy the C tile into shared
//      memory with 16-byte asynchronous copies, so its DRAM latency hides
//      behind the operand loads and the MMAs; after the last chunk each
//      warp reads its 32 TMEM lanes (tcgen05.ld), combines them with the
//      staged C rows, and writes its rows back with warp-wide 512-byte
//      stores.  The rank-64 sweep updates are bound by this C traffic.
// Rows past a problem's M (or N) read other problems' rows or the
// zero fill beyond the array; they only reach accumulator rows (columns)
// that are never stored.
//
// Every wait on an mbarrier is bounded; on expiry the kernel sets DEV_TIMEOUT
// in the status word, waits (bounded) for the copies it issued, frees its
// TMEM and returns.
#pragma once
#include <cuda.h>
#include <stdint.h>

#include <algorithm>

#include "common.h"

namespace cbddc {
namespace tc {

constexpr int BM = 128, BN = 128;             // output tile
constexpr int BKC = 32;                       // K per chunk: 32 x 4 B = one 128-byte swizzle row
constexpr int OPND_BYTES = BM * BKC * 4;      // one operand tile of a chunk (16 KB)
// operand tiles per stage: NP parts of A and NP parts of B (NP = 2: hi, lo;
// NP = 3: three-way split)
template <int NP>
struct TcStage { static constexpr int bytes = 2 * NP * OPND_BYTES; };
constexpr int TC_THREADS = 320;               // GEMM: producer, MMA and eight epilogue warps
constexpr int TMEM_COLS = 128;                // one accumulator slice; the kernel holds two
constexpr int CLD = BN;                       // row pitch (floats) of the C tile in shared memory
constexpr int C_BYTES = BM * CLD * 4;         // 64 KB; 16-byte chunk q of row r sits at q ^ (r % 8)
constexpr uint32_t kWaitLimit = 1u << 25;     // polls of one mbarrier before giving up

// Instruction descriptor of kind::tf32: D = F32 (bits 4-5 = 1), A = B = TF32
// (bits 7-9 and 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(BN >> 3) << 17) |
                            ((uint32_t)(BM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor of a K-major operand in the 128-byte
// swizzled layout that TMA writes: rows of 128 B, 8-row atoms of 1 KB
// stacked along M/N (stride byte offset 1024), descriptor version 1
// (bits 46-47), layout type 2 = 128-byte swizzle (bits 61-63).  The leading
// byte offset is unused for this layout.  Advancing K by 8 TF32 elements
// inside the atom adds 32 bytes to the start address.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Bounded wait for the phase with the given parity; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

// Arrives on bar once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 consecutive TMEM columns of this warp's 32 lanes (one row per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// TF32 rounding (round to nearest, ties away from zero); the low 13
// mantissa bits of the result are zero.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

// x as NP TF32 parts, largest first: NP = 2 rounds twice (x - x1 - x2 is
// about 2^-22 x); NP = 3 leaves no remainder.
template <int NP>
__device__ __forceinline__ void split_tf32(float x, float* p) {
  const float x1 = tf32_round(x);
  const float r = x - x1;  // exact
  const float x2 = tf32_round(r);
  p[0] = x1;
  p[1] = x2;
  if (NP == 3) p[2] = r - x2;  // exact, a few significant bits
}

// Problem of a tensor-core list: sizes, C placement and the first rows of
// its operands in the split arrays.
struct TcProb {
  int M, N, K, ldc;
  int64_t c;
  int ar, br;
};

// Shared-memory footprint of the persistent kernel with NST operand stages
// and NCB C-tile buffers.
template <int NST, int NCB, int NP>
struct TcSmem {
  static constexpr int bytes = NST * TcStage<NP>::bytes + NCB * C_BYTES + 1024 /* alignment */ + 256 /* barriers */;
  static_assert(bytes <= 232448, "shared memory per CTA");
};

// TMA maps of the split operands: parts of op(A) and of op(B)^T.
struct TcMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};

// Persistent grouped GEMM: CTA b takes the tiles b, b + gridDim.x, ... of the
// list ({problem, tile row, tile column}), each C = alpha A B + beta C.
//
// Accumulation: the tensor cores add into TMEM with truncation (measured:
// errors all of one sign on positive data, 5-20x those of FP32 FMAs), and
// the Gauss-Jordan sweeps compound such a bias over their passes.  So every
// KS K-steps of 8 are accumulated on their own in one of two 128-column
// TMEM slices, and the slice sums are added on the CUDA cores in FP32 with
// round-to-nearest (registers of the epilogue threads); the truncated sums
// then span 8 KS products instead of the whole K (KS = 4, one K chunk, for
// long products; KS = 1 for the rank-NB sweep updates).
//
// Warp roles (320 threads):
//   warp 0, one lane: TMA producer of the operand chunks (NST-stage ring);
//   warp 1, one lane: MMA issuer; chunk g of the CTA goes to TMEM slice g % 2;
//   warps 2-9: epilogue; warp w reads TMEM lanes (tile rows) 32 (w % 4) ..
//     + 31 and column half (w - 2) / 4 (64 columns), adds every chunk's
//     slice into 64 FP32 running sums per thread and frees the slice; at the
//     end of a tile it combines them with C, staged in shared memory by
//     16-byte asynchronous copies (the next tile's C rows are copied while
//     this tile's chunks are summed when NCB = 2), and writes its rows back
//     with coalesced 256-byte half-row stores.
// Barriers: full/empty per operand stage, sfull/sempty per TMEM slice
// (sempty counts the eight epilogue warps).
template <int NST, int NCB, int NP, int KS>
__global__ void __launch_bounds__(TC_THREADS, 1)
tc_gemm_kernel(const int4* __restrict__ tiles, int ntiles, const TcProb* __restrict__ probs,
               const __grid_constant__ TcMaps maps, float* __restrict__ C, float alpha, float beta,
               int* __restrict__ status) {
  constexpr int STAGE_BYTES = TcStage<NP>::bytes;
  constexpr int SPC = (BKC / 8) / KS;  // TMEM slices per K chunk (KS K-steps of 8 each)
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte aligned operand stages (the swizzle pattern repeats every 1 KB)
  const uint32_t base = smem_u32(smem_raw);
  uint8_t* smem = smem_raw + ((1024u - (base & 1023u)) & 1023u);
  float* Cbuf = reinterpret_cast<float*>(smem + NST * STAGE_BYTES);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * STAGE_BYTES + NCB * C_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* sfull = empty + NST;
  uint64_t* sempty = sfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ntl = ntiles > (int)blockIdx.x ? (ntiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&sfull[a], 1);
      mbar_init(&sempty[a], 8);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  int issued = 0;  // operand chunks whose copies the producer issued
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      for (int i = 0; i < ntl && !*(volatile int*)abort_flag; ++i) {
        const int4 tl = tiles[blockIdx.x + i * gridDim.x];
        const TcProb p = probs[tl.x];
        const int nk = (p.K + BKC - 1) / BKC;
        const int ya = p.ar + tl.y * BM, yb = p.br + tl.z * BN;
        for (int c = 0; c < nk; ++c, ++g) {
          const int s = g % NST;
          if (g >= NST && !mbar_wait(&empty[s], ((g / NST) - 1) & 1)) {
            atomicExch(abort_flag, 1);
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            tma_load_2d(st + q * OPND_BYTES, &maps.a[q], c * BKC, ya, &full[s]);
            tma_load_2d(st + (NP + q) * OPND_BYTES, &maps.b[q], c * BKC, yb, &full[s]);
          }
          issued = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int g = 0;  // TMEM slices of this CTA so far (SPC per operand chunk)
      bool ok = true;
      for (int i = 0; i < ntl && ok && !*(volatile int*)abort_flag; ++i) {
        const int4 tl = tiles[blockIdx.x + i * gridDim.x];
        const int nk = (probs[tl.x].K + BKC - 1) / BKC;
        for (int c = 0; c < nk; ++c) {
          const int s = (g / SPC) % NST;  // operand stage of chunk c (g counts slices)
          if (!mbar_wait(&full[s], ((g / SPC) / NST) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t st = smem_u32(smem + s * STAGE_BYTES);
          for (int sl = 0; sl < SPC && ok; ++sl, ++g) {
            const int a = g & 1;
            if (g >= 2 && !mbar_wait(&sempty[a], ((g >> 1) - 1) & 1)) {
              ok = false;
              break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(a * TMEM_COLS);
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
              const int k = sl * KS + kk;
              // parts: a_q at tile q, b_q at tile NP + q; small products first
              auto da = [&](int q) { return sw128_desc(st + q * OPND_BYTES + 32 * k); };
              auto db = [&](int q) { return sw128_desc(st + (NP + q) * OPND_BYTES + 32 * k); };
              const uint32_t first = kk > 0 ? 1u : 0u;  // each slice starts afresh
              if (NP == 3) {
                mma_tf32(acc, da(1), db(1), first);
                mma_tf32(acc, da(2), db(0), 1u);
                mma_tf32(acc, da(0), db(2), 1u);
                mma_tf32(acc, da(1), db(0), 1u);
              } else {
                mma_tf32(acc, da(1), db(0), first);
              }
              mma_tf32(acc, da(0), db(1), 1u);
              mma_tf32(acc, da(0), db(0), 1u);
            }
            mma_commit(&sfull[a]);
          }
          if (!ok) break;
          mma_commit(&empty[s]);
        }
        if (!ok) break;
      }
      if (!ok) atomicExch(abort_flag, 1);
    }
  } else {
    // epilogue warps
    const int wq = warp & 3, half = (warp - 2) >> 2;
    const int wrow0 = 32 * wq, col0 = 64 * half;
    // C rows of a tile into buffer (i % NCB): 32 rows x 64 columns, two rows
    // per warp instruction (16 lanes x 16 bytes each)
    auto prefetch = [&](int i) {
      const int4 tl = tiles[blockIdx.x + i * gridDim.x];
      const TcProb p = probs[tl.x];
      if (beta == 0.f || (p.c & 3) || (p.ldc & 3)) return;
      float* Cs = Cbuf + (i % NCB) * (BM * CLD);
      const int m0 = tl.y * BM, n0 = tl.z * BN;
      const int sub = lane >> 4, q = (col0 >> 2) + (lane & 15);  // 16-byte chunk of the row
      for (int r = 0; r < 32; r += 2) {
        const int lr = wrow0 + r + sub, gr = m0 + lr, gc = n0 + 4 * q;
        const int valid = (gr < p.M) ? max(0, min(4, p.N - gc)) : 0;
        const float* src = valid > 0 ? C + p.c + (int64_t)gr * p.ldc + gc : C;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(
                         smem_u32(Cs + lr * CLD + 4 * (q ^ (lr & 7)))),
                     "l"(src), "r"(valid * 4)
                     : "memory");
      }
    };
    if (ntl > 0) prefetch(0);
    asm volatile("cp.async.commit_group;" ::: "memory");
    int g = 0;
    bool ok = true;
    for (int i = 0; i < ntl && ok; ++i) {
      const int4 tl = tiles[blockIdx.x + i * gridDim.x];
      const TcProb p = probs[tl.x];
      const int m0 = tl.y * BM, n0 = tl.z * BN;
      const int nk = (p.K + BKC - 1) / BKC;
      const bool ahead = NCB == 2 && i + 1 < ntl;
      if (ahead) {
        prefetch(i + 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
      float rs[64];
#pragma unroll
      for (int q = 0; q < 64; ++q) rs[q] = 0.f;
      for (int c = 0; c < nk * SPC; ++c, ++g) {
        const int a = g & 1;
        if (!mbar_wait(&sfull[a], (g >> 1) & 1) || *(volatile int*)abort_flag) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + (uint32_t)(a * TMEM_COLS) + ((uint32_t)wrow0 << 16) + (uint32_t)col0;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float v[32];
          tmem_ld32(acc + (uint32_t)(32 * h), v);
#pragma unroll
          for (int q = 0; q < 32; ++q) rs[32 * h + q] += v[q];
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncwarp();
        if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&sempty[a])) : "memory");
      }
      if (!ok) {
        atomicExch(abort_flag, 1);
        break;
      }
      if (ahead) asm volatile("cp.async.wait_group 1;" ::: "memory");
      else asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncwarp();
      const int lr = wrow0 + lane;
      const bool cvec = ((p.c & 3) == 0) && ((p.ldc & 3) == 0);
      float* Cs = Cbuf + (i % NCB) * (BM * CLD);
      if (cvec) {
        float4* c4 = reinterpret_cast<float4*>(Cs + lr * CLD);
#pragma unroll
        for (int qq = 0; qq < 16; ++qq) {
          const int q = ((col0 >> 2) + qq) ^ (lr & 7);  // swizzled 16-byte chunk of this row
          float4 o;
          if (beta != 0.f) {
            const float4 old = c4[q];
            o = make_float4(alpha * rs[4 * qq] + beta * old.x, alpha * rs[4 * qq + 1] + beta * old.y,
                            alpha * rs[4 * qq + 2] + beta * old.z, alpha * rs[4 * qq + 3] + beta * old.w);
          } else {
            o = make_float4(alpha * rs[4 * qq], alpha * rs[4 * qq + 1], alpha * rs[4 * qq + 2],
                            alpha * rs[4 * qq + 3]);
          }
          c4[q] = o;
        }
        __syncwarp();
        const int sub = lane >> 4, q = (col0 >> 2) + (lane & 15);
        for (int r = 0; r < 32; r += 2) {
          const int lr2 = wrow0 + r + sub, gr = m0 + lr2, gc = n0 + 4 * q;
          if (gr >= p.M || gc >= p.N) continue;
          float* dst = C + p.c + (int64_t)gr * p.ldc + gc;
          const float4 o = *reinterpret_cast<const float4*>(Cs + lr2 * CLD + 4 * (q ^ (lr2 & 7)));
          if (gc + 4 <= p.N) {
            *reinterpret_cast<float4*>(dst) = o;
          } else {
            dst[0] = o.x;
            if (gc + 1 < p.N) dst[1] = o.y;
            if (gc + 2 < p.N) dst[2] = o.z;
          }
        }
      } else {
        // unaligned C: each thread updates its own row half in global memory
        const int row = m0 + lr;
        if (row < p.M) {
          float* crow = C + p.c + (int64_t)row * p.ldc + n0 + col0;
          for (int q = 0; q < 64 && n0 + col0 + q < p.N; ++q)
            crow[q] = (beta != 0.f) ? alpha * rs[q] + beta * crow[q] : alpha * rs[q];
        }
      }
      __syncwarp();
      if (NCB == 1 && i + 1 < ntl) {
        prefetch(i + 1);
        asm volatile("cp.async.commit_group;" ::: "memory");
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
  }
  __syncwarp();
  if (*(volatile int*)abort_flag != 0) {
    if (threadIdx.x == 0) atomicOr(status, DEV_TIMEOUT);
    // copies the producer issued may still be in flight: wait (bounded)
    // for the stages it filled before the shared memory is released
    if (warp == 0 && lane == 0)
      for (int g = (issued > NST ? issued - NST : 0); g < issued; ++g)
        (void)mbar_wait(&full[g % NST], (g / NST) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TMEM_COLS)
                 : "memory");
  }
}

// Split of one operand into the K-major hi/lo arrays: output row r (< rows)
// of problem q holds op(X)(r, 0:K) zero-padded to Kp, where op(X)(r, k) is
// X[off + r ld + k] (KMAJ) or X[off + k ld + r] (the transposed read goes
// through a 32 x 33 shared tile so that both sides stay coalesced).
// Grid: (row tiles of 32 x K tiles of 32 flattened, problems); 32 x 8 threads.
struct SplitProb {
  int rows, K, ld;
  int64_t off;
  int r0;  // first output row
};

template <bool KMAJ, int NP>
__global__ void __launch_bounds__(256)
tc_split_kernel(const SplitProb* __restrict__ probs, int Kp, const float* __restrict__ X,
                float* __restrict__ p0, int64_t part_stride) {
  __shared__ float t[32][33];
  const SplitProb q = probs[blockIdx.y];
  const int nkt = Kp / 32;
  const int rt = blockIdx.x / nkt, kt = blockIdx.x % nkt;
  const int rb = rt * 32, kb = kt * 32;
  if (rb >= q.rows) return;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (KMAJ) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int r = rb + ty + 8 * i, k = kb + tx;
      t[ty + 8 * i][tx] = (r < q.rows && k < q.K) ? X[q.off + (int64_t)r * q.ld + k] : 0.f;
    }
  } else {
    // read X[k][r] with r contiguous, store transposed
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = kb + ty + 8 * i, r = rb + tx;
      t[tx][ty + 8 * i] = (r < q.rows && k < q.K) ? X[q.off + (int64_t)k * q.ld + r] : 0.f;
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int r = rb + ty + 8 * i, k = kb + tx;
    if (r < q.rows) {
      const float x = t[ty + 8 * i][tx];
      const int64_t o = (int64_t)(q.r0 + r) * Kp + k;
      float parts[NP];
      split_tf32<NP>(x, parts);
#pragma unroll
      for (int pp = 0; pp < NP; ++pp) p0[o + pp * part_stride] = parts[pp];
    }
  }
}

}  // namespace tc
}  // namespace cbddc

// ------------------------------------------------------------------ host
namespace cbddc {
namespace tc {

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link-time dependence on libcuda).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

inline EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    CB_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    CB_CHECK(q == cudaDriverEntryPointSuccess && p != nullptr, CBDDC_ECUDA,
             "cuTensorMapEncodeTiled is not available from the driver");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map of a K-major [rows][Kp] FP32 array: boxes of 32 (K) x 128 rows,
// 128-byte swizzle, zero fill outside the array.
inline CUtensorMap encode_kmajor(const float* base, int64_t rows, int Kp) {
  CB_CHECK(Kp % BKC == 0 && Kp > 0 && rows > 0, CBDDC_EINVAL, "tensor map: bad K-major array shape");
  CB_CHECK(((uintptr_t)base & 15) == 0, CBDDC_EINVAL, "tensor map: base not 16-byte aligned");
  CUtensorMap m;
  const cuuint64_t dims[2] = {(cuuint64_t)Kp, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)Kp * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)BKC, (cuuint32_t)BM};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CB_CHECK(r == CUDA_SUCCESS, CBDDC_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

template <int NST, int NCB, int NP, int KS>
inline void set_smem_attr_one() {
  CB_CUDA(cudaFuncSetAttribute(tc_gemm_kernel<NST, NCB, NP, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               TcSmem<NST, NCB, NP>::bytes));
}

inline void set_smem_attr() {
  static bool done = false;
  if (!done) {
    set_smem_attr_one<1, 2, 2, 1>();
    set_smem_attr_one<1, 2, 2, 4>();
    set_smem_attr_one<2, 1, 2, 4>();
    set_smem_attr_one<2, 1, 2, 1>();
    set_smem_attr_one<1, 2, 3, 1>();
    set_smem_attr_one<1, 2, 3, 4>();
    done = true;
  }
}

// Persistent CTAs: one per SM (one fits), never more than tiles.
inline int tc_grid(int ntiles) {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    CB_CUDA(cudaGetDevice(&dev));
    CB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return std::max(1, std::min(ntiles, sms));
}

}  // namespace tc
}  // namespace cbddc
