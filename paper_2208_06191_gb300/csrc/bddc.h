// BDDC context (internal).
#pragma once
#include <memory>

#include "common.h"
#include "dense.cuh"
#include "krylov.h"

struct bddc_ctx {
  fem_problem* P = nullptr;
  int precision = CBDDC_FP64, primal = CBDDC_PRIMAL_V;
  int nb = 64;                              // pivot block width of the local sweeps
  int tile_order = 0;                       // setup GEMM tiles: 0 by subdomain, 1 largest first
  float ms_setup_tuned = 0.f, ms_setup_default = 0.f;  // autotuning record (FP32 contexts)
  double pivot_tol = 1e-13;
  int nsub = 0;
  size_t esize = 8;  // bytes per element of the local operators
  // per-subdomain sizes (host)
  std::vector<int> nI, nG, nr, nv, na, nc, ns, ldA, ldS, ldPhi, ldY, ldG;
  std::vector<int64_t> offA, offS, offPhi, offY, offZ, offG, offSPhi, offKc, offX, offYp, offP, offE;
  std::vector<int64_t> offI, offGam, offC, offCon;
  int maxI = 0, maxG = 0, maxR = 0, maxNs = 0, maxC = 0, maxA = 0;
  int n_pi = 0, n_if = 0;
  int64_t totI = 0, totG = 0, totC = 0;
  // device size/offset arrays
  cbddc::DVec<int> d_nI, d_nG, d_nr, d_nv, d_na, d_nc, d_ns, d_ldA, d_ldS, d_ldPhi, d_ldY, d_ldG;
  cbddc::DVec<int64_t> d_offA, d_offS, d_offPhi, d_offY, d_offZ, d_offG, d_offSPhi, d_offKc, d_offE;
  cbddc::DVec<int64_t> d_offI, d_offGam, d_offC, d_offCon, d_offN;
  // local node ordering [I | Gamma_r | Gamma_v]: local node index -> position
  cbddc::DVec<int> perm;
  // local operators (element type float or double, raw storage)
  cbddc::DVec<unsigned char> Aloc, Sw, Phi, Y, Zf, Wf, G, SPhi, Kc, Xp, Yp, Pd, Et;
  cbddc::DVec<float> tc_scratch;            // split operands of the tensor-core GEMMs (FP32)
  cbddc::DVec<float> Xlo, Ylo, DXlo, DYlo;  // second TF32 parts of the sweep panels (FP32)
  cbddc::DVec<float> Xlo2, Ylo2, DXlo2, DYlo2;  // third parts (three-part split)
  int tc_parts_sweep = 0, tc_parts_other = 0;  // TF32 parts per operand chosen at creation
  // apply maps
  cbddc::DVec<int> gdofI, gdofG, gam_if, if_dof, if_ptr, if_src;
  cbddc::DVec<double> Dg;
  cbddc::DVec<int> cons_ptr, cons_idx;   // constraint -> members (local r index)
  cbddc::DVec<double> cons_w;            // weight of each member
  cbddc::DVec<int> gprim, cg_ptr, cg_src;  // coarse rhs gather
  cbddc::DVec<int> ce_key, ce_ptr, ce_src; // coarse matrix entries
  int64_t n_ce = 0;
  cbddc::DVec<double> Sc, ScX, ScY, ScP;   // coarse matrix (inverted in place)
  // work items {subdomain, row block} of the batched apply kernels
  cbddc::DVec<int2> itI, itG, itP, itR;
  int n_itI = 0, n_itG = 0, n_itP = 0, n_itR = 0;
  cbddc::DVec<int> cnch;                   // coarse-restriction chunks per local primal entry
  // sparse interior-interface coupling blocks of the assembled matrix
  // (problems with a global BSR), sliced ELL: gi = rows of the assembled
  // interface nodes, columns = packed interior nodes; ig = rows of the
  // packed interior nodes, columns = interface nodes; per slice its first
  // step (off) and step count (len), per lane slot its row, per step and
  // lane the column and the BSR block (src, -1 = padding); uq / zq: the
  // node-packed inputs (x, y, z, pad) in the operator precision
  bool sparse_cpl = false;
  int n_sgi = 0, n_sig = 0;
  int64_t steps_gi = 0, steps_ig = 0, n_cpl_blocks = 0;
  cbddc::DVec<int> sgi_off, sgi_len, sgi_row, sgi_col, sgi_src;
  cbddc::DVec<int> sig_off, sig_len, sig_row, sig_col, sig_src;
  cbddc::DVec<unsigned char> sgi_val, sig_val, uq, zq;
  // apply work vectors
  cbddc::DVec<double> u0, hG, gI, wG, cl, rc, uc, yG, xI, zl;
  // sweep descriptors and GEMM problem lists
  cbddc::DVec<cbddc::SweepDesc> sw1, sw2, swg, swc;
  int steps1 = 0, steps2 = 0, stepsg = 0, stepsc = 0;
  std::vector<cbddc::GemmList> gl_sw1, gl_sw2, gl_swg, gl_swc;
  cbddc::GemmList gl_E, gl_S, gl_W, gl_T, gl_PhiA, gl_SPhi, gl_Kc;
  cbddc::DVec<double> gl;                  // scaled interface restriction
  // deluxe scaling: blocks b = (edge or face class K, subdomain s sharing
  // it) with the class DoFs' positions in s's interface vector; S_b (class
  // block of s's Schur complement), D_b = Shat_K^-1 S_b (Shat_K = sum of
  // the class's S_b, inverted in place) and E_b = D_b^T share the offsets
  int scaling = CBDDC_SCALING_COUNTING;
  // Petrov coarse space: left basis Psi (layout of Phi), its vertex columns
  // -(S_vr T)^T by one grouped GEMM per setup
  int coarse = CBDDC_COARSE_GALERKIN;
  cbddc::DVec<unsigned char> Psi;
  cbddc::GemmList gl_PsiV;
  int n_dlx = 0, n_dcls = 0, maxDn = 0, stepsd = 0;
  cbddc::DVec<int> dlx_n, dlx_sub, dlx_ld, dlx_pos, dcls_ptr, dcls_blk;
  cbddc::DVec<int64_t> dlx_poff, dlx_off, dcls_off;
  cbddc::DVec<unsigned char> Dsb, Ddb, Deb, Dsh, DX, DY, DP;
  cbddc::DVec<cbddc::SweepDesc> swd;
  std::vector<cbddc::GemmList> gl_swd;
  cbddc::GemmList gl_dlx;
  cbddc::DVec<double> yD;                  // averaging input, deluxe blocks applied
  double setup_flops = 0.0, apply_flops = 0.0;
  int64_t local_bytes = 0;
  // Krylov and Newton workspaces (allocated on first use)
  cbddc::Gmres gm;
  cbddc::DVec<double> nw_r, nw_b, nw_delta, nw_d;
  // multilevel: the coarse problem as an unassembled matrix and its BDDC
  std::vector<int> gprim_h;
  int levels = 2, n_parts2 = 0, primal2 = 0, precision2 = CBDDC_FP64;
  std::vector<int> part2;
  std::unique_ptr<fem_problem> coarse_prob;
  std::unique_ptr<bddc_ctx> next;
  cbddc::DVec<int64_t> d_cbase;  // first coarse contribution block of each subdomain
  int64_t device_bytes() const;
};

namespace cbddc {
void bddc_create(fem_problem* P, const bddc_options* opt, bddc_ctx* C);
void bddc_run_setup(bddc_ctx* C, cudaStream_t s);
void bddc_run_apply(bddc_ctx* C, const double* r, double* z, cudaStream_t s);
void bddc_run_apply_noalloc(bddc_ctx* C, const double* r, double* z, cudaStream_t s);
int64_t bddc_noalloc_scratch_needed(const bddc_ctx* C);
int64_t bddc_noalloc_scratch_capacity();
}  // namespace cbddc
