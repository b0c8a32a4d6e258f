// GMRES workspace and Newton helpers (internal).
#pragma once
#include "common.h"

struct bddc_ctx;

namespace cbddc {

struct Gmres {
  int64_t n = 0;
  int m = 0;
  int nchunks = 0;
  int pstride = 0;           // row stride of the per-CTA partial sums
  int hstride = 0;           // stride of the three CGS coefficient vectors in h
  int reorth = 0;            // second Gram-Schmidt passes of the last solve
  DVec<double> V, Zb, w, r, H, cs, sn, g, y, h, partial, scal;
  DVec<int> flags;
  DVec<unsigned> ticket;
  DVec<double> cpart;        // per-CTA partials of the cooperative orthogonalisation
  int coop_grid = 0;         // its grid size (0: use the multi-launch path)
  DVec<double> mpart;        // per-CTA partials of the cooperative MGS step
  int mgs_grid = 0, mgs_rpt = 0;  // its grid and rows per thread (0: not available)
  double* host_scal = nullptr;
  int* host_flags = nullptr;
  void ensure_small(int64_t n_);
  void ensure(int64_t n_, int m_);
  Gmres() = default;
  Gmres(const Gmres&) = delete;
  Gmres& operator=(const Gmres&) = delete;
  ~Gmres();
};

int gmres_run(fem_problem* P, bddc_ctx* C, Gmres& G, const double* b, double* x, int restart,
              int max_iters, double rtol, int* iters_out, double* relres_out, cudaStream_t s);
double device_norm(fem_problem* P, Gmres& G, const double* v, cudaStream_t s);
void axpby(double a, const double* x, double b, const double* y, double* out, int64_t n, cudaStream_t s);

}  // namespace cbddc
