// Internal definitions shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <string>
#include <vector>

#include "../../include/cardiac_bddc.h"

namespace cbddc {

// Status carried through the host code; converted to the C return code at
// the ABI boundary.
struct Error {
  int code;
  std::string msg;
};

void set_last_error(const std::string& msg);

#define CB_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      throw ::cbddc::Error{CBDDC_ECUDA, std::string(#call) + ": " +          \
                                            cudaGetErrorString(e_)};         \
    }                                                                        \
  } while (0)

#define CB_CHECK(cond, code, msg)                                            \
  do {                                                                       \
    if (!(cond)) throw ::cbddc::Error{(code), (msg)};                        \
  } while (0)

// Counts every kernel launch of the library and checks the launch status.
void count_launch();
#define CB_LAUNCH()                       \
  do {                                    \
    ::cbddc::count_launch();              \
    CB_CUDA(cudaGetLastError());          \
  } while (0)

// Optional CUDA-event timing of one kernel class (see cbddc_timer_start).
bool timer_active(int kernel_class);
void timer_begin(int kernel_class, cudaStream_t s);
void timer_end(int kernel_class, cudaStream_t s, double flops, double bytes);

// Device-side error bits, OR-ed into a status word by kernels.
enum : int {
  DEV_INVERTED = 1,  // J <= 0 at a quadrature point
  DEV_PIVOT = 2,     // tiny or non-finite pivot
  DEV_NONFINITE = 4, // NaN / Inf found
  DEV_TIMEOUT = 8    // a bounded device-side wait expired
};

// Owning device allocation (no copy; move only).
template <typename T>
struct DVec {
  T* p = nullptr;
  size_t n = 0;
  DVec() = default;
  DVec(const DVec&) = delete;
  DVec& operator=(const DVec&) = delete;
  DVec(DVec&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DVec& operator=(DVec&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DVec() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error{CBDDC_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) +
                                    " bytes failed: " + cudaGetErrorString(e)};
    }
    n = count;
  }
  void upload(const std::vector<T>& h) {
    alloc(h.size());
    if (!h.empty()) CB_CUDA(cudaMemcpy(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  }
  size_t bytes() const { return n * sizeof(T); }
};

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }
inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// Per-subdomain description built on the host at problem creation.
struct SubHost {
  std::vector<int> nodes;      // global node ids (free nodes), increasing
  std::vector<int> iface;      // 1 if the node is shared by >= 2 subdomains
};

}  // namespace cbddc

// ---------------------------------------------------------------- problem
struct fem_problem {
  // description
  int elem_type = 0, order = 1, n_en = 8, n_qp = 8, n_fn = 4, n_fqp = 4;
  bool tet = false;                         // tetrahedra (else hexahedra)
  int n_nodes = 0, n_el = 0, n_parts = 0, n_faces = 0, n_robin = 0;
  double rho = 0.0, robin_par[2][4] = {{0}};  // density; Robin K_perp, K_par, C_perp, C_par
  // time state (fem_set_time_state): dt > 0 switches inertia and damping on
  double dt = 0.0;
  const double* d_prev = nullptr;           // borrowed device vectors [n_free]
  const double* d_prev2 = nullptr;
  int64_t n_free_nodes = 0, n_free = 0, nnzb = 0;
  int fiber_kind = 0;
  double fiber[8] = {0};
  double mat[8] = {0};
  double pressure = 0, gamma = 0;
  // host topology kept for BDDC context creation
  std::vector<int> node_to_free;            // -1 for Dirichlet
  std::vector<int> elems_h;                 // n_el * n_en
  std::vector<int> part_h;                  // n_el
  std::vector<cbddc::SubHost> subs;         // per subdomain
  std::vector<int> share_count;             // per node (free nodes only)
  std::vector<int> vertices;                // vertex nodes
  std::vector<std::vector<int>> edges, faces;  // classes (node lists)
  std::vector<double> coords_h;             // n_nodes*3 (fine level only)
  // device data
  cbddc::DVec<double> coords;               // n_nodes*3
  cbddc::DVec<double> fib_nodal;            // n_nodes*6 (f, n) for nodal fibres
  cbddc::DVec<int> elems;                   // n_el*n_en
  cbddc::DVec<int> face_nodes;              // (n_faces+n_robin)*n_fn (outward order)
  cbddc::DVec<int> robin_set;               // n_robin parameter-set ids
  cbddc::DVec<double> acc_full, vel_full;   // n_nodes*3: d-2d'+d'', (d-d')/dt
  cbddc::DVec<int> free_nodes;              // n_free_nodes -> node id
  cbddc::DVec<double> d_full;               // n_nodes*3 displacement
  cbddc::DVec<double> contrib;              // 3x3 blocks of element/face matrices
  cbddc::DVec<double> rcontrib;             // 3-vectors of element/face residuals
  int64_t n_elem_blocks = 0, n_face_blocks = 0;
  int64_t n_elem_vec = 0, n_face_vec = 0;
  cbddc::DVec<int> bsr_row_ptr, bsr_col;
  cbddc::DVec<double> bsr_vals;
  cbddc::DVec<int> slot_ptr, slot_src;      // BSR slot -> contrib blocks
  cbddc::DVec<int> res_ptr, res_src;        // free node -> rcontrib entries
  // subdomain-local slots (for the dense local matrices)
  int64_t n_lslots = 0;
  cbddc::DVec<int> lslot_sub, lslot_row, lslot_col;  // local node indices
  cbddc::DVec<int> lslot_ptr, lslot_src;
  cbddc::DVec<int> status;                  // device error bits
  cbddc::DVec<double> scratch;              // norms etc.
  bool has_tangent = false;
  // autotuned setup per precision (index 0 FP64, 1 FP32): sweep block,
  // tile order (-1: not tuned yet) and the measured setup times
  int tuned_nb[2] = {64, 64}, tuned_to[2] = {-1, -1};
  float tuned_ms[2] = {0.f, 0.f}, default_ms[2] = {0.f, 0.f};
  int64_t device_bytes() const;
};
