// FE assembly and SpMV entry points (internal).
#pragma once
#include "common.h"

namespace cbddc {

void build_problem(const fem_problem_desc* d, fem_problem* P);
void classify_interface(int nn, const std::vector<std::vector<int>>& members,
                        const std::vector<int>& share_count, const std::vector<int>& eptr,
                        const std::vector<int>& eidx, const std::vector<char>* on_bnd,
                        std::vector<int>& vertices, std::vector<std::vector<int>>& edges,
                        std::vector<std::vector<int>>& faces);
void build_local_slots(fem_problem* P, const std::vector<int>& cptr, const std::vector<int>& cidx,
                       const std::vector<int>& cpart, const std::vector<int64_t>& cbase);
void hex_face_node_list(int k, int f, int* out);
void init_shape_tables(int order);

// Element/face residual (and tangent when want_tangent) into the
// contribution buffers, then gathers into residual (may be null) and, with
// the tangent, the BSR values.  Kernels OR DEV_INVERTED into P->status.
void assemble(fem_problem* P, const double* d, double lam, double* residual,
              bool want_tangent, cudaStream_t s);

void bsr_spmv(const fem_problem* P, const double* x, double* y, cudaStream_t s);

}  // namespace cbddc
