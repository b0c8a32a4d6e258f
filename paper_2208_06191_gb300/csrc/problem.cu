// Host-side problem construction: DoF numbering, BSR pattern, gather lists
// from element/face matrices to the global and subdomain matrices, and the
// interface classification of Section 3.2 (faces, edges, vertices).
#include <algorithm>
#include <array>
#include <map>
#include <numeric>

#include "common.h"
#include "fem.h"

namespace cbddc {

namespace {

struct UnionFind {
  std::vector<int> p;
  explicit UnionFind(int n) : p(n) { std::iota(p.begin(), p.end(), 0); }
  int find(int x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
  }
  void unite(int a, int b) {
    a = find(a); b = find(b);
    if (a != b) p[std::max(a, b)] = std::min(a, b);
  }
};

// CSR from (key, value) pairs with keys in [0, nkeys).
void build_csr(int64_t nkeys, const std::vector<std::pair<int64_t, int>>& kv,
               std::vector<int>& ptr, std::vector<int>& src) {
  ptr.assign(nkeys + 1, 0);
  for (auto& e : kv) ptr[e.first + 1]++;
  for (int64_t i = 0; i < nkeys; ++i) ptr[i + 1] += ptr[i];
  src.assign(kv.size(), 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (auto& e : kv) src[fill[e.first]++] = e.second;
}

}  // namespace

// Local node indices of face f of a hexahedron of order k, ordered
// lexicographically in the face parameters (s, t) so that the parametric
// normal d x/ds x d x/dt points out of the element.  Face f fixes reference
// axis face_axis[f] at -1 (even f) or +1 (odd f).
void hex_face_node_list(int k, int f, int* out) {
  static const int axis[6] = {0, 0, 1, 1, 2, 2};
  static const int s_ax[6] = {2, 1, 0, 2, 1, 0};
  static const int t_ax[6] = {1, 2, 2, 0, 0, 1};
  const int m = k + 1;
  const int fixed = (f % 2 == 0) ? 0 : k;
  int n = 0;
  for (int it = 0; it < m; ++it)
    for (int is = 0; is < m; ++is) {
      int idx[3];
      idx[axis[f]] = fixed;
      idx[s_ax[f]] = is;
      idx[t_ax[f]] = it;
      out[n++] = idx[0] + m * (idx[1] + m * idx[2]);
    }
}

// Local node indices of face f (opposite vertex f) of a tetrahedron of
// order k: the three vertices (o, s-end, t-end) with (x_s - x_o) x
// (x_t - x_o) pointing out of the element, then for P2 the midpoints of
// (o, s-end), (s-end, t-end), (o, t-end).
void tet_face_node_list(int k, int f, int* out) {
  static const int ost[4][3] = {{1, 2, 3}, {0, 3, 2}, {0, 1, 3}, {0, 2, 1}};
  static const int edge_of[4][4] = {{-1, 4, 6, 7}, {4, -1, 5, 8}, {6, 5, -1, 9}, {7, 8, 9, -1}};
  const int o = ost[f][0], a = ost[f][1], b = ost[f][2];
  out[0] = o; out[1] = a; out[2] = b;
  if (k == 2) {
    out[3] = edge_of[o][a];
    out[4] = edge_of[a][b];
    out[5] = edge_of[o][b];
  }
}

// Face node list of either element family.
void face_node_list(bool tet, int k, int f, int* out) {
  if (tet) tet_face_node_list(k, f, out);
  else hex_face_node_list(k, f, out);
}

// Interface classes of Section 3.2 from subdomain membership: interface
// nodes (shared by >= 2 subdomains) are grouped by their sharing set and
// split into connected pieces (two nodes are adjacent when an element holds
// both).  A piece shared by 2 subdomains is a face; shared by 3 or more it
// is an edge, except that single-node pieces are vertices and, when the
// outer boundary is known (on_bnd != null), edge nodes on it are vertices
// too (the subdomain corners on the surface).
void classify_interface(int nn, const std::vector<std::vector<int>>& members,
                        const std::vector<int>& share_count, const std::vector<int>& eptr,
                        const std::vector<int>& eidx, const std::vector<char>* on_bnd,
                        std::vector<int>& vertices, std::vector<std::vector<int>>& edges,
                        std::vector<std::vector<int>>& faces) {
  std::map<std::vector<int>, int> key_of;
  std::vector<int> key(nn, -1);
  for (int v = 0; v < nn; ++v)
    if (share_count[v] >= 2) {
      auto it = key_of.find(members[v]);
      if (it == key_of.end()) it = key_of.emplace(members[v], (int)key_of.size()).first;
      key[v] = it->second;
    }
  UnionFind uf(nn);
  const int ne = (int)eptr.size() - 1;
  for (int e = 0; e < ne; ++e) {
    const int* en = &eidx[eptr[e]];
    const int k = eptr[e + 1] - eptr[e];
    for (int a = 0; a < k; ++a) {
      if (key[en[a]] < 0) continue;
      for (int b = a + 1; b < k; ++b)
        if (key[en[b]] == key[en[a]]) uf.unite(en[a], en[b]);
    }
  }
  std::map<int, std::vector<int>> classes;
  for (int v = 0; v < nn; ++v)
    if (key[v] >= 0) classes[uf.find(v)].push_back(v);
  vertices.clear();
  edges.clear();
  faces.clear();
  for (auto& kvp : classes) {
    std::vector<int>& nodes = kvp.second;
    std::sort(nodes.begin(), nodes.end());
    const int s = (int)members[nodes[0]].size();
    if (s == 2) {
      faces.push_back(nodes);
    } else if (nodes.size() == 1) {
      vertices.push_back(nodes[0]);
    } else {
      std::vector<int> rest;
      for (int v : nodes) {
        if (on_bnd && (*on_bnd)[v]) vertices.push_back(v);
        else rest.push_back(v);
      }
      if (!rest.empty()) edges.push_back(rest);
    }
  }
  std::sort(vertices.begin(), vertices.end());
  std::sort(edges.begin(), edges.end());
  std::sort(faces.begin(), faces.end());
}

// Subdomain-local slot lists for the dense local matrices.  Contributor c
// (an element, a face, or a finer subdomain at a coarse level) has nodes
// cidx[cptr[c]..cptr[c+1]), belongs to subdomain cpart[c] and stores its
// 3x3 blocks (a, b) at block index cbase[c] + a * k + b (k = its node count).
// Nodes that are not in the subdomain's node list (Dirichlet nodes) are
// skipped.  Every distinct (subdomain, local row node, local col node)
// becomes one slot with the list of blocks summed into it.
void build_local_slots(fem_problem* P, const std::vector<int>& cptr, const std::vector<int>& cidx,
                       const std::vector<int>& cpart, const std::vector<int64_t>& cbase) {
  const int np = P->n_parts;
  std::vector<int64_t> base(np + 1, 0);
  for (int p = 0; p < np; ++p) {
    const int64_t nl = (int64_t)P->subs[p].nodes.size();
    base[p + 1] = base[p] + nl * nl;
  }
  std::vector<std::pair<int64_t, int>> lkv;
  std::vector<int> loc;
  const int nc = (int)cpart.size();
  for (int c = 0; c < nc; ++c) {
    const int p = cpart[c];
    const auto& nv = P->subs[p].nodes;
    const int64_t nl = (int64_t)nv.size();
    const int k = cptr[c + 1] - cptr[c];
    loc.assign(k, -1);
    for (int a = 0; a < k; ++a) {
      const int v = cidx[cptr[c] + a];
      auto it = std::lower_bound(nv.begin(), nv.end(), v);
      if (it != nv.end() && *it == v) loc[a] = (int)(it - nv.begin());
    }
    for (int a = 0; a < k; ++a) {
      if (loc[a] < 0) continue;
      for (int b = 0; b < k; ++b)
        if (loc[b] >= 0) {
          const int64_t blk = cbase[c] + (int64_t)a * k + b;
          CB_CHECK(blk < INT32_MAX, CBDDC_EINVAL, "too many contribution blocks for 32-bit indices");
          lkv.push_back({base[p] + loc[a] * nl + loc[b], (int)blk});
        }
    }
  }
  std::sort(lkv.begin(), lkv.end());
  std::vector<int> lsub, lrow, lcol, lptr, lsrc;
  lptr.push_back(0);
  int p = 0;
  for (size_t i = 0; i < lkv.size();) {
    size_t j = i;
    while (j < lkv.size() && lkv[j].first == lkv[i].first) ++j;
    const int64_t key = lkv[i].first;
    while (key >= base[p + 1]) ++p;
    const int64_t nl = (int64_t)P->subs[p].nodes.size();
    const int64_t off = key - base[p];
    lsub.push_back(p);
    lrow.push_back((int)(off / nl));
    lcol.push_back((int)(off % nl));
    for (size_t q = i; q < j; ++q) lsrc.push_back(lkv[q].second);
    lptr.push_back((int)lsrc.size());
    i = j;
  }
  P->n_lslots = (int64_t)lsub.size();
  P->lslot_sub.upload(lsub);
  P->lslot_row.upload(lrow);
  P->lslot_col.upload(lcol);
  P->lslot_ptr.upload(lptr);
  P->lslot_src.upload(lsrc);
}

void build_problem(const fem_problem_desc* d, fem_problem* P) {
  CB_CHECK(d != nullptr, CBDDC_EINVAL, "null description");
  CB_CHECK(d->elem_type >= CBDDC_HEX_Q1 && d->elem_type <= CBDDC_TET_P2, CBDDC_EINVAL,
           "unsupported element type");
  CB_CHECK(d->n_nodes > 0 && d->n_elems > 0 && d->coords && d->elems && d->elem_part,
           CBDDC_EINVAL, "empty mesh");
  CB_CHECK(d->n_parts >= 1, CBDDC_EINVAL, "n_parts must be >= 1");
  CB_CHECK(d->fiber_kind == CBDDC_FIBER_SLAB_HELIX || d->fiber_kind == CBDDC_FIBER_NODAL,
           CBDDC_EINVAL, "unsupported fibre kind");
  if (d->fiber_kind == CBDDC_FIBER_SLAB_HELIX)
    CB_CHECK(d->fiber_params[1] != d->fiber_params[0], CBDDC_EINVAL, "degenerate fibre range");
  else
    CB_CHECK(d->fiber_nodal != nullptr, CBDDC_EINVAL, "nodal fibre field missing");
  P->elem_type = d->elem_type;
  P->tet = d->elem_type == CBDDC_TET_P1 || d->elem_type == CBDDC_TET_P2;
  P->order = (d->elem_type == CBDDC_HEX_Q1 || d->elem_type == CBDDC_TET_P1) ? 1 : 2;
  const int k = P->order, m = k + 1;
  const bool tet = P->tet;
  if (tet) {
    P->n_en = k == 1 ? 4 : 10;
    P->n_qp = k == 1 ? 1 : 4;
    P->n_fn = k == 1 ? 3 : 6;
    P->n_fqp = k == 1 ? 1 : 3;
  } else {
    P->n_en = m * m * m;
    P->n_qp = P->n_en;   // (k+1)^3 Gauss points
    P->n_fn = m * m;
    P->n_fqp = m * m;
  }
  const int n_lfaces = tet ? 4 : 6;
  P->n_nodes = d->n_nodes;
  P->n_el = d->n_elems;
  P->n_parts = d->n_parts;
  P->n_faces = d->n_pressure_faces;
  P->n_robin = d->n_robin_faces;
  CB_CHECK(P->n_faces >= 0 && P->n_robin >= 0, CBDDC_EINVAL, "negative face count");
  CB_CHECK(P->n_robin == 0 || d->robin_faces != nullptr, CBDDC_EINVAL, "Robin faces missing");
  CB_CHECK(d->rho >= 0.0, CBDDC_EINVAL, "negative density");
  P->rho = d->rho;
  for (int q = 0; q < 2; ++q)
    for (int c = 0; c < 4; ++c) {
      CB_CHECK(d->robin[q][c] >= 0.0, CBDDC_EINVAL, "negative Robin coefficient");
      P->robin_par[q][c] = d->robin[q][c];
    }
  P->fiber_kind = d->fiber_kind;
  for (int i = 0; i < 8; ++i) { P->fiber[i] = d->fiber_params[i]; P->mat[i] = d->material[i]; }
  P->pressure = d->pressure;
  P->gamma = d->gamma;
  const int nen = P->n_en, nn = P->n_nodes, ne = P->n_el;

  P->elems_h.assign(d->elems, d->elems + (size_t)ne * nen);
  P->part_h.assign(d->elem_part, d->elem_part + ne);
  for (int v : P->elems_h) CB_CHECK(v >= 0 && v < nn, CBDDC_EINVAL, "element node out of range");
  for (int v : P->part_h) CB_CHECK(v >= 0 && v < P->n_parts, CBDDC_EINVAL, "partition id out of range");

  // free-DoF numbering
  std::vector<char> is_dir(nn, 0);
  for (int i = 0; i < d->n_dirichlet; ++i) {
    int v = d->dirichlet_nodes[i];
    CB_CHECK(v >= 0 && v < nn, CBDDC_EINVAL, "Dirichlet node out of range");
    is_dir[v] = 1;
  }
  P->node_to_free.assign(nn, -1);
  std::vector<int> free_nodes;
  for (int v = 0; v < nn; ++v)
    if (!is_dir[v]) { P->node_to_free[v] = (int)free_nodes.size(); free_nodes.push_back(v); }
  P->n_free_nodes = (int64_t)free_nodes.size();
  P->n_free = 3 * P->n_free_nodes;
  CB_CHECK(P->n_free_nodes > 0, CBDDC_EINVAL, "no free nodes");
  const int64_t nf = P->n_free_nodes;
  const std::vector<int>& n2f = P->node_to_free;

  // pressure faces, then Robin faces -> node lists
  const int nfn = P->n_fn;
  const int n_all_faces = P->n_faces + P->n_robin;
  std::vector<int> face_nodes((size_t)n_all_faces * nfn);
  std::vector<int> face_elem(n_all_faces);
  std::vector<int> robin_set(P->n_robin);
  for (int f = 0; f < n_all_faces; ++f) {
    const bool rob = f >= P->n_faces;
    const int g = rob ? f - P->n_faces : f;
    int e = rob ? d->robin_faces[3 * g] : d->pressure_faces[2 * f];
    int lf = rob ? d->robin_faces[3 * g + 1] : d->pressure_faces[2 * f + 1];
    CB_CHECK(e >= 0 && e < ne && lf >= 0 && lf < n_lfaces, CBDDC_EINVAL,
             rob ? "bad Robin face" : "bad pressure face");
    if (rob) {
      robin_set[g] = d->robin_faces[3 * g + 2];
      CB_CHECK(robin_set[g] == 0 || robin_set[g] == 1, CBDDC_EINVAL, "Robin parameter set must be 0 or 1");
    }
    int loc[9];
    face_node_list(tet, k, lf, loc);
    for (int a = 0; a < nfn; ++a) face_nodes[(size_t)f * nfn + a] = P->elems_h[(size_t)e * nen + loc[a]];
    face_elem[f] = e;
  }

  // BSR pattern: free-node pairs sharing an element
  std::vector<int64_t> keys;
  keys.reserve((size_t)ne * nen * nen);
  for (int e = 0; e < ne; ++e) {
    const int* en = &P->elems_h[(size_t)e * nen];
    for (int a = 0; a < nen; ++a) {
      int ra = n2f[en[a]];
      if (ra < 0) continue;
      for (int b = 0; b < nen; ++b) {
        int cb = n2f[en[b]];
        if (cb >= 0) keys.push_back((int64_t)ra * nf + cb);
      }
    }
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  P->nnzb = (int64_t)keys.size();
  CB_CHECK(P->nnzb < INT32_MAX, CBDDC_EINVAL, "matrix too large for 32-bit block indices");
  std::vector<int> row_ptr(nf + 1, 0), col(keys.size());
  for (size_t i = 0; i < keys.size(); ++i) {
    row_ptr[keys[i] / nf + 1]++;
    col[i] = (int)(keys[i] % nf);
  }
  for (int64_t i = 0; i < nf; ++i) row_ptr[i + 1] += row_ptr[i];
  auto slot_of = [&](int r, int c) -> int {
    const int* b = col.data() + row_ptr[r];
    const int* e = col.data() + row_ptr[r + 1];
    const int* it = std::lower_bound(b, e, c);
    return (int)(it - col.data());
  };

  // contribution blocks: elements then faces
  P->n_elem_blocks = (int64_t)ne * nen * nen;
  P->n_face_blocks = (int64_t)n_all_faces * nfn * nfn;
  P->n_elem_vec = (int64_t)ne * nen;
  P->n_face_vec = (int64_t)n_all_faces * nfn;
  CB_CHECK(P->n_elem_blocks + P->n_face_blocks < INT32_MAX, CBDDC_EINVAL,
           "too many element blocks for 32-bit indices");
  std::vector<std::pair<int64_t, int>> kv;
  kv.reserve(P->n_elem_blocks + P->n_face_blocks);
  std::vector<std::pair<int64_t, int>> rkv;
  for (int e = 0; e < ne; ++e) {
    const int* en = &P->elems_h[(size_t)e * nen];
    for (int a = 0; a < nen; ++a) {
      int ra = n2f[en[a]];
      if (ra < 0) continue;
      rkv.push_back({ra, e * nen + a});
      for (int b = 0; b < nen; ++b) {
        int cb = n2f[en[b]];
        if (cb >= 0) kv.push_back({slot_of(ra, cb), (int)((int64_t)e * nen * nen + a * nen + b)});
      }
    }
  }
  for (int f = 0; f < n_all_faces; ++f) {
    const int* fn = &face_nodes[(size_t)f * nfn];
    for (int a = 0; a < nfn; ++a) {
      int ra = n2f[fn[a]];
      if (ra < 0) continue;
      rkv.push_back({ra, (int)(P->n_elem_vec + (int64_t)f * nfn + a)});
      for (int b = 0; b < nfn; ++b) {
        int cb = n2f[fn[b]];
        if (cb >= 0)
          kv.push_back({slot_of(ra, cb), (int)(P->n_elem_blocks + (int64_t)f * nfn * nfn + a * nfn + b)});
      }
    }
  }
  std::vector<int> slot_ptr, slot_src, res_ptr, res_src;
  build_csr(P->nnzb, kv, slot_ptr, slot_src);
  build_csr(nf, rkv, res_ptr, res_src);

  // subdomains: free nodes of their elements and sharing counts
  std::vector<std::vector<int>> members(nn);
  for (int e = 0; e < ne; ++e) {
    int p = P->part_h[e];
    for (int a = 0; a < nen; ++a) {
      int v = P->elems_h[(size_t)e * nen + a];
      if (!is_dir[v]) members[v].push_back(p);
    }
  }
  P->share_count.assign(nn, 0);
  for (int v = 0; v < nn; ++v) {
    auto& mv = members[v];
    std::sort(mv.begin(), mv.end());
    mv.erase(std::unique(mv.begin(), mv.end()), mv.end());
    P->share_count[v] = (int)mv.size();
  }
  P->subs.assign(P->n_parts, SubHost{});
  for (int v = 0; v < nn; ++v)
    for (int p : members[v]) {
      P->subs[p].nodes.push_back(v);
      P->subs[p].iface.push_back(P->share_count[v] >= 2 ? 1 : 0);
    }
  for (int p = 0; p < P->n_parts; ++p)
    CB_CHECK(!P->subs[p].nodes.empty(), CBDDC_EINVAL, "subdomain without free nodes");

  // interface classification
  {
    // outer boundary: element faces (by corner nodes) used by one element
    std::vector<char> on_bnd(nn, 0);
    {
      std::vector<std::pair<std::array<int, 4>, int64_t>> fk;
      fk.reserve((size_t)ne * n_lfaces);
      const int c0 = 0, cK = k;
      auto idx = [m](int a, int b, int c) { return a + m * (b + m * c); };
      const int hcorner[6][4] = {
          {idx(c0, c0, c0), idx(c0, cK, c0), idx(c0, cK, cK), idx(c0, c0, cK)},
          {idx(cK, c0, c0), idx(cK, cK, c0), idx(cK, cK, cK), idx(cK, c0, cK)},
          {idx(c0, c0, c0), idx(cK, c0, c0), idx(cK, c0, cK), idx(c0, c0, cK)},
          {idx(c0, cK, c0), idx(cK, cK, c0), idx(cK, cK, cK), idx(c0, cK, cK)},
          {idx(c0, c0, c0), idx(cK, c0, c0), idx(cK, cK, c0), idx(c0, cK, c0)},
          {idx(c0, c0, cK), idx(cK, c0, cK), idx(cK, cK, cK), idx(c0, cK, cK)}};
      // tetrahedron face f: the three vertices other than f (4th key -1)
      const int tcorner[4][4] = {{1, 2, 3, -1}, {0, 2, 3, -1}, {0, 1, 3, -1}, {0, 1, 2, -1}};
      for (int e = 0; e < ne; ++e)
        for (int f = 0; f < n_lfaces; ++f) {
          std::array<int, 4> c;
          for (int q = 0; q < 4; ++q) {
            const int lc = tet ? tcorner[f][q] : hcorner[f][q];
            c[q] = lc < 0 ? -1 : P->elems_h[(size_t)e * nen + lc];
          }
          std::sort(c.begin(), c.end());
          fk.push_back({c, (int64_t)e * n_lfaces + f});
        }
      std::sort(fk.begin(), fk.end());
      for (size_t i = 0; i < fk.size();) {
        size_t j = i;
        while (j < fk.size() && fk[j].first == fk[i].first) ++j;
        if (j - i == 1) {
          int e = (int)(fk[i].second / n_lfaces), f = (int)(fk[i].second % n_lfaces);
          int loc[9];
          face_node_list(tet, k, f, loc);
          for (int a = 0; a < nfn; ++a) on_bnd[P->elems_h[(size_t)e * nen + loc[a]]] = 1;
        }
        i = j;
      }
    }
    std::vector<int> eptr(ne + 1), eidx(P->elems_h.begin(), P->elems_h.end());
    for (int e = 0; e <= ne; ++e) eptr[e] = e * nen;
    classify_interface(nn, members, P->share_count, eptr, eidx, &on_bnd, P->vertices, P->edges, P->faces);
  }

  // subdomain-local slots: elements then pressure faces as contributors
  {
    std::vector<int> cptr{0}, cidx, cpart;
    std::vector<int64_t> cbase;
    for (int e = 0; e < ne; ++e) {
      for (int a = 0; a < nen; ++a) cidx.push_back(P->elems_h[(size_t)e * nen + a]);
      cptr.push_back((int)cidx.size());
      cpart.push_back(P->part_h[e]);
      cbase.push_back((int64_t)e * nen * nen);
    }
    for (int f = 0; f < n_all_faces; ++f) {
      for (int a = 0; a < nfn; ++a) cidx.push_back(face_nodes[(size_t)f * nfn + a]);
      cptr.push_back((int)cidx.size());
      cpart.push_back(P->part_h[face_elem[f]]);
      cbase.push_back(P->n_elem_blocks + (int64_t)f * nfn * nfn);
    }
    build_local_slots(P, cptr, cidx, cpart, cbase);
  }

  // uploads
  std::vector<double> coords(d->coords, d->coords + (size_t)nn * 3);
  P->coords.upload(coords);
  P->coords_h = std::move(coords);
  if (P->fiber_kind == CBDDC_FIBER_NODAL) {
    std::vector<double> fn(d->fiber_nodal, d->fiber_nodal + (size_t)nn * 6);
    for (int v = 0; v < nn; ++v) {
      const double* q = &fn[(size_t)v * 6];
      CB_CHECK(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] > 0.0 && q[3] * q[3] + q[4] * q[4] + q[5] * q[5] > 0.0,
               CBDDC_EINVAL, "zero nodal fibre direction");
    }
    P->fib_nodal.upload(fn);
  }
  P->elems.upload(P->elems_h);
  P->face_nodes.upload(face_nodes);
  P->robin_set.upload(robin_set);
  P->free_nodes.upload(free_nodes);
  P->d_full.alloc((size_t)nn * 3);
  CB_CUDA(cudaMemset(P->d_full.p, 0, P->d_full.bytes()));
  P->contrib.alloc((size_t)(P->n_elem_blocks + P->n_face_blocks) * 9);
  P->rcontrib.alloc((size_t)(P->n_elem_vec + P->n_face_vec) * 3);
  P->bsr_row_ptr.upload(row_ptr);
  P->bsr_col.upload(col);
  P->bsr_vals.alloc((size_t)P->nnzb * 9);
  P->slot_ptr.upload(slot_ptr);
  P->slot_src.upload(slot_src);
  P->res_ptr.upload(res_ptr);
  P->res_src.upload(res_src);
  P->status.alloc(4);
  CB_CUDA(cudaMemset(P->status.p, 0, P->status.bytes()));
  P->scratch.alloc(4096);
  init_shape_tables(P->order);
}

}  // namespace cbddc

int64_t fem_problem::device_bytes() const {
  return (int64_t)(coords.bytes() + fib_nodal.bytes() + elems.bytes() + face_nodes.bytes() + robin_set.bytes() +
                   acc_full.bytes() + vel_full.bytes() + free_nodes.bytes() +
                   d_full.bytes() + contrib.bytes() + rcontrib.bytes() + bsr_row_ptr.bytes() +
                   bsr_col.bytes() + bsr_vals.bytes() + slot_ptr.bytes() + slot_src.bytes() +
                   res_ptr.bytes() + res_src.bytes() + lslot_sub.bytes() + lslot_row.bytes() +
                   lslot_col.bytes() + lslot_ptr.bytes() + lslot_src.bytes() + status.bytes() +
                   scratch.bytes());
}
