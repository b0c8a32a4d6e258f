"""Two-level BDDC preconditioner, Section 3.2 of the paper, applied to the
whole tangent system through the exact interior/interface block
factorization (first display of Section 3.2).

Setup, per subdomain i (the unassembled local matrix A^(i), A = sum A^(i)):
* interior DoFs I (nodes in one subdomain only) and interface DoFs Gamma;
* interface nodes grouped by the set of subdomains sharing them, split into
  connected pieces: faces (shared by 2), edges (shared by 3 or more),
  vertices (single-node edges, and edge nodes lying on the outer boundary,
  which is where the subdomain corners sit when the coordinates are known);
* primal constraints: vertex values ("V"), and edge ("E") or face ("F")
  arithmetic averages per displacement component (Sections 3.2 and 6.2);
  with "R", also the rigid-body rotations of every averaged class (the
  near-null space taken into the primal space, Section 4);
* counting scaling delta_i^dagger = 1 / #subdomains sharing the DoF, or
  deluxe scaling (Section 3.2 names it as the more robust choice): on every
  edge and face class K, D_K^(i) = (sum_j S_K^(j))^-1 S_K^(i) with S_K^(j)
  the class block of subdomain j's Schur complement onto its interface;
  vertex nodes keep the counting weights;
* coarse basis Phi_i: the minimum-energy extension of each primal
  constraint (the local saddle-point problem with unit constraint values),
  and the coarse matrix S_PiPi = sum_i R_Pi^T Phi_i^T A^(i) Phi_i R_Pi.

Apply z = M^-1 r:
  1. u0 = A_II^-1 r_I                           (block diagonal)
  2. g  = r_Gamma - A_GammaI u0                 (assembled on Gamma)
  3. g_i = D_i R_i g      (deluxe: D_K^(i)^T on each class block)
  4. w_i: local Neumann solve with all primal constraints set to zero
     (vertices eliminated, averages through Lagrange multipliers)
  5. u_c = S_PiPi^-1 sum_i R_Pi^T Phi_i^T g_i;   w_i += Phi_i R_Pi u_c
  6. z_Gamma = sum_i R_i^T D_i w_i   (deluxe: D_K^(i) on each class block)
  7. z_I = A_II^-1 (r_I - A_IGamma z_Gamma)
Steps 2-6 are M_BDDC^-1 = R_D^T S~^-1 R_D applied to the Schur complement
system; steps 1 and 7 are the exact outer block factors.

Multilevel BDDC (Section 3.2, last paragraph; Section 7): the coarse
problem is itself an unassembled matrix whose "elements" are the subdomains
with their local coarse matrices; grouping those subdomains into level-2
subdomains and applying BDDC once to it replaces S_PiPi^-1 in step 5.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

# Rotational constraints whose squared singular value falls below this
# fraction of the class's largest are dropped (the rotation about the axis
# of a straight edge leaves every node of the edge in place).
RIGID_DROP = 1e-8


def class_rotations(X):
    """Rotational primal constraints of one interface class with node
    coordinates X (m, 3): the infinitesimal rotations a -> e_k x (x_a - xbar)
    about the class centroid, k = x, y, z, restricted to the class, as
    orthonormal rows of length 3m (node-major, xyz per node).  Rotations
    about the centroid have zero component sums, so the rows are orthogonal
    to the three averages; together the rows span the rigid motions of the
    class (Section 4, rigid motions as primal degrees of freedom)."""
    X = np.asarray(X, dtype=float)
    y = X - X.mean(axis=0)
    R = np.zeros((3 * len(X), 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        R[:, k] = np.cross(e, y).reshape(-1)
    U, s, _ = np.linalg.svd(R, full_matrices=False)
    if s.size == 0 or s[0] == 0.0:
        return np.zeros((0, 3 * len(X)))
    keep = s ** 2 >= RIGID_DROP * s[0] ** 2
    return U[:, keep].T


def outer_boundary_nodes(fe):
    """Nodes lying on element faces that belong to one element only."""
    from .elements import corner_faces, face_nodes
    et = fe.prob["elem_type"]
    keys = {}
    for f, cn in enumerate(corner_faces(et)):
        fk = np.sort(fe.elems[:, cn], axis=1)
        for e in range(fe.n_el):
            keys.setdefault(tuple(fk[e]), []).append((e, f))
    on = np.zeros(fe.n_nodes, dtype=bool)
    for lst in keys.values():
        if len(lst) == 1:
            e, f = lst[0]
            on[fe.elems[e, face_nodes(et, f)]] = True
    return on


class FineLevel:
    """The fine level of BDDC: element and face matrices of the FE problem.

    Nodes carry 3 DoFs; Dirichlet nodes carry none.  ``elem_nodes`` and
    ``part`` define subdomain membership and node adjacency."""

    def __init__(self, fe, Ke, Kf):
        self.fe = fe
        self.Ke, self.Kf = Ke, Kf
        self.n_nodes = fe.n_nodes
        self.free = ~fe.is_dirichlet
        self.node_to_free = fe.node_to_free
        self.n_free = fe.n_free
        self.elem_nodes = fe.elems
        self.part = np.asarray(fe.prob["elem_part"], dtype=np.int64)
        self.n_parts = int(fe.prob["n_parts"])
        self.on_boundary = outer_boundary_nodes(fe)

    def local_matrix(self, i, dof_map, n):
        return self.fe.assemble(self.Ke, self.Kf, self.part == i, dof_map, n)


class CoarseLevel:
    """The coarse problem of a BDDC level seen as an unassembled matrix:
    its nodes are the coarse nodes (a primal vertex, or an averaged class,
    each with 3 DoFs), its "elements" are the subdomains of the finer level
    with their local coarse matrices Phi_i^T A^(i) Phi_i, and ``part``
    groups those subdomains into the subdomains of this level (Section 3.2,
    multilevel BDDC)."""

    def __init__(self, n_nodes, elem_nodes, elem_K, part, n_parts):
        self.n_nodes = int(n_nodes)
        self.free = np.ones(self.n_nodes, dtype=bool)
        self.node_to_free = np.arange(self.n_nodes)
        self.n_free = 3 * self.n_nodes
        self.elem_nodes = [np.asarray(e, dtype=np.int64) for e in elem_nodes]
        self.elem_K = elem_K
        self.part = np.asarray(part, dtype=np.int64)
        self.n_parts = int(n_parts)
        self.on_boundary = None

    def local_matrix(self, i, dof_map, n):
        rows, cols, vals = [], [], []
        for e in np.nonzero(self.part == i)[0]:
            nodes = self.elem_nodes[e]
            gd = (3 * nodes[:, None] + np.arange(3)).reshape(-1)
            m = dof_map[gd]
            K = self.elem_K[e]
            rows.append(np.repeat(m, m.size))
            cols.append(np.tile(m, m.size))
            vals.append(K.reshape(-1))
        A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(n, n))
        return A.tocsr()


class Classification:
    """Interface classes (faces, edges, vertices) of a partition."""

    def __init__(self, level, elem_part=None, n_parts=None):
        if not isinstance(level, (FineLevel, CoarseLevel)):
            # FE problem given directly: classify its elements
            fe = level
            level = FineLevel.__new__(FineLevel)
            level.n_nodes = fe.n_nodes
            level.free = ~fe.is_dirichlet
            level.elem_nodes = fe.elems
            level.part = np.asarray(elem_part, dtype=np.int64)
            level.n_parts = int(n_parts)
            level.on_boundary = outer_boundary_nodes(fe)
        self.n_parts = level.n_parts
        part = level.part
        n = level.n_nodes
        memb = [set() for _ in range(n)]
        for e, nodes in enumerate(level.elem_nodes):
            p = int(part[e])
            for a in nodes:
                memb[a].add(p)
        self.members = [tuple(sorted(s)) if level.free[a] else ()
                        for a, s in enumerate(memb)]
        self.count = np.array([len(s) for s in self.members])
        iface = self.count >= 2
        self.interface = iface
        key_of = {}
        key = -np.ones(n, dtype=np.int64)
        for a in np.nonzero(iface)[0]:
            key[a] = key_of.setdefault(self.members[a], len(key_of))
        if isinstance(level.elem_nodes, np.ndarray) and level.elem_nodes.ndim == 2:
            en = level.elem_nodes
            ii = np.repeat(en, en.shape[1], axis=1).reshape(-1)
            jj = np.tile(en, (1, en.shape[1])).reshape(-1)
        else:
            ii, jj = [], []
            for nodes in level.elem_nodes:
                nodes = np.asarray(nodes)
                ii.append(np.repeat(nodes, nodes.size))
                jj.append(np.tile(nodes, nodes.size))
            ii = np.concatenate(ii)
            jj = np.concatenate(jj)
        same = (key[ii] >= 0) & (key[ii] == key[jj])
        G = sp.coo_matrix((np.ones(same.sum()), (ii[same], jj[same])), shape=(n, n))
        ncomp, comp = csg.connected_components(G, directed=False)
        on_bnd = level.on_boundary
        classes = {}
        for a in np.nonzero(iface)[0]:
            classes.setdefault(int(comp[a]), []).append(int(a))
        vertices, edges, faces = [], [], []
        for nodes in classes.values():
            s = self.members[nodes[0]]
            if len(s) == 2:
                faces.append(sorted(nodes))
            elif len(nodes) == 1:
                vertices.append(nodes[0])
            else:
                ends = [a for a in nodes if on_bnd is not None and on_bnd[a]]
                vertices.extend(ends)
                rest = sorted(a for a in nodes if on_bnd is None or not on_bnd[a])
                if rest:
                    edges.append(rest)
        self.vertices = sorted(vertices)
        self.edges = sorted(edges)
        self.faces = sorted(faces)


class BDDC:
    """BDDC setup for one tangent.

    ``fe, Ke, Kf``: the FE problem and its element / face matrices (the fine
    level), or a ``CoarseLevel`` as first argument (then Ke, Kf are unused).
    ``level2``: None for the two-level method; otherwise a dict with
    ``part`` (level-2 subdomain of every subdomain of this level),
    ``n_parts`` and ``primal``: the coarse problem is then approximated by
    one application of BDDC on those level-2 subdomains (multilevel BDDC,
    Section 3.2); a nested ``level2`` entry adds a further level.
    ``primal`` holds the letters V, E, F and R (rotations of the averaged
    classes, fine level of a two-level method only: the rotations need node
    coordinates, and a coarse node of the multilevel method carries 3 DoFs).
    ``scaling``: "counting" or "deluxe" on this level (a level-2 method
    takes its own from ``level2["scaling"]``, counting by default).
    ``coarse``: "galerkin" uses the one basis Phi (minimum energy for A) on
    both sides of the coarse problem, Phi^T A Phi; "petrov" is the
    nonsymmetric BDDC with a left basis Psi, the same construction for A^T:
    coarse matrix Psi^T A Phi and coarse right-hand side Psi^T g_i (the two
    agree for a symmetric tangent)."""

    def __init__(self, fe, Ke=None, Kf=None, primal="V", classification=None, level2=None,
                 scaling="counting", coarse="galerkin"):
        if scaling not in ("counting", "deluxe"):
            raise ValueError("scaling is 'counting' or 'deluxe'")
        if coarse not in ("galerkin", "petrov"):
            raise ValueError("coarse is 'galerkin' or 'petrov'")
        self.scaling = scaling
        self.coarse_kind = coarse
        level = fe if isinstance(fe, CoarseLevel) else FineLevel(fe, Ke, Kf)
        self.level = level
        cl = classification or Classification(level)
        self.cl = cl
        use_v = "V" in primal
        use_r = "R" in primal
        if use_r and (not isinstance(level, FineLevel) or level2 is not None):
            raise ValueError("rigid-body constraints need a two-level method on the fine level")
        avg_classes = []
        if "E" in primal:
            avg_classes += cl.edges
        if "F" in primal:
            avg_classes += cl.faces
        rot = [class_rotations(level.fe.coords[c]) if use_r else np.zeros((0, 3 * len(c)))
               for c in avg_classes]
        # global primal numbering: vertex DoFs, then per class its 3 averages
        # and its rotations
        vert = cl.vertices if use_v else []
        ncls = [3 + r.shape[0] for r in rot]
        self.n_pi = 3 * len(vert) + int(sum(ncls))
        vpos = {a: 3 * j for j, a in enumerate(vert)}
        apos = list(3 * len(vert) + np.concatenate([[0], np.cumsum(ncls)[:-1]]).astype(int)) \
            if avg_classes else []
        node_class = {}
        for j, c in enumerate(avg_classes):
            for a in c:
                node_class[a] = j
        self.subs = []
        n2f = level.node_to_free
        part = level.part
        elem_nodes = level.elem_nodes
        sub_nodes = [set() for _ in range(level.n_parts)]
        for e, nodes in enumerate(elem_nodes):
            sub_nodes[int(part[e])].update(int(a) for a in nodes)
        Sc_list = []
        for i in range(level.n_parts):
            nodes = np.array(sorted(sub_nodes[i]), dtype=np.int64)
            nodes = nodes[level.free[nodes]]
            nloc = nodes.size
            dof_map = -np.ones(3 * level.n_nodes, dtype=np.int64)
            for c in range(3):
                dof_map[3 * nodes + c] = 3 * np.arange(nloc) + c
            A = level.local_matrix(i, dof_map, 3 * nloc).tocsr()
            gdof = (3 * n2f[nodes][:, None] + np.arange(3)).reshape(-1)
            iface = cl.count[nodes] >= 2
            ldofI = (3 * np.nonzero(~iface)[0][:, None] + np.arange(3)).ravel()
            ldofG = (3 * np.nonzero(iface)[0][:, None] + np.arange(3)).ravel()
            Dg = np.repeat(1.0 / cl.count[nodes[iface]], 3)
            # primal vertex DoFs (local) and remaining DoFs r
            is_v = np.array([use_v and a in vpos for a in nodes], dtype=bool)
            ldofV = (3 * np.nonzero(is_v)[0][:, None] + np.arange(3)).ravel()
            gV = np.array([vpos[a] + c for a in nodes[is_v] for c in range(3)],
                          dtype=np.int64)
            keep = np.ones(3 * nloc, dtype=bool)
            keep[ldofV] = False
            ldofR = np.nonzero(keep)[0]
            rpos = -np.ones(3 * nloc, dtype=np.int64)
            rpos[ldofR] = np.arange(ldofR.size)
            # averages touching this subdomain
            loc_cls = sorted({node_class[a] for a in nodes if a in node_class})
            rows, cols, vals, gA = [], [], [], []
            for j in loc_cls:
                cnodes = avg_classes[j]
                lidx = np.searchsorted(nodes, cnodes)
                for c in range(3):
                    for li in lidx:
                        rows.append(len(gA))
                        cols.append(rpos[3 * li + c])
                        vals.append(1.0 / len(cnodes))
                    gA.append(apos[j] + c)
                ldof = (3 * lidx[:, None] + np.arange(3)).reshape(-1)
                for k, w in enumerate(rot[j]):
                    rows.extend([len(gA)] * w.size)
                    cols.extend(rpos[ldof])
                    vals.extend(w)
                    gA.append(apos[j] + 3 + k)
            na = len(gA)
            Cr = sp.coo_matrix((vals, (rows, cols)),
                               shape=(na, ldofR.size)).tocsr()
            Krr = A[ldofR][:, ldofR]
            sad = sp.bmat([[Krr, Cr.T], [Cr, None]], format="csc") if na else \
                Krr.tocsc()
            lu_sad = spla.splu(sad)
            # coarse basis: vertex columns then average columns
            nv = ldofV.size
            nc = nv + na
            Phi = np.zeros((3 * nloc, nc))
            if nc:
                rhs = np.zeros((ldofR.size + na, nc))
                if nv:
                    rhs[:ldofR.size, :nv] = -A[ldofR][:, ldofV].toarray()
                    Phi[ldofV, np.arange(nv)] = 1.0
                if na:
                    rhs[ldofR.size:, nv:] = np.eye(na)
                sol = lu_sad.solve(rhs)
                Phi[ldofR, :] = sol[:ldofR.size]
                gP = np.concatenate([gV, np.array(gA, dtype=np.int64)])
                Psi = Phi
                if coarse == "petrov":
                    # left basis: the same saddle problem for A^T
                    AT = A.T.tocsr()
                    sadT = sp.bmat([[AT[ldofR][:, ldofR], Cr.T], [Cr, None]], format="csc") \
                        if na else AT[ldofR][:, ldofR].tocsc()
                    rhsT = np.zeros((ldofR.size + na, nc))
                    Psi = np.zeros((3 * nloc, nc))
                    if nv:
                        rhsT[:ldofR.size, :nv] = -AT[ldofR][:, ldofV].toarray()
                        Psi[ldofV, np.arange(nv)] = 1.0
                    if na:
                        rhsT[ldofR.size:, nv:] = np.eye(na)
                    Psi[ldofR, :] = spla.splu(sadT).solve(rhsT)[:ldofR.size]
                Sc = Psi.T @ (A @ Phi)
            else:
                gP = np.zeros(0, dtype=np.int64)
                Sc = np.zeros((0, 0))
                Psi = Phi
            Sc_list.append(Sc)
            AII = A[ldofI][:, ldofI].tocsc()
            sub = dict(nodes=nodes, A=A, gdof=gdof, ldofI=ldofI, ldofG=ldofG,
                       ldofR=ldofR, Dg=Dg, lu_sad=lu_sad, na=na, Phi=Phi, Psi=Psi,
                       gP=gP, Sc=Sc,
                       luII=spla.splu(AII) if ldofI.size else None,
                       AGI=A[ldofG][:, ldofI], AIG=A[ldofI][:, ldofG])
            self.subs.append(sub)
        self.n_free = level.n_free
        if scaling == "deluxe":
            self._setup_deluxe(cl)
        self.coarse = None
        if level2 is not None and self.n_pi > 0:
            # coarse nodes: 3 consecutive primal DoFs each (node-major)
            clevel = CoarseLevel(self.n_pi // 3, [sub["gP"][::3] // 3 for sub in self.subs],
                                 Sc_list, level2["part"], level2["n_parts"])
            self.coarse = BDDC(clevel, primal=level2.get("primal", "VEF"),
                               level2=level2.get("level2"),
                               scaling=level2.get("scaling", "counting"),
                               coarse=level2.get("coarse", coarse))
            self.S_pipi = None
        else:
            S = np.zeros((self.n_pi, self.n_pi))
            for sub in self.subs:
                if sub["gP"].size:
                    S[np.ix_(sub["gP"], sub["gP"])] += sub["Sc"]
            self.S_pipi = S

    def _setup_deluxe(self, cl):
        """Deluxe scaling: for every edge and face class K and every
        subdomain i sharing it, the block S_K^(i) of the local Schur
        complement S_i = A_GG - A_GI A_II^-1 A_IG on the class DoFs, and
        D_K^(i) = (sum_j S_K^(j))^-1 S_K^(i).  Each subdomain gets
        ``deluxe``: a list of (positions of the class DoFs in its interface
        vector, D_K^(i)); the counting weight of those DoFs becomes 1."""
        blocks = {}
        for i, sub in enumerate(self.subs):
            A = sub["A"]
            AGG = A[sub["ldofG"]][:, sub["ldofG"]].toarray()
            if sub["luII"] is not None:
                S = AGG - sub["AGI"] @ sub["luII"].solve(sub["AIG"].toarray())
            else:
                S = AGG
            sub["S"] = S
            sub["deluxe"] = []
            nodes = sub["nodes"]
            for k, cls in enumerate(cl.edges + cl.faces):
                li = np.searchsorted(nodes, cls)
                if li[0] >= nodes.size or nodes[li[0]] != cls[0]:
                    continue
                ldof = (3 * li[:, None] + np.arange(3)).reshape(-1)
                pos = np.searchsorted(sub["ldofG"], ldof)
                blocks.setdefault(k, []).append((i, pos, S[np.ix_(pos, pos)]))
        for k, lst in blocks.items():
            Shat = sum(Sk for _, _, Sk in lst)
            for i, pos, Sk in lst:
                D = np.linalg.solve(Shat, Sk)
                sub = self.subs[i]
                sub["deluxe"].append((pos, D))
                sub["Dg"][pos] = 1.0

    def _local_solve(self, sub, f_loc):
        """Constrained Neumann solve with zero primal values: w_v = 0,
        C_r w_r = 0, [A_rr C_r^T; C_r 0][w_r; mu] = [f_r; 0]."""
        rhs = np.concatenate([f_loc[sub["ldofR"]], np.zeros(sub["na"])])
        sol = sub["lu_sad"].solve(rhs)
        w = np.zeros(f_loc.size)
        w[sub["ldofR"]] = sol[:sub["ldofR"].size]
        return w

    def coarse_solve(self, c):
        """S_PiPi^-1 c (two levels), or one BDDC application on the coarse
        problem (multilevel)."""
        if c.size == 0:
            return c
        if self.coarse is not None:
            return self.coarse.apply(c)
        return np.linalg.solve(self.S_pipi, c)

    def apply(self, r):
        r = np.asarray(r, dtype=float)
        z = np.zeros_like(r)
        g = r.copy()
        u0 = []
        for sub in self.subs:
            gd = sub["gdof"]
            if sub["luII"] is not None:
                u = sub["luII"].solve(r[gd[sub["ldofI"]]])
                g[gd[sub["ldofG"]]] -= sub["AGI"] @ u
            else:
                u = np.zeros(0)
            u0.append(u)
        c = np.zeros(self.n_pi)
        ws = []
        for sub in self.subs:
            gd = sub["gdof"]
            f = np.zeros(gd.size)
            fG = sub["Dg"] * g[gd[sub["ldofG"]]]
            for pos, D in sub.get("deluxe", ()):
                fG[pos] = D.T @ fG[pos]
            f[sub["ldofG"]] = fG
            w = self._local_solve(sub, f)
            if sub["gP"].size:
                np.add.at(c, sub["gP"], sub["Psi"].T @ f)
            ws.append(w)
        uc = self.coarse_solve(c)
        zG = np.zeros_like(r)
        for sub, w in zip(self.subs, ws):
            gd = sub["gdof"]
            if sub["gP"].size:
                w = w + sub["Phi"] @ uc[sub["gP"]]
            yG = sub["Dg"] * w[sub["ldofG"]]
            for pos, D in sub.get("deluxe", ()):
                yG[pos] = D @ yG[pos]
            np.add.at(zG, gd[sub["ldofG"]], yG)
        z[:] = zG
        for sub, u in zip(self.subs, u0):
            gd = sub["gdof"]
            if sub["luII"] is not None:
                zI = sub["luII"].solve(r[gd[sub["ldofI"]]]
                                       - sub["AIG"] @ zG[gd[sub["ldofG"]]])
                z[gd[sub["ldofI"]]] = zI
        return z
