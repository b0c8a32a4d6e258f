"""Idealised left ventricle: a truncated prolate-ellipsoid shell meshed with
linear (P1) or quadratic (P2) tetrahedra, and its partition.

The paper's swelling and contraction tests run on an ellipsoidal left
ventricle (Section 5); its mesh is not available, so this procedural shell
stands in for it.  Geometry in metres:
* endocardium: semi-axes (a_endo, a_endo, c_endo), epicardium
  (a_epi, a_epi, c_epi); the shell is the part z <= 0, the base plane z = 0
  is clamped;
* node (t, theta, u): transmural t in [0, 1] (0 = endocardium), angle theta,
  longitudinal u in (0, 1] (u = 1 at the base); radii a(t) = a_endo +
  t (a_epi - a_endo), c(t) likewise, polar angle psi = u pi / 2 from the
  apex: X = (a sin(psi) cos(theta), a sin(psi) sin(theta), -c cos(psi)); the
  apex (u = 0) is one node per transmural layer;
* the surface is triangulated ring by ring, the rings' node counts halved
  towards the apex (``ring_sizes``) so that no element degenerates there,
  and every surface triangle is extruded through the wall into prisms cut
  into 3 tetrahedra (``_prisms_to_tets``);
* fibres (nodal input field): the helix angle falls linearly from
  +alpha at the endocardium to -alpha at the epicardium,
  f = cos(a) e_circ + sin(a) e_long, n = outward normal of the ellipsoid
  through the node (transmural direction); P2 edge midpoints take the
  normalised mean of their end nodes' directions;
* partition: surface patches x transmural slabs.  The surface triangles are
  cut by recursive coordinate bisection of their parametric centroids
  (theta, u), scaled to mid-wall lengths, with target weights drawn
  U[1 - w, 1 + w] (seeded) and repaired so that every patch is connected;
  each patch times a range of element layers is a subdomain.  Nested: the
  level-2 subdomains are groups of whole patches (all slabs).

Local numbering of a tetrahedron: vertices 0..3; P2 adds edge midpoints in
the order (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  Local face f is the
face opposite vertex f.
"""
import numpy as np

from .material import default_material, GAMMA_MAX

TET_EDGES = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]


def ring_sizes(ntheta, nu):
    """Nodes per ring: ntheta, halved towards the apex (ntheta / 2^m, m as
    large as divisibility allows) while the circumferential spacing stays
    at least the longitudinal one, 2 pi (k + 1) / N_k >= 1 near the apex."""
    Nk = np.empty(nu, dtype=np.int64)
    for k in range(nu):
        n = ntheta
        while n % 2 == 0 and n // 2 >= 3 and 2 * np.pi * (k + 1) / (n // 2) <= 1.0 + 1e-12:
            n //= 2
        Nk[k] = n
    # a ring never has fewer nodes than the one inside it
    for k in range(1, nu):
        Nk[k] = max(Nk[k], Nk[k - 1])
    return Nk


def _surface_triangles(Nk, first):
    """Triangulation of the parametric surface: a fan from the apex to ring
    0, then the bands between rings (two triangles per quad between rings
    of equal size, three per coarse node where the size doubles)."""
    tri = []
    n0 = Nk[0]
    r0 = 1 + first[0]
    for j in range(n0):
        tri.append((0, r0 + j, r0 + (j + 1) % n0))
    for k in range(len(Nk) - 1):
        a0, b0 = 1 + first[k], 1 + first[k + 1]
        n, m = Nk[k], Nk[k + 1]
        if m == n:
            for j in range(n):
                p, q = a0 + j, a0 + (j + 1) % n
                r, w = b0 + j, b0 + (j + 1) % n
                tri += [(p, r, w), (p, w, q)]
        else:
            assert m == 2 * n, "ring sizes must stay equal or double"
            for j in range(n):
                p, q = a0 + j, a0 + (j + 1) % n
                c, d, e = b0 + 2 * j, b0 + 2 * j + 1, b0 + (2 * j + 2) % m
                tri += [(p, c, d), (p, d, q), (q, d, e)]
    return np.array(tri, dtype=np.int64)


def _prisms_to_tets(tri, nt):
    """Extrude each surface triangle through the nt - 1 transmural layers and
    cut every prism into 3 tetrahedra.  Each quadrilateral side is cut along
    the diagonal through its smallest node id, which both prisms sharing it
    agree on, so the mesh is conforming: with the prism rotated so that its
    smallest node is vertex 0 of the bottom (0,1,2) / top (3,4,5), the tets
    are [0,3,4,5] and, by the diagonal of side (1,2,5,4), either [0,1,2,5],
    [0,1,5,4] or [0,1,2,4], [0,2,5,4]."""
    layers = np.arange(nt - 1)
    bot = (tri[:, None, :] * nt + layers[None, :, None]).reshape(-1, 3)
    pr = np.concatenate([bot, bot + 1], axis=1)            # (n, 6)
    v = np.argmin(pr, axis=1)
    rot = np.array([[0, 1, 2, 3, 4, 5], [1, 2, 0, 4, 5, 3], [2, 0, 1, 5, 3, 4],
                    [3, 4, 5, 0, 1, 2], [4, 5, 3, 1, 2, 0], [5, 3, 4, 2, 0, 1]])
    q = np.take_along_axis(pr, rot[v], axis=1)
    side = q[:, [1, 2, 5, 4]]
    d15 = np.isin(np.argmin(side, axis=1), (0, 2))          # min at 1 or 5
    t1 = q[:, [0, 3, 4, 5]]
    t2 = np.where(d15[:, None], q[:, [0, 1, 2, 5]], q[:, [0, 1, 2, 4]])
    t3 = np.where(d15[:, None], q[:, [0, 1, 5, 4]], q[:, [0, 2, 5, 4]])
    return np.stack([t1, t2, t3], axis=1).reshape(-1, 4)


def lv_problem(nt=3, ntheta=16, nu=8, order=1, a_endo=0.025, c_endo=0.070,
               a_epi=0.035, c_epi=0.080, jitter=0.15, seed=2208, n_parts=8,
               n_parts2=None, n_layers=1, weight_spread=0.3, part_seed=6191,
               pressure=2.0e3, gamma=0.5 * GAMMA_MAX, alpha_deg=60.0,
               load_steps=4, primal="VEF", material=None):
    """P1/P2 tetrahedral mesh of the ventricle shell with nt transmural,
    ntheta circumferential and nu longitudinal node layers (u > 0), plus one
    apex node per transmural layer; n_parts = (surface patches) x n_layers
    transmural slabs (n_layers divides nt - 1).  Also
    apex node per transmural layer."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, nt)
    u = np.linspace(0.0, 1.0, nu + 1)[1:]
    Nk = ring_sizes(ntheta, nu)
    # surface vertices: 0 = apex, then ring k vertex j at 1 + first[k] + j;
    # node id = surface vertex * nt + transmural layer i
    first = np.concatenate([[0], np.cumsum(Nk)[:-1]])
    n_sv = 1 + int(Nk.sum())
    n_nodes = n_sv * nt
    P = np.zeros((n_nodes, 3))   # parametric (t, theta, u)
    P[:nt, 0] = t
    sv_th = np.zeros(n_sv)
    sv_u = np.zeros(n_sv)
    sv_k = -np.ones(n_sv, dtype=np.int64)
    for k in range(nu):
        sl = slice(1 + first[k], 1 + first[k] + Nk[k])
        sv_th[sl] = np.arange(Nk[k]) * (2 * np.pi / Nk[k])
        sv_u[sl] = u[k]
        sv_k[sl] = k
    P[:, 0] = np.tile(t, n_sv)
    P[:, 1] = np.repeat(sv_th, nt)
    P[:, 2] = np.repeat(sv_u, nt)
    P0 = P.copy()
    # jitter in parametric space: interior nodes in (t, theta, u), surface
    # nodes in (theta, u); the apex and the base ring stay put
    if jitter > 0:
        dth = np.repeat(np.where(sv_k >= 0, 2 * np.pi / Nk[np.maximum(sv_k, 0)], 0.0), nt)
        movable = np.repeat((sv_k >= 0) & (sv_k < nu - 1), nt)
        layer = np.tile(np.arange(nt), n_sv)
        inner = movable & (layer > 0) & (layer < nt - 1)
        J = rng.uniform(-jitter, jitter, (n_nodes, 3)) * np.stack(
            [np.full(n_nodes, 1.0 / max(nt - 1, 1)), dth, np.full(n_nodes, 1.0 / nu)], axis=1)
        P[inner] += J[inner]
        P[movable & ~inner, 1:] += J[movable & ~inner, 1:]

    def to_xyz(tt, tht, uu):
        a = a_endo + tt * (a_epi - a_endo)
        c = c_endo + tt * (c_epi - c_endo)
        psi = uu * np.pi / 2
        return np.stack([a * np.sin(psi) * np.cos(tht), a * np.sin(psi) * np.sin(tht),
                         -c * np.cos(psi)], axis=-1)

    X = to_xyz(P[:, 0], P[:, 1], P[:, 2])
    X[np.abs(P[:, 2] - 1.0) < 1e-12, 2] = 0.0  # base plane exactly at z = 0
    tri = _surface_triangles(Nk, first)
    tets = _prisms_to_tets(tri, nt)
    # positive orientation, decided on the unjittered mesh; the jittered
    # one must keep every element positive (no silent re-orientation, which
    # would hide a tangled element)
    def signed_vol(Y):
        v = Y[tets]
        return np.einsum("ij,ij->i", np.cross(v[:, 1] - v[:, 0], v[:, 2] - v[:, 0]), v[:, 3] - v[:, 0])
    neg = signed_vol(to_xyz(P0[:, 0], P0[:, 1], P0[:, 2])) < 0
    tets[neg, 1], tets[neg, 2] = tets[neg, 2].copy(), tets[neg, 1].copy()
    if np.any(signed_vol(X) <= 0):
        raise ValueError("jitter %.3g tangles the mesh; use a smaller value" % jitter)
    # nodal fibres: helix angle alpha(t) from +alpha at t=0 to -alpha at t=1
    alpha = np.deg2rad(alpha_deg) * (1.0 - 2.0 * P[:, 0])
    th_n, psi = P[:, 1], P[:, 2] * np.pi / 2
    e_circ = np.stack([-np.sin(th_n), np.cos(th_n), np.zeros_like(th_n)], axis=1)
    a_n = a_endo + P[:, 0] * (a_epi - a_endo)
    c_n = c_endo + P[:, 0] * (c_epi - c_endo)
    e_long = np.stack([a_n * np.cos(psi) * np.cos(th_n), a_n * np.cos(psi) * np.sin(th_n),
                       c_n * np.sin(psi)], axis=1)
    e_long /= np.linalg.norm(e_long, axis=1)[:, None]
    fib = np.cos(alpha)[:, None] * e_circ + np.sin(alpha)[:, None] * e_long
    # transmural direction: outward normal of the ellipsoid through the node
    nrm = np.stack([X[:, 0] / a_n ** 2, X[:, 1] / a_n ** 2, X[:, 2] / c_n ** 2], axis=1)
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    t_node = P[:, 0]
    # P2: edge midpoints, numbered in order of first appearance
    if order == 2:
        ends = np.sort(np.stack([tets[:, [a for a, _ in TET_EDGES]], tets[:, [b for _, b in TET_EDGES]]],
                                axis=2), axis=2).reshape(-1, 2)
        uniq, first_pos, inv = np.unique(ends, axis=0, return_index=True, return_inverse=True)
        rank = np.empty(uniq.shape[0], dtype=np.int64)
        rank[np.argsort(first_pos, kind="stable")] = np.arange(uniq.shape[0])
        mids = uniq[np.argsort(rank)]
        elems = np.concatenate([tets, n_nodes + rank[inv.reshape(-1)].reshape(-1, 6)], axis=1)
        X = np.concatenate([X, 0.5 * (X[mids[:, 0]] + X[mids[:, 1]])])
        t_node = np.concatenate([t_node, 0.5 * (t_node[mids[:, 0]] + t_node[mids[:, 1]])])
        fm = fib[mids[:, 0]] + fib[mids[:, 1]]
        nm = nrm[mids[:, 0]] + nrm[mids[:, 1]]
        fib = np.concatenate([fib, fm / np.linalg.norm(fm, axis=1)[:, None]])
        nrm = np.concatenate([nrm, nm / np.linalg.norm(nm, axis=1)[:, None]])
        n_nodes = X.shape[0]
    else:
        elems = tets
    # boundary sets: the base plane is clamped; the pressure acts on the
    # element faces whose three vertices lie on the endocardium (t = 0)
    base = np.nonzero(np.abs(X[:, 2]) < 1e-12)[0]
    endo_node = np.abs(t_node) < 1e-12
    faces = []
    for f in range(4):
        vs = [q for q in range(4) if q != f]
        on = np.all(endo_node[tets[:, vs]], axis=1)
        faces.append(np.stack([np.nonzero(on)[0], np.full(on.sum(), f)], axis=1))
    pressure_faces = np.concatenate(faces)
    pressure_faces = pressure_faces[np.lexsort((pressure_faces[:, 1], pressure_faces[:, 0]))]
    # partition: surface patches of triangles (bisection of their parametric
    # centroids, circular mean in theta with the apex left out) times
    # transmural slabs of element layers
    tri_ring = sv_k[tri] >= 0
    cth = np.where(tri_ring, np.cos(sv_th[tri]), 0.0).sum(1)
    sth = np.where(tri_ring, np.sin(sv_th[tri]), 0.0).sum(1)
    tri_th = np.mod(np.arctan2(sth, cth), 2 * np.pi)
    tri_u = sv_u[tri].mean(1)
    if n_parts % n_layers or (nt - 1) % n_layers:
        raise ValueError("n_layers must divide n_parts and nt - 1")
    n_surf = n_parts // n_layers
    n_surf2 = None if n_parts2 is None else n_parts2
    spart, sgroup = _partition(np.stack([tri_th, tri_u], axis=1), n_surf, n_surf2, weight_spread,
                               part_seed, (a_endo + a_epi) / 2, (c_endo + c_epi) / 2)
    spart = _make_connected(spart, _triangle_adjacency(tri))
    slab = np.arange(nt - 1) // ((nt - 1) // n_layers)
    part = (spart[:, None] * n_layers + slab[None, :]).reshape(-1)   # per prism
    part = np.repeat(part, 3)                                        # per tet
    part2, n2 = None, None
    if sgroup is not None:
        part2 = np.repeat(sgroup, n_layers)
        n2 = n_parts2
    prob = {
        "elem_type": "P1" if order == 1 else "P2",
        "coords": X,
        "elems": elems.astype(np.int32),
        "elem_part": part.astype(np.int32),
        "n_parts": int(n_parts),
        "dirichlet_nodes": base.astype(np.int32),
        "pressure_faces": pressure_faces.astype(np.int32),
        "fibers": {"kind": "nodal", "f": fib, "n": nrm},
        "material": dict(material or default_material()),
        "pressure": float(pressure),
        "gamma": float(gamma),
        "load_steps": int(load_steps),
        "primal": primal,
    }
    if part2 is not None:
        prob["part2"] = part2.astype(np.int32)
        prob["n_parts2"] = int(n2)
    return prob


def _rcb(coords, idx, weights, out, base):
    """Recursive coordinate bisection of elements idx into len(weights) parts
    with the given target weights; part ids base, base+1, ..."""
    k = len(weights)
    if k == 1:
        out[idx] = base
        return
    k1 = k // 2
    w1 = sum(weights[:k1]) / sum(weights)
    pts = coords[idx]
    span = pts.max(axis=0) - pts.min(axis=0)
    ax = int(np.argmax(span))
    order = np.argsort(pts[:, ax], kind="stable")
    cut = int(round(w1 * idx.size))
    cut = min(max(cut, 1), idx.size - 1)
    _rcb(coords, idx[order[:cut]], weights[:k1], out, base)
    _rcb(coords, idx[order[cut:]], weights[k1:], out, base + k1)


def _triangle_adjacency(tri):
    """Pairs of surface triangles sharing an edge."""
    import scipy.sparse as sp
    n_tri = tri.shape[0]
    e = np.sort(np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]]), axis=1)
    owner = np.tile(np.arange(n_tri), 3)
    order = np.lexsort((e[:, 1], e[:, 0]))
    e, owner = e[order], owner[order]
    same = np.all(e[1:] == e[:-1], axis=1)
    a, b = owner[:-1][same], owner[1:][same]
    return sp.coo_matrix((np.ones(a.size), (a, b)), shape=(n_tri, n_tri)).tocsr()


def _make_connected(part, adj, max_rounds=20):
    """Moves every piece of a part that is not its largest connected piece
    to the neighbouring part it shares the most faces with, until each part
    is connected (bisection by centroids can leave single columns cut off)."""
    import scipy.sparse as sp
    import scipy.sparse.csgraph as csg
    part = part.copy()
    A = adj.tocoo()
    for _ in range(max_rounds):
        keep = part[A.row] == part[A.col]
        G = sp.coo_matrix((np.ones(keep.sum()), (A.row[keep], A.col[keep])), shape=adj.shape)
        _, lab = csg.connected_components(G, directed=False)
        # largest piece of each part
        order = np.lexsort((lab, part))
        moved = False
        best = {}
        labs, counts = np.unique(lab, return_counts=True)
        size = dict(zip(labs.tolist(), counts.tolist()))
        for q, l in zip(part[order].tolist(), lab[order].tolist()):
            if q not in best or size[l] > size[best[q]]:
                best[q] = l
        stray = np.array([lab[i] != best[part[i]] for i in range(part.size)])
        if not stray.any():
            return part
        for l in np.unique(lab[stray]):
            members = np.nonzero(lab == l)[0]
            nb = adj[members].indices
            nbp = part[nb]
            nbp = nbp[nbp != part[members[0]]]
            if nbp.size:
                part[members] = np.bincount(nbp).argmax()
                moved = True
        if not moved:
            break
    raise ValueError("could not make every subdomain connected")


def _partition(par, n_parts, n_parts2, spread, seed, a_mid, c_mid):
    """Recursive coordinate bisection of the surface triangles (parametric
    centroids par = (theta, u)) into n_parts patches with target weights
    U[1 - spread, 1 + spread]; with n_parts2, first into n_parts2 groups
    (weights: sums of their members) and each group into its patches.
    Returns (patch per triangle, group per patch or None)."""
    rng = np.random.default_rng(seed)
    # coordinates scaled to lengths on the mid-wall surface: circumference
    # r(u) theta and meridian arc length (quarter ellipse) times u
    r = a_mid * np.sin(par[:, 1] * np.pi / 2)
    arc = np.pi / 2 * np.sqrt((a_mid ** 2 + c_mid ** 2) / 2)
    coords = np.stack([par[:, 0] * r, par[:, 1] * arc], axis=1)
    n = par.shape[0]
    out = np.zeros(n, dtype=np.int64)
    w = rng.uniform(1 - spread, 1 + spread, n_parts)
    if n_parts2 is None:
        _rcb(coords, np.arange(n), list(w), out, 0)
        return out, None
    if n_parts % n_parts2:
        raise ValueError("n_parts2 must divide the number of surface patches")
    per = n_parts // n_parts2
    groups = [list(w[g * per:(g + 1) * per]) for g in range(n_parts2)]
    outer = np.zeros(n, dtype=np.int64)
    _rcb(coords, np.arange(n), [sum(g) for g in groups], outer, 0)
    for g in range(n_parts2):
        idx = np.nonzero(outer == g)[0]
        _rcb(coords, idx, groups[g], out, g * per)
    return out, np.repeat(np.arange(n_parts2), per)


# Idealised LV workloads: about 1.0M free DoFs with P1 in 512 parts, and
# about 3.0M with P2 in 4096 parts (2048 surface patches x 2 transmural
# slabs) nested into 64 level-2 parts.  Endocardial pressure 2 kPa and an
# activation of a quarter of the peak, ramped over 8 load steps: at half the
# peak the tangent of the 3M-DoF P2 shell loses so much stability after the
# first Newton step that BDDC-GMRES stagnates (at any grouping, level count
# and precision), which a quarter of the peak avoids.
LV_CONFIGS = {
    "lv_p1": dict(nt=9, ntheta=256, nu=160, order=1, n_parts=512, primal="VEF", load_steps=8,
                  gamma=0.25 * GAMMA_MAX),
    "lv_p2": dict(nt=5, ntheta=176, nu=168, order=2, n_parts=4096, n_parts2=64, n_layers=2,
                  primal="VEF", load_steps=8, gamma=0.25 * GAMMA_MAX),
}


def lv_config(name, **overrides):
    kw = dict(LV_CONFIGS[name])
    kw.update(overrides)
    return lv_problem(**kw)


def lv_part_problem(prob, parts):
    """The part of a ventricle workload that lies in the given level-1
    subdomains, as a workload of its own: their elements, the nodes of those
    renumbered in increasing order, the clamped base nodes and endocardial
    pressure faces among them, the nodal fibres, material and loads
    unchanged, and the subdomains renumbered 0, 1, ... in increasing order.
    Nodes on the cut are left free (traction-free), so it is a sample of the
    workload's element, subdomain and load structure, not a piece of its
    solution."""
    epart = np.asarray(prob["elem_part"])
    keep_part = np.zeros(int(prob["n_parts"]), dtype=bool)
    keep_part[np.asarray(parts)] = True
    sel = np.nonzero(keep_part[epart])[0]
    elems = np.asarray(prob["elems"])[sel]
    nodes = np.unique(elems)
    new_id = -np.ones(len(prob["coords"]), dtype=np.int64)
    new_id[nodes] = np.arange(nodes.size)
    used, local_part = np.unique(epart[sel], return_inverse=True)
    pf = np.asarray(prob["pressure_faces"])
    emap = -np.ones(len(prob["elems"]), dtype=np.int64)
    emap[sel] = np.arange(sel.size)
    keep = emap[pf[:, 0]] >= 0
    dn = np.asarray(prob["dirichlet_nodes"])
    dn = dn[new_id[dn] >= 0]
    fib = prob["fibers"]
    out = dict(prob)
    out.pop("part2", None)
    out.pop("n_parts2", None)
    out.update({
        "coords": np.asarray(prob["coords"])[nodes],
        "elems": new_id[elems].astype(np.int32),
        "elem_part": local_part.astype(np.int32),
        "n_parts": int(used.size),
        "dirichlet_nodes": np.sort(new_id[dn]).astype(np.int32),
        "pressure_faces": np.stack([emap[pf[keep, 0]], pf[keep, 1]], axis=1).astype(np.int32),
        "fibers": {"kind": "nodal", "f": np.asarray(fib["f"])[nodes], "n": np.asarray(fib["n"])[nodes]},
    })
    return out


def clamped_parts(prob):
    """Level-1 subdomains that contain clamped (base) nodes, increasing."""
    isdir = np.zeros(len(prob["coords"]), dtype=bool)
    isdir[np.asarray(prob["dirichlet_nodes"])] = True
    touch = isdir[np.asarray(prob["elems"])].any(axis=1)
    return np.unique(np.asarray(prob["elem_part"])[touch])
