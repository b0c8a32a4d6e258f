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
* cells between rings are cut into 6 Kuhn tetrahedra, the apex prisms into
  3 tetrahedra with matching face diagonals;
* fibres (nodal input field): the helix angle falls linearly from
  +alpha at the endocardium to -alpha at the epicardium,
  f = cos(a) e_circ + sin(a) e_long, n = outward normal of the ellipsoid
  through the node (transmural direction); P2 edge midpoints take the
  normalised mean of their end nodes' directions;
* partition: recursive coordinate bisection of the element centroids in the
  parametric coordinates (theta, u, t) with target weights drawn
  U[1 - w, 1 + w] (seeded), nested so that level-2 subdomains group whole
  level-1 subdomains.

Local numbering of a tetrahedron: vertices 0..3; P2 adds edge midpoints in
the order (0,1), (1,2), (0,2), (0,3), (1,3), (2,3).  Local face f is the
face opposite vertex f.
"""
import numpy as np

from .material import default_material, GAMMA_MAX

TET_EDGES = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]


def _kuhn_tets(c):
    """6 tetrahedra of a cell with corner nodes c[i][j][k] (i: t, j: theta,
    k: u), all sharing the diagonal c000 - c111 (Kuhn/Freudenthal)."""
    out = []
    for p in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        idx = [0, 0, 0]
        path = [c[0][0][0]]
        for ax in p:
            idx[ax] = 1
            path.append(c[idx[0]][idx[1]][idx[2]])
        out.append(path)
    return out


def lv_problem(nt=3, ntheta=16, nu=8, order=1, a_endo=0.025, c_endo=0.070,
               a_epi=0.035, c_epi=0.080, jitter=0.15, seed=2208, n_parts=8,
               n_parts2=None, weight_spread=0.3, part_seed=6191,
               pressure=2.0e3, gamma=0.5 * GAMMA_MAX, alpha_deg=60.0,
               load_steps=4, primal="VEF", material=None):
    """P1/P2 tetrahedral mesh of the ventricle shell with nt transmural,
    ntheta circumferential and nu longitudinal node layers (u > 0), plus one
    apex node per transmural layer."""
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, nt)
    th = np.linspace(0.0, 2 * np.pi, ntheta, endpoint=False)
    u = np.linspace(0.0, 1.0, nu + 1)[1:]
    # node ids: apex(t) = t, ring node (t, j, k) = nt + t + nt*(j + ntheta*k)
    def ring(i, j, k):
        return nt + i + nt * ((j % ntheta) + ntheta * k)

    n_nodes = nt + nt * ntheta * nu
    P = np.zeros((n_nodes, 3))   # parametric (t, theta, u)
    for i in range(nt):
        P[i] = (t[i], 0.0, 0.0)
    for k in range(nu):
        for j in range(ntheta):
            for i in range(nt):
                P[ring(i, j, k)] = (t[i], th[j], u[k])
    P0 = P.copy()
    # jitter interior nodes in parametric space (not on endo/epi/base/apex)
    if jitter > 0:
        dt, dth, du = 1.0 / max(nt - 1, 1), 2 * np.pi / ntheta, 1.0 / nu
        for k in range(nu - 1):
            for j in range(ntheta):
                for i in range(1, nt - 1):
                    q = ring(i, j, k)
                    P[q] += rng.uniform(-jitter, jitter, 3) * (dt, dth, du)
        # circumferential / longitudinal jitter of surface rings too
        for k in range(nu - 1):
            for j in range(ntheta):
                for i in (0, nt - 1):
                    q = ring(i, j, k)
                    P[q, 1:] += rng.uniform(-jitter, jitter, 2) * (dth, du)

    def to_xyz(tt, tht, uu):
        a = a_endo + tt * (a_epi - a_endo)
        c = c_endo + tt * (c_epi - c_endo)
        psi = uu * np.pi / 2
        return np.stack([a * np.sin(psi) * np.cos(tht), a * np.sin(psi) * np.sin(tht),
                         -c * np.cos(psi)], axis=-1)

    X = to_xyz(P[:, 0], P[:, 1], P[:, 2])
    X[np.abs(P[:, 2] - 1.0) < 1e-12, 2] = 0.0  # base plane exactly at z = 0
    tets, cell_par = [], []
    for k in range(nu - 1):
        for j in range(ntheta):
            for i in range(nt - 1):
                c = [[[ring(i + a, j + b, k + cc) for cc in (0, 1)] for b in (0, 1)] for a in (0, 1)]
                for tt in _kuhn_tets(c):
                    tets.append(tt)
                    cell_par.append((t[i] + 0.5 / (nt - 1), th[j] + np.pi / ntheta, (k + 1.5) / nu))
    for j in range(ntheta):
        for i in range(nt - 1):
            A0, A1 = i, i + 1
            B0, B1 = ring(i, j, 0), ring(i + 1, j, 0)
            C0, C1 = ring(i, j + 1, 0), ring(i + 1, j + 1, 0)
            for tt in ([A0, B0, C0, C1], [A0, B0, B1, C1], [A0, A1, B1, C1]):
                tets.append(tt)
                cell_par.append((t[i] + 0.5 / (nt - 1), th[j] + np.pi / ntheta, 0.5 / nu))
    tets = np.array(tets, dtype=np.int64)
    cell_par = np.array(cell_par)
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
    # P2: edge midpoints
    if order == 2:
        edge_id = {}
        mids = []
        elems = np.zeros((tets.shape[0], 10), dtype=np.int64)
        elems[:, :4] = tets
        for e in range(tets.shape[0]):
            for m, (a, b) in enumerate(TET_EDGES):
                key = (min(tets[e, a], tets[e, b]), max(tets[e, a], tets[e, b]))
                if key not in edge_id:
                    edge_id[key] = n_nodes + len(mids)
                    mids.append(key)
                elems[e, 4 + m] = edge_id[key]
        mids = np.array(mids, dtype=np.int64)
        X = np.concatenate([X, 0.5 * (X[mids[:, 0]] + X[mids[:, 1]])])
        P = np.concatenate([P, np.full((mids.shape[0], 3), 0.5)])  # only t is used below
        P[n_nodes:, 0] = 0.5 * (P[mids[:, 0], 0] + P[mids[:, 1], 0])
        fm = fib[mids[:, 0]] + fib[mids[:, 1]]
        nm = nrm[mids[:, 0]] + nrm[mids[:, 1]]
        fib = np.concatenate([fib, fm / np.linalg.norm(fm, axis=1)[:, None]])
        nrm = np.concatenate([nrm, nm / np.linalg.norm(nm, axis=1)[:, None]])
        n_nodes = X.shape[0]
    else:
        elems = tets
    # boundary sets
    base = np.nonzero(np.abs(X[:, 2]) < 1e-12)[0]
    endo_node = np.abs(P[:, 0]) < 1e-12
    faces = []
    for e in range(tets.shape[0]):
        for f in range(4):
            vs = [tets[e, q] for q in range(4) if q != f]
            if all(endo_node[q] for q in vs):
                faces.append((e, f))
    pressure_faces = np.array(faces, dtype=np.int64).reshape(-1, 2)
    # partition of the elements (nested when n_parts2 is given)
    part, part2, n2 = _partition(cell_par, tets.shape[0], n_parts, n_parts2, weight_spread, part_seed)
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


def _partition(cell_par, n_el, n_parts, n_parts2, spread, seed):
    rng = np.random.default_rng(seed)
    # scaled parametric coordinates so that bisection cuts across the
    # longest physical direction: theta (circumference), u (height), t (wall)
    coords = np.stack([cell_par[:, 1] * 2.0, cell_par[:, 2] * 3.0, cell_par[:, 0] * 0.5], axis=1)
    out = np.zeros(n_el, dtype=np.int64)
    if n_parts2 is None:
        w = rng.uniform(1 - spread, 1 + spread, n_parts)
        _rcb(coords, np.arange(n_el), list(w), out, 0)
        return out, None, None
    assert n_parts % n_parts2 == 0
    per = n_parts // n_parts2
    w = rng.uniform(1 - spread, 1 + spread, n_parts)
    groups = [list(w[g * per:(g + 1) * per]) for g in range(n_parts2)]
    # first the level-2 groups (weights = sums of their members), then each
    outer = np.zeros(n_el, dtype=np.int64)
    _rcb(coords, np.arange(n_el), [sum(g) for g in groups], outer, 0)
    for g in range(n_parts2):
        idx = np.nonzero(outer == g)[0]
        _rcb(coords, idx, groups[g], out, g * per)
    part2 = np.repeat(np.arange(n_parts2), per)
    return out, part2, n_parts2


# Idealised LV workloads: about 1.0M free DoFs with P1 in 512 parts, and
# about 3.0M with P2 in 4096 parts nested into 64 level-2 parts.
LV_CONFIGS = {
    "lv_p1": dict(nt=9, ntheta=256, nu=144, order=1, n_parts=512, primal="VEF"),
    "lv_p2": dict(nt=5, ntheta=160, nu=156, order=2, n_parts=4096, n_parts2=64, primal="VEF"),
}


def lv_config(name, **overrides):
    kw = dict(LV_CONFIGS[name])
    kw.update(overrides)
    return lv_problem(**kw)
