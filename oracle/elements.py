"""Reference elements and quadrature: hexahedra (Q1, Q2) and tetrahedra
(P1, P2).

Section 2 ("Space discretization") uses H^1-conforming Q1/Q2 elements on
hexahedra and P1/P2 elements on tetrahedra; the paper does not state the
quadrature, so this oracle uses rules that integrate the stiffness of an
affine element exactly: tensor Gauss with 2 points per direction for Q1 and
3 for Q2 (faces 2x2 and 3x3); the centroid rule for P1 (face: centroid) and
the symmetric 4-point degree-2 rule for P2 (face: the 3-point degree-2 rule
at (1/6, 1/6), (2/3, 1/6), (1/6, 2/3)).

Reference tetrahedron: vertices v0 = 0, v1 = e_x, v2 = e_y, v3 = e_z with
barycentric coordinates L0 = 1 - x - y - z, L1 = x, L2 = y, L3 = z; P2 adds
the edge midpoints of (0,1), (1,2), (0,2), (0,3), (1,3), (2,3); local face f
is the face opposite vertex f.
"""
import numpy as np


def gauss_1d(n):
    """Gauss-Legendre points and weights on [-1, 1] (numpy's routine)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return x, w


def lagrange_1d(k, x):
    """Values and derivatives of the 1-D Lagrange basis of degree k on the
    equispaced nodes -1 + 2a/k, evaluated at points x.  Returns (N, dN) of
    shape (len(x), k+1)."""
    nodes = np.linspace(-1.0, 1.0, k + 1)
    x = np.asarray(x, dtype=float)
    N = np.ones((x.size, k + 1))
    dN = np.zeros((x.size, k + 1))
    for a in range(k + 1):
        others = [b for b in range(k + 1) if b != a]
        denom = np.prod([nodes[a] - nodes[b] for b in others])
        for b in others:
            N[:, a] *= (x - nodes[b])
        N[:, a] /= denom
        # derivative: sum over dropped factor
        for c in others:
            term = np.ones(x.size)
            for b in others:
                if b != c:
                    term *= (x - nodes[b])
            dN[:, a] += term
        dN[:, a] /= denom
    return N, dN


def hex_shape(k, xi):
    """Shape values (n_pts, n_en) and reference gradients (n_pts, n_en, 3)
    of the tensor-product hexahedron of degree k at points xi (n_pts, 3),
    local node a + (k+1)(b + (k+1)c)."""
    xi = np.atleast_2d(xi)
    Nx, dNx = lagrange_1d(k, xi[:, 0])
    Ny, dNy = lagrange_1d(k, xi[:, 1])
    Nz, dNz = lagrange_1d(k, xi[:, 2])
    m = k + 1
    n_en = m ** 3
    N = np.zeros((xi.shape[0], n_en))
    dN = np.zeros((xi.shape[0], n_en, 3))
    for c in range(m):
        for b in range(m):
            for a in range(m):
                i = a + m * (b + m * c)
                N[:, i] = Nx[:, a] * Ny[:, b] * Nz[:, c]
                dN[:, i, 0] = dNx[:, a] * Ny[:, b] * Nz[:, c]
                dN[:, i, 1] = Nx[:, a] * dNy[:, b] * Nz[:, c]
                dN[:, i, 2] = Nx[:, a] * Ny[:, b] * dNz[:, c]
    return N, dN


def hex_volume_rule(k):
    """Tensor Gauss rule with k+1 points per direction: points (n_q, 3),
    weights (n_q,)."""
    x, w = gauss_1d(k + 1)
    P = np.array([[x[i], x[j], x[l]] for l in range(k + 1)
                  for j in range(k + 1) for i in range(k + 1)])
    W = np.array([w[i] * w[j] * w[l] for l in range(k + 1)
                  for j in range(k + 1) for i in range(k + 1)])
    return P, W


# Local face f of the reference hexahedron: (fixed axis, fixed value, s-axis,
# t-axis), with (e_s x e_t) pointing out of the element.
HEX_FACE_PARAM = {
    0: (0, -1.0, 2, 1),
    1: (0, +1.0, 1, 2),
    2: (1, -1.0, 0, 2),
    3: (1, +1.0, 2, 0),
    4: (2, -1.0, 1, 0),
    5: (2, +1.0, 0, 1),
}


def hex_face_rule(k, face):
    """Face quadrature mapped into the volume reference element.

    Returns the volume reference points (n_q, 3), the weights (n_q,), and the
    tangent vectors d xi / ds, d xi / dt (3,) of the face parametrisation."""
    axis, val, sa, ta = HEX_FACE_PARAM[face]
    x, w = gauss_1d(k + 1)
    pts, wts = [], []
    for j in range(k + 1):
        for i in range(k + 1):
            p = np.zeros(3)
            p[axis] = val
            p[sa] = x[i]
            p[ta] = x[j]
            pts.append(p)
            wts.append(w[i] * w[j])
    es = np.zeros(3)
    es[sa] = 1.0
    et = np.zeros(3)
    et[ta] = 1.0
    return np.array(pts), np.array(wts), es, et


def element_order(elem_type):
    return {"Q1": 1, "Q2": 2, "P1": 1, "P2": 2}[elem_type]


def is_tet(elem_type):
    return elem_type in ("P1", "P2")


TET_VERTS = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
TET_EDGES = [(0, 1), (1, 2), (0, 2), (0, 3), (1, 3), (2, 3)]
# Local face f (opposite vertex f): (origin, s-end, t-end) vertices with
# (v_s - v_o) x (v_t - v_o) pointing out of the element.
TET_FACE_PARAM = {0: (1, 2, 3), 1: (0, 3, 2), 2: (0, 1, 3), 3: (0, 2, 1)}


def tet_nodes(k):
    """Reference coordinates of the local nodes, shape (n_en, 3)."""
    if k == 1:
        return TET_VERTS.copy()
    mids = [0.5 * (TET_VERTS[a] + TET_VERTS[b]) for a, b in TET_EDGES]
    return np.vstack([TET_VERTS, np.array(mids)])


def tet_shape(k, xi):
    """Shape values (n_pts, n_en) and reference gradients (n_pts, n_en, 3)
    of the P1 (k = 1) or P2 (k = 2) tetrahedron at points xi (n_pts, 3)."""
    xi = np.atleast_2d(np.asarray(xi, dtype=float))
    L = np.stack([1.0 - xi.sum(1), xi[:, 0], xi[:, 1], xi[:, 2]], axis=1)
    dL = np.array([[-1.0, -1.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    if k == 1:
        return L, np.broadcast_to(dL, (xi.shape[0], 4, 3)).copy()
    N = np.zeros((xi.shape[0], 10))
    dN = np.zeros((xi.shape[0], 10, 3))
    for a in range(4):  # vertex: L_a (2 L_a - 1)
        N[:, a] = L[:, a] * (2.0 * L[:, a] - 1.0)
        dN[:, a] = (4.0 * L[:, a] - 1.0)[:, None] * dL[a]
    for m, (a, b) in enumerate(TET_EDGES):  # edge: 4 L_a L_b
        N[:, 4 + m] = 4.0 * L[:, a] * L[:, b]
        dN[:, 4 + m] = 4.0 * (L[:, b][:, None] * dL[a] + L[:, a][:, None] * dL[b])
    return N, dN


def tet_volume_rule(k):
    """Centroid rule (P1) or the symmetric 4-point degree-2 rule (P2) on the
    reference tetrahedron of volume 1/6: points (n_q, 3), weights (n_q,)."""
    if k == 1:
        return np.array([[0.25, 0.25, 0.25]]), np.array([1.0 / 6.0])
    a = (5.0 + 3.0 * np.sqrt(5.0)) / 20.0
    b = (5.0 - np.sqrt(5.0)) / 20.0
    bary = np.full((4, 4), b) + np.eye(4) * (a - b)
    return bary @ TET_VERTS, np.full(4, 1.0 / 24.0)


def tri_rule(k):
    """Rule on the reference triangle {s, t >= 0, s + t <= 1} (area 1/2):
    points (n_q, 2), weights."""
    if k == 1:
        return np.array([[1.0 / 3.0, 1.0 / 3.0]]), np.array([0.5])
    return (np.array([[1.0 / 6.0, 1.0 / 6.0], [2.0 / 3.0, 1.0 / 6.0], [1.0 / 6.0, 2.0 / 3.0]]),
            np.full(3, 1.0 / 6.0))


def tet_face_rule(k, face):
    """Face quadrature of a tetrahedron mapped into the volume reference
    element: (points (n_q, 3), weights, d xi/ds, d xi/dt)."""
    o, ps, pt = TET_FACE_PARAM[face]
    es = TET_VERTS[ps] - TET_VERTS[o]
    et = TET_VERTS[pt] - TET_VERTS[o]
    st, w = tri_rule(k)
    pts = TET_VERTS[o][None, :] + st[:, :1] * es[None, :] + st[:, 1:] * et[None, :]
    return pts, w, es, et


def tet_face_nodes(k, face):
    """Local node indices on face f (the nodes not involving vertex f)."""
    out = [a for a in range(4) if a != face]
    if k == 2:
        out += [4 + m for m, (a, b) in enumerate(TET_EDGES) if face not in (a, b)]
    return out


def shape(elem_type, xi):
    k = element_order(elem_type)
    return tet_shape(k, xi) if is_tet(elem_type) else hex_shape(k, xi)


def volume_rule(elem_type):
    k = element_order(elem_type)
    return tet_volume_rule(k) if is_tet(elem_type) else hex_volume_rule(k)


def face_rule(elem_type, face):
    k = element_order(elem_type)
    return tet_face_rule(k, face) if is_tet(elem_type) else hex_face_rule(k, face)


def face_nodes(elem_type, face):
    k = element_order(elem_type)
    return tet_face_nodes(k, face) if is_tet(elem_type) else hex_face_nodes(k, face)


def corner_faces(elem_type):
    """Vertex nodes of every local face (used to find the outer boundary:
    a face is on it when no other element has the same vertex set)."""
    if is_tet(elem_type):
        return [[a for a in range(4) if a != f] for f in range(4)]
    m = element_order(elem_type) + 1
    K = m - 1

    def idx(a, b, c):
        return a + m * (b + m * c)
    return [
        [idx(0, 0, 0), idx(0, K, 0), idx(0, K, K), idx(0, 0, K)],
        [idx(K, 0, 0), idx(K, K, 0), idx(K, K, K), idx(K, 0, K)],
        [idx(0, 0, 0), idx(K, 0, 0), idx(K, 0, K), idx(0, 0, K)],
        [idx(0, K, 0), idx(K, K, 0), idx(K, K, K), idx(0, K, K)],
        [idx(0, 0, 0), idx(K, 0, 0), idx(K, K, 0), idx(0, K, 0)],
        [idx(0, 0, K), idx(K, 0, K), idx(K, K, K), idx(0, K, K)],
    ]


def hex_face_nodes(k, face):
    """Local node indices on a face (all nodes of the face, any order)."""
    axis, val, _, _ = HEX_FACE_PARAM[face]
    m = k + 1
    fixed = 0 if val < 0 else k
    out = []
    for c in range(m):
        for b in range(m):
            for a in range(m):
                idx = (a, b, c)
                if idx[axis] == fixed:
                    out.append(a + m * (b + m * c))
    return out
