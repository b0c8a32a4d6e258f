"""Reference hexahedra (Q1, Q2) and Gauss quadrature.

Section 2 ("Space discretization") uses H^1-conforming Q1 and Q2 elements
on hexahedra; the paper does not state the quadrature, so this oracle uses
the tensor Gauss rules that integrate the stiffness of an affine element
exactly: 2 points per direction for Q1, 3 for Q2 (faces: 2x2 and 3x3).
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
    return {"Q1": 1, "Q2": 2}[elem_type]


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
