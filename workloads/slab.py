"""Structured slab workloads: hexahedral Q1/Q2 meshes cut into box subdomains.

The paper's beam test (Section 5) is a structured hexahedral box; these slabs
stand in for its benchmark meshes, which are not available.  Each problem is
a plain dictionary of numpy arrays; see the package docstring for the local
numbering conventions.
"""
import numpy as np

from .material import default_material, GAMMA_MAX


def _box_index(e, n, p):
    """Box index of element layer ``e`` when ``n`` layers are cut into ``p``
    boxes as evenly as possible (ragged when ``p`` does not divide ``n``)."""
    return (e * p) // n


def slab_problem(nx, ny, nz, order=1, lengths=(1.0, 1.0, 1.0),
                 parts=(2, 2, 2), jitter=0.0, seed=2208,
                 pressure=1.0e3, gamma=0.5 * GAMMA_MAX,
                 alpha_deg=(-60.0, 60.0), load_steps=4, primal="V",
                 material=None):
    """Slab [0,Lx]x[0,Ly]x[0,Lz] with nx*ny*nz hexahedra of order 1 or 2.

    * z = 0 face clamped (Dirichlet nodes),
    * follower pressure ``pressure`` on the z = Lz face (local face 5),
    * fibres rotating helically in the xy-plane from ``alpha_deg[0]`` at
      z = 0 to ``alpha_deg[1]`` at z = Lz,
    * box partition ``parts`` = (px, py, pz) of the element grid,
    * ``jitter`` > 0 moves every vertex that is not on the outer boundary by
      U[-jitter, jitter] times the element size (seeded); Q2 mid-nodes then
      sit at the midpoints of the moved vertices (straight-sided elements).
    """
    k = int(order)
    assert k in (1, 2)
    lx, ly, lz = lengths
    mx, my, mz = k * nx + 1, k * ny + 1, k * nz + 1
    # vertex-grid coordinates, optionally jittered, then refined for Q2
    vx = np.linspace(0.0, lx, nx + 1)
    vy = np.linspace(0.0, ly, ny + 1)
    vz = np.linspace(0.0, lz, nz + 1)
    VX, VY, VZ = np.meshgrid(vx, vy, vz, indexing="ij")
    V = np.stack([VX, VY, VZ], axis=-1)  # (nx+1, ny+1, nz+1, 3)
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        h = np.array([lx / nx, ly / ny, lz / nz])
        delta = rng.uniform(-jitter, jitter, size=V.shape) * h
        inner = np.zeros(V.shape[:3], dtype=bool)
        inner[1:-1, 1:-1, 1:-1] = True
        V = V + delta * inner[..., None]
    if k == 1:
        G = V
    else:
        G = np.zeros((mx, my, mz, 3))
        G[::2, ::2, ::2] = V
        G[1::2, :, :] = 0.5 * (G[0:-1:2, :, :] + G[2::2, :, :])
        G[:, 1::2, :] = 0.5 * (G[:, 0:-1:2, :] + G[:, 2::2, :])
        G[:, :, 1::2] = 0.5 * (G[:, :, 0:-1:2] + G[:, :, 2::2])
    # node id = i + mx*(j + my*l); coordinates in that order
    coords = np.ascontiguousarray(G.transpose(2, 1, 0, 3).reshape(-1, 3))

    def nid(i, j, l):
        return i + mx * (j + my * l)

    ex, ey, ez = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz),
                             indexing="ij")
    ex = ex.transpose(2, 1, 0).ravel()
    ey = ey.transpose(2, 1, 0).ravel()
    ez = ez.transpose(2, 1, 0).ravel()  # element id = ex + nx*(ey + ny*ez)
    n_en = (k + 1) ** 3
    elems = np.empty((ex.size, n_en), dtype=np.int32)
    for c in range(k + 1):
        for b in range(k + 1):
            for a in range(k + 1):
                elems[:, a + (k + 1) * (b + (k + 1) * c)] = nid(
                    k * ex + a, k * ey + b, k * ez + c)
    px, py, pz = parts
    part = (_box_index(ex, nx, px)
            + px * (_box_index(ey, ny, py) + py * _box_index(ez, nz, pz)))
    dirichlet = np.nonzero(coords[:, 2] == 0.0)[0].astype(np.int32)
    top = np.nonzero(ez == nz - 1)[0].astype(np.int32)
    pressure_faces = np.stack([top, np.full_like(top, 5)], axis=1)
    return {
        "elem_type": "Q1" if k == 1 else "Q2",
        "coords": coords,
        "elems": elems,
        "elem_part": part.astype(np.int32),
        "n_parts": int(px * py * pz),
        "dirichlet_nodes": dirichlet,
        "pressure_faces": pressure_faces.astype(np.int32),
        "fibers": {"kind": "slab_helix", "z0": 0.0, "z1": float(lz),
                   "alpha0": np.deg2rad(alpha_deg[0]),
                   "alpha1": np.deg2rad(alpha_deg[1])},
        "material": dict(material or default_material()),
        "pressure": float(pressure),
        "gamma": float(gamma),
        "load_steps": int(load_steps),
        "primal": primal,
        "shape": (nx, ny, nz),
    }


# The structured workloads: an 8^3 Q1 cube in 2x2x2 boxes with vertex
# primal space, a 48x48x12 Q1 slab (unit thickness, cubic elements) in 4x4x4
# boxes with vertex + edge averages, and a 24x24x6 Q2 slab in 8x4x2 boxes
# with vertex + edge + face averages.
SLAB_CONFIGS = {
    "slab8_q1": dict(nx=8, ny=8, nz=8, order=1, lengths=(1.0, 1.0, 1.0),
                     parts=(2, 2, 2), primal="V"),
    "slab48_q1": dict(nx=48, ny=48, nz=12, order=1, lengths=(4.0, 4.0, 1.0),
                      parts=(4, 4, 4), primal="VE"),
    "slab24_q2": dict(nx=24, ny=24, nz=6, order=2, lengths=(4.0, 4.0, 1.0),
                      parts=(8, 4, 2), primal="VEF"),
}


def slab_config(name, **overrides):
    kw = dict(SLAB_CONFIGS[name])
    kw.update(overrides)
    return slab_problem(**kw)


def box_groups(parts, groups):
    """Level-2 partition of box subdomains: box (bx, by, bz) of a
    px x py x pz box partition goes to group (bx*gx//px, by*gy//py, bz*gz//pz)
    of a gx x gy x gz grouping.  Returns (group id per subdomain, n_groups)."""
    px, py, pz = parts
    gx, gy, gz = groups
    out = []
    for bz in range(pz):
        for by in range(py):
            for bx in range(px):
                out.append((bx * gx) // px + gx * ((by * gy) // py + gy * ((bz * gz) // pz)))
    return np.array(out, dtype=np.int32), gx * gy * gz
