"""The seeded input generators: partitions the BDDC setup relies on.
Ventricle subdomains (surface patches x transmural slabs, after the repair
pass that moves disconnected pieces) are face-connected, none is empty, and
the level-2 grouping covers every level-2 subdomain; slab box partitions
have equal boxes.  The same seed gives the same problem."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.csgraph as csg

from workloads import lv_problem, slab_problem


def _face_components(elems, part, faces_of):
    keys = {}
    for f, cn in enumerate(faces_of):
        for e, key in enumerate(map(tuple, np.sort(elems[:, cn], axis=1))):
            keys.setdefault(key, []).append(e)
    rows, cols = [], []
    for lst in keys.values():
        if len(lst) == 2 and part[lst[0]] == part[lst[1]]:
            rows.append(lst[0])
            cols.append(lst[1])
    n = len(elems)
    G = sp.coo_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    _, comp = csg.connected_components(G, directed=False)
    return comp


@pytest.mark.parametrize("order", [1, 2])
def test_ventricle_subdomains_are_connected_and_nested(order):
    prob = lv_problem(nt=5, ntheta=48, nu=24, order=order, n_parts=48, n_parts2=6, n_layers=2)
    E = np.asarray(prob["elems"])[:, :4]
    part = np.asarray(prob["elem_part"])
    n = int(prob["n_parts"])
    assert n == 48 and set(np.unique(part)) == set(range(n))
    tri = [[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]]
    comp = _face_components(E, part, tri)
    for i in range(n):
        assert np.unique(comp[part == i]).size == 1, "subdomain %d is not face-connected" % i
    part2 = np.asarray(prob["part2"])
    assert part2.shape == (n,) and set(np.unique(part2)) == set(range(int(prob["n_parts2"])))


def test_slab_boxes_are_equal():
    prob = slab_problem(12, 8, 6, parts=(3, 2, 3))
    part = np.asarray(prob["elem_part"])
    counts = np.bincount(part, minlength=prob["n_parts"])
    assert prob["n_parts"] == 18 and np.all(counts == 12 * 8 * 6 // 18)


def test_generators_are_seeded():
    a = lv_problem(nt=3, ntheta=16, nu=8, n_parts=8)
    b = lv_problem(nt=3, ntheta=16, nu=8, n_parts=8)
    assert np.array_equal(a["coords"], b["coords"]) and np.array_equal(a["elem_part"], b["elem_part"])
    c = slab_problem(6, 6, 4, jitter=0.2)
    d = slab_problem(6, 6, 4, jitter=0.2)
    assert np.array_equal(c["coords"], d["coords"])
