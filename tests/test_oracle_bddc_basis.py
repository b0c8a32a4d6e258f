"""The oracle's BDDC (Section 3.2: constrained local problems through
Lagrange multipliers and the minimum-energy coarse basis Phi) against the
change-of-basis form of the same preconditioner, written independently
here: each subdomain's interface space is rewritten in coordinates where
every primal constraint is one explicit DoF (primal columns C^+ and a
null-space basis of C for the dual part), the partially assembled Schur
complement S~ (primal DoFs assembled, dual DoFs local) is formed and
inverted densely, and

    M_S^-1 = sum_i R_i^T D_i T_i R~_i  S~^-1  sum_j R~_j^T T_j^T D_j^T R_j.

For a symmetric tangent both forms are the same operator (the dense
matrices agree to rounding), for every primal space (vertices, edge and
face averages, rigid-body rotations) and for counting and deluxe scaling.
The tangent is symmetric without follower pressure: the active stress is
the derivative of gamma |F f|.  With follower pressure the tangent is
nonsymmetric; eliminating the dual DoFs of S~ then gives the coarse
problem with a right basis from S and a left basis from S^T, which is the
oracle's "petrov" coarse space, and not its one-basis Galerkin coarse
space."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle.assembly import FEProblem
from oracle.bddc import BDDC, class_rotations
from workloads import slab_problem


def _class_rows(X, rotations):
    m = len(X)
    rows = np.zeros((3, 3 * m))
    for c in range(3):
        rows[c, c::3] = 1.0 / m
    if rotations:
        rows = np.vstack([rows, class_rotations(X)])
    return rows


def _change_of_basis_inverse(fe, subs, cl, primal, deluxe, gamma_dofs):
    """Dense M_S^-1 on the global interface DoFs gamma_dofs."""
    use_v, use_r = "V" in primal, "R" in primal
    classes = (cl.edges if "E" in primal else []) + (cl.faces if "F" in primal else [])
    # global primal numbering
    pidx = {}
    if use_v:
        for a in cl.vertices:
            for c in range(3):
                pidx[("v", a, c)] = len(pidx)
    rows_of = []
    for k, K in enumerate(classes):
        R = _class_rows(fe.coords[K], use_r)
        rows_of.append(R)
        for q in range(R.shape[0]):
            pidx[("c", k, q)] = len(pidx)
    n_pi = len(pidx)
    gpos = {g: i for i, g in enumerate(gamma_dofs)}
    local = []
    for sub in subs:
        nodes = sub["nodes"]
        iface = cl.count[nodes] >= 2
        gnodes = nodes[iface]
        gdofs = (3 * fe.node_to_free[gnodes][:, None] + np.arange(3)).reshape(-1)
        A = sub["A"].toarray()
        lI = (3 * np.nonzero(~iface)[0][:, None] + np.arange(3)).reshape(-1)
        lG = (3 * np.nonzero(iface)[0][:, None] + np.arange(3)).reshape(-1)
        S = A[np.ix_(lG, lG)]
        if lI.size:
            S = S - A[np.ix_(lG, lI)] @ np.linalg.solve(A[np.ix_(lI, lI)], A[np.ix_(lI, lG)])
        n = lG.size
        pos_of_node = {int(a): j for j, a in enumerate(gnodes)}
        # primal columns and dual blocks
        T_cols, p_glob = [], []
        used = np.zeros(n, dtype=bool)
        dual_blocks = []
        if use_v:
            for a in cl.vertices:
                if int(a) in pos_of_node:
                    for c in range(3):
                        col = np.zeros(n)
                        col[3 * pos_of_node[int(a)] + c] = 1.0
                        T_cols.append(col)
                        p_glob.append(pidx[("v", a, c)])
                        used[3 * pos_of_node[int(a)] + c] = True
        for k, K in enumerate(classes):
            if int(K[0]) not in pos_of_node:
                continue
            dofs = np.array([3 * pos_of_node[int(a)] + c for a in K for c in range(3)])
            Ck = rows_of[k]
            pinv = np.linalg.pinv(Ck)
            for q in range(Ck.shape[0]):
                col = np.zeros(n)
                col[dofs] = pinv[:, q]
                T_cols.append(col)
                p_glob.append(pidx[("c", k, q)])
            N = sla.null_space(Ck)
            blk = np.zeros((n, N.shape[1]))
            blk[dofs] = N
            dual_blocks.append(blk)
            used[dofs] = True
        for j in np.nonzero(~used)[0]:
            col = np.zeros((n, 1))
            col[j] = 1.0
            dual_blocks.append(col)
        Tp = np.column_stack(T_cols) if T_cols else np.zeros((n, 0))
        Td = np.hstack(dual_blocks) if dual_blocks else np.zeros((n, 0))
        T = np.hstack([Tp, Td])
        assert T.shape == (n, n) and np.linalg.matrix_rank(T) == n
        counts = np.repeat(cl.count[gnodes], 3).astype(float)
        local.append(dict(S=S, T=T, n_p=Tp.shape[1], p_glob=np.array(p_glob, dtype=int),
                          R=np.array([gpos[g] for g in gdofs]), D=np.diag(1.0 / counts),
                          gnodes=gnodes, pos_of_node=pos_of_node))
    if deluxe:
        # D_K^(i) = (sum_j S_K^(j))^-1 S_K^(i) on every edge and face class
        for K in cl.edges + cl.faces:
            owners = [L for L in local if int(K[0]) in L["pos_of_node"]]
            blocks = []
            for L in owners:
                d = np.array([3 * L["pos_of_node"][int(a)] + c for a in K for c in range(3)])
                blocks.append((L, d, L["S"][np.ix_(d, d)]))
            Shat = sum(b[2] for b in blocks)
            for L, d, SK in blocks:
                L["D"][np.ix_(d, d)] = np.linalg.solve(Shat, SK)
    # partially assembled S~ : primal block first, then each subdomain's duals
    offs, tot = [], n_pi
    for L in local:
        offs.append(tot)
        tot += L["T"].shape[1] - L["n_p"]
    St = np.zeros((tot, tot))
    maps = []
    for L, o in zip(local, offs):
        nd = L["T"].shape[1] - L["n_p"]
        m = np.concatenate([L["p_glob"], o + np.arange(nd)])
        maps.append(m)
        St[np.ix_(m, m)] += L["T"].T @ L["S"] @ L["T"]
    ng = len(gamma_dofs)
    left = np.zeros((ng, tot))
    right = np.zeros((tot, ng))
    for L, m in zip(local, maps):
        E = np.zeros((len(L["R"]), ng))
        E[np.arange(len(L["R"])), L["R"]] = 1.0          # R_i
        left[:, m] += E.T @ L["D"] @ L["T"]
        right[m, :] += L["T"].T @ L["D"].T @ E
    return left @ np.linalg.solve(St, right)


def _dense_pair(pressure, primal, scaling, coarse="galerkin"):
    prob = slab_problem(4, 4, 3, parts=(2, 2, 1), jitter=0.15, pressure=pressure, gamma=3e4)
    fe = FEProblem(prob)
    d = 2e-3 * np.random.default_rng(7).standard_normal(fe.n_free)
    K, (Ke, Kf) = fe.tangent(d, 1.0)
    Kd = K.toarray()
    pc = BDDC(fe, Ke, Kf, primal, scaling=scaling, coarse=coarse)
    cl = pc.cl
    free_nodes = np.nonzero(fe.node_to_free >= 0)[0]
    gnodes = free_nodes[cl.count[free_nodes] >= 2]
    gamma = (3 * fe.node_to_free[gnodes][:, None] + np.arange(3)).reshape(-1)
    # oracle: r with r_I = 0 gives z_Gamma = M_S^-1 r_Gamma
    M_oracle = np.zeros((gamma.size, gamma.size))
    for j, gdof in enumerate(gamma):
        r = np.zeros(fe.n_free)
        r[gdof] = 1.0
        M_oracle[:, j] = pc.apply(r)[gamma]
    M_basis = _change_of_basis_inverse(fe, pc.subs, cl, primal, scaling == "deluxe", gamma)
    return Kd, M_oracle, M_basis


@pytest.mark.parametrize("primal", ["V", "VE", "VEF", "EF", "VER", "EFR"])
@pytest.mark.parametrize("scaling", ["counting", "deluxe"])
def test_lagrange_form_equals_change_of_basis(primal, scaling):
    Kd, M_oracle, M_basis = _dense_pair(0.0, primal, scaling)
    assert np.abs(Kd - Kd.T).max() <= 1e-12 * np.abs(Kd).max()
    assert np.abs(M_oracle - M_basis).max() <= 1e-10 * np.abs(M_basis).max()


@pytest.mark.parametrize("primal", ["VE", "VEF", "EFR"])
@pytest.mark.parametrize("scaling", ["counting", "deluxe"])
def test_nonsymmetric_petrov_coarse_equals_change_of_basis(primal, scaling):
    Kd, M_petrov, M_basis = _dense_pair(2e3, primal, scaling, coarse="petrov")
    asym = np.abs(Kd - Kd.T).max() / np.abs(Kd).max()
    assert asym > 1e-6                      # follower pressure: nonsymmetric
    assert np.abs(M_petrov - M_basis).max() <= 1e-10 * np.abs(M_basis).max()
    _, M_galerkin, _ = _dense_pair(2e3, primal, scaling)
    assert np.abs(M_galerkin - M_basis).max() > 1e-8 * np.abs(M_basis).max()
