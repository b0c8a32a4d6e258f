"""Load-stepped Newton iteration, Eq. (tangent problem) of Section 2.

For each load level lambda_k = k / n_steps (pressure and activation scaled
together), Newton starts from the previous converged displacement
(d^{n,0} = d^{n-1}), solves DF(d)[delta] = -F(d) and updates d += delta,
until ||F(d)|| <= tol ||F(d^{n,0})||.  If an iterate inverts an element
(J <= 0) or Newton does not converge, the load increment is halved.

The tangent systems are solved either exactly (sparse LU, the "truth") or by
GMRES preconditioned by BDDC.
"""
import numpy as np
import scipy.sparse.linalg as spla

from .assembly import FEProblem
from .bddc import BDDC, Classification
from .krylov import gmres


def direct_solver(fe, K, KeKf, r, lam):
    return spla.spsolve(K.tocsc(), -r), 0


def make_bddc_solver(primal, tol=1e-8, restart=100, flexible=False):
    cache = {}

    def solve(fe, K, KeKf, r, lam):
        if "cl" not in cache:
            cache["cl"] = Classification(fe, fe.prob["elem_part"],
                                         fe.prob["n_parts"])
        pc = BDDC(fe, KeKf[0], KeKf[1], primal, cache["cl"])
        x, its, _ = gmres(lambda v: K @ v, -r, pc.apply, tol=tol,
                          restart=restart, flexible=flexible)
        return x, its
    return solve


def newton_solve(prob, linear_solver, tol=1e-8, max_newton=25,
                 max_halvings=6, fe=None, record=None):
    """Returns (d, log) where log lists one dict per Newton step."""
    fe = fe or FEProblem(prob)
    n_steps = int(prob["load_steps"])
    d = np.zeros(fe.n_free)
    log = []
    lam_prev = 0.0
    targets = [k / n_steps for k in range(1, n_steps + 1)]
    halvings = 0
    while targets:
        lam = targets[0]
        d_try = d.copy()
        ok = False
        try:
            r = fe.residual(d_try, lam)
            r0 = np.linalg.norm(r)
            for it in range(max_newton):
                rn = np.linalg.norm(r)
                if rn <= tol * r0 or rn == 0.0:
                    ok = True
                    break
                K, KeKf = fe.tangent(d_try, lam)
                delta, its = linear_solver(fe, K, KeKf, r, lam)
                d_try = d_try + delta
                r = fe.residual(d_try, lam)
                log.append(dict(lam=lam, newton=it, res=float(rn),
                                res_new=float(np.linalg.norm(r)),
                                gmres_its=int(its), r0=float(r0)))
        except FloatingPointError:
            ok = False
        if ok:
            d = d_try
            lam_prev = lam
            targets.pop(0)
        else:
            halvings += 1
            if halvings > max_halvings:
                raise RuntimeError("Newton failed at load %g" % lam)
            targets.insert(0, 0.5 * (lam_prev + lam))
    return d, log
