"""Residual and exact tangent of the quasi-static cardiac mechanics problem.

Follows Section 2 of the paper:
* weak form, Eq. (mechanics weak formulation) / (mechanics time discrete),
  without the inertia term (the workloads are quasi-static load steps):
      F(d) = int_Omega P(F) : grad d*  +  int_endo p J F^{-T} N . d*
* follower pressure on the loaded surface, Eq. (bc endo): traction
  -p J F^{-T} N, written in the weak form as +p J F^{-T} N . d*,
* Newton tangent DF(d)[delta d] of Eq. (tangent problem), taken exactly.

Time-dependent terms (Section 2, time discretization), active when a time
state is set with ``set_time_state``:
* inertia  rho (d^n - 2 d^{n-1} + d^{n-2}) / dt^2 . d*  (the printed /dt is
  read as /dt^2, the dimensionally consistent backward second difference),
  with the consistent mass matrix;
* the generalized Robin condition of Eq. (bc epi) on the listed faces,
  traction -[(N x N)(K_perp d + C_perp v) + (I - N x N)(K_par d + C_par v)]
  with the reference normal N and v = (d^n - d^{n-1}) / dt; without a time
  state only the spring part (v = 0) acts.

Free degrees of freedom: nodes in increasing id, Dirichlet nodes removed,
three interleaved components per node (Section 4, block size 3).
"""
import numpy as np
import scipy.sparse as sp

from . import elements as el
from . import material as mat


class FEProblem:
    """Geometry, quadrature and fibres of one workload (all FP64)."""

    def __init__(self, prob):
        self.prob = prob
        self.k = el.element_order(prob["elem_type"])
        self.coords = np.asarray(prob["coords"], dtype=float)
        self.elems = np.asarray(prob["elems"], dtype=np.int64)
        self.n_nodes = self.coords.shape[0]
        self.n_el, self.n_en = self.elems.shape
        self.par = prob["material"]
        # free-DoF numbering
        is_dir = np.zeros(self.n_nodes, dtype=bool)
        is_dir[np.asarray(prob["dirichlet_nodes"], dtype=np.int64)] = True
        self.is_dirichlet = is_dir
        self.free_nodes = np.nonzero(~is_dir)[0]
        self.node_to_free = -np.ones(self.n_nodes, dtype=np.int64)
        self.node_to_free[self.free_nodes] = np.arange(self.free_nodes.size)
        self.n_free = 3 * self.free_nodes.size
        # volume quadrature
        et = prob["elem_type"]
        pts, wts = el.volume_rule(et)
        N, dN = el.shape(et, pts)
        Xe = self.coords[self.elems]                       # (ne, nen, 3)
        J0 = np.einsum("eai,qaj->eqij", Xe, dN)           # dX_i/dxi_j
        self.detJ0 = np.linalg.det(J0)
        if np.any(self.detJ0 <= 0):
            raise ValueError("inverted reference element")
        invJ0 = np.linalg.inv(J0)                          # dxi_j/dX_i
        self.dNdX = np.einsum("qaj,eqji->eqai", dN, invJ0)
        self.wdet = wts[None, :] * self.detJ0
        Xq = np.einsum("qa,eai->eqi", N, Xe)
        fib = prob["fibers"]
        if fib["kind"] == "nodal":
            # nodal directions interpolated to the quadrature points
            fq = np.einsum("qa,eai->eqi", N, np.asarray(fib["f"], dtype=float)[self.elems])
            nq = np.einsum("qa,eai->eqi", N, np.asarray(fib["n"], dtype=float)[self.elems])
            self.R = mat.nodal_fiber_frame(fq, nq)
        else:
            self.R = mat.fiber_frame(fib, Xq)              # (ne, nq, 3, 3)
        # pressure faces: volume shape data at face quadrature points
        self.faces = []
        for e, f in np.asarray(prob["pressure_faces"], dtype=np.int64):
            fp, fw, es, et_ = el.face_rule(et, int(f))
            Nf, dNf = el.shape(et, fp)
            J0f = np.einsum("ai,qaj->qij", Xe[e], dNf)
            dNdXf = np.einsum("qaj,qji->qai", dNf, np.linalg.inv(J0f))
            Xs = J0f @ es
            Xt = J0f @ et_
            Aref = np.cross(Xs, Xt)                        # N dA / (ds dt)
            self.faces.append((int(e), Nf, dNdXf, Aref, fw))
        # Robin faces: reference normal, area weights, shape values; the
        # parameter set of each face (K_perp, K_par, C_perp, C_par)
        self.robin = []
        sets = prob.get("robin", [])
        for e, f, k in np.asarray(prob.get("robin_faces", np.zeros((0, 3))), dtype=np.int64).reshape(-1, 3):
            fp, fw, es, et_ = el.face_rule(et, int(f))
            Nf, dNf = el.shape(et, fp)
            J0f = np.einsum("ai,qaj->qij", Xe[e], dNf)
            Aref = np.cross(J0f @ es, J0f @ et_)
            area = np.linalg.norm(Aref, axis=1)
            self.robin.append((int(e), Nf, Aref / area[:, None], fw * area, sets[int(k)]))
        # consistent mass: shape values at the volume points
        self.Nq = N
        self.rho = float(prob.get("rho", 0.0))
        self.time = None

    def set_time_state(self, dt, d_prev, d_prev2):
        """Backward-Euler time step dt with the two previous displacements
        (free-DoF vectors); dt = None returns to the quasi-static problem."""
        if dt is None:
            self.time = None
        else:
            self.time = (float(dt), np.asarray(d_prev, dtype=float), np.asarray(d_prev2, dtype=float))

    def _robin_matrix(self, Nn, par, dt):
        """3x3 stiffness of the Robin traction at one point, d g / d d^n."""
        kp = par["k_perp"] + (par["c_perp"] / dt if dt else 0.0)
        kt = par["k_par"] + (par["c_par"] / dt if dt else 0.0)
        nn = np.einsum("qi,qk->qik", Nn, Nn)
        return kp * nn + kt * (np.eye(3) - nn)

    # -- helpers ---------------------------------------------------------
    def full_displacement(self, d_free):
        """Free-DoF vector -> (n_nodes, 3) displacement with zeros on
        Dirichlet nodes."""
        u = np.zeros((self.n_nodes, 3))
        u[self.free_nodes] = np.asarray(d_free).reshape(-1, 3)
        return u

    def to_free(self, v_nodes):
        return v_nodes[self.free_nodes].reshape(-1)

    def deformation_gradient(self, u):
        de = u[self.elems]
        return np.eye(3) + np.einsum("eai,eqaJ->eqiJ", de, self.dNdX)

    # -- residual --------------------------------------------------------
    def element_residuals(self, d_free, lam):
        """Per-element residual contributions (ne, nen, 3) and per-face ones
        (list of (elem, (nen, 3)))."""
        u = self.full_displacement(d_free)
        F = self.deformation_gradient(u)
        if np.any(np.linalg.det(F) <= 0):
            raise FloatingPointError("J <= 0 at a quadrature point")
        gamma = lam * self.prob["gamma"]
        P = mat.first_pk(F, self.R, self.par, gamma)
        re = np.einsum("eqiJ,eqaJ,eq->eai", P, self.dNdX, self.wdet)
        p = lam * self.prob["pressure"]
        rf = []
        for e, Nf, dNdXf, Aref, fw in self.faces:
            Ff = np.eye(3) + np.einsum("ai,qaJ->qiJ", u[self.elems[e]], dNdXf)
            Jf = np.linalg.det(Ff)
            cof = Jf[:, None, None] * np.swapaxes(np.linalg.inv(Ff), -1, -2)
            t = p * np.einsum("qiJ,qJ->qi", cof, Aref)     # p J F^-T N dA
            rf.append((e, np.einsum("q,qa,qi->ai", fw, Nf, t)))
        if self.time is not None and self.rho > 0.0:
            dt, dp, dpp = self.time
            acc = self.full_displacement(np.asarray(d_free) - 2.0 * dp + dpp)
            aq = np.einsum("qa,eai->eqi", self.Nq, acc[self.elems])
            re = re + self.rho / dt ** 2 * np.einsum("qa,eqi,eq->eai", self.Nq, aq, self.wdet)
        if self.robin:
            dt = self.time[0] if self.time is not None else None
            vel = self.full_displacement((np.asarray(d_free) - self.time[1]) / dt) if dt else None
            for e, Nf, Nn, wa, par in self.robin:
                uq = Nf @ u[self.elems[e]]
                nn = np.einsum("qi,qk->qik", Nn, Nn)
                tan = np.eye(3) - nn
                g = par["k_perp"] * np.einsum("qik,qk->qi", nn, uq) + par["k_par"] * np.einsum("qik,qk->qi", tan, uq)
                if vel is not None:
                    vq = Nf @ vel[self.elems[e]]
                    g = g + par["c_perp"] * np.einsum("qik,qk->qi", nn, vq) + par["c_par"] * np.einsum("qik,qk->qi", tan, vq)
                rf.append((e, np.einsum("q,qa,qi->ai", wa, Nf, g)))
        return re, rf

    def residual(self, d_free, lam):
        re, rf = self.element_residuals(d_free, lam)
        r = np.zeros((self.n_nodes, 3))
        np.add.at(r, self.elems, re)
        for e, v in rf:
            np.add.at(r, self.elems[e], v)
        return self.to_free(r)

    # -- tangent ---------------------------------------------------------
    def element_tangents(self, d_free, lam):
        """Element matrices (ne, nen, 3, nen, 3) and face matrices (list of
        (elem, (nen, 3, nen, 3)))."""
        u = self.full_displacement(d_free)
        F = self.deformation_gradient(u)
        gamma = lam * self.prob["gamma"]
        A = mat.tangent(F, self.R, self.par, gamma)
        Ke = np.einsum("eqaJ,eqiJkL,eqbL,eq->eaibk", self.dNdX, A,
                       self.dNdX, self.wdet, optimize=True)
        p = lam * self.prob["pressure"]
        Kf = []
        for e, Nf, dNdXf, Aref, fw in self.faces:
            Ff = np.eye(3) + np.einsum("ai,qaJ->qiJ", u[self.elems[e]], dNdXf)
            Jf = np.linalg.det(Ff)
            Fi = np.linalg.inv(Ff)
            # d cof_iJ / d F_kL = J (Finv_Lk Finv_Ji - Finv_Jk Finv_Li)
            dcof = Jf[:, None, None, None, None] * (
                np.einsum("qLk,qJi->qiJkL", Fi, Fi)
                - np.einsum("qJk,qLi->qiJkL", Fi, Fi))
            dt = p * np.einsum("qiJkL,qJ->qikL", dcof, Aref)
            Kf.append((e, np.einsum("q,qa,qikL,qbL->aibk", fw, Nf, dt,
                                    dNdXf)))
        if self.time is not None and self.rho > 0.0:
            dt = self.time[0]
            M = np.einsum("qa,qb,eq->eab", self.Nq, self.Nq, self.wdet)
            Ke = Ke + self.rho / dt ** 2 * np.einsum("eab,ik->eaibk", M, np.eye(3))
        dt = self.time[0] if self.time is not None else None
        for e, Nf, Nn, wa, par in self.robin:
            Kq = self._robin_matrix(Nn, par, dt)
            Kf.append((e, np.einsum("q,qa,qik,qb->aibk", wa, Nf, Kq, Nf)))
        return Ke, Kf

    def assemble(self, Ke, Kf, elem_subset=None, dof_map=None, n_dof=None):
        """Sum element/face matrices into a sparse matrix.

        By default over all elements, in the global free-DoF numbering.
        ``elem_subset`` (bool mask or index array) restricts the sum, and
        ``dof_map`` (node-DoF index 3*node+comp -> target index or -1) with
        ``n_dof`` renumbers it (used for the subdomain matrices A^(i))."""
        if dof_map is None:
            dof_map = -np.ones(3 * self.n_nodes, dtype=np.int64)
            fn = self.free_nodes
            for c in range(3):
                dof_map[3 * fn + c] = 3 * np.arange(fn.size) + c
            n_dof = self.n_free
        if elem_subset is None:
            sel = np.arange(self.n_el)
        else:
            sel = np.asarray(elem_subset)
            if sel.dtype == bool:
                sel = np.nonzero(sel)[0]
        rows, cols, vals = [], [], []
        nen = self.n_en

        def add(nodes, K):
            gd = (3 * nodes[:, None] + np.arange(3)[None, :]).reshape(-1)
            m = dof_map[gd]
            Kr = K.reshape(nen * 3, nen * 3)
            ok = m >= 0
            ii, jj = np.nonzero(ok[:, None] & ok[None, :])
            rows.append(m[ii])
            cols.append(m[jj])
            vals.append(Kr[ii, jj])

        # vectorised element part
        if sel.size:
            nodes = self.elems[sel]
            gd = (3 * nodes[:, :, None] + np.arange(3)[None, None, :]).reshape(
                sel.size, -1)
            m = dof_map[gd]
            Kr = Ke[sel].reshape(sel.size, nen * 3, nen * 3)
            R = np.broadcast_to(m[:, :, None], Kr.shape)
            C = np.broadcast_to(m[:, None, :], Kr.shape)
            ok = (R >= 0) & (C >= 0)
            rows.append(R[ok])
            cols.append(C[ok])
            vals.append(Kr[ok])
        in_sel = np.zeros(self.n_el, dtype=bool)
        in_sel[sel] = True
        for e, K in Kf:
            if in_sel[e]:
                add(self.elems[e], K)
        if rows:
            rows = np.concatenate(rows)
            cols = np.concatenate(cols)
            vals = np.concatenate(vals)
        A = sp.coo_matrix((vals, (rows, cols)), shape=(n_dof, n_dof))
        return A.tocsr()

    def tangent(self, d_free, lam):
        Ke, Kf = self.element_tangents(d_free, lam)
        return self.assemble(Ke, Kf), (Ke, Kf)

    def min_jacobian(self, d_free):
        u = self.full_displacement(d_free)
        return float(np.min(np.linalg.det(self.deformation_gradient(u))))
