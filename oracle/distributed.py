"""BDDC split over processes, emulated on CPU ranks (test infrastructure).

The paper runs one subdomain per MPI process on an unassembled (MATIS)
matrix, Section 4, and solves the coarse problem on a sub-communicator,
Section 7.  This module spreads the two-level BDDC of ``oracle.bddc`` over
the ranks of a ``torch.distributed`` process group (gloo, CPU) the way a
multi-GPU run would:

* rank q owns a contiguous block of subdomains (``owned``) and works on
  those only: interior solves, restriction, constrained local solves,
  coarse right-hand-side contributions, prolongation, harmonic extension,
  and the unassembled operator product sum_i R_i^T A^(i) R_i x;
* interface sums (step 2, g = r_G - sum_i R_i^T A_GI u0_i, and step 6,
  z_G = sum_i R_i^T D_i w_i) and the assembled operator product are the
  exchanges: every rank contributes its subdomains' terms to a global
  vector and the contributions are gathered and added in rank order
  (an all-gather, so every rank's sum is the same to the bit);
* coarse problem: the ranks' contributions sum_i R_Pi^T Psi_i^T g_i are
  all-gathered and every rank solves the small dense coarse system
  redundantly (no broadcast of the solution).

Vectors are replicated on every rank here (the emulation exchanges whole
vectors instead of only the interface values a real split would send);
each rank's arithmetic is restricted to its own subdomains, and only the
exchanges above combine them.  Setup is done per rank for its subdomains
from the same global description (``oracle.bddc.BDDC``, whose coarse
matrix every rank needs for the redundant solve).
"""
import numpy as np


def owned(n_parts, rank, world):
    """Contiguous block of subdomains of a rank: [lo, hi)."""
    lo = (n_parts * rank) // world
    hi = (n_parts * (rank + 1)) // world
    return lo, hi


def _gather_sum(x, dist, group=None):
    """Sum of x over all ranks, added in rank order (all-gather)."""
    import torch
    world = dist.get_world_size(group)
    t = torch.as_tensor(np.ascontiguousarray(x, dtype=np.float64))
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t, group=group)
    out = np.zeros_like(x, dtype=np.float64)
    for p in parts:
        out = out + p.numpy()
    return out


class DistributedBDDC:
    """Apply and operator product of a two-level ``oracle.bddc.BDDC`` over
    the ranks of ``dist`` (torch.distributed, initialised)."""

    def __init__(self, bddc, dist, group=None):
        if bddc.coarse is not None:
            raise ValueError("the emulated split covers the two-level method")
        self.b = bddc
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.lo, self.hi = owned(len(bddc.subs), self.rank, self.world)
        self.subs = bddc.subs[self.lo:self.hi]
        self.exchanged = 0  # doubles each rank contributed to exchanges

    def _sum(self, x):
        self.exchanged += x.size
        return _gather_sum(x, self.dist, self.group)

    def matvec(self, x):
        """sum_i R_i^T A^(i) R_i x over all subdomains (unassembled form)."""
        x = np.asarray(x, dtype=float)
        y = np.zeros_like(x)
        for sub in self.subs:
            gd = sub["gdof"]
            np.add.at(y, gd, sub["A"] @ x[gd])
        return self._sum(y)

    def apply(self, r):
        b = self.b
        r = np.asarray(r, dtype=float)
        # 1-2. interior solves of owned subdomains, interface sum of g
        dg = np.zeros_like(r)
        u0 = []
        for sub in self.subs:
            gd = sub["gdof"]
            if sub["luII"] is not None:
                u = sub["luII"].solve(r[gd[sub["ldofI"]]])
                np.add.at(dg, gd[sub["ldofG"]], -(sub["AGI"] @ u))
            else:
                u = np.zeros(0)
            u0.append(u)
        g = r + self._sum(dg)
        # 3-4. restriction and constrained local solves, coarse contributions
        c = np.zeros(b.n_pi)
        ws = []
        for sub in self.subs:
            gd = sub["gdof"]
            f = np.zeros(gd.size)
            fG = sub["Dg"] * g[gd[sub["ldofG"]]]
            for pos, D in sub.get("deluxe", ()):
                fG[pos] = D.T @ fG[pos]
            f[sub["ldofG"]] = fG
            ws.append(b._local_solve(sub, f))
            if sub["gP"].size:
                np.add.at(c, sub["gP"], sub["Psi"].T @ f)
        # 5. coarse all-gather and redundant coarse solve on every rank
        uc = b.coarse_solve(self._sum(c))
        # 6. prolongation, scaling, interface sum of z_G
        zG = np.zeros_like(r)
        for sub, w in zip(self.subs, ws):
            gd = sub["gdof"]
            if sub["gP"].size:
                w = w + sub["Phi"] @ uc[sub["gP"]]
            yG = sub["Dg"] * w[sub["ldofG"]]
            for pos, D in sub.get("deluxe", ()):
                yG[pos] = D @ yG[pos]
            np.add.at(zG, gd[sub["ldofG"]], yG)
        zG = self._sum(zG)
        # 7. harmonic extension of owned subdomains (interior DoFs belong to
        # one subdomain each), assembled for the caller
        zI = np.zeros_like(r)
        for sub in self.subs:
            gd = sub["gdof"]
            if sub["luII"] is not None:
                zI[gd[sub["ldofI"]]] = sub["luII"].solve(r[gd[sub["ldofI"]]]
                                                         - sub["AIG"] @ zG[gd[sub["ldofG"]]])
        return zG + self._sum(zI)
