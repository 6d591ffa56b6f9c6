"""A strip window computed by the oracle, for CPU tests of the strip driver
(paper_2506_18867_gb300/strip.py): the same calls as a window context of the
library (gradient, assemble_hessian, energy_rows, pcg_*, axpy, new_vec), on
CPU float64 tensors.  Only the owned rows are computed, from the window's
own rows (its state is embedded into a zero patch, so a missing or stale
halo row changes the result), and every per-row partial sum depends on its
row alone.  Test infrastructure: it runs the oracle.
"""
import numpy as np
import torch


class OracleWindow:
    def __init__(self, orc, patch, window):
        self.orc = orc
        self.prob = orc.Problem.from_patch(patch)
        self.scene = orc.Scene.from_patch(patch, project=True)
        self.nu, self.nv_patch = patch.nu, patch.nv
        self.window = tuple(int(v) for v in window)
        row0, row1, own0, own1 = self.window
        self.nv = row1 - row0
        self.N = self.nu * self.nv
        self.mass = self.prob.lumped_mass()
        self.inv_dt2 = 1.0 / patch.dt ** 2 if patch.dt > 0 else 0.0
        self.grav = np.asarray(patch.gravity, dtype=np.float64)
        self.own = np.arange(own0 * self.nu, own1 * self.nu)      # owned control points, patch numbering
        self.own_local = self.own - row0 * self.nu
        self.dtype = torch.float64

    # -- layout helpers ------------------------------------------------------
    def new_vec(self):
        return torch.zeros((3, self.N), dtype=torch.float64)

    def _embed(self, t):
        full = np.zeros((self.nu * self.nv_patch, 3))
        r0 = self.window[0] * self.nu
        full[r0:r0 + self.N] = t.numpy().T
        return full

    def _row_sums(self, v):
        """(3, n_own_cp) or (n_own_cp,) values -> one sum per owned row."""
        v = np.asarray(v).reshape(-1, len(self.own)).sum(axis=0)
        return v.reshape(-1, self.nu).sum(axis=1)

    # -- the library's calls -------------------------------------------------
    def gradient(self, C, Chat):
        g, _ = self.orc.eval_rows(self.prob, self.scene, self._embed(C), self._embed(Chat), self.own)
        out = self.new_vec()
        out[:, self.own_local] = torch.from_numpy(g.T.copy())
        return out

    def assemble_hessian(self, C, project=True):
        _, K = self.orc.eval_rows(self.prob, self.scene, self._embed(C), self._embed(C), self.own)
        return K

    def energy_rows(self, C, Chat):
        row0, row1, own0, own1 = self.window
        Su, Sv = self.nu - 2, self.nv_patch - 2
        Es, _, _ = self.prob.span_eval(self._embed(C), want_g=False, want_H=False)
        spans = [Es[b * Su:(b + 1) * Su].sum() for b in range(max(own0 - 1, 0), min(own1 - 1, Sv))]
        X, Xh = self._embed(C)[self.own], self._embed(Chat)[self.own]
        m = self.mass[self.own]
        e = -m * (X @ self.grav)
        if self.inv_dt2 > 0:
            e = e + 0.5 * m * self.inv_dt2 * ((X - Xh) ** 2).sum(axis=1)
        return np.array(spans), e.reshape(-1, self.nu).sum(axis=1)

    def pcg_begin(self, K, g, x, p):
        self.K = K
        self.Dinv = np.linalg.inv(K[:, 12])
        self.x, self.p = x, p
        self.r = -g[:, self.own_local].numpy().T.copy()
        self.z = np.einsum("kab,kb->ka", self.Dinv, self.r)
        x[:, self.own_local] = 0.0
        p[:, self.own_local] = torch.from_numpy(self.z.T.copy())
        return np.stack([self._row_sums((self.r * self.z).T), self._row_sums((self.r * self.r).T)])

    def pcg_product(self, K):
        Kf = np.zeros((self.nu * self.nv_patch, 25, 3, 3))
        Kf[self.own] = K
        y = self.orc.stencil_matvec(self.nu, self.nv_patch, Kf, self._embed(self.p))[self.own]
        self.q = y
        pv = self.p[:, self.own_local].numpy().T
        return self._row_sums((pv * y).T)

    def pcg_update(self, alpha):
        pv = self.p[:, self.own_local].numpy().T
        self.x[:, self.own_local] += torch.from_numpy((alpha * pv).T.copy())
        self.r = self.r - alpha * self.q
        self.z = np.einsum("kab,kb->ka", self.Dinv, self.r)
        return np.stack([self._row_sums((self.r * self.z).T), self._row_sums((self.r * self.r).T)])

    def pcg_direction(self, beta):
        pv = self.p[:, self.own_local].numpy().T
        self.p[:, self.own_local] = torch.from_numpy((self.z + beta * pv).T.copy())

    def axpy(self, a, d, alpha, out=None):
        if out is None:
            out = self.new_vec()
        out.copy_(a + alpha * d)
        return out
