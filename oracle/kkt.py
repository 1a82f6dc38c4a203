"""Dense KKT linear algebra of the oracle.  Test infrastructure (see oracle/__init__.py).

The primal-dual Newton system of one interior-point iteration (Wachter & Biegler 2006,
Eq. (13) with the regularisations of their Section 3.1) for problem (10) is

    [ W_s + Sig_s + dw I    0          J_s^T ] [dz_s]   [r_z,s]
    [ 0                     K_dd       b_s^T ] [dd  ] = [r_d  ]      for every scenario s
    [ J_s                   b_s     -dc I    ] [dl_s]   [r_c,s]

where b_s = dc_s/dd.  Only d couples the scenarios (the replicated structure of
Section "Replicated scenario structure"), so the system is bordered block diagonal.
The oracle factors every scenario block

    K_s = [ W_s + Sig_s + dw I , J_s^T ; J_s , -dc I ]      (440 x 440, dense)

with the Bunch-Kaufman symmetric-indefinite LDL^T of LAPACK (scipy.linalg.ldl), reads
its inertia from the 1x1 / 2x2 pivots (Sylvester's law of inertia), and eliminates the
scenarios onto d with a scalar Schur complement

    S_d = K_dd - sum_s bh_s^T K_s^{-1} bh_s,    bh_s = [0; b_s]

whose sign completes the inertia of the whole matrix (Haynsworth inertia additivity).

With a design vector of K entries (the general Eq. (8), dim theta > 1) the border is
b_s = dc_s/dtheta (220 x K), K_dd a K x K block, and the Schur complement the K x K
matrix S_theta = K_dd + dw I - sum_s bh_s^T K_s^{-1} bh_s, whose eigenvalue signs complete
the inertia; the solve takes dtheta from S_theta dtheta = r_theta - sum_s bh_s^T v_s.  A
2-D Jd (K = 1) keeps the scalar shapes throughout.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla


class BlockLDL:
    """Bunch-Kaufman LDL^T of one dense symmetric matrix: A = lu d lu^T, lu[perm] lower
    unit triangular, d block diagonal with 1x1 and 2x2 blocks."""

    def __init__(self, A):
        self.n = A.shape[0]
        self.lu, self.d, self.perm = sla.ldl(A, lower=True, hermitian=False)
        self.Lp = self.lu[self.perm]
        # d is tridiagonal (its 2x2 pivot blocks straddle the diagonal): banded form
        n = self.n
        self.dband = np.zeros((3, n))
        self.dband[0, 1:] = np.diag(self.d, 1)
        self.dband[1, :] = np.diag(self.d)
        self.dband[2, :-1] = np.diag(self.d, -1)

    def inertia(self, zero_tol=0.0):
        """(n_pos, n_neg, n_zero) from the eigenvalues of the pivot blocks of d."""
        d = self.d
        n = self.n
        pos = neg = zero = 0
        i = 0
        while i < n:
            if i + 1 < n and d[i + 1, i] != 0.0:
                ev = np.linalg.eigvalsh(d[i:i + 2, i:i + 2])
                i += 2
            else:
                ev = [d[i, i]]
                i += 1
            for e in ev:
                if abs(e) <= zero_tol:
                    zero += 1
                elif e > 0:
                    pos += 1
                else:
                    neg += 1
        return pos, neg, zero

    def solve(self, b):
        y = sla.solve_triangular(self.Lp, b[self.perm], lower=True, unit_diagonal=True)
        w = sla.solve_banded((1, 1), self.dband, y)
        xp = sla.solve_triangular(self.Lp.T, w, lower=False, unit_diagonal=True)
        x = np.empty_like(xp)
        x[self.perm] = xp
        return x


def scenario_matrix(W, sig, J, dw, dc):
    """K_s = [W + diag(sig) + dw I, J^T; J, -dc I]."""
    n = W.shape[0]
    m = J.shape[0]
    K = np.zeros((n + m, n + m))
    K[:n, :n] = W + np.diag(sig + dw)
    K[n:, :n] = J
    K[:n, n:] = J.T
    K[n:, n:] = -dc * np.eye(m)
    return K


def _border(Jd):
    """b_s as (S, n, K) and whether the shapes are scalar (K = 1 given as (S, n))."""
    return (Jd[:, :, None], True) if Jd.ndim == 2 else (Jd, False)


class SchurKKT:
    """Factorization of the bordered block-diagonal KKT matrix by per-scenario dense
    Bunch-Kaufman LDL^T plus the Schur complement on the design vector (a scalar for d,
    K x K for K sections)."""

    def __init__(self, W, sig, J, Jd, Kdd, dw, dc, zero_tol=0.0):
        S, n, _ = W.shape
        self.S, self.n = S, n
        b3, self.scalar = _border(Jd)
        K = b3.shape[2]
        self.facs = []
        self.inertia_blocks = [0, 0, 0]
        self.U = np.zeros((S, 2 * n, K))
        self.bh = np.zeros((S, 2 * n, K))
        self.bh[:, n:, :] = b3
        for s in range(S):
            f = BlockLDL(scenario_matrix(W[s], sig[s], J[s], dw, dc))
            for k, v in enumerate(f.inertia(zero_tol)):
                self.inertia_blocks[k] += v
            self.facs.append(f)
            self.U[s] = f.solve(self.bh[s])
        # Schur complement of the scenario blocks in the full matrix (K x K)
        self.Smat = (np.atleast_2d(Kdd) + dw * np.eye(K)) - np.einsum("sik,sil->kl", self.bh, self.U)
        self.Sd = float(self.Smat[0, 0]) if self.scalar else self.Smat

    def inertia(self):
        p, m, z = self.inertia_blocks
        for e in np.linalg.eigvalsh(0.5 * (self.Smat + self.Smat.T)):
            if e > 0:
                p += 1
            elif e < 0:
                m += 1
            else:
                z += 1
        return p, m, z

    def solve(self, rz, rd, rc):
        """Solve for (dz (S,n), dd, dl (S,n)) given right-hand sides of the same shapes
        (rd and dd scalars for K = 1, else K-vectors)."""
        S, n = self.S, self.n
        V = np.zeros((S, 2 * n))
        for s in range(S):
            V[s] = self.facs[s].solve(np.concatenate([rz[s], rc[s]]))
        t = np.einsum("sik,si->k", self.bh, V)
        dd = np.linalg.solve(self.Smat, np.atleast_1d(rd) - t)
        X = V - np.einsum("sik,k->si", self.U, dd)
        return X[:, :n], (float(dd[0]) if self.scalar else dd), X[:, n:]


def kkt_residual(W, sig, J, Jd, Kdd, dw, dc, dz, dd, dl, rz, rd, rc):
    """r - K x of the bordered block-diagonal system above, by its block rows:
    z rows (W + Sig + dw I) dz + J^T dl, the design rows (K_dd + dw I) dd + sum b^T dl and
    the constraint rows J dz + b dd - dc dl."""
    b3, scalar = _border(Jd)
    K = b3.shape[2]
    ddv = np.atleast_1d(dd)
    ez = rz - (np.einsum("sij,sj->si", W, dz) + (sig + dw) * dz + np.einsum("sri,sr->si", J, dl))
    ed = np.atleast_1d(rd) - ((np.atleast_2d(Kdd) + dw * np.eye(K)) @ ddv + np.einsum("srk,sr->k", b3, dl))
    ec = rc - (np.einsum("sri,si->sr", J, dz) + np.einsum("srk,k->sr", b3, ddv) - dc * dl)
    return ez, (float(ed[0]) if scalar else ed), ec


def solve_refined(fac, W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc, steps=2):
    """The Schur-reduced solve followed by `steps` rounds of FP64 iterative refinement
    on the whole system (residual by kkt_residual, correction by the same factors): the
    direction the GPU's refined solve is compared with when the KKT matrix is too
    ill-conditioned for an unrefined backward-stable solve to agree with another to
    1e-10."""
    dz, dd, dl = fac.solve(rz, rd, rc)
    for _ in range(steps):
        ez, ed, ec = kkt_residual(W, sig, J, Jd, Kdd, dw, dc, dz, dd, dl, rz, rd, rc)
        cz, cd, cl = fac.solve(ez, ed, ec)
        dz, dd, dl = dz + cz, dd + cd, dl + cl
    return dz, dd, dl


def monolithic_matrix(W, sig, J, Jd, Kdd, dw, dc):
    """The whole KKT matrix, dense, unknowns ordered [d (K entries), (z_s, l_s) for each s]."""
    S, n, _ = W.shape
    b3, _ = _border(Jd)
    nk = b3.shape[2]
    N = nk + 2 * n * S
    K = np.zeros((N, N))
    K[:nk, :nk] = np.atleast_2d(Kdd) + dw * np.eye(nk)
    for s in range(S):
        o = nk + 2 * n * s
        K[o:o + 2 * n, o:o + 2 * n] = scenario_matrix(W[s], sig[s], J[s], dw, dc)
        K[o + n:o + 2 * n, :nk] = b3[s]
        K[:nk, o + n:o + 2 * n] = b3[s].T
    return K


def monolithic_solve(W, sig, J, Jd, Kdd, dw, dc, rz, rd, rc):
    """Dense Bunch-Kaufman LDL^T of the whole matrix (no Schur step); for tiny S only.
    Returns (dz, dd, dl, inertia)."""
    S, n, _ = W.shape
    b3, scalar = _border(Jd)
    nk = b3.shape[2]
    K = monolithic_matrix(W, sig, J, Jd, Kdd, dw, dc)
    rhs = np.zeros(K.shape[0])
    rhs[:nk] = np.atleast_1d(rd)
    for s in range(S):
        o = nk + 2 * n * s
        rhs[o:o + n] = rz[s]
        rhs[o + n:o + 2 * n] = rc[s]
    f = BlockLDL(K)
    x = f.solve(rhs)
    dz = np.stack([x[nk + 2 * n * s:nk + 2 * n * s + n] for s in range(S)])
    dl = np.stack([x[nk + 2 * n * s + n:nk + 2 * n * (s + 1)] for s in range(S)])
    return dz, (float(x[0]) if scalar else x[:nk].copy()), dl, f.inertia()
