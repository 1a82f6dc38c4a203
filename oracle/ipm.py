"""Primal-dual interior-point solve of problem (10), plain and slow.  Test infrastructure.

The method is the filter line-search interior-point algorithm of Wachter & Biegler,
"On the implementation of an interior-point filter line-search algorithm for large-scale
nonlinear programming", Math. Program. 106 (2006) (the published method of Ipopt, the
solver family the paper's MadNLP belongs to), with that paper's default constants:

  * barrier problem min phi_mu = w d - mu sum ln(x - x^L) - mu sum ln(x^U - x), c(x) = 0,
    with the objective scaled by w = S (Ipopt's objective scaling factor; the solution is
    unchanged): unscaled, the barrier terms of the 10 S hydraulic slacks outweigh the
    single objective d until mu << d*/(20 S), so the early central path sits at d's upper
    bound for large S; with w = S it tracks d* for every S;
  * optimality error E_mu with the s_max = 100 scaling, stop when E_0 <= tol = 1e-8 (the
    paper's solver tolerance, Section "Numerical results");
  * monotone barrier update mu <- max(tol/10, min(kappa_mu mu, mu^theta_mu)) while
    E_mu <= kappa_eps mu, tau = max(tau_min, 1 - mu);
  * Newton step from the primal-dual system with bound multipliers eliminated, inertia
    correction of delta_w / delta_c (their Algorithm IC);
  * fraction-to-the-boundary step sizes, backtracking filter line search with the
    switching condition and Armijo rule, filter augmentation, the kappa_Sigma reset of
    the bound multipliers.
  * second-order corrections (their Section 2.4): when the first trial point is rejected
    and increases theta, up to p_max = 4 corrected steps from the same factorization with
    right-hand side c_soc = alpha c(x) + c(x + alpha dx), accepted by the same tests.
  * feasibility restoration (their Section 3.3) when the line search falls below alpha_min:
    the failed iterate's entry joins the filter, then damped Newton steps on the square
    constraint system with d fixed (IPM.restoration) until the point is acceptable to the
    filter with theta reduced by the factor 1 - gamma_theta; a restoration that fails
    stops the solve with status "linesearch".
Not included (as in the GPU path): the watchdog.

Starting point (the paper says only that all configurations used the same one): for
S > 1 the stage states of the expected-value problem's solution (one scenario with the
mean feed, itself solved from the inlet-copy start), see IPM.basecase_start; for S = 1
the inlet-copy start of model.initial_point.

Unknowns: the diameter d (bounds (10c)) and the per-scenario z (S, 220) of model.py with
bounds (10d).  The KKT systems are solved by kkt.SchurKKT (dense per-scenario
Bunch-Kaufman LDL^T + scalar Schur complement on d).

With P["n_sections"] = K > 1 the design vector is the K section diameters theta_k (model.py),
each with the bounds of d, and the objective sum_k w_k theta_k with w_k the sections'
shares of the stages; d, z_L(d), z_U(d) are then K-arrays (floats for K = 1) and the
Schur complement is K x K.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import kkt, model


@dataclass
class Options:
    tol: float = 1e-8
    max_iter: int = 300
    mu_init: float = 0.1
    kappa_eps: float = 10.0
    kappa_mu: float = 0.2
    theta_mu: float = 1.5
    tau_min: float = 0.99
    s_max: float = 100.0
    kappa_sigma: float = 1e10
    bound_push: float = 1e-2
    bound_frac: float = 1e-2
    gamma_theta: float = 1e-5
    gamma_phi: float = 1e-5
    delta: float = 1.0
    s_theta: float = 1.1
    s_phi: float = 2.3
    eta_phi: float = 1e-4
    gamma_alpha: float = 0.05
    lam_init_max: float = 1e3
    dw0: float = 1e-4
    dw_min: float = 1e-20
    dw_max: float = 1e40
    kw_minus: float = 1.0 / 3.0
    kw_plus: float = 8.0
    kw_plus_bar: float = 100.0
    dc_bar: float = 1e-8
    kappa_c: float = 0.25
    max_ls: int = 60
    soc_max: int = 4
    kappa_soc: float = 0.99
    resto_max: int = 20                # feasibility restoration iterations (0: none)
    obj_scaling: float | None = None   # None: the number of scenarios S
    init: str = "basecase"             # "basecase" (S > 1) or "inlet"
    verbose: bool = False


@dataclass
class State:
    d: float
    Z: np.ndarray
    lam: np.ndarray
    zL: np.ndarray
    zU: np.ndarray
    zLd: float
    zUd: float


@dataclass
class Result:
    status: str
    iters: int
    d: float
    Z: np.ndarray
    lam: np.ndarray
    zL: np.ndarray
    zU: np.ndarray
    zLd: float
    zUd: float
    E0: float
    mu: float
    history: list = field(default_factory=list)
    base_iters: int = 0


class Problem:
    """Data of one instance: parameters P, feeds F (18, S), bounds."""

    def __init__(self, P, F, w=1.0):
        self.P, self.F = P, F
        self.w = w                   # objective scaling: the solver minimises w * d
        self.S = F.shape[1]
        self.n = model.NS
        self.K = model.n_sections(P)
        self.wsec = model.section_weights(self.K)
        self.lo, self.hi, self.dlo, self.dhi = model.bounds(P, self.S)
        self.hasL = np.isfinite(self.lo)
        self.hasU = np.isfinite(self.hi)
        self.nL = int(self.hasL.sum()) + self.K   # + the design entries
        self.nU = int(self.hasU.sum()) + self.K
        self.m = self.S * self.n

    def th(self, v):
        """A design-vector quantity in the stored form: a float for K = 1, else an array."""
        v = np.atleast_1d(np.asarray(v, dtype=float))
        return float(v[0]) if self.K == 1 else v.copy()

    # slacks to the bounds (1 where there is no bound, never used)
    def sl(self, Z):
        return np.where(self.hasL, Z - np.where(self.hasL, self.lo, 0.0), 1.0)

    def su(self, Z):
        return np.where(self.hasU, np.where(self.hasU, self.hi, 0.0) - Z, 1.0)


def push_into_bounds(pr, opt, Z, d):
    """Initial-point projection (Wachter & Biegler 2006, Section 3.6)."""
    lo, hi = pr.lo, pr.hi
    width = np.where(pr.hasL & pr.hasU, hi - lo, np.inf)
    pL = np.minimum(opt.bound_push * np.maximum(1.0, np.abs(np.where(pr.hasL, lo, 0.0))),
                    opt.bound_frac * width)
    pU = np.minimum(opt.bound_push * np.maximum(1.0, np.abs(np.where(pr.hasU, hi, 0.0))),
                    opt.bound_frac * width)
    Z = np.where(pr.hasL, np.maximum(Z, np.where(pr.hasL, lo, 0.0) + pL), Z)
    Z = np.where(pr.hasU, np.minimum(Z, np.where(pr.hasU, hi, 0.0) - pU), Z)
    wd = pr.dhi - pr.dlo
    pdl = min(opt.bound_push * max(1.0, abs(pr.dlo)), opt.bound_frac * wd)
    pdu = min(opt.bound_push * max(1.0, abs(pr.dhi)), opt.bound_frac * wd)
    d = np.minimum(np.maximum(np.broadcast_to(np.atleast_1d(d), (pr.K,)), pr.dlo + pdl), pr.dhi - pdu)
    return Z, pr.th(d)


def jd_t(Jd, lam):
    """sum_s b_s^T lam_s: a float for 2-D Jd (K = 1), a K-array for 3-D."""
    v = np.einsum("sr...,sr->...", Jd, lam)
    return float(v) if np.ndim(v) == 0 else v


def dual_residual(pr, st, J, Jd):
    """grad f + J^T lam - z_L + z_U for z (S, n) and for d (K-array)."""
    rz = np.einsum("src,sr->sc", J, st.lam) - st.zL + st.zU
    rd = pr.w * pr.wsec + np.atleast_1d(jd_t(Jd, st.lam)) - np.atleast_1d(st.zLd) + np.atleast_1d(st.zUd)
    return rz, rd


def optimality_error(pr, opt, st, C, J, Jd, mu):
    """E_mu of Wachter & Biegler (2006), Eq. (5), with the s_d, s_c scalings."""
    rz, rd = dual_residual(pr, st, J, Jd)
    sl, su = pr.sl(st.Z), pr.su(st.Z)
    cl = np.where(pr.hasL, st.zL * sl - mu, 0.0)
    cu = np.where(pr.hasU, st.zU * su - mu, 0.0)
    dv, zLd, zUd = np.atleast_1d(st.d), np.atleast_1d(st.zLd), np.atleast_1d(st.zUd)
    cld = zLd * (dv - pr.dlo) - mu
    cud = zUd * (pr.dhi - dv) - mu
    zsum = float(np.abs(st.zL).sum() + np.abs(st.zU).sum() + np.abs(zLd).sum() + np.abs(zUd).sum())
    s_d = max(opt.s_max, (float(np.abs(st.lam).sum()) + zsum) / (pr.m + pr.nL + pr.nU)) / opt.s_max
    s_c = max(opt.s_max, zsum / (pr.nL + pr.nU)) / opt.s_max
    dual = max(float(np.abs(rz).max(initial=0.0)), float(np.abs(rd).max())) / s_d
    primal = float(np.abs(C).max(initial=0.0))
    compl = max(float(np.abs(cl).max(initial=0.0)), float(np.abs(cu).max(initial=0.0)),
                float(np.abs(cld).max()), float(np.abs(cud).max())) / s_c
    return max(dual, primal, compl), dual, primal, compl


def barrier_phi(pr, Z, d, mu):
    sl, su = pr.sl(Z), pr.su(Z)
    dv = np.atleast_1d(d)
    b = np.sum(np.log(sl[pr.hasL])) + np.sum(np.log(su[pr.hasU]))
    b += float(np.sum(np.log(dv - pr.dlo)) + np.sum(np.log(pr.dhi - dv)))
    return pr.w * float(pr.wsec @ dv) - mu * b


def fraction_to_boundary(pr, x, dx, lo_mask, lo, hi_mask, hi, tau):
    """Largest alpha in (0, 1] with x + alpha dx >= (1 - tau)(x - lo) kept inside."""
    a = 1.0
    sl = np.where(lo_mask, x - np.where(lo_mask, lo, 0.0), 1.0)
    neg = lo_mask & (dx < 0)
    if np.any(neg):
        a = min(a, float(np.min(-tau * sl[neg] / dx[neg])))
    su = np.where(hi_mask, np.where(hi_mask, hi, 0.0) - x, 1.0)
    pos = hi_mask & (dx > 0)
    if np.any(pos):
        a = min(a, float(np.min(tau * su[pos] / dx[pos])))
    return a


class IPM:
    def __init__(self, P, F, opt: Options | None = None):
        self.opt = opt or Options()
        w = float(F.shape[1]) if self.opt.obj_scaling is None else float(self.opt.obj_scaling)
        self.pr = Problem(P, F, w)
        self.dw_last = 0.0

    # ---- derivatives -------------------------------------------------------------
    def evaluate(self, st, rows_only=False):
        return model.derivatives(self.pr.P, self.pr.F, st.Z, st.d, st.lam, rows_only)

    def sigma(self, st):
        pr = self.pr
        sig = (np.where(pr.hasL, st.zL / pr.sl(st.Z), 0.0)
               + np.where(pr.hasU, st.zU / pr.su(st.Z), 0.0))
        dv = np.atleast_1d(st.d)
        sigd = np.atleast_1d(st.zLd) / (dv - pr.dlo) + np.atleast_1d(st.zUd) / (pr.dhi - dv)
        return sig, pr.th(sigd)

    def barrier_gradient(self, st, mu):
        pr = self.pr
        gz = (np.where(pr.hasL, -mu / pr.sl(st.Z), 0.0)
              + np.where(pr.hasU, mu / pr.su(st.Z), 0.0))
        dv = np.atleast_1d(st.d)
        gd = pr.w * pr.wsec - mu / (dv - pr.dlo) + mu / (pr.dhi - dv)
        return gz, pr.th(gd)

    # ---- Newton direction with inertia correction -----------------------------------
    def newton_direction(self, st, mu, C, J, Jd, W, Wdd, dw=None, dc=None):
        """Solve the primal-dual system.  With dw/dc given, use them as is (no inertia
        correction); else run Algorithm IC.  Returns (dZ, dd, dlam, dw, dc, fac)."""
        pr, opt = self.pr, self.opt
        sig, sigd = self.sigma(st)
        gz, gd = self.barrier_gradient(st, mu)
        rz = -(gz + np.einsum("src,sr->sc", J, st.lam))
        rd = -(gd + jd_t(Jd, st.lam))
        rc = -C
        Kdd = (float(np.sum(Wdd)) + sigd) if pr.K == 1 else np.diag(Wdd.sum(axis=0) + sigd)
        n_expect, m_expect = pr.K + pr.S * pr.n, pr.S * pr.n

        def factor(w, c):
            return kkt.SchurKKT(W, sig, J, Jd, Kdd, w, c)

        if dw is not None:
            fac = factor(dw, dc)
        else:
            dw, dc = 0.0, 0.0
            fac = factor(0.0, 0.0)
            inert = fac.inertia()
            if inert != (n_expect, m_expect, 0):
                if inert[2] > 0:
                    dc = opt.dc_bar * mu ** opt.kappa_c
                dw = opt.dw0 if self.dw_last == 0.0 else max(opt.dw_min, opt.kw_minus * self.dw_last)
                while True:
                    fac = factor(dw, dc)
                    if fac.inertia() == (n_expect, m_expect, 0):
                        self.dw_last = dw
                        break
                    dw = (opt.kw_plus_bar if self.dw_last == 0.0 else opt.kw_plus) * dw
                    if dw > opt.dw_max:
                        raise RuntimeError("inertia")
        dZ, dd, dlam = fac.solve(rz, rd, rc)
        return dZ, dd, dlam, dw, dc, fac

    def bound_dual_steps(self, st, mu, dZ, dd):
        pr = self.pr
        sl, su = pr.sl(st.Z), pr.su(st.Z)
        dzL = np.where(pr.hasL, mu / sl - st.zL - (st.zL / sl) * dZ, 0.0)
        dzU = np.where(pr.hasU, mu / su - st.zU + (st.zU / su) * dZ, 0.0)
        dv, ddv = np.atleast_1d(st.d), np.atleast_1d(dd)
        zLd, zUd = np.atleast_1d(st.zLd), np.atleast_1d(st.zUd)
        sld, sud = dv - pr.dlo, pr.dhi - dv
        dzLd = mu / sld - zLd - (zLd / sld) * ddv
        dzUd = mu / sud - zUd + (zUd / sud) * ddv
        return dzL, dzU, pr.th(dzLd), pr.th(dzUd)

    # ---- initial point ------------------------------------------------------------
    def initial_state(self, Z0=None, d0=None, lam0=None):
        pr, opt = self.pr, self.opt
        Zi, di = model.initial_point(pr.P, pr.F)
        Z = Zi if Z0 is None else Z0
        d = di if d0 is None else d0
        Z, d = push_into_bounds(pr, opt, Z, d)
        zL = np.where(pr.hasL, 1.0, 0.0)
        zU = np.where(pr.hasU, 1.0, 0.0)
        one = pr.th(np.ones(pr.K))
        st = State(d, Z, np.zeros((pr.S, pr.n)), zL, zU, one, one)
        if lam0 is not None:
            st.lam = lam0.copy()
            return st
        # least-squares multipliers: [I J^T; J 0][w; lam] = [-(grad f - zL + zU); 0]
        C, J, Jd, _, _ = self.evaluate(st, rows_only=True)
        S, n = pr.S, pr.n
        Wid = np.broadcast_to(np.eye(n), (S, n, n))
        fac = kkt.SchurKKT(Wid, np.zeros((S, n)), J, Jd, 1.0 if pr.K == 1 else np.eye(pr.K), 0.0, 0.0)
        rd = pr.th(-(pr.w * pr.wsec - np.atleast_1d(st.zLd) + np.atleast_1d(st.zUd)))
        _, _, lam = fac.solve(-(-zL + zU), rd, np.zeros((S, n)))
        if np.abs(lam).max() <= opt.lam_init_max:
            st.lam = lam
        return st

    def restoration(self, st, mu, tau, filt, theta_k):
        """Feasibility restoration (Wachter & Biegler 2006, Section 3.3) for the square
        constraint system of problem (10): with d fixed, every scenario's c_s(z_s) = 0 is
        220 equations in its 220 unknowns (J_s square), so the phase takes damped Newton
        steps dz_s = -J_s^{-1} c_s, cut by the fraction to the boundary (tau) and halved
        until ||c||_1 decreases (Armijo, 1e-4).  It returns the first point whose theta is
        at most (1 - gamma_theta) theta_k and which the filter (augmented with the failed
        iterate's entry before the phase) accepts; None after resto_max steps."""
        pr, opt = self.pr, self.opt
        Z = st.Z.copy()
        d = st.d
        C = model.residuals(pr.P, pr.F, Z, d)
        theta = float(np.abs(C).sum())
        for _ in range(opt.resto_max):
            _, J, _, _, _ = model.derivatives(pr.P, pr.F, Z, d, np.zeros_like(Z), rows_only=True)
            dZ = np.stack([-np.linalg.solve(J[s], C[s]) for s in range(pr.S)])
            a = fraction_to_boundary(pr, Z, dZ, pr.hasL, pr.lo, pr.hasU, pr.hi, tau)
            while True:
                Zt = Z + a * dZ
                Ct = model.residuals(pr.P, pr.F, Zt, d)
                th_t = float(np.abs(Ct).sum())
                if np.isfinite(th_t) and th_t <= (1.0 - 1e-4 * a) * theta:
                    break
                a *= 0.5
                if a < 1e-10:
                    return None
            Z, C, theta = Zt, Ct, th_t
            if theta <= (1.0 - opt.gamma_theta) * theta_k:
                ph = barrier_phi(pr, Z, d, mu)
                if all(not (theta >= tf and ph >= pf) for (tf, pf) in filt):
                    return Z
        return None

    def state_from_result(self, r):
        """The solver's internal iterate (multipliers of the scaled problem) for a Result."""
        w = self.pr.w
        return State(r.d, r.Z.copy(), r.lam * w, r.zL * w, r.zU * w, r.zLd * w, r.zUd * w)

    def basecase_start(self):
        """Starting states from the expected-value problem (reading of the paper's "same
        initial point"): solve the single scenario whose feed is the mean of the S feeds
        from the inlet-copy start, copy its stage states to every scenario, keep
        d = (d^L + d^U)/2 and set each hydraulic slack from its row.  None when S = 1,
        when init = "inlet", or when the base case does not converge."""
        pr, opt = self.pr, self.opt
        if pr.S == 1 or opt.init != "basecase":
            return None
        from dataclasses import replace
        r1 = IPM(pr.P, pr.F.mean(axis=1, keepdims=True), replace(opt, init="inlet", verbose=False)).solve()
        if r1.status != "ok":
            return None
        Z0 = np.repeat(r1.Z, pr.S, axis=0).reshape(pr.S, model.N, model.NV)
        d0 = 0.5 * (pr.dlo + pr.dhi)
        vol = model.hydraulic_volume(pr.P, pr.F, Z0.reshape(pr.S, -1))
        Z0[:, :, model.IS] = pr.P["u_max"] * math.pi * d0 * d0 / 4.0 - vol
        return Z0.reshape(pr.S, -1), pr.th(np.full(pr.K, d0)), r1.iters

    # ---- main loop ----------------------------------------------------------------
    def solve(self, st=None):
        pr, opt = self.pr, self.opt
        base_iters = 0
        if st is None:
            bc = self.basecase_start()
            if bc is not None:
                st = self.initial_state(Z0=bc[0], d0=bc[1])
                base_iters = bc[2]
            else:
                st = self.initial_state()
        mu = opt.mu_init
        tau = max(opt.tau_min, 1.0 - mu)
        filt = []
        theta0 = None
        hist = []
        status = "maxiter"
        E0 = float("inf")
        k = 0
        for k in range(opt.max_iter + 1):
            C, J, Jd, W, Wdd = self.evaluate(st)
            theta = float(np.abs(C).sum())
            if theta0 is None:
                theta0 = theta
                theta_max = 1e4 * max(1.0, theta0)
                theta_min = 1e-4 * max(1.0, theta0)
            E0 = optimality_error(pr, opt, st, C, J, Jd, 0.0)[0]
            if E0 <= opt.tol:
                status = "ok"
                break
            if k == opt.max_iter:
                break
            # barrier parameter update (monotone)
            while mu > opt.tol / 10.0:
                Emu = optimality_error(pr, opt, st, C, J, Jd, mu)[0]
                if Emu > opt.kappa_eps * mu:
                    break
                mu = max(opt.tol / 10.0, min(opt.kappa_mu * mu, mu ** opt.theta_mu))
                tau = max(opt.tau_min, 1.0 - mu)
                filt = []
            try:
                dZ, dd, dlam, dw, dc, fac = self.newton_direction(st, mu, C, J, Jd, W, Wdd)
            except RuntimeError:
                status = "inertia"
                break
            dzL, dzU, dzLd, dzUd = self.bound_dual_steps(st, mu, dZ, dd)
            # fraction to the boundary
            allK = np.ones(pr.K, dtype=bool)
            a_max = min(fraction_to_boundary(pr, st.Z, dZ, pr.hasL, pr.lo, pr.hasU, pr.hi, tau),
                        fraction_to_boundary(pr, np.atleast_1d(st.d), np.atleast_1d(dd),
                                             allK, np.full(pr.K, pr.dlo), allK, np.full(pr.K, pr.dhi), tau))
            zmask = pr.hasL
            a_z = min(fraction_to_boundary(pr, st.zL, dzL, pr.hasL, np.zeros_like(st.zL),
                                           np.zeros_like(pr.hasU), st.zL, tau),
                      fraction_to_boundary(pr, st.zU, dzU, pr.hasU, np.zeros_like(st.zU),
                                           np.zeros_like(pr.hasU), st.zU, tau),
                      fraction_to_boundary(pr, np.concatenate([np.atleast_1d(st.zLd), np.atleast_1d(st.zUd)]),
                                           np.concatenate([np.atleast_1d(dzLd), np.atleast_1d(dzUd)]),
                                           np.ones(2 * pr.K, dtype=bool), np.zeros(2 * pr.K),
                                           np.zeros(2 * pr.K, dtype=bool), np.zeros(2 * pr.K), tau))
            del zmask
            # filter line search
            phi = barrier_phi(pr, st.Z, st.d, mu)
            gz, gd = self.barrier_gradient(st, mu)
            gphi = float(np.sum(gz * dZ)) + float(np.atleast_1d(gd) @ np.atleast_1d(dd))
            tiny = max(float(np.max(np.abs(dZ) / (1.0 + np.abs(st.Z)))),
                       float(np.max(np.abs(np.atleast_1d(dd)) / (1.0 + np.abs(np.atleast_1d(st.d)))))
                       ) < 10.0 * np.finfo(float).eps
            alpha = a_max
            accepted = False
            ftype = False
            n_ls = 0
            n_soc = 0
            if tiny:
                accepted, alpha = True, a_max
            else:
                if gphi < 0:
                    if theta <= theta_min:
                        a_min = opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta / (-gphi),
                                                      opt.delta * theta ** opt.s_theta / (-gphi) ** opt.s_phi)
                    else:
                        a_min = opt.gamma_alpha * min(opt.gamma_theta, opt.gamma_phi * theta / (-gphi))
                else:
                    a_min = opt.gamma_alpha * opt.gamma_theta
                def acceptable(Zt, dt, a_sw):
                    """filter + sufficient-decrease tests of a trial point; a_sw is the
                    step size used in the switching condition and the Armijo rule."""
                    Ct = model.residuals(pr.P, pr.F, Zt, dt)
                    th_t = float(np.abs(Ct).sum())
                    ph_t = barrier_phi(pr, Zt, dt, mu)
                    ok = np.isfinite(th_t) and np.isfinite(ph_t) and th_t <= theta_max
                    f_t = False
                    if ok:
                        for (tf, pf) in filt:
                            if th_t >= tf and ph_t >= pf:
                                ok = False
                                break
                    if ok:
                        switching = gphi < 0 and a_sw * (-gphi) ** opt.s_phi > opt.delta * theta ** opt.s_theta
                        if theta <= theta_min and switching:
                            ok = ph_t <= phi + opt.eta_phi * a_sw * gphi
                            f_t = ok
                        else:
                            ok = th_t <= (1 - opt.gamma_theta) * theta or ph_t <= phi - opt.gamma_phi * theta
                    return ok, f_t, th_t, Ct

                while n_ls < opt.max_ls:
                    n_ls += 1
                    ok, ftype, th_t, Ct = acceptable(st.Z + alpha * dZ, pr.th(np.atleast_1d(st.d) + alpha * np.atleast_1d(dd)),
                                                     alpha)
                    if ok:
                        accepted = True
                        break
                    if n_ls == 1 and opt.soc_max > 0 and not (th_t < theta):
                        # second-order correction (Section 2.4)
                        a0 = alpha
                        csoc = a0 * C + Ct
                        th_old = theta
                        for p in range(opt.soc_max):
                            sZ, sd, sl = fac.solve(-(gz + np.einsum("src,sr->sc", J, st.lam)),
                                                   -(gd + jd_t(Jd, st.lam)), -csoc)
                            a_soc = min(fraction_to_boundary(pr, st.Z, sZ, pr.hasL, pr.lo, pr.hasU, pr.hi, tau),
                                        fraction_to_boundary(pr, np.atleast_1d(st.d), np.atleast_1d(sd),
                                                             allK, np.full(pr.K, pr.dlo), allK,
                                                             np.full(pr.K, pr.dhi), tau))
                            ok, ftype, th_s, Cs = acceptable(
                                st.Z + a_soc * sZ, pr.th(np.atleast_1d(st.d) + a_soc * np.atleast_1d(sd)), a0)
                            n_soc += 1
                            if ok:
                                dZ, dd, dlam, alpha = sZ, sd, sl, a_soc
                                dzL, dzU, dzLd, dzUd = self.bound_dual_steps(st, mu, dZ, dd)
                                a_z = min(fraction_to_boundary(pr, st.zL, dzL, pr.hasL, np.zeros_like(st.zL),
                                                               np.zeros_like(pr.hasU), st.zL, tau),
                                          fraction_to_boundary(pr, st.zU, dzU, pr.hasU, np.zeros_like(st.zU),
                                                               np.zeros_like(pr.hasU), st.zU, tau),
                                          fraction_to_boundary(pr, np.concatenate([np.atleast_1d(st.zLd),
                                                                                   np.atleast_1d(st.zUd)]),
                                                               np.concatenate([np.atleast_1d(dzLd),
                                                                               np.atleast_1d(dzUd)]),
                                                               np.ones(2 * pr.K, dtype=bool), np.zeros(2 * pr.K),
                                                               np.zeros(2 * pr.K, dtype=bool), np.zeros(2 * pr.K),
                                                               tau))
                                accepted = True
                                break
                            if th_s > opt.kappa_soc * th_old:
                                break
                            th_old = th_s
                            csoc = a_soc * csoc + Cs
                        if accepted:
                            break
                    alpha *= 0.5
                    if alpha < a_min:
                        break
            if not accepted:
                # feasibility restoration: the filter keeps the failed iterate's entry
                filt.append(((1 - opt.gamma_theta) * theta, phi - opt.gamma_phi * theta))
                Zr = self.restoration(st, mu, tau, filt, theta) if opt.resto_max > 0 else None
                if Zr is None:
                    status = "linesearch"
                    break
                hist.append(dict(iter=k, mu=mu, E0=E0, theta=theta, alpha=0.0, alpha_z=0.0,
                                 dw=dw, dc=dc, ls=n_ls, soc=n_soc, d=st.d, resto=True))
                st.Z = Zr
                sl, su = pr.sl(st.Z), pr.su(st.Z)
                ks = opt.kappa_sigma
                st.zL = np.where(pr.hasL, np.clip(st.zL, mu / (ks * sl), ks * mu / sl), 0.0)
                st.zU = np.where(pr.hasU, np.clip(st.zU, mu / (ks * su), ks * mu / su), 0.0)
                continue
            if not ftype and not tiny:
                filt.append(((1 - opt.gamma_theta) * theta, phi - opt.gamma_phi * theta))
            hist.append(dict(iter=k, mu=mu, E0=E0, theta=theta, alpha=alpha, alpha_z=a_z,
                             dw=dw, dc=dc, ls=n_ls, soc=n_soc, d=st.d))
            if opt.verbose:
                print(f"{k:4d} E0={E0:.3e} th={theta:.3e} mu={mu:.2e} a={alpha:.3e} az={a_z:.3e} "
                      f"dw={dw:.1e} ls={n_ls} soc={n_soc} d={st.d}")
            # accept the step
            st.Z = st.Z + alpha * dZ
            st.d = pr.th(np.atleast_1d(st.d) + alpha * np.atleast_1d(dd))
            st.lam = st.lam + alpha * dlam
            st.zL = st.zL + a_z * dzL
            st.zU = st.zU + a_z * dzU
            st.zLd = pr.th(np.atleast_1d(st.zLd) + a_z * np.atleast_1d(dzLd))
            st.zUd = pr.th(np.atleast_1d(st.zUd) + a_z * np.atleast_1d(dzUd))
            # kappa_Sigma safeguard of the bound multipliers (Eq. (16))
            sl, su = pr.sl(st.Z), pr.su(st.Z)
            ks = opt.kappa_sigma
            st.zL = np.where(pr.hasL, np.clip(st.zL, mu / (ks * sl), ks * mu / sl), 0.0)
            st.zU = np.where(pr.hasU, np.clip(st.zU, mu / (ks * su), ks * mu / su), 0.0)
            dv = np.atleast_1d(st.d)
            sld, sud = dv - pr.dlo, pr.dhi - dv
            st.zLd = pr.th(np.minimum(np.maximum(np.atleast_1d(st.zLd), mu / (ks * sld)), ks * mu / sld))
            st.zUd = pr.th(np.minimum(np.maximum(np.atleast_1d(st.zUd), mu / (ks * sud)), ks * mu / sud))
        # report the multipliers of the unscaled problem (min d): those of min w d over w
        w = pr.w
        return Result(status, k, st.d, st.Z, st.lam / w, st.zL / w, st.zU / w,
                      pr.th(np.atleast_1d(st.zLd) / w), pr.th(np.atleast_1d(st.zUd) / w), E0, mu, hist, base_iters)


def solve(P, F, opt=None, **kw):
    return IPM(P, F, opt).solve(**kw)
