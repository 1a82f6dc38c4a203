"""Independent checks of oracle results.  Test infrastructure (see oracle/__init__.py).

Nothing here uses the AD derivatives of model.derivatives; the derivatives these checks
need come from complex-step differentiation of the residuals (Squire & Trapp 1998:
f'(x) = Im f(x + i h) / h, exact to rounding for analytic f), so a mistake in ad.py or
in the Jet path cannot hide behind itself.
"""
from __future__ import annotations

import math

import numpy as np

from . import model

H_CS = 1e-30


def jacobian_complex_step(P, F, Z, d):
    """dc/dz (S, 220, 220) and dc/dd (S, 220) by complex step, one column at a time
    (for an array d of K section diameters dc/dd is (S, 220, K), one column per entry)."""
    S, n = Z.shape
    J = np.zeros((S, n, n))
    for j in range(n):
        Zc = Z.astype(complex)
        Zc[:, j] += 1j * H_CS
        J[:, :, j] = model.residuals(P, F, Zc, d).imag / H_CS
    if np.ndim(d) == 0:
        Jd = model.residuals(P, F, Z.astype(complex), d + 1j * H_CS).imag / H_CS
    else:
        Jd = np.zeros((S, n, np.size(d)))
        for k in range(np.size(d)):
            dc = np.asarray(d, dtype=complex).copy()
            dc[k] += 1j * H_CS
            Jd[:, :, k] = model.residuals(P, F, Z.astype(complex), dc).imag / H_CS
    return J, Jd


def lagrangian_gradient_cs(P, F, Z, d, lam):
    """grad_z (lam^T c) by complex step, (S, 220)."""
    J, _ = jacobian_complex_step(P, F, Z, d)
    return np.einsum("sr,src->sc", lam, J)


# Element and charge content of the 11 species (C, H, N, O, charge).  Formulas:
# MEA C2H7NO, MEAH+ C2H8NO+, H+, MEACOO- C3H6NO3-, HCO3- CHO3-, OH-, CO3-- CO3--,
# CO2, H2O, N2, O2.
ELEMENTS = np.array([
    # C  H  N  O  q
    [2, 7, 1, 1, 0],
    [2, 8, 1, 1, 1],
    [0, 1, 0, 0, 1],
    [3, 6, 1, 3, -1],
    [1, 1, 0, 3, -1],
    [0, 1, 0, 1, -1],
    [1, 0, 0, 3, -2],
    [1, 0, 0, 2, 0],
    [0, 2, 0, 1, 0],
    [0, 0, 2, 0, 0],
    [0, 0, 0, 2, 0],
], dtype=float)


def column_balances(P, F, Z):
    """Element/charge flows (S, 5) and enthalpy flow (S,) in and out of the column.

    In: flue gas (V0, y0, T0) at the bottom, lean solvent (Lin, xin, Tin) at the top.
    Out: gas leaving the top stage, liquid leaving the bottom stage.  Enthalpies are
    evaluated here from the parameter table, independently of model.py.
    """
    off = model.FEED
    full = model.full_layout(P, Z)   # (S, N, 30): x[11], y[11], L, V, T, eps[5]
    S = Z.shape[0]
    xin = np.zeros((S, 11))
    xin[:, :9] = F[off["xin"]:off["xin"] + 9].T
    y0 = np.zeros((S, 11))
    y0[:, 7:11] = F[off["y0"]:off["y0"] + 4].T
    V0, Lin = F[off["V0"]], F[off["Lin"]]
    T0, Tin = F[off["T0"]], F[off["Tin"]]
    x_out = full[:, 0, 0:11]
    L_out, T_bot = full[:, 0, 22], full[:, 0, 24]
    y_out = full[:, -1, 11:22]
    V_out, T_top = full[:, -1, 23], full[:, -1, 24]
    el_in = (V0[:, None] * y0 + Lin[:, None] * xin) @ ELEMENTS
    el_out = (V_out[:, None] * y_out + L_out[:, None] * x_out) @ ELEMENTS

    Tref = P["T_ref"]

    def hL(T):
        dT = (T - Tref)[:, None]
        return (np.asarray(P["hL_ref"]) + np.asarray(P["hL_dh"]) + np.asarray(P["hL_cpa"]) * dT
                + 0.5 * np.asarray(P["hL_cpb"]) * dT ** 2)

    def hV(T):
        dT = (T - Tref)[:, None]
        return (np.asarray(P["hV_ref"]) + np.asarray(P["hV_dh"]) + np.asarray(P["hV_cpa"]) * dT
                + 0.5 * np.asarray(P["hV_cpb"]) * dT ** 2)

    h_in = V0 * np.sum(y0[:, 7:11] * hV(T0), 1) + Lin * np.sum(xin[:, :9] * hL(Tin), 1)
    h_out = V_out * np.sum(y_out[:, 7:11] * hV(T_top), 1) + L_out * np.sum(x_out[:, :9] * hL(T_bot), 1)
    return el_in, el_out, h_in, h_out


def liquid_charge(P, Z):
    """Net charge of the liquid on every stage, sum_i q_i x_i: (S, N)."""
    full = model.full_layout(P, Z)
    return full[:, :, 0:11] @ ELEMENTS[:, 4]


def mesh_newton(P, F, Z0, d, iters=8):
    """Damped-free Newton on each scenario's square MESH system (the 210 rows without the
    hydraulic row, in the 210 unknowns without the slack), Jacobian by complex step.
    Returns (Z, list of max residual norms per iteration)."""
    S = Z0.shape[0]
    keep = np.ones(model.NS, dtype=bool)
    keep[model.NV - 1::model.NV] = False      # slack columns / hydraulic rows
    Z = Z0.copy()
    hist = []
    for _ in range(iters):
        C = model.residuals(P, F, Z, d)
        hist.append(float(np.abs(C[:, keep]).max()))
        J, _ = jacobian_complex_step(P, F, Z, d)
        for s in range(S):
            A = J[s][np.ix_(keep, keep)]
            step = np.linalg.solve(A, C[s, keep])
            Z[s, keep] -= step
        if hist[-1] < 1e-15:
            break
    return Z, hist


def minimum_diameter(P, F, Z):
    """max over scenarios and stages of sqrt(4 V R T / (pi u_max P^abs)): the smallest d
    that satisfies every hydraulic row (10b) at the given states."""
    vol = model.hydraulic_volume(P, F, Z)
    return math.sqrt(4.0 * float(vol.max()) / (math.pi * P["u_max"])), vol


def section_diameters(P, F, Z, K):
    """The smallest diameter of each of K column sections that satisfies the hydraulic
    rows of its stages at the given states: max over scenarios and the section's stages
    of sqrt(4 V R T / (pi u_max P^abs))."""
    vol = model.hydraulic_volume(P, F, Z)
    sec = model.stage_sections(K)
    return np.array([math.sqrt(4.0 * float(vol[:, sec == k].max()) / (math.pi * P["u_max"]))
                     for k in range(K)])


def kkt_error(P, F, d, Z, lam, zL, zU, zLd, zUd, s_max=100.0, chunk=None):
    """E_0 (Wachter & Biegler 2006, Eq. (5) at mu = 0) from the definitions, with the
    constraint Jacobian by complex step.  chunk: scenarios per complex-step Jacobian
    (the Jacobian is block diagonal by scenario; chunking bounds the memory of the
    (S, 220, 220) array and changes no arithmetic)."""
    S = Z.shape[0]
    lo, hi, dlo, dhi = model.bounds(P, S)
    K = np.size(d)
    dv, zLv, zUv = np.atleast_1d(d), np.atleast_1d(zLd), np.atleast_1d(zUd)
    step = S if chunk is None else int(chunk)
    rz = np.zeros_like(Z)
    jdl = np.zeros(K)
    for a in range(0, S, step):
        b = min(S, a + step)
        J, Jd = jacobian_complex_step(P, F[:, a:b], Z[a:b], d)
        rz[a:b] = np.einsum("sr,src->sc", lam[a:b], J)
        jdl += np.atleast_1d(np.einsum("sr...,sr->...", Jd, lam[a:b]))
    C = model.residuals(P, F, Z, d)
    rz = rz - zL + zU
    # gradient of the objective sum_k w_k d_k (w = the sections' shares; 1 for K = 1)
    rd = model.section_weights(K) + jdl - zLv + zUv
    hasL, hasU = np.isfinite(lo), np.isfinite(hi)
    cl = np.where(hasL, zL * (Z - np.where(hasL, lo, 0)), 0.0)
    cu = np.where(hasU, zU * (np.where(hasU, hi, 0) - Z), 0.0)
    cd = max(np.abs(zLv * (dv - dlo)).max(), np.abs(zUv * (dhi - dv)).max())
    nz = hasL.sum() + hasU.sum() + 2 * K
    zs = np.abs(zL).sum() + np.abs(zU).sum() + np.abs(zLv).sum() + np.abs(zUv).sum()
    sd = max(s_max, (np.abs(lam).sum() + zs) / (lam.size + nz)) / s_max
    sc = max(s_max, zs / nz) / s_max
    return max(max(np.abs(rz).max(), np.abs(rd).max()) / sd, np.abs(C).max(),
               max(np.abs(cl).max(), np.abs(cu).max(), cd) / sc)
