"""The scenario absorber NLP (10), written out plainly.  Test infrastructure.

Per scenario and stage n = 0..N-1 (bottom to top) the 22 unknowns, in this order, are
    xt[9]  liquid mole fractions of C_L, scaled (x_i = sx_i xt_i)
    yt[4]  vapour mole fractions of C_V = (CO2, H2O, N2, O2), scaled
    L, V   liquid / vapour molar flows leaving the stage
    Tt     temperature / 100
    eps[5] reaction extents of R1..R5
    s      slack of the hydraulic inequality (10b)
and the 22 rows, in this order, are
    0..10  material balance (1) for the 11 species (Section "Case study" order)
    11     Raoult's law for water (9a)
    12     Henry's law for CO2 (9b)
    13..17 reaction equilibrium (3a) for R1..R5, activities = mole fractions
    18, 19 summation (4) for liquid and vapour
    20     energy balance (6) with the ideal-mixture enthalpies of the case study
    21     hydraulic row (10b) in slack form  V R T / P - u_max pi d^2 / 4 + s = 0, s >= 0
The 90 variable-fixings per scenario of the paper's count (y_i = 0 for the seven
non-volatile species, x_i = 0 for N2 and O2) are eliminated: those entries are exactly
zero and are not unknowns.  Side feeds f, F and heat duty Q are zero and P_n = P^abs.

The per-scenario unknowns are ordered stage-major (index 22 n + j), as are the rows.
The shared design variable is the diameter d.  Derivatives come from ad.Jet, never from
hand-derived formulas.

Design vector with more than one entry (the general Eq. (8) with dim theta > 1): with
P["n_sections"] = K > 1 the column is split into K sections of consecutive stages
(stage n in section floor(n K / N)), each with its own diameter theta_k; the hydraulic
row (10b) of a stage uses its section's diameter.  d is then an array of K entries and
the d-derivatives gain a last axis of K; a scalar d (K = 1) keeps the scalar shapes.
"""
from __future__ import annotations

import math

import numpy as np

from .ad import Jet, jexp, jlog, value

N = 10          # stages N_abs (Section "Problem setup")
NV = 22         # unknowns per stage
NR = 22         # rows per stage
NS = N * NV     # unknowns (and rows) per scenario
K_LOC = 40      # local independent variables of one stage's rows (see _LOCAL)

# Stoichiometric coefficients nu[species, reaction] of R1..R5 (Section "Case study").
# Species: MEA, MEAH+, H+, MEACOO-, HCO3-, OH-, CO3--, CO2, H2O, N2, O2
NU = np.zeros((11, 5))
# R1: MEAH+ <-> MEA + H+
NU[1, 0], NU[0, 0], NU[2, 0] = -1, 1, 1
# R2: HCO3- <-> H+ + CO3--
NU[4, 1], NU[2, 1], NU[6, 1] = -1, 1, 1
# R3: H2O <-> H+ + OH-
NU[8, 2], NU[2, 2], NU[5, 2] = -1, 1, 1
# R4: MEACOO- + H2O <-> MEA + HCO3-
NU[3, 3], NU[8, 3], NU[0, 3], NU[4, 3] = -1, -1, 1, 1
# R5: H2O + CO2 <-> H+ + HCO3-
NU[8, 4], NU[7, 4], NU[2, 4], NU[4, 4] = -1, -1, 1, 1

# Index of each vapour species of C_V in the 11-species order, and back.
VAP_SPECIES = (7, 8, 9, 10)
LIQ_SPECIES = tuple(range(9))

# Local-variable layout of one stage's rows:
#   [0:22)  the stage's own unknowns
#   [22:33) stream from above: xt(9), L, Tt   of stage n+1 (lean feed for the top stage)
#   [33:39) stream from below: yt(4), V, Tt   of stage n-1 (flue gas for stage 1)
#   39      d
IX, IY, IL, IV, IT, IE, IS = 0, 9, 13, 14, 15, 16, 21
A_X, A_L, A_T = 22, 31, 32
B_Y, B_V, B_T = 33, 37, 38
I_D = 39


def feed_rows():
    off, o = {}, 0
    for name, n in (("V0", 1), ("y0", 4), ("T0", 1), ("Lin", 1), ("xin", 9), ("Tin", 1),
                    ("P", 1)):
        off[name] = o
        o += n
    return off


FEED = feed_rows()


def stage_pressures(P, F):
    """Stage pressures (S, N) from the pressure relation (7) with a specified drop:
    P_n = P_top + (N - 1 - n) dP, P_top the scenario's absorber pressure (the top stage,
    n = N - 1) and dP = P["dp_stage"] per stage (0: every stage at P^abs, the case study)."""
    dp = float(P.get("dp_stage", 0.0))
    return F[FEED["P"], :][:, None] + dp * (N - 1 - np.arange(N))[None, :]


def n_sections(P):
    """Number of column sections K, each with its own diameter (1: the case study)."""
    return int(P.get("n_sections", 1))


def stage_sections(K):
    """Section of every stage: floor(n K / N) (consecutive stages, sizes within one)."""
    return (np.arange(N) * K) // N


def section_weights(K):
    """Objective weight of each section's diameter: its share of the stages (its share
    of the column height), so that K = 1 gives the objective d."""
    return np.bincount(stage_sections(K), minlength=K) / float(N)


def local_to_scenario(n):
    """Per-scenario column of each local variable of stage n's rows (-1: not an unknown,
    i.e. boundary feed data; -2: the diameter d)."""
    m = np.full(K_LOC, -1, dtype=np.int64)
    m[:NV] = NV * n + np.arange(NV)
    if n + 1 < N:
        m[A_X:A_X + 9] = NV * (n + 1) + IX + np.arange(9)
        m[A_L] = NV * (n + 1) + IL
        m[A_T] = NV * (n + 1) + IT
    if n > 0:
        m[B_Y:B_Y + 4] = NV * (n - 1) + IY + np.arange(4)
        m[B_V] = NV * (n - 1) + IV
        m[B_T] = NV * (n - 1) + IT
    m[I_D] = -2
    return m


def _lnK(P, r, T):
    """Kent-Eisenberg correlation ln K_r(T) = A + B/T + C ln T + D T (Case study)."""
    return (P["KE_A"][r] + P["KE_B"][r] / T + P["KE_C"][r] * jlog(T) + P["KE_D"][r] * T)


def _hL(P, l, T):
    """Liquid component enthalpy h_l^L(T): reference value, integral of
    cp = cpa + cpb (T - Tref) from Tref to T, and the constant correction dh (F5)."""
    dT = T - P["T_ref"]
    return (P["hL_ref"][l] + P["hL_cpa"][l] * dT + 0.5 * P["hL_cpb"][l] * dT * dT
            + P["hL_dh"][l])


def _hV(P, j, T):
    dT = T - P["T_ref"]
    return (P["hV_ref"][j] + P["hV_cpa"][j] * dT + 0.5 * P["hV_cpb"][j] * dT * dT
            + P["hV_dh"][j])


def stage_rows(P, pres, q):
    """The 22 rows of one stage.  q: list of the 40 local quantities (Jets or arrays);
    pres: the stage's pressure per point (stage_pressures).  Returns a list of 22 values."""
    sx, sy, sT = P["sx"], P["sy"], P["sT"]
    x = [sx[l] * q[IX + l] for l in range(9)]
    y = [sy[j] * q[IY + j] for j in range(4)]
    L, V, T = q[IL], q[IV], sT * q[IT]
    eps = [q[IE + r] for r in range(5)]
    xa = [sx[l] * q[A_X + l] for l in range(9)]
    La, Ta = q[A_L], sT * q[A_T]
    yb = [sy[j] * q[B_Y + j] for j in range(4)]
    Vb, Tb = q[B_V], sT * q[B_T]
    d = q[I_D]

    rows = []
    # (1) material balances: out - in - sum_r nu_ir eps_r = 0
    for c in range(11):
        r = 0.0
        if c < 9:
            r = r + L * x[c] - La * xa[c]
        if c in VAP_SPECIES:
            j = VAP_SPECIES.index(c)
            r = r + V * y[j] - Vb * yb[j]
        for k in range(5):
            if NU[c, k] != 0.0:
                r = r - NU[c, k] * eps[k]
        rows.append(r)
    # (9a) Raoult's law for water: P y_H2O - x_H2O Psat(T)
    psat = jexp(P["psat_a"] - P["psat_b"] / (T + P["psat_c"]))
    rows.append(pres * y[1] - x[8] * psat)
    # (9b) Henry's law for CO2: P y_CO2 - c_CO2 H(T, x_MEA^app, x_H2O^app), c = rho_L x
    a_mea = x[0] + x[1] + x[3]
    a_co2 = x[7] + x[3] + x[4] + x[6]
    a_h2o = x[8] + x[4] + x[6] + x[5]
    tot = a_mea + a_co2 + a_h2o
    lnH = (P["henry_a"] + P["henry_b"] / T + P["henry_m"] * (a_mea / tot)
           + P["henry_w"] * (a_h2o / tot))
    rows.append(pres * y[0] - P["rho_L"] * x[7] * jexp(lnH))
    # (3a) reaction equilibrium: sum_i nu_ir ln x_i - ln K_r(T)
    for k in range(5):
        r = -_lnK(P, k, T)
        for c in range(9):
            if NU[c, k] != 0.0:
                r = r + NU[c, k] * (jlog(q[IX + c]) + math.log(sx[c]))
        rows.append(r)
    # (4) summation
    sumx = -1.0
    for l in range(9):
        sumx = sumx + x[l]
    sumy = -1.0
    for j in range(4):
        sumy = sumy + y[j]
    rows.append(sumx)
    rows.append(sumy)
    # (6) energy balance with ideal-mixture enthalpy flows
    hl = 0.0
    hla = 0.0
    for l in range(9):
        hl = hl + x[l] * _hL(P, l, T)
        hla = hla + xa[l] * _hL(P, l, Ta)
    hv = 0.0
    hvb = 0.0
    for j in range(4):
        hv = hv + y[j] * _hV(P, j, T)
        hvb = hvb + yb[j] * _hV(P, j, Tb)
    rows.append(L * hl + V * hv - La * hla - Vb * hvb)
    # (10b) hydraulic capacity, slack form
    rows.append(V * P["R"] * T / pres - P["u_max"] * math.pi * d * d / 4.0 + q[IS])
    return rows


def _local_values(P, F, Z, d):
    """Values of the 40 local quantities for every (scenario, stage), shape (40, S*N),
    plus boolean masks of which 'above'/'below' entries are unknowns."""
    S = Z.shape[0]
    Zs = Z.reshape(S, N, NV)
    dv = np.atleast_1d(np.asarray(d))
    vals = np.zeros((K_LOC, S, N), dtype=np.result_type(Z.dtype, dv.dtype, np.float64))
    vals[:NV] = np.moveaxis(Zs, 2, 0)
    sx = np.asarray(P["sx"])
    sy = np.asarray(P["sy"])
    # stream from above
    vals[A_X:A_X + 9, :, :N - 1] = np.moveaxis(Zs[:, 1:, IX:IX + 9], 2, 0)
    vals[A_L, :, :N - 1] = Zs[:, 1:, IL]
    vals[A_T, :, :N - 1] = Zs[:, 1:, IT]
    vals[A_X:A_X + 9, :, N - 1] = F[FEED["xin"]:FEED["xin"] + 9, :] / sx[:, None]
    vals[A_L, :, N - 1] = F[FEED["Lin"], :]
    vals[A_T, :, N - 1] = F[FEED["Tin"], :] / P["sT"]
    # stream from below
    vals[B_Y:B_Y + 4, :, 1:] = np.moveaxis(Zs[:, :N - 1, IY:IY + 4], 2, 0)
    vals[B_V, :, 1:] = Zs[:, :N - 1, IV]
    vals[B_T, :, 1:] = Zs[:, :N - 1, IT]
    vals[B_Y:B_Y + 4, :, 0] = F[FEED["y0"]:FEED["y0"] + 4, :] / sy[:, None]
    vals[B_V, :, 0] = F[FEED["V0"], :]
    vals[B_T, :, 0] = F[FEED["T0"], :] / P["sT"]
    vals[I_D] = dv[stage_sections(dv.size)][None, :]     # each stage its section's diameter
    active = np.ones((K_LOC, S, N), dtype=bool)
    active[A_X:B_Y, :, N - 1] = False
    active[B_Y:I_D, :, 0] = False
    pres = stage_pressures(P, F)
    return vals.reshape(K_LOC, S * N), active.reshape(K_LOC, S * N), pres.reshape(S * N)


def residuals(P, F, Z, d):
    """c(z, d) for all scenarios: (S, 220), rows stage-major."""
    S = Z.shape[0]
    vals, _, pres = _local_values(P, F, Z, d)
    rows = stage_rows(P, pres, [vals[i] for i in range(K_LOC)])
    C = np.stack([np.broadcast_to(np.asarray(r, dtype=vals.dtype), (S * N,)) for r in rows])
    return C.reshape(NR, S, N).transpose(1, 2, 0).reshape(S, NS)


def derivatives(P, F, Z, d, lam, rows_only=False):
    """Exact derivatives from second-order AD.

    Returns (C, J, Jd, W, Wdd):
      C   (S, 220)       residuals
      J   (S, 220, 220)  dc_s/dz_s (dense per scenario)
      Jd  (S, 220)       dc_s/dd                   ((S, 220, K) for an array d of K)
      W   (S, 220, 220)  Hessian of lam_s^T c_s with respect to z_s (symmetric)
      Wdd (S,)           d^2 (lam_s^T c_s)/dd^2    ((S, K): diagonal in the sections)
    (the objective is linear in d).
    """
    S = Z.shape[0]
    vals, active, pres = _local_values(P, F, Z, d)
    q = [Jet.variable(vals[i], i, K_LOC, active[i]) for i in range(K_LOC)]
    rows = stage_rows(P, pres, q)
    B = S * N
    lam3 = lam.reshape(S, N, NR).reshape(B, NR)
    C = np.zeros((B, NR))
    G = np.zeros((B, NR, K_LOC))
    Hl = np.zeros((B, K_LOC, K_LOC))
    for r, row in enumerate(rows):
        if not isinstance(row, Jet):  # constant row (cannot happen for this model)
            C[:, r] = row
            continue
        C[:, r] = row.v
        G[:, r, :] = row.g
        if not rows_only:
            Hl += lam3[:, r][:, None, None] * row.h
    C = C.reshape(S, N, NR).reshape(S, NS)
    G = G.reshape(S, N, NR, K_LOC)
    Hl = Hl.reshape(S, N, K_LOC, K_LOC)
    K = np.size(d)
    sec = stage_sections(K)
    J = np.zeros((S, NS, NS))
    Jd = np.zeros((S, NS, K))
    W = np.zeros((S, NS, NS))
    Wdd = np.zeros((S, K))
    for n in range(N):
        m = local_to_scenario(n)
        rws = NR * n + np.arange(NR)
        loc = np.nonzero(m >= 0)[0]
        J[:, rws[:, None], m[loc][None, :]] += G[:, n][:, :, loc]
        Jd[:, rws, sec[n]] = G[:, n, :, I_D]
        if not rows_only:
            W[:, m[loc][:, None], m[loc][None, :]] += Hl[:, n][:, loc[:, None], loc[None, :]]
            Wdd[:, sec[n]] += Hl[:, n, I_D, I_D]
    if np.ndim(d) == 0:
        return C, J, Jd[:, :, 0], W, Wdd[:, 0]
    return C, J, Jd, W, Wdd


def hydraulic_volume(P, F, Z):
    """V R T / P^abs for every (scenario, stage): the gas volumetric flow of (10b)."""
    S = Z.shape[0]
    Zs = Z.reshape(S, N, NV)
    return Zs[:, :, IV] * P["R"] * (P["sT"] * Zs[:, :, IT]) / stage_pressures(P, F)


def bounds(P, S):
    """Lower/upper bounds (10c-d) of the per-scenario unknowns, (S, 220) each (+-inf
    where unbounded), and of d."""
    lo = np.full((N, NV), -np.inf)
    hi = np.full((N, NV), np.inf)
    lo[:, IX:IX + 9] = 0.0
    lo[:, IY:IY + 4] = 0.0
    lo[:, IL] = 0.0
    lo[:, IV] = 0.0
    lo[:, IT] = P["T_lo"] / P["sT"]
    hi[:, IT] = P["T_hi"] / P["sT"]
    lo[:, IS] = 0.0
    lo = np.broadcast_to(lo.reshape(NS), (S, NS)).copy()
    hi = np.broadcast_to(hi.reshape(NS), (S, NS)).copy()
    return lo, hi, P["d_lo"], P["d_hi"]


def initial_point(P, F):
    """Reading F7 of the paper's "same initial point": every stage copies the inlet
    streams (L = Lin, x = xin, V = V0, y = y0), T = (T0 + Tin)/2, eps = 0,
    d = (d^L + d^U)/2; the slack is set from the hydraulic row.  The solver then
    pushes everything inside its bounds."""
    S = F.shape[1]
    Z = np.zeros((S, N, NV))
    sx, sy = np.asarray(P["sx"]), np.asarray(P["sy"])
    Z[:, :, IX:IX + 9] = (F[FEED["xin"]:FEED["xin"] + 9, :] / sx[:, None]).T[:, None, :]
    Z[:, :, IY:IY + 4] = (F[FEED["y0"]:FEED["y0"] + 4, :] / sy[:, None]).T[:, None, :]
    Z[:, :, IL] = F[FEED["Lin"], :][:, None]
    Z[:, :, IV] = F[FEED["V0"], :][:, None]
    Z[:, :, IT] = (0.5 * (F[FEED["T0"], :] + F[FEED["Tin"], :]) / P["sT"])[:, None]
    d = 0.5 * (P["d_lo"] + P["d_hi"])
    vol = (Z[:, :, IV] * P["R"] * P["sT"] * Z[:, :, IT]) / stage_pressures(P, F)
    Z[:, :, IS] = P["u_max"] * math.pi * d * d / 4.0 - vol
    return Z.reshape(S, NS), d


def full_layout(P, Z):
    """The paper-literal 300 unknowns per scenario (x[11], y[11], L, V, T, eps[5] per
    stage, physical units), with the 90 fixed entries exactly zero: (S, N, 30)."""
    S = Z.shape[0]
    Zs = Z.reshape(S, N, NV)
    out = np.zeros((S, N, 30))
    out[:, :, 0:9] = Zs[:, :, IX:IX + 9] * np.asarray(P["sx"])
    for j, c in enumerate(VAP_SPECIES):
        out[:, :, 11 + c] = Zs[:, :, IY + j] * P["sy"][j]
    out[:, :, 22] = Zs[:, :, IL]
    out[:, :, 23] = Zs[:, :, IV]
    out[:, :, 24] = Zs[:, :, IT] * P["sT"]
    out[:, :, 25:30] = Zs[:, :, IE:IE + 5]
    return out


def problem_size(S):
    """Counts of the paper-literal deterministic equivalent (Section "Numerical
    results"): (variables, MESH equalities, variable-fixing constraints, hydraulic
    inequalities).  Per stage: x and y over all 11 species, L, V, T and 5 extents; MESH
    rows = 11 material + 2 phase-equilibrium (9a-b) + 5 reaction (3a) + 2 summation +
    1 energy; fixings = y of the 7 non-volatile species + x of the 2 non-condensables;
    one hydraulic row (10b).  Plus the shared diameter."""
    n_species = 11
    per_stage_vars = 2 * n_species + 3 + NU.shape[1]
    per_stage_mesh = n_species + 2 + NU.shape[1] + 2 + 1
    per_stage_fix = (n_species - len(VAP_SPECIES)) + (n_species - len(LIQ_SPECIES))
    return (1 + S * N * per_stage_vars, S * N * per_stage_mesh, S * N * per_stage_fix, S * N)
