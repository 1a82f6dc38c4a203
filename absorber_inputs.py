"""Seeded synthetic inputs for the scenario absorber design problem (problem (10)).

This module holds *data only*: the model's parameter table, the nominal feed streams
and a counter-based generator for the per-scenario feed perturbations.  It contains
none of the method's arithmetic (no residuals, derivatives, factorizations or solver
steps); both the CPU oracle and the CUDA library take what it returns as input.

Provenance.  The paper states the model's form (Eqs. (1), (3a), (4), (6), (9a-b), (10)
and the Kent-Eisenberg correlation) but prints none of its constants, nominal feeds or
the seven measured operating cases from which it samples scenarios.  Every number below
is therefore either taken from a named public source or marked "project-chosen": a
physically plausible value for a ~30 wt% MEA absorber near 313 K and 1 bar, fixed once
so that the oracle and the GPU path solve the same problem.

Units (the fixed unit system of the solver): flows kmol/s, temperature K (the NLP
variable is T/100), pressure bar, enthalpy MJ/kmol, heat capacity MJ/(kmol K), length m,
velocity m/s, R in bar m^3/(kmol K).
"""
from __future__ import annotations

import math

import numpy as np

N_STAGES = 10
N_FEED_FIELDS = 18

# Species order used everywhere (Section "Case study", component set C).
SPECIES = ("MEA", "MEAH+", "H+", "MEACOO-", "HCO3-", "OH-", "CO3--", "CO2", "H2O", "N2", "O2")
LIQUID = SPECIES[:9]            # C_L: all but the two non-condensables
VAPOR = ("CO2", "H2O", "N2", "O2")  # C_V: the volatile species

# Feed record layout, one column per scenario (structure of arrays, field-major).
FEED_FIELDS = (
    ("V0", 1), ("y0", 4), ("T0", 1),          # flue gas entering stage 1 from below
    ("Lin", 1), ("xin", 9), ("Tin", 1),       # lean solvent entering stage N from above
    ("P", 1),                                 # absorber pressure P^abs (no pressure drop)
)


def feed_offsets():
    """Row offset of each named feed field in the (18, S) feed array."""
    off, o = {}, 0
    for name, n in FEED_FIELDS:
        off[name] = o
        o += n
    assert o == N_FEED_FIELDS
    return off


# --------------------------------------------------------------------------------------
# Parameter table.  Scalars are floats, vectors are tuples in the orders given above.
# --------------------------------------------------------------------------------------
PARAMS = {
    # Ideal-gas constant, bar m^3/(kmol K) (CODATA 2018 R = 8.314462618 J/(mol K)).
    "R": 0.08314462618,
    # Superficial gas velocity limit u_max (project-chosen, ~75 % of flooding for
    # structured packing).
    "u_max": 2.0,
    # Diameter bounds d^L, d^U of (10c) (project-chosen).
    "d_lo": 0.1,
    "d_hi": 20.0,
    # Stage temperature bounds (project-chosen: liquid water range at ~1 bar).
    "T_lo": 273.15,
    "T_hi": 400.0,
    # Reference temperature of the enthalpy model.
    "T_ref": 298.15,
    # Variable scaling of the fixed unit system: x_i = sx_i * xt_i, y_i = sy_i * yt_i,
    # T = sT * Tt.  Chosen near each species' typical magnitude in the column
    # (project-chosen) so that ln-form equilibrium rows have O(1) derivatives.
    "sx": (1.0, 1e-2, 1e-11, 1e-2, 1e-3, 1e-6, 1e-4, 1e-6, 1.0),
    "sy": (1.0, 1.0, 1.0, 1.0),
    "sT": 100.0,
    # Kent-Eisenberg form ln K_r(T) = A + B/T + C ln T + D T, mole-fraction basis (the
    # basis conversion folded into A).  Project-chosen so that K_r(313.15 K) and the van 't
    # Hoff slope match literature-typical pKa values (MEAH+ 9.2, HCO3- 10.2, water
    # 13.5, carbamate reversion ~0.03 M, CO2 hydration 6.3, with c_tot ~ 45 kmol/m^3)
    # and reaction enthalpies 50, 15, 56, 24, 9 kJ/mol for R1..R5.
    "KE_A": (0.332052, -18.160118, -2.359284, -1.311814, -4.894789),
    "KE_B": (-6228.7048, -1960.6603, -7557.6777, -2729.9615, -1503.1447),
    "KE_C": (-1.0, -0.5, -2.0, 0.5, -1.5),
    "KE_D": (1.0e-3, 0.0, -2.0e-3, 0.0, 5.0e-4),
    # Water saturation pressure, ln Psat[bar] = a - b/(T + c): the NIST Chemistry WebBook
    # Antoine parameters for water, 304-333 K (Bridgeman & Aldrich 1964; log10 form
    # A=5.20389, B=1733.926, C=-39.485), converted to natural log.
    "psat_a": 11.982399539580786,
    "psat_b": 3992.512159954794,
    "psat_c": -39.485,
    # Henry coefficient of CO2 (9b): ln H[bar m^3/kmol] = ha + hb/T + hm x_MEA^app +
    # hw x_H2O^app.  hb and the pure-water value H = 2.82e4 exp(-2044/T) follow Versteeg &
    # van Swaaij (1988); the mixing terms hm, hw are project-chosen (ha absorbs hw so that
    # pure water reproduces the cited value).
    "henry_a": 10.047077256926206,
    "henry_b": -2044.0,
    "henry_m": 1.5,
    "henry_w": 0.2,
    # Liquid molar density for c_CO2 = rho_L x_CO2 (project-chosen, 30 wt% MEA at 313 K).
    "rho_L": 44.0,
    # Liquid component enthalpies h_i^L(T) = href + cpa (T-Tref) + cpb/2 (T-Tref)^2 + dh,
    # over C_L.  href of ions = formation offsets consistent with the reaction enthalpies
    # above (H+, MEA, H2O liquid and CO2 gas as zero references); dh of CO2(L) is its
    # heat of absorption.  Project-chosen except water cp (75.3 J/(mol K)) and MEA
    # cp (~195 J/(mol K)).
    "hL_ref": (0.0, -50.0, 0.0, -35.0, -11.0, 56.0, 4.0, 0.0, 0.0),
    "hL_cpa": (0.195, 0.21, 0.03, 0.25, 0.12, 0.08, 0.10, 0.045, 0.0753),
    "hL_cpb": (2.0e-4, 1.0e-4, 1.0e-5, 2.0e-4, 5.0e-5, 5.0e-5, 5.0e-5, 2.0e-5, 1.0e-5),
    "hL_dh": (0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, -20.0, 0.0),
    # Vapour component enthalpies over C_V (CO2, H2O, N2, O2); dh of water vapour is its
    # heat of vaporisation (44.0 kJ/mol at 298 K); cp near ideal-gas values at 313 K.
    "hV_ref": (0.0, 0.0, 0.0, 0.0),
    "hV_cpa": (0.0372, 0.0336, 0.0291, 0.0294),
    "hV_cpb": (4.0e-5, 1.0e-5, 1.0e-6, 4.0e-6),
    "hV_dh": (0.0, 44.0, 0.0, 0.0),
}

# Nominal feed (project-chosen, the paper's measured cases are not available): a
# ~0.1 kmol/s flue gas with 12 mol% CO2 saturated with water at 313 K, and a lean
# 30 wt% MEA solvent (apparent MEA 0.1094, CO2 0.0219, H2O 0.8687: loading 0.2 mol
# CO2/mol MEA) that arrives chemically equilibrated at 313.15 K: xin is the speciation
# of that apparent composition under the reaction-equilibrium constants above (solved
# once with the five equilibria, the MEA, carbon and oxygen balances and
# electroneutrality, stored to 7 digits, then MEAH+ set so the solvent is exactly
# electroneutral and H2O so that it sums to one).
NOMINAL_FEED = {
    "V0": 0.10,
    "y0": (0.12, 0.07, 0.76, 0.05),
    "T0": 313.15,
    "Lin": 0.45,
    "xin": (0.06729314, 0.022461603172326976, 4.673026e-12, 0.02209475, 2.273806e-4,
            3.229917e-6, 6.812133e-5, 9.205931e-8, 0.88785168291669),
    "Tin": 313.15,
    "P": 1.05,
}


# --------------------------------------------------------------------------------------
# Counter-based generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random
# numbers: as easy as 1, 2, 3", SC 2011).  Counter = (scenario, field, stream, 0),
# key = (seed, 0): any scenario subset is reproducible without generating the rest.
# --------------------------------------------------------------------------------------
_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint32(0x9E3779B9)
_PHILOX_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.  ctr: uint32 array (..., 4); key: uint32 array (..., 2)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32).copy() for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = _PHILOX_M0 * c[0].astype(np.uint64)
            p1 = _PHILOX_M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = k0 + _PHILOX_W0
            k1 = k1 + _PHILOX_W1
    return np.stack(c, axis=-1)


def uniform01(seed, idx, field, stream=0):
    """U(0,1) doubles (53-bit, open interval) for counters (idx, field, stream, 0)."""
    idx = np.asarray(idx, dtype=np.uint64)
    ctr = np.zeros(idx.shape + (4,), dtype=np.uint32)
    ctr[..., 0] = (idx & _MASK32).astype(np.uint32)
    ctr[..., 1] = np.uint32(field)
    ctr[..., 2] = np.uint32(stream)
    key = np.zeros(idx.shape + (2,), dtype=np.uint32)
    key[..., 0] = np.uint32(seed)
    out = philox4x32_10(ctr, key)
    a = (out[..., 0] >> np.uint32(5)).astype(np.float64)   # 27 bits
    b = (out[..., 1] >> np.uint32(6)).astype(np.float64)   # 26 bits
    return (a * 67108864.0 + b + 0.5) / 9007199254740992.0


def _ndtri(p):
    from scipy.special import ndtri
    return ndtri(p)


def perturbation_factors(S, seed, dist="uniform", width=0.10, sigma=0.05, cut=0.15,
                         stream=0, first=0):
    """Multiplicative factors (f_V, f_CO2) for scenarios first..first+S-1.

    uniform:   f ~ U[1-width, 1+width]
    truncnorm: f = 1 + sigma*Z with Z standard normal truncated to |sigma Z| <= cut
               (inverse-CDF sampling between Phi(-cut/sigma) and Phi(cut/sigma)).
    """
    idx = np.arange(first, first + S, dtype=np.uint64)
    u = np.stack([uniform01(seed, idx, f, stream) for f in (0, 1)])
    if dist == "uniform":
        return 1.0 - width + 2.0 * width * u
    if dist == "truncnorm":
        from scipy.special import ndtr
        lo, hi = ndtr(-cut / sigma), ndtr(cut / sigma)
        return 1.0 + sigma * _ndtri(lo + (hi - lo) * u)
    raise ValueError(dist)


def make_feeds(S, seed, dist="uniform", width=0.10, sigma=0.05, cut=0.15, stream=0,
               first=0):
    """Feed array (18, S), float64, field-major: the nominal feed with the flue-gas flow
    V0 and its CO2 fraction y_CO2,0 scaled by seeded factors; the other flue-gas
    fractions are rescaled proportionally so the flue gas still sums to one.  All other
    fields stay nominal."""
    off = feed_offsets()
    F = np.empty((N_FEED_FIELDS, S), dtype=np.float64)
    for name, n in FEED_FIELDS:
        v = NOMINAL_FEED[name]
        if n == 1:
            F[off[name], :] = v
        else:
            F[off[name]:off[name] + n, :] = np.asarray(v, dtype=np.float64)[:, None]
    if S == 0:
        return F
    fV, fC = perturbation_factors(S, seed, dist, width, sigma, cut, stream, first)
    y0 = np.asarray(NOMINAL_FEED["y0"], dtype=np.float64)
    yc = y0[0] * fC
    rest = y0[1:][:, None] * ((1.0 - yc) / (1.0 - y0[0]))[None, :]
    F[off["V0"], :] = NOMINAL_FEED["V0"] * fV
    F[off["y0"], :] = yc
    F[off["y0"] + 1:off["y0"] + 4, :] = rest
    return F


def batched_sizes(P=64, seed=3, lo=50, hi=2000):
    """Scenario counts of P independent design problems, log-uniform in [lo, hi]."""
    u = uniform01(seed, np.arange(P, dtype=np.uint64), 7, stream=1)
    return np.rint(np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)).astype(np.int64)


def batched_feeds(sizes, seed=3, dist="uniform"):
    """Independent feed draws of a batch of problems: problem p takes the scenario
    counters after those of problems 0..p-1 on its own stream (2), so no two scenarios
    of the batch share a draw."""
    out, first = [], 0
    for S in sizes:
        out.append(make_feeds(int(S), seed, dist=dist, stream=2, first=first))
        first += int(S)
    return out


# Named workloads (sizes, draws and seeds of the five configurations).
WORKLOADS = {
    "absorber-S10-u10-seed0": dict(S=10, seed=0, dist="uniform"),
    "absorber-S500-u10-seed1": dict(S=500, seed=1, dist="uniform"),
    "absorber-S5000-tn5-seed2": dict(S=5000, seed=2, dist="truncnorm"),
    "absorber-S20000-u10-seed4": dict(S=20000, seed=4, dist="uniform"),
}


def workload_feeds(name):
    w = WORKLOADS[name]
    return make_feeds(w["S"], w["seed"], dist=w["dist"])
