// model.cuh -- the absorber stage equations of the case study with analytic first and
// second derivatives, for one (scenario, stage).  __host__ __device__: the device
// kernels evaluate values with it, and the host runs the same routine once per stage
// type with a recording emitter to derive the sparsity pattern, so the pattern and
// the values written by the kernel come from one piece of code.
//
// Equations (paper, Sections "Equilibrium process model" and "Case study"):
//   (1)  material balance  L x_i + V y_i - L+ x_i+ - V- y_i- - sum_r nu_ir eps_r = 0
//   (9a) Raoult (water)    P y_H2O - x_H2O Psat(T) = 0
//   (9b) Henry (CO2)       P y_CO2 - rho_L x_CO2 H(T, x_MEA^app, x_H2O^app) = 0
//   (3a) reaction equil.   sum_i nu_ir ln x_i - ln K_r(T) = 0,  activities = x
//   (4)  summation         sum x - 1 = 0,  sum y - 1 = 0
//   (6)  energy balance    L h^L + V h^V - L+ h^L+ - V- h^V- = 0 (ideal mixtures, Q = 0)
//   (10b) hydraulic        V R T / P - u_max pi d^2 / 4 + s = 0,  s >= 0
// with Kent-Eisenberg ln K_r = A + B/T + C ln T + D T, Antoine ln Psat = a - b/(T+c),
// ln H = ha + hb/T + hm x_MEA^app + hw x_H2O^app, apparent fractions normalised over
// (MEA, CO2, H2O)_app, and h_i(T) = ref + cpa (T-Tref) + cpb/2 (T-Tref)^2 + dh.
#pragma once

#include <math.h>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace absorber {

constexpr int N_STAGES = 10;
constexpr int NV = 22;          // unknowns per stage
constexpr int NR = 22;          // rows per stage
constexpr int NSC = N_STAGES * NV;  // unknowns (= rows) per scenario
constexpr int NLOC = 40;        // local variables of one stage's rows
constexpr int NFEED = 18;

// local-variable numbering of one stage's rows
constexpr int LX = 0, LY = 9, LL = 13, LV = 14, LT = 15, LE = 16, LS = 21;
constexpr int AX = 22, AL = 31, AT = 32;     // stream from above (stage n+1)
constexpr int BY = 33, BV = 37, BT = 38;     // stream from below (stage n-1)
constexpr int LD_ = 39;                      // the diameter
// rows
constexpr int R_VH = 11, R_VC = 12, R_RX = 13, R_SX = 18, R_SY = 19, R_E = 20, R_H = 21;

// feed record offsets
constexpr int F_V0 = 0, F_Y0 = 1, F_T0 = 5, F_LIN = 6, F_XIN = 7, F_TIN = 16, F_P = 17;

// stoichiometry nu[species][reaction] of R1..R5; species MEA, MEAH+, H+, MEACOO-,
// HCO3-, OH-, CO3--, CO2, H2O, N2, O2
__host__ __device__ constexpr int nu(int c, int r) {
    // R1: MEAH+ -> MEA + H+ ; R2: HCO3- -> H+ + CO3-- ; R3: H2O -> H+ + OH- ;
    // R4: MEACOO- + H2O -> MEA + HCO3- ; R5: H2O + CO2 -> H+ + HCO3-
    constexpr int t[11][5] = {
        {1, 0, 0, 1, 0},     // MEA
        {-1, 0, 0, 0, 0},    // MEAH+
        {1, 1, 1, 0, 1},     // H+
        {0, 0, 0, -1, 0},    // MEACOO-
        {0, -1, 0, 1, 1},    // HCO3-
        {0, 0, 1, 0, 0},     // OH-
        {0, 1, 0, 0, 0},     // CO3--
        {0, 0, 0, 0, -1},    // CO2
        {0, 0, -1, -1, -1},  // H2O
        {0, 0, 0, 0, 0},     // N2
        {0, 0, 0, 0, 0},     // O2
    };
    return t[c][r];
}

// membership of the liquid species in the apparent MEA / CO2 / H2O totals of (9b)
__host__ __device__ constexpr int app_m(int k) { return (k == 0 || k == 1 || k == 3) ? 1 : 0; }
__host__ __device__ constexpr int app_c(int k) { return (k == 7 || k == 3 || k == 4 || k == 6) ? 1 : 0; }
__host__ __device__ constexpr int app_w(int k) { return (k == 8 || k == 4 || k == 6 || k == 5) ? 1 : 0; }
__host__ __device__ constexpr int app_t(int k) { return app_m(k) + app_c(k) + app_w(k); }
__host__ __device__ constexpr bool in_henry(int k) { return app_t(k) > 0; }

struct Params {
    double R, u_max, d_lo, d_hi, T_lo, T_hi, T_ref;
    double sx[9], sy[4], sT;
    double KE_A[5], KE_B[5], KE_C[5], KE_D[5];
    double psat_a, psat_b, psat_c;
    double henry_a, henry_b, henry_m, henry_w, rho_L;
    double hL_ref[9], hL_cpa[9], hL_cpb[9], hL_dh[9];
    double hV_ref[4], hV_cpa[4], hV_cpb[4], hV_dh[4];
    int nsec;        // column sections, each with its own diameter (1 or 2)
    double dp_stage; // specified pressure drop per stage (relation (7)); 0: P^abs everywhere
    // derived at creation
    double lnsx[9];
    double lnsxr[5];   // sum_c nu_ck ln sx_c: the scales' share of each reaction's quotient
    double hL0[9];   // hL_ref + hL_dh
    double hV0[4];
    double Tlo_s, Thi_s;   // T_lo / sT, T_hi / sT: the scaled temperature bounds
};

constexpr int KSEC = 2;   // most column sections (design-vector entries)

// the section of stage n among K: consecutive stages, floor(n K / N)
__host__ __device__ constexpr int stage_sec(int n, int K) { return (n * K) / N_STAGES; }

// objective weight of section k's diameter: its share of the stages
__host__ __device__ inline double sec_weight(int k, int K) {
    int c = 0;
    for (int n = 0; n < N_STAGES; ++n) c += stage_sec(n, K) == k ? 1 : 0;
    return (double)c / N_STAGES;
}

// pressure of stage n by relation (7) with a specified drop, Pt the top stage's
__host__ __device__ inline double stage_pres(const Params& P, double Pt, int n) {
    return Pt + (double)(N_STAGES - 1 - n) * P.dp_stage;
}

struct StageIn {
    double q[NV];     // own scaled unknowns
    double qa[11];    // from above: xt[9], L, Tt  (the lean feed, scaled, on the top stage)
    double qb[6];     // from below: yt[4], V, Tt  (the flue gas, scaled, on stage 0)
    double d, P;
    bool has_above, has_below;   // neighbour stage exists (its values are unknowns)
};

struct StageLam {
    double own[NR];
    double below[10];   // stage n-1: material multipliers of the 9 liquid species, energy
    double above[5];    // stage n+1: material multipliers of the 4 vapour species, energy
};

// Emitter concept:
//   static constexpr bool want_res, want_jac, want_hes;
//   void res(int r, double v); void jac(int r, int lv, double v); void hes(int i, int j, double v);
#ifdef __CUDACC__
#pragma nv_exec_check_disable
#endif
template <class E>
__host__ __device__ inline void stage_eval(const Params& P, const StageIn& in, const StageLam* lam,
                                           E& e) {
    const double sT = P.sT;
    double x[9], y[4];
#pragma unroll
    for (int l = 0; l < 9; ++l) x[l] = P.sx[l] * in.q[LX + l];
#pragma unroll
    for (int j = 0; j < 4; ++j) y[j] = P.sy[j] * in.q[LY + j];
    const double L = in.q[LL], V = in.q[LV], T = sT * in.q[LT];
    double xa[9], yb[4];
#pragma unroll
    for (int l = 0; l < 9; ++l) xa[l] = P.sx[l] * in.qa[l];
#pragma unroll
    for (int j = 0; j < 4; ++j) yb[j] = P.sy[j] * in.qb[j];
    const double La = in.qa[9], Ta = sT * in.qa[10];
    const double Vb = in.qb[4], Tb = sT * in.qb[5];
    const double Pr = in.P;

    // ---- reciprocals of T + C (Antoine), the stage pressure, the apparent-fraction total
    // of (9b) and T from one division: a = Tc Pr, b = tot T, r = 1 / (a b), then
    // 1/Tc = r b Pr, 1/Pr = r b Tc, 1/tot = r a T, 1/T = r a tot (all positive and O(1e-3
    // .. 1e3) at interior points)
    double am = 0, ac = 0, aw = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        am += app_m(k) * x[k];
        ac += app_c(k) * x[k];
        aw += app_w(k) * x[k];
    }
    const double tot = am + ac + aw;
    const double Tc = T + P.psat_c;
    const double ra = Tc * Pr, rb = tot * T;
    const double r4 = 1.0 / (ra * rb);
    const double rbr = r4 * rb, rar = r4 * ra;
    const double iTc = rbr * Pr, iPr = rbr * Tc, it = rar * T, invT = rar * tot;

    // ---- enthalpies ---------------------------------------------------------------
    const double dT = T - P.T_ref, dTa = Ta - P.T_ref, dTb = Tb - P.T_ref;
    double hL[9], cpL[9], hLa[9], cpLa[9], hV[4], cpV[4], hVb[4], cpVb[4];
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        cpL[l] = P.hL_cpa[l] + P.hL_cpb[l] * dT;
        hL[l] = P.hL0[l] + dT * (P.hL_cpa[l] + 0.5 * P.hL_cpb[l] * dT);
        cpLa[l] = P.hL_cpa[l] + P.hL_cpb[l] * dTa;
        hLa[l] = P.hL0[l] + dTa * (P.hL_cpa[l] + 0.5 * P.hL_cpb[l] * dTa);
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        cpV[j] = P.hV_cpa[j] + P.hV_cpb[j] * dT;
        hV[j] = P.hV0[j] + dT * (P.hV_cpa[j] + 0.5 * P.hV_cpb[j] * dT);
        cpVb[j] = P.hV_cpa[j] + P.hV_cpb[j] * dTb;
        hVb[j] = P.hV0[j] + dTb * (P.hV_cpa[j] + 0.5 * P.hV_cpb[j] * dTb);
    }
    double HL = 0, HV = 0, HLa = 0, HVb = 0, CL = 0, CV = 0, CLa = 0, CVb = 0;
#pragma unroll
    for (int l = 0; l < 9; ++l) {
        HL += x[l] * hL[l];
        CL += x[l] * cpL[l];
        HLa += xa[l] * hLa[l];
        CLa += xa[l] * cpLa[l];
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        HV += y[j] * hV[j];
        CV += y[j] * cpV[j];
        HVb += yb[j] * hVb[j];
        CVb += yb[j] * cpVb[j];
    }

    // ---- (9a) water saturation pressure ---------------------------------------------
    const double ps = exp(P.psat_a - P.psat_b * iTc);
    const double bT2 = P.psat_b * iTc * iTc;
    const double ps1 = ps * bT2;                                        // dPsat/dT
    const double ps2 = ps * (bT2 * bT2 - 2.0 * P.psat_b * iTc * iTc * iTc);  // d2Psat/dT2
    // reciprocals of the scaled liquid fractions (derivatives of their logarithms), all
    // nine from one division: prefix products p_c = q_0 ... q_c, r = 1 / p_8, then walking
    // back 1/q_c = r p_{c-1} and r <- r q_c (the fractions are positive and O(1))
    double iq[9];
    if (E::want_jac || E::want_hes) {
        double pre[9];
        pre[0] = in.q[LX];
#pragma unroll
        for (int c = 1; c < 9; ++c) pre[c] = pre[c - 1] * in.q[LX + c];
        double r = 1.0 / pre[8];
#pragma unroll
        for (int c = 8; c > 0; --c) {
            iq[c] = r * pre[c - 1];
            r *= in.q[LX + c];
        }
        iq[0] = r;
    } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) iq[c] = 0.0;
    }

    // ---- (9b) Henry coefficient --------------------------------------------------------
    const double um = am * it, uw = aw * it;
    const double g = P.henry_a + P.henry_b * invT + P.henry_m * um + P.henry_w * uw;
    const double Hh = exp(g);
    const double gT = -P.henry_b * invT * invT;
    const double gTT = 2.0 * P.henry_b * invT * invT * invT;
    double gk[9];   // dg/dx_k (physical x)
#pragma unroll
    for (int k = 0; k < 9; ++k)
        gk[k] = (P.henry_m * (app_m(k) - um * app_t(k)) + P.henry_w * (app_w(k) - uw * app_t(k))) * it;
    const double rhoH = P.rho_L * Hh;
    const double x7 = x[7];

    // ---- residuals ---------------------------------------------------------------------
    if (E::want_res) {
#pragma unroll
        for (int c = 0; c < 11; ++c) {
            double r = 0.0;
            if (c < 9) r += L * x[c] - La * xa[c];
            if (c >= 7) r += V * y[c - 7] - Vb * yb[c - 7];
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (nu(c, k) != 0) r -= nu(c, k) * in.q[LE + k];
            e.res(c, r);
        }
        e.res(R_VH, Pr * y[1] - x[8] * ps);
        e.res(R_VC, Pr * y[0] - rhoH * x7);
        // sum_c nu_ck ln x_c as one logarithm per reaction: every nu is +-1, so it is
        // ln(prod over products of q_c / prod over reactants of q_c) + sum_c nu_ck ln sx_c
        // (the scaled fractions are O(1): the quotients stay far from over- and underflow)
        const double lT = log(T);
        // the five quotients' denominators inverted together from one division (prefix
        // products, then back)
        double qn[5], qd[5], pre[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            double num = 1.0, den = 1.0;
#pragma unroll
            for (int c = 0; c < 9; ++c) {
                if (nu(c, k) > 0) num *= in.q[LX + c];
                if (nu(c, k) < 0) den *= in.q[LX + c];
            }
            qn[k] = num;
            qd[k] = den;
            pre[k] = k ? pre[k - 1] * den : den;
        }
        double rq = 1.0 / pre[4];
#pragma unroll
        for (int k = 4; k >= 0; --k) {
            const double rk = k ? rq * pre[k - 1] : rq;
            if (k) rq *= qd[k];
            const double r = -(P.KE_A[k] + P.KE_B[k] * invT + P.KE_C[k] * lT + P.KE_D[k] * T) + P.lnsxr[k] +
                             log(qn[k] * rk);
            e.res(R_RX + k, r);
        }
        double sx_ = -1.0, sy_ = -1.0;
#pragma unroll
        for (int l = 0; l < 9; ++l) sx_ += x[l];
#pragma unroll
        for (int j = 0; j < 4; ++j) sy_ += y[j];
        e.res(R_SX, sx_);
        e.res(R_SY, sy_);
        e.res(R_E, L * HL + V * HV - La * HLa - Vb * HVb);
        e.res(R_H, V * P.R * T * iPr - P.u_max * M_PI * in.d * in.d * 0.25 + in.q[LS]);
    }

    // ---- Jacobian ----------------------------------------------------------------------
    if (E::want_jac) {
#pragma unroll
        for (int c = 0; c < 11; ++c) {
            if (c < 9) {
                e.jac(c, LX + c, L * P.sx[c]);
                e.jac(c, LL, x[c]);
                if (in.has_above) {
                    e.jac(c, AX + c, -La * P.sx[c]);
                    e.jac(c, AL, -xa[c]);
                }
            }
            if (c >= 7) {
                const int j = c - 7;
                e.jac(c, LY + j, V * P.sy[j]);
                e.jac(c, LV, y[j]);
                if (in.has_below) {
                    e.jac(c, BY + j, -Vb * P.sy[j]);
                    e.jac(c, BV, -yb[j]);
                }
            }
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (nu(c, k) != 0) e.jac(c, LE + k, -(double)nu(c, k));
        }
        // (9a)
        e.jac(R_VH, LY + 1, Pr * P.sy[1]);
        e.jac(R_VH, LX + 8, -P.sx[8] * ps);
        e.jac(R_VH, LT, -x[8] * ps1 * sT);
        // (9b)
        e.jac(R_VC, LY + 0, Pr * P.sy[0]);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            if (in_henry(k)) e.jac(R_VC, LX + k, -rhoH * ((k == 7 ? 1.0 : 0.0) + x7 * gk[k]) * P.sx[k]);
        e.jac(R_VC, LT, -rhoH * x7 * gT * sT);
        // (3a)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
#pragma unroll
            for (int c = 0; c < 9; ++c)
                if (nu(c, k) != 0) e.jac(R_RX + k, LX + c, nu(c, k) * iq[c]);
            e.jac(R_RX + k, LT, -sT * (-P.KE_B[k] * invT * invT + P.KE_C[k] * invT + P.KE_D[k]));
        }
        // (4)
#pragma unroll
        for (int l = 0; l < 9; ++l) e.jac(R_SX, LX + l, P.sx[l]);
#pragma unroll
        for (int j = 0; j < 4; ++j) e.jac(R_SY, LY + j, P.sy[j]);
        // (6)
#pragma unroll
        for (int l = 0; l < 9; ++l) e.jac(R_E, LX + l, L * P.sx[l] * hL[l]);
#pragma unroll
        for (int j = 0; j < 4; ++j) e.jac(R_E, LY + j, V * P.sy[j] * hV[j]);
        e.jac(R_E, LL, HL);
        e.jac(R_E, LV, HV);
        e.jac(R_E, LT, sT * (L * CL + V * CV));
        if (in.has_above) {
#pragma unroll
            for (int l = 0; l < 9; ++l) e.jac(R_E, AX + l, -La * P.sx[l] * hLa[l]);
            e.jac(R_E, AL, -HLa);
            e.jac(R_E, AT, -sT * La * CLa);
        }
        if (in.has_below) {
#pragma unroll
            for (int j = 0; j < 4; ++j) e.jac(R_E, BY + j, -Vb * P.sy[j] * hVb[j]);
            e.jac(R_E, BV, -HVb);
            e.jac(R_E, BT, -sT * Vb * CVb);
        }
        // (10b)
        e.jac(R_H, LV, P.R * T * iPr);
        e.jac(R_H, LT, V * P.R * sT * iPr);
        e.jac(R_H, LS, 1.0);
        e.jac(R_H, LD_, -P.u_max * M_PI * in.d * 0.5);
    }

    // ---- Lagrangian Hessian block of this stage's unknowns (lower triangle) ------------
    // Terms come from this stage's rows and from the neighbours' rows in which this
    // stage's streams appear: the stage below reads (L, x, T) of this stage as its
    // "from above" stream, the stage above reads (V, y, T) as its "from below" stream.
    if (E::want_hes) {
        const double* lo = lam->own;
        double muL[9], muV[4];
#pragma unroll
        for (int c = 0; c < 9; ++c) muL[c] = lo[c] - (in.has_below ? lam->below[c] : 0.0);
#pragma unroll
        for (int j = 0; j < 4; ++j) muV[j] = lo[7 + j] - (in.has_above ? lam->above[j] : 0.0);
        const double muEL = lo[R_E] - (in.has_below ? lam->below[9] : 0.0);
        const double muEV = lo[R_E] - (in.has_above ? lam->above[4] : 0.0);
        const double lVH = lo[R_VH], lVC = lo[R_VC], lH = lo[R_H];

        // Henry block over the species of the apparent totals (and the ln x diagonals)
#pragma unroll
        for (int k = 0; k < 9; ++k) {
#pragma unroll
            for (int l = 0; l <= k; ++l) {
                double v = 0.0;
                bool present = false;
                if (in_henry(k) && in_henry(l)) {
                    const double gkl = (P.henry_m * (-app_m(k) * app_t(l) - app_m(l) * app_t(k) +
                                                     2.0 * um * app_t(k) * app_t(l)) +
                                        P.henry_w * (-app_w(k) * app_t(l) - app_w(l) * app_t(k) +
                                                     2.0 * uw * app_t(k) * app_t(l))) * it * it;
                    const double d2 = (k == 7 ? gk[l] : 0.0) + (l == 7 ? gk[k] : 0.0) +
                                      x7 * (gk[k] * gk[l] + gkl);
                    v += -lVC * rhoH * d2 * P.sx[k] * P.sx[l];
                    present = true;
                }
                if (k == l) {
                    double a = 0.0;
                    bool any = false;
#pragma unroll
                    for (int r = 0; r < 5; ++r)
                        if (nu(k, r) != 0) {
                            a += lo[R_RX + r] * nu(k, r);
                            any = true;
                        }
                    if (any) {
                        v += -a * iq[k] * iq[k];
                        present = true;
                    }
                }
                if (present) e.hes(LX + k, LX + l, v);
            }
        }
        // (L, x_l) and (V, y_j): bilinear flows in (1) and (6)
#pragma unroll
        for (int l = 0; l < 9; ++l) e.hes(LL, LX + l, P.sx[l] * (muL[l] + muEL * hL[l]));
#pragma unroll
        for (int j = 0; j < 4; ++j) e.hes(LV, LY + j, P.sy[j] * (muV[j] + muEV * hV[j]));
        // (T, x_l)
#pragma unroll
        for (int l = 0; l < 9; ++l) {
            double v = sT * P.sx[l] * muEL * L * cpL[l];
            if (l == 8) v += -lVH * P.sx[8] * ps1 * sT;
            if (in_henry(l)) v += -lVC * rhoH * gT * ((l == 7 ? 1.0 : 0.0) + x7 * gk[l]) * P.sx[l] * sT;
            e.hes(LT, LX + l, v);
        }
        // (T, y_j)
#pragma unroll
        for (int j = 0; j < 4; ++j) e.hes(LT, LY + j, sT * P.sy[j] * muEV * V * cpV[j]);
        e.hes(LT, LL, sT * muEL * CL);
        e.hes(LT, LV, sT * muEV * CV + lH * P.R * sT * iPr);
        // (T, T)
        {
            double dCL = 0.0, dCV = 0.0;
#pragma unroll
            for (int l = 0; l < 9; ++l) dCL += x[l] * P.hL_cpb[l];
#pragma unroll
            for (int j = 0; j < 4; ++j) dCV += y[j] * P.hV_cpb[j];
            double v = muEL * L * dCL + muEV * V * dCV - lVH * x[8] * ps2 - lVC * rhoH * x7 * (gT * gT + gTT);
#pragma unroll
            for (int r = 0; r < 5; ++r)
                v -= lo[R_RX + r] * (2.0 * P.KE_B[r] * invT * invT * invT - P.KE_C[r] * invT * invT);
            e.hes(LT, LT, sT * sT * v);
        }
    }
}

}  // namespace absorber
