// vec_kernels.cuh -- interior-point vector kernels (A5-A7) over one or many problems.
//
// One thread per (scenario slot, stage): grid (ceil(S / 128), N_STAGES).  Every scalar of
// the method (mu, tau, step sizes, delta_w, the diameter d and its step) is per problem:
// scalars from ps (BView), d and its step from the problem's d slot [NSC * ld + p] of
// the primal vectors.  Reductions store per-thread partials (store_partials) that
// reduce_kernel combines them per problem in a fixed order.
#pragma once

#include "kernels.cuh"

namespace absorber {

// Schur: r_d and S_d per problem; PS_BASE: 1 if the problem starts from the base states
// PS_RD / PS_SD: the first design entry's right-hand side and the Schur complement (its
// (0,0) entry with two sections, whose other entries are PS_SD01, PS_SD11, PS_RD1)
enum PsExtra { PS_RD = PS_COUNT, PS_SD, PS_BASE, PS_DC, PS_SD01, PS_SD11, PS_RD1, PS_NFIELDS };

__device__ inline double lo_of(const Params& P, int j) { return j == LT ? P.Tlo_s : 0.0; }
__device__ inline double hi_of(const Params& P, int /*j*/) { return P.Thi_s; }

struct RedOps {
    int op[12];
};

// Kernels below with QS = 4 threads per (scenario, stage): a 128-thread block covers 32
// scenarios, lane = scenario and warp q of the block handles the stage's unknowns
// j = q, q + QS, ...  Every lane of a warp works on the same rows, so the sparse-product
// loops have warp-uniform trip counts and table reads, and every load is coalesced over
// 32 scenarios.  Four times the warps of one thread per (scenario, stage): these kernels
// wait on global loads, and 5000 scenarios x 10 stages alone fill only a quarter of the
// GPU's warp slots.  The QS partial values of a (scenario, stage) combine through shared
// memory as (v0 op v1) op (v2 op v3).
constexpr int QS = 4;
constexpr int QS_SCEN = 32;   // scenarios per 128-thread block

__device__ __forceinline__ double comb(int op, double a, double b) {
    return op == RSUM ? a + b : (op == RMAX ? ((b > a || b != b) ? b : a) : fmin(a, b));
}

// combine v[0..NC) over the block's QS warps (ops[k]: RSUM, RMAX or RMIN); warp 0 ends
// with the combined values.  Every thread of the block must call it.
template <int K, int NC>
__device__ __forceinline__ void group_combine(double (&v)[K], double (*sm)[NC][32], const int (&ops)[NC]) {
    const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < NC; ++k) sm[q][k][lane] = v[k];
    __syncthreads();
    if (q == 0) {
#pragma unroll
        for (int k = 0; k < NC; ++k)
            v[k] = comb(ops[k], comb(ops[k], sm[0][k][lane], sm[1][k][lane]), comb(ops[k], sm[2][k][lane], sm[3][k][lane]));
    }
}

// J^T lambda for the stage's unknowns and the optimality-error partials:
// [0] max |J^T l - zL + zU|, [1] sum |lambda|, [2] sum |zL| + |zU|, [3] max and [4] min
// complementarity product over bounded unknowns, [5] the stage's hydraulic multiplier
// (two sections: [5] for the first section's stages, [6] for the second's, each 0 on the
// other's).  QS threads per (scenario, stage); grid (ceil(S / QS_SCEN), N_STAGES), 128 threads.
__global__ void __launch_bounds__(128) dual_kernel(const Params P, int S, int64_t ld, const BView b,
                                                   const double* __restrict__ jac, const double* __restrict__ lam,
                                                   const double* __restrict__ x, const double* __restrict__ zL,
                                                   const double* __restrict__ zU, double* __restrict__ jtl,
                                                   double* part) {
    __shared__ double sm[QS][5][32];
    const int q = threadIdx.x >> 5;
    const int s = blockIdx.x * QS_SCEN + (threadIdx.x & 31);
    const int n = blockIdx.y;
    const bool live = live_prob(b, s, S, PS_ACT) >= 0;
    double v[6] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    if (live) {
        unsigned long long k0 = 0;   // max |J^T l - zL + zU| as an integer key (NaN survives)
#pragma unroll 1
        for (int j = q; j < NV; j += QS) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double gj = jt_one(ld, jac, lam, s, n, j);
            jtl[o] = gj;
            const double zl = zL[o], zu = zU[o];
            k0 = key_max(k0, mag_key(gj - zl + zu));
            v[1] += fabs(lam[o]);
            v[2] += fabs(zl) + fabs(zu);
            const double xv = x[o];
            if (has_lo(j)) {
                const double cp = zl * (xv - lo_of(P, j));
                v[3] = fmax(v[3], cp);
                v[4] = fmin(v[4], cp);
            }
            if (has_hi(j)) {
                const double cp = zu * (hi_of(P, j) - xv);
                v[3] = fmax(v[3], cp);
                v[4] = fmin(v[4], cp);
            }
        }
        v[0] = key_double(k0);
    }
    constexpr int ops[5] = {RMAX, RSUM, RSUM, RMAX, RMIN};
    group_combine<6, 5>(v, sm, ops);
    if (!live || q != 0) return;
    const double lh = lam[(int64_t)(NR * n + R_H) * ld + s];
    if (P.nsec == 1) {
        v[5] = lh;
        store_partials<6>(v, part, ld, s, n);
    } else {
        const bool top = stage_sec(n, P.nsec) == 1;
        const double w7[7] = {v[0], v[1], v[2], v[3], v[4], top ? 0.0 : lh, top ? lh : 0.0};
        store_partials<7>(w7, part, ld, s, n);
    }
}

// Elementwise kernels below: one thread per (entry v, scenario s), grid (ceil(S / 128),
// 220): v = 22 n + j is the block's row, so the bound pattern of unknown j is the same on
// every lane of a block, and every load and store is coalesced over scenarios.

// barrier diagonal Sigma and right-hand sides r_z = -(J^T l - mu/sl + mu/su), r_c = -c;
// the reciprocal slacks are kept for step_kernel
__global__ void __launch_bounds__(128) rhs_kernel(const Params P, int S, int64_t ld, const BView b,
                                                  const double* __restrict__ x, const double* __restrict__ zL,
                                                  const double* __restrict__ zU, const double* __restrict__ jtl,
                                                  const double* __restrict__ c, double* __restrict__ sig,
                                                  double* __restrict__ rz, double* __restrict__ rc,
                                                  double* __restrict__ invL, double* __restrict__ invU) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y, j = v % NV;
    const int p = live_prob(b, s, S, PS_ACT);
    if (p < 0) return;
    const double mu = psv(b, PS_MU, p);
    const int64_t o = (int64_t)v * ld + s;
    const double xv = x[o];
    double sg = 0.0, gb = 0.0;
    if (has_lo(j)) {
        const double inv = 1.0 / (xv - lo_of(P, j));   // one division per bound
        invL[o] = inv;
        sg += zL[o] * inv;
        gb -= mu * inv;
    }
    if (has_hi(j)) {
        const double inv = 1.0 / (hi_of(P, j) - xv);
        invU[o] = inv;
        sg += zU[o] * inv;
        gb += mu * inv;
    }
    sig[o] = sg;
    rz[o] = -(jtl[o] + gb);
    rc[o] = -c[o];
}

// Schur partial sums with H = W + Sigma (W optional), q = J^-1 b for the design entries
// (q1: the second section's, or null for one section): with SCHUR_DD [0] q^T H q,
// [1] q^T q and, with q1, [2] q^T H q1, [3] q^T q1, [6] q1^T H q1, [7] q1^T q1; with
// SCHUR_RHS [2] q^T (r - H p), [3] q^T p and, with q1, [0] q1^T (r - H p), [1] q1^T p;
// always [4] (and with q1 [8]) the scenario's d-d Hessian entry of each section and [5]
// the singular flag.  Terms not asked for are 0.  Optionally the vectors behind them:
// hq = H q, hq1 = H q1 (SCHUR_DD), t = r - H p (SCHUR_RHS), from which dz_fast_kernel
// forms g without another product with H.  TWO: q1 given (the one-entry instance keeps the
// one-entry work and shared memory).
enum { SCHUR_DD = 1, SCHUR_RHS = 2 };

template <bool TWO>
__global__ void __launch_bounds__(128) schur_kernel(int S, int64_t ld, const BView b, const double* __restrict__ hes,
                                                    const double* __restrict__ sig, bool use_w,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    const double* __restrict__ r, const int* __restrict__ sing,
                                                    double* part, int terms, double* __restrict__ hq,
                                                    double* __restrict__ tv, const double* __restrict__ q1 = nullptr,
                                                    double* __restrict__ hq1 = nullptr) {
    constexpr int NC = TWO ? 6 : 4;   // sums combined over the block's row groups
    __shared__ double sm[QS][NC][32];
    const int g = threadIdx.x >> 5;
    const int s = blockIdx.x * QS_SCEN + (threadIdx.x & 31);
    const int n = blockIdx.y;
    const bool live = live_prob(b, s, S, PS_ACT) >= 0;
    if (!TWO) q1 = nullptr;
    double a[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (live) {
#pragma unroll
        for (int j0 = 0; j0 < NV; j0 += QS) {
            const int j = j0 + g;
            if (j < NV) {
                const int64_t o = (int64_t)(NV * n + j) * ld + s;
                const double qj = q[o];
                const double q1j = TWO ? q1[o] : 0.0;
                if (terms & SCHUR_DD) {
                    const double hqj = hv_one(ld, hes, sig, 0.0, use_w, q, s, n, j);
                    if (hq) hq[o] = hqj;
                    a[0] += qj * hqj;
                    a[1] += qj * qj;
                    if (TWO) {
                        const double hq1j = hv_one(ld, hes, sig, 0.0, use_w, q1, s, n, j);
                        if (hq1) hq1[o] = hq1j;
                        a[2] += qj * hq1j;
                        a[3] += qj * q1j;
                        a[4] += q1j * hq1j;
                        a[5] += q1j * q1j;
                    }
                }
                if (terms & SCHUR_RHS) {
                    if (r) {
                        const double tj = r[o] - (p ? hv_one(ld, hes, sig, 0.0, use_w, p, s, n, j) : 0.0);
                        if (tv) tv[o] = tj;
                        a[2] += qj * tj;
                        if (TWO) a[0] += q1j * tj;
                    }
                    if (p) {
                        a[3] += qj * p[o];
                        if (TWO) a[1] += q1j * p[o];
                    }
                }
            }
        }
    }
    constexpr int ops[NC] = {};   // RSUM (0) for every sum
    group_combine<6, NC>(a, sm, ops);
    if (!live || g != 0) return;
    double v[9] = {a[0], a[1], a[2], a[3], 0.0, 0.0, a[4], a[5], 0.0};
    if (n == 0) {
        if (use_w) {
            v[4] = hes[(int64_t)(NHS * N_STAGES) * ld + s];
            if (TWO) v[8] = hes[(int64_t)(NHS * N_STAGES + 1) * ld + s];
        }
        if (sing) v[5] = (double)sing[s];
    }
    if (TWO) store_partials<9>(v, part, ld, s, n);
    else {
        const double w6[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
        store_partials<6>(w6, part, ld, s, n);
    }
}

// dz = p - q dd ;  g = r - (W + Sigma + dw I) dz ;  dd, dw of the slot's problem.
// QS threads per (scenario, stage); each writes its unknowns of dz, then (after the
// block's writes) its entries of g, which read the whole stage's dz.
__global__ void __launch_bounds__(128) dz_kernel(int S, int64_t ld, const BView b, const double* __restrict__ hes,
                                                 const double* __restrict__ sig, bool use_w,
                                                 const double* __restrict__ p, const double* __restrict__ q,
                                                 const double* __restrict__ r, double* dz, double* __restrict__ g) {
    const int gq = threadIdx.x >> 5;
    const int s = blockIdx.x * QS_SCEN + (threadIdx.x & 31);
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_ACT);
    const bool live = pr >= 0;
    if (live) {
        const double dd = dz[(int64_t)NSC * ld + pr];
        for (int j = gq; j < NV; j += QS) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            dz[o] = p[o] - q[o] * dd;
        }
    }
    __syncthreads();   // the block's dz entries are visible to all its threads below
    if (!live) return;
    const double dw = b.ps ? psv(b, PS_DW, pr) : 0.0;
    for (int j = gq; j < NV; j += QS) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        g[o] = r[o] - hv_one(ld, hes, sig, dw, use_w, dz, s, n, j);
    }
}

// dz = p - q dd and g = r - (H + dw I) dz from the Schur pass's vectors t = r - H p and
// hq = H q (H = W + Sigma): g = t - dw p + dd (hq + dw q), no product with H; with a
// second design entry also - q1 dd1 and + dd1 (hq1 + dw q1).  Elementwise.
__global__ void __launch_bounds__(128) dz_fast_kernel(int S, int64_t ld, const BView b, const double* __restrict__ p,
                                                      const double* __restrict__ q, const double* __restrict__ t,
                                                      const double* __restrict__ hq, double* __restrict__ dz,
                                                      double* __restrict__ g, const double* __restrict__ q1 = nullptr,
                                                      const double* __restrict__ hq1 = nullptr) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    const double dd = dz[(int64_t)NSC * ld + pr];
    const double dw = b.ps ? psv(b, PS_DW, pr) : 0.0;
    const int64_t o = (int64_t)blockIdx.y * ld + s;
    const double pj = p[o], qj = q[o];
    if (!q1) {
        dz[o] = pj - qj * dd;
        g[o] = t[o] - dw * pj + dd * (hq[o] + dw * qj);
    } else {
        const double dd1 = dz[(int64_t)NSC * ld + b.NP + pr];
        const double q1j = q1[o];
        dz[o] = pj - qj * dd - q1j * dd1;
        g[o] = t[o] - dw * pj + dd * (hq[o] + dw * qj) + dd1 * (hq1[o] + dw * q1j);
    }
}

// residual of the full KKT system: rho_z = r_z - (H dz + J^T dl), rho_c = r_c - (J dz + b dd).
// The z part is formed from the last block-elimination solve of the refinement: with g =
// r' - H dz' (its right-hand side r' and solution dz', dl' -- the first solve, or the
// last correction), rho_z = g - J^T dl' (r' is r_z or the previous residual, so this is
// r_z - H dz - J^T dl for the accumulated dz, dl without forming H dz again).
// partials: [0] max|rho_z|, [1] max|rho_c|, [2] the stage's hydraulic dl, [3] max|r_z|,
// [4] max|r_c|.  QS threads per (scenario, stage).
__global__ void __launch_bounds__(128) kkt_residual_kernel(int S, int64_t ld, const BView b,
                                                           const double* __restrict__ jac,
                                                           const double* __restrict__ g,
                                                           const double* __restrict__ dlast,
                                                           const double* __restrict__ dz, const double* __restrict__ dl,
                                                           const double* __restrict__ rz, const double* __restrict__ rc,
                                                           double* __restrict__ rhoz, double* __restrict__ rhoc,
                                                           double* part, int nsec = 1) {
    __shared__ double sm[QS][5][32];
    const int gq = threadIdx.x >> 5;
    const int s = blockIdx.x * QS_SCEN + (threadIdx.x & 31);
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_ACT);
    const bool live = pr >= 0;
    const int sec = stage_sec(n, nsec);
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (live) {
        const double dd = dz[(int64_t)NSC * ld + (int64_t)sec * b.NP + pr];   // the stage's section
        bool bad = false;
        for (int j = gq; j < NV; j += QS) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double a = g[o] - jt_one(ld, jac, dlast, s, n, j);
            const double c = rc[o] - jv_one(ld, jac, dz, dd, s, n, j);
            rhoz[o] = a;
            rhoc[o] = c;
            v[0] = fmax(v[0], fabs(a));
            v[1] = fmax(v[1], fabs(c));
            v[3] = fmax(v[3], fabs(rz[o]));
            v[4] = fmax(v[4], fabs(rc[o]));
            bad = bad || a != a || c != c;
        }
        if (bad) v[0] = NAN;   // fmax skips a NaN: any NaN of the rows makes [0] NaN
    }
    constexpr int ops[5] = {RMAX, RMAX, RSUM, RMAX, RMAX};   // [2] is set below
    group_combine<5, 5>(v, sm, ops);
    if (!live || gq != 0) return;
    const double dlh = dl[(int64_t)(NR * n + R_H) * ld + s];
    if (nsec == 1) {
        v[2] = dlh;
        store_partials<5>(v, part, ld, s, n);
    } else {
        // the hydraulic dl by section: [2] the first's, [5] the second's
        const double w6[6] = {v[0], v[1], sec == 0 ? dlh : 0.0, v[3], v[4], sec == 1 ? dlh : 0.0};
        store_partials<6>(w6, part, ld, s, n);
    }
}

// bound-multiplier steps and step-size limits (mu, tau of the problem):
// [0] min primal ratio (alpha_max), [1] min dual ratio (alpha_z),
// [2] barrier gradient . dz, [3] max |dz| / (1 + |z|).  invL, invU: the reciprocal slacks
// rhs_kernel formed at the same x.
__global__ void __launch_bounds__(128) step_kernel(const Params P, int S, int64_t ld, const BView b,
                                                   const double* __restrict__ x, const double* __restrict__ dz,
                                                   const double* __restrict__ zL, const double* __restrict__ zU,
                                                   const double* __restrict__ invL, const double* __restrict__ invU,
                                                   double* __restrict__ dzL, double* __restrict__ dzU, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    const double mu = psv(b, PS_MU, pr), tau = psv(b, PS_TAU, pr);
    // the minima of tau s / |d| (primal) and tau z / |dz| (dual), and the maximum of
    // |d| / (1 + |x|), are carried as fractions num / den (den > 0) compared by
    // cross-multiplication: one division per bound (1 / slack) and one per ratio at the end
    double an = 1.0, ad = 1.0, zn = 1.0, zd = 1.0, rn = 0.0, rd = 1.0;
    double gphi = 0.0;
    bool dnan = false;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        const double xv = x[o], d = dz[o];
        const double ad_ = fabs(d), ax = 1.0 + fabs(xv);
        if (ad_ * rd > rn * ax) {
            rn = ad_;
            rd = ax;
        }
        dnan = dnan || d != d;
        if (has_lo(j)) {
            const double sl = xv - lo_of(P, j), inv = invL[o];
            const double z = zL[o];
            const double dzl = mu * inv - z - (z * inv) * d;
            dzL[o] = dzl;
            if (d < 0.0 && tau * sl * ad < an * -d) {
                an = tau * sl;
                ad = -d;
            }
            if (dzl < 0.0 && tau * z * zd < zn * -dzl) {
                zn = tau * z;
                zd = -dzl;
            }
            gphi += (-mu * inv) * d;
        } else {
            dzL[o] = 0.0;
        }
        if (has_hi(j)) {
            const double su = hi_of(P, j) - xv, inv = invU[o];
            const double z = zU[o];
            const double dzu = mu * inv - z + (z * inv) * d;
            dzU[o] = dzu;
            if (d > 0.0 && tau * su * ad < an * d) {
                an = tau * su;
                ad = d;
            }
            if (dzu < 0.0 && tau * z * zd < zn * -dzu) {
                zn = tau * z;
                zd = -dzu;
            }
            gphi += (mu * inv) * d;
        } else {
            dzU[o] = 0.0;
        }
    }
    const double v[4] = {an / ad, zn / zd, gphi, dnan ? NAN : rn / rd};
    store_partials<4>(v, part, ld, s, n);
}

// primal fraction-to-the-boundary limit of a direction (problems flagged PS_LSACT)
__global__ void __launch_bounds__(128) ftb_kernel(const Params P, int S, int64_t ld, const BView b,
                                                  const double* __restrict__ x, const double* __restrict__ dz,
                                                  double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_LSACT);
    if (pr < 0) return;
    const double tau = psv(b, PS_TAU, pr);
    double an = 1.0, ad = 1.0;   // min of tau s / |d| as a fraction (see step_kernel)
    bool dnan = false;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        const double xv = x[o], d = dz[o];
        if (has_lo(j) && d < 0.0) {
            const double sl = xv - lo_of(P, j);
            if (tau * sl * ad < an * -d) {
                an = tau * sl;
                ad = -d;
            }
        }
        if (has_hi(j) && d > 0.0) {
            const double su = hi_of(P, j) - xv;
            if (tau * su * ad < an * d) {
                an = tau * su;
                ad = d;
            }
        }
        dnan = dnan || d != d;
    }
    const double v[1] = {dnan ? NAN : an / ad};
    store_partials<1>(v, part, ld, s, n);
}

// accept the step of the problems flagged PS_ACT, then the kappa_Sigma safeguard on the
// bound multipliers
__global__ void __launch_bounds__(128) accept_kernel(const Params P, int S, int64_t ld, const BView b, double ksig,
                                                     double* __restrict__ x, const double* __restrict__ dz,
                                                     double* __restrict__ lam, const double* __restrict__ dl,
                                                     double* __restrict__ zL, const double* __restrict__ dzL,
                                                     double* __restrict__ zU, const double* __restrict__ dzU) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y, j = v % NV;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    const double alpha = psv(b, PS_ALPHA, pr), alpha_z = psv(b, PS_ALPHAZ, pr), mu = psv(b, PS_MU, pr);
    const double mlo = mu / ksig, mhi = ksig * mu;
    const int64_t o = (int64_t)v * ld + s;
    const double xv = x[o] + alpha * dz[o];
    x[o] = xv;
    lam[o] += alpha * dl[o];
    // z kept within [mu / (k_sigma s), k_sigma mu / s]: a division only when it clamps
    if (has_lo(j)) {
        const double sl = xv - lo_of(P, j);
        const double z = zL[o] + alpha_z * dzL[o];
        zL[o] = (z * sl < mlo || z * sl > mhi) ? fmin(fmax(z, mlo / sl), mhi / sl) : z;
    }
    if (has_hi(j)) {
        const double su = hi_of(P, j) - xv;
        const double z = zU[o] + alpha_z * dzU[o];
        zU[o] = (z * su < mlo || z * su > mhi) ? fmin(fmax(z, mlo / su), mhi / su) : z;
    }
}

// the problems' own step of their design entries: x[d_p] += alpha_p dz[d_p]   (one thread
// per problem)
__global__ void dstep_kernel(int64_t ld, const BView b, double* __restrict__ x, const double* __restrict__ dz,
                             int nsec = 1) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.NP || psv(b, PS_ACT, p) == 0.0) return;
    for (int k = 0; k < nsec; ++k) {
        const int64_t o = (int64_t)NSC * ld + (int64_t)k * b.NP + p;
        x[o] += psv(b, PS_ALPHA, p) * dz[o];
    }
}

// starting point: every stage copies the inlet streams (or, with base and the problem's
// PS_BASE set, the stage states of problem p's expected-value solution at
// base[v * ldb + p], or of the one shared solution at base[v * ldb]), the slack from the hydraulic row at the problem's d (already in
// x's d slot); pushed into the bounds
__global__ void __launch_bounds__(128) init_kernel(const Params P, int S, int64_t ld, const BView b,
                                                   const double* __restrict__ feed, const double* __restrict__ base,
                                                   int64_t ldb, bool base_shared, double push, double frac,
                                                   double* __restrict__ x,
                                                   double* __restrict__ zL, double* __restrict__ zU,
                                                   double* __restrict__ lam) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    const double d = x[(int64_t)NSC * ld + (int64_t)stage_sec(n, P.nsec) * b.NP + pr];   // the stage's section
    double q[NV];
    if (base && (!b.ps || psv(b, PS_BASE, pr) != 0.0)) {
#pragma unroll
        for (int j = 0; j < NV; ++j) q[j] = base[(int64_t)(NV * n + j) * ldb + (base_shared ? 0 : pr)];
    } else {
#pragma unroll
        for (int l = 0; l < 9; ++l) q[LX + l] = feed[(int64_t)(F_XIN + l) * ld + s] / P.sx[l];
#pragma unroll
        for (int j = 0; j < 4; ++j) q[LY + j] = feed[(int64_t)(F_Y0 + j) * ld + s] / P.sy[j];
        q[LL] = feed[(int64_t)F_LIN * ld + s];
        q[LV] = feed[(int64_t)F_V0 * ld + s];
        q[LT] = 0.5 * (feed[(int64_t)F_T0 * ld + s] + feed[(int64_t)F_TIN * ld + s]) / P.sT;
#pragma unroll
        for (int r = 0; r < 5; ++r) q[LE + r] = 0.0;
    }
    q[LS] = P.u_max * M_PI * d * d * 0.25 - q[LV] * P.R * (P.sT * q[LT]) / stage_pres(P, feed[(int64_t)F_P * ld + s], n);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        double v = q[j];
        const double lo = lo_of(P, j), hi = hi_of(P, j);
        if (has_lo(j)) {
            const double w = has_hi(j) ? frac * (hi - lo) : INFINITY;
            v = fmax(v, lo + fmin(push * fmax(1.0, fabs(lo)), w));
        }
        if (has_hi(j)) {
            const double w = has_lo(j) ? frac * (hi - lo) : INFINITY;
            v = fmin(v, hi - fmin(push * fmax(1.0, fabs(hi)), w));
        }
        x[o] = v;
        zL[o] = has_lo(j) ? 1.0 : 0.0;
        zU[o] = has_hi(j) ? 1.0 : 0.0;
        lam[o] = 0.0;
    }
}

// warm start: push every bounded unknown of x into its bounds as the cold start does and
// put its bound multipliers on the central path of the problem's mu: z = mu / slack
__global__ void __launch_bounds__(128) warm_push_kernel(const Params P, int S, int64_t ld, const BView b, double push,
                                                        double frac, double* __restrict__ x, double* __restrict__ zL,
                                                        double* __restrict__ zU) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    const double mu = psv(b, PS_MU, pr);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        double v = x[o];
        const double lo = lo_of(P, j), hi = hi_of(P, j);
        if (has_lo(j)) {
            const double w = has_hi(j) ? frac * (hi - lo) : INFINITY;
            v = fmax(v, lo + fmin(push * fmax(1.0, fabs(lo)), w));
        }
        if (has_hi(j)) {
            const double w = has_lo(j) ? frac * (hi - lo) : INFINITY;
            v = fmin(v, hi - fmin(push * fmax(1.0, fabs(hi)), w));
        }
        x[o] = v;
        zL[o] = has_lo(j) ? mu / (v - lo) : 0.0;
        zU[o] = has_hi(j) ? mu / (hi - v) : 0.0;
    }
}

// z-part of the least-squares multiplier right-hand side, zL - zU; `one` = 1 (Sigma = I)
__global__ void ls_rhs_kernel(int S, int64_t ld, const BView b, const double* __restrict__ zL,
                              const double* __restrict__ zU, double* __restrict__ rz, double* __restrict__ one) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (live_prob(b, s, S, PS_ACT) < 0) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        rz[o] = zL[o] - zU[o];
        one[o] = 1.0;
    }
}

// y = a x + c y over the per-scenario part; a = ps[afield][p] when afield >= 0.
// flag selects which problems take part (PS_ACT or PS_LSACT).  In place (x == y) is allowed.
__global__ void axpby_kernel(int S, int64_t ld, const BView b, int flag, int afield, double a, const double* xv,
                             double c, double* y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int pr = live_prob(b, s, S, flag);
    if (pr < 0) return;
    const double aa = afield >= 0 ? psv(b, afield, pr) : a;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        y[o] = c == 0.0 ? aa * xv[o] : aa * xv[o] + c * y[o];   // y is not read when c = 0
    }
}

// y1 += x1 (per-scenario part and the problems' design slots) and y2 += x2 (per-scenario
// part).  Elementwise.
__global__ void __launch_bounds__(128) axpy2_kernel(int S, int64_t ld, const BView b, const double* __restrict__ x1,
                                                    double* __restrict__ y1, const double* __restrict__ x2,
                                                    double* __restrict__ y2, int nsec = 1) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.y == 0 && s < b.NP && (!b.ps || psv(b, PS_ACT, s) != 0.0))
        for (int k = 0; k < nsec; ++k)
            y1[(int64_t)NSC * ld + (int64_t)k * b.NP + s] += x1[(int64_t)NSC * ld + (int64_t)k * b.NP + s];
    if (live_prob(b, s, S, PS_ACT) < 0) return;
    const int64_t o = (int64_t)blockIdx.y * ld + s;
    y1[o] += x1[o];
    y2[o] += x2[o];
}

__global__ void max_abs_kernel(int S, int64_t ld, const BView b, const double* __restrict__ v, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (live_prob(b, s, S, PS_ACT) < 0) return;
    double m[1] = {0.0};
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const double a = fabs(v[(int64_t)(NV * n + j) * ld + s]);
        m[0] = (a > m[0] || a != a) ? a : m[0];
    }
    store_partials<1>(m, part, ld, s, n);
}

// ---- reductions per problem ---------------------------------------------------------
// chunk c covers elements [i0, i1) of problem p (element i: stage i / S_p, slot off_p +
// i % S_p); one block per chunk, fixed-order tree; out[k * nchunk + c]
constexpr int RED_T = 128;                  // threads per chunk block
constexpr int RED_PER = 2;                  // elements per thread and plane
constexpr int RED_CHUNK = RED_T * RED_PER;  // elements per chunk
constexpr int RED_KMAX = 12;
constexpr int RED_TAIL = 8;                 // chunk rounds whose loads the last block issues together

__device__ inline double warp_red(int op, double a) {
    // xor tree: every lane ends with the same value (each pair is combined in both orders
    // by commutative operations), in a fixed order
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a = red_op(op, a, __shfl_xor_sync(0xffffffffu, a, o));
    return a;
}

// One block per chunk of a problem's (stage, slot) elements: every plane k < K reduced in
// a fixed order (RED_PER elements per thread, xor trees within warps, warps in order) into
// cout[k][c].  The problem's chunk block that finishes last (a per-problem arrival
// counter; no block waits for another) then combines the problem's chunk results, chunk c
// on lane (c - c0) % 32 in increasing c, then an xor tree, into out[k][p] (and hout[k][p]
// with hout[RED_KMAX][p] = dslots[p], when the host fetches them) and re-arms the
// counter.  Every combination order depends on the problem's own size only.  All of a
// thread's loads are issued before the first combination (one memory latency per block
// instead of one per plane).
template <int K>
__global__ void __launch_bounds__(RED_T) reduce_kernel(const double* __restrict__ part, int64_t ld,
                                                       const RedOps ops, const int* __restrict__ ch, int nchunk,
                                                       const int* __restrict__ pchunk, const double* __restrict__ ps,
                                                       int NP, int flag, double* cout, int* cnt,
                                                       double* __restrict__ out, double* __restrict__ hout,
                                                       const double* __restrict__ dslots) {
    static_assert(K >= 1 && K <= RED_KMAX, "planes per reduction");
    __shared__ double sm[RED_T / 32][K];
    __shared__ int last;
    const int c = blockIdx.x;
    const int p = ch[5 * c + 0], off = ch[5 * c + 1], Sp = ch[5 * c + 2], i0 = ch[5 * c + 3], i1 = ch[5 * c + 4];
    const bool live = !ps || ps[(int64_t)flag * NP + p] != 0.0;
    const int64_t plane = (int64_t)N_STAGES * ld;
    int64_t idx[RED_PER];
    bool ok[RED_PER];
#pragma unroll
    for (int t = 0; t < RED_PER; ++t) {
        const int i = i0 + (int)threadIdx.x + RED_T * t;
        ok[t] = live && i < i1;
        idx[t] = ok[t] ? (int64_t)(i / Sp) * ld + off + i % Sp : 0;
    }
    double v[K][RED_PER];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int t = 0; t < RED_PER; ++t) v[k][t] = ok[t] ? part[(int64_t)k * plane + idx[t]] : 0.0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        const int op = ops.op[k];
        double a = red_id(op);
#pragma unroll
        for (int t = 0; t < RED_PER; ++t)
            if (ok[t]) a = red_op(op, a, v[k][t]);
        a = warp_red(op, a);
        if (lane == 0) sm[warp][k] = a;
    }
    __syncthreads();
    if ((int)threadIdx.x < K) {
        const int k = threadIdx.x, op = ops.op[k];
        double a = red_id(op);
#pragma unroll
        for (int w = 0; w < RED_T / 32; ++w) a = red_op(op, a, sm[w][k]);
        cout[(int64_t)k * nchunk + c] = a;
    }
    const int c0 = pchunk[p], c1 = pchunk[p + 1];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&cnt[p], 1) == c1 - c0 - 1;
    __syncthreads();
    if (!last) return;
    if (threadIdx.x == 0) cnt[p] = 0;
    __threadfence();
    // the problem's chunk results: plane k on warp k % 4, chunk c0 + lane + 32 i on lane
    // `lane` in increasing i (L2 reads: other blocks wrote them).  The loads of RED_TAIL
    // rounds of all the warp's planes are issued before the first combination: one L2
    // latency per RED_TAIL rounds instead of one per round and plane
    constexpr int NW = RED_T / 32;
    constexpr int KW = (K + NW - 1) / NW;   // planes per warp
    int opk[KW];
    double acc[KW];
#pragma unroll
    for (int u = 0; u < KW; ++u) {
        const int k = warp + NW * u;
        opk[u] = k < K ? ops.op[k] : RSUM;
        acc[u] = red_id(opk[u]);
    }
    const int nc = c1 - c0;
    for (int base = 0; base < nc; base += 32 * RED_TAIL) {
        double t[KW][RED_TAIL];
#pragma unroll
        for (int u = 0; u < KW; ++u)
#pragma unroll
            for (int i = 0; i < RED_TAIL; ++i) {
                const int k = warp + NW * u, cc = base + lane + 32 * i;
                t[u][i] = (k < K && cc < nc) ? __ldcg(&cout[(int64_t)k * nchunk + c0 + cc]) : 0.0;
            }
#pragma unroll
        for (int u = 0; u < KW; ++u)
#pragma unroll
            for (int i = 0; i < RED_TAIL; ++i)
                if (base + lane + 32 * i < nc) acc[u] = red_op(opk[u], acc[u], t[u][i]);
    }
#pragma unroll
    for (int u = 0; u < KW; ++u) {
        const int k = warp + NW * u;
        if (k >= K) continue;   // warp-uniform
        const double a = warp_red(opk[u], acc[u]);
        if (lane == 0) {
            out[(int64_t)k * NP + p] = a;
            if (hout) hout[(int64_t)k * NP + p] = a;
        }
    }
    if (hout && dslots && threadIdx.x == 0) hout[(int64_t)RED_KMAX * NP + p] = dslots[p];
}

// dd_p = (r_d - (beta - dw qp)) / S_d from the Schur sums red[2][p], red[3][p]; into the
// problem's d slot of dz
__global__ void finalize_dd_kernel(int64_t ld, const BView b, const double* __restrict__ red, double* __restrict__ dz,
                                   int nsec = 1) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= b.NP || psv(b, PS_ACT, p) == 0.0) return;
    const double beta = red[2 * (int64_t)b.NP + p], qp = red[3 * (int64_t)b.NP + p];
    const double dw = psv(b, PS_DW, p);
    if (nsec == 1) {
        dz[(int64_t)NSC * ld + p] = (psv(b, PS_RD, p) - (beta - dw * qp)) / psv(b, PS_SD, p);
        return;
    }
    // two design entries: S_theta [dd0; dd1] = r_theta - (beta - dw qp), S_theta symmetric
    // positive definite (Algorithm IC), solved by its LDL^T
    const double beta1 = red[0 * (int64_t)b.NP + p], qp1 = red[1 * (int64_t)b.NP + p];
    const double r0 = psv(b, PS_RD, p) - (beta - dw * qp), r1 = psv(b, PS_RD1, p) - (beta1 - dw * qp1);
    const double s00 = psv(b, PS_SD, p), s01 = psv(b, PS_SD01, p), s11 = psv(b, PS_SD11, p);
    const double l = s01 / s00, e = s11 - l * s01;
    const double dd1 = (r1 - l * r0) / e;
    dz[(int64_t)NSC * ld + p] = (r0 - s01 * dd1) / s00;
    dz[(int64_t)NSC * ld + b.NP + p] = dd1;
}

}  // namespace absorber
