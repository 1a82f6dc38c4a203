// absorber_lib.cu -- C ABI (include/absorber.h) of the GB300 absorber design library:
// problem setup, the fused evaluation kernel, the block-LU / Schur-on-d KKT factor and
// solve, FP64 refinement, and the interior-point driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <initializer_list>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "absorber.h"
#include "kernels.cuh"
#include "kernels_warp.cuh"

using namespace absorber;

// ======================================================================================
// IPM vector kernels (one thread per (scenario, stage) unless noted)
// ======================================================================================
namespace absorber {

__device__ inline double lo_of(const Params& P, int j) { return j == LT ? P.T_lo / P.sT : 0.0; }
__device__ inline double hi_of(const Params& P, int j) { return P.T_hi / P.sT; }

// J^T lambda for the stage's unknowns, and the scalars of the optimality error.
// partials: [0] max |J^T l - zL + zU| (z part), [1] sum |lambda|, [2] sum |zL| + |zU|,
// [3] max and [4] min of the complementarity products over bounded unknowns,
// [5] sum of the hydraulic multipliers.
__global__ void __launch_bounds__(128) dual_kernel(const Params P, int S, int64_t ld, const double* __restrict__ jac,
                                                   const double* __restrict__ lam, const double* __restrict__ x,
                                                   const double* __restrict__ zL, const double* __restrict__ zU,
                                                   double* __restrict__ jtl, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double v[6] = {0.0, 0.0, 0.0, -INFINITY, INFINITY, 0.0};
    if (s < S) {
        double g[NV];
        jt_stage(ld, jac, lam, s, n, g);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            jtl[o] = g[j];
            const double zl = zL[o], zu = zU[o];
            const double r = fabs(g[j] - zl + zu);
            v[0] = (r > v[0] || r != r) ? r : v[0];
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
        v[5] = lam[(int64_t)(NR * n + R_H) * ld + s];
    }
    const int ops[6] = {RMAX, RSUM, RSUM, RMAX, RMIN, RSUM};
    block_reduce_store<6>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// barrier diagonal Sigma, right-hand sides r_z = -(J^T l - mu/sl + mu/su), r_c = -c
__global__ void __launch_bounds__(128) rhs_kernel(const Params P, int S, int64_t ld, double mu,
                                                  const double* __restrict__ x, const double* __restrict__ zL,
                                                  const double* __restrict__ zU, const double* __restrict__ jtl,
                                                  const double* __restrict__ c, double* __restrict__ sig,
                                                  double* __restrict__ rz, double* __restrict__ rc) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        const double xv = x[o];
        double sg = 0.0, gb = 0.0;
        if (has_lo(j)) {
            const double sl = xv - lo_of(P, j);
            sg += zL[o] / sl;
            gb -= mu / sl;
        }
        if (has_hi(j)) {
            const double su = hi_of(P, j) - xv;
            sg += zU[o] / su;
            gb += mu / su;
        }
        sig[o] = sg;
        rz[o] = -(jtl[o] + gb);
        rc[o] = -c[o];
    }
}

// Schur-complement partial sums for the stage: with H = W + Sigma (W optional),
// [0] q^T H q, [1] q^T q, [2] q^T (r - H p), [3] q^T p, [4] the d-d Hessian entries.
__global__ void __launch_bounds__(128) schur_kernel(int S, int64_t ld, const double* __restrict__ hes,
                                                    const double* __restrict__ sig, bool use_w,
                                                    const double* __restrict__ p, const double* __restrict__ q,
                                                    const double* __restrict__ r, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (s < S) {
        double hq[NV];
        hv_stage(ld, hes, sig, 0.0, use_w, q, s, n, hq);
        double hp[NV];
        if (p) hv_stage(ld, hes, sig, 0.0, use_w, p, s, n, hp);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double qj = q[o];
            v[0] += qj * hq[j];
            v[1] += qj * qj;
            if (r) v[2] += qj * (r[o] - (p ? hp[j] : 0.0));
            if (p) v[3] += qj * p[o];
        }
        if (use_w && n == 0) v[4] = hes[(int64_t)(NHS * N_STAGES) * ld + s];
    }
    const int ops[5] = {RSUM, RSUM, RSUM, RSUM, RSUM};
    block_reduce_store<5>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// dz = p - q dd ;  g = r - (W + Sigma + dw I) dz ;  dd is read from ddp (the d slot of dz)
__global__ void __launch_bounds__(128) dz_kernel(int S, int64_t ld, const double* __restrict__ hes,
                                                 const double* __restrict__ sig, double dw, bool use_w,
                                                 const double* __restrict__ p, const double* __restrict__ q,
                                                 const double* ddp, const double* __restrict__ r, double* dz,
                                                 double* __restrict__ g) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
    const double dd = *ddp;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        dz[o] = p[o] - q[o] * dd;
    }
    double h[NV];
    hv_stage(ld, hes, sig, dw, use_w, dz, s, n, h);
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        g[o] = r[o] - h[j];
    }
}

// residual of the full KKT system for the stage:  rho_z = r_z - (H dz + J^T dl),
// rho_c = r_c - (J dz + b dd).  partials: [0] max|rho_z|, [1] max|rho_c|,
// [2] sum of the hydraulic dl, [3] max|r_z|, [4] max|r_c|.
__global__ void __launch_bounds__(128) kkt_residual_kernel(int S, int64_t ld, const double* __restrict__ jac,
                                                           const double* __restrict__ hes, const double* __restrict__ sig,
                                                           double dw, bool use_w, const double* __restrict__ dz,
                                                           const double* __restrict__ ddp, const double* __restrict__ dl,
                                                           const double* __restrict__ rz, const double* __restrict__ rc,
                                                           double* __restrict__ rhoz, double* __restrict__ rhoc,
                                                           double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    if (s < S) {
        const double dd = *ddp;
        double h[NV], jt[NV], jv[NR];
        hv_stage(ld, hes, sig, dw, use_w, dz, s, n, h);
        jt_stage(ld, jac, dl, s, n, jt);
        jv_stage(ld, jac, dz, dd, s, n, jv);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double a = rz[o] - (h[j] + jt[j]);
            const double b = rc[o] - jv[j];
            rhoz[o] = a;
            rhoc[o] = b;
            v[0] = fmax(v[0], fabs(a));
            v[1] = fmax(v[1], fabs(b));
            v[3] = fmax(v[3], fabs(rz[o]));
            v[4] = fmax(v[4], fabs(rc[o]));
            if (a != a || b != b) v[0] = NAN;
        }
        v[2] = dl[(int64_t)(NR * n + R_H) * ld + s];
    }
    const int ops[5] = {RMAX, RMAX, RSUM, RMAX, RMAX};
    block_reduce_store<5>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// bound-multiplier steps and step-size limits.  partials: [0] min primal ratio (alpha_max),
// [1] min dual ratio (alpha_z), [2] sum of barrier-gradient . dz, [3] max |dz|/(1+|z|).
__global__ void __launch_bounds__(128) step_kernel(const Params P, int S, int64_t ld, double mu, double tau,
                                                   const double* __restrict__ x, const double* __restrict__ dz,
                                                   const double* __restrict__ zL, const double* __restrict__ zU,
                                                   double* __restrict__ dzL, double* __restrict__ dzU, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double v[4] = {1.0, 1.0, 0.0, 0.0};
    if (s < S) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double xv = x[o], d = dz[o];
            v[3] = fmax(v[3], fabs(d) / (1.0 + fabs(xv)));
            if (d != d) v[3] = NAN;
            if (has_lo(j)) {
                const double sl = xv - lo_of(P, j);
                const double z = zL[o];
                const double dzl = mu / sl - z - (z / sl) * d;
                dzL[o] = dzl;
                if (d < 0.0) v[0] = fmin(v[0], -tau * sl / d);
                if (dzl < 0.0) v[1] = fmin(v[1], -tau * z / dzl);
                v[2] += (-mu / sl) * d;
            } else {
                dzL[o] = 0.0;
            }
            if (has_hi(j)) {
                const double su = hi_of(P, j) - xv;
                const double z = zU[o];
                const double dzu = mu / su - z + (z / su) * d;
                dzU[o] = dzu;
                if (d > 0.0) v[0] = fmin(v[0], tau * su / d);
                if (dzu < 0.0) v[1] = fmin(v[1], -tau * z / dzu);
                v[2] += (mu / su) * d;
            } else {
                dzU[o] = 0.0;
            }
        }
    }
    const int ops[4] = {RMIN, RMIN, RSUM, RMAX};
    block_reduce_store<4>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// accept the step and apply the kappa_Sigma safeguard to the bound multipliers
__global__ void __launch_bounds__(128) accept_kernel(const Params P, int S, int64_t ld, double alpha, double alpha_z,
                                                     double mu, double ksig, double d_new, double* __restrict__ x,
                                                     const double* __restrict__ dz, double* __restrict__ lam,
                                                     const double* __restrict__ dl, double* __restrict__ zL,
                                                     const double* __restrict__ dzL, double* __restrict__ zU,
                                                     const double* __restrict__ dzU) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
    if (s == 0 && n == 0) x[(int64_t)NSC * ld] = d_new;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        const double xv = x[o] + alpha * dz[o];
        x[o] = xv;
        lam[o] += alpha * dl[o];
        if (has_lo(j)) {
            const double sl = xv - lo_of(P, j);
            const double z = zL[o] + alpha_z * dzL[o];
            zL[o] = fmin(fmax(z, mu / (ksig * sl)), ksig * mu / sl);
        }
        if (has_hi(j)) {
            const double su = hi_of(P, j) - xv;
            const double z = zU[o] + alpha_z * dzU[o];
            zU[o] = fmin(fmax(z, mu / (ksig * su)), ksig * mu / su);
        }
    }
}

// default starting point (every stage copies the inlet streams, T the mean inlet
// temperature, eps = 0, the slack from the hydraulic row at d), pushed into the bounds
// (base != null: stage states from the expected-value solution, entry v at base[v * ldb])
__global__ void __launch_bounds__(128) init_kernel(const Params P, int S, int64_t ld, const double* __restrict__ feed,
                                                   const double* __restrict__ base, int64_t ldb, double d, double push,
                                                   double frac, double* __restrict__ x, double* __restrict__ zL,
                                                   double* __restrict__ zU, double* __restrict__ lam) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
    double q[NV];
    if (base) {
#pragma unroll
        for (int j = 0; j < NV; ++j) q[j] = base[(int64_t)(NV * n + j) * ldb];
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
    q[LS] = P.u_max * M_PI * d * d * 0.25 - q[LV] * P.R * (P.sT * q[LT]) / feed[(int64_t)F_P * ld + s];
    if (s == 0 && n == 0) x[(int64_t)NSC * ld] = d;
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

// z-part of the least-squares multiplier right-hand side: -(grad f - zL + zU) = zL - zU
__global__ void ls_rhs_kernel(int S, int64_t ld, const double* __restrict__ zL, const double* __restrict__ zU,
                              double* __restrict__ rz, double* __restrict__ one) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        rz[o] = zL[o] - zU[o];
        one[o] = 1.0;
    }
}

// primal fraction-to-the-boundary limit of a direction: partial [0] = min ratio
__global__ void __launch_bounds__(128) ftb_kernel(const Params P, int S, int64_t ld, double tau,
                                                  const double* __restrict__ x, const double* __restrict__ dz,
                                                  double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double v[1] = {1.0};
    if (s < S) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NV * n + j) * ld + s;
            const double xv = x[o], d = dz[o];
            if (has_lo(j) && d < 0.0) v[0] = fmin(v[0], -tau * (xv - lo_of(P, j)) / d);
            if (has_hi(j) && d > 0.0) v[0] = fmin(v[0], tau * (hi_of(P, j) - xv) / d);
            if (d != d) v[0] = NAN;
        }
    }
    const int ops[1] = {RMIN};
    block_reduce_store<1>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

// y = a * x + b * y on the per-scenario part of row/primal vectors
__global__ void axpby_kernel(int S, int64_t ld, double a, const double* xv, double b, double* y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        y[o] = a * xv[o] + b * y[o];
    }
}

// dd = (rd - (sum_b part[2][b] - dw sum_b part[3][b])) / Sd  (one block, fixed-order tree)
__global__ void __launch_bounds__(256) finalize_dd_kernel(const double* __restrict__ part, int nb, double rd, double dw,
                                                          double Sd, double* out) {
    __shared__ double s2[256], s3[256];
    double a2 = 0.0, a3 = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        a2 += part[2 * (int64_t)nb + b];
        a3 += part[3 * (int64_t)nb + b];
    }
    s2[threadIdx.x] = a2;
    s3[threadIdx.x] = a3;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            s2[threadIdx.x] += s2[threadIdx.x + o];
            s3[threadIdx.x] += s3[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (rd - (s2[0] - dw * s3[0])) / Sd;
}

// y += x on the per-scenario part and on the d slot of primal vectors (d_slot true)
__global__ void axpy_d_kernel(int S, int64_t ld, const double* __restrict__ xv, double* __restrict__ y, bool d_slot) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        y[o] += xv[o];
    }
    if (d_slot && s == 0 && n == 0) y[(int64_t)NSC * ld] += xv[(int64_t)NSC * ld];
}

__global__ void max_abs_kernel(int S, int64_t ld, const double* __restrict__ v, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    double m[1] = {0.0};
    if (s < S) {
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const double a = fabs(v[(int64_t)(NV * n + j) * ld + s]);
            m[0] = (a > m[0] || a != a) ? a : m[0];
        }
    }
    const int ops[1] = {RMAX};
    block_reduce_store<1>(m, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
}

__global__ void axpy_kernel(int S, int64_t ld, double a, const double* __restrict__ xv, double* __restrict__ y) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t o = (int64_t)(NV * n + j) * ld + s;
        y[o] += a * xv[o];
    }
}


}  // namespace absorber

// ======================================================================================
// host side
// ======================================================================================
namespace {

const int kThr = 128;     // threads per block of the (scenario, stage) kernels
const int kThrS = 64;     // threads per block of the per-scenario kernels

thread_local std::string g_err = "no error";

struct PatternTables {
    short slotJ[3][NR][NLOC];
    int segJ[N_STAGES + 1];
    short slotH[NV][NV];
    Ent own[3][MAXOWN], abv[3][MAXABV], blw[3][MAXBLW], hes[NHS];
    int nown[3], nabv[3], nblw[3], dslot[3];
    std::vector<int> jrow, jcol, hrow, hcol;
    bool ok = false;
};

struct Recorder {
    static constexpr bool want_res = false, want_jac = true, want_hes = true;
    std::vector<std::pair<int, int>> J, H;
    void res(int, double) {}
    void jac(int r, int lv, double) { J.push_back({r, lv}); }
    void hes(int i, int j, double) { H.push_back({i, j}); }
};

int local_col(int lv, int n) {
    if (lv < NV) return NV * n + lv;
    if (lv < BY) return NV * (n + 1) + abv_var(lv - AX);
    if (lv < LD_) return NV * (n - 1) + blw_var(lv - BY);
    return NSC;  // d
}

Params dummy_params() {
    Params P;
    std::memset(&P, 0, sizeof(P));
    P.R = 0.08;
    P.u_max = 2.0;
    P.T_lo = 273.0;
    P.T_hi = 400.0;
    P.T_ref = 298.0;
    for (int l = 0; l < 9; ++l) P.sx[l] = 1.0;
    for (int j = 0; j < 4; ++j) P.sy[j] = 1.0;
    P.sT = 100.0;
    P.psat_a = 10.0;
    P.psat_b = 100.0;
    P.psat_c = 10.0;
    P.rho_L = 1.0;
    P.henry_m = 1.0;
    P.henry_w = 1.0;
    return P;
}

// Build the per-scenario CSR patterns and the per-stage-type slot tables by running the
// stage routine with a recording emitter for the three stage types.
bool build_pattern(PatternTables& T, std::string& err) {
    const Params P = dummy_params();
    Recorder rec[3];
    for (int t = 0; t < 3; ++t) {
        StageIn in;
        for (int j = 0; j < NV; ++j) in.q[j] = 1.0;
        for (int a = 0; a < 11; ++a) in.qa[a] = 1.0;
        for (int b = 0; b < 6; ++b) in.qb[b] = 1.0;
        in.d = 1.0;
        in.P = 1.0;
        in.has_below = t != 0;
        in.has_above = t != 2;
        StageLam L;
        for (int r = 0; r < NR; ++r) L.own[r] = 1.0;
        for (int k = 0; k < 10; ++k) L.below[k] = 1.0;
        for (int k = 0; k < 5; ++k) L.above[k] = 1.0;
        stage_eval(P, in, &L, rec[t]);
    }
    // Jacobian: collect (row, col, stage, r, lv), sort in CSR order
    struct E {
        int row, col, n, r, lv;
    };
    std::vector<E> all;
    for (int n = 0; n < N_STAGES; ++n) {
        const int t = stage_type(n);
        for (auto& p : rec[t].J) all.push_back({NR * n + p.first, local_col(p.second, n), n, p.first, p.second});
    }
    std::sort(all.begin(), all.end(), [](const E& a, const E& b) {
        return a.row != b.row ? a.row < b.row : a.col < b.col;
    });
    for (size_t k = 1; k < all.size(); ++k)
        if (all[k].row == all[k - 1].row && all[k].col == all[k - 1].col) {
            err = "duplicate Jacobian entry in the stage routine";
            return false;
        }
    for (int t = 0; t < 3; ++t)
        for (int r = 0; r < NR; ++r)
            for (int l = 0; l < NLOC; ++l) T.slotJ[t][r][l] = -1;
    int next_stage = 0;
    for (size_t k = 0; k < all.size(); ++k) {
        while (next_stage <= all[k].n) T.segJ[next_stage++] = (int)k;
    }
    T.segJ[N_STAGES] = (int)all.size();
    for (int t = 0; t < 3; ++t) T.nown[t] = T.nabv[t] = T.nblw[t] = 0;
    for (size_t k = 0; k < all.size(); ++k) {
        const E& e = all[k];
        const int t = stage_type(e.n);
        const int slot = (int)k - T.segJ[e.n];
        short& sl = T.slotJ[t][e.r][e.lv];
        if (sl == -1) {
            sl = (short)slot;
            Ent en;
            en.slot = (short)slot;
            en.r = (signed char)e.r;
            if (e.lv < NV) {
                en.c = (signed char)e.lv;
                if (T.nown[t] >= MAXOWN) { err = "own table overflow"; return false; }
                T.own[t][T.nown[t]++] = en;
            } else if (e.lv < BY) {
                en.c = (signed char)(e.lv - AX);
                if (T.nabv[t] >= MAXABV) { err = "above table overflow"; return false; }
                T.abv[t][T.nabv[t]++] = en;
            } else if (e.lv < LD_) {
                en.c = (signed char)(e.lv - BY);
                if (T.nblw[t] >= MAXBLW) { err = "below table overflow"; return false; }
                T.blw[t][T.nblw[t]++] = en;
            } else {
                T.dslot[t] = slot;
            }
        } else if (sl != slot) {
            err = "stage segments of one type differ";
            return false;
        }
    }
    T.jrow.resize(all.size());
    T.jcol.resize(all.size());
    // per-scenario pattern: stage segments are the same for all scenarios
    for (size_t k = 0; k < all.size(); ++k) {
        T.jrow[k] = all[k].row;
        T.jcol[k] = all[k].col;
    }
    // Hessian (same entries on every stage type)
    std::vector<std::pair<int, int>> H = rec[1].H;
    std::sort(H.begin(), H.end());
    for (int t = 0; t < 3; ++t) {
        auto h2 = rec[t].H;
        std::sort(h2.begin(), h2.end());
        if (h2 != H) {
            err = "Hessian pattern differs by stage type";
            return false;
        }
    }
    if ((int)H.size() != NHS) {
        err = "unexpected Hessian block size";
        return false;
    }
    for (int i = 0; i < NV; ++i)
        for (int j = 0; j < NV; ++j) T.slotH[i][j] = -1;
    for (int k = 0; k < NHS; ++k) {
        if (H[k].first < H[k].second) {
            err = "upper-triangle Hessian entry";
            return false;
        }
        T.slotH[H[k].first][H[k].second] = (short)k;
        T.hes[k].slot = (short)k;
        T.hes[k].r = (signed char)H[k].first;
        T.hes[k].c = (signed char)H[k].second;
    }
    for (int n = 0; n < N_STAGES; ++n)
        for (int k = 0; k < NHS; ++k) {
            T.hrow.push_back(NV * n + H[k].first);
            T.hcol.push_back(NV * n + H[k].second);
        }
    T.hrow.push_back(NSC);
    T.hcol.push_back(NSC);
    T.ok = true;
    return true;
}

PatternTables& pattern() {
    static PatternTables T;
    static bool tried = false;
    static std::string err;
    if (!tried) {
        tried = true;
        build_pattern(T, err);
        if (!T.ok) std::fprintf(stderr, "absorber: pattern construction failed: %s\n", err.c_str());
    }
    return T;
}

bool g_uploaded[64] = {false};

cudaError_t upload_tables(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_uploaded[dev]) return cudaSuccess;
    PatternTables& T = pattern();
    cudaError_t e;
#define UP(sym, src) \
    if ((e = cudaMemcpyToSymbol(sym, &(src), sizeof(src))) != cudaSuccess) return e;
    UP(c_slotJ, T.slotJ);
    UP(c_segJ, T.segJ);
    UP(c_slotH, T.slotH);
    UP(c_own, T.own);
    UP(c_abv, T.abv);
    UP(c_blw, T.blw);
    UP(c_hes, T.hes);
    UP(c_nown, T.nown);
    UP(c_nabv, T.nabv);
    UP(c_nblw, T.nblw);
    UP(c_dslot, T.dslot);
#undef UP
    g_uploaded[dev] = true;
    return cudaSuccess;
}

}  // namespace

struct abs_problem {
    int dev = 0;
    int64_t S = 0, ld = 0;
    Params P;
    std::vector<double> prob;
    std::string err = "no error";
    int nnzJ = 0, nnzH = 0;
    double* feed = nullptr;          // [18][ld]
    // evaluation / KKT buffers (lazily allocated)
    double* jac = nullptr;           // nnzJ * ld
    double* hes = nullptr;           // nnzH * ld
    double* vec = nullptr;           // pool of primal-size vectors
    int nvec = 0;
    void* LU = nullptr;              // factors of the current precision (points at one of below)
    void* G = nullptr;
    void* LUp[2] = {nullptr, nullptr};   // [ABS_PREC_FP64], [ABS_PREC_FP32]
    void* Gp[2] = {nullptr, nullptr};
    unsigned char* piv = nullptr;
    int* sing = nullptr;
    int* count = nullptr;
    int fac_prec = -1;
    double* part = nullptr;          // partial reductions
    double* hpart = nullptr;         // pinned copy
    int nblk2 = 0;                   // blocks of a (scenario, stage) launch
    // factorization state kept for kkt_solve
    struct {
        bool valid = false;
        int prec = 0;
        const double* jac = nullptr;
        const double* hes = nullptr;
        const double* sig = nullptr;
        double d = 0.0, dw = 0.0, Kdd = 0.0, A0 = 0.0, Q2 = 0.0, Sd = 0.0;
        bool use_w = true;
    } fac;
    // kernel profiler (options.profile): event pairs per hot-kernel launch
    struct Prof {
        bool on = false;
        cudaStream_t st = nullptr;
        std::vector<cudaEvent_t> pool;
        std::vector<std::pair<int, size_t>> marks;   // (kernel id, index of its start event)
        size_t used = 0;
    } prof;
    int64_t nlaunch = 0;   // kernels launched (every launch is followed by launch_check)
    abs_params aparams;              // the caller's table (for the expected-value sub-problem)
    std::vector<double> hfeed;       // host copy of the feeds [18][S]
    abs_problem* base = nullptr;     // one-scenario sub-problem for the expected-value start
};

namespace {

// vector pool indices (each NSC * ld + ld doubles, the d slot at NSC * ld)
enum {
    V_X, V_LAM, V_ZL, V_ZU, V_C, V_JTL, V_SIG, V_RZ, V_RC, V_P, V_Q, V_DZ, V_DL, V_DZL, V_DZU,
    V_G, V_RHOZ, V_RHOC, V_P2, V_CZ, V_CL, V_ONE, V_CT, V_RCS, V_SZ, V_SL, V_COUNT
};

abs_status fail(abs_problem* h, abs_status st, const std::string& msg) {
    if (h) h->err = msg;
    g_err = msg;
    return st;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(h, e_ == cudaErrorMemoryAllocation ? ABS_ERR_OOM : ABS_ERR_CUDA, \
                        std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

int64_t vsize(const abs_problem* h) { return (int64_t)NSC * h->ld + h->ld; }
double* V(abs_problem* h, int k) { return h->vec + (int64_t)k * vsize(h); }
dim3 grid2(const abs_problem* h) { return dim3((unsigned)((h->S + kThr - 1) / kThr), N_STAGES); }

abs_status ensure_buffers(abs_problem* h) {
    if (h->vec) return ABS_OK;
    const int64_t ld = h->ld;
    CK(cudaMalloc(&h->jac, sizeof(double) * (size_t)h->nnzJ * ld));
    CK(cudaMalloc(&h->hes, sizeof(double) * (size_t)h->nnzH * ld));
    h->nvec = V_COUNT;
    CK(cudaMalloc(&h->vec, sizeof(double) * (size_t)vsize(h) * h->nvec));
    CK(cudaMemset(h->vec, 0, sizeof(double) * (size_t)vsize(h) * h->nvec));
    CK(cudaMalloc(&h->piv, (size_t)N_STAGES * NV * ld));
    CK(cudaMalloc(&h->sing, sizeof(int) * (size_t)ld));
    CK(cudaMalloc(&h->count, sizeof(int)));
    h->nblk2 = (int)(((h->S + kThr - 1) / kThr) * N_STAGES);
    const size_t np = (size_t)16 * h->nblk2 + 64;
    CK(cudaMalloc(&h->part, sizeof(double) * np));
    CK(cudaMallocHost(&h->hpart, sizeof(double) * np));
    return ABS_OK;
}

abs_status ensure_factor(abs_problem* h, int prec) {
    if (!h->LUp[prec]) {
        const size_t es = prec == ABS_PREC_FP32 ? sizeof(float) : sizeof(double);
        CK(cudaMalloc(&h->LUp[prec], es * (size_t)N_STAGES * NV * NV * h->ld));
        CK(cudaMalloc(&h->Gp[prec], es * (size_t)N_STAGES * NV * NABV * h->ld));
    }
    h->LU = h->LUp[prec];
    h->G = h->Gp[prec];
    h->fac_prec = prec;
    return ABS_OK;
}

// reduce K partial arrays written by a (scenario, stage) launch, in fixed order on the
// host; the device scalars in `extra` (doubles) and `icount` (an int) are fetched in the
// same round trip through the pinned tail of hpart
abs_status fetch_partials(abs_problem* h, cudaStream_t st, int K, const int* ops, double* out,
                          std::initializer_list<const double*> extra = {}, double* extra_out = nullptr,
                          const int* icount = nullptr, int* icount_out = nullptr) {
    const int nb = h->nblk2;
    double* tail = h->hpart + (size_t)16 * nb;
    if (K > 0) CK(cudaMemcpyAsync(h->hpart, h->part, sizeof(double) * (size_t)K * nb, cudaMemcpyDeviceToHost, st));
    int i = 0;
    for (const double* e : extra) CK(cudaMemcpyAsync(tail + i++, e, sizeof(double), cudaMemcpyDeviceToHost, st));
    if (icount) CK(cudaMemcpyAsync((int*)(tail + 60), icount, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int k = 0; k < i; ++k) extra_out[k] = tail[k];
    if (icount) *icount_out = *(int*)(tail + 60);
    for (int k = 0; k < K; ++k) {
        double a = ops[k] == RSUM ? 0.0 : (ops[k] == RMAX ? -INFINITY : INFINITY);
        const double* p = h->hpart + (size_t)k * nb;
        for (int b = 0; b < nb; ++b) {
            const double v = p[b];
            if (ops[k] == RSUM) a += v;
            else if (ops[k] == RMAX) a = (v > a || v != v) ? v : a;
            else a = (v < a || v != v) ? v : a;
        }
        out[k] = a;
    }
    return ABS_OK;
}

enum { K_EVAL = 0, K_EVAL_TRIAL = 1, K_FACTOR = 2, K_SOLVE = 3, K_SOLVE_T = 4 };

cudaEvent_t prof_event(abs_problem* h) {
    auto& p = h->prof;
    if (p.used == p.pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        p.pool.push_back(e);
    }
    return p.pool[p.used++];
}

// record the start of a hot-kernel launch on stream st (no-op unless profiling)
void prof_begin(abs_problem* h, int kid, cudaStream_t st) {
    if (!h->prof.on) return;
    h->prof.marks.push_back({kid, h->prof.used});
    cudaEventRecord(prof_event(h), st);
}

void prof_end(abs_problem* h, cudaStream_t st) {
    if (!h->prof.on) return;
    cudaEventRecord(prof_event(h), st);
}

abs_status launch_check(abs_problem* h) {
    if (h) h->nlaunch++;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, ABS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ABS_OK;
}

// ---- the KKT machinery ---------------------------------------------------------------
struct KKTSys {
    const double* jac;
    const double* hes;
    const double* sig;
    bool use_w;
    double dw;
    double d;        // current diameter (for b = dc/dd)
    double Kdd;      // W_dd + Sigma_d (without dw)
    double A0, Q2;   // sum q^T (W + Sigma) q, sum q^T q
    double Sd;       // Schur complement with dw
    int prec;
};

dim3 gridw(const abs_problem* h, int wpb) { return dim3((unsigned)((h->S + wpb - 1) / wpb)); }

template <class T>
abs_status factor_launch(abs_problem* h, const double* jac, double pivtol, cudaStream_t st) {
    prof_begin(h, K_FACTOR, st);
    factor_warp_kernel<T><<<gridw(h, WPB_F), 32 * WPB_F, 0, st>>>((int)h->S, h->ld, jac, (T*)h->LU, h->piv, (T*)h->G,
                                                                h->sing, h->count, pivtol);
    prof_end(h, st);
    return launch_check(h);
}

template <class T, int NR_>
abs_status solve_launch(abs_problem* h, const double* jac, const double* xd, const double* r0, const double* r1,
                        double* o0, double* o1, cudaStream_t st) {
    prof_begin(h, K_SOLVE, st);
    solve_warp_kernel<T, NR_><<<gridw(h, WPB_S), 32 * WPB_S, 0, st>>>(h->P, (int)h->S, h->ld, jac, (const T*)h->LU,
                                                                       h->piv, (const T*)h->G, xd, r0, r1, o0, o1);
    prof_end(h, st);
    return launch_check(h);
}

abs_status solve_j(abs_problem* h, int prec, const double* jac, const double* xd, const double* r0,
                   const double* r1, double* o0, double* o1, cudaStream_t st) {
    if (prec == ABS_PREC_FP32) {
        if (o1) return solve_launch<float, 2>(h, jac, xd, r0, r1, o0, o1, st);
        return solve_launch<float, 1>(h, jac, xd, r0, nullptr, o0, nullptr, st);
    }
    if (o1) return solve_launch<double, 2>(h, jac, xd, r0, r1, o0, o1, st);
    return solve_launch<double, 1>(h, jac, xd, r0, nullptr, o0, nullptr, st);
}

abs_status solve_jt(abs_problem* h, int prec, const double* jac, const double* g, double* out, cudaStream_t st) {
    prof_begin(h, K_SOLVE_T, st);
    struct End {
        abs_problem* h;
        cudaStream_t st;
        ~End() { prof_end(h, st); }
    } end{h, st};
    if (prec == ABS_PREC_FP32)
        solve_t_warp_kernel<float><<<gridw(h, WPB_S), 32 * WPB_S, 0, st>>>((int)h->S, h->ld, jac, (const float*)h->LU,
                                                                            h->piv, g, out);
    else
        solve_t_warp_kernel<double><<<gridw(h, WPB_S), 32 * WPB_S, 0, st>>>((int)h->S, h->ld, jac,
                                                                             (const double*)h->LU, h->piv, g, out);
    return launch_check(h);
}

// factor J_s (all scenarios), q = J^-1 b, and the Schur sums A0, Q2, (W_dd sum).
// Returns the number of scenarios with a singular stage block in *nsing.
abs_status kkt_factor_core(abs_problem* h, KKTSys& K, const double* xd, int64_t* nsing, double* wdd,
                           cudaStream_t st) {
    abs_status r;
    if ((r = ensure_factor(h, K.prec)) != ABS_OK) return r;
    CK(cudaMemsetAsync(h->count, 0, sizeof(int), st));
    // FP64: a pivot below 1e-14 of the block's largest entry marks the stage block
    // singular; FP32: only (numerically) zero pivots do -- accuracy is guarded by the FP64
    // refinement instead, with an FP64 refactorization when it stalls
    const double pivtol = K.prec == ABS_PREC_FP32 ? 1e-30 : 1e-14;
    if (K.prec == ABS_PREC_FP32) r = factor_launch<float>(h, K.jac, pivtol, st);
    else r = factor_launch<double>(h, K.jac, pivtol, st);
    if (r != ABS_OK) return r;
    if ((r = solve_j(h, K.prec, K.jac, xd, nullptr, nullptr, V(h, V_Q), nullptr, st)) != ABS_OK) return r;
    schur_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, K.hes, K.sig, K.use_w, nullptr, V(h, V_Q), nullptr,
                                             h->part);
    if ((r = launch_check(h)) != ABS_OK) return r;
    int cnt = 0;
    const int ops[5] = {RSUM, RSUM, RSUM, RSUM, RSUM};
    double red[5];
    if ((r = fetch_partials(h, st, 5, ops, red, {}, nullptr, h->count, &cnt)) != ABS_OK) return r;
    K.A0 = red[0];
    K.Q2 = red[1];
    if (wdd) *wdd = red[4];
    *nsing = cnt;
    return ABS_OK;
}

double schur_value(const KKTSys& K, double dw) { return K.Kdd + dw + K.A0 + dw * K.Q2; }

// one Schur-reduced solve:  given rz (z part), rd, rc  ->  dz (primal, d slot set), dl.
// uses V_P, V_G as scratch.
abs_status kkt_solve_once(abs_problem* h, const KKTSys& K, const double* xd, const double* rz, double rd,
                          const double* rc, double* dz, double* dl, cudaStream_t st) {
    abs_status r;
    if ((r = solve_j(h, K.prec, K.jac, xd, rc, nullptr, V(h, V_P), nullptr, st)) != ABS_OK) return r;
    schur_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, K.hes, K.sig, K.use_w, V(h, V_P), V(h, V_Q), rz,
                                             h->part);
    if ((r = launch_check(h)) != ABS_OK) return r;
    // dd = (rd - beta) / S_d on the device, into the d slot of dz: no host round trip
    double* ddp = dz + (int64_t)NSC * h->ld;
    finalize_dd_kernel<<<1, 256, 0, st>>>(h->part, h->nblk2, rd, K.dw, K.Sd, ddp);
    if ((r = launch_check(h)) != ABS_OK) return r;
    dz_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, K.hes, K.sig, K.dw, K.use_w, V(h, V_P), V(h, V_Q), ddp, rz,
                                          dz, V(h, V_G));
    if ((r = launch_check(h)) != ABS_OK) return r;
    if ((r = solve_jt(h, K.prec, K.jac, V(h, V_G), dl, st)) != ABS_OK) return r;
    return ABS_OK;
}

// Solve with FP64 iterative refinement on the full KKT residual.
abs_status kkt_solve_refined(abs_problem* h, const KKTSys& K, const double* xd, const double* rz, double rd,
                             const double* rc, double* dz, double* dl, int max_refine, double tol, int* steps,
                             double* resid, cudaStream_t st) {
    abs_status r;
    if ((r = kkt_solve_once(h, K, xd, rz, rd, rc, dz, dl, st)) != ABS_OK) return r;
    int k = 0;
    double sc = 0.0;
    double* ddp = dz + (int64_t)NSC * h->ld;
    for (;;) {
        if (max_refine == 0 && !resid) break;   // nothing to refine and no residual asked for
        kkt_residual_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, K.jac, K.hes, K.sig, K.dw, K.use_w, dz, ddp,
                                                        dl, rz, rc, V(h, V_RHOZ), V(h, V_RHOC), h->part);
        if ((r = launch_check(h)) != ABS_OK) return r;
        const int ops[5] = {RMAX, RMAX, RSUM, RMAX, RMAX};
        double red[5], dd = 0.0;
        if ((r = fetch_partials(h, st, 5, ops, red, {ddp}, &dd)) != ABS_OK) return r;
        const double b = -h->P.u_max * M_PI * 0.5 * K.d;
        const double rhod = rd - ((K.Kdd + K.dw) * dd + b * red[2]);
        const double rn = std::max(std::max(red[0], red[1]), std::fabs(rhod));
        const double bn = std::max(std::max(red[3], red[4]), std::fabs(rd));
        sc = rn / (bn + 1e-300);
        if (!(sc == sc)) return fail(h, ABS_ERR_NUMERIC, "NaN in the KKT solve");
        if (sc <= tol || k >= max_refine) break;
        // correction, then add it (including the d slot) to the solution
        if ((r = kkt_solve_once(h, K, xd, V(h, V_RHOZ), rhod, V(h, V_RHOC), V(h, V_CZ), V(h, V_CL), st)) != ABS_OK)
            return r;
        axpy_d_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, V(h, V_CZ), dz, true);
        if ((r = launch_check(h)) != ABS_OK) return r;
        axpy_d_kernel<<<grid2(h), kThr, 0, st>>>((int)h->S, h->ld, V(h, V_CL), dl, false);
        if ((r = launch_check(h)) != ABS_OK) return r;
        ++k;
    }
    if (steps) *steps = k;
    if (resid) *resid = sc;
    return ABS_OK;
}

// feeds: host or device, [18][S] -> device [18][ld]; padding columns copy the last
// scenario so that every padded lane evaluates a valid (ignored) problem
__global__ void pad_feed_kernel(int S, int64_t ld, const double* __restrict__ src, double* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)NFEED * ld) return;
    const int64_t f = i / ld, s = i % ld;
    dst[i] = src[f * S + (s < S ? s : S - 1)];
}

abs_status upload_feeds(abs_problem* h, const double* feeds, cudaStream_t st) {
    const int64_t S = h->S, ld = h->ld;
    cudaPointerAttributes attr;
    const bool on_dev = cudaPointerGetAttributes(&attr, feeds) == cudaSuccess &&
                        (attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (on_dev) {
        // device source: pad on the device (values are the caller's responsibility)
        const int64_t n = (int64_t)NFEED * ld;
        h->hfeed.resize((size_t)NFEED * S);
        CK(cudaMemcpyAsync(h->hfeed.data(), feeds, sizeof(double) * h->hfeed.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        pad_feed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)S, ld, feeds, h->feed);
        return launch_check(h);
    }
    h->hfeed.assign(feeds, feeds + (size_t)NFEED * S);
    std::vector<double> hf((size_t)NFEED * ld, 0.0);
    for (int f = 0; f < NFEED; ++f)
        for (int64_t s = 0; s < ld; ++s) {
            const double v = feeds[(size_t)f * S + (s < S ? s : S - 1)];
            if (!std::isfinite(v)) return fail(h, ABS_ERR_NUMERIC, "non-finite feed value");
            hf[(size_t)f * ld + s] = v;
        }
    CK(cudaMemcpyAsync(h->feed, hf.data(), sizeof(double) * hf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return ABS_OK;
}

}  // namespace

// ======================================================================================
// C ABI
// ======================================================================================
extern "C" {

const char* abs_last_error(const abs_problem* h) { return h ? h->err.c_str() : g_err.c_str(); }

void abs_default_options(abs_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-8;
    o->max_iter = 300;
    o->precision = ABS_PREC_FP64;
    o->max_refine = 0;
    o->refine_tol = 1e-12;
    o->mu_init = 0.1;
    o->kappa_eps = 10.0;
    o->kappa_mu = 0.2;
    o->theta_mu = 1.5;
    o->tau_min = 0.99;
    o->s_max = 100.0;
    o->kappa_sigma = 1e10;
    o->bound_push = 1e-2;
    o->bound_frac = 1e-2;
    o->gamma_theta = 1e-5;
    o->gamma_phi = 1e-5;
    o->delta = 1.0;
    o->s_theta = 1.1;
    o->s_phi = 2.3;
    o->eta_phi = 1e-4;
    o->gamma_alpha = 0.05;
    o->lam_init_max = 1e3;
    o->dw0 = 1e-4;
    o->dw_min = 1e-20;
    o->dw_max = 1e40;
    o->kw_minus = 1.0 / 3.0;
    o->kw_plus = 8.0;
    o->kw_plus_bar = 100.0;
    o->max_ls = 60;
    o->verbose = 0;
    o->profile = 0;
    o->init = 0;
    o->soc_max = 4;
    o->kappa_soc = 0.99;
    o->obj_scaling = 0.0;
}

abs_status absorber_create(const abs_params* p, const double* feeds, const double* prob, int64_t S,
                           abs_problem** out) {
    abs_problem* h = nullptr;
    if (!p || !feeds || !out || S < 1 || S > (int64_t)1 << 26) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    *out = nullptr;
    if (!(p->d_lo < p->d_hi) || !(p->T_lo < p->T_hi) || !(p->d_lo > 0.0))
        return fail(nullptr, ABS_ERR_INFEASIBLE, "inconsistent bounds");
    PatternTables& T = pattern();
    if (!T.ok) return fail(nullptr, ABS_ERR_ARG, "pattern construction failed");
    h = new abs_problem();
    CK(cudaGetDevice(&h->dev));
    CK(upload_tables(h->dev));
    h->S = S;
    h->ld = (S + 31) / 32 * 32;
    std::memcpy(&h->P, p, sizeof(abs_params));
    h->aparams = *p;
    for (int l = 0; l < 9; ++l) {
        if (!(p->sx[l] > 0.0)) {
            delete h;
            return fail(nullptr, ABS_ERR_ARG, "scales must be positive");
        }
        h->P.lnsx[l] = std::log(p->sx[l]);
        h->P.hL0[l] = p->hL_ref[l] + p->hL_dh[l];
    }
    for (int j = 0; j < 4; ++j) h->P.hV0[j] = p->hV_ref[j] + p->hV_dh[j];
    h->nnzJ = (int)T.jrow.size();
    h->nnzH = (int)T.hrow.size();
    if (prob) {
        double sum = 0.0;
        h->prob.assign(prob, prob + S);
        for (double v : h->prob) {
            if (!(v >= 0.0)) {
                delete h;
                return fail(nullptr, ABS_ERR_ARG, "probabilities must be >= 0");
            }
            sum += v;
        }
        if (!(std::fabs(sum - 1.0) <= 1e-9)) {
            delete h;
            return fail(nullptr, ABS_ERR_ARG, "probabilities must sum to 1");
        }
    } else {
        h->prob.assign(S, 1.0 / (double)S);
    }
    CK(cudaMalloc(&h->feed, sizeof(double) * (size_t)NFEED * h->ld));
    abs_status r = upload_feeds(h, feeds, nullptr);
    if (r != ABS_OK) {
        const std::string msg = h->err;
        absorber_destroy(h);
        return fail(nullptr, r, msg);
    }
    *out = h;
    return ABS_OK;
}

abs_status absorber_set_feeds(abs_problem* h, const double* feeds, abs_stream_t stream) {
    if (!h || !feeds) return fail(h, ABS_ERR_ARG, "bad argument");
    return upload_feeds(h, feeds, (cudaStream_t)stream);
}

void absorber_destroy(abs_problem* h) {
    if (!h) return;
    absorber_destroy(h->base);
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    cudaFree(h->feed);
    cudaFree(h->jac);
    cudaFree(h->hes);
    cudaFree(h->vec);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->LUp[k]);
        cudaFree(h->Gp[k]);
    }
    cudaFree(h->piv);
    cudaFree(h->sing);
    cudaFree(h->count);
    cudaFree(h->part);
    cudaFreeHost(h->hpart);
    delete h;
}

abs_status absorber_sizes(const abs_problem* h, abs_sizes* o) {
    if (!h || !o) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    o->S = h->S;
    o->ld = h->ld;
    const int64_t per_stage_vars = 2 * 11 + 3 + 5, per_stage_mesh = 11 + 2 + 5 + 2 + 1, per_stage_fix = 7 + 2;
    o->n_var_paper = 1 + h->S * N_STAGES * per_stage_vars;
    o->n_mesh = h->S * N_STAGES * per_stage_mesh;
    o->n_fix = h->S * N_STAGES * per_stage_fix;
    o->n_hyd = h->S * N_STAGES;
    o->n_unknowns = (int64_t)NSC * h->S + 1;
    o->n_rows = (int64_t)NSC * h->S;
    o->nnzJ_scen = h->nnzJ;
    o->nnzH_scen = h->nnzH;
    return ABS_OK;
}

abs_status abs_scenario_pattern(int32_t* nnzJ_scen, int32_t* nnzH_scen, int32_t* jrow, int32_t* jcol,
                                int32_t* hrow, int32_t* hcol) {
    const PatternTables& T = pattern();
    if (!T.ok) return fail(nullptr, ABS_ERR_ARG, "pattern construction failed");
    if (nnzJ_scen) *nnzJ_scen = (int32_t)T.jrow.size();
    if (nnzH_scen) *nnzH_scen = (int32_t)T.hrow.size();
    for (size_t k = 0; k < T.jrow.size(); ++k) {
        if (jrow) jrow[k] = T.jrow[k];
        if (jcol) jcol[k] = T.jcol[k];
    }
    for (size_t k = 0; k < T.hrow.size(); ++k) {
        if (hrow) hrow[k] = T.hrow[k];
        if (hcol) hcol[k] = T.hcol[k];
    }
    return ABS_OK;
}

int64_t abs_struct_size(int which) {
    switch (which) {
        case 0: return sizeof(abs_params);
        case 1: return sizeof(abs_sizes);
        case 2: return sizeof(abs_kkt_diag);
        case 3: return sizeof(abs_inertia);
        case 4: return sizeof(abs_solve_info);
        case 5: return sizeof(abs_options);
        case 6: return sizeof(abs_result);
        default: return -1;
    }
}

abs_status absorber_pattern(const abs_problem* h, int32_t* jrow, int32_t* jcol, int32_t* hrow, int32_t* hcol) {
    if (!h) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    return abs_scenario_pattern(nullptr, nullptr, jrow, jcol, hrow, hcol);
}

abs_status eval_grad_jac_hess(abs_problem* h, const double* x, const double* lambda, double obj_factor, double* f,
                              double* grad, double* c, double* jac_vals, double* hess_vals, abs_stream_t stream) {
    if (!h || !x || (hess_vals && !lambda)) return fail(h, ABS_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g = grid2(h);
    if (jac_vals && hess_vals)
        eval_kernel<true, true, true><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, x, nullptr, 0.0, lambda, h->feed, c,
                                                          jac_vals, hess_vals, nullptr);
    else if (jac_vals)
        eval_kernel<true, true, false><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, x, nullptr, 0.0, lambda, h->feed, c,
                                                           jac_vals, nullptr, nullptr);
    else if (hess_vals)
        eval_kernel<true, false, true><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, x, nullptr, 0.0, lambda, h->feed, c,
                                                           nullptr, hess_vals, nullptr);
    else if (c)
        eval_kernel<true, false, false><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, x, nullptr, 0.0, lambda, h->feed,
                                                            c, nullptr, nullptr, nullptr);
    abs_status r = launch_check(h);
    if (r != ABS_OK) return r;
    if (grad) {
        CK(cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)vsize(h) - sizeof(double) * (h->ld - 1), st));
        CK(cudaMemcpyAsync(grad + (int64_t)NSC * h->ld, &obj_factor, sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (f) {
        double d = 0.0;
        CK(cudaMemcpyAsync(&d, x + (int64_t)NSC * h->ld, sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *f = obj_factor * d;
    } else if (grad) {
        CK(cudaStreamSynchronize(st));   // obj_factor lives on this stack frame
    }
    return ABS_OK;
}

abs_status kkt_factor(abs_problem* h, const double* x, const double* jac_vals, const double* hess_vals,
                      const abs_kkt_diag* diag, int precision, abs_inertia* inertia, abs_stream_t stream) {
    if (!h || !x || !jac_vals || !hess_vals || !diag || !diag->sigma || !inertia)
        return fail(h, ABS_ERR_ARG, "bad argument");
    if (precision != ABS_PREC_FP64 && precision != ABS_PREC_FP32) return fail(h, ABS_ERR_ARG, "bad precision");
    if (diag->delta_c != 0.0) return fail(h, ABS_ERR_ARG, "delta_c must be 0: J_s is square");
    cudaStream_t st = (cudaStream_t)stream;
    abs_status r = ensure_buffers(h);
    if (r != ABS_OK) return r;
    KKTSys K;
    K.jac = jac_vals;
    K.hes = hess_vals;
    K.sig = diag->sigma;
    K.use_w = true;
    K.dw = diag->delta_w;
    K.prec = precision;
    double sigd = 0.0;
    CK(cudaMemcpyAsync(&K.d, x + (int64_t)NSC * h->ld, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&sigd, diag->sigma + (int64_t)NSC * h->ld, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    int64_t nsing = 0;
    double wdd = 0.0;
    if ((r = kkt_factor_core(h, K, x + (int64_t)NSC * h->ld, &nsing, &wdd, st)) != ABS_OK) return r;
    K.Kdd = wdd + sigd;
    K.Sd = schur_value(K, K.dw);
    const int64_t nb = (int64_t)NSC * h->S;
    inertia->n_pos = nb + (K.Sd > 0 ? 1 : 0);
    inertia->n_neg = nb + (K.Sd < 0 ? 1 : 0);
    inertia->n_zero = (K.Sd == 0 ? 1 : 0);
    inertia->schur_d = K.Sd;
    inertia->n_singular = nsing;
    h->fac.valid = nsing == 0;
    h->fac.prec = precision;
    h->fac.jac = jac_vals;
    h->fac.hes = hess_vals;
    h->fac.sig = diag->sigma;
    h->fac.d = K.d;
    h->fac.dw = K.dw;
    h->fac.Kdd = K.Kdd;
    h->fac.A0 = K.A0;
    h->fac.Q2 = K.Q2;
    h->fac.Sd = K.Sd;
    h->fac.use_w = true;
    if (nsing) return fail(h, ABS_ERR_NUMERIC, "singular stage block in the constraint Jacobian");
    return ABS_OK;
}

abs_status kkt_solve(abs_problem* h, const double* rhs_x, const double* rhs_c, double* sol_x, double* sol_c,
                     int max_refine, double refine_tol, abs_solve_info* info, abs_stream_t stream) {
    if (!h || !rhs_x || !rhs_c || !sol_x || !sol_c || max_refine < 0) return fail(h, ABS_ERR_ARG, "bad argument");
    if (!h->fac.valid) return fail(h, ABS_ERR_ARG, "no valid factorization (call kkt_factor)");
    cudaStream_t st = (cudaStream_t)stream;
    KKTSys K;
    K.jac = h->fac.jac;
    K.hes = h->fac.hes;
    K.sig = h->fac.sig;
    K.use_w = h->fac.use_w;
    K.dw = h->fac.dw;
    K.d = h->fac.d;
    K.Kdd = h->fac.Kdd;
    K.A0 = h->fac.A0;
    K.Q2 = h->fac.Q2;
    K.Sd = h->fac.Sd;
    K.prec = h->fac.prec;
    double rd = 0.0;
    CK(cudaMemcpyAsync(&rd, rhs_x + (int64_t)NSC * h->ld, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    // the d slot of x holds the diameter for b = dc/dd; keep it in a device scalar
    double* xd = V(h, V_ONE) + (int64_t)NSC * h->ld;
    CK(cudaMemcpyAsync(xd, &K.d, sizeof(double), cudaMemcpyHostToDevice, st));
    int steps = 0;
    double resid = 0.0;
    abs_status r = kkt_solve_refined(h, K, xd, rhs_x, rd, rhs_c, sol_x, sol_c, max_refine, refine_tol, &steps,
                                     (info || max_refine > 0) ? &resid : nullptr, st);
    if (r != ABS_OK) return r;
    if (info) {
        info->refine_steps = steps;
        info->residual = resid;
    }
    return ABS_OK;
}

}  // extern "C"

namespace {
template <class T>
__global__ void fma_peak_kernel(int iters, T a0, T b0, T* out) {
    T a[8], b = b0;
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = a0 + (T)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, (T)0.5);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == (T)-1.2345) out[0] = s;   // keeps the chains live; never true for these inputs
}

template <class T>
abs_status fma_peak(double* gflops) {
    abs_problem* h = nullptr;
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    T* out = nullptr;
    CK(cudaMalloc(&out, sizeof(T)));
    const int threads = 256, blocks = sms * 8, iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    fma_peak_kernel<T><<<blocks, threads>>>(iters, (T)1.0, (T)0.999999, out);   // warm-up
    cudaEventRecord(e0);
    for (int r = 0; r < 5; ++r) fma_peak_kernel<T><<<blocks, threads>>>(iters, (T)1.0, (T)0.999999, out);
    cudaEventRecord(e1);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (err != cudaSuccess) return fail(nullptr, ABS_ERR_CUDA, cudaGetErrorString(err));
    const double flops = 5.0 * 2.0 * 8.0 * (double)iters * threads * blocks;
    *gflops = flops / (ms * 1e-3) / 1e9;
    return ABS_OK;
}
}  // namespace

extern "C" abs_status abs_measure_fma_peak(int kind, double* gflops) {
    if (!gflops || (kind != 0 && kind != 1)) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    return kind == 0 ? fma_peak<double>(gflops) : fma_peak<float>(gflops);
}

// the interior-point driver lives in its own file (same translation unit)
#include "ipm.inc"

// ======================================================================================
// Newton direction without any allocation (no handle, no cudaMalloc, no pinned memory)
// ======================================================================================
// For callers that cannot allocate device memory after start-up -- code running under
// a fixed memory budget, inside another runtime's allocator, or between graph
// captures -- this entry runs the FP64 stage-block LU, the Schur step on d and the
// block solves with every intermediate in one file-scope device array.
namespace {

constexpr int64_t NA_MAX_S = ABS_NOALLOC_MAX_SCENARIOS;    // scenarios per call, at most
constexpr int64_t NA_LD = NA_MAX_S;                         // a multiple of 32
constexpr size_t NA_LU = (size_t)N_STAGES * NV * NV * NA_LD;
constexpr size_t NA_G = (size_t)N_STAGES * NV * NABV * NA_LD;
constexpr size_t NA_VEC = (size_t)NSC * NA_LD + NA_LD;
constexpr int NA_NBLK = (int)((NA_MAX_S + 127) / 128) * N_STAGES;
constexpr size_t NA_PART = (size_t)16 * NA_NBLK;
constexpr size_t NA_PIV = ((size_t)N_STAGES * NV * NA_LD + 7) / 8;   // bytes as doubles
constexpr size_t NA_SING = (NA_LD + 1) / 2;                         // ints as doubles
constexpr size_t NA_TOTAL = NA_LU + NA_G + 3 * NA_VEC + NA_PART + NA_PIV + NA_SING + 1;

// the scratch: every device that loads the library holds it until the process exits
static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

double* g_na_base[64] = {nullptr};
double g_na_host_part[NA_PART];   // host copy of the block partials (static, not allocated)

}  // namespace

extern "C" abs_status kkt_newton_noalloc(const abs_params* p, int64_t S, int64_t ld, const double* x,
                                         const double* jac_vals, const double* hess_vals, const double* sigma,
                                         double delta_w, const double* rhs_x, const double* rhs_c, double* sol_x,
                                         double* sol_c, double* schur_d, abs_stream_t stream) {
    abs_problem* h = nullptr;   // for CK(): errors go to the global message
    if (!p || !x || !jac_vals || !hess_vals || !sigma || !rhs_x || !rhs_c || !sol_x || !sol_c)
        return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: NULL argument");
    if (S < 1 || S > NA_MAX_S)
        return fail(nullptr, ABS_ERR_ARG,
                    "kkt_newton_noalloc: S must be in [1, " + std::to_string(NA_MAX_S) + "] (static scratch size)");
    if (ld != (S + 31) / 32 * 32) return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: ld must be S rounded up to 32");
    if (!(delta_w >= 0.0)) return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: delta_w must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: device index out of range");
    if (!g_na_base[dev]) {
        // once per device, with that device current: the array's device address
        double* ptr = nullptr;
        CK(cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch));
        CK(upload_tables(dev));
        g_na_base[dev] = ptr;
    }
    double* LU = g_na_base[dev];
    double* G = LU + NA_LU;
    double* pv = G + NA_G;
    double* qv = pv + NA_VEC;
    double* gv = qv + NA_VEC;
    double* part = gv + NA_VEC;
    unsigned char* piv = (unsigned char*)(part + NA_PART);
    int* sing = (int*)((double*)piv + NA_PIV);
    int* count = (int*)((double*)sing + NA_SING);
    // the problem's constants (derived fields as absorber_create computes them)
    Params P;
    std::memset(&P, 0, sizeof(P));
    std::memcpy(&P, p, sizeof(abs_params));
    for (int l = 0; l < 9; ++l) {
        if (!(p->sx[l] > 0.0)) return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: scales must be positive");
        P.lnsx[l] = std::log(p->sx[l]);
        P.hL0[l] = p->hL_ref[l] + p->hL_dh[l];
    }
    for (int j = 0; j < 4; ++j) P.hV0[j] = p->hV_ref[j] + p->hV_dh[j];
    const dim3 g1((unsigned)((S + kThrS - 1) / kThrS)), g2((unsigned)((S + kThr - 1) / kThr), N_STAGES);
    const int nb = (int)g2.x * N_STAGES;
    const int64_t od = (int64_t)NSC * ld;
    cudaError_t e;
#define NA_LAUNCHED()                                                                                  \
    if ((e = cudaGetLastError()) != cudaSuccess)                                                       \
        return fail(nullptr, ABS_ERR_CUDA, std::string("kkt_newton_noalloc: ") + cudaGetErrorString(e));
    // the singular-block counter must start at zero on every call
    CK(cudaMemsetAsync(count, 0, sizeof(int), st));
    const dim3 gf((unsigned)((S + WPB_F - 1) / WPB_F)), gs((unsigned)((S + WPB_S - 1) / WPB_S));
    factor_warp_kernel<double><<<gf, 32 * WPB_F, 0, st>>>((int)S, ld, jac_vals, LU, piv, G, sing, count, 1e-14);
    NA_LAUNCHED();
    // p = J^-1 r_c, q = J^-1 b
    solve_warp_kernel<double, 2><<<gs, 32 * WPB_S, 0, st>>>(P, (int)S, ld, jac_vals, LU, piv, G, x + od, rhs_c,
                                                            nullptr, pv, qv);
    NA_LAUNCHED();
    schur_kernel<<<g2, kThr, 0, st>>>((int)S, ld, hess_vals, sigma, true, pv, qv, rhs_x, part);
    NA_LAUNCHED();
    int cnt = 0;
    double hx[3] = {0.0, 0.0, 0.0};
    CK(cudaMemcpyAsync(&cnt, count, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hx[0], x + od, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hx[1], sigma + od, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hx[2], rhs_x + od, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(g_na_host_part, part, sizeof(double) * 5 * (size_t)nb, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (cnt) return fail(nullptr, ABS_ERR_NUMERIC, "kkt_newton_noalloc: singular stage block");
    double red[5];
    for (int k = 0; k < 5; ++k) {
        double a = 0.0;
        for (int b = 0; b < nb; ++b) a += g_na_host_part[(size_t)k * nb + b];
        red[k] = a;
    }
    // S_d = K_dd + dw + sum q^T (W + Sigma) q + dw sum q^T q ;  dd = (r_d - beta) / S_d
    const double Kdd = red[4] + hx[1];
    const double Sd = Kdd + delta_w + red[0] + delta_w * red[1];
    if (schur_d) *schur_d = Sd;
    if (!(Sd > 0.0)) return fail(nullptr, ABS_ERR_INERTIA, "kkt_newton_noalloc: Schur complement on d is not positive");
    const double beta = red[2] - delta_w * red[3];
    const double dd = (hx[2] - beta) / Sd;
    CK(cudaMemcpyAsync(sol_x + od, &dd, sizeof(double), cudaMemcpyHostToDevice, st));
    dz_kernel<<<g2, kThr, 0, st>>>((int)S, ld, hess_vals, sigma, delta_w, true, pv, qv, sol_x + od, rhs_x, sol_x, gv);
    NA_LAUNCHED();
    solve_t_warp_kernel<double><<<gs, 32 * WPB_S, 0, st>>>((int)S, ld, jac_vals, LU, piv, gv, sol_c);
    NA_LAUNCHED();
#undef NA_LAUNCHED
    // dd lives on this stack frame until the copy above has completed
    CK(cudaStreamSynchronize(st));
    (void)nb;
    return ABS_OK;
}
