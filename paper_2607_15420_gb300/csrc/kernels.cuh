// kernels.cuh -- device kernels of the absorber library (included once, by absorber_lib.cu).
//
// Layout: structure of arrays over scenarios, leading dimension ld (a multiple of 32):
// per-scenario entry v of scenario s lives at [v * ld + s], so a warp touches 32
// consecutive doubles of one entry (one 256-byte coalesced access).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "model.cuh"

namespace absorber {

constexpr int NABV = 11;   // stream-from-above unknowns of stage n+1 read by stage n
constexpr int NBLW = 6;    // stream-from-below unknowns of stage n-1 read by stage n
constexpr int NHS = 66;    // Hessian lower-triangle entries per stage block
constexpr int MAXOWN = 192, MAXABV = 64, MAXBLW = 32;

__host__ __device__ constexpr int abv_var(int a) { return a < 9 ? a : (a == 9 ? LL : LT); }
__host__ __device__ constexpr int blw_var(int b) { return b < 4 ? LY + b : (b == 4 ? LV : LT); }
__host__ __device__ constexpr int stage_type(int n) { return n == 0 ? 0 : (n == N_STAGES - 1 ? 2 : 1); }

struct Ent {
    short slot;        // entry offset inside the stage's CSR segment
    signed char r;     // row inside the stage
    signed char c;     // column: own unknown (0..21), or above index (0..10), or below (0..5)
};

// Pattern tables, identical for every problem (the model is fixed); uploaded once per
// device.  Built on the host by running stage_eval with a recording emitter.
__constant__ short c_slotJ[3][NR][NLOC];
__constant__ int c_segJ[N_STAGES + 1];
__constant__ short c_slotH[NV][NV];
__constant__ Ent c_own[3][MAXOWN];
__constant__ Ent c_abv[3][MAXABV];
__constant__ Ent c_blw[3][MAXBLW];
__constant__ Ent c_hes[NHS];
__constant__ int c_nown[3], c_nabv[3], c_nblw[3];
__constant__ int c_dslot[3];           // the d entry of the stage's hydraulic row
// The stage tables that the factor and solve kernels read with a different entry on
// every lane (a constant-cache read with 32 different addresses is serialized): one
// global-memory copy, which each factor block stages into shared memory.
struct __align__(16) LaneTables {
    Ent own[3][MAXOWN];
    Ent abv[3][MAXABV];
    Ent blw[3][MAXBLW];
    short blwRp[3][NV + 2];        // row pointers of blw (NV + 1 used; padded to 16 bytes)
    short blwCp[3][NV + 2];        // pointers into blwQ by the stage-below unknown fed
    unsigned char blwQ[3][MAXBLW]; // blw entry indices grouped by that unknown (table order)
};
static_assert(sizeof(LaneTables) % 16 == 0, "LaneTables is copied as 16-byte words");
__device__ LaneTables g_lt;
// The same entries grouped by destination, so that the sparse products below accumulate
// into statically indexed registers (table-indexed register arrays would live in local
// memory): row pointers of the row-ordered tables (J v), copies ordered by the unknown
// they feed (J^T y), and the Hessian block expanded to both triangles by row (H v).
__constant__ short c_ownRp[3][NV + 1], c_abvRp[3][NV + 1], c_blwRp[3][NV + 1];
__constant__ Ent c_ownC[3][MAXOWN], c_abvC[3][MAXABV], c_blwC[3][MAXBLW];
__constant__ short c_ownCp[3][NV + 1], c_abvCp[3][NV + 1], c_blwCp[3][NV + 1];
__constant__ Ent c_hesF[2 * NHS];
__constant__ short c_hesFp[NV + 1];

// bounds of the stage unknowns (10d): lower 0 for fractions, flows and the slack,
// both for T, none for the extents
__host__ __device__ constexpr bool has_lo(int j) { return !(j >= LE && j < LE + 5); }
__host__ __device__ constexpr bool has_hi(int j) { return j == LT; }

// ------------------------------------------------------------------------------------
// problems: a launch covers one or many independent problems (a batch).  Scenario slot
// s belongs to problem pid[s] (-1: padding); per-problem scalars live in device arrays
// ps[field * NP + p].  pid == nullptr means a single problem owning every slot s < S,
// ps == nullptr means no per-problem scalars (every problem active).
// ------------------------------------------------------------------------------------
enum PsField {
    PS_MU = 0,     // barrier parameter
    PS_TAU,        // fraction-to-the-boundary parameter
    PS_ALPHA,      // primal step / trial step
    PS_ALPHAZ,     // bound-multiplier step
    PS_DW,         // primal regularisation delta_w
    PS_ACT,        // 1: problem takes part in this iteration
    PS_LSACT,      // 1: problem takes part in this line-search trial
    PS_SOC,        // 1: the trial follows the second-order-correction direction
    PS_A0,         // coefficient (first trial step) of the SOC right-hand side
    PS_COUNT
};

struct BView {
    const int* pid;
    const double* ps;
    int NP;
};

__device__ inline int prob_of(const BView& b, int s) { return b.pid ? b.pid[s] : 0; }
__device__ inline double psv(const BView& b, int field, int p) { return b.ps[(int64_t)field * b.NP + p]; }
// problem of slot s if it takes part (flag field PS_ACT or PS_LSACT), else -1
__device__ inline int live_prob(const BView& b, int s, int S, int flag) {
    if (s >= S) return -1;
    const int p = prob_of(b, s);
    if (p < 0) return -1;
    if (b.ps && psv(b, flag, p) == 0.0) return -1;
    return p;
}

// ------------------------------------------------------------------------------------
// reductions: every (scenario, stage) thread stores its K partial values at
// part[k * plane + n * ld + s] (plane = N_STAGES * ld); reduce_kernel (vec_kernels.cuh)
// combines them per problem in a fixed order (deterministic)
// ------------------------------------------------------------------------------------
enum RedOp { RSUM = 0, RMAX = 1, RMIN = 2 };

// |a| as an unsigned integer that orders like |a| (the IEEE layout with the sign cleared;
// a NaN orders above +inf): maxima of magnitudes taken on the integer pipe, off the FP64
// pipe, and a NaN among them survives (the key of the maximum is NaN's)
__device__ __forceinline__ unsigned long long mag_key(double a) {
    return (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long key_max(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}
__device__ __forceinline__ double key_double(unsigned long long k) { return __longlong_as_double((long long)k); }

__device__ inline double red_id(int op) { return op == RSUM ? 0.0 : (op == RMAX ? -INFINITY : INFINITY); }

__device__ inline double red_op(int op, double a, double b) {
    if (op == RSUM) return a + b;
    if (op == RMAX) return (b > a || b != b) ? b : a;
    return (b < a || b != b) ? b : a;
}

template <int K>
__device__ inline void store_partials(const double (&v)[K], double* part, int64_t ld, int s, int n) {
    const int64_t plane = (int64_t)N_STAGES * ld;
#pragma unroll
    for (int k = 0; k < K; ++k) part[(int64_t)k * plane + (int64_t)n * ld + s] = v[k];
}

// ------------------------------------------------------------------------------------
// A1 + A2: residuals, Jacobian and Lagrangian Hessian values, one thread per
// (scenario, stage); grid (ceil(S / blockDim), N_STAGES).
// ------------------------------------------------------------------------------------
template <bool WR, bool WJ, bool WH>
struct DevEmit {
    static constexpr bool want_res = WR, want_jac = WJ, want_hes = WH;
    double* cv;
    double* jv;
    double* hv;
    int64_t ld;
    int s, n, t;
    double asum, amax;
    __device__ void res(int r, double v) {
        if (cv) cv[(int64_t)(NR * n + r) * ld + s] = v;
        const double a = fabs(v);
        asum += a;
        amax = (a > amax || a != a) ? a : amax;
    }
    __device__ void jac(int r, int lv, double v) {
        jv[(int64_t)(c_segJ[n] + c_slotJ[t][r][lv]) * ld + s] = v;
    }
    __device__ void hes(int i, int j, double v) {
        hv[(int64_t)(NHS * n + c_slotH[i][j]) * ld + s] = v;
    }
};

__device__ inline void load_stage(const Params& P, int S, int64_t ld, const double* __restrict__ x,
                                  const double* __restrict__ dx, double alpha, const double* __restrict__ feed,
                                  int s, int n, int p, int NP, StageIn& in) {
    const double* xs = x + s;
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        double v = xs[(int64_t)(NV * n + j) * ld];
        if (dx) v += alpha * dx[(int64_t)(NV * n + j) * ld + s];
        in.q[j] = v;
    }
    in.has_above = n + 1 < N_STAGES;
    in.has_below = n > 0;
    if (in.has_above) {
#pragma unroll
        for (int a = 0; a < NABV; ++a) {
            const int64_t o = (int64_t)(NV * (n + 1) + abv_var(a)) * ld + s;
            double v = x[o];
            if (dx) v += alpha * dx[o];
            in.qa[a] = v;
        }
    } else {
#pragma unroll
        for (int l = 0; l < 9; ++l) in.qa[l] = feed[(int64_t)(F_XIN + l) * ld + s] / P.sx[l];
        in.qa[9] = feed[(int64_t)F_LIN * ld + s];
        in.qa[10] = feed[(int64_t)F_TIN * ld + s] / P.sT;
    }
    if (in.has_below) {
#pragma unroll
        for (int b = 0; b < NBLW; ++b) {
            const int64_t o = (int64_t)(NV * (n - 1) + blw_var(b)) * ld + s;
            double v = x[o];
            if (dx) v += alpha * dx[o];
            in.qb[b] = v;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) in.qb[j] = feed[(int64_t)(F_Y0 + j) * ld + s] / P.sy[j];
        in.qb[4] = feed[(int64_t)F_V0 * ld + s];
        in.qb[5] = feed[(int64_t)F_T0 * ld + s] / P.sT;
    }
    const int64_t od = (int64_t)NSC * ld + (int64_t)stage_sec(n, P.nsec) * NP + p;   // its section's diameter
    in.d = x[od] + (dx ? alpha * dx[od] : 0.0);
    in.P = stage_pres(P, feed[(int64_t)F_P * ld + s], n);
}

// partials (if part non-null): [0] |c| summed over the stage's rows, [1] their max,
// [2] sum of the barrier logs of the stage unknowns.  trial = false: evaluation at x of
// the problems flagged PS_ACT; trial = true: at x + alpha_p dir of the problems flagged
// PS_LSACT, dir = dxB where PS_SOC is set, else dxA.
template <bool WR, bool WJ, bool WH>
__global__ void __launch_bounds__(128) eval_kernel(const Params P, int S, int64_t ld, const BView b, bool trial,
                                                   const double* __restrict__ x, const double* __restrict__ dxA,
                                                   const double* __restrict__ dxB, const double* __restrict__ lam,
                                                   const double* __restrict__ feed, double* c, double* jac,
                                                   double* hes, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int p = live_prob(b, s, S, trial ? PS_LSACT : PS_ACT);
    if (p < 0) return;
    DevEmit<WR, WJ, WH> em;
    em.cv = c;
    em.jv = jac;
    em.hv = hes;
    em.ld = ld;
    em.s = s;
    em.n = n;
    em.t = stage_type(n);
    em.asum = 0.0;
    em.amax = 0.0;
    double blog = 0.0;
    StageIn in;
    const double* dx = nullptr;
    double alpha = 0.0;
    if (trial) {
        dx = (b.ps && psv(b, PS_SOC, p) != 0.0) ? dxB : dxA;
        alpha = psv(b, PS_ALPHA, p);
    }
    load_stage(P, S, ld, x, dx, alpha, feed, s, n, p, b.NP, in);
    StageLam L;
    if (WH) {
#pragma unroll
        for (int r = 0; r < NR; ++r) L.own[r] = lam[(int64_t)(NR * n + r) * ld + s];
        if (n > 0) {
#pragma unroll
            for (int k = 0; k < 9; ++k) L.below[k] = lam[(int64_t)(NR * (n - 1) + k) * ld + s];
            L.below[9] = lam[(int64_t)(NR * (n - 1) + R_E) * ld + s];
        }
        if (n + 1 < N_STAGES) {
#pragma unroll
            for (int k = 0; k < 4; ++k) L.above[k] = lam[(int64_t)(NR * (n + 1) + 7 + k) * ld + s];
            L.above[4] = lam[(int64_t)(NR * (n + 1) + R_E) * ld + s];
        }
    }
    stage_eval(P, in, WH ? &L : nullptr, em);
    if (WH && n == 0) {
        // the scenario's share of d-d: -u_max pi / 2 * sum_n lambda_hydraulic, one entry per
        // section (its stages' rows)
        for (int k = 0; k < P.nsec; ++k) {
            double sl = 0.0;
#pragma unroll
            for (int m = 0; m < N_STAGES; ++m)
                if (stage_sec(m, P.nsec) == k) sl += lam[(int64_t)(NR * m + R_H) * ld + s];
            hes[(int64_t)(NHS * N_STAGES + k) * ld + s] = -P.u_max * M_PI * 0.5 * sl;
        }
    }
    if (part) {
        // sum of ln(slack) over the stage's 18 bounds as the logarithm of their product: the
        // product is carried as a mantissa in [1, 2) times a power of two (exponent read from
        // the bit pattern), so it neither overflows nor underflows; a slack that is not
        // positive and finite makes the sum NaN (the trial is rejected as before)
        double m = 1.0;
        long long e2 = 0;
        bool bad = false;
        auto take = [&](double sl) {
            bad = bad || !(sl > 0.0) || !(sl < INFINITY);
            m *= sl;
            const unsigned long long bits = (unsigned long long)__double_as_longlong(m);
            const int ex = (int)((bits >> 52) & 0x7ffull);
            if (ex == 0 || ex == 0x7ff) {
                bad = true;
                return;
            }
            e2 += ex - 1023;
            m = __longlong_as_double((long long)((bits & ~(0x7ffull << 52)) | (1023ull << 52)));
        };
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            if (has_lo(j)) take(in.q[j] - (j == LT ? P.Tlo_s : 0.0));
            if (has_hi(j)) take(P.Thi_s - in.q[j]);
        }
        blog = bad ? NAN : log(m) + (double)e2 * 0.69314718055994530942;   // ln 2
        const double v[3] = {em.asum, em.amax, blog};
        store_partials<3>(v, part, ld, s, n);
    }
}

// ------------------------------------------------------------------------------------
// sparse products with the stage-structured Jacobian / Hessian
// ------------------------------------------------------------------------------------
// (J^T y)_j for unknown j of stage n: rows of stage n (own entries), of stage n-1 (their
// stream-from-above entries) and of stage n+1 (stream-from-below), in a fixed order
__device__ __forceinline__ double jt_one(int64_t ld, const double* __restrict__ jac, const double* __restrict__ y, int s,
                                int n, int j) {
    const int t = stage_type(n);
    const int base = c_segJ[n];
    double a = 0.0;
    for (int k = c_ownCp[t][j]; k < c_ownCp[t][j + 1]; ++k) {
        const Ent e = c_ownC[t][k];
        a += jac[(int64_t)(base + e.slot) * ld + s] * y[(int64_t)(NR * n + e.r) * ld + s];
    }
    if (n > 0) {
        const int tb = stage_type(n - 1), bb = c_segJ[n - 1];
        for (int k = c_abvCp[tb][j]; k < c_abvCp[tb][j + 1]; ++k) {
            const Ent e = c_abvC[tb][k];
            a += jac[(int64_t)(bb + e.slot) * ld + s] * y[(int64_t)(NR * (n - 1) + e.r) * ld + s];
        }
    }
    if (n + 1 < N_STAGES) {
        const int ta = stage_type(n + 1), ba = c_segJ[n + 1];
        for (int k = c_blwCp[ta][j]; k < c_blwCp[ta][j + 1]; ++k) {
            const Ent e = c_blwC[ta][k];
            a += jac[(int64_t)(ba + e.slot) * ld + s] * y[(int64_t)(NR * (n + 1) + e.r) * ld + s];
        }
    }
    return a;
}

// (J v)_r for row r of stage n; v a primal vector, vd the step of the stage's section
// diameter (the hydraulic row's d column)
__device__ __forceinline__ double jv_one(int64_t ld, const double* __restrict__ jac, const double* __restrict__ v, double vd,
                                int s, int n, int r) {
    const int t = stage_type(n);
    const int base = c_segJ[n];
    double a = 0.0;
    for (int k = c_ownRp[t][r]; k < c_ownRp[t][r + 1]; ++k) {
        const Ent e = c_own[t][k];
        a += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * n + e.c) * ld + s];
    }
    if (n + 1 < N_STAGES)
        for (int k = c_abvRp[t][r]; k < c_abvRp[t][r + 1]; ++k) {
            const Ent e = c_abv[t][k];
            a += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * (n + 1) + abv_var(e.c)) * ld + s];
        }
    if (n > 0)
        for (int k = c_blwRp[t][r]; k < c_blwRp[t][r + 1]; ++k) {
            const Ent e = c_blw[t][k];
            a += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * (n - 1) + blw_var(e.c)) * ld + s];
        }
    if (r == R_H) a += jac[(int64_t)(base + c_dslot[t]) * ld + s] * vd;
    return a;
}

// ((W + Sigma + dw I) v)_j for unknown j of stage n (W block diagonal by stage);
// use_w = false gives (Sigma + dw I) v
__device__ __forceinline__ double hv_one(int64_t ld, const double* __restrict__ hes, const double* __restrict__ sig,
                                double dw, bool use_w, const double* __restrict__ v, int s, int n, int j) {
    const int64_t o = (int64_t)(NV * n + j) * ld + s;
    double a = (sig[o] + dw) * v[o];
    if (use_w)
        for (int k = c_hesFp[j]; k < c_hesFp[j + 1]; ++k) {
            const Ent e = c_hesF[k];
            a += hes[(int64_t)(NHS * n + e.slot) * ld + s] * v[(int64_t)(NV * n + e.c) * ld + s];
        }
    return a;
}

}  // namespace absorber
