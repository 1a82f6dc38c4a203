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

// bounds of the stage unknowns (10d): lower 0 for fractions, flows and the slack,
// both for T, none for the extents
__host__ __device__ constexpr bool has_lo(int j) { return !(j >= LE && j < LE + 5); }
__host__ __device__ constexpr bool has_hi(int j) { return j == LT; }

// ------------------------------------------------------------------------------------
// block reductions (deterministic: fixed shuffle tree, fixed smem order)
// ------------------------------------------------------------------------------------
enum RedOp { RSUM = 0, RMAX = 1, RMIN = 2 };

__device__ inline double warp_red(double v, int op) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        if (op == RSUM) v += w;
        else if (op == RMAX) v = (w > v || w != w) ? w : v;
        else v = (w < v || w != w) ? w : v;
    }
    return v;
}

// reduce K values per thread across the block; thread 0 writes part[k * nblk + blk]
template <int K>
__device__ inline void block_reduce_store(double (&v)[K], const int (&ops)[K], double* part,
                                          int nblk, int blk) {
    __shared__ double sm[K][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K; ++k) {
        double w = warp_red(v[k], ops[k]);
        if (lane == 0) sm[k][wid] = w;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            double w = (lane < nw) ? sm[k][lane]
                                   : (ops[k] == RSUM ? 0.0 : (ops[k] == RMAX ? -INFINITY : INFINITY));
            w = warp_red(w, ops[k]);
            if (lane == 0) part[(int64_t)k * nblk + blk] = w;
        }
    }
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
                                  int s, int n, StageIn& in) {
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
    const int64_t od = (int64_t)NSC * ld;
    in.d = x[od] + (dx ? alpha * dx[od] : 0.0);
    in.P = feed[(int64_t)F_P * ld + s];
}

// partials (if non-null): [0] sum |c|, [1] max |c|, [2] sum of barrier logs of the
// stage unknowns (at x + alpha dx), all per block.
template <bool WR, bool WJ, bool WH>
__global__ void __launch_bounds__(128) eval_kernel(const Params P, int S, int64_t ld,
                                                   const double* __restrict__ x, const double* __restrict__ dx,
                                                   double alpha, const double* __restrict__ lam,
                                                   const double* __restrict__ feed, double* c, double* jac,
                                                   double* hes, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
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
    if (s < S) {
        StageIn in;
        load_stage(P, S, ld, x, dx, alpha, feed, s, n, in);
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
            // the scenario's share of d-d: -u_max pi / 2 * sum_n lambda_hydraulic
            double sl = 0.0;
#pragma unroll
            for (int m = 0; m < N_STAGES; ++m) sl += lam[(int64_t)(NR * m + R_H) * ld + s];
            hes[(int64_t)(NHS * N_STAGES) * ld + s] = -P.u_max * M_PI * 0.5 * sl;
        }
        if (part) {
#pragma unroll
            for (int j = 0; j < NV; ++j) {
                if (has_lo(j)) blog += log(in.q[j] - (j == LT ? P.T_lo / P.sT : 0.0));
                if (has_hi(j)) blog += log(P.T_hi / P.sT - in.q[j]);
            }
        }
    }
    if (part) {
        double v[3] = {em.asum, em.amax, blog};
        const int ops[3] = {RSUM, RMAX, RSUM};
        block_reduce_store<3>(v, ops, part, gridDim.x * gridDim.y, blockIdx.y * gridDim.x + blockIdx.x);
    }
}

// ------------------------------------------------------------------------------------
// sparse products with the stage-structured Jacobian / Hessian
// ------------------------------------------------------------------------------------
// (J^T y) for the unknowns of stage n of scenario s: rows of stage n (own entries), of
// stage n-1 (their stream-from-above entries) and of stage n+1 (stream-from-below).
__device__ inline void jt_stage(int64_t ld, const double* __restrict__ jac, const double* __restrict__ y,
                                int s, int n, double (&out)[NV]) {
#pragma unroll
    for (int j = 0; j < NV; ++j) out[j] = 0.0;
    const int t = stage_type(n);
    const int base = c_segJ[n];
    for (int k = 0; k < c_nown[t]; ++k) {
        const Ent e = c_own[t][k];
        out[e.c] += jac[(int64_t)(base + e.slot) * ld + s] * y[(int64_t)(NR * n + e.r) * ld + s];
    }
    if (n > 0) {
        const int tb = stage_type(n - 1), bb = c_segJ[n - 1];
        for (int k = 0; k < c_nabv[tb]; ++k) {
            const Ent e = c_abv[tb][k];
            out[abv_var(e.c)] += jac[(int64_t)(bb + e.slot) * ld + s] * y[(int64_t)(NR * (n - 1) + e.r) * ld + s];
        }
    }
    if (n + 1 < N_STAGES) {
        const int ta = stage_type(n + 1), ba = c_segJ[n + 1];
        for (int k = 0; k < c_nblw[ta]; ++k) {
            const Ent e = c_blw[ta][k];
            out[blw_var(e.c)] += jac[(int64_t)(ba + e.slot) * ld + s] * y[(int64_t)(NR * (n + 1) + e.r) * ld + s];
        }
    }
}

// (J v) for the rows of stage n; v is a primal vector (d at [NSC*ld]) -- dd multiplies
// the d column (set has_d false to leave it out).
__device__ inline void jv_stage(int64_t ld, const double* __restrict__ jac, const double* __restrict__ v,
                                double vd, int s, int n, double (&out)[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) out[r] = 0.0;
    const int t = stage_type(n);
    const int base = c_segJ[n];
    for (int k = 0; k < c_nown[t]; ++k) {
        const Ent e = c_own[t][k];
        out[e.r] += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * n + e.c) * ld + s];
    }
    if (n + 1 < N_STAGES) {
        for (int k = 0; k < c_nabv[t]; ++k) {
            const Ent e = c_abv[t][k];
            out[e.r] += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * (n + 1) + abv_var(e.c)) * ld + s];
        }
    }
    if (n > 0) {
        for (int k = 0; k < c_nblw[t]; ++k) {
            const Ent e = c_blw[t][k];
            out[e.r] += jac[(int64_t)(base + e.slot) * ld + s] * v[(int64_t)(NV * (n - 1) + blw_var(e.c)) * ld + s];
        }
    }
    out[R_H] += jac[(int64_t)(base + c_dslot[t]) * ld + s] * vd;
}

// ((W + Sigma + dw I) v) for the unknowns of stage n (W block diagonal by stage);
// use_w = false gives (Sigma + dw I) v.
__device__ inline void hv_stage(int64_t ld, const double* __restrict__ hes, const double* __restrict__ sig,
                                double dw, bool use_w, const double* __restrict__ v, int s, int n,
                                double (&out)[NV]) {
    double vv[NV];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        vv[j] = v[(int64_t)(NV * n + j) * ld + s];
        out[j] = (sig[(int64_t)(NV * n + j) * ld + s] + dw) * vv[j];
    }
    if (use_w) {
#pragma unroll
        for (int k = 0; k < NHS; ++k) {
            const Ent e = c_hes[k];
            const double h = hes[(int64_t)(NHS * n + e.slot) * ld + s];
            out[e.r] += h * vv[e.c];
            if (e.r != e.c) out[e.c] += h * vv[e.r];
        }
    }
}

// ------------------------------------------------------------------------------------
// A4: block LU of every scenario's constraint Jacobian, one thread per scenario.
// J_s is block tridiagonal: diagonal blocks A_n (22 x 22), sub-diagonal C_n = dc_n/dz_{n-1}
// (only the stream-from-below columns), super-diagonal B_n = dc_n/dz_{n+1} (stream-from-
// above columns).  Recurrence: At_0 = A_0, At_n = A_n - C_n At_{n-1}^{-1} B_{n-1}; each
// At_n is LU-factored with partial pivoting inside the block (P At = L U, the reciprocal
// pivots kept on U's diagonal), and G_n = At_n^{-1} B_n (22 x 11) is stored for the
// back substitution.  Storage (SoA): LU[n][i][j], piv[n][k], G[n][i][a].
// ------------------------------------------------------------------------------------
template <class T>
__device__ inline T& mat(T* base, int64_t ld, int i, int j) { return base[(int64_t)(i * NV + j) * ld]; }

template <class T>
__global__ void __launch_bounds__(64) factor_kernel(int S, int64_t ld, const double* __restrict__ jac,
                                                    T* __restrict__ LU, unsigned char* __restrict__ piv,
                                                    T* __restrict__ G, int* __restrict__ sing, double pivtol) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int singular = 0;
    for (int n = 0; n < N_STAGES; ++n) {
        const int t = stage_type(n);
        const int base = c_segJ[n];
        T* A = LU + (int64_t)n * NV * NV * ld + s;
        for (int k = 0; k < NV * NV; ++k) A[(int64_t)k * ld] = T(0);
        for (int k = 0; k < c_nown[t]; ++k) {
            const Ent e = c_own[t][k];
            mat(A, ld, e.r, e.c) = (T)jac[(int64_t)(base + e.slot) * ld + s];
        }
        if (n > 0) {
            const T* Gp = G + (int64_t)(n - 1) * NV * NABV * ld + s;
            for (int k = 0; k < c_nblw[t]; ++k) {
                const Ent e = c_blw[t][k];
                const T cv = (T)jac[(int64_t)(base + e.slot) * ld + s];
                const int i = blw_var(e.c);
#pragma unroll
                for (int a = 0; a < NABV; ++a)
                    mat(A, ld, e.r, abv_var(a)) -= cv * Gp[(int64_t)(i * NABV + a) * ld];
            }
        }
        T amax = T(0);
        for (int k = 0; k < NV * NV; ++k) amax = fmax(amax, (T)fabs(A[(int64_t)k * ld]));
        const T tiny = (T)pivtol * amax;
        for (int k = 0; k < NV; ++k) {
            int p = k;
            T best = (T)fabs(mat(A, ld, k, k));
            for (int i = k + 1; i < NV; ++i) {
                const T a = (T)fabs(mat(A, ld, i, k));
                if (a > best) {
                    best = a;
                    p = i;
                }
            }
            piv[(int64_t)(n * NV + k) * ld + s] = (unsigned char)p;
            if (p != k) {
                for (int j = 0; j < NV; ++j) {
                    const T tmp = mat(A, ld, k, j);
                    mat(A, ld, k, j) = mat(A, ld, p, j);
                    mat(A, ld, p, j) = tmp;
                }
            }
            T ukk = mat(A, ld, k, k);
            if (!(fabs(ukk) > tiny)) {
                singular = 1;
                ukk = (ukk < T(0) ? -T(1) : T(1)) * (tiny > T(0) ? tiny : T(1));
            }
            const T inv = T(1) / ukk;
            mat(A, ld, k, k) = inv;
            for (int i = k + 1; i < NV; ++i) {
                const T l = mat(A, ld, i, k) * inv;
                mat(A, ld, i, k) = l;
                if (l != T(0)) {
                    for (int j = k + 1; j < NV; ++j) mat(A, ld, i, j) -= l * mat(A, ld, k, j);
                }
            }
        }
        if (n + 1 < N_STAGES) {
            T* Gn = G + (int64_t)n * NV * NABV * ld + s;
            for (int k = 0; k < NV * NABV; ++k) Gn[(int64_t)k * ld] = T(0);
            for (int k = 0; k < c_nabv[t]; ++k) {
                const Ent e = c_abv[t][k];
                Gn[(int64_t)(e.r * NABV + e.c) * ld] = (T)jac[(int64_t)(base + e.slot) * ld + s];
            }
            // G_n <- At_n^{-1} B_n : row swaps, unit-lower forward, upper backward
            for (int k = 0; k < NV; ++k) {
                const int p = piv[(int64_t)(n * NV + k) * ld + s];
                if (p != k) {
#pragma unroll
                    for (int a = 0; a < NABV; ++a) {
                        const T tmp = Gn[(int64_t)(k * NABV + a) * ld];
                        Gn[(int64_t)(k * NABV + a) * ld] = Gn[(int64_t)(p * NABV + a) * ld];
                        Gn[(int64_t)(p * NABV + a) * ld] = tmp;
                    }
                }
            }
            for (int i = 1; i < NV; ++i) {
                for (int k = 0; k < i; ++k) {
                    const T l = mat(A, ld, i, k);
                    if (l != T(0)) {
#pragma unroll
                        for (int a = 0; a < NABV; ++a)
                            Gn[(int64_t)(i * NABV + a) * ld] -= l * Gn[(int64_t)(k * NABV + a) * ld];
                    }
                }
            }
            for (int i = NV - 1; i >= 0; --i) {
                for (int k = i + 1; k < NV; ++k) {
                    const T u = mat(A, ld, i, k);
                    if (u != T(0)) {
#pragma unroll
                        for (int a = 0; a < NABV; ++a)
                            Gn[(int64_t)(i * NABV + a) * ld] -= u * Gn[(int64_t)(k * NABV + a) * ld];
                    }
                }
                const T inv = mat(A, ld, i, i);
#pragma unroll
                for (int a = 0; a < NABV; ++a) Gn[(int64_t)(i * NABV + a) * ld] *= inv;
            }
        }
    }
    sing[s] = singular;
}

// At_n^{-1} v in place (v in registers / local memory)
template <class T>
__device__ inline void lu_apply(const T* A, const unsigned char* pv, int64_t ld, T (&v)[NV]) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        const int p = pv[(int64_t)k * ld];
        if (p != k) {
            const T tmp = v[k];
            v[k] = v[p];
            v[p] = tmp;
        }
    }
#pragma unroll
    for (int i = 1; i < NV; ++i) {
        T acc = v[i];
#pragma unroll
        for (int k = 0; k < i; ++k) acc -= mat(const_cast<T*>(A), ld, i, k) * v[k];
        v[i] = acc;
    }
#pragma unroll
    for (int i = NV - 1; i >= 0; --i) {
        T acc = v[i];
#pragma unroll
        for (int k = i + 1; k < NV; ++k) acc -= mat(const_cast<T*>(A), ld, i, k) * v[k];
        v[i] = acc * mat(const_cast<T*>(A), ld, i, i);
    }
}

// At_n^{-T} v in place:  At^T = U^T L^T P  ->  U^T w = v,  L^T y = w,  v = P^T y
template <class T>
__device__ inline void lu_apply_t(const T* A, const unsigned char* pv, int64_t ld, T (&v)[NV]) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
        T acc = v[i];
#pragma unroll
        for (int k = 0; k < i; ++k) acc -= mat(const_cast<T*>(A), ld, k, i) * v[k];
        v[i] = acc * mat(const_cast<T*>(A), ld, i, i);
    }
#pragma unroll
    for (int i = NV - 2; i >= 0; --i) {
        T acc = v[i];
#pragma unroll
        for (int k = i + 1; k < NV; ++k) acc -= mat(const_cast<T*>(A), ld, k, i) * v[k];
        v[i] = acc;
    }
#pragma unroll
    for (int k = NV - 1; k >= 0; --k) {
        const int p = pv[(int64_t)k * ld];
        if (p != k) {
            const T tmp = v[k];
            v[k] = v[p];
            v[p] = tmp;
        }
    }
}

// J_s x = r for every scenario (one thread each), NRHS right-hand sides.  rhs k is the
// row vector r[k] (or, when r[k] is null, b = dc/dd: -u_max pi d / 2 in every hydraulic
// row).  Solutions are written to out[k] in primal layout (without the d entry).
template <class T, int NRHS>
__global__ void __launch_bounds__(64) solve_kernel(const Params P, int S, int64_t ld, const double* __restrict__ jac,
                                                   const T* __restrict__ LU, const unsigned char* __restrict__ piv,
                                                   const T* __restrict__ G, const double* x_d,
                                                   const double* r0, const double* r1, double* o0, double* o1) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    const double* rr[2] = {r0, r1};
    double* oo[2] = {o0, o1};
    const double bval = -P.u_max * M_PI * 0.5 * x_d[0];
    // forward: w_n = r_n - C_n y_{n-1},  y_n = At_n^{-1} w_n
    for (int n = 0; n < N_STAGES; ++n) {
        const int t = stage_type(n);
        const int base = c_segJ[n];
        const T* A = LU + (int64_t)n * NV * NV * ld + s;
        const unsigned char* pv = piv + (int64_t)n * NV * ld + s;
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
            T w[NV];
            if (rr[k]) {
#pragma unroll
                for (int r = 0; r < NR; ++r) w[r] = (T)rr[k][(int64_t)(NR * n + r) * ld + s];
            } else {
#pragma unroll
                for (int r = 0; r < NR; ++r) w[r] = (r == R_H) ? (T)bval : T(0);
            }
            if (n > 0) {
                for (int q = 0; q < c_nblw[t]; ++q) {
                    const Ent e = c_blw[t][q];
                    w[e.r] -= (T)jac[(int64_t)(base + e.slot) * ld + s] *
                              (T)oo[k][(int64_t)(NV * (n - 1) + blw_var(e.c)) * ld + s];
                }
            }
            lu_apply(A, pv, ld, w);
#pragma unroll
            for (int j = 0; j < NV; ++j) oo[k][(int64_t)(NV * n + j) * ld + s] = (double)w[j];
        }
    }
    // backward: x_n = y_n - G_n x_{n+1}
    for (int n = N_STAGES - 2; n >= 0; --n) {
        const T* Gn = G + (int64_t)n * NV * NABV * ld + s;
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
            T xa[NABV];
#pragma unroll
            for (int a = 0; a < NABV; ++a) xa[a] = (T)oo[k][(int64_t)(NV * (n + 1) + abv_var(a)) * ld + s];
#pragma unroll
            for (int i = 0; i < NV; ++i) {
                T acc = (T)oo[k][(int64_t)(NV * n + i) * ld + s];
#pragma unroll
                for (int a = 0; a < NABV; ++a) acc -= Gn[(int64_t)(i * NABV + a) * ld] * xa[a];
                oo[k][(int64_t)(NV * n + i) * ld + s] = (double)acc;
            }
        }
    }
}

// J_s^T v = g for every scenario (one thread each); g, out: primal layout (no d).
template <class T>
__global__ void __launch_bounds__(64) solve_t_kernel(int S, int64_t ld, const double* __restrict__ jac,
                                                     const T* __restrict__ LU, const unsigned char* __restrict__ piv,
                                                     const double* __restrict__ g, double* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    // forward (U^T of the block LU): u_n = At_n^{-T} (g_n - B_{n-1}^T u_{n-1})
    for (int n = 0; n < N_STAGES; ++n) {
        const T* A = LU + (int64_t)n * NV * NV * ld + s;
        const unsigned char* pv = piv + (int64_t)n * NV * ld + s;
        T w[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) w[j] = (T)g[(int64_t)(NV * n + j) * ld + s];
        if (n > 0) {
            const int tb = stage_type(n - 1), bb = c_segJ[n - 1];
            for (int q = 0; q < c_nabv[tb]; ++q) {
                const Ent e = c_abv[tb][q];
                w[abv_var(e.c)] -= (T)jac[(int64_t)(bb + e.slot) * ld + s] *
                                   (T)out[(int64_t)(NR * (n - 1) + e.r) * ld + s];
            }
        }
        lu_apply_t(A, pv, ld, w);
#pragma unroll
        for (int j = 0; j < NV; ++j) out[(int64_t)(NR * n + j) * ld + s] = (double)w[j];
    }
    // backward (L^T): v_n = u_n - At_n^{-T} C_{n+1}^T v_{n+1}
    for (int n = N_STAGES - 2; n >= 0; --n) {
        const T* A = LU + (int64_t)n * NV * NV * ld + s;
        const unsigned char* pv = piv + (int64_t)n * NV * ld + s;
        const int ta = stage_type(n + 1), ba = c_segJ[n + 1];
        T w[NV];
#pragma unroll
        for (int j = 0; j < NV; ++j) w[j] = T(0);
        for (int q = 0; q < c_nblw[ta]; ++q) {
            const Ent e = c_blw[ta][q];
            w[blw_var(e.c)] += (T)jac[(int64_t)(ba + e.slot) * ld + s] *
                               (T)out[(int64_t)(NR * (n + 1) + e.r) * ld + s];
        }
        lu_apply_t(A, pv, ld, w);
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const int64_t o = (int64_t)(NR * n + j) * ld + s;
            out[o] = (double)((T)out[o] - w[j]);
        }
    }
}

}  // namespace absorber
