// kernels_warp.cuh -- warp-cooperative stage-block LU and block solves (A4, A6).
//
// One warp per scenario.  factor_warp_kernel keeps each 22 x 22 stage block in shared
// memory while the warp works on it: pivot search with rows on lanes, the trailing
// update with columns on lanes (each lane keeps its pivot-row entry in a register and
// walks the rows), the super-diagonal block B_n appended as 11 extra columns so that the
// elimination yields L^-1 P B_n, then U G_n = L^-1 P B_n by backward substitution.
// factor_gj_kernel (FP32) forms the stage-block inverse instead, by Gauss-Jordan exchange
// with row i of the block in lane i's registers.
// Vectors of the solves live one entry per lane; broadcasts are warp shuffles.
//
// Factor storage is per scenario and contiguous (internal layout, not part of the C
// ABI): LU[s][n][22][22], G[s][n][22][11] and the row order piv[s][n][22][2] (see
// PIV_BYTES), so every warp access to the factors is coalesced.  The reciprocal of each
// pivot is kept on U's diagonal.
#pragma once

#include "kernels.cuh"

namespace absorber {

constexpr int NCA = NV + NABV;    // augmented columns [A_n | B_n]
constexpr int PADA = NCA + 1;     // shared-memory row stride of the augmented block
constexpr int PADL = NV + 1;      // shared-memory row stride of a staged LU block
constexpr int WPB_F = 4;          // default warps (scenarios) per block, factor
constexpr int WPB_S = 4;          // default warps (scenarios) per block, solves

// static shared memory of the factor kernel with W warps per block (must stay <= 48 KB)
template <class T, int W>
constexpr bool factor_fits() {
    return (size_t)W * (NV * PADA + NV * NABV) * sizeof(T) + sizeof(LaneTables) <= 48 * 1024;
}

__host__ __device__ constexpr int64_t lu_off(int64_t s, int n) { return (s * N_STAGES + n) * (int64_t)(NV * NV); }
__host__ __device__ constexpr int64_t g_off(int64_t s, int n) { return (s * N_STAGES + n) * (int64_t)(NV * NABV); }
// row order of a factored stage block: (perm[i], ipos[i]) byte pairs for i < 22, perm[i]
// the block row at position i of P A = L U and ipos[j] the position of block row j
constexpr int PIV_BYTES = 2 * NV;
__host__ __device__ constexpr int64_t pv_off(int64_t s, int n) { return (s * N_STAGES + n) * (int64_t)PIV_BYTES; }

template <class T>
__device__ inline T shfl(T v, int src) {
    return __shfl_sync(0xffffffffu, v, src);
}

// |a| as an unsigned integer with the same ordering as |a| itself (IEEE layout with the
// sign cleared): pivot searches and block maxima compare these on the integer pipe,
// keeping them off the floating-point pipe (slow for FP64 on this part)
__device__ inline unsigned long long abs_key(double a) {
    return (unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull;
}
__device__ inline unsigned long long abs_key(float a) {
    return (unsigned long long)(__float_as_uint(a) & 0x7fffffffu);
}
__device__ inline double key_value(unsigned long long k, double) { return __longlong_as_double((long long)k); }
__device__ inline float key_value(unsigned long long k, float) { return __uint_as_float((unsigned)k); }

// warp maximum of 64-bit keys with the hardware 32-bit warp reduction: the high words
// first, then the low words among the lanes holding the highest high word
__device__ inline unsigned long long warp_max_key(unsigned long long key) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mh = __reduce_max_sync(0xffffffffu, hi);
    const unsigned ml = __reduce_max_sync(0xffffffffu, hi == mh ? lo : 0u);
    return ((unsigned long long)mh << 32) | ml;
}

// pivot row: the lowest candidate lane whose key is the largest among the candidates
// (every lane takes part; candidates have cand = true)
__device__ inline int warp_argmax_key(unsigned long long key, bool cand) {
    const unsigned long long m = warp_max_key(cand ? key : 0ull);
    const unsigned won = __ballot_sync(0xffffffffu, cand && key == m);
    return __ffs((int)won) - 1;
}

// FP32 pivot key: |a| with its 5 lowest mantissa bits replaced by 31 - position, so that
// one warp maximum both finds the pivot and breaks ties: the candidate of largest |a| up
// to a relative 2^-18, the lowest position among those (threshold partial pivoting; an
// all-zero column takes its lowest position, a NaN always wins)
__device__ __forceinline__ unsigned pivot_key32(float a, int pos) {
    return (__float_as_uint(a) & 0x7fffffe0u) | (unsigned)(31 - pos);
}
__device__ __forceinline__ int key_position(unsigned key) { return 31 - (int)(key & 31u); }

// reciprocal: FP32 seed refined by two Newton steps r <- r (2 - a r) in T (|a| in the
// normal FP32 range; exact division otherwise)
__device__ inline double recip(double a) {
    const double m = fabs(a);
    if (m > 1e-30 && m < 1e30) {
        double r = (double)(1.0f / (float)a);
        r = r * fma(-a, r, 2.0);
        r = r * fma(-a, r, 2.0);
        return r;
    }
    return 1.0 / a;
}
__device__ inline float recip(float a) { return 1.0f / a; }

// x - a b with one rounding (the factor variants must round identically)
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// the coefficients of a stage-coupling table (<= 32 entries) for scenario s, entry q on
// lane q: one parallel load instead of a dependent load per entry inside the
// sequential coupling loops
template <class T>
__device__ inline T load_coupling(const Ent* tab, int cnt, int base, const double* __restrict__ jac, int64_t ld,
                                  int s, int lane) {
    return lane < cnt ? (T)jac[(int64_t)(base + tab[lane].slot) * ld + s] : T(0);
}

// a stage's LU block and row order fetched into registers ahead of use (the next
// stage's loads overlap the current stage's work), then committed: the block to shared
// memory, lane i's (perm[i], ipos[i]) to registers (lanes >= 22: i itself)
constexpr int LU_PER_LANE = (NV * NV + 31) / 32;
template <class T>
struct LUPrefetch {
    T v[LU_PER_LANE];
    uchar2 p;
    __device__ inline void fetch(const T* __restrict__ LU, const unsigned char* __restrict__ piv, int64_t s, int n,
                                 int lane) {
        const T* src = LU + lu_off(s, n);
#pragma unroll
        for (int i = 0; i < LU_PER_LANE; ++i) {
            const int e = lane + 32 * i;
            v[i] = e < NV * NV ? src[e] : T(0);
        }
        p = lane < NV ? reinterpret_cast<const uchar2*>(piv + pv_off(s, n))[lane]
                      : make_uchar2((unsigned char)lane, (unsigned char)lane);
    }
    __device__ inline void commit(T (*A)[PADL], int& perm, int& ipos, int lane) const {
#pragma unroll
        for (int i = 0; i < LU_PER_LANE; ++i) {
            const int e = lane + 32 * i;
            if (e < NV * NV) A[e / NV][e % NV] = v[i];
        }
        perm = p.x;
        ipos = p.y;
    }
};

// the per-lane stage tables, copied once per block into shared memory (every thread of
// the block takes part; call before any warp leaves)
__device__ inline void stage_lane_tables(LaneTables& lt) {
    const int4* src = reinterpret_cast<const int4*>(&g_lt);
    int4* dst = reinterpret_cast<int4*>(&lt);
    constexpr int NW = (int)(sizeof(LaneTables) / sizeof(int4));
    for (int i = threadIdx.x; i < NW; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
}

constexpr int OWN_PER_LANE = MAXOWN / 32, ABV_PER_LANE = MAXABV / 32;

// the Jacobian values of stage n's own and super-diagonal entries that lane `lane`
// scatters (entries lane, lane + 32, ...), every load issued before the first use
struct StageLoads {
    Ent eo[OWN_PER_LANE];
    double vo[OWN_PER_LANE];
    Ent ea[ABV_PER_LANE];
    double va[ABV_PER_LANE];
    int no, na;
    __device__ inline void fetch(const LaneTables& lt, int n, int64_t ld, int s, int lane,
                                 const double* __restrict__ jac) {
        const int t = stage_type(n);
        const int base = c_segJ[n];
        no = c_nown[t];
        na = n + 1 < N_STAGES ? c_nabv[t] : 0;
#pragma unroll
        for (int i = 0; i < OWN_PER_LANE; ++i) {
            const int k = lane + 32 * i;
            eo[i] = lt.own[t][k < no ? k : 0];
        }
#pragma unroll
        for (int i = 0; i < ABV_PER_LANE; ++i) {
            const int k = lane + 32 * i;
            ea[i] = lt.abv[t][k < na ? k : 0];
        }
#pragma unroll
        for (int i = 0; i < OWN_PER_LANE; ++i)
            vo[i] = lane + 32 * i < no ? jac[(int64_t)(base + eo[i].slot) * ld + s] : 0.0;
#pragma unroll
        for (int i = 0; i < ABV_PER_LANE; ++i)
            va[i] = lane + 32 * i < na ? jac[(int64_t)(base + ea[i].slot) * ld + s] : 0.0;
    }
    // scatter into the augmented block (row stride P, B_n from column NV)
    template <class T, int P>
    __device__ inline void scatter(T* A, int lane) const {
#pragma unroll
        for (int i = 0; i < OWN_PER_LANE; ++i)
            if (lane + 32 * i < no) A[eo[i].r * P + eo[i].c] = (T)vo[i];
#pragma unroll
        for (int i = 0; i < ABV_PER_LANE; ++i)
            if (lane + 32 * i < na) A[ea[i].r * P + NV + ea[i].c] = (T)va[i];
    }
};

// assemble stage n's augmented block [A_n | B_n] of scenario s in shared memory (own
// entries, the super-diagonal coupling B_n, the Schur update A_n -= C_n G_{n-1}) and
// return the threshold below which a pivot marks the block singular
template <class T>
__device__ inline T assemble_stage(int n, int64_t ld, int s, int lane, const double* __restrict__ jac, double pivtol,
                                   const LaneTables& lt, T (*A)[PADA], const T (*Gp)[NABV]) {
    const int t = stage_type(n);
    const int base = c_segJ[n];
    StageLoads L;
    L.fetch(lt, n, ld, s, lane, jac);
    const int nq = n > 0 ? c_nblw[t] : 0;
    const T cvq = load_coupling<T>(lt.blw[t], nq, base, jac, ld, s, lane);
    for (int e = lane; e < NV * NCA; e += 32) A[e / NCA][e % NCA] = T(0);
    __syncwarp();
    L.scatter<T, PADA>(&A[0][0], lane);
    __syncwarp();
    // Schur update with the previous stage: A_n -= C_n G_{n-1}
    for (int k = 0; k < nq; ++k) {
        const Ent e = lt.blw[t][k];
        const T cv = shfl(cvq, k);
        if (lane < NABV) A[e.r][abv_var(lane)] = fma_t(-cv, Gp[blw_var(e.c)][lane], A[e.r][abv_var(lane)]);
        __syncwarp();
    }
    // largest entry of the block (for the singularity test)
    unsigned long long kmax = 0ull;
    for (int e = lane; e < NV * NV; e += 32) {
        const unsigned long long kk = abs_key(A[e / NV][e % NV]);
        kmax = kk > kmax ? kk : kmax;
    }
    kmax = warp_max_key(kmax);
    return (T)pivtol * key_value(kmax, T(0));
}

// mask (optional): only scenarios s with mask[s] != 0 are factored (the FP64 escalation
// of scenarios whose FP32 refinement stalled); the others keep their factors
template <class T, int WPB = WPB_F>
__global__ void __launch_bounds__(32 * WPB) factor_warp_kernel(int S, int64_t ld, const BView b,
                                                                 const double* __restrict__ jac, T* __restrict__ LU,
                                                                 unsigned char* __restrict__ piv, T* __restrict__ G,
                                                                 int* __restrict__ sing, double pivtol,
                                                                 const int* __restrict__ mask = nullptr,
                                                                 const int* __restrict__ skip = nullptr) {
    if (skip && *skip) return;   // the stored factors are those of this Jacobian (every block leaves)
    __shared__ T sA[WPB][NV][PADA];
    __shared__ T sG[WPB][NV][NABV];
    __shared__ LaneTables lt;
    stage_lane_tables(lt);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    // whole warps leave together; no block-level barriers below
    if (live_prob(b, s, S, PS_ACT) < 0) return;
    if (mask && mask[s] == 0) return;
    T(*A)[PADA] = sA[warp];
    T(*Gp)[NABV] = sG[warp];
    int singular = 0;
    for (int n = 0; n < N_STAGES; ++n) {
        const T tiny = assemble_stage<T>(n, ld, s, lane, jac, pivtol, lt, A, Gp);
        const unsigned long long ktiny = abs_key(tiny);
        unsigned char* pv = piv + pv_off(s, n);
        int orig = lane;   // block row now at position lane
        // LU with partial pivoting, row operations on all 33 columns.  FP64: fully unrolled
        // (static shared-memory offsets, independent row updates; measured 3 % faster);
        // FP32: rolled (the unrolled body's size costs more than it gains)
        constexpr int UNR = sizeof(T) == 8 ? NV : 1;
#pragma unroll UNR
        for (int k = 0; k < NV; ++k) {
            // key 0 marks lanes outside the candidate rows.  FP64: exact |value| keys, ties to
            // the lowest row (an exact zero candidate also has key 0: the singular test below
            // catches it); FP32: pivot_key32 (the rule of factor_gj_kernel)
            const bool cand = lane >= k && lane < NV;
            int p;
            if constexpr (sizeof(T) == 4) {
                p = key_position(__reduce_max_sync(0xffffffffu, cand ? pivot_key32(A[lane][k], lane) : 0u));
            } else {
                p = warp_argmax_key(cand ? abs_key(A[lane][k]) : 0ull, cand);
                if (p < 0 || p >= NV) p = k;
            }
            if (p != k) {
                for (int j = lane; j < NCA; j += 32) {
                    const T a = A[k][j];
                    A[k][j] = A[p][j];
                    A[p][j] = a;
                }
                const int ok = __shfl_sync(0xffffffffu, orig, k), op = __shfl_sync(0xffffffffu, orig, p);
                if (lane == k) orig = op;
                if (lane == p) orig = ok;
            }
            __syncwarp();
            T ukk = A[k][k];
            if (!(abs_key(ukk) > ktiny) || ukk != ukk) {
                singular = 1;
                ukk = (ukk < T(0) ? T(-1) : T(1)) * (tiny > T(0) ? tiny : T(1));
            }
            const T inv = recip(ukk);
            if (lane > k && lane < NV) A[lane][k] *= inv;
            __syncwarp();
            const int j = k + 1 + lane;
            if (j < NCA) {
                const T akj = A[k][j];
                constexpr int UNI = sizeof(T) == 8 ? NV : 4;
#pragma unroll UNI
                for (int i = k + 1; i < NV; ++i) A[i][j] = fma_t(-A[i][k], akj, A[i][j]);
            }
            if (lane == 0) A[k][k] = inv;
            __syncwarp();
        }
        // U G = L^-1 P B: lanes 0..21 = (column a = lane % 11, row parity lane / 11)
        if (n + 1 < N_STAGES) {
            const int a = lane % NABV, grp = lane / NABV;
#pragma unroll UNR
            for (int i = NV - 1; i >= 0; --i) {
                const T g = A[i][NV + a] * A[i][i];
                __syncwarp();
                if (grp < 2) {
                    constexpr int UNG = sizeof(T) == 8 ? NV : 4;
#pragma unroll UNG
                    for (int r = grp; r < i; r += 2) A[r][NV + a] = fma_t(-A[r][i], g, A[r][NV + a]);
                    if (grp == 0) A[i][NV + a] = g;
                }
                __syncwarp();
            }
            T* Gn = G + g_off(s, n);
            for (int e = lane; e < NV * NABV; e += 32) {
                const T g = A[e / NABV][NV + e % NABV];
                Gn[e] = g;
                Gp[e / NABV][e % NABV] = g;
            }
        }
        T* Ln = LU + lu_off(s, n);
        for (int e = lane; e < NV * NV; e += 32) Ln[e] = A[e / NV][e % NV];
        if (lane < NV) {
            pv[2 * lane] = (unsigned char)orig;
            pv[2 * orig + 1] = (unsigned char)lane;
        }
        __syncwarp();
    }
    if (lane == 0) sing[s] = singular;
}

// FP32 stage-block inverses (the FP32 path's factorization): Gauss-Jordan elimination
// in place, with partial pivoting, on [A_n | B_n] with rows in registers.  Lane i < 22
// keeps row i (17 float pairs) for the whole elimination; rows are never moved, each lane
// tracks the position its row takes.  Step k exchanges unknown k with the equation of the
// pivot row p (one warp maximum of pivot_key32 over the rows not yet chosen: ties go to
// the lowest position): with inv = 1 / a_pk, the pivot row becomes u_j = -a_pj inv
// (j != k), u_k = inv, and every other row i becomes a_ij + a_ik u_j (j != k),
// a_ik inv (j = k).  After the 22 exchanges the row at position i expresses unknown i:
// its first 22 entries are row i of A_n^-1 with columns in position order (column c: the
// equation of the row at position c) and its last 11 are row i of -G_n.  The block solves
// take the row order (perm, ipos as for the LU factors) to match the columns.
constexpr int NPR = (NCA + 1) / 2;   // float pairs of [A_n | B_n] per row (column 33: padding)
constexpr int NBLWV = 6;             // unknowns of the stage below in a row's coupling (C_n)
constexpr int PADQ = 36;             // assembly row stride (rows 16-byte aligned)
constexpr int UINV = 36;             // broadcast buffer: the pivot's reciprocal

__device__ __forceinline__ float& rv(float2* r, int j) { return (j & 1) ? r[j >> 1].y : r[j >> 1].x; }

// (W <= 4: at least 24 resident warps per SM, 85 registers per thread at most)
template <int WPB = WPB_F>
__global__ void __launch_bounds__(32 * WPB, WPB >= 8 ? 3 : 24 / WPB) factor_gj_kernel(int S, int64_t ld, const BView b,
                                                             const double* __restrict__ jac, float* __restrict__ AI,
                                                             unsigned char* __restrict__ piv, float* __restrict__ G,
                                                             int* __restrict__ sing, double pivtol,
                                                             const int* __restrict__ skip = nullptr) {
    if (skip && *skip) return;   // the stored inverses are those of this Jacobian (every block leaves)
    // per warp: the assembly block (reused as the row-major inverse on the way out), G_n
    // by unknown (the next stage's Schur update reads it), and the broadcast row
    __shared__ __align__(16) float sA[WPB][NV * PADQ];
    __shared__ __align__(16) float sG[WPB][NV * NABV + 2];
    __shared__ __align__(16) float sU[WPB][40];
    __shared__ LaneTables lt;
    stage_lane_tables(lt);
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    if (live_prob(b, s, S, PS_ACT) < 0) return;   // whole warps leave together
    float* A = sA[warp];
    float* Gs = sG[warp];
    float* U = sU[warp];
    const bool rowlane = lane < NV;
    int singular = 0;
#pragma unroll 1
    for (int n = 0; n < N_STAGES; ++n) {
        const int t = stage_type(n);
        const int base = c_segJ[n];
        // assemble: every Jacobian load of the lane first (its scatter entries and its row's
        // entries of C_n), rows zeroed, entries scattered, rows to registers
        StageLoads L;
        L.fetch(lt, n, ld, s, lane, jac);
        int q0 = 0, nb = 0;
        if (n > 0 && rowlane) {
            q0 = lt.blwRp[t][lane];
            nb = lt.blwRp[t][lane + 1] - q0;
        }
        Ent eb[NBLWV];
        double vb[NBLWV];
#pragma unroll
        for (int i = 0; i < NBLWV; ++i) {
            eb[i] = lt.blw[t][i < nb ? q0 + i : 0];
            vb[i] = i < nb ? jac[(int64_t)(base + eb[i].slot) * ld + s] : 0.0;
        }
        if (rowlane) {
#pragma unroll
            for (int q = 0; q < PADQ / 4; ++q) *reinterpret_cast<float4*>(&A[lane * PADQ + 4 * q]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        L.scatter<float, PADQ>(A, lane);
        __syncwarp();
        float2 r2[NPR];
        if (rowlane) {
#pragma unroll
            for (int q = 0; q < NPR / 2; ++q) {
                const float4 a4 = *reinterpret_cast<const float4*>(&A[lane * PADQ + 4 * q]);
                r2[2 * q] = make_float2(a4.x, a4.y);
                r2[2 * q + 1] = make_float2(a4.z, a4.w);
            }
            r2[NPR - 1] = *reinterpret_cast<const float2*>(&A[lane * PADQ + 2 * (NPR - 1)]);
        } else {
#pragma unroll
            for (int m = 0; m < NPR; ++m) r2[m] = make_float2(0.f, 0.f);
        }
        // Schur update with the previous stage, A_n -= C_n G_{n-1}: each row applies its own
        // entries of C_n in table order (at most one per unknown of the stage below)
#pragma unroll
        for (int i = 0; i < NBLWV; ++i) {
            if (i < nb) {
                const float cv = (float)vb[i];
                const float* gr = Gs + blw_var(eb[i].c) * NABV;
#pragma unroll
                for (int a = 0; a < NABV; ++a) rv(r2, abv_var(a)) = fmaf(-cv, gr[a], rv(r2, abv_var(a)));
            }
        }
        // the largest |entry| of the block gives the singularity threshold
        unsigned km = 0u;
#pragma unroll
        for (int j = 0; j < NV; ++j) km = max(km, __float_as_uint(rv(r2, j)) & 0x7fffffffu);
        km = __reduce_max_sync(full, km);
        const float tiny = (float)pivtol * __uint_as_float(km);
        const unsigned ktiny = __float_as_uint(tiny) & 0x7fffffffu;
        int cur = lane;             // position of this lane's row
        bool done = !rowlane;       // row already chosen (lanes >= 22 never take part)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            const float xk = rv(r2, k);
            const unsigned key = done ? 0u : pivot_key32(xk, cur);
            const unsigned mx = __reduce_max_sync(full, key);
            // every lane forms the reciprocal of its candidate while the maximum is found
            // (off the step's dependency chain); operands outside [2^-60, 2^60] are replaced
            // so that no lane takes the division's slow path, and the pivot row recomputes
            // in that case
            const float ax = fabsf(xk);
            const bool easy = ax > 0x1p-60f && ax < 0x1p60f;
            const float sinv = recip(easy ? xk : 1.0f);
            const int pos = key_position(mx);
            const bool isp = !done && key == mx;
            if (cur == k) cur = pos;
            if (isp) {
                cur = k;
                done = true;
                // the pivot row: singular test, reciprocal, u_j = -a_pj inv, u_k = inv, to
                // shared memory
                float ukk = xk;
                float inv = sinv;
                if (!((__float_as_uint(ukk) & 0x7fffffffu) > ktiny) || ukk != ukk) {
                    singular = 1;
                    ukk = (ukk < 0.0f ? -1.0f : 1.0f) * (tiny > 0.0f ? tiny : 1.0f);
                    inv = recip(ukk);
                } else if (!easy) {
                    inv = recip(ukk);
                }
                const float2 niv = make_float2(-inv, -inv);
#pragma unroll
                for (int m = 0; m < NPR; ++m) r2[m] = __fmul2_rn(r2[m], niv);
                rv(r2, k) = inv;
#pragma unroll
                for (int q = 0; q < NPR / 2; ++q)
                    *reinterpret_cast<float4*>(&U[4 * q]) = make_float4(r2[2 * q].x, r2[2 * q].y, r2[2 * q + 1].x,
                                                                        r2[2 * q + 1].y);
                *reinterpret_cast<float2*>(&U[2 * (NPR - 1)]) = r2[NPR - 1];
            }
            __syncwarp();
            if (rowlane && !isp) {
                const float f = rv(r2, k);
                const float2 nf = make_float2(f, f);
#pragma unroll
                for (int q = 0; q < NPR / 2; ++q) {
                    const float4 u4 = *reinterpret_cast<const float4*>(&U[4 * q]);
                    r2[2 * q] = __ffma2_rn(nf, make_float2(u4.x, u4.y), r2[2 * q]);
                    r2[2 * q + 1] = __ffma2_rn(nf, make_float2(u4.z, u4.w), r2[2 * q + 1]);
                }
                r2[NPR - 1] = __ffma2_rn(nf, *reinterpret_cast<const float2*>(&U[2 * (NPR - 1)]), r2[NPR - 1]);
                rv(r2, k) = f * U[k];   // U[k] holds inv
            }
            __syncwarp();
        }
        // rows to shared memory at their positions (G_n = -(the B part)), row order, then
        // coalesced stores
        if (rowlane) {
#pragma unroll
            for (int m = 0; m < NV / 2; ++m) *reinterpret_cast<float2*>(&A[cur * NV + 2 * m]) = r2[m];
            if (n + 1 < N_STAGES) {
#pragma unroll
                for (int a = 0; a < NABV; ++a) Gs[cur * NABV + a] = -rv(r2, NV + a);
            }
            piv[pv_off(s, n) + 2 * cur] = (unsigned char)lane;
            piv[pv_off(s, n) + 2 * lane + 1] = (unsigned char)cur;
        }
        __syncwarp();
        float4* Ln = reinterpret_cast<float4*>(AI + lu_off(s, n));
        for (int e = lane; e < NV * NV / 4; e += 32) Ln[e] = reinterpret_cast<const float4*>(A)[e];
        if (n + 1 < N_STAGES) {
            float2* Gn = reinterpret_cast<float2*>(G + g_off(s, n));
            for (int e = lane; e < NV * NABV / 2; e += 32) Gn[e] = reinterpret_cast<const float2*>(Gs)[e];
        }
        __syncwarp();
    }
    singular = __any_sync(0xffffffffu, singular);
    if (lane == 0) sing[s] = singular;
}

// w <- At^-1 w, lane i holding w_i (lanes >= 22 carry zeros): P w in one shuffle, then
// L forward and U backward (unrolled: the loads of A run ahead of the shuffle chain)
template <class T>
__device__ inline T lu_apply_warp(const T (*A)[PADL], int perm, int lane, T w) {
    w = shfl(w, perm);
#pragma unroll
    for (int k = 0; k < NV - 1; ++k) {
        const T wk = shfl(w, k);
        if (lane > k && lane < NV) w -= A[lane][k] * wk;
    }
#pragma unroll
    for (int k = NV - 1; k >= 0; --k) {
        if (lane == k) w *= A[k][k];
        const T wk = shfl(w, k);
        if (lane < k) w -= A[lane][k] * wk;
    }
    return w;
}

// w <- At^-T w:  U^T forward, L^T backward, then P^T w in one shuffle
template <class T>
__device__ inline T lu_apply_t_warp(const T (*A)[PADL], int ipos, int lane, T w) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        if (lane == k) w *= A[k][k];
        const T wk = shfl(w, k);
        if (lane > k && lane < NV) w -= A[k][lane] * wk;
    }
#pragma unroll
    for (int k = NV - 1; k > 0; --k) {
        const T wk = shfl(w, k);
        if (lane < k) w -= A[k][lane] * wk;
    }
    return shfl(w, ipos);
}

// FP32 path (factor_gj_kernel): lane i's row i of the stage-block inverse, fetched a
// stage ahead; the block solve y = A_n^-1 w is y_i = sum_j a_ij w_j (two interleaved
// accumulations: even and odd j)
// FP32 path (factor_gj_kernel): lane i's row i of the stage-block inverse M (columns in
// position order) and its row-order pair, fetched a stage ahead.  The block solve
// y = A_n^-1 w is y_i = sum_c M_ic w_perm[c] (two interleaved accumulations: even and odd c)
constexpr int NPI = NV / 2;
struct InvRowFetch {
    float2 a[NPI];
    uchar2 p;
    __device__ inline void fetch(const float* __restrict__ AI, const unsigned char* __restrict__ piv, int64_t s,
                                 int n, int lane) {
        const float2* src = reinterpret_cast<const float2*>(AI + lu_off(s, n) + (lane < NV ? lane : 0) * NV);
#pragma unroll
        for (int m = 0; m < NPI; ++m) a[m] = lane < NV ? src[m] : make_float2(0.f, 0.f);
        p = lane < NV ? reinterpret_cast<const uchar2*>(piv + pv_off(s, n))[lane]
                      : make_uchar2((unsigned char)lane, (unsigned char)lane);
    }
    __device__ inline float apply(float w) const {
        w = shfl(w, (int)p.x);
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int m = 0; m < NPI; ++m) {
            e = fmaf(a[m].x, shfl(w, 2 * m), e);
            o = fmaf(a[m].y, shfl(w, 2 * m + 1), o);
        }
        return e + o;
    }
};
// ... and lane c's column c, for the transposed block solve: u_c = sum_i M_ic w_i, then
// v_j = u_ipos[j]
struct InvColFetch {
    float c[NV];
    uchar2 p;
    __device__ inline void fetch(const float* __restrict__ AI, const unsigned char* __restrict__ piv, int64_t s,
                                 int n, int lane) {
        const float* src = AI + lu_off(s, n) + (lane < NV ? lane : 0);
#pragma unroll
        for (int i = 0; i < NV; ++i) c[i] = lane < NV ? src[i * NV] : 0.f;
        p = lane < NV ? reinterpret_cast<const uchar2*>(piv + pv_off(s, n))[lane]
                      : make_uchar2((unsigned char)lane, (unsigned char)lane);
    }
    __device__ inline float apply(float w) const {
        float e = 0.f, o = 0.f;
#pragma unroll
        for (int i = 0; i < NV; i += 2) {
            e = fmaf(c[i], shfl(w, i), e);
            o = fmaf(c[i + 1], shfl(w, i + 1), o);
        }
        return shfl(e + o, (int)p.y);
    }
};

// the coupling of stage n to the stage below (C_n: entry q on lane q), fetched a stage
// ahead of use: the entry's Jacobian value (kept in double until used, so that the load
// does not stall the fetch), the stage-below unknown it multiplies (row solves) or its
// row (transposed solves), and lane j's group of entries -- those of row j (row solves)
// or those feeding stage-below unknown j (transposed solves), in table order
constexpr int NBLWC = 8;   // entries feeding one stage-below unknown, at most
struct CouplingFetch {
    double cv;
    int src, q0, nb;
    unsigned char qi[NBLWC];   // transposed solves: the group's entry indices
    template <bool TRANS>
    __device__ inline void fetch(int n, int64_t ld, int s, int lane, const double* __restrict__ jac) {
        const int t = stage_type(n), base = c_segJ[n], nq = c_nblw[t];
        const Ent e = g_lt.blw[t][lane < nq ? lane : 0];
        cv = lane < nq ? jac[(int64_t)(base + e.slot) * ld + s] : 0.0;
        src = lane < nq ? (TRANS ? (int)e.r : blw_var(e.c)) : 0;
        const short* ptr = TRANS ? g_lt.blwCp[t] : g_lt.blwRp[t];
        q0 = lane < NV ? ptr[lane] : 0;
        nb = lane < NV ? ptr[lane + 1] - q0 : 0;
        if (TRANS) {
#pragma unroll
            for (int i = 0; i < NBLWC; ++i) qi[i] = g_lt.blwQ[t][i < nb ? q0 + i : 0];
        }
    }
};

// J_s x = r (NRHS right-hand sides; a null r[k] means b = dc/dtheta_bsec, the border
// column of design entry bsec: nonzero in the hydraulic rows of that section's stages),
// one warp per scenario.
// INV (FP32 only): LU holds the stage-block inverses of factor_gj_kernel and each block
// solve is a matrix-vector product; otherwise LU factors and row order.
// the block solves of scenario s (problem pr) by its warp; A: the warp's shared-memory
// staging block for LU factors (unused with INV)
template <class T, int NRHS, bool INV>
__device__ __forceinline__ void solve_warp_body(const Params& P, int s, int pr, int lane, int64_t ld,
                                                const double* __restrict__ jac, const T* __restrict__ LU,
                                                const unsigned char* __restrict__ piv, const T* __restrict__ G,
                                                const double* x, const double* r0, const double* r1, double* o0,
                                                double* o1, T (*A)[PADL], int NP, int bsec) {
    static_assert(!INV || sizeof(T) == 4, "stage-block inverses are FP32");
    int perm = lane, ipos = lane;
    const double* rr[2] = {r0, r1};
    double* oo[2] = {o0, o1};
    // b = dc/dtheta of the problem's design entry bsec
    const T bval = (T)(-P.u_max * M_PI * 0.5 * x[(int64_t)NSC * ld + (int64_t)bsec * NP + pr]);
    const bool row = lane < NV;
    T y[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) y[k] = T(0);
    LUPrefetch<T> pre;
    InvRowFetch ipre;
    if constexpr (INV) ipre.fetch((const float*)LU, piv, s, 0, lane);
    else pre.fetch(LU, piv, s, 0, lane);
    double rnext[NRHS];
#pragma unroll
    for (int k = 0; k < NRHS; ++k) rnext[k] = (rr[k] && row) ? rr[k][(int64_t)lane * ld + s] : 0.0;
    CouplingFetch cnext;
    cnext.fetch<false>(1, ld, s, lane, jac);
    // forward: w_n = r_n - C_n y_{n-1},  y_n = At_n^-1 w_n
    for (int n = 0; n < N_STAGES; ++n) {
        InvRowFetch icur;
        if constexpr (INV) icur = ipre;
        else pre.commit(A, perm, ipos, lane);
        const CouplingFetch cc = cnext;
        T w[NRHS];
#pragma unroll
        for (int k = 0; k < NRHS; ++k)
            w[k] = rr[k] ? (T)rnext[k] : ((lane == R_H && stage_sec(n, P.nsec) == bsec) ? bval : T(0));
        if (n + 1 < N_STAGES) {
            if constexpr (INV) ipre.fetch((const float*)LU, piv, s, n + 1, lane);
            else pre.fetch(LU, piv, s, n + 1, lane);
#pragma unroll
            for (int k = 0; k < NRHS; ++k)
                rnext[k] = (rr[k] && row) ? rr[k][(int64_t)(NR * (n + 1) + lane) * ld + s] : 0.0;
            cnext.fetch<false>(n + 1, ld, s, lane, jac);
        }
        if (n > 0) {
            // products of C_n's entries (entry q on lane q) with y_{n-1}, then subtracted in
            // each row in entry order
            const T cv = (T)cc.cv;
#pragma unroll
            for (int k = 0; k < NRHS; ++k) {
                const T pq = cv * shfl(y[k], cc.src);
#pragma unroll
                for (int i = 0; i < NBLWV; ++i) {
                    const T pp = shfl(pq, (cc.q0 + i) & 31);
                    if (i < cc.nb) w[k] -= pp;
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
            if constexpr (INV) y[k] = icur.apply(w[k]);
            else y[k] = lu_apply_warp<T>(A, perm, lane, w[k]);
            if (row) oo[k][(int64_t)(NV * n + lane) * ld + s] = (double)y[k];
        }
        __syncwarp();
    }
    // backward: x_n = y_n - G_n x_{n+1}   (y currently holds x_9 = y_9); the forward
    // values y_n and G_n of the next stage down are fetched one stage ahead
    T gnext[NABV];
    T ynext[NRHS];
    auto fetch_back = [&](int n) {
        const T* Gn = G + g_off(s, n);
#pragma unroll
        for (int a = 0; a < NABV; ++a) gnext[a] = row ? Gn[lane * NABV + a] : T(0);
#pragma unroll
        for (int k = 0; k < NRHS; ++k) ynext[k] = row ? (T)oo[k][(int64_t)(NV * n + lane) * ld + s] : T(0);
    };
    fetch_back(N_STAGES - 2);
    for (int n = N_STAGES - 2; n >= 0; --n) {
        T gc[NABV], yc[NRHS];
#pragma unroll
        for (int a = 0; a < NABV; ++a) gc[a] = gnext[a];
#pragma unroll
        for (int k = 0; k < NRHS; ++k) yc[k] = ynext[k];
        if (n > 0) fetch_back(n - 1);
#pragma unroll
        for (int k = 0; k < NRHS; ++k) {
            T acc = yc[k];
#pragma unroll
            for (int a = 0; a < NABV; ++a) {
                const T xa = shfl(y[k], abv_var(a));
                if (row) acc -= gc[a] * xa;
            }
            y[k] = acc;
            if (row) oo[k][(int64_t)(NV * n + lane) * ld + s] = (double)acc;
        }
    }
}

template <class T, int NRHS, int WPB = WPB_S, bool INV = false>
__global__ void __launch_bounds__(32 * WPB) solve_warp_kernel(const Params P, int S, int64_t ld, const BView b,
                                                                const double* __restrict__ jac, const T* __restrict__ LU,
                                                                const unsigned char* __restrict__ piv,
                                                                const T* __restrict__ G, const double* x,
                                                                const double* r0, const double* r1, double* o0,
                                                                double* o1, int bsec = 0) {
    __shared__ T sL[INV ? 1 : WPB][NV][PADL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    solve_warp_body<T, NRHS, INV>(P, s, pr, lane, ld, jac, LU, piv, G, x, r0, r1, o0, o1, sL[INV ? 0 : warp], b.NP,
                                  bsec);
}

// the same with factors of mixed precision: scenarios with esc[s] != 0 use their FP64 LU
// factors (escalated), the others their FP32 stage-block inverses
template <int NRHS, int WPB = WPB_S>
__global__ void __launch_bounds__(32 * WPB) solve_mixed_kernel(const Params P, int S, int64_t ld, const BView b,
                                                                 const double* __restrict__ jac,
                                                                 const float* __restrict__ AI,
                                                                 const double* __restrict__ LU,
                                                                 const unsigned char* __restrict__ piv,
                                                                 const float* __restrict__ G32,
                                                                 const double* __restrict__ G64,
                                                                 const int* __restrict__ esc, const double* x,
                                                                 const double* r0, const double* r1, double* o0,
                                                                 double* o1, int bsec = 0) {
    __shared__ double sL[WPB][NV][PADL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    const int pr = live_prob(b, s, S, PS_ACT);
    if (pr < 0) return;
    if (esc[s])
        solve_warp_body<double, NRHS, false>(P, s, pr, lane, ld, jac, LU, piv, G64, x, r0, r1, o0, o1, sL[warp], b.NP,
                                             bsec);
    else
        solve_warp_body<float, NRHS, true>(P, s, pr, lane, ld, jac, AI, piv, G32, x, r0, r1, o0, o1, nullptr, b.NP,
                                           bsec);
}

// stage unknown j -> its index among the 11 stream-from-above unknowns (-1: none)
__host__ __device__ constexpr int abv_index(int j) { return j < 9 ? j : (j == LL ? 9 : (j == LT ? 10 : -1)); }

// J_s^T v = g, one warp per scenario; g in primal layout (no d), out in row layout.
// With the block LU J = L U (L: diagonal blocks At_n, sub-diagonal C_n; U: identity
// diagonal, super-diagonal G_n = At_n^-1 B_n), J^T = U^T L^T:
//   forward   w_0 = g_0,  w_{n+1} = g_{n+1} - G_n^T w_n   (into stage n+1's 11 unknowns
//             that stage n reads: products with the stored G blocks, no block solve)
//   backward  v_9 = At_9^-T w_9,  v_n = At_n^-T (w_n - C_{n+1}^T v_{n+1})
// one transposed block solve per stage.
// INV (FP32 only): LU holds the stage-block inverses (see solve_warp_kernel).
template <class T, bool INV>
__device__ __forceinline__ void solve_t_warp_body(int s, int lane, int64_t ld, const double* __restrict__ jac,
                                                  const T* __restrict__ LU, const unsigned char* __restrict__ piv,
                                                  const T* __restrict__ G, const double* __restrict__ g, double* out,
                                                  T (*A)[PADL]) {
    static_assert(!INV || sizeof(T) == 4, "stage-block inverses are FP32");
    int perm = lane, ipos = lane;
    const bool row = lane < NV;
    const int my_abv = abv_index(lane);   // lane j takes the product of column abv_index(j)
    // forward sweep with the G blocks (fetched one stage ahead); w_n kept in out
    T w = row ? (T)g[(int64_t)lane * ld + s] : T(0);
    if (row) out[(int64_t)lane * ld + s] = (double)w;
    T gn[NV];
    auto fetch_g = [&](int n) {
        const T* Gn = G + g_off(s, n);
#pragma unroll
        for (int i = 0; i < NV; ++i) gn[i] = lane < NABV ? Gn[i * NABV + lane] : T(0);
    };
    fetch_g(0);
    for (int n = 1; n < N_STAGES; ++n) {
        T gc[NV];
#pragma unroll
        for (int i = 0; i < NV; ++i) gc[i] = gn[i];
        if (n + 1 < N_STAGES) fetch_g(n);
        const T gnext = row ? (T)g[(int64_t)(NV * n + lane) * ld + s] : T(0);
        // lane a < 11: (G_{n-1}^T w_{n-1})_a = sum_i G_{n-1}[i][a] w_{n-1,i}
        T acc = T(0);
#pragma unroll
        for (int i = 0; i < NV; ++i) acc += gc[i] * shfl(w, i);
        const T t = shfl(acc, my_abv >= 0 ? my_abv : 0);
        w = gnext - (my_abv >= 0 ? t : T(0));
        if (row) out[(int64_t)(NV * n + lane) * ld + s] = (double)w;
    }
    // backward sweep: one transposed block solve per stage
    LUPrefetch<T> pre;
    InvColFetch ipre;
    if constexpr (INV) ipre.fetch((const float*)LU, piv, s, N_STAGES - 1, lane);
    else pre.fetch(LU, piv, s, N_STAGES - 1, lane);
    double rnext = row ? out[(int64_t)(NV * (N_STAGES - 1) + lane) * ld + s] : 0.0;
    CouplingFetch cnext;
    cnext.fetch<true>(N_STAGES - 1, ld, s, lane, jac);
    T v = T(0);
    for (int n = N_STAGES - 1; n >= 0; --n) {
        InvColFetch icur;
        if constexpr (INV) icur = ipre;
        else pre.commit(A, perm, ipos, lane);
        T rhs = (T)rnext;
        const CouplingFetch cc = cnext;
        if (n > 0) {
            if constexpr (INV) ipre.fetch((const float*)LU, piv, s, n - 1, lane);
            else pre.fetch(LU, piv, s, n - 1, lane);
            rnext = row ? out[(int64_t)(NV * (n - 1) + lane) * ld + s] : 0.0;
            cnext.fetch<true>(n, ld, s, lane, jac);
        }
        if (n + 1 < N_STAGES) {
            // C_{n+1}^T v_{n+1}: entry q's product (lane q) subtracted from the stage-n
            // unknown it multiplies, each unknown's entries in table order
            const T pq = (T)cc.cv * shfl(v, cc.src);
#pragma unroll
            for (int i = 0; i < NBLWC; ++i) {
                const T pp = shfl(pq, cc.qi[i]);
                if (i < cc.nb) rhs -= pp;
            }
        }
        __syncwarp();
        if constexpr (INV) v = icur.apply(rhs);
        else v = lu_apply_t_warp<T>(A, ipos, lane, rhs);
        if (row) out[(int64_t)(NR * n + lane) * ld + s] = (double)v;
        __syncwarp();
    }
}

template <class T, int WPB = WPB_S, bool INV = false>
__global__ void __launch_bounds__(32 * WPB) solve_t_warp_kernel(int S, int64_t ld, const BView b,
                                                                const double* __restrict__ jac,
                                                                const T* __restrict__ LU,
                                                                const unsigned char* __restrict__ piv,
                                                                const T* __restrict__ G,
                                                                const double* __restrict__ g, double* out) {
    __shared__ T sL[INV ? 1 : WPB][NV][PADL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    if (live_prob(b, s, S, PS_ACT) < 0) return;
    solve_t_warp_body<T, INV>(s, lane, ld, jac, LU, piv, G, g, out, sL[INV ? 0 : warp]);
}

// mixed precision (see solve_mixed_kernel)
template <int WPB = WPB_S>
__global__ void __launch_bounds__(32 * WPB) solve_t_mixed_kernel(int S, int64_t ld, const BView b,
                                                                   const double* __restrict__ jac,
                                                                   const float* __restrict__ AI,
                                                                   const double* __restrict__ LU,
                                                                   const unsigned char* __restrict__ piv,
                                                                   const float* __restrict__ G32,
                                                                   const double* __restrict__ G64,
                                                                   const int* __restrict__ esc,
                                                                   const double* __restrict__ g, double* out) {
    __shared__ double sL[WPB][NV][PADL];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    if (live_prob(b, s, S, PS_ACT) < 0) return;
    if (esc[s]) solve_t_warp_body<double, false>(s, lane, ld, jac, LU, piv, G64, g, out, sL[warp]);
    else solve_t_warp_body<float, true>(s, lane, ld, jac, AI, piv, G32, g, out, nullptr);
}

}  // namespace absorber
