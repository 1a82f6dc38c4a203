// kernels_ldl.cuh -- regularised symmetric indefinite factorization of the scenario
// blocks (included once, by absorber_lib.cu).
//
// The scenario block of the primal-dual matrix with both regularisations of Wachter &
// Biegler (2006, Eq. (13) and Section 3.1),
//     K_s = [ W_s + Sigma_s + dw I , J_s^T ; J_s , -dc I ],
// is ordered stage by stage, each stage's 22 unknowns followed by its 22 rows, so that
// it is block tridiagonal with 44 x 44 blocks: diagonal blocks K_nn and coupling blocks
// E_n = K_{n+1,n} (the rows of stage n+1 against the unknowns of stage n, J_{n+1,n}, and
// the unknowns of stage n+1 against the rows of stage n, J_{n,n+1}^T).  The block LDL^T
// recurrence in stage order
//     Dt_0 = K_00,   Dt_n = K_nn - E_{n-1} Dt_{n-1}^-1 E_{n-1}^T,
// factors every Dt_n by the Bunch-Kaufman partial pivoting rule (symmetric interchanges,
// 1 x 1 and 2 x 2 pivots; Bunch & Kaufman 1977, alpha = (1 + sqrt 17) / 8); by
// Sylvester's law the inertia of K_s is the sum of the inertias of the pivot blocks.
// Each Dt_n is stored as its explicit inverse (from the factors) for the block solves.
// Unlike the block LU of J_s this needs no square nonsingular J_s: it is the
// factorization for dc > 0 (Algorithm IC's branch for a singular Jacobian) and for
// solves that must count the inertia of every scenario block.  One warp per scenario,
// FP64, the working blocks in dynamic shared memory.
#pragma once

#include "kernels.cuh"

namespace absorber {

constexpr int NB = NV + NR;                        // unknowns of a stage block of K_s
constexpr int LDP = NB + 1;                        // shared-memory row stride
constexpr int LDL_BUF = NB * LDP;                  // doubles per working block
constexpr int64_t LDL_BLOCK = (int64_t)NB * NB;    // doubles per stored inverse
// factor: W (the block being factored), Dinv (the previous stage's inverse, then this
// stage's), E (coupling), T (products, inverse columns); dd, od (pivot blocks); perm, blk
constexpr size_t LDL_FACTOR_SMEM = sizeof(double) * (4 * LDL_BUF + 2 * NB) + sizeof(int) * 2 * NB;
// solve: the inverse, the coupling, the ten stage vectors and one work vector
constexpr size_t LDL_SOLVE_SMEM = sizeof(double) * (2 * LDL_BUF + N_STAGES * NB + NB);

__device__ inline int64_t ldl_off(int s, int n) { return ((int64_t)s * N_STAGES + n) * LDL_BLOCK; }

__device__ inline double warp_max_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// the diagonal block K_nn: [W_nn + Sigma_n + dw I, J_nn^T; J_nn, -dc I] (W omitted when
// use_w is false)
__device__ inline void ldl_assemble_diag(double* W, int64_t ld, int s, int n, const double* __restrict__ jac,
                                         const double* __restrict__ hes, const double* __restrict__ sig, bool use_w,
                                         double dw, double dc, int lane) {
    for (int e = lane; e < LDL_BUF; e += 32) W[e] = 0.0;
    __syncwarp();
    const int t = stage_type(n);
    if (use_w)
        for (int k = lane; k < NHS; k += 32) {
            const Ent e = c_hes[k];
            const double v = hes[(int64_t)(NHS * n + e.slot) * ld + s];
            W[e.r * LDP + e.c] = v;
            W[e.c * LDP + e.r] = v;
        }
    const int base = c_segJ[n];
    for (int k = lane; k < c_nown[t]; k += 32) {
        const Ent e = c_own[t][k];
        const double v = jac[(int64_t)(base + e.slot) * ld + s];
        W[(NV + e.r) * LDP + e.c] = v;
        W[e.c * LDP + NV + e.r] = v;
    }
    __syncwarp();
    if (lane < NV) {
        W[lane * LDP + lane] += sig[(int64_t)(NV * n + lane) * ld + s] + dw;
        W[(NV + lane) * LDP + NV + lane] = -dc;
    }
    __syncwarp();
}

// the coupling block E_{n-1} = K_{n,n-1} (n >= 1): rows of stage n on the unknowns of
// stage n-1 (its stream from below) and, transposed, rows of stage n-1 on the unknowns of
// stage n (their stream from above)
__device__ inline void ldl_assemble_coupling(double* E, int64_t ld, int s, int n, const double* __restrict__ jac,
                                             int lane) {
    for (int e = lane; e < LDL_BUF; e += 32) E[e] = 0.0;
    __syncwarp();
    const int t = stage_type(n), tb = stage_type(n - 1);
    for (int k = lane; k < c_nblw[t]; k += 32) {
        const Ent e = c_blw[t][k];
        E[(NV + e.r) * LDP + blw_var(e.c)] = jac[(int64_t)(c_segJ[n] + e.slot) * ld + s];
    }
    for (int k = lane; k < c_nabv[tb]; k += 32) {
        const Ent e = c_abv[tb][k];
        E[abv_var(e.c) * LDP + NV + e.r] = jac[(int64_t)(c_segJ[n - 1] + e.slot) * ld + s];
    }
    __syncwarp();
}

// Bunch-Kaufman factorization of the symmetric block W (full storage, kept symmetric on
// the trailing part) in place: afterwards W's strict lower triangle holds the unit lower
// factor L (zero inside 2 x 2 pivots), dd / od the pivot blocks (od[k] the off-diagonal
// of a 2 x 2 pivot starting at k), blk[k] 1 (1 x 1 pivot), 2 (a 2 x 2 pivot starts), 0
// (its second index), perm[i] the original index at position i:  P^T W P = L D L^T.
// Pivots of magnitude <= tiny (and exactly singular 2 x 2 blocks) count as zero.
__device__ inline void bk_factor(double* W, double* dd, double* od, int* perm, int* blk, int lane, double tiny,
                                 int& npos, int& nneg, int& nzero) {
    const double alpha = 0.64038820320220756872;   // (1 + sqrt(17)) / 8
    for (int i = lane; i < NB; i += 32) {
        perm[i] = i;
        od[i] = 0.0;
        blk[i] = 1;
    }
    __syncwarp();
    int k = 0;
    while (k < NB) {
        // lambda: the largest |entry| below the diagonal in column k, r its lowest row
        double lam = 0.0;
        int r = NB;
        for (int i = lane; i < NB; i += 32)
            if (i > k) {
                const double a = fabs(W[i * LDP + k]);
                if (a > lam) {
                    lam = a;
                    r = i;
                }
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double l2 = __shfl_xor_sync(0xffffffffu, lam, o);
            const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
            if (l2 > lam || (l2 == lam && r2 < r)) {
                lam = l2;
                r = r2;
            }
        }
        const double akk = fabs(W[k * LDP + k]);
        int kind = 1, swp = -1;
        if (!(fmax(akk, lam) > 0.0)) {
            kind = 0;   // zero column (or NaN): a zero pivot
        } else if (akk < alpha * lam) {
            // sigma: the largest off-diagonal |entry| of row r in the trailing block
            double sg = 0.0;
            for (int j = lane; j < NB; j += 32)
                if (j >= k && j != r) sg = fmax(sg, fabs(W[r * LDP + j]));
            sg = warp_max_d(sg);
            if (akk * sg >= alpha * lam * lam) {
                kind = 1;
            } else if (fabs(W[r * LDP + r]) >= alpha * sg) {
                kind = 1;
                swp = r;
            } else {
                kind = 2;
                swp = r;
            }
        }
        // symmetric interchange of positions p and q (rows over every column -- the rows of
        // L computed so far move with them --, then columns over the trailing rows)
        if (swp >= 0) {
            const int p = kind == 2 ? k + 1 : k, q = swp;
            if (p != q) {
                for (int j = lane; j < NB; j += 32) {
                    const double a = W[p * LDP + j];
                    W[p * LDP + j] = W[q * LDP + j];
                    W[q * LDP + j] = a;
                }
                __syncwarp();
                for (int i = lane; i < NB; i += 32)
                    if (i >= k) {
                        const double a = W[i * LDP + p];
                        W[i * LDP + p] = W[i * LDP + q];
                        W[i * LDP + q] = a;
                    }
                if (lane == 0) {
                    const int t = perm[p];
                    perm[p] = perm[q];
                    perm[q] = t;
                }
                __syncwarp();
            }
        }
        if (kind == 0) {
            ++nzero;
            if (lane == 0) dd[k] = 0.0;
            for (int i = lane; i < NB; i += 32)
                if (i > k) W[i * LDP + k] = 0.0;
            __syncwarp();
            k += 1;
            continue;
        }
        if (kind == 1) {
            const double d = W[k * LDP + k];
            if (fabs(d) <= tiny) ++nzero;
            else if (d > 0.0) ++npos;
            else ++nneg;
            const double dinv = 1.0 / d;
            if (lane == 0) dd[k] = d;
            // every row i > k: l_i = w_ik / d, w_ij -= l_i w_kj (k < j <= i, mirrored)
            for (int i = lane; i < NB; i += 32)
                if (i > k) {
                    const double l = W[i * LDP + k] * dinv;
                    for (int j = k + 1; j <= i; ++j) {
                        const double v = fma(-l, W[k * LDP + j], W[i * LDP + j]);
                        W[i * LDP + j] = v;
                        W[j * LDP + i] = v;
                    }
                    W[i * LDP + k] = l;
                }
            __syncwarp();
            k += 1;
        } else {
            const double a = W[k * LDP + k], b = W[(k + 1) * LDP + k], c = W[(k + 1) * LDP + k + 1];
            const double det = a * c - b * b;   // < 0 for a Bunch-Kaufman 2 x 2 pivot
            if (det < 0.0) {
                ++npos;
                ++nneg;
            } else if (det > 0.0) {
                if (a > 0.0) npos += 2;
                else nneg += 2;
            } else {
                ++nzero;
                if (a + c > 0.0) ++npos;
                else if (a + c < 0.0) ++nneg;
                else ++nzero;
            }
            const double idet = 1.0 / det;
            const double i11 = c * idet, i12 = -b * idet, i22 = a * idet;
            if (lane == 0) {
                dd[k] = a;
                dd[k + 1] = c;
                od[k] = b;
                blk[k] = 2;
                blk[k + 1] = 0;
            }
            for (int i = lane; i < NB; i += 32)
                if (i > k + 1) {
                    const double w0 = W[i * LDP + k], w1 = W[i * LDP + k + 1];
                    const double l0 = w0 * i11 + w1 * i12, l1 = w0 * i12 + w1 * i22;
                    for (int j = k + 2; j <= i; ++j) {
                        const double v = W[i * LDP + j] - l0 * W[k * LDP + j] - l1 * W[(k + 1) * LDP + j];
                        W[i * LDP + j] = v;
                        W[j * LDP + i] = v;
                    }
                    W[i * LDP + k] = l0;
                    W[i * LDP + k + 1] = l1;
                }
            __syncwarp();
            if (lane == 0) W[(k + 1) * LDP + k] = 0.0;   // inside the pivot block: part of D, not of L
            __syncwarp();
            k += 2;
        }
    }
}

// Dinv = W^-1 in the original index order from the factors of bk_factor: column b of
// (L D L^T)^-1 by a forward sweep with L, the pivot blocks, a backward sweep with L^T
// (lane b, in T's column b), then scattered through perm.  A zero pivot contributes 0.
__device__ inline void bk_inverse(const double* W, const double* dd, const double* od, const int* perm,
                                  const int* blk, double* T, double* Dinv, int lane) {
    for (int b = lane; b < NB; b += 32) {
        for (int i = 0; i < NB; ++i) T[i * LDP + b] = i == b ? 1.0 : 0.0;
        for (int j = 0; j < NB; ++j) {
            const double yj = T[j * LDP + b];
            for (int i = j + 1; i < NB; ++i) T[i * LDP + b] = fma(-W[i * LDP + j], yj, T[i * LDP + b]);
        }
        for (int k = 0; k < NB;) {
            if (blk[k] == 2) {
                const double a = dd[k], c = dd[k + 1], o = od[k];
                const double det = a * c - o * o;
                const double y0 = T[k * LDP + b], y1 = T[(k + 1) * LDP + b];
                const double z0 = det != 0.0 ? (c * y0 - o * y1) / det : 0.0;
                const double z1 = det != 0.0 ? (a * y1 - o * y0) / det : 0.0;
                T[k * LDP + b] = z0;
                T[(k + 1) * LDP + b] = z1;
                k += 2;
            } else {
                const double d = dd[k];
                T[k * LDP + b] = d != 0.0 ? T[k * LDP + b] / d : 0.0;
                k += 1;
            }
        }
        for (int j = NB - 1; j >= 0; --j) {
            double acc = T[j * LDP + b];
            for (int i = j + 1; i < NB; ++i) acc = fma(-W[i * LDP + j], T[i * LDP + b], acc);
            T[j * LDP + b] = acc;
        }
    }
    __syncwarp();
    for (int e = lane; e < NB * NB; e += 32) {
        const int a = e / NB, b = e - a * NB;
        Dinv[perm[a] * LDP + perm[b]] = T[a * LDP + b];
    }
    __syncwarp();
}

// factor K_s of every active scenario (dw = PS_DW, dc = PS_DC of its problem): the
// inverses of Dt_0 .. Dt_9 to Dinv_g, and per scenario (partials at stage 0, the other
// stages 0) [2] positive, [3] negative, [6] zero pivots of K_s, [5] 1 if any pivot is zero.
// Only exactly zero pivots count as zero (a zero column of the trailing block, or a
// singular 2 x 2 pivot): near-singular blocks are factored, as LAPACK's Bunch-Kaufman
// does, and their inertia read from the signs.  One warp per block.
__global__ void __launch_bounds__(32) ldl_factor_kernel(int S, int64_t ld, const BView b,
                                                        const double* __restrict__ jac, const double* __restrict__ hes,
                                                        const double* __restrict__ sig, bool use_w,
                                                        double* __restrict__ Dinv_g, double* __restrict__ part) {
    extern __shared__ __align__(16) double ldl_sm[];
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x;
    const int p = live_prob(b, s, S, PS_ACT);
    if (p < 0) return;
    double* W = ldl_sm;
    double* Dv = W + LDL_BUF;
    double* E = Dv + LDL_BUF;
    double* T = E + LDL_BUF;
    double* dd = T + LDL_BUF;
    double* od = dd + NB;
    int* perm = reinterpret_cast<int*>(od + NB);
    int* blk = perm + NB;
    const double dw = b.ps ? psv(b, PS_DW, p) : 0.0;
    const double dc = b.ps ? psv(b, PS_DC, p) : 0.0;
    int npos = 0, nneg = 0, nzero = 0;
    for (int n = 0; n < N_STAGES; ++n) {
        ldl_assemble_diag(W, ld, s, n, jac, hes, sig, use_w, dw, dc, lane);
        if (n > 0) {
            // W -= E Dinv_{n-1} E^T: T = E Dinv (row a on lane a), then the lower triangle
            // of T E^T, mirrored
            ldl_assemble_coupling(E, ld, s, n, jac, lane);
            for (int a = lane; a < NB; a += 32)
                for (int j = 0; j < NB; ++j) {
                    double acc = 0.0;
                    for (int i = 0; i < NB; ++i) acc = fma(E[a * LDP + i], Dv[i * LDP + j], acc);
                    T[a * LDP + j] = acc;
                }
            __syncwarp();
            for (int a = lane; a < NB; a += 32)
                for (int c = 0; c <= a; ++c) {
                    double acc = 0.0;
                    for (int j = 0; j < NB; ++j) acc = fma(T[a * LDP + j], E[c * LDP + j], acc);
                    const double v = W[a * LDP + c] - acc;
                    W[a * LDP + c] = v;
                    W[c * LDP + a] = v;
                }
            __syncwarp();
        }
        bk_factor(W, dd, od, perm, blk, lane, 0.0, npos, nneg, nzero);
        bk_inverse(W, dd, od, perm, blk, T, Dv, lane);
        double* dst = Dinv_g + ldl_off(s, n);
        for (int e = lane; e < NB * NB; e += 32) {
            const int a = e / NB;
            dst[e] = Dv[a * LDP + (e - a * NB)];
        }
        __syncwarp();
    }
    if (lane < N_STAGES) {
        const int64_t plane = (int64_t)N_STAGES * ld;
        const int64_t o = (int64_t)lane * ld + s;
        const bool z = lane == 0;
        part[2 * plane + o] = z ? (double)npos : 0.0;
        part[3 * plane + o] = z ? (double)nneg : 0.0;
        part[5 * plane + o] = z ? (nzero > 0 ? 1.0 : 0.0) : 0.0;
        part[6 * plane + o] = z ? (double)nzero : 0.0;
    }
}

// v = K_s^-1 r of every active scenario with the inverses of ldl_factor_kernel:
// forward g_0 = r_0, g_n = r_n - E_{n-1} Dinv_{n-1} g_{n-1}; backward x_9 = Dinv_9 g_9,
// x_n = Dinv_n (g_n - E_n^T x_{n+1}).  r: z part rz (primal layout), row part rc (row
// layout); rhs_b: r = [0; b] instead, b = dc/dd (the d entries of the hydraulic rows).
// Out: xz (primal layout, d slots untouched), xl (row layout); partial plane `pl` of each
// scenario: sgn * b^T x_l at stage 0 (the other stages 0).  fac_planes (the factorization's
// u = K_s^-1 [0; b], pl = 0): plane 1 zero and plane 4 the scenario's d-d Hessian entry
// (hes, or 0 without), as the block-LU path's Schur sums lay them out; otherwise (a solve,
// pl = 2) planes 0, 1 and 3 zero.  One warp per block.
__global__ void __launch_bounds__(32) ldl_solve_kernel(int S, int64_t ld, const BView b,
                                                       const double* __restrict__ jac,
                                                       const double* __restrict__ Dinv_g,
                                                       const double* __restrict__ rz, const double* __restrict__ rc,
                                                       bool rhs_b, double* __restrict__ xz, double* __restrict__ xl,
                                                       double* __restrict__ part, int pl, double sgn, bool fac_planes,
                                                       const double* __restrict__ hes) {
    extern __shared__ __align__(16) double ldl_sm[];
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x;
    const int p = live_prob(b, s, S, PS_ACT);
    if (p < 0) return;
    double* Dv = ldl_sm;
    double* E = Dv + LDL_BUF;
    double* G = E + LDL_BUF;
    double* H = G + N_STAGES * NB;
    for (int e = lane; e < N_STAGES * NB; e += 32) {
        const int n = e / NB, i = e - n * NB;
        double v;
        if (rhs_b) v = (i == NV + R_H) ? jac[(int64_t)(c_segJ[n] + c_dslot[stage_type(n)]) * ld + s] : 0.0;
        else v = i < NV ? rz[(int64_t)(NV * n + i) * ld + s] : rc[(int64_t)(NR * n + i - NV) * ld + s];
        G[e] = v;
    }
    __syncwarp();
    auto load_inv = [&](int n) {
        const double* src = Dinv_g + ldl_off(s, n);
        for (int e = lane; e < NB * NB; e += 32) {
            const int a = e / NB;
            Dv[a * LDP + (e - a * NB)] = src[e];
        }
        __syncwarp();
    };
    // forward
    for (int n = 1; n < N_STAGES; ++n) {
        load_inv(n - 1);
        const double* gp = G + (n - 1) * NB;
        for (int a = lane; a < NB; a += 32) {
            double acc = 0.0;
            for (int j = 0; j < NB; ++j) acc = fma(Dv[a * LDP + j], gp[j], acc);
            H[a] = acc;
        }
        ldl_assemble_coupling(E, ld, s, n, jac, lane);   // its syncs order H before the reads below
        double* gn = G + n * NB;
        for (int a = lane; a < NB; a += 32) {
            double acc = gn[a];
            for (int i = 0; i < NB; ++i) acc = fma(-E[a * LDP + i], H[i], acc);
            gn[a] = acc;
        }
        __syncwarp();
    }
    // backward
    for (int n = N_STAGES - 1; n >= 0; --n) {
        double* gn = G + n * NB;
        if (n + 1 < N_STAGES) {
            ldl_assemble_coupling(E, ld, s, n + 1, jac, lane);   // E_n = K_{n+1,n}
            const double* xn1 = G + (n + 1) * NB;
            for (int i = lane; i < NB; i += 32) {
                double acc = gn[i];
                for (int a = 0; a < NB; ++a) acc = fma(-E[a * LDP + i], xn1[a], acc);
                H[i] = acc;
            }
        } else {
            for (int i = lane; i < NB; i += 32) H[i] = gn[i];
        }
        __syncwarp();
        load_inv(n);
        for (int a = lane; a < NB; a += 32) {
            double acc = 0.0;
            for (int j = 0; j < NB; ++j) acc = fma(Dv[a * LDP + j], H[j], acc);
            gn[a] = acc;
        }
        __syncwarp();
    }
    double bs = 0.0;
    for (int e = lane; e < N_STAGES * NB; e += 32) {
        const int n = e / NB, i = e - n * NB;
        if (i < NV) xz[(int64_t)(NV * n + i) * ld + s] = G[e];
        else xl[(int64_t)(NR * n + i - NV) * ld + s] = G[e];
        if (i == NV + R_H) bs += jac[(int64_t)(c_segJ[n] + c_dslot[stage_type(n)]) * ld + s] * G[e];
    }
    // the lanes' terms combined in a fixed order (lane order of the stages)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bs += __shfl_xor_sync(0xffffffffu, bs, o);
    if (lane < N_STAGES) {
        const int64_t plane = (int64_t)N_STAGES * ld;
        const int64_t o = (int64_t)lane * ld + s;
        part[pl * plane + o] = lane == 0 ? sgn * bs : 0.0;
        if (fac_planes) {
            part[1 * plane + o] = 0.0;
            part[4 * plane + o] = (lane == 0 && hes) ? hes[(int64_t)(NHS * N_STAGES) * ld + s] : 0.0;
        } else {
            part[0 * plane + o] = 0.0;
            part[1 * plane + o] = 0.0;
            part[3 * plane + o] = 0.0;
        }
    }
}

// the back-substitution of the Schur step on d: x = v - u dd for the z part (dz, d slots
// untouched) and the row part (dl), dd the problem's (dz's d slot).  One thread per
// (scenario, stage).
__global__ void __launch_bounds__(128) ldl_back_kernel(int S, int64_t ld, const BView b, const double* __restrict__ uz,
                                                       const double* __restrict__ ul, double* __restrict__ dz,
                                                       double* __restrict__ dl) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int p = live_prob(b, s, S, PS_ACT);
    if (p < 0) return;
    const double dd = dz[(int64_t)NSC * ld + p];
#pragma unroll
    for (int j = 0; j < NV; ++j) {
        const int64_t oz = (int64_t)(NV * n + j) * ld + s, ol = (int64_t)(NR * n + j) * ld + s;
        dz[oz] = fma(-uz[oz], dd, dz[oz]);
        dl[ol] = fma(-ul[ol], dd, dl[ol]);
    }
}

// the KKT residual of the regularised system, every term formed directly:
// rho_z = r_z - (W + Sigma + dw I) dz - J^T dl,  rho_c = r_c - J dz - b dd + dc dl;
// partials as kkt_residual_kernel's: [0] max|rho_z|, [1] max|rho_c|, [2] the stage's
// hydraulic dl, [3] max|r_z|, [4] max|r_c|.  One thread per (scenario, stage).
__global__ void __launch_bounds__(128) kkt_residual_reg_kernel(int S, int64_t ld, const BView b,
                                                               const double* __restrict__ jac,
                                                               const double* __restrict__ hes,
                                                               const double* __restrict__ sig, bool use_w,
                                                               const double* __restrict__ dz,
                                                               const double* __restrict__ dl,
                                                               const double* __restrict__ rz,
                                                               const double* __restrict__ rc, double* __restrict__ rhoz,
                                                               double* __restrict__ rhoc, double* part) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    const int p = live_prob(b, s, S, PS_ACT);
    if (p < 0) return;
    const double dw = b.ps ? psv(b, PS_DW, p) : 0.0;
    const double dc = b.ps ? psv(b, PS_DC, p) : 0.0;
    const double dd = dz[(int64_t)NSC * ld + p];
    double v[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int j = 0; j < NV; ++j) {
        const int64_t oz = (int64_t)(NV * n + j) * ld + s, ol = (int64_t)(NR * n + j) * ld + s;
        const double a = rz[oz] - hv_one(ld, hes, sig, dw, use_w, dz, s, n, j) - jt_one(ld, jac, dl, s, n, j);
        const double c = rc[ol] - jv_one(ld, jac, dz, dd, s, n, j) + dc * dl[ol];
        rhoz[oz] = a;
        rhoc[ol] = c;
        v[0] = fmax(v[0], fabs(a));
        v[1] = fmax(v[1], fabs(c));
        v[3] = fmax(v[3], fabs(rz[oz]));
        v[4] = fmax(v[4], fabs(rc[ol]));
        if (a != a || c != c) v[0] = NAN;
    }
    v[2] = dl[(int64_t)(NR * n + R_H) * ld + s];
    store_partials<5>(v, part, ld, s, n);
}

}  // namespace absorber
