// kernels_tc.cuh -- FP32 stage-block inverses by blocked Gauss-Jordan exchange with the
// dense trailing updates on the tensor cores (warp-level mma.sync, TF32 operands split in
// three products for FP32-level accuracy).  Same input and output as factor_gj_kernel:
// the inverse rows of every stage block in position order, -G_n, the row order, the
// singular flag.
//
// One warp per scenario; the augmented block M = [A_n | B_n] (22 x 33) stays in shared
// memory.  The 22 pivot columns are taken in panels K of 8 (8, 8, 6).  Inside a panel the
// exchanges run on the panel's columns only, lane i holding row i's panel entries: the
// pivot search (one warp maximum of position-tagged keys, ties to the lowest position, the
// rule of factor_gj_kernel), the pivot row's scaling and the rank-1 updates of the other
// rows.  With R the panel's pivot rows in step order, the panel's exchanges turn
// [A_RK B_RN; C_OK D_ON] into [A_RK^-1, -A_RK^-1 B_RN; C_OK A_RK^-1, D_ON - C_OK A_RK^-1 B_RN]
// (the principal pivot transform), so with the new panel columns M'_K (22 x 8) the other
// columns follow from one product T = M'_K B_R (22 x 8 times 8 x 33, B_R the pivot rows'
// entries before the panel):  M'_RN = -T_R,  M'_ON = M_ON - T_O.  That product runs as
// m16n8k8 MMAs (2 row tiles x 5 column tiles), each operand a = hi + lo with hi, lo TF32
// and T = hi hi' + hi lo' + lo hi' accumulated in FP32.
#pragma once

#include "kernels_warp.cuh"

namespace absorber {

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo, both TF32 (hi the rounded value, lo the rounded remainder)
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

// D += A B for one m16n8k8 tile (A row-major 16 x 8, B column-major 8 x 8, FP32 accumulate)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int TC_PANEL = 8;
constexpr int TC_NT = 5;   // column tiles of 8 over the 33 columns of [A_n | B_n]

template <int WPB = WPB_F>
__global__ void __launch_bounds__(32 * WPB, WPB >= 8 ? 3 : 24 / WPB) factor_gj_tc_kernel(
    int S, int64_t ld, const BView b, const double* __restrict__ jac, float* __restrict__ AI,
    unsigned char* __restrict__ piv, float* __restrict__ G, int* __restrict__ sing, double pivtol) {
    __shared__ __align__(16) float sM[WPB][NV * PADQ];
    __shared__ __align__(16) float sG[WPB][NV * NABV + 2];
    __shared__ __align__(16) float sU[WPB][TC_PANEL];
    __shared__ int sR[WPB][TC_PANEL];
    __shared__ int sIn[WPB][32];
    __shared__ LaneTables lt;
    stage_lane_tables(lt);
    const unsigned full = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int s = blockIdx.x * WPB + warp;
    if (live_prob(b, s, S, PS_ACT) < 0) return;   // whole warps leave together
    float* M = sM[warp];
    float* Gs = sG[warp];
    float* U = sU[warp];
    int* R = sR[warp];
    int* In = sIn[warp];
    const bool rowlane = lane < NV;
    const int g = lane >> 2, t4 = lane & 3;   // MMA fragment coordinates
    int singular = 0;
#pragma unroll 1
    for (int n = 0; n < N_STAGES; ++n) {
        const int t = stage_type(n);
        const int base = c_segJ[n];
        // assemble as factor_gj_kernel: every Jacobian load of the lane first, rows zeroed,
        // entries scattered, then the Schur update A_n -= C_n G_{n-1} on the lane's row
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
            for (int q = 0; q < PADQ / 4; ++q) *reinterpret_cast<float4*>(&M[lane * PADQ + 4 * q]) = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        L.scatter<float, PADQ>(M, lane);
        __syncwarp();
        if (rowlane) {
#pragma unroll
            for (int i = 0; i < NBLWV; ++i) {
                if (i < nb) {
                    const float cv = (float)vb[i];
                    const float* gr = Gs + blw_var(eb[i].c) * NABV;
#pragma unroll
                    for (int a = 0; a < NABV; ++a)
                        M[lane * PADQ + abv_var(a)] = fmaf(-cv, gr[a], M[lane * PADQ + abv_var(a)]);
                }
            }
        }
        // the largest |entry| of the block gives the singularity threshold
        unsigned km = 0u;
        if (rowlane) {
#pragma unroll
            for (int j = 0; j < NV; ++j) km = max(km, __float_as_uint(M[lane * PADQ + j]) & 0x7fffffffu);
        }
        km = __reduce_max_sync(full, km);
        const float tiny = (float)pivtol * __uint_as_float(km);
        const unsigned ktiny = __float_as_uint(tiny) & 0x7fffffffu;
        int cur = lane;             // position of this lane's row
        bool done = !rowlane;       // row already chosen (lanes >= 22 never take part)
#pragma unroll 1
        for (int k0 = 0; k0 < NV; k0 += TC_PANEL) {
            const int nbp = min(TC_PANEL, NV - k0);
            // ---- the panel's exchanges, on the panel's columns --------------------------
            float pc[TC_PANEL];
#pragma unroll
            for (int j = 0; j < TC_PANEL; ++j) pc[j] = (rowlane && j < nbp) ? M[lane * PADQ + k0 + j] : 0.f;
            int inR = 0;
#pragma unroll
            for (int j = 0; j < TC_PANEL; ++j) {
                if (j < nbp) {
                    const int k = k0 + j;
                    const float xk = pc[j];
                    const unsigned key = done ? 0u : pivot_key32(xk, cur);
                    const unsigned mx = __reduce_max_sync(full, key);
                    const int pos = key_position(mx);
                    const bool isp = !done && key == mx;
                    if (cur == k) cur = pos;
                    if (isp) {
                        cur = k;
                        done = true;
                        inR = 1;
                        R[j] = lane;
                        float ukk = xk;
                        if (!((__float_as_uint(ukk) & 0x7fffffffu) > ktiny) || ukk != ukk) {
                            singular = 1;
                            ukk = (ukk < 0.0f ? -1.0f : 1.0f) * (tiny > 0.0f ? tiny : 1.0f);
                        }
                        const float inv = recip(ukk);
#pragma unroll
                        for (int m = 0; m < TC_PANEL; ++m) pc[m] = -pc[m] * inv;
                        pc[j] = inv;
#pragma unroll
                        for (int m = 0; m < TC_PANEL; ++m) U[m] = pc[m];
                    }
                    __syncwarp();
                    if (rowlane && !isp) {
                        const float f = pc[j];
#pragma unroll
                        for (int m = 0; m < TC_PANEL; ++m)
                            if (m != j) pc[m] = fmaf(f, U[m], pc[m]);
                        pc[j] = f * U[j];
                    }
                    __syncwarp();
                }
            }
            In[lane] = inR;
            if (rowlane) {
#pragma unroll
                for (int j = 0; j < TC_PANEL; ++j)
                    if (j < nbp) M[lane * PADQ + k0 + j] = pc[j];
            }
            if (lane >= nbp && lane < TC_PANEL) R[lane] = 0;   // padding rows of a short panel
            __syncwarp();
            // ---- trailing update: T = M'_K B_R on the tensor cores ----------------------
            // A fragments (rows of M'_K; k = panel column), split hi + lo
            uint32_t ahi[2][4], alo[2][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int row = mt * 16 + g + ((e & 1) ? 8 : 0);
                    const int col = t4 + ((e & 2) ? 4 : 0);
                    const float v = (row < NV && col < nbp) ? M[row * PADQ + k0 + col] : 0.f;
                    tf32_split(v, ahi[mt][e], alo[mt][e]);
                }
            }
            const int r0 = R[t4], r1 = R[t4 + 4];
            const bool k0ok = t4 < nbp, k1ok = t4 + 4 < nbp;
            const bool in0 = In[g] != 0, in1 = In[g + 8] != 0, in2 = In[16 + g] != 0, in3 = In[24 + g] != 0;
#pragma unroll
            for (int nt = 0; nt < TC_NT; ++nt) {
                // B fragment: the pivot rows' entries of this column tile, before the update
                const int colb = nt * 8 + g;
                const float b0 = (k0ok && colb < NCA) ? M[r0 * PADQ + colb] : 0.f;
                const float b1 = (k1ok && colb < NCA) ? M[r1 * PADQ + colb] : 0.f;
                uint32_t bhi[2], blo[2];
                tf32_split(b0, bhi[0], blo[0]);
                tf32_split(b1, bhi[1], blo[1]);
                float d[2][4];
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) d[mt][e] = 0.f;
                    mma_tf32(d[mt], alo[mt], bhi);
                    mma_tf32(d[mt], ahi[mt], blo);
                    mma_tf32(d[mt], ahi[mt], bhi);
                }
                __syncwarp();   // every lane has read its B entries of this tile
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int row = mt * 16 + g + ((e & 2) ? 8 : 0);
                        const int col = nt * 8 + 2 * t4 + (e & 1);
                        const bool inrow = mt == 0 ? ((e & 2) ? in1 : in0) : ((e & 2) ? in3 : in2);
                        if (row < NV && col < NCA && (col < k0 || col >= k0 + nbp)) {
                            float& mv = M[row * PADQ + col];
                            mv = inrow ? -d[mt][e] : mv - d[mt][e];
                        }
                    }
                }
                __syncwarp();
            }
        }
        // the lane's row to registers, then to shared memory at its position (inverse
        // rows; -G_n by unknown for the next stage's Schur update), row order, stores
        float row[NPR * 2];
        if (rowlane) {
#pragma unroll
            for (int j = 0; j < NCA; ++j) row[j] = M[lane * PADQ + j];
        }
        __syncwarp();
        if (rowlane) {
#pragma unroll
            for (int j = 0; j < NV; ++j) M[cur * NV + j] = row[j];
            if (n + 1 < N_STAGES) {
#pragma unroll
                for (int a = 0; a < NABV; ++a) Gs[cur * NABV + a] = -row[NV + a];
            }
            piv[pv_off(s, n) + 2 * cur] = (unsigned char)lane;
            piv[pv_off(s, n) + 2 * lane + 1] = (unsigned char)cur;
        }
        __syncwarp();
        float4* Ln = reinterpret_cast<float4*>(AI + lu_off(s, n));
        for (int e = lane; e < NV * NV / 4; e += 32) Ln[e] = reinterpret_cast<const float4*>(M)[e];
        if (n + 1 < N_STAGES) {
            float2* Gn = reinterpret_cast<float2*>(G + g_off(s, n));
            for (int e = lane; e < NV * NABV / 2; e += 32) Gn[e] = reinterpret_cast<const float2*>(Gs)[e];
        }
        __syncwarp();
    }
    singular = __any_sync(0xffffffffu, singular);
    if (lane == 0) sing[s] = singular;
}

}  // namespace absorber
