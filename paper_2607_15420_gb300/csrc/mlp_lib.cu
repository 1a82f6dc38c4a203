// mlp_lib.cu -- the warm-start network of the learned warm start: a 3 -> 256 -> 256 ->
// 256 -> 440 perceptron with GELU activations, bfloat16 weights and FP32 accumulation,
// trained on the GPU by the kernels below (forward, reverse-mode backward, Adam).
//
//   a0 = (X - in_shift) / in_scale
//   a_l = gelu(a_{l-1} W_l^T + b_l),  l = 1..3;   gelu(x) = x Phi(x) (exact erf form)
//   yhat = a3 W4^T + b4                 (normalised outputs; raw = yhat * out_scale + out_shift)
//   loss = sum (yhat - (Y - out_shift) / out_scale)^2 / (2 n 440)
// The weight matrices enter every product as bfloat16 copies (round to nearest even)
// of FP32 master weights; biases, activations and sums are FP32.  Gradients are taken
// with respect to the rounded weights and applied to the masters by Adam (Kingma & Ba
// 2015, Algorithm 1).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "absorber.h"
#include "kernels_umma.cuh"

namespace {

constexpr int NIN = ABS_MLP_IN, NH = ABS_MLP_HIDDEN, NOUT = ABS_MLP_OUT;
constexpr int64_t NPAR = ABS_MLP_PARAMS;
// layer l: fan-in, fan-out, offsets of W_l ([out][in], row-major) and b_l in the flat vector
constexpr int L_IN[4] = {NIN, NH, NH, NH};
constexpr int L_OUT[4] = {NH, NH, NH, NOUT};
constexpr int64_t OFF_W[4] = {0, NIN * NH + NH, NIN * NH + NH + NH * NH + NH,
                              NIN * NH + NH + 2 * (NH * NH + NH)};
constexpr int64_t OFF_B[4] = {OFF_W[0] + NIN * NH, OFF_W[1] + NH * NH, OFF_W[2] + NH * NH, OFF_W[3] + NH * NOUT};
static_assert(OFF_B[3] + NOUT == NPAR, "parameter layout");

constexpr int CHUNK_ROWS = 8192;   // inference rows per pass (bounds the activation workspace)

thread_local std::string g_mlp_err = "no error";

}  // namespace

struct abs_mlp {
    int dev = 0;
    float* theta = nullptr;          // FP32 master parameters [NPAR]
    __nv_bfloat16* wb = nullptr;     // bfloat16 copies at the same offsets (weights only are read)
    float* grad = nullptr;           // [NPAR]
    float* m = nullptr;              // Adam moments [NPAR]
    float* v = nullptr;
    int64_t step = 0;                // Adam steps taken
    float* norm = nullptr;           // device: in_shift[3], in_scale[3], out_shift[440], out_scale[440]
    double hnorm[2 * NIN + 2 * NOUT];
    // activation workspace for cap rows
    int64_t cap = 0;
    float* a0 = nullptr;             // [cap][3] normalised inputs
    float* z[3] = {nullptr, nullptr, nullptr};   // pre-activations [cap][256]
    float* a[3] = {nullptr, nullptr, nullptr};   // activations [cap][256]
    float* yh = nullptr;             // [cap][440]
    float* g = nullptr;              // dloss/dyhat [cap][440]
    float* da = nullptr;             // [cap][256]
    float* dz = nullptr;             // [cap][256]
    float* xb = nullptr;             // gathered minibatch inputs [cap][3]
    float* ybt = nullptr;            // gathered minibatch targets [cap][440]
    int* perm = nullptr;             // [perm_cap]
    int64_t perm_cap = 0;
    double* lpart = nullptr;         // loss partial sums
    int64_t lpart_cap = 0;
    double* lacc = nullptr;          // per-epoch loss accumulators
    int64_t lacc_cap = 0;
    bool tc = true;                  // tensor-core products for the 256-input layers
    int* hfault = nullptr;           // mapped host flag: a tensor-core wait gave up
    int* dfault = nullptr;
    std::string err = "no error";
};

namespace {

abs_status mfail(abs_mlp* n, abs_status st, const std::string& msg) {
    if (n) n->err = msg;
    g_mlp_err = msg;
    return st;
}

#define MCK(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return mfail(net, e_ == cudaErrorMemoryAllocation ? ABS_ERR_OOM : ABS_ERR_CUDA, \
                         std::string(#call) + ": " + cudaGetErrorString(e_));             \
    } while (0)

abs_status mlaunch(abs_mlp* net) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mfail(net, ABS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ABS_OK;
}

__device__ __forceinline__ float gelu_f(float x) { return x * 0.5f * (1.0f + erff(x * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_prime_f(float x) {
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) + x * 0.39894228040143268f * expf(-0.5f * x * x);
}

__device__ __forceinline__ float ld_el(const float* p, int64_t i) { return p[i]; }
__device__ __forceinline__ float ld_el(const __nv_bfloat16* p, int64_t i) { return __bfloat162float(p[i]); }

enum { EPI_STORE = 0, EPI_BIAS_GELU = 1, EPI_BIAS = 2, EPI_GELU_GRAD = 3, EPI_DENORM = 4 };

constexpr int BM = 64, BN = 64, BK = 16, GT = 256;

// C[m][n] = sum_k A(m, k) B(k, n) with A(m, k) = A[m sam + k sak] and
// B(k, n) = B[k sbk + n sbn]; 64x64 tile per block, 4x4 outputs per thread, K in steps
// of 16 staged in shared memory.  Epilogues:
//   EPI_STORE      C = acc
//   EPI_BIAS_GELU  Z = acc + bias[n] (stored), C = gelu(Z)
//   EPI_BIAS       C = acc + bias[n]
//   EPI_GELU_GRAD  C = acc * gelu'(aux[m][n])
//   EPI_DENORM     C = (acc + bias[n]) * scale[n] + shift[n]
// Row-major C, Z and aux with leading dimension ldc = N.
template <class TB, int EPI>
__global__ void __launch_bounds__(GT) gemm_kernel(int M, int N, int K, const float* __restrict__ A, int64_t sam,
                                                  int64_t sak, const TB* __restrict__ B, int64_t sbk, int64_t sbn,
                                                  const float* __restrict__ bias, const float* __restrict__ aux,
                                                  float* __restrict__ Z, float* __restrict__ C,
                                                  const float* __restrict__ scale, const float* __restrict__ shift) {
    __shared__ __align__(16) float As[BK][BM + 4];
    __shared__ __align__(16) float Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tr = tid / 16, tc = tid % 16;   // this thread's 4 rows tr*4.. and 4 columns tc*4..
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.0f;
    const bool a_kfast = sak == 1, b_nfast = sbn == 1;
    for (int k0 = 0; k0 < K; k0 += BK) {
#pragma unroll
        for (int r = 0; r < (BM * BK) / GT; ++r) {
            const int e = tid + r * GT;
            int mm, kk;
            if (a_kfast) {
                mm = e / BK;
                kk = e % BK;
            } else {
                kk = e / BM;
                mm = e % BM;
            }
            const int gm = m0 + mm, gk = k0 + kk;
            As[kk][mm] = (gm < M && gk < K) ? A[(int64_t)gm * sam + (int64_t)gk * sak] : 0.0f;
        }
#pragma unroll
        for (int r = 0; r < (BN * BK) / GT; ++r) {
            const int e = tid + r * GT;
            int nn, kk;
            if (b_nfast) {
                kk = e / BN;
                nn = e % BN;
            } else {
                nn = e / BK;
                kk = e % BK;
            }
            const int gn = n0 + nn, gk = k0 + kk;
            Bs[kk][nn] = (gn < N && gk < K) ? ld_el(B, (int64_t)gk * sbk + (int64_t)gn * sbn) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 av = *reinterpret_cast<const float4*>(&As[kk][tr * 4]);
            const float4 bv = *reinterpret_cast<const float4*>(&Bs[kk][tc * 4]);
            const float ar[4] = {av.x, av.y, av.z, av.w};
            const float br[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(ar[i], br[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int gm = m0 + tr * 4 + i;
        if (gm >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int gn = n0 + tc * 4 + j;
            if (gn >= N) continue;
            const int64_t o = (int64_t)gm * N + gn;
            float vv = acc[i][j];
            if (EPI == EPI_BIAS_GELU) {
                vv += bias[gn];
                Z[o] = vv;
                vv = gelu_f(vv);
            } else if (EPI == EPI_BIAS) {
                vv += bias[gn];
            } else if (EPI == EPI_GELU_GRAD) {
                vv *= gelu_prime_f(aux[o]);
            } else if (EPI == EPI_DENORM) {
                vv = (vv + bias[gn]) * scale[gn] + shift[gn];
            }
            C[o] = vv;
        }
    }
}

// The forward products on the tensor cores (kernels_umma.cuh): A FP32 [M][K] row-major, W
// bfloat16 [N][K] row-major, K a multiple of 64; epilogues EPI_BIAS_GELU, EPI_BIAS,
// EPI_DENORM as gemm_kernel's.  Grid (ceil(N / 64), ceil(M / 128)), 128 threads,
// umma::SMEM bytes of dynamic shared memory.  fault: set when a wait for the MMAs gave up
// (the block then frees its tensor memory and leaves its outputs unwritten).  idle (the
// self-test of that path): no MMA and no commit are issued, so the first wait runs out
// after wait_limit polls.
template <int EPI>
__global__ void __launch_bounds__(umma::T) gemm_tc_kernel(int M, int N, int K, const float* __restrict__ A,
                                                          const __nv_bfloat16* __restrict__ W,
                                                          const float* __restrict__ bias, float* __restrict__ Z,
                                                          float* __restrict__ C, const float* __restrict__ scale,
                                                          const float* __restrict__ shift, int* __restrict__ fault,
                                                          int idle, long long wait_limit) {
    using namespace umma;
    extern __shared__ unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tbase;
    unsigned char* sm = (unsigned char*)(((uintptr_t)tc_smem + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const uint32_t sa = smem_u32(sm), sb = sa + 3 * A_PLANE, mb = smem_u32(&mbar);
    if (warp == 0) {
        tmem_alloc(smem_u32(&tbase), TN);
        tmem_relinquish();
    }
    if (tid == 0) mbar_init(mb, 1);
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = tbase;
    bool ok = true;
    for (int c = 0; c < K / KC; ++c) {
        const int k0 = c * KC;
        // A chunk: 128 x 64 FP32 as float4, W chunk: 64 x 64 bfloat16 as 16-byte rows of core
        // matrices; every load in flight before the first store.  Float4 e of the A chunk
        // fills half a row of core matrix cm = e / 16 (row group cm / 8, K block cm % 8) and
        // W's row v of core matrix v / 8 (row group (v / 8) / 8, K block (v / 8) % 8): a
        // half-warp's stores cover whole 128-byte core matrices.  A is split into its three
        // bfloat16 terms (8-byte stores into the three term planes)
        constexpr int NA = (TM * KC / 4) / T, NB = (TN * KC / 8) / T;
        float4 av[NA];
        uint4 wv[NB];
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int e = i * T + tid, cm = e >> 4, q = e & 15;
            const int r = ((cm >> 3) << 3) + (q >> 1), k = ((cm & 7) << 3) + ((q & 1) << 2);
            av[i] = m0 + r < M ? *reinterpret_cast<const float4*>(A + (int64_t)(m0 + r) * K + k0 + k)
                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int v = i * T + tid, cm = v >> 3;
            const int n = ((cm >> 3) << 3) + (v & 7), k = (cm & 7) << 3;
            wv[i] = n0 + n < N ? *reinterpret_cast<const uint4*>(W + (int64_t)(n0 + n) * K + k0 + k)
                               : make_uint4(0u, 0u, 0u, 0u);
        }
#pragma unroll
        for (int i = 0; i < NA; ++i) {
            const int e = i * T + tid, cm = e >> 4, q = e & 15;
            const int r = ((cm >> 3) << 3) + (q >> 1), k = ((cm & 7) << 3) + ((q & 1) << 2);
            const float a4[4] = {av[i].x, av[i].y, av[i].z, av[i].w};
            __nv_bfloat16 t[3][4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const __nv_bfloat16 h = __float2bfloat16_rn(a4[j]);
                const float r1 = a4[j] - __bfloat162float(h);
                const __nv_bfloat16 m = __float2bfloat16_rn(r1);
                t[0][j] = h;
                t[1][j] = m;
                t[2][j] = __float2bfloat16_rn(r1 - __bfloat162float(m));
            }
            const uint32_t o = core_off(r, k, TM / 8);
#pragma unroll
            for (int p = 0; p < 3; ++p)
                *reinterpret_cast<uint2*>(sm + p * A_PLANE + o) = make_uint2(pack2(t[p][0], t[p][1]), pack2(t[p][2], t[p][3]));
        }
#pragma unroll
        for (int i = 0; i < NB; ++i) {
            const int v = i * T + tid, cm = v >> 3;
            const int n = ((cm >> 3) << 3) + (v & 7), k = (cm & 7) << 3;
            *reinterpret_cast<uint4*>(sm + 3 * A_PLANE + core_off(n, k, TN / 8)) = wv[i];
        }
        fence_smem_async();
        __syncthreads();
        if (tid == 0 && !idle) {
            fence_after();
#pragma unroll
            for (int s = 0; s < KC / 16; ++s)
#pragma unroll
                for (int p = 0; p < 3; ++p)
                    mma(tmem, desc(sa + p * A_PLANE + s * 2 * (TM / 8) * 128, A_LBO, A_SBO),
                        desc(sb + s * 2 * (TN / 8) * 128, B_LBO, B_SBO), IDESC, (c | s | p) != 0);
            commit(mb);
        }
        // the chunk's MMAs are done before its shared memory is refilled
        ok = __syncthreads_and(ok && mbar_wait(mb, (uint32_t)(c & 1), wait_limit));
        if (!ok) break;
        fence_after();
    }
    if (ok) {
        // accumulator rows + bias into a padded shared tile over the A planes (the MMAs are
        // done): warp w its lanes (rows) 32 (w % 4) + 0..31, columns TN / 2 (w / 4) + ...
        // Then rows written with the lanes along the columns (coalesced), the epilogue's
        // nonlinearity on the way
        constexpr int LDS = TN + 1;
        float* tile = reinterpret_cast<float*>(sm);
        const int q4 = warp & 3, ch = warp >> 2;
        const int r = q4 * 32 + lane;
#pragma unroll
        for (int cb = ch * (TN / 2); cb < (ch + 1) * (TN / 2); cb += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)cb, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int gn = n0 + cb + j;
                tile[r * LDS + cb + j] = v[j] + (gn < N ? bias[gn] : 0.0f);
            }
        }
        __syncthreads();
        for (int rr = warp; rr < TM; rr += T / 32) {
            const int row = m0 + rr;
            if (row >= M) break;   // warp-uniform
#pragma unroll
            for (int h = 0; h < TN / 32; ++h) {
                const int c = lane + 32 * h, gn = n0 + c;
                if (gn >= N) continue;
                const int64_t o = (int64_t)row * N + gn;
                float vv = tile[rr * LDS + c];
                if (EPI == EPI_BIAS_GELU) {
                    Z[o] = vv;
                    vv = gelu_f(vv);
                } else if (EPI == EPI_DENORM) {
                    vv = vv * scale[gn] + shift[gn];
                }
                C[o] = vv;
            }
        }
    }
    fence_before();
    __syncthreads();
    if (warp == 0) tmem_dealloc(tmem, TN);
    if (!ok && tid == 0) atomicExch(fault, 1);
}

template <int EPI>
abs_status gemm_tc(abs_mlp* net, cudaStream_t st, int M, int N, int K, const float* A, const __nv_bfloat16* W,
                   float* C, const float* bias, float* Z, const float* scale, const float* shift,
                   bool idle = false) {
    static bool attr = false;
    if (!attr) {
        MCK(cudaFuncSetAttribute(gemm_tc_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize, umma::SMEM));
        attr = true;
    }
    const dim3 grid((unsigned)((N + umma::TN - 1) / umma::TN), (unsigned)((M + umma::TM - 1) / umma::TM));
    gemm_tc_kernel<EPI><<<grid, umma::T, umma::SMEM, st>>>(M, N, K, A, W, bias, Z, C, scale, shift, net->dfault,
                                                           idle ? 1 : 0, idle ? 1024ll : umma::WAIT_LIMIT);
    return mlaunch(net);
}

template <class TB, int EPI>
abs_status gemm(abs_mlp* net, cudaStream_t st, int M, int N, int K, const float* A, int64_t sam, int64_t sak,
                const TB* B, int64_t sbk, int64_t sbn, float* C, const float* bias = nullptr,
                const float* aux = nullptr, float* Z = nullptr, const float* scale = nullptr,
                const float* shift = nullptr) {
    if (M <= 0 || N <= 0) return ABS_OK;
    if constexpr (std::is_same<TB, __nv_bfloat16>::value &&
                  (EPI == EPI_BIAS_GELU || EPI == EPI_BIAS || EPI == EPI_DENORM)) {
        // a forward product of a 256-input layer: A [M][K], W [N][K] row-major, aligned
        if (net->tc && K % umma::KC == 0 && sak == 1 && sam == K && sbk == 1 && sbn == K &&
            ((uintptr_t)A & 15) == 0 && ((uintptr_t)B & 15) == 0)
            return gemm_tc<EPI>(net, st, M, N, K, A, B, C, bias, Z, scale, shift);
    }
    const dim3 grid((unsigned)((N + BN - 1) / BN), (unsigned)((M + BM - 1) / BM));
    gemm_kernel<TB, EPI><<<grid, GT, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, aux, Z, C, scale, shift);
    return mlaunch(net);
}

__global__ void normalize_kernel(int64_t n, const float* __restrict__ X, const float* __restrict__ norm,
                                 float* __restrict__ a0) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * NIN) return;
    const int k = (int)(i % NIN);
    a0[i] = (X[i] - norm[k]) / norm[NIN + k];
}

// g = (yhat - t) / (n * 440) with t the normalised target; block partial sums of r^2
__global__ void __launch_bounds__(256) loss_grad_kernel(int64_t n, const float* __restrict__ yh,
                                                        const float* __restrict__ Y, const float* __restrict__ norm,
                                                        float inv, float* __restrict__ g, double* __restrict__ part) {
    __shared__ double sh[256];
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double r2 = 0.0;
    if (i < n * NOUT) {
        const int k = (int)(i % NOUT);
        const float t = (Y[i] - norm[2 * NIN + k]) / norm[2 * NIN + NOUT + k];
        const float r = yh[i] - t;
        g[i] = r * inv;
        r2 = (double)r * (double)r;
    }
    sh[threadIdx.x] = r2;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// out[slot] (+)= scale * sum of part[0..np) in a fixed order (one block)
__global__ void __launch_bounds__(256) sum_partials_kernel(const double* __restrict__ part, int64_t np, double scale,
                                                           bool accumulate, double* __restrict__ out) {
    __shared__ double sh[256];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < np; i += 256) a += part[i];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = (accumulate ? *out : 0.0) + scale * sh[0];
}

// db[o] = sum over rows of dz[row][o]  (one thread per column, rows in order)
__global__ void colsum_kernel(int rows, int cols, const float* __restrict__ dz, float* __restrict__ db) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= cols) return;
    float a = 0.0f;
    for (int r = 0; r < rows; ++r) a += dz[(int64_t)r * cols + o];
    db[o] = a;
}

__global__ void to_bf16_kernel(int64_t n, const float* __restrict__ src, __nv_bfloat16* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = __float2bfloat16_rn(src[i]);
}

__global__ void adam_kernel(int64_t n, float* __restrict__ th, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2,
                            __nv_bfloat16* __restrict__ wb) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float t = th[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    th[i] = t;
    wb[i] = __float2bfloat16_rn(t);
}

__global__ void gather_rows_kernel(int64_t rows, int cols, const int* __restrict__ idx, const float* __restrict__ src,
                                   float* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= rows * cols) return;
    const int64_t r = i / cols, c = i % cols;
    dst[i] = src[(int64_t)idx[r] * cols + c];
}

// per-column mean and standard deviation of X [n][cols] (double sums in a fixed order);
// a column whose spread is below 1e-7 of its magnitude keeps scale 1
__global__ void __launch_bounds__(256) column_stats_kernel(int64_t n, int cols, const float* __restrict__ X,
                                                           float* __restrict__ shift, float* __restrict__ scale) {
    __shared__ double sh[256];
    const int c = blockIdx.x;
    double a = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) a += X[r * cols + c];
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double mean = sh[0] / (double)n;
    __syncthreads();
    a = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) {
        const double d = X[r * cols + c] - mean;
        a += d * d;
    }
    sh[threadIdx.x] = a;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sd = sqrt(sh[0] / (double)n);
        shift[c] = (float)mean;
        scale[c] = (sd > 1e-7 * fmax(1.0, fabs(mean))) ? (float)sd : 1.0f;
    }
}

unsigned grid1(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

abs_status ensure_cap(abs_mlp* net, int64_t rows) {
    if (rows <= net->cap) return ABS_OK;
    cudaFree(net->a0);
    for (int l = 0; l < 3; ++l) {
        cudaFree(net->z[l]);
        cudaFree(net->a[l]);
    }
    cudaFree(net->yh);
    cudaFree(net->g);
    cudaFree(net->da);
    cudaFree(net->dz);
    cudaFree(net->xb);
    cudaFree(net->ybt);
    cudaFree(net->lpart);
    net->cap = 0;
    MCK(cudaMalloc(&net->a0, sizeof(float) * rows * NIN));
    for (int l = 0; l < 3; ++l) {
        MCK(cudaMalloc(&net->z[l], sizeof(float) * rows * NH));
        MCK(cudaMalloc(&net->a[l], sizeof(float) * rows * NH));
    }
    MCK(cudaMalloc(&net->yh, sizeof(float) * rows * NOUT));
    MCK(cudaMalloc(&net->g, sizeof(float) * rows * NOUT));
    MCK(cudaMalloc(&net->da, sizeof(float) * rows * NH));
    MCK(cudaMalloc(&net->dz, sizeof(float) * rows * NH));
    MCK(cudaMalloc(&net->xb, sizeof(float) * rows * NIN));
    MCK(cudaMalloc(&net->ybt, sizeof(float) * rows * NOUT));
    net->lpart_cap = (rows * NOUT + 255) / 256;
    MCK(cudaMalloc(&net->lpart, sizeof(double) * net->lpart_cap));
    net->cap = rows;
    return ABS_OK;
}

// forward pass of rows X [n][3] (raw); train: normalised outputs in net->yh and the
// layer values kept for backward; else raw outputs into Yout
abs_status forward_rows(abs_mlp* net, const float* X, int64_t n, bool train, float* Yout, cudaStream_t st) {
    abs_status r;
    normalize_kernel<<<grid1(n * NIN), 256, 0, st>>>(n, X, net->norm, net->a0);
    if ((r = mlaunch(net)) != ABS_OK) return r;
    const float* prev = net->a0;
    for (int l = 0; l < 3; ++l) {
        const int in = L_IN[l];
        if ((r = gemm<__nv_bfloat16, EPI_BIAS_GELU>(net, st, (int)n, NH, in, prev, in, 1, net->wb + OFF_W[l], 1, in,
                                                    net->a[l], net->theta + OFF_B[l], nullptr, net->z[l])) != ABS_OK)
            return r;
        prev = net->a[l];
    }
    if (train)
        return gemm<__nv_bfloat16, EPI_BIAS>(net, st, (int)n, NOUT, NH, prev, NH, 1, net->wb + OFF_W[3], 1, NH,
                                            net->yh, net->theta + OFF_B[3]);
    return gemm<__nv_bfloat16, EPI_DENORM>(net, st, (int)n, NOUT, NH, prev, NH, 1, net->wb + OFF_W[3], 1, NH, Yout,
                                          net->theta + OFF_B[3], nullptr, nullptr, net->norm + 2 * NIN + NOUT,
                                          net->norm + 2 * NIN);
}

// loss and gradient of the rows last passed through forward_rows(train) against raw
// targets Y [n][440]; gradient into net->grad, loss*scale into *loss_dev (+= if acc)
abs_status backward_rows(abs_mlp* net, const float* Y, int64_t n, double* loss_dev, double scale, bool acc,
                         cudaStream_t st) {
    abs_status r;
    const int64_t nel = n * NOUT;
    const unsigned nb = grid1(nel);
    loss_grad_kernel<<<nb, 256, 0, st>>>(n, net->yh, Y, net->norm, 1.0f / (float)nel, net->g, net->lpart);
    if ((r = mlaunch(net)) != ABS_OK) return r;
    sum_partials_kernel<<<1, 256, 0, st>>>(net->lpart, nb, scale / (2.0 * (double)nel), acc, loss_dev);
    if ((r = mlaunch(net)) != ABS_OK) return r;
    // layer 4: dW4 = g^T a3, db4 = colsum g, da3 = g W4
    const float* dcur = net->g;
    int ocur = NOUT;
    for (int l = 3; l >= 0; --l) {
        const int in = L_IN[l];
        const float* aprev = l > 0 ? net->a[l - 1] : net->a0;
        if ((r = gemm<float, EPI_STORE>(net, st, ocur, in, (int)n, dcur, 1, ocur, aprev, in, 1,
                                        net->grad + OFF_W[l])) != ABS_OK)
            return r;
        colsum_kernel<<<grid1(ocur, 128), 128, 0, st>>>((int)n, ocur, dcur, net->grad + OFF_B[l]);
        if ((r = mlaunch(net)) != ABS_OK) return r;
        if (l == 0) break;
        // dz_{l-1} = (dcur W_l) * gelu'(z_{l-1}); dcur and the result alternate buffers
        float* dst = (dcur == net->dz) ? net->da : net->dz;
        if ((r = gemm<__nv_bfloat16, EPI_GELU_GRAD>(net, st, (int)n, in, ocur, dcur, ocur, 1, net->wb + OFF_W[l], in,
                                                    1, dst, nullptr, net->z[l - 1])) != ABS_OK)
            return r;
        dcur = dst;
        ocur = in;
    }
    return ABS_OK;
}

uint64_t splitmix64(uint64_t& s) {
    // splitmix64 (Steele, Lea & Flood 2014)
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

abs_status upload_norm(abs_mlp* net) {
    float f[2 * NIN + 2 * NOUT];
    for (int i = 0; i < 2 * NIN + 2 * NOUT; ++i) f[i] = (float)net->hnorm[i];
    MCK(cudaMemcpy(net->norm, f, sizeof(f), cudaMemcpyHostToDevice));
    return ABS_OK;
}

}  // namespace

extern "C" {

const char* abs_mlp_last_error(const abs_mlp* net) { return net ? net->err.c_str() : g_mlp_err.c_str(); }

abs_status abs_mlp_create(uint64_t seed, abs_mlp** out) {
    abs_mlp* net = nullptr;
    if (!out) return mfail(nullptr, ABS_ERR_ARG, "bad argument");
    *out = nullptr;
    net = new abs_mlp();
    abs_status r = ABS_OK;
    auto bad = [&](abs_status st) {
        const std::string msg = net->err;
        abs_mlp_destroy(net);
        return mfail(nullptr, st, msg);
    };
#define MCK2(call)                                                                                    \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            mfail(net, e_ == cudaErrorMemoryAllocation ? ABS_ERR_OOM : ABS_ERR_CUDA,                  \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                                \
            return bad(e_ == cudaErrorMemoryAllocation ? ABS_ERR_OOM : ABS_ERR_CUDA);                 \
        }                                                                                             \
    } while (0)
    MCK2(cudaGetDevice(&net->dev));
    MCK2(cudaMalloc(&net->theta, sizeof(float) * NPAR));
    MCK2(cudaMalloc(&net->wb, sizeof(__nv_bfloat16) * NPAR));
    MCK2(cudaMalloc(&net->grad, sizeof(float) * NPAR));
    MCK2(cudaMalloc(&net->m, sizeof(float) * NPAR));
    MCK2(cudaMalloc(&net->v, sizeof(float) * NPAR));
    MCK2(cudaMalloc(&net->norm, sizeof(float) * (2 * NIN + 2 * NOUT)));
    MCK2(cudaHostAlloc(&net->hfault, sizeof(int), cudaHostAllocMapped));
    *net->hfault = 0;
    MCK2(cudaHostGetDevicePointer(&net->dfault, net->hfault, 0));
#undef MCK2
    // Glorot-uniform weights (Glorot & Bengio 2010), zero biases, identity normalisation
    std::vector<float> th(NPAR, 0.0f);
    uint64_t s = seed;
    for (int l = 0; l < 4; ++l) {
        const double lim = std::sqrt(6.0 / (double)(L_IN[l] + L_OUT[l]));
        for (int64_t i = 0; i < (int64_t)L_IN[l] * L_OUT[l]; ++i) {
            const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
            th[OFF_W[l] + i] = (float)((2.0 * u - 1.0) * lim);
        }
    }
    for (int i = 0; i < NIN; ++i) {
        net->hnorm[i] = 0.0;
        net->hnorm[NIN + i] = 1.0;
    }
    for (int i = 0; i < NOUT; ++i) {
        net->hnorm[2 * NIN + i] = 0.0;
        net->hnorm[2 * NIN + NOUT + i] = 1.0;
    }
    if ((r = upload_norm(net)) != ABS_OK) return bad(r);
    if ((r = abs_mlp_set_params(net, th.data())) != ABS_OK) return bad(r);
    *out = net;
    return ABS_OK;
}

void abs_mlp_destroy(abs_mlp* net) {
    if (!net) return;
    if (net->hfault) cudaFreeHost(net->hfault);
    cudaFree(net->theta);
    cudaFree(net->wb);
    cudaFree(net->grad);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->norm);
    cudaFree(net->a0);
    for (int l = 0; l < 3; ++l) {
        cudaFree(net->z[l]);
        cudaFree(net->a[l]);
    }
    cudaFree(net->yh);
    cudaFree(net->g);
    cudaFree(net->da);
    cudaFree(net->dz);
    cudaFree(net->xb);
    cudaFree(net->ybt);
    cudaFree(net->perm);
    cudaFree(net->lpart);
    cudaFree(net->lacc);
    delete net;
}

abs_status abs_mlp_set_params(abs_mlp* net, const float* params) {
    if (!net || !params) return mfail(net, ABS_ERR_ARG, "bad argument");
    MCK(cudaMemcpy(net->theta, params, sizeof(float) * NPAR, cudaMemcpyHostToDevice));
    MCK(cudaMemset(net->m, 0, sizeof(float) * NPAR));
    MCK(cudaMemset(net->v, 0, sizeof(float) * NPAR));
    net->step = 0;
    to_bf16_kernel<<<grid1(NPAR), 256>>>(NPAR, net->theta, net->wb);
    abs_status r = mlaunch(net);
    if (r != ABS_OK) return r;
    MCK(cudaDeviceSynchronize());
    return ABS_OK;
}

abs_status abs_mlp_get_params(const abs_mlp* cnet, float* params) {
    abs_mlp* net = const_cast<abs_mlp*>(cnet);
    if (!net || !params) return mfail(net, ABS_ERR_ARG, "bad argument");
    MCK(cudaMemcpy(params, net->theta, sizeof(float) * NPAR, cudaMemcpyDeviceToHost));
    return ABS_OK;
}

abs_status abs_mlp_set_normalization(abs_mlp* net, const double* in_shift, const double* in_scale,
                                     const double* out_shift, const double* out_scale) {
    if (!net || !in_shift || !in_scale || !out_shift || !out_scale) return mfail(net, ABS_ERR_ARG, "bad argument");
    for (int i = 0; i < NIN; ++i)
        if (!(in_scale[i] > 0.0)) return mfail(net, ABS_ERR_ARG, "scales must be positive");
    for (int i = 0; i < NOUT; ++i)
        if (!(out_scale[i] > 0.0)) return mfail(net, ABS_ERR_ARG, "scales must be positive");
    std::memcpy(net->hnorm, in_shift, sizeof(double) * NIN);
    std::memcpy(net->hnorm + NIN, in_scale, sizeof(double) * NIN);
    std::memcpy(net->hnorm + 2 * NIN, out_shift, sizeof(double) * NOUT);
    std::memcpy(net->hnorm + 2 * NIN + NOUT, out_scale, sizeof(double) * NOUT);
    return upload_norm(net);
}

abs_status abs_mlp_get_normalization(const abs_mlp* net, double* in_shift, double* in_scale, double* out_shift,
                                     double* out_scale) {
    if (!net) return mfail(nullptr, ABS_ERR_ARG, "bad argument");
    if (in_shift) std::memcpy(in_shift, net->hnorm, sizeof(double) * NIN);
    if (in_scale) std::memcpy(in_scale, net->hnorm + NIN, sizeof(double) * NIN);
    if (out_shift) std::memcpy(out_shift, net->hnorm + 2 * NIN, sizeof(double) * NOUT);
    if (out_scale) std::memcpy(out_scale, net->hnorm + 2 * NIN + NOUT, sizeof(double) * NOUT);
    return ABS_OK;
}

abs_status abs_mlp_fit_normalization(abs_mlp* net, const float* X, const float* Y, int64_t n, abs_stream_t stream) {
    if (!net || !X || !Y || n < 1) return mfail(net, ABS_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    column_stats_kernel<<<NIN, 256, 0, st>>>(n, NIN, X, net->norm, net->norm + NIN);
    abs_status r = mlaunch(net);
    if (r != ABS_OK) return r;
    column_stats_kernel<<<NOUT, 256, 0, st>>>(n, NOUT, Y, net->norm + 2 * NIN, net->norm + 2 * NIN + NOUT);
    if ((r = mlaunch(net)) != ABS_OK) return r;
    float f[2 * NIN + 2 * NOUT];
    MCK(cudaMemcpyAsync(f, net->norm, sizeof(f), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    for (int i = 0; i < 2 * NIN + 2 * NOUT; ++i) net->hnorm[i] = f[i];
    return ABS_OK;
}

int32_t abs_mlp_device_fault(const abs_mlp* net) { return net && net->hfault ? *(volatile int*)net->hfault : 0; }

abs_status abs_mlp_set_tensor_cores(abs_mlp* net, int32_t on) {
    if (!net || (on != 0 && on != 1)) return mfail(net, ABS_ERR_ARG, "bad argument");
    net->tc = on != 0;
    return ABS_OK;
}

abs_status abs_mlp_selftest_wait(abs_mlp* net, abs_stream_t stream) {
    if (!net) return mfail(net, ABS_ERR_ARG, "bad argument");
    if (abs_mlp_device_fault(net)) return mfail(net, ABS_ERR_TIMEOUT, "a tensor-core product gave up waiting");
    cudaStream_t st = (cudaStream_t)stream;
    abs_status r;
    if ((r = ensure_cap(net, umma::TM)) != ABS_OK) return r;
    // one 128 x 256 x 256 product with its MMAs withheld, on the activation workspace
    if ((r = gemm_tc<EPI_BIAS_GELU>(net, st, umma::TM, NH, NH, net->a[0], net->wb + OFF_W[1], net->a[1],
                                     net->theta + OFF_B[1], net->z[1], nullptr, nullptr, true)) != ABS_OK)
        return r;
    MCK(cudaStreamSynchronize(st));
    const bool expired = abs_mlp_device_fault(net) != 0;
    *(volatile int*)net->hfault = 0;
    if (!expired) return mfail(net, ABS_ERR_CUDA, "the withheld wait did not report its expiry");
    return mfail(net, ABS_ERR_TIMEOUT, "a tensor-core product gave up waiting (self-test)");
}

abs_status abs_mlp_forward(abs_mlp* net, const float* X, int64_t n, float* Y, abs_stream_t stream) {
    if (!net || n < 0 || (n > 0 && (!X || !Y))) return mfail(net, ABS_ERR_ARG, "bad argument");
    if (abs_mlp_device_fault(net)) return mfail(net, ABS_ERR_TIMEOUT, "a tensor-core product gave up waiting");
    cudaStream_t st = (cudaStream_t)stream;
    abs_status r;
    for (int64_t r0 = 0; r0 < n; r0 += CHUNK_ROWS) {
        const int64_t rows = std::min<int64_t>(CHUNK_ROWS, n - r0);
        if ((r = ensure_cap(net, rows)) != ABS_OK) return r;
        if ((r = forward_rows(net, X + r0 * NIN, rows, false, Y + r0 * NOUT, st)) != ABS_OK) return r;
    }
    return ABS_OK;
}

abs_status abs_mlp_loss_grad(abs_mlp* net, const float* X, const float* Y, int64_t n, double* loss, float* grad,
                             abs_stream_t stream) {
    if (!net || !X || !Y || n < 1) return mfail(net, ABS_ERR_ARG, "bad argument");
    if (abs_mlp_device_fault(net)) return mfail(net, ABS_ERR_TIMEOUT, "a tensor-core product gave up waiting");
    cudaStream_t st = (cudaStream_t)stream;
    abs_status r;
    if ((r = ensure_cap(net, n)) != ABS_OK) return r;
    if (!net->lacc) {
        MCK(cudaMalloc(&net->lacc, sizeof(double) * 64));
        net->lacc_cap = 64;
    }
    if ((r = forward_rows(net, X, n, true, nullptr, st)) != ABS_OK) return r;
    if ((r = backward_rows(net, Y, n, net->lacc, 1.0, false, st)) != ABS_OK) return r;
    if (grad) MCK(cudaMemcpyAsync(grad, net->grad, sizeof(float) * NPAR, cudaMemcpyDeviceToDevice, st));
    double l = 0.0;
    MCK(cudaMemcpyAsync(&l, net->lacc, sizeof(double), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    if (loss) *loss = l;
    return ABS_OK;
}

void abs_default_train_options(abs_train_options* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->epochs = 200;
    o->batch = 512;
    o->lr = 1e-3;
    o->lr_final = 1e-5;
    o->beta1 = 0.9;
    o->beta2 = 0.999;
    o->eps = 1e-8;
    o->seed = 1;
}

abs_status abs_mlp_train(abs_mlp* net, const float* X, const float* Y, int64_t n, const abs_train_options* opt_in,
                         double* epoch_loss, abs_stream_t stream) {
    if (!net || !X || !Y || n < 1) return mfail(net, ABS_ERR_ARG, "bad argument");
    if (abs_mlp_device_fault(net)) return mfail(net, ABS_ERR_TIMEOUT, "a tensor-core product gave up waiting");
    abs_train_options o;
    if (opt_in) o = *opt_in;
    else abs_default_train_options(&o);
    if (o.epochs < 1 || o.batch < 1 || !(o.lr > 0) || !(o.lr_final > 0) || !(o.beta1 >= 0 && o.beta1 < 1) ||
        !(o.beta2 >= 0 && o.beta2 < 1) || !(o.eps > 0) || n > INT32_MAX)
        return mfail(net, ABS_ERR_ARG, "bad training option");
    cudaStream_t st = (cudaStream_t)stream;
    abs_status r;
    const int64_t B = std::min<int64_t>(o.batch, n);
    if ((r = ensure_cap(net, B)) != ABS_OK) return r;
    if (net->perm_cap < n) {
        cudaFree(net->perm);
        net->perm = nullptr;
        MCK(cudaMalloc(&net->perm, sizeof(int) * n));
        net->perm_cap = n;
    }
    if (net->lacc_cap < o.epochs) {
        cudaFree(net->lacc);
        net->lacc = nullptr;
        MCK(cudaMalloc(&net->lacc, sizeof(double) * o.epochs));
        net->lacc_cap = o.epochs;
    }
    std::vector<int> perm(n);
    uint64_t rs = o.seed;
    for (int e = 0; e < o.epochs; ++e) {
        // this epoch's order: Fisher-Yates shuffle with splitmix64 draws
        for (int64_t i = 0; i < n; ++i) perm[i] = (int)i;
        for (int64_t i = n - 1; i > 0; --i) {
            const int64_t j = (int64_t)(splitmix64(rs) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        // the copy reads perm before this host loop writes it again (synchronised below)
        MCK(cudaMemcpyAsync(net->perm, perm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
        const double lr =
            o.epochs > 1 ? o.lr * std::pow(o.lr_final / o.lr, (double)e / (double)(o.epochs - 1)) : o.lr;
        bool first = true;
        for (int64_t b0 = 0; b0 < n; b0 += B) {
            const int64_t nb = std::min<int64_t>(B, n - b0);
            gather_rows_kernel<<<grid1(nb * NIN), 256, 0, st>>>(nb, NIN, net->perm + b0, X, net->xb);
            if ((r = mlaunch(net)) != ABS_OK) return r;
            gather_rows_kernel<<<grid1(nb * NOUT), 256, 0, st>>>(nb, NOUT, net->perm + b0, Y, net->ybt);
            if ((r = mlaunch(net)) != ABS_OK) return r;
            if ((r = forward_rows(net, net->xb, nb, true, nullptr, st)) != ABS_OK) return r;
            if ((r = backward_rows(net, net->ybt, nb, net->lacc + e, (double)nb / (double)n, !first, st)) != ABS_OK)
                return r;
            first = false;
            net->step++;
            const double c1 = 1.0 - std::pow(o.beta1, (double)net->step);
            const double c2 = 1.0 - std::pow(o.beta2, (double)net->step);
            adam_kernel<<<grid1(NPAR), 256, 0, st>>>(NPAR, net->theta, net->grad, net->m, net->v, (float)lr,
                                                     (float)o.beta1, (float)o.beta2, (float)o.eps, (float)c1,
                                                     (float)c2, net->wb);
            if ((r = mlaunch(net)) != ABS_OK) return r;
        }
        MCK(cudaStreamSynchronize(st));
    }
    if (epoch_loss)
        MCK(cudaMemcpyAsync(epoch_loss, net->lacc, sizeof(double) * o.epochs, cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    return ABS_OK;
}

}  // extern "C"
