// absorber_lib.cu -- C ABI (include/absorber.h) of the GB300 absorber design library:
// problem setup, the fused evaluation kernel, the block-LU / Schur-on-d KKT factor and
// solve with FP64 refinement, and the interior-point engine for one problem or a batch
// of independent problems.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <initializer_list>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>
#include <string>
#include <vector>

#include "absorber.h"
#include "kernels.cuh"
#include "kernels_warp.cuh"
#include "kernels_tc.cuh"
#include "vec_kernels.cuh"
#include "kernels_ldl.cuh"

using namespace absorber;

// ======================================================================================
// sparsity pattern (host): derived from the stage routine itself
// ======================================================================================
namespace {

const int kThr = 128;     // threads per block of the (scenario, stage) kernels

thread_local std::string g_err = "no error";

struct PatternTables {
    short slotJ[3][NR][NLOC];
    int segJ[N_STAGES + 1];
    short slotH[NV][NV];
    Ent own[3][MAXOWN], abv[3][MAXABV], blw[3][MAXBLW], hes[NHS];
    int nown[3], nabv[3], nblw[3], dslot[3];
    // the same entries grouped by destination (see kernels.cuh)
    short ownRp[3][NV + 1], abvRp[3][NV + 1], blwRp[3][NV + 1];
    Ent ownC[3][MAXOWN], abvC[3][MAXABV], blwC[3][MAXBLW];
    short ownCp[3][NV + 1], abvCp[3][NV + 1], blwCp[3][NV + 1];
    Ent hesF[2 * NHS];
    short hesFp[NV + 1];
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
    // destination-grouped copies: row pointers of the (row-ordered) tables, and copies
    // ordered by the unknown they feed in J^T y (own column, abv_var, blw_var)
    auto rowptr = [](const Ent* tab, int cnt, short* ptr) {
        for (int r = 0; r <= NV; ++r) {
            int k = 0;
            while (k < cnt && tab[k].r < r) ++k;
            ptr[r] = (short)k;
        }
    };
    auto bydest = [](const Ent* tab, int cnt, int kind, Ent* out, short* ptr) {
        auto dest = [kind](const Ent& e) { return kind == 0 ? (int)e.c : (kind == 1 ? abv_var(e.c) : blw_var(e.c)); };
        int m = 0;
        for (int j = 0; j < NV; ++j) {
            ptr[j] = (short)m;
            for (int k = 0; k < cnt; ++k)
                if (dest(tab[k]) == j) out[m++] = tab[k];
        }
        ptr[NV] = (short)m;
    };
    for (int t = 0; t < 3; ++t) {
        auto rowsorted = [](const Ent* tab, int cnt) {
            for (int k = 1; k < cnt; ++k)
                if (tab[k].r < tab[k - 1].r) return false;
            return true;
        };
        if (!rowsorted(T.own[t], T.nown[t]) || !rowsorted(T.abv[t], T.nabv[t]) || !rowsorted(T.blw[t], T.nblw[t])) {
            err = "stage table not in row order";
            return false;
        }
        rowptr(T.own[t], T.nown[t], T.ownRp[t]);
        rowptr(T.abv[t], T.nabv[t], T.abvRp[t]);
        rowptr(T.blw[t], T.nblw[t], T.blwRp[t]);
        for (int r = 0; r < NV; ++r)
            if (T.blwRp[t][r + 1] - T.blwRp[t][r] > 6) {   // one entry per unknown of the stage below
                err = "coupling row with more than 6 entries";
                return false;
            }
        for (int j = 0; j < NBLW; ++j) {
            int cnt = 0;
            for (int q = 0; q < T.nblw[t]; ++q) cnt += T.blw[t][q].c == j;
            if (cnt > 8) {   // the transposed block solve sums at most 8 entries per unknown
                err = "coupling column with more than 8 entries";
                return false;
            }
        }
        bydest(T.own[t], T.nown[t], 0, T.ownC[t], T.ownCp[t]);
        bydest(T.abv[t], T.nabv[t], 1, T.abvC[t], T.abvCp[t]);
        bydest(T.blw[t], T.nblw[t], 2, T.blwC[t], T.blwCp[t]);
    }
    // the symmetric Hessian block expanded to both triangles, grouped by row
    {
        int m = 0;
        for (int r = 0; r < NV; ++r) {
            T.hesFp[r] = (short)m;
            for (int k = 0; k < NHS; ++k) {
                const Ent& e = T.hes[k];
                if (e.r == r) T.hesF[m++] = e;
                else if (e.c == r) {
                    Ent f = e;
                    f.r = e.c;
                    f.c = e.r;
                    T.hesF[m++] = f;
                }
            }
        }
        T.hesFp[NV] = (short)m;
    }
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
std::mutex g_upload_mu;   // handles may be created from several host threads

cudaError_t upload_tables(int dev) {
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_upload_mu);
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
    UP(c_ownRp, T.ownRp);
    UP(c_abvRp, T.abvRp);
    UP(c_blwRp, T.blwRp);
    UP(c_ownC, T.ownC);
    UP(c_abvC, T.abvC);
    UP(c_blwC, T.blwC);
    UP(c_ownCp, T.ownCp);
    UP(c_abvCp, T.abvCp);
    UP(c_blwCp, T.blwCp);
    UP(c_hesF, T.hesF);
    UP(c_hesFp, T.hesFp);
    {
        static LaneTables lt;
        std::memset(&lt, 0, sizeof(lt));
        std::memcpy(lt.own, T.own, sizeof(lt.own));
        std::memcpy(lt.abv, T.abv, sizeof(lt.abv));
        std::memcpy(lt.blw, T.blw, sizeof(lt.blw));
        for (int t = 0; t < 3; ++t) {
            for (int r = 0; r <= NV; ++r) lt.blwRp[t][r] = T.blwRp[t][r];
            int m = 0;
            for (int j = 0; j < NV; ++j) {
                lt.blwCp[t][j] = (short)m;
                for (int q = 0; q < T.nblw[t]; ++q)
                    if (blw_var(T.blw[t][q].c) == j) lt.blwQ[t][m++] = (unsigned char)q;
            }
            lt.blwCp[t][NV] = (short)m;
        }
        UP(g_lt, lt);
    }
#undef UP
    g_uploaded[dev] = true;
    return cudaSuccess;
}

}  // namespace

// ---- state of the interior-point method on the device (engine.inc) -----------------------
namespace {
// the method's scalar options, passed by value to the control kernels
struct DevOpt {
    double tol, mu_init, kappa_eps, kappa_mu, theta_mu, tau_min, s_max, kappa_sigma, bound_push, bound_frac;
    double gamma_theta, gamma_phi, delta, s_theta, s_phi, eta_phi, gamma_alpha, lam_init_max;
    double dw0, dw_min, dw_max, kw_minus, kw_plus, kw_plus_bar, kappa_soc, obj_scaling, refine_tol;
    double dlo, dhi, u_max;
    double dc_bar, kappa_c;     // delta_c = dc_bar mu^kappa_c when a pivot is zero (block LDL^T)
    double wsec[KSEC];          // objective weights of the design entries
    int max_iter, max_refine, max_ls, soc_max, resto_max, kkt, nsec;
};

// one problem's state of the method
struct DState {
    int status, iters, ls_trials, soc_steps, inertia_corr, refine_steps, fallbacks, esc_scen;
    int have_theta0, tiny, ftype, soc_taken, ls, nls, nsoc, soc_new, nfilt, stepped;
    int resto, resto_it, resto_bt, resto_phases, resto_now;   // feasibility restoration state
    double w, mu, tau, theta_max, theta_min, dw_last;
    // the design vector (section diameters; one entry for the single d) and its bound
    // multipliers, slacks, steps
    double d[KSEC], zLd[KSEC], zUd[KSEC], jtl_d[KSEC], sld[KSEC], sud[KSEC], dd[KSEC];
    double dzLd[KSEC], dzUd[KSEC], sd[KSEC], Kdd[KSEC], rd[KSEC];
    double theta_k, ra, th_r, blog_r;              // restoration: entry theta, step, trial theta / logs
    double E0, inf_pr, inf_du, theta, phi;
    double a_max, a_z, gphi, alpha, a_min, a0, th_old, a_soc, ct_coef;
    double dw, Sd, S01, S11, resid;                // Sd (and S01, S11): the design Schur complement
    int ic_trial;                                  // Algorithm IC trial of the block LDL^T path
    double dc;                                     // its delta_c of the iteration
    // the learned start's acceptance test at the first evaluation: the inlet-copy start's
    // (E_0, theta) and the learned start's
    double gate_E0, gate_theta, first_E0, first_theta;
    // the switching condition's powers at the iterate, for every trial of its line search:
    // (-grad phi . d)^s_phi (when negative) and delta theta^s_theta
    double pw_phi, pw_th;
};

// state shared by the problems of a run
struct DGlobal {
    int k;              // iteration
    int rk;             // refinement round of the current solve (shared, as the launches are)
    int esc_any;        // an FP64 escalation took place in this iteration
    int guard_iter, guard_ls;   // executions of the iteration / line-search loop bodies
    int esc_blocks;     // blocks of esc_kernel done (its last block decides; reset there)
    int lsfac;          // the stored factors of J are those of the least-squares estimate at x
    int fac_skip;       // the Newton step's factorization keeps them (iteration 0 only)
    long long launches; // kernels of this library launched by graph execution
};
}  // namespace

// kernel profiler (options.profile): event pairs around each hot-kernel launch
struct Prof {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    std::vector<std::pair<int, size_t>> marks;   // (kernel id, index of its start event)
    size_t used = 0;
};

constexpr int KMAX = 10;         // partial values per (scenario, stage) thread, at most
constexpr int PS_RING = 16;      // pinned staging buffers for per-problem scalar uploads
constexpr int CHUNK = RED_CHUNK;  // reduction elements per chunk

struct abs_problem {
    int dev = 0;
    int64_t S = 0, ld = 0;       // scenario slots in use and leading dimension
    Params P;
    abs_params aparams;
    std::vector<double> prob;
    std::string err = "no error";
    int nnzJ = 0, nnzH = 0;
    double* feed = nullptr;      // device [18][ld]
    std::vector<double> hfeed;   // host [18][S]
    // the problems this handle holds: one, or P independent ones (a batch)
    int NP = 1;
    std::vector<int> off;        // NP + 1 slot offsets (problem p owns slots [off[p], off[p+1]))
    int* pid = nullptr;          // device problem index per slot (null when NP == 1)
    // workspaces (allocated on first use)
    double* jac = nullptr;       // nnzJ * ld
    double* hes = nullptr;       // nnzH * ld
    double* vec = nullptr;       // pool of primal-size vectors
    void* LUp[2] = {nullptr, nullptr};   // factors per precision [ABS_PREC_FP64], [ABS_PREC_FP32]
    void* Gp[2] = {nullptr, nullptr};
    void* LU = nullptr;
    void* G = nullptr;
    unsigned char* piv = nullptr;
    int* sing = nullptr;
    double* part = nullptr;      // per-thread partials [KMAX][N_STAGES][ld]
    int* chunks = nullptr;       // [nchunk][5]: problem, slot offset, slots, first, last element
    int nchunk = 0;
    int* pchunk = nullptr;       // [NP + 1]
    double* cred = nullptr;      // [KMAX][nchunk]
    int* rcnt = nullptr;         // [NP] chunk arrivals of the running reduction (zero between launches)
    double* red = nullptr;       // [KMAX][NP]
    double* hred = nullptr;      // pinned [KMAX + 2][NP] staging for scalar copies
    double* hmap = nullptr;      // pinned, device-mapped [RED_KMAX + 1][NP]: fetched reductions
    double* hmap_dev = nullptr;  // (the reduction kernel writes them straight to host memory)
    double* ps = nullptr;        // device per-problem scalars [PS_NFIELDS][NP]
    double* hps = nullptr;       // host values of ps
    double* hring = nullptr;     // pinned staging ring [PS_RING][PS_NFIELDS][NP]
    int ring_next = 0;
    long long ring_epoch[PS_RING] = {0};
    long long sync_epoch = 1;
    // factorization kept for kkt_solve (single-problem API)
    struct {
        bool valid = false;
        int prec = 0;
        const double* jac = nullptr;
        const double* hes = nullptr;
        const double* sig = nullptr;
        double d = 0.0, dw = 0.0, dc = 0.0, Kdd = 0.0, A0 = 0.0, Q2 = 0.0, Sd = 0.0;
        bool ldl = false;            // factored by the block LDL^T (kernels_ldl.cuh)
    } fac;
    double* ldl_inv = nullptr;       // [S][N_STAGES][44][44] inverses of the block LDL^T pivot blocks
    Prof prof;
    int autotune = 1;                // tile autotuner on (options.autotune)
    int factor_tile = 0;             // forced FP32 factor shape (options.factor_tile; 0: none)
    int factor_kernel = 0;           // FP32 factor: 0 Gauss-Jordan on the FP32 pipes, 1 tensor-core panels
    // the engine's own stream (stream capture needs a non-default stream) and the event
    // that orders it after the caller's stream
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr;
    cudaEvent_t ev_b[2] = {nullptr, nullptr};   // around the expected-value start's run
    // whole runs of the method captured into CUDA graphs (engine.inc), by configuration
    struct RunGraph {
        std::vector<char> key;
        int eager_runs = 0;          // eager runs of this configuration (capture on the second)
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<RunGraph> rgraphs;
    std::vector<cudaStream_t> cap;   // capture streams of conditional bodies, by depth
    int64_t graph_replays = 0;
    // the method's state on the device
    DState* dst = nullptr;           // [NP]
    DGlobal* dglob = nullptr;
    double* gate = nullptr;          // [2][NP] the inlet-copy start's E_0 and theta (learned-start test)
    double* filt = nullptr;          // [NP][fcap][2]
    int fcap = 0;
    int* esc = nullptr;              // [ld] per-scenario FP64 escalation flags of the iteration
    int* escn = nullptr;             // [NP] escalated scenarios per problem (reset by the control kernel)
    int* doff = nullptr;             // [NP + 1] slot offsets of the problems
    int* hcond = nullptr;            // mapped host memory: conditions of eager runs
    int* hcond_dev = nullptr;
    int tile[4] = {4, 4, 4, 4};      // warps per block last used: factor, solve, solve x2, solve^T
    int64_t nlaunch = 0;         // kernels launched (every launch is followed by launch_check)
    int64_t kcount[ABS_N_KINDS] = {0};   // ... by kind
    float* mlp_x = nullptr;          // learned warm start: network inputs [ld][3] and outputs [ld][440]
    float* mlp_y = nullptr;
    double* wd0 = nullptr;           // learned warm start: its d0 (device)
    // bound multipliers of d at the end of the last engine run, per problem, of the scaled
    // problem, and each problem's objective scaling w (absorber_bound_multipliers)
    std::vector<double> zLd_last, zUd_last, w_last;
    bool sol_valid = false;
    abs_problem* base = nullptr;     // expected-value sub-problem(s) for the starting point
    abs_problem* batch = nullptr;    // cached batch handle of ipm_solve_batched (on probs[0])
    abs_problem* aux = nullptr;      // ipm_solve_learned: the inlet-copy start's evaluation (same problem)
    cudaEvent_t gate_ev = nullptr;   // recorded after that evaluation's (E_0, theta) reached gate
    std::vector<int64_t> batch_key;  // the sizes it was built for
};

namespace {

// vector pool indices (each NSC * ld + ld doubles; the problems' d slots at NSC * ld + p)
enum {
    V_X, V_LAM, V_ZL, V_ZU, V_C, V_JTL, V_SIG, V_RZ, V_RC, V_P, V_Q, V_DZ, V_DL, V_DZL, V_DZU,
    V_G, V_RHOZ, V_RHOC, V_CZ, V_CL, V_ONE, V_CT, V_RCS, V_RCN, V_SZ, V_SL, V_HQ, V_T, V_IL, V_IU, V_QL, V_Q1, V_HQ1,
    V_COUNT
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

// vector length: the scenario entries, then room for every problem's design entries
// (problem p's section k at NSC ld + k NP + p)
int64_t vsize(const abs_problem* h) { return (int64_t)NSC * h->ld + (int64_t)h->P.nsec * h->ld; }
double* V(abs_problem* h, int k) { return h->vec + (int64_t)k * vsize(h); }
dim3 grid2(const abs_problem* h) { return dim3((unsigned)((h->S + kThr - 1) / kThr), N_STAGES); }
// the trial evaluation (FP64-pipe-bound, limited by registers) in 32-thread blocks: the
// blocks spread more evenly over the SMs (measured 7 % faster; the full evaluation is not)
constexpr int EVAL_T = 32;
dim3 geval(const abs_problem* h) { return dim3((unsigned)((h->S + EVAL_T - 1) / EVAL_T), N_STAGES); }
// elementwise kernels: one thread per (entry, scenario)
dim3 gride(const abs_problem* h) { return dim3((unsigned)((h->S + kThr - 1) / kThr), NSC); }
// kernels with QS threads per (scenario, stage)
dim3 gridq(const abs_problem* h) { return dim3((unsigned)((h->S + QS_SCEN - 1) / QS_SCEN), N_STAGES); }
dim3 gridw(const abs_problem* h, int wpb) { return dim3((unsigned)((h->S + wpb - 1) / wpb)); }
BView view(const abs_problem* h) { return BView{h->pid, h->ps, h->NP}; }
double& PSV(abs_problem* h, int field, int p) { return h->hps[(size_t)field * h->NP + p]; }

// kernel kinds of abs_result.kind_launches (include/absorber.h, ABS_N_KINDS)
enum {
    KD_EVAL = 0, KD_EVAL_TRIAL, KD_FACTOR, KD_SOLVE, KD_SOLVE_T, KD_RESIDUAL, KD_SCHUR, KD_DUAL, KD_REDUCE, KD_RHS,
    KD_DZ, KD_STEP, KD_ACCEPT, KD_VEC, KD_CTL, KD_EVAL_JAC
};

// after every launch: count it (by kind; a reduction counts its planes) and check it
abs_status launch_check(abs_problem* h, int kind = KD_VEC, int weight = 1) {
    if (h) {
        h->nlaunch++;
        h->kcount[kind] += weight;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, ABS_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return ABS_OK;
}

enum { K_EVAL = 0, K_EVAL_TRIAL = 1, K_FACTOR = 2, K_SOLVE = 3, K_SOLVE_T = 4 };
enum { TK_FACTOR = 0, TK_SOLVE1 = 1, TK_SOLVE2 = 2, TK_SOLVE_T = 3 };

cudaEvent_t prof_event(abs_problem* h) {
    auto& p = h->prof;
    if (p.used == p.pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        p.pool.push_back(e);
    }
    return p.pool[p.used++];
}

void prof_begin(abs_problem* h, int kid, cudaStream_t st) {
    if (!h->prof.on) return;
    h->prof.marks.push_back({kid, h->prof.used});
    cudaEventRecord(prof_event(h), st);
}

void prof_end(abs_problem* h, cudaStream_t st) {
    if (!h->prof.on) return;
    cudaEventRecord(prof_event(h), st);
}

abs_status ensure_buffers(abs_problem* h) {
    if (h->vec) return ABS_OK;
    const int64_t ld = h->ld;
    CK(cudaMalloc(&h->jac, sizeof(double) * (size_t)h->nnzJ * ld));
    CK(cudaMalloc(&h->hes, sizeof(double) * (size_t)h->nnzH * ld));
    CK(cudaMalloc(&h->vec, sizeof(double) * (size_t)vsize(h) * V_COUNT));
    CK(cudaMemset(h->vec, 0, sizeof(double) * (size_t)vsize(h) * V_COUNT));
    CK(cudaMalloc(&h->piv, (size_t)N_STAGES * PIV_BYTES * ld));
    CK(cudaMalloc(&h->sing, sizeof(int) * (size_t)ld));
    CK(cudaMemset(h->sing, 0, sizeof(int) * (size_t)ld));
    CK(cudaMalloc(&h->part, sizeof(double) * (size_t)KMAX * N_STAGES * ld));
    // reduction chunks: each problem's (stage, slot) elements in pieces of CHUNK
    std::vector<int> ch, pc(h->NP + 1, 0);
    for (int p = 0; p < h->NP; ++p) {
        pc[p] = (int)(ch.size() / 5);
        const int Sp = h->off[p + 1] - h->off[p];
        const int E = N_STAGES * Sp;
        for (int i0 = 0; i0 < E; i0 += CHUNK) {
            ch.push_back(p);
            ch.push_back(h->off[p]);
            ch.push_back(Sp);
            ch.push_back(i0);
            ch.push_back(std::min(E, i0 + CHUNK));
        }
    }
    pc[h->NP] = (int)(ch.size() / 5);
    h->nchunk = pc[h->NP];
    CK(cudaMalloc(&h->chunks, sizeof(int) * ch.size()));
    CK(cudaMemcpy(h->chunks, ch.data(), sizeof(int) * ch.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&h->pchunk, sizeof(int) * pc.size()));
    CK(cudaMemcpy(h->pchunk, pc.data(), sizeof(int) * pc.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&h->cred, sizeof(double) * (size_t)KMAX * h->nchunk));
    CK(cudaMalloc(&h->rcnt, sizeof(int) * (size_t)h->NP));
    CK(cudaMemset(h->rcnt, 0, sizeof(int) * (size_t)h->NP));
    CK(cudaMalloc(&h->red, sizeof(double) * (size_t)KMAX * h->NP));
    CK(cudaMallocHost(&h->hred, sizeof(double) * (size_t)(KMAX + 2) * h->NP));
    CK(cudaHostAlloc(&h->hmap, sizeof(double) * (size_t)(RED_KMAX + 1) * h->NP, cudaHostAllocMapped));
    CK(cudaHostGetDevicePointer(&h->hmap_dev, h->hmap, 0));
    CK(cudaMalloc(&h->ps, sizeof(double) * (size_t)PS_NFIELDS * h->NP));
    h->hps = new double[(size_t)PS_NFIELDS * h->NP]();
    CK(cudaMallocHost(&h->hring, sizeof(double) * (size_t)PS_RING * PS_NFIELDS * h->NP));
    for (int p = 0; p < h->NP; ++p) {
        PSV(h, PS_ACT, p) = 1.0;
        PSV(h, PS_LSACT, p) = 1.0;
        PSV(h, PS_SD, p) = 1.0;
    }
    return ABS_OK;
}

abs_status ensure_stream(abs_problem* h) {
    if (h->stream) return ABS_OK;
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreate(&h->ev_b[0]));
    CK(cudaEventCreate(&h->ev_b[1]));
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
    return ABS_OK;
}

// the block LDL^T's inverses (allocated on first use) and its kernels' shared memory
abs_status ensure_ldl(abs_problem* h) {
    if (!h->ldl_inv) {
        CK(cudaMalloc(&h->ldl_inv, sizeof(double) * (size_t)LDL_BLOCK * N_STAGES * h->S));
        CK(cudaFuncSetAttribute(ldl_factor_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)LDL_FACTOR_SMEM));
    }
    return ABS_OK;
}

// host synchronisation point: every copy issued before it has completed
abs_status sync(abs_problem* h, cudaStream_t st) {
    CK(cudaStreamSynchronize(st));
    h->sync_epoch++;
    return ABS_OK;
}

// copy the per-problem scalars to the device through a pinned staging slot that no
// pending copy still reads
abs_status upload_ps(abs_problem* h, cudaStream_t st) {
    const size_t n = (size_t)PS_NFIELDS * h->NP;
    const int slot = h->ring_next;
    h->ring_next = (h->ring_next + 1) % PS_RING;
    if (h->ring_epoch[slot] == h->sync_epoch) {
        abs_status r = sync(h, st);
        if (r != ABS_OK) return r;
    }
    double* stage = h->hring + (size_t)slot * n;
    std::memcpy(stage, h->hps, sizeof(double) * n);
    CK(cudaMemcpyAsync(h->ps, stage, sizeof(double) * n, cudaMemcpyHostToDevice, st));
    h->ring_epoch[slot] = h->sync_epoch;
    return ABS_OK;
}

RedOps make_ops(std::initializer_list<int> l) {
    RedOps o;
    int i = 0;
    for (int v : l) o.op[i++] = v;
    for (; i < 12; ++i) o.op[i] = RSUM;
    return o;
}

// combine the K partial planes per problem (device result in h->red[k][p]); with fetch,
// the reduction kernel also writes them (and the problems' d slots of `dslots`, if given)
// to mapped host memory, read after one stream synchronization (no copy round trip)
abs_status reduce(abs_problem* h, cudaStream_t st, int K, const RedOps& ops, int flag, bool fetch,
                  const double* dslots = nullptr) {
    double* hout = fetch ? h->hmap_dev : nullptr;
    const double* ds = fetch ? dslots : nullptr;
    switch (K) {
#define RK(k)                                                                                                      \
    case k:                                                                                                        \
        reduce_kernel<k><<<(unsigned)h->nchunk, RED_T, 0, st>>>(h->part, h->ld, ops, h->chunks, h->nchunk, h->pchunk, \
                                                                 h->ps, h->NP, flag, h->cred, h->rcnt, h->red, hout, ds); \
        break;
        RK(1) RK(2) RK(3) RK(4) RK(5) RK(6) RK(7) RK(8) RK(9) RK(10)
#undef RK
        default: return fail(h, ABS_ERR_ARG, "reduction with more than 10 planes");
    }
    abs_status r = launch_check(h, KD_REDUCE, K);
    if (r != ABS_OK) return r;
    if (!fetch) return ABS_OK;
    return sync(h, st);
}

double RED(const abs_problem* h, int k, int p) { return h->hmap[(size_t)k * h->NP + p]; }

// ---- the KKT machinery (every active problem at once) ----------------------------------
// factor precision of a KKT system: ABS_PREC_FP64, ABS_PREC_FP32, or mixed -- the FP32
// stage-block inverses of most scenarios with FP64 LU factors of the scenarios escalated
// in this iteration (esc flags)
constexpr int ABS_PREC_MIXED = 2;

struct KKTSys {
    const double* jac = nullptr;
    const double* hes = nullptr;
    const double* sig = nullptr;
    bool use_w = true;
    int prec = ABS_PREC_FP64;
    // block LDL^T of every scenario block (FP64, dw = PS_DW, dc = PS_DC) instead of the
    // block LU of J_s
    bool ldl = false;
    // set before kkt_factor_core: p = J^-1 rc is solved together with q = J^-1 b (one
    // two-right-hand-side launch) and the first KKT solve with this rc reuses it
    const double* pre_rc = nullptr;
    // with pre_rc (one design entry): the Schur pass of kkt_factor_core also forms the
    // right-hand-side sums of the first solve with this rz (q^T (rz - H p), q^T p and
    // t = rz - H p; they do not depend on dw), so that solve skips its own Schur pass
    const double* pre_rz = nullptr;
    // device flag: when set, kkt_factor_core keeps the stored factors of J (those of the
    // least-squares multiplier estimate at the same point)
    const int* skip = nullptr;
};

// ---- block-tile autotuner ----------------------------------------------------------------
// The warp kernels run one scenario per warp; how many warps share a block (and with it
// the block's static shared memory) sets the resident blocks per SM and the tail of the
// last wave.  The first launch of a kernel kind, precision and size bucket (powers of
// two of S) on a device times every candidate (best of two timings) on that launch's own data -- each
// candidate computes the same values bit for bit, one warp per scenario -- and keeps the
// fastest for every later launch with that key.  Launches below TUNE_MIN_S scenarios are
// latency-bound and use the default shape.
constexpr int TUNE_MIN_S = 256;
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, int> g_tuned;   // (device, kind, element size, bucket)

int size_bucket(int64_t S) {
    int b = 0;
    while (((int64_t)1 << (b + 1)) <= S) ++b;
    return b;
}

template <class Launch>
abs_status tuned_launch(abs_problem* h, int kind, int es, std::initializer_list<int> cands, int dflt,
                        Launch&& launch, cudaStream_t st) {
    int w = dflt;
    // no timing inside a stream capture (a capture admits no synchronization): an untuned
    // key launches its default shape there
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) cap = cudaStreamCaptureStatusNone;
    if (h->autotune && h->S >= TUNE_MIN_S) {
        const auto key = std::make_tuple(h->dev, kind, es, size_bucket(h->S));
        bool found = false;
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tuned.find(key);
            if (it != g_tuned.end()) {
                w = it->second;
                found = true;
            }
        }
        if (!found && cap != cudaStreamCaptureStatusNone) {
            h->tile[kind] = w;
            return launch(w);
        }
        if (!found) {
            cudaEvent_t e0, e1;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            float best = INFINITY;
            for (int c : cands)
                for (int rep = 0; rep < 2; ++rep) {   // the better of two timings per candidate
                    cudaEventRecord(e0, st);
                    abs_status r = launch(c);
                    cudaEventRecord(e1, st);
                    if (r != ABS_OK) {
                        cudaEventDestroy(e0);
                        cudaEventDestroy(e1);
                        return r;
                    }
                    float ms = 0.f;
                    if (cudaEventSynchronize(e1) == cudaSuccess &&
                        cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) {
                        best = ms;
                        w = c;
                    }
                }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            std::lock_guard<std::mutex> lk(g_tune_mu);
            g_tuned[key] = w;
            h->tile[kind] = w;
            return ABS_OK;   // the candidates' outputs are identical: the last one stands
        }
    }
    h->tile[kind] = w;
    return launch(w);
}

// factor launch shape: W warps per block.  FP32: stage-block inverses and G by
// Gauss-Jordan (factor_gj_kernel); FP64: LU factors, row order and G (factor_warp_kernel),
// of the scenarios with mask[s] != 0 only when mask is given
template <class T, int W>
void factor_w(abs_problem* h, const double* jac, double pivtol, const int* mask, cudaStream_t st,
              const int* skip) {
    if constexpr (std::is_same<T, float>::value) {
        if (h->factor_kernel == 1)
            factor_gj_tc_kernel<W><<<gridw(h, W), 32 * W, 0, st>>>((int)h->S, h->ld, view(h), jac,
                                                                   (float*)h->LUp[ABS_PREC_FP32], h->piv,
                                                                   (float*)h->Gp[ABS_PREC_FP32], h->sing, pivtol);
        else
            factor_gj_kernel<W><<<gridw(h, W), 32 * W, 0, st>>>((int)h->S, h->ld, view(h), jac,
                                                                (float*)h->LUp[ABS_PREC_FP32], h->piv,
                                                                (float*)h->Gp[ABS_PREC_FP32], h->sing, pivtol,
                                                                skip);
    }
    else if constexpr (factor_fits<T, W>())
        factor_warp_kernel<T, W><<<gridw(h, W), 32 * W, 0, st>>>((int)h->S, h->ld, view(h), jac,
                                                                (T*)h->LUp[ABS_PREC_FP64], h->piv,
                                                                (T*)h->Gp[ABS_PREC_FP64], h->sing, pivtol, mask,
                                                                skip);
}

// skip (device flag, optional): when set at run time the launch leaves the stored factors
// as they are (they are those of this Jacobian)
template <class T>
abs_status factor_launch(abs_problem* h, const double* jac, double pivtol, cudaStream_t st,
                         const int* mask = nullptr, const int* skip = nullptr) {
    prof_begin(h, K_FACTOR, st);
    auto go = [&](int w) {
        switch (w) {
            case 1: factor_w<T, 1>(h, jac, pivtol, mask, st, skip); break;
            case 2: factor_w<T, 2>(h, jac, pivtol, mask, st, skip); break;
            case 8: factor_w<T, 8>(h, jac, pivtol, mask, st, skip); break;
            default: factor_w<T, 4>(h, jac, pivtol, mask, st, skip); break;
        }
        return launch_check(h, KD_FACTOR);
    };
    abs_status r;
    if (std::is_same<T, float>::value && h->factor_tile != 0) {
        h->tile[TK_FACTOR] = h->factor_tile;
        r = go(h->factor_tile);
    } else if (std::is_same<T, float>::value)
        r = tuned_launch(h, TK_FACTOR, h->factor_kernel == 1 ? 5 : (int)sizeof(T), {1, 2, 4, 8}, WPB_F, go, st);
    else if (mask)
        r = go(WPB_F);   // the escalation's masked factorization: the default shape
    else
        r = factor_fits<T, 8>() ? tuned_launch(h, TK_FACTOR, sizeof(T), {1, 2, 4, 8}, WPB_F, go, st)
                                : tuned_launch(h, TK_FACTOR, sizeof(T), {1, 2, 4}, WPB_F, go, st);
    prof_end(h, st);
    return r;
}

template <class T, int NR_, int W>
void solve_w(abs_problem* h, const double* jac, const double* x, const double* r0, const double* r1, double* o0,
             double* o1, cudaStream_t st, int bsec) {
    const int pi = std::is_same<T, float>::value ? ABS_PREC_FP32 : ABS_PREC_FP64;
    solve_warp_kernel<T, NR_, W, std::is_same<T, float>::value><<<gridw(h, W), 32 * W, 0, st>>>(
        h->P, (int)h->S, h->ld, view(h), jac, (const T*)h->LUp[pi], h->piv, (const T*)h->Gp[pi], x, r0, r1, o0, o1,
        bsec);
}

// bsec: the design entry whose border column a null right-hand side stands for
template <class T, int NR_>
abs_status solve_launch(abs_problem* h, const double* jac, const double* x, const double* r0, const double* r1,
                        double* o0, double* o1, cudaStream_t st, int bsec = 0) {
    prof_begin(h, K_SOLVE, st);
    auto go = [&](int w) {
        switch (w) {
            case 1: solve_w<T, NR_, 1>(h, jac, x, r0, r1, o0, o1, st, bsec); break;
            case 2: solve_w<T, NR_, 2>(h, jac, x, r0, r1, o0, o1, st, bsec); break;
            case 8: solve_w<T, NR_, 8>(h, jac, x, r0, r1, o0, o1, st, bsec); break;
            default: solve_w<T, NR_, 4>(h, jac, x, r0, r1, o0, o1, st, bsec); break;
        }
        return launch_check(h, KD_SOLVE);
    };
    abs_status r = tuned_launch(h, NR_ == 1 ? TK_SOLVE1 : TK_SOLVE2, sizeof(T), {1, 2, 4, 8}, WPB_S, go, st);
    prof_end(h, st);
    return r;
}

// mixed factor precision (escalated scenarios FP64, the others FP32), default shape
template <int NR_>
abs_status solve_mixed(abs_problem* h, const double* jac, const double* x, const double* r0, const double* r1,
                       double* o0, double* o1, cudaStream_t st, int bsec = 0) {
    prof_begin(h, K_SOLVE, st);
    solve_mixed_kernel<NR_, WPB_S><<<gridw(h, WPB_S), 32 * WPB_S, 0, st>>>(
        h->P, (int)h->S, h->ld, view(h), jac, (const float*)h->LUp[ABS_PREC_FP32], (const double*)h->LUp[ABS_PREC_FP64],
        h->piv, (const float*)h->Gp[ABS_PREC_FP32], (const double*)h->Gp[ABS_PREC_FP64], h->esc, x, r0, r1, o0, o1,
        bsec);
    prof_end(h, st);
    return launch_check(h, KD_SOLVE);
}

abs_status solve_j(abs_problem* h, int prec, const double* jac, const double* x, const double* r0, double* o0,
                   cudaStream_t st, int bsec = 0) {
    if (prec == ABS_PREC_MIXED) return solve_mixed<1>(h, jac, x, r0, nullptr, o0, nullptr, st, bsec);
    if (prec == ABS_PREC_FP32) return solve_launch<float, 1>(h, jac, x, r0, nullptr, o0, nullptr, st, bsec);
    return solve_launch<double, 1>(h, jac, x, r0, nullptr, o0, nullptr, st, bsec);
}

// two right-hand sides in one launch (a null r means b = dc/dd)
abs_status solve_j2(abs_problem* h, int prec, const double* jac, const double* x, const double* r0, const double* r1,
                    double* o0, double* o1, cudaStream_t st) {
    if (prec == ABS_PREC_MIXED) return solve_mixed<2>(h, jac, x, r0, r1, o0, o1, st);
    if (prec == ABS_PREC_FP32) return solve_launch<float, 2>(h, jac, x, r0, r1, o0, o1, st);
    return solve_launch<double, 2>(h, jac, x, r0, r1, o0, o1, st);
}

template <class T, int W>
void solve_t_w(abs_problem* h, const double* jac, const double* g, double* out, cudaStream_t st) {
    const int pi = std::is_same<T, float>::value ? ABS_PREC_FP32 : ABS_PREC_FP64;
    solve_t_warp_kernel<T, W, std::is_same<T, float>::value><<<gridw(h, W), 32 * W, 0, st>>>(
        (int)h->S, h->ld, view(h), jac, (const T*)h->LUp[pi], h->piv, (const T*)h->Gp[pi], g, out);
}

template <class T>
abs_status solve_jt_t(abs_problem* h, const double* jac, const double* g, double* out, cudaStream_t st) {
    auto go = [&](int w) {
        switch (w) {
            case 1: solve_t_w<T, 1>(h, jac, g, out, st); break;
            case 2: solve_t_w<T, 2>(h, jac, g, out, st); break;
            case 8: solve_t_w<T, 8>(h, jac, g, out, st); break;
            default: solve_t_w<T, 4>(h, jac, g, out, st); break;
        }
        return launch_check(h, KD_SOLVE_T);
    };
    return tuned_launch(h, TK_SOLVE_T, sizeof(T), {1, 2, 4, 8}, WPB_S, go, st);
}

abs_status solve_jt(abs_problem* h, int prec, const double* jac, const double* g, double* out, cudaStream_t st) {
    prof_begin(h, K_SOLVE_T, st);
    abs_status r;
    if (prec == ABS_PREC_MIXED) {
        solve_t_mixed_kernel<WPB_S><<<gridw(h, WPB_S), 32 * WPB_S, 0, st>>>(
            (int)h->S, h->ld, view(h), jac, (const float*)h->LUp[ABS_PREC_FP32], (const double*)h->LUp[ABS_PREC_FP64],
            h->piv, (const float*)h->Gp[ABS_PREC_FP32], (const double*)h->Gp[ABS_PREC_FP64], h->esc, g, out);
        r = launch_check(h, KD_SOLVE_T);
    } else {
        r = prec == ABS_PREC_FP32 ? solve_jt_t<float>(h, jac, g, out, st) : solve_jt_t<double>(h, jac, g, out, st);
    }
    prof_end(h, st);
    return r;
}

// factor every active problem's J_s, q = J^-1 b (with p = J^-1 pre_rc when set) and the
// Schur sums into h->red per problem: [0] A0 = sum q^T (W + Sigma) q, [1] Q2 = sum q^T q,
// [4] the d-d Hessian entries, [5] singular stage blocks (fetch: also to the host, RED).
// Mixed precision: FP64 factors of the escalated scenarios only (the others keep their
// FP32 inverses).  x: primal vector whose d slots hold the problems' d.
abs_status kkt_factor_core(abs_problem* h, const KKTSys& K, const double* x, cudaStream_t st, bool fetch) {
    abs_status r;
    if (K.ldl) {
        // block LDL^T: the pivot inverses and the inertia counts ([2] positive, [3] negative,
        // [6] zero pivots, [5] scenarios with a zero pivot), then u = K_s^-1 [0; b] with
        // [0] A0 = -sum b^T u_l (so that S_d = K_dd + dw + A0), [1] 0, [4] the d-d entries
        if ((r = ensure_ldl(h)) != ABS_OK) return r;
        ldl_factor_kernel<<<(unsigned)h->S, 32, LDL_FACTOR_SMEM, st>>>((int)h->S, h->ld, view(h), K.jac, K.hes, K.sig,
                                                                       K.use_w, h->ldl_inv, h->part);
        if ((r = launch_check(h, KD_FACTOR)) != ABS_OK) return r;
        ldl_solve_kernel<<<(unsigned)h->S, 32, LDL_SOLVE_SMEM, st>>>((int)h->S, h->ld, view(h), K.jac, h->ldl_inv,
                                                                     nullptr, nullptr, true, V(h, V_Q), V(h, V_QL),
                                                                     h->part, 0, -1.0, true,
                                                                     K.use_w ? K.hes : nullptr);
        if ((r = launch_check(h, KD_SOLVE)) != ABS_OK) return r;
        return reduce(h, st, 7, make_ops({RSUM, RSUM, RSUM, RSUM, RSUM, RSUM, RSUM}), PS_ACT, fetch);
    }
    if (K.prec == ABS_PREC_MIXED) {
        if ((r = ensure_factor(h, ABS_PREC_FP64)) != ABS_OK) return r;
        if ((r = ensure_factor(h, ABS_PREC_FP32)) != ABS_OK) return r;
        r = factor_launch<double>(h, K.jac, 1e-14, st, h->esc);
    } else {
        if ((r = ensure_factor(h, K.prec)) != ABS_OK) return r;
        // FP64: a pivot below 1e-14 of the block's largest entry marks the stage block
        // singular; FP32: only (numerically) zero pivots do -- accuracy is guarded by the
        // FP64 refinement instead, with FP64 escalation where it stalls
        if (K.prec == ABS_PREC_FP32) r = factor_launch<float>(h, K.jac, 1e-30, st, nullptr, K.skip);
        else r = factor_launch<double>(h, K.jac, 1e-14, st, nullptr, K.skip);
    }
    if (r != ABS_OK) return r;
    r = K.pre_rc ? solve_j2(h, K.prec, K.jac, x, K.pre_rc, nullptr, V(h, V_P), V(h, V_Q), st)
                 : solve_j(h, K.prec, K.jac, x, nullptr, V(h, V_Q), st);
    if (r != ABS_OK) return r;
    // a second design entry: q1 = J^-1 b1, b1 the border column of the second section
    const bool two = h->P.nsec == 2;
    if (two && (r = solve_j(h, K.prec, K.jac, x, nullptr, V(h, V_Q1), st, 1)) != ABS_OK) return r;
    if (two)
        schur_kernel<true><<<gridq(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), K.hes, K.sig, K.use_w, nullptr,
                                                       V(h, V_Q), nullptr, h->sing, h->part, SCHUR_DD, V(h, V_HQ),
                                                       nullptr, V(h, V_Q1), V(h, V_HQ1));
    else if (K.pre_rc && K.pre_rz)
        // the matrix sums and the first solve's right-hand-side sums in one pass: planes
        // [0] q^T H q, [1] q^T q, [2] q^T (rz - H p), [3] q^T p, [4] d-d, [5] singular
        schur_kernel<false><<<gridq(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), K.hes, K.sig, K.use_w, V(h, V_P),
                                                        V(h, V_Q), K.pre_rz, h->sing, h->part, SCHUR_DD | SCHUR_RHS,
                                                        V(h, V_HQ), V(h, V_T));
    else
        schur_kernel<false><<<gridq(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), K.hes, K.sig, K.use_w, nullptr,
                                                        V(h, V_Q), nullptr, h->sing, h->part, SCHUR_DD, V(h, V_HQ),
                                                        nullptr);
    if ((r = launch_check(h, KD_SCHUR)) != ABS_OK) return r;
    if (two) return reduce(h, st, 9, make_ops({RSUM, RSUM, RSUM, RSUM, RSUM, RSUM, RSUM, RSUM, RSUM}), PS_ACT, fetch);
    return reduce(h, st, 6, make_ops({RSUM, RSUM, RSUM, RSUM, RSUM, RSUM}), PS_ACT, fetch);
}

// one Schur-reduced solve for every active problem: rz (z part), rc -> dz (d slots set),
// dl.  PS_RD, PS_SD, PS_DW must be on the device.  No host round trip.  have_p: V_P
// already holds J^-1 rc (solved with q in kkt_factor_core).
abs_status kkt_solve_launches(abs_problem* h, const KKTSys& K, const double* x, const double* rz, const double* rc,
                              double* dz, double* dl, cudaStream_t st, bool have_p = false) {
    abs_status r;
    if (K.ldl) {
        // v = K_s^-1 [rz; rc] into dz, dl with [2] b^T v_l ([3] zero), dd, then x = v - u dd
        ldl_solve_kernel<<<(unsigned)h->S, 32, LDL_SOLVE_SMEM, st>>>((int)h->S, h->ld, view(h), K.jac, h->ldl_inv,
                                                                     rz, rc, false, dz, dl, h->part, 2, 1.0, false,
                                                                     nullptr);
        if ((r = launch_check(h, KD_SOLVE)) != ABS_OK) return r;
        if ((r = reduce(h, st, 4, make_ops({RSUM, RSUM, RSUM, RSUM}), PS_ACT, false)) != ABS_OK) return r;
        finalize_dd_kernel<<<(unsigned)((h->NP + 127) / 128), 128, 0, st>>>(h->ld, view(h), h->red, dz);
        if ((r = launch_check(h, KD_VEC)) != ABS_OK) return r;
        ldl_back_kernel<<<dim3((unsigned)((h->S + 127) / 128), N_STAGES), 128, 0, st>>>((int)h->S, h->ld, view(h),
                                                                                       V(h, V_Q), V(h, V_QL), dz, dl);
        return launch_check(h, KD_DZ);
    }
    if (!have_p && (r = solve_j(h, K.prec, K.jac, x, rc, V(h, V_P), st)) != ABS_OK) return r;
    const bool two = h->P.nsec == 2;
    // the Schur pass of kkt_factor_core already formed this solve's sums (h->red [2], [3])
    const bool sums_ready = have_p && !two && K.pre_rc == rc && K.pre_rz == rz;
    if (sums_ready) {
        // nothing: t, hq and the reduced sums are in place
    } else if (two)
        schur_kernel<true><<<gridq(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), K.hes, K.sig, K.use_w, V(h, V_P),
                                                       V(h, V_Q), rz, nullptr, h->part, SCHUR_RHS, nullptr, V(h, V_T),
                                                       V(h, V_Q1), nullptr);
    else
        schur_kernel<false><<<gridq(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), K.hes, K.sig, K.use_w, V(h, V_P),
                                                        V(h, V_Q), rz, nullptr, h->part, SCHUR_RHS, nullptr,
                                                        V(h, V_T));
    if (!sums_ready) {
        if ((r = launch_check(h, KD_SCHUR)) != ABS_OK) return r;
        if ((r = reduce(h, st, 4, make_ops({RSUM, RSUM, RSUM, RSUM}), PS_ACT, false)) != ABS_OK) return r;
    }
    finalize_dd_kernel<<<(unsigned)((h->NP + 127) / 128), 128, 0, st>>>(h->ld, view(h), h->red, dz, h->P.nsec);
    if ((r = launch_check(h, KD_VEC)) != ABS_OK) return r;
    dz_fast_kernel<<<gride(h), kThr, 0, st>>>((int)h->S, h->ld, view(h), V(h, V_P), V(h, V_Q), V(h, V_T),
                                              V(h, V_HQ), dz, V(h, V_G), two ? V(h, V_Q1) : nullptr,
                                              two ? V(h, V_HQ1) : nullptr);
    if ((r = launch_check(h, KD_DZ)) != ABS_OK) return r;
    return solve_jt(h, K.prec, K.jac, V(h, V_G), dl, st);
}

// the paper's layout (Section "Numerical results"): [d, z_1 .. z_S], z_s = per stage x
// over the 11 species, y over the 11 species, L, V, T, the 5 extents (physical units);
// the fixed entries (y of the 7 non-volatile species, x of N2 and O2) exactly 0
__global__ void __launch_bounds__(128) paper_layout_kernel(const Params P, int S, int64_t ld,
                                                           const double* __restrict__ x, double* __restrict__ out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (s >= S) return;
    constexpr int PER = 30;
    double* z = out + 1 + (int64_t)s * (N_STAGES * PER) + PER * n;
    auto xv = [&](int j) { return x[(int64_t)(NV * n + j) * ld + s]; };
#pragma unroll
    for (int k = 0; k < PER; ++k) z[k] = 0.0;
#pragma unroll
    for (int l = 0; l < 9; ++l) z[l] = xv(LX + l) * P.sx[l];
#pragma unroll
    for (int j = 0; j < 4; ++j) z[11 + 7 + j] = xv(LY + j) * P.sy[j];   // CO2, H2O, N2, O2 are species 7..10
    z[22] = xv(LL);
    z[23] = xv(LV);
    z[24] = xv(LT) * P.sT;
#pragma unroll
    for (int r = 0; r < 5; ++r) z[25 + r] = xv(LE + r);
    if (s == 0 && n == 0) out[0] = x[(int64_t)NSC * ld];
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
        const int64_t n = (int64_t)NFEED * ld;
        h->hfeed.resize((size_t)NFEED * S);
        CK(cudaMemcpyAsync(h->hfeed.data(), feeds, sizeof(double) * h->hfeed.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        pad_feed_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((int)S, ld, feeds, h->feed);
        return launch_check(h, KD_VEC);
    }
    std::vector<double> hf((size_t)NFEED * ld, 0.0);
    for (int f = 0; f < NFEED; ++f)
        for (int64_t s = 0; s < ld; ++s) {
            const double v = feeds[(size_t)f * S + (s < S ? s : S - 1)];
            if (!std::isfinite(v)) return fail(h, ABS_ERR_NUMERIC, "non-finite feed value");
            hf[(size_t)f * ld + s] = v;
        }
    h->hfeed.assign(feeds, feeds + (size_t)NFEED * S);
    CK(cudaMemcpyAsync(h->feed, hf.data(), sizeof(double) * hf.size(), cudaMemcpyHostToDevice, st));
    CK(cudaStreamSynchronize(st));
    return ABS_OK;
}

// the device parameter block of a parameter table: the table itself plus the derived
// fields (logarithms of the liquid scales, enthalpy offsets, scaled temperature bounds);
// false if a liquid scale is not positive
bool make_params(const abs_params* p, Params* P) {
    std::memset(P, 0, sizeof(*P));
    std::memcpy(P, p, sizeof(abs_params));
    for (int l = 0; l < 9; ++l) {
        if (!(p->sx[l] > 0.0)) return false;
        P->lnsx[l] = std::log(p->sx[l]);
        for (int k = 0; k < 5; ++k) P->lnsxr[k] += nu(l, k) * P->lnsx[l];
        P->hL0[l] = p->hL_ref[l] + p->hL_dh[l];
    }
    for (int j = 0; j < 4; ++j) P->hV0[j] = p->hV_ref[j] + p->hV_dh[j];
    P->Tlo_s = p->T_lo / p->sT;
    P->Thi_s = p->T_hi / p->sT;
    return p->n_sections >= 1 && p->n_sections <= KSEC;
}

abs_status init_handle(abs_problem* h, const abs_params* p, int64_t S) {
    CK(cudaGetDevice(&h->dev));
    CK(upload_tables(h->dev));
    h->S = S;
    h->ld = (S + 31) / 32 * 32;
    h->aparams = *p;
    if (!make_params(p, &h->P)) return fail(h, ABS_ERR_ARG, "scales must be positive, n_sections 1 or 2");
    const PatternTables& T = pattern();
    h->nnzJ = (int)T.jrow.size();
    h->nnzH = (int)T.hrow.size() + h->P.nsec - 1;   // one d-d entry per section
    h->NP = 1;
    h->off = {0, (int)S};
    CK(cudaMalloc(&h->feed, sizeof(double) * (size_t)NFEED * h->ld));
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
    o->refine_tol = 1e-10;
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
    o->warm_mu_init = 1e-3;
    o->warm_bound_push = 1e-8;
    o->autotune = 1;
    o->graphs = 1;
    o->resto_max = 20;
    o->kkt = 0;
}

abs_status absorber_create(const abs_params* p, const double* feeds, const double* prob, int64_t S,
                           abs_problem** out) {
    if (!p || !feeds || !out || S < 1 || S > (int64_t)1 << 26) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    *out = nullptr;
    if (!(p->d_lo < p->d_hi) || !(p->T_lo < p->T_hi) || !(p->d_lo > 0.0))
        return fail(nullptr, ABS_ERR_INFEASIBLE, "inconsistent bounds");
    PatternTables& T = pattern();
    if (!T.ok) return fail(nullptr, ABS_ERR_ARG, "pattern construction failed");
    abs_problem* h = new abs_problem();
    abs_status r = init_handle(h, p, S);
    if (r == ABS_OK && prob) {
        double sum = 0.0;
        h->prob.assign(prob, prob + S);
        for (double v : h->prob) {
            if (!(v >= 0.0)) r = fail(h, ABS_ERR_ARG, "probabilities must be >= 0");
            sum += v;
        }
        if (r == ABS_OK && !(std::fabs(sum - 1.0) <= 1e-9)) r = fail(h, ABS_ERR_ARG, "probabilities must sum to 1");
    } else if (r == ABS_OK) {
        h->prob.assign(S, 1.0 / (double)S);
    }
    if (r == ABS_OK) r = upload_feeds(h, feeds, nullptr);
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
    absorber_destroy(h->batch);
    absorber_destroy(h->aux);
    if (h->gate_ev) cudaEventDestroy(h->gate_ev);
    for (auto e : h->prof.pool) cudaEventDestroy(e);
    for (auto& g : h->rgraphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto s : h->cap) cudaStreamDestroy(s);
    if (h->ev_in) cudaEventDestroy(h->ev_in);
    for (auto e : h->ev_b)
        if (e) cudaEventDestroy(e);
    if (h->stream) cudaStreamDestroy(h->stream);
    cudaFree(h->dst);
    cudaFree(h->dglob);
    cudaFree(h->gate);
    cudaFree(h->filt);
    cudaFree(h->esc);
    cudaFree(h->escn);
    cudaFree(h->doff);
    if (h->hcond) cudaFreeHost(h->hcond);
    cudaFree(h->feed);
    cudaFree(h->pid);
    cudaFree(h->mlp_x);
    cudaFree(h->mlp_y);
    cudaFree(h->wd0);
    cudaFree(h->jac);
    cudaFree(h->hes);
    cudaFree(h->vec);
    cudaFree(h->ldl_inv);
    for (int k = 0; k < 2; ++k) {
        cudaFree(h->LUp[k]);
        cudaFree(h->Gp[k]);
    }
    cudaFree(h->piv);
    cudaFree(h->sing);
    cudaFree(h->part);
    cudaFree(h->chunks);
    cudaFree(h->pchunk);
    cudaFree(h->cred);
    cudaFree(h->rcnt);
    cudaFree(h->red);
    cudaFreeHost(h->hred);
    cudaFreeHost(h->hmap);
    cudaFree(h->ps);
    delete[] h->hps;
    cudaFreeHost(h->hring);
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
        case 7: return sizeof(abs_train_options);
        default: return -1;
    }
}

abs_status absorber_pattern(const abs_problem* h, int32_t* jrow, int32_t* jcol, int32_t* hrow, int32_t* hcol) {
    if (!h) return fail(nullptr, ABS_ERR_ARG, "bad argument");
    if (h->P.nsec != 1) return fail(const_cast<abs_problem*>(h), ABS_ERR_ARG, "absorber_pattern: one section only");
    return abs_scenario_pattern(nullptr, nullptr, jrow, jcol, hrow, hcol);
}

abs_status eval_grad_jac_hess(abs_problem* h, const double* x, const double* lambda, double obj_factor, double* f,
                              double* grad, double* c, double* jac_vals, double* hess_vals, abs_stream_t stream) {
    if (!h || !x || (hess_vals && !lambda)) return fail(h, ABS_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const dim3 g = grid2(h);
    const BView b{h->pid, nullptr, h->NP};   // each scenario reads its own problem's d slot
    if (jac_vals && hess_vals)
        eval_kernel<true, true, true><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, b, false, x, nullptr, nullptr,
                                                          lambda, h->feed, c, jac_vals, hess_vals, nullptr);
    else if (jac_vals)
        eval_kernel<true, true, false><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, b, false, x, nullptr, nullptr,
                                                           lambda, h->feed, c, jac_vals, nullptr, nullptr);
    else if (hess_vals)
        eval_kernel<true, false, true><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, b, false, x, nullptr, nullptr,
                                                           lambda, h->feed, c, nullptr, hess_vals, nullptr);
    else if (c)
        eval_kernel<true, false, false><<<g, kThr, 0, st>>>(h->P, (int)h->S, h->ld, b, false, x, nullptr, nullptr,
                                                            lambda, h->feed, c, nullptr, nullptr, nullptr);
    abs_status r = launch_check(h, KD_EVAL);
    if (r != ABS_OK) return r;
    // the objective sum_k w_k theta_k (w = 1, the single d, for one section)
    const int K = h->P.nsec;
    double gk[KSEC];
    for (int k = 0; k < K; ++k) gk[k] = obj_factor * sec_weight(k, K);
    if (grad) {
        CK(cudaMemsetAsync(grad, 0, sizeof(double) * (size_t)((int64_t)NSC * h->ld + (K - 1) * h->NP + 1), st));
        for (int k = 0; k < K; ++k)
            CK(cudaMemcpyAsync(grad + (int64_t)NSC * h->ld + (int64_t)k * h->NP, &gk[k], sizeof(double),
                               cudaMemcpyHostToDevice, st));
    }
    if (f) {
        double d[KSEC] = {0.0, 0.0};
        for (int k = 0; k < K; ++k)
            CK(cudaMemcpyAsync(&d[k], x + (int64_t)NSC * h->ld + (int64_t)k * h->NP, sizeof(double),
                               cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double fv = 0.0;
        for (int k = 0; k < K; ++k) fv += gk[k] * d[k];
        *f = fv;
    } else if (grad) {
        CK(cudaStreamSynchronize(st));   // gk lives on this stack frame
    }
    return ABS_OK;
}

abs_status absorber_scenario_status(const abs_problem* ch, int32_t* status) {
    abs_problem* h = const_cast<abs_problem*>(ch);
    if (!h || !status) return fail(h, ABS_ERR_ARG, "bad argument");
    std::vector<int> sg((size_t)h->S, 0);
    if (h->sing) CK(cudaMemcpy(sg.data(), h->sing, sizeof(int) * (size_t)h->S, cudaMemcpyDeviceToHost));
    for (int64_t s = 0; s < h->S; ++s) status[s] = sg[(size_t)s] ? ABS_ERR_NUMERIC : ABS_OK;
    return ABS_OK;
}

abs_status absorber_paper_layout(abs_problem* h, const double* x, double* out, abs_stream_t stream) {
    if (!h || !x || !out) return fail(h, ABS_ERR_ARG, "bad argument");
    if (h->NP != 1 || h->P.nsec != 1)
        return fail(h, ABS_ERR_ARG, "absorber_paper_layout needs a single-problem, single-diameter handle");
    cudaStream_t st = (cudaStream_t)stream;
    paper_layout_kernel<<<grid2(h), kThr, 0, st>>>(h->P, (int)h->S, h->ld, x, out);
    return launch_check(h, KD_VEC);
}

}  // extern "C"

// the interior-point engine lives in its own file (same translation unit)
#include "engine.inc"
#include "warm.inc"

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


// ======================================================================================
// Newton direction without any allocation (no handle, no cudaMalloc, no pinned memory)
// ======================================================================================
// For callers that cannot allocate device memory after start-up -- code running under
// a fixed memory budget, inside another runtime's allocator, or between graph
// captures -- this entry runs the FP64 stage-block LU, the Schur step on d and the
// block solves with every intermediate in one file-scope device array.  Nothing in the
// array has to start at zero: every word a call reads was written earlier in that call
// (the factor kernel writes every scenario's singular flag; every live (scenario,
// stage) thread writes its partial sums; the per-problem scalars are copied in first).
namespace {

constexpr int64_t NA_MAX_S = ABS_NOALLOC_MAX_SCENARIOS;    // scenarios per call, at most
constexpr int64_t NA_LD = NA_MAX_S;                         // a multiple of 32
constexpr size_t NA_LU = (size_t)N_STAGES * NV * NV * NA_LD;
constexpr size_t NA_G = (size_t)N_STAGES * NV * NABV * NA_LD;
constexpr size_t NA_VEC = (size_t)NSC * NA_LD + NA_LD;
constexpr int NA_K = 6;                                     // Schur partial planes
constexpr size_t NA_PART = (size_t)NA_K * N_STAGES * NA_LD;
constexpr size_t NA_PIV = ((size_t)N_STAGES * PIV_BYTES * NA_LD + 7) / 8;   // bytes as doubles
constexpr size_t NA_SING = (NA_LD + 1) / 2;                         // ints as doubles
constexpr size_t NA_PS = PS_NFIELDS;                                // one problem's scalars
constexpr size_t NA_TOTAL = NA_LU + NA_G + 3 * NA_VEC + NA_PART + NA_PIV + NA_SING + NA_PS;

// the scratch: every device that loads the library holds it until the process exits
static __device__ __align__(256) double g_noalloc_scratch[NA_TOTAL];

double* g_na_base[64] = {nullptr};
double g_na_host_part[NA_PART];   // host copy of the partial sums (static, not allocated)
double g_na_host_ps[NA_PS];       // host source of the per-problem scalars
// one call at a time in the process: the host arrays above and the device scratch are
// shared by every call (the lock is held until the call's stream has drained)
std::mutex g_na_mu;

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
    std::lock_guard<std::mutex> lock(g_na_mu);
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
    double* psd = (double*)sing + NA_SING;
    // the problem's constants (derived fields as absorber_create computes them)
    Params P;
    if (!make_params(p, &P) || P.nsec != 1)
        return fail(nullptr, ABS_ERR_ARG, "kkt_newton_noalloc: scales must be positive, one section");
    const dim3 g2((unsigned)((S + kThr - 1) / kThr), N_STAGES);
    const dim3 gq((unsigned)((S + QS_SCEN - 1) / QS_SCEN), N_STAGES);
    const int64_t od = (int64_t)NSC * ld;
    cudaError_t e;
#define NA_LAUNCHED()                                                                                  \
    if ((e = cudaGetLastError()) != cudaSuccess)                                                       \
        return fail(nullptr, ABS_ERR_CUDA, std::string("kkt_newton_noalloc: ") + cudaGetErrorString(e));
    // one problem, taking part in every kernel, with this call's delta_w
    std::memset(g_na_host_ps, 0, sizeof(g_na_host_ps));
    g_na_host_ps[PS_ACT] = 1.0;
    g_na_host_ps[PS_LSACT] = 1.0;
    g_na_host_ps[PS_DW] = delta_w;
    CK(cudaMemcpyAsync(psd, g_na_host_ps, sizeof(g_na_host_ps), cudaMemcpyHostToDevice, st));
    const BView bv{nullptr, psd, 1};
    const dim3 gf((unsigned)((S + WPB_F - 1) / WPB_F)), gs((unsigned)((S + WPB_S - 1) / WPB_S));
    factor_warp_kernel<double><<<gf, 32 * WPB_F, 0, st>>>((int)S, ld, bv, jac_vals, LU, piv, G, sing, 1e-14);
    NA_LAUNCHED();
    // p = J^-1 r_c, q = J^-1 b
    solve_warp_kernel<double, 2><<<gs, 32 * WPB_S, 0, st>>>(P, (int)S, ld, bv, jac_vals, LU, piv, G, x, rhs_c, nullptr,
                                                            pv, qv);
    NA_LAUNCHED();
    schur_kernel<false><<<gq, kThr, 0, st>>>((int)S, ld, bv, hess_vals, sigma, true, pv, qv, rhs_x, sing, part,
                                      SCHUR_DD | SCHUR_RHS, nullptr, nullptr);
    NA_LAUNCHED();
    double hx[2] = {0.0, 0.0};   // Sigma_dd and r_d
    const int64_t plane = (int64_t)N_STAGES * ld;
    CK(cudaMemcpyAsync(&hx[0], sigma + od, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&hx[1], rhs_x + od, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(g_na_host_part, part, sizeof(double) * NA_K * (size_t)plane, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    double red[NA_K];
    for (int k = 0; k < NA_K; ++k) {
        double a = 0.0;
        for (int n = 0; n < N_STAGES; ++n)
            for (int64_t s = 0; s < S; ++s) a += g_na_host_part[k * plane + n * ld + s];
        red[k] = a;
    }
    if (red[5] != 0.0) return fail(nullptr, ABS_ERR_NUMERIC, "kkt_newton_noalloc: singular stage block");
    // S_d = K_dd + dw + sum q^T (W + Sigma) q + dw sum q^T q ;  dd = (r_d - beta) / S_d
    const double Kdd = red[4] + hx[0];
    const double Sd = Kdd + delta_w + red[0] + delta_w * red[1];
    if (schur_d) *schur_d = Sd;
    if (!(Sd > 0.0)) return fail(nullptr, ABS_ERR_INERTIA, "kkt_newton_noalloc: Schur complement on d is not positive");
    const double beta = red[2] - delta_w * red[3];
    const double dd = (hx[1] - beta) / Sd;
    CK(cudaMemcpyAsync(sol_x + od, &dd, sizeof(double), cudaMemcpyHostToDevice, st));
    dz_kernel<<<gq, kThr, 0, st>>>((int)S, ld, bv, hess_vals, sigma, true, pv, qv, rhs_x, sol_x, gv);
    NA_LAUNCHED();
    solve_t_warp_kernel<double><<<gs, 32 * WPB_S, 0, st>>>((int)S, ld, bv, jac_vals, LU, piv, G, gv, sol_c);
    NA_LAUNCHED();
#undef NA_LAUNCHED
    // dd lives on this stack frame until the copy above has completed
    CK(cudaStreamSynchronize(st));
    return ABS_OK;
}
