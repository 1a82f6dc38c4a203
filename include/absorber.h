/*
 * absorber.h -- C ABI of the GB300 (sm_103a) library for the scenario-based absorber
 * diameter design problem of "Harnessing GPU Acceleration in Large-Scale Process
 * Optimization" (Huang, Shu, Schanen, Anitescu, Gandhi, Shin).
 *
 * Problem (10) of the paper:  min d  s.t. for every scenario w and stage n the MESH
 * equations (1) material, (3a) reaction equilibrium, (4) summation, (6) energy,
 * (9a) Raoult / (9b) Henry phase equilibrium; the hydraulic rows (10b)
 *     V_nw R T_nw / P_w - u_max pi d^2 / 4 <= 0;
 * and the bounds (10c-d).  The shared diameter d is the only coupling between
 * scenarios (Section "Replicated scenario structure").
 *
 * Unknown layout (per scenario, 220 = 10 stages x 22, stage-major, stage 0 = bottom):
 *   j = 0..8   xt_i  scaled liquid mole fraction of MEA, MEAH+, H+, MEACOO-, HCO3-,
 *                    OH-, CO3--, CO2, H2O   (x_i = sx_i * xt_i)
 *   j = 9..12  yt_i  scaled vapour mole fraction of CO2, H2O, N2, O2
 *   j = 13, 14 L, V  liquid / vapour molar flow leaving the stage [kmol/s]
 *   j = 15     Tt    temperature / sT  (sT = 100 K)
 *   j = 16..20 eps_r reaction extents of R1..R5 [kmol/s]
 *   j = 21     s     slack of the stage's hydraulic row, s >= 0
 * Row layout (per scenario, 220, stage-major):
 *   r = 0..10 material balance per species (order above plus N2, O2); 11 (9a);
 *   12 (9b); 13..17 (3a) for R1..R5; 18, 19 (4) liquid / vapour; 20 (6);
 *   21 (10b) as  V R T / P - u_max pi d^2/4 + s = 0.
 * The paper's 90 variable-fixings per scenario (y = 0 for the 7 non-volatile species,
 * x = 0 for N2, O2) are eliminated; abs_sizes reports the paper's counts.
 *
 * Device vectors are structure-of-arrays over scenarios with leading dimension
 * ld = S rounded up to a multiple of 32 (abs_sizes.ld): entry v of scenario s is at
 * [v * ld + s]; padding entries s >= S are ignored on input and unspecified on output.
 * A "primal vector" has 220*ld + 1 doubles, the last one being d.  A "row vector" has
 * 220*ld doubles.
 *
 * Ownership: the library owns the opaque abs_problem and every workspace inside it
 * (freed by absorber_destroy).  The caller owns every buffer passed by pointer.
 * Pointers documented "device" must be CUDA device (or managed) memory on the
 * handle's device; "host" pointers are ordinary host memory.
 * Streams: calls are asynchronous on the given stream unless documented otherwise.
 * Errors: no exception crosses the ABI; every call returns an abs_status, and
 * abs_last_error(h) gives a static description of the last error on that handle.
 * A handle is not thread-safe: serialise calls on one handle.
 */
#ifndef ABSORBER_H
#define ABSORBER_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct abs_problem abs_problem;
typedef struct CUstream_st* abs_stream_t; /* same type as cudaStream_t; NULL = default */

typedef int abs_status;
#define ABS_OK              0
#define ABS_ERR_ARG        -1   /* invalid argument (NULL pointer, S < 1, bad option) */
#define ABS_ERR_CUDA       -2   /* a CUDA runtime call failed */
#define ABS_ERR_OOM        -3   /* device allocation failed */
#define ABS_ERR_INERTIA    -4   /* inertia correction exceeded delta_w_max */
#define ABS_ERR_LINESEARCH -5   /* step size fell below alpha_min and restoration failed */
#define ABS_ERR_MAXITER    -6   /* iteration limit reached */
#define ABS_ERR_NUMERIC    -7   /* NaN/Inf, or a singular stage Jacobian block */
#define ABS_ERR_TIMEOUT    -8   /* a device-side wait gave up */
#define ABS_ERR_INFEASIBLE -9   /* bounds inconsistent (e.g. d_lo >= d_hi) */

#define ABS_NV_STAGE 22
#define ABS_N_STAGES 10
#define ABS_NV_SCEN 220
#define ABS_N_FEED 18

/* Model parameter table (problem data).  Units: flows kmol/s, T K, P bar, enthalpy
 * MJ/kmol, cp MJ/(kmol K), d m, u m/s, R bar m^3/(kmol K).  Each field is one
 * constant of the case-study model (Section "Case study"): the Kent-Eisenberg
 * correlation ln K_r = A + B/T + C ln T + D T, Antoine water Psat
 * ln Psat = a - b/(T + c), Henry ln H = ha + hb/T + hm x_MEA^app + hw x_H2O^app
 * with c_CO2 = rho_L x_CO2, ideal-mixture enthalpies
 * h_i(T) = ref + cpa (T - Tref) + cpb/2 (T - Tref)^2 + dh. */
typedef struct abs_params {
    double R, u_max, d_lo, d_hi, T_lo, T_hi, T_ref;
    double sx[9], sy[4], sT;
    double KE_A[5], KE_B[5], KE_C[5], KE_D[5];
    double psat_a, psat_b, psat_c;
    double henry_a, henry_b, henry_m, henry_w, rho_L;
    double hL_ref[9], hL_cpa[9], hL_cpb[9], hL_dh[9];
    double hV_ref[4], hV_cpa[4], hV_cpb[4], hV_dh[4];
    int32_t n_sections;   /* design vector (Eq. (8) with dim theta = n_sections): 1 the case
                             study's single diameter d; 2 a column of two sections of 5
                             stages (bottom, top), each with its own diameter theta_k in
                             [d_lo, d_hi] used by its stages' hydraulic rows (10b), the
                             objective (theta_0 + theta_1) / 2.  Design entries of a primal
                             vector: problem q's theta_k at 220 ld + k P + q (P problems) */
    double dp_stage;      /* pressure relation (7) with a specified drop: stage n (0 bottom, 9
                             top) at P_n = P + (9 - n) dp_stage, P the feed's absorber (top)
                             pressure; 0 (the case study): every stage at P */
} abs_params;

typedef struct abs_sizes {
    int64_t S, ld;
    /* the paper's counts for this S (Section "Numerical results") */
    int64_t n_var_paper, n_mesh, n_fix, n_hyd;
    /* the solver's NLP after eliminating the fixings: n = 220 S + 1, m = 220 S */
    int64_t n_unknowns, n_rows;
    /* per-scenario sparsity (identical for every scenario) */
    int32_t nnzJ_scen, nnzH_scen;
} abs_sizes;

/* Create a problem instance (Section "Problem setup"; Eq. (8) with (10)).
 *   p      host; the parameter table (copied).
 *   feeds  host or device; [18][S] doubles, field-major: V0, y0[CO2,H2O,N2,O2], T0,
 *          Lin, xin[9 liquid species], Tin, P  (flue gas in at the bottom, lean
 *          solvent in at the top, absorber pressure).  Copied.
 *   prob   host, S probabilities p_w of (8a) or NULL (1/S each).  Problem (10a) has no
 *          operating cost, so they do not enter the solution; they are validated and
 *          kept for completeness.
 *   S      number of scenarios, >= 1.
 *   out    receives the handle.
 * Uses the current CUDA device.  Synchronous.  Errors: ABS_ERR_ARG, ABS_ERR_OOM,
 * ABS_ERR_CUDA, ABS_ERR_INFEASIBLE (bad bounds). */
abs_status absorber_create(const abs_params* p, const double* feeds, const double* prob,
                           int64_t S, abs_problem** out);

/* Replace the feeds of an existing problem (same S), e.g. to re-solve with new scenario
 * data without reallocating.  feeds: host or device, [18][S] as in absorber_create; a
 * host array is copied synchronously, a device array asynchronously on the stream.
 * Errors: ABS_ERR_ARG, ABS_ERR_NUMERIC (non-finite host value), ABS_ERR_CUDA. */
abs_status absorber_set_feeds(abs_problem* h, const double* feeds, abs_stream_t stream);

/* Release the handle and every workspace it owns.  NULL is a no-op. */
void absorber_destroy(abs_problem* h);

/* Static text describing the last error recorded on h (or a global one if h is NULL). */
const char* abs_last_error(const abs_problem* h);

/* Sizes: the paper's counts (1 + 300 S variables, 210 S MESH rows, 90 S fixings,
 * 10 S hydraulic rows) and the solver's. */
abs_status absorber_sizes(const abs_problem* h, abs_sizes* out);

/* Host-only (no device needed): the per-scenario pattern sizes and patterns, as
 * absorber_pattern returns them.  Any of the array pointers may be NULL. */
abs_status abs_scenario_pattern(int32_t* nnzJ_scen, int32_t* nnzH_scen, int32_t* jrow,
                                int32_t* jcol, int32_t* hrow, int32_t* hcol);

/* Host-only: sizeof of the ABI structs, for binding checks.  which: 0 abs_params,
 * 1 abs_sizes, 2 abs_kkt_diag, 3 abs_inertia, 4 abs_solve_info, 5 abs_options,
 * 6 abs_result, 7 abs_train_options; -1 for an unknown index. */
int64_t abs_struct_size(int which);

/* Per-scenario status of the last factorization (kkt_factor or the last one of a solve):
 * status[s] = ABS_ERR_NUMERIC when a stage block of scenario s was singular or not
 * finite, else ABS_OK.  status: host, S entries.  Synchronous. */
abs_status absorber_scenario_status(const abs_problem* h, int32_t* status);

/* A primal vector in the paper's layout (Section "Numerical results"): out = [d, z_1 ..
 * z_S] with 300 entries per scenario -- per stage x over the 11 species, y over the 11
 * species, L, V, T, the 5 reaction extents, in physical units -- and the 90 fixed
 * entries per scenario (y of the 7 non-volatile species, x of N2 and O2) exactly 0.
 *   x    device primal vector of a single-problem handle.
 *   out  device, 1 + 300 S doubles.  Asynchronous. */
abs_status absorber_paper_layout(abs_problem* h, const double* x, double* out, abs_stream_t stream);

/* Per-scenario sparsity patterns (host arrays), identical for every scenario.
 *   jrow, jcol: nnzJ_scen entries of dc_s/d(z_s, d) in CSR order (row ascending, then
 *               column ascending); columns 0..219 are z_s, column 220 is d.
 *   hrow, hcol: nnzH_scen entries of the lower triangle (row >= col) of the
 *               Lagrangian Hessian in CSR order; the last entry is (220, 220), the
 *               scenario's contribution to d-d (entries over scenarios are summed).
 * Value arrays of eval_grad_jac_hess hold entry k of scenario s at [k * ld + s]. */
abs_status absorber_pattern(const abs_problem* h, int32_t* jrow, int32_t* jcol,
                            int32_t* hrow, int32_t* hcol);

/* Objective, gradient, constraints, Jacobian and Lagrangian-Hessian values in one
 * fused pass over (scenario, stage) -- the replicated constraint families of Eqs.
 * (1), (3a), (4), (6), (9a-b), (10b) with analytic derivatives.
 *   x         device, primal vector (220*ld + 1).
 *   lambda    device, row vector: equality multipliers (may be NULL if hess_vals is).
 *   obj_factor  multiplies the objective (d) and its derivatives.
 *   f         host, receives obj_factor * d (may be NULL).
 *   grad      device primal vector or NULL: obj_factor * e_d.
 *   c         device row vector or NULL: residuals.
 *   jac_vals  device, nnzJ_scen * ld, or NULL.
 *   hess_vals device, nnzH_scen * ld, or NULL: Hessian of sum_rows lambda c (the
 *             objective is linear).
 * Asynchronous except when f != NULL (reads d back). */
abs_status eval_grad_jac_hess(abs_problem* h, const double* x, const double* lambda,
                              double obj_factor, double* f, double* grad, double* c,
                              double* jac_vals, double* hess_vals, abs_stream_t stream);

#define ABS_PREC_FP64 0   /* stage-block LU and solves in FP64 */
#define ABS_PREC_FP32 1   /* stage-block LU and solves in FP32, FP64 refinement */
#define ABS_PREC_FP32_TC 3 /* kkt_factor only: FP32 as ABS_PREC_FP32, the stage-block inverses
                              by the tensor-core panel kernel (abs_options.factor_kernel = 1) */
#define ABS_PREC_FP64_LDL 4 /* kkt_factor only: every scenario block K_s by the regularised
                              block LDL^T in FP64 (taken whenever delta_c > 0) */

typedef struct abs_kkt_diag {
    const double* sigma;  /* device primal vector: barrier diagonal Sigma (d last) */
    double delta_w;       /* primal regularisation, >= 0 */
    double delta_c;       /* dual regularisation, >= 0 (> 0: the block LDL^T of kkt_factor) */
} abs_kkt_diag;

typedef struct abs_inertia {
    int64_t n_pos, n_neg, n_zero;   /* inertia of the whole KKT matrix */
    double schur_d;                 /* the scalar Schur complement on d */
    int64_t n_singular;             /* scenarios whose factorization met a tiny pivot */
} abs_inertia;

/* Factor the primal-dual matrix of one interior-point iteration (Wachter & Biegler
 * 2006, Eq. (13) with the regularisations of their Section 3.1; the paper's KKT step,
 * Section "GPU-resident solution")
 *     K = [ W + Sigma + dw I , J^T ; J , -dc I ]
 * for the bordered block-diagonal structure of (10), the scenarios eliminated onto d by
 * a scalar Schur complement S_d = K_dd + dw - sum_s bh_s^T K_s^{-1} bh_s (bh_s = [0; b_s],
 * b_s = dc_s/dd); the inertia of K is that of the scenario blocks plus the sign of S_d
 * (Haynsworth).  Two factorizations of the scenario blocks K_s:
 *  - delta_c = 0 (ABS_PREC_FP64 / FP32 / FP32_TC): the constraint Jacobian J_s (220 x 220,
 *    block tridiagonal with 22 x 22 stage blocks) by a block LU with partial pivoting
 *    inside each stage block; then S_d = K_dd + sum_s q_s^T (W_s + Sigma_s + dw I) q_s,
 *    q_s = J_s^{-1} b_s, and with J_s nonsingular every K_s has inertia (220, 220, 0)
 *    whatever W_s is.  A singular stage block is reported in n_singular and by
 *    ABS_ERR_NUMERIC;
 *  - delta_c > 0 or ABS_PREC_FP64_LDL: K_s itself by a block LDL^T over its 44 x 44 stage
 *    blocks (unknowns and rows of a stage together) with Bunch-Kaufman pivoting inside
 *    each, in FP64; its inertia counted from the pivots.  A zero pivot is reported in
 *    n_zero and n_singular and by ABS_ERR_NUMERIC.
 *   x, jac_vals, hess_vals  device, as produced by eval_grad_jac_hess at the iterate.
 *   diag       host struct (delta_w, delta_c >= 0, else ABS_ERR_ARG).
 *   precision  ABS_PREC_FP64, ABS_PREC_FP32, ABS_PREC_FP32_TC or ABS_PREC_FP64_LDL;
 *              delta_c > 0 needs ABS_PREC_FP64 or ABS_PREC_FP64_LDL (else ABS_ERR_ARG).
 *   inertia    host, receives the inertia (the call synchronises the stream).
 * The factorization stays in the handle for kkt_solve, which reads jac_vals, hess_vals
 * and diag->sigma again (its products with H and its FP64 refinement): those buffers
 * are referenced, not copied, and must stay allocated and unchanged until the last
 * kkt_solve of this factorization. */
abs_status kkt_factor(abs_problem* h, const double* x, const double* jac_vals,
                      const double* hess_vals, const abs_kkt_diag* diag, int precision,
                      abs_inertia* inertia, abs_stream_t stream);

typedef struct abs_solve_info {
    int32_t refine_steps;       /* FP64 refinement steps taken */
    double residual;            /* final scaled residual ||r - K s||_inf / (||r||_inf + tiny) */
} abs_solve_info;

/* Solve K sol = rhs with the last kkt_factor: per-scenario forward/backward block
 * solves, the Schur step on d, back-substitution, then FP64 iterative refinement on
 * the full residual (computed from the FP64 jac/hess values) until the scaled residual
 * is <= refine_tol or max_refine steps were taken.
 *   rhs_x, sol_x  device primal vectors (220*ld + 1).
 *   rhs_c, sol_c  device row vectors (220*ld).
 *   info          host or NULL (if non-NULL the call synchronises).          */
abs_status kkt_solve(abs_problem* h, const double* rhs_x, const double* rhs_c,
                     double* sol_x, double* sol_c, int max_refine, double refine_tol,
                     abs_solve_info* info, abs_stream_t stream);

/* Options of the interior-point solve.  abs_default_options fills the published
 * defaults of Wachter & Biegler (2006) and tol = 1e-8 (the paper's tolerance). */
typedef struct abs_options {
    double tol;            /* stop when E_0 <= tol */
    int32_t max_iter;
    int32_t precision;     /* ABS_PREC_FP64 / ABS_PREC_FP32 */
    int32_t max_refine;    /* refinement steps per Newton solve */
    double refine_tol;     /* scaled residual target of the refinement */
    double mu_init, kappa_eps, kappa_mu, theta_mu, tau_min, s_max, kappa_sigma;
    double bound_push, bound_frac;
    double gamma_theta, gamma_phi, delta, s_theta, s_phi, eta_phi, gamma_alpha;
    double lam_init_max;
    double dw0, dw_min, dw_max, kw_minus, kw_plus, kw_plus_bar;
    int32_t max_ls;        /* maximum line-search trials per iteration */
    int32_t verbose;       /* 1: print one line per iteration to stdout */
    int32_t profile;       /* 1: time the hot kernels with CUDA events (abs_result.kernel_*) */
    int32_t init;          /* 0: expected-value start (S > 1, see ipm_solve), 1: inlet copy,
                              2: one expected-value start shared by every problem of a
                              batch (the mean over all its scenarios) */
    int32_t soc_max;       /* second-order corrections per iteration (0 disables) */
    double kappa_soc;      /* required theta reduction between corrections */
    double obj_scaling;    /* the solver minimises obj_scaling * d; <= 0 means S */
    double warm_mu_init;   /* ipm_solve_learned: barrier parameter of the learned start */
    double warm_bound_push;/* ipm_solve_learned: bound push and fraction at the learned start */
    int32_t warm_multipliers; /* ipm_solve_learned: 0 least-squares estimate at the learned
                                 point, 1 the network's multipliers */
    int32_t autotune;      /* 1: the first factor / solve launch of each kernel, precision and
                              size bucket (S rounded down to a power of two, S >= 256) times
                              every warps-per-block candidate and keeps the fastest
                              (results are identical); 0: 4 warps per block */
    int32_t graphs;        /* 1: the whole solve (every iteration, refinement round, line-search
                              round and restoration step, with the device's decisions as
                              conditional nodes) is captured into one CUDA graph on the second
                              solve of a launch configuration and replayed from then on (the
                              first runs eagerly and tunes the tile shapes); 0: every solve is
                              launched eagerly, the host reading each decision */
    int32_t factor_tile;   /* FP32 factor launches only: 0 shape from autotune; 1, 2, 4, 8:
                              that many warps (scenarios) per block (identical results);
                              other values are rejected with ABS_ERR_ARG */
    int32_t resto_max;     /* feasibility restoration (Wachter & Biegler 2006, Section 3.3)
                              when the line search fails: at most this many damped Newton
                              steps on the square constraint system with d fixed, until the
                              filter accepts a point with theta reduced by 1 - gamma_theta;
                              0 disables it (the solve then stops with ABS_ERR_LINESEARCH) */
    int32_t factor_kernel; /* FP32 stage-block inverses: 0 Gauss-Jordan exchanges on the FP32
                              pipes; 1 blocked Gauss-Jordan (panels of 8 pivot columns) with
                              the trailing updates on the tensor cores (mma.sync TF32, split
                              in three products for FP32 accuracy).  Same outputs up to
                              rounding; kkt_factor uses the last value an ipm_solve set */
    int32_t kkt;           /* factorization of the scenario blocks: 0 block LU of J_s (inertia
                              from the Schur scalar alone; a singular stage block ends the solve
                              with ABS_ERR_NUMERIC); 1 the regularised block LDL^T of kkt_factor
                              (FP64 only), with Algorithm IC complete: the inertia of every
                              scenario block from its pivots, delta_c = 1e-8 mu^(1/4) when a
                              pivot is zero, every delta_w trial refactored */
} abs_options;

void abs_default_options(abs_options* o);

#define ABS_N_PHASES 6   /* eval, factor, solve, linesearch, step, other */
#define ABS_N_KINDS 16   /* kernel kinds counted in abs_result.kind_launches: 0 evaluation with
                            the Hessian, 1 line-search trial evaluation, 2 stage-block factor,
                            3 block solve J x = r, 4 block solve J^T y = g, 5 KKT residual,
                            6 Schur sums, 7 dual residual J^T lambda, 8 reduction planes (one
                            count per plane reduced), 9 barrier diagonal and right-hand
                            sides, 10 dz and g, 11 step sizes, 12 accept, 13 other vector
                            kernels, 14 control kernels, 15 evaluation without the Hessian */
#define ABS_N_KERNELS 5  /* eval (residual+Jacobian+Hessian), eval (line-search trial),
                            stage-block LU, block solve J x = r, block solve J^T y = g */

typedef struct abs_result {
    abs_status status;
    int32_t iters;
    int32_t ls_trials;           /* line-search trial evaluations in total */
    int32_t inertia_corrections; /* iterations that needed delta_w > 0 */
    int32_t refine_steps;        /* refinement steps in total */
    double d, obj, E0, mu;
    double inf_pr, inf_du;
    double solve_ms;             /* wall time of ipm_solve (host clock) */
    double phase_ms[ABS_N_PHASES];  /* CUDA-event time per phase */
    double kernel_ms[ABS_N_KERNELS];        /* with options.profile: summed kernel time */
    int32_t kernel_launches[ABS_N_KERNELS]; /* ... and launch counts */
    int64_t launches;            /* every kernel this library launched during the solve */
    int32_t base_iters;          /* iterations of the expected-value start solve */
    int32_t soc_steps;           /* second-order correction steps taken */
    int32_t fp64_fallbacks;      /* FP32 factors: iterations in which the FP64 refinement
                                    stalled and the scenarios behind it were refactored in FP64 */
    double base_ms;              /* host time of the expected-value start solve */
    int32_t warm_status;         /* ipm_solve_learned: 1 learned start used, 0 rejected */
    int32_t fp64_scenarios;      /* FP32 factors: scenario factorizations escalated to FP64 in
                                    total (over the iterations; see fp64_fallbacks) */
    double warm_ms;              /* ipm_solve_learned: host time of the prediction and of queueing
                                    the inlet-copy start's evaluation */
    double warm_E0, cold_E0;     /* E_0 at the learned start and at the inlet-copy start */
    double warm_theta, cold_theta;  /* constraint violation ||c||_1 at the same two starts */
    int32_t tiles[4];            /* warps per block last used: factor, solve (1 and 2 right-hand
                                    sides), transposed solve */
    int32_t graph_replays;       /* graph launches of the solve (whole runs replayed from
                                    captured CUDA graphs) */
    int32_t resto_phases;        /* feasibility restoration phases entered */
    int64_t kind_launches[ABS_N_KINDS];  /* launches per kernel kind issued by the host during
                                    the solve (eager runs, captures; a replayed graph adds none) */
    double d_sec[2];             /* the design entries (abs_params.n_sections of them; d_sec[0] =
                                    d); obj = their stage-weighted sum */
} abs_result;

/* Diagnostic: measured throughput of dependent-free fused multiply-adds on the current
 * device, in GFLOP/s (2 flops per FMA).  kind 0: FP64, kind 1: FP32.  Synchronous. */
abs_status abs_measure_fma_peak(int kind, double* gflops);

/* Interior-point solve of problem (10) on the device (the paper's GPU-resident
 * solution, Section "GPU-resident solution with MadNLP.jl"): filter line-search
 * primal-dual method after Wachter & Biegler (2006) with second-order corrections and
 * the objective scaled by S, with the eval kernel, the block-LU + Schur KKT
 * factorization and solve, every vector update and every scalar decision of the method
 * (barrier update, Algorithm IC, refinement test, FP64 escalation, filter line search,
 * feasibility restoration) running in this library's kernels; with options.graphs the
 * solve is one replay of a captured CUDA graph whose loops and branches are conditional
 * nodes set by those kernels.
 * Starting point (unless warm_x is given): for S > 1 and init = 0 the stage states of
 * the expected-value problem -- one scenario whose feed is the mean of the S feeds,
 * solved first by this same method from the inlet-copy start, always with FP64 factors
 * -- copied to every scenario, d = (d_lo + d_hi)/2 and each hydraulic slack from its
 * row; otherwise every stage copies the inlet streams.  A warm start (warm_x) is pushed
 * into the bounds by bound_push / bound_frac and its bound multipliers set to
 * mu_init / slack; without warm_y the row multipliers are the least-squares estimate.  The returned multipliers (y_out) are those of the
 * unscaled problem min d.
 *   opt     host (NULL = defaults).
 *   warm_x  device primal vector or NULL; warm_y device row vector or NULL.
 *   res     host, required.
 *   x_out   device primal vector or NULL;  y_out device row vector or NULL.
 * Synchronous (returns when the solve has finished). */
abs_status ipm_solve(abs_problem* h, const abs_options* opt, const double* warm_x,
                     const double* warm_y, abs_result* res, double* x_out, double* y_out,
                     abs_stream_t stream);

/* Bound multipliers z_L, z_U of the bounds (10c-d) at the point the last ipm_solve,
 * ipm_solve_batch or ipm_solve_learned on this handle returned (the primal-dual iterate
 * of the interior-point method, Wachter & Biegler 2006, Eq. (4); the KKT point of the
 * paper's Section "GPU-resident solution with MadNLP.jl"), for the unscaled problem
 * min d (the solver's scaled multipliers divided by each problem's obj_scaling), so that
 * with x_out and y_out of the same solve they give every term of the optimality error
 * E_0.  Unknowns without a lower (upper) bound carry 0.
 *   zl_out, zu_out  device primal vectors in the handle's layout (the design slots receive
 *                   each problem's multipliers of d >= d_lo / d <= d_hi), or NULL.
 *   zd_out          host, 2 K P doubles (K = n_sections: z_L of the design entries, entry k
 *                   of problem q at k P + q, then z_U likewise), or NULL.
 * Errors: ABS_ERR_ARG (no finished solve on the handle), ABS_ERR_CUDA.  Synchronous. */
abs_status absorber_bound_multipliers(abs_problem* h, double* zl_out, double* zu_out, double* zd_out,
                                      abs_stream_t stream);

/* A handle holding P independent design problems side by side: problem q has sizes[q]
 * scenarios, and its feeds are columns [off_q, off_q + sizes[q]) of feeds (off_q = the
 * sum of the earlier sizes).
 *   feeds  host or device, [18][sum(sizes)] as in absorber_create.
 *   sizes  host, P counts >= 1.
 * Vectors of a batch handle use S = sum(sizes) and ld = S rounded up to 32; the primal
 * vectors hold the P diameters in their last ld entries (problem q's at 220*ld + q).
 * eval_grad_jac_hess evaluates every problem at its own diameter; kkt_factor,
 * kkt_solve and ipm_solve need single-problem handles (ipm_solve_batch solves a batch
 * handle).  Synchronous.  Errors as absorber_create. */
abs_status absorber_create_batched(const abs_params* p, const double* feeds, const int64_t* sizes,
                                   int32_t P, abs_problem** out);

/* Number of problems a handle holds (1 for absorber_create; 0 for NULL). */
int32_t absorber_num_problems(const abs_problem* h);

/* Batched interior-point solve of P independent design problems of form (10), each
 * with its own scenario count, feeds, diameter, barrier parameter, filter and
 * inertia-correction state (the batching form of the scenario workflow: many design
 * studies of Section "Case study: absorber diameter minimization" side by side on one GPU).  Every kernel launch
 * covers the scenarios of all problems still iterating, laid out side by side in one
 * structure-of-arrays (problem p owns a contiguous run of scenario slots); per-problem
 * sums, maxima and minima come from segmented reductions; the control kernels take each
 * problem's scalar decisions on the device (one thread per problem).  A problem
 * that has converged or failed stops taking part.  The method and its starting point are
 * those of ipm_solve with warm_x = warm_y = NULL, applied to each problem: the
 * expected-value starts of all problems are themselves solved as one batch of P
 * one-scenario problems.
 *   probs   host array of P handles from absorber_create (each a single problem; all
 *           with the same parameter table).  The batch workspace is built on the first
 *           call and cached on probs[0] for later calls with the same scenario counts; it
 *           is freed with probs[0].
 *   opt     host (NULL = defaults); obj_scaling <= 0 scales problem p by its own S_p.
 *   res     host array of P results, one per problem (timings and launch counts are
 *           those of the whole batch).
 *   x_out   host array of P device primal vectors (each in its own problem's layout,
 *           220*ld_p + 1) or NULL; entries may be NULL.
 * Returns ABS_OK when the batch ran (each problem's outcome is in res[p].status) or an
 * error of the batch as a whole (bad argument, CUDA error).  Synchronous. */
abs_status ipm_solve_batched(abs_problem** probs, int32_t P, const abs_options* opt,
                             abs_result* res, double** x_out, abs_stream_t stream);

/* The batched solve of the P problems of a handle from absorber_create_batched (or of a
 * single-problem handle, P = 1), with the method of ipm_solve_batched.
 *   res    host array of absorber_num_problems(h) results.
 *   x_out  device primal vector in the batch handle's layout, or NULL.
 *   y_out  device row vector, or NULL: each problem's multipliers of its unscaled
 *          problem min d.
 * Returns ABS_OK when the batch ran (outcomes in res[q].status).  Synchronous. */
abs_status ipm_solve_batch(abs_problem* h, const abs_options* opt, abs_result* res,
                           double* x_out, double* y_out, abs_stream_t stream);

/* ---- learned warm start ------------------------------------------------------------
 * The paper solves every instance from a fixed starting point; this is the learned-
 * warm-start form of its workflow: a network, trained on the GPU from solutions of
 * single-scenario instances of problem (10), predicts the starting point of a new
 * instance, which the interior-point method then accepts or rejects.
 *
 * The network (abs_mlp): 3 -> 256 -> 256 -> 256 -> 440 perceptron with GELU
 * (x Phi(x)) activations, bfloat16 weights and FP32 activations and sums:
 *   a0 = (X - in_shift) / in_scale;  a_l = gelu(a_{l-1} W_l^T + b_l), l = 1..3;
 *   yhat = a3 W4^T + b4;  prediction = yhat * out_scale + out_shift.
 * Inputs per scenario: V0 (flue-gas flow), y_CO2,0 (its CO2 fraction), d.  Outputs: the
 * scenario's 220 unknowns (this header's per-scenario order, with the 13 species
 * fractions xt, yt of each stage as natural logarithms) then its 220 row multipliers
 * (of the unscaled problem).  Training minimises
 *   loss = sum (yhat - (Y - out_shift) / out_scale)^2 / (2 n 440)
 * with Adam (Kingma & Ba 2015); W_l enter every product rounded to bfloat16 (nearest,
 * ties to even) from FP32 master weights.  Parameters, flat (ABS_MLP_PARAMS floats):
 * W1 [256][3], b1, W2 [256][256], b2, W3 [256][256], b3, W4 [440][256], b4.
 * Device arrays X are [n][3] and Y [n][440] floats, row-major.  A network is not
 * thread-safe; its calls use the current device. */
#define ABS_MLP_IN 3
#define ABS_MLP_HIDDEN 256
#define ABS_MLP_OUT 440
#define ABS_MLP_PARAMS 245688
typedef struct abs_mlp abs_mlp;

/* New network: Glorot-uniform weights from seed (splitmix64 draws), zero biases,
 * identity normalisation.  Errors: ABS_ERR_ARG, ABS_ERR_OOM, ABS_ERR_CUDA. */
abs_status abs_mlp_create(uint64_t seed, abs_mlp** out);
void abs_mlp_destroy(abs_mlp* net);
const char* abs_mlp_last_error(const abs_mlp* net);

/* Host copies of the FP32 master parameters (ABS_MLP_PARAMS floats).  set_params
 * refreshes the bfloat16 copies and resets Adam's moments and step count.  Synchronous. */
abs_status abs_mlp_set_params(abs_mlp* net, const float* params);
abs_status abs_mlp_get_params(const abs_mlp* net, float* params);

/* Normalisation constants (host, 3 + 3 + 440 + 440 doubles; scales > 0; stored as
 * float).  fit_normalization sets them to the per-column mean and standard deviation
 * of device data X [n][3], Y [n][440] (scale 1 for a column with no spread). */
abs_status abs_mlp_set_normalization(abs_mlp* net, const double* in_shift, const double* in_scale,
                                     const double* out_shift, const double* out_scale);
abs_status abs_mlp_get_normalization(const abs_mlp* net, double* in_shift, double* in_scale,
                                     double* out_shift, double* out_scale);
abs_status abs_mlp_fit_normalization(abs_mlp* net, const float* X, const float* Y, int64_t n,
                                     abs_stream_t stream);

/* Prediction: raw inputs X [n][3] -> raw outputs Y [n][440] (device).  Asynchronous. */
abs_status abs_mlp_forward(abs_mlp* net, const float* X, int64_t n, float* Y, abs_stream_t stream);

/* The products of the layers with 256 inputs (layers 2-4, forward) run on the tensor cores
 * (tcgen05 MMAs of bfloat16 operands with FP32 accumulation in tensor memory; each FP32
 * activation enters as the sum of three bfloat16 terms, so the product keeps FP32
 * accuracy) when on = 1, the default, or as FP32 FMAs on the CUDA cores when on = 0.
 * Returns ABS_ERR_ARG for another value. */
abs_status abs_mlp_set_tensor_cores(abs_mlp* net, int32_t on);

/* Nonzero once a tensor-core product of this network gave up waiting for its MMAs (after
 * about 4M polls of its mbarrier; that block's outputs are left unwritten and its tensor
 * memory freed).  Read after the stream the network ran on has synchronised;
 * abs_mlp_forward, abs_mlp_loss_grad and abs_mlp_train then return ABS_ERR_TIMEOUT. */
int32_t abs_mlp_device_fault(const abs_mlp* net);

/* Self-test of that path: one 128 x 256 x 256 tensor-core product whose MMAs are withheld,
 * so that its wait runs out after 1024 polls; the kernel frees its tensor memory and sets
 * the fault flag, which this call reads after synchronising the stream and then clears.
 * Returns ABS_ERR_TIMEOUT (the expected outcome: the expiry was reported), ABS_ERR_CUDA
 * when it was not reported or a CUDA call failed. */
abs_status abs_mlp_selftest_wait(abs_mlp* net, abs_stream_t stream);

/* Loss of the n pairs (X, Y) (raw, device) and its gradient with respect to the
 * parameters (device, ABS_MLP_PARAMS floats, or NULL).  *loss: host.  Synchronous. */
abs_status abs_mlp_loss_grad(abs_mlp* net, const float* X, const float* Y, int64_t n, double* loss,
                             float* grad, abs_stream_t stream);

typedef struct abs_train_options {
    int32_t epochs;        /* passes over the data */
    int32_t batch;         /* rows per Adam step (the last step of an epoch takes the rest) */
    double lr, lr_final;   /* learning rate, decayed geometrically from lr to lr_final */
    double beta1, beta2, eps;
    uint64_t seed;         /* order of the rows in each epoch (Fisher-Yates, splitmix64) */
} abs_train_options;
void abs_default_train_options(abs_train_options* o);

/* Train on n pairs (raw, device) with the network's current normalisation: each epoch
 * visits the rows in a seeded random order in minibatches, one Adam step per batch.
 * epoch_loss: host, opt->epochs doubles (mean loss of each epoch's batches) or NULL.
 * Synchronous. */
abs_status abs_mlp_train(abs_mlp* net, const float* X, const float* Y, int64_t n,
                         const abs_train_options* opt, double* epoch_loss, abs_stream_t stream);

/* Training pairs from a solved handle (typically a batch of one-scenario problems),
 * one row per (scenario of a kept problem, diameter copy a = 0..n_aug-1):
 *   X row = (V0, y_CO2,0 of the scenario, d),  d = d_p (1 + d_spread a / (n_aug - 1))
 *           with d_p the problem's optimal diameter (x's d slot; copy 0 is d_p itself);
 *   Y row = (the scenario's 220 entries of x -- species fractions as logarithms,
 *            hydraulic slacks recomputed at d -- then its 220 entries of y).
 * The stage states of a scenario do not depend on d (its MESH system is square in
 * them), so the copies teach the network that; only the slacks follow d.
 *   x, y   device primal / row vectors of the solved handle (unscaled multipliers, as
 *          ipm_solve_batch writes them).
 *   keep   host, one flag per problem (nonzero = use), or NULL for all.
 *   X, Y   device [rows][3], [rows][440] floats, or NULL to only count.
 *   rows   host, receives the number of rows.
 * Synchronous. */
abs_status abs_mlp_make_dataset(const abs_problem* h, const double* x, const double* y,
                                const int32_t* keep, int32_t n_aug, double d_spread, float* X,
                                float* Y, int64_t* rows, abs_stream_t stream);

/* Interior-point solve of a single-problem handle from the network's predicted start
 * (one network pass at the mean training diameter; its targets do not depend on d):
 * stage states from the network; d0 solves stationarity in d when every scenario's
 * largest-volume hydraulic row carries the multiplier warm_mu_init / slack; slacks from
 * the hydraulic rows at d0; unknowns pushed into their bounds by warm_bound_push and
 * bound multipliers warm_mu_init / slack; row multipliers from the least-squares
 * estimate at that point (warm_multipliers = 0) or the network's, scaled onto the same
 * central path (1).  The start is accepted when its E_0 and ||c||_1 do not exceed those
 * of the inlet-copy start (evaluated with zero iterations on a second handle of the same
 * problem, created on first use, while the prediction runs); the solve runs from it
 * with mu_init = warm_mu_init and takes the test at its first evaluation, where a
 * rejected start ends that run and the solve restarts from the default start
 * (res.warm_status says which).  Outputs as ipm_solve.  Synchronous. */
abs_status ipm_solve_learned(abs_problem* h, abs_mlp* net, const abs_options* opt,
                             abs_result* res, double* x_out, double* y_out, abs_stream_t stream);

/* Newton direction of one interior-point iteration without any allocation.
 *
 * The paper has no counterpart: this entry exists for callers that cannot allocate
 * GPU memory once they are running -- code under a fixed device-memory budget, code
 * whose memory belongs to another runtime's allocator, or code that must not trigger
 * allocator synchronisation between CUDA graph captures.  It computes what
 * kkt_factor (FP64, delta_c = 0) followed by kkt_solve (no refinement) compute, with
 * no handle: the caller passes the problem's parameter table and its own device
 * buffers, and every intermediate (stage-block LU factors, G blocks, pivots, the
 * Schur vectors and block partial sums) lives in one static device array of the
 * library, sized for ABS_NOALLOC_MAX_SCENARIOS scenarios (about 8 MB), which every GPU
 * that loads the library holds until the process exits.  The call makes no cudaMalloc,
 * cudaFree, pinned-host or other allocating call.
 *   p          host, the parameter table.
 *   S, ld      scenarios (1 <= S <= ABS_NOALLOC_MAX_SCENARIOS; larger S is rejected
 *              with ABS_ERR_ARG) and the leading dimension (S rounded up to 32).
 *   x          device primal vector (only d, its last entry, is read).
 *   jac_vals, hess_vals  device, as eval_grad_jac_hess writes them at the iterate.
 *   sigma      device primal vector, the barrier diagonal (d last); delta_w >= 0.
 *   rhs_x, rhs_c, sol_x, sol_c  device primal / row vectors, as for kkt_solve.
 *   schur_d    host or NULL: receives the Schur complement on d.
 * Errors: ABS_ERR_ARG, ABS_ERR_NUMERIC (singular stage block), ABS_ERR_INERTIA (Schur
 * complement not positive: increase delta_w), ABS_ERR_CUDA.
 * The first call on each device looks up the array's device address and uploads the
 * pattern tables.  All calls share the one array, which keeps the last call's contents;
 * the library serialises every call of this entry point in the process (a lock held
 * until the call's stream has drained), so two calls never overlap on the GPU -- but
 * other work the caller queues on other streams must not touch the same output buffers
 * meanwhile.  The call copies a few scalars through pageable host memory and
 * synchronises the stream before returning, so it cannot be recorded into a CUDA graph;
 * it makes no allocation at any point. */
#define ABS_NOALLOC_MAX_SCENARIOS 128
abs_status kkt_newton_noalloc(const abs_params* p, int64_t S, int64_t ld, const double* x,
                              const double* jac_vals, const double* hess_vals,
                              const double* sigma, double delta_w, const double* rhs_x,
                              const double* rhs_c, double* sol_x, double* sol_c,
                              double* schur_d, abs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* ABSORBER_H */
