// Internal declarations of the WP-CCC CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/wpccc.h"

namespace wpccc {

// ---------------------------------------------------------------------------
// error reporting
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
wpccc_status fail(wpccc_status st, const std::string& msg);
wpccc_status cuda_fail(cudaError_t e, const char* what);

#define WPCCC_CUDA(call)                                          \
    do {                                                          \
        cudaError_t e_ = (call);                                  \
        if (e_ != cudaSuccess) return ::wpccc::cuda_fail(e_, #call); \
    } while (0)

#define WPCCC_CHECK_LAUNCH(name)                                  \
    do {                                                          \
        cudaError_t e_ = cudaGetLastError();                      \
        if (e_ != cudaSuccess) return ::wpccc::cuda_fail(e_, name); \
    } while (0)

// ---------------------------------------------------------------------------
// device-resident basis
// ---------------------------------------------------------------------------
struct CentreDev {
    double Z = 0.0;
    int n_rad = 0, n_states = 0, lmax = 0, nlam = 0;  // nlam = 2*lmax+1 multipoles
    double* f = nullptr;        // [n_rad][Nr]
    int* rad_l = nullptr;       // [n_rad]
    int* st_rad = nullptr;      // [n_states]
    int* st_l = nullptr;        // [n_states]
    int* st_m = nullptr;        // [n_states]
    double* st_eps = nullptr;   // [n_states]
    int* st_index = nullptr;    // [n_rad][2*WPCCC_LMAX+1]: state of (radial, m) or -1
    // Eq. 7 table: entry e holds F_{a b lam}(r_i) for a <= b
    int n_fent = 0;
    double* F = nullptr;        // [n_fent][Nr]
    int* Foff = nullptr;        // [n_rad][n_rad][nlam]: entry or -1 (symmetric in a, b)
    int* fent_a = nullptr;      // [n_fent]
    int* fent_b = nullptr;
    int* fent_lam = nullptr;
    double* ang = nullptr;      // [LM][LM][nlam]: Eq. 6 coefficient of the angular parts (l', m'), (l, m)
                                // without the sqrt((lam-mu)!/(lam+mu)!) factor (carried by the Legendre
                                // table); it does not depend on the radial functions
    int* st_lm = nullptr;       // [n_states]: angular index l^2 + l + m of each state
    int LM = 0;                 // (lmax + 1)^2 angular parts
    // host copies used to build launch lists
    std::vector<int> h_rad_l, h_st_rad, h_st_m;
};

// Derivative tables of one centre (differentiation form), for the parameters whose tangent of this
// centre's radial functions is not identically zero.
struct CentreTan {
    int n_tan = 0;
    int par[WPCCC_MAX_PARAMS] = {};     // parameter of each stored table
    int slot[WPCCC_MAX_PARAMS] = {};    // stored table of each parameter, or -1
    double* df = nullptr;               // [n_tan][n_rad][Nr]
    double* dF = nullptr;               // [n_tan][n_fent][Nr]: derivative of the Eq. 7 table
};

// Per-category launch counts and (optionally) event-timed device durations.
struct Profiler {
    bool on = false;
    double ms[WPCCC_PROF_N] = {};
    long long launches[WPCCC_PROF_N] = {};
    std::vector<cudaEvent_t> pool;
    std::vector<cudaEvent_t> pending[WPCCC_PROF_N];   // start, stop, start, stop, ...
    cudaEvent_t begin(int cat, cudaStream_t st);
    void end(int cat, cudaStream_t st, cudaEvent_t e0);
    cudaError_t flush();
    void release();
};

}  // namespace wpccc

struct wpccc_basis_s {
    int device = 0;
    int n_centres = 1;
    int Nr = 0;
    int N_T = 0, N_P = 0, N = 0;
    double* r = nullptr;
    double* w = nullptr;
    double* inv_den = nullptr;  // [Nr-4][5] Lagrange denominators of the 5-point stencils
    wpccc::CentreDev T, P;
    // two-centre quadrature
    int Geta = 0, Gtau = 0, G = 0;
    double* s = nullptr;
    double* ws = nullptr;
    double* tau = nullptr;
    double* wtau = nullptr;
    double gamma = 0.5;
    int dmax = 0;               // lmax_T + lmax_P: largest |q - q'|
    int nlq_T = 0, nlq_P = 0;   // (l, q >= 0) pairs per centre
    // projectile states with q >= 0 ("half columns") of the molecular-frame integrals
    int n_half = 0;
    int* half_state = nullptr;  // [n_half] projectile state
    int* half_of = nullptr;     // [n_rad_P][WPCCC_LMAX+1]: half column of (radial, q>=0) or -1
    // work items of the Eq. 8 rotation (k_rotate): radial pairs grouped by (l_T, l_P), several pairs per warp
    int* rot_plan = nullptr;    // [n_rot_items][4] (first pair, pairs, l_T, l_P), then [pairs][2] (a, b)
    int n_rot_items = 0;
    int rot_cap = 0;            // largest block of one item: pairs x 2 (2 l_T + 1)(2 l_P + 1) entries
    // column tiles of the FP32 contraction: up to 16 half columns sharing one q
    int n_qtiles = 0;
    int* qtile_q = nullptr;     // [n_qtiles]
    int* qtile_cols = nullptr;  // [n_qtiles][16], -1 padded
    // scratch owned by the basis
    void* ws_ptr = nullptr;
    size_t ws_bytes = 0;
    size_t ws_limit = (size_t)8 << 30;
    int solve_mode = WPCCC_SOLVE_STAGE;
    int rk4_layout = WPCCC_RK4_AUTO;
    // short-range part of a Li-like target potential, V_T(r) = -[Z_T + mp_c e^{-mp_a r}(1 + mp_b r)]/r
    double mp_c = 0.0, mp_a = 0.0, mp_b = 0.0;
    // differentiation form
    int n_par = 0;
    double dexp[WPCCC_MAX_PARAMS][4] = {};   // d(Z_P, mp_c, mp_a, mp_b)/d theta_p
    double* deps = nullptr;                  // [n_par][N]: d eps_i / d theta_p per state
    wpccc::CentreTan tanT, tanP;
    int refine_iters = 2;       // FP64 refinement iterations of the mixed-precision form
    double refine_tol = 1e-3;   // largest last correction / solution of a refinement (<= 0: not checked)
    long wait_polls = 1L << 20; // polls of an mbarrier before a tensor-core kernel's wait gives up
    // tensor-core contraction (precision mode 3): node tables carry the split operand tables
    bool tc_layout = false;
    int n_qgroups = 0;          // row tiles: target states of one q', at most 56 per tile
    int* tc_row = nullptr;      // [2 N_T]: row of each target state in a split table, then its group's size
    int* tc_err = nullptr;      // device flag: a wait of the tensor-core pipeline gave up
    // tensor-core Schur update (schur_tc.cu): (A tile, B tile) pairs for N_P = su_np
    int* su_tiles = nullptr;
    int su_np = 0, su_ntiles = 0;
    int schur_update = WPCCC_SCHUR_UPDATE_AUTO;   // where the mixed Schur forms form I - K^+ K
    int* tc_halfq = nullptr;    // [n_half]: q of each half column
    float2* fT2 = nullptr;      // [n_rad_T][Nr]: the target's radial tables as double-floats (hi, lo)
    float2* fP2 = nullptr;      // the projectile's
    int* qg_off = nullptr;      // [n_qgroups + 1]: first split-table row of each tile (2 x cumulative size),
                                // then [n_qgroups]: the tile's q'
    int* qg_rows = nullptr;     // [n_qgroups][max tile size]: target state of each row of a tile
    int qg_max = 0;
    // second stream of wpccc_propagate (RK4 sweeps overlap the next chunk's assembly) and its events
    cudaStream_t rk_stream = nullptr;
    cudaEvent_t ev_asm[2] = {nullptr, nullptr}, ev_rk[2] = {nullptr, nullptr};
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    wpccc::Profiler prof;
};

namespace wpccc {

// one projectile position to evaluate
// The element kernels take one grid row (gridDim.y) per position, so one launch holds at most this many.
constexpr int MAX_EVALS_PER_LAUNCH = 65535;

struct EvalDesc {
    double b, v, z;
    int path;
    int pad;
};

// Layout of the per-evaluation scratch of the two-centre element kernels.
struct ElemScratch {
    size_t node_doubles;   // node tables per evaluation (in doubles, even)
    size_t w_off;          // offset of the complex node weights within them (even)
    size_t w_off_f;        // the same in the FP32 layout of the mixed-precision form (floats, even)
    size_t mol_elems;      // molecular-frame integrals per evaluation (complex)
    size_t bytes_per_eval;
    size_t et_doubles;     // small per-position tables (Wigner d, Legendre, stencil, F at R, phases), even
    size_t ph_off;         // offset of the per-state energy phases exp(i eps_i z / v) (complex, N of them)
    int dtot, npb;         // sizes of their Wigner-d and Legendre parts
    size_t cp_off[2];      // per centre: Eq. 6 coefficients of the position, [LM][LM][nlam] (see k_direct_coef)
    int tc_rows;           // rows of the tensor-core slice planes (2 N_T), when the basis enables the layout
    // tensor-core layout (precision modes 3-5): up to seven bf16 slice planes [7][tc_rows][G], then
    // (offsets in floats) the window scales, A_P and W_K / r_T as double-floats
    size_t t6_sc_off, t6_ap_off, t6_w_off;
};
ElemScratch elem_scratch_layout(const wpccc_basis_s* B);

// Queue the element kernels for `nev` evaluations (device list `evals`), writing
// S and H (matrix k at S + k*N*N).  S may be null (one-centre propagation).
// `scratch` must hold elem_scratch_layout(B).bytes_per_eval * nev bytes (unused in
// one-centre mode).
// precision 0: FP64 throughout; 1: the Eq. 9 contraction on the FP32 pipe (mixed-precision form).
wpccc_status launch_elements(wpccc_basis_s* B, const EvalDesc* evals, int nev,
                             double2* S, double2* H, void* scratch, cudaStream_t st, int precision = 0);

// Queue only the per-position tables of the element pipeline (k_eval_tables and, two-centre, the FP64
// node tables) for `nev` evaluations into `scratch` (layout of elem_scratch_layout).
wpccc_status launch_node_stage(wpccc_basis_s* B, const EvalDesc* evals, int nev, void* scratch, cudaStream_t st);

// Body of wpccc_propagate (argument checks, plan, kernels, status) on caller-owned amplitudes.
wpccc_status propagate_internal(wpccc_basis_s* B, const wpccc_paths* paths, int precision_mode, double2* c,
                                cudaStream_t st);

// Grows the basis-owned scratch buffer to at least `bytes`.
wpccc_status ensure_workspace(wpccc_basis_s* B, size_t bytes);

enum ProfCat { PROF_NODES = 0, PROF_MOL = 1, PROF_ROT_DIRECT = 2, PROF_SOLVE = 3, PROF_RK4 = 4, PROF_ADJ = 5 };

// Tensor-core form of the Eq. 9 contraction (precision mode 3): from the node tables of the tensor-core
// layout into the molecular-frame blocks, for `nev` evaluations.
wpccc_status tc_prepare(wpccc_basis_s* B);
wpccc_status rotation_plan(wpccc_basis_s* B);
// The tensor-core contraction over the slice planes: slices = 7 to FP64 accuracy (precision modes 4, 5),
// 3 at FP32 level (precision mode 3).
wpccc_status launch_mol_tc64(wpccc_basis_s* B, int nev, const void* node, double2* mol, int* err, cudaStream_t st,
                             int slices);

// Queue the batched FP32 factorisation P S = L U of FP64 matrices (mixed-precision form).
wpccc_status launch_factor_f32(int N, int batch, const double2* S, float2* LU, int* ipiv, int* info,
                               cudaStream_t st);

// Queue the batched Schur-complement factorisation of two-centre overlap matrices S (Cholesky factor of
// I - K^+ K into the lower triangle of S's projectile block; info as ZPOTRF).
wpccc_status launch_schur_factor(int N, int N_T, int batch, double2* S, int* info, cudaStream_t st);
// The same in FP32 into D (K rounded to FP32 and the Cholesky factor), S only read: the preconditioner
// of the mixed-precision forms' refinement.
wpccc_status launch_schur_factor_f32(int N, int N_T, int batch, const double2* S, float2* D, int* info,
                                     cudaStream_t st);

// The Cholesky factor of a trailing matrix I - K^+ K already in D's projectile block (K in FP32 in D).
wpccc_status launch_schur_cholesky_f32(int N, int N_T, int batch, float2* D, int* info, cudaStream_t st);
// The FP32 preconditioner of the mixed Schur forms with the rank-N_T update I - K^+ K on the tensor cores
// (schur_tc.cu); `scratch` holds at least `scratch_per_eval` bytes per evaluation.
bool schur_tc_applicable(const wpccc_basis_s* B, size_t scratch_per_eval);
// Its tile list and timeout flag, made on the host before any launch (and before a graph capture).
wpccc_status schur_tc_prepare(wpccc_basis_s* B);
wpccc_status launch_schur_factor_f32_tc(wpccc_basis_s* B, int nev, const double2* S, float2* D, int* info,
                                        void* scratch, size_t scratch_per_eval, cudaStream_t st);
// Allocates the device flag of the tensor-core kernels' bounded waits, if the basis has none yet.
wpccc_status ensure_tc_err(wpccc_basis_s* B);

// Queue the batched solve of S X = H (results in place).
wpccc_status launch_solve(int N, int batch, double2* S, double2* H, int* ipiv, int* info,
                          cudaStream_t st);

}  // namespace wpccc

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
