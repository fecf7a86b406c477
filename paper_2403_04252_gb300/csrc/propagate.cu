// Propagation of the amplitudes (Algorithm 1) and the probabilities.
//
// M(z) = -(i/v) S(z)^{-1} H(z) depends on the path and z only, never on the
// amplitudes, so the positions an RK4 step needs (z_mid and z_new; z of the
// first node once per path) are evaluated ahead of the sweep: for a chunk of
// steps of every path, all matrix elements are assembled and all systems
// solved in batched launches, then one fused RK4 kernel per chunk advances
// every path through the chunk's steps.  The matrix at the last node of a
// chunk is carried over to the next.
#include <algorithm>
#include <cmath>
#include <vector>

#include "rk_device.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

struct PathChunk {
    int path;
    int nsteps;
    int start_local;   // eval (within the chunk) holding X at the first node, or -1: use the carry
    int first_local;   // eval of step 0's midpoint; step s uses first_local + 2s (mid), + 2s + 1 (new)
    int z0;            // index of the chunk's first node in the concatenated z array
    int pad;
    double v;
};


struct RkArgs {
    int N;
    int N_T;                // target states (two-centre: S = [[I, K], [K^+, I]])
    int iters;              // refinement iterations (mixed-precision form)
    int df_rhs;             // reduced-precision forms: H y in double-float arithmetic (matvec_df)
    int stage_cols;         // > 0: H streamed through shared memory, this many columns per slot (matvec_df_staged)
    long long stage_off;    // byte offset of the staging slots in the dynamic shared memory
    long polls;             // bound of a staging wait
    double tol;             // convergence tolerance of the refinement's last sweep (<= 0: unchecked)
    const float2* LU32;     // chunk: FP32 factors per evaluation (mixed forms: LU, or K and the Schur factor)
    float2* carryLU32;      // per path (mixed form)
    const double2* H;       // chunk: H (one-centre, or X = S^{-1} H in matrix mode) per evaluation
    const double2* LU;      // chunk: LU factors of S (stage mode) or S itself (mixed form) per evaluation
    const int* piv;         // chunk: pivots per evaluation (stage mode)
    const int* info;        // chunk: solve status per evaluation (two-centre), else null
    double2* carryH;        // per path: the matrix (or H) at the last node of the previous chunk
    double2* carryLU;       // per path (stage mode)
    int* carryPiv;          // per path (stage mode)
    double2* c;             // [n_paths][N]
    const double* z;
    const PathChunk* pcs;
    int* flags;
};

enum RkMode { RK_MATRIX = 0, RK_STAGE = 1, RK_MIXED = 2, RK_SCHUR = 3, RK_MIXED_SCHUR = 4 };

// Matrices of one position as the RK4 kernel sees them.
struct PosMats {
    const double2* H;     // H (or X = S^{-1} H in matrix mode)
    const double2* S;     // FP64 LU factors (stage mode) or FP64 S (mixed form)
    const float2* L32;    // FP32 factors (mixed form)
    const int* piv;
};

// One block per path: the chunk's RK4 steps (Algorithm 1) with M(z) y = -(i/v) S(z)^{-1} H(z) y:
//   RK_MATRIX  X = S^{-1} H stored (the paper's form; one-centre: X = H)
//   RK_STAGE   S^{-1} applied from FP64 LU factors at every stage
//   RK_SCHUR   S^{-1} applied through the Schur complement's Cholesky factor at every stage
//   RK_MIXED   S^{-1} applied by FP64 refinement on FP32 LU factors
//   RK_MIXED_SCHUR  the same on the FP32 Schur factors
template <int MODE>
__global__ void __launch_bounds__(RK_THREADS, 1) k_rk4(RkArgs A) {
    extern __shared__ double2 rk_smem[];
    const int N = A.N;
    double2* c = rk_smem;
    double2* y = c + N;
    double2* kv = y + N;
    double2* acc = kv + N;
    double2* t = acc + N;                       // stage: scratch; mixed: b
    double2* xs = t + N;                        // mixed: x
    double2* rs = xs + N;                       // mixed: r
    float2* ds = reinterpret_cast<float2*>(rs + N);   // mixed: d
    // 32 x 32 diagonal block of the triangular solves (after the vectors of the mode)
    double2* us = t + N;                        // Schur: scratch of the projectile part
    float2* us32 = ds + N + (N & 1);            // mixed Schur: FP32 scratch of the projectile part
    constexpr bool MIX = MODE == RK_MIXED || MODE == RK_MIXED_SCHUR;
    void* blk = MODE == RK_MIXED ? (void*)(ds + N + (N & 1))
                                 : MODE == RK_MIXED_SCHUR ? (void*)(us32 + N + (N & 1))
                                                          : (MODE == RK_SCHUR ? (void*)(us + N) : (void*)(t + N));
    const PathChunk pc = A.pcs[blockIdx.x];
    const size_t mat = (size_t)N * N;
    double2* cg = A.c + (size_t)pc.path * N;
    const double v = pc.v;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) c[i] = cg[i];
    if (A.info && threadIdx.x == 0) {
        int bad = 0;
        if (pc.start_local >= 0 && A.info[pc.start_local] != 0) bad = 1;
        for (int s = 0; s < 2 * pc.nsteps; ++s)
            if (A.info[pc.first_local + s] != 0) bad = 1;
        if (bad) atomicOr(A.flags, FLAG_SINGULAR);
    }
    __syncthreads();
    auto at = [&](int e) {
        PosMats m;
        m.H = A.H + (size_t)e * mat;
        m.S = MODE != RK_MATRIX ? A.LU + (size_t)e * mat : nullptr;
        m.L32 = MIX ? A.LU32 + (size_t)e * mat : nullptr;
        m.piv = MODE != RK_MATRIX ? A.piv + (size_t)e * N : nullptr;
        return m;
    };
    // the staging slots of H for the reduced-precision forms' right-hand side (after the mode's vectors)
    Staging sg{};
    const Staging* sgp = nullptr;
    if (MIX && A.stage_cols > 0) {
        sg.buf = reinterpret_cast<double2*>(reinterpret_cast<char*>(rk_smem) + A.stage_off);
        sg.bars = reinterpret_cast<uint64_t*>(sg.buf + (size_t)2 * A.stage_cols * N);
        sg.cols = A.stage_cols;
        sg.polls = A.polls;
        sgp = &sg;
    }
    auto apply = [&](const PosMats& m, const double2* in, double2* out) {
        if (MODE == RK_MATRIX) {
            matvec(m.H, N, in, out);
            for (int i = threadIdx.x; i < N; i += RK_THREADS) out[i] = make_double2(out[i].y / v, -out[i].x / v);
            __syncthreads();
        } else if (MODE == RK_SCHUR) {
            apply_schur(m.S, m.H, N, A.N_T, v, in, out, t, us, static_cast<double2*>(blk));
        } else if (MODE == RK_STAGE) {
            apply_LU(m.S, m.piv, m.H, N, v, in, out, t, static_cast<double2*>(blk));
        } else if (MODE == RK_MIXED_SCHUR) {
            apply_schur_mixed(m.S, m.L32, m.H, N, A.N_T, v, A.iters, in, out, t, xs, rs, ds, us32,
                              static_cast<float2*>(blk), A.tol, A.flags, A.df_rhs != 0, sgp);
        } else {
            apply_LU_mixed(m.S, m.L32, m.piv, m.H, N, A.N_T, v, A.iters, in, out, t, xs, rs, ds,
                           static_cast<float2*>(blk), A.tol, A.flags, A.df_rhs != 0, sgp);
        }
    };
    PosMats Mz;
    if (pc.start_local >= 0) {
        Mz = at(pc.start_local);
    } else {
        Mz.H = A.carryH + (size_t)pc.path * mat;
        Mz.S = MODE != RK_MATRIX ? A.carryLU + (size_t)pc.path * mat : nullptr;
        Mz.L32 = MIX ? A.carryLU32 + (size_t)pc.path * mat : nullptr;
        Mz.piv = MODE != RK_MATRIX ? A.carryPiv + (size_t)pc.path * N : nullptr;
    }
    for (int s = 0; s < pc.nsteps; ++s) {
        const PosMats Mmid = at(pc.first_local + 2 * s), Mnew = at(pc.first_local + 2 * s + 1);
        const double h = A.z[pc.z0 + s + 1] - A.z[pc.z0 + s];
        const double h2 = 0.5 * h, h6 = h / 6.0;
        // K1 = M_z c
        apply(Mz, c, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = kv[i];
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K2 = M_mid (c + h/2 K1)
        apply(Mmid, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K3 = M_mid (c + h/2 K2)
        apply(Mmid, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h, kv[i].x, c[i].x), fma(h, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K4 = M_new (c + h K3)
        apply(Mnew, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 a = make_double2(acc[i].x + kv[i].x, acc[i].y + kv[i].y);
            c[i] = make_double2(fma(h6, a.x, c[i].x), fma(h6, a.y, c[i].y));
        }
        __syncthreads();
        Mz = Mnew;
    }
    bool finite = true;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        cg[i] = c[i];
        if (!isfinite(c[i].x) || !isfinite(c[i].y)) finite = false;
    }
    if (!finite) atomicOr(A.flags, FLAG_NONFINITE);
    // carry the matrices at the chunk's last node into the next chunk
    double2* cH = A.carryH + (size_t)pc.path * mat;
    if (Mz.H != cH) {
        for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cH[q] = Mz.H[q];
        if (MODE != RK_MATRIX) {
            double2* cL = A.carryLU + (size_t)pc.path * mat;
            int* cP = A.carryPiv + (size_t)pc.path * N;
            for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cL[q] = Mz.S[q];
            for (int q = threadIdx.x; q < N; q += RK_THREADS) cP[q] = Mz.piv[q];
        }
        if (MIX) {
            float2* cL32 = A.carryLU32 + (size_t)pc.path * mat;
            for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cL32[q] = Mz.L32[q];
        }
    }
}

// ---------------------------------------------------------------------------
// RK4 with the vectors in global memory (one-centre form, any N): one launch per stage for all paths of
// a chunk.  Stage 1 reads c and writes y_a, stage 2 reads y_a and writes y_b, stage 3 reads y_b and
// writes y_a, stage 4 reads y_a and updates c; each thread owns one row of every vector, so the
// per-row updates need no further synchronisation, and the launch boundary orders the stages.
// ---------------------------------------------------------------------------
constexpr int WIDE_ROWS = 128;   // rows (threads) per block
constexpr int WIDE_TJ = 256;     // columns of the input vector staged in shared memory at a time

struct WideArgs {
    int N;
    const double2* H;        // chunk: H per evaluation (M = -(i/v) H)
    const PathChunk* pcs;
    double2* c;              // [n_paths][N]
    double2 *ya, *yb, *acc;  // [chunk paths][N]
    const double* z;
    int* flags;
};

__global__ void __launch_bounds__(WIDE_ROWS) k_rk4_wide(WideArgs A, int s, int stage) {
    __shared__ double2 sy[WIDE_TJ];
    const PathChunk pc = A.pcs[blockIdx.y];
    if (s >= pc.nsteps) return;   // the whole block: the path has fewer steps in this chunk
    const int N = A.N;
    const int i = blockIdx.x * WIDE_ROWS + threadIdx.x;
    // position of the stage: the step's first node (the chunk's first evaluation, or the previous
    // step's last node), its midpoint twice, then its last node
    const int e = stage == 1 ? (s == 0 ? pc.start_local : pc.first_local + 2 * s - 1)
                             : (stage == 4 ? pc.first_local + 2 * s + 1 : pc.first_local + 2 * s);
    const double2* M = A.H + (size_t)e * N * N;
    double2* cp = A.c + (size_t)pc.path * N;
    const size_t vo = (size_t)blockIdx.y * N;
    const double2* in = stage == 1 ? cp : (stage == 3 ? A.yb + vo : A.ya + vo);
    double re = 0.0, im = 0.0;
    for (int j0 = 0; j0 < N; j0 += WIDE_TJ) {
        const int nj = min(WIDE_TJ, N - j0);
        for (int q = threadIdx.x; q < nj; q += WIDE_ROWS) sy[q] = in[j0 + q];
        __syncthreads();
        if (i < N) {
            const double2* col = M + i + (size_t)j0 * N;   // column-major: consecutive rows coalesce
            for (int q = 0; q < nj; ++q) {
                const double2 a = col[(size_t)q * N];
                const double2 b = sy[q];
                re = fma(a.x, b.x, re);
                re = fma(-a.y, b.y, re);
                im = fma(a.x, b.y, im);
                im = fma(a.y, b.x, im);
            }
        }
        __syncthreads();
    }
    if (i >= N) return;
    const double v = pc.v;
    const double h = A.z[pc.z0 + s + 1] - A.z[pc.z0 + s];
    const double2 k = make_double2(im / v, -re / v);   // -(i/v) (H y)_i
    const double2 ci = cp[i];
    double2* acc = A.acc + vo;
    if (stage == 1) {
        acc[i] = k;
        A.ya[vo + i] = make_double2(ci.x + 0.5 * h * k.x, ci.y + 0.5 * h * k.y);
    } else if (stage == 2) {
        acc[i] = make_double2(acc[i].x + 2.0 * k.x, acc[i].y + 2.0 * k.y);
        A.yb[vo + i] = make_double2(ci.x + 0.5 * h * k.x, ci.y + 0.5 * h * k.y);
    } else if (stage == 3) {
        acc[i] = make_double2(acc[i].x + 2.0 * k.x, acc[i].y + 2.0 * k.y);
        A.ya[vo + i] = make_double2(ci.x + h * k.x, ci.y + h * k.y);
    } else {
        const double2 a = acc[i];
        const double2 cn = make_double2(ci.x + (h / 6.0) * (a.x + k.x), ci.y + (h / 6.0) * (a.y + k.y));
        if (!isfinite(cn.x) || !isfinite(cn.y)) atomicOr(A.flags, FLAG_NONFINITE);
        cp[i] = cn;
    }
}

size_t rk_smem_bytes(int mode, int N) {
    if (mode == RK_SCHUR) return (size_t)N * 6 * sizeof(double2) + 32 * 32 * sizeof(double2);
    if (mode == RK_MIXED_SCHUR)
        return (size_t)N * 7 * sizeof(double2) + 2 * (size_t)(N + (N & 1)) * sizeof(float2) + 32 * 32 * sizeof(float2);
    return mode == RK_MIXED ? (size_t)N * 7 * sizeof(double2) + (size_t)(N + (N & 1)) * sizeof(float2) +
                                  32 * 32 * sizeof(float2)
                            : (size_t)N * 5 * sizeof(double2) + 32 * 32 * sizeof(double2);
}

__global__ void k_probabilities(long long n, const double2* __restrict__ c, double* __restrict__ P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double2 a = c[i];
        P[i] = a.x * a.x + a.y * a.y;
    }
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_probabilities(int n_paths, int N, const void* c, double* P, void* stream) {
    if (n_paths < 0 || N < 1) return fail(WPCCC_EINVAL, "wpccc_probabilities: bad sizes");
    if (n_paths == 0) return WPCCC_OK;
    if (!c || !P) return fail(WPCCC_EINVAL, "wpccc_probabilities: null pointer");
    long long n = (long long)n_paths * N;
    k_probabilities<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, static_cast<const double2*>(c), P);
    WPCCC_CHECK_LAUNCH("k_probabilities");
    return WPCCC_OK;
}

namespace wpccc {

// ---------------------------------------------------------------------------
// propagation plan: the positions every chunk of RK4 steps needs, the buffer layout, and the
// launch sequence (used directly by wpccc_propagate and captured into a graph by wpccc_batch)
// ---------------------------------------------------------------------------
struct PropPlan {
    wpccc_basis_s* B = nullptr;
    int np = 0, N = 0, mode = RK_MATRIX, elem_precision = 0, C = 1, n_chunks = 0, max_chunk_evals = 0;
    int max_steps = 0;
    bool two = false, mixed = false, stage = false, schur = false;
    bool schur_tc = false;   // mixed Schur forms: the trailing update I - K^+ K on the tensor cores
    bool df_rhs = false;     // reduced-precision forms (1, 2, 3): H y on the FP32 pipe in double-float arithmetic
    bool wide = false;       // one-centre RK4 with the vectors in global memory (k_rk4_wide)
    size_t per_eval = 0, fixed = 0;
    std::vector<double> z;
    std::vector<EvalDesc> ev;
    std::vector<PathChunk> pcs;
    std::vector<int> ev_begin, pc_begin;
    size_t sz_carry = 0, sz_carryLU = 0, sz_carryPiv = 0, sz_carryLU32 = 0, sz_LU32 = 0, sz_z = 0, sz_ev = 0,
           sz_pc = 0, sz_flags = 0, sz_S = 0, sz_H = 0, sz_piv = 0, sz_info = 0, sz_scr = 0, sz_vec = 0, bytes = 0;
    double2 *d_carry = nullptr, *d_carryLU = nullptr, *d_S = nullptr, *d_H = nullptr, *d_vec = nullptr;
    int *d_carryPiv = nullptr, *d_flags = nullptr, *d_piv = nullptr, *d_info = nullptr;
    float2 *d_carryLU32 = nullptr, *d_LU32 = nullptr;
    double* d_z = nullptr;
    EvalDesc* d_ev = nullptr;
    PathChunk* d_pc = nullptr;
    void* d_scr = nullptr;
};

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Validates the paths and lays out the plan.  C_request > 0 fixes the RK4 steps per chunk,
// otherwise they are chosen from the workspace limit and the SM count.
static wpccc_status plan_build(wpccc_basis_s* B, const wpccc_paths* paths, int precision_mode, int C_request,
                               size_t ws_limit, PropPlan& P) {
    if (precision_mode < 0 || precision_mode > 5)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: precision_mode must be 0 to 5");
    if ((precision_mode == 1 || precision_mode >= 3) && B->n_centres == 2 && B->mp_c != 0.0)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: model-potential targets need FP64 elements (mode 0 or 2)");
    if (precision_mode >= 3 && B->n_centres == 2) {
        if (B->G % 128 != 0)
            return fail(WPCCC_EUNSUPPORTED, "precision modes 3-5 need a node count that is a multiple of 128");
        wpccc_status ts = tc_prepare(B);
        if (ts != WPCCC_OK) return ts;
    }
    const int np = paths->n_paths;
    if (np < 1 || !paths->b || !paths->v || !paths->n_z || !paths->z)
        return fail(WPCCC_EINVAL, "wpccc_propagate: empty or null path description");
    std::vector<int> zoff(np + 1, 0);
    for (int p = 0; p < np; ++p) {
        if (!(paths->b[p] > 0.0) || !(paths->v[p] > 0.0))
            return fail(WPCCC_EINVAL, "wpccc_propagate: b and v must be > 0");
        if (paths->n_z[p] < 1) return fail(WPCCC_EINVAL, "wpccc_propagate: n_z < 1");
        zoff[p + 1] = zoff[p] + paths->n_z[p];
        for (int k = zoff[p] + 1; k < zoff[p + 1]; ++k)
            if (!(paths->z[k] > paths->z[k - 1]))
                return fail(WPCCC_EINVAL, "wpccc_propagate: z nodes must increase strictly");
    }
    const int N = B->N;
    if (N > WPCCC_NMAX) return fail(WPCCC_EINVAL, "wpccc_propagate: N too large");
    P = PropPlan();
    P.B = B;
    P.np = np;
    P.N = N;
    P.two = B->n_centres == 2;
    // 1: FP32 contraction + FP32 factors + FP64 refinement; 2: FP64 elements + FP32 factors + FP64
    // refinement; 3: as 1 with the contraction on the tensor cores (three bf16 slices); 4: FP64 form with
    // the contraction on the tensor cores to FP64 accuracy (seven slices); 5: as 2 with mode 4's elements
    P.mixed = P.two && precision_mode >= 1 && precision_mode != 4;
    P.df_rhs = P.mixed && precision_mode != 5;
    P.elem_precision = !P.two ? 0
                       : (precision_mode == 1 || precision_mode == 3) ? precision_mode
                       : (precision_mode == 4 || precision_mode == 5) ? 4 : 0;
    P.stage = P.two && !P.mixed && B->solve_mode != WPCCC_SOLVE_MATRIX;
    P.schur = P.two && B->solve_mode == WPCCC_SOLVE_SCHUR;
    const bool want_tc = B->schur_update == WPCCC_SCHUR_UPDATE_TENSOR ||
                         (B->schur_update == WPCCC_SCHUR_UPDATE_AUTO && B->N_P >= 256);
    P.schur_tc = P.mixed && P.schur && want_tc && schur_tc_applicable(B, elem_scratch_layout(B).bytes_per_eval);
    if (P.schur_tc) {
        wpccc_status ts = schur_tc_prepare(B);
        if (ts != WPCCC_OK) return ts;
    }
    P.mode = P.mixed ? (P.schur ? RK_MIXED_SCHUR : RK_MIXED) : (P.schur ? RK_SCHUR : (P.stage ? RK_STAGE : RK_MATRIX));
    // 227 KB per block, less the kernels' static shared memory (the refinement check's reduction)
    const bool fits = rk_smem_bytes(P.mode, N) + 1024 <= (size_t)227 * 1024;
    if (P.two && B->rk4_layout == WPCCC_RK4_GLOBAL)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: the global-memory RK4 layout is one-centre only");
    P.wide = !P.two && (B->rk4_layout == WPCCC_RK4_GLOBAL || (B->rk4_layout == WPCCC_RK4_AUTO && !fits));
    if (!P.wide && !fits)
        return fail(WPCCC_EINVAL, "wpccc_propagate: N too large for the RK4 kernel's shared memory in this mode");
    const size_t mat = (size_t)N * N;
    const ElemScratch L = elem_scratch_layout(B);
    // device bytes per evaluation: S (two-centre only), H, FP32 factors, pivots and info, element scratch
    P.per_eval = (P.two ? 2 : 1) * mat * sizeof(double2) + (P.mixed ? mat * sizeof(float2) : 0) + L.bytes_per_eval +
                 (P.two ? (size_t)N * sizeof(int) + sizeof(int) : 0) + sizeof(EvalDesc);
    long long total_evals = 0;
    for (int p = 0; p < np; ++p) {
        int ns = paths->n_z[p] - 1;
        P.max_steps = std::max(P.max_steps, ns);
        if (ns > 0) total_evals += 2LL * ns + 1;
    }
    P.z.assign(paths->z, paths->z + zoff[np]);
    if (P.max_steps == 0) return WPCCC_OK;
    P.fixed = (P.wide ? align256((size_t)3 * np * N * sizeof(double2))
                      : align256((size_t)np * mat * sizeof(double2)) * (P.mode != RK_MATRIX ? 2 : 1)) +
              (P.mixed ? align256((size_t)np * mat * sizeof(float2)) : 0) + align256((size_t)np * N * sizeof(int)) +
              align256((size_t)zoff[np] * sizeof(double)) + align256((size_t)total_evals * sizeof(EvalDesc)) +
              align256((size_t)np * P.max_steps * sizeof(PathChunk)) + 16 * 256;
    // a chunk evaluates at most 2C + 1 positions per path in one launch of each element kernel
    if (3LL * np > MAX_EVALS_PER_LAUNCH)
        return fail(WPCCC_EINVAL, "wpccc_propagate: more than " + std::to_string(MAX_EVALS_PER_LAUNCH / 3) +
                                      " paths in one call");
    const int C_launch = (int)((MAX_EVALS_PER_LAUNCH / np - 1) / 2);
    int C;
    if (C_request > 0) {
        C = std::min({C_request, P.max_steps, C_launch});
    } else {
        // Two chunks are in flight (the RK4 sweep of one overlaps the assembly of the next), so each
        // buffer set gets half the budget.  Aim for at least four chunks per call, each with enough
        // positions (>= 2 per SM) to fill the GPU.
        size_t budget = ws_limit > P.fixed ? ws_limit - P.fixed : 0;
        long long cap_evals = (long long)(budget / (2 * P.per_eval));
        int dev_sms = 0;
        WPCCC_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, B->device));
        const long long cap_steps = std::max<long long>(1, (cap_evals - np) / (2LL * np));
        const long long fill_steps = std::max<long long>(1, (2LL * dev_sms / np + 1) / 2);
        long long want = std::max<long long>((P.max_steps + 3) / 4, fill_steps);
        C = (int)std::max<long long>(1, std::min<long long>({(long long)P.max_steps, cap_steps, want,
                                                              (long long)C_launch}));
    }
    P.C = C;
    P.n_chunks = (P.max_steps + C - 1) / C;
    P.ev.reserve(total_evals);
    P.ev_begin.assign(P.n_chunks + 1, 0);
    P.pc_begin.assign(P.n_chunks + 1, 0);
    for (int ch = 0; ch < P.n_chunks; ++ch) {
        P.ev_begin[ch] = (int)P.ev.size();
        P.pc_begin[ch] = (int)P.pcs.size();
        const int s0 = ch * C;
        for (int p = 0; p < np; ++p) {
            const int ns = paths->n_z[p] - 1;
            if (s0 >= ns) continue;
            const int n = std::min(C, ns - s0);
            const double* zp = paths->z + zoff[p];
            PathChunk pc;
            pc.path = p;
            pc.nsteps = n;
            pc.v = paths->v[p];
            pc.z0 = zoff[p] + s0;
            pc.pad = 0;
            pc.start_local = -1;
            const int base = P.ev_begin[ch];
            if (s0 == 0 || P.wide) {
                // the path's first node; in the global-memory layout every chunk evaluates its first node
                // again (instead of carrying an N x N matrix over)
                pc.start_local = (int)P.ev.size() - base;
                P.ev.push_back(EvalDesc{paths->b[p], paths->v[p], zp[s0], p, 0});
            }
            pc.first_local = (int)P.ev.size() - base;
            for (int s = s0; s < s0 + n; ++s) {
                const double za = zp[s], zb = zp[s + 1];
                P.ev.push_back(EvalDesc{paths->b[p], paths->v[p], (za + zb) / 2.0, p, 0});
                P.ev.push_back(EvalDesc{paths->b[p], paths->v[p], zb, p, 0});
            }
            P.pcs.push_back(pc);
        }
    }
    P.ev_begin[P.n_chunks] = (int)P.ev.size();
    P.pc_begin[P.n_chunks] = (int)P.pcs.size();
    for (int ch = 0; ch < P.n_chunks; ++ch)
        P.max_chunk_evals = std::max(P.max_chunk_evals, P.ev_begin[ch + 1] - P.ev_begin[ch]);
    const int mce = P.max_chunk_evals;
    P.sz_carry = P.wide ? 0 : align256((size_t)np * mat * sizeof(double2));
    P.sz_vec = P.wide ? align256((size_t)3 * np * N * sizeof(double2)) : 0;
    P.sz_carryLU = P.mode != RK_MATRIX ? P.sz_carry : 0;
    P.sz_carryPiv = P.mode != RK_MATRIX ? align256((size_t)np * N * sizeof(int)) : 0;
    P.sz_carryLU32 = P.mixed ? align256((size_t)np * mat * sizeof(float2)) : 0;
    P.sz_LU32 = P.mixed ? align256((size_t)mce * mat * sizeof(float2)) * 2 : 0;
    P.sz_z = align256((size_t)zoff[np] * sizeof(double));
    P.sz_ev = align256(P.ev.size() * sizeof(EvalDesc));
    P.sz_pc = align256(P.pcs.size() * sizeof(PathChunk));
    P.sz_flags = 256;
    // two buffer sets (chunk parity) for what the RK4 sweep reads
    P.sz_S = P.two ? align256((size_t)mce * mat * sizeof(double2)) * 2 : 0;
    P.sz_H = align256((size_t)mce * mat * sizeof(double2)) * 2;
    P.sz_piv = P.two ? align256((size_t)mce * N * sizeof(int)) * 2 : 0;
    P.sz_info = P.two ? align256((size_t)mce * sizeof(int)) * 2 : 0;
    P.sz_scr = align256((size_t)mce * L.bytes_per_eval);
    P.bytes = P.sz_carry + P.sz_carryLU + P.sz_carryPiv + P.sz_carryLU32 + P.sz_LU32 + P.sz_z + P.sz_ev + P.sz_pc +
              P.sz_flags + P.sz_S + P.sz_H + P.sz_piv + P.sz_info + P.sz_scr + P.sz_vec;
    return WPCCC_OK;
}

static void plan_bind(PropPlan& P, void* ws) {
    char* w = static_cast<char*>(ws);
    auto take = [&](size_t n) {
        char* p = n ? w : nullptr;
        w += n;
        return p;
    };
    P.d_carry = reinterpret_cast<double2*>(take(P.sz_carry));
    P.d_carryLU = reinterpret_cast<double2*>(take(P.sz_carryLU));
    P.d_carryPiv = reinterpret_cast<int*>(take(P.sz_carryPiv));
    P.d_carryLU32 = reinterpret_cast<float2*>(take(P.sz_carryLU32));
    P.d_LU32 = reinterpret_cast<float2*>(take(P.sz_LU32));
    P.d_z = reinterpret_cast<double*>(take(P.sz_z));
    P.d_ev = reinterpret_cast<EvalDesc*>(take(P.sz_ev));
    P.d_pc = reinterpret_cast<PathChunk*>(take(P.sz_pc));
    P.d_flags = reinterpret_cast<int*>(take(P.sz_flags));
    P.d_S = reinterpret_cast<double2*>(take(P.sz_S));
    P.d_H = reinterpret_cast<double2*>(take(P.sz_H));
    P.d_piv = reinterpret_cast<int*>(take(P.sz_piv));
    P.d_info = reinterpret_cast<int*>(take(P.sz_info));
    P.d_scr = take(P.sz_scr);
    P.d_vec = reinterpret_cast<double2*>(take(P.sz_vec));
}

// Copies the plan's node, position and chunk lists to the device (from its host vectors, which
// must stay alive until the copies have run).
static wpccc_status plan_upload(PropPlan& P, cudaStream_t st) {
    if (P.max_steps == 0) return WPCCC_OK;
    WPCCC_CUDA(cudaMemcpyAsync(P.d_z, P.z.data(), P.z.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(P.d_ev, P.ev.data(), P.ev.size() * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(P.d_pc, P.pcs.data(), P.pcs.size() * sizeof(PathChunk), cudaMemcpyHostToDevice, st));
    return WPCCC_OK;
}

struct PlanStreams {
    cudaStream_t st, rs;          // assembly (and the caller's order), RK4 sweeps
    cudaEvent_t asm_done[2], rk_done[2], fork, join;
};

// Queues every kernel of the plan: the flags reset, then per chunk the element kernels and the
// solve on S.st, the RK4 sweep on S.rs, with double-buffered chunks.  Capturable into a graph.
static wpccc_status plan_enqueue(PropPlan& P, double2* c, const PlanStreams& S) {
    if (P.max_steps == 0) return WPCCC_OK;
    wpccc_basis_s* B = P.B;
    const int N = P.N;
    cudaStream_t st = S.st, rs = S.rs;
    WPCCC_CUDA(cudaMemsetAsync(P.d_flags, 0, sizeof(int), st));
    int rk_smem = P.wide ? 0 : (int)rk_smem_bytes(P.mode, N);
    // reduced-precision forms with N <= RK_THREADS: H streamed through two shared-memory slots of up to eight
    // columns each, in what the mode's vectors leave of the 227 KB
    int stage_cols = 0;
    size_t stage_off = 0;
    const size_t rk_cap = (size_t)227 * 1024 - 1024;
    if (!P.wide && P.df_rhs && N <= RK_THREADS) {
        stage_off = ((size_t)rk_smem + 127) / 128 * 128;
        if (rk_cap > stage_off + 16)
            stage_cols = (int)std::min<size_t>(8, (rk_cap - stage_off - 16) / (2 * (size_t)N * sizeof(double2)));
        if (stage_cols >= 1) rk_smem = (int)(stage_off + 2 * (size_t)stage_cols * N * sizeof(double2) + 16);
        else stage_cols = 0;
    }
    if (!P.wide) {
        // the largest any plan takes (a batch graph holds launches of several plans)
        const int mx = (int)rk_cap;
        WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_MATRIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_SCHUR>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
        WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_MIXED_SCHUR>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx));
    }
    const size_t hS = P.sz_S / 2 / sizeof(double2), hH = P.sz_H / 2 / sizeof(double2);
    const size_t hL = P.sz_LU32 / 2 / sizeof(float2), hP = P.sz_piv / 2 / sizeof(int), hI = P.sz_info / 2 / sizeof(int);
    RkArgs ra;
    ra.N = N;
    ra.N_T = B->N_T;
    ra.iters = B->refine_iters;
    ra.df_rhs = P.df_rhs ? 1 : 0;
    ra.stage_cols = stage_cols;
    ra.stage_off = (long long)stage_off;
    ra.polls = B->wait_polls;
    ra.tol = B->refine_tol;
    ra.carryH = P.d_carry;
    ra.carryLU = P.d_carryLU;
    ra.carryPiv = P.d_carryPiv;
    ra.carryLU32 = P.d_carryLU32;
    ra.c = c;
    ra.z = P.d_z;
    ra.flags = P.d_flags;
    // the RK4 stream starts after everything queued so far on the assembly stream
    WPCCC_CUDA(cudaEventRecord(S.fork, st));
    WPCCC_CUDA(cudaStreamWaitEvent(rs, S.fork, 0));
    wpccc_status s;
    for (int ch = 0; ch < P.n_chunks; ++ch) {
        const int nev = P.ev_begin[ch + 1] - P.ev_begin[ch];
        const int npc = P.pc_begin[ch + 1] - P.pc_begin[ch];
        const int k = ch & 1;
        double2* bS = P.two ? P.d_S + k * hS : nullptr;
        double2* bH = P.d_H + k * hH;
        float2* bL = P.mixed ? P.d_LU32 + k * hL : nullptr;
        int* bP = P.two ? P.d_piv + k * hP : nullptr;
        int* bI = P.two ? P.d_info + k * hI : nullptr;
        // buffer set k is free once the RK4 sweep of chunk ch - 2 is done
        if (ch >= 2) WPCCC_CUDA(cudaStreamWaitEvent(st, S.rk_done[k], 0));
        s = launch_elements(B, P.d_ev + P.ev_begin[ch], nev, bS, bH, P.d_scr, st, P.elem_precision);
        if (s != WPCCC_OK) return s;
        if (P.two) {
            cudaEvent_t e0 = B->prof.begin(PROF_SOLVE, st);
            if (P.mixed && P.schur && P.schur_tc)
                s = launch_schur_factor_f32_tc(B, nev, bS, bL, bI, P.d_scr, elem_scratch_layout(B).bytes_per_eval, st);
            else if (P.mixed && P.schur) s = launch_schur_factor_f32(N, B->N_T, nev, bS, bL, bI, st);
            else if (P.mixed) s = launch_factor_f32(N, nev, bS, bL, bP, bI, st);
            else if (P.schur) s = launch_schur_factor(N, B->N_T, nev, bS, bI, st);
            else s = launch_solve(N, nev, bS, P.stage ? nullptr : bH, bP, bI, st);
            if (s != WPCCC_OK) return s;
            B->prof.end(PROF_SOLVE, st, e0);
        }
        WPCCC_CUDA(cudaEventRecord(S.asm_done[k], st));
        WPCCC_CUDA(cudaStreamWaitEvent(rs, S.asm_done[k], 0));
        cudaEvent_t e1 = B->prof.begin(PROF_RK4, rs);
        ra.pcs = P.d_pc + P.pc_begin[ch];
        ra.H = bH;
        ra.LU = P.mode != RK_MATRIX ? bS : nullptr;
        ra.LU32 = bL;
        ra.piv = P.mode != RK_MATRIX ? bP : nullptr;
        ra.info = bI;
        if (P.wide) {
            WideArgs wa;
            wa.N = N;
            wa.H = bH;
            wa.pcs = ra.pcs;
            wa.c = c;
            wa.ya = P.d_vec;
            wa.yb = P.d_vec + (size_t)P.np * N;
            wa.acc = P.d_vec + (size_t)2 * P.np * N;
            wa.z = P.d_z;
            wa.flags = P.d_flags;
            const int steps = std::min(P.C, P.max_steps - ch * P.C);
            const dim3 grid((N + WIDE_ROWS - 1) / WIDE_ROWS, npc);
            for (int s2 = 0; s2 < steps; ++s2)
                for (int stage = 1; stage <= 4; ++stage) k_rk4_wide<<<grid, WIDE_ROWS, 0, rs>>>(wa, s2, stage);
        } else if (P.mode == RK_MIXED) k_rk4<RK_MIXED><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else if (P.mode == RK_MIXED_SCHUR) k_rk4<RK_MIXED_SCHUR><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else if (P.mode == RK_SCHUR) k_rk4<RK_SCHUR><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else if (P.mode == RK_STAGE) k_rk4<RK_STAGE><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else k_rk4<RK_MATRIX><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        WPCCC_CHECK_LAUNCH("k_rk4");
        B->prof.end(PROF_RK4, rs, e1);
        WPCCC_CUDA(cudaEventRecord(S.rk_done[k], rs));
    }
    // the assembly stream resumes after the last sweep
    WPCCC_CUDA(cudaEventRecord(S.join, rs));
    WPCCC_CUDA(cudaStreamWaitEvent(st, S.join, 0));
    return WPCCC_OK;
}

static wpccc_status flags_status(int flags) {
    if (flags & FLAG_SINGULAR) return fail(WPCCC_ESINGULAR, "an overlap matrix had a zero pivot");
    if (flags & FLAG_NONFINITE) return fail(WPCCC_ENONFINITE, "amplitudes became non-finite");
    if (flags & FLAG_TIMEOUT)
        return fail(WPCCC_ETIMEOUT, "a wait of the RK4 sweep's matrix staging timed out");
    if (flags & FLAG_NOCONV)
        return fail(WPCCC_ENOCONV, "the FP64 refinement of a reduced-precision solve did not converge (last "
                                   "correction above the tolerance relative to the solution)");
    return WPCCC_OK;
}

static wpccc_status basis_streams(wpccc_basis_s* B) {
    if (B->rk_stream) return WPCCC_OK;
    WPCCC_CUDA(cudaStreamCreateWithFlags(&B->rk_stream, cudaStreamNonBlocking));
    for (int k = 0; k < 2; ++k) {
        WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_asm[k], cudaEventDisableTiming));
        WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_rk[k], cudaEventDisableTiming));
    }
    WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
    WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming));
    return WPCCC_OK;
}

}  // namespace wpccc

namespace wpccc {

wpccc_status propagate_internal(wpccc_basis_s* B, const wpccc_paths* paths, int precision_mode, double2* c,
                                cudaStream_t st) {
    PropPlan P;
    wpccc_status s = plan_build(B, paths, precision_mode, 0, B->ws_limit, P);
    if (s != WPCCC_OK) return s;
    if (P.max_steps == 0) return WPCCC_OK;
    if ((s = ensure_workspace(B, P.bytes)) != WPCCC_OK) return s;
    plan_bind(P, B->ws_ptr);
    if ((s = basis_streams(B)) != WPCCC_OK) return s;
    if ((s = plan_upload(P, st)) != WPCCC_OK) return s;
    PlanStreams S{st, B->rk_stream, {B->ev_asm[0], B->ev_asm[1]}, {B->ev_rk[0], B->ev_rk[1]}, B->ev_fork,
                  B->ev_join};
    if ((s = plan_enqueue(P, c, S)) != WPCCC_OK) return s;
    int flags = 0;
    WPCCC_CUDA(cudaMemcpyAsync(&flags, P.d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaStreamSynchronize(st));
    if (B->tc_err) {
        int e = 0;
        WPCCC_CUDA(cudaMemcpy(&e, B->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            WPCCC_CUDA(cudaMemset(B->tc_err, 0, sizeof(int)));
            return fail(WPCCC_ETIMEOUT, "wpccc_propagate: a wait of a tensor-core kernel timed out (stage " +
                                         std::to_string(e) + ")");
        }
    }
    s = flags_status(flags);
    if (s != WPCCC_OK) set_error(std::string("wpccc_propagate: ") + wpccc_last_error());
    return s;
}

}  // namespace wpccc

extern "C" wpccc_status wpccc_propagate(wpccc_basis B, const wpccc_paths* paths, int precision_mode,
                                        int batch_mode, void* c, void* stream) {
    if (!B || !paths || !c) return fail(WPCCC_EINVAL, "wpccc_propagate: null argument");
    if (batch_mode != 0) return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: only batch_mode 0");
    WPCCC_CUDA(cudaSetDevice(B->device));
    return propagate_internal(B, paths, precision_mode, static_cast<double2*>(c), static_cast<cudaStream_t>(stream));
}

// ---------------------------------------------------------------------------
// batches: several (basis, paths) sets propagated together by one CUDA graph launch
// ---------------------------------------------------------------------------
struct wpccc_batch_s {
    int device = 0;
    int n_sets = 0;
    std::vector<wpccc::PropPlan> plans;
    std::vector<double2*> c;
    void* ws = nullptr;
    std::vector<cudaStream_t> streams;      // two per set (assembly, RK4), plus the capture stream
    std::vector<cudaEvent_t> events;        // six per set, plus the capture fork
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<int> chunk_steps;
    std::vector<double> tuned_ms_per_step;
};

namespace wpccc {

static void batch_free(wpccc_batch_s* X) {
    if (!X) return;
    cudaSetDevice(X->device);
    for (cudaStream_t s : X->streams)
        if (s) cudaStreamSynchronize(s);
    if (X->exec) cudaGraphExecDestroy(X->exec);
    if (X->graph) cudaGraphDestroy(X->graph);
    for (cudaEvent_t e : X->events)
        if (e) cudaEventDestroy(e);
    for (cudaStream_t s : X->streams)
        if (s) cudaStreamDestroy(s);
    if (X->ws) cudaFree(X->ws);
    delete X;
}

// Times one candidate schedule of a set on its first steps: a warm run, then a timed run.
static wpccc_status tune_trial(wpccc_basis_s* B, const wpccc_paths* paths, int precision, int C, double2* c_src,
                               double* ms_per_step) {
    // the set's paths cut to 2C steps (at least two chunks, so the overlap is part of the timing)
    const int np = paths->n_paths;
    std::vector<int> nz(np);
    std::vector<double> z;
    int steps = 0;
    int off = 0;
    for (int p = 0; p < np; ++p) {
        const int n = std::min(paths->n_z[p], 2 * C + 1);
        nz[p] = n;
        z.insert(z.end(), paths->z + off, paths->z + off + n);
        off += paths->n_z[p];
        steps = std::max(steps, n - 1);
    }
    if (steps == 0) {
        *ms_per_step = 0.0;
        return WPCCC_OK;
    }
    wpccc_paths tp{np, paths->b, paths->v, nz.data(), z.data()};
    PropPlan P;
    wpccc_status s = plan_build(B, &tp, precision, C, B->ws_limit, P);
    if (s != WPCCC_OK) return s;
    void* ws = nullptr;
    double2* c = nullptr;
    cudaStream_t st = nullptr, rs = nullptr;
    cudaEvent_t ev[8] = {};
    float ms = 0.f;
    auto cleanup = [&]() {
        if (st) cudaStreamSynchronize(st);
        for (cudaEvent_t e : ev)
            if (e) cudaEventDestroy(e);
        if (st) cudaStreamDestroy(st);
        if (rs) cudaStreamDestroy(rs);
        if (ws) cudaFree(ws);
        if (c) cudaFree(c);
    };
    cudaError_t e = cudaMalloc(&ws, P.bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c, (size_t)np * P.N * sizeof(double2));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&rs, cudaStreamNonBlocking);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&ev[k], cudaEventDisableTiming);
    for (int k = 6; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreate(&ev[k]);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c, c_src, (size_t)np * P.N * sizeof(double2), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) {
        cleanup();
        return cuda_fail(e, "autotuner trial set-up");
    }
    plan_bind(P, ws);
    PlanStreams S{st, rs, {ev[0], ev[1]}, {ev[2], ev[3]}, ev[4], ev[5]};
    for (int rep = 0; rep < 2 && s == WPCCC_OK; ++rep) {
        if ((s = plan_upload(P, st)) != WPCCC_OK) break;
        if (rep == 1) cudaEventRecord(ev[6], st);
        s = plan_enqueue(P, c, S);
        if (rep == 1) cudaEventRecord(ev[7], st);
        if (cudaStreamSynchronize(st) != cudaSuccess && s == WPCCC_OK) s = cuda_fail(cudaGetLastError(), "trial");
    }
    if (s == WPCCC_OK) {
        cudaEventElapsedTime(&ms, ev[6], ev[7]);
        *ms_per_step = ms / steps;
    }
    cleanup();
    return s;
}

}  // namespace wpccc

extern "C" wpccc_status wpccc_batch_create(int n_sets, const wpccc_basis* bases, const wpccc_paths* paths,
                                           int precision_mode, void* const* c, int autotune, wpccc_batch* out) {
    if (!bases || !paths || !c || !out || n_sets < 1) return fail(WPCCC_EINVAL, "wpccc_batch_create: bad arguments");
    *out = nullptr;
    const int device = bases[0] ? bases[0]->device : -1;
    for (int k = 0; k < n_sets; ++k) {
        if (!bases[k] || !c[k]) return fail(WPCCC_EINVAL, "wpccc_batch_create: null basis or amplitudes");
        if (bases[k]->device != device) return fail(WPCCC_EINVAL, "wpccc_batch_create: bases on different devices");
    }
    WPCCC_CUDA(cudaSetDevice(device));
    wpccc_batch_s* X = new wpccc_batch_s();
    X->device = device;
    X->n_sets = n_sets;
    X->plans.resize(n_sets);
    X->c.resize(n_sets);
    X->chunk_steps.assign(n_sets, 0);
    X->tuned_ms_per_step.assign(n_sets, 0.0);
    auto bail = [&](wpccc_status st) {
        std::string keep = wpccc_last_error();
        batch_free(X);
        set_error(keep);
        return st;
    };
    wpccc_status s;
    for (int k = 0; k < n_sets; ++k) {
        wpccc_basis_s* B = bases[k];
        X->c[k] = static_cast<double2*>(c[k]);
        PropPlan P;
        if ((s = plan_build(B, &paths[k], precision_mode, 0, B->ws_limit, P)) != WPCCC_OK) return bail(s);
        int best = P.C;
        if (autotune && P.max_steps > 1) {
            // schedules tried: the default chunk and half and twice as many RK4 steps per chunk
            std::vector<int> cand{P.C};
            if (P.C / 2 >= 1) cand.push_back(P.C / 2);
            if (2 * P.C <= P.max_steps) cand.push_back(2 * P.C);
            double best_ms = -1.0;
            for (int C : cand) {
                double ms = 0.0;
                const bool was_on = B->prof.on;
                B->prof.on = false;
                s = tune_trial(B, &paths[k], precision_mode, C, X->c[k], &ms);
                B->prof.on = was_on;
                if (s != WPCCC_OK) return bail(s);
                if (best_ms < 0.0 || ms < best_ms) {
                    best_ms = ms;
                    best = C;
                }
            }
            X->tuned_ms_per_step[k] = best_ms;
        }
        if ((s = plan_build(B, &paths[k], precision_mode, best, B->ws_limit, X->plans[k])) != WPCCC_OK) return bail(s);
        X->chunk_steps[k] = X->plans[k].C;
    }
    // one workspace for every set
    size_t total = 0;
    for (auto& P : X->plans) total += align256(P.bytes);
    {
        cudaError_t e = cudaMalloc(&X->ws, std::max<size_t>(total, 256));
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaMalloc(batch workspace)"));
    }
    size_t off = 0;
    for (auto& P : X->plans) {
        plan_bind(P, static_cast<char*>(X->ws) + off);
        off += align256(P.bytes);
    }
    // streams and events, then the plans' lists on the device (before the capture)
    X->streams.assign(2 * n_sets + 1, nullptr);
    X->events.assign(6 * n_sets + 1, nullptr);
    for (auto& st : X->streams) {
        cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamCreate(batch)"));
    }
    for (auto& ev : X->events) {
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return bail(cuda_fail(e, "cudaEventCreate(batch)"));
    }
    cudaStream_t cap = X->streams[2 * n_sets];
    for (int k = 0; k < n_sets; ++k)
        if ((s = plan_upload(X->plans[k], cap)) != WPCCC_OK) return bail(s);
    {
        cudaError_t e = cudaStreamSynchronize(cap);
        if (e != cudaSuccess) return bail(cuda_fail(e, "batch upload"));
    }
    // capture every set's launch sequence into one graph: fork from the capture stream, join back
    std::vector<bool> prof_on(n_sets);
    for (int k = 0; k < n_sets; ++k) {
        prof_on[k] = bases[k]->prof.on;
        bases[k]->prof.on = false;
    }
    auto restore = [&]() {
        for (int k = 0; k < n_sets; ++k) bases[k]->prof.on = prof_on[k];
    };
    {
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            restore();
            return bail(cuda_fail(e, "cudaStreamBeginCapture"));
        }
    }
    cudaEvent_t fork = X->events[6 * n_sets];
    wpccc_status cs = WPCCC_OK;
    if (cudaEventRecord(fork, cap) != cudaSuccess) cs = cuda_fail(cudaGetLastError(), "capture fork");
    for (int k = 0; k < n_sets && cs == WPCCC_OK; ++k) {
        cudaStream_t st = X->streams[2 * k], rs = X->streams[2 * k + 1];
        cudaEvent_t* ev = &X->events[6 * k];
        if (cudaStreamWaitEvent(st, fork, 0) != cudaSuccess) {
            cs = cuda_fail(cudaGetLastError(), "capture fork wait");
            break;
        }
        PlanStreams S{st, rs, {ev[0], ev[1]}, {ev[2], ev[3]}, ev[4], ev[5]};
        cs = plan_enqueue(X->plans[k], X->c[k], S);
        if (cs != WPCCC_OK) break;
        // join: the capture stream waits for this set's assembly stream (which waits for its sweeps)
        if (cudaEventRecord(ev[5], st) != cudaSuccess || cudaStreamWaitEvent(cap, ev[5], 0) != cudaSuccess)
            cs = cuda_fail(cudaGetLastError(), "capture join");
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cap, &graph);
    restore();
    if (cs != WPCCC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return bail(cs);
    }
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaStreamEndCapture"));
    X->graph = graph;
    e = cudaGraphInstantiate(&X->exec, graph, 0);
    if (e != cudaSuccess) return bail(cuda_fail(e, "cudaGraphInstantiate"));
    *out = X;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_batch_launch(wpccc_batch X, void* stream) {
    if (!X) return fail(WPCCC_EINVAL, "wpccc_batch_launch: null batch");
    WPCCC_CUDA(cudaSetDevice(X->device));
    WPCCC_CUDA(cudaGraphLaunch(X->exec, static_cast<cudaStream_t>(stream)));
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_batch_status(wpccc_batch X, void* stream) {
    if (!X) return fail(WPCCC_EINVAL, "wpccc_batch_status: null batch");
    WPCCC_CUDA(cudaSetDevice(X->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<int> flags(X->n_sets, 0);
    for (int k = 0; k < X->n_sets; ++k)
        if (X->plans[k].d_flags)
            WPCCC_CUDA(cudaMemcpyAsync(&flags[k], X->plans[k].d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaStreamSynchronize(st));
    for (int k = 0; k < X->n_sets; ++k) {
        wpccc_basis_s* B = X->plans[k].B;
        if (B && B->tc_err) {
            int e = 0;
            WPCCC_CUDA(cudaMemcpy(&e, B->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
            if (e) {
                WPCCC_CUDA(cudaMemset(B->tc_err, 0, sizeof(int)));
                return fail(WPCCC_ETIMEOUT, "wpccc_batch_status: a wait of the tensor-core contraction timed out");
            }
        }
    }
    int all = 0;
    for (int f : flags) all |= f;
    wpccc_status s = flags_status(all);
    if (s != WPCCC_OK) set_error(std::string("wpccc_batch_status: ") + wpccc_last_error());
    return s;
}

extern "C" wpccc_status wpccc_batch_info(wpccc_batch X, int* chunk_steps, double* tuned_ms_per_step) {
    if (!X) return fail(WPCCC_EINVAL, "wpccc_batch_info: null batch");
    for (int k = 0; k < X->n_sets; ++k) {
        if (chunk_steps) chunk_steps[k] = X->chunk_steps[k];
        if (tuned_ms_per_step) tuned_ms_per_step[k] = X->tuned_ms_per_step[k];
    }
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_batch_destroy(wpccc_batch X) {
    batch_free(X);
    return WPCCC_OK;
}
