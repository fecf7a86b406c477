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

#include "wpccc_internal.cuh"

namespace wpccc {

wpccc_status ensure_workspace(wpccc_basis_s* B, size_t bytes);

struct PathChunk {
    int path;
    int nsteps;
    int start_local;   // eval (within the chunk) holding X at the first node, or -1: use the carry
    int first_local;   // eval of step 0's midpoint; step s uses first_local + 2s (mid), + 2s + 1 (new)
    int z0;            // index of the chunk's first node in the concatenated z array
    int pad;
    double v;
};

enum : int { FLAG_SINGULAR = 1, FLAG_NONFINITE = 2 };

constexpr int RK_THREADS = 512;

// k = -(i/v) X y   (X column-major N x N)
__device__ inline void apply_X(const double2* __restrict__ X, int N, double v, const double2* y, double2* k) {
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        double re = 0.0, im = 0.0;
        const double2* row = X + i;
        for (int j = 0; j < N; ++j) {
            const double2 a = row[(size_t)j * N];
            const double2 b = y[j];
            re = fma(a.x, b.x, re);
            re = fma(-a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(a.y, b.x, im);
        }
        // -(i/v) (re + i im) = (im - i re)/v
        k[i] = make_double2(im / v, -re / v);
    }
    __syncthreads();
}

// t <- S^{-1} t in place from the factors P S = L U (LAPACK layout, pivots 1-based);
// C2 = double2 (FP64 factors) or float2 (FP32 factors of the mixed-precision form).
// Blocked by 32 rows: each 32 x 32 diagonal block is staged in shared memory (blk) and solved by
// one warp; the off-diagonal updates run on every thread.
template <typename C2>
__device__ void lu_solve_inplace(const C2* __restrict__ LU, const int* __restrict__ piv, int N, C2* t, C2* blk) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        for (int r = 0; r < N; ++r) {
            const int p = piv[r] - 1;
            if (p != r) {
                const C2 q = t[r];
                t[r] = t[p];
                t[p] = q;
            }
        }
    // L z = P t, unit lower triangular
    for (int kb = 0; kb < N; kb += 32) {
        const int nb = min(32, N - kb);
        for (int q = tid; q < 32 * 32; q += RK_THREADS) {
            const int i = q & 31, j = q >> 5;
            if (i < nb && j < nb) blk[q] = LU[(size_t)(kb + i) + (size_t)(kb + j) * N];
        }
        __syncthreads();
        if (warp == 0) {
            C2 x = t[kb + (lane < nb ? lane : 0)];
            for (int j = 0; j < nb - 1; ++j) {
                const auto xr = __shfl_sync(0xffffffffu, x.x, j);
                const auto xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane > j && lane < nb) {
                    const C2 l = blk[j * 32 + lane];
                    x.x = fma(-l.x, xr, x.x);
                    x.x = fma(l.y, xi, x.x);
                    x.y = fma(-l.x, xi, x.y);
                    x.y = fma(-l.y, xr, x.y);
                }
            }
            if (lane < nb) t[kb + lane] = x;
        }
        __syncthreads();
        for (int i = kb + nb + tid; i < N; i += RK_THREADS) {
            C2 a = t[i];
            for (int j = 0; j < nb; ++j) {
                const C2 l = LU[(size_t)i + (size_t)(kb + j) * N];
                const C2 b = t[kb + j];
                a.x = fma(-l.x, b.x, a.x);
                a.x = fma(l.y, b.y, a.x);
                a.y = fma(-l.x, b.y, a.y);
                a.y = fma(-l.y, b.x, a.y);
            }
            t[i] = a;
        }
        __syncthreads();
    }
    // U x = z, upper triangular, from the bottom
    const int last = ((N - 1) / 32) * 32;
    for (int kb = last; kb >= 0; kb -= 32) {
        const int nb = min(32, N - kb);
        for (int q = tid; q < 32 * 32; q += RK_THREADS) {
            const int i = q & 31, j = q >> 5;
            if (i < nb && j < nb) blk[q] = LU[(size_t)(kb + i) + (size_t)(kb + j) * N];
        }
        __syncthreads();
        if (warp == 0) {
            C2 x = t[kb + (lane < nb ? lane : 0)];
            for (int j = nb - 1; j >= 0; --j) {
                if (lane == j) {
                    const C2 u = blk[j * 32 + j];
                    const auto d = u.x * u.x + u.y * u.y;
                    const auto ir = u.x / d, ii = -u.y / d;
                    const auto xr0 = x.x;
                    x.x = x.x * ir - x.y * ii;
                    x.y = xr0 * ii + x.y * ir;
                }
                const auto xr = __shfl_sync(0xffffffffu, x.x, j);
                const auto xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane < j) {
                    const C2 u = blk[j * 32 + lane];
                    x.x = fma(-u.x, xr, x.x);
                    x.x = fma(u.y, xi, x.x);
                    x.y = fma(-u.x, xi, x.y);
                    x.y = fma(-u.y, xr, x.y);
                }
            }
            if (lane < nb) t[kb + lane] = x;
        }
        __syncthreads();
        for (int i = tid; i < kb; i += RK_THREADS) {
            C2 a = t[i];
            for (int j = 0; j < nb; ++j) {
                const C2 u = LU[(size_t)i + (size_t)(kb + j) * N];
                const C2 b = t[kb + j];
                a.x = fma(-u.x, b.x, a.x);
                a.x = fma(u.y, b.y, a.x);
                a.y = fma(-u.x, b.y, a.y);
                a.y = fma(-u.y, b.x, a.y);
            }
            t[i] = a;
        }
        __syncthreads();
    }
}

// out = M y (FP64 matvec, M column-major N x N); out = b - M y when `residual` (b given).
__device__ inline void matvec(const double2* __restrict__ M, int N, const double2* y, double2* out,
                              const double2* b = nullptr) {
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        double re = 0.0, im = 0.0;
        const double2* row = M + i;
        for (int j = 0; j < N; ++j) {
            const double2 a = row[(size_t)j * N];
            const double2 q = y[j];
            re = fma(a.x, q.x, re);
            re = fma(-a.y, q.y, re);
            im = fma(a.x, q.y, im);
            im = fma(a.y, q.x, im);
        }
        out[i] = b ? make_double2(b[i].x - re, b[i].y - im) : make_double2(re, im);
    }
    __syncthreads();
}

// k = -(i/v) S^{-1} (H y) with S given by its FP64 LU factors.  t: shared scratch of N.
__device__ void apply_LU(const double2* __restrict__ LU, const int* __restrict__ piv,
                         const double2* __restrict__ Hm, int N, double v, const double2* y, double2* k,
                         double2* t, double2* blk) {
    matvec(Hm, N, y, t);
    lu_solve_inplace<double2>(LU, piv, N, t, blk);
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(t[i].y / v, -t[i].x / v);
    __syncthreads();
}

// Mixed-precision form: k = -(i/v) x with S x = H y solved by FP64 iterative refinement
// preconditioned by FP32 factors: x_0 = 0, r = H y - S x_n (FP64), x_{n+1} = x_n + (LU_32)^{-1} r.
// Shared scratch: b, x, r (double2) and d (float2), N each.
__device__ void apply_LU_mixed(const double2* __restrict__ S64, const float2* __restrict__ LU32,
                               const int* __restrict__ piv, const double2* __restrict__ Hm, int N, double v,
                               int iters, const double2* y, double2* k, double2* b, double2* x, double2* r,
                               float2* d, float2* blk) {
    matvec(Hm, N, y, b);
    for (int it = 0; it < iters; ++it) {
        const double2* rr = b;
        if (it > 0) {
            matvec(S64, N, x, r, b);
            rr = r;
        }
        for (int i = threadIdx.x; i < N; i += RK_THREADS) d[i] = make_float2((float)rr[i].x, (float)rr[i].y);
        __syncthreads();
        lu_solve_inplace<float2>(LU32, piv, N, d, blk);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 dx = make_double2((double)d[i].x, (double)d[i].y);
            x[i] = it == 0 ? dx : make_double2(x[i].x + dx.x, x[i].y + dx.y);
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(x[i].y / v, -x[i].x / v);
    __syncthreads();
}

struct RkArgs {
    int N;
    int iters;              // refinement iterations (mixed-precision form)
    const float2* LU32;     // chunk: FP32 factors per evaluation (mixed form)
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

enum RkMode { RK_MATRIX = 0, RK_STAGE = 1, RK_MIXED = 2 };

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
//   RK_MIXED   S^{-1} applied by FP64 refinement on FP32 factors
template <int MODE>
__global__ void __launch_bounds__(RK_THREADS) k_rk4(RkArgs A) {
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
    void* blk = MODE == RK_MIXED ? (void*)(ds + N + (N & 1)) : (void*)(t + N);
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
        m.L32 = MODE == RK_MIXED ? A.LU32 + (size_t)e * mat : nullptr;
        m.piv = MODE != RK_MATRIX ? A.piv + (size_t)e * N : nullptr;
        return m;
    };
    auto apply = [&](const PosMats& m, const double2* in, double2* out) {
        if (MODE == RK_MATRIX) {
            matvec(m.H, N, in, out);
            for (int i = threadIdx.x; i < N; i += RK_THREADS) out[i] = make_double2(out[i].y / v, -out[i].x / v);
            __syncthreads();
        } else if (MODE == RK_STAGE) {
            apply_LU(m.S, m.piv, m.H, N, v, in, out, t, static_cast<double2*>(blk));
        } else {
            apply_LU_mixed(m.S, m.L32, m.piv, m.H, N, v, A.iters, in, out, t, xs, rs, ds, static_cast<float2*>(blk));
        }
    };
    PosMats Mz;
    if (pc.start_local >= 0) {
        Mz = at(pc.start_local);
    } else {
        Mz.H = A.carryH + (size_t)pc.path * mat;
        Mz.S = MODE != RK_MATRIX ? A.carryLU + (size_t)pc.path * mat : nullptr;
        Mz.L32 = MODE == RK_MIXED ? A.carryLU32 + (size_t)pc.path * mat : nullptr;
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
        if (MODE == RK_MIXED) {
            float2* cL32 = A.carryLU32 + (size_t)pc.path * mat;
            for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cL32[q] = Mz.L32[q];
        }
    }
}

size_t rk_smem_bytes(int mode, int N) {
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

extern "C" wpccc_status wpccc_propagate(wpccc_basis B, const wpccc_paths* paths, int precision_mode,
                                        int batch_mode, void* c, void* stream) {
    if (!B || !paths || !c) return fail(WPCCC_EINVAL, "wpccc_propagate: null argument");
    if (precision_mode < 0 || precision_mode > 2)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: precision_mode must be 0, 1 or 2");
    if (batch_mode != 0) return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: only batch_mode 0");
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

    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool two = B->n_centres == 2;
    // 1: FP32 contraction + FP32 LU + FP64 refinement; 2: FP64 elements + FP32 LU + FP64 refinement
    const bool mixed = two && precision_mode >= 1;
    const int elem_precision = (two && precision_mode == 1) ? 1 : 0;
    const bool stage = two && !mixed && B->solve_mode == WPCCC_SOLVE_STAGE;
    const int mode = mixed ? RK_MIXED : (stage ? RK_STAGE : RK_MATRIX);
    const size_t mat = (size_t)N * N;
    const ElemScratch L = elem_scratch_layout(B);
    if (rk_smem_bytes(mode, N) > (size_t)227 * 1024)
        return fail(WPCCC_EINVAL, "wpccc_propagate: N too large for the RK4 kernel's shared memory in this mode");
    // device bytes per evaluation: S (two-centre only), H, pivots and info, element scratch
    const size_t per_eval = (two ? 2 : 1) * mat * sizeof(double2) + (mixed ? mat * sizeof(float2) : 0) +
                            L.bytes_per_eval + (two ? (size_t)N * sizeof(int) + sizeof(int) : 0) + sizeof(EvalDesc);

    int max_steps = 0;
    long long total_evals = 0;
    for (int p = 0; p < np; ++p) {
        int ns = paths->n_z[p] - 1;
        max_steps = std::max(max_steps, ns);
        if (ns > 0) total_evals += 2LL * ns + 1;
    }
    if (max_steps == 0) return WPCCC_OK;

    // fixed part of the workspace: carry matrices, z nodes, plan, flags
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t fixed = align((size_t)np * mat * sizeof(double2)) * (mode != RK_MATRIX ? 2 : 1) +
                         (mixed ? align((size_t)np * mat * sizeof(float2)) : 0) +
                         align((size_t)np * N * sizeof(int)) + align((size_t)zoff[np] * sizeof(double)) +
                         align((size_t)total_evals * sizeof(EvalDesc)) +
                         align((size_t)np * max_steps * sizeof(PathChunk)) + 16 * 256;
    // Steps per chunk.  Two chunks are in flight (the RK4 sweep of one overlaps the assembly of the
    // next), so each buffer set gets half the budget.  Aim for at least four chunks per call, each
    // with enough positions (>= 2 per SM) to fill the GPU.
    size_t budget = B->ws_limit > fixed ? B->ws_limit - fixed : 0;
    long long cap_evals = (long long)(budget / (2 * per_eval));
    int dev_sms = 0;
    WPCCC_CUDA(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, B->device));
    const long long cap_steps = std::max<long long>(1, (cap_evals - np) / (2LL * np));
    const long long fill_steps = std::max<long long>(1, (2LL * dev_sms / np + 1) / 2);
    long long want = std::max<long long>((max_steps + 3) / 4, fill_steps);
    int C = (int)std::max<long long>(1, std::min<long long>({(long long)max_steps, cap_steps, want}));
    const int n_chunks = (max_steps + C - 1) / C;

    // plan: evaluations and path chunks for every chunk
    std::vector<EvalDesc> ev;
    ev.reserve(total_evals);
    std::vector<PathChunk> pcs;
    std::vector<int> ev_begin(n_chunks + 1), pc_begin(n_chunks + 1);
    for (int ch = 0; ch < n_chunks; ++ch) {
        ev_begin[ch] = (int)ev.size();
        pc_begin[ch] = (int)pcs.size();
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
            const int base = ev_begin[ch];
            if (s0 == 0) {
                pc.start_local = (int)ev.size() - base;
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], zp[0], p, 0});
            }
            pc.first_local = (int)ev.size() - base;
            for (int s = s0; s < s0 + n; ++s) {
                const double za = zp[s], zb = zp[s + 1];
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], (za + zb) / 2.0, p, 0});
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], zb, p, 0});
            }
            pcs.push_back(pc);
        }
    }
    ev_begin[n_chunks] = (int)ev.size();
    pc_begin[n_chunks] = (int)pcs.size();
    int max_chunk_evals = 0;
    for (int ch = 0; ch < n_chunks; ++ch) max_chunk_evals = std::max(max_chunk_evals, ev_begin[ch + 1] - ev_begin[ch]);

    // workspace carve-up
    const size_t sz_carry = align((size_t)np * mat * sizeof(double2));
    const size_t sz_carryLU = mode != RK_MATRIX ? sz_carry : 0;
    const size_t sz_carryPiv = mode != RK_MATRIX ? align((size_t)np * N * sizeof(int)) : 0;
    const size_t sz_carryLU32 = mixed ? align((size_t)np * mat * sizeof(float2)) : 0;
    const size_t sz_LU32 = mixed ? align((size_t)max_chunk_evals * mat * sizeof(float2)) * 2 : 0;
    const size_t sz_z = align((size_t)zoff[np] * sizeof(double));
    const size_t sz_ev = align(ev.size() * sizeof(EvalDesc));
    const size_t sz_pc = align(pcs.size() * sizeof(PathChunk));
    const size_t sz_flags = 256;
    // two buffer sets (chunk parity) for what the RK4 sweep reads
    const size_t sz_S = two ? align((size_t)max_chunk_evals * mat * sizeof(double2)) * 2 : 0;
    const size_t sz_H = align((size_t)max_chunk_evals * mat * sizeof(double2)) * 2;
    const size_t sz_piv = two ? align((size_t)max_chunk_evals * N * sizeof(int)) * 2 : 0;
    const size_t sz_info = two ? align((size_t)max_chunk_evals * sizeof(int)) * 2 : 0;
    const size_t sz_scr = align((size_t)max_chunk_evals * L.bytes_per_eval);
    const size_t need = sz_carry + sz_carryLU + sz_carryPiv + sz_carryLU32 + sz_LU32 + sz_z + sz_ev + sz_pc +
                        sz_flags + sz_S + sz_H + sz_piv + sz_info + sz_scr;
    wpccc_status s = ensure_workspace(B, need);
    if (s != WPCCC_OK) return s;
    char* w = static_cast<char*>(B->ws_ptr);
    double2* d_carry = reinterpret_cast<double2*>(w);
    w += sz_carry;
    double2* d_carryLU = mode != RK_MATRIX ? reinterpret_cast<double2*>(w) : nullptr;
    w += sz_carryLU;
    int* d_carryPiv = mode != RK_MATRIX ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_carryPiv;
    float2* d_carryLU32 = mixed ? reinterpret_cast<float2*>(w) : nullptr;
    w += sz_carryLU32;
    float2* d_LU32 = mixed ? reinterpret_cast<float2*>(w) : nullptr;
    w += sz_LU32;
    double* d_z = reinterpret_cast<double*>(w);
    w += sz_z;
    EvalDesc* d_ev = reinterpret_cast<EvalDesc*>(w);
    w += sz_ev;
    PathChunk* d_pc = reinterpret_cast<PathChunk*>(w);
    w += sz_pc;
    int* d_flags = reinterpret_cast<int*>(w);
    w += sz_flags;
    double2* d_S = two ? reinterpret_cast<double2*>(w) : nullptr;
    w += sz_S;
    double2* d_H = reinterpret_cast<double2*>(w);
    w += sz_H;
    int* d_piv = two ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_piv;
    int* d_info = two ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_info;
    void* d_scr = w;

    // half-buffers of each set
    const size_t hS = sz_S / 2 / sizeof(double2), hH = sz_H / 2 / sizeof(double2);
    const size_t hL = sz_LU32 / 2 / sizeof(float2), hP = sz_piv / 2 / sizeof(int), hI = sz_info / 2 / sizeof(int);
    if (!B->rk_stream) {
        WPCCC_CUDA(cudaStreamCreateWithFlags(&B->rk_stream, cudaStreamNonBlocking));
        for (int k = 0; k < 2; ++k) {
            WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_asm[k], cudaEventDisableTiming));
            WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_rk[k], cudaEventDisableTiming));
        }
        WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
        WPCCC_CUDA(cudaEventCreateWithFlags(&B->ev_join, cudaEventDisableTiming));
    }
    cudaStream_t rs = B->rk_stream;

    WPCCC_CUDA(cudaMemcpyAsync(d_z, paths->z, (size_t)zoff[np] * sizeof(double), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(d_ev, ev.data(), ev.size() * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(d_pc, pcs.data(), pcs.size() * sizeof(PathChunk), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), st));
    const int rk_smem = (int)rk_smem_bytes(mode, N);
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_MATRIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<RK_MIXED>, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));
    RkArgs ra;
    ra.N = N;
    ra.iters = B->refine_iters;
    ra.H = d_H;
    ra.LU = mode != RK_MATRIX ? d_S : nullptr;
    ra.LU32 = d_LU32;
    ra.carryLU32 = d_carryLU32;
    ra.piv = mode != RK_MATRIX ? d_piv : nullptr;
    ra.info = d_info;
    ra.carryH = d_carry;
    ra.carryLU = d_carryLU;
    ra.carryPiv = d_carryPiv;
    ra.c = static_cast<double2*>(c);
    ra.z = d_z;
    ra.flags = d_flags;

    // the RK4 stream starts after everything queued so far on the caller's stream
    WPCCC_CUDA(cudaEventRecord(B->ev_fork, st));
    WPCCC_CUDA(cudaStreamWaitEvent(rs, B->ev_fork, 0));
    for (int ch = 0; ch < n_chunks; ++ch) {
        const int nev = ev_begin[ch + 1] - ev_begin[ch];
        const int npc = pc_begin[ch + 1] - pc_begin[ch];
        const int k = ch & 1;
        double2* bS = two ? d_S + k * hS : nullptr;
        double2* bH = d_H + k * hH;
        float2* bL = mixed ? d_LU32 + k * hL : nullptr;
        int* bP = two ? d_piv + k * hP : nullptr;
        int* bI = two ? d_info + k * hI : nullptr;
        // buffer set k is free once the RK4 sweep of chunk ch - 2 is done
        if (ch >= 2) WPCCC_CUDA(cudaStreamWaitEvent(st, B->ev_rk[k], 0));
        s = launch_elements(B, d_ev + ev_begin[ch], nev, bS, bH, d_scr, st, elem_precision);
        if (s != WPCCC_OK) return s;
        if (two) {
            cudaEvent_t e0 = B->prof.begin(PROF_SOLVE, st);
            if (mixed) s = launch_factor_f32(N, nev, bS, bL, bP, bI, st);
            else s = launch_solve(N, nev, bS, stage ? nullptr : bH, bP, bI, st);
            if (s != WPCCC_OK) return s;
            B->prof.end(PROF_SOLVE, st, e0);
        }
        WPCCC_CUDA(cudaEventRecord(B->ev_asm[k], st));
        WPCCC_CUDA(cudaStreamWaitEvent(rs, B->ev_asm[k], 0));
        cudaEvent_t e1 = B->prof.begin(PROF_RK4, rs);
        ra.pcs = d_pc + pc_begin[ch];
        ra.H = bH;
        ra.LU = mode != RK_MATRIX ? bS : nullptr;
        ra.LU32 = bL;
        ra.piv = mode != RK_MATRIX ? bP : nullptr;
        ra.info = bI;
        if (mode == RK_MIXED) k_rk4<RK_MIXED><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else if (mode == RK_STAGE) k_rk4<RK_STAGE><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        else k_rk4<RK_MATRIX><<<npc, RK_THREADS, rk_smem, rs>>>(ra);
        WPCCC_CHECK_LAUNCH("k_rk4");
        B->prof.end(PROF_RK4, rs, e1);
        WPCCC_CUDA(cudaEventRecord(B->ev_rk[k], rs));
    }
    // the caller's stream resumes after the last sweep
    WPCCC_CUDA(cudaEventRecord(B->ev_join, rs));
    WPCCC_CUDA(cudaStreamWaitEvent(st, B->ev_join, 0));
    int flags = 0;
    WPCCC_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaStreamSynchronize(st));
    if (flags & FLAG_SINGULAR) return fail(WPCCC_ESINGULAR, "wpccc_propagate: an overlap matrix had a zero pivot");
    if (flags & FLAG_NONFINITE) return fail(WPCCC_ENONFINITE, "wpccc_propagate: amplitudes became non-finite");
    return WPCCC_OK;
}
