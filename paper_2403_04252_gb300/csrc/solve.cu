// Batched complex linear solve S X = H with partial pivoting (the paper's ZGESV
// step of Eq. 4), one thread block per system, in FP64.
//
// Blocked right-looking elimination of the augmented matrix [S | H]:
//   for each panel of NB columns
//     1. unblocked LU of the panel with partial pivoting (largest |re|+|im|,
//        lowest row on ties, as LAPACK's izamax)
//     2. the panel's row interchanges applied to every other column of S and H
//     3. U12 = L11^{-1} A12 for the trailing columns of S and all columns of H
//     4. trailing update A22 -= L21 U12 (complex GEMM on the FP64 pipe)
//   then blocked back substitution X = U^{-1} Y on H.
// S is left holding L and U of P S = L U (LAPACK layout), H holds X.
#include <algorithm>

#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int NB = 32;            // panel width (the triangular solves map one row per lane)
static_assert(NB == 32, "NB must equal the warp size");
constexpr int LU_THREADS = 256;
constexpr int TM = 64, TN = 32;   // update tile, complex elements

// C[m x n] -= A[m x k] * B[k x n], column-major, k <= NB, whole block cooperating.
__device__ void cta_gemm_sub(double2* __restrict__ C, int ldc, const double2* __restrict__ A, int lda,
                             const double2* __restrict__ B, int ldb, int m, int n, int k,
                             double2* sA, double2* sB) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int i0 = 0; i0 < m; i0 += TM) {
        // A tile: sA[kk][ii]
        for (int idx = tid; idx < TM * NB; idx += LU_THREADS) {
            int ii = idx % TM, kk = idx / TM;
            sA[kk * TM + ii] = (i0 + ii < m && kk < k) ? A[(size_t)(i0 + ii) + (size_t)kk * lda]
                                                       : make_double2(0.0, 0.0);
        }
        for (int j0 = 0; j0 < n; j0 += TN) {
            for (int idx = tid; idx < NB * TN; idx += LU_THREADS) {
                int kk = idx % NB, jj = idx / NB;
                sB[kk * TN + jj] = (j0 + jj < n && kk < k) ? B[(size_t)kk + (size_t)(j0 + jj) * ldb]
                                                           : make_double2(0.0, 0.0);
            }
            __syncthreads();
            double2 acc[4][2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) acc[a][c] = make_double2(0.0, 0.0);
            for (int kk = 0; kk < k; ++kk) {
                double2 av[4], bv[2];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = sA[kk * TM + ty + 16 * a];
#pragma unroll
                for (int c = 0; c < 2; ++c) bv[c] = sB[kk * TN + tx + 16 * c];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        acc[a][c].x = fma(av[a].x, bv[c].x, acc[a][c].x);
                        acc[a][c].x = fma(-av[a].y, bv[c].y, acc[a][c].x);
                        acc[a][c].y = fma(av[a].x, bv[c].y, acc[a][c].y);
                        acc[a][c].y = fma(av[a].y, bv[c].x, acc[a][c].y);
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                int i = i0 + ty + 16 * a;
                if (i >= m) continue;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    int j = j0 + tx + 16 * c;
                    if (j >= n) continue;
                    double2* p = C + (size_t)i + (size_t)j * ldc;
                    double2 v = *p;
                    v.x -= acc[a][c].x;
                    v.y -= acc[a][c].y;
                    *p = v;
                }
            }
            __syncthreads();
        }
    }
}

__device__ inline double2 crecip(double2 a) {
    double d = a.x * a.x + a.y * a.y;
    return make_double2(a.x / d, -a.y / d);
}

__global__ void __launch_bounds__(LU_THREADS) k_lu_solve(int N, double2* __restrict__ Sall,
                                                         double2* __restrict__ Hall, int* __restrict__ ipiv_all,
                                                         int* __restrict__ info_all) {
    extern __shared__ double2 lu_smem[];
    double2* sA = lu_smem;                 // TM * NB
    double2* sB = sA + TM * NB;            // NB * TN
    double2* sT = sB + NB * TN;            // NB * NB triangular block
    double2* sD = sT + NB * NB;            // NB reciprocals of U's diagonal
    __shared__ double red_v[LU_THREADS / 32];
    __shared__ int red_i[LU_THREADS / 32];
    __shared__ int s_piv[NB];
    __shared__ int s_info;

    const int sys = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t mat = (size_t)N * N;
    double2* A = Sall + (size_t)sys * mat;
    double2* Bm = Hall ? Hall + (size_t)sys * mat : nullptr;
    int* ipiv = ipiv_all + (size_t)sys * N;
    if (tid == 0) s_info = 0;
    __syncthreads();

    for (int k0 = 0; k0 < N; k0 += NB) {
        const int nb = min(NB, N - k0);
        // ---- 1. panel factorisation
        for (int kk = 0; kk < nb; ++kk) {
            const int k = k0 + kk;
            double best = -1.0;
            int bi = N;
            for (int i = k + tid; i < N; i += LU_THREADS) {
                double2 a = A[(size_t)i + (size_t)k * N];
                double v = fabs(a.x) + fabs(a.y);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                double ov = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                red_v[warp] = best;
                red_i[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                double bv = red_v[0];
                int bix = red_i[0];
                for (int w = 1; w < LU_THREADS / 32; ++w)
                    if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bix)) {
                        bv = red_v[w];
                        bix = red_i[w];
                    }
                if (bix >= N) bix = k;
                s_piv[kk] = bix;
                ipiv[k] = bix + 1;
                if (bv == 0.0 && s_info == 0) s_info = k + 1;
            }
            __syncthreads();
            const int p = s_piv[kk];
            if (p != k && tid < nb) {
                const int c = k0 + tid;
                double2 t = A[(size_t)k + (size_t)c * N];
                A[(size_t)k + (size_t)c * N] = A[(size_t)p + (size_t)c * N];
                A[(size_t)p + (size_t)c * N] = t;
            }
            __syncthreads();
            const double2 piv = A[(size_t)k + (size_t)k * N];
            if (piv.x != 0.0 || piv.y != 0.0) {
                const double2 inv = crecip(piv);
                for (int i = k + 1 + tid; i < N; i += LU_THREADS) {
                    double2* q = A + (size_t)i + (size_t)k * N;
                    *q = cmul(*q, inv);
                }
            }
            __syncthreads();
            const int ncol = nb - kk - 1, nrow = N - k - 1;
            for (int idx = tid; idx < ncol * nrow; idx += LU_THREADS) {
                const int i = k + 1 + idx % nrow, j = k + 1 + idx / nrow;
                const double2 l = A[(size_t)i + (size_t)k * N];
                const double2 u = A[(size_t)k + (size_t)j * N];
                double2* q = A + (size_t)i + (size_t)j * N;
                double2 v = *q;
                v.x = fma(-l.x, u.x, v.x);
                v.x = fma(l.y, u.y, v.x);
                v.y = fma(-l.x, u.y, v.y);
                v.y = fma(-l.y, u.x, v.y);
                *q = v;
            }
            __syncthreads();
        }
        // ---- 2. interchanges on every column outside the panel (S) and on H
        const int nS = N - nb;
        const int nH = Bm ? N : 0;
        for (int c = tid; c < nS + nH; c += LU_THREADS) {
            double2* col;
            if (c < nS) {
                const int cc = c < k0 ? c : c + nb;
                col = A + (size_t)cc * N;
            } else {
                col = Bm + (size_t)(c - nS) * N;
            }
            for (int kk = 0; kk < nb; ++kk) {
                const int p = s_piv[kk], k = k0 + kk;
                if (p != k) {
                    double2 t = col[k];
                    col[k] = col[p];
                    col[p] = t;
                }
            }
        }
        // L11 (unit lower) into shared memory
        for (int idx = tid; idx < NB * NB; idx += LU_THREADS) {
            const int i = idx % NB, j = idx / NB;
            sT[idx] = (i < nb && j < nb) ? A[(size_t)(k0 + i) + (size_t)(k0 + j) * N] : make_double2(0.0, 0.0);
        }
        __syncthreads();
        // ---- 3. U12 = L11^{-1} A12 for trailing S columns and all H columns:
        //         one warp per column, lane i holds row k0 + i (NB == warp size)
        const int nTr = N - k0 - nb;
        for (int c = warp; c < nTr + nH; c += LU_THREADS / 32) {
            double2* col = (c < nTr) ? A + (size_t)(k0 + nb + c) * N + k0 : Bm + (size_t)(c - nTr) * N + k0;
            double2 x = lane < nb ? col[lane] : make_double2(0.0, 0.0);
            for (int j = 0; j < nb - 1; ++j) {
                const double xr = __shfl_sync(0xffffffffu, x.x, j);
                const double xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane > j) {
                    const double2 l = sT[j * NB + lane];
                    x.x = fma(-l.x, xr, x.x);
                    x.x = fma(l.y, xi, x.x);
                    x.y = fma(-l.x, xi, x.y);
                    x.y = fma(-l.y, xr, x.y);
                }
            }
            if (lane < nb) col[lane] = x;
        }
        __syncthreads();
        // ---- 4. trailing update
        const int m = N - k0 - nb;
        if (m > 0) {
            const double2* L21 = A + (size_t)(k0 + nb) + (size_t)k0 * N;
            if (nTr > 0)
                cta_gemm_sub(A + (size_t)(k0 + nb) + (size_t)(k0 + nb) * N, N, L21, N,
                             A + (size_t)k0 + (size_t)(k0 + nb) * N, N, m, nTr, nb, sA, sB);
            if (Bm) cta_gemm_sub(Bm + (size_t)(k0 + nb), N, L21, N, Bm + (size_t)k0, N, m, N, nb, sA, sB);
        }
        __syncthreads();
    }

    const int info = s_info;
    if (tid == 0) info_all[sys] = info;
    if (info != 0 || !Bm) return;   // factor only, or no solution for a singular system (as ZGESV)

    // ---- back substitution X = U^{-1} Y
    const int last = ((N - 1) / NB) * NB;
    for (int kb = last; kb >= 0; kb -= NB) {
        const int nb = min(NB, N - kb);
        for (int idx = tid; idx < NB * NB; idx += LU_THREADS) {
            const int i = idx % NB, j = idx / NB;
            sT[idx] = (i < nb && j < nb) ? A[(size_t)(kb + i) + (size_t)(kb + j) * N] : make_double2(0.0, 0.0);
        }
        if (tid < NB) sD[tid] = tid < nb ? crecip(A[(size_t)(kb + tid) + (size_t)(kb + tid) * N]) : make_double2(0.0, 0.0);
        __syncthreads();
        for (int c = warp; c < N; c += LU_THREADS / 32) {
            double2* col = Bm + (size_t)c * N + kb;
            double2 x = lane < nb ? col[lane] : make_double2(0.0, 0.0);
            for (int j = nb - 1; j >= 0; --j) {
                if (lane == j) x = cmul(x, sD[j]);
                const double xr = __shfl_sync(0xffffffffu, x.x, j);
                const double xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane < j) {
                    const double2 u = sT[j * NB + lane];
                    x.x = fma(-u.x, xr, x.x);
                    x.x = fma(u.y, xi, x.x);
                    x.y = fma(-u.x, xi, x.y);
                    x.y = fma(-u.y, xr, x.y);
                }
            }
            if (lane < nb) col[lane] = x;
        }
        __syncthreads();
        if (kb > 0)
            cta_gemm_sub(Bm, N, A + (size_t)kb * N, N, Bm + kb, N, kb, N, nb, sA, sB);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// FP32 factorisation for the mixed-precision form: P S = L U with S read in FP64,
// rounded to FP32 and factorised on the FP32 pipe.  The factors serve as the
// preconditioner of FP64 iterative refinement (the residuals use the FP64 S).
// ---------------------------------------------------------------------------
__device__ inline float2 cmulf(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ void cta_gemm_sub_f(float2* __restrict__ C, int ldc, const float2* __restrict__ A, int lda,
                               const float2* __restrict__ B, int ldb, int m, int n, int k, float2* sA,
                               float2* sB) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int i0 = 0; i0 < m; i0 += TM) {
        for (int idx = tid; idx < TM * NB; idx += LU_THREADS) {
            int ii = idx % TM, kk = idx / TM;
            sA[kk * TM + ii] = (i0 + ii < m && kk < k) ? A[(size_t)(i0 + ii) + (size_t)kk * lda] : make_float2(0.f, 0.f);
        }
        for (int j0 = 0; j0 < n; j0 += TN) {
            for (int idx = tid; idx < NB * TN; idx += LU_THREADS) {
                int kk = idx % NB, jj = idx / NB;
                sB[kk * TN + jj] = (j0 + jj < n && kk < k) ? B[(size_t)kk + (size_t)(j0 + jj) * ldb] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            float2 acc[4][2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) acc[a][c] = make_float2(0.f, 0.f);
            for (int kk = 0; kk < k; ++kk) {
                float2 av[4], bv[2];
#pragma unroll
                for (int a = 0; a < 4; ++a) av[a] = sA[kk * TM + ty + 16 * a];
#pragma unroll
                for (int c = 0; c < 2; ++c) bv[c] = sB[kk * TN + tx + 16 * c];
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        acc[a][c].x = fmaf(av[a].x, bv[c].x, acc[a][c].x);
                        acc[a][c].x = fmaf(-av[a].y, bv[c].y, acc[a][c].x);
                        acc[a][c].y = fmaf(av[a].x, bv[c].y, acc[a][c].y);
                        acc[a][c].y = fmaf(av[a].y, bv[c].x, acc[a][c].y);
                    }
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                int i = i0 + ty + 16 * a;
                if (i >= m) continue;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    int j = j0 + tx + 16 * c;
                    if (j >= n) continue;
                    float2* p = C + (size_t)i + (size_t)j * ldc;
                    float2 v = *p;
                    v.x -= acc[a][c].x;
                    v.y -= acc[a][c].y;
                    *p = v;
                }
            }
            __syncthreads();
        }
    }
}

__global__ void __launch_bounds__(LU_THREADS) k_lu_factor_f32(int N, const double2* __restrict__ Sall,
                                                              float2* __restrict__ LUall, int* __restrict__ ipiv_all,
                                                              int* __restrict__ info_all) {
    extern __shared__ float2 luf_smem[];
    float2* sA = luf_smem;            // TM * NB
    float2* sB = sA + TM * NB;        // NB * TN
    float2* sT = sB + NB * TN;        // NB * NB
    __shared__ float red_v[LU_THREADS / 32];
    __shared__ int red_i[LU_THREADS / 32];
    __shared__ int s_piv[NB];
    __shared__ int s_info;
    const int sys = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const size_t mat = (size_t)N * N;
    const double2* S = Sall + (size_t)sys * mat;
    float2* A = LUall + (size_t)sys * mat;
    int* ipiv = ipiv_all + (size_t)sys * N;
    for (size_t q = tid; q < mat; q += LU_THREADS) A[q] = make_float2((float)S[q].x, (float)S[q].y);
    if (tid == 0) s_info = 0;
    __syncthreads();
    for (int k0 = 0; k0 < N; k0 += NB) {
        const int nb = min(NB, N - k0);
        for (int kk = 0; kk < nb; ++kk) {
            const int k = k0 + kk;
            float best = -1.f;
            int bi = N;
            for (int i = k + tid; i < N; i += LU_THREADS) {
                float2 a = A[(size_t)i + (size_t)k * N];
                float v = fabsf(a.x) + fabsf(a.y);
                if (v > best) {
                    best = v;
                    bi = i;
                }
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                float ov = __shfl_down_sync(0xffffffffu, best, off);
                int oi = __shfl_down_sync(0xffffffffu, bi, off);
                if (ov > best || (ov == best && oi < bi)) {
                    best = ov;
                    bi = oi;
                }
            }
            if (lane == 0) {
                red_v[warp] = best;
                red_i[warp] = bi;
            }
            __syncthreads();
            if (tid == 0) {
                float bv = red_v[0];
                int bix = red_i[0];
                for (int w = 1; w < LU_THREADS / 32; ++w)
                    if (red_v[w] > bv || (red_v[w] == bv && red_i[w] < bix)) {
                        bv = red_v[w];
                        bix = red_i[w];
                    }
                if (bix >= N) bix = k;
                s_piv[kk] = bix;
                ipiv[k] = bix + 1;
                if (bv == 0.f && s_info == 0) s_info = k + 1;
            }
            __syncthreads();
            const int p = s_piv[kk];
            if (p != k && tid < nb) {
                const int c = k0 + tid;
                float2 t = A[(size_t)k + (size_t)c * N];
                A[(size_t)k + (size_t)c * N] = A[(size_t)p + (size_t)c * N];
                A[(size_t)p + (size_t)c * N] = t;
            }
            __syncthreads();
            const float2 piv = A[(size_t)k + (size_t)k * N];
            if (piv.x != 0.f || piv.y != 0.f) {
                const float d = piv.x * piv.x + piv.y * piv.y;
                const float2 inv = make_float2(piv.x / d, -piv.y / d);
                for (int i = k + 1 + tid; i < N; i += LU_THREADS) {
                    float2* q = A + (size_t)i + (size_t)k * N;
                    *q = cmulf(*q, inv);
                }
            }
            __syncthreads();
            const int ncol = nb - kk - 1, nrow = N - k - 1;
            for (int idx = tid; idx < ncol * nrow; idx += LU_THREADS) {
                const int i = k + 1 + idx % nrow, j = k + 1 + idx / nrow;
                const float2 l = A[(size_t)i + (size_t)k * N];
                const float2 u = A[(size_t)k + (size_t)j * N];
                float2* q = A + (size_t)i + (size_t)j * N;
                float2 v = *q;
                v.x = fmaf(-l.x, u.x, v.x);
                v.x = fmaf(l.y, u.y, v.x);
                v.y = fmaf(-l.x, u.y, v.y);
                v.y = fmaf(-l.y, u.x, v.y);
                *q = v;
            }
            __syncthreads();
        }
        const int nS = N - nb;
        for (int c = tid; c < nS; c += LU_THREADS) {
            const int cc = c < k0 ? c : c + nb;
            float2* col = A + (size_t)cc * N;
            for (int kk = 0; kk < nb; ++kk) {
                const int p = s_piv[kk], k = k0 + kk;
                if (p != k) {
                    float2 t = col[k];
                    col[k] = col[p];
                    col[p] = t;
                }
            }
        }
        for (int idx = tid; idx < NB * NB; idx += LU_THREADS) {
            const int i = idx % NB, j = idx / NB;
            sT[idx] = (i < nb && j < nb) ? A[(size_t)(k0 + i) + (size_t)(k0 + j) * N] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        const int nTr = N - k0 - nb;
        for (int c = warp; c < nTr; c += LU_THREADS / 32) {
            float2* col = A + (size_t)(k0 + nb + c) * N + k0;
            float2 x = lane < nb ? col[lane] : make_float2(0.f, 0.f);
            for (int j = 0; j < nb - 1; ++j) {
                const float xr = __shfl_sync(0xffffffffu, x.x, j);
                const float xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane > j) {
                    const float2 l = sT[j * NB + lane];
                    x.x = fmaf(-l.x, xr, x.x);
                    x.x = fmaf(l.y, xi, x.x);
                    x.y = fmaf(-l.x, xi, x.y);
                    x.y = fmaf(-l.y, xr, x.y);
                }
            }
            if (lane < nb) col[lane] = x;
        }
        __syncthreads();
        if (nTr > 0)
            cta_gemm_sub_f(A + (size_t)(k0 + nb) + (size_t)(k0 + nb) * N, N, A + (size_t)(k0 + nb) + (size_t)k0 * N, N,
                           A + (size_t)k0 + (size_t)(k0 + nb) * N, N, nTr, nTr, nb, sA, sB);
        __syncthreads();
    }
    if (tid == 0) info_all[sys] = s_info;
}

wpccc_status launch_factor_f32(int N, int batch, const double2* S, float2* LU, int* ipiv, int* info, cudaStream_t st) {
    if (batch == 0) return WPCCC_OK;
    const int smem = (int)(sizeof(float2) * (TM * NB + NB * TN + NB * NB));
    WPCCC_CUDA(cudaFuncSetAttribute(k_lu_factor_f32, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_lu_factor_f32<<<batch, LU_THREADS, smem, st>>>(N, S, LU, ipiv, info);
    WPCCC_CHECK_LAUNCH("k_lu_factor_f32");
    return WPCCC_OK;
}

size_t solve_smem_bytes() { return sizeof(double2) * (TM * NB + NB * TN + NB * NB + NB); }

// H == nullptr: factorisation only (P S = L U), no right-hand sides.
wpccc_status launch_solve(int N, int batch, double2* S, double2* H, int* ipiv, int* info, cudaStream_t st) {
    if (batch == 0) return WPCCC_OK;
    const int smem = (int)solve_smem_bytes();
    WPCCC_CUDA(cudaFuncSetAttribute(k_lu_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_lu_solve<<<batch, LU_THREADS, smem, st>>>(N, S, H, ipiv, info);
    WPCCC_CHECK_LAUNCH("k_lu_solve");
    return WPCCC_OK;
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_solve(int N, int batch, void* S, void* H, int* ipiv, int* info, int precision_mode,
                                    void* stream) {
    if (N < 1 || N > WPCCC_NMAX) return fail(WPCCC_EINVAL, "wpccc_solve: N out of range 1..WPCCC_NMAX");
    if (batch < 0) return fail(WPCCC_EINVAL, "wpccc_solve: batch < 0");
    if (batch > 0 && (!S || !H || !ipiv || !info)) return fail(WPCCC_EINVAL, "wpccc_solve: null pointer");
    if (precision_mode != 0) return fail(WPCCC_EUNSUPPORTED, "wpccc_solve: only precision_mode 0 (FP64)");
    return launch_solve(N, batch, static_cast<double2*>(S), static_cast<double2*>(H), ipiv, info,
                        static_cast<cudaStream_t>(stream));
}
