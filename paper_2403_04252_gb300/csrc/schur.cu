// Schur-complement factorisation of the two-centre overlap matrix (solve mode WPCCC_SOLVE_SCHUR).
//
// S = [[I, K], [K^+, I]] (Eq. 1) is a Gram matrix, Hermitian positive definite.  Eliminating the target
// block gives the Schur complement C = I - K^+ K (N_P x N_P, Hermitian positive definite), factorised
// by Cholesky, C = L L^+.  Then S k = t is
//   k_P = C^{-1} (t_P - K^+ t_T),   k_T = t_T - K k_P,
// i.e. two matrix-vector products with K and two triangular solves with L per RK4 stage, instead of the
// pivoted LU of the whole S.  Per position: the rank-N_T update K^+ K of the lower triangle (4 N_P^2 N_T
// real flops) and the Cholesky ((4/3) N_P^3), against (8/3) N^3 for the LU of S.
//
// One thread block per system; L overwrites the lower triangle of S's projectile-projectile block
// (the identity block, which the propagation never reads otherwise); K stays in place.  The mixed-
// precision forms take the same factorisation in FP32 into a separate buffer, as the preconditioner of
// their FP64 iterative refinement.
#include <algorithm>

#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int SC_NB = 32;          // Cholesky panel width
constexpr int SC_THREADS = 256;
constexpr int SC_TM = 64, SC_TN = 32;

template <typename R> struct SchurC;
template <> struct SchurC<double> { using type = double2; };
template <> struct SchurC<float> { using type = float2; };

// C[m x n] -= sum_kk A(i, kk) B(kk, j) over the tiles that touch the lower triangle (i >= j) of C, for a
// reduction of kd terms taken SC_NB at a time; A and B are element loaders.
template <typename R, typename LA, typename LB>
__device__ void cta_update_lower(typename SchurC<R>::type* __restrict__ C, int ldc, int m, int kd, LA loadA,
                                 LB loadB, typename SchurC<R>::type* sA, typename SchurC<R>::type* sB) {
    using C2 = typename SchurC<R>::type;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int i0 = 0; i0 < m; i0 += SC_TM) {
        for (int j0 = 0; j0 < m && j0 < i0 + SC_TM; j0 += SC_TN) {
            C2 acc[4][2];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) acc[a][c] = C2{R(0), R(0)};
            for (int k0 = 0; k0 < kd; k0 += SC_NB) {
                for (int idx = tid; idx < SC_TM * SC_NB; idx += SC_THREADS) {
                    const int ii = idx % SC_TM, kk = idx / SC_TM;
                    sA[kk * SC_TM + ii] = (i0 + ii < m && k0 + kk < kd) ? loadA(i0 + ii, k0 + kk) : C2{R(0), R(0)};
                }
                for (int idx = tid; idx < SC_NB * SC_TN; idx += SC_THREADS) {
                    const int kk = idx % SC_NB, jj = idx / SC_NB;
                    sB[kk * SC_TN + jj] = (j0 + jj < m && k0 + kk < kd) ? loadB(k0 + kk, j0 + jj) : C2{R(0), R(0)};
                }
                __syncthreads();
                const int kn = min(SC_NB, kd - k0);
                for (int kk = 0; kk < kn; ++kk) {
                    C2 av[4], bv[2];
#pragma unroll
                    for (int a = 0; a < 4; ++a) av[a] = sA[kk * SC_TM + ty + 16 * a];
#pragma unroll
                    for (int c = 0; c < 2; ++c) bv[c] = sB[kk * SC_TN + tx + 16 * c];
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
                __syncthreads();
            }
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const int i = i0 + ty + 16 * a;
                if (i >= m) continue;
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const int j = j0 + tx + 16 * c;
                    if (j >= m || j > i) continue;
                    C2* p = C + (size_t)i + (size_t)j * ldc;
                    C2 v = *p;
                    v.x -= acc[a][c].x;
                    v.y -= acc[a][c].y;
                    *p = v;
                }
            }
        }
    }
}

// One system per block.  R = double: D is S itself (FP64, in place).  R = float (preconditioner of the
// mixed-precision form): D is a separate FP32 N x N buffer that receives K rounded to FP32 in its
// target-projectile block and the FP32 Cholesky factor in its projectile block; S is only read.
// given = true: D already holds K in FP32 and the trailing matrix I - K^+ K in the projectile block's
// lower triangle (formed on the tensor cores, schur_tc.cu); only the Cholesky factor is computed.
template <typename R>
__global__ void __launch_bounds__(SC_THREADS) k_schur_factor(int N, int N_T, const double2* Sall,
                                                             typename SchurC<R>::type* __restrict__ Dall,
                                                             int* __restrict__ info_all, bool given) {
    using C2 = typename SchurC<R>::type;
    extern __shared__ __align__(16) unsigned char sc_smem_raw[];
    C2* sA = reinterpret_cast<C2*>(sc_smem_raw);   // SC_TM * SC_NB
    C2* sB = sA + SC_TM * SC_NB;                    // SC_NB * SC_TN
    __shared__ int s_info;
    __shared__ R s_d;
    const int sys = blockIdx.x, tid = threadIdx.x;
    const int NP = N - N_T;
    const size_t mat = (size_t)N * N;
    C2* D = Dall + (size_t)sys * mat;
    C2* C = D + N_T + (size_t)N_T * N;           // projectile block, leading dimension N
    const C2* K = D + (size_t)N_T * N;           // K[i][j] = D[i][N_T + j], i < N_T
    if (tid == 0) s_info = 0;
    if (sizeof(R) == 4 && !given) {
        // K to FP32, identity into the lower triangle of the projectile block
        const double2* S = Sall + (size_t)sys * mat;
        for (size_t q = tid; q < (size_t)N_T * NP; q += SC_THREADS) {
            const int i = (int)(q % N_T), j = (int)(q / N_T);
            const double2 a = S[(size_t)i + (size_t)(N_T + j) * N];
            D[(size_t)i + (size_t)(N_T + j) * N] = C2{(R)a.x, (R)a.y};
        }
        for (size_t q = tid; q < (size_t)NP * NP; q += SC_THREADS) {
            const int i = (int)(q % NP), j = (int)(q / NP);
            if (i >= j) C[(size_t)i + (size_t)j * N] = C2{R(i == j ? 1 : 0), R(0)};
        }
        __syncthreads();
    }
    // C = I - K^+ K on the lower triangle (the block holds I already)
    if (!given)
        cta_update_lower<R>(
            C, N, NP, N_T,
            [&](int i, int kk) {   // (K^+)[i][kk] = conj(K[kk][i])
                const C2 a = K[(size_t)kk + (size_t)i * N];
                return C2{a.x, -a.y};
            },
            [&](int kk, int j) { return K[(size_t)kk + (size_t)j * N]; }, sA, sB);
    __syncthreads();
    // blocked right-looking Cholesky of C, lower
    for (int k0 = 0; k0 < NP; k0 += SC_NB) {
        const int nb = min(SC_NB, NP - k0);
        for (int kk = 0; kk < nb; ++kk) {
            const int k = k0 + kk;
            if (tid == 0) {
                R d = C[(size_t)k + (size_t)k * N].x;
                if (!(d > R(0))) {
                    if (s_info == 0) s_info = k + 1;
                    d = R(1);
                }
                s_d = sqrt(d);
                C[(size_t)k + (size_t)k * N] = C2{s_d, R(0)};
            }
            __syncthreads();
            const R inv = R(1) / s_d;
            for (int i = k + 1 + tid; i < NP; i += SC_THREADS) {
                C2* q = C + (size_t)i + (size_t)k * N;
                *q = C2{q->x * inv, q->y * inv};
            }
            __syncthreads();
            // rank-1 update of the rest of the panel: C[i][j] -= C[i][k] conj(C[j][k]), k < j <= i
            const int ncol = k0 + nb - (k + 1), nrow = NP - (k + 1);
            for (int idx = tid; idx < ncol * nrow; idx += SC_THREADS) {
                const int j = k + 1 + idx / nrow, i = k + 1 + idx % nrow;
                if (i < j) continue;
                const C2 l = C[(size_t)i + (size_t)k * N];
                const C2 u = C[(size_t)j + (size_t)k * N];
                C2* q = C + (size_t)i + (size_t)j * N;
                C2 v = *q;
                v.x -= l.x * u.x + l.y * u.y;
                v.y -= l.y * u.x - l.x * u.y;
                *q = v;
            }
            __syncthreads();
        }
        // trailing update C22 -= L21 L21^+
        const int m2 = NP - (k0 + nb);
        if (m2 > 0) {
            C2* C22 = C + (size_t)(k0 + nb) + (size_t)(k0 + nb) * N;
            const C2* L21 = C + (size_t)(k0 + nb) + (size_t)k0 * N;
            cta_update_lower<R>(
                C22, N, m2, nb, [&](int i, int kk) { return L21[(size_t)i + (size_t)kk * N]; },
                [&](int kk, int j) {
                    const C2 a = L21[(size_t)j + (size_t)kk * N];
                    return C2{a.x, -a.y};
                },
                sA, sB);
        }
        __syncthreads();
    }
    if (tid == 0) info_all[sys] = s_info;
}

wpccc_status launch_schur_factor(int N, int N_T, int batch, double2* S, int* info, cudaStream_t st) {
    if (batch == 0) return WPCCC_OK;
    const int smem = (int)(sizeof(double2) * (SC_TM * SC_NB + SC_NB * SC_TN));   // 48 KB: needs the opt-in
    WPCCC_CUDA(cudaFuncSetAttribute(k_schur_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    k_schur_factor<double><<<batch, SC_THREADS, smem, st>>>(N, N_T, S, S, info, false);
    WPCCC_CHECK_LAUNCH("k_schur_factor<double>");
    return WPCCC_OK;
}

wpccc_status launch_schur_factor_f32(int N, int N_T, int batch, const double2* S, float2* D, int* info,
                                     cudaStream_t st) {
    if (batch == 0) return WPCCC_OK;
    const int smem = (int)(sizeof(float2) * (SC_TM * SC_NB + SC_NB * SC_TN));
    k_schur_factor<float><<<batch, SC_THREADS, smem, st>>>(N, N_T, S, D, info, false);
    WPCCC_CHECK_LAUNCH("k_schur_factor<float>");
    return WPCCC_OK;
}

wpccc_status launch_schur_cholesky_f32(int N, int N_T, int batch, float2* D, int* info, cudaStream_t st) {
    if (batch == 0) return WPCCC_OK;
    const int smem = (int)(sizeof(float2) * (SC_TM * SC_NB + SC_NB * SC_TN));
    k_schur_factor<float><<<batch, SC_THREADS, smem, st>>>(N, N_T, nullptr, D, info, true);
    WPCCC_CHECK_LAUNCH("k_schur_factor<float> (Cholesky of the given trailing matrix)");
    return WPCCC_OK;
}

}  // namespace wpccc
