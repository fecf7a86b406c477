// The Schur complement's rank-N_T update on the 5th-generation tensor cores, for the FP32 preconditioner
// of the mixed-precision forms (solve mode WPCCC_SOLVE_SCHUR).
//
// S = [[I, K], [K^+, I]] (Eq. 1).  One step of block elimination (the paper solves S X = H by LU, Sec. II
// and Eq. 4) with the identity block as pivot leaves the trailing matrix C = I - K^+ K, which the
// preconditioner factorises by Cholesky.  This trailing update is the bulk of the factorisation
// (4 N_P^2 N_T real flops for its lower triangle against 4/3 N_P^3 for the Cholesky), and it is a dense
// contraction over the target index, so it runs here as a real GEMM on tcgen05:
//   (K^+ K)_re[m][n] = sum_kappa X[m][kappa] X[n][kappa],   (K^+ K)_im[m][n] = sum_kappa X[m][kappa] Y[n][kappa]
// with kappa = 2 t + (0, 1) over the target states t and, per projectile state m,
//   X[m][2t] = Re K[t][m], X[m][2t+1] = Im K[t][m],   Y[m][2t] = Im K[t][m], Y[m][2t+1] = -Re K[t][m].
// The operands are written by k_schur_slices in the fixed-point slicing of the Eq. 9 contraction
// (ozaki.cuh): per 128-wide window of kappa and per row a power-of-two scale, OZ_FAST_SLICES bf16 slices,
// every level sum (i + j = L <= 3, at most four products over 128 terms) held exactly by an FP32 TMEM
// accumulator, the window's sum drained with its two scales into a double-float running sum.  The B
// operand rows are [X; Y] (2 N_P rows), the A operand rows the first N_P of them.  Only tiles that touch
// the lower triangle are formed.  The Cholesky factor itself stays on the CUDA cores (k_schur_factor
// with the trailing matrix given).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "ozaki.cuh"
#include "tc_ptx.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int SU_SL = OZ_FAST_SLICES;                 // slices per operand
constexpr int SU_M = 128;                             // A rows per CTA (MMA M)
constexpr int SU_N = 64;                              // B rows per CTA (MMA N)
constexpr int SU_K = 32;                              // kappa per chunk: one 64-byte bf16 row
constexpr int SU_WIN = 4;                             // chunks per scaling window (128 kappa)
constexpr int SU_STAGES = 3;                          // TMA ring
constexpr int SU_A_TILE = SU_M * 64;                  // bytes of one slice of the A tile
constexpr int SU_B_TILE = SU_N * 64;                  // bytes of one slice of the B tile
constexpr int SU_STAGE_BYTES = SU_SL * (SU_A_TILE + SU_B_TILE);   // 48 KB, a multiple of 1024
constexpr int SU_EPI_WARPS = 8;                       // two per TMEM lane quadrant, 32 columns each
constexpr int SU_THREADS = (SU_EPI_WARPS + 1) * 32;
constexpr int SU_BUF_COLS = SU_SL * SU_N;             // four level accumulators per buffer
constexpr int SU_TMEM_COLS = 512;                     // two buffers
static_assert(2 * SU_BUF_COLS <= SU_TMEM_COLS, "two buffers of accumulators fit the TMEM allocation");
static_assert(SU_STAGE_BYTES % 1024 == 0, "1024-byte aligned stages");
static_assert(SU_SL == 4, "the epilogue combines four exact levels");

// Scratch layout of one position: slice planes [SU_SL][2 N_P][KP] bf16, then scales [KP / 128][2 N_P] float.
struct SchurTcLayout {
    int NP2, KP, nwin;
    size_t plane_bytes, sc_off, bytes;
};
static SchurTcLayout su_layout(int N, int N_T) {
    SchurTcLayout L;
    L.NP2 = 2 * (N - N_T);
    L.KP = (2 * N_T + 127) / 128 * 128;
    L.nwin = L.KP / 128;
    L.plane_bytes = (size_t)SU_SL * L.NP2 * L.KP * 2;
    L.sc_off = L.plane_bytes;
    L.bytes = (L.sc_off + (size_t)L.nwin * L.NP2 * sizeof(float) + 255) / 256 * 256;
    return L;
}

// Operand slices: warp per (row, window), lanes over kappa = 32 j + lane; also K rounded to FP32 into D's
// target-projectile block (read by the preconditioner's solves).
__global__ void __launch_bounds__(128) k_schur_slices(int N, int N_T, const double2* __restrict__ Sall,
                                                      float2* __restrict__ Dall, unsigned char* __restrict__ scr,
                                                      size_t scr_stride, int KP) {
    const int NP = N - N_T, NP2 = 2 * NP;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = blockIdx.x * 4 + warp, w = blockIdx.y, e = blockIdx.z;
    if (r >= NP2) return;
    const size_t mat = (size_t)N * N;
    const double2* S = Sall + (size_t)e * mat;
    float2* D = Dall + (size_t)e * mat;
    unsigned char* base = scr + (size_t)e * scr_stride;
    __nv_bfloat16* plane = reinterpret_cast<__nv_bfloat16*>(base);
    float* sc = reinterpret_cast<float*>(base + (size_t)SU_SL * NP2 * KP * 2);
    const bool ys = r >= NP;
    const int m = ys ? r - NP : r;
    float2 xv[4];
    float mx = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int kap = w * 128 + 32 * j + lane;
        double val = 0.0;
        if (kap < 2 * N_T) {
            const int t = kap >> 1, part = kap & 1;
            const size_t o = (size_t)t + (size_t)(N_T + m) * N;
            const double2 z = S[o];
            val = !ys ? (part == 0 ? z.x : z.y) : (part == 0 ? z.y : -z.x);
            if (!ys && part == 0) D[o] = make_float2((float)z.x, (float)z.y);
        }
        xv[j] = df_split(val);
        mx = fmaxf(mx, fabsf(xv[j].x));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const int sh = oz_shift(mx);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        __nv_bfloat16 q[SU_SL];
        oz_slices<SU_SL>(xv[j].x, xv[j].y, sh, q);
        const size_t o = (size_t)r * KP + w * 128 + 32 * j + lane;
#pragma unroll
        for (int i = 0; i < SU_SL; ++i) plane[(size_t)i * NP2 * KP + o] = q[i];
    }
    if (lane == 0) sc[(size_t)w * NP2 + r] = ldexpf(1.f, -sh);
}

struct SuMaps {
    CUtensorMap a, b;   // slice planes with box heights SU_M and SU_N
};

struct SuArgs {
    int N, N_T, NP, NP2, KP, nwin;
    int n_tiles;             // (m-tile, B-tile) pairs per position
    const int* tiles;        // [n_tiles][2]: A row start, B row start
    const unsigned char* scr;
    size_t scr_stride, sc_off;
    float2* D;               // [nev][N][N]: the trailing matrix I - K^+ K into the projectile block (lower)
    int* err;
    long wait_limit;
};

// One CTA per (position, A tile of 128 rows, B tile of 64 rows): warp 8 issues the TMA loads and MMAs
// (one thread), warps 0-7 drain the accumulators per window and write the tile's lower triangle.
__global__ void __launch_bounds__(SU_THREADS, 1) k_schur_gemm_tc(const __grid_constant__ SuMaps maps, SuArgs A) {
    extern __shared__ __align__(1024) unsigned char su_smem_raw[];
    unsigned char* sm = su_smem_raw + ((1024 - (smem_u32(su_smem_raw) & 1023)) & 1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + SU_STAGES * SU_STAGE_BYTES);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tile = blockIdx.x, e = blockIdx.y;
    const int a0 = A.tiles[2 * tile], b0 = A.tiles[2 * tile + 1];
    // tfull[3], tempty[3], accf[2], acce[2]
    const uint32_t tfull0 = smem_u32(bars), tempty0 = tfull0 + 8 * SU_STAGES, accf0 = tempty0 + 8 * SU_STAGES,
                   acce0 = accf0 + 16;
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < SU_STAGES; ++s) {
            mbar_init(tfull0 + 8 * s, 1);
            mbar_init(tempty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, SU_EPI_WARPS * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(SU_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    const int nk = A.KP / SU_K;

    if (warp == SU_EPI_WARPS) {
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc_mn(SU_M, SU_N);
            const uint32_t tx = (uint32_t)SU_STAGE_BYTES;
            auto issue_tma = [&](int k) {
                const int s = k % SU_STAGES;
                unsigned char* st = sm + s * SU_STAGE_BYTES;
                const uint32_t bar = tfull0 + 8 * s;
                mbar_arrive_tx(bar, tx);
                for (int sp = 0; sp < SU_SL; ++sp) {
                    tma_load_3d(smem_u32(st + sp * SU_A_TILE), &maps.a, k * SU_K, sp * A.NP2 + a0, e, bar);
                    tma_load_3d(smem_u32(st + SU_SL * SU_A_TILE + sp * SU_B_TILE), &maps.b, k * SU_K,
                                sp * A.NP2 + b0, e, bar);
                }
            };
            int issued = 0;
            for (; issued < SU_STAGES && issued < nk; ++issued) issue_tma(issued);
            bool ok = true;
            int last_mma = -1;
            for (int k = 0; k < nk && ok; ++k) {
                const int s = k % SU_STAGES, w = k / SU_WIN, b = w & 1;
                ok = mbar_wait(tfull0 + 8 * s, (k / SU_STAGES) & 1, abort_flag, A.err, 21, A.wait_limit);
                if (ok && k % SU_WIN == 0 && w >= 2)
                    ok = mbar_wait(acce0 + 8 * b, ((w - 2) >> 1) & 1, abort_flag, A.err, 22, A.wait_limit);
                if (!ok) break;
                tc_fence_after();
                const uint32_t sa = smem_u32(sm + s * SU_STAGE_BYTES);
                const uint32_t sb = sa + SU_SL * SU_A_TILE;
                const uint32_t dbase = tmem + (uint32_t)(b * SU_BUF_COLS);
                const uint64_t da = sw64_desc(sa), db = sw64_desc(sb);
                const uint32_t fresh = k % SU_WIN == 0 ? 0u : 1u;
#pragma unroll
                for (int L = SU_SL - 1; L >= 0; --L) {
                    const uint32_t d = dbase + (uint32_t)(L * SU_N);
#pragma unroll
                    for (int i = 0; i <= L; ++i) {
#pragma unroll
                        for (int kk = 0; kk < SU_K / 16; ++kk) {
                            const bool first = i == 0 && kk == 0;
                            tc_mma(d, da + (uint64_t)((i * SU_A_TILE + kk * 32) >> 4),
                                   db + (uint64_t)(((L - i) * SU_B_TILE + kk * 32) >> 4), idesc, first ? fresh : 1u);
                        }
                    }
                }
                tc_commit(tempty0 + 8 * s);
                last_mma = k;
                if (k % SU_WIN == SU_WIN - 1) tc_commit(accf0 + 8 * b);
                if (k >= 1 && issued < nk) {
                    const int kp = k - 1, sp = kp % SU_STAGES;
                    ok = mbar_wait(tempty0 + 8 * sp, (kp / SU_STAGES) & 1, abort_flag, A.err, 23, A.wait_limit);
                    if (ok) issue_tma(issued++);
                }
            }
            if (!ok) {
                // the copies in flight land before the CTA exits
                for (int k = issued > SU_STAGES ? issued - SU_STAGES : 0; k < issued; ++k) {
                    const int s = k % SU_STAGES;
                    for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(tfull0 + 8 * s, (k / SU_STAGES) & 1); ++it) {
                    }
                }
            }
            // and the MMAs issued complete before the tensor memory is released
            if (last_mma >= 0) {
                const int s = last_mma % SU_STAGES;
                for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(tempty0 + 8 * s, (last_mma / SU_STAGES) & 1); ++it) {
                }
            }
        }
    } else {
        // epilogue: TMEM lanes 32 qd .. 32 qd + 31 (A rows), 32 columns from col0 (B rows)
        const int qd = warp & 3, col0 = (warp >> 2) * 32;
        const int lrow = qd * 32 + lane;
        const int m = a0 + lrow;
        const float* scA = reinterpret_cast<const float*>(A.scr + (size_t)e * A.scr_stride + A.sc_off);
        float hi[32], lo[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
            hi[k] = 0.f;
            lo[k] = 0.f;
        }
        bool ok = true;
        for (int j = 0; j < A.nwin && ok; ++j) {
            const int b = j & 1;
            ok = mbar_wait(accf0 + 8 * b, (j >> 1) & 1, abort_flag, A.err, 24, A.wait_limit);
            if (!ok) break;
            tc_fence_after();
            const float* scw = scA + (size_t)j * A.NP2;
            const float sa = m < A.NP ? scw[m] : 0.f;
            const uint32_t base = tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * SU_BUF_COLS + col0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                float v[SU_SL][8];
#pragma unroll
                for (int lv = 0; lv < SU_SL; ++lv) tmem_ld8(base + lv * SU_N + 8 * q, v[lv]);
                asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int k = 8 * q + u;
                    const int nb = b0 + col0 + k;
                    const float sc = nb < A.NP2 ? sa * scw[nb] : 0.f;
                    // exact: L0 + round(L1), frac(L1) + L2; L3 as it is (see ozaki.cuh)
                    const float l1h = rintf(v[1][u]);
                    const float xa = __fadd_rn(v[0][u], l1h);
                    const float xb = __fadd_rn(__fsub_rn(v[1][u], l1h), v[2][u]);
                    float r1, r2;
                    hi[k] = two_sum(hi[k], xa * sc, r1);
                    hi[k] = two_sum(hi[k], xb * sc, r2);
                    lo[k] = __fadd_rn(lo[k], __fadd_rn(__fadd_rn(r1, r2), v[3][u] * sc));
                }
            }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * b);
        }
        // the lower triangle of the tile: C = I - K^+ K, real part from B rows < N_P, imaginary part from
        // the Y rows (B rows >= N_P)
        if (ok && m < A.NP) {
            float2* D = A.D + (size_t)e * A.N * A.N;
#pragma unroll
            for (int k = 0; k < 32; ++k) {
                const int nb = b0 + col0 + k;
                if (nb >= A.NP2) continue;
                const bool im = nb >= A.NP;
                const int n = im ? nb - A.NP : nb;
                if (n > m) continue;
                const float c = hi[k] + lo[k];
                float* p = reinterpret_cast<float*>(D + (size_t)(A.N_T + m) + (size_t)(A.N_T + n) * A.N);
                if (im) p[1] = -c;
                else p[0] = (m == n ? 1.f : 0.f) - c;
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(SU_TMEM_COLS));
    }
}

// The (A tile, B tile) pairs that touch the lower triangle, kept on the basis for its N_P.
static wpccc_status su_tiles(wpccc_basis_s* B, int NP) {
    if (B->su_tiles && B->su_np == NP) return WPCCC_OK;
    std::vector<int> t;
    for (int a = 0; a < NP; a += SU_M) {
        const int amax = std::min(NP, a + SU_M) - 1;   // last A row of the tile
        for (int half = 0; half < 2; ++half)
            for (int bb = 0; bb <= amax; bb += SU_N) {
                t.push_back(a);
                t.push_back(half * NP + bb);
            }
    }
    if (B->su_tiles) cudaFree(B->su_tiles);
    B->su_tiles = nullptr;
    WPCCC_CUDA(cudaMalloc((void**)&B->su_tiles, t.size() * sizeof(int)));
    WPCCC_CUDA(cudaMemcpy(B->su_tiles, t.data(), t.size() * sizeof(int), cudaMemcpyHostToDevice));
    B->su_np = NP;
    B->su_ntiles = (int)(t.size() / 2);
    return WPCCC_OK;
}

wpccc_status schur_tc_prepare(wpccc_basis_s* B) {
    wpccc_status s = su_tiles(B, B->N - B->N_T);
    if (s == WPCCC_OK) s = ensure_tc_err(B);
    return s;
}

bool schur_tc_applicable(const wpccc_basis_s* B, size_t scratch_per_eval) {
    if (!encode_fn() || B->n_centres != 2) return false;
    const SchurTcLayout L = su_layout(B->N, B->N_T);
    return L.bytes <= scratch_per_eval && B->N - B->N_T >= 1;
}

wpccc_status launch_schur_factor_f32_tc(wpccc_basis_s* B, int nev, const double2* S, float2* D, int* info,
                                        void* scratch, size_t scratch_per_eval, cudaStream_t st) {
    if (nev == 0) return WPCCC_OK;
    const int N = B->N, N_T = B->N_T, NP = N - N_T;
    const SchurTcLayout L = su_layout(N, N_T);
    if (L.bytes > scratch_per_eval) return fail(WPCCC_EINVAL, "tensor-core Schur update: scratch too small");
    if (!B->su_tiles || B->su_np != NP || !B->tc_err)
        return fail(WPCCC_EINVAL, "tensor-core Schur update: schur_tc_prepare was not called");
    const size_t stride = L.bytes;   // per evaluation, a multiple of 256 and at most scratch_per_eval
    // operand slices and K in FP32
    k_schur_slices<<<dim3((L.NP2 + 3) / 4, L.nwin, nev), 128, 0, st>>>(N, N_T, S, D, static_cast<unsigned char*>(scratch),
                                                                       stride, L.KP);
    WPCCC_CHECK_LAUNCH("k_schur_slices");
    SuMaps maps;
    const cuuint64_t dims[3] = {(cuuint64_t)L.KP, (cuuint64_t)SU_SL * L.NP2, (cuuint64_t)nev};
    const cuuint64_t strides[2] = {(cuuint64_t)L.KP * 2, (cuuint64_t)stride};
    const cuuint32_t estr[3] = {1, 1, 1};
    const cuuint32_t boxa[3] = {(cuuint32_t)SU_K, (cuuint32_t)SU_M, 1};
    const cuuint32_t boxb[3] = {(cuuint32_t)SU_K, (cuuint32_t)SU_N, 1};
    if ((uintptr_t)scratch % 16 != 0)
        return fail(WPCCC_EINVAL, "tensor-core Schur update: scratch not 16-byte aligned");
    CUresult r = encode_fn()(&maps.a, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, scratch, dims, strides, boxa, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        r = encode_fn()(&maps.b, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, scratch, dims, strides, boxb, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(WPCCC_ECUDA, "cuTensorMapEncodeTiled failed for the Schur operand planes");
    SuArgs a;
    a.N = N;
    a.N_T = N_T;
    a.NP = NP;
    a.NP2 = L.NP2;
    a.KP = L.KP;
    a.nwin = L.nwin;
    a.n_tiles = B->su_ntiles;
    a.tiles = B->su_tiles;
    a.scr = static_cast<const unsigned char*>(scratch);
    a.scr_stride = stride;
    a.sc_off = L.sc_off;
    a.D = D;
    a.err = B->tc_err;
    a.wait_limit = B->wait_polls;
    const size_t smem = 1024 + (size_t)SU_STAGES * SU_STAGE_BYTES + 8 * (2 * SU_STAGES + 4);
    WPCCC_CUDA(cudaFuncSetAttribute(k_schur_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_schur_gemm_tc<<<dim3(a.n_tiles, nev), SU_THREADS, smem, st>>>(maps, a);
    WPCCC_CHECK_LAUNCH("k_schur_gemm_tc");
    // the Cholesky factor of the trailing matrix on the CUDA cores
    return launch_schur_cholesky_f32(N, N_T, nev, D, info, st);
}

}  // namespace wpccc
