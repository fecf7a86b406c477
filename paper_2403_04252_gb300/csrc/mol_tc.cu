// Eq. 9 contraction on the 5th-generation tensor cores (precision mode 3).
//
// For the target states of one molecular-frame projection q' (a "group") the two-centre integrals are
//   X_K[i][c] = sum_g A_T[i][g] W_{|q_c - q'|}(g) A_P[c][g],   X_Q[i][c] = the same with A_T V_T(r_T),
// i.e. one real contraction over the quadrature nodes g of
//   generated rows   m = (half column c, re/im):   Bw[m][g] = re/im(W_{|q_c - q'|}(g) / r_T) A_P[c][g]
//   table rows       n = (A_T r_T rows of the group, then A_T r_T V_T rows):   from the node tables
// (the weight's factor (eta^2 - tau^2) = 4 r_T r_P / R^2 gives the r_T that cancels the 1/r_T of V_T, so
// both operands stay bounded where the transfer potential diverges);
// into D[m][n] (M = 128 generated rows per CTA, N = twice the group size rounded up to 16).
//
// Precision (error-free slicing after Ozaki, Ogita, Oishi and Rump): within each 32-node chunk every row
// of both operands is written in fixed point, x = s (k0 + k1 2^-8 + k2 2^-16), with s a power of two from
// the row's largest |x| in the chunk and k0..k2 integers in [-128, 128] (exact in bf16).  The main product sum_g k0 k0' is a sum of integers below 2^20, which the tensor
// core's FP32 accumulator holds exactly whatever its rounding; the 2^-8-weighted correction terms
// (k0 k1' + k1 k0' + 2^-8 (k0 k2' + k1 k1' + k2 k0')) go to a second accumulator, whose rounding is
// 2^-8 smaller.  Per chunk the epilogue
// forms s s' (main + 2^-8 corr) (powers of two: exact) and adds it to compensated (Kahan) FP32 sums.
//
// Pipeline per CTA (288 threads): warps 0-7 generate the Bw tiles (64-byte swizzled K-major layout) and
// drain the accumulators; warp 8 issues the TMA loads of the table tiles (cp.async.bulk.tensor, 64-byte
// swizzle) and the tcgen05.mma instructions.  Three shared-memory stages, two TMEM buffers of two
// accumulators, mbarriers between the roles; every wait is bounded and records a timeout in a device flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "tc_ptx.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int TC_M = 128;          // generated rows per CTA (MMA M)
constexpr int TC_K = 32;           // nodes per chunk: one 64-byte bf16 row
constexpr int TC_STAGES = 4;
constexpr int TC_PE_WARPS = 8;     // producer / epilogue warps
constexpr int TC_THREADS = (TC_PE_WARPS + 1) * 32;
constexpr int TC_BN_MAX = 128;     // table rows per box (MMA N at most), so 64 accumulators per thread
// target states per row tile: 2 x 56 = 112 table rows keep this kernel's four stages within 227 KB of
// shared memory (64-state tiles would need 228 KB)
constexpr int TC_TILE_STATES = 56;
constexpr int TC_TMEM_COLS = 512;  // two buffers x (main, correction) accumulators of up to 128 columns
constexpr int TC_A_TILE = TC_M * 64;          // bytes of one slice of the generated tile
constexpr int TC_A_SLICES = 4;                // k0, k1, k2 2^-8, k1 2^-8
constexpr int TC_B_SLICES = 3;                // k0', k1', k2' 2^-8

static __device__ __forceinline__ uint32_t bf16_idesc(int n) { return bf16_idesc_mn(TC_M, n); }

struct TcArgs {
    int G, N_T, n_half, nchunks, BN, n_mtiles, dmax;
    const int* qg_off;     // [groups + 1] first split-table row of each group
    const int* qg_q;       // [groups] q' of each group
    const int* qg_rows;    // [groups][qg_max] target state of each A_T row
    int qg_max;
    const int* half_q;     // [n_half] q of each half column
    const char* node;      // node tables (tensor-core layout) of the launch's evaluations
    size_t node_bytes;     // stride between evaluations
    size_t ap_off_f, w_off_f, sc_off_f;
    int tc_rows;
    double* mol;           // [nev][2][N_T][n_half] complex, written as (re, im) doubles
    int* err;
};

__global__ void __launch_bounds__(TC_THREADS, 1) k_mol_tc(const __grid_constant__ CUtensorMap tmap, TcArgs A) {
    extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
    // 1024-byte aligned base (the swizzle atoms repeat every 512 bytes)
    unsigned char* sm = tc_smem_raw + ((1024 - (smem_u32(tc_smem_raw) & 1023)) & 1023);
    const int b_tile = A.BN * 64;                          // bytes of one slice of the table tile
    // stage: A slices | B slices | A scales (128 floats) | B scales (BN floats)
    const int sc_bytes = (TC_M + A.BN) * 4;
    const int stage_bytes = ((TC_A_SLICES * TC_A_TILE + TC_B_SLICES * b_tile + sc_bytes) + 1023) / 1024 * 1024;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TC_STAGES * stage_bytes);
    // full[s], empty[s], accf[2], acce[2]
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mt = blockIdx.x % A.n_mtiles, grp = blockIdx.x / A.n_mtiles, e = blockIdx.y;
    const int row0 = A.qg_off[grp], ng = (A.qg_off[grp + 1] - row0) / 2;
    const int Ng = (2 * ng + 15) / 16 * 16;               // MMA N of this group
    const int qp = A.qg_q[grp];
    const uint32_t full0 = smem_u32(bars), empty0 = full0 + 8 * TC_STAGES, accf0 = empty0 + 8 * TC_STAGES,
                   acce0 = accf0 + 16;
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(full0 + 8 * s, TC_PE_WARPS * 32 + 1);
            mbar_init(empty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, TC_PE_WARPS * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    const char* nb = A.node + (size_t)e * A.node_bytes;
    const int nk = A.nchunks;

    if (warp == TC_PE_WARPS) {
        // ---- TMA and MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc(Ng);
            const uint32_t tx = (uint32_t)(TC_B_SLICES * b_tile);
            auto issue_tma = [&](int k) {
                const int s = k % TC_STAGES;
                unsigned char* st = sm + s * stage_bytes;
                const uint32_t bar = full0 + 8 * s;
                mbar_arrive_tx(bar, tx);
                for (int sp = 0; sp < TC_B_SLICES; ++sp)
                    tma_load_3d(smem_u32(st + TC_A_SLICES * TC_A_TILE + sp * b_tile), &tmap, k * TC_K,
                                sp * A.tc_rows + row0, e, bar);
            };
            int issued = 0;
            for (; issued < TC_STAGES && issued < nk; ++issued) issue_tma(issued);
            bool ok = true;
            // correction products (A slice, B slice), the smallest first; then the main product
            const int ca[5] = {3, 2, 0, 1, 0}, cb[5] = {1, 0, 2, 0, 1};
            for (int k = 0; k < nk && ok; ++k) {
                const int s = k % TC_STAGES, b = k & 1;
                ok = mbar_wait(full0 + 8 * s, (k / TC_STAGES) & 1, abort_flag, A.err, 1);
                if (ok && k >= 2) ok = mbar_wait(acce0 + 8 * b, ((k - 2) >> 1) & 1, abort_flag, A.err, 2);
                if (!ok) break;
                tc_fence_after();
                unsigned char* st = sm + s * stage_bytes;
                const uint32_t a0 = smem_u32(st), bt0 = smem_u32(st + TC_A_SLICES * TC_A_TILE);
                const uint32_t dmain = tmem + (uint32_t)(b * 256), dcorr = dmain + 128;
                uint32_t acc = 0;
                for (int p = 0; p < 5; ++p)
                    for (int kk = 0; kk < TC_K / 16; ++kk) {
                        tc_mma(dcorr, sw64_desc(a0 + ca[p] * TC_A_TILE + kk * 32),
                               sw64_desc(bt0 + cb[p] * b_tile + kk * 32), idesc, acc);
                        acc = 1;
                    }
                for (int kk = 0; kk < TC_K / 16; ++kk)
                    tc_mma(dmain, sw64_desc(a0 + kk * 32), sw64_desc(bt0 + kk * 32), idesc, kk > 0 ? 1u : 0u);
                tc_commit(empty0 + 8 * s);
                tc_commit(accf0 + 8 * b);
                if (k >= 1 && issued < nk) {
                    // refill the stage of the previous chunk once its MMAs have completed (this chunk's MMAs
                    // are already queued behind them, so the tensor pipe does not wait for the refill)
                    const int kp = k - 1, sp = kp % TC_STAGES;
                    ok = mbar_wait(empty0 + 8 * sp, (kp / TC_STAGES) & 1, abort_flag, A.err, 3);
                    if (ok) issue_tma(issued++);
                }
            }
            if (!ok) {
                // give the copies still in flight time to land before the CTA exits
                for (int k = issued > TC_STAGES ? issued - TC_STAGES : 0; k < issued; ++k) {
                    const int s = k % TC_STAGES;
                    for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(full0 + 8 * s, (k / TC_STAGES) & 1); ++it) {
                    }
                }
            }
        }
    } else {
        // ---- producers of the generated operand (two threads per row, 16 nodes each), and the epilogue
        const int r = tid >> 1, half = tid & 1;
        const int m = mt * TC_M + r, c = m >> 1, ri = m & 1;
        const bool valid = c < A.n_half;
        const float* aP = reinterpret_cast<const float*>(nb) + A.ap_off_f + (size_t)(valid ? c : 0) * A.G;
        int d = 0;
        if (valid) {
            d = A.half_q[c] - qp;
            d = d < 0 ? -d : d;
        }
        const float2* Wk = reinterpret_cast<const float2*>(reinterpret_cast<const float*>(nb) + A.w_off_f) +
                           (size_t)d * A.G;
        const float* scT = reinterpret_cast<const float*>(nb) + A.sc_off_f;   // [chunk][tc_rows]
        // epilogue: this thread's accumulator lane and half of the columns
        const int quarter = warp & 3, chalf = warp >> 2;
        const int lrow = quarter * 32 + lane;
        const int ncol = Ng / 2, n8 = ncol / 8, col0 = chalf * ncol;
        float tot[TC_BN_MAX / 2], cmp[TC_BN_MAX / 2];
#pragma unroll
        for (int k = 0; k < TC_BN_MAX / 2; ++k) {
            tot[k] = 0.f;
            cmp[k] = 0.f;
        }
        bool ok = true;
        auto drain = [&](int j) {
            const int b = j & 1;
            ok = ok && mbar_wait(accf0 + 8 * b, (j >> 1) & 1, abort_flag, A.err, 4);
            if (!ok) return;
            tc_fence_after();
            const float* scl = reinterpret_cast<const float*>(sm + (j % TC_STAGES) * stage_bytes +
                                                              TC_A_SLICES * TC_A_TILE + TC_B_SLICES * b_tile);
            const float sa = scl[lrow];
            const uint32_t base = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * 256 + col0);
            // eight-column groups: main and correction loads, one wait, then the sums
#pragma unroll
            for (int q = 0; q < TC_BN_MAX / 16; ++q)
                if (q < n8) {
                    float vm[8], vc[8];
                    tmem_ld8(base + 8 * q, vm);
                    tmem_ld8(base + 128 + 8 * q, vc);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = 8 * q + u;
                        const float x = fmaf(vc[u], 1.f / 256.f, vm[u]) * (sa * scl[TC_M + col0 + k]);
                        const float y = __fsub_rn(x, cmp[k]);
                        const float t = __fadd_rn(tot[k], y);
                        cmp[k] = __fsub_rn(__fsub_rn(t, tot[k]), y);
                        tot[k] = t;
                    }
                }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * b);
        };
        for (int k = 0; k < nk && ok; ++k) {
            const int s = k % TC_STAGES;
            if (k >= TC_STAGES) ok = mbar_wait(empty0 + 8 * s, ((k - TC_STAGES) / TC_STAGES) & 1, abort_flag, A.err, 5);
            if (!ok) break;
            unsigned char* at = sm + s * stage_bytes;
            float* scl = reinterpret_cast<float*>(at + TC_A_SLICES * TC_A_TILE + TC_B_SLICES * b_tile);
            const int g0 = k * TC_K + half * 16;
            float x[16];
            float mx = 0.f;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int g = g0 + j;
                x[j] = 0.f;
                if (valid && g < A.G) {
                    const float2 w = Wk[g];
                    x[j] = (ri ? w.y : w.x) * aP[g];
                }
                mx = fmaxf(mx, fabsf(x[j]));
            }
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
            int E = 0;
            if (mx > 0.f) frexpf(mx, &E);
            const int sh = mx > 0.f ? 7 - E : 0;
            if (half == 0) scl[r] = ldexpf(1.f, -sh);
            // the table rows' scales of this chunk
            if (tid < A.BN) {
                const int row = row0 + tid;
                scl[TC_M + tid] = row < A.tc_rows ? scT[(size_t)k * A.tc_rows + row] : 0.f;
            }
            uint32_t w4[TC_A_SLICES][8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                __nv_bfloat16 q[TC_A_SLICES][2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float xs = ldexpf(x[j + h], sh);
                    const float k0 = rintf(xs);
                    const float r1 = (xs - k0) * 256.f;
                    const float k1 = rintf(r1);
                    const float k2 = rintf((r1 - k1) * 256.f);
                    q[0][h] = __float2bfloat16_rn(k0);
                    q[1][h] = __float2bfloat16_rn(k1);
                    q[2][h] = __float2bfloat16_rn(k2 * (1.f / 256.f));
                    q[3][h] = __float2bfloat16_rn(k1 * (1.f / 256.f));
                }
#pragma unroll
                for (int sp = 0; sp < TC_A_SLICES; ++sp) w4[sp][j >> 1] = bf16x2(q[sp][0], q[sp][1]);
            }
            // row r of each slice tile: 64 bytes, 16-byte chunk qq at (qq ^ ((r >> 1) & 3))
#pragma unroll
            for (int sp = 0; sp < TC_A_SLICES; ++sp)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int qq = half * 2 + h;
                    *reinterpret_cast<uint4*>(at + sp * TC_A_TILE + r * 64 + ((qq ^ ((r >> 1) & 3)) << 4)) =
                        make_uint4(w4[sp][4 * h], w4[sp][4 * h + 1], w4[sp][4 * h + 2], w4[sp][4 * h + 3]);
                }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(full0 + 8 * s);
            if (k >= 1) drain(k - 1);
        }
        if (ok) drain(nk - 1);
        // results: column n of D is A_T row n of the group (overlap K) or, from ng on, its A_T V_T row (Q)
        const int mo = mt * TC_M + lrow, co = mo >> 1, rio = mo & 1;
        if (ok && co < A.n_half) {
            const size_t plane = (size_t)A.N_T * A.n_half;
            double* out = A.mol + (size_t)e * 2 * plane * 2;
#pragma unroll
            for (int k = 0; k < TC_BN_MAX / 2; ++k) {
                if (k >= ncol) continue;
                const int n = col0 + k;
                if (n >= 2 * ng) continue;
                const int x = n < ng ? 0 : 1;
                const int i = A.qg_rows[grp * A.qg_max + (n < ng ? n : n - ng)];
                out[((size_t)x * plane + (size_t)i * A.n_half + co) * 2 + rio] = (double)tot[k] - (double)cmp[k];
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// Row tiles of the tensor-core layout: the target states grouped by their molecular-frame q', each group
// cut into tiles of at most 56 states (near-equal sizes).  A tile of n states owns 2 n consecutive rows of
// the split tables: its A_T rows, then its A_T V_T rows.  Enables the layout on the basis.
wpccc_status tc_prepare(wpccc_basis_s* B) {
    if (B->tc_layout) return WPCCC_OK;
    if (B->n_centres != 2) return fail(WPCCC_EUNSUPPORTED, "the tensor-core contraction needs a two-centre basis");
    if (!encode_fn()) return fail(WPCCC_EUNSUPPORTED, "tensor-core contraction: cuTensorMapEncodeTiled unavailable");
    if (B->G % 32 != 0) return fail(WPCCC_EUNSUPPORTED, "tensor-core contraction: the node count must be a multiple of 32");
    const int L = B->T.lmax;
    std::vector<std::vector<int>> groups(2 * L + 1);
    for (int i = 0; i < B->N_T; ++i) groups[B->T.h_st_m[i] + L].push_back(i);
    std::vector<std::vector<int>> tiles;
    std::vector<int> tq;
    for (int gq = 0; gq < 2 * L + 1; ++gq) {
        const int n = (int)groups[gq].size();
        if (n == 0) continue;
        const int nt = (n + TC_TILE_STATES - 1) / TC_TILE_STATES;
        for (int t = 0; t < nt; ++t) {
            const int a = (int)((long)n * t / nt), b = (int)((long)n * (t + 1) / nt);
            tiles.emplace_back(groups[gq].begin() + a, groups[gq].begin() + b);
            tq.push_back(gq - L);
        }
    }
    const int ntl = (int)tiles.size();
    int qmax = 0;
    for (auto& t : tiles) qmax = std::max<int>(qmax, (int)t.size());
    std::vector<int> off(ntl + 1, 0), rows((size_t)ntl * qmax, 0), trow(2 * (size_t)B->N_T);
    for (int t = 0; t < ntl; ++t) {
        off[t + 1] = off[t] + 2 * (int)tiles[t].size();
        for (size_t n = 0; n < tiles[t].size(); ++n) {
            const int i = tiles[t][n];
            rows[(size_t)t * qmax + n] = i;
            trow[i] = off[t] + (int)n;
            trow[B->N_T + i] = (int)tiles[t].size();
        }
    }
    auto up = [&](int** dst, const std::vector<int>& v) -> wpccc_status {
        WPCCC_CUDA(cudaMalloc((void**)dst, v.size() * sizeof(int)));
        WPCCC_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice));
        return WPCCC_OK;
    };
    std::vector<int> qg(ntl + 1 + ntl);
    std::copy(off.begin(), off.end(), qg.begin());
    std::copy(tq.begin(), tq.end(), qg.begin() + ntl + 1);
    std::vector<int> halfq(B->n_half);
    {
        std::vector<int> hs(B->n_half);
        WPCCC_CUDA(cudaMemcpy(hs.data(), B->half_state, B->n_half * sizeof(int), cudaMemcpyDeviceToHost));
        for (int h = 0; h < B->n_half; ++h) halfq[h] = B->P.h_st_m[hs[h]];
    }
    wpccc_status s;
    if ((s = up(&B->tc_row, trow)) != WPCCC_OK) return s;
    if ((s = up(&B->qg_off, qg)) != WPCCC_OK) return s;
    if ((s = up(&B->qg_rows, rows)) != WPCCC_OK) return s;
    if ((s = up(&B->tc_halfq, halfq)) != WPCCC_OK) return s;
    WPCCC_CUDA(cudaMalloc((void**)&B->tc_err, sizeof(int)));
    WPCCC_CUDA(cudaMemset(B->tc_err, 0, sizeof(int)));
    B->n_qgroups = ntl;
    B->qg_max = qmax;
    B->tc_layout = true;
    return WPCCC_OK;
}

wpccc_status launch_mol_tc(wpccc_basis_s* B, int nev, const void* node, double2* mol, int* err, cudaStream_t st) {
    if (!B->tc_layout) return fail(WPCCC_EINVAL, "tensor-core layout not prepared");
    const ElemScratch L = elem_scratch_layout(B);
    const size_t node_bytes = L.node_doubles * sizeof(double);
    const int BN = (2 * B->qg_max + 15) / 16 * 16;
    // split tables as one 3-D bf16 tensor: x = node (G), y = split-table row (3 x 2 N_T), z = evaluation
    CUtensorMap map;
    const cuuint64_t dims[3] = {(cuuint64_t)B->G, (cuuint64_t)TC_B_SLICES * L.tc_rows, (cuuint64_t)nev};
    const cuuint64_t strides[2] = {(cuuint64_t)B->G * 2, (cuuint64_t)node_bytes};
    const cuuint32_t box[3] = {(cuuint32_t)TC_K, (cuuint32_t)BN, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = encode_fn()(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(node), dims, strides, box,
                             estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(WPCCC_ECUDA, "cuTensorMapEncodeTiled failed for the split tables");
    TcArgs a;
    a.G = B->G;
    a.N_T = B->N_T;
    a.n_half = B->n_half;
    a.nchunks = (B->G + TC_K - 1) / TC_K;
    a.BN = BN;
    a.n_mtiles = (2 * B->n_half + TC_M - 1) / TC_M;
    a.dmax = B->dmax;
    a.qg_off = B->qg_off;
    a.qg_q = B->qg_off + B->n_qgroups + 1;
    a.qg_rows = B->qg_rows;
    a.qg_max = B->qg_max;
    a.half_q = B->tc_halfq;
    a.node = static_cast<const char*>(node);
    a.node_bytes = node_bytes;
    a.ap_off_f = L.tc_ap_off;
    a.w_off_f = L.tc_w_off;
    a.sc_off_f = L.tc_sc_off;
    a.tc_rows = L.tc_rows;
    a.mol = reinterpret_cast<double*>(mol);
    a.err = err;
    const int stage_bytes =
        ((TC_A_SLICES * TC_A_TILE + TC_B_SLICES * BN * 64 + (TC_M + BN) * 4) + 1023) / 1024 * 1024;
    const size_t smem = 1024 + (size_t)TC_STAGES * stage_bytes + 8 * (2 * TC_STAGES + 4);
    WPCCC_CUDA(cudaFuncSetAttribute(k_mol_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_mol_tc<<<dim3(a.n_mtiles * B->n_qgroups, nev), TC_THREADS, smem, st>>>(map, a);
    WPCCC_CHECK_LAUNCH("k_mol_tc");
    return WPCCC_OK;
}

}  // namespace wpccc
