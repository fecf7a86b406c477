// Eq. 9 contraction on the 5th-generation tensor cores: to FP64 accuracy with seven slices per operand
// (precision modes 4 and 5), and with four (precision mode 3, the reduced-precision form).
//
// The two-centre integrals of one row tile (target states of one molecular-frame projection q') are
//   X_K[i][c] = sum_g (A_T r_T)[i][g] Bw[c][g],   X_Q[i][c] = sum_g (A_T r_T V_T)[i][g] Bw[c][g],
//   Bw[(c, re/im)][g] = re/im(W_{|q_c - q'|}(g) / r_T(g)) A_P[c][g],
// one real contraction over the quadrature nodes g of
//   table rows      m (M = 128: the tile's A_T r_T rows, then its A_T r_T V_T rows), from the node tables
//   generated rows  n (N = 48: 24 half columns x re/im), formed here from double-float W and A_P
// into D[m][n].
//
// Precision (error-free slicing after Ozaki, Ogita, Oishi and Rump; see ozaki.cuh): per window of four
// 32-node chunks (128 nodes) both operands are written in fixed point with SL = 7 bf16 slices,
// a_g = s_m sum_i alpha_i and b_g = s_n sum_j beta_j with alpha_i, beta_j integers times 2^(-8 i),
// 2^(-8 j) and s_m, s_n powers of two per row and window.  The products with i + j = L form level L
// (weight 2^(-8 L)); levels 0-3 go to four accumulators that hold their window sums exactly (integers
// times 2^(-8 L) below 2^24 units: at most four products of |k| <= 129 over 128 nodes), levels 4-6 to a
// fifth, whose FP32 rounding over its 144 MMAs stays near 2^-48 of the window's largest term; levels
// >= 7 are dropped (below 2^-53).  Per window the epilogue forms s_m s_n (L0 + L1 + L2 + L3 + T) with
// the exact parts folded into double-float running sums (two TwoSums), so the result carries about
// 2^-46 of the largest term.  With SL = 4 (levels 0-3, ten products, four exact accumulators, no tail) each
// operand keeps 31 bits below its row's window maximum, and a window's sum errs by up to about 2^-28 of its
// largest term, without the truncation bias of the tensor core's FP32 accumulation.
//
// Pipeline per CTA (416 threads): warps 0-11 generate the Bw tiles (64-byte swizzled K-major rows) and
// drain the accumulators; warp 12 issues the TMA loads of the table tiles (cp.async.bulk.tensor, 64-byte
// swizzle) and the tcgen05.mma instructions.  Three table tiles and two generated tiles in flight in
// shared memory, a ring of scale slots (one per window), two TMEM buffers of five accumulators (one per
// window), mbarriers between the roles; every wait is bounded and records a timeout in a device flag.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "ozaki.cuh"
#include "tc_ptx.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int T6_M = 128;                              // table rows per CTA (MMA M)
constexpr int T6_K = 32;                               // nodes per chunk: one 64-byte bf16 row
constexpr int T6_WIN = 4;                              // chunks per scaling window (128 nodes)
// Per slice count: accumulators (SL = 7: levels 0, 1, 2, 3 exact and >= 4; SL = 4: levels 0-3, all exact)
// and generated rows per CTA (MMA N), two buffers of accumulators within the 512 TMEM columns
// (2 x 5 x 48 = 480, 2 x 4 x 48 = 384); eight producer threads per generated row.
template <int SL> struct Tc64Cfg {
    static constexpr int ACC = SL == 7 ? 5 : SL;
    static constexpr int N = 48;
    static constexpr int PE_WARPS = N / 4;                       // producer / epilogue warps
    static constexpr int THREADS = (PE_WARPS + 1) * 32;
    static constexpr int BUF_COLS = ACC * N;                    // column offset of the second buffer
    static constexpr int B_TILE = N * 64;                       // bytes of one slice of the generated tile
    static constexpr int TSTAGE_BYTES = SL * T6_M * 64;         // a multiple of 1024
    static constexpr int GSTAGE_BYTES = SL * N * 64;            // a multiple of 1024
    static constexpr int SC_FLOATS = T6_M + N;                  // per scale slot: table rows, generated rows
    static constexpr int COLS_PER_WARP = N / (PE_WARPS / 4);    // 16 columns per epilogue warp
    static_assert(PE_WARPS * 32 == N * 8, "eight producer threads (4 nodes each) per generated row");
    static_assert(2 * BUF_COLS <= 512, "two buffers of accumulators fit the TMEM allocation");
    static_assert(TSTAGE_BYTES % 1024 == 0 && GSTAGE_BYTES % 1024 == 0, "1024-byte aligned stages");
};
constexpr int T6_TSTAGES = 3;                          // table tiles in flight (TMA ring)
constexpr int T6_GSTAGES = 2;                          // generated tiles (producer ring)
constexpr int T6_SC_SLOTS = 2;                         // scale ring, one slot per window (see the drain)
constexpr int T6_TMEM_COLS = 512;
constexpr int T6_A_TILE = T6_M * 64;                   // bytes of one slice of the table tile
constexpr int T6_BOXES = T6_M / 32;                    // table box heights 32, 64, 96, 128 rows

template <int SL>
static size_t tc64_smem_bytes() {
    using CF = Tc64Cfg<SL>;
    return 1024 + (size_t)T6_TSTAGES * CF::TSTAGE_BYTES + (size_t)T6_GSTAGES * CF::GSTAGE_BYTES +
           sizeof(float) * T6_SC_SLOTS * CF::SC_FLOATS + 8 * (2 * T6_TSTAGES + 2 * T6_GSTAGES + 4);
}

// Tensor maps of the slice planes with box heights 32, 64, 96 and 128 rows: a row tile loads only the
// 32-row multiple that covers its rows (rows past its end are loaded from the next tile, or left stale,
// and only feed accumulator lanes that are never read).
struct Tc64Maps {
    CUtensorMap m[T6_BOXES];
};

struct Tc64Args {
    int G, N_T, n_half, nchunks, n_ntiles, tc_rows, qg_max;
    const int* qg_off;     // [tiles + 1] first split-table row of each row tile
    const int* qg_q;       // [tiles] q' of each row tile
    const int* qg_rows;    // [tiles][qg_max] target state of each A_T row of a tile
    const int* half_q;     // [n_half] q of each half column
    const char* node;      // node tables (FP64-accurate tensor-core layout) of the launch's evaluations
    size_t node_bytes;     // stride between evaluations
    size_t sc_off_f, ap_off_f, w_off_f;
    double* mol;           // [nev][2][N_T][n_half] complex, written as (re, im) doubles
    int* err;
    long wait_limit;       // polls of an mbarrier wait before it gives up
};

template <int SL>
__global__ void __launch_bounds__(Tc64Cfg<SL>::THREADS, 1) k_mol_tc64(const __grid_constant__ Tc64Maps maps, Tc64Args A) {
    using CF = Tc64Cfg<SL>;
    constexpr int T6_ACC = CF::ACC;
    constexpr int T6_N = CF::N;
    constexpr int T6_PE_WARPS = CF::PE_WARPS;
    constexpr int T6_BUF_COLS = CF::BUF_COLS;
    constexpr int T6_B_TILE = CF::B_TILE;
    constexpr int T6_TSTAGE_BYTES = CF::TSTAGE_BYTES;
    constexpr int T6_GSTAGE_BYTES = CF::GSTAGE_BYTES;
    constexpr int T6_SC_FLOATS = CF::SC_FLOATS;
    constexpr int T6_COLS_PER_WARP = CF::COLS_PER_WARP;
    extern __shared__ __align__(1024) unsigned char t6_smem_raw[];
    unsigned char* sm = t6_smem_raw + ((1024 - (smem_u32(t6_smem_raw) & 1023)) & 1023);
    unsigned char* gsm = sm + T6_TSTAGES * T6_TSTAGE_BYTES;                        // generated tiles
    float* ring = reinterpret_cast<float*>(gsm + T6_GSTAGES * T6_GSTAGE_BYTES);  // [slot][T6_SC_FLOATS]
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + T6_SC_SLOTS * T6_SC_FLOATS);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntile = blockIdx.x % A.n_ntiles, tile = blockIdx.x / A.n_ntiles, e = blockIdx.y;
    const int row0 = A.qg_off[tile], ns = (A.qg_off[tile + 1] - row0) / 2;   // states of the row tile
    const int qp = A.qg_q[tile];
    const int box = (2 * ns + 31) / 32;                  // table box height of this tile, in 32-row units
    // tfull[3] (TMA), tempty[3], gfull[2] (producers), gempty[2], accf[2], acce[2]
    const uint32_t tfull0 = smem_u32(bars), tempty0 = tfull0 + 8 * T6_TSTAGES, gfull0 = tempty0 + 8 * T6_TSTAGES,
                   gempty0 = gfull0 + 8 * T6_GSTAGES, accf0 = gempty0 + 8 * T6_GSTAGES, acce0 = accf0 + 16;
    if (tid == 0) {
        s_abort = 0;
        for (int s = 0; s < T6_TSTAGES; ++s) {
            mbar_init(tfull0 + 8 * s, 1);
            mbar_init(tempty0 + 8 * s, 1);
        }
        for (int s = 0; s < T6_GSTAGES; ++s) {
            mbar_init(gfull0 + 8 * s, T6_PE_WARPS * 32);
            mbar_init(gempty0 + 8 * s, 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf0 + 8 * b, 1);
            mbar_init(acce0 + 8 * b, T6_PE_WARPS * 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&s_tmem)),
                     "r"(T6_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
        tc_fence_before();
    }
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = s_tmem;
    volatile int* abort_flag = &s_abort;
    const char* nb = A.node + (size_t)e * A.node_bytes;
    const int nk = A.nchunks;

    if (warp == T6_PE_WARPS) {
        // ---- TMA and MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc_mn(T6_M, T6_N);
            const uint32_t tx = (uint32_t)(SL * box * 32 * 64);
            const CUtensorMap* tmap = &maps.m[box - 1];
            auto issue_tma = [&](int k) {
                const int s = k % T6_TSTAGES;
                unsigned char* st = sm + s * T6_TSTAGE_BYTES;
                const uint32_t bar = tfull0 + 8 * s;
                mbar_arrive_tx(bar, tx);
                for (int sp = 0; sp < SL; ++sp)
                    tma_load_3d(smem_u32(st + sp * T6_A_TILE), tmap, k * T6_K, sp * A.tc_rows + row0, e, bar);
            };
            int issued = 0;
            for (; issued < T6_TSTAGES && issued < nk; ++issued) issue_tma(issued);
            bool ok = true;
            int last_mma = -1;   // the last chunk whose MMAs were issued (their completion commits to tempty)
            for (int k = 0; k < nk && ok; ++k) {
                const int s = k % T6_TSTAGES, s2 = k % T6_GSTAGES, w = k / T6_WIN, b = w & 1;
                ok = mbar_wait(tfull0 + 8 * s, (k / T6_TSTAGES) & 1, abort_flag, A.err, 11, A.wait_limit);
                if (ok) ok = mbar_wait(gfull0 + 8 * s2, (k / T6_GSTAGES) & 1, abort_flag, A.err, 16, A.wait_limit);
                if (ok && k % T6_WIN == 0 && w >= 2) ok = mbar_wait(acce0 + 8 * b, ((w - 2) >> 1) & 1, abort_flag, A.err, 12, A.wait_limit);
                if (!ok) break;
                tc_fence_after();
                const uint32_t a0 = smem_u32(sm + s * T6_TSTAGE_BYTES), b0 = smem_u32(gsm + s2 * T6_GSTAGE_BYTES);
                const uint32_t dbase = tmem + (uint32_t)(b * T6_BUF_COLS);
                // levels from the smallest up; in a window's first chunk the first product into each
                // accumulator overwrites it.  Fully unrolled: the descriptors of the slices are the base
                // descriptors plus compile-time offsets (16-byte units; no carry out of the address field)
                const uint64_t da = sw64_desc(a0), db = sw64_desc(b0);
                const uint32_t fresh = k % T6_WIN == 0 ? 0u : 1u;
#pragma unroll
                for (int L = SL - 1; L >= 0; --L) {
                    const int lv = L < T6_ACC - 1 ? L : T6_ACC - 1;
                    const uint32_t d = dbase + (uint32_t)(lv * T6_N);
#pragma unroll
                    for (int i = 0; i <= L; ++i) {
#pragma unroll
                        for (int kk = 0; kk < T6_K / 16; ++kk) {
                            const bool first = (L == SL - 1 || L < T6_ACC - 1) && i == 0 && kk == 0;
                            tc_mma(d, da + (uint64_t)((i * T6_A_TILE + kk * 32) >> 4),
                                   db + (uint64_t)(((L - i) * T6_B_TILE + kk * 32) >> 4), idesc, first ? fresh : 1u);
                        }
                    }
                }
                tc_commit(tempty0 + 8 * s);
                tc_commit(gempty0 + 8 * s2);
                last_mma = k;
                if (k % T6_WIN == T6_WIN - 1) tc_commit(accf0 + 8 * b);
                if (k >= 1 && issued < nk) {
                    // refill the table slot of the previous chunk (for chunk k + 2) once its MMAs have completed
                    const int kp = k - 1, sp = kp % T6_TSTAGES;
                    ok = mbar_wait(tempty0 + 8 * sp, (kp / T6_TSTAGES) & 1, abort_flag, A.err, 13, A.wait_limit);
                    if (ok) issue_tma(issued++);
                }
            }
            if (!ok) {
                // give the copies still in flight time to land before the CTA exits
                for (int k = issued > T6_TSTAGES ? issued - T6_TSTAGES : 0; k < issued; ++k) {
                    const int s = k % T6_TSTAGES;
                    for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(tfull0 + 8 * s, (k / T6_TSTAGES) & 1); ++it) {
                    }
                }
            }
            // the MMAs issued complete before the tensor memory is released (they finish in order: the last
            // chunk's commit covers them all); on the normal path the epilogue has waited for them already,
            // on a give-up path nobody else does
            if (last_mma >= 0) {
                const int s = last_mma % T6_TSTAGES;
                for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(tempty0 + 8 * s, (last_mma / T6_TSTAGES) & 1); ++it) {
                }
            }
        }
    } else {
        // ---- producers of the generated operand (eight threads per row, four nodes each), and the epilogue
        const int n = tid >> 3, part = tid & 7;
        const int gr = ntile * T6_N + n, c = gr >> 1, ri = gr & 1;
        const bool valid = c < A.n_half;
        int d = 0;
        if (valid) {
            d = A.half_q[c] - qp;
            d = d < 0 ? -d : d;
        }
        const float* nbf = reinterpret_cast<const float*>(nb);
        const float2* ap = reinterpret_cast<const float2*>(nbf + A.ap_off_f) + (size_t)(valid ? c : 0) * A.G;
        const float2* wd = reinterpret_cast<const float2*>(nbf + A.w_off_f) + ((size_t)d * 2 + ri) * A.G;
        const float* scT = nbf + A.sc_off_f;   // [chunk][tc_rows]
        // epilogue: accumulator lanes 32 qd .. 32 qd + 31 (table rows), 16 columns from col0
        const int qd = warp & 3, col0 = (warp >> 2) * T6_COLS_PER_WARP;
        const int lrow = qd * 32 + lane;
        const bool live = qd * 32 < 2 * ns;    // warps whose rows all lie past the tile skip the arithmetic
        float hi[T6_COLS_PER_WARP], lo[T6_COLS_PER_WARP];
#pragma unroll
        for (int k = 0; k < T6_COLS_PER_WARP; ++k) {
            hi[k] = 0.f;
            lo[k] = 0.f;
        }
        bool ok = true;
        // drain of window j: its accumulators with the window's scales
        auto drain = [&](int j) {
            const int b = j & 1;
            ok = ok && mbar_wait(accf0 + 8 * b, (j >> 1) & 1, abort_flag, A.err, 14, A.wait_limit);
            if (!ok) return;
            tc_fence_after();
            if (live) {
                const float* scl = ring + (j % T6_SC_SLOTS) * T6_SC_FLOATS;
                const float sa = scl[lrow];
                const uint32_t base =
                    tmem + ((uint32_t)(qd * 32) << 16) + (uint32_t)(b * T6_BUF_COLS + col0);
#pragma unroll
                for (int q = 0; q < T6_COLS_PER_WARP / 8; ++q) {
                    float v[T6_ACC][8];
#pragma unroll
                    for (int lv = 0; lv < T6_ACC; ++lv) tmem_ld8(base + lv * T6_N + 8 * q, v[lv]);
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int k = 8 * q + u;
                        const float sc = sa * scl[T6_M + col0 + k];
                        // exact: L0 + round(L1) (integers below 2^22), frac(L1) + L2 (multiples of
                        // 2^-16 below 2^7); rounded: L3 + T (below 1, its rounding under 2^-24)
                        const float l1h = rintf(v[1][u]);
                        const float xa = __fadd_rn(v[0][u], l1h);
                        const float xb = __fadd_rn(__fsub_rn(v[1][u], l1h), v[2][u]);
                        const float xc = T6_ACC == 5 ? __fadd_rn(v[3][u], v[T6_ACC - 1][u])
                                         : T6_ACC == 4 ? v[T6_ACC - 1][u] : 0.f;
                        float r1, r2;
                        hi[k] = two_sum(hi[k], xa * sc, r1);
                        hi[k] = two_sum(hi[k], xb * sc, r2);
                        lo[k] = __fadd_rn(lo[k], __fadd_rn(__fadd_rn(r1, r2), xc * sc));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * b);
        };
        const int nwin = nk / T6_WIN;
        const int trow = row0 + tid;
        for (int w = 0; w < nwin && ok; ++w) {
            // this thread's 16 generated values of the window (four per chunk), their row maximum over the
            // window's 128 nodes (the row's eight threads), and the window's scales
            float2 xw[T6_WIN * 4];
            float mx = 0.f;
#pragma unroll
            for (int cc = 0; cc < T6_WIN; ++cc) {
                const int g0 = (w * T6_WIN + cc) * T6_K + part * 4;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 wq = valid ? reinterpret_cast<const float4*>(wd + g0)[h] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 aq = valid ? reinterpret_cast<const float4*>(ap + g0)[h] : make_float4(0.f, 0.f, 0.f, 0.f);
                    xw[4 * cc + 2 * h] = df_mul(make_float2(wq.x, wq.y), make_float2(aq.x, aq.y));
                    xw[4 * cc + 2 * h + 1] = df_mul(make_float2(wq.z, wq.w), make_float2(aq.z, aq.w));
                }
            }
#pragma unroll
            for (int jj = 0; jj < T6_WIN * 4; ++jj) mx = fmaxf(mx, fabsf(xw[jj].x));
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int sh = oz_shift(mx);
            float* scl = ring + (w % T6_SC_SLOTS) * T6_SC_FLOATS;
            if (part == 0) scl[T6_M + n] = ldexpf(1.f, -sh);
            // the table rows' scales of this window (rows past the table read as zero scale)
            if (tid < T6_M) scl[tid] = trow < A.tc_rows ? scT[(size_t)w * A.tc_rows + trow] : 0.f;
#pragma unroll
            for (int cc = 0; cc < T6_WIN; ++cc) {
                const int k = w * T6_WIN + cc, s = k % T6_GSTAGES;
                if (k >= T6_GSTAGES)
                    ok = ok && mbar_wait(gempty0 + 8 * s, ((k - T6_GSTAGES) / T6_GSTAGES) & 1, abort_flag, A.err, 15, A.wait_limit);
                if (!ok) break;
                unsigned char* bt = gsm + s * T6_GSTAGE_BYTES;
                __nv_bfloat16 q[4][SL];
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) oz_slices<SL>(xw[4 * cc + jj].x, xw[4 * cc + jj].y, sh, q[jj]);
                // row n of each slice tile: 64 bytes, 16-byte chunk qq at (qq ^ ((n >> 1) & 3)); this
                // thread holds the 8-byte half (part & 1) of chunk part >> 1
                const int off = n * 64 + (((part >> 1) ^ ((n >> 1) & 3)) << 4) + (part & 1) * 8;
#pragma unroll
                for (int sp = 0; sp < SL; ++sp)
                    *reinterpret_cast<uint2*>(bt + sp * T6_B_TILE + off) =
                        make_uint2(bf16x2(q[0][sp], q[1][sp]), bf16x2(q[2][sp], q[3][sp]));
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(gfull0 + 8 * s);
                // the previous window's drain overlaps this window's MMAs
                if (cc == 0 && w >= 1) drain(w - 1);
            }
        }
        if (ok) drain(nwin - 1);
        // results: row m of D is A_T row m of the tile (overlap K) or, from ns on, its A_T V_T row (Q)
        if (ok && live && lrow < 2 * ns) {
            const int x = lrow < ns ? 0 : 1;
            const int i = A.qg_rows[tile * A.qg_max + (lrow < ns ? lrow : lrow - ns)];
            const size_t plane = (size_t)A.N_T * A.n_half;
            double* out = A.mol + (size_t)e * 2 * plane * 2;
#pragma unroll
            for (int k = 0; k < T6_COLS_PER_WARP; ++k) {
                const int go = ntile * T6_N + col0 + k, co = go >> 1, rio = go & 1;
                if (co >= A.n_half) continue;
                out[((size_t)x * plane + (size_t)i * A.n_half + co) * 2 + rio] = (double)hi[k] + (double)lo[k];
            }
        }
    }
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(T6_TMEM_COLS));
    }
}

wpccc_status launch_mol_tc64(wpccc_basis_s* B, int nev, const void* node, double2* mol, int* err, cudaStream_t st,
                             int slices) {
    if (slices != OZ_FAST_SLICES && slices != OZ_SLICES)
        return fail(WPCCC_EINVAL, "tensor-core contraction: 4 or 7 slices");
    if (!B->tc_layout) return fail(WPCCC_EINVAL, "tensor-core layout not prepared");
    if (B->G % (T6_K * T6_WIN) != 0) return fail(WPCCC_EUNSUPPORTED, "the node count must be a multiple of 128");
    const ElemScratch L = elem_scratch_layout(B);
    const size_t node_bytes = L.node_doubles * sizeof(double);
    // seven slice planes as one 3-D bf16 tensor: x = node (G), y = slice plane row (7 x tc_rows), z = evaluation
    Tc64Maps maps;
    const cuuint64_t dims[3] = {(cuuint64_t)B->G, (cuuint64_t)slices * L.tc_rows, (cuuint64_t)nev};
    const cuuint64_t strides[2] = {(cuuint64_t)B->G * 2, (cuuint64_t)node_bytes};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int h = 0; h < T6_BOXES; ++h) {
        const cuuint32_t box[3] = {(cuuint32_t)T6_K, (cuuint32_t)(32 * (h + 1)), 1};
        CUresult r = encode_fn()(&maps.m[h], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(node), dims, strides,
                                 box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(WPCCC_ECUDA, "cuTensorMapEncodeTiled failed for the slice planes");
    }
    Tc64Args a;
    a.G = B->G;
    a.N_T = B->N_T;
    a.n_half = B->n_half;
    a.nchunks = B->G / T6_K;
    a.n_ntiles = 0;   // per slice count, below
    a.tc_rows = L.tc_rows;
    a.qg_max = B->qg_max;
    a.qg_off = B->qg_off;
    a.qg_q = B->qg_off + B->n_qgroups + 1;
    a.qg_rows = B->qg_rows;
    a.half_q = B->tc_halfq;
    a.node = static_cast<const char*>(node);
    a.node_bytes = node_bytes;
    a.sc_off_f = L.t6_sc_off;
    a.ap_off_f = L.t6_ap_off;
    a.w_off_f = L.t6_w_off;
    a.mol = reinterpret_cast<double*>(mol);
    a.err = err;
    a.wait_limit = B->wait_polls;
    if (slices == OZ_SLICES) {
        using CF = Tc64Cfg<OZ_SLICES>;
        a.n_ntiles = (2 * B->n_half + CF::N - 1) / CF::N;
        const size_t smem = tc64_smem_bytes<OZ_SLICES>();
        WPCCC_CUDA(cudaFuncSetAttribute(k_mol_tc64<OZ_SLICES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_mol_tc64<OZ_SLICES><<<dim3(a.n_ntiles * B->n_qgroups, nev), CF::THREADS, smem, st>>>(maps, a);
    } else {
        using CF = Tc64Cfg<OZ_FAST_SLICES>;
        a.n_ntiles = (2 * B->n_half + CF::N - 1) / CF::N;
        const size_t smem = tc64_smem_bytes<OZ_FAST_SLICES>();
        WPCCC_CUDA(cudaFuncSetAttribute(k_mol_tc64<OZ_FAST_SLICES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        k_mol_tc64<OZ_FAST_SLICES><<<dim3(a.n_ntiles * B->n_qgroups, nev), CF::THREADS, smem, st>>>(maps, a);
    }
    WPCCC_CHECK_LAUNCH("k_mol_tc64");
    return WPCCC_OK;
}

}  // namespace wpccc
