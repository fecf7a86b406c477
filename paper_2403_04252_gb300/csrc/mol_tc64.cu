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
// Pipeline per CTA: warps 0-11 generate the Bw tiles (64-byte swizzled K-major rows) from the window's
// W and A_P, which warp 13 stages in shared memory by TMA one window ahead; warp 13 also streams the table
// tiles (cp.async.bulk.tensor, 64-byte swizzle) into their ring; warp 12 issues the tcgen05.mma
// instructions.  The accumulators (two TMEM buffers, one per window) are drained with seven slices by
// the producer warps, with four slices by four drain warps (14-17) that keep the double-float running
// sums in the spare TMEM columns.  Mbarriers between the roles; every wait is bounded and records a
// timeout in a device flag.
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
    static constexpr int MMA_WARP = PE_WARPS;                    // one thread issues the MMAs
    static constexpr int TMA_WARP = PE_WARPS + 1;                // one thread issues the TMA loads
    // four slices: four drain warps (one per TMEM lane quarter) fold the accumulators into double-float
    // running sums held in the spare TMEM columns, so that the producers never wait for a drain; seven
    // slices: the producers drain (their accumulators leave no spare columns)
    static constexpr int DRAIN_WARPS = SL == 7 ? 0 : 4;
    static constexpr int DRAIN0 = PE_WARPS + 2;                  // first drain warp
    static constexpr int THREADS = (PE_WARPS + 2 + DRAIN_WARPS) * 32;
    static constexpr int SUM_COL = 2 * ACC * N;                  // TMEM column of the running sums (hi, then lo)
    static constexpr int HALF = N / 2;                           // half columns of a CTA
    // table tiles in flight: four with four slices, two with seven (shared memory)
    static constexpr int TSTAGES = SL == 7 ? 2 : 4;
    static constexpr int BUF_COLS = ACC * N;                    // column offset of the second buffer
    static constexpr int B_TILE = N * 64;                       // bytes of one slice of the generated tile
    static constexpr int TSTAGE_BYTES = SL * T6_M * 64;         // a multiple of 1024
    static constexpr int GSTAGE_BYTES = SL * N * 64;            // a multiple of 1024
    static constexpr int SC_FLOATS = T6_M + N;                  // per scale slot: table rows, generated rows
    static constexpr int COLS_PER_WARP = N / (PE_WARPS / 4);    // 16 columns per epilogue warp
    // generated tiles in flight: four with four slices (the producers run up to four chunks ahead of the
    // MMAs); two with seven (shared memory; the producers drain window w - 1 after the first chunk of
    // window w)
    static constexpr int GSTAGES = SL == 7 ? 2 : 4;
    // scale slots, one per window.  Seven slices: a thread may start window w + 1 only after every producer
    // has drained window w - 1.  Four slices: while the drain warps fold window j, the MMAs may finish
    // window j + 1 (window j + 2 needs the accumulators that drain frees) and the producers run four chunks
    // further, into window j + 3, so four slots.
    static constexpr int SC_SLOTS = SL == 7 ? 2 : 4;
    static_assert(PE_WARPS * 32 == N * 8, "eight producer threads (4 nodes each) per generated row");
    static_assert(2 * BUF_COLS <= 512, "two buffers of accumulators fit the TMEM allocation");
    static_assert(DRAIN_WARPS == 0 || SUM_COL + 2 * N <= 512, "the running sums fit the spare TMEM columns");
    static_assert(TSTAGE_BYTES % 1024 == 0 && GSTAGE_BYTES % 1024 == 0, "1024-byte aligned stages");
};
constexpr int T6_TMEM_COLS = 512;
constexpr int T6_WIN_BYTES = T6_WIN * T6_K * 8;        // one row of a window's double-floats (128 nodes)
constexpr int T6_A_TILE = T6_M * 64;                   // bytes of one slice of the table tile
constexpr int T6_BOXES = T6_M / 32;                    // table box heights 32, 64, 96, 128 rows

// Dynamic shared memory: the table ring, the generated ring, one window of the generated operand's inputs
// (A_P of the CTA's half columns, then hw rows of W / r_T), the scale slots and the mbarriers.
template <int SL>
static size_t tc64_smem_bytes(int hw) {
    using CF = Tc64Cfg<SL>;
    return 1024 + (size_t)CF::TSTAGES * CF::TSTAGE_BYTES + (size_t)CF::GSTAGES * CF::GSTAGE_BYTES +
           (size_t)(CF::HALF + hw) * T6_WIN_BYTES + sizeof(float) * CF::SC_SLOTS * CF::SC_FLOATS +
           8 * (2 * CF::TSTAGES + 2 * CF::GSTAGES + 6);
}

// Tensor maps of the slice planes with box heights 32, 64, 96 and 128 rows: a row tile loads only the
// 32-row multiple that covers its rows (rows past its end are loaded from the next tile, or left stale,
// and only feed accumulator lanes that are never read).
// mA, mW: the double-float A_P rows and W / r_T rows of the node tables as FP32 tensors (x = float within a
// row, y = row, z = evaluation) with boxes of one window (256 floats) by the CTA's half columns / hw rows.
struct Tc64Maps {
    CUtensorMap m[T6_BOXES];
    CUtensorMap mA, mW;
};

struct Tc64Args {
    int G, N_T, n_half, nchunks, n_ntiles, tc_rows, qg_max;
    const int* qg_off;     // [tiles + 1] first split-table row of each row tile
    const int* qg_q;       // [tiles] q' of each row tile
    const int* qg_rows;    // [tiles][qg_max] target state of each A_T row of a tile
    const int* half_q;     // [n_half] q of each half column
    const char* node;      // node tables (FP64-accurate tensor-core layout) of the launch's evaluations
    size_t node_bytes;     // stride between evaluations
    size_t sc_off_f;
    int hw;                // W rows staged per window: 2 (l_P + 1), every d = |q - q'| one CTA can meet
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
    constexpr int T6_GSTAGES = CF::GSTAGES;
    constexpr int T6_TSTAGES = CF::TSTAGES;
    constexpr int T6_SC_SLOTS = CF::SC_SLOTS;
    constexpr bool X2 = SL == OZ_FAST_SLICES;   // four slices: packed FP32x2 producer and drain
    extern __shared__ __align__(1024) unsigned char t6_smem_raw[];
    unsigned char* sm = t6_smem_raw + ((1024 - (smem_u32(t6_smem_raw) & 1023)) & 1023);
    unsigned char* gsm = sm + T6_TSTAGES * T6_TSTAGE_BYTES;                        // generated tiles
    unsigned char* raw = gsm + T6_GSTAGES * T6_GSTAGE_BYTES;                     // A_P rows, then W rows
    float* ring = reinterpret_cast<float*>(raw + (CF::HALF + A.hw) * T6_WIN_BYTES);  // [slot][T6_SC_FLOATS]
    uint64_t* bars = reinterpret_cast<uint64_t*>(ring + T6_SC_SLOTS * T6_SC_FLOATS);
    __shared__ uint32_t s_tmem;
    __shared__ int s_abort, s_dlo;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntile = blockIdx.x % A.n_ntiles, tile = blockIdx.x / A.n_ntiles, e = blockIdx.y;
    const int row0 = A.qg_off[tile], ns = (A.qg_off[tile + 1] - row0) / 2;   // states of the row tile
    const int qp = A.qg_q[tile];
    const int box = (2 * ns + 31) / 32;                  // table box height of this tile, in 32-row units
    // tfull[TSTAGES] (TMA), tempty[TSTAGES] (MMA commit), gfull[GSTAGES] (producers), gempty[GSTAGES] (MMA
    // commit), accf[2] (MMA commit), acce[2] (drain), rawfull (TMA), rawempty (producers)
    const uint32_t tfull0 = smem_u32(bars), tempty0 = tfull0 + 8 * T6_TSTAGES, gfull0 = tempty0 + 8 * T6_TSTAGES,
                   gempty0 = gfull0 + 8 * T6_GSTAGES, accf0 = gempty0 + 8 * T6_GSTAGES, acce0 = accf0 + 16,
                   rawfull = acce0 + 16, rawempty = rawfull + 8;
    const int c0 = ntile * CF::HALF;                     // first half column of this CTA
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
            mbar_init(acce0 + 8 * b, (CF::DRAIN_WARPS > 0 ? CF::DRAIN_WARPS : T6_PE_WARPS) * 32);
        }
        mbar_init(rawfull, 1);
        mbar_init(rawempty, T6_PE_WARPS * 32);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        // the smallest d = |q_c - q'| over the CTA's half columns: the first W row the window loads hold
        int dl = 1 << 20;
        if (lane < CF::HALF && c0 + lane < A.n_half) {
            dl = A.half_q[c0 + lane] - qp;
            dl = dl < 0 ? -dl : dl;
        }
        for (int o = 16; o > 0; o >>= 1) dl = min(dl, __shfl_xor_sync(0xffffffffu, dl, o));
        if (lane == 0) s_dlo = dl < (1 << 20) ? dl : 0;
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

    if (warp == CF::TMA_WARP) {
        // ---- TMA issue (one thread): the table tiles chunk by chunk into their ring, a slot refilled as soon as
        // the MMAs that read it have completed; the generated operand's inputs window by window into the
        // staged-input buffer, refilled as soon as every producer has read the previous window
        if (lane == 0) {
            const uint32_t tx = (uint32_t)(SL * box * 32 * 64);
            const uint32_t rtx = (uint32_t)((CF::HALF + A.hw) * T6_WIN_BYTES);
            const CUtensorMap* tmap = &maps.m[box - 1];
            const int dlo = s_dlo, nwin = nk / T6_WIN;
            auto issue_table = [&](int k) {
                const int s = k % T6_TSTAGES;
                unsigned char* st = sm + s * T6_TSTAGE_BYTES;
                const uint32_t bar = tfull0 + 8 * s;
                mbar_arrive_tx(bar, tx);
                for (int sp = 0; sp < SL; ++sp)
                    tma_load_3d(smem_u32(st + sp * T6_A_TILE), tmap, k * T6_K, sp * A.tc_rows + row0, e, bar);
            };
            auto issue_raw = [&](int w) {
                mbar_arrive_tx(rawfull, rtx);
                tma_load_3d(smem_u32(raw), &maps.mA, w * T6_WIN * T6_K * 2, c0, e, rawfull);
                tma_load_3d(smem_u32(raw + CF::HALF * T6_WIN_BYTES), &maps.mW, w * T6_WIN * T6_K * 2, 2 * dlo, e, rawfull);
            };
            bool ok = true;
            int issued = 0, issued_raw = 0;
            if (nwin > 0) issue_raw(issued_raw++);
            for (; issued < T6_TSTAGES && issued < nk; ++issued) issue_table(issued);
            // then whichever is free first: the staged-input buffer once every producer has read the previous
            // window, a table slot once the MMAs of its previous chunk have completed (non-blocking tests, so
            // that neither refill waits behind the other); a run of `wait_limit` idle polls gives up
            long idle = 0;
            while (ok && (issued < nk || issued_raw < nwin)) {
                bool moved = false;
                if (issued_raw < nwin && mbar_test(rawempty, (issued_raw - 1) & 1)) {
                    issue_raw(issued_raw++);
                    moved = true;
                }
                if (issued < nk) {
                    const int kp = issued - T6_TSTAGES;
                    if (mbar_test(tempty0 + 8 * (kp % T6_TSTAGES), (kp / T6_TSTAGES) & 1)) {
                        issue_table(issued++);
                        moved = true;
                    }
                }
                if (moved) {
                    idle = 0;
                } else if (*abort_flag) {
                    ok = false;
                } else if (++idle >= A.wait_limit) {
                    *abort_flag = 1;
                    atomicExch(A.err, 13);
                    ok = false;
                } else {
                    __nanosleep(32);   // leave the issue slots to the producers while nothing is free
                }
            }
            // every copy issued has landed before the CTA exits: at once on the normal path (the consumers
            // waited for them), bounded where a role gave up before reading its data
            for (int k = issued > T6_TSTAGES ? issued - T6_TSTAGES : 0; k < issued; ++k) {
                const int s = k % T6_TSTAGES;
                for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(tfull0 + 8 * s, (k / T6_TSTAGES) & 1); ++it) {
                }
            }
            if (issued_raw > 0)
                for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(rawfull, (issued_raw - 1) & 1); ++it) {
                }
        }
    } else if (warp == CF::MMA_WARP) {
        // ---- MMA issue (one thread)
        if (lane == 0) {
            const uint32_t idesc = bf16_idesc_mn(T6_M, T6_N);
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
                if constexpr (SL == OZ_FAST_SLICES) {
                    // four slices: the generated tile's slices B_0..B_3 lie one after the other, so one MMA
                    // per table slice A_i and K step forms A_i [B_0 .. B_{3-i}] (N = (4 - i) 48) into the
                    // columns of levels i .. 3: product (i, j) lands on level i + j's accumulator.  Each table
                    // slice is read once per K step (4 MMAs instead of 10); A_0 [B_0 .. B_3] opens a window.
#pragma unroll
                    for (int kk = 0; kk < T6_K / 16; ++kk) {
#pragma unroll
                        for (int i = 0; i < SL; ++i) {
                            tc_mma(dbase + (uint32_t)(i * T6_N), da + (uint64_t)((i * T6_A_TILE + kk * 32) >> 4),
                                   db + (uint64_t)((kk * 32) >> 4), bf16_idesc_mn(T6_M, (SL - i) * T6_N),
                                   kk == 0 && i == 0 ? fresh : 1u);
                        }
                    }
                } else {
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
                }
                tc_commit(tempty0 + 8 * s);
                tc_commit(gempty0 + 8 * s2);
                last_mma = k;
                if (k % T6_WIN == T6_WIN - 1) tc_commit(accf0 + 8 * b);
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
    } else if (CF::DRAIN_WARPS > 0 && warp >= CF::DRAIN0) {
        // ---- drain warps (four slices): per window, the four level accumulators of this warp's 32 TMEM
        // lanes (table rows) and 48 columns folded with the window's scales into the double-float running
        // sums in TMEM columns SUM_COL (high parts) and SUM_COL + N (low parts), 8 columns at a time, two
        // per packed FP32x2 instruction: L0 + rint(L1) exact into the TwoSum high part, frac(L1) + L2 + L3
        // rounded once (below 2^8 units, its rounding under 2^-16 units: 2^-30 of one node's largest
        // product) into the low part.  After the last window the sums go to the output.
        const int qd = warp & 3, lrow = qd * 32 + lane;
        const bool live = qd * 32 < 2 * ns;
        const int nwin = nk / T6_WIN;
        const uint32_t lb = tmem + ((uint32_t)(qd * 32) << 16);
        const f32x2 CM = x2_pack(12582912.f, 12582912.f);
        const size_t plane = (size_t)A.N_T * A.n_half;
        double* out = A.mol + (size_t)e * 2 * plane * 2;
        int xo = 0, io = 0;
        if (lrow < 2 * ns) {
            xo = lrow < ns ? 0 : 1;
            io = A.qg_rows[tile * A.qg_max + (lrow < ns ? lrow : lrow - ns)];
        }
        bool ok = true;
        for (int j = 0; j < nwin && ok; ++j) {
            const int b = j & 1;
            ok = mbar_wait(accf0 + 8 * b, (j >> 1) & 1, abort_flag, A.err, 14, A.wait_limit);
            if (!ok) break;
            tc_fence_after();
            if (live) {
                const float* scl = ring + (j % T6_SC_SLOTS) * T6_SC_FLOATS;
                const float sa = scl[lrow];
                const f32x2 sa2 = x2_pack(sa, sa);
#pragma unroll 1
                for (int g = 0; g < T6_N / 8; ++g) {
                    float v[T6_ACC][8], hv[8], lv[8];
#pragma unroll
                    for (int a = 0; a < T6_ACC; ++a) tmem_ld8(lb + (uint32_t)(b * T6_BUF_COLS + a * T6_N + 8 * g), v[a]);
                    if (j > 0) {
                        tmem_ld8(lb + (uint32_t)(CF::SUM_COL + 8 * g), hv);
                        tmem_ld8(lb + (uint32_t)(CF::SUM_COL + T6_N + 8 * g), lv);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
                    if (j == 0) {
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            hv[u] = 0.f;
                            lv[u] = 0.f;
                        }
                    }
#pragma unroll
                    for (int u = 0; u < 8; u += 2) {
                        const float2 sn = *reinterpret_cast<const float2*>(scl + T6_M + 8 * g + u);
                        const f32x2 sc = x2_mul(sa2, x2_pack(sn.x, sn.y));
                        const f32x2 L0 = x2_pack(v[0][u], v[0][u + 1]), L1 = x2_pack(v[1][u], v[1][u + 1]),
                                    L2 = x2_pack(v[2][u], v[2][u + 1]), L3 = x2_pack(v[3][u], v[3][u + 1]);
                        const f32x2 l1h = x2_sub(x2_add(L1, CM), CM);
                        const f32x2 xa = x2_add(L0, l1h);
                        const f32x2 xbc = x2_add(x2_add(x2_sub(L1, l1h), L2), L3);
                        f32x2 r1;
                        const f32x2 hi2 = two_sum_x2(x2_pack(hv[u], hv[u + 1]), x2_mul(xa, sc), r1);
                        const f32x2 lo2 = x2_fma(xbc, sc, x2_add(x2_pack(lv[u], lv[u + 1]), r1));
                        x2_unpack(hi2, hv[u], hv[u + 1]);
                        x2_unpack(lo2, lv[u], lv[u + 1]);
                    }
                    if (j + 1 < nwin) {
                        tmem_st8(lb + (uint32_t)(CF::SUM_COL + 8 * g), hv);
                        tmem_st8(lb + (uint32_t)(CF::SUM_COL + T6_N + 8 * g), lv);
                    } else if (lrow < 2 * ns) {
                        // results: row lrow of D is A_T row lrow of the tile (overlap K) or, from ns on, its
                        // A_T V_T row (Q)
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int go = ntile * T6_N + 8 * g + u, co = go >> 1, rio = go & 1;
                            if (co < A.n_half)
                                out[((size_t)xo * plane + (size_t)io * A.n_half + co) * 2 + rio] =
                                    (double)hv[u] + (double)lv[u];
                        }
                    }
                }
                asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
            }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * b);
        }
    } else {
        // ---- producers of the generated operand (eight threads per row, four nodes each), and the epilogue
        const int n = tid >> 3, part = tid & 7;
        const int gr = ntile * T6_N + n, c = gr >> 1, ri = gr & 1;
        const bool valid = c < A.n_half;
        // this row's window inputs in the raw buffer: A_P row n / 2 (zero past the last half column), W row
        // 2 (d - d_lo) + re/im
        int lw = ri;
        if (valid) {
            int d = A.half_q[c] - qp;
            d = d < 0 ? -d : d;
            lw = 2 * (d - s_dlo) + ri;
        }
        // seven slices: this thread's nodes 4 part .. 4 part + 3 of each chunk (32 bytes of each row); four
        // slices: nodes 2 part, 2 part + 1 and 16 + 2 part, 17 + 2 part (16 bytes at part 16 and 128 + part 16),
        // so that the eight threads of a row read 128 contiguous bytes per load, free of bank conflicts
        const int pofs = X2 ? part * 16 : part * 32;
        const unsigned char* ap_s = raw + (n >> 1) * T6_WIN_BYTES + pofs;
        const unsigned char* wd_s = raw + (CF::HALF + lw) * T6_WIN_BYTES + pofs;
        const float* nbf = reinterpret_cast<const float*>(nb);
        const float* scT = nbf + A.sc_off_f;   // [chunk][tc_rows]
        // epilogue: accumulator lanes 32 qd .. 32 qd + 31 (table rows), 16 columns from col0
        const int qd = warp & 3, col0 = (warp >> 2) * T6_COLS_PER_WARP;
        const int lrow = qd * 32 + lane;
        const bool live = qd * 32 < 2 * ns;    // warps whose rows all lie past the tile skip the arithmetic
        // seven slices: this thread's running sums (four slices: held in TMEM by the drain warps)
        float hi[X2 ? 1 : T6_COLS_PER_WARP], lo[X2 ? 1 : T6_COLS_PER_WARP];
#pragma unroll
        for (int k = 0; k < (X2 ? 1 : T6_COLS_PER_WARP); ++k) {
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
                        // 2^-16 below 2^7)
                        const float l1h = rintf(v[1][u]);
                        const float xa = __fadd_rn(v[0][u], l1h);
                        const float xb = __fadd_rn(__fsub_rn(v[1][u], l1h), v[2][u]);
                        // seven slices: frac(L1) + L2 exact into the high part as well; L3 + T rounded
                        // (below 1, its rounding under 2^-24)
                        float r1, r2;
                        hi[k] = two_sum(hi[k], xa * sc, r1);
                        hi[k] = two_sum(hi[k], xb * sc, r2);
                        const float xc = __fadd_rn(v[3][u], v[T6_ACC - 1][u]);
                        lo[k] = __fadd_rn(lo[k], __fadd_rn(__fadd_rn(r1, r2), xc * sc));
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * b);
        };
        const int nwin = nk / T6_WIN;
        const int trow = row0 + tid;
        // the table rows' scales (rows past the table read as zero scale), loaded one window ahead of the
        // window that stores them in its scale slot
        const bool has_trow = tid < T6_M && trow < A.tc_rows;
        float tsc = has_trow ? scT[trow] : 0.f;
        if constexpr (X2) {
        // four slices, two nodes per packed FP32x2 instruction: the products as unnormalised pairs p + e,
        // sliced by rounding to each slice's grid
        for (int w = 0; w < nwin && ok; ++w) {
            f32x2 pw[T6_WIN * 2], ew[T6_WIN * 2];
            float mx = 0.f;
            ok = mbar_wait(rawfull, w & 1, abort_flag, A.err, 18, A.wait_limit);
            if (!ok) break;
#pragma unroll
            for (int cc = 0; cc < T6_WIN; ++cc) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 wq = *reinterpret_cast<const float4*>(wd_s + cc * T6_K * 8 + h * 128);
                    const float4 aq = *reinterpret_cast<const float4*>(ap_s + cc * T6_K * 8 + h * 128);
                    const int j = 2 * cc + h;
                    df_mul_pe_x2(x2_pack(wq.x, wq.z), x2_pack(wq.y, wq.w), x2_pack(aq.x, aq.z), x2_pack(aq.y, aq.w),
                                 pw[j], ew[j]);
                    float p0, p1;
                    x2_unpack(pw[j], p0, p1);
                    mx = fmaxf(mx, fmaxf(fabsf(p0), fabsf(p1)));
                }
            }
            // this thread has read the window's inputs: its shared-memory reads ordered before the TMA
            // (async proxy) writes of the next window, then the release to the TMA thread
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(rawempty);
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int sh = min(oz_shift(mx), 127);
            const float sc2 = __int_as_float((sh + 127) << 23);
            const f32x2 s2 = x2_pack(sc2, sc2);
            float* scl = ring + (w % T6_SC_SLOTS) * T6_SC_FLOATS;
            if (part == 0) scl[T6_M + n] = ldexpf(1.f, -sh);
            if (tid < T6_M) scl[tid] = tsc;
            if (has_trow && w + 1 < nwin) tsc = scT[(size_t)(w + 1) * A.tc_rows + trow];
#pragma unroll
            for (int cc = 0; cc < T6_WIN; ++cc) {
                const int k = w * T6_WIN + cc, s = k % T6_GSTAGES;
                if (k >= T6_GSTAGES)
                    ok = ok && mbar_wait(gempty0 + 8 * s, ((k - T6_GSTAGES) / T6_GSTAGES) & 1, abort_flag, A.err, 15, A.wait_limit);
                if (!ok) break;
                unsigned char* bt = gsm + s * T6_GSTAGE_BYTES;
                f32x2 t0[4], t1[4];
                oz_slices4_pe_x2(pw[2 * cc], ew[2 * cc], s2, t0);
                oz_slices4_pe_x2(pw[2 * cc + 1], ew[2 * cc + 1], s2, t1);
                // row n of each slice tile: 64 bytes, 16-byte chunk qq at (qq ^ ((n >> 1) & 3)); nodes 2 part, 2 part
                // + 1 are bytes 4 part .. 4 part + 3 (chunk part >> 2), nodes 16 + 2 part, 17 + 2 part two
                // chunks further
                const int sw = (n >> 1) & 3, within = (part & 3) * 4;
                const int off0 = n * 64 + (((part >> 2) ^ sw) << 4) + within;
                const int off1 = n * 64 + (((2 + (part >> 2)) ^ sw) << 4) + within;
#pragma unroll
                for (int sp = 0; sp < 4; ++sp) {
                    float a0, a1, b0, b1;
                    x2_unpack(t0[sp], a0, a1);
                    x2_unpack(t1[sp], b0, b1);
                    *reinterpret_cast<uint32_t*>(bt + sp * T6_B_TILE + off0) = bf16x2_exact(a0, a1);
                    *reinterpret_cast<uint32_t*>(bt + sp * T6_B_TILE + off1) = bf16x2_exact(b0, b1);
                }
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_arrive(gfull0 + 8 * s);
            }
        }
        } else {
        for (int w = 0; w < nwin && ok; ++w) {
            // this thread's 16 generated values of the window (four per chunk), their row maximum over the
            // window's 128 nodes (the row's eight threads), and the window's scales
            float2 xw[T6_WIN * 4];
            float mx = 0.f;
            ok = mbar_wait(rawfull, w & 1, abort_flag, A.err, 18, A.wait_limit);
            if (!ok) break;
#pragma unroll
            for (int cc = 0; cc < T6_WIN; ++cc) {
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float4 wq = *reinterpret_cast<const float4*>(wd_s + cc * T6_K * 8 + h * 16);
                    const float4 aq = *reinterpret_cast<const float4*>(ap_s + cc * T6_K * 8 + h * 16);
                    xw[4 * cc + 2 * h] = df_mul(make_float2(wq.x, wq.y), make_float2(aq.x, aq.y));
                    xw[4 * cc + 2 * h + 1] = df_mul(make_float2(wq.z, wq.w), make_float2(aq.z, aq.w));
                }
            }
            asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
            mbar_arrive(rawempty);
#pragma unroll
            for (int jj = 0; jj < T6_WIN * 4; ++jj) mx = fmaxf(mx, fabsf(xw[jj].x));
#pragma unroll
            for (int o = 1; o < 8; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            const int sh = oz_shift(mx);
            float* scl = ring + (w % T6_SC_SLOTS) * T6_SC_FLOATS;
            if (part == 0) scl[T6_M + n] = ldexpf(1.f, -sh);
            if (tid < T6_M) scl[tid] = tsc;
            if (has_trow && w + 1 < nwin) tsc = scT[(size_t)(w + 1) * A.tc_rows + trow];
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
        }
        if constexpr (!X2) {
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
    // the generated operand's inputs as FP32 tensors (a double-float is two floats): A_P [n_half][2 G] and
    // W / r_T [d][re, im][2 G] per evaluation; boxes of one window by 24 half columns / hw rows (rows past
    // the tensor read as zero)
    const int hw = 2 * (B->P.lmax + 1);
    if (hw > 2 * (B->dmax + 1) || hw > 256) return fail(WPCCC_EINVAL, "tensor-core contraction: W rows");
    {
        const char* nodef = static_cast<const char*>(node);
        const cuuint64_t fstr[2] = {(cuuint64_t)B->G * 2 * sizeof(float), (cuuint64_t)node_bytes};
        const cuuint64_t dA[3] = {(cuuint64_t)B->G * 2, (cuuint64_t)B->n_half, (cuuint64_t)nev};
        const cuuint64_t dW[3] = {(cuuint64_t)B->G * 2, (cuuint64_t)2 * (B->dmax + 1), (cuuint64_t)nev};
        const cuuint32_t bA[3] = {(cuuint32_t)(T6_WIN * T6_K * 2), (cuuint32_t)(Tc64Cfg<OZ_FAST_SLICES>::HALF), 1};
        const cuuint32_t bW[3] = {(cuuint32_t)(T6_WIN * T6_K * 2), (cuuint32_t)hw, 1};
        CUresult r = encode_fn()(&maps.mA, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                                 const_cast<char*>(nodef + L.t6_ap_off * sizeof(float)), dA, fstr, bA, estr,
                                 CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                 CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r == CUDA_SUCCESS)
            r = encode_fn()(&maps.mW, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3,
                            const_cast<char*>(nodef + L.t6_w_off * sizeof(float)), dW, fstr, bW, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(WPCCC_ECUDA, "cuTensorMapEncodeTiled failed for the node weights");
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
    a.hw = hw;
    a.mol = reinterpret_cast<double*>(mol);
    a.err = err;
    a.wait_limit = B->wait_polls;
    if (slices == OZ_SLICES) {
        using CF = Tc64Cfg<OZ_SLICES>;
        a.n_ntiles = (2 * B->n_half + CF::N - 1) / CF::N;
        const size_t smem = tc64_smem_bytes<OZ_SLICES>(hw);
        WPCCC_CUDA(cudaFuncSetAttribute(k_mol_tc64<OZ_SLICES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_mol_tc64<OZ_SLICES><<<dim3(a.n_ntiles * B->n_qgroups, nev), CF::THREADS, smem, st>>>(maps, a);
    } else {
        using CF = Tc64Cfg<OZ_FAST_SLICES>;
        a.n_ntiles = (2 * B->n_half + CF::N - 1) / CF::N;
        const size_t smem = tc64_smem_bytes<OZ_FAST_SLICES>(hw);
        WPCCC_CUDA(cudaFuncSetAttribute(k_mol_tc64<OZ_FAST_SLICES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)smem));
        k_mol_tc64<OZ_FAST_SLICES><<<dim3(a.n_ntiles * B->n_qgroups, nev), CF::THREADS, smem, st>>>(maps, a);
    }
    WPCCC_CHECK_LAUNCH("k_mol_tc64");
    return WPCCC_OK;
}

}  // namespace wpccc
