// Device helpers shared by the RK4 kernels of the propagation and of its adjoint: the FP64 matrix-vector
// product, the triangular solves with LAPACK-layout LU factors, and the stage operator -(i/v) S^{-1} H.
// Every helper is called by all RK_THREADS threads of a block and ends with a block barrier.
#pragma once

#include "ozaki.cuh"
#include "tc_ptx.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int RK_THREADS = 512;

// Status bits the RK4 kernels raise in the propagation's flag word.
enum : int { FLAG_SINGULAR = 1, FLAG_NONFINITE = 2, FLAG_NOCONV = 4, FLAG_TIMEOUT = 8 };

// Convergence test of a refinement's last sweep: max|dx| <= tol max|x| over the block's vector, else
// FLAG_NOCONV (dmax, xmax: this thread's maxima).  Called by all threads; ends with a block barrier.
static __device__ void refine_check(double dmax, double xmax, double tol, int* flags) {
    __shared__ double red[2][RK_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = dmax;
        red[1][threadIdx.x >> 5] = xmax;
    }
    __syncthreads();
    if (threadIdx.x == 0 && flags) {
        double d = 0.0, x = 0.0;
        for (int i = 0; i < RK_THREADS / 32; ++i) {
            d = fmax(d, red[0][i]);
            x = fmax(x, red[1][i]);
        }
        if (!(d <= tol * x)) atomicOr(flags, FLAG_NOCONV);
    }
    __syncthreads();
}

// t <- S^{-1} t in place from the factors P S = L U (LAPACK layout, pivots 1-based);
// C2 = double2 (FP64 factors) or float2 (FP32 factors of the mixed-precision form).
// Blocked by 32 rows: each 32 x 32 diagonal block is staged in shared memory (blk) and solved by
// one warp; the off-diagonal updates run on every thread.
template <typename C2>
static __device__ void lu_solve_inplace(const C2* __restrict__ LU, const int* __restrict__ piv, int N, C2* t, C2* blk) {
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
#pragma unroll 4
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

// An FP64 value as a double-float (hi, lo), by integer operations on its bits (no FP64 arithmetic): hi is x
// truncated to 24 significant bits, lo the next 23 bits (exact: the bits are taken, not rounded), so
// |x - hi - lo| < 2^-46 |x|.  For 2^-126 <= |x| < 2^-80 lo is dropped (an absolute error below 2^-104), below
// 2^-126 x reads as zero; infinities and NaNs go through the FP64 conversion and stay non-finite.
static __device__ __forceinline__ float2 split_bits(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t h = (uint32_t)(u >> 32), l = (uint32_t)u;
    const uint32_t e = (h >> 20) & 0x7FFu, sg = h & 0x80000000u;
    if (e - 897u > 253u) return make_float2(e < 897u ? 0.f : __double2float_rn(x), 0.f);
    const float hi = __uint_as_float(sg | ((e - 896u) << 23) | ((h & 0xFFFFFu) << 3) | (l >> 29));
    const uint32_t r = (l >> 6) & 0x7FFFFFu;   // mantissa bits 28..6, the value r 2^(e - 1069)
    const float rf = __fsub_rn(__uint_as_float(0x4B000000u | r), 8388608.f);
    const float lo = e >= 943u ? __fmul_rn(rf, __uint_as_float((e - 942u) << 23)) : 0.f;
    return make_float2(hi, __uint_as_float(__float_as_uint(lo) | sg));
}

// (s, c) += a b for double-floats a = (a.x, a.y) pairs, two real products at once (one per half of the
// FP32x2 registers): the products' high parts join s by TwoSum, their residuals and the TwoSum errors
// join c (the compensated dot product of Ogita, Rump and Oishi, with double-float operands).
static __device__ __forceinline__ void dot2_acc_x2(f32x2& s, f32x2& c, f32x2 ah, f32x2 al, f32x2 bh, f32x2 bl) {
    const f32x2 p = x2_mul(ah, bh);
    f32x2 e = x2_fma(ah, bh, x2_neg(p));
    e = x2_fma(ah, bl, e);
    e = x2_fma(al, bh, e);
    f32x2 t;
    s = two_sum_x2(s, p, t);
    c = x2_add(c, x2_add(t, e));
}

// out = M y like matvec, for the reduced-precision forms' right-hand side H y: M's FP64 entries and y taken
// as double-floats (split_bits), the sums compensated on the FP32 pipe (dot2_acc_x2, the real and the
// imaginary part in the two halves), about 2^-44 of sum_j |M_ij| |y_j|.  ys: scratch of N float4.
__device__ inline void matvec_df(const double2* __restrict__ M, int N, const double2* y, double2* out, float4* ys) {
    for (int j = threadIdx.x; j < N; j += RK_THREADS) {
        const float2 a = split_bits(y[j].x), b = split_bits(y[j].y);
        ys[j] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        f32x2 s = x2_pack(0.f, 0.f), c = x2_pack(0.f, 0.f);   // (re, im)
        const double2* row = M + i;
#pragma unroll 4
        for (int j = 0; j < N; ++j) {
            const double2 m = row[(size_t)j * N];
            const float2 mr = split_bits(m.x), mi = split_bits(m.y);
            const float4 q = ys[j];   // (Re y hi, Re y lo, Im y hi, Im y lo)
            // re += mr yr - mi yi, im += mr yi + mi yr
            dot2_acc_x2(s, c, x2_pack(mr.x, mr.x), x2_pack(mr.y, mr.y), x2_pack(q.x, q.z), x2_pack(q.y, q.w));
            dot2_acc_x2(s, c, x2_pack(-mi.x, mi.x), x2_pack(-mi.y, mi.y), x2_pack(q.z, q.x), x2_pack(q.w, q.y));
        }
        float sr, si, cr, ci;
        x2_unpack(s, sr, si);
        x2_unpack(c, cr, ci);
        out[i] = make_double2((double)sr + (double)cr, (double)si + (double)ci);
    }
    __syncthreads();
}

// Shared-memory staging of a column-major matrix for matvec_df_staged: `cols` columns per slot, two slots,
// then their two mbarriers; `polls` bounds every wait.
struct Staging {
    double2* buf;        // [2][cols][N]
    uint64_t* bars;      // [2]
    int cols;
    long polls;
};

// matvec_df with M streamed through shared memory: blocks of `cols` consecutive columns (contiguous in the
// column-major storage) are brought in by bulk asynchronous copies, one block ahead, issued by thread 0; every
// thread reads its row of the block from shared memory.  The sums, and so the result, are those of
// matvec_df (the same terms in the same order).  Needs N <= RK_THREADS.  A wait that gives up raises
// FLAG_TIMEOUT and the sweep goes on (with what the slot holds); the copies in flight land before return.
__device__ inline void matvec_df_staged(const double2* __restrict__ M, int N, const double2* y, double2* out,
                                        float4* ys, const Staging& sg, int* flags) {
    const int tid = threadIdx.x;
    for (int j = tid; j < N; j += RK_THREADS) {
        const float2 a = split_bits(y[j].x), b = split_bits(y[j].y);
        ys[j] = make_float4(a.x, a.y, b.x, b.y);
    }
    const uint32_t bar0 = smem_u32(sg.bars);
    if (tid == 0) {
        mbar_init(bar0, 1);
        mbar_init(bar0 + 8, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    const int nblk = (N + sg.cols - 1) / sg.cols;
    auto issue = [&](int blk) {
        const int c0 = blk * sg.cols, nc = min(sg.cols, N - c0);
        const uint32_t bytes = (uint32_t)nc * (uint32_t)N * (uint32_t)sizeof(double2);
        const uint32_t bar = bar0 + 8 * (blk & 1);
        // the slot's previous contents were read through the generic proxy: order those reads first
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        mbar_arrive_tx(bar, bytes);
        asm volatile(
            "{\n.reg .u64 g;\ncvta.to.global.u64 g, %1;\n"
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [g], %2, [%3];\n}\n" ::"r"(
                smem_u32(sg.buf + (size_t)(blk & 1) * sg.cols * N)),
            "l"(M + (size_t)c0 * N), "r"(bytes), "r"(bar)
            : "memory");
    };
    if (tid == 0) {
        issue(0);
        if (nblk > 1) issue(1);
    }
    f32x2 s = x2_pack(0.f, 0.f), c = x2_pack(0.f, 0.f);   // (re, im) of row tid
    for (int blk = 0; blk < nblk; ++blk) {
        const uint32_t bar = bar0 + 8 * (blk & 1), par = (blk >> 1) & 1;
        long it = 0;
        while (!mbar_try(bar, par) && ++it < sg.polls) {
        }
        if (it >= sg.polls && flags) atomicOr(flags, FLAG_TIMEOUT);
        const int c0 = blk * sg.cols, nc = min(sg.cols, N - c0);
        if (tid < N) {
            const double2* col = sg.buf + (size_t)(blk & 1) * sg.cols * N + tid;
            for (int cc = 0; cc < nc; ++cc) {
                const double2 m = col[(size_t)cc * N];
                const float2 mr = split_bits(m.x), mi = split_bits(m.y);
                const float4 q = ys[c0 + cc];
                dot2_acc_x2(s, c, x2_pack(mr.x, mr.x), x2_pack(mr.y, mr.y), x2_pack(q.x, q.z), x2_pack(q.y, q.w));
                dot2_acc_x2(s, c, x2_pack(-mi.x, mi.x), x2_pack(-mi.y, mi.y), x2_pack(q.z, q.x), x2_pack(q.w, q.y));
            }
        }
        __syncthreads();
        if (tid == 0 && blk + 2 < nblk) issue(blk + 2);
    }
    if (tid < N) {
        float sr, si, cr, ci;
        x2_unpack(s, sr, si);
        x2_unpack(c, cr, ci);
        out[tid] = make_double2((double)sr + (double)cr, (double)si + (double)ci);
    }
    // after a give-up the last copies may still be in flight: let them land (bounded) before the slots are reused
    if (tid == 0)
        for (int blk = nblk > 2 ? nblk - 2 : 0; blk < nblk; ++blk)
            for (long it = 0; it < TC_WAIT_LIMIT && !mbar_try(bar0 + 8 * (blk & 1), (blk >> 1) & 1); ++it) {
            }
    __syncthreads();
}

// out = b - S y for S = [[I, K], [K^+, I]] (two-centre overlap, FP64, column-major): only the
// off-diagonal blocks are read, rows i < N_T against columns j >= N_T and the other way round.
__device__ inline void residual_S(const double2* __restrict__ S, int N, int N_T, const double2* y, const double2* b,
                                  double2* out) {
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        double re = 0.0, im = 0.0;
        const int j0 = i < N_T ? N_T : 0, j1 = i < N_T ? N : N_T;
        const double2* row = S + i;
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            const double2 a = row[(size_t)j * N];
            const double2 q = y[j];
            re = fma(a.x, q.x, re);
            re = fma(-a.y, q.y, re);
            im = fma(a.x, q.y, im);
            im = fma(a.y, q.x, im);
        }
        out[i] = make_double2(b[i].x - y[i].x - re, b[i].y - y[i].y - im);
    }
    __syncthreads();
}

// k = -(i/v) S^{-1} (H y) with S given by its FP64 LU factors.  t: shared scratch of N.
static __device__ void apply_LU(const double2* __restrict__ LU, const int* __restrict__ piv,
                         const double2* __restrict__ Hm, int N, double v, const double2* y, double2* k,
                         double2* t, double2* blk) {
    matvec(Hm, N, y, t);
    lu_solve_inplace<double2>(LU, piv, N, t, blk);
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(t[i].y / v, -t[i].x / v);
    __syncthreads();
}

// Mixed-precision form: k = -(i/v) x with S x = H y solved by FP64 iterative refinement
// preconditioned by FP32 factors: x_0 = 0, r = H y - S x_n (FP64), x_{n+1} = x_n + (LU_32)^{-1} r; the
// last sweep's correction is checked against the solution (refine_check) when tol > 0.
// Shared scratch: b, x, r (double2) and d (float2), N each.
static __device__ void apply_LU_mixed(const double2* __restrict__ S64, const float2* __restrict__ LU32,
                               const int* __restrict__ piv, const double2* __restrict__ Hm, int N, int N_T, double v,
                               int iters, const double2* y, double2* k, double2* b, double2* x, double2* r,
                               float2* d, float2* blk, double tol = 0.0, int* flags = nullptr, bool df_rhs = false,
                               const Staging* sg = nullptr) {
    if (df_rhs && sg) matvec_df_staged(Hm, N, y, b, reinterpret_cast<float4*>(r), *sg, flags);
    else if (df_rhs) matvec_df(Hm, N, y, b, reinterpret_cast<float4*>(r));
    else matvec(Hm, N, y, b);
    for (int it = 0; it < iters; ++it) {
        const double2* rr = b;
        if (it > 0) {
            residual_S(S64, N, N_T, x, b, r);
            rr = r;
        }
        for (int i = threadIdx.x; i < N; i += RK_THREADS) d[i] = make_float2((float)rr[i].x, (float)rr[i].y);
        __syncthreads();
        lu_solve_inplace<float2>(LU32, piv, N, d, blk);
        double dm = 0.0, xm = 0.0;
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 dx = make_double2((double)d[i].x, (double)d[i].y);
            x[i] = it == 0 ? dx : make_double2(x[i].x + dx.x, x[i].y + dx.y);
            dm = fmax(dm, fmax(fabs(dx.x), fabs(dx.y)));
            xm = fmax(xm, fmax(fabs(x[i].x), fabs(x[i].y)));
        }
        __syncthreads();
        if (it > 0 && it == iters - 1 && tol > 0.0) refine_check(dm, xm, tol, flags);
    }
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(x[i].y / v, -x[i].x / v);
    __syncthreads();
}

// x <- C^{-1} x with C = L L^+ (L lower, real positive diagonal, column-major with leading dimension ld),
// n unknowns; C2 = double2 (FP64 factor) or float2 (FP32 factor of the mixed-precision form).  Blocked by
// 32 rows: the diagonal block is staged in shared memory (blk) and solved by one warp; off-diagonal
// updates: rows below (forward) by all threads, rows above (backward) a warp per row.
template <typename C2>
static __device__ void chol_solve_inplace(const C2* __restrict__ L, int ld, int n, C2* x, C2* blk) {
    using R = decltype(C2().x);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // L z = x
    for (int kb = 0; kb < n; kb += 32) {
        const int nb = min(32, n - kb);
        for (int q = tid; q < 32 * 32; q += RK_THREADS) {
            const int i = q & 31, j = q >> 5;
            if (i < nb && j < nb) blk[q] = L[(size_t)(kb + i) + (size_t)(kb + j) * ld];
        }
        __syncthreads();
        if (warp == 0) {
            C2 v = x[kb + (lane < nb ? lane : 0)];
            for (int j = 0; j < nb; ++j) {
                if (lane == j) {
                    const R d = R(1) / blk[j * 32 + j].x;
                    v.x *= d;
                    v.y *= d;
                }
                const R vr = __shfl_sync(0xffffffffu, v.x, j);
                const R vi = __shfl_sync(0xffffffffu, v.y, j);
                if (lane > j && lane < nb) {
                    const C2 l = blk[j * 32 + lane];
                    v.x = fma(-l.x, vr, v.x);
                    v.x = fma(l.y, vi, v.x);
                    v.y = fma(-l.x, vi, v.y);
                    v.y = fma(-l.y, vr, v.y);
                }
            }
            if (lane < nb) x[kb + lane] = v;
        }
        __syncthreads();
        for (int i = kb + nb + tid; i < n; i += RK_THREADS) {
            C2 a = x[i];
            for (int j = 0; j < nb; ++j) {
                const C2 l = L[(size_t)i + (size_t)(kb + j) * ld];
                const C2 b = x[kb + j];
                a.x = fma(-l.x, b.x, a.x);
                a.x = fma(l.y, b.y, a.x);
                a.y = fma(-l.x, b.y, a.y);
                a.y = fma(-l.y, b.x, a.y);
            }
            x[i] = a;
        }
        __syncthreads();
    }
    // L^+ x = z, from the bottom: (L^+)[i][j] = conj(L[j][i]), j >= i
    const int last = ((n - 1) / 32) * 32;
    for (int kb = last; kb >= 0; kb -= 32) {
        const int nb = min(32, n - kb);
        for (int q = tid; q < 32 * 32; q += RK_THREADS) {
            const int i = q & 31, j = q >> 5;
            if (i < nb && j < nb) blk[q] = L[(size_t)(kb + i) + (size_t)(kb + j) * ld];
        }
        __syncthreads();
        if (warp == 0) {
            C2 v = x[kb + (lane < nb ? lane : 0)];
            for (int j = nb - 1; j >= 0; --j) {
                if (lane == j) {
                    const R d = R(1) / blk[j * 32 + j].x;
                    v.x *= d;
                    v.y *= d;
                }
                const R vr = __shfl_sync(0xffffffffu, v.x, j);
                const R vi = __shfl_sync(0xffffffffu, v.y, j);
                if (lane < j) {
                    const C2 l = blk[lane * 32 + j];   // L[j][lane], conjugated below
                    v.x = fma(-l.x, vr, v.x);
                    v.x = fma(-l.y, vi, v.x);
                    v.y = fma(-l.x, vi, v.y);
                    v.y = fma(l.y, vr, v.y);
                }
            }
            if (lane < nb) x[kb + lane] = v;
        }
        __syncthreads();
        // rows i < kb: x_i -= sum_jj conj(L[kb + jj][i]) x[kb + jj], a warp per row, lanes over jj
        for (int i = warp; i < kb; i += RK_THREADS / 32) {
            R re = 0, im = 0;
            if (lane < nb) {
                const C2 l = L[(size_t)(kb + lane) + (size_t)i * ld];
                const C2 b = x[kb + lane];
                re = l.x * b.x + l.y * b.y;
                im = l.x * b.y - l.y * b.x;
            }
            for (int o = 16; o > 0; o >>= 1) {
                re += __shfl_xor_sync(0xffffffffu, re, o);
                im += __shfl_xor_sync(0xffffffffu, im, o);
            }
            if (lane == 0) {
                C2 q = x[i];
                q.x -= re;
                q.y -= im;
                x[i] = q;
            }
        }
        __syncthreads();
    }
}

// t <- S^{-1} t for S = [[I, K], [K^+, I]] held as K (rows 0..N_T-1 of columns N_T..N-1 of D) and the
// Cholesky factor L of the Schur complement I - K^+ K (lower triangle of D's projectile block), D
// column-major N x N:  u_P = t_P - K^+ t_T,  t_P = (L L^+)^{-1} u_P,  t_T = t_T - K t_P.
// u: shared scratch of N - N_T.  C2 = double2 (FP64) or float2 (FP32 preconditioner).
template <typename C2>
static __device__ void schur_solve_inplace(const C2* __restrict__ D, int N, int N_T, C2* t, C2* u, C2* blk) {
    using R = decltype(C2().x);
    const int NP = N - N_T, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const C2* K = D + (size_t)N_T * N;
    for (int j = warp; j < NP; j += RK_THREADS / 32) {
        R re = 0, im = 0;
        const C2* col = K + (size_t)j * N;
        for (int i = lane; i < N_T; i += 32) {
            const C2 a = col[i], b = t[i];
            re = fma(a.x, b.x, re);
            re = fma(a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(-a.y, b.x, im);
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_xor_sync(0xffffffffu, re, o);
            im += __shfl_xor_sync(0xffffffffu, im, o);
        }
        if (lane == 0) {
            C2 q = t[N_T + j];
            q.x -= re;
            q.y -= im;
            u[j] = q;
        }
    }
    __syncthreads();
    chol_solve_inplace<C2>(D + N_T + (size_t)N_T * N, N, NP, u, blk);
    for (int i = threadIdx.x; i < N_T; i += RK_THREADS) {
        R re = 0, im = 0;
#pragma unroll 4
        for (int j = 0; j < NP; ++j) {
            const C2 a = K[(size_t)i + (size_t)j * N];
            const C2 b = u[j];
            re = fma(a.x, b.x, re);
            re = fma(-a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(a.y, b.x, im);
        }
        C2 q = t[i];
        q.x -= re;
        q.y -= im;
        t[i] = q;
    }
    for (int j = threadIdx.x; j < NP; j += RK_THREADS) t[N_T + j] = u[j];
    __syncthreads();
}

// Schur form of the stage operator: k = -(i/v) S^{-1} (H y) with S's Schur factors in place of S
// (FP64).  t, u: shared scratch of N.
static __device__ void apply_schur(const double2* __restrict__ S, const double2* __restrict__ Hm, int N, int N_T,
                                   double v, const double2* y, double2* k, double2* t, double2* u, double2* blk) {
    matvec(Hm, N, y, t);
    schur_solve_inplace<double2>(S, N, N_T, t, u, blk);
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(t[i].y / v, -t[i].x / v);
    __syncthreads();
}

// Mixed-precision Schur form: k = -(i/v) x with S x = H y solved by FP64 iterative refinement
// preconditioned by the FP32 Schur factors D32 (K in FP32 and the FP32 Cholesky factor of I - K^+ K):
// x_0 = 0, r = H y - S x_n (FP64, S's off-diagonal blocks), x_{n+1} = x_n + S_32^{-1} r.
// Shared scratch: b, x, r (double2, N each), d (float2, N) and u (float2, N - N_T).
static __device__ void apply_schur_mixed(const double2* __restrict__ S64, const float2* __restrict__ D32,
                                         const double2* __restrict__ Hm, int N, int N_T, double v, int iters,
                                         const double2* y, double2* k, double2* b, double2* x, double2* r, float2* d,
                                         float2* u, float2* blk, double tol = 0.0, int* flags = nullptr,
                                         bool df_rhs = false, const Staging* sg = nullptr) {
    if (df_rhs && sg) matvec_df_staged(Hm, N, y, b, reinterpret_cast<float4*>(r), *sg, flags);
    else if (df_rhs) matvec_df(Hm, N, y, b, reinterpret_cast<float4*>(r));
    else matvec(Hm, N, y, b);
    for (int it = 0; it < iters; ++it) {
        const double2* rr = b;
        if (it > 0) {
            residual_S(S64, N, N_T, x, b, r);
            rr = r;
        }
        for (int i = threadIdx.x; i < N; i += RK_THREADS) d[i] = make_float2((float)rr[i].x, (float)rr[i].y);
        __syncthreads();
        schur_solve_inplace<float2>(D32, N, N_T, d, u, blk);
        double dm = 0.0, xm = 0.0;
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 dx = make_double2((double)d[i].x, (double)d[i].y);
            x[i] = it == 0 ? dx : make_double2(x[i].x + dx.x, x[i].y + dx.y);
            dm = fmax(dm, fmax(fabs(dx.x), fabs(dx.y)));
            xm = fmax(xm, fmax(fabs(x[i].x), fabs(x[i].y)));
        }
        __syncthreads();
        if (it > 0 && it == iters - 1 && tol > 0.0) refine_check(dm, xm, tol, flags);
    }
    for (int i = threadIdx.x; i < N; i += RK_THREADS) k[i] = make_double2(x[i].y / v, -x[i].x / v);
    __syncthreads();
}

}  // namespace wpccc
