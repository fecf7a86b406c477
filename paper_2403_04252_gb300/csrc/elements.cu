// Matrix-element assembly (Eq. 1, 6-9) for a batch of projectile positions.
//
// Two-centre pipeline per batch of positions (one "evaluation" = one (b, v, z)):
//   k_node_tables  per quadrature node (eta, tau): geometry, radial functions
//                  interpolated at r_T and r_P (5-point Lagrange, Sec. II),
//                  normalised Legendre functions at the two centres' cosines, and
//                  the complex node weights W_d = (R^3/8) w (eta^2-tau^2)
//                  exp(i v z eta tau/2) (-i)^d J_d(x) times 1 (overlap K) and -Z_T/r_T (transfer Q)
//   k_mol_gemm     molecular-frame integrals (Eq. 9) as a contraction over the
//                  nodes: X[i][c] = sum_g A_T[i][g] A_P[c][g] W_{|q_c - q'_i|}[g]
//                  for every target state i and projectile state c with q >= 0
//   k_rotate       Eq. 8 rotation to the collision frame (q < 0 columns from the
//                  q -> -q reflection), energy phases, writes the off-diagonal
//                  blocks of S and H
//   k_direct       Eq. 6 direct elements D_T and D_P (F of Eq. 7 interpolated at R),
//                  energy phases; identity diagonal blocks of S
//   k_direct_sr    (model-potential target only) the short-range part of the target
//                  potential between projectile states, on the (eta, tau) rule, added to D_P
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <vector>

#include <cuda_bf16.h>

#include "angular.cuh"
#include "geometry.cuh"
#include "ozaki.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

// Two-centre integrals per position: the overlap K and the transfer Q (Eq. 1); the lower-left
// block of H is Q^+, as Eq. 1 prints it, so no third integral is formed.
constexpr int NX = 2;

// ---------------------------------------------------------------------------
// Bessel functions of the first kind J_0(x) .. J_dmax(x), x >= 0, all orders from one pass:
//   x >= dmax       forward recurrence J_{n+1} = (2n/x) J_n - J_{n-1} from J_0, J_1 (stable while the
//                   order stays below the argument);
//   1e-5 <= x < dmax  Miller's backward recurrence (J. C. P. Miller; Abramowitz & Stegun 9.12): start
//                   from f_{M+1} = 0, f_M = 1 at an order M well above x and dmax, recur downwards with
//                   the same relation, rescale against overflow, and normalise by J_0 (or J_1 when that
//                   is larger, so a zero of J_0 costs no accuracy);
//   x < 1e-5        the first two terms of the power series, (x/2)^n/n! (1 - (x/2)^2/(n+1)).
// J_0 and J_1 come from CUDA's j0 and j1.
// ---------------------------------------------------------------------------
constexpr int BESSEL_MAX = 2 * WPCCC_LMAX;

__device__ inline void bessel_j_orders(int dmax, double x, double* J) {
    if (x < 1e-5) {
        const double h = 0.5 * x;
        double t = 1.0;
        for (int n = 0; n <= dmax; ++n) {
            J[n] = t * (1.0 - h * h / (n + 1));
            t *= h / (n + 1);
        }
        return;
    }
    const double j0v = j0(x), j1v = j1(x);
    if (x >= (double)dmax) {
        J[0] = j0v;
        if (dmax >= 1) J[1] = j1v;
        const double ix2 = 2.0 / x;
        for (int n = 1; n < dmax; ++n) J[n + 1] = (n * ix2) * J[n] - J[n - 1];
        return;
    }
    const int M = dmax + 26 + (int)x;
    const double ix2 = 2.0 / x;
    double fn1 = 0.0, fn = 1.0;   // f_{n+1}, f_n
    for (int n = M; n >= 1; --n) {
        const double fm = (n * ix2) * fn - fn1;   // f_{n-1}
        fn1 = fn;
        fn = fm;
        if (n - 1 <= dmax) J[n - 1] = fm;
        if (fabs(fn) > 1e200) {
            fn *= 1e-200;
            fn1 *= 1e-200;
            for (int k = n - 1; k <= dmax; ++k) J[k] *= 1e-200;
        }
    }
    const double scale = fabs(j0v) >= fabs(j1v) ? j0v / J[0] : j1v / J[1];
    for (int n = 0; n <= dmax; ++n) J[n] *= scale;
}

// ---------------------------------------------------------------------------
// k_node_tables
// ---------------------------------------------------------------------------
struct NodeArgs {
    int Nr, G, Gtau, nradT, nradP, lmaxT, lmaxP, nlqT, nlqP, dmax;
    double gamma, Z_T, Z_P;
    double mp_c, mp_a, mp_b;   // short-range part of a model-potential target (mp_c = 0: bare nucleus)
    const double *r, *fT, *fP, *s, *ws, *tau, *wtau;
    const float2 *fT2, *fP2;   // the radial tables as double-floats (tensor-core layout)
    const double* inv_den;   // Lagrange denominators per stencil start
    double* node;            // per evaluation: [fT | fP | thT | thP | pad | W] (see elem_scratch_layout)
    size_t node_doubles;     // stride between evaluations, in doubles
    size_t w_off;            // offset of W in elements of the table type (even, so W stays aligned)
    // T = float: per-state products instead of per-radial values (one rounding of f * Theta * sign)
    int N_T, n_half;
    const int *stT_index, *half_of, *radT_l, *radP_l;
    // tensor-core layout (T = float, precision modes 3-5): bf16 slice planes of A_T r_T and A_T r_T V_T
    // (tc_slices of them: OZ_FAST_SLICES for the reduced-precision form, 7 for FP64 accuracy) with scales per
    // 128-node window, and
    // A_P and W_K / r_T as double-floats
    int tc, tc_slices;
    const int* tc_row;          // [2 N_T]: row of each target state in the slice planes, then its tile's size
    int tc_rows;
    size_t t6_ap_off, t6_w_off, t6_sc_off;
    // sqrt((2l+1)/2 (l-q)!/(l+q)!) at l(l+1)/2 + q, and 1/k for k = 0..WPCCC_LMAX (entry 0 unused): the
    // Legendre recurrence's constants, formed once on the host instead of per node
    double th_nrm[(WPCCC_LMAX + 1) * (WPCCC_LMAX + 2) / 2];
    double inv_int[WPCCC_LMAX + 1];
};

// Radial functions of the tensor-core layout's target rows processed per shared-memory batch.
constexpr int TC_NA = 16;

// Normalised Legendre functions Theta_lq(c) = sqrt((2l+1)/2 (l-q)!/(l+q)!) P_l^q(c) (Condon-Shortley phase)
// for 0 <= q <= l <= lmax, by the upward recurrence in l at fixed q, handed to put(l (l+1)/2 + q, value).
template <typename F>
__device__ inline void theta_lq(double c, int lmax, const NodeArgs& A, F put) {
    const double sq = sqrt((1.0 - c) * (1.0 + c));
    double pmm = 1.0;   // P_q^q, built up from P_0^0 = 1
    for (int q = 0; q <= lmax; ++q) {
        if (q > 0) pmm *= -(2.0 * q - 1.0) * sq;
        double pa = 0.0, pb = pmm;   // P_{l-2}^q, P_{l-1}^q
        for (int l = q; l <= lmax; ++l) {
            double pl;
            if (l == q) pl = pmm;
            else if (l == q + 1) pl = c * (2.0 * q + 1.0) * pmm;
            else pl = (c * (2.0 * l - 1.0) * pb - (l + q - 1.0) * pa) * A.inv_int[l - q];
            if (l > q) {
                pa = pb;
                pb = pl;
            }
            const int t = l * (l + 1) / 2 + q;
            put(t, A.th_nrm[t] * pl);
        }
    }
}

template <typename T> struct Vec2;
template <> struct Vec2<double> { using type = double2; };
template <> struct Vec2<float> { using type = float2; };

// The per-node factors are computed in FP64; T = double keeps them in FP64, T = float (mixed-precision
// form) stores them rounded to FP32 for the FP32 contraction.  In the tensor-core layout a block is one
// 128-node scaling window and needs dynamic shared memory (see node_tables_smem).
template <typename T>
__global__ void __launch_bounds__(128) k_node_tables(NodeArgs A, const EvalDesc* __restrict__ ev) {
    using T2 = typename Vec2<T>::type;
    const int e = blockIdx.y;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= A.G) return;
    const int k = g / A.Gtau, t = g - k * A.Gtau;
    const double b = ev[e].b, v = ev[e].v, z = ev[e].z;
    const double R = dist_R(b, z);
    const double gR = __dmul_rn(A.gamma, R);
    const double eta = __dadd_rn(1.0, __ddiv_rn(A.s[k], gR));
    const double tau = A.tau[t];
    const double halfR = __dmul_rn(0.5, R);
    const double rT = __dmul_rn(halfR, __dadd_rn(eta, tau));
    const double rP = __dmul_rn(halfR, __dsub_rn(eta, tau));
    const double cT = (eta * tau + 1.0) / (eta + tau);
    const double cP = (eta * tau - 1.0) / (eta - tau);
    const double x = 0.5 * v * b * sqrt((eta * eta - 1.0) * (1.0 - tau * tau));
    const double wgt = (A.ws[k] / gR) * A.wtau[t];
    const double amp = (R * R * R / 8.0) * wgt * (eta * eta - tau * tau);
    double sph, cph;
    sincos(0.5 * v * z * eta * tau, &sph, &cph);

    T* base = reinterpret_cast<T*>(A.node + (size_t)e * A.node_doubles);
    T* oT = base;
    T* oP = oT + (size_t)A.nradT * A.G;
    T* thT = oP + (size_t)A.nradP * A.G;
    T* thP = thT + (size_t)A.nlqT * A.G;
    T2* W = reinterpret_cast<T2*>(base + A.w_off);

    // radial functions at the node radii
    int sT, sP;
    double LT[5], LP[5];
    const bool inT = stencil5_fast(A.r, A.inv_den, A.Nr, rT, sT, LT);
    const bool inP = stencil5_fast(A.r, A.inv_den, A.Nr, rP, sP, LP);
    auto interp = [&](const double* f, int a, bool in, int st, const double* Lw) {
        if (!in) return 0.0;
        const double* fa = f + (size_t)a * A.Nr + st;
        return Lw[0] * fa[0] + Lw[1] * fa[1] + Lw[2] * fa[2] + Lw[3] * fa[3] + Lw[4] * fa[4];
    };
    if (sizeof(T) == 8) {
        for (int a = 0; a < A.nradT; ++a) oT[(size_t)a * A.G + g] = (T)interp(A.fT, a, inT, sT, LT);
        for (int a = 0; a < A.nradP; ++a) oP[(size_t)a * A.G + g] = (T)interp(A.fP, a, inP, sP, LP);
        // Theta_lq(c) = sqrt((2l+1)/2 (l-q)!/(l+q)!) P_l^q(c), index l(l+1)/2 + q
        theta_lq(cT, A.lmaxT, A, [&](int q, double val) { thT[(size_t)q * A.G + g] = (T)val; });
        theta_lq(cP, A.lmaxP, A, [&](int q, double val) { thP[(size_t)q * A.G + g] = (T)val; });
    } else if (A.tc) {
        // tensor-core layout: A_T r_T and A_T r_T V_T per target state (rows of the row tiles), each as
        // tc_slices bf16 slices against a power-of-two scale per 128-node window (this block); the
        // products are formed in double-float arithmetic from FP64 factors split once per node.
        // Shared memory: th [nlq][128] (this thread's column only while it builds A_P from the projectile's
        // Theta, then the target's Theta for every warp), r [2][128] (r_T, r_T V_T), f [TC_NA][128]
        // (a batch of target radial functions at the window's nodes).
        extern __shared__ float2 s_tc[];
        // the 5-point interpolation in double-float arithmetic on the FP32 pipe (the FP64 pipe is two
        // operations per clock per SM on this part): Lagrange weights split once per node, tables stored
        // split; each term's product is exact in its high parts (FMA residual) and the sum a TwoSum chain
        float2 LT2[5], LP2[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            LT2[k] = df_split(LT[k]);
            LP2[k] = df_split(LP[k]);
        }
        auto interp2 = [&](const float2* f2, int a, bool in, int st, const float2* Lw) {
            if (!in) return make_float2(0.f, 0.f);
            const float2* fa = f2 + (size_t)a * A.Nr + st;
            float hi = 0.f, lo = 0.f;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float2 v = fa[k];
                const float p = Lw[k].x * v.x;
                float e = fmaf(Lw[k].x, v.x, -p);
                e = fmaf(Lw[k].x, v.y, e);
                e = fmaf(Lw[k].y, v.x, e);
                float r;
                hi = two_sum(hi, p, r);
                lo += r + e;
            }
            const float s = hi + lo;
            return make_float2(s, lo - (s - hi));
        };
        const int nlq = A.nlqT > A.nlqP ? A.nlqT : A.nlqP;
        float2* s_th = s_tc;
        float2* s_r = s_th + (size_t)nlq * 128;
        float2* s_f = s_r + 2 * 128;
        const int tx = threadIdx.x, wid = tx >> 5, lid = tx & 31;
        // A_P per half column as double-floats
        theta_lq(cP, A.lmaxP, A, [&](int q, double val) { s_th[q * 128 + tx] = df_split(val); });
        float2* aP = reinterpret_cast<float2*>(reinterpret_cast<float*>(base) + A.t6_ap_off);
        for (int b2 = 0; b2 < A.nradP; ++b2) {
            const float2 fv = interp2(A.fP2, b2, inP, sP, LP2);
            const int l = A.radP_l[b2];
            for (int q = 0; q <= l; ++q) {
                const int j = A.half_of[b2 * (WPCCC_LMAX + 1) + q];
                aP[(size_t)j * A.G + g] = df_mul(fv, s_th[(l * (l + 1) / 2 + q) * 128 + tx]);
            }
        }
        theta_lq(cT, A.lmaxT, A, [&](int q, double val) { s_th[q * 128 + tx] = df_split(val); });
        const double rTV = A.mp_c == 0.0 ? -A.Z_T : -A.Z_T + (-A.mp_c * exp(-A.mp_a * rT)) * (1.0 + A.mp_b * rT);
        s_r[tx] = df_split(rT);
        s_r[128 + tx] = df_split(rTV);
        __nv_bfloat16* sp = reinterpret_cast<__nv_bfloat16*>(base);
        float* sc = reinterpret_cast<float*>(base) + A.t6_sc_off + (size_t)blockIdx.x * A.tc_rows;
        const size_t split = (size_t)A.tc_rows * A.G;
        const int g0 = blockIdx.x * 128;
        // one row of the slice planes at the window's 128 nodes: lane holds nodes lid + 32 j
        auto put_row = [&](size_t row, const float2* xv, float mx) {
            const int sh = oz_shift(mx);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                __nv_bfloat16 q[OZ_SLICES];
                const size_t o = row * A.G + g0 + lid + 32 * j;
                if (A.tc_slices == OZ_FAST_SLICES) {
                    oz_slices<OZ_FAST_SLICES>(xv[j].x, xv[j].y, sh, q);
#pragma unroll
                    for (int i = 0; i < OZ_FAST_SLICES; ++i) sp[i * split + o] = q[i];
                } else {
                    oz_slices<OZ_SLICES>(xv[j].x, xv[j].y, sh, q);
#pragma unroll
                    for (int i = 0; i < OZ_SLICES; ++i) sp[i * split + o] = q[i];
                }
            }
            if (lid == 0) sc[row] = ldexpf(1.f, -sh);
        };
        for (int a0 = 0; a0 < A.nradT; a0 += TC_NA) {
            const int na = A.nradT - a0 < TC_NA ? A.nradT - a0 : TC_NA;
            __syncthreads();   // the previous batch's rows are written (and, first time, Theta_T and r are in)
            for (int j = 0; j < na; ++j) s_f[j * 128 + tx] = interp2(A.fT2, a0 + j, inT, sT, LT2);
            __syncthreads();
            // the batch's states, one per warp in turn: (radial function, m) pairs in order
            int pair = 0;
            for (int j = 0; j < na; ++j) {
                const int a = a0 + j, l = A.radT_l[a];
                for (int m = -l; m <= l; ++m, ++pair) {
                    if ((pair & 3) != wid) continue;
                    const int i = A.stT_index[a * (2 * WPCCC_LMAX + 1) + m + WPCCC_LMAX];
                    const int am = m < 0 ? -m : m;
                    const bool neg = m < 0 && (am & 1);
                    const float2* th = s_th + (l * (l + 1) / 2 + am) * 128;
                    float2 x1[4], x2[4];
                    float m1 = 0.f, m2 = 0.f;
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) {
                        const int n = lid + 32 * jj;
                        float2 tv = df_mul(s_f[j * 128 + n], th[n]);
                        if (neg) tv = make_float2(-tv.x, -tv.y);
                        x1[jj] = df_mul(tv, s_r[n]);
                        x2[jj] = df_mul(tv, s_r[128 + n]);
                        m1 = fmaxf(m1, fabsf(x1[jj].x));
                        m2 = fmaxf(m2, fabsf(x2[jj].x));
                    }
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        m1 = fmaxf(m1, __shfl_xor_sync(0xffffffffu, m1, o));
                        m2 = fmaxf(m2, __shfl_xor_sync(0xffffffffu, m2, o));
                    }
                    const int row = A.tc_row[i];
                    const int tsz = A.tc_row[A.N_T + i];
                    put_row((size_t)row, x1, m1);
                    put_row((size_t)(row + tsz), x2, m2);
                }
            }
        }
    } else {
        // per state: A_T[i][g] = f_a(r_T) Theta_{l|m|}(c_T) (-1)^m [m < 0], A_P[j][g] = f_b(r_P) Theta_{lq}(c_P)
        double thv[(WPCCC_LMAX + 1) * (WPCCC_LMAX + 2) / 2];
        T* aT = base;
        T* aP = aT + (size_t)A.N_T * A.G;
        theta_lq(cT, A.lmaxT, A, [&](int q, double val) { thv[q] = val; });
        for (int a = 0; a < A.nradT; ++a) {
            const double val = interp(A.fT, a, inT, sT, LT);
            const int l = A.radT_l[a];
            for (int m = -l; m <= l; ++m) {
                const int i = A.stT_index[a * (2 * WPCCC_LMAX + 1) + m + WPCCC_LMAX];
                const int am = m < 0 ? -m : m;
                const double sg = (m < 0 && (am & 1)) ? -1.0 : 1.0;
                aT[(size_t)i * A.G + g] = (T)(val * thv[l * (l + 1) / 2 + am] * sg);
            }
        }
        theta_lq(cP, A.lmaxP, A, [&](int q, double val) { thv[q] = val; });
        for (int b2 = 0; b2 < A.nradP; ++b2) {
            const double val = interp(A.fP, b2, inP, sP, LP);
            const int l = A.radP_l[b2];
            for (int q = 0; q <= l; ++q) {
                const int j = A.half_of[b2 * (WPCCC_LMAX + 1) + q];
                aP[(size_t)j * A.G + g] = (T)(val * thv[l * (l + 1) / 2 + q]);
            }
        }
    }
    // node weights for the two integrands, d = |q - q'| = 0..dmax; Q carries the target potential
    const double irT = 1.0 / rT;
    const double uQ = A.mp_c == 0.0 ? -A.Z_T * irT
                                    : (-A.Z_T + (-A.mp_c * exp(-A.mp_a * rT)) * (1.0 + A.mp_b * rT)) * irT;
    const size_t stride = (size_t)(A.dmax + 1) * A.G;
    double Jd[BESSEL_MAX + 1];
    bessel_j_orders(A.dmax, x, Jd);
    for (int d = 0; d <= A.dmax; ++d) {
        const double J = Jd[d] * amp;
        // (-i)^d exp(i phi)
        double re, im;
        switch (d & 3) {
            case 0: re = cph; im = sph; break;
            case 1: re = sph; im = -cph; break;
            case 2: re = -cph; im = -sph; break;
            default: re = -sph; im = cph; break;
        }
        const double2 w0 = make_double2(J * re, J * im);
        const size_t o = (size_t)d * A.G + g;
        if (sizeof(T) == 4 && A.tc) {
            // tensor-core layout: W_K / r_T as double-floats, [d][re, im][G] (r_T and the transfer
            // potential sit in the slice planes)
            float2* w6 = reinterpret_cast<float2*>(reinterpret_cast<float*>(base) + A.t6_w_off);
            w6[((size_t)d * 2) * A.G + g] = df_split(w0.x * irT);
            w6[((size_t)d * 2 + 1) * A.G + g] = df_split(w0.y * irT);
        } else {
            T2 a, bq;
            a.x = (T)w0.x;
            a.y = (T)w0.y;
            bq.x = (T)(w0.x * uQ);
            bq.y = (T)(w0.y * uQ);
            W[o] = a;
            W[stride + o] = bq;
        }
    }
}

// Dynamic shared memory of k_node_tables: the tensor-core layout's per-window tables, else none.
static size_t node_tables_smem(const wpccc_basis_s* B, bool tc) {
    if (!tc) return 0;
    const int nlq = std::max(B->nlq_T, B->nlq_P);
    return (size_t)(nlq + 2 + TC_NA) * 128 * sizeof(float2);
}

// ---------------------------------------------------------------------------
// k_mol_gemm: Eq. 9 contraction over the quadrature nodes (FP64)
// ---------------------------------------------------------------------------
constexpr int GT_I = 32, GT_J = 32, GT_K = 32;

struct GemmArgs {
    int G, N_T, n_half, nradT, nradP, nlqT, nlqP, dmax, n_col_tiles;
    const int *stT_rad, *stT_l, *stT_m;   // target states
    const int *stP_rad, *stP_l, *stP_m;   // projectile states
    const int* half_state;
    const double* node;
    size_t node_doubles, w_off;
    double2* mol;                         // [nev][NX][N_T][n_half]
};

template <typename R> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

// R = double: FP64 throughout.  R = float (mixed-precision form): node values are rounded to FP32 in
// shared memory, products and sums run on the FP32 pipe, with the sum over each chunk of GT_K nodes
// formed separately and then added to the running total (two-level summation).
template <typename R>
__global__ void __launch_bounds__(256) k_mol_gemm(GemmArgs A) {
    using R2 = typename Cplx<R>::type;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* sAT = reinterpret_cast<R*>(smem_raw);                      // [GT_K][GT_I + 1]
    R* sAP = sAT + GT_K * (GT_I + 1);                             // [GT_K][GT_J + 1]
    R2* sW = reinterpret_cast<R2*>(sAP + GT_K * (GT_J + 1));      // [NX][dmax+1][GT_K]
    __shared__ int s_rrad[GT_I], s_rlq[GT_I], s_rq[GT_I];
    __shared__ R s_rsgn[GT_I];
    __shared__ int s_crad[GT_J], s_clq[GT_J], s_cq[GT_J];

    const int e = blockIdx.y;
    const int rt = blockIdx.x / A.n_col_tiles, ct = blockIdx.x % A.n_col_tiles;
    const int i0 = rt * GT_I, j0 = ct * GT_J;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const R* base = reinterpret_cast<const R*>(A.node + (size_t)e * A.node_doubles);
    const R* fT = base;
    const R* fP = fT + (size_t)A.nradT * A.G;
    const R* thT = fP + (size_t)A.nradP * A.G;
    const R* thP = thT + (size_t)A.nlqT * A.G;
    const R2* W = reinterpret_cast<const R2*>(base + A.w_off);

    if (tid < GT_I) {
        int i = i0 + tid;
        if (i < A.N_T) {
            int l = A.stT_l[i], m = A.stT_m[i], am = m < 0 ? -m : m;
            s_rrad[tid] = A.stT_rad[i];
            s_rlq[tid] = l * (l + 1) / 2 + am;
            s_rq[tid] = m;
            s_rsgn[tid] = (m < 0 && (am & 1)) ? R(-1) : R(1);   // Theta_{l,-q} = (-1)^q Theta_{l,q}
        } else {
            s_rrad[tid] = -1;
            s_rlq[tid] = 0;
            s_rq[tid] = 0;
            s_rsgn[tid] = R(0);
        }
    } else if (tid < GT_I + GT_J) {
        int c = tid - GT_I, j = j0 + c;
        if (j < A.n_half) {
            int st = A.half_state[j];
            int l = A.stP_l[st], q = A.stP_m[st];
            s_crad[c] = A.stP_rad[st];
            s_clq[c] = l * (l + 1) / 2 + q;
            s_cq[c] = q;
        } else {
            s_crad[c] = -1;
            s_clq[c] = 0;
            s_cq[c] = 0;
        }
    }
    __syncthreads();

    int dd[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int d = s_cq[tx * 2 + c] - s_rq[ty * 2 + a];
            dd[a][c] = d < 0 ? -d : d;
        }
    R acc[2][2][2 * NX], tot[2][2][2 * NX];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int q = 0; q < 2 * NX; ++q) {
                acc[a][c][q] = R(0);
                tot[a][c][q] = R(0);
            }

    const int nd = A.dmax + 1;
    const size_t wstride = (size_t)nd * A.G;
    for (int g0 = 0; g0 < A.G; g0 += GT_K) {
        // A_T[i][g] = f_a(r_T) Theta_{l|q'|}(c_T) * sign, transposed into sAT[g][i]
        if (sizeof(R) == 8) {
            for (int idx = tid; idx < GT_I * GT_K; idx += 256) {
                int ii = idx / GT_K, gg = idx % GT_K, g = g0 + gg;
                R val = R(0);
                if (s_rrad[ii] >= 0 && g < A.G)
                    val = fT[(size_t)s_rrad[ii] * A.G + g] * thT[(size_t)s_rlq[ii] * A.G + g] * s_rsgn[ii];
                sAT[gg * (GT_I + 1) + ii] = val;
            }
            for (int idx = tid; idx < GT_J * GT_K; idx += 256) {
                int cc = idx / GT_K, gg = idx % GT_K, g = g0 + gg;
                R val = R(0);
                if (s_crad[cc] >= 0 && g < A.G)
                    val = fP[(size_t)s_crad[cc] * A.G + g] * thP[(size_t)s_clq[cc] * A.G + g];
                sAP[gg * (GT_J + 1) + cc] = val;
            }
        } else {
            // mixed-precision form: per-state products from k_node_tables<float>
            const R* aT = base;
            const R* aP = aT + (size_t)A.N_T * A.G;
            for (int idx = tid; idx < GT_I * GT_K; idx += 256) {
                int ii = idx / GT_K, gg = idx % GT_K, g = g0 + gg;
                sAT[gg * (GT_I + 1) + ii] = (s_rrad[ii] >= 0 && g < A.G) ? aT[(size_t)(i0 + ii) * A.G + g] : R(0);
            }
            for (int idx = tid; idx < GT_J * GT_K; idx += 256) {
                int cc = idx / GT_K, gg = idx % GT_K, g = g0 + gg;
                sAP[gg * (GT_J + 1) + cc] = (s_crad[cc] >= 0 && g < A.G) ? aP[(size_t)(j0 + cc) * A.G + g] : R(0);
            }
        }
        for (int idx = tid; idx < NX * nd * GT_K; idx += 256) {
            int gg = idx % GT_K, xd = idx / GT_K, g = g0 + gg;
            int X = xd / nd, d = xd % nd;
            R2 wr;
            if (g < A.G) {
                wr = W[(size_t)X * wstride + (size_t)d * A.G + g];
            } else {
                wr.x = R(0);
                wr.y = R(0);
            }
            sW[idx] = wr;
        }
        __syncthreads();
#pragma unroll 4
        for (int gg = 0; gg < GT_K; ++gg) {
            R at[2], ap[2];
            at[0] = sAT[gg * (GT_I + 1) + ty * 2];
            at[1] = sAT[gg * (GT_I + 1) + ty * 2 + 1];
            ap[0] = sAP[gg * (GT_J + 1) + tx * 2];
            ap[1] = sAP[gg * (GT_J + 1) + tx * 2 + 1];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const R p = at[a] * ap[c];
                    const R2* wp = sW + dd[a][c] * GT_K + gg;
                    const R2 w0 = wp[0], w1 = wp[nd * GT_K];
                    acc[a][c][0] = fma(p, w0.x, acc[a][c][0]);
                    acc[a][c][1] = fma(p, w0.y, acc[a][c][1]);
                    acc[a][c][2] = fma(p, w1.x, acc[a][c][2]);
                    acc[a][c][3] = fma(p, w1.y, acc[a][c][3]);
                }
        }
        if (sizeof(R) == 4) {
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int c = 0; c < 2; ++c)
#pragma unroll
                    for (int q = 0; q < 2 * NX; ++q) {
                        tot[a][c][q] += acc[a][c][q];
                        acc[a][c][q] = R(0);
                    }
        }
        __syncthreads();
    }
    if (sizeof(R) == 8) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int c = 0; c < 2; ++c)
#pragma unroll
                for (int q = 0; q < 2 * NX; ++q) tot[a][c][q] = acc[a][c][q];
    }
    const size_t plane = (size_t)A.N_T * A.n_half;
    double2* out = A.mol + (size_t)e * NX * plane;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        int i = i0 + ty * 2 + a;
        if (i >= A.N_T) continue;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            int j = j0 + tx * 2 + c;
            if (j >= A.n_half) continue;
            size_t o = (size_t)i * A.n_half + j;
            out[o] = make_double2(tot[a][c][0], tot[a][c][1]);
            out[plane + o] = make_double2(tot[a][c][2], tot[a][c][3]);
        }
    }
}

// ---------------------------------------------------------------------------
// k_mol_gemm_f32q: the FP32 contraction of the mixed-precision form with column tiles of one q.
// All columns of a tile share q, so row i needs the single weight W_{|q - q'_i|}: the row operand is
// pre-multiplied by it once per node, B_x[i][g] = A_T[i][g] W_x[d_i][g] (x = three complex integrands),
// and the inner loop is a plain 6-accumulator product with the column operand A_P[j][g].
// Sums run per chunk of QT_K nodes and are then added to the running totals by compensated summation.
// ---------------------------------------------------------------------------
constexpr int QT_I = 32, QT_J = 16, QT_K = 32, QT_THREADS = 64;   // 8 x 4 thread grid per warp pair
constexpr int QT_AS = QT_K + 4;   // row stride of the staged row operand (16-byte rows, distinct banks)

struct Gemm32Args {
    int G, N_T, n_half, dmax, n_col_tiles;
    const int* stT_m;
    const int* ctile_q;       // [n_col_tiles]
    const int* ctile_cols;    // [n_col_tiles][QT_J] half columns (-1: padding)
    const double* node;
    size_t node_doubles, w_off_f;
    double2* mol;
};

__device__ inline void cp_async4(void* sdst, const void* gsrc, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 4 : 0));
}
__device__ inline void cp_async8(void* sdst, const void* gsrc, bool valid) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(gsrc), "r"(valid ? 8 : 0));
}
__device__ inline void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gsrc));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(QT_THREADS) k_mol_gemm_f32q(Gemm32Args A) {
    extern __shared__ __align__(16) float qsm[];
    const int nd = A.dmax + 1;
    float* sA = qsm;                                   // [2][QT_I][QT_AS]   row operand A_T
    float* sP = sA + 2 * QT_I * QT_AS;                 // [2][QT_K][QT_J]    column operand A_P
    float2* sW = reinterpret_cast<float2*>(sP + 2 * QT_K * QT_J);   // [2][NX][nd][QT_K] weights
    __shared__ int s_d[QT_I], s_col[QT_J];
    const int e = blockIdx.y;
    const int rt = blockIdx.x / A.n_col_tiles, ct = blockIdx.x % A.n_col_tiles;
    const int i0 = rt * QT_I;
    const int tid = threadIdx.x, tx = tid & 3, ty = tid >> 2;
    const int q = A.ctile_q[ct];
    const float* base = reinterpret_cast<const float*>(A.node + (size_t)e * A.node_doubles);
    const float* aT = base;
    const float* aP = aT + (size_t)A.N_T * A.G;
    const float2* W = reinterpret_cast<const float2*>(base + A.w_off_f);
    const size_t wstride = (size_t)nd * A.G;
    for (int r = tid; r < QT_I; r += QT_THREADS) {
        const int i = i0 + r;
        int d = -1;
        if (i < A.N_T) {
            d = q - A.stT_m[i];
            d = d < 0 ? -d : d;
        }
        s_d[r] = d;
    }
    for (int c = tid; c < QT_J; c += QT_THREADS) s_col[c] = A.ctile_cols[ct * QT_J + c];
    __syncthreads();
    const bool vec = (A.G & 3) == 0;
    auto stage = [&](int buf, int g0) {
        float* a = sA + buf * QT_I * QT_AS;
        for (int t = tid; t < QT_I * (QT_K / 4); t += QT_THREADS) {
            const int r = t / (QT_K / 4), k4 = (t % (QT_K / 4)) * 4, g = g0 + k4;
            const bool rv = s_d[r] >= 0;
            const float* src = aT + (size_t)(rv ? i0 + r : 0) * A.G;
            if (vec && rv && g + 3 < A.G) {
                cp_async16(a + r * QT_AS + k4, src + g);
            } else {
                for (int u = 0; u < 4; ++u) {
                    const bool ok = rv && g + u < A.G;
                    cp_async4(a + r * QT_AS + k4 + u, ok ? src + g + u : aT, ok);
                }
            }
        }
        float* p = sP + buf * QT_K * QT_J;
        for (int t = tid; t < QT_K * QT_J; t += QT_THREADS) {
            const int c = t / QT_K, k = t % QT_K, g = g0 + k;
            const int j = s_col[c];
            const bool ok = j >= 0 && g < A.G;
            cp_async4(p + k * QT_J + c, ok ? aP + (size_t)j * A.G + g : aP, ok);
        }
        float2* w = sW + (size_t)buf * NX * nd * QT_K;
        for (int t = tid; t < NX * nd * QT_K; t += QT_THREADS) {
            const int k = t % QT_K, xd = t / QT_K, g = g0 + k;
            const int x = xd / nd, d = xd % nd;
            const bool ok = g < A.G;
            cp_async8(w + t, ok ? W + (size_t)x * wstride + (size_t)d * A.G + g : W, ok);
        }
        cp_async_commit();
    };

    // chunk sums in FP32; running totals as compensated (Kahan) FP32 sums of the chunk sums, whose
    // rounding error does not grow with the number of chunks
    float acc[2][4][2 * NX], tot[2][4][2 * NX], cmp[2][4][2 * NX];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int x = 0; x < 2 * NX; ++x) {
                acc[a][c][x] = 0.f;
                tot[a][c][x] = 0.f;
                cmp[a][c][x] = 0.f;
            }
    const int r0 = ty * 2;
    const int d0 = s_d[r0] < 0 ? 0 : s_d[r0], d1 = s_d[r0 + 1] < 0 ? 0 : s_d[r0 + 1];
    const int nchunks = (A.G + QT_K - 1) / QT_K;
    stage(0, 0);
    for (int kc = 0; kc < nchunks; ++kc) {
        const int buf = kc & 1;
        if (kc + 1 < nchunks) {
            stage(buf ^ 1, (kc + 1) * QT_K);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const float* a = sA + buf * QT_I * QT_AS;
        const float* p = sP + buf * QT_K * QT_J;
        const float2* w = sW + (size_t)buf * NX * nd * QT_K;
#pragma unroll 4
        for (int gg = 0; gg < QT_K; ++gg) {
            const float4 pv = *reinterpret_cast<const float4*>(p + gg * QT_J + tx * 4);
            const float pc[4] = {pv.x, pv.y, pv.z, pv.w};
            float bv[2][2 * NX];
#pragma unroll
            for (int rr = 0; rr < 2; ++rr) {
                const int d = rr == 0 ? d0 : d1;
                const float at = a[(r0 + rr) * QT_AS + gg];
                const float2 w0 = w[d * QT_K + gg];
                const float2 w1 = w[(nd + d) * QT_K + gg];
                bv[rr][0] = at * w0.x;
                bv[rr][1] = at * w0.y;
                bv[rr][2] = at * w1.x;
                bv[rr][3] = at * w1.y;
            }
#pragma unroll
            for (int rr = 0; rr < 2; ++rr)
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                    for (int x = 0; x < 2 * NX; ++x) acc[rr][c][x] = fmaf(bv[rr][x], pc[c], acc[rr][c][x]);
        }
#pragma unroll
        for (int rr = 0; rr < 2; ++rr)
#pragma unroll
            for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int x = 0; x < 2 * NX; ++x) {
                    const float y = __fsub_rn(acc[rr][c][x], cmp[rr][c][x]);
                    const float t = __fadd_rn(tot[rr][c][x], y);
                    cmp[rr][c][x] = __fsub_rn(__fsub_rn(t, tot[rr][c][x]), y);
                    tot[rr][c][x] = t;
                    acc[rr][c][x] = 0.f;
                }
        __syncthreads();
    }
    const size_t plane = (size_t)A.N_T * A.n_half;
    double2* out = A.mol + (size_t)e * NX * plane;
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
        const int i = i0 + r0 + rr;
        if (i >= A.N_T) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int j = s_col[tx * 4 + c];
            if (j < 0) continue;
            const size_t o = (size_t)i * A.n_half + j;
            out[o] = make_double2((double)tot[rr][c][0] - (double)cmp[rr][c][0],
                                  (double)tot[rr][c][1] - (double)cmp[rr][c][1]);
            out[plane + o] = make_double2((double)tot[rr][c][2] - (double)cmp[rr][c][2],
                                          (double)tot[rr][c][3] - (double)cmp[rr][c][3]);
        }
    }
}

size_t mol_gemm_f32q_smem(int dmax) {
    return sizeof(float) * (2 * QT_I * QT_AS + 2 * QT_K * QT_J) + sizeof(float2) * 2 * NX * (dmax + 1) * QT_K;
}

// ---------------------------------------------------------------------------
// k_eval_tables: the small per-position tables shared by k_rotate and k_direct:
//   Wigner d^l_{m q}(theta) for l <= lrot      at [off_l + (m + l)(2l+1) + (q + l)]
//   Pbar(lam, mu) = sqrt((lam-mu)!/(lam+mu)!) P_lam^mu(cos Theta), lam < nlam, at dtot + lam(lam+1)/2 + mu
//   the 5-point stencil of Eq. 7's table at R: start, beyond-grid flag, Lagrange weights
//   F of every Eq. 7 table entry at R
//   the energy phase of every state, exp(i eps_i z / v), so that an element's phase
//   exp(i (eps_i - eps_j) z / v) is one complex product
// ---------------------------------------------------------------------------
struct EtArgs {
    int lrot, nlam, Nr;
    int dtot, npb;           // sizes of the d and Pbar parts
    int nfT, nfP;            // Eq. 7 table entries of the two centres (F interpolated at R follows the stencil)
    const double *FT, *FP;
    const double* r;
    int N_T, N;              // states (target first)
    const double *epsT, *epsP;
    size_t ph_off;
    double* et;              // [nev][et_doubles]
    size_t et_doubles;
};

__global__ void __launch_bounds__(128) k_eval_tables(EtArgs A, const EvalDesc* __restrict__ ev) {
    const int e = blockIdx.x;
    const double b = ev[e].b, z = ev[e].z;
    const double R = dist_R(b, z);
    const double cth = z / R;
    const double ch = sqrt(0.5 * (1.0 + cth)), sh = sqrt(0.5 * (1.0 - cth));
    double* et = A.et + (size_t)e * A.et_doubles;
    for (int idx = threadIdx.x; idx < A.dtot; idx += blockDim.x) {
        int l = 0, off = 0;
        while (idx >= off + (2 * l + 1) * (2 * l + 1)) {
            off += (2 * l + 1) * (2 * l + 1);
            ++l;
        }
        int loc = idx - off, m = loc / (2 * l + 1) - l, q = loc % (2 * l + 1) - l;
        et[idx] = wigner_small_d(l, m, q, ch, sh);
    }
    for (int t = threadIdx.x; t < A.npb; t += blockDim.x) {
        int lam = 0;
        while ((lam + 1) * (lam + 2) / 2 <= t) ++lam;
        int mu = t - lam * (lam + 1) / 2;
        et[A.dtot + t] = sqrt(dfact(lam - mu) / dfact(lam + mu)) * assoc_legendre(lam, mu, cth);
    }
    __shared__ int s_s, s_out;
    __shared__ double s_L[5];
    if (threadIdx.x == 0) {
        double* st = et + A.dtot + A.npb;
        int s;
        double L[5];
        if (R > A.r[A.Nr - 1]) {
            st[0] = (double)(A.Nr - 1);
            st[1] = 1.0;
            for (int k = 0; k < 5; ++k) st[2 + k] = 0.0;
            s_s = A.Nr - 1;
            s_out = 1;
        } else {
            stencil5(A.r, A.Nr, R, s, L);
            st[0] = (double)s;
            st[1] = 0.0;
            for (int k = 0; k < 5; ++k) st[2 + k] = L[k];
            s_s = s;
            s_out = 0;
            for (int k = 0; k < 5; ++k) s_L[k] = L[k];
        }
    }
    __syncthreads();
    // F of every Eq. 7 table entry at R (5-point interpolation, or the multipole tail beyond the grid)
    double* Fint = et + A.dtot + A.npb + 8;
    const double ratio = A.r[A.Nr - 1] / R;
    for (int t = threadIdx.x; t < A.nfT + A.nfP; t += blockDim.x) {
        const double* Fe = t < A.nfT ? A.FT + (size_t)t * A.Nr : A.FP + (size_t)(t - A.nfT) * A.Nr;
        double Fv;
        if (s_out) {
            // lam of the entry is not needed here: the tail factor (r_max/R)^{lam+1} is applied in k_direct
            Fv = Fe[A.Nr - 1];
        } else {
            const int s = s_s;
            Fv = s_L[0] * Fe[s] + s_L[1] * Fe[s + 1] + s_L[2] * Fe[s + 2] + s_L[3] * Fe[s + 3] + s_L[4] * Fe[s + 4];
        }
        Fint[t] = Fv;
    }
    (void)ratio;
    double2* ph = reinterpret_cast<double2*>(et + A.ph_off);
    const double v = ev[e].v;
    for (int i = threadIdx.x; i < A.N; i += blockDim.x) {
        const double eps = i < A.N_T ? A.epsT[i] : A.epsP[i - A.N_T];
        double sp, cp;
        sincos(eps * z / v, &sp, &cp);
        ph[i] = make_double2(cp, sp);
    }
}

// ---------------------------------------------------------------------------
// k_rotate: Eq. 8 and the off-diagonal blocks of S and H
// ---------------------------------------------------------------------------
struct RotArgs {
    int N_T, N_P, N, n_half, lmax, n_radT, n_radP;
    int rot_block;            // complex entries of one warp's block: NX (2 lmax_T + 1)(2 lmax_P + 1)
    int dtot;                 // size of the Wigner-d part of the per-position tables
    const double* et;         // per-position tables (k_eval_tables)
    size_t et_doubles, ph_off;
    const int *stT_rad, *stT_l, *stT_m, *stT_index;
    const int *stP_rad, *stP_l, *stP_m, *half_of, *stP_index;
    const int *radT_l, *radP_l;
    const double *epsT, *epsP;
    const double2* mol;
    double2 *S, *H;
    size_t mat;   // N*N
    const int* items;         // [n_items][4]: first pair, pairs, l_T, l_P
    const int* pairs;         // [pairs][2]: target radial, projectile radial
    int n_items;
};

constexpr int ROT_WARPS_MAX = 8;
constexpr int ROT_LANE_CAP = 256;   // block entries one item may hold (more when a single pair has more)

// Work items of k_rotate: the radial pairs (a, b) grouped by (l_a, l_b), and per group the number P of
// pairs one warp takes so that its P NX (2 l_a + 1)(2 l_b + 1) block entries fill the lanes best (the
// passes run over all entries of the item, lane by lane).
wpccc_status rotation_plan(wpccc_basis_s* B) {
    std::vector<int> items, pairs;
    int cap = 0;
    for (int la = 0; la <= B->T.lmax; ++la)
        for (int lb = 0; lb <= B->P.lmax; ++lb) {
            std::vector<int> cls;
            for (int ra = 0; ra < B->T.n_rad; ++ra)
                if (B->T.h_rad_l[ra] == la)
                    for (int rb = 0; rb < B->P.n_rad; ++rb)
                        if (B->P.h_rad_l[rb] == lb) {
                            cls.push_back(ra);
                            cls.push_back(rb);
                        }
            const int np = (int)cls.size() / 2;
            if (np == 0) continue;
            const int E = NX * (2 * la + 1) * (2 * lb + 1);
            int best = 1;
            double bu = (double)E / (32.0 * ((E + 31) / 32));
            for (int P = 2; P <= np && P * E <= std::max(ROT_LANE_CAP, E); ++P) {
                const double u = (double)(P * E) / (32.0 * ((P * E + 31) / 32));
                if (u > bu + 1e-12) {
                    bu = u;
                    best = P;
                }
            }
            const int first = (int)pairs.size() / 2;
            pairs.insert(pairs.end(), cls.begin(), cls.end());
            for (int k = 0; k < np; k += best) {
                const int cnt = std::min(best, np - k);
                items.insert(items.end(), {first + k, cnt, la, lb});
                cap = std::max(cap, cnt * E);
            }
        }
    std::vector<int> plan(items);
    plan.insert(plan.end(), pairs.begin(), pairs.end());
    WPCCC_CUDA(cudaMalloc((void**)&B->rot_plan, plan.size() * sizeof(int)));
    WPCCC_CUDA(cudaMemcpy(B->rot_plan, plan.data(), plan.size() * sizeof(int), cudaMemcpyHostToDevice));
    B->n_rot_items = (int)items.size() / 4;
    B->rot_cap = cap;
    return WPCCC_OK;
}

// One warp per work item: P radial pairs (a, b) of one (l_a, l_b).  For each pair the (2l_a+1) x (2l_b+1)
// molecular-frame block of each integral (q < 0 columns from the reflection) is rotated in two passes
// through shared memory, T[q'][m_b] = sum_q d^{l_b}_{m_b q} X[q'][q], then K[m_a][m_b] =
// sum_q' d^{l_a}_{m_a q'} T[q'][m_b] with the energy phases; every pass runs over the item's P NX blk
// entries, lane by lane.
__global__ void __launch_bounds__(32 * ROT_WARPS_MAX) k_rotate(RotArgs A, const EvalDesc* __restrict__ ev) {
    extern __shared__ double sd[];     // Wigner d^l_{m q}(theta) for l <= lmax, then per-warp blocks
    const int e = blockIdx.y;
    const int total = A.dtot;
    const double* etd = A.et + (size_t)e * A.et_doubles;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) sd[idx] = etd[idx];
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = blockIdx.x * (blockDim.x >> 5) + warp;
    if (item >= A.n_items) return;
    const int p0 = A.items[4 * item], P = A.items[4 * item + 1], la = A.items[4 * item + 2],
              lb = A.items[4 * item + 3];
    const int* pr = A.pairs + 2 * p0;
    const int na = 2 * la + 1, nbq = 2 * lb + 1, blk = na * nbq, E = NX * blk, PE = P * E;
    const int tot_pad = (total + 1) & ~1;
    double2* X = reinterpret_cast<double2*>(sd + tot_pad) + (size_t)warp * 2 * A.rot_block;
    double2* T = X + A.rot_block;
    int offa = 0, offb = 0;
    for (int l = 0; l < la; ++l) offa += (2 * l + 1) * (2 * l + 1);
    for (int l = 0; l < lb; ++l) offb += (2 * l + 1) * (2 * l + 1);
    const double* da = sd + offa;   // da[(m + la) * na + (q + la)] = d^{la}_{m q}
    const double* db = sd + offb;
    const size_t plane = (size_t)A.N_T * A.n_half;
    const double2* mol = A.mol + (size_t)e * NX * plane;
    // molecular blocks, entry p E + x blk + (q' + la) nbq + (q + lb)
    for (int t = lane; t < PE; t += 32) {
        const int p = t / E, r0 = t - p * E, x = r0 / blk, r = r0 - x * blk, qp = r / nbq - la, q = r % nbq - lb;
        const int ra = pr[2 * p], rb = pr[2 * p + 1];
        int row, col;
        bool neg = false;
        if (q >= 0) {
            row = A.stT_index[ra * (2 * WPCCC_LMAX + 1) + qp + WPCCC_LMAX];
            col = A.half_of[rb * (WPCCC_LMAX + 1) + q];
        } else {
            row = A.stT_index[ra * (2 * WPCCC_LMAX + 1) - qp + WPCCC_LMAX];
            col = A.half_of[rb * (WPCCC_LMAX + 1) - q];
            neg = (qp + q) & 1;
        }
        double2 val = mol[(size_t)x * plane + (size_t)row * A.n_half + col];
        if (neg) val = make_double2(-val.x, -val.y);
        X[t] = val;
    }
    __syncwarp();
    // T[p][x][q'][m_b] = sum_q d^{lb}_{m_b q} X[p][x][q'][q]
    for (int t = lane; t < PE; t += 32) {
        const int r = t % blk, qi = r / nbq, mb = r % nbq;
        const double2* xr = X + (t - r) + qi * nbq;
        const double* dr = db + mb * nbq;
        double re = 0.0, im = 0.0;
        for (int q = 0; q < nbq; ++q) {
            re = fma(dr[q], xr[q].x, re);
            im = fma(dr[q], xr[q].y, im);
        }
        T[t] = make_double2(re, im);
    }
    __syncwarp();
    // K, Q [p][x][m_a][m_b] = sum_q' d^{la}_{m_a q'} T[p][x][q'][m_b] with the energy phases, into X
    const double2* phs = reinterpret_cast<const double2*>(etd + A.ph_off);
    for (int t = lane; t < PE; t += 32) {
        const int p = t / E, r = t % blk, mi = r / nbq, mb = r % nbq;
        const double* dr = da + mi * na;
        const double2* tc = T + (t - r) + mb;
        double re = 0.0, im = 0.0;
        for (int qi = 0; qi < na; ++qi) {
            const double w = dr[qi];
            const double2 tv = tc[qi * nbq];
            re = fma(w, tv.x, re);
            im = fma(w, tv.y, im);
        }
        const int ra = pr[2 * p], rb = pr[2 * p + 1];
        const int i = A.stT_index[ra * (2 * WPCCC_LMAX + 1) + (mi - la) + WPCCC_LMAX];
        const int j = A.stP_index[rb * (2 * WPCCC_LMAX + 1) + (mb - lb) + WPCCC_LMAX];
        const double2 ph = cmul(phs[i], cconj(phs[A.N_T + j]));
        X[t] = cmul(make_double2(re, im), ph);
    }
    __syncwarp();
    // S and H entries: the upper blocks with the target index fastest (consecutive rows of a column), the
    // lower blocks with the projectile index fastest, so that both writes run along memory
    double2* S = A.S + (size_t)e * A.mat;
    double2* H = A.H + (size_t)e * A.mat;
    for (int t = lane; t < P * blk; t += 32) {
        const int p = t / blk, r = t - p * blk, mi = r % na, mb = r / na;
        const int ra = pr[2 * p], rb = pr[2 * p + 1];
        const int i = A.stT_index[ra * (2 * WPCCC_LMAX + 1) + (mi - la) + WPCCC_LMAX];
        const int j = A.stP_index[rb * (2 * WPCCC_LMAX + 1) + (mb - lb) + WPCCC_LMAX];
        const size_t up = (size_t)i + (size_t)(A.N_T + j) * A.N;     // row i, column N_T + j
        S[up] = X[p * E + mi * nbq + mb];
        H[up] = X[p * E + blk + mi * nbq + mb];
    }
    for (int t = lane; t < P * blk; t += 32) {
        const int p = t / blk, r = t - p * blk, mi = r / nbq, mb = r % nbq;
        const int ra = pr[2 * p], rb = pr[2 * p + 1];
        const int i = A.stT_index[ra * (2 * WPCCC_LMAX + 1) + (mi - la) + WPCCC_LMAX];
        const int j = A.stP_index[rb * (2 * WPCCC_LMAX + 1) + (mb - lb) + WPCCC_LMAX];
        const size_t lo = (size_t)(A.N_T + j) + (size_t)i * A.N;     // row N_T + j, column i
        S[lo] = cconj(X[p * E + r]);
        H[lo] = cconj(X[p * E + blk + r]);     // Eq. 1: the lower-left block of H is Q^+
    }
}

// ---------------------------------------------------------------------------
// k_direct: Eq. 6 blocks (and identity blocks of S)
// ---------------------------------------------------------------------------
struct DirArgs {
    int Nr, N, off, Nc, n_rad, nlam;
    int dtot, npb;                // layout of the per-position tables
    int foff0;                    // first interpolated F entry of this centre in the per-position tables
    const double* et;
    size_t et_doubles, ph_off;
    double Z_other, parity;       // parity = -1: the other nucleus sits at -R
    const double *r, *F, *ang, *eps;
    const int *Foff, *st_rad, *st_m, *st_lm;
    int LM;
    size_t cp_off;                // this centre's Eq. 6 coefficients within the per-position tables
    double2 *S, *H;
    size_t mat;
};

// Eq. 6 coefficients of one position and centre, per pair of angular parts and multipole:
//   cp[(l'm', lm)][lam] = -Z_other parity^lam A(l'm', lm, lam) Pbar_lam^|mu|(cos theta) (-1)^mu [mu < 0, odd]
//                         x (r_max / R)^(lam + 1) when R lies beyond the radial grid,
// so that D[(a', m')][(a, m)] = sum_lam cp[..][lam] F_lam^{a'a}(R) takes one multiply-add per term.
__global__ void k_direct_coef(DirArgs A0, DirArgs A1, const EvalDesc* __restrict__ ev) {
    const DirArgs& A = blockIdx.z == 0 ? A0 : A1;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long n = (long long)A.LM * A.LM * A.nlam;
    if (idx >= n) return;
    const int e = blockIdx.y;
    const int lam = (int)(idx % A.nlam);
    const long long pr = idx / A.nlam;
    const int a = (int)(pr / A.LM), b2 = (int)(pr % A.LM);
    int lp = 0, l = 0;
    while ((lp + 1) * (lp + 1) <= a) ++lp;
    while ((l + 1) * (l + 1) <= b2) ++l;
    const int mu = (a - lp * lp - lp) - (b2 - l * l - l);
    const int amu = mu < 0 ? -mu : mu;
    double* et = const_cast<double*>(A.et) + (size_t)e * A.et_doubles;
    const double c = A.ang[idx];
    double v = 0.0;
    if (c != 0.0) {
        double P = et[A.dtot + lam * (lam + 1) / 2 + amu];
        if (mu < 0 && (amu & 1)) P = -P;
        double sc = (lam & 1) ? A.parity : 1.0;
        const double* st = et + A.dtot + A.npb;
        if (st[1] != 0.0) {
            const double R = dist_R(ev[e].b, ev[e].z);
            const double ratio = A.r[A.Nr - 1] / R;
            double p = ratio;
            for (int k = 0; k < lam; ++k) p *= ratio;
            sc *= p;
        }
        v = -A.Z_other * sc * c * P;
    }
    et[A.cp_off + idx] = v;
}

__global__ void __launch_bounds__(256) k_direct(DirArgs A0, DirArgs A1, const EvalDesc* __restrict__ ev) {
    const DirArgs& A = blockIdx.z == 0 ? A0 : A1;
    const int e = blockIdx.y;
    const double* et = A.et + (size_t)e * A.et_doubles;
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)A.Nc * A.Nc) return;
    // consecutive threads take consecutive rows of a column: the writes run along column-major memory
    const int i = (int)(idx % A.Nc), j = (int)(idx / A.Nc);
    const int ra = A.st_rad[i], rb = A.st_rad[j];
    const double* cp = et + A.cp_off + ((size_t)A.st_lm[i] * A.LM + A.st_lm[j]) * A.nlam;
    const int* foff = A.Foff + ((size_t)ra * A.n_rad + rb) * A.nlam;
    const double* Fint = et + A.dtot + A.npb + 8 + A.foff0;
    double D = 0.0;
    for (int lam = 0; lam < A.nlam; ++lam) {
        const double c = cp[lam];
        if (c == 0.0) continue;
        D = fma(c, Fint[foff[lam]], D);
    }
    const double2* phs = reinterpret_cast<const double2*>(et + A.ph_off);
    const double2 ph = cmul(phs[A.off + i], cconj(phs[A.off + j]));
    const size_t o = (size_t)(A.off + i) + (size_t)(A.off + j) * A.N;
    A.H[(size_t)e * A.mat + o] = make_double2(D * ph.x, D * ph.y);
    if (A.S) A.S[(size_t)e * A.mat + o] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

// ---------------------------------------------------------------------------
// k_direct_sr: short-range part of a model-potential target between projectile states.
// In the molecular frame the potential is symmetric about the axis, so only equal q couple:
//   I[b][q] = (R^3/8) sum_g w_g (eta^2 - tau^2) V_s(r_T) f_a(r_P) Theta_{l_a q}(c_P) f_b(r_P) Theta_{l_b q}(c_P)
// (Theta_{l,-q} = (-1)^q Theta_{l,q}, so I does not depend on the sign of q).  One block per
// (projectile radial a, position): a warp per (b, q) sums over the nodes, then the rows of a are
// rotated with d^{l}(theta) on both sides, given their energy phases and added to H.
// ---------------------------------------------------------------------------
struct SrArgs {
    int G, Gtau, nradT, nradP, lmaxP, nlqT, N_T, N_P, N, dtot;
    double gamma, mp_c, mp_a, mp_b;
    const double *s, *ws, *tau, *wtau;
    const double* node;        // FP64 node tables per evaluation
    size_t node_doubles;
    const double* et;          // per-position tables (Wigner d first, energy phases at ph_off)
    size_t et_doubles, ph_off;
    const int *radP_l, *stP_index, *stP_rad, *stP_m;
    const double* epsP;
    double2* H;
    size_t mat;
};

__global__ void __launch_bounds__(256) k_direct_sr(SrArgs A, const EvalDesc* __restrict__ ev) {
    extern __shared__ double srm[];   // [G] V_s-weighted f_a, then I[n_radP][lmaxP+1], then Wigner d
    const int a = blockIdx.x, e = blockIdx.y;
    const double b = ev[e].b, z = ev[e].z;
    const double R = dist_R(b, z);
    const double gR = __dmul_rn(A.gamma, R);
    const double halfR = __dmul_rn(0.5, R);
    const double* base = A.node + (size_t)e * A.node_doubles;
    const double* oP = base + (size_t)A.nradT * A.G;
    const double* thP = oP + (size_t)A.nradP * A.G + (size_t)A.nlqT * A.G;
    const int LQ = A.lmaxP + 1;
    double* ufa = srm;
    double* I = srm + A.G;
    double* dt = I + A.nradP * LQ;
    for (int g = threadIdx.x; g < A.G; g += blockDim.x) {
        const int k = g / A.Gtau, t = g - k * A.Gtau;
        const double eta = __dadd_rn(1.0, __ddiv_rn(A.s[k], gR));
        const double tau = A.tau[t];
        const double rT = __dmul_rn(halfR, __dadd_rn(eta, tau));
        const double wgt = (A.ws[k] / gR) * A.wtau[t];
        const double vol = (R * R * R / 8.0) * wgt * (eta * eta - tau * tau);
        const double Vs = (-A.mp_c * exp(-A.mp_a * rT)) * (1.0 + A.mp_b * rT) / rT;
        ufa[g] = vol * Vs * oP[(size_t)a * A.G + g];
    }
    const double* etd = A.et + (size_t)e * A.et_doubles;
    for (int t = threadIdx.x; t < A.dtot; t += blockDim.x) dt[t] = etd[t];
    __syncthreads();
    const int la = A.radP_l[a];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int pq = warp; pq < A.nradP * LQ; pq += nw) {
        const int bb = pq / LQ, q = pq - bb * LQ;
        const int lb = A.radP_l[bb];
        double acc = 0.0;
        if (q <= la && q <= lb) {
            const double* ta = thP + (size_t)(la * (la + 1) / 2 + q) * A.G;
            const double* tb = thP + (size_t)(lb * (lb + 1) / 2 + q) * A.G;
            const double* fb = oP + (size_t)bb * A.G;
            for (int g = lane; g < A.G; g += 32) acc = fma(ufa[g] * ta[g], fb[g] * tb[g], acc);
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) I[pq] = acc;
    }
    __syncthreads();
    // lab frame: D[(a, m)][(b, m')] = sum_q d^{la}_{m q} d^{lb}_{m' q} I[b][|q|]
    int offa = 0;
    for (int l = 0; l < la; ++l) offa += (2 * l + 1) * (2 * l + 1);
    double2* H = A.H + (size_t)e * A.mat;
    for (int idx = threadIdx.x; idx < (2 * la + 1) * A.N_P; idx += blockDim.x) {
        const int mi = idx / A.N_P - la, j = idx % A.N_P;
        const int bb = A.stP_rad[j], lb = A.radP_l[bb], mj = A.stP_m[j];
        int offb = 0;
        for (int l = 0; l < lb; ++l) offb += (2 * l + 1) * (2 * l + 1);
        const int qm = la < lb ? la : lb;
        double D = 0.0;
        for (int q = -qm; q <= qm; ++q) {
            const double da = dt[offa + (mi + la) * (2 * la + 1) + (q + la)];
            const double db = dt[offb + (mj + lb) * (2 * lb + 1) + (q + lb)];
            D = fma(da * db, I[bb * LQ + (q < 0 ? -q : q)], D);
        }
        const int i = A.stP_index[a * (2 * WPCCC_LMAX + 1) + mi + WPCCC_LMAX];
        const double2* phs = reinterpret_cast<const double2*>(etd + A.ph_off);
        const double2 ph = cmul(phs[A.N_T + i], cconj(phs[A.N_T + j]));
        const size_t o = (size_t)(A.N_T + i) + (size_t)(A.N_T + j) * A.N;
        const double2 h = H[o];
        H[o] = make_double2(fma(D, ph.x, h.x), fma(D, ph.y, h.y));
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
ElemScratch elem_scratch_layout(const wpccc_basis_s* B) {
    ElemScratch L{};
    const int lrot = std::max(B->T.lmax, B->n_centres == 2 ? B->P.lmax : 0);
    for (int l = 0; l <= lrot; ++l) L.dtot += (2 * l + 1) * (2 * l + 1);
    const int nlam = 2 * lrot + 1;
    L.npb = nlam * (nlam + 1) / 2;
    L.et_doubles = (size_t)L.dtot + L.npb + 8 + B->T.n_fent + (B->n_centres == 2 ? B->P.n_fent : 0);
    L.et_doubles += L.et_doubles & 1;
    L.ph_off = L.et_doubles;
    L.et_doubles += 2 * (size_t)B->N;
    L.cp_off[0] = L.et_doubles;
    L.et_doubles += (size_t)B->T.LM * B->T.LM * B->T.nlam;
    L.cp_off[1] = L.et_doubles;
    if (B->n_centres == 2) L.et_doubles += (size_t)B->P.LM * B->P.LM * B->P.nlam;
    L.et_doubles += L.et_doubles & 1;
    if (B->n_centres == 2) {
        size_t nd = (size_t)(B->T.n_rad + B->P.n_rad + B->nlq_T + B->nlq_P) * B->G;
        nd += nd & 1;   // keep the complex weights 16-byte aligned
        L.w_off = nd;
        nd += (size_t)NX * (B->dmax + 1) * B->G * 2;
        // FP32 layout of the mixed-precision form: per-state products, then the weights (floats)
        size_t nf = (size_t)(B->N_T + B->n_half) * B->G;
        nf += nf & 1;
        L.w_off_f = nf;
        nf += (size_t)NX * (B->dmax + 1) * B->G * 2;
        L.node_doubles = std::max(nd, (nf + 1) / 2);
        if (B->tc_layout) {
            L.tc_rows = 2 * B->N_T;
            // tensor-core layout (precision modes 3-5): up to seven bf16 slice planes [7][tc_rows][G], the
            // scales per 128-node window, A_P [n_half][G] and W_K / r_T [d][re, im][G] as double-floats
            size_t n6 = ((size_t)OZ_SLICES * L.tc_rows * B->G + 7) / 8 * 4;
            L.t6_sc_off = n6;
            n6 += ((size_t)L.tc_rows * ((B->G + 127) / 128) + 3) / 4 * 4;
            L.t6_ap_off = n6;
            n6 += (size_t)2 * B->n_half * B->G;
            L.t6_w_off = n6;
            n6 += (size_t)4 * (B->dmax + 1) * B->G;
            L.node_doubles = std::max(L.node_doubles, (n6 + 1) / 2);
        }
        L.node_doubles += L.node_doubles & 1;
        L.mol_elems = (size_t)NX * B->N_T * B->n_half;
        L.bytes_per_eval = L.node_doubles * sizeof(double) + L.mol_elems * sizeof(double2);
    }
    L.bytes_per_eval += L.et_doubles * sizeof(double);
    return L;
}

static DirArgs dir_args(const wpccc_basis_s* B, const CentreDev& c, int off, double Z_other, double parity,
                        double2* S, double2* H) {
    DirArgs a;
    a.Nr = B->Nr;
    a.N = B->N;
    a.off = off;
    a.Nc = c.n_states;
    a.n_rad = c.n_rad;
    a.nlam = c.nlam;
    a.Z_other = Z_other;
    a.parity = parity;
    a.r = B->r;
    a.F = c.F;
    a.ang = c.ang;
    a.st_lm = c.st_lm;
    a.LM = c.LM;
    a.eps = c.st_eps;
    a.Foff = c.Foff;
    a.st_rad = c.st_rad;
    a.st_m = c.st_m;
    a.S = S;
    a.H = H;
    a.mat = (size_t)B->N * B->N;
    const ElemScratch L = elem_scratch_layout(B);
    a.cp_off = L.cp_off[off == 0 ? 0 : 1];
    a.dtot = L.dtot;
    a.npb = L.npb;
    a.et = nullptr;
    a.et_doubles = L.et_doubles;
    a.ph_off = L.ph_off;
    return a;
}

// Per-position tables (k_eval_tables) and, two-centre, the node tables of Eq. 9 (k_node_tables).
static wpccc_status launch_tables(wpccc_basis_s* B, const EvalDesc* evals, int nev, void* scratch,
                                  cudaStream_t st, int precision) {
    const bool two = B->n_centres == 2;
    const ElemScratch L = elem_scratch_layout(B);
    double* node = static_cast<double*>(scratch);
    double2* mol = reinterpret_cast<double2*>(node + L.node_doubles * nev);
    double* et = reinterpret_cast<double*>(mol + L.mol_elems * nev);
    {
        EtArgs ea;
        ea.lrot = std::max(B->T.lmax, two ? B->P.lmax : 0);
        ea.nlam = 2 * ea.lrot + 1;
        ea.Nr = B->Nr;
        ea.dtot = L.dtot;
        ea.npb = L.npb;
        ea.r = B->r;
        ea.nfT = B->T.n_fent;
        ea.nfP = two ? B->P.n_fent : 0;
        ea.FT = B->T.F;
        ea.FP = two ? B->P.F : nullptr;
        ea.N_T = B->N_T;
        ea.N = B->N;
        ea.epsT = B->T.st_eps;
        ea.epsP = two ? B->P.st_eps : nullptr;
        ea.ph_off = L.ph_off;
        ea.et = et;
        ea.et_doubles = L.et_doubles;
        cudaEvent_t e0 = B->prof.begin(PROF_NODES, st);
        k_eval_tables<<<nev, 128, 0, st>>>(ea, evals);
        WPCCC_CHECK_LAUNCH("k_eval_tables");
        B->prof.end(PROF_NODES, st, e0);
    }
    if (!two) return WPCCC_OK;
    NodeArgs na;
    na.Nr = B->Nr;
    na.G = B->G;
    na.Gtau = B->Gtau;
    na.nradT = B->T.n_rad;
    na.nradP = B->P.n_rad;
    na.lmaxT = B->T.lmax;
    na.lmaxP = B->P.lmax;
    na.nlqT = B->nlq_T;
    na.nlqP = B->nlq_P;
    na.dmax = B->dmax;
    na.gamma = B->gamma;
    na.Z_T = B->T.Z;
    na.Z_P = B->P.Z;
    na.mp_c = B->mp_c;
    na.mp_a = B->mp_a;
    na.mp_b = B->mp_b;
    na.r = B->r;
    na.fT = B->T.f;
    na.fP = B->P.f;
    na.fT2 = B->fT2;
    na.fP2 = B->fP2;
    na.s = B->s;
    na.ws = B->ws;
    na.tau = B->tau;
    na.wtau = B->wtau;
    na.inv_den = B->inv_den;
    na.node = node;
    na.node_doubles = L.node_doubles;
    na.w_off = precision == 0 ? L.w_off : L.w_off_f;
    na.N_T = B->N_T;
    na.n_half = B->n_half;
    na.stT_index = B->T.st_index;
    na.half_of = B->half_of;
    na.radT_l = B->T.rad_l;
    na.radP_l = B->P.rad_l;
    na.tc = precision == 3 || precision == 4;
    na.tc_slices = precision == 3 ? OZ_FAST_SLICES : OZ_SLICES;
    na.tc_row = B->tc_row;
    na.tc_rows = L.tc_rows;
    na.t6_ap_off = L.t6_ap_off;
    na.t6_w_off = L.t6_w_off;
    na.t6_sc_off = L.t6_sc_off;
    for (int l = 0; l <= WPCCC_LMAX; ++l) {
        na.inv_int[l] = l > 0 ? 1.0 / l : 0.0;
        for (int q = 0; q <= l; ++q) {
            double num = 1.0, den = 1.0;   // (l-q)!, (l+q)!
            for (int k = 2; k <= l - q; ++k) num *= k;
            for (int k = 2; k <= l + q; ++k) den *= k;
            na.th_nrm[l * (l + 1) / 2 + q] = std::sqrt((2.0 * l + 1.0) * 0.5 * num / den);
        }
    }
    if (na.tc && !B->tc_layout) return fail(WPCCC_EINVAL, "tensor-core layout not prepared");
    if (na.tc && B->G % 128 != 0) return fail(WPCCC_EUNSUPPORTED, "the tensor-core layout needs a multiple of 128 nodes");
    const size_t nsm = node_tables_smem(B, na.tc);
    cudaEvent_t e0 = B->prof.begin(PROF_NODES, st);
    if (precision == 0) {
        k_node_tables<double><<<dim3((B->G + 127) / 128, nev), 128, 0, st>>>(na, evals);
    } else {
        if (nsm > 48 * 1024)
            WPCCC_CUDA(cudaFuncSetAttribute(k_node_tables<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)nsm));
        k_node_tables<float><<<dim3((B->G + 127) / 128, nev), 128, nsm, st>>>(na, evals);
    }
    WPCCC_CHECK_LAUNCH("k_node_tables");
    B->prof.end(PROF_NODES, st, e0);
    return WPCCC_OK;
}

wpccc_status launch_node_stage(wpccc_basis_s* B, const EvalDesc* evals, int nev, void* scratch, cudaStream_t st) {
    if (nev <= 0) return WPCCC_OK;
    return launch_tables(B, evals, nev, scratch, st, 0);
}

wpccc_status launch_elements(wpccc_basis_s* B, const EvalDesc* evals, int nev, double2* S,
                             double2* H, void* scratch, cudaStream_t st, int precision) {
    if (nev <= 0) return WPCCC_OK;
    const bool two = B->n_centres == 2;
    if (two && B->mp_c != 0.0 && precision != 0)
        return fail(WPCCC_EUNSUPPORTED, "model-potential targets need FP64 elements (precision mode 0 or 2)");
    const ElemScratch L = elem_scratch_layout(B);
    double* node = static_cast<double*>(scratch);
    double2* mol = reinterpret_cast<double2*>(node + L.node_doubles * nev);
    double* et = reinterpret_cast<double*>(mol + L.mol_elems * nev);
    wpccc_status ts = launch_tables(B, evals, nev, scratch, st, precision);
    if (ts != WPCCC_OK) return ts;
    if (two) {
        GemmArgs ga;
        ga.G = B->G;
        ga.N_T = B->N_T;
        ga.n_half = B->n_half;
        ga.nradT = B->T.n_rad;
        ga.nradP = B->P.n_rad;
        ga.nlqT = B->nlq_T;
        ga.nlqP = B->nlq_P;
        ga.dmax = B->dmax;
        ga.n_col_tiles = (B->n_half + GT_J - 1) / GT_J;
        ga.stT_rad = B->T.st_rad;
        ga.stT_l = B->T.st_l;
        ga.stT_m = B->T.st_m;
        ga.stP_rad = B->P.st_rad;
        ga.stP_l = B->P.st_l;
        ga.stP_m = B->P.st_m;
        ga.half_state = B->half_state;
        ga.node = node;
        ga.node_doubles = L.node_doubles;
        ga.w_off = precision == 0 ? L.w_off : L.w_off_f;
        ga.mol = mol;
        const int n_row_tiles = (B->N_T + GT_I - 1) / GT_I;
        cudaEvent_t e0 = B->prof.begin(PROF_MOL, st);
        if (precision == 0) {
            const size_t gsm = (size_t)GT_K * (GT_I + 1 + GT_J + 1) * sizeof(double) +
                               (size_t)NX * (B->dmax + 1) * GT_K * sizeof(double2);
            WPCCC_CUDA(cudaFuncSetAttribute(k_mol_gemm<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)gsm));
            k_mol_gemm<double><<<dim3(n_row_tiles * ga.n_col_tiles, nev), 256, gsm, st>>>(ga);
        } else if (precision == 3 || precision == 4) {
            wpccc_status ms = launch_mol_tc64(B, nev, node, mol, B->tc_err, st,
                                               precision == 3 ? OZ_FAST_SLICES : OZ_SLICES);
            if (ms != WPCCC_OK) return ms;
        } else {
            Gemm32Args g32;
            g32.G = B->G;
            g32.N_T = B->N_T;
            g32.n_half = B->n_half;
            g32.dmax = B->dmax;
            g32.n_col_tiles = B->n_qtiles;
            g32.stT_m = B->T.st_m;
            g32.ctile_q = B->qtile_q;
            g32.ctile_cols = B->qtile_cols;
            g32.node = node;
            g32.node_doubles = L.node_doubles;
            g32.w_off_f = L.w_off_f;
            g32.mol = mol;
            const int rtiles = (B->N_T + QT_I - 1) / QT_I;
            const size_t qsm = mol_gemm_f32q_smem(B->dmax);
            WPCCC_CUDA(cudaFuncSetAttribute(k_mol_gemm_f32q, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)qsm));
            k_mol_gemm_f32q<<<dim3(rtiles * B->n_qtiles, nev), QT_THREADS, qsm, st>>>(g32);
        }
        WPCCC_CHECK_LAUNCH("k_mol_gemm");
        B->prof.end(PROF_MOL, st, e0);

        RotArgs ra;
        ra.N_T = B->N_T;
        ra.N_P = B->N_P;
        ra.N = B->N;
        ra.n_half = B->n_half;
        ra.lmax = std::max(B->T.lmax, B->P.lmax);
        ra.stT_rad = B->T.st_rad;
        ra.stT_l = B->T.st_l;
        ra.stT_m = B->T.st_m;
        ra.stT_index = B->T.st_index;
        ra.stP_rad = B->P.st_rad;
        ra.stP_l = B->P.st_l;
        ra.stP_m = B->P.st_m;
        ra.half_of = B->half_of;
        ra.stP_index = B->P.st_index;
        ra.n_radT = B->T.n_rad;
        ra.n_radP = B->P.n_rad;
        ra.radT_l = B->T.rad_l;
        ra.radP_l = B->P.rad_l;
        ra.epsT = B->T.st_eps;
        ra.epsP = B->P.st_eps;
        ra.mol = mol;
        ra.S = S;
        ra.H = H;
        ra.mat = (size_t)B->N * B->N;
        int dtot = 0;
        for (int l = 0; l <= ra.lmax; ++l) dtot += (2 * l + 1) * (2 * l + 1);
        ra.rot_block = B->rot_cap;
        ra.items = B->rot_plan;
        ra.pairs = B->rot_plan + 4 * B->n_rot_items;
        ra.n_items = B->n_rot_items;
        ra.dtot = L.dtot;
        ra.et = et;
        ra.et_doubles = L.et_doubles;
        ra.ph_off = L.ph_off;
        const size_t per_warp = (size_t)2 * ra.rot_block * sizeof(double2);
        const size_t dbytes = (size_t)((dtot + 1) & ~1) * sizeof(double);
        int rwarps = (int)std::min<size_t>(ROT_WARPS_MAX, ((size_t)200 * 1024 - dbytes) / per_warp);
        if (rwarps < 1) rwarps = 1;
        const size_t rsm = dbytes + (size_t)rwarps * per_warp;
        const dim3 rgrid((unsigned)((B->n_rot_items + rwarps - 1) / rwarps), nev);
        e0 = B->prof.begin(PROF_ROT_DIRECT, st);
        WPCCC_CUDA(cudaFuncSetAttribute(k_rotate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rsm));
        k_rotate<<<rgrid, 32 * rwarps, rsm, st>>>(ra, evals);
        WPCCC_CHECK_LAUNCH("k_rotate");
        B->prof.end(PROF_ROT_DIRECT, st, e0);
    }
    DirArgs d0 = dir_args(B, B->T, 0, B->P.Z, 1.0, S, H);
    DirArgs d1 = two ? dir_args(B, B->P, B->N_T, B->T.Z, -1.0, S, H) : d0;
    d0.et = et;
    d1.et = et;
    d0.foff0 = 0;
    d1.foff0 = B->T.n_fent;
    int ncmax = two ? std::max(B->N_T, B->N_P) : B->N_T;
    long long cells = (long long)ncmax * ncmax;
    cudaEvent_t ed = B->prof.begin(PROF_ROT_DIRECT, st);
    const long long ncoef = std::max((long long)B->T.LM * B->T.LM * B->T.nlam,
                                     two ? (long long)B->P.LM * B->P.LM * B->P.nlam : 0LL);
    k_direct_coef<<<dim3((unsigned)((ncoef + 255) / 256), nev, two ? 2 : 1), 256, 0, st>>>(d0, d1, evals);
    WPCCC_CHECK_LAUNCH("k_direct_coef");
    k_direct<<<dim3((unsigned)((cells + 255) / 256), nev, two ? 2 : 1), 256, 0, st>>>(d0, d1, evals);
    WPCCC_CHECK_LAUNCH("k_direct");
    B->prof.end(PROF_ROT_DIRECT, st, ed);
    if (two && B->mp_c != 0.0) {
        SrArgs sa;
        sa.G = B->G;
        sa.Gtau = B->Gtau;
        sa.nradT = B->T.n_rad;
        sa.nradP = B->P.n_rad;
        sa.lmaxP = B->P.lmax;
        sa.nlqT = B->nlq_T;
        sa.N_T = B->N_T;
        sa.N_P = B->N_P;
        sa.N = B->N;
        sa.dtot = L.dtot;
        sa.gamma = B->gamma;
        sa.mp_c = B->mp_c;
        sa.mp_a = B->mp_a;
        sa.mp_b = B->mp_b;
        sa.s = B->s;
        sa.ws = B->ws;
        sa.tau = B->tau;
        sa.wtau = B->wtau;
        sa.node = node;
        sa.node_doubles = L.node_doubles;
        sa.et = et;
        sa.et_doubles = L.et_doubles;
        sa.ph_off = L.ph_off;
        sa.radP_l = B->P.rad_l;
        sa.stP_index = B->P.st_index;
        sa.stP_rad = B->P.st_rad;
        sa.stP_m = B->P.st_m;
        sa.epsP = B->P.st_eps;
        sa.H = H;
        sa.mat = (size_t)B->N * B->N;
        const size_t srsm = ((size_t)B->G + (size_t)B->P.n_rad * (B->P.lmax + 1) + L.dtot) * sizeof(double);
        WPCCC_CUDA(cudaFuncSetAttribute(k_direct_sr, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)srsm));
        ed = B->prof.begin(PROF_ROT_DIRECT, st);
        k_direct_sr<<<dim3(B->P.n_rad, nev), 256, srsm, st>>>(sa, evals);
        WPCCC_CHECK_LAUNCH("k_direct_sr");
        B->prof.end(PROF_ROT_DIRECT, st, ed);
    }
    return WPCCC_OK;
}

// Grows the basis-owned scratch buffer to at least `bytes`.
wpccc_status ensure_workspace(wpccc_basis_s* B, size_t bytes) {
    if (B->ws_bytes >= bytes) return WPCCC_OK;
    if (B->ws_ptr) {
        cudaError_t e = cudaFree(B->ws_ptr);
        B->ws_ptr = nullptr;
        B->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_fail(e, "cudaFree(workspace)");
    }
    cudaError_t e = cudaMalloc(&B->ws_ptr, bytes);
    if (e != cudaSuccess) {
        B->ws_ptr = nullptr;
        return cuda_fail(e, "cudaMalloc(workspace)");
    }
    B->ws_bytes = bytes;
    return WPCCC_OK;
}

}  // namespace wpccc

using namespace wpccc;

namespace wpccc {
static wpccc_status matrix_elements_prec(wpccc_basis B, double b, double v, int nz, const double* z, void* S,
                                         void* H, int precision, void* stream);
}

extern "C" wpccc_status wpccc_matrix_elements(wpccc_basis B, double b, double v, int nz, const double* z,
                                              void* S, void* H, void* stream) {
    return matrix_elements_prec(B, b, v, nz, z, S, H, 0, stream);
}

extern "C" wpccc_status wpccc_matrix_elements_precision(wpccc_basis B, double b, double v, int nz, const double* z,
                                                        void* S, void* H, int precision_mode, void* stream) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_matrix_elements_precision: null basis");
    if (precision_mode != 0 && precision_mode != 1 && precision_mode != 3 && precision_mode != 4)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_matrix_elements_precision: element precision 0, 1, 3 or 4");
    if (precision_mode != 0 && B->n_centres != 2)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_matrix_elements_precision: reduced precision needs two centres");
    if (precision_mode != 0 && B->mp_c != 0.0)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_matrix_elements_precision: model-potential targets need FP64");
    if (precision_mode >= 3 && B->G % 128 != 0)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_matrix_elements_precision: modes 3 and 4 need a node count that is a multiple of 128");
    return matrix_elements_prec(B, b, v, nz, z, S, H, precision_mode, stream);
}

namespace wpccc {
static wpccc_status matrix_elements_prec(wpccc_basis B, double b, double v, int nz, const double* z, void* S,
                                         void* H, int precision, void* stream) {
    if (!B || !z || !S || !H) return fail(WPCCC_EINVAL, "wpccc_matrix_elements: null argument");
    if (nz < 1) return fail(WPCCC_EINVAL, "wpccc_matrix_elements: nz < 1");
    if (!(b > 0.0) || !(v > 0.0)) return fail(WPCCC_EINVAL, "wpccc_matrix_elements: b and v must be > 0");
    if (precision == 3 || precision == 4) {
        WPCCC_CUDA(cudaSetDevice(B->device));
        wpccc_status ts = tc_prepare(B);
        if (ts != WPCCC_OK) return ts;
    }
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const ElemScratch L = elem_scratch_layout(B);
    // evaluations per launch bounded by the workspace limit
    size_t per = L.bytes_per_eval + sizeof(EvalDesc);
    int chunk = (int)std::min<size_t>({(size_t)nz, (size_t)MAX_EVALS_PER_LAUNCH,
                                       std::max<size_t>(1, (B->ws_limit - 256) / per)});
    size_t need = (size_t)chunk * L.bytes_per_eval + 256 + (size_t)chunk * sizeof(EvalDesc);
    wpccc_status s = ensure_workspace(B, need);
    if (s != WPCCC_OK) return s;
    char* wsb = static_cast<char*>(B->ws_ptr);
    EvalDesc* dev_ev = reinterpret_cast<EvalDesc*>(wsb);
    void* scratch = wsb + ((chunk * sizeof(EvalDesc) + 255) / 256) * 256;
    std::vector<EvalDesc> ev(chunk);
    const size_t mat = (size_t)B->N * B->N;
    for (int k0 = 0; k0 < nz; k0 += chunk) {
        int n = std::min(chunk, nz - k0);
        for (int k = 0; k < n; ++k) ev[k] = EvalDesc{b, v, z[k0 + k], 0, 0};
        WPCCC_CUDA(cudaMemcpyAsync(dev_ev, ev.data(), n * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
        s = launch_elements(B, dev_ev, n, static_cast<double2*>(S) + k0 * mat, static_cast<double2*>(H) + k0 * mat,
                            scratch, st, precision);
        if (s != WPCCC_OK) return s;
        // the host list is reused: wait for the copy before refilling it
        WPCCC_CUDA(cudaStreamSynchronize(st));
    }
    if (precision == 3 || precision == 4) {
        int e = 0;
        WPCCC_CUDA(cudaMemcpy(&e, B->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (e) {
            WPCCC_CUDA(cudaMemset(B->tc_err, 0, sizeof(int)));
            return fail(WPCCC_ETIMEOUT, "a wait of the tensor-core contraction timed out (stage " + std::to_string(e) + ")");
        }
    }
    return WPCCC_OK;
}
}  // namespace wpccc
