// Differentiation form: derivatives of observables P_o = sum_i g[o][i] |c_i|^2 at the end of every path
// with respect to the basis parameters theta (projectile charge, model-potential parameters), by the
// discrete adjoint of Algorithm 1 and of the element assembly.
//
// Notation.  One RK4 step (Algorithm 1, stage form) from c to c':
//   x1 = c, x2 = c + h/2 k1, x3 = c + h/2 k2, x4 = c + h k3,  k_s = M_s x_s,
//   c' = c + h/6 (k1 + 2 k2 + 2 k3 + k4),  M_s = -(i/v) S_s^{-1} H_s  (S, H at z, z_mid, z_mid, z_new).
// With dL = 2 Re(lam'^+ dc') the reverse stages are
//   kb4 = h/6 lam', kb3 = h/3 lam' + h xb4, kb2 = h/3 lam' + h/2 xb3, kb1 = h/6 lam' + h/2 xb2,
//   xi_s = S_s^{-1} kb_s,  xb_s = M_s^+ kb_s = (i/v) H_s xi_s   (S and H are Hermitian),
//   lam = lam' + xb1 + xb2 + xb3 + xb4,
// and every stage adds  2 Re[ -(i/v) xi_s^+ (dH_s) x_s - xi_s^+ (dS_s) k_s ]  to dL/dtheta
// (dM = -(i/v) S^{-1} (dH - dS S^{-1} H) and S^{-1} H x = i v k).
//
// dS and dH never appear as matrices.  Their energy-phase part (i z/v)(d eps_i - d eps_j) X_ij is a
// sum over states of the stage's own vectors (H x, H xi, S k = -(i/v) H x, S xi = kb) and is added by
// the adjoint RK4 kernel.  The rest is the same Eq. 6-9 integrals with one ingredient differentiated;
// each stage needs only the bilinear forms xi^+ dX x, which the element-adjoint kernels evaluate on
// the quadrature nodes: the vectors are rotated into the molecular frame (Eq. 8), projected onto
// the node tables, and combined with the node weights (Eq. 9), O(N G) work per form.
//
// Memory: the forward sweep keeps c every `checkpoint_every` steps; the reverse sweep recomputes S,
// H and the LU factors of one segment (all its paths), replays its steps to record the stage
// vectors, then runs the reverse stages and the element adjoint of that segment.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "geometry.cuh"
#include "rk_device.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

constexpr int ADJ_MAXTAN = 2;   // derivative tables per centre handled by the element adjoint
constexpr int ADJ_LMAX = 6;     // largest l of a basis the element adjoint handles
constexpr int ADJ_NODES = 128;  // quadrature nodes per block of k_adj_mol
constexpr int ADJ_KINDS = 5;    // bilinear forms per stage: K(xi,k), K(k,xi), Q(xi,x), Q(x,xi), Ds(xi,x)

// One stage of one step of one path, for one observable.
struct AdjTerm {
    int pos;      // position within the segment's list
    int slot;     // path slot within the group
    int obs;
    int rec;      // (slot * K + step) * 4 + stage: the x, k, H x records
    int xi;       // rec * n_obs + obs: the xi record
    int pad;
    double v, z;
};

__device__ inline double2 cmulc(double2 a, double2 b) {   // conj(a) * b
    return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// k_rk4_adjoint: one block per path slot.  Phase 1 replays the segment's steps from its checkpoint
// and records x_s, k_s and H_s x_s of every stage; phase 2 runs the reverse stages, records xi_s and
// adds the energy-phase part of the parameter derivatives.
// ---------------------------------------------------------------------------
struct AdjRkArgs {
    int N, n_obs, npar, K;
    const double2* H;        // segment matrices, position e at e * N * N
    const double2* LU;
    const int* piv;
    const int* info;
    const int* slots;        // active slot of each block
    const int* pos0;         // [slots] first position of the slot
    const int* nsteps;       // [slots]
    const double* z;         // [slots][K + 1] node positions of the segment
    const double* v;         // [slots]
    const double2* ckpt;     // [slots][N] amplitudes at the segment start
    double2* lam;            // [slots][n_obs][N] cotangent of c at the segment end (in) / start (out)
    double2 *rx, *rk, *rhx;  // [slots][K][4][N]
    double2* rxi;            // [slots][K][4][n_obs][N]
    const double* deps;      // [npar][N]
    double* gphase;          // [slots][n_obs][npar], accumulated
    int* flags;
};

constexpr int ADJ_RED = 2 * WPCCC_MAX_PARAMS;

__global__ void __launch_bounds__(RK_THREADS) k_rk4_adjoint(AdjRkArgs A) {
    extern __shared__ double2 adj_smem[];
    __shared__ double red[RK_THREADS / 32][ADJ_RED];
    const int N = A.N;
    double2* c = adj_smem;
    double2* y = c + N;
    double2* kv = y + N;
    double2* t = kv + N;
    double2* xb = t + N;
    double2* xs = xb + N;
    double2* lam = xs + N;                       // [n_obs][N]
    double2* blk = lam + (size_t)A.n_obs * N;    // 32 x 32
    const int sl = A.slots[blockIdx.x];
    const int n = A.nsteps[sl], p0 = A.pos0[sl];
    const double v = A.v[sl];
    const double* zs = A.z + (size_t)sl * (A.K + 1);
    const size_t mat = (size_t)N * N;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (A.info && tid == 0) {
        int bad = 0;
        for (int e = 0; e <= 2 * n; ++e)
            if (A.info[p0 + e] != 0) bad = 1;
        if (bad) atomicOr(A.flags, 1);
    }
    auto Hm = [&](int e) { return A.H + (size_t)(p0 + e) * mat; };
    auto Lm = [&](int e) { return A.LU + (size_t)(p0 + e) * mat; };
    auto Pv = [&](int e) { return A.piv + (size_t)(p0 + e) * N; };
    auto stage_pos = [&](int s, int st) { return st == 0 ? 2 * s : (st == 3 ? 2 * s + 2 : 2 * s + 1); };
    auto rec = [&](int s, int st) { return ((size_t)sl * A.K + s) * 4 + st; };

    // ---- phase 1: replay, recording the stage vectors
    for (int i = tid; i < N; i += RK_THREADS) c[i] = A.ckpt[(size_t)sl * N + i];
    __syncthreads();
    for (int s = 0; s < n; ++s) {
        const double h = zs[s + 1] - zs[s];
        const double h2 = 0.5 * h, h6 = h / 6.0;
        for (int i = tid; i < N; i += RK_THREADS) {
            y[i] = c[i];
            xb[i] = make_double2(0.0, 0.0);   // running sum of the stage derivatives
        }
        __syncthreads();
        for (int st = 0; st < 4; ++st) {
            const int e = stage_pos(s, st);
            const size_t r = rec(s, st) * N;
            matvec(Hm(e), N, y, t);
            for (int i = tid; i < N; i += RK_THREADS) {
                A.rhx[r + i] = t[i];
                A.rx[r + i] = y[i];
            }
            __syncthreads();   // the solve permutes t in place
            lu_solve_inplace<double2>(Lm(e), Pv(e), N, t, blk);
            const double hn = st == 2 ? h : h2;
            const double wk = (st == 0 || st == 3) ? 1.0 : 2.0;
            for (int i = tid; i < N; i += RK_THREADS) {
                const double2 k = make_double2(t[i].y / v, -t[i].x / v);
                A.rk[r + i] = k;
                xb[i] = make_double2(fma(wk, k.x, xb[i].x), fma(wk, k.y, xb[i].y));
                if (st < 3) y[i] = make_double2(fma(hn, k.x, c[i].x), fma(hn, k.y, c[i].y));
            }
            __syncthreads();
        }
        for (int i = tid; i < N; i += RK_THREADS) c[i] = make_double2(fma(h6, xb[i].x, c[i].x), fma(h6, xb[i].y, c[i].y));
        __syncthreads();
    }

    // ---- phase 2: reverse stages
    for (int q = tid; q < A.n_obs * N; q += RK_THREADS) lam[q] = A.lam[(size_t)sl * A.n_obs * N + q];
    __syncthreads();
    double gacc[4][WPCCC_MAX_PARAMS] = {};   // thread 0 keeps the per-observable phase contributions
    for (int s = n - 1; s >= 0; --s) {
        const double h = zs[s + 1] - zs[s];
        const double zst[4] = {zs[s], 0.5 * (zs[s] + zs[s + 1]), 0.5 * (zs[s] + zs[s + 1]), zs[s + 1]};
        for (int o = 0; o < A.n_obs; ++o) {
            double2* lo = lam + (size_t)o * N;
            for (int i = tid; i < N; i += RK_THREADS) {
                xs[i] = make_double2(0.0, 0.0);
                xb[i] = make_double2(0.0, 0.0);
            }
            __syncthreads();
            for (int st = 3; st >= 0; --st) {
                const int e = stage_pos(s, st);
                const size_t r = rec(s, st) * N;
                const double cl = (st == 0 || st == 3) ? h / 6.0 : h / 3.0;
                const double cx = st == 3 ? 0.0 : (st == 2 ? h : 0.5 * h);
                // kb = cl lam' + cx xb(previous stage); xi = S^{-1} kb (in t); kb kept in y
                for (int i = tid; i < N; i += RK_THREADS) {
                    const double2 kb = make_double2(fma(cx, xb[i].x, cl * lo[i].x), fma(cx, xb[i].y, cl * lo[i].y));
                    y[i] = kb;
                    t[i] = kb;
                }
                __syncthreads();
                lu_solve_inplace<double2>(Lm(e), Pv(e), N, t, blk);
                matvec(Hm(e), N, t, kv);   // u = H xi
                // energy-phase part: Re A_p and Im B_p with
                //   A = sum_i deps_i (conj(xi_i) (Hx)_i - conj(u_i) x_i)
                //   B = sum_i deps_i (conj(xi_i) (Sk)_i - conj(kb_i) k_i),  S k = -(i/v) H x
                double part[ADJ_RED] = {};
                for (int i = tid; i < N; i += RK_THREADS) {
                    const double2 xi = t[i], u = kv[i], kb = y[i];
                    const double2 hx = A.rhx[r + i], xx = A.rx[r + i], kk = A.rk[r + i];
                    const double2 sk = make_double2(hx.y / v, -hx.x / v);
                    const double2 a1 = cmulc(xi, hx), a2 = cmulc(u, xx);
                    const double2 b1 = cmulc(xi, sk), b2 = cmulc(kb, kk);
                    const double ra = a1.x - a2.x, ib = b1.y - b2.y;
                    for (int p = 0; p < A.npar; ++p) {
                        const double de = A.deps[(size_t)p * N + i];
                        part[2 * p] = fma(de, ra, part[2 * p]);
                        part[2 * p + 1] = fma(de, ib, part[2 * p + 1]);
                    }
                }
                for (int k = 0; k < 2 * A.npar; ++k) {
                    double val = part[k];
                    for (int off = 16; off > 0; off >>= 1) val += __shfl_xor_sync(0xffffffffu, val, off);
                    if (lane == 0) red[warp][k] = val;
                }
                // record xi, then xb = (i/v) u and its running sum
                const size_t rxo = (rec(s, st) * A.n_obs + o) * N;
                for (int i = tid; i < N; i += RK_THREADS) {
                    A.rxi[rxo + i] = t[i];
                    const double2 x = make_double2(-kv[i].y / v, kv[i].x / v);
                    xb[i] = x;
                    xs[i] = cadd(xs[i], x);
                }
                __syncthreads();
                if (tid == 0) {
                    const double z = zst[st];
                    for (int p = 0; p < A.npar; ++p) {
                        double ra = 0.0, ib = 0.0;
                        for (int w = 0; w < RK_THREADS / 32; ++w) {
                            ra += red[w][2 * p];
                            ib += red[w][2 * p + 1];
                        }
                        // 2 Re[(z/v^2) A - (i z/v) B] = 2 (z/v^2) Re A + 2 (z/v) Im B
                        gacc[o][p] += 2.0 * (z / (v * v)) * ra + 2.0 * (z / v) * ib;
                    }
                }
                __syncthreads();
            }
            for (int i = tid; i < N; i += RK_THREADS) lo[i] = cadd(lo[i], xs[i]);
            __syncthreads();
        }
    }
    for (int q = tid; q < A.n_obs * N; q += RK_THREADS) {
        const double2 l = lam[q];
        A.lam[(size_t)sl * A.n_obs * N + q] = l;
        if (!isfinite(l.x) || !isfinite(l.y)) atomicOr(A.flags, 2);
    }
    if (tid == 0)
        for (int o = 0; o < A.n_obs; ++o)
            for (int p = 0; p < A.npar; ++p) A.gphase[((size_t)sl * A.n_obs + o) * A.npar + p] += gacc[o][p];
}

size_t adj_rk_smem_bytes(int N, int n_obs) { return ((size_t)(6 + n_obs) * N + 32 * 32) * sizeof(double2); }

// lam = g o c at the end of the paths, P = g |c|^2
__global__ void k_adj_init(int N, int n_obs, int n_slots, const double* __restrict__ g,
                           const double2* __restrict__ c, double2* __restrict__ lam, double* __restrict__ P) {
    const int sl = blockIdx.x;
    __shared__ double red[32];
    for (int o = 0; o < n_obs; ++o) {
        double acc = 0.0;
        for (int i = threadIdx.x; i < N; i += blockDim.x) {
            const double2 ci = c[(size_t)sl * N + i];
            const double gi = g[(size_t)o * N + i];
            lam[((size_t)sl * n_obs + o) * N + i] = make_double2(gi * ci.x, gi * ci.y);
            acc += gi * (ci.x * ci.x + ci.y * ci.y);
        }
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0 && P) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            P[(size_t)sl * n_obs + o] = s;
        }
        __syncthreads();
    }
    (void)n_slots;
}

// ---------------------------------------------------------------------------
// element adjoint, per position: derivative node tables
//   tn = [dfT at r_T: nT][nradT][G] | [dfP at r_P: nP][nradP][G] | vol[G] | V_s(r_T)[G] | dV_s/dtheta_p[npar][G]
//        | d F/dtheta at R: [nT][nfT] | [nP][nfP]
// ---------------------------------------------------------------------------
struct TanLayout {
    size_t dfT, dfP, vol, Vs, dVs, dFT, dFP, doubles;
};

static TanLayout tan_layout(const wpccc_basis_s* B) {
    TanLayout t;
    const size_t G = B->G;
    t.dfT = 0;
    t.dfP = t.dfT + (size_t)B->tanT.n_tan * B->T.n_rad * G;
    t.vol = t.dfP + (size_t)B->tanP.n_tan * B->P.n_rad * G;
    t.Vs = t.vol + G;
    t.dVs = t.Vs + G;
    t.dFT = t.dVs + (size_t)B->n_par * G;
    t.dFP = t.dFT + (size_t)B->tanT.n_tan * B->T.n_fent;
    t.doubles = t.dFP + (size_t)B->tanP.n_tan * B->P.n_fent;
    t.doubles += t.doubles & 1;
    return t;
}

struct TanNodeArgs {
    int Nr, G, Gtau, nradT, nradP, nT, nP, npar;
    double gamma, mp_c, mp_a, mp_b;
    double dexp[WPCCC_MAX_PARAMS][4];
    const double *r, *inv_den, *s, *ws, *tau, *wtau;
    const double *dfT, *dfP;   // [nT][nradT][Nr], [nP][nradP][Nr]
    double* tn;
    size_t tn_doubles;
    TanLayout L;
};

__global__ void __launch_bounds__(128) k_adj_tan_nodes(TanNodeArgs A, const EvalDesc* __restrict__ ev) {
    const int e = blockIdx.y;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= A.G) return;
    const int k = g / A.Gtau, t = g - k * A.Gtau;
    const double b = ev[e].b, z = ev[e].z;
    const double R = dist_R(b, z);
    const double gR = __dmul_rn(A.gamma, R);
    const double eta = __dadd_rn(1.0, __ddiv_rn(A.s[k], gR));
    const double tau = A.tau[t];
    const double halfR = __dmul_rn(0.5, R);
    const double rT = __dmul_rn(halfR, __dadd_rn(eta, tau));
    const double rP = __dmul_rn(halfR, __dsub_rn(eta, tau));
    const double wgt = (A.ws[k] / gR) * A.wtau[t];
    const double vol = (R * R * R / 8.0) * wgt * (eta * eta - tau * tau);
    double* tn = A.tn + (size_t)e * A.tn_doubles;
    int sT, sP;
    double LT[5], LP[5];
    const bool inT = stencil5_fast(A.r, A.inv_den, A.Nr, rT, sT, LT);
    const bool inP = stencil5_fast(A.r, A.inv_den, A.Nr, rP, sP, LP);
    for (int q = 0; q < A.nT; ++q)
        for (int a = 0; a < A.nradT; ++a) {
            double val = 0.0;
            if (inT) {
                const double* fa = A.dfT + ((size_t)q * A.nradT + a) * A.Nr + sT;
                val = LT[0] * fa[0] + LT[1] * fa[1] + LT[2] * fa[2] + LT[3] * fa[3] + LT[4] * fa[4];
            }
            tn[A.L.dfT + ((size_t)q * A.nradT + a) * A.G + g] = val;
        }
    for (int q = 0; q < A.nP; ++q)
        for (int a = 0; a < A.nradP; ++a) {
            double val = 0.0;
            if (inP) {
                const double* fa = A.dfP + ((size_t)q * A.nradP + a) * A.Nr + sP;
                val = LP[0] * fa[0] + LP[1] * fa[1] + LP[2] * fa[2] + LP[3] * fa[3] + LP[4] * fa[4];
            }
            tn[A.L.dfP + ((size_t)q * A.nradP + a) * A.G + g] = val;
        }
    const double ex = exp(-A.mp_a * rT);
    tn[A.L.vol + g] = vol;
    tn[A.L.Vs + g] = (-A.mp_c * ex) * (1.0 + A.mp_b * rT) / rT;
    for (int p = 0; p < A.npar; ++p) {
        // d V_s / d theta_p through d(c, a, b)/d theta_p, V_s = -c e^{-a r}(1 + b r)/r
        const double dc = A.dexp[p][1], da = A.dexp[p][2], db = A.dexp[p][3];
        const double d = dc * (-ex * (1.0 + A.mp_b * rT) / rT) + da * (A.mp_c * ex * (1.0 + A.mp_b * rT)) +
                         db * (-A.mp_c * ex);
        tn[A.L.dVs + (size_t)p * A.G + g] = d;
    }
}

// derivative Eq. 7 tables interpolated at R (the stencil of k_eval_tables)
struct TanFArgs {
    int Nr, nT, nP, nfT, nfP, dtot, npb;
    const double *dFT, *dFP;
    const double* et;
    size_t et_doubles;
    double* tn;
    size_t tn_doubles;
    TanLayout L;
};

__global__ void __launch_bounds__(256) k_adj_ftan(TanFArgs A) {
    const int e = blockIdx.x;
    const double* st = A.et + (size_t)e * A.et_doubles + A.dtot + A.npb;
    const int s = (int)st[0];
    const bool out = st[1] != 0.0;
    double* tn = A.tn + (size_t)e * A.tn_doubles;
    const int tot = A.nT * A.nfT + A.nP * A.nfP;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        const double* Fe;
        size_t o;
        if (q < A.nT * A.nfT) {
            Fe = A.dFT + (size_t)q * A.Nr;
            o = A.L.dFT + q;
        } else {
            const int q2 = q - A.nT * A.nfT;
            Fe = A.dFP + (size_t)q2 * A.Nr;
            o = A.L.dFP + q2;
        }
        tn[o] = out ? Fe[A.Nr - 1]
                    : st[2] * Fe[s] + st[3] * Fe[s + 1] + st[4] * Fe[s + 2] + st[5] * Fe[s + 3] + st[6] * Fe[s + 4];
    }
}

// ---------------------------------------------------------------------------
// k_adj_vec: per term, the three vectors (xi, x, k) with the energy phases taken out,
//   tv_i = v_i e^{-i eps_i z / v}   (so that xi^+ (X o phases) x = tv_xi^+ X tv_x),
// and rotated into the molecular frame of each centre, mv_(a,q) = sum_m d^{l_a}_{m q}(theta) tv_(a,m).
// ---------------------------------------------------------------------------
struct VecArgs {
    int N, N_T, N_P, n_obs, dtot, pos_first;
    const AdjTerm* terms;
    const double* et;
    size_t et_doubles, ph_off;
    const double2 *rx, *rk, *rxi;
    const double *epsT, *epsP;
    const int *stT_rad, *stT_m, *radT_l, *stT_index;
    const int *stP_rad, *stP_m, *radP_l, *stP_index;
    double2 *tv, *mv;   // [term][3][N]
};

__global__ void __launch_bounds__(256) k_adj_vec(VecArgs A) {
    const AdjTerm T = A.terms[blockIdx.x];
    const int N = A.N;
    const double2* src[3] = {A.rxi + (size_t)T.xi * N, A.rx + (size_t)T.rec * N, A.rk + (size_t)T.rec * N};
    double2* tv = A.tv + (size_t)blockIdx.x * 3 * N;
    double2* mv = A.mv + (size_t)blockIdx.x * 3 * N;
    const double* d = A.et + (size_t)(T.pos - A.pos_first) * A.et_doubles;
    const double2* ph = reinterpret_cast<const double2*>(d + A.ph_off);   // exp(i eps_i z / v)
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const int k = q / N, i = q - k * N;
        tv[q] = cmul(src[k][i], cconj(ph[i]));
    }
    __syncthreads();
    for (int q = threadIdx.x; q < 3 * N; q += blockDim.x) {
        const int k = q / N, i = q - k * N;
        const bool tgt = i < A.N_T;
        const int ii = tgt ? i : i - A.N_T;
        const int a = tgt ? A.stT_rad[ii] : A.stP_rad[ii];
        const int l = tgt ? A.radT_l[a] : A.radP_l[a];
        const int qq = tgt ? A.stT_m[ii] : A.stP_m[ii];
        const int* idx = (tgt ? A.stT_index : A.stP_index) + a * (2 * WPCCC_LMAX + 1) + WPCCC_LMAX;
        const int off = tgt ? 0 : A.N_T;
        int offl = 0;
        for (int j = 0; j < l; ++j) offl += (2 * j + 1) * (2 * j + 1);
        double2 acc = make_double2(0.0, 0.0);
        for (int m = -l; m <= l; ++m) {
            const double w = d[offl + (m + l) * (2 * l + 1) + (qq + l)];
            const double2 x = tv[(size_t)k * N + off + idx[m]];
            acc.x = fma(w, x.x, acc.x);
            acc.y = fma(w, x.y, acc.y);
        }
        mv[q] = acc;
    }
}

// ---------------------------------------------------------------------------
// k_adj_mol: one bilinear form alpha^+ dX beta of a two-centre integral (molecular frame) for every
// parameter, on one tile of quadrature nodes.  Kinds 0/1 K (weight W_K), 2/3 Q (weight W_Q = W_K
// V_T(r_T), and d V_T/d theta times W_K), 4 the short-range D_P part (weight vol V_s, diagonal in q).
// Per node:  a_q'(g) = sum_{i: q_i = q'} conj(alpha_i) f_{a_i}(g) Theta_{l_i q'}(g), the same with the
// derivative table of f, and b_q(g) likewise on the projectile side; then
//   sum_{q', q} W_{|q - q'|}(g) (da_q' b_q + a_q' db_q) [+ dV(g) W_K a_q' b_q].
// ---------------------------------------------------------------------------
struct AdjJob {
    int term;   // term within the sub-batch
    int kind;
    int pos;    // position within the sub-batch
    int va, vb; // vector index (0 xi, 1 x, 2 k) of alpha and beta
};

struct MolAdjArgs {
    int G, N, N_T, N_P, nradT, nradP, nlqT, nlqP, dmax, npar, n_tiles;
    int nT, nP, slotT[WPCCC_MAX_PARAMS], slotP[WPCCC_MAX_PARAMS];
    const int *radT_l, *radP_l, *stT_index, *stP_index;
    const double* node;
    size_t node_doubles, w_off;
    const double* tn;
    size_t tn_doubles;
    TanLayout L;
    const double2* mv;
    const AdjJob* jobs;
    double2* part;   // [job][tile][npar]
};

// Projection of one vector onto the node tables of one centre at node g:
// out[(q + lm) * (1 + nt) + 0] primal, [.. + 1 + k] with derivative table k.
template <int LM>
__device__ inline void adj_project(const double2* vec, bool conj_vec, int nrad, const int* rad_l, const int* st_index,
                                   const double* f, const double* th, const double* df, int nt, int G, int g,
                                   double2 out[2 * LM + 1][1 + ADJ_MAXTAN]) {
    for (int q = 0; q < 2 * LM + 1; ++q)
        for (int k = 0; k <= ADJ_MAXTAN; ++k) out[q][k] = make_double2(0.0, 0.0);
    for (int a = 0; a < nrad; ++a) {
        const int l = rad_l[a];
        const double fv = f[(size_t)a * G + g];
        double dv[ADJ_MAXTAN];
        for (int k = 0; k < nt; ++k) dv[k] = df[((size_t)k * nrad + a) * G + g];
        for (int q = -l; q <= l; ++q) {
            const int aq = q < 0 ? -q : q;
            double thv = th[(size_t)(l * (l + 1) / 2 + aq) * G + g];
            if (q < 0 && (aq & 1)) thv = -thv;
            double2 x = vec[st_index[a * (2 * WPCCC_LMAX + 1) + q + WPCCC_LMAX]];
            if (conj_vec) x.y = -x.y;
            const double A = fv * thv;
            out[q + LM][0].x = fma(A, x.x, out[q + LM][0].x);
            out[q + LM][0].y = fma(A, x.y, out[q + LM][0].y);
            for (int k = 0; k < nt; ++k) {
                const double dA = dv[k] * thv;
                out[q + LM][1 + k].x = fma(dA, x.x, out[q + LM][1 + k].x);
                out[q + LM][1 + k].y = fma(dA, x.y, out[q + LM][1 + k].y);
            }
        }
    }
}

template <int LM>
__global__ void __launch_bounds__(ADJ_NODES) k_adj_mol(MolAdjArgs A) {
    extern __shared__ double2 mvs[];   // alpha then beta
    __shared__ double2 red[ADJ_NODES / 32][WPCCC_MAX_PARAMS];
    const AdjJob J = A.jobs[blockIdx.y];
    const int tile = blockIdx.x;
    const int g = tile * ADJ_NODES + threadIdx.x;
    const bool ds = J.kind == 4;
    const int na = ds ? A.N_P : A.N_T, nb = A.N_P;
    const int offa = ds ? A.N_T : 0;
    const double2* mv = A.mv + (size_t)J.term * 3 * A.N;
    double2* al = mvs;
    double2* be = mvs + na;
    for (int i = threadIdx.x; i < na; i += blockDim.x) al[i] = mv[(size_t)J.va * A.N + offa + i];
    for (int i = threadIdx.x; i < nb; i += blockDim.x) be[i] = mv[(size_t)J.vb * A.N + A.N_T + i];
    __syncthreads();
    double2 val[WPCCC_MAX_PARAMS];
    for (int p = 0; p < WPCCC_MAX_PARAMS; ++p) val[p] = make_double2(0.0, 0.0);
    if (g < A.G) {
        const double* base = A.node + (size_t)J.pos * A.node_doubles;
        const double* fT = base;
        const double* fP = fT + (size_t)A.nradT * A.G;
        const double* thT = fP + (size_t)A.nradP * A.G;
        const double* thP = thT + (size_t)A.nlqT * A.G;
        const double2* W = reinterpret_cast<const double2*>(base + A.w_off);
        const double* tn = A.tn + (size_t)J.pos * A.tn_doubles;
        double2 pa[2 * LM + 1][1 + ADJ_MAXTAN], pb[2 * LM + 1][1 + ADJ_MAXTAN];
        adj_project<LM>(be, false, A.nradP, A.radP_l, A.stP_index, fP, thP, tn + A.L.dfP, A.nP, A.G, g, pb);
        if (!ds) {
            adj_project<LM>(al, true, A.nradT, A.radT_l, A.stT_index, fT, thT, tn + A.L.dfT, A.nT, A.G, g, pa);
            const bool isQ = J.kind >= 2;
            const size_t stride = (size_t)(A.dmax + 1) * A.G;
            const double2* Wx = W + (isQ ? stride : 0);
            // cb[q'] = sum_q W_{|q-q'|} b_q (and with the derivative tables), ck[q'] with W_K (Q only)
            for (int qp = -LM; qp <= LM; ++qp) {
                double2 cb[1 + ADJ_MAXTAN], ck = make_double2(0.0, 0.0);
                for (int k = 0; k <= ADJ_MAXTAN; ++k) cb[k] = make_double2(0.0, 0.0);
                for (int q = -LM; q <= LM; ++q) {
                    const int d = q > qp ? q - qp : qp - q;
                    if (d > A.dmax) continue;
                    const double2 w = Wx[(size_t)d * A.G + g];
                    for (int k = 0; k <= A.nP; ++k) cb[k] = cadd(cb[k], cmul(w, pb[q + LM][k]));
                    if (isQ) ck = cadd(ck, cmul(W[(size_t)d * A.G + g], pb[q + LM][0]));
                }
                const double2 a0 = pa[qp + LM][0];
                for (int p = 0; p < A.npar; ++p) {
                    double2 acc = make_double2(0.0, 0.0);
                    if (A.slotT[p] >= 0) acc = cadd(acc, cmul(pa[qp + LM][1 + A.slotT[p]], cb[0]));
                    if (A.slotP[p] >= 0) acc = cadd(acc, cmul(a0, cb[1 + A.slotP[p]]));
                    if (isQ) acc = cadd(acc, cscale(cmul(a0, ck), tn[A.L.dVs + (size_t)p * A.G + g]));
                    val[p] = cadd(val[p], acc);
                }
            }
        } else {
            adj_project<LM>(al, true, A.nradP, A.radP_l, A.stP_index, fP, thP, tn + A.L.dfP, A.nP, A.G, g, pa);
            const double vol = tn[A.L.vol + g], us = vol * tn[A.L.Vs + g];
            for (int q = -LM; q <= LM; ++q) {
                const double2 c0 = pa[q + LM][0], e0 = pb[q + LM][0];
                const double2 ce = cmul(c0, e0);
                for (int p = 0; p < A.npar; ++p) {
                    double2 acc = cscale(ce, vol * tn[A.L.dVs + (size_t)p * A.G + g]);
                    if (A.slotP[p] >= 0) {
                        const int k = 1 + A.slotP[p];
                        acc = cadd(acc, cscale(cadd(cmul(pa[q + LM][k], e0), cmul(c0, pb[q + LM][k])), us));
                    }
                    val[p] = cadd(val[p], acc);
                }
            }
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < A.npar; ++p) {
        double x = val[p].x, y = val[p].y;
        for (int off = 16; off > 0; off >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, off);
            y += __shfl_xor_sync(0xffffffffu, y, off);
        }
        if (lane == 0) red[warp][p] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < A.npar) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < ADJ_NODES / 32; ++w) s = cadd(s, red[w][threadIdx.x]);
        A.part[((size_t)blockIdx.y * A.n_tiles + tile) * A.npar + threadIdx.x] = s;
    }
}

// ---------------------------------------------------------------------------
// k_adj_direct: the direct blocks' bilinear forms (Eq. 6 with the derivative Eq. 7 tables at R, and
// the explicit projectile-charge factor of D_T).  blockIdx.y = 0: D_T between target states (charge
// Z_P), 1: the Coulomb part of D_P between projectile states (charge Z_T, other nucleus at -R).
// ---------------------------------------------------------------------------
struct DirAdjArgs {
    int Nr, N, N_T, npar, dtot, npb, pos_first, nfT, nfP;
    double Z_T, Z_P;
    double dexp[WPCCC_MAX_PARAMS][4];
    int slotT[WPCCC_MAX_PARAMS], slotP[WPCCC_MAX_PARAMS];
    const AdjTerm* terms;
    const EvalDesc* ev;   // positions of the sub-batch
    const double* r;
    const double* et;
    size_t et_doubles;
    const double* tn;
    size_t tn_doubles;
    TanLayout L;
    // per centre
    int Nc[2], n_rad[2], nlam[2], nt[2];
    const double* ang[2];
    const int* st_lm[2];
    int LM[2];
    const int* Foff[2];
    const int* st_rad[2];
    const int* st_m[2];
    const double2* tv;
    double2* bd;   // [term][2][npar]
};

__global__ void __launch_bounds__(256) k_adj_direct(DirAdjArgs A) {
    const int cen = blockIdx.y;
    const AdjTerm T = A.terms[blockIdx.x];
    const int e = T.pos - A.pos_first;
    const double* et = A.et + (size_t)e * A.et_doubles;
    const double* tn = A.tn + (size_t)e * A.tn_doubles;
    const double* st = et + A.dtot + A.npb;
    const bool out = st[1] != 0.0;
    const double R = dist_R(A.ev[e].b, A.ev[e].z);
    const double ratio = A.r[A.Nr - 1] / R;   // beyond the grid F_lam(R) = F_lam(r_max) (r_max/R)^{lam+1}
    const double* Fint = et + A.dtot + A.npb + 8 + (cen == 0 ? 0 : A.nfT);
    const double* dF = tn + (cen == 0 ? A.L.dFT : A.L.dFP);
    const int Nc = A.Nc[cen], nrad = A.n_rad[cen], nlam = A.nlam[cen], nt = A.nt[cen];
    const int nf = cen == 0 ? A.nfT : A.nfP;
    const int off = cen == 0 ? 0 : A.N_T;
    const double parity = cen == 0 ? 1.0 : -1.0;
    const double2* xi = A.tv + (size_t)blockIdx.x * 3 * A.N + off;
    const double2* xx = xi + A.N;
    __shared__ double2 red[8][WPCCC_MAX_PARAMS];
    double2 acc[WPCCC_MAX_PARAMS];
    for (int p = 0; p < WPCCC_MAX_PARAMS; ++p) acc[p] = make_double2(0.0, 0.0);
    for (long long idx = threadIdx.x; idx < (long long)Nc * Nc; idx += blockDim.x) {
        const int i = (int)(idx / Nc), j = (int)(idx % Nc);
        const int ra = A.st_rad[cen][i], rb = A.st_rad[cen][j];
        const int mu = A.st_m[cen][i] - A.st_m[cen][j];
        const int amu = mu < 0 ? -mu : mu;
        const double* ang = A.ang[cen] + ((size_t)A.st_lm[cen][i] * A.LM[cen] + A.st_lm[cen][j]) * nlam;
        const int* foff = A.Foff[cen] + ((size_t)ra * nrad + rb) * nlam;
        double D1 = 0.0, dD[ADJ_MAXTAN] = {};
        double sgn = 1.0;
        for (int lam = 0; lam < nlam; ++lam, sgn *= parity) {
            const double c = ang[lam];
            if (c == 0.0) continue;
            double P = et[A.dtot + lam * (lam + 1) / 2 + amu];
            if (mu < 0 && (amu & 1)) P = -P;
            double tail = 1.0;
            if (out)
                for (int k = 0; k <= lam; ++k) tail *= ratio;
            const double w = sgn * c * P * tail;
            const int ent = foff[lam];
            D1 = fma(w, Fint[ent], D1);
            for (int k = 0; k < nt; ++k) dD[k] = fma(w, dF[(size_t)k * nf + ent], dD[k]);
        }
        const double2 wij = cmulc(xi[i], xx[j]);
        for (int p = 0; p < A.npar; ++p) {
            double d;
            if (cen == 0) {
                d = -A.dexp[p][0] * D1;
                if (A.slotT[p] >= 0) d -= A.Z_P * dD[A.slotT[p]];
            } else {
                d = A.slotP[p] >= 0 ? -A.Z_T * dD[A.slotP[p]] : 0.0;
            }
            acc[p] = make_double2(fma(d, wij.x, acc[p].x), fma(d, wij.y, acc[p].y));
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int p = 0; p < A.npar; ++p) {
        double x = acc[p].x, y = acc[p].y;
        for (int o = 16; o > 0; o >>= 1) {
            x += __shfl_xor_sync(0xffffffffu, x, o);
            y += __shfl_xor_sync(0xffffffffu, y, o);
        }
        if (lane == 0) red[warp][p] = make_double2(x, y);
    }
    __syncthreads();
    if (threadIdx.x < A.npar) {
        double2 s = make_double2(0.0, 0.0);
        for (int w = 0; w < 8; ++w) s = cadd(s, red[w][threadIdx.x]);
        A.bd[((size_t)blockIdx.x * 2 + cen) * A.npar + threadIdx.x] = s;
    }
}

// Per term and parameter: 2 Im(xi^+ dH x)/v - 2 Re(xi^+ dS k) from the bilinear forms
//   xi^+ dH x = D_T + D_P(Coulomb) + D_P(short range) + Q(xi, x) + conj(Q(x, xi))
//   xi^+ dS k = K(xi, k) + conj(K(k, xi))
__global__ void k_adj_combine(int n_terms, int npar, int n_tiles, const AdjTerm* __restrict__ terms,
                              const double2* __restrict__ part, const double2* __restrict__ bd,
                              double* __restrict__ tg) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n_terms * npar) return;
    const int t = q / npar, p = q - t * npar;
    double2 mol[ADJ_KINDS];
    for (int k = 0; k < ADJ_KINDS; ++k) {
        double2 s = make_double2(0.0, 0.0);
        for (int tile = 0; tile < n_tiles; ++tile)
            s = cadd(s, part[(((size_t)t * ADJ_KINDS + k) * n_tiles + tile) * npar + p]);
        mol[k] = s;
    }
    const double2 dT = bd[((size_t)t * 2 + 0) * npar + p], dP = bd[((size_t)t * 2 + 1) * npar + p];
    const double2 BH = cadd(cadd(cadd(dT, dP), cadd(mol[4], mol[2])), cconj(mol[3]));
    const double2 BS = cadd(mol[0], cconj(mol[1]));
    tg[q] = 2.0 * BH.y / terms[t].v - 2.0 * BS.x;
}

}  // namespace wpccc

// ---------------------------------------------------------------------------
// host driver
// ---------------------------------------------------------------------------
namespace wpccc {

wpccc_status launch_solve(int N, int batch, double2* S, double2* H, int* ipiv, int* info, cudaStream_t st);

namespace {

// Device buffers of one path group, freed on scope exit.
struct DevBufs {
    std::vector<void*> ptrs;
    ~DevBufs() {
        for (void* p : ptrs) cudaFree(p);
    }
    template <class T>
    wpccc_status get(T** out, size_t n, const char* what) {
        void* p = nullptr;
        cudaError_t e = cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T));
        if (e != cudaSuccess) return cuda_fail(e, what);
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return WPCCC_OK;
    }
};

template <int LM>
wpccc_status launch_mol_adj(const MolAdjArgs& a, int n_jobs, size_t smem, cudaStream_t st) {
    WPCCC_CUDA(cudaFuncSetAttribute(k_adj_mol<LM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_adj_mol<LM><<<dim3(a.n_tiles, n_jobs), ADJ_NODES, smem, st>>>(a);
    WPCCC_CHECK_LAUNCH("k_adj_mol");
    return WPCCC_OK;
}

}  // namespace

static wpccc_status adjoint_group(wpccc_basis_s* B, const wpccc_paths* paths, int g0, int gs, const int* zoff,
                                  int n_obs, const double* g_dev, int K, double2* c, double* P_out,
                                  std::vector<double>& grad, cudaStream_t st) {
    const int N = B->N, npar = B->n_par;
    const size_t mat = (size_t)N * N;
    int max_steps = 0;
    for (int q = 0; q < gs; ++q) max_steps = std::max(max_steps, paths->n_z[g0 + q] - 1);
    const int nseg = max_steps == 0 ? 0 : (max_steps + K - 1) / K;
    DevBufs D;
    wpccc_status s;
    double2* lam;
    if ((s = D.get(&lam, (size_t)gs * n_obs * N, "adjoint lam")) != WPCCC_OK) return s;
    // sub-path descriptor of the group, rebuilt per segment
    std::vector<double> sb(gs), sv(gs), sz;
    std::vector<int> snz(gs);
    for (int q = 0; q < gs; ++q) {
        sb[q] = paths->b[g0 + q];
        sv[q] = paths->v[g0 + q];
    }
    auto seg_steps = [&](int q, int seg) {
        const int ns = paths->n_z[g0 + q] - 1;
        return std::max(0, std::min(K, ns - seg * K));
    };
    double2* ckpt = nullptr;
    if (nseg > 0) {
        if ((s = D.get(&ckpt, (size_t)nseg * gs * N, "adjoint checkpoints")) != WPCCC_OK) return s;
    }
    // ---- forward sweep with checkpoints
    for (int seg = 0; seg < nseg; ++seg) {
        WPCCC_CUDA(cudaMemcpyAsync(ckpt + (size_t)seg * gs * N, c, (size_t)gs * N * sizeof(double2),
                                   cudaMemcpyDeviceToDevice, st));
        sz.clear();
        for (int q = 0; q < gs; ++q) {
            const int n = seg_steps(q, seg);
            const double* zp = paths->z + zoff[g0 + q] + seg * K;
            snz[q] = n + 1;
            if (n == 0) {
                sz.push_back(paths->z[zoff[g0 + q]]);
                snz[q] = 1;
            } else {
                sz.insert(sz.end(), zp, zp + n + 1);
            }
        }
        wpccc_paths sub{gs, sb.data(), sv.data(), snz.data(), sz.data()};
        if ((s = propagate_internal(B, &sub, 0, c, st)) != WPCCC_OK) return s;
    }
    // ---- observables and the cotangent at the end
    k_adj_init<<<gs, 256, 0, st>>>(N, n_obs, gs, g_dev, c, lam, P_out ? P_out + (size_t)g0 * n_obs : nullptr);
    WPCCC_CHECK_LAUNCH("k_adj_init");
    if (nseg == 0) {
        WPCCC_CUDA(cudaStreamSynchronize(st));
        return WPCCC_OK;
    }
    // ---- buffers of one segment
    const int max_pos = gs * (2 * K + 1);
    double2 *segS, *segH, *rx, *rk, *rhx, *rxi;
    int *piv, *info, *d_slots, *d_pos0, *d_nst, *flags;
    double *d_z, *d_v, *gphase;
    EvalDesc* d_ev;
    if ((s = D.get(&segS, (size_t)max_pos * mat, "adjoint S")) != WPCCC_OK) return s;
    if ((s = D.get(&segH, (size_t)max_pos * mat, "adjoint H")) != WPCCC_OK) return s;
    if ((s = D.get(&piv, (size_t)max_pos * N, "adjoint piv")) != WPCCC_OK) return s;
    if ((s = D.get(&info, (size_t)max_pos, "adjoint info")) != WPCCC_OK) return s;
    if ((s = D.get(&rx, (size_t)gs * K * 4 * N, "adjoint rx")) != WPCCC_OK) return s;
    if ((s = D.get(&rk, (size_t)gs * K * 4 * N, "adjoint rk")) != WPCCC_OK) return s;
    if ((s = D.get(&rhx, (size_t)gs * K * 4 * N, "adjoint rhx")) != WPCCC_OK) return s;
    if ((s = D.get(&rxi, (size_t)gs * K * 4 * n_obs * N, "adjoint rxi")) != WPCCC_OK) return s;
    if ((s = D.get(&d_slots, (size_t)gs, "adjoint slots")) != WPCCC_OK) return s;
    if ((s = D.get(&d_pos0, (size_t)gs, "adjoint pos0")) != WPCCC_OK) return s;
    if ((s = D.get(&d_nst, (size_t)gs, "adjoint nsteps")) != WPCCC_OK) return s;
    if ((s = D.get(&flags, 1, "adjoint flags")) != WPCCC_OK) return s;
    if ((s = D.get(&d_z, (size_t)gs * (K + 1), "adjoint z")) != WPCCC_OK) return s;
    if ((s = D.get(&d_v, (size_t)gs, "adjoint v")) != WPCCC_OK) return s;
    if ((s = D.get(&gphase, (size_t)gs * n_obs * npar, "adjoint gphase")) != WPCCC_OK) return s;
    if ((s = D.get(&d_ev, (size_t)max_pos, "adjoint positions")) != WPCCC_OK) return s;
    WPCCC_CUDA(cudaMemsetAsync(gphase, 0, (size_t)gs * n_obs * npar * sizeof(double), st));
    WPCCC_CUDA(cudaMemsetAsync(flags, 0, sizeof(int), st));
    WPCCC_CUDA(cudaMemcpyAsync(d_v, sv.data(), gs * sizeof(double), cudaMemcpyHostToDevice, st));
    // element-adjoint sub-batches: positions per launch and the scratch they need
    const ElemScratch EL = elem_scratch_layout(B);
    const TanLayout TL = tan_layout(B);
    const int NB = std::max(1, std::min(max_pos, 256));
    const int n_tiles = (B->G + ADJ_NODES - 1) / ADJ_NODES;
    const int max_terms = NB * 2 * n_obs;
    double2 *tv, *mv, *part, *bd;
    double *tg, *tnode;
    AdjTerm* d_terms;
    AdjJob* d_jobs;
    if ((s = D.get(&tv, (size_t)max_terms * 3 * N, "adjoint tv")) != WPCCC_OK) return s;
    if ((s = D.get(&mv, (size_t)max_terms * 3 * N, "adjoint mv")) != WPCCC_OK) return s;
    if ((s = D.get(&part, (size_t)max_terms * ADJ_KINDS * n_tiles * npar, "adjoint part")) != WPCCC_OK) return s;
    if ((s = D.get(&bd, (size_t)max_terms * 2 * npar, "adjoint bd")) != WPCCC_OK) return s;
    if ((s = D.get(&tg, (size_t)max_terms * npar, "adjoint tg")) != WPCCC_OK) return s;
    if ((s = D.get(&tnode, (size_t)NB * TL.doubles, "adjoint node derivatives")) != WPCCC_OK) return s;
    if ((s = D.get(&d_terms, (size_t)max_pos * 2 * n_obs, "adjoint terms")) != WPCCC_OK) return s;
    if ((s = D.get(&d_jobs, (size_t)max_terms * ADJ_KINDS, "adjoint jobs")) != WPCCC_OK) return s;
    if ((s = ensure_workspace(B, (size_t)NB * EL.bytes_per_eval)) != WPCCC_OK) return s;
    double* node = static_cast<double*>(B->ws_ptr);
    const int adj_smem = (int)adj_rk_smem_bytes(N, n_obs);
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, adj_smem));
    int LMX = std::max(B->T.lmax, B->P.lmax);

    std::vector<EvalDesc> ev;
    std::vector<int> pos0(gs), nst(gs), slots;
    std::vector<double> zseg((size_t)gs * (K + 1));
    std::vector<AdjTerm> terms;
    std::vector<double> h_tg;
    std::vector<double> gel((size_t)gs * n_obs * npar, 0.0);
    for (int seg = nseg - 1; seg >= 0; --seg) {
        ev.clear();
        slots.clear();
        terms.clear();
        for (int q = 0; q < gs; ++q) {
            const int n = seg_steps(q, seg);
            nst[q] = n;
            pos0[q] = (int)ev.size();
            if (n == 0) continue;
            slots.push_back(q);
            const double* zp = paths->z + zoff[g0 + q] + seg * K;
            for (int k = 0; k <= n; ++k) zseg[(size_t)q * (K + 1) + k] = zp[k];
            ev.push_back(EvalDesc{sb[q], sv[q], zp[0], q, 0});
            for (int k = 0; k < n; ++k) {
                ev.push_back(EvalDesc{sb[q], sv[q], (zp[k] + zp[k + 1]) / 2.0, q, 0});
                ev.push_back(EvalDesc{sb[q], sv[q], zp[k + 1], q, 0});
            }
            // terms in position order: position 2s holds stage 4 of step s-1 and stage 1 of step s,
            // 2s+1 stages 2 and 3 of step s
            for (int lp = 0; lp <= 2 * n; ++lp) {
                int use[2][2], nu = 0;
                if (lp & 1) {
                    use[nu][0] = lp / 2; use[nu++][1] = 1;
                    use[nu][0] = lp / 2; use[nu++][1] = 2;
                } else {
                    const int sn = lp / 2;
                    if (sn > 0) { use[nu][0] = sn - 1; use[nu++][1] = 3; }
                    if (sn < n) { use[nu][0] = sn; use[nu++][1] = 0; }
                }
                for (int u = 0; u < nu; ++u)
                    for (int o = 0; o < n_obs; ++o) {
                        AdjTerm t;
                        t.pos = pos0[q] + lp;
                        t.slot = q;
                        t.obs = o;
                        t.rec = (q * K + use[u][0]) * 4 + use[u][1];
                        t.xi = t.rec * n_obs + o;
                        t.pad = 0;
                        t.v = sv[q];
                        t.z = ev[pos0[q] + lp].z;
                        terms.push_back(t);
                    }
            }
        }
        const int npos = (int)ev.size();
        if (npos == 0) continue;
        WPCCC_CUDA(cudaMemcpyAsync(d_ev, ev.data(), npos * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
        WPCCC_CUDA(cudaMemcpyAsync(d_pos0, pos0.data(), gs * sizeof(int), cudaMemcpyHostToDevice, st));
        WPCCC_CUDA(cudaMemcpyAsync(d_nst, nst.data(), gs * sizeof(int), cudaMemcpyHostToDevice, st));
        WPCCC_CUDA(cudaMemcpyAsync(d_slots, slots.data(), slots.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        WPCCC_CUDA(cudaMemcpyAsync(d_z, zseg.data(), zseg.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        WPCCC_CUDA(cudaMemcpyAsync(d_terms, terms.data(), terms.size() * sizeof(AdjTerm), cudaMemcpyHostToDevice, st));
        // S, H and the LU factors of every position of the segment
        for (int p0 = 0; p0 < npos; p0 += NB) {
            const int nb = std::min(NB, npos - p0);
            if ((s = launch_elements(B, d_ev + p0, nb, segS + (size_t)p0 * mat, segH + (size_t)p0 * mat, B->ws_ptr, st,
                                     0)) != WPCCC_OK)
                return s;
            if ((s = launch_solve(N, nb, segS + (size_t)p0 * mat, nullptr, piv + (size_t)p0 * N, info + p0, st)) !=
                WPCCC_OK)
                return s;
        }
        // replay and reverse stages
        AdjRkArgs ra;
        ra.N = N;
        ra.n_obs = n_obs;
        ra.npar = npar;
        ra.K = K;
        ra.H = segH;
        ra.LU = segS;
        ra.piv = piv;
        ra.info = info;
        ra.slots = d_slots;
        ra.pos0 = d_pos0;
        ra.nsteps = d_nst;
        ra.z = d_z;
        ra.v = d_v;
        ra.ckpt = ckpt + (size_t)seg * gs * N;
        ra.lam = lam;
        ra.rx = rx;
        ra.rk = rk;
        ra.rhx = rhx;
        ra.rxi = rxi;
        ra.deps = B->deps;
        ra.gphase = gphase;
        ra.flags = flags;
        cudaEvent_t pa = B->prof.begin(PROF_ADJ, st);
        k_rk4_adjoint<<<(unsigned)slots.size(), RK_THREADS, adj_smem, st>>>(ra);
        WPCCC_CHECK_LAUNCH("k_rk4_adjoint");
        B->prof.end(PROF_ADJ, st, pa);
        // element adjoint, sub-batch by sub-batch of positions
        size_t t0 = 0;
        for (int p0 = 0; p0 < npos; p0 += NB) {
            const int nb = std::min(NB, npos - p0);
            size_t t1 = t0;
            while (t1 < terms.size() && terms[t1].pos < p0 + nb) ++t1;
            const int nt = (int)(t1 - t0);
            if (nt == 0) continue;
            if ((s = launch_node_stage(B, d_ev + p0, nb, B->ws_ptr, st)) != WPCCC_OK) return s;
            // the per-position tables follow the node tables and the (unused) molecular-frame blocks
            double* et = node + EL.node_doubles * nb + EL.mol_elems * nb * 2;
            cudaEvent_t pe = B->prof.begin(PROF_ADJ, st);
            TanNodeArgs tna;
            tna.Nr = B->Nr;
            tna.G = B->G;
            tna.Gtau = B->Gtau;
            tna.nradT = B->T.n_rad;
            tna.nradP = B->P.n_rad;
            tna.nT = B->tanT.n_tan;
            tna.nP = B->tanP.n_tan;
            tna.npar = npar;
            tna.gamma = B->gamma;
            tna.mp_c = B->mp_c;
            tna.mp_a = B->mp_a;
            tna.mp_b = B->mp_b;
            std::memcpy(tna.dexp, B->dexp, sizeof(tna.dexp));
            tna.r = B->r;
            tna.inv_den = B->inv_den;
            tna.s = B->s;
            tna.ws = B->ws;
            tna.tau = B->tau;
            tna.wtau = B->wtau;
            tna.dfT = B->tanT.df;
            tna.dfP = B->tanP.df;
            tna.tn = tnode;
            tna.tn_doubles = TL.doubles;
            tna.L = TL;
            k_adj_tan_nodes<<<dim3((B->G + 127) / 128, nb), 128, 0, st>>>(tna, d_ev + p0);
            WPCCC_CHECK_LAUNCH("k_adj_tan_nodes");
            TanFArgs tfa;
            tfa.Nr = B->Nr;
            tfa.nT = B->tanT.n_tan;
            tfa.nP = B->tanP.n_tan;
            tfa.nfT = B->T.n_fent;
            tfa.nfP = B->P.n_fent;
            tfa.dtot = EL.dtot;
            tfa.npb = EL.npb;
            tfa.dFT = B->tanT.dF;
            tfa.dFP = B->tanP.dF;
            tfa.et = et;
            tfa.et_doubles = EL.et_doubles;
            tfa.tn = tnode;
            tfa.tn_doubles = TL.doubles;
            tfa.L = TL;
            k_adj_ftan<<<nb, 256, 0, st>>>(tfa);
            WPCCC_CHECK_LAUNCH("k_adj_ftan");
            VecArgs va;
            va.N = N;
            va.N_T = B->N_T;
            va.N_P = B->N_P;
            va.n_obs = n_obs;
            va.dtot = EL.dtot;
            va.pos_first = p0;
            va.terms = d_terms + t0;
            va.et = et;
            va.et_doubles = EL.et_doubles;
            va.ph_off = EL.ph_off;
            va.rx = rx;
            va.rk = rk;
            va.rxi = rxi;
            va.epsT = B->T.st_eps;
            va.epsP = B->P.st_eps;
            va.stT_rad = B->T.st_rad;
            va.stT_m = B->T.st_m;
            va.radT_l = B->T.rad_l;
            va.stT_index = B->T.st_index;
            va.stP_rad = B->P.st_rad;
            va.stP_m = B->P.st_m;
            va.radP_l = B->P.rad_l;
            va.stP_index = B->P.st_index;
            va.tv = tv;
            va.mv = mv;
            k_adj_vec<<<nt, 256, 0, st>>>(va);
            WPCCC_CHECK_LAUNCH("k_adj_vec");
            // five bilinear forms per term: K(xi,k), K(k,xi), Q(xi,x), Q(x,xi), Ds(xi,x)
            std::vector<AdjJob> jobs((size_t)nt * ADJ_KINDS);
            const int vab[ADJ_KINDS][2] = {{0, 2}, {2, 0}, {0, 1}, {1, 0}, {0, 1}};
            for (int t = 0; t < nt; ++t)
                for (int k = 0; k < ADJ_KINDS; ++k) {
                    AdjJob& j = jobs[(size_t)t * ADJ_KINDS + k];
                    j.term = t;
                    j.kind = k;
                    j.pos = terms[t0 + t].pos - p0;
                    j.va = vab[k][0];
                    j.vb = vab[k][1];
                }
            WPCCC_CUDA(cudaMemcpyAsync(d_jobs, jobs.data(), jobs.size() * sizeof(AdjJob), cudaMemcpyHostToDevice, st));
            MolAdjArgs ma;
            ma.G = B->G;
            ma.N = N;
            ma.N_T = B->N_T;
            ma.N_P = B->N_P;
            ma.nradT = B->T.n_rad;
            ma.nradP = B->P.n_rad;
            ma.nlqT = B->nlq_T;
            ma.nlqP = B->nlq_P;
            ma.dmax = B->dmax;
            ma.npar = npar;
            ma.n_tiles = n_tiles;
            ma.nT = B->tanT.n_tan;
            ma.nP = B->tanP.n_tan;
            for (int p = 0; p < WPCCC_MAX_PARAMS; ++p) {
                ma.slotT[p] = p < npar ? B->tanT.slot[p] : -1;
                ma.slotP[p] = p < npar ? B->tanP.slot[p] : -1;
            }
            ma.radT_l = B->T.rad_l;
            ma.radP_l = B->P.rad_l;
            ma.stT_index = B->T.st_index;
            ma.stP_index = B->P.st_index;
            ma.node = node;
            ma.node_doubles = EL.node_doubles;
            ma.w_off = EL.w_off;
            ma.tn = tnode;
            ma.tn_doubles = TL.doubles;
            ma.L = TL;
            ma.mv = mv;
            ma.jobs = d_jobs;
            ma.part = part;
            const size_t msm = (size_t)(std::max(B->N_T, B->N_P) + B->N_P) * sizeof(double2);
            const int nj = nt * ADJ_KINDS;
            switch (LMX) {
                case 0:
                case 1: s = launch_mol_adj<1>(ma, nj, msm, st); break;
                case 2: s = launch_mol_adj<2>(ma, nj, msm, st); break;
                case 3: s = launch_mol_adj<3>(ma, nj, msm, st); break;
                case 4: s = launch_mol_adj<4>(ma, nj, msm, st); break;
                case 5: s = launch_mol_adj<5>(ma, nj, msm, st); break;
                default: s = launch_mol_adj<6>(ma, nj, msm, st); break;
            }
            if (s != WPCCC_OK) return s;
            DirAdjArgs da;
            da.Nr = B->Nr;
            da.N = N;
            da.N_T = B->N_T;
            da.npar = npar;
            da.dtot = EL.dtot;
            da.npb = EL.npb;
            da.pos_first = p0;
            da.nfT = B->T.n_fent;
            da.nfP = B->P.n_fent;
            da.Z_T = B->T.Z;
            da.Z_P = B->P.Z;
            std::memcpy(da.dexp, B->dexp, sizeof(da.dexp));
            for (int p = 0; p < WPCCC_MAX_PARAMS; ++p) {
                da.slotT[p] = ma.slotT[p];
                da.slotP[p] = ma.slotP[p];
            }
            da.terms = d_terms + t0;
            da.ev = d_ev + p0;
            da.r = B->r;
            da.et = et;
            da.et_doubles = EL.et_doubles;
            da.tn = tnode;
            da.tn_doubles = TL.doubles;
            da.L = TL;
            const CentreDev* cs[2] = {&B->T, &B->P};
            const CentreTan* ts[2] = {&B->tanT, &B->tanP};
            for (int k = 0; k < 2; ++k) {
                da.Nc[k] = cs[k]->n_states;
                da.n_rad[k] = cs[k]->n_rad;
                da.nlam[k] = cs[k]->nlam;
                da.nt[k] = ts[k]->n_tan;
                da.ang[k] = cs[k]->ang;
                da.st_lm[k] = cs[k]->st_lm;
                da.LM[k] = cs[k]->LM;
                da.Foff[k] = cs[k]->Foff;
                da.st_rad[k] = cs[k]->st_rad;
                da.st_m[k] = cs[k]->st_m;
            }
            da.tv = tv;
            da.bd = bd;
            k_adj_direct<<<dim3(nt, 2), 256, 0, st>>>(da);
            WPCCC_CHECK_LAUNCH("k_adj_direct");
            k_adj_combine<<<(nt * npar + 127) / 128, 128, 0, st>>>(nt, npar, n_tiles, d_terms + t0, part, bd, tg);
            WPCCC_CHECK_LAUNCH("k_adj_combine");
            B->prof.end(PROF_ADJ, st, pe);
            h_tg.resize((size_t)nt * npar);
            WPCCC_CUDA(cudaMemcpyAsync(h_tg.data(), tg, h_tg.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
            WPCCC_CUDA(cudaStreamSynchronize(st));
            for (int t = 0; t < nt; ++t) {
                const AdjTerm& T = terms[t0 + t];
                for (int p = 0; p < npar; ++p) gel[((size_t)T.slot * n_obs + T.obs) * npar + p] += h_tg[(size_t)t * npar + p];
            }
            t0 = t1;
        }
    }
    std::vector<double> gph((size_t)gs * n_obs * npar);
    int hflags = 0;
    WPCCC_CUDA(cudaMemcpyAsync(gph.data(), gphase, gph.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaMemcpyAsync(&hflags, flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaStreamSynchronize(st));
    if (hflags & 1) return fail(WPCCC_ESINGULAR, "wpccc_propagate_adjoint: an overlap matrix had a zero pivot");
    if (hflags & 2) return fail(WPCCC_ENONFINITE, "wpccc_propagate_adjoint: the adjoint became non-finite");
    for (size_t k = 0; k < gph.size(); ++k) grad[(size_t)g0 * n_obs * npar + k] = gph[k] + gel[k];
    return WPCCC_OK;
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_propagate_adjoint(wpccc_basis B, const wpccc_paths* paths, int n_obs, const double* g,
                                                int K, void* c, double* P, double* grad, void* stream) {
    if (!B || !paths || !g || !c || !grad) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: null argument");
    if (B->n_centres != 2) return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate_adjoint: two-centre bases only");
    if (B->n_par < 1) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: call wpccc_basis_set_tangents first");
    if (n_obs < 1 || n_obs > 4) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: n_obs must be 1..4");
    if (K < 1) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: checkpoint_every must be >= 1");
    if (std::max(B->T.lmax, B->P.lmax) > ADJ_LMAX)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate_adjoint: l above 6");
    if (B->tanT.n_tan > ADJ_MAXTAN || B->tanP.n_tan > ADJ_MAXTAN)
        return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate_adjoint: more than 2 derivative tables on one centre");
    const int N = B->N;
    if (adj_rk_smem_bytes(N, n_obs) + 2048 > (size_t)227 * 1024)
        return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: N too large for the adjoint RK4 kernel");
    const int np = paths->n_paths;
    if (np < 1 || !paths->b || !paths->v || !paths->n_z || !paths->z)
        return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: empty or null path description");
    std::vector<int> zoff(np + 1, 0);
    for (int p = 0; p < np; ++p) {
        if (!(paths->b[p] > 0.0) || !(paths->v[p] > 0.0))
            return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: b and v must be > 0");
        if (paths->n_z[p] < 1) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: n_z < 1");
        zoff[p + 1] = zoff[p] + paths->n_z[p];
        for (int k = zoff[p] + 1; k < zoff[p + 1]; ++k)
            if (!(paths->z[k] > paths->z[k - 1]))
                return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: z nodes must increase strictly");
    }
    for (int k = 0; k < n_obs * N; ++k)
        if (!std::isfinite(g[k])) return fail(WPCCC_EINVAL, "wpccc_propagate_adjoint: non-finite weights");
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    double* g_dev = nullptr;
    WPCCC_CUDA(cudaMalloc(&g_dev, (size_t)n_obs * N * sizeof(double)));
    cudaError_t e = cudaMemcpyAsync(g_dev, g, (size_t)n_obs * N * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFree(g_dev);
        return cuda_fail(e, "wpccc_propagate_adjoint: weights");
    }
    // paths per group: one segment's S, H and records of every path of the group within twice the
    // workspace limit
    const int K_eff = K;
    const size_t per_path = (size_t)(2 * K_eff + 1) * ((size_t)N * N * 2 * sizeof(double2) + N * sizeof(int)) +
                            (size_t)K_eff * 4 * (3 + n_obs) * N * sizeof(double2);
    const int gsz = (int)std::max<size_t>(1, std::min<size_t>((size_t)np, 2 * B->ws_limit / per_path));
    std::vector<double> hgrad((size_t)np * n_obs * B->n_par, 0.0);
    wpccc_status s = WPCCC_OK;
    for (int g0 = 0; g0 < np && s == WPCCC_OK; g0 += gsz) {
        const int gs = std::min(gsz, np - g0);
        s = adjoint_group(B, paths, g0, gs, zoff.data(), n_obs, g_dev, K_eff,
                          static_cast<double2*>(c) + (size_t)g0 * N, P, hgrad, st);
    }
    if (s == WPCCC_OK) {
        e = cudaMemcpyAsync(grad, hgrad.data(), hgrad.size() * sizeof(double), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) s = cuda_fail(e, "wpccc_propagate_adjoint: gradient copy");
    }
    cudaStreamSynchronize(st);
    cudaFree(g_dev);
    return s;
}
