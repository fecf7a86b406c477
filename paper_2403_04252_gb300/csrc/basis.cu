// Basis set-up: upload of the generated inputs and the z-independent tables,
// built once per basis and kept in device memory (Sec. II keeps the same
// quantities resident on the GPU before the equations are integrated).
//   * Eq. 7 radial multipole integrals F_{ab lam}(r_i) at every grid radius
//   * Eq. 6 angular coefficients sqrt((2l+1)/(2l'+1)) C^{l'0}_{lam0 l0} C^{l'm'}_{lam mu lm}
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "angular.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

wpccc_status fail(wpccc_status st, const std::string& msg) {
    g_last_error = msg;
    return st;
}

wpccc_status cuda_fail(cudaError_t e, const char* what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? WPCCC_ENOMEM : WPCCC_ECUDA;
}

// ---------------------------------------------------------------------------
// profiler
// ---------------------------------------------------------------------------
cudaEvent_t Profiler::begin(int cat, cudaStream_t st) {
    ++launches[cat];
    if (!on) return nullptr;
    cudaEvent_t e;
    if (pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    } else {
        e = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(e, st);
    return e;
}

void Profiler::end(int cat, cudaStream_t st, cudaEvent_t e0) {
    if (!on || !e0) return;
    cudaEvent_t e;
    if (pool.empty()) {
        if (cudaEventCreate(&e) != cudaSuccess) {
            pool.push_back(e0);
            return;
        }
    } else {
        e = pool.back();
        pool.pop_back();
    }
    cudaEventRecord(e, st);
    pending[cat].push_back(e0);
    pending[cat].push_back(e);
}

cudaError_t Profiler::flush() {
    cudaError_t err = cudaSuccess;
    for (int c = 0; c < WPCCC_PROF_N; ++c) {
        for (size_t k = 0; k + 1 < pending[c].size(); k += 2) {
            float t = 0.f;
            cudaError_t e = cudaEventSynchronize(pending[c][k + 1]);
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, pending[c][k], pending[c][k + 1]);
            if (e != cudaSuccess) err = e;
            ms[c] += t;
            pool.push_back(pending[c][k]);
            pool.push_back(pending[c][k + 1]);
        }
        pending[c].clear();
    }
    return err;
}

void Profiler::release() {
    flush();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
    pool.clear();
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
__device__ inline double ipow(double x, int n) {
    double p = 1.0;
    for (int k = 0; k < n; ++k) p *= x;
    return p;
}

// F_{ab lam}(r_i) = r_i^{-lam-1} sum_{j<=i} g_j r_j^lam + r_i^lam sum_{j>i} g_j r_j^{-lam-1},
// g_j = w_j r_j^2 f_a(r_j) f_b(r_j): Eq. 7 on the grid's own rule, split at r = R = r_i.
// One block per table entry; the two sums are a forward and a backward block scan.
// With derivative tables df (differentiation form), g_j = w_j r_j^2 (df_a f_b + f_a df_b): the
// derivative of the table, which is bilinear in the two radial functions.
__device__ inline double fpair(const double* fa, const double* fb, const double* dfa, const double* dfb, int j) {
    return dfa ? dfa[j] * fb[j] + fa[j] * dfb[j] : fa[j] * fb[j];
}

__global__ void __launch_bounds__(256) k_ftable(int Nr, const double* __restrict__ r,
                                                const double* __restrict__ w,
                                                const double* __restrict__ f,
                                                const int* __restrict__ ea, const int* __restrict__ eb,
                                                const int* __restrict__ elam, double* __restrict__ F,
                                                const double* __restrict__ df = nullptr) {
    __shared__ double s_fwd[256], s_bwd[256];
    const int e = blockIdx.x, tid = threadIdx.x;
    const int a = ea[e], b = eb[e], lam = elam[e];
    const double* fa = f + (size_t)a * Nr;
    const double* fb = f + (size_t)b * Nr;
    const double* dfa = df ? df + (size_t)a * Nr : nullptr;
    const double* dfb = df ? df + (size_t)b * Nr : nullptr;
    double* out = F + (size_t)e * Nr;
    const int chunk = (Nr + 255) / 256;
    const int j0 = min(Nr, tid * chunk), j1 = min(Nr, j0 + chunk);
    double sa = 0.0, sb = 0.0;
    for (int j = j0; j < j1; ++j) {
        double rj = r[j];
        double g = w[j] * rj * rj * fpair(fa, fb, dfa, dfb, j);
        double rl = ipow(rj, lam);
        sa += g * rl;
        sb += g / (rl * rj);
    }
    s_fwd[tid] = sa;
    s_bwd[tid] = sb;
    __syncthreads();
    if (tid == 0) {
        double run = 0.0;
        for (int t = 0; t < 256; ++t) {  // exclusive forward
            double v = s_fwd[t];
            s_fwd[t] = run;
            run += v;
        }
        run = 0.0;
        for (int t = 255; t >= 0; --t) {  // exclusive backward
            double v = s_bwd[t];
            s_bwd[t] = run;
            run += v;
        }
    }
    __syncthreads();
    double acc = s_fwd[tid];
    for (int j = j0; j < j1; ++j) {
        double rj = r[j];
        acc += w[j] * rj * rj * fpair(fa, fb, dfa, dfb, j) * ipow(rj, lam);
        out[j] = acc;  // inclusive inner sum, finished below
    }
    double accb = s_bwd[tid];
    for (int j = j1 - 1; j >= j0; --j) {
        double rj = r[j];
        double rl = ipow(rj, lam);
        double inner = out[j];
        out[j] = inner / (rl * rj) + rl * accb;
        accb += w[j] * rj * rj * fpair(fa, fb, dfa, dfb, j) / (rl * rj);
    }
}

// 1 / prod_{c != a} (r_{s+a} - r_{s+c}) for every 5-point stencil start s.
__global__ void k_lagrange_den(int Nr, const double* __restrict__ r, double* __restrict__ inv_den) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s > Nr - 5) return;
    for (int a = 0; a < 5; ++a) {
        double p = 1.0;
        for (int c = 0; c < 5; ++c)
            if (c != a) p *= r[s + a] - r[s + c];
        inv_den[(size_t)s * 5 + a] = 1.0 / p;
    }
}

// Eq. 6 angular factor per pair of angular parts ((l', m'), (l, m)) and lam, without
// sqrt((lam-mu)!/(lam+mu)!); angular index l^2 + l + m.
__global__ void k_direct_angular(int LM, int nlam, double* __restrict__ ang) {
    long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)LM * LM) return;
    const int a = (int)(idx / LM), b2 = (int)(idx % LM);
    int lp = 0, l = 0;
    while ((lp + 1) * (lp + 1) <= a) ++lp;
    while ((l + 1) * (l + 1) <= b2) ++l;
    const int mp = a - lp * lp - lp, m = b2 - l * l - l;
    int mu = mp - m;
    double pre = sqrt((2.0 * l + 1.0) / (2.0 * lp + 1.0));
    for (int lam = 0; lam < nlam; ++lam) {
        double v = 0.0;
        if (lam >= abs(lp - l) && lam <= lp + l && ((lp + l + lam) & 1) == 0 && abs(mu) <= lam)
            v = pre * clebsch_gordan(lam, 0, l, 0, lp, 0) * clebsch_gordan(lam, mu, l, m, lp, mp);
        ang[idx * nlam + lam] = v;
    }
}

// ---------------------------------------------------------------------------
// host helpers
// ---------------------------------------------------------------------------
template <class T>
static wpccc_status upload(T** dst, const T* src, size_t n, const char* what) {
    *dst = nullptr;
    if (n == 0) return WPCCC_OK;
    WPCCC_CUDA(cudaMalloc((void**)dst, n * sizeof(T)));
    if (src) {
        cudaError_t e = cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, what);
    }
    return WPCCC_OK;
}

static void free_centre(CentreDev& c) {
    void* ptrs[] = {c.f, c.rad_l, c.st_rad, c.st_l, c.st_m, c.st_eps, c.st_index,
                    c.F, c.Foff, c.fent_a, c.fent_b, c.fent_lam, c.ang, c.st_lm};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    c = CentreDev();
}

static bool all_finite(const double* x, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

static wpccc_status check_centre(const wpccc_centre_desc& d, int Nr, bool all_m, const char* name) {
    std::string n(name);
    if (d.n_rad < 1 || !d.rad_l || !d.f) return fail(WPCCC_EINVAL, n + ": n_rad < 1 or null rad_l/f");
    if (d.n_states < 1 || !d.st_rad || !d.st_m || !d.st_eps)
        return fail(WPCCC_EINVAL, n + ": n_states < 1 or null state arrays");
    if (!std::isfinite(d.Z)) return fail(WPCCC_EINVAL, n + ": non-finite charge");
    if (!all_finite(d.f, (size_t)d.n_rad * Nr)) return fail(WPCCC_EINVAL, n + ": non-finite radial table");
    if (!all_finite(d.st_eps, (size_t)d.n_states)) return fail(WPCCC_EINVAL, n + ": non-finite state energy");
    for (int a = 0; a < d.n_rad; ++a)
        if (d.rad_l[a] < 0 || d.rad_l[a] > WPCCC_LMAX)
            return fail(WPCCC_EINVAL, n + ": rad_l out of range 0..WPCCC_LMAX");
    std::vector<int> seen((size_t)d.n_rad * (2 * WPCCC_LMAX + 1), 0);
    for (int i = 0; i < d.n_states; ++i) {
        int a = d.st_rad[i];
        if (a < 0 || a >= d.n_rad) return fail(WPCCC_EINVAL, n + ": st_rad out of range");
        int l = d.rad_l[a], m = d.st_m[i];
        if (m < -l || m > l) return fail(WPCCC_EINVAL, n + ": |st_m| > l");
        if (seen[(size_t)a * (2 * WPCCC_LMAX + 1) + m + WPCCC_LMAX]++)
            return fail(WPCCC_EINVAL, n + ": a (radial, m) pair appears twice");
    }
    if (all_m)
        for (int a = 0; a < d.n_rad; ++a)
            for (int m = -d.rad_l[a]; m <= d.rad_l[a]; ++m)
                if (!seen[(size_t)a * (2 * WPCCC_LMAX + 1) + m + WPCCC_LMAX])
                    return fail(WPCCC_EINVAL, n + ": two-centre mode needs every m of every radial function");
    return WPCCC_OK;
}

static wpccc_status build_centre(const wpccc_centre_desc& d, int Nr, const double* r_dev,
                                 const double* w_dev, CentreDev& c) {
    wpccc_status st;
    c.Z = d.Z;
    c.n_rad = d.n_rad;
    c.n_states = d.n_states;
    c.h_rad_l.assign(d.rad_l, d.rad_l + d.n_rad);
    c.h_st_rad.assign(d.st_rad, d.st_rad + d.n_states);
    c.h_st_m.assign(d.st_m, d.st_m + d.n_states);
    c.lmax = 0;
    for (int l : c.h_rad_l) c.lmax = l > c.lmax ? l : c.lmax;
    c.nlam = 2 * c.lmax + 1;
    std::vector<int> st_l(d.n_states), st_lm(d.n_states);
    for (int i = 0; i < d.n_states; ++i) {
        st_l[i] = d.rad_l[d.st_rad[i]];
        st_lm[i] = st_l[i] * st_l[i] + st_l[i] + d.st_m[i];
    }
    c.LM = (c.lmax + 1) * (c.lmax + 1);
    std::vector<int> st_index((size_t)d.n_rad * (2 * WPCCC_LMAX + 1), -1);
    for (int i = 0; i < d.n_states; ++i)
        st_index[(size_t)d.st_rad[i] * (2 * WPCCC_LMAX + 1) + d.st_m[i] + WPCCC_LMAX] = i;
    if ((st = upload(&c.f, d.f, (size_t)d.n_rad * Nr, "upload f")) != WPCCC_OK) return st;
    if ((st = upload(&c.rad_l, d.rad_l, d.n_rad, "upload rad_l")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_rad, d.st_rad, d.n_states, "upload st_rad")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_l, st_l.data(), d.n_states, "upload st_l")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_lm, st_lm.data(), d.n_states, "upload st_lm")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_m, d.st_m, d.n_states, "upload st_m")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_eps, d.st_eps, d.n_states, "upload st_eps")) != WPCCC_OK) return st;
    if ((st = upload(&c.st_index, st_index.data(), st_index.size(), "upload st_index")) != WPCCC_OK) return st;

    // Eq. 7 table entries: radial pairs a <= b and multipoles allowed by the triangle and parity rules
    std::vector<int> ea, eb, el, off((size_t)c.n_rad * c.n_rad * c.nlam, -1);
    for (int a = 0; a < c.n_rad; ++a)
        for (int b = a; b < c.n_rad; ++b) {
            int la = c.h_rad_l[a], lb = c.h_rad_l[b];
            for (int lam = abs(la - lb); lam <= la + lb; lam += 2) {
                int e = (int)ea.size();
                ea.push_back(a);
                eb.push_back(b);
                el.push_back(lam);
                off[((size_t)a * c.n_rad + b) * c.nlam + lam] = e;
                off[((size_t)b * c.n_rad + a) * c.nlam + lam] = e;
            }
        }
    c.n_fent = (int)ea.size();
    if ((st = upload(&c.fent_a, ea.data(), ea.size(), "upload fent")) != WPCCC_OK) return st;
    if ((st = upload(&c.fent_b, eb.data(), eb.size(), "upload fent")) != WPCCC_OK) return st;
    if ((st = upload(&c.fent_lam, el.data(), el.size(), "upload fent")) != WPCCC_OK) return st;
    if ((st = upload(&c.Foff, off.data(), off.size(), "upload Foff")) != WPCCC_OK) return st;
    if ((st = upload<double>(&c.F, nullptr, (size_t)c.n_fent * Nr, "alloc F")) != WPCCC_OK) return st;
    k_ftable<<<c.n_fent, 256>>>(Nr, r_dev, w_dev, c.f, c.fent_a, c.fent_b, c.fent_lam, c.F);
    WPCCC_CHECK_LAUNCH("k_ftable");
    size_t nang = (size_t)c.LM * c.LM;
    if ((st = upload<double>(&c.ang, nullptr, nang * c.nlam, "alloc ang")) != WPCCC_OK) return st;
    k_direct_angular<<<(unsigned)((nang + 255) / 256), 256>>>(c.LM, c.nlam, c.ang);
    WPCCC_CHECK_LAUNCH("k_direct_angular");
    return WPCCC_OK;
}

static void free_basis(wpccc_basis_s* B) {
    if (!B) return;
    cudaSetDevice(B->device);
    B->prof.release();
    if (B->rk_stream) {
        cudaStreamSynchronize(B->rk_stream);
        cudaStreamDestroy(B->rk_stream);
    }
    cudaEvent_t evs[] = {B->ev_asm[0], B->ev_asm[1], B->ev_rk[0], B->ev_rk[1], B->ev_fork, B->ev_join};
    for (cudaEvent_t e : evs)
        if (e) cudaEventDestroy(e);
    free_centre(B->T);
    free_centre(B->P);
    void* tptrs[] = {B->tanT.df, B->tanT.dF, B->tanP.df, B->tanP.dF, B->deps, B->tc_row, B->qg_off, B->qg_rows,
                     B->tc_err, B->tc_halfq, B->su_tiles, B->fT2, B->fP2, B->rot_plan};
    for (void* p : tptrs)
        if (p) cudaFree(p);
    void* ptrs[] = {B->r, B->w, B->inv_den, B->s, B->ws, B->tau, B->wtau, B->half_state, B->half_of, B->qtile_q,
                    B->qtile_cols, B->ws_ptr};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete B;
}

}  // namespace wpccc

using namespace wpccc;

extern "C" const char* wpccc_last_error(void) { return g_last_error.c_str(); }

extern "C" wpccc_status wpccc_basis_create(const wpccc_basis_desc* d, int device, wpccc_basis* out) {
    if (!d || !out) return fail(WPCCC_EINVAL, "wpccc_basis_create: null argument");
    *out = nullptr;
    if (d->n_centres != 1 && d->n_centres != 2) return fail(WPCCC_EINVAL, "n_centres must be 1 or 2");
    if (d->Nr < 5 || !d->r || !d->w) return fail(WPCCC_EINVAL, "Nr < 5 or null r/w");
    if (!(d->r[0] > 0.0)) return fail(WPCCC_EINVAL, "r[0] must be > 0");
    for (int i = 1; i < d->Nr; ++i)
        if (!(d->r[i] > d->r[i - 1])) return fail(WPCCC_EINVAL, "r must be strictly increasing");
    if (!std::isfinite(d->r[d->Nr - 1]) || !all_finite(d->w, (size_t)d->Nr))
        return fail(WPCCC_EINVAL, "non-finite r or w");
    const bool two = d->n_centres == 2;
    wpccc_status st = check_centre(d->T, d->Nr, two, "target");
    if (st != WPCCC_OK) return st;
    if (two) {
        if ((st = check_centre(d->P, d->Nr, true, "projectile")) != WPCCC_OK) return st;
        if (d->Geta < 1 || d->Gtau < 1 || !d->s || !d->ws || !d->tau || !d->wtau)
            return fail(WPCCC_EINVAL, "two-centre mode needs the (eta, tau) quadrature");
        if (!(d->gamma > 0.0) || !std::isfinite(d->gamma)) return fail(WPCCC_EINVAL, "gamma must be finite and > 0");
        if (!all_finite(d->s, (size_t)d->Geta) || !all_finite(d->ws, (size_t)d->Geta) ||
            !all_finite(d->tau, (size_t)d->Gtau) || !all_finite(d->wtau, (size_t)d->Gtau) ||
            !std::isfinite(d->mp_c) || !std::isfinite(d->mp_a) || !std::isfinite(d->mp_b))
            return fail(WPCCC_EINVAL, "non-finite quadrature or model-potential parameter");
    }
    int N = d->T.n_states + (two ? d->P.n_states : 0);
    if (N > WPCCC_NMAX) return fail(WPCCC_EINVAL, "N exceeds WPCCC_NMAX");
    int ndev = 0;
    WPCCC_CUDA(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) return fail(WPCCC_EINVAL, "device out of range");
    WPCCC_CUDA(cudaSetDevice(device));

    wpccc_basis_s* B = new wpccc_basis_s();
    B->device = device;
    B->n_centres = d->n_centres;
    B->Nr = d->Nr;
    B->N_T = d->T.n_states;
    B->N_P = two ? d->P.n_states : 0;
    B->N = N;
    auto bail = [&](wpccc_status s) {
        std::string keep = g_last_error;
        free_basis(B);
        g_last_error = keep;
        return s;
    };
    if ((st = upload(&B->r, d->r, d->Nr, "upload r")) != WPCCC_OK) return bail(st);
    if ((st = upload(&B->w, d->w, d->Nr, "upload w")) != WPCCC_OK) return bail(st);
    if ((st = upload<double>(&B->inv_den, nullptr, (size_t)(d->Nr - 4) * 5, "alloc inv_den")) != WPCCC_OK)
        return bail(st);
    k_lagrange_den<<<(d->Nr - 4 + 127) / 128, 128>>>(d->Nr, B->r, B->inv_den);
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return bail(cuda_fail(e, "k_lagrange_den"));
    }
    if ((st = build_centre(d->T, d->Nr, B->r, B->w, B->T)) != WPCCC_OK) return bail(st);
    if (two) {
        if ((st = build_centre(d->P, d->Nr, B->r, B->w, B->P)) != WPCCC_OK) return bail(st);
        B->Geta = d->Geta;
        B->Gtau = d->Gtau;
        B->G = d->Geta * d->Gtau;
        B->gamma = d->gamma;
        if ((st = upload(&B->s, d->s, d->Geta, "upload s")) != WPCCC_OK) return bail(st);
        if ((st = upload(&B->ws, d->ws, d->Geta, "upload ws")) != WPCCC_OK) return bail(st);
        if ((st = upload(&B->tau, d->tau, d->Gtau, "upload tau")) != WPCCC_OK) return bail(st);
        if ((st = upload(&B->wtau, d->wtau, d->Gtau, "upload wtau")) != WPCCC_OK) return bail(st);
        if (!std::isfinite(d->mp_c) || !std::isfinite(d->mp_a) || !std::isfinite(d->mp_b))
            return bail(fail(WPCCC_EINVAL, "model-potential parameters must be finite"));
        B->mp_c = d->mp_c;
        B->mp_a = d->mp_a;
        B->mp_b = d->mp_b;
        B->dmax = B->T.lmax + B->P.lmax;
        B->nlq_T = (B->T.lmax + 1) * (B->T.lmax + 2) / 2;
        B->nlq_P = (B->P.lmax + 1) * (B->P.lmax + 2) / 2;
        std::vector<int> half_state, half_of((size_t)B->P.n_rad * (WPCCC_LMAX + 1), -1);
        for (int j = 0; j < B->N_P; ++j) {
            int m = d->P.st_m[j];
            if (m < 0) continue;
            half_of[(size_t)d->P.st_rad[j] * (WPCCC_LMAX + 1) + m] = (int)half_state.size();
            half_state.push_back(j);
        }
        B->n_half = (int)half_state.size();
        // column tiles of one q for the FP32 contraction
        std::vector<int> tq, tc;
        for (int q = 0; q <= B->P.lmax; ++q) {
            std::vector<int> cols;
            for (int h = 0; h < B->n_half; ++h)
                if (d->P.st_m[half_state[h]] == q) cols.push_back(h);
            for (size_t k = 0; k < cols.size(); k += 16) {
                tq.push_back(q);
                for (size_t c = 0; c < 16; ++c) tc.push_back(k + c < cols.size() ? cols[k + c] : -1);
            }
        }
        B->n_qtiles = (int)tq.size();
        if ((st = upload(&B->qtile_q, tq.data(), tq.size(), "upload qtile_q")) != WPCCC_OK) return bail(st);
        if ((st = upload(&B->qtile_cols, tc.data(), tc.size(), "upload qtile_cols")) != WPCCC_OK) return bail(st);
        if ((st = upload(&B->half_state, half_state.data(), half_state.size(), "upload half")) != WPCCC_OK)
            return bail(st);
        if ((st = upload(&B->half_of, half_of.data(), half_of.size(), "upload half_of")) != WPCCC_OK)
            return bail(st);
        if ((st = rotation_plan(B)) != WPCCC_OK) return bail(st);
    } else {
        B->P.Z = d->P.Z;
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return bail(cuda_fail(e, "basis set-up kernels"));
    *out = B;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_destroy(wpccc_basis B) {
    if (!B) return WPCCC_OK;
    cudaSetDevice(B->device);
    cudaDeviceSynchronize();
    free_basis(B);
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_info(wpccc_basis B, int* N_T, int* N_P) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_info: null basis");
    if (N_T) *N_T = B->N_T;
    if (N_P) *N_P = B->N_P;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_profile_enable(wpccc_basis B, int on) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_profile_enable: null basis");
    WPCCC_CUDA(cudaSetDevice(B->device));
    B->prof.flush();
    for (int c = 0; c < WPCCC_PROF_N; ++c) {
        B->prof.ms[c] = 0.0;
        B->prof.launches[c] = 0;
    }
    B->prof.on = on != 0;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_profile_read(wpccc_basis B, double* ms, long long* launches) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_profile_read: null basis");
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaError_t e = B->prof.flush();
    if (e != cudaSuccess) return cuda_fail(e, "wpccc_profile_read");
    for (int c = 0; c < WPCCC_PROF_N; ++c) {
        if (ms) ms[c] = B->prof.ms[c];
        if (launches) launches[c] = B->prof.launches[c];
    }
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_solve_mode(wpccc_basis B, int mode) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_solve_mode: null basis");
    if (mode != WPCCC_SOLVE_STAGE && mode != WPCCC_SOLVE_MATRIX && mode != WPCCC_SOLVE_SCHUR)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_solve_mode: unknown mode");
    B->solve_mode = mode;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_rk4_layout(wpccc_basis B, int layout) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_rk4_layout: null basis");
    if (layout != WPCCC_RK4_AUTO && layout != WPCCC_RK4_SHARED && layout != WPCCC_RK4_GLOBAL)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_rk4_layout: unknown layout");
    B->rk4_layout = layout;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_refine_iters(wpccc_basis B, int iters) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_refine_iters: null basis");
    if (iters < 1 || iters > WPCCC_MAX_REFINE)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_refine_iters: iterations must be 1 to " + std::to_string(WPCCC_MAX_REFINE));
    B->refine_iters = iters;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_schur_update(wpccc_basis B, int mode) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_schur_update: null basis");
    if (mode != WPCCC_SCHUR_UPDATE_AUTO && mode != WPCCC_SCHUR_UPDATE_TENSOR && mode != WPCCC_SCHUR_UPDATE_CUDA_CORES)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_schur_update: unknown mode");
    B->schur_update = mode;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_refine_tolerance(wpccc_basis B, double tol) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_refine_tolerance: null basis");
    if (!std::isfinite(tol)) return fail(WPCCC_EINVAL, "wpccc_basis_set_refine_tolerance: non-finite tolerance");
    B->refine_tol = tol;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_wait_limit(wpccc_basis B, long polls) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_wait_limit: null basis");
    if (polls < 1) return fail(WPCCC_EINVAL, "wpccc_basis_set_wait_limit: polls must be >= 1");
    B->wait_polls = polls;
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_basis_set_workspace_limit(wpccc_basis B, size_t bytes) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_workspace_limit: null basis");
    if (bytes < ((size_t)64 << 20)) return fail(WPCCC_EINVAL, "workspace limit below 64 MiB");
    B->ws_limit = bytes;
    return WPCCC_OK;
}

// ---------------------------------------------------------------------------
// differentiation form: derivative tables of the inputs
// ---------------------------------------------------------------------------
namespace wpccc {

// Keeps the derivative tables of one centre for the parameters whose tangent is not identically
// zero, and builds the derivative of its Eq. 7 table from them.
static wpccc_status centre_tangents(wpccc_basis_s* B, CentreDev& c, CentreTan& t, int n_par, const double* df) {
    const size_t per = (size_t)c.n_rad * B->Nr;
    t = CentreTan();
    for (int p = 0; p < WPCCC_MAX_PARAMS; ++p) t.slot[p] = -1;
    std::vector<int> keep;
    for (int p = 0; p < n_par; ++p) {
        const double* d = df + (size_t)p * per;
        bool nz = false;
        for (size_t k = 0; k < per && !nz; ++k) {
            if (!std::isfinite(d[k])) return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: non-finite derivative");
            nz = d[k] != 0.0;
        }
        if (nz) {
            t.slot[p] = (int)keep.size();
            t.par[keep.size()] = p;
            keep.push_back(p);
        }
    }
    t.n_tan = (int)keep.size();
    if (t.n_tan == 0) return WPCCC_OK;
    std::vector<double> packed(per * t.n_tan);
    for (int k = 0; k < t.n_tan; ++k)
        std::memcpy(packed.data() + per * k, df + per * keep[k], per * sizeof(double));
    wpccc_status st;
    if ((st = upload(&t.df, packed.data(), packed.size(), "upload df")) != WPCCC_OK) return st;
    if ((st = upload<double>(&t.dF, nullptr, (size_t)t.n_tan * c.n_fent * B->Nr, "alloc dF")) != WPCCC_OK) return st;
    for (int k = 0; k < t.n_tan; ++k) {
        k_ftable<<<c.n_fent, 256>>>(B->Nr, B->r, B->w, c.f, c.fent_a, c.fent_b, c.fent_lam,
                                    t.dF + (size_t)k * c.n_fent * B->Nr, t.df + per * k);
        WPCCC_CHECK_LAUNCH("k_ftable (derivative)");
    }
    return WPCCC_OK;
}

}  // namespace wpccc

extern "C" wpccc_status wpccc_basis_set_tangents(wpccc_basis B, int n_par, const double* dfT, const double* depsT,
                                                 const double* dfP, const double* depsP, const double* dexplicit) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: null basis");
    if (B->n_centres != 2) return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: two-centre bases only");
    if (n_par < 1 || n_par > WPCCC_MAX_PARAMS)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: n_par must be 1..WPCCC_MAX_PARAMS");
    if (!dfT || !depsT || !dfP || !depsP || !dexplicit)
        return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: null pointer");
    for (int k = 0; k < 4 * n_par; ++k)
        if (!std::isfinite(dexplicit[k])) return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: non-finite dexplicit");
    if (!all_finite(dfT, (size_t)n_par * B->T.n_rad * B->Nr) || !all_finite(dfP, (size_t)n_par * B->P.n_rad * B->Nr))
        return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: non-finite radial derivative table");
    WPCCC_CUDA(cudaSetDevice(B->device));
    WPCCC_CUDA(cudaDeviceSynchronize());
    void* old[] = {B->tanT.df, B->tanT.dF, B->tanP.df, B->tanP.dF, B->deps};
    for (void* p : old)
        if (p) cudaFree(p);
    B->tanT = CentreTan();
    B->tanP = CentreTan();
    B->deps = nullptr;
    B->n_par = 0;
    // energy derivatives per state, target states first
    std::vector<double> de((size_t)n_par * B->N);
    for (int p = 0; p < n_par; ++p) {
        for (int i = 0; i < B->N_T; ++i) de[(size_t)p * B->N + i] = depsT[(size_t)p * B->T.n_rad + B->T.h_st_rad[i]];
        for (int j = 0; j < B->N_P; ++j)
            de[(size_t)p * B->N + B->N_T + j] = depsP[(size_t)p * B->P.n_rad + B->P.h_st_rad[j]];
    }
    for (double x : de)
        if (!std::isfinite(x)) return fail(WPCCC_EINVAL, "wpccc_basis_set_tangents: non-finite energy derivative");
    wpccc_status st;
    if ((st = upload(&B->deps, de.data(), de.size(), "upload deps")) != WPCCC_OK) return st;
    if ((st = centre_tangents(B, B->T, B->tanT, n_par, dfT)) != WPCCC_OK) return st;
    if ((st = centre_tangents(B, B->P, B->tanP, n_par, dfP)) != WPCCC_OK) return st;
    for (int p = 0; p < n_par; ++p)
        for (int k = 0; k < 4; ++k) B->dexp[p][k] = dexplicit[4 * p + k];
    WPCCC_CUDA(cudaDeviceSynchronize());
    B->n_par = n_par;
    return WPCCC_OK;
}
