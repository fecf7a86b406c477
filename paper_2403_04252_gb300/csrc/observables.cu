// Observables at the end of the paths (Sec. II, after Algorithm 1: the amplitudes at z_max give the
// transition probabilities, from which capture and excitation cross sections follow):
//   wpccc_observables     P[p][o] = sum_i g[o][i] |c_p,i|^2 (capture: g = 1 on the projectile's bound
//                         states; excitation of a level: g = 1 on its states)
//   wpccc_cross_sections  sigma_o = 2 pi int_0^inf b P_o(b) db by the trapezoid rule on the impact
//                         parameters plus b = 0 (where b P(b) = 0)
//   wpccc_overlap_norms   c^+ S(z) c and c^+ c of every path at a given position: in the non-orthogonal
//                         two-centre basis the probability carried by the amplitudes is c^+ S c
//   wpccc_basis_states    the quantum numbers and energies of the basis' states, in state order
#include <algorithm>
#include <cmath>
#include <vector>

#include "wpccc_internal.cuh"

namespace wpccc {

static __device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 acc) {
    return make_double2(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
}

// One block per (path, observable): a block-wide sum over the states.
__global__ void __launch_bounds__(256) k_observables(int N, int n_obs, const double2* __restrict__ c,
                                                     const double* __restrict__ g, double* __restrict__ P) {
    const int p = blockIdx.x, o = blockIdx.y;
    const double2* cp = c + (size_t)p * N;
    const double* go = g + (size_t)o * N;
    double s = 0.0;
    for (int i = threadIdx.x; i < N; i += blockDim.x) {
        const double2 a = cp[i];
        s += go[i] * (a.x * a.x + a.y * a.y);
    }
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) P[(size_t)p * n_obs + o] = red[0];
}

constexpr int XS_MAX_B = 2048;   // impact parameters per cross-section call (the weights travel as kernel arguments)

struct XsArgs {
    int n_b, n_obs;
    double wb[XS_MAX_B];   // 2 pi b_j w_j
};

// One block per observable: sigma_o = sum_j wb_j P[j][o] (sum in a fixed order: per-thread strides, then
// a tree over the block).
__global__ void __launch_bounds__(256) k_cross_sections(const __grid_constant__ XsArgs A, const double* __restrict__ P,
                                                        double* __restrict__ sigma) {
    const int o = blockIdx.x;
    double s = 0.0;
    for (int j = threadIdx.x; j < A.n_b; j += blockDim.x) s += A.wb[j] * P[(size_t)j * A.n_obs + o];
    __shared__ double red[256];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) sigma[o] = red[0];
}

// One block per path: c^+ S c (S column-major, complex) and c^+ c.
__global__ void __launch_bounds__(256) k_overlap_norms(int N, const double2* __restrict__ c,
                                                       const double2* __restrict__ S, double* __restrict__ out) {
    const int p = blockIdx.x;
    const double2* cp = c + (size_t)p * N;
    const double2* Sp = S + (size_t)p * N * N;
    double sre = 0.0, n2 = 0.0;
    // c^+ S c = sum_j conj(c_j) (S c)_j with (S c)_j = sum_k S[j + k N] c_k
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        double2 y = make_double2(0.0, 0.0);
        for (int k = 0; k < N; ++k) y = cfma(Sp[j + (size_t)k * N], cp[k], y);
        const double2 a = cp[j];
        sre += a.x * y.x + a.y * y.y;   // Re(conj(a) y); the imaginary parts cancel for Hermitian S
        n2 += a.x * a.x + a.y * a.y;
    }
    __shared__ double red[2][256];
    red[0][threadIdx.x] = sre;
    red[1][threadIdx.x] = n2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            red[0][threadIdx.x] += red[0][threadIdx.x + w];
            red[1][threadIdx.x] += red[1][threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * p] = red[0][0];
        out[2 * p + 1] = red[1][0];
    }
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_observables(int n_paths, int N, int n_obs, const double* g, const void* c, double* P,
                                          void* stream) {
    if (n_paths < 0 || N < 1 || n_obs < 1 || n_obs > 65535 || n_paths > 0x7fffffff / 2)
        return fail(WPCCC_EINVAL, "wpccc_observables: bad sizes");
    if (n_paths == 0) return WPCCC_OK;
    if (!g || !c || !P) return fail(WPCCC_EINVAL, "wpccc_observables: null pointer");
    k_observables<<<dim3(n_paths, n_obs), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        N, n_obs, static_cast<const double2*>(c), g, P);
    WPCCC_CHECK_LAUNCH("k_observables");
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_cross_sections(int n_b, const double* b, int n_obs, const double* P, double* sigma,
                                             void* stream) {
    if (n_b < 1 || n_b > XS_MAX_B || n_obs < 1 || n_obs > 65535)
        return fail(WPCCC_EINVAL, "wpccc_cross_sections: n_b must be 1.." + std::to_string(XS_MAX_B) +
                                      " and n_obs >= 1");
    if (!b || !P || !sigma) return fail(WPCCC_EINVAL, "wpccc_cross_sections: null pointer");
    XsArgs a;
    a.n_b = n_b;
    a.n_obs = n_obs;
    // trapezoid weights on the nodes 0, b_1, ..., b_n: w_j = (b_{j+1} - b_{j-1}) / 2, the last (b_n - b_{n-1}) / 2
    double prev = 0.0;
    for (int j = 0; j < n_b; ++j) {
        if (!std::isfinite(b[j]) || !(b[j] > prev))
            return fail(WPCCC_EINVAL, "wpccc_cross_sections: impact parameters must be finite, > 0 and increasing");
        const double next = j + 1 < n_b ? b[j + 1] : b[j];
        a.wb[j] = 2.0 * M_PI * b[j] * (0.5 * (next - prev));
        prev = b[j];
    }
    k_cross_sections<<<n_obs, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, P, sigma);
    WPCCC_CHECK_LAUNCH("k_cross_sections");
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_overlap_norms(wpccc_basis B, int n_paths, const double* b, const double* v,
                                            const double* z, const void* c, double* out, void* stream) {
    if (!B || !b || !v || !z || !c || !out) return fail(WPCCC_EINVAL, "wpccc_overlap_norms: null argument");
    if (n_paths < 1 || n_paths > MAX_EVALS_PER_LAUNCH) return fail(WPCCC_EINVAL, "wpccc_overlap_norms: bad n_paths");
    for (int p = 0; p < n_paths; ++p)
        if (!(b[p] > 0.0) || !(v[p] > 0.0) || !std::isfinite(z[p]))
            return fail(WPCCC_EINVAL, "wpccc_overlap_norms: b and v must be > 0, z finite");
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t N = (size_t)B->N;
    const ElemScratch L = elem_scratch_layout(B);
    // positions in groups that the workspace limit holds (scratch of the element kernels), S and H per group
    const int per = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_paths,
                                                               (B->ws_limit - 256) / (L.bytes_per_eval + sizeof(EvalDesc))));
    const size_t need = (size_t)per * L.bytes_per_eval + 256 + (size_t)per * sizeof(EvalDesc);
    wpccc_status s = ensure_workspace(B, need);
    if (s != WPCCC_OK) return s;
    double2* SH = nullptr;
    if (cudaMalloc(&SH, 2 * (size_t)per * N * N * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        return fail(WPCCC_ENOMEM, "wpccc_overlap_norms: cudaMalloc(S, H)");
    }
    char* wsb = static_cast<char*>(B->ws_ptr);
    EvalDesc* dev_ev = reinterpret_cast<EvalDesc*>(wsb);
    void* scratch = wsb + ((per * sizeof(EvalDesc) + 255) / 256) * 256;
    std::vector<EvalDesc> ev(per);
    for (int p0 = 0; p0 < n_paths && s == WPCCC_OK; p0 += per) {
        const int n = std::min(per, n_paths - p0);
        for (int k = 0; k < n; ++k) ev[k] = EvalDesc{b[p0 + k], v[p0 + k], z[p0 + k], p0 + k, 0};
        cudaError_t e = cudaMemcpyAsync(dev_ev, ev.data(), n * sizeof(EvalDesc), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) {
            s = cuda_fail(e, "cudaMemcpyAsync(positions)");
            break;
        }
        s = launch_elements(B, dev_ev, n, SH, SH + (size_t)per * N * N, scratch, st, 0);
        if (s != WPCCC_OK) break;
        k_overlap_norms<<<n, 256, 0, st>>>((int)N, static_cast<const double2*>(c) + (size_t)p0 * N, SH, out + 2 * p0);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // the host list and S, H are reused
        if (e != cudaSuccess) s = cuda_fail(e, "k_overlap_norms");
    }
    cudaFree(SH);
    return s;
}

extern "C" wpccc_status wpccc_basis_states(wpccc_basis B, int* qn, double* eps) {
    if (!B) return fail(WPCCC_EINVAL, "wpccc_basis_states: null basis");
    const int two = B->n_centres == 2;
    if (qn) {
        int k = 0;
        for (int cen = 0; cen < 1 + two; ++cen) {
            const CentreDev& C = cen == 0 ? B->T : B->P;
            for (int i = 0; i < C.n_states; ++i, ++k) {
                const int a = C.h_st_rad[i];
                qn[4 * k] = cen;
                qn[4 * k + 1] = a;
                qn[4 * k + 2] = C.h_rad_l[a];
                qn[4 * k + 3] = C.h_st_m[i];
            }
        }
    }
    if (eps) {
        WPCCC_CUDA(cudaSetDevice(B->device));
        WPCCC_CUDA(cudaMemcpy(eps, B->T.st_eps, B->N_T * sizeof(double), cudaMemcpyDeviceToHost));
        if (two) WPCCC_CUDA(cudaMemcpy(eps + B->N_T, B->P.st_eps, B->N_P * sizeof(double), cudaMemcpyDeviceToHost));
    }
    return WPCCC_OK;
}
