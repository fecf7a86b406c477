// Propagation of the amplitudes (Algorithm 1) and the probabilities.
//
// M(z) = -(i/v) S(z)^{-1} H(z) depends on the path and z only, never on the
// amplitudes, so the positions an RK4 step needs (z_mid and z_new; z of the
// first node once per path) are evaluated ahead of the sweep: for a chunk of
// steps of every path, all matrix elements are assembled and all systems
// solved in batched launches, then one fused RK4 kernel per chunk advances
// every path through the chunk's steps.  The matrix at the last node of a
// chunk is carried over to the next.
#include <algorithm>
#include <cmath>
#include <vector>

#include "wpccc_internal.cuh"

namespace wpccc {

wpccc_status ensure_workspace(wpccc_basis_s* B, size_t bytes);

struct PathChunk {
    int path;
    int nsteps;
    int start_local;   // eval (within the chunk) holding X at the first node, or -1: use the carry
    int first_local;   // eval of step 0's midpoint; step s uses first_local + 2s (mid), + 2s + 1 (new)
    int z0;            // index of the chunk's first node in the concatenated z array
    int pad;
    double v;
};

enum : int { FLAG_SINGULAR = 1, FLAG_NONFINITE = 2 };

constexpr int RK_THREADS = 512;

// k = -(i/v) X y   (X column-major N x N)
__device__ inline void apply_M(const double2* __restrict__ X, int N, double v, const double2* y, double2* k) {
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        double re = 0.0, im = 0.0;
        const double2* row = X + i;
        for (int j = 0; j < N; ++j) {
            const double2 a = row[(size_t)j * N];
            const double2 b = y[j];
            re = fma(a.x, b.x, re);
            re = fma(-a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(a.y, b.x, im);
        }
        // -(i/v) (re + i im) = (im - i re)/v
        k[i] = make_double2(im / v, -re / v);
    }
}

__global__ void __launch_bounds__(RK_THREADS) k_rk4(int N, const double2* __restrict__ Hc,
                                                    double2* __restrict__ carry, double2* __restrict__ c_all,
                                                    const double* __restrict__ z, const PathChunk* __restrict__ pcs,
                                                    const int* __restrict__ info, int* __restrict__ flags) {
    extern __shared__ double2 rk_smem[];
    double2* c = rk_smem;
    double2* y = c + N;
    double2* kv = y + N;
    double2* acc = kv + N;
    const PathChunk pc = pcs[blockIdx.x];
    const size_t mat = (size_t)N * N;
    double2* cg = c_all + (size_t)pc.path * N;
    double2* carry_p = carry + (size_t)pc.path * mat;
    const double v = pc.v;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) c[i] = cg[i];
    if (info && threadIdx.x == 0) {
        int bad = 0;
        if (pc.start_local >= 0 && info[pc.start_local] != 0) bad = 1;
        for (int s = 0; s < 2 * pc.nsteps; ++s)
            if (info[pc.first_local + s] != 0) bad = 1;
        if (bad) atomicOr(flags, FLAG_SINGULAR);
    }
    __syncthreads();
    const double2* Xz = pc.start_local >= 0 ? Hc + (size_t)pc.start_local * mat : carry_p;
    for (int s = 0; s < pc.nsteps; ++s) {
        const double2* Xmid = Hc + (size_t)(pc.first_local + 2 * s) * mat;
        const double2* Xnew = Xmid + mat;
        const double h = z[pc.z0 + s + 1] - z[pc.z0 + s];
        const double h2 = 0.5 * h, h6 = h / 6.0;
        // K1 = M_z c
        apply_M(Xz, N, v, c, kv);
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = kv[i];
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K2 = M_mid (c + h/2 K1)
        apply_M(Xmid, N, v, y, kv);
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K3 = M_mid (c + h/2 K2)
        apply_M(Xmid, N, v, y, kv);
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h, kv[i].x, c[i].x), fma(h, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K4 = M_new (c + h K3)
        apply_M(Xnew, N, v, y, kv);
        __syncthreads();
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 a = make_double2(acc[i].x + kv[i].x, acc[i].y + kv[i].y);
            c[i] = make_double2(fma(h6, a.x, c[i].x), fma(h6, a.y, c[i].y));
        }
        __syncthreads();
        Xz = Xnew;
    }
    bool finite = true;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        cg[i] = c[i];
        if (!isfinite(c[i].x) || !isfinite(c[i].y)) finite = false;
    }
    if (!finite) atomicOr(flags, FLAG_NONFINITE);
    // carry the matrix at the chunk's last node into the next chunk
    if (Xz != carry_p)
        for (size_t t = threadIdx.x; t < mat; t += RK_THREADS) carry_p[t] = Xz[t];
}

__global__ void k_probabilities(long long n, const double2* __restrict__ c, double* __restrict__ P) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const double2 a = c[i];
        P[i] = a.x * a.x + a.y * a.y;
    }
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_probabilities(int n_paths, int N, const void* c, double* P, void* stream) {
    if (n_paths < 0 || N < 1) return fail(WPCCC_EINVAL, "wpccc_probabilities: bad sizes");
    if (n_paths == 0) return WPCCC_OK;
    if (!c || !P) return fail(WPCCC_EINVAL, "wpccc_probabilities: null pointer");
    long long n = (long long)n_paths * N;
    k_probabilities<<<(unsigned)((n + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        n, static_cast<const double2*>(c), P);
    WPCCC_CHECK_LAUNCH("k_probabilities");
    return WPCCC_OK;
}

extern "C" wpccc_status wpccc_propagate(wpccc_basis B, const wpccc_paths* paths, int precision_mode,
                                        int batch_mode, void* c, void* stream) {
    if (!B || !paths || !c) return fail(WPCCC_EINVAL, "wpccc_propagate: null argument");
    if (precision_mode != 0) return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: only precision_mode 0 (FP64)");
    if (batch_mode != 0) return fail(WPCCC_EUNSUPPORTED, "wpccc_propagate: only batch_mode 0");
    const int np = paths->n_paths;
    if (np < 1 || !paths->b || !paths->v || !paths->n_z || !paths->z)
        return fail(WPCCC_EINVAL, "wpccc_propagate: empty or null path description");
    std::vector<int> zoff(np + 1, 0);
    for (int p = 0; p < np; ++p) {
        if (!(paths->b[p] > 0.0) || !(paths->v[p] > 0.0))
            return fail(WPCCC_EINVAL, "wpccc_propagate: b and v must be > 0");
        if (paths->n_z[p] < 1) return fail(WPCCC_EINVAL, "wpccc_propagate: n_z < 1");
        zoff[p + 1] = zoff[p] + paths->n_z[p];
        for (int k = zoff[p] + 1; k < zoff[p + 1]; ++k)
            if (!(paths->z[k] > paths->z[k - 1]))
                return fail(WPCCC_EINVAL, "wpccc_propagate: z nodes must increase strictly");
    }
    const int N = B->N;
    if (N > WPCCC_NMAX) return fail(WPCCC_EINVAL, "wpccc_propagate: N too large");
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool two = B->n_centres == 2;
    const size_t mat = (size_t)N * N;
    const ElemScratch L = elem_scratch_layout(B);
    // device bytes per evaluation: S (two-centre only), H, pivots and info, element scratch
    const size_t per_eval = (two ? 2 : 1) * mat * sizeof(double2) + L.bytes_per_eval +
                            (two ? (size_t)N * sizeof(int) + sizeof(int) : 0) + sizeof(EvalDesc);

    int max_steps = 0;
    long long total_evals = 0;
    for (int p = 0; p < np; ++p) {
        int ns = paths->n_z[p] - 1;
        max_steps = std::max(max_steps, ns);
        if (ns > 0) total_evals += 2LL * ns + 1;
    }
    if (max_steps == 0) return WPCCC_OK;

    // fixed part of the workspace: carry matrices, z nodes, plan, flags
    auto align = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t fixed = align((size_t)np * mat * sizeof(double2)) + align((size_t)zoff[np] * sizeof(double)) +
                         align((size_t)total_evals * sizeof(EvalDesc)) +
                         align((size_t)np * max_steps * sizeof(PathChunk)) + 16 * 256;
    // steps per chunk: every path with steps left contributes 2 evaluations per step
    size_t budget = B->ws_limit > fixed ? B->ws_limit - fixed : 0;
    long long cap_evals = (long long)(budget / per_eval);
    int C = (int)std::min<long long>(max_steps, std::max<long long>(1, (cap_evals - np) / (2LL * np)));
    if (cap_evals < 2LL * np + np) C = 1;
    const int n_chunks = (max_steps + C - 1) / C;

    // plan: evaluations and path chunks for every chunk
    std::vector<EvalDesc> ev;
    ev.reserve(total_evals);
    std::vector<PathChunk> pcs;
    std::vector<int> ev_begin(n_chunks + 1), pc_begin(n_chunks + 1);
    for (int ch = 0; ch < n_chunks; ++ch) {
        ev_begin[ch] = (int)ev.size();
        pc_begin[ch] = (int)pcs.size();
        const int s0 = ch * C;
        for (int p = 0; p < np; ++p) {
            const int ns = paths->n_z[p] - 1;
            if (s0 >= ns) continue;
            const int n = std::min(C, ns - s0);
            const double* zp = paths->z + zoff[p];
            PathChunk pc;
            pc.path = p;
            pc.nsteps = n;
            pc.v = paths->v[p];
            pc.z0 = zoff[p] + s0;
            pc.pad = 0;
            pc.start_local = -1;
            const int base = ev_begin[ch];
            if (s0 == 0) {
                pc.start_local = (int)ev.size() - base;
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], zp[0], p, 0});
            }
            pc.first_local = (int)ev.size() - base;
            for (int s = s0; s < s0 + n; ++s) {
                const double za = zp[s], zb = zp[s + 1];
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], (za + zb) / 2.0, p, 0});
                ev.push_back(EvalDesc{paths->b[p], paths->v[p], zb, p, 0});
            }
            pcs.push_back(pc);
        }
    }
    ev_begin[n_chunks] = (int)ev.size();
    pc_begin[n_chunks] = (int)pcs.size();
    int max_chunk_evals = 0;
    for (int ch = 0; ch < n_chunks; ++ch) max_chunk_evals = std::max(max_chunk_evals, ev_begin[ch + 1] - ev_begin[ch]);

    // workspace carve-up
    const size_t sz_carry = align((size_t)np * mat * sizeof(double2));
    const size_t sz_z = align((size_t)zoff[np] * sizeof(double));
    const size_t sz_ev = align(ev.size() * sizeof(EvalDesc));
    const size_t sz_pc = align(pcs.size() * sizeof(PathChunk));
    const size_t sz_flags = 256;
    const size_t sz_S = two ? align((size_t)max_chunk_evals * mat * sizeof(double2)) : 0;
    const size_t sz_H = align((size_t)max_chunk_evals * mat * sizeof(double2));
    const size_t sz_piv = two ? align((size_t)max_chunk_evals * N * sizeof(int)) : 0;
    const size_t sz_info = two ? align((size_t)max_chunk_evals * sizeof(int)) : 0;
    const size_t sz_scr = align((size_t)max_chunk_evals * L.bytes_per_eval);
    const size_t need = sz_carry + sz_z + sz_ev + sz_pc + sz_flags + sz_S + sz_H + sz_piv + sz_info + sz_scr;
    wpccc_status s = ensure_workspace(B, need);
    if (s != WPCCC_OK) return s;
    char* w = static_cast<char*>(B->ws_ptr);
    double2* d_carry = reinterpret_cast<double2*>(w);
    w += sz_carry;
    double* d_z = reinterpret_cast<double*>(w);
    w += sz_z;
    EvalDesc* d_ev = reinterpret_cast<EvalDesc*>(w);
    w += sz_ev;
    PathChunk* d_pc = reinterpret_cast<PathChunk*>(w);
    w += sz_pc;
    int* d_flags = reinterpret_cast<int*>(w);
    w += sz_flags;
    double2* d_S = two ? reinterpret_cast<double2*>(w) : nullptr;
    w += sz_S;
    double2* d_H = reinterpret_cast<double2*>(w);
    w += sz_H;
    int* d_piv = two ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_piv;
    int* d_info = two ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_info;
    void* d_scr = w;

    WPCCC_CUDA(cudaMemcpyAsync(d_z, paths->z, (size_t)zoff[np] * sizeof(double), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(d_ev, ev.data(), ev.size() * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemcpyAsync(d_pc, pcs.data(), pcs.size() * sizeof(PathChunk), cudaMemcpyHostToDevice, st));
    WPCCC_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), st));
    const int rk_smem = (int)(4 * (size_t)N * sizeof(double2));
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));

    for (int ch = 0; ch < n_chunks; ++ch) {
        const int nev = ev_begin[ch + 1] - ev_begin[ch];
        const int npc = pc_begin[ch + 1] - pc_begin[ch];
        s = launch_elements(B, d_ev + ev_begin[ch], nev, d_S, d_H, d_scr, st);
        if (s != WPCCC_OK) return s;
        if (two) {
            cudaEvent_t e0 = B->prof.begin(PROF_SOLVE, st);
            s = launch_solve(N, nev, d_S, d_H, d_piv, d_info, st);
            if (s != WPCCC_OK) return s;
            B->prof.end(PROF_SOLVE, st, e0);
        }
        cudaEvent_t e1 = B->prof.begin(PROF_RK4, st);
        k_rk4<<<npc, RK_THREADS, rk_smem, st>>>(N, d_H, d_carry, static_cast<double2*>(c), d_z,
                                                 d_pc + pc_begin[ch], d_info, d_flags);
        WPCCC_CHECK_LAUNCH("k_rk4");
        B->prof.end(PROF_RK4, st, e1);
    }
    int flags = 0;
    WPCCC_CUDA(cudaMemcpyAsync(&flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, st));
    WPCCC_CUDA(cudaStreamSynchronize(st));
    if (flags & FLAG_SINGULAR) return fail(WPCCC_ESINGULAR, "wpccc_propagate: an overlap matrix had a zero pivot");
    if (flags & FLAG_NONFINITE) return fail(WPCCC_ENONFINITE, "wpccc_propagate: amplitudes became non-finite");
    return WPCCC_OK;
}
