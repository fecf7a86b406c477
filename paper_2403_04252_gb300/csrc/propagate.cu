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
__device__ inline void apply_X(const double2* __restrict__ X, int N, double v, const double2* y, double2* k) {
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
    __syncthreads();
}

// k = -(i/v) S^{-1} (H y) with S given by its LU factors (P S = L U, LAPACK layout) and pivots.
// t is shared scratch of N elements.
__device__ void apply_LU(const double2* __restrict__ LU, const int* __restrict__ piv,
                         const double2* __restrict__ Hm, int N, double v, const double2* y, double2* k,
                         double2* t) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < N; i += RK_THREADS) {
        double re = 0.0, im = 0.0;
        const double2* row = Hm + i;
        for (int j = 0; j < N; ++j) {
            const double2 a = row[(size_t)j * N];
            const double2 b = y[j];
            re = fma(a.x, b.x, re);
            re = fma(-a.y, b.y, re);
            im = fma(a.x, b.y, im);
            im = fma(a.y, b.x, im);
        }
        t[i] = make_double2(re, im);
    }
    __syncthreads();
    if (tid == 0)
        for (int r = 0; r < N; ++r) {
            const int p = piv[r] - 1;
            if (p != r) {
                const double2 q = t[r];
                t[r] = t[p];
                t[p] = q;
            }
        }
    __syncthreads();
    // L z = P H y, unit lower triangular, blocks of 32 rows
    for (int kb = 0; kb < N; kb += 32) {
        const int nb = min(32, N - kb);
        if (warp == 0) {
            double2 x = lane < nb ? t[kb + lane] : make_double2(0.0, 0.0);
            for (int j = 0; j < nb - 1; ++j) {
                const double xr = __shfl_sync(0xffffffffu, x.x, j);
                const double xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane > j && lane < nb) {
                    const double2 l = LU[(size_t)(kb + lane) + (size_t)(kb + j) * N];
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
            double2 a = t[i];
            for (int j = 0; j < nb; ++j) {
                const double2 l = LU[(size_t)i + (size_t)(kb + j) * N];
                const double2 b = t[kb + j];
                a.x = fma(-l.x, b.x, a.x);
                a.x = fma(l.y, b.y, a.x);
                a.y = fma(-l.x, b.y, a.y);
                a.y = fma(-l.y, b.x, a.y);
            }
            t[i] = a;
        }
        __syncthreads();
    }
    // U x = z, upper triangular, blocks of 32 rows from the bottom
    const int last = ((N - 1) / 32) * 32;
    for (int kb = last; kb >= 0; kb -= 32) {
        const int nb = min(32, N - kb);
        if (warp == 0) {
            double2 x = lane < nb ? t[kb + lane] : make_double2(0.0, 0.0);
            for (int j = nb - 1; j >= 0; --j) {
                if (lane == j) {
                    const double2 u = LU[(size_t)(kb + j) + (size_t)(kb + j) * N];
                    const double d = u.x * u.x + u.y * u.y;
                    x = cmul(x, make_double2(u.x / d, -u.y / d));
                }
                const double xr = __shfl_sync(0xffffffffu, x.x, j);
                const double xi = __shfl_sync(0xffffffffu, x.y, j);
                if (lane < j) {
                    const double2 u = LU[(size_t)(kb + lane) + (size_t)(kb + j) * N];
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
            double2 a = t[i];
            for (int j = 0; j < nb; ++j) {
                const double2 u = LU[(size_t)i + (size_t)(kb + j) * N];
                const double2 b = t[kb + j];
                a.x = fma(-u.x, b.x, a.x);
                a.x = fma(u.y, b.y, a.x);
                a.y = fma(-u.x, b.y, a.y);
                a.y = fma(-u.y, b.x, a.y);
            }
            t[i] = a;
        }
        __syncthreads();
    }
    for (int i = tid; i < N; i += RK_THREADS) k[i] = make_double2(t[i].y / v, -t[i].x / v);
    __syncthreads();
}

struct RkArgs {
    int N;
    const double2* H;       // chunk: H (one-centre, or X = S^{-1} H in matrix mode) per evaluation
    const double2* LU;      // chunk: LU factors of S per evaluation (stage mode), else null
    const int* piv;         // chunk: pivots per evaluation (stage mode)
    const int* info;        // chunk: solve status per evaluation (two-centre), else null
    double2* carryH;        // per path: the matrix (or H) at the last node of the previous chunk
    double2* carryLU;       // per path (stage mode)
    int* carryPiv;          // per path (stage mode)
    double2* c;             // [n_paths][N]
    const double* z;
    const PathChunk* pcs;
    int* flags;
};

// One block per path: the chunk's RK4 steps (Algorithm 1) with M(z) y = -(i/v) X(z) y, where
// X = S^{-1} H is either stored (matrix mode, one-centre) or applied from the LU factors (stage mode).
template <bool STAGE>
__global__ void __launch_bounds__(RK_THREADS) k_rk4(RkArgs A) {
    extern __shared__ double2 rk_smem[];
    const int N = A.N;
    double2* c = rk_smem;
    double2* y = c + N;
    double2* kv = y + N;
    double2* acc = kv + N;
    double2* t = acc + N;
    const PathChunk pc = A.pcs[blockIdx.x];
    const size_t mat = (size_t)N * N;
    double2* cg = A.c + (size_t)pc.path * N;
    const double v = pc.v;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) c[i] = cg[i];
    if (A.info && threadIdx.x == 0) {
        int bad = 0;
        if (pc.start_local >= 0 && A.info[pc.start_local] != 0) bad = 1;
        for (int s = 0; s < 2 * pc.nsteps; ++s)
            if (A.info[pc.first_local + s] != 0) bad = 1;
        if (bad) atomicOr(A.flags, FLAG_SINGULAR);
    }
    __syncthreads();
    // matrices at the current node
    const double2* Hz;
    const double2* LUz = nullptr;
    const int* Pz = nullptr;
    if (pc.start_local >= 0) {
        Hz = A.H + (size_t)pc.start_local * mat;
        if (STAGE) {
            LUz = A.LU + (size_t)pc.start_local * mat;
            Pz = A.piv + (size_t)pc.start_local * N;
        }
    } else {
        Hz = A.carryH + (size_t)pc.path * mat;
        if (STAGE) {
            LUz = A.carryLU + (size_t)pc.path * mat;
            Pz = A.carryPiv + (size_t)pc.path * N;
        }
    }
    for (int s = 0; s < pc.nsteps; ++s) {
        const int em = pc.first_local + 2 * s, en = em + 1;
        const double2* Hmid = A.H + (size_t)em * mat;
        const double2* Hnew = A.H + (size_t)en * mat;
        const double2* LUmid = STAGE ? A.LU + (size_t)em * mat : nullptr;
        const double2* LUnew = STAGE ? A.LU + (size_t)en * mat : nullptr;
        const int* Pmid = STAGE ? A.piv + (size_t)em * N : nullptr;
        const int* Pnew = STAGE ? A.piv + (size_t)en * N : nullptr;
        const double h = A.z[pc.z0 + s + 1] - A.z[pc.z0 + s];
        const double h2 = 0.5 * h, h6 = h / 6.0;
        // K1 = M_z c
        if (STAGE) apply_LU(LUz, Pz, Hz, N, v, c, kv, t);
        else apply_X(Hz, N, v, c, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = kv[i];
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K2 = M_mid (c + h/2 K1)
        if (STAGE) apply_LU(LUmid, Pmid, Hmid, N, v, y, kv, t);
        else apply_X(Hmid, N, v, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h2, kv[i].x, c[i].x), fma(h2, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K3 = M_mid (c + h/2 K2)
        if (STAGE) apply_LU(LUmid, Pmid, Hmid, N, v, y, kv, t);
        else apply_X(Hmid, N, v, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            acc[i] = make_double2(fma(2.0, kv[i].x, acc[i].x), fma(2.0, kv[i].y, acc[i].y));
            y[i] = make_double2(fma(h, kv[i].x, c[i].x), fma(h, kv[i].y, c[i].y));
        }
        __syncthreads();
        // K4 = M_new (c + h K3)
        if (STAGE) apply_LU(LUnew, Pnew, Hnew, N, v, y, kv, t);
        else apply_X(Hnew, N, v, y, kv);
        for (int i = threadIdx.x; i < N; i += RK_THREADS) {
            const double2 a = make_double2(acc[i].x + kv[i].x, acc[i].y + kv[i].y);
            c[i] = make_double2(fma(h6, a.x, c[i].x), fma(h6, a.y, c[i].y));
        }
        __syncthreads();
        Hz = Hnew;
        LUz = LUnew;
        Pz = Pnew;
    }
    bool finite = true;
    for (int i = threadIdx.x; i < N; i += RK_THREADS) {
        cg[i] = c[i];
        if (!isfinite(c[i].x) || !isfinite(c[i].y)) finite = false;
    }
    if (!finite) atomicOr(A.flags, FLAG_NONFINITE);
    // carry the matrices at the chunk's last node into the next chunk
    double2* cH = A.carryH + (size_t)pc.path * mat;
    if (Hz != cH) {
        for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cH[q] = Hz[q];
        if (STAGE) {
            double2* cL = A.carryLU + (size_t)pc.path * mat;
            int* cP = A.carryPiv + (size_t)pc.path * N;
            for (size_t q = threadIdx.x; q < mat; q += RK_THREADS) cL[q] = LUz[q];
            for (int q = threadIdx.x; q < N; q += RK_THREADS) cP[q] = Pz[q];
        }
    }
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
    if ((size_t)5 * N * sizeof(double2) > (size_t)227 * 1024)
        return fail(WPCCC_EINVAL, "wpccc_propagate: N too large for the RK4 kernel's shared memory");
    WPCCC_CUDA(cudaSetDevice(B->device));
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool two = B->n_centres == 2;
    const bool stage = two && B->solve_mode == WPCCC_SOLVE_STAGE;
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
    const size_t fixed = align((size_t)np * mat * sizeof(double2)) * (stage ? 2 : 1) +
                         align((size_t)np * N * sizeof(int)) + align((size_t)zoff[np] * sizeof(double)) +
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
    const size_t sz_carryLU = stage ? sz_carry : 0;
    const size_t sz_carryPiv = stage ? align((size_t)np * N * sizeof(int)) : 0;
    const size_t sz_z = align((size_t)zoff[np] * sizeof(double));
    const size_t sz_ev = align(ev.size() * sizeof(EvalDesc));
    const size_t sz_pc = align(pcs.size() * sizeof(PathChunk));
    const size_t sz_flags = 256;
    const size_t sz_S = two ? align((size_t)max_chunk_evals * mat * sizeof(double2)) : 0;
    const size_t sz_H = align((size_t)max_chunk_evals * mat * sizeof(double2));
    const size_t sz_piv = two ? align((size_t)max_chunk_evals * N * sizeof(int)) : 0;
    const size_t sz_info = two ? align((size_t)max_chunk_evals * sizeof(int)) : 0;
    const size_t sz_scr = align((size_t)max_chunk_evals * L.bytes_per_eval);
    const size_t need = sz_carry + sz_carryLU + sz_carryPiv + sz_z + sz_ev + sz_pc + sz_flags + sz_S + sz_H +
                        sz_piv + sz_info + sz_scr;
    wpccc_status s = ensure_workspace(B, need);
    if (s != WPCCC_OK) return s;
    char* w = static_cast<char*>(B->ws_ptr);
    double2* d_carry = reinterpret_cast<double2*>(w);
    w += sz_carry;
    double2* d_carryLU = stage ? reinterpret_cast<double2*>(w) : nullptr;
    w += sz_carryLU;
    int* d_carryPiv = stage ? reinterpret_cast<int*>(w) : nullptr;
    w += sz_carryPiv;
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
    const int rk_smem = (int)(5 * (size_t)N * sizeof(double2));
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));
    WPCCC_CUDA(cudaFuncSetAttribute(k_rk4<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, rk_smem));
    RkArgs ra;
    ra.N = N;
    ra.H = d_H;
    ra.LU = stage ? d_S : nullptr;
    ra.piv = stage ? d_piv : nullptr;
    ra.info = d_info;
    ra.carryH = d_carry;
    ra.carryLU = d_carryLU;
    ra.carryPiv = d_carryPiv;
    ra.c = static_cast<double2*>(c);
    ra.z = d_z;
    ra.flags = d_flags;

    for (int ch = 0; ch < n_chunks; ++ch) {
        const int nev = ev_begin[ch + 1] - ev_begin[ch];
        const int npc = pc_begin[ch + 1] - pc_begin[ch];
        s = launch_elements(B, d_ev + ev_begin[ch], nev, d_S, d_H, d_scr, st);
        if (s != WPCCC_OK) return s;
        if (two) {
            cudaEvent_t e0 = B->prof.begin(PROF_SOLVE, st);
            s = launch_solve(N, nev, d_S, stage ? nullptr : d_H, d_piv, d_info, st);
            if (s != WPCCC_OK) return s;
            B->prof.end(PROF_SOLVE, st, e0);
        }
        cudaEvent_t e1 = B->prof.begin(PROF_RK4, st);
        ra.pcs = d_pc + pc_begin[ch];
        if (stage) k_rk4<true><<<npc, RK_THREADS, rk_smem, st>>>(ra);
        else k_rk4<false><<<npc, RK_THREADS, rk_smem, st>>>(ra);
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
