// Row tiles of the tensor-core contractions (precision modes 3, 4 and 5): the target states grouped by
// their molecular-frame projection q', and each group cut into tiles that one 128-row MMA tile holds.
// The contraction itself is in mol_tc64.cu.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <vector>

#include "tc_ptx.cuh"
#include "wpccc_internal.cuh"

namespace wpccc {

// The radial tables as double-floats, for the node tables' interpolation on the FP32 pipe.
__global__ void k_split_table(long long n, const double* __restrict__ f, float2* __restrict__ out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const float h = __double2float_rn(f[i]);
        out[i] = make_float2(h, __double2float_rn(f[i] - (double)h));
    }
}

static wpccc_status split_table(const double* f, long long n, float2** out) {
    WPCCC_CUDA(cudaMalloc((void**)out, n * sizeof(float2)));
    k_split_table<<<(unsigned)((n + 255) / 256), 256>>>(n, f, *out);
    WPCCC_CHECK_LAUNCH("k_split_table");
    WPCCC_CUDA(cudaDeviceSynchronize());
    return WPCCC_OK;
}

// target states per row tile: A_T r_T and A_T r_T V_T rows of at most 56 states (112 of the 128 rows)
constexpr int TC_TILE_STATES = 56;

// Row tiles: each q' group cut into tiles of at most 56 states (near-equal sizes).  A tile of n states owns
// 2 n consecutive rows of the slice planes: its A_T r_T rows, then its A_T r_T V_T rows.  Enables the
// layout on the basis.
wpccc_status tc_prepare(wpccc_basis_s* B) {
    if (B->tc_layout) return WPCCC_OK;
    if (B->n_centres != 2) return fail(WPCCC_EUNSUPPORTED, "the tensor-core contraction needs a two-centre basis");
    if (!encode_fn()) return fail(WPCCC_EUNSUPPORTED, "tensor-core contraction: cuTensorMapEncodeTiled unavailable");
    if (B->G % 128 != 0)
        return fail(WPCCC_EUNSUPPORTED, "tensor-core contraction: the node count must be a multiple of 128");
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
    if ((s = ensure_tc_err(B)) != WPCCC_OK) return s;
    if ((s = split_table(B->T.f, (long long)B->T.n_rad * B->Nr, &B->fT2)) != WPCCC_OK) return s;
    if ((s = split_table(B->P.f, (long long)B->P.n_rad * B->Nr, &B->fP2)) != WPCCC_OK) return s;
    B->n_qgroups = ntl;
    B->qg_max = qmax;
    B->tc_layout = true;
    return WPCCC_OK;
}

wpccc_status ensure_tc_err(wpccc_basis_s* B) {
    if (B->tc_err) return WPCCC_OK;
    WPCCC_CUDA(cudaMalloc((void**)&B->tc_err, sizeof(int)));
    WPCCC_CUDA(cudaMemset(B->tc_err, 0, sizeof(int)));
    return WPCCC_OK;
}

}  // namespace wpccc
