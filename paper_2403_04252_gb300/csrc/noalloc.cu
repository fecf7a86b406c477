// wpccc_matrix_elements_noalloc: matrix elements without any device allocation.
//
// Some callers cannot let a library allocate device memory during a call: a host
// framework that has reserved the device memory up front (so a further cudaMalloc
// fails or fragments its pool), or a latency-critical loop that cannot absorb the
// device-wide synchronisation of cudaMalloc/cudaFree.  For them this entry point
// runs the same element kernels as wpccc_matrix_elements with its scratch memory
// (node tables, molecular-frame blocks, the position list) in the fixed array
// below, which every GPU that loads this library holds until the process exits.
#include <algorithm>
#include <mutex>
#include <vector>

#include "wpccc_internal.cuh"

namespace wpccc {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;   // 64 MiB
static_assert(NOALLOC_SCRATCH_BYTES == WPCCC_NOALLOC_SCRATCH_BYTES, "header and library disagree");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once per device and kept for the
// life of the process: a cudaDeviceReset (a new primary context) leaves the kept address stale, so the
// library does not support calls on a device after it has been reset.
static wpccc_status noalloc_scratch(int device, void** out) {
    if (device < 0 || device >= NOALLOC_MAX_DEVICES)
        return fail(WPCCC_EINVAL, "wpccc_matrix_elements_noalloc: device index beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_noalloc_ptr[device] = p;
    }
    *out = g_noalloc_ptr[device];
    return WPCCC_OK;
}

}  // namespace wpccc

using namespace wpccc;

extern "C" wpccc_status wpccc_matrix_elements_noalloc(wpccc_basis B, double b, double v, int nz, const double* z,
                                                      void* S, void* H, void* stream) {
    if (!B || !z || !S || !H) return fail(WPCCC_EINVAL, "wpccc_matrix_elements_noalloc: null argument");
    if (nz < 1) return fail(WPCCC_EINVAL, "wpccc_matrix_elements_noalloc: nz < 1");
    if (!(b > 0.0) || !(v > 0.0)) return fail(WPCCC_EINVAL, "wpccc_matrix_elements_noalloc: b and v must be > 0");
    const ElemScratch L = elem_scratch_layout(B);
    // one position needs its element scratch plus its entry of the position list (the list is rounded up
    // to 256 bytes, so 256 bytes cover that rounding and any list of up to 256 / sizeof(EvalDesc) entries)
    if (L.bytes_per_eval + 256 > NOALLOC_SCRATCH_BYTES)
        return fail(WPCCC_EINVAL, "wpccc_matrix_elements_noalloc: one position of this basis needs " +
                                      std::to_string(L.bytes_per_eval + 256) +
                                      " bytes of scratch, more than the fixed " +
                                      std::to_string(NOALLOC_SCRATCH_BYTES) + " bytes");
    WPCCC_CUDA(cudaSetDevice(B->device));
    void* base = nullptr;
    wpccc_status s = noalloc_scratch(B->device, &base);
    if (s != WPCCC_OK) return s;
    // positions per launch: the list (rounded up to 256 bytes) and the scratch fit the array, and the element
    // kernels take one grid row per position (at most 65535)
    const int chunk = (int)std::min<size_t>(
        {(size_t)nz, (size_t)MAX_EVALS_PER_LAUNCH, (NOALLOC_SCRATCH_BYTES - 256) / (L.bytes_per_eval + sizeof(EvalDesc))});
    char* wsb = static_cast<char*>(base);
    EvalDesc* dev_ev = reinterpret_cast<EvalDesc*>(wsb);
    void* scratch = wsb + ((chunk * sizeof(EvalDesc) + 255) / 256) * 256;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    std::vector<EvalDesc> ev(chunk);
    const size_t mat = (size_t)B->N * B->N;
    for (int k0 = 0; k0 < nz; k0 += chunk) {
        const int n = chunk < nz - k0 ? chunk : nz - k0;
        for (int k = 0; k < n; ++k) ev[k] = EvalDesc{b, v, z[k0 + k], 0, 0};
        WPCCC_CUDA(cudaMemcpyAsync(dev_ev, ev.data(), n * sizeof(EvalDesc), cudaMemcpyHostToDevice, st));
        s = launch_elements(B, dev_ev, n, static_cast<double2*>(S) + k0 * mat, static_cast<double2*>(H) + k0 * mat,
                            scratch, st);
        if (s != WPCCC_OK) return s;
        // the host list and the scratch are reused by the next chunk
        WPCCC_CUDA(cudaStreamSynchronize(st));
    }
    return WPCCC_OK;
}
