// Geometry helpers of the element kernels and of their adjoint (one definition, so both pick the
// same node radii and interpolation stencils).
#pragma once

#include <cuda_runtime.h>

namespace wpccc {

// ---------------------------------------------------------------------------
// geometry shared by the kernels; explicit round-to-nearest operations so that
// the interpolation stencils are chosen from exactly the same radii as a plain
// IEEE evaluation of the same formulas (no contraction into FMA)
// ---------------------------------------------------------------------------
static __device__ inline double dist_R(double b, double z) {
    return __dsqrt_rn(__dadd_rn(__dmul_rn(b, b), __dmul_rn(z, z)));
}

// Largest j with r[j] <= x (-1 if x < r[0]); 5-point stencil start and Lagrange weights.
// Returns false when x lies beyond the last grid point (the function is zero there).
static __device__ inline bool stencil5(const double* __restrict__ r, int Nr, double x, int& s, double L[5]) {
    if (x > r[Nr - 1]) return false;
    int lo = -1, hi = Nr;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (r[mid] <= x) lo = mid;
        else hi = mid;
    }
    s = min(max(lo - 2, 0), Nr - 5);
    double rn[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) rn[k] = r[s + k];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        double p = 1.0;
#pragma unroll
        for (int c = 0; c < 5; ++c)
            if (c != a) p *= (x - rn[c]) / (rn[a] - rn[c]);
        L[a] = p;
    }
    return true;
}

// The same stencil with the Lagrange denominators 1/prod_{c != a}(r_{s+a} - r_{s+c}) read from a
// table made at set-up (inv_den[s][a], 5 per stencil start), so no division per interpolation.
static __device__ inline bool stencil5_fast(const double* __restrict__ r, const double* __restrict__ inv_den, int Nr,
                                     double x, int& s, double L[5]) {
    if (x > r[Nr - 1]) return false;
    int lo = -1, hi = Nr;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (r[mid] <= x) lo = mid;
        else hi = mid;
    }
    s = min(max(lo - 2, 0), Nr - 5);
    double dx[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) dx[k] = x - r[s + k];
#pragma unroll
    for (int a = 0; a < 5; ++a) {
        double p = inv_den[(size_t)s * 5 + a];
#pragma unroll
        for (int c = 0; c < 5; ++c)
            if (c != a) p *= dx[c];
        L[a] = p;
    }
    return true;
}

}  // namespace wpccc
