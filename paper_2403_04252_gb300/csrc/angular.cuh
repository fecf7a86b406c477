// Angular-momentum functions evaluated on the device: factorials, Clebsch-Gordan
// coefficients, Wigner small-d matrices and associated Legendre functions.
#pragma once

#include <cuda_runtime.h>

namespace wpccc {

// n! in double; exact for n <= 22, correctly ordered products beyond.
__device__ inline double dfact(int n) {
    double p = 1.0;
    for (int k = 2; k <= n; ++k) p *= (double)k;
    return p;
}

// <j1 m1 j2 m2 | J M> for integer arguments (Racah's closed formula).
__device__ inline double clebsch_gordan(int j1, int m1, int j2, int m2, int J, int M) {
    if (m1 + m2 != M || abs(m1) > j1 || abs(m2) > j2 || abs(M) > J) return 0.0;
    if (J < abs(j1 - j2) || J > j1 + j2) return 0.0;
    double pre = (2.0 * J + 1.0) * dfact(J + j1 - j2) * dfact(J - j1 + j2) * dfact(j1 + j2 - J) /
                 dfact(j1 + j2 + J + 1);
    pre *= dfact(J + M) * dfact(J - M) * dfact(j1 - m1) * dfact(j1 + m1) * dfact(j2 - m2) * dfact(j2 + m2);
    double sum = 0.0;
    for (int k = 0; k <= j1 + j2 - J; ++k) {
        int d1 = j1 + j2 - J - k, d2 = j1 - m1 - k, d3 = j2 + m2 - k;
        int d4 = J - j2 + m1 + k, d5 = J - j1 - m2 + k;
        if (d1 < 0 || d2 < 0 || d3 < 0 || d4 < 0 || d5 < 0) continue;
        double t = 1.0 / (dfact(k) * dfact(d1) * dfact(d2) * dfact(d3) * dfact(d4) * dfact(d5));
        sum += (k & 1) ? -t : t;
    }
    return sqrt(pre) * sum;
}

// d^j_{mp m}(beta) = <j mp| exp(-i beta J_y) |j m>, given c = cos(beta/2), s = sin(beta/2).
__device__ inline double wigner_small_d(int j, int mp, int m, double c, double s) {
    double pre = sqrt(dfact(j + mp) * dfact(j - mp) * dfact(j + m) * dfact(j - m));
    double tot = 0.0;
    for (int k = 0; k <= 2 * j; ++k) {
        int a = j + m - k, cc = mp - m + k, d = j - mp - k;
        if (a < 0 || cc < 0 || d < 0) continue;
        double t = pre / (dfact(a) * dfact(k) * dfact(cc) * dfact(d));
        int pc = 2 * j + m - mp - 2 * k, ps = mp - m + 2 * k;
        for (int e = 0; e < pc; ++e) t *= c;
        for (int e = 0; e < ps; ++e) t *= s;
        tot += ((mp - m + k) & 1) ? -t : t;
    }
    return tot;
}

// Associated Legendre P_l^m(x), 0 <= m <= l, with the Condon-Shortley phase, by the
// standard upward recurrence in l from P_m^m = (-1)^m (2m-1)!! (1-x^2)^{m/2}.
__device__ inline double assoc_legendre(int l, int m, double x) {
    double pmm = 1.0;
    if (m > 0) {
        double sq = sqrt((1.0 - x) * (1.0 + x));
        double fct = 1.0;
        for (int i = 1; i <= m; ++i) {
            pmm *= -fct * sq;
            fct += 2.0;
        }
    }
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pl = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pl = (x * (2.0 * ll - 1.0) * pm1 - (ll + m - 1.0) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = pl;
    }
    return pl;
}

}  // namespace wpccc
