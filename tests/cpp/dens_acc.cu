// CPU check of the compensated FP32 density accumulator of the mixed path
// (DensAcc<float> in roks_impl.cuh, compiled here as host code): sums of
// positive terms of mixed magnitude, as the |psi|^2 contributions of many
// bands to one grid point, accumulated term by term with add() and, split
// into groups, merged with add2() as the band-group slots are.  Compared with
// the sum in FP64 (exact to far below FP32 rounding at these lengths) and
// with the plain FP32 sum.  Prints one line per case:
//   n rel_err_pair rel_err_plain value_within_one_ulp
#include <cmath>
#include <cstdio>
#include <random>
#include <vector>

#include "roks_impl.cuh"

using roks::DensAcc;

int main() {
    std::mt19937_64 rng(2024);
    std::uniform_real_distribution<double> u(0.0, 1.0);
    for (int n : {10, 1000, 100000, 1000000}) {
        std::vector<float> v(n);
        for (int i = 0; i < n; ++i) v[i] = (float)(u(rng) * std::pow(10.0, -4.0 * u(rng)));
        double exact = 0.0;
        float plain = 0.0f;
        for (float x : v) { exact += (double)x; plain += x; }
        // term by term
        DensAcc<float>::S a = DensAcc<float>::make(v[0]);
        for (int i = 1; i < n; ++i) a = DensAcc<float>::add(a, v[i]);
        // eight groups merged in order (the band-group slots)
        const int ng = 8, gs = (n + ng - 1) / ng;
        DensAcc<float>::S g = DensAcc<float>::make(0.0f);
        for (int k = 0; k < ng; ++k) {
            DensAcc<float>::S p = DensAcc<float>::make(0.0f);
            for (int i = k * gs; i < std::min(n, (k + 1) * gs); ++i) p = DensAcc<float>::add(p, v[i]);
            g = k == 0 ? p : DensAcc<float>::add2(g, p);
        }
        const double pair = (double)a.x + (double)a.y;
        const double grouped = (double)g.x + (double)g.y;
        const double err_pair = std::fmax(std::fabs(pair - exact), std::fabs(grouped - exact)) / exact;
        const double err_plain = std::fabs((double)plain - exact) / exact;
        const float val = DensAcc<float>::value(a);
        const float ref = (float)exact;
        const bool ulp_ok = std::fabs((double)val - (double)ref) <= (double)std::nextafter(ref, 2.0f * ref) - ref;
        std::printf("%d %.3e %.3e %d\n", n, err_pair, err_plain, ulp_ok ? 1 : 0);
    }
    return 0;
}
