// CPU run of the DIIS window test and coefficient solve of the CUDA path
// (diis_window_coefficients in roks_diis.cuh).  Reads cases from stdin:
//   ncase, then per case: n tol, then n x n Gram matrix rows (oldest pair first)
// and prints per case: h d_0 .. d_{h-1}.
#include <cstdio>

#include "roks_diis.cuh"

int main() {
    int ncase = 0;
    if (std::scanf("%d", &ncase) != 1) return 1;
    for (int c = 0; c < ncase; ++c) {
        int n = 0;
        double tol = 0.0;
        if (std::scanf("%d %lf", &n, &tol) != 2 || n < 1 || n > roks::kDiisMax) return 1;
        double B[roks::kDiisMax * roks::kDiisMax] = {0.0};
        roks::DiisOrder ord{};
        ord.n = n;
        // ring slots in a rotated order, as after the ring has wrapped
        for (int k = 0; k < n; ++k) ord.slot[k] = (k + 3) % roks::kDiisMax;
        for (int j = 0; j < n; ++j)
            for (int k = 0; k < n; ++k)
                if (std::scanf("%lf", &B[ord.slot[j] * roks::kDiisMax + ord.slot[k]]) != 1) return 1;
        double d[roks::kDiisMax];
        int slot[roks::kDiisMax];
        const int h = roks::diis_window_coefficients(B, ord, tol, d, slot);
        std::printf("%d", h);
        for (int i = 0; i < h; ++i) {
            if (slot[i] != ord.slot[n - h + i]) return 2;
            std::printf(" %.17g", d[i]);
        }
        std::printf("\n");
    }
    return 0;
}
