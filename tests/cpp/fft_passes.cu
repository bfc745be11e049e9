// CPU check of the transform arithmetic of the CUDA path (fft_core.cuh):
// every compiled grid length runs its pass sequence (radix plan, codelets,
// twiddles, Stockham index map) on random lines in both directions and is
// compared with the DFT sum X_k = sum_j x_j exp(dir 2 pi i j k / N) written
// out here.  Prints one line per length and direction: N dir max_rel_err.
#include <cmath>
#include <cstdio>
#include <random>

#include "fft_core.cuh"

using roks::host_passes;

template <int N, int DIR>
double check(std::mt19937_64& rng) {
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    double2 tw[N], x[N], y[N];
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < N; ++t) tw[t] = make_double2(std::cos(-two_pi * t / N), std::sin(-two_pi * t / N));
    double worst = 0.0;
    for (int trial = 0; trial < 4; ++trial) {
        for (int j = 0; j < N; ++j) x[j] = y[j] = make_double2(u(rng), u(rng));
        host_passes<double2, N, DIR, 0>(y, tw);
        double scale = 0.0, err = 0.0;
        for (int k = 0; k < N; ++k) {
            long double re = 0, im = 0;
            for (int j = 0; j < N; ++j) {
                const long double a = DIR * (long double)two_pi * (long double)((j * k) % N) / N;
                re += x[j].x * std::cos(a) - x[j].y * std::sin(a);
                im += x[j].x * std::sin(a) + x[j].y * std::cos(a);
            }
            scale = std::fmax(scale, std::hypot((double)re, (double)im));
            err = std::fmax(err, std::hypot(y[k].x - (double)re, y[k].y - (double)im));
        }
        worst = std::fmax(worst, err / scale);
    }
    return worst;
}

template <int N>
void both(std::mt19937_64& rng) {
    std::printf("%d -1 %.3e\n", N, check<N, -1>(rng));
    std::printf("%d 1 %.3e\n", N, check<N, 1>(rng));
}

int main() {
    std::mt19937_64 rng(12345);
    both<16>(rng);
    both<24>(rng);
    both<32>(rng);
    both<48>(rng);
    both<72>(rng);
    both<96>(rng);
    both<120>(rng);
    return 0;
}
