// CPU check of the transform arithmetic of the CUDA path (fft_core.cuh):
// every compiled grid length runs its pass sequence (radix plan, codelets,
// twiddles, Stockham index map) on random lines in both directions and is
// compared with the DFT sum X_k = sum_j x_j exp(dir 2 pi i j k / N) written
// out here.  Prints one line per length and direction: N dir max_rel_err.
//
// Then the sphere-pruned first pass: lines whose entries are random for the
// frequencies |i| <= (N - 1) / 4 and zero elsewhere, transformed with the
// first pass's known-zero inputs left out (sphere_zero_mask), against the
// same DFT sum; and, independently of the arithmetic, every input the mask
// drops is checked to be an element outside that frequency range.  Prints
// "prune N dir max_rel_err zero_inputs_of_R0 mask_ok".
//
// Last, every pruned codelet (radix 2, 3, 4, 5, 8) for every mask it accepts,
// against the plain codelet on random inputs with zeros at the mask: prints
// "codelet R dir max_rel_err masks_checked".
#include <cmath>
#include <cstdio>
#include <random>
#include <utility>

#include "fft_core.cuh"

using roks::host_passes;

template <int N, int DIR, bool PRUNE = false>
double check(std::mt19937_64& rng) {
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    double2 tw[N], x[N], y[N];
    const double two_pi = 6.283185307179586476925286766559;
    const int nb = roks::sphere_prune_nmax(N);
    for (int t = 0; t < N; ++t) tw[t] = make_double2(std::cos(-two_pi * t / N), std::sin(-two_pi * t / N));
    double worst = 0.0;
    for (int trial = 0; trial < 4; ++trial) {
        for (int j = 0; j < N; ++j) {
            const int i = j <= N / 2 ? j : j - N;
            x[j] = y[j] = (!PRUNE || (i >= -nb && i <= nb)) ? make_double2(u(rng), u(rng)) : make_double2(0.0, 0.0);
        }
        if constexpr (PRUNE)
            host_passes<double2, N, DIR, 0, roks::sphere_zero_mask(N)>(y, tw);
        else
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

// every dropped input r (elements j + r S, j < S) lies outside |i| <= nb
template <int N>
bool mask_ok() {
    constexpr unsigned Z = roks::sphere_zero_mask(N);
    constexpr int R0 = roks::plan_radix(N, 0), S = N / R0;
    const int nb = roks::sphere_prune_nmax(N);
    for (int r = 0; r < R0; ++r) {
        if (!((Z >> r) & 1u)) continue;
        for (int j = 0; j < S; ++j) {
            const int e = j + r * S, i = e <= N / 2 ? e : e - N;
            if (i >= -nb && i <= nb) return false;
        }
    }
    return true;
}

template <int R, int DIR, unsigned Z>
double codelet_err(std::mt19937_64& rng) {
    std::uniform_real_distribution<double> u(-1.0, 1.0);
    double worst = 0.0;
    for (int trial = 0; trial < 3; ++trial) {
        double2 a[R], b[R];
        for (int r = 0; r < R; ++r)
            a[r] = b[r] = ((Z >> r) & 1u) ? make_double2(0.0, 0.0) : make_double2(u(rng), u(rng));
        roks::Dft<R, DIR, double2>::run(a);
        roks::DftZ<R, DIR, double2, Z>::run(b);
        double scale = 1e-300, err = 0.0;
        for (int r = 0; r < R; ++r) {
            scale = std::fmax(scale, std::hypot(a[r].x, a[r].y));
            err = std::fmax(err, std::hypot(a[r].x - b[r].x, a[r].y - b[r].y));
        }
        worst = std::fmax(worst, err / scale);
    }
    return worst;
}

// masks a pruned codelet accepts: input 0 is never pruned (for radix 8 the
// first even and the first odd input, the inputs 0 of its 4-point parts)
template <int R>
constexpr bool accepted(unsigned z) {
    return R == 8 ? !(z & 3u) : !(z & 1u);
}

template <int R, int DIR, unsigned Z>
void one_mask(std::mt19937_64& rng, double& worst, int& count) {
    if constexpr (accepted<R>(Z)) {
        worst = std::fmax(worst, codelet_err<R, DIR, Z>(rng));
        ++count;
    }
}

template <int R, int DIR, unsigned... Z>
void all_masks(std::mt19937_64& rng, double& worst, int& count, std::integer_sequence<unsigned, Z...>) {
    (one_mask<R, DIR, Z>(rng, worst, count), ...);
}

template <int R, int DIR>
void codelet_masks(std::mt19937_64& rng) {
    double worst = 0.0;
    int count = 0;
    all_masks<R, DIR>(rng, worst, count, std::make_integer_sequence<unsigned, (1u << R)>{});
    std::printf("codelet %d %d %.3e %d\n", R, DIR, worst, count);
}

template <int N>
void both(std::mt19937_64& rng) {
    std::printf("%d -1 %.3e\n", N, check<N, -1>(rng));
    std::printf("%d 1 %.3e\n", N, check<N, 1>(rng));
    const int nz = __builtin_popcount(roks::sphere_zero_mask(N));
    const int ok = mask_ok<N>() ? 1 : 0;
    std::printf("prune %d -1 %.3e %d %d\n", N, check<N, -1, true>(rng), nz, ok);
    std::printf("prune %d 1 %.3e %d %d\n", N, check<N, 1, true>(rng), nz, ok);
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
    codelet_masks<2, -1>(rng);
    codelet_masks<2, 1>(rng);
    codelet_masks<3, -1>(rng);
    codelet_masks<3, 1>(rng);
    codelet_masks<4, -1>(rng);
    codelet_masks<4, 1>(rng);
    codelet_masks<5, -1>(rng);
    codelet_masks<5, 1>(rng);
    codelet_masks<8, -1>(rng);
    codelet_masks<8, 1>(rng);
    return 0;
}
