// fft_core.cuh -- complex helpers, radix-2/3/4/5/8 codelets and the
// shared-memory Stockham pass used by every transform of the library.
//
// A tile holds TL independent lines of length N in shared memory, element e
// of line l at buf[e * LS + l] (LS = TL + 1), so that a warp touching
// consecutive lines touches consecutive words.  A transform is a sequence of
// Stockham autosort passes (radices 8, 5, 4, 3, 2 in that order of
// extraction); each pass reads its butterfly inputs into registers, waits,
// and writes the outputs back in place.  Functions are __host__ __device__
// so the pass arithmetic can also be exercised on the CPU.
#pragma once

#include <vector_types.h>

#ifndef __CUDACC__
#ifndef __forceinline__
#define __forceinline__ inline
#endif
#endif

namespace roks {

template <typename T> struct cplx_t;
template <> struct cplx_t<float> { using type = float2; };
template <> struct cplx_t<double> { using type = double2; };
template <typename T> using c2 = typename cplx_t<T>::type;

template <typename T>
__host__ __device__ __forceinline__ c2<T> mk(T x, T y) { c2<T> r; r.x = x; r.y = y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V cadd(V a, V b) { V r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V csub(V a, V b) { V r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename V>
__host__ __device__ __forceinline__ V cmul(V a, V b) {
    V r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// conj(a) * b
template <typename V>
__host__ __device__ __forceinline__ V cmulc(V a, V b) {
    V r; r.x = a.x * b.x + a.y * b.y; r.y = a.x * b.y - a.y * b.x; return r;
}
template <typename V, typename S>
__host__ __device__ __forceinline__ V cscale(V a, S s) { V r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by dir * i  (dir = +1 or -1)
template <int DIR, typename V>
__host__ __device__ __forceinline__ V mul_i(V a) {
    V r;
    if (DIR > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

// ---------------------------------------------------------------- plans
// Radix sequence of a length: factors of 8 first, then 5, 4, 3, 2.
__host__ __device__ constexpr int plan_radix(int n, int pass) {
    const int cand[5] = {8, 5, 4, 3, 2};
    int p = 0;
    for (int c = 0; c < 5; ++c) {
        while (n % cand[c] == 0 && n > 1) {
            if (p == pass) return cand[c];
            n /= cand[c];
            ++p;
        }
    }
    return 1;
}
__host__ __device__ constexpr int plan_passes(int n) {
    int p = 0;
    while (plan_radix(n, p) > 1) ++p;
    return p;
}
// product of the radices of passes before `pass` (Stockham Ns)
__host__ __device__ constexpr int plan_ns(int n, int pass) {
    int ns = 1;
    for (int p = 0; p < pass; ++p) ns *= plan_radix(n, p);
    return ns;
}
__host__ __device__ constexpr bool plan_ok(int n) {
    int m = n;
    for (int p = 0; p < 32 && m > 1; ++p) {
        int r = plan_radix(n, p);
        if (r <= 1) return false;
        m /= r;
    }
    return m == 1;
}

// ---------------------------------------------------------------- codelets
// In-place DFT of R points: v_r <- sum_s v_s exp(DIR * 2 pi i r s / R).
template <int R, int DIR, typename V> struct Dft;

template <int DIR, typename V> struct Dft<2, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        V a = cadd(v[0], v[1]); V b = csub(v[0], v[1]); v[0] = a; v[1] = b;
    }
};

template <int DIR, typename V> struct Dft<3, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        using T = decltype(v[0].x);
        const T h = T(0.86602540378443864676);         // sin(2 pi / 3)
        V t = cadd(v[1], v[2]);
        V u = mul_i<DIR>(cscale(csub(v[1], v[2]), h));
        V m = csub(v[0], cscale(t, T(0.5)));
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, u);
        v[2] = csub(m, u);
    }
};

template <int DIR, typename V> struct Dft<4, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), t3 = mul_i<DIR>(csub(v[1], v[3]));
        v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
        v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
    }
};

template <int DIR, typename V> struct Dft<5, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        using T = decltype(v[0].x);
        const T c1 = T(0.30901699437494742410);   // cos(2 pi / 5)
        const T c2 = T(-0.80901699437494742410);  // cos(4 pi / 5)
        const T s1 = T(0.95105651629515357212);   // sin(2 pi / 5)
        const T s2 = T(0.58778525229247312917);   // sin(4 pi / 5)
        V t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
        V u1 = csub(v[1], v[4]), u2 = csub(v[2], v[3]);
        V a1 = cadd(v[0], cadd(cscale(t1, c1), cscale(t2, c2)));
        V a2 = cadd(v[0], cadd(cscale(t1, c2), cscale(t2, c1)));
        V b1 = mul_i<DIR>(cadd(cscale(u1, s1), cscale(u2, s2)));
        V b2 = mul_i<DIR>(csub(cscale(u1, s2), cscale(u2, s1)));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd(a1, b1); v[4] = csub(a1, b1);
        v[2] = cadd(a2, b2); v[3] = csub(a2, b2);
    }
};

template <int DIR, typename V> struct Dft<8, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        using T = decltype(v[0].x);
        const T r2 = T(0.70710678118654752440);    // cos(pi / 4)
        V e[4] = {v[0], v[2], v[4], v[6]};
        V o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR, V>::run(e);
        Dft<4, DIR, V>::run(o);
        // twiddles exp(DIR i pi k / 4), k = 1, 2, 3
        V w1 = cscale(cadd(o[1], mul_i<DIR>(o[1])), r2);
        V w2 = mul_i<DIR>(o[2]);
        V w3 = cscale(csub(mul_i<DIR>(o[3]), o[3]), r2);
        v[0] = cadd(e[0], o[0]); v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1);   v[5] = csub(e[1], w1);
        v[2] = cadd(e[2], w2);   v[6] = csub(e[2], w2);
        v[3] = cadd(e[3], w3);   v[7] = csub(e[3], w3);
    }
};

// ---------------------------------------------------------------- Stockham
// One pass of radix R with Ns = NS over all TL lines of a tile, in place.
// tw[t] = exp(-2 pi i t / N); the inverse (DIR = +1) uses its conjugate.
// Butterfly b of a line reads elements b + r N/R and writes
// (b / NS) NS R + (b mod NS) + r NS.
template <typename V, int N, int R, int NS, int DIR>
__host__ __device__ __forceinline__ void twiddle_dft(V* v, const V* tw, int j) {
    const int k = j % NS;
    if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            const int t = r * k * (N / (NS * R));
            V w = tw[t];
            if (DIR > 0) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
    Dft<R, DIR, V>::run(v);
}

#ifdef __CUDACC__
template <typename V, int N, int R, int NS, int DIR, int TL, int LS, int NT>
__device__ __forceinline__ void stockham_pass(V* buf, const V* tw) {
    constexpr int NBF = N / R;
    constexpr int TOT = NBF * TL;
    constexpr int PER = (TOT + NT - 1) / NT;
    V v[PER][R];
    const int tid = threadIdx.x;
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int beta = tid + q * NT;
        if (beta < TOT) {
            const int line = beta % TL, j = beta / TL;
#pragma unroll
            for (int r = 0; r < R; ++r) v[q][r] = buf[(j + r * NBF) * LS + line];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int beta = tid + q * NT;
        if (beta < TOT) {
            const int line = beta % TL, j = beta / TL;
            twiddle_dft<V, N, R, NS, DIR>(v[q], tw, j);
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) buf[(base + r * NS) * LS + line] = v[q][r];
        }
    }
    __syncthreads();
}

template <typename V, int N, int DIR, int TL, int LS, int NT, int P>
__device__ __forceinline__ void run_passes(V* buf, const V* tw) {
    if constexpr (P < plan_passes(N)) {
        stockham_pass<V, N, plan_radix(N, P), plan_ns(N, P), DIR, TL, LS, NT>(buf, tw);
        run_passes<V, N, DIR, TL, LS, NT, P + 1>(buf, tw);
    }
}

// Full N-point transform of all TL lines of the tile (unnormalised).
template <typename V, int N, int DIR, int TL, int LS, int NT>
__device__ __forceinline__ void tile_fft(V* buf, const V* tw) {
    static_assert(plan_ok(N), "unsupported transform length");
    run_passes<V, N, DIR, TL, LS, NT, 0>(buf, tw);
}
#endif

// Host-side reference of the same pass sequence on one line (used by a CPU
// test of the pass arithmetic).
template <typename V, int N, int DIR, int P>
__host__ void host_passes(V* line, const V* tw) {
    if constexpr (P < plan_passes(N)) {
        constexpr int R = plan_radix(N, P);
        constexpr int NS = plan_ns(N, P);
        constexpr int NBF = N / R;
        V out[N];
        for (int j = 0; j < NBF; ++j) {
            V v[R];
            for (int r = 0; r < R; ++r) v[r] = line[j + r * NBF];
            twiddle_dft<V, N, R, NS, DIR>(v, tw, j);
            const int base = (j / NS) * NS * R + (j % NS);
            for (int r = 0; r < R; ++r) out[base + r * NS] = v[r];
        }
        for (int e = 0; e < N; ++e) line[e] = out[e];
        host_passes<V, N, DIR, P + 1>(line, tw);
    }
}

}  // namespace roks
