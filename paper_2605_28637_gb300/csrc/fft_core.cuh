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

#include <utility>
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
// a * s + c with s real
template <typename V, typename S>
__host__ __device__ __forceinline__ V cfma(V a, S s, V c) {
    V r; r.x = a.x * s + c.x; r.y = a.y * s + c.y; return r;
}
// a + dir i b and a - dir i b, without forming i b (its components swap
// places, which paired instructions cannot do)
template <int DIR, typename V>
__host__ __device__ __forceinline__ V cadd_i(V a, V b) {
    V r;
    if (DIR > 0) { r.x = a.x - b.y; r.y = a.y + b.x; } else { r.x = a.x + b.y; r.y = a.y - b.x; }
    return r;
}
template <int DIR, typename V>
__host__ __device__ __forceinline__ V csub_i(V a, V b) { return cadd_i<-DIR, V>(a, b); }

// Paired FP32 arithmetic (sm_100 and later): the complex float2 add,
// subtract, real scale and real multiply-add are each one instruction on
// both components, rounded to nearest like the scalar forms.  These
// overloads take precedence over the templates above in device code; the
// codelets below are written so that every swap of components (the factor i)
// stays in cadd_i / csub_i.
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return __fmul2_rn(a, make_float2(s, s)); }
__device__ __forceinline__ float2 cfma(float2 a, float s, float2 c) { return __ffma2_rn(a, make_float2(s, s), c); }
#endif

// ---------------------------------------------------------------- plans
// Radix sequence of a transform length.  The grid sizes of the workloads get
// two passes with register codelets up to 16 points (96 = 12 x 8,
// 120 = 15 x 8, 72 = 9 x 8, 48 = 8 x 6, 24 = 8 x 3, 32 = 8 x 4, 16 = 4 x 4);
// other lengths fall back to factors of 8, 5, 4, 3, 2 in that order.
__host__ __device__ constexpr int plan_radix(int n, int pass) {
    switch (n) {
        case 96: return pass == 0 ? 12 : (pass == 1 ? 8 : 1);
        case 120: return pass == 0 ? 15 : (pass == 1 ? 8 : 1);
        case 72: return pass == 0 ? 9 : (pass == 1 ? 8 : 1);
        case 48: return pass == 0 ? 8 : (pass == 1 ? 6 : 1);
        case 16: return pass == 0 ? 4 : (pass == 1 ? 4 : 1);
        default: break;
    }
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
        if (r <= 1 || m % r != 0) return false;
        m /= r;
    }
    return m == 1;
}

// Sphere pruning of the first pass.  When only the frequencies |i| <= nb of
// a line are nonzero, input r of every butterfly of the first pass (element
// j + r S of the line, S = N / R0 for the pass's radix R0, j < S) is zero for
// nb / S < r <= (N - nb) / S - 1.  The kernels prune for
// nb = sphere_prune_nmax(N) = (N - 1) / 4, which covers every sphere whose
// density fits the grid without aliasing (N >= 4 nmax + 1); a larger sphere
// takes the full first pass.
__host__ __device__ constexpr int sphere_prune_nmax(int n) { return (n - 1) / 4; }
__host__ __device__ constexpr unsigned sphere_zero_mask(int n) {
    const int r0 = plan_radix(n, 0), S = n / r0, nb = sphere_prune_nmax(n);
    unsigned m = 0;
    for (int r = nb / S + 1; r <= (n - nb) / S - 1 && r < r0; ++r) m |= 1u << r;
    return m;
}

// ---------------------------------------------------------------- compile-time trigonometry
// cos and sin of 2 pi m / R from their Taylor series (argument reduced to
// [-pi, pi]; 30 terms give full double precision there).  Used only to fold
// the internal twiddles of the composite codelets into constants.
__host__ __device__ constexpr double ct_pi() { return 3.14159265358979323846264338327950288; }
__host__ __device__ constexpr double ct_series(double x, bool sine) {
    double term = sine ? x : 1.0, sum = term;
    const double x2 = x * x;
    for (int k = 1; k < 30; ++k) {
        const double a = sine ? (2.0 * k) * (2.0 * k + 1.0) : (2.0 * k - 1.0) * (2.0 * k);
        term = -term * x2 / a;
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double ct_angle(int m, int r) {
    double x = 2.0 * ct_pi() * double(m % r) / double(r);
    if (x > ct_pi()) x -= 2.0 * ct_pi();
    return x;
}
__host__ __device__ constexpr double ct_cos(int m, int r) { return ct_series(ct_angle(m, r), false); }
__host__ __device__ constexpr double ct_sin(int m, int r) { return ct_series(ct_angle(m, r), true); }

template <int... I, typename F>
__host__ __device__ __forceinline__ void sfor_impl(std::integer_sequence<int, I...>, F&& f) {
    (f(std::integral_constant<int, I>{}), ...);
}
// f(integral_constant<int, 0>) ... f(integral_constant<int, N-1>)
template <int N, typename F>
__host__ __device__ __forceinline__ void sfor(F&& f) {
    sfor_impl(std::make_integer_sequence<int, N>{}, f);
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
        V d = cscale(csub(v[1], v[2]), h);
        V m = cfma(t, T(-0.5), v[0]);
        v[0] = cadd(v[0], t);
        v[1] = cadd_i<DIR>(m, d);
        v[2] = csub_i<DIR>(m, d);
    }
};

template <int DIR, typename V> struct Dft<4, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        V t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
        V t2 = cadd(v[1], v[3]), d = csub(v[1], v[3]);
        v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
        v[1] = cadd_i<DIR>(t1, d); v[3] = csub_i<DIR>(t1, d);
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
        V a1 = cfma(t2, c2, cfma(t1, c1, v[0]));
        V a2 = cfma(t2, c1, cfma(t1, c2, v[0]));
        V b1 = cfma(u2, s2, cscale(u1, s1));
        V b2 = cfma(u2, -s1, cscale(u1, s2));
        v[0] = cadd(v[0], cadd(t1, t2));
        v[1] = cadd_i<DIR>(a1, b1); v[4] = csub_i<DIR>(a1, b1);
        v[2] = cadd_i<DIR>(a2, b2); v[3] = csub_i<DIR>(a2, b2);
    }
};

// The last butterflies of the 8-point DFT from the 4-point DFTs of the even
// (e) and odd (o) inputs, with the twiddles exp(DIR i pi k / 4), k = 1, 2, 3:
// (1 + DIR i) / sqrt 2, DIR i, (DIR i - 1) / sqrt 2.
template <int DIR, typename V> struct Dft8Combine {
    __host__ __device__ static __forceinline__ void run(V* v, const V* e, const V* o) {
        using T = decltype(v[0].x);
        const T r2 = T(0.70710678118654752440);    // cos(pi / 4)
        V w1 = cscale(cadd_i<DIR>(o[1], o[1]), r2);
        V w3 = cscale(csub_i<DIR>(o[3], o[3]), -r2);
        v[0] = cadd(e[0], o[0]);         v[4] = csub(e[0], o[0]);
        v[1] = cadd(e[1], w1);           v[5] = csub(e[1], w1);
        v[2] = cadd_i<DIR>(e[2], o[2]);  v[6] = csub_i<DIR>(e[2], o[2]);
        v[3] = cadd(e[3], w3);           v[7] = csub(e[3], w3);
    }
};

template <int DIR, typename V> struct Dft<8, DIR, V> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        V e[4] = {v[0], v[2], v[4], v[6]};
        V o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, DIR, V>::run(e);
        Dft<4, DIR, V>::run(o);
        Dft8Combine<DIR, V>::run(v, e, o);
    }
};

// x * exp(DIR 2 pi i M / R) with M, R compile-time constants.
template <int R, int M, int DIR, typename V>
__host__ __device__ __forceinline__ V twiddle_const(V x) {
    using T = decltype(x.x);
    constexpr int m = M % R;
    if constexpr (m == 0) {
        return x;
    } else if constexpr (2 * m == R) {
        V r; r.x = -x.x; r.y = -x.y; return r;
    } else if constexpr (4 * m == R) {
        return mul_i<DIR>(x);
    } else if constexpr (4 * m == 3 * R) {
        return mul_i<-DIR>(x);
    } else {
        constexpr double c = ct_cos(m, R);
        constexpr double sn = DIR * ct_sin(m, R);
        V r;
        r.x = x.x * T(c) - x.y * T(sn);
        r.y = x.x * T(sn) + x.y * T(c);
        return r;
    }
}

// Composite DFT of R = A * B points in registers (Cooley-Tukey, decimation
// in time): inputs n = B n1 + n2, outputs k = k1 + A k2,
// X[k] = sum_n2 W_B^{n2 k2} W_R^{n2 k1} sum_n1 x[B n1 + n2] W_A^{n1 k1}.
template <int A, int B, int DIR, typename V>
struct DftAB {
    __host__ __device__ static __forceinline__ void run(V* v) {
        constexpr int R = A * B;
        V y[B][A];
        sfor<B>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            V t[A];
            sfor<A>([&](auto n1c) { t[decltype(n1c)::value] = v[B * decltype(n1c)::value + n2]; });
            Dft<A, DIR, V>::run(t);
            sfor<A>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                y[n2][k1] = twiddle_const<R, n2 * k1, DIR>(t[k1]);
            });
        });
        sfor<A>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            V t[B];
            sfor<B>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value][k1]; });
            Dft<B, DIR, V>::run(t);
            sfor<B>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = t[decltype(k2c)::value]; });
        });
    }
};

template <int DIR, typename V> struct Dft<6, DIR, V> : DftAB<3, 2, DIR, V> {};
template <int DIR, typename V> struct Dft<9, DIR, V> : DftAB<3, 3, DIR, V> {};
template <int DIR, typename V> struct Dft<10, DIR, V> : DftAB<5, 2, DIR, V> {};
template <int DIR, typename V> struct Dft<12, DIR, V> : DftAB<4, 3, DIR, V> {};
template <int DIR, typename V> struct Dft<15, DIR, V> : DftAB<5, 3, DIR, V> {};
template <int DIR, typename V> struct Dft<16, DIR, V> : DftAB<4, 4, DIR, V> {};

// ---------------------------------------------------------------- pruned codelets
// The same DFTs when some inputs are known at compile time to be zero (bit n
// of Z: input n is zero and holds 0).  Additions with a known zero are left
// out, a difference with a zero first operand carries its sign into the next
// constant or into the choice of cadd_i / csub_i, and the remaining operations
// are those of the plain codelet in the same order, so a pruned codelet gives
// the plain codelet's result exactly.  Z = 0 is the plain codelet.  Input 0
// is never pruned (the first pass's butterflies all read a frequency near 0
// there).  The first pass of an inverse x or y transform uses them: x and y
// planes outside the sphere are zero for every butterfly.
template <bool ZA, bool ZB, typename V>
__host__ __device__ __forceinline__ V zadd(V a, V b) {
    if constexpr (ZB) return a;          // also a = b = 0
    else if constexpr (ZA) return b;
    else return cadd(a, b);
}

template <int R, int DIR, typename V, unsigned Z> struct DftZ {
    static_assert(Z == 0, "no pruned codelet for this radix");
    __host__ __device__ static __forceinline__ void run(V* v) { Dft<R, DIR, V>::run(v); }
};

template <int DIR, typename V, unsigned Z> struct DftZ<2, DIR, V, Z> {
    static_assert(!(Z & 1u), "input 0 of a pruned codelet is not zero");
    __host__ __device__ static __forceinline__ void run(V* v) {
        if constexpr (Z & 2u) v[1] = v[0];
        else Dft<2, DIR, V>::run(v);
    }
};

template <int DIR, typename V, unsigned Z> struct DftZ<3, DIR, V, Z> {
    static_assert(!(Z & 1u), "input 0 of a pruned codelet is not zero");
    __host__ __device__ static __forceinline__ void run(V* v) {
        using T = decltype(v[0].x);
        constexpr bool z1 = Z & 2u, z2 = Z & 4u;
        if constexpr (Z == 0) {
            Dft<3, DIR, V>::run(v);
        } else if constexpr (z1 && z2) {
            v[1] = v[0]; v[2] = v[0];
        } else {
            const T h = T(0.86602540378443864676);
            V t = zadd<z1, z2>(v[1], v[2]);
            V d;
            if constexpr (z1) d = cscale(v[2], -h);
            else d = cscale(v[1], h);
            V m = cfma(t, T(-0.5), v[0]);
            v[0] = cadd(v[0], t);
            v[1] = cadd_i<DIR>(m, d);
            v[2] = csub_i<DIR>(m, d);
        }
    }
};

template <int DIR, typename V, unsigned Z> struct DftZ<4, DIR, V, Z> {
    static_assert(!(Z & 1u), "input 0 of a pruned codelet is not zero");
    __host__ __device__ static __forceinline__ void run(V* v) {
        constexpr bool z1 = Z & 2u, z2 = Z & 4u, z3 = Z & 8u;
        if constexpr (Z == 0) {
            Dft<4, DIR, V>::run(v);
        } else {
            V t0, t1;
            if constexpr (z2) { t0 = v[0]; t1 = v[0]; }
            else { t0 = cadd(v[0], v[2]); t1 = csub(v[0], v[2]); }
            if constexpr (z1 && z3) {
                v[0] = t0; v[1] = t1; v[2] = t0; v[3] = t1;
            } else {
                V t2, o1, o3;
                if constexpr (z1) {            // d = -v3
                    t2 = v[3];
                    o1 = csub_i<DIR>(t1, v[3]); o3 = cadd_i<DIR>(t1, v[3]);
                } else if constexpr (z3) {     // d = v1
                    t2 = v[1];
                    o1 = cadd_i<DIR>(t1, v[1]); o3 = csub_i<DIR>(t1, v[1]);
                } else {
                    t2 = cadd(v[1], v[3]);
                    V d = csub(v[1], v[3]);
                    o1 = cadd_i<DIR>(t1, d); o3 = csub_i<DIR>(t1, d);
                }
                v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
                v[1] = o1; v[3] = o3;
            }
        }
    }
};

template <int DIR, typename V, unsigned Z> struct DftZ<5, DIR, V, Z> {
    static_assert(!(Z & 1u), "input 0 of a pruned codelet is not zero");
    __host__ __device__ static __forceinline__ void run(V* v) {
        if constexpr (Z == 0) {
            Dft<5, DIR, V>::run(v);
        } else {
            using T = decltype(v[0].x);
            const T c1 = T(0.30901699437494742410);   // cos(2 pi / 5)
            const T c2 = T(-0.80901699437494742410);  // cos(4 pi / 5)
            const T s1 = T(0.95105651629515357212);   // sin(2 pi / 5)
            const T s2 = T(0.58778525229247312917);   // sin(4 pi / 5)
            constexpr bool z1 = Z & 2u, z2 = Z & 4u, z3 = Z & 8u, z4 = Z & 16u;
            constexpr bool p1 = !(z1 && z4), p2 = !(z2 && z3);   // pair (1, 4), pair (2, 3) present
            // sums t and differences u = g * w of the pairs, g = -1 when the
            // pair's first member is zero (then w is the second member)
            constexpr T g1 = z1 ? T(-1) : T(1), g2 = z2 ? T(-1) : T(1);
            V t1 = zadd<z1, z4>(v[1], v[4]), t2 = zadd<z2, z3>(v[2], v[3]);
            V w1, w2;
            if constexpr (z1 || z4) w1 = t1; else w1 = csub(v[1], v[4]);
            if constexpr (z2 || z3) w2 = t2; else w2 = csub(v[2], v[3]);
            if constexpr (!p1 && !p2) {
                v[1] = v[0]; v[2] = v[0]; v[3] = v[0]; v[4] = v[0];
            } else {
                V a1, a2, b1, b2, s0;
                if constexpr (p1 && p2) {
                    a1 = cfma(t2, c2, cfma(t1, c1, v[0]));
                    a2 = cfma(t2, c1, cfma(t1, c2, v[0]));
                    b1 = cfma(w2, g2 * s2, cscale(w1, g1 * s1));
                    b2 = cfma(w2, -g2 * s1, cscale(w1, g1 * s2));
                    s0 = cadd(v[0], cadd(t1, t2));
                } else if constexpr (p1) {
                    a1 = cfma(t1, c1, v[0]);
                    a2 = cfma(t1, c2, v[0]);
                    b1 = cscale(w1, g1 * s1);
                    b2 = cscale(w1, g1 * s2);
                    s0 = cadd(v[0], t1);
                } else {
                    a1 = cfma(t2, c2, v[0]);
                    a2 = cfma(t2, c1, v[0]);
                    b1 = cscale(w2, g2 * s2);
                    b2 = cscale(w2, -g2 * s1);
                    s0 = cadd(v[0], t2);
                }
                v[0] = s0;
                v[1] = cadd_i<DIR>(a1, b1); v[4] = csub_i<DIR>(a1, b1);
                v[2] = cadd_i<DIR>(a2, b2); v[3] = csub_i<DIR>(a2, b2);
            }
        }
    }
};

template <int DIR, typename V, unsigned Z> struct DftZ<8, DIR, V, Z> {
    __host__ __device__ static __forceinline__ void run(V* v) {
        if constexpr (Z == 0) {
            Dft<8, DIR, V>::run(v);
        } else {
            // even inputs 0, 2, 4, 6 and odd inputs 1, 3, 5, 7
            constexpr unsigned ZE = (Z & 1u) | ((Z >> 1) & 2u) | ((Z >> 2) & 4u) | ((Z >> 3) & 8u);
            constexpr unsigned ZO = ((Z >> 1) & 1u) | ((Z >> 2) & 2u) | ((Z >> 3) & 4u) | ((Z >> 4) & 8u);
            V e[4] = {v[0], v[2], v[4], v[6]};
            V o[4] = {v[1], v[3], v[5], v[7]};
            DftZ<4, DIR, V, ZE>::run(e);
            DftZ<4, DIR, V, ZO>::run(o);
            Dft8Combine<DIR, V>::run(v, e, o);
        }
    }
};

// Composite A * B with known-zero inputs: each A-point DFT over n1 (inputs
// B n1 + n2) drops the zeros of its own group.  No group may be all zero.
template <int A, int B, int DIR, typename V, unsigned Z>
struct DftABZ {
    template <int N2>
    __host__ __device__ static constexpr unsigned group_mask() {
        unsigned m = 0;
        for (int n1 = 0; n1 < A; ++n1)
            if (Z & (1u << (B * n1 + N2))) m |= 1u << n1;
        return m;
    }
    __host__ __device__ static __forceinline__ void run(V* v) {
        constexpr int R = A * B;
        V y[B][A];
        sfor<B>([&](auto n2c) {
            constexpr int n2 = decltype(n2c)::value;
            constexpr unsigned G = group_mask<n2>();
            static_assert(G != (1u << A) - 1u, "a pruned composite codelet keeps every input group");
            V t[A];
            sfor<A>([&](auto n1c) { t[decltype(n1c)::value] = v[B * decltype(n1c)::value + n2]; });
            DftZ<A, DIR, V, G>::run(t);
            sfor<A>([&](auto k1c) {
                constexpr int k1 = decltype(k1c)::value;
                y[n2][k1] = twiddle_const<R, n2 * k1, DIR>(t[k1]);
            });
        });
        sfor<A>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            V t[B];
            sfor<B>([&](auto n2c) { t[decltype(n2c)::value] = y[decltype(n2c)::value][k1]; });
            Dft<B, DIR, V>::run(t);
            sfor<B>([&](auto k2c) { v[k1 + A * decltype(k2c)::value] = t[decltype(k2c)::value]; });
        });
    }
};

template <int DIR, typename V, unsigned Z> struct DftZ<6, DIR, V, Z> : DftABZ<3, 2, DIR, V, Z> {};
template <int DIR, typename V, unsigned Z> struct DftZ<9, DIR, V, Z> : DftABZ<3, 3, DIR, V, Z> {};
template <int DIR, typename V, unsigned Z> struct DftZ<10, DIR, V, Z> : DftABZ<5, 2, DIR, V, Z> {};
template <int DIR, typename V, unsigned Z> struct DftZ<12, DIR, V, Z> : DftABZ<4, 3, DIR, V, Z> {};
template <int DIR, typename V, unsigned Z> struct DftZ<15, DIR, V, Z> : DftABZ<5, 3, DIR, V, Z> {};
template <int DIR, typename V, unsigned Z> struct DftZ<16, DIR, V, Z> : DftABZ<4, 4, DIR, V, Z> {};

// ---------------------------------------------------------------- Stockham
// One pass of radix R with Ns = NS over all TL lines of a tile, in place.
// tw[t] = exp(-2 pi i t / N); the inverse (DIR = +1) uses its conjugate.
// Butterfly b of a line reads elements b + r N/R and writes
// (b / NS) NS R + (b mod NS) + r NS.
// Z: inputs known to be zero (pruned codelet; their twiddles are skipped).
template <typename V, int N, int R, int NS, int DIR, unsigned Z = 0>
__host__ __device__ __forceinline__ void twiddle_dft(V* v, const V* tw, int j) {
    const int k = j % NS;
    if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
            if ((Z >> r) & 1u) continue;
            const int t = r * k * (N / (NS * R));
            V w = tw[t];
            if (DIR > 0) w.y = -w.y;
            v[r] = cmul(v[r], w);
        }
    }
    DftZ<R, DIR, V, Z>::run(v);
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

// One pass with caller-supplied input and output: ld(line, e) returns
// element e of a line, st(line, e, v, q, r) receives output element e (q, r
// identify the register slot, the same for every call with the same tile
// shape).  SYNC waits between the reads and the writes (needed when both go
// to the same shared tile).
// Z: inputs of the pass's codelet known to be zero for every butterfly; they
// are neither loaded nor added.
template <typename V, int N, int P, int DIR, int TL, int NT, bool SYNC, unsigned Z = 0, class Ld, class St>
__device__ __forceinline__ void pass_io(const V* tw, Ld&& ld, St&& st) {
    constexpr int R = plan_radix(N, P);
    constexpr int NS = plan_ns(N, P);
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
            for (int r = 0; r < R; ++r) {
                if ((Z >> r) & 1u) {
                    v[q][r].x = 0;
                    v[q][r].y = 0;
                } else {
                    v[q][r] = ld(line, j + r * NBF);
                }
            }
        }
    }
    if constexpr (SYNC) __syncthreads();
#pragma unroll
    for (int q = 0; q < PER; ++q) {
        const int beta = tid + q * NT;
        if (beta < TOT) {
            const int line = beta % TL, j = beta / TL;
            twiddle_dft<V, N, R, NS, DIR, Z>(v[q], tw, j);
            const int base = (j / NS) * NS * R + (j % NS);
#pragma unroll
            for (int r = 0; r < R; ++r) st(line, base + r * NS, v[q][r], q, r);
        }
    }
}

template <typename V, int N, int DIR, int TL, int LS, int NT, int P, class Sl, class Ss>
__device__ __forceinline__ void middle_passes(V* buf, const V* tw, Sl& sl, Ss& ss) {
    if constexpr (P < plan_passes(N) - 1) {
        pass_io<V, N, P, DIR, TL, NT, true>(tw, sl, ss);
        __syncthreads();
        middle_passes<V, N, DIR, TL, LS, NT, P + 1>(buf, tw, sl, ss);
    }
}

// Full transform of TL lines whose first pass reads through ld and whose last
// pass writes through st; the passes in between use the shared tile buf.
// FIRST_SMEM: ld reads buf (the caller has synchronised).  LAST_SMEM: st
// writes buf (the caller synchronises before reading it).  Z0: inputs of the
// first pass's codelet that are zero for every butterfly (sphere_zero_mask).
template <typename V, int N, int DIR, int TL, int LS, int NT, bool FIRST_SMEM, bool LAST_SMEM, unsigned Z0 = 0,
          class Ld, class St>
__device__ __forceinline__ void fft_io(V* buf, const V* tw, Ld&& ld, St&& st) {
    static_assert(plan_ok(N), "unsupported transform length");
    constexpr int NP = plan_passes(N);
    auto sl = [&](int line, int e) { return buf[e * LS + line]; };
    auto ss = [&](int line, int e, V v, int, int) { buf[e * LS + line] = v; };
    if constexpr (NP == 1) {
        pass_io<V, N, 0, DIR, TL, NT, FIRST_SMEM || LAST_SMEM, Z0>(tw, ld, st);
    } else {
        pass_io<V, N, 0, DIR, TL, NT, FIRST_SMEM, Z0>(tw, ld, ss);
        __syncthreads();
        middle_passes<V, N, DIR, TL, LS, NT, 1>(buf, tw, sl, ss);
        pass_io<V, N, NP - 1, DIR, TL, NT, LAST_SMEM>(tw, sl, st);
    }
}

// Register slots of the last pass of an N-point transform over TL lines:
// slot (q, r) of thread tid holds output element e of line `line`.
template <int N, int TL, int NT>
struct LastPassSlots {
    static constexpr int P = plan_passes(N) - 1;
    static constexpr int R = plan_radix(N, P);
    static constexpr int NS = plan_ns(N, P);
    static constexpr int TOT = (N / R) * TL;
    static constexpr int PER = (TOT + NT - 1) / NT;
    __device__ static __forceinline__ bool point(int tid, int q, int r, int& line, int& e) {
        const int beta = tid + q * NT;
        if (beta >= TOT) return false;
        line = beta % TL;
        const int j = beta / TL;
        e = (j / NS) * NS * R + (j % NS) + r * NS;
        return true;
    }
};

// The same pass sequence on one line, on the host: tests/cpp/fft_passes.cu
// runs it for every compiled length against the DFT sum.
// Z0: the first pass's known-zero inputs (sphere_zero_mask), not read.
template <typename V, int N, int DIR, int P, unsigned Z0 = 0>
__host__ void host_passes(V* line, const V* tw) {
    if constexpr (P < plan_passes(N)) {
        constexpr int R = plan_radix(N, P);
        constexpr int NS = plan_ns(N, P);
        constexpr int NBF = N / R;
        constexpr unsigned Z = P == 0 ? Z0 : 0u;
        V out[N];
        for (int j = 0; j < NBF; ++j) {
            V v[R];
            for (int r = 0; r < R; ++r) {
                v[r].x = 0;
                v[r].y = 0;
                if (!((Z >> r) & 1u)) v[r] = line[j + r * NBF];
            }
            twiddle_dft<V, N, R, NS, DIR, Z>(v, tw, j);
            const int base = (j / NS) * NS * R + (j % NS);
            for (int r = 0; r < R; ++r) out[base + r * NS] = v[r];
        }
        for (int e = 0; e < N; ++e) line[e] = out[e];
        host_passes<V, N, DIR, P + 1, Z0>(line, tw);
    }
}

}  // namespace roks
