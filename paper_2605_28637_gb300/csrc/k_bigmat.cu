// k_bigmat.cu -- band-space matrices too large for one SM's shared memory
// (more than 64 bands): blocked right-looking Cholesky with the inverse of
// L, and the matrix exponential by Taylor + squaring on a tiled square GEMM.
// Element type U is float2 (mixed path) or double2 (FP64 path); the work is
// spread over many blocks because GB300's FP64 rate per SM is small.
#include <algorithm>
#include <cmath>

#include "roks_impl.cuh"

namespace roks {

constexpr int BK = 32;   // block size of the blocked algorithms

template <typename U> struct Real;
template <> struct Real<float2> { using type = float; };
template <> struct Real<double2> { using type = double; };

template <typename U>
__device__ __forceinline__ U ld_as(const double2 v) {
    U r;
    r.x = (typename Real<U>::type)v.x;
    r.y = (typename Real<U>::type)v.y;
    return r;
}

// A (n x n, column major, type U) <- O (double2), Hermitian part.
template <typename U>
__global__ void k_big_load(int n, const double2* __restrict__ O, U* __restrict__ A) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int i = idx % n, j = idx / n;
    const double2 a = O[idx], b = O[(int64_t)i * n + j];
    A[idx] = ld_as<U>(make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y)));
}

// Factor the diagonal block kb (one block): L_kk and D = L_kk^{-1} (BK x BK).
template <typename U>
__global__ void __launch_bounds__(256) k_big_diag(int n, int kb, U* __restrict__ A, U* __restrict__ Dinv, int* flag) {
    using R = typename Real<U>::type;
    __shared__ U L[BK][BK + 1];
    __shared__ U X[BK][BK + 1];
    __shared__ R piv_inv[BK];
    const int k0 = kb * BK;
    const int m = min(BK, n - k0);
    for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
        const int i = t % BK, j = t / BK;
        U v;
        v.x = 0; v.y = 0;
        if (i < m && j < m) v = A[(int64_t)(k0 + j) * n + k0 + i];
        L[j][i] = v;                 // L[col][row]
        U z; z.x = (i == j) ? R(1) : R(0); z.y = 0;
        X[j][i] = z;
    }
    __syncthreads();
    for (int j = 0; j < m; ++j) {
        if (threadIdx.x == 0) {
            R d = L[j][j].x;
            if (!(d > R(0))) {
                if (flag) atomicCAS(flag, 0, k0 + j + 1);
                d = R(1);
            }
            const R p = sqrt(d);
            L[j][j].x = p;
            L[j][j].y = 0;
            piv_inv[j] = R(1) / p;
        }
        __syncthreads();
        const R inv = piv_inv[j];
        for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) {
            L[j][i].x *= inv;
            L[j][i].y *= inv;
        }
        __syncthreads();
        const int r = m - j - 1;
        for (int t = threadIdx.x; t < r * r; t += blockDim.x) {
            const int i = j + 1 + t % r, k = j + 1 + t / r;
            if (k > i) continue;
            const U a = L[j][i], b = L[j][k];
            L[k][i].x -= a.x * b.x + a.y * b.y;
            L[k][i].y -= a.y * b.x - a.x * b.y;
        }
        __syncthreads();
    }
    // X = L^{-1}: column c by one thread (BK <= 32 columns)
    if (threadIdx.x < m) {
        const int c = threadIdx.x;
        for (int i = c; i < m; ++i) {
            R sr = (i == c) ? R(1) : R(0), si = 0;
            for (int k = c; k < i; ++k) {
                const U l = L[k][i], x = X[c][k];
                sr -= l.x * x.x - l.y * x.y;
                si -= l.x * x.y + l.y * x.x;
            }
            X[c][i].x = sr * piv_inv[i];
            X[c][i].y = si * piv_inv[i];
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
        const int i = t % BK, j = t / BK;
        if (i < m && j < m) A[(int64_t)(k0 + j) * n + k0 + i] = L[j][i];
        U z; z.x = 0; z.y = 0;
        Dinv[(int64_t)kb * BK * BK + j * BK + i] = (i < m && j < m) ? X[j][i] : z;
    }
}

// Panel: L_ik = A_ik D^H for the row blocks i > kb (one block per row block).
template <typename U>
__global__ void __launch_bounds__(256) k_big_panel(int n, int kb, U* __restrict__ A, const U* __restrict__ Dinv) {
    using R = typename Real<U>::type;
    __shared__ U S[BK][BK + 1];
    __shared__ U Dm[BK][BK + 1];
    const int k0 = kb * BK;
    const int i0 = (kb + 1 + blockIdx.x) * BK;
    const int rows = min(BK, n - i0), cols = min(BK, n - k0);
    for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
        const int r = t % BK, c = t / BK;
        U v; v.x = 0; v.y = 0;
        if (r < rows && c < cols) v = A[(int64_t)(k0 + c) * n + i0 + r];
        S[c][r] = v;
        Dm[c][r] = Dinv[(int64_t)kb * BK * BK + c * BK + r];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
        const int r = t % BK, c = t / BK;
        if (r >= rows || c >= cols) continue;
        // (A D^H)_rc = sum_m A_rm conj(D_cm), D lower: m <= c
        R sr = 0, si = 0;
        for (int mm = 0; mm <= c; ++mm) {
            const U a = S[mm][r], d = Dm[mm][c];
            sr += a.x * d.x + a.y * d.y;
            si += a.y * d.x - a.x * d.y;
        }
        U o; o.x = sr; o.y = si;
        A[(int64_t)(k0 + c) * n + i0 + r] = o;
    }
}

// Trailing update: A_ij -= L_ik L_jk^H for block pairs kb < jb <= ib.
template <typename U>
__global__ void __launch_bounds__(256) k_big_update(int n, int kb, U* __restrict__ A) {
    using R = typename Real<U>::type;
    __shared__ U Li[BK][BK + 1];
    __shared__ U Lj[BK][BK + 1];
    // blockIdx.x enumerates the lower-triangle block pairs of the trailing matrix
    int t = blockIdx.x, ib = 0;
    while ((ib + 1) * (ib + 2) / 2 <= t) ++ib;
    const int jb = t - ib * (ib + 1) / 2;
    const int k0 = kb * BK;
    const int i0 = (kb + 1 + ib) * BK, j0 = (kb + 1 + jb) * BK;
    const int ri = min(BK, n - i0), rj = min(BK, n - j0), cc = min(BK, n - k0);
    for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
        const int r = q % BK, c = q / BK;
        U z; z.x = 0; z.y = 0;
        Li[c][r] = (r < ri && c < cc) ? A[(int64_t)(k0 + c) * n + i0 + r] : z;
        Lj[c][r] = (r < rj && c < cc) ? A[(int64_t)(k0 + c) * n + j0 + r] : z;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
        const int r = q % BK, c = q / BK;
        if (r >= ri || c >= rj) continue;
        if (ib == jb && c > r) continue;
        R sr = 0, si = 0;
        for (int mm = 0; mm < cc; ++mm) {
            const U a = Li[mm][r], b = Lj[mm][c];
            sr += a.x * b.x + a.y * b.y;
            si += a.y * b.x - a.x * b.y;
        }
        U* dst = A + (int64_t)(j0 + c) * n + i0 + r;
        U o = *dst;
        o.x -= sr;
        o.y -= si;
        *dst = o;
    }
}

// Inverse, block row ib: X_ij = -D_i sum_{m=j}^{i-1} L_im X_mj for jb < ib
// (X_ii = D_i); X lives in the upper... separate buffer Xm (n x n).
template <typename U>
__global__ void __launch_bounds__(256) k_big_inv_row(int n, int ib, const U* __restrict__ A,
                                                     const U* __restrict__ Dinv, U* __restrict__ Xm) {
    using R = typename Real<U>::type;
    __shared__ U Sacc[BK][BK + 1];
    __shared__ U Lt[BK][BK + 1];
    __shared__ U Xt[BK][BK + 1];
    const int jb = blockIdx.x;          // 0 .. ib
    const int i0 = ib * BK, j0 = jb * BK;
    const int ri = min(BK, n - i0), cj = min(BK, n - j0);
    if (jb == ib) {
        for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
            const int r = q % BK, c = q / BK;
            if (r < ri && c < cj) Xm[(int64_t)(j0 + c) * n + i0 + r] = Dinv[(int64_t)ib * BK * BK + c * BK + r];
        }
        return;
    }
    R accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};
    for (int mb = jb; mb < ib; ++mb) {
        const int m0 = mb * BK, cm = min(BK, n - m0);
        for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
            const int r = q % BK, c = q / BK;
            U z; z.x = 0; z.y = 0;
            Lt[c][r] = (r < ri && c < cm) ? A[(int64_t)(m0 + c) * n + i0 + r] : z;        // L_im (r, c)
            Xt[c][r] = (r < cm && c < cj) ? Xm[(int64_t)(j0 + c) * n + m0 + r] : z;       // X_mj (r, c)
        }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const int q = threadIdx.x + s * 256;
            const int r = q % BK, c = q / BK;
            for (int mm = 0; mm < BK; ++mm) {
                const U a = Lt[mm][r], b = Xt[c][mm];
                accr[s] += a.x * b.x - a.y * b.y;
                acci[s] += a.x * b.y + a.y * b.x;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int q = threadIdx.x + s * 256;
        const int r = q % BK, c = q / BK;
        U v; v.x = accr[s]; v.y = acci[s];
        Sacc[c][r] = v;
    }
    __syncthreads();
    const U* D = Dinv + (int64_t)ib * BK * BK;
    for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
        const int r = q % BK, c = q / BK;
        if (r >= ri || c >= cj) continue;
        R sr = 0, si = 0;
        for (int mm = 0; mm <= r; ++mm) {
            const U d = D[mm * BK + r], b = Sacc[c][mm];
            sr += d.x * b.x - d.y * b.y;
            si += d.x * b.y + d.y * b.x;
        }
        U o; o.x = -sr; o.y = -si;
        Xm[(int64_t)(j0 + c) * n + i0 + r] = o;
    }
}

// LinvH (double2) = X^H, with X lower triangular (upper part written as zero).
template <typename U>
__global__ void k_big_store_inverse(int n, const U* __restrict__ Xm, double2* __restrict__ LinvH) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int c = idx % n, i = idx / n;     // LinvH(row c, col i) = conj X(i, c)
    if (i < c) {
        LinvH[idx] = make_double2(0.0, 0.0);
        return;
    }
    const U x = Xm[(int64_t)c * n + i];
    LinvH[idx] = make_double2((double)x.x, -(double)x.y);
}

template <typename U>
void cholesky_big_impl(int n, const double2* O, U* A, U* Dinv, U* Xm, double2* LinvH, int* flag, cudaStream_t st) {
    const int nbk = (n + BK - 1) / BK;
    const int blocks = (n * n + 255) / 256;
    roks::count_launch(), k_big_load<U><<<blocks, 256, 0, st>>>(n, O, A);
    for (int kb = 0; kb < nbk; ++kb) {
        roks::count_launch(), k_big_diag<U><<<1, 256, 0, st>>>(n, kb, A, Dinv, flag);
        const int nt = nbk - kb - 1;
        if (nt > 0) {
            roks::count_launch(), k_big_panel<U><<<nt, 256, 0, st>>>(n, kb, A, Dinv);
            roks::count_launch(), k_big_update<U><<<nt * (nt + 1) / 2, 256, 0, st>>>(n, kb, A);
        }
    }
    for (int ib = 0; ib < nbk; ++ib) roks::count_launch(), k_big_inv_row<U><<<ib + 1, 256, 0, st>>>(n, ib, A, Dinv, Xm);
    roks::count_launch(), k_big_store_inverse<U><<<blocks, 256, 0, st>>>(n, Xm, LinvH);
}

size_t cholesky_big_work_bytes(int n, bool fp64) {
    const size_t e = fp64 ? sizeof(double2) : sizeof(float2);
    const int nbk = (n + BK - 1) / BK;
    return e * ((size_t)2 * n * n + (size_t)nbk * BK * BK) + 256;
}

void cholesky_inverse_big(int n, const double2* O, void* work, bool fp64, double2* LinvH, int* flag,
                          cudaStream_t st) {
    const int nbk = (n + BK - 1) / BK;
    if (fp64) {
        double2* A = static_cast<double2*>(work);
        double2* Xm = A + (size_t)n * n;
        double2* D = Xm + (size_t)n * n;
        cholesky_big_impl<double2>(n, O, A, D, Xm, LinvH, flag, st);
    } else {
        float2* A = static_cast<float2*>(work);
        float2* Xm = A + (size_t)n * n;
        float2* D = Xm + (size_t)n * n;
        cholesky_big_impl<float2>(n, O, A, D, Xm, LinvH, flag, st);
    }
    (void)nbk;
}

// ------------------------------------------------------------------ matrix exponential, large n
// C = alpha A B (+ I when add_identity), n x n, 32 x 32 output tiles per
// block of 256 threads, thread (tx, ty) owning rows ty + 16 i and columns
// tx + 16 j (i, j < 2), K in slices of 16 staged in shared memory (two
// shared-memory loads per complex multiply-add pair of the tile).  With
// guard, launches past the device's squaring count copy A through.
constexpr int SQ_K = 16;

template <typename U>
__global__ void __launch_bounds__(256) k_sq_gemm(int n, const U* __restrict__ A, const U* __restrict__ B,
                                                 U* __restrict__ C, typename Real<U>::type alpha, int add_identity,
                                                 const double* __restrict__ guard, int step) {
    using R = typename Real<U>::type;
    __shared__ U As[SQ_K][BK + 1];
    __shared__ U Bs[SQ_K][BK + 1];
    const int i0 = blockIdx.x * BK, j0 = blockIdx.y * BK;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (guard && step >= int(guard[0])) {
        // squaring beyond q: copy through
        for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
            const int r = q % BK, c = q / BK;
            if (i0 + r < n && j0 + c < n) C[(int64_t)(j0 + c) * n + i0 + r] = A[(int64_t)(j0 + c) * n + i0 + r];
        }
        return;
    }
    R ar[2][2], ai[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) ar[a][b] = ai[a][b] = R(0);
    for (int k0 = 0; k0 < n; k0 += SQ_K) {
        for (int q = threadIdx.x; q < BK * SQ_K; q += blockDim.x) {
            // A(i0 + r, k0 + c): rows contiguous; B(k0 + c, j0 + r): K contiguous
            const int r = q % BK, c = q / BK;
            U z;
            z.x = 0;
            z.y = 0;
            As[c][r] = (i0 + r < n && k0 + c < n) ? A[(int64_t)(k0 + c) * n + i0 + r] : z;
            const int kr = q % SQ_K, jc = q / SQ_K;
            Bs[kr][jc] = (k0 + kr < n && j0 + jc < n) ? B[(int64_t)(j0 + jc) * n + k0 + kr] : z;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SQ_K; ++kk) {
            const U a0 = As[kk][ty], a1 = As[kk][ty + 16];
            const U b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            const U av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    ar[a][b] += av[a].x * bv[b].x - av[a].y * bv[b].y;
                    ai[a][b] += av[a].x * bv[b].y + av[a].y * bv[b].x;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int r = ty + 16 * a, c = tx + 16 * b;
            if (i0 + r < n && j0 + c < n) {
                U o;
                o.x = alpha * ar[a][b] + ((add_identity && i0 + r == j0 + c) ? R(1) : R(0));
                o.y = alpha * ai[a][b];
                C[(int64_t)(j0 + c) * n + i0 + r] = o;
            }
        }
}

// Column sums sum_r (|Re a| + |Im a|) of A (a bound of the 1-norm with
// fewer FP64 operations than the moduli): one warp per column.
__global__ void k_big_colsum(int n, const double2* __restrict__ A, double* __restrict__ colsum) {
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (c >= n) return;
    double sum = 0.0;
    for (int r = lane; r < n; r += 32) {
        const double2 a = A[(int64_t)c * n + r];
        sum += fabs(a.x) + fabs(a.y);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) colsum[c] = sum;
}

// X = s A / 2^q with ||s A||_1 / 2^q <= 1/4 (q on the device in info[0]);
// P = I + X / degree.  Every block finds the largest column sum itself
// (n values) and fills its share of the elements.
template <typename U>
__global__ void k_big_expm_scale(int n, const double2* __restrict__ A, const double* __restrict__ s,
                                 const double* __restrict__ colsum, U* __restrict__ X, U* __restrict__ P,
                                 double* __restrict__ info, int degree) {
    __shared__ double red[256];
    __shared__ double fsh;
    double best = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) best = fmax(best, colsum[c]);
    red[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double scaled = fabs(s[0]) * red[0];
        int q = 0;
        while (scaled > 0.25 && q < 40) {
            scaled *= 0.5;
            ++q;
        }
        if (blockIdx.x == 0) info[0] = double(q);
        fsh = s[0] * ldexp(1.0, -q);
    }
    __syncthreads();
    const double f = fsh, fd = fsh / degree;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
        const double2 a = A[idx];
        X[idx] = ld_as<U>(make_double2(f * a.x, f * a.y));
        const int m = idx % n, c = idx / n;
        P[idx] = ld_as<U>(make_double2((m == c ? 1.0 : 0.0) + fd * a.x, fd * a.y));
    }
}

template <typename U>
__global__ void k_big_to_double(int n, const U* __restrict__ P, double2* __restrict__ E) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < n * n) E[idx] = make_double2((double)P[idx].x, (double)P[idx].y);
}

template <typename U>
void expm_big_impl(int n, const double2* A, const double* s, double2* E, U* X, U* P, U* Q, double* info, int degree,
                   int max_square, cudaStream_t st) {
    using R = typename Real<U>::type;
    // the column sums go to E's storage (n doubles), overwritten at the end
    double* colsum = reinterpret_cast<double*>(E);
    roks::count_launch(), k_big_colsum<<<(unsigned)((32 * n + 255) / 256), 256, 0, st>>>(n, A, colsum);
    const int fill_blocks = std::min(152, (n * n + 255) / 256);
    roks::count_launch(), k_big_expm_scale<U><<<fill_blocks, 256, 0, st>>>(n, A, s, colsum, X, P, info, degree);
    const int nt = (n + BK - 1) / BK;
    dim3 g(nt, nt);
    for (int k = degree - 1; k >= 1; --k) {
        roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, X, P, Q, R(1) / R(k), 1, nullptr, 0);
        U* t = P; P = Q; Q = t;
    }
    for (int r = 0; r < max_square; ++r) {
        roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, P, P, Q, R(1), 0, info, r);
        U* t = P; P = Q; Q = t;
    }
    roks::count_launch(), k_big_to_double<U><<<(n * n + 255) / 256, 256, 0, st>>>(n, P, E);
}

size_t expm_big_work_bytes(int n, bool fp64) { return (fp64 ? sizeof(double2) : sizeof(float2)) * 3 * (size_t)n * n; }

void expm_big(int n, const double2* A, const double* scale_dev, double2* E, void* work, double* info, bool fp64,
              cudaStream_t st) {
    // FP64: degree 16 (||X|| <= 1/4 gives 1e-26); FP32: degree 8 (1e-11);
    // at most 24 squarings (the launches past the device's q copy through).
    if (fp64) {
        double2* X = static_cast<double2*>(work);
        expm_big_impl<double2>(n, A, scale_dev, E, X, X + (size_t)n * n, X + 2 * (size_t)n * n, info, 16, 24, st);
    } else {
        float2* X = static_cast<float2*>(work);
        expm_big_impl<float2>(n, A, scale_dev, E, X, X + (size_t)n * n, X + 2 * (size_t)n * n, info, 8, 24, st);
    }
}

}  // namespace roks
