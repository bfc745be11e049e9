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

// Factor the diagonal block kb (one block of 256 threads): L_kk, and
// D = L_kk^{-1} by a column sweep in the same loop (solve L D = I for all
// right-hand sides at once: row j of D is scaled by 1/L_jj as soon as
// column j of L is final, then subtracted from the rows below).
// Thread (lane i, warp w) keeps the elements (row i, column w + 8 q), q < 4,
// of L and of D in registers.  Step j: the warp owning column j forms the
// pivot (a shuffle from lane j), scales the column and publishes it with
// 1/L_jj; after one barrier every thread updates its own elements, and the
// lane owning row j + 1 of D publishes that row for the next step.  The
// published column and row are double-buffered by the parity of j, so one
// barrier per step suffices.  D goes to Dinv and to X = L^{-1} (block kb, kb).
template <typename U>
__global__ void __launch_bounds__(256) k_big_diag(int n, int kb, U* __restrict__ A, U* __restrict__ Dinv,
                                                  U* __restrict__ Xm, int* flag) {
    using R = typename Real<U>::type;
    __shared__ U colbuf[2][BK];    // column j of L (scaled), by row
    __shared__ U xrow[2][BK];      // row j of D before its scaling, by column
    __shared__ R invbuf[2];
    const int k0 = kb * BK;
    const int m = min(BK, n - k0);
    const int i = threadIdx.x & 31, w = threadIdx.x >> 5;
    U Lr[4], Xr[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = w + 8 * q;
        U v;
        v.x = 0;
        v.y = 0;
        if (i < m && k < m) v = A[(int64_t)(k0 + k) * n + k0 + i];
        Lr[q] = v;
        Xr[q].x = (i == k) ? R(1) : R(0);
        Xr[q].y = 0;
    }
    // row 0 of D (D[0][0] = 1 before scaling) for step 0
    if (w == 0 && i == 0) xrow[0][0] = Xr[0];
    for (int j = 0; j < m; ++j) {
        const int b = j & 1;
        const int wj = j & 7, qj = j >> 3;
        if (w == wj) {
            // this warp owns column j: pivot from lane j
            U lj = Lr[0];
#pragma unroll
            for (int q = 1; q < 4; ++q)
                if (q == qj) lj = Lr[q];
            R d = __shfl_sync(0xffffffffu, lj.x, j);
            if (!(d > R(0))) {
                if (i == 0 && flag) atomicCAS(flag, 0, k0 + j + 1);
                d = R(1);
            }
            const R p = sqrt(d);
            const R inv = R(1) / p;
            if (i > j) {
                lj.x *= inv;
                lj.y *= inv;
            } else if (i == j) {
                lj.x = p;
                lj.y = 0;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q == qj) Lr[q] = lj;
            colbuf[b][i] = lj;
            if (i == 0) invbuf[b] = inv;
        }
        __syncthreads();
        const R inv = invbuf[b];
        const U a = colbuf[b][i];   // L(i, j)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = w + 8 * q;
            if (k > j && i >= k) {
                // trailing L(i, k) -= L(i, j) conj(L(k, j))
                const U c = colbuf[b][k];
                Lr[q].x -= a.x * c.x + a.y * c.y;
                Lr[q].y -= a.y * c.x - a.x * c.y;
            } else if (k <= j) {
                if (i == j) {
                    // row j of D, final: scaled by 1 / L_jj
                    Xr[q].x *= inv;
                    Xr[q].y *= inv;
                } else if (i > j) {
                    // D(i, k) -= L(i, j) D(j, k), D(j, k) = xrow * inv
                    const U xv = xrow[b][k];
                    const R xr = xv.x * inv, xi = xv.y * inv;
                    Xr[q].x -= a.x * xr - a.y * xi;
                    Xr[q].y -= a.x * xi + a.y * xr;
                }
            }
        }
        // row j + 1 of D (columns k <= j + 1) for the next step
        if (i == j + 1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int k = w + 8 * q;
                if (k <= j + 1) xrow[b ^ 1][k] = Xr[q];
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int k = w + 8 * q;
        if (i < m && k < m) {
            A[(int64_t)(k0 + k) * n + k0 + i] = Lr[q];
            Xm[(int64_t)(k0 + k) * n + k0 + i] = Xr[q];
        }
        U z;
        z.x = 0;
        z.y = 0;
        Dinv[(int64_t)kb * BK * BK + k * BK + i] = (i < m && k < m) ? Xr[q] : z;
    }
}

// Blocks 0 .. nt-1, panel: L_ik = A_ik D^H for the row blocks i > kb.
// Blocks nt .. nt+kb-1, row kb of X = L^{-1}: X_kj = D_kb W_kj for j < kb,
// in place (W_kj, accumulated in Xm by the updates of the earlier steps,
// holds -sum_{m<kb} L_km X_mj).
template <typename U>
__global__ void __launch_bounds__(256) k_big_panel(int n, int kb, int nt, U* __restrict__ A,
                                                   const U* __restrict__ Dinv, U* __restrict__ Xm) {
    using R = typename Real<U>::type;
    __shared__ U S[BK][BK + 1];
    __shared__ U Dm[BK][BK + 1];
    const int k0 = kb * BK;
    for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
        const int r = t % BK, c = t / BK;
        Dm[c][r] = Dinv[(int64_t)kb * BK * BK + c * BK + r];
    }
    if ((int)blockIdx.x < nt) {
        const int i0 = (kb + 1 + blockIdx.x) * BK;
        const int rows = min(BK, n - i0), cols = min(BK, n - k0);
        for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
            const int r = t % BK, c = t / BK;
            U v; v.x = 0; v.y = 0;
            if (r < rows && c < cols) v = A[(int64_t)(k0 + c) * n + i0 + r];
            S[c][r] = v;
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
    } else {
        const int j0 = (blockIdx.x - nt) * BK;
        const int rows = min(BK, n - k0);   // j0 + BK <= k0: full columns
        for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
            const int r = t % BK, c = t / BK;
            U v; v.x = 0; v.y = 0;
            if (r < rows) v = Xm[(int64_t)(j0 + c) * n + k0 + r];
            S[c][r] = v;
        }
        __syncthreads();
        for (int t = threadIdx.x; t < BK * BK; t += blockDim.x) {
            const int r = t % BK, c = t / BK;
            if (r >= rows) continue;
            // (D W)_rc = sum_{m <= r} D_rm W_mc
            R sr = 0, si = 0;
            for (int mm = 0; mm <= r; ++mm) {
                const U d = Dm[mm][r], w = S[c][mm];
                sr += d.x * w.x - d.y * w.y;
                si += d.x * w.y + d.y * w.x;
            }
            U o; o.x = sr; o.y = si;
            Xm[(int64_t)(j0 + c) * n + k0 + r] = o;
        }
    }
}

// Blocks 0 .. ntri-1, trailing update: A_ij -= L_ik L_jk^H for the block
// pairs kb < jb <= ib.  Blocks ntri .. ntri + nt (kb+1) - 1, the inverse's
// right-looking update: W_ij -= L_ik X_kj for the row blocks i > kb and the
// column blocks j <= kb (X_kj final after the panel of this step).
template <typename U>
__global__ void __launch_bounds__(256) k_big_update(int n, int kb, int nt, U* __restrict__ A, U* __restrict__ Xm) {
    using R = typename Real<U>::type;
    __shared__ U Li[BK][BK + 1];
    __shared__ U Lj[BK][BK + 1];
    const int ntri = nt * (nt + 1) / 2;
    const int k0 = kb * BK;
    const int cc = min(BK, n - k0);
    if ((int)blockIdx.x < ntri) {
        // blockIdx.x enumerates the lower-triangle block pairs of the trailing matrix
        int t = blockIdx.x, ib = 0;
        while ((ib + 1) * (ib + 2) / 2 <= t) ++ib;
        const int jb = t - ib * (ib + 1) / 2;
        const int i0 = (kb + 1 + ib) * BK, j0 = (kb + 1 + jb) * BK;
        const int ri = min(BK, n - i0), rj = min(BK, n - j0);
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
    } else {
        const int q0 = blockIdx.x - ntri;
        const int i0 = (kb + 1 + q0 % nt) * BK, j0 = (q0 / nt) * BK;
        const int ri = min(BK, n - i0);
        // Li: L_ik (r, m); Lj: X_kj stored as [col][row] = X(m, c)
        for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
            const int r = q % BK, c = q / BK;
            U z; z.x = 0; z.y = 0;
            Li[c][r] = (r < ri && c < cc) ? A[(int64_t)(k0 + c) * n + i0 + r] : z;
            Lj[c][r] = (r < cc) ? Xm[(int64_t)(j0 + c) * n + k0 + r] : z;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < BK * BK; q += blockDim.x) {
            const int r = q % BK, c = q / BK;
            if (r >= ri) continue;
            R sr = 0, si = 0;
            for (int mm = 0; mm < cc; ++mm) {
                const U a = Li[mm][r], x = Lj[c][mm];
                sr += a.x * x.x - a.y * x.y;
                si += a.x * x.y + a.y * x.x;
            }
            U* dst = Xm + (int64_t)(j0 + c) * n + i0 + r;
            U o = *dst;
            o.x -= sr;
            o.y -= si;
            *dst = o;
        }
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

// Right-looking blocked Cholesky with the inverse X = L^{-1} formed along
// the way: step kb factors the diagonal block (and its inverse D_kb), forms
// the panel below it and row kb of X (X_kj = D_kb W_kj), then updates the
// trailing matrix and the accumulated rows W_ij -= L_ik X_kj of X below.
// Three launches per block step, each spread over the blocks it touches.
template <typename U>
void cholesky_big_impl(int n, const double2* O, U* A, U* Dinv, U* Xm, double2* LinvH, int* flag, cudaStream_t st) {
    const int nbk = (n + BK - 1) / BK;
    const int blocks = (n * n + 255) / 256;
    cudaMemsetAsync(Xm, 0, sizeof(U) * (size_t)n * n, st);
    roks::count_launch(), k_big_load<U><<<blocks, 256, 0, st>>>(n, O, A);
    for (int kb = 0; kb < nbk; ++kb) {
        roks::count_launch(), k_big_diag<U><<<1, 256, 0, st>>>(n, kb, A, Dinv, Xm, flag);
        const int nt = nbk - kb - 1;
        if (nt + kb > 0) roks::count_launch(), k_big_panel<U><<<nt + kb, 256, 0, st>>>(n, kb, nt, A, Dinv, Xm);
        if (nt > 0)
            roks::count_launch(), k_big_update<U><<<nt * (nt + 1) / 2 + nt * (kb + 1), 256, 0, st>>>(n, kb, nt, A, Xm);
    }
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
// C = alpha A B (+ D when D is given) (+ I when add_identity), n x n.  A
// block owns a 16 x 16 output tile and splits K over four groups of 64
// threads (contiguous K ranges, 16-deep slices staged in shared memory);
// each thread keeps a 2 x 2 complex tile, and the four partial tiles are
// added in group order at the end (deterministic).  At n = 430 this is 729
// blocks, enough to keep every SM busy, where 32 x 32 tiles over all of K
// gave 196 blocks with one slice in flight each.  With guard, launches past
// the device's squaring count (guard[0]) return at once: the result then
// stays in the buffer the last real squaring wrote (k_big_to_double picks it).
constexpr int SQ_T = 16;   // output tile
constexpr int SQ_K = 16;   // K slice
constexpr int SQ_G = 4;    // K groups per block

template <typename U>
__global__ void __launch_bounds__(256) k_sq_gemm(int n, const U* __restrict__ A, const U* __restrict__ B,
                                                 U* __restrict__ C, typename Real<U>::type alpha,
                                                 const U* __restrict__ D, int add_identity,
                                                 const double* __restrict__ guard, int step) {
    using R = typename Real<U>::type;
    __shared__ U As[SQ_G][SQ_K][SQ_T + 1];
    __shared__ U Bs[SQ_G][SQ_K][SQ_T + 1];
    if (guard && step >= int(guard[0])) return;
    const int i0 = blockIdx.x * SQ_T, j0 = blockIdx.y * SQ_T;
    const int g = threadIdx.x >> 6, t = threadIdx.x & 63;
    const int tx = t & 7, ty = t >> 3;
    // K range of group g: [kb, ke), the same slice count for every group
    const int kr = ((n + SQ_G - 1) / SQ_G + SQ_K - 1) / SQ_K * SQ_K;
    const int kb = g * kr, ke = min(n, kb + kr);
    R ar[2][2], ai[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) ar[a][b] = ai[a][b] = R(0);
    for (int k0 = 0; k0 < kr; k0 += SQ_K) {
#pragma unroll
        for (int q = t; q < SQ_T * SQ_K; q += 64) {
            // A(i0 + r, kb + k0 + c): rows contiguous; B(kb + k0 + kk, j0 + c): K contiguous
            const int r = q % SQ_T, c = q / SQ_T;
            const int ka = kb + k0 + c;
            U z;
            z.x = 0;
            z.y = 0;
            As[g][c][r] = (i0 + r < n && ka < ke) ? A[(int64_t)ka * n + i0 + r] : z;
            const int kk = q % SQ_K, jc = q / SQ_K;
            const int kbb = kb + k0 + kk;
            Bs[g][kk][jc] = (kbb < ke && j0 + jc < n) ? B[(int64_t)(j0 + jc) * n + kbb] : z;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < SQ_K; ++kk) {
            const U av[2] = {As[g][kk][ty], As[g][kk][ty + 8]};
            const U bv[2] = {Bs[g][kk][tx], Bs[g][kk][tx + 8]};
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
    // partial tiles of the groups, added in group order by group 0
    U* part = &As[0][0][0];   // SQ_G x SQ_T x SQ_T fits in As (SQ_K >= SQ_T)
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            U v;
            v.x = ar[a][b];
            v.y = ai[a][b];
            part[(g * SQ_T + ty + 8 * a) * SQ_T + tx + 8 * b] = v;
        }
    __syncthreads();
    if (g != 0) return;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int r = ty + 8 * a, c = tx + 8 * b;
            if (i0 + r >= n || j0 + c >= n) continue;
            R sr = 0, si = 0;
            for (int gg = 0; gg < SQ_G; ++gg) {
                const U v = part[(gg * SQ_T + r) * SQ_T + c];
                sr += v.x;
                si += v.y;
            }
            const int64_t idx = (int64_t)(j0 + c) * n + i0 + r;
            U o;
            o.x = alpha * sr + ((add_identity && i0 + r == j0 + c) ? R(1) : R(0));
            o.y = alpha * si;
            if (D) {
                o.x += D[idx].x;
                o.y += D[idx].y;
            }
            C[idx] = o;
        }
}

// Paterson-Stockmeyer blocks of the Taylor polynomial: B = c0 I + c1 X +
// c2 X^2 + c3 X^3 + c4 X^4 (elementwise over the four powers).
template <typename U>
__global__ void k_big_ps_block(int n, const U* __restrict__ X1, const U* __restrict__ X2, const U* __restrict__ X3,
                               const U* __restrict__ X4, typename Real<U>::type c0, typename Real<U>::type c1,
                               typename Real<U>::type c2, typename Real<U>::type c3, typename Real<U>::type c4,
                               U* __restrict__ Bo) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int r = idx % n, c = idx / n;
    U o;
    o.x = c1 * X1[idx].x + c2 * X2[idx].x + c3 * X3[idx].x + c4 * X4[idx].x + (r == c ? c0 : 0);
    o.y = c1 * X1[idx].y + c2 * X2[idx].y + c3 * X3[idx].y + c4 * X4[idx].y;
    Bo[idx] = o;
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

// X = s A / 2^q with ||s A||_1 / 2^q <= 1/4 (q on the device in info[0]).
// Every block finds the largest column sum itself (n values) and fills its
// share of the elements.
template <typename U>
__global__ void k_big_expm_scale(int n, const double2* __restrict__ A, const double* __restrict__ s,
                                 const double* __restrict__ colsum, U* __restrict__ X, double* __restrict__ info) {
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
    const double f = fsh;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < n * n; idx += gridDim.x * blockDim.x) {
        const double2 a = A[idx];
        X[idx] = ld_as<U>(make_double2(f * a.x, f * a.y));
    }
}

// E = the squared polynomial: buffer P0 after an even number of squarings
// (min(q, max_square), q = info[0]), P1 after an odd one.
template <typename U>
__global__ void k_big_to_double(int n, const U* __restrict__ P0, const U* __restrict__ P1,
                                const double* __restrict__ info, int max_square, double2* __restrict__ E) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int q = min(int(info[0]), max_square);
    const U v = (q & 1) ? P1[idx] : P0[idx];
    E[idx] = make_double2((double)v.x, (double)v.y);
}

// exp(s A) = (p(X))^(2^q), X = s A / 2^q, p the Taylor polynomial of degree
// 4 r (FP32: r = 2, degree 8; FP64: r = 4, degree 16) evaluated by
// Paterson-Stockmeyer: X^2, X^3, X^4 (three products), blocks B_j =
// sum_{i<4} c_{4j+i} X^i (the last one with c_{4r} X^4), then
// p = B_0 + X^4 (B_1 + X^4 (B_2 + ...)) (r - 1 products), instead of the
// 4 r - 1 products of Horner's rule.  Work: seven n x n buffers.
template <typename U>
void expm_big_impl(int n, const double2* A, const double* s, double2* E, U* W, double* info, int r, int max_square,
                   cudaStream_t st) {
    using R = typename Real<U>::type;
    const size_t nn = (size_t)n * n;
    U* X1 = W;
    U* X2 = W + nn;
    U* X3 = W + 2 * nn;
    U* X4 = W + 3 * nn;
    U* Bj = W + 4 * nn;
    U* P = W + 5 * nn;
    U* Q = W + 6 * nn;
    // the column sums go to E's storage (n doubles), overwritten at the end
    double* colsum = reinterpret_cast<double*>(E);
    roks::count_launch(), k_big_colsum<<<(unsigned)((32 * n + 255) / 256), 256, 0, st>>>(n, A, colsum);
    const int fill_blocks = std::min(152, (n * n + 255) / 256);
    roks::count_launch(), k_big_expm_scale<U><<<fill_blocks, 256, 0, st>>>(n, A, s, colsum, X1, info);
    const int nt = (n + SQ_T - 1) / SQ_T;
    dim3 g(nt, nt);
    const int eb = (n * n + 255) / 256;
    roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, X1, X1, X2, R(1), nullptr, 0, nullptr, 0);
    roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, X2, X1, X3, R(1), nullptr, 0, nullptr, 0);
    roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, X2, X2, X4, R(1), nullptr, 0, nullptr, 0);
    // Taylor coefficients 1/k!
    double cf[17];
    cf[0] = 1.0;
    for (int k = 1; k <= 16; ++k) cf[k] = cf[k - 1] / k;
    const int d = 4 * r;
    // innermost block (with the top coefficient on X^4), then Horner in X^4
    int j = r - 1;
    roks::count_launch(), k_big_ps_block<U><<<eb, 256, 0, st>>>(n, X1, X2, X3, X4, R(cf[4 * j]), R(cf[4 * j + 1]),
                                                                  R(cf[4 * j + 2]), R(cf[4 * j + 3]), R(cf[d]), P);
    for (j = r - 2; j >= 0; --j) {
        roks::count_launch(), k_big_ps_block<U><<<eb, 256, 0, st>>>(n, X1, X2, X3, X4, R(cf[4 * j]),
                                                                      R(cf[4 * j + 1]), R(cf[4 * j + 2]),
                                                                      R(cf[4 * j + 3]), R(0), Bj);
        roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, X4, P, Q, R(1), Bj, 0, nullptr, 0);
        U* t = P; P = Q; Q = t;
    }
    // squarings: the device's q of them, the rest return at once
    for (int k = 0; k < max_square; ++k) {
        U* src = (k & 1) ? Q : P;
        U* dst = (k & 1) ? P : Q;
        roks::count_launch(), k_sq_gemm<U><<<g, 256, 0, st>>>(n, src, src, dst, R(1), nullptr, 0, info, k);
    }
    roks::count_launch(), k_big_to_double<U><<<eb, 256, 0, st>>>(n, P, Q, info, max_square, E);
}

size_t expm_big_work_bytes(int n, bool fp64) { return (fp64 ? sizeof(double2) : sizeof(float2)) * 7 * (size_t)n * n; }

void expm_big(int n, const double2* A, const double* scale_dev, double2* E, void* work, double* info, bool fp64,
              cudaStream_t st) {
    // FP64: degree 16 (||X|| <= 1/4 gives 1e-26); FP32: degree 8 (1e-11);
    // at most 24 squarings (the launches past the device's q return at once).
    if (fp64) expm_big_impl<double2>(n, A, scale_dev, E, static_cast<double2*>(work), info, 4, 24, st);
    else expm_big_impl<float2>(n, A, scale_dev, E, static_cast<float2*>(work), info, 2, 24, st);
}

}  // namespace roks
