// k_exx_grid.cuh -- the grid work of the exact exchange for one batch of
// pairs, with the pointwise steps fused into the transform passes:
//
//   x pass, forward : rho_jn = conj(psi_j) psi_n formed while the x lines load
//   y pass, forward : plain strided pass
//   z pass          : forward transform, times v(G) / N^3 (and the partial
//                     sums of the pair integrals), inverse transform, in one
//                     tile (the z lines are contiguous)
//   y, x passes, inverse: plain strided passes (W_jn)
//   accumulation    : X_n += c(n, j) psi_j W_jn and X_j += c(j, n) psi_n
//                     conj(W_jn), one thread per grid point over the
//                     batch's pairs in order
//
// Against the separate pair-density, 3D-transform, multiply and
// accumulation kernels this saves six of the sixteen passes over the batch
// buffer per pair.  (Folding the accumulation into the inverse x pass, with
// each block looping over the batch's pairs to own its grid points, left
// too few blocks in flight: 137 ms per hybrid-72 apply against 104.)
#pragma once

#include "k_fft_impl.cuh"
#include "roks_exx.cuh"

namespace roks {

// grid index p = (x N + y) N + z; a block of the x passes owns the TL lines
// z0 .. z0 + TL - 1 of one y
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_exx_x_fwd(const c2<T>* __restrict__ tw, const c2<T>* __restrict__ Phi,
                                                        const int* __restrict__ pj, const int* __restrict__ pn,
                                                        int p0, c2<T>* __restrict__ buf) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    constexpr int64_t N3 = (int64_t)N * N * N, NN = (int64_t)N * N;
    extern __shared__ __align__(16) unsigned char smem[];
    V* bs = reinterpret_cast<V*>(smem);
    V* tws = bs + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL, y = blockIdx.y, b = blockIdx.z;
    const int j = pj[p0 + b], n = pn[p0 + b];
    const V* Pj = Phi + (int64_t)j * N3 + y * N + z0;
    const V* Pn = Phi + (int64_t)n * N3 + y * N + z0;
    V* out = buf + (int64_t)b * N3 + y * N + z0;
    fft_io<V, N, -1, TL, LS, kThreads, false, false>(
        bs, tws,
        [&](int line, int e) {
            if (z0 + line >= N) return mk<T>(T(0), T(0));
            const int64_t o = e * NN + line;
            return cmulc(Pj[o], Pn[o]);
        },
        [&](int line, int e, V v, int, int) {
            if (z0 + line < N) out[e * NN + line] = v;
        });
}

// z lines (contiguous), tiles t = blockIdx.x, blockIdx.x + gridDim.x, ...:
// forward transform, times vG = v(G) / N^3, inverse transform; the block's
// sum of vG |rho(G)|^2 goes to part[b * gridDim.x + blockIdx.x]
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_exx_z_mult(const c2<T>* __restrict__ tw, const T* __restrict__ vG,
                                                         c2<T>* __restrict__ buf, double* __restrict__ part) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    constexpr int64_t N3 = (int64_t)N * N * N;
    constexpr int NLINE = N * N;
    constexpr int NT = (NLINE + TL - 1) / TL;
    extern __shared__ __align__(16) unsigned char smem[];
    V* bs = reinterpret_cast<V*>(smem);
    V* tws = bs + N * LS;
    __shared__ double red[kThreads];
    load_twiddles<V, N>(tws, tw);
    const int b = blockIdx.y;
    V* d = buf + (int64_t)b * N3;
    T acc = T(0);
    for (int t = blockIdx.x; t < NT; t += gridDim.x) {
        const int l0 = t * TL;
        __syncthreads();
        for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
            const int line = idx / N, e = idx - line * N;
            const int l = l0 + line;
            bs[e * LS + line] = l < NLINE ? d[(int64_t)l * N + e] : mk<T>(T(0), T(0));
        }
        __syncthreads();
        tile_fft<V, N, -1, TL, LS, kThreads>(bs, tws);
        for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
            const int line = idx / N, e = idx - line * N;
            const int l = l0 + line;
            const T w = l < NLINE ? vG[(int64_t)l * N + e] : T(0);
            const V v = bs[e * LS + line];
            acc += w * (v.x * v.x + v.y * v.y);
            bs[e * LS + line] = mk<T>(v.x * w, v.y * w);
        }
        __syncthreads();
        tile_fft<V, N, +1, TL, LS, kThreads>(bs, tws);
        for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
            const int line = idx / N, e = idx - line * N;
            const int l = l0 + line;
            if (l < NLINE) d[(int64_t)l * N + e] = bs[e * LS + line];
        }
    }
    red[threadIdx.x] = double(acc);
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = red[0];
}

// Exchange field accumulation, one thread per grid point, pairs in order
// (n ascending, j ascending): X_n += c(n, j) psi_j W, X_j += c(j, n) psi_n conj(W).
template <typename T>
__global__ void k_exx_accumulate(int64_t N3, const c2<T>* __restrict__ Phi, const c2<T>* __restrict__ W,
                                 const int* __restrict__ pj, const int* __restrict__ pn, int p0, int np,
                                 ExxCoef cf, c2<T>* __restrict__ X) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N3) return;
    int cur = -1;
    T ax = 0, ay = 0;
    for (int b = 0; b < np; ++b) {
        const int j = pj[p0 + b], n = pn[p0 + b];
        if (n != cur) {
            if (cur >= 0) {
                c2<T> o = X[(int64_t)cur * N3 + p];
                X[(int64_t)cur * N3 + p] = mk<T>(o.x + ax, o.y + ay);
            }
            cur = n;
            ax = ay = T(0);
        }
        const c2<T> w = W[(int64_t)b * N3 + p];
        const int kn = n < cf.n_closed ? 0 : n - cf.n_closed + 1;
        const int kj = j < cf.n_closed ? 0 : j - cf.n_closed + 1;
        const c2<T> pjv = Phi[(int64_t)j * N3 + p];
        const T cnj = T(cf.c[kn][kj]);
        const c2<T> t = cmul(pjv, w);
        ax += cnj * t.x;
        ay += cnj * t.y;
        if (j != n) {
            const c2<T> pnv = Phi[(int64_t)n * N3 + p];
            const T cjn = T(cf.c[kj][kn]);
            // psi_n conj(W)
            const T ux = pnv.x * w.x + pnv.y * w.y, uy = pnv.y * w.x - pnv.x * w.y;
            c2<T> o = X[(int64_t)j * N3 + p];
            X[(int64_t)j * N3 + p] = mk<T>(o.x + cjn * ux, o.y + cjn * uy);
        }
    }
    if (cur >= 0) {
        c2<T> o = X[(int64_t)cur * N3 + p];
        X[(int64_t)cur * N3 + p] = mk<T>(o.x + ax, o.y + ay);
    }
}

template <typename T, int N>
struct ExxGrid {
    using V = c2<T>;
    static constexpr int TL = tile_lines(N);
    static constexpr size_t SM = tile_smem_bytes<V, N, TL + 1>();
    static void batch(const ExxArgs<T>& a, int p0, int np, bool want_field, cudaStream_t st) {
        const int64_t N3 = (int64_t)N * N * N;
        set_smem(k_exx_x_fwd<T, N>, SM);
        set_smem(k_exx_z_mult<T, N>, SM);
        set_smem(k_grid_fft_strided<T, N>, SM);
        const dim3 gx((N + TL - 1) / TL, N, np);
        roks::count_launch(), k_exx_x_fwd<T, N><<<gx, kThreads, SM, st>>>(a.tw, a.Phi, a.pj, a.pn, p0, a.buf);
        // y lines: outer x (stride N^2), elements along y (stride N)
        roks::count_launch(), k_grid_fft_strided<T, N><<<gx, kThreads, SM, st>>>(a.tw, a.buf, (int64_t)N * N,
                                                                                (int64_t)N, -1, N3);
        roks::count_launch(), k_exx_z_mult<T, N><<<dim3(kExxBlocks, np), kThreads, SM, st>>>(a.tw, a.vG, a.buf,
                                                                                             a.part);
        if (!want_field) return;
        roks::count_launch(), k_grid_fft_strided<T, N><<<gx, kThreads, SM, st>>>(a.tw, a.buf, (int64_t)N * N,
                                                                                (int64_t)N, +1, N3);
        // x lines: outer y (stride N), elements along x (stride N^2)
        roks::count_launch(), k_grid_fft_strided<T, N><<<gx, kThreads, SM, st>>>(a.tw, a.buf, (int64_t)N,
                                                                                (int64_t)N * N, +1, N3);
        roks::count_launch(), k_exx_accumulate<T><<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(
                                  N3, a.Phi, a.buf, a.pj, a.pn, p0, np, a.cf, a.X);
    }
};

// One batch of pairs p0 .. p0 + np - 1: the pair integrals' block partials
// in a.part (np x kExxBlocks) and, with want_field, the fields added to a.X.
template <typename T>
void exx_batch_grid(const ExxArgs<T>& a, int p0, int np, bool want_field, cudaStream_t st) {
    ROKS_GRID_DISPATCH(a.N, (ExxGrid<T, NN>::batch(a, p0, np, want_field, st)));
}

}  // namespace roks
