// k_fft_impl.cuh -- the band transforms of the plane-wave apply and density
// passes, and the full-grid 3D transform.  Included by one translation unit
// per precision.
//
// Band path (inverse direction, coefficients -> real space):
//   z stage : for every (i, j) column of the sphere, scatter the contiguous
//             coefficients k = -kmax..kmax into a z line and transform it;
//   y stage : for every plane i and every z, gather the columns of the plane
//             into a y line and transform it;
//   x stage : for every (y, z), gather the 2 nmax + 1 nonzero planes into an
//             x line and transform it -> psi(r) line.
// Only the x stage touches full grid lines; columns and planes outside the
// sphere are never stored.  The forward direction mirrors it and keeps only
// the outputs that lie in the sphere.
#pragma once

#include "roks_impl.cuh"

namespace roks {

template <typename V, int N>
__device__ __forceinline__ void load_twiddles(V* tws, const V* tw) {
    for (int t = threadIdx.x; t < N; t += blockDim.x) tws[t] = tw[t];
}

template <typename V, int N, int LS>
__device__ __forceinline__ V* tile_buf(unsigned char* smem) { return reinterpret_cast<V*>(smem); }

template <typename V, int N, int LS>
constexpr size_t tile_smem_bytes() { return sizeof(V) * (size_t(N) * LS + N); }

// ------------------------------------------------------------------ z stage
// Lines (sphere columns) per tile of the z stages.  For N = 120 16, half the
// other stages' 32: the z stages' short gathers and scatters gain from more
// blocks in flight (forward z at mgo-120: 0.413 -> 0.331 ms; 24 lines 0.346).
__host__ __device__ constexpr int tile_lines_z(int n) { return n == 120 ? 16 : tile_lines(n); }

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_band_z_inv(Sphere s, const c2<T>* __restrict__ tw,
                                                         const c2<T>* __restrict__ psi, int64_t ld,
                                                         int b0, c2<T>* __restrict__ Zc) {
    using V = c2<T>;
    constexpr int TL = tile_lines_z(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    __shared__ int cstart[TL], ckmax[TL];
    load_twiddles<V, N>(tws, tw);
    const int c0 = blockIdx.x * TL;
    const int bb = blockIdx.y;
    const V* p = psi + (int64_t)(b0 + bb) * ld;
    // the lines' column descriptors once per block; then every coefficient
    // load of a thread is independent of the others (all in flight at once)
    if (threadIdx.x < TL) {
        const int c = c0 + threadIdx.x;
        cstart[threadIdx.x] = c < s.ncol ? s.col_start[c] : 0;
        ckmax[threadIdx.x] = c < s.ncol ? s.col_kmax[c] : -1;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < (TL * N + kThreads - 1) / kThreads; ++r) {
        const int idx = threadIdx.x + r * kThreads;
        if (idx < TL * N) {
            const int line = idx / N, e = idx - line * N;
            const int k = signed_freq(e, N);
            const int km = ckmax[line];
            V v = mk<T>(T(0), T(0));
            if (k >= -km && k <= km) v = p[cstart[line] + k + km];
            buf[e * LS + line] = v;
        }
    }
    __syncthreads();
    tile_fft<V, N, +1, TL, LS, kThreads>(buf, tws);
    V* out = Zc + (int64_t)bb * s.ncol * N;
    for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
        const int line = idx / N, e = idx - line * N;
        const int c = c0 + line;
        if (c < s.ncol) out[(int64_t)c * N + e] = buf[e * LS + line];
    }
}

// KIN: add the kinetic term w_k |G|^2/2 psi(G) while scattering out; without
// it the transform alone (the Gamma-point unpack adds the kinetic term)
template <typename T, int N, bool KIN>
__global__ void __launch_bounds__(kThreads) k_band_z_fwd(Sphere s, const c2<T>* __restrict__ tw,
                                                         const c2<T>* __restrict__ Zc,
                                                         c2<T>* __restrict__ out, int64_t ldo,
                                                         const c2<T>* __restrict__ psi, int64_t ldp,
                                                         const T* __restrict__ g2half,
                                                         const T* __restrict__ wk, int b0, int n_closed) {
    using V = c2<T>;
    constexpr int TL = tile_lines_z(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    __shared__ int cstart[TL], ckmax[TL];
    load_twiddles<V, N>(tws, tw);
    const int c0 = blockIdx.x * TL;
    const int bb = blockIdx.y;
    const int b = b0 + bb;
    const V* in = Zc + (int64_t)bb * s.ncol * N;
    if (threadIdx.x < TL) {
        const int c = c0 + threadIdx.x;
        cstart[threadIdx.x] = c < s.ncol ? s.col_start[c] : 0;
        ckmax[threadIdx.x] = c < s.ncol ? s.col_kmax[c] : -1;
    }
#pragma unroll
    for (int r = 0; r < (TL * N + kThreads - 1) / kThreads; ++r) {
        const int idx = threadIdx.x + r * kThreads;
        if (idx < TL * N) {
            const int line = idx / N, e = idx - line * N;
            const int c = c0 + line;
            buf[e * LS + line] = (c < s.ncol) ? in[(int64_t)c * N + e] : mk<T>(T(0), T(0));
        }
    }
    __syncthreads();
    tile_fft<V, N, -1, TL, LS, kThreads>(buf, tws);
    const int cls = b < n_closed ? 0 : b - n_closed + 1;
    const T w = KIN ? wk[cls] : T(0);
    V* o = out + (int64_t)b * ldo;
    const V* p = KIN ? psi + (int64_t)b * ldp : nullptr;
#pragma unroll
    for (int r = 0; r < (TL * N + kThreads - 1) / kThreads; ++r) {
        const int idx = threadIdx.x + r * kThreads;
        if (idx < TL * N) {
            const int line = idx / N, e = idx - line * N;
            const int k = signed_freq(e, N);
            const int km = ckmax[line];
            if (k >= -km && k <= km) {
                const int g = cstart[line] + k + km;
                const V loc = buf[e * LS + line];
                if constexpr (KIN) {
                    const V ps = p[g];
                    const T kin = w * g2half[g];
                    o[g] = mk<T>(loc.x + kin * ps.x, loc.y + kin * ps.y);
                } else {
                    o[g] = loc;
                }
            }
        }
    }
}

// ------------------------------------------------------------------ y stage
// PRUNE (y_inv and the inverse x stages): the sphere's frequencies lie within
// |i|, |j| <= sphere_prune_nmax(N), so the first pass leaves out the inputs
// that are zero for every butterfly (sphere_zero_mask).
template <typename T, int N, bool PRUNE>
__global__ void __launch_bounds__(kThreads) k_band_y_inv(Sphere s, const c2<T>* __restrict__ tw,
                                                         const c2<T>* __restrict__ Zc,
                                                         c2<T>* __restrict__ Yp) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL;
    const int p = blockIdx.y;
    const int bb = blockIdx.z;
    const int jm = s.plane_jmax[p];
    const V* in = Zc + ((int64_t)bb * s.ncol + s.plane_col0[p] + jm) * N;
    V* out = Yp + ((int64_t)bb * s.np + p) * N * N;
    fft_io<V, N, +1, TL, LS, kThreads, false, false, PRUNE ? sphere_zero_mask(N) : 0u>(
        buf, tws,
        [&](int line, int e) {
            const int z = z0 + line, j = signed_freq(e, N);
            return (z < N && j >= -jm && j <= jm) ? in[(int64_t)j * N + z] : mk<T>(T(0), T(0));
        },
        [&](int line, int e, V v, int, int) {
            const int z = z0 + line;
            if (z < N) out[(int64_t)e * N + z] = v;
        });
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_band_y_fwd(Sphere s, const c2<T>* __restrict__ tw,
                                                         const c2<T>* __restrict__ Yp,
                                                         c2<T>* __restrict__ Zc) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL;
    const int p = blockIdx.y;
    const int bb = blockIdx.z;
    const V* in = Yp + ((int64_t)bb * s.np + p) * N * N;
    const int jm = s.plane_jmax[p];
    V* out = Zc + ((int64_t)bb * s.ncol + s.plane_col0[p] + jm) * N;
    fft_io<V, N, -1, TL, LS, kThreads, false, false>(
        buf, tws,
        [&](int line, int e) {
            const int z = z0 + line;
            return (z < N) ? in[(int64_t)e * N + z] : mk<T>(T(0), T(0));
        },
        [&](int line, int e, V v, int, int) {
            const int z = z0 + line, j = signed_freq(e, N);
            if (z < N && j >= -jm && j <= jm) out[(int64_t)j * N + z] = v;
        });
}

// ------------------------------------------------------------------ x stage
template <typename T, int N>
__device__ __forceinline__ void load_x_lines(const Sphere& s, c2<T>* buf, const c2<T>* Ypb, int y, int z0) {
    constexpr int TL = tile_lines(N), LS = TL + 1;
    for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
        const int e = idx / TL, line = idx - e * TL;
        const int z = z0 + line;
        const int i = signed_freq(e, N);
        c2<T> v = mk<T>(T(0), T(0));
        if (z < N && i >= -s.nmax && i <= s.nmax) v = Ypb[((int64_t)(i + s.nmax) * N + y) * N + z];
        buf[e * LS + line] = v;
    }
}

// SPLIT: every band of the launch holds two real orbitals as (re, im) with
// the classes a and b (the Gamma-point packing of the open pair): re is
// multiplied by V^a, im by V^b.
template <typename T, int N, bool SPLIT, bool PRUNE>
__global__ void __launch_bounds__(x_threads(N)) k_band_x_apply(Sphere s, const c2<T>* __restrict__ tw,
                                                               c2<T>* __restrict__ Yp,
                                                               const T* __restrict__ Vk,
                                                               const c2<T>* __restrict__ Xx, int b0,
                                                               int n_closed, T scale) {
    constexpr int NT = x_threads(N);
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL;
    const int y = blockIdx.y;
    const int bb = blockIdx.z;
    const int b = b0 + bb;
    const int cls = SPLIT ? 1 : (b < n_closed ? 0 : b - n_closed + 1);
    // offsets within one band's planes and within one N^3 grid fit in 32 bits
    V* Ypb = Yp + (int64_t)bb * s.np * N * N + y * N + z0;
    const T* Vc = Vk + (int64_t)cls * N * N * N + y * N + z0;
    const T* Vc2 = Vk + (int64_t)2 * N * N * N + y * N + z0;
    const c2<T>* Xb = Xx ? Xx + (int64_t)b * N * N * N + y * N + z0 : nullptr;
    const int nmax = s.nmax;
    constexpr int NN = N * N;
    // inverse x transform; the last pass forms (V psi + X) * scale in the tile,
    // X being the exchange field of the band (absent without exact exchange)
    fft_io<V, N, +1, TL, LS, NT, false, true, PRUNE ? sphere_zero_mask(N) : 0u>(
        buf, tws,
        [&](int line, int e) {
            const int i = signed_freq(e, N);
            return (z0 + line < N && i >= -nmax && i <= nmax) ? Ypb[(i + nmax) * NN + line] : mk<T>(T(0), T(0));
        },
        [&](int line, int e, V v, int, int) {
            const bool in = z0 + line < N;
            const int gi = e * NN + line;
            const T w = in ? Vc[gi] * scale : T(0);
            T w2 = w;
            if constexpr (SPLIT) w2 = in ? Vc2[gi] * scale : T(0);
            V o = mk<T>(v.x * w, v.y * w2);
            if (Xb && in) {
                const V xv = Xb[gi];
                o.x += xv.x * scale;
                o.y += xv.y * scale;
            }
            buf[e * LS + line] = o;
        });
    __syncthreads();
    // forward x transform; the last pass keeps the planes of the sphere
    fft_io<V, N, -1, TL, LS, NT, true, false>(
        buf, tws, [&](int line, int e) { return buf[e * LS + line]; },
        [&](int line, int e, V v, int, int) {
            const int i = signed_freq(e, N);
            if (z0 + line < N && i >= -nmax && i <= nmax) Ypb[(i + nmax) * NN + line] = v;
        });
}

// Real-space orbitals on the full grid: Phi[b] = scale * inverse x transform
// of the plane data (used by the exact-exchange pair densities).
template <typename T, int N, bool PRUNE>
__global__ void __launch_bounds__(kThreads) k_band_x_inv_full(Sphere s, const c2<T>* __restrict__ tw,
                                                              const c2<T>* __restrict__ Yp,
                                                              c2<T>* __restrict__ Phi, int b0, T scale) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL;
    const int y = blockIdx.y;
    const int bb = blockIdx.z;
    const V* Ypb = Yp + (int64_t)bb * s.np * N * N;
    V* out = Phi + (int64_t)(b0 + bb) * N * N * N;
    const int nmax = s.nmax;
    fft_io<V, N, +1, TL, LS, kThreads, false, false, PRUNE ? sphere_zero_mask(N) : 0u>(
        buf, tws,
        [&](int line, int e) {
            const int z = z0 + line, i = signed_freq(e, N);
            return (z < N && i >= -nmax && i <= nmax) ? Ypb[((int64_t)(i + nmax) * N + y) * N + z]
                                                      : mk<T>(T(0), T(0));
        },
        [&](int line, int e, V v, int, int) {
            const int z = z0 + line;
            if (z < N) out[((int64_t)e * N + y) * N + z] = mk<T>(v.x * scale, v.y * scale);
        });
}

// Density: block (z tile, y, g) transforms the bands of group g (bands
// b0 + g*gs ...).  The last pass of each inverse x transform leaves every
// thread the same set of output points, so |psi|^2 is summed in registers
// (FP32 partial sums of up to 16 bands, added in FP64).  Closed-shell sums go
// to the group's own slot (slot[g], N^3 doubles, written in full so no
// clearing is needed); the open bands a and b, one band each, go straight to
// rho3.  k_density_reduce adds the slots in group order.
// The staging buffers hold full x lines, element e of line l at e * TL + l:
// the rows of the planes outside the sphere (and the lines past N of the
// last z tile) are zeroed once, so the first pass loads without tests.
// SEL: (Re psi)^2 (part_sel 1) or (Im psi)^2 (part_sel 2) instead of |psi|^2.
template <typename T, int N, bool SEL, bool PRUNE>
__global__ void __launch_bounds__(kThreads) k_band_x_density(Sphere s, const c2<T>* __restrict__ tw,
                                                             const c2<T>* __restrict__ Yp,
                                                             typename DensAcc<T>::S* __restrict__ rho3,
                                                             typename DensAcc<T>::S* __restrict__ slot,
                                                             int b0, int nbb, int gs, int n_closed, T scale,
                                                             int part_sel, int cls_override) {
    using V = c2<T>;
    using DA = DensAcc<T>;
    using DS = typename DA::S;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    using Slots = LastPassSlots<N, TL, kThreads>;
    constexpr int PER = Slots::PER, R = Slots::R;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    V* stg = tws + N;   // two staging buffers of N x TL (x lines) for the next band
    load_twiddles<V, N>(tws, tw);
    const int z0 = blockIdx.x * TL;
    const int y = blockIdx.y;
    const int g = blockIdx.z;
    const int N3 = N * N * N;
    const int nmax = s.nmax, np = s.np;
    const int gbeg = g * gs, gend = min(nbb, gbeg + gs);
    // rows of TL lines are 16-byte aligned in both memories (N even, TL a
    // multiple of 16): copy them with 16-byte cp.async, only the chunks of
    // lines z < N (the last tile may overhang the row)
    constexpr int CH = TL * (int)sizeof(V) / 16;   // 16-byte chunks per row
    const int chv = min(CH, (N - z0) * (int)sizeof(V) / 16);
    for (int t = threadIdx.x; t < 2 * N * TL; t += blockDim.x) stg[t] = mk<T>(T(0), T(0));
    __syncthreads();
    auto stage = [&](int band, int which) {
        const char* src = reinterpret_cast<const char*>(Yp + (int64_t)band * np * N * N + y * N + z0);
        char* dst = reinterpret_cast<char*>(stg + which * N * TL);
        for (int c = threadIdx.x; c < np * CH; c += blockDim.x) {
            const int row = c / CH, k = c - row * CH;
            if (k >= chv) continue;
            // plane row (i + nmax) -> x index e = i mod N
            const int e = row >= nmax ? row - nmax : N + row - nmax;
            const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst + e * TL * sizeof(V) + 16 * k));
            const char* sp = src + (int64_t)row * N * N * sizeof(V) + 16 * k;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(sp) : "memory");
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    if (gbeg < gend) stage(gbeg, 0);
    DS* slot_g = slot + (int64_t)g * N3;
    bool slot_written = false;
    int bb = gbeg;
    while (bb < gend) {
        const int b = b0 + bb;
        const int cls = cls_override >= 0 ? cls_override : (b < n_closed ? 0 : b - n_closed + 1);
        const int seg_end = cls == 0 ? min(gend, n_closed - b0) : bb + 1;
        DS* rr = cls == 0 ? slot_g : rho3 + (int64_t)cls * N3;
        while (bb < seg_end) {
            T part[PER][R];
#pragma unroll
            for (int q = 0; q < PER; ++q)
#pragma unroll
                for (int r = 0; r < R; ++r) part[q][r] = T(0);
            const int chunk_end = min(seg_end, bb + 16);
            for (; bb < chunk_end; ++bb) {
                // the next band's planes stream in while this one is transformed
                if (bb + 1 < gend) {
                    stage(bb + 1, (bb + 1 - gbeg) & 1);
                    asm volatile("cp.async.wait_group 1;" ::: "memory");
                } else {
                    asm volatile("cp.async.wait_group 0;" ::: "memory");
                }
                __syncthreads();
                const V* sb = stg + ((bb - gbeg) & 1) * N * TL;
                fft_io<V, N, +1, TL, LS, kThreads, false, false, PRUNE ? sphere_zero_mask(N) : 0u>(
                    buf, tws, [&](int line, int e) { return sb[e * TL + line]; },
                    [&](int, int, V v, int q, int r) {
                        if constexpr (SEL)
                            part[q][r] += part_sel == 1 ? v.x * v.x : v.y * v.y;
                        else
                            part[q][r] += v.x * v.x + v.y * v.y;
                    });
                __syncthreads();
            }
            const bool first = cls == 0 && !slot_written;
#pragma unroll
            for (int q = 0; q < PER; ++q)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int line = 0, e = 0;
                    if (Slots::point(threadIdx.x, q, r, line, e) && z0 + line < N) {
                        DS* dst = rr + (e * N + y) * N + z0 + line;
                        const T add = part[q][r] * scale;
                        *dst = (cls != 0 || !first) ? DA::add(*dst, add) : DA::make(add);
                    }
                }
            if (cls == 0) slot_written = true;
        }
    }
    if (!slot_written && slot) {
        // a group without closed bands still owns its slot
#pragma unroll
        for (int q = 0; q < PER; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                int line = 0, e = 0;
                if (Slots::point(threadIdx.x, q, r, line, e) && z0 + line < N)
                    slot_g[(e * N + y) * N + z0 + line] = DA::make(T(0));
            }
    }
}

// rho3[0] = sum of the closed-shell slots in group order
template <typename T>
__global__ void k_density_reduce(int N3, int ng, const typename DensAcc<T>::S* __restrict__ slot,
                                 typename DensAcc<T>::S* __restrict__ rho) {
    using DA = DensAcc<T>;
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N3) return;
    typename DA::S s = slot[p];
    for (int g = 1; g < ng; ++g) s = DA::add2(s, slot[(int64_t)g * N3 + p]);
    rho[p] = s;
}

// ------------------------------------------------------------------ full grid
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_grid_fft_z(const c2<T>* __restrict__ tw, c2<T>* data, int dir,
                                                         int64_t bstride) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    data += (int64_t)blockIdx.y * bstride;
    const int l0 = blockIdx.x * TL;           // line = x * N + y
    for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
        const int line = idx / N, e = idx - line * N;
        const int l = l0 + line;
        buf[e * LS + line] = (l < N * N) ? data[(int64_t)l * N + e] : mk<T>(T(0), T(0));
    }
    __syncthreads();
    if (dir > 0) tile_fft<V, N, +1, TL, LS, kThreads>(buf, tws);
    else tile_fft<V, N, -1, TL, LS, kThreads>(buf, tws);
    for (int idx = threadIdx.x; idx < TL * N; idx += kThreads) {
        const int line = idx / N, e = idx - line * N;
        const int l = l0 + line;
        if (l < N * N) data[(int64_t)l * N + e] = buf[e * LS + line];
    }
}

// Lines along y (outer = x, estride = N) or x (outer = y, ostride = N,
// estride = N^2); the tile runs over consecutive z.
template <typename T, int N>
__global__ void __launch_bounds__(kThreads) k_grid_fft_strided(const c2<T>* __restrict__ tw, c2<T>* data,
                                                               int64_t ostride, int64_t estride, int dir,
                                                               int64_t bstride) {
    using V = c2<T>;
    constexpr int TL = tile_lines(N), LS = TL + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    V* buf = reinterpret_cast<V*>(smem);
    V* tws = buf + N * LS;
    load_twiddles<V, N>(tws, tw);
    __syncthreads();
    const int z0 = blockIdx.x * TL;
    V* base = data + (int64_t)blockIdx.z * bstride + (int64_t)blockIdx.y * ostride;
    auto ld = [&](int line, int e) {
        const int z = z0 + line;
        return (z < N) ? base[e * estride + z] : mk<T>(T(0), T(0));
    };
    auto st = [&](int line, int e, V v, int, int) {
        const int z = z0 + line;
        if (z < N) base[e * estride + z] = v;
    };
    // every element is read in the first pass before any is written in the
    // last (the tile sits between), so the transform may work in place
    if (dir > 0) fft_io<V, N, +1, TL, LS, kThreads, false, false>(buf, tws, ld, st);
    else fft_io<V, N, -1, TL, LS, kThreads, false, false>(buf, tws, ld, st);
}

// ------------------------------------------------------------------ launchers
template <typename K>
static void set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <typename T, int N>
struct BandFft {
    using V = c2<T>;
    static constexpr int TL = tile_lines(N);
    static constexpr size_t SM = tile_smem_bytes<V, N, TL + 1>();
    static constexpr int TLZ = tile_lines_z(N);
    static constexpr size_t SMZ = tile_smem_bytes<V, N, TLZ + 1>();

    static void z_inv(const Sphere& s, const V* tw, const V* psi, int64_t ld, int b0, int nbb, V* Zc,
                      cudaStream_t st) {
        set_smem(k_band_z_inv<T, N>, SMZ);
        dim3 gz((s.ncol + TLZ - 1) / TLZ, nbb);
        roks::count_launch(), k_band_z_inv<T, N><<<gz, kThreads, SMZ, st>>>(s, tw, psi, ld, b0, Zc);
    }
    // the sphere fits the pruned first passes
    static bool prune(const Sphere& s) { return s.nmax <= sphere_prune_nmax(N); }
    static void y_inv(const Sphere& s, const V* tw, const V* Zc, V* Yp, int nbb, cudaStream_t st) {
        dim3 gy((N + TL - 1) / TL, s.np, nbb);
        if (prune(s)) {
            set_smem(k_band_y_inv<T, N, true>, SM);
            roks::count_launch(), k_band_y_inv<T, N, true><<<gy, kThreads, SM, st>>>(s, tw, Zc, Yp);
        } else {
            set_smem(k_band_y_inv<T, N, false>, SM);
            roks::count_launch(), k_band_y_inv<T, N, false><<<gy, kThreads, SM, st>>>(s, tw, Zc, Yp);
        }
    }
    // split_band (if within the launch) takes the SPLIT instance, alone
    static void x_apply(const Sphere& s, const V* tw, V* Yp, const T* Vk, const V* Xx, int b0, int nbb, int nc,
                        int split_band, T scale, cudaStream_t st) {
        const bool pr = prune(s);
        auto run = [&](bool split, int first, int count) {
            if (count <= 0) return;
            // the kernel indexes the planes from the launch's first band
            V* Y = Yp + (int64_t)(first - b0) * s.np * N * N;
            dim3 g((N + TL - 1) / TL, N, count);
            auto go = [&](auto kernel) {
                set_smem(kernel, SM);
                roks::count_launch(), kernel<<<g, x_threads(N), SM, st>>>(s, tw, Y, Vk, Xx, first, nc, scale);
            };
            if (split)
                pr ? go(k_band_x_apply<T, N, true, true>) : go(k_band_x_apply<T, N, true, false>);
            else
                pr ? go(k_band_x_apply<T, N, false, true>) : go(k_band_x_apply<T, N, false, false>);
        };
        if (split_band < b0 || split_band >= b0 + nbb) {
            run(false, b0, nbb);
        } else {
            run(false, b0, split_band - b0);
            run(true, split_band, 1);
            run(false, split_band + 1, b0 + nbb - split_band - 1);
        }
    }
    static void x_inv_full(const Sphere& s, const V* tw, const V* Yp, V* Phi, int b0, int nbb, T scale,
                           cudaStream_t st) {
        dim3 g((N + TL - 1) / TL, N, nbb);
        if (prune(s)) {
            set_smem(k_band_x_inv_full<T, N, true>, SM);
            roks::count_launch(), k_band_x_inv_full<T, N, true><<<g, kThreads, SM, st>>>(s, tw, Yp, Phi, b0, scale);
        } else {
            set_smem(k_band_x_inv_full<T, N, false>, SM);
            roks::count_launch(), k_band_x_inv_full<T, N, false><<<g, kThreads, SM, st>>>(s, tw, Yp, Phi, b0, scale);
        }
    }
    static void y_fwd(const Sphere& s, const V* tw, const V* Yp, V* Zc, int nbb, cudaStream_t st) {
        set_smem(k_band_y_fwd<T, N>, SM);
        dim3 gy((N + TL - 1) / TL, s.np, nbb);
        roks::count_launch(), k_band_y_fwd<T, N><<<gy, kThreads, SM, st>>>(s, tw, Yp, Zc);
    }
    static void z_fwd(const Sphere& s, const V* tw, const V* Zc, V* out, int64_t ldo, const V* psi, int64_t ldp,
                      const T* g2half, const T* wk, int b0, int nbb, int nc, cudaStream_t st) {
        dim3 gz((s.ncol + TLZ - 1) / TLZ, nbb);
        if (psi) {
            set_smem(k_band_z_fwd<T, N, true>, SMZ);
            roks::count_launch(), k_band_z_fwd<T, N, true><<<gz, kThreads, SMZ, st>>>(s, tw, Zc, out, ldo, psi, ldp,
                                                                                      g2half, wk, b0, nc);
        } else {
            set_smem(k_band_z_fwd<T, N, false>, SMZ);
            roks::count_launch(), k_band_z_fwd<T, N, false><<<gz, kThreads, SMZ, st>>>(s, tw, Zc, out, ldo, psi,
                                                                                       ldp, g2half, wk, b0, nc);
        }
    }
    // slot null: the bands are open-shell ones (or cls_override >= 0) and go
    // straight to rho3, no group slots are written and none are reduced
    static void x_density(const Sphere& s, const V* tw, const V* Yp, double* rho3, double* slot, int ngroups,
                          int b0, int nbb, int nc, double scale, int part_sel, int cls_override,
                          cudaStream_t st) {
        // tile, twiddles and two staging buffers of N x TL
        const size_t sm = SM + 2 * sizeof(V) * (size_t)N * TL;
        const int gs = (nbb + ngroups - 1) / ngroups;
        const int ng = (nbb + gs - 1) / gs;
        dim3 g((N + TL - 1) / TL, N, ng);
        using DS = typename DensAcc<T>::S;
        DS* r3 = reinterpret_cast<DS*>(rho3);
        DS* sl = reinterpret_cast<DS*>(slot);
        auto go = [&](auto kernel) {
            set_smem(kernel, sm);
            roks::count_launch(),
                kernel<<<g, kThreads, sm, st>>>(s, tw, Yp, r3, sl, b0, nbb, gs, nc, T(scale), part_sel, cls_override);
        };
        const bool pr = prune(s);
        if (part_sel == 0)
            pr ? go(k_band_x_density<T, N, false, true>) : go(k_band_x_density<T, N, false, false>);
        else
            pr ? go(k_band_x_density<T, N, true, true>) : go(k_band_x_density<T, N, true, false>);
        if (!sl) return;
        const int N3 = N * N * N;
        roks::count_launch(), k_density_reduce<T><<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N3, ng, sl, r3);
    }
    static void grid3(const V* tw, V* data, int dir, int batch, int64_t bstride, cudaStream_t st) {
        set_smem(k_grid_fft_z<T, N>, SM);
        set_smem(k_grid_fft_strided<T, N>, SM);
        dim3 gz((N * N + TL - 1) / TL, batch);
        roks::count_launch(), k_grid_fft_z<T, N><<<gz, kThreads, SM, st>>>(tw, data, dir, bstride);
        dim3 g((N + TL - 1) / TL, N, batch);
        roks::count_launch(), k_grid_fft_strided<T, N><<<g, kThreads, SM, st>>>(tw, data, (int64_t)N * N, (int64_t)N,
                                                                               dir, bstride);
        roks::count_launch(), k_grid_fft_strided<T, N><<<g, kThreads, SM, st>>>(tw, data, (int64_t)N, (int64_t)N * N,
                                                                               dir, bstride);
    }
};

#define ROKS_GRID_DISPATCH(N_, CALL)    \
    switch (N_) {                       \
        case 16: { constexpr int NN = 16; CALL; } break;   \
        case 24: { constexpr int NN = 24; CALL; } break;   \
        case 32: { constexpr int NN = 32; CALL; } break;   \
        case 48: { constexpr int NN = 48; CALL; } break;   \
        case 72: { constexpr int NN = 72; CALL; } break;   \
        case 96: { constexpr int NN = 96; CALL; } break;   \
        case 120: { constexpr int NN = 120; CALL; } break; \
        default: break;                 \
    }

template <typename T>
void band_z_inv(const Sphere& s, const c2<T>* tw, const c2<T>* psi, int64_t ld, int b0, int nbb, c2<T>* Zc,
                cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::z_inv(s, tw, psi, ld, b0, nbb, Zc, st)));
}
template <typename T>
void band_y_inv(const Sphere& s, const c2<T>* tw, const c2<T>* Zc, c2<T>* Yp, int nbb, cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::y_inv(s, tw, Zc, Yp, nbb, st)));
}
template <typename T>
void band_x_apply(const Sphere& s, const c2<T>* tw, c2<T>* Yp, const T* Vk, const c2<T>* Xx, int b0, int nbb,
                  int n_closed, int split_band, T scale, cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::x_apply(s, tw, Yp, Vk, Xx, b0, nbb, n_closed, split_band, scale, st)));
}
template <typename T>
void band_x_inv_full(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, c2<T>* Phi, int b0, int nbb, T scale,
                     cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::x_inv_full(s, tw, Yp, Phi, b0, nbb, scale, st)));
}
template <typename T>
void band_y_fwd(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, c2<T>* Zc, int nbb, cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::y_fwd(s, tw, Yp, Zc, nbb, st)));
}
template <typename T>
void band_z_fwd(const Sphere& s, const c2<T>* tw, const c2<T>* Zc, c2<T>* out, int64_t ldo, const c2<T>* psi,
                int64_t ldp, const T* g2half, const T* wk, int b0, int nbb, int n_closed, cudaStream_t st) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::z_fwd(s, tw, Zc, out, ldo, psi, ldp, g2half, wk, b0, nbb, n_closed,
                                                   st)));
}
template <typename T>
void band_x_density(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, double* rho3, double* slot, int ngroups,
                    int b0, int nbb, int n_closed, double scale, cudaStream_t st, int part_sel, int cls_override) {
    ROKS_GRID_DISPATCH(s.N, (BandFft<T, NN>::x_density(s, tw, Yp, rho3, slot, ngroups, b0, nbb, n_closed, scale,
                                                       part_sel, cls_override, st)));
}
template <typename T>
void grid_fft3(int N, const c2<T>* tw, c2<T>* data, int dir, cudaStream_t st) {
    ROKS_GRID_DISPATCH(N, (BandFft<T, NN>::grid3(tw, data, dir, 1, 0, st)));
}
template <typename T>
void grid_fft3_batched(int N, const c2<T>* tw, c2<T>* data, int batch, int64_t bstride, int dir, cudaStream_t st) {
    ROKS_GRID_DISPATCH(N, (BandFft<T, NN>::grid3(tw, data, dir, batch, bstride, st)));
}

#define ROKS_INSTANTIATE_FFT(T)                                                                              \
    template void band_z_inv<T>(const Sphere&, const c2<T>*, const c2<T>*, int64_t, int, int, c2<T>*,           \
                                cudaStream_t);                                                                   \
    template void band_y_inv<T>(const Sphere&, const c2<T>*, const c2<T>*, c2<T>*, int, cudaStream_t);          \
    template void band_x_apply<T>(const Sphere&, const c2<T>*, c2<T>*, const T*, const c2<T>*, int, int, int, int, \
                                  T, cudaStream_t);                                                              \
    template void band_x_inv_full<T>(const Sphere&, const c2<T>*, const c2<T>*, c2<T>*, int, int, T, cudaStream_t); \
    template void grid_fft3_batched<T>(int, const c2<T>*, c2<T>*, int, int64_t, int, cudaStream_t);             \
    template void band_y_fwd<T>(const Sphere&, const c2<T>*, const c2<T>*, c2<T>*, int, cudaStream_t);          \
    template void band_z_fwd<T>(const Sphere&, const c2<T>*, const c2<T>*, c2<T>*, int64_t, const c2<T>*,        \
                                int64_t, const T*, const T*, int, int, int, cudaStream_t);                      \
    template void band_x_density<T>(const Sphere&, const c2<T>*, const c2<T>*, double*, double*, int, int, int,  \
                                    int, double, cudaStream_t, int, int);                                        \
    template void grid_fft3<T>(int, const c2<T>*, c2<T>*, int, cudaStream_t);

}  // namespace roks
