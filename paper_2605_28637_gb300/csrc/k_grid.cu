// k_grid.cu -- pointwise and reduction kernels on the real-space grid and on
// plane-wave coefficient blocks: model set-up (local wells, projectors),
// per-band sums, potentials (Hartree, Slater exchange, class potentials),
// and the pointwise steps of the PCG iteration (TPA preconditioner, axpy).
#include "roks_grid.cuh"

namespace roks {

constexpr double kPi = 3.14159265358979323846;
constexpr int RB = 256;   // threads of the reduction blocks

__device__ __forceinline__ double block_sum(double v, double* sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = RB / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// Block sum of per-thread values of the element type, in FP64, valid in
// thread 0.  FP32: each warp reduces (sum, error) pairs with Knuth's
// two-sum and only the warp results are widened, so no per-thread FP64
// arithmetic or conversion runs (both are slow on this part) while the sum
// keeps about FP64 accuracy.  FP64: the plain tree.
template <typename T>
__device__ __forceinline__ double block_sum_t(T v, double* sh) {
    if constexpr (sizeof(T) == 8) {
        return block_sum(v, sh);
    } else {
        float s = v, c = 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float so = __shfl_xor_sync(0xffffffffu, s, o);
            const float co = __shfl_xor_sync(0xffffffffu, c, o);
            const float t = s + so;
            const float bp = t - s;
            c = c + co + ((s - (t - bp)) + (so - bp));
            s = t;
        }
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) sh[warp] = double(s) + double(c);
        __syncthreads();
        double r = 0.0;
        if (threadIdx.x == 0)
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r += sh[w];
        __syncthreads();
        return r;
    }
}

// ------------------------------------------------------------------ set-up
// V(G) = -(1/Omega) sum_a d_a (2 pi w^2)^{3/2} exp(-G^2 w^2 / 2) exp(-i G.R_a)
// on the grid (signed frequencies, N/2 -> +N/2), zero on Nyquist planes.
__global__ void k_vloc_G(int N, double b, double omega, int natoms, const double* __restrict__ atoms,
                         double2* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N3 = (int64_t)N * N * N;
    if (idx >= N3) return;
    const int z = idx % N, y = (idx / N) % N, x = idx / ((int64_t)N * N);
    const int fx = signed_freq(x, N), fy = signed_freq(y, N), fz = signed_freq(z, N);
    double2 v = make_double2(0.0, 0.0);
    const bool nyq = (N % 2 == 0) && (fx == N / 2 || fy == N / 2 || fz == N / 2);
    if (!nyq) {
        const double gx = b * fx, gy = b * fy, gz = b * fz;
        const double g2 = gx * gx + gy * gy + gz * gz;
        for (int a = 0; a < natoms; ++a) {
            const double* at = atoms + 5 * a;   // x, y, z, depth, width
            const double w = at[4];
            const double amp = -at[3] * pow(2.0 * kPi * w * w, 1.5) / omega * exp(-0.5 * g2 * w * w);
            const double ph = -(gx * at[0] + gy * at[1] + gz * at[2]);
            double sn, cs;
            sincos(ph, &sn, &cs);
            v.x += amp * cs;
            v.y += amp * sn;
        }
    }
    out[idx] = v;
}

__global__ void k_real_part(int64_t n, const double2* __restrict__ in, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i].x;
}

// p_i(G) = Omega^{-1/2} N_l (2 pi rc^2)^{3/2} exp(-G^2 rc^2/2) Y(G) exp(-iG.R)
// proj[i] = {x, y, z, rc, l, m}; G from the Miller vectors.
template <typename T>
__global__ void k_projectors(int npw, int nproj, double b, double omega, const int* __restrict__ miller,
                             const double* __restrict__ proj, c2<T>* __restrict__ P, int64_t ldp) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (g >= npw) return;
    const double* pr = proj + 6 * i;
    const double gx = b * miller[3 * g], gy = b * miller[3 * g + 1], gz = b * miller[3 * g + 2];
    const double g2 = gx * gx + gy * gy + gz * gz;
    const double rc = pr[3];
    const int l = int(pr[4]), m = int(pr[5]);
    double norm = pow(kPi * rc * rc, -0.75);
    if (l == 1) norm *= sqrt(2.0 / (rc * rc));
    const double pref = norm * pow(2.0 * kPi * rc * rc, 1.5) / sqrt(omega) * exp(-0.5 * g2 * rc * rc);
    double sn, cs;
    sincos(-(gx * pr[0] + gy * pr[1] + gz * pr[2]), &sn, &cs);
    double re = pref * cs, im = pref * sn;
    if (l == 1) {
        // multiply by -i rc^2 G_m
        const double gm = (m == 0 ? gx : (m == 1 ? gy : gz)) * rc * rc;
        const double r2 = im * gm, i2 = -re * gm;
        re = r2;
        im = i2;
    }
    P[(int64_t)i * ldp + g] = mk<T>(T(re), T(im));
}

// Output i of SplitMix64 seeded with `seed` (counter based: Vigna's mixing
// function applied to seed + (i + 1) * 0x9E3779B97F4A7C15), mapped to
// [-1, 1) through its top 53 bits: -1 + 2 (z >> 11) 2^-53.
__device__ __forceinline__ double splitmix64_pm1(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    const double u = (double)(z >> 11) * 0x1p-53;
    return -1.0 + 2.0 * u;
}

// Bands band0 .. band0 + gridDim.y - 1: c_nG = (u_re + i u_im) / (1 + |G|^2),
// the pair (u_re, u_im) read from u (numbered from band0) or, when u is
// null, drawn as numbers 2 (n npw + g) and 2 (n npw + g) + 1 of the seed's
// stream.
template <typename T>
__global__ void k_init_orbitals(int npw, int band0, const double* __restrict__ u, uint64_t seed,
                                const double* __restrict__ g2, c2<T>* __restrict__ psi, int64_t ld) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = band0 + blockIdx.y;
    if (g >= npw) return;
    const double d = 1.0 / (1.0 + g2[g]);
    double ur, ui;
    if (u) {
        const double* un = u + ((int64_t)blockIdx.y * npw + g) * 2;
        ur = un[0];
        ui = un[1];
    } else {
        const uint64_t i = ((uint64_t)n * (uint64_t)npw + (uint64_t)g) * 2u;
        ur = splitmix64_pm1(seed, i);
        ui = splitmix64_pm1(seed, i + 1);
    }
    psi[(int64_t)n * ld + g] = mk<T>(T(ur * d), T(ui * d));
}

template <typename T>
__global__ void k_to_real(int64_t n, const double* __restrict__ in, T* __restrict__ out, double scale) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = T(in[i] * scale);
}

// ------------------------------------------------------------------ per-band sums
// part[(op_out * nb + n) * nsplit + split]; ops:
//  0: sum 0.5 g2 |x|^2           (kinetic)
//  1: sum |x|^2, sum g2 |x|^2    (TPA scale)
//  2: sum Re(conj(x) y)          (inner product)
//  3: sum |x|^2
template <typename T, int OP>
__global__ void __launch_bounds__(RB) k_colred(int npw, int nb, const c2<T>* __restrict__ x, int64_t ldx,
                                               const c2<T>* __restrict__ y, int64_t ldy,
                                               const T* __restrict__ g2h, int nsplit, double* __restrict__ part) {
    __shared__ double sh[RB];
    const int n = blockIdx.x, sp = blockIdx.y;
    const int per = (npw + nsplit - 1) / nsplit;
    const int g0 = sp * per, g1 = min(npw, g0 + per);
    // per-thread sums in the element type (a handful of terms), block sums in FP64
    T t0 = T(0), t1 = T(0);
    const c2<T>* xc = x + (int64_t)n * ldx;
#pragma unroll 4
    for (int g = g0 + threadIdx.x; g < g1; g += RB) {
        const c2<T> a = xc[g];
        const T m = a.x * a.x + a.y * a.y;
        if (OP == 0) t0 += g2h[g] * m;
        if (OP == 1) {
            t0 += m;
            t1 += T(2) * g2h[g] * m;
        }
        if (OP == 2) {
            const c2<T> bb = y[(int64_t)n * ldy + g];
            t0 += a.x * bb.x + a.y * bb.y;
        }
        if (OP == 3) t0 += m;
    }
    double s0 = block_sum_t<T>(t0, sh);
    double s1 = 0.0;
    if (OP == 1) s1 = block_sum_t<T>(t1, sh);
    if (threadIdx.x == 0) {
        part[((int64_t)0 * nb + n) * nsplit + sp] = s0;
        if (OP == 1) part[((int64_t)1 * nb + n) * nsplit + sp] = s1;
    }
}

// Op 1 (TPA sums): out[n] = |g_n|^2, out[nb + n] = sum g2 |g_n|^2 (as
// k_colred_final sums them), then out[2 nb + 2 n] = 1/X_n and
// out[2 nb + 2 n + 1] = -2/X_n with X_n = 1.5 out[nb + n] / out[n] (Eqs. 17, 18,
// reading R1).
__global__ void k_colred_final_tpa(int nb, int nsplit, const double* __restrict__ part, double* __restrict__ out) {
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= nb) return;
    double v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const double* p = part + (int64_t)(h * nb + n) * nsplit;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < nsplit; k += 4) {
            s0 += p[k];
            s1 += p[k + 1];
            s2 += p[k + 2];
            s3 += p[k + 3];
        }
        v[h] = (s0 + s1) + (s2 + s3);
        out[h * nb + n] = v[h];
    }
    const double X = 1.5 * v[1] / fmax(v[0], 1e-300);
    out[2 * nb + 2 * n] = 1.0 / X;
    out[2 * nb + 2 * n + 1] = -2.0 / X;
}

// out[i] = sum of the nsplit partials of column i (nsplit a multiple of 4):
// four interleaved FP64 chains, combined pairwise (fixed order)
__global__ void k_colred_final(int count, int nsplit, const double* __restrict__ part, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const double* p = part + (int64_t)i * nsplit;
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int k = 0; k < nsplit; k += 4) {
        s0 += p[k];
        s1 += p[k + 1];
        s2 += p[k + 2];
        s3 += p[k + 3];
    }
    out[i] = (s0 + s1) + (s2 + s3);
}

// dst = scale * sum over the columns of their nsplit partials (nsplit a
// multiple of 4), in the order of k_colred_final then k_sum_to: lane l sums
// columns l, l + 32, ..., each as four interleaved chains, then a shuffle tree.
__global__ void k_colred_total(int count, int nsplit, const double* __restrict__ part, double* dst, double scale) {
    const int lane = threadIdx.x;
    double s = 0;
    for (int i = lane; i < count; i += 32) {
        const double* p = part + (int64_t)i * nsplit;
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int k = 0; k < nsplit; k += 4) {
            s0 += p[k];
            s1 += p[k + 1];
            s2 += p[k + 2];
            s3 += p[k + 3];
        }
        s += (s0 + s1) + (s2 + s3);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dst[0] = scale * s;
}

template <typename T>
void column_sums(int op, int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy,
                 const T* g2, double* part, double* out, cudaStream_t st) {
    constexpr int nsplit = 16;
    dim3 g(nb, nsplit);
    switch (op) {
        case 0: roks::count_launch(), k_colred<T, 0><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part); break;
        case 1: roks::count_launch(), k_colred<T, 1><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part); break;
        case 2: roks::count_launch(), k_colred<T, 2><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part); break;
        default: roks::count_launch(), k_colred<T, 3><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part); break;
    }
    if (op == 1) {
        roks::count_launch(), k_colred_final_tpa<<<(nb + 127) / 128, 128, 0, st>>>(nb, nsplit, part, out);
        return;
    }
    roks::count_launch(), k_colred_final<<<(nb + 127) / 128, 128, 0, st>>>(nb, nsplit, part, out);
}

template <typename T>
void column_total(int op, int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy, const T* g2,
                  double* part, double* dst, double scale, cudaStream_t st) {
    constexpr int nsplit = 16;
    dim3 g(nb, nsplit);
    if (op == 2) roks::count_launch(), k_colred<T, 2><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part);
    else roks::count_launch(), k_colred<T, 3><<<g, RB, 0, st>>>(npw, nb, x, ldx, y, ldy, g2, nsplit, part);
    roks::count_launch(), k_colred_total<<<1, 32, 0, st>>>(nb, nsplit, part, dst, scale);
}

// ------------------------------------------------------------------ projector blocks
// B: nproj x nb (double2, ld nproj).  Block-diagonal D, Q stored by rows:
// row i holds blk_n[i] entries for projectors blk_off[i] ... (<= kMaxBlk).
__global__ void k_apply_DQ(int nproj, int nb, const double2* __restrict__ B, const int* __restrict__ blk_off,
                           const int* __restrict__ blk_n, const double* __restrict__ Drow,
                           const double* __restrict__ Qrow, const double* __restrict__ wband,
                           double2* __restrict__ DB, double2* __restrict__ QB) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= nproj * nb) return;
    const int i = idx % nproj, n = idx / nproj;
    const int o = blk_off[i], cnt = blk_n[i];
    double dr = 0, di = 0, qr = 0, qi = 0;
    for (int j = 0; j < cnt; ++j) {
        const double2 bj = B[(int64_t)n * nproj + o + j];
        const double d = Drow[i * kMaxBlk + j], q = Qrow[i * kMaxBlk + j];
        dr += d * bj.x;
        di += d * bj.y;
        qr += q * bj.x;
        qi += q * bj.y;
    }
    const double w = wband ? wband[n] : 1.0;
    if (DB) DB[idx] = make_double2(w * dr, w * di);
    if (QB) QB[idx] = make_double2(qr, qi);
}

// NL_n = Re sum_i conj(B_in) (D B)_in  (DB unweighted)
__global__ void k_band_quadratic(int nproj, int nb, const double2* __restrict__ B,
                                 const double2* __restrict__ DB, double* __restrict__ out) {
    __shared__ double sh[RB];
    const int n = blockIdx.x;
    double s = 0.0;
    for (int i = threadIdx.x; i < nproj; i += RB) {
        const double2 a = B[(int64_t)n * nproj + i], d = DB[(int64_t)n * nproj + i];
        s += a.x * d.x + a.y * d.y;
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) out[n] = s;
}

// ------------------------------------------------------------------ potentials
// Channel densities rho^{ch} = sum_k f[k][ch] rho_k; total rho = up M + down M.
// xc3[k] = sum_ch C[k][ch] v^{ch},  v = -(1-alpha) (6 rho / pi)^{1/3};
// partial sums of (1-alpha) Slater energies per configuration and of V_loc rho.
template <typename T>
__global__ void __launch_bounds__(RB) k_pot_xc(int N3, const typename DensAcc<T>::S* __restrict__ rho3,
                                               const T* __restrict__ vloc, PotCoefT<T> cf, T c6, T cx,
                                               c2<T>* __restrict__ rho_grid, T* __restrict__ xc3,
                                               double* __restrict__ part) {
    // pointwise arithmetic in the element type T (constants come from the
    // host: FP64 arithmetic per thread is slow on this part); per-thread
    // partial energies in T over a few points, block and grid sums in FP64
    __shared__ double sh[RB];
    T exM = 0, exT = 0, eloc = 0;
    const T xs = cf.xscale;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        using DA = DensAcc<T>;
        const T rk[3] = {T(DA::value(rho3[p])), T(DA::value(rho3[N3 + p])), T(DA::value(rho3[2 * N3 + p]))};
        T v[4];
        T rho_tot = 0;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            T r = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) r += cf.f[k][ch] * rk[k];
            r = r > T(0) ? r : T(0);
            const T c = cbrt(r);
            v[ch] = -xs * c6 * c;
            const T e = -xs * cx * c * r;
            if (ch < 2) { exM += e; rho_tot += r; } else exT += e;
        }
        eloc += vloc[p] * rho_tot;
        rho_grid[p] = mk<T>(rho_tot, T(0));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s = 0;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) s += cf.C[k][ch] * v[ch];
            xc3[k * N3 + p] = s;
        }
    }
    const double dexM = block_sum_t<T>(exM, sh);
    const double dexT = block_sum_t<T>(exT, sh);
    const double deloc = block_sum_t<T>(eloc, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 0] = dexM;
        part[blockIdx.x * 4 + 1] = dexT;
        part[blockIdx.x * 4 + 2] = deloc;
        part[blockIdx.x * 4 + 3] = 0.0;
    }
}

// ------------------------------------------------------------------ PBE exchange
// Channel densities (clamped at 0) packed in pairs, gg = (up M + i down M,
// up T + i down T); the total density for the Hartree solve; V_loc rho.
template <typename T>
__global__ void __launch_bounds__(RB) k_gga_pack(int N3, const typename DensAcc<T>::S* __restrict__ rho3,
                                                 const T* __restrict__ vloc, PotCoefT<T> cf,
                                                 c2<T>* __restrict__ rho_grid, c2<T>* __restrict__ gg,
                                                 double* __restrict__ part) {
    __shared__ double sh[RB];
    T eloc = 0;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        using DA = DensAcc<T>;
        const T rk[3] = {T(DA::value(rho3[p])), T(DA::value(rho3[N3 + p])), T(DA::value(rho3[2 * N3 + p]))};
        T r[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            T v = 0;
#pragma unroll
            for (int k = 0; k < 3; ++k) v += cf.f[k][ch] * rk[k];
            r[ch] = v > T(0) ? v : T(0);
        }
        gg[p] = mk<T>(r[0], r[1]);
        gg[N3 + p] = mk<T>(r[2], r[3]);
        const T rt = r[0] + r[1];
        rho_grid[p] = mk<T>(rt, T(0));
        eloc += vloc[p] * rt;
    }
    const double d = block_sum_t<T>(eloc, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 2] = d;
        part[blockIdx.x * 4 + 3] = 0.0;
    }
}

// grid index p = (x N + y) N + z; the spectral derivative along axis c
// multiplies by i G_c, with G_c = b f_c and the Nyquist index left out
template <typename T>
__device__ __forceinline__ void gga_gvec(int p, int N, T b, T g[3]) {
    const int z = p % N, y = (p / N) % N, x = p / (N * N);
    const int idx[3] = {x, y, z};
#pragma unroll
    for (int c = 0; c < 3; ++c) g[c] = (2 * idx[c] == N) ? T(0) : b * T(signed_freq(idx[c], N));
}

// dd[3 P + c] = i G_c gg[P] / N^3 (after the forward transform of gg)
template <typename T>
__global__ void __launch_bounds__(RB) k_gga_grad(int N, T b, T inv, const c2<T>* __restrict__ gg,
                                                 c2<T>* __restrict__ dd) {
    const int N3 = N * N * N;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        T g[3];
        gga_gvec<T>(p, N, b, g);
#pragma unroll
        for (int P = 0; P < 2; ++P) {
            const c2<T> s = gg[(int64_t)P * N3 + p];
#pragma unroll
            for (int c = 0; c < 3; ++c)
                dd[(int64_t)(3 * P + c) * N3 + p] = mk<T>(-g[c] * s.y * inv, g[c] * s.x * inv);
        }
    }
}

// Per point and channel (the gradients in dd after the inverse transform):
// e, v1 = de/drho (-> v4) and the flux f grad rho, f = 2 de/d|grad rho|^2
// (-> dd, in place), all times xscale; partial sums of E_x^M, E_x^T.
template <typename T>
__global__ void __launch_bounds__(RB) k_gga_point(int N3, const typename DensAcc<T>::S* __restrict__ rho3,
                                                  PotCoefT<T> cf, T cx, T k2, T mu, T kappa, T rho_min,
                                                  c2<T>* __restrict__ dd, T* __restrict__ v4,
                                                  double* __restrict__ part) {
    __shared__ double sh[RB];
    T exM = 0, exT = 0;
    const T xs = cf.xscale;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        using DA = DensAcc<T>;
        const T rk[3] = {T(DA::value(rho3[p])), T(DA::value(rho3[N3 + p])), T(DA::value(rho3[2 * N3 + p]))};
#pragma unroll
        for (int P = 0; P < 2; ++P) {
            c2<T> gr[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) gr[c] = dd[(int64_t)(3 * P + c) * N3 + p];
            T fl[2][3];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int ch = 2 * P + h;
                T r = 0;
#pragma unroll
                for (int k = 0; k < 3; ++k) r += cf.f[k][ch] * rk[k];
                r = r > T(0) ? r : T(0);
                const T gx = h ? gr[0].y : gr[0].x, gy = h ? gr[1].y : gr[1].x, gz = h ? gr[2].y : gr[2].x;
                T e = 0, v1 = 0, f = 0;
                if (r > rho_min) {
                    const T c = cbrt(r);
                    const T s2 = (gx * gx + gy * gy + gz * gz) / (T(4) * k2 * r * r * c * c);
                    const T den = T(1) + mu * s2 / kappa;
                    const T F = T(1) + mu * s2 / den;
                    const T dF = mu / (den * den);
                    e = -xs * cx * r * c * F;
                    v1 = -(T(4) / T(3)) * xs * cx * c * (F - T(2) * s2 * dF);
                    f = -xs * cx * dF / (T(2) * k2 * r * c);
                }
                v4[(int64_t)ch * N3 + p] = v1;
                fl[h][0] = f * gx;
                fl[h][1] = f * gy;
                fl[h][2] = f * gz;
                if (P == 0) exM += e;
                else exT += e;
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) dd[(int64_t)(3 * P + c) * N3 + p] = mk<T>(fl[0][c], fl[1][c]);
        }
    }
    const double dM = block_sum_t<T>(exM, sh);
    const double dT = block_sum_t<T>(exT, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 4 + 0] = dM;
        part[blockIdx.x * 4 + 1] = dT;
    }
}

// gg[P] = sum_c i G_c dd[3 P + c] / N^3 (after the forward transform of dd)
template <typename T>
__global__ void __launch_bounds__(RB) k_gga_div(int N, T b, T inv, const c2<T>* __restrict__ dd,
                                                c2<T>* __restrict__ gg) {
    const int N3 = N * N * N;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        T g[3];
        gga_gvec<T>(p, N, b, g);
#pragma unroll
        for (int P = 0; P < 2; ++P) {
            T re = 0, im = 0;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const c2<T> s = dd[(int64_t)(3 * P + c) * N3 + p];
                re -= g[c] * s.y;
                im += g[c] * s.x;
            }
            gg[(int64_t)P * N3 + p] = mk<T>(re * inv, im * inv);
        }
    }
}

// v^{ch} = v1 - div (gg after the inverse transform); xc3[k] = sum_ch C[k][ch] v^{ch}
template <typename T>
__global__ void __launch_bounds__(RB) k_gga_combine(int N3, PotCoefT<T> cf, const T* __restrict__ v4,
                                                    const c2<T>* __restrict__ gg, T* __restrict__ xc3) {
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        const c2<T> d0 = gg[p], d1 = gg[N3 + p];
        const T v[4] = {v4[p] - d0.x, v4[N3 + p] - d0.y, v4[2 * N3 + p] - d1.x, v4[3 * N3 + p] - d1.y};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T s = 0;
#pragma unroll
            for (int ch = 0; ch < 4; ++ch) s += cf.C[k][ch] * v[ch];
            xc3[(int64_t)k * N3 + p] = s;
        }
    }
}

// After the forward transform: rho(G) = grid / N^3; E_H partial
// sum 4 pi |rho(G)|^2 / G^2; grid <- V_H(G) = 4 pi rho(G) / G^2 (G = 0 -> 0).
template <typename T>
__global__ void __launch_bounds__(RB) k_hartree_G(int N, T inv, T fpb, c2<T>* __restrict__ grid,
                                                  double* __restrict__ part) {
    // inv = 1 / N^3, fpb = 4 pi / b^2 with b = 2 pi / L (from the host)
    __shared__ double sh[RB];
    const int N3 = N * N * N;
    T eh = 0;
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        const int z = p % N, y = (p / N) % N, x = p / (N * N);
        const int fx = signed_freq(x, N), fy = signed_freq(y, N), fz = signed_freq(z, N);
        const int m2 = fx * fx + fy * fy + fz * fz;
        const c2<T> gv = grid[p];
        const T rx = gv.x * inv, ry = gv.y * inv;
        c2<T> o = mk<T>(T(0), T(0));
        if (m2 > 0) {
            const T k = fpb / T(m2);              // 4 pi / G^2
            eh += k * (rx * rx + ry * ry);
            o = mk<T>(k * rx, k * ry);
        }
        grid[p] = o;
    }
    const double deh = block_sum_t<T>(eh, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = deh;
}

// V^k = w_k (V_loc + V_H) + xc3[k]; partial sums <a|V^c|a>, <b|V^c|b> (rho_a, rho_b).
template <typename T>
__global__ void __launch_bounds__(RB) k_pot_class(int N3, const T* __restrict__ vloc,
                                                  const c2<T>* __restrict__ vh, const T* __restrict__ xc3,
                                                  const typename DensAcc<T>::S* __restrict__ rho3, PotCoef cf,
                                                  T* __restrict__ Vk,
                                                  double* __restrict__ Vk64, double* __restrict__ part) {
    __shared__ double sh[RB];
    T ea = 0, eb = 0;
    const T w0 = T(cf.w[0]), w1 = T(cf.w[1]), w2 = T(cf.w[2]);
    for (int p = blockIdx.x * RB + threadIdx.x; p < N3; p += gridDim.x * RB) {
        const T v0 = vloc[p] + vh[p].x;
        const T vc = w0 * v0 + xc3[p];
        const T va = w1 * v0 + xc3[N3 + p];
        const T vb = w2 * v0 + xc3[2 * N3 + p];
        Vk[p] = vc;
        Vk[N3 + p] = va;
        Vk[2 * N3 + p] = vb;
        if (Vk64) {
            Vk64[p] = double(vc);
            Vk64[N3 + p] = double(va);
            Vk64[2 * N3 + p] = double(vb);
        }
        ea += vc * T(DensAcc<T>::value(rho3[N3 + p]));
        eb += vc * T(DensAcc<T>::value(rho3[2 * N3 + p]));
    }
    const double dea = block_sum_t<T>(ea, sh);
    const double deb = block_sum_t<T>(eb, sh);
    if (threadIdx.x == 0) {
        part[blockIdx.x * 2 + 0] = dea;
        part[blockIdx.x * 2 + 1] = deb;
    }
}

// Sum per-block partials in a fixed order: out[q] = scale[q] * sum_b part[b * nq + q];
// one block per quantity.
__global__ void __launch_bounds__(RB) k_partials_final(int nblocks, int nq, const double* __restrict__ part,
                                                       double* __restrict__ out, double s0, double s1, double s2,
                                                       double s3) {
    __shared__ double sh[RB];
    const int q = blockIdx.x;
    double s = 0;
    for (int b = threadIdx.x; b < nblocks; b += RB) s += part[b * nq + q];
    s = block_sum(s, sh);
    const double sc[4] = {s0, s1, s2, s3};
    if (threadIdx.x == 0) out[q] = s * sc[q];
}

// ------------------------------------------------------------------ PCG pointwise
// K g: K(G, n) = -(2 / X_n) tpa(|G|^2 / X_n), X_n = 1.5 sum g2 |g|^2 / sum |g|^2.
template <typename T>
__global__ void k_precond(int npw, const c2<T>* __restrict__ gI, int64_t ld, const T* __restrict__ g2h,
                          const double* __restrict__ sums /* [4 nb]: |g|^2, g2 |g|^2, then 1/X, -2/X */,
                          int nb, c2<T>* __restrict__ out, int64_t ldo) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (g >= npw) return;
    // the band's coefficients come from the column-sum kernel (FP64 divisions
    // once per band, not once per block)
    const T X0 = T(sums[2 * nb + 2 * n]), X1 = T(sums[2 * nb + 2 * n + 1]);
    const T x = T(2) * g2h[g] * X0;
    const T num = T(27) + x * (T(18) + x * (T(12) + T(8) * x));
    const T K = X1 * num / (num + T(16) * x * x * x * x);
    const c2<T> a = gI[(int64_t)n * ld + g];
    out[(int64_t)n * ldo + g] = mk<T>(K * a.x, K * a.y);
}

// out = x + coef[0] * y  (coef on the device; y may be null -> copy)
template <typename T>
__global__ void k_axpy(int npw, const c2<T>* __restrict__ x, int64_t ldx, const c2<T>* __restrict__ y, int64_t ldy,
                       const double* __restrict__ coef, double csign, c2<T>* __restrict__ out, int64_t ldo) {
    // the coefficient is formed once per block (FP64 arithmetic per element is slow on this part)
    __shared__ T cs;
    if (threadIdx.x == 0 && y) cs = T(csign * coef[0]);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (g >= npw) return;
    c2<T> a = x[(int64_t)n * ldx + g];
    if (y) {
        const T c = cs;
        const c2<T> b = y[(int64_t)n * ldy + g];
        a.x += c * b.x;
        a.y += c * b.y;
    }
    out[(int64_t)n * ldo + g] = a;
}

// ------------------------------------------------------------------ host wrappers
void vloc_setup(int N, double L, int natoms, const double* atoms_dev, double2* grid, double* vloc,
                const double2* tw64, cudaStream_t st) {
    const int64_t N3 = (int64_t)N * N * N;
    const double omega = L * L * L;
    roks::count_launch(), k_vloc_G<<<(N3 + 255) / 256, 256, 0, st>>>(N, 2.0 * kPi / L, omega, natoms, atoms_dev, grid);
    grid_fft3<double>(N, tw64, grid, +1, st);
    roks::count_launch(), k_real_part<<<(N3 + 255) / 256, 256, 0, st>>>(N3, grid, vloc);
}

template <typename T>
void projectors_setup(int npw, int nproj, double L, const int* miller_dev, const double* proj_dev, c2<T>* P,
                      int64_t ldp, cudaStream_t st) {
    if (nproj == 0) return;
    dim3 g((npw + 255) / 256, nproj);
    roks::count_launch(), k_projectors<T><<<g, 256, 0, st>>>(npw, nproj, 2.0 * kPi / L, L * L * L, miller_dev, proj_dev, P, ldp);
}

template <typename T>
void init_orbitals(int npw, int band0, int nbands, const double* u_dev, uint64_t seed, const double* g2, c2<T>* psi,
                   int64_t ld, cudaStream_t st) {
    if (nbands <= 0) return;
    dim3 g((npw + 255) / 256, nbands);
    roks::count_launch(), k_init_orbitals<T><<<g, 256, 0, st>>>(npw, band0, u_dev, seed, g2, psi, ld);
}

template <typename T>
void to_real_type(int64_t n, const double* in, T* out, double scale, cudaStream_t st) {
    roks::count_launch(), k_to_real<T><<<(n + 255) / 256, 256, 0, st>>>(n, in, out, scale);
}

void apply_DQ(int nproj, int nb, const double2* B, const int* blk_off, const int* blk_n, const double* Drow,
              const double* Qrow, const double* wband, double2* DB, double2* QB, cudaStream_t st) {
    if (nproj == 0) return;
    roks::count_launch(), k_apply_DQ<<<(nproj * nb + 127) / 128, 128, 0, st>>>(nproj, nb, B, blk_off, blk_n, Drow, Qrow, wband, DB, QB);
}

void band_quadratic(int nproj, int nb, const double2* B, const double2* DB, double* out, cudaStream_t st) {
    if (nproj == 0) {
        cudaMemsetAsync(out, 0, sizeof(double) * nb, st);
        return;
    }
    roks::count_launch(), k_band_quadratic<<<nb, RB, 0, st>>>(nproj, nb, B, DB, out);
}

// Grid densities of the element type's storage -> FP64 (API output)
template <typename T>
__global__ void k_density_to_f64(int64_t n, const typename DensAcc<T>::S* __restrict__ in, double* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if constexpr (sizeof(T) == 4) out[i] = double(in[i].x) + double(in[i].y);
    else out[i] = in[i];
}

template <typename T>
void density_to_f64(int64_t n, const double* rho3, double* out, cudaStream_t st) {
    using DS = typename DensAcc<T>::S;
    roks::count_launch(), k_density_to_f64<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        n, reinterpret_cast<const DS*>(rho3), out);
}
template void density_to_f64<float>(int64_t, const double*, double*, cudaStream_t);
template void density_to_f64<double>(int64_t, const double*, double*, cudaStream_t);

constexpr int kPotBlocks = 512;

template <typename T>
void potentials(int N, double L, const double* rho3, const T* vloc, const PotCoef& cf, c2<T>* grid,
                T* xc3, const c2<T>* tw, T* Vk, double* Vk64, double* part, double* out6,
                cudaStream_t st, bool energies_only, const GgaWork* gga) {
    // out6: [E_x^M, E_x^T, E_loc, E_H, <a|V^c|a>, <b|V^c|b>]; energies_only
    // stops after E_H (out6[4..5] and Vk are left as they were)
    const int N3 = N * N * N;
    const double dvol = L * L * L / double(N3);
    const double c6 = std::cbrt(6.0 / kPi);                 // (6 / pi)^{1/3}
    const double b = 2.0 * kPi / L;
    using DS = typename DensAcc<T>::S;
    const DS* r3 = reinterpret_cast<const DS*>(rho3);
    PotCoefT<T> ct;
    for (int k = 0; k < 3; ++k)
        for (int ch = 0; ch < 4; ++ch) {
            ct.f[k][ch] = T(cf.f[k][ch]);
            ct.C[k][ch] = T(cf.C[k][ch]);
        }
    ct.xscale = T(cf.xscale);
    c2<T>* gg = gga ? static_cast<c2<T>*>(gga->gg) : nullptr;
    c2<T>* dd = gga ? static_cast<c2<T>*>(gga->dd) : nullptr;
    if (!gga) {
        roks::count_launch(), k_pot_xc<T><<<kPotBlocks, RB, 0, st>>>(N3, r3, vloc, ct, T(c6), T(0.75 * c6), grid,
                                                                      xc3, part);
    } else {
        // PBE exchange: the channels' gradients by two forward and six
        // inverse grid transforms, then the pointwise energy, de/drho and flux
        const T inv = T(1.0 / double(N3));
        roks::count_launch(), k_gga_pack<T><<<kPotBlocks, RB, 0, st>>>(N3, r3, vloc, ct, grid, gg, part);
        grid_fft3_batched<T>(N, tw, gg, 2, (int64_t)N3, -1, st);
        roks::count_launch(), k_gga_grad<T><<<kPotBlocks, RB, 0, st>>>(N, T(b), inv, gg, dd);
        grid_fft3_batched<T>(N, tw, dd, 6, (int64_t)N3, +1, st);
        roks::count_launch(), k_gga_point<T><<<kPotBlocks, RB, 0, st>>>(
                                  N3, r3, ct, T(0.75 * c6), T(std::pow(6.0 * kPi * kPi, 2.0 / 3.0)), T(gga->mu),
                                  T(gga->kappa), T(gga->rho_min), dd, static_cast<T*>(gga->v4), part);
    }
    roks::count_launch(), k_partials_final<<<4, RB, 0, st>>>(kPotBlocks, 4, part, out6, dvol, dvol, dvol, 0.0);
    grid_fft3<T>(N, tw, grid, -1, st);
    roks::count_launch(), k_hartree_G<T><<<kPotBlocks, RB, 0, st>>>(N, T(1.0 / double(N3)), T(4.0 * kPi / (b * b)),
                                                                     grid, part);
    roks::count_launch(), k_partials_final<<<1, RB, 0, st>>>(kPotBlocks, 1, part, out6 + 3, 0.5 * L * L * L, 0, 0, 0);
    if (energies_only) return;
    if (gga) {
        // the divergence of the fluxes: six forward transforms, i G . flux,
        // two inverse transforms
        const T inv = T(1.0 / double(N3));
        grid_fft3_batched<T>(N, tw, dd, 6, (int64_t)N3, -1, st);
        roks::count_launch(), k_gga_div<T><<<kPotBlocks, RB, 0, st>>>(N, T(b), inv, dd, gg);
        grid_fft3_batched<T>(N, tw, gg, 2, (int64_t)N3, +1, st);
        roks::count_launch(), k_gga_combine<T><<<kPotBlocks, RB, 0, st>>>(N3, ct, static_cast<const T*>(gga->v4),
                                                                           gg, xc3);
    }
    grid_fft3<T>(N, tw, grid, +1, st);
    roks::count_launch(), k_pot_class<T><<<kPotBlocks, RB, 0, st>>>(N3, vloc, grid, xc3, r3, cf, Vk, Vk64, part);
    roks::count_launch(), k_partials_final<<<2, RB, 0, st>>>(kPotBlocks, 2, part, out6 + 4, dvol, dvol, 0, 0);
}

size_t potentials_part_elems() { return (size_t)kPotBlocks * 4; }

template <typename T>
void precondition(int npw, int nb, const c2<T>* gI, int64_t ld, const T* g2h, const double* sums, c2<T>* out,
                  int64_t ldo, cudaStream_t st) {
    dim3 g((npw + 255) / 256, nb);
    roks::count_launch(), k_precond<T><<<g, 256, 0, st>>>(npw, gI, ld, g2h, sums, nb, out, ldo);
}

template <typename T>
void axpy(int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy, const double* coef,
          double csign, c2<T>* out, int64_t ldo, cudaStream_t st) {
    dim3 g((npw + 255) / 256, nb);
    roks::count_launch(), k_axpy<T><<<g, 256, 0, st>>>(npw, x, ldx, y, ldy, coef, csign, out, ldo);
}

#define ROKS_INSTANTIATE_GRID(T)                                                                               \
    template void projectors_setup<T>(int, int, double, const int*, const double*, c2<T>*, int64_t,            \
                                      cudaStream_t);                                                           \
    template void init_orbitals<T>(int, int, int, const double*, uint64_t, const double*, c2<T>*, int64_t,     \
                                   cudaStream_t);                                                              \
    template void to_real_type<T>(int64_t, const double*, T*, double, cudaStream_t);                           \
    template void column_sums<T>(int, int, int, const c2<T>*, int64_t, const c2<T>*, int64_t, const T*,       \
                                 double*, double*, cudaStream_t);                                              \
    template void column_total<T>(int, int, int, const c2<T>*, int64_t, const c2<T>*, int64_t, const T*,      \
                                  double*, double*, double, cudaStream_t);                                     \
    template void potentials<T>(int, double, const double*, const T*, const PotCoef&, c2<T>*, T*,             \
                                const c2<T>*, T*, double*, double*, double*, cudaStream_t, bool,              \
                                const GgaWork*);                                                               \
    template void precondition<T>(int, int, const c2<T>*, int64_t, const T*, const double*, c2<T>*,           \
                                  int64_t, cudaStream_t);                                                      \
    template void axpy<T>(int, int, const c2<T>*, int64_t, const c2<T>*, int64_t, const double*, double,      \
                          c2<T>*, int64_t, cudaStream_t);

ROKS_INSTANTIATE_GRID(float)
ROKS_INSTANTIATE_GRID(double)

}  // namespace roks
