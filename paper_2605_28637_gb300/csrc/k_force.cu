// k_force.cu -- kernels of the ROKS forces (Sec. II B): the Hellmann-Feynman
// terms of the local wells and of the projectors, and the overlap term with
// the constraint multipliers gamma,
//   dE/dR_Inu = Omega sum_G (-i G_nu) v_I(G) e^{-iG.R_I} conj(rho_w(G))
//             + 2 Re sum_{i in I} sum_n conj(dB_inu,n) [w_n (D B)_in - (Q B Gam)_in],
// with B = P^H Psi, dB_nu = (dP_nu)^H Psi, dp_i/dR_nu = -i G_nu p_i and
// Gam_mn = (theta_mn + conj theta_nm)/2 (so that sum_mn gamma_mn <m|dS|n>
// = 2 Re sum_im conj(dB_im) (Q B Gam)_im).  The band-block products and the
// grid transform reuse the PCG path's kernels.
#include <cmath>

#include "roks_force.cuh"

namespace roks {

constexpr double kTwoPi = 6.28318530717958647692;

// e^{-i 2 pi f s_c} for f = signed frequency of grid index x, s_c = R_c / L
// (fractional coordinate, reduced so that the phase is exact to FP64 before
// the conversion to the element type).
template <typename T>
__global__ void k_force_tables(int natoms, int N, double L, const double* __restrict__ atoms,
                               c2<T>* __restrict__ tab) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= natoms * 3 * N) return;
    const int x = idx % N, c = (idx / N) % 3, a = idx / (3 * N);
    const double s = atoms[5 * a + c] / L;
    double t = double(signed_freq(x, N)) * s;
    t -= rint(t);
    double sn, cs;
    sincospi(-2.0 * t, &sn, &cs);
    tab[idx] = mk<T>(T(cs), T(sn));
}

// rho_w(r) = sum_k w_k rho_k(r) into the complex grid (imaginary part zero)
template <typename T>
__global__ void k_force_rho(int N3, const typename DensAcc<T>::S* __restrict__ rho3, T w0, T w1, T w2,
                            c2<T>* __restrict__ grid) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N3; p += gridDim.x * blockDim.x) {
        using DA = DensAcc<T>;
        const T r = w0 * T(DA::value(rho3[p])) + w1 * T(DA::value(rho3[N3 + p])) + w2 * T(DA::value(rho3[2 * N3 + p]));
        grid[p] = mk<T>(r, T(0));
    }
}

// Block (bx, a): partial sums over a slice of the grid of
// f_nu v_a(G) (sin phi rho_re - cos phi rho_im), e^{i phi} = e^{-iG.R_a},
// rho = the unnormalised forward transform of rho_w; Nyquist planes skipped
// (the local potential has none).  part[(a * 3 + nu) * gridDim.x + bx].
template <typename T>
__global__ void __launch_bounds__(256) k_force_loc(int N, const c2<T>* __restrict__ tab, const T* __restrict__ amp,
                                                   const T* __restrict__ w2h, T b2, const c2<T>* __restrict__ rho,
                                                   double* __restrict__ part) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2<T>* t = reinterpret_cast<c2<T>*>(smem_raw);
    const int a = blockIdx.y;
    for (int i = threadIdx.x; i < 3 * N; i += blockDim.x) t[i] = tab[(int64_t)a * 3 * N + i];
    __syncthreads();
    const T A = amp[a], wh = w2h[a];
    const int N3 = N * N * N;
    const int half = N / 2;
    const bool even = (N % 2) == 0;
    T acc0 = T(0), acc1 = T(0), acc2 = T(0);
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < N3; p += gridDim.x * blockDim.x) {
        const int z = p % N, y = (p / N) % N, x = p / (N * N);
        const int fx = signed_freq(x, N), fy = signed_freq(y, N), fz = signed_freq(z, N);
        if (even && (fx == half || fy == half || fz == half)) continue;
        const T g2 = b2 * T(fx * fx + fy * fy + fz * fz);
        const T v = A * exp(-g2 * wh);
        const c2<T> ex = t[x], ey = t[N + y], ez = t[2 * N + z];
        // e = ex ey ez
        const T pr = ex.x * ey.x - ex.y * ey.y, pi = ex.x * ey.y + ex.y * ey.x;
        const T er = pr * ez.x - pi * ez.y, ei = pr * ez.y + pi * ez.x;
        const c2<T> r = rho[p];
        const T core = v * (ei * r.x - er * r.y);
        acc0 += T(fx) * core;
        acc1 += T(fy) * core;
        acc2 += T(fz) * core;
    }
    __shared__ double sh[3][8];
    double v3[3] = {double(acc0), double(acc1), double(acc2)};
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double v = v3[c];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) sh[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[threadIdx.x][w];
        part[((int64_t)a * 3 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
}

// dP_nu[g, i] = -i G_nu(g) P[g, i]
template <typename T>
__global__ void k_force_dP(int npw, const c2<T>* __restrict__ P, int64_t ld, const int* __restrict__ miller, T b,
                           int nu, c2<T>* __restrict__ out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    if (g >= npw) return;
    const T c = b * T(miller[3 * g + nu]);
    const c2<T> p = P[(int64_t)i * ld + g];
    out[(int64_t)i * ld + g] = mk<T>(c * p.y, -c * p.x);
}

// c[nu * nproj + i] = 2 Re sum_n conj(dB_nu[i, n]) (DBw[i, n] - Y[i, n])
__global__ void k_force_nl(int nproj, int nb, const double2* __restrict__ dB, const double2* __restrict__ DBw,
                           const double2* __restrict__ Y, double* __restrict__ c) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 3 * nproj) return;
    const int i = idx % nproj, nu = idx / nproj;
    const double2* d = dB + (int64_t)nu * nproj * nb;
    double s = 0.0;
    for (int n = 0; n < nb; ++n) {
        const int64_t e = (int64_t)n * nproj + i;
        const double2 x = d[e];
        const double zr = DBw[e].x - Y[e].x, zi = DBw[e].y - Y[e].y;
        s += x.x * zr + x.y * zi;
    }
    c[idx] = 2.0 * s;
}

// forces[a * 3 + nu] = -(scale sum_bx part + sum over the projectors of atom a of c)
__global__ void k_force_collect(int natoms, int nproj, int nblk, const int* __restrict__ owner,
                                const double* __restrict__ c, const double* __restrict__ part, double scale,
                                double* __restrict__ forces) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= natoms * 3) return;
    const int a = idx / 3, nu = idx % 3;
    double loc = 0.0;
    for (int k = 0; k < nblk; ++k) loc += part[(int64_t)idx * nblk + k];
    double s = scale * loc;
    for (int i = 0; i < nproj; ++i)
        if (owner[i] == a) s += c[nu * nproj + i];
    forces[idx] = -s;
}

// ------------------------------------------------------------------ host wrappers
template <typename T>
void force_local(int N, double L, int natoms, const double* atoms, const double* rho3, const double* w, const T* amp,
                 const T* w2h, c2<T>* tab, c2<T>* grid, const c2<T>* tw, double* part, cudaStream_t st) {
    const int N3 = N * N * N;
    const double b = kTwoPi / L;
    count_launch(), k_force_tables<T><<<(natoms * 3 * N + 255) / 256, 256, 0, st>>>(natoms, N, L, atoms, tab);
    using DS = typename DensAcc<T>::S;
    count_launch(), k_force_rho<T><<<1024, 256, 0, st>>>(N3, reinterpret_cast<const DS*>(rho3), T(w[0]), T(w[1]),
                                                         T(w[2]), grid);
    grid_fft3<T>(N, tw, grid, -1, st);
    const dim3 g(kForceLocBlocks, natoms);
    count_launch(), k_force_loc<T><<<g, 256, sizeof(c2<T>) * 3 * N, st>>>(N, tab, amp, w2h, T(b * b), grid, part);
}

template <typename T>
void force_dP(int npw, int nproj, const c2<T>* P, int64_t ld, const int* miller, double b, int nu, c2<T>* out,
              cudaStream_t st) {
    const dim3 g((npw + 255) / 256, nproj);
    count_launch(), k_force_dP<T><<<g, 256, 0, st>>>(npw, P, ld, miller, T(b), nu, out);
}

void force_nl(int nproj, int nb, const double2* dB, const double2* DBw, const double2* Y, double* c,
              cudaStream_t st) {
    if (nproj <= 0) return;
    count_launch(), k_force_nl<<<(3 * nproj + 127) / 128, 128, 0, st>>>(nproj, nb, dB, DBw, Y, c);
}

void force_collect(int natoms, int nproj, const int* owner, const double* c, const double* part, double scale,
                   double* forces, cudaStream_t st) {
    count_launch(), k_force_collect<<<(natoms * 3 + 127) / 128, 128, 0, st>>>(natoms, nproj, kForceLocBlocks, owner,
                                                                               c, part, scale, forces);
}

#define ROKS_INSTANTIATE_FORCE(T)                                                                              \
    template void force_local<T>(int, double, int, const double*, const double*, const double*, const T*,      \
                                 const T*, c2<T>*, c2<T>*, const c2<T>*, double*, cudaStream_t);               \
    template void force_dP<T>(int, int, const c2<T>*, int64_t, const int*, double, int, c2<T>*, cudaStream_t);
ROKS_INSTANTIATE_FORCE(float)
ROKS_INSTANTIATE_FORCE(double)

}  // namespace roks
