// k_exx.cu -- exact exchange with a spherically truncated Coulomb kernel (the
// screened-hybrid workload): pair densities rho_jn = psi_j^* psi_n on the
// full grid, W_jn = sum_G v(G) rho_jn(G) e^{iGr}, the exchange field
// X_n = -alpha Omega^{1/2} sum_j w(k_n, k_j) psi_j W_jn that the x-stage apply
// adds next to V psi, and the pair integrals K_jn = Omega sum_G v |rho_jn(G)|^2.
// Pairs j <= n are used once: W_nj = conj(W_jn).  The grid work of a batch
// of pairs (k_exx_grid.cuh) fuses the pointwise steps into the transforms.
#include "roks_exx.cuh"

namespace roks {

constexpr double kPiX = 3.14159265358979323846;

// v(G) / N^3 on the grid: 4 pi (1 - cos(|G| Rc)) / G^2, v(0) = 2 pi Rc^2
// (spherical truncation); with bare != 0, 4 pi / G^2 and v(0) = 0.
template <typename T>
__global__ void k_exx_kernel(int N, double b, double Rc, int bare, T* __restrict__ vG) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N3 = (int64_t)N * N * N;
    if (p >= N3) return;
    const int z = p % N, y = (p / N) % N, x = p / ((int64_t)N * N);
    const int fx = signed_freq(x, N), fy = signed_freq(y, N), fz = signed_freq(z, N);
    const double g2 = b * b * double(fx * fx + fy * fy + fz * fz);
    double v;
    if (g2 > 0) {
        const double g = sqrt(g2);
        v = bare ? 4.0 * kPiX / g2 : 4.0 * kPiX * (1.0 - cos(g * Rc)) / g2;
    } else {
        v = bare ? 0.0 : 2.0 * kPiX * Rc * Rc;
    }
    vG[p] = T(v / double(N3));
}

// K_pair = (Omega / N^3) sum of the block partials; fills both triangles of Kmat.
__global__ void k_exx_pair_sum(int np, int nblk, const double* __restrict__ part, const int* __restrict__ pj,
                               const int* __restrict__ pn, int p0, double scale, int nb, double* __restrict__ Kmat) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= np) return;
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s += part[(int64_t)b * nblk + k];
    s *= scale;
    const int j = pj[p0 + b], n = pn[p0 + b];
    Kmat[(int64_t)n * nb + j] = s;
    Kmat[(int64_t)j * nb + n] = s;
}

// hf2[L] = -1/2 sum_ij (sum_sigma f_i^{sigma L} f_j^{sigma L}) K_ij, L = M, T.
__global__ void k_exx_energy(int nb, const double* __restrict__ Kmat, ExxCoef cf, double* __restrict__ hf2) {
    __shared__ double sM[256], sT[256];
    double eM = 0, eT = 0;
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const int i = idx % nb, j = idx / nb;
        const int ki = i < cf.n_closed ? 0 : i - cf.n_closed + 1;
        const int kj = j < cf.n_closed ? 0 : j - cf.n_closed + 1;
        const double k = Kmat[idx];
        eM += cf.fM[ki][kj] * k;
        eT += cf.fT[ki][kj] * k;
    }
    sM[threadIdx.x] = eM;
    sT[threadIdx.x] = eT;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sM[threadIdx.x] += sM[threadIdx.x + s];
            sT[threadIdx.x] += sT[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        hf2[0] = -0.5 * sM[0];
        hf2[1] = -0.5 * sT[0];
    }
}

// Exchange part of <m|F^c|m> for the open bands: -alpha sum_j wx(c, k_j) K_jm.
__global__ void k_exx_open_diag(int nb, const double* __restrict__ Kmat, ExxCoef cf, double* __restrict__ out2) {
    const int o = threadIdx.x;
    if (o >= 2) return;
    const int m = cf.n_closed + o;
    if (m >= nb) {
        out2[o] = 0.0;
        return;
    }
    double s = 0.0;
    for (int j = 0; j < nb; ++j) {
        const int kj = j < cf.n_closed ? 0 : j - cf.n_closed + 1;
        s += cf.wxc[kj] * Kmat[(int64_t)m * nb + j];
    }
    out2[o] = -cf.alpha * s;
}

// ------------------------------------------------------------------ host side
template <typename T>
void exx_setup_kernel(int N, double L, int bare, T* vG, cudaStream_t st) {
    const int64_t N3 = (int64_t)N * N * N;
    const double Rc = cbrt(3.0 * L * L * L / (4.0 * kPiX));
    roks::count_launch(), k_exx_kernel<T><<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(N, 2.0 * kPiX / L, Rc, bare,
                                                                                        vG);
}

template <typename T>
void exx_pairs(const ExxArgs<T>& a, bool want_field, cudaStream_t st) {
    const int64_t N3 = (int64_t)a.N * a.N * a.N;
    const int nblk = kExxBlocks;
    const double omega = a.L * a.L * a.L;
    if (want_field) cudaMemsetAsync(a.X, 0, sizeof(c2<T>) * N3 * a.nb, st);
    for (int p0 = 0; p0 < a.npairs; p0 += a.batch) {
        const int np = a.npairs - p0 < a.batch ? a.npairs - p0 : a.batch;
        exx_batch_grid<T>(a, p0, np, want_field, st);
        roks::count_launch(), k_exx_pair_sum<<<(np + 127) / 128, 128, 0, st>>>(np, nblk, a.part, a.pj, a.pn, p0,
                                                                              omega / double(N3), a.nb, a.Kmat);
    }
    roks::count_launch(), k_exx_energy<<<1, 256, 0, st>>>(a.nb, a.Kmat, a.cf, a.hf2);
    roks::count_launch(), k_exx_open_diag<<<1, 32, 0, st>>>(a.nb, a.Kmat, a.cf, a.open_diag);
}

template void exx_setup_kernel<float>(int, double, int, float*, cudaStream_t);
template void exx_setup_kernel<double>(int, double, int, double*, cudaStream_t);
template void exx_pairs<float>(const ExxArgs<float>&, bool, cudaStream_t);
template void exx_pairs<double>(const ExxArgs<double>&, bool, cudaStream_t);

}  // namespace roks
