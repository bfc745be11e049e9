// k_exx.cu -- exact exchange with a spherically truncated Coulomb kernel (the
// screened-hybrid workload): pair densities rho_jn = psi_j^* psi_n on the
// full grid, W_jn = sum_G v(G) rho_jn(G) e^{iGr}, the exchange field
// X_n = -alpha Omega^{1/2} sum_j w(k_n, k_j) psi_j W_jn that the x-stage apply
// adds next to V psi, and the pair integrals K_jn = Omega sum_G v |rho_jn(G)|^2.
// Pairs j <= n are used once: W_nj = conj(W_jn).
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

template <typename T>
__global__ void k_exx_pair_density(int64_t N3, const c2<T>* __restrict__ Phi, const int* __restrict__ pj,
                                   const int* __restrict__ pn, int p0, c2<T>* __restrict__ out) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int b = blockIdx.y;
    if (p >= N3) return;
    const int j = pj[p0 + b], n = pn[p0 + b];
    const c2<T> a = Phi[(int64_t)j * N3 + p], c = Phi[(int64_t)n * N3 + p];
    out[(int64_t)b * N3 + p] = cmulc(a, c);
}

// data <- data * v(G)/N^3 and partial sums of (v/N^3) |data|^2 per pair and block.
constexpr int XB = 256;
template <typename T>
__global__ void __launch_bounds__(XB) k_exx_mult(int64_t N3, const T* __restrict__ vG, c2<T>* __restrict__ data,
                                                 double* __restrict__ part) {
    __shared__ double sh[XB];
    const int b = blockIdx.y;
    c2<T>* d = data + (int64_t)b * N3;
    T acc = 0;
    for (int64_t p = (int64_t)blockIdx.x * XB + threadIdx.x; p < N3; p += (int64_t)gridDim.x * XB) {
        const c2<T> v = d[p];
        const T w = vG[p];
        acc += w * (v.x * v.x + v.y * v.y);
        d[p] = mk<T>(v.x * w, v.y * w);
    }
    sh[threadIdx.x] = double(acc);
    __syncthreads();
    for (int s = XB / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)b * gridDim.x + blockIdx.x] = sh[0];
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
        dim3 gp((unsigned)((N3 + 255) / 256), np);
        roks::count_launch(), k_exx_pair_density<T><<<gp, 256, 0, st>>>(N3, a.Phi, a.pj, a.pn, p0, a.buf);
        grid_fft3_batched<T>(a.N, a.tw, a.buf, np, N3, -1, st);
        dim3 gm(nblk, np);
        roks::count_launch(), k_exx_mult<T><<<gm, XB, 0, st>>>(N3, a.vG, a.buf, a.part);
        roks::count_launch(), k_exx_pair_sum<<<(np + 127) / 128, 128, 0, st>>>(np, nblk, a.part, a.pj, a.pn, p0,
                                                                              omega / double(N3), a.nb, a.Kmat);
        if (want_field) {
            grid_fft3_batched<T>(a.N, a.tw, a.buf, np, N3, +1, st);
            roks::count_launch(), k_exx_accumulate<T><<<(unsigned)((N3 + 255) / 256), 256, 0, st>>>(
                N3, a.Phi, a.buf, a.pj, a.pn, p0, np, a.cf, a.X);
        }
    }
    roks::count_launch(), k_exx_energy<<<1, 256, 0, st>>>(a.nb, a.Kmat, a.cf, a.hf2);
    roks::count_launch(), k_exx_open_diag<<<1, 32, 0, st>>>(a.nb, a.Kmat, a.cf, a.open_diag);
}

template void exx_setup_kernel<float>(int, double, int, float*, cudaStream_t);
template void exx_setup_kernel<double>(int, double, int, double*, cudaStream_t);
template void exx_pairs<float>(const ExxArgs<float>&, bool, cudaStream_t);
template void exx_pairs<double>(const ExxArgs<double>&, bool, cudaStream_t);

}  // namespace roks
