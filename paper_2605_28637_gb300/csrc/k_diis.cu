// k_diis.cu -- kernels of the DIIS solver on the ROKS residual (Sec. II A):
// the multipliers of the residual with the coupling coefficients lambda,
// the extrapolation coefficients of the history window, and the
// extrapolated orbitals.  The band-block products, the preconditioner and the
// reductions reuse the PCG path's kernels.
#include <cmath>

#include "roks_diis.cuh"

namespace roks {

// Lambda_mn = theta_mn - lambda_mn (theta_mn - conj theta_nm).  With every
// lambda = 1/2 this is gamma of Eq. 11 and the residual is the gradient.
__global__ void k_diis_multipliers(int nb, const double2* __restrict__ Th, int ia, int ib, double lab, double lba,
                                   double2* __restrict__ Lam) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb * nb; i += gridDim.x * blockDim.x) {
        const int m = i % nb, n = i / nb;
        double lam = 0.5;
        if (m == ia && n == ib) lam = lab;
        if (m == ib && n == ia) lam = lba;
        const double2 t = Th[(int64_t)n * nb + m];
        const double2 u = Th[(int64_t)m * nb + n];   // theta_nm
        // theta_mn - conj theta_nm
        const double dx = t.x - u.x, dy = t.y + u.y;
        Lam[(int64_t)n * nb + m] = make_double2(t.x - lam * dx, t.y - lam * dy);
    }
}

// One thread: symmetric completion of the newest row of B, the window test
// on the normalised Gram matrix and the coefficients of the accepted window.
__global__ void k_diis_solve(DiisState* __restrict__ s, DiisOrder ord, double tol) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = ord.n;
    const int ns = ord.slot[n - 1];
    for (int k = 0; k < n; ++k) s->B[ord.slot[k] * kDiisMax + ns] = s->B[ns * kDiisMax + ord.slot[k]];
    for (int h = n; h >= 2; --h) {
        const int o = n - h;
        double q[kDiisMax], L[kDiisMax][kDiisMax];
        bool ok = true;
        for (int j = 0; j < h && ok; ++j) {
            const double bjj = s->B[ord.slot[o + j] * kDiisMax + ord.slot[o + j]];
            ok = bjj > 0.0 && isfinite(bjj);
            q[j] = ok ? 1.0 / sqrt(bjj) : 0.0;
        }
        // Cholesky of Bn = D^-1/2 B D^-1/2, pivots L_jj^2 >= tol
        for (int j = 0; j < h && ok; ++j) {
            for (int i = j; i < h; ++i) {
                double v = s->B[ord.slot[o + i] * kDiisMax + ord.slot[o + j]] * q[i] * q[j];
                for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(v >= tol)) {
                        ok = false;
                        break;
                    }
                    L[j][j] = sqrt(v);
                } else {
                    L[i][j] = v / L[j][j];
                }
            }
        }
        if (!ok) continue;
        // Bn z = D^-1/2 1, y = D^-1/2 z = B^-1 1, d = y / sum y
        double w[kDiisMax];
        for (int i = 0; i < h; ++i) {
            double v = q[i];
            for (int k = 0; k < i; ++k) v -= L[i][k] * w[k];
            w[i] = v / L[i][i];
        }
        for (int i = h - 1; i >= 0; --i) {
            double v = w[i];
            for (int k = i + 1; k < h; ++k) v -= L[k][i] * w[k];
            w[i] = v / L[i][i];
        }
        double sum = 0.0;
        for (int i = 0; i < h; ++i) {
            w[i] *= q[i];
            sum += w[i];
        }
        if (!(sum != 0.0 && isfinite(sum))) continue;
        for (int i = 0; i < h; ++i) {
            s->d[i] = w[i] / sum;
            s->slot[i] = ord.slot[o + i];
        }
        s->h = h;
        return;
    }
    // the newest pair alone: d = 1 (unless its residual is not finite)
    const double bnn = s->B[ns * kDiisMax + ns];
    s->d[0] = 1.0;
    s->slot[0] = ns;
    s->h = isfinite(bnn) ? 1 : 0;
}

template <typename T>
__global__ void k_diis_combine(int npw, const DiisState* __restrict__ s, const c2<T>* __restrict__ psi_ring,
                               const c2<T>* __restrict__ e_ring, int64_t blk, int64_t ld, double tau,
                               c2<T>* __restrict__ out, int64_t ldo) {
    // coefficients in the element type, formed once per block
    __shared__ T cp[kDiisMax], ce[kDiisMax];
    __shared__ int off[kDiisMax];
    __shared__ int hh;
    if (threadIdx.x == 0) hh = s->h;
    if (threadIdx.x < kDiisMax) {
        const int k = threadIdx.x;
        const double d = k < s->h ? s->d[k] : 0.0;
        cp[k] = T(d);
        ce[k] = T(d * tau);
        off[k] = k < s->h ? s->slot[k] : 0;
    }
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = blockIdx.y;
    if (g >= npw) return;
    const int64_t e = (int64_t)n * ld + g;
    c2<T> acc;
    acc.x = T(0);
    acc.y = T(0);
    for (int k = 0; k < hh; ++k) {
        const c2<T> p = psi_ring[off[k] * blk + e];
        const c2<T> r = e_ring[off[k] * blk + e];
        acc.x += cp[k] * p.x + ce[k] * r.x;
        acc.y += cp[k] * p.y + ce[k] * r.y;
    }
    out[(int64_t)n * ldo + g] = acc;
}

// ------------------------------------------------------------------ host wrappers
void diis_multipliers(int nb, const double2* Theta, int ia, int ib, double lab, double lba, double2* Lam,
                      cudaStream_t st) {
    const int blocks = (nb * nb + 255) / 256;
    count_launch(), k_diis_multipliers<<<blocks, 256, 0, st>>>(nb, Theta, ia, ib, lab, lba, Lam);
}

void diis_solve(DiisState* s, const DiisOrder& ord, double tol, cudaStream_t st) {
    count_launch(), k_diis_solve<<<1, 32, 0, st>>>(s, ord, tol);
}

template <typename T>
void diis_combine(int npw, int nb, const DiisState* s, const c2<T>* psi_ring, const c2<T>* e_ring, int64_t blk,
                  int64_t ld, double tau, c2<T>* out, int64_t ldo, cudaStream_t st) {
    const dim3 g((npw + 255) / 256, nb);
    count_launch(), k_diis_combine<T><<<g, 256, 0, st>>>(npw, s, psi_ring, e_ring, blk, ld, tau, out, ldo);
}

template void diis_combine<float>(int, int, const DiisState*, const c2<float>*, const c2<float>*, int64_t, int64_t,
                                  double, c2<float>*, int64_t, cudaStream_t);
template void diis_combine<double>(int, int, const DiisState*, const c2<double>*, const c2<double>*, int64_t,
                                   int64_t, double, c2<double>*, int64_t, cudaStream_t);

}  // namespace roks
