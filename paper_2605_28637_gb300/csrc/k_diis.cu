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

// Row `ns` of B from one pass over the error vectors: block (bx, n) takes
// kGramPer x 256 coefficients of band n, sums Re <e_new|e_k> for every pair
// of the window (per-thread sums in the element type over a few terms, block
// sums in FP64) into part[k * nblocks + block].
constexpr int kGramPer = 8;
template <typename T>
__global__ void __launch_bounds__(256) k_diis_gram(int npw, const c2<T>* __restrict__ enew,
                                                   const c2<T>* __restrict__ ering, int64_t blk, int64_t ld,
                                                   DiisOrder ord, double* __restrict__ part) {
    __shared__ double sh[kDiisMax][8];
    const int n = blockIdx.y;
    const int g0 = blockIdx.x * kGramPer * 256;
    const int g1 = min(npw, g0 + kGramPer * 256);
    T acc[kDiisMax];
#pragma unroll
    for (int k = 0; k < kDiisMax; ++k) acc[k] = T(0);
    const int64_t col = (int64_t)n * ld;
    for (int g = g0 + threadIdx.x; g < g1; g += 256) {
        const c2<T> a = enew[col + g];
#pragma unroll
        for (int k = 0; k < kDiisMax; ++k) {
            if (k < ord.n) {
                const c2<T> b = ering[ord.slot[k] * blk + col + g];
                acc[k] += a.x * b.x + a.y * b.y;
            }
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < kDiisMax; ++k) {
        if (k < ord.n) {
            double v = double(acc[k]);
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) sh[k][warp] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x < ord.n) {
        const int k = threadIdx.x;
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += sh[k][w];
        const int nblocks = gridDim.x * gridDim.y;
        part[(int64_t)k * nblocks + blockIdx.y * gridDim.x + blockIdx.x] = v;
    }
}

// Warp k sums the partials of pair k in a fixed order into B[ns][slot_k].
__global__ void k_diis_gram_final(int nblocks, const double* __restrict__ part, DiisOrder ord,
                                  DiisState* __restrict__ s) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= ord.n) return;
    double v = 0.0;
    for (int i = lane; i < nblocks; i += 32) v += part[(int64_t)k * nblocks + i];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int ns = ord.slot[ord.n - 1];
    if (lane == 0) s->B[ns * kDiisMax + ord.slot[k]] = v;
}

// One warp: B and the residual's band norms are loaded in parallel, then one
// thread completes the newest row symmetrically, tests the windows on the
// normalised Gram matrix and solves for the coefficients of the accepted one
// (the loads dominate a single thread's time: the arithmetic is a few
// hundred FP64 operations).
__global__ void k_diis_solve(DiisState* __restrict__ s, DiisOrder ord, double tol, const double* __restrict__ rn,
                             int nb) {
    __shared__ double Bs[kDiisMax * kDiisMax];
    const int lane = threadIdx.x;
    for (int i = lane; i < kDiisMax * kDiisMax; i += 32) Bs[i] = s->B[i];
    double r = 0.0;
    for (int i = lane; i < nb; i += 32) r += rn[i];
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    __syncwarp();
    if (lane != 0) return;
    s->rnorm2 = r;
    const int n = ord.n;
    const int ns = ord.slot[n - 1];
    for (int k = 0; k < n; ++k) {
        const double v = Bs[ns * kDiisMax + ord.slot[k]];
        Bs[ord.slot[k] * kDiisMax + ns] = v;
        s->B[ord.slot[k] * kDiisMax + ns] = v;
    }
    s->h = diis_window_coefficients(Bs, ord, tol, s->d, s->slot);
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

void diis_solve(DiisState* s, const DiisOrder& ord, double tol, const double* rn, int nb, cudaStream_t st) {
    count_launch(), k_diis_solve<<<1, 32, 0, st>>>(s, ord, tol, rn, nb);
}

int diis_gram_blocks(int npw, int nb) { return ((npw + kGramPer * 256 - 1) / (kGramPer * 256)) * nb; }

template <typename T>
void diis_gram(int npw, int nb, const c2<T>* enew, const c2<T>* ering, int64_t blk, int64_t ld,
               const DiisOrder& ord, double* part, DiisState* s, cudaStream_t st) {
    const dim3 g((npw + kGramPer * 256 - 1) / (kGramPer * 256), nb);
    count_launch(), k_diis_gram<T><<<g, 256, 0, st>>>(npw, enew, ering, blk, ld, ord, part);
    count_launch(), k_diis_gram_final<<<1, 32 * kDiisMax, 0, st>>>(int(g.x * g.y), part, ord, s);
}

template <typename T>
void diis_combine(int npw, int nb, const DiisState* s, const c2<T>* psi_ring, const c2<T>* e_ring, int64_t blk,
                  int64_t ld, double tau, c2<T>* out, int64_t ldo, cudaStream_t st) {
    const dim3 g((npw + 255) / 256, nb);
    count_launch(), k_diis_combine<T><<<g, 256, 0, st>>>(npw, s, psi_ring, e_ring, blk, ld, tau, out, ldo);
}

template void diis_gram<float>(int, int, const c2<float>*, const c2<float>*, int64_t, int64_t, const DiisOrder&,
                               double*, DiisState*, cudaStream_t);
template void diis_gram<double>(int, int, const c2<double>*, const c2<double>*, int64_t, int64_t, const DiisOrder&,
                                double*, DiisState*, cudaStream_t);
template void diis_combine<float>(int, int, const DiisState*, const c2<float>*, const c2<float>*, int64_t, int64_t,
                                  double, c2<float>*, int64_t, cudaStream_t);
template void diis_combine<double>(int, int, const DiisState*, const c2<double>*, const c2<double>*, int64_t,
                                   int64_t, double, c2<double>*, int64_t, cudaStream_t);

}  // namespace roks
