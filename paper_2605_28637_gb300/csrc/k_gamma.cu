// k_gamma.cu -- the Gamma-point form of the band path (the paper samples the
// Brillouin zone at Gamma alone, Sec. III): real orbitals on the half sphere
// of plane waves, two of them packed into one complex transform.
//
// A real orbital has c(-G) = conj c(G), so the half sphere (G = 0 and the
// Miller triples after it in the basis order) carries all of it.  The basis
// is sorted by (i, j, k) ascending and the sphere is symmetric, so negation
// reverses the order: the partner of full row g is npw_full - 1 - g, the
// half sphere is the tail from h0 = (npw_full - 1) / 2 (G = 0 itself), and
// the partner of row h0 + h is h0 - h.
//
// Stored form: c'(0) = c(0) (real), c'(G) = sqrt 2 c(G) otherwise.  Then
// Re sum_half conj(a') b' = sum_full conj(a) b for real orbitals a, b, so
// every contraction, norm and dot product of the complex path gives the
// full-sphere value once its real part is taken (gamma_real_part for the
// band-space products; the column sums take Re already).
//
// Packing: for real orbitals a(r), b(r), C(G) = c_a(G) + i c_b(G) transforms
// to a(r) + i b(r), so |C(r)|^2 = a^2 + b^2 (the density of both) and V C is
// V a + i V b; the forward transform X of (V a + i V b) separates into
// A(G) = (X(G) + conj X(-G)) / 2 and B(G) = (X(G) - conj X(-G)) / 2i.
#include "roks_impl.cuh"

namespace roks {

namespace {

template <typename T>
__device__ __forceinline__ T sqrt2() { return T(1.4142135623730950488); }
template <typename T>
__device__ __forceinline__ T inv_sqrt2() { return T(0.70710678118654752440); }

// thread (h, k): rows h0 + h and h0 - h of packed band k
template <typename T>
__global__ void k_gamma_expand(int nh, int h0, int nb, const c2<T>* __restrict__ psi, int64_t ld,
                               c2<T>* __restrict__ Cpk, int64_t ldc) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (h >= nh) return;
    const int na = 2 * k, nbb = 2 * k + 1;
    c2<T> a = psi[(int64_t)na * ld + h];
    c2<T> b = nbb < nb ? psi[(int64_t)nbb * ld + h] : mk<T>(T(0), T(0));
    c2<T>* out = Cpk + (int64_t)k * ldc;
    if (h == 0) {
        // G = 0: real coefficients, a + i b
        out[h0] = mk<T>(a.x, b.x);
        return;
    }
    const T s = inv_sqrt2<T>();
    a = mk<T>(a.x * s, a.y * s);
    b = mk<T>(b.x * s, b.y * s);
    out[h0 + h] = mk<T>(a.x - b.y, a.y + b.x);      // a + i b
    out[h0 - h] = mk<T>(a.x + b.y, b.x - a.y);      // conj(a) + i conj(b)
}

template <typename T>
__global__ void k_gamma_unpack(int nh, int h0, int nb, int n_closed, const c2<T>* __restrict__ Fpk, int64_t ldc,
                               const c2<T>* __restrict__ psi, int64_t ldp, const T* __restrict__ g2half,
                               const T* __restrict__ wk, c2<T>* __restrict__ F, int64_t ldf) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int k = blockIdx.y;
    if (h >= nh) return;
    const c2<T>* in = Fpk + (int64_t)k * ldc;
    const c2<T> X = in[h0 + h];
    const c2<T> Y = in[h0 - h];   // the -G entry (X itself at G = 0)
    const T s = h == 0 ? T(1) : sqrt2<T>();
    const T half = T(0.5);
    // A = (X + conj Y) / 2, B = (X - conj Y) / 2i
    const c2<T> A = mk<T>(half * (X.x + Y.x) * s, half * (X.y - Y.y) * s);
    const c2<T> B = mk<T>(half * (X.y + Y.y) * s, half * (Y.x - X.x) * s);
    const T g2 = g2half[h];
#pragma unroll
    for (int part = 0; part < 2; ++part) {
        const int n = 2 * k + part;
        if (n >= nb) break;
        const int cls = n < n_closed ? 0 : n - n_closed + 1;
        const c2<T> p = psi[(int64_t)n * ldp + h];
        const T kin = wk[cls] * g2;
        const c2<T> v = part == 0 ? A : B;
        F[(int64_t)n * ldf + h] = mk<T>(v.x + kin * p.x, v.y + kin * p.y);
    }
}

template <typename T>
__global__ void k_gamma_scale_rows(int nh, int ncols, c2<T>* __restrict__ X, int64_t ld) {
    const int h = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (h >= nh || c >= ncols) return;
    c2<T>& v = X[(int64_t)c * ld + h];
    if (h == 0) {
        v.y = T(0);
    } else {
        const T s = sqrt2<T>();
        v.x *= s;
        v.y *= s;
    }
}

__global__ void k_gamma_real_part(int M, int N, double2* __restrict__ C, int ldc) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * N) return;
    const int m = (int)(i % M), n = (int)(i / M);
    C[(int64_t)n * ldc + m].y = 0.0;
}

}  // namespace

template <typename T>
void gamma_expand(int nh, int h0, int nb, const c2<T>* psi, int64_t ld, c2<T>* Cpk, int64_t ldc, cudaStream_t st) {
    const int nk = (nb + 1) / 2;
    if (nh <= 0 || nk <= 0) return;
    dim3 g((nh + 255) / 256, nk);
    count_launch();
    k_gamma_expand<T><<<g, 256, 0, st>>>(nh, h0, nb, psi, ld, Cpk, ldc);
}

template <typename T>
void gamma_unpack(int nh, int h0, int nb, int n_closed, const c2<T>* Fpk, int64_t ldc, const c2<T>* psi,
                  int64_t ldp, const T* g2half, const T* wk, c2<T>* F, int64_t ldf, cudaStream_t st) {
    const int nk = (nb + 1) / 2;
    if (nh <= 0 || nk <= 0) return;
    dim3 g((nh + 255) / 256, nk);
    count_launch();
    k_gamma_unpack<T><<<g, 256, 0, st>>>(nh, h0, nb, n_closed, Fpk, ldc, psi, ldp, g2half, wk, F, ldf);
}

template <typename T>
void gamma_scale_rows(int nh, int ncols, c2<T>* X, int64_t ld, cudaStream_t st) {
    if (nh <= 0 || ncols <= 0) return;
    dim3 g((nh + 255) / 256, ncols);
    count_launch();
    k_gamma_scale_rows<T><<<g, 256, 0, st>>>(nh, ncols, X, ld);
}

void gamma_real_part(int M, int N, double2* C, int ldc, cudaStream_t st) {
    const int64_t n = (int64_t)M * N;
    if (n <= 0) return;
    count_launch();
    k_gamma_real_part<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, N, C, ldc);
}

#define ROKS_INSTANTIATE_GAMMA(T)                                                                            \
    template void gamma_expand<T>(int, int, int, const c2<T>*, int64_t, c2<T>*, int64_t, cudaStream_t);      \
    template void gamma_unpack<T>(int, int, int, int, const c2<T>*, int64_t, const c2<T>*, int64_t, const T*,  \
                                  const T*, c2<T>*, int64_t, cudaStream_t);                                  \
    template void gamma_scale_rows<T>(int, int, c2<T>*, int64_t, cudaStream_t);
ROKS_INSTANTIATE_GAMMA(float)
ROKS_INSTANTIATE_GAMMA(double)

}  // namespace roks
