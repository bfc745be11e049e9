// k_dense.cu -- complex contractions of the apply and PCG step (projector
// coefficients B = P^H Psi, back-projection P X, subspace matrices
// Psi^H X, rotations Psi U) and the small FP64 band-space matrix kernels
// (Cholesky inverse, Taylor exponential).
//
// The contractions here are SIMT tiled kernels with register blocking.
#include "roks_impl.cuh"

namespace roks {

// ------------------------------------------------------------------ C = A^H B, split over K
// A: K x M, B: K x N (column major).  Each block: 32 x 32 outputs over one
// K chunk; 256 threads, 2 x 2 outputs each.  Chunk sums are exact FP64
// additions of FP32 (or FP64) partial sums.
constexpr int CN_T = 32, CN_KT = 16, CN_KC = 1024;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_cn(int M, int N, int K, const c2<T>* __restrict__ A, int64_t lda,
                                                 const c2<T>* __restrict__ B, int64_t ldb, double2* __restrict__ part) {
    using V = c2<T>;
    __shared__ V As[CN_KT][CN_T + 1];
    __shared__ V Bs[CN_KT][CN_T + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * CN_T, n0 = blockIdx.y * CN_T;
    const int kbeg = blockIdx.z * CN_KC, kend = min(K, kbeg + CN_KC);
    V acc[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) acc[a][b] = mk<T>(T(0), T(0));
    for (int k0 = kbeg; k0 < kend; k0 += CN_KT) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int t = threadIdx.x + q * 256;
            const int kk = t & 15, mm = t >> 4;      // 16 x 32
            const int k = k0 + kk;
            const int m = m0 + mm, n = n0 + mm;
            As[kk][mm] = (k < kend && m < M) ? A[(int64_t)m * lda + k] : mk<T>(T(0), T(0));
            Bs[kk][mm] = (k < kend && n < N) ? B[(int64_t)n * ldb + k] : mk<T>(T(0), T(0));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < CN_KT; ++kk) {
            V a0 = As[kk][ty], a1 = As[kk][ty + 16];
            V b0 = Bs[kk][tx], b1 = Bs[kk][tx + 16];
            acc[0][0] = cadd(acc[0][0], cmulc(a0, b0));
            acc[0][1] = cadd(acc[0][1], cmulc(a0, b1));
            acc[1][0] = cadd(acc[1][0], cmulc(a1, b0));
            acc[1][1] = cadd(acc[1][1], cmulc(a1, b1));
        }
        __syncthreads();
    }
    double2* P = part + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int m = m0 + ty + 16 * a, n = n0 + tx + 16 * b;
            if (m < M && n < N) P[(int64_t)n * M + m] = make_double2(double(acc[a][b].x), double(acc[a][b].y));
        }
}

__global__ void k_chunk_sum(int M, int N, int nchunk, const double2* __restrict__ part, double2* __restrict__ C,
                            int ldc) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int m = idx % M, n = idx / M;
    double2 s = make_double2(0.0, 0.0);
    for (int c = 0; c < nchunk; ++c) {
        const double2 v = part[(int64_t)c * M * N + idx];
        s.x += v.x;
        s.y += v.y;
    }
    C[(int64_t)n * ldc + m] = s;
}

size_t gemm_cn_work(int M, int N, int K) {
    const int nchunk = (K + CN_KC - 1) / CN_KC;
    return (size_t)nchunk * M * N;
}

template <typename T>
void gemm_cn(int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb, double2* C, int ldc,
             double2* work, size_t work_elems, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    const int nchunk = K > 0 ? (K + CN_KC - 1) / CN_KC : 1;
    (void)work_elems;
    dim3 g((M + CN_T - 1) / CN_T, (N + CN_T - 1) / CN_T, nchunk);
    if (K > 0) k_gemm_cn<T><<<g, 256, 0, st>>>(M, N, K, A, lda, B, ldb, work);
    else cudaMemsetAsync(work, 0, sizeof(double2) * M * N, st);
    k_chunk_sum<<<(M * N + 255) / 256, 256, 0, st>>>(M, N, nchunk, work, C, ldc);
}

// ------------------------------------------------------------------ C = alpha A B + beta C
// A: M x K (tall, column major, element type T), B: K x N FP64 (small).
// Block: 64 rows x 32 columns; thread (tx < 64, ty < 4) owns rows m0+tx and
// columns n0 + ty + 4 c, c < 8.
constexpr int NN_TM = 64, NN_TN = 32, NN_KT = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_gemm_nn(int M, int N, int K, const c2<T>* __restrict__ A, int64_t lda,
                                                 const double2* __restrict__ B, int ldb, c2<T>* __restrict__ C,
                                                 int64_t ldc, T alpha, T beta) {
    using V = c2<T>;
    __shared__ V As[NN_KT][NN_TM];
    __shared__ V Bs[NN_KT][NN_TN];
    const int tx = threadIdx.x & 63, ty = threadIdx.x >> 6;
    const int m0 = blockIdx.x * NN_TM, n0 = blockIdx.y * NN_TN;
    V acc[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] = mk<T>(T(0), T(0));
    for (int k0 = 0; k0 < K; k0 += NN_KT) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = threadIdx.x + q * 256;       // 16 x 64
            const int mm = t & 63, kk = t >> 6;
            const int m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < M && k < K) ? A[(int64_t)k * lda + m] : mk<T>(T(0), T(0));
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const int t = threadIdx.x + q * 256;       // 16 x 32
            const int kk = t & 15, nn = t >> 4;
            const int k = k0 + kk, n = n0 + nn;
            double2 b = (k < K && n < N) ? B[(int64_t)n * ldb + k] : make_double2(0.0, 0.0);
            Bs[kk][nn] = mk<T>(T(b.x), T(b.y));
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < NN_KT; ++kk) {
            const V a = As[kk][tx];
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[c] = cadd(acc[c], cmul(a, Bs[kk][ty + 4 * c]));
        }
        __syncthreads();
    }
    const int m = m0 + tx;
    if (m >= M) return;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const int n = n0 + ty + 4 * c;
        if (n < N) {
            V* dst = C + (int64_t)n * ldc + m;
            V r = cscale(acc[c], alpha);
            if (beta != T(0)) r = cadd(r, cscale(*dst, beta));
            *dst = r;
        }
    }
}

template <typename T>
void gemm_nn(int M, int N, int K, const c2<T>* A, int64_t lda, const double2* B, int ldb, c2<T>* C, int64_t ldc,
             double alpha, double beta, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    dim3 g((M + NN_TM - 1) / NN_TM, (N + NN_TN - 1) / NN_TN);
    k_gemm_nn<T><<<g, 256, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, T(alpha), T(beta));
}

template void gemm_cn<float>(int, int, int, const float2*, int64_t, const float2*, int64_t, double2*, int,
                             double2*, size_t, cudaStream_t);
template void gemm_cn<double>(int, int, int, const double2*, int64_t, const double2*, int64_t, double2*, int,
                              double2*, size_t, cudaStream_t);
template void gemm_nn<float>(int, int, int, const float2*, int64_t, const double2*, int, float2*, int64_t, double,
                             double, cudaStream_t);
template void gemm_nn<double>(int, int, int, const double2*, int64_t, const double2*, int, double2*, int64_t,
                              double, double, cudaStream_t);

// ------------------------------------------------------------------ small FP64 matrices
__global__ void k_small_gemm(int M, int N, int K, const double2* __restrict__ A, int lda, int ca,
                             const double2* __restrict__ B, int ldb, int cb, double2* __restrict__ C, int ldc,
                             double alpha, double beta) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= M * N) return;
    const int m = idx % M, n = idx / M;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < K; ++k) {
        double2 a = ca ? A[(int64_t)m * lda + k] : A[(int64_t)k * lda + m];
        double2 b = cb ? B[(int64_t)k * ldb + n] : B[(int64_t)n * ldb + k];
        if (ca) a.y = -a.y;
        if (cb) b.y = -b.y;
        sr += a.x * b.x - a.y * b.y;
        si += a.x * b.y + a.y * b.x;
    }
    double2* c = C + (int64_t)n * ldc + m;
    double2 r = make_double2(alpha * sr, alpha * si);
    if (beta != 0.0) { r.x += beta * c->x; r.y += beta * c->y; }
    *c = r;
}

// op(A): A (M x K) or A^H when ca (A stored K x M); op(B) likewise.
void small_gemm(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb, bool cb,
                double2* C, int ldc, double alpha, double beta, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    k_small_gemm<<<(M * N + 127) / 128, 128, 0, st>>>(M, N, K, A, lda, ca, B, ldb, cb, C, ldc, alpha, beta);
}

// Cholesky O = L L^H (Crout, column by column) and the inverse of L, one
// block.  LinvH[k, i] = conj(Linv[i, k]) so that Psi LinvH = Psi L^{-H}.
__global__ void __launch_bounds__(1024) k_cholesky_inverse(int n, const double2* __restrict__ O, double2* L,
                                                           double2* LinvH, int* flag) {
    __shared__ double piv;
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) L[idx] = make_double2(0.0, 0.0);
    __syncthreads();
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = O[(int64_t)j * n + j].x;
            for (int k = 0; k < j; ++k) {
                const double2 l = L[(int64_t)k * n + j];
                d -= l.x * l.x + l.y * l.y;
            }
            if (!(d > 0.0)) {
                bad = j + 1;
                d = 1.0;
            }
            piv = sqrt(d);
            L[(int64_t)j * n + j] = make_double2(piv, 0.0);
        }
        __syncthreads();
        const double inv = 1.0 / piv;
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            double2 s = O[(int64_t)j * n + i];
            for (int k = 0; k < j; ++k) {
                const double2 a = L[(int64_t)k * n + i];
                const double2 b = L[(int64_t)k * n + j];
                // a * conj(b)
                s.x -= a.x * b.x + a.y * b.y;
                s.y -= a.y * b.x - a.x * b.y;
            }
            L[(int64_t)j * n + i] = make_double2(s.x * inv, s.y * inv);
        }
        __syncthreads();
    }
    // columns c of X = L^{-1}: X[i, c] = (delta_ic - sum_{c<=k<i} L[i,k] X[k,c]) / L[i,i]
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        for (int i = 0; i < c; ++i) LinvH[(int64_t)i * n + c] = make_double2(0.0, 0.0);
        for (int i = c; i < n; ++i) {
            double sr = (i == c) ? 1.0 : 0.0, si = 0.0;
            for (int k = c; k < i; ++k) {
                const double2 l = L[(int64_t)k * n + i];
                const double2 x = LinvH[(int64_t)k * n + c];   // conj(X[k, c]) stored at row c, column k
                // l * X[k,c] = l * conj(x)
                sr -= l.x * x.x + l.y * x.y;
                si -= l.y * x.x - l.x * x.y;
            }
            const double d = 1.0 / L[(int64_t)i * n + i].x;
            // conj(X[i, c]) is element (row c, column i) of L^{-H}
            LinvH[(int64_t)i * n + c] = make_double2(sr * d, -si * d);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && bad) flag[0] = bad;
}

void cholesky_inverse(int n, const double2* O, double2* Lw, double2* LinvH, int* flag, cudaStream_t st) {
    k_cholesky_inverse<<<1, 1024, 0, st>>>(n, O, Lw, LinvH, flag);
}

// ------------------------------------------------------------------ exp(s A)
// Scaling: X = s A / 2^q with ||s A||_1 / 2^q <= 1/2; Taylor degree 16 by
// Horner, E_k = I + X E_{k+1} / k; then q squarings.  q is decided on the
// device and the squaring launches past q copy through.
constexpr int kExpmDegree = 16;
constexpr int kExpmMaxSquare = 16;

__global__ void k_expm_scale(int n, const double2* __restrict__ A, const double* __restrict__ s,
                             double2* __restrict__ X, double* __restrict__ info) {
    __shared__ double colmax[1024];
    double best = 0.0;
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double sum = 0.0;
        for (int r = 0; r < n; ++r) {
            const double2 a = A[(int64_t)c * n + r];
            sum += sqrt(a.x * a.x + a.y * a.y);
        }
        best = fmax(best, sum);
    }
    colmax[threadIdx.x] = best;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) colmax[threadIdx.x] = fmax(colmax[threadIdx.x], colmax[threadIdx.x + w]);
        __syncthreads();
    }
    const double norm = fabs(s[0]) * colmax[0];
    int q = 0;
    double scaled = norm;
    while (scaled > 0.5 && q < kExpmMaxSquare) {
        scaled *= 0.5;
        ++q;
    }
    const double f = s[0] * ldexp(1.0, -q);
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const double2 a = A[idx];
        X[idx] = make_double2(f * a.x, f * a.y);
    }
    if (threadIdx.x == 0) info[0] = double(q);
}

__global__ void k_expm_horner(int n, const double2* __restrict__ X, const double2* __restrict__ Ein,
                              double2* __restrict__ Eout, double invk, int first) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int m = idx % n, c = idx / n;
    double sr = 0.0, si = 0.0;
    if (first) {
        const double2 x = X[idx];
        sr = x.x;
        si = x.y;
    } else {
        for (int k = 0; k < n; ++k) {
            const double2 a = X[(int64_t)k * n + m];
            const double2 b = Ein[(int64_t)c * n + k];
            sr += a.x * b.x - a.y * b.y;
            si += a.x * b.y + a.y * b.x;
        }
    }
    Eout[idx] = make_double2((m == c ? 1.0 : 0.0) + sr * invk, si * invk);
}

__global__ void k_expm_square(int n, const double2* __restrict__ E, double2* __restrict__ Eout, int step,
                              const double* __restrict__ info) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    if (step >= int(info[0])) {
        Eout[idx] = E[idx];
        return;
    }
    const int m = idx % n, c = idx / n;
    double sr = 0.0, si = 0.0;
    for (int k = 0; k < n; ++k) {
        const double2 a = E[(int64_t)k * n + m];
        const double2 b = E[(int64_t)c * n + k];
        sr += a.x * b.x - a.y * b.y;
        si += a.x * b.y + a.y * b.x;
    }
    Eout[idx] = make_double2(sr, si);
}

void expm_scaled(int n, const double2* A, const double* scale_dev, double2* E, double2* w1, double2* w2,
                 double2* w3, double* sdev, cudaStream_t st) {
    k_expm_scale<<<1, 256, 0, st>>>(n, A, scale_dev, w1, sdev);
    const int blocks = (n * n + 127) / 128;
    // Horner: E_deg = I + X / deg, ..., E_1 = I + X E_2
    double2* cur = w2;
    double2* nxt = w3;
    k_expm_horner<<<blocks, 128, 0, st>>>(n, w1, nullptr, cur, 1.0 / kExpmDegree, 1);
    for (int k = kExpmDegree - 1; k >= 1; --k) {
        k_expm_horner<<<blocks, 128, 0, st>>>(n, w1, cur, nxt, 1.0 / k, 0);
        double2* t = cur; cur = nxt; nxt = t;
    }
    for (int q = 0; q < kExpmMaxSquare; ++q) {
        double2* dst = (q == kExpmMaxSquare - 1) ? E : nxt;
        k_expm_square<<<blocks, 128, 0, st>>>(n, cur, dst, q, sdev);
        if (q == kExpmMaxSquare - 1) break;
        double2* t = cur; cur = nxt; nxt = t;
    }
}

}  // namespace roks
