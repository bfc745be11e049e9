// roks_impl.cuh -- internal declarations shared by the library's translation
// units: geometry of the plane-wave sphere on the FFT grid, the launchers of
// the CUDA kernels, and small helpers.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "fft_core.cuh"

namespace roks {

// Grid sizes with compiled transforms.
constexpr int kGrids[] = {16, 24, 32, 48, 72, 96, 120};

// Lines per shared-memory tile for a transform length.
// Lines per transform tile.  N = 120 takes 32 lines with the 15 x 8 plan:
// its two passes then hold 256 and 480 butterflies (one and two nearly full
// rounds of 256 threads); 24 lines with 12 x 10 left the second round of the
// radix-10 pass 1/8 busy.  Measured at mgo-120 (ms per launch): x-stage
// density 1.99 -> 1.33, x-stage apply 2.99 -> 2.60, y stage 0.56 -> 0.48.
__host__ __device__ constexpr int tile_lines(int n) {
    return n == 16 ? 16 : (n == 32 || n == 96 || n == 120) ? 32 : 24;
}
constexpr int kThreads = 256;
// Threads of the x-stage apply: for N = 96 (radix 12 then 8 over 32 lines:
// 256 and 384 butterflies) 128 threads take 2 and 3 butterflies each with
// none idle; other lengths keep kThreads.
__host__ __device__ constexpr int x_threads(int n) { return n == 96 ? 128 : kThreads; }

// The plane-wave sphere seen from the grid.  Basis order is i, j, k
// ascending, so the coefficients of one (i, j) column are contiguous with
// k running from -kmax to kmax; the columns of one i plane are contiguous
// with j running from -jmax to jmax.
struct Sphere {
    int N;        // grid points per side
    int nmax;     // largest |i|, |j|, |k|
    int np;       // planes i = -nmax .. nmax  (2 nmax + 1)
    int ncol;     // (i, j) columns
    const int* col_start;   // [ncol] first coefficient (k = -kmax)
    const int* col_kmax;    // [ncol]
    const int* plane_col0;  // [np] first column of plane i
    const int* plane_jmax;  // [np]
};

__host__ __device__ __forceinline__ int signed_freq(int e, int n) { return e <= n / 2 ? e : e - n; }

// Host-side count of the kernel launches issued by the library (every launch
// site calls count_launch(); read and reset through the profiling API).
void count_launch();
void count_launches(long long n);   // n launches at once (a graph replay)
long long launches_now();
long long launches_take();

// ------------------------------------------------------------ band FFTs
// Bands b0 .. b0+nbb-1 of psi (column major, ld).  Zc holds nbb x ncol x N
// z-lines, Yp holds nbb x np x N x N plane data (y, z).
// z stage, inverse: sphere columns -> Zc
template <typename T>
void band_z_inv(const Sphere& s, const c2<T>* tw, const c2<T>* psi, int64_t ld, int b0, int nbb, c2<T>* Zc,
                cudaStream_t st);
// y stage, inverse: Zc -> Yp
template <typename T>
void band_y_inv(const Sphere& s, const c2<T>* tw, const c2<T>* Zc, c2<T>* Yp, int nbb, cudaStream_t st);
// x stage, in place on Yp: inverse transform, multiply by V^{class(b)} * scale,
// forward transform, keep the planes of the sphere.  Band split_band (-1:
// none) holds two real orbitals as (re, im): re is multiplied by V^a, im by V^b.
template <typename T>
void band_x_apply(const Sphere& s, const c2<T>* tw, c2<T>* Yp, const T* Vk, const c2<T>* Xx, int b0, int nbb,
                  int n_closed, int split_band, T scale, cudaStream_t st);
// x stage, inverse, full real-space lines: Phi[b0 + b] = scale * psi~ (N^3 each)
template <typename T>
void band_x_inv_full(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, c2<T>* Phi, int b0, int nbb, T scale,
                     cudaStream_t st);
// y stage, forward: Yp -> Zc (columns of the sphere only)
template <typename T>
void band_y_fwd(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, c2<T>* Zc, int nbb, cudaStream_t st);
// z stage, forward: Zc -> out[b] = gathered coefficients + wk[class] g2half psi[b]
// (psi null: the gathered coefficients alone)
template <typename T>
void band_z_fwd(const Sphere& s, const c2<T>* tw, const c2<T>* Zc, c2<T>* out, int64_t ldo, const c2<T>* psi,
                int64_t ldp, const T* g2half, const T* wk, int b0, int nbb, int n_closed, cudaStream_t st);
// Grid densities: FP64 in the FP64 path; in the mixed path a compensated FP32
// pair (hi, lo) in the same 8 bytes per point, summed with Knuth's two-sum,
// so that no per-point FP64 arithmetic or conversion runs (both are slow on
// this part) while the sums keep about FP64 accuracy.
template <typename T> struct DensAcc;
template <> struct DensAcc<double> {
    using S = double;
    __host__ __device__ static S make(double v) { return v; }
    __host__ __device__ static S add(S a, double v) { return a + v; }
    __host__ __device__ static S add2(S a, S b) { return a + b; }
    __host__ __device__ static double value(S a) { return a; }
};
template <> struct DensAcc<float> {
    using S = float2;
    __host__ __device__ static S make(float v) { return make_float2(v, 0.f); }
    __host__ __device__ static S add(S a, float v) {
        const float t = a.x + v;
        const float bp = t - a.x;
        const float err = (a.x - (t - bp)) + (v - bp);
        return make_float2(t, a.y + err);
    }
    __host__ __device__ static S add2(S a, S b) {
        S r = add(a, b.x);
        r.y += b.y;
        return r;
    }
    __host__ __device__ static float value(S a) { return a.x + a.y; }
};

// x stage, inverse: rho3 (3 x N^3 DensAcc<T>::S, in a buffer of doubles) =
// sum |psi|^2 * scale per class, bands split into up to ngroups groups; slot
// holds ngroups x N^3 values.  rho3 classes a, b must be zero on entry (class
// 0 is overwritten).  part_sel 1 / 2 sums (Re psi)^2 / (Im psi)^2 instead of
// |psi|^2, and cls_override >= 0 sends every band to that class of rho3
// (with slot null: no group slots; the Gamma-point open pair).
constexpr int kDensityGroups = 4;
constexpr int kDensityGroupsMax = 8;   // the autotuner's largest candidate
template <typename T>
void band_x_density(const Sphere& s, const c2<T>* tw, const c2<T>* Yp, double* rho3, double* slot, int ngroups,
                    int b0, int nbb, int n_closed, double scale, cudaStream_t st, int part_sel = 0,
                    int cls_override = -1);

// ------------------------------------------------------------ Gamma point (k_gamma.cu)
// Real orbitals are stored on the half sphere (G = 0 and the Miller triples
// after it in the basis order, the contiguous tail of the full basis from
// row h0 = (npw_full - 1) / 2), with every coefficient of G != 0 scaled by
// sqrt 2.  With that scaling the real part of a half-sphere sum of
// conj(a) b equals the full-sphere inner product of the real orbitals, so
// the contractions, norms and dot products of the complex path carry over.
// The partner -G of full row h0 + h is row h0 - h.
//
// Cpk[k] (full sphere, ldc) = a + i b for the bands a = 2k, b = 2k + 1 (b
// absent: 0), unscaled and expanded with c(-G) = conj(c(G)).
template <typename T>
void gamma_expand(int nh, int h0, int nb, const c2<T>* psi, int64_t ld, c2<T>* Cpk, int64_t ldc, cudaStream_t st);
// F[n] (half sphere, scaled) = the transform of real orbital n taken out of
// the packed transform Fpk[n / 2] (A = (X + conj X~) / 2 for the real part,
// (X - conj X~) / 2i for the imaginary one, X~ the -G entry), plus the
// kinetic term wk[class(n)] g2half psi[n].
template <typename T>
void gamma_unpack(int nh, int h0, int nb, int n_closed, const c2<T>* Fpk, int64_t ldc, const c2<T>* psi,
                  int64_t ldp, const T* g2half, const T* wk, c2<T>* F, int64_t ldf, cudaStream_t st);
// rows 1 .. nh-1 of ncols columns times sqrt 2; row 0 (G = 0) keeps its real
// part only (the half-sphere form of a real-space-real set)
template <typename T>
void gamma_scale_rows(int nh, int ncols, c2<T>* X, int64_t ld, cudaStream_t st);
// C (M x N, ldc) <- Re C: the band-space products of real orbitals
void gamma_real_part(int M, int N, double2* C, int ldc, cudaStream_t st);

// ------------------------------------------------------------ full-grid 3D FFT (in place)
template <typename T>
void grid_fft3(int N, const c2<T>* tw, c2<T>* data, int dir, cudaStream_t st);
// batch grids data + k bstride, k < batch
template <typename T>
void grid_fft3_batched(int N, const c2<T>* tw, c2<T>* data, int batch, int64_t bstride, int dir, cudaStream_t st);

// ------------------------------------------------------------ dense complex contractions
// Cpart[chunk] (element type T, M x N column major) = sum over the k of the
// chunk of conj(A[k, m]) B[k, n]; then C = sum_chunks Cpart (double2, ldc)
// in a fixed order.  work holds work_elems double2.  Large FP32 blocks go to
// the tensor cores (gemm_cn_tcg), the others to the streamed SIMT kernel.
template <typename T>
void gemm_cn(int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb,
             double2* C, int ldc, double2* work, size_t work_elems, cudaStream_t st);
size_t gemm_cn_work(int M, int N, int K);
// C (ldc) = fixed-order sum of nchunk partials (M x N double2 each)
void chunk_sum(int M, int N, int nchunk, const double2* part, double2* C, int ldc, cudaStream_t st);
// FP32 partials (nchunk x M x N float2) summed like chunk_sum, with compensation.
void chunk_sum_f32(int M, int N, int nchunk, const float2* part, double2* C, int ldc, cudaStream_t st);
// Streamed FP32 contractions (bulk copies into a shared-memory ring, one CTA
// per SM); false when the shape, the alignment (16-byte bases, even leading
// dimensions) or the buffers do not allow them, and the caller falls back.
// ROKS_STREAM=0 switches them off.
bool stream_enabled();
bool gemm_cn_stream(int M, int N, int K, const float2* A, int64_t lda, const float2* B, int64_t ldb, double2* C,
                    int ldc, double2* work, size_t work_elems, cudaStream_t st);
bool gemm_nn_stream(int M, int N, int K, const float2* A, int64_t lda, const double2* B, int ldb, void* bwork,
                    const float2* Cin, int64_t ldcin, float2* Cout, int64_t ldc, float alpha, float beta,
                    cudaStream_t st);
// 1 if a streamed-contraction wait gave up since the last call (then cleared);
// the flag's device address, for asynchronous reads.
int stream_timeout_take();
// Polls of every bounded work-loop wait in the contraction kernels launched
// from now on: 0 the default (2^26), < 0 none (every such wait gives up).
void set_wait_cap(int cap);
uint32_t wait_polls();
int* stream_timeout_flag();
// Same, with at most max_chunks K chunks (work holds max_chunks * M * N).
template <typename T>
void gemm_cn_capped(int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb,
                    double2* C, int ldc, double2* work, int max_chunks, cudaStream_t st);
// C[m, n] = alpha sum_k A[m, k] B[k, n] + beta C[m, n]; B is FP64 (small).
// For T = float, bwork receives an FP32 copy of B (K x N float2); it may be
// the partial-sum buffer of gemm_cn (not in use across calls).
// bwork_bytes: size of bwork; the tensor-core path (FP32, large blocks)
// needs tcg_nn_work_bytes(N, K) and is skipped when it is 0 or too small.
template <typename T>
void gemm_nn(int M, int N, int K, const c2<T>* A, int64_t lda, const double2* B, int ldb,
             c2<T>* C, int64_t ldc, double alpha, double beta, void* bwork, cudaStream_t st,
             size_t bwork_bytes = 0);

// Cout (ldc) = alpha A B + beta Cin (ldcin); Cin may differ from Cout (when
// beta != 0 and it does, Cin is not modified).
template <typename T>
void gemm_nn_io(int M, int N, int K, const c2<T>* A, int64_t lda, const double2* B, int ldb, const c2<T>* Cin,
                int64_t ldcin, c2<T>* Cout, int64_t ldc, double alpha, double beta, void* bwork, cudaStream_t st,
                size_t bwork_bytes = 0);

// ------------------------------------------------------------ tensor-core contractions (k_tcgemm.cu)
// Complex FP32 contractions of large blocks on tcgen05 (three TF32 products
// per FP32 product, every K-step drained into round-to-nearest FP32 sums).
bool tcg_enabled();
bool tcg_cn_takes(int M, int N, int K);
bool tcg_nn_takes(int M, int N, int K);
// K-split depth of the A^H B products: about waves_x2 / 2 waves of CTAs
// (the work buffer is sized for the deepest candidate, 4 waves)
void tcg_set_waves(int waves_x2);
size_t tcg_cn_work_bytes(int M, int N, int K);
size_t tcg_nn_work_bytes(int N, int K);
bool gemm_cn_tcg(int M, int N, int K, const float2* A, int64_t lda, const float2* B, int64_t ldb, double2* C, int ldc,
                 void* work, size_t work_bytes, cudaStream_t st);
bool gemm_nn_tcg(int M, int N, int K, const float2* A, int64_t lda, const double2* B, int ldb, const float2* Cin,
                 int64_t ldcin, float2* Cout, int64_t ldc, float alpha, float beta, void* bwork, size_t bwork_bytes,
                 cudaStream_t st);
// An operand that does not change (the projector matrix) split once into
// TF32 hi/lo blocks in the kernels' operand layout: the tall products A B
// whose A is that matrix (same address, leading dimension and shape) then
// copy it instead of converting it.  out holds tcg_presplit_bytes(M, K);
// false when not registered.
size_t tcg_presplit_bytes(int M, int K);
bool tcg_presplit(int M, int K, const float2* A, int64_t lda, void* out, cudaStream_t st);
void tcg_presplit_forget(const void* split);
// 1 if a tensor-core wait gave up since the last call (then cleared)
int tcg_timeout_take();
// tensor-core contraction launches since the last call
long long tcg_launches_take();

// ------------------------------------------------------------ small FP64 matrices (n x n, column major)
void small_gemm(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb,
                bool cb, double2* C, int ldc, double alpha, double beta, cudaStream_t st);
// Same with FP32 arithmetic (FP64 storage, alpha and beta applied in FP64).
// work (optional, work_bytes): the large products pack both operands into
// FP32 there first.
void small_gemm_f32(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb, bool cb,
                    double2* C, int ldc, double alpha, double beta, cudaStream_t st, void* work = nullptr,
                    size_t work_bytes = 0);
// O (Hermitian) -> LinvH = L^{-H}, L L^H = O.  flag[0] set to 1 + column on failure.
void cholesky_inverse(int n, const double2* O, double2* Lw, double2* LinvH, int* flag, cudaStream_t st);
// n within the single-block factorisations
bool cholesky_small_supported(int n);
// Cholesky inverse of a near-identity Hermitian O in deviation form, FP32,
// one block (n <= 64): L = I + Lambda, L^{-1} = I + Xi; writes XiH = Xi^H
// (so that L^{-H} = I + XiH).  The rounding errors scale with |O - I|, not
// with 1.  O's two triangles are averaged.  flag[0] = 1 + column on failure.
void cholesky_dev_f32(int n, const double2* O, double2* XiH, int* flag, cudaStream_t st);
// Blocked multi-block Cholesky inverse for any n (FP32 or FP64 arithmetic);
// work: cholesky_big_work_bytes(n, fp64).
size_t cholesky_big_work_bytes(int n, bool fp64);
void cholesky_inverse_big(int n, const double2* O, void* work, bool fp64, double2* LinvH, int* flag,
                          cudaStream_t st);
// exp(scale A) for any n on a tiled square GEMM (FP32 degree 8 or FP64
// degree 16); work: expm_big_work_bytes(n, fp64); info: 1 double.
size_t expm_big_work_bytes(int n, bool fp64);
void expm_big(int n, const double2* A, const double* scale_dev, double2* E, void* work, double* info, bool fp64,
              cudaStream_t st);
// E = expm(scale_dev[0] * A), A anti-Hermitian, Taylor + scaling and squaring.
void expm_scaled(int n, const double2* A, const double* scale_dev, double2* E, double2* w1, double2* w2,
                 double2* w3, double* sdev, cudaStream_t st);
// Single-precision, single-block variant for n <= 64; false if n is larger.
bool expm_small_f32(int n, const double2* A, const double* scale_dev, double2* E, cudaStream_t st);

}  // namespace roks
