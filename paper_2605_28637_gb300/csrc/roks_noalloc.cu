// roks_noalloc.cu -- roks_orthonormalize_noalloc: Cholesky orthonormalisation
// of a band block (overlap S = 1) that allocates no device memory.
//
// Who needs it: callers that cannot call cudaMalloc, e.g. code running
// inside a framework that has reserved the GPU's memory for its own caching
// allocator, or an embedded solver loop that must not allocate once it is
// running.  The scratch of this entry point (split-K partial sums, the
// overlap matrix, L^{-H} and a status flag) lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded; every
// GPU that loads the library holds it until the process exits.
#include <cstddef>

#include "../../include/roks.h"
#include "roks_impl.cuh"

using namespace roks;

namespace {

constexpr int kNaMaxBands = 64;    // largest band count accepted
constexpr int kNaMaxChunks = 64;   // K chunks of the overlap contraction
constexpr size_t kNaPart = (size_t)kNaMaxChunks * kNaMaxBands * kNaMaxBands;   // double2
constexpr size_t kNaMat = (size_t)kNaMaxBands * kNaMaxBands;                   // double2
// layout (double2 units): partials | O | LinvH | L | flag (int, 256-byte slot)
constexpr size_t kNaBytes = sizeof(double2) * (kNaPart + 3 * kNaMat) + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

// Device address of the scratch array on the current device (the host name
// g_noalloc_scratch is only a stand-in and must never reach a kernel).  It
// is resolved on every call: the lookup is cheap next to the synchronising
// call, and a cached address would go stale if the module were reloaded
// (after cudaDeviceReset, for instance).
cudaError_t scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<unsigned char*>(p);
    return cudaSuccess;
}

// psi <- psi U in place, U upper triangular (nb x nb, FP64, column major).
// A block owns 64 rows: it reads them into shared memory before writing.
template <typename T>
__global__ void __launch_bounds__(256) k_rows_times_upper(int npw, int nb, c2<T>* psi, int64_t ld,
                                                          const double2* __restrict__ U) {
    using V = c2<T>;
    constexpr int RT = 64;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    V* tile = reinterpret_cast<V*>(smem_raw);       // [nb][RT]
    V* Us = tile + (size_t)nb * RT;                 // [nb][nb] column major
    const int g0 = blockIdx.x * RT;
    for (int idx = threadIdx.x; idx < nb * RT; idx += blockDim.x) {
        const int r = idx % RT, j = idx / RT;
        const int g = g0 + r;
        tile[idx] = g < npw ? psi[(int64_t)j * ld + g] : mk<T>(T(0), T(0));
    }
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
        const double2 u = U[idx];
        Us[idx] = mk<T>(T(u.x), T(u.y));
    }
    __syncthreads();
    const int r = threadIdx.x % RT;
    const int g = g0 + r;
    if (g >= npw) return;
    for (int j = threadIdx.x / RT; j < nb; j += blockDim.x / RT) {
        T sr = T(0), si = T(0);
        for (int k = 0; k <= j; ++k) {
            const V a = tile[k * RT + r], b = Us[j * nb + k];
            sr += a.x * b.x - a.y * b.y;
            si += a.x * b.y + a.y * b.x;
        }
        psi[(int64_t)j * ld + g] = mk<T>(sr, si);
    }
}

template <typename T>
roks_status run(int npw, int nb, void* psi, int64_t ld, cudaStream_t st, unsigned char* base) {
    using V = c2<T>;
    double2* part = reinterpret_cast<double2*>(base);
    double2* O = part + kNaPart;
    double2* LinvH = O + kNaMat;
    double2* Lw = LinvH + kNaMat;
    int* flag = reinterpret_cast<int*>(Lw + kNaMat);
    // the flag keeps the previous call's value: clear it first
    if (cudaMemsetAsync(flag, 0, sizeof(int), st) != cudaSuccess) return ROKS_ECUDA;
    V* X = static_cast<V*>(psi);
    gemm_cn_capped<T>(nb, nb, npw, X, ld, X, ld, O, nb, part, kNaMaxChunks, st);
    cholesky_inverse(nb, O, Lw, LinvH, flag, st);
    int h = 0;
    if (cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return ROKS_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return ROKS_ECUDA;
    if (h) return ROKS_ENOTPOSDEF;
    const size_t sm = sizeof(V) * ((size_t)nb * 64 + (size_t)nb * nb);
    if (sm > 48 * 1024 &&
        cudaFuncSetAttribute(k_rows_times_upper<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) !=
            cudaSuccess)
        return ROKS_ECUDA;
    count_launch();
    k_rows_times_upper<T><<<(npw + 63) / 64, 256, sm, st>>>(npw, nb, X, ld, LinvH);
    if (cudaGetLastError() != cudaSuccess) return ROKS_ECUDA;
    return ROKS_OK;
}

}  // namespace

extern "C" roks_status roks_orthonormalize_noalloc(int precision, int npw, int nbands, void* psi, int64_t ld,
                                                   void* cuda_stream) {
    if (precision != ROKS_FP64 && precision != ROKS_MIXED) return ROKS_EINVAL;
    if (!psi || npw <= 0 || nbands <= 0 || ld < npw) return ROKS_EINVAL;
    if (nbands > kNaMaxBands) return ROKS_EINVAL;     // beyond the fixed scratch
    unsigned char* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return ROKS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    return precision == ROKS_FP64 ? run<double>(npw, nbands, psi, ld, st, base)
                                  : run<float>(npw, nbands, psi, ld, st, base);
}
