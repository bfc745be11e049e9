// k_dense.cu -- complex contractions of the apply and PCG step (projector
// coefficients B = P^H Psi, back-projection P X, subspace matrices
// Psi^H X, rotations Psi U) and the small FP64 band-space matrix kernels
// (Cholesky inverse, Taylor exponential).
//
// The contractions here are SIMT tiled kernels with register blocking.
#include <atomic>
#include <mutex>
#include <vector>

#include <cooperative_groups.h>

#include "roks_impl.cuh"

namespace roks {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_now() { return g_launches.load(std::memory_order_relaxed); }
long long launches_take() { return g_launches.exchange(0); }

// ------------------------------------------------------------------ complex multiply-accumulate
namespace {
template <typename T> __device__ __forceinline__ T fmat(T a, T b, T c);
template <> __device__ __forceinline__ float fmat<float>(float a, float b, float c) { return fmaf(a, b, c); }
template <> __device__ __forceinline__ double fmat<double>(double a, double b, double c) { return fma(a, b, c); }

// acc += conj(a) b as four fused multiply-adds
template <typename T>
__device__ __forceinline__ void mac_cn(c2<T>& acc, const c2<T>& a, const c2<T>& b) {
    acc.x = fmat(a.x, b.x, acc.x);
    acc.x = fmat(a.y, b.y, acc.x);
    acc.y = fmat(a.x, b.y, acc.y);
    acc.y = fmat(-a.y, b.x, acc.y);
}
// acc += a b
template <typename T>
__device__ __forceinline__ void mac_nn(c2<T>& acc, const c2<T>& a, const c2<T>& b) {
    acc.x = fmat(a.x, b.x, acc.x);
    acc.x = fmat(-a.y, b.y, acc.x);
    acc.y = fmat(a.x, b.y, acc.y);
    acc.y = fmat(a.y, b.x, acc.y);
}

// Asynchronous global -> shared copy of one complex element (8 or 16
// bytes); the destination is zero-filled when !valid (nothing is read).
template <typename T>
__device__ __forceinline__ void cp_elem(c2<T>* dst, const c2<T>* src, bool valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    const int n = valid ? (int)sizeof(c2<T>) : 0;
    if constexpr (sizeof(c2<T>) == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int NPEND>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(NPEND) : "memory"); }

// Shared-memory position of tile row r when each thread owns R consecutive
// rows: one pad element after every R rows for even R, so that the 16
// threads of a row group read 16 different bank pairs.
template <int R> __host__ __device__ constexpr int padpos(int r) { return (R % 2 == 0) ? r + r / R : r; }
template <int R> __host__ __device__ constexpr int padgroup() { return (R % 2 == 0) ? R + 1 : R; }
// row stride of a k slice: covers 16 row groups and is odd (conflict-free transposed stores)
template <int R> __host__ __device__ constexpr int padstride() { return (16 * padgroup<R>()) | 1; }
}  // namespace

// ------------------------------------------------------------------ C = A^H B, split over K
// A: K x M, B: K x N (column major, K contiguous).  A block of TY x TX
// threads (runtime, at most 16 x 16) owns an output tile of (TY RM) x (TX RN)
// and one K chunk; thread (tx, ty) keeps the RM x RN register tile of rows
// ty RM + i and columns tx RN + j.  K slices of KT are double-buffered in
// shared memory by cp.async.  Chunk partials (element type T) are summed in a
// fixed order by k_chunk_sum.
template <typename T> struct CnTile { static constexpr int KT = sizeof(T) == 4 ? 32 : 16; };

template <typename T, int RM, int RN>
__global__ void __launch_bounds__(256) k_gemm_cn(int M, int N, int K, int kchunk, int TY, int TX, int SA, int SB,
                                                 const c2<T>* __restrict__ A, int64_t lda,
                                                 const c2<T>* __restrict__ B, int64_t ldb, c2<T>* __restrict__ part) {
    // SA, SB: odd row strides of the k slices, at least TY (TX) padded row groups
    using V = c2<T>;
    constexpr int KT = CnTile<T>::KT;
    extern __shared__ __align__(16) unsigned char cn_smem[];
    V* As = reinterpret_cast<V*>(cn_smem);   // [2][KT][SA]
    V* Bs = As + 2 * KT * SA;                // [2][KT][SB]
    const int nthr = TX * TY, tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    const int TM = TY * RM, TN = TX * RN;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);
    const int nk = kend > kbeg ? (kend - kbeg + KT - 1) / KT : 0;

    auto stage_in = [&](int s, int k0) {
        V* as = As + s * KT * SA;
        V* bs = Bs + s * KT * SB;
        for (int e = tid; e < TM * KT; e += nthr) {
            const int r = e / KT, kk = e % KT;
            const int m = m0 + r, k = k0 + kk;
            const bool ok = m < M && k < kend;
            cp_elem<T>(as + kk * SA + padpos<RM>(r), ok ? A + (int64_t)m * lda + k : A, ok);
        }
        for (int e = tid; e < TN * KT; e += nthr) {
            const int c = e / KT, kk = e % KT;
            const int n = n0 + c, k = k0 + kk;
            const bool ok = n < N && k < kend;
            cp_elem<T>(bs + kk * SB + padpos<RN>(c), ok ? B + (int64_t)n * ldb + k : B, ok);
        }
        cp_commit();
    };

    V acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = mk<T>(T(0), T(0));
    if (nk > 0) stage_in(0, kbeg);
    for (int t = 0; t < nk; ++t) {
        if (t + 1 < nk) {
            stage_in((t + 1) & 1, kbeg + (t + 1) * KT);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const V* as = As + (t & 1) * KT * SA + ty * padgroup<RM>();
        const V* bs = Bs + (t & 1) * KT * SB + tx * padgroup<RN>();
#pragma unroll 8
        for (int kk = 0; kk < KT; ++kk) {
            V a[RM], b[RN];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = as[i];
#pragma unroll
            for (int j = 0; j < RN; ++j) b[j] = bs[j];
            as += SA;
            bs += SB;
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) mac_cn<T>(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    // stage the tile (column n at Cs[n TM + r]) and write it out along m
    V* Cs = As;
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) Cs[(tx * RN + j) * TM + ty * RM + i] = acc[i][j];
    __syncthreads();
    V* P = part + (int64_t)blockIdx.z * M * N;
    for (int e = tid; e < TM * TN; e += nthr) {
        const int c = e / TM, r = e - c * TM;
        const int m = m0 + r, n = n0 + c;
        if (m < M && n < N) P[(int64_t)n * M + m] = Cs[e];
    }
}

namespace {
// s + v with its rounding error accumulated in c (Knuth's two-sum)
__device__ __forceinline__ void two_sum_acc(float& s, float& c, float v) {
    const float t = s + v;
    const float bp = t - s;
    c += (s - (t - bp)) + (v - bp);
    s = t;
}
}  // namespace

// C[n ldc + m] = sum over the chunks of part[c][n][m] in a fixed order.  A
// block covers 32 consecutive outputs (lanes) and its 32 warps take every
// 32nd chunk (many loads in flight: the reduction is latency-bound); FP32
// partials are summed with compensation (two-sum) and the 32 group sums
// combined by a fixed pairwise tree of compensated FP32 additions; FP64
// partials are summed directly, by the same tree.
constexpr int kSumGroups = 32;
// (s1, c1) += (s2, c2) for compensated sums: the rounding error of s1 + s2
// joins the compensations
__device__ __forceinline__ void comp_add(float& s1, float& c1, float s2, float c2) {
    const float t = s1 + s2;
    const float bp = t - s1;
    c1 += c2 + ((s1 - (t - bp)) + (s2 - bp));
    s1 = t;
}
template <typename P>
__global__ void __launch_bounds__(32 * kSumGroups) k_chunk_sum(int M, int MN, int nchunk, const P* __restrict__ part,
                                                               double2* __restrict__ C, int ldc) {
    const int lane = threadIdx.x & 31, g = threadIdx.x >> 5;
    const int w = blockIdx.x * 32 + lane;
    if constexpr (sizeof(P) == 8) {
        // FP32 partials: compensated FP32 throughout (FP64 arithmetic is slow
        // on this part), one conversion per output at the end
        __shared__ float4 red[kSumGroups][32];
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
        if (w < MN) {
#pragma unroll 8
            for (int c = g; c < nchunk; c += kSumGroups) {
                const P v = part[(int64_t)c * MN + w];
                two_sum_acc(sx, cx, v.x);
                two_sum_acc(sy, cy, v.y);
            }
        }
        red[g][lane] = make_float4(sx, cx, sy, cy);
        __syncthreads();
#pragma unroll
        for (int h = kSumGroups / 2; h > 0; h >>= 1) {
            if (g < h) {
                float4 a = red[g][lane];
                const float4 b = red[g + h][lane];
                comp_add(a.x, a.y, b.x, b.y);
                comp_add(a.z, a.w, b.z, b.w);
                red[g][lane] = a;
            }
            __syncthreads();
        }
        if (g == 0 && w < MN) {
            const float4 r = red[0][lane];
            C[(int64_t)(w / M) * ldc + (w % M)] = make_double2((double)r.x + (double)r.y, (double)r.z + (double)r.w);
        }
    } else {
        __shared__ double2 red[kSumGroups][32];
        double2 r = make_double2(0.0, 0.0);
        if (w < MN) {
#pragma unroll 4
            for (int c = g; c < nchunk; c += kSumGroups) {
                const P v = part[(int64_t)c * MN + w];
                r.x += v.x;
                r.y += v.y;
            }
        }
        red[g][lane] = r;
        __syncthreads();
        // pairwise, in a fixed tree (five dependent levels instead of 32)
#pragma unroll
        for (int h = kSumGroups / 2; h > 0; h >>= 1) {
            if (g < h) {
                red[g][lane].x += red[g + h][lane].x;
                red[g][lane].y += red[g + h][lane].y;
            }
            __syncthreads();
        }
        if (g == 0 && w < MN) C[(int64_t)(w / M) * ldc + (w % M)] = red[0][lane];
    }
}

template <typename P>
static void chunk_sum_t(int M, int N, int nchunk, const P* part, double2* C, int ldc, cudaStream_t st) {
    const int MN = M * N;
    roks::count_launch(), k_chunk_sum<P><<<(MN + 31) / 32, 32 * kSumGroups, 0, st>>>(M, MN, nchunk, part, C, ldc);
}

void chunk_sum(int M, int N, int nchunk, const double2* part, double2* C, int ldc, cudaStream_t st) {
    chunk_sum_t<double2>(M, N, nchunk, part, C, ldc, st);
}

void chunk_sum_f32(int M, int N, int nchunk, const float2* part, double2* C, int ldc, cudaStream_t st) {
    chunk_sum_t<float2>(M, N, nchunk, part, C, ldc, st);
}

namespace {
struct CnPlan {
    int rm, rn, ty, tx, mt, nt, kchunk, nchunk;
};

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

// register-tile shapes: all of 1..4 x 1..4, and with 6 in FP32 only
#define CN_TILES4(X) X(1, 1) X(1, 2) X(1, 3) X(1, 4) X(2, 1) X(2, 2) X(2, 3) X(2, 4) \
                     X(3, 1) X(3, 2) X(3, 3) X(3, 4) X(4, 1) X(4, 2) X(4, 3) X(4, 4)
#define CN_TILES6(X) X(1, 6) X(2, 6) X(3, 6) X(4, 6) X(6, 1) X(6, 2) X(6, 3) X(6, 4) X(6, 6)

constexpr int padgroup_rt(int r) { return (r % 2 == 0) ? r + 1 : r; }

// odd row strides of the k slices for a thread grid, and the dynamic
// shared memory of a launch (two slices of A and B, or the output tile)
template <typename T>
void cn_layout(const CnPlan& p, int& SA, int& SB, size_t& smem) {
    constexpr int KT = CnTile<T>::KT;
    SA = (p.ty * padgroup_rt(p.rm)) | 1;
    SB = (p.tx * padgroup_rt(p.rn)) | 1;
    const size_t slices = (size_t)2 * KT * (SA + SB);
    const size_t tile = (size_t)p.ty * p.rm * p.tx * p.rn;
    smem = sizeof(c2<T>) * (slices > tile ? slices : tile);
}

template <typename T, int RM, int RN>
size_t cn_smem_max() {
    constexpr int KT = CnTile<T>::KT;
    const size_t slices = (size_t)2 * KT * (padstride<RM>() + padstride<RN>());
    const size_t tile = (size_t)16 * RM * 16 * RN;
    return sizeof(c2<T>) * (slices > tile ? slices : tile);
}

template <typename T, int RM, int RN>
void cn_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_gemm_cn<T, RM, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)cn_smem_max<T, RM, RN>());
        done = true;
    }
}

// Blocks of the chosen contraction kernel resident on one SM (occupancy API),
// so that the split-K grid fills whole waves of the GPU.
template <typename T>
int cn_resident_blocks(int rm, int rn, int threads, size_t smem) {
    // cached per (tile, block size, shared memory): the first call of each shape queries
    struct Ent {
        int rm, rn, threads;
        size_t smem;
        int nb;
    };
    static std::vector<Ent> cache;
    static std::mutex mu;
    {
        std::lock_guard<std::mutex> g(mu);
        for (const Ent& c : cache)
            if (c.rm == rm && c.rn == rn && c.threads == threads && c.smem == smem) return c.nb;
    }
    int nb = 0;
    cudaError_t e = cudaErrorInvalidValue;
#define CN_OCC(RM_, RN_)                                                                              \
    if (rm == RM_ && rn == RN_) {                                                                   \
        cn_attr<T, RM_, RN_>();                                                                     \
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_gemm_cn<T, RM_, RN_>, threads, smem); \
    }
    CN_TILES4(CN_OCC)
    if constexpr (sizeof(T) == 4) { CN_TILES6(CN_OCC) }
#undef CN_OCC
    if (e != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 2;
    }
    std::lock_guard<std::mutex> g(mu);
    cache.push_back(Ent{rm, rn, threads, smem, nb});
    return nb;
}

// Register tile and thread grid with the least padded work (plus the
// shared-memory loads per multiply-add), then K chunks for whole waves of
// resident blocks, each at least two K slices long.
template <typename T>
CnPlan cn_plan(int M, int N, int K, int max_chunks) {
    constexpr int KT = CnTile<T>::KT;
    CnPlan best{};
    double best_cost = 1e300;
    // register tiles up to 4 x 4 (6-wide tiles, compiled for FP32, measured no
    // faster on these shapes: the kernel is issue-bound at any tile size)
    const int rcand[5] = {1, 2, 3, 4, 6};
    const int nc = 4;
    for (int ia = 0; ia < nc; ++ia)
        for (int ib = 0; ib < nc; ++ib) {
            const int rm = rcand[ia], rn = rcand[ib];
            const int mt = (M + 16 * rm - 1) / (16 * rm), nt = (N + 16 * rn - 1) / (16 * rn);
            const int ty = (M + mt * rm - 1) / (mt * rm), tx = (N + nt * rn - 1) / (nt * rn);
            const double covered = (double)mt * ty * rm * nt * tx * rn;
            double cost = covered * (1.0 + (rm + rn) / (4.0 * rm * rn));
            if (ty * tx < 64) cost *= 1.5;   // too few threads per block to hide latency
            if (cost < best_cost) {
                best_cost = cost;
                best = CnPlan{rm, rn, ty, tx, mt, nt, 0, 0};
            }
        }
    const int tiles = best.mt * best.nt;
    int SA = 0, SB = 0;
    size_t smem = 0;
    cn_layout<T>(best, SA, SB, smem);
    int want = (cn_resident_blocks<T>(best.rm, best.rn, best.ty * best.tx, smem) * sm_count() + tiles - 1) / tiles;
    const int by_len = (K + 2 * KT - 1) / (2 * KT);
    if (want > by_len) want = by_len;
    if (max_chunks > 0 && want > max_chunks) want = max_chunks;
    if (want < 1) want = 1;
    int kc = (K + want - 1) / want;
    kc = ((kc + KT - 1) / KT) * KT;
    if (kc < KT) kc = KT;
    best.kchunk = kc;
    best.nchunk = K > 0 ? (K + kc - 1) / kc : 1;
    return best;
}

template <typename T, int RM, int RN>
void launch_cn(const CnPlan& p, int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb,
               c2<T>* part, cudaStream_t st) {
    int SA = 0, SB = 0;
    size_t smem = 0;
    cn_layout<T>(p, SA, SB, smem);
    cn_attr<T, RM, RN>();
    dim3 g(p.mt, p.nt, p.nchunk);
    roks::count_launch();
    k_gemm_cn<T, RM, RN><<<g, p.ty * p.tx, smem, st>>>(M, N, K, p.kchunk, p.ty, p.tx, SA, SB, A, lda, B, ldb, part);
}

template <typename T>
void run_cn(const CnPlan& p, int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb,
            double2* C, int ldc, double2* work, cudaStream_t st) {
    c2<T>* part = reinterpret_cast<c2<T>*>(work);
    if (K <= 0) {
        cudaMemsetAsync(part, 0, sizeof(c2<T>) * M * N, st);
    } else {
#define CN_CASE(RM_, RN_) \
    if (p.rm == RM_ && p.rn == RN_) launch_cn<T, RM_, RN_>(p, M, N, K, A, lda, B, ldb, part, st);
        CN_TILES4(CN_CASE)
        if constexpr (sizeof(T) == 4) { CN_TILES6(CN_CASE) }
#undef CN_CASE
    }
    chunk_sum_t<c2<T>>(M, N, K > 0 ? p.nchunk : 1, part, C, ldc, st);
}
}  // namespace

// Partial-sum buffer of a contraction, in double2 elements (enough for
// either precision).
size_t gemm_cn_work(int M, int N, int K) {
    const CnPlan a = cn_plan<float>(M, N, K, 0), b = cn_plan<double>(M, N, K, 0);
    const int nc = a.nchunk > b.nchunk ? a.nchunk : b.nchunk;
    return (size_t)nc * M * N;
}

template <typename T>
void gemm_cn(int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb, double2* C, int ldc,
             double2* work, size_t work_elems, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    const int max_chunks = (int)(work_elems / ((size_t)M * N));
    if constexpr (sizeof(T) == 4) {
        // mixed path: large blocks on the tcgen05 tensor cores, the rest on
        // the TMA-streamed SIMT kernel
        if (gemm_cn_tcg(M, N, K, reinterpret_cast<const float2*>(A), lda, reinterpret_cast<const float2*>(B), ldb, C,
                        ldc, work, work_elems * sizeof(double2), st))
            return;
        if (gemm_cn_stream(M, N, K, reinterpret_cast<const float2*>(A), lda, reinterpret_cast<const float2*>(B), ldb,
                           C, ldc, work, work_elems, st))
            return;
    }
    run_cn<T>(cn_plan<T>(M, N, K, max_chunks), M, N, K, A, lda, B, ldb, C, ldc, work, st);
}

// Same contraction with the number of K chunks capped at max_chunks, for
// callers whose partial-sum buffer has a fixed size (max_chunks * M * N
// double2).
template <typename T>
void gemm_cn_capped(int M, int N, int K, const c2<T>* A, int64_t lda, const c2<T>* B, int64_t ldb, double2* C,
                    int ldc, double2* work, int max_chunks, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    run_cn<T>(cn_plan<T>(M, N, K, max_chunks), M, N, K, A, lda, B, ldb, C, ldc, work, st);
}

template void gemm_cn_capped<float>(int, int, int, const float2*, int64_t, const float2*, int64_t, double2*, int,
                                    double2*, int, cudaStream_t);
template void gemm_cn_capped<double>(int, int, int, const double2*, int64_t, const double2*, int64_t, double2*, int,
                                     double2*, int, cudaStream_t);

// ------------------------------------------------------------------ C = alpha A B + beta C
// A: M x K (tall, column major), B: K x N (small, element type T).  A block
// of 32 x TY threads owns (32 RM) rows x (TY RN) columns; thread (tx, ty)
// keeps rows m0 + tx + 32 i and columns n0 + ty RN + j.  K slices of 16 are
// double-buffered in shared memory by cp.async.
constexpr int NN_KT = 16;

template <typename T, int RM, int RN>
__global__ void __launch_bounds__(256) k_gemm_nn(int M, int N, int K, int TY, const c2<T>* __restrict__ A,
                                                 int64_t lda, const c2<T>* __restrict__ B, int ldb,
                                                 c2<T>* __restrict__ C, int64_t ldc, T alpha, T beta) {
    using V = c2<T>;
    constexpr int TM = 32 * RM, SBN = 8 * RN + 1;   // odd B stride: conflict-free transposed staging
    extern __shared__ __align__(16) unsigned char nn_smem[];
    V* As = reinterpret_cast<V*>(nn_smem);   // [2][NN_KT][TM]
    V* Bs = As + 2 * NN_KT * TM;             // [2][NN_KT][SBN]
    V* Cs = Bs + 2 * NN_KT * SBN;            // [SBN][TM]: beta C, staged before the main loop
    const int nthr = 32 * TY, tid = threadIdx.x;
    const int tx = tid & 31, ty = tid >> 5;
    const int TN = TY * RN;
    const int m0 = blockIdx.x * TM, n0 = blockIdx.y * TN;
    const int nk = (K + NN_KT - 1) / NN_KT;

    auto stage_in = [&](int s, int k0) {
        V* as = As + s * NN_KT * TM;
        V* bs = Bs + s * NN_KT * SBN;
        for (int e = tid; e < NN_KT * TM; e += nthr) {
            const int kk = e / TM, r = e - kk * TM;
            const int m = m0 + r, k = k0 + kk;
            const bool ok = m < M && k < K;
            cp_elem<T>(as + e, ok ? A + (int64_t)k * lda + m : A, ok);
        }
        for (int e = tid; e < NN_KT * TN; e += nthr) {
            const int c = e / NN_KT, kk = e % NN_KT;
            const int n = n0 + c, k = k0 + kk;
            const bool ok = n < N && k < K;
            cp_elem<T>(bs + kk * SBN + c, ok ? B + (int64_t)n * ldb + k : B, ok);
        }
        cp_commit();
    };

    V acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = mk<T>(T(0), T(0));
    // beta C is copied to shared memory asynchronously before the main loop,
    // so its loads overlap the contraction instead of waiting one by one
    // behind the stores of C in the epilogue
    if (beta != T(0)) {
        for (int e = tid; e < TN * TM; e += nthr) {
            const int c = e / TM, r = e - c * TM;
            const int m = m0 + r, n = n0 + c;
            const bool ok = m < M && n < N;
            cp_elem<T>(Cs + e, ok ? C + (int64_t)n * ldc + m : C, ok);
        }
    }
    cp_commit();
    if (nk > 0) stage_in(0, 0);
    for (int t = 0; t < nk; ++t) {
        if (t + 1 < nk) {
            stage_in((t + 1) & 1, (t + 1) * NN_KT);
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        const V* as = As + (t & 1) * NN_KT * TM + tx;
        const V* bs = Bs + (t & 1) * NN_KT * SBN + ty * RN;
#pragma unroll 4
        for (int kk = 0; kk < NN_KT; ++kk) {
            V a[RM], b[RN];
#pragma unroll
            for (int i = 0; i < RM; ++i) a[i] = as[kk * TM + 32 * i];
#pragma unroll
            for (int j = 0; j < RN; ++j) b[j] = bs[kk * SBN + j];
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) mac_nn<T>(acc[i][j], a[i], b[j]);
        }
        __syncthreads();
    }
    cp_wait<0>();
    __syncthreads();
#pragma unroll
    for (int i = 0; i < RM; ++i) {
        const int m = m0 + tx + 32 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < RN; ++j) {
            const int n = n0 + ty * RN + j;
            if (n < N) {
                V r = cscale(acc[i][j], alpha);
                if (beta != T(0)) r = cadd(r, cscale(Cs[(ty * RN + j) * TM + tx + 32 * i], beta));
                C[(int64_t)n * ldc + m] = r;
            }
        }
    }
}

// FP64 small matrix (K x N, ldb) -> contiguous FP32 copy (K x N, ld K)
__global__ void k_b_to_f32(int K, int N, const double2* __restrict__ B, int ldb, float2* __restrict__ Bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * N) return;
    const int n = i / K, k = i - n * K;
    const double2 v = B[(int64_t)n * ldb + k];
    Bf[i] = make_float2((float)v.x, (float)v.y);
}

namespace {
template <typename T, int RN>
void launch_nn(int M, int N, int K, int ty, int nt, const c2<T>* A, int64_t lda, const c2<T>* B, int ldb, c2<T>* C,
               int64_t ldc, T alpha, T beta, cudaStream_t st) {
    constexpr int RM = 4;
    const size_t smem = sizeof(c2<T>) * (2 * NN_KT * (32 * RM + 8 * RN + 1) + (size_t)(8 * RN) * (32 * RM));
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_gemm_nn<T, RM, RN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        attr = true;
    }
    dim3 g((M + 32 * RM - 1) / (32 * RM), nt);
    roks::count_launch();
    k_gemm_nn<T, RM, RN><<<g, 32 * ty, smem, st>>>(M, N, K, ty, A, lda, B, ldb, C, ldc, alpha, beta);
}
}  // namespace

template <typename T>
void gemm_nn(int M, int N, int K, const c2<T>* A, int64_t lda, const double2* B, int ldb, c2<T>* C, int64_t ldc,
             double alpha, double beta, void* bwork, cudaStream_t st, size_t bwork_bytes) {
    if (M <= 0 || N <= 0) return;
    if constexpr (sizeof(T) == 4) {
        if (bwork_bytes > 0 &&
            gemm_nn_tcg(M, N, K, reinterpret_cast<const float2*>(A), lda, B, ldb,
                        beta != 0.0 ? reinterpret_cast<const float2*>(C) : nullptr, ldc, reinterpret_cast<float2*>(C),
                        ldc, (float)alpha, (float)beta, bwork, bwork_bytes, st))
            return;
    }
    // column tiles of at most 64: RN = ceil(tile / 8) columns per thread, TY <= 8 warps
    const int nt = (N + 63) / 64;
    const int tn = (N + nt - 1) / nt;
    const int rn = (tn + 7) / 8;
    const int ty = (tn + rn - 1) / rn;
    const c2<T>* Bt;
    int ldbt;
    if constexpr (sizeof(T) == 4) {
        if (gemm_nn_stream(M, N, K, reinterpret_cast<const float2*>(A), lda, B, ldb, bwork,
                           reinterpret_cast<const float2*>(C), ldc, reinterpret_cast<float2*>(C), ldc, (float)alpha,
                           (float)beta, st))
            return;
        float2* Bf = static_cast<float2*>(bwork);
        if (K > 0) {
            roks::count_launch();
            k_b_to_f32<<<(K * N + 255) / 256, 256, 0, st>>>(K, N, B, ldb, Bf);
        }
        Bt = Bf;
        ldbt = K;
    } else {
        Bt = B;
        ldbt = ldb;
    }
#define NN_CASE(RN_) \
    if (rn == RN_) launch_nn<T, RN_>(M, N, K, ty, nt, A, lda, Bt, ldbt, C, ldc, T(alpha), T(beta), st);
    NN_CASE(1) NN_CASE(2) NN_CASE(3) NN_CASE(4) NN_CASE(5) NN_CASE(6) NN_CASE(7) NN_CASE(8)
#undef NN_CASE
}

template <typename T>
void gemm_nn_io(int M, int N, int K, const c2<T>* A, int64_t lda, const double2* B, int ldb, const c2<T>* Cin,
                int64_t ldcin, c2<T>* Cout, int64_t ldc, double alpha, double beta, void* bwork, cudaStream_t st,
                size_t bwork_bytes) {
    if (M <= 0 || N <= 0) return;
    if constexpr (sizeof(T) == 4) {
        if (bwork_bytes > 0 &&
            gemm_nn_tcg(M, N, K, reinterpret_cast<const float2*>(A), lda, B, ldb, reinterpret_cast<const float2*>(Cin),
                        ldcin, reinterpret_cast<float2*>(Cout), ldc, (float)alpha, (float)beta, bwork, bwork_bytes,
                        st))
            return;
        if (gemm_nn_stream(M, N, K, reinterpret_cast<const float2*>(A), lda, B, ldb, bwork,
                           reinterpret_cast<const float2*>(Cin), ldcin, reinterpret_cast<float2*>(Cout), ldc,
                           (float)alpha, (float)beta, st))
            return;
    }
    if (beta != 0.0 && (Cin != Cout || ldcin != ldc))
        cudaMemcpy2DAsync(Cout, ldc * sizeof(c2<T>), Cin, ldcin * sizeof(c2<T>), M * sizeof(c2<T>), N,
                          cudaMemcpyDeviceToDevice, st);
    gemm_nn<T>(M, N, K, A, lda, B, ldb, Cout, ldc, alpha, beta, bwork, st, 0);
}

template void gemm_nn_io<float>(int, int, int, const float2*, int64_t, const double2*, int, const float2*, int64_t,
                                float2*, int64_t, double, double, void*, cudaStream_t, size_t);
template void gemm_nn_io<double>(int, int, int, const double2*, int64_t, const double2*, int, const double2*,
                                 int64_t, double2*, int64_t, double, double, void*, cudaStream_t, size_t);

template void gemm_cn<float>(int, int, int, const float2*, int64_t, const float2*, int64_t, double2*, int,
                             double2*, size_t, cudaStream_t);
template void gemm_cn<double>(int, int, int, const double2*, int64_t, const double2*, int64_t, double2*, int,
                              double2*, size_t, cudaStream_t);
template void gemm_nn<float>(int, int, int, const float2*, int64_t, const double2*, int, float2*, int64_t, double,
                             double, void*, cudaStream_t, size_t);
template void gemm_nn<double>(int, int, int, const double2*, int64_t, const double2*, int, double2*, int64_t,
                              double, double, void*, cudaStream_t, size_t);

// ------------------------------------------------------------------ small FP64 matrices
// One warp per output element; the lanes split K and reduce with shuffles.
__global__ void k_small_gemm(int M, int N, int K, const double2* __restrict__ A, int lda, int ca,
                             const double2* __restrict__ B, int ldb, int cb, double2* __restrict__ C, int ldc,
                             double alpha, double beta) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= M * N) return;
    const int m = warp % M, n = warp / M;
    double sr = 0.0, si = 0.0;
    for (int k = lane; k < K; k += 32) {
        double2 a = ca ? A[(int64_t)m * lda + k] : A[(int64_t)k * lda + m];
        double2 b = cb ? B[(int64_t)k * ldb + n] : B[(int64_t)n * ldb + k];
        if (ca) a.y = -a.y;
        if (cb) b.y = -b.y;
        sr += a.x * b.x - a.y * b.y;
        si += a.x * b.y + a.y * b.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane != 0) return;
    double2* c = C + (int64_t)n * ldc + m;
    double2 r = make_double2(alpha * sr, alpha * si);
    if (beta != 0.0) { r.x += beta * c->x; r.y += beta * c->y; }
    *c = r;
}

// ------------------------------------------------------------------ large band-space products
// C = alpha op(A) op(B) + beta C on FP64 storage, for products too large for
// one warp per element (hundreds of bands, thousands of projectors): 32 x 32
// output tiles per block of 256 threads (enough blocks to fill the GPU at a
// few hundred bands), thread (tx, ty) owning rows ty + 16 i and columns
// tx + 16 j (i, j < 2); K in slices of 16 staged in shared memory, each load
// coalesced along the operand's contiguous index.  Arithmetic type R (float
// on the mixed path): every slice is summed on its own before it joins the
// running sum, so that rounding grows with K / 16.  TI: the stored operand
// type (double2, or float2 packed once by k_pack_f32 on the mixed path, so
// that the FP64 -> FP32 conversions, which run on the narrow FP64 pipe, are
// made once per element instead of once per output tile).
constexpr int BS_T = 32, BS_K = 16, BS_R = 2;

template <typename R, typename TI>
__global__ void __launch_bounds__(256) k_bs_gemm(int M, int N, int K, const TI* __restrict__ A, int lda,
                                                 int ca, const TI* __restrict__ B, int ldb, int cb,
                                                 double2* __restrict__ C, int ldc, double alpha, double beta) {
    __shared__ c2<R> As[BS_K][BS_T + 1];
    __shared__ c2<R> Bs[BS_K][BS_T + 1];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * BS_T, n0 = blockIdx.y * BS_T;
    c2<R> acc[BS_R][BS_R];
#pragma unroll
    for (int i = 0; i < BS_R; ++i)
#pragma unroll
        for (int j = 0; j < BS_R; ++j) acc[i][j].x = acc[i][j].y = R(0);
    for (int k0 = 0; k0 < K; k0 += BS_K) {
        for (int e = tid; e < BS_T * BS_K; e += 256) {
            // op(A)[m][k]: A^H of a K x M matrix (k contiguous) or an M x K one (m contiguous)
            const int ka = ca ? e % BS_K : e / BS_T, ma = ca ? e / BS_K : e % BS_T;
            c2<R> v;
            v.x = v.y = R(0);
            if (m0 + ma < M && k0 + ka < K) {
                const TI d = ca ? A[(int64_t)(m0 + ma) * lda + k0 + ka] : A[(int64_t)(k0 + ka) * lda + m0 + ma];
                v.x = (R)d.x;
                v.y = ca ? -(R)d.y : (R)d.y;
            }
            As[ka][ma] = v;
            // op(B)[k][n]: B^H of an N x K matrix (n contiguous) or a K x N one (k contiguous)
            const int kb = cb ? e / BS_T : e % BS_K, nb = cb ? e % BS_T : e / BS_K;
            c2<R> w;
            w.x = w.y = R(0);
            if (n0 + nb < N && k0 + kb < K) {
                const TI d = cb ? B[(int64_t)(k0 + kb) * ldb + n0 + nb] : B[(int64_t)(n0 + nb) * ldb + k0 + kb];
                w.x = (R)d.x;
                w.y = cb ? -(R)d.y : (R)d.y;
            }
            Bs[kb][nb] = w;
        }
        __syncthreads();
        c2<R> t[BS_R][BS_R];
#pragma unroll
        for (int i = 0; i < BS_R; ++i)
#pragma unroll
            for (int j = 0; j < BS_R; ++j) t[i][j].x = t[i][j].y = R(0);
#pragma unroll 4
        for (int kk = 0; kk < BS_K; ++kk) {
            c2<R> a[BS_R], b[BS_R];
#pragma unroll
            for (int i = 0; i < BS_R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < BS_R; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < BS_R; ++i)
#pragma unroll
                for (int j = 0; j < BS_R; ++j) mac_nn<R>(t[i][j], a[i], b[j]);
        }
#pragma unroll
        for (int i = 0; i < BS_R; ++i)
#pragma unroll
            for (int j = 0; j < BS_R; ++j) {
                acc[i][j].x += t[i][j].x;
                acc[i][j].y += t[i][j].y;
            }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < BS_R; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < BS_R; ++j) {
            const int n = n0 + tx + 16 * j;
            if (n >= N) continue;
            double2* c = C + (int64_t)n * ldc + m;
            double2 r = make_double2(alpha * (double)acc[i][j].x, alpha * (double)acc[i][j].y);
            if (beta != 0.0) {
                r.x += beta * c->x;
                r.y += beta * c->y;
            }
            *c = r;
        }
    }
}

// Products with at least this many outputs (and 32 or more terms each) go to
// the tiled kernel; smaller ones keep one warp per element.
static bool bs_tiled(int M, int N, int K) { return (long long)M * N >= 16384 && K >= 32; }

template <typename R>
static void bs_gemm(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb, bool cb,
             double2* C, int ldc, double alpha, double beta, cudaStream_t st) {
    const dim3 g((unsigned)((M + BS_T - 1) / BS_T), (unsigned)((N + BS_T - 1) / BS_T));
    roks::count_launch();
    k_bs_gemm<R, double2><<<g, 256, 0, st>>>(M, N, K, A, lda, ca ? 1 : 0, B, ldb, cb ? 1 : 0, C, ldc, alpha, beta);
}

// dst (rows x cols, leading dimension rows) = src (FP64, leading dimension ld) in FP32
__global__ void k_pack_f32(int rows, int cols, const double2* __restrict__ src, int ld, float2* __restrict__ dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)rows * cols) return;
    const int r = (int)(i % rows), c = (int)(i / rows);
    const double2 v = src[(int64_t)c * ld + r];
    dst[i] = make_float2((float)v.x, (float)v.y);
}

// op(A): A (M x K) or A^H when ca (A stored K x M); op(B) likewise.
void small_gemm(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb, bool cb,
                double2* C, int ldc, double alpha, double beta, cudaStream_t st) {
    if (M <= 0 || N <= 0) return;
    if (bs_tiled(M, N, K)) {
        bs_gemm<double>(M, N, K, A, lda, ca, B, ldb, cb, C, ldc, alpha, beta, st);
        return;
    }
    const long long threads = (long long)M * N * 32;
    roks::count_launch(), k_small_gemm<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, N, K, A, lda, ca, B, ldb, cb, C, ldc, alpha, beta);
}

// Same product with FP32 arithmetic on FP64 storage (the mixed-precision
// path): the conversions are once per loaded element, the dot products and
// the shuffle reduction in FP32, alpha and beta applied in FP64.
__global__ void k_small_gemm_f32(int M, int N, int K, const double2* __restrict__ A, int lda, int ca,
                                 const double2* __restrict__ B, int ldb, int cb, double2* __restrict__ C, int ldc,
                                 double alpha, double beta) {
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= M * N) return;
    const int m = warp % M, n = warp / M;
    float sr = 0.f, si = 0.f;
    for (int k = lane; k < K; k += 32) {
        const double2 ad = ca ? A[(int64_t)m * lda + k] : A[(int64_t)k * lda + m];
        const double2 bd = cb ? B[(int64_t)k * ldb + n] : B[(int64_t)n * ldb + k];
        const float ax = (float)ad.x, ay = ca ? -(float)ad.y : (float)ad.y;
        const float bx = (float)bd.x, by = cb ? -(float)bd.y : (float)bd.y;
        sr = fmaf(ax, bx, sr);
        sr = fmaf(-ay, by, sr);
        si = fmaf(ax, by, si);
        si = fmaf(ay, bx, si);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
    }
    if (lane != 0) return;
    double2* c = C + (int64_t)n * ldc + m;
    double2 r = make_double2(alpha * (double)sr, alpha * (double)si);
    if (beta != 0.0) {
        r.x += beta * c->x;
        r.y += beta * c->y;
    }
    *c = r;
}

void small_gemm_f32(int M, int N, int K, const double2* A, int lda, bool ca, const double2* B, int ldb, bool cb,
                    double2* C, int ldc, double alpha, double beta, cudaStream_t st, void* work, size_t work_bytes) {
    if (M <= 0 || N <= 0) return;
    if (bs_tiled(M, N, K)) {
        // the stored shapes of A (K x M for A^H, else M x K) and B (N x K for B^H, else K x N)
        const int ra = ca ? K : M, na = ca ? M : K, rb = cb ? N : K, nbc = cb ? K : N;
        const size_t need = sizeof(float2) * ((size_t)ra * na + (size_t)rb * nbc);
        if (work && need <= work_bytes) {
            float2* Ap = static_cast<float2*>(work);
            float2* Bp = Ap + (size_t)ra * na;
            const int64_t ta = (int64_t)ra * na, tb = (int64_t)rb * nbc;
            roks::count_launch(), k_pack_f32<<<(unsigned)((ta + 255) / 256), 256, 0, st>>>(ra, na, A, lda, Ap);
            roks::count_launch(), k_pack_f32<<<(unsigned)((tb + 255) / 256), 256, 0, st>>>(rb, nbc, B, ldb, Bp);
            const dim3 g((unsigned)((M + BS_T - 1) / BS_T), (unsigned)((N + BS_T - 1) / BS_T));
            roks::count_launch();
            k_bs_gemm<float, float2><<<g, 256, 0, st>>>(M, N, K, Ap, ra, ca ? 1 : 0, Bp, rb, cb ? 1 : 0, C, ldc, alpha,
                                                        beta);
        } else {
            bs_gemm<float>(M, N, K, A, lda, ca, B, ldb, cb, C, ldc, alpha, beta, st);
        }
        return;
    }
    const long long threads = (long long)M * N * 32;
    roks::count_launch(), k_small_gemm_f32<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(
                              M, N, K, A, lda, ca, B, ldb, cb, C, ldc, alpha, beta);
}

// Cholesky inverse held in shared memory (n <= kSmallN), FP64: right-looking
// factorisation O = L L^H (two barriers per column), then X = L^{-1} by
// forward substitution with one warp per column (lanes split the dot
// products); LinvH = X^H.
constexpr int kSmallN = 64;

__global__ void __launch_bounds__(1024) k_cholesky_small(int n, const double2* __restrict__ O,
                                                         double2* __restrict__ LinvH, int* flag) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2* L = reinterpret_cast<double2*>(smem_raw);          // n x n, column major
    double2* X = L + n * n;                                      // n x n, column major
    __shared__ int bad;
    __shared__ double dinv[kSmallN];                             // 1 / L_jj
    if (threadIdx.x == 0) bad = 0;
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        L[idx] = O[idx];
        X[idx] = make_double2(0.0, 0.0);
    }
    __syncthreads();
    // FP64 throughput is a per-SM resource: the pivot square root and
    // reciprocal are computed once, by one thread, not by every thread.
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x == 0) {
            double d = L[j * n + j].x;
            if (!(d > 0.0)) {
                if (!bad) bad = j + 1;
                d = 1.0;
            }
            const double piv = sqrt(d);
            L[j * n + j] = make_double2(piv, 0.0);
            dinv[j] = 1.0 / piv;
        }
        __syncthreads();
        const double inv = dinv[j];
        for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
            const double2 v = L[j * n + i];
            L[j * n + i] = make_double2(v.x * inv, v.y * inv);
        }
        __syncthreads();
        // trailing update A_ik -= L_ij conj(L_kj), j < k <= i
        const int m = n - j - 1;
        for (int t = threadIdx.x; t < m * m; t += blockDim.x) {
            const int k = t / m;
            const int i = t - k * m;
            if (k > i) continue;
            const double2 a = L[j * n + j + 1 + i], b = L[j * n + j + 1 + k];
            double2 c = L[(j + 1 + k) * n + j + 1 + i];
            c.x -= a.x * b.x + a.y * b.y;
            c.y -= a.y * b.x - a.x * b.y;
            L[(j + 1 + k) * n + j + 1 + i] = c;
        }
        __syncthreads();
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < n; c += nw) {
        for (int i = c; i < n; ++i) {
            double sr = 0.0, si = 0.0;
            for (int k = c + lane; k < i; k += 32) {
                const double2 l = L[k * n + i], x = X[c * n + k];
                sr += l.x * x.x - l.y * x.y;
                si += l.x * x.y + l.y * x.x;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                sr += __shfl_xor_sync(0xffffffffu, sr, o);
                si += __shfl_xor_sync(0xffffffffu, si, o);
            }
            if (lane == 0) {
                const double di = dinv[i];
                X[c * n + i] = make_double2(((i == c) ? 1.0 - sr : -sr) * di, -si * di);
            }
            __syncwarp();
        }
    }
    __syncthreads();
    // LinvH (row c, column i) = conj X (row i, column c)
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int c = idx % n, i = idx / n;
        const double2 x = X[c * n + i];
        LinvH[idx] = make_double2(x.x, -x.y);
    }
    if (threadIdx.x == 0 && bad) flag[0] = bad;
}

bool cholesky_small_supported(int n) { return n <= kSmallN; }

// Deviation form of the Cholesky inverse for O = I + Delta (FP32, one block,
// n <= kSmallN).  W holds the working lower triangle of Delta (its diagonal
// real), L = I + Lambda is built column by column with the pivot deviation
// lambda_jj = w / (1 + sqrt(1 + w)) (no cancellation), and the columns of
// Xi = L^{-1} - I solve (I + Lambda) xi_c = -Lambda e_c by a right-looking
// sweep, one warp per column.
constexpr int kCholFactorThreads = 256;   // threads of the factorisation steps
// NP: trailing-update pairs per factorisation thread, >= n (n - 1) / 2 / 256
template <int NP>
__global__ void __launch_bounds__(1024) k_cholesky_dev_f32(int n, const double2* __restrict__ O,
                                                           double2* __restrict__ XiH, int* flag) {
    constexpr int kCholPairs = NP;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* W = reinterpret_cast<float2*>(smem_raw);   // Delta (lower), updated in place
    float2* Lm = W + n * n;                             // Lambda (lower, diagonal deviation in .x)
    // trailing-update pairs (i, k), i >= k >= 1, by k descending: the pairs of
    // step j (k > j) are the first (n - 1 - j)(n - j) / 2
    int* pk = reinterpret_cast<int*>(Lm + n * n);
    __shared__ float dinv[kSmallN];
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int i = idx % n, j = idx / n;
        if (i < j) continue;
        // average of the two triangles, minus the identity, before rounding to FP32
        const double2 a = O[(int64_t)j * n + i], b = O[(int64_t)i * n + j];
        const double re = 0.5 * (a.x + b.x) - (i == j ? 1.0 : 0.0);
        const double im = i == j ? 0.0 : 0.5 * (a.y - b.y);
        W[idx] = make_float2((float)re, (float)im);
        if (j >= 1) {
            const int d = n - 1 - j;
            pk[d * (d + 1) / 2 + (i - j)] = (i << 8) | j;
        }
    }
    __syncthreads();
    int bad = 0;
    for (int j = 0; j < n; ++j) {
        if (threadIdx.x < kCholFactorThreads) {
            float w = W[j * n + j].x;
            if (!(1.f + w > 0.f)) {
                if (!bad) bad = j + 1;
                w = 0.f;
            }
            const float piv = sqrtf(1.f + w), inv = 1.f / piv, invd = inv * inv;
            if (threadIdx.x == 0) dinv[j] = inv;
            for (int i = j + threadIdx.x; i < n; i += kCholFactorThreads) {
                const float2 v = W[j * n + i];
                Lm[j * n + i] = (i == j) ? make_float2(w / (1.f + piv), 0.f) : make_float2(v.x * inv, v.y * inv);
            }
            // trailing update W(i, k) -= W(i, j) conj(W(k, j)) / (1 + w_jj), k > j, i >= k:
            // all loads of a thread first, then its stores (they never alias)
            const int npair = (n - 1 - j) * (n - j) / 2;
            int ii[kCholPairs], kk[kCholPairs];
            float2 a[kCholPairs], b[kCholPairs], c[kCholPairs];
#pragma unroll
            for (int q = 0; q < kCholPairs; ++q) {
                const int e = threadIdx.x + q * kCholFactorThreads;
                const int code = e < npair ? pk[e] : 0;
                ii[q] = code >> 8;
                kk[q] = code & 255;
                if (e < npair) {
                    a[q] = W[j * n + ii[q]];
                    b[q] = W[j * n + kk[q]];
                    c[q] = W[kk[q] * n + ii[q]];
                }
            }
#pragma unroll
            for (int q = 0; q < kCholPairs; ++q) {
                const int e = threadIdx.x + q * kCholFactorThreads;
                if (e < npair) {
                    float2 t = c[q];
                    t.x = fmaf(-(a[q].x * b[q].x + a[q].y * b[q].y), invd, t.x);
                    t.y = fmaf(-(a[q].y * b[q].x - a[q].x * b[q].y), invd, t.y);
                    W[kk[q] * n + ii[q]] = t;
                }
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && bad) flag[0] = bad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int c = warp; c < n; c += nw) {
        // right-hand side -Lambda e_c: rows lane and lane + 32
        float2 r0 = make_float2(0.f, 0.f), r1 = make_float2(0.f, 0.f);
        if (lane >= c && lane < n) r0 = make_float2(-Lm[c * n + lane].x, -Lm[c * n + lane].y);
        if (lane + 32 >= c && lane + 32 < n) r1 = make_float2(-Lm[c * n + lane + 32].x, -Lm[c * n + lane + 32].y);
        for (int k = c; k < n; ++k) {
            const float2 own = k < 32 ? r0 : r1;
            const float sx = __shfl_sync(0xffffffffu, own.x, k & 31);
            const float sy = __shfl_sync(0xffffffffu, own.y, k & 31);
            const float di = dinv[k];
            const float2 xk = make_float2(sx * di, sy * di);
            if (lane == (k & 31)) {
                if (k < 32) r0 = xk;
                else r1 = xk;
            }
            if (lane > k && lane < n) {
                const float2 l = Lm[k * n + lane];
                r0.x -= l.x * xk.x - l.y * xk.y;
                r0.y -= l.x * xk.y + l.y * xk.x;
            }
            if (lane + 32 > k && lane + 32 < n) {
                const float2 l = Lm[k * n + lane + 32];
                r1.x -= l.x * xk.x - l.y * xk.y;
                r1.y -= l.x * xk.y + l.y * xk.x;
            }
        }
        // XiH (row c, column i) = conj Xi (row i, column c); zero above the diagonal of Xi
        if (lane < n) {
            const float2 x = lane >= c ? r0 : make_float2(0.f, 0.f);
            XiH[(int64_t)lane * n + c] = make_double2((double)x.x, -(double)x.y);
        }
        if (lane + 32 < n) {
            const float2 x = lane + 32 >= c ? r1 : make_float2(0.f, 0.f);
            XiH[(int64_t)(lane + 32) * n + c] = make_double2((double)x.x, -(double)x.y);
        }
    }
}

void cholesky_dev_f32(int n, const double2* O, double2* XiH, int* flag, cudaStream_t st) {
    const size_t sm = sizeof(float2) * 2 * n * n + sizeof(int) * n * (n - 1) / 2;
    roks::count_launch();
    if (n * (n - 1) / 2 <= 4 * kCholFactorThreads) {
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(k_cholesky_dev_f32<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_cholesky_dev_f32<4><<<1, 1024, sm, st>>>(n, O, XiH, flag);
    } else {
        if (sm > 48 * 1024)
            cudaFuncSetAttribute(k_cholesky_dev_f32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        k_cholesky_dev_f32<8><<<1, 1024, sm, st>>>(n, O, XiH, flag);
    }
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
    if (n <= kSmallN) {
        const size_t sm = sizeof(double2) * 2 * n * n;
        if (sm > 48 * 1024) cudaFuncSetAttribute(k_cholesky_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        roks::count_launch(), k_cholesky_small<<<1, 1024, sm, st>>>(n, O, LinvH, flag);
        return;
    }
    roks::count_launch(), k_cholesky_inverse<<<1, 1024, 0, st>>>(n, O, Lw, LinvH, flag);
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


// exp(s A) for n <= kSmallN in single precision on one thread-block cluster:
// X = s A / 2^q (||s A||_1 / 2^q <= 1/4), Taylor degree 8 (truncation below
// 1e-11, so that the squarings amplify FP32 rounding alone), q squarings.
// Used by the mixed-precision path, whose orbitals are re-orthonormalised
// after every rotation.
//
// Every CTA of the cluster keeps all the n x n matrices (column major,
// leading dimension ldm) in its shared memory.  A product is split by
// columns: CTA r computes its slice, one output element per thread, and
// stores it into the shared memory of every CTA of the cluster; a cluster
// barrier then publishes the product.  Each output element is accumulated
// in the same order as by a single block, so the result does not depend on
// the cluster size.
constexpr int kExpmCluster = 8;
constexpr int kExpmThreads = 256;
namespace cg = cooperative_groups;

// C[:, c0:c1) = A B + a0 I + a1 X + a2 X2 (A, B may be null: no product),
// written to the C of every CTA in the cluster
__device__ __forceinline__ void cluster_mm_poly(cg::cluster_group& cluster, int n, int ldm, int c0, int c1,
                                                const float2* A, const float2* B, const float2* X,
                                                const float2* X2, float a0, float a1, float a2, float2* C) {
    const int cols = c1 - c0;
    for (int t = threadIdx.x; t < n * cols; t += blockDim.x) {
        const int m = t % n, c = c0 + t / n;
        const float2 x = X[c * ldm + m], x2 = X2[c * ldm + m];
        float2 v = make_float2((m == c ? a0 : 0.f) + a1 * x.x + a2 * x2.x, a1 * x.y + a2 * x2.y);
        if (A) {
#pragma unroll 6
            for (int k = 0; k < n; ++k) {
                const float2 a = A[k * ldm + m], b = B[c * ldm + k];
                v.x = fmaf(a.x, b.x, v.x);
                v.y = fmaf(a.x, b.y, v.y);
                v.x = fmaf(-a.y, b.y, v.x);
                v.y = fmaf(a.y, b.x, v.y);
            }
        }
#pragma unroll
        for (int r = 0; r < kExpmCluster; ++r) cluster.map_shared_rank(C, r)[c * ldm + m] = v;
    }
    cluster.sync();
}

__global__ void __cluster_dims__(kExpmCluster, 1, 1) __launch_bounds__(kExpmThreads)
    k_expm_small_f32(int n, const double2* __restrict__ A, const double* __restrict__ s, double2* __restrict__ E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cluster = cg::this_cluster();
    const int rank = (int)cluster.block_rank();
    const int ldm = (n + 1) & ~1;
    const int nn = ldm * ldm;
    float2* X = reinterpret_cast<float2*>(smem_raw);
    float2* X2 = X + nn;
    float2* X3 = X2 + nn;
    float2* T1 = X3 + nn;
    float2* T2 = T1 + nn;
    __shared__ float wmax[kExpmThreads / 32];
    __shared__ int qs;
    const int cp = (n + kExpmCluster - 1) / kExpmCluster;
    const int c0 = min(n, rank * cp), c1 = min(n, c0 + cp);
    for (int idx = threadIdx.x; idx < 5 * nn; idx += blockDim.x) X[idx] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
        const int r = idx % n, c = idx / n;
        const double2 a = A[idx];
        X[c * ldm + r] = make_float2((float)a.x, (float)a.y);
    }
    __syncthreads();
    // 1-norm (every CTA the same way): one warp per column, lanes over rows
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    float best = 0.f;
    for (int c = warp; c < n; c += nw) {
        float sum = 0.f;
        for (int r = lane; r < n; r += 32) {
            const float2 a = X[c * ldm + r];
            sum += sqrtf(a.x * a.x + a.y * a.y);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
        best = fmaxf(best, sum);
    }
    if (lane == 0) wmax[warp] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        float m = 0.f;
        for (int w = 0; w < nw; ++w) m = fmaxf(m, wmax[w]);
        float scaled = fabsf((float)s[0]) * m;
        int q = 0;
        while (scaled > 0.25f && q < 30) {
            scaled *= 0.5f;
            ++q;
        }
        qs = q;
    }
    __syncthreads();
    const int q = qs;
    const float f = (float)s[0] * ldexpf(1.f, -q);
    for (int idx = threadIdx.x; idx < nn; idx += blockDim.x) X[idx] = make_float2(f * X[idx].x, f * X[idx].y);
    // the peers write into this CTA's matrices from here on
    cluster.sync();
    constexpr float c3 = 1.f / 6.f, c4 = 1.f / 24.f, c5 = 1.f / 120.f, c6 = 1.f / 720.f, c7 = 1.f / 5040.f,
                    c8 = 1.f / 40320.f;
    cluster_mm_poly(cluster, n, ldm, c0, c1, X, X, X, X, 0.f, 0.f, 0.f, X2);                  // X^2
    cluster_mm_poly(cluster, n, ldm, c0, c1, X2, X, X, X2, 0.f, 0.f, 0.f, X3);                // X^3
    cluster_mm_poly(cluster, n, ldm, c0, c1, nullptr, nullptr, X, X2, c6, c7, c8, T1);        // B2
    cluster_mm_poly(cluster, n, ldm, c0, c1, X3, T1, X, X2, c3, c4, c5, T2);                  // B1 + X^3 B2
    cluster_mm_poly(cluster, n, ldm, c0, c1, X3, T2, X, X2, 1.f, 1.f, 0.5f, T1);              // B0 + X^3 (...)
    float2* P = T1;
    float2* Q = T2;
    for (int r = 0; r < q; ++r) {
        cluster_mm_poly(cluster, n, ldm, c0, c1, P, P, X, X2, 0.f, 0.f, 0.f, Q);
        float2* t = P;
        P = Q;
        Q = t;
    }
    for (int idx = threadIdx.x; idx < n * (c1 - c0); idx += blockDim.x) {
        const int r = idx % n, c = c0 + idx / n;
        const float2 v = P[c * ldm + r];
        E[(int64_t)c * n + r] = make_double2(v.x, v.y);
    }
}

bool expm_small_f32(int n, const double2* A, const double* scale_dev, double2* E, cudaStream_t st) {
    if (n > kSmallN) return false;
    const int ldm = (n + 1) & ~1;
    const size_t sm = sizeof(float2) * 5 * ldm * ldm;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_expm_small_f32, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(float2) * 5 * kSmallN * kSmallN));
        attr = true;
    }
    roks::count_launch(), k_expm_small_f32<<<kExpmCluster, kExpmThreads, sm, st>>>(n, A, scale_dev, E);
    return true;
}

void expm_scaled(int n, const double2* A, const double* scale_dev, double2* E, double2* w1, double2* w2,
                 double2* w3, double* sdev, cudaStream_t st) {
    roks::count_launch(), k_expm_scale<<<1, 256, 0, st>>>(n, A, scale_dev, w1, sdev);
    const int blocks = (n * n + 127) / 128;
    // Horner: E_deg = I + X / deg, ..., E_1 = I + X E_2
    double2* cur = w2;
    double2* nxt = w3;
    roks::count_launch(), k_expm_horner<<<blocks, 128, 0, st>>>(n, w1, nullptr, cur, 1.0 / kExpmDegree, 1);
    for (int k = kExpmDegree - 1; k >= 1; --k) {
        roks::count_launch(), k_expm_horner<<<blocks, 128, 0, st>>>(n, w1, cur, nxt, 1.0 / k, 0);
        double2* t = cur; cur = nxt; nxt = t;
    }
    for (int q = 0; q < kExpmMaxSquare; ++q) {
        double2* dst = (q == kExpmMaxSquare - 1) ? E : nxt;
        roks::count_launch(), k_expm_square<<<blocks, 128, 0, st>>>(n, cur, dst, q, sdev);
        if (q == kExpmMaxSquare - 1) break;
        double2* t = cur; cur = nxt; nxt = t;
    }
}

}  // namespace roks
