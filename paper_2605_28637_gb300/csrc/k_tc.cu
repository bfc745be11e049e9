// k_tc.cu -- complex contractions C = A^H B on the tcgen05 tensor cores
// (mixed-precision path).  A: K x M, B: K x N complex FP32, column major
// (K contiguous).  Real formulation: with a = (re, im) interleaved along K,
//   C_re[m, n] = sum over 2K reals of A'[m, :] . B'[n, :],
//   C_im[m, n] = sum over 2K reals of A'[m, :] . B''[n, :],
// where A' and B' are the columns as stored and B'' = (im, -re) pairs.  One
// MMA with a (2 N16)-row B operand [B'; B''] yields both.  Each FP32 value is
// split into three TF32 parts (hi + mid + lo, exact to 2^-33) and the six
// products down to that order (hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid)
// are accumulated in FP32 in tensor memory, so the contraction is as
// accurate as an FP32 one.  Split K over CTAs; partial sums in FP64 are
// reduced by the same fixed-order kernel as the SIMT contraction.
#include <atomic>
#include <cstdlib>

#include "roks_impl.cuh"
#include "tc_sm103.cuh"

namespace roks {

static __device__ int g_tc_timeout;        // set when an mbarrier wait gave up

namespace {

constexpr int TC_M = 128;                  // MMA rows (A tile)
constexpr int TC_KC = 16;                  // complex K elements per stage
constexpr int TC_KR = 2 * TC_KC;           // real K elements per stage (4 MMAs of K = 8)
constexpr uint32_t TC_WAIT = 1u << 26;     // mbarrier polls before giving up

// byte offset of element (row, kr) in the core-matrix layout of a tile with TC_KR reals per row
__device__ __forceinline__ uint32_t core_off(int row, int kr) {
    return (uint32_t)(((row >> 3) * (TC_KR / 4) + (kr >> 2)) * 128 + (row & 7) * 16 + (kr & 3) * 4);
}

template <int NP>
__global__ void __launch_bounds__(128) k_gemm_cn_tc(int M, int N, int K, int kchunk, const float2* __restrict__ A,
                                                    int64_t lda, const float2* __restrict__ B, int64_t ldb,
                                                    double2* __restrict__ part) {
    constexpr int N16 = NP / 2;
    constexpr uint32_t TCOLS = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : 256));
    constexpr int A_BYTES = TC_M * TC_KR * 4;
    constexpr int B_BYTES = NP * TC_KR * 4;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* Ahi = smem;
    unsigned char* Amd = Ahi + A_BYTES;
    unsigned char* Alo = Amd + A_BYTES;
    unsigned char* Bhi = Alo + A_BYTES;
    unsigned char* Bmd = Bhi + B_BYTES;
    unsigned char* Blo = Bmd + B_BYTES;
    __shared__ uint64_t mbar;
    __shared__ uint32_t tbase;
    __shared__ int failed;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TC_M;
    const int kbeg = blockIdx.z * kchunk, kend = min(K, kbeg + kchunk);

    if (warp == 0) tc::tmem_alloc(&tbase, TCOLS);
    if (tid == 0) {
        tc::mbar_init(&mbar, 1);
        tc::fence_mbar_init();
        failed = 0;
    }
    // zero the B tiles once: padding rows stay zero
    for (int i = tid; i < 3 * B_BYTES / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(Bhi)[i] = make_uint4(0, 0, 0, 0);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    const uint32_t idesc = tc::idesc_tf32(TC_M, NP);

    int stage = 0;
    for (int k0 = kbeg; k0 < kend; k0 += TC_KC, ++stage) {
        // ---- stage the A tile: 128 rows x 16 complex (split hi / lo)
        for (int i = tid; i < TC_M * TC_KC; i += blockDim.x) {
            const int row = i / TC_KC, kc = i % TC_KC;
            const int m = m0 + row, k = k0 + kc;
            float2 v = make_float2(0.f, 0.f);
            if (m < M && k < kend) v = A[(int64_t)m * lda + k];
            float hx, mx, lx, hy, my, ly;
            tc::split3_tf32(v.x, hx, mx, lx);
            tc::split3_tf32(v.y, hy, my, ly);
            const uint32_t off = core_off(row, 2 * kc);
            *reinterpret_cast<float2*>(Ahi + off) = make_float2(hx, hy);
            *reinterpret_cast<float2*>(Amd + off) = make_float2(mx, my);
            *reinterpret_cast<float2*>(Alo + off) = make_float2(lx, ly);
        }
        // ---- stage B' (rows 0..N-1) and B'' (rows N16..N16+N-1)
        for (int i = tid; i < N * TC_KC; i += blockDim.x) {
            const int n = i / TC_KC, kc = i % TC_KC;
            const int k = k0 + kc;
            float2 v = make_float2(0.f, 0.f);
            if (k < kend) v = B[(int64_t)n * ldb + k];
            float hx, mx, lx, hy, my, ly;
            tc::split3_tf32(v.x, hx, mx, lx);
            tc::split3_tf32(v.y, hy, my, ly);
            const uint32_t o1 = core_off(n, 2 * kc), o2 = core_off(N16 + n, 2 * kc);
            *reinterpret_cast<float2*>(Bhi + o1) = make_float2(hx, hy);
            *reinterpret_cast<float2*>(Bmd + o1) = make_float2(mx, my);
            *reinterpret_cast<float2*>(Blo + o1) = make_float2(lx, ly);
            *reinterpret_cast<float2*>(Bhi + o2) = make_float2(hy, -hx);
            *reinterpret_cast<float2*>(Bmd + o2) = make_float2(my, -mx);
            *reinterpret_cast<float2*>(Blo + o2) = make_float2(ly, -lx);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0 && !failed) {
            const uint32_t ah = tc::smem_u32(Ahi), am = tc::smem_u32(Amd), al = tc::smem_u32(Alo);
            const uint32_t bh = tc::smem_u32(Bhi), bm = tc::smem_u32(Bmd), bl = tc::smem_u32(Blo);
            constexpr uint32_t LBO = 128, SBO = (TC_KR / 4) * 128;
#pragma unroll
            for (int kk = 0; kk < TC_KR / 8; ++kk) {
                const uint32_t ko = kk * 2 * 128;   // 8 reals = two K chunks
                const uint32_t acc0 = (stage > 0 || kk > 0) ? 1u : 0u;
                // smallest terms first
                tc::mma_tf32(tmem, tc::make_desc(am + ko, LBO, SBO), tc::make_desc(bm + ko, LBO, SBO), idesc, acc0);
                tc::mma_tf32(tmem, tc::make_desc(ah + ko, LBO, SBO), tc::make_desc(bl + ko, LBO, SBO), idesc, 1u);
                tc::mma_tf32(tmem, tc::make_desc(al + ko, LBO, SBO), tc::make_desc(bh + ko, LBO, SBO), idesc, 1u);
                tc::mma_tf32(tmem, tc::make_desc(ah + ko, LBO, SBO), tc::make_desc(bm + ko, LBO, SBO), idesc, 1u);
                tc::mma_tf32(tmem, tc::make_desc(am + ko, LBO, SBO), tc::make_desc(bh + ko, LBO, SBO), idesc, 1u);
                tc::mma_tf32(tmem, tc::make_desc(ah + ko, LBO, SBO), tc::make_desc(bh + ko, LBO, SBO), idesc, 1u);
            }
            tc::commit(&mbar);
        }
        // every thread waits for the MMAs before the tiles are overwritten
        if (!tc::mbar_wait(&mbar, (uint32_t)(stage & 1), TC_WAIT)) {
            failed = 1;
            g_tc_timeout = 1;
        }
        tc::fence_after_sync();
        __syncthreads();
        if (failed) break;
    }
    if (failed && tid == 0) {
        // give MMAs still in flight a second bounded chance before freeing TMEM
        tc::mbar_wait(&mbar, (uint32_t)(stage & 1), TC_WAIT);
    }
    // ---- epilogue: warp w reads lanes 32 w .. 32 w + 31 (rows of C)
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (!failed && stage > 0) {
        const int m = m0 + 32 * warp + lane;
        double2* P = part + (int64_t)blockIdx.z * M * N;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * warp) << 16);
        for (int n0 = 0; n0 < N; n0 += 8) {
            float re[8], im[8];
            tc::tmem_ld8(lane_addr + (uint32_t)n0, re);
            tc::tmem_ld8(lane_addr + (uint32_t)(N16 + n0), im);
            if (m < M) {
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (n0 + q < N) P[(int64_t)(n0 + q) * M + m] = make_double2((double)re[q], (double)im[q]);
            }
        }
    } else if (stage == 0) {
        const int m = m0 + 32 * warp + lane;
        double2* P = part + (int64_t)blockIdx.z * M * N;
        if (m < M)
            for (int n = 0; n < N; ++n) P[(int64_t)n * M + m] = make_double2(0.0, 0.0);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

}  // namespace

// Opt-in (ROKS_TENSOR_CORES=1): on the thin contractions of the apply and
// the PCG step (M, N <= 128, K ~ 10^4 - 10^5) this kernel is slower than the
// SIMT one, and the tensor cores' FP32 accumulation truncates instead of
// rounding, which biases long sums of positive terms (norms, overlaps).
bool tc_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("ROKS_TENSOR_CORES");
        on = (e && e[0] == '1') ? 1 : 0;
    }
    return on == 1;
}

// Tensor-core path of C = A^H B for N <= 128; false when not applicable.
// max_chunks bounds the partial-sum buffer (max_chunks * M * N double2).
bool gemm_cn_tc(int M, int N, int K, const float2* A, int64_t lda, const float2* B, int64_t ldb, double2* C, int ldc,
                double2* work, int max_chunks, cudaStream_t st) {
    if (!tc_enabled() || max_chunks <= 0 || M <= 0 || N <= 0 || N > 128 || K <= 0) return false;
    const int n16 = ((N + 7) / 8) * 8;
    const int np = 2 * n16;
    const int npad = np <= 32 ? 32 : (np <= 64 ? 64 : (np <= 128 ? 128 : 256));
    const int mt = (M + TC_M - 1) / TC_M;
    int want = (2 * 152 + mt - 1) / mt;
    if (want > max_chunks) want = max_chunks;
    if (want < 1) want = 1;
    int kc = (K + want - 1) / want;
    kc = ((kc + TC_KC - 1) / TC_KC) * TC_KC;
    const int nchunk = (K + kc - 1) / kc;
    if (nchunk > max_chunks) return false;
    dim3 g(mt, 1, nchunk);
    const size_t smem = 3 * (size_t)TC_M * TC_KR * 4 + 3 * (size_t)npad * TC_KR * 4;
#define TC_CASE(NP_)                                                                                             \
    if (npad == NP_) {                                                                                           \
        cudaFuncSetAttribute(k_gemm_cn_tc<NP_>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);         \
        roks::count_launch(), k_gemm_cn_tc<NP_><<<g, 128, smem, st>>>(M, N, K, kc, A, lda, B, ldb, work);        \
    }
    TC_CASE(32) TC_CASE(64) TC_CASE(128) TC_CASE(256)
#undef TC_CASE
    chunk_sum(M, N, nchunk, work, C, ldc, st);
    return true;
}

int tc_timeout_take() {
    if (!tc_enabled()) return 0;   // the flag is only ever set by the tensor-core kernel
    int h = 0;
    cudaMemcpyFromSymbol(&h, g_tc_timeout, sizeof(int));
    if (h) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(int));
    }
    return h;
}

}  // namespace roks
