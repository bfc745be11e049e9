// k_stream.cu -- FP32 complex contractions over the plane-wave dimension,
// streamed through shared memory by the tensor-memory-access engine (TMA).
//
// Both kernels run one CTA per SM over a contiguous range of rows (plane
// waves).  One thread of the last warp is the producer: for every row slice
// it issues one 2-D tensor copy per operand (a box of rows x all columns of a
// column-major band block) into a ring of shared-memory stages, and the
// copies complete the transaction count of the stage's "full" mbarrier.  The
// other warps multiply out of shared memory and release a stage by one
// arrival per warp on its "empty" mbarrier.  No thread computes an address
// for a single element, and the loads of later slices overlap the
// arithmetic of the current one.  Rows past the end of a matrix arrive as
// zeros (the copy's out-of-bounds fill).
//
//  * k_cn_stream: Cpart[cta] = A^H B over the CTA's rows (A: K x M, B: K x N
//    column major, K the plane-wave dimension), slices of 16 rows stored
//    with the 128-byte swizzle (one 128-byte row per column, its 16-byte
//    pairs permuted by the column index) so that loads of different columns
//    hit different banks; the per-CTA partials are summed in a fixed order,
//    with compensation, by the chunk-sum kernel.
//  * k_nn_stream: Cout = alpha A B + beta Cin (A: M x K tall, B: K x N
//    small, loaded once into shared memory, by a bulk copy of an FP32 copy
//    or, when small, converted from FP64 by the consumer warps), one row
//    tile of A (and of Cin) per stage.
//
// Every wait is bounded: a wait that gives up sets a device flag (read and
// cleared by stream_timeout_take), the kernel then waits (again bounded)
// for its own copies in flight and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdlib>
#include <mutex>

#include "roks_impl.cuh"
#include "tc_sm103.cuh"

namespace roks {

static __device__ int g_stream_timeout;

namespace {

constexpr uint32_t ST_WAIT = 1u << 26;   // mbarrier polls before giving up
constexpr int ST_MAXS = 8;               // most stages of a ring
constexpr int CN_KT = 16;                // rows per slice of the A^H B kernel (128 bytes: the swizzle span)
constexpr size_t ST_SMEM = 225 * 1024;   // dynamic shared memory of one CTA, alignment slack included
constexpr size_t ST_ALIGN = 1024;        // stage alignment (the 128-byte swizzle repeats every 1024 bytes)

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mb_arrive_expect(uint64_t* b, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mb_arrive(uint64_t* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
// global -> shared bulk copy; bytes a multiple of 16, both addresses 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     su32(dst)),
                 "l"(src), "r"(bytes), "r"(su32(bar))
                 : "memory");
}
// 2-D tensor copy of the box at (x = first row, y = first column)
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(su32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
        : "memory");
}

// A wait of the work loop gives up after `cap` polls (the context's wait
// cap); the waits for copies already in flight before the CTA exits use
// the default cap, so that no copy outlives its CTA.
__device__ __forceinline__ bool wait_or_flag(uint64_t* b, uint32_t parity, uint32_t cap) {
    if (tc::mbar_wait(b, parity, cap)) return true;
    g_stream_timeout = 1;
    return false;
}

__host__ __device__ constexpr size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// first ST_ALIGN-aligned byte of the dynamic shared memory
__device__ __forceinline__ unsigned char* aligned_smem(unsigned char* raw) {
    const uint32_t a = su32(raw);
    return raw + ((ST_ALIGN - (a & (ST_ALIGN - 1))) & (ST_ALIGN - 1));
}

// ------------------------------------------------------------------ Cpart = A^H B
// Thread t < TY TX KS: K-split group g = t / (TY TX), then (ty, tx); it owns
// rows m = ty + TY i (i < RM) and columns n = tx + TX j (j < RN) of the
// output, and the row pairs p = g, g + KS, ... of every slice.  Element
// (column c, row pair p) of a stage lies at byte c * 128 + ((p ^ (c & 7)) * 16).
// threads per CTA a register tile allows (registers: 65536 / threads)
__host__ __device__ constexpr int cn_maxt(int rm, int rn) {
    return rm * rn <= 4 ? 1024 : (rm * rn <= 9 ? 832 : (rm * rn <= 16 ? 512 : 384));
}

template <int RM, int RN, int KS>
__global__ void __launch_bounds__(cn_maxt(RM, RN)) k_cn_stream(int M, int N, int K, int rows_per_cta, int TY, int TX,
                                                   int NS, const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmB,
                                                   float2* __restrict__ part, uint32_t wcap) {
    extern __shared__ __align__(1024) unsigned char st_smem[];
    __shared__ __align__(8) uint64_t full[ST_MAXS], empty[ST_MAXS];
    unsigned char* ring = aligned_smem(st_smem);
    const uint32_t a_bytes = (uint32_t)align_up((size_t)128 * M, ST_ALIGN);
    const uint32_t stage_bytes = a_bytes + (uint32_t)align_up((size_t)128 * N, ST_ALIGN);
    const uint32_t tx_bytes = 128u * (uint32_t)(M + N);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5, cwarps = nwarps - 1;
    const int rb = blockIdx.x * rows_per_cta;
    const int re = min(K, rb + rows_per_cta);
    const int ns = re > rb ? (re - rb + CN_KT - 1) / CN_KT : 0;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], (uint32_t)cwarps);
        }
        tc::fence_mbar_init();
    }
    __syncthreads();

    const int tyx = TY * TX, nact = tyx * KS;
    const bool active = tid < nact;
    const int g = tid / tyx, t = tid - g * tyx, ty = t / TX, tx = t - ty * TX;
    float2 acc[RM][RN];
#pragma unroll
    for (int i = 0; i < RM; ++i)
#pragma unroll
        for (int j = 0; j < RN; ++j) acc[i][j] = make_float2(0.f, 0.f);

    if (warp == nwarps - 1) {
        // producer (one thread)
        if (lane == 0) {
            int issued = 0;
            for (int s = 0; s < ns; ++s) {
                const int sg = s % NS;
                if (s >= NS && !wait_or_flag(&empty[sg], (uint32_t)((s / NS - 1) & 1), wcap)) break;
                unsigned char* st = ring + (size_t)sg * stage_bytes;
                const int k0 = rb + s * CN_KT;
                mb_arrive_expect(&full[sg], tx_bytes);
                tma_2d(st, &tmA, k0, 0, &full[sg]);
                tma_2d(st + a_bytes, &tmB, k0, 0, &full[sg]);
                issued = s + 1;
            }
            // copies still in flight complete before the CTA may exit
            for (int s = (issued > NS ? issued - NS : 0); s < issued; ++s)
                wait_or_flag(&full[s % NS], (uint32_t)((s / NS) & 1), ST_WAIT);
        }
        __syncwarp();
    } else {
        // byte offset of row pair p of column c in a stage: (c * 128 + 16 * (c & 7)) ^ (16 p)
        uint32_t ob[RM + RN];
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const uint32_t m = (uint32_t)min(ty + TY * i, M - 1);
            ob[i] = m * 128u + ((m & 7u) << 4);
        }
#pragma unroll
        for (int j = 0; j < RN; ++j) {
            const uint32_t n = (uint32_t)min(tx + TX * j, N - 1);
            ob[RM + j] = a_bytes + n * 128u + ((n & 7u) << 4);
        }
        auto pair_mac = [&](const unsigned char* st, uint32_t (&sb)[RM + RN], int p) {
            const uint32_t px = (uint32_t)p << 4;
            float4 v[RM + RN];
#pragma unroll
            for (int q = 0; q < RM + RN; ++q) v[q] = *reinterpret_cast<const float4*>(st + (sb[q] ^ px));
            // operation-major order: consecutive multiply-adds go to different
            // accumulators, so none waits on the one before it
#define CN_PASS(OUT, AX, BX, SGN)                                   \
    _Pragma("unroll") for (int i = 0; i < RM; ++i)                  \
        _Pragma("unroll") for (int j = 0; j < RN; ++j)              \
            acc[i][j].OUT = fmaf(SGN v[i].AX, v[RM + j].BX, acc[i][j].OUT);
            CN_PASS(x, x, x, ) CN_PASS(y, x, y, ) CN_PASS(x, y, y, ) CN_PASS(y, y, x, -)
            CN_PASS(x, z, z, ) CN_PASS(y, z, w, ) CN_PASS(x, w, w, ) CN_PASS(y, w, z, -)
#undef CN_PASS
        };
        for (int s = 0; s < ns; ++s) {
            const int sg = s % NS;
            if (!wait_or_flag(&full[sg], (uint32_t)((s / NS) & 1), wcap)) break;
            const int rows = min(CN_KT, re - (rb + s * CN_KT));
            const int pairs = (rows + 1) >> 1;
            if (active) {
                // stage bases are multiples of 1024: the swizzle acts on bits 4-6 of the offset alone
                uint32_t sb[RM + RN];
#pragma unroll
                for (int q = 0; q < RM + RN; ++q) sb[q] = (uint32_t)sg * stage_bytes + ob[q];
                if (pairs == CN_KT / 2) {
#pragma unroll
                    for (int q = 0; q < CN_KT / 2 / KS; ++q) pair_mac(ring, sb, g + KS * q);
                } else {
                    for (int p = g; p < pairs; p += KS) pair_mac(ring, sb, p);
                }
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&empty[sg]);
        }
    }
    __syncthreads();
    // K-split groups: groups 1.. park their sums in the (idle) ring, group 0
    // adds them in group order
    if (KS > 1) {
        float2* red = reinterpret_cast<float2*>(ring);
        if (active && g > 0) {
#pragma unroll
            for (int i = 0; i < RM; ++i)
#pragma unroll
                for (int j = 0; j < RN; ++j) red[((size_t)(g - 1) * tyx + t) * (RM * RN) + i * RN + j] = acc[i][j];
        }
        __syncthreads();
        if (active && g == 0) {
            for (int q = 1; q < KS; ++q)
#pragma unroll
                for (int i = 0; i < RM; ++i)
#pragma unroll
                    for (int j = 0; j < RN; ++j) {
                        const float2 v = red[((size_t)(q - 1) * tyx + t) * (RM * RN) + i * RN + j];
                        acc[i][j].x += v.x;
                        acc[i][j].y += v.y;
                    }
        }
    }
    if (active && g == 0) {
        float2* P = part + (int64_t)blockIdx.x * M * N;
#pragma unroll
        for (int i = 0; i < RM; ++i) {
            const int m = ty + TY * i;
            if (m >= M) continue;
#pragma unroll
            for (int j = 0; j < RN; ++j) {
                const int n = tx + TX * j;
                if (n < N) P[(int64_t)n * M + m] = acc[i][j];
            }
        }
    }
}

// ------------------------------------------------------------------ Cout = alpha A B + beta Cin
// Row tiles of TR = 32 RR WS rows: consumer warp (h, w), h < WS, w < W, owns
// rows 32 RR h + RR l .. + RR - 1 (lane l) and the column pairs 2 (w + W j),
// j < RN / 2.  K is taken in nkc chunks of KC columns: a work item is (tile,
// chunk), and its stage holds the A box of the chunk (KC columns x TR rows)
// and, for the tile's last chunk, the Cin box (N columns x TR rows).  B
// (K x N row major, N even) is resident in shared memory.
template <int RR, int RN, int WS>
__global__ void __launch_bounds__(768) k_nn_stream(int M, int N, int K, int KC, int nkc, int rows_per_cta, int W,
                                                   int NS, int load_c, const __grid_constant__ CUtensorMap tmA,
                                                   const __grid_constant__ CUtensorMap tmC,
                                                   const float2* __restrict__ Bf, const double2* __restrict__ Bd,
                                                   int ldb, float2* Cout, int64_t ldc, float alpha, float beta,
                                                   uint32_t wcap) {
    constexpr int TR = 32 * RR * WS;
    constexpr int RP = RN / 2;
    extern __shared__ __align__(1024) unsigned char st_smem[];
    __shared__ __align__(8) uint64_t full[ST_MAXS], empty[ST_MAXS], bbar;
    unsigned char* base = aligned_smem(st_smem);
    float2* Bs = reinterpret_cast<float2*>(base);
    const uint32_t b_bytes = (uint32_t)K * (uint32_t)N * 8u;
    unsigned char* ring = base + align_up(b_bytes, 128);
    const uint32_t a_bytes = (uint32_t)KC * TR * 8u;
    const uint32_t a_span = (uint32_t)align_up(a_bytes, 128);
    const uint32_t c_bytes = load_c ? (uint32_t)N * TR * 8u : 0u;
    const uint32_t stage_bytes = (uint32_t)align_up(a_span + c_bytes, 128);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = blockDim.x >> 5;
    const int rb = blockIdx.x * rows_per_cta;
    const int re = min(M, rb + rows_per_cta);
    const int nt = re > rb ? (re - rb + TR - 1) / TR : 0;
    const int items = nt * nkc;
    if (tid == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], (uint32_t)(W * WS));
        }
        tc::mbar_init(&bbar, 1);
        tc::fence_mbar_init();
    }
    __syncthreads();

    if (warp == nwarps - 1) {
        // producer (one thread): B once (unless the consumers convert it), then the (tile, chunk) items
        if (lane == 0 && nt > 0) {
            if (!Bd) {
                mb_arrive_expect(&bbar, b_bytes);
                bulk_g2s(Bs, Bf, b_bytes, &bbar);
            }
            int issued = 0;
            for (int it = 0; it < items; ++it) {
                const int sg = it % NS;
                if (it >= NS && !wait_or_flag(&empty[sg], (uint32_t)((it / NS - 1) & 1), wcap)) break;
                unsigned char* st = ring + (size_t)sg * stage_bytes;
                const int kc = it % nkc;
                const int r0 = rb + (it / nkc) * TR;
                const bool last = kc == nkc - 1;
                mb_arrive_expect(&full[sg], a_bytes + (last ? c_bytes : 0u));
                tma_2d(st, &tmA, r0, kc * KC, &full[sg]);
                if (last && load_c) tma_2d(st + a_span, &tmC, r0, 0, &full[sg]);
                issued = it + 1;
            }
            if (!Bd) wait_or_flag(&bbar, 0u, ST_WAIT);
            for (int it = (issued > NS ? issued - NS : 0); it < issued; ++it)
                wait_or_flag(&full[it % NS], (uint32_t)((it / NS) & 1), ST_WAIT);
        }
        __syncwarp();
    } else if (warp < W * WS && nt > 0) {
        bool ok = true;
        if (Bd) {
            // small FP64 B: the consumers convert it (row major) while the first tiles are in flight
            for (int i = tid; i < K * N; i += 32 * W * WS) {
                const int k = i / N, n = i - k * N;
                const double2 v = Bd[(int64_t)n * ldb + k];
                Bs[i] = make_float2((float)v.x, (float)v.y);
            }
            asm volatile("bar.sync 1, %0;" ::"r"(32 * W * WS) : "memory");
        } else {
            ok = wait_or_flag(&bbar, 0u, wcap);
        }
        const int w = warp % W, hb = (warp / W) * 32 * RR;
        int ncp[RP];
#pragma unroll
        for (int j = 0; j < RP; ++j) ncp[j] = min(2 * (w + W * j), N - 2);
        float2 acc[RR][RN];
        for (int it = 0; it < items && ok; ++it) {
            const int sg = it % NS;
            if (!wait_or_flag(&full[sg], (uint32_t)((it / NS) & 1), wcap)) break;
            const int kc = it % nkc;
            const int r0 = rb + (it / nkc) * TR;
            const int rows = min(TR, re - r0);
            const int k0 = kc * KC, kn = min(KC, K - k0);
            const float2* As = reinterpret_cast<const float2*>(ring + (size_t)sg * stage_bytes);
            const float2* Bk = Bs + (size_t)k0 * N;
            if (kc == 0) {
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int j = 0; j < RN; ++j) acc[r][j] = make_float2(0.f, 0.f);
            }
            // four k at a time: all shared-memory loads first, then the multiply-adds
            auto kstep = [&](const float4 (&av)[4], const float4 (&bv)[4][RP], int u) {
                float a[2 * RR];
                if constexpr (RR == 2) {
                    a[0] = av[u].x; a[1] = av[u].y; a[2] = av[u].z; a[3] = av[u].w;
                } else {
                    a[0] = av[u].x; a[1] = av[u].y;
                }
                float b[2 * RN];
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                    b[4 * j] = bv[u][j].x; b[4 * j + 1] = bv[u][j].y;
                    b[4 * j + 2] = bv[u][j].z; b[4 * j + 3] = bv[u][j].w;
                }
                // operation-major order (no multiply-add waits on the one before it)
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < RN; ++c) acc[r][c].x = fmaf(a[2 * r], b[2 * c], acc[r][c].x);
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < RN; ++c) acc[r][c].y = fmaf(a[2 * r], b[2 * c + 1], acc[r][c].y);
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < RN; ++c) acc[r][c].x = fmaf(-a[2 * r + 1], b[2 * c + 1], acc[r][c].x);
#pragma unroll
                for (int r = 0; r < RR; ++r)
#pragma unroll
                    for (int c = 0; c < RN; ++c) acc[r][c].y = fmaf(a[2 * r + 1], b[2 * c], acc[r][c].y);
            };
            auto load_a = [&](int k) -> float4 {
                if constexpr (RR == 2) return *reinterpret_cast<const float4*>(As + (size_t)k * TR + hb + 2 * lane);
                const float2 v = As[(size_t)k * TR + hb + lane];
                return make_float4(v.x, v.y, 0.f, 0.f);
            };
            int k = 0;
            for (; k + 4 <= kn; k += 4) {
                float4 av[4], bv[4][RP];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    av[u] = load_a(k + u);
#pragma unroll
                    for (int j = 0; j < RP; ++j)
                        bv[u][j] = *reinterpret_cast<const float4*>(Bk + (size_t)(k + u) * N + ncp[j]);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) kstep(av, bv, u);
            }
            for (; k < kn; ++k) {
                float4 av[4], bv[4][RP];
                av[0] = load_a(k);
#pragma unroll
                for (int j = 0; j < RP; ++j) bv[0][j] = *reinterpret_cast<const float4*>(Bk + (size_t)k * N + ncp[j]);
                kstep(av, bv, 0);
            }
            if (kc == nkc - 1) {
                // epilogue: rows RR lane + r of the tile, columns ncp[j], ncp[j] + 1
                const float2* Cs = reinterpret_cast<const float2*>(ring + (size_t)sg * stage_bytes + a_span);
                const int lr = hb + RR * lane;
#pragma unroll
                for (int j = 0; j < RP; ++j) {
                    if (2 * (w + W * j) >= N) continue;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int n = ncp[j] + h;
                        float2 v[RR];
#pragma unroll
                        for (int r = 0; r < RR; ++r) {
                            v[r] = make_float2(alpha * acc[r][2 * j + h].x, alpha * acc[r][2 * j + h].y);
                            if (load_c) {
                                const float2 c = Cs[(size_t)n * TR + lr + r];
                                v[r].x = fmaf(beta, c.x, v[r].x);
                                v[r].y = fmaf(beta, c.y, v[r].y);
                            }
                        }
                        float2* out = Cout + (int64_t)n * ldc + r0 + lr;
                        if (RR == 2 && lr + 1 < rows) {
                            *reinterpret_cast<float4*>(out) = make_float4(v[0].x, v[0].y, v[RR - 1].x, v[RR - 1].y);
                        } else {
#pragma unroll
                            for (int r = 0; r < RR; ++r)
                                if (lr + r < rows) out[r] = v[r];
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) mb_arrive(&empty[sg]);
        }
    }
    __syncthreads();
}

// B (K x N, FP64, column major, ldb) -> Bf (K x N, FP32, row major)
__global__ void k_b_rowmajor_f32(int K, int N, const double2* __restrict__ B, int ldb, float2* __restrict__ Bf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * N) return;
    const int k = i / N, n = i - k * N;
    const double2 v = B[(int64_t)n * ldb + k];
    Bf[i] = make_float2((float)v.x, (float)v.y);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// 2-D map of a column-major complex FP32 block (rows x cols, ld elements per
// column), moved as 8-byte elements in boxes of box_rows x box_cols
bool encode_block(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                  int box_cols, bool swizzle128) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 8u};
    const cuuint32_t box[2] = {(cuuint32_t)box_rows, (cuuint32_t)box_cols};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE,
                          swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int st_sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// polls of the work-loop waits of the next launches (set_wait_cap)
uint32_t g_wait_polls = ST_WAIT;

template <typename F>
void set_smem(F* f, size_t bytes) {
    cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

bool tensor_map_2d(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                   int box_cols, bool swizzle128) {
    return encode_block(map, ptr, rows, cols, ld, box_rows, box_cols, swizzle128);
}

bool stream_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("ROKS_STREAM");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

void set_wait_cap(int cap) { g_wait_polls = cap == 0 ? ST_WAIT : (cap < 0 ? 0u : (uint32_t)cap); }
uint32_t wait_polls() { return g_wait_polls; }

int stream_timeout_take() {
    int h = 0;
    cudaMemcpyFromSymbol(&h, g_stream_timeout, sizeof(int));
    if (h) {
        const int z = 0;
        cudaMemcpyToSymbol(g_stream_timeout, &z, sizeof(int));
    }
    return h;
}

int* stream_timeout_flag() {
    constexpr int kMaxDev = 64;
    static int* addr[kMaxDev] = {nullptr};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    if (!addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_stream_timeout) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        addr[dev] = static_cast<int*>(p);
    }
    return addr[dev];
}

// Cpart = A^H B streamed, then the fixed-order sum; false when the shape,
// the alignment or the partial buffer does not allow it.
bool gemm_cn_stream(int M, int N, int K, const float2* A, int64_t lda, const float2* B, int64_t ldb, double2* C,
                    int ldc, double2* work, size_t work_elems, cudaStream_t st) {
    if (!stream_enabled() || M <= 0 || N <= 0 || M > 256 || N > 256 || K < 2 * CN_KT) return false;
    if ((lda & 1) || (ldb & 1) || !aligned16(A) || !aligned16(B) || !aligned16(work)) return false;
    // register tile: least padded work plus shared-memory loads per multiply-add,
    // weighted by the warps per SM it leaves (fewer than 16 hide latency poorly)
    struct Cand { int rm, rn; };
    const Cand cands[] = {{3, 3}, {4, 4}, {4, 6}, {2, 2}};
    int best = -1, ty = 0, tx = 0, ks = 1;
    double best_cost = 1e300;
    for (int c = 0; c < 4; ++c) {
        const int rm = cands[c].rm, rn = cands[c].rn;
        const int TY = (M + rm - 1) / rm, TX = (N + rn - 1) / rn;
        const int thr = TY * TX;
        const int maxt = cn_maxt(rm, rn);
        int KS = 0;
        for (int k = 8; k >= 1 && !KS; k /= 2)
            if (((thr * k + 31) / 32) * 32 + 32 <= maxt) KS = k;
        if (!KS) continue;
        const int warps = (thr * KS + 31) / 32;
        const double cost = (double)TY * rm * TX * rn * (1.0 + (rm + rn) / (2.0 * rm * rn)) *
                            (warps < 16 ? 16.0 / warps : 1.0);
        if (cost < best_cost) {
            best_cost = cost;
            best = c;
            ty = TY;
            tx = TX;
            ks = KS;
        }
    }
    if (best < 0) return false;
    const size_t stage = align_up((size_t)128 * M, ST_ALIGN) + align_up((size_t)128 * N, ST_ALIGN);
    int NS = (int)((ST_SMEM - ST_ALIGN) / stage);
    if (NS > ST_MAXS) NS = ST_MAXS;
    if (NS < 2) return false;
    const size_t red = (size_t)(ks - 1) * ty * tx * cands[best].rm * cands[best].rn * sizeof(float2);
    if (red > NS * stage) return false;
    int G = st_sm_count();
    const int gmax = (K + CN_KT - 1) / CN_KT;
    if (G > gmax) G = gmax;
    int rows = (K + G - 1) / G;
    rows = (rows + 1) & ~1;   // interior range ends stay even: a row pair never spans two CTAs
    G = (K + rows - 1) / rows;
    if ((size_t)G * M * N * sizeof(float2) > work_elems * sizeof(double2)) return false;
    CUtensorMap tmA, tmB;
    if (!encode_block(&tmA, A, K, M, lda, CN_KT, M, true) || !encode_block(&tmB, B, K, N, ldb, CN_KT, N, true))
        return false;
    const int cons = ty * tx * ks;
    const int threads = ((cons + 31) / 32) * 32 + 32;
    const size_t smem = NS * stage + ST_ALIGN;
    float2* part = reinterpret_cast<float2*>(work);
#define CNS_CASE(RM_, RN_, KS_)                                                                            \
    if (cands[best].rm == RM_ && cands[best].rn == RN_ && ks == KS_) {                                    \
        static bool attr = false;                                                                          \
        if (!attr) {                                                                                       \
            set_smem(k_cn_stream<RM_, RN_, KS_>, ST_SMEM);                                                 \
            attr = true;                                                                                   \
        }                                                                                                  \
        roks::count_launch();                                                                              \
        k_cn_stream<RM_, RN_, KS_><<<G, threads, smem, st>>>(M, N, K, rows, ty, tx, NS, tmA, tmB, part,      \
                                                             g_wait_polls);                                 \
    }
#define CNS_KS(RM_, RN_) CNS_CASE(RM_, RN_, 1) CNS_CASE(RM_, RN_, 2) CNS_CASE(RM_, RN_, 4) CNS_CASE(RM_, RN_, 8)
    CNS_KS(3, 3) CNS_KS(4, 4) CNS_KS(4, 6) CNS_KS(2, 2)
#undef CNS_KS
#undef CNS_CASE
    chunk_sum_f32(M, N, G, part, C, ldc, st);
    return true;
}

// Cout (ldc) = alpha A B + beta Cin (ldcin) streamed (B: K x N FP64 small,
// converted into bwork as K x N FP32 row major); false when the shape or the
// alignment does not allow it.
bool gemm_nn_stream(int M, int N, int K, const float2* A, int64_t lda, const double2* B, int ldb, void* bwork,
                    const float2* Cin, int64_t ldcin, float2* Cout, int64_t ldc, float alpha, float beta,
                    cudaStream_t st) {
    if (!stream_enabled() || M <= 0 || N <= 0 || K <= 0 || (N & 1) || N > 96 || K > 256) return false;
    const bool load_c = beta != 0.f;
    if ((lda & 1) || (ldc & 1) || !aligned16(A) || !aligned16(bwork) || !aligned16(Cout) ||
        (load_c && (!aligned16(Cin) || (ldcin & 1))))
        return false;
    // columns per thread (even) so that at most 11 warps cover N
    const int pairs = N / 2;
    const int rp = (pairs + 10) / 11;
    const int RN = 2 * rp;
    if (RN > 12) return false;
    const int W = (pairs + rp - 1) / rp;
    const size_t bbytes = align_up((size_t)K * N * sizeof(float2), 128);
    // rows per lane RR, warp sets WS and K chunks: the largest row tile, then
    // the fewest chunks, with two stages beside the resident B
    int RR = 0, WS = 0, NS = 0, KC = 0, nkc = 0;
    size_t stage = 0;
    const int shapes[3][2] = {{2, 2}, {2, 1}, {1, 1}};
    for (int c = 0; c < 3 && !RR; ++c) {
        const int rr = shapes[c][0], ws = shapes[c][1], tr = 32 * rr * ws;
        for (int q = 1; q <= 8 && !RR; ++q) {
            const int kc = (K + q - 1) / q;
            stage = align_up(align_up((size_t)kc * tr * sizeof(float2), 128) +
                                 (load_c ? (size_t)N * tr * sizeof(float2) : 0),
                             128);
            if (ST_ALIGN + bbytes + 2 * stage > ST_SMEM) continue;
            RR = rr;
            WS = ws;
            KC = kc;
            nkc = (K + kc - 1) / kc;
            NS = (int)((ST_SMEM - ST_ALIGN - bbytes) / stage);
            if (NS > 4) NS = 4;
        }
    }
    if (!RR) return false;
    const int TR = 32 * RR * WS;
    int G = st_sm_count();
    const int gmax = (M + TR - 1) / TR;
    if (G > gmax) G = gmax;
    int rows = (M + G - 1) / G;
    rows = (rows + 1) & ~1;
    G = (M + rows - 1) / rows;
    CUtensorMap tmA, tmC;
    if (!encode_block(&tmA, A, M, K, lda, TR, KC, false)) return false;
    if (load_c) {
        if (!encode_block(&tmC, Cin, M, N, ldcin, TR, N, false)) return false;
    } else {
        tmC = tmA;   // not read
    }
    float2* Bf = static_cast<float2*>(bwork);
    // a small B is converted by the kernel's consumers; a large one by a kernel of its own
    const bool convert_in = K * N <= 2048;
    if (!convert_in) {
        roks::count_launch();
        k_b_rowmajor_f32<<<(K * N + 255) / 256, 256, 0, st>>>(K, N, B, ldb, Bf);
    }
    const size_t smem = ST_ALIGN + bbytes + (size_t)NS * stage;
    const int threads = 32 * (W * WS + 1);
#define NNS_CASE(RR_, RN_, WS_)                                                                              \
    if (RR == RR_ && RN == RN_ && WS == WS_) {                                                              \
        static bool attr = false;                                                                           \
        if (!attr) {                                                                                        \
            set_smem(k_nn_stream<RR_, RN_, WS_>, ST_SMEM);                                                  \
            attr = true;                                                                                    \
        }                                                                                                   \
        roks::count_launch();                                                                               \
        k_nn_stream<RR_, RN_, WS_><<<G, threads, smem, st>>>(M, N, K, KC, nkc, rows, W, NS, load_c ? 1 : 0,  \
                                                             tmA, tmC, Bf, convert_in ? B : nullptr, ldb,   \
                                                             Cout, ldc, alpha, beta, g_wait_polls);         \
        return true;                                                                                        \
    }
#define NNS_RN(RR_, WS_) NNS_CASE(RR_, 2, WS_) NNS_CASE(RR_, 4, WS_) NNS_CASE(RR_, 6, WS_) NNS_CASE(RR_, 8, WS_) \
    NNS_CASE(RR_, 10, WS_) NNS_CASE(RR_, 12, WS_)
    NNS_RN(2, 2) NNS_RN(2, 1) NNS_RN(1, 1)
#undef NNS_RN
#undef NNS_CASE
    return false;
}

}  // namespace roks
