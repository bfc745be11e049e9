// k_tcgemm.cu -- complex FP32 contractions of the large blocks (hundreds of
// bands, thousands of projectors) on the 5th-generation tensor cores
// (tcgen05, kind::tf32), mixed-precision path:
//
//   CN:  C (M x N, FP64 out) = A^H B,          A: K x M, B: K x N (K: plane waves)
//   NN:  Cout (M x N) = alpha A B + beta Cin,   A: M x K tall, B: K x N small (FP64)
//
// Real formulation.  Complex vectors are stored as interleaved (re, im)
// pairs, so a complex dot product is a real one over 2K numbers taken as
// stored from one operand (a'), against a rearranged copy of the other:
//   CN  Re = a'.(br, bi),   Im = a'.(bi, -br)      (a' = conj taken by the pairing)
//   NN  Re = a'.(br, -bi),  Im = a'.(bi, br)
// The MMA's N side holds 64 complex columns as 128 rows: the 64 rows that
// give the real parts, then the 64 that give the imaginary parts; one MMA of
// M = 128, N = 128 yields both.
//
// Precision (three TF32 products per FP32 product): each operand value x is
// split as x = hi + lo, hi = tf32(x), lo = tf32(x - hi), and each product is
// lo.hi + hi.lo + hi.hi.  The tensor cores' FP32 accumulation truncates
// instead of rounding, which biases long sums of like-signed terms (norms,
// overlaps, diagonal-dominated rotations).  So every stage (32 reals: four
// K-steps of 8) goes into a fresh tensor-memory accumulator, in the order
// of the eight small cross terms first and the four hi.hi products last:
// only those four additions meet a large partial sum (a bias near 1e-7 of
// the stage's sum at most), and the drain warps add the stage's result into
// FP32 sums in registers (round to nearest).  Four accumulators of 128
// columns rotate, so the MMAs of the next stages run while the previous
// ones drain.  (A drain per K-step was measured a third slower on the
// mgo-120 products.)
//
// One CTA per SM (200 KB of shared memory, all 512 tensor-memory columns),
// 18 warps:
//   warp 0      producer: 2-D tensor copies of the raw FP32 operand slices
//               into three raw stages; NN: bulk copies of the pre-split B;
//   warp 1      one thread issues the MMAs;
//   warps 2-17  workers.  In iteration i a worker converts its share of
//               stage i (split into TF32 hi and lo, build the N-side rows,
//               store K-major core matrices of 8 rows x 16 bytes, no
//               swizzle, into one of two operand stages) and then drains its
//               block of stage i - 2's accumulator: the lane quadrant
//               warp % 4 and 16 complex columns.  The lag of two cannot
//               deadlock: converting stage i waits for the MMAs of stage
//               i - 2, which need the drain of stage i - 6 (iteration i - 4)
//               and the conversion of stage i - 2 (iteration i - 2), and
//               draining stage i - 2 waits for those same MMAs.
// Every wait is bounded (the context's wait cap); a wait that gives up sets
// a device flag and the CTA winds down: copies and MMAs in flight are waited
// for with the default bound before the tensor memory is freed.
#include <cuda.h>

#include <algorithm>
#include <cstdint>
#include <cstdlib>

#include "roks_impl.cuh"
#include "tc_sm103.cuh"

namespace roks {

// 2-D tensor map of a column-major complex FP32 block (k_stream.cu)
bool tensor_map_2d(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, int64_t ld, int box_rows,
                   int box_cols, bool swizzle128);

static __device__ int g_tcg_timeout;

namespace {

constexpr int GB_M = 128;      // tile rows (tensor-memory lanes)
constexpr int GB_NC = 64;      // complex columns of a tile
constexpr int GB_NR = 128;     // N-side rows of a tile (real parts, then imaginary parts)
constexpr int GB_KC = 16;      // complex K per stage
constexpr int GB_KR = 32;      // real K per stage (four MMA K-steps of 8)
constexpr int GB_RAW = 3;      // raw stages
constexpr int GB_CONV = 2;     // operand stages
constexpr int GB_ACC = 4;      // tensor-memory accumulators
constexpr int GB_WORKERS = 16;    // worker warps
constexpr int GB_THREADS = (2 + GB_WORKERS) * 32;
constexpr uint32_t GB_PART = GB_M * GB_KR * 4;   // one split part (hi or lo) of a 128-row operand: 16 KB
constexpr uint32_t GB_SLOT = 4 * GB_PART;        // A hi | A lo | B hi | B lo
constexpr uint32_t GB_RAWA = GB_M * GB_KC * 8;   // 16 KB
constexpr uint32_t GB_RAWB = GB_NC * GB_KC * 8;  // 8 KB (CN)
constexpr uint32_t GB_TCOLS = GB_ACC * GB_NR;    // 512 columns
constexpr uint32_t GB_DEFAULT_WAIT = 1u << 26;

// byte offset of real element kr of row r in a K-major operand tile of
// 32 reals per row: core matrix (r / 8, kr / 4) of 128 bytes, row r % 8 at
// 16 (r % 8), element kr % 4 at 4 (kr % 4)
__device__ __forceinline__ uint32_t cofs(int r, int kr) {
    return (uint32_t)((((r >> 3) * (GB_KR / 4) + (kr >> 2)) << 7) + ((r & 7) << 4) + ((kr & 3) << 2));
}

__device__ __forceinline__ void split4(const float4 v, float4& hi, float4& lo) {
    hi.x = tc::to_tf32(v.x);
    hi.y = tc::to_tf32(v.y);
    hi.z = tc::to_tf32(v.z);
    hi.w = tc::to_tf32(v.w);
    lo.x = tc::to_tf32(v.x - hi.x);
    lo.y = tc::to_tf32(v.y - hi.y);
    lo.z = tc::to_tf32(v.z - hi.z);
    lo.w = tc::to_tf32(v.w - hi.w);
}

__device__ __forceinline__ void put_split(unsigned char* hi_base, uint32_t off, const float4 v) {
    float4 h, l;
    split4(v, h, l);
    *reinterpret_cast<float4*>(hi_base + off) = h;
    *reinterpret_cast<float4*>(hi_base + GB_PART + off) = l;
}

// Bounded wait on a phase; gives up after `cap` polls, or early once another
// role of the CTA has given up (checked every 1024 polls).
__device__ __forceinline__ bool gwait(uint64_t* bar, uint32_t parity, uint32_t cap, volatile int* failed) {
    for (uint32_t i = 0; i < cap; ++i) {
        if (tc::mbar_try(bar, parity)) return true;
        if ((i & 1023u) == 1023u && *failed) return false;
    }
    return false;
}

// The same wait by every lane of a warp, with one outcome for the warp (the
// warp-wide instructions after it need all lanes): true only if every lane
// saw the phase complete.
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint32_t cap, volatile int* failed) {
    const bool ok = gwait(bar, parity, cap, failed);
    return __all_sync(0xffffffffu, ok) != 0;
}

__device__ __forceinline__ void give_up(volatile int* failed) {
    *failed = 1;
    g_tcg_timeout = 1;
}

// Shared-memory plan of a variant: operand slots (A hi | A lo | B hi | B lo)
// and raw stages.  APRE: A arrives pre-split (k_tcg_asplit), copied by the
// producer straight into the slot, so the slots can be three deep; the tall
// product P Y takes it (B is pre-split as well: no raw stage, no conversion,
// the worker warps only drain).  The plan also covers A^H B with a pre-split
// A (raw stages of B alone), which gemm_cn_tcg does not launch: it measured
// slower than converting both operands in the kernel.
template <bool NN, bool APRE>
struct GbPlan {
    static constexpr int SLOTS = APRE ? 3 : GB_CONV;
    static constexpr uint32_t RAWA = APRE ? 0u : GB_RAWA;       // raw A bytes per stage
    static constexpr uint32_t RAWB = NN ? 0u : GB_RAWB;         // raw B bytes per stage
    static constexpr uint32_t RAWS = RAWA + RAWB;                // bytes of one raw stage
    static constexpr bool RAW = RAWA + RAWB > 0;                // a TMA raw stage per K stage
    static constexpr bool CONVERT = RAW;                        // workers convert raw operands
    static constexpr bool BULK = NN || APRE;                    // bulk copies into the slot
    static constexpr uint32_t BULK_BYTES = (NN ? 2 * GB_PART : 0u) + (APRE ? 2 * GB_PART : 0u);
    static constexpr size_t SMEM = (size_t)SLOTS * GB_SLOT + (RAW ? (size_t)GB_RAW * RAWS : 0) + 1024;
    static constexpr int LAG = CONVERT ? 2 : 0;                 // drain of stage i - LAG in iteration i
};

// CTA-loop schedules (the kernel's SK instance), one CTA per SM:
// * A^H B, stream-K: CTA c takes units units * c / ctas .. units * (c + 1) /
//   ctas - 1 of the (tile, stage) sequence, stage fastest (tile t: M tile
//   t % fast, N tile t / fast), and writes the partial sums of each tile it
//   touches to its segment slot c * maxseg + (t - its first tile);
// * A B, persistent: units = tiles, CTA c takes the whole tiles c, c + ctas,
//   ... (tile t: N tile t % fast, M tile t / fast), its pipeline running on
//   across them, and writes each tile's result as it completes.
// ctas = 0: one tile (and one K range) per CTA of a 3-D grid.
struct SkPlan {
    int64_t units = 0;
    int ctas = 0, maxseg = 0, fast = 0;
};

template <bool NN, bool APRE, bool SK = false>
__global__ void __launch_bounds__(GB_THREADS, 1)
    k_tcgemm(int M, int N, int stages_per_cta, int total_stages, SkPlan sk, const __grid_constant__ CUtensorMap tmA,
             const __grid_constant__ CUtensorMap tmB, const unsigned char* __restrict__ bsplit,
             const unsigned char* __restrict__ asplit, float2* __restrict__ part, const float2* Cin, int64_t ldcin,
             float2* Cout, int64_t ldc, float alpha, float beta, uint32_t wcap) {
    using PL = GbPlan<NN, APRE>;
    constexpr int SL = PL::SLOTS;
    extern __shared__ __align__(1024) unsigned char gb_smem[];
    __shared__ __align__(8) uint64_t raw_full[GB_RAW], raw_empty[GB_RAW], conv_full[SL], conv_empty[SL], b_full[SL],
        acc_full[GB_ACC], acc_empty[GB_ACC], mma_done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int failed;
    unsigned char* base = gb_smem + ((1024u - (tc::smem_u32(gb_smem) & 1023u)) & 1023u);
    unsigned char* conv = base;                                // SL operand slots
    unsigned char* raw = base + (size_t)SL * GB_SLOT;          // GB_RAW raw stages (1024-byte aligned)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // CN: grid (M tiles, N tiles, K splits).  NN: grid (N tiles, M tiles),
    // so that the CTAs sharing one tile of the tall A run side by side and A
    // comes from DRAM about once (M fastest re-read it once per N tile)
    const int mi = NN ? blockIdx.y : blockIdx.x, ni = NN ? blockIdx.x : blockIdx.y;
    const int m0 = mi * GB_M, n0 = ni * GB_NC;
    const int s0 = NN ? 0 : blockIdx.z * stages_per_cta;
    const int64_t u0 = (SK && !NN) ? sk.units * blockIdx.x / sk.ctas : 0;
    // CTA loop: the first tile and stage (the loops then step them); after a
    // tile's last stage the next tile is t + tstep
    const int t_first = SK ? (NN ? (int)blockIdx.x : (int)(u0 / total_stages)) : 0;
    const int s_first = (SK && !NN) ? (int)(u0 - (int64_t)t_first * total_stages) : 0;
    const int tstep = (SK && NN) ? sk.ctas : 1;
    const int ns = NN ? (SK ? (int)((sk.units - blockIdx.x + sk.ctas - 1) / sk.ctas) * total_stages : total_stages)
                      : (SK ? (int)(sk.units * (blockIdx.x + 1) / sk.ctas - u0)
                            : max(0, min(total_stages, s0 + stages_per_cta) - s0));

    if (tid == 0) {
        for (int s = 0; s < GB_RAW; ++s) {
            tc::mbar_init(&raw_full[s], 1);
            tc::mbar_init(&raw_empty[s], GB_WORKERS);
        }
        for (int s = 0; s < SL; ++s) {
            tc::mbar_init(&conv_full[s], GB_WORKERS);
            tc::mbar_init(&conv_empty[s], 1);
            tc::mbar_init(&b_full[s], 1);
        }
        for (int s = 0; s < GB_ACC; ++s) {
            tc::mbar_init(&acc_full[s], 1);
            tc::mbar_init(&acc_empty[s], GB_WORKERS);
        }
        tc::mbar_init(&mma_done, 1);
        failed = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(&tmem_base, GB_TCOLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        // ------------------------------------------------ producer
        if (lane == 0) {
            int issued = 0, bissued = 0;
            int t_cur = t_first, s_cur = s_first;
            for (int i = 0; i < ns; ++i) {
                // this stage's tile (M tile ma, N tile nb_) and K stage ks_
                int ma = mi, nb_ = ni, ks_ = s0 + i;
                if (SK) {
                    ma = NN ? t_cur / sk.fast : t_cur % sk.fast;
                    nb_ = NN ? t_cur % sk.fast : t_cur / sk.fast;
                    ks_ = s_cur;
                    if (++s_cur == total_stages) {
                        s_cur = 0;
                        t_cur += tstep;
                    }
                }
                if (PL::RAW) {
                    const int rs = i % GB_RAW;
                    if (i >= GB_RAW && !gwait(&raw_empty[rs], (uint32_t)((i / GB_RAW - 1) & 1), wcap, &failed)) {
                        give_up(&failed);
                        break;
                    }
                    unsigned char* ra = raw + (size_t)rs * PL::RAWS;
                    const int k0 = ks_ * GB_KC, am = ma * GB_M, bn = nb_ * GB_NC;
                    if (NN) {
                        tc::mbar_arrive_expect_tx(&raw_full[rs], GB_RAWA);
                        tc::tma_2d(ra, &tmA, am, k0, &raw_full[rs]);
                    } else {
                        tc::mbar_arrive_expect_tx(&raw_full[rs], PL::RAWA + PL::RAWB);
                        if (!APRE) tc::tma_2d(ra, &tmA, k0, am, &raw_full[rs]);
                        tc::tma_2d(ra + PL::RAWA, &tmB, k0, bn, &raw_full[rs]);
                    }
                    issued = i + 1;
                }
                if (PL::BULK) {
                    // pre-split operands go straight into the operand slot
                    const int cs = i % SL;
                    if (i >= SL && !gwait(&conv_empty[cs], (uint32_t)((i / SL - 1) & 1), wcap, &failed)) {
                        give_up(&failed);
                        break;
                    }
                    unsigned char* sl = conv + (size_t)cs * GB_SLOT;
                    tc::mbar_arrive_expect_tx(&b_full[cs], PL::BULK_BYTES);
                    if (APRE)
                        tc::bulk_g2s(sl, asplit + ((size_t)ma * total_stages + ks_) * (2 * GB_PART),
                                     2 * GB_PART, &b_full[cs]);
                    if (NN)
                        tc::bulk_g2s(sl + 2 * GB_PART,
                                     bsplit + ((size_t)nb_ * total_stages + ks_) * (2 * GB_PART), 2 * GB_PART,
                                     &b_full[cs]);
                    bissued = i + 1;
                }
            }
            // copies still in flight complete before the CTA may exit
            for (int i = issued > GB_RAW ? issued - GB_RAW : 0; i < issued; ++i)
                gwait(&raw_full[i % GB_RAW], (uint32_t)((i / GB_RAW) & 1), GB_DEFAULT_WAIT, &failed);
            for (int i = bissued > SL ? bissued - SL : 0; i < bissued; ++i)
                gwait(&b_full[i % SL], (uint32_t)((i / SL) & 1), GB_DEFAULT_WAIT, &failed);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issue
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_tf32(GB_M, GB_NR);
            constexpr uint32_t LBO = 128, SBO = (GB_KR / 4) * 128;
            bool ok = true;
            int u = 0;
            for (int i = 0; i < ns && ok; ++i) {
                const int cs = i % SL;
                const uint32_t par = (uint32_t)((i / SL) & 1);
                if ((PL::CONVERT && !gwait(&conv_full[cs], par, wcap, &failed)) ||
                    (PL::BULK && !gwait(&b_full[cs], par, wcap, &failed))) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t sa = tc::smem_u32(conv + (size_t)cs * GB_SLOT);
                // one accumulator per stage
                const int b = u % GB_ACC;
                if (u >= GB_ACC && !gwait(&acc_empty[b], (uint32_t)((u / GB_ACC - 1) & 1), wcap, &failed)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(b * GB_NR);
                // small cross terms of the four K-steps first (8 reals = two K chunks of 128 bytes) ...
                for (int kk = 0; kk < GB_KR / 8; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 256u;
                    tc::mma_tf32(d, tc::make_desc(sa + GB_PART + ko, LBO, SBO),
                                 tc::make_desc(sa + 2 * GB_PART + ko, LBO, SBO), idesc, kk > 0 ? 1u : 0u);
                    tc::mma_tf32(d, tc::make_desc(sa + ko, LBO, SBO), tc::make_desc(sa + 3 * GB_PART + ko, LBO, SBO),
                                 idesc, 1u);
                }
                // ... then the hi.hi products
                for (int kk = 0; kk < GB_KR / 8; ++kk) {
                    const uint32_t ko = (uint32_t)kk * 256u;
                    tc::mma_tf32(d, tc::make_desc(sa + ko, LBO, SBO), tc::make_desc(sa + 2 * GB_PART + ko, LBO, SBO),
                                 idesc, 1u);
                }
                tc::commit(&acc_full[b]);
                ++u;
                tc::commit(&conv_empty[cs]);   // the operand slot is free once these MMAs complete
            }
            if (!ok) give_up(&failed);
            // every MMA issued completes before the tensor memory is freed
            tc::commit(&mma_done);
            gwait(&mma_done, 0u, GB_DEFAULT_WAIT, &failed);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ workers: conversion, then drain
        const int wt = tid - 64;                // 0 .. 32 GB_WORKERS - 1
        const int q = warp & 3;                 // lane quadrant
        const int cg = (warp - 2) >> 2;         // complex columns 16 cg .. 16 cg + 15
        const int r = 32 * q + lane;            // tile row of the drain
        const int rr = wt & 127, c0 = wt >> 7;  // conversion of A: row rr, chunks c0 and c0 + 4
        float re[16], im[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) re[j] = im[j] = 0.f;
        bool ok = true;
        // CTA loop: stages left in the current tile's segment, its index,
        // and its tile
        int left = total_stages - s_first, seg = 0, t_drain = t_first;
        // A B: this thread's row and 16 columns of the tile at (mo, no),
        // times alpha, plus beta Cin
        auto write_nn = [&](int mo, int no) {
            const int m = mo + r;
            if (m >= M) return;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int n = no + 16 * cg + j;
                if (n < N) {
                    float2 o = make_float2(alpha * re[j], alpha * im[j]);
                    if (beta != 0.f) {
                        const float2 ci = Cin[(int64_t)n * ldcin + m];
                        o.x = fmaf(beta, ci.x, o.x);
                        o.y = fmaf(beta, ci.y, o.y);
                    }
                    Cout[(int64_t)n * ldc + m] = o;
                }
            }
        };
        for (int i = 0; i < ns + PL::LAG; ++i) {
            if (PL::CONVERT && i < ns) {
                const int rs = i % GB_RAW, cs = i % SL;
                if (!warp_wait(&raw_full[rs], (uint32_t)((i / GB_RAW) & 1), wcap, &failed) ||
                    (i >= SL && !warp_wait(&conv_empty[cs], (uint32_t)((i / SL - 1) & 1), wcap, &failed))) {
                    ok = false;
                    break;
                }
                const unsigned char* ra = raw + (size_t)rs * PL::RAWS;
                unsigned char* sl = conv + (size_t)cs * GB_SLOT;
                if (!NN) {
                    if (!APRE) {
                        // A row rr (column rr of A): 16 complex in eight 16-byte chunks,
                        // stored by the copy with the 128-byte swizzle
#pragma unroll
                        for (int h2 = 0; h2 < 2; ++h2) {
                            const int ch = c0 + 4 * h2;
                            const float4 v =
                                *reinterpret_cast<const float4*>(ra + rr * 128 + ((ch ^ (rr & 7)) << 4));
                            put_split(sl, cofs(rr, 4 * ch), v);
                        }
                    }
                    // B column j, chunk ch: the real-part row (re, im) and the
                    // imaginary-part row (im, -re)
                    const int j = wt & 63, ch = wt >> 6;
                    const float4 v =
                        *reinterpret_cast<const float4*>(ra + PL::RAWA + j * 128 + ((ch ^ (j & 7)) << 4));
                    put_split(sl + 2 * GB_PART, cofs(j, 4 * ch), v);
                    put_split(sl + 2 * GB_PART, cofs(GB_NC + j, 4 * ch), make_float4(v.y, -v.x, v.w, -v.z));
                } else {
                    // A row rr (plane wave m0 + rr): the raw slice is [k][m], 1 KB per k
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const int ch = c0 + 4 * h2;
                        const float2 a0 = *reinterpret_cast<const float2*>(ra + (2 * ch) * 1024 + rr * 8);
                        const float2 a1 = *reinterpret_cast<const float2*>(ra + (2 * ch + 1) * 1024 + rr * 8);
                        put_split(sl, cofs(rr, 4 * ch), make_float4(a0.x, a0.y, a1.x, a1.y));
                    }
                }
                tc::fence_async_smem();   // generic-proxy stores become visible to the tensor cores
                __syncwarp();
                if (lane == 0) {
                    tc::mbar_arrive(&raw_empty[rs]);
                    tc::mbar_arrive(&conv_full[cs]);
                }
            }
            const int dsg = i - PL::LAG;
            if (dsg >= 0) {
                const int b = dsg % GB_ACC;
                if (!warp_wait(&acc_full[b], (uint32_t)((dsg / GB_ACC) & 1), wcap, &failed)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t ta = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * GB_NR + 16 * cg);
                float v[16], w[16];
                tc::tmem_ld16_nowait(ta, v);
                tc::tmem_ld16_nowait(ta + GB_NC, w);
                tc::tmem_wait_ld();
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    re[j] += v[j];
                    im[j] += w[j];
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(&acc_empty[b]);
                if (SK) {
                    // the last stage of a tile in this CTA's run: its sums
                    // go out (A B: the result; A^H B: the partial sums to
                    // the segment slot), and the sums restart
                    if (--left == 0 || dsg == ns - 1) {
                        if (NN) {
                            write_nn((t_drain / sk.fast) * GB_M, (t_drain % sk.fast) * GB_NC);
                        } else {
                            float2* Pp = part + ((int64_t)blockIdx.x * sk.maxseg + seg) * GB_NC * GB_M;
#pragma unroll
                            for (int j = 0; j < 16; ++j) Pp[(int64_t)(16 * cg + j) * GB_M + r] = make_float2(re[j], im[j]);
                        }
#pragma unroll
                        for (int j = 0; j < 16; ++j) re[j] = im[j] = 0.f;
                        ++seg;
                        t_drain += tstep;
                        left = total_stages;
                    }
                }
            }
        }
        if (!ok) give_up(&failed);
        if (ok && !SK) {
            if (NN) {
                write_nn(m0, n0);
            } else {
                const int tile = blockIdx.x + blockIdx.y * gridDim.x;
                const int tiles = gridDim.x * gridDim.y;
                float2* P = part + ((int64_t)blockIdx.z * tiles + tile) * GB_NC * GB_M;
#pragma unroll
                for (int j = 0; j < 16; ++j) P[(int64_t)(16 * cg + j) * GB_M + r] = make_float2(re[j], im[j]);
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, GB_TCOLS);
    }
}

// A pre-split for the tall product A B, once per operand that does not
// change (the projector matrix): for each (128-row tile t, stage s of 16
// complex K) a block of hi (16 KB) then lo (16 KB) in the operand-slot
// layout, element (r, kr) = real part kr & 1 of A(128 t + r, 16 s + kr / 2)
// (A is M x K, column major).  Zero beyond M and K.
__global__ void k_tcg_asplit(int M, int K, const float2* __restrict__ A, int64_t lda, int nst, int mt,
                             unsigned char* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)mt * nst * GB_M * 8;
    if (idx >= total) return;
    const int ch = (int)(idx % 8);
    const int rr = (int)((idx / 8) % GB_M);
    const int s = (int)((idx / (8 * GB_M)) % nst);
    const int t = (int)(idx / (8 * GB_M * nst));
    const int m = t * GB_M + rr;
    float v[4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int k = s * GB_KC + 2 * ch + e;
        float2 a = make_float2(0.f, 0.f);
        if (k < K && m < M) a = A[(int64_t)k * lda + m];
        v[2 * e] = a.x;
        v[2 * e + 1] = a.y;
    }
    unsigned char* blk = out + ((size_t)t * nst + s) * (2 * GB_PART);
    float4 hi, lo;
    split4(make_float4(v[0], v[1], v[2], v[3]), hi, lo);
    *reinterpret_cast<float4*>(blk + cofs(rr, 4 * ch)) = hi;
    *reinterpret_cast<float4*>(blk + GB_PART + cofs(rr, 4 * ch)) = lo;
}

// B (K x N complex FP64, ldb) -> the NN kernel's N-side operand: for each
// (64-column tile t, stage s) a block of hi (16 KB) then lo (16 KB), rows
// j < 64 (re, -im) and 64 + j (im, re) of column 64 t + j, K-major core
// matrices; zero beyond K and N.
__global__ void k_tcg_bsplit(int K, int N, const double2* __restrict__ B, int ldb, int nst, int nt,
                             unsigned char* __restrict__ out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t total = (int64_t)nt * nst * GB_NR * 8;
    if (idx >= total) return;
    const int ch = (int)(idx % 8);
    const int r = (int)((idx / 8) % GB_NR);
    const int s = (int)((idx / (8 * GB_NR)) % nst);
    const int t = (int)(idx / (8 * GB_NR * nst));
    const int n = t * GB_NC + (r % GB_NC);
    float v[4];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const int k = s * GB_KC + 2 * ch + e;
        double2 b = make_double2(0.0, 0.0);
        if (k < K && n < N) b = B[(int64_t)n * ldb + k];
        if (r < GB_NC) {
            v[2 * e] = (float)b.x;
            v[2 * e + 1] = -(float)b.y;
        } else {
            v[2 * e] = (float)b.y;
            v[2 * e + 1] = (float)b.x;
        }
    }
    unsigned char* blk = out + ((size_t)t * nst + s) * (2 * GB_PART);
    const uint32_t off = (uint32_t)((((r >> 3) * (GB_KR / 4) + ch) << 7) + ((r & 7) << 4));
    float4 hi, lo;
    split4(make_float4(v[0], v[1], v[2], v[3]), hi, lo);
    *reinterpret_cast<float4*>(blk + off) = hi;
    *reinterpret_cast<float4*>(blk + GB_PART + off) = lo;
}

// C (M x N, FP64, ldc) = sum over the K splits of the CN partials, in split
// order (FP64 sums).
__global__ void k_tcg_reduce(int M, int N, int mt, int tiles, int ks, const float2* __restrict__ part,
                             double2* __restrict__ C, int ldc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * N) return;
    const int m = (int)(idx % M), n = (int)(idx / M);
    const int tile = (m / GB_M) + (n / GB_NC) * mt;
    const int64_t off = ((int64_t)tile * GB_NC + (n % GB_NC)) * GB_M + (m % GB_M);
    double sr = 0.0, si = 0.0;
    for (int z = 0; z < ks; ++z) {
        const float2 p = part[(int64_t)z * tiles * GB_NC * GB_M + off];
        sr += (double)p.x;
        si += (double)p.y;
    }
    C[(int64_t)n * ldc + m] = make_double2(sr, si);
}

// The stream-K partials of tile t: the CTAs whose unit runs meet the tile's
// units t T .. (t + 1) T - 1, in CTA (that is K) order, summed in FP64.
__global__ void k_tcg_reduce_sk(int M, int N, int mt, int T, SkPlan sk, const float2* __restrict__ part,
                                double2* __restrict__ C, int ldc) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)M * N) return;
    const int m = (int)(idx % M), n = (int)(idx / M);
    const int t = (m / GB_M) + (n / GB_NC) * mt;
    const int64_t off = (int64_t)(n % GB_NC) * GB_M + (m % GB_M);
    const int64_t ta = (int64_t)t * T, tb = ta + T;
    int c = (int)(ta * sk.ctas / sk.units) - 1;
    if (c < 0) c = 0;
    double sr = 0.0, si = 0.0;
    for (; c < sk.ctas; ++c) {
        const int64_t a = sk.units * c / sk.ctas, b = sk.units * (c + 1) / sk.ctas;
        if (a >= tb) break;
        if (b <= ta || a == b) continue;   // no unit of the tile (or none at all)
        const int seg = t - (int)(a / T);
        const float2 p = part[((int64_t)c * sk.maxseg + seg) * GB_NC * GB_M + off];
        sr += (double)p.x;
        si += (double)p.y;
    }
    C[(int64_t)n * ldc + m] = make_double2(sr, si);
}

int sm_count() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) {
            cudaGetLastError();
            n = 152;
        }
    }
    return n;
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

template <bool NN, bool APRE, bool SK = false>
void set_attr() {
    static bool done = false;
    if (!done) {
        cudaFuncSetAttribute(k_tcgemm<NN, APRE, SK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)GbPlan<NN, APRE>::SMEM);
        done = true;
    }
}

// Operands split once (tcg_presplit): looked up by address, leading
// dimension and shape, so that a call on another matrix never takes them.
struct PreSplit {
    const void* A;
    int64_t lda;
    int M, K;
    const unsigned char* split;
};
constexpr int kMaxPreSplit = 32;
PreSplit g_pre[kMaxPreSplit];
int g_npre = 0;

const unsigned char* find_presplit(const void* A, int64_t lda, int M, int K) {
    static int on = -1;
    if (on < 0) {
        // ROKS_TC_PRESPLIT=0 converts every operand in the kernel (for comparisons)
        const char* e = std::getenv("ROKS_TC_PRESPLIT");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    if (!on) return nullptr;
    for (int i = 0; i < g_npre; ++i) {
        const PreSplit& p = g_pre[i];
        if (p.A == A && p.lda == lda && p.M == M && p.K == K) return p.split;
    }
    return nullptr;
}

// Schedule of A^H B (tcg_set_waves): 2 (the default) is the stream-K
// schedule over one wave of one CTA per SM; 5 and 8 split K into 2.5 or 4
// waves.  Stream-K removes the partial last wave of the split (P^H Psi at
// mgo-120: 385 CTAs ran as 3 waves of 148): 1.45 -> 1.23 ms.
int g_waves_x2 = 2;

// K splits of a CN product: about g_waves_x2 / 2 waves of CTAs
// waves_x2 = 2: the stream-K schedule over one wave (one CTA per SM)
SkPlan cn_stream_k(int mt, int nt, int total) {
    SkPlan p;
    if (g_waves_x2 != 2) return p;
    p.ctas = sm_count();
    p.fast = mt;
    p.units = (int64_t)mt * nt * total;
    const int64_t len = (p.units + p.ctas - 1) / p.ctas;
    p.maxseg = (int)((len + total - 1) / total) + 1;
    return p;
}

int cn_splits(int tiles, int total) {
    int ks = (g_waves_x2 * sm_count() / 2 + tiles - 1) / tiles;
    if (ks > total) ks = total;
    if (ks < 1) ks = 1;
    const int per = (total + ks - 1) / ks;
    return (total + per - 1) / per;
}

}  // namespace

// The tensor-core path is the default for shapes it takes; ROKS_TENSOR_CORES=0
// keeps every contraction on the SIMT kernels.
bool tcg_enabled() {
    static int on = -1;
    if (on < 0) {
        const char* e = std::getenv("ROKS_TENSOR_CORES");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

void tcg_set_waves(int waves_x2) { g_waves_x2 = waves_x2 >= 1 ? waves_x2 : 2; }

bool tcg_cn_takes(int M, int N, int K) { return tcg_enabled() && M >= 128 && N >= 64 && K >= 1024; }
bool tcg_nn_takes(int M, int N, int K) { return tcg_enabled() && M >= 4096 && N >= 64 && K >= 64; }

size_t tcg_cn_work_bytes(int M, int N, int K) {
    // the larger of the split-K and the stream-K partials (the autotuner
    // may take either after the buffer is sized)
    const int mt = (M + GB_M - 1) / GB_M, nt = (N + GB_NC - 1) / GB_NC, total = (K + GB_KC - 1) / GB_KC;
    size_t split = 0;
    for (int w : {3, 5, 8}) {
        const int keep = g_waves_x2;
        g_waves_x2 = w;
        split = std::max(split, (size_t)mt * nt * cn_splits(mt * nt, total));
        g_waves_x2 = keep;
    }
    const int ctas = sm_count();
    const int64_t len = ((int64_t)mt * nt * total + ctas - 1) / ctas;
    const size_t sk = (size_t)ctas * (size_t)((len + total - 1) / total + 1);
    return std::max(split, sk) * GB_NC * GB_M * sizeof(float2);
}

size_t tcg_nn_work_bytes(int N, int K) {
    const int nt = (N + GB_NC - 1) / GB_NC, total = (K + GB_KC - 1) / GB_KC;
    return (size_t)nt * total * 2 * GB_PART;
}

size_t tcg_presplit_bytes(int M, int K) {
    const size_t mt = (M + GB_M - 1) / GB_M, nst = (K + GB_KC - 1) / GB_KC;
    return mt * nst * 2 * GB_PART;
}

bool tcg_presplit(int M, int K, const float2* A, int64_t lda, void* out, cudaStream_t st) {
    if (g_npre >= kMaxPreSplit || !aligned(out, 16)) return false;
    const int mt = (M + GB_M - 1) / GB_M, nst = (K + GB_KC - 1) / GB_KC;
    const int64_t n = (int64_t)mt * nst * GB_M * 8;
    unsigned char* o = static_cast<unsigned char*>(out);
    roks::count_launch();
    k_tcg_asplit<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(M, K, A, lda, nst, mt, o);
    if (cudaGetLastError() != cudaSuccess) return false;
    g_pre[g_npre++] = PreSplit{A, lda, M, K, o};
    return true;
}

void tcg_presplit_forget(const void* split) {
    int w = 0;
    for (int i = 0; i < g_npre; ++i)
        if (g_pre[i].split != split) g_pre[w++] = g_pre[i];
    g_npre = w;
}

static long long g_tcg_launches = 0;
long long tcg_launches_take() {
    const long long n = g_tcg_launches;
    g_tcg_launches = 0;
    return n;
}

// C = A^H B on the tensor cores; false when the shape, the alignment or the
// work buffer does not allow it (the caller then takes the SIMT kernels).
bool gemm_cn_tcg(int M, int N, int K, const float2* A, int64_t lda, const float2* B, int64_t ldb, double2* C, int ldc,
                 void* work, size_t work_bytes, cudaStream_t st) {
    if (!tcg_cn_takes(M, N, K)) return false;
    if ((lda & 1) || (ldb & 1) || !aligned(A, 16) || !aligned(B, 16) || !aligned(work, 16)) return false;
    const int mt = (M + GB_M - 1) / GB_M, nt = (N + GB_NC - 1) / GB_NC, total = (K + GB_KC - 1) / GB_KC;
    const SkPlan sk = cn_stream_k(mt, nt, total);
    const int ks = sk.ctas > 0 ? 1 : cn_splits(mt * nt, total);
    const int per = (total + ks - 1) / ks;
    if (tcg_cn_work_bytes(M, N, K) > work_bytes) return false;
    // (A^H B converts both operands in the kernel: a pre-split A, copied as
    // 32 KB hi/lo blocks while the workers still convert B, measured slower
    // on P^H Psi at mgo-120, 1.45 -> 1.49 ms)
    CUtensorMap tmA, tmB;
    if (!tensor_map_2d(&tmA, A, K, M, lda, GB_KC, GB_M, true) || !tensor_map_2d(&tmB, B, K, N, ldb, GB_KC, GB_NC, true))
        return false;
    float2* part = static_cast<float2*>(work);
    roks::count_launch();
    g_tcg_launches += 1;
    if (sk.ctas > 0) {
        set_attr<false, false, true>();
        k_tcgemm<false, false, true><<<dim3(sk.ctas, 1, 1), GB_THREADS, GbPlan<false, false>::SMEM, st>>>(
            M, N, per, total, sk, tmA, tmB, nullptr, nullptr, part, nullptr, 0, nullptr, 0, 0.f, 0.f, wait_polls());
    } else {
        set_attr<false, false>();
        k_tcgemm<false, false><<<dim3(mt, nt, ks), GB_THREADS, GbPlan<false, false>::SMEM, st>>>(
            M, N, per, total, sk, tmA, tmB, nullptr, nullptr, part, nullptr, 0, nullptr, 0, 0.f, 0.f, wait_polls());
    }
    const int64_t outs = (int64_t)M * N;
    roks::count_launch();
    if (sk.ctas > 0)
        k_tcg_reduce_sk<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(M, N, mt, total, sk, part, C, ldc);
    else
        k_tcg_reduce<<<(unsigned)((outs + 255) / 256), 256, 0, st>>>(M, N, mt, mt * nt, ks, part, C, ldc);
    return true;
}

// Cout = alpha A B + beta Cin on the tensor cores (B FP64, small); false when
// not applicable.  Cout may be Cin; it must not overlap A.
bool gemm_nn_tcg(int M, int N, int K, const float2* A, int64_t lda, const double2* B, int ldb, const float2* Cin,
                 int64_t ldcin, float2* Cout, int64_t ldc, float alpha, float beta, void* bwork, size_t bwork_bytes,
                 cudaStream_t st) {
    if (!tcg_nn_takes(M, N, K) || !bwork) return false;
    if ((lda & 1) || !aligned(A, 16) || !aligned(bwork, 16) || !aligned(Cout, 8)) return false;
    if (beta != 0.f && (!Cin || !aligned(Cin, 8))) return false;
    if (static_cast<const void*>(A) == static_cast<const void*>(Cout)) return false;
    const int nt = (N + GB_NC - 1) / GB_NC, total = (K + GB_KC - 1) / GB_KC;
    if (tcg_nn_work_bytes(N, K) > bwork_bytes) return false;
    const unsigned char* as = find_presplit(A, lda, M, K);
    CUtensorMap tmA{};
    if (!as && !tensor_map_2d(&tmA, A, M, K, lda, GB_M, GB_KC, false)) return false;
    unsigned char* bs = static_cast<unsigned char*>(bwork);
    const int64_t nsplit = (int64_t)nt * total * GB_NR * 8;
    roks::count_launch();
    k_tcg_bsplit<<<(unsigned)((nsplit + 255) / 256), 256, 0, st>>>(K, N, B, ldb, total, nt, bs);
    roks::count_launch();
    g_tcg_launches += 1;
    const int mt = (M + GB_M - 1) / GB_M;
    const dim3 grid(nt, mt, 1);
    // more tiles than SMs: persistent CTAs, one per SM, each looping over
    // whole tiles (tile t: N tile t % nt, M tile t / nt) with its pipeline
    // running on across them
    SkPlan pp;
    if ((int64_t)mt * nt > sm_count()) {
        pp.ctas = sm_count();
        pp.units = (int64_t)mt * nt;
        pp.fast = nt;
    }
    if (pp.ctas > 0) {
        const dim3 g1(pp.ctas, 1, 1);
        if (as) {
            set_attr<true, true, true>();
            k_tcgemm<true, true, true><<<g1, GB_THREADS, GbPlan<true, true>::SMEM, st>>>(
                M, N, total, total, pp, tmA, tmA, bs, as, nullptr, Cin, ldcin, Cout, ldc, alpha, beta,
                wait_polls());
        } else {
            set_attr<true, false, true>();
            k_tcgemm<true, false, true><<<g1, GB_THREADS, GbPlan<true, false>::SMEM, st>>>(
                M, N, total, total, pp, tmA, tmA, bs, nullptr, nullptr, Cin, ldcin, Cout, ldc, alpha, beta,
                wait_polls());
        }
        return true;
    }
    if (as) {
        set_attr<true, true>();
        k_tcgemm<true, true><<<grid, GB_THREADS, GbPlan<true, true>::SMEM, st>>>(
            M, N, total, total, SkPlan{}, tmA, tmA, bs, as, nullptr, Cin, ldcin, Cout, ldc, alpha, beta,
            wait_polls());
    } else {
        set_attr<true, false>();
        k_tcgemm<true, false><<<grid, GB_THREADS, GbPlan<true, false>::SMEM, st>>>(
            M, N, total, total, SkPlan{}, tmA, tmA, bs, nullptr, nullptr, Cin, ldcin, Cout, ldc, alpha, beta,
            wait_polls());
    }
    return true;
}

int tcg_timeout_take() {
    int h = 0;
    if (cudaMemcpyFromSymbol(&h, g_tcg_timeout, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (h) {
        const int z = 0;
        cudaMemcpyToSymbol(g_tcg_timeout, &z, sizeof(int));
    }
    return h;
}

}  // namespace roks
