// k_mlp.cu -- the learned correction of the TPA preconditioner: a per
// (plane wave, band) network with three inputs, two tanh layers of 64 and one
// output s; the TPA step is scaled by m = exp(clip(s, -3, 3)).
//
// Training runs on the GPU in these kernels: a forward/backward pass over
// blocks of samples writes per-block gradient partials (samples summed in a
// fixed order), a second kernel sums the partials in block order with
// two-sum compensation, and an Adam kernel updates the FP32 master weights.
// Inference (the fused preconditioner inside the PCG step) holds the weights
// in shared memory rounded to BF16.
//
// Parameter layout (4481 floats): W1 (64 x 3, row major), b1 (64), W2
// (64 x 64, row major), b2 (64), w3 (64), b3 (1).
#include <cuda_bf16.h>

#include "roks_grid.cuh"
#include "roks_mlp.cuh"

namespace roks {

namespace {

constexpr int H = kMlpHidden;
constexpr int OW1 = 0, OB1 = 3 * H, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H, OB3 = OW3 + H;
static_assert(OB3 + 1 == kMlpParams, "layout");

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Loads the parameters into shared memory (optionally rounded to BF16).
__device__ __forceinline__ void load_params(const float* __restrict__ p, float* w, bool bf16) {
    for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = bf16 ? bf16_round(p[i]) : p[i];
}

// s for one feature vector; h1, h2 receive the activations when non-null.
__device__ __forceinline__ float mlp_eval(const float* w, float u0, float u1, float u2, float* h1o, float* h2o) {
    float h1[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float z = w[OB1 + j];
        z = fmaf(w[OW1 + 3 * j + 0], u0, z);
        z = fmaf(w[OW1 + 3 * j + 1], u1, z);
        z = fmaf(w[OW1 + 3 * j + 2], u2, z);
        h1[j] = tanhf(z);
        if (h1o) h1o[j] = h1[j];
    }
    float s = w[OB3];
#pragma unroll 4
    for (int k = 0; k < H; ++k) {
        const float4* row = reinterpret_cast<const float4*>(w + OW2 + H * k);
        float z = w[OB2 + k];
#pragma unroll
        for (int q = 0; q < H / 4; ++q) {
            const float4 c = row[q];
            z = fmaf(c.x, h1[4 * q + 0], z);
            z = fmaf(c.y, h1[4 * q + 1], z);
            z = fmaf(c.z, h1[4 * q + 2], z);
            z = fmaf(c.w, h1[4 * q + 3], z);
        }
        const float h2 = tanhf(z);
        if (h2o) h2o[k] = h2;
        s = fmaf(w[OW3 + k], h2, s);
    }
    return s;
}

__global__ void __launch_bounds__(256) k_mlp_forward(int n, const float* __restrict__ U,
                                                     const float* __restrict__ params, int bf16,
                                                     float* __restrict__ s) {
    extern __shared__ __align__(16) float mlp_w[];
    load_params(params, mlp_w, bf16 != 0);
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    s[i] = mlp_eval(mlp_w, U[3 * i], U[3 * i + 1], U[3 * i + 2], nullptr, nullptr);
}

// Per-block gradient partials of sum_i w_i (s_i - t_i)^2 over the block's
// samples (one thread per sample in the forward pass), plus [sum w r^2,
// sum w] at the end: part[block][kMlpParams + 2].
constexpr int GB = 128;   // samples (and threads) per block
constexpr int HP = H + 1; // padded row of the activation tiles

__global__ void __launch_bounds__(GB) k_mlp_grad_partial(int n, const float* __restrict__ U,
                                                         const float* __restrict__ t, const float* __restrict__ wt,
                                                         const float* __restrict__ params, float* __restrict__ part) {
    extern __shared__ __align__(16) float sm[];
    float* w = sm;                          // kMlpParams (+ pad to 4)
    float* h1s = w + ((kMlpParams + 3) / 4) * 4;
    float* h2s = h1s + GB * HP;             // h2, then dz2
    float* d1s = h2s + GB * HP;             // dz1
    float* us = d1s + GB * HP;              // GB x 3
    float* dss = us + GB * 3;               // ds
    __shared__ float lw[2][GB];
    load_params(params, w, false);
    __syncthreads();
    const int tid = threadIdx.x;
    const int i = blockIdx.x * GB + tid;
    const bool valid = i < n;
    float ds = 0.f, wi = 0.f, lnum = 0.f;
    {
        float h1[H];
        const float u0 = valid ? U[3 * i] : 0.f, u1 = valid ? U[3 * i + 1] : 0.f, u2 = valid ? U[3 * i + 2] : 0.f;
        us[3 * tid] = u0;
        us[3 * tid + 1] = u1;
        us[3 * tid + 2] = u2;
        const float s = mlp_eval(w, u0, u1, u2, h1, h2s + tid * HP);
#pragma unroll
        for (int j = 0; j < H; ++j) h1s[tid * HP + j] = h1[j];
        if (valid) {
            wi = wt[i];
            const float r = s - t[i];
            ds = 2.f * wi * r;
            lnum = wi * r * r;
        }
        dss[tid] = ds;
        lw[0][tid] = lnum;
        lw[1][tid] = wi;
    }
    __syncthreads();
    float* P = part + (int64_t)blockIdx.x * (kMlpParams + 2);
    // output layer: gw3[k] = sum_i ds_i h2[i][k], gb3 = sum_i ds_i
    for (int k = tid; k <= H; k += GB) {
        float a = 0.f;
        if (k < H)
            for (int q = 0; q < GB; ++q) a = fmaf(dss[q], h2s[q * HP + k], a);
        else
            for (int q = 0; q < GB; ++q) a += dss[q];
        P[k < H ? OW3 + k : OB3] = a;
    }
    if (tid == 0) {
        float a = 0.f, b = 0.f;
        for (int q = 0; q < GB; ++q) {
            a += lw[0][q];
            b += lw[1][q];
        }
        P[kMlpParams] = a;
        P[kMlpParams + 1] = b;
    }
    __syncthreads();
    // per sample: dz2 = ds w3 (1 - h2^2) (over h2), dz1 = (W2^T dz2) (1 - h1^2)
    {
        float d2[H];
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const float h2 = h2s[tid * HP + k];
            d2[k] = ds * w[OW3 + k] * (1.f - h2 * h2);
            h2s[tid * HP + k] = d2[k];
        }
#pragma unroll 4
        for (int j = 0; j < H; ++j) {
            float a = 0.f;
#pragma unroll
            for (int k = 0; k < H; ++k) a = fmaf(w[OW2 + H * k + j], d2[k], a);
            const float h1 = h1s[tid * HP + j];
            d1s[tid * HP + j] = a * (1.f - h1 * h1);
        }
    }
    __syncthreads();
    // gW2[k][j] = sum_i dz2[i][k] h1[i][j]; gb2[k] = sum_i dz2[i][k]
    for (int e = tid; e < H * H; e += GB) {
        const int k = e / H, j = e % H;
        float a = 0.f;
        for (int q = 0; q < GB; ++q) a = fmaf(h2s[q * HP + k], h1s[q * HP + j], a);
        P[OW2 + e] = a;
    }
    for (int k = tid; k < H; k += GB) {
        float a = 0.f, b = 0.f;
        for (int q = 0; q < GB; ++q) {
            a += h2s[q * HP + k];
            b += d1s[q * HP + k];
        }
        P[OB2 + k] = a;
        P[OB1 + k] = b;
    }
    // gW1[j][c] = sum_i dz1[i][j] u[i][c]
    for (int e = tid; e < H * 3; e += GB) {
        const int j = e / 3, c = e % 3;
        float a = 0.f;
        for (int q = 0; q < GB; ++q) a = fmaf(d1s[q * HP + j], us[3 * q + c], a);
        P[OW1 + e] = a;
    }
}

// grad[p] = sum_b part[b][p] / sum w (block order, two-sum); loss likewise.
__global__ void k_mlp_grad_reduce(int nblk, const float* __restrict__ part, float* __restrict__ grad,
                                  float* __restrict__ loss) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p > kMlpParams) return;
    auto sum_col = [&](int col) {
        float s = 0.f, c = 0.f;
        for (int b = 0; b < nblk; ++b) {
            const float v = part[(int64_t)b * (kMlpParams + 2) + col];
            const float t = s + v, bp = t - s;
            c += (s - (t - bp)) + (v - bp);
            s = t;
        }
        return s + c;
    };
    const float sw = sum_col(kMlpParams + 1);
    const float inv = sw > 0.f ? 1.f / sw : 0.f;
    if (p < kMlpParams) grad[p] = sum_col(p) * inv;
    else if (loss) loss[0] = sum_col(kMlpParams) * inv;
}

__global__ void k_mlp_adam(int np, float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ g, float lr, float b1, float b2, float c1, float c2, float eps) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// Fused preconditioner of the PCG step: out = K m g_I with K the TPA factor
// (X_n = 1.5 T_n, T_n the kinetic energy of the residual) and m the network's
// multiplier on the features (log1p(x), log1p(|g|/rms_n), eps_n); m = 1 while
// the correction is suspended (sc->mlp_off > 0) or no weights are set.
template <typename T>
__global__ void __launch_bounds__(256) k_precond_mlp(int npw, const c2<T>* __restrict__ gI, int64_t ld,
                                                     const T* __restrict__ g2h, const double* __restrict__ sums,
                                                     int nb, const double2* __restrict__ Theta,
                                                     const double* __restrict__ wband,
                                                     const float* __restrict__ params, const PcgScalars* sc,
                                                     c2<T>* __restrict__ out, int64_t ldo) {
    extern __shared__ __align__(16) float mlp_w[];
    __shared__ float band[5];   // 1/X, -2/X, 1/T, 1/rms, eps
    __shared__ int use;
    const int n = blockIdx.y;
    if (threadIdx.x == 0) {
        const double s0 = fmax(sums[n], 1e-300), s1 = sums[nb + n];
        const double X = 1.5 * s1 / s0;           // sums carry |G|^2 |g|^2
        const double Tn = 0.5 * s1 / s0;
        band[0] = float(1.0 / X);
        band[1] = float(-2.0 / X);
        band[2] = float(1.0 / fmax(Tn, 1e-300));
        band[3] = float(1.0 / sqrt(s0 / npw));
        band[4] = float(Theta[(int64_t)n * nb + n].x / wband[n]);
        use = (params != nullptr && (sc == nullptr || sc->mlp_off <= 0.0)) ? 1 : 0;
    }
    __syncthreads();
    if (use) load_params(params, mlp_w, true);
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npw) return;
    const c2<T> a = gI[(int64_t)n * ld + g];
    const float gh = float(g2h[g]);
    const float x = 2.f * gh * band[0];
    const float num = 27.f + x * (18.f + x * (12.f + 8.f * x));
    float K = band[1] * num / (num + 16.f * x * x * x * x);
    if (use) {
        const float amp = sqrtf(float(a.x) * float(a.x) + float(a.y) * float(a.y));
        const float s = mlp_eval(mlp_w, log1pf(gh * band[2]), log1pf(amp * band[3]), band[4], nullptr, nullptr);
        K *= expf(fminf(fmaxf(s, -3.f), 3.f));
    }
    out[(int64_t)n * ldo + g] = mk<T>(T(K) * a.x, T(K) * a.y);
}

template <typename T>
__global__ void k_mlp_features(int npw, const c2<T>* __restrict__ gI, int64_t ld, const T* __restrict__ g2h,
                               const double* __restrict__ sums, int nb, const double2* __restrict__ Theta,
                               const double* __restrict__ wband, float* __restrict__ U) {
    __shared__ float band[3];   // 1/T, 1/rms, eps
    const int n = blockIdx.y;
    if (threadIdx.x == 0) {
        const double s0 = fmax(sums[n], 1e-300), s1 = sums[nb + n];
        band[0] = float(1.0 / fmax(0.5 * s1 / s0, 1e-300));
        band[1] = float(1.0 / sqrt(s0 / npw));
        band[2] = float(Theta[(int64_t)n * nb + n].x / wband[n]);
    }
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= npw) return;
    const c2<T> a = gI[(int64_t)n * ld + g];
    const float amp = sqrtf(float(a.x) * float(a.x) + float(a.y) * float(a.y));
    float* u = U + 3 * ((int64_t)n * npw + g);
    u[0] = log1pf(float(g2h[g]) * band[0]);
    u[1] = log1pf(amp * band[1]);
    u[2] = band[2];
}

size_t grad_smem() {
    return sizeof(float) * (((kMlpParams + 3) / 4) * 4 + 3 * GB * HP + GB * 3 + GB);
}

}  // namespace

void mlp_forward(int n, const float* U, const float* params, bool bf16, float* s, cudaStream_t st) {
    if (n <= 0) return;
    const size_t sm = sizeof(float) * kMlpParams;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    roks::count_launch(), k_mlp_forward<<<(n + 255) / 256, 256, sm, st>>>(n, U, params, bf16 ? 1 : 0, s);
}

size_t mlp_grad_work_floats(int n) { return (size_t)((n + GB - 1) / GB) * (kMlpParams + 2); }

void mlp_grad(int n, const float* U, const float* t, const float* w, const float* params, float* work, float* grad,
              float* loss, cudaStream_t st) {
    const int nblk = (n + GB - 1) / GB;
    if (nblk <= 0) return;
    const size_t sm = grad_smem();
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_grad_partial, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    roks::count_launch(), k_mlp_grad_partial<<<nblk, GB, sm, st>>>(n, U, t, w, params, work);
    roks::count_launch(), k_mlp_grad_reduce<<<(kMlpParams + 1 + 255) / 256, 256, 0, st>>>(nblk, work, grad, loss);
}

void mlp_adam(float* p, float* m, float* v, const float* g, int step, float lr, float b1, float b2, float eps,
              cudaStream_t st) {
    const double c1 = 1.0 / (1.0 - std::pow((double)b1, step));
    const double c2 = 1.0 / (1.0 - std::pow((double)b2, step));
    roks::count_launch(), k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(kMlpParams, p, m, v, g, lr, b1, b2,
                                                                             (float)c1, (float)c2, eps);
}

template <typename T>
void precondition_mlp(int npw, int nb, const c2<T>* gI, int64_t ld, const T* g2h, const double* sums,
                      const double2* Theta, const double* wband, const float* params, const PcgScalars* sc,
                      c2<T>* out, int64_t ldo, cudaStream_t st) {
    const size_t sm = sizeof(float) * kMlpParams;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_precond_mlp<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        attr = true;
    }
    dim3 g((npw + 255) / 256, nb);
    roks::count_launch(), k_precond_mlp<T><<<g, 256, sm, st>>>(npw, gI, ld, g2h, sums, nb, Theta, wband, params, sc,
                                                               out, ldo);
}

template <typename T>
void mlp_features(int npw, int nb, const c2<T>* g, int64_t ld, const T* g2h, const double* sums,
                  const double2* Theta, const double* wband, float* U, cudaStream_t st) {
    dim3 grid((npw + 255) / 256, nb);
    roks::count_launch(), k_mlp_features<T><<<grid, 256, 0, st>>>(npw, g, ld, g2h, sums, nb, Theta, wband, U);
}
template void mlp_features<float>(int, int, const float2*, int64_t, const float*, const double*, const double2*,
                                  const double*, float*, cudaStream_t);
template void mlp_features<double>(int, int, const double2*, int64_t, const double*, const double*, const double2*,
                                   const double*, float*, cudaStream_t);

template void precondition_mlp<float>(int, int, const float2*, int64_t, const float*, const double*, const double2*,
                                      const double*, const float*, const PcgScalars*, float2*, int64_t, cudaStream_t);
template void precondition_mlp<double>(int, int, const double2*, int64_t, const double*, const double*,
                                       const double2*, const double*, const float*, const PcgScalars*, double2*,
                                       int64_t, cudaStream_t);

}  // namespace roks
