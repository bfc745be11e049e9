// roks_mlp.cuh -- the learned correction of the TPA preconditioner (internal).
#pragma once

#include <cmath>

#include "roks_grid.cuh"

namespace roks {

constexpr int kMlpHidden = 64;
constexpr int kMlpParams = kMlpHidden * 3 + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden + kMlpHidden + 1;

// s[i] for the n feature rows U (n x 3); bf16: round the weights to BF16.
void mlp_forward(int n, const float* U, const float* params, bool bf16, float* s, cudaStream_t st);
// grad = d/dp sum w (s - t)^2 / sum w, loss = that mean (device scalars);
// work holds mlp_grad_work_floats(n) floats.
size_t mlp_grad_work_floats(int n);
void mlp_grad(int n, const float* U, const float* t, const float* w, const float* params, float* work, float* grad,
              float* loss, cudaStream_t st);
// One Adam step (step counts from 1) on the FP32 master weights.
void mlp_adam(float* p, float* m, float* v, const float* g, int step, float lr, float b1, float b2, float eps,
              cudaStream_t st);
// out = K m g (TPA factor times the network's multiplier) for a residual
// block; sums = column sums (|g|^2, |G|^2 |g|^2) per band; eps_n = Theta_nn /
// wband_n; m = 1 when params is null or sc->mlp_off > 0 (sc may be null: on).
template <typename T>
void precondition_mlp(int npw, int nb, const c2<T>* gI, int64_t ld, const T* g2h, const double* sums,
                      const double2* Theta, const double* wband, const float* params, const PcgScalars* sc,
                      c2<T>* out, int64_t ldo, cudaStream_t st);
// The features (npw * nb rows of 3, band by band) of a residual block.
template <typename T>
void mlp_features(int npw, int nb, const c2<T>* g, int64_t ld, const T* g2h, const double* sums,
                  const double2* Theta, const double* wband, float* U, cudaStream_t st);

}  // namespace roks
