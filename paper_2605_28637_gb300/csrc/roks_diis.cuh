// roks_diis.cuh -- device state and kernels' host wrappers of the DIIS
// solver on the ROKS residual (Sec. II A; Pulay extrapolation in the form of
// Hutter, Luthi and Parrinello 1994).  Internal to the library.
#pragma once

#include <cmath>

#include "roks_impl.cuh"

namespace roks {

constexpr int kDiisMax = 8;   // longest history (ring slots)

// Device state of the DIIS history.  B is indexed by ring slot,
// B[j * kDiisMax + k] = sum_n Re <e_jn|e_kn>; the window (the pairs the
// extrapolation uses, oldest first) and its coefficients are written by
// diis_solve.
struct DiisState {
    double B[kDiisMax * kDiisMax];
    double d[kDiisMax];
    int slot[kDiisMax];
    int h;          // window size; 0 if no window passed (non-finite B)
    int pad;
    double E0, Enew, rnorm2;
};

// Ring slots of the pairs stored so far, oldest first; the last is the newest.
struct DiisOrder {
    int n;
    int slot[kDiisMax];
};

// The window test and the coefficients (host and device): B by ring slot
// (B[j * kDiisMax + k], symmetric over the slots of ord).  For h from ord.n
// down to 2, the h most recent pairs pass when every Cholesky pivot of the
// normalised Gram matrix D^-1/2 B D^-1/2 (D = diag B) satisfies L_kk^2 >= tol;
// their coefficients are d = B^-1 1 / (1^T B^-1 1), solved through that
// factor.  Otherwise the newest pair alone (d = 1).  Writes d and the ring
// slots of the window (oldest first); returns h, or 0 when the newest
// diagonal entry is not finite.
__host__ __device__ inline int diis_window_coefficients(const double* B, const DiisOrder& ord, double tol,
                                                        double* d, int* slot_out) {
    const int n = ord.n;
    const int ns = ord.slot[n - 1];
    for (int h = n; h >= 2; --h) {
        const int o = n - h;
        double q[kDiisMax], L[kDiisMax][kDiisMax];
        bool ok = true;
        for (int j = 0; j < h && ok; ++j) {
            const double bjj = B[ord.slot[o + j] * kDiisMax + ord.slot[o + j]];
            ok = bjj > 0.0 && isfinite(bjj);
            q[j] = ok ? 1.0 / sqrt(bjj) : 0.0;
        }
        for (int j = 0; j < h && ok; ++j) {
            for (int i = j; i < h; ++i) {
                double v = B[ord.slot[o + i] * kDiisMax + ord.slot[o + j]] * q[i] * q[j];
                for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
                if (i == j) {
                    if (!(v >= tol)) {
                        ok = false;
                        break;
                    }
                    L[j][j] = sqrt(v);
                } else {
                    L[i][j] = v / L[j][j];
                }
            }
        }
        if (!ok) continue;
        // Bn z = D^-1/2 1, y = D^-1/2 z = B^-1 1, d = y / sum y
        double w[kDiisMax];
        for (int i = 0; i < h; ++i) {
            double v = q[i];
            for (int k = 0; k < i; ++k) v -= L[i][k] * w[k];
            w[i] = v / L[i][i];
        }
        for (int i = h - 1; i >= 0; --i) {
            double v = w[i];
            for (int k = i + 1; k < h; ++k) v -= L[k][i] * w[k];
            w[i] = v / L[i][i];
        }
        double sum = 0.0;
        for (int i = 0; i < h; ++i) {
            w[i] *= q[i];
            sum += w[i];
        }
        if (!(sum != 0.0 && isfinite(sum))) continue;
        for (int i = 0; i < h; ++i) {
            d[i] = w[i] / sum;
            slot_out[i] = ord.slot[o + i];
        }
        return h;
    }
    d[0] = 1.0;
    slot_out[0] = ns;
    return isfinite(B[ns * kDiisMax + ns]) ? 1 : 0;
}

// Lambda_mn = theta_mn - lambda_mn (theta_mn - conj theta_nm), lambda_mn = 1/2
// except lambda[ia, ib] = lab and lambda[ib, ia] = lba (ia < 0: none).
// Column major, nb x nb, FP64.
void diis_multipliers(int nb, const double2* Theta, int ia, int ib, double lab, double lba, double2* Lam,
                      cudaStream_t st);
// Row of the newest pair: B[ns][slot_k] = sum_n Re <e_new,n|e_k,n> for every
// pair of ord (ns = its last slot), in one pass over the error vectors; the
// pair of ring slot j is e_ring + j blk, leading dimension ld.  part holds
// kDiisMax * diis_gram_blocks(npw, nb) doubles.
int diis_gram_blocks(int npw, int nb);
template <typename T>
void diis_gram(int npw, int nb, const c2<T>* enew, const c2<T>* ering, int64_t blk, int64_t ld,
               const DiisOrder& ord, double* part, DiisState* s, cudaStream_t st);
// Completes B symmetrically from the newest row, then picks the largest
// window of the most recent pairs whose normalised Gram matrix passes the
// Cholesky pivot test (every L_kk^2 >= tol) and solves for the coefficients
// d = B^-1 1 / (1^T B^-1 1) of that window (FP64).  rnorm2 = sum of the nb
// band norms rn (the squared residual norm).
void diis_solve(DiisState* s, const DiisOrder& ord, double tol, const double* rn, int nb, cudaStream_t st);
// out[g, n] = sum_k d_k (Psi_k[g, n] + tau e_k[g, n]) over the window; the
// pair of ring slot j is (psi_ring + j blk, e_ring + j blk), leading dimension ld.
template <typename T>
void diis_combine(int npw, int nb, const DiisState* s, const c2<T>* psi_ring, const c2<T>* e_ring, int64_t blk,
                  int64_t ld, double tau, c2<T>* out, int64_t ldo, cudaStream_t st);

}  // namespace roks
