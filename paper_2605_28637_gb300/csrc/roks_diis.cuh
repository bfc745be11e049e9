// roks_diis.cuh -- device state and kernels' host wrappers of the DIIS
// solver on the ROKS residual (Sec. II A; Pulay extrapolation in the form of
// Hutter, Luthi and Parrinello 1994).  Internal to the library.
#pragma once

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
