// roks_force.cuh -- host wrappers of the force kernels (Sec. II B).  Internal
// to the library.
#pragma once

#include "roks_impl.cuh"

namespace roks {

constexpr int kForceLocBlocks = 64;   // grid slices per atom of the local term

// Local term: tab (natoms x 3 x N) <- e^{-iG_c R_c} per axis; grid <- the
// forward transform of rho_w = sum_k w[k] rho_k (rho3 in DensAcc<T> storage);
// part (natoms x 3 x kForceLocBlocks) <- slices of
// sum_G f_nu v_a(G) Im(e^{-iG.R_a} conj(rho)), v_a(G) = amp[a] exp(-|G|^2 w2h[a]).
// The derivative is Omega b / N^3 times the sum of a row of part.
template <typename T>
void force_local(int N, double L, int natoms, const double* atoms, const double* rho3, const double* w, const T* amp,
                 const T* w2h, c2<T>* tab, c2<T>* grid, const c2<T>* tw, double* part, cudaStream_t st);
// out = -i G_nu P (all projectors), leading dimension ld
template <typename T>
void force_dP(int npw, int nproj, const c2<T>* P, int64_t ld, const int* miller, double b, int nu, c2<T>* out,
              cudaStream_t st);
// c[nu * nproj + i] = 2 Re sum_n conj(dB_nu[i, n]) (DBw - Y)[i, n]; dB holds the
// three derivatives one after the other (nproj x nb each, column major)
void force_nl(int nproj, int nb, const double2* dB, const double2* DBw, const double2* Y, double* c,
              cudaStream_t st);
// forces[a * 3 + nu] = -(scale * sum part row + sum of c over the projectors of atom a)
void force_collect(int natoms, int nproj, const int* owner, const double* c, const double* part, double scale,
                   double* forces, cudaStream_t st);

}  // namespace roks
