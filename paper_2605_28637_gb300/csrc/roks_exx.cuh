// roks_exx.cuh -- exact-exchange launch arguments (internal).
#pragma once

#include "roks_impl.cuh"

namespace roks {

constexpr int kExxBlocks = 64;   // reduction blocks per pair in k_exx_mult

// Coefficients derived from the occupations: c[k][k'] = -alpha Omega^{1/2}
// w(k, k') for the exchange field, fM/fT[k][k'] = sum over the spins of a
// configuration of f_k f_k', wxc[k'] = w(closed, k').
struct ExxCoef {
    double c[3][3];
    double fM[3][3];
    double fT[3][3];
    double wxc[3];
    double alpha;
    int n_closed;
};

template <typename T>
struct ExxArgs {
    int N, nb, npairs, batch;
    double L;
    const c2<T>* tw;      // grid twiddles
    const T* vG;          // v(G) / N^3
    const c2<T>* Phi;     // real-space orbitals, nb x N^3
    c2<T>* X;             // exchange fields, nb x N^3
    c2<T>* buf;           // batch x N^3
    const int* pj;        // pair list (n ascending, then j)
    const int* pn;
    double* part;         // batch x kExxBlocks
    double* Kmat;         // nb x nb
    double* hf2;          // [E_hf^M, E_hf^T] before alpha
    double* open_diag;    // exchange part of <a|F^c|a>, <b|F^c|b>
    ExxCoef cf;
};

template <typename T>
void exx_setup_kernel(int N, double L, int bare, T* vG, cudaStream_t st);
// K for all pairs, the energies and the open-band diagonal; the exchange
// fields X too when want_field.
template <typename T>
void exx_pairs(const ExxArgs<T>& a, bool want_field, cudaStream_t st);
// The grid work of one batch of pairs p0 .. p0 + np - 1 (k_exx_grid.cuh):
// pair densities, transforms, v(G) and the block partials of the pair
// integrals in a.part (np x kExxBlocks), and with want_field the fields
// added to a.X.
template <typename T>
void exx_batch_grid(const ExxArgs<T>& a, int p0, int np, bool want_field, cudaStream_t st);

}  // namespace roks
