// roks_grid.cuh -- declarations of the grid, reduction and PCG-step kernels'
// host wrappers (internal to the library).
#pragma once

#include "roks_impl.cuh"

namespace roks {

constexpr int kMaxBlk = 16;   // projectors per atom

// Occupation-derived coefficients of the class potentials (Eq. 13):
// f[k][ch] = f_k^{sigma L}, C[k][ch] = c_L f_k^{sigma L}, w[k] = sum_ch C[k][ch],
// channels (up M, down M, up T, down T); xscale = 1 - alpha.
struct PotCoef {
    double f[3][4];
    double C[3][4];
    double w[3];
    double xscale;
};
// The same coefficients in the element type, converted once on the host.
template <typename T>
struct PotCoefT {
    T f[3][4];
    T C[3][4];
    T xscale;
};

void vloc_setup(int N, double L, int natoms, const double* atoms_dev, double2* grid, double* vloc,
                const double2* tw64, cudaStream_t st);
template <typename T>
void projectors_setup(int npw, int nproj, double L, const int* miller_dev, const double* proj_dev, c2<T>* P,
                      int64_t ldp, cudaStream_t st);
// Bands band0 .. band0 + nbands - 1 of the seeded start from uniforms u_dev
// (numbered from band0) or, when u_dev is null, from SplitMix64(seed).
template <typename T>
void init_orbitals(int npw, int band0, int nbands, const double* u_dev, uint64_t seed, const double* g2, c2<T>* psi,
                   int64_t ld, cudaStream_t st);
template <typename T>
void to_real_type(int64_t n, const double* in, T* out, double scale, cudaStream_t st);
// op 0: kinetic 0.5 g2 |x|^2; 1: (|x|^2, g2 |x|^2) -> out[0..nb), out[nb..2nb), and the TPA
// coefficients (1/X_n, -2/X_n) -> out[2nb..4nb) (out holds 4 nb for op 1); 2: Re <x|y>; 3: |x|^2.
// g2h = |G|^2 / 2 in the element type.  part must hold 2 * nb * 16 doubles.
template <typename T>
void column_sums(int op, int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy,
                 const T* g2h, double* part, double* out, cudaStream_t st);
// dst = scale * sum over the columns of column_sums' op 2 or 3 (out unused),
// summed in the same order as column_sums followed by sum_to.
template <typename T>
void column_total(int op, int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy,
                  const T* g2h, double* part, double* dst, double scale, cudaStream_t st);
void apply_DQ(int nproj, int nb, const double2* B, const int* blk_off, const int* blk_n, const double* Drow,
              const double* Qrow, const double* wband, double2* DB, double2* QB, cudaStream_t st);
void band_quadratic(int nproj, int nb, const double2* B, const double2* DB, double* out, cudaStream_t st);
// rho3 (3 x N^3) in DensAcc<T> storage -> FP64 values (out may not alias rho3)
template <typename T>
void density_to_f64(int64_t n, const double* rho3, double* out, cudaStream_t st);
// Grid transforms in the element type T (FP32 for the mixed path), energies
// in FP64.  rho3 in DensAcc<T> storage; vloc and the exchange-correlation
// fields xc3 (3 x N^3) in the element type T.  energies_only: out6[0..3]
// alone (no inverse transform, no class potentials Vk).
//
// gga: work grids of PBE exchange (the GGA); null keeps the Slater exchange.
// Per spin channel e = e_Slater F_x(s), F_x = 1 + mu s^2 / (1 + mu s^2 /
// kappa), s^2 = |grad rho|^2 / (4 (6 pi^2)^{2/3} rho^{8/3}), and v = de/drho -
// div(2 de/d|grad rho|^2 grad rho), with spectral derivatives (i G_c, the
// Nyquist index of axis c left out); a channel at or below rho_min carries
// no exchange.
struct GgaWork {
    void* gg = nullptr;   // 2 N^3 complex T: the channel pairs (up M + i down M, up T + i down T)
    void* dd = nullptr;   // 6 N^3 complex T: their three derivatives, then the fluxes
    void* v4 = nullptr;   // 4 N^3 T: de/drho per channel
    double mu = 0, kappa = 0, rho_min = 0;
};
template <typename T>
void potentials(int N, double L, const double* rho3, const T* vloc, const PotCoef& cf, c2<T>* grid,
                T* xc3, const c2<T>* tw, T* Vk, double* Vk64, double* part, double* out6,
                cudaStream_t st, bool energies_only = false, const GgaWork* gga = nullptr);
size_t potentials_part_elems();
template <typename T>
void precondition(int npw, int nb, const c2<T>* gI, int64_t ld, const T* g2h, const double* sums, c2<T>* out,
                  int64_t ldo, cudaStream_t st);
template <typename T>
void axpy(int npw, int nb, const c2<T>* x, int64_t ldx, const c2<T>* y, int64_t ldy, const double* coef,
          double csign, c2<T>* out, int64_t ldo, cudaStream_t st);

// ------------------------------------------------------------ PCG step, band-space part (k_pcg.cu)
// Device scalars of one PCG iteration.
struct PcgScalars {
    double E0, Et, Enew;      // energies at the start, trial, new point
    double pg, pg_prev;       // <p|g> now and at the previous step (0 = none)
    double beta;              // Fletcher-Reeves ratio in use
    double a1, a2, r1, r2;    // Re<u|G>, Re<v|G>, Re sum A^* Gin, Re sum A_prev^* Gin
    double pgI;               // Re <p_I|g_I>
    double rot_pg;            // (1/2) Re sum A^* Gin
    double dE0;               // directional derivative
    double dt;                // trial step
    double step;              // accepted step
    double rot;               // 1 when the rotation is used
    double restarted;
    double has_prev;          // 1 when a previous direction exists
    double cur;               // scalar used by launches that scale by a device value
    double gnorm2;
    double coup_re, coup_im;
    double neg_one;           // constant -1 for device-scaled axpy
    double mlp_off;           // iterations left with the learned correction suspended
};

// Gam = (Theta + Theta^H)/2, Gin = Theta - Theta^H, R (Eq. 20) -> A (Eqs. 22-23),
// and the open-shell coupling; shell[n] is the shell index of band n.  The
// diagonal d_m = <m|F^c|m> is Re theta_mm for closed bands and is formed from
// expectation values for open ones (w_c (<m|T|m> + <m|V_nl|m>) + <m|V^c|m>,
// plus the exchange term when open_x is given).
//
// Empty bands (n_occ <= n < nb, the empty shell of Eq. 20): their columns of
// theta hold <m|F^c|n>.  The energy's operator there is F^e = 0, so Gam, Gin
// and the inter-shell R take theta with those columns zero; R within the
// empty shell is F^c.  An occupied band m of class k and an empty band n
// rotate by A_mn = (1/2) atan2(2|R|, <n|F^k|n> - <m|F^k|m>) R/|R|, which
// takes m to the lower eigenvector of the pair's 2 x 2 block of F^k;
// dk[k * n_empty + (n - n_occ)] = <n|F^k|n>.  n_occ = nb: no empty bands.
void pcg_rotation(int nb, int n_closed, const double2* Theta, const double* kin_b, const double* nl_b,
                  const double* open_vc, const double* open_x, double wc, const int* shell, int suppress_ab, int ia,
                  int ib, double2* Gam, double2* Gin, double2* A, PcgScalars* sc, cudaStream_t st, int n_occ,
                  const double* dk);
// <e|F^k|e> = w_k (<e|T|e> + <e|V_nl|e>) + dvol sum_r V^k(r) rho_e(r) of the
// n_empty empty bands e = n_occ + i, k = 0, 1, 2 (w_k = w0, w1, w2; class potentials Vk, 3 x N3
// in the element type; rho_e: the band densities in the element type's
// density storage, band i at rho_e + (i + 1) N3) -> dk[k * n_empty + i].
// part: at least 3 n_empty x 64 doubles.
template <typename T>
void empty_band_diagonal(int64_t N3, int n_empty, int n_occ, const double* rho_e, const T* Vk, double dvol,
                         const double* kin_b, const double* nl_b, double w0, double w1, double w2, double* part,
                         double* dk, cudaStream_t st);
// sc->rot_pg = 1/2 Re sum conj(A) Gin; sc->r1, r2 as named.
void pcg_rot_dots(int nb, const double2* A, const double2* Aprev, const double2* Gin, double* part, PcgScalars* sc,
                  cudaStream_t st);
// Decide beta / restart / rotation, set dE0 and the trial step.
void pcg_direction(PcgScalars* sc, cudaStream_t st);
// A_tot = rot * (A + beta Aprev)
void pcg_total_rotation(int nb, const double2* A, const double2* Aprev, PcgScalars* sc, double2* Atot,
                        cudaStream_t st);
// Parabola through E0, dE0, Et -> step; next trial; pg_prev.
void pcg_line_search(PcgScalars* sc, cudaStream_t st);
// sc->cur = sc->(field); used to feed device-scaled launches.
void pcg_set_cur(PcgScalars* sc, int field, cudaStream_t st);
// Energy combination on the device: out (11 doubles) from the pieces.
void energy_combine(const double* kin_b, const double* nl_b, int nb, const double* wband, const double* out6,
                    double cM, double cT, double alpha, const double* hf2, double* E, cudaStream_t st);
// Copy E[total] into a scalar field.
void pcg_take_energy(const double* E, PcgScalars* sc, int field, cudaStream_t st);
// Hermitian part: O <- (O + O^H)/2
void hermitize(int n, double2* O, cudaStream_t st);


}  // namespace roks
