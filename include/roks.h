/*
 * roks.h -- C ABI of the GB300 (sm_103a) ROKS plane-wave hot path.
 *
 * The method: restricted open-shell Kohn-Sham DFT for the lowest excited
 * singlet, E_S = 2 E(Phi_1) - E(Phi_3) (Eq. 1), minimised over one set of
 * spatial orbitals shared by the mixed-spin configuration Phi_1 (a up,
 * b down) and the triplet Phi_3 (a up, b up), subject to <m|S|n> = delta_mn
 * (Eq. 2), by all-band preconditioned conjugate gradients (Sec. II A,
 * Eqs. 5-24).  Orbitals are expanded in plane waves on a cubic cell at the
 * Gamma point.  The Hamiltonian model: kinetic energy, Gaussian local wells,
 * separable s/p projectors sum |p_i> D_ij <p_j| with overlap
 * S = 1 + sum |p_i> Q_ij <p_j| (Eq. 3), Hartree, LSDA Slater exchange per
 * spin channel and an optional exact-exchange fraction alpha with a
 * spherically truncated Coulomb kernel.
 *
 * Conventions for every entry point:
 *  - Orbitals Psi are column-major, npw x nbands complex numbers stored as
 *    interleaved (re, im) pairs, leading dimension ld >= npw (in complex
 *    elements).  Element type: double for ROKS_FP64, float for ROKS_MIXED.
 *    Column order is closed bands, then open band a, then open band b.
 *  - Coefficient index g follows the basis order of roks_basis().
 *  - Device pointers belong to the caller; they must stay valid for the
 *    duration of the call (stream ordered).  The library owns its internal
 *    workspaces and frees them in roks_destroy().
 *  - All work is ordered on the CUDA stream given to roks_setup().  Calls
 *    that return host values (roks_potential, roks_pcg_step, roks_diis_step,
 *    roks_forces, roks_energies_get) synchronise that stream; the others do
 *    not.
 *  - Errors are returned as roks_status; roks_last_error() gives text.  No
 *    C++ exception crosses this interface.  A context is not thread safe.
 */
#ifndef ROKS_H
#define ROKS_H

#include <stdint.h>

#if defined(__GNUC__)
#define ROKS_API __attribute__((visibility("default")))
#else
#define ROKS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct roks_ctx roks_ctx;

typedef enum {
    ROKS_OK = 0,
    ROKS_EINVAL = 1,      /* invalid argument or unsupported size            */
    ROKS_ENOMEM = 2,      /* device or host allocation failed                 */
    ROKS_ECUDA = 3,       /* a CUDA runtime call failed                       */
    ROKS_ENOTPOSDEF = 4,  /* overlap matrix not positive definite (Cholesky) */
    ROKS_ENOCONV = 5,     /* iteration limit reached without convergence      */
    ROKS_ETIMEOUT = 6,    /* a bounded device wait ran out                    */
    ROKS_EDIVERGED = 7    /* non-finite energy or gradient                    */
} roks_status;

enum { ROKS_FP64 = 0, ROKS_MIXED = 1 };
/* Occupation modes (Sec. II A): 0 closed-shell ground state, one
 * configuration with c = 1; 1 ROKS singlet, c_M = 2, c_T = -1 (Eq. 1);
 * 2 triplet configuration alone, c_T = 1. */
enum { ROKS_MODE_GS = 0, ROKS_MODE_SINGLET = 1, ROKS_MODE_TRIPLET = 2 };

/* Cubic cell of side L (Bohr) with an N x N x N FFT grid.  Supported N:
 * 16, 24, 32, 48, 72, 96, 120. */
typedef struct {
    double L;
    int grid;
} roks_cell;

/* Atom: position (Bohr), species index, Gaussian local well
 * V(r) = -depth * exp(-|r-R|^2 / (2 width^2)), summed over periodic images
 * and band limited to the grid (Nyquist planes excluded). */
typedef struct {
    double pos[3];
    int species;
    double depth;   /* Ha */
    double width;   /* Bohr */
} roks_atom;

/* Projector set of a species: nproj channels, channel c has angular
 * momentum l[c] (0 = s, 1 = p), Cartesian component m[c] (p only: 0 x,
 * 1 y, 2 z) and Gaussian radius rc[c] (Bohr).  In reciprocal space
 * p_c(G) = Omega^{-1/2} N_l (2 pi rc^2)^{3/2} exp(-G^2 rc^2/2) Y(G) exp(-iG.R),
 * Y = 1 (s) or -i rc^2 G_m (p), N_l giving unit norm.  D (Ha) and Q
 * (dimensionless) are nproj x nproj symmetric, row major.  The arrays are
 * read during roks_setup only. */
typedef struct {
    int nproj;
    const int* l;
    const int* m;
    const double* rc;
    const double* D;
    const double* Q;
} roks_species;

/* n_closed doubly occupied bands; modes 1 and 2 add the two singly
 * occupied bands a, b (Fig. 1A).  n_open states the open-shell size and must
 * be 0 for ROKS_MODE_GS and 2 for the other modes (ROKS_EINVAL otherwise).
 *
 * n_empty unoccupied bands (the empty shell of Eq. 20) follow: bands are
 * ordered closed, a, b, empty.  They carry no occupation in any
 * configuration, so the densities, energies and forces are those of the
 * occupied bands.  In a PCG step they enter the R matrix (F^s between an
 * occupied shell s and the empty shell, F^c within it), an occupied-empty
 * pair rotates the occupied band to the lower eigenvector of the pair's
 * 2 x 2 block of its own operator, and each empty band moves along its
 * preconditioned F^c residual, so the empty bands relax to the lowest
 * eigenvectors of F^c outside the occupied space.  roks_apply_h applies F^c
 * to them; the gradient roks_gradient_parts writes is the energy's
 * (F^e = 0) and its g_I the F^c residual.  Not with exact exchange
 * (alpha != 0) or the Gamma-point form (ROKS_EINVAL); roks_diis_step
 * returns ROKS_EINVAL on a context with empty bands. */
typedef struct {
    int n_closed;
    int n_open;
    int mode;
    int n_empty;
} roks_occ;

/* Exact-exchange kernels v(G) of the pair potentials (Sec. III hybrid). */
enum {
    ROKS_EXX_TRUNCATED = 0,   /* spherical truncation, v = 4 pi (1 - cos(|G| R_c)) / G^2,
                                 v(0) = 2 pi R_c^2, R_c = (3 Omega / 4 pi)^(1/3) */
    ROKS_EXX_BARE = 1         /* bare Coulomb 4 pi / G^2 without the G = 0 term  */
};

/* Exchange functional of the spin channels (Eq. 8's v_x^{sigma L}), scaled
 * by (1 - alpha).  Per channel density rho (a spin density):
 *   SLATER: e = -(3/4) (6/pi)^{1/3} rho^{4/3}, v = -(6 rho/pi)^{1/3} (LSDA);
 *   PBE_X:  the GGA exchange of Perdew, Burke and Ernzerhof (the paper's
 *           molecules use PBE, Sec. III): e = e_Slater F_x(s), F_x = 1 +
 *           mu s^2 / (1 + mu s^2/kappa), kappa = 0.804, mu = beta pi^2/3,
 *           s^2 = |grad rho|^2 / (4 (6 pi^2)^{2/3} rho^{8/3}), and v =
 *           de/drho - div(2 de/d|grad rho|^2 grad rho), the derivatives
 *           spectral on the grid (i G, the Nyquist index of each axis left
 *           out); a channel at or below 1e-10 Bohr^-3 carries no exchange.
 *           Without correlation, like the Slater model. */
enum {
    ROKS_XC_SLATER = 0,
    ROKS_XC_PBE_X = 1
};

/* Options.  Every field after e_tol takes its default when zero. */
typedef struct {
    int precision;     /* ROKS_FP64, or ROKS_MIXED: FP32 transforms and
                          contractions, band-space work in FP32 on FP64
                          storage (the overlap Cholesky in deviation form
                          O = I + Delta up to 64 bands, so that its rounding
                          scales with |Delta|), FP64 energy combination and
                          PCG scalars, compensated FP32 block sums           */
    double alpha;      /* exact-exchange fraction (0 = none); Slater exchange
                          is scaled by (1 - alpha)                           */
    int suppress_ab;   /* 1: zero the open-shell a-b block of R (Eq. 20),
                          the coupling suppression of Sec. II A              */
    double e_tol;      /* convergence: |E_i+1 - E_i| < e_tol (Ha) on two
                          consecutive steps (0: 1e-6)                        */
    double g_tol;      /* and, when > 0, the gradient norm |g| (PCG) or the
                          residual norm |R| (DIIS) of the last step < g_tol  */
    int max_iter;      /* > 0: a step that is the max_iter-th since the last
                          roks_init_orbitals, roks_orthonormalize or
                          roks_invalidate without having converged returns
                          ROKS_ENOCONV (its update is kept)                  */
    uint64_t seed;     /* SplitMix64 seed of roks_init_orbitals when it is
                          given no host random numbers                       */
    int precond;       /* ROKS_PRECOND_TPA (0) or ROKS_PRECOND_TPA_MLP: the
                          learned correction with all-zero weights (m = 1,
                          TPA itself) until roks_set_preconditioner loads
                          trained ones                                       */
    int autotune;      /* 1: roks_setup times the candidate launch shapes of
                          the band transforms and keeps the fastest          */
    int exx_kernel;    /* ROKS_EXX_TRUNCATED (0) or ROKS_EXX_BARE            */
    int wait_cap;      /* polls of every bounded device wait (mbarrier waits
                          of the streamed and tensor-core contractions) before
                          it gives up with ROKS_ETIMEOUT; 0: 2^26; < 0: no
                          poll at all, so every such wait gives up (a test of
                          the timeout path).  Copies already in flight are
                          still waited for with the default cap.             */
    int gamma;         /* 1: real orbitals at the Gamma point (the only
                          k-point the paper samples, Sec. III) on the half
                          sphere.  The basis is G = 0 and the Miller triples
                          after it in the basis order (npw_half =
                          (npw_full + 1) / 2); every orbital-shaped array the
                          calls take or return holds, per band, c(0) (real)
                          and sqrt(2) c(G) for the other half-sphere G, so
                          that Re sum conj(a) b over the rows is the full
                          inner product.  Two bands share one complex
                          transform.  Requires alpha = 0 and, with an open
                          shell, an even n_closed (ROKS_EINVAL otherwise).   */
    int xc;            /* ROKS_XC_SLATER (default) or ROKS_XC_PBE_X.  PBE
                          exchange holds 8 complex and 4 real grids of work
                          space and adds 16 grid transforms to a potential. */
} roks_options;

/* Energy terms (Ha).  E_kin, E_loc, E_nl carry the occupation weights;
 * E_M, E_T are the two configuration energies, E_total = c_M E_M + c_T E_T
 * (E_S for the singlet, Eq. 1). */
typedef struct {
    double E_kin, E_loc, E_nl, E_H;
    double E_x_M, E_x_T;          /* (1 - alpha) Slater exchange per configuration */
    double E_hf_M, E_hf_T;        /* exact-exchange integrals (before alpha)       */
    double E_M, E_T, E_total;
} roks_energies;

/* Result of one PCG iteration. */
typedef struct {
    double E;            /* energy at the start of the step                 */
    double E_new;        /* energy after the step                           */
    double step;         /* Delta of Eqs. 5 and 24                          */
    double grad_norm;    /* Frobenius norm of the constrained gradient g    */
    double coupling_re;  /* <a|F^a - F^b|b> at the start (Eq. 15)           */
    double coupling_im;
    double beta;         /* Fletcher-Reeves ratio used (0 after a restart)  */
    double dE0;          /* directional derivative of E along the step      */
    int restarted;       /* 1 when the CG direction was reset               */
    int converged;       /* 1 once |dE| < e_tol on two consecutive steps
                            (and grad_norm < g_tol when g_tol > 0)           */
} roks_step_info;

/* Builds the plane-wave basis (Miller vectors with |G|^2/2 <= ecut, tested
 * in integers as i^2+j^2+k^2 <= floor(2 ecut (L/2pi)^2); loops i, j, k
 * ascending from -n to n), the local potential, the projectors and all
 * device workspaces, on `cuda_stream` (a cudaStream_t, or NULL for the
 * legacy default stream) of the current device.  Returns ROKS_EINVAL for an
 * unsupported grid, a grid smaller than 2 n + 1, or bad counts.  On success
 * *out owns device memory until roks_destroy(). */
ROKS_API roks_status roks_setup(const roks_cell* cell, double ecut, int natoms,
                       const roks_atom* atoms, int nspecies,
                       const roks_species* species, const roks_occ* occ,
                       const roks_options* opt, void* cuda_stream,
                       roks_ctx** out);

/* Basis size, band count, the minimal leading dimension, and a host
 * pointer to the npw x 3 Miller indices (row major, owned by the context).
 * With roks_options.gamma these are the half-sphere rows. */
ROKS_API roks_status roks_basis(roks_ctx* ctx, int* npw, int* nbands, int* ld_min,
                       const int32_t** miller);

/* Initial orbitals (seeded start): u_host holds nbands x npw x 2 uniform
 * numbers in [-1, 1) (band major, re/im innermost); the library forms
 * c_nG = (u_re + i u_im)/(1 + |G|^2) and S-orthonormalises them into psi
 * (device, ld >= npw).  u_host is read before the call returns.  With
 * u_host NULL the numbers are drawn on the device: number i (same order) is
 * -1 + 2 (z_i >> 11) 2^-53, z_i output i of SplitMix64 seeded with
 * roks_options.seed (z_i = mix(seed + (i + 1) 0x9E3779B97F4A7C15) with
 * Vigna's mixing function).  Allocates nothing (host numbers are staged in
 * the context's workspaces).  Resets the direction and DIIS histories.
 * With roks_options.gamma, npw is the half sphere's: c(0) keeps its real
 * part and the other rows are stored times sqrt(2) before the
 * orthonormalisation. */
ROKS_API roks_status roks_init_orbitals(roks_ctx* ctx, const double* u_host,
                               void* psi, int64_t ld);

/* Forgets everything the context derived from orbital buffers: the density
 * and potentials, the projector coefficients P^H psi, the transform planes,
 * the PCG direction and DIIS histories.  Steps and force calls key these on
 * the buffer address and leading dimension alone, so a caller that writes
 * new values into a buffer a step or force call has used (a copy from the
 * host, an in-place edit) calls this before the next call on it. */
ROKS_API roks_status roks_invalidate(roks_ctx* ctx);

/* Class densities rho_k(r) = sum_{n in k} |psi_n(r)|^2, k = closed, a, b
 * (the inputs of the spin densities of Eq. 8), plus the kinetic and
 * non-local energy terms of psi.  rho_out (optional, device, 3 x N^3 double,
 * grid index (x N + y) N + z) receives a copy. */
ROKS_API roks_status roks_density(roks_ctx* ctx, const void* psi, int64_t ld,
                         double* rho_out);

/* From the last roks_density: channel densities rho^{sigma L}, one Hartree
 * solve (rho_M = rho_T), Slater exchange per channel and the class
 * potentials V^k = w_k (V_loc + V_H) + sum_{sigma L} c_L f_k v_x (Eqs. 8, 13).
 * Fills *e (host; may be NULL).  vclass_out (optional, device, 3 x N^3 of
 * the orbital element type) receives V^closed, V^a, V^b.  Synchronises. */
ROKS_API roks_status roks_potential(roks_ctx* ctx, roks_energies* e, void* vclass_out);

/* Shell operators applied to each band with the last roks_potential:
 * fpsi_n = F^{k(n)}|n> (Eq. 13: kinetic + local + non-local, and exact
 * exchange if alpha != 0).  spsi (optional) = S|n>.  grad (optional)
 * = g_n = F^n|n> - sum_m S|m> gamma_nm with gamma of Eq. 11.  All outputs
 * are device arrays with the same ld as psi. */
ROKS_API roks_status roks_apply_h(roks_ctx* ctx, const void* psi, int64_t ld,
                         void* fpsi, void* spsi, void* grad);

/* roks_apply_h with both gradients of the step (Eqs. 7, 11, 12), from
 * theta = Psi^H F Psi: grad = F|n> - sum_m S|m> gamma_nm (gamma = (theta +
 * theta^H) / 2) and grad_I = F|n> - sum_m S|m> theta_mn, the part the
 * preconditioner of Eq. 16 takes.  spsi, grad and grad_I may each be NULL;
 * fpsi may not.  Device arrays with the same ld as psi; the call also leaves
 * theta for roks_precondition's band energies. */
ROKS_API roks_status roks_gradient_parts(roks_ctx* ctx, const void* psi, int64_t ld, void* fpsi, void* spsi,
                                void* grad, void* grad_I);

/* In place S-orthonormalisation: O = Psi^H S Psi = L L^H (Cholesky: FP64
 * on the FP64 path; on the mixed path FP32 in deviation form up to 64 bands
 * and blocked FP32 beyond), Psi <- Psi L^{-H}; band order closed, a, b.
 * ROKS_ENOTPOSDEF if O is not positive definite. */
ROKS_API roks_status roks_orthonormalize(roks_ctx* ctx, void* psi, int64_t ld);

/* One PCG iteration on psi (in place, S-orthonormal on entry and exit):
 * gradient and gamma (Eqs. 7, 11), split (Eq. 12), TPA preconditioning
 * (Eqs. 17, 18), Fletcher-Reeves direction (Eq. 6), R-matrix rotation
 * generator (Eqs. 20-23), parabolic line search on E (Eq. 5) and the update
 * orth((Psi + Delta s) exp(Delta (A^i + beta A^{i-1}))) (Eq. 24).  The
 * direction history lives in the context; the first call (or the first after
 * roks_init_orbitals / roks_orthonormalize) starts with steepest descent.
 * psi must not be modified by the caller between consecutive steps (or
 * roks_invalidate must be called after such a change).  ROKS_EDIVERGED for
 * a non-finite energy or gradient (checked before any other status);
 * ROKS_ENOCONV past roks_options.max_iter.  Fills *info (host).
 * Synchronises. */
ROKS_API roks_status roks_pcg_step(roks_ctx* ctx, void* psi, int64_t ld,
                          roks_step_info* info);

/* ------------------------------------------------------------------
 * DIIS on the ROKS residual (Sec. II A): the paper minimises E_S also with
 * a DIIS solver (Pulay extrapolation as in Hutter, Luthi and Parrinello
 * 1994) on the residual of Frank et al.,
 *   R_n = F^n|n> - sum_m S|m> Lambda_mn,
 *   Lambda_mn = theta_mn - lambda_mn (theta_mn - theta_nm^*),
 *   theta_mn = <m|F^n|n>,
 * lambda_mn = 1/2 for every pair (then R is the gradient g of Eq. 7) except
 * the open pair: lambda_ab (component along |a> of the residual of b) and
 * lambda_ba (component along |b> of the residual of a); the paper's choice
 * for excited singlets of the same symmetry as the ground state is
 * lambda_ab = 1/2, lambda_ba = -1/2.  One step:
 *   e = tau K R with the TPA preconditioner K (Eqs. 17, 18), no S-projection;
 *   the pair (Psi, e) joins the last `history` pairs;
 *   B_jk = sum_n Re <e_jn|e_kn>; the window is the largest set of the most
 *   recent pairs whose normalised Gram matrix D^-1/2 B D^-1/2 (D = diag B)
 *   has every Cholesky pivot L_kk^2 >= 1e-7;
 *   d = B^-1 1 / (1^T B^-1 1) over the window (real, sum d = 1: the
 *   minimiser of |sum d_j e_j|^2);
 *   psi <- orth(sum_j d_j (Psi_j + e_j)) (Cholesky S-orthonormalisation).
 * The history lives in the context.  It starts afresh on the first call, on
 * a change of psi, ld or any option, after a PCG step, roks_init_orbitals
 * or roks_orthonormalize; a DIIS step likewise makes the next PCG step start
 * with steepest descent.  DIIS uses the TPA preconditioner alone (the learned
 * correction, if set, applies to PCG only). */
#define ROKS_DIIS_MAX 8
typedef struct {
    int history;       /* pairs kept, 1 .. ROKS_DIIS_MAX (1: preconditioned
                          steepest descent with step tau)                   */
    double tau;        /* step scale of the error vector, > 0               */
    double lambda_ab;  /* coupling coefficients of the open pair (singlet   */
    double lambda_ba;  /*   mode only; other modes ignore them)             */
} roks_diis_options;

typedef struct {
    double E;          /* energy at the start of the step                   */
    double E_new;      /* energy of the extrapolated, orthonormal orbitals  */
    double res_norm;   /* Frobenius norm of the residual R at the start     */
    int window;        /* pairs the extrapolation used                      */
    double coef[ROKS_DIIS_MAX];   /* their coefficients, oldest first        */
    int converged;     /* 1 once |E_new - E| < e_tol on two consecutive steps
                          (and res_norm < g_tol when g_tol > 0)             */
} roks_diis_info;

/* One DIIS step on psi (in place, S-orthonormal on entry and exit; psi
 * unmodified by the caller between steps, as for roks_pcg_step).  opt
 * NULL takes history 6, tau 1/2, lambda_ab = lambda_ba = 1/2.  ROKS_EINVAL
 * for options out of range; ROKS_EDIVERGED for a non-finite residual or
 * energy; ROKS_ENOTPOSDEF if the extrapolated orbitals are linearly
 * dependent.  Fills *info (host).  Synchronises. */
ROKS_API roks_status roks_diis_step(roks_ctx* ctx, void* psi, int64_t ld, const roks_diis_options* opt,
                                    roks_diis_info* info);

/* Forces on the atoms (Sec. II B, generalised Hellmann-Feynman theorem):
 *   F_Inu = -dE/dR_Inu,
 *   dE/dR_Inu = sum_{L sigma n} c_L f_n^{sigma L} <n|dH^{sigma L}/dR_Inu|n>
 *             - sum_mn gamma_mn <m|dS/dR_Inu|n>,
 * with gamma of Eq. 11 formed from psi.  In this model the wells and the
 * projectors carry the dependence on the atoms:
 *   local:     Omega sum_G (-i G_nu) v_I(G) e^{-iG.R_I} conj(rho_w(G)),
 *              rho_w = sum_n w_n |psi_n|^2, grid G without the Nyquist planes;
 *   projector: 2 Re sum_{i in I} sum_n conj(<dp_i|n>) [w_n (D B)_in - (Q B Gam)_in],
 *              B = P^H psi, dp_i/dR_nu = -i G_nu p_i, Gam_mn = gamma_nm.
 * The paper sums the overlap term in the basis that diagonalises gamma; the
 * double sum used here has the same value.  At stationary orbitals this is
 * the total derivative of the minimised E_S; at other orbitals it is the
 * derivative at fixed orbitals and multipliers of E - sum gamma (S - 1).
 * forces_host: natoms x 3 doubles (Ha/Bohr, atom order of roks_setup, x y z
 * innermost), written before the call returns.  Uses the density and
 * potentials of psi when a PCG or DIIS step (or a force call) on the same
 * buffer and leading dimension left them current, and forms them otherwise;
 * after writing new orbitals into such a buffer, call roks_invalidate first.
 * The call leaves the step's own state (potentials, projector coefficients,
 * direction history) as it was: the next step on psi proceeds unchanged.
 * ROKS_EDIVERGED for a non-finite force.  Synchronises. */
ROKS_API roks_status roks_forces(roks_ctx* ctx, const void* psi, int64_t ld, double* forces_host);

/* Launch shapes in use (the autotuner's choices when roks_options.autotune
 * was set, else the defaults): the number of band groups of the density's
 * x-stage transform (2, 4 or 8; default 4) and the schedule of the
 * tensor-core A^H B products: 2 is a stream-K schedule over one wave of
 * one CTA per SM (each CTA an equal run of the (tile, K stage) units, the
 * tiles' partial sums added in K order; the default), 5 and 8 split K over
 * 2.5 or 4 waves.  candidate_ms: the timed candidates in that order (ms
 * per launch; 0 when not timed).  Host struct, filled before the call
 * returns. */
typedef struct {
    int density_groups;
    int tc_split_waves_x2;
    double candidate_ms[6];
} roks_tuning;
ROKS_API roks_status roks_tuning_get(const roks_ctx* ctx, roks_tuning* t);

/* Energies of the last completed density/potential evaluation.  Synchronises. */
ROKS_API roks_status roks_energies_get(roks_ctx* ctx, roks_energies* e);

/* Kernel-family timing (tracing).  While enabled, CUDA events are recorded
 * on the context's stream around each instrumented launch group (the band
 * transform stages, projector contractions, potentials, orthonormalisation,
 * subspace and rotation steps). */
typedef struct {
    char name[32];     /* family name, NUL terminated                        */
    int launches;      /* event pairs recorded since the last read          */
    double ms;         /* summed device time between the pairs (ms)         */
} roks_profile_entry;

ROKS_API roks_status roks_profile_enable(roks_ctx* ctx, int enable);

/* Synchronises the stream, writes up to cap entries to out (host), sets
 * *count to the number of entries and clears the record.  The last two
 * entries, with ms = 0, count the kernels the library launched (in any
 * context of the process) since the last read: "kernel_launches" all of
 * them, "tensor_core_launches" the tcgen05 contractions among them. */
ROKS_API roks_status roks_profile_read(roks_ctx* ctx, roks_profile_entry* out, int cap,
                                       int* count);

/* Allocation-free orthonormalisation of a band block with overlap S = 1
 * (no counterpart in the paper; it exists for callers that cannot call
 * cudaMalloc, such as code inside a framework that has reserved the GPU's
 * memory for its own allocator, or a solver loop that must not allocate once
 * running).  psi (device, npw x nbands complex, column major, ld >= npw,
 * double for ROKS_FP64 or float for ROKS_MIXED) is replaced in place by
 * psi L^{-H} with psi^H psi = L L^H (FP64 Cholesky), exactly what
 * roks_orthonormalize does on a context without projectors.  Needs no
 * context and allocates nothing: its scratch (4.2 MiB: split-K partial sums,
 * the overlap, L^{-H} and a status flag) is a fixed array in the library's
 * device memory, present on every GPU that loads the library until the
 * process exits.  Every call looks up that array's device address on the
 * current device (cudaGetSymbolAddress) before it launches anything; the
 * call synchronises its stream, so it is not for use under stream capture.
 * All calls share the array
 * and it keeps the last call's contents, so calls that overlap on the GPU
 * (different streams or threads at once) race; serialise them.
 * Limits: nbands <= 64 (ROKS_EINVAL beyond).  Synchronises the stream;
 * ROKS_ENOTPOSDEF leaves psi unchanged. */
ROKS_API roks_status roks_orthonormalize_noalloc(int precision, int npw, int nbands,
                                                 void* psi, int64_t ld, void* cuda_stream);

/* ------------------------------------------------------------------
 * Learned correction of the TPA preconditioner.  The paper preconditions
 * the out-of-subspace gradient with the TPA kinetic factor K alone (Eqs.
 * 16-18); this part multiplies K, per plane wave G and band n, by
 * m = exp(clip(s, -3, 3)), s the output of a network 3 -> 64 -> 64 -> 1
 * (tanh) of the features
 *   u0 = log(1 + (|G|^2/2) / T_n), T_n = sum (|G|^2/2)|g_nG|^2 / sum |g_nG|^2,
 *   u1 = log(1 + |g_nG| / rms_n),   rms_n = (sum |g_nG|^2 / N_pw)^(1/2),
 *   u2 = eps_n = Theta_nn / w_n     (band energy, Ha).
 * Parameters: ROKS_MLP_PARAMS floats, W1 (64 x 3, row major), b1 (64), W2
 * (64 x 64, row major), b2 (64), w3 (64), b3.  The network is trained with
 * the three calls below (all device pointers, FP32, stream-ordered, no
 * synchronisation; ROKS_EINVAL on bad sizes or null pointers). */
#define ROKS_MLP_PARAMS 4481
#define ROKS_PRECOND_TPA 0
#define ROKS_PRECOND_TPA_MLP 1

/* s[i] = network output for the feature rows feats (n x 3, row major);
 * bf16 != 0 rounds the weights to BF16 first (as the preconditioner does). */
ROKS_API roks_status roks_mlp_forward(int n, const float* feats, const float* params, int bf16, float* s,
                                      void* cuda_stream);
/* Floats of the work buffer roks_mlp_grad needs for n samples. */
ROKS_API size_t roks_mlp_grad_work(int n);
/* loss[0] = sum_i w_i (s_i - t_i)^2 / sum_i w_i and grad = d loss / d params
 * (ROKS_MLP_PARAMS floats), summed in a fixed order (deterministic). */
ROKS_API roks_status roks_mlp_grad(int n, const float* feats, const float* target, const float* weight,
                                   const float* params, float* work, float* grad, float* loss, void* cuda_stream);
/* One Adam step (step counts from 1) on params, with moment buffers m, v
 * (ROKS_MLP_PARAMS floats each, zero before the first step). */
ROKS_API roks_status roks_mlp_adam(float* params, float* m, float* v, const float* grad, int step, float lr,
                                   float beta1, float beta2, float eps, void* cuda_stream);
/* Selects the preconditioner of roks_pcg_step: ROKS_PRECOND_TPA, or
 * ROKS_PRECOND_TPA_MLP with params (device, ROKS_MLP_PARAMS floats, copied).
 * With the correction on, an accepted step that raises the energy or a CG
 * restart suspends it for three iterations (TPA is the fallback). */
ROKS_API roks_status roks_set_preconditioner(roks_ctx* ctx, int kind, const float* params);
/* out = K m grad (the preconditioner in use, before the S-projection of Eq.
 * 16) for a gradient block (device, npw x nbands, ld), and, when feats is
 * not NULL, the features of every coefficient (device, npw * nbands rows of
 * 3, band by band).  eps_n comes from Theta of the last roks_apply_h call
 * that returned a gradient. */
ROKS_API roks_status roks_precondition(roks_ctx* ctx, const void* grad, int64_t ld, void* out, float* feats);

/* Text of the last error on this context ("" if none).  Never NULL. */
ROKS_API const char* roks_last_error(const roks_ctx* ctx);

/* Frees every device and host resource of the context.  NULL is a no-op. */
ROKS_API void roks_destroy(roks_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* ROKS_H */
