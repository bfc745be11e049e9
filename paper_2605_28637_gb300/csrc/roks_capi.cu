// roks_capi.cu -- the C ABI (include/roks.h): set-up of the plane-wave model
// on one GPU and the host-side ordering of the kernels of each entry point.
// All arithmetic of the method runs in the kernels; the host only validates
// arguments, builds integer index maps and launches.
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstdlib>
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/roks.h"
#include "roks_diis.cuh"
#include "roks_exx.cuh"
#include "roks_force.cuh"
#include "roks_grid.cuh"
#include "roks_mlp.cuh"

using namespace roks;

namespace roks {
void sum_to(const double* v, int n, double* dst, double scale, cudaStream_t st);
void pcg_finish(PcgScalars* sc, cudaStream_t st);
}

#define SC_FIELD(f) int(offsetof(PcgScalars, f) / sizeof(double))

struct roks_ctx {
    std::string err;
    cudaStream_t st = nullptr;
    int prec = ROKS_FP64;
    // model
    double L = 0, omega = 0, ecut = 0, alpha = 0, e_tol = 1e-6, g_tol = 0;
    int max_iter = 0, wait_cap = 0, exx_kernel = 0, autotune = 0;
    // launch shapes (the autotuner's choices, or the defaults)
    int dens_groups = kDensityGroups, tc_waves_x2 = 2;   // 2: stream-K A^H B
    double tune_ms[6] = {0, 0, 0, 0, 0, 0};
    uint64_t seed = 0;
    long long steps = 0;   // PCG and DIIS steps since the orbitals were last set
    int N = 0, npw = 0, ld_min = 0, nmax = 0, M = 0, ncol = 0, np = 0;
    int nb = 0, nc = 0, mode = 1, nproj = 0, natoms = 0, suppress_ab = 0;
    // empty shell (Eq. 20): bands nocc .. nb - 1 carry no occupation; ne of them
    int nocc = 0, ne = 0;
    double* d_rho_e = nullptr;   // their densities, band i at (i + 1) N^3 (density storage)
    // exchange functional (roks_options.xc) and PBE exchange's work grids
    int xc = ROKS_XC_SLATER;
    GgaWork gga{};
    double* d_dk = nullptr;      // <e|F^k|e>, 3 x ne
    // Gamma point (roks_options.gamma): npw counts the half sphere, the tail
    // of the full basis from row h0; the transforms run on nbt packed bands
    // (two real orbitals each) with n_closed nct, and band split_t (-1: none)
    // holds the open pair a, b.  Without it nbt = nb, nct = nc, split_t = -1.
    int gamma = 0, npw_full = 0, h0 = 0, nbt = 0, nct = 0, split_t = -1;
    int64_t ldc_pk = 0;
    void* d_Cpk = nullptr;   // packed full-sphere coefficients (npw_full rows, ldc_pk, nbt bands)
    // the projector matrix split once into TF32 hi/lo operand blocks for the
    // tensor-core tall products P Y, where they take it
    void* d_Psplit_nn = nullptr;
    double cM = 0, cT = 0;
    PotCoef cf{};
    std::vector<int32_t> miller;
    // device: index maps and model tables
    int *d_col_start = nullptr, *d_col_kmax = nullptr, *d_plane_col0 = nullptr, *d_plane_jmax = nullptr;
    int* d_miller = nullptr;
    int* d_shell = nullptr;
    double* d_g2 = nullptr;        // |G|^2 (FP64)
    void* d_g2half = nullptr;      // |G|^2 / 2 (T)
    void* d_wk = nullptr;          // class weights (T)
    double* d_wband = nullptr;     // weight per band (FP64)
    double* d_vloc = nullptr;      // V_loc(r)
    void* d_vloc_t = nullptr;      // V_loc(r) in the element type (the FP64 path aliases d_vloc)
    void* d_P = nullptr;           // projectors npw x nproj (T complex, ld = ld_min)
    int *d_blk_off = nullptr, *d_blk_n = nullptr;
    double *d_Drow = nullptr, *d_Qrow = nullptr;
    void* d_tw = nullptr;          // twiddles (T)
    double2* d_tw64 = nullptr;     // twiddles (FP64)
    // band transforms
    void *d_Zc = nullptr, *d_Yp = nullptr;
    // grid
    double* d_rho3 = nullptr;
    double* d_rho_slot = nullptr;   // closed-shell density partials per band group
    double* d_xc3 = nullptr;
    double2* d_grid = nullptr;
    void* d_Vk = nullptr;
    double* d_part = nullptr;
    double* d_out6 = nullptr;
    double* d_E = nullptr;
    // band blocks (T complex, ld_min x nb)
    void *W_F = nullptr, *W_S = nullptr, *W_G = nullptr, *W_gI = nullptr, *W_K = nullptr, *W_u = nullptr,
         *W_v = nullptr, *W_s = nullptr, *W_sprev = nullptr, *W_Y = nullptr, *W_Y2 = nullptr;
    // band-space FP64
    double2 *d_Th = nullptr, *d_Gam = nullptr, *d_Gin = nullptr, *d_A = nullptr, *d_Aprev = nullptr,
            *d_Atot = nullptr, *d_U = nullptr, *d_O = nullptr, *d_L = nullptr, *d_LinvH = nullptr,
            *d_Msm = nullptr, *d_e1 = nullptr, *d_e2 = nullptr, *d_e3 = nullptr;
    double2 *d_B = nullptr, *d_DB = nullptr, *d_QB = nullptr, *d_B2 = nullptr;
    double2* d_gemm_work = nullptr;
    size_t gemm_work_elems = 0;
    double *d_kin_b = nullptr, *d_nl_b = nullptr, *d_colpart = nullptr, *d_colout = nullptr;
    double* d_expm_info = nullptr;
    void* d_bigwork = nullptr;      // blocked Cholesky / exponential for more than 64 bands
    int* d_flag = nullptr;
    // pinned host copy of the PCG scalars and the status flag: one round trip per step
    PcgScalars* h_sc = nullptr;
    int* h_flag = nullptr;
    PcgScalars* d_sc = nullptr;
    // exact exchange (alpha != 0)
    void *d_Phi = nullptr, *d_Xx = nullptr, *d_exbuf = nullptr, *d_vG = nullptr;
    int *d_pj = nullptr, *d_pn = nullptr;
    double *d_expart = nullptr, *d_Kmat = nullptr, *d_hf2 = nullptr, *d_exopen = nullptr;
    int npairs = 0, exx_batch = 0;
    ExxCoef exc{};
    // state: the density/potentials and d_B = P^H psi belong to the buffer
    // (address and leading dimension) a step or force call last used
    const void* cache_psi = nullptr;
    int64_t cache_ld = 0;
    const void* b_psi = nullptr;
    int64_t b_ld = 0;
    // Yp holds the y-stage planes of every band of this buffer (leading
    // dimension yp_ld): the density's x stage only reads them, so the next
    // apply of the same orbitals starts at the x stage
    const void* yp_psi = nullptr;
    int64_t yp_ld = 0;
    bool pot_valid = false;
    int n_small = 0;
    // DIIS history: ring of (Psi_j, e_j) pairs, the device state of B and
    // the window, and the host bookkeeping of the ring (pushes so far, the
    // options and buffer it belongs to).  pcg_fresh: the next PCG step starts
    // with steepest descent (a DIIS step has moved the orbitals).
    void* diis_ring = nullptr;
    int diis_slots = 0;
    DiisState* d_diis = nullptr;
    double* d_diis_part = nullptr;   // block partials of the Gram row
    DiisState* h_diis = nullptr;
    long long diis_count = 0;
    int diis_small = 0;
    roks_diis_options diis_opt{};
    const void* diis_psi = nullptr;
    int64_t diis_ld = 0;
    bool pcg_fresh = false;
    // forces (roks_forces): atom table (x, y, z, depth, width), owner atom of
    // every projector, and scratch allocated on the first call
    std::vector<double> atoms_h;
    std::vector<int> proj_atom_h;
    double* d_atoms = nullptr;
    int* d_proj_atom = nullptr;
    void *d_fdP = nullptr, *d_ftab = nullptr, *d_famp = nullptr, *d_fw2h = nullptr;
    double2 *d_fdB = nullptr, *d_fY = nullptr;
    double *d_fc = nullptr, *d_fpart = nullptr, *d_forces = nullptr;
    // learned correction of the preconditioner; once its run meets the
    // convergence criterion, TPA alone continues and must meet it again
    float* d_mlp = nullptr;
    int mlp_kind = ROKS_PRECOND_TPA;
    bool mlp_judging = false;
    // one PCG iteration as a CUDA graph, captured on a private stream the
    // second time in a row the same orbital buffer is stepped, replayed on st
    bool graphs = true;
    cudaStream_t cap_st = nullptr;
    // the rotation exponential (one SM) runs on a side stream beside the
    // band-block updates that do not need it
    cudaStream_t side_st = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
    cudaGraphExec_t pcg_exec = nullptr;
    const void* graph_psi = nullptr;
    const void* last_psi = nullptr;
    int64_t graph_ld = 0, last_ld = 0;
    long long graph_launches = 0;
    std::vector<void*> allocs;
    // kernel-family timing (roks_profile_enable / roks_profile_read)
    struct Rec {
        int fam;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<std::string> prof_names;
    std::vector<Rec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
};

namespace {

roks_status fail(roks_ctx* c, roks_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                      \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess)                                                        \
            return fail(ctx, ROKS_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

template <typename P>
cudaError_t dalloc(roks_ctx* ctx, P** p, size_t bytes) {
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes > 0 ? bytes : 16);
    if (e == cudaSuccess) {
        ctx->allocs.push_back(q);
        cudaMemsetAsync(q, 0, bytes > 0 ? bytes : 16, ctx->st);
    }
    *p = static_cast<P*>(q);
    return e;
}

cudaEvent_t prof_event(roks_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records CUDA events around the launches issued while it is alive.
struct ProfScope {
    roks_ctx* c;
    int fam = -1;
    cudaEvent_t a = nullptr;
    ProfScope(roks_ctx* ctx, const char* name) : c(ctx) {
        if (!c->prof_on) return;
        for (size_t i = 0; i < c->prof_names.size(); ++i)
            if (c->prof_names[i] == name) fam = (int)i;
        if (fam < 0) {
            fam = (int)c->prof_names.size();
            c->prof_names.push_back(name);
        }
        a = prof_event(c);
        cudaEventRecord(a, c->st);
    }
    ~ProfScope() {
        if (fam < 0) return;
        cudaEvent_t b = prof_event(c);
        cudaEventRecord(b, c->st);
        c->prof_recs.push_back({fam, a, b});
    }
};
#define PROF_CAT2(a, b) a##b
#define PROF_CAT(a, b) PROF_CAT2(a, b)
#define PROF(name) ProfScope PROF_CAT(prof_scope_, __LINE__)(ctx, name)

Sphere sphere(const roks_ctx* c) {
    Sphere s;
    s.N = c->N;
    s.nmax = c->nmax;
    s.np = c->np;
    s.ncol = c->ncol;
    s.col_start = c->d_col_start;
    s.col_kmax = c->d_col_kmax;
    s.plane_col0 = c->d_plane_col0;
    s.plane_jmax = c->d_plane_jmax;
    return s;
}

bool grid_supported(int n) {
    for (int g : kGrids)
        if (g == n) return true;
    return false;
}

int isqrt_floor(long v) {
    long r = (long)std::sqrt((double)v);
    while (r * r > v) --r;
    while ((r + 1) * (r + 1) <= v) ++r;
    return (int)r;
}

// ------------------------------------------------------------------ typed implementation
template <typename T>
struct Impl {
    using V = c2<T>;
    static V* cv(void* p) { return static_cast<V*>(p); }
    static const V* ccv(const void* p) { return static_cast<const V*>(p); }

    // C = A^H B over the basis rows; at the Gamma point its real part (the
    // full-sphere product of real orbitals in the stored half-sphere form)
    static void cn(roks_ctx* ctx, int M, int N, int K, const V* A, int64_t lda, const V* B, int64_t ldb, double2* C,
                   int ldc, cudaStream_t st) {
        gemm_cn<T>(M, N, K, A, lda, B, ldb, C, ldc, ctx->d_gemm_work, ctx->gemm_work_elems, st);
        if (ctx->gamma) gamma_real_part(M, N, C, ldc, st);
    }

    // Yp <- y-stage planes of the transform bands of psi (at the Gamma point
    // two real orbitals per band, expanded to the full sphere first)
    static void inv_planes(roks_ctx* ctx, const void* psi, int64_t ld) {
        const Sphere s = sphere(ctx);
        cudaStream_t st = ctx->st;
        const V* src = ccv(psi);
        int64_t lds = ld;
        if (ctx->gamma) {
            PROF("fft_z_inv");
            gamma_expand<T>(ctx->npw, ctx->h0, ctx->nb, src, ld, cv(ctx->d_Cpk), ctx->ldc_pk, st);
            src = ccv(ctx->d_Cpk);
            lds = ctx->ldc_pk;
        }
        { PROF("fft_z_inv"); band_z_inv<T>(s, ccv(ctx->d_tw), src, lds, 0, ctx->nbt, cv(ctx->d_Zc), st); }
        { PROF("fft_y_inv"); band_y_inv<T>(s, ccv(ctx->d_tw), cv(ctx->d_Zc), cv(ctx->d_Yp), ctx->nbt, st); }
        ctx->yp_psi = psi;
        ctx->yp_ld = ld;
    }

    // Exact exchange of the bands whose plane data sit in Yp: real-space
    // orbitals, pair integrals, energies and (want_field) the exchange fields.
    static void exchange(roks_ctx* ctx, bool want_field) {
        const Sphere s = sphere(ctx);
        cudaStream_t st = ctx->st;
        band_x_inv_full<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp), cv(ctx->d_Phi), 0, ctx->nb, T(1.0 / std::sqrt(ctx->omega)),
                           st);
        ExxArgs<T> a;
        a.N = ctx->N;
        a.nb = ctx->nb;
        a.npairs = ctx->npairs;
        a.batch = ctx->exx_batch;
        a.L = ctx->L;
        a.tw = ccv(ctx->d_tw);
        a.vG = static_cast<const T*>(ctx->d_vG);
        a.Phi = ccv(ctx->d_Phi);
        a.X = cv(ctx->d_Xx);
        a.buf = cv(ctx->d_exbuf);
        a.pj = ctx->d_pj;
        a.pn = ctx->d_pn;
        a.part = ctx->d_expart;
        a.Kmat = ctx->d_Kmat;
        a.hf2 = ctx->d_hf2;
        a.open_diag = ctx->d_exopen;
        a.cf = ctx->exc;
        exx_pairs<T>(a, want_field, st);
    }

    // rho3, kin_b, nl_b of psi.  Bgiven: projector coefficients of psi if known.
    static roks_status density(roks_ctx* ctx, const void* psi, int64_t ld, const double2* Bgiven) {
        const Sphere s = sphere(ctx);
        cudaStream_t st = ctx->st;
        const V* p = ccv(psi);
        inv_planes(ctx, psi, ld);
        if (ctx->alpha != 0.0) {
            PROF("exchange");
            exchange(ctx, false);
        }
        CK(cudaMemsetAsync(ctx->d_rho3, 0, sizeof(double) * 3 * (size_t)ctx->N * ctx->N * ctx->N, st));
        {
            PROF("fft_x_density");
            if (ctx->split_t < 0) {
                // the occupied bands (the empty ones carry no density)
                band_x_density<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp), ctx->d_rho3, ctx->d_rho_slot, ctx->dens_groups,
                                  0, ctx->nbt - ctx->ne, ctx->nct, 1.0 / ctx->omega, st);
                if (ctx->ne > 0) {
                    // each empty band's own density, for its <e|V^k|e> (the
                    // kernel indexes the planes from the launch's first band
                    // and adds class 1 of the rho3 it is given)
                    const int64_t N3 = (int64_t)ctx->N * ctx->N * ctx->N;
                    CK(cudaMemsetAsync(ctx->d_rho_e + N3, 0, sizeof(double) * ctx->ne * N3, st));
                    for (int i = 0; i < ctx->ne; ++i) {
                        const int e = ctx->nocc + i;
                        const V* yo = ccv(ctx->d_Yp) + (int64_t)e * ctx->np * ctx->N * ctx->N;
                        band_x_density<T>(s, ccv(ctx->d_tw), yo, ctx->d_rho_e + i * N3, nullptr, 1, e, 1, ctx->nc,
                                          1.0 / ctx->omega, st, 0, 1);
                    }
                }
            } else {
                // Gamma point: the closed pairs, then the packed open pair's
                // real part (a) and imaginary part (b) into their own classes
                if (ctx->nct > 0)
                    band_x_density<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp), ctx->d_rho3, ctx->d_rho_slot,
                                      ctx->dens_groups, 0, ctx->nct, ctx->nct, 1.0 / ctx->omega, st);
                // (the kernel indexes the plane buffer from the launch's first band)
                const V* yo = ccv(ctx->d_Yp) + (int64_t)ctx->split_t * ctx->np * ctx->N * ctx->N;
                for (int part = 1; part <= 2; ++part)
                    band_x_density<T>(s, ccv(ctx->d_tw), yo, ctx->d_rho3, nullptr, 1, ctx->split_t, 1, ctx->nct,
                                      1.0 / ctx->omega, st, part, part);
            }
        }
        column_sums<T>(0, ctx->npw, ctx->nb, p, ld, nullptr, 0, static_cast<const T*>(ctx->d_g2half), ctx->d_colpart, ctx->d_kin_b, st);
        const double2* B = Bgiven;
        if (!B) {
            PROF("proj_PhPsi");
            cn(ctx, ctx->nproj, ctx->nb, ctx->npw, ccv(ctx->d_P), ctx->ld_min, p, ld, ctx->d_B, ctx->nproj, st);
            B = ctx->d_B;
        }
        if (B == ctx->d_B) {
            ctx->b_psi = psi;
            ctx->b_ld = ld;
        }
        apply_DQ(ctx->nproj, ctx->nb, B, ctx->d_blk_off, ctx->d_blk_n, ctx->d_Drow, ctx->d_Qrow, nullptr,
                 ctx->d_DB, nullptr, st);
        band_quadratic(ctx->nproj, ctx->nb, B, ctx->d_DB, ctx->d_nl_b, st);
        CK(cudaGetLastError());
        return ROKS_OK;
    }

    // energies_only: the energy of the density (out6[0..3], d_E) without the
    // class potentials, for points whose potentials no apply will use
    static roks_status potential(roks_ctx* ctx, bool energies_only = false) {
        cudaStream_t st = ctx->st;
        PROF("potential");
        potentials<T>(ctx->N, ctx->L, ctx->d_rho3, static_cast<const T*>(ctx->d_vloc_t), ctx->cf,
                      reinterpret_cast<V*>(ctx->d_grid), reinterpret_cast<T*>(ctx->d_xc3), ccv(ctx->d_tw),
                      static_cast<T*>(ctx->d_Vk), nullptr, ctx->d_part, ctx->d_out6, st, energies_only,
                      ctx->xc == ROKS_XC_PBE_X ? &ctx->gga : nullptr);
        energy_combine(ctx->d_kin_b, ctx->d_nl_b, ctx->nocc, ctx->d_wband, ctx->d_out6, ctx->cM, ctx->cT,
                       ctx->alpha, ctx->alpha != 0.0 ? ctx->d_hf2 : nullptr, ctx->d_E, st);
        CK(cudaGetLastError());
        return ROKS_OK;
    }

    // F = F^{k(n)}|n>, S = S|n> (S optional), with the current potentials.
    // reuse_B: d_B already holds P^H psi (the PCG chain keeps it from the
    // orthonormalisation of the accepted point)
    // Yp <- y-stage planes of psi
    static void planes(roks_ctx* ctx, const void* psi, int64_t ld) { inv_planes(ctx, psi, ld); }

    // planes_ready: Yp already holds the planes of psi (yp_psi), so the
    // transform starts at the x stage
    static roks_status apply(roks_ctx* ctx, const void* psi, int64_t ld, void* F, int64_t ldf, void* S,
                             int64_t lds, bool reuse_B = false, bool planes_ready = false) {
        const Sphere s = sphere(ctx);
        cudaStream_t st = ctx->st;
        const V* p = ccv(psi);
        const int N = ctx->N;
        if (!planes_ready) planes(ctx, psi, ld);
        if (ctx->alpha != 0.0) {
            PROF("exchange");
            exchange(ctx, true);
        }
        {
            PROF("fft_x_apply");
            const int nx = ctx->nbt - ctx->ne;
            band_x_apply<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp), static_cast<const T*>(ctx->d_Vk),
                            ctx->alpha != 0.0 ? ccv(ctx->d_Xx) : nullptr, 0, nx, ctx->nct, ctx->split_t,
                            T(1.0 / (double(N) * N * N)), st);
            // empty bands: F^c (a closed count past the last band gives class 0)
            if (ctx->ne > 0)
                band_x_apply<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp) + (int64_t)nx * ctx->np * N * N,
                                static_cast<const T*>(ctx->d_Vk), nullptr, nx, ctx->ne, ctx->nb, -1,
                                T(1.0 / (double(N) * N * N)), st);
        }
        ctx->yp_psi = nullptr;   // the x stage works in place
        { PROF("fft_y_fwd"); band_y_fwd<T>(s, ccv(ctx->d_tw), cv(ctx->d_Yp), cv(ctx->d_Zc), ctx->nbt, st); }
        {
            PROF("fft_z_fwd");
            if (ctx->gamma) {
                // packed transforms on the full sphere, then each real
                // orbital's half with its kinetic term
                band_z_fwd<T>(s, ccv(ctx->d_tw), cv(ctx->d_Zc), cv(ctx->d_Cpk), ctx->ldc_pk, nullptr, 0,
                              static_cast<const T*>(ctx->d_g2half), static_cast<const T*>(ctx->d_wk), 0, ctx->nbt,
                              ctx->nct, st);
                gamma_unpack<T>(ctx->npw, ctx->h0, ctx->nb, ctx->nc, ccv(ctx->d_Cpk), ctx->ldc_pk, p, ld,
                                static_cast<const T*>(ctx->d_g2half), static_cast<const T*>(ctx->d_wk), cv(F), ldf,
                                st);
            } else {
                band_z_fwd<T>(s, ccv(ctx->d_tw), cv(ctx->d_Zc), cv(F), ldf, p, ld,
                              static_cast<const T*>(ctx->d_g2half), static_cast<const T*>(ctx->d_wk), 0, ctx->nocc,
                              ctx->nc, st);
                if (ctx->ne > 0)
                    band_z_fwd<T>(s, ccv(ctx->d_tw), cv(ctx->d_Zc) + (int64_t)ctx->nocc * ctx->ncol * N, cv(F), ldf,
                                  p, ld, static_cast<const T*>(ctx->d_g2half), static_cast<const T*>(ctx->d_wk),
                                  ctx->nocc, ctx->ne, ctx->nb, st);
            }
        }
        if (ctx->nproj > 0) {
            if (!reuse_B) {
                PROF("proj_PhPsi");
                cn(ctx, ctx->nproj, ctx->nb, ctx->npw, ccv(ctx->d_P), ctx->ld_min, p, ld, ctx->d_B, ctx->nproj, st);
                ctx->b_psi = psi;
                ctx->b_ld = ld;
            }
            apply_DQ(ctx->nproj, ctx->nb, ctx->d_B, ctx->d_blk_off, ctx->d_blk_n, ctx->d_Drow, ctx->d_Qrow,
                     ctx->d_wband, ctx->d_DB, ctx->d_QB, st);
            PROF("proj_PX");
            gemm_nn<T>(ctx->npw, ctx->nb, ctx->nproj, ccv(ctx->d_P), ctx->ld_min, ctx->d_DB, ctx->nproj, cv(F), ldf,
                       1.0, 1.0, ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
        }
        if (S) {
            CK(cudaMemcpy2DAsync(S, lds * sizeof(V), psi, ld * sizeof(V), ctx->npw * sizeof(V), ctx->nb,
                                 cudaMemcpyDeviceToDevice, st));
            if (ctx->nproj > 0) {
                PROF("proj_PX");
                gemm_nn<T>(ctx->npw, ctx->nb, ctx->nproj, ccv(ctx->d_P), ctx->ld_min, ctx->d_QB, ctx->nproj, cv(S),
                           lds, 1.0, 1.0, ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
            }
        }
        CK(cudaGetLastError());
        return ROKS_OK;
    }

    // out = in L^{-H} with in^H S in = L L^H; Bout = P^H out.
    static roks_status orth(roks_ctx* ctx, const void* in, int64_t ldi, void* out, int64_t ldo, double2* Bout) {
        cudaStream_t st = ctx->st;
        const int nb = ctx->nb;
        {
            PROF("orth_overlap");
            cn(ctx, nb, nb, ctx->npw, ccv(in), ldi, ccv(in), ldi, ctx->d_O, nb, st);
        }
        if (ctx->nproj > 0) {
            {
                PROF("proj_PhPsi");
                cn(ctx, ctx->nproj, nb, ctx->npw, ccv(ctx->d_P), ctx->ld_min, ccv(in), ldi, ctx->d_B2, ctx->nproj, st);
            }
            PROF("orth_small");
            apply_DQ(ctx->nproj, nb, ctx->d_B2, ctx->d_blk_off, ctx->d_blk_n, ctx->d_Drow, ctx->d_Qrow, nullptr,
                     nullptr, ctx->d_QB, st);
            if (ctx->prec == ROKS_MIXED)
                small_gemm_f32(nb, nb, ctx->nproj, ctx->d_B2, ctx->nproj, true, ctx->d_QB, ctx->nproj, false, ctx->d_O,
                               nb, 1.0, 1.0, st, ctx->d_gemm_work, ctx->gemm_work_elems * sizeof(double2));
            else
                small_gemm(nb, nb, ctx->nproj, ctx->d_B2, ctx->nproj, true, ctx->d_QB, ctx->nproj, false, ctx->d_O, nb,
                           1.0, 1.0, st);
        }
        // mixed path, small n: L^{-H} = I + Xi^H in deviation form (FP32 errors
        // relative to |O - I|); out = in + in Xi^H keeps the identity exact
        const bool dev = ctx->prec == ROKS_MIXED && cholesky_small_supported(nb);
        {
            PROF("orth_cholesky");
            if (dev) {
                cholesky_dev_f32(nb, ctx->d_O, ctx->d_LinvH, ctx->d_flag, st);
            } else {
                hermitize(nb, ctx->d_O, st);
                if (nb > 64)
                    cholesky_inverse_big(nb, ctx->d_O, ctx->d_bigwork, ctx->prec == ROKS_FP64, ctx->d_LinvH,
                                         ctx->d_flag, st);
                else
                    cholesky_inverse(nb, ctx->d_O, ctx->d_L, ctx->d_LinvH, ctx->d_flag, st);
            }
        }
        {
            PROF("orth_apply");
            if (dev)
                gemm_nn_io<T>(ctx->npw, nb, nb, ccv(in), ldi, ctx->d_LinvH, nb, ccv(in), ldi, cv(out), ldo, 1.0, 1.0,
                              ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
            else
                gemm_nn<T>(ctx->npw, nb, nb, ccv(in), ldi, ctx->d_LinvH, nb, cv(out), ldo, 1.0, 0.0,
                           ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
        }
        if (Bout && ctx->nproj > 0) {
            PROF("orth_small");
            if (dev)
                CK(cudaMemcpyAsync(Bout, ctx->d_B2, sizeof(double2) * ctx->nproj * nb, cudaMemcpyDeviceToDevice, st));
            if (ctx->prec == ROKS_MIXED)
                small_gemm_f32(ctx->nproj, nb, nb, ctx->d_B2, ctx->nproj, false, ctx->d_LinvH, nb, false, Bout,
                               ctx->nproj, 1.0, dev ? 1.0 : 0.0, st, ctx->d_gemm_work,
                               ctx->gemm_work_elems * sizeof(double2));
            else
                small_gemm(ctx->nproj, nb, nb, ctx->d_B2, ctx->nproj, false, ctx->d_LinvH, nb, false, Bout, ctx->nproj,
                           1.0, dev ? 1.0 : 0.0, st);
        }
        CK(cudaGetLastError());
        return ROKS_OK;
    }

    static roks_status check_flag(roks_ctx* ctx) {
        int flag = 0;
        CK(cudaMemcpyAsync(&flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        const bool tc_out = tcg_timeout_take() != 0;
        const bool st_out = stream_timeout_take() != 0;
        if (flag || tc_out || st_out) {
            CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), ctx->st));
            CK(cudaStreamSynchronize(ctx->st));
        }
        if (tc_out) return fail(ctx, ROKS_ETIMEOUT, "a tensor-core completion wait ran out (bounded mbarrier wait)");
        if (st_out)
            return fail(ctx, ROKS_ETIMEOUT, "a bulk-copy wait of a streamed contraction ran out (bounded mbarrier wait)");
        if (flag)
            return fail(ctx, ROKS_ENOTPOSDEF,
                        "overlap matrix not positive definite at band " + std::to_string(flag - 1));
        return ROKS_OK;
    }

    // s-projection: out = x - Psi ((S Psi)^H x)
    static void project(roks_ctx* ctx, const void* psi, int64_t ld, const void* x, void* out) {
        cudaStream_t st = ctx->st;
        const int nb = ctx->nb;
        const int64_t l = ctx->ld_min;
        PROF("subspace_project");
        cn(ctx, nb, nb, ctx->npw, ccv(ctx->W_S), l, ccv(x), l, ctx->d_Msm, nb, st);
        gemm_nn_io<T>(ctx->npw, nb, nb, ccv(psi), ld, ctx->d_Msm, nb, ccv(x), l, cv(out), l, -1.0, 1.0,
                      ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
    }

    // dst field = sum_n Re <x_n|y_n>
    static void dot_to(roks_ctx* ctx, const void* x, const void* y, int field, int ncols = -1) {
        const int64_t l = ctx->ld_min;
        column_total<T>(2, ctx->npw, ncols < 0 ? ctx->nb : ncols, ccv(x), l, ccv(y), l, static_cast<const T*>(ctx->d_g2half),
                        ctx->d_colpart, reinterpret_cast<double*>(ctx->d_sc) + field, 1.0, ctx->st);
    }

    // U = exp(step A_tot) on the side stream, after everything already
    // enqueued on st; join_U makes st wait for it.
    static roks_status fork_U(roks_ctx* ctx, int step_field) {
        const int nb = ctx->nb;
        double* scd = reinterpret_cast<double*>(ctx->d_sc);
        if (!ctx->side_st) {
            CK(cudaStreamCreateWithFlags(&ctx->side_st, cudaStreamNonBlocking));
            CK(cudaEventCreateWithFlags(&ctx->fork_ev, cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&ctx->join_ev, cudaEventDisableTiming));
        }
        CK(cudaEventRecord(ctx->fork_ev, ctx->st));
        CK(cudaStreamWaitEvent(ctx->side_st, ctx->fork_ev, 0));
        // profiled (eager) steps time the exponential as a family of its own
        // on the main stream; otherwise it runs beside the band-block updates
        cudaStream_t ss = ctx->prof_on ? ctx->st : ctx->side_st;
        PROF("expm");
        if (nb > 64) {
            expm_big(nb, ctx->d_Atot, scd + step_field, ctx->d_U, ctx->d_bigwork, ctx->d_expm_info,
                     ctx->prec == ROKS_FP64, ss);
        } else {
            const bool small32 =
                (ctx->prec == ROKS_MIXED) && expm_small_f32(nb, ctx->d_Atot, scd + step_field, ctx->d_U, ss);
            if (!small32)
                expm_scaled(nb, ctx->d_Atot, scd + step_field, ctx->d_U, ctx->d_e1, ctx->d_e2, ctx->d_e3,
                            ctx->d_expm_info, ss);
        }
        CK(cudaGetLastError());
        CK(cudaEventRecord(ctx->join_ev, ss));
        return ROKS_OK;
    }
    static roks_status join_U(roks_ctx* ctx) {
        CK(cudaStreamWaitEvent(ctx->st, ctx->join_ev, 0));
        return ROKS_OK;
    }

    // out = orth((psi + step s) exp(step Atot)), U forked before (fork_U);
    // energies of out in d_E (and its potentials unless energies_only).
    static roks_status move(roks_ctx* ctx, const void* psi, int64_t ld, int step_field, void* out, int64_t ldo,
                            bool energies_only = false) {
        cudaStream_t st = ctx->st;
        const int nb = ctx->nb;
        const int64_t l = ctx->ld_min;
        double* scd = reinterpret_cast<double*>(ctx->d_sc);
        {
            PROF("rotate");
            // the trial point (energies only) moves the occupied bands alone:
            // the empty bands' directions do not change the energy to first
            // order, and their second order would distort the parabola
            const int nmv = (energies_only && ctx->ne > 0) ? ctx->nocc : nb;
            axpy<T>(ctx->npw, nmv, ccv(psi), ld, ccv(ctx->W_s), l, scd + step_field, 1.0, cv(ctx->W_Y), l, st);
            if (nmv < nb)
                CK(cudaMemcpy2DAsync(static_cast<V*>(ctx->W_Y) + (int64_t)nmv * l, l * sizeof(V),
                                     static_cast<const V*>(psi) + (int64_t)nmv * ld, ld * sizeof(V),
                                     ctx->npw * sizeof(V), nb - nmv, cudaMemcpyDeviceToDevice, st));
            roks_status r = join_U(ctx);
            if (r != ROKS_OK) return r;
            gemm_nn<T>(ctx->npw, nb, nb, ccv(ctx->W_Y), l, ctx->d_U, nb, cv(ctx->W_Y2), l, 1.0, 0.0, ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
        }
        roks_status r = orth(ctx, ctx->W_Y2, l, out, ldo, ctx->d_B);
        if (r != ROKS_OK) return r;
        r = density(ctx, out, ldo, ctx->nproj > 0 ? ctx->d_B : nullptr);
        if (r != ROKS_OK) return r;
        return potential(ctx, energies_only);
    }

    // The device work of one PCG iteration from a valid potential: no host
    // synchronisation and no host-side state change, so it can be captured.
    static roks_status pcg_enqueue(roks_ctx* ctx, void* psi, int64_t ld) {
        cudaStream_t st = ctx->st;
        const int nb = ctx->nb, npw = ctx->npw;
        const int64_t l = ctx->ld_min;
        roks_status r;
        pcg_take_energy(ctx->d_E, ctx->d_sc, SC_FIELD(E0), st);
        // F Psi, S Psi, theta, d
        r = apply(ctx, psi, ld, ctx->W_F, l, ctx->W_S, l, true, true);
        if (r != ROKS_OK) return r;
        {
            PROF("subspace_theta");
            cn(ctx, nb, nb, npw, ccv(psi), ld, ccv(ctx->W_F), l, ctx->d_Th, nb, st);
        }
        const int ia = (ctx->mode == ROKS_MODE_SINGLET) ? ctx->nc : -1;
        const int ib = (ctx->mode == ROKS_MODE_SINGLET) ? ctx->nc + 1 : -1;
        if (ctx->ne > 0)
            empty_band_diagonal<T>((int64_t)ctx->N * ctx->N * ctx->N, ctx->ne, ctx->nocc, ctx->d_rho_e,
                                   static_cast<const T*>(ctx->d_Vk), ctx->omega / (double(ctx->N) * ctx->N * ctx->N),
                                   ctx->d_kin_b, ctx->d_nl_b, ctx->cf.w[0], ctx->cf.w[1], ctx->cf.w[2],
                                   ctx->d_dk + 3 * ctx->ne, ctx->d_dk, st);
        pcg_rotation(nb, ctx->nc, ctx->d_Th, ctx->d_kin_b, ctx->d_nl_b, ctx->d_out6 + 4,
                     ctx->alpha != 0.0 ? ctx->d_exopen : nullptr, ctx->cf.w[0], ctx->d_shell,
                     ctx->suppress_ab && ctx->mode == ROKS_MODE_SINGLET, ia, ib, ctx->d_Gam, ctx->d_Gin, ctx->d_A,
                     ctx->d_sc, st, ctx->nocc, ctx->d_dk);
        // gI = F - S theta ; G = F - S Gam, with F^e = 0 in the empty columns
        // (their g_I is the F^c residual, the empty bands' own direction)
        {
        PROF("gradient_precond");
        gemm_nn_io<T>(npw, nb, nb, ccv(ctx->W_S), l, ctx->d_Th, nb, ccv(ctx->W_F), l, cv(ctx->W_gI), l, -1.0, 1.0,
                      ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
        if (ctx->ne > 0) CK(cudaMemsetAsync(static_cast<V*>(ctx->W_F) + (int64_t)ctx->nocc * l, 0,
                                            sizeof(V) * l * ctx->ne, st));
        gemm_nn_io<T>(npw, nb, nb, ccv(ctx->W_S), l, ctx->d_Gam, nb, ccv(ctx->W_F), l, cv(ctx->W_G), l, -1.0, 1.0,
                      ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
        column_total<T>(3, npw, nb, ccv(ctx->W_G), l, nullptr, 0, static_cast<const T*>(ctx->d_g2half), ctx->d_colpart,
                        reinterpret_cast<double*>(ctx->d_sc) + SC_FIELD(gnorm2), 1.0, st);
        // p_I = K g_I - Psi (S Psi)^H K g_I
        column_sums<T>(1, npw, nb, ccv(ctx->W_gI), l, nullptr, 0, static_cast<const T*>(ctx->d_g2half), ctx->d_colpart, ctx->d_colout, st);
        if (ctx->mlp_kind == ROKS_PRECOND_TPA_MLP)
            precondition_mlp<T>(npw, nb, ccv(ctx->W_gI), l, static_cast<const T*>(ctx->d_g2half), ctx->d_colout,
                                ctx->d_Th, ctx->d_wband, ctx->d_mlp, ctx->d_sc, cv(ctx->W_K), l, st);
        else
            precondition<T>(npw, nb, ccv(ctx->W_gI), l, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, cv(ctx->W_K), l, st);
        }
        project(ctx, psi, ld, ctx->W_K, ctx->W_K);
        // the Fletcher-Reeves ratio of the energy's gradient: occupied bands
        dot_to(ctx, ctx->W_K, ctx->W_gI, SC_FIELD(pgI), ctx->nocc);
        pcg_rot_dots(nb, ctx->d_A, ctx->d_Aprev, ctx->d_Gin, ctx->d_colpart, ctx->d_sc, st);
        // u = p_I (projected above; the S-projector is idempotent on
        // S-orthonormal orbitals, so projecting again changes nothing),
        // v = proj(s_prev) (s_prev was projected against the previous orbitals)
        project(ctx, psi, ld, ctx->W_sprev, ctx->W_v);
        dot_to(ctx, ctx->W_K, ctx->W_G, SC_FIELD(a1));
        dot_to(ctx, ctx->W_v, ctx->W_G, SC_FIELD(a2));
        pcg_direction(ctx->d_sc, st);
        // A_tot = rot (A + beta A_prev) and its exponential beside s = u + beta v
        pcg_total_rotation(nb, ctx->d_A, ctx->d_Aprev, ctx->d_sc, ctx->d_Atot, st);
        r = fork_U(ctx, SC_FIELD(dt));
        if (r != ROKS_OK) return r;
        axpy<T>(npw, nb, ccv(ctx->W_K), l, ccv(ctx->W_v), l, reinterpret_cast<double*>(ctx->d_sc) + SC_FIELD(beta),
                1.0, cv(ctx->W_s), l, st);
        // trial point: its energy alone (the accepted point's potentials replace it)
        r = move(ctx, psi, ld, SC_FIELD(dt), ctx->W_F, l, true);
        if (r != ROKS_OK) return r;
        pcg_take_energy(ctx->d_E, ctx->d_sc, SC_FIELD(Et), st);
        pcg_line_search(ctx->d_sc, st);
        // accepted point (written to W_F, then copied over psi)
        r = fork_U(ctx, SC_FIELD(step));
        if (r != ROKS_OK) return r;
        r = move(ctx, psi, ld, SC_FIELD(step), ctx->W_F, l);
        if (r != ROKS_OK) return r;
        pcg_take_energy(ctx->d_E, ctx->d_sc, SC_FIELD(Enew), st);
        CK(cudaMemcpy2DAsync(psi, ld * sizeof(V), ctx->W_F, l * sizeof(V), npw * sizeof(V), nb,
                             cudaMemcpyDeviceToDevice, st));
        // history
        CK(cudaMemcpyAsync(ctx->W_sprev, ctx->W_s, sizeof(V) * l * nb, cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->d_Aprev, ctx->d_A, sizeof(double2) * nb * nb, cudaMemcpyDeviceToDevice, st));
        pcg_finish(ctx->d_sc, st);
        // the accepted point's density left its planes in Yp; psi now holds it
        ctx->yp_psi = psi;
        ctx->yp_ld = ld;
        CK(cudaGetLastError());
        return ROKS_OK;
    }

    // Replays the captured iteration, capturing it first when the buffer is
    // stepped for the second time in a row (the first, eager call has set
    // up every kernel attribute).  Profiling runs eagerly (events per
    // kernel family); so does a context whose capture failed.
    static roks_status pcg_run(roks_ctx* ctx, void* psi, int64_t ld) {
        const bool repeat = ctx->last_psi == psi && ctx->last_ld == ld;
        ctx->last_psi = psi;
        ctx->last_ld = ld;
        if (!ctx->graphs || ctx->prof_on || !repeat) return pcg_enqueue(ctx, psi, ld);
        if (!(ctx->pcg_exec && ctx->graph_psi == psi && ctx->graph_ld == ld)) {
            if (ctx->pcg_exec) {
                cudaGraphExecDestroy(ctx->pcg_exec);
                ctx->pcg_exec = nullptr;
            }
            if (!ctx->cap_st) CK(cudaStreamCreateWithFlags(&ctx->cap_st, cudaStreamNonBlocking));
            const long long n0 = launches_now();
            CK(cudaStreamBeginCapture(ctx->cap_st, cudaStreamCaptureModeThreadLocal));
            cudaStream_t user = ctx->st;
            ctx->st = ctx->cap_st;
            const roks_status r = pcg_enqueue(ctx, psi, ld);
            ctx->st = user;
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(ctx->cap_st, &g);
            const long long n = launches_now() - n0;
            count_launches(-n);   // recorded, not launched
            if (r != ROKS_OK) {
                if (g) cudaGraphDestroy(g);
                return r;
            }
            if (e == cudaSuccess && g) e = cudaGraphInstantiate(&ctx->pcg_exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess || !ctx->pcg_exec) {
                // capture refused: keep launching the same kernels one by one
                cudaGetLastError();
                ctx->pcg_exec = nullptr;
                ctx->graphs = false;
                return pcg_enqueue(ctx, psi, ld);
            }
            ctx->graph_psi = psi;
            ctx->graph_ld = ld;
            ctx->graph_launches = n;
        }
        CK(cudaGraphLaunch(ctx->pcg_exec, ctx->st));
        count_launches(ctx->graph_launches);
        return ROKS_OK;
    }

    static roks_status pcg_step(roks_ctx* ctx, void* psi, int64_t ld, roks_step_info* info) {
        cudaStream_t st = ctx->st;
        roks_status r;
        if (!(ctx->pot_valid && ctx->cache_psi == psi && ctx->cache_ld == ld)) {
            r = density(ctx, psi, ld, nullptr);
            if (r != ROKS_OK) return r;
            r = potential(ctx);
            if (r != ROKS_OK) return r;
        }
        if (ctx->nproj > 0 && !(ctx->b_psi == psi && ctx->b_ld == ld)) {
            // the iteration reuses P^H psi from d_B: form it if another call replaced it
            PROF("proj_PhPsi");
            cn(ctx, ctx->nproj, ctx->nb, ctx->npw, ccv(ctx->d_P), ctx->ld_min, ccv(psi), ld, ctx->d_B, ctx->nproj, st);
            ctx->b_psi = psi;
            ctx->b_ld = ld;
        }
        // the iteration's apply starts from the planes in Yp (a captured
        // iteration leaves those of its accepted point there)
        if (!(ctx->yp_psi == psi && ctx->yp_ld == ld)) planes(ctx, psi, ld);
        r = pcg_run(ctx, psi, ld);
        if (r != ROKS_OK) return r;
        ctx->b_psi = psi;   // d_B: projector coefficients of the accepted point, now in psi
        ctx->b_ld = ld;
        ctx->yp_psi = psi;
        ctx->yp_ld = ld;
        // scalars and status flag in one round trip (pinned host copies)
        CK(cudaMemcpyAsync(ctx->h_sc, ctx->d_sc, sizeof(PcgScalars), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        int* sflag = stream_timeout_flag();
        ctx->h_flag[1] = 0;
        if (sflag) CK(cudaMemcpyAsync(ctx->h_flag + 1, sflag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        // a wait that ran out comes first (the step's numbers are then
        // meaningless), then non-finite numbers, then a failed Cholesky
        const bool tc_out = tcg_timeout_take() != 0;
        const bool st_out = ctx->h_flag[1] != 0;
        if (st_out) stream_timeout_take();
        const PcgScalars h = *ctx->h_sc;
        const bool finite = std::isfinite(h.E0) && std::isfinite(h.Enew) && std::isfinite(h.gnorm2);
        if (tc_out || st_out || !finite || *ctx->h_flag) {
            const int band = *ctx->h_flag - 1;
            CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
            CK(cudaStreamSynchronize(st));
            ctx->pot_valid = false;
            if (tc_out)
                return fail(ctx, ROKS_ETIMEOUT, "a tensor-core completion wait ran out (bounded mbarrier wait)");
            if (st_out)
                return fail(ctx, ROKS_ETIMEOUT,
                            "a bulk-copy wait of a streamed contraction ran out (bounded mbarrier wait)");
            if (info) {
                info->E = h.E0;
                info->E_new = h.Enew;
                info->grad_norm = std::sqrt(h.gnorm2);
            }
            if (!finite) return fail(ctx, ROKS_EDIVERGED, "non-finite energy or gradient");
            return fail(ctx, ROKS_ENOTPOSDEF, "overlap matrix not positive definite at band " + std::to_string(band));
        }
        ctx->cache_psi = psi;
        ctx->cache_ld = ld;
        ctx->pot_valid = true;
        if (info) {
            info->E = h.E0;
            info->E_new = h.Enew;
            info->step = h.step;
            info->grad_norm = std::sqrt(h.gnorm2);
            info->coupling_re = h.coup_re;
            info->coupling_im = h.coup_im;
            info->beta = h.beta;
            info->dE0 = h.dE0;
            info->restarted = h.restarted != 0.0;
        }
        return ROKS_OK;
    }

    // Forces (roks_forces): potentials, F Psi and gamma of psi, the
    // projector derivatives dB_nu = (dP_nu)^H Psi, the projector terms per
    // projector and the local term per atom (k_force.cu), summed per atom.
    static roks_status forces(roks_ctx* ctx, const void* psi, int64_t ld, double* out_host) {
        cudaStream_t st = ctx->st;
        // the occupied bands (the first nocc) alone carry the energy
        const int nb = ctx->nocc, npw = ctx->npw, np_ = ctx->nproj;
        const int64_t l = ctx->ld_min;
        roks_status r = ROKS_OK;
        // the density and potentials of psi are current after a PCG or DIIS
        // step on it (or a previous force call); otherwise form them
        if (!(ctx->pot_valid && ctx->cache_psi == psi && ctx->cache_ld == ld)) {
            r = density(ctx, psi, ld, nullptr);
            if (r != ROKS_OK) return r;
            r = potential(ctx);
            if (r != ROKS_OK) return r;
            ctx->cache_psi = psi;
            ctx->cache_ld = ld;
            ctx->pot_valid = true;
        }
        r = apply(ctx, psi, ld, ctx->W_F, l, nullptr, 0, np_ > 0 && ctx->b_psi == psi && ctx->b_ld == ld,
                  ctx->yp_psi == psi && ctx->yp_ld == ld);
        if (r != ROKS_OK) return r;
        const double b = 2.0 * M_PI / ctx->L;
        {
            PROF("force");
            cn(ctx, nb, nb, npw, ccv(psi), ld, ccv(ctx->W_F), l, ctx->d_Th, nb, st);
            diis_multipliers(nb, ctx->d_Th, -1, -1, 0.5, 0.5, ctx->d_Gam, st);   // Gam = (theta + theta^H)/2
            if (np_ > 0) {
                for (int nu = 0; nu < 3; ++nu) {
                    force_dP<T>(npw, np_, ccv(ctx->d_P), l, ctx->d_miller, b, nu, cv(ctx->d_fdP), st);
                    cn(ctx, np_, nb, npw, ccv(ctx->d_fdP), l, ccv(psi), ld, ctx->d_fdB + (int64_t)nu * np_ * nb, np_,
                       st);
                }
                apply_DQ(np_, nb, ctx->d_B, ctx->d_blk_off, ctx->d_blk_n, ctx->d_Drow, ctx->d_Qrow, ctx->d_wband,
                         ctx->d_DB, ctx->d_QB, st);
                small_gemm(np_, nb, nb, ctx->d_QB, np_, false, ctx->d_Gam, nb, false, ctx->d_fY, np_, 1.0, 0.0, st);
                force_nl(np_, nb, ctx->d_fdB, ctx->d_DB, ctx->d_fY, ctx->d_fc, st);
            }
            force_local<T>(ctx->N, ctx->L, ctx->natoms, ctx->d_atoms, ctx->d_rho3, ctx->cf.w,
                           static_cast<const T*>(ctx->d_famp), static_cast<const T*>(ctx->d_fw2h), cv(ctx->d_ftab),
                           reinterpret_cast<V*>(ctx->d_grid), ccv(ctx->d_tw), ctx->d_fpart, st);
            const double N3 = double(ctx->N) * ctx->N * ctx->N;
            force_collect(ctx->natoms, np_, ctx->d_proj_atom, ctx->d_fc, ctx->d_fpart, ctx->omega * b / N3,
                          ctx->d_forces, st);
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(out_host, ctx->d_forces, sizeof(double) * 3 * ctx->natoms, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (tcg_timeout_take())
            return fail(ctx, ROKS_ETIMEOUT, "a tensor-core completion wait ran out (bounded mbarrier wait)");
        if (stream_timeout_take())
            return fail(ctx, ROKS_ETIMEOUT, "a bulk-copy wait of a streamed contraction ran out (bounded mbarrier wait)");
        for (int i = 0; i < 3 * ctx->natoms; ++i)
            if (!std::isfinite(out_host[i])) return fail(ctx, ROKS_EDIVERGED, "non-finite force");
        return ROKS_OK;
    }

    // One DIIS step (roks_diis_step): residual with the coupling
    // coefficients, e = K R into the ring, the new row of B, the window and
    // its coefficients on the device, the extrapolated orbitals, their
    // orthonormalisation and energy.  Launched eagerly: the ring slots change
    // from step to step.
    static roks_status diis_step(roks_ctx* ctx, void* psi, int64_t ld, const roks_diis_options& o,
                                 roks_diis_info* info) {
        cudaStream_t st = ctx->st;
        const int nb = ctx->nb, npw = ctx->npw;
        const int64_t l = ctx->ld_min;
        const int64_t blk = l * nb;
        roks_status r;
        if (!(ctx->pot_valid && ctx->cache_psi == psi && ctx->cache_ld == ld)) {
            r = density(ctx, psi, ld, nullptr);
            if (r != ROKS_OK) return r;
            r = potential(ctx);
            if (r != ROKS_OK) return r;
        }
        if (ctx->nproj > 0 && !(ctx->b_psi == psi && ctx->b_ld == ld)) {
            PROF("proj_PhPsi");
            cn(ctx, ctx->nproj, nb, npw, ccv(ctx->d_P), ctx->ld_min, ccv(psi), ld, ctx->d_B, ctx->nproj, st);
            ctx->b_psi = psi;
            ctx->b_ld = ld;
        }
        CK(cudaMemcpyAsync(&ctx->d_diis->E0, ctx->d_E + 10, sizeof(double), cudaMemcpyDeviceToDevice, st));
        r = apply(ctx, psi, ld, ctx->W_F, l, ctx->W_S, l, ctx->nproj > 0, ctx->yp_psi == psi && ctx->yp_ld == ld);
        if (r != ROKS_OK) return r;
        {
            PROF("subspace_theta");
            cn(ctx, nb, nb, npw, ccv(psi), ld, ccv(ctx->W_F), l, ctx->d_Th, nb, st);
        }
        const int slot = int(ctx->diis_count % o.history);
        V* Pj = cv(ctx->diis_ring) + slot * blk;
        V* Ej = cv(ctx->diis_ring) + (int64_t)(o.history + slot) * blk;
        {
            PROF("diis_residual");
            const bool singlet = ctx->mode == ROKS_MODE_SINGLET;
            diis_multipliers(nb, ctx->d_Th, singlet ? ctx->nc : -1, singlet ? ctx->nc + 1 : -1, o.lambda_ab,
                             o.lambda_ba, ctx->d_Gam, st);
            // R = F - S Lambda
            gemm_nn_io<T>(npw, nb, nb, ccv(ctx->W_S), l, ctx->d_Gam, nb, ccv(ctx->W_F), l, cv(ctx->W_G), l, -1.0,
                          1.0, ctx->d_gemm_work, st, ctx->gemm_work_elems * sizeof(double2));
            // e = K R (tau enters the extrapolation; d does not depend on a common
            // scale of e); the band norms |R_n|^2 stay in d_colout[0, nb) for rnorm2
            column_sums<T>(1, npw, nb, ccv(ctx->W_G), l, nullptr, 0, static_cast<const T*>(ctx->d_g2half),
                           ctx->d_colpart, ctx->d_colout, st);
            precondition<T>(npw, nb, ccv(ctx->W_G), l, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, Ej, l,
                            st);
            CK(cudaMemcpy2DAsync(Pj, l * sizeof(V), psi, ld * sizeof(V), npw * sizeof(V), nb,
                                 cudaMemcpyDeviceToDevice, st));
        }
        DiisOrder ord{};
        ord.n = int(std::min<long long>(ctx->diis_count + 1, o.history));
        for (int k = 0; k < ord.n; ++k) ord.slot[k] = int((ctx->diis_count + 1 - ord.n + k) % o.history);
        {
            PROF("diis_gram");
            diis_gram<T>(npw, nb, Ej, cv(ctx->diis_ring) + (int64_t)o.history * blk, blk, l, ord, ctx->d_diis_part,
                         ctx->d_diis, st);
            diis_solve(ctx->d_diis, ord, 1e-7, ctx->d_colout, nb, st);
        }
        {
            PROF("diis_combine");
            diis_combine<T>(npw, nb, ctx->d_diis, cv(ctx->diis_ring), cv(ctx->diis_ring) + (int64_t)o.history * blk,
                            blk, l, o.tau, cv(ctx->W_Y), l, st);
        }
        ctx->diis_count += 1;
        r = orth(ctx, ctx->W_Y, l, psi, ld, ctx->nproj > 0 ? ctx->d_B : nullptr);
        if (r != ROKS_OK) return r;
        ctx->b_psi = ctx->nproj > 0 ? psi : nullptr;
        ctx->b_ld = ld;
        r = density(ctx, psi, ld, ctx->nproj > 0 ? ctx->d_B : nullptr);
        if (r != ROKS_OK) return r;
        r = potential(ctx);
        if (r != ROKS_OK) return r;
        CK(cudaMemcpyAsync(&ctx->d_diis->Enew, ctx->d_E + 10, sizeof(double), cudaMemcpyDeviceToDevice, st));
        CK(cudaMemcpyAsync(ctx->h_diis, ctx->d_diis, sizeof(DiisState), cudaMemcpyDeviceToHost, st));
        CK(cudaMemcpyAsync(ctx->h_flag, ctx->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        int* sflag = stream_timeout_flag();
        ctx->h_flag[1] = 0;
        if (sflag) CK(cudaMemcpyAsync(ctx->h_flag + 1, sflag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        ctx->cache_psi = psi;
        ctx->cache_ld = ld;
        ctx->pot_valid = true;
        const bool tc_out = tcg_timeout_take() != 0;
        const bool st_out = ctx->h_flag[1] != 0;
        if (st_out) stream_timeout_take();
        if (tc_out || st_out) {
            CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
            CK(cudaStreamSynchronize(st));
            ctx->pot_valid = false;
            return fail(ctx, ROKS_ETIMEOUT, tc_out ? "a tensor-core completion wait ran out (bounded mbarrier wait)"
                                                   : "a bulk-copy wait of a streamed contraction ran out "
                                                     "(bounded mbarrier wait)");
        }
        const DiisState& h = *ctx->h_diis;
        if (*ctx->h_flag) {
            const int band = *ctx->h_flag - 1;
            CK(cudaMemsetAsync(ctx->d_flag, 0, sizeof(int), st));
            ctx->pot_valid = false;
            if (h.h == 0) return fail(ctx, ROKS_EDIVERGED, "non-finite residual");
            return fail(ctx, ROKS_ENOTPOSDEF, "extrapolated orbitals linearly dependent at band " + std::to_string(band));
        }
        if (info) {
            info->E = h.E0;
            info->E_new = h.Enew;
            info->res_norm = std::sqrt(h.rnorm2);
            info->window = h.h;
            for (int k = 0; k < ROKS_DIIS_MAX; ++k) info->coef[k] = k < h.h ? h.d[k] : 0.0;
        }
        if (h.h == 0 || !std::isfinite(h.Enew) || !std::isfinite(h.rnorm2))
            return fail(ctx, ROKS_EDIVERGED, "non-finite residual or energy");
        return ROKS_OK;
    }
};

void reset_history(roks_ctx* ctx) {
    PcgScalars h;
    std::memset(&h, 0, sizeof(h));
    h.dt = 0.3;
    h.neg_one = -1.0;
    cudaMemcpyAsync(ctx->d_sc, &h, sizeof(h), cudaMemcpyHostToDevice, ctx->st);
    const size_t bytes = (ctx->prec == ROKS_FP64 ? sizeof(double2) : sizeof(float2)) * (size_t)ctx->ld_min * ctx->nb;
    cudaMemsetAsync(ctx->W_sprev, 0, bytes, ctx->st);
    cudaMemsetAsync(ctx->d_Aprev, 0, sizeof(double2) * ctx->nb * ctx->nb, ctx->st);
    ctx->pot_valid = false;
    ctx->cache_psi = nullptr;
    ctx->b_psi = nullptr;
    ctx->n_small = 0;
    ctx->mlp_judging = false;
    ctx->diis_count = 0;
    ctx->diis_small = 0;
    ctx->pcg_fresh = false;
    ctx->yp_psi = nullptr;
    ctx->steps = 0;
    cudaStreamSynchronize(ctx->st);
}

// The context's wait cap and tensor-core split depth for the launches of
// one entry point.
void enter(roks_ctx* ctx) {
    set_wait_cap(ctx->wait_cap);
    tcg_set_waves(ctx->tc_waves_x2);
}

// Times fn(candidate) (three launches after one warm-up, CUDA events on the
// context's stream) and returns the fastest candidate; ms[i] gets the times.
template <typename F>
int pick_fastest(roks_ctx* ctx, const int* cand, int nc, double* ms, F fn) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    int best = cand[0];
    double best_ms = 1e300;
    for (int i = 0; i < nc; ++i) {
        fn(cand[i]);
        cudaEventRecord(a, ctx->st);
        for (int r = 0; r < 3; ++r) fn(cand[i]);
        cudaEventRecord(b, ctx->st);
        cudaEventSynchronize(b);
        float t = 0.f;
        cudaEventElapsedTime(&t, a, b);
        ms[i] = t / 3.0;
        if (ms[i] < best_ms) {
            best_ms = ms[i];
            best = cand[i];
        }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

// Autotuner (roks_options.autotune): the band grouping of the density's x
// stage (grid depth against the fixed-order reduction of the group slots)
// and, on the mixed path, the split depth of the tensor-core A^H B products,
// each timed on the context's own buffers and sizes.
roks_status autotune(roks_ctx* ctx) {
    enter(ctx);
    const Sphere s = sphere(ctx);
    const int g_cand[3] = {2, 4, 8};
    if (ctx->prec == ROKS_FP64)
        ctx->dens_groups = pick_fastest(ctx, g_cand, 3, ctx->tune_ms, [&](int g) {
            band_x_density<double>(s, static_cast<const double2*>(ctx->d_tw), static_cast<double2*>(ctx->d_Yp),
                                   ctx->d_rho3, ctx->d_rho_slot, g, 0, ctx->nbt - ctx->ne, ctx->nct, 1.0 / ctx->omega, ctx->st);
        });
    else
        ctx->dens_groups = pick_fastest(ctx, g_cand, 3, ctx->tune_ms, [&](int g) {
            band_x_density<float>(s, static_cast<const float2*>(ctx->d_tw), static_cast<float2*>(ctx->d_Yp),
                                  ctx->d_rho3, ctx->d_rho_slot, g, 0, ctx->nbt - ctx->ne, ctx->nct, 1.0 / ctx->omega, ctx->st);
        });
    // the largest A^H B product of a step that runs on the tensor cores
    const int M = ctx->nproj >= ctx->nb ? ctx->nproj : ctx->nb;
    const void* A = ctx->nproj >= ctx->nb ? ctx->d_P : ctx->W_Y;
    if (ctx->prec == ROKS_MIXED && tcg_cn_takes(M, ctx->nb, ctx->npw)) {
        // 2: stream-K over one wave; 5, 8: K split into 2.5 or 4 waves
        const int w_cand[3] = {2, 5, 8};
        ctx->tc_waves_x2 = pick_fastest(ctx, w_cand, 3, ctx->tune_ms + 3, [&](int w) {
            tcg_set_waves(w);
            gemm_cn<float>(M, ctx->nb, ctx->npw, static_cast<const float2*>(A), ctx->ld_min,
                           static_cast<const float2*>(ctx->W_Y), ctx->ld_min, ctx->d_B2, M, ctx->d_gemm_work,
                           ctx->gemm_work_elems, ctx->st);
        });
        tcg_set_waves(ctx->tc_waves_x2);
    }
    const cudaError_t e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) return fail(ctx, ROKS_ECUDA, std::string("autotune: ") + cudaGetErrorString(e));
    return ROKS_OK;
}

}  // namespace

// ====================================================================== C ABI
extern "C" {

roks_status roks_setup(const roks_cell* cell, double ecut, int natoms, const roks_atom* atoms, int nspecies,
                       const roks_species* species, const roks_occ* occ, const roks_options* opt,
                       void* cuda_stream, roks_ctx** out) {
    if (!out) return ROKS_EINVAL;
    *out = nullptr;
    if (!cell || !occ || !opt || (natoms > 0 && !atoms) || (nspecies > 0 && !species) || natoms < 0 ||
        nspecies < 0)
        return ROKS_EINVAL;
    if (!(cell->L > 0) || !(ecut > 0) || !grid_supported(cell->grid)) return ROKS_EINVAL;
    if (occ->n_closed < 0 || occ->mode < 0 || occ->mode > 2) return ROKS_EINVAL;
    if (occ->n_open != (occ->mode == ROKS_MODE_GS ? 0 : 2)) return ROKS_EINVAL;
    if (opt->precision != ROKS_FP64 && opt->precision != ROKS_MIXED) return ROKS_EINVAL;
    if (!(opt->alpha >= 0.0 && opt->alpha <= 1.0)) return ROKS_EINVAL;
    if (!(opt->e_tol >= 0.0) || !(opt->g_tol >= 0.0) || opt->max_iter < 0) return ROKS_EINVAL;
    if (opt->precond != ROKS_PRECOND_TPA && opt->precond != ROKS_PRECOND_TPA_MLP) return ROKS_EINVAL;
    if (opt->exx_kernel != ROKS_EXX_TRUNCATED && opt->exx_kernel != ROKS_EXX_BARE) return ROKS_EINVAL;
    if (opt->autotune != 0 && opt->autotune != 1) return ROKS_EINVAL;
    if (opt->gamma != 0 && opt->gamma != 1) return ROKS_EINVAL;
    if (opt->xc != ROKS_XC_SLATER && opt->xc != ROKS_XC_PBE_X) return ROKS_EINVAL;
    // the Gamma-point packing pairs bands (2k, 2k + 1): an open pair must be
    // one packed band, and exact exchange runs on the complex path only
    if (opt->gamma && (opt->alpha != 0.0 || (occ->mode != ROKS_MODE_GS && (occ->n_closed & 1)))) return ROKS_EINVAL;
    // empty bands: the complex path without exact exchange
    if (occ->n_empty < 0 || (occ->n_empty > 0 && (opt->gamma || opt->alpha != 0.0))) return ROKS_EINVAL;
    roks_ctx* ctx = new (std::nothrow) roks_ctx();
    if (!ctx) return ROKS_ENOMEM;
    ctx->st = static_cast<cudaStream_t>(cuda_stream);
    {
        // ROKS_GRAPHS=0 launches every PCG iteration kernel by kernel
        const char* g = std::getenv("ROKS_GRAPHS");
        ctx->graphs = !(g && g[0] == '0');
    }
    ctx->prec = opt->precision;
    ctx->L = cell->L;
    ctx->N = cell->grid;
    ctx->omega = cell->L * cell->L * cell->L;
    ctx->ecut = ecut;
    ctx->alpha = opt->alpha;
    ctx->e_tol = opt->e_tol > 0 ? opt->e_tol : 1e-6;
    ctx->g_tol = opt->g_tol;
    ctx->max_iter = opt->max_iter;
    ctx->seed = opt->seed;
    ctx->wait_cap = opt->wait_cap;
    ctx->exx_kernel = opt->exx_kernel;
    ctx->autotune = opt->autotune;
    ctx->gamma = opt->gamma;
    ctx->xc = opt->xc;
    ctx->mlp_kind = opt->precond;   // all-zero network weights until trained ones are set
    ctx->suppress_ab = opt->suppress_ab;
    ctx->mode = occ->mode;
    ctx->nc = occ->n_closed;
    ctx->nocc = occ->n_closed + (occ->mode == ROKS_MODE_GS ? 0 : 2);
    ctx->ne = occ->n_empty;
    ctx->nb = ctx->nocc + ctx->ne;
    ctx->natoms = natoms;
    auto bail = [&](roks_status s, const std::string& m) {
        roks_destroy(ctx);
        (void)m;
        return s;
    };
    if (ctx->nb <= 0) return bail(ROKS_EINVAL, "no bands");
    // -------- basis: i^2 + j^2 + k^2 <= floor(2 ecut (L / 2 pi)^2)
    const double q = cell->L / (2.0 * M_PI);
    const double Mq = std::floor(2.0 * ecut * q * q);
    if (Mq > 1e7) return bail(ROKS_EINVAL, "cut-off too large");
    ctx->M = (int)Mq;
    ctx->nmax = isqrt_floor(ctx->M);
    const int n = ctx->nmax, N = ctx->N;
    if (N < 2 * n + 1) return bail(ROKS_EINVAL, "grid smaller than 2 n + 1");
    std::vector<int> col_start, col_kmax, plane_col0, plane_jmax;
    for (int i = -n; i <= n; ++i) {
        const int ji = isqrt_floor(ctx->M - i * i);
        plane_col0.push_back((int)col_kmax.size());
        plane_jmax.push_back(ji);
        for (int j = -ji; j <= ji; ++j) {
            const int kj = isqrt_floor(ctx->M - i * i - j * j);
            col_start.push_back((int)(ctx->miller.size() / 3));
            col_kmax.push_back(kj);
            for (int k = -kj; k <= kj; ++k) {
                ctx->miller.push_back(i);
                ctx->miller.push_back(j);
                ctx->miller.push_back(k);
            }
        }
    }
    ctx->npw = (int)(ctx->miller.size() / 3);
    ctx->npw_full = ctx->npw;
    if (ctx->gamma) {
        // the half sphere: G = 0 (row h0, the middle of the symmetric,
        // lexicographically sorted basis) and every row after it
        ctx->h0 = (ctx->npw - 1) / 2;
        const int32_t* g0 = &ctx->miller[3 * (size_t)ctx->h0];
        if (g0[0] != 0 || g0[1] != 0 || g0[2] != 0) return bail(ROKS_EINVAL, "basis without G = 0 at its middle");
        ctx->miller.erase(ctx->miller.begin(), ctx->miller.begin() + 3 * (size_t)ctx->h0);
        ctx->npw = ctx->npw_full - ctx->h0;
    }
    ctx->ld_min = (ctx->npw + 31) / 32 * 32;
    ctx->ncol = (int)col_kmax.size();
    ctx->np = 2 * n + 1;
    if (ctx->nb > ctx->npw) return bail(ROKS_EINVAL, "more bands than plane waves");
    if (ctx->gamma) {
        ctx->nbt = (ctx->nb + 1) / 2;
        ctx->nct = ctx->mode == ROKS_MODE_GS ? ctx->nbt : ctx->nc / 2;
        ctx->split_t = ctx->mode == ROKS_MODE_GS ? -1 : ctx->nc / 2;
        ctx->ldc_pk = ((int64_t)ctx->npw_full + 31) / 32 * 32;
    } else {
        ctx->nbt = ctx->nb;
        ctx->nct = ctx->nc;
        ctx->split_t = -1;
    }
    // -------- occupations (Eqs. 7, 13): f table and c_L
    const double ftab[3][4] = {{1, 1, 1, 1}, {1, 0, 1, 0}, {0, 1, 1, 0}};
    ctx->cM = occ->mode == 0 ? 1.0 : (occ->mode == 1 ? 2.0 : 0.0);
    ctx->cT = occ->mode == 0 ? 0.0 : (occ->mode == 1 ? -1.0 : 1.0);
    const double cch[4] = {ctx->cM, ctx->cM, ctx->cT, ctx->cT};
    for (int k = 0; k < 3; ++k) {
        double w = 0;
        for (int ch = 0; ch < 4; ++ch) {
            ctx->cf.f[k][ch] = ftab[k][ch];
            ctx->cf.C[k][ch] = cch[ch] * ftab[k][ch];
            w += ctx->cf.C[k][ch];
        }
        ctx->cf.w[k] = w;
    }
    ctx->cf.xscale = 1.0 - opt->alpha;
    // exchange pair weights w(k, k') = sum_ch c_L f_k f_k' (Eq. 13 with the
    // exact-exchange energy of each configuration)
    {
        const double sq = std::sqrt(ctx->omega);
        for (int k = 0; k < 3; ++k)
            for (int k2 = 0; k2 < 3; ++k2) {
                double w = 0, fm = 0, ft = 0;
                for (int ch = 0; ch < 4; ++ch) {
                    const double ff = ftab[k][ch] * ftab[k2][ch];
                    w += cch[ch] * ff;
                    if (ch < 2) fm += ff;
                    else ft += ff;
                }
                ctx->exc.c[k][k2] = -opt->alpha * sq * w;
                ctx->exc.fM[k][k2] = fm;
                ctx->exc.fT[k][k2] = ft;
                if (k == 0) ctx->exc.wxc[k2] = w;
            }
        ctx->exc.alpha = opt->alpha;
        ctx->exc.n_closed = ctx->nc;
    }
    // -------- projectors: per-projector table and block-diagonal rows
    std::vector<double> proj, Drow, Qrow, atomtab;
    std::vector<int> blk_off, blk_n;
    for (int a = 0; a < natoms; ++a) {
        const roks_atom& at = atoms[a];
        if (at.species < 0 || at.species >= nspecies || !(at.width > 0)) return bail(ROKS_EINVAL, "bad atom");
        atomtab.insert(atomtab.end(), {at.pos[0], at.pos[1], at.pos[2], at.depth, at.width});
        const roks_species& sp = species[at.species];
        if (sp.nproj < 0 || sp.nproj > kMaxBlk) return bail(ROKS_EINVAL, "bad projector count");
        if (sp.nproj > 0 && (!sp.l || !sp.m || !sp.rc || !sp.D || !sp.Q)) return bail(ROKS_EINVAL, "bad species");
        const int off = (int)blk_off.size();
        for (int c = 0; c < sp.nproj; ++c) ctx->proj_atom_h.push_back(a);
        for (int c = 0; c < sp.nproj; ++c) {
            if ((sp.l[c] != 0 && sp.l[c] != 1) || sp.m[c] < 0 || sp.m[c] > 2 || !(sp.rc[c] > 0))
                return bail(ROKS_EINVAL, "bad projector channel");
            proj.insert(proj.end(), {at.pos[0], at.pos[1], at.pos[2], sp.rc[c], (double)sp.l[c], (double)sp.m[c]});
            blk_off.push_back(off);
            blk_n.push_back(sp.nproj);
            for (int j = 0; j < kMaxBlk; ++j) {
                Drow.push_back(j < sp.nproj ? sp.D[c * sp.nproj + j] : 0.0);
                Qrow.push_back(j < sp.nproj ? sp.Q[c * sp.nproj + j] : 0.0);
            }
        }
    }
    ctx->nproj = (int)blk_off.size();
    ctx->atoms_h = atomtab;
    // -------- device allocations
    const bool f64 = ctx->prec == ROKS_FP64;
    const size_t cs = f64 ? sizeof(double2) : sizeof(float2);
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    const size_t N3 = (size_t)N * N * N;
    const int nb = ctx->nb, l = ctx->ld_min, npw = ctx->npw;
    cudaError_t e = cudaSuccess;
#define AL(p, bytes)                                                   \
    do {                                                               \
        e = dalloc(ctx, &(p), (bytes));                                \
        if (e != cudaSuccess) return bail(ROKS_ENOMEM, "cudaMalloc"); \
    } while (0)
    AL(ctx->d_col_start, sizeof(int) * ctx->ncol);
    AL(ctx->d_col_kmax, sizeof(int) * ctx->ncol);
    AL(ctx->d_plane_col0, sizeof(int) * ctx->np);
    AL(ctx->d_plane_jmax, sizeof(int) * ctx->np);
    AL(ctx->d_miller, sizeof(int) * 3 * npw);
    AL(ctx->d_shell, sizeof(int) * nb);
    AL(ctx->d_g2, sizeof(double) * npw);
    AL(ctx->d_g2half, rs * npw);
    AL(ctx->d_wk, rs * 3);
    AL(ctx->d_wband, sizeof(double) * nb);
    AL(ctx->d_vloc, sizeof(double) * N3);
    AL(ctx->d_mlp, sizeof(float) * ROKS_MLP_PARAMS);
    if (ctx->prec != ROKS_FP64) AL(ctx->d_vloc_t, sizeof(float) * N3);
    AL(ctx->d_P, cs * (size_t)l * (ctx->nproj > 0 ? ctx->nproj : 1));
    AL(ctx->d_blk_off, sizeof(int) * (ctx->nproj + 1));
    AL(ctx->d_blk_n, sizeof(int) * (ctx->nproj + 1));
    AL(ctx->d_Drow, sizeof(double) * (Drow.size() + 1));
    AL(ctx->d_Qrow, sizeof(double) * (Qrow.size() + 1));
    AL(ctx->d_tw, cs * N);
    AL(ctx->d_tw64, sizeof(double2) * N);
    AL(ctx->d_Zc, cs * (size_t)ctx->nbt * ctx->ncol * N);
    AL(ctx->d_Yp, cs * (size_t)ctx->nbt * ctx->np * N * N);
    if (ctx->gamma) AL(ctx->d_Cpk, cs * (size_t)ctx->ldc_pk * ctx->nbt);
    AL(ctx->d_rho3, sizeof(double) * 3 * N3);
    AL(ctx->d_rho_slot, sizeof(double) * (opt->autotune ? kDensityGroupsMax : kDensityGroups) * N3);
    if (ctx->xc == ROKS_XC_PBE_X) {
        AL(ctx->gga.gg, 2 * rs * 2 * N3);
        AL(ctx->gga.dd, 2 * rs * 6 * N3);
        AL(ctx->gga.v4, rs * 4 * N3);
        // PBE's kappa and mu = beta pi^2 / 3 (beta of the gradient expansion)
        ctx->gga.kappa = 0.804;
        ctx->gga.mu = 0.06672455060314922 * M_PI * M_PI / 3.0;
        ctx->gga.rho_min = 1e-10;
    }
    if (ctx->ne > 0) {
        AL(ctx->d_rho_e, sizeof(double) * (size_t)(ctx->ne + 1) * N3);
        AL(ctx->d_dk, sizeof(double) * 3 * ctx->ne * (1 + 64));   // values, then block partials
    }
    AL(ctx->d_xc3, sizeof(double) * 3 * N3);
    AL(ctx->d_grid, sizeof(double2) * N3);
    AL(ctx->d_Vk, rs * 3 * N3);
    AL(ctx->d_part, sizeof(double) * potentials_part_elems());
    AL(ctx->d_out6, sizeof(double) * 8);
    AL(ctx->d_E, sizeof(double) * 12);
    void** bands[] = {&ctx->W_F, &ctx->W_S, &ctx->W_G, &ctx->W_gI, &ctx->W_K, &ctx->W_u,
                      &ctx->W_v, &ctx->W_s, &ctx->W_sprev, &ctx->W_Y, &ctx->W_Y2};
    for (void** b : bands) AL(*b, cs * (size_t)l * nb);
    double2** smalls[] = {&ctx->d_Th, &ctx->d_Gam, &ctx->d_Gin, &ctx->d_A, &ctx->d_Aprev, &ctx->d_Atot, &ctx->d_U,
                          &ctx->d_O, &ctx->d_L, &ctx->d_LinvH, &ctx->d_Msm, &ctx->d_e1, &ctx->d_e2, &ctx->d_e3};
    for (double2** b : smalls) AL(*b, sizeof(double2) * nb * nb);
    const int np_ = ctx->nproj > 0 ? ctx->nproj : 1;
    AL(ctx->d_B, sizeof(double2) * np_ * nb);
    AL(ctx->d_DB, sizeof(double2) * np_ * nb);
    AL(ctx->d_QB, sizeof(double2) * np_ * nb);
    AL(ctx->d_B2, sizeof(double2) * np_ * nb);
    size_t gw = gemm_cn_work(np_ > nb ? np_ : nb, nb, npw);
    if (!f64) {
        // partial sums of the tensor-core contractions and the split B blocks
        // of their tall products share the buffer
        // (sized for the deepest split the autotuner may choose)
        tcg_set_waves(opt->autotune ? 8 : ctx->tc_waves_x2);
        const size_t tb = std::max(std::max(tcg_cn_work_bytes(np_, nb, npw), tcg_cn_work_bytes(nb, nb, npw)),
                                   std::max(tcg_nn_work_bytes(nb, np_), tcg_nn_work_bytes(nb, nb)));
        gw = std::max(gw, (tb + sizeof(double2) - 1) / sizeof(double2));
    }
    ctx->gemm_work_elems = gw;
    tcg_set_waves(ctx->tc_waves_x2);
    AL(ctx->d_gemm_work, sizeof(double2) * gw);
    AL(ctx->d_kin_b, sizeof(double) * nb);
    AL(ctx->d_nl_b, sizeof(double) * nb);
    AL(ctx->d_colpart, sizeof(double) * 2 * nb * 16);
    AL(ctx->d_colout, sizeof(double) * 4 * nb);   // op-1 sums (2 nb), then the TPA coefficients (2 nb)
    AL(ctx->d_expm_info, sizeof(double) * 2);
    if (nb > 64) {
        const size_t w1 = cholesky_big_work_bytes(nb, f64), w2 = expm_big_work_bytes(nb, f64);
        AL(ctx->d_bigwork, w1 > w2 ? w1 : w2);
    }
    AL(ctx->d_flag, sizeof(int) * 2);
    {
        void* hp = nullptr;
        if (cudaMallocHost(&hp, sizeof(PcgScalars) + 64) != cudaSuccess) return bail(ROKS_ENOMEM, "cudaMallocHost");
        ctx->h_sc = static_cast<PcgScalars*>(hp);
        ctx->h_flag = reinterpret_cast<int*>(static_cast<char*>(hp) + sizeof(PcgScalars) + 32);
        *ctx->h_flag = 0;
    }
    AL(ctx->d_sc, sizeof(PcgScalars));
    std::vector<int> pj, pn;
    if (opt->alpha != 0.0) {
        for (int n2 = 0; n2 < nb; ++n2)
            for (int j2 = 0; j2 <= n2; ++j2) {
                pj.push_back(j2);
                pn.push_back(n2);
            }
        ctx->npairs = (int)pj.size();
        const size_t grid_bytes = cs * N3;
        int batch = (int)((256u << 20) / grid_bytes);
        if (batch < 1) batch = 1;
        if (batch > 64) batch = 64;
        if (batch > ctx->npairs) batch = ctx->npairs;
        ctx->exx_batch = batch;
        AL(ctx->d_Phi, cs * N3 * nb);
        AL(ctx->d_Xx, cs * N3 * nb);
        AL(ctx->d_exbuf, cs * N3 * batch);
        AL(ctx->d_vG, rs * N3);
        AL(ctx->d_pj, sizeof(int) * ctx->npairs);
        AL(ctx->d_pn, sizeof(int) * ctx->npairs);
        AL(ctx->d_expart, sizeof(double) * batch * kExxBlocks);
        AL(ctx->d_Kmat, sizeof(double) * nb * nb);
        AL(ctx->d_hf2, sizeof(double) * 2);
        AL(ctx->d_exopen, sizeof(double) * 2);
    }
    if (!f64 && ctx->nproj > 0 && tcg_nn_takes(npw, nb, ctx->nproj))
        AL(ctx->d_Psplit_nn, tcg_presplit_bytes(npw, ctx->nproj));
    double* d_atoms = nullptr;
    double* d_proj = nullptr;
    AL(d_atoms, sizeof(double) * (atomtab.size() + 1));
    AL(d_proj, sizeof(double) * (proj.size() + 1));
    ctx->d_atoms = d_atoms;
#undef AL
    // -------- uploads
    // shells of Eq. 20: closed 0, open a 1 and b 2 (the triplet's a, b: one
    // open shell 1), empty 3; the operator applied to an empty band is F^c
    std::vector<int> shell(nb), dummy;
    auto band_class = [&](int b) { return (b < ctx->nc || b >= ctx->nocc) ? 0 : b - ctx->nc + 1; };
    for (int b = 0; b < nb; ++b) {
        const int cls = band_class(b);
        shell[b] = b >= ctx->nocc ? 3 : ((ctx->mode == ROKS_MODE_TRIPLET && cls > 0) ? 1 : cls);
    }
    std::vector<double> g2(npw), wband(nb);
    const double bq = 2.0 * M_PI / cell->L;
    for (int g = 0; g < npw; ++g) {
        const double gx = bq * ctx->miller[3 * g], gy = bq * ctx->miller[3 * g + 1], gz = bq * ctx->miller[3 * g + 2];
        g2[g] = gx * gx + gy * gy + gz * gz;
    }
    for (int b = 0; b < nb; ++b) wband[b] = ctx->cf.w[band_class(b)];
    std::vector<double2> tw64(N);
    for (int t = 0; t < N; ++t) tw64[t] = make_double2(std::cos(-2.0 * M_PI * t / N), std::sin(-2.0 * M_PI * t / N));
    auto up = [&](void* dst, const void* src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, ctx->st) : cudaSuccess;
    };
    e = up(ctx->d_col_start, col_start.data(), sizeof(int) * col_start.size());
    if (e == cudaSuccess) e = up(ctx->d_col_kmax, col_kmax.data(), sizeof(int) * col_kmax.size());
    if (e == cudaSuccess) e = up(ctx->d_plane_col0, plane_col0.data(), sizeof(int) * plane_col0.size());
    if (e == cudaSuccess) e = up(ctx->d_plane_jmax, plane_jmax.data(), sizeof(int) * plane_jmax.size());
    if (e == cudaSuccess) e = up(ctx->d_miller, ctx->miller.data(), sizeof(int) * ctx->miller.size());
    if (e == cudaSuccess) e = up(ctx->d_shell, shell.data(), sizeof(int) * nb);
    if (e == cudaSuccess) e = up(ctx->d_g2, g2.data(), sizeof(double) * npw);
    if (e == cudaSuccess) e = up(ctx->d_wband, wband.data(), sizeof(double) * nb);
    if (e == cudaSuccess) e = up(ctx->d_tw64, tw64.data(), sizeof(double2) * N);
    if (e == cudaSuccess) e = up(ctx->d_blk_off, blk_off.data(), sizeof(int) * blk_off.size());
    if (e == cudaSuccess) e = up(ctx->d_blk_n, blk_n.data(), sizeof(int) * blk_n.size());
    if (e == cudaSuccess) e = up(ctx->d_Drow, Drow.data(), sizeof(double) * Drow.size());
    if (e == cudaSuccess) e = up(ctx->d_Qrow, Qrow.data(), sizeof(double) * Qrow.size());
    if (e == cudaSuccess) e = up(d_atoms, atomtab.data(), sizeof(double) * atomtab.size());
    if (e == cudaSuccess) e = up(d_proj, proj.data(), sizeof(double) * proj.size());
    if (e == cudaSuccess && ctx->npairs > 0) e = up(ctx->d_pj, pj.data(), sizeof(int) * pj.size());
    if (e == cudaSuccess && ctx->npairs > 0) e = up(ctx->d_pn, pn.data(), sizeof(int) * pn.size());
    if (e != cudaSuccess) return bail(ROKS_ECUDA, "upload");
    // typed tables
    std::vector<double> wk(ctx->cf.w, ctx->cf.w + 3);
    double* d_tmp = nullptr;
    e = cudaMalloc(&d_tmp, sizeof(double) * (npw + 8));
    if (e != cudaSuccess) return bail(ROKS_ENOMEM, "cudaMalloc");
    std::vector<double> g2h(npw);
    for (int g = 0; g < npw; ++g) g2h[g] = 0.5 * g2[g];
    std::vector<double> twf(2 * N);
    for (int t = 0; t < N; ++t) { twf[2 * t] = tw64[t].x; twf[2 * t + 1] = tw64[t].y; }
    cudaMemcpyAsync(d_tmp, g2h.data(), sizeof(double) * npw, cudaMemcpyHostToDevice, ctx->st);
    if (f64) to_real_type<double>(npw, d_tmp, static_cast<double*>(ctx->d_g2half), 1.0, ctx->st);
    else to_real_type<float>(npw, d_tmp, static_cast<float*>(ctx->d_g2half), 1.0, ctx->st);
    cudaStreamSynchronize(ctx->st);
    cudaMemcpyAsync(d_tmp, wk.data(), sizeof(double) * 3, cudaMemcpyHostToDevice, ctx->st);
    if (f64) to_real_type<double>(3, d_tmp, static_cast<double*>(ctx->d_wk), 1.0, ctx->st);
    else to_real_type<float>(3, d_tmp, static_cast<float*>(ctx->d_wk), 1.0, ctx->st);
    cudaStreamSynchronize(ctx->st);
    cudaFree(d_tmp);
    if (f64) {
        cudaMemcpyAsync(ctx->d_tw, tw64.data(), sizeof(double2) * N, cudaMemcpyHostToDevice, ctx->st);
    } else {
        std::vector<float2> t32(N);
        for (int t = 0; t < N; ++t) t32[t] = make_float2((float)tw64[t].x, (float)tw64[t].y);
        cudaMemcpyAsync(ctx->d_tw, t32.data(), sizeof(float2) * N, cudaMemcpyHostToDevice, ctx->st);
        cudaStreamSynchronize(ctx->st);
    }
    // -------- model on the device
    vloc_setup(N, cell->L, natoms, d_atoms, ctx->d_grid, ctx->d_vloc, ctx->d_tw64, ctx->st);
    if (ctx->prec == ROKS_FP64) ctx->d_vloc_t = ctx->d_vloc;
    else to_real_type<float>(N3, ctx->d_vloc, static_cast<float*>(ctx->d_vloc_t), 1.0, ctx->st);
    if (f64) projectors_setup<double>(npw, ctx->nproj, cell->L, ctx->d_miller, d_proj,
                                      static_cast<double2*>(ctx->d_P), l, ctx->st);
    else projectors_setup<float>(npw, ctx->nproj, cell->L, ctx->d_miller, d_proj, static_cast<float2*>(ctx->d_P), l,
                                 ctx->st);
    if (ctx->gamma && ctx->nproj > 0) {
        // real-space-real projectors in the stored half-sphere form
        if (f64) gamma_scale_rows<double>(npw, ctx->nproj, static_cast<double2*>(ctx->d_P), l, ctx->st);
        else gamma_scale_rows<float>(npw, ctx->nproj, static_cast<float2*>(ctx->d_P), l, ctx->st);
    }
    if (ctx->d_Psplit_nn &&
        !tcg_presplit(npw, ctx->nproj, static_cast<const float2*>(ctx->d_P), l, ctx->d_Psplit_nn, ctx->st))
        return bail(ROKS_ECUDA, "projector split");
    if (opt->alpha != 0.0) {
        const int bare = opt->exx_kernel == ROKS_EXX_BARE ? 1 : 0;
        if (f64) exx_setup_kernel<double>(N, cell->L, bare, static_cast<double*>(ctx->d_vG), ctx->st);
        else exx_setup_kernel<float>(N, cell->L, bare, static_cast<float*>(ctx->d_vG), ctx->st);
    }
    e = cudaStreamSynchronize(ctx->st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return bail(ROKS_ECUDA, cudaGetErrorString(e));
    reset_history(ctx);
    if (opt->autotune) {
        const roks_status r = autotune(ctx);
        if (r != ROKS_OK) return bail(r, ctx->err);
        reset_history(ctx);
    }
    *out = ctx;
    return ROKS_OK;
}

roks_status roks_tuning_get(const roks_ctx* ctx, roks_tuning* t) {
    if (!ctx || !t) return ROKS_EINVAL;
    t->density_groups = ctx->dens_groups;
    t->tc_split_waves_x2 = ctx->tc_waves_x2;
    for (int i = 0; i < 6; ++i) t->candidate_ms[i] = ctx->tune_ms[i];
    return ROKS_OK;
}

roks_status roks_basis(roks_ctx* ctx, int* npw, int* nbands, int* ld_min, const int32_t** miller) {
    if (!ctx) return ROKS_EINVAL;
    if (npw) *npw = ctx->npw;
    if (nbands) *nbands = ctx->nb;
    if (ld_min) *ld_min = ctx->ld_min;
    if (miller) *miller = ctx->miller.data();
    return ROKS_OK;
}

static roks_status check_psi(roks_ctx* ctx, const void* psi, int64_t ld) {
    if (!psi) return fail(ctx, ROKS_EINVAL, "null orbital pointer");
    if (ld < ctx->npw) return fail(ctx, ROKS_EINVAL, "leading dimension smaller than npw");
    return ROKS_OK;
}

roks_status roks_init_orbitals(roks_ctx* ctx, const double* u_host, void* psi, int64_t ld) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    const int64_t l = ctx->ld_min;
    const bool f64 = ctx->prec == ROKS_FP64;
    // host numbers are staged, a few bands at a time, in a band block the
    // orthonormalisation below does not use (no allocation)
    const size_t stage_doubles = (f64 ? sizeof(double2) : sizeof(float2)) * (size_t)l * ctx->nb / sizeof(double);
    const int per = u_host ? (int)(stage_doubles / (2 * (size_t)ctx->npw)) : ctx->nb;
    if (per < 1) return fail(ctx, ROKS_EINVAL, "staging block too small");
    double* stage = static_cast<double*>(ctx->W_u);
    for (int b0 = 0; b0 < ctx->nb; b0 += per) {
        const int nbk = std::min(per, ctx->nb - b0);
        const double* u = nullptr;
        if (u_host) {
            CK(cudaMemcpyAsync(stage, u_host + 2 * (size_t)ctx->npw * b0, sizeof(double) * 2 * (size_t)ctx->npw * nbk,
                               cudaMemcpyHostToDevice, ctx->st));
            u = stage;
        }
        if (f64)
            init_orbitals<double>(ctx->npw, b0, nbk, u, ctx->seed, ctx->d_g2, static_cast<double2*>(ctx->W_Y), l,
                                  ctx->st);
        else
            init_orbitals<float>(ctx->npw, b0, nbk, u, ctx->seed, ctx->d_g2, static_cast<float2*>(ctx->W_Y), l,
                                 ctx->st);
    }
    if (ctx->gamma) {
        // real orbitals: c(0) real, the other half-sphere rows in the stored form
        if (f64) gamma_scale_rows<double>(ctx->npw, ctx->nb, static_cast<double2*>(ctx->W_Y), l, ctx->st);
        else gamma_scale_rows<float>(ctx->npw, ctx->nb, static_cast<float2*>(ctx->W_Y), l, ctx->st);
    }
    CK(cudaGetLastError());
    r = f64 ? Impl<double>::orth(ctx, ctx->W_Y, l, psi, ld, nullptr) : Impl<float>::orth(ctx, ctx->W_Y, l, psi, ld, nullptr);
    cudaStreamSynchronize(ctx->st);
    if (r != ROKS_OK) return r;
    reset_history(ctx);
    return ctx->prec == ROKS_FP64 ? Impl<double>::check_flag(ctx) : Impl<float>::check_flag(ctx);
}

roks_status roks_invalidate(roks_ctx* ctx) {
    if (!ctx) return ROKS_EINVAL;
    reset_history(ctx);
    return ROKS_OK;
}

roks_status roks_density(roks_ctx* ctx, const void* psi, int64_t ld, double* rho_out) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    ctx->pot_valid = false;
    r = ctx->prec == ROKS_FP64 ? Impl<double>::density(ctx, psi, ld, nullptr)
                               : Impl<float>::density(ctx, psi, ld, nullptr);
    if (r != ROKS_OK) return r;
    if (rho_out) {
        const int64_t n3 = 3 * (int64_t)ctx->N * ctx->N * ctx->N;
        if (ctx->prec == ROKS_FP64) density_to_f64<double>(n3, ctx->d_rho3, static_cast<double*>(rho_out), ctx->st);
        else density_to_f64<float>(n3, ctx->d_rho3, static_cast<double*>(rho_out), ctx->st);
        CK(cudaGetLastError());
    }
    return ROKS_OK;
}

static void fill_energies(const double* h, roks_energies* e) {
    e->E_kin = h[0]; e->E_loc = h[1]; e->E_nl = h[2]; e->E_H = h[3];
    e->E_x_M = h[4]; e->E_x_T = h[5]; e->E_hf_M = h[6]; e->E_hf_T = h[7];
    e->E_M = h[8]; e->E_T = h[9]; e->E_total = h[10];
}

roks_status roks_energies_get(roks_ctx* ctx, roks_energies* e) {
    if (!ctx || !e) return ROKS_EINVAL;
    double h[12];
    CK(cudaMemcpyAsync(h, ctx->d_E, sizeof(double) * 11, cudaMemcpyDeviceToHost, ctx->st));
    CK(cudaStreamSynchronize(ctx->st));
    fill_energies(h, e);
    return ROKS_OK;
}

roks_status roks_potential(roks_ctx* ctx, roks_energies* e, void* vclass_out) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = ctx->prec == ROKS_FP64 ? Impl<double>::potential(ctx) : Impl<float>::potential(ctx);
    if (r != ROKS_OK) return r;
    const size_t N3 = (size_t)ctx->N * ctx->N * ctx->N;
    if (vclass_out)
        CK(cudaMemcpyAsync(vclass_out, ctx->d_Vk, (ctx->prec == ROKS_FP64 ? 8 : 4) * 3 * N3, cudaMemcpyDeviceToDevice,
                           ctx->st));
    if (e) return roks_energies_get(ctx, e);
    CK(cudaStreamSynchronize(ctx->st));
    return ROKS_OK;
}

roks_status roks_apply_h(roks_ctx* ctx, const void* psi, int64_t ld, void* fpsi, void* spsi, void* grad) {
    return roks_gradient_parts(ctx, psi, ld, fpsi, spsi, grad, nullptr);
}

roks_status roks_gradient_parts(roks_ctx* ctx, const void* psi, int64_t ld, void* fpsi, void* spsi, void* grad,
                                void* grad_I) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    if (!fpsi) return fail(ctx, ROKS_EINVAL, "null output");
    const int64_t l = ctx->ld_min;
    const int nb = ctx->nb;
    void* S = spsi ? spsi : ((grad || grad_I) ? ctx->W_S : nullptr);
    const int64_t lds = spsi ? ld : l;
    if (ctx->prec == ROKS_FP64) r = Impl<double>::apply(ctx, psi, ld, fpsi, ld, S, lds);
    else r = Impl<float>::apply(ctx, psi, ld, fpsi, ld, S, lds);
    if (r != ROKS_OK || !(grad || grad_I)) return r;
    // theta = Psi^H F Psi; g = F - S Gam, Gam_mn = (theta_mn + conj theta_nm) / 2; g_I = F - S theta
    if (ctx->prec == ROKS_FP64) {
        gemm_cn<double>(nb, nb, ctx->npw, static_cast<const double2*>(psi), ld, static_cast<const double2*>(fpsi), ld,
                        ctx->d_Th, nb, ctx->d_gemm_work, ctx->gemm_work_elems, ctx->st);
    } else {
        gemm_cn<float>(nb, nb, ctx->npw, static_cast<const float2*>(psi), ld, static_cast<const float2*>(fpsi), ld,
                       ctx->d_Th, nb, ctx->d_gemm_work, ctx->gemm_work_elems, ctx->st);
    }
    if (ctx->gamma) gamma_real_part(nb, nb, ctx->d_Th, nb, ctx->st);
    const size_t es = ctx->prec == ROKS_FP64 ? sizeof(double2) : sizeof(float2);
    for (int part = 0; part < 2; ++part) {
        void* out = part == 0 ? grad : grad_I;
        if (!out) continue;
        const double2* M = ctx->d_Th;
        if (part == 0) {
            CK(cudaMemcpyAsync(ctx->d_Gam, ctx->d_Th, sizeof(double2) * nb * nb, cudaMemcpyDeviceToDevice, ctx->st));
            // the energy's operator of an empty band is F^e = 0
            if (ctx->ne > 0)
                CK(cudaMemsetAsync(ctx->d_Gam + (int64_t)ctx->nocc * nb, 0, sizeof(double2) * nb * ctx->ne, ctx->st));
            hermitize(nb, ctx->d_Gam, ctx->st);
            M = ctx->d_Gam;
        }
        CK(cudaMemcpy2DAsync(out, ld * es, fpsi, ld * es, ctx->npw * es, nb, cudaMemcpyDeviceToDevice, ctx->st));
        if (part == 0 && ctx->ne > 0)
            CK(cudaMemset2DAsync(static_cast<char*>(out) + (size_t)ctx->nocc * ld * es, ld * es, 0, ctx->npw * es,
                                 ctx->ne, ctx->st));
        if (ctx->prec == ROKS_FP64)
            gemm_nn<double>(ctx->npw, nb, nb, static_cast<const double2*>(S), lds, M, nb, static_cast<double2*>(out),
                            ld, -1.0, 1.0, ctx->d_gemm_work, ctx->st, ctx->gemm_work_elems * sizeof(double2));
        else
            gemm_nn<float>(ctx->npw, nb, nb, static_cast<const float2*>(S), lds, M, nb, static_cast<float2*>(out), ld,
                           -1.0, 1.0, ctx->d_gemm_work, ctx->st, ctx->gemm_work_elems * sizeof(double2));
    }
    CK(cudaGetLastError());
    return ROKS_OK;
}

roks_status roks_orthonormalize(roks_ctx* ctx, void* psi, int64_t ld) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    const int64_t l = ctx->ld_min;
    const size_t es = ctx->prec == ROKS_FP64 ? sizeof(double2) : sizeof(float2);
    CK(cudaMemcpy2DAsync(ctx->W_Y, l * es, psi, ld * es, ctx->npw * es, ctx->nb, cudaMemcpyDeviceToDevice, ctx->st));
    r = ctx->prec == ROKS_FP64 ? Impl<double>::orth(ctx, ctx->W_Y, l, psi, ld, nullptr)
                               : Impl<float>::orth(ctx, ctx->W_Y, l, psi, ld, nullptr);
    if (r != ROKS_OK) return r;
    reset_history(ctx);
    return ctx->prec == ROKS_FP64 ? Impl<double>::check_flag(ctx) : Impl<float>::check_flag(ctx);
}

roks_status roks_pcg_step(roks_ctx* ctx, void* psi, int64_t ld, roks_step_info* info) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    // after DIIS steps the direction history belongs to other orbitals
    if (ctx->pcg_fresh) reset_history(ctx);
    ctx->diis_count = 0;
    roks_step_info tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    r = ctx->prec == ROKS_FP64 ? Impl<double>::pcg_step(ctx, psi, ld, &tmp) : Impl<float>::pcg_step(ctx, psi, ld, &tmp);
    if (r != ROKS_OK) {
        if (info) *info = tmp;
        return r;
    }
    ctx->steps += 1;
    // convergence: |E_new - E| < e_tol on two consecutive steps, and the
    // gradient norm below g_tol when one is set
    if (std::fabs(tmp.E_new - tmp.E) < ctx->e_tol) ctx->n_small += 1;
    else ctx->n_small = 0;
    tmp.converged = (ctx->n_small >= 2 && (ctx->g_tol <= 0 || tmp.grad_norm < ctx->g_tol)) ? 1 : 0;
    if (tmp.converged && ctx->mlp_kind == ROKS_PRECOND_TPA_MLP && !ctx->mlp_judging) {
        // TPA judges the convergence of the corrected run: switch the
        // correction off for good (a device flag the captured step reads) and
        // require the criterion again with TPA steps
        const double off = 1e30;
        const size_t at = offsetof(PcgScalars, mlp_off);
        CK(cudaMemcpyAsync(reinterpret_cast<char*>(ctx->d_sc) + at, &off, sizeof(double), cudaMemcpyHostToDevice,
                           ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
        ctx->mlp_judging = true;
        ctx->n_small = 0;
        tmp.converged = 0;
    }
    if (info) *info = tmp;
    if (!tmp.converged && ctx->max_iter > 0 && ctx->steps >= ctx->max_iter)
        return fail(ctx, ROKS_ENOCONV, "no convergence within max_iter steps");
    return ROKS_OK;
}

roks_status roks_diis_step(roks_ctx* ctx, void* psi, int64_t ld, const roks_diis_options* opt,
                           roks_diis_info* info) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    if (ctx->ne > 0) return fail(ctx, ROKS_EINVAL, "the DIIS solver takes occupied bands only (no empty shell)");
    roks_diis_options o;
    if (opt) {
        o = *opt;
    } else {
        o.history = 6;
        o.tau = 0.5;
        o.lambda_ab = 0.5;
        o.lambda_ba = 0.5;
    }
    if (o.history < 1 || o.history > ROKS_DIIS_MAX || !(o.tau > 0.0) || !std::isfinite(o.tau) ||
        !std::isfinite(o.lambda_ab) || !std::isfinite(o.lambda_ba))
        return fail(ctx, ROKS_EINVAL, "DIIS options out of range (history 1..8, tau > 0, finite lambdas)");
    const roks_diis_options& p = ctx->diis_opt;
    const bool same = ctx->diis_count > 0 && ctx->diis_psi == psi && ctx->diis_ld == ld &&
                      o.history == p.history && o.tau == p.tau && o.lambda_ab == p.lambda_ab &&
                      o.lambda_ba == p.lambda_ba;
    if (!same) {
        ctx->diis_count = 0;
        ctx->diis_small = 0;
    }
    ctx->diis_opt = o;
    ctx->diis_psi = psi;
    ctx->diis_ld = ld;
    if (!ctx->d_diis) {
        CK(dalloc(ctx, &ctx->d_diis, sizeof(DiisState)));
        CK(dalloc(ctx, &ctx->d_diis_part, sizeof(double) * kDiisMax * (size_t)diis_gram_blocks(ctx->npw, ctx->nb)));
        void* hp = nullptr;
        CK(cudaMallocHost(&hp, sizeof(DiisState)));
        ctx->h_diis = static_cast<DiisState*>(hp);
    }
    if (ctx->diis_slots < o.history) {
        if (ctx->diis_ring) {
            CK(cudaStreamSynchronize(ctx->st));
            for (auto& q : ctx->allocs)
                if (q == ctx->diis_ring) q = nullptr;
            cudaFree(ctx->diis_ring);
            ctx->diis_ring = nullptr;
            ctx->diis_slots = 0;
        }
        const size_t es = ctx->prec == ROKS_FP64 ? sizeof(double2) : sizeof(float2);
        if (dalloc(ctx, &ctx->diis_ring, es * (size_t)ctx->ld_min * ctx->nb * 2 * o.history) != cudaSuccess)
            return fail(ctx, ROKS_ENOMEM, "DIIS history ring");
        ctx->diis_slots = o.history;
    }
    roks_diis_info tmp;
    std::memset(&tmp, 0, sizeof(tmp));
    r = ctx->prec == ROKS_FP64 ? Impl<double>::diis_step(ctx, psi, ld, o, &tmp)
                               : Impl<float>::diis_step(ctx, psi, ld, o, &tmp);
    ctx->pcg_fresh = true;
    if (r != ROKS_OK) {
        if (info) *info = tmp;
        return r;
    }
    ctx->steps += 1;
    if (std::fabs(tmp.E_new - tmp.E) < ctx->e_tol) ctx->diis_small += 1;
    else ctx->diis_small = 0;
    tmp.converged = (ctx->diis_small >= 2 && (ctx->g_tol <= 0 || tmp.res_norm < ctx->g_tol)) ? 1 : 0;
    if (info) *info = tmp;
    if (!tmp.converged && ctx->max_iter > 0 && ctx->steps >= ctx->max_iter)
        return fail(ctx, ROKS_ENOCONV, "no convergence within max_iter steps");
    return ROKS_OK;
}

roks_status roks_forces(roks_ctx* ctx, const void* psi, int64_t ld, double* forces_host) {
    if (!ctx) return ROKS_EINVAL;
    roks_status r = check_psi(ctx, psi, ld);
    if (r != ROKS_OK) return r;
    enter(ctx);
    if (!forces_host) return fail(ctx, ROKS_EINVAL, "null force array");
    if (ctx->natoms == 0) return ROKS_OK;
    const bool f64 = ctx->prec == ROKS_FP64;
    if (!ctx->d_forces) {
        const size_t cs = f64 ? sizeof(double2) : sizeof(float2);
        const size_t rs = f64 ? sizeof(double) : sizeof(float);
        const int na = ctx->natoms, np_ = ctx->nproj, nb = ctx->nb;
        cudaError_t e = cudaSuccess;
        auto al = [&](auto** p, size_t bytes) {
            if (e == cudaSuccess) e = dalloc(ctx, p, bytes);
        };
        al(&ctx->d_proj_atom, sizeof(int) * (np_ + 1));
        al(&ctx->d_fdP, cs * (size_t)ctx->ld_min * (np_ > 0 ? np_ : 1));
        al(&ctx->d_fdB, sizeof(double2) * 3 * (size_t)(np_ > 0 ? np_ : 1) * nb);
        al(&ctx->d_fY, sizeof(double2) * (size_t)(np_ > 0 ? np_ : 1) * nb);
        al(&ctx->d_fc, sizeof(double) * 3 * (np_ + 1));
        al(&ctx->d_ftab, cs * (size_t)na * 3 * ctx->N);
        al(&ctx->d_famp, rs * na);
        al(&ctx->d_fw2h, rs * na);
        al(&ctx->d_fpart, sizeof(double) * (size_t)na * 3 * kForceLocBlocks);
        al(&ctx->d_forces, sizeof(double) * 3 * na);
        if (e != cudaSuccess) return fail(ctx, ROKS_ENOMEM, "force workspaces");
        // per atom: amplitude -d (2 pi w^2)^{3/2} / Omega and w^2 / 2 of the well
        std::vector<double> amp(na), w2h(na);
        for (int a = 0; a < na; ++a) {
            const double d = ctx->atoms_h[5 * a + 3], w = ctx->atoms_h[5 * a + 4];
            amp[a] = -d * std::pow(2.0 * M_PI * w * w, 1.5) / ctx->omega;
            w2h[a] = 0.5 * w * w;
        }
        if (f64) {
            CK(cudaMemcpyAsync(ctx->d_famp, amp.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(ctx->d_fw2h, w2h.data(), sizeof(double) * na, cudaMemcpyHostToDevice, ctx->st));
        } else {
            std::vector<float> a32(amp.begin(), amp.end()), w32(w2h.begin(), w2h.end());
            CK(cudaMemcpyAsync(ctx->d_famp, a32.data(), sizeof(float) * na, cudaMemcpyHostToDevice, ctx->st));
            CK(cudaMemcpyAsync(ctx->d_fw2h, w32.data(), sizeof(float) * na, cudaMemcpyHostToDevice, ctx->st));
        }
        if (np_ > 0)
            CK(cudaMemcpyAsync(ctx->d_proj_atom, ctx->proj_atom_h.data(), sizeof(int) * np_, cudaMemcpyHostToDevice,
                               ctx->st));
        CK(cudaStreamSynchronize(ctx->st));
    }
    return f64 ? Impl<double>::forces(ctx, psi, ld, forces_host) : Impl<float>::forces(ctx, psi, ld, forces_host);
}

roks_status roks_profile_enable(roks_ctx* ctx, int enable) {
    if (!ctx) return ROKS_EINVAL;
    ctx->prof_on = enable != 0;
    if (ctx->prof_on) launches_take();
    return ROKS_OK;
}

roks_status roks_profile_read(roks_ctx* ctx, roks_profile_entry* out, int cap, int* count) {
    if (!ctx || cap < 0 || (cap > 0 && !out)) return ROKS_EINVAL;
    CK(cudaStreamSynchronize(ctx->st));
    const size_t nf = ctx->prof_names.size();
    std::vector<double> ms(nf, 0.0);
    std::vector<int> cnt(nf, 0);
    for (const auto& r : ctx->prof_recs) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            ms[r.fam] += t;
            cnt[r.fam] += 1;
        }
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_recs.clear();
    const long long kernels = launches_take();
    int n = 0;
    for (size_t f = 0; f < nf; ++f) {
        if (cnt[f] == 0) continue;
        if (n < cap) {
            std::memset(out[n].name, 0, sizeof(out[n].name));
            std::strncpy(out[n].name, ctx->prof_names[f].c_str(), sizeof(out[n].name) - 1);
            out[n].launches = cnt[f];
            out[n].ms = ms[f];
        }
        ++n;
    }
    if (n < cap) {
        std::memset(out[n].name, 0, sizeof(out[n].name));
        std::strncpy(out[n].name, "kernel_launches", sizeof(out[n].name) - 1);
        out[n].launches = (int)kernels;
        out[n].ms = 0.0;
    }
    ++n;
    const long long tensor = tcg_launches_take();
    if (n < cap) {
        std::memset(out[n].name, 0, sizeof(out[n].name));
        std::strncpy(out[n].name, "tensor_core_launches", sizeof(out[n].name) - 1);
        out[n].launches = (int)tensor;
        out[n].ms = 0.0;
    }
    ++n;
    if (count) *count = n;
    return ROKS_OK;
}

roks_status roks_mlp_forward(int n, const float* feats, const float* params, int bf16, float* s, void* stream) {
    if (n < 0 || (n > 0 && (!feats || !params || !s))) return ROKS_EINVAL;
    mlp_forward(n, feats, params, bf16 != 0, s, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? ROKS_OK : ROKS_ECUDA;
}

size_t roks_mlp_grad_work(int n) { return n > 0 ? mlp_grad_work_floats(n) : 0; }

roks_status roks_mlp_grad(int n, const float* feats, const float* target, const float* weight, const float* params,
                          float* work, float* grad, float* loss, void* stream) {
    if (n <= 0 || !feats || !target || !weight || !params || !work || !grad) return ROKS_EINVAL;
    mlp_grad(n, feats, target, weight, params, work, grad, loss, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? ROKS_OK : ROKS_ECUDA;
}

roks_status roks_mlp_adam(float* params, float* m, float* v, const float* grad, int step, float lr, float beta1,
                          float beta2, float eps, void* stream) {
    if (!params || !m || !v || !grad || step < 1 || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f))
        return ROKS_EINVAL;
    mlp_adam(params, m, v, grad, step, lr, beta1, beta2, eps, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? ROKS_OK : ROKS_ECUDA;
}

roks_status roks_set_preconditioner(roks_ctx* ctx, int kind, const float* params) {
    if (!ctx) return ROKS_EINVAL;
    if (kind != ROKS_PRECOND_TPA && kind != ROKS_PRECOND_TPA_MLP)
        return fail(ctx, ROKS_EINVAL, "unknown preconditioner kind");
    if (kind == ROKS_PRECOND_TPA_MLP) {
        if (!params) return fail(ctx, ROKS_EINVAL, "null network parameters");
        CK(cudaMemcpyAsync(ctx->d_mlp, params, sizeof(float) * ROKS_MLP_PARAMS, cudaMemcpyDeviceToDevice, ctx->st));
    }
    if (kind != ctx->mlp_kind && ctx->pcg_exec) {
        // the captured iteration launches the other preconditioner: capture again
        CK(cudaStreamSynchronize(ctx->st));
        cudaGraphExecDestroy(ctx->pcg_exec);
        ctx->pcg_exec = nullptr;
        ctx->graph_psi = nullptr;
    }
    ctx->mlp_kind = kind;
    return ROKS_OK;
}

roks_status roks_precondition(roks_ctx* ctx, const void* grad, int64_t ld, void* out, float* feats) {
    if (!ctx) return ROKS_EINVAL;
    if (!grad || !out || ld < ctx->npw) return fail(ctx, ROKS_EINVAL, "bad gradient or output");
    const int npw = ctx->npw, nb = ctx->nb;
    cudaStream_t st = ctx->st;
    if (ctx->prec == ROKS_FP64) {
        using T = double;
        const auto* g = static_cast<const double2*>(grad);
        column_sums<T>(1, npw, nb, g, ld, nullptr, 0, static_cast<const T*>(ctx->d_g2half), ctx->d_colpart,
                       ctx->d_colout, st);
        if (feats) mlp_features<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, ctx->d_Th,
                                   ctx->d_wband, feats, st);
        if (ctx->mlp_kind == ROKS_PRECOND_TPA_MLP)
            precondition_mlp<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, ctx->d_Th,
                                ctx->d_wband, ctx->d_mlp, nullptr, static_cast<double2*>(out), ld, st);
        else
            precondition<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout,
                            static_cast<double2*>(out), ld, st);
    } else {
        using T = float;
        const auto* g = static_cast<const float2*>(grad);
        column_sums<T>(1, npw, nb, g, ld, nullptr, 0, static_cast<const T*>(ctx->d_g2half), ctx->d_colpart,
                       ctx->d_colout, st);
        if (feats) mlp_features<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, ctx->d_Th,
                                   ctx->d_wband, feats, st);
        if (ctx->mlp_kind == ROKS_PRECOND_TPA_MLP)
            precondition_mlp<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout, ctx->d_Th,
                                ctx->d_wband, ctx->d_mlp, nullptr, static_cast<float2*>(out), ld, st);
        else
            precondition<T>(npw, nb, g, ld, static_cast<const T*>(ctx->d_g2half), ctx->d_colout,
                            static_cast<float2*>(out), ld, st);
    }
    CK(cudaGetLastError());
    return ROKS_OK;
}

const char* roks_last_error(const roks_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void roks_destroy(roks_ctx* ctx) {
    if (!ctx) return;
    if (ctx->st) cudaStreamSynchronize(ctx->st);
    else cudaDeviceSynchronize();
    if (ctx->pcg_exec) cudaGraphExecDestroy(ctx->pcg_exec);
    if (ctx->d_Psplit_nn) tcg_presplit_forget(ctx->d_Psplit_nn);
    if (ctx->h_sc) cudaFreeHost(ctx->h_sc);
    if (ctx->h_diis) cudaFreeHost(ctx->h_diis);
    if (ctx->cap_st) cudaStreamDestroy(ctx->cap_st);
    if (ctx->side_st) cudaStreamDestroy(ctx->side_st);
    if (ctx->fork_ev) cudaEventDestroy(ctx->fork_ev);
    if (ctx->join_ev) cudaEventDestroy(ctx->join_ev);
    for (void* p : ctx->allocs) cudaFree(p);
    for (const auto& r : ctx->prof_recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    delete ctx;
}

}  // extern "C"
