// k_pcg.cu -- band-space part of one PCG iteration, kept on the device so
// that a step needs no host round trip: gamma and the gradient split
// (Eqs. 11, 12), the ROKS R matrix (Eq. 20), the rotation generator
// (Eqs. 22-23), the Fletcher-Reeves ratio (Eq. 6) with restarts, the
// parabolic line search (Eq. 5) and the energy combination (Eq. 1).
#include <cstddef>

#include "roks_grid.cuh"

namespace roks {

// Gam_mn = gamma_nm = (theta_mn + conj theta_nm)/2; Gin_mn = theta_mn - conj theta_nm;
// R_mn: same shell theta_mn; shell(m) < shell(n): conj theta_nm - theta_mn;
// shell(m) > shell(n): theta_mn - conj theta_nm; a-b zeroed when suppressed.
// A_mn = -(1/2) atan2(2|R|, |d_m - d_n|) sgn(d_m - d_n) R/|R| for m < n,
// A_nm = -conj A_mn (|R| < 1e-14 -> 0).
// d_m = <m|F^c|m>.  Closed bands: Re theta_mm.  Open bands:
// w_c (<m|T|m> + <m|V_nl|m>) + <m|V^c|m> with the local part from rho_m.
__device__ __forceinline__ double band_diag(int m, int nb, int n_closed, int n_occ, const double2* __restrict__ Th,
                                            const double* __restrict__ kin_b, const double* __restrict__ nl_b,
                                            const double* __restrict__ open_vc, const double* __restrict__ open_x,
                                            double wc) {
    // closed and empty bands: F^c was applied to them
    if (m < n_closed || m >= n_occ) return Th[(int64_t)m * nb + m].x;
    double v = wc * (kin_b[m] + nl_b[m]) + open_vc[m - n_closed];
    if (open_x) v += open_x[m - n_closed];
    return v;
}

// Gamma, the rotation gradient and A (Eqs. 11, 20-23) with the diagonal d
// formed per pair; block 0 also forms the a-b coupling of the open shells.
__global__ void k_pcg_rotation(int nb, int n_closed, const double2* __restrict__ Th, const double* __restrict__ kin_b,
                               const double* __restrict__ nl_b, const double* __restrict__ open_vc,
                               const double* __restrict__ open_x, double wc, const int* __restrict__ shell,
                               int suppress_ab, int ia, int ib, double2* __restrict__ Gam, double2* __restrict__ Gin,
                               double2* __restrict__ A, PcgScalars* sc, int n_occ, const double* __restrict__ dk) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx == 0) {
        if (ia < 0) {
            sc->coup_re = sc->coup_im = 0.0;
        } else {
            // <a|F^a - F^b|b> = conj(theta_ba) - theta_ab
            const double2 tab = Th[(int64_t)ib * nb + ia];
            const double2 tba = Th[(int64_t)ia * nb + ib];
            sc->coup_re = tba.x - tab.x;
            sc->coup_im = -tba.y - tab.y;
        }
    }
    if (idx >= nb * nb) return;
    const int m = idx % nb, n = idx / nb;
    const double2 z2 = make_double2(0.0, 0.0);
    // theta of the energy: <m|F^e|n> = 0 in the empty columns
    const double2 tmn = n < n_occ ? Th[(int64_t)n * nb + m] : z2;
    const double2 tnm = m < n_occ ? Th[(int64_t)m * nb + n] : z2;
    Gam[idx] = make_double2(0.5 * (tmn.x + tnm.x), 0.5 * (tmn.y - tnm.y));
    Gin[idx] = make_double2(tmn.x - tnm.x, tmn.y + tnm.y);
    double2 a = z2;
    if (m != n) {
        // the element of the upper triangle that defines this pair
        const int p = m < n ? m : n, q = m < n ? n : m;
        const double2 tpq = q < n_occ ? Th[(int64_t)q * nb + p] : z2;
        const double2 tqp = p < n_occ ? Th[(int64_t)p * nb + q] : z2;
        double2 r;
        if (shell[p] == shell[q]) r = Th[(int64_t)q * nb + p];   // same shell (the empty one: F^c)
        else if (shell[p] < shell[q]) r = make_double2(tqp.x - tpq.x, -tqp.y - tpq.y);
        else r = make_double2(tpq.x - tqp.x, tpq.y + tqp.y);
        if (suppress_ab && ((p == ia && q == ib) || (p == ib && q == ia))) r = make_double2(0.0, 0.0);
        const double ar = sqrt(r.x * r.x + r.y * r.y);
        if (ar >= 1e-14) {
            double2 apq;
            if (p < n_occ && q >= n_occ) {
                // occupied p of class k, empty q: p to the lower state of F^k
                const int k = p < n_closed ? 0 : p - n_closed + 1;
                const double gap = dk[k * (nb - n_occ) + (q - n_occ)] - Th[(int64_t)p * nb + p].x;
                const double phi = 0.5 * atan2(2.0 * ar, gap);
                apq = make_double2(phi * r.x / ar, phi * r.y / ar);
            } else {
                const double dd = band_diag(p, nb, n_closed, n_occ, Th, kin_b, nl_b, open_vc, open_x, wc) -
                                  band_diag(q, nb, n_closed, n_occ, Th, kin_b, nl_b, open_vc, open_x, wc);
                const double sg = dd >= 0.0 ? 1.0 : -1.0;
                const double phi = 0.5 * atan2(2.0 * ar, fabs(dd));
                apq = make_double2(-phi * sg * r.x / ar, -phi * sg * r.y / ar);
            }
            a = (m == p) ? apq : make_double2(-apq.x, apq.y);
        }
    }
    A[idx] = a;
}

void pcg_rotation(int nb, int n_closed, const double2* Theta, const double* kin_b, const double* nl_b,
                  const double* open_vc, const double* open_x, double wc, const int* shell, int suppress_ab, int ia,
                  int ib, double2* Gam, double2* Gin, double2* A, PcgScalars* sc, cudaStream_t st, int n_occ,
                  const double* dk) {
    roks::count_launch(), k_pcg_rotation<<<(nb * nb + 127) / 128, 128, 0, st>>>(
                              nb, n_closed, Theta, kin_b, nl_b, open_vc, open_x, wc, shell, suppress_ab, ia, ib, Gam,
                              Gin, A, sc, n_occ, dk);
}

// Empty bands: block partial sums of dvol V^k rho_e (grid-stride, one block
// row per (band, class)), then the fixed-order total plus the
// kinetic/non-local part.
template <typename T>
__global__ void k_empty_vexp(int64_t N3, int n_empty, const typename DensAcc<T>::S* __restrict__ rho_e,
                             const T* __restrict__ Vk, double* __restrict__ part) {
    using DA = DensAcc<T>;
    __shared__ double red[256];
    const int i = blockIdx.y % n_empty, k = blockIdx.y / n_empty;
    const typename DA::S* r = rho_e + (int64_t)(i + 1) * N3;
    const T* v = Vk + (int64_t)k * N3;
    double acc = 0.0;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < N3; p += (int64_t)gridDim.x * blockDim.x)
        acc += double(v[p]) * double(DA::value(r[p]));
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

__global__ void k_empty_diag_final(int nblk, int n_empty, int n_occ, const double* __restrict__ part, double dvol,
                                   const double* __restrict__ kin_b, const double* __restrict__ nl_b, double w0,
                                   double w1, double w2, double* __restrict__ dk) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 3 * n_empty) return;
    const int i = j % n_empty, k = j / n_empty;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)j * nblk + b];
    const int e = n_occ + i;
    const double w = k == 0 ? w0 : (k == 1 ? w1 : w2);
    dk[j] = w * (kin_b[e] + nl_b[e]) + dvol * s;
}

template <typename T>
void empty_band_diagonal(int64_t N3, int n_empty, int n_occ, const double* rho_e, const T* Vk, double dvol,
                         const double* kin_b, const double* nl_b, double w0, double w1, double w2, double* part,
                         double* dk, cudaStream_t st) {
    if (n_empty <= 0) return;
    constexpr int kBlk = 64;
    using DS = typename DensAcc<T>::S;
    roks::count_launch(), k_empty_vexp<T><<<dim3(kBlk, 3 * n_empty), 256, 0, st>>>(
                              N3, n_empty, reinterpret_cast<const DS*>(rho_e), Vk, part);
    roks::count_launch(), k_empty_diag_final<<<(3 * n_empty + 127) / 128, 128, 0, st>>>(kBlk, n_empty, n_occ, part,
                                                                                        dvol, kin_b, nl_b, w0, w1, w2,
                                                                                        dk);
}
template void empty_band_diagonal<float>(int64_t, int, int, const double*, const float*, double, const double*,
                                         const double*, double, double, double, double*, double*, cudaStream_t);
template void empty_band_diagonal<double>(int64_t, int, int, const double*, const double*, double, const double*,
                                          const double*, double, double, double, double*, double*, cudaStream_t);

// r1 = Re <A, Gin>, r2 = Re <A_prev, Gin> (sums over all n^2 elements).
// One block (up to 64 bands), or block partials of a grid-stride sum and a
// fixed-order final sum (larger n: the FP64 chains of one block take
// hundreds of microseconds at a few hundred bands).
__global__ void k_pcg_rot_dots(int nb, const double2* __restrict__ A, const double2* __restrict__ Ap,
                               const double2* __restrict__ Gin, double* __restrict__ part, PcgScalars* sc) {
    __shared__ double s1[256], s2[256];
    double r1 = 0, r2 = 0;
    const int64_t n2 = (int64_t)nb * nb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += (int64_t)gridDim.x * blockDim.x) {
        const double2 g = Gin[i], a = A[i], p = Ap[i];
        r1 += a.x * g.x + a.y * g.y;
        r2 += p.x * g.x + p.y * g.y;
    }
    s1[threadIdx.x] = r1;
    s2[threadIdx.x] = r2;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (gridDim.x == 1) {
            sc->r1 = s1[0];
            sc->r2 = s2[0];
            sc->rot_pg = 0.5 * s1[0];
        } else {
            part[2 * blockIdx.x] = s1[0];
            part[2 * blockIdx.x + 1] = s2[0];
        }
    }
}

__global__ void k_pcg_rot_dots_final(int nblk, const double* __restrict__ part, PcgScalars* sc) {
    if (threadIdx.x != 0) return;
    double r1 = 0, r2 = 0;
    for (int b = 0; b < nblk; ++b) {
        r1 += part[2 * b];
        r2 += part[2 * b + 1];
    }
    sc->r1 = r1;
    sc->r2 = r2;
    sc->rot_pg = 0.5 * r1;
}

void pcg_rot_dots(int nb, const double2* A, const double2* Aprev, const double2* Gin, double* part, PcgScalars* sc,
                  cudaStream_t st) {
    if (nb <= 64) {
        roks::count_launch(), k_pcg_rot_dots<<<1, 256, 0, st>>>(nb, A, Aprev, Gin, part, sc);
        return;
    }
    // part holds at least 2 x 16 x nb doubles (the column-sum partials): 2 nblk fit
    int nblk = (nb * nb + 2047) / 2048;
    if (nblk > 152) nblk = 152;
    roks::count_launch(), k_pcg_rot_dots<<<nblk, 256, 0, st>>>(nb, A, Aprev, Gin, part, sc);
    roks::count_launch(), k_pcg_rot_dots_final<<<1, 32, 0, st>>>(nblk, part, sc);
}

// beta = pg / pg_prev; dE(beta) = 2 a1 + 2 beta a2 + r1 + beta r2.
// Not descent with beta != 0: restart (beta = 0).  Still not descent: drop
// the rotation.
__global__ void k_pcg_direction(PcgScalars* sc) {
    if (threadIdx.x != 0) return;
    sc->pg = sc->pgI + sc->rot_pg;
    double beta = (sc->has_prev != 0.0) ? sc->pg / sc->pg_prev : 0.0;
    double dE = 2.0 * sc->a1 + 2.0 * beta * sc->a2 + sc->r1 + beta * sc->r2;
    double rot = 1.0, restarted = 0.0;
    if (dE >= 0.0 && beta != 0.0) {
        beta = 0.0;
        restarted = 1.0;
        dE = 2.0 * sc->a1 + sc->r1;
    }
    if (dE >= 0.0) {
        rot = 0.0;
        restarted = 1.0;
        dE = 2.0 * sc->a1 + 2.0 * beta * sc->a2;
    }
    sc->beta = beta;
    sc->dE0 = dE;
    sc->rot = rot;
    sc->restarted = restarted;
}

void pcg_direction(PcgScalars* sc, cudaStream_t st) { roks::count_launch(), k_pcg_direction<<<1, 32, 0, st>>>(sc); }

__global__ void k_pcg_total_rotation(int nb, const double2* __restrict__ A, const double2* __restrict__ Ap,
                                     const PcgScalars* __restrict__ sc, double2* __restrict__ At) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb * nb) return;
    const double r = sc->rot, b = sc->beta;
    const double2 a = A[i], p = Ap[i];
    At[i] = make_double2(r * (a.x + b * p.x), r * (a.y + b * p.y));
}

void pcg_total_rotation(int nb, const double2* A, const double2* Aprev, PcgScalars* sc, double2* Atot,
                        cudaStream_t st) {
    roks::count_launch(), k_pcg_total_rotation<<<(nb * nb + 127) / 128, 128, 0, st>>>(nb, A, Aprev, sc, Atot);
}

// Parabola E(x) = E0 + dE0 x + c x^2 through E(dt) = Et; c > 0 gives the
// minimum -dE0/(2c), otherwise the trial step is kept; capped at 3 dt.
__global__ void k_pcg_line_search(PcgScalars* sc) {
    if (threadIdx.x != 0) return;
    const double dt = sc->dt;
    const double c = (sc->Et - sc->E0 - sc->dE0 * dt) / (dt * dt);
    double step = c > 0.0 ? -sc->dE0 / (2.0 * c) : dt;
    step = fmin(step, 3.0 * dt);
    sc->step = step;
}

void pcg_line_search(PcgScalars* sc, cudaStream_t st) { roks::count_launch(), k_pcg_line_search<<<1, 32, 0, st>>>(sc); }

// After the step: next trial step, history.
__global__ void k_pcg_finish(PcgScalars* sc) {
    if (threadIdx.x != 0) return;
    sc->dt = fmin(fmax(sc->step, 0.05), 2.0);
    sc->pg_prev = sc->pg;
    sc->has_prev = 1.0;
    // TPA stays the fallback of the learned correction: an accepted step that
    // raised the energy, or a CG restart, suspends it for three iterations
    if (sc->Enew > sc->E0 || sc->restarted != 0.0) sc->mlp_off = 3.0;
    else sc->mlp_off = fmax(sc->mlp_off - 1.0, 0.0);
}

__global__ void k_set_cur(PcgScalars* sc, int field) {
    if (threadIdx.x == 0) sc->cur = reinterpret_cast<double*>(sc)[field];
}

void pcg_set_cur(PcgScalars* sc, int field, cudaStream_t st) { roks::count_launch(), k_set_cur<<<1, 32, 0, st>>>(sc, field); }

void pcg_finish(PcgScalars* sc, cudaStream_t st) { roks::count_launch(), k_pcg_finish<<<1, 32, 0, st>>>(sc); }

// E[0..10] = kin, loc, nl, H, xM, xT, hfM, hfT, M, T, total
__global__ void k_energy_combine(const double* __restrict__ kin_b, const double* __restrict__ nl_b, int nb,
                                 const double* __restrict__ wband, const double* __restrict__ out6, double cM,
                                 double cT, double alpha, const double* __restrict__ hf2, double* __restrict__ E) {
    // band sums: lane l takes bands l, l + 32, ..., then a fixed shuffle tree
    // (FP64 adds are long-latency: few dependent levels)
    const int lane = threadIdx.x;
    double kin = 0, nl = 0;
    for (int n = lane; n < nb; n += 32) {
        kin += wband[n] * kin_b[n];
        nl += wband[n] * nl_b[n];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        kin += __shfl_xor_sync(0xffffffffu, kin, o);
        nl += __shfl_xor_sync(0xffffffffu, nl, o);
    }
    if (lane != 0) return;
    const double loc = out6[2], H = out6[3], xM = out6[0], xT = out6[1];
    const double hfM = hf2 ? hf2[0] : 0.0, hfT = hf2 ? hf2[1] : 0.0;
    const double one = kin + loc + nl + H;
    const double M = one + xM + alpha * hfM;
    const double T = one + xT + alpha * hfT;
    E[0] = kin; E[1] = loc; E[2] = nl; E[3] = H; E[4] = xM; E[5] = xT; E[6] = hfM; E[7] = hfT;
    E[8] = M; E[9] = T; E[10] = cM * M + cT * T;
}

void energy_combine(const double* kin_b, const double* nl_b, int nb, const double* wband, const double* out6,
                    double cM, double cT, double alpha, const double* hf2, double* E, cudaStream_t st) {
    roks::count_launch(), k_energy_combine<<<1, 32, 0, st>>>(kin_b, nl_b, nb, wband, out6, cM, cT, alpha, hf2, E);
}

__global__ void k_take_energy(const double* __restrict__ E, PcgScalars* sc, int field) {
    if (threadIdx.x == 0) reinterpret_cast<double*>(sc)[field] = E[10];
}

void pcg_take_energy(const double* E, PcgScalars* sc, int field, cudaStream_t st) {
    roks::count_launch(), k_take_energy<<<1, 32, 0, st>>>(E, sc, field);
}

__global__ void k_hermitize(int n, double2* O) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * n) return;
    const int m = idx % n, c = idx / n;
    if (m > c) return;
    const double2 a = O[(int64_t)c * n + m], b = O[(int64_t)m * n + c];
    const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
    O[(int64_t)c * n + m] = h;
    O[(int64_t)m * n + c] = make_double2(h.x, -h.y);
}

void hermitize(int n, double2* O, cudaStream_t st) { roks::count_launch(), k_hermitize<<<(n * n + 127) / 128, 128, 0, st>>>(n, O); }

// dst = scale * sum_i v[i]: lane l sums v[l], v[l + 32], ..., then a fixed
// shuffle tree (FP64 adds are long-latency: few dependent levels)
__global__ void k_sum_to(const double* __restrict__ v, int n, double* dst, double scale) {
    const int lane = threadIdx.x;
    double s = 0;
    for (int i = lane; i < n; i += 32) s += v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) dst[0] = scale * s;
}

void sum_to(const double* v, int n, double* dst, double scale, cudaStream_t st) {
    roks::count_launch(), k_sum_to<<<1, 32, 0, st>>>(v, n, dst, scale);
}

}  // namespace roks
