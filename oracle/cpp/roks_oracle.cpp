// roks_oracle.cpp -- plain FP64 C++ oracle of the ROKS plane-wave apply
// path (TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and the
// CPU-baseline legs of bench.py load it; the library never does).
//
// A second, independent restatement of what the path computes, beside the
// NumPy oracle (oracle/roks.py): the same model, written out in C++ with a
// textbook recursive mixed-radix FFT and OpenMP over bands.  It shares no
// code with the CUDA path and none with the NumPy oracle; tests check the two
// oracles against each other (tests/test_oracle_cpp.py).
//
// What it computes (paper notation):
//   * plane-wave basis: Miller triples with (2 pi / L)^2 |m|^2 / 2 <= Ecut,
//     tested in integers, loops i, j, k ascending (full sphere, Gamma point);
//   * orbitals on the grid psi(r) = Omega^{-1/2} sum_G c_G e^{iG.r} and the
//     class densities rho_k = sum_{n in k} |psi_n|^2 (closed, a, b);
//   * channel densities rho^{sigma L} = sum_k f_k^{sigma L} rho_k, one
//     Hartree solve (rho_M = rho_T), Slater exchange per channel scaled by
//     (1 - alpha), class potentials V^k = w_k (V_loc + V_H) + sum c_L f_k v_x
//     (Eqs. 8, 13);
//   * F^k|n> = w_k (T + V_nl)|n> + V^k psi_n, S|n> = |n> + sum |p_i> Q_ij
//     <p_j|n> (Eqs. 3, 13), with Gaussian wells for V_loc and Gaussian s/p
//     projectors (the model that stands in for the paper's PAW sets).
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <vector>

#ifdef _OPENMP
#include <omp.h>
#endif

namespace {

using cd = std::complex<double>;
constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- FFT
// Unnormalised DFT X[k] = sum_n x[n] exp(sign 2 pi i n k / n_len), by the
// textbook recursive Cooley-Tukey split on the smallest prime factor p of
// the length: p interleaved sub-sequences transformed recursively, then
// combined with twiddles by a direct p-point DFT.
struct Fft1 {
    int N = 0;
    std::vector<cd> w;   // w[t] = exp(+2 pi i t / N); the forward sign conjugates

    explicit Fft1(int n) : N(n), w(n) {
        for (int t = 0; t < n; ++t) w[t] = std::polar(1.0, 2.0 * kPi * t / n);
    }
    static int smallest_factor(int n) {
        for (int p = 2; p * p <= n; ++p)
            if (n % p == 0) return p;
        return n;
    }
    // out[k * os] for k < n from in[j * is] for j < n; scratch holds >= 3 n
    // (this level's twiddles exp(sign 2 pi i t / n), t < n, then the
    // sub-transforms and the deeper levels' scratch)
    void rec(const cd* in, int is, cd* out, int os, int n, int sign, cd* scratch) const {
        if (n == 1) {
            out[0] = in[0];
            return;
        }
        cd* wn = scratch;
        const int step = N / n;
        for (int t = 0; t < n; ++t) wn[t] = sign > 0 ? w[(int64_t)t * step] : std::conj(w[(int64_t)t * step]);
        const int p = smallest_factor(n);
        const int m = n / p;
        if (m == 1) {
            // direct DFT of a prime length: exponent j k mod n kept incrementally
            for (int k = 0; k < n; ++k) {
                cd s = 0;
                int t = 0;
                for (int j = 0; j < n; ++j) {
                    s += in[(int64_t)j * is] * wn[t];
                    t += k;
                    if (t >= n) t -= n;
                }
                out[(int64_t)k * os] = s;
            }
            return;
        }
        // sub-sequence r (elements r, r + p, ...) transformed into y[r * m .. r * m + m)
        cd* y = scratch + n;
        cd* rest = scratch + 2 * n;
        for (int r = 0; r < p; ++r) rec(in + (int64_t)r * is, is * p, y + (int64_t)r * m, 1, m, sign, rest);
        // X[k] = sum_r exp(sign 2 pi i r k / n) Y_r[k mod m]
        for (int k = 0; k < n; ++k) {
            const int k1 = k % m;
            cd s = 0;
            int t = 0;
            for (int r = 0; r < p; ++r) {
                s += y[(int64_t)r * m + k1] * wn[t];
                t += k;
                if (t >= n) t -= n;
            }
            out[(int64_t)k * os] = s;
        }
    }
    // in-place transform of a contiguous line of length N
    void line(cd* a, int sign, cd* scratch) const {
        rec(a, 1, scratch, 1, N, sign, scratch + N);
        for (int j = 0; j < N; ++j) a[j] = scratch[j];
    }
    size_t scratch_size() const { return (size_t)8 * N + 64; }
};

// 3D transform of an N^3 grid (index (i N + j) N + k), lines along each
// axis.  Lines along j and i are gathered kB at a time (consecutive k), so
// that every row read from the grid is a run of kB neighbours.
void fft3(const Fft1& f, cd* g, int sign) {
    const int N = f.N;
    constexpr int kB = 8;
    std::vector<cd> scratch(f.scratch_size()), buf((size_t)kB * N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) f.line(g + ((int64_t)i * N + j) * N, sign, scratch.data());
    for (int pass = 0; pass < 2; ++pass) {
        // pass 0: lines along j (stride N) for each i; pass 1: along i (stride N^2) for each j
        const int64_t stride = pass == 0 ? N : (int64_t)N * N;
        for (int o = 0; o < N; ++o) {
            const int64_t base = pass == 0 ? (int64_t)o * N * N : (int64_t)o * N;
            for (int k0 = 0; k0 < N; k0 += kB) {
                const int nb = N - k0 < kB ? N - k0 : kB;
                for (int e = 0; e < N; ++e)
                    for (int b = 0; b < nb; ++b) buf[(size_t)b * N + e] = g[base + e * stride + k0 + b];
                for (int b = 0; b < nb; ++b) f.line(buf.data() + (size_t)b * N, sign, scratch.data());
                for (int e = 0; e < N; ++e)
                    for (int b = 0; b < nb; ++b) g[base + e * stride + k0 + b] = buf[(size_t)b * N + e];
            }
        }
    }
}

// ---------------------------------------------------------------- the model
// Occupations f_k^{sigma L} of the classes (closed, a, b) in the channels
// (up M, down M, up T, down T): the mixed configuration has a up and b down,
// the triplet a and b up (Fig. 1A, Eq. 7).
constexpr double kF[3][4] = {{1, 1, 1, 1}, {1, 0, 1, 0}, {0, 1, 1, 0}};

struct RoSys {
    double L = 0, omega = 0, ecut = 0, alpha = 0;
    int N = 0, npw = 0, nproj = 0, nb = 0, n_closed = 0, mode = 1;
    double cL[2] = {0, 0};             // c_M, c_T (Eq. 1)
    double C[3][4] = {};               // c_L f_k^{sigma L}
    double w[3] = {};                  // sum over channels of C[k]: weight of T, V_loc, V_H, V_nl in F^k
    std::vector<int32_t> miller;       // npw x 3
    std::vector<int64_t> gidx;         // grid index of each basis vector
    std::vector<double> g2;            // |G|^2 per basis vector
    std::vector<double> G2grid;        // |G|^2 on the grid (index N/2 taken as +N/2)
    std::vector<double> vloc;          // V_loc(r), real
    std::vector<cd> P;                 // npw x nproj, column major
    std::vector<double> D, Q;          // nproj x nproj, block diagonal (row major)
    Fft1* fft = nullptr;
};

int signed_index(int e, int N) { return e <= N / 2 ? e : e - N; }

// occupations and the basis
bool setup_basis(RoSys& s) {
    const double q = s.L / (2.0 * kPi);
    const long M = (long)std::floor(2.0 * s.ecut * q * q);
    long n = (long)std::floor(std::sqrt((double)M));
    while ((n + 1) * (n + 1) <= M) ++n;
    while (n * n > M) --n;
    if (s.N < 2 * n + 1) return false;
    const double b = 2.0 * kPi / s.L;
    for (long i = -n; i <= n; ++i)
        for (long j = -n; j <= n; ++j)
            for (long k = -n; k <= n; ++k) {
                if (i * i + j * j + k * k > M) continue;
                s.miller.push_back((int32_t)i);
                s.miller.push_back((int32_t)j);
                s.miller.push_back((int32_t)k);
                const long mi = (i % s.N + s.N) % s.N, mj = (j % s.N + s.N) % s.N, mk = (k % s.N + s.N) % s.N;
                s.gidx.push_back(((int64_t)mi * s.N + mj) * s.N + mk);
                s.g2.push_back(b * b * (double)(i * i + j * j + k * k));
            }
    s.npw = (int)(s.miller.size() / 3);
    const int N = s.N;
    s.G2grid.resize((size_t)N * N * N);
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            for (int k = 0; k < N; ++k) {
                const double gx = b * signed_index(i, N), gy = b * signed_index(j, N), gz = b * signed_index(k, N);
                s.G2grid[((size_t)i * N + j) * N + k] = gx * gx + gy * gy + gz * gz;
            }
    return true;
}

void setup_occupations(RoSys& s) {
    // c_L: singlet (2, -1); triplet (0, 1); closed-shell ground state (1, 0)
    s.cL[0] = s.mode == 1 ? 2.0 : (s.mode == 2 ? 0.0 : 1.0);
    s.cL[1] = s.mode == 1 ? -1.0 : (s.mode == 2 ? 1.0 : 0.0);
    for (int k = 0; k < 3; ++k) {
        s.w[k] = 0;
        for (int ch = 0; ch < 4; ++ch) {
            s.C[k][ch] = s.cL[ch / 2] * kF[k][ch];
            s.w[k] += s.C[k][ch];
        }
    }
}

// Gaussian wells: V(G) = -(1/Omega) sum_a d_a (2 pi w^2)^{3/2} exp(-|G|^2 w^2 / 2)
// exp(-i G.R_a) on every grid vector except the Nyquist planes (left out so
// that V(r) is real), then V(r) = sum_G V(G) e^{iG.r}.
void setup_vloc(RoSys& s, int natoms, const double* pos, const double* depth, const double* width) {
    const int N = s.N;
    const double b = 2.0 * kPi / s.L;
    std::vector<cd> V((size_t)N * N * N, cd(0, 0));
    for (int a = 0; a < natoms; ++a) {
        const double d = depth[a], wd = width[a];
        const double pref = -d * std::pow(2.0 * kPi * wd * wd, 1.5) / s.omega;
        std::vector<cd> ph[3];
        for (int c = 0; c < 3; ++c) {
            ph[c].resize(N);
            for (int e = 0; e < N; ++e) ph[c][e] = std::polar(1.0, -b * signed_index(e, N) * pos[3 * a + c]);
        }
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j)
                for (int k = 0; k < N; ++k) {
                    const size_t g = ((size_t)i * N + j) * N + k;
                    V[g] += pref * std::exp(-0.5 * s.G2grid[g] * wd * wd) * ph[0][i] * ph[1][j] * ph[2][k];
                }
    }
    if (N % 2 == 0) {
        const int h = N / 2;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j)
                for (int k = 0; k < N; ++k)
                    if (i == h || j == h || k == h) V[((size_t)i * N + j) * N + k] = 0;
    }
    fft3(*s.fft, V.data(), +1);
    s.vloc.resize(V.size());
    for (size_t g = 0; g < V.size(); ++g) s.vloc[g] = V[g].real();
}

// Gaussian s/p projectors (Eq. 3's |p_i>):
// p_i(G) = Omega^{-1/2} n_l (2 pi rc^2)^{3/2} exp(-|G|^2 rc^2 / 2) Y(G) exp(-i G.R),
// Y = 1 for s and -i rc^2 G_m for p_m; n_l = (pi rc^2)^{-3/4}, times
// sqrt(2 / rc^2) for p, normalises the continuum functions.
void setup_projectors(RoSys& s, int natoms, const double* pos, const int* species, const int* sp_nproj,
                      const int* sp_l, const int* sp_m, const double* sp_rc, const double* sp_D, const double* sp_Q) {
    // per-species offsets into the channel and matrix arrays
    int nsp = 0;
    for (int a = 0; a < natoms; ++a) nsp = species[a] + 1 > nsp ? species[a] + 1 : nsp;
    std::vector<int> ch_off(nsp + 1, 0), mat_off(nsp + 1, 0);
    for (int t = 0; t < nsp; ++t) {
        ch_off[t + 1] = ch_off[t] + sp_nproj[t];
        mat_off[t + 1] = mat_off[t] + sp_nproj[t] * sp_nproj[t];
    }
    int np = 0;
    for (int a = 0; a < natoms; ++a) np += sp_nproj[species[a]];
    s.nproj = np;
    s.P.assign((size_t)s.npw * np, cd(0, 0));
    s.D.assign((size_t)np * np, 0.0);
    s.Q.assign((size_t)np * np, 0.0);
    const double b = 2.0 * kPi / s.L;
    int col = 0;
    for (int a = 0; a < natoms; ++a) {
        const int t = species[a], nc = sp_nproj[t];
        for (int c = 0; c < nc; ++c) {
            const int l = sp_l[ch_off[t] + c], m = sp_m[ch_off[t] + c];
            const double rc = sp_rc[ch_off[t] + c];
            double norm = std::pow(kPi * rc * rc, -0.75);
            if (l == 1) norm *= std::sqrt(2.0 / (rc * rc));
            const double pref = norm * std::pow(2.0 * kPi * rc * rc, 1.5) / std::sqrt(s.omega);
            for (int g = 0; g < s.npw; ++g) {
                const double G[3] = {b * s.miller[3 * g], b * s.miller[3 * g + 1], b * s.miller[3 * g + 2]};
                const double GR = G[0] * pos[3 * a] + G[1] * pos[3 * a + 1] + G[2] * pos[3 * a + 2];
                const cd ang = l == 0 ? cd(1, 0) : cd(0, -rc * rc * G[m]);
                s.P[(size_t)(col + c) * s.npw + g] = pref * ang * std::exp(-0.5 * s.g2[g] * rc * rc) *
                                                     std::polar(1.0, -GR);
            }
            for (int c2 = 0; c2 < nc; ++c2) {
                s.D[(size_t)(col + c) * np + col + c2] = sp_D[mat_off[t] + c * nc + c2];
                s.Q[(size_t)(col + c) * np + col + c2] = sp_Q[mat_off[t] + c * nc + c2];
            }
        }
        col += nc;
    }
}

// ---------------------------------------------------------------- grid transforms
// psi(r) = Omega^{-1/2} sum_G c_G e^{iG.r}
void to_real(const RoSys& s, const cd* c, cd* grid) {
    std::fill(grid, grid + (size_t)s.N * s.N * s.N, cd(0, 0));
    for (int g = 0; g < s.npw; ++g) grid[s.gidx[g]] = c[g];
    fft3(*s.fft, grid, +1);
    const double f = 1.0 / std::sqrt(s.omega);
    for (size_t g = 0; g < (size_t)s.N * s.N * s.N; ++g) grid[g] *= f;
}

// <e_G|f> = Omega^{-1/2} int e^{-iG.r} f(r) dr, on the grid, G in the sphere
void to_pw(const RoSys& s, cd* grid, cd* c) {
    fft3(*s.fft, grid, -1);
    const double f = std::sqrt(s.omega) / ((double)s.N * s.N * s.N);
    for (int g = 0; g < s.npw; ++g) c[g] = grid[s.gidx[g]] * f;
}

int class_of(const RoSys& s, int n) { return n < s.n_closed ? 0 : n - s.n_closed + 1; }

// ---------------------------------------------------------------- densities
// rho3[k] += sum over the given bands of class k of |psi_n(r)|^2; bands are
// spread over threads, each with its own partial sums, added in thread order.
void densities(const RoSys& s, const cd* psi, int64_t ld, int b0, int nbands, double* rho3, int threads) {
    const size_t N3 = (size_t)s.N * s.N * s.N;
#ifdef _OPENMP
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    const int nt = 1;
    (void)threads;
#endif
    std::vector<std::vector<double>> part(nt, std::vector<double>(3 * N3, 0.0));
#pragma omp parallel for num_threads(nt) schedule(static)
    for (int t = 0; t < nt; ++t) {
        std::vector<cd> grid(N3);
        for (int n = t; n < nbands; n += nt) {
            to_real(s, psi + (int64_t)n * ld, grid.data());
            double* r = part[t].data() + (size_t)class_of(s, b0 + n) * N3;
            for (size_t g = 0; g < N3; ++g) r[g] += std::norm(grid[g]);
        }
    }
    for (int t = 0; t < nt; ++t)
        for (size_t g = 0; g < 3 * N3; ++g) rho3[g] += part[t][g];
}

// ---------------------------------------------------------------- potentials (Eqs. 8, 13)
// Vk (3 x N^3) and the energies E = {E_H, E_x_M, E_x_T, E_loc}
void potentials(const RoSys& s, const double* rho3, double* Vk, double* E) {
    const int N = s.N;
    const size_t N3 = (size_t)N * N * N;
    const double dV = s.omega / (double)N3;
    std::vector<double> rch(4 * N3, 0.0);
    for (int ch = 0; ch < 4; ++ch)
        for (int k = 0; k < 3; ++k)
            if (kF[k][ch] != 0.0)
                for (size_t g = 0; g < N3; ++g) rch[ch * N3 + g] += kF[k][ch] * rho3[k * N3 + g];
    // Hartree: one solve for rho = rho_up^M + rho_down^M (= rho^T)
    std::vector<cd> rG(N3);
    for (size_t g = 0; g < N3; ++g) rG[g] = cd(rch[g] + rch[N3 + g], 0.0);
    fft3(*s.fft, rG.data(), -1);
    double eh = 0.0;
    for (size_t g = 0; g < N3; ++g) {
        rG[g] /= (double)N3;
        if (s.G2grid[g] > 0) {
            eh += 4.0 * kPi * std::norm(rG[g]) / s.G2grid[g];
            rG[g] *= 4.0 * kPi / s.G2grid[g];
        } else {
            rG[g] = 0.0;
        }
    }
    fft3(*s.fft, rG.data(), +1);   // V_H(r) (real part)
    E[0] = 0.5 * s.omega * eh;
    // Slater exchange per channel, scaled by (1 - alpha)
    const double scale = 1.0 - s.alpha;
    const double cx = 0.75 * std::cbrt(6.0 / kPi);
    double ex[4] = {0, 0, 0, 0};
    std::vector<double> vx(4 * N3);
    for (int ch = 0; ch < 4; ++ch)
        for (size_t g = 0; g < N3; ++g) {
            const double r = rch[ch * N3 + g];
            vx[ch * N3 + g] = -scale * std::cbrt(6.0 * r / kPi);
            ex[ch] += std::cbrt(r) * r;
        }
    E[1] = -scale * cx * dV * (ex[0] + ex[1]);
    E[2] = -scale * cx * dV * (ex[2] + ex[3]);
    double eloc = 0.0;
    for (size_t g = 0; g < N3; ++g) eloc += s.vloc[g] * (rch[g] + rch[N3 + g]);
    E[3] = dV * eloc;
    // V^k = w_k (V_loc + V_H) + sum_ch c_L f_k^ch v_x^ch
    for (int k = 0; k < 3; ++k)
        for (size_t g = 0; g < N3; ++g) {
            double v = s.w[k] * (s.vloc[g] + rG[g].real());
            for (int ch = 0; ch < 4; ++ch) v += s.C[k][ch] * vx[ch * N3 + g];
            Vk[k * N3 + g] = v;
        }
}

// ---------------------------------------------------------------- apply (Eqs. 3, 13)
// F^k|n> = w_k (|G|^2 / 2 c_n + P D P^H c_n) + <G|V^k psi_n>, S|n> = c_n + P Q P^H c_n
void apply_band(const RoSys& s, const cd* c, int k, const double* Vk, cd* F, cd* Sn, cd* grid, cd* B, cd* DB) {
    const size_t N3 = (size_t)s.N * s.N * s.N;
    const int np = s.nproj;
    to_real(s, c, grid);
    const double* V = Vk + (size_t)k * N3;
    for (size_t g = 0; g < N3; ++g) grid[g] *= V[g];
    to_pw(s, grid, F);
    for (int g = 0; g < s.npw; ++g) F[g] += s.w[k] * 0.5 * s.g2[g] * c[g];
    // B = P^H c
    for (int i = 0; i < np; ++i) {
        cd b = 0;
        const cd* p = s.P.data() + (size_t)i * s.npw;
        for (int g = 0; g < s.npw; ++g) b += std::conj(p[g]) * c[g];
        B[i] = b;
    }
    // F += w_k P (D B); S = c + P (Q B)
    for (int i = 0; i < np; ++i) {
        cd d = 0, q = 0;
        for (int j = 0; j < np; ++j) {
            d += s.D[(size_t)i * np + j] * B[j];
            q += s.Q[(size_t)i * np + j] * B[j];
        }
        DB[i] = d * s.w[k];
        DB[np + i] = q;
    }
    if (Sn)
        for (int g = 0; g < s.npw; ++g) Sn[g] = c[g];
    for (int i = 0; i < np; ++i) {
        const cd* p = s.P.data() + (size_t)i * s.npw;
        const cd d = DB[i], q = DB[np + i];
        for (int g = 0; g < s.npw; ++g) {
            F[g] += p[g] * d;
            if (Sn) Sn[g] += p[g] * q;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------- C interface
// Arrays of complex numbers are interleaved (re, im) doubles; band blocks are
// column major with leading dimension ld (complex elements).
extern "C" {

// Species arrays: sp_nproj[t] channels each, channel arrays (l, m, rc)
// concatenated over the species, D and Q blocks (nproj_t x nproj_t, row
// major) concatenated likewise.  mode: 0 ground state, 1 singlet, 2
// triplet.  Returns null for a grid smaller than the sphere.
void* ro_create(double L, int N, double ecut, int mode, int n_closed, double alpha, int natoms, const double* pos,
                const int* species, const double* depth, const double* width, const int* sp_nproj, const int* sp_l,
                const int* sp_m, const double* sp_rc, const double* sp_D, const double* sp_Q) {
    RoSys* s = new RoSys();
    s->L = L;
    s->N = N;
    s->omega = L * L * L;
    s->ecut = ecut;
    s->mode = mode;
    s->n_closed = n_closed;
    s->alpha = alpha;
    s->nb = n_closed + (mode == 0 ? 0 : 2);
    s->fft = new Fft1(N);
    setup_occupations(*s);
    if (!setup_basis(*s)) {
        delete s->fft;
        delete s;
        return nullptr;
    }
    setup_vloc(*s, natoms, pos, depth, width);
    setup_projectors(*s, natoms, pos, species, sp_nproj, sp_l, sp_m, sp_rc, sp_D, sp_Q);
    return s;
}

void ro_destroy(void* h) {
    RoSys* s = static_cast<RoSys*>(h);
    if (!s) return;
    delete s->fft;
    delete s;
}

int ro_npw(void* h) { return static_cast<RoSys*>(h)->npw; }
int ro_nproj(void* h) { return static_cast<RoSys*>(h)->nproj; }
const int32_t* ro_miller(void* h) { return static_cast<RoSys*>(h)->miller.data(); }
const double* ro_vloc(void* h) { return static_cast<RoSys*>(h)->vloc.data(); }
const double* ro_projectors(void* h) { return reinterpret_cast<const double*>(static_cast<RoSys*>(h)->P.data()); }

// rho3 (3 x N^3) += the class densities of bands b0 .. b0 + nbands - 1 (psi
// holds those bands)
void ro_densities(void* h, const double* psi, int64_t ld, int b0, int nbands, double* rho3, int threads) {
    densities(*static_cast<RoSys*>(h), reinterpret_cast<const cd*>(psi), ld, b0, nbands, rho3, threads);
}

// Vk (3 x N^3) and E[0..3] = E_H, E_x_M, E_x_T, E_loc from the class densities
void ro_potentials(void* h, const double* rho3, double* Vk, double* E) {
    potentials(*static_cast<RoSys*>(h), rho3, Vk, E);
}

// F (and S, when not null) of nbands bands with classes cls[n] (0 closed,
// 1 a, 2 b), at the class potentials Vk; bands spread over threads
void ro_apply(void* h, const double* psi, int64_t ld, int nbands, const int* cls, const double* Vk, double* F,
              double* S, int threads) {
    const RoSys& s = *static_cast<RoSys*>(h);
    const cd* c = reinterpret_cast<const cd*>(psi);
    cd* Fo = reinterpret_cast<cd*>(F);
    cd* So = reinterpret_cast<cd*>(S);
    const size_t N3 = (size_t)s.N * s.N * s.N;
#ifdef _OPENMP
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#else
    const int nt = 1;
    (void)threads;
#endif
#pragma omp parallel num_threads(nt)
    {
        std::vector<cd> grid(N3), B(s.nproj + 1), DB(2 * s.nproj + 2);
#pragma omp for schedule(dynamic, 1)
        for (int n = 0; n < nbands; ++n)
            apply_band(s, c + (int64_t)n * ld, cls[n], Vk, Fo + (int64_t)n * ld, So ? So + (int64_t)n * ld : nullptr,
                       grid.data(), B.data(), DB.data());
    }
}

}  // extern "C"
