// qmc_oracle.cpp -- plain, slow FP64 CPU oracle for the VMC energy / force /
// force-covariance path and the accelerated Langevin step of Sorella & Mazzola,
// "Accelerated ab-initio Molecular Dynamics" (arXiv:1605.08423).
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, import or
// execute this file: it is used by tests/, by __graft_entry__.smoke() and by the
// cpu_baseline leg of bench.py.  It shares no code, header, table or helper with
// the CUDA library; the only common ground is the seeded synthetic inputs, which
// are passed in as arguments.
//
// Every function below states the passage it follows.  Derivatives with respect
// to the nuclear positions R are taken by forward-mode dual numbers (type D3),
// never by hand, so that this file contains no adjoint code.
//
// Readings of passages that the paper leaves open are stated at each function.
//
// Parity status (each function is pinned by a test under tests/ against a
// closed form, a textbook constant, a finite difference or brute force):
//   philox4x32_10 ........ published known-answer vectors
//   ewald ................ NaCl and simple-cubic Madelung constants, kappa invariance
//   wavefunction / E_L ... exact hydrogen atom, finite differences in r and R,
//                          translation / permutation / coefficient invariances, cusps
//   vmc chain ............ importance-sampled brute-force integral on a tiny system
//   reduce ............... i.i.d. synthetic samples with known covariance
//   U_{3+4} Jastrow ...... closed form on one nucleus, finite differences in r
//                          and R, permutation invariance, linearity in f, the
//                          Metropolis delta against full evaluations
//   langevin_step ........ harmonic closed forms (steepest descent, Newton step,
//                          stationary covariance, autocorrelation); fast and
//                          simple-rule variants against their closed forms; in
//                          the periodic box, invariance under whole-box shifts
//                          of R_prev and the canonical <cos 2 pi x / L> of a
//                          periodic potential with position-dependent S
//   twisted form ......... Bloch Gaussians against their Fourier series
//                          (Poisson summation) and the Bloch property; psi's
//                          Bloch phases and time reversal; the complex kinetic
//                          energy and the R-derivatives against finite
//                          differences; the plane-wave limit; the chain against
//                          a brute-force integral; the twist-average rule
//   empirical S .......... closed forms of one pair (with and without images
//                          inside the cutoff), finite differences of the
//                          energy, symmetry, translation sum rule, mu shift
//   toy model ............ finite differences of U, H, S^{-1}; the S-difference
//                          corrections against the cumbersome term (Gauss-Hermite
//                          averages); stationary <U> against quadratures of the
//                          canonical density and of the simple rule's density
//   "parity unpinned": the statistical quality of the random-coefficient
//   wavefunction itself (nothing in the paper fixes it).

#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <algorithm>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace orc {

// ---------------------------------------------------------------------------
// Philox4x32-10 counter-based generator, from its published definition
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11): ten rounds of two 32x32->64 multiplies with the Weyl key schedule.
// ---------------------------------------------------------------------------
static void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Counter layout shared by definition with the device library (each side has
// its own implementation): ctr = {stream, md_step, index, purpose}.
enum Purpose : uint32_t {
    P_PROP_X = 0, P_PROP_Y = 1, P_PROP_Z = 2, P_ACCEPT = 3,
    P_INIT_X = 4, P_INIT_Y = 5, P_INIT_Z = 6, P_LANGEVIN = 7
};

// 53-bit uniform in the open interval (0,1) from two 32-bit words.
static double uniform53(uint32_t a, uint32_t b) {
    uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}

struct Rng {
    uint32_t key[2];
    explicit Rng(uint64_t seed) { key[0] = (uint32_t)seed; key[1] = (uint32_t)(seed >> 32); }
    void block(uint32_t s, uint32_t m, uint32_t idx, uint32_t purpose, uint32_t out[4]) const {
        uint32_t ctr[4] = {s, m, idx, purpose};
        philox4x32_10(ctr, key, out);
    }
    double uniform(uint32_t s, uint32_t m, uint32_t idx, uint32_t purpose) const {
        uint32_t w[4]; block(s, m, idx, purpose, w);
        return uniform53(w[0], w[1]);
    }
    // Box-Muller (cosine branch) on the two uniforms of one block.
    double normal(uint32_t s, uint32_t m, uint32_t idx, uint32_t purpose) const {
        uint32_t w[4]; block(s, m, idx, purpose, w);
        double u1 = uniform53(w[0], w[1]), u2 = uniform53(w[2], w[3]);
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(2.0 * M_PI * u2);
    }
};

// ---------------------------------------------------------------------------
// Dual number with three tangent components: d/dR_{a,x}, d/dR_{a,y}, d/dR_{a,z}
// of one nucleus a.  Used only to differentiate with respect to R.
// ---------------------------------------------------------------------------
struct D3 {
    double v; double d[3];
    D3() : v(0), d{0, 0, 0} {}
    D3(double x) : v(x), d{0, 0, 0} {}
};
static inline double val(double x) { return x; }
static inline double val(const D3& x) { return x.v; }
static inline D3 operator+(const D3& a, const D3& b) { D3 r(a.v + b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] + b.d[k]; return r; }
static inline D3 operator-(const D3& a, const D3& b) { D3 r(a.v - b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] - b.d[k]; return r; }
static inline D3 operator-(const D3& a) { D3 r(-a.v); for (int k = 0; k < 3; ++k) r.d[k] = -a.d[k]; return r; }
static inline D3 operator*(const D3& a, const D3& b) { D3 r(a.v * b.v); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b.v + a.v * b.d[k]; return r; }
static inline D3 operator/(const D3& a, const D3& b) { D3 r(a.v / b.v); for (int k = 0; k < 3; ++k) r.d[k] = (a.d[k] * b.v - a.v * b.d[k]) / (b.v * b.v); return r; }
static inline D3 operator+(const D3& a, double b) { return a + D3(b); }
static inline D3 operator+(double a, const D3& b) { return D3(a) + b; }
static inline D3 operator-(const D3& a, double b) { return a - D3(b); }
static inline D3 operator-(double a, const D3& b) { return D3(a) - b; }
static inline D3 operator*(const D3& a, double b) { D3 r(a.v * b); for (int k = 0; k < 3; ++k) r.d[k] = a.d[k] * b; return r; }
static inline D3 operator*(double a, const D3& b) { return b * a; }
static inline D3 operator/(const D3& a, double b) { return a * (1.0 / b); }
static inline D3 operator/(double a, const D3& b) { return D3(a) / b; }
static inline D3& operator+=(D3& a, const D3& b) { a = a + b; return a; }
static inline D3& operator-=(D3& a, const D3& b) { a = a - b; return a; }
static inline D3& operator*=(D3& a, const D3& b) { a = a * b; return a; }
static inline D3 chain(const D3& x, double f, double fp) { D3 r(f); for (int k = 0; k < 3; ++k) r.d[k] = fp * x.d[k]; return r; }
static inline D3 exp(const D3& x) { double e = std::exp(x.v); return chain(x, e, e); }
static inline D3 sin(const D3& x) { return chain(x, std::sin(x.v), std::cos(x.v)); }
static inline D3 cos(const D3& x) { return chain(x, std::cos(x.v), -std::sin(x.v)); }
static inline D3 sqrt(const D3& x) { double s = std::sqrt(x.v); return chain(x, s, 0.5 / s); }
static inline D3 log(const D3& x) { return chain(x, std::log(x.v), 1.0 / x.v); }
static inline D3 erfc(const D3& x) { return chain(x, std::erfc(x.v), -2.0 / std::sqrt(M_PI) * std::exp(-x.v * x.v)); }

// ---------------------------------------------------------------------------
// Complex number over a real scalar S (double or D3), for the twisted
// (complex) orbitals; only the operations the determinant algebra needs.
// ---------------------------------------------------------------------------
template <class S>
struct Cx {
    S re, im;
    Cx() : re(0.0), im(0.0) {}
    Cx(const S& r, const S& i) : re(r), im(i) {}
};
template <class S> static inline Cx<S> operator+(const Cx<S>& a, const Cx<S>& b) { return Cx<S>(a.re + b.re, a.im + b.im); }
template <class S> static inline Cx<S> operator-(const Cx<S>& a, const Cx<S>& b) { return Cx<S>(a.re - b.re, a.im - b.im); }
template <class S> static inline Cx<S> operator*(const Cx<S>& a, const Cx<S>& b) {
    return Cx<S>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class S> static inline Cx<S> operator/(const Cx<S>& a, const Cx<S>& b) {
    const S q = b.re * b.re + b.im * b.im;
    return Cx<S>((a.re * b.re + a.im * b.im) / q, (a.im * b.re - a.re * b.im) / q);
}
template <class S> static inline Cx<S> scale(const Cx<S>& a, double r) { return Cx<S>(a.re * r, a.im * r); }
template <class S> static inline Cx<S>& operator+=(Cx<S>& a, const Cx<S>& b) { a = a + b; return a; }
template <class S> static inline Cx<S>& operator-=(Cx<S>& a, const Cx<S>& b) { a = a - b; return a; }
template <class S> static inline double abs2v(const Cx<S>& a) { return val(a.re) * val(a.re) + val(a.im) * val(a.im); }
using std::exp; using std::sin; using std::cos; using std::sqrt; using std::log; using std::erfc;

// ---------------------------------------------------------------------------
// System description.  Mirrors the C-ABI parameters of the library but is
// declared independently here.
// ---------------------------------------------------------------------------
struct Params {
    int32_t N;            // nuclei (protons)
    int32_t n_up, n_dn;   // electrons of each spin
    int32_t n_orb;        // orbitals (columns of coeff); >= max(n_up, n_dn)
    int32_t n_gauss;      // s-Gaussians per nucleus
    int32_t periodic;     // 1: periodic box (sin periodisation + Ewald); 0: open
    int32_t mmax;         // reciprocal cutoff |m| <= mmax
    int32_t pad_;
    double  L;            // box side (bohr)
    double  b_ee, b_ep;   // Pade Jastrow parameters
    double  Z;            // nuclear charge (1 for hydrogen)
    double  Zj;           // e-n Jastrow cusp amplitude (Z for the cusp; 0 switches U_1 off)
    double  kappa;        // Ewald splitting parameter
    const double* zeta;   // [n_gauss]
    const double* coeff;  // [N*n_gauss][n_orb], row b = a*n_gauss + g
    // 3- and 4-body e-e-n-n Jastrow U_{3+4} (SI, Jastrow section), one
    // periodised Gaussian exp(-zeta_j |d|^2) per nucleus; fj = null: term off
    double zeta_j;
    const double* fj;     // [N][N] symmetric coefficients f^{ab}
    // Twisted boundary conditions (SI, basis section): null keeps the real
    // sin-periodised orbitals; otherwise the twist vector theta [3] of the
    // spin-up determinant (spin down: -theta) and Bloch-summed Gaussians
    const double* twist;
};

// ---------------------------------------------------------------------------
// Periodised displacement (SI, "periodized with the trivial substitution"):
// each Cartesian component r_mu -> (L/pi) sin(pi r_mu / L), applied to the raw
// difference.  Reading: used for both the Jastrow and the determinant orbitals.
// For each component returns d, its first and second derivatives with respect
// to the electron coordinate.
// ---------------------------------------------------------------------------
template <class S>
static void periodised(const Params& p, double x, const S& R, S& d, S& dd, S& ddd) {
    if (p.periodic) {
        S arg = (x - R) * (M_PI / p.L);
        d = (p.L / M_PI) * sin(arg);
        dd = cos(arg);
        ddd = -(M_PI / p.L) * sin(arg);
    } else {
        d = x - R; dd = S(1.0); ddd = S(0.0);
    }
}

// Gaussian basis function chi = exp(-zeta |d|^2) with gradient and Laplacian
// in the electron coordinate (SI basis of s-Gaussians per nucleus).
template <class S>
static void gaussian(const Params& p, const double x[3], const S Rc[3], double zeta,
                     S& chi, S grad[3], S& lap) {
    S d[3], dd[3], ddd[3];
    S t(0.0);
    for (int mu = 0; mu < 3; ++mu) { periodised(p, x[mu], Rc[mu], d[mu], dd[mu], ddd[mu]); t += d[mu] * d[mu]; }
    chi = exp(-zeta * t);
    lap = S(0.0);
    for (int mu = 0; mu < 3; ++mu) {
        S dt = 2.0 * d[mu] * dd[mu];                    // d t / d x_mu
        S d2t = 2.0 * (dd[mu] * dd[mu] + d[mu] * ddd[mu]);  // d^2 t / d x_mu^2
        grad[mu] = -zeta * dt * chi;
        lap += (zeta * zeta * dt * dt - zeta * d2t) * chi;
    }
}

// Pade pair functions (SI, U_2 and the e-n term).  Reading of the sign garble:
// the electron-electron term is +r/(2(1+b r)) (cusp +1/2 under J = e^U) and the
// electron-nucleus term is -Z r/(1+b r) (cusp -Z).
static void u_ee(double b, double r, double& u, double& up, double& upp) {
    double q = 1.0 + b * r;
    u = r / (2.0 * q); up = 1.0 / (2.0 * q * q); upp = -b / (q * q * q);
}
template <class S>
static void u_ep(double b, double Z, const S& r, S& u, S& up, S& upp) {
    S q = 1.0 + b * r;
    u = -Z * r / q; up = -Z / (q * q); upp = 2.0 * Z * b / (q * q * q);
}

// Value, gradient and Laplacian (in the electron coordinate x) of a radial
// pair function u(|d(x - c)|).
template <class S, class F>
static void pair_term(const Params& p, const double x[3], const S c[3], F ufun,
                      S& u, S grad[3], S& lap) {
    S d[3], dd[3], ddd[3];
    S t(0.0);
    for (int mu = 0; mu < 3; ++mu) { periodised(p, x[mu], c[mu], d[mu], dd[mu], ddd[mu]); t += d[mu] * d[mu]; }
    S r = sqrt(t);
    S up, upp;
    ufun(r, u, up, upp);
    lap = S(0.0);
    for (int mu = 0; mu < 3; ++mu) {
        S dt = 2.0 * d[mu] * dd[mu];
        S d2t = 2.0 * (dd[mu] * dd[mu] + d[mu] * ddd[mu]);
        S dr = dt / (2.0 * r);
        S d2r = d2t / (2.0 * r) - dt * dt / (4.0 * r * r * r);
        grad[mu] = up * dr;
        lap += upp * dr * dr + up * d2r;
    }
}

// LU factorisation with partial pivoting (Golub & Van Loan, Alg. 3.4.1) and
// the inverse by forward / back substitution.  Returns log|det| and the sign.
template <class S>
static bool lu_inverse(int n, std::vector<S> A, std::vector<S>& inv, S& logdet, int& sign) {
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    sign = 1;
    logdet = S(0.0);
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(val(A[i * n + k])) > std::fabs(val(A[piv * n + k]))) piv = i;
        if (val(A[piv * n + k]) == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
            std::swap(perm[k], perm[piv]);
            sign = -sign;
        }
        S pivot = A[k * n + k];
        if (val(pivot) < 0) sign = -sign;
        logdet += log(val(pivot) < 0 ? -pivot : pivot);
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] = A[i * n + k] / pivot;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    inv.assign((size_t)n * n, S(0.0));
    for (int col = 0; col < n; ++col) {
        std::vector<S> y(n);
        for (int i = 0; i < n; ++i) {          // solve L y = P e_col
            S s = (perm[i] == col) ? S(1.0) : S(0.0);
            for (int j = 0; j < i; ++j) s -= A[i * n + j] * y[j];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {     // solve U x = y
            S s = y[i];
            for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * inv[j * n + col];
            inv[i * n + col] = s / A[i * n + i];
        }
    }
    return true;
}

// ---------------------------------------------------------------------------
// Ewald sum over point charges in the cubic box (reading of the paper's
// periodic Coulomb Hamiltonian; the truncation is part of the definition):
//   V = sum_{k<l} q_k q_l sum_{n : |r_kl + nL| < L} erfc(kappa |r_kl+nL|)/|r_kl+nL|
//     + 1/2 sum_k q_k^2 sum_{0 < |nL| < L} erfc(kappa |n| L)/(|n| L)      (empty)
//     + (4 pi / L^3) sum_{half space, 0 < |m| <= mmax} exp(-k^2/4kappa^2)/k^2 |rho(k)|^2
//     - kappa/sqrt(pi) sum_k q_k^2
//     [- pi Q^2 / (2 L^3 kappa^2)   neutralising background, only if requested]
// with k = 2 pi m / L and rho(k) = sum_k q_k exp(i k.r_k).
// ---------------------------------------------------------------------------
template <class S>
static S ewald(int nq, const double* q, const S* pos, double L, double kappa, int mmax, bool background) {
    S V(0.0);
    for (int k = 0; k < nq; ++k)
        for (int l = k + 1; l < nq; ++l) {
            S r[3];
            for (int mu = 0; mu < 3; ++mu) r[mu] = pos[3 * k + mu] - pos[3 * l + mu];
            for (int nx = -3; nx <= 3; ++nx)
                for (int ny = -3; ny <= 3; ++ny)
                    for (int nz = -3; nz <= 3; ++nz) {
                        S a = r[0] + nx * L, b = r[1] + ny * L, c = r[2] + nz * L;
                        S d = sqrt(a * a + b * b + c * c);
                        if (val(d) < L) V += q[k] * q[l] * erfc(kappa * d) / d;
                    }
        }
    for (int k = 0; k < nq; ++k)
        for (int nx = -1; nx <= 1; ++nx)
            for (int ny = -1; ny <= 1; ++ny)
                for (int nz = -1; nz <= 1; ++nz) {
                    int n2 = nx * nx + ny * ny + nz * nz;
                    double d = std::sqrt((double)n2) * L;
                    if (n2 > 0 && d < L) V += 0.5 * q[k] * q[k] * std::erfc(kappa * d) / d;
                }
    const double vol = L * L * L;
    for (int mx = 0; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz) {
                bool half = (mx > 0) || (mx == 0 && my > 0) || (mx == 0 && my == 0 && mz > 0);
                int m2 = mx * mx + my * my + mz * mz;
                if (!half || m2 > mmax * mmax) continue;
                double kx = 2 * M_PI * mx / L, ky = 2 * M_PI * my / L, kz = 2 * M_PI * mz / L;
                double k2 = kx * kx + ky * ky + kz * kz;
                S re(0.0), im(0.0);
                for (int j = 0; j < nq; ++j) {
                    S ph = kx * pos[3 * j] + ky * pos[3 * j + 1] + kz * pos[3 * j + 2];
                    re += q[j] * cos(ph);
                    im += q[j] * sin(ph);
                }
                V += (4 * M_PI / vol) * std::exp(-k2 / (4 * kappa * kappa)) / k2 * (re * re + im * im);
            }
    double q2 = 0, Q = 0;
    for (int k = 0; k < nq; ++k) { q2 += q[k] * q[k]; Q += q[k]; }
    V -= kappa / std::sqrt(M_PI) * q2;
    if (background) V -= M_PI * Q * Q / (2 * vol * kappa * kappa);
    return V;
}

// Bare Coulomb energy of point charges (open boundary; hydrogen atom pin).
template <class S>
static S coulomb_open(int nq, const double* q, const S* pos) {
    S V(0.0);
    for (int k = 0; k < nq; ++k)
        for (int l = k + 1; l < nq; ++l) {
            S a = pos[3 * k] - pos[3 * l], b = pos[3 * k + 1] - pos[3 * l + 1], c = pos[3 * k + 2] - pos[3 * l + 2];
            V += q[k] * q[l] / sqrt(a * a + b * b + c * c);
        }
    return V;
}

// ---------------------------------------------------------------------------
// Jastrow-Slater wavefunction psi = det(Phi_up) det(Phi_dn) exp(U) (Eq. for
// V(R), SI Jastrow J = e^U with U = U_1 + U_2 restricted to the Pade e-n and
// e-e terms) and its local energy
//   E_L = -1/2 sum_i [ lap_i ln psi + |grad_i ln psi|^2 ] + V.
// Electrons 0..n_up-1 carry spin up.  Orbital j of either spin is
// phi_j(r) = sum_b C[b][j] chi_b(r) (same coefficients for both spins).
// ---------------------------------------------------------------------------
template <class S>
struct WfOut {
    S lnpsi;          // ln |psi|
    int sign;
    S ekin, epot, el;
    std::vector<double> grad;  // grad_i ln psi, [Ne][3] (values only)
    bool ok;
};

template <class S>
static void slater_block(const Params& p, const S* R, const double* X, int i0, int ne,
                         S& logdet, int& sign, std::vector<S>& g, std::vector<S>& l, bool& ok) {
    const int G = p.n_gauss, nb = p.N * G, no = p.n_orb;
    std::vector<S> A((size_t)ne * ne), D[3], Lp((size_t)ne * ne);
    for (int mu = 0; mu < 3; ++mu) D[mu].assign((size_t)ne * ne, S(0.0));
    for (int i = 0; i < ne; ++i) {
        const double* x = X + 3 * (i0 + i);
        std::vector<S> chi(nb), dchi[3], lchi(nb);
        for (int mu = 0; mu < 3; ++mu) dchi[mu].resize(nb);
        for (int a = 0; a < p.N; ++a)
            for (int gg = 0; gg < G; ++gg) {
                S c, gr[3], lp;
                gaussian(p, x, R + 3 * a, p.zeta[gg], c, gr, lp);
                int b = a * G + gg;
                chi[b] = c; lchi[b] = lp;
                for (int mu = 0; mu < 3; ++mu) dchi[mu][b] = gr[mu];
            }
        for (int j = 0; j < ne; ++j) {
            S v(0.0), lv(0.0), dv[3] = {S(0.0), S(0.0), S(0.0)};
            for (int b = 0; b < nb; ++b) {
                double cbj = p.coeff[(size_t)b * no + j];
                v += cbj * chi[b]; lv += cbj * lchi[b];
                for (int mu = 0; mu < 3; ++mu) dv[mu] += cbj * dchi[mu][b];
            }
            A[i * ne + j] = v; Lp[i * ne + j] = lv;
            for (int mu = 0; mu < 3; ++mu) D[mu][i * ne + j] = dv[mu];
        }
    }
    std::vector<S> inv;
    ok = lu_inverse(ne, A, inv, logdet, sign);
    g.assign((size_t)ne * 3, S(0.0)); l.assign(ne, S(0.0));
    if (!ok) return;
    // grad_i ln det = sum_j dphi_j(r_i) G_ji ;  lap_i det / det = sum_j lap phi_j(r_i) G_ji
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) {
            for (int mu = 0; mu < 3; ++mu) g[i * 3 + mu] += D[mu][i * ne + j] * inv[j * ne + i];
            l[i] += Lp[i * ne + j] * inv[j * ne + i];
        }
}

// Jastrow exponent U with grad_i U and lap_i U of every electron (SI, J = e^U:
// the Pade e-e and e-n terms and, with p.fj, the e-e-n-n term).
template <class S>
static void jastrow_all(const Params& p, const S* R, const double* X, S& U, std::vector<S>& gU, std::vector<S>& lU) {
    const int Ne = p.n_up + p.n_dn;
    gU.assign((size_t)Ne * 3, S(0.0));
    lU.assign(Ne, S(0.0));
    U = S(0.0);
    auto fee = [&](const S& r, S& u, S& up, S& upp) {
        double uu, a, b; u_ee(p.b_ee, val(r), uu, a, b); u = S(uu); up = S(a); upp = S(b);
    };
    auto fep = [&](const S& r, S& u, S& up, S& upp) { u_ep(p.b_ep, p.Zj, r, u, up, upp); };
    for (int i = 0; i < Ne; ++i) {
        for (int j = 0; j < Ne; ++j) {
            if (j == i) continue;
            S cj[3] = {S(X[3 * j]), S(X[3 * j + 1]), S(X[3 * j + 2])};
            S u, gr[3], lp;
            pair_term(p, X + 3 * i, cj, fee, u, gr, lp);
            if (j > i) U += u;
            for (int mu = 0; mu < 3; ++mu) gU[i * 3 + mu] += gr[mu];
            lU[i] += lp;
        }
        for (int a = 0; a < p.N; ++a) {
            S u, gr[3], lp;
            pair_term(p, X + 3 * i, R + 3 * a, fep, u, gr, lp);
            U += u;
            for (int mu = 0; mu < 3; ++mu) gU[i * 3 + mu] += gr[mu];
            lU[i] += lp;
        }
    }
    // U_{3+4} = sum_{i<j} sum_{a,b} f^{ab} chi_a(r_i) chi_b(r_j) (SI, e-e-n-n term with
    // one Jastrow orbital per nucleus); its gradient and Laplacian in r_i are
    // the pair terms containing i differentiated in r_i.  Written as the
    // plain pair sum: O(Ne^2 N^2).
    if (p.fj) {
        const int N = p.N;
        std::vector<S> chi((size_t)Ne * N), gchi((size_t)Ne * N * 3), lchi((size_t)Ne * N);
        for (int i = 0; i < Ne; ++i)
            for (int a = 0; a < N; ++a) {
                S gr[3];
                gaussian(p, X + 3 * i, R + 3 * a, p.zeta_j, chi[(size_t)i * N + a], gr, lchi[(size_t)i * N + a]);
                for (int mu = 0; mu < 3; ++mu) gchi[((size_t)i * N + a) * 3 + mu] = gr[mu];
            }
        for (int i = 0; i < Ne; ++i)
            for (int j = 0; j < Ne; ++j) {
                if (j == i) continue;
                for (int a = 0; a < N; ++a) {
                    S fx(0.0);   // sum_b f^{ab} chi_b(r_j)
                    for (int b = 0; b < N; ++b) fx += p.fj[(size_t)a * N + b] * chi[(size_t)j * N + b];
                    if (j > i) U += chi[(size_t)i * N + a] * fx;
                    for (int mu = 0; mu < 3; ++mu) gU[i * 3 + mu] += gchi[((size_t)i * N + a) * 3 + mu] * fx;
                    lU[i] += lchi[(size_t)i * N + a] * fx;
                }
            }
    }
}

// Potential energy of all 2N charges (Ewald sum in the periodic box).
template <class S>
static S potential(const Params& p, const S* R, const double* X) {
    const int Ne = p.n_up + p.n_dn;
    std::vector<double> q;
    std::vector<S> pos;
    for (int i = 0; i < Ne; ++i) { q.push_back(-1.0); for (int mu = 0; mu < 3; ++mu) pos.push_back(S(X[3 * i + mu])); }
    for (int a = 0; a < p.N; ++a) { q.push_back(p.Z); for (int mu = 0; mu < 3; ++mu) pos.push_back(R[3 * a + mu]); }
    if (p.periodic) return ewald((int)q.size(), q.data(), pos.data(), p.L, p.kappa, p.mmax, false);
    return coulomb_open((int)q.size(), q.data(), pos.data());
}

template <class S>
static WfOut<S> wavefunction(const Params& p, const S* R, const double* X) {
    WfOut<S> out;
    const int Ne = p.n_up + p.n_dn;
    out.ok = true;
    out.sign = 1;
    out.lnpsi = S(0.0);
    std::vector<S> g((size_t)Ne * 3, S(0.0)), l(Ne, S(0.0));
    for (int s = 0; s < 2; ++s) {
        int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up;
        if (ne == 0) continue;
        S ld; int sg; bool ok;
        std::vector<S> gs, ls;
        slater_block(p, R, X, i0, ne, ld, sg, gs, ls, ok);
        if (!ok) { out.ok = false; return out; }
        out.lnpsi += ld; out.sign *= sg;
        for (int i = 0; i < ne; ++i) {
            for (int mu = 0; mu < 3; ++mu) g[(i0 + i) * 3 + mu] = gs[i * 3 + mu];
            l[i0 + i] = ls[i];
        }
    }
    // Jastrow U, grad_i U, lap_i U
    std::vector<S> gU, lU;
    S U;
    jastrow_all(p, R, X, U, gU, lU);
    out.lnpsi += U;
    // kinetic energy: lap_i ln psi = (l_i - |g_i|^2) + lap_i U ; grad_i ln psi = g_i + grad_i U
    S kin(0.0);
    out.grad.assign((size_t)Ne * 3, 0.0);
    for (int i = 0; i < Ne; ++i) {
        S g2(0.0), t2(0.0);
        for (int mu = 0; mu < 3; ++mu) {
            S t = g[i * 3 + mu] + gU[i * 3 + mu];
            g2 += g[i * 3 + mu] * g[i * 3 + mu];
            t2 += t * t;
            out.grad[i * 3 + mu] = val(t);
        }
        S lap_lnpsi = l[i] - g2 + lU[i];
        kin += lap_lnpsi + t2;
    }
    out.ekin = -0.5 * kin;
    // potential energy of all 2N charges
    out.epot = potential(p, R, X);
    out.el = out.ekin + out.epot;
    return out;
}

// Value-only evaluation plus all R-derivatives by one D3 pass per nucleus.
struct ConfigResult {
    double lnpsi, el, ekin, epot; int sign; bool ok;
    std::vector<double> grad, dlnpsi, del;
};
static ConfigResult eval_config(const Params& p, const double* R, const double* X, bool derivs) {
    ConfigResult res;
    WfOut<double> w = wavefunction<double>(p, R, X);
    res.ok = w.ok; res.lnpsi = w.lnpsi; res.el = w.el; res.ekin = w.ekin; res.epot = w.epot;
    res.sign = w.sign; res.grad = w.grad;
    if (!derivs || !w.ok) return res;
    res.dlnpsi.assign((size_t)3 * p.N, 0.0);
    res.del.assign((size_t)3 * p.N, 0.0);
    std::vector<D3> Rd((size_t)3 * p.N);
    for (int a = 0; a < p.N; ++a) {
        for (int k = 0; k < 3 * p.N; ++k) Rd[k] = D3(R[k]);
        for (int mu = 0; mu < 3; ++mu) Rd[3 * a + mu].d[mu] = 1.0;
        WfOut<D3> wd = wavefunction<D3>(p, Rd.data(), X);
        for (int mu = 0; mu < 3; ++mu) {
            res.dlnpsi[3 * a + mu] = wd.lnpsi.d[mu];
            res.del[3 * a + mu] = wd.el.d[mu];
        }
    }
    return res;
}

static double wrap(double x, double L) { return x - L * std::floor(x / L); }

// ---------------------------------------------------------------------------
// Metropolis VMC chain of one walker (standard single-electron Metropolis;
// the paper defers the sampler to its references).  Readings:
//   * walker start: up electron i at nucleus i, down electron i at nucleus
//     n_up + i (modulo N), plus 0.5 bohr Gaussian noise;
//   * sweep = electrons 0..Ne-1 in order; proposal r' = r + sigma xi;
//   * accept when u < |psi'/psi|^2 (strict);
//   * after sweep s >= n_warmup, a sample is taken when
//     (s - n_warmup + 1) % measure_every == 0.
// Per-walker accumulators (layout [cnt, sE, sE2, sO(3N), sEO(3N), sdE(3N)]).
// The ratio is det(A')/det(A) from a fresh LU of the moved block; the Jastrow
// ratio uses the pair terms containing electron i (all others cancel).
// ---------------------------------------------------------------------------
static void slater_row(const Params& p, const double* R, const double* x, int ne, double* row) {
    const int G = p.n_gauss, no = p.n_orb;
    for (int j = 0; j < ne; ++j) row[j] = 0;
    for (int a = 0; a < p.N; ++a)
        for (int gg = 0; gg < G; ++gg) {
            double c, gr[3], lp;
            gaussian<double>(p, x, R + 3 * a, p.zeta[gg], c, gr, lp);
            int b = a * G + gg;
            for (int j = 0; j < ne; ++j) row[j] += p.coeff[(size_t)b * no + j] * c;
        }
}

static double pair_u(const Params& p, const double* x, const double* c, bool ee) {
    double t = 0;
    for (int mu = 0; mu < 3; ++mu) {
        double d, dd, ddd;
        periodised<double>(p, x[mu], c[mu], d, dd, ddd);
        t += d * d;
    }
    double r = std::sqrt(t), u, up, upp;
    if (ee) u_ee(p.b_ee, r, u, up, upp);
    else u_ep<double>(p.b_ep, p.Zj, r, u, up, upp);
    return u;
}

static double jastrow_orbital(const Params& p, const double* x, const double* Ra) {
    double c, gr[3], lp;
    gaussian<double>(p, x, Ra, p.zeta_j, c, gr, lp);
    return c;
}

static double jastrow_delta(const Params& p, const double* R, const double* X, int i, const double* xn) {
    const int Ne = p.n_up + p.n_dn;
    double du = 0;
    for (int j = 0; j < Ne; ++j) {
        if (j == i) continue;
        du += pair_u(p, xn, X + 3 * j, true) - pair_u(p, X + 3 * i, X + 3 * j, true);
    }
    for (int a = 0; a < p.N; ++a) du += pair_u(p, xn, R + 3 * a, false) - pair_u(p, X + 3 * i, R + 3 * a, false);
    if (p.fj) {   // U_{3+4}: the pairs (i, j) with chi(r_i) replaced
        const int N = p.N;
        for (int a = 0; a < N; ++a) {
            const double dchi = jastrow_orbital(p, xn, R + 3 * a) - jastrow_orbital(p, X + 3 * i, R + 3 * a);
            for (int j = 0; j < Ne; ++j) {
                if (j == i) continue;
                for (int b = 0; b < N; ++b)
                    du += dchi * p.fj[(size_t)a * N + b] * jastrow_orbital(p, X + 3 * j, R + 3 * b);
            }
        }
    }
    return du;
}

static double logdet_of(int n, const std::vector<double>& A, int& sign, bool& ok) {
    std::vector<double> inv; double ld;
    ok = lu_inverse<double>(n, A, inv, ld, sign);
    return ld;
}

struct ChainArgs {
    int32_t W, n_sweeps, n_warmup, measure_every;
    int32_t init_walkers;   // 1: place walkers from Philox; 0: X holds them already
    int32_t forces;         // 1: accumulate R-derivatives (D3 passes)
    uint32_t md_step;
    int32_t pad_;
    double sigma;
    uint64_t seed;
};

static void init_walker(const Params& p, const Rng& rng, uint32_t w, const double* R, double* X) {
    const int Ne = p.n_up + p.n_dn;
    for (int i = 0; i < Ne; ++i) {
        int site = (i < p.n_up ? i : p.n_up + (i - p.n_up)) % p.N;
        for (int mu = 0; mu < 3; ++mu) {
            double z = rng.normal(w, 0u, (uint32_t)i, P_INIT_X + mu);
            double x = R[3 * site + mu] + 0.5 * z;
            X[3 * i + mu] = p.periodic ? wrap(x, p.L) : x;
        }
    }
}

static void run_walker(const Params& p, const ChainArgs& c, const Rng& rng, uint32_t w, const double* R,
                       double* X, double* acc, double* vacc, long long* n_acc, long long* n_try) {
    const int Ne = p.n_up + p.n_dn, N3 = 3 * p.N;
    if (c.init_walkers) init_walker(p, rng, w, R, X);
    // Slater matrices of both spin blocks, rows = electrons
    std::vector<double> A[2];
    double ld[2] = {0, 0}; int sg[2] = {1, 1};
    for (int s = 0; s < 2; ++s) {
        int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up;
        A[s].assign((size_t)ne * ne, 0.0);
        for (int i = 0; i < ne; ++i) slater_row(p, R, X + 3 * (i0 + i), ne, &A[s][(size_t)i * ne]);
        bool ok = true;
        if (ne) ld[s] = logdet_of(ne, A[s], sg[s], ok);
    }
    const int total = c.n_warmup + c.n_sweeps;
    for (int sw = 0; sw < total; ++sw) {
        for (int i = 0; i < Ne; ++i) {
            const int s = i < p.n_up ? 0 : 1;
            const int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up, il = i - i0;
            const uint32_t idx = (uint32_t)(sw * Ne + i);
            double xn[3];
            for (int mu = 0; mu < 3; ++mu) xn[mu] = X[3 * i + mu] + c.sigma * rng.normal(w, c.md_step, idx, P_PROP_X + mu);
            std::vector<double> An = A[s];
            slater_row(p, R, xn, ne, &An[(size_t)il * ne]);
            int sgn; bool ok;
            double ldn = logdet_of(ne, An, sgn, ok);
            double du = jastrow_delta(p, R, X, i, xn);
            double prob = ok ? std::exp(2.0 * (ldn - ld[s]) + 2.0 * du) : 0.0;
            double u = rng.uniform(w, c.md_step, idx, P_ACCEPT);
            ++*n_try;
            if (u < prob) {
                ++*n_acc;
                A[s] = An; ld[s] = ldn; sg[s] = sgn;
                for (int mu = 0; mu < 3; ++mu) X[3 * i + mu] = p.periodic ? wrap(xn[mu], p.L) : xn[mu];
            }
        }
        if (sw >= c.n_warmup && ((sw - c.n_warmup + 1) % c.measure_every) == 0) {
            ConfigResult r = eval_config(p, R, X, c.forces != 0);
            acc[0] += 1; acc[1] += r.el; acc[2] += r.el * r.el;
            if (vacc) vacc[0] += r.epot;
            if (c.forces)
                for (int k = 0; k < N3; ++k) {
                    acc[3 + k] += r.dlnpsi[k];
                    acc[3 + N3 + k] += r.el * r.dlnpsi[k];
                    acc[3 + 2 * N3 + k] += r.del[k];
                }
        }
    }
}

// ---------------------------------------------------------------------------
// Twisted boundary conditions (SI, basis section: the orbitals obey
// phi(r + n L) = exp(i theta.n) phi(r) for integer vectors n).  Reading: the
// Gaussians are turned into Bloch functions by the standard lattice sum
//   chi_{a,g}(r) = sum_n exp(i theta.n) exp(-zeta_g |r - R_a - n L|^2),
// which has that property for every n; the spin-up determinant uses theta and
// the spin-down one -theta (the SI's opposite twists for opposite spins) with
// the same real coefficients, so the down orbitals are the complex conjugates
// of the up ones and psi(-theta) = conj psi(theta).  The Jastrow factor stays
// the real sin-periodised one.  Truncation (part of the definition): with k
// the nearest integer vector to (r - R_a)/L, the images n = k + m with m in
// [-M, M]^3 and
//   M = max(1, ceil(sqrt(40 / zeta_min) / L - 1/2)),
// so that every omitted image lies more than sqrt(40 / zeta_min) away (each
// omitted term below e^-40 of the largest one).
// With complex psi the sampled density is |psi|^2, and the estimators take the
// real parts: E_L = Re(H psi / psi), d ln|psi| / dR = Re(d ln psi / dR) and
// d E_L / dR = Re(d (H psi / psi) / dR) (H is Hermitian, so
// E = <|psi|^2 Re E_L> / <|psi|^2> and its R-derivative take these forms).
// ---------------------------------------------------------------------------
static int bloch_images(const Params& p) {
    double zmin = p.zeta[0];
    for (int g = 1; g < p.n_gauss; ++g) zmin = std::min(zmin, p.zeta[g]);
    const int M = (int)std::ceil(std::sqrt(40.0 / zmin) / p.L - 0.5);
    return M < 1 ? 1 : M;
}

// Bloch-summed Gaussian, its gradient and its Laplacian in the electron
// coordinate x, as the plain sum over the (2M+1)^3 images.
template <class S>
static void bloch_gaussian(double L, const double x[3], const S Rc[3], double zeta, const double th[3], int M,
                           Cx<S>& chi, Cx<S> grad[3], Cx<S>& lap) {
    chi = Cx<S>(); lap = Cx<S>();
    for (int mu = 0; mu < 3; ++mu) grad[mu] = Cx<S>();
    S d[3];
    int k[3];
    for (int mu = 0; mu < 3; ++mu) {
        d[mu] = x[mu] - Rc[mu];
        k[mu] = (int)std::nearbyint(val(d[mu]) / L);
    }
    for (int m0 = -M; m0 <= M; ++m0)
        for (int m1 = -M; m1 <= M; ++m1)
            for (int m2 = -M; m2 <= M; ++m2) {
                const int n[3] = {k[0] + m0, k[1] + m1, k[2] + m2};
                S u[3], r2(0.0);
                for (int mu = 0; mu < 3; ++mu) { u[mu] = d[mu] - (double)n[mu] * L; r2 += u[mu] * u[mu]; }
                const S e = exp(-zeta * r2);
                const double ph = th[0] * n[0] + th[1] * n[1] + th[2] * n[2];
                const double c = std::cos(ph), s = std::sin(ph);
                chi += Cx<S>(c * e, s * e);
                for (int mu = 0; mu < 3; ++mu) {
                    const S gm = -2.0 * zeta * u[mu] * e;
                    grad[mu] += Cx<S>(c * gm, s * gm);
                }
                const S lp = (4.0 * zeta * zeta * r2 - 6.0 * zeta) * e;
                lap += Cx<S>(c * lp, s * lp);
            }
}

// Complex LU with partial pivoting (largest modulus; Golub & Van Loan,
// Alg. 3.4.1) and the inverse; returns ln|det| and arg det (value only).
template <class S>
static bool lu_inverse_c(int n, std::vector<Cx<S>> A, std::vector<Cx<S>>& inv, S& logabs, double& phase) {
    std::vector<int> perm(n);
    for (int i = 0; i < n; ++i) perm[i] = i;
    logabs = S(0.0);
    phase = 0.0;
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (abs2v(A[i * n + k]) > abs2v(A[piv * n + k])) piv = i;
        if (abs2v(A[piv * n + k]) == 0.0) return false;
        if (piv != k) {
            for (int j = 0; j < n; ++j) std::swap(A[k * n + j], A[piv * n + j]);
            std::swap(perm[k], perm[piv]);
            phase += M_PI;
        }
        const Cx<S> pivot = A[k * n + k];
        logabs += 0.5 * log(pivot.re * pivot.re + pivot.im * pivot.im);
        phase += std::atan2(val(pivot.im), val(pivot.re));
        for (int i = k + 1; i < n; ++i) {
            A[i * n + k] = A[i * n + k] / pivot;
            for (int j = k + 1; j < n; ++j) A[i * n + j] -= A[i * n + k] * A[k * n + j];
        }
    }
    phase = std::remainder(phase, 2.0 * M_PI);
    inv.assign((size_t)n * n, Cx<S>());
    for (int col = 0; col < n; ++col) {
        std::vector<Cx<S>> y(n);
        for (int i = 0; i < n; ++i) {
            Cx<S> s = (perm[i] == col) ? Cx<S>(S(1.0), S(0.0)) : Cx<S>();
            for (int j = 0; j < i; ++j) s -= A[i * n + j] * y[j];
            y[i] = s;
        }
        for (int i = n - 1; i >= 0; --i) {
            Cx<S> s = y[i];
            for (int j = i + 1; j < n; ++j) s -= A[i * n + j] * inv[j * n + col];
            inv[i * n + col] = s / A[i * n + i];
        }
    }
    return true;
}

// Twisted Slater block of electrons i0..i0+ne-1 with twist th: ln|det|,
// arg det, and per electron g_i = grad_i det / det, l_i = lap_i det / det.
template <class S>
static void slater_block_twist(const Params& p, const S* R, const double* X, int i0, int ne, const double th[3],
                               S& logabs, double& phase, std::vector<Cx<S>>& g, std::vector<Cx<S>>& l, bool& ok) {
    const int G = p.n_gauss, nb = p.N * G, no = p.n_orb, M = bloch_images(p);
    std::vector<Cx<S>> A((size_t)ne * ne), D[3], Lp((size_t)ne * ne);
    for (int mu = 0; mu < 3; ++mu) D[mu].assign((size_t)ne * ne, Cx<S>());
    for (int i = 0; i < ne; ++i) {
        const double* x = X + 3 * (i0 + i);
        std::vector<Cx<S>> chi(nb), dchi[3], lchi(nb);
        for (int mu = 0; mu < 3; ++mu) dchi[mu].resize(nb);
        for (int a = 0; a < p.N; ++a)
            for (int gg = 0; gg < G; ++gg) {
                Cx<S> c, gr[3], lp;
                bloch_gaussian(p.L, x, R + 3 * a, p.zeta[gg], th, M, c, gr, lp);
                const int b = a * G + gg;
                chi[b] = c; lchi[b] = lp;
                for (int mu = 0; mu < 3; ++mu) dchi[mu][b] = gr[mu];
            }
        for (int j = 0; j < ne; ++j) {
            Cx<S> v, lv, dv[3];
            for (int b = 0; b < nb; ++b) {
                const double cbj = p.coeff[(size_t)b * no + j];
                v += scale(chi[b], cbj); lv += scale(lchi[b], cbj);
                for (int mu = 0; mu < 3; ++mu) dv[mu] += scale(dchi[mu][b], cbj);
            }
            A[i * ne + j] = v; Lp[i * ne + j] = lv;
            for (int mu = 0; mu < 3; ++mu) D[mu][i * ne + j] = dv[mu];
        }
    }
    std::vector<Cx<S>> inv;
    ok = lu_inverse_c(ne, A, inv, logabs, phase);
    g.assign((size_t)ne * 3, Cx<S>()); l.assign(ne, Cx<S>());
    if (!ok) return;
    for (int i = 0; i < ne; ++i)
        for (int j = 0; j < ne; ++j) {
            for (int mu = 0; mu < 3; ++mu) g[i * 3 + mu] += D[mu][i * ne + j] * inv[j * ne + i];
            l[i] += Lp[i * ne + j] * inv[j * ne + i];
        }
}

template <class S>
struct WfTwist {
    S lnpsi;          // ln |psi|
    double phase;     // arg psi (value only)
    S ekin, epot, el; // Re of the kinetic and local energies
    double ekin_im;   // Im of the kinetic energy (value only)
    std::vector<double> grad;  // Re grad_i ln psi, [Ne][3]
    bool ok;
};

// Twisted wavefunction psi = det(Phi_up(theta)) det(Phi_dn(-theta)) e^U and
//   H psi / psi = -1/2 sum_i [ l_i + 2 g_i . grad_i U + lap_i U + |grad_i U|^2 ] + V
// (complex l_i, g_i of the blocks; U real), E_L its real part.
template <class S>
static WfTwist<S> wavefunction_twist(const Params& p, const S* R, const double* X) {
    WfTwist<S> out;
    const int Ne = p.n_up + p.n_dn;
    out.ok = true;
    out.lnpsi = S(0.0);
    out.phase = 0.0;
    std::vector<Cx<S>> g((size_t)Ne * 3), l(Ne);
    for (int s = 0; s < 2; ++s) {
        const int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up;
        if (ne == 0) continue;
        const double sg = s ? -1.0 : 1.0;
        const double th[3] = {sg * p.twist[0], sg * p.twist[1], sg * p.twist[2]};
        S la; double ph; bool ok;
        std::vector<Cx<S>> gs, ls;
        slater_block_twist(p, R, X, i0, ne, th, la, ph, gs, ls, ok);
        if (!ok) { out.ok = false; return out; }
        out.lnpsi += la; out.phase += ph;
        for (int i = 0; i < ne; ++i) {
            for (int mu = 0; mu < 3; ++mu) g[(i0 + i) * 3 + mu] = gs[i * 3 + mu];
            l[i0 + i] = ls[i];
        }
    }
    out.phase = std::remainder(out.phase, 2.0 * M_PI);
    std::vector<S> gU, lU;
    S U;
    jastrow_all(p, R, X, U, gU, lU);
    out.lnpsi += U;
    S kin(0.0);
    double kin_im = 0.0;
    out.grad.assign((size_t)Ne * 3, 0.0);
    for (int i = 0; i < Ne; ++i) {
        S re = l[i].re + lU[i];
        double im = val(l[i].im);
        for (int mu = 0; mu < 3; ++mu) {
            re += 2.0 * g[i * 3 + mu].re * gU[i * 3 + mu] + gU[i * 3 + mu] * gU[i * 3 + mu];
            im += 2.0 * val(g[i * 3 + mu].im) * val(gU[i * 3 + mu]);
            out.grad[i * 3 + mu] = val(g[i * 3 + mu].re + gU[i * 3 + mu]);
        }
        kin += re;
        kin_im += im;
    }
    out.ekin = -0.5 * kin;
    out.ekin_im = -0.5 * kin_im;
    out.epot = potential(p, R, X);
    out.el = out.ekin + out.epot;
    return out;
}

struct TwistResult {
    double lnpsi, phase, el, ekin, ekin_im, epot; bool ok;
    std::vector<double> grad, dlnpsi, del;
};
static TwistResult eval_config_twist(const Params& p, const double* R, const double* X, bool derivs) {
    TwistResult res;
    WfTwist<double> w = wavefunction_twist<double>(p, R, X);
    res.ok = w.ok; res.lnpsi = w.lnpsi; res.phase = w.phase; res.el = w.el; res.ekin = w.ekin;
    res.ekin_im = w.ekin_im; res.epot = w.epot; res.grad = w.grad;
    if (!derivs || !w.ok) return res;
    res.dlnpsi.assign((size_t)3 * p.N, 0.0);
    res.del.assign((size_t)3 * p.N, 0.0);
    std::vector<D3> Rd((size_t)3 * p.N);
    for (int a = 0; a < p.N; ++a) {
        for (int k = 0; k < 3 * p.N; ++k) Rd[k] = D3(R[k]);
        for (int mu = 0; mu < 3; ++mu) Rd[3 * a + mu].d[mu] = 1.0;
        WfTwist<D3> wd = wavefunction_twist<D3>(p, Rd.data(), X);
        for (int mu = 0; mu < 3; ++mu) {
            res.dlnpsi[3 * a + mu] = wd.lnpsi.d[mu];
            res.del[3 * a + mu] = wd.el.d[mu];
        }
    }
    return res;
}

// Row of twisted orbitals at x (values only).
static void slater_row_twist(const Params& p, const double* R, const double* x, int ne, const double th[3],
                             Cx<double>* row) {
    const int G = p.n_gauss, no = p.n_orb, M = bloch_images(p);
    for (int j = 0; j < ne; ++j) row[j] = Cx<double>();
    for (int a = 0; a < p.N; ++a)
        for (int gg = 0; gg < G; ++gg) {
            Cx<double> c, gr[3], lp;
            bloch_gaussian<double>(p.L, x, R + 3 * a, p.zeta[gg], th, M, c, gr, lp);
            const int b = a * G + gg;
            for (int j = 0; j < ne; ++j) row[j] += scale(c, p.coeff[(size_t)b * no + j]);
        }
}

// The Metropolis chain of run_walker with twisted orbitals (the spin-up block
// with twist theta = p.twist, spin down with -theta): acceptance |psi'/psi|^2
// from ln|det| of fresh complex LUs; the same Philox draws, sweep order and
// sampling rule; samples from eval_config_twist.
static void run_walker_twist(const Params& p, const ChainArgs& c, const Rng& rng, uint32_t w, const double* R,
                             double* X, double* acc, double* vacc, long long* n_acc, long long* n_try) {
    const int Ne = p.n_up + p.n_dn, N3 = 3 * p.N;
    if (c.init_walkers) init_walker(p, rng, w, R, X);
    std::vector<Cx<double>> A[2];
    double ld[2] = {0, 0};
    double th[2][3];
    for (int s = 0; s < 2; ++s) {
        const double sg = s ? -1.0 : 1.0;
        for (int mu = 0; mu < 3; ++mu) th[s][mu] = sg * p.twist[mu];
        const int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up;
        A[s].assign((size_t)ne * ne, Cx<double>());
        for (int i = 0; i < ne; ++i) slater_row_twist(p, R, X + 3 * (i0 + i), ne, th[s], &A[s][(size_t)i * ne]);
        std::vector<Cx<double>> inv; double ph;
        if (ne) lu_inverse_c(ne, A[s], inv, ld[s], ph);
    }
    const int total = c.n_warmup + c.n_sweeps;
    for (int sw = 0; sw < total; ++sw) {
        for (int i = 0; i < Ne; ++i) {
            const int s = i < p.n_up ? 0 : 1;
            const int i0 = s ? p.n_up : 0, ne = s ? p.n_dn : p.n_up, il = i - i0;
            const uint32_t idx = (uint32_t)(sw * Ne + i);
            double xn[3];
            for (int mu = 0; mu < 3; ++mu) xn[mu] = X[3 * i + mu] + c.sigma * rng.normal(w, c.md_step, idx, P_PROP_X + mu);
            std::vector<Cx<double>> An = A[s];
            slater_row_twist(p, R, xn, ne, th[s], &An[(size_t)il * ne]);
            std::vector<Cx<double>> inv; double ldn, ph;
            const bool ok = lu_inverse_c(ne, An, inv, ldn, ph);
            const double du = jastrow_delta(p, R, X, i, xn);
            const double prob = ok ? std::exp(2.0 * (ldn - ld[s]) + 2.0 * du) : 0.0;
            const double u = rng.uniform(w, c.md_step, idx, P_ACCEPT);
            ++*n_try;
            if (u < prob) {
                ++*n_acc;
                for (int mu = 0; mu < 3; ++mu) X[3 * i + mu] = p.periodic ? wrap(xn[mu], p.L) : xn[mu];
                // the row of the wrapped position differs from An's by a phase only
                slater_row_twist(p, R, X + 3 * i, ne, th[s], &An[(size_t)il * ne]);
                A[s] = An; ld[s] = ldn;
            }
        }
        if (sw >= c.n_warmup && ((sw - c.n_warmup + 1) % c.measure_every) == 0) {
            TwistResult r = eval_config_twist(p, R, X, c.forces != 0);
            acc[0] += 1; acc[1] += r.el; acc[2] += r.el * r.el;
            if (vacc) vacc[0] += r.epot;
            if (c.forces)
                for (int k = 0; k < N3; ++k) {
                    acc[3 + k] += r.dlnpsi[k];
                    acc[3 + N3 + k] += r.el * r.dlnpsi[k];
                    acc[3 + 2 * N3 + k] += r.del[k];
                }
        }
    }
}

// ---------------------------------------------------------------------------
// Statistics (covariance matrix definition of the paper):
//   E = mean E_L;  f = -<dE_L/dR> - 2(<E_L dlnpsi/dR> - E <dlnpsi/dR>)
//   per-walker block forces f_w (same formula with walker means and the global E)
//   S = sum_w (f_w - f)(f_w - f)^T / (W (W-1))   (covariance of the mean)
//   E_err^2 = sum_w (E_w - E)^2 / (W (W-1)),  N_c = number of samples.
// ---------------------------------------------------------------------------
static void reduce(int W, int N3, const double* acc, double* E, double* Eerr, double* f, double* S, double* Nc) {
    const int stride = 3 + 3 * N3;
    double cnt = 0, sE = 0;
    std::vector<double> sO(N3, 0), sEO(N3, 0), sdE(N3, 0);
    for (int w = 0; w < W; ++w) {
        const double* a = acc + (size_t)w * stride;
        cnt += a[0]; sE += a[1];
        for (int k = 0; k < N3; ++k) { sO[k] += a[3 + k]; sEO[k] += a[3 + N3 + k]; sdE[k] += a[3 + 2 * N3 + k]; }
    }
    *Nc = cnt;
    double Em = sE / cnt;
    *E = Em;
    for (int k = 0; k < N3; ++k) f[k] = -sdE[k] / cnt - 2.0 * (sEO[k] / cnt - Em * sO[k] / cnt);
    std::vector<double> fw((size_t)W * N3);
    double ve = 0;
    for (int w = 0; w < W; ++w) {
        const double* a = acc + (size_t)w * stride;
        double c = a[0];
        double ew = a[1] / c;
        ve += (ew - Em) * (ew - Em);
        for (int k = 0; k < N3; ++k)
            fw[(size_t)w * N3 + k] = -a[3 + 2 * N3 + k] / c - 2.0 * (a[3 + N3 + k] / c - Em * a[3 + k] / c);
    }
    *Eerr = W > 1 ? std::sqrt(ve / ((double)W * (W - 1))) : 0.0;
    for (int i = 0; i < N3; ++i)
        for (int j = 0; j < N3; ++j) {
            double s = 0;
            for (int w = 0; w < W; ++w) s += (fw[(size_t)w * N3 + i] - f[i]) * (fw[(size_t)w * N3 + j] - f[j]);
            S[(size_t)i * N3 + j] = W > 1 ? s / ((double)W * (W - 1)) : 0.0;
        }
}

// ---------------------------------------------------------------------------
// Twist average (main text: k-point sampling of the Brillouin zone on a
// Monkhorst-Pack mesh, whose points have equal weights).  Walkers come in K
// contiguous blocks of W/K, block t sampling twist t; each block is reduced on
// its own (its force with its own energy E_t, the estimator holding per twist)
// and the K independent estimates are averaged:
//   E = (1/K) sum_t E_t,  f = (1/K) sum_t f_t,  S = (1/K^2) sum_t S_t,
//   E_err^2 = (1/K^2) sum_t E_err,t^2,  N_c = sum_t N_c,t.
// ---------------------------------------------------------------------------
static void reduce_twists(int K, int W, int N3, const double* acc, double* E, double* Eerr, double* f, double* S,
                          double* Nc) {
    const int Wk = W / K, stride = 3 + 3 * N3;
    *E = 0; *Nc = 0;
    double e2 = 0;
    for (int k = 0; k < N3; ++k) f[k] = 0;
    for (size_t k = 0; k < (size_t)N3 * N3; ++k) S[k] = 0;
    std::vector<double> ft(N3), St((size_t)N3 * N3);
    for (int t = 0; t < K; ++t) {
        double Et, Eet, Nct;
        reduce(Wk, N3, acc + (size_t)t * Wk * stride, &Et, &Eet, ft.data(), St.data(), &Nct);
        *E += Et / K; e2 += Eet * Eet; *Nc += Nct;
        for (int k = 0; k < N3; ++k) f[k] += ft[k] / K;
        for (size_t k = 0; k < (size_t)N3 * N3; ++k) S[k] += St[k] / ((double)K * K);
    }
    *Eerr = std::sqrt(e2) / K;
}

// ---------------------------------------------------------------------------
// Empirical acceleration matrix (main text, conclusions: S = H + mu I with H
// the Hessian of an accurate and cheap empirical potential, mu > 0 chosen
// where H is not positive definite; the paper names no potential).  Reading:
// the screened-Coulomb (Yukawa) pair potential of the protons in the electron
// gas,
//   V(R) = sum_{a<b} sum_{n : |d_ab + nL| < L} v(|d_ab + nL|),  v(r) = exp(-r / lambda) / r,
// with d_ab = R_a - R_b and the images n taken within one box side, lambda the
// screening length.  H = d^2 V / dR dR by nested forward-mode dual numbers.
// ---------------------------------------------------------------------------
template <class V>
struct D1 {   // value and one tangent over a value type that may itself be a D1
    V v, d;
    D1() : v(0.0), d(0.0) {}
    D1(double c) : v(c), d(0.0) {}
    D1(const V& a, const V& b) : v(a), d(b) {}
};
template <class V> static inline D1<V> operator+(const D1<V>& a, const D1<V>& b) { return D1<V>(a.v + b.v, a.d + b.d); }
template <class V> static inline D1<V> operator-(const D1<V>& a, const D1<V>& b) { return D1<V>(a.v - b.v, a.d - b.d); }
template <class V> static inline D1<V> operator*(const D1<V>& a, const D1<V>& b) {
    return D1<V>(a.v * b.v, a.d * b.v + a.v * b.d);
}
template <class V> static inline D1<V> operator/(const D1<V>& a, const D1<V>& b) {
    const V q = a.v / b.v;
    return D1<V>(q, (a.d - q * b.d) / b.v);
}
template <class V> static inline D1<V> operator*(double c, const D1<V>& a) { return D1<V>(c * a.v, c * a.d); }
template <class V> static inline D1<V> operator-(const D1<V>& a, double c) { return D1<V>(a.v - c, a.d); }
template <class V> static inline D1<V>& operator+=(D1<V>& a, const D1<V>& b) { a = a + b; return a; }
template <class V> static inline D1<V> exp(const D1<V>& a) { const V e = exp(a.v); return D1<V>(e, e * a.d); }
template <class V> static inline D1<V> sqrt(const D1<V>& a) { const V r = sqrt(a.v); return D1<V>(r, a.d / (2.0 * r)); }
template <class V> static inline double val(const D1<V>& a) { return val(a.v); }

template <class E>
static E empirical_energy(int N, double L, const E* R, double lambda) {
    E V(0.0);
    for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) {
            E d[3];
            for (int mu = 0; mu < 3; ++mu) {
                d[mu] = R[3 * a + mu] - R[3 * b + mu];
                d[mu] = d[mu] - L * std::nearbyint(val(d[mu]) / L);   // minimum image
            }
            for (int n0 = -2; n0 <= 2; ++n0)
                for (int n1 = -2; n1 <= 2; ++n1)
                    for (int n2 = -2; n2 <= 2; ++n2) {
                        const int nn[3] = {n0, n1, n2};
                        E r2(0.0);
                        for (int mu = 0; mu < 3; ++mu) {
                            const E x = d[mu] - (-L * nn[mu]);
                            r2 += x * x;
                        }
                        if (!(val(r2) < L * L)) continue;
                        const E r = sqrt(r2);
                        V += exp(E(0.0) - (1.0 / lambda) * r) / r;
                    }
        }
    return V;
}

// S = H + mu I ([3N][3N]); one pass of second-order duals per pair of coordinates.
static void empirical_s(int N, double L, const double* R, double lambda, double mu, double* S) {
    typedef D1<D1<double>> E2;
    const int n3 = 3 * N;
    std::vector<E2> x(n3);
    for (int i = 0; i < n3; ++i)
        for (int j = i; j < n3; ++j) {
            for (int k = 0; k < n3; ++k) x[k] = E2(R[k]);
            x[i].d.v = 1.0;     // outer tangent along coordinate i
            x[j].v.d = 1.0;     // inner tangent along coordinate j
            const E2 V = empirical_energy<E2>(N, L, x.data(), lambda);
            const double h = V.d.d;
            S[(size_t)i * n3 + j] = h + (i == j ? mu : 0.0);
            S[(size_t)j * n3 + i] = h + (i == j ? mu : 0.0);
        }
}

// ---------------------------------------------------------------------------
// Adopted integrator (SI, "Better integration scheme, the adopted one"):
//   R' = R + Dt S^{-1} [ f - (S_prev - S)(R_prev - R) / (2 Db) ] + sqrt(2 T Db) z,
//   <z z^T> = S^{-1},  Dt = (1-e^{-a D})/a,  Db = (1-e^{-2 a D})/(2a)  (Dt = Db = D at a = 0).
// z = L^{-T} xi with S = L L^T (Cholesky) and xi ~ N(0, I).  Optional noise
// correction (SI "Noise correction"): T -> T - D/2.  box > 0 wraps R' into [0, box).
// R_prev - R is the displacement of the previous step: in the periodic box
// (box > 0) its minimum image, each component reduced by the nearest multiple
// of box (a position wrapped into the box between the two steps would
// otherwise enter with a jump of one box side).
// scheme selects the variant of the SI:
//   LV_ADOPTED  the equation above;
//   LV_FAST     the faster iteration scheme (Eq. finaldyn):
//               R' = R + D S^{-1} f + sqrt(2 T D) z - (1/2) S^{-1} (S_prev - S)(R_prev - R);
//   LV_NOROGNA  the same without the S_prev term (Eq. norogna), which the SI
//               shows samples a wrong distribution when S depends on R.
// ---------------------------------------------------------------------------
enum LangevinScheme { LV_ADOPTED = 0, LV_FAST = 1, LV_NOROGNA = 2 };

static int langevin(int n, const double* R, const double* Rprev, const double* f, const double* S,
                    const double* Sprev, double T, double delta, double alpha, const double* xi,
                    int noise_correction, double box, int scheme, double* Rout) {
    double Dt = delta, Db = delta;
    if (scheme == LV_ADOPTED && alpha > 0) {
        Dt = (1.0 - std::exp(-alpha * delta)) / alpha;
        Db = (1.0 - std::exp(-2.0 * alpha * delta)) / (2.0 * alpha);
    }
    if (noise_correction) T = T - 0.5 * delta;
    std::vector<double> Lc((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {                       // Cholesky, S = L L^T
        double s = S[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
        if (!(s > 0)) return -1;
        Lc[(size_t)j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = S[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
            Lc[(size_t)i * n + j] = t / Lc[(size_t)j * n + j];
        }
    }
    std::vector<double> g(n), y(n), x(n), z(n), dR(n);
    for (int j = 0; j < n; ++j) {
        dR[j] = Rprev[j] - R[j];
        if (box > 0) dR[j] -= box * std::nearbyint(dR[j] / box);
    }
    for (int i = 0; i < n; ++i) {
        double s = 0;
        if (scheme != LV_NOROGNA)
            for (int j = 0; j < n; ++j) s += (Sprev[(size_t)i * n + j] - S[(size_t)i * n + j]) * dR[j];
        g[i] = f[i] - s / (2.0 * Db);
    }
    for (int i = 0; i < n; ++i) {                       // L y = g
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= Lc[(size_t)i * n + k] * y[k];
        y[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {                  // L^T x = y
        double s = y[i];
        for (int k = i + 1; k < n; ++k) s -= Lc[(size_t)k * n + i] * x[k];
        x[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {                  // L^T z = xi
        double s = xi[i];
        for (int k = i + 1; k < n; ++k) s -= Lc[(size_t)k * n + i] * z[k];
        z[i] = s / Lc[(size_t)i * n + i];
    }
    double amp = (T > 0) ? std::sqrt(2.0 * T * Db) : 0.0;
    for (int i = 0; i < n; ++i) {
        double r = R[i] + Dt * x[i] + amp * z[i];
        Rout[i] = box > 0 ? wrap(r, box) : r;
    }
    return 0;
}


// ---------------------------------------------------------------------------
// First simplified scheme (SI, Eq. smartMarkov) for a given S(R) and S(y), in
// its two halves: predict  y = R + sqrt(2 T D) z,  <z z^T> = S^{-1}(R)
// (z = L^{-T} xi, S(R) = L L^T), and correct
//   R' = y + D S^{-1}(R) f(R) - 1/2 S^{-1}(R) [S(y) - S(R)] (y - R).
// box > 0 wraps R' (not y) into [0, box).  Both return -1 when S(R) is not
// positive definite.
// ---------------------------------------------------------------------------
static bool cholesky(int n, const double* S, std::vector<double>& Lc) {
    Lc.assign((size_t)n * n, 0.0);
    for (int j = 0; j < n; ++j) {
        double s = S[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
        if (!(s > 0)) return false;
        Lc[(size_t)j * n + j] = std::sqrt(s);
        for (int i = j + 1; i < n; ++i) {
            double t = S[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
            Lc[(size_t)i * n + j] = t / Lc[(size_t)j * n + j];
        }
    }
    return true;
}

static int first_predict(int n, const double* R, const double* S, double T, double delta, const double* xi,
                         double* y) {
    std::vector<double> Lc;
    if (!cholesky(n, S, Lc)) return -1;
    std::vector<double> z(n);
    for (int i = n - 1; i >= 0; --i) {                  // L^T z = xi
        double s = xi[i];
        for (int k = i + 1; k < n; ++k) s -= Lc[(size_t)k * n + i] * z[k];
        z[i] = s / Lc[(size_t)i * n + i];
    }
    const double amp = T > 0 ? std::sqrt(2.0 * T * delta) : 0.0;
    for (int i = 0; i < n; ++i) y[i] = R[i] + amp * z[i];
    return 0;
}

static int first_correct(int n, const double* R, const double* f, const double* S, const double* Sy,
                         const double* y, double delta, double box, double* Rout) {
    std::vector<double> Lc;
    if (!cholesky(n, S, Lc)) return -1;
    std::vector<double> g(n), w(n), x(n);
    for (int i = 0; i < n; ++i) {
        double v = 0;
        for (int j = 0; j < n; ++j) v += (Sy[(size_t)i * n + j] - S[(size_t)i * n + j]) * (y[j] - R[j]);
        g[i] = delta * f[i] - 0.5 * v;
    }
    for (int i = 0; i < n; ++i) {                       // L w = g
        double s = g[i];
        for (int k = 0; k < i; ++k) s -= Lc[(size_t)i * n + k] * w[k];
        w[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {                  // L^T x = w
        double s = w[i];
        for (int k = i + 1; k < n; ++k) s -= Lc[(size_t)k * n + i] * x[k];
        x[i] = s / Lc[(size_t)i * n + i];
    }
    for (int i = 0; i < n; ++i) {
        const double r = y[i] + x[i];
        Rout[i] = box > 0 ? wrap(r, box) : r;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// Rotating-spring toy model (SI, "A simple toy model") and the integrator
// variants compared on it.  The end point R = (x, y) of a spring of rest
// length a and stiffness k, free to rotate about the origin:
//   U(x, y) = k/2 (sqrt(x^2 + y^2) - a)^2,   f = -grad U.
// Acceleration matrices (gamma = 0, Euclidean canonical measure):
//   TOY_S_G   S = G_lambda, the matrix printed in the SI (identity at lambda = 1)
//   TOY_S_HG  S = H + mu G_lambda, H = grad grad U (the SI's regularised Hessian)
// Schemes, one step from R (and R_prev for the two-point ones), <z z^T> = S^{-1}(R):
//   TOY_PLAIN     S = I: R' = R + D f + sqrt(2 T D) xi
//   TOY_STANDARD  Eq. standard: R' = R + D S^{-1} f + T D Gamma + sqrt(2 T D) z,
//                 Gamma_j = sum_i d_i (S^{-1})_{ji}  (the "cumbersome term")
//   TOY_FIRST     Eq. smartMarkov: y = R + sqrt(2 T D) z,
//                 R' = y + D S^{-1}(R) f(R) - 1/2 S^{-1}(R) [S(y) - S(R)] (y - R)
//   TOY_FAST      Eq. finaldyn: R' = R + D S^{-1} f + sqrt(2 T D) z
//                                 - 1/2 S^{-1} [S(R_prev) - S(R)] (R_prev - R)
//   TOY_ADOPTED   Eq. finaldyn_new: R' = R + Dt S^{-1} [f - (S(R_prev) - S(R))(R_prev - R)/(2 Db)]
//                                 + sqrt(2 T Db) z,  Dt, Db as in the hydrogen step
//   TOY_NOROGNA   Eq. norogna: R' = R + D S^{-1} f + sqrt(2 T D) z
// On the first step R_prev = R.  Derivatives (f, H, Gamma) come from nested
// forward-mode dual numbers, never from hand-derived formulas.
// ---------------------------------------------------------------------------
enum ToyScheme { TOY_PLAIN = 0, TOY_STANDARD = 1, TOY_FIRST = 2, TOY_FAST = 3, TOY_ADOPTED = 4, TOY_NOROGNA = 5 };
enum ToySMode { TOY_S_G = 0, TOY_S_HG = 1 };
constexpr uint32_t P_TOY = 8;   // Philox purpose word of the toy-model noise

// Dual number with the two tangents d/dx, d/dy over a value type V that may
// itself be a dual number (nesting gives second and third derivatives).
template <class V> struct Du {
    V v, dx, dy;
    Du() : v(0.0), dx(0.0), dy(0.0) {}
    Du(double c) : v(c), dx(0.0), dy(0.0) {}
    Du(V a, V b, V c) : v(a), dx(b), dy(c) {}
};
template <class V> Du<V> operator+(const Du<V>& a, const Du<V>& b) { return Du<V>(a.v + b.v, a.dx + b.dx, a.dy + b.dy); }
template <class V> Du<V> operator-(const Du<V>& a, const Du<V>& b) { return Du<V>(a.v - b.v, a.dx - b.dx, a.dy - b.dy); }
template <class V> Du<V> operator-(const Du<V>& a) { return Du<V>(-a.v, -a.dx, -a.dy); }
template <class V> Du<V> operator*(const Du<V>& a, const Du<V>& b) {
    return Du<V>(a.v * b.v, a.dx * b.v + a.v * b.dx, a.dy * b.v + a.v * b.dy);
}
template <class V> Du<V> operator/(const Du<V>& a, const Du<V>& b) {
    const V q = a.v / b.v;
    return Du<V>(q, (a.dx - q * b.dx) / b.v, (a.dy - q * b.dy) / b.v);
}
template <class V> Du<V> operator+(const Du<V>& a, double c) { return a + Du<V>(c); }
template <class V> Du<V> operator+(double c, const Du<V>& a) { return Du<V>(c) + a; }
template <class V> Du<V> operator-(const Du<V>& a, double c) { return a - Du<V>(c); }
template <class V> Du<V> operator-(double c, const Du<V>& a) { return Du<V>(c) - a; }
template <class V> Du<V> operator*(const Du<V>& a, double c) { return a * Du<V>(c); }
template <class V> Du<V> operator*(double c, const Du<V>& a) { return Du<V>(c) * a; }
template <class V> Du<V> operator/(const Du<V>& a, double c) { return a / Du<V>(c); }
template <class V> Du<V> operator/(double c, const Du<V>& a) { return Du<V>(c) / a; }
template <class V> Du<V> sqrt(const Du<V>& a) {
    using std::sqrt;
    const V s = sqrt(a.v);
    return Du<V>(s, a.dx / (s + s), a.dy / (s + s));
}
template <class V> Du<V> lift(const V& c) { return Du<V>(c, V(0.0), V(0.0)); }
template <class V> Du<V> seed_x(const V& x) { return Du<V>(x, V(1.0), V(0.0)); }
template <class V> Du<V> seed_y(const V& y) { return Du<V>(y, V(0.0), V(1.0)); }

struct ToyModel {
    double k, a;        // spring stiffness and rest length
    double lambda;      // G_lambda parameter, as printed
    double mu;          // weight of G_lambda in S = H + mu G_lambda
    int s_mode;         // TOY_S_G or TOY_S_HG
};

template <class V> V toy_U(const ToyModel& m, const V& x, const V& y) {
    using std::sqrt;
    const V d = sqrt(x * x + y * y) - m.a;
    return 0.5 * m.k * d * d;
}
// grad U by one level of dual numbers.
template <class V> void toy_grad(const ToyModel& m, const V& x, const V& y, V g[2]) {
    const Du<V> ux = toy_U(m, seed_x(x), lift(y));
    const Du<V> uy = toy_U(m, lift(x), seed_y(y));
    g[0] = ux.dx; g[1] = uy.dy;
}
// H = grad grad U: one more level of dual numbers on toy_grad.
template <class V> void toy_hess(const ToyModel& m, const V& x, const V& y, V H[2][2]) {
    Du<V> gx[2], gy[2];
    toy_grad(m, seed_x(x), lift(y), gx);
    toy_grad(m, lift(x), seed_y(y), gy);
    for (int i = 0; i < 2; ++i) { H[i][0] = gx[i].dx; H[i][1] = gy[i].dy; }
}
// G_lambda as printed in the SI.
template <class V> void toy_G(const ToyModel& m, const V& x, const V& y, V G[2][2]) {
    const double l = m.lambda;
    const V r2 = x * x + y * y;
    G[0][0] = (x * x + y * y * l) / (r2 * l);
    G[0][1] = (x * y * (1.0 - l)) / (r2 * l);
    G[1][0] = G[0][1];
    G[1][1] = (x * x * l + y * y) / (r2 * l);
}
template <class V> void toy_S(const ToyModel& m, const V& x, const V& y, V S[2][2]) {
    toy_G(m, x, y, S);
    if (m.s_mode == TOY_S_HG) {
        V H[2][2];
        toy_hess(m, x, y, H);
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) S[i][j] = H[i][j] + m.mu * S[i][j];
    }
}
// S^{-1} by the 2x2 adjugate formula.
template <class V> void toy_Sinv(const ToyModel& m, const V& x, const V& y, V Si[2][2]) {
    V S[2][2];
    toy_S(m, x, y, S);
    const V det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
    Si[0][0] = S[1][1] / det; Si[0][1] = -S[0][1] / det;
    Si[1][0] = -S[1][0] / det; Si[1][1] = S[0][0] / det;
}
// Gamma_j = sum_i d_i (S^{-1})_{ji} (SI, Eq. for the cumbersome term).
static void toy_gamma(const ToyModel& m, double x, double y, double Gam[2]) {
    Du<double> Sx[2][2], Sy[2][2];
    toy_Sinv(m, seed_x(x), lift(y), Sx);
    toy_Sinv(m, lift(x), seed_y(y), Sy);
    for (int j = 0; j < 2; ++j) Gam[j] = Sx[j][0].dx + Sy[j][1].dy;
}

// 2x2 Cholesky S = L L^T; false if S is not positive definite.
static bool chol2(const double S[2][2], double L[2][2]) {
    if (!(S[0][0] > 0)) return false;
    L[0][0] = std::sqrt(S[0][0]); L[0][1] = 0.0;
    L[1][0] = S[1][0] / L[0][0];
    const double d = S[1][1] - L[1][0] * L[1][0];
    if (!(d > 0)) return false;
    L[1][1] = std::sqrt(d);
    return true;
}
static void chol2_solve(const double L[2][2], const double b[2], double x[2]) {     // S x = b
    const double y0 = b[0] / L[0][0], y1 = (b[1] - L[1][0] * y0) / L[1][1];
    x[1] = y1 / L[1][1];
    x[0] = (y0 - L[1][0] * x[1]) / L[0][0];
}
static void chol2_noise(const double L[2][2], const double xi[2], double z[2]) {   // z = L^{-T} xi
    z[1] = xi[1] / L[1][1];
    z[0] = (xi[0] - L[1][0] * z[1]) / L[0][0];
}

struct ToyStep {
    ToyModel m;
    double T, delta, alpha;
    int scheme;
};

// One step of the selected scheme from R (R_prev used by TOY_FAST / TOY_ADOPTED).
// Returns false when S(R) is not positive definite.
static bool toy_step(const ToyStep& c, const double R[2], const double Rp[2], const double xi[2], double Rn[2]) {
    const ToyModel& m = c.m;
    double g[2];
    toy_grad(m, R[0], R[1], g);
    const double f[2] = {-g[0], -g[1]};
    const double D = c.delta, T = c.T > 0 ? c.T : 0.0;
    if (c.scheme == TOY_PLAIN) {
        const double amp = std::sqrt(2.0 * T * D);
        for (int j = 0; j < 2; ++j) Rn[j] = R[j] + D * f[j] + amp * xi[j];
        return true;
    }
    double S[2][2], L[2][2], z[2], sf[2];
    toy_S(m, R[0], R[1], S);
    if (!chol2(S, L)) return false;
    chol2_noise(L, xi, z);
    chol2_solve(L, f, sf);
    const double amp = std::sqrt(2.0 * T * D);
    switch (c.scheme) {
    case TOY_STANDARD: {
        double Gam[2];
        toy_gamma(m, R[0], R[1], Gam);
        for (int j = 0; j < 2; ++j) Rn[j] = R[j] + D * sf[j] + T * D * Gam[j] + amp * z[j];
        return true;
    }
    case TOY_FIRST: {
        double y[2], Sy[2][2], v[2], w[2];
        for (int j = 0; j < 2; ++j) y[j] = R[j] + amp * z[j];
        toy_S(m, y[0], y[1], Sy);
        for (int i = 0; i < 2; ++i) {
            v[i] = 0.0;
            for (int j = 0; j < 2; ++j) v[i] += (Sy[i][j] - S[i][j]) * (y[j] - R[j]);
        }
        chol2_solve(L, v, w);
        for (int j = 0; j < 2; ++j) Rn[j] = y[j] + D * sf[j] - 0.5 * w[j];
        return true;
    }
    case TOY_FAST: {
        double Sp[2][2], v[2], w[2];
        toy_S(m, Rp[0], Rp[1], Sp);
        for (int i = 0; i < 2; ++i) {
            v[i] = 0.0;
            for (int j = 0; j < 2; ++j) v[i] += (Sp[i][j] - S[i][j]) * (Rp[j] - R[j]);
        }
        chol2_solve(L, v, w);
        for (int j = 0; j < 2; ++j) Rn[j] = R[j] + D * sf[j] + amp * z[j] - 0.5 * w[j];
        return true;
    }
    case TOY_ADOPTED: {
        double Dt = D, Db = D;
        if (c.alpha > 0) {
            Dt = (1.0 - std::exp(-c.alpha * D)) / c.alpha;
            Db = (1.0 - std::exp(-2.0 * c.alpha * D)) / (2.0 * c.alpha);
        }
        double Sp[2][2], h[2], x[2];
        toy_S(m, Rp[0], Rp[1], Sp);
        for (int i = 0; i < 2; ++i) {
            double v = 0.0;
            for (int j = 0; j < 2; ++j) v += (Sp[i][j] - S[i][j]) * (Rp[j] - R[j]);
            h[i] = f[i] - v / (2.0 * Db);
        }
        chol2_solve(L, h, x);
        const double ampb = std::sqrt(2.0 * T * Db);
        for (int j = 0; j < 2; ++j) Rn[j] = R[j] + Dt * x[j] + ampb * z[j];
        return true;
    }
    default:   // TOY_NOROGNA
        for (int j = 0; j < 2; ++j) Rn[j] = R[j] + D * sf[j] + amp * z[j];
        return true;
    }
}

// Two standard normals from one Philox block (Box-Muller, both branches),
// counter = (trajectory, step, 0, P_TOY).
static void toy_noise(const Rng& rng, uint32_t traj, uint32_t step, double xi[2]) {
    uint32_t w[4];
    rng.block(traj, step, 0u, P_TOY, w);
    const double u1 = uniform53(w[0], w[1]), u2 = uniform53(w[2], w[3]);
    const double rho = std::sqrt(-2.0 * std::log(u1));
    xi[0] = rho * std::cos(2.0 * M_PI * u2);
    xi[1] = rho * std::sin(2.0 * M_PI * u2);
}

// One trajectory of n_steps steps from xy0.  out = [x, y, sum U, sum U^2,
// sum |R|, unwrapped polar angle travelled, status]; the sums run over the
// positions after steps n_burn..n_steps-1; status = 0, or s+1 when S was not
// positive definite at step s (the trajectory stops there).
static void toy_run(const ToyStep& c, const Rng& rng, uint32_t traj, int n_steps, int n_burn, const double xy0[2],
                    double out[7]) {
    double R[2] = {xy0[0], xy0[1]}, Rp[2] = {xy0[0], xy0[1]}, Rn[2], xi[2];
    double su = 0.0, su2 = 0.0, sr = 0.0, theta = 0.0, status = 0.0;
    for (int s = 0; s < n_steps; ++s) {
        toy_noise(rng, traj, (uint32_t)s, xi);
        if (!toy_step(c, R, Rp, xi, Rn)) { status = s + 1; break; }
        theta += std::atan2(R[0] * Rn[1] - R[1] * Rn[0], R[0] * Rn[0] + R[1] * Rn[1]);
        Rp[0] = R[0]; Rp[1] = R[1];
        R[0] = Rn[0]; R[1] = Rn[1];
        if (s >= n_burn) {
            const double u = toy_U(c.m, R[0], R[1]);
            su += u; su2 += u * u; sr += std::sqrt(R[0] * R[0] + R[1] * R[1]);
        }
    }
    out[0] = R[0]; out[1] = R[1]; out[2] = su; out[3] = su2; out[4] = sr; out[5] = theta; out[6] = status;
}

}  // namespace orc

// ===========================================================================
// extern "C" surface used by the Python test harness (oracle/oracle.py)
// ===========================================================================
extern "C" {

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { orc::philox4x32_10(ctr, key, out); }

double orc_uniform(uint64_t seed, uint32_t s, uint32_t m, uint32_t idx, uint32_t purpose) {
    return orc::Rng(seed).uniform(s, m, idx, purpose);
}
double orc_normal(uint64_t seed, uint32_t s, uint32_t m, uint32_t idx, uint32_t purpose) {
    return orc::Rng(seed).normal(s, m, idx, purpose);
}

double orc_ewald(int nq, const double* q, const double* pos, double L, double kappa, int mmax, int background) {
    return orc::ewald<double>(nq, q, pos, L, kappa, mmax, background != 0);
}

// One configuration X ([Ne][3]) at nuclei R ([N][3]).  out_scalars = {lnpsi,
// sign, E_L, E_kin, E_pot}; grad = grad_i ln psi [Ne][3]; dlnpsi, del = d/dR
// [N][3] (only when derivs != 0).  Returns 0, or -1 for a singular Slater block.
int orc_eval_config(const orc::Params* p, const double* R, const double* X, int derivs,
                    double* out_scalars, double* grad, double* dlnpsi, double* del) {
    orc::ConfigResult r = orc::eval_config(*p, R, X, derivs != 0);
    if (!r.ok) return -1;
    out_scalars[0] = r.lnpsi; out_scalars[1] = r.sign; out_scalars[2] = r.el;
    out_scalars[3] = r.ekin; out_scalars[4] = r.epot;
    const int Ne = p->n_up + p->n_dn;
    if (grad) std::memcpy(grad, r.grad.data(), sizeof(double) * 3 * Ne);
    if (derivs) {
        std::memcpy(dlnpsi, r.dlnpsi.data(), sizeof(double) * 3 * p->N);
        std::memcpy(del, r.del.data(), sizeof(double) * 3 * p->N);
    }
    return 0;
}

// Many configurations at once (walker-parallel): X [nconf][Ne][3].
// The R-derivatives take one dual-number pass per (configuration, nucleus);
// the passes are independent, so the threads share them out over both indices
// (each pass is the same computation as in eval_config).
int orc_eval_configs(const orc::Params* p, const double* R, int nconf, const double* X, int derivs,
                     double* lnpsi, double* el, double* dlnpsi, double* del) {
    const int Ne = p->n_up + p->n_dn, N3 = 3 * p->N, N = p->N;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
    for (int c = 0; c < nconf; ++c) {
        orc::ConfigResult r = orc::eval_config(*p, R, X + (size_t)c * 3 * Ne, false);
        if (!r.ok) { ++bad; continue; }
        lnpsi[c] = r.lnpsi; el[c] = r.el;
    }
    if (bad || !derivs) return bad ? -1 : 0;
#pragma omp parallel for schedule(dynamic) collapse(2)
    for (int c = 0; c < nconf; ++c)
        for (int a = 0; a < N; ++a) {
            std::vector<orc::D3> Rd((size_t)N3);
            for (int k = 0; k < N3; ++k) Rd[k] = orc::D3(R[k]);
            for (int mu = 0; mu < 3; ++mu) Rd[3 * a + mu].d[mu] = 1.0;
            orc::WfOut<orc::D3> wd = orc::wavefunction<orc::D3>(*p, Rd.data(), X + (size_t)c * 3 * Ne);
            for (int mu = 0; mu < 3; ++mu) {
                dlnpsi[(size_t)c * N3 + 3 * a + mu] = wd.lnpsi.d[mu];
                del[(size_t)c * N3 + 3 * a + mu] = wd.el.d[mu];
            }
        }
    return 0;
}

// Slater matrices at one configuration X [Ne][3]: out [Ne][n_orb], row i =
// phi_j(r_i) for j < n_orb (spin-up rows first, then spin-down rows); used by
// the tests to state the condition numbers of their inputs.
void orc_slater_matrices(const orc::Params* p, const double* R, const double* X, double* out) {
    const int Ne = p->n_up + p->n_dn;
    for (int i = 0; i < Ne; ++i) orc::slater_row(*p, R, X + 3 * i, p->n_orb, out + (size_t)i * p->n_orb);
}

// Change of U when electron i of X moves to xn (the Metropolis Jastrow ratio's exponent).
double orc_jastrow_delta(const orc::Params* p, const double* R, const double* X, int i, const double* xn) {
    return orc::jastrow_delta(*p, R, X, i, xn);
}

// Walker start positions, X [W][Ne][3].
void orc_init_walkers(const orc::Params* p, const double* R, int W, uint64_t seed, double* X) {
    const int Ne = p->n_up + p->n_dn;
    orc::Rng rng(seed);
    for (int w = 0; w < W; ++w) orc::init_walker(*p, rng, (uint32_t)w, R, X + (size_t)w * 3 * Ne);
}

// VMC chains of W walkers; X [W][Ne][3] in/out; acc [W][3 + 9N] accumulated
// (caller zeroes it); n_accept / n_try summed over walkers.
// vacc [W] (or null) accumulates each walker's sum of the sampled potential energy V_L.
void orc_vmc_v(const orc::Params* p, const double* R, const orc::ChainArgs* c, double* X, double* acc, double* vacc,
               long long* n_accept, long long* n_try) {
    const int Ne = p->n_up + p->n_dn, stride = 3 + 9 * p->N;
    orc::Rng rng(c->seed);
    long long na = 0, nt = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : na, nt)
    for (int w = 0; w < c->W; ++w) {
        long long a = 0, t = 0;
        orc::run_walker(*p, *c, rng, (uint32_t)w, R, X + (size_t)w * 3 * Ne, acc + (size_t)w * stride,
                        vacc ? vacc + w : nullptr, &a, &t);
        na += a; nt += t;
    }
    *n_accept = na; *n_try = nt;
}

void orc_vmc(const orc::Params* p, const double* R, const orc::ChainArgs* c, double* X, double* acc,
             long long* n_accept, long long* n_try) {
    orc_vmc_v(p, R, c, X, acc, nullptr, n_accept, n_try);
}

// Pressure of a cubic cell of volume omega from the chains' accumulators (the
// paper reports P(rho) along isotherms but does not state its estimator;
// reading: the virial of the Coulomb system).  Every term of the Hamiltonian
// is a kinetic term (degree -2) or a Coulomb term (degree -1) in the lengths,
// so the trial state scaled with the cell has E(lambda) = <T>/lambda^2 +
// <V>/lambda, and -dE/dOmega = (2<T> + <V>)/(3 Omega), with <T> = <E_L> - <V_L>.
// Classical nuclei at temperature T_nuc add the ideal-gas term N T_nuc / Omega.
// out = [P, error bar from walker blocks, electronic part, <V_L>, <T_L>].
void orc_pressure(int W, int N, const double* acc, const double* vacc, double omega, double T_nuc, double* out) {
    const int stride = 3 + 9 * N;
    double c = 0, e = 0, v = 0;
    for (int w = 0; w < W; ++w) { c += acc[(size_t)w * stride]; e += acc[(size_t)w * stride + 1]; v += vacc[w]; }
    const double E = e / c, V = v / c, T = E - V;
    const double Pel = (2.0 * T + V) / (3.0 * omega);
    double d2 = 0;
    for (int w = 0; w < W; ++w) {
        const double cw = acc[(size_t)w * stride];
        const double Ew = acc[(size_t)w * stride + 1] / cw, Vw = vacc[w] / cw;
        const double pw = (2.0 * (Ew - Vw) + Vw) / (3.0 * omega);
        d2 += (pw - Pel) * (pw - Pel);
    }
    out[0] = Pel + N * T_nuc / omega;
    out[1] = W > 1 ? std::sqrt(d2 / ((double)W * (W - 1))) : 0.0;
    out[2] = Pel;
    out[3] = V;
    out[4] = T;
}

void orc_reduce(int W, int N3, const double* acc, double* E, double* Eerr, double* f, double* S, double* Nc) {
    orc::reduce(W, N3, acc, E, Eerr, f, S, Nc);
}

void orc_reduce_twists(int K, int W, int N3, const double* acc, double* E, double* Eerr, double* f, double* S,
                       double* Nc) {
    orc::reduce_twists(K, W, N3, acc, E, Eerr, f, S, Nc);
}

// ---- empirical acceleration matrix S = H + mu I ----

double orc_empirical_energy(int N, double L, const double* R, double lambda) {
    return orc::empirical_energy<double>(N, L, R, lambda);
}

void orc_empirical_s(int N, double L, const double* R, double lambda, double mu, double* S) {
    orc::empirical_s(N, L, R, lambda, mu, S);
}

// ---- twisted boundary conditions (p->twist set) ----

int orc_bloch_images(const orc::Params* p) { return orc::bloch_images(*p); }

// One Bloch-summed Gaussian at x for a nucleus at Rc: out [10] = chi (re, im),
// grad chi (re, im per component), lap chi (re, im).
void orc_bloch_gaussian(double L, const double* x, const double* Rc, double zeta, const double* th, int M,
                        double* out) {
    orc::Cx<double> c, g[3], l;
    orc::bloch_gaussian<double>(L, x, Rc, zeta, th, M, c, g, l);
    out[0] = c.re; out[1] = c.im;
    for (int mu = 0; mu < 3; ++mu) { out[2 + 2 * mu] = g[mu].re; out[3 + 2 * mu] = g[mu].im; }
    out[8] = l.re; out[9] = l.im;
}

// One configuration with twisted orbitals: out_scalars = {ln|psi|, arg psi,
// E_L, Re E_kin, Im E_kin, E_pot}; grad = Re grad_i ln psi; dlnpsi, del as in
// orc_eval_config.  Returns 0, or -1 for a singular Slater block.
int orc_eval_config_twist(const orc::Params* p, const double* R, const double* X, int derivs, double* out_scalars,
                          double* grad, double* dlnpsi, double* del) {
    if (!p->twist) return -2;
    orc::TwistResult r = orc::eval_config_twist(*p, R, X, derivs != 0);
    if (!r.ok) return -1;
    out_scalars[0] = r.lnpsi; out_scalars[1] = r.phase; out_scalars[2] = r.el;
    out_scalars[3] = r.ekin; out_scalars[4] = r.ekin_im; out_scalars[5] = r.epot;
    const int Ne = p->n_up + p->n_dn;
    if (grad) std::memcpy(grad, r.grad.data(), sizeof(double) * 3 * Ne);
    if (derivs) {
        std::memcpy(dlnpsi, r.dlnpsi.data(), sizeof(double) * 3 * p->N);
        std::memcpy(del, r.del.data(), sizeof(double) * 3 * p->N);
    }
    return 0;
}

// Many configurations, twist twists[3 * (c / (nconf / K))] for configuration c
// (K contiguous blocks); outputs as orc_eval_configs.
int orc_eval_configs_twist(const orc::Params* p, const double* R, int nconf, const double* X, int K,
                           const double* twists, int derivs, double* lnpsi, double* el, double* dlnpsi, double* del) {
    const int Ne = p->n_up + p->n_dn, N3 = 3 * p->N;
    if (K < 1 || nconf % K) return -2;
    const int per = nconf / K;
    int bad = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : bad)
    for (int c = 0; c < nconf; ++c) {
        orc::Params q = *p;
        q.twist = twists + 3 * (c / per);
        orc::TwistResult r = orc::eval_config_twist(q, R, X + (size_t)c * 3 * Ne, derivs != 0);
        if (!r.ok) { ++bad; continue; }
        lnpsi[c] = r.lnpsi; el[c] = r.el;
        if (derivs)
            for (int k = 0; k < N3; ++k) {
                dlnpsi[(size_t)c * N3 + k] = r.dlnpsi[k];
                del[(size_t)c * N3 + k] = r.del[k];
            }
    }
    return bad ? -1 : 0;
}

// VMC chains with twisted orbitals: walker w samples twist
// twists[3 * (w / (W / K))] (K contiguous blocks, W a multiple of K); the
// rest as orc_vmc_v.
int orc_vmc_twists(const orc::Params* p, const double* R, const orc::ChainArgs* c, int K, const double* twists,
                   double* X, double* acc, double* vacc, long long* n_accept, long long* n_try) {
    if (K < 1 || c->W % K) return -2;
    const int Ne = p->n_up + p->n_dn, stride = 3 + 9 * p->N, per = c->W / K;
    orc::Rng rng(c->seed);
    long long na = 0, nt = 0;
#pragma omp parallel for schedule(dynamic) reduction(+ : na, nt)
    for (int w = 0; w < c->W; ++w) {
        orc::Params q = *p;
        q.twist = twists + 3 * (w / per);
        long long a = 0, t = 0;
        orc::run_walker_twist(q, *c, rng, (uint32_t)w, R, X + (size_t)w * 3 * Ne, acc + (size_t)w * stride,
                              vacc ? vacc + w : nullptr, &a, &t);
        na += a; nt += t;
    }
    *n_accept = na; *n_try = nt;
    return 0;
}

int orc_langevin(int n, const double* R, const double* Rprev, const double* f, const double* S,
                 const double* Sprev, double T, double delta, double alpha, const double* xi,
                 int noise_correction, double box, int scheme, double* Rout) {
    return orc::langevin(n, R, Rprev, f, S, Sprev, T, delta, alpha, xi, noise_correction, box, scheme, Rout);
}

int orc_langevin_first_predict(int n, const double* R, const double* S, double T, double delta, const double* xi,
                               double* y) {
    return orc::first_predict(n, R, S, T, delta, xi, y);
}
int orc_langevin_first_correct(int n, const double* R, const double* f, const double* S, const double* Sy,
                               const double* y, double delta, double box, double* Rout) {
    return orc::first_correct(n, R, f, S, Sy, y, delta, box, Rout);
}

// Langevin noise xi_c for component c of MD step m (Philox, purpose P_LANGEVIN).
void orc_langevin_noise(uint64_t seed, uint32_t md_step, int n, double* xi) {
    orc::Rng rng(seed);
    for (int c = 0; c < n; ++c) xi[c] = rng.normal((uint32_t)c, md_step, 0u, orc::P_LANGEVIN);
}

// ---- toy model ----
struct ToyArgs {
    double k, a, T, delta, lambda, mu, alpha;
    int32_t scheme, s_mode, n_steps, n_burn;
    uint64_t seed;
};
static orc::ToyStep toy_cfg(const ToyArgs* a) {
    orc::ToyStep c;
    c.m.k = a->k; c.m.a = a->a; c.m.lambda = a->lambda; c.m.mu = a->mu; c.m.s_mode = a->s_mode;
    c.T = a->T; c.delta = a->delta; c.alpha = a->alpha; c.scheme = a->scheme;
    return c;
}
// Model quantities at (x, y): out = [U, f_x, f_y, S (4), S^{-1} (4), H (4), Gamma (2)].
void orc_toy_eval(const ToyArgs* a, double x, double y, double* out) {
    const orc::ToyStep c = toy_cfg(a);
    double g[2], S[2][2], Si[2][2], H[2][2], Gam[2];
    orc::toy_grad(c.m, x, y, g);
    orc::toy_S(c.m, x, y, S);
    orc::toy_Sinv(c.m, x, y, Si);
    orc::toy_hess(c.m, x, y, H);
    orc::toy_gamma(c.m, x, y, Gam);
    out[0] = orc::toy_U(c.m, x, y); out[1] = -g[0]; out[2] = -g[1];
    for (int i = 0; i < 4; ++i) { out[3 + i] = S[i / 2][i % 2]; out[7 + i] = Si[i / 2][i % 2]; out[11 + i] = H[i / 2][i % 2]; }
    out[15] = Gam[0]; out[16] = Gam[1];
}
// One step of the scheme in a->scheme from R (R_prev = Rp) with the given xi; 0 or -1 (S not PD).
int orc_toy_step(const ToyArgs* a, const double* R, const double* Rp, const double* xi, double* Rn) {
    return orc::toy_step(toy_cfg(a), R, Rp, xi, Rn) ? 0 : -1;
}
// n_traj independent trajectories (OpenMP over trajectories); xy0 [n_traj][2], out [n_traj][7].
void orc_toy_run(const ToyArgs* a, int n_traj, const double* xy0, double* out) {
    const orc::ToyStep c = toy_cfg(a);
    const orc::Rng rng(a->seed);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n_traj; ++t)
        orc::toy_run(c, rng, (uint32_t)t, a->n_steps, a->n_burn, xy0 + 2 * (size_t)t, out + 7 * (size_t)t);
}
// The same for selected trajectories of a larger run: ids [n] are their indices
// there (the Philox stream), xy0 [n][2] their start points, out [n][7].
void orc_toy_run_ids(const ToyArgs* a, int n, const int* ids, const double* xy0, double* out) {
    const orc::ToyStep c = toy_cfg(a);
    const orc::Rng rng(a->seed);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < n; ++t)
        orc::toy_run(c, rng, (uint32_t)ids[t], a->n_steps, a->n_burn, xy0 + 2 * (size_t)t, out + 7 * (size_t)t);
}
// The two toy-model normals of (trajectory, step).
void orc_toy_noise(uint64_t seed, uint32_t traj, uint32_t step, double* xi) {
    orc::toy_noise(orc::Rng(seed), traj, step, xi);
}

int orc_num_threads() {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

}  // extern "C"
