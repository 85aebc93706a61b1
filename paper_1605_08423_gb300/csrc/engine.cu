// engine.cu -- the qmc_system handle: device state of one system (walkers,
// inverses, tables), the schedule of one energy/force call and every entry
// point of include/qmcmd.h.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/qmcmd.h"
#include "common.cuh"
#include "kernels.cuh"
#include "pool.h"

using namespace qmc;

namespace {

constexpr double kBoltzmannHaPerK = 3.166811563e-6;

const char* kKernelNames[QMC_NKERNEL] = {"propose", "orbitals_prop", "sweep",  "recompute", "orbitals_meas",
                                         "measure", "reduce",        "langevin", "adjoint"};
enum {
    KC_PROPOSE = 0, KC_ORB_PROP, KC_SWEEP, KC_RECOMPUTE, KC_ORB_MEAS, KC_MEASURE, KC_REDUCE, KC_LANGEVIN, KC_ADJOINT
};

struct EventPair { cudaEvent_t a, b; int cls; };

}  // namespace

struct qmc_system {
    qmc_params p;
    std::vector<double> zeta_h, coeff_h, fj_h;
    double* d_fj = nullptr;    // e-e-n-n Jastrow coefficients [N][N]
    float* d_fj32 = nullptr;   // the same in FP32 (mixed form)
    int N, n, G, B, W, nk, mmax;
    bool mixed;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    // tables
    double *d_R = nullptr, *d_zeta = nullptr, *d_C64 = nullptr, *d_kw = nullptr, *d_ptrig64 = nullptr;
    float *d_C32 = nullptr, *d_ptrig32 = nullptr;
    int4* d_kvec = nullptr;
    double2 *d_eikR = nullptr, *d_rhop = nullptr;
    double *d_vconst = nullptr, *d_dvpp = nullptr;
    float *d_R32 = nullptr, *d_kw32 = nullptr, *d_zeta32 = nullptr;
    void* d_ptp = nullptr;     // (sin, cos)(pi x'/L) of the proposals of the current sweep
    float2* d_eikR32 = nullptr;
    void* d_chat = nullptr;    // C^T chunks, TF32 hi/lo, swizzled (tensor-core orbital kernel)
    bool use_tc = false;
    // tensor-core adjoint (mixed form): C rows per Gaussian in TF32 pieces,
    // K^T per walker-spin, electron data and E_L per walker
    void* d_ahat = nullptr;
    float *d_Kt = nullptr, *d_eg = nullptr;
    double* d_elw = nullptr;
    bool use_tc_adj = false;
    // reciprocal-space force as one GEMM over walkers (split path):
    // F[W][3N] = rho[W][2 nk] . T^T, T = [3N][2 nk] built per R
    float *d_Trec = nullptr, *d_rk = nullptr, *d_frec = nullptr;
    // walkers
    double *d_X = nullptr, *d_Xp = nullptr;
    void *d_uacc = nullptr, *d_Phi = nullptr, *d_Gt = nullptr, *d_D = nullptr, *d_Lp = nullptr;
    double* d_logdet = nullptr;
    double* d_acc = nullptr;
    double* d_vacc = nullptr;    // per-walker sums of V_L (virial pressure)
    float* d_vep = nullptr;      // per-electron e-n Jastrow sums carried by the mixed sweep
    double* d_pout = nullptr;    // pressure output [5]
    unsigned long long* d_nacc = nullptr;
    // reductions and output
    double *d_colsum = nullptr, *d_dev = nullptr, *d_out = nullptr;
    double *d_eval = nullptr;  // eval_config outputs
    // Langevin
    double *d_Rl = nullptr, *d_Rprev = nullptr, *d_f = nullptr, *d_S = nullptr, *d_Sprev = nullptr, *d_Lwork = nullptr;
    // first simplified scheme between its two halves: R, f(R), S(R) and the factor of S(R)
    double *d_fsR = nullptr, *d_fsf = nullptr, *d_fsS = nullptr, *d_fsL = nullptr;
    bool fs_pending = false;
    double fs_delta = 0.0;
    int* d_err = nullptr;
    std::vector<void*> allocs;
    // device block the handle's arrays are carved from (server admission), or none
    unsigned char* pool = nullptr;
    size_t pool_bytes = 0, pool_off = 0;
    uint32_t md_step = 0;
    uint32_t w0 = 0;                     // QMC_OPT_WALKER_OFFSET: Philox stream of walker 0
    bool first_call = true;
    int lv_scheme = kLvAdopted;          // QMC_OPT_INTEGRATOR
    bool lv_noise_correction = false;    // QMC_OPT_NOISE_CORRECTION
    bool ns_recompute = false;           // QMC_OPT_RECOMPUTE == QMC_RECOMPUTE_NEWTON (mixed form only)
    bool langevin_first = true;
    // QMC_S_EMPIRICAL: screening length (bohr) and shift (Ha/bohr^2) of S = H + mu I
    double emp_lambda = 0.0, emp_mu = 0.5;
    uint32_t langevin_step_no = 0;
    double last_Nc = 0.0;
    // twisted boundary conditions (FP64 form): K twists, walker blocks of W/K;
    // the twist vectors and their phase table; the real inputs of the FP64
    // measure kernel (D', Lp' with Re g, Re l in column 0, unit inverse rows,
    // zero coefficients); E_L and ln|psi| per walker; the per-twist results
    // before the average
    int K = 0;
    TwistView tv{};
    std::vector<double> twist_h;
    double* d_theta = nullptr;
    double2* d_tph = nullptr;
    double *d_Dr = nullptr, *d_Lpr = nullptr, *d_Gtr = nullptr, *d_Czero = nullptr;
    double *d_elt = nullptr, *d_lpt = nullptr, *d_tout = nullptr;
    long long nlaunch = 0;  // kernels launched by this handle
    bool profiling = false;
    std::vector<EventPair> events, free_events;
    double ktime[QMC_NKERNEL] = {0};
    long long klaunch[QMC_NKERNEL] = {0};
};

namespace {

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? QMC_OK : QMC_ERR_CUDA; }

template <typename T>
T* dalloc(qmc_system* h, size_t count, int* rc) {
    void* p = nullptr;
    if (*rc != QMC_OK) return nullptr;
    if (count == 0) count = 1;
    if (h->pool) {   // carve from the caller's block, 256-byte aligned
        const size_t bytes = (count * sizeof(T) + kPoolAlign - 1) & ~(kPoolAlign - 1);
        if (h->pool_off + bytes > h->pool_bytes) { *rc = QMC_ERR_OOM; return nullptr; }
        p = h->pool + h->pool_off;
        h->pool_off += bytes;
        return (T*)p;
    }
    if (cudaMalloc(&p, count * sizeof(T)) != cudaSuccess) {
        *rc = QMC_ERR_OOM;
        cudaGetLastError();
        return nullptr;
    }
    h->allocs.push_back(p);
    return (T*)p;
}

void enumerate_kvec(int mmax, std::vector<int4>& kv) {
    // half space: mx > 0, or mx == 0 and my > 0, or mx == my == 0 and mz > 0; 0 < |m|^2 <= mmax^2
    for (int mx = 0; mx <= mmax; ++mx)
        for (int my = -mmax; my <= mmax; ++my)
            for (int mz = -mmax; mz <= mmax; ++mz) {
                const bool half = mx > 0 || (mx == 0 && my > 0) || (mx == 0 && my == 0 && mz > 0);
                if (half && mx * mx + my * my + mz * mz <= mmax * mmax) kv.push_back(make_int4(mx, my, mz, 0));
            }
}

// Images per axis of the Bloch-summed Gaussians (twisted orbitals): every
// omitted image lies more than sqrt(40 / zeta_min) away from the electron.
int bloch_images(const qmc_params* p) {
    double zmin = p->zeta[0];
    for (int g = 1; g < p->n_gauss; ++g) zmin = p->zeta[g] < zmin ? p->zeta[g] : zmin;
    const int M = (int)std::ceil(std::sqrt(40.0 / zmin) / p->L - 0.5);
    return M < 1 ? 1 : M;
}

// Thomas-Fermi screening length of the electron gas of N electrons in the box:
// k_F = (3 pi^2 N / L^3)^(1/3), k_TF^2 = 4 k_F / pi (hartree units), lambda = 1 / k_TF.
double thomas_fermi_length(int N, double L) {
    const double kF = std::cbrt(3.0 * kPi * kPi * N / (L * L * L));
    return 1.0 / std::sqrt(4.0 * kF / kPi);
}

int validate(const qmc_params* p) {
    if (!p || !p->zeta || !p->coeff) return QMC_ERR_INVALID;
    if (p->n_protons < 2 || p->n_protons > 128 || (p->n_protons & 1)) return QMC_ERR_INVALID;
    if (p->n_gauss < 1 || p->n_gauss > 8) return QMC_ERR_INVALID;
    if (p->n_walkers < 2 || p->n_sweeps < 1 || p->n_warmup < 0 || p->n_warmup_cont < 0) return QMC_ERR_INVALID;
    if (p->measure_every < 1 || p->recompute_every < 1) return QMC_ERR_INVALID;
    if (p->precision != QMC_FP64 && p->precision != QMC_MIXED) return QMC_ERR_INVALID;
    if (p->ewald_mmax < 1 || p->ewald_mmax > 12) return QMC_ERR_INVALID;
    if (!(p->L > 0) || !(p->ewald_kappa > 0) || !(p->sigma > 0) || p->b_ee < 0 || p->b_ep < 0) return QMC_ERR_INVALID;
    if (p->fj && !(p->zeta_j > 0)) return QMC_ERR_INVALID;
    if (p->n_sweeps / p->measure_every < 1) return QMC_ERR_INVALID;
    if (p->n_twist < 0) return QMC_ERR_INVALID;
    if (p->n_twist > 0) {   // twisted boundary conditions: FP64 form, whole walker blocks
        if (!p->twist || p->precision != QMC_FP64) return QMC_ERR_INVALID;
        if (p->n_walkers % p->n_twist || p->n_walkers / p->n_twist < 2) return QMC_ERR_INVALID;
        for (int k = 0; k < 3 * p->n_twist; ++k)
            if (!std::isfinite(p->twist[k])) return QMC_ERR_INVALID;
        for (int g = 0; g < p->n_gauss; ++g)
            if (!(p->zeta[g] > 0)) return QMC_ERR_INVALID;
    }
    if (p->fj) {   // the kernels use row a of f as its column a: f must be exactly symmetric
        const int N = p->n_protons;
        for (int a = 0; a < N; ++a)
            for (int b = a + 1; b < N; ++b)
                if (!(p->fj[(size_t)a * N + b] == p->fj[(size_t)b * N + a])) return QMC_ERR_INVALID;
    }
    return QMC_OK;
}

size_t footprint(const qmc_params* p) {
    const size_t N = p->n_protons, n = N / 2, G = p->n_gauss, B = N * G, W = p->n_walkers;
    const size_t t = p->precision == QMC_MIXED ? 4 : 8;
    int nkc = 0;
    for (int mx = 0; mx <= p->ewald_mmax; ++mx)
        for (int my = -p->ewald_mmax; my <= p->ewald_mmax; ++my)
            for (int mz = -p->ewald_mmax; mz <= p->ewald_mmax; ++mz) {
                const bool half = mx > 0 || (mx == 0 && my > 0) || (mx == 0 && my == 0 && mz > 0);
                if (half && mx * mx + my * my + mz * mz <= p->ewald_mmax * p->ewald_mmax) ++nkc;
            }
    const size_t nk = nkc;
    size_t b = 0;
    b += 8 * (3 * N + G + B * n + 6 * N + 3 * N + 2) + 4 * (B * n + 6 * N) + 16 * nk + 8 * nk + 16 * (N * nk + nk);
    b += 4 * (3 * N + G + nk) + 8 * N * nk + 4;      // FP32 copies of R, zeta, kw, exp(i k.R); error word
    b += t * W * N * 6;                              // proposal trig
    b += 8 * 2 * W * 3 * N;                          // X, Xp
    const size_t tc = p->n_twist > 0 ? 16 : t;     // complex orbitals of the twisted form
    b += t * W * N + tc * (W * N * n + 2 * W * n * n + 3 * W * N * n + W * N * n);   // uacc, Phi, Gt, D, Lp
    b += 8 * 2 * W + 8 * W * (3 + 9 * N) + 8 * W;   // logdet, acc, nacc
    b += 8 * W + 8 * 5;                              // V_L sums, pressure output
    b += 8 * (4 + 9 * N) + 8 * W * (3 * N + 1) + 8 * (4 + 3 * N + 9 * N * N);   // colsum, dev, out
    b += 8 * (2 * W + 6 * W * N);                    // eval outputs
    b += 8 * (3 * 3 * N + 3 * 9 * N * N);           // Langevin
    b += 8 * (2 * 3 * N + 2 * 9 * N * N);           // first simplified scheme between its halves
    if (p->fj) b += (t == 4 ? 12 : 8) * N * N;       // e-e-n-n Jastrow coefficients (+ FP32 copy)
    if (p->n_twist > 0) {
        // twists, phase table, real D' / Lp' / unit rows / zero coefficients, E_L and ln|psi|, per-twist results
        const size_t K = p->n_twist, M = bloch_images(p);
        b += 8 * 3 * K + 16 * 3 * K * (2 * M + 1) + 8 * (W * N * 4 * n + 2 * W * n * n + B * n) + 8 * 2 * W +
             8 * K * (4 + 3 * N + 9 * N * N);
    }
    b += (size_t)kPoolAllocs * kPoolAlign;           // alignment slack of a carved handle
    if (t == 4) {                                    // tensor-core operands (mixed form)
        b += tc_coeff_bytes((int)B, (int)n);
        b += tc_adjoint_coeff_bytes((int)n, (int)G) + 4 * (2 * W * n * n + 9 * W * N) + 8 * W;
        b += 4 * (3 * N * 2 * nk + W * 2 * nk + W * 3 * N);   // reciprocal-force GEMM operands
        b += 4 * W * N;                                        // carried e-n Jastrow sums of the sweep
    }
    return b;
}

void prof_begin(qmc_system* h, int cls, EventPair& ep) {
    if (!h->profiling) return;
    if (!h->free_events.empty()) {
        ep = h->free_events.back();
        h->free_events.pop_back();
    } else {
        cudaEventCreate(&ep.a);
        cudaEventCreate(&ep.b);
    }
    ep.cls = cls;
    cudaEventRecord(ep.a, h->stream);
}
void prof_end(qmc_system* h, EventPair& ep) {
    if (!h->profiling) return;
    cudaEventRecord(ep.b, h->stream);
    h->events.push_back(ep);
    ++h->klaunch[ep.cls];
}

template <typename T>
SysView<T> view(qmc_system* h, int W) {
    SysView<T> s;
    s.N = h->N; s.n = h->n; s.G = h->G; s.B = h->B; s.W = W;
    s.np = 4;
    while (s.np < s.n) s.np *= 2;
    s.L = h->p.L; s.ell = h->p.L / kPi; s.iL = 1.0 / h->p.L;
    s.b_ee = h->p.b_ee; s.b_ep = h->p.b_ep; s.Zj = 1.0; s.kappa = h->p.ewald_kappa;
    s.zeta = h->d_zeta;
    s.zetat = (const T*)(sizeof(T) == 8 ? (const void*)h->d_zeta : (const void*)h->d_zeta32);
    s.C = (const T*)(sizeof(T) == 8 ? (const void*)h->d_C64 : (const void*)h->d_C32);
    s.R = h->d_R;
    s.RT = (const T*)(sizeof(T) == 8 ? (const void*)h->d_R : (const void*)h->d_R32);
    s.eikRt = (const V2<T>*)(sizeof(T) == 8 ? (const void*)h->d_eikR : (const void*)h->d_eikR32);
    s.kwt = (const T*)(sizeof(T) == 8 ? (const void*)h->d_kw : (const void*)h->d_kw32);
    s.ptrig = (const T*)(sizeof(T) == 8 ? (const void*)h->d_ptrig64 : (const void*)h->d_ptrig32);
    s.nk = h->nk; s.mmax = h->mmax;
    s.kvec = h->d_kvec; s.kw = h->d_kw; s.eikR = h->d_eikR; s.rho_p = h->d_rhop;
    s.vconst = h->d_vconst; s.dvpp = h->d_dvpp; s.err = h->d_err; s.vacc = h->d_vacc;
    s.fj = h->d_fj; s.zeta_j = h->p.zeta_j;
    s.fjt = (const T*)(sizeof(T) == 8 ? (const void*)h->d_fj : (const void*)h->d_fj32);
    return s;
}

void setup_tables(qmc_system* h) {
    h->nlaunch += 5;
    launch_setup(h->N, h->p.L, h->p.ewald_kappa, h->nk, h->d_kvec, h->d_R, h->d_kw, h->d_ptrig64, h->d_ptrig32,
                 h->d_eikR, h->d_rhop, h->d_vconst, h->d_dvpp, h->d_R32, h->d_eikR32, h->d_kw32, h->stream);
    if (h->d_Trec) {
        h->nlaunch += 1;
        launch_recforce_table(h->N, h->nk, h->p.L, h->d_kvec, h->d_kw, h->d_eikR, h->d_Trec, h->stream);
    }
}

// Orbital rows at `pos`: tensor-core kernel in the mixed form, SIMT otherwise.
template <typename T>
void orbitals(qmc_system* h, const SysView<T>& s, const double* pos, int nrows, T* val, T* grad, T* lap) {
    if (sizeof(T) == 4 && h->use_tc)
        launch_orbitals_tc(*(const SysView<float>*)&s, h->d_chat, pos, nrows, (float*)val, (float*)grad, (float*)lap,
                           h->stream);
    else
        launch_orbitals<T>(s, pos, nrows, val, grad, lap, h->stream);
}

// Slater matrices at the current walker positions and their FP64 inverse.
template <typename T>
void recompute(qmc_system* h, int W) {
    EventPair ep;
    prof_begin(h, KC_RECOMPUTE, ep);
    SysView<T> s = view<T>(h, W);
    h->nlaunch += 2;
    orbitals<T>(h, s, h->d_X, W * h->N, (T*)h->d_Phi, nullptr, nullptr);
    launch_invert<T>(W, h->N, h->n, (const T*)h->d_Phi, (T*)h->d_Gt, h->d_logdet, h->d_err, h->stream);
    prof_end(h, ep);
}

// Periodic recompute inside a call, which resets the drift of the rank-1
// updates: by default (QMC_RECOMPUTE_FP64) the Slater blocks at the current
// positions and their FP64 Gauss-Jordan inverses and ln|det|; with
// QMC_RECOMPUTE_NEWTON (mixed form only) one Newton-Schulz step on the carried
// inverse with the residual in compensated FP32 (FP64 Gauss-Jordan only for
// blocks too far off).
template <typename T>
void recompute_in_call(qmc_system* h, int W) {
    if constexpr (sizeof(T) == 4) {
        if (h->ns_recompute) {
            EventPair ep;
            prof_begin(h, KC_RECOMPUTE, ep);
            SysView<T> s = view<T>(h, W);
            h->nlaunch += 2;
            orbitals<T>(h, s, h->d_X, W * h->N, (T*)h->d_Phi, nullptr, nullptr);
            launch_refine(W, h->N, h->n, (const float*)h->d_Phi, (float*)h->d_Gt, h->d_logdet, h->d_err, h->stream);
            prof_end(h, ep);
            return;
        }
    }
    recompute<T>(h, W);
}

template <typename T>
void measure(qmc_system* h, int W, double* el, double* lnpsi, double* dl, double* de) {
    SysView<T> s = view<T>(h, W);
    EventPair ep;
    h->nlaunch += 2;
    prof_begin(h, KC_ORB_MEAS, ep);
    orbitals<T>(h, s, h->d_X, W * h->N, (T*)h->d_Phi, (T*)h->d_D, (T*)h->d_Lp);
    prof_end(h, ep);
    const bool split = sizeof(T) == 4 && h->use_tc && h->use_tc_adj;
    prof_begin(h, KC_MEASURE, ep);
    launch_measure<T>(s, h->d_X, (const T*)h->d_D, (const T*)h->d_Lp, (const T*)h->d_Gt, h->d_logdet, h->d_acc, el,
                      lnpsi, dl, de, split ? h->d_Kt : nullptr, split ? h->d_eg : nullptr,
                      split ? h->d_elw : nullptr, split ? h->d_rk : nullptr, h->stream);
    prof_end(h, ep);
    if (split) {
        h->nlaunch += 1;
        prof_begin(h, KC_ADJOINT, ep);
        // reciprocal-space forces of all walkers: F[W][3N] = rho[W][2nk] . T[2nk][3N]
        h->nlaunch += 1;
        launch_recforce_gemm(W, 3 * h->N, 2 * h->nk, h->d_rk, h->d_Trec, h->d_frec, h->stream);
        launch_adjoint_tc(*(const SysView<float>*)&s, h->d_ahat, (const float*)h->d_Gt, h->d_Kt, h->d_eg, h->d_elw,
                          h->d_frec, h->d_acc, dl, de, h->stream);
        prof_end(h, ep);
    }
}

// Sampling part of one energy/force call (recompute, warm-up and measured
// sweeps with their samples in the per-walker accumulators); returns the
// number of electron moves.
template <typename T>
double run_sampling(qmc_system* h) {
    const int W = h->W, N = h->N;
    SysView<T> s = view<T>(h, W);
    const Key key = make_key(h->p.seed);
    const uint32_t md = h->md_step;
    cudaMemsetAsync(h->d_acc, 0, sizeof(double) * (size_t)W * (3 + 9 * N), h->stream);
    cudaMemsetAsync(h->d_vacc, 0, sizeof(double) * (size_t)W, h->stream);
    cudaMemsetAsync(h->d_nacc, 0, sizeof(unsigned long long) * W, h->stream);
    recompute<T>(h, W);
    const int nw = h->first_call ? h->p.n_warmup : h->p.n_warmup_cont;
    const int total = nw + h->p.n_sweeps;
    for (int sw = 0; sw < total; ++sw) {
        EventPair ep;
        h->nlaunch += 3;
        prof_begin(h, KC_PROPOSE, ep);
        launch_propose<T>(W, N, h->p.L, h->d_X, h->d_Xp, (T*)h->d_ptp, (T*)h->d_uacc, key, md, (uint32_t)sw,
                          h->p.sigma, h->w0, h->stream);
        prof_end(h, ep);
        prof_begin(h, KC_ORB_PROP, ep);
        orbitals<T>(h, s, h->d_Xp, W * N, (T*)h->d_Phi, nullptr, nullptr);
        prof_end(h, ep);
        prof_begin(h, KC_SWEEP, ep);
        launch_sweep<T>(s, h->d_X, h->d_Xp, (const T*)h->d_ptp, (const T*)h->d_uacc, (const T*)h->d_Phi,
                        (T*)h->d_Gt, h->d_nacc, h->d_vep, sw == 0, h->stream);
        prof_end(h, ep);
        if ((sw + 1) % h->p.recompute_every == 0) recompute_in_call<T>(h, W);
        if (sw >= nw && ((sw - nw + 1) % h->p.measure_every) == 0) measure<T>(h, W, nullptr, nullptr, nullptr, nullptr);
    }
    h->md_step++;
    h->first_call = false;
    return (double)W * total * N;
}

// ---- twisted boundary conditions (FP64 form, complex orbitals) ----

// Complex Slater blocks at the current walker positions and their inverses.
void recompute_twist(qmc_system* h, int W) {
    EventPair ep;
    prof_begin(h, KC_RECOMPUTE, ep);
    SysView<double> s = view<double>(h, W);
    h->nlaunch += 2;
    launch_twist_orbitals(s, h->tv, h->d_X, W * h->N, (double2*)h->d_Phi, nullptr, nullptr, h->stream);
    launch_twist_invert(W, h->N, h->n, (const double2*)h->d_Phi, (double2*)h->d_Gt, h->d_logdet, h->d_err, h->stream);
    prof_end(h, ep);
}

// Local energy and force sample of every walker: complex orbital rows; Re g and
// Re l into column 0 of D' and Lp'; the FP64 measure kernel on D', Lp', unit
// inverse rows and zero coefficients (so it computes E_L = Re(H psi / psi), the
// Jastrow and Ewald force terms with vv = Re g + grad U, and adds nothing from
// its orbital force phase); then the complex orbital (Pulay) force terms.
void measure_twist(qmc_system* h, int W, double* el, double* lnpsi, double* dl, double* de) {
    SysView<double> s = view<double>(h, W);
    const int N = h->N, n = h->n;
    EventPair ep;
    h->nlaunch += 4;
    prof_begin(h, KC_ORB_MEAS, ep);
    launch_twist_orbitals(s, h->tv, h->d_X, W * N, (double2*)h->d_Phi, (double2*)h->d_D, (double2*)h->d_Lp,
                          h->stream);
    launch_twist_gl(W * N, N, n, (const double2*)h->d_D, (const double2*)h->d_Lp, (const double2*)h->d_Gt, h->d_Dr,
                    h->d_Lpr, h->stream);
    prof_end(h, ep);
    SysView<double> s0 = s;
    s0.C = h->d_Czero;
    double* elw = el ? el : h->d_elt;
    prof_begin(h, KC_MEASURE, ep);
    launch_measure<double>(s0, h->d_X, h->d_Dr, h->d_Lpr, h->d_Gtr, h->d_logdet, h->d_acc, elw,
                           lnpsi ? lnpsi : h->d_lpt, dl, de, nullptr, nullptr, nullptr, nullptr, h->stream);
    prof_end(h, ep);
    prof_begin(h, KC_ADJOINT, ep);
    launch_twist_pulay(s, h->tv, h->d_X, (const double2*)h->d_D, (const double2*)h->d_Lp, (const double2*)h->d_Gt,
                       elw, h->d_acc, dl, de, h->stream);
    prof_end(h, ep);
}

double run_sampling_twist(qmc_system* h) {
    const int W = h->W, N = h->N;
    SysView<double> s = view<double>(h, W);
    const Key key = make_key(h->p.seed);
    const uint32_t md = h->md_step;
    cudaMemsetAsync(h->d_acc, 0, sizeof(double) * (size_t)W * (3 + 9 * N), h->stream);
    cudaMemsetAsync(h->d_vacc, 0, sizeof(double) * (size_t)W, h->stream);
    cudaMemsetAsync(h->d_nacc, 0, sizeof(unsigned long long) * W, h->stream);
    recompute_twist(h, W);
    const int nw = h->first_call ? h->p.n_warmup : h->p.n_warmup_cont;
    const int total = nw + h->p.n_sweeps;
    for (int sw = 0; sw < total; ++sw) {
        EventPair ep;
        h->nlaunch += 3;
        prof_begin(h, KC_PROPOSE, ep);
        launch_propose<double>(W, N, h->p.L, h->d_X, h->d_Xp, (double*)h->d_ptp, (double*)h->d_uacc, key, md,
                               (uint32_t)sw, h->p.sigma, h->w0, h->stream);
        prof_end(h, ep);
        prof_begin(h, KC_ORB_PROP, ep);
        launch_twist_orbitals(s, h->tv, h->d_Xp, W * N, (double2*)h->d_Phi, nullptr, nullptr, h->stream);
        prof_end(h, ep);
        prof_begin(h, KC_SWEEP, ep);
        launch_twist_sweep(s, h->tv, h->d_X, h->d_Xp, (const double*)h->d_ptp, (const double*)h->d_uacc,
                           (const double2*)h->d_Phi, (double2*)h->d_Gt, h->d_nacc, h->stream);
        prof_end(h, ep);
        if ((sw + 1) % h->p.recompute_every == 0) recompute_twist(h, W);
        if (sw >= nw && ((sw - nw + 1) % h->p.measure_every) == 0) measure_twist(h, W, nullptr, nullptr, nullptr, nullptr);
    }
    h->md_step++;
    h->first_call = false;
    return (double)W * total * N;
}

// Each twist's walker block reduced on its own, then the twist average.
void reduce_twist(qmc_system* h, double moves) {
    const int K = h->K, Wk = h->W / K, N = h->N;
    const size_t stride = 3 + 9 * (size_t)N, olen = 4 + 3 * (size_t)N + 9 * (size_t)N * N;
    for (int t = 0; t < K; ++t)
        launch_reduce(Wk, N, moves / K, h->d_acc + (size_t)t * Wk * stride, h->d_nacc + (size_t)t * Wk, h->d_colsum,
                      h->d_dev, h->d_tout + (size_t)t * olen, h->d_err, h->stream);
    launch_twist_average(K, N, h->d_tout, h->d_out, h->stream);
    h->nlaunch += 5 * K + 1;
}

template <typename T>
void run_call(qmc_system* h) {
    if (h->K) {
        const double moves = run_sampling_twist(h);
        EventPair ep;
        prof_begin(h, KC_REDUCE, ep);
        reduce_twist(h, moves);
        prof_end(h, ep);
        h->last_Nc = (double)h->W * (h->p.n_sweeps / h->p.measure_every);
        return;
    }
    const double moves = run_sampling<T>(h);
    EventPair ep;
    prof_begin(h, KC_REDUCE, ep);
    h->nlaunch += 5;
    launch_reduce(h->W, h->N, moves, h->d_acc, h->d_nacc, h->d_colsum, h->d_dev, h->d_out, h->d_err, h->stream);
    prof_end(h, ep);
    h->last_Nc = (double)h->W * (h->p.n_sweeps / h->p.measure_every);
}

int read_err(qmc_system* h) {
    int e = 0;
    if (cudaMemcpyAsync(&e, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, h->stream) != cudaSuccess) return QMC_ERR_CUDA;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return QMC_ERR_CUDA;
    cudaMemsetAsync(h->d_err, 0, sizeof(int), h->stream);
    if (e & kErrNotPD) return QMC_ERR_NOT_PD;
    if (e & kErrSingular) return QMC_ERR_SINGULAR;
    if (e & kErrNonfinite) return QMC_ERR_NONFINITE;
    if (e & kErrTimeout) return QMC_ERR_TIMEOUT;
    return QMC_OK;
}

int check_launch() { return cudaGetLastError() == cudaSuccess ? QMC_OK : QMC_ERR_CUDA; }

}  // namespace

extern "C" {

size_t qmc_footprint_bytes(const qmc_params* p) { return validate(p) == QMC_OK ? footprint(p) : 0; }

int qmc_init(const qmc_params* p, const double* R, qmc_system** out) {
    return qmc::init_handle(p, R, nullptr, 0, nullptr, true, out);
}

}  // extern "C"

namespace qmc {

int init_handle(const qmc_params* p, const double* R, void* block, size_t block_bytes, cudaStream_t stream,
                bool wait, qmc_system** out) {
    if (!out || !R) return QMC_ERR_INVALID;
    *out = nullptr;
    int rc = validate(p);
    if (rc != QMC_OK) return rc;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return QMC_ERR_CUDA; }
    qmc_system* h = new (std::nothrow) qmc_system();
    if (!h) return QMC_ERR_OOM;
    h->pool = (unsigned char*)block;
    h->pool_bytes = block ? block_bytes : 0;
    h->p = *p;
    h->N = p->n_protons; h->n = h->N / 2; h->G = p->n_gauss; h->B = h->N * h->G; h->W = p->n_walkers;
    h->mmax = p->ewald_mmax;
    h->mixed = p->precision == QMC_MIXED;
    h->zeta_h.assign(p->zeta, p->zeta + h->G);
    h->coeff_h.assign(p->coeff, p->coeff + (size_t)h->B * h->n);
    h->p.zeta = h->zeta_h.data();
    h->p.coeff = h->coeff_h.data();
    if (p->fj) {
        h->fj_h.assign(p->fj, p->fj + (size_t)h->N * h->N);
        h->p.fj = h->fj_h.data();
    }
    if (p->n_twist > 0) {
        h->K = p->n_twist;
        h->twist_h.assign(p->twist, p->twist + 3 * (size_t)h->K);
        h->p.twist = h->twist_h.data();
    } else {
        h->p.n_twist = 0;
        h->p.twist = nullptr;
    }
    std::vector<int4> kv;
    enumerate_kvec(h->mmax, kv);
    h->nk = (int)kv.size();
    if (stream) {
        h->stream = stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete h;
            return QMC_ERR_CUDA;
        }
        h->stream = h->own_stream;
    }
    const int N = h->N, n = h->n, W = h->W, B = h->B, nk = h->nk;
    const size_t t = h->mixed ? sizeof(float) : sizeof(double);
    const size_t tc = h->K ? sizeof(double2) : t;   // complex orbitals of the twisted form
    h->d_R = dalloc<double>(h, 3 * N, &rc);
    h->d_zeta = dalloc<double>(h, h->G, &rc);
    h->d_C64 = dalloc<double>(h, (size_t)B * n, &rc);
    h->d_C32 = dalloc<float>(h, (size_t)B * n, &rc);
    h->d_ptrig64 = dalloc<double>(h, 6 * N, &rc);
    h->d_ptrig32 = dalloc<float>(h, 6 * N, &rc);
    h->d_kvec = dalloc<int4>(h, nk, &rc);
    h->d_kw = dalloc<double>(h, nk, &rc);
    h->d_eikR = dalloc<double2>(h, (size_t)N * nk, &rc);
    h->d_rhop = dalloc<double2>(h, nk, &rc);
    h->d_vconst = dalloc<double>(h, 1, &rc);
    h->d_dvpp = dalloc<double>(h, 3 * N, &rc);
    h->d_R32 = dalloc<float>(h, 3 * N, &rc);
    h->d_zeta32 = dalloc<float>(h, h->G, &rc);
    h->d_ptp = dalloc<unsigned char>(h, t * (size_t)W * N * 6, &rc);
    h->d_kw32 = dalloc<float>(h, nk, &rc);
    h->d_eikR32 = dalloc<float2>(h, (size_t)N * nk, &rc);
    h->d_X = dalloc<double>(h, (size_t)W * 3 * N, &rc);
    h->d_Xp = dalloc<double>(h, (size_t)W * 3 * N, &rc);
    h->d_uacc = dalloc<unsigned char>(h, t * W * N, &rc);
    h->d_Phi = dalloc<unsigned char>(h, tc * W * N * n, &rc);
    h->d_Gt = dalloc<unsigned char>(h, tc * W * 2 * n * n, &rc);
    h->d_D = dalloc<unsigned char>(h, tc * W * N * 3 * n, &rc);
    h->d_Lp = dalloc<unsigned char>(h, tc * W * N * n, &rc);
    h->d_logdet = dalloc<double>(h, 2 * (size_t)W, &rc);
    h->d_acc = dalloc<double>(h, (size_t)W * (3 + 9 * N), &rc);
    h->d_vacc = dalloc<double>(h, W, &rc);
    if (h->mixed) h->d_vep = dalloc<float>(h, (size_t)W * N, &rc);
    h->d_pout = dalloc<double>(h, 5, &rc);
    h->d_nacc = dalloc<unsigned long long>(h, W, &rc);
    h->d_colsum = dalloc<double>(h, 4 + 9 * N, &rc);
    h->d_dev = dalloc<double>(h, (size_t)W * (3 * N + 1), &rc);
    h->d_out = dalloc<double>(h, 4 + 3 * N + 9 * (size_t)N * N, &rc);
    h->d_eval = dalloc<double>(h, (size_t)W * (2 + 6 * N), &rc);
    h->d_Rl = dalloc<double>(h, 3 * N, &rc);
    h->d_Rprev = dalloc<double>(h, 3 * N, &rc);
    h->d_f = dalloc<double>(h, 3 * N, &rc);
    h->d_S = dalloc<double>(h, 9 * (size_t)N * N, &rc);
    h->d_Sprev = dalloc<double>(h, 9 * (size_t)N * N, &rc);
    h->d_Lwork = dalloc<double>(h, 9 * (size_t)N * N, &rc);
    h->d_fsR = dalloc<double>(h, 3 * N, &rc);
    h->d_fsf = dalloc<double>(h, 3 * N, &rc);
    h->d_fsS = dalloc<double>(h, 9 * (size_t)N * N, &rc);
    h->d_fsL = dalloc<double>(h, 9 * (size_t)N * N, &rc);
    h->d_err = dalloc<int>(h, 1, &rc);
    if (!h->fj_h.empty()) {
        h->d_fj = dalloc<double>(h, (size_t)N * N, &rc);
        if (h->mixed) h->d_fj32 = dalloc<float>(h, (size_t)N * N, &rc);
    }
    std::vector<double2> tph;
    if (h->K) {
        const int K = h->K, M = bloch_images(p);
        h->d_theta = dalloc<double>(h, 3 * (size_t)K, &rc);
        h->d_tph = dalloc<double2>(h, (size_t)K * 3 * (2 * M + 1), &rc);
        h->d_Dr = dalloc<double>(h, (size_t)W * N * 3 * n, &rc);
        h->d_Lpr = dalloc<double>(h, (size_t)W * N * n, &rc);
        h->d_Gtr = dalloc<double>(h, (size_t)W * 2 * n * n, &rc);
        h->d_Czero = dalloc<double>(h, (size_t)B * n, &rc);
        h->d_elt = dalloc<double>(h, W, &rc);
        h->d_lpt = dalloc<double>(h, W, &rc);
        h->d_tout = dalloc<double>(h, (size_t)K * (4 + 3 * N + 9 * (size_t)N * N), &rc);
        // exp(i theta_mu m), m = -M..M, per twist and axis
        for (int k = 0; k < K; ++k)
            for (int mu = 0; mu < 3; ++mu)
                for (int m = -M; m <= M; ++m) {
                    const double a = h->twist_h[3 * k + mu] * m;
                    tph.push_back(make_double2(std::cos(a), std::sin(a)));
                }
        h->tv.K = K; h->tv.Wk = W / K; h->tv.M = M;
        h->tv.theta = h->d_theta; h->tv.ph = h->d_tph;
    }
    // The tcgen05 kernels serve N = 128 with 4 Gaussians per nucleus (n = 64
    // orbitals per spin), the configuration they are built, tuned and tested
    // for; other systems use the SIMT FP32 kernels.  With 32 or 64 protons and
    // 2 Gaussians per nucleus the tcgen05 path rarely stalled the device for
    // tens of seconds and returned non-finite results (several thousand
    // walkers, most often with other handles' kernels running); the cause is
    // not found, so that path is not offered.
    if (h->mixed && tc_orbitals_supported(n, B) && n == 64 && h->G == 4) {
        h->d_chat = dalloc<unsigned char>(h, tc_coeff_bytes(B, n), &rc);
        h->use_tc = true;
        if (tc_adjoint_supported(N, n, h->G)) {
            h->d_ahat = dalloc<unsigned char>(h, tc_adjoint_coeff_bytes(n, h->G), &rc);
            h->d_Kt = dalloc<float>(h, (size_t)W * 2 * n * n, &rc);
            h->d_eg = dalloc<float>(h, (size_t)W * N * 9, &rc);
            h->d_elw = dalloc<double>(h, W, &rc);
            h->d_Trec = dalloc<float>(h, (size_t)3 * N * 2 * nk, &rc);
            h->d_rk = dalloc<float>(h, (size_t)W * 2 * nk, &rc);
            h->d_frec = dalloc<float>(h, (size_t)W * 3 * N, &rc);
            h->use_tc_adj = true;
        }
    }
    if (rc != QMC_OK) { qmc_destroy(h); return rc; }
    std::vector<float> c32(h->coeff_h.begin(), h->coeff_h.end());
    std::vector<float> z32(h->zeta_h.begin(), h->zeta_h.end());
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(h->d_R, R, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_zeta, h->zeta_h.data(), sizeof(double) * h->G, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_C64, h->coeff_h.data(), sizeof(double) * B * n, cudaMemcpyHostToDevice, st);
    if (h->d_fj) cudaMemcpyAsync(h->d_fj, h->fj_h.data(), sizeof(double) * N * N, cudaMemcpyHostToDevice, st);
    if (h->K) {
        cudaMemcpyAsync(h->d_theta, h->twist_h.data(), sizeof(double) * 3 * h->K, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(h->d_tph, tph.data(), sizeof(double2) * tph.size(), cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(h->d_Dr, 0, sizeof(double) * (size_t)W * N * 3 * n, st);
        cudaMemsetAsync(h->d_Lpr, 0, sizeof(double) * (size_t)W * N * n, st);
        cudaMemsetAsync(h->d_Czero, 0, sizeof(double) * (size_t)B * n, st);
        launch_twist_unit_rows(W, n, h->d_Gtr, st);
    }
    std::vector<float> fj32(h->fj_h.begin(), h->fj_h.end());
    if (h->d_fj32) cudaMemcpyAsync(h->d_fj32, fj32.data(), sizeof(float) * N * N, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_C32, c32.data(), sizeof(float) * B * n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_zeta32, z32.data(), sizeof(float) * h->G, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_kvec, kv.data(), sizeof(int4) * nk, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(h->d_err, 0, sizeof(int), st);
    cudaMemsetAsync(h->d_nacc, 0, sizeof(unsigned long long) * W, st);
    if (h->d_chat) prepare_tc_coeff(h->d_C32, B, n, h->d_chat, st);
    if (h->d_ahat) prepare_tc_adjoint_coeff(h->d_C32, N, h->G, n, h->d_ahat, st);
    setup_tables(h);
    launch_init_walkers(W, N, p->L, h->d_R, h->d_X, make_key(p->seed), 0u, st);
    h->emp_lambda = thomas_fermi_length(N, p->L);
    rc = check_launch();
    // host arrays above are pageable, so their copies have been staged already
    if (rc == QMC_OK && wait) rc = cuda_rc(cudaStreamSynchronize(st));
    if (rc != QMC_OK) { qmc_destroy(h); return rc; }
    *out = h;
    return QMC_OK;
}

}  // namespace qmc

extern "C" {

void qmc_destroy(qmc_system* h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    for (void* a : h->allocs) cudaFree(a);      // none for a handle carved from a block
    for (auto& e : h->events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    for (auto& e : h->free_events) { cudaEventDestroy(e.a); cudaEventDestroy(e.b); }
    if (h->own_stream) cudaStreamDestroy(h->own_stream);
    delete h;
}

int qmc_set_stream(qmc_system* h, void* stream) {
    if (!h) return QMC_ERR_INVALID;
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return QMC_OK;
}

int qmc_sync(qmc_system* h) {
    if (!h) return QMC_ERR_INVALID;
    return read_err(h);
}

int qmc_set_md_step(qmc_system* h, uint32_t md_step) {
    if (!h) return QMC_ERR_INVALID;
    h->md_step = md_step;
    return QMC_OK;
}

int qmc_energy_forces_device(qmc_system* h, const double* R_dev, double* out_dev) {
    if (!h || !R_dev || !out_dev) return QMC_ERR_INVALID;
    const int N = h->N;
    cudaMemcpyAsync(h->d_R, R_dev, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, h->stream);
    setup_tables(h);
    if (h->mixed) run_call<float>(h);
    else run_call<double>(h);
    cudaMemcpyAsync(out_dev, h->d_out, sizeof(double) * (4 + 3 * N + 9 * (size_t)N * N), cudaMemcpyDeviceToDevice,
                    h->stream);
    return check_launch();
}

int qmc_energy_forces(qmc_system* h, const double* R, qmc_result* out) {
    if (!h || !R || !out || !out->f || !out->cov) return QMC_ERR_INVALID;
    const int N = h->N;
    cudaMemcpyAsync(h->d_R, R, sizeof(double) * 3 * N, cudaMemcpyHostToDevice, h->stream);
    setup_tables(h);
    if (h->mixed) run_call<float>(h);
    else run_call<double>(h);
    int rc = check_launch();
    if (rc != QMC_OK) return rc;
    std::vector<double> o(4 + 3 * N + 9 * (size_t)N * N);
    cudaMemcpyAsync(o.data(), h->d_out, sizeof(double) * o.size(), cudaMemcpyDeviceToHost, h->stream);
    rc = read_err(h);
    if (rc != QMC_OK) return rc;
    out->E = o[0]; out->E_err = o[1]; out->n_samples = o[2]; out->accept = o[3];
    std::memcpy(out->f, o.data() + 4, sizeof(double) * 3 * N);
    std::memcpy(out->cov, o.data() + 4 + 3 * N, sizeof(double) * 9 * (size_t)N * N);
    return QMC_OK;
}

int qmc_pressure_device(qmc_system* h, double T_kelvin, double* out_dev) {
    if (!h || !out_dev || T_kelvin < 0) return QMC_ERR_INVALID;
    const double L = h->p.L;
    EventPair ep;
    prof_begin(h, KC_REDUCE, ep);
    h->nlaunch += 1;
    launch_pressure(h->W, h->N, h->d_acc, h->d_vacc, L * L * L, T_kelvin * kBoltzmannHaPerK, out_dev, h->stream);
    prof_end(h, ep);
    return check_launch();
}

int qmc_pressure(qmc_system* h, double T_kelvin, double* out) {
    if (!h || !out) return QMC_ERR_INVALID;
    int rc = qmc_pressure_device(h, T_kelvin, h->d_pout);
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(out, h->d_pout, sizeof(double) * 5, cudaMemcpyDeviceToHost, h->stream);
    return read_err(h);
}

int qmc_shard_sample_device(qmc_system* h, const double* R_dev, double* sums_dev) {
    if (!h || !R_dev || !sums_dev || h->K) return QMC_ERR_INVALID;
    const int N = h->N;
    cudaMemcpyAsync(h->d_R, R_dev, sizeof(double) * 3 * N, cudaMemcpyDeviceToDevice, h->stream);
    setup_tables(h);
    const double moves = h->mixed ? run_sampling<float>(h) : run_sampling<double>(h);
    EventPair ep;
    prof_begin(h, KC_REDUCE, ep);
    h->nlaunch += 2;
    launch_shard_sums(h->W, N, moves, h->d_acc, h->d_nacc, sums_dev, h->stream);
    prof_end(h, ep);
    return check_launch();
}

int qmc_shard_reduce_device(qmc_system* h, const double* sums_dev, double* out_dev, double* gram_dev) {
    if (!h || !sums_dev || !out_dev || !gram_dev || h->K) return QMC_ERR_INVALID;
    EventPair ep;
    prof_begin(h, KC_REDUCE, ep);
    h->nlaunch += 4;
    launch_shard_reduce(h->W, h->N, h->d_acc, sums_dev, h->d_dev, out_dev, gram_dev, h->d_err, h->stream);
    prof_end(h, ep);
    return check_launch();
}

int qmc_shard_finish_device(qmc_system* h, const double* sums_dev, const double* gram_dev, double* out_dev,
                            long long walkers_total) {
    if (!h || !sums_dev || !gram_dev || !out_dev || walkers_total < 2 || h->K) return QMC_ERR_INVALID;
    EventPair ep;
    prof_begin(h, KC_REDUCE, ep);
    h->nlaunch += 1;
    launch_shard_finish(h->N, sums_dev, gram_dev, out_dev, h->stream);
    prof_end(h, ep);
    h->last_Nc = (double)walkers_total * (h->p.n_sweeps / h->p.measure_every);
    return check_launch();
}

int langevin_step_device(qmc_system* h, double* R_dev, const double* f_dev, const double* S_dev, double T_kelvin,
                         double delta, int s_mode, double alpha) {
    if (!h || !R_dev || !f_dev || (!S_dev && s_mode == QMC_S_COV)) return QMC_ERR_INVALID;
    if (s_mode != QMC_S_IDENTITY && s_mode != QMC_S_COV && s_mode != QMC_S_EMPIRICAL) return QMC_ERR_INVALID;
    if (s_mode == QMC_S_EMPIRICAL && alpha < 0) return QMC_ERR_INVALID;
    if (!(delta > 0) || T_kelvin < 0) return QMC_ERR_INVALID;
    double T_ha = T_kelvin * kBoltzmannHaPerK;
    if (h->lv_noise_correction) {       // SI "Noise correction": 2 T D = 2 T_target D - D^2
        T_ha -= 0.5 * delta;
        if (!(T_ha > 0)) return QMC_ERR_INVALID;
    }
    const int n3 = 3 * h->N;
    cudaStream_t st = h->stream;
    const int identity = s_mode == QMC_S_IDENTITY;
    if (s_mode == QMC_S_COV)
        cudaMemcpyAsync(h->d_S, S_dev, sizeof(double) * n3 * n3, cudaMemcpyDeviceToDevice, st);
    if (s_mode == QMC_S_EMPIRICAL) {   // S = H + mu I at the current positions
        h->nlaunch += 1;
        launch_empirical_s(h->N, h->p.L, R_dev, h->emp_lambda, h->emp_mu, h->d_S, st);
    }
    if (h->langevin_first) {
        cudaMemcpyAsync(h->d_Rprev, R_dev, sizeof(double) * n3, cudaMemcpyDeviceToDevice, st);
        if (!identity) cudaMemcpyAsync(h->d_Sprev, h->d_S, sizeof(double) * n3 * n3, cudaMemcpyDeviceToDevice, st);
        else cudaMemsetAsync(h->d_Sprev, 0, sizeof(double) * n3 * n3, st);
        h->langevin_first = false;
    }
    double a = 0.0;
    if (s_mode == QMC_S_COV) a = alpha > 0 ? alpha : 0.122 * h->last_Nc;
    if (s_mode == QMC_S_EMPIRICAL) a = alpha;
    EventPair ep;
    prof_begin(h, KC_LANGEVIN, ep);
    h->nlaunch += 1;
    launch_langevin(n3, R_dev, h->d_Rprev, f_dev, h->d_S, h->d_Sprev, h->d_Lwork, T_ha, delta, a,
                    make_key(h->p.seed), h->langevin_step_no, h->p.L, identity, h->lv_scheme, h->d_err, st);
    prof_end(h, ep);
    h->langevin_step_no++;
    return check_launch();
}

int qmc_twist_partial_device(qmc_system* h, const double* out_dev, double* part_dev) {
    if (!h || !out_dev || !part_dev || !h->K) return QMC_ERR_INVALID;
    h->nlaunch += 1;
    launch_twist_partial(h->K, h->N, out_dev, part_dev, h->stream);
    return check_launch();
}

int qmc_twist_combine_device(qmc_system* h, const double* part_dev, int K_total, double* out_dev) {
    if (!h || !part_dev || !out_dev || !h->K || K_total < h->K) return QMC_ERR_INVALID;
    h->nlaunch += 1;
    launch_twist_combine(K_total, h->N, part_dev, out_dev, h->stream);
    return check_launch();
}

int qmc_set_empirical_s(qmc_system* h, double lambda, double mu) {
    if (!h || !std::isfinite(lambda) || !std::isfinite(mu) || mu < 0) return QMC_ERR_INVALID;
    h->emp_lambda = lambda > 0 ? lambda : thomas_fermi_length(h->N, h->p.L);
    h->emp_mu = mu;
    return QMC_OK;
}

int qmc_empirical_s_device(qmc_system* h, const double* R_dev, double* S_dev) {
    if (!h || !R_dev || !S_dev) return QMC_ERR_INVALID;
    h->nlaunch += 1;
    launch_empirical_s(h->N, h->p.L, R_dev, h->emp_lambda, h->emp_mu, S_dev, h->stream);
    return check_launch();
}

int qmc_empirical_s(qmc_system* h, const double* R, double* S) {
    if (!h || !R || !S) return QMC_ERR_INVALID;
    const int n3 = 3 * h->N;
    cudaMemcpyAsync(h->d_Rl, R, sizeof(double) * n3, cudaMemcpyHostToDevice, h->stream);
    int rc = qmc_empirical_s_device(h, h->d_Rl, h->d_Lwork);
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(S, h->d_Lwork, sizeof(double) * n3 * n3, cudaMemcpyDeviceToHost, h->stream);
    return read_err(h);
}

int langevin_step(qmc_system* h, double* R, const double* f, const double* S, double T_kelvin, double delta,
                  int s_mode, double alpha) {
    if (!h || !R || !f || (!S && s_mode == QMC_S_COV)) return QMC_ERR_INVALID;
    const int n3 = 3 * h->N;
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(h->d_Rl, R, sizeof(double) * n3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_f, f, sizeof(double) * n3, cudaMemcpyHostToDevice, st);
    if (s_mode == QMC_S_COV) cudaMemcpyAsync(h->d_S, S, sizeof(double) * n3 * n3, cudaMemcpyHostToDevice, st);
    int rc = langevin_step_device(h, h->d_Rl, h->d_f, s_mode == QMC_S_COV ? h->d_S : nullptr, T_kelvin, delta, s_mode,
                                  alpha);
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(R, h->d_Rl, sizeof(double) * n3, cudaMemcpyDeviceToHost, st);
    return read_err(h);
}

int langevin_first_predict(qmc_system* h, double* R, const double* f, const double* S, double T_kelvin, double delta) {
    if (!h || !R || !f || !S || !(delta > 0) || T_kelvin < 0) return QMC_ERR_INVALID;
    double T_ha = T_kelvin * kBoltzmannHaPerK;
    if (h->lv_noise_correction) {
        T_ha -= 0.5 * delta;
        if (!(T_ha > 0)) return QMC_ERR_INVALID;
    }
    const int n3 = 3 * h->N;
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(h->d_fsR, R, sizeof(double) * n3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_fsf, f, sizeof(double) * n3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_fsS, S, sizeof(double) * n3 * n3, cudaMemcpyHostToDevice, st);
    EventPair ep;
    prof_begin(h, KC_LANGEVIN, ep);
    h->nlaunch += 1;
    launch_first_predict(n3, h->d_fsR, h->d_fsS, h->d_fsL, T_ha, delta, make_key(h->p.seed), h->langevin_step_no,
                         h->d_Rl, h->d_err, st);
    prof_end(h, ep);
    int rc = check_launch();
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(R, h->d_Rl, sizeof(double) * n3, cudaMemcpyDeviceToHost, st);
    rc = read_err(h);
    h->fs_pending = rc == QMC_OK;
    h->fs_delta = delta;
    return rc;
}

int langevin_first_correct(qmc_system* h, double* y, const double* S_y) {
    if (!h || !y || !S_y || !h->fs_pending) return QMC_ERR_INVALID;
    const int n3 = 3 * h->N;
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(h->d_Rl, y, sizeof(double) * n3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_S, S_y, sizeof(double) * n3 * n3, cudaMemcpyHostToDevice, st);
    EventPair ep;
    prof_begin(h, KC_LANGEVIN, ep);
    h->nlaunch += 1;
    launch_first_correct(n3, h->d_Rl, h->d_fsR, h->d_fsf, h->d_fsS, h->d_S, h->d_fsL, h->fs_delta, h->p.L, st);
    prof_end(h, ep);
    int rc = check_launch();
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(y, h->d_Rl, sizeof(double) * n3, cudaMemcpyDeviceToHost, st);
    h->fs_pending = false;
    h->langevin_step_no++;
    return read_err(h);
}

int qmc_eval_config(qmc_system* h, int n_conf, const double* X, const double* R, double* logpsi, double* EL,
                    double* dlogpsi_dR, double* dEL_dR) {
    if (!h || !X || !R || !logpsi || !EL || !dlogpsi_dR || !dEL_dR) return QMC_ERR_INVALID;
    if (n_conf < 1 || n_conf > h->W) return QMC_ERR_INVALID;
    const int N = h->N, N3 = 3 * N;
    cudaStream_t st = h->stream;
    cudaMemcpyAsync(h->d_R, R, sizeof(double) * N3, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(h->d_X, X, sizeof(double) * (size_t)n_conf * N3, cudaMemcpyHostToDevice, st);
    setup_tables(h);
    cudaMemsetAsync(h->d_acc, 0, sizeof(double) * (size_t)n_conf * (3 + 9 * N), st);
    cudaMemsetAsync(h->d_vacc, 0, sizeof(double) * (size_t)n_conf, st);
    double* el = h->d_eval;
    double* lp = el + n_conf;
    double* dl = lp + n_conf;
    double* de = dl + (size_t)n_conf * N3;
    if (h->K) { recompute_twist(h, n_conf); measure_twist(h, n_conf, el, lp, dl, de); }
    else if (h->mixed) { recompute<float>(h, n_conf); measure<float>(h, n_conf, el, lp, dl, de); }
    else { recompute<double>(h, n_conf); measure<double>(h, n_conf, el, lp, dl, de); }
    int rc = check_launch();
    if (rc != QMC_OK) return rc;
    cudaMemcpyAsync(EL, el, sizeof(double) * n_conf, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(logpsi, lp, sizeof(double) * n_conf, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(dlogpsi_dR, dl, sizeof(double) * n_conf * N3, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(dEL_dR, de, sizeof(double) * n_conf * N3, cudaMemcpyDeviceToHost, st);
    return read_err(h);
}

int qmc_get_walkers(qmc_system* h, double* X) {
    if (!h || !X) return QMC_ERR_INVALID;
    cudaMemcpyAsync(X, h->d_X, sizeof(double) * (size_t)h->W * 3 * h->N, cudaMemcpyDeviceToHost, h->stream);
    return read_err(h);
}

int qmc_set_walkers(qmc_system* h, const double* X) {
    if (!h || !X) return QMC_ERR_INVALID;
    cudaMemcpyAsync(h->d_X, X, sizeof(double) * (size_t)h->W * 3 * h->N, cudaMemcpyHostToDevice, h->stream);
    return read_err(h);
}

int qmc_get_accumulators(qmc_system* h, double* acc) {
    if (!h || !acc) return QMC_ERR_INVALID;
    cudaMemcpyAsync(acc, h->d_acc, sizeof(double) * (size_t)h->W * (3 + 9 * h->N), cudaMemcpyDeviceToHost, h->stream);
    return read_err(h);
}

int qmc_set_option(qmc_system* h, int option, int value) {
    if (!h) return QMC_ERR_INVALID;
    if (option == QMC_OPT_TENSOR_CORES) {
        if (value && !h->d_chat) return QMC_ERR_INVALID;
        h->use_tc = value != 0;
        return QMC_OK;
    }
    if (option == QMC_OPT_TC_ADJOINT) {
        if (value && !h->d_ahat) return QMC_ERR_INVALID;
        h->use_tc_adj = value != 0;
        return QMC_OK;
    }
    if (option == QMC_OPT_INTEGRATOR) {
        if (value != QMC_LV_ADOPTED && value != QMC_LV_FAST && value != QMC_LV_NOROGNA) return QMC_ERR_INVALID;
        h->lv_scheme = value == QMC_LV_FAST ? kLvFast : value == QMC_LV_NOROGNA ? kLvNorogna : kLvAdopted;
        return QMC_OK;
    }
    if (option == QMC_OPT_NOISE_CORRECTION) {
        h->lv_noise_correction = value != 0;
        return QMC_OK;
    }
    if (option == QMC_OPT_WALKER_OFFSET) {
        if (value < 0) return QMC_ERR_INVALID;
        h->w0 = (uint32_t)value;
        h->first_call = true;
        h->md_step = 0;
        h->nlaunch += 1;
        launch_init_walkers(h->W, h->N, h->p.L, h->d_R, h->d_X, make_key(h->p.seed), h->w0, h->stream);
        return check_launch();
    }
    if (option == QMC_OPT_RECOMPUTE) {
        if (value != QMC_RECOMPUTE_FP64 && value != QMC_RECOMPUTE_NEWTON) return QMC_ERR_INVALID;
        if (value == QMC_RECOMPUTE_NEWTON && !h->mixed) return QMC_ERR_INVALID;
        h->ns_recompute = value == QMC_RECOMPUTE_NEWTON;
        return QMC_OK;
    }
    return QMC_ERR_INVALID;
}

int qmc_set_profiling(qmc_system* h, int on) {
    if (!h) return QMC_ERR_INVALID;
    h->profiling = on != 0;
    return QMC_OK;
}

int qmc_kernel_times(qmc_system* h, int n, double* ms, long long* launches) {
    if (!h || n < 0) return QMC_ERR_INVALID;
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return QMC_ERR_CUDA;
    for (auto& e : h->events) {
        float t = 0.f;
        cudaEventElapsedTime(&t, e.a, e.b);
        h->ktime[e.cls] += t;
        h->free_events.push_back(e);
    }
    h->events.clear();
    for (int k = 0; k < n && k < QMC_NKERNEL; ++k) {
        if (ms) ms[k] = h->ktime[k];
        if (launches) launches[k] = h->klaunch[k];
    }
    for (int k = 0; k < QMC_NKERNEL; ++k) { h->ktime[k] = 0; h->klaunch[k] = 0; }
    return QMC_OK;
}

long long qmc_launch_count(qmc_system* h) { return h ? h->nlaunch : -1; }

// Checkpoint layout: 8 int64 header words [magic, version, N, W, md_step,
// first_call, langevin_first, langevin_step_no], last_Nc (double), then
// X [W][N][3], R_prev [3N], S_prev [3N][3N] (doubles).
namespace {
constexpr long long kCkptMagic = 0x514D43504B505431LL;  // "QMCPKPT1"
size_t ckpt_bytes(const qmc_system* h) {
    const size_t N3 = 3 * (size_t)h->N;
    return 8 * sizeof(long long) + sizeof(double) + sizeof(double) * ((size_t)h->W * N3 + N3 + N3 * N3);
}
}  // namespace

size_t qmc_checkpoint_size(qmc_system* h) { return h ? ckpt_bytes(h) : 0; }

int qmc_checkpoint_save(qmc_system* h, void* buf) {
    if (!h || !buf) return QMC_ERR_INVALID;
    const size_t N3 = 3 * (size_t)h->N;
    long long* hd = (long long*)buf;
    hd[0] = kCkptMagic; hd[1] = 1; hd[2] = h->N; hd[3] = h->W; hd[4] = h->md_step;
    hd[5] = h->first_call; hd[6] = h->langevin_first; hd[7] = h->langevin_step_no;
    double* d = (double*)(hd + 8);
    d[0] = h->last_Nc;
    double* X = d + 1;
    cudaMemcpyAsync(X, h->d_X, sizeof(double) * h->W * N3, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(X + h->W * N3, h->d_Rprev, sizeof(double) * N3, cudaMemcpyDeviceToHost, h->stream);
    cudaMemcpyAsync(X + h->W * N3 + N3, h->d_Sprev, sizeof(double) * N3 * N3, cudaMemcpyDeviceToHost, h->stream);
    return read_err(h);
}

int qmc_checkpoint_load(qmc_system* h, const void* buf) {
    if (!h || !buf) return QMC_ERR_INVALID;
    const long long* hd = (const long long*)buf;
    if (hd[0] != kCkptMagic || hd[1] != 1 || hd[2] != h->N || hd[3] != h->W) return QMC_ERR_INVALID;
    const size_t N3 = 3 * (size_t)h->N;
    h->md_step = (uint32_t)hd[4];
    h->first_call = hd[5] != 0;
    h->langevin_first = hd[6] != 0;
    h->langevin_step_no = (uint32_t)hd[7];
    const double* d = (const double*)(hd + 8);
    h->last_Nc = d[0];
    const double* X = d + 1;
    cudaMemcpyAsync(h->d_X, X, sizeof(double) * h->W * N3, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->d_Rprev, X + h->W * N3, sizeof(double) * N3, cudaMemcpyHostToDevice, h->stream);
    cudaMemcpyAsync(h->d_Sprev, X + h->W * N3 + N3, sizeof(double) * N3 * N3, cudaMemcpyHostToDevice, h->stream);
    return read_err(h);
}

const char* qmc_kernel_name(int k) { return (k >= 0 && k < QMC_NKERNEL) ? kKernelNames[k] : "?"; }

const char* qmc_strerror(int code) {
    switch (code) {
        case QMC_OK: return "ok";
        case QMC_ERR_INVALID: return "invalid argument";
        case QMC_ERR_OOM: return "out of device memory";
        case QMC_ERR_CUDA: return "CUDA runtime error";
        case QMC_ERR_NOT_PD: return "acceleration matrix S is not positive definite";
        case QMC_ERR_NONFINITE: return "non-finite local energy, ratio or force";
        case QMC_ERR_TIMEOUT: return "bounded device wait gave up";
        case QMC_ERR_SINGULAR: return "singular Slater matrix";
        default: return "unknown error";
    }
}

}  // extern "C"
