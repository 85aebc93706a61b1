/*
 * qmcmd.h -- C ABI of the GB300 library for the data-parallel hot path of
 * Sorella & Mazzola, "Accelerated ab-initio Molecular Dynamics" (arXiv:1605.08423):
 * Variational Monte Carlo (VMC) evaluation of the Born-Oppenheimer energy, the
 * nuclear forces and their covariance for N protons in a periodic cubic box,
 * and the accelerated first-order Langevin step that consumes them.
 *
 * Conventions shared by every entry point
 *   - Units: bohr, hartree.  Temperatures are given in kelvin and converted with
 *     k_B = 3.166811563e-6 Ha/K.
 *   - Arrays are dense, row-major, FP64 unless stated.  R is [N][3]; electron
 *     configurations are [W][N][3] with electrons 0..N/2-1 spin up and
 *     N/2..N-1 spin down.
 *   - Ownership: the caller owns every pointer it passes.  The library copies
 *     what it needs during the call and keeps no caller pointer afterwards.
 *     All device state (walkers, inverses, tables) is owned by the handle and
 *     released by qmc_destroy.
 *   - "_device" variants take device pointers and are asynchronous on the
 *     handle's stream (qmc_set_stream); errors they raise on the GPU are
 *     reported by the next qmc_sync.  All other calls take host pointers and
 *     return only after the result is on the host.
 *   - Return value: QMC_OK (0) or a negative QMC_ERR_* code; qmc_strerror
 *     gives its text.  A failed call leaves caller arrays unspecified.
 *   - Threading: one handle per host thread at a time.
 */
#ifndef QMCMD_H
#define QMCMD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    QMC_OK = 0,
    QMC_ERR_INVALID = -1,   /* bad argument (sizes, parity of N, null pointer) */
    QMC_ERR_OOM = -2,       /* device allocation failed / footprint above the cap */
    QMC_ERR_CUDA = -3,      /* CUDA runtime error (no device, launch failure) */
    QMC_ERR_NOT_PD = -4,    /* S is not positive definite (Cholesky failed) */
    QMC_ERR_NONFINITE = -5, /* a local energy, ratio or force was not finite */
    QMC_ERR_TIMEOUT = -6,   /* a bounded device wait gave up */
    QMC_ERR_SINGULAR = -7   /* a Slater matrix was exactly singular */
};

enum { QMC_FP64 = 0, QMC_MIXED = 1 };          /* precision forms */
enum { QMC_S_IDENTITY = 0, QMC_S_COV = 1, QMC_S_EMPIRICAL = 2 };   /* acceleration matrix of langevin_step */

/*
 * System and sampler parameters (the wavefunction of the paper's Eq. for
 * V(R) restricted to a Jastrow-Slater form: psi = det(Phi_up) det(Phi_dn) e^U,
 * orbitals phi_j(r) = sum_b coeff[b][j] exp(-zeta_g |d(r - R_a)|^2), b = a*n_gauss + g,
 * d the sin-periodised displacement of the SI, U = Pade e-e + e-n terms).
 */
typedef struct {
    int32_t n_protons;        /* N, even, 2..128; N electrons, N/2 per spin             */
    int32_t n_gauss;          /* Gaussians per proton, 1..8                              */
    int32_t n_walkers;        /* W >= 2                                                  */
    int32_t n_sweeps;         /* measured sweeps per qmc_energy_forces call              */
    int32_t n_warmup;         /* sweeps before the first measurement of the first call   */
    int32_t n_warmup_cont;    /* same, for later calls (walkers carried over)            */
    int32_t measure_every;    /* sweeps between samples, >= 1                           */
    int32_t recompute_every;  /* sweeps between periodic inverse recomputes, >= 1 (see   */
                              /* QMC_OPT_RECOMPUTE for how each form recomputes)         */
    int32_t precision;        /* QMC_FP64 or QMC_MIXED                                   */
    int32_t ewald_mmax;       /* reciprocal cutoff |m| <= mmax (k = 2 pi m / L)          */
    double L;                 /* box side, bohr                                          */
    double b_ee, b_ep;        /* Pade Jastrow parameters                                 */
    double ewald_kappa;       /* Ewald splitting parameter, bohr^-1 (e.g. 5/L)           */
    double sigma;             /* Gaussian proposal width, bohr                           */
    uint64_t seed;            /* Philox4x32-10 key                                       */
    const double* zeta;       /* [n_gauss] exponents, bohr^-2 (copied)                   */
    const double* coeff;      /* [N*n_gauss][N/2] orbital coefficients (copied)          */
    /* 3- and 4-body e-e-n-n Jastrow term of the SI, one periodised Gaussian
     * chi_a(r) = exp(-zeta_j |d(r - R_a)|^2) per proton:
     *   U += sum_{i<j} sum_{a,b} fj[a][b] chi_a(r_i) chi_b(r_j).
     * fj = NULL switches it off.  Both forms (the mixed form in FP32), and fj
     * must be exactly symmetric (fj[a][b] == fj[b][a]); INVALID otherwise. */
    double zeta_j;            /* Jastrow-orbital exponent, bohr^-2 (the SI uses 0.7933844) */
    const double* fj;         /* [N][N] symmetric coefficients (copied), or NULL         */
    /* Twisted boundary conditions (SI, basis section: phi(r + nL) = e^{i theta.n} phi(r))
     * and the k-point average of the main text.  n_twist = 0: the real
     * Gamma-point form above.  n_twist = K > 0: FP64 form only (fj allowed),
     * W a multiple of K with W/K >= 2 (INVALID otherwise).  The orbitals are then
     * Bloch-summed Gaussians
     *   chi_{a,g}(r) = sum_n e^{i theta.n} exp(-zeta_g |r - R_a - nL|^2)
     * (images n = k + m, m in [-M, M]^3 around the nearest one k, with
     * M = max(1, ceil(sqrt(40 / zeta_min) / L - 1/2))), complex, with the same
     * real coefficients; the spin-up determinant carries theta and the
     * spin-down one -theta; the Jastrow factor is unchanged.  Walkers come in K
     * contiguous blocks of W/K, block t sampling |psi_t|^2 with twist
     * twist[3t..3t+2]; E_L and the estimators take real parts.  Each block is
     * reduced on its own and the results averaged with equal weights:
     * E, f and the acceptance are the means over the twists, n_samples the
     * sum, E_err = sqrt(sum E_err_t^2) / K and S = sum S_t / K^2.  Served
     * trajectories may be twisted; the walker-sharded calls reject twisted
     * handles (the twists shard instead: qmc_twist_partial_device). */
    int32_t n_twist;          /* K, number of twists (0: Gamma point)                    */
    int32_t pad_twist;        /* unused, 0                                               */
    const double* twist;      /* [K][3] twist vectors theta, radians (copied), or NULL   */
} qmc_params;

/* Result of one energy/force evaluation.  f and cov are caller-allocated host
 * arrays of 3N and 3N*3N doubles. */
typedef struct {
    double E;          /* VMC energy, hartree                                   */
    double E_err;      /* its error bar (walker blocks)                         */
    double* f;         /* [3N] mean force -dE/dR, Ha/bohr                       */
    double* cov;       /* [3N][3N] covariance of the mean force (S)             */
    double n_samples;  /* N_c = walkers x measured sweeps / measure_every       */
    double accept;     /* Metropolis acceptance ratio of the call               */
} qmc_result;

typedef struct qmc_system qmc_system;

/* Create a handle: validates p, allocates all device state on the current
 * CUDA device, uploads R ([N][3], host) and places the walkers (each electron
 * next to a proton plus 0.5 bohr Philox noise).  Errors: INVALID, OOM, CUDA. */
int qmc_init(const qmc_params* p, const double* R, qmc_system** out);

/* Release every device allocation of h (h may be NULL). */
void qmc_destroy(qmc_system* h);

/* Bytes of device memory a handle with parameters p holds (admission control). */
size_t qmc_footprint_bytes(const qmc_params* p);

/* Launch subsequent work of h on `stream` (a cudaStream_t; NULL = the handle's
 * own stream, so pass cudaStreamLegacy for the legacy default stream). */
int qmc_set_stream(qmc_system* h, void* stream);

/* Wait for h's stream and return the device-side error status (QMC_OK or a code). */
int qmc_sync(qmc_system* h);

/*
 * The hot path.  For nuclei R (host [N][3]): full inverse recompute, n_warmup
 * (first call) or n_warmup_cont sweeps, then n_sweeps Metropolis sweeps with a
 * local-energy and force sample every measure_every sweeps, then the
 * reductions of the paper's covariance-matrix definition:
 *   E = <E_L>,  f = -<dE_L/dR> - 2(<E_L dlnpsi/dR> - E <dlnpsi/dR>)   (Hellmann-Feynman + Pulay)
 *   S = Cov(f) of the mean, from walker blocks.
 * Walkers carry over to the next call.  Errors: INVALID, CUDA, NONFINITE, SINGULAR.
 */
int qmc_energy_forces(qmc_system* h, const double* R, qmc_result* out);

/* Same, device pointers, asynchronous: R_dev [N][3]; out_dev receives
 * [E, E_err, n_samples, accept, f(3N), S(3N*3N)] as FP64. */
int qmc_energy_forces_device(qmc_system* h, const double* R_dev, double* out_dev);

/*
 * Pressure of the last qmc_energy_forces call (the paper's equations of state;
 * the paper does not state its estimator).  The Coulomb potential, including
 * its Ewald sum with kappa L and the k cutoff in units of 2 pi / L held fixed,
 * is homogeneous of degree -1 in all lengths, so for the trial state scaled
 * with the box E(lambda) = T / lambda^2 + V / lambda and the virial gives
 *   P = (2 <T_L> + <V_L>) / (3 L^3) + N k_B T / L^3
 * (electrons, then the ideal-gas term of classical nuclei at temperature
 * T_kelvin; pass 0 for the electronic part alone).  out [5] = [P, its error bar
 * from walker blocks, the electronic part, <V_L>, <T_L>], hartree / bohr^3
 * (1 Ha/bohr^3 = 29421.0 GPa) and hartree.  qmc_pressure takes a host array and
 * returns after the result is there; qmc_pressure_device writes device memory
 * asynchronously.  For this handle's walkers only (a sharded evaluation would
 * need its per-walker sums combined).  Errors: INVALID, CUDA.
 */
int qmc_pressure(qmc_system* h, double T_kelvin, double* out);
int qmc_pressure_device(qmc_system* h, double T_kelvin, double* out_dev);

/*
 * Walker sharding.  Walkers are independent Markov chains, so one energy/force
 * evaluation can be split over P processes (one GPU each), each holding a
 * slice of the walkers (QMC_OPT_WALKER_OFFSET = index of its first walker).
 * The reduction of qmc_energy_forces then takes three calls around two sums
 * over the processes (e.g. an all-reduce); every pointer is a device pointer
 * and every call is asynchronous on the handle's stream:
 *   qmc_shard_sample_device   sampling at nuclei R_dev ([N][3]) as in
 *                             qmc_energy_forces_device, then this handle's
 *                             sums_dev [3 + 9N + 3] = [column sums of the
 *                             per-walker accumulators (layout of
 *                             qmc_get_accumulators), accepted moves, walkers,
 *                             moves]                      -> sum over processes
 *   qmc_shard_reduce_device   from the summed sums_dev: E, N_c, acceptance and
 *                             f into out_dev (layout of qmc_energy_forces_device),
 *                             and this handle's gram_dev [1 + 9N^2] =
 *                             [sum_w (E_w - E)^2, sum_w (f_w - f)(f_w - f)^T] with
 *                             the global E and f         -> sum over processes
 *   qmc_shard_finish_device   E_err and S into out_dev from the summed gram_dev;
 *                             walkers_total (the walkers of all processes) sets
 *                             N_c for the alpha of a later langevin_step.
 * The result equals that of one handle holding all walkers, up to the order
 * of the FP64 sums.  Every process then applies the same Langevin step (same
 * seed, same MD step, same inputs: the same R').  Errors: INVALID, CUDA; device
 * errors via qmc_sync.
 */
int qmc_shard_sample_device(qmc_system* h, const double* R_dev, double* sums_dev);
int qmc_shard_reduce_device(qmc_system* h, const double* sums_dev, double* out_dev, double* gram_dev);
int qmc_shard_finish_device(qmc_system* h, const double* sums_dev, const double* gram_dev, double* out_dev,
                            long long walkers_total);

/*
 * Accelerated first-order Langevin step (SI, adopted integrator):
 *   R' = R + Dt S^{-1} [ f - (S_prev - S)(R_prev - R) / (2 Db) ] + sqrt(2 T Db) z,  <z z^T> = S^{-1},
 *   Dt = (1 - e^{-alpha Delta})/alpha,  Db = (1 - e^{-2 alpha Delta})/(2 alpha)
 * with (R_prev, S_prev) the pair of the previous call kept in h (equal to the
 * current pair on the first call).  s_mode QMC_S_IDENTITY: S = I, alpha = 0
 * (conventional first-order Langevin); QMC_S_COV: S as given and
 * alpha = 0.122 N_c of the last qmc_energy_forces call unless alpha > 0;
 * QMC_S_EMPIRICAL: S = H + mu I at the current R built on the device (see
 * qmc_set_empirical_s; the S argument is ignored), alpha as given (>= 0; 0
 * gives Dt = Db = Delta).  In the periodic box R_prev - R is taken as the
 * minimum image (the previous step's displacement).
 * R (host, [3N]) is updated in place and wrapped into [0, L).  Noise from
 * Philox (key = seed, counter = (component, step, 0, 7)).
 * Errors: INVALID, NOT_PD, CUDA.
 */
int langevin_step(qmc_system* h, double* R, const double* f, const double* S,
                  double T_kelvin, double delta, int s_mode, double alpha);

/* Same, device pointers, asynchronous (R_dev in/out). */
int langevin_step_device(qmc_system* h, double* R_dev, const double* f_dev, const double* S_dev,
                         double T_kelvin, double delta, int s_mode, double alpha);

/*
 * Twists sharded over processes (one GPU each; twisted handles only): each
 * process's handle samples its own K_r of the K twists, all with the same
 * walkers per twist, and qmc_energy_forces_device gives its average over them
 * in out_dev.  qmc_twist_partial_device turns that into the process's
 * contribution part_dev = [K_r E, (K_r E_err)^2, N_c, K_r accept, K_r f, K_r^2 S]
 * (4 + 3N + 9N^2 doubles); after the caller sums the contributions over the
 * processes (an all-reduce), qmc_twist_combine_device writes the average over
 * all K_total twists in the layout of qmc_energy_forces_device (the rule of the
 * n_twist comment: means, N_c summed, E_err = sqrt(sum E_err_t^2) / K,
 * S = sum S_t / K^2).  Device pointers, asynchronous.  Errors: INVALID (a
 * handle without twists, K_total below its K), CUDA.
 */
int qmc_twist_partial_device(qmc_system* h, const double* out_dev, double* part_dev);
int qmc_twist_combine_device(qmc_system* h, const double* part_dev, int K_total, double* out_dev);

/*
 * Empirical acceleration matrix (main text, conclusions: S = H + mu I with H the
 * Hessian of an accurate and cheap empirical potential and mu > 0 where H is
 * not positive definite; the paper names no potential).  H here is the Hessian
 * of the screened-Coulomb (Yukawa) pair potential of the protons,
 *   V = sum_{a<b} sum_{n : |d_ab + nL| < L} exp(-r/lambda) / r,  r = |d_ab + nL|,
 * images within one box side.  It has the three uniform translations as zero
 * modes, so mu > 0 is needed for a positive definite S.
 * qmc_set_empirical_s sets lambda (bohr; <= 0: the Thomas-Fermi length
 * 1/sqrt(4 k_F / pi), k_F = (3 pi^2 N / L^3)^(1/3), the default) and mu
 * (hartree / bohr^2, >= 0; default 0.5) for s_mode QMC_S_EMPIRICAL.  A mu
 * below minus the lowest eigenvalue of H makes the step fail with NOT_PD (its
 * Cholesky factorisation of S), and the caller raises mu.
 * qmc_empirical_s writes S = H + mu I at nuclei R (host [N][3]) into S (host
 * [3N][3N]); the _device form takes device pointers and is asynchronous.
 * Errors: INVALID, CUDA.
 */
int qmc_set_empirical_s(qmc_system* h, double lambda, double mu);
int qmc_empirical_s(qmc_system* h, const double* R, double* S);
int qmc_empirical_s_device(qmc_system* h, const double* R_dev, double* S_dev);

/*
 * First simplified scheme of the SI (Eq. smartMarkov), which needs S at the
 * predicted point and therefore a second energy/force evaluation per MD step,
 * in two calls around it:
 *   langevin_first_predict  R (host [3N], in) -> y = R + sqrt(2 T Delta) z,
 *                           <z z^T> = S^{-1}(R) (R overwritten with y, not
 *                           wrapped); keeps R, f(R), S(R) and the Cholesky
 *                           factor of S(R) in h.  Noise as in langevin_step.
 *   (the caller evaluates S(y), e.g. qmc_energy_forces at y)
 *   langevin_first_correct  y (host [3N], in) -> R' = y + Delta S^{-1}(R) f(R)
 *                           - 1/2 S^{-1}(R) [S(y) - S(R)] (y - R), wrapped into
 *                           [0, L); advances the MD step counter.
 * QMC_OPT_NOISE_CORRECTION applies to the predict half.  A correct call
 * without a pending predict is INVALID; a checkpoint does not carry a pending
 * predict.  Errors: INVALID, NOT_PD (S(R)), CUDA.
 */
int langevin_first_predict(qmc_system* h, double* R, const double* f, const double* S, double T_kelvin,
                           double delta);
int langevin_first_correct(qmc_system* h, double* y, const double* S_y);

/*
 * The same Langevin step for callers that cannot allocate device memory (the
 * paper has no counterpart: this is a deployment entry point).  cudaMalloc and
 * cudaFree may synchronise the device, which a host overlapping many
 * trajectories on streams or running a latency-bound MD loop cannot afford, and
 * some embedding hosts own all device memory and hand the library only
 * pre-allocated buffers.  This call allocates nothing and needs no handle:
 *   R      device [n3], in: R_n, out: R_{n+1} (wrapped into [0, box) if box > 0)
 *   Rprev  device [n3], R_{n-1} (pass R itself on the first step)
 *   f      device [n3] force; S, Sprev device [n3][n3] (ignored for QMC_S_IDENTITY;
 *          pass S as Sprev on the first step)
 *   alpha  >= 0, used as given (0: Dt = Db = delta); seed/step: Philox key and MD step
 *   stream cudaStream_t (NULL = default stream); the call returns after the step.
 * Workspace: a statically allocated device array of QMC_STATIC_MAX_N3^2 doubles
 * (1.18 MB) that every GPU which loads the library holds until exit.  The first
 * call on each device looks its address up (make it before any stream capture).
 * Calls that overlap on the GPU share the array and race.  n3 > QMC_STATIC_MAX_N3
 * is rejected.  Errors: INVALID, NOT_PD, CUDA.
 */
enum { QMC_STATIC_MAX_N3 = 384 };
int qmc_langevin_step_static(int n3, double* R, const double* Rprev, const double* f, const double* S,
                             const double* Sprev, double T_kelvin, double delta, int s_mode, double alpha,
                             uint64_t seed, uint32_t step, double box, void* stream);

/*
 * Per-configuration evaluation (parity checks): for n_conf <= n_walkers
 * configurations X (host [n_conf][N][3]) at nuclei R, returns ln|psi|, E_L
 * and the R-derivatives d ln|psi|/dR, dE_L/dR ([n_conf][N][3]) from the same
 * kernels the sampler uses.  Overwrites the first n_conf walkers.  With
 * twists, configuration c is evaluated as walker c: twist c / (n_walkers / K).
 */
int qmc_eval_config(qmc_system* h, int n_conf, const double* X, const double* R,
                    double* logpsi, double* EL, double* dlogpsi_dR, double* dEL_dR);

/* Copy walker positions out of / into the handle (host [n_walkers][N][3]). */
int qmc_get_walkers(qmc_system* h, double* X);
int qmc_set_walkers(qmc_system* h, const double* X);

/* Per-walker accumulators of the last call, host [n_walkers][3 + 9N]:
 * [count, sum E_L, sum E_L^2, sum dlnpsi/dR (3N), sum E_L dlnpsi/dR (3N), sum dE_L/dR (3N)]. */
int qmc_get_accumulators(qmc_system* h, double* acc);

/* Handle options.  QMC_OPT_TENSOR_CORES (mixed form with N = 128 and n_gauss =
 * 4, default 1; other systems always use the SIMT kernels): evaluate the
 * orbital contractions with the tcgen05 tensor-core kernel (2xTF32 split,
 * FP32-level accuracy); 0 selects the SIMT FP32 kernel.
 * QMC_OPT_TC_ADJOINT (where QMC_OPT_TENSOR_CORES is available; default 1):
 * while tensor cores are on, the B x n contractions of the orbital force terms
 * (Z = C G, P = C G Y G) and their basis-derivative epilogue run in a separate
 * tcgen05 kernel (2xTF32 pieces, 3 products); 0 keeps them in the SIMT
 * measure kernel.  INVALID for an unknown option or when the form has no such
 * kernel. */
enum { QMC_OPT_TENSOR_CORES = 1, QMC_OPT_TC_ADJOINT = 2 };
/* QMC_OPT_INTEGRATOR selects the scheme of later langevin_step /
 * langevin_step_device calls with s_mode QMC_S_COV (SI, integration schemes):
 *   QMC_LV_ADOPTED (default)  the adopted step written at langevin_step;
 *   QMC_LV_FAST               Eq. finaldyn, the same with Dt = Db = Delta whatever
 *                             alpha: R' = R + Delta S^{-1} f + sqrt(2 T Delta) z
 *                                         - 1/2 S^{-1} (S_prev - S)(R_prev - R);
 *   QMC_LV_NOROGNA            Eq. norogna, without the S_prev term (samples a wrong
 *                             distribution when S depends on R; kept for comparison).
 * QMC_OPT_NOISE_CORRECTION (default 0): 1 lowers the temperature of the step to
 * T - Delta/2 (SI "Noise correction", 2 T Delta = 2 T_target Delta - Delta^2, T
 * in hartree); a step with Delta >= 2 T is then INVALID. */
enum { QMC_OPT_INTEGRATOR = 3, QMC_OPT_NOISE_CORRECTION = 4 };
enum { QMC_LV_ADOPTED = 0, QMC_LV_FAST = 1, QMC_LV_NOROGNA = 2 };
/* QMC_OPT_RECOMPUTE selects the periodic inverse recompute inside a call
 * (every recompute_every sweeps; the recompute at the start of every call is
 * always the FP64 one):
 *   QMC_RECOMPUTE_FP64 (default)  Slater blocks at the current positions, then
 *                                 FP64 Gauss-Jordan inverse and ln|det| (resets the
 *                                 drift of the Sherman-Morrison updates);
 *   QMC_RECOMPUTE_NEWTON          mixed form only: one Newton-Schulz step
 *                                 G <- G + G (I - A G) on the carried inverse, the
 *                                 residual I - A G formed with a compensated (error-
 *                                 free product, TwoSum) FP32 dot product, so that G
 *                                 becomes the inverse of the FP32 Slater block to
 *                                 FP32 rounding; FP64 Gauss-Jordan for blocks with
 *                                 max|I - A G| >= 0.01.  ln|det| is not updated.
 *                                 About a third of the FP64 recompute's time on
 *                                 parts whose FP64 rate is 1/64 of FP32.
 * INVALID for other values, and for QMC_RECOMPUTE_NEWTON in the FP64 form. */
enum { QMC_OPT_RECOMPUTE = 5 };
/* QMC_OPT_WALKER_OFFSET (value >= 0, default 0): the handle's walker w draws
 * its random numbers from Philox stream value + w, so that handles holding
 * consecutive slices of one walker population (walker sharding, below)
 * reproduce the chains of a single handle holding all of them.  Setting it
 * places the walkers again (as qmc_init does, with the new streams) and makes
 * the next call a first call (n_warmup sweeps, MD step counter 0); set it
 * right after qmc_init. */
enum { QMC_OPT_WALKER_OFFSET = 6 };
enum { QMC_RECOMPUTE_FP64 = 0, QMC_RECOMPUTE_NEWTON = 1 };
int qmc_set_option(qmc_system* h, int option, int value);

/*
 * Rotating-spring toy model (SI, "A simple toy model"): the planar spring end
 * point R = (x, y) with U = k/2 (|R| - a)^2, free to rotate, integrated by the
 * SI's schemes for many independent trajectories at once (one GPU thread
 * each, FP64).  The acceleration matrix is
 *   QMC_TOY_S_G   S = G_lambda, the matrix printed in the SI
 *                 (G_lambda = P_r/lambda + P_t, P_r = R R^T/|R|^2, P_t = I - P_r);
 *   QMC_TOY_S_HG  S = H + mu G_lambda, H = grad grad U (positive definite only for
 *                 |R| > k a / (k + mu)).
 * Schemes (z = L^{-T} xi with S(R) = L L^T, xi ~ N(0, I); R_prev = R on the first step):
 *   QMC_TOY_PLAIN     S = I: R' = R + D f + sqrt(2 T D) xi
 *   QMC_TOY_STANDARD  Eq. standard with the cumbersome term Gamma_j = sum_i d_i S^{-1}_{ji}:
 *                     R' = R + D S^{-1} f + T D Gamma + sqrt(2 T D) z
 *   QMC_TOY_FIRST     Eq. smartMarkov: y = R + sqrt(2 T D) z,
 *                     R' = y + D S^{-1} f - 1/2 S^{-1} [S(y) - S(R)] (y - R)
 *   QMC_TOY_FAST      Eq. finaldyn: R' = R + D S^{-1} f + sqrt(2 T D) z
 *                                       - 1/2 S^{-1} [S(R_prev) - S(R)] (R_prev - R)
 *   QMC_TOY_ADOPTED   Eq. finaldyn_new with Dt, Db of alpha (as langevin_step)
 *   QMC_TOY_NOROGNA   Eq. norogna: R' = R + D S^{-1} f + sqrt(2 T D) z
 * Noise: Philox4x32-10, key = seed, counter = (trajectory, step, 0, 8); the two
 * normals are the cosine and sine branches of Box-Muller on the block's two
 * 53-bit uniforms.
 * xy0 is [n_traj][2]; out is [n_traj][QMC_TOY_NOUT] =
 *   [x, y, sum U, sum U^2, sum |R|, polar angle travelled (unwrapped), status]
 * with the sums over the positions after steps n_burn .. n_steps-1 and status
 * s + 1 if S(R) was not positive definite at step s (that trajectory stops
 * there; others continue), else 0.
 * qmc_toy_langevin takes host arrays, returns after the run and gives
 * QMC_ERR_NOT_PD (with out filled) when any trajectory stopped;
 * qmc_toy_langevin_device takes device arrays and is asynchronous on `stream`
 * (a cudaStream_t, NULL = default stream); read the status column.
 * Errors: INVALID (unknown scheme or s_mode, delta <= 0, lambda <= 0, T < 0,
 * alpha < 0, n_burn outside [0, n_steps], null arrays), OOM, CUDA, NOT_PD.
 */
enum { QMC_TOY_PLAIN = 0, QMC_TOY_STANDARD = 1, QMC_TOY_FIRST = 2, QMC_TOY_FAST = 3, QMC_TOY_ADOPTED = 4,
       QMC_TOY_NOROGNA = 5 };
enum { QMC_TOY_S_G = 0, QMC_TOY_S_HG = 1 };
enum { QMC_TOY_NOUT = 7 };
typedef struct {
    double k, a;        /* spring stiffness and rest length                    */
    double T;           /* temperature, energy units of U                      */
    double delta;       /* time step D                                         */
    double lambda;      /* G_lambda parameter as printed (> 0; 1 gives S = I)  */
    double mu;          /* weight of G_lambda in QMC_TOY_S_HG                  */
    double alpha;       /* QMC_TOY_ADOPTED (0: Dt = Db = D)                    */
    int32_t scheme;     /* QMC_TOY_*                                           */
    int32_t s_mode;     /* QMC_TOY_S_G or QMC_TOY_S_HG                         */
    int32_t n_steps, n_burn;
    uint64_t seed;
} qmc_toy_params;
int qmc_toy_langevin(const qmc_toy_params* p, int n_traj, const double* xy0, double* out);
int qmc_toy_langevin_device(const qmc_toy_params* p, int n_traj, const double* xy0_dev, double* out_dev,
                            void* stream);

/* Set the MD step counter used in the Philox counters of the next call. */
int qmc_set_md_step(qmc_system* h, uint32_t md_step);

/* Kernel timing: when enabled, CUDA events on h's stream bracket every kernel
 * class; qmc_kernel_times fills ms[k] (total ms) and launches[k] for the
 * n <= QMC_NKERNEL classes named by qmc_kernel_name(k), then resets them. */
enum { QMC_NKERNEL = 9 };
int qmc_set_profiling(qmc_system* h, int on);
int qmc_kernel_times(qmc_system* h, int n, double* ms, long long* launches);
const char* qmc_kernel_name(int k);

/* Number of CUDA kernels this handle has launched so far (monotonic). */
long long qmc_launch_count(qmc_system* h);

/* Checkpoint / resume of a handle's sampler and MD state: walker positions,
 * the MD step counters and the Langevin history (R_prev, S_prev) -- everything a
 * later qmc_energy_forces / langevin_step depends on besides the parameters
 * (every call starts from a full inverse recompute, so inverses are not
 * stored).  qmc_checkpoint_size gives the byte size; save writes into a
 * caller-allocated host buffer; load restores into a handle created with the
 * same parameters (INVALID otherwise).  A handle restored from a checkpoint
 * continues bit-identically to the one that wrote it. */
size_t qmc_checkpoint_size(qmc_system* h);
int qmc_checkpoint_save(qmc_system* h, void* buf);
int qmc_checkpoint_load(qmc_system* h, const void* buf);

/*
 * Serving: continuous batching of MD-step requests from many concurrent
 * Langevin trajectories (each with its own N, density and temperature) on one
 * GPU.  A trajectory keeps its walkers resident between requests; a request is
 * one MD step (qmc_energy_forces at the trajectory's current nuclei, then
 * langevin_step).  Requests of one trajectory run in order; up to max_active
 * requests of different trajectories run at once on separate streams, so their
 * kernels overlap.  Admission is by device-memory footprint against
 * hbm_budget_bytes; idle trajectories are evicted least-recently-used with
 * their state checkpointed to host memory and restored on re-admission, so a
 * request's result is the same alone, in the mix and after an eviction.
 * qmc_server_progress never blocks: the caller's loop calls it to retire
 * finished requests and start queued ones, and qmc_server_fetch collects a
 * finished request (1 = done, 0 = still pending).
 * The budget is allocated as one device arena by qmc_server_create (OOM if it
 * cannot be); trajectories are carved from it, so admission and eviction
 * allocate and free no device memory.
 */
typedef struct qmc_server qmc_server;
typedef struct {
    int traj, status;                    /* trajectory id, QMC_OK or the request's error */
    double E, E_err, n_samples, accept;
    double* f;                           /* [3N] or NULL (caller-allocated)          */
    double* cov;                         /* [3N][3N] or NULL                        */
    double* R_next;                      /* [3N] nuclei after the Langevin step, or NULL */
    double latency_ms, wait_ms, run_ms;  /* submit->done, submit->start, start->done */
    double gpu_start_ms, gpu_end_ms;     /* the request's work on the device: from its start
                                            event to its end event, ms after the server was
                                            created (-1 if not timed) */
} qmc_served;
int qmc_server_create(size_t hbm_budget_bytes, int max_active, qmc_server** out);
void qmc_server_destroy(qmc_server* s);
/* Register a trajectory (device memory is taken only when it is admitted).
 * Parameters with the e-e-n-n Jastrow term (p->fj != NULL) are INVALID here. */
int qmc_server_add_trajectory(qmc_server* s, const qmc_params* p, const double* R0, double T_kelvin, double delta,
                              int s_mode, int* traj);
int qmc_server_submit(qmc_server* s, int traj, long long* ticket);
/* Retire finished requests and start queued ones; returns how many finished. */
int qmc_server_progress(qmc_server* s);
int qmc_server_fetch(qmc_server* s, long long ticket, qmc_served* out);
/* stats[8]: resident bytes, resident trajectories, active, queued, evictions,
 * completed, admissions, budget. */
int qmc_server_stats(qmc_server* s, long long* stats);

/* Text of an error code. */
const char* qmc_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif /* QMCMD_H */
