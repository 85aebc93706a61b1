// kernels.cuh -- host-side launchers of the qmcmd kernels (one per kernel class).
#pragma once
#include "common.cuh"

namespace qmc {

// k_orbitals.cu
template <typename T>
void launch_orbitals(const SysView<T>& s, const double* pos, int nrows, T* val, T* grad, T* lap, cudaStream_t st);
template <typename T>
void launch_propose(int W, int N, double L, double* X, double* Xp, T* ptp, T* uacc, Key key, uint32_t md,
                    uint32_t sweep, double sigma, uint32_t w0, cudaStream_t st);
void launch_init_walkers(int W, int N, double L, const double* R, double* X, Key key, uint32_t w0, cudaStream_t st);

// k_orbitals_tc.cu (tensor-core form of the value-only contraction)
bool tc_orbitals_supported(int n, int B);
void launch_orbitals_tc(const SysView<float>& s, const void* chat, const double* pos, int nrows, float* val,
                        float* grad, float* lap, cudaStream_t st);
void prepare_tc_coeff(const float* C, int B, int n, void* chat, cudaStream_t st);
size_t tc_coeff_bytes(int B, int n);

// k_adjoint_tc.cu (tensor-core form of the orbital part of the force
// estimators; the measure kernel then runs with kt_out/eg_out/elw set)
bool tc_adjoint_supported(int N, int n, int G);
size_t tc_adjoint_coeff_bytes(int n, int G);
void prepare_tc_adjoint_coeff(const float* C, int N, int G, int n, void* ahat, cudaStream_t st);
void launch_adjoint_tc(const SysView<float>& s, const void* ahat, const float* Gt, const float* Kt, const float* eg,
                       const double* elw, const float* frec, double* acc, double* out_dl, double* out_de,
                       cudaStream_t st);

// k_invert.cu: FP64 Gauss-Jordan inverse of each walker's two Slater blocks.
template <typename T>
void launch_invert(int W, int N, int n, const T* Phi, T* Gt, double* logdet, int* err, cudaStream_t st);

// k_invert.cu: mixed-form periodic recompute (one Newton-Schulz step, FP64
// Gauss-Jordan where the carried inverse is too far off).
void launch_refine(int W, int N, int n, const float* Phi, float* Gt, double* logdet, int* err, cudaStream_t st);

// k_sweep.cu: one Metropolis sweep per walker (warp per walker).
template <typename T>
// vep: [W][N] per-electron e-n Jastrow sums carried between the sweeps of a
// call by the mixed-form register sweep (computed when vep_init, i.e. in the
// call's first sweep); unused by the other sweep kernels.
void launch_sweep(const SysView<T>& s, double* X, const double* Xp, const T* ptp, const T* uacc, const T* Phi, T* Gt,
                  unsigned long long* nacc, float* vep, bool vep_init, cudaStream_t st);

// k_measure.cu: local energy, d ln psi / dR and dE_L / dR per walker.
template <typename T>
void launch_measure(const SysView<T>& s, const double* X, const T* D, const T* Lp, const T* Gt,
                    const double* logdet, double* acc, double* out_el, double* out_lnpsi, double* out_dl,
                    double* out_de, float* kt_out, float* eg_out, double* elw, float* rk_out, cudaStream_t st);
template <typename T>
size_t measure_smem_bytes(int N, int n, int nk, int mmax, bool split);

// k_setup.cu: per-R tables (proton trig, structure factors, p-p Ewald terms).
void launch_setup(int N, double L, double kappa, int nk, const int4* kvec, const double* R, double* kw,
                  double* ptrig64, float* ptrig32, double2* eikR, double2* rho_p, double* vconst, double* dvpp,
                  float* R32, float2* eikR32, float* kw32, cudaStream_t st);

// k_setup.cu: the reciprocal-space force as a [3N][2 nk] matrix on rho(k) (split measure path).
void launch_recforce_table(int N, int nk, double L, const int4* kvec, const double* kw, const double2* eikR, float* T,
                           cudaStream_t st);

// k_recforce.cu: F[W][M] = rho[W][K] . T[K][M] (reciprocal-space force of every walker sample).
void launch_recforce_gemm(int W, int M, int K, const float* rho, const float* T, float* F, cudaStream_t st);

// k_reduce.cu: walker reductions and the covariance matrix.
void launch_reduce(int W, int N, double moves, const double* acc, const unsigned long long* nacc,
                   double* colsum, double* dev, double* out, int* err, cudaStream_t st);
// k_reduce.cu: virial pressure of the last call's samples, out [5].
void launch_pressure(int W, int N, const double* acc, const double* vacc, double omega, double T_nuc, double* out,
                     cudaStream_t st);
// k_reduce.cu: walker-sharded form of the same reduction (see there): local
// sums [3 + 9N + 3], then E, f and local deviation sums gram [1 + 9N^2] from
// the summed sums, then E_err and S from the summed gram.
void launch_shard_sums(int W, int N, double moves, const double* acc, const unsigned long long* nacc, double* sums,
                       cudaStream_t st);
void launch_shard_reduce(int W, int N, const double* acc, const double* sums, double* dev, double* out, double* gram,
                         int* err, cudaStream_t st);
void launch_shard_finish(int N, const double* sums, const double* gram, double* out, cudaStream_t st);

// k_twist.cu: twisted boundary conditions (FP64 form, complex orbitals).
void launch_twist_orbitals(const SysView<double>& s, const TwistView& tv, const double* pos, int nrows,
                           double2* val, double2* grad, double2* lap, cudaStream_t st);
void launch_twist_invert(int W, int N, int n, const double2* Phi, double2* Gt, double* logdet, int* err,
                         cudaStream_t st);
void launch_twist_sweep(const SysView<double>& s, const TwistView& tv, double* X, const double* Xp, const double* ptp,
                        const double* uacc, const double2* Phi, double2* Gt, unsigned long long* nacc,
                        cudaStream_t st);
void launch_twist_gl(int rows, int N, int n, const double2* D, const double2* Lp, const double2* Gt, double* Dr,
                     double* Lpr, cudaStream_t st);
void launch_twist_unit_rows(int W, int n, double* Gtr, cudaStream_t st);
void launch_twist_pulay(const SysView<double>& s, const TwistView& tv, const double* X, const double2* D,
                        const double2* Lp, const double2* Gt, const double* elw, double* acc, double* out_dl,
                        double* out_de, cudaStream_t st);
size_t twist_pulay_smem_bytes(int N, int n, bool j34);
void launch_twist_average(int K, int N, const double* tout, double* out, cudaStream_t st);
void launch_twist_partial(int Kr, int N, const double* out, double* part, cudaStream_t st);
void launch_twist_combine(int K, int N, const double* part, double* out, cudaStream_t st);

// k_empirical.cu: S = H + mu I, H the Hessian of the screened-Coulomb proton pair potential.
void launch_empirical_s(int N, double L, const double* R, double lambda, double mu, double* S, cudaStream_t st);

// k_langevin.cu (scheme: kLvAdopted, kLvFast or kLvNorogna)
enum : int { kLvAdopted = 0, kLvFast = 1, kLvNorogna = 2 };
void launch_langevin(int n3, double* R, double* Rprev, const double* f, const double* S, double* Sprev,
                     double* Lwork, double T_ha, double delta, double alpha, Key key, uint32_t md, double box,
                     int identity, int scheme, int* err, cudaStream_t st);

// k_langevin.cu: first simplified scheme, predict (y) and correct (R') halves
void launch_first_predict(int n3, const double* R, const double* S, double* Lwork, double T_ha, double delta, Key key,
                          uint32_t md, double* y, int* err, cudaStream_t st);
void launch_first_correct(int n3, double* y, const double* R, const double* f, const double* S, const double* Sy,
                          const double* Lwork, double delta, double box, cudaStream_t st);

// k_toy.cu: rotating-spring toy model, one thread per trajectory (FP64).
struct ToyDev {
    double k, a;          // U = k/2 (|R| - a)^2
    double sr_const;      // radial eigenvalue of S: 1/lambda (G_lambda) or k + mu/lambda (H + mu G_lambda)
    double mu;            // tangential eigenvalue of S is 1 (G_lambda) or k (1 - a/r) + mu
    double T, delta;
    double dt, db;        // adopted scheme: (1 - e^{-alpha D})/alpha, (1 - e^{-2 alpha D})/(2 alpha)
    double half_idb;      // 1 / (2 db)
    double amp, ampb;     // sqrt(2 T D), sqrt(2 T Db)
    int scheme, s_mode, n_steps, n_burn;
    Key key;
};
void launch_toy(const ToyDev& p, int n_traj, const double* xy0, double* out, cudaStream_t st);

}  // namespace qmc
