// k_langevin.cu -- accelerated first-order Langevin step (SI, adopted integrator):
//   R' = R + Dt S^{-1} [ f - (S_prev - S)(R_prev - R) / (2 Db) ] + sqrt(2 T Db) z,   <z z^T> = S^{-1}
//   Dt = (1 - e^{-alpha D}) / alpha,  Db = (1 - e^{-2 alpha D}) / (2 alpha)   (both D at alpha = 0)
// with S = L L^T (Cholesky), x = S^{-1} g by two triangular solves and z = L^{-T} xi,
// xi ~ N(0, I) from Philox (counter = (component, md step, 0, 7)).  One CTA, FP64.
// identity != 0 runs the conventional dynamics (S = I, alpha = 0).
// scheme selects the SI's variant: kLvAdopted (above), kLvFast (Eq. finaldyn:
// Dt = Db = D whatever alpha, i.e. R' = R + D S^{-1} f + sqrt(2 T D) z
// - 1/2 S^{-1}(S_prev - S)(R_prev - R)) or kLvNorogna (Eq. norogna: no S_prev
// term, Dt = Db = D).  T arrives already lowered by the noise correction when
// the caller asked for it.
// On exit (R_prev, S_prev) hold the pair of this step for the next call.
// first_predict_kernel / first_correct_kernel: the first simplified scheme
// (Eq. smartMarkov) in two halves, around the caller's evaluation of S(y).
#include "common.cuh"
#include "kernels.cuh"
#include "langevin_core.cuh"

namespace qmc {

__global__ void __launch_bounds__(1024) langevin_kernel(int n, double* R, double* Rprev, const double* __restrict__ f,
                                                        const double* __restrict__ S, double* Sprev, double* Lc,
                                                        double T, double delta, double alpha, Key key, uint32_t md,
                                                        double box, int identity, int scheme, int* err) {
    extern __shared__ double v[];
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    double* r1 = nullptr;
    if (!cta_langevin_step(n, R, Rprev, f, S, Sprev, Lc, T, delta, alpha, key, md, box, identity, scheme, v, red,
                           &r1)) {
        if (tid == 0) raise_err(err, kErrNotPD);
        return;
    }
    const double* r0 = r1 - n;   // R, kept by the step before any write
    for (int i = tid; i < n; i += nt) {
        Rprev[i] = r0[i];
        R[i] = r1[i];
    }
    for (size_t idx = tid; idx < (size_t)n * n; idx += nt) Sprev[idx] = identity ? (idx % (n + 1) == 0 ? 1.0 : 0.0) : S[idx];
}

// First simplified scheme (SI, Eq. smartMarkov), predict half: Cholesky of
// S(R) into Lc (kept for the correct half) and y = R + sqrt(2 T D) z,
// z = L^{-T} xi with the step's Philox noise; y is not wrapped (the correct
// half needs y - R).
__global__ void __launch_bounds__(1024) first_predict_kernel(int n, const double* __restrict__ R,
                                                             const double* __restrict__ S, double* Lc, double T,
                                                             double delta, Key key, uint32_t md, double* y, int* err) {
    extern __shared__ double v[];
    double* w = v;          // [n] xi, consumed by the solve
    double* z = w + n;      // [n]
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    if (!cta_cholesky(n, S, Lc, red)) {
        if (tid == 0) raise_err(err, kErrNotPD);
        return;
    }
    for (int i = tid; i < n; i += nt) w[i] = Draw<double>::normal(philox((uint32_t)i, md, 0u, kLangevin, key));
    __syncthreads();
    cta_backward(n, Lc, w, z);
    const double amp = T > 0.0 ? sqrt(2.0 * T * delta) : 0.0;
    for (int i = tid; i < n; i += nt) y[i] = R[i] + amp * z[i];
}

// Correct half: R' = y + S(R)^{-1} (D f(R) - 1/2 [S(y) - S(R)] (y - R)) with the
// kept factor of S(R); R' (in y) wrapped into [0, box) if box > 0.
__global__ void __launch_bounds__(1024) first_correct_kernel(int n, double* y, const double* __restrict__ R,
                                                             const double* __restrict__ f,
                                                             const double* __restrict__ S,
                                                             const double* __restrict__ Sy,
                                                             const double* __restrict__ Lc, double delta, double box) {
    extern __shared__ double v[];
    double* g = v;          // [n]
    double* x = g + n;      // [n]
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < n; i += nt) {
        double s = 0.0;
        for (int j = 0; j < n; ++j) s += (Sy[(size_t)i * n + j] - S[(size_t)i * n + j]) * (y[j] - R[j]);
        g[i] = delta * f[i] - 0.5 * s;
    }
    __syncthreads();
    cta_forward(n, Lc, g);
    cta_backward(n, Lc, g, x);
    for (int i = tid; i < n; i += nt) {
        double r = y[i] + x[i];
        if (box > 0.0) r -= box * floor(r / box);
        y[i] = r;
    }
}

void launch_first_predict(int n3, const double* R, const double* S, double* Lwork, double T_ha, double delta, Key key,
                          uint32_t md, double* y, int* err, cudaStream_t st) {
    first_predict_kernel<<<1, 1024, 2 * (size_t)n3 * sizeof(double), st>>>(n3, R, S, Lwork, T_ha, delta, key, md, y,
                                                                          err);
}

void launch_first_correct(int n3, double* y, const double* R, const double* f, const double* S, const double* Sy,
                          const double* Lwork, double delta, double box, cudaStream_t st) {
    first_correct_kernel<<<1, 1024, 2 * (size_t)n3 * sizeof(double), st>>>(n3, y, R, f, S, Sy, Lwork, delta, box);
}

void launch_langevin(int n3, double* R, double* Rprev, const double* f, const double* S, double* Sprev,
                     double* Lwork, double T_ha, double delta, double alpha, Key key, uint32_t md, double box,
                     int identity, int scheme, int* err, cudaStream_t st) {
    const size_t smem = 5 * (size_t)n3 * sizeof(double);
    langevin_kernel<<<1, 1024, smem, st>>>(n3, R, Rprev, f, S, Sprev, Lwork, T_ha, delta, alpha, key, md, box,
                                           identity, scheme, err);
}

}  // namespace qmc
