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

namespace qmc {

namespace {

// Cholesky S = L L^T of an n x n SPD matrix (row-major) by one CTA,
// left-looking, column by column, into the lower triangle of Lc.  Returns
// false on every thread if S is not positive definite (the pivot test uses a
// block-wide sum, so all threads see the same value).
__device__ bool cta_cholesky(int n, const double* __restrict__ S, double* Lc, double* red) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < n; ++j) {
        double p = 0.0;
        for (int k = tid; k < j; k += nt) p += Lc[(size_t)j * n + k] * Lc[(size_t)j * n + k];
        p = block_sum(p, red);
        const double d = S[(size_t)j * n + j] - p;
        if (!(d > 0.0)) return false;
        const double ljj = sqrt(d);
        if (tid == 0) Lc[(size_t)j * n + j] = ljj;
        for (int i = j + 1 + tid; i < n; i += nt) {
            double t = S[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= Lc[(size_t)i * n + k] * Lc[(size_t)j * n + k];
            Lc[(size_t)i * n + j] = t / ljj;
        }
        __syncthreads();
    }
    return true;
}

// In-place forward solve L w = g (g in shared memory), column oriented.
__device__ void cta_forward(int n, const double* Lc, double* g) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = 0; k < n; ++k) {
        const double wk = g[k] / Lc[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) g[k] = wk;
        for (int i = k + 1 + tid; i < n; i += nt) g[i] -= Lc[(size_t)i * n + k] * wk;
        __syncthreads();
    }
}

// Back solve L^T x = w (w in shared memory, consumed), column oriented.
__device__ void cta_backward(int n, const double* Lc, double* w, double* x) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = n - 1; k >= 0; --k) {
        const double xk = w[k] / Lc[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) x[k] = xk;
        for (int i = tid; i < k; i += nt) w[i] -= Lc[(size_t)k * n + i] * xk;
        __syncthreads();
    }
}

}  // namespace

__global__ void __launch_bounds__(1024) langevin_kernel(int n, double* R, double* Rprev, const double* __restrict__ f,
                                                        const double* __restrict__ S, double* Sprev, double* Lc,
                                                        double T, double delta, double alpha, Key key, uint32_t md,
                                                        double box, int identity, int scheme, int* err) {
    extern __shared__ double v[];
    double* g = v;          // [n]
    double* x = g + n;      // [n]
    double* z = x + n;      // [n]
    double* r0 = z + n;     // [n]
    __shared__ double red[32];
    const int tid = threadIdx.x, nt = blockDim.x;
    double Dt = delta, Db = delta;
    if (!identity && scheme == kLvAdopted && alpha > 0.0) {
        Dt = (1.0 - exp(-alpha * delta)) / alpha;
        Db = (1.0 - exp(-2.0 * alpha * delta)) / (2.0 * alpha);
    }
    if (!identity && !cta_cholesky(n, S, Lc, red)) {
        if (tid == 0) raise_err(err, kErrNotPD);
        return;
    }
    // g = f - (S_prev - S)(R_prev - R) / (2 Db);  xi;  keep R
    for (int i = tid; i < n; i += nt) {
        double t = f[i];
        if (!identity && scheme != kLvNorogna) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += (Sprev[(size_t)i * n + j] - S[(size_t)i * n + j]) * (Rprev[j] - R[j]);
            t -= s / (2.0 * Db);
        }
        g[i] = t;
        const uint4 w = philox((uint32_t)i, md, 0u, kLangevin, key);
        z[i] = Draw<double>::normal(w);
        r0[i] = R[i];
    }
    __syncthreads();
    if (!identity) {
        // forward solve L y = g (column oriented), y stored in g
        for (int k = 0; k < n; ++k) {
            const double yk = g[k] / Lc[(size_t)k * n + k];
            __syncthreads();
            if (tid == 0) g[k] = yk;
            for (int i = k + 1 + tid; i < n; i += nt) g[i] -= Lc[(size_t)i * n + k] * yk;
            __syncthreads();
        }
        // back solves L^T x = y and L^T z = xi
        for (int k = n - 1; k >= 0; --k) {
            const double xk = g[k] / Lc[(size_t)k * n + k];
            const double zk = z[k] / Lc[(size_t)k * n + k];
            __syncthreads();
            if (tid == 0) { x[k] = xk; z[k] = zk; }
            for (int i = tid; i < k; i += nt) {
                g[i] -= Lc[(size_t)k * n + i] * xk;
                z[i] -= Lc[(size_t)k * n + i] * zk;
            }
            __syncthreads();
        }
    } else {
        for (int i = tid; i < n; i += nt) x[i] = g[i];
        __syncthreads();
    }
    const double amp = T > 0.0 ? sqrt(2.0 * T * Db) : 0.0;
    for (int i = tid; i < n; i += nt) {
        double r = r0[i] + Dt * x[i] + amp * z[i];
        if (box > 0.0) r -= box * floor(r / box);
        Rprev[i] = r0[i];
        R[i] = r;
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
    const size_t smem = 4 * (size_t)n3 * sizeof(double);
    langevin_kernel<<<1, 1024, smem, st>>>(n3, R, Rprev, f, S, Sprev, Lwork, T_ha, delta, alpha, key, md, box,
                                           identity, scheme, err);
}

}  // namespace qmc
