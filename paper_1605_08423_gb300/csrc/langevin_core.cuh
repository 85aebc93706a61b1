// langevin_core.cuh -- one-CTA FP64 building blocks of the accelerated
// first-order Langevin step (SI, integration schemes), shared by the handle's
// kernel (k_langevin.cu) and the allocation-free entry point
// (k_langevin_static.cu), so that both compute the step with the same code.
#pragma once
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

// Cholesky S = L L^T of an n x n SPD matrix (row-major) by one CTA,
// left-looking, column by column, into the lower triangle of Lc.  Returns
// false on every thread if S is not positive definite (the pivot test uses a
// block-wide sum, so all threads see the same value).
__device__ inline bool cta_cholesky(int n, const double* __restrict__ S, double* Lc, double* red) {
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
__device__ inline void cta_forward(int n, const double* Lc, double* g) {
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
__device__ inline void cta_backward(int n, const double* Lc, double* w, double* x) {
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int k = n - 1; k >= 0; --k) {
        const double xk = w[k] / Lc[(size_t)k * n + k];
        __syncthreads();
        if (tid == 0) x[k] = xk;
        for (int i = tid; i < k; i += nt) w[i] -= Lc[(size_t)k * n + i] * xk;
        __syncthreads();
    }
}

// One step of the SI's adopted scheme (or a variant) by one CTA:
//   R' = R + Dt S^{-1} [f - (S_prev - S)(R_prev - R) / (2 Db)] + sqrt(2 T Db) z,  <z z^T> = S^{-1}
// with Dt = (1 - e^{-alpha D})/alpha, Db = (1 - e^{-2 alpha D})/(2 alpha) for
// the adopted scheme with alpha > 0 and Dt = Db = D otherwise; kLvNorogna drops
// the S_prev term; identity != 0 takes S = I (no Cholesky, no S_prev term).
// R_prev - R is the previous step's displacement: in the periodic box (box > 0)
// its minimum image, each component reduced by the nearest multiple of box (a
// position wrapped into the box between the steps would otherwise enter with a
// jump of one box side).
// xi ~ N(0, I) from Philox (counter = (component, md, 0, kLangevin)).
//
// Aliasing: R, Rprev, f, S and Sprev are read, R' is returned in the shared
// array r1 and nothing is written to global memory except Lc.  Every read of
// R and Rprev happens before the barrier that precedes the return, so the
// caller may write R' over R (or over Rprev) afterwards.  Shared memory v
// holds 5 n doubles.  Returns false on every thread if S is not positive
// definite (nothing else is computed then).
__device__ inline bool cta_langevin_step(int n, const double* R, const double* Rprev, const double* f,
                                         const double* S, const double* Sprev, double* Lc, double T, double delta,
                                         double alpha, Key key, uint32_t md, double box, int identity, int scheme,
                                         double* v, double* red, double** r1_out) {
    double* g = v;          // [n]
    double* x = g + n;      // [n]
    double* z = x + n;      // [n]
    double* r0 = z + n;     // [n] R
    double* r1 = r0 + n;    // [n] R'
    const int tid = threadIdx.x, nt = blockDim.x;
    double Dt = delta, Db = delta;
    if (!identity && scheme == kLvAdopted && alpha > 0.0) {
        Dt = (1.0 - exp(-alpha * delta)) / alpha;
        Db = (1.0 - exp(-2.0 * alpha * delta)) / (2.0 * alpha);
    }
    if (!identity && !cta_cholesky(n, S, Lc, red)) return false;
    const bool two_time = !identity && scheme != kLvNorogna;
    if (two_time) {   // R_prev - R (minimum image), kept in r1 until R' is formed
        for (int j = tid; j < n; j += nt) {
            double dj = Rprev[j] - R[j];
            if (box > 0.0) dj -= box * rint(dj / box);
            r1[j] = dj;
        }
        __syncthreads();
    }
    // g = f - (S_prev - S)(R_prev - R) / (2 Db);  xi;  keep R
    for (int i = tid; i < n; i += nt) {
        double t = f[i];
        if (two_time) {
            double s = 0.0;
            for (int j = 0; j < n; ++j) s += (Sprev[(size_t)i * n + j] - S[(size_t)i * n + j]) * r1[j];
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
        r1[i] = r;
    }
    __syncthreads();
    *r1_out = r1;
    return true;
}

}  // namespace qmc
