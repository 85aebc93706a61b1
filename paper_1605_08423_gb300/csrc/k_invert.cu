// k_invert.cu -- full FP64 inverse of every walker's two Slater blocks.
//
// A_s[i][j] = phi_j(r_i) for the n electrons of spin s.  In-place Gauss-Jordan
// with partial (row) pivoting (Golub & Van Loan sec. 3.4); row interchanges
// turn into column interchanges of the inverse, undone at the end.  Always
// FP64: this is the periodic recompute that resets the drift of the rank-1
// (Sherman-Morrison) updates of the sweep kernel.  Output: Gt[i][j] = (A^-1)_{j,i}
// in the working precision, ln|det A| and the pivot sign.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

template <typename T>
__global__ void __launch_bounds__(256) invert_kernel(int N, int n, const T* __restrict__ Phi, T* __restrict__ Gt,
                                                     double* __restrict__ logdet, int* err) {
    extern __shared__ double sm[];
    const int ld = n + 1;
    double* M = sm;                      // [n][n+1]
    double* col = M + (size_t)n * ld;    // [n]
    int* perm = (int*)(col + n);         // [n]
    __shared__ int piv_row;
    __shared__ int singular;
    __shared__ double ipv_s;
    __shared__ int sgn;
    const int w = blockIdx.x >> 1, sp = blockIdx.x & 1;
    const int tid = threadIdx.x, nt = blockDim.x;
    const T* A = Phi + ((size_t)w * N + (size_t)sp * n) * n;
    for (int idx = tid; idx < n * n; idx += nt) M[(idx / n) * ld + idx % n] = (double)A[idx];
    if (tid == 0) { sgn = 1; singular = 0; }
    // ln|det| as mantissa product and exponent sum (one log at the end): the
    // FP64 pipe is the bound here, so no per-step log or per-thread division
    double mant = 1.0;
    int expo = 0;
    // rank-1 update: thread owns column jj of rows i0, i0 + istep, ... (no index division per element)
    const bool tiled = nt % n == 0;
    const int jj = tid % n, i0 = tid / n, istep = nt / n;
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {                      // argmax |M[i][k]|, i >= k (ties -> lowest row)
            // magnitudes compared as the bit patterns of |x| (monotonic for
            // finite doubles): integer work instead of FP64 compares
            unsigned long long best = 0ull; int bi = n;
            for (int i = k + tid; i < n; i += 32) {
                const unsigned long long v = (unsigned long long)__double_as_longlong(M[i * ld + k]) & 0x7FFFFFFFFFFFFFFFull;
                if (bi == n || v > best) { best = v; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (oi < n && (bi == n || ob > best || (ob == best && oi < bi))) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                piv_row = bi;
                perm[k] = bi;
                if (best == 0ull) singular = 1;
            }
        }
        __syncthreads();
        if (singular) break;
        const int p = piv_row;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                const double t = M[k * ld + j];
                M[k * ld + j] = M[p * ld + j];
                M[p * ld + j] = t;
            }
            __syncthreads();
        }
        if (tid == 0) {
            const double pv = M[k * ld + k];
            int e1, e2;
            const double m1 = frexp(fabs(pv), &e1);
            mant = frexp(mant * m1, &e2);
            expo += e1 + e2;
            sgn *= (p != k ? -1 : 1) * (pv < 0 ? -1 : 1);
            ipv_s = 1.0 / pv;
        }
        for (int i = tid; i < n; i += nt) col[i] = (i == k) ? 0.0 : M[i * ld + k];
        __syncthreads();
        const double ipv = ipv_s;
        for (int j = tid; j < n; j += nt) M[k * ld + j] = (j == k ? 1.0 : M[k * ld + j]) * ipv;
        __syncthreads();
        if (tiled) {
            const double mkj = M[k * ld + jj];
            for (int i = i0; i < n; i += istep) {
                if (i == k) continue;
                const double base = (jj == k) ? 0.0 : M[i * ld + jj];
                M[i * ld + jj] = base - col[i] * mkj;
            }
        } else {
            for (int idx = tid; idx < n * n; idx += nt) {
                const int i = idx / n, j = idx - i * n;
                if (i == k) continue;
                const double base = (j == k) ? 0.0 : M[i * ld + j];
                M[i * ld + j] = base - col[i] * M[k * ld + j];
            }
        }
        __syncthreads();
    }
    if (singular) {
        if (tid == 0) {
            raise_err(err, kErrSingular);
            logdet[2 * w + sp] = -INFINITY;
        }
        return;
    }
    for (int k = n - 1; k >= 0; --k) {       // undo the interchanges on the columns
        const int p = perm[k];
        if (p != k)
            for (int i = tid; i < n; i += nt) {
                const double t = M[i * ld + k];
                M[i * ld + k] = M[i * ld + p];
                M[i * ld + p] = t;
            }
        __syncthreads();
    }
    T* out = Gt + ((size_t)w * 2 + sp) * n * n;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int i = idx / n, j = idx - i * n;       // Gt[i][j] = inv[j][i]
        out[idx] = (T)M[j * ld + i];
    }
    if (tid == 0) logdet[2 * w + sp] = log(mant) + expo * 0.69314718055994530942;
}

template <typename T>
void launch_invert(int W, int N, int n, const T* Phi, T* Gt, double* logdet, int* err, cudaStream_t st) {
    const size_t smem = (size_t)n * (n + 1) * sizeof(double) + n * sizeof(double) + n * sizeof(int);
    const int threads = n >= 32 ? 256 : 64;
    invert_kernel<T><<<2 * W, threads, smem, st>>>(N, n, Phi, Gt, logdet, err);
}

template void launch_invert<double>(int, int, int, const double*, double*, double*, int*, cudaStream_t);
template void launch_invert<float>(int, int, int, const float*, float*, double*, int*, cudaStream_t);

}  // namespace qmc
