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

// Gauss-Jordan inverse of walker w's spin block sp by the whole CTA, in the
// FP64 work space sm (n (n + 1) + n doubles and n ints).
template <typename T>
__device__ void gj_invert(int N, int n, const T* __restrict__ Phi, T* __restrict__ Gt, double* __restrict__ logdet,
                          int* err, int w, int sp, double* sm) {
    const int ld = n + 1;
    double* M = sm;                      // [n][n+1]
    double* col = M + (size_t)n * ld;    // [n]
    int* perm = (int*)(col + n);         // [n]
    __shared__ int piv_row;
    __shared__ int singular;
    __shared__ double ipv_s;
    __shared__ int sgn;
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
__global__ void __launch_bounds__(256) invert_kernel(int N, int n, const T* __restrict__ Phi, T* __restrict__ Gt,
                                                     double* __restrict__ logdet, int* err) {
    extern __shared__ double sm[];
    gj_invert<T>(N, n, Phi, Gt, logdet, err, blockIdx.x >> 1, blockIdx.x & 1, sm);
}

// Mixed form, periodic recompute inside a call: one Newton-Schulz step
//   R = I - A G,  G <- G + G R
// on the inverse the Sherman-Morrison updates have carried since the last
// recompute; A = the Slater block just evaluated at the current positions.
// With E = G - A^-1 the step leaves G' - A^-1 = -E A E, second order in the
// drift.  The residual is formed without rounding error of consequence: each
// product a*g is split exactly into its FP32 value and error (one FMA) and the
// sum is carried as an unevaluated pair hi + lo with Knuth's TwoSum (the
// compensated dot product of Ogita, Rump and Oishi, SIAM J. Sci. Comput. 26,
// 2005), so R is the residual of the FP32 A and G to FP32 relative accuracy
// although A G agrees with I to a few units of FP32 rounding.  G R is small
// and formed in plain FP32.  The result is the inverse of the FP32 Slater
// block to FP32 rounding (what FP64 Gauss-Jordan rounded to FP32 gives) from
// about ten FP32 operations per term of one n^3 product plus one plain n^3
// product; FP64 runs at 1/64 of the FP32 rate on this part.  If max |R_ij| >=
// 0.01 (or is not finite) the block is inverted from scratch by Gauss-Jordan in
// FP64 instead.  ln|det| is not updated here (nothing in a call reads it
// after the first recompute, which is always Gauss-Jordan).
__global__ void __launch_bounds__(256) refine_kernel(int N, int n, int np, const float* __restrict__ Phi,
                                                     float* __restrict__ Gt, double* __restrict__ logdet, int* err) {
    extern __shared__ double sm[];
    const int ld = np + 4, ng = np / 4;
    float* AT = (float*)sm;                  // A^T [j][i]; later G'^T
    float* Gm = AT + (size_t)np * ld;        // G [j][k] = Gt[k][j]
    float* R = Gm + (size_t)np * ld;         // R [i][k]
    __shared__ float rmax_s[8];
    const int w = blockIdx.x >> 1, sp = blockIdx.x & 1;
    const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
    const float* A = Phi + ((size_t)w * N + (size_t)sp * n) * n;
    float* Go = Gt + ((size_t)w * 2 + sp) * n * n;
    for (int idx = tid; idx < np * np; idx += nt) {
        const int i = idx / np, j = idx - i * np;
        const bool in = i < n && j < n;
        AT[j * ld + i] = in ? A[i * n + j] : 0.f;
        Gm[j * ld + i] = in ? Go[i * n + j] : 0.f;
    }
    __syncthreads();
    const int r0 = 4 * (tid / ng), c0 = 4 * (tid % ng);
    const bool act = tid < ng * ng;
    float acc[4][4] = {};
    float rm = 0.f;
    if (act) {                               // (A G)[i][k] = sum_j A[i][j] G[j][k] as hi + lo
        float lo[4][4] = {};
        for (int j = 0; j < np; ++j) {
            const float4 a4 = *(const float4*)(AT + j * ld + r0), g4 = *(const float4*)(Gm + j * ld + c0);
            const float av[4] = {a4.x, a4.y, a4.z, a4.w}, gv[4] = {g4.x, g4.y, g4.z, g4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    // explicit-rounding intrinsics: no contraction into FMAs,
                    // which would void the error-free transformations
                    const float p = __fmul_rn(av[a], gv[b]);
                    const float e = __fmaf_rn(av[a], gv[b], -p);     // a g - p exactly
                    const float s = acc[a][b], t = __fadd_rn(s, p);
                    const float z = __fsub_rn(t, s);
                    const float d = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));   // s + p - t exactly
                    lo[a][b] = __fadd_rn(lo[a][b], __fadd_rn(d, e));
                    acc[a][b] = t;
                }
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = r0 + a, k = c0 + b;
                // (delta - hi) is exact (hi is within a few units of rounding
                // of delta); one rounding when lo is taken off
                const float r = (i < n && k < n) ? __fsub_rn(__fsub_rn(i == k ? 1.f : 0.f, acc[a][b]), lo[a][b]) : 0.f;
                R[i * ld + k] = r;
                rm = fmaxf(rm, isfinite(r) ? fabsf(r) : 1e30f);
            }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rm = fmaxf(rm, __shfl_xor_sync(0xffffffffu, rm, o));
    if (lane == 0) rmax_s[warp] = rm;
    __syncthreads();
    float rmax = 0.f;
    for (int q = 0; q < nt / 32; ++q) rmax = fmaxf(rmax, rmax_s[q]);
    if (!(rmax < 0.01f)) {                   // too far off: FP64 Gauss-Jordan from scratch
        __syncthreads();
        gj_invert<float>(N, n, Phi, Gt, logdet, err, w, sp, sm);
        return;
    }
    if (act) {                               // G'[j][k] = G[j][k] + sum_i G[j][i] R[i][k]
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = Gm[(r0 + a) * ld + c0 + b];
        for (int i = 0; i < np; ++i) {
            const float4 r4 = *(const float4*)(R + i * ld + c0);
            const float rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                const float gji = Gm[(r0 + a) * ld + i];
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] += gji * rv[b];
            }
        }
    }
    __syncthreads();                         // every read of A^T done: it takes G'^T
    if (act)
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) AT[(c0 + b) * ld + r0 + a] = acc[a][b];
    __syncthreads();
    for (int idx = tid; idx < n * n; idx += nt) {
        const int k = idx / n, j = idx - k * n;     // Gt[k][j] = G'[j][k]
        Go[idx] = AT[k * ld + j];
    }
}

void launch_refine(int W, int N, int n, const float* Phi, float* Gt, double* logdet, int* err, cudaStream_t st) {
    int np = 4;
    while (np < n) np *= 2;
    const size_t gj = (size_t)n * (n + 1) * sizeof(double) + n * sizeof(double) + n * sizeof(int);
    const size_t ns = (size_t)3 * np * (np + 4) * sizeof(float);
    const size_t smem = gj > ns ? gj : ns;
    // raise the dynamic shared-memory limit to what this launch needs (the
    // kernel also holds static shared memory, so not to the opt-in maximum)
    static size_t attr = 0;
    if (smem > attr &&
        cudaFuncSetAttribute(refine_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
        attr = smem;
    refine_kernel<<<2 * W, 256, smem, st>>>(N, n, np, Phi, Gt, logdet, err);
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
