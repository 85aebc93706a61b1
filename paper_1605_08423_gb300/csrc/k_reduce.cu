// k_reduce.cu -- walker reductions: E, its error bar, the mean force and the
// covariance matrix S of the paper's covariance definition,
//   f   = -<dE_L/dR> - 2(<E_L dlnpsi/dR> - E <dlnpsi/dR>)
//   f_w = same with the means of walker w (global E)
//   S   = sum_w (f_w - f)(f_w - f)^T / (W (W-1))     (covariance of the mean)
//   E_err^2 = sum_w (E_w - E)^2 / (W (W-1)),  N_c = number of samples.
// FP64, fixed-order trees (bitwise reproducible; no atomics).
// Output layout: [E, E_err, N_c, accept, f(3N), S(3N x 3N)].
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

// colsum[c] = sum_w acc[w][c] for c < ncol; colsum[ncol] = sum_w nacc[w].
__global__ void colsum_kernel(int W, int ncol, const double* __restrict__ acc, const unsigned long long* __restrict__ nacc,
                              double* colsum) {
    __shared__ double red[32];
    const int c = blockIdx.x;
    double s = 0.0;
    if (c < ncol)
        for (int w = threadIdx.x; w < W; w += blockDim.x) s += acc[(size_t)w * ncol + c];
    else
        for (int w = threadIdx.x; w < W; w += blockDim.x) s += (double)nacc[w];
    s = block_sum(s, red);
    if (threadIdx.x == 0) colsum[c] = s;
}

__global__ void finalize_kernel(int W, int N, double moves, const double* __restrict__ colsum, double* out, int* err) {
    const int N3 = 3 * N, ncol = 3 + 9 * N;
    const double cnt = colsum[0];
    const double E = colsum[1] / cnt;
    for (int c = threadIdx.x; c < N3; c += blockDim.x) {
        const double f = -colsum[3 + 2 * N3 + c] / cnt - 2.0 * (colsum[3 + N3 + c] / cnt - E * colsum[3 + c] / cnt);
        out[4 + c] = f;
        if (!isfinite(f)) raise_err(err, kErrNonfinite);
    }
    if (threadIdx.x == 0) {
        out[0] = E;
        out[2] = cnt;
        out[3] = colsum[ncol] / moves;
        if (!isfinite(E)) raise_err(err, kErrNonfinite);
    }
}

// dev[w][c] = f_w[c] - f[c] (c < 3N), dev[w][3N] = E_w - E.
__global__ void deviation_kernel(int W, int N, const double* __restrict__ acc, const double* __restrict__ out,
                                 double* dev) {
    const int N3 = 3 * N, ncol = 3 + 9 * N;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (size_t)W * (N3 + 1)) return;
    const int w = (int)(t / (N3 + 1)), c = (int)(t - (size_t)w * (N3 + 1));
    const double* a = acc + (size_t)w * ncol;
    const double cnt = a[0], E = out[0];
    if (c < N3) {
        const double fw = -a[3 + 2 * N3 + c] / cnt - 2.0 * (a[3 + N3 + c] / cnt - E * a[3 + c] / cnt);
        dev[t] = fw - out[4 + c];
    } else {
        dev[t] = a[1] / cnt - E;
    }
}

__global__ void eerr_kernel(int W, int N, const double* __restrict__ dev, double* out) {
    __shared__ double red[32];
    const int N3 = 3 * N;
    double s = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double d = dev[(size_t)w * (N3 + 1) + N3];
        s += d * d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) out[1] = W > 1 ? sqrt(s / ((double)W * (W - 1))) : 0.0;
}

// S tile (32 x 32) per block; 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256) gram_kernel(int W, int N, const double* __restrict__ dev, double* out) {
    __shared__ double A[32][33], Bm[32][33];
    const int N3 = 3 * N, ld = N3 + 1;
    const int i0 = blockIdx.y * 32, j0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    double acc[4] = {0, 0, 0, 0};
    for (int w0 = 0; w0 < W; w0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int w = w0 + r;
            A[r][tx] = (w < W && i0 + tx < N3) ? dev[(size_t)w * ld + i0 + tx] : 0.0;
            Bm[r][tx] = (w < W && j0 + tx < N3) ? dev[(size_t)w * ld + j0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 8
        for (int r = 0; r < 32; ++r) {
            const double b = Bm[r][tx];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] += A[r][ty + 8 * q] * b;
        }
        __syncthreads();
    }
    const double scale = W > 1 ? 1.0 / ((double)W * (W - 1)) : 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < N3 && j < N3) out[4 + N3 + (size_t)i * N3 + j] = acc[q] * scale;
    }
}

void launch_reduce(int W, int N, double moves, const double* acc, const unsigned long long* nacc, double* colsum,
                        double* dev, double* out, int* err, cudaStream_t st) {
    const int ncol = 3 + 9 * N, N3 = 3 * N;
    colsum_kernel<<<ncol + 1, 256, 0, st>>>(W, ncol, acc, nacc, colsum);
    finalize_kernel<<<1, 256, 0, st>>>(W, N, moves, colsum, out, err);
    const size_t tot = (size_t)W * (N3 + 1);
    deviation_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, N, acc, out, dev);
    eerr_kernel<<<1, 256, 0, st>>>(W, N, dev, out);
    dim3 g((N3 + 31) / 32, (N3 + 31) / 32);
    gram_kernel<<<g, 256, 0, st>>>(W, N, dev, out);
}

}  // namespace qmc
