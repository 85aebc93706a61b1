// k_reduce.cu -- walker reductions: E, its error bar, the mean force and the
// covariance matrix S of the paper's covariance definition,
//   f   = -<dE_L/dR> - 2(<E_L dlnpsi/dR> - E <dlnpsi/dR>)
//   f_w = same with the means of walker w (global E)
//   S   = sum_w (f_w - f)(f_w - f)^T / (W (W-1))     (covariance of the mean)
//   E_err^2 = sum_w (E_w - E)^2 / (W (W-1)),  N_c = number of samples.
// FP64, fixed-order trees (bitwise reproducible; no atomics).
// Output layout: [E, E_err, N_c, accept, f(3N), S(3N x 3N)].
//
// Walker-sharded form (walkers split over processes, one GPU each): the same
// reduction in three steps around two sums over the processes --
//   local column sums (plus walkers and moves)          -> summed over processes
//   E, f from the global sums; local sums of (E_w - E)^2 and of
//   (f_w - f)(f_w - f)^T with the global E, f          -> summed over processes
//   E_err and S from the global sums and walker count.
// The result equals the single-process reduction over all walkers up to the
// order of the FP64 sums.
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

// E, f, N_c and the acceptance ratio from column sums (moves < 0: read the
// number of moves from colsum[ncol + 2], as the sharded form stores it).
__global__ void finalize_kernel(int N, double moves, const double* __restrict__ colsum, double* out, int* err) {
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
        out[3] = colsum[ncol] / (moves < 0.0 ? colsum[ncol + 2] : moves);
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

// sum_w (E_w - E)^2: written as sqrt(sum / (W (W - 1))) when finish != 0, else as the plain sum.
__global__ void eerr_kernel(int W, int N, const double* __restrict__ dev, double* dst, int finish) {
    __shared__ double red[32];
    const int N3 = 3 * N;
    double s = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double d = dev[(size_t)w * (N3 + 1) + N3];
        s += d * d;
    }
    s = block_sum(s, red);
    if (threadIdx.x == 0) dst[0] = finish ? (W > 1 ? sqrt(s / ((double)W * (W - 1))) : 0.0) : s;
}

// dst[i][j] = scale * sum_w dev[w][i] dev[w][j]: a 32 x 32 tile per block,
// 256 threads, 4 outputs each.
__global__ void __launch_bounds__(256) gram_kernel(int W, int N, const double* __restrict__ dev, double* dst,
                                                   double scale) {
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
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + ty + 8 * q, j = j0 + tx;
        if (i < N3 && j < N3) dst[(size_t)i * N3 + j] = acc[q] * scale;
    }
}

void launch_reduce(int W, int N, double moves, const double* acc, const unsigned long long* nacc, double* colsum,
                        double* dev, double* out, int* err, cudaStream_t st) {
    const int ncol = 3 + 9 * N, N3 = 3 * N;
    colsum_kernel<<<ncol + 1, 256, 0, st>>>(W, ncol, acc, nacc, colsum);
    finalize_kernel<<<1, 256, 0, st>>>(N, moves, colsum, out, err);
    const size_t tot = (size_t)W * (N3 + 1);
    deviation_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, N, acc, out, dev);
    eerr_kernel<<<1, 256, 0, st>>>(W, N, dev, out + 1, 1);
    dim3 g((N3 + 31) / 32, (N3 + 31) / 32);
    gram_kernel<<<g, 256, 0, st>>>(W, N, dev, out + 4 + N3, W > 1 ? 1.0 / ((double)W * (W - 1)) : 0.0);
}

// ---------------------------------------------------------------------------
// Walker-sharded form.
// ---------------------------------------------------------------------------
__global__ void shard_counts_kernel(int N, double walkers, double moves, double* sums) {
    const int ncol = 3 + 9 * N;
    sums[ncol + 1] = walkers;
    sums[ncol + 2] = moves;
}

// E_err and S from the summed partial sums: scale by 1 / (W (W - 1)), W the
// summed walker count.
__global__ void shard_finish_kernel(int N, const double* __restrict__ sums, const double* __restrict__ gram,
                                    double* out) {
    const int N3 = 3 * N, ncol = 3 + 9 * N;
    const double W = sums[ncol + 1];
    const double scale = W > 1.0 ? 1.0 / (W * (W - 1.0)) : 0.0;
    const size_t tot = (size_t)N3 * N3;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot; i += (size_t)gridDim.x * blockDim.x)
        out[4 + N3 + i] = gram[1 + i] * scale;
    if (blockIdx.x == 0 && threadIdx.x == 0) out[1] = sqrt(gram[0] * scale);
}

// Virial pressure of the last call's samples (the potential is homogeneous of
// degree -1 in all lengths -- the Ewald sum with kappa L and the k cutoff in
// units of 2 pi / L fixed included -- so for the trial state scaled with the
// box, E(lambda) = T / lambda^2 + V / lambda and -dE/dOmega = (2 T + V) / (3 Omega)):
//   P_w = (2 E_w - V_w) / (3 Omega)   per walker (T = E - V),
//   P   = (2 E - V) / (3 Omega) + N T_nuc / Omega   (classical nuclei, ideal-gas term),
//   P_err^2 = sum_w (P_w - P_el)^2 / (W (W - 1)).
// out = [P, P_err, P_el, <V_L>, <T_L>] (hartree / bohr^3, hartree).
__global__ void pressure_kernel(int W, int N, const double* __restrict__ acc, const double* __restrict__ vacc,
                                double omega, double T_nuc, double* out) {
    __shared__ double red[32];
    const int ncol = 3 + 9 * N;
    double c = 0.0, e = 0.0, v = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        c += acc[(size_t)w * ncol];
        e += acc[(size_t)w * ncol + 1];
        v += vacc[w];
    }
    c = block_sum(c, red);
    e = block_sum(e, red);
    v = block_sum(v, red);
    const double E = e / c, V = v / c;
    const double Pel = (2.0 * E - V) / (3.0 * omega);
    double d2 = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) {
        const double cw = acc[(size_t)w * ncol];
        const double pw = (2.0 * acc[(size_t)w * ncol + 1] / cw - vacc[w] / cw) / (3.0 * omega);
        d2 += (pw - Pel) * (pw - Pel);
    }
    d2 = block_sum(d2, red);
    if (threadIdx.x == 0) {
        out[0] = Pel + N * T_nuc / omega;
        out[1] = W > 1 ? sqrt(d2 / ((double)W * (W - 1))) : 0.0;
        out[2] = Pel;
        out[3] = V;
        out[4] = E - V;
    }
}

void launch_pressure(int W, int N, const double* acc, const double* vacc, double omega, double T_nuc, double* out,
                     cudaStream_t st) {
    pressure_kernel<<<1, 256, 0, st>>>(W, N, acc, vacc, omega, T_nuc, out);
}

void launch_shard_sums(int W, int N, double moves, const double* acc, const unsigned long long* nacc, double* sums,
                       cudaStream_t st) {
    const int ncol = 3 + 9 * N;
    colsum_kernel<<<ncol + 1, 256, 0, st>>>(W, ncol, acc, nacc, sums);
    shard_counts_kernel<<<1, 1, 0, st>>>(N, (double)W, moves, sums);
}

void launch_shard_reduce(int W, int N, const double* acc, const double* sums, double* dev, double* out, double* gram,
                         int* err, cudaStream_t st) {
    const int N3 = 3 * N;
    finalize_kernel<<<1, 256, 0, st>>>(N, -1.0, sums, out, err);
    const size_t tot = (size_t)W * (N3 + 1);
    deviation_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(W, N, acc, out, dev);
    eerr_kernel<<<1, 256, 0, st>>>(W, N, dev, gram, 0);
    dim3 g((N3 + 31) / 32, (N3 + 31) / 32);
    gram_kernel<<<g, 256, 0, st>>>(W, N, dev, gram + 1, 1.0);
}

void launch_shard_finish(int N, const double* sums, const double* gram, double* out, cudaStream_t st) {
    shard_finish_kernel<<<64, 256, 0, st>>>(N, sums, gram, out);
}

}  // namespace qmc
