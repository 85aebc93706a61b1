// k_empirical.cu -- empirical acceleration matrix S = H + mu I (main text,
// conclusions: S from the Hessian H of an accurate and cheap empirical
// potential, with mu > 0 where H is not positive definite).  H is the Hessian
// of the screened-Coulomb (Yukawa) pair potential of the protons,
//   V = sum_{a<b} sum_{n : |d_ab + nL| < L} v(|d_ab + nL|),  v(r) = exp(-r / lambda) / r,
// images within one box side: the minimum image has |d_mu| <= L/2, so only its
// 27 neighbours n in {-1, 0, 1}^3 can lie within L.  Per image vector x, r = |x|:
//   h(x) = v''(r) x x^T / r^2 + v'(r) / r (I - x x^T / r^2),
//   v' = -e (1/r^2 + 1/(lambda r)),  v'' = e (2/r^3 + 2/(lambda r^2) + 1/(lambda^2 r)),  e = exp(-r / lambda);
// block (a, b != a) of H is -sum_images h(x_ab), the diagonal block
// sum_{b != a} sum_images h(x_ab).  One thread per 3 x 3 block, FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

__device__ inline void yukawa_pair_hessian(const double* __restrict__ Ra, const double* __restrict__ Rb, double L,
                                           double lambda, double h[9]) {
    double d[3];
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        d[mu] = Ra[mu] - Rb[mu];
        d[mu] -= L * rint(d[mu] / L);
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) h[k] = 0.0;
    const double il = 1.0 / lambda;
    for (int c = 0; c < 27; ++c) {
        const double x[3] = {d[0] + L * (c % 3 - 1), d[1] + L * ((c / 3) % 3 - 1), d[2] + L * (c / 9 - 1)};
        const double r2 = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
        if (!(r2 < L * L) || !(r2 > 0.0)) continue;
        const double r = sqrt(r2), ir = 1.0 / r;
        const double e = exp(-r * il);
        const double v1 = -e * (ir * ir + il * ir);
        const double v2 = e * (2.0 * ir * ir * ir + 2.0 * il * ir * ir + il * il * ir);
        const double radial = (v2 - v1 * ir) / r2, trans = v1 * ir;
#pragma unroll
        for (int mu = 0; mu < 3; ++mu)
#pragma unroll
            for (int nu = 0; nu < 3; ++nu) h[3 * mu + nu] += radial * x[mu] * x[nu] + (mu == nu ? trans : 0.0);
    }
}

__global__ void empirical_s_kernel(int N, double L, const double* __restrict__ R, double lambda, double mu,
                                   double* __restrict__ S) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * N) return;
    const int a = t / N, b = t - a * N, n3 = 3 * N;
    double h[9];
    if (a != b) {
        yukawa_pair_hessian(R + 3 * a, R + 3 * b, L, lambda, h);
#pragma unroll
        for (int k = 0; k < 9; ++k) S[(size_t)(3 * a + k / 3) * n3 + 3 * b + k % 3] = -h[k];
        return;
    }
    double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int c = 0; c < N; ++c) {
        if (c == a) continue;
        yukawa_pair_hessian(R + 3 * a, R + 3 * c, L, lambda, h);
#pragma unroll
        for (int k = 0; k < 9; ++k) acc[k] += h[k];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) S[(size_t)(3 * a + k / 3) * n3 + 3 * a + k % 3] = acc[k] + (k % 4 == 0 ? mu : 0.0);
}

void launch_empirical_s(int N, double L, const double* R, double lambda, double mu, double* S, cudaStream_t st) {
    empirical_s_kernel<<<(N * N + 127) / 128, 128, 0, st>>>(N, L, R, lambda, mu, S);
}

}  // namespace qmc
