// k_setup.cu -- per-configuration tables of the nuclei (once per R).
//
//  * (sin, cos)(pi R_a / L) for the periodised displacements,
//  * exp(i k.R_a) and the proton structure factor rho_p(k) = sum_a Z exp(i k.R_a),
//  * the proton-proton real-space Ewald energy and its gradient, plus the
//    constant self-interaction term -kappa/sqrt(pi) sum_q q^2 over all 2N charges.
// Everything here is FP64.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

__global__ void ptrig_kernel(int N, double L, const double* __restrict__ R, double* ptrig64, float* ptrig32,
                             float* R32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N) return;
    R32[t] = (float)R[t];
    const int a = t / 3, mu = t % 3;
    double sn, cs;
    sincospi(R[t] / L, &sn, &cs);
    ptrig64[6 * a + mu] = sn; ptrig64[6 * a + 3 + mu] = cs;
    ptrig32[6 * a + mu] = (float)sn; ptrig32[6 * a + 3 + mu] = (float)cs;
}

__global__ void eikr_kernel(int N, int nk, double L, const int4* __restrict__ kvec, const double* __restrict__ R,
                            double2* eikR, float2* eikR32) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N * nk) return;
    const int a = t / nk, k = t - a * nk;
    const int4 m = kvec[k];
    const double ph = 2.0 * (m.x * R[3 * a] + m.y * R[3 * a + 1] + m.z * R[3 * a + 2]) / L;
    double sn, cs;
    sincospi(ph, &sn, &cs);
    eikR[t] = make_double2(cs, sn);
    eikR32[t] = make_float2((float)cs, (float)sn);
}

__global__ void rhop_kernel(int N, int nk, const double2* __restrict__ eikR, double2* rho_p) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    double re = 0, im = 0;
    for (int a = 0; a < N; ++a) { re += eikR[(size_t)a * nk + k].x; im += eikR[(size_t)a * nk + k].y; }
    rho_p[k] = make_double2(re, im);
}

// One block: proton-proton real-space energy (+ self term) and gradient.
__global__ void pp_kernel(int N, double L, double kappa, const double* __restrict__ R, double* vconst, double* dvpp) {
    __shared__ double red[64];
    double e = 0.0;
    for (int a = threadIdx.x; a < N; a += blockDim.x) {
        double g[3] = {0, 0, 0};
        for (int b = 0; b < N; ++b) {
            if (b == a) continue;
            double gr[3];
            const double v = ewald_real<double>(R[3 * a] - R[3 * b], R[3 * a + 1] - R[3 * b + 1],
                                                R[3 * a + 2] - R[3 * b + 2], L, kappa, gr);
            e += 0.5 * v;
            g[0] += gr[0]; g[1] += gr[1]; g[2] += gr[2];
        }
        dvpp[3 * a] = g[0]; dvpp[3 * a + 1] = g[1]; dvpp[3 * a + 2] = g[2];
    }
    const double tot = block_sum(e, red);
    if (threadIdx.x == 0) vconst[0] = tot - kappa / sqrt(kPi) * (2.0 * N);
}

// Reciprocal weights (4 pi / L^3) exp(-k^2 / 4 kappa^2) / k^2 of the half-space vectors.
__global__ void kw_kernel(int nk, double L, double kappa, const int4* __restrict__ kvec, double* kw, float* kw32) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nk) return;
    const int4 m = kvec[k];
    const double tp = 2.0 * kPi / L;
    const double k2 = tp * tp * (double)(m.x * m.x + m.y * m.y + m.z * m.z);
    kw[k] = 4.0 * kPi / (L * L * L) * exp(-k2 / (4.0 * kappa * kappa)) / k2;
    kw32[k] = (float)kw[k];
}

// Reciprocal-space force on the nuclei as a matrix acting on the electron
// structure factor of a sample: with rho(k) = rho_p(k) - rho_e(k) = (rr, ri),
//   F_{a,mu} = sum_k 2 Z w_k (2 pi m_mu / L) [ri cos(k.R_a) - rr sin(k.R_a)],
// T is [3N][2 nk] column-major (column 2k multiplies rr(k), 2k + 1 ri(k)).
__global__ void recforce_table_kernel(int N, int nk, double L, const int4* __restrict__ kvec,
                                      const double* __restrict__ kw, const double2* __restrict__ eikR, float* T) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * N * nk) return;
    const int k = t / (3 * N), c = t - k * 3 * N, a = c / 3, mu = c - 3 * a;
    const int4 m = kvec[k];
    const double mm = mu == 0 ? m.x : (mu == 1 ? m.y : m.z);
    const double f = 2.0 * kw[k] * (2.0 * kPi / L) * mm;   // proton charge 1
    const double2 e = eikR[(size_t)a * nk + k];
    T[(size_t)(2 * k) * 3 * N + c] = (float)(-f * e.y);
    T[(size_t)(2 * k + 1) * 3 * N + c] = (float)(f * e.x);
}

void launch_recforce_table(int N, int nk, double L, const int4* kvec, const double* kw, const double2* eikR, float* T,
                           cudaStream_t st) {
    recforce_table_kernel<<<(3 * N * nk + 255) / 256, 256, 0, st>>>(N, nk, L, kvec, kw, eikR, T);
}

void launch_setup(int N, double L, double kappa, int nk, const int4* kvec, const double* R, double* kw,
                  double* ptrig64, float* ptrig32, double2* eikR, double2* rho_p, double* vconst, double* dvpp,
                  float* R32, float2* eikR32, float* kw32, cudaStream_t st) {
    kw_kernel<<<(nk + 127) / 128, 128, 0, st>>>(nk, L, kappa, kvec, kw, kw32);
    ptrig_kernel<<<(3 * N + 127) / 128, 128, 0, st>>>(N, L, R, ptrig64, ptrig32, R32);
    eikr_kernel<<<(N * nk + 255) / 256, 256, 0, st>>>(N, nk, L, kvec, R, eikR, eikR32);
    rhop_kernel<<<(nk + 127) / 128, 128, 0, st>>>(N, nk, eikR, rho_p);
    pp_kernel<<<1, 256, 0, st>>>(N, L, kappa, R, vconst, dvpp);
}

}  // namespace qmc
