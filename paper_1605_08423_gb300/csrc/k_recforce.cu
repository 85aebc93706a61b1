// k_recforce.cu -- reciprocal-space Ewald force on the nuclei for every walker
// sample of the mixed form, as one FP32 matrix product over walkers.
//
// The Ewald k-sum's force on nucleus a is linear in the sample's structure
// factor rho(k) = rho_p(k) - rho_e(k) = (rr, ri):
//   F_{a,mu} = sum_k 2 Z w_k (2 pi m_mu / L) [ri cos(k.R_a) - rr sin(k.R_a)]
// so with the per-R table T ([3N][2 nk], built in k_setup.cu) the forces of all
// walkers are F[w][c] = sum_q rho[w][q] T[q][c]  (q = 2k or 2k + 1), an
// M = walkers, N = 3N, K = 2 nk product: 2 * 16384 * 384 * 924 = 11.6 GFLOP
// per sample at N = 128 -- dense and regular, plain FP32 FMAs in the order of
// q (FP32-level, like every other FP32 pair term of the mixed form).
//
// Tiling: a CTA owns 128 walkers x 128 columns, K in steps of 16 staged in
// shared memory (double-buffered: the next step's tile is loaded into
// registers while the current one is multiplied); 256 threads, 8 x 8 outputs
// each, read as two 4-wide groups 64 apart in both directions so that the
// shared-memory reads of a warp are conflict-free.  Ragged walkers, columns and
// K are zero-filled on load and masked on store.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

namespace {
constexpr int kBW = 128, kBC = 128, kBK = 16, kThr = 256;
constexpr int kPadW = kBW + 4, kPadC = kBC + 4;
}  // namespace

__global__ void __launch_bounds__(kThr, 1)
    recforce_gemm_kernel(int W, int M, int K, const float* __restrict__ rho, const float* __restrict__ T,
                         float* __restrict__ F) {
    __shared__ __align__(16) float As[2][kBK][kPadW];   // rho tile, transposed: As[q][w]
    __shared__ __align__(16) float Bs[2][kBK][kPadC];   // T tile: Bs[q][c]
    const int tid = threadIdx.x;
    const int w0 = blockIdx.x * kBW, c0 = blockIdx.y * kBC;
    const int tw = tid >> 4, tc = tid & 15;             // 16 x 16 threads
    // load mapping: rho element (w0 + lw, q0 + lq), lw = idx / 16, lq = idx % 16
    //               T element   (q0 + tq, c0 + tcc), tq = idx / 128, tcc = idx % 128
    float ra[8], rb[8];
    auto load = [&](int q0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = tid + kThr * i;
            const int lw = idx >> 4, lq = idx & 15;
            const int w = w0 + lw, q = q0 + lq;
            ra[i] = (w < W && q < K) ? rho[(size_t)w * K + q] : 0.f;
            const int tq = idx >> 7, tcc = idx & 127;
            const int qq = q0 + tq, c = c0 + tcc;
            rb[i] = (qq < K && c < M) ? T[(size_t)qq * M + c] : 0.f;
        }
    };
    auto store = [&](int b) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int idx = tid + kThr * i;
            As[b][idx & 15][idx >> 4] = ra[i];
            Bs[b][idx >> 7][idx & 127] = rb[i];
        }
    };
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = 0.f;
    const int nsteps = (K + kBK - 1) / kBK;
    load(0);
    store(0);
    __syncthreads();
    for (int s = 0; s < nsteps; ++s) {
        const int b = s & 1;
        if (s + 1 < nsteps) load((s + 1) * kBK);
#pragma unroll
        for (int q = 0; q < kBK; ++q) {
            float av[8], bv[8];
            load4(&As[b][q][4 * tw], av);
            load4(&As[b][q][64 + 4 * tw], av + 4);
            load4(&Bs[b][q][4 * tc], bv);
            load4(&Bs[b][q][64 + 4 * tc], bv + 4);
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int c = 0; c < 8; ++c) acc[a][c] = fmaf(av[a], bv[c], acc[a][c]);
        }
        if (s + 1 < nsteps) store(b ^ 1);
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 8; ++a) {
        const int w = w0 + (a < 4 ? 4 * tw + a : 64 + 4 * tw + a - 4);
        if (w >= W) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int col = c0 + (c < 4 ? 4 * tc + c : 64 + 4 * tc + c - 4);
            if (col < M) F[(size_t)w * M + col] = acc[a][c];
        }
    }
}

void launch_recforce_gemm(int W, int M, int K, const float* rho, const float* T, float* F, cudaStream_t st) {
    const dim3 grid((W + kBW - 1) / kBW, (M + kBC - 1) / kBC);
    recforce_gemm_kernel<<<grid, kThr, 0, st>>>(W, M, K, rho, T, F);
}

}  // namespace qmc
