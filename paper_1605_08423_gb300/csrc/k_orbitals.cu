// k_orbitals.cu -- walker-batched molecular-orbital evaluation, Metropolis
// proposals and walker placement.
//
// Orbitals (SI, determinant basis; Gaussians periodised by the SI's
// r_mu -> (L/pi) sin(pi r_mu / L) substitution):
//   phi_j(r) = sum_b C[b][j] chi_b(r),  chi_b(r) = exp(-zeta_g t),  t = |d(r - R_a)|^2,  b = a*G + g.
// For a batch of rows (one electron position each) this is the dense
// contraction [rows x B] . [B x n]; the basis tile is produced on the fly in
// shared memory and never written to HBM.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

// Q = 1: values only (proposal rows / Slater matrix).
// Q = 5: value, d/dx, d/dy, d/dz, Laplacian (local energy).
template <typename T, int Q, int NP>
__global__ void __launch_bounds__(512) orbitals_simt(SysView<T> s, const double* __restrict__ pos, int nrows,
                                                     T* __restrict__ val, T* __restrict__ grad, T* __restrict__ lap) {
    constexpr int RT = 32, KC = 16, CG = NP / 4;
    __shared__ T rtrig[RT][6];
    __shared__ T chi[Q][KC][RT];
    __shared__ __align__(16) T csm[KC][NP];
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int row0 = blockIdx.x * RT;
    const int n = s.n, B = s.B, G = s.G;
    const T ell = (T)s.ell;

    for (int idx = tid; idx < RT * 3; idx += nthr) {
        const int r = idx / 3, mu = idx % 3, row = row0 + r;
        T sn = 0, cs = 1;
        if (row < nrows) qsincospi((T)(pos[(size_t)row * 3 + mu] / s.L), &sn, &cs);
        rtrig[r][mu] = sn;
        rtrig[r][3 + mu] = cs;
    }
    const int rg = tid / CG, cg = tid % CG;
    const int r0 = 2 * rg, c0 = 4 * cg;
    T acc[Q][2][4];
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int m = 0; m < 4; ++m) acc[q][a][m] = T(0);

    for (int k0 = 0; k0 < B; k0 += KC) {
        __syncthreads();
        for (int idx = tid; idx < KC * NP; idx += nthr) {
            const int kk = idx / NP, j = idx % NP, b = k0 + kk;
            csm[kk][j] = (b < B && j < n) ? s.C[(size_t)b * n + j] : T(0);
        }
        for (int idx = tid; idx < KC * RT; idx += nthr) {
            const int kk = idx / RT, r = idx % RT, b = k0 + kk;
            T v[Q];
#pragma unroll
            for (int q = 0; q < Q; ++q) v[q] = T(0);
            if (b < B && row0 + r < nrows) {
                const int a = b / G, g = b - a * G;
                const T* pt = s.ptrig + 6 * a;
                T sd[3], cd[3], t = 0;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    const T sx = rtrig[r][mu], cx = rtrig[r][3 + mu], sr = pt[mu], cr = pt[3 + mu];
                    sd[mu] = sx * cr - cx * sr;
                    cd[mu] = cx * cr + sx * sr;
                    t += sd[mu] * sd[mu];
                }
                t *= ell * ell;
                const T z = s.zetat[g];
                const T e = qexp(-z * t);
                v[0] = e;
                if (Q == 5) {
                    const T f1 = -z * e, f2 = z * z * e;
                    T pp = 0, sq = 0;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        const T p = ell * sd[mu] * cd[mu], qq = cd[mu] * cd[mu] - sd[mu] * sd[mu];
                        v[1 + mu] = T(2) * f1 * p;
                        pp += p * p; sq += qq;
                    }
                    v[Q - 1] = T(4) * f2 * pp + T(2) * f1 * sq;
                }
            }
#pragma unroll
            for (int q = 0; q < Q; ++q) chi[q][kk][r] = v[q];
        }
        __syncthreads();
        if (rg * 2 < RT) {
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                T c[4];
#pragma unroll
                for (int m = 0; m < 4; ++m) c[m] = csm[kk][c0 + m];
#pragma unroll
                for (int q = 0; q < Q; ++q) {
                    const T x0 = chi[q][kk][r0], x1 = chi[q][kk][r0 + 1];
#pragma unroll
                    for (int m = 0; m < 4; ++m) {
                        acc[q][0][m] += x0 * c[m];
                        acc[q][1][m] += x1 * c[m];
                    }
                }
            }
        }
    }
    if (rg * 2 >= RT) return;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const int row = row0 + r0 + a;
        if (row >= nrows) continue;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int j = c0 + m;
            if (j >= n) continue;
            val[(size_t)row * n + j] = acc[0][a][m];
            if (Q == 5) {
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) grad[((size_t)row * 3 + mu) * n + j] = acc[1 + mu][a][m];
                lap[(size_t)row * n + j] = acc[Q - 1][a][m];
            }
        }
    }
}

template <typename T, int Q>
static void launch_orb(const SysView<T>& s, const double* pos, int nrows, T* val, T* grad, T* lap, cudaStream_t st) {
    const int grid = (nrows + 31) / 32;
    if (s.n <= 16)
        orbitals_simt<T, Q, 16><<<grid, 16 * 4, 0, st>>>(s, pos, nrows, val, grad, lap);
    else if (s.n <= 32)
        orbitals_simt<T, Q, 32><<<grid, 16 * 8, 0, st>>>(s, pos, nrows, val, grad, lap);
    else
        orbitals_simt<T, Q, 64><<<grid, 16 * 16, 0, st>>>(s, pos, nrows, val, grad, lap);
}

template <typename T>
void launch_orbitals(const SysView<T>& s, const double* pos, int nrows, T* val, T* grad, T* lap, cudaStream_t st) {
    if (grad) launch_orb<T, 5>(s, pos, nrows, val, grad, lap, st);
    else launch_orb<T, 1>(s, pos, nrows, val, nullptr, nullptr, st);
}

// ---------------------------------------------------------------------------
// Proposals of one sweep: Xp = X + sigma xi (Philox normals, purposes 0..2),
// their (sin, cos)(pi x'/L) in the working precision, and the acceptance
// uniforms (purpose 3), index = sweep * N + electron.  A move of electron i
// only ever changes r_i, so every proposal of the sweep is known when the
// sweep starts.  X is wrapped into [0, L) first (the mixed sweep stores
// accepted positions unwrapped).  The Philox stream of walker w is w0 + w
// (w0: the handle's first walker in a walker-sharded run).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void propose_kernel(int W, int N, double L, double* __restrict__ X, double* __restrict__ Xp,
                               T* __restrict__ ptp, T* __restrict__ uacc, Key key, uint32_t md, uint32_t sweep,
                               double sigma, uint32_t w0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * N) return;
    const int w = t / N, i = t - w * N;
    const uint32_t idx = sweep * (uint32_t)N + (uint32_t)i;
    const double iL = 1.0 / L;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        double x = X[(size_t)t * 3 + mu];
        x -= L * floor(x * iL);
        X[(size_t)t * 3 + mu] = x;
        const T z = Draw<T>::normal(philox(w0 + (uint32_t)w, md, idx, kPropX + mu, key));
        const double xp = x + sigma * (double)z;
        Xp[(size_t)t * 3 + mu] = xp;
        T sn, cs;
        qsincospi((T)(xp * iL), &sn, &cs);
        ptp[(size_t)t * 6 + mu] = sn;
        ptp[(size_t)t * 6 + 3 + mu] = cs;
    }
    uacc[t] = Draw<T>::uniform(philox(w0 + (uint32_t)w, md, idx, kAccept, key));
}

template <typename T>
void launch_propose(int W, int N, double L, double* X, double* Xp, T* ptp, T* uacc, Key key, uint32_t md,
                    uint32_t sweep, double sigma, uint32_t w0, cudaStream_t st) {
    const int tot = W * N;
    propose_kernel<T><<<(tot + 255) / 256, 256, 0, st>>>(W, N, L, X, Xp, ptp, uacc, key, md, sweep, sigma, w0);
}

// Walker start: electron i next to proton i (up electrons on protons 0..N/2-1,
// down electrons on N/2..N-1) plus 0.5 bohr Gaussian noise, wrapped; the
// Philox stream of walker w is w0 + w.
__global__ void init_walkers_kernel(int W, int N, double L, const double* __restrict__ R, double* __restrict__ X,
                                    Key key, uint32_t w0) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= W * N) return;
    const int w = t / N, i = t - w * N;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const double z = Draw<double>::normal(philox(w0 + (uint32_t)w, 0u, (uint32_t)i, kInitX + mu, key));
        const double x = R[3 * i + mu] + 0.5 * z;
        X[(size_t)t * 3 + mu] = x - L * floor(x / L);
    }
}

void launch_init_walkers(int W, int N, double L, const double* R, double* X, Key key, uint32_t w0, cudaStream_t st) {
    init_walkers_kernel<<<(W * N + 255) / 256, 256, 0, st>>>(W, N, L, R, X, key, w0);
}

template void launch_orbitals<double>(const SysView<double>&, const double*, int, double*, double*, double*, cudaStream_t);
template void launch_orbitals<float>(const SysView<float>&, const double*, int, float*, float*, float*, cudaStream_t);
template void launch_propose<double>(int, int, double, double*, double*, double*, double*, Key, uint32_t, uint32_t,
                                     double, uint32_t, cudaStream_t);
template void launch_propose<float>(int, int, double, double*, double*, float*, float*, Key, uint32_t, uint32_t,
                                    double, uint32_t, cudaStream_t);

}  // namespace qmc
