// k_twist.cu -- twisted boundary conditions in the FP64 form: Bloch-summed
// Gaussian orbitals, complex Slater inverses, complex Sherman-Morrison sweeps,
// the orbital parts of E_L and of the force estimators, and the twist average.
//
// SI, basis section: orbitals with phi(r + nL) = exp(i theta.n) phi(r) for
// integer vectors n.  The Gaussians become Bloch functions by the lattice sum
//   chi_{a,g}(r) = sum_n exp(i theta.n) exp(-zeta_g |r - R_a - nL|^2),
// truncated to the images n = k + m, m in [-M, M]^3 around the nearest one k
// (M from the smallest exponent: every omitted image lies more than
// sqrt(40 / zeta_min) away).  The sum factorises over the axes:
//   chi = exp(i theta.k) s_x s_y s_z,
//   s_mu = sum_{m=-M..M} exp(i theta_mu m) exp(-zeta (d_mu - m L)^2),  d = r - R_a - kL,
// and a derivative in r_mu acts on s_mu alone.  The spin-up determinant takes
// the walker's twist theta, the spin-down one -theta (the SI's opposite
// twists); the Jastrow factor is the real one of the Gamma-point form.
// Walkers come in K contiguous blocks of Wk = W / K, block t on twist t.  The
// sampled density is |psi|^2 and the estimators take real parts:
//   E_L = Re(H psi / psi),  d ln|psi| / dR = Re(d ln psi / dR),  dE_L / dR = Re(d (H psi / psi) / dR).
// Complex values are double2 (x = real, y = imaginary part).
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cinv(double2 a) {
    const double q = a.x * a.x + a.y * a.y;
    return make_double2(a.x / q, -a.y / q);
}
__device__ __forceinline__ double2 czero() { return make_double2(0.0, 0.0); }

// One axis of a Bloch-summed Gaussian at the minimum-image coordinate d0:
// s[q] = d^q s / dx^q for q = 0..ND, with the phases ph[m + M] = exp(i theta_mu m)
// (conjugated when sg < 0, the spin-down twist).
//   g = e^{-zeta u^2}: g' = -2 zeta u g,  g'' = (4 zeta^2 u^2 - 2 zeta) g,  g''' = (12 zeta^2 u - 8 zeta^3 u^3) g.
template <int ND>
__device__ __forceinline__ void axis_sums(double d0, double zeta, double L, int M, const double2* __restrict__ ph,
                                          double sg, double2 s[ND + 1]) {
#pragma unroll
    for (int q = 0; q <= ND; ++q) s[q] = czero();
    for (int m = -M; m <= M; ++m) {
        const double u = d0 - m * L;
        const double e = exp(-zeta * u * u);
        double2 p = ph[m + M];
        p.y *= sg;
        const double2 pe = cscale(p, e);
        s[0] = cadd(s[0], pe);
        if (ND >= 1) s[1] = cadd(s[1], cscale(pe, -2.0 * zeta * u));
        if (ND >= 2) s[2] = cadd(s[2], cscale(pe, 4.0 * zeta * zeta * u * u - 2.0 * zeta));
        if (ND >= 3) s[3] = cadd(s[3], cscale(pe, 12.0 * zeta * zeta * u - 8.0 * zeta * zeta * zeta * u * u * u));
    }
}

// Minimum-image split of r - R_a and the Bloch phase exp(i sg theta.k) of the
// nearest image k.
__device__ __forceinline__ double2 min_image(const double x[3], const double* __restrict__ Ra, double L, double iL,
                                             const double* __restrict__ th, double sg, double d0[3]) {
    double kth = 0.0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const double d = x[mu] - Ra[mu];
        const double k = rint(d * iL);
        d0[mu] = d - k * L;
        kth += th[mu] * k;
    }
    double sn, cs;
    sincos(sg * kth, &sn, &cs);
    return make_double2(cs, sn);
}

// ---------------------------------------------------------------------------
// Orbital rows: one warp per row (walker w = row / N, electron i = row % N).
// The warp first evaluates the B Bloch-summed basis functions (lanes over the
// basis; Q = 1: values, Q = 5: value, gradient, Laplacian) into its slice of
// shared memory, then contracts them with the real coefficients (lanes over
// the orbitals).  Same layouts as the real kernels: val [rows][n], grad
// [rows][3][n], lap [rows][n], complex.
// ---------------------------------------------------------------------------
template <int Q>
__global__ void __launch_bounds__(256) twist_orbitals_kernel(SysView<double> s, TwistView tv,
                                                             const double* __restrict__ pos, int nrows,
                                                             double2* __restrict__ val, double2* __restrict__ grad,
                                                             double2* __restrict__ lap) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    const int row = blockIdx.x * wpb + warp;
    if (row >= nrows) return;   // whole warps leave; the kernel has no block-wide barrier
    const int N = s.N, n = s.n, B = s.B, G = s.G, M = tv.M;
    double2* chi = (double2*)smraw + (size_t)warp * B * Q;   // [B][Q]
    const int w = row / N, i = row - w * N, t = w / tv.Wk;
    const double sg = i < n ? 1.0 : -1.0;
    const double* th = tv.theta + 3 * t;
    const double2* ph = tv.ph + (size_t)t * 3 * (2 * M + 1);
    const double x[3] = {pos[(size_t)row * 3], pos[(size_t)row * 3 + 1], pos[(size_t)row * 3 + 2]};
    constexpr int ND = Q == 1 ? 0 : 2;
    for (int b = lane; b < B; b += 32) {
        const int a = b / G, g = b - a * G;
        double d0[3];
        const double2 P = min_image(x, s.R + 3 * a, s.L, s.iL, th, sg, d0);
        const double z = s.zeta[g];
        double2 sa[3][ND + 1];
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) axis_sums<ND>(d0[mu], z, s.L, M, ph + mu * (2 * M + 1), sg, sa[mu]);
        const double2 yz = cmul(sa[1][0], sa[2][0]);
        chi[(size_t)b * Q] = cmul(P, cmul(sa[0][0], yz));
        if constexpr (Q == 5) {
            const double2 xz = cmul(sa[0][0], sa[2][0]), xy = cmul(sa[0][0], sa[1][0]);
            chi[(size_t)b * Q + 1] = cmul(P, cmul(sa[0][1], yz));
            chi[(size_t)b * Q + 2] = cmul(P, cmul(sa[1][1], xz));
            chi[(size_t)b * Q + 3] = cmul(P, cmul(sa[2][1], xy));
            chi[(size_t)b * Q + 4] = cmul(P, cadd(cadd(cmul(sa[0][2], yz), cmul(sa[1][2], xz)), cmul(sa[2][2], xy)));
        }
    }
    __syncwarp();
    for (int j = lane; j < n; j += 32) {
        double2 acc[Q];
#pragma unroll
        for (int q = 0; q < Q; ++q) acc[q] = czero();
        for (int b = 0; b < B; ++b) {
            const double c = s.C[(size_t)b * n + j];
#pragma unroll
            for (int q = 0; q < Q; ++q) acc[q] = cadd(acc[q], cscale(chi[(size_t)b * Q + q], c));
        }
        val[(size_t)row * n + j] = acc[0];
        if constexpr (Q == 5) {
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) grad[((size_t)row * 3 + mu) * n + j] = acc[1 + mu];
            lap[(size_t)row * n + j] = acc[4];
        }
    }
}

// Warps per CTA of the orbital kernel: as many [B][Q] slices as fit in 200 KB, at most 8.
static int twist_orb_warps(int B, int Q) {
    const size_t per = (size_t)B * Q * sizeof(double2);
    size_t w = (200u * 1024u) / per;
    return (int)(w < 1 ? 1 : (w > 8 ? 8 : w));
}

void launch_twist_orbitals(const SysView<double>& s, const TwistView& tv, const double* pos, int nrows,
                           double2* val, double2* grad, double2* lap, cudaStream_t st) {
    const int Q = grad ? 5 : 1;
    const int wpb = twist_orb_warps(s.B, Q);
    const size_t smem = (size_t)wpb * s.B * Q * sizeof(double2);
    const int grid = (nrows + wpb - 1) / wpb;
    if (Q == 5) {
        static size_t attr = 0;
        if (smem > attr && cudaFuncSetAttribute(twist_orbitals_kernel<5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem) == cudaSuccess)
            attr = smem;
        twist_orbitals_kernel<5><<<grid, 32 * wpb, smem, st>>>(s, tv, pos, nrows, val, grad, lap);
    } else {
        static size_t attr = 0;
        if (smem > attr && cudaFuncSetAttribute(twist_orbitals_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                (int)smem) == cudaSuccess)
            attr = smem;
        twist_orbitals_kernel<1><<<grid, 32 * wpb, smem, st>>>(s, tv, pos, nrows, val, nullptr, nullptr);
    }
}

// ---------------------------------------------------------------------------
// Complex Gauss-Jordan inverse of walker w's spin block sp (one CTA per block):
// in place with partial pivoting on the largest modulus (Golub & Van Loan
// sec. 3.4), row interchanges undone on the columns at the end.  Output
// Gt[i][j] = (A^-1)_{j,i} and ln|det A| (the sum of ln|pivot|).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) twist_invert_kernel(int N, int n, const double2* __restrict__ Phi,
                                                           double2* __restrict__ Gt, double* __restrict__ logdet,
                                                           int* err) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int w = blockIdx.x >> 1, sp = blockIdx.x & 1;
    const int ld = n + 1;
    double2* Mx = (double2*)smraw;                 // [n][n+1]
    double2* col = Mx + (size_t)n * ld;            // [n]
    int* perm = (int*)(col + n);                   // [n]
    __shared__ int piv_row;
    __shared__ int singular;
    __shared__ double2 ipv_s;
    __shared__ double lsum;
    const int tid = threadIdx.x, nt = blockDim.x;
    const double2* A = Phi + ((size_t)w * N + (size_t)sp * n) * n;
    for (int idx = tid; idx < n * n; idx += nt) Mx[(idx / n) * ld + idx % n] = A[idx];
    if (tid == 0) { singular = 0; lsum = 0.0; }
    __syncthreads();
    for (int k = 0; k < n; ++k) {
        if (tid < 32) {   // argmax |M[i][k]|^2, i >= k (ties -> lowest row)
            double best = -1.0;
            int bi = n;
            for (int i = k + tid; i < n; i += 32) {
                const double2 v = Mx[i * ld + k];
                const double a = v.x * v.x + v.y * v.y;
                if (a > best) { best = a; bi = i; }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(0xffffffffu, best, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
                if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
            }
            if (tid == 0) {
                piv_row = bi;
                perm[k] = bi < n ? bi : k;
                if (!(best > 0.0)) singular = 1;
            }
        }
        __syncthreads();
        if (singular) break;
        const int p = piv_row;
        if (p != k) {
            for (int j = tid; j < n; j += nt) {
                const double2 tmp = Mx[k * ld + j];
                Mx[k * ld + j] = Mx[p * ld + j];
                Mx[p * ld + j] = tmp;
            }
            __syncthreads();
        }
        if (tid == 0) {
            const double2 pv = Mx[k * ld + k];
            lsum += 0.5 * log(pv.x * pv.x + pv.y * pv.y);
            ipv_s = cinv(pv);
        }
        for (int i = tid; i < n; i += nt) col[i] = (i == k) ? czero() : Mx[i * ld + k];
        __syncthreads();
        const double2 ipv = ipv_s;
        for (int j = tid; j < n; j += nt) Mx[k * ld + j] = cmul(j == k ? make_double2(1.0, 0.0) : Mx[k * ld + j], ipv);
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx - i * n;
            if (i == k) continue;
            const double2 base = (j == k) ? czero() : Mx[i * ld + j];
            Mx[i * ld + j] = csub(base, cmul(col[i], Mx[k * ld + j]));
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
                const double2 tmp = Mx[i * ld + k];
                Mx[i * ld + k] = Mx[i * ld + p];
                Mx[i * ld + p] = tmp;
            }
        __syncthreads();
    }
    double2* out = Gt + ((size_t)w * 2 + sp) * n * n;
    for (int idx = tid; idx < n * n; idx += nt) {
        const int i = idx / n, j = idx - i * n;       // Gt[i][j] = inv[j][i]
        out[idx] = Mx[j * ld + i];
    }
    if (tid == 0) logdet[2 * w + sp] = lsum;
}

void launch_twist_invert(int W, int N, int n, const double2* Phi, double2* Gt, double* logdet, int* err,
                         cudaStream_t st) {
    const size_t smem = (size_t)n * (n + 1) * sizeof(double2) + n * sizeof(double2) + n * sizeof(int);
    static size_t attr = 0;
    if (smem > attr &&
        cudaFuncSetAttribute(twist_invert_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
        attr = smem;
    twist_invert_kernel<<<2 * W, n >= 32 ? 256 : 64, smem, st>>>(N, n, Phi, Gt, logdet, err);
}

// ---------------------------------------------------------------------------
// Metropolis sweep with complex Sherman-Morrison updates (one warp per walker;
// the moving spin block's G^T staged in shared memory, row stride n + 1):
//   ratio  R = sum_j phi'_j G^T[i][j],   accept if u < |R|^2 exp(2 dU),
//   G^T[l] <- G^T[l] - (w_l - delta_{l,i}) / R * G^T[i],  w_l = sum_j phi'_j G^T[l][j].
// dU is the real Jastrow difference of the Gamma-point form (with the e-e-n-n
// term when s.fj is set: c_a = sum_j chi_a(r_j) kept per walker, and the pairs
// (i, j != i) change by sum_a (chi_a(r'_i) - chi_a(r_i)) sum_b f_ab (c_b - chi_b(r_i))).  An accepted
// position is wrapped into the box, x = x' - kL; the orbital row of x is
// exp(-i sg theta.k) times that of x', so row i of G^T (column i of the
// inverse) takes the factor exp(i sg theta.k) to stay the inverse of the
// Slater block at the stored positions.
// ---------------------------------------------------------------------------
__host__ __device__ inline size_t twist_sweep_warp_bytes(int N, int n, bool j34) {
    const size_t b = ((size_t)n * (n + 1) + 2 * (size_t)n) * sizeof(double2) + (size_t)(j34 ? 9 : 6) * N * sizeof(double);
    return (b + 15) & ~size_t(15);
}

// e-e-n-n Jastrow orbital exp(-zeta |d|^2) between two points given by their
// (sin, cos)(pi x / L) triples (d the sin-periodised displacement)
__device__ __forceinline__ double tw_jas_orbital(const double* a, const double* b, double ell, double zeta) {
    double t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const double sd = a[mu] * b[3 + mu] - a[3 + mu] * b[mu];
        t += sd * sd;
    }
    return exp(-zeta * ell * ell * t);
}

__device__ __forceinline__ double tw_pair_dist(const double* a, const double* b, double ell) {
    double t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const double sd = a[mu] * b[3 + mu] - a[3 + mu] * b[mu];
        t += sd * sd;
    }
    return ell * sqrt(t);
}

__global__ void __launch_bounds__(256) twist_sweep_kernel(SysView<double> s, TwistView tv, double* __restrict__ X,
                                                          const double* __restrict__ Xp,
                                                          const double* __restrict__ ptp,
                                                          const double* __restrict__ uacc,
                                                          const double2* __restrict__ Phi, double2* __restrict__ Gt,
                                                          unsigned long long* __restrict__ nacc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = s.N, n = s.n, ld = n + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    double* ptr_s = (double*)smraw;                                   // [N][6] proton trig
    const size_t off = ((size_t)6 * N * sizeof(double) + 15) & ~size_t(15);
    const bool j34 = s.fj != nullptr;
    unsigned char* mine = smraw + off + (size_t)warp * twist_sweep_warp_bytes(N, n, j34);
    double2* Gs = (double2*)mine;            // [n][ld]
    double2* rowb = Gs + (size_t)n * ld;     // [n]
    double2* phi = rowb + n;                 // [n]
    double* et = (double*)(phi + n);         // [N][6] electron trig
    double* c34 = et + 6 * N;                // [N] sum over electrons of chi_a (e-e-n-n term)
    double* cho = c34 + N;                   // [N] chi_a at the moving electron
    double* chn = cho + N;                   // [N] chi_a at its proposal
    for (int idx = threadIdx.x; idx < 6 * N; idx += blockDim.x) ptr_s[idx] = s.ptrig[idx];
    __syncthreads();
    const int w = blockIdx.x * wpb + warp;
    if (w >= s.W) return;   // whole warps leave; only warp-level barriers follow

    const double ell = s.ell, bee = s.b_ee, bep = s.b_ep, Zj = s.Zj, L = s.L;
    double* Xw = X + (size_t)w * 3 * N;
    for (int idx = lane; idx < 3 * N; idx += 32) {
        const int i = idx / 3, mu = idx % 3;
        double sn, cs;
        sincospi(Xw[idx] / L, &sn, &cs);
        et[6 * i + mu] = sn;
        et[6 * i + 3 + mu] = cs;
    }
    __syncwarp();
    const double zj = s.zeta_j;
    if (j34) {
        for (int a = lane; a < N; a += 32) {
            double c = 0;
            for (int j = 0; j < N; ++j) c += tw_jas_orbital(et + 6 * j, ptr_s + 6 * a, ell, zj);
            c34[a] = c;
        }
        __syncwarp();
    }
    const double* th = tv.theta + 3 * (w / tv.Wk);
    unsigned long long naccept = 0;
    for (int sp = 0; sp < 2; ++sp) {
        double2* G = Gt + ((size_t)w * 2 + sp) * n * n;
        const double sg = sp == 0 ? 1.0 : -1.0;
        for (int idx = lane; idx < n * n; idx += 32) Gs[(idx / n) * ld + idx % n] = G[idx];
        __syncwarp();
        for (int il = 0; il < n; ++il) {
            const int i = sp * n + il;
            const size_t row = (size_t)w * N + i;
            double pt[6];
#pragma unroll
            for (int mu = 0; mu < 6; ++mu) pt[mu] = ptp[row * 6 + mu];
            for (int j = lane; j < n; j += 32) phi[j] = Phi[row * n + j];
            const double u = uacc[row];
            __syncwarp();
            double2 part = czero();
            for (int j = lane; j < n; j += 32) part = cadd(part, cmul(phi[j], Gs[il * ld + j]));
            const double2 ratio = make_double2(warp_sum(part.x), warp_sum(part.y));
            double du = 0;
            const double* ei = et + 6 * i;
            for (int j = lane; j < N; j += 32) {
                const double* ej = et + 6 * j;
                double u1, u0, d1, d2;
                pade_ee(bee, tw_pair_dist(pt, ej, ell), u1, d1, d2);
                pade_ee(bee, tw_pair_dist(ei, ej, ell), u0, d1, d2);
                du += (j != i) ? u1 - u0 : 0.0;
            }
            for (int a = lane; a < N; a += 32) {
                const double* pa = ptr_s + 6 * a;
                double u1, u0, d1, d2, d3;
                pade_ep(bep, Zj, tw_pair_dist(pt, pa, ell), u1, d1, d2, d3);
                pade_ep(bep, Zj, tw_pair_dist(ei, pa, ell), u0, d1, d2, d3);
                du += u1 - u0;
            }
            if (j34) {
                for (int a = lane; a < N; a += 32) {
                    chn[a] = tw_jas_orbital(pt, ptr_s + 6 * a, ell, zj);
                    cho[a] = tw_jas_orbital(ei, ptr_s + 6 * a, ell, zj);
                }
                __syncwarp();
                for (int a = lane; a < N; a += 32) {
                    const double* fa = s.fj + a;   // f symmetric: column a = row a, consecutive over lanes
                    double wa = 0;
                    for (int b = 0; b < N; ++b) wa += fa[(size_t)b * N] * (c34[b] - cho[b]);
                    du += (chn[a] - cho[a]) * wa;
                }
            }
            du = warp_sum(du);
            const double prob = (ratio.x * ratio.x + ratio.y * ratio.y) * exp(2.0 * du);
            if (u < prob) {
                for (int j = lane; j < n; j += 32) rowb[j] = Gs[il * ld + j];
                __syncwarp();
                const double2 ir = cinv(ratio);
                for (int l = lane; l < n; l += 32) {
                    double2 wl = czero();
                    for (int j = 0; j < n; ++j) wl = cadd(wl, cmul(phi[j], Gs[l * ld + j]));
                    if (l == il) wl.x -= 1.0;
                    const double2 coef = cmul(wl, ir);
                    for (int j = 0; j < n; ++j) Gs[l * ld + j] = csub(Gs[l * ld + j], cmul(coef, rowb[j]));
                }
                __syncwarp();
                double kth = 0.0;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    const double xpl = Xp[row * 3 + mu];
                    kth += th[mu] * floor(xpl / L);
                }
                if (lane < 3) {
                    const double xpl = Xp[row * 3 + lane];
                    const double x = xpl - L * floor(xpl / L);
                    Xw[3 * i + lane] = x;
                    double sn, cs;
                    sincospi(x / L, &sn, &cs);
                    et[6 * i + lane] = sn;
                    et[6 * i + 3 + lane] = cs;
                }
                if (kth != 0.0) {
                    double sn, cs;
                    sincos(sg * kth, &sn, &cs);
                    const double2 f = make_double2(cs, sn);
                    for (int j = lane; j < n; j += 32) Gs[il * ld + j] = cmul(Gs[il * ld + j], f);
                }
                if (j34)
                    for (int a = lane; a < N; a += 32) c34[a] += chn[a] - cho[a];
                ++naccept;
            }
            __syncwarp();
        }
        for (int idx = lane; idx < n * n; idx += 32) G[idx] = Gs[(idx / n) * ld + idx % n];
        __syncwarp();
    }
    if (lane == 0) nacc[w] += naccept;
}

void launch_twist_sweep(const SysView<double>& s, const TwistView& tv, double* X, const double* Xp, const double* ptp,
                        const double* uacc, const double2* Phi, double2* Gt, unsigned long long* nacc,
                        cudaStream_t st) {
    const size_t wb = twist_sweep_warp_bytes(s.N, s.n, s.fj != nullptr);
    const size_t base = ((size_t)6 * s.N * sizeof(double) + 15) & ~size_t(15);
    int wpb = (int)((200u * 1024u - base) / wb);
    wpb = wpb < 1 ? 1 : (wpb > 8 ? 8 : wpb);
    const size_t smem = base + (size_t)wpb * wb;
    static size_t attr = 0;
    if (smem > attr &&
        cudaFuncSetAttribute(twist_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
        attr = smem;
    twist_sweep_kernel<<<(s.W + wpb - 1) / wpb, 32 * wpb, smem, st>>>(s, tv, X, Xp, ptp, uacc, Phi, Gt, nacc);
}

// ---------------------------------------------------------------------------
// g_i = sum_j D_ij G^T[i][j] and l_i = sum_j Lp_ij G^T[i][j] of every electron.
// Their real parts are the only way the complex determinant enters E_L:
//   Re(H psi / psi) = -1/2 sum_i [ Re l_i + 2 Re g_i . grad_i U + lap_i U + |grad_i U|^2 ] + V,
// and the e-n Jastrow force terms take vv_i = Re g_i + grad_i U.  The FP64
// measure kernel computes all of that from real rows D, Lp and inverse rows
// G^T: it is handed D' and Lp' whose column 0 holds Re g_i and Re l_i (the
// other columns stay zero) and G'^T rows e_0 (twist_unit_rows), so its
// sum_j D'_ij G'^T[i][j] is Re g_i exactly.  One warp per electron.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) twist_gl_kernel(int rows, int n, const double2* __restrict__ D,
                                                       const double2* __restrict__ Lp, const double2* __restrict__ Gt,
                                                       int N, double* __restrict__ Dr, double* __restrict__ Lpr) {
    const int lane = threadIdx.x & 31, r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (r >= rows) return;
    const int w = r / N, i = r - w * N, sp = i / n, il = i - sp * n;
    const double2* grow = Gt + (((size_t)w * 2 + sp) * n + il) * n;
    const double2* drow = D + (size_t)r * 3 * n;
    const double2* lrow = Lp + (size_t)r * n;
    double g0 = 0, g1 = 0, g2 = 0, l = 0;
    for (int j = lane; j < n; j += 32) {
        const double2 gj = grow[j];
        const double2 d0 = drow[j], d1 = drow[n + j], d2 = drow[2 * n + j], lj = lrow[j];
        g0 += d0.x * gj.x - d0.y * gj.y;
        g1 += d1.x * gj.x - d1.y * gj.y;
        g2 += d2.x * gj.x - d2.y * gj.y;
        l += lj.x * gj.x - lj.y * gj.y;
    }
    g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2); l = warp_sum(l);
    if (lane == 0) {
        Dr[(size_t)r * 3 * n] = g0;
        Dr[((size_t)r * 3 + 1) * n] = g1;
        Dr[((size_t)r * 3 + 2) * n] = g2;
        Lpr[(size_t)r * n] = l;
    }
}

void launch_twist_gl(int rows, int N, int n, const double2* D, const double2* Lp, const double2* Gt, double* Dr,
                     double* Lpr, cudaStream_t st) {
    twist_gl_kernel<<<(rows + 7) / 8, 256, 0, st>>>(rows, n, D, Lp, Gt, N, Dr, Lpr);
}

// G'^T[w][sp][i][j] = (j == 0) for every walker-spin block (written once per handle).
__global__ void twist_unit_rows_kernel(size_t total, int n, double* __restrict__ Gtr) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < total) Gtr[k] = (k % (size_t)n) == 0 ? 1.0 : 0.0;
}

void launch_twist_unit_rows(int W, int n, double* Gtr, cudaStream_t st) {
    const size_t total = (size_t)W * 2 * n * n;
    twist_unit_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(total, n, Gtr);
}

// ---------------------------------------------------------------------------
// Orbital (Pulay) terms of the force estimators with complex orbitals, one CTA
// per walker, after the measure kernel has accumulated everything else of the
// sample (the Jastrow and Ewald terms; its own orbital force phase runs on zero
// coefficients and adds nothing) and written E_L.  grad_i U (the Pade e-e and
// e-n terms of the sin-periodised Jastrow, and with s.fj the e-e-n-n term
// grad_i U34 = sum_a grad chi_a(r_i) w_ia, w_ia = sum_b f_ab (c_b - chi_b(r_i)),
// c = sum_j chi(r_j)) is formed here again.  Per spin
// block, with G the inverse (G[j][i] = G^T[i][j]),
//   Y_ij = -1/2 Lp_ij - grad_i U . D_ij,  K = G Y G,  Z_bi = sum_j C_bj G_ji,  P_bi = sum_j C_bj K_ji,
//   d ln|psi| / dR_a += -Re sum_i sum_{b in a} Z_bi grad chi_b(r_i)
//   dE_L / dR_a      +=  Re sum_i sum_{b in a} [ P_bi grad chi_b + Z_bi (H_b grad_i U + 1/2 grad lap chi_b) ]
// (chi depends on r - R_a, so d/dR_a = -grad; the Hermitian H makes the R-
// derivative of E the real part).  The sample adds dl, E_L dl and de to the
// walker's accumulators like the measure kernel does.  A warp handles one
// nucleus at a time, lanes over its (Gaussian, electron) pairs: fixed order.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) twist_pulay_kernel(SysView<double> s, TwistView tv,
                                                          const double* __restrict__ X,
                                                          const double2* __restrict__ D,
                                                          const double2* __restrict__ Lp,
                                                          const double2* __restrict__ Gt,
                                                          const double* __restrict__ elw, double* __restrict__ acc,
                                                          double* __restrict__ out_dl, double* __restrict__ out_de) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = s.N, n = s.n, G = s.G, M = tv.M, N3 = 3 * N;
    const int w = blockIdx.x, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    double2* Gm = (double2*)smraw;              // [n][n]  G[j][i]
    double2* YK = Gm + (size_t)n * n;           // [n][n]  Y[i][j], then K[j][i]
    double2* T1 = YK + (size_t)n * n;           // [n][n]  (Y G)[i][i']
    double* fdl = (double*)(T1 + (size_t)n * n); // [3N]
    double* fde = fdl + N3;                      // [3N]
    double* et = fde + N3;                       // [N][6] (sin, cos)(pi x / L) of the electrons
    double* gUw = et + 6 * N;                    // [N][3] grad_i U
    double* c34 = gUw + 3 * N;                   // [N] sum over electrons of chi_a (e-e-n-n term)
    double* rows = c34 + N;                      // per warp [N]: chi_b(r_i)
    const double* th = tv.theta + 3 * (w / tv.Wk);
    const double2* ph = tv.ph + (size_t)(w / tv.Wk) * 3 * (2 * M + 1);
    for (int c = tid; c < N3; c += nt) {
        fdl[c] = 0.0; fde[c] = 0.0;
        double sn, cs;
        sincospi(X[(size_t)w * N3 + c] * s.iL, &sn, &cs);
        et[6 * (c / 3) + c % 3] = sn;
        et[6 * (c / 3) + 3 + c % 3] = cs;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) {          // grad_i U: d t / dx = 2 p, p = (L/pi) sin cos
        double g[3] = {0, 0, 0};
        const double* ei = et + 6 * i;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double sd[3], cd[3], t;
            disp_trig(ei, et + 6 * j, s.ell, sd, cd, t);
            const double r = qsqrt_pair(t);
            double u, u1, u2, f1, f2, f3;
            pade_ee(s.b_ee, r, u, u1, u2);
            rho_to_t(r, u1, u2, 0.0, f1, f2, f3);
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) g[mu] += 2.0 * f1 * (s.ell * sd[mu] * cd[mu]);
        }
        for (int a = 0; a < N; ++a) {
            double sd[3], cd[3], t;
            disp_trig(ei, s.ptrig + 6 * a, s.ell, sd, cd, t);
            const double r = qsqrt_pair(t);
            double u, u1, u2, u3, f1, f2, f3;
            pade_ep(s.b_ep, s.Zj, r, u, u1, u2, u3);
            rho_to_t(r, u1, u2, 0.0, f1, f2, f3);
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) g[mu] += 2.0 * f1 * (s.ell * sd[mu] * cd[mu]);
        }
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) gUw[3 * i + mu] = g[mu];
    }
    __syncthreads();
    if (s.fj) {   // grad chi = -zeta chi grad t, grad t = 2 p, p = (L/pi) sin cos
        const double zj = s.zeta_j;
        for (int a = tid; a < N; a += nt) {
            double c = 0;
            for (int j = 0; j < N; ++j) c += tw_jas_orbital(et + 6 * j, s.ptrig + 6 * a, s.ell, zj);
            c34[a] = c;
        }
        __syncthreads();
        double* row = rows + (size_t)warp * N;
        for (int i = warp; i < N; i += nw) {
            for (int b = lane; b < N; b += 32) row[b] = tw_jas_orbital(et + 6 * i, s.ptrig + 6 * b, s.ell, zj);
            __syncwarp();
            double g[3] = {0, 0, 0};
            for (int a = lane; a < N; a += 32) {
                const double* fa = s.fj + a;   // f symmetric: column a = row a
                double wa = 0;
                for (int b = 0; b < N; ++b) wa += fa[(size_t)b * N] * (c34[b] - row[b]);
                double sd[3], cd[3], t;
                disp_trig(et + 6 * i, s.ptrig + 6 * a, s.ell, sd, cd, t);
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) g[mu] += -2.0 * zj * row[a] * (s.ell * sd[mu] * cd[mu]) * wa;
            }
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) g[mu] = warp_sum(g[mu]);
            if (lane == 0)
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) gUw[3 * i + mu] += g[mu];
            __syncwarp();
        }
        __syncthreads();
    }
    for (int sp = 0; sp < 2; ++sp) {
        const double sg = sp == 0 ? 1.0 : -1.0;
        const double2* Gsp = Gt + ((size_t)w * 2 + sp) * n * n;
        for (int idx = tid; idx < n * n; idx += nt) {
            const int i = idx / n, j = idx - i * n;
            Gm[j * n + i] = Gsp[idx];                     // G[j][i] = G^T[i][j]
            const int e = sp * n + i;
            const size_t r = (size_t)w * N + e;
            const double2* dr = D + r * 3 * n;
            const double2 lp = Lp[r * n + j];
            const double gx = gUw[3 * e], gy = gUw[3 * e + 1], gz = gUw[3 * e + 2];
            YK[idx] = make_double2(-0.5 * lp.x - (gx * dr[j].x + gy * dr[n + j].x + gz * dr[2 * n + j].x),
                                   -0.5 * lp.y - (gx * dr[j].y + gy * dr[n + j].y + gz * dr[2 * n + j].y));
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += nt) {     // T1 = Y G
            const int i = idx / n, c = idx - i * n;
            double2 a = czero();
            for (int j = 0; j < n; ++j) a = cadd(a, cmul(YK[i * n + j], Gm[j * n + c]));
            T1[idx] = a;
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += nt) {     // K = G T1 (over Y)
            const int j = idx / n, c = idx - j * n;
            double2 a = czero();
            for (int i = 0; i < n; ++i) a = cadd(a, cmul(Gm[j * n + i], T1[i * n + c]));
            YK[idx] = a;
        }
        __syncthreads();
        for (int a = warp; a < N; a += nw) {
            double dl[3] = {0, 0, 0}, de[3] = {0, 0, 0};
            for (int pr = lane; pr < G * n; pr += 32) {
                const int g = pr / n, il = pr - g * n, b = a * G + g, e = sp * n + il;
                double2 z = czero(), p = czero();
                for (int j = 0; j < n; ++j) {
                    const double c = s.C[(size_t)b * n + j];
                    z = cadd(z, cscale(Gm[j * n + il], c));
                    p = cadd(p, cscale(YK[j * n + il], c));
                }
                const double x[3] = {X[((size_t)w * N + e) * 3], X[((size_t)w * N + e) * 3 + 1],
                                     X[((size_t)w * N + e) * 3 + 2]};
                double d0[3];
                const double2 P = min_image(x, s.R + 3 * a, s.L, s.iL, th, sg, d0);
                double2 sa[3][4];
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) axis_sums<3>(d0[mu], s.zeta[g], s.L, M, ph + mu * (2 * M + 1), sg, sa[mu]);
                // grad chi, Hessian, grad lap chi of the Bloch Gaussian (each times P)
                double2 gr[3], hs[3][3], tl[3];
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    const int m1 = (mu + 1) % 3, m2 = (mu + 2) % 3;
                    gr[mu] = cmul(P, cmul(sa[mu][1], cmul(sa[m1][0], sa[m2][0])));
                    hs[mu][mu] = cmul(P, cmul(sa[mu][2], cmul(sa[m1][0], sa[m2][0])));
                    hs[mu][m1] = cmul(P, cmul(cmul(sa[mu][1], sa[m1][1]), sa[m2][0]));
                    hs[mu][m2] = cmul(P, cmul(cmul(sa[mu][1], sa[m2][1]), sa[m1][0]));
                    tl[mu] = cmul(P, cadd(cmul(sa[mu][3], cmul(sa[m1][0], sa[m2][0])),
                                          cmul(sa[mu][1], cadd(cmul(sa[m1][2], sa[m2][0]), cmul(sa[m1][0], sa[m2][2])))));
                }
                const double* gu = gUw + 3 * e;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    const double2 hg = cadd(cadd(cscale(hs[mu][0], gu[0]), cscale(hs[mu][1], gu[1])),
                                            cscale(hs[mu][2], gu[2]));
                    const double2 zt = cmul(z, cadd(hg, cscale(tl[mu], 0.5)));
                    const double2 pg = cmul(p, gr[mu]);
                    dl[mu] -= cmul(z, gr[mu]).x;
                    de[mu] += pg.x + zt.x;
                }
            }
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) { dl[mu] = warp_sum(dl[mu]); de[mu] = warp_sum(de[mu]); }
            if (lane == 0)
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) { fdl[3 * a + mu] += dl[mu]; fde[3 * a + mu] += de[mu]; }
        }
        __syncthreads();
    }
    const double EL = elw[w];
    const size_t stride = 3 + 9 * (size_t)N;
    double* aw = acc + (size_t)w * stride;
    bool bad = false;
    for (int c = tid; c < N3; c += nt) {
        const double dl = fdl[c], de = fde[c];
        if (!isfinite(dl) || !isfinite(de)) bad = true;
        aw[3 + c] += dl;
        aw[3 + N3 + c] += EL * dl;
        aw[3 + 2 * N3 + c] += de;
        if (out_dl) { out_dl[(size_t)w * N3 + c] += dl; out_de[(size_t)w * N3 + c] += de; }
    }
    if (bad) raise_err(s.err, kErrNonfinite);
}

size_t twist_pulay_smem_bytes(int N, int n, bool j34) {
    return (size_t)3 * n * n * sizeof(double2) + (size_t)(j34 ? 15 + 1 + 8 : 15) * N * sizeof(double);
}

void launch_twist_pulay(const SysView<double>& s, const TwistView& tv, const double* X, const double2* D,
                        const double2* Lp, const double2* Gt, const double* elw, double* acc, double* out_dl,
                        double* out_de, cudaStream_t st) {
    const size_t smem = twist_pulay_smem_bytes(s.N, s.n, s.fj != nullptr);
    static size_t attr = 0;
    if (smem > attr &&
        cudaFuncSetAttribute(twist_pulay_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
        attr = smem;
    twist_pulay_kernel<<<s.W, 256, smem, st>>>(s, tv, X, D, Lp, Gt, elw, acc, out_dl, out_de);
}

// ---------------------------------------------------------------------------
// Twist average of K per-twist results [E, E_err, N_c, accept, f (3N), S (9N^2)]
// (main text: k-point sampling on a Monkhorst-Pack mesh, equal weights; the
// twists are independent estimates):
//   E, accept, f: means;  E_err = sqrt(sum E_err,t^2) / K;  N_c: sum;  S = sum S_t / K^2.
// ---------------------------------------------------------------------------
__global__ void twist_average_kernel(int K, int N3, const double* __restrict__ tout, double* __restrict__ out) {
    const int len = 4 + N3 + N3 * N3;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= len) return;
    double v = 0.0;
    if (c == 1) {
        for (int t = 0; t < K; ++t) {
            const double e = tout[(size_t)t * len + 1];
            v += e * e;
        }
        out[c] = sqrt(v) / K;
        return;
    }
    for (int t = 0; t < K; ++t) v += tout[(size_t)t * len + c];
    if (c == 2) out[c] = v;                                  // N_c
    else if (c < 4 + N3) out[c] = v / K;                     // E, accept, f
    else out[c] = v / ((double)K * K);                       // S
}

void launch_twist_average(int K, int N, const double* tout, double* out, cudaStream_t st) {
    const int len = 4 + 3 * N + 9 * N * N;
    twist_average_kernel<<<(len + 255) / 256, 256, 0, st>>>(K, 3 * N, tout, out);
}

// Twists sharded over processes: a process whose handle averaged K_r of the K
// twists contributes [K_r E, (K_r E_err)^2, N_c, K_r accept, K_r f, K_r^2 S];
// the sum of the contributions over the processes, divided as below, is the
// average over all K twists (the same combination rule, since
// K_r^2 E_err,r^2 = sum_{t in r} E_err,t^2 and K_r^2 S_r = sum_{t in r} S_t).
__global__ void twist_partial_kernel(double Kr, int N3, const double* __restrict__ out, double* __restrict__ part) {
    const int len = 4 + N3 + N3 * N3;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= len) return;
    const double v = out[c];
    if (c == 1) part[c] = (Kr * v) * (Kr * v);
    else if (c == 2) part[c] = v;
    else if (c < 4 + N3) part[c] = Kr * v;
    else part[c] = Kr * Kr * v;
}

__global__ void twist_combine_kernel(double K, int N3, const double* __restrict__ part, double* __restrict__ out) {
    const int len = 4 + N3 + N3 * N3;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= len) return;
    const double v = part[c];
    if (c == 1) out[c] = sqrt(v) / K;
    else if (c == 2) out[c] = v;
    else if (c < 4 + N3) out[c] = v / K;
    else out[c] = v / (K * K);
}

void launch_twist_partial(int Kr, int N, const double* out, double* part, cudaStream_t st) {
    const int len = 4 + 3 * N + 9 * N * N;
    twist_partial_kernel<<<(len + 255) / 256, 256, 0, st>>>((double)Kr, 3 * N, out, part);
}

void launch_twist_combine(int K, int N, const double* part, double* out, cudaStream_t st) {
    const int len = 4 + 3 * N + 9 * N * N;
    twist_combine_kernel<<<(len + 255) / 256, 256, 0, st>>>((double)K, 3 * N, part, out);
}

}  // namespace qmc
