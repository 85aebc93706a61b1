// k_measure.cu -- local energy and nuclear-force sample of every walker.
//
// One CTA per walker.  From the orbital derivative rows (D = grad phi, Lp =
// lap phi at the current electrons), the inverse G of each spin block and
// the positions it computes
//   E_L = -1/2 sum_i [ l_i - |g_i|^2 + lap_i U + |g_i + grad_i U|^2 ] + V_Ewald
//     g_i = sum_j D_ij G_ji,  l_i = sum_j Lp_ij G_ji
// and, by a hand-written reverse-mode pass (recomputing the basis instead of
// storing it), the derivatives with respect to every nucleus R_a:
//   d ln psi / dR_a = - sum_i sum_{b in a} Z_bi grad chi_b(r_i) - sum_i grad_i u_en(i,a)
//   dE_L / dR_a     =   sum_i sum_{b in a} [ P_bi grad chi_b + Z_bi (H_b grad_i U + 1/2 grad lap chi_b) ]
//                     + sum_i [ (g_i + grad_i U) . H(u_en) + 1/2 grad lap u_en ] + dV/dR_a
//   Z = C G,  P = C (G Y G),  Y_ij = -1/2 Lp_ij - grad_i U . D_ij
// (Hellmann-Feynman term dV/dR plus the Pulay terms through the basis centres
// and the e-n Jastrow).  The force sample f = -dE_L/dR - 2(E_L - E) d ln psi/dR
// is assembled later from the per-walker sums accumulated here:
//   [count, sum E_L, sum E_L^2, sum dlnpsi (3N), sum E_L dlnpsi (3N), sum dE_L (3N)].
// Every reduction is a fixed-order warp or block tree (bitwise reproducible).
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

template <typename T>
struct MLayout {
    size_t xs, xt, et, gU, lU, Ui, gi, vv, li, facc, gacc, rhot, red, stage, cmask, uni, total;
    // split: the B x n orbital contractions run in the adjoint kernel, so the
    // spin-block work space only holds Y^T / M1 and G (and no epilogue stage)
    __host__ __device__ MLayout(int N, int n, int nk, int mmax, bool split = false) {
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = (o + bytes + 15) & ~size_t(15); return r; };
        xs = take(sizeof(double) * 3 * N);
        xt = take(sizeof(T) * 3 * N);
        et = take(sizeof(T) * 6 * N);
        gU = take(sizeof(T) * 3 * N);
        lU = take(sizeof(T) * N);
        Ui = take(sizeof(T) * N);
        gi = take(sizeof(T) * 3 * N);
        vv = take(sizeof(T) * 3 * N);
        li = take(sizeof(T) * N);
        facc = take(sizeof(double) * 9 * N);
        gacc = take(sizeof(T) * 9 * N);
        rhot = take(sizeof(V2<T>) * nk);
        red = take(sizeof(double) * 64);
        stage = take(split ? 0 : sizeof(double) * 64 * 6);
        cmask = take(sizeof(unsigned) * (size_t)N * ((N + 31) / 32));
        // phase table e^{i m theta}, m = 0..mmax (negative m by conjugation)
        const size_t etab = sizeof(V2<T>) * (size_t)N * 3 * (mmax + 1);
        int np = 4;
        while (np < n) np *= 2;
        const size_t spin = split ? sizeof(T) * 2 * (size_t)np * (np + 4) : sizeof(T) * (size_t)np * (3 * (np + 4) + 68);
        // P1 partials: nparts * N <= 256 rows of 5, and (mixed form, N a
        // multiple of 32) the e-e tiles' rows of 5 per electron and partner block
        const size_t jpart = sizeof(T) * 5 * (256 + (size_t)(N / 32) * N);
        // e-e-n-n Jastrow work space: c [N], S [N][3], 8 warps x 5N
        const size_t j34 = sizeof(T) * 44 * (size_t)N;
        size_t u = etab > spin ? etab : spin;
        u = u > j34 ? u : j34;
        uni = take(u > jpart ? u : jpart);
        total = o;
    }
};

// One electron-proton pair: real-space Ewald value v = phi(r) summed over
// images and its gradient g with respect to the electron-proton vector; the
// e-n Jastrow contributions dl (to d ln psi/dR_a) and de (to dE_L/dR_a, given
// vv = g_i + grad_i U).  sd, cd: sin, cos(pi (x - R_a)/L) per component.
// FP32 radial factors of the Pade pair functions in t = rho^2, from one
// reciprocal square root and one reciprocal (the FP64 form goes through
// pade_* and rho_to_t):  f1 = u'/(2 rho),  f2 = (u''/rho^2 - u'/rho^3)/4,
// f3 = (u'''/rho^3 - 3 u''/rho^4 + 3 u'/rho^5)/8.
__device__ __forceinline__ void jas_ee_f32(float t, float b, float& u, float& f1, float& f2) {
    const float ir = rsqrtf(t), r = t * ir, ir2 = ir * ir;
    const float iq = __fdividef(1.0f, 1.0f + b * r), iq2 = iq * iq;
    u = 0.5f * r * iq;
    const float u1 = 0.5f * iq2, u2 = -b * iq2 * iq;
    f1 = 0.5f * u1 * ir;
    f2 = 0.25f * (u2 - u1 * ir) * ir2;
}
__device__ __forceinline__ void jas_ep_f32(float t, float b, float Zj, float& u, float& f1, float& f2, float& f3) {
    const float ir = rsqrtf(t), r = t * ir, ir2 = ir * ir;
    const float iq = __fdividef(1.0f, 1.0f + b * r), iq2 = iq * iq;
    u = -Zj * r * iq;
    const float u1 = -Zj * iq2, u2 = 2.0f * Zj * b * iq2 * iq, u3 = -6.0f * Zj * b * b * iq2 * iq2;
    f1 = 0.5f * u1 * ir;
    f2 = 0.25f * (u2 - u1 * ir) * ir2;
    f3 = 0.125f * (u3 - 3.0f * (u2 - u1 * ir) * ir) * ir2 * ir;
}

// FP32 e-n pair terms of d ln psi / dR and dE_L / dR (same quantities as
// ep_jastrow): g = 2 f1 p, H v = 4 f2 p (p.v) + 2 f1 q o v,
// grad lap u = p o (8 f3 |p|^2 + 8 f2 q + 4 f2 sum q - 2 k^2 f1).
__device__ __forceinline__ void ep_jastrow_f32(const float sd[3], const float cd[3], float ell, float k2, float bep,
                                               float Zj, const float vv[3], float dl[3], float de[3]) {
    float p[3], q[3], s2 = 0.f;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        p[mu] = ell * sd[mu] * cd[mu];
        q[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
        s2 += sd[mu] * sd[mu];
    }
    float u, f1, f2, f3;
    jas_ep_f32(ell * ell * s2, bep, Zj, u, f1, f2, f3);
    const float pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    const float sq = q[0] + q[1] + q[2];
    const float pv = p[0] * vv[0] + p[1] * vv[1] + p[2] * vv[2];
    const float c2 = 2.f * f1, c4 = 4.f * f2;
    const float common = 8.f * f3 * pp + c4 * sq - 2.f * k2 * f1;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        dl[mu] = -c2 * p[mu];
        de[mu] = c4 * p[mu] * pv + c2 * q[mu] * vv[mu] + 0.5f * p[mu] * (common + 8.f * f2 * q[mu]);
    }
}

template <typename S>
__device__ __forceinline__ void ep_jastrow(const S sd[3], const S cd[3], S ell, S k2, S bep, S Zj, const S vv[3],
                                           S dl[3], S de[3]) {
    S p[3], q[3], t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        p[mu] = ell * sd[mu] * cd[mu];
        q[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
        t += sd[mu] * sd[mu];
    }
    t *= ell * ell;
    const S r = qsqrt_pair(t);
    S u, u1, u2, u3, f1, f2, f3;
    pade_ep(bep, Zj, r, u, u1, u2, u3);
    rho_to_t(r, u1, u2, u3, f1, f2, f3);
    RadialDerivs<S> rd;
    radial_chain(p, q, f1, f2, f3, k2, rd);
    S hv[3];
    hess_mul(rd.h, vv, hv);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) { dl[mu] = -rd.g[mu]; de[mu] = hv[mu] + S(0.5) * rd.tl[mu]; }
}

template <typename S>
__device__ __forceinline__ void ep_pair(const S sd[3], const S cd[3], S ell, S k2, S bep, S Zj, S dx, S dy, S dz, S L,
                                        S kap, const S vv[3], S& v, S g[3], S dl[3], S de[3]) {
    S p[3], q[3], t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        p[mu] = ell * sd[mu] * cd[mu];
        q[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
        t += sd[mu] * sd[mu];
    }
    t *= ell * ell;
    const S r = qsqrt_pair(t);
    S u, u1, u2, u3, f1, f2, f3;
    pade_ep(bep, Zj, r, u, u1, u2, u3);
    rho_to_t(r, u1, u2, u3, f1, f2, f3);
    RadialDerivs<S> rd;
    radial_chain(p, q, f1, f2, f3, k2, rd);
    S hv[3];
    hess_mul(rd.h, vv, hv);
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) { dl[mu] = -rd.g[mu]; de[mu] = hv[mu] + S(0.5) * rd.tl[mu]; }
    v = ewald_real<S>(dx, dy, dz, L, kap, g);
}

// e-e-n-n Jastrow orbital chi_a(r_i) = exp(-zeta |d|^2) of electron trig ei and
// nucleus trig pa with its gradient, Hessian, Laplacian and gradient of the
// Laplacian in the electron coordinate (radial chain of f(t) = exp(-zeta t)).
template <typename T>
__device__ __forceinline__ T jas34_orbital(const T* ei, const T* pa, T ell, T zeta, T k2, RadialDerivs<T>& rd) {
    T sd[3], cd[3], t;
    disp_trig(ei, pa, ell, sd, cd, t);
    T p[3], q[3];
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        p[mu] = ell * sd[mu] * cd[mu];
        q[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
    }
    const T e = qexp(-zeta * t);
    radial_chain(p, q, -zeta * e, zeta * zeta * e, -zeta * zeta * zeta * e, k2, rd);
    return e;
}

// kSplit: the B x n orbital contractions and their basis-derivative epilogue
// are left to the tensor-core adjoint kernel; this kernel then writes what
// that kernel needs: K^T per spin block (kt_out), the electrons' (sin, cos)
// and grad U (eg_out, 9 per electron) and E_L of the sample (elw); the
// reciprocal-space force, a fixed [3N][2 nk] matrix times rho(k), is left to a
// GEMM over all walkers, so the structure factor goes out too (rk_out).
template <typename T, bool kSplit>
__global__ void __launch_bounds__(256, kSplit ? 3 : 1) measure_kernel(SysView<T> s, int mmax, const double* __restrict__ X,
                                                      const T* __restrict__ D, const T* __restrict__ Lp,
                                                      const T* __restrict__ Gt, const double* __restrict__ logdet,
                                                      double* __restrict__ acc, double* __restrict__ out_el,
                                                      double* __restrict__ out_lnpsi, double* __restrict__ out_dl,
                                                      double* __restrict__ out_de, float* __restrict__ kt_out,
                                                      float* __restrict__ eg_out, double* __restrict__ elw,
                                                      float* __restrict__ rk_out) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int N = s.N, n = s.n, G = s.G, nk = s.nk;
    const MLayout<T> lay(N, n, nk, mmax, kSplit);
    double* xs = (double*)(sm + lay.xs);
    T* xt = (T*)(sm + lay.xt);
    T* et = (T*)(sm + lay.et);
    T* gU = (T*)(sm + lay.gU);
    T* lU = (T*)(sm + lay.lU);
    T* Ui = (T*)(sm + lay.Ui);
    T* gi = (T*)(sm + lay.gi);
    T* vvs = (T*)(sm + lay.vv);
    T* li = (T*)(sm + lay.li);
    double* f_dl = (double*)(sm + lay.facc);
    double* f_de = f_dl + 3 * N;
    double* f_dv = f_de + 3 * N;
    // FP32-phase partials per nucleus component (one writer each; FP64 sums
    // above hold the FP64 close-pair terms and the SIMT Pulay epilogue)
    T* g_dl = (T*)(sm + lay.gacc);
    T* g_de = g_dl + 3 * N;
    T* g_dv = g_de + 3 * N;
    V2<T>* rhot = (V2<T>*)(sm + lay.rhot);
    double* red = (double*)(sm + lay.red);
    double* stage = (double*)(sm + lay.stage);
    unsigned* cmask = (unsigned*)(sm + lay.cmask);
    unsigned char* uni = sm + lay.uni;

    const int w = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const double L = s.L;
    const T ell = (T)s.ell, bee = (T)s.b_ee, bep = (T)s.b_ep, Zj = (T)s.Zj, kap = (T)s.kappa;
    const double iL = s.iL;
    const T twopiL = T(2.0 * kPi * iL), k2 = twopiL * twopiL;
    const double Zn = 1.0;  // proton charge

    // ---- P0: positions and their (sin, cos)(pi x / L)
    for (int idx = tid; idx < 3 * N; idx += nt) {
        const double x = X[(size_t)w * 3 * N + idx];
        xs[idx] = x;
        xt[idx] = (T)x;
        T sn, cs;
        qsincospi((T)(x * iL), &sn, &cs);
        et[6 * (idx / 3) + idx % 3] = sn;
        et[6 * (idx / 3) + 3 + idx % 3] = cs;
    }
    for (int idx = tid; idx < 9 * N; idx += nt) { f_dl[idx] = 0.0; g_dl[idx] = T(0); }
    for (int idx = tid; idx < N * ((N + 31) / 32); idx += nt) cmask[idx] = 0u;
    __syncthreads();

    // ---- P1: Jastrow gradient / Laplacian per electron, U partial sums.  The
    // partner range is split into nparts slices so that every thread works;
    // the slices are summed in order afterwards.
    const int nparts = nt >= N ? nt / N : 1;
    T* jpart = (T*)uni;
    // Mixed form with N a multiple of 32: each e-e pair is evaluated once, in
    // 32 x 32 tiles of electron blocks (I, J), I <= J, one warp per tile: lane
    // l holds electron 32 I + l and at step k meets electron 32 J + (l + k) mod
    // 32; its row sums stay in the lane and the partner's column sums move one
    // lane per step (shuffle), so that after the tile lane l holds electron
    // 32 J + l's.  A diagonal tile takes steps 1..16 (step 16 on lanes 0-15
    // only).  Each (electron, partner block) has one slot of 5; the slots are
    // summed in block order with the e-n slices below.
    const bool ee_tiles = sizeof(T) == 4 && (N & 31) == 0 && N >= 64;
    T* eepart = jpart + (size_t)5 * 256;   // [N / 32][N][5]
    for (int tt = tid; tt < nparts * N; tt += nt) {
        const int i = tt % N, pi = tt / N;
        const int j0 = (N * pi) / nparts, j1 = (N * (pi + 1)) / nparts;
        T g[3] = {0, 0, 0}, lp = 0, ui = 0;
        const T* ei = et + 6 * i;
        for (int j = ee_tiles ? j1 : j0; j < j1; ++j) {
            if (j == i) continue;
            T sd[3], cd[3], t;
            disp_trig(ei, et + 6 * j, ell, sd, cd, t);
            T u, f1, f2;
            if constexpr (sizeof(T) == 4) {
                jas_ee_f32(t, bee, u, f1, f2);
            } else {
                const T r = qsqrt_pair(t);
                T u1, u2, f3;
                pade_ee(bee, r, u, u1, u2);
                rho_to_t(r, u1, u2, T(0), f1, f2, f3);
            }
            T pp = 0, sq = 0;
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                const T p = ell * sd[mu] * cd[mu];
                g[mu] += T(2) * f1 * p;
                pp += p * p; sq += cd[mu] * cd[mu] - sd[mu] * sd[mu];
            }
            lp += T(4) * f2 * pp + T(2) * f1 * sq;
            if (j > i) ui += u;
        }
        for (int a = j0; a < j1; ++a) {
            T sd[3], cd[3], t;
            disp_trig(ei, s.ptrig + 6 * a, ell, sd, cd, t);
            T u, f1, f2;
            if constexpr (sizeof(T) == 4) {
                float f3;
                jas_ep_f32(t, bep, Zj, u, f1, f2, f3);
            } else {
                const T r = qsqrt_pair(t);
                T u1, u2, u3, f3;
                pade_ep(bep, Zj, r, u, u1, u2, u3);
                rho_to_t(r, u1, u2, T(0), f1, f2, f3);
            }
            T pp = 0, sq = 0;
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                const T p = ell * sd[mu] * cd[mu];
                g[mu] += T(2) * f1 * p;
                pp += p * p; sq += cd[mu] * cd[mu] - sd[mu] * sd[mu];
            }
            lp += T(4) * f2 * pp + T(2) * f1 * sq;
            ui += u;
        }
        T* o = jpart + ((size_t)pi * N + i) * 5;
        o[0] = g[0]; o[1] = g[1]; o[2] = g[2]; o[3] = lp; o[4] = ui;
    }
    if constexpr (sizeof(T) == 4) {
        if (ee_tiles) {
            const int nb = N >> 5, noff = nb * (nb - 1) / 2, ntiles = noff + nb;
            for (int tile = warp; tile < ntiles; tile += nw) {
                int I = 0, J = 0;
                if (tile < noff) {   // off-diagonal tiles, I < J in row-major order
                    int r = tile;
                    while (r >= nb - 1 - I) { r -= nb - 1 - I; ++I; }
                    J = I + 1 + r;
                } else {
                    I = J = tile - noff;
                }
                const bool diag = I == J;
                const int i = 32 * I + lane;
                float ei[6];
#pragma unroll
                for (int c = 0; c < 6; ++c) ei[c] = et[6 * i + c];
                float rg[3] = {0.f, 0.f, 0.f}, rl = 0.f, ru = 0.f, cg[3] = {0.f, 0.f, 0.f}, cl = 0.f;
                const int k0 = diag ? 1 : 0, k1 = diag ? 17 : 32;
                for (int k = k0; k < k1; ++k) {
                    if (!diag || k < 16 || lane < 16) {
                        const int j = 32 * J + ((lane + k) & 31);
                        float sd[3], cd[3], t;
                        disp_trig(ei, et + 6 * j, ell, sd, cd, t);
                        float u, f1, f2;
                        jas_ee_f32(t, bee, u, f1, f2);
                        float pp = 0.f, sq = 0.f;
#pragma unroll
                        for (int mu = 0; mu < 3; ++mu) {
                            const float pm = ell * sd[mu] * cd[mu], gm = 2.f * f1 * pm;
                            rg[mu] += gm;
                            cg[mu] -= gm;   // p is odd under the exchange of the pair
                            pp += pm * pm;
                            sq += cd[mu] * cd[mu] - sd[mu] * sd[mu];
                        }
                        const float lpv = 4.f * f2 * pp + 2.f * f1 * sq;
                        rl += lpv;
                        cl += lpv;
                        ru += u;
                    }
                    // the column sums move to the lane that meets their electron next
                    const int src = (lane + 1) & 31;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) cg[mu] = __shfl_sync(0xffffffffu, cg[mu], src);
                    cl = __shfl_sync(0xffffffffu, cl, src);
                }
                if (diag) {   // lane l holds column (l + 17) mod 32: column l's come from lane (l + 15) mod 32
                    const int src = (lane + 15) & 31;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) cg[mu] = __shfl_sync(0xffffffffu, cg[mu], src);
                    cl = __shfl_sync(0xffffffffu, cl, src);
                    T* o = eepart + ((size_t)I * N + i) * 5;
                    o[0] = rg[0] + cg[0]; o[1] = rg[1] + cg[1]; o[2] = rg[2] + cg[2]; o[3] = rl + cl; o[4] = ru;
                } else {
                    T* o = eepart + ((size_t)J * N + i) * 5;
                    o[0] = rg[0]; o[1] = rg[1]; o[2] = rg[2]; o[3] = rl; o[4] = ru;
                    T* oc = eepart + ((size_t)I * N + 32 * J + lane) * 5;
                    oc[0] = cg[0]; oc[1] = cg[1]; oc[2] = cg[2]; oc[3] = cl; oc[4] = 0.f;
                }
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) {
        T v[5] = {0, 0, 0, 0, 0};
        for (int pi = 0; pi < nparts; ++pi)
#pragma unroll
            for (int c = 0; c < 5; ++c) v[c] += jpart[((size_t)pi * N + i) * 5 + c];
        if (ee_tiles)
            for (int pb = 0; pb < (N >> 5); ++pb)
#pragma unroll
                for (int c = 0; c < 5; ++c) v[c] += eepart[((size_t)pb * N + i) * 5 + c];
        gU[3 * i] = v[0]; gU[3 * i + 1] = v[1]; gU[3 * i + 2] = v[2];
        lU[i] = v[3]; Ui[i] = v[4];
    }

    // ---- P2: g_i = sum_j D_ij G_ji, l_i = sum_j Lp_ij G_ji (warp per electron,
    // lanes over the orbitals: coalesced rows of D, Lp and G^T)
    for (int i = warp; i < N; i += nw) {
        const int sp = i / n, il = i - sp * n;
        const T* grow = Gt + (((size_t)w * 2 + sp) * n + il) * n;
        const T* drow = D + ((size_t)w * N + i) * 3 * n;
        const T* lrow = Lp + ((size_t)w * N + i) * n;
        T g0 = 0, g1 = 0, g2 = 0, l = 0;
        for (int j = lane; j < n; j += 32) {
            const T gj = grow[j];
            g0 += drow[j] * gj; g1 += drow[n + j] * gj; g2 += drow[2 * n + j] * gj;
            l += lrow[j] * gj;
        }
        g0 = warp_sum(g0); g1 = warp_sum(g1); g2 = warp_sum(g2); l = warp_sum(l);
        if (lane == 0) { gi[3 * i] = g0; gi[3 * i + 1] = g1; gi[3 * i + 2] = g2; li[i] = l; }
    }
    __syncthreads();

    // ---- P2b (FP64 form with the e-e-n-n Jastrow term):
    //   U34 = sum_{i<j} chi_i^T F chi_j = 1/2 sum_i chi_i . w_i,  w_i = F (c - chi_i),  c = sum_j chi_j,
    //   grad_i U34 = sum_a grad chi_a(r_i) w_ia,  lap_i U34 = sum_a lap chi_a(r_i) w_ia,
    // added to grad U, lap U and the per-electron U sums.  c and S_a = sum_j grad chi_a(r_j)
    // stay in the work space for the force terms after P3.
    T* j34c = (T*)uni;               // [N]
    T* j34S = j34c + N;              // [N][3]
    T* j34w = j34S + 3 * N;          // per warp: chi_i [N], grad chi_i [N][3], lap chi_i [N]
    {
        if (s.fjt) {
            const T zj = (T)s.zeta_j;
            for (int a = tid; a < N; a += nt) {
                T c = 0, g[3] = {0, 0, 0};
                for (int j = 0; j < N; ++j) {
                    RadialDerivs<T> rd;
                    c += jas34_orbital(et + 6 * j, s.ptrig + 6 * a, ell, zj, k2, rd);
                    for (int mu = 0; mu < 3; ++mu) g[mu] += rd.g[mu];
                }
                j34c[a] = c;
                for (int mu = 0; mu < 3; ++mu) j34S[3 * a + mu] = g[mu];
            }
            __syncthreads();
            T* stc = j34w + (size_t)warp * 5 * N;
            for (int i = warp; i < N; i += nw) {
                for (int a = lane; a < N; a += 32) {
                    RadialDerivs<T> rd;
                    stc[a] = jas34_orbital(et + 6 * i, s.ptrig + 6 * a, ell, zj, k2, rd);
                }
                __syncwarp();
                T g[3] = {0, 0, 0}, l = 0, u = 0;
                for (int a = lane; a < N; a += 32) {
                    RadialDerivs<T> rd;
                    const T chi = jas34_orbital(et + 6 * i, s.ptrig + 6 * a, ell, zj, k2, rd);
                    const T* fa = s.fjt + a;   // column a = row a (f symmetric): coalesced over lanes
                    T w = 0;
                    for (int b = 0; b < N; ++b) w += fa[(size_t)b * N] * (j34c[b] - stc[b]);
                    for (int mu = 0; mu < 3; ++mu) g[mu] += rd.g[mu] * w;
                    l += rd.lap * w;
                    u += chi * w;
                }
                for (int mu = 0; mu < 3; ++mu) g[mu] = warp_sum(g[mu]);
                l = warp_sum(l);
                u = warp_sum(u);
                if (lane == 0) {
                    for (int mu = 0; mu < 3; ++mu) gU[3 * i + mu] += g[mu];
                    lU[i] += l;
                    Ui[i] += T(0.5) * u;
                }
                __syncwarp();
            }
            __syncthreads();
        }
    }

    // ---- P3: kinetic energy and U
    double kin_p = 0.0, u_p = 0.0;
    for (int i = tid; i < N; i += nt) {
        T g2 = 0, t2 = 0;
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const T g = gi[3 * i + mu], t = g + gU[3 * i + mu];
            g2 += g * g; t2 += t * t;
            vvs[3 * i + mu] = t;     // grad_i ln psi, for the e-n pair terms
        }
        kin_p += (double)(li[i] - g2 + lU[i] + t2);
        u_p += (double)Ui[i];
    }
    const double kin = block_sum(kin_p, red);
    const double Utot = block_sum(u_p, red + 32);

    // ---- P3b (with the e-e-n-n Jastrow term): its terms of d ln psi / dR_a
    // and dE_L / dR_a.  With s_a^(i) = S_a - grad chi_a(r_i), v_ia = sum_b grad chi_b(r_i) f_ba,
    // lam_ia = sum_b lap chi_b(r_i) f_ba and vv_i = g_i + grad_i U:
    //   dlnpsi/dR_a += -sum_i grad chi_a(r_i) w_ia
    //   dE_L/dR_a   += sum_i [ 1/2 (grad lap chi_a(r_i) w_ia + lam_ia s_a^(i))
    //                          + (Hess chi_a(r_i) vv_i) w_ia + (vv_i . v_ia) s_a^(i) ]
    // (the R_a-derivative of -1/2 sum_i [lap_i U34 + 2 vv_i . grad_i U34]).
    {
        if (s.fjt) {
            const T zj = (T)s.zeta_j;
            T* st = j34w + (size_t)warp * 5 * N;   // chi_i [N], grad chi_i [N][3], lap chi_i [N]
            for (int i = warp; i < N; i += nw) {
                for (int a = lane; a < N; a += 32) {
                    RadialDerivs<T> rd;
                    st[a] = jas34_orbital(et + 6 * i, s.ptrig + 6 * a, ell, zj, k2, rd);
                    for (int mu = 0; mu < 3; ++mu) st[N + 3 * a + mu] = rd.g[mu];
                    st[4 * N + a] = rd.lap;
                }
                __syncwarp();
                T vv[3];
                for (int mu = 0; mu < 3; ++mu) vv[mu] = gi[3 * i + mu] + gU[3 * i + mu];
                for (int a = lane; a < N; a += 32) {
                    RadialDerivs<T> rd;
                    jas34_orbital(et + 6 * i, s.ptrig + 6 * a, ell, zj, k2, rd);
                    const T* fa = s.fjt + a;   // column a = row a (f symmetric): coalesced over lanes
                    T w = 0, v[3] = {0, 0, 0}, lam = 0;
                    for (int b = 0; b < N; ++b) {
                        const T f = fa[(size_t)b * N];
                        w += f * (j34c[b] - st[b]);
                        for (int mu = 0; mu < 3; ++mu) v[mu] += st[N + 3 * b + mu] * f;
                        lam += st[4 * N + b] * f;
                    }
                    T hv[3];
                    hess_mul(rd.h, vv, hv);
                    const T vvv = vv[0] * v[0] + vv[1] * v[1] + vv[2] * v[2];
                    for (int mu = 0; mu < 3; ++mu) {
                        const T sa = j34S[3 * a + mu] - rd.g[mu];
                        atomicAdd(&f_dl[3 * a + mu], (double)(-rd.g[mu] * w));
                        atomicAdd(&f_de[3 * a + mu],
                                  (double)(T(0.5) * (rd.tl[mu] * w + lam * sa) + hv[mu] * w + vvv * sa));
                    }
                }
                __syncwarp();
            }
            __syncthreads();
        }
    }

    // ---- P4a: electron-electron real-space Ewald
    double vee_p = 0.0;
    const T Lt = (T)L;
    const float iLt = 1.f / (float)Lt, rc2 = kRealCut2Mixed * (float)Lt * (float)Lt;
    // balanced cyclic pairing: electron i with i+d (mod N), d = 1..N/2 (d = N/2 only for i < N/2),
    // the distance range split into nparts slices
    for (int tt = tid; tt < nparts * N; tt += nt) {
        const int i = tt % N, pi = tt / N, half = N / 2;
        const int d0 = 1 + (half * pi) / nparts, d1 = 1 + (half * (pi + 1)) / nparts;
        T v = 0;
        for (int d = d0; d < d1; ++d) {
            const bool skip = 2 * d == N && i >= half;
            const int j = i + d < N ? i + d : i + d - N;      // (i + d) mod N, d < N
            if (skip) continue;
            if constexpr (sizeof(T) == 4) {
                v += ewald_real_cut<false>(xt[3 * i] - xt[3 * j], xt[3 * i + 1] - xt[3 * j + 1],
                                           xt[3 * i + 2] - xt[3 * j + 2], false, Lt, iLt, rc2, kap, nullptr);
                continue;
            }
            v += ewald_real<T>(xt[3 * i] - xt[3 * j], xt[3 * i + 1] - xt[3 * j + 1], xt[3 * i + 2] - xt[3 * j + 2], Lt,
                               kap, nullptr);
        }
        vee_p += (double)v;
    }
    // ---- P4b: electron-proton pairs (warp per proton, lanes over electrons): the
    // real-space Ewald energy and its R-gradient (Hellmann-Feynman) together with
    // the e-n Jastrow terms of d ln psi/dR and dE_L/dR.  In the mixed form, pairs
    // closer than 0.3 bohr are only flagged here and evaluated afterwards in FP64
    // (one thread per proton, electrons in increasing order): there the 1/r^2
    // Coulomb force and the 1/r^2 part of grad lap u_en cancel (cusp
    // condition), and FP32 rounding of either term would survive the
    // cancellation.  Deferring them keeps FP64 off the common path.
    double vep_p = 0.0;
    T vep_t = 0;
    const int nwords = (N + 31) / 32;
    for (int a = warp; a < N; a += nw) {
        T v = 0, gv[3] = {0, 0, 0}, dl[3] = {0, 0, 0}, de[3] = {0, 0, 0};
        // the nucleus' trig values and position stay in registers over its electrons
        T pa[6], ra[3];
#pragma unroll
        for (int c = 0; c < 6; ++c) pa[c] = s.ptrig[6 * a + c];
#pragma unroll
        for (int c = 0; c < 3; ++c) ra[c] = s.RT[3 * a + c];
        for (int i = lane; i < N; i += 32) {
            T sd[3], cd[3], t;
            disp_trig(et + 6 * i, pa, ell, sd, cd, t);
            const bool close = sizeof(T) == 4 && t < T(0.09);
            if (close) atomicOr(&cmask[a * nwords + (i >> 5)], 1u << (i & 31));
            if constexpr (sizeof(T) == 4) {
                // FP32: Jastrow terms unless close; the Ewald images inside the
                // FP32-level cutoff (a close pair's nearest image is done in FP64)
                if (!close) {
                    T vv[3], pl[3], pe[3];
                    for (int mu = 0; mu < 3; ++mu) vv[mu] = vvs[3 * i + mu];
                    ep_jastrow_f32(sd, cd, ell, k2, bep, Zj, vv, pl, pe);
                    for (int mu = 0; mu < 3; ++mu) { dl[mu] += pl[mu]; de[mu] += pe[mu]; }
                }
                v += ewald_real_cut<true>(xt[3 * i] - ra[0], xt[3 * i + 1] - ra[1], xt[3 * i + 2] - ra[2], close, Lt,
                                          iLt, rc2, kap, gv);
                continue;
            }
            if (close) {   // only the images other than the nearest one here
                T pg[3] = {0, 0, 0};
                v += ewald_real<T>(xt[3 * i] - ra[0], xt[3 * i + 1] - ra[1], xt[3 * i + 2] - ra[2], Lt, kap, pg, true);
                for (int mu = 0; mu < 3; ++mu) gv[mu] += pg[mu];
                continue;
            }
            T vv[3], pv, pg[3], pl[3], pe[3];
            for (int mu = 0; mu < 3; ++mu) vv[mu] = gi[3 * i + mu] + gU[3 * i + mu];
            ep_pair<T>(sd, cd, ell, k2, bep, Zj, xt[3 * i] - ra[0], xt[3 * i + 1] - ra[1], xt[3 * i + 2] - ra[2],
                       Lt, kap, vv, pv, pg, pl, pe);
            v += pv;
            for (int mu = 0; mu < 3; ++mu) { gv[mu] += pg[mu]; dl[mu] += pl[mu]; de[mu] += pe[mu]; }
        }
        v = warp_sum(v);
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) { gv[mu] = warp_sum(gv[mu]); dl[mu] = warp_sum(dl[mu]); de[mu] = warp_sum(de[mu]); }
        if (lane == 0) {   // FP32 partials; FP64 only where the sample is accumulated
            vep_t += -(T)Zn * v;
            for (int mu = 0; mu < 3; ++mu) {
                g_dv[3 * a + mu] = (T)Zn * gv[mu];
                g_dl[3 * a + mu] = dl[mu];
                g_de[3 * a + mu] = de[mu];
            }
        }
    }
    if (sizeof(T) == 4) {
        // Close pairs in FP64, one thread per pair: the e-n Jastrow terms and
        // the nearest-image real-space Coulomb term (the pair's other images
        // were summed in FP32 above).  Pairs are numbered nucleus by nucleus,
        // electrons in increasing order; each nucleus sums its pairs' results
        // in that order, so the sums do not depend on the thread count.
        int* coff = (int*)uni;                                       // [N + 1] pair offsets
        double* slot = (double*)(uni + (((size_t)(N + 1) * sizeof(int) + 15) & ~size_t(15)));
        const size_t uni_bytes = lay.total - lay.uni;
        const int CH = (int)((uni_bytes - ((size_t)(slot) - (size_t)uni)) / (10 * sizeof(double)));
        __syncthreads();
        if (warp == 0) {   // exclusive scan of the per-nucleus counts
            const int per = (N + 31) / 32, a0 = lane * per;
            int loc = 0;
            for (int a = a0; a < a0 + per && a < N; ++a)
                for (int wd = 0; wd < nwords; ++wd) loc += __popc(cmask[a * nwords + wd]);
            int inc = loc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += y;
            }
            int run = inc - loc;
            for (int a = a0; a < a0 + per && a < N; ++a) {
                coff[a] = run;
                for (int wd = 0; wd < nwords; ++wd) run += __popc(cmask[a * nwords + wd]);
            }
            if (lane == 31) coff[N] = inc;
        }
        __syncthreads();
        const int total = coff[N];
        const double k2d = (2.0 * kPi * iL) * (2.0 * kPi * iL);
        for (int base = 0; base < total; base += CH) {
            const int end = base + CH < total ? base + CH : total;
            for (int t = base + tid; t < end; t += nt) {
                int lo = 0, hi = N;   // nucleus: coff[a] <= t < coff[a + 1]
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (coff[mid] <= t) lo = mid; else hi = mid;
                }
                const int a = lo;
                int k = t - coff[a], i = 0;
                for (int wd = 0; wd < nwords; ++wd) {
                    const unsigned m = cmask[a * nwords + wd];
                    const int c = __popc(m);
                    if (k < c) { i = wd * 32 + nth_set_bit(m, k); break; }
                    k -= c;
                }
                const double dx = xs[3 * i] - s.R[3 * a], dy = xs[3 * i + 1] - s.R[3 * a + 1],
                             dz = xs[3 * i + 2] - s.R[3 * a + 2];
                double sdd[3], cdd[3], vv[3], pl[3], pe[3];
                sincospi(dx * iL, &sdd[0], &cdd[0]);
                sincospi(dy * iL, &sdd[1], &cdd[1]);
                sincospi(dz * iL, &sdd[2], &cdd[2]);
                for (int mu = 0; mu < 3; ++mu) vv[mu] = (double)gi[3 * i + mu] + (double)gU[3 * i + mu];
                ep_jastrow<double>(sdd, cdd, s.ell, k2d, s.b_ep, s.Zj, vv, pl, pe);
                const double mx = dx - L * rint(dx * iL), my = dy - L * rint(dy * iL), mz = dz - L * rint(dz * iL);
                const double r2 = mx * mx + my * my + mz * mz, r = sqrt(r2), ir = 1.0 / r;
                const double ec = erfc(s.kappa * r);
                const double sg = -(ec * ir + 1.1283791670955126 * s.kappa * exp(-s.kappa * s.kappa * r2)) * ir * ir;
                double* o = slot + (size_t)(t - base) * 10;
                o[0] = ec * ir;
                o[1] = sg * mx; o[2] = sg * my; o[3] = sg * mz;
                for (int mu = 0; mu < 3; ++mu) { o[4 + mu] = pl[mu]; o[7 + mu] = pe[mu]; }
            }
            __syncthreads();
            for (int a = tid; a < N; a += nt) {
                const int lo = coff[a] > base ? coff[a] : base, hi = coff[a + 1] < end ? coff[a + 1] : end;
                if (lo >= hi) continue;
                double vC = 0, gC[3] = {0, 0, 0}, dlC[3] = {0, 0, 0}, deC[3] = {0, 0, 0};
                for (int t = lo; t < hi; ++t) {
                    const double* o = slot + (size_t)(t - base) * 10;
                    vC += o[0];
                    for (int mu = 0; mu < 3; ++mu) { gC[mu] += o[1 + mu]; dlC[mu] += o[4 + mu]; deC[mu] += o[7 + mu]; }
                }
                vep_p += -Zn * vC;
                for (int mu = 0; mu < 3; ++mu) {
                    f_dv[3 * a + mu] += Zn * gC[mu];
                    f_dl[3 * a + mu] += dlC[mu];
                    f_de[3 * a + mu] += deC[mu];
                }
            }
            __syncthreads();
        }
    }
    // ---- P4c: reciprocal space: electron structure factor from per-electron phase tables
    V2<T>* etab = (V2<T>*)uni;
    const int nm = mmax + 1;   // m = 0..mmax; e^{-i m theta} = conj(e^{i m theta})
    for (int idx = tid; idx < 3 * N; idx += nt) {
        T sn, cs;
        qsincospi((T)(2.0 * iL) * xt[idx], &sn, &cs);
        V2<T>* e = etab + (size_t)idx * nm;
        V2<T> cur{T(1), T(0)};
        e[0] = cur;
        for (int m = 1; m <= mmax; ++m) {
            cur = V2<T>{cur.x * cs - cur.y * sn, cur.x * sn + cur.y * cs};
            e[m] = cur;
        }
    }
    __syncthreads();
    double vrec_p = 0.0;
    T vrec_t = 0;
    for (int k = tid; k < nk; k += nt) {
        const int4 m = s.kvec[k];
        T re = 0, im = 0;
        for (int i = 0; i < N; ++i) {
            const V2<T> a = etab[(3 * i) * nm + m.x];   // m.x >= 0 in the half space
            V2<T> b = etab[(3 * i + 1) * nm + (m.y < 0 ? -m.y : m.y)], c = etab[(3 * i + 2) * nm + (m.z < 0 ? -m.z : m.z)];
            if (m.y < 0) b.y = -b.y;
            if (m.z < 0) c.y = -c.y;
            const T abx = a.x * b.x - a.y * b.y, aby = a.x * b.y + a.y * b.x;
            re += abx * c.x - aby * c.y;
            im += abx * c.y + aby * c.x;
        }
        const double2 rp = s.rho_p[k];
        const T rr = (T)rp.x - re, ri = (T)rp.y - im;   // electrons carry -1
        rhot[k] = V2<T>{rr, ri};
        if constexpr (kSplit) {
            rk_out[(size_t)w * 2 * nk + 2 * k] = (float)rr;
            rk_out[(size_t)w * 2 * nk + 2 * k + 1] = (float)ri;
        }
        vrec_t += s.kwt[k] * (rr * rr + ri * ri);
    }
    vrec_p += (double)vrec_t;
    __syncthreads();
    // ---- P4d: reciprocal-space force on the protons (warp per proton; the
    // split path leaves it to the GEMM)
    for (int a = warp; a < (kSplit ? 0 : N); a += nw) {
        T gx = 0, gy = 0, gz = 0;
#pragma unroll 4
        for (int k = lane; k < nk; k += 32) {
            const V2<T> e = s.eikRt[(size_t)a * nk + k];
            const V2<T> rd = rhot[k];
            const T c = T(2) * (T)Zn * s.kwt[k] * (rd.y * e.x - rd.x * e.y);
            const int4 m = s.kvec[k];
            gx += c * twopiL * (T)m.x; gy += c * twopiL * (T)m.y; gz += c * twopiL * (T)m.z;
        }
        gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
        if (lane == 0) { g_dv[3 * a] += gx; g_dv[3 * a + 1] += gy; g_dv[3 * a + 2] += gz; }
    }
    vep_p += (double)vep_t;
    const double vee = block_sum(vee_p, red);
    const double vep = block_sum(vep_p, red + 32);
    const double vrec = block_sum(vrec_p, red);

    __syncthreads();

    // ---- P6: orbital (Pulay) terms, one spin block at a time.  All n x n and
    // B x n products are register-tiled 4 x 4 per thread on a zero-padded
    // np x np block (np = padded n, a power of two >= 4):
    //   M1 = Y G,  K = G M1  (= G Y G),  Z = C G,  P = C K  (per 64-row tile of C)
    // and the basis-derivative contraction is fused onto each Z/P tile.
    const int np = s.np, ldt = np + 4, ng = np / 4;
    const int lnp = __ffs(np) - 1;   // np is a power of two: index arithmetic by shifts (no integer division)
    if constexpr (kSplit) {
        // K = G Y G per spin block for the adjoint kernel, in two buffers: the
        // 4 x 4 register tiles of M1 = Y G overwrite Y^T once every thread has
        // read it, and K^T goes out through the G buffer (coalesced stores).
        T* bufY = (T*)uni;                       // Y^T [j][i], then M1 [i][i']
        T* bufG2 = bufY + (size_t)np * ldt;      // G [j][i], then K^T [i'][j]
        const int r0 = 4 * (tid / ng), c0 = 4 * (tid % ng);
        const bool act = tid < ng * ng;
        for (int sp = 0; sp < 2; ++sp) {
            const T* Gsp = Gt + ((size_t)w * 2 + sp) * n * n;
            for (int idx = tid; idx < np * np; idx += nt) {
                const int il = idx >> lnp, j = idx & (np - 1);
                T g = 0, y = 0;
                if (il < n && j < n) {
                    const int i = sp * n + il;
                    g = Gsp[il * n + j];
                    const size_t rr = (size_t)w * N + i;
                    const T* dr = D + rr * 3 * n;
                    y = T(-0.5) * Lp[rr * n + j] -
                        (gU[3 * i] * dr[j] + gU[3 * i + 1] * dr[n + j] + gU[3 * i + 2] * dr[2 * n + j]);
                }
                bufG2[j * ldt + il] = g;
                bufY[j * ldt + il] = y;
            }
            __syncthreads();
            T acc4[4][4] = {};
            if (act) {                           // M1[i][i'] = sum_j Y[i][j] G[j][i']
                for (int j = 0; j < np; ++j) {
                    T y4[4], g4[4];
                    load4(bufY + j * ldt + r0, y4);
                    load4(bufG2 + j * ldt + c0, g4);
#pragma unroll
                    for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                        for (int b_ = 0; b_ < 4; ++b_) acc4[a_][b_] += y4[a_] * g4[b_];
                }
            }
            __syncthreads();
            if (act)
#pragma unroll
                for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                    for (int b_ = 0; b_ < 4; ++b_) bufY[(r0 + a_) * ldt + c0 + b_] = acc4[a_][b_];
            __syncthreads();
            if (act) {                           // K[j][i'] = sum_i G[j][i] M1[i][i']
#pragma unroll
                for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                    for (int b_ = 0; b_ < 4; ++b_) acc4[a_][b_] = 0;
                for (int i = 0; i < np; ++i) {
                    T m4[4];
                    load4(bufY + i * ldt + c0, m4);
#pragma unroll
                    for (int a_ = 0; a_ < 4; ++a_) {
                        const T gji = bufG2[(r0 + a_) * ldt + i];
#pragma unroll
                        for (int b_ = 0; b_ < 4; ++b_) acc4[a_][b_] += gji * m4[b_];
                    }
                }
            }
            __syncthreads();
            if (act)
#pragma unroll
                for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                    for (int b_ = 0; b_ < 4; ++b_) bufG2[(c0 + b_) * ldt + r0 + a_] = acc4[a_][b_];
            __syncthreads();
            float* ko = kt_out + ((size_t)w * 2 + sp) * n * n;
            for (int idx = tid; idx < np * np; idx += nt) {
                const int i = idx >> lnp, j = idx & (np - 1);
                if (i < n && j < n) ko[i * n + j] = (float)bufG2[i * ldt + j];
            }
            __syncthreads();
        }
    } else {
    T* bufA = (T*)uni;                       // Y^T [j][i], later K [j][i]
    T* bufG = bufA + (size_t)np * ldt;       // G   [j][i] = G_{j,i}
    T* bufS = bufG + (size_t)np * ldt;       // G^T [i][j], later C^T tile [j][b] (stride 68)
    T* bufM = bufS + (size_t)np * 68;        // M1  [i][i']
    for (int sp = 0; sp < 2; ++sp) {
        const T* Gsp = Gt + ((size_t)w * 2 + sp) * n * n;
        for (int idx = tid; idx < np * np; idx += nt) {
            const int il = idx >> lnp, j = idx & (np - 1);
            T g = 0, y = 0;
            if (il < n && j < n) {
                const int i = sp * n + il;
                g = Gsp[il * n + j];
                const size_t rr = (size_t)w * N + i;
                const T* dr = D + rr * 3 * n;
                y = T(-0.5) * Lp[rr * n + j] - (gU[3 * i] * dr[j] + gU[3 * i + 1] * dr[n + j] + gU[3 * i + 2] * dr[2 * n + j]);
            }
            bufS[il * ldt + j] = g;
            bufG[j * ldt + il] = g;
            bufA[j * ldt + il] = y;
        }
        __syncthreads();
        if (tid < ng * ng) {                     // M1[i][i'] = sum_j Y[i][j] G[j][i']
            const int r0 = 4 * (tid / ng), c0 = 4 * (tid % ng);
            T acc4[4][4] = {};
            for (int j = 0; j < np; ++j) {
                T y4[4], g4[4];
                load4(bufA + j * ldt + r0, y4);
                load4(bufG + j * ldt + c0, g4);
#pragma unroll
                for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                    for (int b_ = 0; b_ < 4; ++b_) acc4[a_][b_] += y4[a_] * g4[b_];
            }
#pragma unroll
            for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                for (int b_ = 0; b_ < 4; ++b_) bufM[(r0 + a_) * ldt + c0 + b_] = acc4[a_][b_];
        }
        __syncthreads();
        if (tid < ng * ng) {                     // K[j][i'] = sum_i G[j][i] M1[i][i']
            const int r0 = 4 * (tid / ng), c0 = 4 * (tid % ng);
            T acc4[4][4] = {};
            for (int i = 0; i < np; ++i) {
                T g4[4], m4[4];
                load4(bufS + i * ldt + r0, g4);
                load4(bufM + i * ldt + c0, m4);
#pragma unroll
                for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                    for (int b_ = 0; b_ < 4; ++b_) acc4[a_][b_] += g4[a_] * m4[b_];
            }
#pragma unroll
            for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                for (int b_ = 0; b_ < 4; ++b_) bufA[(r0 + a_) * ldt + c0 + b_] = acc4[a_][b_];
        }
        __syncthreads();
        const int B = s.B;
        for (int b0 = 0; b0 < B; b0 += 64) {
            for (int idx = tid; idx < 64 * np; idx += nt) {   // C^T tile
                const int bl = idx >> lnp, j = idx & (np - 1);
                bufS[j * 68 + bl] = (b0 + bl < B && j < n) ? s.C[(size_t)(b0 + bl) * n + j] : T(0);
            }
            __syncthreads();
            const bool act = tid < 16 * ng;
            const int bg = tid / ng, ig = tid % ng;
            T z4[4][4] = {}, p4[4][4] = {};
            if (act) {
                for (int j = 0; j < np; ++j) {
                    T c4[4], g4[4], k4[4];
                    load4(bufS + j * 68 + 4 * bg, c4);
                    load4(bufG + j * ldt + 4 * ig, g4);
                    load4(bufA + j * ldt + 4 * ig, k4);
#pragma unroll
                    for (int a_ = 0; a_ < 4; ++a_)
#pragma unroll
                        for (int b_ = 0; b_ < 4; ++b_) {
                            z4[a_][b_] += c4[a_] * g4[b_];
                            p4[a_][b_] += c4[a_] * k4[b_];
                        }
                }
            }
            // Epilogue.  For chi = exp(-zeta t) with f' = -zeta chi, f'' = zeta^2 chi,
            // f''' = -zeta^3 chi, the radial chain contracts to
            //   grad chi = 2 f' p,  H v = 4 f'' p (p.v) + 2 f' q o v,
            //   grad lap chi = p o (8 f''' |p|^2 + 4 f'' sum q - 2 k^2 f' + 8 f'' q),
            // so the geometry (p, q, p.gU, q o gU) is computed once per
            // (nucleus, electron) and shared by that nucleus' Gaussians.
            T fl[4][3] = {}, fe[4][3] = {};
#pragma unroll
            for (int ii = 0; ii < 4; ++ii) {
                const int il = 4 * ig + ii;
                if (!act || il >= n) continue;
                const int i = sp * n + il;
                const T* gu = gU + 3 * i;
                int a_prev = -1;
                T t = 0, pv[3] = {0, 0, 0}, qv[3] = {0, 0, 0}, pp = 0, sq = 0, pg = 0, qg[3] = {0, 0, 0};
#pragma unroll
                for (int bb = 0; bb < 4; ++bb) {
                    const int b = b0 + 4 * bg + bb;
                    if (b >= B) continue;
                    const int a = b / G, g = b - a * G;
                    if (a != a_prev) {
                        a_prev = a;
                        T sd[3], cd[3];
                        disp_trig(et + 6 * i, s.ptrig + 6 * a, ell, sd, cd, t);
                        pp = 0; sq = 0; pg = 0;
#pragma unroll
                        for (int mu = 0; mu < 3; ++mu) {
                            pv[mu] = ell * sd[mu] * cd[mu];
                            qv[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
                            pp += pv[mu] * pv[mu];
                            sq += qv[mu];
                            pg += pv[mu] * gu[mu];
                            qg[mu] = qv[mu] * gu[mu];
                        }
                    }
                    const T z = s.zetat[g];
                    const T e = qexp(-z * t);
                    const T f1 = -z * e, f2 = z * z * e, f3 = -z * z * z * e;
                    const T A = T(8) * f3 * pp + T(4) * f2 * sq - T(2) * k2 * f1;
                    const T zb = z4[bb][ii], pb = p4[bb][ii];
                    const T g1 = T(2) * f1;
                    const T cp = pb * g1 + zb * T(4) * f2 * pg;   // p terms of pb grad chi + zb H gU
                    const T cq = zb * g1;                          // q o gU term of zb H gU
                    const T hz = T(0.5) * zb;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        // dl -= zb grad chi;  de += pb grad chi + zb (H gU + 1/2 grad lap chi)
                        fl[bb][mu] -= zb * g1 * pv[mu];
                        fe[bb][mu] += cp * pv[mu] + cq * qg[mu] + hz * pv[mu] * (A + T(8) * f2 * qv[mu]);
                    }
                }
            }
            // reduce over the ng threads that share these four basis functions
#pragma unroll
            for (int bb = 0; bb < 4; ++bb)
#pragma unroll
                for (int mu = 0; mu < 3; ++mu)
                    for (int o = 1; o < ng; o <<= 1) {
                        fl[bb][mu] += __shfl_xor_sync(0xffffffffu, fl[bb][mu], o);
                        fe[bb][mu] += __shfl_xor_sync(0xffffffffu, fe[bb][mu], o);
                    }
            if (act && ig == 0)
                for (int bb = 0; bb < 4; ++bb)
                    for (int mu = 0; mu < 3; ++mu) {
                        stage[(4 * bg + bb) * 6 + mu] = (double)fl[bb][mu];
                        stage[(4 * bg + bb) * 6 + 3 + mu] = (double)fe[bb][mu];
                    }
            __syncthreads();
            {   // one thread per nucleus of this tile sums its basis functions in order
                const int bend = (b0 + 64 < B) ? b0 + 64 : B;
                const int a_first = b0 / G, a_last = (bend - 1) / G;
                const int a = a_first + tid;
                if (a <= a_last) {
                    const int lo = (a * G > b0) ? a * G : b0, hi = ((a + 1) * G < bend) ? (a + 1) * G : bend;
                    for (int b = lo; b < hi; ++b)
                        for (int mu = 0; mu < 3; ++mu) {
                            f_dl[3 * a + mu] += stage[(b - b0) * 6 + mu];
                            f_de[3 * a + mu] += stage[(b - b0) * 6 + 3 + mu];
                        }
                }
            }
            __syncthreads();
        }
    }

    }

    // ---- P7: accumulate the sample
    const double EL = -0.5 * kin + vee + vep + vrec + s.vconst[0];
    const int N3 = 3 * N;
    const size_t stride = 3 + 9 * (size_t)N;
    double* aw = acc + (size_t)w * stride;
    bool bad = !isfinite(EL);
    for (int c = tid; c < N3; c += nt) {
        const double dl = f_dl[c] + (double)g_dl[c];
        const double de = (f_de[c] + (double)g_de[c]) + (f_dv[c] + (double)g_dv[c]) + s.dvpp[c];
        if (!isfinite(dl) || !isfinite(de)) bad = true;
        aw[3 + c] += dl;
        aw[3 + N3 + c] += EL * dl;
        aw[3 + 2 * N3 + c] += de;
        if (out_dl) { out_dl[(size_t)w * N3 + c] = dl; out_de[(size_t)w * N3 + c] = de; }
    }
    if constexpr (kSplit) {
        for (int idx = tid; idx < 9 * N; idx += nt) {
            const int i = idx / 9, c = idx - 9 * i;
            eg_out[(size_t)w * 9 * N + idx] = (float)(c < 6 ? et[6 * i + c] : gU[3 * i + c - 6]);
        }
        if (tid == 0) elw[w] = EL;
    }
    if (tid == 0) {
        aw[0] += 1.0; aw[1] += EL; aw[2] += EL * EL;
        if (s.vacc) s.vacc[w] += vee + vep + vrec + s.vconst[0];   // V_L, for the virial pressure
        if (out_el) { out_el[w] = EL; out_lnpsi[w] = logdet[2 * w] + logdet[2 * w + 1] + Utot; }
    }
    if (bad) raise_err(s.err, kErrNonfinite);
}

template <typename T>
size_t measure_smem_bytes(int N, int n, int nk, int mmax, bool split) {
    return MLayout<T>(N, n, nk, mmax, split).total;
}

template <typename T>
void launch_measure(const SysView<T>& s, const double* X, const T* D, const T* Lp, const T* Gt, const double* logdet,
                    double* acc, double* out_el, double* out_lnpsi, double* out_dl, double* out_de, float* kt_out,
                    float* eg_out, double* elw, float* rk_out, cudaStream_t st) {
    const bool split = sizeof(T) == 4 && kt_out != nullptr;
    const size_t smem = measure_smem_bytes<T>(s.N, s.n, s.nk, s.mmax, split);
    static bool attr_set[3] = {false, false, false};
    const int which = sizeof(T) == 8 ? 1 : (split ? 2 : 0);
    if constexpr (sizeof(T) == 4) {
        if (split) {
            if (!attr_set[which]) {
                cudaFuncSetAttribute(measure_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     227 * 1024);
                attr_set[which] = true;
            }
            measure_kernel<T, true><<<s.W, 256, smem, st>>>(s, s.mmax, X, D, Lp, Gt, logdet, acc, out_el, out_lnpsi,
                                                            out_dl, out_de, kt_out, eg_out, elw, rk_out);
            return;
        }
    }
    {
        if (!attr_set[which]) {
            cudaFuncSetAttribute(measure_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
            attr_set[which] = true;
        }
        measure_kernel<T, false><<<s.W, 256, smem, st>>>(s, s.mmax, X, D, Lp, Gt, logdet, acc, out_el, out_lnpsi,
                                                         out_dl, out_de, nullptr, nullptr, nullptr, nullptr);
    }
}

template size_t measure_smem_bytes<double>(int, int, int, int, bool);
template size_t measure_smem_bytes<float>(int, int, int, int, bool);
template void launch_measure<double>(const SysView<double>&, const double*, const double*, const double*,
                                     const double*, const double*, double*, double*, double*, double*, double*,
                                     float*, float*, double*, float*, cudaStream_t);
template void launch_measure<float>(const SysView<float>&, const double*, const float*, const float*, const float*,
                                    const double*, double*, double*, double*, double*, double*, float*, float*,
                                    double*, float*, cudaStream_t);

}  // namespace qmc
