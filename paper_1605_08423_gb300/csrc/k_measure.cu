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
    size_t xs, xt, et, gU, lU, Ui, gi, li, facc, rho, red, uni, total;
    __host__ __device__ MLayout(int N, int n, int nk, int mmax) {
        size_t o = 0;
        auto take = [&](size_t bytes) { size_t r = o; o = (o + bytes + 15) & ~size_t(15); return r; };
        xs = take(sizeof(double) * 3 * N);
        xt = take(sizeof(T) * 3 * N);
        et = take(sizeof(T) * 6 * N);
        gU = take(sizeof(T) * 3 * N);
        lU = take(sizeof(T) * N);
        Ui = take(sizeof(T) * N);
        gi = take(sizeof(T) * 3 * N);
        li = take(sizeof(T) * N);
        facc = take(sizeof(double) * 9 * N);
        rho = take(sizeof(double2) * nk);
        red = take(sizeof(double) * 64);
        const size_t etab = sizeof(V2<T>) * (size_t)N * 3 * (2 * mmax + 1);
        const size_t spin = sizeof(T) * 3 * (size_t)n * (n + 1);
        uni = take(etab > spin ? etab : spin);
        total = o;
    }
};

// One electron-proton pair: real-space Ewald value v = phi(r) summed over
// images and its gradient g with respect to the electron-proton vector; the
// e-n Jastrow contributions dl (to d ln psi/dR_a) and de (to dE_L/dR_a, given
// vv = g_i + grad_i U).  sd, cd: sin, cos(pi (x - R_a)/L) per component.
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
    const S r = qsqrt(t);
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

template <typename T>
__global__ void __launch_bounds__(256) measure_kernel(SysView<T> s, int mmax, const double* __restrict__ X,
                                                      const T* __restrict__ D, const T* __restrict__ Lp,
                                                      const T* __restrict__ Gt, const double* __restrict__ logdet,
                                                      double* __restrict__ acc, double* __restrict__ out_el,
                                                      double* __restrict__ out_lnpsi, double* __restrict__ out_dl,
                                                      double* __restrict__ out_de) {
    extern __shared__ __align__(16) unsigned char sm[];
    const int N = s.N, n = s.n, G = s.G, nk = s.nk;
    const MLayout<T> lay(N, n, nk, mmax);
    double* xs = (double*)(sm + lay.xs);
    T* xt = (T*)(sm + lay.xt);
    T* et = (T*)(sm + lay.et);
    T* gU = (T*)(sm + lay.gU);
    T* lU = (T*)(sm + lay.lU);
    T* Ui = (T*)(sm + lay.Ui);
    T* gi = (T*)(sm + lay.gi);
    T* li = (T*)(sm + lay.li);
    double* f_dl = (double*)(sm + lay.facc);
    double* f_de = f_dl + 3 * N;
    double* f_dv = f_de + 3 * N;
    double2* rho = (double2*)(sm + lay.rho);
    double* red = (double*)(sm + lay.red);
    unsigned char* uni = sm + lay.uni;

    const int w = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
    const double L = s.L;
    const T ell = (T)s.ell, bee = (T)s.b_ee, bep = (T)s.b_ep, Zj = (T)s.Zj, kap = (T)s.kappa;
    const T twopiL = T(2.0 * kPi / L), k2 = twopiL * twopiL;
    const double Zn = 1.0;  // proton charge

    // ---- P0: positions and their (sin, cos)(pi x / L)
    for (int idx = tid; idx < 3 * N; idx += nt) {
        const double x = X[(size_t)w * 3 * N + idx];
        xs[idx] = x;
        xt[idx] = (T)x;
        T sn, cs;
        qsincospi((T)(x / L), &sn, &cs);
        et[6 * (idx / 3) + idx % 3] = sn;
        et[6 * (idx / 3) + 3 + idx % 3] = cs;
    }
    for (int idx = tid; idx < 9 * N; idx += nt) f_dl[idx] = 0.0;
    __syncthreads();

    // ---- P1: Jastrow gradient / Laplacian per electron, U partial sums
    for (int i = tid; i < N; i += nt) {
        T g[3] = {0, 0, 0}, lp = 0, ui = 0;
        const T* ei = et + 6 * i;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            T sd[3], cd[3], t;
            disp_trig(ei, et + 6 * j, ell, sd, cd, t);
            const T r = qsqrt(t);
            T u, u1, u2, f1, f2, f3;
            pade_ee(bee, r, u, u1, u2);
            rho_to_t(r, u1, u2, T(0), f1, f2, f3);
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
        for (int a = 0; a < N; ++a) {
            T sd[3], cd[3], t;
            disp_trig(ei, s.ptrig + 6 * a, ell, sd, cd, t);
            const T r = qsqrt(t);
            T u, u1, u2, u3, f1, f2, f3;
            pade_ep(bep, Zj, r, u, u1, u2, u3);
            rho_to_t(r, u1, u2, T(0), f1, f2, f3);
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
        gU[3 * i] = g[0]; gU[3 * i + 1] = g[1]; gU[3 * i + 2] = g[2];
        lU[i] = lp; Ui[i] = ui;
    }

    // ---- P2: g_i = sum_j D_ij G_ji, l_i = sum_j Lp_ij G_ji
    for (int i = tid; i < N; i += nt) {
        const int sp = i / n, il = i - sp * n;
        const T* grow = Gt + (((size_t)w * 2 + sp) * n + il) * n;
        const T* drow = D + ((size_t)w * N + i) * 3 * n;
        const T* lrow = Lp + ((size_t)w * N + i) * n;
        T g0 = 0, g1 = 0, g2 = 0, l = 0;
        for (int j = 0; j < n; ++j) {
            const T gj = grow[j];
            g0 += drow[j] * gj; g1 += drow[n + j] * gj; g2 += drow[2 * n + j] * gj;
            l += lrow[j] * gj;
        }
        gi[3 * i] = g0; gi[3 * i + 1] = g1; gi[3 * i + 2] = g2; li[i] = l;
    }
    __syncthreads();

    // ---- P3: kinetic energy and U
    double kin_p = 0.0, u_p = 0.0;
    for (int i = tid; i < N; i += nt) {
        T g2 = 0, t2 = 0;
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            const T g = gi[3 * i + mu], t = g + gU[3 * i + mu];
            g2 += g * g; t2 += t * t;
        }
        kin_p += (double)(li[i] - g2 + lU[i] + t2);
        u_p += (double)Ui[i];
    }
    const double kin = block_sum(kin_p, red);
    const double Utot = block_sum(u_p, red + 32);

    // ---- P4a: electron-electron real-space Ewald
    double vee_p = 0.0;
    const T Lt = (T)L;
    for (int i = tid; i < N; i += nt) {
        T v = 0;
        for (int j = i + 1; j < N; ++j)
            v += ewald_real<T>(xt[3 * i] - xt[3 * j], xt[3 * i + 1] - xt[3 * j + 1], xt[3 * i + 2] - xt[3 * j + 2], Lt,
                               kap, nullptr);
        vee_p += (double)v;
    }
    // ---- P4b: electron-proton pairs (warp per proton, lanes over electrons): the
    // real-space Ewald energy and its R-gradient (Hellmann-Feynman) together with
    // the e-n Jastrow terms of d ln psi/dR and dE_L/dR.  In the mixed form, pairs
    // closer than 0.3 bohr are evaluated and summed in FP64: there the 1/r^2
    // Coulomb force and the 1/r^2 part of grad lap u_en cancel (cusp condition),
    // and FP32 rounding of either term would survive the cancellation.
    double vep_p = 0.0;
    for (int a = warp; a < N; a += nw) {
        T v = 0, gv[3] = {0, 0, 0}, dl[3] = {0, 0, 0}, de[3] = {0, 0, 0};
        double vC = 0, gC[3] = {0, 0, 0}, dlC[3] = {0, 0, 0}, deC[3] = {0, 0, 0};
        const T* pa = s.ptrig + 6 * a;
        for (int i = lane; i < N; i += 32) {
            const double dx = xs[3 * i] - s.R[3 * a], dy = xs[3 * i + 1] - s.R[3 * a + 1],
                         dz = xs[3 * i + 2] - s.R[3 * a + 2];
            T sd[3], cd[3], t;
            disp_trig(et + 6 * i, pa, ell, sd, cd, t);
            if (sizeof(T) == 4 && t < T(0.09)) {
                double sdd[3], cdd[3], vv[3], pv, pg[3], pl[3], pe[3];
                sincospi(dx / L, &sdd[0], &cdd[0]);
                sincospi(dy / L, &sdd[1], &cdd[1]);
                sincospi(dz / L, &sdd[2], &cdd[2]);
                for (int mu = 0; mu < 3; ++mu) vv[mu] = (double)gi[3 * i + mu] + (double)gU[3 * i + mu];
                ep_pair<double>(sdd, cdd, s.ell, (double)k2, s.b_ep, s.Zj, dx, dy, dz, L, s.kappa, vv, pv, pg, pl, pe);
                vC += pv;
                for (int mu = 0; mu < 3; ++mu) { gC[mu] += pg[mu]; dlC[mu] += pl[mu]; deC[mu] += pe[mu]; }
            } else {
                T vv[3], pv, pg[3], pl[3], pe[3];
                for (int mu = 0; mu < 3; ++mu) vv[mu] = gi[3 * i + mu] + gU[3 * i + mu];
                const T* ra = s.RT + 3 * a;
                ep_pair<T>(sd, cd, ell, k2, bep, Zj, xt[3 * i] - ra[0], xt[3 * i + 1] - ra[1], xt[3 * i + 2] - ra[2],
                           Lt, kap, vv, pv, pg, pl, pe);
                v += pv;
                for (int mu = 0; mu < 3; ++mu) { gv[mu] += pg[mu]; dl[mu] += pl[mu]; de[mu] += pe[mu]; }
            }
        }
        v = warp_sum(v); vC = warp_sum(vC);
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            gv[mu] = warp_sum(gv[mu]); dl[mu] = warp_sum(dl[mu]); de[mu] = warp_sum(de[mu]);
            gC[mu] = warp_sum(gC[mu]); dlC[mu] = warp_sum(dlC[mu]); deC[mu] = warp_sum(deC[mu]);
        }
        if (lane == 0) {
            vep_p += -Zn * ((double)v + vC);
            for (int mu = 0; mu < 3; ++mu) {
                f_dv[3 * a + mu] += Zn * ((double)gv[mu] + gC[mu]);
                f_dl[3 * a + mu] += (double)dl[mu] + dlC[mu];
                f_de[3 * a + mu] += (double)de[mu] + deC[mu];
            }
        }
    }
    // ---- P4c: reciprocal space: electron structure factor from per-electron phase tables
    V2<T>* etab = (V2<T>*)uni;
    const int nm = 2 * mmax + 1;
    for (int idx = tid; idx < 3 * N; idx += nt) {
        T sn, cs;
        qsincospi((T)(2.0 * xs[idx] / L), &sn, &cs);
        V2<T>* e = etab + (size_t)idx * nm;
        V2<T> cur{T(1), T(0)};
        e[mmax] = cur;
        for (int m = 1; m <= mmax; ++m) {
            cur = V2<T>{cur.x * cs - cur.y * sn, cur.x * sn + cur.y * cs};
            e[mmax + m] = cur;
            e[mmax - m] = V2<T>{cur.x, -cur.y};
        }
    }
    __syncthreads();
    double vrec_p = 0.0;
    for (int k = tid; k < nk; k += nt) {
        const int4 m = s.kvec[k];
        T re = 0, im = 0;
        for (int i = 0; i < N; ++i) {
            const V2<T> a = etab[(3 * i) * nm + m.x + mmax], b = etab[(3 * i + 1) * nm + m.y + mmax],
                        c = etab[(3 * i + 2) * nm + m.z + mmax];
            const T abx = a.x * b.x - a.y * b.y, aby = a.x * b.y + a.y * b.x;
            re += abx * c.x - aby * c.y;
            im += abx * c.y + aby * c.x;
        }
        const double2 rp = s.rho_p[k];
        const double rr = rp.x - (double)re, ri = rp.y - (double)im;   // electrons carry -1
        rho[k] = make_double2(rr, ri);
        vrec_p += s.kw[k] * (rr * rr + ri * ri);
    }
    __syncthreads();
    // ---- P4d: reciprocal-space force on the protons (warp per proton)
    for (int a = warp; a < N; a += nw) {
        T gx = 0, gy = 0, gz = 0;
        for (int k = lane; k < nk; k += 32) {
            const V2<T> e = s.eikRt[(size_t)a * nk + k];
            const double2 rd = rho[k];
            const T c = T(2) * (T)Zn * s.kwt[k] * ((T)rd.y * e.x - (T)rd.x * e.y);
            const int4 m = s.kvec[k];
            gx += c * twopiL * (T)m.x; gy += c * twopiL * (T)m.y; gz += c * twopiL * (T)m.z;
        }
        gx = warp_sum(gx); gy = warp_sum(gy); gz = warp_sum(gz);
        if (lane == 0) { f_dv[3 * a] += (double)gx; f_dv[3 * a + 1] += (double)gy; f_dv[3 * a + 2] += (double)gz; }
    }
    const double vee = block_sum(vee_p, red);
    const double vep = block_sum(vep_p, red + 32);
    const double vrec = block_sum(vrec_p, red);

    __syncthreads();

    // ---- P6: orbital (Pulay) terms, one spin block at a time
    const int ld = n + 1;
    T* Gs = (T*)uni;
    T* Ys = Gs + (size_t)n * ld;
    T* Ks = Ys + (size_t)n * ld;
    for (int sp = 0; sp < 2; ++sp) {
        const T* Gsp = Gt + ((size_t)w * 2 + sp) * n * n;
        for (int idx = tid; idx < n * n; idx += nt) {
            const int il = idx / n, j = idx - il * n, i = sp * n + il;
            Gs[il * ld + j] = Gsp[idx];
            const size_t rr = (size_t)w * N + i;
            const T* dr = D + rr * 3 * n;
            Ys[il * ld + j] = T(-0.5) * Lp[rr * n + j] -
                              (gU[3 * i] * dr[j] + gU[3 * i + 1] * dr[n + j] + gU[3 * i + 2] * dr[2 * n + j]);
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += nt) {          // M1 = Y G  ->  Ks
            const int il = idx / n, ip = idx - il * n;
            T acc_ = 0;
            for (int j = 0; j < n; ++j) acc_ += Ys[il * ld + j] * Gs[ip * ld + j];
            Ks[il * ld + ip] = acc_;
        }
        __syncthreads();
        for (int idx = tid; idx < n * n; idx += nt) {          // (G M1)^T -> Ys : Kt[ip][j] = sum_i G_ji M1[i][ip]
            const int ip = idx / n, j = idx - ip * n;
            T acc_ = 0;
            for (int i = 0; i < n; ++i) acc_ += Gs[i * ld + j] * Ks[i * ld + ip];
            Ys[ip * ld + j] = acc_;
        }
        __syncthreads();
        for (int a = warp; a < N; a += nw) {
            T dl[3] = {0, 0, 0}, de[3] = {0, 0, 0};
            const T* pa = s.ptrig + 6 * a;
            for (int il = lane; il < n; il += 32) {
                const int i = sp * n + il;
                T sd[3], cd[3], t, p[3], q[3];
                disp_trig(et + 6 * i, pa, ell, sd, cd, t);
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) { p[mu] = ell * sd[mu] * cd[mu]; q[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu]; }
                const T* gu = gU + 3 * i;
                const T* grow = Gs + il * ld;
                const T* krow = Ys + il * ld;
                for (int g = 0; g < G; ++g) {
                    const T* cb = s.C + ((size_t)a * G + g) * n;
                    T zb = 0, pb = 0;
                    for (int j = 0; j < n; ++j) {
                        const T c = cb[j];
                        zb += c * grow[j];
                        pb += c * krow[j];
                    }
                    const T z = (T)s.zeta[g];
                    const T e = qexp(-z * t);
                    RadialDerivs<T> rd;
                    radial_chain(p, q, -z * e, z * z * e, -z * z * z * e, k2, rd);
                    T hv[3];
                    hess_mul(rd.h, gu, hv);
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        dl[mu] -= zb * rd.g[mu];
                        de[mu] += pb * rd.g[mu] + zb * (hv[mu] + T(0.5) * rd.tl[mu]);
                    }
                }
            }
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) { dl[mu] = warp_sum(dl[mu]); de[mu] = warp_sum(de[mu]); }
            if (lane == 0)
                for (int mu = 0; mu < 3; ++mu) { f_dl[3 * a + mu] += (double)dl[mu]; f_de[3 * a + mu] += (double)de[mu]; }
        }
        __syncthreads();
    }

    // ---- P7: accumulate the sample
    const double EL = -0.5 * kin + vee + vep + vrec + s.vconst[0];
    const int N3 = 3 * N;
    const size_t stride = 3 + 9 * (size_t)N;
    double* aw = acc + (size_t)w * stride;
    bool bad = !isfinite(EL);
    for (int c = tid; c < N3; c += nt) {
        const double dl = f_dl[c];
        const double de = f_de[c] + f_dv[c] + s.dvpp[c];
        if (!isfinite(dl) || !isfinite(de)) bad = true;
        aw[3 + c] += dl;
        aw[3 + N3 + c] += EL * dl;
        aw[3 + 2 * N3 + c] += de;
        if (out_dl) { out_dl[(size_t)w * N3 + c] = dl; out_de[(size_t)w * N3 + c] = de; }
    }
    if (tid == 0) {
        aw[0] += 1.0; aw[1] += EL; aw[2] += EL * EL;
        if (out_el) { out_el[w] = EL; out_lnpsi[w] = logdet[2 * w] + logdet[2 * w + 1] + Utot; }
    }
    if (bad) raise_err(s.err, kErrNonfinite);
}

template <typename T>
size_t measure_smem_bytes(int N, int n, int nk, int mmax) {
    return MLayout<T>(N, n, nk, mmax).total;
}

template <typename T>
void launch_measure(const SysView<T>& s, const double* X, const T* D, const T* Lp, const T* Gt, const double* logdet,
                    double* acc, double* out_el, double* out_lnpsi, double* out_dl, double* out_de, cudaStream_t st) {
    const size_t smem = measure_smem_bytes<T>(s.N, s.n, s.nk, s.mmax);
    static bool attr_set[2] = {false, false};
    const int which = sizeof(T) == 8;
    if (!attr_set[which]) {
        cudaFuncSetAttribute(measure_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_set[which] = true;
    }
    measure_kernel<T><<<s.W, 256, smem, st>>>(s, s.mmax, X, D, Lp, Gt, logdet, acc, out_el, out_lnpsi, out_dl, out_de);
}

template size_t measure_smem_bytes<double>(int, int, int, int);
template size_t measure_smem_bytes<float>(int, int, int, int);
template void launch_measure<double>(const SysView<double>&, const double*, const double*, const double*,
                                     const double*, const double*, double*, double*, double*, double*, double*,
                                     cudaStream_t);
template void launch_measure<float>(const SysView<float>&, const double*, const float*, const float*, const float*,
                                    const double*, double*, double*, double*, double*, double*, cudaStream_t);

}  // namespace qmc
