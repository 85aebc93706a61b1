// k_sweep.cu -- one Metropolis sweep of every walker (single-electron moves).
//
// One warp per walker.  For electron i (up block first, then down) with
// proposal r'_i (precomputed by the proposal kernel) and its orbital row
// phi'_j = phi_j(r'_i) (precomputed by the orbital kernel for the whole sweep):
//   ratio   R  = sum_j phi'_j G_{j,i}                     (determinant ratio)
//   Jastrow dU = sum_{j != i} [u_ee(r'_i,r_j) - u_ee(r_i,r_j)] + sum_a [u_en(r'_i,R_a) - u_en(r_i,R_a)]
//   accept if u < R^2 exp(2 dU)
// and on acceptance the Sherman-Morrison rank-1 update of the inverse of the
// spin block:  G' = G - G_{:,i} (phi'^T G - e_i^T) / R.
// The inverse of the moving spin block is staged in shared memory (row stride
// n+1: conflict-free per-lane rows) for the n moves of that block.
#include "common.cuh"
#include "kernels.cuh"

namespace qmc {

template <typename T>
struct SweepSmem {
    // Rows of the staged inverse are 16-byte vectors: nv = n rounded up to a
    // whole vector (zero padded), row stride ld = nv + one vector, so that the
    // 16-byte accesses of 8 consecutive lanes (one per row) hit distinct banks.
    static constexpr int VE = 16 / sizeof(T);   // elements per 16-byte vector
    __host__ __device__ static int nv(int n) { return (n + VE - 1) / VE * VE; }
    __host__ __device__ static int ld(int n) { return nv(n) + VE; }
    // per warp: G^T [n][ld], old row [nv], phi' [nv], trig [6N], and only with
    // the e-e-n-n Jastrow term (j34) three [N] vectors (sum over electrons of
    // chi_a, chi_a at the moving electron and at its proposal)
    __host__ __device__ static size_t warp_bytes(int N, int n, bool j34) {
        size_t b = ((size_t)n * ld(n) + 2 * (size_t)nv(n)) * sizeof(T);
        b += (size_t)(j34 ? 9 : 6) * N * sizeof(T);
        return (b + 15) & ~size_t(15);
    }
};

template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; };
template <> struct Vec16<double> { using type = double2; };

__device__ __forceinline__ float vdot(float4 a, float4 b, float acc[4]) {
    acc[0] += a.x * b.x; acc[1] += a.y * b.y; acc[2] += a.z * b.z; acc[3] += a.w * b.w;
    return 0.f;
}
__device__ __forceinline__ double vdot(double2 a, double2 b, double acc[4]) {
    acc[0] += a.x * b.x; acc[1] += a.y * b.y;
    return 0.0;
}
__device__ __forceinline__ float4 vaxpy(float4 g, float c, float4 r) {
    return make_float4(g.x - c * r.x, g.y - c * r.y, g.z - c * r.z, g.w - c * r.w);
}
__device__ __forceinline__ double2 vaxpy(double2 g, double c, double2 r) {
    return make_double2(g.x - c * r.x, g.y - c * r.y);
}

// exp(-zeta |d|^2) for the periodised displacement between two points given
// by their (sin, cos)(pi x / L) triples (e-e-n-n Jastrow orbital)
template <typename T>
__device__ __forceinline__ T jas_orbital(const T* a, const T* b, T ell, T zeta) {
    T t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const T sd = a[mu] * b[3 + mu] - a[3 + mu] * b[mu];
        t += sd * sd;
    }
    return qexp(-zeta * ell * ell * t);
}

template <typename T>
__device__ __forceinline__ T pair_dist(const T* a, const T* b, T ell) {
    // |d| for the periodised displacement between two points given by their
    // (sin, cos)(pi x / L) triples
    T t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        const T sd = a[mu] * b[3 + mu] - a[3 + mu] * b[mu];
        t += sd * sd;
    }
    return ell * qsqrt_pair(t);
}

template <typename T>
__global__ void __launch_bounds__(512) sweep_kernel(SysView<T> s, double* __restrict__ X, const double* __restrict__ Xp,
                                                    const T* __restrict__ ptp, const T* __restrict__ uacc,
                                                    const T* __restrict__ Phi,
                                                    T* __restrict__ Gt, unsigned long long* __restrict__ nacc) {
    extern __shared__ __align__(16) unsigned char smraw[];
    using V = typename Vec16<T>::type;
    constexpr int VE = SweepSmem<T>::VE;
    const int N = s.N, n = s.n, nv = SweepSmem<T>::nv(n), ld = SweepSmem<T>::ld(n), nvv = nv / VE;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    T* ptr_s = (T*)smraw;                                    // [N][6] proton trig
    size_t off = ((size_t)6 * N * sizeof(T) + 15) & ~size_t(15);
    const bool j34 = sizeof(T) == 8 && s.fjt != nullptr;
    unsigned char* mine = smraw + off + (size_t)warp * SweepSmem<T>::warp_bytes(N, n, j34);
    T* Gs = (T*)mine;
    T* rowb = Gs + (size_t)n * ld;
    T* phi = rowb + nv;
    T* et = phi + nv;
    T* c34 = et + 6 * N;     // [N] sum over electrons of chi_a (e-e-n-n Jastrow term, FP64 form)
    T* cho = c34 + N;        // [N] chi_a at the moving electron
    T* chn = cho + N;        // [N] chi_a at its proposal

    for (int idx = threadIdx.x; idx < 6 * N; idx += blockDim.x) ptr_s[idx] = s.ptrig[idx];
    __syncthreads();
    const int w = blockIdx.x * wpb + warp;
    if (w >= s.W) return;

    const T ell = (T)s.ell, bee = (T)s.b_ee, bep = (T)s.b_ep, Zj = (T)s.Zj;
    const double L = s.L;
    double* Xw = X + (size_t)w * 3 * N;   // positions stay in HBM; accepted moves are written through
    const double iL = 1.0 / L;
    for (int idx = lane; idx < 3 * N; idx += 32) {
        const int i = idx / 3, mu = idx % 3;
        T sn, cs;
        qsincospi((T)(Xw[idx] * iL), &sn, &cs);
        et[6 * i + mu] = sn;
        et[6 * i + 3 + mu] = cs;
    }
    __syncwarp();
    const T zj = (T)s.zeta_j;
    if (j34) {
        for (int a = lane; a < N; a += 32) {
            T c = 0;
            for (int j = 0; j < N; ++j) c += jas_orbital(et + 6 * j, ptr_s + 6 * a, ell, zj);
            c34[a] = c;
        }
        __syncwarp();
    }
    for (int j = n + lane; j < nv; j += 32) phi[j] = T(0);   // padding stays zero
    unsigned long long naccept = 0;
    // the next move's proposal trig, orbital row (n <= 64: two per lane) and
    // uniform are loaded one move ahead, so their HBM latency overlaps a move
    T pt_nx[6], ph_nx[2], u_nx;
    auto fetch = [&](int i) {
        const size_t row = (size_t)w * N + i;
#pragma unroll
        for (int mu = 0; mu < 6; ++mu) pt_nx[mu] = ptp[row * 6 + mu];
#pragma unroll
        for (int k = 0; k < 2; ++k) ph_nx[k] = (lane + 32 * k < n) ? Phi[row * n + lane + 32 * k] : T(0);
        u_nx = uacc[row];
    };
    fetch(0);
    for (int sp = 0; sp < 2; ++sp) {
        T* G = Gt + ((size_t)w * 2 + sp) * n * n;
        for (int idx = lane; idx < n * nv; idx += 32) {
            const int r = idx / nv, c = idx - r * nv;
            Gs[r * ld + c] = c < n ? G[r * n + c] : T(0);
        }
        __syncwarp();
        for (int il = 0; il < n; ++il) {
            const int i = sp * n + il;
            const size_t row = (size_t)w * N + i;
            T pt[6];
#pragma unroll
            for (int mu = 0; mu < 6; ++mu) pt[mu] = pt_nx[mu];
#pragma unroll
            for (int k = 0; k < 2; ++k)
                if (lane + 32 * k < n) phi[lane + 32 * k] = ph_nx[k];
            const T u = u_nx;
            if (i + 1 < N) fetch(i + 1);
            __syncwarp();
            T part = 0;
            for (int j = lane; j < n; j += 32) part += phi[j] * Gs[il * ld + j];
            const T ratio = warp_sum(part);
            T du = 0;
            const T* ei = et + 6 * i;
#pragma unroll 4
            for (int j = lane; j < N; j += 32) {
                const T* ej = et + 6 * j;
                T u1, u0, d1, d2;
                pade_ee(bee, pair_dist(pt, ej, ell), u1, d1, d2);
                pade_ee(bee, pair_dist(ei, ej, ell), u0, d1, d2);
                du += (j != i) ? u1 - u0 : T(0);
            }
#pragma unroll 4
            for (int a = lane; a < N; a += 32) {
                const T* pa = ptr_s + 6 * a;
                T u1, u0, d1, d2, d3;
                pade_ep(bep, Zj, pair_dist(pt, pa, ell), u1, d1, d2, d3);
                pade_ep(bep, Zj, pair_dist(ei, pa, ell), u0, d1, d2, d3);
                du += u1 - u0;
            }
            if (j34) {
                // e-e-n-n term: the pairs (i, j != i) change by
                // sum_a (chi_a(r'_i) - chi_a(r_i)) sum_b f_ab (c_b - chi_b(r_i))
                for (int a = lane; a < N; a += 32) {
                    chn[a] = jas_orbital(pt, ptr_s + 6 * a, ell, zj);
                    cho[a] = jas_orbital(ei, ptr_s + 6 * a, ell, zj);
                }
                __syncwarp();
                for (int a = lane; a < N; a += 32) {
                    // f is symmetric (checked at qmc_init): column a = row a,
                    // and the lanes' loads of a column element are consecutive
                    const T* fa = s.fjt + a;
                    T wa = 0;
                    for (int b = 0; b < N; ++b) wa += fa[(size_t)b * N] * (c34[b] - cho[b]);
                    du += (chn[a] - cho[a]) * wa;
                }
            }
            du = warp_sum(du);
            const T prob = ratio * ratio * qexp(T(2) * du);
            if (u < prob) {
                for (int j = lane; j < nv; j += 32) rowb[j] = Gs[il * ld + j];
                __syncwarp();
                const T ir = T(1) / ratio;
                const V* phv = (const V*)phi;
                const V* rbv = (const V*)rowb;
                for (int l = lane; l < n; l += 32) {
                    V* gl = (V*)(Gs + l * ld);
                    T w4[4] = {0, 0, 0, 0};   // partial sums per vector component: short chains
                    for (int jv = 0; jv < nvv; ++jv) vdot(phv[jv], gl[jv], w4);
                    const T wl = (w4[0] + w4[1]) + (w4[2] + w4[3]);
                    const T coef = (wl - (l == il ? T(1) : T(0))) * ir;
                    for (int jv = 0; jv < nvv; ++jv) gl[jv] = vaxpy(gl[jv], coef, rbv[jv]);
                }
                if (lane < 3) {
                    // FP64 form: wrap into [0, L) at once (as the reference chain does).
                    // Mixed form: keep the proposal as is (every function of the
                    // positions is periodic; the next proposal pass wraps), so no
                    // FP64 arithmetic runs per move.
                    const double xpl = Xp[row * 3 + lane];
                    if (sizeof(T) == 8) {
                        const double x = xpl - L * floor(xpl / L);
                        Xw[3 * i + lane] = x;
                        T sn, cs;
                        qsincospi((T)(x / L), &sn, &cs);
                        et[6 * i + lane] = sn;
                        et[6 * i + 3 + lane] = cs;
                    } else {
                        Xw[3 * i + lane] = xpl;
                        et[6 * i + lane] = pt[lane];
                        et[6 * i + 3 + lane] = pt[3 + lane];
                    }
                }
                if (j34)
                    for (int a = lane; a < N; a += 32) c34[a] += chn[a] - cho[a];
                ++naccept;
            }
            __syncwarp();
        }
        for (int idx = lane; idx < n * n; idx += 32) G[idx] = Gs[(idx / n) * ld + idx % n];
        (void)VE;
        __syncwarp();
    }
    if (lane == 0) nacc[w] += naccept;
}


// Mixed form, n <= 64: two warps per walker and the inverse in registers.
// Thread tw (0..63) of a walker owns row tw of the staged inverse (G^T row,
// zero-padded to 64 columns), so a move touches no shared-memory copy of G:
//   w_l = sum_j phi'_j G^T[l][j] for every row (the ratio is w_il),
//   on acceptance every thread applies G^T[l] -= (w_l - delta_{l,il}) / R * G^T[il].
// The Jastrow difference is split over the 64 threads (two e-e and two e-n
// partners each).  The two warps of a walker meet at a named barrier (one
// per walker of the CTA), once per move: before it every thread has put its
// share of the Jastrow difference, the owner of row il its row and w_il, and
// every thread its element of the next move's orbital row into shared
// buffers that alternate between moves; after it the acceptance decision and
// the update need nothing else.  Electron i's (sin, cos) after an accepted
// move are written by the thread that has i among its partners (tw = i mod
// 64), the only thread that reads them later in the sweep.  Same proposals, uniforms and acceptance rule as
// sweep_kernel; the mixed form keeps accepted proposals unwrapped.
// With the e-e-n-n Jastrow term (s.fjt set) the CTA stages f (FP32, N x N) in
// shared memory and each walker keeps c_a = sum_j chi_a(r_j); a move of
// electron i changes U by sum_a (chi_a(r'_i) - chi_a(r_i)) w_a with
// w_a = sum_b f_ab (c_b - chi_b(r_i)), each thread taking nuclei tw and
// tw + 64 (one more barrier per move to publish chi_b(r_i)).
constexpr int kSwWalkers = 4;   // walkers per CTA (8 warps)
constexpr int kSwRow = 64;      // register row length (n <= 64)

// Stride of one point's (sin, cos)(pi x / L) triples in sweep_reg_kernel's
// shared memory: 7 floats, so that the 32 lanes reading 32 consecutive points
// hit 32 distinct banks (a stride of 6 pairs them up).
constexpr int kTS = 7;

// Shared-memory floats per walker of sweep_reg_kernel: phi [2][64], row
// [2][64], red [2][8], trig [kTS N], V [N], and with the e-e-n-n term c [N]
// and chi(r_i) [N]; rounded up to whole 16-byte vectors (phi and the row are
// read as float4).
__host__ __device__ inline size_t sweep_reg_walker_floats(int N, bool j34) {
    return (4 * kSwRow + 16 + (kTS + 1) * (size_t)N + (j34 ? 2 * (size_t)N : 0) + 3) & ~size_t(3);
}

__global__ void __launch_bounds__(64 * kSwWalkers) sweep_reg_kernel(SysView<float> s, double* __restrict__ X,
                                                                  const double* __restrict__ Xp,
                                                                  const float* __restrict__ ptp,
                                                                  const float* __restrict__ uacc,
                                                                  const float* __restrict__ Phi,
                                                                  float* __restrict__ Gt,
                                                                  unsigned long long* __restrict__ nacc,
                                                                  float* __restrict__ Vep, int vep_init) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int N = s.N, n = s.n;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int p = warp >> 1, h = warp & 1, tw = tid & 63;
    const bool j34 = s.fjt != nullptr;
    float* ptr_s = (float*)smraw;                                       // [N][kTS] proton trig
    float* f_s = ptr_s + ((kTS * N + 3) & ~3);                            // [N][N] e-e-n-n coefficients (j34)
    float* mine = f_s + (j34 ? (size_t)N * N : 0) + (size_t)p * sweep_reg_walker_floats(N, j34);
    float* phi = mine;                  // [2][64] orbital row at the proposal (zero beyond n)
    float* rowb = phi + 2 * kSwRow;     // [2][64] row il of G^T
    float* red = rowb + 2 * kSwRow;     // [2][8] e-e du halves, ratio, new e-n sum halves
    float* et = red + 16;               // [N][kTS] (sin, cos)(pi x / L) of the current positions
    float* vj = et + kTS * N;           // [N] V_i = sum_a u_en(r_i, R_a) at the current positions
    float* c34 = vj + N;                // [N] sum_j chi_a(r_j) (j34)
    float* cho = c34 + N;               // [N] chi_a at the moving electron (j34)
    for (int idx = tid; idx < 6 * N; idx += blockDim.x) ptr_s[kTS * (idx / 6) + idx % 6] = s.ptrig[idx];
    if (j34)
        for (int idx = tid; idx < N * N; idx += blockDim.x) f_s[idx] = s.fjt[idx];
    __syncthreads();
    const int w = blockIdx.x * kSwWalkers + p;
    if (w >= s.W) return;              // whole walkers only: both of its warps leave
    auto bar = [&]() { asm volatile("bar.sync %0, 64;\n" ::"r"(1 + p) : "memory"); };

    const float ell = (float)s.ell, bee = (float)s.b_ee, bep = (float)s.b_ep, Zj = (float)s.Zj;
    const double iL = 1.0 / s.L;
    double* Xw = X + (size_t)w * 3 * N;
    for (int idx = tw; idx < 3 * N; idx += 64) {
        const int i = idx / 3, mu = idx % 3;
        float sn, cs;
        sincospif((float)(Xw[idx] * iL), &sn, &cs);
        et[kTS * i + mu] = sn;
        et[kTS * i + 3 + mu] = cs;
    }
    const float zj = (float)s.zeta_j;
    bar();   // et complete
    // V_i: computed from the positions in the first sweep of a call, carried
    // in Vep between the call's sweeps (an accepted move sets V_i to the sum
    // of its new e-n terms), so a move evaluates the e-n Pade terms only at
    // the proposal
    for (int i = tw; i < N; i += 64) {
        float v = 0.f;
        if (vep_init) {
            for (int a = 0; a < N; ++a) {
                float u0, d1, d2, d3;
                pade_ep(bep, Zj, pair_dist(et + kTS * i, ptr_s + kTS * a, ell), u0, d1, d2, d3);
                v += u0;
            }
        } else {
            v = Vep[(size_t)w * N + i];
        }
        vj[i] = v;
    }
    if (j34) {
        for (int a = tw; a < N; a += 64) {
            float c = 0.f;
            for (int j = 0; j < N; ++j) c += jas_orbital(et + kTS * j, ptr_s + kTS * a, ell, zj);
            c34[a] = c;
        }
    }
    // proposal trig and uniform of a row; the orbital value phi_tw of a row
    auto ld_pt = [&](int i, float* pt_, float& u_) {
        const size_t row = (size_t)w * N + i;
#pragma unroll
        for (int mu = 0; mu < 6; ++mu) pt_[mu] = ptp[row * 6 + mu];
        u_ = uacc[row];
    };
    auto ld_ph = [&](int i) { return tw < n ? Phi[((size_t)w * N + i) * n + tw] : 0.f; };
    unsigned long long naccept = 0;
    const bool vec4 = (n & 3) == 0;
    for (int sp = 0; sp < 2; ++sp) {
        float* G = Gt + ((size_t)w * 2 + sp) * n * n;
        float g[kSwRow];
#pragma unroll
        for (int jv = 0; jv < kSwRow / 4; ++jv) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            const int j = 4 * jv;
            if (tw < n && j < n) {
                if (vec4) {
                    v = *(const float4*)(G + (size_t)tw * n + j);
                } else {
                    v.x = G[(size_t)tw * n + j];
                    if (j + 1 < n) v.y = G[(size_t)tw * n + j + 1];
                    if (j + 2 < n) v.z = G[(size_t)tw * n + j + 2];
                    if (j + 3 < n) v.w = G[(size_t)tw * n + j + 3];
                }
            }
            g[j] = v.x; g[j + 1] = v.y; g[j + 2] = v.z; g[j + 3] = v.w;
        }
        const int i0 = sp * n;
        phi[tw] = ld_ph(i0);                      // the spin's first move: buffer 0
        float ph_nx = n > 1 ? ld_ph(i0 + 1) : 0.f;   // the next move's value, stored during this move
        float pt_nx[6], u_nx;
        ld_pt(i0, pt_nx, u_nx);
        bar();   // buffer 0 and the positions visible; the previous spin's reads done
        for (int il = 0; il < n; ++il) {
            const int i = i0 + il, buf = il & 1;
            const size_t row = (size_t)w * N + i;
            float pt[6];
#pragma unroll
            for (int mu = 0; mu < 6; ++mu) pt[mu] = pt_nx[mu];
            const float u = u_nx;
            const float ph_wr = ph_nx;
            if (il + 1 < n) ld_pt(i + 1, pt_nx, u_nx);
            if (il + 2 < n) ph_nx = ld_ph(i + 2);
            // w_l for this thread's row: four partial sums
            const float4* phv = (const float4*)(phi + buf * kSwRow);
            float a4[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int jv = 0; jv < kSwRow / 4; ++jv) {
                const float4 ph = phv[jv];
                a4[0] += ph.x * g[4 * jv]; a4[1] += ph.y * g[4 * jv + 1];
                a4[2] += ph.z * g[4 * jv + 2]; a4[3] += ph.w * g[4 * jv + 3];
            }
            const float wl = (a4[0] + a4[1]) + (a4[2] + a4[3]);
            // Jastrow difference: partners tw and tw + 64 (e-e: new minus old
            // pair terms; e-n: the new terms, less V_i after the barrier)
            float du = 0.f, vnew = 0.f;
            const float* ei = et + kTS * i;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const int j = tw + 64 * k;
                if (j < N) {
                    const float* ej = et + kTS * j;
                    float u1, u0, d1, d2;
                    pade_ee(bee, pair_dist(pt, ej, ell), u1, d1, d2);
                    pade_ee(bee, pair_dist(ei, ej, ell), u0, d1, d2);
                    du += (j != i) ? u1 - u0 : 0.f;
                    const float* pa = ptr_s + kTS * j;
                    float d3;
                    pade_ep(bep, Zj, pair_dist(pt, pa, ell), u1, d1, d2, d3);
                    vnew += u1;
                }
            }
            float chn_r[2] = {0.f, 0.f}, cho_r[2] = {0.f, 0.f};
            if (j34) {
                // chi_a at the electron and at its proposal for this thread's nuclei
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int a = tw + 64 * k;
                    if (a < N) {
                        chn_r[k] = jas_orbital(pt, ptr_s + kTS * a, ell, zj);
                        cho_r[k] = jas_orbital(ei, ptr_s + kTS * a, ell, zj);
                        cho[a] = cho_r[k];
                    }
                }
                bar();   // chi_b(r_i) of every nucleus and the previous move's c_b visible
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int a = tw + 64 * k;
                    if (a < N) {
                        float wa = 0.f;
                        for (int b = 0; b < N; ++b) wa += f_s[(size_t)b * N + a] * (c34[b] - cho[b]);
                        du += (chn_r[k] - cho_r[k]) * wa;
                    }
                }
            }
            du = warp_sum(du);
            vnew = warp_sum(vnew);
            float* rd = red + 8 * buf;
            float* rb = rowb + buf * kSwRow;
            if (lane == 0) { rd[h] = du; rd[4 + h] = vnew; }
            if (tw == il) {
                rd[2] = wl;
#pragma unroll
                for (int jv = 0; jv < kSwRow / 4; ++jv)
                    ((float4*)rb)[jv] = make_float4(g[4 * jv], g[4 * jv + 1], g[4 * jv + 2], g[4 * jv + 3]);
            }
            if (il + 1 < n) phi[(buf ^ 1) * kSwRow + tw] = ph_wr;
            const float v_old = vj[i];   // before the barrier: an accepted move rewrites it after
            bar();
            const float ratio = rd[2];
            const float vin = rd[4] + rd[5];
            const float dut = (rd[0] + rd[1]) + (vin - v_old);
            const float prob = ratio * ratio * expf(2.f * dut);
            if (u < prob) {
                const float coef = (wl - (tw == il ? 1.f : 0.f)) * __fdividef(1.f, ratio);
                const float4* rbv = (const float4*)rb;
#pragma unroll
                for (int jv = 0; jv < kSwRow / 4; ++jv) {
                    const float4 r4 = rbv[jv];
                    g[4 * jv] -= coef * r4.x; g[4 * jv + 1] -= coef * r4.y;
                    g[4 * jv + 2] -= coef * r4.z; g[4 * jv + 3] -= coef * r4.w;
                }
                // keep the proposal as is (periodic functions; the next proposal pass wraps)
                if (tw < 3) Xw[3 * i + tw] = Xp[row * 3 + tw];
                if (tw == (i & 63)) {
#pragma unroll
                    for (int mu = 0; mu < 6; ++mu) et[kTS * i + mu] = pt[mu];
                    vj[i] = vin;   // read again only in the next sweep
                }
                if (j34) {      // c_a of this thread's nuclei (read by others only after the next barrier)
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const int a = tw + 64 * k;
                        if (a < N) c34[a] += chn_r[k] - cho_r[k];
                    }
                }
                ++naccept;
            }
        }
        if (tw < n) {
#pragma unroll
            for (int j = 0; j < kSwRow; ++j)
                if (j < n) G[(size_t)tw * n + j] = g[j];
        }
    }
    bar();   // the last accepted moves' V_i
    for (int i = tw; i < N; i += 64) Vep[(size_t)w * N + i] = vj[i];
    if (tw == 0) nacc[w] += naccept;
}

template <typename T>
void launch_sweep(const SysView<T>& s, double* X, const double* Xp, const T* ptp, const T* uacc, const T* Phi, T* Gt,
                  unsigned long long* nacc, float* vep, bool vep_init, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (s.n <= kSwRow) {   // mixed form: inverse rows in registers
            const bool j34 = s.fjt != nullptr;
            const size_t smem = sizeof(float) * (((kTS * s.N + 3) & ~3) + (j34 ? (size_t)s.N * s.N : 0) +
                                                 kSwWalkers * sweep_reg_walker_floats(s.N, j34));
            static size_t attr = 0;
            if (smem > attr &&
                cudaFuncSetAttribute(sweep_reg_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) ==
                    cudaSuccess)
                attr = smem;
            sweep_reg_kernel<<<(s.W + kSwWalkers - 1) / kSwWalkers, 64 * kSwWalkers, smem, st>>>(
                *(const SysView<float>*)&s, X, Xp, (const float*)ptp, (const float*)uacc, (const float*)Phi,
                (float*)Gt, nacc, vep, vep_init ? 1 : 0);
            return;
        }
    }
    const size_t wb = SweepSmem<T>::warp_bytes(s.N, s.n, sizeof(T) == 8 && s.fjt != nullptr);
    const size_t head = ((size_t)6 * s.N * sizeof(T) + 15) & ~size_t(15);
    // as many walkers per CTA as the shared memory of one SM holds (one CTA per SM)
    int wpb = (int)((226 * 1024 - head) / wb);
    if (wpb > 16) wpb = 16;
    if (wpb < 1) wpb = 1;
    const size_t smem = head + wpb * wb;
    static bool attr_set[2] = {false, false};
    const int which = sizeof(T) == 8;
    if (!attr_set[which]) {
        cudaFuncSetAttribute(sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr_set[which] = true;
    }
    sweep_kernel<T><<<(s.W + wpb - 1) / wpb, 32 * wpb, smem, st>>>(s, X, Xp, ptp, uacc, Phi, Gt, nacc);
}

template void launch_sweep<double>(const SysView<double>&, double*, const double*, const double*, const double*,
                                   const double*, double*, unsigned long long*, float*, bool, cudaStream_t);
template void launch_sweep<float>(const SysView<float>&, double*, const double*, const float*, const float*,
                                  const float*, float*, unsigned long long*, float*, bool, cudaStream_t);

}  // namespace qmc
