// common.cuh -- device helpers shared by the qmcmd kernels (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace qmc {

constexpr double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Counter words:
// {stream (walker or component), md step, index (move / electron), purpose}.
// ---------------------------------------------------------------------------
enum : uint32_t {
    kPropX = 0, kPropY = 1, kPropZ = 2, kAccept = 3,
    kInitX = 4, kInitY = 5, kInitZ = 6, kLangevin = 7
};

struct Key { uint32_t k0, k1; };

__host__ __device__ inline Key make_key(uint64_t seed) { return Key{(uint32_t)seed, (uint32_t)(seed >> 32)}; }

__device__ __forceinline__ uint4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, Key key) {
    uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
        k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// (0,1) uniforms: 53-bit for FP64, 24-bit for FP32.
__device__ __forceinline__ double u53(uint32_t a, uint32_t b) {
    const uint64_t k = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
    return ((double)k + 0.5) * (1.0 / 9007199254740992.0);
}
__device__ __forceinline__ float u24(uint32_t a) { return ((float)(a >> 8) + 0.5f) * (1.0f / 16777216.0f); }

// Standard normal from one Philox block (Box-Muller, cosine branch) and the
// acceptance uniform, in the precision of the form.
template <typename T> struct Draw;
template <> struct Draw<double> {
    __device__ static double normal(uint4 w) {
        const double a = u53(w.x, w.y), b = u53(w.z, w.w);
        return sqrt(-2.0 * log(a)) * cospi(2.0 * b);
    }
    __device__ static double uniform(uint4 w) { return u53(w.x, w.y); }
};
template <> struct Draw<float> {
    __device__ static float normal(uint4 w) {
        const float a = u24(w.x), b = u24(w.z);
        return sqrtf(-2.0f * logf(a)) * cospif(2.0f * b);
    }
    __device__ static float uniform(uint4 w) { return u24(w.x); }
};

// ---------------------------------------------------------------------------
// Math overloads for the two precision forms.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double qexp(double x) { return exp(x); }
__device__ __forceinline__ float qexp(float x) { return expf(x); }
__device__ __forceinline__ double qsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float qsqrt(float x) { return sqrtf(x); }
// Reciprocal and square root of the pair loops: IEEE in FP64; in FP32 the
// hardware approximations (a few ulp), well inside the FP32-level tolerance of
// the mixed form.
__device__ __forceinline__ double qrcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float qrcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double qsqrt_pair(double x) { return sqrt(x); }
__device__ __forceinline__ float qsqrt_pair(float x) { return x > 0.f ? x * rsqrtf(x) : 0.f; }
__device__ __forceinline__ double qerfc(double x) { return erfc(x); }
__device__ __forceinline__ float qerfc(float x) { return erfcf(x); }
__device__ __forceinline__ double qrint(double x) { return rint(x); }
__device__ __forceinline__ float qrint(float x) { return rintf(x); }
__device__ __forceinline__ void qsincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ void qsincospi(float x, float* s, float* c) { sincospif(x, s, c); }

// Four consecutive elements from 16-byte-aligned shared memory.
__device__ __forceinline__ void load4(const float* p, float o[4]) {
    const float4 v = *(const float4*)p;
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const double* p, double o[4]) {
    const double2 a = *(const double2*)p, b = *(const double2*)(p + 2);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block reduction (fixed tree) of one value per thread; result
// valid in all threads.  `scratch` holds >= 32 elements.
template <typename T>
__device__ T block_sum(T v, T* scratch) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    v = warp_sum(v);
    __syncthreads();
    if (lane == 0) scratch[wid] = v;
    __syncthreads();
    T t = (lane < nw) ? scratch[lane] : T(0);
    t = warp_sum(t);
    return t;
}

// Device error word bits.
enum : int { kErrNonfinite = 1, kErrSingular = 2, kErrNotPD = 4, kErrTimeout = 8 };

__device__ __forceinline__ void raise_err(int* err, int bit) { atomicOr(err, bit); }

// ---------------------------------------------------------------------------
// Read-only view of one system on the device (passed by value to kernels).
// ---------------------------------------------------------------------------
template <typename T> struct V2 { T x, y; };

template <typename T>
struct SysView {
    int N, n, G, B, W;
    int np;                 // n padded to a power of two >= 4 (tiled products)
    double L, ell;          // box side, L/pi
    double iL;              // 1/L
    double b_ee, b_ep, Zj;  // Jastrow parameters (Zj = e-n cusp amplitude)
    double kappa;           // Ewald splitting
    const double* zeta;     // [G]
    const T* zetat;         // [G] in the working precision
    const T* C;             // [B][n]
    const double* R;        // [N][3]
    const T* RT;            // [N][3] in the working precision
    const T* ptrig;         // [N][6]: sin(pi R/L) xyz, cos(pi R/L) xyz
    int nk;                 // half-space reciprocal vectors
    int mmax;               // reciprocal cutoff |m| <= mmax
    const int4* kvec;       // [nk] (mx, my, mz, 0)
    const double* kw;       // [nk] (4 pi / L^3) exp(-k^2/4 kappa^2) / k^2
    const double2* eikR;    // [N][nk] exp(i k.R_a)
    const V2<T>* eikRt;     // the same in the working precision
    const T* kwt;           // kw in the working precision
    const double2* rho_p;   // [nk] sum_a Z exp(i k.R_a)
    const double* vconst;   // [1] proton-proton real-space + self energy
    const double* dvpp;     // [3N] d(proton-proton real-space energy)/dR
    int* err;
    double* vacc;           // [W] per-walker sums of the sample's potential energy V_L (pressure), or null
    const double* fj;       // [N][N] e-e-n-n Jastrow coefficients (symmetric), or null
    const T* fjt;           // the same in the working precision, or null
    double zeta_j;          // their Gaussians' exponent
};

// Twisted boundary conditions: walker w samples twist t = w / Wk (K contiguous
// blocks); the spin-up orbitals carry theta_t, the spin-down ones -theta_t.
struct TwistView {
    int K, Wk;              // twists, walkers per twist
    int M;                  // Bloch-sum images per axis: m = -M..M around the nearest one
    const double* theta;    // [K][3]
    const double2* ph;      // [K][3][2M+1]: exp(i theta_mu m), m = -M..M
};

// Radial-function chain for f(t), t = |d|^2 with d the sin-periodised
// displacement.  Per component: s = sin(pi D/L), c = cos(pi D/L),
//   p = (L/pi) s c  (so dt/dx = 2p),  q = c^2 - s^2  (dp/dx = q),  dq/dx = -(2pi/L)^2 p.
// Given f', f'', f''' (derivatives in t) this returns the gradient, the
// Hessian (symmetric, xx yy zz xy xz yz), the Laplacian and grad(Laplacian).
template <typename T>
struct RadialDerivs {
    T g[3], h[6], lap, tl[3];
};
template <typename T>
__device__ __forceinline__ void radial_chain(const T p[3], const T q[3], T f1, T f2, T f3, T k2,
                                             RadialDerivs<T>& o) {
    const T pp = p[0] * p[0] + p[1] * p[1] + p[2] * p[2];
    const T sq = q[0] + q[1] + q[2];
#pragma unroll
    for (int m = 0; m < 3; ++m) o.g[m] = T(2) * f1 * p[m];
    o.h[0] = T(4) * f2 * p[0] * p[0] + T(2) * f1 * q[0];
    o.h[1] = T(4) * f2 * p[1] * p[1] + T(2) * f1 * q[1];
    o.h[2] = T(4) * f2 * p[2] * p[2] + T(2) * f1 * q[2];
    o.h[3] = T(4) * f2 * p[0] * p[1];
    o.h[4] = T(4) * f2 * p[0] * p[2];
    o.h[5] = T(4) * f2 * p[1] * p[2];
    o.lap = T(4) * f2 * pp + T(2) * f1 * sq;
#pragma unroll
    for (int m = 0; m < 3; ++m)
        o.tl[m] = p[m] * (T(8) * f3 * pp + T(8) * f2 * q[m] + T(4) * f2 * sq - T(2) * k2 * f1);
}

// H v for the packed symmetric Hessian.
template <typename T>
__device__ __forceinline__ void hess_mul(const T h[6], const T v[3], T out[3]) {
    out[0] = h[0] * v[0] + h[3] * v[1] + h[4] * v[2];
    out[1] = h[3] * v[0] + h[1] * v[1] + h[5] * v[2];
    out[2] = h[4] * v[0] + h[5] * v[1] + h[2] * v[2];
}

// Pade pair functions u(rho) and their rho-derivatives:
//   e-e: u = rho / (2 (1 + b rho))      (cusp +1/2)
//   e-n: u = -Zj rho / (1 + b rho)      (cusp -Zj)
template <typename T>
__device__ __forceinline__ void pade_ee(T b, T r, T& u, T& u1, T& u2) {
    const T q = T(1) + b * r, iq = qrcp(q);
    u = T(0.5) * r * iq; u1 = T(0.5) * iq * iq; u2 = -b * iq * iq * iq;
}
template <typename T>
__device__ __forceinline__ void pade_ep(T b, T Zj, T r, T& u, T& u1, T& u2, T& u3) {
    const T q = T(1) + b * r, iq = qrcp(q), iq2 = iq * iq;
    u = -Zj * r * iq; u1 = -Zj * iq2; u2 = T(2) * Zj * b * iq2 * iq; u3 = T(-6) * Zj * b * b * iq2 * iq2;
}

// From u(rho) derivatives to derivatives in t = rho^2.
template <typename T>
__device__ __forceinline__ void rho_to_t(T r, T u1, T u2, T u3, T& f1, T& f2, T& f3) {
    const T ir = qrcp(r), ir2 = ir * ir, ir3 = ir2 * ir;
    f1 = T(0.5) * u1 * ir;
    f2 = T(0.25) * (u2 * ir2 - u1 * ir3);
    f3 = T(0.125) * (u3 * ir3 - T(3) * u2 * ir2 * ir2 + T(3) * u1 * ir3 * ir2);
}

// Real-space Ewald pair sum over the images r0 + nL with |r0 + nL| < L of the
// minimum-image vector r0, phi(r) = erfc(kappa r)/r; optionally the gradient
// with respect to r0.
template <typename T>
__device__ __forceinline__ T ewald_real(T dx, T dy, T dz, T Lt, T kappa, T* grad, bool skip_min = false) {
    const T iL = T(1) / Lt;
    dx -= Lt * qrint(dx * iL); dy -= Lt * qrint(dy * iL); dz -= Lt * qrint(dz * iL);
    const T r0[3] = {dx, dy, dz};
    T sh[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) sh[m] = r0[m] >= T(0) ? -Lt : Lt;
    T v = 0;
    if (grad) grad[0] = grad[1] = grad[2] = 0;
    const T c2 = T(1.1283791670955126);  // 2 / sqrt(pi)
    // the (at most 8) candidate images inside the cutoff, compacted into a bit
    // mask so that a warp runs the erfc body only max(popcount) times
    unsigned mask = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const T a = r0[0] + ((c & 1) ? sh[0] : T(0));
        const T b = r0[1] + ((c & 2) ? sh[1] : T(0));
        const T e = r0[2] + ((c & 4) ? sh[2] : T(0));
        const T r2 = a * a + b * b + e * e;
        if (r2 < Lt * Lt && r2 > T(0)) mask |= 1u << c;
    }
    if (skip_min) mask &= ~1u;   // the minimum image is evaluated elsewhere
    while (mask) {
        const int c = __ffs(mask) - 1;
        mask &= mask - 1;
        const T a = r0[0] + ((c & 1) ? sh[0] : T(0));
        const T b = r0[1] + ((c & 2) ? sh[1] : T(0));
        const T e = r0[2] + ((c & 4) ? sh[2] : T(0));
        const T r2 = a * a + b * b + e * e;
        const T r = qsqrt(r2), ir = T(1) / r;
        const T ec = qerfc(kappa * r);
        v += ec * ir;
        if (grad) {
            const T dphi = -(ec * ir + c2 * kappa * qexp(-kappa * kappa * r2)) * ir;  // phi'(r)
            const T s = dphi * ir;
            grad[0] += s * a; grad[1] += s * b; grad[2] += s * e;
        }
    }
    return v;
}

// Position of the n-th (0-based) set bit of m (n < popc(m)), by halving.
__device__ __forceinline__ int nth_set_bit(unsigned m, int n) {
    int r = 0;
#pragma unroll
    for (int w = 16; w >= 1; w >>= 1) {
        const int cnt = __popc(m & ((1u << w) - 1u));
        if (n >= cnt) { n -= cnt; m >>= w; r += w; }
    }
    return r;
}

// Mixed form: real-space Ewald cutoff radius squared.  erfc(kappa r) at
// r = 0.8 L with kappa = 5 / L is 1.5e-8, below FP32 resolution of the pair
// sums, so images beyond it are dropped (the FP64 form keeps r < L).
constexpr float kRealCut2Mixed = 0.64f;

// erfc(x) for 0 <= x <= 4.1 in FP32 given e = exp(-x^2):
//   erfc(x) = e t P(t),  t = 1 / (1 + x / 2),
// P a degree-8 polynomial fitted (least squares, relative weight) to
// erfc(x) exp(x^2) / t; relative error 3.1e-7 in FP32 arithmetic (the fit and
// its check are in fit_erfc.py beside this package).
__device__ __forceinline__ float erfc_scaled_fit(float x, float e) {
    const float t = __fdividef(1.0f, 1.0f + 0.5f * x);
    float p = -4.711474106e-02f;
    p = p * t + 2.220349312e-01f;
    p = p * t - 3.470333517e-01f;
    p = p * t + 1.025151908e-01f;
    p = p * t + 1.076001227e-01f;
    p = p * t + 1.385983676e-01f;
    p = p * t + 2.617502213e-01f;
    p = p * t + 2.793540657e-01f;
    p = p * t + 2.822951376e-01f;
    return e * t * p;
}

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32, a few ulp)
__device__ __forceinline__ float ex2_fast(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Nearest integer of x (|x| < 2^22) in FP32 arithmetic: adding and removing
// 1.5 * 2^23 leaves no fraction bits, and round-to-nearest-even does the
// rounding (IEEE rounding of each addition; no reassociation in this build).
// The FMA pipe does it, where rintf's rounding instruction runs on the FP64
// pipe, a fraction of whose rate this part has.
__device__ __forceinline__ float rint_fma(float x) {
    const float m = 12582912.0f;   // 1.5 * 2^23
    return __fsub_rn(__fadd_rn(x, m), m);
}

// Mixed-form real-space Ewald sum of one pair: the images of the minimum-image
// vector inside the FP32-level cutoff (skip_min: leave out the minimum image),
// phi(r) = erfc(kappa r) / r and, when grad, its gradient added to grad.
// iL = 1/Lt and rc2 = kRealCut2Mixed Lt^2 come from the caller (loop invariants).
template <bool kGrad>
__device__ __forceinline__ float ewald_real_cut(float dx, float dy, float dz, bool skip_min, float Lt, float iL,
                                                float rc2, float kappa, float* grad) {
    dx -= Lt * rint_fma(dx * iL); dy -= Lt * rint_fma(dy * iL); dz -= Lt * rint_fma(dz * iL);
    // moving component m of the minimum image by L away from zero adds
    // L (L - 2 |d_m|) > 0 to r^2 (so only the minimum image can sit at r = 0)
    const float r0 = dx * dx + dy * dy + dz * dz;
    const float e0 = Lt * (Lt - 2.f * fabsf(dx)), e1 = Lt * (Lt - 2.f * fabsf(dy)), e2 = Lt * (Lt - 2.f * fabsf(dz));
    const float r1 = r0 + e0, r2_ = r0 + e1, r3 = r1 + e1, r4 = r0 + e2;
    unsigned mask = (r0 < rc2 && r0 > 0.f && !skip_min) ? 1u : 0u;
    mask |= (r1 < rc2 ? 2u : 0u) | (r2_ < rc2 ? 4u : 0u) | (r3 < rc2 ? 8u : 0u) | (r4 < rc2 ? 16u : 0u) |
            (r1 + e2 < rc2 ? 32u : 0u) | (r2_ + e2 < rc2 ? 64u : 0u) | (r3 + e2 < rc2 ? 128u : 0u);
    const float sx = dx >= 0.f ? -Lt : Lt, sy = dy >= 0.f ? -Lt : Lt, sz = dz >= 0.f ? -Lt : Lt;
    const float c2k = 1.1283791670955126f * kappa;      // 2 kappa / sqrt(pi)
    const float nk2 = -1.4426950408889634f * kappa * kappa;   // -kappa^2 log2(e)
    float v = 0.f;
    while (mask) {
        const int c = __ffs(mask) - 1;
        mask &= mask - 1;
        const float a = dx + ((c & 1) ? sx : 0.f), b = dy + ((c & 2) ? sy : 0.f), e = dz + ((c & 4) ? sz : 0.f);
        const float r2 = a * a + b * b + e * e;
        const float ir = rsqrtf(r2), r = r2 * ir;
        const float ex = ex2_fast(nk2 * r2);              // exp(-kappa^2 r^2)
        const float ec = erfc_scaled_fit(kappa * r, ex);
        v += ec * ir;
        if (kGrad) {
            const float s = -(ec * ir + c2k * ex) * ir * ir;   // phi'(r) / r
            grad[0] += s * a; grad[1] += s * b; grad[2] += s * e;
        }
    }
    return v;
}

template <typename T>
__device__ __forceinline__ void disp_trig(const T* ei, const T* pj, T ell, T sd[3], T cd[3], T& t) {
    t = 0;
#pragma unroll
    for (int mu = 0; mu < 3; ++mu) {
        sd[mu] = ei[mu] * pj[3 + mu] - ei[3 + mu] * pj[mu];
        cd[mu] = ei[3 + mu] * pj[3 + mu] + ei[mu] * pj[mu];
        t += sd[mu] * sd[mu];
    }
    t *= ell * ell;
}

}  // namespace qmc
