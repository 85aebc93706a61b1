// k_adjoint_tc.cu -- tensor-core (tcgen05) form of the orbital (Pulay) part of
// the force estimators for the mixed-precision path.
//
// For one walker and one spin block (n electrons, orbitals j, inverse G = A^-1
// with A_ij = phi_j(r_i), K = G Y G with Y_ij = -1/2 lap phi_j(r_i) -
// grad_i U . grad phi_j(r_i)), the derivatives of ln det and of the kinetic
// part of E_L with respect to the nucleus a of basis function b are
//   d ln det / dR_a = - sum_{b in a} sum_i Z_bi grad chi_b(r_i),  Z = C G,
//   d E_kin / dR_a  = sum_{b in a} sum_i [P_bi grad chi_b + Z_bi (H chi_b gU_i + 1/2 grad lap chi_b)],  P = C K,
// (chain rule through phi_j = sum_b C_bj chi_b(r - R_a)).  Z and P are
// B x n contractions over the orbitals with a coefficient matrix shared by
// all walkers: they run on the tensor cores here, and the basis-derivative
// contraction is fused onto the accumulators in tensor memory.
//
// Layout.  The basis index b = a * G + g is split as (g, a): the MMA's M = 128
// rows are the nuclei a (zero rows beyond N), one accumulator block per
// Gaussian g.  Block g holds [Z | P] as N_mma = 2 * n16 columns (electron i of
// Z at column i, of P at n16 + i).  So the 128 TMEM lanes are the nuclei and
// a thread of the epilogue owns one nucleus for all G blocks: the geometry of
// a (nucleus, electron) pair is computed once and shared by its Gaussians, as
// in the SIMT epilogue, and the sum over the nucleus' basis functions is a
// register sum.
//
// Operands: A_g = C rows of Gaussian g (128 x n, K-major, prepared once per
// handle, two TF32 pieces, 128-byte swizzle) streamed from L2 by bulk copies
// into two shared buffers; B = [G^T ; K^T] (N_mma x n, K-major, two TF32
// pieces) built per walker-spin from the inverse and from K (written by the
// measure kernel).  Products A0 B0 + A0 B1 + A1 B0 (dropped A1 B1 below
// 2^-24 relative): FP32-level accuracy.
//
// One CTA per SM (persistent), 256 threads: warps w and w + 4 read TMEM lane
// quarter w % 4 and split the electrons in halves.  Every mbarrier wait is
// bounded; on a timeout the kernel records kErrTimeout, waits (bounded) for
// its copies in flight, frees tensor memory and returns.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace qmc {

namespace {
constexpr int kRowsA = 128;                 // MMA M (nuclei)
constexpr int kKc = 32;                     // orbitals per K chunk (128 bytes of FP32)
constexpr int kTileA = kRowsA * kKc * 4;    // 16 KB
constexpr int kPcs = 2;                     // TF32 pieces per operand
constexpr long long kWaitIter = 1ll << 26;

__host__ __device__ inline int adj_n16(int n) { return n <= 16 ? 16 : ((n + 15) / 16) * 16; }
__host__ __device__ inline int adj_nkc(int n) { return (n + kKc - 1) / kKc; }
__host__ __device__ inline size_t adj_abytes(int n) { return (size_t)kPcs * adj_nkc(n) * kTileA; }
__host__ __device__ inline size_t adj_bbytes(int n) { return (size_t)kPcs * adj_nkc(n) * 2 * adj_n16(n) * 128; }
__host__ __device__ inline uint32_t adj_tmem_cols(int n, int G) {
    uint32_t c = 32;
    while (c < (uint32_t)(G * 2 * adj_n16(n))) c <<= 1;
    return c;
}
inline size_t adj_smem(int n) {
    return 1024 + 2 * adj_abytes(n) + adj_bbytes(n) + sizeof(float) * 64 * 9 + sizeof(double) * 2 * 128 * 6;
}
}  // namespace

bool tc_adjoint_supported(int N, int n, int G) {
    return N <= kRowsA && n >= 1 && n <= 64 && G >= 1 && G <= 4 && G * 2 * adj_n16(n) <= 512 &&
           adj_smem(n) <= 227 * 1024;
}

size_t tc_adjoint_coeff_bytes(int n, int G) { return (size_t)G * adj_abytes(n); }

// A_g tiles: Gaussian g at g * abytes; within it piece p, chunk kc at
// (p * nkc + kc) * 16 KB; element (a, k) of a tile at sw128_off(a, k).
__global__ void prepare_adj_coeff_kernel(const float* __restrict__ C, int N, int G, int n, unsigned char* out) {
    const int nkc = adj_nkc(n);
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const int per_g = nkc * kRowsA * kKc;
    if (t >= G * per_g) return;
    const int g = t / per_g, rem = t - g * per_g;
    const int kc = rem / (kRowsA * kKc), rem2 = rem - kc * kRowsA * kKc;
    const int a = rem2 / kKc, k = rem2 - a * kKc;
    const int j = kc * kKc + k;
    const float x = (a < N && j < n) ? C[(size_t)(a * G + g) * n + j] : 0.f;
    float x0, x1;
    tc::split_tf32(x, x0, x1);
    unsigned char* base = out + (size_t)g * adj_abytes(n);
    *(float*)(base + (size_t)(0 * nkc + kc) * kTileA + tc::sw128_off(a, k)) = x0;
    *(float*)(base + (size_t)(1 * nkc + kc) * kTileA + tc::sw128_off(a, k)) = x1;
}

void prepare_tc_adjoint_coeff(const float* C, int N, int G, int n, void* ahat, cudaStream_t st) {
    const int tot = G * adj_nkc(n) * kRowsA * kKc;
    prepare_adj_coeff_kernel<<<(tot + 255) / 256, 256, 0, st>>>(C, N, G, n, (unsigned char*)ahat);
}

namespace {

// State of the A-operand pipeline, kept by the issuing thread only.
struct APipe {
    int held[2];      // Gaussian whose A tiles are (or are being) loaded into buffer b
    bool pend[2];     // a load into buffer b has not been waited for yet
    uint32_t phf[2];  // parity of the next phase of full[b]
    uint32_t phe[2];  // parity of the next phase of empty[b]
};

}  // namespace

__global__ void __launch_bounds__(256, 1)
    adjoint_tc_kernel(SysView<float> s, const unsigned char* __restrict__ ahat, const float* __restrict__ Gt,
                      const float* __restrict__ Kt, const float* __restrict__ eg, const double* __restrict__ elw,
                      double* __restrict__ acc, double* __restrict__ out_dl, double* __restrict__ out_de) {
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    const int N = s.N, n = s.n, G = s.G, W = s.W;
    const int n16 = adj_n16(n), NN = 2 * n16, nkc = adj_nkc(n), nK = nkc * kKc;
    const size_t abytes = adj_abytes(n), bbytes = adj_bbytes(n);
    unsigned char* sB = base + 2 * abytes;
    float* se = (float*)(sB + bbytes);                  // [n][9]: sin, cos (pi x / L), grad U of the spin's electrons
    double* stage = (double*)(se + 64 * 9);             // [2][128][6]
    __shared__ uint64_t full[2], empty[2], done;
    __shared__ uint32_t tbase;
    __shared__ int abort_flag;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t ncols = adj_tmem_cols(n, G);

    if (warp == 0) { tc::tmem_alloc(&tbase, ncols); tc::tmem_relinquish(); }
    if (tid == 0) {
        tc::mbar_init(&full[0], 1); tc::mbar_init(&full[1], 1);
        tc::mbar_init(&empty[0], 1); tc::mbar_init(&empty[1], 1);
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    const uint32_t idesc = tc::idesc_tf32(kRowsA, NN);

    // epilogue role: nucleus a = lane quarter row, electron half h
    const int quarter = warp & 3, half = warp >> 2;
    const int a = quarter * 32 + lane;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
    const float ell = (float)s.ell;
    const float twopiL = (float)(2.0 * kPi / s.L), k2 = twopiL * twopiL;
    float pt[6], zt[4];
#pragma unroll
    for (int c = 0; c < 6; ++c) pt[c] = a < N ? s.ptrig[6 * a + c] : 0.f;
#pragma unroll
    for (int g = 0; g < 4; ++g) zt[g] = g < G ? s.zetat[g] : 0.f;
    const int hn = n16 / 2;
    const int i_lo = half * hn, i_hi = (half + 1) * hn < n ? (half + 1) * hn : n;

    APipe ap{{-1, -1}, {false, false}, {0u, 0u}, {0u, 0u}};
    uint32_t ph_done = 0;
    bool ok = true;
    auto load_a = [&](int b, int g) {
        tc::mbar_arrive_expect_tx(&full[b], (uint32_t)abytes);
        tc::bulk_g2s(base + (size_t)b * abytes, ahat + (size_t)g * abytes, (uint32_t)abytes, &full[b]);
        ap.held[b] = g;
        ap.pend[b] = true;
    };
    if (tid == 0) {
        load_a(0, 0);
        if (G > 1) load_a(1, 1);
    }

    for (int w = blockIdx.x; w < W; w += gridDim.x) {
        double dfl[3] = {0.0, 0.0, 0.0}, dfe[3] = {0.0, 0.0, 0.0};
        for (int sp = 0; sp < 2; ++sp) {
            // ---- B operand [G^T ; K^T] (two TF32 pieces) and the electron data
            const float* gsrc = Gt + ((size_t)w * 2 + sp) * n * n;
            const float* ksrc = Kt + ((size_t)w * 2 + sp) * n * n;
            const int kg = nK / 4;
            for (int item = tid; item < NN * kg; item += blockDim.x) {
                const int r = item / kg, k0 = 4 * (item - r * kg);
                const int rr = r < n16 ? r : r - n16;
                const float* src = (r < n16 ? gsrc : ksrc) + (size_t)rr * n;
                float v[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = (rr < n && k0 + q < n) ? src[k0 + q] : 0.f;
                float4 x0, x1;
                tc::split_tf32(v[0], x0.x, x1.x);
                tc::split_tf32(v[1], x0.y, x1.y);
                tc::split_tf32(v[2], x0.z, x1.z);
                tc::split_tf32(v[3], x0.w, x1.w);
                const int kc = k0 / kKc;
                const uint32_t off = tc::sw128_off(r, k0 - kc * kKc);
                *(float4*)(sB + (size_t)(0 * nkc + kc) * NN * 128 + off) = x0;
                *(float4*)(sB + (size_t)(1 * nkc + kc) * NN * 128 + off) = x1;
            }
            for (int idx = tid; idx < 9 * n; idx += blockDim.x) se[idx] = eg[((size_t)w * N + sp * n) * 9 + idx];
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (abort_flag) break;

            // ---- MMAs (one thread): block g += A_g [G^T ; K^T]^T over the orbitals
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t b0 = tc::smem_addr(sB), bstep = (uint32_t)NN * 128;
                bool epend[2] = {false, false};
                for (int g = 0; g < G && ok; ++g) {
                    const int b = g & 1;
                    if (ap.held[b] != g) load_a(b, g);   // only if no refill was issued for it
                    if (ap.pend[b]) {
                        if (!tc::mbar_wait(&full[b], ap.phf[b], kWaitIter)) { ok = false; break; }
                        ap.phf[b] ^= 1u;
                        ap.pend[b] = false;
                    }
                    const uint32_t a0 = tc::smem_addr(base + (size_t)b * abytes);
                    const uint32_t d = tmem + (uint32_t)(g * NN);
                    for (int kc = 0; kc < nkc; ++kc)
#pragma unroll
                        for (int ks = 0; ks < kKc / 8; ++ks) {
                            const uint32_t o = 32u * ks;
                            const uint32_t aa = a0 + (uint32_t)kc * kTileA + o, bb = b0 + (uint32_t)kc * bstep + o;
                            const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
                            // A1 B0, A0 B1, A0 B0 (smallest first)
                            tc::mma_tf32(d, tc::desc_sw128(aa + (uint32_t)nkc * kTileA), tc::desc_sw128(bb), idesc,
                                         first);
                            tc::mma_tf32(d, tc::desc_sw128(aa), tc::desc_sw128(bb + (uint32_t)nkc * bstep), idesc, 1u);
                            tc::mma_tf32(d, tc::desc_sw128(aa), tc::desc_sw128(bb), idesc, 1u);
                        }
                    // buffer b will take A_{g+2}: signal when these MMAs have read it
                    if (g + 2 < G) { tc::mma_commit(&empty[b]); epend[b] = true; }
                    // refill the other buffer with A_{g+1} once the MMAs of g-1 are done,
                    // while the MMAs of g run
                    const int b1 = b ^ 1;
                    if (g + 1 < G && ap.held[b1] != g + 1) {
                        if (epend[b1]) {
                            if (!tc::mbar_wait(&empty[b1], ap.phe[b1], kWaitIter)) { ok = false; break; }
                            ap.phe[b1] ^= 1u;
                            epend[b1] = false;
                        }
                        load_a(b1, g + 1);
                    }
                }
                tc::mma_commit(&done);
                if (!ok) abort_flag = 1;
            }
            if (!tc::mbar_wait(&done, ph_done, kWaitIter)) ok = false;
            ph_done ^= 1u;
            tc::fence_after_sync();
            if (!ok) abort_flag = 1;
            // prefetch A_0, A_1 for the next walker-spin while the epilogue runs
            const bool more = sp == 0 || w + (int)gridDim.x < W;
            if (tid == 0 && ok && more)
                for (int b = 0; b < 2 && b < G; ++b)
                    if (ap.held[b] != b) load_a(b, b);

            // ---- epilogue: thread (a, half) over its electrons, 8 at a time
            float fl[3] = {0.f, 0.f, 0.f}, fe[3] = {0.f, 0.f, 0.f};
            for (int i0 = i_lo; i0 < i_hi; i0 += 8) {
                uint32_t zr[4][8], pr[4][8];
#pragma unroll
                for (int g = 0; g < 4; ++g)
                    if (g < G) {
                        tc::tmem_ld8(taddr + (uint32_t)(g * NN + i0), zr[g]);
                        tc::tmem_ld8(taddr + (uint32_t)(g * NN + n16 + i0), pr[g]);
                    }
                tc::tmem_wait_ld();
#pragma unroll
                for (int ii = 0; ii < 8; ++ii) {
                    const int i = i0 + ii;
                    if (i >= i_hi) break;
                    const float* e = se + 9 * i;
                    float sd[3], cd[3], pv[3], qv[3], t = 0.f, pp = 0.f, sq = 0.f, pg = 0.f;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        sd[mu] = e[mu] * pt[3 + mu] - e[3 + mu] * pt[mu];
                        cd[mu] = e[3 + mu] * pt[3 + mu] + e[mu] * pt[mu];
                        t += sd[mu] * sd[mu];
                    }
                    t *= ell * ell;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        pv[mu] = ell * sd[mu] * cd[mu];
                        qv[mu] = cd[mu] * cd[mu] - sd[mu] * sd[mu];
                        pp += pv[mu] * pv[mu];
                        sq += qv[mu];
                        pg += pv[mu] * e[6 + mu];
                    }
                    // chi = exp(-zeta t): f' = -zeta chi, f'' = zeta^2 chi, f''' = -zeta^3 chi;
                    // grad chi = 2 f' p, H v = 4 f'' p (p.v) + 2 f' q o v,
                    // grad lap chi = p o (8 f''' |p|^2 + 4 f'' sum q - 2 k^2 f' + 8 f'' q)
                    float cl = 0.f, cp = 0.f, cpq = 0.f;
#pragma unroll
                    for (int g = 0; g < 4; ++g)
                        if (g < G) {
                            const float z = zt[g];
                            const float ex = expf(-z * t);
                            const float f1 = -z * ex, f2 = z * z * ex, f3 = -z * z * z * ex;
                            const float A = 8.f * f3 * pp + 4.f * f2 * sq - 2.f * k2 * f1;
                            const float zb = __uint_as_float(zr[g][ii]), pb = __uint_as_float(pr[g][ii]);
                            cl += zb * f1;
                            cp += pb * 2.f * f1 + zb * (4.f * f2 * pg + 0.5f * A);
                            cpq += zb * 4.f * f2;
                        }
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        fl[mu] -= 2.f * cl * pv[mu];
                        fe[mu] += cp * pv[mu] + 2.f * cl * qv[mu] * e[6 + mu] + cpq * pv[mu] * qv[mu];
                    }
                }
            }
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) { dfl[mu] += (double)fl[mu]; dfe[mu] += (double)fe[mu]; }
            tc::fence_before_sync();
            __syncthreads();   // TMEM and the B operand are free for the next walker-spin
            if (abort_flag) break;
        }
        if (abort_flag) break;
        // ---- per nucleus: the two electron halves, in order, into the walker's sums
#pragma unroll
        for (int mu = 0; mu < 3; ++mu) {
            stage[((size_t)half * 128 + a) * 6 + mu] = dfl[mu];
            stage[((size_t)half * 128 + a) * 6 + 3 + mu] = dfe[mu];
        }
        __syncthreads();
        if (tid < N) {
            const int N3 = 3 * N;
            const double EL = elw[w];
            double* aw = acc + (size_t)w * (3 + 9 * (size_t)N);
            bool bad = false;
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                const int c = 3 * tid + mu;
                const double dl = stage[(size_t)tid * 6 + mu] + stage[((size_t)128 + tid) * 6 + mu];
                const double de = stage[(size_t)tid * 6 + 3 + mu] + stage[((size_t)128 + tid) * 6 + 3 + mu];
                if (!isfinite(dl) || !isfinite(de)) bad = true;
                aw[3 + c] += dl;
                aw[3 + N3 + c] += EL * dl;
                aw[3 + 2 * N3 + c] += de;
                if (out_dl) { out_dl[(size_t)w * N3 + c] += dl; out_de[(size_t)w * N3 + c] += de; }
            }
            if (bad) raise_err(s.err, kErrNonfinite);
        }
        __syncthreads();
    }

    // leave cleanly: no bulk copy of ours may still be in flight
    if (tid == 0) {
        if (!ok || abort_flag) raise_err(s.err, kErrTimeout);
        for (int b = 0; b < 2; ++b)
            if (ap.pend[b]) {
                tc::mbar_wait(&full[b], ap.phf[b], kWaitIter);
                ap.pend[b] = false;
            }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

void launch_adjoint_tc(const SysView<float>& s, const void* ahat, const float* Gt, const float* Kt, const float* eg,
                       const double* elw, double* acc, double* out_dl, double* out_de, cudaStream_t st) {
    static int sms[64] = {0};
    static size_t set_smem = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (sms[dev] == 0) cudaDeviceGetAttribute(&sms[dev], cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = adj_smem(s.n);
    if (smem > set_smem &&
        cudaFuncSetAttribute(adjoint_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess)
        set_smem = smem;
    const int grid = s.W < sms[dev] ? s.W : sms[dev];
    adjoint_tc_kernel<<<grid, 256, smem, st>>>(s, (const unsigned char*)ahat, Gt, Kt, eg, elw, acc, out_dl, out_de);
}

}  // namespace qmc
