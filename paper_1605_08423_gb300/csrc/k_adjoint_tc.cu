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
// One CTA per SM (persistent), 17 warps.  TMEM holds two slots of 256
// columns; a unit is two Gaussians of one walker-spin.  Warp 16 issues the
// MMAs of unit u + 1 into one slot while warps 0-15 run the epilogue of unit u
// from the other (warps w, w + 4, w + 8, w + 12 read lane quarter w % 4 and
// split the electrons in four parts); mbarriers hand the slots, the B operand
// and the A buffers back and forth.  Every mbarrier wait is bounded; after a
// timeout the kernel records kErrTimeout and every later wait returns at once,
// so all threads reach the exit (bulk copies in flight are waited for, TMEM is
// freed).
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
constexpr int kThreads = 512;               // 16 warps: 4 per TMEM lane quarter
constexpr int kParts = kThreads / 128;      // electron parts per nucleus
constexpr int kPreItems = 4;                // B items (4 orbitals) per thread: 128 rows x 16 / 512
constexpr int kPreElec = 2;                 // electron-data floats per thread: 9 x 64 / 512, rounded up

__host__ __device__ inline int adj_n16(int n) { return n <= 16 ? 16 : ((n + 15) / 16) * 16; }
__host__ __device__ inline int adj_nkc(int n) { return (n + kKc - 1) / kKc; }
__host__ __device__ inline size_t adj_abytes(int n) { return (size_t)kPcs * adj_nkc(n) * kTileA; }
__host__ __device__ inline size_t adj_bbytes(int n) { return (size_t)kPcs * adj_nkc(n) * 2 * adj_n16(n) * 128; }
inline size_t adj_smem(int n) {
    return 1024 + 2 * adj_abytes(n) + adj_bbytes(n) + sizeof(float) * 3 * 64 * 12 + sizeof(float) * kParts * 128 * 6;
}
}  // namespace

bool tc_adjoint_supported(int N, int n, int G) {
    return N <= kRowsA && n >= 1 && n <= 64 && G >= 1 && G <= 4 && 2 * 2 * adj_n16(n) <= 256 &&
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

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32, relative error of
// a few ulp; the exponents here stay above -126, so flushing subnormals to
// zero changes nothing).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// State of the A-operand pipeline, kept by the issuing thread only.
struct APipe {
    int held[2];      // Gaussian whose A tiles are (or are being) loaded into buffer b
    bool pend[2];     // a load into buffer b has not been waited for yet
    uint32_t phf[2];  // parity of the next phase of full[b]
    uint32_t phe[2];  // parity of the next phase of empty[b]
};

}  // namespace

// Registers of one thread's share of the next walker-spin's operands, loaded
// from HBM while the current epilogue runs.
struct BPrefetch {
    float4 v[kPreItems];   // four consecutive orbitals of one B row
    float e[kPreElec];     // electron data (sin, cos, grad U)
};

__global__ void __launch_bounds__(kThreads + 32, 1)
    adjoint_tc_kernel(SysView<float> s, const unsigned char* __restrict__ ahat, const float* __restrict__ Gt,
                      const float* __restrict__ Kt, const float* __restrict__ eg, const double* __restrict__ elw,
                      const float* __restrict__ frec, double* __restrict__ acc, double* __restrict__ out_dl,
                      double* __restrict__ out_de) {
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    const int N = s.N, n = s.n, G = s.G, W = s.W;
    const int n16 = adj_n16(n), NN = 2 * n16, nkc = adj_nkc(n), nK = nkc * kKc, kg = nK / 4;
    const int kg_shift = nkc == 1 ? 3 : 4;   // kg = 8 nkc is a power of two (nkc <= 2): no integer division
    const size_t abytes = adj_abytes(n), bbytes = adj_bbytes(n);
    unsigned char* sB = base + 2 * abytes;
    // electron data of walker-spin t in buffer t % 3: [64][12] sin, cos (pi x / L), grad U, pad.
    // Three buffers: t + 1 is written while some warps may still read t, and
    // t - 2 has been released by every warp (its TMEM slot was freed).
    float* se3 = (float*)(sB + bbytes);
    float* stage = se3 + 3 * 64 * 12;                   // [kParts][128][6]
    __shared__ uint64_t afull[2], aempty[2], bfull, mdone[2], sfree[2];
    __shared__ uint32_t tbase;
    __shared__ volatile int abort_flag;
    __shared__ float gcon[6][4];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const bool issuer = warp == kThreads / 32;          // warp 16 issues the MMAs; warps 0-15 do the rest
    const int H = (G + 1) / 2;                          // Gaussian pairs per walker-spin (TMEM units)

    if (warp == 0) { tc::tmem_alloc(&tbase, 512u); tc::tmem_relinquish(); }
    if (tid == 0) {
        tc::mbar_init(&afull[0], 1); tc::mbar_init(&afull[1], 1);
        tc::mbar_init(&aempty[0], 1); tc::mbar_init(&aempty[1], 1);
        tc::mbar_init(&bfull, kThreads / 32);
        tc::mbar_init(&mdone[0], 1); tc::mbar_init(&mdone[1], 1);
        tc::mbar_init(&sfree[0], kThreads / 32); tc::mbar_init(&sfree[1], kThreads / 32);
        tc::fence_mbar_init();
        abort_flag = 0;
    }
    for (int idx = tid; idx < 3 * 64 * 12; idx += blockDim.x) se3[idx] = 0.f;
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    const uint32_t idesc = tc::idesc_tf32(kRowsA, NN);
    // a wait that gives up after kWaitIter polls and then makes every later
    // wait of the CTA return at once (all threads run through to the exit)
    auto wait = [&](uint64_t* mb, uint32_t parity) {
        if (abort_flag) return;
        if (!tc::mbar_wait(mb, parity, kWaitIter)) abort_flag = 1;
    };

    // walker-spins t = 0, 1, ... of this CTA -> walker blockIdx.x + (t / 2) * gridDim.x, spin t % 2;
    // unit u = (t, hg): Gaussians 2 hg, 2 hg + 1 of walker-spin t in TMEM slot u % 2 (256 columns)
    const int nws = 2 * ((W - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x);
    const int nunits = nws * H;

    if (issuer) {
        // ---- MMA warp (one lane): A_g streamed by bulk copies through two
        // buffers (buffer g % 2), refilled one Gaussian group behind
        if (lane == 0) {
            APipe ap{{-1, -1}, {false, false}, {0u, 0u}, {0u, 0u}};
            bool epend[2] = {false, false};
            int nxt[2] = {-1, -1};
            auto load_a = [&](int b, int g) {
                tc::mbar_arrive_expect_tx(&afull[b], (uint32_t)abytes);
                tc::bulk_g2s(base + (size_t)b * abytes, ahat + (size_t)g * abytes, (uint32_t)abytes, &afull[b]);
                ap.held[b] = g;
                ap.pend[b] = true;
            };
            if (nunits > 0) {
                load_a(0, 0);
                if (G > 1) load_a(1, 1);
            }
            const uint32_t b0 = tc::smem_addr(sB), bstep = (uint32_t)NN * 128;
            for (int u = 0; u < nunits; ++u) {
                const int t = u / H, hg = u - t * H, slot = u & 1;
                if (hg == 0) wait(&bfull, (uint32_t)(t & 1));                       // B of walker-spin t
                if (u >= 2) wait(&sfree[slot], (uint32_t)(((u >> 1) - 1) & 1));    // slot read out
                tc::fence_after_sync();
                const int g_end = 2 * hg + 2 < G ? 2 * hg + 2 : G;
                for (int g = 2 * hg; g < g_end; ++g) {
                    const int b = g & 1;
                    if (ap.held[b] != g) {                  // no refill was issued for it
                        if (epend[b]) { wait(&aempty[b], ap.phe[b]); ap.phe[b] ^= 1u; epend[b] = false; }
                        load_a(b, g);
                    }
                    if (ap.pend[b]) { wait(&afull[b], ap.phf[b]); ap.phf[b] ^= 1u; ap.pend[b] = false; }
                    if (!abort_flag) {
                        const uint32_t a0 = tc::smem_addr(base + (size_t)b * abytes);
                        const uint32_t d = tmem + (uint32_t)(slot * 256 + (g - 2 * hg) * NN);
                        for (int kc = 0; kc < nkc; ++kc)
#pragma unroll
                            for (int ks = 0; ks < kKc / 8; ++ks) {
                                const uint32_t o = 32u * ks;
                                const uint32_t aa = a0 + (uint32_t)kc * kTileA + o, bb = b0 + (uint32_t)kc * bstep + o;
                                const uint32_t first = (kc == 0 && ks == 0) ? 0u : 1u;
                                // A1 B0, A0 B1, A0 B0 (smallest first)
                                tc::mma_tf32(d, tc::desc_sw128(aa + (uint32_t)nkc * kTileA), tc::desc_sw128(bb),
                                             idesc, first);
                                tc::mma_tf32(d, tc::desc_sw128(aa), tc::desc_sw128(bb + (uint32_t)nkc * bstep),
                                             idesc, 1u);
                                tc::mma_tf32(d, tc::desc_sw128(aa), tc::desc_sw128(bb), idesc, 1u);
                            }
                    }
                    // the next Gaussian buffer b takes (cyclically over walker-spins)
                    const int gn = g + 2 < G ? g + 2 : (g & 1);
                    if (gn != g) { tc::mma_commit(&aempty[b]); epend[b] = true; nxt[b] = gn; }
                    // refill the other buffer once its previous MMAs are done, while these run
                    const int b1 = b ^ 1;
                    if (epend[b1] && nxt[b1] >= 0 && ap.held[b1] != nxt[b1]) {
                        wait(&aempty[b1], ap.phe[b1]);
                        ap.phe[b1] ^= 1u;
                        epend[b1] = false;
                        load_a(b1, nxt[b1]);
                    }
                }
                tc::mma_commit(&mdone[slot]);
            }
            // no bulk copy of ours may still be in flight at exit
            for (int b = 0; b < 2; ++b)
                if (ap.pend[b]) tc::mbar_wait(&afull[b], ap.phf[b], kWaitIter);
        }
        __syncwarp();
    } else {
        // ---- epilogue warps: thread (nucleus a = TMEM lane, electron part)
        const int quarter = warp & 3, part = warp >> 2;
        const int a = quarter * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
        const float ell = (float)s.ell;
        const float twopiL = (float)(2.0 * kPi / s.L), k2 = twopiL * twopiL;
        // per-Gaussian constants of the epilogue (chi = exp(-zeta t) = 2^(-zl t)):
        //   sum_g zb f'   = -sum zeta (e zb),       4 f'' zb = 4 zeta^2 (e zb),
        //   pb 2 f' + zb (4 f'' p.gU + A/2) = -2 zeta (e pb) + (e zb) Q_g,
        //   Q_g = 4 zeta^2 p.gU - 4 zeta^3 |p|^2 + 2 zeta^2 sum q + k^2 zeta
        float pt[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) pt[c] = a < N ? s.ptrig[6 * a + c] : 0.f;
        if (tid < 4) {   // gcon[k][g]: zeta log2(e), zeta, 4 zeta^2, -4 zeta^3, 2 zeta^2, k^2 zeta
            const float z = tid < G ? s.zetat[tid] : 0.f;
            gcon[0][tid] = z * 1.4426950408889634f;
            gcon[1][tid] = z;
            gcon[2][tid] = 4.f * z * z;
            gcon[3][tid] = -4.f * z * z * z;
            gcon[4][tid] = 2.f * z * z;
            gcon[5][tid] = k2 * z;
        }
        asm volatile("bar.sync 1, %0;\n" ::"n"(kThreads) : "memory");   // epilogue warps only
        const int pn = n16 / kParts;
        const int i_lo = part * pn, i_hi = (part + 1) * pn < n ? (part + 1) * pn : n;
        const bool vec4 = (n & 3) == 0;
        auto prefetch = [&](int t, BPrefetch& pf) {
            const int w = blockIdx.x + (t >> 1) * gridDim.x, sp = t & 1;
            const float* gsrc = Gt + ((size_t)w * 2 + sp) * n * n;
            const float* ksrc = Kt + ((size_t)w * 2 + sp) * n * n;
#pragma unroll
            for (int k = 0; k < kPreItems; ++k) {
                const int item = tid + k * kThreads;
                const int r = item >> kg_shift, k0 = 4 * (item & (kg - 1));
                const int rr = r < n16 ? r : r - n16;
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (item < NN * kg && rr < n && k0 < n) {
                    const float* src = (r < n16 ? gsrc : ksrc) + (size_t)rr * n + k0;
                    if (vec4) {
                        v = *(const float4*)src;
                    } else {
                        v.x = src[0];
                        if (k0 + 1 < n) v.y = src[1];
                        if (k0 + 2 < n) v.z = src[2];
                        if (k0 + 3 < n) v.w = src[3];
                    }
                }
                pf.v[k] = v;
            }
            const float* esrc = eg + ((size_t)w * N + sp * n) * 9;
#pragma unroll
            for (int k = 0; k < kPreElec; ++k) {
                const int idx = tid + k * kThreads;
                pf.e[k] = idx < 9 * n ? esrc[idx] : 0.f;
            }
        };
        // B of walker-spin t into sB, its electron data into se buffer t % 3,
        // then this warp's arrival on bfull
        auto store = [&](const BPrefetch& pf, int t) {
#pragma unroll
            for (int k = 0; k < kPreItems; ++k) {
                const int item = tid + k * kThreads;
                if (item < NN * kg) {
                    const int r = item >> kg_shift, k0 = 4 * (item & (kg - 1));
                    float4 x0, x1;
                    tc::split_tf32(pf.v[k].x, x0.x, x1.x);
                    tc::split_tf32(pf.v[k].y, x0.y, x1.y);
                    tc::split_tf32(pf.v[k].z, x0.z, x1.z);
                    tc::split_tf32(pf.v[k].w, x0.w, x1.w);
                    const int kc = k0 / kKc;
                    const uint32_t off = tc::sw128_off(r, k0 - kc * kKc);
                    *(float4*)(sB + (size_t)(0 * nkc + kc) * NN * 128 + off) = x0;
                    *(float4*)(sB + (size_t)(1 * nkc + kc) * NN * 128 + off) = x1;
                }
            }
            float* se = se3 + (t % 3) * 64 * 12;
#pragma unroll
            for (int k = 0; k < kPreElec; ++k) {
                const int idx = tid + k * kThreads;
                if (idx < 9 * n) se[(idx / 9) * 12 + idx % 9] = pf.e[k];
            }
            tc::fence_proxy_async();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&bfull);
        };

        // (operands are loaded right before they are stored: 17 warps leave 96
        // registers a thread, too few to carry them through an epilogue)
        BPrefetch pf;
        if (nws > 0) {
            prefetch(0, pf);
            store(pf, 0);
        }
        float dfl[3] = {0.f, 0.f, 0.f}, dfe[3] = {0.f, 0.f, 0.f};   // this thread's share, both spins
        for (int u = 0; u < nunits; ++u) {
            const int t = u / H, hg = u - t * H, slot = u & 1;
            const int w = blockIdx.x + (t >> 1) * gridDim.x, sp = t & 1;
            wait(&mdone[slot], (uint32_t)((u >> 1) & 1));
            tc::fence_after_sync();
            if (hg == H - 1 && t + 1 < nws) {
                // every MMA of walker-spin t is done: B is free for t + 1
                prefetch(t + 1, pf);
                store(pf, t + 1);
            }
            if (sp == 0 && hg == 0)
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) { dfl[mu] = 0.f; dfe[mu] = 0.f; }
            const float* se = se3 + (t % 3) * 64 * 12;
            const int ng = (2 * hg + 2 < G ? 2 : G - 2 * hg);
            const uint32_t tslot = taddr + (uint32_t)(slot * 256);
            // this unit's two Gaussians' constants
            float uzl[2], ucz[2], uc4[2], uq3[2], uq2[2], uq0[2];
#pragma unroll
            for (int gg = 0; gg < 2; ++gg) {
                const int g = (2 * hg + gg) & 3;
                uzl[gg] = gcon[0][g]; ucz[gg] = gcon[1][g]; uc4[gg] = gcon[2][g];
                uq3[gg] = gcon[3][g]; uq2[gg] = gcon[4][g]; uq0[gg] = gcon[5][g];
            }
            for (int i0 = i_lo; i0 < i_hi; i0 += 4) {
                uint32_t zr[2][4], pr[2][4];
#pragma unroll
                for (int gg = 0; gg < 2; ++gg)
                    if (gg < ng) {
                        tc::tmem_ld4(tslot + (uint32_t)(gg * NN + i0), zr[gg]);
                        tc::tmem_ld4(tslot + (uint32_t)(gg * NN + n16 + i0), pr[gg]);
                    }
                tc::tmem_wait_ld();
                // electrons i0 .. i0 + 3 < n16: beyond n the accumulator columns
                // and the electron data are zero, so those terms vanish
#pragma unroll
                for (int ii = 0; ii < 4; ++ii) {
                    const int i = i0 + ii;
                    const float4 e0 = *(const float4*)(se + 12 * i), e1 = *(const float4*)(se + 12 * i + 4),
                                 e2 = *(const float4*)(se + 12 * i + 8);
                    const float sx[3] = {e0.x, e0.y, e0.z}, cx[3] = {e0.w, e1.x, e1.y}, gu[3] = {e1.z, e1.w, e2.x};
                    float pv[3], qv[3], t2 = 0.f, pp = 0.f, sq = 0.f, pg = 0.f;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        const float sd = sx[mu] * pt[3 + mu] - cx[mu] * pt[mu];
                        const float cd = cx[mu] * pt[3 + mu] + sx[mu] * pt[mu];
                        t2 += sd * sd;
                        pv[mu] = ell * sd * cd;
                        qv[mu] = cd * cd - sd * sd;
                    }
                    t2 *= ell * ell;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        pp += pv[mu] * pv[mu];
                        sq += qv[mu];
                        pg += pv[mu] * gu[mu];
                    }
                    // chi = exp(-zeta t): f' = -zeta chi, f'' = zeta^2 chi, f''' = -zeta^3 chi;
                    // grad chi = 2 f' p, H v = 4 f'' p (p.v) + 2 f' q o v,
                    // grad lap chi = p o (8 f''' |p|^2 + 4 f'' sum q - 2 k^2 f' + 8 f'' q)
                    float cl = 0.f, cp = 0.f, cpq = 0.f;
#pragma unroll
                    for (int gg = 0; gg < 2; ++gg)
                        if (gg < ng) {
                            const float ex = ex2_approx(-uzl[gg] * t2);
                            const float ez = ex * __uint_as_float(zr[gg][ii]), ep = ex * __uint_as_float(pr[gg][ii]);
                            const float Q = uc4[gg] * pg + uq3[gg] * pp + uq2[gg] * sq + uq0[gg];
                            cl -= ucz[gg] * ez;
                            cpq += uc4[gg] * ez;
                            cp += ez * Q - 2.f * ucz[gg] * ep;
                        }
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        dfl[mu] -= 2.f * cl * pv[mu];
                        dfe[mu] += cp * pv[mu] + 2.f * cl * qv[mu] * gu[mu] + cpq * pv[mu] * qv[mu];
                    }
                }
            }
            // this warp has read the slot out
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(&sfree[slot]);
            if (sp == 1 && hg == H - 1) {
                // ---- per nucleus: the electron parts, in order, into the walker's sums
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    stage[((size_t)part * 128 + a) * 6 + mu] = dfl[mu];
                    stage[((size_t)part * 128 + a) * 6 + 3 + mu] = dfe[mu];
                }
                asm volatile("bar.sync 1, %0;\n" ::"n"(kThreads) : "memory");   // epilogue warps only
                if (tid < N && !abort_flag) {
                    const int N3 = 3 * N;
                    const double EL = elw[w];
                    double* aw = acc + (size_t)w * (3 + 9 * (size_t)N) + 3 + 3 * tid;
                    double dl[3], de[3], s0[3], s1[3], s2[3];
                    bool bad = false;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {   // all loads first, then the updates
                        s0[mu] = aw[mu];
                        s1[mu] = aw[N3 + mu];
                        s2[mu] = aw[2 * N3 + mu];
                        float l = 0.f, e = 0.f;
#pragma unroll
                        for (int q = 0; q < kParts; ++q) {
                            l += stage[((size_t)q * 128 + tid) * 6 + mu];
                            e += stage[((size_t)q * 128 + tid) * 6 + 3 + mu];
                        }
                        // plus the reciprocal-space force of this sample (GEMM over walkers)
                        if (frec) e += frec[(size_t)w * N3 + 3 * tid + mu];
                        if (!isfinite(l) || !isfinite(e)) bad = true;
                        dl[mu] = (double)l;
                        de[mu] = (double)e;
                    }
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        aw[mu] = s0[mu] + dl[mu];
                        aw[N3 + mu] = s1[mu] + EL * dl[mu];
                        aw[2 * N3 + mu] = s2[mu] + de[mu];
                    }
                    if (out_dl)
#pragma unroll
                        for (int mu = 0; mu < 3; ++mu) {
                            out_dl[(size_t)w * N3 + 3 * tid + mu] += dl[mu];
                            out_de[(size_t)w * N3 + 3 * tid + mu] += de[mu];
                        }
                    if (bad) raise_err(s.err, kErrNonfinite);
                }
                asm volatile("bar.sync 1, %0;\n" ::"n"(kThreads) : "memory");   // stage free again
            }
        }
    }

    if (tid == 0 && abort_flag) raise_err(s.err, kErrTimeout);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512u);
}

void launch_adjoint_tc(const SysView<float>& s, const void* ahat, const float* Gt, const float* Kt, const float* eg,
                       const double* elw, const float* frec, double* acc, double* out_dl, double* out_de,
                       cudaStream_t st) {
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
    adjoint_tc_kernel<<<grid, kThreads + 32, smem, st>>>(s, (const unsigned char*)ahat, Gt, Kt, eg, elw, frec, acc, out_dl,
                                                         out_de);
}

}  // namespace qmc
