// k_orbitals_tc.cu -- tensor-core (tcgen05) form of the walker-batched
// molecular-orbital contraction for the mixed-precision path.
//
//   phi_j(r) = sum_b C[b][j] chi_b(r)   (and grad, Laplacian for Q = 4)
//
// A CTA owns 128 rows (electron positions).  For each chunk of 32 basis
// functions the threads evaluate the periodised Gaussians (value, or
// gradient and Laplacian) of the 128 rows straight into shared memory, in the
// K-major 128-byte-swizzled layout the tensor core reads, split into P exact
// TF32 pieces.  One thread then issues, per quantity, the piece products with
// i + j <= P - 1 (tcgen05.mma kind::tf32), accumulating in tensor memory
// (FP32).  With P = 2 (x = x0 + x1, representation error 2^-24 |x|):
//   D += A1 B0 + A0 B1 + A0 B0,
// the dropped A1 B1 is below 2^-22 relative: FP32-level, which is what the
// results are stored in.  (P = 3, six products, reaches 2^-33.)
// B = C^T chunk, prepared once per handle in the same swizzled layout.
//
// Accumulation per chunk.  The tensor core's FP32 accumulation over all B
// basis functions of a row is the largest error of the contraction (the
// diffuse Gaussians make every nucleus contribute, and the Slater inverse
// amplifies the error of the orbital values and derivatives alike).  So chunk
// 0 accumulates into the running total T and every later chunk into a fresh
// TMEM block C (reset by its first product), which the threads then add into
// T (tcgen05.ld of C and T, FP32 add, tcgen05.st to T): a chunk's 32 products
// are summed by the tensor core, the 16 chunk sums at N = 128 by the threads
// with round-to-nearest.  After the last chunk T goes TMEM -> registers ->
// shared -> HBM.
#include "common.cuh"
#include "kernels.cuh"
#include "tc.cuh"

namespace qmc {

// 2^x by the hardware approximation (PTX ex2.approx.ftz.f32; a few ulp, the
// exponents here stay far above the subnormal range)
__device__ __forceinline__ float tc_ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

namespace {
constexpr int kRows = 128;     // MMA M
constexpr int kKc = 32;        // basis functions per chunk (128 bytes of FP32 per row)
constexpr int kTileA = kRows * kKc * 4;   // 16 KB
}

// pieces used per operand: orbital values (Slater rows) and their derivatives
constexpr int kPiecesVal = 2;
constexpr int kPiecesDer = 2;
constexpr int kPieces = kPiecesVal > kPiecesDer ? kPiecesVal : kPiecesDer;   // prepared coefficient pieces

__host__ __device__ inline int tc_nm(int n) { return n <= 16 ? 16 : ((n + 15) / 16) * 16; }

size_t tc_coeff_bytes(int B, int n) {
    const int nch = (B + kKc - 1) / kKc;
    return (size_t)nch * kPieces * tc_nm(n) * 128;
}

bool tc_orbitals_supported(int n, int B) { (void)B; return n >= 1 && n <= 64; }

// C^T chunks, kPieces TF32 pieces, swizzled: chunk c at c * kPieces * NM * 128
// bytes, piece p at p * NM * 128.
__global__ void prepare_coeff_kernel(const float* __restrict__ C, int B, int n, int NM, unsigned char* chat) {
    const int nch = (B + kKc - 1) / kKc;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nch * NM * kKc) return;
    const int c = t / (NM * kKc), rem = t - c * NM * kKc, j = rem / kKc, k = rem - j * kKc;
    const int b = c * kKc + k;
    const float x = (b < B && j < n) ? C[(size_t)b * n + j] : 0.f;
    float xp[3];
    if (kPieces == 3) tc::split3_tf32(x, xp[0], xp[1], xp[2]);
    else tc::split_tf32(x, xp[0], xp[1]);
    unsigned char* base = chat + (size_t)c * kPieces * NM * 128;
    for (int p = 0; p < kPieces; ++p) *(float*)(base + (size_t)p * NM * 128 + tc::sw128_off(j, k)) = xp[p];
}

void prepare_tc_coeff(const float* C, int B, int n, void* chat, cudaStream_t st) {
    const int NM = tc_nm(n), nch = (B + kKc - 1) / kKc;
    const int tot = nch * NM * kKc;
    prepare_coeff_kernel<<<(tot + 255) / 256, 256, 0, st>>>(C, B, n, NM, (unsigned char*)chat);
}

// Q = 1: values (Slater rows / proposals).  Q = 4: d/dx, d/dy, d/dz and the
// Laplacian (local energy; the values are not needed there).
template <int Q, int P>
__global__ void __launch_bounds__(Q == 1 ? 256 : 544, Q == 1 ? 4 : 1)
    orbitals_tc_kernel(SysView<float> s, const unsigned char* __restrict__ chat, const double* __restrict__ pos,
                       int nrows, int NM, float* __restrict__ val, float* __restrict__ grad, float* __restrict__ lap) {
    extern __shared__ unsigned char smraw[];
    unsigned char* base = (unsigned char*)((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~uintptr_t(1023));
    unsigned char* sA = base;                                    // [Q][piece] tiles of 16 KB
    unsigned char* sB = base + (size_t)Q * P * kTileA;           // [buffer][piece] tiles of NM * 128 bytes
    constexpr int kBbuf = Q == 4 ? 2 : 1;                        // B buffers
    float* ptr_s = (float*)(sB + (size_t)kBbuf * P * NM * 128);  // [N][6] proton trig
    __shared__ float rtrig[kRows][6];
    __shared__ float zs[16];   // zeta_g and zeta_g log2(e), g < 8
    __shared__ uint64_t mbarh[2], fullh[2], bbar, freeh0, foldab[2];
    __shared__ uint32_t tbase;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nt = blockDim.x;
    const int row0 = blockIdx.x * kRows;
    const int n = s.n, B = s.B, G = s.G, N = s.N;
    const float ell = (float)s.ell;
    constexpr uint32_t kSub = (Q == 1) ? 64u : 256u;       // columns of one accumulator block (>= Q * NM)
    constexpr uint32_t kCols = 2 * kSub;                   // running total T at 0, chunk block C at kSub
    // Add the chunk block C into the running total T: warps split by TMEM lane
    // quarter (warp % 4) and 16-column groups; warp-collective.
    auto fold_chunk = [&](int nwarps) {
        const int quarter = warp & 3, cg = warp >> 2, ngr = nwarps >> 2;
        const uint32_t tl = tbase + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = cg * 16; c0 < Q * NM; c0 += 16 * ngr) {
            float cv[16], tv[16];
            tc::tmem_ld16(tl + kSub + (uint32_t)c0, cv);
            tc::tmem_ld16(tl + (uint32_t)c0, tv);
#pragma unroll
            for (int j = 0; j < 16; ++j) tv[j] += cv[j];
            tc::tmem_st16(tl + (uint32_t)c0, tv);
        }
    };

    if (warp == 0) { tc::tmem_alloc(&tbase, kCols); tc::tmem_relinquish(); }
    if (tid == 0) {
        tc::mbar_init(&mbarh[0], 1); tc::mbar_init(&mbarh[1], 1);
        tc::mbar_init(&fullh[0], 16); tc::mbar_init(&fullh[1], 16);   // one arrival per producer warp
        tc::mbar_init(&bbar, 1);                                         // B chunk bulk copies (value kernel)
        tc::mbar_init(&freeh0, 1);                                       // derivative kernel: half 0 read
        tc::mbar_init(&foldab[0], 16); tc::mbar_init(&foldab[1], 16);   // derivative kernel: folds done
        tc::fence_mbar_init();
    }
    for (int idx = tid; idx < kRows * 3; idx += nt) {
        const int r = idx / 3, mu = idx % 3, row = row0 + r;
        float sn = 0.f, cs = 1.f;
        if (row < nrows) sincospif((float)(pos[(size_t)row * 3 + mu] * (1.0 / s.L)), &sn, &cs);
        rtrig[r][mu] = sn;
        rtrig[r][3 + mu] = cs;
    }
    for (int idx = tid; idx < 6 * N; idx += nt) ptr_s[idx] = s.ptrig[idx];
    if (tid < 8) {
        const float z = tid < G ? s.zetat[tid] : 0.f;
        zs[tid] = z;
        zs[8 + tid] = z * 1.4426950408889634f;
    }
    const int gshift = (G & (G - 1)) == 0 ? __ffs(G) - 1 : -1;
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tbase;
    const uint32_t idesc = tc::idesc_tf32(kRows, NM);
    const int nch = (B + kKc - 1) / kKc;
    const size_t chunk_bytes = (size_t)kPieces * NM * 128;
    bool ok = true;

    if constexpr (Q == 4 && P == 2) {
    // Derivative kernel (Q = 4).  A chunk of 32 basis functions is produced in
    // two halves (basis 0-15 and 16-31 = k-steps 0-1 and 2-3, disjoint 16-byte
    // pieces of every A row) by warps 0-15, which arrive on fullh[h]; warp 16
    // issues the MMAs.  Each later chunk accumulates into the chunk block C,
    // split by quantity group: C_a (d/dx, d/dy) and C_b (d/dz, Laplacian).  The
    // MMAs of chunk c run in four steps
    //   S1 half 0 into C_a, S2 half 0 into C_b (commit freeh0),
    //   S3 half 1 into C_a (commit doneA = mbarh[0]), S4 half 1 into C_b (commit doneB = mbarh[1]).
    // Producer order for chunk c >= 1: half 0 of c (once freeh0 of c - 1 says
    // S1, S2 of c - 1 have read half 0), fold C_a of c - 1 into T (after doneA),
    // fold C_b of c - 1 (after doneB), store the B chunk c + 1 into the buffer
    // chunk c - 1 used, half 1 of c.  S1 of chunk c also waits for the fold of
    // C_a of c - 1 (folda), S2 for that of C_b (foldb).  So the production of
    // half 0 runs under S3, S4 of the previous chunk and the folds under S1 of
    // this one: the tensor core does not wait for a fold.  Every barrier
    // completes once per chunk (folds: once per chunk >= 1) and cannot complete
    // again before its waiters have seen the previous completion (each
    // completion needs work that follows that wait), so parity waits are
    // unambiguous.
    constexpr int kProd = 512;                 // producer threads
    constexpr int kBv4 = 2;                    // P * NM * 8 <= 1024 vectors over 512 producers
    const int nbv4 = P * NM * 8;
    const size_t bbytes = (size_t)P * NM * 128;
    uint4 bnx[kBv4];
    auto fetch_b4 = [&](int c) {
        const uint4* src = (const uint4*)(chat + (size_t)c * chunk_bytes);
#pragma unroll
        for (int v = 0; v < kBv4; ++v) {
            const int idx = tid + v * kProd;
            if (idx < nbv4) bnx[v] = src[idx];
        }
    };
    auto store_b4 = [&](int buf) {
        uint4* dst = (uint4*)(sB + (size_t)buf * bbytes);
#pragma unroll
        for (int v = 0; v < kBv4; ++v) {
            const int idx = tid + v * kProd;
            if (idx < nbv4) dst[idx] = bnx[v];
        }
    };
    // C of quantity group grp added into T (columns grp * 2 NM .. + 2 NM) by
    // the 16 producer warps: warp % 4 picks the TMEM lane quarter, warp / 4 a
    // 16-column group; all loads of a warp are issued before one wait, the
    // stores before one wait.
    auto fold_group = [&](int grp) {
        const int quarter = warp & 3, cg = warp >> 2;
        const uint32_t tl = tbase + ((uint32_t)(quarter * 32) << 16);
        const int c_lo = grp * 2 * NM, c_hi = c_lo + 2 * NM;
        for (int c0 = c_lo + cg * 16; c0 < c_hi; c0 += 64) {
            float cv[16], tv[16];
            tc::tmem_ld16(tl + kSub + (uint32_t)c0, cv);
            tc::tmem_ld16(tl + (uint32_t)c0, tv);
#pragma unroll
            for (int j = 0; j < 16; ++j) tv[j] += cv[j];
            tc::tmem_st16(tl + (uint32_t)c0, tv);
        }
    };
    // one item = (row, 4 consecutive basis functions of half h of chunk c);
    // the displacement to a nucleus is computed once for its Gaussians.  Warp
    // wp owns rows 8 wp .. 8 wp + 7 (one swizzle block); each quarter-warp (the
    // 8 lanes of one phase of a 16-byte store) takes rows q and q + 4 of the
    // block, whose swizzled 16-byte pieces of this half lie in opposite halves
    // of the 128-byte row: the phase covers all 32 banks once.
    auto produce = [&](int c, int h) {
        const int wl = tid & 31;
        const int r = 8 * (tid >> 5) + ((wl >> 3) & 3) + 4 * ((wl >> 2) & 1), k0 = 16 * h + 4 * (wl & 3);
        float v[Q][4];
        if (G == 4) {
            // 4 Gaussians per nucleus: the item is the 4 Gaussians of nucleus
            // (c * 32 + k0) / 4, one geometry and four exponentials
            const int a = (c * kKc + k0) >> 2;
            const bool on = a < N && row0 + r < nrows;
            const float* pt = ptr_s + 6 * (on ? a : 0);
            float t = 0.f, pp = 0.f, sq = 0.f, pv[3];
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                const float sx = rtrig[r][mu], cx = rtrig[r][3 + mu];
                const float sd = sx * pt[3 + mu] - cx * pt[mu];
                const float cd = cx * pt[3 + mu] + sx * pt[mu];
                t += sd * sd;
                pv[mu] = ell * sd * cd;
                pp += pv[mu] * pv[mu];
                sq += cd * cd - sd * sd;
            }
            t *= ell * ell;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float z = zs[kk];
                const float e = tc_ex2(-zs[8 + kk] * t);
                const float f1 = -z * e, f2 = z * z * e;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) v[mu][kk] = on ? 2.f * f1 * pv[mu] : 0.f;
                v[Q - 1][kk] = on ? 4.f * f2 * pp + 2.f * f1 * sq : 0.f;
            }
        } else {
            int a_prev = -1;
            float t = 0.f, pp = 0.f, sq = 0.f, pv[3] = {0.f, 0.f, 0.f};
            const int b0 = c * kKc + k0;
            int a0, g0;
            if (gshift >= 0) { a0 = b0 >> gshift; g0 = b0 & (G - 1); }
            else { a0 = b0 / G; g0 = b0 - a0 * G; }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int b = b0 + kk;
                int a = a0, g = g0 + kk;
                while (g >= G) { g -= G; ++a; }
#pragma unroll
                for (int q = 0; q < Q; ++q) v[q][kk] = 0.f;
                if (b >= B || row0 + r >= nrows) continue;
                if (a != a_prev) {
                    a_prev = a;
                    const float* pt = ptr_s + 6 * a;
                    t = 0.f; pp = 0.f; sq = 0.f;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        const float sx = rtrig[r][mu], cx = rtrig[r][3 + mu];
                        const float sd = sx * pt[3 + mu] - cx * pt[mu];
                        const float cd = cx * pt[3 + mu] + sx * pt[mu];
                        t += sd * sd;
                        pv[mu] = ell * sd * cd;
                        pp += pv[mu] * pv[mu];
                        sq += cd * cd - sd * sd;
                    }
                    t *= ell * ell;
                }
                const float z = zs[g];
                const float e = tc_ex2(-zs[8 + g] * t);
                const float f1 = -z * e, f2 = z * z * e;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) v[mu][kk] = 2.f * f1 * pv[mu];
                v[Q - 1][kk] = 4.f * f2 * pp + 2.f * f1 * sq;
            }
        }
        const uint32_t off = tc::sw128_off(r, k0);
#pragma unroll
        for (int q = 0; q < Q; ++q) {
            unsigned char* tq = sA + (size_t)(P * q) * kTileA + off;
            float4 x0, x1;
            tc::split_tf32_fast(v[q][0], x0.x, x1.x);
            tc::split_tf32_fast(v[q][1], x0.y, x1.y);
            tc::split_tf32_fast(v[q][2], x0.z, x1.z);
            tc::split_tf32_fast(v[q][3], x0.w, x1.w);
            *(float4*)(tq) = x0;
            *(float4*)(tq + kTileA) = x1;
        }
        // this warp's share of half h is in shared memory
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&fullh[h]);
    };
    // a fold is complete in this warp: make its TMEM stores visible to the MMAs
    auto arrive_fold = [&](uint64_t* bar) {
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(bar);
    };
    if (tid < kProd) {
        fetch_b4(0);
        store_b4(0);
        if (nch > 1) fetch_b4(1);
    }
    const bool issuer = warp == kProd / 32;
    if (issuer) {
        if (lane == 0) {
            // MMAs of half h of chunk c for quantities q0, q0 + 1: chunk 0 into
            // the running total, later chunks into the chunk block
            auto issue = [&](int c, int h, int q0) {
                const uint32_t b0 = tc::smem_addr(sB + (size_t)(c & 1) * bbytes), bstep = (uint32_t)NM * 128;
#pragma unroll
                for (int q = q0; q < q0 + 2; ++q) {
                    const uint32_t a0 = tc::smem_addr(sA + (size_t)(P * q) * kTileA);
                    const uint32_t d = tmem + (c > 0 ? kSub : 0u) + (uint32_t)(q * NM);
#pragma unroll
                    for (int kh = 0; kh < 2; ++kh) {
                        const int ks = 2 * h + kh;
                        const uint32_t o = 32u * ks;
                        // products A_i B_j with i + j <= 1, smallest first
                        const int pi[3] = {1, 0, 0}, pj[3] = {0, 1, 0};
#pragma unroll
                        for (int m = 0; m < 3; ++m)
                            tc::mma_tf32(d, tc::desc_sw128(a0 + pi[m] * kTileA + o),
                                         tc::desc_sw128(b0 + pj[m] * bstep + o), idesc, (ks > 0 || m > 0) ? 1u : 0u);
                    }
                }
            };
            for (int c = 0; c < nch; ++c) {
                const uint32_t par = (uint32_t)(c & 1);
                // S1: half 0 of (d/dx, d/dy), once the half is produced and C_a folded
                if (!tc::mbar_wait(&fullh[0], par, 1ll << 26)) ok = false;
                if (c >= 2 && !tc::mbar_wait(&foldab[0], par, 1ll << 26)) ok = false;
                tc::fence_after_sync();
                issue(c, 0, 0);
                // S2: half 0 of (d/dz, Laplacian), once C_b is folded; half 0 is then read
                if (c >= 2 && !tc::mbar_wait(&foldab[1], par, 1ll << 26)) ok = false;
                tc::fence_after_sync();
                issue(c, 0, 2);
                tc::mma_commit(&freeh0);
                // S3: half 1 of (d/dx, d/dy); C_a of this chunk complete
                if (!tc::mbar_wait(&fullh[1], par, 1ll << 26)) ok = false;
                tc::fence_after_sync();
                issue(c, 1, 0);
                tc::mma_commit(&mbarh[0]);
                // S4: half 1 of (d/dz, Laplacian); the chunk is read, C_b complete
                issue(c, 1, 2);
                tc::mma_commit(&mbarh[1]);
            }
        }
        __syncwarp();
    } else {
        for (int c = 0; c < nch; ++c) {
            const uint32_t pp_ = (uint32_t)((c - 1) & 1);
            if (c >= 1) {
                if (!tc::mbar_wait(&freeh0, pp_, 1ll << 26)) ok = false;     // S2 of c - 1 done
                tc::fence_after_sync();
            }
            produce(c, 0);
            if (c >= 1) {
                if (!tc::mbar_wait(&mbarh[0], pp_, 1ll << 26)) ok = false;   // S3 of c - 1 done
                tc::fence_after_sync();
                if (c >= 2) { fold_group(0); arrive_fold(&foldab[0]); }
                if (!tc::mbar_wait(&mbarh[1], pp_, 1ll << 26)) ok = false;   // S4 of c - 1 done
                tc::fence_after_sync();
                if (c >= 2) { fold_group(1); arrive_fold(&foldab[1]); }
            }
            // the B buffer of chunk c + 1 was last read by chunk c - 1, done
            if (c + 1 < nch) {
                store_b4((c + 1) & 1);
                if (c + 2 < nch) fetch_b4(c + 2);
            }
            produce(c, 1);
        }
        // the last chunk's blocks (chunk 0 went straight into T)
        const uint32_t pl = (uint32_t)((nch - 1) & 1);
        if (!tc::mbar_wait(&mbarh[0], pl, 1ll << 26)) ok = false;
        tc::fence_after_sync();
        if (nch >= 2) fold_group(0);
        if (!tc::mbar_wait(&mbarh[1], pl, 1ll << 26)) ok = false;
        tc::fence_after_sync();
        if (nch >= 2) fold_group(1);
        tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
    } else {
    // B operand: the first P pieces of each prepared C^T chunk (16-byte
    // vectors).  Q = 4 (one CTA per SM): fetched into registers one chunk
    // ahead and stored once the previous chunk's MMAs are done.  Q = 1 (several
    // CTAs per SM hide the latency): copied at the start of each chunk.
    constexpr int kBv = Q == 4 ? 2 : 4;   // P * NM * 8 <= 1024 vectors over 512 (Q = 4) or 256 threads
    const int nbv = P * NM * 8;
    uint4 bnext[kBv];
    auto fetch_b = [&](int c) {
        const uint4* src = (const uint4*)(chat + (size_t)c * chunk_bytes);
#pragma unroll
        for (int v = 0; v < kBv; ++v) {
            const int idx = tid + v * nt;
            if (idx < nbv) bnext[v] = src[idx];
        }
    };
    auto store_b = [&]() {
        uint4* dst = (uint4*)sB;
#pragma unroll
        for (int v = 0; v < kBv; ++v) {
            const int idx = tid + v * nt;
            if (idx < nbv) dst[idx] = bnext[v];
        }
    };
    // Q = 1: B comes by one bulk copy per chunk (a single thread, no
    // registers), issued as soon as the previous chunk's MMAs are done, so it
    // lands while the threads evaluate the chunk's basis functions; the
    // issuing thread waits for it before the MMAs.
    const uint32_t bcopy = (uint32_t)(P * NM * 128);   // a whole chunk: the prepared pieces are the P used
    if constexpr (Q == 1) {
        if (tid == 0) {
            tc::mbar_arrive_expect_tx(&bbar, bcopy);
            tc::bulk_g2s(sB, chat, bcopy, &bbar);
        }
    } else {
        fetch_b(0);
        store_b();
    }
    for (int c = 0; c < nch; ++c) {
        if constexpr (Q == 4) {
            if (c + 1 < nch) fetch_b(c + 1);
        }
        // A operand: one item = (row, 4 consecutive basis functions); the
        // displacement to a nucleus is computed once for its Gaussians.  In the
        // value kernel all items of a thread are evaluated before any is
        // stored, so their arithmetic overlaps (the stores could alias the
        // tables it reads); the derivative kernel stores item by item.
        constexpr int IT = kRows * (kKc / 4) / (Q == 1 ? 256 : 512);   // items per thread
        float vv[IT][Q][4];
        auto store_item = [&](int u) {
            const int item = tid + u * nt;
            const int r = item / (kKc / 4), k0 = 4 * (item - r * (kKc / 4));
            const uint32_t off = tc::sw128_off(r, k0);
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                unsigned char* tq = sA + (size_t)(P * q) * kTileA + off;
                const float* v = vv[u][q];
                if constexpr (P == 3) {
                    float4 x0, x1, x2;
                    tc::split3_tf32(v[0], x0.x, x1.x, x2.x);
                    tc::split3_tf32(v[1], x0.y, x1.y, x2.y);
                    tc::split3_tf32(v[2], x0.z, x1.z, x2.z);
                    tc::split3_tf32(v[3], x0.w, x1.w, x2.w);
                    *(float4*)(tq) = x0;
                    *(float4*)(tq + kTileA) = x1;
                    *(float4*)(tq + 2 * kTileA) = x2;
                } else {
                    // hi rounded to TF32; lo = x - hi exactly, whose low bits the
                    // tensor core drops (sign-symmetric, below 2^-22 |x|)
                    float4 x0, x1;
                    tc::split_tf32_fast(v[0], x0.x, x1.x);
                    tc::split_tf32_fast(v[1], x0.y, x1.y);
                    tc::split_tf32_fast(v[2], x0.z, x1.z);
                    tc::split_tf32_fast(v[3], x0.w, x1.w);
                    *(float4*)(tq) = x0;
                    *(float4*)(tq + kTileA) = x1;
                }
            }
        };
        // Value kernel with 4 Gaussians per nucleus (256 threads): the items of
        // a thread are rows tid / 8 + 32 u of the one nucleus c * 8 + tid % 8,
        // so its trig values are loaded once per chunk and the exponent needs
        // only the squared periodised distance.
        const bool fast4 = Q == 1 && G == 4 && nt == 256;
        if (fast4) {
            const int a = c * (kKc / 4) + (tid & 7);
            const bool a_ok = a < N;
            float ps[3], pc[3];
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) {
                ps[mu] = a_ok ? ptr_s[6 * a + mu] : 0.f;
                pc[mu] = a_ok ? ptr_s[6 * a + 3 + mu] : 1.f;
            }
            const float ell2 = ell * ell;
#pragma unroll
            for (int u = 0; u < IT; ++u) {
                const int r = (tid >> 3) + 32 * u;
                float t = 0.f;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu) {
                    const float sd = rtrig[r][mu] * pc[mu] - rtrig[r][3 + mu] * ps[mu];
                    t += sd * sd;
                }
                t *= ell2;
                const bool on = a_ok && row0 + r < nrows;
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) vv[u][0][kk] = on ? tc_ex2(-zs[8 + kk] * t) : 0.f;
            }
        }
#pragma unroll
        for (int u = 0; u < (fast4 ? 0 : IT); ++u) {
            const int item = tid + u * nt;
            const int r = item / (kKc / 4), k0 = 4 * (item - r * (kKc / 4));
            int a_prev = -1;
            float t = 0.f, pp = 0.f, sq = 0.f, pv[3] = {0.f, 0.f, 0.f};
            // nucleus and Gaussian of basis function b = a G + g (shifts when G is a power of two)
            const int b0 = c * kKc + k0;
            int a0, g0;
            if (gshift >= 0) { a0 = b0 >> gshift; g0 = b0 & (G - 1); }
            else { a0 = b0 / G; g0 = b0 - a0 * G; }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const int b = b0 + kk;
                int a = a0, g = g0 + kk;
                while (g >= G) { g -= G; ++a; }
#pragma unroll
                for (int q = 0; q < Q; ++q) vv[u][q][kk] = 0.f;
                if (b >= B || row0 + r >= nrows) continue;
                if (a != a_prev) {
                    a_prev = a;
                    const float* pt = ptr_s + 6 * a;
                    t = 0.f; pp = 0.f; sq = 0.f;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        const float sx = rtrig[r][mu], cx = rtrig[r][3 + mu];
                        const float sd = sx * pt[3 + mu] - cx * pt[mu];
                        const float cd = cx * pt[3 + mu] + sx * pt[mu];
                        t += sd * sd;
                        pv[mu] = ell * sd * cd;
                        pp += pv[mu] * pv[mu];
                        sq += cd * cd - sd * sd;
                    }
                    t *= ell * ell;
                }
                const float z = zs[g];
                const float e = tc_ex2(-zs[8 + g] * t);
                if (Q == 1) {
                    vv[u][0][kk] = e;
                } else {
                    const float f1 = -z * e, f2 = z * z * e;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) vv[u][mu][kk] = 2.f * f1 * pv[mu];
                    vv[u][Q - 1][kk] = 4.f * f2 * pp + 2.f * f1 * sq;
                }
            }
            if constexpr (Q != 1) store_item(u);   // register budget: one item at a time
        }
        if constexpr (Q == 1) {
#pragma unroll
            for (int u = 0; u < IT; ++u) store_item(u);
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            if (Q == 1 && !tc::mbar_wait(&bbar, (uint32_t)(c & 1), 1ll << 26)) ok = false;   // B of chunk c
            tc::fence_after_sync();
            const uint32_t b0 = tc::smem_addr(sB), bstep = (uint32_t)NM * 128;
#pragma unroll
            for (int q = 0; q < Q; ++q) {
                const uint32_t a0 = tc::smem_addr(sA + (size_t)(P * q) * kTileA);
                // chunk 0 into the running total, later chunks into the chunk block
                const uint32_t d = tmem + (c > 0 ? kSub : 0u) + (uint32_t)(q * NM);
#pragma unroll
                for (int ks = 0; ks < kKc / 8; ++ks) {
                    const uint32_t o = 32u * ks;
                    // products A_i B_j with i + j <= P - 1, smallest first
                    constexpr int np = P == 3 ? 6 : 3;
                    const int pi[6] = {2, 1, 0, 1, 0, 0}, pj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
                    for (int m = 6 - np; m < 6; ++m)
                        tc::mma_tf32(d, tc::desc_sw128(a0 + pi[m] * kTileA + o), tc::desc_sw128(b0 + pj[m] * bstep + o),
                                     idesc, (ks > 0 || m > 6 - np) ? 1u : 0u);
                }
            }
            tc::mma_commit(&mbarh[0]);
        }
        // the other lanes of the issuing warp wait here, not in the mbarrier
        // poll below, so they do not hold up the single issuing lane; one warp
        // polls for the MMAs, the others wait at the block barrier and take no
        // issue slots from the other CTAs on the SM meanwhile
        __syncwarp();
        if (warp == 0 && !tc::mbar_wait(&mbarh[0], (uint32_t)(c & 1), 1ll << 26)) ok = false;
        __syncthreads();
        tc::fence_after_sync();
        if (c > 0) {                             // chunk c into the running total
            fold_chunk(nt / 32);
            tc::fence_before_sync();
        }
        if (Q == 4 && c + 1 < nch) store_b();   // the MMAs of chunk c have read sB
        if (Q == 1 && tid == 0 && c + 1 < nch) {
            tc::mbar_arrive_expect_tx(&bbar, bcopy);
            tc::bulk_g2s(sB, chat + (size_t)(c + 1) * chunk_bytes, bcopy, &bbar);
        }
        __syncthreads();
    }
    // a copy still in flight after a wait that gave up lands before the CTA leaves
    if (Q == 1 && tid == 0 && !ok) tc::mbar_wait(&bbar, (uint32_t)((nch - 1) & 1), 1ll << 26);
    }
    if (!ok && lane == 0) raise_err(s.err, kErrTimeout);

    // Epilogue, one quantity at a time: TMEM -> registers -> shared staging
    // tile [128][NM + 4] (the A tiles are free now) -> coalesced HBM stores.
    float* stage = (float*)sA;
    const int lds = NM + 4;
    const int quarter = warp & 3, cgroup = warp >> 2, ngroups = nt / 128;
    const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16);
    const int r = quarter * 32 + lane;
    const int rows_here = (nrows - row0) < kRows ? (nrows - row0) : kRows;
    // rows of n floats go out as 16-byte vectors when n / 4 is a power of two
    // (index arithmetic by shifts; every output row then starts 16-byte aligned)
    const int nv = n >> 2;
    const int vshift = ((n & 3) == 0 && (nv & (nv - 1)) == 0) ? __ffs(nv) - 1 : -1;
    for (int q = 0; q < Q; ++q) {
        for (int c0 = cgroup * 16; c0 < NM; c0 += 16 * ngroups) {
            float v[16];
            tc::tmem_ld16(taddr + (uint32_t)(q * NM + c0), v);
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                *(float4*)(stage + (size_t)r * lds + c0 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        }
        __syncthreads();
        float* dst = Q == 1 ? val : (q == Q - 1 ? lap : grad + (size_t)q * n);
        const size_t pitch = (Q == 1 || q == Q - 1) ? (size_t)n : (size_t)3 * n;   // floats between rows
        if (vshift >= 0) {
            for (int idx = tid; idx < (rows_here << vshift); idx += nt) {
                const int rr = idx >> vshift, j = (idx & (nv - 1)) << 2;
                *(float4*)(dst + (size_t)(row0 + rr) * pitch + j) = *(const float4*)(stage + (size_t)rr * lds + j);
            }
        } else {
            for (int idx = tid; idx < rows_here * n; idx += nt) {
                const int rr = idx / n, j = idx - rr * n;
                dst[(size_t)(row0 + rr) * pitch + j] = stage[(size_t)rr * lds + j];
            }
        }
        __syncthreads();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kCols);
}

void launch_orbitals_tc(const SysView<float>& s, const void* chat, const double* pos, int nrows, float* val,
                        float* grad, float* lap, cudaStream_t st) {
    const int NM = tc_nm(s.n);
    const int grid = (nrows + kRows - 1) / kRows;
    // the dynamic shared-memory limit is raised to what a launch needs (the
    // kernel also holds static shared memory, so the opt-in maximum minus that)
    static size_t set4 = 0, set1 = 0;
    if (grad) {
        const size_t smem = 1024 + (size_t)4 * kPiecesDer * kTileA + (size_t)2 * kPiecesDer * NM * 128 + 24 * (size_t)s.N;
        if (smem > set4 &&
            cudaFuncSetAttribute(orbitals_tc_kernel<4, kPiecesDer>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess)
            set4 = smem;
        orbitals_tc_kernel<4, kPiecesDer>
            <<<grid, 544, smem, st>>>(s, (const unsigned char*)chat, pos, nrows, NM, val, grad, lap);
    } else {
        const size_t smem = 1024 + (size_t)kPiecesVal * kTileA + (size_t)kPiecesVal * NM * 128 + 24 * (size_t)s.N;
        if (smem > set1 &&
            cudaFuncSetAttribute(orbitals_tc_kernel<1, kPiecesVal>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) == cudaSuccess)
            set1 = smem;
        orbitals_tc_kernel<1, kPiecesVal>
            <<<grid, 256, smem, st>>>(s, (const unsigned char*)chat, pos, nrows, NM, val, nullptr, nullptr);
    }
}

}  // namespace qmc
