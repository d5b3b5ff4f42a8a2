// Reduced density operators of pure states (TensorLy-Quantum Sec. 2: partial traces of
// density operators; Sec. 3, Fig. 1 left: full-rank partial traces from n to m qubits).
//
// For rho = |psi><psi| and a kept qubit set A (m qubits) with complement B,
//   rho_A[i][j] = sum_k Psi[i][k] conj(Psi[j][k]),   Psi[i][k] = psi(kept bits i, traced bits k),
// i.e. rho_A = Psi Psi^dagger with Psi a 2^m x 2^(n-m) matrix: a Hermitian rank-K update.
// Kernels:
//   * psi_gather_kernel lays Psi out row-major (row i contiguous in k) from the state, where
//     bit t of i is the t-th lowest kept qubit and bit u of k the u-th lowest traced one;
//   * herk_ws_kernel (m >= 7 with at least one whole tile per SM) computes 128 x 128 tiles of
//     the upper block triangle on the tensor cores (tcgen05, TF32 high/low split, FP32
//     accumulators in tensor memory): persistent CTAs with producer, MMA and epilogue warps,
//     two accumulator sets, TMA tensor stores of off-diagonal tiles and their conjugate mirrors;
//   * herk_tc_kernel (m >= 7, fewer tiles: k split over CTAs) does the same arithmetic one
//     tile per CTA, all warps taking turns at loading and storing;
//   * herk_tile_kernel (m < 7) computes 64 x 64 tiles on FP32 CUDA cores with 4 x 4 complex
//     register blocks per thread from 16-wide k chunks staged in shared memory.
// Entries above the diagonal are written twice (as computed, and conjugate-transposed below
// it) and the diagonal as real numbers, so the output is exactly Hermitian. When the output
// has few tiles (small m, long k) the k range is split over CTAs; the splits are summed in a
// fixed order by herk_reduce_kernel, so results are deterministic. Complex64 output.
#include <cuda.h>   // CUtensorMap and its enums (the encoder is fetched through the runtime)
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>

#include "internal.h"

namespace tlq {

namespace {

constexpr int kTileR = 64;     // output tile edge
constexpr int kChunkK = 16;    // k chunk staged per step
constexpr int kHerkThreads = 256;

// Psi[i * K + k] = psi[x(i, k)], x = deposit(i, keep bits) | deposit(k, traced bits).
__global__ void psi_gather_kernel(const float2* __restrict__ psi, float2* __restrict__ Psi, int n, int m,
                                  const __grid_constant__ QubitMap Q) {
    __shared__ int32_t s_kept[32], s_traced[32];
    if (threadIdx.x < m) s_kept[threadIdx.x] = Q.kept[threadIdx.x];
    if (threadIdx.x < n - m) s_traced[threadIdx.x] = Q.traced[threadIdx.x];
    __syncthreads();
    const uint64_t N = 1ull << n;
    const int kb = n - m;
    for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N; y += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t k = y & ((1ull << kb) - 1);
        const uint64_t i = y >> kb;
        uint64_t x = 0;
        for (int t = 0; t < m; ++t) x |= ((i >> t) & 1ull) << s_kept[t];
        for (int u = 0; u < kb; ++u) x |= ((k >> u) & 1ull) << s_traced[u];
        Psi[y] = psi[x];
    }
}

// Upper block-triangle tile u -> (bi, bj), bi <= bj: u = bj (bj + 1) / 2 + bi.
__device__ __forceinline__ void tri_tile(uint32_t u, int& bi, int& bj) {
    int r = (int)((sqrtf(8.0f * (float)u + 1.0f) - 1.0f) * 0.5f);   // within one of the root; fixed below
    while ((uint64_t)(r + 1) * (uint64_t)(r + 2) / 2 <= u) ++r;
    while ((uint64_t)r * (uint64_t)(r + 1) / 2 > u) --r;
    bj = r;
    bi = (int)(u - (uint32_t)((uint64_t)r * (uint64_t)(r + 1) / 2));
}

// Stage rows [r0, r0 + 64) x k [k0, k0 + 16) of Psi transposed into s[k][row]; rows >= D and
// k >= kend read as zero.
__device__ __forceinline__ void load_chunk(const float2* __restrict__ Psi, int64_t D, int64_t K, int64_t r0,
                                           int64_t k0, int64_t kend, float2 (&reg)[4], int tid) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int idx = tid + kHerkThreads * e;   // 0 .. 1023 = 64 rows x 16 k
        const int row = idx >> 4, kk = idx & 15;
        const int64_t r = r0 + row, k = k0 + kk;
        reg[e] = (r < D && k < kend) ? Psi[r * K + k] : make_float2(0.f, 0.f);
    }
}

__device__ __forceinline__ void store_chunk(float2 (*s)[kTileR + 2], const float2 (&reg)[4], int tid) {
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int idx = tid + kHerkThreads * e;
        s[idx & 15][idx >> 4] = reg[e];
    }
}

// grid.x = upper tiles, grid.y = k splits. out = rho (splits == 1) or partial + split * D * D.
__global__ void __launch_bounds__(kHerkThreads) herk_tile_kernel(const float2* __restrict__ Psi, int64_t D,
                                                                  int64_t K, int64_t k_per_split,
                                                                  float2* __restrict__ out) {
    __shared__ __align__(16) float2 sA[kChunkK][kTileR + 2];
    __shared__ __align__(16) float2 sB[kChunkK][kTileR + 2];
    int bi, bj;
    tri_tile(blockIdx.x, bi, bj);
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t i0 = (int64_t)bi * kTileR, j0 = (int64_t)bj * kTileR;
    const int64_t kbeg = (int64_t)blockIdx.y * k_per_split;
    const int64_t kend = kbeg + k_per_split < K ? kbeg + k_per_split : K;
    float2* dst = out + (int64_t)blockIdx.y * (gridDim.y > 1 ? D * D : 0);

    float ar[4][4], ai[4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) ar[r][c] = ai[r][c] = 0.f;

    float2 ra[4], rb[4];
    load_chunk(Psi, D, K, i0, kbeg, kend, ra, tid);
    load_chunk(Psi, D, K, j0, kbeg, kend, rb, tid);
    for (int64_t k0 = kbeg; k0 < kend; k0 += kChunkK) {
        __syncthreads();   // the previous chunk has been consumed
        store_chunk(sA, ra, tid);
        store_chunk(sB, rb, tid);
        __syncthreads();
        if (k0 + kChunkK < kend) {   // prefetch the next chunk while this one is used
            load_chunk(Psi, D, K, i0, k0 + kChunkK, kend, ra, tid);
            load_chunk(Psi, D, K, j0, k0 + kChunkK, kend, rb, tid);
        }
#pragma unroll
        for (int kk = 0; kk < kChunkK; ++kk) {
            float2 a[4], b[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) a[r] = sA[kk][ty * 4 + r];
#pragma unroll
            for (int c = 0; c < 4; ++c) b[c] = sB[kk][tx * 4 + c];
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    // a * conj(b)
                    ar[r][c] = fmaf(a[r].x, b[c].x, fmaf(a[r].y, b[c].y, ar[r][c]));
                    ai[r][c] = fmaf(a[r].y, b[c].x, fmaf(-a[r].x, b[c].y, ai[r][c]));
                }
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int64_t i = i0 + ty * 4 + r;
        if (i >= D) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int64_t j = j0 + tx * 4 + c;
            if (j >= D || j < i) continue;   // the upper triangle; the lower one is its mirror
            if (j == i) {
                dst[i * D + i] = make_float2(ar[r][c], 0.f);   // rho is Hermitian: real diagonal
            } else {
                dst[i * D + j] = make_float2(ar[r][c], ai[r][c]);
                dst[j * D + i] = make_float2(ar[r][c], -ai[r][c]);
            }
        }
    }
}

// rho[e] = sum over splits s = 0, 1, ... of partial[s][e] (FP64 sum in split order).
__global__ void herk_reduce_kernel(const float2* __restrict__ partial, int splits, int64_t DD,
                                   float2* __restrict__ rho) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < DD; e += (int64_t)gridDim.x * blockDim.x) {
        double re = 0.0, im = 0.0;
        for (int s = 0; s < splits; ++s) {
            const float2 v = partial[(int64_t)s * DD + e];
            re += v.x;
            im += v.y;
        }
        rho[e] = make_float2((float)re, (float)im);
    }
}

// ---- tensor-core path (tcgen05, TMEM accumulators) ------------------------------------------
//
// rho_A = Psi Psi^dagger in real arithmetic with planar operands (re, im of Psi rows):
//   Re rho = A_re B_re^T + A_im B_im^T,   Im rho = A_im B_re^T + A_re (-B_im)^T,
// A = rows i of the output tile, B = rows j. Each FP32 operand x is split into TF32 parts
// x_hi (x with the low 13 mantissa bits cleared, exact in TF32) and x_lo = x - x_hi; every
// product is x_hi y_hi + x_hi y_lo + x_lo y_hi (the dropped x_lo y_lo is 2^-20 relative),
// accumulated in FP32 in tensor memory: Re in TMEM columns 0..127 of the accumulator, Im in
// 128..255. The twelve products of a chunk go as six MMAs of N = 256 (M = 128, K = 8,
// kind::tf32): an A part times a stack of two B parts [X; Y] adds A X^T to Re and A Y^T to Im.
// The B parts are laid out as [B_im hi][B_re hi][-B_im hi] [B_im lo][B_re lo][-B_im lo], so
// every stack needed is two neighbouring parts:
//   A_re hi x [B_re hi; -B_im hi],  A_re hi x [B_re lo; -B_im lo],  A_re lo x [B_re hi; -B_im hi],
//   A_im hi x [B_im hi;  B_re hi],  A_im hi x [B_im lo;  B_re lo],  A_im lo x [B_im hi;  B_re hi].
// Shared-memory operands use the no-swizzle K-major layout: 8-row x 16-byte core matrices,
// 128 bytes apart along K and 256 bytes apart along M/N (one 4 KB tile per operand part, a
// 256-row stack spanning two neighbouring parts).
//
// herk_tc_kernel: one CTA (8 warps) owns a 128 x 128 output tile. The k range is walked in
// chunks of 8 complex values, double-buffered in shared memory: all threads load and split a
// chunk while the tensor core works on the previous one, and thread 0 issues the chunk's MMAs
// and commits them to that buffer's mbarrier; the global loads of the following chunk are
// issued right after, so their latency overlaps the tensor core's work.

constexpr int kTcTile = 128;
constexpr int kTcThreads = 256;
constexpr int kTcChunk = 8;                         // complex k per stage (one MMA K-step)
constexpr int kTcPartBytes = kTcTile * kTcChunk * 4; // 4 KB: 128 rows x 8 TF32
constexpr int kTcParts = 10;                        // A: re/im hi/lo; B: im, re, -im, each hi and lo
constexpr int kTcStageBytes = kTcParts * kTcPartBytes;
constexpr int kTcTmemCols = 2 * kTcTile;            // Re and Im accumulators
constexpr unsigned long long kTcWaitNs = 1000000000ull;   // bound on every mbarrier wait

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t gtimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ bool mbar_done(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the given phase of an mbarrier, giving up after kTcWaitNs.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const uint64_t t0 = gtimer();
    while (!mbar_done(bar, parity)) {
        if (gtimer() - t0 > kTcWaitNs) return false;
        __nanosleep(32);
    }
    return true;
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K-direction) and stride
// (M/N-direction) byte offsets of the core matrices, descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor: FP32 accumulator, TF32 A and B, both K-major, M = 128, N = 256.
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)((2 * kTcTile) >> 3) << 17) |
                              ((uint32_t)(kTcTile >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kTcIdesc), "r"(accumulate)
        : "memory");
}

// 16 consecutive FP32 columns of this warp's 32 TMEM lanes, one lane per thread.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes, one lane per thread.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// Split 4 complex values of row `row` (k = 4 * half .. +3 of the chunk) into the operand parts
// at `base`: A side (re hi, re lo, im hi, im lo), or B side (im hi, re hi, -im hi, im lo,
// re lo, -im lo); 16-byte stores.
__device__ __forceinline__ void put_row4(unsigned char* base, int row, int half, const float4& p0, const float4& p1,
                                         bool b_side) {
    const int off = (row >> 3) * 256 + half * 128 + (row & 7) * 16;
    const float re[4] = {p0.x, p0.z, p1.x, p1.z};
    const float im[4] = {p0.y, p0.w, p1.y, p1.w};
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        rh[e] = tf32_hi(re[e]);
        rl[e] = re[e] - rh[e];
        ih[e] = tf32_hi(im[e]);
        il[e] = im[e] - ih[e];
    }
    if (!b_side) {
        *reinterpret_cast<float4*>(base + 0 * kTcPartBytes + off) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4*>(base + 1 * kTcPartBytes + off) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<float4*>(base + 2 * kTcPartBytes + off) = make_float4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<float4*>(base + 3 * kTcPartBytes + off) = make_float4(il[0], il[1], il[2], il[3]);
    } else {
        *reinterpret_cast<float4*>(base + 0 * kTcPartBytes + off) = make_float4(ih[0], ih[1], ih[2], ih[3]);
        *reinterpret_cast<float4*>(base + 1 * kTcPartBytes + off) = make_float4(rh[0], rh[1], rh[2], rh[3]);
        *reinterpret_cast<float4*>(base + 2 * kTcPartBytes + off) = make_float4(-ih[0], -ih[1], -ih[2], -ih[3]);
        *reinterpret_cast<float4*>(base + 3 * kTcPartBytes + off) = make_float4(il[0], il[1], il[2], il[3]);
        *reinterpret_cast<float4*>(base + 4 * kTcPartBytes + off) = make_float4(rl[0], rl[1], rl[2], rl[3]);
        *reinterpret_cast<float4*>(base + 5 * kTcPartBytes + off) = make_float4(-il[0], -il[1], -il[2], -il[3]);
    }
}

// The six MMAs of one staged chunk (parts at shared address `st`) into the accumulator at TMEM
// column `d` (Re at d, Im at d + 128); `acc` = 0 starts a new tile.
__device__ __forceinline__ void issue_chunk(uint32_t d, uint32_t st, uint32_t acc) {
    const uint64_t a0 = sdesc(st, 128, 256);   // part 0; part p is + p * kTcPartBytes / 16
    auto dp = [&](int part) { return a0 + (uint64_t)(part * (kTcPartBytes >> 4)); };
    mma_tf32(d, dp(0), dp(5), acc);   // A_re hi x [B_re hi; -B_im hi]
    mma_tf32(d, dp(0), dp(8), 1u);    // A_re hi x [B_re lo; -B_im lo]
    mma_tf32(d, dp(1), dp(5), 1u);    // A_re lo x [B_re hi; -B_im hi]
    mma_tf32(d, dp(2), dp(4), 1u);    // A_im hi x [B_im hi;  B_re hi]
    mma_tf32(d, dp(2), dp(7), 1u);    // A_im hi x [B_im lo;  B_re lo]
    mma_tf32(d, dp(3), dp(4), 1u);    // A_im lo x [B_im hi;  B_re hi]
}

__device__ __forceinline__ void load_rows(const float2* __restrict__ Psi, int64_t D, int64_t K, int64_t r0, int64_t k0,
                                          int64_t kend, int row, int half, float4& p0, float4& p1) {
    const int64_t r = r0 + row, k = k0 + 4 * half;
    p0 = make_float4(0.f, 0.f, 0.f, 0.f);
    p1 = p0;
    if (r >= D) return;
    const float2* src = Psi + r * K + k;
    if (k + 4 <= kend) {
        p0 = *reinterpret_cast<const float4*>(src);
        p1 = *reinterpret_cast<const float4*>(src + 2);
    } else {
        float2 v[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) v[e] = (k + e < kend) ? src[e] : make_float2(0.f, 0.f);
        p0 = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
        p1 = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
    }
}

// One chunk of the tile's k loop: wait until the MMAs that last read this stage are done,
// split the chunk held in registers into the stage, issue its 12 MMAs (thread 0), then load
// the chunk two ahead into the same registers. Returns false when a wait gave up.
__device__ __forceinline__ bool tc_chunk(int c, int nchunks, unsigned char* stage0, uint64_t* bars, uint32_t tmem,
                                         const float2* __restrict__ Psi, int64_t D, int64_t K, int64_t i0,
                                         int64_t j0, int64_t kbeg, int64_t kend, int row, int half, int tid,
                                         float4& a0, float4& a1, float4& b0, float4& b1) {
    const int s = c & 1;
    unsigned char* st = stage0 + s * kTcStageBytes;
    bool bad = false;
    if (c >= 2) bad = !mbar_wait(su32(&bars[s]), (uint32_t)(((c >> 1) - 1) & 1));   // MMAs of chunk c-2 done
    if (__syncthreads_or(bad)) return false;
    put_row4(st, row, half, a0, a1, false);                    // parts 0-3: A re/im hi/lo
    put_row4(st + 4 * kTcPartBytes, row, half, b0, b1, true);  // parts 4-9: B im, re, -im
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        issue_chunk(tmem, su32(st), c > 0 ? 1u : 0u);
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(&bars[s]))
                     : "memory");
    }
    if (c + 2 < nchunks) {
        const int64_t k2 = kbeg + (int64_t)(c + 2) * kTcChunk;
        load_rows(Psi, D, K, i0, k2, kend, row, half, a0, a1);
        load_rows(Psi, D, K, j0, k2, kend, row, half, b0, b1);
    }
    return true;
}

constexpr int kTcStagePitch = 64 + 1;   // complex per staged output row (64 columns + 1 pad)

// grid.x = upper 128-tiles, grid.y = k splits; out = rho or partial + split * D * D.
__global__ void __launch_bounds__(kTcThreads, 2) herk_tc_kernel(const float2* __restrict__ Psi, int64_t D, int64_t K,
                                                                int64_t k_per_split, float2* __restrict__ out,
                                                                int32_t* __restrict__ err,
                                                                const __grid_constant__ CUtensorMap tm_rows,
                                                                const __grid_constant__ CUtensorMap tm_mirror,
                                                                int use_tma) {
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    unsigned char* stage0 = tc_smem;                                 // 2 stages x 40 KB
    uint64_t* bars = reinterpret_cast<uint64_t*>(tc_smem + 2 * kTcStageBytes);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int bi, bj;
    tri_tile(blockIdx.x, bi, bj);
    const int64_t i0 = (int64_t)bi * kTcTile, j0 = (int64_t)bj * kTcTile;
    const int64_t kbeg = (int64_t)blockIdx.y * k_per_split;
    const int64_t kend = kbeg + k_per_split < K ? kbeg + k_per_split : K;
    const int nchunks = (int)((kend - kbeg + kTcChunk - 1) / kTcChunk);
    float2* dst = out + (int64_t)blockIdx.y * (gridDim.y > 1 ? D * D : 0);

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[0])) : "memory");
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&bars[1])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_slot)),
                     "r"(kTcTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    const int row = tid >> 1, half = tid & 1;   // this thread's row of A and of B, and k half
    // chunks c (even) and c + 1 (odd) in two register sets, each refilled two chunks ahead
    float4 a0, a1, b0, b1, e0, e1, f0, f1;
    if (nchunks > 0) {
        load_rows(Psi, D, K, i0, kbeg, kend, row, half, a0, a1);
        load_rows(Psi, D, K, j0, kbeg, kend, row, half, b0, b1);
    }
    if (nchunks > 1) {
        load_rows(Psi, D, K, i0, kbeg + kTcChunk, kend, row, half, e0, e1);
        load_rows(Psi, D, K, j0, kbeg + kTcChunk, kend, row, half, f0, f1);
    }
    bool bad = false;
    for (int c = 0; c < nchunks; c += 2) {
        if (!tc_chunk(c, nchunks, stage0, bars, tmem, Psi, D, K, i0, j0, kbeg, kend, row, half, tid, a0, a1, b0, b1)) {
            bad = true;
            break;
        }
        if (c + 1 < nchunks &&
            !tc_chunk(c + 1, nchunks, stage0, bars, tmem, Psi, D, K, i0, j0, kbeg, kend, row, half, tid, e0, e1, f0,
                      f1)) {
            bad = true;
            break;
        }
    }
    if (!bad && nchunks > 0) {
        const int cl = nchunks - 1;
        bad = !mbar_wait(su32(&bars[cl & 1]), (uint32_t)((cl >> 1) & 1));   // every MMA of the tile done
    }
    bad = __syncthreads_or(bad) != 0;
    if (!bad && nchunks > 0 && use_tma && bi != bj) {
        // Off-diagonal tile, TMA epilogue in 8 steps of 16 columns, double-buffered: a step's
        // TMEM values are staged as 128-byte-swizzled boxes (16 complex wide) -- one box of 128
        // rows for rho[i][j] and eight boxes of 16 rows for the mirror rho[j][i] = conj -- and
        // written by tensor stores that one thread issues; staging the next step overlaps them,
        // and a buffer is restaged only after the stores that read it are done.
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = warp & 3, hh = warp >> 2;            // TMEM lanes 32q.., 8-column half hh
        const int r = 32 * q + lane;                       // this thread's row of the tile
        const int ci = r & 15;
        const uint64_t mr = reinterpret_cast<uint64_t>(&tm_rows);
        const uint64_t mm = reinterpret_cast<uint64_t>(&tm_mirror);
#pragma unroll 1
        for (int st = 0; st < kTcTile / 16; ++st) {
            unsigned char* buf = tc_smem + (st & 1) * 32768;   // [16 KB rows box][8 x 2 KB mirror boxes]
            if (tid == 0 && st >= 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
            __syncthreads();   // this buffer's previous stores have read it
            const int col = 16 * st + 8 * hh;              // tile column of this thread's 8 values
            float vr[8], vi[8];
            tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, vr);
            tmem_ld8(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kTcTile + col), vi);
            // rows: row r, 16-byte chunk c (two complex) at chunk c ^ (r & 7); this thread has
            // chunks 4 hh .. 4 hh + 3 of the row
            unsigned char* rb = buf + r * 128;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int cc = 4 * hh + c;
                *reinterpret_cast<float4*>(rb + ((cc ^ (r & 7)) << 4)) =
                    make_float4(vr[2 * c], vi[2 * c], vr[2 * c + 1], vi[2 * c + 1]);
            }
            // mirror: box r / 16 (16 rows x 128 B), row jl = 8 hh + e, complex r % 16
            unsigned char* mb = buf + 16384 + (r >> 4) * 2048;
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int jl = 8 * hh + e;
                *reinterpret_cast<float2*>(mb + jl * 128 + ((((ci >> 1) ^ (jl & 7))) << 4) + ((ci & 1) << 3)) =
                    make_float2(vr[e], -vi[e]);
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(mr),
                             "r"((int)(2 * (j0 + 16 * st))), "r"((int)i0), "r"(su32(buf))
                             : "memory");
                for (int b = 0; b < 8; ++b)
                    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(mm),
                                 "r"((int)(2 * (i0 + 16 * b))), "r"((int)(j0 + 16 * st)),
                                 "r"(su32(buf + 16384 + b * 2048))
                                 : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
            }
        }
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
    } else if (!bad && nchunks > 0) {
        // Epilogue through shared memory (the stages are free now), one 128 x 64 half of the
        // tile at a time: TMEM -> staged rows, then coalesced row writes of the entries on or
        // above the diagonal and coalesced writes of their conjugate mirrors (rows of rho^T).
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        float2* S = reinterpret_cast<float2*>(tc_smem);   // [128][kTcStagePitch]
        const int q = warp & 3, hh = warp >> 2;          // TMEM lanes 32q.., 32-column quarter hh
#pragma unroll 1
        for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll 1
            for (int cc = 0; cc < 2; ++cc) {
                const int col = 64 * h2 + 32 * hh + 16 * cc;   // tile column of this load
                float vr[16], vi[16];
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col, vr);
                tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(kTcTile + col), vi);
                float2* srow = S + (32 * q + lane) * kTcStagePitch + (col - 64 * h2);
#pragma unroll
                for (int e = 0; e < 16; ++e) srow[e] = make_float2(vr[e], vi[e]);
            }
            __syncthreads();
            // rows: entry (i, j) for j >= i (the diagonal as a real number)
#pragma unroll 4
            for (int t = tid; t < kTcTile * 64; t += kTcThreads) {
                const int r = t >> 6, cj = t & 63;
                const int64_t i = i0 + r, j = j0 + 64 * h2 + cj;
                if (i >= D || j >= D || j < i) continue;
                float2 v = S[r * kTcStagePitch + cj];
                if (j == i) v.y = 0.f;
                dst[i * D + j] = v;
            }
            // mirrors: entry (j, i) = conj(i, j) for j > i, written along rows j
#pragma unroll 4
            for (int t = tid; t < kTcTile * 64; t += kTcThreads) {
                const int cj = t >> 7, r = t & 127;
                const int64_t i = i0 + r, j = j0 + 64 * h2 + cj;
                if (i >= D || j >= D || j <= i) continue;
                const float2 v = S[r * kTcStagePitch + cj];
                dst[j * D + i] = make_float2(v.x, -v.y);
            }
            __syncthreads();
        }
    }
    if (bad && tid == 0) atomicExch(err, 3);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTcTmemCols) : "memory");
}

constexpr size_t kTcSmem = 2 * (size_t)kTcStageBytes + 64;

// ---- persistent warp-specialised tensor-core path -------------------------------------------
//
// The arithmetic of herk_tc_kernel (TF32 hi/lo planes, 12 MMAs per 8-complex chunk into Re/Im
// accumulators), organised so that operand loads, tensor-core work and output stores overlap.
// One CTA per SM walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... with three roles:
//   * 8 producer warps: half an A row and half a B row (4 complex each) per thread, loaded
//     kWsAhead chunks ahead into registers, split into the TF32 planes of a shared-memory stage
//     (kWsStages stages) and announced on the stage's "full" mbarrier;
//   * 1 MMA warp: one thread waits for a full stage, issues its six MMAs into one of two TMEM
//     accumulator sets (tiles alternate between them), commits them to the stage's "empty"
//     mbarrier, and after a tile's last chunk commits to the set's "ready" mbarrier;
//   * 8 epilogue warps (warp w: TMEM lane quadrant w % 4, i.e. one tile row per thread, and the
//     8-column half w / 4 of each 16-column step): wait for a ready set, read it, hand it back
//     ("freed" mbarrier) after the last read, and stage the values as 128-byte-swizzled boxes
//     for TMA tensor stores (two staging buffers), as herk_tc_kernel does; diagonal tiles are
//     written from registers (upper triangle, its conjugate mirror, real diagonal) so the output
//     stays exactly Hermitian.
// Every wait is bounded (kTcWaitNs): a role that gives up raises the abort flag and the error
// word, the others stop at their next wait, and all threads meet at the end, after the MMA
// thread has waited for its last MMAs, to release tensor memory.
constexpr int kWsStages = 3;
constexpr int kWsAhead = 3;                        // chunks in flight per producer thread
constexpr int kWsEpi = 256;                        // epilogue threads (warps 0-7)
constexpr int kWsProd = 256;                       // producer threads (warps 8-15)
constexpr int kWsMmaWarp = 16;
constexpr int kWsThreads = 17 * 32;
constexpr int kWsEpiBytes = 32768;                 // one staging buffer: rows box + 8 mirror boxes
constexpr int kWsTmemCols = 2 * kTcTmemCols;       // two accumulator sets
constexpr size_t kWsBarOff = (size_t)kWsStages * kTcStageBytes + 2 * kWsEpiBytes;
constexpr size_t kWsSmem = kWsBarOff + 256;

struct WsBars {
    uint64_t full[kWsStages], empty[kWsStages], ready[2], freed[2], done;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(bar) : "memory");
}

// One potentially blocking test of an mbarrier phase: the hardware suspends the thread until
// the phase completes or a short system time limit passes.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the given phase of an mbarrier; false when another role aborted or after kTcWaitNs
// (then this thread raises the abort flag).
__device__ __forceinline__ bool ws_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (!mbar_try(bar, parity)) {
        if (*abort) return false;
        if (gtimer() - t0 > kTcWaitNs) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// OR of `v` over the 128 epilogue threads (named barrier 1): they leave their loop together,
// so none is left waiting at a barrier the others no longer reach.
__device__ __forceinline__ bool epi_any(bool v) {
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n barrier.red.or.pred q, 1, 256, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)v)
        : "memory");
    return r != 0;
}

__global__ void __launch_bounds__(kWsThreads, 1) herk_ws_kernel(const float2* __restrict__ Psi, int64_t D, int64_t K,
                                                                int64_t tiles, float2* __restrict__ rho,
                                                                int32_t* __restrict__ err,
                                                                const __grid_constant__ CUtensorMap tm_rows,
                                                                const __grid_constant__ CUtensorMap tm_mirror) {
    extern __shared__ __align__(1024) unsigned char ws_smem[];
    unsigned char* stage0 = ws_smem;
    unsigned char* epi0 = ws_smem + (size_t)kWsStages * kTcStageBytes;
    WsBars* B = reinterpret_cast<WsBars*>(ws_smem + kWsBarOff);
    volatile int* abort = &B->abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nch = (int)(K / kTcChunk);                       // chunks per tile
    const int64_t nloc = tiles > blockIdx.x ? (tiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;   // this CTA's tiles
    const int64_t G = nloc * nch;                              // this CTA's chunks

    if (tid == 0) {
        for (int s = 0; s < kWsStages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&B->full[s])), "r"(kWsProd) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&B->empty[s])) : "memory");
        }
        for (int a = 0; a < 2; ++a) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&B->ready[a])) : "memory");
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(&B->freed[a])), "r"(kWsEpi) : "memory");
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&B->done)) : "memory");
        B->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kWsMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&B->tmem)),
                     "r"(kWsTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = B->tmem;

    if (warp >= kWsEpi / 32 && warp < kWsMmaWarp) {
        // ---- producers: k half `half` of row `row` of A (tile rows i0..) and of B (rows j0..) ----
        const int pt = tid - kWsEpi, row = pt >> 1, half = pt & 1;
        float4 pa[kWsAhead][2], pb[kWsAhead][2];
        // chunks are fetched in order: the next one is chunk f_c of this CTA's tile f_lt, whose
        // block coordinates are (f_bi, f_bj)
        int64_t f_lt = 0;
        int f_c = 0, f_bi = 0, f_bj = 0;
        if (nloc > 0) tri_tile((uint32_t)blockIdx.x, f_bi, f_bj);
        auto fetch = [&](float4 (&a)[2], float4 (&b)[2]) {
            const int bi = f_bi, bj = f_bj;
            const int64_t k = (int64_t)f_c * kTcChunk + 4 * half;
            const float4* sa = reinterpret_cast<const float4*>(Psi + ((int64_t)bi * kTcTile + row) * K + k);
            const float4* sb = reinterpret_cast<const float4*>(Psi + ((int64_t)bj * kTcTile + row) * K + k);
            a[0] = sa[0];
            a[1] = sa[1];
            b[0] = sb[0];
            b[1] = sb[1];
            if (++f_c == nch) {
                f_c = 0;
                if (++f_lt < nloc) tri_tile((uint32_t)(blockIdx.x + f_lt * gridDim.x), f_bi, f_bj);
            }
        };
        auto put = [&](int64_t g, const float4 (&a)[2], const float4 (&b)[2]) -> bool {
            const int s = (int)(g % kWsStages);
            const uint32_t ph = (uint32_t)((g / kWsStages) & 1);
            if (!ws_wait(su32(&B->empty[s]), ph ^ 1u, abort)) return false;   // its last MMAs are done
            unsigned char* st = stage0 + (size_t)s * kTcStageBytes;
            put_row4(st, row, half, a[0], a[1], false);
            put_row4(st + 4 * kTcPartBytes, row, half, b[0], b[1], true);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(su32(&B->full[s]));
            return true;
        };
#pragma unroll
        for (int e = 0; e < kWsAhead; ++e)
            if (e < G) fetch(pa[e], pb[e]);
        bool ok = true;
        for (int64_t g0 = 0; g0 < G && ok; g0 += kWsAhead) {
#pragma unroll
            for (int e = 0; e < kWsAhead; ++e) {
                const int64_t g = g0 + e;
                if (g >= G) break;
                if (!put(g, pa[e], pb[e])) {
                    ok = false;
                    break;
                }
                if (g + kWsAhead < G) fetch(pa[e], pb[e]);
            }
        }
    } else if (warp == kWsMmaWarp) {
        // ---- MMA issue: one thread ----
        if (lane == 0) {
            for (int64_t lt = 0; lt < nloc; ++lt) {
                const int a = (int)(lt & 1);
                if (!ws_wait(su32(&B->freed[a]), (uint32_t)(((lt >> 1) & 1) ^ 1), abort)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t dr = tmem + (uint32_t)(a * kTcTmemCols);
                bool ok = true;
                for (int c = 0; c < nch; ++c) {
                    const int64_t g = lt * nch + c;
                    const int s = (int)(g % kWsStages);
                    if (!ws_wait(su32(&B->full[s]), (uint32_t)((g / kWsStages) & 1), abort)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    issue_chunk(dr, su32(stage0 + (size_t)s * kTcStageBytes), c > 0 ? 1u : 0u);
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     su32(&B->empty[s]))
                                 : "memory");
                }
                if (!ok) break;
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 su32(&B->ready[a]))
                             : "memory");
            }
            // every MMA issued so far has completed once this commit arrives
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             su32(&B->done))
                         : "memory");
            const uint64_t t0 = gtimer();
            while (!mbar_done(su32(&B->done), 0u) && gtimer() - t0 <= kTcWaitNs) __nanosleep(32);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp w reads TMEM lanes 32 (w % 4).. (its thread's tile row r) and the
        // 8-column half w / 4 of each 16-column step ----
        const int q4 = warp & 3, hh = warp >> 2;
        const int r = 32 * q4 + lane;
        const int ci = r & 15;
        const uint64_t mr = reinterpret_cast<uint64_t>(&tm_rows);
        const uint64_t mm = reinterpret_cast<uint64_t>(&tm_mirror);
        int64_t q = 0;   // staging steps issued (buffer q & 1)
        for (int64_t lt = 0; lt < nloc; ++lt) {
            const int a = (int)(lt & 1);
            const bool ok = ws_wait(su32(&B->ready[a]), (uint32_t)((lt >> 1) & 1), abort);
            if (epi_any(!ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int bi, bj;
            tri_tile((uint32_t)(blockIdx.x + lt * gridDim.x), bi, bj);
            const int64_t i0 = (int64_t)bi * kTcTile, j0 = (int64_t)bj * kTcTile;
            const uint32_t tr = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(a * kTcTmemCols);
            for (int st = 0; st < kTcTile / 16; ++st) {
                const int col = 16 * st + 8 * hh;   // tile column of this thread's 8 values
                float vr[8], vi[8];
                if (bi != bj) {
                    unsigned char* buf = epi0 + (q & 1) * kWsEpiBytes;
                    if (tid == 0 && q >= 2) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
                    asm volatile("bar.sync 1, 256;" ::: "memory");   // this buffer's previous stores have read it
                    tmem_ld8(tr + (uint32_t)col, vr);
                    tmem_ld8(tr + (uint32_t)(kTcTile + col), vi);
                    if (st == kTcTile / 16 - 1) {   // the accumulator set is free for the tile after next
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        mbar_arrive(su32(&B->freed[a]));
                    }
                    // rows box: row r, 16-byte chunk cc (two complex) at chunk cc ^ (r & 7); this
                    // thread has chunks 4 hh .. 4 hh + 3
                    unsigned char* rb = buf + r * 128;
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int cc = 4 * hh + c;
                        *reinterpret_cast<float4*>(rb + ((cc ^ (r & 7)) << 4)) =
                            make_float4(vr[2 * c], vi[2 * c], vr[2 * c + 1], vi[2 * c + 1]);
                    }
                    // mirror boxes: box r / 16 (16 rows x 128 B), row jl = 8 hh + e, complex r % 16
                    unsigned char* mb = buf + 16384 + (r >> 4) * 2048;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int jl = 8 * hh + e;
                        *reinterpret_cast<float2*>(mb + jl * 128 + ((((ci >> 1) ^ (jl & 7))) << 4) + ((ci & 1) << 3)) =
                            make_float2(vr[e], -vi[e]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    asm volatile("bar.sync 1, 256;" ::: "memory");
                    if (tid == 0) {
                        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(mr),
                                     "r"((int)(2 * (j0 + 16 * st))), "r"((int)i0), "r"(su32(buf))
                                     : "memory");
                        for (int bx = 0; bx < 8; ++bx)
                            asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(mm),
                                         "r"((int)(2 * (i0 + 16 * bx))), "r"((int)(j0 + 16 * st)),
                                         "r"(su32(buf + 16384 + bx * 2048))
                                         : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    }
                    ++q;
                } else {
                    // diagonal tile: entries (i, j) with j >= i from registers, their mirrors, a
                    // real diagonal
                    tmem_ld8(tr + (uint32_t)col, vr);
                    tmem_ld8(tr + (uint32_t)(kTcTile + col), vi);
                    if (st == kTcTile / 16 - 1) {
                        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                        mbar_arrive(su32(&B->freed[a]));
                    }
                    const int64_t i = i0 + r;
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int cj = col + e;
                        const int64_t j = j0 + cj;
                        if (cj > r) {
                            rho[i * D + j] = make_float2(vr[e], vi[e]);
                            rho[j * D + i] = make_float2(vr[e], -vi[e]);
                        } else if (cj == r) {
                            rho[i * D + i] = make_float2(vr[e], 0.f);
                        }
                    }
                }
            }
        }
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");   // stores complete
    }
    if (tid == 0 && *abort) atomicExch(err, 3);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0 && *abort) atomicExch(err, 3);
    if (warp == kWsMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWsTmemCols) : "memory");
}

}  // namespace

// Tensor maps of rho (D x D complex64, viewed as float32 [D][2D]) for the TMA epilogue:
// boxes 32 floats (16 complex, 128 bytes) wide, 128 rows (rho[i][j]) or 16 rows (mirrors),
// 128-byte swizzle. The encoder is fetched from the driver through the runtime, so the
// library does not link libcuda. False (no TMA) when rho is not 16-byte aligned or the
// encoder is unavailable.
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static bool encode_rho_maps(float2* rho, int64_t D, CUtensorMap* rows, CUtensorMap* mirror) {
    if ((reinterpret_cast<uintptr_t>(rho) & 15u) != 0) return false;
    static const EncodeTiledFn fn = []() -> EncodeTiledFn {   // looked up once (thread-safe)
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        const bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                            cudaSuccess &&
                        q == cudaDriverEntryPointSuccess;
        cudaGetLastError();
        return ok ? reinterpret_cast<EncodeTiledFn>(f) : nullptr;
    }();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)(2 * D), (cuuint64_t)D};
    const cuuint64_t strides[1] = {(cuuint64_t)(8 * D)};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t box_rows[2] = {32, (cuuint32_t)kTcTile};
    const cuuint32_t box_mirror[2] = {32, 16};
    if (fn(rows, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rho, dims, strides, box_rows, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    if (fn(mirror, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, rho, dims, strides, box_mirror, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return false;
    return true;
}

// Tile and k-split plan shared by the workspace size and the launch: the tensor-core kernel
// for outputs of at least one 128-tile (m >= 7), the CUDA-core kernel below that; the k range
// is split (each split a whole number of chunks) while the launch still fits one wave (one CTA
// per SM for the tensor-core kernel, two for the CUDA-core one): every split adds a full
// partial output to write and sum. Long k ranges (>= 256 chunks a split) split further, up to
// two tensor-core CTAs per SM, whose epilogues then overlap the other CTA's MMAs.
struct HerkPlan {
    bool tc;
    int64_t tiles;
    int splits;
    int64_t kps;   // k values per split
};

static HerkPlan herk_plan(int n, int m, int sm_count) {
    HerkPlan P;
    P.tc = m >= 7;
    const int tile = P.tc ? kTcTile : kTileR;
    const int chunk = P.tc ? kTcChunk : kChunkK;
    const int64_t D = 1ll << m, K = 1ll << (n - m);
    const int64_t T = (D + tile - 1) / tile;
    P.tiles = T * (T + 1) / 2;
    int64_t s = 1;
    const int64_t wave = P.tc ? sm_count : 2ll * sm_count;
    while (K / (s * 2) >= 8 * chunk &&
           (P.tiles * s * 2 <= wave || (P.tc && P.tiles * s < 2ll * sm_count && K / (s * 2) >= 256 * chunk)))
        s *= 2;
    P.kps = ((K + s - 1) / s + chunk - 1) / chunk * chunk;
    P.splits = (int)((K + P.kps - 1) / P.kps);
    return P;
}

int herk_splits(int n, int m, int sm_count) { return herk_plan(n, m, sm_count).splits; }

size_t partial_trace_workspace_bytes(int n, int m, int sm_count) {
    const int s = herk_splits(n, m, sm_count);
    size_t b = ((size_t)8 << n) + 256;
    if (s > 1) b += (size_t)s * ((size_t)8 << (2 * m)) + 256;
    return b + 1024;
}

int launch_partial_trace(const void* psi_v, int n, const QubitMap& Q, int m, void* rho_v, void* workspace,
                         int sm_count, int32_t* err, void* stream, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    const float2* psi = (const float2*)psi_v;
    float2* rho = (float2*)rho_v;
    const int64_t D = 1ll << m, K = 1ll << (n - m);
    float2* Psi = (float2*)workspace;
    const HerkPlan P = herk_plan(n, m, sm_count);
    float2* partial = P.splits > 1 ? (float2*)((char*)workspace + (((size_t)8 << n) + 255) / 256 * 256) : nullptr;
    float2* dst = P.splits > 1 ? partial : rho;
    psi_gather_kernel<<<sm_count * 8, 256, 0, st>>>(psi, Psi, n, m, Q);
    dim3 grid((unsigned)P.tiles, (unsigned)P.splits);
    if (P.tc) {
        cudaError_t e = cudaFuncSetAttribute(herk_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmem);
        if (e != cudaSuccess) return (int)e;
        CUtensorMap tm_rows, tm_mirror;
        std::memset(&tm_rows, 0, sizeof(tm_rows));
        std::memset(&tm_mirror, 0, sizeof(tm_mirror));
        const int use_tma = P.splits == 1 && encode_rho_maps(rho, D, &tm_rows, &tm_mirror) ? 1 : 0;
        if (use_tma && n - m >= 3 && P.tiles >= sm_count) {
            // enough whole tiles for every SM: the persistent warp-specialised kernel
            e = cudaFuncSetAttribute(herk_ws_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmem);
            if (e != cudaSuccess) return (int)e;
            const unsigned g = (unsigned)(P.tiles < sm_count ? P.tiles : sm_count);
            herk_ws_kernel<<<g, kWsThreads, kWsSmem, st>>>(Psi, D, K, P.tiles, rho, err, tm_rows, tm_mirror);
        } else {
            herk_tc_kernel<<<grid, kTcThreads, kTcSmem, st>>>(Psi, D, K, P.kps, dst, err, tm_rows, tm_mirror, use_tma);
        }
    } else {
        herk_tile_kernel<<<grid, kHerkThreads, 0, st>>>(Psi, D, K, P.kps, dst);
    }
    int nl = 2;
    if (P.splits > 1) {
        herk_reduce_kernel<<<sm_count * 4, 256, 0, st>>>(partial, P.splits, D * D, rho);
        ++nl;
    }
    if (launches) *launches = nl;
    return (int)cudaGetLastError();
}

}  // namespace tlq
