// Dense statevector path on GB300: circuits whose two-qubit gates are not nearest-neighbour
// (e.g. QAOA on a random 3-regular graph). TensorLy-Quantum (arXiv:2112.10239) contrasts its
// factorised networks with the "traditional vector representation" of a state (Sec. 1);
// this file is that representation, tuned for HBM streaming.
//
// The 2^n complex64 state lives in HBM. Each layer (rotations, then commuting diagonal
// gates) is applied in passes over tiles of 2^12 amplitudes staged in shared memory:
//   * a low tile is 2^12 contiguous amplitudes (qubits 0..11);
//   * a strided tile keeps qubits 0..3 (16 contiguous amplitudes = 128 bytes per row) and
//     8 higher qubits a..a+7 as its 256 rows.
// Inside a tile the rotations on the tile's qubits run as 16-amplitude register passes
// (gates.cuh). The layer's diagonal gates are applied in the layer's last pass: RZ/RZZ gates
// sharing one angle form a class whose phase exp(-i a/2 (N - 2c)) depends only on the count
// c of "odd" terms, obtained with popcounts over per-distance masks and looked up in a small
// per-layer table; CZ gates contribute (-1)^(count of 11 pairs). The energy of Z/ZZ terms is
// accumulated in the final pass from the same counts; X/Y terms are measured by a separate
// streaming kernel. Reductions run in a fixed order, so results are deterministic.
// Layer 0 acts on |0..0>, so the forward starts from its product state written in one kernel
// and streams the remaining layers; the gradient's reverse passes (the adjoint) walk the
// fused schedule of all layers.
//
// The plain per-gate path (one full-state sweep per gate, per-term measurement sweeps, and
// for the gradient one sweep per gate and state) is kept as the baseline the fused passes are
// compared against.
#include "gates.cuh"
#include "tc.cuh"

#include <algorithm>
#include <cstdio>

namespace tlq {

namespace {

constexpr int kTile = 1 << kDenseTileBits;        // 4096 amplitudes
__host__ __device__ constexpr int padded_amps_c(int W) { return (1 << W) + (1 << (W - 3)); }
constexpr int kThreads = kTile / 16;                // 16 amplitudes per thread per register pass
constexpr int kMaxLayerClasses = kDenseMaxLayerClasses;
constexpr int kMaxDistWords = kDenseMaxDistWords;  // (d, mask) int pairs staged in shared memory
constexpr int kMaxTab = kDenseMaxTab;              // phase-table entries staged per layer

// Edge-word tables of XOR classes (see class_count): up to kEwTabs per pass, each four rows of
// 256 words over 8-bit chunks of the index, then the 32 per-qubit words they are built from.
// A row keeps one padding word per 16 entries, so that lanes reading entries 16 apart (the
// thread bases of a register group at bit 0) hit distinct banks.
constexpr int kEwTabs = 2;
constexpr int kEwRow = 256 + 16;
__host__ __device__ constexpr size_t ew_bytes(int ntabs) { return (size_t)ntabs * (4 * kEwRow + 32) * sizeof(uint64_t); }
__device__ __forceinline__ int ew_slot(uint32_t b) { return (int)(b + (b >> 4)); }

// ---- layer 0 as a product state ----------------------------------------------------------
//
// Layer 0 acts on |0..0>, so the state after it is written directly instead of streamed: a
// product of single-qubit factors, amplitude(x) = prod_q f_q(x_q) with f_q(0) = cos(a_q/2) and
// f_q(1) = sin(a_q/2) (RY) or -i sin(a_q/2) (RX), 1 and 0 for a qubit without a rotation; then
// layer 0's diagonal classes (phase exp(-i a/2 (N - 2c)) from the phase table, or the CZ sign
// (-1)^c). Sixteen consecutive amplitudes are built at once: the product over bits 4.. once,
// the low four bits by doubling, the classes by split counts over bits 0..3. The product over
// bits 4.. is four rows of per-chunk products (bits 4..11, 12..19, 20..27, 28..30), and one XOR
// class of at most 64 terms takes its count at the base index from the rows' edge-parity words
// (see class_count): both are linear over the chunks.
struct InitGates { int32_t gate[32]; };
struct InitRow {
    float2 f;      // product of the chunk's factors f_q(x_q)
    uint64_t w;    // edge-parity word of the chunk's bits for class InitStage::ewc
};

__device__ __forceinline__ float2 init_factor(const InitGates& I, const tlq_gate* gates, const float2* GT, int q,
                                              int bit) {
    const int g = I.gate[q];
    if (g < 0) return make_float2(bit ? 0.f : 1.f, 0.f);
    const float2 cs = GT[g];
    if (!bit) return make_float2(cs.x, 0.f);
    return gates[g].kind == TLQ_RY ? make_float2(cs.y, 0.f) : make_float2(0.f, -cs.y);
}

// Shared-memory staging of the product state's per-qubit factors and layer 0's classes.
struct InitStage {
    float2 f[32][2];
    DenseClassDev cls[kMaxLayerClasses];
    DensePassClassDev pcd[kMaxLayerClasses];
    int32_t dist[kMaxDistWords];
    int32_t woff[kMaxLayerClasses];
    int32_t toff[kMaxLayerClasses];
    float2 tab[kMaxTab];
    InitRow thr[256];     // bits 4..11: a thread's base in the generating register group
    InitRow hi[2][256];   // bits 12..19 and 20..27
    InitRow top[8];       // bits 28..30
    int nc;
    int staged;   // the phase tables fit: read from shared memory, else from global memory
    int ewc;      // the class counted from the rows' words (-1: none)
};

// Bit e of the result: term e of XOR class C (pairs in distance-mask order, then singles) is
// odd at index x. Linear over GF(2) in x, so the words of disjoint bit chunks XOR together.
__device__ uint64_t edge_parity(const DenseClassDev& C, const int32_t* dist, uint32_t x) {
    uint64_t w = 0;
    int e = 0;
    for (int k = 0; k < C.ndist; ++k) {
        const uint32_t M = (uint32_t)dist[2 * k + 1];
        const uint32_t odd = (x ^ (x >> dist[2 * k])) & M;
        for (uint32_t m = M; m; m &= m - 1u, ++e)
            if (odd & m & (0u - m)) w |= 1ull << e;
    }
    for (uint32_t m = C.single; m; m &= m - 1u, ++e)
        if (x & m & (0u - m)) w |= 1ull << e;
    return w;
}

// Stage the factors and layer 0's classes (every thread of the block calls this; ends with a
// barrier).
__device__ void stage_init(InitStage& S, int n_eff, const InitGates& I, const tlq_gate* gates, const float2* GT,
                           const DenseClassDev* classes, int cls_off, int ncls, const DensePassClassDev* pcd,
                           const int32_t* dists, const float2* ptab, int tid, int nthreads) {
    if (tid < 32) {
        S.f[tid][0] = tid < n_eff ? init_factor(I, gates, GT, tid, 0) : make_float2(1.f, 0.f);
        S.f[tid][1] = tid < n_eff ? init_factor(I, gates, GT, tid, 1) : make_float2(0.f, 0.f);
    }
    const int nc = ncls < kMaxLayerClasses ? ncls : kMaxLayerClasses;
    if (tid < nc) {
        S.cls[tid] = classes[cls_off + tid];
        S.pcd[tid] = pcd[tid];
    }
    __syncthreads();
    if (tid == 0) {
        int w = 0, t = 0, ewc = -1;
        for (int c = 0; c < nc; ++c) {
            S.woff[c] = w;
            w += 2 * S.cls[c].ndist;
            S.toff[c] = t;
            t += S.cls[c].kind == 0 ? S.cls[c].nterms + 1 : 0;
            if (ewc < 0 && S.cls[c].kind != 1 && S.cls[c].nterms <= 64 && w <= kMaxDistWords) ewc = c;
        }
        S.staged = t <= kMaxTab;
        S.nc = nc;
        S.ewc = ewc;
    }
    __syncthreads();
    for (int c = 0; c < nc; ++c) {
        for (int k = tid; k < 2 * S.cls[c].ndist; k += nthreads)
            if (S.woff[c] + k < kMaxDistWords) S.dist[S.woff[c] + k] = dists[2 * S.cls[c].dist_off + k];
        if (S.staged && S.cls[c].kind == 0)
            for (int e = tid; e <= S.cls[c].nterms; e += nthreads) S.tab[S.toff[c] + e] = ptab[S.cls[c].tab_off + e];
    }
    __syncthreads();
    // chunk rows: thr (bits 4..11), hi[0] (12..19), hi[1] (20..27), top (28..30)
    for (int e = tid; e < 3 * 256 + 8; e += nthreads) {
        const int chunk = e >> 8;   // 3: top
        const uint32_t b = (uint32_t)(e & 255);
        const int lo = 4 + 8 * chunk, nb = chunk < 3 ? 8 : 3;
        float2 f = make_float2(1.f, 0.f);
        for (int i = 0; i < nb; ++i) f = cmul(f, S.f[lo + i][(b >> i) & 1u]);
        const uint64_t w = S.ewc >= 0 ? edge_parity(S.cls[S.ewc], S.dist + S.woff[S.ewc], b << lo) : 0ull;
        InitRow& r = chunk == 0 ? S.thr[b] : chunk < 3 ? S.hi[chunk - 1][b] : S.top[b];
        r.f = f;
        r.w = w;
    }
    __syncthreads();
}

__device__ __forceinline__ int class_count(const DenseClassDev& c, const int32_t* dist, const uint64_t* ew,
                                           uint32_t x);
__device__ __forceinline__ void split_deltas(const DenseClassDev& C, const DensePassClassDev& pc, uint32_t xb,
                                             int (&Ak)[4]);
__device__ __forceinline__ int split_count(const DensePassClassDev& pc, int cnt0, const int (&Ak)[4], int j);

// The 16 amplitudes x0 | j (x0 a multiple of 16) of the state after layer 0.
__device__ __forceinline__ void gen16(const InitStage& S, const float2* ptab, uint32_t x0, float2 (&v)[16]) {
    const InitRow& r0 = S.thr[(x0 >> 4) & 255u];
    const InitRow& r1 = S.hi[0][(x0 >> 12) & 255u];
    const InitRow& r2 = S.hi[1][(x0 >> 20) & 255u];
    const InitRow& r3 = S.top[(x0 >> 28) & 7u];
    v[0] = cmul(cmul(r0.f, r1.f), cmul(r2.f, r3.f));
    const uint64_t W = r0.w ^ r1.w ^ r2.w ^ r3.w;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float2 f0 = S.f[k][0], f1 = S.f[k][1];
#pragma unroll
        for (int j = 0; j < (1 << k); ++j) {
            v[j | (1 << k)] = cmul(v[j], f1);
            v[j] = cmul(v[j], f0);
        }
    }
    for (int ci = 0; ci < S.nc; ++ci) {
        const DenseClassDev& C = S.cls[ci];
        const DensePassClassDev& pc = S.pcd[ci];
        const int cnt0 = ci == S.ewc ? __popcll(W) : class_count(C, S.dist + S.woff[ci], nullptr, x0);
        int Ak[4];
        split_deltas(C, pc, x0, Ak);
        const float2* tab = S.staged ? S.tab + S.toff[ci] : ptab + C.tab_off;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int cnt = split_count(pc, cnt0, Ak, j);
            if (C.kind == 0) v[j] = cmul(v[j], tab[cnt]);
            else if (cnt & 1) v[j] = make_float2(-v[j].x, -v[j].y);
        }
    }
}

struct PassArgs {
    DensePassDev pass;
    const DenseLayerDev* layers;
    const DenseClassDev* classes;
    const DensePassClassDev* pcd;
    const int32_t* stage;
    const int32_t* dists;
    int32_t energy_class_off, energy_nclass;
    const DenseZTermDev* zterms;
    int32_t n_zterms;
    const tlq_gate* gates;
    const float2* GT;       // gate table of this set
    const float2* ptab;     // phase tables of this set
    float2* state;
    int32_t n_eff;
    double* partial;        // per-CTA energy partials
    double* npartial;       // tensor-core passes: per-half <psi|psi> partials
    int32_t* err;           // kernel error word
    float2* lam;            // gradient mode, final pass: lam = (diagonal part of H) psi, else null
    // generating pass (dense_pass_kernel<true>): layer 0's product state replaces the input tiles
    InitGates init;
    int32_t init_class_off, init_nclass;
    const DensePassClassDev* init_pcd;
};

// Global amplitude index of local tile index t.
__device__ __forceinline__ uint32_t tile_x(const DensePassDev& p, uint32_t tile, uint32_t t) {
    if (!p.strided) return (tile << kDenseTileBits) | t;
    const uint32_t lo = tile & ((1u << (p.a - 4)) - 1u);
    const uint32_t hi = tile >> (p.a - 4);
    return (t & 15u) | (lo << 4) | ((t >> 4) << p.a) | (hi << (p.a + kDenseStridedBits));
}

// The global index of amplitude j of a register group at bit s is tile_x(base) + j * step:
// register bits map to consecutive global bits (s = 0: the tile's low 4 bits; s >= 4: in a
// strided tile, bits a + s - 4 ..).
__device__ __forceinline__ uint32_t tile_step(const DensePassDev& p, int s) {
    return (!p.strided || s == 0) ? (1u << s) : (1u << (s - 4 + p.a));
}

// Count of class c at index x. An XOR class (kind 0 or 2) with a staged edge-word table
// (c.ew >= 0) takes four table reads: number its terms e = 0..N-1 and let E_q be the word with
// bit e set for every term that contains qubit q; bit e of the XOR of E_q over the qubits set in
// x is then x_u ^ x_v for a pair term (u, v) and x_q for a single term, so the count is the
// popcount of that XOR, and row k of the table holds the XORs over the 256 values of bits
// 8k..8k+7. Otherwise, popcounts over the class's distance masks.
__device__ __forceinline__ int class_count(const DenseClassDev& c, const int32_t* dist, const uint64_t* ew,
                                           uint32_t x) {
    if (c.ew >= 0) {
        const uint64_t* T = ew + (size_t)c.ew * (4 * kEwRow);
        return __popcll(T[ew_slot(x & 255u)] ^ T[kEwRow + ew_slot((x >> 8) & 255u)] ^
                        T[2 * kEwRow + ew_slot((x >> 16) & 255u)] ^ T[3 * kEwRow + ew_slot(x >> 24)]);
    }
    int cnt;
    if (c.kind == 1) {
        cnt = 0;
        for (int k = 0; k < c.ndist; ++k) cnt += __popc((x & (x >> dist[2 * k])) & (uint32_t)dist[2 * k + 1]);
    } else {
        cnt = __popc(x & c.single);
        for (int k = 0; k < c.ndist; ++k) cnt += __popc((x ^ (x >> dist[2 * k])) & (uint32_t)dist[2 * k + 1]);
    }
    return cnt;
}

// ---- asynchronous tile copies ------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Each thread copies its 8 x 16 bytes (2 amplitudes each) of tile `t` into the padded
// shared buffer with cp.async (global -> shared without a register round trip), then
// commits them as one group.
// Copy k of a thread covers tile index i = 2 (tid + kThreads k): both its global index (the
// row bits t >> 4 advance by 2 kThreads / 16 per k) and its padded shared slot advance by a
// fixed step per k.
__device__ __forceinline__ void issue_tile(const DensePassDev& P, uint32_t t, const float2* state, float2* buf,
                                           int tid) {
    const uint32_t i0 = 2u * (uint32_t)tid;
    const float2* src = state + tile_x(P, t, i0);
    const uint32_t gstep = P.strided ? ((2u * kThreads / 16u) << P.a) : 2u * kThreads;
    uint32_t dst = smem_u32(buf + pad16((int)i0));
#pragma unroll
    for (int k = 0; k < kTile / 2 / kThreads; ++k) {
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
        src += gstep;
        dst += (uint32_t)(pad16(2 * kThreads) * sizeof(float2));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

__device__ __forceinline__ void wait_tiles() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// The 32 per-qubit edge words E_q of XOR class C (see class_count), from its distance masks.
__device__ void build_edge_words(const DenseClassDev& C, const int32_t* dists, uint64_t* E) {
    for (int q = 0; q < 32; ++q) E[q] = 0;
    int e = 0;
    for (int k = 0; k < C.ndist; ++k) {
        const int d = dists[2 * (C.dist_off + k)];
        for (uint32_t m = (uint32_t)dists[2 * (C.dist_off + k) + 1]; m; m &= m - 1u) {
            const int u = __ffs((int)m) - 1;   // pair (u, u + d)
            const uint64_t bit = 1ull << e++;
            E[u] ^= bit;
            if (u + d < 32) E[u + d] ^= bit;
        }
    }
    for (uint32_t m = C.single; m; m &= m - 1u) E[__ffs((int)m) - 1] ^= 1ull << e++;
}

// Stage a pass's classes (diagonal phases of the layers it completes, and the energy
// classes in the final pass) with their distance words, phase tables and split counts, and
// edge-word tables (s_ew, ew_bytes(n_ew)) for the first n_ew XOR classes of at most 64 terms.
// Called by every thread of the CTA; ends with a barrier.
template <int NT = kThreads>
__device__ void stage_classes(const DensePassDev& P, const DenseClassDev* classes, const DensePassClassDev* pcd,
                              const int32_t* stage, const int32_t* dists, const float2* ptab, DenseClassDev* s_cls,
                              DensePassClassDev* s_pcd, int32_t* s_woff, int32_t* s_toff, int32_t* s_dist,
                              float2* s_tab, uint64_t* s_ew, int n_ew, int tid) {
    const int nst = P.nstage;
    if (tid < nst) s_cls[tid] = classes[stage[P.stage_off + tid]];
    __syncthreads();
    if (tid == 0) {
        int woff = 0, toff = 0, slot = 0;
        for (int c = 0; c < nst; ++c) {
            s_woff[c] = woff;
            s_toff[c] = toff;
            woff += 2 * s_cls[c].ndist;
            toff += s_cls[c].kind == 0 ? s_cls[c].nterms + 1 : 0;
            const bool tab = s_cls[c].kind != 1 && s_cls[c].nterms <= 64 && slot < n_ew;
            s_cls[c].ew = tab ? slot++ : -1;
        }
    }
    for (int g = 0; g < P.ngroups; ++g)
        for (int k = tid; k < P.group_ncls[g]; k += NT) s_pcd[P.group_cls[g] + k] = pcd[P.group_pcd[g] + k];
    __syncthreads();
    uint64_t* s_eq = s_ew + (size_t)n_ew * 4 * kEwRow;   // [n_ew][32] per-qubit words
    if ((tid & 31) == 0 && (tid >> 5) < n_ew) {            // lane 0 of warp w: slot w (zero if unused)
        const int slot = tid >> 5;
        int c = 0;
        while (c < nst && s_cls[c].ew != slot) ++c;
        if (c < nst) build_edge_words(s_cls[c], dists, s_eq + 32 * slot);
        else for (int q = 0; q < 32; ++q) s_eq[32 * slot + q] = 0;
    }
    for (int c = 0; c < nst; ++c) {
        const DenseClassDev& C = s_cls[c];
        for (int w = tid; w < 2 * C.ndist; w += NT) s_dist[s_woff[c] + w] = dists[2 * C.dist_off + w];
        if (C.kind == 0)
            for (int e = tid; e <= C.nterms; e += NT) s_tab[s_toff[c] + e] = ptab[C.tab_off + e];
    }
    if (n_ew > 0) {
        __syncthreads();
        for (int i = tid; i < n_ew * 4 * 256; i += NT) {
            const int slot = i >> 10, k = (i >> 8) & 3, b = i & 255;
            const uint64_t* Eq = s_eq + 32 * slot + 8 * k;
            uint64_t w = 0;
            for (int t = 0; t < 8; ++t)
                if ((b >> t) & 1) w ^= Eq[t];
            s_ew[(size_t)slot * (4 * kEwRow) + k * kEwRow + ew_slot((uint32_t)b)] = w;
        }
    }
    __syncthreads();
}

// The rotations of a pass's register groups, staged once per CTA: kind (-1 where the group has
// no rotation on that bit) and (cos a/2, sin a/2) of slot 4 g + k. Ends without a barrier.
__device__ __forceinline__ void stage_group_gates(const DensePassDev& P, const tlq_gate* gates, const float2* GT,
                                                  int* s_gkind, float2* s_gcs, int tid) {
    if (tid < 4 * kDenseMaxGroups) {
        const int g = tid >> 2, k = tid & 3;
        int kind = -1;
        float2 cs = make_float2(1.f, 0.f);
        if (g < P.ngroups && ((P.group_mask[g] >> k) & 1u)) {
            const int gate = P.gate[g][k];
            kind = gates[gate].kind;
            cs = GT[gate];
        }
        s_gkind[tid] = kind;
        s_gcs[tid] = cs;
    }
}

// Split class count of amplitude j of a register pass: count(x_b | j) from the count at the
// thread's base index, the per-bit deltas A_k and the in-group pairs C[j] (see DensePassClassDev).
__device__ __forceinline__ void split_deltas(const DenseClassDev& C, const DensePassClassDev& pc, uint32_t xb,
                                             int (&Ak)[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int inter = __popc(xb & pc.N[k]);
        Ak[k] = C.kind == 1 ? inter : __popc(pc.N[k]) - 2 * inter + (int)((pc.single >> k) & 1u);
    }
}

__device__ __forceinline__ int split_count(const DensePassClassDev& pc, int cnt0, const int (&Ak)[4], int j) {
    const uint32_t cw = pc.C[j >> 2];
    int cnt = cnt0 + (int)((cw >> (8 * (j & 3))) & 255u);
    if (j & 1) cnt += Ak[0];
    if (j & 2) cnt += Ak[1];
    if (j & 4) cnt += Ak[2];
    if (j & 8) cnt += Ak[3];
    return cnt;
}

// After group g of a pass: the diagonal phases of a completed layer and/or the energy, from
// split class counts over the thread's 16 amplitudes v (register bits at s.., thread base index
// `base` in tile t_id); accumulates the energy into eacc and, in gradient mode, writes lam.
template <bool NORM = false>
__device__ __forceinline__ void group_epilogue(const PassArgs& A, const DensePassDev& P, int g, uint32_t t_id,
                                               int base, int s, float2 (&v)[16], float& eacc, float& nacc,
                                               const DenseClassDev* s_cls, const DensePassClassDev* s_pcd,
                                               const int32_t* s_woff, const int32_t* s_toff, const int32_t* s_dist,
                                               const float2* s_tab, const uint64_t* s_ew) {
    // after this group: diagonal phases of a completed layer and/or the energy, from split
    // class counts; the last group then writes straight to HBM from registers
    const int ncls = P.group_ncls[g];
    if (ncls > 0 || g == P.measure_group) {
        const uint32_t xb = tile_x(P, t_id, (uint32_t)base);   // register bits are zero in base
        float ez[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) ez[j] = 0.f;
        bool any_energy = g == P.measure_group;
        for (int ci = P.group_cls[g]; ci < P.group_cls[g] + ncls; ++ci) {
            const DenseClassDev& C = s_cls[ci];
            const DensePassClassDev& pc = s_pcd[ci];
            const int woff = s_woff[ci], toff = s_toff[ci];
            any_energy |= C.kind == 2;
            const int cnt0 = class_count(C, s_dist + woff, s_ew, xb);
            int Ak[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int inter = __popc(xb & pc.N[k]);
                Ak[k] = C.kind == 1 ? inter : __popc(pc.N[k]) - 2 * inter + (int)((pc.single >> k) & 1u);
            }
            const uint32_t cw0 = pc.C[0], cw1 = pc.C[1], cw2 = pc.C[2], cw3 = pc.C[3];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint32_t cw = (j >> 2) == 0 ? cw0 : (j >> 2) == 1 ? cw1 : (j >> 2) == 2 ? cw2 : cw3;
                int cnt = cnt0 + (int)((cw >> (8 * (j & 3))) & 255u);
                if (j & 1) cnt += Ak[0];
                if (j & 2) cnt += Ak[1];
                if (j & 4) cnt += Ak[2];
                if (j & 8) cnt += Ak[3];
                // phases multiply the amplitudes directly (|v|^2, and so the energy, does not
                // depend on their order; lam below takes the final amplitudes)
                if (C.kind == 0) v[j] = cmul(v[j], s_tab[toff + cnt]);
                else if (C.kind == 1) { if (cnt & 1) { v[j].x = -v[j].x; v[j].y = -v[j].y; } }
                else ez[j] += (float)C.coeff * (float)(C.nterms - 2 * cnt);
            }
        }
        const uint32_t xstep = tile_step(P, s);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (any_energy) {
                if (A.n_zterms > 0) {
                    const uint32_t x = xb + j * xstep;
                    for (int k = 0; k < A.n_zterms; ++k) {
                        const DenseZTermDev Z = A.zterms[k];
                        ez[j] += (__popc(x & Z.mask) & 1) ? -(float)Z.coeff : (float)Z.coeff;
                    }
                }
                const float pj = v[j].x * v[j].x + v[j].y * v[j].y;
                eacc += pj * ez[j];
                if (NORM) nacc += pj;
                if (A.lam)
                    A.lam[xb + j * xstep] = make_float2(ez[j] * v[j].x, ez[j] * v[j].y);
            }
        }
    }
}

// Persistent pass kernel: each CTA walks tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// in one of two forms. SINGLE: one shared-memory tile buffer and three CTAs per SM (80
// registers); once every thread holds its amplitudes of the last register pass, the cp.async
// copy of the CTA's next tile starts, and the other CTAs of the SM keep it busy meanwhile.
// Otherwise: two tile buffers and two CTAs per SM; the copy of the next tile runs while the
// current one is processed. Energy-only calls take the first form, the forward of a gradient
// call the second (measured faster for each). The last register pass writes its 16 amplitudes
// straight to HBM.
__host__ __device__ constexpr int dense_pass_bufs(bool single) { return single ? 1 : 2; }
__host__ __device__ constexpr int dense_pass_ctas(bool single) { return single ? 3 : 2; }
// The generating pass keeps no edge-word tables (its layer 0 staging takes their room).
__host__ __device__ constexpr int dense_pass_ew_tabs(bool gen) { return gen ? 0 : kEwTabs; }
__host__ __device__ constexpr size_t dense_pass_smem_base(bool single, bool gen) {
    return ((dense_pass_bufs(single) * (size_t)padded_amps_c(kDenseTileBits) * sizeof(float2) + kMaxTab * sizeof(float2) +
             kMaxDistWords * sizeof(int32_t) + kMaxLayerClasses * (sizeof(DenseClassDev) + sizeof(DensePassClassDev)) +
             2 * kMaxLayerClasses * sizeof(int32_t) + 16 * sizeof(float) + ew_bytes(dense_pass_ew_tabs(gen))) + 15) /
           16 * 16;
}

// GEN: the first forward pass of a low tile whose first group starts at bit 0 -- its input is
// layer 0's product state, generated in registers for group 0 (gen16) instead of read from HBM.
template <bool GEN, bool SINGLE>
__global__ void __launch_bounds__(kThreads, dense_pass_ctas(SINGLE)) dense_pass_kernel(const __grid_constant__ PassArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* bufs = reinterpret_cast<float2*>(smem_raw);                     // 1 or 2 x padded_amps(12)
    float2* s_tab = bufs + dense_pass_bufs(SINGLE) * padded_amps(kDenseTileBits);   // kMaxTab
    int32_t* s_dist = reinterpret_cast<int32_t*>(s_tab + kMaxTab);                   // kMaxDistWords
    DenseClassDev* s_cls = reinterpret_cast<DenseClassDev*>(s_dist + kMaxDistWords); // kMaxLayerClasses
    DensePassClassDev* s_pcd = reinterpret_cast<DensePassClassDev*>(s_cls + kMaxLayerClasses);
    int32_t* s_woff = reinterpret_cast<int32_t*>(s_pcd + kMaxLayerClasses);        // kMaxLayerClasses
    int32_t* s_toff = s_woff + kMaxLayerClasses;                                    // kMaxLayerClasses
    float* s_red = reinterpret_cast<float*>(s_toff + kMaxLayerClasses);              // 16
    uint64_t* s_ew = reinterpret_cast<uint64_t*>(s_red + 16);                       // ew_bytes(n_ew)
    constexpr int n_ew = dense_pass_ew_tabs(GEN);
    const DensePassDev& P = A.pass;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    InitStage* S = reinterpret_cast<InitStage*>(smem_raw + dense_pass_smem_base(SINGLE, GEN));   // GEN only
    const uint32_t ntiles = 1u << (A.n_eff - kDenseTileBits);

    __shared__ int s_gkind[4 * kDenseMaxGroups];
    __shared__ float2 s_gcs[4 * kDenseMaxGroups];
    if (!GEN && blockIdx.x < ntiles) issue_tile(P, blockIdx.x, A.state, bufs, tid);

    stage_group_gates(P, A.gates, A.GT, s_gkind, s_gcs, tid);   // visible after the barriers below
    stage_classes(P, A.classes, A.pcd, A.stage, A.dists, A.ptab, s_cls, s_pcd, s_woff, s_toff, s_dist, s_tab, s_ew,
                  n_ew, tid);
    if (GEN)
        stage_init(*S, A.n_eff, A.init, A.gates, A.GT, A.classes, A.init_class_off, A.init_nclass, A.init_pcd, A.dists,
                   A.ptab, tid, kThreads);

    float eacc = 0.f;
    int i = 0;
    for (uint32_t t_id = blockIdx.x; t_id < ntiles; t_id += gridDim.x, ++i) {
        float2* tile = bufs + (SINGLE ? 0 : (i & 1) * padded_amps(kDenseTileBits));
        if (!GEN) {
            wait_tiles();        // this thread's copies of tile t_id have landed
            __syncthreads();     // ... and everyone else's
            const uint32_t next = t_id + gridDim.x;
            if (!SINGLE && next < ntiles)
                issue_tile(P, next, A.state, bufs + ((i & 1) ^ 1) * padded_amps(kDenseTileBits), tid);
        }
        for (int g = 0; g < P.ngroups; ++g) {
            const int s = P.group_s[g];
            int kd[4];
            float c[4], sn[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                kd[k] = s_gkind[4 * g + k];
                const float2 v = s_gcs[4 * g + k];
                c[k] = v.x;
                sn[k] = v.y;
            }
            const int lowmask = (1 << s) - 1;
            const int base = (tid & lowmask) | ((tid >> s) << (s + 4));
            float2* p = tile + pad16(base);
            pk64 u[16];   // the 16 amplitudes as packed (re, im) registers
            if (GEN && g == 0) {   // s == 0
                float2 v[16];
                gen16(*S, A.ptab, tile_x(P, t_id, (uint32_t)base), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) u[j] = pk2(v[j].x, v[j].y);
            } else {
                load16ps(u, p, s);
            }
            if (SINGLE && g == P.ngroups - 1) {   // every thread holds its last amplitudes: the buffer is free
                __syncthreads();
                const uint32_t next = t_id + gridDim.x;
                if (!GEN && next < ntiles) issue_tile(P, next, A.state, bufs, tid);
            }
            if (kd[0] >= 0) apply_rot_p<0>(u, kd[0], c[0], sn[0]);
            if (kd[1] >= 0) apply_rot_p<1>(u, kd[1], c[1], sn[1]);
            if (kd[2] >= 0) apply_rot_p<2>(u, kd[2], c[2], sn[2]);
            if (kd[3] >= 0) apply_rot_p<3>(u, kd[3], c[3], sn[3]);
            if (P.group_ncls[g] > 0 || g == P.measure_group) {
                float2 v[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = upk2(u[j]);
                group_epilogue(A, P, g, t_id, base, s, v, eacc, eacc, s_cls, s_pcd, s_woff, s_toff, s_dist, s_tab,
                               s_ew);
#pragma unroll
                for (int j = 0; j < 16; ++j) u[j] = pk2(v[j].x, v[j].y);
            }
            if (g < P.ngroups - 1) {
                store16ps(u, p, s);
                __syncthreads();
            } else if (P.store) {
                pk64* dst = reinterpret_cast<pk64*>(A.state) + tile_x(P, t_id, (uint32_t)base);
                const uint32_t step = tile_step(P, s);
#pragma unroll
                for (int j = 0; j < 16; ++j) dst[j * step] = u[j];
            }
        }
        if (!SINGLE) __syncthreads();   // the buffer is free for the copy issued in the next iteration
    }
    if (P.measure_group >= 0) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) eacc += __shfl_xor_sync(0xffffffffu, eacc, off);
        if (lane == 0) s_red[warp] = eacc;
        __syncthreads();
        if (tid == 0) {
            float e = 0.f;
            for (int w = 0; w < kThreads / 32; ++w) e += s_red[w];
            A.partial[blockIdx.x] = (double)e;
        }
    }
}

size_t dense_pass_smem(bool single) { return dense_pass_smem_base(single, false); }

// The generating pass keeps layer 0's staging (InitStage) after the pass kernel's own data.
size_t dense_pass_gen_smem(bool single) { return dense_pass_smem_base(single, true) + sizeof(InitStage); }

// ---- tensor-core passes (mixed precision: split TF32 products, FP32 accumulation) ----------
//
// A register group's rotations (up to four, on the group's four tile bits) form one 16 x 16
// complex block U = R_3 (x) R_2 (x) R_1 (x) R_0 acting on a thread's 16 amplitudes, y = U a.
// Written in real arithmetic on a row of 32 reals [Re a_0..a_15 | Im a_0..a_15] this is one
// product with the 32 x 32 matrix M = [[Re U, -Im U], [Im U, Re U]]. On the tensor cores
// (tcgen05, kind::tf32, FP32 accumulators in tensor memory) a group is then one GEMM per 128
// rows of the tile: A = the rows (tensor memory, written by the threads with tcgen05.st),
// B = M in the K-major layout (shared memory), D = the rotated rows (tensor memory).
// FP32 accuracy comes from splitting both operands into TF32 parts, x = x_hi + x_lo with x_hi
// and x_lo rounded to TF32 (|x - x_hi - x_lo| <= 2^-22 |x|): D = A_hi [B_hi | B_lo] +
// A_lo B_hi, where [B_hi | B_lo] stacks the two parts of M along N (N = 64; the two 32-column
// halves of D are added when D is read back) and the dropped A_lo B_lo is at most 2^-22 of the
// product. The diagonal layers and the energy stay on the CUDA cores, unchanged.
//
// dense_tc_pass_kernel: one CTA per SM, 512 threads as two independent halves of 256 (named
// barriers 1 and 2), each streaming its own tiles (double-buffered with cp.async) through the
// pass's groups, as dense_pass_kernel does. The halves share the B operands of the pass's
// groups (8 KB each, built once per CTA from the gate table) and the staged class tables; each
// half owns 256 of the CTA's 512 tensor-memory columns: per 128-row chunk, A_hi (32 columns),
// A_lo (32) and D (64). One thread per half issues the 16 MMAs of a group (2 chunks x 4 K-steps
// x 2 products) and commits them to the half's mbarrier, which every thread of the half waits
// on (bounded: an MMA that has not completed after 1 s sets error word 4 and the CTA stops).

constexpr int kTcPassThreads = 2 * kThreads;
constexpr int kTcBlockBytes = 8192;       // one group's B: 4 K-steps x (64 rows x 8 TF32)
constexpr int kTcTmemCols = 512;
constexpr int kMaxSms = 1024;             // bound on the tensor-core pass grid (norm partials)

// Offsets in the dynamic shared memory of the tensor-core pass kernel for nblk B blocks:
// [0] tiles (2 halves x 2 buffers), [1] B blocks, [2] phase tables, [3] distance words,
// [4] classes, [5] split counts, [6] word offsets, [7] table offsets, [8] energy partials,
// [9] mbarriers, [10] tensor-memory address, [11] total.
__host__ __device__ inline void tc_pass_layout(int nblk, size_t (&off)[12]) {
    size_t o = 0;
    auto put = [&](int k, size_t bytes, size_t align) {
        o = (o + align - 1) / align * align;
        off[k] = o;
        o += bytes;
    };
    put(0, 4 * (size_t)padded_amps(kDenseTileBits) * sizeof(float2), 1024);
    put(1, (size_t)nblk * kTcBlockBytes, 1024);
    put(2, kMaxTab * sizeof(float2), 16);
    put(3, kMaxDistWords * sizeof(int32_t), 16);
    put(4, kMaxLayerClasses * sizeof(DenseClassDev), 16);
    put(5, kMaxLayerClasses * sizeof(DensePassClassDev), 16);
    put(6, kMaxLayerClasses * sizeof(int32_t), 16);
    put(7, kMaxLayerClasses * sizeof(int32_t), 16);
    put(8, 4 * (kThreads / 32) * sizeof(float), 16);
    put(9, 2 * sizeof(uint64_t), 8);
    put(10, sizeof(uint32_t), 4);
    off[11] = o;
}

// B operand of every rotation group of the pass: M = [[Re U, -Im U], [Im U, Re U]] (row n =
// output real, column k = input real), rounded TF32 parts in rows 0..31 (hi) and 32..63 (lo),
// K-major core matrices (8 rows x 16 bytes; 128 bytes apart along K, 256 along N), one 2 KB
// block per K-step of 8. Entries of U are products of the four 2 x 2 factors, in FP64 from the
// FP32 (cos, sin) of the gate table.
__device__ void build_tc_blocks(const DensePassDev& P, const tlq_gate* gates, const float2* GT, unsigned char* bblk,
                                int tid, int nthreads) {
    for (int e = tid; e < P.ngroups * 1024; e += nthreads) {
        const int g = e >> 10, n = (e >> 5) & 31, k = e & 31;
        const unsigned m = P.group_mask[g];
        if (m == 0) continue;
        const int i = n & 15, j = k & 15;
        double ur = 1.0, ui = 0.0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int ib = (i >> b) & 1, jb = (j >> b) & 1;
            double fr = ib == jb ? 1.0 : 0.0, fi = 0.0;
            if ((m >> b) & 1u) {
                const int gate = P.gate[g][b];
                const float2 cs = GT[gate];
                if (ib == jb) fr = (double)cs.x;
                else if (gates[gate].kind == TLQ_RY) fr = ib ? (double)cs.y : -(double)cs.y;   // [[c,-s],[s,c]]
                else { fr = 0.0; fi = -(double)cs.y; }                                           // [[c,-is],[-is,c]]
            }
            const double nr = ur * fr - ui * fi, ni = ur * fi + ui * fr;
            ur = nr;
            ui = ni;
        }
        const double mv = n < 16 ? (k < 16 ? ur : -ui) : (k < 16 ? ui : ur);
        const float mh = tc::tf32_rna((float)mv);
        const float ml = tc::tf32_rna((float)(mv - (double)mh));
        const int kk = k >> 3, kin = k & 7;
        const int o = g * kTcBlockBytes + kk * 2048 + (n >> 3) * 256 + (kin >> 2) * 128 + (n & 7) * 16 + (kin & 3) * 4;
        *reinterpret_cast<float*>(bblk + o) = mh;
        *reinterpret_cast<float*>(bblk + o + 4 * 256) = ml;   // row n + 32
    }
}

// The 16 MMAs of one group for one half: tm = the half's tensor-memory columns, b = the
// group's B block (shared address).
__device__ __forceinline__ void issue_group_mmas(uint32_t tm, uint32_t b) {
    constexpr uint32_t kN64 = tc::idesc_tf32(128, 64), kN32 = tc::idesc_tf32(128, 32);
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint64_t bd = tc::sdesc(b + kk * 2048, 128, 256);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t cb = tm + 128 * c;
            tc::mma_tf32_ts(cb + 64, cb + 8 * kk, bd, kN64, kk > 0 ? 1u : 0u);   // A_hi [B_hi | B_lo]
        }
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const uint64_t bd = tc::sdesc(b + kk * 2048, 128, 256);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const uint32_t cb = tm + 128 * c;
            tc::mma_tf32_ts(cb + 64, cb + 32 + 8 * kk, bd, kN32, 1u);              // A_lo B_hi
        }
    }
}

// Rotate the thread's 16 amplitudes by group g's block on the tensor cores (every thread of
// the half calls this). taddr = this thread's lanes and chunk columns; tm = the half's
// columns; returns false (uniformly over the half) when the MMAs did not complete in time.
__device__ __forceinline__ bool tc_rotate(float2 (&v)[16], uint32_t taddr, uint32_t tm, uint32_t bblock, int th,
                                          int bar_id, uint64_t* bar, uint32_t& phase) {
    float hi[16], lo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        hi[j] = tc::tf32_rna(v[j].x);
        lo[j] = tc::tf32_rna(v[j].x - hi[j]);
    }
    tc::tmem_st16(taddr + 0, hi);
    tc::tmem_st16(taddr + 32, lo);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        hi[j] = tc::tf32_rna(v[j].y);
        lo[j] = tc::tf32_rna(v[j].y - hi[j]);
    }
    tc::tmem_st16(taddr + 16, hi);
    tc::tmem_st16(taddr + 48, lo);
    tc::tmem_wait_st();
    tc::fence_before();
    tc::bar_sync(bar_id, kThreads);
    if (th == 0) {
        tc::fence_after();
        issue_group_mmas(tm, bblock);
        tc::commit(bar);
    }
    const bool ok = tc::mbar_wait(bar, phase);
    phase ^= 1u;
    if (tc::bar_or(bar_id, kThreads, !ok)) return false;
    tc::fence_after();
    float d0[16], d1[16];
    tc::tmem_ld16x2(taddr + 64, taddr + 96, d0, d1);    // Re y: A B_hi part, A_hi B_lo part
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j].x = d0[j] + d1[j];
    tc::tmem_ld16x2(taddr + 80, taddr + 112, d0, d1);   // Im y
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j].y = d0[j] + d1[j];
    tc::fence_before();   // the loads are ordered before the next group's MMAs by the next barrier
    return true;
}

__global__ void __launch_bounds__(kTcPassThreads, 1) dense_tc_pass_kernel(const __grid_constant__ PassArgs A, int nblk) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    size_t off[12];
    tc_pass_layout(nblk, off);
    float2* tiles = reinterpret_cast<float2*>(smem_raw + off[0]);
    unsigned char* bblk = smem_raw + off[1];
    float2* s_tab = reinterpret_cast<float2*>(smem_raw + off[2]);
    int32_t* s_dist = reinterpret_cast<int32_t*>(smem_raw + off[3]);
    DenseClassDev* s_cls = reinterpret_cast<DenseClassDev*>(smem_raw + off[4]);
    DensePassClassDev* s_pcd = reinterpret_cast<DensePassClassDev*>(smem_raw + off[5]);
    int32_t* s_woff = reinterpret_cast<int32_t*>(smem_raw + off[6]);
    int32_t* s_toff = reinterpret_cast<int32_t*>(smem_raw + off[7]);
    float* s_red = reinterpret_cast<float*>(smem_raw + off[8]);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + off[9]);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem_raw + off[10]);
    const DensePassDev& P = A.pass;
    const int tid = threadIdx.x;
    const int h = tid >> 8, th = tid & (kThreads - 1);   // half, thread within the half
    const int warp = tid >> 5, lane = tid & 31;
    const int bar_id = 1 + h;
    const uint32_t ntiles = 1u << (A.n_eff - kDenseTileBits);
    const uint32_t first = 2u * blockIdx.x + (uint32_t)h, step = 2u * gridDim.x;
    float2* buf0 = tiles + 2 * h * padded_amps(kDenseTileBits);

    if (first < ntiles) issue_tile(P, first, A.state, buf0, th);
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(tslot, kTcTmemCols);
    build_tc_blocks(P, A.gates, A.GT, bblk, tid, kTcPassThreads);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // B is read by the tensor core
    stage_classes<kTcPassThreads>(P, A.classes, A.pcd, A.stage, A.dists, A.ptab, s_cls, s_pcd, s_woff, s_toff,
                                  s_dist, s_tab, nullptr, 0, tid);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    const uint32_t tmem = *tslot;
    const uint32_t tm = tmem + 256u * (uint32_t)h;                       // this half's columns
    const uint32_t taddr = tm + 128u * (uint32_t)(th >> 7) + ((uint32_t)(32 * (warp & 3)) << 16);
    const uint32_t bbase = tc::su32(bblk);
    uint32_t phase = 0;
    bool bad = false;

    float eacc = 0.f, nacc = 0.f;
    int i = 0;
    for (uint32_t t_id = first; t_id < ntiles && !bad; t_id += step, ++i) {
        const int b = i & 1;
        float2* tile = buf0 + b * padded_amps(kDenseTileBits);
        wait_tiles();
        tc::bar_sync(bar_id, kThreads);
        const uint32_t next = t_id + step;
        if (next < ntiles) issue_tile(P, next, A.state, buf0 + (b ^ 1) * padded_amps(kDenseTileBits), th);
        for (int g = 0; g < P.ngroups; ++g) {
            const int s = P.group_s[g];
            const int stride = pass_stride(s);
            const int base = (th & ((1 << s) - 1)) | ((th >> s) << (s + 4));
            float2* p = tile + pad16(base);
            float2 v[16];
            load16(v, p, stride);
            if (P.group_mask[g] != 0 &&
                !tc_rotate(v, taddr, tm, bbase + (uint32_t)(g * kTcBlockBytes), th, bar_id, &bars[h], phase)) {
                bad = true;
                break;
            }
            group_epilogue<true>(A, P, g, t_id, base, s, v, eacc, nacc, s_cls, s_pcd, s_woff, s_toff, s_dist, s_tab,
                                 nullptr);
            if (g < P.ngroups - 1) {
                store16(v, p, stride);
                tc::bar_sync(bar_id, kThreads);
            } else if (P.store) {
#pragma unroll
                for (int j = 0; j < 16; ++j) A.state[tile_x(P, t_id, (uint32_t)(base | (j << s)))] = v[j];
            }
        }
        if (!bad) tc::bar_sync(bar_id, kThreads);   // the buffer is free for the next copy
    }
    wait_tiles();   // no copy of this thread is left in flight
    if (P.measure_group >= 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            eacc += __shfl_xor_sync(0xffffffffu, eacc, o);
            nacc += __shfl_xor_sync(0xffffffffu, nacc, o);
        }
        if (lane == 0) {
            s_red[h * (kThreads / 32) + (warp & 7)] = eacc;
            s_red[2 * (kThreads / 32) + h * (kThreads / 32) + (warp & 7)] = nacc;
        }
        tc::bar_sync(bar_id, kThreads);
        if (th == 0) {
            float e = 0.f, nn = 0.f;
            for (int w = 0; w < kThreads / 32; ++w) {
                e += s_red[h * (kThreads / 32) + w];
                nn += s_red[2 * (kThreads / 32) + h * (kThreads / 32) + w];
            }
            A.partial[(size_t)h * gridDim.x + blockIdx.x] = (double)e;
            A.npartial[(size_t)h * gridDim.x + blockIdx.x] = (double)nn;   // <psi|psi> partials
        }
    }
    if (bad) {
        if (th == 0) {
            atomicOr(A.err, 4);
            tc::mbar_wait(&bars[h], phase ^ 1u);   // the group's MMAs, once more (bounded)
        }
    }
    tc::fence_before();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTcTmemCols);
}

// ---- adjoint passes (gradient) ----------------------------------------------------------------
//
// The gradient follows the adjoint method: with lam = H psi at the end of the circuit, walk the
// gates backwards; a gate exp(-i a G/2) contributes dE/da = Im <lam|G|psi> with both states
// taken right after it, then is un-applied to both. Gates that commute with G may sit between
// that point and the one where the sum is taken, which lets a whole register group (rotations on
// four distinct qubits) and a whole diagonal layer be handled at once:
//   * diagonal class with angle a: sum_x Im(conj(lam_x) psi_x) (N - 2c(x)), then both states
//     times the conjugate phase (the sum is unchanged by a common phase, so its order is free);
//   * RX / RY on register bit k: the pair sums of gates.cuh, then the inverse rotation.
// One adjoint kernel reverses one forward pass: groups in reverse order, each group's diagonal
// classes before its rotations. psi and lam tiles share the CTA's shared memory (one buffer
// each); the next tile's copies start as soon as the last group has read its registers.

struct AdjArgs {
    DensePassDev pass;
    const DenseClassDev* classes;
    const DensePassClassDev* pcd;
    const int32_t* stage;
    const int32_t* dists;
    const tlq_gate* gates;
    const float2* GT;       // gate table of this set
    const float2* ptab;     // phase tables of this set
    float2* psi;
    float2* lam;
    int32_t n_eff;
    double* gpart;          // [kDenseAdjSlots][gridDim.x] gradient partials of this pass
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) x += __shfl_xor_sync(0xffffffffu, x, off);
    return x;
}

// The thread's share of Im<lam|G|psi> for the rotation on register bit K (kind and
// (cos a/2, sin a/2) from the staged group gates), which is then un-applied from psi and lam.
template <int K>
__device__ __forceinline__ float adjoint_bit(int kind, float2 cs, float2 (&v)[16], float2 (&u)[16]) {
    return adjoint_rot<K, float2, float>(v, u, kind, cs.x, -cs.y);
}

// Layer-0 rotation on register bit K: gradient only (see DensePassDev::group_rot0).
template <int K>
__device__ __forceinline__ float gradient_bit(int kind, const float2 (&v)[16], const float2 (&u)[16]) {
    return kind == TLQ_RY ? grad_y<K, float2, float>(v, u) : grad_x<K, float2, float>(v, u);
}

__global__ void __launch_bounds__(kThreads, 2) dense_adjoint_kernel(const __grid_constant__ AdjArgs A) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2* bpsi = reinterpret_cast<float2*>(smem_raw);                               // padded_amps(12)
    float2* blam = bpsi + padded_amps(kDenseTileBits);                                // padded_amps(12)
    double* s_gacc = reinterpret_cast<double*>(blam + padded_amps(kDenseTileBits));   // [warps][slots]
    float2* s_tab = reinterpret_cast<float2*>(s_gacc + (kThreads / 32) * kDenseAdjSlots);
    int32_t* s_dist = reinterpret_cast<int32_t*>(s_tab + kMaxTab);
    DenseClassDev* s_cls = reinterpret_cast<DenseClassDev*>(s_dist + kMaxDistWords);
    DensePassClassDev* s_pcd = reinterpret_cast<DensePassClassDev*>(s_cls + kMaxLayerClasses);
    int32_t* s_woff = reinterpret_cast<int32_t*>(s_pcd + kMaxLayerClasses);
    int32_t* s_toff = s_woff + kMaxLayerClasses;
    uint64_t* s_ew = reinterpret_cast<uint64_t*>(s_toff + kMaxLayerClasses);   // ew_bytes(kEwTabs)
    const DensePassDev& P = A.pass;
    const int tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const uint32_t ntiles = 1u << (A.n_eff - kDenseTileBits);

    if (blockIdx.x < ntiles) {
        issue_tile(P, blockIdx.x, A.psi, bpsi, tid);
        issue_tile(P, blockIdx.x, A.lam, blam, tid);
    }
    for (int k = tid; k < (kThreads / 32) * kDenseAdjSlots; k += kThreads) s_gacc[k] = 0.0;
    __shared__ int s_gkind[4 * kDenseMaxGroups];
    __shared__ float2 s_gcs[4 * kDenseMaxGroups];
    stage_group_gates(P, A.gates, A.GT, s_gkind, s_gcs, tid);   // visible after the barriers below
    stage_classes(P, A.classes, A.pcd, A.stage, A.dists, A.ptab, s_cls, s_pcd, s_woff, s_toff, s_dist, s_tab, s_ew,
                  kEwTabs, tid);
    double* acc = s_gacc + warp * kDenseAdjSlots;   // written by one lane of this warp per slot

    for (uint32_t t_id = blockIdx.x; t_id < ntiles; t_id += gridDim.x) {
        wait_tiles();
        __syncthreads();
        for (int g = P.ngroups - 1; g >= 0; --g) {
            const int s = P.group_s[g];
            const int stride = pass_stride(s);
            const int base = (tid & ((1 << s) - 1)) | ((tid >> s) << (s + 4));
            float2 v[16], u[16];
            load16s(v, bpsi + pad16(base), s);
            load16s(u, blam + pad16(base), s);
            if (g == 0) {
                __syncthreads();   // every thread holds its amplitudes: both buffers are free
                const uint32_t next = t_id + gridDim.x;
                if (next < ntiles) {
                    issue_tile(P, next, A.psi, bpsi, tid);
                    issue_tile(P, next, A.lam, blam, tid);
                }
            }
            // the diagonal classes applied after this group in the forward pass
            const int ncls = P.group_ncls[g];
            if (ncls > 0) {
                const uint32_t xb = tile_x(P, t_id, (uint32_t)base);
                for (int ci = P.group_cls[g]; ci < P.group_cls[g] + ncls; ++ci) {
                    const DenseClassDev& C = s_cls[ci];
                    if (C.kind == 2) continue;   // energy classes: nothing to undo
                    const DensePassClassDev& pc = s_pcd[ci];
                    const int cnt0 = class_count(C, s_dist + s_woff[ci], s_ew, xb);
                    int Ak[4];
                    split_deltas(C, pc, xb, Ak);
                    if (C.kind == 0) {
                        const int toff = s_toff[ci];
                        float gsum = 0.f;
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const int cnt = split_count(pc, cnt0, Ak, j);
                            gsum += (u[j].x * v[j].y - u[j].y * v[j].x) * (float)(C.nterms - 2 * cnt);
                            float2 ph = s_tab[toff + cnt];
                            ph.y = -ph.y;
                            v[j] = cmul(v[j], ph);
                            u[j] = cmul(u[j], ph);
                        }
                        gsum = warp_sum(gsum);
                        if (lane == 0) acc[4 * kDenseMaxGroups + ci] += (double)gsum;
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            if (split_count(pc, cnt0, Ak, j) & 1) {
                                v[j].x = -v[j].x;
                                v[j].y = -v[j].y;
                                u[j].x = -u[j].x;
                                u[j].y = -u[j].y;
                            }
                        }
                    }
                }
            }
            // the group's rotations: gradient, then the inverse rotation on both states; layer 0's
            // rotations commute and nothing after them needs the state, so they only give gradients
            const unsigned m = P.group_mask[g];
            float g0 = 0.f, g1 = 0.f, g2 = 0.f, g3 = 0.f;
            const int* gk = s_gkind + 4 * g;
            const float2* gcs = s_gcs + 4 * g;
            if ((P.group_rot0 >> g) & 1u) {
                if (m & 1u) g0 = gradient_bit<0>(gk[0], v, u);
                if (m & 2u) g1 = gradient_bit<1>(gk[1], v, u);
                if (m & 4u) g2 = gradient_bit<2>(gk[2], v, u);
                if (m & 8u) g3 = gradient_bit<3>(gk[3], v, u);
            } else {
                if (m & 1u) g0 = adjoint_bit<0>(gk[0], gcs[0], v, u);
                if (m & 2u) g1 = adjoint_bit<1>(gk[1], gcs[1], v, u);
                if (m & 4u) g2 = adjoint_bit<2>(gk[2], gcs[2], v, u);
                if (m & 8u) g3 = adjoint_bit<3>(gk[3], gcs[3], v, u);
            }
            {   // the group's four warp sums in one transposing reduction: lane 8 k holds bit k's
                const float gk = warp_sum4(g0, g1, g2, g3, lane);
                const int k = lane >> 3;
                if ((lane & 7) == 0 && ((m >> k) & 1u)) acc[4 * g + k] += (double)gk;
            }
            if (g > 0) {
                store16s(v, bpsi + pad16(base), s);
                store16s(u, blam + pad16(base), s);
                __syncthreads();
            } else if (P.store) {
                const uint32_t x0 = tile_x(P, t_id, (uint32_t)base), step = tile_step(P, s);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    A.psi[x0 + j * step] = v[j];
                    A.lam[x0 + j * step] = u[j];
                }
            }
        }
    }
    __syncthreads();
    for (int k = tid; k < kDenseAdjSlots; k += kThreads) {
        double sum = 0.0;
        for (int w = 0; w < kThreads / 32; ++w) sum += s_gacc[w * kDenseAdjSlots + k];
        A.gpart[(size_t)k * gridDim.x + blockIdx.x] = sum;
    }
}

size_t dense_adjoint_smem() {
    return 2 * (size_t)padded_amps(kDenseTileBits) * sizeof(float2) +
           (size_t)(kThreads / 32) * kDenseAdjSlots * sizeof(double) + kMaxTab * sizeof(float2) +
           kMaxDistWords * sizeof(int32_t) + kMaxLayerClasses * (sizeof(DenseClassDev) + sizeof(DensePassClassDev)) +
           2 * kMaxLayerClasses * sizeof(int32_t) + ew_bytes(kEwTabs);
}

// lam (+)= sum_t c_t P_t psi over Pauli strings given by (flip, zy, ny):
// (P psi)_x = (-i)^ny (-1)^popc(x & zy) psi_{x ^ flip}.
__global__ void lambda_terms_kernel(const float2* psi, float2* lam, uint64_t N, const DenseXTermDev* terms, int nterms,
                                    int accumulate) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
        float2 out = accumulate ? lam[x] : make_float2(0.f, 0.f);
        for (int t = 0; t < nterms; ++t) {
            const DenseXTermDev T = terms[t];
            const int q = T.ny & 3;
            const float2 f0 = make_float2(q == 0 ? 1.f : q == 2 ? -1.f : 0.f, q == 1 ? -1.f : q == 3 ? 1.f : 0.f);
            float2 v = cmul(f0, psi[x ^ T.flip]);
            const float c = (__popc((uint32_t)x & T.zy) & 1) ? -(float)T.coeff : (float)T.coeff;
            out.x += c * v.x;
            out.y += c * v.y;
        }
        lam[x] = out;
    }
}

// grad[p] = sum over the entries of parameter p of sum over CTAs of the pass partials, one warp
// per parameter; each lane sums a fixed subset in order, then a fixed shuffle tree.
__global__ void dense_grad_reduce_kernel(const double* gpart, int grid, const int32_t* off, const int32_t* idx,
                                         int n_params, double* grad) {
    const int p = (int)((blockIdx.x * (uint32_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (p >= n_params) return;
    double s = 0.0, c = 0.0;   // Neumaier
    for (int e = off[p]; e < off[p + 1]; ++e) {
        const double* row = gpart + (size_t)idx[e] * grid;
        for (int k = lane; k < grid; k += 32) {
            const double x = row[k];
            const double t = s + x;
            if (fabs(s) >= fabs(x)) c += (s - t) + x;
            else c += (x - t) + s;
            s = t;
        }
    }
    double v = s + c;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) grad[p] = v;
}

// ---- gate tables and phase tables ---------------------------------------------------------

__global__ void dense_gate_table_kernel(const tlq_gate* gates, int n_gates, const double* theta, int n_params,
                                        float2* out) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_gates) return;
    const tlq_gate G = gates[g];
    const double a = G.param >= 0 ? theta[G.param] : G.angle;
    double s, c;
    sincos(0.5 * a, &s, &c);
    out[g] = make_float2((float)c, (float)s);
}

// entry e: exp(-i a/2 * mult[e]) with a the angle of gate tab_gate[e]
__global__ void dense_phase_table_kernel(const tlq_gate* gates, const int32_t* tab_gate, const int32_t* tab_mult,
                                         int entries, const double* theta, float2* out) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= entries) return;
    const tlq_gate G = gates[tab_gate[e]];
    const double a = G.param >= 0 ? theta[G.param] : G.angle;
    double s, c;
    sincos(0.5 * a * (double)tab_mult[e], &s, &c);
    out[e] = make_float2((float)c, (float)-s);
}

// ---- measurement of one Pauli term (X/Y letters, or any term on the per-gate path) ---------

constexpr int kMeasBlocks = 1024;
constexpr int kMeasThreads = 256;

__global__ void __launch_bounds__(kMeasThreads) term_measure_kernel(const float2* psi, uint64_t N, uint32_t flip,
                                                                    uint32_t zy, int ny, double* partial) {
    float2 f0;   // (-i)^ny
    const int q = ny & 3;
    f0.x = q == 0 ? 1.f : q == 2 ? -1.f : 0.f;
    f0.y = q == 1 ? -1.f : q == 3 ? 1.f : 0.f;
    float acc = 0.f;
    for (uint64_t x = (uint64_t)blockIdx.x * kMeasThreads + threadIdx.x; x < N; x += (uint64_t)gridDim.x * kMeasThreads) {
        const float2 a = psi[x];
        const float2 v = psi[x ^ flip];
        float2 t = cmul(f0, v);
        if (__popc((uint32_t)x & zy) & 1) { t.x = -t.x; t.y = -t.y; }
        acc += a.x * t.x + a.y * t.y;
    }
    __shared__ float red[kMeasThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = 0.f;
        for (int w = 0; w < kMeasThreads / 32; ++w) e += red[w];
        partial[blockIdx.x] = (double)e;
    }
}

struct Neumaier {
    double s = 0, c = 0;
    __device__ void add(double x) {
        const double t = s + x;
        if (fabs(s) >= fabs(x)) c += (s - t) + x;
        else c += (x - t) + s;
        s = t;
    }
    __device__ double value() const { return s + c; }
};

// out[0] (+)= coeff * sum of partial[0..n) in fixed order
// One warp: lane l sums partials l, l + 32, ... (compensated), then lane 0 adds the 32 lane
// sums in lane order after the value already in *out; the order is fixed, whatever the launch.
__global__ void reduce_partials_kernel(const double* partial, int n, double coeff, double* out, int accumulate) {
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    const int lane = threadIdx.x;
    Neumaier mine;
    for (int i = lane; i < n; i += 32) mine.add(coeff * partial[i]);
    const double v = mine.value();
    Neumaier acc;
    if (lane == 0 && accumulate) acc.add(*out);
    for (int l = 0; l < 32; ++l) {
        const double x = __shfl_sync(0xffffffffu, v, l);
        if (lane == 0) acc.add(x);
    }
    if (lane == 0) *out = acc.value();
}

// Tensor-core mode: divide the energy (and the gradient) by <psi|psi> = sum of the norm
// partials (FP64, fixed order). In exact arithmetic the state has unit norm and nothing
// changes; the tensor cores' FP32 accumulation truncates, which shrinks the state by a nearly
// uniform factor over the passes, and the ratio cancels that factor to first order.
__global__ void normalize_kernel(const double* npart, int n, double* energy, double* grad, int n_params) {
    __shared__ double s_norm;
    if (threadIdx.x == 0) {
        Neumaier acc;
        for (int i = 0; i < n; ++i) acc.add(npart[i]);
        s_norm = acc.value();
    }
    __syncthreads();
    const double inv = 1.0 / s_norm;
    if (threadIdx.x == 0) *energy *= inv;
    if (grad)
        for (int p = threadIdx.x; p < n_params; p += blockDim.x) grad[p] *= inv;
}

// ---- plain per-gate sweeps (baseline) -----------------------------------------------------

// sgn = -1 applies the inverse rotation (adjoint sweep)
__global__ void pergate_rot_kernel(float2* psi, uint64_t half, int q, int kind, const float2* GT, int gate, float sgn) {
    const float2 cs = GT[gate];
    const float c = cs.x, s = sgn * cs.y;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < half; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x0 = ((i >> q) << (q + 1)) | (i & ((1ull << q) - 1));
        const uint64_t x1 = x0 | (1ull << q);
        const float2 a0 = psi[x0], a1 = psi[x1];
        float2 b0, b1;
        if (kind == TLQ_RY) {
            b0 = make_float2(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
            b1 = make_float2(s * a0.x + c * a1.x, s * a0.y + c * a1.y);
        } else {
            b0 = make_float2(c * a0.x + s * a1.y, c * a0.y - s * a1.x);
            b1 = make_float2(c * a1.x + s * a0.y, c * a1.y - s * a0.x);
        }
        psi[x0] = b0;
        psi[x1] = b1;
    }
}

__global__ void pergate_diag_kernel(float2* psi, uint64_t N, int kind, int q0, int q1, const float2* GT, int gate,
                                    float sgn) {
    float2 f0 = make_float2(1.f, 0.f), f1 = f0;
    if (kind != TLQ_CZ) {
        const float2 cs = GT[gate];
        f0 = make_float2(cs.x, -sgn * cs.y);   // z = +1
        f1 = make_float2(cs.x, sgn * cs.y);    // z = -1
    }
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
        const int b0 = (int)((x >> q0) & 1);
        if (kind == TLQ_RZ) {
            psi[x] = cmul(psi[x], b0 ? f1 : f0);
        } else {
            const int b1 = (int)((x >> q1) & 1);
            if (kind == TLQ_CZ) {
                if (b0 & b1) { float2 v = psi[x]; psi[x] = make_float2(-v.x, -v.y); }
            } else {
                psi[x] = cmul(psi[x], (b0 ^ b1) ? f1 : f0);
            }
        }
    }
}

// Im <lam| G |psi> of one gate over the whole state (G = X_q, Y_q, Z_q or Z_q0 Z_q1), per block.
__global__ void __launch_bounds__(kMeasThreads) pergate_grad_kernel(const float2* psi, const float2* lam, uint64_t N,
                                                                    int kind, int q0, int q1, double* partial) {
    float acc = 0.f;
    if (kind == TLQ_RX || kind == TLQ_RY) {
        const uint64_t half = N / 2;
        for (uint64_t i = (uint64_t)blockIdx.x * kMeasThreads + threadIdx.x; i < half;
             i += (uint64_t)gridDim.x * kMeasThreads) {
            const uint64_t x0 = ((i >> q0) << (q0 + 1)) | (i & ((1ull << q0) - 1));
            const uint64_t x1 = x0 | (1ull << q0);
            const float2 p0 = psi[x0], p1 = psi[x1], l0 = lam[x0], l1 = lam[x1];
            if (kind == TLQ_RY) acc += (l1.x * p0.x + l1.y * p0.y) - (l0.x * p1.x + l0.y * p1.y);
            else acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
        }
    } else {
        for (uint64_t x = (uint64_t)blockIdx.x * kMeasThreads + threadIdx.x; x < N;
             x += (uint64_t)gridDim.x * kMeasThreads) {
            const float2 p = psi[x], l = lam[x];
            int odd = (int)((x >> q0) & 1);
            if (kind == TLQ_RZZ) odd ^= (int)((x >> q1) & 1);
            const float w = l.x * p.y - l.y * p.x;
            acc += odd ? -w : w;
        }
    }
    __shared__ float red[kMeasThreads / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = 0.f;
        for (int w = 0; w < kMeasThreads / 32; ++w) e += red[w];
        partial[blockIdx.x] = (double)e;
    }
}

// The state after layer 0 from |0..0> (layer 0 acts on |0..0>): single-qubit rotations give a
// product state, amplitude(x) = prod_q f_q(x_q) with f_q(0) = cos(a_q/2) and f_q(1) = sin(a_q/2)
// (RY) or -i sin(a_q/2) (RX), 1 and 0 for a qubit without a rotation; then layer 0's diagonal
// classes (phase exp(-i a/2 (N - 2c)) from the phase table, or the CZ sign (-1)^c). Each
// thread writes 16 consecutive amplitudes: the product over bits 4.. once, the low four bits
// by doubling. Replaces the layer-0 passes of the forward sweep.
__global__ void __launch_bounds__(256) dense_product_init_kernel(float2* psi, int n_eff,
                                                                  const __grid_constant__ InitGates I,
                                                                  const tlq_gate* gates, const float2* GT,
                                                                  const DenseClassDev* classes, int cls_off, int ncls,
                                                                  const DensePassClassDev* pcd, const int32_t* dists,
                                                                  const float2* ptab) {
    __shared__ InitStage S;
    stage_init(S, n_eff, I, gates, GT, classes, cls_off, ncls, pcd, dists, ptab, threadIdx.x, blockDim.x);
    const uint64_t nblk = 1ull << (n_eff - 4);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nblk; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t x0 = (uint32_t)(t << 4);
        float2 v[16];
        gen16(S, ptab, x0, v);
        float4* out = reinterpret_cast<float4*>(psi + x0);
#pragma unroll
        for (int i = 0; i < 8; ++i) out[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
    }
}

__global__ void init_state_kernel(float2* psi, uint64_t N) {
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x)
        psi[x] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
}

}  // namespace

// Energy partials (one per CTA of a pass, or per measurement block), then, from
// dense_norm_offset on, the tensor-core passes' norm partials (two per CTA, one CTA per SM).
size_t dense_norm_offset(int n_eff) {
    const size_t tiles = (size_t)1 << (n_eff - kDenseTileBits);
    return tiles > (size_t)kMeasBlocks ? tiles : (size_t)kMeasBlocks;
}

size_t dense_partial_count(int n_eff) { return dense_norm_offset(n_eff) + 2 * kMaxSms; }

int dense_grid(int n_eff, int sm_count) {
    const int ntiles = 1 << (n_eff - kDenseTileBits);
    return ntiles < 2 * sm_count ? ntiles : 2 * sm_count;   // two CTAs per SM (the adjoint)
}

static int dense_fwd_grid(int n_eff, int sm_count, bool single) {
    const int ntiles = 1 << (n_eff - kDenseTileBits);
    const int g = dense_pass_ctas(single) * sm_count;
    return ntiles < g ? ntiles : g;
}

namespace {

// Plain path: one sweep per gate forward, per-term measurement sweeps, and for the gradient
// lam = H psi by one gather sweep, then per gate (last to first) one gradient sweep and the
// inverse gate on both states.
int launch_pergate(DenseLaunch& L, cudaStream_t st, int b, const float2* GT, double* eout, double* gout, int& launches) {
    const uint64_t N = 1ull << L.n_eff;
    const int grid_sweep = L.sm_count * 8;
    float2* psi = (float2*)L.state;
    float2* lam = (float2*)L.lam;
    for (int g = 0; g < L.n_gates; ++g) {
        const tlq_gate G = L.host_gates[g];
        if (G.kind == TLQ_RX || G.kind == TLQ_RY)
            pergate_rot_kernel<<<grid_sweep, 256, 0, st>>>(psi, N / 2, G.q0, G.kind, GT, g, 1.f);
        else
            pergate_diag_kernel<<<grid_sweep, 256, 0, st>>>(psi, N, G.kind, G.q0, G.q1, GT, g, 1.f);
        ++launches;
    }
    for (int t = 0; t < L.n_all_terms; ++t) {
        const DenseXTermDev T = L.host_all_terms[t];
        term_measure_kernel<<<kMeasBlocks, kMeasThreads, 0, st>>>(psi, N, T.flip, T.zy, T.ny, L.partial);
        reduce_partials_kernel<<<1, 32, 0, st>>>(L.partial, kMeasBlocks, T.coeff, eout, 1);
        launches += 2;
    }
    if (!gout) return 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(gout, 0, sizeof(double) * (size_t)L.n_params, st)) != cudaSuccess) return (int)e;
    lambda_terms_kernel<<<grid_sweep, 256, 0, st>>>(psi, lam, N, L.all_terms, L.n_all_terms, 0);
    ++launches;
    for (int g = L.n_gates - 1; g >= 0; --g) {
        const tlq_gate G = L.host_gates[g];
        if (G.param >= 0) {
            pergate_grad_kernel<<<kMeasBlocks, kMeasThreads, 0, st>>>(psi, lam, N, G.kind, G.q0, G.q1, L.partial);
            reduce_partials_kernel<<<1, 32, 0, st>>>(L.partial, kMeasBlocks, 1.0, gout + G.param, 1);
            launches += 2;
        }
        if (g == 0) break;
        for (float2* st_ptr : {psi, lam}) {
            if (G.kind == TLQ_RX || G.kind == TLQ_RY)
                pergate_rot_kernel<<<grid_sweep, 256, 0, st>>>(st_ptr, N / 2, G.q0, G.kind, GT, g, -1.f);
            else
                pergate_diag_kernel<<<grid_sweep, 256, 0, st>>>(st_ptr, N, G.kind, G.q0, G.q1, GT, g, -1.f);
            ++launches;
        }
    }
    (void)b;
    return 0;
}

}  // namespace

int launch_dense(DenseLaunch& L, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    const uint64_t N = 1ull << L.n_eff;
    const int grid_sweep = L.sm_count * 8;
    float2* psi = (float2*)L.state;
    float2* lam = (float2*)L.lam;
    int launches = 0;
    // forward passes run single-buffered at three CTAs per SM, except the pass that measures
    // the energy of a gradient call (it also writes lambda), which runs double-buffered at two
    // (measured faster for it)
    const bool single = L.grad == nullptr;
    const size_t smem = dense_pass_smem(true), smem2 = dense_pass_smem(false);
    const size_t asmem = dense_adjoint_smem();
    // layer 0's product state generated inside the first forward pass (no start kernel, no read
    // of the start state) when that pass is a low tile whose first group starts at bit 0
    const bool gen_first = !L.per_gate && !L.tc && L.product_init && L.gen_first;
    const size_t gsmem = dense_pass_gen_smem(true), gsmem2 = dense_pass_gen_smem(false);
    // each kernel with its dynamic shared memory and the largest shared-memory carveout, so
    // that its CTAs per SM fit
    auto prepare = [](const void* k, size_t bytes) {
        cudaError_t r = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (r == cudaSuccess) r = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
        return r;
    };
    if ((e = prepare((const void*)dense_pass_kernel<false, true>, smem)) != cudaSuccess) return (int)e;
    if (gen_first && (e = prepare((const void*)dense_pass_kernel<true, true>, gsmem)) != cudaSuccess) return (int)e;
    if (!single) {
        if ((e = prepare((const void*)dense_pass_kernel<false, false>, smem2)) != cudaSuccess) return (int)e;
        if (gen_first && (e = prepare((const void*)dense_pass_kernel<true, false>, gsmem2)) != cudaSuccess)
            return (int)e;
    }
    size_t tc_smem = 0;
    int tc_nblk = 0;
    if (L.tc && !L.per_gate) {
        const DensePassDev* fw = L.product_init ? L.host_fwd_passes : L.host_passes;
        const int nf = L.product_init ? L.n_fwd_passes : L.n_passes;
        for (int p = 0; p < nf; ++p) tc_nblk = fw[p].ngroups > tc_nblk ? fw[p].ngroups : tc_nblk;
        size_t off[12];
        tc_pass_layout(tc_nblk, off);
        tc_smem = off[11];
        if ((e = cudaFuncSetAttribute(dense_tc_pass_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)tc_smem)) != cudaSuccess)
            return (int)e;
    }
    if (L.grad && !L.per_gate &&
        (e = cudaFuncSetAttribute(dense_adjoint_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)asmem)) !=
            cudaSuccess)
        return (int)e;
    for (int b = 0; b < L.B; ++b) {
        const double* th = L.theta + (size_t)b * L.n_params;
        float2* GT = (float2*)L.gate_table + (size_t)b * L.n_gates;
        float2* PT = (float2*)L.phase_tab + (size_t)b * (L.tab_entries > 0 ? L.tab_entries : 1);
        double* gout = L.grad ? L.grad + (size_t)b * L.n_params : nullptr;
        if (L.n_gates > 0) {
            dense_gate_table_kernel<<<(L.n_gates + 255) / 256, 256, 0, st>>>(L.gates, L.n_gates, th, L.n_params, GT);
            ++launches;
        }
        if (L.tab_entries > 0 && !L.per_gate) {
            dense_phase_table_kernel<<<(L.tab_entries + 255) / 256, 256, 0, st>>>(L.gates, L.tab_gate, L.tab_mult,
                                                                                 L.tab_entries, th, PT);
            ++launches;
        }
        if (b == 0 && L.ev_begin && (e = cudaEventRecord((cudaEvent_t)L.ev_begin, st)) != cudaSuccess) return (int)e;
        const bool product_init = !L.per_gate && L.product_init;
        InitGates I;
        for (int q = 0; q < 32; ++q) I.gate[q] = q < L.n_eff ? L.host_init_gate[q] : -1;
        if (product_init && !gen_first) {   // the state after layer 0, written directly
            dense_product_init_kernel<<<grid_sweep, 256, 0, st>>>(psi, L.n_eff, I, L.gates, GT, L.classes,
                                                                  L.init_class_off, L.init_nclass, L.init_pcd,
                                                                  L.dists, PT);
            ++launches;
        } else if (!product_init) {
            init_state_kernel<<<grid_sweep, 256, 0, st>>>(psi, N);
            ++launches;
        }
        double* eout = L.energy + b;
        if ((e = cudaMemsetAsync(eout, 0, sizeof(double), st)) != cudaSuccess) return (int)e;
        if (L.per_gate) {
            const int rc = launch_pergate(L, st, b, GT, eout, gout, launches);
            if (rc) return rc;
        } else {
            PassArgs A;
            A.layers = L.layers;
            A.classes = L.classes;
            A.pcd = L.pcd;
            A.stage = L.stage;
            A.dists = L.dists;
            A.energy_class_off = L.energy_class_off;
            A.energy_nclass = L.energy_nclass;
            A.zterms = L.zterms;
            A.n_zterms = L.n_zterms;
            A.gates = L.gates;
            A.GT = GT;
            A.ptab = PT;
            A.state = psi;
            A.n_eff = L.n_eff;
            A.partial = L.partial;
            A.npartial = L.partial + dense_norm_offset(L.n_eff);
            A.err = L.err;
            A.lam = nullptr;
            A.init = I;
            A.init_class_off = L.init_class_off;
            A.init_nclass = L.init_nclass;
            A.init_pcd = L.init_pcd;
            const int grid = dense_fwd_grid(L.n_eff, L.sm_count, true);
            const int grid2 = dense_fwd_grid(L.n_eff, L.sm_count, false);
            int mgrid = grid;   // CTAs of the measuring pass: its energy partials
            const int agrid = dense_grid(L.n_eff, L.sm_count);   // the adjoint (two CTAs per SM)
            const int ntiles = 1 << (L.n_eff - kDenseTileBits);
            const int tc_grid = std::min(std::min((ntiles + 1) / 2, L.sm_count), kMaxSms);   // one CTA per SM
            bool measured = false;
            const DensePassDev* fwd = product_init ? L.host_fwd_passes : L.host_passes;
            const int n_fwd = product_init ? L.n_fwd_passes : L.n_passes;
            for (int p = 0; p < n_fwd; ++p) {
                A.pass = fwd[p];
                if (gout) {
                    A.pass.store = 1;   // the adjoint starts from the final state in HBM
                    if (A.pass.measure_group >= 0) A.lam = lam;
                } else if (p == n_fwd - 1 && L.n_xterms == 0 && !L.keep_state) {
                    A.pass.store = 0;   // energies only: nothing reads the final state
                }
                const bool sp = single || A.pass.measure_group < 0;
                if (A.pass.measure_group >= 0) mgrid = sp ? grid : grid2;
                if (L.tc) dense_tc_pass_kernel<<<tc_grid, kTcPassThreads, tc_smem, st>>>(A, tc_nblk);
                else if (gen_first && p == 0 && sp) dense_pass_kernel<true, true><<<grid, kThreads, gsmem, st>>>(A);
                else if (gen_first && p == 0) dense_pass_kernel<true, false><<<grid2, kThreads, gsmem2, st>>>(A);
                else if (sp) dense_pass_kernel<false, true><<<grid, kThreads, smem, st>>>(A);
                else dense_pass_kernel<false, false><<<grid2, kThreads, smem2, st>>>(A);
                ++launches;
                if (A.pass.measure_group >= 0) measured = true;
            }
            if (measured) {
                reduce_partials_kernel<<<1, 32, 0, st>>>(L.partial, L.tc ? 2 * tc_grid : mgrid, 1.0, eout, 1);
                ++launches;
            }
            for (int t = 0; t < L.n_xterms; ++t) {
                const DenseXTermDev T = L.host_xterms[t];
                term_measure_kernel<<<kMeasBlocks, kMeasThreads, 0, st>>>(psi, N, T.flip, T.zy, T.ny, L.partial);
                reduce_partials_kernel<<<1, 32, 0, st>>>(L.partial, kMeasBlocks, T.coeff, eout, 1);
                launches += 2;
            }
            if (gout) {
                // lam = H psi: the diagonal part was written by the measuring pass; X/Y strings here
                if (L.n_xterms > 0 || !measured) {
                    lambda_terms_kernel<<<grid_sweep, 256, 0, st>>>(psi, lam, N, L.xterms, L.n_xterms, measured ? 1 : 0);
                    ++launches;
                }
                AdjArgs R;
                R.classes = L.classes;
                R.pcd = L.pcd;
                R.stage = L.stage;
                R.dists = L.dists;
                R.gates = L.gates;
                R.GT = GT;
                R.ptab = PT;
                R.psi = psi;
                R.lam = lam;
                R.n_eff = L.n_eff;
                for (int p = L.n_passes - 1; p >= 0; --p) {
                    R.pass = L.host_passes[p];
                    R.pass.store = L.host_rev_store[p];   // see DensePlan::rev_store
                    R.gpart = L.gpart + (size_t)p * kDenseAdjSlots * agrid;
                    dense_adjoint_kernel<<<agrid, kThreads, asmem, st>>>(R);
                    ++launches;
                }
                if (L.n_params > 0) {
                    dense_grad_reduce_kernel<<<(L.n_params + 7) / 8, 256, 0, st>>>(L.gpart, agrid, L.adj_off, L.adj_idx,
                                                                                 L.n_params, gout);
                    ++launches;
                }
            }
            if (L.tc && measured) {
                normalize_kernel<<<1, 256, 0, st>>>(L.partial + dense_norm_offset(L.n_eff), 2 * tc_grid, eout, gout,
                                                    L.n_params);
                ++launches;
            }
        }
        if (b == L.B - 1 && L.ev_end && (e = cudaEventRecord((cudaEvent_t)L.ev_end, st)) != cudaSuccess) return (int)e;
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    L.launches = launches;
    return 0;
}

}  // namespace tlq
