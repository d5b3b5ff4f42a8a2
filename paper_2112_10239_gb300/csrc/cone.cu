// Causal-cone expectation values and adjoint gradients on GB300 (sm_103a).
//
// TensorLy-Quantum (arXiv:2112.10239) evaluates <H> = sum_t c_t <psi|P_t|psi> by
// contracting the ket network, each term's operator and the bra network (Sec. 1,
// Sec. 3), and its full gradient by backpropagation (Sec. 3). Here each term is
// contracted over its causal cone only (Sec. 4's "causality-simplified contraction"):
// the planner hands every (term, parameter set) pair a window of W <= 20 qubits and
// the gates of the cone; the reduced state of the window is a 2^W complex vector.
//
// Kernels
//   gate_table_kernel  (K0) FP64 angles -> (cos a/2, sin a/2) per (set, gate), rounded
//                           to the state precision.
//   cone_kernel        (K1-K3) persistent and batched: CTAs pull chunks of equal-width
//                           (cone, set) items from an atomic counter; a chunk is split into
//                           teams of tt = 2^(W-4) threads (one cone per team) so cones of
//                           every width share one launch. Each thread holds 16 amplitudes
//                           (4 window bits) in registers; a "pass" loads them from the
//                           shared-memory state, applies all rotations on those 4 bits,
//                           optionally multiplies by the layer's diagonal phase, and
//                           stores them back. The adjoint walks the layers backwards with
//                           psi and lambda = P psi, emitting Im<lambda|G|psi> per gate.
//   reduce_kernel      (K5) energies and gradients in one launch: fixed-order Neumaier sums in FP64, so a
//                           result does not depend on batching or scheduling.
//
// The global-memory tier's kernels (cone_kernel<real, GRAD, true>) are compiled in their own
// translation unit, cone_global.cu, which includes this file with TLQ_CONE_GLOBAL_TU defined
// and emits only launch_cone_global and launch_batch_global: the two tiers then take
// different ptxas optimisation levels (the build gives this file -O1, under which the
// shared-memory tier measured faster, and cone_global.cu the default -O3).
#include "internal.h"

#include <cuda_runtime.h>
#include <cstdio>

#include "gates.cuh"
#include "tc.cuh"

namespace tlq {

// ---- per-team shared-memory layout ----------------------------------------------------
//
// [psi][lam] padded states (shared tier only), the diagonal phase table (chunk 0: the
// low 7 window bits, padded by one entry per 16; chunk 1: bits 7..13 plus the crossing
// bit 6; chunk 2: bits 14.. plus crossing bit 13), two layer-info buffers (rotation
// (c, s), kind and gradient slot per window qubit; alternating by layer) and the
// double-buffered per-warp gradient partials.
//
// A team may hold half a window: when the window's top qubit carries gates of layer 0 only
// and no measured term, the state is the sum of two branches (top bit 0 and 1) that no
// later gate mixes and no term connects, so each branch is an independent item of W - 1
// qubits (`W` below is the state width) whose energies and gradients add up to the
// window's. Tables and layer records still cover the whole window (`Wt` qubits); the
// branch's top bit enters every phase lookup as the constant `hi`.

// Global-tier tiles (FP32 states wider than a tile): 2^12 amplitudes, 16 per thread of a
// 256-thread half of the CTA; the two halves take alternate tiles, each with its own buffers.
// A high tile keeps window bits 0..7 (see TileMap). The per-sweep partial sums: three rotation
// groups of four (slots 0..11), then the diagonal gates (an RZ and a pair per qubit, from 16).
constexpr int kTileBits = 12;
constexpr int kTileLowBits = 8;
constexpr int kTileTeams = 2;
constexpr int kMaxSweepSlots = 16 + 2 * 20;

__host__ __device__ inline bool tiled_state(int W, int real_bytes, bool smem_state) {
    return !smem_state && real_bytes == 4 && W > kTileBits;
}

struct TeamLayout {
    int psi, lam, tab, info, fac, red, bytes;
    int tile;           // tiled global tier: the psi tile, then (gradients) the lam tile
    int tab1, tab2;     // entry offsets of chunk tables 1 and 2
    int tab_entries;    // total table entries (unpadded) built per layer
};

__host__ __device__ inline int nwarps_of(int tt) { return tt >= 32 ? tt / 32 : 1; }
__host__ __device__ inline int info_bytes(int real_bytes) { return 32 * 2 * real_bytes + 4 * 32 * 4; }

__host__ __device__ inline TeamLayout team_layout(int W, int Wt, int tt, int real_bytes, bool grad, bool smem_state) {
    TeamLayout L{};
    const int r2 = 2 * real_bytes;
    int off = 0;
    L.psi = off;
    if (smem_state) off += padded_amps(W) * r2;
    L.lam = off;
    if (smem_state && grad) off += padded_amps(W) * r2;
    const bool tiled = tiled_state(W, real_bytes, smem_state);
    L.tile = off;
    if (tiled) off += kTileTeams * padded_amps(kTileBits) * r2 * 2;   // psi and lam, or two psi buffers
    const int b1 = (Wt - 7) < 7 ? (Wt - 7) : 7;
    const int b2 = Wt > 14 ? Wt - 14 : 0;
    L.tab1 = 136;
    L.tab2 = L.tab1 + (1 << (b1 + 1));
    const int slots = L.tab2 + (b2 > 0 ? (1 << (b2 + 1)) : 0);
    L.tab_entries = 128 + (1 << (b1 + 1)) + (b2 > 0 ? (1 << (b2 + 1)) : 0);
    L.tab = off;
    off += slots * r2;
    off = (off + 15) & ~15;
    L.info = off;
    off += 2 * info_bytes(real_bytes);
    L.fac = off;   // per-qubit diagonal factors of the layer being staged (info_fac): 32 x 4 complex
    off += 128 * r2;
    off = (off + 15) & ~15;
    L.red = off;
    off += 2 * (tiled ? kMaxSweepSlots : kMaxPassSlots) * nwarps_of(tt) * real_bytes;
    L.bytes = (off + 15) & ~15;
    return L;
}

// ---- team synchronisation ---------------------------------------------------------------

struct Team {
    int tid;        // thread index within the team
    int tt;         // team size (power of two)
    int id;         // team index within the CTA
    unsigned mask;  // lanes of the team within its warp (tt <= 32)
    __device__ __forceinline__ void sync() const {
        if (tt >= kCtaThreads) {
            __syncthreads();
        } else if (tt > 32) {
            asm volatile("bar.sync %0, %1;" ::"r"(id + 1), "r"(tt) : "memory");
        } else {
            __syncwarp(mask);
        }
    }
};

template <typename real>
__device__ __forceinline__ real team_warp_sum(real v, const Team& tm) {
    if (tm.tt >= 32) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    } else {
        for (int off = tm.tt >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(tm.mask, v, off);
    }
    return v;
}


// Diagonal phase of window index x: the product of the chunk-table entries.
template <typename T2>
__device__ __forceinline__ T2 phase_of(const T2* tab, int tab1, int tab2, int W, int x) {
    const int t0 = x & 127;
    T2 ph = tab[t0 + (t0 >> 4)];
    const int b1 = (W - 7) < 7 ? (W - 7) : 7;
    const int i1 = ((x >> 7) & ((1 << b1) - 1)) | (((x >> 6) & 1) << b1);
    ph = cmul(ph, tab[tab1 + i1]);
    if (W > 14) {
        const int b2 = W - 14;
        const int i2 = ((x >> 14) & ((1 << b2) - 1)) | (((x >> 13) & 1) << b2);
        ph = cmul(ph, tab[tab2 + i2]);
    }
    return ph;
}

// Diagonal phases of the 16 amplitudes xb | (j << s), j < 16 (register bits [s, s + 4)), handed
// to use(j, phase) one at a time. A chunk table whose index bits (its qubits and its crossing bit)
// lie outside the register bits gives the same entry for all 16 amplitudes and is read once. Same
// products as phase_of (up to the order of the factors when three chunks are used).
template <typename T2, typename F>
__device__ __forceinline__ void for_phases16(const T2* tab, int tab1, int tab2, int W, int xb, int s, F use) {
    const int b1 = (W - 7) < 7 ? (W - 7) : 7;
    const bool v0 = s < 7;                           // chunk 0: bits 0..6
    const bool v1 = s <= 6 + b1 && s + 3 >= 6;       // chunk 1: crossing bit 6, bits 7..6 + b1
    const bool v2 = W > 14 && s + 3 >= 13;           // chunk 2: crossing bit 13, bits 14..
    auto e0 = [&](int x) {
        const int t0 = x & 127;
        return tab[t0 + (t0 >> 4)];
    };
    auto e1 = [&](int x) { return tab[tab1 + (((x >> 7) & ((1 << b1) - 1)) | (((x >> 6) & 1) << b1))]; };
    auto e2 = [&](int x) {
        const int b2 = W - 14;
        return tab[tab2 + (((x >> 14) & ((1 << b2) - 1)) | (((x >> 13) & 1) << b2))];
    };
    if (!v0 && v1 && !v2) {          // the register bits lie in chunk 1
        T2 h = e0(xb);
        if (W > 14) h = cmul(h, e2(xb));
#pragma unroll
        for (int j = 0; j < 16; ++j) use(j, cmul(h, e1(xb | (j << s))));
    } else if (v0 && !v1 && !v2) {   // the register bits lie in chunk 0
        T2 h = e1(xb);
        if (W > 14) h = cmul(h, e2(xb));
#pragma unroll
        for (int j = 0; j < 16; ++j) use(j, cmul(e0(xb | (j << s)), h));
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) use(j, phase_of(tab, tab1, tab2, W, xb | (j << s)));
    }
}

// ---- kernel parameters ---------------------------------------------------------------------

struct ConeArgs {
    const ConeDev* cones;
    const MeasDev* meas;
    const double* term_coeff;
    const int32_t* prog;
    const int32_t* items;
    const ChunkDev* chunks;
    int32_t chunk_begin, chunk_end;
    const void* gate_table;
    int32_t n_gates, n_terms, n_slots;
    double* e_part;
    double* g_part;
    int32_t* counter;
    int32_t* err;
    void* gscratch;
    size_t gscratch_slot;
    const SetRec* sets;     // per-set records (serving batches), or null: one plan, strided sets
};

template <typename T2>
struct TeamMem {
    T2* psi;
    T2* lam;
    T2* tile;              // tiled global tier: the psi tile (the lam tile follows it)
    T2* tab;
    unsigned char* info;   // two buffers of info_bytes, then the per-qubit factor staging area
    void* red;
    int tab1, tab2, tab_entries;
    int W;                 // qubits of the state held (the window, or its branch)
    int Wt;                // qubits of the window (tables, layer records)
    int hi;                // index bits above the state: the branch's top bit (0 for a whole window)
};

template <typename T2>
__device__ __forceinline__ T2* info_cs(const TeamMem<T2>& M, int par) {
    return reinterpret_cast<T2*>(M.info + par * info_bytes((int)sizeof(T2) / 2));
}
template <typename T2>
__device__ __forceinline__ int* info_kinds(const TeamMem<T2>& M, int par) {
    return reinterpret_cast<int*>(M.info + par * info_bytes((int)sizeof(T2) / 2) + 32 * sizeof(T2));
}
template <typename T2>
__device__ __forceinline__ int* info_rslot(const TeamMem<T2>& M, int par) {
    return info_kinds(M, par) + 32;
}
template <typename T2>
__device__ __forceinline__ int* info_zslot(const TeamMem<T2>& M, int par) {
    return info_kinds(M, par) + 64;
}
template <typename T2>
__device__ __forceinline__ int* info_pslot(const TeamMem<T2>& M, int par) {
    return info_kinds(M, par) + 96;
}
// The factor staging area follows the two info buffers (TeamLayout::fac).
template <typename T2>
__device__ __forceinline__ T2* info_fac(const TeamMem<T2>& M) {
    return reinterpret_cast<T2*>(M.info + 2 * info_bytes((int)sizeof(T2) / 2));
}

// Stage one layer from its per-qubit records: rotation parameters and gradient slots into
// info buffer `par`, and the diagonal phase table (conjugated for the adjoint direction).
// A table entry is the product, over its chunk's qubits q, of the RZ factor of q and the
// RZZ/CZ factor of the pair (q - 1, q) (q - 1 is the chunk's crossing bit for its first
// qubit). Those two factors depend only on the bits of q - 1 and q, so they are first staged
// per qubit as h_q(prev, bit) (one global read of the layer's records each), and an entry
// costs one complex multiply per qubit. Ends with a team barrier.
template <typename real, typename T2>
__device__ void stage_layer(const int32_t* lp, const T2* GT, const Team& tm, const TeamMem<T2>& M, int par,
                            bool conj_phase) {
    const int W = M.Wt;
    T2* cs = info_cs(M, par);
    int* kinds = info_kinds(M, par);
    int* rslot = info_rslot(M, par);
    int* zslot = info_zslot(M, par);
    int* pslot = info_pslot(M, par);
    const int has_diag = lp[0];
    const int32_t* R = lp + kLayerHeader;
    T2* hq = info_fac(M);   // hq[4 q + 2 prev + bit]
    T2 one;
    one.x = 1;
    one.y = 0;
    for (int j = tm.tid; j < W; j += tm.tt) {
        const int32_t* r = R + j * kRecWords;
        const int rg = r[0];
        kinds[j] = rg >= 0 ? (r[1] & 255) : -1;
        if (rg >= 0) cs[j] = GT[rg];
        rslot[j] = (r[1] >> 8) - 1;
        zslot[j] = r[3];
        pslot[j] = (r[5] >> 8) - 1;
        if (has_diag) {
            const T2 g = r[2] >= 0 ? GT[r[2]] : one;   // RZ on j: (cos, sin) of a/2
            int pk = -1;                                // the (j - 1, j) gate sits in record j - 1
            T2 pf = one;
            if (j > 0) {
                const int32_t* rp = r - kRecWords;
                if (rp[4] >= 0) {
                    pk = rp[5] & 255;
                    if (pk != TLQ_CZ) pf = GT[rp[4]];
                }
            }
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int prev = e >> 1, bq = e & 1;
                // RZ(a): e^{-ia/2} for bit 0, e^{+ia/2} for bit 1 (identity when absent)
                T2 f;
                f.x = g.x;
                f.y = bq ? g.y : -g.y;
                if (pk == TLQ_CZ) {
                    if (prev & bq) { f.x = -f.x; f.y = -f.y; }
                } else if (pk >= 0) {   // RZZ: e^{-ia/2} for equal bits, e^{+ia/2} otherwise
                    T2 h;
                    h.x = pf.x;
                    h.y = (prev ^ bq) ? pf.y : -pf.y;
                    f = cmul(f, h);
                }
                hq[4 * j + e] = f;
            }
        }
    }
    if (has_diag) {
        tm.sync();   // the per-qubit factors are staged
        const int b1 = (W - 7) < 7 ? (W - 7) : 7;
        for (int e = tm.tid; e < M.tab_entries; e += tm.tt) {
            int lo, bc, idx, slot;
            if (e < 128) {
                lo = 0; bc = 7; idx = e; slot = e + (e >> 4);
            } else if (e < 128 + (2 << b1)) {
                lo = 7; bc = b1; idx = e - 128; slot = M.tab1 + idx;
            } else {
                lo = 14; bc = W - 14; idx = e - 128 - (2 << b1); slot = M.tab2 + idx;
            }
            int prev = lo > 0 ? (idx >> bc) & 1 : 0;   // bit of qubit lo - 1 (crossing bit)
            T2 ph = hq[4 * lo + 2 * prev + (idx & 1)];
            prev = idx & 1;
            for (int k = 1; k < bc; ++k) {
                const int bq = (idx >> k) & 1;
                ph = cmul(ph, hq[4 * (lo + k) + 2 * prev + bq]);
                prev = bq;
            }
            if (conj_phase) ph.y = -ph.y;
            M.tab[slot] = ph;
        }
    }
    tm.sync();
}

// ---- global tier: tiles ---------------------------------------------------------------------
//
// A state too wide for shared memory lives in global memory, and a layer is applied in a few
// sweeps over it. A sweep stages one tile of 2^12 amplitudes at a time in shared memory, runs
// one or more register passes on it and writes it back. A low tile holds window bits 0..11
// (the tile index gives the bits above); a high tile holds window bits 0..7 and one 4-bit
// register group g..g+3 (the tile index gives the bits in between and above). Window bits 0..4
// stay the lane bits of every pass, so the passes' warp reductions are unchanged.
struct TileMap {
    int a;       // tile bits [0, a) are window bits [0, a)
    int g;       // tile bits [a, 12) are window bits [g, g + 12 - a)
    int fix;     // window bits given by the tile index
    int s_loc;   // tile position of the pass's register bits
    bool first;  // the half's first tile of a sweep: the pass's partial sums start from zero
    int nw;      // partial sums: warps of the CTA (the slot stride) ...
    int warp0;   // ... and the CTA warp index of the half's first warp
    __device__ __forceinline__ int x(int i) const { return (i & ((1 << a) - 1)) | ((i >> a) << g) | fix; }
};

// Forward pass on register bits [s, s+4): rotations on the bits in `m`, then the
// layer's diagonal phase when `diag`.
// TILE: psi is a shared-memory tile (tmap gives its bits); s is the window position of the
// register bits and tmap->s_loc their tile position.
template <typename real, typename T2, bool TILE = false>
__device__ void pass_fwd(T2* psi, int s, unsigned m, bool diag, const Team& tm, const TeamMem<T2>& M, int par,
                         const TileMap* tmap = nullptr) {
    const int W = M.W;
    const T2* cs = info_cs(M, par);
    const int* kinds = info_kinds(M, par);
    int kd[4];
    real c[4], sn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kd[k] = (m >> k) & 1 ? kinds[s + k] : -1;
        const T2 v = cs[s + k];
        c[k] = v.x;
        sn[k] = v.y;
    }
    const int sl = TILE ? tmap->s_loc : s;
    const int nout = 1 << ((TILE ? kTileBits : W) - 4);
    const int lowmask = (1 << sl) - 1;
    const int stride = pass_stride(sl);
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int base = (o & lowmask) | ((o >> sl) << (sl + 4));
        T2* p = psi + pad16(base);
        T2 v[16];
        load16(v, p, stride);
        if (kd[0] >= 0) apply_rot<0>(v, kd[0], c[0], sn[0]);
        if (kd[1] >= 0) apply_rot<1>(v, kd[1], c[1], sn[1]);
        if (kd[2] >= 0) apply_rot<2>(v, kd[2], c[2], sn[2]);
        if (kd[3] >= 0) apply_rot<3>(v, kd[3], c[3], sn[3]);
        if (diag) {
            const int xb = (TILE ? tmap->x(base) : base) | M.hi;
            for_phases16(M.tab, M.tab1, M.tab2, M.Wt, xb, s, [&](int j, T2 ph) { v[j] = cmul(v[j], ph); });
        }
        store16(v, p, stride);
    }
}

// Adjoint pass on register bits [s, s+4): when `diag`, emit Im<lam|Z..|psi> for the layer's
// parametrised diagonal gates and un-apply the diagonal; then for each rotation on the bits
// in `m`, emit Im<lam|G|psi> and un-apply it from psi and lam. Per-warp partial sums go to
// red[slot * nw + warp]: slots 0..3 rotations (register bit), 4.. diagonal gates in program
// order.
template <typename real, typename T2, bool DIAG, bool FINAL = false, bool TILE = false>
__device__ void pass_bwd(T2* psi, T2* lam, int s, unsigned m, const Team& tm, const TeamMem<T2>& M, int par,
                         real* red, const TileMap* tmap = nullptr) {
    const int W = M.W;
    const T2* cs = info_cs(M, par);
    const int* kinds = info_kinds(M, par);
    const int nw = TILE ? tmap->nw : nwarps_of(tm.tt);
    const int warp = TILE ? tmap->warp0 + (tm.tid >> 5) : (tm.tt >= 32 ? (tm.tid >> 5) : 0);
    const bool leader = tm.tt >= 32 ? ((tm.tid & 31) == 0) : (tm.tid == 0);
    int kd[4];
    real c[4], sn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kd[k] = (m >> k) & 1 ? kinds[s + k] : -1;
        const T2 v = cs[s + k];
        c[k] = v.x;
        sn[k] = -v.y;   // un-apply: angle -> -angle
    }
    const int sl = TILE ? tmap->s_loc : s;
    const int nout = 1 << ((TILE ? kTileBits : W) - 4);
    const int lowmask = (1 << sl) - 1;
    const int stride = pass_stride(sl);
    bool first = TILE ? tmap->first : true;
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int base = (o & lowmask) | ((o >> sl) << (sl + 4));
        T2* pp = psi + pad16(base);
        T2* lp = lam + pad16(base);
        T2 p[16], l[16];
        load16(p, pp, stride);
        load16(l, lp, stride);
        if constexpr (DIAG) {
            // w_x = Im(conj(lam_x) psi_x); dE/da is sum_x z_q(x) w_x for RZ on q and
            // sum_x z_q0(x) z_q1(x) w_x for RZZ on (q0, q1 = q0 + 1).
            real S = 0, Sk0 = 0, Sk1 = 0, Sk2 = 0, Sk3 = 0, Sp0 = 0, Sp1 = 0, Sp2 = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const real w = l[j].x * p[j].y - l[j].y * p[j].x;
                S += w;
                Sk0 += (j & 1) ? -w : w;
                Sk1 += (j & 2) ? -w : w;
                Sk2 += (j & 4) ? -w : w;
                Sk3 += (j & 8) ? -w : w;
                Sp0 += ((j ^ (j >> 1)) & 1) ? -w : w;
                Sp1 += (((j >> 1) ^ (j >> 2)) & 1) ? -w : w;
                Sp2 += (((j >> 2) ^ (j >> 3)) & 1) ? -w : w;
            }
            const int* zslot = info_zslot(M, par);
            const int* pslot = info_pslot(M, par);
            const int xb = (TILE ? tmap->x(base) : base) | M.hi;   // the index bits outside the register bits
            if (tm.tt >= 32) {
                // Whole warps (W >= 9, so s >= 5: window bits 0..4 are the lane bits, the bits
                // from 5 up to s - 1 and above the register bits are the same across the warp).
                // A Walsh transform of S over the lanes gives every sign pattern of the lane
                // bits at once: lane m holds F[m] = sum_l (-1)^popc(l & m) S_l, so the sum for an
                // RZ on lane bit j is F[2^j], for a pair of lane bits F[2^j0 + 2^j1], and for
                // uniform bits F[0] with the warp's sign. The register-bit sums are reduced four
                // at a time. Each slot is written by the lane that holds its value.
                const int lane = tm.tid & 31;
                real F = S;
#pragma unroll
                for (int off = 1; off < 32; off <<= 1) {
                    const real o2 = __shfl_xor_sync(0xffffffffu, F, off);
                    F = (lane & off) ? (o2 - F) : (F + o2);
                }
                const real sk = warp_sum4(Sk0, Sk1, Sk2, Sk3, lane);   // lane 8 k: sum of Sk_k
                bool pin = false;                                      // RZZ inside the register block
                for (int j0 = s; j0 < s + 3; ++j0) pin |= pslot[j0] >= 0;
                const real sp = pin ? warp_sum4(Sp0, Sp1, Sp2, (real)0, lane) : (real)0;
                auto put = [&](int t, int owner, real val) {
                    if (lane == owner) {
                        real* dst = red + t * nw + warp;
                        *dst = first ? val : *dst + val;
                    }
                };
                for (int j0 = 0; j0 < M.Wt; ++j0) {
                    const int k0 = j0 - s;
                    const bool in0 = (unsigned)k0 < 4u;
                    if (zslot[j0] >= 0) {
                        if (in0) put(4 + 2 * j0, 8 * k0, sk);
                        else if (j0 < 5) put(4 + 2 * j0, 1 << j0, F);
                        else put(4 + 2 * j0, 0, ((xb >> j0) & 1) ? -F : F);
                    }
                    if (pslot[j0] >= 0) {   // RZZ on (j0, j0 + 1)
                        const int j1 = j0 + 1;
                        const bool in1 = (unsigned)(j1 - s) < 4u;
                        if (in0 && in1) {
                            put(5 + 2 * j0, 8 * k0, sp);
                        } else if (in0) {   // j0 = s + 3, j1 above the block: the same across the warp
                            put(5 + 2 * j0, 24, ((xb >> j1) & 1) ? -sk : sk);
                        } else if (in1) {   // j1 = s, j0 = s - 1
                            if (j0 < 5) {   // a lane bit (s = 5): signed sum of Sk0 over the warp
                                const real v = team_warp_sum(((xb >> j0) & 1) ? -Sk0 : Sk0, tm);
                                put(5 + 2 * j0, 0, v);
                            } else {
                                put(5 + 2 * j0, 0, ((xb >> j0) & 1) ? -sk : sk);
                            }
                        } else if (j1 < 5) {
                            put(5 + 2 * j0, (1 << j0) | (1 << j1), F);
                        } else if (j0 < 5) {   // j0 = 4, j1 = 5
                            put(5 + 2 * j0, 16, ((xb >> j1) & 1) ? -F : F);
                        } else {
                            put(5 + 2 * j0, 0, (((xb >> j0) ^ (xb >> j1)) & 1) ? -F : F);
                        }
                    }
                }
            } else
            for (int j0 = 0; j0 < M.Wt; ++j0) {
                const int k0 = j0 - s;
                const bool in0 = (unsigned)k0 < 4u;
                if (zslot[j0] >= 0) {
                    real val;
                    if (in0) val = k0 == 0 ? Sk0 : k0 == 1 ? Sk1 : k0 == 2 ? Sk2 : Sk3;
                    else val = ((xb >> j0) & 1) ? -S : S;
                    val = team_warp_sum(val, tm);
                    if (leader) {
                        real* dst = red + (4 + 2 * j0) * nw + warp;
                        *dst = first ? val : *dst + val;
                    }
                }
                if (pslot[j0] >= 0) {   // RZZ on (j0, j0 + 1)
                    const int j1 = j0 + 1;
                    const bool in1 = (unsigned)(j1 - s) < 4u;
                    real val;
                    if (in0 && in1) val = k0 == 0 ? Sp0 : k0 == 1 ? Sp1 : Sp2;
                    else if (in0) val = ((xb >> j1) & 1) ? -Sk3 : Sk3;   // j0 = s + 3
                    else if (in1) val = ((xb >> j0) & 1) ? -Sk0 : Sk0;   // j1 = s
                    else val = (((xb >> j0) ^ (xb >> j1)) & 1) ? -S : S;
                    val = team_warp_sum(val, tm);
                    if (leader) {
                        real* dst = red + (5 + 2 * j0) * nw + warp;
                        *dst = first ? val : *dst + val;
                    }
                }
            }
            for_phases16(M.tab, M.tab1, M.tab2, M.Wt, xb, s, [&](int j, T2 ph) {   // conjugated table
                p[j] = cmul(p[j], ph);
                l[j] = cmul(l[j], ph);
            });
        }
        if constexpr (!DIAG) {
            real g0 = 0, g1 = 0, g2 = 0, g3 = 0;
            if constexpr (FINAL) {
                // layer 0: the states are not needed afterwards, and its rotations commute, so
                // every gradient is taken at this state with nothing un-applied or stored
                if (kd[0] >= 0) g0 = kd[0] == TLQ_RY ? grad_y<0, T2, real, false>(p, l) : grad_x<0, T2, real>(p, l);
                if (kd[1] >= 0) g1 = kd[1] == TLQ_RY ? grad_y<1, T2, real, false>(p, l) : grad_x<1, T2, real>(p, l);
                if (kd[2] >= 0) g2 = kd[2] == TLQ_RY ? grad_y<2, T2, real, false>(p, l) : grad_x<2, T2, real>(p, l);
                if (kd[3] >= 0) g3 = kd[3] == TLQ_RY ? grad_y<3, T2, real, false>(p, l) : grad_x<3, T2, real>(p, l);
            } else {
                if (kd[0] >= 0) g0 = adjoint_rot<0, T2, real, false>(p, l, kd[0], c[0], sn[0]);
                if (kd[1] >= 0) g1 = adjoint_rot<1, T2, real, false>(p, l, kd[1], c[1], sn[1]);
                if (kd[2] >= 0) g2 = adjoint_rot<2, T2, real, false>(p, l, kd[2], c[2], sn[2]);
                if (kd[3] >= 0) g3 = adjoint_rot<3, T2, real, false>(p, l, kd[3], c[3], sn[3]);
                store16(p, pp, stride);
                store16(l, lp, stride);
            }
            if (tm.tt >= 32) {
                const int lane = tm.tid & 31;
                const real val = warp_sum4(g0, g1, g2, g3, lane);   // value k = (lane >> 3) & 3
                const int k = (lane >> 3) & 3;
                const int kdk = k == 0 ? kd[0] : k == 1 ? kd[1] : k == 2 ? kd[2] : kd[3];
                if ((lane & 7) == 0 && kdk >= 0) {
                    real* dst = red + k * nw + warp;
                    *dst = first ? val : *dst + val;
                }
            } else {
                const real gk[4] = {g0, g1, g2, g3};
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    if (kd[k] < 0) continue;
                    const real val = team_warp_sum(gk[k], tm);
                    if (leader) {
                        real* dst = red + k * nw + warp;
                        *dst = first ? val : *dst + val;
                    }
                }
            }
        } else {
            store16(p, pp, stride);
            store16(l, lp, stride);
        }
        first = false;
    }
}

// Sum the per-warp partials of one adjoint pass in fixed order and store them as FP64 slots.
template <typename real, typename T2>
__device__ void flush_pass(const real* red, int nw, unsigned m, int s, const TeamMem<T2>& M, int par, bool diag,
                           double* gdst, const Team& tm) {
    const int* kinds = info_kinds(M, par);
    const int* rslot = info_rslot(M, par);
    const int* zslot = info_zslot(M, par);
    const int* pslot = info_pslot(M, par);
    const int nred = diag ? 4 + 2 * M.Wt : 4;
    for (int t = tm.tid; t < nred; t += tm.tt) {
        int slot;
        if (t < 4) {
            if (!((m >> t) & 1) || kinds[s + t] < 0) continue;
            slot = rslot[s + t];
        } else {
            const int j = (t - 4) >> 1;
            slot = ((t - 4) & 1) ? pslot[j] : zslot[j];
        }
        if (slot < 0) continue;
        real acc = 0;
        for (int w = 0; w < nw; ++w) acc += red[t * nw + w];
        // a branch adds its share onto zeroed slots: two addends, so the order does not matter
        if (M.Wt > M.W) atomicAdd(gdst + slot, (double)acc);
        else gdst[slot] = (double)acc;
    }
}

// Factor of window qubit j with bit value `bit` in the product state that layer 0's
// rotations make from |0..0> (staged in info buffer `par`): f_j(0) = cos(a_j/2) and
// f_j(1) = sin(a_j/2) (RY) or -i sin(a_j/2) (RX); a qubit without a live rotation gives 1
// for bit 0 and 0 for bit 1.
template <typename T2>
__device__ __forceinline__ T2 init_factor(const T2* cs, const int* kinds, unsigned live, int j, int bit) {
    T2 f;
    const bool rot = ((live >> j) & 1u) && kinds[j] >= 0;
    if (!rot) {
        f.x = bit ? 0 : 1;
        f.y = 0;
    } else if (bit == 0) {
        f.x = cs[j].x;
        f.y = 0;
    } else if (kinds[j] == TLQ_RY) {
        f.x = cs[j].y;
        f.y = 0;
    } else {   // RX
        f.x = 0;
        f.y = -cs[j].y;
    }
    return f;
}

// The 16 amplitudes x = base | j (j < 16) of the product state over the state's qubits,
// prod_{q < M.W} f_q(x_q): the product over the fixed high bits times the 16 products over
// the low four bits (built by doubling).
template <typename T2>
__device__ __forceinline__ void product16(const T2* cs, const int* kinds, int W, unsigned live, int base,
                                          T2 (&v)[16]) {
    v[0].x = 1;
    v[0].y = 0;
    for (int j = 4; j < W; ++j) v[0] = cmul(v[0], init_factor(cs, kinds, live, j, (base >> j) & 1));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const T2 f0 = init_factor(cs, kinds, live, k, 0), f1 = init_factor(cs, kinds, live, k, 1);
#pragma unroll
        for (int j = 0; j < (1 << k); ++j) {
            v[j | (1 << k)] = cmul(v[j], f1);
            v[j] = cmul(v[j], f0);
        }
    }
}

// The window state after layer 0 (staged in info buffer `par`), from |0..0>: the product
// state of its rotations, times the branch's top-qubit factor for half a window, then
// layer 0's diagonal phase when `diag`. Each thread writes 16 contiguous amplitudes.
// Replaces the register passes of layer 0 (and its diagonal pass) in the forward sweep.
template <typename real, typename T2>
__device__ void init_product_state(const TeamMem<T2>& M, unsigned live, bool diag, const Team& tm, int par) {
    const int W = M.W;
    const int nout = 1 << (W - 4);
    const T2* cs = info_cs(M, par);
    const int* kinds = info_kinds(M, par);
    T2 top;
    top.x = 1;
    top.y = 0;
    if (M.Wt > W) top = init_factor(cs, kinds, live, W, (M.hi >> W) & 1);
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int base = o << 4;
        T2 v[16];
        product16(cs, kinds, W, live, base, v);
        if (M.Wt > W) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = cmul(v[j], top);
        }
        if (diag) {
            const int xb = base | M.hi;
            for_phases16(M.tab, M.tab1, M.tab2, M.Wt, xb, 0, [&](int j, T2 ph) { v[j] = cmul(v[j], ph); });
        }
        store16(v, M.psi + pad16(base), 1);
    }
}

// Gradient of layer 0's rotation on the top qubit of a branch (bit value h): Im<lam|G|psi>
// pairs amplitudes of the two branches, and this branch holds only lam and psi with top bit
// h. At this point (layer 0's diagonal un-applied) psi is the product state of layer 0's
// rotations, so the other branch's amplitude is known exactly: f_top(1 - h) times the
// product over the state's qubits. The branch adds its half of the pair sums:
// RY, G = Y: h = 0 gives -Re(conj(l0) p1), h = 1 gives +Re(conj(l1) p0);
// RX, G = X: Im(conj(l_h) p_{1-h}) for either h.
// Per-warp partial sums go to red[warp]. Ends without a barrier.
template <typename real, typename T2>
__device__ void top_rotation_grad(const TeamMem<T2>& M, unsigned live, int par, const Team& tm, real* red) {
    const int W = M.W;
    const int h = (M.hi >> W) & 1;
    const int nout = 1 << (W - 4);
    const T2* cs = info_cs(M, par);
    const int* kinds = info_kinds(M, par);
    const int kind = kinds[W];
    const T2 f = init_factor(cs, kinds, live, W, 1 - h);   // the other branch's top factor
    const int warp = tm.tt >= 32 ? (tm.tid >> 5) : 0;
    const bool leader = tm.tt >= 32 ? ((tm.tid & 31) == 0) : (tm.tid == 0);
    real acc = 0;
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int base = o << 4;
        T2 u[16], l[16];
        product16(cs, kinds, W, live, base, u);
        load16(l, M.lam + pad16(base), 1);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const T2 q = cmul(f, u[j]);   // psi of the paired amplitude in the other branch
            if (kind == TLQ_RY) acc += (h ? (real)1 : (real)-1) * (l[j].x * q.x + l[j].y * q.y);
            else acc += l[j].x * q.y - l[j].y * q.x;
        }
    }
    acc = team_warp_sum(acc, tm);
    if (leader) red[warp] = acc;
}

// One pass over the window for up to kMeasBatch terms: per-warp partial sums of
// <psi|P_t|psi> go to red[k * nw + warp]; when GRAD, lam += sum_t c_t P_t psi over these
// terms (lam starts at zero unless ADD, in which case each thread reads back the values it
// wrote in the previous batch). Each block of 16 amplitudes is read once per pass.
constexpr int kMeasBatch = 8;
template <typename real, typename T2, bool GRAD, bool ADD>
__device__ void measure_batch(const TeamMem<T2>& M, const MeasDev* mt, int nmt, const double* coeff, const Team& tm,
                              real* red) {
    const int W = M.W;
    const int nout = 1 << (W - 4);
    const int nw = nwarps_of(tm.tt);
    const int warp = tm.tt >= 32 ? (tm.tid >> 5) : 0;
    const bool leader = tm.tt >= 32 ? ((tm.tid & 31) == 0) : (tm.tid == 0);
    real acc[kMeasBatch];
#pragma unroll
    for (int k = 0; k < kMeasBatch; ++k) acc[k] = 0;
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int x0 = o << 4;
        T2 a[16];
        load16(a, M.psi + pad16(x0), 1);
        T2 lv[16];
        if (GRAD) {
            if (ADD) {
                load16(lv, M.lam + pad16(x0), 1);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) lv[j].x = lv[j].y = 0;
            }
        }
#pragma unroll
        for (int k = 0; k < kMeasBatch; ++k) {
            if (k >= nmt) break;
            const MeasDev md = mt[k];
            T2 f0;   // (-i)^ny
            const int ny = md.ny & 3;
            f0.x = ny == 0 ? 1 : ny == 2 ? -1 : 0;
            f0.y = ny == 1 ? -1 : ny == 3 ? 1 : 0;
            const real ck = GRAD ? (real)coeff[md.term] : (real)0;
            real sk = 0;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int x = x0 | j;
                const T2 v = M.psi[pad16(x ^ (int)md.flip)];
                T2 t = cmul(f0, v);
                if (__popc((unsigned)x & md.zy) & 1) { t.x = -t.x; t.y = -t.y; }
                sk += a[j].x * t.x + a[j].y * t.y;
                if (GRAD) {
                    lv[j].x += ck * t.x;
                    lv[j].y += ck * t.y;
                }
            }
            acc[k] += sk;
        }
        if (GRAD) store16(lv, M.lam + pad16(x0), 1);
    }
#pragma unroll
    for (int k = 0; k < kMeasBatch; ++k) {
        if (k >= nmt) break;
        const real v = team_warp_sum(acc[k], tm);
        if (leader) red[k * nw + warp] = v;
    }
}

// <psi|P_t|psi> for every term t measured on this window, written to e_out[term] (added for
// a branch); when GRAD also lam = sum_t c_t P_t psi (the term coefficients folded into the
// adjoint). Terms go kMeasBatch per pass over the window (at most kMaxGroupTerms in all).
// Ends with a team barrier.
template <typename real, typename T2, bool GRAD>
__device__ void measure(const TeamMem<T2>& M, const MeasDev* mt, int nmt, const double* coeff, double* e_out,
                        const Team& tm, real* red) {
    const int nw = nwarps_of(tm.tt);
    measure_batch<real, T2, GRAD, false>(M, mt, nmt < kMeasBatch ? nmt : kMeasBatch, coeff, tm, red);
    for (int k0 = kMeasBatch; k0 < nmt; k0 += kMeasBatch)
        measure_batch<real, T2, GRAD, true>(M, mt + k0, nmt - k0 < kMeasBatch ? nmt - k0 : kMeasBatch, coeff, tm,
                                            red + k0 * nw);
    tm.sync();
    for (int k = tm.tid; k < nmt; k += tm.tt) {
        real e = 0;
        for (int w = 0; w < nw; ++w) e += red[k * nw + w];
        if (M.Wt > M.W) atomicAdd(e_out + mt[k].term, (double)e);   // a branch: two addends onto zero
        else e_out[mt[k].term] = (double)e;
    }
    tm.sync();
}

// One (cone, set) item: the whole window (half = 0), or the branch with the window's top
// bit half - 1 (W = the window's width - 1). Ends with a team barrier.
// ---- global tier: tile sweeps ----------------------------------------------------------------

// The sweeps of one layer on a tiled state of W qubits (14 <= W <= 20), in forward order: the
// low sweep takes the layer's rotations below the high groups (register groups at 0, 4 and 8,
// as in the untiled forward), then each high sweep one group g..g+3, g = W - 4, W - 8 (at least
// 8) while g > 12. Sweeps without rotations are dropped; the layer's diagonal goes into the last
// forward sweep (an empty low sweep when there is none).
struct LayerSweeps {
    int n;
    int g[3];           // 0 for the low sweep, else the high group's base bit (at least 8)
    int ng[3];          // register groups of the sweep
    int s[3][3];        // window base bit of each group
    unsigned m[3][3];   // its rotation bits
};

__device__ __forceinline__ void layer_sweeps(unsigned todo, int W, bool diag, LayerSweeps& L) {
    int gh[2], nh = 0;
    for (int g = W - 4; nh < 2; g = g - 4 > kTileLowBits ? g - 4 : kTileLowBits) {
        gh[nh++] = g;
        if (g <= kTileBits) break;
    }
    const int lowtop = gh[nh - 1] < kTileBits ? gh[nh - 1] : kTileBits;
    L.n = 0;
    unsigned bits = todo & ((1u << lowtop) - 1u);
    L.g[0] = 0;
    L.ng[0] = 0;
    while (bits && L.ng[0] < 3) {
        const int bt = __ffs(bits) - 1;
        const int sg = bt < 4 ? 0 : (bt < kTileBits - 4 ? bt : kTileBits - 4);
        L.s[0][L.ng[0]] = sg;
        L.m[0][L.ng[0]] = (bits >> sg) & 15u;
        ++L.ng[0];
        bits &= ~(15u << sg);
    }
    if (L.ng[0] > 0) L.n = 1;
    for (int h = 0; h < nh; ++h) {
        const unsigned m = (todo >> gh[h]) & 15u;
        if (!m) continue;
        L.g[L.n] = gh[h];
        L.ng[L.n] = 1;
        L.s[L.n][0] = gh[h];
        L.m[L.n][0] = m;
        ++L.n;
    }
    if (L.n == 0 && diag) {
        L.g[0] = 0;
        L.ng[0] = 0;
        L.n = 1;
    }
}

// Tile t of a sweep whose high group starts at g (g = 0: the low tile), for half `half`.
__device__ __forceinline__ TileMap sweep_tile(int g, int t, int half) {
    TileMap tp;
    if (g == 0) {
        tp.a = kTileBits;
        tp.g = kTileBits;
        tp.fix = t << kTileBits;
    } else {   // tile index bits: window bits kTileLowBits..g-1, then g+4..
        const int nlo = g - kTileLowBits;
        tp.a = kTileLowBits;
        tp.g = g;
        tp.fix = ((t & ((1 << nlo) - 1)) << kTileLowBits) | ((t >> nlo) << (g + 4));
    }
    tp.s_loc = kTileLowBits;
    tp.first = t < kTileTeams;
    tp.nw = kGlobalCtaThreads / 32;
    tp.warp0 = half * (kGlobalCtaThreads / kTileTeams / 32);
    return tp;
}

// Tile transfers on the bulk-copy engine (cp.async.bulk). In the padded layout a low tile is
// one contiguous block of the global state (2^12 amplitudes and their padding, 36,864 bytes)
// and a high tile is 16 blocks, one per value of its register group (256 amplitudes and their
// padding, 2,304 bytes each); in shared memory the blocks follow one another. One thread of a
// half issues the copies: loads complete on the half's mbarrier (one phase per tile), stores go
// into bulk groups that the same thread retires before its buffers are loaded again.
struct TileSync {
    uint64_t* bar;     // two mbarriers per half, one per tile buffer (shared memory)
    uint32_t phase;    // this thread's half: bit k = parity of the next load into buffer k
};

__device__ __forceinline__ int tile_blocks(const TileMap& tp) { return tp.a == kTileBits ? 1 : 1 << (kTileBits - kTileLowBits); }
__device__ __forceinline__ uint32_t tile_block_bytes(const TileMap& tp) {
    return (uint32_t)padded_amps(tp.a) * (uint32_t)sizeof(float2);
}

// Issued by one thread of the half: load the tile of nst states (gs[k] -> tiles[k]).
__device__ __forceinline__ void tile_fetch(float2* const (&tiles)[2], float2* const (&gs)[2], int nst,
                                           const TileMap& tp, uint64_t* bar) {
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");   // earlier stores have read the buffers
    const int nb = tile_blocks(tp);
    const uint32_t bytes = tile_block_bytes(tp);
    const uint32_t b = tc::su32(bar);
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes * nb * nst) : "memory");
    for (int k = 0; k < nst; ++k)
        for (int r = 0; r < nb; ++r)
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             tc::su32(tiles[k] + pad16(r << tp.a))),
                         "l"(gs[k] + pad16(tp.x(r << tp.a))), "r"(bytes), "r"(b)
                         : "memory");
}

// Issued by one thread of the half after a barrier that follows every thread's proxy fence.
__device__ __forceinline__ void tile_store(float2* const (&tiles)[2], float2* const (&gs)[2], int nst, const TileMap& tp) {
    const int nb = tile_blocks(tp);
    const uint32_t bytes = tile_block_bytes(tp);
    for (int k = 0; k < nst; ++k)
        for (int r = 0; r < nb; ++r)
            asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gs[k] + pad16(tp.x(r << tp.a))),
                         "r"(tc::su32(tiles[k] + pad16(r << tp.a))), "r"(bytes)
                         : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Every thread of the half: wait (bounded) for the load of the half's current tile.
__device__ __forceinline__ void tile_wait(TileSync& ts, int half, int buf, const ConeArgs& A) {
    if (!tc::mbar_wait(ts.bar + 2 * half + buf, (ts.phase >> buf) & 1u)) atomicOr(A.err, 1);
    ts.phase ^= 1u << buf;
}

// End of a sweep, before the CTA barrier: the half's stores are complete and visible to the
// loads and plain reads that follow.
__device__ __forceinline__ void tile_sweep_done(const Team& ht) {
    if (ht.tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async;" ::: "memory");
}

// The half of the CTA (256 threads, named barrier 1 or 2) that a thread works in during a sweep.
__device__ __forceinline__ Team tile_half(const Team& tm) {
    Team h;
    const int per = kGlobalCtaThreads / kTileTeams;
    h.id = tm.tid / per;
    h.tid = tm.tid - h.id * per;
    h.tt = per;
    h.mask = 0xffffffffu;
    return h;
}

// Forward layers 1.. of a tiled state (layer 0's product state is already in M.psi).
template <typename real>
__device__ void tiled_forward(const ConeArgs& A, const TeamMem<float2>& M, const Team& tm, const int32_t* body,
                              const int32_t* lofs, int nl, const float2* GT, TileSync& ts) {
    const int W = M.W;
    const int ntiles = 1 << (W - kTileBits);
    const Team ht = tile_half(tm);
    // two psi buffers per half (the adjoint's psi and lam tiles): the load of the half's next
    // tile runs while the current one is processed
    float2* const buf[2] = {M.tile + 2 * ht.id * padded_amps(kTileBits),
                            M.tile + (2 * ht.id + 1) * padded_amps(kTileBits)};
    float2* const gs[2] = {M.psi, M.psi};
    for (int li = 1; li < nl; ++li) {
        const int32_t* lp = body + lofs[li];
        const int ndiag = lp[0];
        const int par = li & 1;
        const unsigned todo = (unsigned)lp[1];
        if (todo >> W) {   // a branch's top qubit has gates of layer 0 only
            if (tm.tid == 0) atomicOr(A.err, 1);
            return;
        }
        asm volatile("fence.proxy.async;" ::: "memory");   // plain writes of the state before the loads
        stage_layer<real, float2>(lp, GT, tm, M, par, false);
        LayerSweeps LS;
        layer_sweeps(todo, W, ndiag > 0, LS);
        for (int k = 0; k < LS.n; ++k) {
            const bool dg = ndiag > 0 && k == LS.n - 1;
            const bool low = LS.g[k] == 0;
            int cur = 0;
            if (ht.tid == 0 && ht.id < ntiles) {
                float2* const t0[2] = {buf[0], buf[0]};
                tile_fetch(t0, gs, 1, sweep_tile(LS.g[k], ht.id, ht.id), ts.bar + 2 * ht.id);
            }
            for (int t = ht.id; t < ntiles; t += kTileTeams, cur ^= 1) {
                TileMap tp = sweep_tile(LS.g[k], t, ht.id);
                tile_wait(ts, ht.id, cur, A);
                if (ht.tid == 0 && t + kTileTeams < ntiles) {   // every thread left buf[cur ^ 1] behind
                    float2* const tn[2] = {buf[cur ^ 1], buf[cur ^ 1]};
                    tile_fetch(tn, gs, 1, sweep_tile(LS.g[k], t + kTileTeams, ht.id), ts.bar + 2 * ht.id + (cur ^ 1));
                }
                float2* tile = buf[cur];
                if (LS.ng[k] == 0)   // the diagonal alone
                    pass_fwd<real, float2, true>(tile, kTileLowBits, 0u, true, ht, M, par, &tp);
                for (int gi = 0; gi < LS.ng[k]; ++gi) {
                    tp.s_loc = low ? LS.s[k][gi] : kTileLowBits;
                    pass_fwd<real, float2, true>(tile, LS.s[k][gi], LS.m[k][gi], dg && gi == LS.ng[k] - 1, ht, M, par,
                                                 &tp);
                    if (gi < LS.ng[k] - 1) ht.sync();
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                ht.sync();
                if (ht.tid == 0) {
                    float2* const tc2[2] = {tile, tile};
                    tile_store(tc2, gs, 1, tp);
                }
            }
            tile_sweep_done(ht);
            tm.sync();   // the next sweep reads tiles of both halves
        }
    }
}

// The adjoint of a tiled state, layers nl-1 .. 0: each layer's sweeps in reverse order, the
// first of them un-applying the diagonal before its rotations. A sweep's partial sums
// accumulate over each half's tiles (in tile order) in per-warp slots and are flushed once.
// Layer 0 only takes gradients (its rotations are not un-applied): only its diagonal sweep
// writes the tiles back, and the branch's top-qubit gradient follows the sweeps.
template <typename real>
__device__ void tiled_adjoint(const ConeArgs& A, const TeamMem<float2>& M, const Team& tm, const int32_t* body,
                              const int32_t* lofs, int nl, const float2* GT, real* red, double* gdst, TileSync& ts) {
    const int W = M.W;
    const int ntiles = 1 << (W - kTileBits);
    const int nw = nwarps_of(tm.tt);
    const Team ht = tile_half(tm);
    float2* tp_psi = M.tile + 2 * ht.id * padded_amps(kTileBits);
    float2* tp_lam = tp_psi + padded_amps(kTileBits);
    float2* const tiles[2] = {tp_psi, tp_lam};
    float2* const gs[2] = {M.psi, M.lam};
    int rpar = 0;
    for (int li = nl - 1; li >= 0; --li) {
        const int32_t* lp = body + lofs[li];
        const int ndiag = lp[0];
        const int par = li & 1;
        unsigned todo = (unsigned)lp[1];
        const bool top = li == 0 && ((todo >> W) & 1u);   // a branch: layer 0's rotation on the top qubit
        if (top) todo &= ~(1u << W);
        if (todo >> W) {
            if (tm.tid == 0) atomicOr(A.err, 1);
            return;
        }
        asm volatile("fence.proxy.async;" ::: "memory");   // plain writes of the states before the loads
        stage_layer<real, float2>(lp, GT, tm, M, par, true);
        LayerSweeps LS;
        layer_sweeps(todo, W, ndiag > 0, LS);
        for (int k = LS.n - 1; k >= 0; --k) {
            const bool dg = ndiag > 0 && k == LS.n - 1;
            const bool low = LS.g[k] == 0;
            const bool store = li > 0 || dg;
            real* rb = red + rpar * kMaxSweepSlots * nw;
            for (int t = ht.id; t < ntiles; t += kTileTeams) {
                TileMap tp = sweep_tile(LS.g[k], t, ht.id);
                if (ht.tid == 0) tile_fetch(tiles, gs, 2, tp, ts.bar + 2 * ht.id);
                tile_wait(ts, ht.id, 0, A);
                if (dg) {
                    pass_bwd<real, float2, true, false, true>(tp_psi, tp_lam, low ? kTileLowBits : LS.g[k], 0u, ht, M,
                                                              par, rb + 12 * nw, &tp);
                    if (LS.ng[k] > 0 || !store) ht.sync();
                }
                for (int gi = 0; gi < LS.ng[k]; ++gi) {
                    tp.s_loc = low ? LS.s[k][gi] : kTileLowBits;
                    if (li == 0)
                        pass_bwd<real, float2, false, true, true>(tp_psi, tp_lam, LS.s[k][gi], LS.m[k][gi], ht, M, par,
                                                                  rb + 4 * gi * nw, &tp);
                    else
                        pass_bwd<real, float2, false, false, true>(tp_psi, tp_lam, LS.s[k][gi], LS.m[k][gi], ht, M,
                                                                   par, rb + 4 * gi * nw, &tp);
                    if (gi < LS.ng[k] - 1 || !store) ht.sync();
                }
                if (store) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    ht.sync();
                    if (ht.tid == 0) tile_store(tiles, gs, 2, tp);
                }
            }
            tile_sweep_done(ht);
            tm.sync();   // both halves' tiles written back and partial sums complete
            for (int gi = 0; gi < LS.ng[k]; ++gi)
                flush_pass<real, float2>(rb + 4 * gi * nw, nw, LS.m[k][gi], LS.s[k][gi], M, par, false, gdst, tm);
            if (dg) flush_pass<real, float2>(rb + 12 * nw, nw, 0u, 0, M, par, true, gdst, tm);
            rpar ^= 1;
        }
        if (top) {
            real* rb = red + rpar * kMaxSweepSlots * nw;
            top_rotation_grad<real, float2>(M, (unsigned)lp[1], par, tm, rb);
            tm.sync();
            flush_pass<real, float2>(rb, nw, 1u, W, M, par, false, gdst, tm);
            rpar ^= 1;
        }
    }
}

template <typename real, bool GRAD, bool GLOBAL>
__device__ void run_cone(const ConeArgs& A, int cone_idx, int half, int b, const Team& tm, unsigned char* tb, int W,
                         int team_bytes, TileSync& ts) {
    using T2 = typename R2<real>::T;
    const SetRec* R = A.sets ? A.sets + b : nullptr;
    const ConeDev cd = R ? R->cones[cone_idx] : A.cones[cone_idx];
    const TeamLayout TL = team_layout(W, cd.W, tm.tt, (int)sizeof(real), GRAD, !GLOBAL);
    if (half > 2 || cd.W != W + (half ? 1 : 0) || TL.bytes > team_bytes || (half && (R ? R->prog : A.prog)[cd.prog_off] < 1)) {
        if (tm.tid == 0) atomicOr(A.err, 1);
        return;
    }
    TeamMem<T2> M;
    if (GLOBAL) {
        unsigned char* g = reinterpret_cast<unsigned char*>(A.gscratch) + (size_t)blockIdx.x * A.gscratch_slot;
        M.psi = reinterpret_cast<T2*>(g);
        M.lam = M.psi + padded_amps(W);
        M.tile = reinterpret_cast<T2*>(tb + TL.tile);
    } else {
        M.psi = reinterpret_cast<T2*>(tb + TL.psi);
        M.lam = reinterpret_cast<T2*>(tb + TL.lam);
    }
    M.tab = reinterpret_cast<T2*>(tb + TL.tab);
    M.info = tb + TL.info;
    M.red = tb + TL.red;
    M.tab1 = TL.tab1;
    M.tab2 = TL.tab2;
    M.tab_entries = TL.tab_entries;
    M.W = W;
    M.Wt = cd.W;
    M.hi = half ? (half - 1) << W : 0;
    const T2* GT = reinterpret_cast<const T2*>(A.gate_table) + (R ? (size_t)R->gt_off : (size_t)b * A.n_gates);
    real* red = reinterpret_cast<real*>(M.red);
    const int nw = nwarps_of(tm.tt);
    const int32_t* prog = (R ? R->prog : A.prog) + cd.prog_off;
    const int nl = prog[0];
    const int32_t* lofs = prog + 1;
    const int32_t* body = prog + 1 + nl;
    if (nl > 0) {   // layer 0 acts on |0..0>: write its product state (and phase) directly
        const int32_t* lp = body + lofs[0];
        stage_layer<real, T2>(lp, GT, tm, M, 0, false);
        init_product_state<real, T2>(M, (unsigned)lp[1], lp[0] > 0, tm, 0);
    } else {        // |0...0>
        for (int x = tm.tid; x < padded_amps(W); x += tm.tt) {
            T2 z;
            z.x = x == 0 ? 1 : 0;
            z.y = 0;
            M.psi[x] = z;   // pad16(0) == 0
        }
    }
    tm.sync();
    constexpr bool tiled = GLOBAL && sizeof(real) == 4;   // FP32 global-tier states are wider than a tile
    if constexpr (tiled) {
        if (W <= kTileBits) {
            if (tm.tid == 0) atomicOr(A.err, 1);
            return;
        }
        tiled_forward<real>(A, M, tm, body, lofs, nl, GT, ts);
    }
    for (int li = 1; li < nl && !tiled; ++li) {
        const int32_t* lp = body + lofs[li];
        const int ndiag = lp[0];
        const int par = li & 1;
        unsigned todo = (unsigned)lp[1];
        if (todo >> W) {   // a branch's top qubit has gates of layer 0 only
            if (tm.tid == 0) atomicOr(A.err, 1);
            return;
        }
        stage_layer<real, T2>(lp, GT, tm, M, par, false);
        bool first = true;
        while (todo || (first && ndiag > 0)) {
            int s;
            unsigned m;
            if (todo) {
                const int bt = __ffs(todo) - 1;
                s = bt < 4 ? 0 : (bt < W - 4 ? bt : W - 4);
                m = (todo >> s) & 15u;
                todo &= ~(15u << s);
            } else {
                s = W - 4;
                m = 0;
            }
            pass_fwd<real, T2>(M.psi, s, m, todo == 0 && ndiag > 0, tm, M, par);
            tm.sync();
            first = false;
        }
    }
    measure<real, T2, GRAD>(M, (R ? R->meas : A.meas) + cd.mterm_off, cd.nmterms, R ? R->term_coeff : A.term_coeff,
                            A.e_part + (R ? (size_t)R->e_off : (size_t)b * A.n_terms), tm, red);
    if (!GRAD) return;
    double* gdst = A.g_part + (R ? (size_t)R->g_off : (size_t)b * A.n_slots) + cd.slot_off;
    if constexpr (tiled) {
        tiled_adjoint<real>(A, M, tm, body, lofs, nl, GT, red, gdst, ts);
        return;
    }
    int rpar = 0;
    for (int li = nl - 1; li >= 0; --li) {
        const int32_t* lp = body + lofs[li];
        const int ndiag = lp[0];
        const int par = li & 1;
        unsigned todo = (unsigned)lp[1];
        stage_layer<real, T2>(lp, GT, tm, M, par, true);
        if (ndiag > 0) {   // the layer's diagonal first: its gradients, then its conjugate phase
            real* rb = red + rpar * kMaxPassSlots * nw;
            pass_bwd<real, T2, true>(M.psi, M.lam, W - 4, 0u, tm, M, par, rb);
            tm.sync();
            flush_pass<real, T2>(rb, nw, 0u, W - 4, M, par, true, gdst, tm);
            rpar ^= 1;
        }
        if (li == 0 && ((todo >> W) & 1u)) {   // a branch: layer 0's rotation on the window's top qubit
            real* rb = red + rpar * kMaxPassSlots * nw;
            top_rotation_grad<real, T2>(M, (unsigned)lp[1], par, tm, rb);
            tm.sync();
            flush_pass<real, T2>(rb, nw, 1u, W, M, par, false, gdst, tm);
            rpar ^= 1;
            todo &= ~(1u << W);
        }
        if (todo >> W) {
            if (tm.tid == 0) atomicOr(A.err, 1);
            return;
        }
        while (todo) {
            const int bt = 31 - __clz(todo);
            int s = bt - 3;
            if (s < 4) s = bt >= 4 ? 4 : 0;
            if (s > W - 4) s = W - 4;
            const unsigned m = (todo >> s) & 15u;
            todo &= ~(15u << s);
            real* rb = red + rpar * kMaxPassSlots * nw;
            if (li == 0) pass_bwd<real, T2, false, true>(M.psi, M.lam, s, m, tm, M, par, rb);
            else pass_bwd<real, T2, false>(M.psi, M.lam, s, m, tm, M, par, rb);
            tm.sync();
            flush_pass<real, T2>(rb, nw, m, s, M, par, false, gdst, tm);
            rpar ^= 1;
        }
    }
}

template <typename real, bool GRAD, bool GLOBAL>
__global__ void __launch_bounds__(GLOBAL ? kGlobalCtaThreads : kCtaThreads, GLOBAL ? kGlobalCtasPerSm : 1)
cone_kernel(ConeArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_chunk;
    __shared__ __align__(8) uint64_t s_tile_bar[2 * kTileTeams];   // tiled global tier: two per half
    TileSync ts{s_tile_bar, 0u};
    if constexpr (GLOBAL && sizeof(real) == 4) {
        if (threadIdx.x == 0) {
            for (int h = 0; h < 2 * kTileTeams; ++h) tc::mbar_init(s_tile_bar + h, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncthreads();
    }
    for (;;) {
        if (threadIdx.x == 0) s_chunk = A.chunk_begin + atomicAdd(A.counter, 1);
        __syncthreads();
        const int c = s_chunk;
        __syncthreads();
        if (c >= A.chunk_end) break;
        const ChunkDev ch = A.chunks[c];
        const int tt = ch.tt;
        const int team = threadIdx.x / tt;
        if (ch.W < kMinConeW || ch.W > kMaxConeW || tt < 16 || tt > (int)blockDim.x || ch.count > (int)blockDim.x / tt ||
            (!GLOBAL && ((1 << (ch.W - 4)) < kCtaThreads ? (1 << (ch.W - 4)) : kCtaThreads) != tt)) {
            if (threadIdx.x == 0) atomicOr(A.err, 1);
            continue;
        }
        if (team < ch.count) {
            Team tm;
            tm.tid = threadIdx.x - team * tt;
            tm.tt = tt;
            tm.id = team;
            const int lane = threadIdx.x & 31;
            tm.mask = tt >= 32 ? 0xffffffffu : (((1u << tt) - 1u) << (lane & ~(tt - 1)));
            const int item = ch.first + team;
            const int cw = A.items[2 * item], b = A.items[2 * item + 1];
            run_cone<real, GRAD, GLOBAL>(A, cw & kItemConeMask, (cw >> kItemHalfShift) & 3, b, tm,
                                         smem + (size_t)team * ch.team_bytes, ch.W, ch.team_bytes, ts);
        }
        __syncthreads();
    }
}

// ---- K0: gate tables ---------------------------------------------------------------------

// The same launch zeroes the cone kernel's work counters and, when window branches add into
// them, the partial energies and gradient slots (z0[0..n0), z1[0..n1)).
template <typename real>
__global__ void gate_table_kernel(const tlq_gate* gates, int n_gates, const double* theta, int n_params, int B,
                                  typename R2<real>::T* out, int32_t* counters, double* z0, long long n0, double* z1,
                                  long long n1) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * blockDim.x;
    if (i < 2) counters[i] = 0;
    for (long long k = i; k < n0; k += nth) z0[k] = 0.0;
    for (long long k = i; k < n1; k += nth) z1[k] = 0.0;
    if (i >= (long long)B * n_gates) return;
    const int b = (int)(i / n_gates), g = (int)(i % n_gates);
    const tlq_gate G = gates[g];
    const double a = G.param >= 0 ? theta[(size_t)b * n_params + G.param] : G.angle;
    double s, c;
    sincos(0.5 * a, &s, &c);
    typename R2<real>::T v;
    v.x = (real)c;
    v.y = (real)s;
    out[i] = v;
}

// ---- K5: fixed-order compensated reductions ---------------------------------------------

constexpr int kReduceThreads = 64;

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

// E_b = sum_t c_t e_{t,b}: one warp per set; lane l sums the terms t = l, l + 32, ... with a
// compensated sum (coalesced reads), then lane 0 adds the 32 partials in lane order. The
// order is fixed, so the result does not depend on the launch.
__device__ __forceinline__ void energy_warp(const double* e, const double* coeff, int T, int lane, double* out) {
    Neumaier acc;
    for (int t = lane; t < T; t += 32) acc.add(coeff[t] * e[t]);
    const double mine = acc.value();
    Neumaier tot;
    for (int l = 0; l < 32; ++l) {
        const double v = __shfl_sync(0xffffffffu, mine, l);
        if (lane == 0) tot.add(v);
    }
    if (lane == 0) *out = tot.value();
}

// g_p = sum over the slots k of parameter p of c_term(k) g_slot(k), compensated, in slot order;
// the slots are loaded eight at a time before they are added, so their latencies overlap.
__device__ __forceinline__ double grad_slots(const double* g, const int32_t* idx, const int32_t* term,
                                             const double* coeff, int k0, int k1) {
    Neumaier acc;
    for (int k = k0; k < k1; k += 8) {
        double v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (k + e < k1) {
                const int t = term[k + e];
                v[e] = (t >= 0 ? coeff[t] : 1.0) * g[idx[k + e]];
            }
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (k + e < k1) acc.add(v[e]);
    }
    return acc.value();
}

#ifndef TLQ_CONE_GLOBAL_TU
// Energies and gradients of a launch in one kernel: blocks [0, eb) hold one warp per set for
// the energies, the others one thread per (set, parameter) for the gradients (P = 0: none).
__global__ void reduce_kernel(const double* e_part, const double* coeff, int T, int B, double* energy, int eb,
                              const double* g_part, const int32_t* off, const int32_t* idx, const int32_t* term,
                              int P, int S, double* grad) {
    if ((int)blockIdx.x < eb) {
        const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
        if (b < B) energy_warp(e_part + (size_t)b * T, coeff, T, threadIdx.x & 31, energy + b);
        return;
    }
    const long long i = (long long)(blockIdx.x - eb) * blockDim.x + threadIdx.x;
    if (i >= (long long)B * P) return;
    const int b = (int)(i / P), p = (int)(i % P);
    grad[i] = grad_slots(g_part + (size_t)b * S, idx, term, coeff, off[p], off[p + 1]);
}
#endif

// ---- launchers -----------------------------------------------------------------------------

// The global-memory tier's launches (defined in the cone_global.cu translation unit).
int launch_cone_global(const ConeLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                       int32_t* counter, bool fp64, bool grad);
struct BatchLaunch;
int launch_batch_global(const BatchLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                        int32_t* counter, bool fp64, bool grad);

template <typename real, bool GRAD, bool GLOBAL>
static int launch_cone_t(const ConeLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                         int32_t* counter, int threads) {
    if (end <= begin) return 0;
    auto kern = cone_kernel<real, GRAD, GLOBAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    ConeArgs A;
    A.cones = L.cones;
    A.meas = L.meas;
    A.term_coeff = L.term_coeff;
    A.prog = L.prog;
    A.items = L.items;
    A.chunks = L.chunks;
    A.chunk_begin = begin;
    A.chunk_end = end;
    A.gate_table = L.gate_table;
    A.n_gates = L.n_gates;
    A.n_terms = L.n_terms;
    A.n_slots = L.n_slots;
    A.e_part = L.e_part;
    A.g_part = L.g_part;
    A.counter = counter;
    A.err = L.err;
    A.gscratch = L.gscratch;
    A.gscratch_slot = L.gscratch_slot;
    A.sets = nullptr;
    const int n = end - begin;
    if (grid > n) grid = n;
    kern<<<grid, GLOBAL ? kGlobalCtaThreads : threads, smem, st>>>(A);
    return (int)cudaGetLastError();
}

#ifdef TLQ_CONE_GLOBAL_TU
int launch_cone_global(const ConeLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                       int32_t* counter, bool fp64, bool grad) {
    if (fp64)
        return grad ? launch_cone_t<double, true, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads)
                    : launch_cone_t<double, false, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads);
    return grad ? launch_cone_t<float, true, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads)
                : launch_cone_t<float, false, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads);
}
#else
int cone_smem_grid(bool fp64, bool grad, int smem_bytes, int sm_count, int threads) {
    int per_sm = 0;
    cudaError_t e;
    if (fp64) {
        e = grad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<double, true, false>, threads, smem_bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<double, false, false>, threads, smem_bytes);
    } else {
        e = grad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<float, true, false>, threads, smem_bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<float, false, false>, threads, smem_bytes);
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * sm_count;
}

int team_bytes_host(int W, int Wt, int tt, bool fp64, bool grad, bool smem_state) {
    return team_layout(W, Wt, tt, fp64 ? 8 : 4, grad, smem_state).bytes;
}

int launch_cone(ConeLaunch& L, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const bool grad = L.grad != nullptr;
    cudaError_t e;
    // K0 (also zeroes the work counters and, for branch items, the partial sums they add into)
    {
        const long long n = (long long)L.B * L.n_gates;
        const int thr = 256;
        const int blocks = (int)((n + thr - 1) / thr) > 0 ? (int)((n + thr - 1) / thr) : 1;
        const long long n0 = L.accum ? (long long)L.B * L.n_terms : 0;
        const long long n1 = L.accum && grad ? (long long)L.B * L.n_slots : 0;
        if (L.fp64)
            gate_table_kernel<double><<<blocks, thr, 0, st>>>(L.gates, L.n_gates, L.theta, L.n_params, L.B,
                                                              (double2*)L.gate_table, L.counters, L.e_part, n0, L.g_part, n1);
        else
            gate_table_kernel<float><<<blocks, thr, 0, st>>>(L.gates, L.n_gates, L.theta, L.n_params, L.B,
                                                             (float2*)L.gate_table, L.counters, L.e_part, n0, L.g_part, n1);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    L.launches = 1 + (L.n_chunks_smem > 0) + (L.n_chunks > L.n_chunks_smem) + 1;
    const int smem_grid = cone_smem_grid(L.fp64, grad, L.smem_bytes, L.sm_count, L.smem_threads);
    if (L.ev_begin && (e = cudaEventRecord((cudaEvent_t)L.ev_begin, st)) != cudaSuccess) return (int)e;
    int rc;
    if (L.fp64) {
        rc = grad ? launch_cone_t<double, true, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters, L.smem_threads)
                  : launch_cone_t<double, false, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters, L.smem_threads);
    } else {
        rc = grad ? launch_cone_t<float, true, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters, L.smem_threads)
                  : launch_cone_t<float, false, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters, L.smem_threads);
    }
    if (rc) return rc;
    rc = launch_cone_global(L, st, L.n_chunks_smem, L.n_chunks, L.gsmem_bytes, L.g_grid, L.counters + 1, L.fp64, grad);
    if (rc) return rc;
    if (L.ev_end && (e = cudaEventRecord((cudaEvent_t)L.ev_end, st)) != cudaSuccess) return (int)e;
    {
        // small blocks (two warps): the compensated FP64 sums spread over every SM's FP64 units
        const int thr = kReduceThreads;
        const int eb = (L.B + thr / 32 - 1) / (thr / 32);   // one warp per set
        const int P = grad ? L.n_params : 0;
        const long long n = (long long)L.B * P;
        const int gb = (int)((n + thr - 1) / thr);
        reduce_kernel<<<eb + gb, thr, 0, st>>>(L.e_part, L.term_coeff, L.n_terms, L.B, L.energy, eb, L.g_part,
                                               L.pmap_off, L.pmap_idx, L.pmap_term, P, L.n_slots, L.grad);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    return 0;
}
#endif

// ---- serving batches: per-set records --------------------------------------------------------

// Also zeroes the batch's four work counters and, when window branches add into them, its
// partial energies and gradient slots (z0[0..n0), z1[0..n1)).
template <typename real>
__global__ void batch_gate_table_kernel(const SetRec* sets, typename R2<real>::T* out, int32_t* counters, double* z0,
                                        long long n0, double* z1, long long n1) {
    const long long t = ((long long)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    const long long nth = (long long)gridDim.x * gridDim.y * blockDim.x;
    if (t < 4) counters[t] = 0;
    for (long long k = t; k < n0; k += nth) z0[k] = 0.0;
    for (long long k = t; k < n1; k += nth) z1[k] = 0.0;
    const SetRec& R = sets[blockIdx.y];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= R.n_gates) return;
    const tlq_gate G = R.gates[g];
    const double a = G.param >= 0 ? R.theta[G.param] : G.angle;
    double s, c;
    sincos(0.5 * a, &s, &c);
    typename R2<real>::T v;
    v.x = (real)c;
    v.y = (real)s;
    out[R.gt_off + g] = v;
}

// The serving batch's energies and gradients in one kernel, in the summation orders of
// reduce_kernel, so a set's results are bit-identical served or computed synchronously:
// blocks [0, eb) hold one warp per set, the others cover (set, parameter) pairs, gx blocks of
// 256 parameters per set.
#ifndef TLQ_CONE_GLOBAL_TU
__global__ void batch_reduce_kernel(const SetRec* sets, int n_sets, const double* e_part, const double* g_part,
                                    int eb, int gx) {
    if ((int)blockIdx.x < eb) {
        const int b = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
        if (b >= n_sets) return;
        const SetRec& R = sets[b];
        energy_warp(e_part + R.e_off, R.term_coeff, R.n_terms, threadIdx.x & 31, R.energy);
        return;
    }
    const int q = (int)blockIdx.x - eb;
    const int b = q / gx;
    if (b >= n_sets) return;
    const SetRec& R = sets[b];
    const int p = (q - b * gx) * blockDim.x + threadIdx.x;
    if (!R.grad || p >= R.n_params) return;
    R.grad[p] = grad_slots(g_part + R.g_off, R.pmap_idx, R.pmap_term, R.term_coeff, R.pmap_off[p], R.pmap_off[p + 1]);
}
#endif

template <typename real, bool GRAD, bool GLOBAL>
static int launch_batch_t(const BatchLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                          int32_t* counter, int threads) {
    if (end <= begin) return 0;
    auto kern = cone_kernel<real, GRAD, GLOBAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    ConeArgs A{};
    A.items = L.items;
    A.chunks = L.chunks;
    A.chunk_begin = begin;
    A.chunk_end = end;
    A.gate_table = L.gate_table;
    A.e_part = L.e_part;
    A.g_part = L.g_part;
    A.counter = counter;
    A.err = L.err;
    A.gscratch = L.gscratch;
    A.gscratch_slot = L.gscratch_slot;
    A.sets = L.sets;
    const int n = end - begin;
    if (grid > n) grid = n;
    if (grid < 1) grid = 1;
    kern<<<grid, GLOBAL ? kGlobalCtaThreads : threads, smem, st>>>(A);
    return (int)cudaGetLastError();
}

#ifdef TLQ_CONE_GLOBAL_TU
int launch_batch_global(const BatchLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                        int32_t* counter, bool fp64, bool grad) {
    if (fp64)
        return grad ? launch_batch_t<double, true, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads)
                    : launch_batch_t<double, false, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads);
    return grad ? launch_batch_t<float, true, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads)
                : launch_batch_t<float, false, true>(L, st, begin, end, smem, grid, counter, kGlobalCtaThreads);
}
#else
template <typename real>
static int launch_batch_all(BatchLaunch& L, cudaStream_t st) {
    int rc;
    const int g0 = cone_smem_grid(sizeof(real) == 8, false, L.smem_bytes[0] > 0 ? L.smem_bytes[0] : 1024, L.sm_count,
                                  L.smem_threads[0]);
    const int g1 = cone_smem_grid(sizeof(real) == 8, true, L.smem_bytes[1] > 0 ? L.smem_bytes[1] : 1024, L.sm_count,
                                  L.smem_threads[1]);
    if ((rc = launch_batch_t<real, false, false>(L, st, L.range[0], L.range[1], L.smem_bytes[0], g0, L.counters + 0,
                                                 L.smem_threads[0])))
        return rc;
    if ((rc = launch_batch_global(L, st, L.range[1], L.range[2], L.gsmem_bytes[0], L.g_grid, L.counters + 1,
                                  sizeof(real) == 8, false)))
        return rc;
    if ((rc = launch_batch_t<real, true, false>(L, st, L.range[2], L.range[3], L.smem_bytes[1], g1, L.counters + 2,
                                                L.smem_threads[1])))
        return rc;
    if ((rc = launch_batch_global(L, st, L.range[3], L.range[4], L.gsmem_bytes[1], L.g_grid, L.counters + 3,
                                  sizeof(real) == 8, true)))
        return rc;
    for (int k = 0; k < 4; ++k) L.launches += L.range[k + 1] > L.range[k];
    return 0;
}

int launch_cone_batch(BatchLaunch& L, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e;
    L.launches = 0;
    if (L.n_sets <= 0) return 0;
    const dim3 gk((L.max_gates + 255) / 256 > 0 ? (L.max_gates + 255) / 256 : 1, L.n_sets);
    // the gate tables, the work counters and (branch items add their shares) the partial sums
    const long long n0 = L.accum ? (long long)L.e_count : 0, n1 = L.accum ? (long long)L.g_count : 0;
    if (L.fp64)
        batch_gate_table_kernel<double><<<gk, 256, 0, st>>>(L.sets, (double2*)L.gate_table, L.counters, L.e_part, n0,
                                                            L.g_part, n1);
    else
        batch_gate_table_kernel<float><<<gk, 256, 0, st>>>(L.sets, (float2*)L.gate_table, L.counters, L.e_part, n0,
                                                           L.g_part, n1);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    const int rc = L.fp64 ? launch_batch_all<double>(L, st) : launch_batch_all<float>(L, st);
    if (rc) return rc;
    {
        const int eb = (L.n_sets + 7) / 8;   // 8 warps per block
        const int gx = (L.max_params > 0 && L.range[4] > L.range[2]) ? (L.max_params + 255) / 256 : 0;
        batch_reduce_kernel<<<eb + gx * L.n_sets, 256, 0, st>>>(L.sets, L.n_sets, L.e_part, L.g_part, eb, gx);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    L.launches += 2;
    return 0;
}
#endif

}  // namespace tlq
