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
//   energy_reduce / grad_reduce (K5) fixed-order Neumaier sums over terms in FP64, so a
//                           result does not depend on batching or scheduling.
#include "internal.h"

#include <cuda_runtime.h>
#include <cstdio>

namespace tlq {

template <typename real> struct R2;
template <> struct R2<float> { using T = float2; };
template <> struct R2<double> { using T = double2; };

// Bank-conflict-free placement of amplitude a: XOR the low 4 index bits with bits 4..7.
// For every pass (registers on bits [s, s+4) with s = 0 or s >= 4) the 16 lanes of a
// half-warp (8-byte words) or 8 lanes of a quarter-warp (16-byte words) then hit distinct
// banks. It is a bijection on [0, 2^W).
__host__ __device__ __forceinline__ int swz(int a) { return a ^ ((a >> 4) & 15); }

// ---- per-team shared-memory layout ----------------------------------------------------

struct TeamLayout {
    int psi, lam, tab, cs, kinds, rslot, red, bytes;
    int nch;            // phase-table chunks
    int tab_off[3];     // entry offsets of the chunk tables
};

__host__ __device__ inline int nwarps_of(int tt) { return tt >= 32 ? tt / 32 : 1; }

__host__ __device__ inline TeamLayout team_layout(int W, int tt, int real_bytes, bool grad, bool smem_state) {
    TeamLayout L{};
    const int r2 = 2 * real_bytes;
    int off = 0;
    L.psi = off;
    if (smem_state) off += (1 << W) * r2;
    L.lam = off;
    if (smem_state && grad) off += (1 << W) * r2;
    L.nch = (W + 6) / 7;
    int ent = 0;
    for (int c = 0; c < L.nch; ++c) {
        int bc = (W - 7 * c) < 7 ? (W - 7 * c) : 7;
        L.tab_off[c] = ent;
        ent += c == 0 ? (1 << bc) : (1 << (bc + 1));
    }
    L.tab = off;
    off += ent * r2;
    L.cs = off;
    off += 32 * r2;
    L.kinds = off;
    off += 32 * 4;
    L.rslot = off;
    off += 32 * 4;
    off = (off + 15) & ~15;
    L.red = off;
    off += 2 * kMaxPassSlots * nwarps_of(tt) * real_bytes;
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
    const int top = tm.tt < 32 ? tm.tt : 32;
    for (int off = top >> 1; off > 0; off >>= 1) v += __shfl_xor_sync(tm.mask, v, off);
    return v;
}

// ---- complex helpers ---------------------------------------------------------------------

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

// RY(a) on register bit K: [[c,-s],[s,c]] on (amp with bit 0, amp with bit 1).
template <int K, typename T2, typename real>
__device__ __forceinline__ void apply_ry(T2 (&v)[16], real c, real s) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        T2 a0 = v[j], a1 = v[j | (1 << K)];
        v[j].x = c * a0.x - s * a1.x;
        v[j].y = c * a0.y - s * a1.y;
        v[j | (1 << K)].x = s * a0.x + c * a1.x;
        v[j | (1 << K)].y = s * a0.y + c * a1.y;
    }
}

// RX(a) on register bit K: [[c,-is],[-is,c]].
template <int K, typename T2, typename real>
__device__ __forceinline__ void apply_rx(T2 (&v)[16], real c, real s) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        T2 a0 = v[j], a1 = v[j | (1 << K)];
        v[j].x = c * a0.x + s * a1.y;
        v[j].y = c * a0.y - s * a1.x;
        v[j | (1 << K)].x = c * a1.x + s * a0.y;
        v[j | (1 << K)].y = c * a1.y - s * a0.x;
    }
}

template <int K, typename T2, typename real>
__device__ __forceinline__ void apply_rot(T2 (&v)[16], int kind, real c, real s) {
    if (kind == TLQ_RY) apply_ry<K>(v, c, s);
    else apply_rx<K>(v, c, s);
}

// Im <lam| G |psi> over the pairs of register bit K, G = Y (RY) or X (RX).
template <int K, typename T2, typename real>
__device__ __forceinline__ real grad_rot(const T2 (&p)[16], const T2 (&l)[16], int kind) {
    real acc = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const T2 p0 = p[j], p1 = p[j | (1 << K)], l0 = l[j], l1 = l[j | (1 << K)];
        if (kind == TLQ_RY) {
            // Y|0> = i|1>, Y|1> = -i|0>: Im<l|Y p> = Re(conj(l1) p0) - Re(conj(l0) p1)
            acc += (l1.x * p0.x + l1.y * p0.y) - (l0.x * p1.x + l0.y * p1.y);
        } else {
            // Im<l|X p> = Im(conj(l0) p1 + conj(l1) p0)
            acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
        }
    }
    return acc;
}

// Diagonal phase of window index x: product of the per-chunk table entries.
template <typename T2>
__device__ __forceinline__ T2 phase_of(const T2* tab, const TeamLayout& TL, int W, int x) {
    T2 ph = tab[x & 127];
    if (W > 7) {
#pragma unroll
        for (int c = 1; c < 3; ++c) {
            if (c >= TL.nch) break;
            const int bc = (W - 7 * c) < 7 ? (W - 7 * c) : 7;
            const int idx = ((x >> (7 * c)) & ((1 << bc) - 1)) | (((x >> (7 * c - 1)) & 1) << bc);
            ph = cmul(ph, tab[TL.tab_off[c] + idx]);
        }
    }
    return ph;
}

// ---- kernel parameters ---------------------------------------------------------------------

struct ConeArgs {
    const ConeDev* cones;
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
};

// Stage one layer's rotation parameters and build its diagonal phase table (conjugated
// for the adjoint direction). Returns the live-group mask (bit g: window bits [4g,4g+4)).
template <typename real, typename T2>
__device__ unsigned stage_layer(const int32_t* lp, int W, const T2* GT, const Team& tm, const TeamLayout& TL,
                                unsigned char* tb, bool conj_phase) {
    T2* cs = reinterpret_cast<T2*>(tb + TL.cs);
    int* kinds = reinterpret_cast<int*>(tb + TL.kinds);
    int* rslot = reinterpret_cast<int*>(tb + TL.rslot);
    T2* tab = reinterpret_cast<T2*>(tb + TL.tab);
    const int nrot = lp[0], ndiag = lp[1];
    const int32_t* rot = lp + 2;
    const int32_t* dg = rot + 3 * nrot;
    tm.sync();   // previous users of cs/kinds/rslot/tab are done
    for (int j = tm.tid; j < 32; j += tm.tt) kinds[j] = -1;
    tm.sync();
    for (int k = tm.tid; k < nrot; k += tm.tt) {
        const int w0 = rot[3 * k];
        const int j = w0 & 255;
        kinds[j] = w0 >> 8;
        T2 v = GT[rot[3 * k + 1]];
        cs[j] = v;
        rslot[j] = rot[3 * k + 2];
    }
    if (ndiag > 0) {
        int total = TL.nch == 1 ? (1 << W) : 0;
        if (TL.nch > 1) {
            const int bl = (W - 7 * (TL.nch - 1));
            total = TL.tab_off[TL.nch - 1] + (1 << (bl + 1));
        }
        for (int e = tm.tid; e < total; e += tm.tt) {
            int c = 0;
            while (c + 1 < TL.nch && e >= TL.tab_off[c + 1]) ++c;
            const int idx = e - TL.tab_off[c];
            const int lo = 7 * c;
            const int bc = (W - lo) < 7 ? (W - lo) : 7;
            T2 ph;
            ph.x = 1;
            ph.y = 0;
            for (int k = 0; k < ndiag; ++k) {
                const int w0 = dg[3 * k];
                const int kind = w0 & 255, j0 = (w0 >> 8) & 255, j1 = (w0 >> 16) & 255;
                const bool two = (kind != TLQ_RZ);
                const int own = two ? j1 : j0;
                if (own < lo || own >= lo + bc) continue;
                auto bit_of = [&](int q) -> int {
                    if (q >= lo) return (idx >> (q - lo)) & 1;
                    return (idx >> bc) & 1;   // q == lo - 1, the crossing bit
                };
                if (kind == TLQ_CZ) {
                    if (bit_of(j0) & bit_of(j1)) { ph.x = -ph.x; ph.y = -ph.y; }
                    continue;
                }
                const T2 g = GT[dg[3 * k + 1]];
                const int odd = two ? (bit_of(j0) ^ bit_of(j1)) : bit_of(j0);
                T2 f;
                f.x = g.x;
                f.y = odd ? g.y : -g.y;   // exp(-i a z/2): z = +1 -> e^{-ia/2}
                ph = cmul(ph, f);
            }
            if (conj_phase) ph.y = -ph.y;
            tab[e] = ph;
        }
    }
    tm.sync();
    unsigned live = 0;
    for (int g = 0; 4 * g < W; ++g) {
        bool any = false;
        for (int q = 4 * g; q < 4 * g + 4 && q < W; ++q) any |= kinds[q] >= 0;
        if (any) live |= 1u << g;
    }
    return live;
}

// Forward pass over register bits [s, s+4): rotations on `apply` bits, then the
// diagonal phase when `diag`.
template <typename real, typename T2>
__device__ void pass_fwd(T2* psi, int W, int s, unsigned apply, bool diag, const Team& tm, const TeamLayout& TL,
                         unsigned char* tb) {
    const T2* cs = reinterpret_cast<const T2*>(tb + TL.cs);
    const int* kinds = reinterpret_cast<const int*>(tb + TL.kinds);
    const T2* tab = reinterpret_cast<const T2*>(tb + TL.tab);
    int kd[4];
    real c[4], sn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kd[k] = (apply >> k) & 1 ? kinds[s + k] : -1;
        T2 v = cs[s + k];
        c[k] = v.x;
        sn[k] = v.y;
    }
    const int nout = 1 << (W - 4);
    const int lowmask = (1 << s) - 1;
    for (int o = tm.tid; o < nout; o += tm.tt) {
        const int base = (o & lowmask) | ((o >> s) << (s + 4));
        T2 v[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = psi[swz(base | (j << s))];
        if (kd[0] >= 0) apply_rot<0>(v, kd[0], c[0], sn[0]);
        if (kd[1] >= 0) apply_rot<1>(v, kd[1], c[1], sn[1]);
        if (kd[2] >= 0) apply_rot<2>(v, kd[2], c[2], sn[2]);
        if (kd[3] >= 0) apply_rot<3>(v, kd[3], c[3], sn[3]);
        if (diag) {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = cmul(v[j], phase_of(tab, TL, W, base | (j << s)));
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) psi[swz(base | (j << s))] = v[j];
    }
}

// Adjoint pass over register bits [s, s+4): when `diag`, emit Im<lam|Z..|psi> for the
// layer's parametrised diagonal gates and un-apply the diagonal; then for each rotation
// on `apply` bits emit Im<lam|G|psi> and un-apply it from psi and lam.
// Per-warp partial sums go to red[slot * nw + warp]: slots 0..3 rotations (register bit),
// slots 4.. diagonal gates in program order.
template <typename real, typename T2>
__device__ void pass_bwd(T2* psi, T2* lam, int W, int s, unsigned apply, bool diag, const int32_t* dg, int ndiag,
                         const Team& tm, const TeamLayout& TL, unsigned char* tb, real* red) {
    const T2* cs = reinterpret_cast<const T2*>(tb + TL.cs);
    const int* kinds = reinterpret_cast<const int*>(tb + TL.kinds);
    const T2* tab = reinterpret_cast<const T2*>(tb + TL.tab);
    const int nw = nwarps_of(tm.tt);
    const int warp = tm.tt >= 32 ? (tm.tid >> 5) : 0;
    const bool leader = tm.tt >= 32 ? ((tm.tid & 31) == 0) : (tm.tid == 0);
    int kd[4];
    real c[4], sn[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        kd[k] = (apply >> k) & 1 ? kinds[s + k] : -1;
        T2 v = cs[s + k];
        c[k] = v.x;
        sn[k] = -v.y;   // un-apply: angle -> -angle
    }
    const int nout = 1 << (W - 4);
    const int lowmask = (1 << s) - 1;
    bool first = true;
    for (int o = tm.tid; o < nout || (first && o - tm.tid < nout); o += tm.tt) {
        // every team thread takes part in the reductions, even without an amplitude block
        const bool has = o < nout;
        const int base = has ? ((o & lowmask) | ((o >> s) << (s + 4))) : 0;
        T2 p[16], l[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (has) {
                p[j] = psi[swz(base | (j << s))];
                l[j] = lam[swz(base | (j << s))];
            } else {
                p[j].x = p[j].y = 0;
                l[j].x = l[j].y = 0;
            }
        }
        if (diag) {
            // w_x = Im(conj(lam_x) psi_x); dE/da for RZ on q: sum_x z_q(x) w_x; RZZ: z_q0 z_q1 w_x.
            real S = 0, Sk[4] = {0, 0, 0, 0}, Sp[3] = {0, 0, 0};
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const real w = l[j].x * p[j].y - l[j].y * p[j].x;
                S += w;
#pragma unroll
                for (int k = 0; k < 4; ++k) Sk[k] += ((j >> k) & 1) ? -w : w;
#pragma unroll
                for (int k = 0; k < 3; ++k) Sp[k] += (((j >> k) ^ (j >> (k + 1))) & 1) ? -w : w;
            }
            int sl = 4;
            for (int k = 0; k < ndiag; ++k) {
                const int w0 = dg[3 * k];
                if (dg[3 * k + 2] < 0) continue;
                const int kind = w0 & 255, j0 = (w0 >> 8) & 255, j1 = (w0 >> 16) & 255;
                real val;
                const bool in0 = j0 >= s && j0 < s + 4;
                if (kind == TLQ_RZ) {
                    if (in0) {
                        const int k0 = j0 - s;
                        val = k0 == 0 ? Sk[0] : k0 == 1 ? Sk[1] : k0 == 2 ? Sk[2] : Sk[3];
                    } else {
                        val = ((base >> j0) & 1) ? -S : S;
                    }
                } else {   // RZZ on (j0, j1 = j0 + 1)
                    const bool in1 = j1 >= s && j1 < s + 4;
                    if (in0 && in1) {
                        const int k0 = j0 - s;
                        val = k0 == 0 ? Sp[0] : k0 == 1 ? Sp[1] : Sp[2];
                    } else if (in0) {   // j0 = s + 3, j1 outside
                        val = ((base >> j1) & 1) ? -Sk[3] : Sk[3];
                    } else if (in1) {   // j1 = s, j0 = s - 1 outside
                        val = ((base >> j0) & 1) ? -Sk[0] : Sk[0];
                    } else {
                        val = (((base >> j0) ^ (base >> j1)) & 1) ? -S : S;
                    }
                }
                val = team_warp_sum(val, tm);
                if (leader) {
                    real* dst = red + sl * nw + warp;
                    *dst = first ? val : *dst + val;
                }
                ++sl;
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const T2 ph = phase_of(tab, TL, W, base | (j << s));   // already conjugated
                p[j] = cmul(p[j], ph);
                l[j] = cmul(l[j], ph);
            }
        }
        real gk[4] = {0, 0, 0, 0};
        if (kd[0] >= 0) { gk[0] = grad_rot<0, T2, real>(p, l, kd[0]); apply_rot<0>(p, kd[0], c[0], sn[0]); apply_rot<0>(l, kd[0], c[0], sn[0]); }
        if (kd[1] >= 0) { gk[1] = grad_rot<1, T2, real>(p, l, kd[1]); apply_rot<1>(p, kd[1], c[1], sn[1]); apply_rot<1>(l, kd[1], c[1], sn[1]); }
        if (kd[2] >= 0) { gk[2] = grad_rot<2, T2, real>(p, l, kd[2]); apply_rot<2>(p, kd[2], c[2], sn[2]); apply_rot<2>(l, kd[2], c[2], sn[2]); }
        if (kd[3] >= 0) { gk[3] = grad_rot<3, T2, real>(p, l, kd[3]); apply_rot<3>(p, kd[3], c[3], sn[3]); apply_rot<3>(l, kd[3], c[3], sn[3]); }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (kd[k] < 0) continue;
            const real val = team_warp_sum(gk[k], tm);
            if (leader) {
                real* dst = red + k * nw + warp;
                *dst = first ? val : *dst + val;
            }
        }
        if (has) {
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                psi[swz(base | (j << s))] = p[j];
                lam[swz(base | (j << s))] = l[j];
            }
        }
        first = false;
    }
}

// Sum the per-warp partials of one pass in fixed order and store them as FP64 slots.
template <typename real>
__device__ void flush_pass(const real* red, int nw, unsigned apply, int s, const int* kinds, const int* rslot,
                           const int32_t* dg, int ndiag, bool diag, double* gdst, const Team& tm) {
    // rotation slots
    for (int k = tm.tid; k < 4; k += tm.tt) {
        if (!((apply >> k) & 1) || kinds[s + k] < 0) continue;
        const int slot = rslot[s + k];
        if (slot < 0) continue;
        double acc = 0;
        for (int w = 0; w < nw; ++w) acc += (double)red[k * nw + w];
        gdst[slot] = acc;
    }
    if (!diag) return;
    int sl = 4;
    for (int k = 0; k < ndiag; ++k) {
        const int slot = dg[3 * k + 2];
        if (slot < 0) continue;
        if (((sl - 4) % tm.tt) == tm.tid) {
            double acc = 0;
            for (int w = 0; w < nw; ++w) acc += (double)red[sl * nw + w];
            gdst[slot] = acc;
        }
        ++sl;
    }
}

// <psi|P|psi> for the cone's Pauli term; when GRAD also lam = P psi.
template <typename real, typename T2, bool GRAD>
__device__ double measure(T2* psi, T2* lam, int W, const ConeDev& cd, const Team& tm, real* red) {
    const int nout = 1 << (W - 4);
    T2 f0;   // (-i)^ny
    const int ny = cd.ny & 3;
    f0.x = ny == 0 ? 1 : ny == 2 ? -1 : 0;
    f0.y = ny == 1 ? -1 : ny == 3 ? 1 : 0;
    real acc = 0;
    for (int o = tm.tid; o < nout; o += tm.tt) {
#pragma unroll 4
        for (int j = 0; j < 16; ++j) {
            const int x = (o << 4) | j;
            const T2 a = psi[swz(x)];
            const T2 v = psi[swz(x ^ (int)cd.flip)];
            T2 lv = cmul(f0, v);
            if (__popc((unsigned)x & cd.zy) & 1) { lv.x = -lv.x; lv.y = -lv.y; }
            if (GRAD) lam[swz(x)] = lv;
            acc += a.x * lv.x + a.y * lv.y;
        }
    }
    acc = team_warp_sum(acc, tm);
    const int nw = nwarps_of(tm.tt);
    const int warp = tm.tt >= 32 ? (tm.tid >> 5) : 0;
    const bool leader = tm.tt >= 32 ? ((tm.tid & 31) == 0) : (tm.tid == 0);
    if (leader) red[warp] = acc;
    tm.sync();
    double e = 0;
    for (int w = 0; w < nw; ++w) e += (double)red[w];
    tm.sync();
    return e;
}

template <typename real, bool GRAD, bool GLOBAL>
__device__ void run_cone(const ConeArgs& A, int cone_idx, int b, const Team& tm, unsigned char* tb, int W) {
    using T2 = typename R2<real>::T;
    const ConeDev cd = A.cones[cone_idx];
    const TeamLayout TL = team_layout(W, tm.tt, (int)sizeof(real), GRAD, !GLOBAL);
    T2* psi;
    T2* lam;
    if (GLOBAL) {
        unsigned char* g = reinterpret_cast<unsigned char*>(A.gscratch) + (size_t)blockIdx.x * A.gscratch_slot;
        psi = reinterpret_cast<T2*>(g);
        lam = psi + (1 << W);
    } else {
        psi = reinterpret_cast<T2*>(tb + TL.psi);
        lam = reinterpret_cast<T2*>(tb + TL.lam);
    }
    const T2* GT = reinterpret_cast<const T2*>(A.gate_table) + (size_t)b * A.n_gates;
    real* red = reinterpret_cast<real*>(tb + TL.red);
    const int nw = nwarps_of(tm.tt);
    // |0...0>
    for (int x = tm.tid; x < (1 << W); x += tm.tt) {
        T2 z;
        z.x = x == 0 ? 1 : 0;
        z.y = 0;
        psi[x] = z;   // swz(0) == 0
    }
    const int32_t* prog = A.prog + cd.prog_off;
    const int nl = prog[0];
    const int32_t* lofs = prog + 1;
    const int32_t* body = prog + 1 + nl;
    for (int li = 0; li < nl; ++li) {
        const int32_t* lp = body + lofs[li];
        const int ndiag = lp[1];
        unsigned live = stage_layer<real, T2>(lp, W, GT, tm, TL, tb, false);
        int last = -1;
        for (int g = 0; 4 * g < W; ++g) if ((live >> g) & 1) last = g;
        if (last < 0 && ndiag > 0) { live = 1; last = 0; }
        for (int g = 0; g <= last; ++g) {
            if (!((live >> g) & 1)) continue;
            const int s = 4 * g < W - 4 ? 4 * g : W - 4;
            unsigned apply = 0;
            for (int k = 0; k < 4; ++k) {
                const int q = s + k;
                if (q >= 4 * g && q < 4 * g + 4) apply |= 1u << k;
            }
            pass_fwd<real, T2>(psi, W, s, apply, g == last && ndiag > 0, tm, TL, tb);
            tm.sync();
        }
    }
    const double e = measure<real, T2, GRAD>(psi, lam, W, cd, tm, red);
    if (tm.tid == 0) A.e_part[(size_t)b * A.n_terms + cd.term] = e;
    if (!GRAD) return;
    tm.sync();
    double* gdst = A.g_part + (size_t)b * A.n_slots + cd.slot_off;
    const int* kinds = reinterpret_cast<const int*>(tb + TL.kinds);
    const int* rslot = reinterpret_cast<const int*>(tb + TL.rslot);
    int parity = 0;
    for (int li = nl - 1; li >= 0; --li) {
        const int32_t* lp = body + lofs[li];
        const int nrot = lp[0], ndiag = lp[1];
        const int32_t* dg = lp + 2 + 3 * nrot;
        unsigned live = stage_layer<real, T2>(lp, W, GT, tm, TL, tb, true);
        int first = -1;
        for (int g = 0; 4 * g < W; ++g) if ((live >> g) & 1) { first = g; break; }
        if (first < 0 && ndiag > 0) { live = 1; first = 0; }
        for (int g = first; g >= 0 && 4 * g < W; ++g) {
            if (!((live >> g) & 1)) continue;
            const int s = 4 * g < W - 4 ? 4 * g : W - 4;
            unsigned apply = 0;
            for (int k = 0; k < 4; ++k) {
                const int q = s + k;
                if (q >= 4 * g && q < 4 * g + 4) apply |= 1u << k;
            }
            real* rb = red + parity * kMaxPassSlots * nw;
            const bool dpass = (g == first) && ndiag > 0;
            pass_bwd<real, T2>(psi, lam, W, s, apply, dpass, dg, ndiag, tm, TL, tb, rb);
            tm.sync();
            flush_pass<real>(rb, nw, apply, s, kinds, rslot, dg, ndiag, dpass, gdst, tm);
            parity ^= 1;
        }
    }
}

template <typename real, bool GRAD, bool GLOBAL>
__global__ void __launch_bounds__(kCtaThreads, 1) cone_kernel(ConeArgs A) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_chunk;
    for (;;) {
        if (threadIdx.x == 0) s_chunk = A.chunk_begin + atomicAdd(A.counter, 1);
        __syncthreads();
        const int c = s_chunk;
        __syncthreads();
        if (c >= A.chunk_end) break;
        const ChunkDev ch = A.chunks[c];
        const int tt = ch.tt;
        const int team = threadIdx.x / tt;
        const int nteams = kCtaThreads / tt;
        if (ch.W < kMinConeW || ch.W > kMaxConeW || tt < 16 || (!GLOBAL && (1 << (ch.W - 4)) != tt && tt != kCtaThreads)) {
            if (threadIdx.x == 0) atomicOr(A.err, 1);
            continue;
        }
        if (team < ch.count && team < nteams) {
            Team tm;
            tm.tid = threadIdx.x - team * tt;
            tm.tt = tt;
            tm.id = team;
            const int lane = threadIdx.x & 31;
            tm.mask = tt >= 32 ? 0xffffffffu : (((1u << tt) - 1u) << (lane & ~(tt - 1)));
            const int item = ch.first + team;
            const int cone = A.items[2 * item], b = A.items[2 * item + 1];
            run_cone<real, GRAD, GLOBAL>(A, cone, b, tm, smem + (size_t)team * ch.team_bytes, ch.W);
        }
        __syncthreads();
    }
}

// ---- K0: gate tables ---------------------------------------------------------------------

template <typename real>
__global__ void gate_table_kernel(const tlq_gate* gates, int n_gates, const double* theta, int n_params, int B,
                                  typename R2<real>::T* out) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
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

__global__ void energy_reduce_kernel(const double* e_part, const double* coeff, int T, int B, double* energy) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    Neumaier acc;
    for (int t = 0; t < T; ++t) acc.add(coeff[t] * e_part[(size_t)b * T + t]);
    energy[b] = acc.value();
}

__global__ void grad_reduce_kernel(const double* g_part, const int32_t* off, const int32_t* idx, const double* coeff,
                                   int P, int S, int B, double* grad) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)B * P) return;
    const int b = (int)(i / P), p = (int)(i % P);
    Neumaier acc;
    for (int k = off[p]; k < off[p + 1]; ++k) acc.add(coeff[k] * g_part[(size_t)b * S + idx[k]]);
    grad[i] = acc.value();
}

// ---- launchers -----------------------------------------------------------------------------

template <typename real, bool GRAD, bool GLOBAL>
static int launch_cone_t(const ConeLaunch& L, cudaStream_t st, int begin, int end, int smem, int grid,
                         int32_t* counter) {
    if (end <= begin) return 0;
    auto kern = cone_kernel<real, GRAD, GLOBAL>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return (int)e;
    ConeArgs A;
    A.cones = L.cones;
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
    const int n = end - begin;
    if (grid > n) grid = n;
    kern<<<grid, kCtaThreads, smem, st>>>(A);
    return (int)cudaGetLastError();
}

int cone_smem_grid(bool fp64, bool grad, int smem_bytes, int sm_count) {
    int per_sm = 0;
    cudaError_t e;
    if (fp64) {
        e = grad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<double, true, false>, kCtaThreads, smem_bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<double, false, false>, kCtaThreads, smem_bytes);
    } else {
        e = grad ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<float, true, false>, kCtaThreads, smem_bytes)
                 : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cone_kernel<float, false, false>, kCtaThreads, smem_bytes);
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * sm_count;
}

int team_bytes_host(int W, int tt, bool fp64, bool grad, bool smem_state) {
    return team_layout(W, tt, fp64 ? 8 : 4, grad, smem_state).bytes;
}

int launch_cone(ConeLaunch& L, void* stream) {
    cudaStream_t st = (cudaStream_t)stream;
    const bool grad = L.grad != nullptr;
    cudaError_t e;
    // K0
    {
        const long long n = (long long)L.B * L.n_gates;
        const int thr = 256;
        const int blocks = (int)((n + thr - 1) / thr);
        if (L.fp64) gate_table_kernel<double><<<blocks, thr, 0, st>>>(L.gates, L.n_gates, L.theta, L.n_params, L.B, (double2*)L.gate_table);
        else gate_table_kernel<float><<<blocks, thr, 0, st>>>(L.gates, L.n_gates, L.theta, L.n_params, L.B, (float2*)L.gate_table);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    if ((e = cudaMemsetAsync(L.counters, 0, 2 * sizeof(int32_t), st)) != cudaSuccess) return (int)e;
    L.launches = 1 + (L.n_chunks_smem > 0) + (L.n_chunks > L.n_chunks_smem) + 1 + (grad ? 1 : 0);
    if (L.ev_begin && (e = cudaEventRecord((cudaEvent_t)L.ev_begin, st)) != cudaSuccess) return (int)e;
    int rc;
    const int smem_grid = cone_smem_grid(L.fp64, grad, L.smem_bytes, L.sm_count);
    if (L.fp64) {
        rc = grad ? launch_cone_t<double, true, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters)
                  : launch_cone_t<double, false, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters);
        if (rc) return rc;
        rc = grad ? launch_cone_t<double, true, true>(L, st, L.n_chunks_smem, L.n_chunks, L.gsmem_bytes, L.g_grid, L.counters + 1)
                  : launch_cone_t<double, false, true>(L, st, L.n_chunks_smem, L.n_chunks, L.gsmem_bytes, L.g_grid, L.counters + 1);
    } else {
        rc = grad ? launch_cone_t<float, true, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters)
                  : launch_cone_t<float, false, false>(L, st, 0, L.n_chunks_smem, L.smem_bytes, smem_grid, L.counters);
        if (rc) return rc;
        rc = grad ? launch_cone_t<float, true, true>(L, st, L.n_chunks_smem, L.n_chunks, L.gsmem_bytes, L.g_grid, L.counters + 1)
                  : launch_cone_t<float, false, true>(L, st, L.n_chunks_smem, L.n_chunks, L.gsmem_bytes, L.g_grid, L.counters + 1);
    }
    if (rc) return rc;
    if (L.ev_end && (e = cudaEventRecord((cudaEvent_t)L.ev_end, st)) != cudaSuccess) return (int)e;
    energy_reduce_kernel<<<(L.B + 127) / 128, 128, 0, st>>>(L.e_part, L.term_coeff, L.n_terms, L.B, L.energy);
    if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    if (grad) {
        const long long n = (long long)L.B * L.n_params;
        grad_reduce_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(L.g_part, L.pmap_off, L.pmap_idx, L.pmap_coeff,
                                                                   L.n_params, L.n_slots, L.B, L.grad);
        if ((e = cudaGetLastError()) != cudaSuccess) return (int)e;
    }
    return 0;
}

}  // namespace tlq
