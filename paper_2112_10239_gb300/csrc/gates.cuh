// Register-level gate helpers shared by the cone kernel (cone.cu) and the dense
// statevector passes (dense.cu): a thread holds 16 amplitudes that differ in 4 index bits
// ("register bits"); rotations on those bits are 2x2 updates of amplitude pairs.
#pragma once

#include <cuda_runtime.h>

#include "internal.h"

namespace tlq {

template <typename real> struct R2;
template <> struct R2<float> { using T = float2; };
template <> struct R2<double> { using T = double2; };

// Shared-memory placement of amplitude a: two padding slots after every 16 amplitudes,
// P(a) = a + 2*floor(a/16). A pass holds 16 amplitudes per thread on window bits
// [s, s+4). For s = 0 a thread's 16 amplitudes are contiguous (vector loads) and
// consecutive threads start 18 slots apart, so the 8 lanes of a 128-bit phase hit distinct
// banks; for s >= 4 the 16 lanes of a half-warp read consecutive slots. In both cases
// amplitude j of a thread sits at P(base) + j * stride, stride = 1 (s = 0) or
// 2^s + 2^(s-3) (s >= 4), so addressing costs one add per amplitude.
__host__ __device__ __forceinline__ int pad16(int a) { return a + ((a >> 4) << 1); }
__host__ __device__ __forceinline__ int padded_amps(int W) { return (1 << W) + (1 << (W - 3)); }
__host__ __device__ __forceinline__ int pass_stride(int s) { return s == 0 ? 1 : (1 << s) + (1 << (s - 3)); }

// ---- complex helpers ---------------------------------------------------------------------

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
    T2 r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}

template <typename T2>
__device__ __forceinline__ void load16(T2 (&v)[16], const T2* p, int stride) {
    if (stride == 1) {
        if constexpr (sizeof(T2) == 8) {
            const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 t = q[i];
                v[2 * i].x = t.x;
                v[2 * i].y = t.y;
                v[2 * i + 1].x = t.z;
                v[2 * i + 1].y = t.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = p[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = p[j * stride];
    }
}

template <typename T2>
__device__ __forceinline__ void store16(const T2 (&v)[16], T2* p, int stride) {
    if (stride == 1) {
        if constexpr (sizeof(T2) == 8) {
            float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
            for (int i = 0; i < 8; ++i) q[i] = make_float4(v[2 * i].x, v[2 * i].y, v[2 * i + 1].x, v[2 * i + 1].y);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) p[j] = v[j];
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) p[j * stride] = v[j];
    }
}

// The same loads and stores with the register bits' position s dispatched to a compile-time
// stride (s = 0 or 4..8, the positions a 2^12-amplitude tile has), so the 16 addresses are
// immediate offsets from one register; other s take the runtime form.
__host__ __device__ constexpr int stride_of(int s) { return s == 0 ? 1 : (1 << s) + (1 << (s - 3)); }

// Calls f(stride) with a literal stride for s = 0, 4..8 (each case inlines its own copy).
template <typename F>
__device__ __forceinline__ void with_stride(int s, F f) {
    switch (s) {
        case 0: f(stride_of(0)); break;
        case 4: f(stride_of(4)); break;
        case 5: f(stride_of(5)); break;
        case 6: f(stride_of(6)); break;
        case 7: f(stride_of(7)); break;
        case 8: f(stride_of(8)); break;
        default: f(stride_of(s)); break;
    }
}

template <typename T2>
__device__ __forceinline__ void load16s(T2 (&v)[16], const T2* p, int s) {
    with_stride(s, [&](int st) { load16(v, p, st); });
}

template <typename T2>
__device__ __forceinline__ void store16s(const T2 (&v)[16], T2* p, int s) {
    with_stride(s, [&](int st) { store16(v, p, st); });
}

// Warp sums of four values at once (a transposing reduction: 6 shuffles instead of 4 x 5).
// Lane l receives the sum over the warp of value (l >> 3) & 3.
template <typename real>
__device__ __forceinline__ real warp_sum4(real a0, real a1, real a2, real a3, int lane) {
    const bool u = (lane & 16) != 0;
    real k0 = u ? a2 : a0, k1 = u ? a3 : a1;   // kept: values 2u and 2u + 1
    const real s0 = u ? a0 : a2, s1 = u ? a1 : a3;
    k0 += __shfl_xor_sync(0xffffffffu, s0, 16);
    k1 += __shfl_xor_sync(0xffffffffu, s1, 16);
    const bool v = (lane & 8) != 0;
    real k = v ? k1 : k0;                      // value 2u + v
    k += __shfl_xor_sync(0xffffffffu, v ? k0 : k1, 8);
    k += __shfl_xor_sync(0xffffffffu, k, 4);
    k += __shfl_xor_sync(0xffffffffu, k, 2);
    k += __shfl_xor_sync(0xffffffffu, k, 1);
    return k;
}

// ---- packed two-wide FP32 (f32x2): one instruction updates the (re, im) pair of an
// amplitude. A real factor (RY's cos and sin, and the gradient sums of Y) acts on both parts
// alike, so these updates take half the instructions of the scalar form; the kernels that use
// them are bound by instruction issue, not by the FMA pipe.

__device__ __forceinline__ unsigned long long pk2(float x, float y) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(x), "f"(y));
    return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
    float2 v;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
    return v;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// ---- packed register state: each amplitude lives in one 64-bit register pair (re, im) from
// its load to its store, so the packed updates need no conversions between them.
using pk64 = unsigned long long;

__device__ __forceinline__ void load16p(pk64 (&v)[16], const float2* p, int stride) {
    if (stride == 1) {
        const ulonglong2* q = reinterpret_cast<const ulonglong2*>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const ulonglong2 t = q[i];
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    } else {
        const pk64* q = reinterpret_cast<const pk64*>(p);
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] = q[j * stride];
    }
}

__device__ __forceinline__ void store16p(const pk64 (&v)[16], float2* p, int stride) {
    if (stride == 1) {
        ulonglong2* q = reinterpret_cast<ulonglong2*>(p);
#pragma unroll
        for (int i = 0; i < 8; ++i) q[i] = make_ulonglong2(v[2 * i], v[2 * i + 1]);
    } else {
        pk64* q = reinterpret_cast<pk64*>(p);
#pragma unroll
        for (int j = 0; j < 16; ++j) q[j * stride] = v[j];
    }
}

__device__ __forceinline__ void load16ps(pk64 (&v)[16], const float2* p, int s) {
    with_stride(s, [&](int st) { load16p(v, p, st); });
}

__device__ __forceinline__ void store16ps(const pk64 (&v)[16], float2* p, int s) {
    with_stride(s, [&](int st) { store16p(v, p, st); });
}

// RY(a) on register bit K of a packed state; C = (c, c), S = (s, s), NS = (-s, -s).
template <int K>
__device__ __forceinline__ void apply_ry_p(pk64 (&v)[16], pk64 C, pk64 S, pk64 NS) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const pk64 a0 = v[j], a1 = v[j | (1 << K)];
        v[j] = fma2(C, a0, mul2(NS, a1));           // c a0 - s a1
        v[j | (1 << K)] = fma2(C, a1, mul2(S, a0));  // s a0 + c a1
    }
}

// RX(a) on register bit K of a packed state (scalar arithmetic on the unpacked pairs).
template <int K>
__device__ __forceinline__ void apply_rx_p(pk64 (&v)[16], float c, float s) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const float2 a0 = upk2(v[j]), a1 = upk2(v[j | (1 << K)]);
        v[j] = pk2(c * a0.x + s * a1.y, c * a0.y - s * a1.x);
        v[j | (1 << K)] = pk2(c * a1.x + s * a0.y, c * a1.y - s * a0.x);
    }
}

template <int K>
__device__ __forceinline__ void apply_rot_p(pk64 (&v)[16], int kind, float c, float s) {
    if (kind == TLQ_RY) apply_ry_p<K>(v, pk2(c, c), pk2(s, s), pk2(-s, -s));
    else apply_rx_p<K>(v, c, s);
}

// Im <lam| Y |psi> over the pairs of register bit K on packed states (see grad_y).
template <int K>
__device__ __forceinline__ float grad_y_p(const pk64 (&p)[16], const pk64 (&l)[16]) {
    pk64 sa = pk2(0.f, 0.f), sb = pk2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        sa = fma2(l[j | (1 << K)], p[j], sa);
        sb = fma2(l[j], p[j | (1 << K)], sb);
    }
    const float2 a = upk2(sa), b = upk2(sb);
    return (a.x + a.y) - (b.x + b.y);
}

// Im <lam| X |psi> over the pairs of register bit K on packed states (see grad_x).
template <int K>
__device__ __forceinline__ float grad_x_p(const pk64 (&p)[16], const pk64 (&l)[16]) {
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const float2 p0 = upk2(p[j]), p1 = upk2(p[j | (1 << K)]), l0 = upk2(l[j]), l1 = upk2(l[j | (1 << K)]);
        acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
    }
    return acc;
}

// Adjoint step of one rotation on register bit K of packed states: gradient, then un-apply
// (angle -> -angle: s_neg = -sin(a/2)) on psi and lam.
template <int K>
__device__ __forceinline__ float adjoint_rot_p(pk64 (&p)[16], pk64 (&l)[16], int kind, float c, float s_neg) {
    float g;
    if (kind == TLQ_RY) {
        g = grad_y_p<K>(p, l);
        const pk64 C = pk2(c, c), S = pk2(s_neg, s_neg), NS = pk2(-s_neg, -s_neg);
        apply_ry_p<K>(p, C, S, NS);
        apply_ry_p<K>(l, C, S, NS);
    } else {
        g = grad_x_p<K>(p, l);
        apply_rx_p<K>(p, c, s_neg);
        apply_rx_p<K>(l, c, s_neg);
    }
    return g;
}

// RY(a) on register bit K: [[c,-s],[s,c]] on (amp with bit 0, amp with bit 1). PACK selects
// the packed form for FP32 (callers whose register budget is tight keep the scalar form).
template <int K, typename T2, typename real, bool PACK = true>
__device__ __forceinline__ void apply_ry(T2 (&v)[16], real c, real s) {
    if constexpr (sizeof(real) == 4 && PACK) {
        const unsigned long long C = pk2(c, c), S = pk2(s, s), NS = pk2(-s, -s);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << K)) continue;
            const unsigned long long a0 = pk2(v[j].x, v[j].y), a1 = pk2(v[j | (1 << K)].x, v[j | (1 << K)].y);
            const float2 r0 = upk2(fma2(C, a0, mul2(NS, a1)));   // c a0 - s a1
            const float2 r1 = upk2(fma2(C, a1, mul2(S, a0)));    // s a0 + c a1
            v[j].x = r0.x;
            v[j].y = r0.y;
            v[j | (1 << K)].x = r1.x;
            v[j | (1 << K)].y = r1.y;
        }
    } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << K)) continue;
            const T2 a0 = v[j], a1 = v[j | (1 << K)];
            v[j].x = c * a0.x - s * a1.x;
            v[j].y = c * a0.y - s * a1.y;
            v[j | (1 << K)].x = s * a0.x + c * a1.x;
            v[j | (1 << K)].y = s * a0.y + c * a1.y;
        }
    }
}

// RX(a) on register bit K: [[c,-is],[-is,c]].
template <int K, typename T2, typename real>
__device__ __forceinline__ void apply_rx(T2 (&v)[16], real c, real s) {
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const T2 a0 = v[j], a1 = v[j | (1 << K)];
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

// Im <lam| Y |psi> over the pairs of register bit K (Y|0> = i|1>, Y|1> = -i|0>):
// sum over pairs of Re(conj(l1) p0) - Re(conj(l0) p1).
template <int K, typename T2, typename real, bool PACK = true>
__device__ __forceinline__ real grad_y(const T2 (&p)[16], const T2 (&l)[16]) {
    if constexpr (sizeof(real) == 4 && PACK) {
        // two packed sums: (l1 . p0) and (l0 . p1) componentwise, folded at the end
        unsigned long long sa = pk2(0.f, 0.f), sb = pk2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << K)) continue;
            const int j1 = j | (1 << K);
            sa = fma2(pk2(l[j1].x, l[j1].y), pk2(p[j].x, p[j].y), sa);
            sb = fma2(pk2(l[j].x, l[j].y), pk2(p[j1].x, p[j1].y), sb);
        }
        const float2 a = upk2(sa), b = upk2(sb);
        return (a.x + a.y) - (b.x + b.y);
    } else {
        real acc = 0;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            if (j & (1 << K)) continue;
            const T2 p0 = p[j], p1 = p[j | (1 << K)], l0 = l[j], l1 = l[j | (1 << K)];
            acc += (l1.x * p0.x + l1.y * p0.y) - (l0.x * p1.x + l0.y * p1.y);
        }
        return acc;
    }
}

// Im <lam| X |psi> = sum over pairs of Im(conj(l0) p1 + conj(l1) p0).
template <int K, typename T2, typename real>
__device__ __forceinline__ real grad_x(const T2 (&p)[16], const T2 (&l)[16]) {
    real acc = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        if (j & (1 << K)) continue;
        const T2 p0 = p[j], p1 = p[j | (1 << K)], l0 = l[j], l1 = l[j | (1 << K)];
        acc += (l0.x * p1.y - l0.y * p1.x) + (l1.x * p0.y - l1.y * p0.x);
    }
    return acc;
}

// Adjoint step of one rotation on register bit K: gradient, then un-apply on psi and lam.
template <int K, typename T2, typename real, bool PACK = true>
__device__ __forceinline__ real adjoint_rot(T2 (&p)[16], T2 (&l)[16], int kind, real c, real s_neg) {
    real g;
    if (kind == TLQ_RY) {
        g = grad_y<K, T2, real, PACK>(p, l);
        apply_ry<K, T2, real, PACK>(p, c, s_neg);
        apply_ry<K, T2, real, PACK>(l, c, s_neg);
    } else {
        g = grad_x<K, T2, real>(p, l);
        apply_rx<K>(p, c, s_neg);
        apply_rx<K>(l, c, s_neg);
    }
    return g;
}

}  // namespace tlq
