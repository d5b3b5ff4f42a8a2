// Energies of small circuits (n <= kTinyMaxQubits) for the latency-bound single call.
//
// <psi(theta)|H|psi(theta)> (Sec. 1 objective, Sec. 3) with the whole 2^n state of one
// parameter set in one CTA's shared memory: the gates are applied one at a time in circuit
// order (the plain definition of the circuit), then every Pauli term is measured and the terms
// are summed in FP64 in term order. At a few hundred amplitudes the cost of a call is launch
// latency and instruction fetch, not arithmetic: this one short kernel replaces the cone
// kernel (a large, fully unrolled kernel run by one 16-thread team at this size), the gate
// table and the reduction launches.
#include "internal.h"

#include <cuda_runtime.h>

namespace tlq {

namespace {

constexpr int kTinyThreads = 256;

// One CTA per parameter set (blockIdx.x). Dynamic shared memory: the state (2^n complex64),
// the gates' (cos a/2, sin a/2) and the per-warp partial sums of every term.
__global__ void __launch_bounds__(kTinyThreads) tiny_energy_kernel(const tlq_gate* __restrict__ gates, int n_gates,
                                                                   const double* __restrict__ theta, int n_params,
                                                                   int n, const DenseXTermDev* __restrict__ terms,
                                                                   int n_terms, double* __restrict__ energy) {
    extern __shared__ __align__(16) unsigned char tiny_smem[];
    const int N = 1 << n;
    float2* psi = reinterpret_cast<float2*>(tiny_smem);
    float2* cs = psi + N;                                        // [n_gates]
    float* part = reinterpret_cast<float*>(cs + n_gates);        // [n_terms][warps]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    constexpr int nw = kTinyThreads / 32;
    const double* th = theta + (size_t)blockIdx.x * n_params;

    for (int g = tid; g < n_gates; g += kTinyThreads) {
        const tlq_gate G = gates[g];
        const double a = G.param >= 0 ? th[G.param] : G.angle;
        double s, c;
        sincos(0.5 * a, &s, &c);
        cs[g] = make_float2((float)c, (float)s);
    }
    for (int x = tid; x < N; x += kTinyThreads) psi[x] = make_float2(x == 0 ? 1.f : 0.f, 0.f);
    __syncthreads();

    for (int g = 0; g < n_gates; ++g) {
        const tlq_gate G = gates[g];
        const float c = cs[g].x, s = cs[g].y;
        if (G.kind == TLQ_RX || G.kind == TLQ_RY) {
            // pairs (x0, x1 = x0 | 2^q): RY = [[c, -s], [s, c]], RX = [[c, -is], [-is, c]]
            const int q = G.q0;
            const int lowm = (1 << q) - 1;
            for (int i = tid; i < N / 2; i += kTinyThreads) {
                const int x0 = ((i & ~lowm) << 1) | (i & lowm), x1 = x0 | (1 << q);
                const float2 a0 = psi[x0], a1 = psi[x1];
                if (G.kind == TLQ_RY) {
                    psi[x0] = make_float2(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
                    psi[x1] = make_float2(s * a0.x + c * a1.x, s * a0.y + c * a1.y);
                } else {
                    psi[x0] = make_float2(c * a0.x + s * a1.y, c * a0.y - s * a1.x);
                    psi[x1] = make_float2(c * a1.x + s * a0.y, c * a1.y - s * a0.x);
                }
            }
        } else {
            // diagonal: RZ e^{-ia/2} / e^{+ia/2} by the bit; RZZ the same by the parity of the
            // two bits; CZ -1 where both bits are 1
            for (int x = tid; x < N; x += kTinyThreads) {
                const int b0 = (x >> G.q0) & 1;
                if (G.kind == TLQ_CZ) {
                    if (b0 & (x >> G.q1) & 1) psi[x] = make_float2(-psi[x].x, -psi[x].y);
                } else {
                    const int odd = G.kind == TLQ_RZ ? b0 : b0 ^ ((x >> G.q1) & 1);
                    const float2 v = psi[x];
                    const float ps = odd ? s : -s;
                    psi[x] = make_float2(c * v.x - ps * v.y, c * v.y + ps * v.x);
                }
            }
        }
        __syncthreads();
    }

    // <psi|P_t|psi> = sum_x Re(conj(psi_x) (-i)^ny (-1)^popc(x & zy) psi_{x ^ flip})
    for (int t = 0; t < n_terms; ++t) {
        const DenseXTermDev T = terms[t];
        const int ny = T.ny & 3;
        const float fx = ny == 0 ? 1.f : ny == 2 ? -1.f : 0.f, fy = ny == 1 ? -1.f : ny == 3 ? 1.f : 0.f;
        float acc = 0.f;
        for (int x = tid; x < N; x += kTinyThreads) {
            const float2 a = psi[x], v = psi[x ^ (int)T.flip];
            float re = fx * v.x - fy * v.y, im = fx * v.y + fy * v.x;
            if (__popc((unsigned)x & T.zy) & 1) { re = -re; im = -im; }
            acc += a.x * re + a.y * im;
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) part[t * nw + warp] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        // E = sum_t c_t e_t, compensated (Neumaier) in term order; e_t from the warps in order
        double sum = 0.0, comp = 0.0;
        for (int t = 0; t < n_terms; ++t) {
            float e = 0.f;
            for (int w = 0; w < nw; ++w) e += part[t * nw + w];
            const double x = terms[t].coeff * (double)e;
            const double y = sum + x;
            comp += fabs(sum) >= fabs(x) ? (sum - y) + x : (x - y) + sum;
            sum = y;
        }
        energy[blockIdx.x] = sum + comp;
    }
}

}  // namespace

size_t tiny_smem_bytes(int n, int n_gates, int n_terms) {
    return ((size_t)1 << n) * sizeof(float2) + (size_t)n_gates * sizeof(float2) +
           (size_t)n_terms * (kTinyThreads / 32) * sizeof(float);
}

bool tiny_fits(int n, int n_gates, int n_terms) {
    return n >= 1 && n <= kTinyMaxQubits && n_gates >= 0 && tiny_smem_bytes(n, n_gates, n_terms) <= 48 * 1024;
}

int launch_tiny_energy(const tlq_gate* gates, int n_gates, const double* theta, int n_params, int n,
                       const DenseXTermDev* terms, int n_terms, int B, double* energy, void* stream) {
    tiny_energy_kernel<<<B, kTinyThreads, tiny_smem_bytes(n, n_gates, n_terms), (cudaStream_t)stream>>>(
        gates, n_gates, theta, n_params, n, terms, n_terms, energy);
    return (int)cudaGetLastError();
}

}  // namespace tlq
