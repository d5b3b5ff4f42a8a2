// Exact matrix-product-state (tensor-train) route for chain circuits (TensorLy-Quantum Sec. 1 and
// Sec. 2: factorized, MPS / tensor-train representations of circuits and states; Sec. 3: the
// expectation value <H> of a transverse-field Ising Hamiltonian and its full gradient).
//
// Construction. A two-qubit gate on neighbours (q, q+1) is a sum of two products of single-site
// operators: CZ = |0><0| (x) I + |1><1| (x) Z and RZZ(g) = cos(g/2) I (x) I - i sin(g/2) Z (x) Z.
// The k-th such gate on a pair is bit k of the bond index between q and q+1, so a column
// (alpha, beta) of the site tensor A_q[s, alpha, beta] is the product of the site's operators in
// circuit order applied to |0>, the two-qubit gates contributing the factor selected by their bit
// (the left factor carries the coefficient). The state is psi[s_0..s_{n-1}] = prod_q A_q[s_q],
// exact, with bond dimension 2^(gates on the pair).
//
// Contraction. Bond k lies between sites k-1 and k. Left environments Ln[k] (sites < k, no
// operator) and LH[k] (sites < k with every term that ends before k inserted, each times its
// coefficient), right environments Rn[k] and RH[k] likewise, and for a term spanning sites
// i..j its partial chains OL_t[k], OR_t[k] on the bonds inside its span. A transfer through site q
// with Pauli P maps M to sum_s A_q[s]^dagger M (P A_q)[s]; the right sweep is the same map on the
// transposed site tensors. Then, per site, Gamma_q = dE / d conj(A_q) is a sum of
// Lx (P A_q) Rx^T over (LH, Rn), (Ln, RH) and every term covering q, the energy of a term is
// read where it ends, and the gradient of a gate on site q is 2 Re <dA_q, Gamma_q> through the
// site's operator product (forward products kept per column, then one backward pass).
//
// Kernels (one CTA per parameter set for the two sweeps, one per (set, site) otherwise):
//   mps_table_kernel   half-angle cos / sin per (set, gate)
//   mps_build_kernel   A_q for every (set, site)
//   mps_sweep_kernel   left and right sweeps (blockIdx.x & 1), sequential over sites
//   mps_site_kernel    term energies, Gamma_q and per-gate gradients per (set, site)
//   mps_reduce_kernel  E_b = sum_t c_t e_t and g_{b,p} = sum over the gates of p (FP64, fixed order)
// States and environments are FP32 (or FP64) complex; the sums of the last step are FP64.
#include "internal.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

namespace tlq {

constexpr int kMpsMaxCover = 32;     // terms covering one site
constexpr int kMpsThreads = 256;     // CTA size of every MPS kernel but the table and reduction

// One operator on a site, in circuit order.
enum MpsOpKind : int32_t {
    kOpRX = 0,
    kOpRY = 1,
    kOpRZ = 2,
    kOpLeftCZ = 3,    // |b><b| by bit `bit` of the right bond
    kOpLeftRZZ = 4,   // cos(g/2) I (bit 0) or -i sin(g/2) Z (bit 1), bit of the right bond
    kOpRightZ = 5,    // Z^b, bit of the left bond
};

struct MpsOp {
    int32_t kind;
    int32_t bit;
    int32_t gate;    // index into the gate list (angle table, gradient slot)
    int32_t param;   // parameter of the gate, -1 for a fixed angle or CZ
};

// Per-term data: span [lo, hi], coefficient, Pauli codes of sites lo..hi (0 I, 1 X, 2 Y, 3 Z) from
// pauli_off, and the element offsets of its chain matrices on bonds lo+1..hi from chain_off.
struct MpsTermDev {
    int32_t lo, hi;
    int32_t pauli_off;
    int32_t chain_idx;   // index of bond lo+1 in chain_boff
    double coeff;
};

// Output group of a sweep step or of the per-site kernel, and its contributions.
struct MpsGroup {
    int64_t dst;     // sweep: the matrix written; site kernel: Rx
    int32_t c0, nc;  // contributions [c0, c0 + nc)
    int32_t term;    // site kernel: the term whose energy the group yields, or -1
    int32_t pad;
};
struct MpsContrib {
    int64_t src;     // sweep: the input matrix; site kernel: Lx
    double coef;
    int32_t pauli;
    int32_t pad;
};

// Where the descriptors of one (kernel role, site) start: kinds 0/1 the left sweep without /
// with gradients, 2/3 the right sweep, 4/5 the per-site kernel; entry kind * n + q.
struct MpsDescIdx {
    int32_t g_off, ng, c_off, nc;
};

struct MpsPlan {
    int n = 0, n_gates = 0, n_params = 0, n_terms = 0;
    int max_bits = 0;
    int max_site_elems = 0;      // max over sites of chi_left * chi_right
    int max_site_ops = 0;        // max operators on one site
    int max_groups = 0;          // max output groups of one sweep step / one site
    int max_contribs = 0;        // max contributions (transfers) of one sweep step
    int64_t a_tot = 0, env_tot = 0, chain_tot = 0;   // complex elements per set
    std::vector<int32_t> bits;        // [n + 1] bond bits (bonds 0 and n: 0)
    std::vector<int64_t> a_off;       // [n] site tensor offsets
    std::vector<int64_t> env_off;     // [n + 1] bond offsets inside one environment array
    std::vector<int32_t> op_off;      // [n + 1]
    std::vector<MpsOp> ops;
    std::vector<int32_t> act_off;     // [n + 1] terms covering each site, in term order
    std::vector<int32_t> act;
    std::vector<MpsTermDev> terms;
    std::vector<uint8_t> pauli;
    std::vector<int64_t> chain_boff;  // element offset of each (term, bond) chain matrix
    std::vector<int32_t> pg_off;      // [n_params + 1] gates of each parameter, in gate order
    std::vector<int32_t> pg_idx;
    std::vector<tlq_gate> gates;
    std::vector<MpsDescIdx> dsc;      // [6 n] precomputed groups and contributions per site
    std::vector<MpsGroup> dgroups;
    std::vector<MpsContrib> dcontribs;
    // device copies
    int32_t* d_bits = nullptr;
    int64_t* d_a_off = nullptr;
    int64_t* d_env_off = nullptr;
    int32_t* d_op_off = nullptr;
    MpsOp* d_ops = nullptr;
    int32_t* d_act_off = nullptr;
    int32_t* d_act = nullptr;
    MpsTermDev* d_terms = nullptr;
    uint8_t* d_pauli = nullptr;
    int64_t* d_chain_boff = nullptr;
    int32_t* d_pg_off = nullptr;
    int32_t* d_pg_idx = nullptr;
    tlq_gate* d_gates = nullptr;
    MpsDescIdx* d_dsc = nullptr;
    MpsGroup* d_dgroups = nullptr;
    MpsContrib* d_dcontribs = nullptr;
    size_t device_bytes = 0;
    bool uploaded = false;
    ~MpsPlan();
};

MpsPlan::~MpsPlan() {
    cudaFree(d_bits);
    cudaFree(d_a_off);
    cudaFree(d_env_off);
    cudaFree(d_op_off);
    cudaFree(d_ops);
    cudaFree(d_act_off);
    cudaFree(d_act);
    cudaFree(d_terms);
    cudaFree(d_pauli);
    cudaFree(d_chain_boff);
    cudaFree(d_pg_off);
    cudaFree(d_pg_idx);
    cudaFree(d_gates);
    cudaFree(d_dsc);
    cudaFree(d_dgroups);
    cudaFree(d_dcontribs);
}

static void build_descriptors(MpsPlan& p);

std::shared_ptr<MpsPlan> make_mps_plan(const Circuit& c, const Ham& h, std::string* err) {
    auto p = std::make_shared<MpsPlan>();
    const int n = c.n;
    p->n = n;
    p->n_gates = (int)c.gates.size();
    p->n_params = c.n_params;
    p->n_terms = (int)h.terms.size();
    p->gates = c.gates;
    p->bits.assign(n + 1, 0);
    std::vector<std::vector<MpsOp>> site_ops(n);
    for (int g = 0; g < p->n_gates; ++g) {
        const tlq_gate& G = c.gates[g];
        if (G.kind == TLQ_RZZ || G.kind == TLQ_CZ) {
            const int lo = std::min(G.q0, G.q1), hi = std::max(G.q0, G.q1);
            if (hi != lo + 1) {
                *err = "MPS route: gate " + std::to_string(g) + " acts on non-neighbouring qubits";
                return nullptr;
            }
            const int bit = p->bits[hi]++;   // bond hi lies between sites lo and hi
            const int32_t param = G.kind == TLQ_RZZ ? G.param : -1;
            site_ops[lo].push_back({G.kind == TLQ_CZ ? kOpLeftCZ : kOpLeftRZZ, bit, g, param});
            site_ops[hi].push_back({kOpRightZ, bit, g, -1});
        } else {
            const int32_t k = G.kind == TLQ_RX ? kOpRX : G.kind == TLQ_RY ? kOpRY : kOpRZ;
            site_ops[G.q0].push_back({k, 0, g, G.param});
        }
    }
    p->op_off.assign(n + 1, 0);
    for (int q = 0; q < n; ++q) {
        if ((int)site_ops[q].size() > kMpsMaxSiteOps) {
            *err = "MPS route: more than " + std::to_string(kMpsMaxSiteOps) + " gates on qubit " + std::to_string(q);
            return nullptr;
        }
        p->op_off[q + 1] = p->op_off[q] + (int)site_ops[q].size();
        p->ops.insert(p->ops.end(), site_ops[q].begin(), site_ops[q].end());
    }
    for (int k = 0; k <= n; ++k) p->max_bits = std::max(p->max_bits, p->bits[k]);
    if (p->max_bits > kMpsMaxBondBitsF32) {
        *err = "MPS route: " + std::to_string(p->max_bits) + " two-qubit gates on one pair (bond dimension 2^" +
               std::to_string(p->max_bits) + ", at most 2^" + std::to_string(kMpsMaxBondBitsF32) + ")";
        return nullptr;
    }
    p->a_off.resize(n);
    int64_t acc = 0;
    for (int q = 0; q < n; ++q) {
        p->a_off[q] = acc;
        const int64_t e = (int64_t)1 << (p->bits[q] + p->bits[q + 1]);
        p->max_site_elems = std::max(p->max_site_elems, (int)e);
        acc += 2 * e;
    }
    p->a_tot = acc;
    p->env_off.resize(n + 1);
    acc = 0;
    for (int k = 0; k <= n; ++k) {
        p->env_off[k] = acc;
        acc += (int64_t)1 << (2 * p->bits[k]);
    }
    p->env_tot = acc;
    // terms: span, Pauli codes over the span, chain matrices on the bonds inside the span
    std::vector<std::vector<int32_t>> cover(n);
    acc = 0;
    for (int t = 0; t < p->n_terms; ++t) {
        const Term& T = h.terms[t];
        MpsTermDev d{};
        d.lo = *std::min_element(T.sites.begin(), T.sites.end());
        d.hi = *std::max_element(T.sites.begin(), T.sites.end());
        d.coeff = T.coeff;
        d.pauli_off = (int32_t)p->pauli.size();
        d.chain_idx = (int32_t)p->chain_boff.size();
        std::vector<uint8_t> code(d.hi - d.lo + 1, 0);
        for (size_t k = 0; k < T.sites.size(); ++k) {
            const char l = T.letters[k];
            code[T.sites[k] - d.lo] = l == 'X' ? 1 : l == 'Y' ? 2 : 3;
        }
        p->pauli.insert(p->pauli.end(), code.begin(), code.end());
        for (int k = d.lo + 1; k <= d.hi; ++k) {
            p->chain_boff.push_back(acc);
            acc += (int64_t)1 << (2 * p->bits[k]);
        }
        for (int q = d.lo; q <= d.hi; ++q) cover[q].push_back(t);
        p->terms.push_back(d);
    }
    p->chain_tot = acc;
    p->act_off.assign(n + 1, 0);
    int max_cover = 0;
    for (int q = 0; q < n; ++q) {
        p->act_off[q + 1] = p->act_off[q] + (int)cover[q].size();
        p->act.insert(p->act.end(), cover[q].begin(), cover[q].end());
        max_cover = std::max(max_cover, (int)cover[q].size());
    }
    if (max_cover > kMpsMaxCover) {
        *err = "MPS route: more than " + std::to_string(kMpsMaxCover) + " terms cover one qubit";
        return nullptr;
    }
    // a sweep step writes the norm environment, the H environment and one chain per covering
    // term that continues (contributions: one each, plus the terms folded into the H group); the
    // site kernel forms (LH, Rn), (Ln, RH) and one group per covering term
    p->max_groups = 2 + max_cover;
    p->max_contribs = 2 + max_cover;
    for (int q = 0; q < n; ++q) p->max_site_ops = std::max(p->max_site_ops, p->op_off[q + 1] - p->op_off[q]);
    // parameter -> gates (gradient reduction), in gate order
    p->pg_off.assign(p->n_params + 1, 0);
    for (const MpsOp& o : p->ops)
        if (o.param >= 0) p->pg_off[o.param + 1]++;
    for (int k = 0; k < p->n_params; ++k) p->pg_off[k + 1] += p->pg_off[k];
    p->pg_idx.assign(p->pg_off[p->n_params], 0);
    {
        std::vector<int32_t> fill(p->pg_off.begin(), p->pg_off.end() - 1);
        for (int g = 0; g < p->n_gates; ++g) {
            const tlq_gate& G = c.gates[g];
            if (G.kind != TLQ_CZ && G.param >= 0) p->pg_idx[fill[G.param]++] = g;
        }
    }
    build_descriptors(*p);
    return p;
}

template <typename V>
static int up(const std::vector<V>& v, V** out, size_t* bytes) {
    *out = nullptr;
    if (v.empty()) return 0;
    cudaError_t e = cudaMalloc((void**)out, v.size() * sizeof(V));
    if (e != cudaSuccess) return (int)e;
    *bytes += v.size() * sizeof(V);
    return (int)cudaMemcpy(*out, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice);
}

int mps_upload(MpsPlan& p) {
    if (p.uploaded) return 0;
    int rc = 0;
    size_t b = 0;
    if (!rc) rc = up(p.bits, &p.d_bits, &b);
    if (!rc) rc = up(p.a_off, &p.d_a_off, &b);
    if (!rc) rc = up(p.env_off, &p.d_env_off, &b);
    if (!rc) rc = up(p.op_off, &p.d_op_off, &b);
    if (!rc) rc = up(p.ops, &p.d_ops, &b);
    if (!rc) rc = up(p.act_off, &p.d_act_off, &b);
    if (!rc) rc = up(p.act, &p.d_act, &b);
    if (!rc) rc = up(p.terms, &p.d_terms, &b);
    if (!rc) rc = up(p.pauli, &p.d_pauli, &b);
    if (!rc) rc = up(p.chain_boff, &p.d_chain_boff, &b);
    if (!rc) rc = up(p.pg_off, &p.d_pg_off, &b);
    if (!rc) rc = up(p.pg_idx, &p.d_pg_idx, &b);
    if (!rc) rc = up(p.gates, &p.d_gates, &b);
    if (!rc) rc = up(p.dsc, &p.d_dsc, &b);
    if (!rc) rc = up(p.dgroups, &p.d_dgroups, &b);
    if (!rc) rc = up(p.dcontribs, &p.d_dcontribs, &b);
    p.device_bytes = b;
    p.uploaded = rc == 0;
    return rc;
}

void mps_info(const MpsPlan& p, int* max_bond_bits, int64_t* elems_per_set, size_t* device_bytes) {
    if (max_bond_bits) *max_bond_bits = p.max_bits;
    if (elems_per_set) *elems_per_set = p.a_tot + 4 * p.env_tot + 2 * p.chain_tot;
    if (device_bytes) *device_bytes = p.device_bytes;
}

// Contraction flops per parameter set (8 per complex multiply-add) of the sweeps and the
// per-site kernel, counted with the groups those kernels form: a transfer through a site with
// input dimension din and output dout costs 2 din dout din (M (P A)[s]) per contribution plus
// 2 dout dout din (sum_s A[s]^dagger Y[s]) per output; a site group costs 2 dl dr (dl + dr).
double mps_flops(const MpsPlan& p, bool grad) {
    double cmac = 0;
    for (int q = 0; q < p.n; ++q) {
        const double dl = (double)(1 << p.bits[q]), dr = (double)(1 << p.bits[q + 1]);
        int ends_l = 0, cont_l = 0, ends_r = 0, cont_r = 0, end_here = 0, cover = 0;
        for (int k = p.act_off[q]; k < p.act_off[q + 1]; ++k) {
            const MpsTermDev& t = p.terms[p.act[k]];
            ++cover;
            if (t.hi == q) ++ends_l, ++end_here;
            else ++cont_l;
            if (t.lo == q) ++ends_r;
            else ++cont_r;
        }
        // left sweep: din = dl, dout = dr; right sweep: din = dr, dout = dl
        const int ncl = 1 + (grad ? 1 + ends_l : 0) + cont_l, ngl = 1 + (grad ? 1 : 0) + cont_l;
        const int ncr = 1 + (grad ? 1 + ends_r + cont_r : 0), ngr = 1 + (grad ? 1 + cont_r : 0);
        cmac += ncl * 2 * dl * dr * dl + ngl * 2 * dr * dr * dl;
        cmac += ncr * 2 * dr * dl * dr + ngr * 2 * dl * dl * dr;
        const int ngs = grad ? 2 + cover : end_here;
        cmac += ngs * 2 * dl * dr * (dl + dr);
    }
    return 8.0 * cmac;
}

// ---- device side -------------------------------------------------------------------------
// The kernel bodies are host-and-device templates over the barrier, so that the same code is
// what every CTA runs; the kernels below instantiate them with __syncthreads.

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

template <typename V> __host__ __device__ __forceinline__ V cx(decltype(V::x) re, decltype(V::x) im) {
    V r;
    r.x = re;
    r.y = im;
    return r;
}
// acc + a * b
template <typename V> __host__ __device__ __forceinline__ V cfma(V a, V b, V acc) {
    acc.x += a.x * b.x - a.y * b.y;
    acc.y += a.x * b.y + a.y * b.x;
    return acc;
}
// acc + conj(a) * b
template <typename V> __host__ __device__ __forceinline__ V cfma_cj(V a, V b, V acc) {
    acc.x += a.x * b.x + a.y * b.y;
    acc.y += a.x * b.y - a.y * b.x;
    return acc;
}
template <typename V> __host__ __device__ __forceinline__ V cmul(V a, V b) {
    return cx<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// (P A)[s] = f * A[s']: I (s, 1), X (1 - s, 1), Y (1 - s, -i for s = 0, +i for s = 1), Z (s, (-1)^s)
template <typename V> __host__ __device__ __forceinline__ void pauli_row(int P, int s, int* sp, V* f) {
    *sp = (P == 1 || P == 2) ? 1 - s : s;
    if (P == 2) *f = cx<V>(0, s ? 1 : -1);
    else if (P == 3 && s) *f = cx<V>(-1, 0);
    else *f = cx<V>(1, 0);
}

// v <- M v for one site operator of column (al, be); (c, s) = cos, sin of the gate's half angle.
template <typename V, typename T>
__host__ __device__ __forceinline__ void op_apply(const MpsOp& o, T c, T s, int al, int be, V& a0, V& a1) {
    switch (o.kind) {
        case kOpRX: {   // [[c, -is], [-is, c]]
            const V n0 = cx<V>(c * a0.x + s * a1.y, c * a0.y - s * a1.x);
            const V n1 = cx<V>(c * a1.x + s * a0.y, c * a1.y - s * a0.x);
            a0 = n0;
            a1 = n1;
            break;
        }
        case kOpRY: {   // [[c, -s], [s, c]]
            const V n0 = cx<V>(c * a0.x - s * a1.x, c * a0.y - s * a1.y);
            const V n1 = cx<V>(s * a0.x + c * a1.x, s * a0.y + c * a1.y);
            a0 = n0;
            a1 = n1;
            break;
        }
        case kOpRZ:     // diag(c - is, c + is)
            a0 = cx<V>(c * a0.x + s * a0.y, c * a0.y - s * a0.x);
            a1 = cx<V>(c * a1.x - s * a1.y, c * a1.y + s * a1.x);
            break;
        case kOpLeftCZ:
            if ((be >> o.bit) & 1) a0 = cx<V>(0, 0);
            else a1 = cx<V>(0, 0);
            break;
        case kOpLeftRZZ:
            if ((be >> o.bit) & 1) {   // -is Z
                a0 = cx<V>(s * a0.y, -s * a0.x);
                a1 = cx<V>(-s * a1.y, s * a1.x);
            } else {
                a0 = cx<V>(c * a0.x, c * a0.y);
                a1 = cx<V>(c * a1.x, c * a1.y);
            }
            break;
        default:        // kOpRightZ
            if ((al >> o.bit) & 1) a1 = cx<V>(-a1.x, -a1.y);
            break;
    }
}

// w <- M^dagger w
template <typename V, typename T>
__host__ __device__ __forceinline__ void op_adjoint(const MpsOp& o, T c, T s, int al, int be, V& w0, V& w1) {
    switch (o.kind) {
        case kOpRX: {   // [[c, is], [is, c]]
            const V n0 = cx<V>(c * w0.x - s * w1.y, c * w0.y + s * w1.x);
            const V n1 = cx<V>(c * w1.x - s * w0.y, c * w1.y + s * w0.x);
            w0 = n0;
            w1 = n1;
            break;
        }
        case kOpRY: {   // [[c, s], [-s, c]]
            const V n0 = cx<V>(c * w0.x + s * w1.x, c * w0.y + s * w1.y);
            const V n1 = cx<V>(c * w1.x - s * w0.x, c * w1.y - s * w0.y);
            w0 = n0;
            w1 = n1;
            break;
        }
        case kOpRZ:     // diag(c + is, c - is)
            w0 = cx<V>(c * w0.x - s * w0.y, c * w0.y + s * w0.x);
            w1 = cx<V>(c * w1.x + s * w1.y, c * w1.y - s * w1.x);
            break;
        case kOpLeftRZZ:
            if ((be >> o.bit) & 1) {   // +is Z
                w0 = cx<V>(-s * w0.y, s * w0.x);
                w1 = cx<V>(s * w1.y, -s * w1.x);
            } else {
                w0 = cx<V>(c * w0.x, c * w0.y);
                w1 = cx<V>(c * w1.x, c * w1.y);
            }
            break;
        default:        // the projector and Z^b are Hermitian
            op_apply(o, c, s, al, be, w0, w1);
            break;
    }
}

// 2 Re <dM v, w> for the operator's angle: rotations dM = (-i/2) G M (u = M v, the vector after
// the operator), the RZZ left factor d(c)/da = -s/2 (bit 0), d(-is)/da = -ic/2 (bit 1) on v.
template <typename V, typename T>
__host__ __device__ __forceinline__ T op_grad(const MpsOp& o, T c, T s, int be, V v0, V v1, V u0, V u1, V w0,
                                              V w1) {
    V d0, d1;
    switch (o.kind) {
        case kOpRX:   // (-i/2) X u
            d0 = cx<V>(T(0.5) * u1.y, -T(0.5) * u1.x);
            d1 = cx<V>(T(0.5) * u0.y, -T(0.5) * u0.x);
            break;
        case kOpRY:   // (-i/2) Y u = (-u1 / 2, u0 / 2)
            d0 = cx<V>(-T(0.5) * u1.x, -T(0.5) * u1.y);
            d1 = cx<V>(T(0.5) * u0.x, T(0.5) * u0.y);
            break;
        case kOpRZ:   // (-i/2) Z u
            d0 = cx<V>(T(0.5) * u0.y, -T(0.5) * u0.x);
            d1 = cx<V>(-T(0.5) * u1.y, T(0.5) * u1.x);
            break;
        default:      // kOpLeftRZZ
            if ((be >> o.bit) & 1) {   // (-ic/2) Z v
                d0 = cx<V>(T(0.5) * c * v0.y, -T(0.5) * c * v0.x);
                d1 = cx<V>(-T(0.5) * c * v1.y, T(0.5) * c * v1.x);
            } else {
                d0 = cx<V>(-T(0.5) * s * v0.x, -T(0.5) * s * v0.y);
                d1 = cx<V>(-T(0.5) * s * v1.x, -T(0.5) * s * v1.y);
            }
            break;
    }
    return T(2) * (d0.x * w0.x + d0.y * w0.y + d1.x * w1.x + d1.y * w1.y);
}

template <typename T>
struct MpsArgs {
    using V = typename Cx<T>::t;
    int n, B, n_gates, n_params, n_terms, grad;
    const int32_t* bits;
    const int64_t* a_off;
    const int64_t* env_off;
    const int32_t* op_off;
    const MpsOp* ops;
    const int32_t* act_off;
    const int32_t* act;
    const MpsTermDev* terms;
    const uint8_t* pauli;
    const int64_t* chain_boff;
    const MpsDescIdx* dsc;
    const MpsGroup* dgroups;
    const MpsContrib* dcontribs;
    int64_t a_tot, env_tot, chain_tot, stride;
    int max_elems, max_groups, max_ops;
    int ygroups_sweep, ygroups_site;
    V* work;                 // B blocks of `stride` elements
    const double2* tab;      // [B][n_gates] (cos, sin) of the half angles
    double* e;               // [B][n_terms] <P_t>
    double* gslot;           // [B][n_gates] gradient of each parametrised gate
};

// Bytes of the per-site kernel's shared region: Z buffers and energy partials, or the gradient
// partials, whichever is larger (16-byte multiple).
template <typename T>
__host__ __device__ inline size_t site_region_bytes(int ygroups, int max_elems, int max_ops, int nt) {
    const size_t zb = (size_t)ygroups * 2 * max_elems * sizeof(typename Cx<T>::t) + (size_t)ygroups * nt * sizeof(double);
    const size_t gb = (size_t)max_ops * nt * sizeof(T);
    const size_t r = zb > gb ? zb : gb;
    return (r + 15) & ~(size_t)15;
}

// Groups of the sweep step through site q (dir 0: left to right, 1: right to left); returns the
// group count. Norm environment first, then (with gradients) the H environment with the terms
// that end here folded in, then one chain per covering term that continues.
template <typename T>
__host__ __device__ int sweep_desc(const MpsArgs<T>& a, int q, int dir, MpsGroup* G, MpsContrib* C) {
    const int64_t E0 = a.a_tot + (dir ? 2 : 0) * a.env_tot;
    const int64_t EH = E0 + a.env_tot;
    const int64_t CH = a.a_tot + 4 * a.env_tot + (dir ? a.chain_tot : 0);
    const int kin = dir ? q + 1 : q, kout = dir ? q : q + 1;
    int ng = 0, nc = 0;
    G[ng] = MpsGroup{E0 + a.env_off[kout], nc, 1, -1, 0};
    C[nc++] = MpsContrib{E0 + a.env_off[kin], 1.0, 0, 0};
    ++ng;
    if (a.grad) {
        G[ng] = MpsGroup{EH + a.env_off[kout], nc, 0, -1, 0};
        C[nc++] = MpsContrib{EH + a.env_off[kin], 1.0, 0, 0};
        for (int k = a.act_off[q]; k < a.act_off[q + 1]; ++k) {
            const MpsTermDev& t = a.terms[a.act[k]];
            if ((dir ? t.lo : t.hi) != q) continue;
            const bool starts = (dir ? t.hi : t.lo) == q;
            const int64_t src = starts ? E0 + a.env_off[kin] : CH + a.chain_boff[t.chain_idx + kin - t.lo - 1];
            C[nc++] = MpsContrib{src, t.coeff, a.pauli[t.pauli_off + q - t.lo], 0};
        }
        G[ng].nc = nc - G[ng].c0;
        ++ng;
    }
    if (dir == 0 || a.grad) {
        for (int k = a.act_off[q]; k < a.act_off[q + 1]; ++k) {
            const MpsTermDev& t = a.terms[a.act[k]];
            if ((dir ? t.lo : t.hi) == q) continue;
            const bool starts = (dir ? t.hi : t.lo) == q;
            const int64_t src = starts ? E0 + a.env_off[kin] : CH + a.chain_boff[t.chain_idx + kin - t.lo - 1];
            G[ng++] = MpsGroup{CH + a.chain_boff[t.chain_idx + kout - t.lo - 1], nc, 1, -1, 0};
            C[nc++] = MpsContrib{src, 1.0, a.pauli[t.pauli_off + q - t.lo], 0};
        }
    }
    return ng;
}

// Groups of the per-site kernel at site q: (LH, Rn) and (Ln, RH) with gradients, then every
// covering term (Lx its left chain or Ln, Rx its right chain or Rn); without gradients only the
// terms that end at q. One contribution each.
template <typename T>
__host__ __device__ int site_desc(const MpsArgs<T>& a, int q, MpsGroup* G, MpsContrib* C) {
    const int64_t Ln = a.a_tot, LH = Ln + a.env_tot, Rn = LH + a.env_tot, RH = Rn + a.env_tot;
    const int64_t OL = a.a_tot + 4 * a.env_tot, OR = OL + a.chain_tot;
    int ng = 0;
    if (a.grad) {
        G[ng] = MpsGroup{Rn + a.env_off[q + 1], ng, 1, -1, 0};
        C[ng] = MpsContrib{LH + a.env_off[q], 1.0, 0, 0};
        ++ng;
        G[ng] = MpsGroup{RH + a.env_off[q + 1], ng, 1, -1, 0};
        C[ng] = MpsContrib{Ln + a.env_off[q], 1.0, 0, 0};
        ++ng;
    }
    for (int k = a.act_off[q]; k < a.act_off[q + 1]; ++k) {
        const int ti = a.act[k];
        const MpsTermDev& t = a.terms[ti];
        if (!a.grad && t.hi != q) continue;
        const int64_t lx = t.lo == q ? Ln + a.env_off[q] : OL + a.chain_boff[t.chain_idx + q - t.lo - 1];
        const int64_t rx = t.hi == q ? Rn + a.env_off[q + 1] : OR + a.chain_boff[t.chain_idx + q - t.lo];
        G[ng] = MpsGroup{rx, ng, 1, t.hi == q ? ti : -1, 0};
        C[ng] = MpsContrib{lx, t.coeff, a.pauli[t.pauli_off + q - t.lo], 0};
        ++ng;
    }
    return ng;
}

// Precomputes every (role, site) descriptor list with the functions above on the plan's host
// tables; the kernels copy a site's list into shared memory with one load per entry.
static void build_descriptors(MpsPlan& p) {
    MpsArgs<float> a{};
    a.n = p.n;
    a.bits = p.bits.data();
    a.a_off = p.a_off.data();
    a.env_off = p.env_off.data();
    a.act_off = p.act_off.data();
    a.act = p.act.data();
    a.terms = p.terms.data();
    a.pauli = p.pauli.data();
    a.chain_boff = p.chain_boff.data();
    a.a_tot = p.a_tot;
    a.env_tot = p.env_tot;
    a.chain_tot = p.chain_tot;
    std::vector<MpsGroup> G(p.max_groups);
    std::vector<MpsContrib> C(p.max_contribs);
    p.dsc.assign((size_t)6 * p.n, MpsDescIdx{0, 0, 0, 0});
    for (int kind = 0; kind < 6; ++kind) {
        a.grad = kind & 1;
        for (int q = 0; q < p.n; ++q) {
            int ng;
            if (kind < 4) {
                ng = sweep_desc(a, q, kind >> 1, G.data(), C.data());
            } else {
                ng = site_desc(a, q, G.data(), C.data());
            }
            int nc = 0;
            for (int g = 0; g < ng; ++g) nc = std::max(nc, G[g].c0 + G[g].nc);
            p.dsc[(size_t)kind * p.n + q] = MpsDescIdx{(int32_t)p.dgroups.size(), ng, (int32_t)p.dcontribs.size(), nc};
            p.dgroups.insert(p.dgroups.end(), G.begin(), G.begin() + ng);
            p.dcontribs.insert(p.dcontribs.end(), C.begin(), C.begin() + nc);
        }
    }
}

// Shared-memory layout of the per-site kernel (bytes from the start): Aw, Gam, the Z / partials
// region, gacc (even count of doubles), the site's (cos, sin) table and operators, groups,
// contributions.
template <typename T>
__host__ __device__ inline void site_smem_offsets(int max_elems, int ygroups, int max_ops, int max_groups, int nt,
                                                  size_t off[7]) {
    const size_t el = (size_t)2 * max_elems * sizeof(typename Cx<T>::t);
    off[0] = 2 * el;                                                        // region
    off[1] = off[0] + site_region_bytes<T>(ygroups, max_elems, max_ops, nt); // gacc
    off[2] = off[1] + (size_t)((max_ops + 1) & ~1) * sizeof(double);        // cos / sin
    off[3] = off[2] + (size_t)max_ops * sizeof(double2);                    // operators
    off[4] = off[3] + (size_t)max_ops * sizeof(MpsOp);                      // groups
    off[5] = off[4] + (size_t)max_groups * sizeof(MpsGroup);                // contributions
    off[6] = off[5] + (size_t)max_groups * sizeof(MpsContrib);              // end
}

// Stages the operators of site q and their (cos, sin) into shared memory.
template <typename T>
__host__ __device__ inline void stage_ops(const MpsArgs<T>& a, int q, int b, MpsOp* sop, double2* scs, int tid,
                                          int nt) {
    const int o0 = a.op_off[q], m = a.op_off[q + 1] - o0;
    const double2* tab = a.tab + (int64_t)b * a.n_gates;
    for (int k = tid; k < m; k += nt) {
        const MpsOp o = a.ops[o0 + k];
        sop[k] = o;
        scs[k] = tab[o.gate];
    }
}

// Site tensors: block (set b, site q); each thread builds columns (al, be) of A_q from the
// site's operators staged in shared memory (smem: [max_ops] (cos, sin), [max_ops] operators).
#pragma nv_exec_check_disable
template <typename T, typename Sync>
__host__ __device__ void build_body(const MpsArgs<T>& a, int bid, int tid, int nt, unsigned char* smem, Sync sync) {
    using V = typename Cx<T>::t;
    const int q = bid % a.n, b = bid / a.n;
    const int dl = 1 << a.bits[q], dr = 1 << a.bits[q + 1];
    const int m = a.op_off[q + 1] - a.op_off[q];
    double2* scs = reinterpret_cast<double2*>(smem);
    MpsOp* sop = reinterpret_cast<MpsOp*>(scs + a.max_ops);
    stage_ops(a, q, b, sop, scs, tid, nt);
    sync();
    V* A = a.work + (int64_t)b * a.stride + a.a_off[q];
    for (int col = tid; col < dl * dr; col += nt) {
        const int al = col / dr, be = col - al * dr;
        V v0 = cx<V>(1, 0), v1 = cx<V>(0, 0);
        for (int k = 0; k < m; ++k) op_apply(sop[k], (T)scs[k].x, (T)scs[k].y, al, be, v0, v1);
        A[col] = v0;
        A[dl * dr + col] = v1;
    }
}

// Stages A_q into shared memory as Aw[s][in][out]: natural order (in = left bond) for dir 0,
// transposed (in = right bond) for dir 1.
template <typename T>
__host__ __device__ void stage_site(const MpsArgs<T>& a, const typename Cx<T>::t* base, int q, int dir,
                                    typename Cx<T>::t* Aw, int tid, int nt) {
    const int dl = 1 << a.bits[q], dr = 1 << a.bits[q + 1];
    const typename Cx<T>::t* A = base + a.a_off[q];
    for (int idx = tid; idx < 2 * dl * dr; idx += nt) {
        if (!dir) {
            Aw[idx] = A[idx];
        } else {
            const int s = idx / (dl * dr), r = idx - s * dl * dr, al = r / dr, be = r - al * dr;
            Aw[s * dl * dr + be * dl + al] = A[idx];
        }
    }
}

// Both sweeps: block 2b + dir. Shared memory: Aw [2 max_elems], Y [ygroups][2 max_elems], groups,
// contributions. Per site: Y_g[s] = sum_c coef_c f_c(s) M_c Aw[s'_c(s)] (in x out), then
// out_g = sum_s Aw[s]^dagger Y_g[s] (out x out), written to the group's matrix.
#pragma nv_exec_check_disable
template <typename T, typename Sync>
__host__ __device__ void sweep_body(const MpsArgs<T>& a, int bid, int tid, int nt, unsigned char* smem, Sync sync) {
    using V = typename Cx<T>::t;
    const int dir = bid & 1, b = bid >> 1;
    V* base = a.work + (int64_t)b * a.stride;
    V* Aw = reinterpret_cast<V*>(smem);
    V* Y = Aw + 2 * a.max_elems;
    MpsGroup* G = reinterpret_cast<MpsGroup*>(Y + (size_t)a.ygroups_sweep * 2 * a.max_elems);
    MpsContrib* C = reinterpret_cast<MpsContrib*>(G + a.max_groups);
    if (tid == 0) {
        const int kb = dir ? a.n : 0;
        const int64_t E0 = a.a_tot + (dir ? 2 : 0) * a.env_tot;
        base[E0 + a.env_off[kb]] = cx<V>(1, 0);
        if (a.grad) base[E0 + a.env_tot + a.env_off[kb]] = cx<V>(0, 0);
    }
    for (int step = 0; step < a.n; ++step) {
        const int q = dir ? a.n - 1 - step : step;
        const MpsDescIdx d = a.dsc[(size_t)(dir * 2 + a.grad) * a.n + q];
        for (int i = tid; i < d.ng; i += nt) G[i] = a.dgroups[d.g_off + i];
        for (int i = tid; i < d.nc; i += nt) C[i] = a.dcontribs[d.c_off + i];
        stage_site(a, base, q, dir, Aw, tid, nt);
        sync();
        const int ng = d.ng;
        const int din = 1 << a.bits[dir ? q + 1 : q], dout = 1 << a.bits[dir ? q : q + 1];
        const int ys = 2 * din * dout;
        for (int g0 = 0; g0 < ng; g0 += a.ygroups_sweep) {
            const int nb = ng - g0 < a.ygroups_sweep ? ng - g0 : a.ygroups_sweep;
            for (int idx = tid; idx < nb * ys; idx += nt) {
                const int gi = idx / ys, r = idx - gi * ys;
                const int s = r / (din * dout), r2 = r - s * din * dout, i = r2 / dout, o = r2 - i * dout;
                const MpsGroup g = G[g0 + gi];
                V acc = cx<V>(0, 0);
                for (int c = g.c0; c < g.c0 + g.nc; ++c) {
                    const MpsContrib cc = C[c];
                    int sp;
                    V f;
                    pauli_row(cc.pauli, s, &sp, &f);
                    const V* M = base + cc.src + (int64_t)i * din;
                    const V* Ac = Aw + sp * din * dout + o;
                    V d = cx<V>(0, 0);
                    for (int ip = 0; ip < din; ++ip) d = cfma(M[ip], Ac[ip * dout], d);
                    const V w = cx<V>((T)cc.coef * f.x, (T)cc.coef * f.y);
                    acc = cfma(w, d, acc);
                }
                Y[gi * ys + r] = acc;
            }
            sync();
            for (int idx = tid; idx < nb * dout * dout; idx += nt) {
                const int gi = idx / (dout * dout), r = idx - gi * dout * dout, o = r / dout, o2 = r - o * dout;
                const V* Yg = Y + gi * ys;
                V acc = cx<V>(0, 0);
                for (int s = 0; s < 2; ++s)
                    for (int i = 0; i < din; ++i)
                        acc = cfma_cj(Aw[s * din * dout + i * dout + o], Yg[s * din * dout + i * dout + o2], acc);
                base[G[g0 + gi].dst + r] = acc;
            }
            sync();
        }
    }
}

// Per (set, site): term energies where terms end, Gamma_q and the site's gate gradients.
// Shared memory: Aw [2 max_elems], Gam [2 max_elems], then a region holding either the Z
// buffers [ygroups][2 max_elems] with the energy partials [ygroups][nt] (doubles), or the
// gradient partials [max_ops][nt]; then gacc [max_ops] (doubles), groups, contributions.
#pragma nv_exec_check_disable
template <typename T, typename Sync>
__host__ __device__ void site_body(const MpsArgs<T>& a, int bid, int tid, int nt, unsigned char* smem, Sync sync) {
    using V = typename Cx<T>::t;
    const int q = bid % a.n, b = bid / a.n;
    const int dl = 1 << a.bits[q], dr = 1 << a.bits[q + 1], ne = dl * dr, ys = 2 * ne;
    V* base = a.work + (int64_t)b * a.stride;
    V* Aw = reinterpret_cast<V*>(smem);
    V* Gam = Aw + 2 * a.max_elems;
    size_t off[7];
    site_smem_offsets<T>(a.max_elems, a.ygroups_site, a.max_ops, a.max_groups, nt, off);
    unsigned char* region = smem + off[0];
    V* Z = reinterpret_cast<V*>(region);
    double* red = reinterpret_cast<double*>(Z + (size_t)a.ygroups_site * 2 * a.max_elems);
    T* cg = reinterpret_cast<T*>(region);
    double* gacc = reinterpret_cast<double*>(smem + off[1]);
    double2* scs = reinterpret_cast<double2*>(smem + off[2]);
    MpsOp* sop = reinterpret_cast<MpsOp*>(smem + off[3]);
    MpsGroup* G = reinterpret_cast<MpsGroup*>(smem + off[4]);
    MpsContrib* C = reinterpret_cast<MpsContrib*>(smem + off[5]);
    const int m = a.op_off[q + 1] - a.op_off[q];
    const MpsDescIdx d = a.dsc[(size_t)(4 + a.grad) * a.n + q];
    for (int i = tid; i < d.ng; i += nt) G[i] = a.dgroups[d.g_off + i];
    for (int i = tid; i < d.nc; i += nt) C[i] = a.dcontribs[d.c_off + i];
    if (a.grad) stage_ops(a, q, b, sop, scs, tid, nt);
    stage_site(a, base, q, 0, Aw, tid, nt);
    if (a.grad)
        for (int idx = tid; idx < ys; idx += nt) Gam[idx] = cx<V>(0, 0);
    for (int k = tid; k < m; k += nt) gacc[k] = 0.0;
    sync();
    const int ng = d.ng;
    for (int g0 = 0; g0 < ng; g0 += a.ygroups_site) {
        const int nb = ng - g0 < a.ygroups_site ? ng - g0 : a.ygroups_site;
        // Z_g[s] = f(s) Lx Aw[s']   (dl x dr)
        for (int idx = tid; idx < nb * ys; idx += nt) {
            const int gi = idx / ys, r = idx - gi * ys;
            const int s = r / ne, r2 = r - s * ne, al = r2 / dr, be = r2 - al * dr;
            const MpsContrib cc = C[G[g0 + gi].c0];
            int sp;
            V f;
            pauli_row(cc.pauli, s, &sp, &f);
            const V* Lx = base + cc.src + (int64_t)al * dl;
            const V* Ac = Aw + sp * ne + be;
            V d = cx<V>(0, 0);
            for (int ap = 0; ap < dl; ++ap) d = cfma(Lx[ap], Ac[ap * dr], d);
            Z[gi * ys + r] = cmul(f, d);
        }
        sync();
        // prod = Z_g[s] Rx^T; Gam += coef prod; energy partials Re(conj(A) prod)
        bool any_e = false;
        for (int gi = 0; gi < nb; ++gi) {
            const MpsGroup g = G[g0 + gi];
            const V* Rx = base + g.dst;
            const T coef = (T)C[g.c0].coef;
            double ep = 0.0;
            for (int idx = tid; idx < ys; idx += nt) {
                const int s = idx / ne, r2 = idx - s * ne, al = r2 / dr, be = r2 - al * dr;
                const V* Zr = Z + gi * ys + s * ne + al * dr;
                const V* Rr = Rx + (int64_t)be * dr;
                V prod = cx<V>(0, 0);
                for (int bp = 0; bp < dr; ++bp) prod = cfma(Zr[bp], Rr[bp], prod);
                if (a.grad) {
                    Gam[idx].x += coef * prod.x;
                    Gam[idx].y += coef * prod.y;
                }
                if (g.term >= 0) ep += (double)(Aw[idx].x * prod.x + Aw[idx].y * prod.y);
            }
            if (g.term >= 0) {
                red[gi * nt + tid] = ep;
                any_e = true;
            }
        }
        sync();
        if (any_e) {
            for (int stride = nt / 2; stride > 0; stride >>= 1) {
                if (tid < stride)
                    for (int gi = 0; gi < nb; ++gi)
                        if (G[g0 + gi].term >= 0) red[gi * nt + tid] += red[gi * nt + tid + stride];
                sync();
            }
            if (tid == 0)
                for (int gi = 0; gi < nb; ++gi)
                    if (G[g0 + gi].term >= 0) a.e[(int64_t)b * a.n_terms + G[g0 + gi].term] = red[gi * nt];
            sync();
        }
    }
    if (!a.grad) return;
    // gradients: per column, forward products kept, then the backward pass from Gamma
    for (int r0 = 0; r0 < ne; r0 += nt) {
        const int col = r0 + tid;
        if (col < ne) {
            const int al = col / dr, be = col - al * dr;
            V f0[kMpsMaxSiteOps + 1], f1[kMpsMaxSiteOps + 1];
            f0[0] = cx<V>(1, 0);
            f1[0] = cx<V>(0, 0);
            for (int k = 0; k < m; ++k) {
                V v0 = f0[k], v1 = f1[k];
                op_apply(sop[k], (T)scs[k].x, (T)scs[k].y, al, be, v0, v1);
                f0[k + 1] = v0;
                f1[k + 1] = v1;
            }
            V w0 = Gam[col], w1 = Gam[ne + col];
            for (int k = m - 1; k >= 0; --k) {
                const MpsOp o = sop[k];
                const T c = (T)scs[k].x, sn = (T)scs[k].y;
                cg[k * nt + tid] = o.param >= 0 ? op_grad(o, c, sn, be, f0[k], f1[k], f0[k + 1], f1[k + 1], w0, w1)
                                                : T(0);
                op_adjoint(o, c, sn, al, be, w0, w1);
            }
        } else {
            for (int k = 0; k < m; ++k) cg[k * nt + tid] = T(0);
        }
        sync();
        for (int stride = nt / 2; stride > 0; stride >>= 1) {
            if (tid < stride)
                for (int k = 0; k < m; ++k) cg[k * nt + tid] += cg[k * nt + tid + stride];
            sync();
        }
        for (int k = tid; k < m; k += nt) gacc[k] += (double)cg[k * nt];
        sync();
    }
    for (int k = tid; k < m; k += nt) {
        const MpsOp o = sop[k];
        if (o.param >= 0) a.gslot[(int64_t)b * a.n_gates + o.gate] = gacc[k];
    }
}

namespace {

struct DevSync {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};

__global__ void mps_table_kernel(const tlq_gate* __restrict__ gates, int n_gates, const double* __restrict__ theta,
                                 int n_params, int B, double2* __restrict__ tab) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)B * n_gates) return;
    const int b = (int)(i / n_gates), g = (int)(i - (int64_t)b * n_gates);
    const tlq_gate G = gates[g];
    const double ang = G.param >= 0 ? theta[(int64_t)b * n_params + G.param] : G.angle;
    double sn, c;
    sincos(0.5 * ang, &sn, &c);
    tab[i] = make_double2(c, sn);
}

template <typename T>
__global__ void __launch_bounds__(kMpsThreads) mps_build_kernel(MpsArgs<T> a) {
    extern __shared__ __align__(16) unsigned char mps_smem[];
    build_body(a, blockIdx.x, threadIdx.x, blockDim.x, mps_smem, DevSync{});
}

template <typename T>
__global__ void __launch_bounds__(kMpsThreads) mps_sweep_kernel(MpsArgs<T> a) {
    extern __shared__ __align__(16) unsigned char mps_smem[];
    sweep_body(a, blockIdx.x, threadIdx.x, blockDim.x, mps_smem, DevSync{});
}

template <typename T>
__global__ void __launch_bounds__(kMpsThreads) mps_site_kernel(MpsArgs<T> a) {
    extern __shared__ __align__(16) unsigned char mps_smem[];
    site_body(a, blockIdx.x, threadIdx.x, blockDim.x, mps_smem, DevSync{});
}

// E_b = sum_t c_t <P_t> (Neumaier, term order) for i < B; g_{b,p} = sum of the gradients of the
// gates of p (Neumaier, gate order) for B <= i < B + B * n_params.
__global__ void mps_reduce_kernel(const MpsTermDev* __restrict__ terms, int n_terms, const double* __restrict__ e,
                                  const int32_t* __restrict__ pg_off, const int32_t* __restrict__ pg_idx,
                                  int n_params, int n_gates, const double* __restrict__ gslot, int B,
                                  double* __restrict__ energy, double* __restrict__ grad) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < B) {
        double sum = 0.0, comp = 0.0;
        for (int t = 0; t < n_terms; ++t) {
            const double x = terms[t].coeff * e[i * n_terms + t];
            const double y = sum + x;
            comp += fabs(sum) >= fabs(x) ? (sum - y) + x : (x - y) + sum;
            sum = y;
        }
        energy[i] = sum + comp;
        return;
    }
    if (!grad) return;
    const int64_t j = i - B;
    if (j >= (int64_t)B * n_params) return;
    const int b = (int)(j / n_params), p = (int)(j - (int64_t)b * n_params);
    double sum = 0.0, comp = 0.0;   // Neumaier, gate order (as the energy above)
    for (int k = pg_off[p]; k < pg_off[p + 1]; ++k) {
        const double x = gslot[(int64_t)b * n_gates + pg_idx[k]];
        const double y = sum + x;
        comp += fabs(sum) >= fabs(x) ? (sum - y) + x : (x - y) + sum;
        sum = y;
    }
    grad[j] = sum + comp;
}

constexpr size_t kMpsSmemCap = 220 * 1024;

struct MpsSizes {
    int ygroups_sweep = 0, ygroups_site = 0;
    size_t sweep_smem = 0, site_smem = 0, build_smem = 0;
};

template <typename T>
MpsSizes mps_sizes(const MpsPlan& p) {
    using V = typename Cx<T>::t;
    MpsSizes z;
    const size_t el = (size_t)2 * p.max_site_elems * sizeof(V);
    const size_t desc = (size_t)p.max_groups * sizeof(MpsGroup) + (size_t)p.max_contribs * sizeof(MpsContrib);
    for (int y = p.max_groups; y >= 1; --y) {
        const size_t b = el + (size_t)y * el + desc;
        if (b <= kMpsSmemCap) { z.ygroups_sweep = y; z.sweep_smem = b; break; }
    }
    for (int y = p.max_groups; y >= 1; --y) {
        size_t off[7];
        site_smem_offsets<T>(p.max_site_elems, y, p.max_site_ops, p.max_groups, kMpsThreads, off);
        if (off[6] <= kMpsSmemCap) { z.ygroups_site = y; z.site_smem = off[6]; break; }
    }
    z.build_smem = (size_t)p.max_site_ops * (sizeof(double2) + sizeof(MpsOp));
    return z;
}

template <typename T>
size_t work_bytes(const MpsPlan& p, int B) {
    const size_t per = (size_t)(p.a_tot + 4 * p.env_tot + 2 * p.chain_tot) * sizeof(typename Cx<T>::t);
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return al(per * B) + al((size_t)B * p.n_gates * sizeof(double2)) + al((size_t)B * p.n_terms * sizeof(double)) +
           al((size_t)B * p.n_gates * sizeof(double));
}

template <typename T>
int launch_t(const MpsPlan& p, const double* theta, int B, double* energy, double* grad, void* work, cudaStream_t st,
             int* launches) {
    const MpsSizes z = mps_sizes<T>(p);
    if (!z.ygroups_sweep || !z.ygroups_site) return (int)cudaErrorInvalidConfiguration;
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t per = (size_t)(p.a_tot + 4 * p.env_tot + 2 * p.chain_tot) * sizeof(typename Cx<T>::t);
    unsigned char* w = static_cast<unsigned char*>(work);
    MpsArgs<T> a{};
    a.n = p.n;
    a.B = B;
    a.n_gates = p.n_gates;
    a.n_params = p.n_params;
    a.n_terms = p.n_terms;
    a.grad = grad != nullptr;
    a.bits = p.d_bits;
    a.a_off = p.d_a_off;
    a.env_off = p.d_env_off;
    a.op_off = p.d_op_off;
    a.ops = p.d_ops;
    a.act_off = p.d_act_off;
    a.act = p.d_act;
    a.terms = p.d_terms;
    a.pauli = p.d_pauli;
    a.chain_boff = p.d_chain_boff;
    a.dsc = p.d_dsc;
    a.dgroups = p.d_dgroups;
    a.dcontribs = p.d_dcontribs;
    a.a_tot = p.a_tot;
    a.env_tot = p.env_tot;
    a.chain_tot = p.chain_tot;
    a.stride = p.a_tot + 4 * p.env_tot + 2 * p.chain_tot;
    a.max_elems = p.max_site_elems;
    a.max_groups = p.max_groups;
    a.max_ops = p.max_site_ops;
    a.ygroups_sweep = z.ygroups_sweep;
    a.ygroups_site = z.ygroups_site;
    a.work = reinterpret_cast<typename Cx<T>::t*>(w);
    w += al(per * B);
    double2* tab = reinterpret_cast<double2*>(w);
    a.tab = tab;
    w += al((size_t)B * p.n_gates * sizeof(double2));
    a.e = reinterpret_cast<double*>(w);
    w += al((size_t)B * p.n_terms * sizeof(double));
    a.gslot = reinterpret_cast<double*>(w);
    int nl = 0;
    if (p.n_gates > 0) {
        const int64_t tot = (int64_t)B * p.n_gates;
        mps_table_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(p.d_gates, p.n_gates, theta, p.n_params, B,
                                                                        tab);
        ++nl;
    }
    const unsigned sites = (unsigned)((int64_t)p.n * B);
    mps_build_kernel<T><<<sites, kMpsThreads, z.build_smem, st>>>(a);
    ++nl;
    cudaError_t e = cudaFuncSetAttribute(mps_sweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)z.sweep_smem);
    if (e != cudaSuccess) return (int)e;
    mps_sweep_kernel<T><<<2 * B, kMpsThreads, z.sweep_smem, st>>>(a);
    ++nl;
    e = cudaFuncSetAttribute(mps_site_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)z.site_smem);
    if (e != cudaSuccess) return (int)e;
    mps_site_kernel<T><<<sites, kMpsThreads, z.site_smem, st>>>(a);
    ++nl;
    const int64_t rt = (int64_t)B + (grad ? (int64_t)B * p.n_params : 0);
    mps_reduce_kernel<<<(unsigned)((rt + 255) / 256), 256, 0, st>>>(p.d_terms, p.n_terms, a.e, p.d_pg_off, p.d_pg_idx,
                                                                   p.n_params, p.n_gates, a.gslot, B, energy, grad);
    ++nl;
    if (launches) *launches = nl;
    return (int)cudaGetLastError();
}

}  // namespace

size_t mps_workspace_bytes(const MpsPlan& p, int B, bool fp64) {
    return fp64 ? work_bytes<double>(p, B) : work_bytes<float>(p, B);
}

bool mps_fits(const MpsPlan& p, bool fp64, std::string* why) {
    if (fp64 && p.max_bits > kMpsMaxBondBitsF64) {
        *why = "MPS route: bond dimension 2^" + std::to_string(p.max_bits) + " above 2^" +
               std::to_string(kMpsMaxBondBitsF64) + " in FP64";
        return false;
    }
    const MpsSizes z = fp64 ? mps_sizes<double>(p) : mps_sizes<float>(p);
    if (!z.ygroups_sweep || !z.ygroups_site) {
        *why = "MPS route: the site tensors do not fit in shared memory";
        return false;
    }
    return true;
}

int launch_mps(const MpsPlan& p, const double* theta, int B, bool fp64, double* energy, double* grad, void* work,
               void* stream, int* launches) {
    cudaStream_t st = (cudaStream_t)stream;
    return fp64 ? launch_t<double>(p, theta, B, energy, grad, work, st, launches)
                : launch_t<float>(p, theta, B, energy, grad, work, st, launches);
}

}  // namespace tlq
