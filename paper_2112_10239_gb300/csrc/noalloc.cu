// Allocation-free variant of the batched cone kernel launch (tlq_expectation_grad_static).
//
// Some callers cannot allocate device memory when they evaluate a circuit: a host
// application whose own memory manager owns the whole GPU and must account for every
// byte, or a latency-critical loop that cannot afford the implicit device
// synchronisation of cudaMalloc/cudaFree. For them this entry point takes all of its
// working memory -- the copy of the plan, the work list, the gate tables, the per-term
// partial energies, the gradient slots and the work counters -- from one fixed array
// compiled into the library, instead of the context's growable workspace.
//
// The array is a file-scope __device__ object of kStaticScratchBytes; every GPU that
// loads the library holds it until the process exits. Host code cannot use the array's
// name as a device address, so its address is looked up with cudaGetSymbolAddress once
// per device (on the first call on that device, with that device current) and that
// pointer is handed to the kernels. All calls share the one array and it keeps whatever
// the last call left there; the work counters that must start at zero are cleared by
// every call. Two calls whose work overlaps on the GPU (different streams, or the same
// context used from two threads) race on the array and must be serialised by the caller.
#include "runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>

namespace tlq {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;   // 16 MiB

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];


namespace {

std::mutex g_mu;           // guards the scratch addresses and the host-plan cache
std::mutex g_enqueue_mu;   // makes each call's sequence of copies and launches one unit
void* g_scratch_ptr[256] = {nullptr};   // device address of g_static_scratch per device

// Set-up, once per device: the device must be current.
tlq_status static_scratch(int device, void** out) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (device < 0 || device >= 256) {
        set_error("static scratch: device ordinal out of range");
        return TLQ_EINVAL;
    }
    if (!g_scratch_ptr[device]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess || !p) {
            set_error(std::string("static scratch: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
            return TLQ_ECUDA;
        }
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return TLQ_OK;
}

// Host-side plan and work list for one (context, device, circuit, Hamiltonian, batch size,
// gradient flag). An entry is immutable once published and is held by shared_ptr for the
// whole of a call, so a concurrent call that evicts it from the cache cannot free what this
// call still reads. A cache hit is confirmed by comparing the stored circuit and Hamiltonian
// contents, not the fingerprint alone.
struct HostPlan {
    const Context* ctx = nullptr;
    int device = -1;
    uint64_t key[2] = {0, 0};
    int n = 0, n_params = 0;
    std::vector<tlq_gate> gates;
    std::vector<Term> terms;
    std::shared_ptr<Plan> plan;
    int B = -1;
    bool grad = false;
    std::vector<int32_t> items;
    std::vector<ChunkDev> chunks;
    int n_chunks_smem = 0, smem_bytes = 0, smem_threads = kCtaThreads, gsmem_bytes = 0, g_maxW = 0;
    bool accum = false;
};
std::vector<std::shared_ptr<const HostPlan>> g_plans;   // small LRU (most recent last), guarded by g_mu
constexpr size_t kMaxHostPlans = 16;

uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
    return h;
}

void fingerprint(const Circuit& c, const Ham& h, uint64_t out[2]) {
    uint64_t a = mix((uint64_t)c.n, (uint64_t)c.n_params);
    for (const tlq_gate& g : c.gates) {
        a = mix(a, ((uint64_t)(uint32_t)g.kind << 32) | (uint32_t)g.q0);
        a = mix(a, ((uint64_t)(uint32_t)g.q1 << 32) | (uint32_t)g.param);
        uint64_t bits;
        std::memcpy(&bits, &g.angle, 8);
        a = mix(a, bits);
    }
    uint64_t b = mix(0x243f6a8885a308d3ull, (uint64_t)h.n);
    for (const Term& t : h.terms) {
        uint64_t bits;
        std::memcpy(&bits, &t.coeff, 8);
        b = mix(b, bits);
        for (int s : t.sites) b = mix(b, (uint64_t)(uint32_t)s);
        for (char ch : t.letters) b = mix(b, (uint64_t)(unsigned char)ch);
    }
    out[0] = a;
    out[1] = b;
}

bool same_gate(const tlq_gate& x, const tlq_gate& y) {
    return x.kind == y.kind && x.q0 == y.q0 && x.q1 == y.q1 && x.param == y.param &&
           std::memcmp(&x.angle, &y.angle, sizeof(double)) == 0;
}

bool same_term(const Term& x, const Term& y) {
    return std::memcmp(&x.coeff, &y.coeff, sizeof(double)) == 0 && x.sites == y.sites && x.letters == y.letters;
}

bool matches(const HostPlan& hp, const Context* ctx, int device, const uint64_t key[2], const Circuit& c,
             const Ham& h, int B, bool grad) {
    if (hp.ctx != ctx || hp.device != device || hp.B != B || hp.grad != grad) return false;
    if (hp.key[0] != key[0] || hp.key[1] != key[1] || hp.n != c.n || hp.n_params != c.n_params) return false;
    if (hp.gates.size() != c.gates.size() || hp.terms.size() != h.terms.size()) return false;
    for (size_t i = 0; i < c.gates.size(); ++i)
        if (!same_gate(hp.gates[i], c.gates[i])) return false;
    for (size_t i = 0; i < h.terms.size(); ++i)
        if (!same_term(hp.terms[i], h.terms[i])) return false;
    return true;
}

void build_host_worklist(HostPlan& hp, int B, bool grad, int smax) {
    const Plan& P = *hp.plan;
    std::vector<WorkItem> its;
    for (int t = 0; t < (int)P.cones.size(); ++t)
        for (int b = 0; b < B; ++b) push_cone_items(P, t, b, grad, its);
    hp.items.clear();
    ChunkSet cs;
    build_chunks(its, false, grad, smax, hp.items, cs);
    hp.chunks = cs.smem;
    hp.chunks.insert(hp.chunks.end(), cs.glob.begin(), cs.glob.end());
    hp.n_chunks_smem = (int)cs.smem.size();
    hp.smem_bytes = cs.smem_bytes;
    hp.smem_threads = cs.smem_threads;
    hp.gsmem_bytes = cs.gsmem_bytes;
    hp.g_maxW = cs.g_maxW;
    hp.accum = cs.accum;
    hp.B = B;
    hp.grad = grad;
}

// A kernel that finds an inconsistent work item sets the error word; this call cannot read
// it back without synchronising, so the error is made visible in the outputs instead: every
// energy (and gradient entry) of the call becomes NaN. Runs after the reductions.
__global__ void poison_on_error_kernel(const int32_t* err, double* energy, int B, double* grad, int64_t n_grad) {
    if (*err == 0) return;
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    for (int64_t i = threadIdx.x; i < B; i += blockDim.x) energy[i] = nan;
    if (grad)
        for (int64_t i = threadIdx.x; i < n_grad; i += blockDim.x) grad[i] = nan;
}

struct Carve {
    unsigned char* base;
    size_t used = 0;
    void* take(size_t bytes) {
        used = (used + 255) & ~(size_t)255;
        void* p = base + used;
        used += bytes;
        return p;
    }
};

}  // namespace

// Drops the cached host plans of a context that is being destroyed.
void noalloc_forget(const Context* ctx) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_plans.erase(std::remove_if(g_plans.begin(), g_plans.end(),
                                 [&](const std::shared_ptr<const HostPlan>& p) { return p->ctx == ctx; }),
                  g_plans.end());
}

}  // namespace tlq

using namespace tlq;

extern "C" tlq_status tlq_expectation_grad_static(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev,
                                                  int32_t B, double* energy_dev, double* grad_dev, void* cuda_stream) {
    Context* C = reinterpret_cast<Context*>(ctx);
    Circuit* Ci = reinterpret_cast<Circuit*>(c);
    Ham* Hm = reinterpret_cast<Ham*>(h);
    if (!C || !Ci || !Hm) { set_error("tlq_expectation_grad_static: NULL handle"); return TLQ_EINVAL; }
    if (Ci->ctx != C || Hm->ctx != C) { set_error("tlq_expectation_grad_static: handle from another context"); return TLQ_EINVAL; }
    if (Ci->n != Hm->n) { set_error("tlq_expectation_grad_static: qubit counts differ"); return TLQ_EINVAL; }
    if (B <= 0) { set_error("tlq_expectation_grad_static: B must be positive"); return TLQ_EINVAL; }
    if ((!theta_dev && Ci->n_params > 0) || !energy_dev) { set_error("tlq_expectation_grad_static: NULL device pointer"); return TLQ_EINVAL; }
    if (C->host_only()) { set_error("tlq_expectation_grad_static: host-only context"); return TLQ_EUNSUPPORTED; }
    std::lock_guard<std::mutex> lk(C->mu);
    cudaError_t e = cudaSetDevice(C->device);
    if (e != cudaSuccess) { set_error(std::string("cudaSetDevice: ") + cudaGetErrorString(e)); return TLQ_ECUDA; }
    void* scratch = nullptr;
    tlq_status st = static_scratch(C->device, &scratch);
    if (st != TLQ_OK) return st;
    const bool grad = grad_dev != nullptr;

    uint64_t key[2];
    fingerprint(*Ci, *Hm, key);
    std::shared_ptr<const HostPlan> hp;
    {
        std::lock_guard<std::mutex> g(g_mu);
        for (size_t i = 0; i < g_plans.size(); ++i)
            if (matches(*g_plans[i], C, C->device, key, *Ci, *Hm, B, grad)) {
                hp = g_plans[i];
                g_plans.erase(g_plans.begin() + (std::ptrdiff_t)i);   // most recently used goes last
                g_plans.push_back(hp);
                break;
            }
    }
    if (!hp) {
        // planning is host work on this call's own copy; the entry is published only when complete
        std::string err;
        auto plan = make_plan(*Ci, *Hm, &err);
        if (!plan) { set_error(err); return TLQ_EINVAL; }
        if (plan->path != TLQ_PATH_CONE) {
            set_error("tlq_expectation_grad_static: only nearest-neighbour circuits (cone path) are supported");
            return TLQ_EUNSUPPORTED;
        }
        auto fresh = std::make_shared<HostPlan>();
        fresh->ctx = C;
        fresh->device = C->device;
        fresh->key[0] = key[0];
        fresh->key[1] = key[1];
        fresh->n = Ci->n;
        fresh->n_params = Ci->n_params;
        fresh->gates = Ci->gates;
        fresh->terms = Hm->terms;
        fresh->plan = plan;
        int smax = 0;
        cudaDeviceGetAttribute(&smax, cudaDevAttrMaxSharedMemoryPerBlockOptin, C->device);
        smax = smax > 2048 ? smax - 1024 : 48 * 1024;
        build_host_worklist(*fresh, B, grad, smax);
        hp = fresh;
        std::lock_guard<std::mutex> g(g_mu);
        if (g_plans.size() >= kMaxHostPlans) g_plans.erase(g_plans.begin());
        g_plans.push_back(hp);
    }
    const Plan& P = *hp->plan;
    const int G = (int)Ci->gates.size();
    const int T = (int)P.term_coeff.size();
    const int S = std::max<int32_t>(1, P.n_slots);
    const int n_glob = (int)hp->chunks.size() - hp->n_chunks_smem;
    const int g_grid = std::max(0, std::min(n_glob, kGlobalCtasPerSm * C->sm_count));
    const size_t amps = hp->g_maxW > 0 ? ((size_t)1 << hp->g_maxW) + ((size_t)1 << (hp->g_maxW - 3)) : 0;
    const size_t gslot = ((amps * 8 * (grad ? 2 : 1)) + 255) & ~(size_t)255;

    // carve the static array
    Carve cv{reinterpret_cast<unsigned char*>(scratch)};
    tlq_gate* d_gates = (tlq_gate*)cv.take((size_t)std::max(1, G) * sizeof(tlq_gate));
    ConeDev* d_cones = (ConeDev*)cv.take(P.cones.size() * sizeof(ConeDev));
    MeasDev* d_meas = (MeasDev*)cv.take(P.meas.size() * sizeof(MeasDev));
    int32_t* d_prog = (int32_t*)cv.take(P.prog.size() * sizeof(int32_t));
    double* d_tc = (double*)cv.take(P.term_coeff.size() * sizeof(double));
    int32_t* d_poff = (int32_t*)cv.take(P.pmap_off.size() * sizeof(int32_t));
    int32_t* d_pidx = (int32_t*)cv.take(std::max<size_t>(1, P.pmap_idx.size()) * sizeof(int32_t));
    int32_t* d_pterm = (int32_t*)cv.take(std::max<size_t>(1, P.pmap_term.size()) * sizeof(int32_t));
    int32_t* d_items = (int32_t*)cv.take(hp->items.size() * sizeof(int32_t));
    ChunkDev* d_chunks = (ChunkDev*)cv.take(hp->chunks.size() * sizeof(ChunkDev));
    void* d_gt = cv.take((size_t)B * std::max(1, G) * sizeof(float2));
    double* d_e = (double*)cv.take((size_t)B * T * sizeof(double));
    double* d_g = grad ? (double*)cv.take((size_t)B * S * sizeof(double)) : nullptr;
    int32_t* d_cnt = (int32_t*)cv.take(64);
    void* d_gs = g_grid > 0 ? cv.take((size_t)g_grid * gslot) : nullptr;
    if (cv.used > kStaticScratchBytes) {
        set_error("tlq_expectation_grad_static: this call needs " + std::to_string(cv.used) +
                  " bytes of scratch; the library's static array holds " + std::to_string(kStaticScratchBytes) +
                  " bytes (use tlq_expectation_grad_dev, or a smaller batch)");
        return TLQ_ENOMEM;
    }
    cudaStream_t strm = cuda_stream ? (cudaStream_t)cuda_stream : (cudaStream_t)C->stream;
    // Calls from several threads on one stream must not interleave their copies and launches
    // (they share the array), so the whole enqueue sequence is one critical section.
    std::lock_guard<std::mutex> enq(g_enqueue_mu);
    auto put = [&](void* dst, const void* src, size_t bytes) {
        if (bytes && e == cudaSuccess) e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, strm);
    };
    put(d_gates, Ci->gates.data(), (size_t)G * sizeof(tlq_gate));
    put(d_cones, P.cones.data(), P.cones.size() * sizeof(ConeDev));
    put(d_meas, P.meas.data(), P.meas.size() * sizeof(MeasDev));
    put(d_prog, P.prog.data(), P.prog.size() * sizeof(int32_t));
    put(d_tc, P.term_coeff.data(), P.term_coeff.size() * sizeof(double));
    put(d_poff, P.pmap_off.data(), P.pmap_off.size() * sizeof(int32_t));
    put(d_pidx, P.pmap_idx.data(), P.pmap_idx.size() * sizeof(int32_t));
    put(d_pterm, P.pmap_term.data(), P.pmap_term.size() * sizeof(int32_t));
    put(d_items, hp->items.data(), hp->items.size() * sizeof(int32_t));
    put(d_chunks, hp->chunks.data(), hp->chunks.size() * sizeof(ChunkDev));
    if (e == cudaSuccess) e = cudaMemsetAsync(d_cnt, 0, 64, strm);   // work counters and error word start at 0
    if (e != cudaSuccess) { set_error(std::string("tlq_expectation_grad_static: copy: ") + cudaGetErrorString(e)); return TLQ_ECUDA; }

    ConeLaunch L;
    L.cones = d_cones;
    L.meas = d_meas;
    L.prog = d_prog;
    L.term_coeff = d_tc;
    L.pmap_off = d_poff;
    L.pmap_idx = d_pidx;
    L.pmap_term = d_pterm;
    L.gates = d_gates;
    L.n_gates = G;
    L.n_params = Ci->n_params;
    L.n_terms = T;
    L.n_slots = P.n_slots;
    L.B = B;
    L.theta = theta_dev;
    L.items = d_items;
    L.chunks = d_chunks;
    L.n_chunks_smem = hp->n_chunks_smem;
    L.n_chunks = (int)hp->chunks.size();
    L.smem_bytes = hp->smem_bytes;
    L.smem_threads = hp->smem_threads;
    L.accum = hp->accum;
    L.gsmem_bytes = hp->gsmem_bytes;
    L.g_maxW = hp->g_maxW;
    L.gate_table = d_gt;
    L.e_part = d_e;
    L.g_part = d_g;
    L.gscratch = d_gs;
    L.gscratch_slot = gslot;
    L.g_grid = g_grid;
    L.counters = d_cnt;
    L.err = d_cnt + 4;
    L.energy = energy_dev;
    L.grad = grad_dev;
    L.fp64 = false;
    L.sm_count = C->sm_count;
    int rc = launch_cone(L, strm);
    if (rc == 0) {
        poison_on_error_kernel<<<1, 256, 0, strm>>>(L.err, energy_dev, B, grad_dev,
                                                   grad ? (int64_t)B * Ci->n_params : 0);
        rc = (int)cudaGetLastError();
    }
    if (rc != 0) {
        set_error(std::string("tlq_expectation_grad_static: launch: ") + cudaGetErrorString((cudaError_t)rc));
        return TLQ_ECUDA;
    }
    return TLQ_OK;
}
