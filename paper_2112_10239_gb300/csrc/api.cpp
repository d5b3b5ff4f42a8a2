// C-ABI implementation: validation, handles, plan cache, workspace and the synchronous
// and device-pointer entry points. Serving (tlq_submit / tlq_poll) is in serving.cpp.
#include "runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <set>

namespace tlq {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }
const char* get_error() { return t_err.c_str(); }

#define TLQ_CUDA(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                  \
            return TLQ_ECUDA;                                                               \
        }                                                                                   \
    } while (0)

PlanEntry::~PlanEntry() {
    if (graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)graph_exec);
    cudaFree(d_cones);
    cudaFree(d_meas);
    cudaFree(d_prog);
    cudaFree(d_term_coeff);
    cudaFree(d_pmap_off);
    cudaFree(d_pmap_idx);
    cudaFree(d_pmap_term);
    cudaFree(d_gates);
    cudaFree(d_dlayers);
    cudaFree(d_dclasses);
    cudaFree(d_dpcd);
    cudaFree(d_dstage);
    cudaFree(d_ddists);
    cudaFree(d_dzterms);
    cudaFree(d_dtab_gate);
    cudaFree(d_dtab_mult);
    cudaFree(d_dxterms);
    cudaFree(d_dallterms);
    cudaFree(d_dfgates);
    cudaFree(d_dfxterms);
    cudaFree(d_dadj_off);
    cudaFree(d_dadj_idx);
    cudaFree(d_dinit_pcd);
    cudaFree(d_items);
    cudaFree(d_chunks);
}

template <typename T>
static tlq_status upload(const std::vector<T>& v, T** out, size_t* bytes) {
    *out = nullptr;
    if (v.empty()) return TLQ_OK;
    TLQ_CUDA(cudaMalloc((void**)out, v.size() * sizeof(T)));
    TLQ_CUDA(cudaMemcpy(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *bytes += v.size() * sizeof(T);
    return TLQ_OK;
}

#define TLQ_TRY(x)                          \
    do {                                    \
        tlq_status s_ = (x);                \
        if (s_ != TLQ_OK) return s_;        \
    } while (0)

tlq_status get_plan(Context* ctx, Circuit* c, Ham* h, std::shared_ptr<PlanEntry>* out) {
    auto key = std::make_pair(c->id, h->id);
    auto it = ctx->plans.find(key);
    if (it != ctx->plans.end()) { *out = it->second; return TLQ_OK; }
    std::string err;
    auto plan = make_plan(*c, *h, &err);
    if (!plan) { set_error(err); return TLQ_EUNSUPPORTED; }
    auto pe = std::make_shared<PlanEntry>();
    pe->plan = plan;
    pe->circ_id = c->id;
    pe->ham_id = h->id;
    if (!ctx->host_only()) {
        size_t bytes = 0;
        std::vector<tlq_gate> gates = c->gates;
        TLQ_TRY(upload(gates, &pe->d_gates, &bytes));
        TLQ_TRY(upload(plan->term_coeff, &pe->d_term_coeff, &bytes));
        if (plan->path == TLQ_PATH_CONE) {
            TLQ_TRY(upload(plan->cones, &pe->d_cones, &bytes));
            TLQ_TRY(upload(plan->meas, &pe->d_meas, &bytes));
            TLQ_TRY(upload(plan->prog, &pe->d_prog, &bytes));
            TLQ_TRY(upload(plan->pmap_off, &pe->d_pmap_off, &bytes));
            TLQ_TRY(upload(plan->pmap_idx, &pe->d_pmap_idx, &bytes));
            TLQ_TRY(upload(plan->pmap_term, &pe->d_pmap_term, &bytes));
        }
        if (plan->dense) {
            const DensePlan& D = *plan->dense;
            TLQ_TRY(upload(D.layers, &pe->d_dlayers, &bytes));
            TLQ_TRY(upload(D.classes, &pe->d_dclasses, &bytes));
            TLQ_TRY(upload(D.pcd, &pe->d_dpcd, &bytes));
            TLQ_TRY(upload(D.stage, &pe->d_dstage, &bytes));
            TLQ_TRY(upload(D.dists, &pe->d_ddists, &bytes));
            TLQ_TRY(upload(D.zterms, &pe->d_dzterms, &bytes));
            TLQ_TRY(upload(D.tab_gate, &pe->d_dtab_gate, &bytes));
            TLQ_TRY(upload(D.tab_mult, &pe->d_dtab_mult, &bytes));
            TLQ_TRY(upload(D.xterms, &pe->d_dxterms, &bytes));
            TLQ_TRY(upload(D.all_terms, &pe->d_dallterms, &bytes));
            TLQ_TRY(upload(D.fgates, &pe->d_dfgates, &bytes));
            TLQ_TRY(upload(D.fxterms, &pe->d_dfxterms, &bytes));
            TLQ_TRY(upload(D.adj_off, &pe->d_dadj_off, &bytes));
            TLQ_TRY(upload(D.adj_idx, &pe->d_dadj_idx, &bytes));
            TLQ_TRY(upload(D.init_pcd, &pe->d_dinit_pcd, &bytes));
        }
        pe->device_bytes = bytes;
        ctx->held += bytes;
    }
    ctx->plans[key] = pe;
    *out = pe;
    return TLQ_OK;
}

static int smem_optin(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v > 2048 ? v - 1024 : 48 * 1024;
}

tlq_status ensure_worklist(Context* ctx, PlanEntry& pe, const Circuit& c, int B, bool fp64, bool grad) {
    (void)c;
    if (pe.wl_B == B && pe.wl_fp64 == fp64 && pe.wl_grad == grad) return TLQ_OK;
    const Plan& P = *pe.plan;
    const int T = (int)P.cones.size();
    std::vector<WorkItem> its;
    its.reserve((size_t)T * B * 2);
    for (int t = 0; t < T; ++t)
        for (int b = 0; b < B; ++b) push_cone_items(P, t, b, grad, its);
    std::vector<int32_t> items;
    ChunkSet cs;
    build_chunks(its, fp64, grad, smem_optin(ctx->device), items, cs);
    std::vector<ChunkDev> chunks = cs.smem;
    chunks.insert(chunks.end(), cs.glob.begin(), cs.glob.end());
    cudaFree(pe.d_items);
    cudaFree(pe.d_chunks);
    pe.d_items = nullptr;
    pe.d_chunks = nullptr;
    size_t bytes = 0;
    TLQ_TRY(upload(items, &pe.d_items, &bytes));
    TLQ_TRY(upload(chunks, &pe.d_chunks, &bytes));
    pe.n_chunks_smem = (int)cs.smem.size();
    pe.n_chunks = (int)chunks.size();
    pe.smem_bytes = cs.smem_bytes;
    pe.smem_threads = cs.smem_threads;
    pe.gsmem_bytes = cs.gsmem_bytes;
    pe.g_maxW = cs.g_maxW;
    pe.accum = cs.accum;
    pe.wl_B = B;
    pe.wl_fp64 = fp64;
    pe.wl_grad = grad;
    return TLQ_OK;
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of one CTA's global-memory cone states (padded psi, and lam for gradients).
static size_t global_slot_bytes(int W, bool fp64, bool grad) {
    const size_t amps = ((size_t)1 << W) + ((size_t)1 << (W - 3));
    return align256(amps * (fp64 ? 16 : 8) * (grad ? 2 : 1));
}

static int global_grid(const PlanEntry& pe, int sm_count) {
    const int ng = pe.n_chunks - pe.n_chunks_smem;
    return std::max(0, std::min(ng, kGlobalCtasPerSm * sm_count));
}

size_t cone_workspace_bytes(const PlanEntry& pe, const Circuit& c, int B, bool fp64, bool grad, int g_grid) {
    const Plan& P = *pe.plan;
    const size_t r2 = fp64 ? 16 : 8;
    size_t s = 0;
    s += align256((size_t)B * c.gates.size() * r2);
    s += align256((size_t)B * P.term_coeff.size() * sizeof(double));
    if (grad) s += align256((size_t)B * std::max<int32_t>(1, P.n_slots) * sizeof(double));
    if (g_grid > 0) s += align256((size_t)g_grid * global_slot_bytes(pe.g_maxW, fp64, grad));
    return s + 1024;
}

// gradient mode adds the adjoint state and the per-pass gradient partials
static size_t dense_gpart_count(const DensePlan& D, int sm_count) {
    return std::max<size_t>(1, D.passes.size()) * kDenseAdjSlots * (size_t)dense_grid(D.n_eff, std::max(1, sm_count));
}

size_t dense_workspace_bytes(const PlanEntry& pe, const Circuit& c, int B, bool grad, int sm_count) {
    const DensePlan& D = *pe.plan->dense;
    size_t s = 0;
    s += align256((size_t)B * std::max<size_t>(1, c.gates.size()) * 8);
    s += align256((size_t)B * std::max<size_t>(1, D.tab_gate.size()) * 8);
    s += align256(((size_t)1 << D.n_eff) * 8);
    s += align256(dense_partial_count(D.n_eff) * sizeof(double));
    if (grad) {
        s += align256(((size_t)1 << D.n_eff) * 8);
        s += align256(dense_gpart_count(D, sm_count) * sizeof(double));
    }
    return s + 1024;
}

static tlq_status run_dense(Context* ctx, PlanEntry& pe, const Circuit& c, const double* theta_dev, int B,
                            double* energy_dev, double* grad_dev, bool per_gate, void* stream, Workspace* ws,
                            void** state_out = nullptr, bool tc = false) {
    // The fused passes of an expectation run in the rotation frame (DensePlan::frame_mask); a
    // call that hands out the state (state_out) and the per-gate sweeps use the plain frame.
    const bool framed = !per_gate && !state_out && pe.plan->dense->frame_mask != 0;
    const DensePlan& D = *pe.plan->dense;
    const bool grad = grad_dev != nullptr;
    const size_t need = dense_workspace_bytes(pe, c, B, grad, ctx->sm_count);
    if (ws->cap - ws->used < need) {
        set_error("workspace too small for the dense state");
        return TLQ_ENOMEM;
    }
    DenseLaunch L;
    L.n_eff = D.n_eff;
    L.n_passes = (int32_t)D.passes.size();
    L.layers = pe.d_dlayers;
    L.classes = pe.d_dclasses;
    L.pcd = pe.d_dpcd;
    L.stage = pe.d_dstage;
    L.dists = pe.d_ddists;
    L.energy_class_off = D.energy_class_off;
    L.energy_nclass = D.energy_nclass;
    L.zterms = pe.d_dzterms;
    L.n_zterms = (int32_t)D.zterms.size();
    L.n_xterms = (int32_t)D.xterms.size();
    L.tab_gate = pe.d_dtab_gate;
    L.tab_mult = pe.d_dtab_mult;
    L.tab_entries = (int32_t)D.tab_gate.size();
    L.gates = framed ? pe.d_dfgates : pe.d_gates;
    L.n_gates = (int32_t)c.gates.size();
    L.n_params = c.n_params;
    L.B = B;
    L.theta = theta_dev;
    L.gate_table = ws->take((size_t)B * std::max<size_t>(1, c.gates.size()) * 8);
    L.phase_tab = ws->take((size_t)B * std::max<size_t>(1, D.tab_gate.size()) * 8);
    L.state = ws->take(((size_t)1 << D.n_eff) * 8);
    if (state_out) *state_out = L.state;
    L.partial = (double*)ws->take(dense_partial_count(D.n_eff) * sizeof(double));
    if (grad) {
        L.lam = ws->take(((size_t)1 << D.n_eff) * 8);
        L.gpart = (double*)ws->take(dense_gpart_count(D, ctx->sm_count) * sizeof(double));
    }
    L.xterms = framed ? pe.d_dfxterms : pe.d_dxterms;
    L.all_terms = pe.d_dallterms;
    L.adj_off = pe.d_dadj_off;
    L.adj_idx = pe.d_dadj_idx;
    L.energy = energy_dev;
    L.grad = grad_dev;
    L.err = ctx->d_err;
    L.per_gate = per_gate;
    L.tc = tc;
    L.keep_state = state_out != nullptr;
    L.gen_first = D.gen_first;
    L.sm_count = ctx->sm_count;
    L.host_gates = c.gates.data();
    L.host_passes = D.passes.data();
    L.product_init = D.product_init;
    L.host_fwd_passes = D.fwd_passes.data();
    L.host_rev_store = D.rev_store.data();
    L.n_fwd_passes = (int32_t)D.fwd_passes.size();
    L.host_init_gate = D.init_gate.data();
    L.init_class_off = D.init_class_off;
    L.init_nclass = D.init_nclass;
    L.init_pcd = pe.d_dinit_pcd;
    L.host_xterms = framed ? D.fxterms.data() : D.xterms.data();
    L.host_all_terms = D.all_terms.data();
    L.n_all_terms = (int32_t)D.all_terms.size();
    if (ctx->profile) { L.ev_begin = ctx->prof_ev[0]; L.ev_end = ctx->prof_ev[1]; }
    const int rc = launch_dense(L, stream);
    ctx->last_launches = L.launches;
    if (rc != 0) {
        set_error(std::string("dense launch: ") + cudaGetErrorString((cudaError_t)rc));
        return TLQ_ECUDA;
    }
    return TLQ_OK;
}

tlq_status run_device(Context* ctx, Circuit* c, Ham* h, const double* theta_dev, int B, tlq_precision prec,
                      double* energy_dev, double* grad_dev, void* stream, Workspace* ws) {
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    const Plan& P = *pe->plan;
    const bool fp64 = prec == TLQ_FP64_REF;
    const bool grad = grad_dev != nullptr;
    const bool plain = ctx->cfg.fuse_k == 1;
    if (!grad && !fp64 && !plain && P.dense &&
        tiny_fits(c->n, (int)c->gates.size(), (int)P.dense->all_terms.size())) {
        // a small circuit, energies only: one CTA per set with the whole state (tiny.cu)
        if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[0], (cudaStream_t)stream));
        const int rc = launch_tiny_energy(pe->d_gates, (int)c->gates.size(), theta_dev, c->n_params, c->n,
                                          pe->d_dallterms, (int)P.dense->all_terms.size(), B, energy_dev, stream);
        if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[1], (cudaStream_t)stream));
        ctx->last_launches = 1;
        if (rc != 0) {
            set_error(std::string("tiny launch: ") + cudaGetErrorString((cudaError_t)rc));
            return TLQ_ECUDA;
        }
        return TLQ_OK;
    }
    if (P.path != TLQ_PATH_CONE || plain) {
        if (!P.dense) {
            set_error("no dense statevector plan for this request (n > " + std::to_string(kDenseMaxQubits) + ")");
            return TLQ_EUNSUPPORTED;
        }
        if (fp64) {
            set_error(std::string("the dense statevector path runs in FP32 only (") +
                      (P.path == TLQ_PATH_DENSE ? P.why_dense : std::string("plain per-gate mode")) + ")");
            return TLQ_EUNSUPPORTED;
        }
        return run_dense(ctx, *pe, *c, theta_dev, B, energy_dev, grad_dev, plain || !P.dense->fits_fused, stream, ws,
                         nullptr, prec == TLQ_MIXED_TC);
    }
    TLQ_TRY(ensure_worklist(ctx, *pe, *c, B, fp64, grad));
    const int g_grid = global_grid(*pe, ctx->sm_count);
    const size_t need = cone_workspace_bytes(*pe, *c, B, fp64, grad, g_grid);
    if (ws->cap - ws->used < need) {
        set_error("workspace too small");
        return TLQ_ENOMEM;
    }
    ConeLaunch L;
    L.cones = pe->d_cones;
    L.meas = pe->d_meas;
    L.prog = pe->d_prog;
    L.term_coeff = pe->d_term_coeff;
    L.pmap_off = pe->d_pmap_off;
    L.pmap_idx = pe->d_pmap_idx;
    L.pmap_term = pe->d_pmap_term;
    L.gates = pe->d_gates;
    L.n_gates = (int32_t)c->gates.size();
    L.n_params = c->n_params;
    L.n_terms = (int32_t)P.term_coeff.size();
    L.n_slots = P.n_slots;
    L.B = B;
    L.theta = theta_dev;
    L.items = pe->d_items;
    L.chunks = pe->d_chunks;
    L.n_chunks_smem = pe->n_chunks_smem;
    L.n_chunks = pe->n_chunks;
    L.smem_bytes = pe->smem_bytes;
    L.smem_threads = pe->smem_threads;
    L.accum = pe->accum;
    L.gsmem_bytes = pe->gsmem_bytes;
    L.g_maxW = pe->g_maxW;
    const size_t r2 = fp64 ? 16 : 8;
    L.gate_table = ws->take((size_t)B * c->gates.size() * r2);
    L.e_part = (double*)ws->take((size_t)B * P.term_coeff.size() * sizeof(double));
    L.g_part = grad ? (double*)ws->take((size_t)B * std::max<int32_t>(1, P.n_slots) * sizeof(double)) : nullptr;
    L.g_grid = g_grid;
    L.gscratch_slot = g_grid > 0 ? global_slot_bytes(pe->g_maxW, fp64, grad) : 0;
    L.gscratch = g_grid > 0 ? ws->take((size_t)g_grid * L.gscratch_slot) : nullptr;
    L.counters = ctx->d_counters;
    L.err = ctx->d_err;
    L.energy = energy_dev;
    L.grad = grad_dev;
    L.fp64 = fp64;
    L.sm_count = ctx->sm_count;
    if (ctx->profile) { L.ev_begin = ctx->prof_ev[0]; L.ev_end = ctx->prof_ev[1]; }
    int rc = launch_cone(L, stream);
    ctx->last_launches = L.launches;
    if (rc != 0) {
        set_error(std::string("cone launch: ") + cudaGetErrorString((cudaError_t)rc));
        return TLQ_ECUDA;
    }
    return TLQ_OK;
}

// Size the context workspace for one call (plus its I/O buffers); grow-only.
static tlq_status reserve(Context* ctx, size_t bytes) {
    ctx->ws.used = 0;
    if (ctx->ws.cap >= bytes) return TLQ_OK;
    const size_t others = ctx->held - ctx->ws.cap;
    if (others + bytes > ctx->budget) {
        set_error("request needs " + std::to_string(bytes) + " bytes of workspace; budget " +
                  std::to_string(ctx->budget) + " bytes, " + std::to_string(others) + " held elsewhere");
        return TLQ_ENOMEM;
    }
    size_t nb = std::max(bytes, ctx->ws.cap + ctx->ws.cap / 2);
    if (others + nb > ctx->budget) nb = bytes;
    TLQ_CUDA(cudaStreamSynchronize((cudaStream_t)ctx->stream));
    if (ctx->ws.base) cudaFree(ctx->ws.base);
    ctx->held -= ctx->ws.cap;
    ctx->ws.base = nullptr;
    ctx->ws.cap = 0;
    cudaError_t e = cudaMalloc(&ctx->ws.base, nb);
    if (e != cudaSuccess) {
        set_error(std::string("workspace cudaMalloc: ") + cudaGetErrorString(e));
        return TLQ_ENOMEM;
    }
    ctx->ws.cap = nb;
    ctx->held += nb;
    return TLQ_OK;
}

static tlq_status ensure_pinned(Context* ctx, size_t bytes) {
    if (ctx->h_pinned_cap >= bytes) return TLQ_OK;
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    ctx->h_pinned = nullptr;
    ctx->h_pinned_cap = 0;
    TLQ_CUDA(cudaMallocHost(&ctx->h_pinned, bytes));
    ctx->h_pinned_cap = bytes;
    return TLQ_OK;
}

}  // namespace tlq

using namespace tlq;

struct tlq_ctx_s : Context {};
struct tlq_circuit_s : Circuit {};
struct tlq_ham_s : Ham {};

extern "C" {

int32_t tlq_version(void) { return 10000; }

const char* tlq_last_error(tlq_ctx) { return get_error(); }

tlq_status tlq_init(const tlq_config* cfg_in, tlq_ctx* out) {
    if (!out) { set_error("tlq_init: out is NULL"); return TLQ_EINVAL; }
    tlq_config cfg{};
    cfg.device = 0;
    if (cfg_in) cfg = *cfg_in;
    if (cfg.max_slots <= 0) cfg.max_slots = 64;
    if (cfg.default_prec < TLQ_FP32 || cfg.default_prec > TLQ_FP64_REF) {
        set_error("tlq_init: unknown default precision");
        return TLQ_EINVAL;
    }
    auto* ctx = new tlq_ctx_s();
    ctx->cfg = cfg;
    ctx->device = cfg.device;
    if (cfg.device >= 0) {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || cfg.device >= ndev) {
            set_error(std::string("tlq_init: no CUDA device ") + std::to_string(cfg.device) +
                      (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : std::string()));
            delete ctx;
            return e != cudaSuccess ? TLQ_ECUDA : TLQ_EINVAL;
        }
        auto fail = [&](cudaError_t err, const char* what) {
            set_error(std::string("tlq_init: ") + what + ": " + cudaGetErrorString(err));
            delete ctx;
            return TLQ_ECUDA;
        };
        if ((e = cudaSetDevice(cfg.device)) != cudaSuccess) return fail(e, "cudaSetDevice");
        cudaStream_t st;
        if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "stream");
        ctx->stream = st;
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, cfg.device);
        size_t freeb = 0, totalb = 0;
        cudaMemGetInfo(&freeb, &totalb);
        ctx->budget = cfg.mem_budget ? cfg.mem_budget : (size_t)(0.8 * (double)freeb);
        if ((e = cudaMalloc((void**)&ctx->d_counters, 64)) != cudaSuccess) return fail(e, "counters");
        ctx->d_err = ctx->d_counters + 4;
        ctx->held = 64;
    }
    *out = ctx;
    return TLQ_OK;
}

tlq_status tlq_destroy(tlq_ctx ctx) {
    if (!ctx) return TLQ_OK;
    scheduler_stop(ctx);
    noalloc_forget(ctx);
    if (!ctx->host_only()) {
        cudaSetDevice(ctx->device);
        cudaStreamSynchronize((cudaStream_t)ctx->stream);
    }
    ctx->plans.clear();
    ctx->mps_plans.clear();
    for (Circuit* c : ctx->circuits) delete static_cast<tlq_circuit_s*>(c);
    for (Ham* h : ctx->hams) delete static_cast<tlq_ham_s*>(h);
    if (!ctx->host_only()) {
        cudaFree(ctx->ws.base);
        cudaFree(ctx->d_counters);
        if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
        if (ctx->prof_ev[0]) cudaEventDestroy((cudaEvent_t)ctx->prof_ev[0]);
        if (ctx->prof_ev[1]) cudaEventDestroy((cudaEvent_t)ctx->prof_ev[1]);
        cudaStreamDestroy((cudaStream_t)ctx->stream);
    }
    delete ctx;
    return TLQ_OK;
}

tlq_status tlq_circuit_create(tlq_ctx ctx, int32_t n, const tlq_gate* gates, int32_t n_gates, int32_t n_params,
                              tlq_circuit* out) {
    if (!ctx || !out) { set_error("tlq_circuit_create: NULL context or out"); return TLQ_EINVAL; }
    if (n < 1 || n > (1 << 20)) { set_error("tlq_circuit_create: n_qubits out of [1, 2^20]"); return TLQ_EINVAL; }
    if (n_gates < 0 || (n_gates > 0 && !gates)) { set_error("tlq_circuit_create: bad gate array"); return TLQ_EINVAL; }
    if (n_params < 0) { set_error("tlq_circuit_create: n_params < 0"); return TLQ_EINVAL; }
    for (int i = 0; i < n_gates; ++i) {
        const tlq_gate& g = gates[i];
        std::string where = "tlq_circuit_create: gate " + std::to_string(i) + ": ";
        if (g.kind < TLQ_RX || g.kind > TLQ_CZ) { set_error(where + "unknown kind"); return TLQ_EINVAL; }
        if (g.q0 < 0 || g.q0 >= n) { set_error(where + "qubit out of range"); return TLQ_EINVAL; }
        const bool two = g.kind == TLQ_RZZ || g.kind == TLQ_CZ;
        if (two) {
            if (g.q1 < 0 || g.q1 >= n) { set_error(where + "second qubit out of range"); return TLQ_EINVAL; }
            if (g.q1 == g.q0) { set_error(where + "q0 == q1"); return TLQ_EINVAL; }
        }
        if (g.kind != TLQ_CZ && (g.param < -1 || g.param >= n_params)) {
            set_error(where + "param index out of range");
            return TLQ_EINVAL;
        }
    }
    auto* c = new tlq_circuit_s();
    c->ctx = ctx;
    c->n = n;
    c->n_params = n_params;
    c->gates.assign(gates, gates + n_gates);
    for (auto& g : c->gates) {
        if (g.kind != TLQ_RZZ && g.kind != TLQ_CZ) g.q1 = -1;
        if (g.kind == TLQ_CZ) g.param = -1;
    }
    plan_circuit_layers(*c);
    c->id = ctx->next_id++;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->circuits.push_back(c);
    }
    *out = c;
    return TLQ_OK;
}

static void evict_plans(Context* ctx, uint64_t circ_id, uint64_t ham_id) {
    for (auto it = ctx->plans.begin(); it != ctx->plans.end();) {
        if (it->first.first == circ_id || it->first.second == ham_id) {
            ctx->held -= it->second->device_bytes;
            it = ctx->plans.erase(it);
        } else {
            ++it;
        }
    }
    for (auto it = ctx->mps_plans.begin(); it != ctx->mps_plans.end();) {
        if (it->first.first == circ_id || it->first.second == ham_id) {
            size_t b = 0;
            mps_info(*it->second, nullptr, nullptr, &b);
            ctx->held -= b;
            it = ctx->mps_plans.erase(it);
        } else {
            ++it;
        }
    }
}

tlq_status tlq_circuit_destroy(tlq_circuit c) {
    if (!c) return TLQ_OK;
    Context* ctx = c->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->host_only()) cudaStreamSynchronize((cudaStream_t)ctx->stream);
    evict_plans(ctx, c->id, 0);
    ctx->circuits.erase(std::remove(ctx->circuits.begin(), ctx->circuits.end(), (Circuit*)c), ctx->circuits.end());
    delete c;
    return TLQ_OK;
}

tlq_status tlq_hamiltonian_create(tlq_ctx ctx, int32_t n, const tlq_term* terms, int32_t n_terms, tlq_ham* out) {
    if (!ctx || !out) { set_error("tlq_hamiltonian_create: NULL context or out"); return TLQ_EINVAL; }
    if (n < 1 || n > (1 << 20)) { set_error("tlq_hamiltonian_create: n_qubits out of [1, 2^20]"); return TLQ_EINVAL; }
    if (n_terms < 1 || !terms) { set_error("tlq_hamiltonian_create: need at least one term"); return TLQ_EINVAL; }
    auto* h = new tlq_ham_s();
    h->ctx = ctx;
    h->n = n;
    for (int t = 0; t < n_terms; ++t) {
        const tlq_term& T = terms[t];
        std::string where = "tlq_hamiltonian_create: term " + std::to_string(t) + ": ";
        if (T.nsites < 1 || !T.sites || !T.paulis) { set_error(where + "empty term"); delete h; return TLQ_EINVAL; }
        Term tm;
        tm.coeff = T.coeff;
        std::set<int> seen;
        for (int k = 0; k < T.nsites; ++k) {
            const int s = T.sites[k];
            const char l = T.paulis[k];
            if (s < 0 || s >= n) { set_error(where + "site out of range"); delete h; return TLQ_EINVAL; }
            if (l != 'X' && l != 'Y' && l != 'Z') { set_error(where + "unknown Pauli letter"); delete h; return TLQ_EINVAL; }
            if (!seen.insert(s).second) { set_error(where + "duplicate site"); delete h; return TLQ_EINVAL; }
            tm.sites.push_back(s);
            tm.letters.push_back(l);
        }
        h->terms.push_back(std::move(tm));
    }
    h->id = ctx->next_id++;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->hams.push_back(h);
    }
    *out = h;
    return TLQ_OK;
}

tlq_status tlq_hamiltonian_destroy(tlq_ham h) {
    if (!h) return TLQ_OK;
    Context* ctx = h->ctx;
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (!ctx->host_only()) cudaStreamSynchronize((cudaStream_t)ctx->stream);
    evict_plans(ctx, 0, h->id);
    ctx->hams.erase(std::remove(ctx->hams.begin(), ctx->hams.end(), (Ham*)h), ctx->hams.end());
    delete h;
    return TLQ_OK;
}

static tlq_status check_pair(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t B, tlq_precision prec) {
    if (!ctx || !c || !h) { set_error("NULL context, circuit or Hamiltonian"); return TLQ_EINVAL; }
    if (c->ctx != ctx || h->ctx != ctx) { set_error("circuit or Hamiltonian belongs to another context"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    if (B <= 0) { set_error("B must be positive"); return TLQ_EINVAL; }
    if (prec < TLQ_FP32 || prec > TLQ_FP64_REF) { set_error("unknown precision"); return TLQ_EINVAL; }
    if (ctx->host_only()) { set_error("host-only context: no device work"); return TLQ_EUNSUPPORTED; }
    return TLQ_OK;
}

// Enqueue the synchronous call's device work on `st`: clear the error word, copy the angles
// from the pinned staging buffer, run the path, copy energies (gradients) and the error word
// back into the staging buffer.
static tlq_status sync_enqueue(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t B, tlq_precision prec, bool want_grad,
                               cudaStream_t st, size_t th_b, size_t e_b, size_t g_b) {
    // Small circuits, energies only (the small-circuit kernel): the kernel reads the angles from
    // the pinned staging buffer and writes the energies into it through its device mapping, so
    // the call is one kernel, with no copies (the error word in the staging buffer is cleared by
    // the host before every launch; this kernel never sets it).
    if (!want_grad && prec != TLQ_FP64_REF && ctx->cfg.fuse_k != 1) {
        std::shared_ptr<PlanEntry> pe;
        TLQ_TRY(get_plan(ctx, c, h, &pe));
        const Plan& P = *pe->plan;
        void* dhp = nullptr;
        if (P.dense && tiny_fits(c->n, (int)c->gates.size(), (int)P.dense->all_terms.size()) &&
            cudaHostGetDevicePointer(&dhp, ctx->h_pinned, 0) == cudaSuccess && dhp) {
            if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[0], st));
            const int rc = launch_tiny_energy(pe->d_gates, (int)c->gates.size(), (const double*)dhp, c->n_params, c->n,
                                              pe->d_dallterms, (int)P.dense->all_terms.size(), B,
                                              (double*)((char*)dhp + th_b), st);
            if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[1], st));
            ctx->last_launches = 1;
            if (rc != 0) {
                set_error(std::string("tiny launch: ") + cudaGetErrorString((cudaError_t)rc));
                return TLQ_ECUDA;
            }
            return TLQ_OK;
        }
        cudaGetLastError();   // no device mapping: the copy path below
    }
    ctx->ws.used = 0;
    double* d_theta = (double*)ctx->ws.take(th_b);
    double* d_e = (double*)ctx->ws.take(e_b);
    double* d_g = want_grad ? (double*)ctx->ws.take(g_b) : nullptr;
    char* hp = (char*)ctx->h_pinned;
    TLQ_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), st));
    if (c->n_params > 0)
        TLQ_CUDA(cudaMemcpyAsync(d_theta, hp, (size_t)B * c->n_params * sizeof(double), cudaMemcpyHostToDevice, st));
    TLQ_TRY(run_device(ctx, c, h, d_theta, B, prec, d_e, d_g, st, &ctx->ws));
    TLQ_CUDA(cudaMemcpyAsync(hp + th_b, d_e, e_b, cudaMemcpyDeviceToHost, st));
    if (want_grad)
        TLQ_CUDA(cudaMemcpyAsync(hp + th_b + e_b, d_g, (size_t)B * c->n_params * sizeof(double), cudaMemcpyDeviceToHost, st));
    TLQ_CUDA(cudaMemcpyAsync(hp + th_b + e_b + g_b, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    return TLQ_OK;
}

static tlq_status sync_call(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B, tlq_precision prec,
                            double* energy, double* grad) {
    TLQ_TRY(check_pair(ctx, c, h, B, prec));
    if (!theta && c->n_params > 0) { set_error("theta is NULL"); return TLQ_EINVAL; }
    if (!energy) { set_error("energy is NULL"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    const bool fp64 = prec == TLQ_FP64_REF;
    const bool want_grad = grad != nullptr;
    size_t work = 0;
    if (pe->plan->path == TLQ_PATH_CONE && ctx->cfg.fuse_k != 1) {
        TLQ_TRY(ensure_worklist(ctx, *pe, *c, B, fp64, want_grad));
        work = cone_workspace_bytes(*pe, *c, B, fp64, want_grad, global_grid(*pe, ctx->sm_count));
    } else if (pe->plan->dense) {
        work = dense_workspace_bytes(*pe, *c, B, want_grad, ctx->sm_count);
    }
    const size_t P = (size_t)std::max(1, c->n_params);
    const size_t th_b = (size_t)B * P * sizeof(double);
    const size_t e_b = (size_t)B * sizeof(double);
    const size_t g_b = want_grad ? (size_t)B * P * sizeof(double) : 0;
    TLQ_TRY(reserve(ctx, work + th_b + e_b + g_b + 4096));
    TLQ_TRY(ensure_pinned(ctx, th_b + e_b + g_b + 64));
    cudaStream_t st = (cudaStream_t)ctx->stream;
    char* hp = (char*)ctx->h_pinned;
    if (c->n_params > 0) std::memcpy(hp, theta, (size_t)B * c->n_params * sizeof(double));
    // The device work is a fixed launch sequence for a given plan, batch size, precision and
    // buffers: capture it once as a CUDA graph and replay it (one launch instead of about ten
    // runtime calls). Profiling records events around single kernels, so it runs uncaptured;
    // a capture that fails also falls back to direct launches.
    PlanEntry::GraphKey key;
    key.B = B;
    key.prec = (int)prec;
    key.grad = want_grad ? 1 : 0;
    key.fuse_k = ctx->cfg.fuse_k;
    key.ws_base = ctx->ws.base;
    key.ws_cap = ctx->ws.cap;
    key.pinned = ctx->h_pinned;
    key.pinned_cap = ctx->h_pinned_cap;
    *(int32_t*)(hp + th_b + e_b + g_b) = 0;   // the error word (the copy path overwrites it)
    bool launched = false;
    if (!ctx->profile) {
        if (!(pe->graph_exec && pe->graph_key == key)) {
            if (pe->graph_exec) cudaGraphExecDestroy((cudaGraphExec_t)pe->graph_exec);
            pe->graph_exec = nullptr;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const tlq_status s = sync_enqueue(ctx, c, h, B, prec, want_grad, st, th_b, e_b, g_b);
                const cudaError_t ce = cudaStreamEndCapture(st, &g);
                cudaGraphExec_t ex = nullptr;
                if (s == TLQ_OK && ce == cudaSuccess && g && cudaGraphInstantiate(&ex, g, 0) == cudaSuccess) {
                    pe->graph_exec = ex;
                    pe->graph_key = key;
                }
                if (g) cudaGraphDestroy(g);
            }
            cudaGetLastError();   // a failed capture leaves nothing behind: run uncaptured below
        }
        if (pe->graph_exec) {
            TLQ_CUDA(cudaGraphLaunch((cudaGraphExec_t)pe->graph_exec, st));
            launched = true;
        }
    }
    if (!launched) TLQ_TRY(sync_enqueue(ctx, c, h, B, prec, want_grad, st, th_b, e_b, g_b));
    TLQ_CUDA(cudaStreamSynchronize(st));
    const int32_t* h_err = (const int32_t*)(hp + th_b + e_b + g_b);
    if (*h_err != 0) {
        set_error("kernel error word " + std::to_string(*h_err));
        return TLQ_EKERNEL;
    }
    std::memcpy(energy, hp + th_b, e_b);
    if (want_grad) std::memcpy(grad, hp + th_b + e_b, (size_t)B * c->n_params * sizeof(double));
    return TLQ_OK;
}

tlq_status tlq_expectation(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B, tlq_precision prec,
                           double* energy) {
    return sync_call(ctx, c, h, theta, B, prec, energy, nullptr);
}

tlq_status tlq_expectation_grad(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B,
                                tlq_precision prec, double* energy, double* grad) {
    if (!grad) { set_error("grad is NULL"); return TLQ_EINVAL; }
    return sync_call(ctx, c, h, theta, B, prec, energy, grad);
}

tlq_status tlq_expectation_grad_dev(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev, int32_t B,
                                    tlq_precision prec, double* energy_dev, double* grad_dev, void* cuda_stream) {
    TLQ_TRY(check_pair(ctx, c, h, B, prec));
    if ((!theta_dev && c->n_params > 0) || !energy_dev) { set_error("NULL device pointer"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    const bool fp64 = prec == TLQ_FP64_REF;
    size_t work = 0;
    if (pe->plan->path == TLQ_PATH_CONE && ctx->cfg.fuse_k != 1) {
        TLQ_TRY(ensure_worklist(ctx, *pe, *c, B, fp64, grad_dev != nullptr));
        work = cone_workspace_bytes(*pe, *c, B, fp64, grad_dev != nullptr,
                                    global_grid(*pe, ctx->sm_count));
    } else if (pe->plan->dense) {
        work = dense_workspace_bytes(*pe, *c, B, grad_dev != nullptr, ctx->sm_count);
    }
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : (cudaStream_t)ctx->stream;
    if (ctx->ws.cap < work + 4096) {
        // the workspace is reallocated: make sure no earlier call on another stream still uses it
        TLQ_CUDA(cudaDeviceSynchronize());
    }
    TLQ_TRY(reserve(ctx, work + 4096));
    return run_device(ctx, c, h, theta_dev, B, prec, energy_dev, grad_dev, st, &ctx->ws);
}

// ---- reduced density operators ----------------------------------------------------------

// Validates keep[0..m) against n qubits and returns it sorted ascending.
static tlq_status check_keep(int n, const int32_t* keep, int32_t m, std::vector<int32_t>* sorted) {
    if (!keep) { set_error("keep is NULL"); return TLQ_EINVAL; }
    if (m < 1 || m > n) { set_error("m must be in [1, n]"); return TLQ_EINVAL; }
    if (m > kMaxDensityQubits) {
        set_error("at most " + std::to_string(kMaxDensityQubits) + " kept qubits");
        return TLQ_EINVAL;
    }
    sorted->assign(keep, keep + m);
    for (int32_t q : *sorted)
        if (q < 0 || q >= n) { set_error("kept qubit out of range"); return TLQ_EINVAL; }
    std::sort(sorted->begin(), sorted->end());
    for (int t = 1; t < m; ++t)
        if ((*sorted)[t] == (*sorted)[t - 1]) { set_error("kept qubit listed twice"); return TLQ_EINVAL; }
    return TLQ_OK;
}

// Kept / traced qubit lists of a state on n <= 31 qubits (keep validated and sorted).
static QubitMap keep_map(int n, const std::vector<int32_t>& keep) {
    QubitMap Q{};
    std::vector<char> in(n, 0);
    for (int32_t q : keep) in[q] = 1;
    int a = 0, b = 0;
    for (int q = 0; q < n && q < 32; ++q) {
        if (in[q]) Q.kept[a++] = q;
        else Q.traced[b++] = q;
    }
    return Q;
}

tlq_status tlq_partial_trace_dev(tlq_ctx ctx, const float* psi_dev, int32_t n, const int32_t* keep, int32_t m,
                                 float* rho_dev, void* cuda_stream) {
    if (!ctx) { set_error("NULL context"); return TLQ_EINVAL; }
    if (!psi_dev || !rho_dev) { set_error("NULL device pointer"); return TLQ_EINVAL; }
    if (n < 1 || n > kDenseMaxQubits) { set_error("n must be in [1, 31]"); return TLQ_EINVAL; }
    std::vector<int32_t> ks;
    TLQ_TRY(check_keep(n, keep, m, &ks));
    if (ctx->host_only()) { set_error("host-only context"); return TLQ_EUNSUPPORTED; }
    const QubitMap Q = keep_map(n, ks);
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    const size_t work = partial_trace_workspace_bytes(n, m, ctx->sm_count);
    if (ctx->ws.cap < work + 4096) TLQ_CUDA(cudaDeviceSynchronize());
    TLQ_TRY(reserve(ctx, work + 4096));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : (cudaStream_t)ctx->stream;
    if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[0], st));
    int nl = 0;
    const int rc = launch_partial_trace(psi_dev, n, Q, m, rho_dev, ctx->ws.take(work), ctx->sm_count, ctx->d_err, st, &nl);
    if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[1], st));
    ctx->last_launches = nl;
    if (rc != 0) {
        set_error(std::string("partial trace launch: ") + cudaGetErrorString((cudaError_t)rc));
        return TLQ_ECUDA;
    }
    return TLQ_OK;
}

tlq_status tlq_reduced_density(tlq_ctx ctx, tlq_circuit c, const double* theta, const int32_t* keep, int32_t m,
                               double* rho) {
    if (!ctx || !c) { set_error("NULL handle"); return TLQ_EINVAL; }
    if (!rho) { set_error("rho is NULL"); return TLQ_EINVAL; }
    if (!theta && c->n_params > 0) { set_error("theta is NULL"); return TLQ_EINVAL; }
    std::vector<int32_t> kq;
    TLQ_TRY(check_keep(c->n, keep, m, &kq));
    if (m > kMaxDensityQubits - 1) { set_error("at most 14 kept qubits through the host API"); return TLQ_EINVAL; }
    if (ctx->host_only()) { set_error("host-only context"); return TLQ_EUNSUPPORTED; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    // the state to trace: the whole circuit (n <= 31), or for a nearest-neighbour circuit the
    // window of the kept qubits' backward light cone, simulated from |0..0> on its own
    Circuit* src = c;
    std::unique_ptr<Circuit> sub;
    if (c->n > kDenseMaxQubits) {
        if (!c->nearest_neighbour) {
            set_error("reduced density of a non-local circuit on more than 31 qubits");
            return TLQ_EUNSUPPORTED;
        }
        int lo = 0, hi = 0;
        const std::vector<int> gates = light_cone_gates(*c, std::vector<int>(kq.begin(), kq.end()), &lo, &hi);
        if (hi - lo + 1 > kDenseMaxQubits) {
            set_error("light cone of the kept qubits wider than 31 qubits");
            return TLQ_EUNSUPPORTED;
        }
        sub.reset(new Circuit());
        sub->ctx = ctx;
        sub->n = hi - lo + 1;
        sub->n_params = c->n_params;
        for (int g : gates) {
            tlq_gate G = c->gates[g];
            G.q0 -= lo;
            if (G.q1 >= 0) G.q1 -= lo;
            sub->gates.push_back(G);
        }
        plan_circuit_layers(*sub);
        sub->id = ctx->next_id++;
        for (int32_t& q : kq) q -= lo;
        src = sub.get();
    }
    Ham empty;
    empty.ctx = ctx;
    empty.n = src->n;
    empty.id = 0;
    std::shared_ptr<PlanEntry> pe;
    tlq_status s = get_plan(ctx, src, &empty, &pe);
    auto drop_sub = [&]() { if (sub) evict_plans(ctx, sub->id, ~(uint64_t)0); };
    if (s != TLQ_OK) { drop_sub(); return s; }
    const DensePlan& D = *pe->plan->dense;
    const QubitMap Q = keep_map(D.n_eff, kq);
    const size_t P = (size_t)std::max(1, src->n_params);
    const size_t rho_b = ((size_t)8 << (2 * m));
    const size_t work = dense_workspace_bytes(*pe, *src, 1, false, ctx->sm_count) +
                        partial_trace_workspace_bytes(D.n_eff, m, ctx->sm_count) + P * 8 + 8 + rho_b + 8192;
    if ((s = reserve(ctx, work)) != TLQ_OK || (s = ensure_pinned(ctx, std::max(rho_b, P * 8) + 64)) != TLQ_OK) {
        drop_sub();
        return s;
    }
    cudaStream_t st = (cudaStream_t)ctx->stream;
    double* d_theta = (double*)ctx->ws.take(P * 8);
    double* d_e = (double*)ctx->ws.take(8);
    float* d_rho = (float*)ctx->ws.take(rho_b);
    char* hp = (char*)ctx->h_pinned;
    cudaError_t ce = cudaMemsetAsync(ctx->d_err, 0, sizeof(int32_t), st);
    if (ce == cudaSuccess && src->n_params > 0) {
        std::memcpy(hp, theta, (size_t)src->n_params * 8);
        ce = cudaMemcpyAsync(d_theta, hp, (size_t)src->n_params * 8, cudaMemcpyHostToDevice, st);
    }
    void* state = nullptr;
    if (ce == cudaSuccess)
        s = run_dense(ctx, *pe, *src, d_theta, 1, d_e, nullptr, ctx->cfg.fuse_k == 1 || !D.fits_fused, st, &ctx->ws,
                      &state);
    if (ce == cudaSuccess && s == TLQ_OK) {
        const size_t pt = partial_trace_workspace_bytes(D.n_eff, m, ctx->sm_count);
        int nl = 0;
        const int rc = launch_partial_trace(state, D.n_eff, Q, m, d_rho, ctx->ws.take(pt), ctx->sm_count, ctx->d_err, st, &nl);
        ce = (cudaError_t)rc;
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(hp, d_rho, rho_b, cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(hp + rho_b, ctx->d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    }
    drop_sub();
    if (s != TLQ_OK) return s;
    if (ce != cudaSuccess) { set_error(std::string("reduced density: ") + cudaGetErrorString(ce)); return TLQ_ECUDA; }
    int32_t kerr = 0;
    std::memcpy(&kerr, hp + rho_b, sizeof(int32_t));
    if (kerr != 0) { set_error("kernel error word " + std::to_string(kerr)); return TLQ_EKERNEL; }
    const float* f = (const float*)hp;
    const size_t entries = (size_t)2 << (2 * m);
    for (size_t e = 0; e < entries; ++e) rho[e] = (double)f[e];
    return TLQ_OK;
}

tlq_status tlq_plan_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* path, int32_t* lo, int32_t* w,
                         int32_t* ngates) {
    if (!ctx || !c || !h) { set_error("NULL handle"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    const Plan& P = *pe->plan;
    if (path) *path = P.path;
    if (P.path == TLQ_PATH_CONE) {
        for (size_t t = 0; t < P.cone_lo.size(); ++t) {
            if (lo) lo[t] = P.cone_lo[t];
            if (w) w[t] = P.cone_wtrue[t];
            if (ngates) ngates[t] = P.cone_gates[t];
        }
    }
    return TLQ_OK;
}

}  // extern "C"

extern "C" {

tlq_status tlq_plan_cone_stats(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* ncones, int32_t* nrot, int32_t* ndiag,
                               int32_t* npdiag, int32_t* weff, int32_t* wtrue, int32_t* nterms, int32_t* split) {
    if (!ctx || !c || !h) { set_error("NULL handle"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    const Plan& P = *pe->plan;
    if (P.path != TLQ_PATH_CONE) { set_error("not on the cone path"); return TLQ_EUNSUPPORTED; }
    if (ncones) *ncones = (int32_t)P.cones.size();
    for (size_t t = 0; t < P.cones.size(); ++t) {
        if (nrot) nrot[t] = P.cone_nrot[t];
        if (ndiag) ndiag[t] = P.cone_ndiag[t];
        if (npdiag) npdiag[t] = P.cone_npdiag[t];
        if (weff) weff[t] = P.cones[t].W;
        if (wtrue) wtrue[t] = P.group_wtrue[t];
        if (nterms) nterms[t] = P.cones[t].nmterms;
        if (split) split[t] = P.cones[t].split;
    }
    return TLQ_OK;
}

tlq_status tlq_plan_dense_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* n_eff, int32_t* n_passes,
                               int32_t* n_fwd_passes, int32_t* n_rev_store, int32_t* n_xterms, int32_t* fused) {
    if (!ctx || !c || !h) { set_error("NULL handle"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    if (!pe->plan->dense) { set_error("no dense statevector plan (more than 31 qubits)"); return TLQ_EUNSUPPORTED; }
    const DensePlan& D = *pe->plan->dense;
    if (n_eff) *n_eff = D.n_eff;
    if (n_passes) *n_passes = (int32_t)D.passes.size();
    if (n_fwd_passes) *n_fwd_passes = D.product_init ? (int32_t)D.fwd_passes.size() : (int32_t)D.passes.size();
    if (n_rev_store) {
        int32_t k = 0;
        for (int32_t v : D.rev_store) k += v;
        *n_rev_store = k;
    }
    if (n_xterms) *n_xterms = (int32_t)D.xterms.size();
    if (fused) *fused = D.fits_fused ? 1 : 0;
    return TLQ_OK;
}

tlq_status tlq_plan_dense_bytes(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int want_grad, tlq_precision prec,
                                double* bytes) {
    if (!ctx || !c || !h || !bytes) { set_error("NULL handle or out pointer"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    if (prec < TLQ_FP32 || prec > TLQ_FP64_REF) { set_error("unknown precision"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::shared_ptr<PlanEntry> pe;
    TLQ_TRY(get_plan(ctx, c, h, &pe));
    if (!pe->plan->dense) { set_error("no dense statevector plan (more than 31 qubits)"); return TLQ_EUNSUPPORTED; }
    const DensePlan& D = *pe->plan->dense;
    const double S = 8.0 * (double)(1ull << D.n_eff);
    const bool tc = prec == TLQ_MIXED_TC;
    const bool gen = D.product_init && D.gen_first && !tc;
    const std::vector<DensePassDev>& fwd = D.product_init ? D.fwd_passes : D.passes;
    const int nx = (int)D.xterms.size();
    double b = gen ? 0.0 : S;                              // the start state, written once
    for (size_t p = 0; p < fwd.size(); ++p) {
        if (!(gen && p == 0)) b += S;                      // read
        const bool last = p + 1 == fwd.size();
        if (want_grad || !last || nx > 0) b += S;          // write (not the last one of an energy)
    }
    b += nx * S;                                           // X/Y terms: one read each
    if (want_grad) {
        b += S;                                            // lam = (diagonal part of H) psi
        if (nx > 0) b += 3 * S;                            // lam += X/Y strings of psi
        for (size_t p = 0; p < D.passes.size(); ++p)      // reverse passes: read both, write both
            b += 2 * S + (D.rev_store[p] ? 2 * S : 0.0);
    }
    *bytes = b;
    return TLQ_OK;
}

tlq_status tlq_profile_enable(tlq_ctx ctx, int on) {
    if (!ctx) { set_error("NULL context"); return TLQ_EINVAL; }
    if (ctx->host_only()) { set_error("host-only context"); return TLQ_EUNSUPPORTED; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    if (on && !ctx->prof_ev[0]) {
        cudaEvent_t a, b;
        TLQ_CUDA(cudaEventCreate(&a));
        TLQ_CUDA(cudaEventCreate(&b));
        ctx->prof_ev[0] = a;
        ctx->prof_ev[1] = b;
    }
    ctx->profile = on != 0;
    return TLQ_OK;
}

tlq_status tlq_profile_last(tlq_ctx ctx, float* kernel_ms, int32_t* launches) {
    if (!ctx) { set_error("NULL context"); return TLQ_EINVAL; }
    if (!ctx->profile || !ctx->prof_ev[0]) { set_error("profiling is not enabled"); return TLQ_EINVAL; }
    TLQ_CUDA(cudaEventSynchronize((cudaEvent_t)ctx->prof_ev[1]));
    float ms = 0;
    TLQ_CUDA(cudaEventElapsedTime(&ms, (cudaEvent_t)ctx->prof_ev[0], (cudaEvent_t)ctx->prof_ev[1]));
    if (kernel_ms) *kernel_ms = ms;
    if (launches) *launches = ctx->last_launches;
    return TLQ_OK;
}

}  // extern "C"

// ---- exact MPS route ----------------------------------------------------------------------

namespace tlq {

// Cached MPS plan of (circuit, Hamiltonian); uploaded to the device when `upload`.
static tlq_status get_mps_plan(Context* ctx, Circuit* c, Ham* h, bool upload, std::shared_ptr<MpsPlan>* out) {
    auto key = std::make_pair(c->id, h->id);
    auto it = ctx->mps_plans.find(key);
    std::shared_ptr<MpsPlan> p;
    if (it != ctx->mps_plans.end()) {
        p = it->second;
    } else {
        std::string err;
        p = make_mps_plan(*c, *h, &err);
        if (!p) { set_error(err); return TLQ_EUNSUPPORTED; }
        ctx->mps_plans[key] = p;
    }
    if (upload) {
        size_t before = 0, after = 0;
        mps_info(*p, nullptr, nullptr, &before);
        const int rc = mps_upload(*p);
        if (rc != 0) {
            set_error(std::string("MPS plan upload: ") + cudaGetErrorString((cudaError_t)rc));
            return TLQ_ECUDA;
        }
        mps_info(*p, nullptr, nullptr, &after);
        ctx->held += after - before;
    }
    *out = p;
    return TLQ_OK;
}

// Launch on `st` with device buffers; the caller holds ctx->mu and has checked the arguments.
// `pre` bytes at the front of the workspace are the caller's (angles and results of the host
// call); the MPS buffers follow them.
static tlq_status mps_run(Context* ctx, Circuit* c, Ham* h, const double* theta_dev, int B, tlq_precision prec,
                          double* energy_dev, double* grad_dev, cudaStream_t st, size_t pre, void** pre_ptr,
                          const double* theta_host) {
    std::shared_ptr<MpsPlan> p;
    TLQ_TRY(get_mps_plan(ctx, c, h, true, &p));
    const bool fp64 = prec == TLQ_FP64_REF;
    std::string why;
    if (!mps_fits(*p, fp64, &why)) { set_error(why); return TLQ_EUNSUPPORTED; }
    if ((int64_t)c->n * B > INT32_MAX) { set_error("MPS route: n * B above 2^31"); return TLQ_EINVAL; }
    const size_t work = mps_workspace_bytes(*p, B, fp64);
    if (ctx->ws.cap < work + pre + 4096) TLQ_CUDA(cudaDeviceSynchronize());
    TLQ_TRY(reserve(ctx, work + pre + 4096));
    if (pre) {
        *pre_ptr = ctx->ws.take(pre);
        // host call: the angles are the first B * n_params doubles of the caller's block
        if (theta_host && c->n_params > 0)
            TLQ_CUDA(cudaMemcpyAsync(*pre_ptr, theta_host, (size_t)B * c->n_params * sizeof(double),
                                     cudaMemcpyHostToDevice, st));
        if (theta_host) theta_dev = (const double*)*pre_ptr;
        energy_dev = (double*)((char*)*pre_ptr + ((size_t)B * c->n_params * sizeof(double) + 255) / 256 * 256);
        if (grad_dev) grad_dev = energy_dev + ((size_t)B * sizeof(double) + 255) / 256 * 256 / sizeof(double);
    }
    void* w = ctx->ws.take(work);
    if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[0], st));
    int nl = 0;
    const int rc = launch_mps(*p, c->n_params > 0 ? theta_dev : nullptr, B, fp64, energy_dev, grad_dev, w, st, &nl);
    if (ctx->profile) TLQ_CUDA(cudaEventRecord((cudaEvent_t)ctx->prof_ev[1], st));
    ctx->last_launches = nl;
    if (rc != 0) {
        set_error(std::string("MPS launch: ") + cudaGetErrorString((cudaError_t)rc));
        return TLQ_ECUDA;
    }
    return TLQ_OK;
}

}  // namespace tlq

extern "C" {

tlq_status tlq_mps_expectation_grad_dev(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev, int32_t B,
                                        tlq_precision prec, double* energy_dev, double* grad_dev, void* cuda_stream) {
    TLQ_TRY(check_pair(ctx, c, h, B, prec));
    if ((!theta_dev && c->n_params > 0) || !energy_dev) { set_error("NULL device pointer"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : (cudaStream_t)ctx->stream;
    return mps_run(ctx, c, h, theta_dev, B, prec, energy_dev, grad_dev, st, 0, nullptr, nullptr);
}

tlq_status tlq_mps_expectation_grad(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B,
                                    tlq_precision prec, double* energy, double* grad) {
    TLQ_TRY(check_pair(ctx, c, h, B, prec));
    if (!theta && c->n_params > 0) { set_error("theta is NULL"); return TLQ_EINVAL; }
    if (!energy) { set_error("energy is NULL"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    TLQ_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)ctx->stream;
    const size_t P = (size_t)c->n_params;
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    // [angles | energies | gradients] at the front of the workspace
    const size_t pre = al(B * P * sizeof(double)) + al(B * sizeof(double)) + (grad ? al(B * P * sizeof(double)) : 0);
    void* blk = nullptr;
    double dummy = 0;
    TLQ_TRY(mps_run(ctx, c, h, nullptr, B, prec, &dummy, grad ? &dummy : nullptr, st, pre, &blk, theta));
    const double* d_e = (const double*)((const char*)blk + al(B * P * sizeof(double)));
    const double* d_g = d_e + al(B * sizeof(double)) / sizeof(double);
    TLQ_CUDA(cudaMemcpyAsync(energy, d_e, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (grad && P > 0) TLQ_CUDA(cudaMemcpyAsync(grad, d_g, B * P * sizeof(double), cudaMemcpyDeviceToHost, st));
    TLQ_CUDA(cudaStreamSynchronize(st));
    return TLQ_OK;
}

tlq_status tlq_plan_mps_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* max_bond_bits, int64_t* elems_per_set,
                             double* flops_energy, double* flops_grad) {
    if (!ctx || !c || !h) { set_error("NULL handle"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    std::lock_guard<std::mutex> lk(ctx->mu);
    std::shared_ptr<MpsPlan> p;
    TLQ_TRY(get_mps_plan(ctx, c, h, false, &p));
    int bits = 0;
    int64_t el = 0;
    mps_info(*p, &bits, &el, nullptr);
    if (max_bond_bits) *max_bond_bits = bits;
    if (elems_per_set) *elems_per_set = el;
    if (flops_energy) *flops_energy = mps_flops(*p, false);
    if (flops_grad) *flops_grad = mps_flops(*p, true);
    return TLQ_OK;
}

}  // extern "C"
