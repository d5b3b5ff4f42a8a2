// Host runtime objects behind the C-ABI (context, device plan cache, workspace).
#pragma once

#include "internal.h"

#include <atomic>
#include <condition_variable>
#include <deque>
#include <thread>
#include <unordered_map>

namespace tlq {

void set_error(const std::string& msg);
const char* get_error();

// Device copy of a Plan plus the work list for the last batch size used.
struct PlanEntry {
    std::shared_ptr<Plan> plan;
    uint64_t circ_id = 0, ham_id = 0;
    // cone path device buffers
    ConeDev* d_cones = nullptr;
    MeasDev* d_meas = nullptr;
    int32_t* d_prog = nullptr;
    double* d_term_coeff = nullptr;
    int32_t* d_pmap_off = nullptr;
    int32_t* d_pmap_idx = nullptr;
    int32_t* d_pmap_term = nullptr;
    tlq_gate* d_gates = nullptr;
    // dense path device buffers
    DenseLayerDev* d_dlayers = nullptr;
    DenseClassDev* d_dclasses = nullptr;
    DensePassClassDev* d_dpcd = nullptr;
    int32_t* d_dstage = nullptr;
    int32_t* d_ddists = nullptr;
    DenseZTermDev* d_dzterms = nullptr;
    int32_t* d_dtab_gate = nullptr;
    int32_t* d_dtab_mult = nullptr;
    DenseXTermDev* d_dxterms = nullptr;
    DenseXTermDev* d_dallterms = nullptr;
    tlq_gate* d_dfgates = nullptr;           // DensePlan::fgates (rotation frame of the fused passes)
    DenseXTermDev* d_dfxterms = nullptr;     // DensePlan::fxterms
    int32_t* d_dadj_off = nullptr;
    int32_t* d_dadj_idx = nullptr;
    DensePassClassDev* d_dinit_pcd = nullptr;
    // work list cache (keyed by batch size and precision)
    int wl_B = -1;
    bool wl_fp64 = false;
    bool wl_grad = false;
    int32_t* d_items = nullptr;
    ChunkDev* d_chunks = nullptr;
    int n_chunks_smem = 0, n_chunks = 0;
    int smem_bytes = 0, gsmem_bytes = 0, g_maxW = 0;
    int smem_threads = 512;   // CTA size of the shared tier
    bool accum = false;       // branch items: the launcher zeroes the partial sums
    size_t device_bytes = 0;
    // CUDA graph of the synchronous call's device work (input copy, kernels, output copies),
    // replayed while the key below is unchanged; see sync_call in api.cpp
    void* graph_exec = nullptr;   // cudaGraphExec_t
    struct GraphKey {
        int B = -1, prec = -1, grad = -1, fuse_k = -1;
        void* ws_base = nullptr;
        size_t ws_cap = 0;
        void* pinned = nullptr;
        size_t pinned_cap = 0;
        bool operator==(const GraphKey& o) const {
            return B == o.B && prec == o.prec && grad == o.grad && fuse_k == o.fuse_k && ws_base == o.ws_base &&
                   ws_cap == o.ws_cap && pinned == o.pinned && pinned_cap == o.pinned_cap;
        }
    } graph_key;
    ~PlanEntry();
};

struct Workspace {
    void* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    void* take(size_t bytes) {
        used = (used + 255) & ~(size_t)255;
        void* p = (char*)base + used;
        used += bytes;
        return p;
    }
};


struct Scheduler;

struct Context {
    int device = -1;
    tlq_config cfg{};
    void* stream = nullptr;          // cudaStream_t
    int sm_count = 0;
    size_t budget = 0;
    size_t held = 0;                 // bytes currently held (plans + workspace)
    Workspace ws;
    int32_t* d_counters = nullptr;   // [2]
    int32_t* d_err = nullptr;        // kernel error word
    void* h_pinned = nullptr;        // pinned staging
    size_t h_pinned_cap = 0;
    std::mutex mu;                   // guards the plan cache and workspace
    std::map<std::pair<uint64_t, uint64_t>, std::shared_ptr<PlanEntry>> plans;
    std::map<std::pair<uint64_t, uint64_t>, std::shared_ptr<MpsPlan>> mps_plans;   // exact MPS route
    std::vector<Circuit*> circuits;
    std::vector<Ham*> hams;
    std::atomic<uint64_t> next_id{1};
    Scheduler* sched = nullptr;
    bool profile = false;            // record events around the dominant kernel
    void* prof_ev[2] = {nullptr, nullptr};
    int last_launches = 0;
    bool host_only() const { return device < 0; }
};

// Prepared launch of one (circuit, Hamiltonian, batch) on the cone path.
tlq_status get_plan(Context* ctx, Circuit* c, Ham* h, std::shared_ptr<PlanEntry>* out);
tlq_status ensure_worklist(Context* ctx, PlanEntry& pe, const Circuit& c, int B, bool fp64, bool grad);
// Bytes of workspace a launch needs (excluding the work list).
size_t cone_workspace_bytes(const PlanEntry& pe, const Circuit& c, int B, bool fp64, bool grad, int g_grid);
tlq_status run_device(Context* ctx, Circuit* c, Ham* h, const double* theta_dev, int B, tlq_precision prec,
                      double* energy_dev, double* grad_dev, void* stream, Workspace* ws);

void scheduler_stop(Context* ctx);
// Drops the allocation-free entry point's cached host plans of a context (noalloc.cu).
void noalloc_forget(const Context* ctx);

}  // namespace tlq
