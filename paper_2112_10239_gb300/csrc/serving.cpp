// Serving loop: tlq_submit / tlq_poll with continuous batching.
//
// A scheduler thread per context takes submitted requests in arrival order and admits
// them while request slots (tlq_config.max_slots) and the device-memory budget allow.
// Admitted requests are packed into one batch: each parameter set becomes a record
// (SetRec) that points at its request's plan, angles and outputs, and the (cone, set)
// items of all requests are merged into one width-sorted work list, so requests of
// different n and depth share one persistent cone launch. Each batch owns one device
// buffer and one pinned host buffer (one H2D copy of the packed inputs, one D2H copy of
// the outputs). Two batch slots with their own streams let a new batch start while the
// previous one is still running, so work of requests that arrive while others are on the
// GPU overlaps on the device. A set's result does not depend on its batch: every cone is
// computed by the same code with the same team shape and fixed-order reductions.
//
// Plans are cached by circuit/Hamiltonian structure (gate kinds, qubits, parameter
// indices, term sites and letters -- not angles or coefficients), so repeated structures
// with new angles or fields skip planning.
#include "runtime.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <list>
#include <unordered_map>

namespace tlq {

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int kMaxBatchSets = 8192;

struct ServeRequest {
    tlq_ticket id = 0;
    Circuit* c = nullptr;                 // borrowed until the request completes
    Ham* h = nullptr;
    int B = 0;
    bool grad = false;
    bool fp64 = false;
    int n_params = 0;
    const double* theta = nullptr;
    double* energy = nullptr;
    double* grad_out = nullptr;
    std::shared_ptr<const Plan> plan;
    std::vector<tlq_gate> gates;          // copy (the circuit may be destroyed after completion)
    std::vector<double> term_coeff;
    size_t bytes = 0;                     // packed device bytes of this request
    double t_submit = 0, t_done = 0;
    tlq_status status = TLQ_OK;
    std::string err;
    bool done = false;
    // placement inside its batch
    size_t o_energy = 0, o_grad = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    void* dbuf = nullptr;
    size_t dcap = 0;
    unsigned char* hbuf = nullptr;
    size_t hcap = 0;
    std::vector<ServeRequest*> reqs;
    bool busy = false;
    size_t out_begin = 0, out_end = 0;    // output region (same offsets on host and device)
    size_t err_off = 0;
};

uint64_t mix64(uint64_t h, uint64_t v) {
    v *= 0x9e3779b97f4a7c15ull;
    v ^= v >> 29;
    h ^= v + 0x632be59bd9b4e019ull + (h << 7) + (h >> 3);
    return h;
}

// Structure key of a (circuit, Hamiltonian) pair: two independent 64-bit hashes.
std::pair<uint64_t, uint64_t> structure_key(const Circuit& c, const Ham& h) {
    uint64_t a = mix64(1, (uint64_t)c.n), b = mix64(7, (uint64_t)c.n_params);
    for (const tlq_gate& g : c.gates) {
        const uint64_t w = ((uint64_t)(uint32_t)g.kind << 48) ^ ((uint64_t)(uint32_t)g.q0 << 28) ^
                           ((uint64_t)(uint32_t)(g.q1 + 1) << 8) ^ (uint64_t)(uint32_t)(g.param + 1) * 0x100000001ull;
        a = mix64(a, w);
        b = mix64(b ^ 0x5555, w + 17);
    }
    for (const Term& t : h.terms) {
        a = mix64(a, 0xabcdefull + t.sites.size());
        for (size_t k = 0; k < t.sites.size(); ++k) {
            const uint64_t w = ((uint64_t)(uint32_t)t.sites[k] << 8) | (uint64_t)(unsigned char)t.letters[k];
            a = mix64(a, w);
            b = mix64(b, w * 31 + k);
        }
    }
    return {a, b ^ ((uint64_t)c.gates.size() << 32) ^ h.terms.size()};
}

struct PairHash {
    size_t operator()(const std::pair<uint64_t, uint64_t>& k) const { return (size_t)(k.first ^ (k.second * 3)); }
};

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct Scheduler {
    Context* ctx = nullptr;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServeRequest*> queue;        // planned, waiting for admission
    std::deque<ServeRequest*> plan_queue;   // submitted, waiting for a planner thread
    std::condition_variable cv_plan;
    std::vector<std::thread> planners;
    int planning = 0;
    std::unordered_map<tlq_ticket, ServeRequest*> all;
    uint64_t next_ticket = 1;
    bool stop = false;
    Slot slots[2];
    size_t bytes_in_flight = 0;
    int reqs_in_flight = 0;
    // structure-keyed plan cache (LRU)
    std::mutex plan_mu;
    std::list<std::pair<std::pair<uint64_t, uint64_t>, std::shared_ptr<const Plan>>> lru;
    std::unordered_map<std::pair<uint64_t, uint64_t>, decltype(lru)::iterator, PairHash> plan_index;
    // statistics
    std::vector<double> latencies;
    int64_t batches = 0, batched_requests = 0;

    std::shared_ptr<const Plan> plan_for(const Circuit& c, const Ham& h, std::string* err) {
        const auto key = structure_key(c, h);
        {
            std::lock_guard<std::mutex> lk(plan_mu);
            auto it = plan_index.find(key);
            if (it != plan_index.end()) {
                lru.splice(lru.begin(), lru, it->second);
                return it->second->second;
            }
        }
        std::shared_ptr<const Plan> p = make_plan(c, h, err);
        if (!p) return nullptr;
        std::lock_guard<std::mutex> lk(plan_mu);
        if (plan_index.find(key) == plan_index.end()) {
            lru.emplace_front(key, p);
            plan_index[key] = lru.begin();
            if (lru.size() > 2048) {
                plan_index.erase(lru.back().first);
                lru.pop_back();
            }
        }
        return p;
    }

    void run();
    void plan_loop();
    bool launch(Slot& s, std::vector<ServeRequest*>& batch);
    void finish(Slot& s);
    size_t request_bytes(const ServeRequest& r) const;
};

}  // namespace tlq

namespace tlq {

namespace {

size_t global_slot(int W, bool fp64, bool grad) {
    const size_t amps = ((size_t)1 << W) + ((size_t)1 << (W - 3));
    return al(amps * (fp64 ? 16 : 8) * (grad ? 2 : 1));
}

int smem_optin_dev(int device) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    return v > 2048 ? v - 1024 : 48 * 1024;
}

}  // namespace

size_t Scheduler::request_bytes(const ServeRequest& r) const {
    const Plan& P = *r.plan;
    const size_t G = r.gates.size(), T = P.term_coeff.size(), E = P.pmap_idx.size();
    const size_t r2 = r.fp64 ? 16 : 8;
    size_t s = 0;
    s += al(G * sizeof(tlq_gate)) + al(P.cones.size() * sizeof(ConeDev)) + al(P.meas.size() * sizeof(MeasDev)) +
         al(P.prog.size() * 4) + al(T * 8);
    s += al((P.pmap_off.size()) * 4) + 2 * al(std::max<size_t>(1, E) * 4);
    s += al((size_t)r.B * std::max(1, r.n_params) * 8);                      // theta
    s += (size_t)r.B * (sizeof(SetRec) + P.cones.size() * (16 + 2 * sizeof(ChunkDev)));   // records, items, chunks
    s += (size_t)r.B * 8 + (r.grad ? (size_t)r.B * r.n_params * 8 : 0);       // outputs
    s += al((size_t)r.B * std::max<size_t>(1, G) * r2) + al((size_t)r.B * T * 8);
    if (r.grad) s += al((size_t)r.B * std::max<int32_t>(1, P.n_slots) * 8);
    return s + 4096;
}

bool Scheduler::launch(Slot& sl, std::vector<ServeRequest*>& batch) {
    const bool fp64 = batch.front()->fp64;
    const size_t r2 = fp64 ? 16 : 8;
    int n_sets = 0, max_gates = 0, max_params = 0;
    for (ServeRequest* r : batch) {
        n_sets += r->B;
        max_gates = std::max(max_gates, (int)r->gates.size());
        max_params = std::max(max_params, r->n_params);
    }
    // ---- work list: (grad, tier, W desc) groups, chunked per width class ----
    const int smax = smem_optin_dev(ctx->device);
    std::vector<WorkItem> its[2];
    {
        int gs = 0;
        for (ServeRequest* r : batch) {
            const Plan& P = *r->plan;
            for (int b = 0; b < r->B; ++b, ++gs)
                for (size_t t = 0; t < P.cones.size(); ++t) push_cone_items(P, (int)t, gs, r->grad, its[r->grad ? 1 : 0]);
        }
    }
    std::vector<int32_t> items;
    std::vector<ChunkDev> chunks;
    BatchLaunch L;
    int g_maxW = 0;
    bool g_grad = false;
    int n_glob_max = 0;
    for (int gr = 0; gr < 2; ++gr) {
        ChunkSet cs;
        build_chunks(its[gr], fp64, gr == 1, smax, items, cs);
        L.smem_bytes[gr] = cs.smem_bytes;
        L.smem_threads[gr] = cs.smem_threads;
        L.gsmem_bytes[gr] = cs.gsmem_bytes;
        L.accum |= cs.accum;
        if (!cs.glob.empty()) {
            g_maxW = std::max(g_maxW, cs.g_maxW);
            g_grad |= gr == 1;
        }
        L.range[2 * gr] = (int32_t)chunks.size();
        chunks.insert(chunks.end(), cs.smem.begin(), cs.smem.end());
        L.range[2 * gr + 1] = (int32_t)chunks.size();
        chunks.insert(chunks.end(), cs.glob.begin(), cs.glob.end());
        n_glob_max = std::max(n_glob_max, (int)cs.glob.size());
    }
    L.range[4] = (int32_t)chunks.size();
    const int g_grid = std::min(n_glob_max, kGlobalCtasPerSm * ctx->sm_count);
    const size_t gslot = g_maxW > 0 ? global_slot(g_maxW, fp64, g_grad) : 0;

    // ---- layout ----
    size_t off = 0;
    auto take = [&](size_t bytes) { off = al(off); size_t o = off; off += bytes; return o; };
    const size_t o_sets = take((size_t)n_sets * sizeof(SetRec));
    const size_t o_items = take(items.size() * 4);
    const size_t o_chunks = take(chunks.size() * sizeof(ChunkDev));
    struct ROff { size_t gates, cones, meas, prog, tc, poff, pidx, pterm, theta; };
    std::vector<ROff> ro(batch.size());
    for (size_t i = 0; i < batch.size(); ++i) {
        const ServeRequest& r = *batch[i];
        const Plan& P = *r.plan;
        ro[i].gates = take(std::max<size_t>(1, r.gates.size()) * sizeof(tlq_gate));
        ro[i].cones = take(P.cones.size() * sizeof(ConeDev));
        ro[i].meas = take(P.meas.size() * sizeof(MeasDev));
        ro[i].prog = take(P.prog.size() * 4);
        ro[i].tc = take(r.term_coeff.size() * 8);
        ro[i].poff = take(P.pmap_off.size() * 4);
        ro[i].pidx = take(std::max<size_t>(1, P.pmap_idx.size()) * 4);
        ro[i].pterm = take(std::max<size_t>(1, P.pmap_term.size()) * 4);
        ro[i].theta = take((size_t)r.B * std::max(1, r.n_params) * 8);
    }
    const size_t in_end = off;
    const size_t out_begin = take(0);
    for (ServeRequest* r : batch) {
        r->o_energy = take((size_t)r->B * 8);
        r->o_grad = r->grad ? take((size_t)r->B * r->n_params * 8) : 0;
    }
    const size_t o_err = take(16);
    const size_t out_end = off;
    size_t gt_total = 0, e_total = 0, g_total = 0;
    for (ServeRequest* r : batch) {
        gt_total += (size_t)r->B * r->gates.size();
        e_total += (size_t)r->B * r->plan->term_coeff.size();
        if (r->grad) g_total += (size_t)r->B * r->plan->n_slots;
    }
    const size_t o_gt = take(std::max<size_t>(1, gt_total) * r2);
    const size_t o_e = take(std::max<size_t>(1, e_total) * 8);
    const size_t o_g = take(std::max<size_t>(1, g_total) * 8);
    const size_t o_cnt = take(64);
    const size_t o_gs = take((size_t)g_grid * gslot);
    const size_t total = al(off);

    // ---- buffers (grow only; the slot is idle here) ----
    if (sl.dcap < total) {
        if (sl.dbuf) cudaFree(sl.dbuf);
        sl.dbuf = nullptr;
        sl.dcap = 0;
        const size_t want = std::max(total, (size_t)64 << 20);
        if (cudaMalloc(&sl.dbuf, want) != cudaSuccess) return false;
        sl.dcap = want;
    }
    if (sl.hcap < out_end) {
        if (sl.hbuf) cudaFreeHost(sl.hbuf);
        sl.hbuf = nullptr;
        sl.hcap = 0;
        const size_t want = std::max(out_end, (size_t)16 << 20);
        if (cudaMallocHost((void**)&sl.hbuf, want) != cudaSuccess) return false;
        sl.hcap = want;
    }
    unsigned char* H = sl.hbuf;
    unsigned char* D = (unsigned char*)sl.dbuf;

    // ---- pack inputs ----
    SetRec* sets = (SetRec*)(H + o_sets);
    size_t gt = 0, e = 0, g = 0;
    int gs = 0;
    for (size_t i = 0; i < batch.size(); ++i) {
        const ServeRequest& r = *batch[i];
        const Plan& P = *r.plan;
        std::memcpy(H + ro[i].gates, r.gates.data(), r.gates.size() * sizeof(tlq_gate));
        std::memcpy(H + ro[i].cones, P.cones.data(), P.cones.size() * sizeof(ConeDev));
        std::memcpy(H + ro[i].meas, P.meas.data(), P.meas.size() * sizeof(MeasDev));
        std::memcpy(H + ro[i].prog, P.prog.data(), P.prog.size() * 4);
        std::memcpy(H + ro[i].tc, r.term_coeff.data(), r.term_coeff.size() * 8);
        std::memcpy(H + ro[i].poff, P.pmap_off.data(), P.pmap_off.size() * 4);
        std::memcpy(H + ro[i].pidx, P.pmap_idx.data(), P.pmap_idx.size() * 4);
        std::memcpy(H + ro[i].pterm, P.pmap_term.data(), P.pmap_term.size() * 4);
        if (r.n_params > 0) std::memcpy(H + ro[i].theta, r.theta, (size_t)r.B * r.n_params * 8);
        for (int b = 0; b < r.B; ++b, ++gs) {
            SetRec& R = sets[gs];
            R.cones = (const ConeDev*)(D + ro[i].cones);
            R.meas = (const MeasDev*)(D + ro[i].meas);
            R.prog = (const int32_t*)(D + ro[i].prog);
            R.gates = (const tlq_gate*)(D + ro[i].gates);
            R.theta = (const double*)(D + ro[i].theta) + (size_t)b * r.n_params;
            R.term_coeff = (const double*)(D + ro[i].tc);
            R.pmap_off = (const int32_t*)(D + ro[i].poff);
            R.pmap_idx = (const int32_t*)(D + ro[i].pidx);
            R.pmap_term = (const int32_t*)(D + ro[i].pterm);
            R.energy = (double*)(D + r.o_energy) + b;
            R.grad = r.grad ? (double*)(D + r.o_grad) + (size_t)b * r.n_params : nullptr;
            R.gt_off = (int64_t)gt;
            R.e_off = (int64_t)e;
            R.g_off = (int64_t)g;
            R.n_gates = (int32_t)r.gates.size();
            R.n_params = r.n_params;
            R.n_terms = (int32_t)P.term_coeff.size();
            R.n_slots = P.n_slots;
            gt += r.gates.size();
            e += P.term_coeff.size();
            if (r.grad) g += P.n_slots;
        }
    }
    std::memcpy(H + o_items, items.data(), items.size() * 4);
    std::memcpy(H + o_chunks, chunks.data(), chunks.size() * sizeof(ChunkDev));

    // ---- transfer, launch, read back ----
    cudaError_t ce = cudaMemcpyAsync(D, H, in_end, cudaMemcpyHostToDevice, sl.stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(D + o_err, 0, 16, sl.stream);
    if (ce != cudaSuccess) return false;
    L.sets = (const SetRec*)(D + o_sets);
    L.n_sets = n_sets;
    L.max_gates = max_gates;
    L.max_params = max_params;
    L.items = (const int32_t*)(D + o_items);
    L.chunks = (const ChunkDev*)(D + o_chunks);
    L.gate_table = D + o_gt;
    L.e_part = (double*)(D + o_e);
    L.g_part = (double*)(D + o_g);
    L.e_count = e_total;
    L.g_count = g_total;
    L.gscratch = g_grid > 0 ? D + o_gs : nullptr;
    L.gscratch_slot = gslot;
    L.g_grid = g_grid;
    L.counters = (int32_t*)(D + o_cnt);
    L.err = (int32_t*)(D + o_err);
    L.fp64 = fp64;
    L.sm_count = ctx->sm_count;
    if (launch_cone_batch(L, sl.stream) != 0) return false;
    ce = cudaMemcpyAsync(H + out_begin, D + out_begin, out_end - out_begin, cudaMemcpyDeviceToHost, sl.stream);
    if (ce == cudaSuccess) ce = cudaEventRecord(sl.ev, sl.stream);
    if (ce != cudaSuccess) return false;
    sl.out_begin = out_begin;
    sl.out_end = out_end;
    sl.err_off = o_err;
    sl.reqs = batch;
    sl.busy = true;
    return true;
}

void Scheduler::finish(Slot& sl) {
    const int32_t kerr = *(const int32_t*)(sl.hbuf + sl.err_off);
    const double t = now_s();
    for (ServeRequest* r : sl.reqs) {
        if (kerr != 0) {
            r->status = TLQ_EKERNEL;
            r->err = "kernel error word " + std::to_string(kerr);
        } else {
            std::memcpy(r->energy, sl.hbuf + r->o_energy, (size_t)r->B * 8);
            if (r->grad) std::memcpy(r->grad_out, sl.hbuf + r->o_grad, (size_t)r->B * r->n_params * 8);
        }
        r->t_done = t;
        r->done = true;
        latencies.push_back(t - r->t_submit);
        bytes_in_flight -= r->bytes;
        --reqs_in_flight;
    }
    ++batches;
    batched_requests += (int64_t)sl.reqs.size();
    sl.reqs.clear();
    sl.busy = false;
}

// Planner threads: plan (or fetch the cached plan of) each submitted request, copy what the
// batch needs, and hand it to the scheduler. Failures complete the request with an error.
void Scheduler::plan_loop() {
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_plan.wait(lk, [&] { return stop || !plan_queue.empty(); });
        if (plan_queue.empty()) {
            if (stop) break;
            continue;
        }
        ServeRequest* r = plan_queue.front();
        plan_queue.pop_front();
        ++planning;
        lk.unlock();
        std::string err;
        auto plan = plan_for(*r->c, *r->h, &err);
        tlq_status st = TLQ_OK;
        if (!plan) {
            st = TLQ_EUNSUPPORTED;
            r->err = "tlq_submit: " + err;
        } else if (plan->path != TLQ_PATH_CONE) {
            st = TLQ_EUNSUPPORTED;
            r->err = "tlq_submit: only nearest-neighbour circuits (the causal-cone path) are served; use tlq_expectation";
        } else {
            r->plan = plan;
            r->gates = r->c->gates;
            r->term_coeff.reserve(r->h->terms.size());
            for (const Term& t : r->h->terms) r->term_coeff.push_back(t.coeff);
            r->bytes = request_bytes(*r);
            if (r->bytes > ctx->budget / 2) {
                st = TLQ_ENOMEM;
                r->err = "tlq_submit: request needs " + std::to_string(r->bytes) + " bytes; a batch may hold " +
                         std::to_string(ctx->budget / 2);
            }
        }
        lk.lock();
        --planning;
        if (st != TLQ_OK) {
            r->status = st;
            r->done = true;
            cv_done.notify_all();
        } else {
            queue.push_back(r);
            cv_work.notify_one();
        }
    }
}

void Scheduler::run() {
    cudaSetDevice(ctx->device);
    for (Slot& s : slots) {
        cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking);
        cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    }
    const size_t slot_budget = ctx->budget / 2;
    const int max_slots = std::max(1, ctx->cfg.max_slots);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        for (Slot& s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.ev);
            if (q == cudaSuccess) {
                finish(s);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                for (ServeRequest* r : s.reqs) {
                    r->status = TLQ_ECUDA;
                    r->err = std::string("batch failed: ") + cudaGetErrorString(q);
                    r->done = true;
                    bytes_in_flight -= r->bytes;
                    --reqs_in_flight;
                }
                s.reqs.clear();
                s.busy = false;
                progressed = true;
            }
        }
        if (progressed) cv_done.notify_all();
        for (Slot& s : slots) {
            if (s.busy || queue.empty()) continue;
            std::vector<ServeRequest*> batch;
            size_t bytes = 0;
            int sets = 0;
            while (!queue.empty()) {
                ServeRequest* r = queue.front();
                if (!batch.empty() && r->fp64 != batch.front()->fp64) break;
                if (reqs_in_flight + (int)batch.size() + 1 > max_slots) break;
                if (bytes + r->bytes > slot_budget) break;
                if (sets + r->B > kMaxBatchSets && !batch.empty()) break;
                batch.push_back(r);
                bytes += r->bytes;
                sets += r->B;
                queue.pop_front();
            }
            if (batch.empty()) break;
            bytes_in_flight += bytes;
            reqs_in_flight += (int)batch.size();
            lk.unlock();
            const bool ok = launch(s, batch);
            lk.lock();
            if (!ok) {
                const cudaError_t e = cudaGetLastError();
                for (ServeRequest* r : batch) {
                    r->status = TLQ_ECUDA;
                    r->err = std::string("batch launch failed: ") + cudaGetErrorString(e);
                    r->done = true;
                    bytes_in_flight -= r->bytes;
                    --reqs_in_flight;
                }
                cv_done.notify_all();
            }
            progressed = true;
        }
        if (stop && queue.empty() && plan_queue.empty() && planning == 0 && !slots[0].busy && !slots[1].busy) break;
        if (!progressed) {
            if (slots[0].busy || slots[1].busy) {
                lk.unlock();
                std::this_thread::sleep_for(std::chrono::microseconds(20));
                lk.lock();
            } else {
                cv_work.wait(lk);
            }
        }
    }
    lk.unlock();
    for (Slot& s : slots) {
        if (s.dbuf) cudaFree(s.dbuf);
        if (s.hbuf) cudaFreeHost(s.hbuf);
        if (s.ev) cudaEventDestroy(s.ev);
        if (s.stream) cudaStreamDestroy(s.stream);
        s = Slot();
    }
}

void scheduler_stop(Context* ctx) {
    Scheduler* S = ctx->sched;
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_plan.notify_all();
    for (std::thread& t : S->planners)
        if (t.joinable()) t.join();
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (auto& kv : S->all) delete kv.second;
    for (ServeRequest* r : S->queue)
        if (S->all.find(r->id) == S->all.end()) delete r;
    delete S;
    ctx->sched = nullptr;
}

}  // namespace tlq

using namespace tlq;

extern "C" {

tlq_status tlq_submit(tlq_ctx ctx_h, tlq_circuit c_h, tlq_ham h_h, const double* theta, int32_t B, int want_grad,
                      tlq_precision prec, double* energy, double* grad, tlq_ticket* out) {
    Context* ctx = reinterpret_cast<Context*>(ctx_h);
    Circuit* c = reinterpret_cast<Circuit*>(c_h);
    Ham* h = reinterpret_cast<Ham*>(h_h);
    if (!ctx || !c || !h || !out) { set_error("tlq_submit: NULL argument"); return TLQ_EINVAL; }
    if (c->ctx != ctx || h->ctx != ctx) { set_error("tlq_submit: handle from another context"); return TLQ_EINVAL; }
    if (c->n != h->n) { set_error("tlq_submit: circuit and Hamiltonian qubit counts differ"); return TLQ_EINVAL; }
    if (B <= 0) { set_error("tlq_submit: B must be positive"); return TLQ_EINVAL; }
    if (B > kMaxBatchSets) { set_error("tlq_submit: B exceeds the batch limit of " + std::to_string(kMaxBatchSets)); return TLQ_ENOMEM; }
    if ((!theta && c->n_params > 0) || !energy || (want_grad && !grad)) { set_error("tlq_submit: NULL buffer"); return TLQ_EINVAL; }
    if (prec < TLQ_FP32 || prec > TLQ_FP64_REF) { set_error("tlq_submit: unknown precision"); return TLQ_EINVAL; }
    if (ctx->host_only()) { set_error("tlq_submit: host-only context"); return TLQ_EUNSUPPORTED; }
    Scheduler* S;
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        if (!ctx->sched) {
            ctx->sched = new Scheduler();
            ctx->sched->ctx = ctx;
            ctx->sched->th = std::thread([s = ctx->sched] { s->run(); });
            const unsigned hw = std::thread::hardware_concurrency();
            const int np = (int)std::max(1u, std::min(8u, hw / 2));
            for (int k = 0; k < np; ++k) ctx->sched->planners.emplace_back([s = ctx->sched] { s->plan_loop(); });
        }
        S = ctx->sched;
    }
    auto* r = new ServeRequest();
    r->c = c;
    r->h = h;
    r->B = B;
    r->grad = want_grad != 0;
    r->fp64 = prec == TLQ_FP64_REF;
    r->n_params = c->n_params;
    r->theta = theta;
    r->energy = energy;
    r->grad_out = want_grad ? grad : nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = S->next_ticket++;
        r->t_submit = std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
        S->all[r->id] = r;
        S->plan_queue.push_back(r);
        *out = r->id;
    }
    S->cv_plan.notify_one();
    return TLQ_OK;
}

tlq_status tlq_poll(tlq_ctx ctx_h, tlq_ticket t, int64_t timeout_us) {
    Context* ctx = reinterpret_cast<Context*>(ctx_h);
    if (!ctx) { set_error("tlq_poll: NULL context"); return TLQ_EINVAL; }
    Scheduler* S = ctx->sched;
    if (!S) { set_error("tlq_poll: unknown ticket"); return TLQ_EINVAL; }
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(t);
    if (it == S->all.end()) { set_error("tlq_poll: unknown or retired ticket"); return TLQ_EINVAL; }
    ServeRequest* r = it->second;
    if (!r->done) {
        if (timeout_us == 0) return TLQ_EAGAIN;
        if (timeout_us < 0) {
            S->cv_done.wait(lk, [&] { return r->done; });
        } else if (!S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return r->done; })) {
            return TLQ_ETIMEOUT;
        }
    }
    const tlq_status st = r->status;
    if (st != TLQ_OK) set_error(r->err);
    S->all.erase(it);
    delete r;
    return st;
}

tlq_status tlq_serving_stats(tlq_ctx ctx_h, int64_t* completed, double* p50_s, double* p99_s, double* mean_batch) {
    Context* ctx = reinterpret_cast<Context*>(ctx_h);
    if (!ctx) { set_error("tlq_serving_stats: NULL context"); return TLQ_EINVAL; }
    Scheduler* S = ctx->sched;
    std::vector<double> lat;
    int64_t nb = 0, nr = 0;
    if (S) {
        std::lock_guard<std::mutex> lk(S->mu);
        lat = S->latencies;
        nb = S->batches;
        nr = S->batched_requests;
    }
    std::sort(lat.begin(), lat.end());
    auto pct = [&](double q) {
        if (lat.empty()) return 0.0;
        size_t i = (size_t)std::ceil(q * (double)lat.size());
        if (i > 0) --i;
        return lat[std::min(i, lat.size() - 1)];
    };
    if (completed) *completed = (int64_t)lat.size();
    if (p50_s) *p50_s = pct(0.50);
    if (p99_s) *p99_s = pct(0.99);
    if (mean_batch) *mean_batch = nb ? (double)nr / (double)nb : 0.0;
    return TLQ_OK;
}

}  // extern "C"
