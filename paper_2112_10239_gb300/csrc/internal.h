// Internal structures shared by the host runtime (api.cpp, planner.cpp, serving.cpp)
// and the kernel launchers (cone.cu, dense.cu). Not part of the C-ABI.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <mutex>
#include <memory>
#include <map>

#include "tlq.h"

namespace tlq {

// ---------------------------------------------------------------------------------------
// Device-side plan records (plain old data, copied to the GPU as-is).
// ---------------------------------------------------------------------------------------

// One term's causal cone: a window of W qubits starting at chain site `lo` (window
// qubit j is chain qubit lo + j; qubits past the chain end are padding and stay |0>).
struct ConeDev {
    int32_t term;       // term index (row of the per-term energy buffer)
    int32_t W;          // effective window width (>= kMinConeW)
    int32_t prog_off;   // offset of the cone's program in the int32 program array
    int32_t slot_off;   // first gradient slot of this cone
    uint32_t flip;      // window-bit mask of X/Y letters
    uint32_t zy;        // window-bit mask of Y/Z letters (sign (-1)^bit)
    int32_t ny;         // number of Y letters: overall factor (-i)^ny
    int32_t nslots;     // gradient slots of this cone
};

// A chunk of work for one CTA: `count` (cone, set) items of equal width W starting at
// item `first`; the CTA splits into teams of `tt` threads, one item per team.
struct ChunkDev {
    int32_t W;
    int32_t first;
    int32_t count;
    int32_t tt;         // team size (threads)
    int32_t team_bytes; // dynamic shared memory per team
    int32_t pad[3];
};

// Program encoding (int32 words) of one cone:
//   [nlayers, off_0 .. off_{nlayers-1}, body]
// where body + off_l holds layer l (forward order): a header
//   [has_diag, live (window-bit mask of rotations), 0, 0]
// followed by one record of kRecWords words per window qubit j:
//   [rot_gate, rot_kind | (slot+1) << 8, rz_gate, rz_slot, pair_gate, pair_kind | (slot+1) << 8]
// rot_* is the layer's RX/RY on j, rz_* its RZ on j, pair_* its RZZ or CZ on (j, j+1);
// gate = -1 and slot = -1 mean absent / no parameter. Gates index the circuit's gate list.
constexpr int kRecWords = 6;
constexpr int kLayerHeader = 4;
constexpr int kMinConeW = 8;       // narrower cones are padded to this width
constexpr int kMaxSmemConeW = 13;  // widest cone kept in shared memory (FP32)
constexpr int kMaxConeW = 20;      // widest cone on the cone path (global-memory tier)
constexpr int kCtaThreads = 512;
constexpr int kMaxPassSlots = 4 + 2 * 20;  // gradient values per adjoint pass: 4 rotations + RZ/pair per qubit

// ---------------------------------------------------------------------------------------
// Host-side objects.
// ---------------------------------------------------------------------------------------

struct Context;

struct Circuit {
    Context* ctx = nullptr;
    int n = 0;
    int n_params = 0;
    std::vector<tlq_gate> gates;
    // Layer structure: layers[l] = (rotation gates, diagonal gates), leading diagonal
    // gates (acting on |0...0>, a global phase) dropped.
    struct Layer { std::vector<int> rot, diag; };
    std::vector<Layer> layers;
    bool nearest_neighbour = true;   // every two-qubit gate acts on (q, q+1)
    uint64_t id = 0;
};

struct Term {
    double coeff;
    std::vector<int> sites;
    std::string letters;
};

struct Ham {
    Context* ctx = nullptr;
    int n = 0;
    std::vector<Term> terms;
    uint64_t id = 0;
};

// Result of planning one (circuit, Hamiltonian) pair; cached on the context.
struct Plan {
    tlq_path path = TLQ_PATH_CONE;
    // cone path
    std::vector<ConeDev> cones;           // one per term
    std::vector<int32_t> prog;            // programs of all cones
    std::vector<int32_t> cone_gates;      // gates in each cone (introspection)
    std::vector<int32_t> cone_lo;         // window start per term
    std::vector<int32_t> cone_wtrue;      // true (unpadded, clipped) width per term
    std::vector<int32_t> cone_nrot;       // rotations in each cone
    std::vector<int32_t> cone_ndiag;      // layers with diagonal gates in each cone
    std::vector<int32_t> cone_npdiag;     // parametrised diagonal gates in each cone
    int32_t n_slots = 0;                  // gradient slots per parameter set
    // slot -> parameter map, CSR by parameter: g[p] = sum_i coeff[i] * part[idx[i]]
    std::vector<int32_t> pmap_off;        // n_params + 1
    std::vector<int32_t> pmap_idx;
    std::vector<double> pmap_coeff;
    std::vector<double> term_coeff;       // per term
    int max_w = 0;
    std::string why_dense;                // reason the dense path was chosen
};

std::string plan_circuit_layers(Circuit& c);   // fills c.layers; returns "" or error
std::shared_ptr<Plan> make_plan(const Circuit& c, const Ham& h, std::string* err);

// ---------------------------------------------------------------------------------------
// Kernel launchers (cone.cu / dense.cu). All return cudaError_t as int (0 = success).
// ---------------------------------------------------------------------------------------

struct DevPlan;   // device copy of a Plan (owned by the context cache)

struct ConeLaunch {
    // device pointers
    const ConeDev* cones = nullptr;
    const int32_t* prog = nullptr;
    const double* term_coeff = nullptr;
    const int32_t* pmap_off = nullptr;
    const int32_t* pmap_idx = nullptr;
    const double* pmap_coeff = nullptr;
    const tlq_gate* gates = nullptr;      // circuit gate list on the device
    int32_t n_gates = 0;
    int32_t n_params = 0;
    int32_t n_terms = 0;
    int32_t n_slots = 0;
    int32_t B = 0;
    const double* theta = nullptr;        // [B][n_params]
    // work list
    const int32_t* items = nullptr;       // [2 * n_items]: (cone, set)
    const ChunkDev* chunks = nullptr;
    int32_t n_chunks_smem = 0;            // chunks [0, n_chunks_smem) use shared memory
    int32_t n_chunks = 0;                 // chunks [n_chunks_smem, n_chunks) use global memory
    int32_t smem_bytes = 0;               // dynamic shared memory for the shared tier
    int32_t gsmem_bytes = 0;              // dynamic shared memory for the global tier
    int32_t g_maxW = 0;                   // widest cone of the global tier
    // workspace
    void* gate_table = nullptr;           // [B][n_gates] real2
    double* e_part = nullptr;             // [B][n_terms]
    double* g_part = nullptr;             // [B][n_slots]
    void* gscratch = nullptr;             // global-tier states
    size_t gscratch_slot = 0;             // bytes per CTA slot
    int32_t g_grid = 0;                   // CTAs of the global-tier launch
    int32_t* counters = nullptr;          // [2] work counters (zeroed by the launcher)
    int32_t* err = nullptr;               // kernel error word
    // outputs
    double* energy = nullptr;             // [B]
    double* grad = nullptr;               // [B][n_params] or null
    bool fp64 = false;
    int sm_count = 0;
    void* ev_begin = nullptr;             // optional cudaEvent_t pair around the cone kernels
    void* ev_end = nullptr;
    int launches = 0;                     // out: kernels launched
};

int launch_cone(ConeLaunch& L, void* stream);
int cone_smem_grid(bool fp64, bool grad, int smem_bytes, int sm_count);

struct DenseLaunch {
    int n = 0;
    const int32_t* prog = nullptr;        // dense layer program (device)
    int32_t prog_len = 0;
    const tlq_gate* gates = nullptr;
    int32_t n_gates = 0, n_params = 0, B = 0;
    const double* theta = nullptr;
    const int32_t* term_desc = nullptr;   // per term: flip, zy, ny (int32 x4)
    const double* term_coeff = nullptr;
    int32_t n_terms = 0;
    void* gate_table = nullptr;
    void* state = nullptr;                // 2^n real2
    double* partial = nullptr;            // reduction scratch
    int32_t* err = nullptr;
    double* energy = nullptr;
    bool fp64 = false;
    bool per_gate = false;                // plain per-gate sweeps (baseline)
    int sm_count = 0;
};

int launch_dense(const DenseLaunch& L, void* stream);

}  // namespace tlq
