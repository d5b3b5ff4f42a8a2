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
// One cone of work: a window shared by one or more terms (a term whose own causal cone fits
// inside another term's window is measured on that window).
struct ConeDev {
    int32_t W;          // effective window width (>= kMinConeW)
    int32_t prog_off;   // offset of the cone's program in the int32 program array
    int32_t slot_off;   // first gradient slot of this cone
    int32_t nslots;     // gradient slots of this cone
    int32_t mterm_off;  // first of this cone's measured terms in the MeasDev array
    int32_t nmterms;    // terms measured on this window
    int32_t split;      // 1: run as two branches of W - 1 qubits (the top qubit has gates of
                        // layer 0 only and no measured term); 0: one item of W qubits
    int32_t pad;
};

// Work-list items are (cone word, set) pairs; the cone word carries the branch:
// cone | half << kItemHalfShift, half 0 = the whole window, 1 / 2 = top bit 0 / 1.
constexpr int kItemHalfShift = 28;
constexpr int32_t kItemConeMask = (1 << kItemHalfShift) - 1;
constexpr int kSplitMinW = 13;     // windows at least this wide are split when they can be

// A term measured on a cone's window: P = (-i)^ny (-1)^popc(x & zy) X^flip.
struct MeasDev {
    int32_t term;       // term index (row of the per-term energy buffer, coefficient index)
    uint32_t flip;      // window-bit mask of X/Y letters
    uint32_t zy;        // window-bit mask of Y/Z letters (sign (-1)^bit)
    int32_t ny;         // number of Y letters
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
constexpr int kMaxGroupTerms = 16; // terms measured on one shared window
constexpr int kMaxSmemConeW = 14;  // widest cone kept in shared memory (when it fits: FP32 forward at 14)
constexpr int kMaxConeW = 20;      // widest cone on the cone path (global-memory tier)
constexpr int kCtaThreads = 512;
// Global-memory tier: one window per CTA of kGlobalCtaThreads, kGlobalCtasPerSm CTAs per SM,
// each with its own state slot in HBM/L2. (Two 256-thread CTAs per SM measured 9 % slower on
// 15- and 17-qubit windows than one 512-thread CTA: twice the blocks per thread per pass.)
constexpr int kGlobalCtaThreads = 512;
constexpr int kGlobalCtasPerSm = 1;
constexpr int kMaxPassSlots = 4 + 2 * 20;  // gradient values per adjoint pass: 4 rotations + RZ/pair per qubit

// Dense statevector path (circuits with non-adjacent two-qubit gates): the 2^n state lives
// in HBM and is processed in passes over tiles of 2^12 amplitudes (256 threads; two CTAs
// share an SM). A "low" tile is 2^12 contiguous amplitudes (qubits 0..11); a "strided" tile
// keeps qubits 0..3 (16 contiguous amplitudes, 128 bytes) and 8 higher qubits a..a+7.
// Inside a tile, rotations run as 16-amplitude register passes; the diagonal gates of a
// layer are grouped into angle classes and applied from a phase table indexed by a popcount.
constexpr int kDenseTileBits = 12;
constexpr int kDenseStridedBits = 8;
constexpr int kDenseMaxQubits = 31;
constexpr int kDenseMaxLayerClasses = 48;  // per layer (+ energy classes)
constexpr int kDenseMaxDistWords = 512;
constexpr int kDenseMaxTab = 768;

constexpr int kDenseMaxGroups = 8;
// Gradient slots of one adjoint pass: 4 rotations per register group, then one per staged class.
constexpr int kDenseAdjSlots = 4 * kDenseMaxGroups + kDenseMaxLayerClasses;

// One streaming pass over all tiles. Its register passes ("groups") may span a layer
// boundary: the group that completes a layer's rotations is followed by that layer's
// diagonal, and later groups already apply the next layer's rotations on this tile's qubits.
struct DensePassDev {
    int32_t strided;                      // 0: low tile, 1: strided tile
    int32_t a;                            // strided: global qubit of local bit 4
    int32_t ngroups;
    int32_t store;                        // write the tile back (0: read-only measurement pass)
    int32_t nstage;                       // classes staged in shared memory for this pass
    int32_t stage_off;                    // their indices in DensePlan::stage
    int32_t measure_group;                // group after which the energy is accumulated (-1 none)
    uint32_t group_rot0;                  // bit g: group g rotates layer 0 (the adjoint needs only
                                          // their gradients: nothing after them uses the state)
    int32_t group_s[kDenseMaxGroups];     // local start bit of each register pass
    uint32_t group_mask[kDenseMaxGroups]; // register bits carrying a rotation
    int32_t group_cls[kDenseMaxGroups];   // first staged class evaluated after the group's rotations
    int32_t group_ncls[kDenseMaxGroups];  // how many (diagonal phases and/or energy classes)
    int32_t group_pcd[kDenseMaxGroups];   // first DensePassClassDev of those classes
    int32_t gate[kDenseMaxGroups][4];     // rotation gate per register bit (-1 none)
};

// Per pass and class, the split of the class's count over the last register pass: with x_b
// the thread's base index (the 4 register bits zero) and j the register bits,
//   count(x_b | j) = count(x_b) + sum_k j_k A_k + C[j],
// A_k = popc(N_k) - 2 popc(x_b & N_k) + single_k (XOR counts) or popc(x_b & N_k) (AND counts),
// N_k = partners outside the register bits of register bit k, C[j] = count of the pairs inside.
struct DensePassClassDev {
    uint32_t N[4];
    uint32_t single;          // bit k: register bit k carries a single-qubit term
    uint32_t C[4];            // C[j] in byte j % 4 of word j / 4
    uint32_t pad[3];
};

// A class of diagonal terms counted by popcounts over distance masks:
//   kind 0: RZ/RZZ gates sharing one angle; phase exp(-i a/2 (N - 2 c)), c = sum_d popc((x ^ x>>d) & M_d)
//           + popc(x & single), looked up in a table of N+1 entries at tab_off;
//   kind 1: CZ gates; sign (-1)^c with c = sum_d popc((x & x>>d) & M_d);
//   kind 2: Z / ZZ energy terms sharing one coefficient; energy coeff * (N - 2 c) per amplitude.
struct DenseClassDev {
    int32_t kind;
    int32_t gate;
    int32_t nterms;
    int32_t ndist;
    int32_t dist_off;         // (d, mask) pairs in the distance array
    int32_t tab_off;
    uint32_t single;
    int32_t ew;               // a pass's staged copy: its edge-word table in shared memory (-1: none)
    double coeff;
};
struct DenseLayerDev { int32_t nclass, class_off, pad0, pad1; };
struct DenseXTermDev { uint32_t flip, zy; int32_t ny, pad; double coeff; };   // terms with X/Y letters
struct DenseZTermDev { uint32_t mask; int32_t pad; double coeff; };           // Z strings of 3+ sites

struct DensePlan {
    int n_eff = 0;                          // qubits of the state (>= kDenseTileBits; extra qubits stay |0>)
    std::vector<DensePassDev> passes;
    std::vector<DenseLayerDev> layers;
    std::vector<DenseClassDev> classes;     // diagonal-layer classes, then energy classes
    std::vector<int32_t> dists;             // (d, mask) pairs
    int32_t energy_class_off = 0, energy_nclass = 0;
    std::vector<DenseZTermDev> zterms;
    std::vector<DenseXTermDev> xterms;
    std::vector<int32_t> tab_gate;          // per phase-table entry: gate providing the angle
    std::vector<int32_t> tab_mult;          // per entry: N - 2c
    std::vector<DenseXTermDev> all_terms;   // every term (plain per-gate path measures them one by one)
    std::vector<DensePassClassDev> pcd;     // per (pass, group, class): split counts
    std::vector<int32_t> stage;             // per pass: classes staged in shared memory
    // Product-state start (two or more layers): the forward writes layer 0's result directly --
    // the init_gate rotations (per qubit, -1 none) on |0..0> times layer 0's diagonal classes
    // [init_class_off, +init_nclass) with split counts init_pcd over bits 0..3 -- and then runs
    // fwd_passes (layers 1..); the adjoint walks `passes` (all layers) in reverse.
    bool product_init = false;
    std::vector<DensePassDev> fwd_passes;
    // per pass of `passes`: 1 when its reverse (adjoint) pass writes psi and lambda back -- not
    // the first pass, nor a pass that only gives layer 0's rotation gradients
    std::vector<int32_t> rev_store;
    std::vector<int32_t> init_gate;
    int32_t init_class_off = 0, init_nclass = 0;
    std::vector<DensePassClassDev> init_pcd;
    // adjoint: for parameter p, entries adj_idx[adj_off[p] .. adj_off[p+1]) are the
    // (pass * kDenseAdjSlots + slot) gradient slots that carry it, in a fixed order
    std::vector<int32_t> adj_off;
    std::vector<int32_t> adj_idx;
    int max_classes_per_layer = 0;
    int max_dists = 0;
    bool fits_fused = true;                 // staged class data fits the pass kernel's shared memory
    // Rotation frame of the fused passes. On a qubit whose rotations are all RX the passes carry
    // psi' = S psi with S = diag(1, i) on that qubit: S RX(a) S^dagger = RY(a), S commutes with
    // every diagonal gate and S|0> = |0>, so the RX gates run as the real RY form and only the
    // X/Y letters of the measured terms change (S X S^dagger = Y, S Y S^dagger = -X).
    // The first forward pass generates layer 0's product state in registers instead of reading
    // a start state written by a separate kernel (a low tile whose first group starts at bit 0).
    bool gen_first = false;
    uint32_t frame_mask = 0;                // qubits carried in the rotated frame
    std::vector<tlq_gate> fgates;           // the circuit's gates with RX -> RY on those qubits
    std::vector<DenseXTermDev> fxterms;     // xterms with the letters converted on those qubits
};

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
    std::vector<ConeDev> cones;           // one per term group (shared window)
    std::vector<MeasDev> meas;            // measured terms of all cones
    std::vector<int32_t> group_wtrue;     // true width of each group's window
    std::vector<int32_t> prog;            // programs of all cones
    std::vector<int32_t> cone_gates;      // gates in each cone (introspection)
    std::vector<int32_t> cone_lo;         // window start per term
    std::vector<int32_t> cone_wtrue;      // true (unpadded, clipped) width per term
    std::vector<int32_t> cone_nrot;       // rotations in each group cone
    std::vector<int32_t> cone_ndiag;      // layers with diagonal gates in each group cone
    std::vector<int32_t> cone_npdiag;     // parametrised diagonal gates in each group cone
    int32_t n_slots = 0;                  // gradient slots per parameter set
    // slot -> parameter map, CSR by parameter: g[p] = sum_i part[idx[i]] (the term coefficients are
    // folded into the adjoint's lambda; term[i] = -1)
    std::vector<int32_t> pmap_off;        // n_params + 1
    std::vector<int32_t> pmap_idx;
    std::vector<int32_t> pmap_term;       // term owning each entry (its coefficient scales the slot)
    std::vector<double> term_coeff;       // per term
    int max_w = 0;
    std::string why_dense;                // reason the dense path was chosen
    std::shared_ptr<DensePlan> dense;     // dense statevector plan (when n <= kDenseMaxQubits)
};

std::shared_ptr<DensePlan> make_dense_plan(const Circuit& c, const Ham& h, std::string* err);

std::string plan_circuit_layers(Circuit& c);   // fills c.layers; returns "" or error
std::shared_ptr<Plan> make_plan(const Circuit& c, const Ham& h, std::string* err);

// ---------------------------------------------------------------------------------------
// Kernel launchers (cone.cu / dense.cu). All return cudaError_t as int (0 = success).
// ---------------------------------------------------------------------------------------

struct DevPlan;   // device copy of a Plan (owned by the context cache)

struct ConeLaunch {
    // device pointers
    const ConeDev* cones = nullptr;
    const MeasDev* meas = nullptr;
    const int32_t* prog = nullptr;
    const double* term_coeff = nullptr;
    const int32_t* pmap_off = nullptr;
    const int32_t* pmap_idx = nullptr;
    const int32_t* pmap_term = nullptr;
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
    int32_t smem_threads = kCtaThreads;   // CTA size of the shared tier
    int32_t gsmem_bytes = 0;              // dynamic shared memory for the global tier
    int32_t g_maxW = 0;                   // widest cone of the global tier
    bool accum = false;                   // branch items: partial energies and slots are added
                                          // (zeroed by the launcher)
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

// ---- small circuits (tiny.cu) ----
// Energies of circuits of at most kTinyMaxQubits qubits: one CTA per parameter set holds the
// whole state in shared memory and applies the gates in circuit order (FP32), then measures
// every term (terms as in DensePlan::all_terms) and sums them in FP64 in term order.
constexpr int kTinyMaxQubits = 10;
bool tiny_fits(int n, int n_gates, int n_terms);
int launch_tiny_energy(const tlq_gate* gates, int n_gates, const double* theta, int n_params, int n,
                       const DenseXTermDev* terms, int n_terms, int B, double* energy, void* stream);

// ---- exact matrix-product states (mps.cu) ----
// Chain circuits (every two-qubit gate on neighbours q, q+1) as an exact MPS: each two-qubit
// gate splits into a sum of two products of single-site operators, so the bond between q and
// q+1 carries one bit per gate on that pair (bond dimension 2^gates, no truncation).
constexpr int kMpsMaxBondBitsF32 = 6;     // bond dimension <= 64 in FP32
constexpr int kMpsMaxBondBitsF64 = 5;     // <= 32 in FP64
constexpr int kMpsMaxSiteOps = 48;        // operators on one site (gates touching the qubit)
struct MpsPlan;                           // host + device plan (mps.cu)
// Plans a (circuit, Hamiltonian) pair on the host; nullptr with *err set when the circuit is
// not a chain circuit or exceeds the limits above.
std::shared_ptr<MpsPlan> make_mps_plan(const Circuit& c, const Ham& h, std::string* err);
// Uploads the plan's tables (once); 0 or a cudaError_t.
int mps_upload(MpsPlan& p);
void mps_info(const MpsPlan& p, int* max_bond_bits, int64_t* elems_per_set, size_t* device_bytes);
// Contraction flops per parameter set of one call (energies, or energies and gradients).
double mps_flops(const MpsPlan& p, bool grad);
size_t mps_workspace_bytes(const MpsPlan& p, int B, bool fp64);
// Whether the plan runs in the given precision (bond limit, shared-memory fit); *why otherwise.
bool mps_fits(const MpsPlan& p, bool fp64, std::string* why);
// Energies (and gradients when grad != nullptr) of B parameter sets; theta, energy and grad
// are device pointers, work a workspace of mps_workspace_bytes. 0 or a cudaError_t.
int launch_mps(const MpsPlan& p, const double* theta, int B, bool fp64, double* energy, double* grad,
               void* work, void* stream, int* launches);

// ---- work lists (planner.cpp) ----
// One work item before chunking: the cone word (cone | half << kItemHalfShift), the set, the
// state width W, the window width Wt (W + 1 for a branch) and the estimated amplitude visits.
struct WorkItem {
    int32_t cone, set, W, Wt;
    double work;
};
// Chunks of one launch group (shared and global tier) and what their launches need.
struct ChunkSet {
    std::vector<ChunkDev> smem, glob;
    int smem_bytes = 0, smem_threads = kCtaThreads, gsmem_bytes = 0, g_maxW = 0;
    bool accum = false;   // branch items present
};
// Amplitude visits of one (cone, set) item as the cone kernel schedules its register passes:
// the layer-0 product state, one pass per 4-bit group of live rotations per later layer (the
// diagonal folded into the last), the measurement, and in the adjoint the diagonal pass plus
// the rotation passes of every layer over both states.
double cone_visits(const Plan& P, int cone, bool grad);
// The items of one (cone, set): the whole window, or its two branches when the cone splits.
void push_cone_items(const Plan& P, int cone, int set, bool grad, std::vector<WorkItem>& out);
// Sorts `its` (widest state first, then most work first), appends the (cone word, set) pairs
// to `items` and fills `cs` with the chunks of each width class: teams of 2^(W-4) threads as
// many as fit a CTA in the shared tier, one 512-thread team per CTA in the global tier.
void build_chunks(std::vector<WorkItem>& its, bool fp64, bool grad, int smax, std::vector<int32_t>& items,
                  ChunkSet& cs);
int team_bytes_host(int W, int Wt, int tt, bool fp64, bool grad, bool smem_state);

// One parameter set of a serving batch: where its plan, angles, partial sums and outputs
// live. Sets of different circuits share one launch through these records.
struct SetRec {
    const ConeDev* cones;
    const MeasDev* meas;
    const int32_t* prog;
    const tlq_gate* gates;
    const double* theta;        // this set's angles [n_params]
    const double* term_coeff;
    const int32_t* pmap_off;
    const int32_t* pmap_idx;
    const int32_t* pmap_term;
    double* energy;             // this set's energy (device)
    double* grad;               // this set's gradient [n_params] (device) or null
    int64_t gt_off, e_off, g_off;   // offsets into the batch's gate table, term energies, slots
    int32_t n_gates, n_params, n_terms, n_slots;
};

struct BatchLaunch {
    const SetRec* sets = nullptr;     // device [n_sets]
    int32_t n_sets = 0, max_gates = 0, max_params = 0;
    const int32_t* items = nullptr;   // (cone, set) pairs
    const ChunkDev* chunks = nullptr;
    // chunk ranges: forward-only smem, forward-only global, gradient smem, gradient global
    int32_t range[5] = {0, 0, 0, 0, 0};
    int32_t smem_bytes[2] = {0, 0};   // shared tier: forward, gradient
    int32_t smem_threads[2] = {kCtaThreads, kCtaThreads};   // shared tier CTA sizes
    int32_t gsmem_bytes[2] = {0, 0};  // global tier: forward, gradient
    size_t e_count = 0, g_count = 0;  // doubles in e_part / g_part (zeroed when `accum`)
    bool accum = false;               // branch items present
    void* gate_table = nullptr;
    double* e_part = nullptr;
    double* g_part = nullptr;
    void* gscratch = nullptr;
    size_t gscratch_slot = 0;
    int32_t g_grid = 0;
    int32_t* counters = nullptr;      // [4]
    int32_t* err = nullptr;
    bool fp64 = false;
    int sm_count = 0;
    int launches = 0;
};
int launch_cone_batch(BatchLaunch& L, void* stream);
int cone_smem_grid(bool fp64, bool grad, int smem_bytes, int sm_count, int threads);

struct DenseLaunch {
    int n_eff = 0;
    const DensePassDev* passes = nullptr;
    int32_t n_passes = 0;
    const DenseLayerDev* layers = nullptr;
    const DenseClassDev* classes = nullptr;
    const DensePassClassDev* pcd = nullptr;
    const int32_t* stage = nullptr;
    const int32_t* dists = nullptr;
    int32_t energy_class_off = 0, energy_nclass = 0;
    const DenseZTermDev* zterms = nullptr;
    int32_t n_zterms = 0;
    const DenseXTermDev* xterms = nullptr;
    int32_t n_xterms = 0;
    const DenseXTermDev* all_terms = nullptr;   // device copy (per-gate adjoint)
    const int32_t* adj_off = nullptr;           // DensePlan::adj_off / adj_idx (device)
    const int32_t* adj_idx = nullptr;
    const int32_t* tab_gate = nullptr;
    const int32_t* tab_mult = nullptr;
    int32_t tab_entries = 0;
    int32_t max_classes = 0, max_dists = 0;
    const tlq_gate* gates = nullptr;
    int32_t n_gates = 0, n_params = 0, B = 0;
    const double* theta = nullptr;        // [B][n_params]
    // workspace
    void* gate_table = nullptr;           // [B][n_gates] float2
    void* phase_tab = nullptr;            // [B][tab_entries] float2
    void* state = nullptr;                // 2^n_eff float2
    double* partial = nullptr;            // per-CTA / per-block partial sums
    double* xpart = nullptr;              // [n_xterms] per set
    int32_t* err = nullptr;               // kernel error word
    bool product_init = false;            // DensePlan::product_init
    const DensePassDev* host_fwd_passes = nullptr;   // DensePlan::fwd_passes
    const int32_t* host_rev_store = nullptr;          // DensePlan::rev_store
    int32_t n_fwd_passes = 0;
    const int32_t* host_init_gate = nullptr;   // DensePlan::init_gate (n_eff entries)
    int32_t init_class_off = 0, init_nclass = 0;
    const DensePassClassDev* init_pcd = nullptr;   // device copy of DensePlan::init_pcd
    void* lam = nullptr;                  // gradient mode: 2^n_eff float2 adjoint state
    double* gpart = nullptr;              // gradient mode: [n_passes][kDenseAdjSlots][grid] partials
    // outputs
    double* energy = nullptr;             // [B]
    double* grad = nullptr;               // [B][n_params] or null (energies only)
    bool per_gate = false;                // plain per-gate sweeps (baseline)
    bool tc = false;                      // forward rotation groups on the tensor cores (TLQ_MIXED_TC)
    bool gen_first = false;               // DensePlan::gen_first (FP32 passes only)
    bool keep_state = false;              // the caller reads the final state (else an energy-only
                                          // call skips the last pass's store when no X/Y term needs it)
    int sm_count = 0;
    void* ev_begin = nullptr;
    void* ev_end = nullptr;
    int launches = 0;
    // host copies (pass descriptors go to the kernel by value)
    const tlq_gate* host_gates = nullptr;
    const DensePassDev* host_passes = nullptr;
    const DenseXTermDev* host_xterms = nullptr;
    const DenseXTermDev* host_all_terms = nullptr;
    int32_t n_all_terms = 0;
};
size_t dense_partial_count(int n_eff);
int dense_grid(int n_eff, int sm_count);

int launch_dense(DenseLaunch& L, void* stream);

// Partial trace of a pure state (density.cu): kept[t] = t-th lowest kept qubit, traced[u] =
// u-th lowest traced qubit.
constexpr int kMaxDensityQubits = 15;   // largest kept set (a 2^15 x 2^15 complex64 output)
struct QubitMap { int32_t kept[32]; int32_t traced[32]; };
int herk_splits(int n, int m, int sm_count);
size_t partial_trace_workspace_bytes(int n, int m, int sm_count);
int launch_partial_trace(const void* psi, int n, const QubitMap& Q, int m, void* rho, void* workspace, int sm_count,
                         int32_t* err, void* stream, int* launches);
// Gates in the backward light cone of the qubit set S on a circuit's layers (every operator
// on S); *lo / *hi bound the qubits they touch together with S.
std::vector<int> light_cone_gates(const Circuit& c, const std::vector<int>& S, int* lo, int* hi);

}  // namespace tlq
