// Host planner: layer structure of a circuit and per-term causal cones.
//
// TensorLy-Quantum (arXiv:2112.10239) contracts the whole ket network, the operator and
// the bra network along an optimised path (Sec. 1, Sec. 3) and lists
// "causality-simplified contraction" as future work (Sec. 4). This planner implements
// that restriction: for each Pauli term it walks the circuit backwards and keeps only
// the gates that can influence the term, so each term becomes a small dense problem on
// a window of W chain sites whose size does not depend on the qubit count.
//
// Light-cone rule (Heisenberg picture, backwards through layer l = (rotations R_l,
// diagonal gates D_l)):
//   * D_l: the diagonal gates commute with each other. If the operator is still
//     diagonal (Z-only) they commute with it and drop out. Otherwise every diagonal gate
//     touching the support is kept and its qubits join the support (one step per layer,
//     because the new qubits only carry Z factors, which commute with D_l).
//   * R_l: rotations on support qubits are kept; after one the operator is no longer
//     diagonal. Rotations never grow the support.
// Gates outside the cone commute past the operator and cancel, so simulating only the
// kept gates on the window from |0...0> gives the exact term value.
#include "internal.h"

#include <algorithm>
#include <cstring>
#include <iterator>
#include <map>

namespace tlq {

static bool is_diag(int kind) { return kind == TLQ_RZ || kind == TLQ_RZZ || kind == TLQ_CZ; }
static bool is_two(int kind) { return kind == TLQ_RZZ || kind == TLQ_CZ; }

std::string plan_circuit_layers(Circuit& c) {
    // Greedy grouping in gate order: a rotation joins the open rotation step if its qubit
    // is still free there; diagonal gates join the open diagonal step. No reordering.
    struct Step { bool diag; std::vector<int> g; std::vector<char> used; };
    std::vector<Step> steps;
    c.nearest_neighbour = true;
    for (int i = 0; i < (int)c.gates.size(); ++i) {
        const tlq_gate& g = c.gates[i];
        if (is_two(g.kind) && std::abs(g.q0 - g.q1) != 1) c.nearest_neighbour = false;
        if (is_diag(g.kind)) {
            if (steps.empty() || !steps.back().diag) steps.push_back(Step{true, {}, {}});
            steps.back().g.push_back(i);
        } else {
            if (steps.empty() || steps.back().diag || steps.back().used[g.q0]) {
                steps.push_back(Step{false, {}, std::vector<char>(c.n, 0)});
            }
            steps.back().g.push_back(i);
            steps.back().used[g.q0] = 1;
        }
    }
    c.layers.clear();
    size_t k = 0;
    while (k < steps.size() && steps[k].diag) ++k;   // diagonal gates on |0..0>: global phase
    for (; k < steps.size(); ++k) {
        Circuit::Layer L;
        L.rot = steps[k].g;
        if (k + 1 < steps.size() && steps[k + 1].diag) { L.diag = steps[k + 1].g; ++k; }
        c.layers.push_back(std::move(L));
    }
    return "";
}

namespace {

struct LayerIndex {
    // per layer: rotation gate on qubit q (or -1); diagonal gates touching q
    std::vector<std::vector<int>> rot_at;                 // [L][n]
    std::vector<std::vector<std::vector<int>>> diag_at;   // [L][n] -> gates
    std::vector<int> layer_of;                            // gate -> layer (-1: dropped)
    std::vector<char> is_rot;                             // gate is a layer rotation
};

LayerIndex index_layers(const Circuit& c) {
    LayerIndex ix;
    const int L = (int)c.layers.size();
    ix.rot_at.assign(L, std::vector<int>(c.n, -1));
    ix.diag_at.assign(L, std::vector<std::vector<int>>(c.n));
    ix.layer_of.assign(c.gates.size(), -1);
    ix.is_rot.assign(c.gates.size(), 0);
    for (int l = 0; l < L; ++l) {
        for (int g : c.layers[l].rot) { ix.layer_of[g] = l; ix.is_rot[g] = 1; }
        for (int g : c.layers[l].diag) ix.layer_of[g] = l;
        for (int g : c.layers[l].rot) ix.rot_at[l][c.gates[g].q0] = g;
        for (int g : c.layers[l].diag) {
            const tlq_gate& G = c.gates[g];
            ix.diag_at[l][G.q0].push_back(g);
            if (is_two(G.kind)) ix.diag_at[l][G.q1].push_back(g);
        }
    }
    return ix;
}

}  // namespace

std::shared_ptr<Plan> make_plan(const Circuit& c, const Ham& h, std::string* err) {
    auto P = std::make_shared<Plan>();
    const int T = (int)h.terms.size();
    const int L = (int)c.layers.size();
    P->term_coeff.resize(T);
    for (int t = 0; t < T; ++t) P->term_coeff[t] = h.terms[t].coeff;

    if (c.n <= kDenseMaxQubits) {
        std::string derr;
        P->dense = make_dense_plan(c, h, &derr);
    }
    if (!c.nearest_neighbour) {
        P->path = TLQ_PATH_DENSE;
        P->why_dense = "two-qubit gate between non-adjacent qubits";
        if (!P->dense && err) *err = "non-local circuit on more than " + std::to_string(kDenseMaxQubits) + " qubits";
        return P->dense ? P : nullptr;
    }
    const LayerIndex ix = index_layers(c);
    std::vector<char> inS(c.n, 0), inc(c.gates.size(), 0);
    P->cone_lo.resize(T);
    P->cone_wtrue.resize(T);
    P->cone_gates.resize(T);
    struct PEntry { int32_t param, slot, term; };
    std::vector<PEntry> pentries;   // gradient slots in emission order
    int32_t slot_total = 0;

    std::vector<std::pair<int, int>> dpart;   // (diagonal gate, sub-layer) of one layer
    std::vector<uint32_t> zmask, pmask;
    // ---- phase 1: each term's own causal cone ----
    std::vector<std::vector<int>> tkept(T);
    std::vector<int> tlo(T), thi(T);
    for (int t = 0; t < T; ++t) {
        const Term& term = h.terms[t];
        std::vector<int> S(term.sites.begin(), term.sites.end());
        for (int q : S) inS[q] = 1;
        bool diag_op = true;
        for (char ch : term.letters) if (ch != 'Z') diag_op = false;
        std::vector<int>& kept = tkept[t];   // gate indices in the cone
        for (int l = L - 1; l >= 0; --l) {
            if (!diag_op && !c.layers[l].diag.empty()) {
                std::vector<int> grow;
                for (int q : S) {
                    for (int g : ix.diag_at[l][q]) {
                        if (inc[g]) continue;
                        inc[g] = 1;
                        kept.push_back(g);
                        const tlq_gate& G = c.gates[g];
                        if (!inS[G.q0]) { inS[G.q0] = 1; grow.push_back(G.q0); }
                        if (is_two(G.kind) && !inS[G.q1]) { inS[G.q1] = 1; grow.push_back(G.q1); }
                    }
                }
                S.insert(S.end(), grow.begin(), grow.end());
            }
            for (int q : S) {
                int g = ix.rot_at[l][q];
                if (g >= 0 && !inc[g]) { inc[g] = 1; kept.push_back(g); diag_op = false; }
            }
        }
        const int lo = *std::min_element(S.begin(), S.end());
        const int hi = *std::max_element(S.begin(), S.end());
        for (int q : S) inS[q] = 0;
        for (int g : kept) inc[g] = 0;
        std::sort(kept.begin(), kept.end());
        tlo[t] = lo;
        thi[t] = hi;
        const int wtrue = hi - lo + 1;
        P->cone_lo[t] = lo;
        P->cone_wtrue[t] = wtrue;
        P->cone_gates[t] = (int32_t)kept.size();
        const int W = std::max(wtrue, kMinConeW);
        P->max_w = std::max(P->max_w, W);
        if (W > kMaxConeW) {
            P->path = TLQ_PATH_DENSE;
            P->why_dense = "light cone wider than " + std::to_string(kMaxConeW) + " qubits";
            if (!P->dense && err) *err = "light cones wider than " + std::to_string(kMaxConeW) + " qubits on more than " +
                                         std::to_string(kDenseMaxQubits) + " qubits";
            return P->dense ? P : nullptr;
        }
    }
    // ---- phase 2: terms whose window lies inside another term's window share its cone ----
    // (one forward pass and one adjoint pass with lambda = sum_t c_t P_t psi serve all of them;
    // the window simulates the union of the members' cone gates, exact for each member)
    std::vector<int> order(T);
    for (int t = 0; t < T; ++t) order[t] = t;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return thi[a] - tlo[a] > thi[b] - tlo[b]; });
    std::vector<std::vector<int>> members;
    std::vector<int> glo, ghi;
    std::vector<std::vector<int>> by_lo(c.n);
    for (int t : order) {
        int found = -1;
        for (int lo = tlo[t]; lo >= 0 && lo >= tlo[t] - kMaxConeW && found < 0; --lo)
            for (int gidx : by_lo[lo])
                if (ghi[gidx] >= thi[t] && members[gidx].size() < (size_t)kMaxGroupTerms) { found = gidx; break; }
        if (found < 0) {
            found = (int)members.size();
            members.emplace_back();
            glo.push_back(tlo[t]);
            ghi.push_back(thi[t]);
            by_lo[tlo[t]].push_back(found);
        }
        members[found].push_back(t);
    }
    const int NG = (int)members.size();
    P->cones.resize(NG);
    P->cone_nrot.assign(NG, 0);
    P->cone_ndiag.assign(NG, 0);
    P->cone_npdiag.assign(NG, 0);
    P->group_wtrue.assign(NG, 0);
    // ---- phase 3: one program per group ----
    for (int t = 0; t < NG; ++t) {
        std::sort(members[t].begin(), members[t].end());
        std::vector<int> kept;
        for (int m : members[t]) {
            std::vector<int> merged;
            std::set_union(kept.begin(), kept.end(), tkept[m].begin(), tkept[m].end(), std::back_inserter(merged));
            kept.swap(merged);
        }
        const int lo = glo[t];
        const int W = std::max(ghi[t] - glo[t] + 1, kMinConeW);
        P->group_wtrue[t] = ghi[t] - glo[t] + 1;
        // A wide window whose top qubit is busy after the first layer (or measured) but whose
        // bottom qubit is free is laid out mirrored (window qubit j = chain qubit hi - j), so
        // that the free end is the top and the window can run as two branches (see below).
        bool mirror = false;
        if (W >= kSplitMinW && P->group_wtrue[t] == W && !kept.empty()) {
            const int l0 = ix.layer_of[kept.front()];
            auto end_free = [&](int q) {
                for (int m : members[t])
                    for (int site : h.terms[m].sites)
                        if (site == q) return false;
                for (int g : kept) {
                    const tlq_gate& G = c.gates[g];
                    const bool touches = G.q0 == q || (is_two(G.kind) && G.q1 == q);
                    if (touches && ix.layer_of[g] != l0) return false;
                }
                return true;
            };
            mirror = !end_free(ghi[t]) && end_free(lo);
        }
        const int top_q = lo + W - 1;
        auto pos1 = [&](int q) { return mirror ? top_q - q : q - lo; };                  // window qubit of q
        auto pos2 = [&](int a, int b) { return mirror ? top_q - std::max(a, b) : std::min(a, b) - lo; };   // of pair (a, a+1)
        // Emit the program in forward layer order: per layer a header and one fixed record
        // per window qubit (see internal.h). A layer whose cone gates put two RZ on one
        // qubit or two two-qubit gates on one pair is split into several layers (the
        // diagonal gates commute, so any split is exact).
        ConeDev cd{};
        cd.W = W;
        cd.prog_off = (int32_t)P->prog.size();
        cd.slot_off = slot_total;
        int32_t nslot = 0;
        std::vector<int32_t> body, layer_off;
        int32_t nlayers = 0;
        // gates of a layer have consecutive indices, so the sorted cone gates come in layer order
        size_t kp = 0;
        while (kp < kept.size()) {
            const int l = ix.layer_of[kept[kp]];
            size_t kp2 = kp;
            while (kp2 < kept.size() && ix.layer_of[kept[kp2]] == l) ++kp2;
            // sub-layers: each diagonal gate goes to the first part where its position is free
            int nparts = 1;
            dpart.clear();
            zmask.assign(1, 0u);
            pmask.assign(1, 0u);
            for (size_t k = kp; k < kp2; ++k) {
                const int g = kept[k];
                if (ix.is_rot[g]) continue;
                const tlq_gate& G = c.gates[g];
                const bool two = is_two(G.kind);
                const uint32_t bit = 1u << (two ? pos2(G.q0, G.q1) : pos1(G.q0));
                int part = 0;
                while (part < nparts && ((two ? pmask[part] : zmask[part]) & bit)) ++part;
                if (part == nparts) {
                    ++nparts;
                    zmask.push_back(0u);
                    pmask.push_back(0u);
                }
                (two ? pmask[part] : zmask[part]) |= bit;
                dpart.push_back({g, part});
            }
            for (int part = 0; part < nparts; ++part) {
                layer_off.push_back((int32_t)body.size());
                const size_t hdr = body.size();
                body.resize(hdr + kLayerHeader + (size_t)W * kRecWords, -1);
                int32_t* rec = body.data() + hdr + kLayerHeader;
                for (int jj = 0; jj < W; ++jj) {
                    rec[(size_t)jj * kRecWords + 1] = 0;
                    rec[(size_t)jj * kRecWords + 5] = 0;
                }
                uint32_t live = 0;
                if (part == 0) {
                    for (size_t k = kp; k < kp2; ++k) {
                        const int g = kept[k];
                        if (!ix.is_rot[g]) continue;
                        const int jj = pos1(c.gates[g].q0);
                        rec[(size_t)jj * kRecWords + 0] = g;
                        live |= 1u << jj;
                    }
                }
                bool any_diag = false;
                for (const auto& dp : dpart) {
                    if (dp.second != part) continue;
                    const tlq_gate& G = c.gates[dp.first];
                    const bool two = is_two(G.kind);
                    const int jj = two ? pos2(G.q0, G.q1) : pos1(G.q0);
                    rec[(size_t)jj * kRecWords + (two ? 4 : 2)] = dp.first;
                    any_diag = true;
                }
                // gradient slots: rotations by window position, then RZ / pair gates by position
                for (int jj = 0; jj < W; ++jj) {
                    int32_t* r = rec + (size_t)jj * kRecWords;
                    if (r[0] < 0) continue;
                    const tlq_gate& G = c.gates[r[0]];
                    const int32_t slot = G.param >= 0 ? nslot++ : -1;
                    if (slot >= 0) pentries.push_back({G.param, slot_total + slot, -1});
                    r[1] = G.kind | ((slot + 1) << 8);
                    P->cone_nrot[t] += 1;
                }
                for (int jj = 0; jj < W; ++jj) {
                    int32_t* r = rec + (size_t)jj * kRecWords;
                    if (r[2] >= 0) {
                        const tlq_gate& G = c.gates[r[2]];
                        const int32_t slot = G.param >= 0 ? nslot++ : -1;
                        if (slot >= 0) {
                            pentries.push_back({G.param, slot_total + slot, -1});
                            P->cone_npdiag[t] += 1;
                        }
                        r[3] = slot;
                    }
                    if (r[4] >= 0) {
                        const tlq_gate& G = c.gates[r[4]];
                        const int32_t slot = (G.param >= 0 && G.kind != TLQ_CZ) ? nslot++ : -1;
                        if (slot >= 0) {
                            pentries.push_back({G.param, slot_total + slot, -1});
                            P->cone_npdiag[t] += 1;
                        }
                        r[5] = G.kind | ((slot + 1) << 8);
                    }
                }
                if (any_diag) P->cone_ndiag[t] += 1;
                body[hdr + 0] = any_diag ? 1 : 0;
                body[hdr + 1] = (int32_t)live;
                body[hdr + 2] = 0;
                body[hdr + 3] = 0;
                ++nlayers;
            }
            kp = kp2;
        }
        P->prog.push_back(nlayers);
        P->prog.insert(P->prog.end(), layer_off.begin(), layer_off.end());
        P->prog.insert(P->prog.end(), body.begin(), body.end());
        cd.nslots = nslot;
        slot_total += nslot;
        cd.mterm_off = (int32_t)P->meas.size();
        cd.nmterms = (int32_t)members[t].size();
        for (int m : members[t]) {
            const Term& term = h.terms[m];
            MeasDev md{};
            md.term = m;
            for (size_t q = 0; q < term.sites.size(); ++q) {
                const uint32_t bit = 1u << pos1(term.sites[q]);
                const char ch = term.letters[q];
                if (ch == 'X' || ch == 'Y') md.flip |= bit;
                if (ch == 'Y' || ch == 'Z') md.zy |= bit;
                if (ch == 'Y') ++md.ny;
            }
            P->meas.push_back(md);
        }
        // Two branches of W - 1 qubits instead of one window when the window is real (no
        // padding), wide, its top qubit has gates of program layer 0 only and no measured
        // term touches it: the branches with top bit 0 and 1 are then independent items.
        cd.split = 0;
        if (W >= kSplitMinW && P->group_wtrue[t] == W && nlayers >= 1) {
            const int top = W - 1;
            bool ok = true;
            for (int m = cd.mterm_off; m < cd.mterm_off + cd.nmterms; ++m)
                if (((P->meas[m].flip | P->meas[m].zy) >> top) & 1u) ok = false;
            for (int li = 1; li < nlayers && ok; ++li) {
                const int32_t* lp = body.data() + layer_off[li];
                const int32_t* rec = lp + kLayerHeader;
                if (((uint32_t)lp[1] >> top) & 1u) ok = false;                 // rotation on top
                if (rec[top * kRecWords + 2] >= 0) ok = false;                 // RZ on top
                if (rec[(top - 1) * kRecWords + 4] >= 0) ok = false;           // pair (top - 1, top)
            }
            cd.split = ok ? 1 : 0;
        }
        P->cones[t] = cd;
    }
    P->n_slots = slot_total;
    P->pmap_off.assign(c.n_params + 1, 0);
    // CSR by parameter (counting sort keeps emission order within a parameter)
    for (const PEntry& e : pentries) P->pmap_off[e.param + 1] += 1;
    for (int q = 0; q < c.n_params; ++q) P->pmap_off[q + 1] += P->pmap_off[q];
    P->pmap_idx.assign(pentries.size(), 0);
    P->pmap_term.assign(pentries.size(), 0);
    {
        std::vector<int32_t> fill(P->pmap_off.begin(), P->pmap_off.end() - 1);
        for (const PEntry& e : pentries) {
            const int32_t k = fill[e.param]++;
            P->pmap_idx[k] = e.slot;
            P->pmap_term[k] = e.term;
        }
    }
    (void)err;
    return P;
}


// ---------------------------------------------------------------------------------------
// Work lists of the cone kernel.
// ---------------------------------------------------------------------------------------

double cone_visits(const Plan& P, int cone, bool grad) {
    const ConeDev& cd = P.cones[cone];
    const int W = cd.W;
    const int32_t* prog = P.prog.data() + cd.prog_off;
    const int nl = prog[0];
    const int32_t* body = prog + 1 + nl;
    double passes = 1 + 1;   // layer 0 (or the |0..0> start) and the measurement
    for (int li = 0; li < nl; ++li) {
        const int32_t* lp = body + prog[1 + li];
        const bool diag = lp[0] > 0;
        const unsigned live = (unsigned)lp[1];
        if (li > 0) {
            unsigned todo = live;
            int n = 0;
            while (todo) {
                const int bt = __builtin_ctz(todo);
                const int sh = bt < 4 ? 0 : std::min(bt, W - 4);
                todo &= ~(15u << sh);
                ++n;
            }
            passes += std::max(n, diag ? 1 : 0);
        }
        if (grad) {
            unsigned todo = live;
            int n = diag ? 1 : 0;
            while (todo) {
                const int bt = 31 - __builtin_clz(todo);
                int sh = bt - 3;
                if (sh < 4) sh = bt >= 4 ? 4 : 0;
                if (sh > W - 4) sh = W - 4;
                todo &= ~(15u << sh);
                ++n;
            }
            passes += 2.0 * n;
        }
    }
    return passes * (double)(1u << W);
}

void push_cone_items(const Plan& P, int cone, int set, bool grad, std::vector<WorkItem>& out) {
    const ConeDev& cd = P.cones[cone];
    const double w = cone_visits(P, cone, grad);
    if (cd.split) {
        out.push_back({cone | (1 << kItemHalfShift), set, cd.W - 1, cd.W, 0.5 * w});
        out.push_back({cone | (2 << kItemHalfShift), set, cd.W - 1, cd.W, 0.5 * w});
    } else {
        out.push_back({cone, set, cd.W, cd.W, w});
    }
}

void build_chunks(std::vector<WorkItem>& its, bool fp64, bool grad, int smax, std::vector<int32_t>& items,
                  ChunkSet& cs) {
    // widest state first; within a width the most amplitude visits first, so that the items
    // left for the last round of a width class are its cheapest
    std::stable_sort(its.begin(), its.end(), [](const WorkItem& a, const WorkItem& b) {
        if (a.W != b.W) return a.W > b.W;
        return a.work > b.work;
    });
    struct Class {
        size_t k, k2;
        int W, tt, tb;
        bool global;
    };
    std::vector<Class> cls;
    int max_tt = 0;
    for (size_t k = 0; k < its.size();) {
        Class c{};
        c.k = k;
        c.W = its[k].W;
        int wt = c.W;   // widest window of the class (tables of branch items cover the whole window)
        size_t k2 = k;
        while (k2 < its.size() && its[k2].W == c.W) {
            wt = std::max(wt, its[k2].Wt);
            ++k2;
        }
        c.k2 = k2;
        c.tt = std::min(kCtaThreads, 1 << (c.W - 4));
        c.tb = team_bytes_host(c.W, wt, c.tt, fp64, grad, true);
        c.global = c.W > kMaxSmemConeW || c.tb > smax;
        if (c.global) {
            c.tt = kGlobalCtaThreads;
            c.tb = team_bytes_host(c.W, wt, c.tt, fp64, grad, false);
        } else {
            max_tt = std::max(max_tt, c.tt);
        }
        cls.push_back(c);
        k = k2;
    }
    // Shared-tier CTAs of 256 threads when the widest teams have 256: two CTAs per SM with one
    // such team each take their items independently (finer load balance at the end of a
    // launch); 512 threads otherwise.
    cs.smem_threads = max_tt == 256 ? 256 : kCtaThreads;
    for (const Class& c : cls) {
        const int nteams = c.global ? 1 : std::max(1, std::min(cs.smem_threads / c.tt, smax / c.tb));
        const int first = (int)items.size() / 2;
        for (size_t i = c.k; i < c.k2; ++i) {
            items.push_back(its[i].cone);
            items.push_back(its[i].set);
            if (its[i].Wt > its[i].W) cs.accum = true;
        }
        const int nit = (int)(c.k2 - c.k);
        for (int f = 0; f < nit; f += nteams) {
            ChunkDev ch{};
            ch.W = c.W;
            ch.first = first + f;
            ch.count = std::min(nteams, nit - f);
            ch.tt = c.tt;
            ch.team_bytes = c.tb;
            (c.global ? cs.glob : cs.smem).push_back(ch);
        }
        if (c.global) {
            cs.gsmem_bytes = std::max(cs.gsmem_bytes, c.tb);
            cs.g_maxW = std::max(cs.g_maxW, c.W);
        } else {
            cs.smem_bytes = std::max(cs.smem_bytes, nteams * c.tb);
        }
    }
}

// ---------------------------------------------------------------------------------------
// Dense statevector plan.
// ---------------------------------------------------------------------------------------

namespace {

// Collects pairs/singles of one class; returns false if the position is already used
// (the caller then opens another class with the same angle).
struct ClassBuild {
    int kind = 0, gate = -1;
    double coeff = 0;
    std::map<int, uint32_t> dist;   // d -> mask of lower qubits
    uint32_t single = 0;
    int nterms = 0;
    bool add_pair(int u, int v) {
        if (u > v) std::swap(u, v);
        uint32_t& m = dist[v - u];
        if (m & (1u << u)) return false;
        m |= 1u << u;
        ++nterms;
        return true;
    }
    bool add_single(int q) {
        if (single & (1u << q)) return false;
        single |= 1u << q;
        ++nterms;
        return true;
    }
};

void emit_class(DensePlan& D, const ClassBuild& cb) {
    DenseClassDev c{};
    c.kind = cb.kind;
    c.gate = cb.gate;
    c.nterms = cb.nterms;
    c.dist_off = (int32_t)D.dists.size() / 2;
    c.ndist = (int32_t)cb.dist.size();
    for (auto& kv : cb.dist) { D.dists.push_back(kv.first); D.dists.push_back((int32_t)kv.second); }
    c.single = cb.single;
    c.coeff = cb.coeff;
    c.tab_off = -1;
    c.ew = -1;
    if (cb.kind == 0) {
        c.tab_off = (int32_t)D.tab_gate.size();
        for (int k = 0; k <= cb.nterms; ++k) {
            D.tab_gate.push_back(cb.gate);
            D.tab_mult.push_back(cb.nterms - 2 * k);
        }
    }
    D.max_dists = std::max(D.max_dists, c.ndist);
    D.classes.push_back(c);
}

// Adds one term to the first class of `list` that accepts it, or opens a new class.
template <typename F>
void place(std::vector<ClassBuild>& list, const ClassBuild& proto, F add) {
    for (auto& cb : list)
        if (add(cb)) return;
    list.push_back(proto);
    add(list.back());
}

}  // namespace

std::vector<int> light_cone_gates(const Circuit& c, const std::vector<int>& S0, int* lo, int* hi) {
    // Walk the layers from last to first. A layer's diagonal gates commute with each other,
    // so conjugating a general operator on the support S by all of them involves only the
    // gates that touch S as it stands before the layer: each joins the cone and its other
    // qubit joins S (partners added here pull in no further gate of the same layer). Then
    // the layer's rotations on S join. Gates outside commute with the operator and drop out
    // (the rule of the term cones, for a non-diagonal operator).
    std::vector<char> in(c.n, 0);
    std::vector<int> S;
    for (int q : S0) if (!in[q]) { in[q] = 1; S.push_back(q); }
    std::vector<int> kept, grow;
    for (int l = (int)c.layers.size() - 1; l >= 0; --l) {
        grow.clear();
        for (int g : c.layers[l].diag) {
            const tlq_gate& G = c.gates[g];
            const bool two = G.kind == TLQ_RZZ || G.kind == TLQ_CZ;
            if (!in[G.q0] && !(two && in[G.q1])) continue;
            kept.push_back(g);
            if (two) grow.push_back(in[G.q0] ? G.q1 : G.q0);
        }
        for (int q : grow)
            if (!in[q]) { in[q] = 1; S.push_back(q); }
        for (int g : c.layers[l].rot)
            if (in[c.gates[g].q0]) kept.push_back(g);
    }
    std::sort(kept.begin(), kept.end());
    *lo = *std::min_element(S.begin(), S.end());
    *hi = *std::max_element(S.begin(), S.end());
    return kept;
}

std::shared_ptr<DensePlan> make_dense_plan(const Circuit& c, const Ham& h, std::string* err) {
    if (c.n > kDenseMaxQubits) {
        if (err) *err = "dense statevector path needs n <= " + std::to_string(kDenseMaxQubits);
        return nullptr;
    }
    auto D = std::make_shared<DensePlan>();
    const int n_eff = std::max(c.n, kDenseTileBits);
    D->n_eff = n_eff;
    // diagonal classes per layer
    const int L = (int)c.layers.size();
    for (int l = 0; l < L; ++l) {
        DenseLayerDev ld{};
        ld.class_off = (int32_t)D->classes.size();
        std::map<std::pair<int, uint64_t>, std::vector<ClassBuild>> xor_cls;   // key: (param or -1, angle bits)
        std::vector<ClassBuild> and_cls;
        for (int g : c.layers[l].diag) {
            const tlq_gate& G = c.gates[g];
            if (G.kind == TLQ_CZ) {
                ClassBuild proto;
                proto.kind = 1;
                place(and_cls, proto, [&](ClassBuild& cb) { return cb.add_pair(G.q0, G.q1); });
                continue;
            }
            uint64_t bits = 0;
            if (G.param < 0) std::memcpy(&bits, &G.angle, 8);
            auto& list = xor_cls[{G.param, bits}];
            ClassBuild proto;
            proto.kind = 0;
            proto.gate = g;
            if (G.kind == TLQ_RZZ) place(list, proto, [&](ClassBuild& cb) { return cb.add_pair(G.q0, G.q1); });
            else place(list, proto, [&](ClassBuild& cb) { return cb.add_single(G.q0); });
        }
        for (auto& kv : xor_cls)
            for (auto& cb : kv.second) emit_class(*D, cb);
        for (auto& cb : and_cls) emit_class(*D, cb);
        ld.nclass = (int32_t)D->classes.size() - ld.class_off;
        D->max_classes_per_layer = std::max(D->max_classes_per_layer, (int)ld.nclass);
        D->layers.push_back(ld);
    }
    // energy: Z/ZZ terms in coefficient classes, longer Z strings, and X/Y terms
    D->energy_class_off = (int32_t)D->classes.size();
    std::map<uint64_t, std::vector<ClassBuild>> ecls;
    for (const Term& t : h.terms) {
        bool zonly = true;
        for (char ch : t.letters) zonly &= (ch == 'Z');
        if (zonly && t.sites.size() <= 2) {
            uint64_t bits;
            std::memcpy(&bits, &t.coeff, 8);
            ClassBuild proto;
            proto.kind = 2;
            proto.coeff = t.coeff;
            if (t.sites.size() == 2)
                place(ecls[bits], proto, [&](ClassBuild& cb) { return cb.add_pair(t.sites[0], t.sites[1]); });
            else
                place(ecls[bits], proto, [&](ClassBuild& cb) { return cb.add_single(t.sites[0]); });
        } else if (zonly) {
            DenseZTermDev z{};
            for (int s : t.sites) z.mask |= 1u << s;
            z.coeff = t.coeff;
            D->zterms.push_back(z);
        }
        {
            DenseXTermDev x{};
            for (size_t k = 0; k < t.sites.size(); ++k) {
                const uint32_t bit = 1u << t.sites[k];
                const char ch = t.letters[k];
                if (ch == 'X' || ch == 'Y') x.flip |= bit;
                if (ch == 'Y' || ch == 'Z') x.zy |= bit;
                if (ch == 'Y') ++x.ny;
            }
            x.coeff = t.coeff;
            D->all_terms.push_back(x);
        }
        if (!zonly) {
            DenseXTermDev x{};
            for (size_t k = 0; k < t.sites.size(); ++k) {
                const uint32_t bit = 1u << t.sites[k];
                const char ch = t.letters[k];
                if (ch == 'X' || ch == 'Y') x.flip |= bit;
                if (ch == 'Y' || ch == 'Z') x.zy |= bit;
                if (ch == 'Y') ++x.ny;
            }
            x.coeff = t.coeff;
            D->xterms.push_back(x);
        }
    }
    for (auto& kv : ecls)
        for (auto& cb : kv.second) emit_class(*D, cb);
    D->energy_nclass = (int32_t)D->classes.size() - D->energy_class_off;

    // rotation frame: qubits whose rotations are all RX (see DensePlan::frame_mask)
    {
        std::vector<int> nrx(c.n, 0), nry(c.n, 0);
        for (const tlq_gate& g : c.gates) {
            if (g.kind == TLQ_RX) ++nrx[g.q0];
            if (g.kind == TLQ_RY) ++nry[g.q0];
        }
        for (int q = 0; q < c.n && q < 32; ++q)
            if (nrx[q] > 0 && nry[q] == 0) D->frame_mask |= 1u << q;
        D->fgates = c.gates;
        for (tlq_gate& g : D->fgates)
            if (g.kind == TLQ_RX && ((D->frame_mask >> g.q0) & 1u)) g.kind = TLQ_RY;
        D->fxterms = D->xterms;
        for (DenseXTermDev& x : D->fxterms) {
            const uint32_t xs = x.flip & ~x.zy & D->frame_mask;   // X letters in the frame: -> Y
            const uint32_t ys = x.flip & x.zy & D->frame_mask;    // Y letters in the frame: -> -X
            x.zy = (x.zy | xs) & ~ys;
            x.ny += __builtin_popcount(xs) - __builtin_popcount(ys);
            if (__builtin_popcount(ys) & 1) x.coeff = -x.coeff;
        }
    }

    // Pass schedule. Tile patterns: the low tile (qubits 0..11) and strided tiles covering 8
    // higher qubits each. Greedy: each pass takes the pattern covering the most pending
    // rotations of the current layer; when a pass completes a layer it applies the layer's
    // diagonal right there and continues with the next layer's rotations on the same tile.
    std::vector<int> chunk_a;
    for (int a = kDenseTileBits; a < n_eff; a += kDenseStridedBits)
        chunk_a.push_back(std::min(a, n_eff - kDenseStridedBits));
    auto blank = [](int strided, int a) {
        DensePassDev p{};
        p.strided = strided;
        p.a = a;
        p.store = 1;
        p.measure_group = -1;
        for (int g = 0; g < kDenseMaxGroups; ++g) {
            p.group_cls[g] = -1;
            p.group_pcd[g] = -1;
            for (int k = 0; k < 4; ++k) p.gate[g][k] = -1;
        }
        return p;
    };
    // local bit of global qubit q in a pattern (-1: not in the tile); patterns: -1 low, else chunk
    auto local_of = [&](int pat, int q) -> int {
        if (pat < 0) return q < kDenseTileBits ? q : -1;
        const int a = chunk_a[pat];
        if (q < 4) return q;
        return (q >= a && q < a + kDenseStridedBits) ? 4 + q - a : -1;
    };
    struct GroupDiag { int pass, group, layer; };     // diagonal (or energy: layer = -1) after a group
    // Greedy schedule of layers [l0, l1) into `out` (pass indices in gdiag are into `out`).
    auto schedule = [&](int l0, int l1, std::vector<DensePassDev>& out, std::vector<GroupDiag>& gdiag) {
        std::vector<int> pend;                        // pending rotation gates of layer l
        int l = l0;
        auto load_layer = [&]() {
            pend.clear();
            if (l < l1) pend = c.layers[l].rot;
        };
        load_layer();
        while (l < l1) {
            // choose the pattern with the most pending rotations
            int best = -1, bestn = -1;
            for (int pat = -1; pat < (int)chunk_a.size(); ++pat) {
                int cnt = 0;
                for (int g : pend) cnt += local_of(pat, c.gates[g].q0) >= 0;
                if (cnt > bestn) { bestn = cnt; best = pat; }
            }
            DensePassDev pass = blank(best >= 0, best >= 0 ? chunk_a[best] : 0);
            const int pi = (int)out.size();
            for (;;) {
                // rotations of layer l on this tile
                uint32_t bits = 0;
                int gate_at[16];
                for (int k = 0; k < 16; ++k) gate_at[k] = -1;
                std::vector<int> rest;
                for (int g : pend) {
                    const int lb = local_of(best, c.gates[g].q0);
                    if (lb >= 0 && !((bits >> lb) & 1)) { bits |= 1u << lb; gate_at[lb] = g; }
                    else rest.push_back(g);
                }
                int need = 0;
                for (uint32_t b2 = bits; b2;) {
                    const int b = __builtin_ctz(b2);
                    const int s = b < 4 ? 0 : std::min(b, kDenseTileBits - 4);
                    b2 &= ~(15u << s);
                    ++need;
                }
                const bool completes = rest.empty();
                if (pass.ngroups + std::max(need, completes ? 1 : 0) > kDenseMaxGroups) break;
                while (bits) {
                    const int b = __builtin_ctz(bits);
                    const int s = b < 4 ? 0 : std::min(b, kDenseTileBits - 4);
                    const int gi = pass.ngroups++;
                    if (l == 0) pass.group_rot0 |= 1u << gi;
                    pass.group_s[gi] = s;
                    pass.group_mask[gi] = (bits >> s) & 15u;
                    for (int k = 0; k < 4; ++k)
                        if ((pass.group_mask[gi] >> k) & 1) pass.gate[gi][k] = gate_at[s + k];
                    bits &= ~(15u << s);
                }
                pend = rest;
                if (!completes) break;
                // layer l done on the whole state: its diagonal follows the last group
                if (pass.ngroups == 0) {
                    pass.group_s[0] = kDenseTileBits - 4;
                    pass.group_mask[0] = 0;
                    pass.ngroups = 1;
                }
                if (!c.layers[l].diag.empty()) gdiag.push_back({pi, pass.ngroups - 1, l});
                ++l;
                load_layer();
                if (l >= l1) break;
                if (pass.ngroups >= kDenseMaxGroups) break;
            }
            if (pass.ngroups == 0) {   // nothing fit (cannot happen with 8 groups) -- keep the loop finite
                pass.group_s[0] = kDenseTileBits - 4;
                pass.group_mask[0] = 0;
                pass.ngroups = 1;
            }
            out.push_back(pass);
        }
    };
    // Split counts of class `cl` over register bits gbit[0..3] (global qubits; see
    // DensePassClassDev): partners outside the bits per bit, in-group counts C[j].
    auto split_counts = [&](const DenseClassDev& cl, const int (&gbit)[4]) {
        auto kof = [&](int q) { for (int k = 0; k < 4; ++k) if (gbit[k] == q) return k; return -1; };
        DensePassClassDev pc{};
        uint32_t cnt[16] = {0};
        for (int k = 0; k < cl.ndist; ++k) {
            const int d = D->dists[2 * (cl.dist_off + k)];
            const uint32_t M = (uint32_t)D->dists[2 * (cl.dist_off + k) + 1];
            for (int u = 0; u < 32; ++u) {
                if (!((M >> u) & 1)) continue;
                const int v = u + d;
                const int ku = kof(u), kv = kof(v);
                if (ku >= 0 && kv >= 0) {
                    for (int jj = 0; jj < 16; ++jj) {
                        const int bu = (jj >> ku) & 1, bv = (jj >> kv) & 1;
                        cnt[jj] += cl.kind == 1 ? (bu & bv) : (bu ^ bv);
                    }
                } else if (ku >= 0) {
                    pc.N[ku] |= 1u << v;
                } else if (kv >= 0) {
                    pc.N[kv] |= 1u << u;
                }
            }
        }
        for (int k = 0; k < 4; ++k)
            if ((cl.single >> gbit[k]) & 1) pc.single |= 1u << k;
        for (int jj = 0; jj < 16; ++jj) pc.C[jj >> 2] |= cnt[jj] << (8 * (jj & 3));
        return pc;
    };
    // The energy after the last pass of P, then per pass the staged classes of every group
    // that evaluates some, with their split counts (shared pools D->stage and D->pcd).
    const bool want_energy = D->energy_nclass > 0 || !D->zterms.empty();
    auto finalize = [&](std::vector<DensePassDev>& P, std::vector<GroupDiag>& gdiag) {
        if (want_energy) {
            if (P.empty()) {
                DensePassDev p = blank(0, 0);
                p.ngroups = 1;
                p.group_s[0] = kDenseTileBits - 4;
                p.store = 0;
                P.push_back(p);
            }
            gdiag.push_back({(int)P.size() - 1, P.back().ngroups - 1, -1});
            P.back().measure_group = P.back().ngroups - 1;
        }
        for (int pi = 0; pi < (int)P.size(); ++pi) {
            DensePassDev& pass = P[pi];
            pass.stage_off = (int32_t)D->stage.size();
            for (const GroupDiag& gd : gdiag) {
                if (gd.pass != pi) continue;
                const int gi = gd.group;
                int first_cls, ncls;
                if (gd.layer >= 0) {
                    first_cls = D->layers[gd.layer].class_off;
                    ncls = D->layers[gd.layer].nclass;
                } else {
                    first_cls = D->energy_class_off;
                    ncls = D->energy_nclass;
                }
                if (pass.group_ncls[gi] == 0) {
                    pass.group_cls[gi] = (int32_t)D->stage.size() - pass.stage_off;
                    pass.group_pcd[gi] = (int32_t)D->pcd.size();
                }
                pass.group_ncls[gi] += ncls;
                const int s = pass.group_s[gi];
                int gbit[4];
                for (int k = 0; k < 4; ++k) {
                    const int local = s + k;
                    gbit[k] = pass.strided ? (local < 4 ? local : pass.a + local - 4) : local;
                }
                for (int ci = first_cls; ci < first_cls + ncls; ++ci) {
                    D->stage.push_back(ci);
                    D->pcd.push_back(split_counts(D->classes[ci], gbit));
                }
            }
            pass.nstage = (int32_t)D->stage.size() - pass.stage_off;
        }
    };
    // The full schedule (used by the adjoint, and by the forward from |0..0>) and, for two or
    // more layers, a forward schedule of layers 1.. that starts from layer 0's product state.
    std::vector<GroupDiag> gd_all, gd_fwd;
    D->init_gate.assign(n_eff, -1);
    schedule(0, L, D->passes, gd_all);
    finalize(D->passes, gd_all);
    D->rev_store.assign(D->passes.size(), 0);
    for (size_t p = 1; p < D->passes.size(); ++p) {
        const DensePassDev& ps = D->passes[p];
        bool rot0_only = ps.group_rot0 == (1u << ps.ngroups) - 1u;
        for (int g = 0; g < ps.ngroups; ++g) rot0_only &= ps.group_ncls[g] == 0;
        D->rev_store[p] = rot0_only ? 0 : 1;
    }
    D->product_init = L >= 2;
    if (D->product_init) {
        schedule(1, L, D->fwd_passes, gd_fwd);
        finalize(D->fwd_passes, gd_fwd);
        for (int g : c.layers[0].rot) D->init_gate[c.gates[g].q0] = g;
        D->init_class_off = D->layers[0].class_off;
        D->init_nclass = D->layers[0].nclass;
        const int gbit0[4] = {0, 1, 2, 3};
        for (int ci = D->init_class_off; ci < D->init_class_off + D->init_nclass; ++ci)
            D->init_pcd.push_back(split_counts(D->classes[ci], gbit0));
        D->gen_first = !D->fwd_passes.empty() && D->fwd_passes[0].strided == 0 && D->fwd_passes[0].group_s[0] == 0 &&
                       D->init_nclass <= kDenseMaxLayerClasses;
    }
    // adjoint slots: rotation k of group g -> 4g + k; staged class ci (kind 0, a parameter) ->
    // 4 * kDenseMaxGroups + ci; collected per parameter with a counting sort (pass-major order)
    {
        std::vector<std::pair<int32_t, int32_t>> ent;   // (param, pass * slots + slot)
        for (int pi = 0; pi < (int)D->passes.size(); ++pi) {
            const DensePassDev& pass = D->passes[pi];
            for (int g = 0; g < pass.ngroups; ++g)
                for (int k = 0; k < 4; ++k) {
                    const int gate = pass.gate[g][k];
                    if (gate >= 0 && c.gates[gate].param >= 0)
                        ent.push_back({c.gates[gate].param, pi * kDenseAdjSlots + 4 * g + k});
                }
            for (int ci = 0; ci < pass.nstage && ci < kDenseMaxLayerClasses; ++ci) {
                const DenseClassDev& cl = D->classes[D->stage[pass.stage_off + ci]];
                if (cl.kind == 0 && c.gates[cl.gate].param >= 0)
                    ent.push_back({c.gates[cl.gate].param, pi * kDenseAdjSlots + 4 * kDenseMaxGroups + ci});
            }
        }
        D->adj_off.assign(c.n_params + 1, 0);
        for (auto& e : ent) ++D->adj_off[e.first + 1];
        for (int p = 0; p < c.n_params; ++p) D->adj_off[p + 1] += D->adj_off[p];
        D->adj_idx.assign(ent.size(), 0);
        std::vector<int32_t> fill(D->adj_off.begin(), D->adj_off.end() - 1);
        for (auto& e : ent) D->adj_idx[fill[e.first]++] = e.second;
    }
    // shared-memory capacity of the pass kernel
    std::vector<DensePassDev> all_passes = D->passes;
    all_passes.insert(all_passes.end(), D->fwd_passes.begin(), D->fwd_passes.end());
    for (const DensePassDev& pass : all_passes) {
        int words = 0, tab = 0;
        for (int k = 0; k < pass.nstage; ++k) {
            const DenseClassDev& cl = D->classes[D->stage[pass.stage_off + k]];
            words += 2 * cl.ndist;
            tab += cl.kind == 0 ? cl.nterms + 1 : 0;
        }
        if (pass.nstage > kDenseMaxLayerClasses || words > kDenseMaxDistWords || tab > kDenseMaxTab)
            D->fits_fused = false;
    }
    return D;
}

}  // namespace tlq
