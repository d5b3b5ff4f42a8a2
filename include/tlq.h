/*
 * tlq.h -- C-ABI of the GB300 expectation-value / gradient engine.
 *
 * What the library computes (TensorLy-Quantum, arXiv:2112.10239):
 *   Sec. 2: circuits are built from pre-defined gates, operators and states;
 *   Sec. 3: the forward pass is the expectation value <H> of a circuit's output
 *           state against a Hamiltonian given as a sum of local Pauli terms (the
 *           transverse-field Ising model there), and the backward pass is the full
 *           gradient nabla <H> with respect to every rotation angle;
 *   Sec. 4: "causality-simplified contraction" (listed there as future work) --
 *           for nearest-neighbour circuits each term is contracted over its causal
 *           cone only, so the cost does not grow with the qubit count.
 *
 * Conventions fixed by this library (the paper states none of them):
 *   - the initial state is |0...0>; qubit q is bit q of the amplitude index;
 *   - RX(a) = exp(-i a X/2), RY(a) = exp(-i a Y/2) = [[c,-s],[s,c]],
 *     RZ(a) = exp(-i a Z/2), RZZ(a) = exp(-i a Z(x)Z/2), CZ = diag(1,1,1,-1),
 *     with c = cos(a/2), s = sin(a/2);
 *   - a gate takes theta[param] when param >= 0, else its fixed `angle`;
 *   - gradients are dE/dtheta_p summed over every gate carrying parameter p.
 *
 * General rules:
 *   - Every call returns a tlq_status; nothing throws across the ABI and nothing
 *     aborts the process. On failure tlq_last_error() gives a message
 *     (thread-local; valid until the thread's next failing call).
 *   - Handles are owned by the library from *_create until *_destroy. Gate and term
 *     arrays are copied at create time; the caller keeps ownership of its arrays.
 *   - theta/energy/grad buffers are borrowed for the duration of a synchronous call,
 *     or, for tlq_submit, until tlq_poll returns TLQ_OK for that ticket.
 *   - Angles are FP64 on the boundary; energies and gradients are FP64.
 *   - A context and its handles may be used from one thread at a time, except
 *     tlq_submit / tlq_poll, which are thread-safe.
 */
#ifndef TLQ_H
#define TLQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tlq_ctx_s* tlq_ctx;
typedef struct tlq_circuit_s* tlq_circuit;
typedef struct tlq_ham_s* tlq_ham;
typedef uint64_t tlq_ticket;

typedef enum {
    TLQ_OK = 0,
    TLQ_EINVAL = 1,       /* malformed argument or descriptor */
    TLQ_ENOMEM = 2,       /* device memory budget or allocation exceeded */
    TLQ_EAGAIN = 3,       /* tlq_poll: request still pending */
    TLQ_ETIMEOUT = 4,     /* tlq_poll: waited timeout_us without completion */
    TLQ_ECUDA = 5,        /* a CUDA runtime call failed */
    TLQ_EKERNEL = 6,      /* a kernel reported an internal error word */
    TLQ_EUNSUPPORTED = 7  /* valid request outside what the library implements */
} tlq_status;

typedef enum {
    TLQ_FP32 = 0,      /* complex64 states, FP32 arithmetic; FP64 gate tables' source
                          angles and FP64 reductions across terms */
    TLQ_MIXED_TC = 1,  /* dense statevector path: each group of up to four rotations of a
                          forward pass is one 16 x 16 complex block applied on the tensor
                          cores (tcgen05, split-TF32 products, FP32 accumulation), and the
                          energy and gradient are divided by the computed <psi|psi>, which
                          cancels the tensor cores' truncating accumulation to first order;
                          the same accuracy contract as TLQ_FP32. The adjoint passes, the
                          causal-cone path and circuits of at most 10 qubits run their FP32
                          kernels in this mode. */
    TLQ_FP64_REF = 2   /* complex128 correctness mode of the same kernels (slow) */
} tlq_precision;

typedef enum { TLQ_RX = 0, TLQ_RY = 1, TLQ_RZ = 2, TLQ_RZZ = 3, TLQ_CZ = 4 } tlq_gate_kind;

/* One gate. q1 is the second qubit of RZZ/CZ (ignored, conventionally -1, for
 * one-qubit gates). param = -1 selects the fixed `angle` (radians); CZ ignores both. */
typedef struct {
    int32_t kind;     /* tlq_gate_kind */
    int32_t q0, q1;
    int32_t param;
    double angle;
} tlq_gate;

/* One Pauli term coeff * P, P = prod_k letter_k acting on sites[k].
 * `paulis` holds nsites letters from {'X','Y','Z'} (no terminator needed). */
typedef struct {
    double coeff;
    int32_t nsites;
    const int32_t* sites;
    const char* paulis;
} tlq_term;

typedef struct {
    int device;              /* CUDA device ordinal; -1 = host-only context (validation and
                                planning only; every compute call returns TLQ_EUNSUPPORTED) */
    size_t mem_budget;       /* bytes of device memory the context may hold (0 = 80% of free) */
    int max_slots;           /* tlq_submit: requests admitted concurrently (0 = 64) */
    tlq_precision default_prec;
    int fuse_k;              /* reserved (fused block size); 0 = default */
} tlq_config;

/* Create a context on cfg->device: one CUDA stream, a device workspace and, for the
 * serving calls, a scheduler thread started on first tlq_submit. cfg may be NULL
 * (device 0, defaults). *out is set only on TLQ_OK. */
tlq_status tlq_init(const tlq_config* cfg, tlq_ctx* out);

/* Wait for all submitted work, stop the scheduler and free every device resource of
 * the context. Circuits and Hamiltonians created on it must not be used afterwards
 * (destroy them first; tlq_destroy also frees any that are left). NULL is a no-op. */
tlq_status tlq_destroy(tlq_ctx ctx);

/* Validate and copy a gate list (Sec. 2: circuits composed of gates).
 * EINVAL when: n_qubits < 1 or > 2^20; a qubit is out of [0, n_qubits); q0 == q1 for a
 * two-qubit gate; an unknown kind; param >= n_params or param < -1; n_gates < 0.
 * The execution path (per-term light cones for nearest-neighbour circuits, a dense
 * statevector otherwise) is chosen when the circuit is first paired with a Hamiltonian. */
tlq_status tlq_circuit_create(tlq_ctx ctx, int32_t n_qubits, const tlq_gate* gates, int32_t n_gates,
                              int32_t n_params, tlq_circuit* out);
tlq_status tlq_circuit_destroy(tlq_circuit c);

/* Validate and copy a Pauli-sum Hamiltonian (Sec. 3: H as a sum of local terms, never a
 * dense matrix). EINVAL when: a site is out of range; a letter is not X/Y/Z; a site
 * repeats inside one term; nsites < 1; n_terms < 1. */
tlq_status tlq_hamiltonian_create(tlq_ctx ctx, int32_t n_qubits, const tlq_term* terms, int32_t n_terms,
                                  tlq_ham* out);
tlq_status tlq_hamiltonian_destroy(tlq_ham h);

/* Forward pass (Sec. 3, <H>): energy[b] = <psi(theta_b)| H |psi(theta_b)> for b < B.
 * theta: host, row-major [B][n_params] FP64. energy: host [B] FP64. Synchronous. The device
 * work of a call (input copy, kernels, output copies) is captured once as a CUDA graph per
 * (circuit, Hamiltonian, B, precision, gradient or not) and replayed by later calls with the
 * same key, unless kernel profiling is enabled. Circuits of at most 10 qubits (FP32) are
 * evaluated by one small kernel that applies the gates in order to the whole state; their
 * energies agree with tlq_expectation_grad's to rounding, not bit for bit.
 * EINVAL: B <= 0, null pointers, circuit/Hamiltonian qubit counts differ.
 * ENOMEM: the call's workspace exceeds the context's budget. */
tlq_status tlq_expectation(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B,
                           tlq_precision prec, double* energy);

/* Forward + backward (Sec. 3, <H> and nabla <H>): as tlq_expectation plus
 * grad[b][p] = dE_b / dtheta_p (host, row-major [B][n_params], FP64). Synchronous.
 * A parameter shared by several gates gets the sum of their derivatives; parameters no
 * gate uses get 0. Both paths compute the gradient by the adjoint method; on the dense
 * statevector path it holds a second 2^n complex64 state (lambda = H psi) while it runs,
 * and TLQ_FP64_REF returns TLQ_EUNSUPPORTED there (that path is FP32 only). */
tlq_status tlq_expectation_grad(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B,
                                tlq_precision prec, double* energy, double* grad);

/* Device-pointer variant for callers that keep tensors on the GPU (the PyTorch path):
 * theta_dev [B][n_params], energy_dev [B], grad_dev [B][n_params] (nullable: energy
 * only) are device pointers on the context's device; all work is enqueued on
 * cuda_stream (a cudaStream_t; NULL = the context's own stream) and the call returns
 * without synchronising. The outputs are valid once that stream reaches this point.
 * The workspace is owned by the context: do not enqueue a second call on another
 * stream until this one has completed. */
tlq_status tlq_expectation_grad_dev(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev,
                                    int32_t B, tlq_precision prec, double* energy_dev, double* grad_dev,
                                    void* cuda_stream);

/* Allocation-free variant of tlq_expectation_grad_dev (FP32, nearest-neighbour circuits).
 * The paper has no counterpart: this serves callers that cannot allocate device memory
 * when they evaluate -- e.g. a host application whose own allocator owns the whole GPU and
 * accounts for every byte, or a latency-critical loop that cannot take the implicit device
 * synchronisation of cudaMalloc. Arguments are as for tlq_expectation_grad_dev (device
 * pointers; grad_dev may be NULL for energies only; work enqueued on cuda_stream, NULL =
 * the context's stream; no synchronisation). All working memory (a copy of the plan, the
 * work list, gate tables, per-term partials, gradient slots, counters) comes from one
 * 16 MiB array compiled into the library, which every GPU that loads the library holds
 * until the process exits; no cudaMalloc/cudaFree or other allocating routine is called.
 * The first call on a device looks up that array's device address (cudaGetSymbolAddress).
 * Calls share the array:
 * calls whose work overlaps on the GPU race and must be serialised by the caller (for
 * example by enqueueing them on one stream: each call enqueues its copies and launches as
 * one unit, so calls made from several threads onto one stream do not interleave). Plans and work lists are cached on the host
 * (16 entries, keyed by context, device, batch size, gradient flag and the full circuit and
 * Hamiltonian contents); the cache is safe to use from several threads and contexts, and a
 * context's entries are dropped by tlq_destroy. The call does not synchronise, so it cannot
 * return a kernel's error status: if a kernel of the call finds an inconsistent work item,
 * every energy (and gradient entry) the call writes is NaN instead.
 * TLQ_ENOMEM (with the byte count in tlq_last_error) when the call needs more than the
 * array holds; TLQ_EUNSUPPORTED for circuits that need the dense statevector path. */
tlq_status tlq_expectation_grad_static(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev, int32_t B,
                                       double* energy_dev, double* grad_dev, void* cuda_stream);

/* Serving (continuous batching): enqueue one request; returns at once with a ticket.
 * theta: host [B][n_params]; energy: host [B]; grad: host [B][n_params] when want_grad.
 * The buffers are borrowed until tlq_poll returns for the ticket; the circuit and the
 * Hamiltonian must stay alive until then too. Planning runs on the library's planner
 * threads (plans are cached by circuit/Hamiltonian structure). Requests are admitted as
 * request slots and device memory free up, packed with the other admitted requests into
 * batched launches, and overlap on the device with batches already in flight. Results do
 * not depend on what else is in the batch. The call itself fails with EINVAL as
 * tlq_expectation does (and ENOMEM for B above 8192); failures found while planning --
 * EUNSUPPORTED for circuits that need the dense statevector path, ENOMEM for a request
 * that can never fit half of the memory budget -- are returned by tlq_poll. */
tlq_status tlq_submit(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B, int want_grad,
                      tlq_precision prec, double* energy, double* grad, tlq_ticket* out);

/* TLQ_OK: done (outputs written, ticket retired); TLQ_EAGAIN: pending and
 * timeout_us == 0; TLQ_ETIMEOUT: still pending after timeout_us microseconds (a negative
 * timeout waits until completion); any other status: the request failed (ticket retired,
 * message in tlq_last_error). EINVAL for an unknown or already retired ticket. */
tlq_status tlq_poll(tlq_ctx ctx, tlq_ticket t, int64_t timeout_us);

/* Thread-local message of the calling thread's last failure ("" if none). */
const char* tlq_last_error(tlq_ctx ctx);

/* ---- introspection (host-side; no device work) -------------------------------------- */

/* Partial trace of a pure state (Sec. 2: partial traces of density operators; Sec. 3,
 * Fig. 1 left: full-rank partial traces from n to m qubits): for rho = |psi><psi| and the
 * kept qubits A = keep[0..m) (any order, distinct),
 *   rho_A[i][j] = sum_k psi(i, k) conj(psi(j, k)),
 * where psi(i, k) is the amplitude whose kept qubits hold the bits of i and whose traced
 * qubits hold the bits of k. Bit q of a state index is qubit q; bit t of i (and j) is the
 * t-th lowest kept qubit, bit u of k the u-th lowest traced qubit.
 * psi_dev: device, 2^n complex64 as interleaved (re, im) floats, 1 <= n <= 31, not modified.
 * rho_dev: device, 2^m x 2^m complex64 row-major (interleaved), 1 <= m <= min(n, 15); the
 * full matrix is written and is exactly Hermitian (real diagonal; each entry below the
 * diagonal is the conjugate of its mirror). keep: host array of m qubit indices, read
 * during the call.
 * Work is enqueued on cuda_stream (NULL = the context's stream) without synchronising; a
 * workspace of about 8 * 2^n bytes is taken from the context (plus 8 * 4^m bytes per k-range
 * split when the output is small). Outputs of m >= 7 run on the tensor cores (TF32 operands
 * split into high and low parts, three products each, FP32 accumulation: about 2^-20
 * relative error per product), smaller ones on FP32 CUDA cores; results are deterministic.
 * A tensor-core wait that gives up (after about a second) leaves the output incomplete and
 * sets the context's kernel error word, which tlq_reduced_density reports as EKERNEL.
 * EINVAL: NULL pointers, n or m out of range, a kept qubit out of range or repeated. */
tlq_status tlq_partial_trace_dev(tlq_ctx ctx, const float* psi_dev, int32_t n, const int32_t* keep, int32_t m,
                                 float* rho_dev, void* cuda_stream);

/* Reduced density operator of a circuit's output state on the kept qubits (Sec. 2):
 * rho_A of U(theta)|0..0> as above, for one parameter set theta (host, [n_params] FP64).
 * rho: host, 2^m x 2^m complex128 row-major as interleaved (re, im) doubles, 1 <= m <= 14.
 * Circuits on n <= 31 qubits run on the dense statevector path; a nearest-neighbour circuit
 * on more qubits is simulated on the window of the kept qubits' backward light cone (exact:
 * gates outside the cone do not change rho_A), which must span at most 31 qubits.
 * Synchronous; FP32 state and sums. EINVAL as for tlq_partial_trace_dev; EUNSUPPORTED for a
 * non-local circuit on more than 31 qubits or a light cone wider than 31 qubits. */
tlq_status tlq_reduced_density(tlq_ctx ctx, tlq_circuit c, const double* theta, const int32_t* keep, int32_t m,
                               double* rho);

/* Exact matrix-product-state (tensor-train) route (Sec. 2: MPS / tensor-train factorized
 * representations; Sec. 1: contraction of factorized tensors; Sec. 3: <H> and its full
 * gradient), for chain circuits: every RZZ / CZ acts on neighbours (q, q+1). Each such gate is
 * split exactly into two products of single-site operators, so the bond between q and q+1
 * carries one bit per two-qubit gate on that pair: bond dimension 2^(gates on the pair), no
 * truncation, result exact up to rounding. The energies E[b] and, when grad is not NULL, the
 * gradients grad[b][p] are those of tlq_expectation_grad (same definitions, same layouts:
 * theta [B][n_params], energy [B], grad [B][n_params], row-major FP64), computed from the MPS
 * by left and right environment sweeps and one pass per site. The Hamiltonian's terms may
 * span any sites (a term costs one transfer per site of its span). Precision: TLQ_FP32 (and
 * TLQ_MIXED_TC) keep site tensors and environments in complex64, TLQ_FP64_REF in complex128;
 * the term and gradient sums are FP64 in a fixed order (results are deterministic).
 * tlq_mps_expectation_grad_dev: device pointers, work enqueued on cuda_stream (NULL = the
 * context's stream) without synchronising; tlq_mps_expectation_grad: host pointers,
 * synchronous. Workspace from the context: about B * elems_per_set complex entries (see
 * tlq_plan_mps_info) plus per-set tables.
 * EINVAL: NULL handles or pointers, B <= 0, qubit counts that differ, n * B >= 2^31.
 * EUNSUPPORTED: a two-qubit gate on non-neighbouring qubits, more than 6 two-qubit gates on
 * one pair (5 in FP64), more than 48 gates on one qubit, more than 32 terms covering one qubit.
 * ENOMEM: the workspace exceeds the context's memory budget. */
tlq_status tlq_mps_expectation_grad_dev(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta_dev, int32_t B,
                                        tlq_precision prec, double* energy_dev, double* grad_dev, void* cuda_stream);
tlq_status tlq_mps_expectation_grad(tlq_ctx ctx, tlq_circuit c, tlq_ham h, const double* theta, int32_t B,
                                    tlq_precision prec, double* energy, double* grad);

/* MPS plan of (c, h): the largest bond's bit count *max_bond_bits (bond dimension
 * 2^max_bond_bits), the complex entries one parameter set's site tensors, environments and
 * term chains take (*elems_per_set), and the contraction flops per parameter set of an
 * energy-only call (*flops_energy) and of an energy + gradient call (*flops_grad), 8 per
 * complex multiply-add of the environment transfers and site contractions. Any pointer may be
 * NULL. Works on host-only contexts; EUNSUPPORTED as for tlq_mps_expectation_grad. */
tlq_status tlq_plan_mps_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* max_bond_bits, int64_t* elems_per_set,
                             double* flops_energy, double* flops_grad);

typedef enum { TLQ_PATH_CONE = 0, TLQ_PATH_DENSE = 1 } tlq_path;

/* Plan summary for (c, h): the chosen path; for the cone path, per term t < n_terms the
 * window start lo[t] and width w[t] (clipped to the chain) and the number of gates in its
 * cone ngates[t]. Any of lo/w/ngates may be NULL. Works on host-only contexts. */
tlq_status tlq_plan_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* path, int32_t* lo, int32_t* w,
                         int32_t* ngates);

/* Work-cone statistics for (c, h) on the cone path. Terms whose causal cone lies inside
 * another term's window are measured on that window, so the plan has *ncones <= n_terms
 * work cones. For cone k: rotations nrot[k], diagonal layers ndiag[k] and parametrised
 * diagonal gates npdiag[k] it simulates, the width weff[k] of its window (padded to at
 * least 8 qubits), its true width wtrue[k], the number of terms nterms[k] measured on it,
 * and split[k] = 1 when the kernel runs it as two independent branches of weff[k] - 1 qubits
 * (the window's top qubit carries gates of the first layer only and no measured term, so the
 * states with that qubit 0 and 1 never mix; their energies and gradients add up). Arrays
 * must hold n_terms entries; any pointer may be NULL. Used to count the algorithmic work of a
 * call. TLQ_EUNSUPPORTED on the dense path. */
tlq_status tlq_plan_cone_stats(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* ncones, int32_t* nrot, int32_t* ndiag,
                               int32_t* npdiag, int32_t* weff, int32_t* wtrue, int32_t* nterms, int32_t* split);

/* Dense statevector plan of (c, h): the state's qubit count *n_eff (n, at least 12); the
 * number of streaming passes *n_passes the adjoint makes over the state (in reverse); the
 * number *n_fwd_passes the forward makes -- with two or more layers the forward first writes
 * layer 0's result directly (one write of the state, layer 0 acting on |0..0>) and then runs
 * a schedule of the remaining layers; the number of reverse passes *n_rev_store that write psi
 * and lambda back (the others only read: the first pass, and passes that only give layer 0's
 * rotation gradients); the number of Pauli strings with X/Y letters *n_xterms
 * measured by separate sweeps; and *fused = 1 when the fused passes are used (0: the plan's
 * staged data exceed the pass kernel's shared memory and the plain per-gate sweeps run
 * instead). Any out pointer may be NULL. TLQ_EUNSUPPORTED when (c, h) has no dense plan (more
 * than 31 qubits). */
tlq_status tlq_plan_dense_info(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int32_t* n_eff, int32_t* n_passes,
                               int32_t* n_fwd_passes, int32_t* n_rev_store, int32_t* n_xterms, int32_t* fused);

/* HBM bytes that one evaluation (one parameter set) on the dense statevector path moves by
 * its pass schedule in precision `prec`, with (want_grad != 0) or without the gradient: the
 * start state written once (none when the first forward pass generates layer 0's product
 * state itself), each forward pass reading and writing the 2^n complex64 state (an
 * energy-only evaluation without X/Y terms does not write the final state back), one read per
 * term with X/Y letters, and with the gradient lambda written, the X/Y strings' gather sweep
 * (two reads, one write) and each reverse pass reading psi and lambda and writing both back
 * unless nothing after it needs them. Works on host-only contexts; EUNSUPPORTED without a
 * dense plan. Used as the algorithmic byte count of the dense path's roofline. */
tlq_status tlq_plan_dense_bytes(tlq_ctx ctx, tlq_circuit c, tlq_ham h, int want_grad, tlq_precision prec,
                                double* bytes);

/* Kernel timing for benchmarks. While enabled, every compute call records CUDA events
 * around its dominant kernel (the batched cone kernel, the dense pass sequence, the partial
 * trace's kernels, or all five kernels of the MPS route) on the stream it launches on. tlq_profile_last waits for the last call's events and returns
 * that kernel's device time in milliseconds and the number of kernels the call launched. */
tlq_status tlq_profile_enable(tlq_ctx ctx, int on);
tlq_status tlq_profile_last(tlq_ctx ctx, float* kernel_ms, int32_t* launches);

/* Serving statistics since the context was created: completed requests, latency
 * percentiles (seconds from tlq_submit to completion on the device) and the mean number
 * of requests per batched launch. Any out pointer may be NULL. */
tlq_status tlq_serving_stats(tlq_ctx ctx, int64_t* completed, double* p50_s, double* p99_s,
                             double* mean_batch);

/* Version of this ABI (major * 10000 + minor * 100 + patch). */
int32_t tlq_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TLQ_H */
