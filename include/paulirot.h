/*
 * paulirot.h -- C ABI of the GB300 Pauli-rotation statevector library
 * (libpaulirot.so, CUDA kernels for sm_103a plus host C++).
 *
 * What it computes (arXiv 2602.09020):
 *   * R_P(theta) = exp(-i theta/2 P) on an n-qubit statevector, every rotation
 *     pairing amplitude k with f_P(k) = k XOR x and the phase
 *     i^{nY} (-1)^{popc(k & z)} (Sec. "Multi-qubit rotations in a fullstate
 *     simulator" and App. "Amplitude update rule for multi-qubit rotations").
 *   * Pauli gates kept in a Pauli frame Q, so that the represented state is
 *     |psi> = Q |phi> and a rotation about P acts on |phi> about Q^dag P Q =
 *     +-P (Sec. "Pauli Frame as a Lookup Table", Eq. single_to_multirot, with
 *     the frame restricted to Pauli gates).
 *   * <psi|sum_j c_j P_j|psi> = sum_j c_j <phi|Q^dag P_j Q|phi>
 *     (Sec. "Extraction of Expectation Values", Eqs. Fmap and chfsexp).
 *   * First-order Trotter products, Eq. (trotter), and a symmetric
 *     second-order product (not in the paper; see trotter_expand).
 *   * dE/dtheta_j of E = <psi|H|psi> by an adjoint sweep (not in the paper).
 *   * General Clifford frames in the backward interpretation (Sec.
 *     "Clifford-Fullstate Hybrid Simulator"): Clifford gates update a host
 *     frame, non-Clifford rotations run on the state about the rewritten
 *     axis, the frame is applied to the state as <= 4n rotations by pi/2
 *     (App. "Efficiently implementing Clifford unitaries with multi-qubit
 *     rotations"), and Pauli measurement / qubit preparation act on the
 *     rewritten axis (App. "Complete workflow of the hybrid Clifford
 *     fullstate simulation"); see the cliff_* and cfhs_* calls.
 *
 * Conventions
 *   * qubit j is bit j of the amplitude index (qubit 0 least significant);
 *   * a Pauli string is a pair of uint64 masks (x, z): X on bits x & ~z,
 *     Z on z & ~x, Y on x & z; bits >= n must be zero;
 *   * theta is the angle of exp(-i theta/2 P), FP64;
 *   * amplitudes are interleaved (re, im): SV_C128 = 2 x double per amplitude,
 *     SV_C64 = 2 x float.  Angle trigonometry and every reduction are FP64 in
 *     both modes.
 *
 * Errors: every function returns an int status (SV_OK = 0, negative on
 * failure) and never aborts or exits.  sv_last_error() gives a thread-local
 * message for the last failure on the calling thread.
 *
 * Threads: a handle (state, plan or Clifford frame) is used by one host
 * thread at a time.  The library's shared state (tuned fusion depths, the
 * cached batched launch, phase tables, per-kernel grid sizes) is guarded, so
 * different handles may be driven from different threads.
 *
 * Ownership: host arrays passed in are read (or written) before the call
 * returns and stay owned by the caller.  Device memory made by sv_alloc and
 * all internal scratch belong to the library and are released by sv_free.
 * sv_wrap borrows caller memory, which must outlive the handle.
 *
 * Streams: all device work of a handle is enqueued on its CUDA stream
 * (cudaStream_t passed as void*, NULL = legacy default stream).  Calls that
 * return host values (expval_pauli_sum, rotation_grads, sv_to_host, ...)
 * synchronise that stream before returning.
 */
#ifndef PAULIROT_H
#define PAULIROT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define SV_OK 0
#define SV_EINVAL (-1)       /* bad argument: null pointer, mask bit >= n, NaN/Inf angle, ... */
#define SV_ENOMEM (-2)       /* device or host allocation failed, or n too large */
#define SV_ECUDA (-3)        /* a CUDA runtime call failed (message has the CUDA error) */
#define SV_ETIMEOUT (-4)     /* a bounded device wait gave up (batched launch) */
#define SV_EUNSUPPORTED (-5) /* valid request this build does not handle */
#define SV_EIO (-6)          /* a checkpoint file could not be written or read, or is corrupt */

/* ---- amplitude types ------------------------------------------------------- */
#define SV_C128 0 /* complex128: 16 bytes per amplitude, n <= 33 */
#define SV_C64 1  /* complex64:   8 bytes per amplitude, n <= 34 */

typedef struct sv_state sv_state; /* opaque: amplitudes, n, dtype, stream, frame, scratch */
typedef struct sv_plan sv_plan;   /* opaque: a rotation list compiled into fused runs */

/* Thread-local description of the last failure on this thread ("" if none). */
const char *sv_last_error(void);

/* Library version, (major << 16) | minor. */
int sv_version(void);

/* ---- statevector handles ----------------------------------------------------- */

/* Allocate a 2^n-amplitude state on the current CUDA device, set to |0..0>,
 * frame = identity.  dtype is SV_C128 or SV_C64.  SV_ENOMEM if n exceeds the
 * dtype's limit or the allocation fails (nothing is left allocated). */
int sv_alloc(sv_state **out, int n_qubits, int dtype, void *cuda_stream);

/* Wrap caller-owned device memory of 2^n amplitudes (16-byte aligned); the
 * contents are taken as |phi> with the identity frame.  Not freed by sv_free. */
int sv_wrap(sv_state **out, void *dev_amps, int n_qubits, int dtype, void *cuda_stream);

/* Release the handle (and the amplitudes if sv_alloc made them). NULL is OK. */
int sv_free(sv_state *sv);

/* Change the stream used by later calls on this handle. */
int sv_set_stream(sv_state *sv, void *cuda_stream);

/* Device pointer to the stored amplitudes |phi> (not materialised). */
int sv_device_ptr(sv_state *sv, void **out);

/* Query n and dtype. */
int sv_info(sv_state *sv, int *n_qubits, int *dtype);

/* |phi> = |k>, frame = identity. */
int sv_set_basis_state(sv_state *sv, uint64_t k);

/* |phi> = host amplitudes (2^n of the handle's dtype), frame = identity. */
int sv_from_host(sv_state *sv, const void *host_amps);

/* Copy amplitudes to host memory (2^n of the handle's dtype).  With
 * materialize_frame != 0 the frame is first applied to the device state (see
 * sv_materialize), so the copy is |psi>; with 0 the copy is |phi>. */
int sv_to_host(sv_state *sv, void *host_amps, int materialize_frame);

/* Apply the frame Q to the stored amplitudes in place (|phi> <- Q|phi>, one
 * pass), then reset the frame: the represented state |psi> is unchanged
 * (paper, Sec. "Extraction of Expectation Values": (F, Phi) -> (F_origin, Psi),
 * here for a Pauli-only frame with its exact phase). */
int sv_materialize(sv_state *sv);

/* Copy state and frame of src into dst (same n and dtype). */
int sv_copy(sv_state *dst, const sv_state *src);

/* ---- checkpoint / resume (not in the paper) -------------------------------------
 * sv_save writes the amplitudes phi as they lie in device memory, the Pauli
 * frame Q (the represented state Q phi is restored exactly, nothing is
 * materialised) and a caller tag (e.g. the index of the next plan of a Trotter
 * sequence compiled as several plans) to path, through path + ".tmp" renamed
 * over it, so an existing checkpoint is replaced only by a complete one.  The
 * file is a 72-byte header (magic "PRCKPT01", version, n, dtype, frame, tag,
 * sizes, FNV-1a checksums of the amplitudes and of the header) followed by
 * the amplitudes.  It waits for the handle's stream.  SV_EIO on a file error.
 *
 * sv_load reads a checkpoint into a handle of the same n and dtype: SV_EINVAL
 * if the file is not a checkpoint or its n / dtype differ (nothing changed),
 * SV_EIO if it is truncated or a checksum fails (header problems change
 * nothing; an amplitude checksum failure is found after the copy, so the
 * amplitudes are then unspecified and the frame unchanged).  On success the
 * frame is the saved one and *out_tag (nullable) the saved tag. */
int sv_save(sv_state *sv, const char *path, uint64_t tag);
int sv_load(sv_state *sv, const char *path, uint64_t *out_tag);

/* ---- Pauli frame (host only, O(1) per call) --------------------------------- */

/* Reset the frame to the identity. */
int frame_reset(sv_state *sv);

/* Apply the Pauli gate pauli ('X', 'Y' or 'Z') on qubit to the represented
 * state by updating the frame only: Q <- G Q with the exact phase (paper,
 * Fig. "CFHS gate flow": Clifford gates update F, here Pauli gates). */
int frame_apply_pauli(sv_state *sv, char pauli, int qubit);

/* Read the frame Q = i^phase X^xq Z^zq (phase in 0..3). */
int frame_get(sv_state *sv, uint64_t *xq, uint64_t *zq, int *phase);

/* ---- rotations ----------------------------------------------------------------- */

/* Apply R_{P_0}(angles[0]) first, then P_1, ... to the represented state.
 * R_P(theta) = exp(-i theta/2 P) = cos(theta/2) I - i sin(theta/2) P, applied
 * as the pair update of amplitudes k and k XOR x (paper, Sec. "Multi-qubit
 * rotations in a fullstate simulator" and App. "Amplitude update rule for
 * multi-qubit rotations").  Host arrays of length count.  Each rotation is rewritten by the frame
 * (sign flip where P anticommutes with Q), the list is compiled into fused
 * runs (the runs and launches of plan_create with fusion_depth = -1 followed by
 * plan_apply, so the result is the same bit for bit) and launched on the
 * handle's stream while the rest of the list is still being compiled: runs go
 * out in batches, their records copied from pinned staging into a device
 * buffer that the handle keeps for later calls (grown as needed, released by
 * sv_free).  The host arrays may be reused when the call returns; it returns
 * before the device work finishes. */
int apply_pauli_rotations(sv_state *sv, const uint64_t *x, const uint64_t *z,
                          const double *angles, size_t count);

/* Compile a rotation list once for states of n qubits and this dtype: the
 * rotations of Sec. "Multi-qubit rotations in a fullstate simulator", in list
 * order, grouped into fused runs (one pass over the amplitudes per run; the
 * grouping is this library's, the paper applies one rotation per pass).
 * fusion_depth = maximum dimension of the span of x-masks fused into one
 * pass (0..5; -1 = the depth plan_tuned_depth reports: the autotuned one for
 * (n, dtype) if one is recorded, else 3 for complex128 and 4 for complex64).  The plan's device buffers
 * are uploaded on cuda_stream; plan_apply then launches kernels only (no
 * host-to-device copy), so it can be captured into a CUDA graph. */
int plan_create(sv_plan **out, int n_qubits, int dtype, const uint64_t *x, const uint64_t *z,
                const double *angles, size_t count, int fusion_depth, void *cuda_stream);

/* Apply a plan to a state (same n and dtype): its rotations in list order, as
 * apply_pauli_rotations would (Sec. "Multi-qubit rotations in a fullstate
 * simulator").  The frame signs are taken from
 * the handle's frame at call time (a captured graph replays the frame it was
 * captured with).  Updates the handle's frame on the host. */
int plan_apply(sv_state *sv, sv_plan *plan);

int plan_free(sv_plan *plan);

/* ---- fusion-depth autotuner ----------------------------------------------------
 * The best fusion depth trades HBM passes against per-pass work and depends on
 * the kernel variant, n and the rotation list (fused pass of the paper's
 * Sec. "Implementation"; the depth is not fixed there).  A process-wide table
 * maps (n, dtype) to a depth that plan_create(-1) and apply_pauli_rotations
 * use.  If the environment variable PAULIROT_TUNE_CACHE names a file, the table
 * is read from it before its first use and written back after each
 * plan_autotune; the file holds "<c64|c128> <n> <depth>" lines.
 *
 * plan_autotune compiles x/z/angles (count rotations, as for plan_create) at
 * every depth 1..max_depth (max_depth <= 0 means 5; capped at n), applies each
 * plan once untimed and then reps times (reps <= 0 means 3) in two interleaved
 * rounds on sv's stream, timed with CUDA events, and records the fastest
 * depth for (sv's n, sv's dtype); ties go to the smaller depth.  sv is the
 * scratch: its represented state is overwritten (evolved by the timed
 * applications), so initialise it afterwards.  out_ms (nullable, 5 doubles)
 * receives the milliseconds per application for depths 1..5, -1 where not
 * timed.  Batched launches take plans of depth <= 4: tune with max_depth 4
 * for them.  Synchronizes sv's stream. */
int plan_autotune(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *angles, size_t count,
                  int max_depth, int reps, int *out_depth, double *out_ms);

/* Fusion depth for a batched launch (batch_run), timed on the launch itself:
 * for every depth 1..max_depth (max_depth <= 0 or > 4 means 4, the batched
 * kernel's limit) each state's list x[i], z[i], angles[i] (counts[i]
 * rotations) is compiled as by plan_create, the batch is run once untimed and
 * then reps times (reps <= 0 means 3) with CUDA events on states[0]'s stream
 * (use_graph as for batch_run).  The fastest depth is recorded for every
 * (n, dtype) in the batch (replacing single-state entries for those sizes),
 * so plan_create(-1) compiles for it; ties go to the smaller depth.  The
 * states are scratch: overwritten.  out_ms (nullable, 4 doubles) receives
 * the best milliseconds per batched launch for depths 1..4, -1 where not
 * timed. */
int batch_autotune(sv_state **states, const uint64_t *const *x, const uint64_t *const *z,
                   const double *const *angles, const size_t *counts, size_t count, int max_depth, int reps,
                   int use_graph, int *out_depth, double *out_ms);

/* The depth plan_create(-1) would use for (n, dtype) (capped at n);
 * *out_tuned (nullable) = 1 if it comes from the table, 0 if it is the default. */
int plan_tuned_depth(int n_qubits, int dtype, int *out_depth, int *out_tuned);

/* Record depth (1..5) for (n, dtype) in the table, or remove the entry
 * (depth = -1).  Host only; does not write the cache file. */
int plan_set_tuned_depth(int n_qubits, int dtype, int depth);

/* Merge the entries of a cache file into the table (a missing file is empty;
 * a malformed one is SV_EINVAL and changes nothing), or write the table to a
 * file (through a temporary file of the calling process renamed over it).
 * Host only. */
int plan_tune_cache_load(const char *path);
int plan_tune_cache_save(const char *path);

/* The runs a plan is made of, computed on the host only (no device work):
 * the same planning as plan_create with these arguments.  Runs cover the
 * rotations in list order, identity strings left out: run i holds the next
 * runs[i].count of them.  kind 0 = fused coset run (one pass; its x-masks
 * lie in the span of basis[0..d-1], a reduced basis whose vectors' highest set
 * bits are distinct), kind 1 = diagonal phase-sum run (x = 0 only; d = 0; at
 * most 1024 rotations and 128 distinct z patterns on index bits 0..8, so a
 * longer stretch of diagonal rotations becomes several runs).  A
 * run may hold no rotation when it only folds the running scale.  At most cap
 * runs are written; *out_runs (nullable) = all runs, *out_rotations (nullable)
 * = rotations after dropping identities. */
typedef struct sv_run_info {
  int32_t kind;
  int32_t d;
  int32_t count;
  int32_t reserved;
  uint64_t basis[5];
} sv_run_info;
int plan_inspect(int n_qubits, int dtype, const uint64_t *x, const uint64_t *z, const double *angles,
                 size_t count, int fusion_depth, sv_run_info *runs, size_t cap, size_t *out_runs,
                 size_t *out_rotations);

/* Plan statistics: number of rotations (after dropping identities), number
 * of fused runs, of which diagonal phase-sum runs.  Each run is one HBM pass
 * unless plan_sweeps says fewer. */
int plan_stats(const sv_plan *plan, size_t *n_rotations, size_t *n_runs, size_t *n_diag_runs);

/* *n_sweeps = passes over the state that plan_apply launches.  A complex64
 * plan with n >= 13 applies pairs of consecutive runs in one chained pass when
 * their spans and index bits 0..3 fit in 12 dimensions (Sec. "Multi-qubit
 * rotations in a fullstate simulator": each rotation pairs k with k ^ x inside
 * a coset of its run's span, so a coset of the joint span is closed under both
 * runs); then n_sweeps < n_runs.  Setting the environment variable
 * PAULIROT_CHAIN=0 before plan_create turns chaining off (same results, bit for
 * bit).  SV_EINVAL for a null argument. */
int plan_sweeps(const sv_plan *plan, size_t *n_sweeps);

/* ---- Trotter products (host) ----------------------------------------------------- */

/* Expand H = sum_j c_j P_j (T terms) into a rotation list.
 * order 1, Eq. (trotter): per step exp(-i c_j P_j dt) for j = 1..T, theta = 2 c_j dt.
 * order 2 (symmetric, not in the paper): per step theta = c_j dt for j = 1..T then
 * for j = T..1.  With merge != 0 neighbouring rotations about the same string
 * are merged into one (exact), which for order 2 joins the middle pair and
 * the pair across step boundaries.  Writes at most cap entries; *out_count is
 * the full length (call with cap = 0 to size the arrays). */
int trotter_expand(const uint64_t *x, const uint64_t *z, const double *c, size_t n_terms,
                   double dt, int steps, int order, int merge, uint64_t *out_x, uint64_t *out_z,
                   double *out_theta, size_t cap, size_t *out_count);

/* ---- reductions (FP64) ----------------------------------------------------------- */

/* out_energy = <psi|sum_j c_j P_j|psi> for the represented state, FP64, as
 * sum_j c_j <phi|Q^dag P_j Q|phi> with the Pauli frame Q (paper, Sec.
 * "Extraction of Expectation Values", Eqs. Fmap and chfsexp).
 * out_norm2 (nullable) = <psi|psi>.  Terms are grouped by x-mask and several
 * groups are evaluated per pass; partial sums are reduced in a fixed order,
 * so repeated calls give bitwise-equal results.  Arithmetic (n >= 4): every
 * per-term sum is an exact 64-bit integer sum on a grid 2^-S chosen from the
 * state's norm (S = 60 - ceil(log2 <psi|psi>)); complex64 products are exact
 * and rounded once onto the grid, complex128 products are 62-bit fixed-point
 * products on one exponent per 16 amplitudes, rounded once per transform
 * entry.  n < 4: FP64 products and sums.  SV_EUNSUPPORTED if the norm is not
 * finite (complex64: also if it exceeds about 2^52). */
int expval_pauli_sum(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *coeff,
                     size_t count, double *out_energy, double *out_norm2);

/* Allocation-free variant of expval_pauli_sum (the paper has no counterpart).
 * Same result and tolerance, but the call allocates nothing: no cudaMalloc,
 * cudaFree, pinned or heap memory.  It is meant for callers that cannot
 * allocate while they run -- code living inside a memory budget that an outer
 * framework has already carved up, latency-critical loops that cannot afford
 * the device-wide synchronisation an allocation can cause, and hosts that
 * forbid allocation after start-up.
 * Scratch: a fixed 4 MiB device array inside the library (held by every GPU
 * that loads the library until the process exits) plus a static host buffer.
 * Limits: at most 4096 terms and at most 1024 internal passes (groups of
 * terms whose x-masks span <= 4 dimensions); larger requests fail with
 * SV_EINVAL and a message, before any device work.
 * Set-up: the first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current.
 * Sharing: every call uses the same array and it keeps the last call's
 * contents; nothing in it needs to start at zero (every value is written before
 * it is read).  Calls that overlap on the GPU (other host threads, other streams)
 * race on the array; host threads are serialised by a lock, GPU work is not. */
int expval_pauli_sum_noalloc(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *coeff,
                             size_t count, double *out_energy, double *out_norm2);

/* dst <- sum_j c_j P_j applied to src's represented state (dst gets the
 * identity frame): each P_j maps amplitude k to k XOR x_j with the phase
 * i^{nY} (-1)^{popc(k & z_j)} (Sec. "Multi-qubit rotations in a fullstate
 * simulator"); the sum is the seed H psi of the adjoint gradient (not in the
 * paper).  Same n and dtype; dst must not be src. */
int apply_pauli_sum(sv_state *dst, sv_state *src, const uint64_t *x, const uint64_t *z,
                    const double *coeff, size_t count);

/* ---- adjoint gradient (not in the paper) -------------------------------------------- */

/* E = <psi|H|psi> with psi = R_{n_rot-1} ... R_0 psi0 (psi0 = the represented
 * state of the handle, left unchanged), and out_grads[j] = dE/dtheta_j for all
 * j, FP64.  Adjoint method: lambda = H psi, then for j = n_rot-1 .. 0:
 * g_j = Im <lambda|P_j|phi_j>, phi <- R_j^dag phi, lambda <- R_j^dag lambda,
 * walked in fused runs (consecutive rotations whose x-masks span <= 3
 * dimensions share one pass over phi and lambda).  Precision: complex128
 * applies the rotations in 64-bit fixed point with one exponent per coset of
 * each vector (resolution 2^-58 of the coset's largest component or finer) and
 * forms each coset's share of a gradient from fixed-point products summed
 * exactly, then in FP64 (a rotation of a diagonal stretch with |angle| > pi/2
 * takes an FP64 pass of its own); complex64 applies the rotations to phi and lambda in FP32
 * and sums every gradient term in FP64 (each FP32 term widened exactly; a term
 * below 1.2e-38 in magnitude counts as zero), and lambda = H psi sums each
 * element's coefficients exactly in 64-bit fixed point before one FP64
 * multiply-add per term group.  The two work states (phi, lambda; psi0's size
 * and type) are allocated on the first call, kept on psi0's handle for later
 * calls and released by sv_free(psi0). */
int rotation_grads(sv_state *psi0, const uint64_t *x, const uint64_t *z, const double *angles,
                   size_t n_rot, const uint64_t *hx, const uint64_t *hz, const double *hc,
                   size_t n_terms, double *out_energy, double *out_grads);

/* ---- gate-decomposed comparison path -------------------------------------------------- */

/* The same rotations applied the textbook way, one HBM pass per gate: basis
 * change per X/Y qubit (H, or Sdg then H), a CNOT ladder over the support,
 * Rz on its top qubit, the ladder and basis change undone (paper, Sec.
 * "Preliminaries of Hamiltonian Simulation", CNOT-staircase figure, 2(k-1)
 * CNOTs).  Frame signs are applied as in apply_pauli_rotations.  Used as the
 * same-GPU baseline; *out_gates (nullable) receives the number of gate
 * kernels launched. */
int apply_pauli_rotations_gates(sv_state *sv, const uint64_t *x, const uint64_t *z,
                                const double *angles, size_t count, size_t *out_gates);

/* ---- batched independent states (not in the paper) --------------------------------------- */

/* Apply plans[i] to states[i] for i < count (independent problems of uneven
 * sizes, all SV_C64 or all SV_C128) in one persistent launch on the stream of
 * states[0].  With use_graph != 0 the launch is captured into a CUDA graph
 * once per (states, plans) set and replayed.  Device waits are bounded: a
 * wait that runs out sets an error word and the call returns SV_ETIMEOUT. */
int batch_run(sv_state **states, sv_plan **plans, size_t count, int use_graph);

/* Options of batch_run_ex. */
typedef struct sv_batch_opts {
  double wait_timeout_s; /* limit on each device-side barrier wait, seconds (<= 0: 1.0) */
  int test_skip_arrival; /* testing only: one CTA of the first state that spans several CTAs
                            skips its first barrier arrival, so its peers' waits run out and
                            the call returns SV_ETIMEOUT (the failure path, without a fault) */
} sv_batch_opts;

/* batch_run with options (opts may be NULL).  Plans must use fusion_depth <= 4.
 * The work assignment and device buffers are cached for the last (states,
 * plans) set; with use_graph the launch is captured once into a CUDA graph and
 * replayed (the state handles' streams must not be the legacy default stream;
 * if capture is unavailable the launch is issued directly).  Each call
 * synchronises the stream of states[0] to read the error word. */
int batch_run_ex(sv_state **states, sv_plan **plans, size_t count, int use_graph, const sv_batch_opts *opts);

/* The batched launch's work assignment, computed on the host only by the rule
 * batch_run uses: state i has n_qubits[i] qubits and a plan of rotations[i]
 * rotations in passes[i] passes; the grid has grid_ctas CTAs.  A state's cost
 * is taken as 2^n (rotations + 4 (passes + 1)); states of n >= 16 costing more than
 * one CTA's share span several CTAs, the rest are packed onto CTAs.
 * out_ctas[i] (nullable) = CTAs state i spans (1 when packed with others);
 * *out_max_over_mean (nullable) = the largest CTA load over the mean load. */
int batch_inspect(const int *n_qubits, const size_t *rotations, const size_t *passes, size_t count, int grid_ctas,
                  int *out_ctas, double *out_max_over_mean);

/* Shape of the last batched launch: CTAs in the grid, states that spanned
 * several CTAs, and how it was launched: 1 = cooperative launch replayed from a
 * CUDA graph, 0 = no graph, negative = graph capture failed with that
 * cudaError_t (the cooperative launch then runs directly; a plain launch, whose
 * CTAs need not all be resident at once, is never used for the barriers). */
int batch_info(int *grid_ctas, int *multi_cta_states, int *graph_used);

/* ---- tracing (not in the paper) --------------------------------------------------------- */

/* One row per kernel name: launches, summed device time and algorithmic HBM
 * bytes (reads + writes the kernel must make, counted from its inputs). */
typedef struct sv_trace_row {
  char name[40];
  int64_t launches;
  double total_ms;
  double bytes; /* algorithmic HBM bytes, summed over launches */
  double flops; /* algorithmic floating-point operations (FMA = 2), summed */
} sv_trace_row;

/* Start recording a CUDA event pair around every kernel this handle launches
 * (on the handle's stream), including the kernels rotation_grads runs on the
 * handle's internal work states.  Recording adds two event records per launch. */
int sv_trace_start(sv_state *sv);

/* Trace modes.  SV_TRACE_LAUNCHES = sv_trace_start.  SV_TRACE_BLOCKS records one
 * event wherever the launched kernel changes (and one at sv_trace_stop): a
 * block of consecutive launches of one kernel runs as it does untraced
 * (chained passes overlap their prologues), and its elapsed time, which
 * includes anything else the handle enqueues inside the block, is
 * attributed to that kernel.  SV_EINVAL for another mode. */
#define SV_TRACE_LAUNCHES 0
#define SV_TRACE_BLOCKS 1
int sv_trace_start_ex(sv_state *sv, int mode);

/* Stop recording, synchronise the stream and aggregate per kernel name into
 * rows (at most cap; *n_rows = rows written).  Events are recycled. */
int sv_trace_stop(sv_state *sv, sv_trace_row *rows, int cap, int *n_rows);

/* ---- arithmetic-rate probe (not in the paper) ----------------------------------------- */

/* Launch one probe kernel on cuda_stream (no synchronisation) that keeps one
 * arithmetic pipe busy: `blocks` CTAs of 256 threads, each thread running eight
 * independent dependency chains of `iters` operations.  kind 0: FP64 fused
 * multiply-add; kind 1: 32 x 32 -> 64-bit signed integer multiply-add (the
 * operation the complex128 passes are built from); kind 2: packed FP32x2 fused
 * multiply-add (two FP32 FMAs per operation, the complex64 passes' update).
 * The caller times the launch
 * with CUDA events; *out_ops (nullable) = operations the launch performs
 * (blocks * 256 * iters * 8).  dev_out: caller-owned device buffer of
 * blocks * 256 eight-byte values, overwritten with the chains' results.
 * SV_EINVAL for another kind, blocks < 1, iters < 1 or a null buffer. */
int sv_probe_rate(int kind, int blocks, int iters, void *dev_out, void *cuda_stream, double *out_ops);

/* ---- Clifford-fullstate hybrid: general Clifford frames ------------------------------------ *
 *
 * Sec. "Clifford-Fullstate Hybrid Simulator".  A frame F represents a Clifford
 * unitary U in the backward interpretation, F = U^dag F_origin U (Eq. framemat):
 * entry j is the pair (U^dag Z_j U, U^dag X_j U), each a Hermitian Pauli string
 * with a sign.  The pair (F, state) represents psi = U phi (Eq. cfhsstate),
 * where phi is what the state handle holds (including its own Pauli frame).
 * Clifford gates only update F on the host; a rotation about P acts on phi
 * about F(P) = U^dag P U (Eq. single_to_multirot, Eq. Fmap); <P>_psi =
 * <F(P)>_phi (Eq. chfsexp).  Frames are host objects: the cliff_* calls do no
 * device work and need no GPU.  n <= 63. */
typedef struct sv_cliff sv_cliff; /* opaque: 2n signed Pauli strings */

/* Gate codes of a gate stream.  One-qubit gates use q0; CNOT (control q0,
 * target q1), CZ and SWAP use q0 and q1 (distinct).  RX/RY/RZ(q0, theta) =
 * exp(-i theta/2 sigma_q0) are the non-Clifford gates: they change the state,
 * not the frame. */
#define SV_CG_H 0
#define SV_CG_S 1   /* diag(1, i) */
#define SV_CG_SDG 2 /* diag(1, -i) */
#define SV_CG_X 3
#define SV_CG_Y 4
#define SV_CG_Z 5
#define SV_CG_CNOT 6
#define SV_CG_CZ 7
#define SV_CG_SWAP 8
#define SV_CG_RX 9
#define SV_CG_RY 10
#define SV_CG_RZ 11

/* Create an origin frame (U = I) on n qubits.  *out is owned by the caller and
 * released by cliff_free. */
int cliff_create(sv_cliff **out, int n_qubits);
int cliff_free(sv_cliff *f);
int cliff_reset(sv_cliff *f); /* back to the origin frame */
int cliff_num_qubits(const sv_cliff *f, int *out);

/* Apply a gate stream to the frame.  Clifford gates update F (each new entry a
 * product of old entries: U' = g U, F'(P) = F(g^dag P g)); each RX/RY/RZ gate
 * appends, in order, the rotation phi must undergo: masks of F(sigma_q0) and
 * the angle times its sign, to out_x/out_z/out_theta (capacity cap; *out_count
 * = rotations written).  The whole stream (gate codes, qubits, finite angles,
 * capacity) is checked first: SV_EINVAL leaves the frame unchanged.  gate, q0
 * are arrays of count; q1 may be NULL if no two-qubit gate occurs, theta if no
 * rotation gate occurs. */
int cliff_apply_gates(sv_cliff *f, const int *gate, const int *q0, const int *q1, const double *theta, size_t count,
                      uint64_t *out_x, uint64_t *out_z, double *out_theta, size_t cap, size_t *out_count);

/* F(P_k) = out_sign[k] * (string with masks out_x[k], out_z[k]) for the
 * Hermitian strings P_k = (x[k], z[k]) (Eq. Fmap).  Bits >= n: SV_EINVAL. */
int cliff_map_paulis(const sv_cliff *f, const uint64_t *x, const uint64_t *z, size_t count, uint64_t *out_x,
                     uint64_t *out_z, int *out_sign);

/* Entry `qubit` of F: U^dag Z_q U = ez_sign * (ez_x, ez_z) and
 * U^dag X_q U = ex_sign * (ex_x, ex_z). */
int cliff_entry(const sv_cliff *f, int qubit, uint64_t *ez_x, uint64_t *ez_z, int *ez_sign, uint64_t *ex_x,
                uint64_t *ex_z, int *ex_sign);

/* *out = 1 if F is the origin frame (U proportional to I), else 0. */
int cliff_is_origin(const sv_cliff *f, int *out);

/* Rotations R_1..R_m, R_k = exp(-i theta_k/2 P_k) with theta_k = +-pi/2 (that is
 * exp(-i pi/4 Q_k) for a signed Pauli Q_k), such that U = R_m ... R_1 up to a
 * global phase: applying R_1 first, then R_2, ... to phi gives U phi (App.
 * "Efficiently implementing Clifford unitaries with multi-qubit rotations";
 * construction in csrc/clifford.cu).  m <= 4n; cap >= 4n always suffices. */
int cliff_inverse_rotations(const sv_cliff *f, uint64_t *out_x, uint64_t *out_z, double *out_theta, size_t cap,
                            size_t *out_count);

/* Gate stream on (F, sv): Clifford gates update F, the rotation gates run on
 * sv's amplitudes through apply_pauli_rotations (one plan for the stream).
 * The frame and the state must have the same n. */
int cfhs_apply_gates(sv_state *sv, sv_cliff *f, const int *gate, const int *q0, const int *q1, const double *theta,
                     size_t count);

/* Multi-qubit rotations exp(-i theta_k/2 P_k) applied to psi = U phi: each
 * runs on sv about F(P_k) with its sign folded into the angle. */
int cfhs_apply_rotations(sv_state *sv, const sv_cliff *f, const uint64_t *x, const uint64_t *z, const double *theta,
                         size_t count);

/* <psi| sum_k c_k P_k |psi> = sum_k c_k <phi|F(P_k)|phi> (Eq. chfsexp), with the
 * reductions of expval_pauli_sum; *out_norm2 (nullable) = <phi|phi>. */
int cfhs_expval(sv_state *sv, const sv_cliff *f, const uint64_t *x, const uint64_t *z, const double *coeff,
                size_t count, double *out_energy, double *out_norm2);

/* Apply U to sv's amplitudes (the rotations of cliff_inverse_rotations) and
 * reset F to the origin frame, so that sv alone holds psi -- up to a global
 * phase, which a Clifford frame does not fix. */
int cfhs_materialize(sv_state *sv, sv_cliff *f);

/* Projective measurement of the Hermitian Pauli string P = (x, z) on
 * psi = U phi (f may be NULL: U = I), App. "Complete workflow of the hybrid
 * Clifford fullstate simulation" (Meas on the frame-rewritten axis).  The +1
 * probability is p = (1 + <psi|P|psi>/<psi|psi>)/2, from the reductions of
 * expval_pauli_sum; the outcome is +1 if u < p, else -1, with u a uniform
 * number in [0, 1) the caller draws (SV_EINVAL otherwise).  An outcome whose
 * probability is below 1e-14 is never taken.  The state becomes the
 * normalised projection (I + outcome P) psi / |(I + outcome P) psi| (one pass
 * over the amplitudes).  *out_outcome = +-1, *out_prob = its probability
 * (both nullable). */
int cfhs_measure_pauli(sv_state *sv, const sv_cliff *f, uint64_t x, uint64_t z, double u, int *out_outcome,
                       double *out_prob);

/* Prepare `qubit` in the +1 eigenstate of pauli ('X', 'Y' or 'Z') of psi =
 * U phi (f may be NULL), the workflow's Prep: measure that axis as
 * cfhs_measure_pauli does (uniform u) and, on outcome -1, apply an
 * anticommuting partner (Z for X and Y, X for Z) through the frames, so that
 * no extra pass runs.  *out_outcome (nullable) = the measured outcome. */
int cfhs_prepare_qubit(sv_state *sv, const sv_cliff *f, int qubit, char pauli, double u, int *out_outcome);

/* ---- global-qubit sharding (host planning) ---------------------------------------------- *
 *
 * Paper, Sec. "Multi-qubit rotations in a fullstate simulator", distributed-
 * memory paragraph: the amplitudes of n qubits are split over 2^g ranks by their
 * top g index bits (the global qubits); rank r holds the slice of L = n - g local
 * qubits whose top bits are r.  A rotation whose x-mask has no global bit acts
 * inside every slice; one whose global x-part is X pairs rank r with rank r ^ X,
 * and the two exchange slices.  A rank places the slice it receives beside its
 * own: the two form a state of L + 1 qubits (bit L = 0 for its own slice, 1 for
 * the partner's), its "pair state", on which the rotations of that exchange act
 * as ordinary rotations.  These calls rewrite rotations and terms for one rank;
 * they do no device work and need no GPU (the exchange and the passes are the
 * caller's: see paper_2602_09020_gb300/shard.py). */
typedef struct sv_shard_step {
  int32_t kind;    /* 0: on the rank's own slice (L qubits); 1: on its pair state (L + 1 qubits) */
  int32_t partner; /* kind 1: the rank whose slice is exchanged (rank ^ X); kind 0: the rank */
  int64_t first;   /* entries [first, first + count) of the rewritten arrays */
  int64_t count;
} sv_shard_step;

/* Rewrite the rotation list (x, z, theta; count entries, masks on n_qubits) for
 * `rank` of 2^global_qubits ranks.  With a Clifford frame F (nullable; on
 * n_qubits, see the cliff_* calls below) each rotation about P is first taken
 * about F(P) with its sign folded into theta, as cfhs_apply_rotations does.  The list is cut, in order, into steps: a step
 * of kind 0 holds rotations with no global x-bit; a step of kind 1 holds the
 * rotations from one with global x-part X to the last one with that X before a
 * rotation with another non-zero global x-part (rotations with no global x-bit in
 * between stay in it).  The cut depends only on the masks, so every rank gets the
 * same steps.  Rotation j is written to out_x[j], out_z[j], out_theta[j] (arrays of
 * count) in its step's frame: local masks and theta (-1)^{popc(r & z_g)} for kind
 * 0; pair masks (bit L set in x when the rotation crosses, in z when
 * popc(X & z_g) is odd) and theta times the pair sign for kind 1 (derivation in
 * csrc/shard.cu).  At most step_cap steps are written; *out_steps = steps needed
 * (SV_EINVAL if above step_cap).  SV_EINVAL for masks with bits >= n_qubits,
 * global_qubits outside 0..n-1 or rank outside 0..2^g - 1. */
int shard_rotations(int n_qubits, int global_qubits, int rank, const sv_cliff *frame, const uint64_t *x,
                    const uint64_t *z, const double *theta, size_t count, sv_shard_step *steps, size_t step_cap,
                    size_t *out_steps, uint64_t *out_x, uint64_t *out_z, double *out_theta);

/* Rewrite the Pauli sum sum_j c_j P_j for `rank` (terms mapped through the
 * nullable frame F first, as cfhs_expval does): group 0 (kind 0, always first,
 * possibly empty) holds the terms with no global x-bit, as local strings with
 * coefficient c_j (-1)^{popc(r & z_g)}; then one group (kind 1) per distinct
 * non-zero global x-part X, in order of first appearance, as pair strings with
 * coefficient c_j sigma / 2 (each of the two ranks of a pair evaluates the term
 * over the same pair state).  The sum over all ranks of <own|group 0|own> plus
 * <pair|group k|pair> for every group k is <psi|H|psi>.  Terms are written group
 * by group to out_x/out_z/out_coeff (arrays of count); at most group_cap groups;
 * *out_groups = groups needed. */
int shard_terms(int n_qubits, int global_qubits, int rank, const sv_cliff *frame, const uint64_t *x,
                const uint64_t *z, const double *coeff, size_t count, sv_shard_step *groups, size_t group_cap,
                size_t *out_groups, uint64_t *out_x, uint64_t *out_z, double *out_coeff);

#ifdef __cplusplus
}
#endif

#endif /* PAULIROT_H */
