// Internal declarations shared by the translation units of libpaulirot.so.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "paulirot.h"

namespace pr {

// ---------------------------------------------------------------- limits
constexpr int kDMax = 5;            // max dimension of a fused run's x-span
constexpr int kMaxRunRots = 256;    // rotations per fused coset run (shared memory)
constexpr int kMaxDiagRots = 1024;  // rotations per diagonal phase-sum run
constexpr int kDiagClassBits = 4;   // index bits resolved by the in-thread Walsh-Hadamard step
constexpr int kDiagClassLo = 5;     // lowest of those bits (above the lane bits)
constexpr int kDiagMinQubits = kDiagClassLo + kDiagClassBits;
constexpr int kDiagSlotBits = kDiagClassLo + kDiagClassBits;  // index bits 0..8: lane and class bits
constexpr int kDiagSlots = 128;  // distinct z patterns on those bits per diagonal run
constexpr int kMaxExpGroupTerms = 4096;  // terms per expectation run (shared memory)
constexpr int kThreads = 256;

inline int max_qubits(int dtype) { return dtype == SV_C128 ? 33 : 34; }
inline size_t amp_bytes(int dtype) { return dtype == SV_C128 ? 16 : 8; }
// fusion depth of plan_create(-1) when no tuned value is recorded
inline int default_depth(int dtype) { return dtype == SV_C128 ? 3 : 4; }

// ---------------------------------------------------------------- errors
int fail(int code, const char *fmt, ...);
void clear_error();

#define PR_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return ::pr::fail(SV_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

#define PR_CHECK_LAUNCH() PR_CUDA(cudaGetLastError())

// ---------------------------------------------------------------- Pauli algebra (host)
// A Pauli operator i^q X^x Z^z (X part left of the Z part, qubit-wise).
struct Pauli {
  uint64_t x = 0, z = 0;
  int q = 0;
};

inline int popc64(uint64_t v) { return __builtin_popcountll(v); }

#ifdef __CUDACC__
// FP64 value of an FP32 number by integer work without branches (rebias the
// exponent, shift the mantissa): exact for normal numbers, zeros, infinities
// and NaN; subnormals (below 1.2e-38 in magnitude) become zero.  On GB300 the
// conversion instruction occupies the narrow FP64 pipe as much as an add.
__device__ __forceinline__ double widen_f64(double v) { return v; }
__device__ __forceinline__ double widen_f64(float v) {
  const uint32_t b = __float_as_uint(v);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint64_t exp64 = e == 0u ? 0ULL : (e == 0xffu ? 0x7ffULL : (uint64_t)(e + 896u));
  const uint64_t mant = e == 0u ? 0ULL : (uint64_t)(b & 0x7fffffu) << 29;
  return __longlong_as_double((long long)(((uint64_t)(b >> 31) << 63) | (exp64 << 52) | mant));
}
#endif

// symplectic product: 1 if the two strings anticommute
inline int anticommute(uint64_t x1, uint64_t z1, uint64_t x2, uint64_t z2) {
  return popc64((x1 & z2) ^ (z1 & x2)) & 1;
}

// (i^a X^x1 Z^z1)(i^b X^x2 Z^z2) = i^{a+b+2|z1&x2|} X^{x1^x2} Z^{z1^z2}
inline Pauli pauli_mul(const Pauli &a, const Pauli &b) {
  Pauli r;
  r.x = a.x ^ b.x;
  r.z = a.z ^ b.z;
  r.q = (a.q + b.q + 2 * popc64(a.z & b.x)) & 3;
  return r;
}

// the Hermitian string with masks (x, z): Y = iXZ on every Y position
inline Pauli pauli_string(uint64_t x, uint64_t z) {
  Pauli p;
  p.x = x;
  p.z = z;
  p.q = popc64(x & z) & 3;
  return p;
}

// ---------------------------------------------------------------- device plan records
// One rotation of a fused coset run, tan form: the run applies
//   a_k <- a_k + t * kappa * s_k * a_{k^x},  kappa = (-i)^{nY+1},  s_k = (-1)^{popc(k&z)}
// with the factor (-1) of kappa's real/imaginary sign and the plan-frame sign
// folded into t; code = 2*u + imag where u are the coordinates of x in the
// run's basis and imag = (nY even); zt bit l = popc(s_l & z) & 1 for coset
// element l.
struct RotDev {
  uint64_t x, z;
  double t;
  uint32_t zt;
  uint32_t code;  // (u << 1) | imag in the low 16 bits; segment length above
};
// A segment is a stretch of consecutive rotations of a run with the same code
// (same pairing and part).  Its first rotation carries the stretch length in
// the bits above kCodeMask (the others carry 0 there), so a kernel can apply
// the whole segment under one dispatch, two rotations per sweep of the pairs.
constexpr int kSegShift = 16;
constexpr uint32_t kCodeMask = (1u << kSegShift) - 1;
static_assert(sizeof(RotDev) == 32, "RotDev layout");

// One rotation of a diagonal phase-sum run: a = theta/2 as a fixed-point
// fraction of a full turn (units of 2 pi / 2^64), plan-frame sign applied.
// slot = rank of the rotation's z pattern on index bits 0..8 among the run's
// distinct patterns (the run's rotations are sorted by that pattern).
struct DiagDev {
  uint64_t z;
  uint64_t a;
  uint32_t slot;
  uint32_t pad;
};

struct RunDev {
  uint64_t basis[kDMax];  // reduced x-span basis; basis[b] has pivot bit piv[b]
  int32_t piv[kDMax];     // ascending pivot positions
  int32_t d;
  int32_t kind;           // 0 = coset run, 1 = diagonal phase-sum run
  int32_t first, count;   // range in the plan's RotDev or DiagDev array
  int32_t fold;           // multiply by (fold_re + i fold_im) at the end
  double fold_re, fold_im;
  int32_t seg[(1 << kDiagClassBits) + 1];  // diag runs: slot ranges per class (z bits 5..8)
};

// Two consecutive complex64 coset runs applied in one HBM pass (chain.cu).  A
// CTA owns a block of 2^kChainDim amplitudes: a coset of a subspace W that
// contains both runs' spans and index bits 0..3.  Block coordinate i stands for
// the index-space vector w[i] (w[i] = 2^i for i < 4, bits 0..3 clear above);
// amplitude index = block base ^ (xor of w[i] over the set bits i).
constexpr int kChainDim = 12;  // 2^12 amplitudes per block: 128 threads x 32 amplitudes
struct ChainSubDev {
  uint64_t off[16];   // element offsets (the run's basis padded to 4 vectors)
  uint64_t padv[4];   // index-space vector of basis slot b >= d, else 0
  uint16_t offc[16];  // the same offsets in block coordinates
  int32_t pivc[4];    // pivots of the padded span in block coordinates, ascending
  int32_t d, first, count, fold;
  double fold_re, fold_im;
};
struct ChainDev {
  uint64_t w[kChainDim];
  int32_t wpiv[kChainDim];  // pivot bits of W, ascending (block bases have zeros there)
  int32_t pad;
  ChainSubDev sub[2];
};
// one launch of a plan: run `run` alone (chain < 0) or runs run, run + 1 as
// the chained pass chains[chain]
struct PlanStep {
  int32_t run, chain;
};

// Expectation-value run: groups of terms whose x-masks lie in one span.
struct ExpTermDev {
  uint64_t z;
  double coef;    // c_j * frame sign * (-1)^{floor(nY/2)} (times 2 for pairs)
  uint32_t zt;    // coset sign table as in RotDev
  uint32_t imag;  // nY odd: the term reads Im(conj(a_k) a_{k^x})
};
struct ExpGroupDev {
  int32_t u;      // coordinates of the group's x in the run basis
  int32_t first, count;
  int32_t pad;    // Hpsi runs: bit 0 = some term has even nY, bit 1 = some has odd nY
};
struct ExpRunDev {
  uint64_t basis[kDMax];
  int32_t piv[kDMax];
  int32_t d;
  int32_t n_groups;
  int32_t with_norm;
  double qscale;  // H psi runs: a term's coefficient is its fixed-point value times qscale
};

// ---------------------------------------------------------------- host objects
struct HostRun {
  RunDev dev;
};

}  // namespace pr

namespace pr {
struct TraceRec {
  int name;       // index into the kernel name table (trace.cu)
  double bytes;   // algorithmic bytes of this launch
  double flops;   // algorithmic floating-point operations of this launch
  int ev0, ev1;   // event pool slots
  int64_t launches;  // launches in the record (block mode: a run of one kernel)
};
// kernel name ids for tracing
enum KernelId {
  KN_COSET0 = 0, KN_COSET1, KN_COSET2, KN_COSET3, KN_COSET4, KN_COSET5,
  KN_DIAG_SUM, KN_EXPVAL, KN_FINISH, KN_PAULI_SUM, KN_MATERIALIZE, KN_SET_BASIS,
  KN_ADJOINT, KN_SUM_ROWS, KN_GATE1, KN_DIAG1, KN_CNOT, KN_PROJECT, KN_ADJOINT_RUN, KN_CHAIN, KN_COUNT
};
}  // namespace pr

struct sv_state {
  void *amps = nullptr;
  int n = 0;
  int dtype = SV_C128;
  bool owns = false;
  int device = 0;
  cudaStream_t stream = nullptr;
  pr::Pauli frame;
  // scratch: block partial sums and run results (device), results (pinned host)
  double *d_partials = nullptr;
  size_t partials_cap = 0;  // doubles
  double *d_results = nullptr;
  size_t results_cap = 0;
  double *h_results = nullptr;
  size_t h_results_cap = 0;
  // staging for per-call rotation lists (device + pinned host)
  void *d_stage = nullptr;
  size_t stage_cap = 0;
  void *h_stage = nullptr;
  size_t h_stage_cap = 0;
  // work states of rotation_grads (phi and lambda), kept for the next call and
  // released with this handle
  sv_state *work[2] = {nullptr, nullptr};
  // a work state records its launches in its owner's trace (null: its own)
  sv_state *trace_owner = nullptr;
  // packed complex64 passes launched on this handle (their parity sets the
  // direction the next one walks the cosets in)
  uint32_t packed_passes = 0;
  // rotation records of apply_pauli_rotations: device buffer and pinned
  // staging, kept for the next call; events after the last copy and after the
  // last launch that reads the buffer
  void *d_rec = nullptr;
  size_t d_rec_cap = 0;
  void *h_rec = nullptr;
  size_t h_rec_cap = 0;
  cudaEvent_t rec_copied = nullptr;
  cudaEvent_t rec_done = nullptr;
  // tracing
  bool tracing = false;
  bool trace_blocks = false;  // one event per change of kernel instead of per launch
  std::vector<cudaEvent_t> events;
  int events_used = 0;
  std::vector<pr::TraceRec> trace;
};

struct sv_plan {
  int n = 0, dtype = SV_C128, dmax = 0;
  std::vector<pr::RunDev> runs;
  // launch order of apply_plan; empty: one launch per run
  std::vector<pr::PlanStep> steps;
  std::vector<pr::ChainDev> chains;
  pr::RotDev *d_rots = nullptr;
  pr::DiagDev *d_diag = nullptr;
  size_t n_rots = 0, n_diag = 0;
  size_t n_input = 0, n_effective = 0, n_diag_runs = 0;
  pr::Pauli frame;  // product of the frame factors taken out by angle reduction
  // for the adjoint sweep, in applied order: original index, applied angle in
  // the plan frame (sign and reduction included) and the plan-frame sign
  std::vector<int64_t> order;
  std::vector<double> beta;
  std::vector<int8_t> sigma;
  std::vector<uint64_t> ox, oz;
  bool owns_device = true;
};

namespace pr {
// tracing (trace.cu): call trace_begin before a launch and trace_end after it
int trace_begin(sv_state *sv, int name);
void trace_end(sv_state *sv, int slot, int name, double bytes, double flops = 0.0);
void trace_release(sv_state *sv);

// batched launches (batch.cu): forget a cached batch that uses a freed handle
void batch_forget(const sv_state *sv, const sv_plan *plan);

// device memory helpers (state.cu)
int ensure_scratch(sv_state *sv, size_t partial_doubles, size_t result_doubles);
int ensure_stage(sv_state *sv, size_t bytes);
int device_sm_count();

// launch one run of a plan (rotate.cu)
int launch_run(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz);
// chained passes (chain.cu): pair up consecutive runs of a complex64 plan
// (fills plan->steps and plan->chains), and launch one chained pass
void build_chains(sv_plan *plan);
bool chains_enabled(const sv_plan *plan);
// runs i and i + 1 of the plan as one chained pass, if they qualify
bool chain_pair(const sv_plan *plan, size_t i, ChainDev *out);
int launch_chain(sv_state *sv, const sv_plan *plan, const ChainDev &chain, uint64_t fx, uint64_t fz);
int prepare_tables(int dtype);
int table_pointer(int dtype, const void **out);
// basis state and in-place frame application (state.cu)
int launch_materialize(sv_state *sv, uint64_t x, uint64_t z, int q);
int launch_set_basis(sv_state *sv, uint64_t k);

// plan building (plan.cu)
// Receives the plan's runs while build_plan makes them: run(p, rots, diags) after
// each run is appended (its rotation records are final; the newest run's fold
// may still change), finish(p, rots, diags) once the plan is complete.
struct PlanSink {
  virtual int run(sv_plan *p, const std::vector<RotDev> &rots, const std::vector<DiagDev> &diags) = 0;
  virtual int finish(sv_plan *p, const std::vector<RotDev> &rots, const std::vector<DiagDev> &diags) = 0;
  virtual ~PlanSink() = default;
};
// upload = false: plan on the host only (no device allocation, no upload);
// with a sink the records go to the sink instead of a device copy of the plan
int build_plan(sv_plan *p, int n, int dtype, const uint64_t *x, const uint64_t *z,
               const double *theta, size_t count, int fusion_depth, cudaStream_t stream, bool upload = true,
               PlanSink *sink = nullptr);
int apply_plan(sv_state *sv, sv_plan *plan);
int validate_masks(int n, const uint64_t *x, const uint64_t *z, size_t count);
// tuned fusion depth for (n, dtype), or -1 if none is recorded (tune.cu)
int tuned_depth(int n, int dtype);

// reductions (reduce.cu)
int expval_impl(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
                double *energy, double *norm2);
int pauli_sum_impl(sv_state *dst, sv_state *src, const uint64_t *x, const uint64_t *z,
                   const double *c, size_t count);
// adjoint one-rotation step (adjoint.cu)
// max_blocks > 0 caps the grid (the partial sums it writes per block)
int adjoint_step(sv_state *phi, sv_state *lam, uint64_t x, uint64_t z, double beta, double *d_out,
                 int max_blocks = 0);
}  // namespace pr
