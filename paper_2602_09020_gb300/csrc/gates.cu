// Gate-decomposed comparison path: every rotation exp(-i theta/2 P) applied as
// its textbook circuit (paper, Sec. "Preliminaries of Hamiltonian Simulation",
// CNOT-staircase figure): per X qubit H, per Y qubit Sdg then H; CNOTs from
// each support qubit to the next (ascending), Rz(theta) on the top support
// qubit, the ladder backwards, then H (X) or H then S (Y).  Each gate is its own
// kernel and its own pass over the state, which is what a gate-level simulator
// does; this path exists to measure the same-GPU speedup of the pair pass.
#include <cmath>

#include "internal.h"

namespace pr {

namespace {

template <typename R>
struct Cx;
template <>
struct Cx<float> {
  using T = float2;
};
template <>
struct Cx<double> {
  using T = double2;
};

// Hadamard on qubit q, in the amplitude precision
template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_hadamard(typename Cx<R>::T *__restrict__ amp, uint64_t half, int q) {
  using C = typename Cx<R>::T;
  const R r = (R)0.70710678118654752440;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t lowmask = (1ULL << q) - 1ULL;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride) {
    const uint64_t k0 = ((t >> q) << (q + 1)) | (t & lowmask), k1 = k0 | (1ULL << q);
    const C a = amp[k0], b = amp[k1];
    C o0, o1;
    o0.x = r * (a.x + b.x);
    o0.y = r * (a.y + b.y);
    o1.x = r * (a.x - b.x);
    o1.y = r * (a.y - b.y);
    amp[k0] = o0;
    amp[k1] = o1;
  }
}

// diag(p0, p1) on qubit q (S, Sdg, Rz, global phases), in the amplitude precision
template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_diag1(typename Cx<R>::T *__restrict__ amp, uint64_t half, int q, double2 p0d, double2 p1d) {
  using C = typename Cx<R>::T;
  const R p0x = (R)p0d.x, p0y = (R)p0d.y, p1x = (R)p1d.x, p1y = (R)p1d.y;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t lowmask = (1ULL << q) - 1ULL;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < half; t += stride) {
    const uint64_t k0 = ((t >> q) << (q + 1)) | (t & lowmask), k1 = k0 | (1ULL << q);
    const C a = amp[k0], b = amp[k1];
    C o0, o1;
    o0.x = p0x * a.x - p0y * a.y;
    o0.y = p0x * a.y + p0y * a.x;
    o1.x = p1x * b.x - p1y * b.y;
    o1.y = p1x * b.y + p1y * b.x;
    amp[k0] = o0;
    amp[k1] = o1;
  }
}

// CNOT(c, t): swap amplitudes with bit c set that differ in bit t
template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_cnot(typename Cx<R>::T *__restrict__ amp, uint64_t quarter, int lo, int hi, uint64_t bc, uint64_t bt) {
  using C = typename Cx<R>::T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < quarter; s += stride) {
    uint64_t k = ((s >> lo) << (lo + 1)) | (s & ((1ULL << lo) - 1ULL));
    k = ((k >> hi) << (hi + 1)) | (k & ((1ULL << hi) - 1ULL));
    k |= bc;
    const C a = amp[k], b = amp[k | bt];
    amp[k] = b;
    amp[k | bt] = a;
  }
}

struct GateCtx {
  sv_state *sv;
  unsigned blocks_half, blocks_quarter;
  size_t launched = 0;
};

int hadamard(GateCtx &g, int q) {
  const uint64_t half = (1ULL << g.sv->n) >> 1;
  const int tr = trace_begin(g.sv, KN_GATE1);
  if (g.sv->dtype == SV_C128)
    k_hadamard<double><<<g.blocks_half, kThreads, 0, g.sv->stream>>>((double2 *)g.sv->amps, half, q);
  else
    k_hadamard<float><<<g.blocks_half, kThreads, 0, g.sv->stream>>>((float2 *)g.sv->amps, half, q);
  PR_CHECK_LAUNCH();
  trace_end(g.sv, tr, KN_GATE1, 4.0 * (double)amp_bytes(g.sv->dtype) * (double)half);
  ++g.launched;
  return SV_OK;
}

int diag1(GateCtx &g, int q, double2 p0, double2 p1) {
  const uint64_t half = (1ULL << g.sv->n) >> 1;
  const int tr = trace_begin(g.sv, KN_DIAG1);
  if (g.sv->dtype == SV_C128)
    k_diag1<double><<<g.blocks_half, kThreads, 0, g.sv->stream>>>((double2 *)g.sv->amps, half, q, p0, p1);
  else
    k_diag1<float><<<g.blocks_half, kThreads, 0, g.sv->stream>>>((float2 *)g.sv->amps, half, q, p0, p1);
  PR_CHECK_LAUNCH();
  trace_end(g.sv, tr, KN_DIAG1, 4.0 * (double)amp_bytes(g.sv->dtype) * (double)half);
  ++g.launched;
  return SV_OK;
}

int cnot(GateCtx &g, int c, int t) {
  const uint64_t quarter = (1ULL << g.sv->n) >> 2;
  const int lo = c < t ? c : t, hi = c < t ? t : c;
  const int tr = trace_begin(g.sv, KN_CNOT);
  if (g.sv->dtype == SV_C128)
    k_cnot<double><<<g.blocks_quarter, kThreads, 0, g.sv->stream>>>((double2 *)g.sv->amps, quarter, lo, hi,
                                                                    1ULL << c, 1ULL << t);
  else
    k_cnot<float><<<g.blocks_quarter, kThreads, 0, g.sv->stream>>>((float2 *)g.sv->amps, quarter, lo, hi,
                                                                   1ULL << c, 1ULL << t);
  PR_CHECK_LAUNCH();
  trace_end(g.sv, tr, KN_CNOT, 4.0 * (double)amp_bytes(g.sv->dtype) * (double)quarter);
  ++g.launched;
  return SV_OK;
}

unsigned blocks_for(uint64_t work) {
  uint64_t need = (work + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)device_sm_count() * 8;
  uint64_t b = need < cap ? need : cap;
  return b ? (unsigned)b : 1u;
}

}  // namespace

}  // namespace pr

using namespace pr;

extern "C" {

int apply_pauli_rotations_gates(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *angles,
                                size_t count, size_t *out_gates) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (count && (!x || !z || !angles)) return fail(SV_EINVAL, "NULL rotation arrays");
  if (sv->n < 2) return fail(SV_EUNSUPPORTED, "gate path needs n >= 2");
  int rc = validate_masks(sv->n, x, z, count);
  if (rc) return rc;
  for (size_t j = 0; j < count; ++j)
    if (!std::isfinite(angles[j])) return fail(SV_EINVAL, "angle %zu is not finite", j);
  GateCtx g;
  g.sv = sv;
  g.blocks_half = blocks_for((1ULL << sv->n) >> 1);
  g.blocks_quarter = blocks_for((1ULL << sv->n) >> 2);
  const double2 one = make_double2(1.0, 0.0), pi_ = make_double2(0.0, 1.0), mi = make_double2(0.0, -1.0);
  const Pauli q = sv->frame;
  int sup[64];
  for (size_t j = 0; j < count; ++j) {
    double th = angles[j];
    if (anticommute(x[j], z[j], q.x, q.z)) th = -th;  // Q^dag P Q = -P
    int k = 0;
    for (int b = 0; b < sv->n; ++b)
      if (((x[j] | z[j]) >> b) & 1ULL) sup[k++] = b;
    if (k == 0) {
      // identity string: global phase e^{-i theta/2} on both halves of qubit 0
      const double2 ph = make_double2(std::cos(0.5 * th), -std::sin(0.5 * th));
      if ((rc = diag1(g, 0, ph, ph))) return rc;
      continue;
    }
    for (int m = 0; m < k; ++m) {
      const int b = sup[m];
      const bool xb = (x[j] >> b) & 1ULL, zb = (z[j] >> b) & 1ULL;
      if (xb && zb) {
        if ((rc = diag1(g, b, one, mi))) return rc;  // Sdg
        if ((rc = hadamard(g, b))) return rc;
      } else if (xb) {
        if ((rc = hadamard(g, b))) return rc;
      }
    }
    for (int m = 0; m + 1 < k; ++m)
      if ((rc = cnot(g, sup[m], sup[m + 1]))) return rc;
    const double2 e0 = make_double2(std::cos(0.5 * th), -std::sin(0.5 * th));
    const double2 e1 = make_double2(std::cos(0.5 * th), std::sin(0.5 * th));
    if ((rc = diag1(g, sup[k - 1], e0, e1))) return rc;
    for (int m = k - 2; m >= 0; --m)
      if ((rc = cnot(g, sup[m], sup[m + 1]))) return rc;
    for (int m = 0; m < k; ++m) {
      const int b = sup[m];
      const bool xb = (x[j] >> b) & 1ULL, zb = (z[j] >> b) & 1ULL;
      if (xb && zb) {
        if ((rc = hadamard(g, b))) return rc;
        if ((rc = diag1(g, b, one, pi_))) return rc;  // S
      } else if (xb) {
        if ((rc = hadamard(g, b))) return rc;
      }
    }
  }
  if (out_gates) *out_gates = g.launched;
  return SV_OK;
}

}  // extern "C"
