// Projective Pauli measurement and qubit preparation on a (frame, state) pair
// (App. "Complete workflow of the hybrid Clifford fullstate simulation": a
// measurement or preparation on qubit i acts on the full state about the
// frame-rewritten axis).
//
// With psi = U Q phi (U the Clifford frame, Q the state's Pauli frame, phi the
// amplitudes), measuring a Hermitian Pauli P gives +1 with probability
// p = (1 + <psi|P|psi>/<psi|psi>)/2 and leaves (I + s P) psi / norm.  Since
// P U = U M with M = F(P) (a signed Pauli string) and M Q = sigma Q M with
// sigma = (-1)^{<M,Q>}, the post-measurement amplitudes are
//   phi' = (phi + s sigma M phi) / (2 sqrt(p_s <psi|psi>)),
// one pass over pairs (k, k^x) of M.  The outcome is decided by a uniform
// number u in [0, 1) that the caller draws: +1 if u < p_+, else -1.
#include <cmath>
#include <vector>

#include "internal.h"

namespace pr {
namespace {

template <typename R>
struct Cplx;
template <>
struct Cplx<double> {
  using T = double2;
};
template <>
struct Cplx<float> {
  using T = float2;
};

// times i^k
template <typename C>
__device__ __forceinline__ C ipow(C v, int k) {
  switch (k & 3) {
    case 0: return v;
    case 1: { C r; r.x = -v.y; r.y = v.x; return r; }
    case 2: { C r; r.x = -v.x; r.y = -v.y; return r; }
    default: { C r; r.x = v.y; r.y = -v.x; return r; }
  }
}

// phi <- scale (phi + s M phi), M = i^{nY} X^x Z^z: (M phi)_k = i^{nY} (-1)^{popc((k^x)&z)} phi_{k^x}.
// x = 0: one thread per amplitude; else one thread per pair (leaders have bit h = msb(x) clear).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_project(typename Cplx<R>::T *__restrict__ amp, uint64_t count,
                                                     uint64_t x, uint64_t z, int h, int ny, R s, R scale) {
  using C = typename Cplx<R>::T;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < count; t += stride) {
    if (x == 0) {
      const R f = scale * (R(1) + ((__popcll(t & z) & 1) ? -s : s));
      C v = amp[t];
      v.x *= f;
      v.y *= f;
      amp[t] = v;
    } else {
      const uint64_t k = ((t >> h) << (h + 1)) | (t & ((1ULL << h) - 1));
      const uint64_t m = k ^ x;
      const C a = amp[k], b = amp[m];
      C mb = ipow(b, ny), ma = ipow(a, ny);  // (M phi)_k from phi_m and (M phi)_m from phi_k
      if (__popcll(m & z) & 1) { mb.x = -mb.x; mb.y = -mb.y; }
      if (__popcll(k & z) & 1) { ma.x = -ma.x; ma.y = -ma.y; }
      C na, nb;
      na.x = scale * (a.x + s * mb.x);
      na.y = scale * (a.y + s * mb.y);
      nb.x = scale * (b.x + s * ma.x);
      nb.y = scale * (b.y + s * ma.y);
      amp[k] = na;
      amp[m] = nb;
    }
  }
}

template <typename R>
int launch_project(sv_state *sv, const Pauli &M, double s, double scale) {
  const uint64_t N = 1ULL << sv->n;
  const int h = M.x ? 63 - __builtin_clzll(M.x) : 0;
  const uint64_t count = M.x ? N / 2 : N;
  const uint64_t need = (count + kThreads - 1) / kThreads;
  const unsigned blocks = (unsigned)(need < (uint64_t)device_sm_count() * 8 ? (need ? need : 1) : device_sm_count() * 8);
  const int tr = trace_begin(sv, KN_PROJECT);
  k_project<R><<<blocks, kThreads, 0, sv->stream>>>((typename Cplx<R>::T *)sv->amps, count, M.x, M.z, h,
                                                    popc64(M.x & M.z) & 3, (R)s, (R)scale);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_PROJECT, 2.0 * (double)amp_bytes(sv->dtype) * (double)N);
  return SV_OK;
}

int pauli_masks_ok(const sv_state *sv, uint64_t x, uint64_t z) {
  const uint64_t lim = sv->n >= 64 ? ~0ULL : ((1ULL << sv->n) - 1);
  if ((x | z) & ~lim) return fail(SV_EINVAL, "Pauli masks have bits at or above n = %d", sv->n);
  return SV_OK;
}

// The signed string M = F(P) (P itself without a frame), as (masks, sign).
int rewrite(const sv_state *sv, const sv_cliff *f, uint64_t x, uint64_t z, Pauli *M, int *sign) {
  if (!f) {
    *M = pauli_string(x, z);
    *sign = 1;
    return SV_OK;
  }
  int nf = 0;
  int rc = cliff_num_qubits(f, &nf);
  if (rc) return rc;
  if (nf != sv->n) return fail(SV_EINVAL, "frame has %d qubits, state %d", nf, sv->n);
  uint64_t mx = 0, mz = 0;
  rc = cliff_map_paulis(f, &x, &z, 1, &mx, &mz, sign);
  if (rc) return rc;
  *M = pauli_string(mx, mz);
  return SV_OK;
}

int measure(sv_state *sv, const sv_cliff *f, uint64_t x, uint64_t z, double u, int *out_outcome, double *out_prob) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (!(u >= 0.0 && u < 1.0)) return fail(SV_EINVAL, "u = %g is not in [0, 1)", u);
  int rc = pauli_masks_ok(sv, x, z);
  if (rc) return rc;
  Pauli M;
  int sign = 1;
  rc = rewrite(sv, f, x, z, &M, &sign);
  if (rc) return rc;
  // <psi|P|psi> = sign <Q phi|M|Q phi>: the reductions of expval_pauli_sum
  const double one = (double)sign;
  double e = 0.0, nrm = 0.0;
  rc = expval_pauli_sum(sv, &M.x, &M.z, &one, 1, &e, &nrm);
  if (rc) return rc;
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return fail(SV_EINVAL, "state norm %g cannot be measured", nrm);
  const double p_plus = std::fmin(1.0, std::fmax(0.0, 0.5 * (1.0 + e / nrm)));
  int s = u < p_plus ? 1 : -1;
  double p = s > 0 ? p_plus : 1.0 - p_plus;
  // an outcome of probability zero up to rounding is not taken
  if (p <= 1e-14) {
    s = -s;
    p = 1.0 - p;
  }
  // (I + s P) U Q = U Q (I + s sign sigma M), sigma = (-1)^{<M, Q>}
  const int sigma = anticommute(M.x, M.z, sv->frame.x, sv->frame.z) ? -1 : 1;
  const double scale = 0.5 / std::sqrt(p * nrm);
  rc = sv->dtype == SV_C128 ? launch_project<double>(sv, M, (double)(s * sign * sigma), scale)
                            : launch_project<float>(sv, M, (double)(s * sign * sigma), scale);
  if (rc) return rc;
  if (out_outcome) *out_outcome = s;
  if (out_prob) *out_prob = p;
  return SV_OK;
}

}  // namespace
}  // namespace pr

using namespace pr;

extern "C" {

int cfhs_measure_pauli(sv_state *sv, const sv_cliff *f, uint64_t x, uint64_t z, double u, int *out_outcome,
                       double *out_prob) {
  return measure(sv, f, x, z, u, out_outcome, out_prob);
}

int cfhs_prepare_qubit(sv_state *sv, const sv_cliff *f, int qubit, char pauli, double u, int *out_outcome) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (qubit < 0 || qubit >= sv->n) return fail(SV_EINVAL, "qubit %d out of range", qubit);
  const uint64_t b = 1ULL << qubit;
  uint64_t x = 0, z = 0, fx = 0, fz = 0;  // the axis and a Pauli that anticommutes with it
  switch (pauli) {
    case 'X': case 'x': x = b; fz = b; break;
    case 'Y': case 'y': x = b; z = b; fz = b; break;
    case 'Z': case 'z': z = b; fx = b; break;
    default: return fail(SV_EINVAL, "pauli must be 'X', 'Y' or 'Z'");
  }
  int s = 0;
  int rc = measure(sv, f, x, z, u, &s, nullptr);
  if (rc) return rc;
  if (out_outcome) *out_outcome = s;
  if (s < 0) {
    // flip to the +1 eigenstate: apply the anticommuting partner F(fbar) to psi,
    // which the state's Pauli frame absorbs (Q <- F(fbar) Q, exact phase)
    Pauli G;
    int sign = 1;
    rc = rewrite(sv, f, fx, fz, &G, &sign);
    if (rc) return rc;
    if (sign < 0) G.q = (G.q + 2) & 3;
    sv->frame = pauli_mul(G, sv->frame);
  }
  return SV_OK;
}

}  // extern "C"
