// Global-qubit sharding of the statevector (host planning only).
//
// The paper distributes the amplitudes over 2^g ranks by the top g index bits
// (the "global" qubits): a rotation whose x-mask has no global bit pairs
// amplitudes inside every rank's slice, one whose x-mask has global part X
// pairs rank r with rank r ^ X, and the two exchange slices (Sec.
// "Multi-qubit rotations in a fullstate simulator", distributed-memory
// paragraph).  Here the exchanged slice is placed beside the rank's own one,
// and the pair of slices is treated as a state of L + 1 qubits (L = n - g local
// qubits, bit L = "which of the two ranks"), so the rotations that act inside
// the pair run through the ordinary fused passes.  This file rewrites
// rotations and Pauli terms into those local and pair frames; it does no
// device work.
//
// Pair frame.  With q = bit L and the pair's global parts r (q = 0) and r ^ X
// (q = 1), a string P = (x, z) whose global x-part x_g is 0 or X acts on the
// pair as sigma * P', where
//   P' = (x_l | u << L, z_l | v << L),  u = [x_g != 0],  v = popc(X & z_g) & 1,
//   sigma = (-1)^{popc(r & z_g) + (w - (u & v)) / 2},  w = popc(x_g & z_g),
// because popc(k & z) over the pair is popc(r & z_g) + q v + popc(i & z_l)
// and the factor i^{nY} of P differs from that of P' by i^{w - (u & v)}, an
// even power.  A string with x_g = 0 acts on the rank's own slice alone as
// (-1)^{popc(r & z_g)} (x_l, z_l).  Rotation angles take the sign sigma;
// expectation terms take it on their coefficient, and a pair term is halved
// because both ranks of the pair evaluate it over the same two slices.
#include <cstring>
#include <unordered_map>
#include <vector>

#include "internal.h"

namespace pr {
namespace {

struct Split {
  uint64_t xl, zl, xg, zg;
};

inline Split split(uint64_t x, uint64_t z, int L) {
  const uint64_t m = (L >= 64) ? ~0ULL : ((1ULL << L) - 1ULL);
  return {x & m, z & m, x >> L, z >> L};
}

// the string in the pair frame of partner mask X (x_g in {0, X}); returns sigma
inline int pair_map(const Split &s, uint64_t X, int L, uint64_t rank, uint64_t *px, uint64_t *pz) {
  const int u = s.xg != 0;
  const int v = popc64(X & s.zg) & 1;
  const int w = popc64(s.xg & s.zg);
  *px = s.xl | ((uint64_t)u << L);
  *pz = s.zl | ((uint64_t)v << L);
  const int e = popc64(rank & s.zg) + (w - (u & v)) / 2;
  return (e & 1) ? -1 : 1;
}

// strings mapped through an optional Clifford frame (Eq. Fmap): masks of F(P_j)
// and the values times the sign of F(P_j)
int frame_mapped(const sv_cliff *frame, const uint64_t *x, const uint64_t *z, const double *v, size_t count,
                 std::vector<uint64_t> &mx, std::vector<uint64_t> &mz, std::vector<double> &mv) {
  mx.assign(x, x + count);
  mz.assign(z, z + count);
  mv.assign(v, v + count);
  if (!frame || !count) return SV_OK;
  std::vector<int> sg(count);
  const int rc = cliff_map_paulis(frame, x, z, count, mx.data(), mz.data(), sg.data());
  if (rc) return rc;
  for (size_t j = 0; j < count; ++j) mv[j] = sg[j] * v[j];
  return SV_OK;
}

int check_shape(int n, int g, int rank) {
  if (n < 1 || n > 63) return fail(SV_EINVAL, "n_qubits must be in 1..63");
  if (g < 0 || g >= n) return fail(SV_EINVAL, "global_qubits must be in 0..n-1");
  if (g > 16) return fail(SV_EUNSUPPORTED, "at most 2^16 ranks");
  if (rank < 0 || rank >= (1 << g)) return fail(SV_EINVAL, "rank %d outside 0..%d", rank, (1 << g) - 1);
  return SV_OK;
}

}  // namespace
}  // namespace pr

extern "C" int shard_rotations(int n_qubits, int global_qubits, int rank, const sv_cliff *frame, const uint64_t *x0,
                               const uint64_t *z0, const double *theta0, size_t count, sv_shard_step *steps,
                               size_t step_cap, size_t *out_steps, uint64_t *out_x, uint64_t *out_z,
                               double *out_theta) {
  using namespace pr;
  clear_error();
  int rc = check_shape(n_qubits, global_qubits, rank);
  if (rc) return rc;
  if (count && (!x0 || !z0 || !theta0)) return fail(SV_EINVAL, "NULL rotation arrays");
  if (count && (!out_x || !out_z || !out_theta)) return fail(SV_EINVAL, "NULL output arrays");
  if (step_cap && !steps) return fail(SV_EINVAL, "steps is NULL");
  rc = validate_masks(n_qubits, x0, z0, count);
  if (rc) return rc;
  int fn = n_qubits;
  if (frame && (cliff_num_qubits(frame, &fn) || fn != n_qubits))
    return fail(SV_EINVAL, "the frame is not on %d qubits", n_qubits);
  std::vector<uint64_t> mx, mz;
  std::vector<double> mt;
  rc = frame_mapped(frame, x0, z0, theta0, count, mx, mz, mt);
  if (rc) return rc;
  const uint64_t *x = mx.data(), *z = mz.data();
  const double *theta = mt.data();
  const int L = n_qubits - global_qubits;
  // the global x-part of the next rotation after j whose global x-part is not 0
  std::vector<uint64_t> next(count + 1, 0);
  for (size_t j = count; j-- > 0;) {
    const uint64_t xg = x[j] >> L;
    next[j] = xg ? xg : next[j + 1];
  }
  size_t ns = 0;
  int kind = -1;
  uint64_t X = 0;
  auto open = [&](int k, uint64_t mask, size_t first) {
    if (ns < step_cap) {
      steps[ns].kind = k;
      steps[ns].partner = k ? (int32_t)((uint64_t)rank ^ mask) : rank;
      steps[ns].first = (int64_t)first;
      steps[ns].count = 0;
    }
    ++ns;
    kind = k;
    X = mask;
  };
  for (size_t j = 0; j < count; ++j) {
    const Split s = split(x[j], z[j], L);
    if (s.xg == 0) {
      // a local rotation stays in an open pair step only if that step's
      // partner is also the next one needed (no extra exchange either way)
      if (kind < 0 || (kind == 1 && next[j] != X)) open(0, 0, j);
    } else if (kind != 1 || s.xg != X) {
      open(1, s.xg, j);
    }
    if (kind == 0) {
      out_x[j] = s.xl;
      out_z[j] = s.zl;
      out_theta[j] = (popc64((uint64_t)rank & s.zg) & 1) ? -theta[j] : theta[j];
    } else {
      const int sg = pair_map(s, X, L, (uint64_t)rank, &out_x[j], &out_z[j]);
      out_theta[j] = sg * theta[j];
    }
    if (ns - 1 < step_cap) steps[ns - 1].count++;
  }
  if (out_steps) *out_steps = ns;
  if (ns > step_cap) return fail(SV_EINVAL, "step capacity %zu is below the %zu steps needed", step_cap, ns);
  return SV_OK;
}

extern "C" int shard_terms(int n_qubits, int global_qubits, int rank, const sv_cliff *frame, const uint64_t *x0,
                           const uint64_t *z0, const double *coeff0, size_t count, sv_shard_step *groups,
                           size_t group_cap, size_t *out_groups, uint64_t *out_x, uint64_t *out_z,
                           double *out_coeff) {
  using namespace pr;
  clear_error();
  int rc = check_shape(n_qubits, global_qubits, rank);
  if (rc) return rc;
  if (count && (!x0 || !z0 || !coeff0)) return fail(SV_EINVAL, "NULL term arrays");
  if (count && (!out_x || !out_z || !out_coeff)) return fail(SV_EINVAL, "NULL output arrays");
  if (group_cap && !groups) return fail(SV_EINVAL, "groups is NULL");
  rc = validate_masks(n_qubits, x0, z0, count);
  if (rc) return rc;
  int fn = n_qubits;
  if (frame && (cliff_num_qubits(frame, &fn) || fn != n_qubits))
    return fail(SV_EINVAL, "the frame is not on %d qubits", n_qubits);
  std::vector<uint64_t> mx, mz;
  std::vector<double> mc;
  rc = frame_mapped(frame, x0, z0, coeff0, count, mx, mz, mc);
  if (rc) return rc;
  const uint64_t *x = mx.data(), *z = mz.data();
  const double *coeff = mc.data();
  const int L = n_qubits - global_qubits;
  // group 0: terms local to the slice; then one group per distinct global x-part
  std::vector<uint64_t> keys{0};
  std::unordered_map<uint64_t, size_t> index{{0, 0}};
  std::vector<std::vector<size_t>> members(1);
  for (size_t j = 0; j < count; ++j) {
    const uint64_t xg = x[j] >> L;
    auto it = index.find(xg);
    if (it == index.end()) {
      it = index.emplace(xg, keys.size()).first;
      keys.push_back(xg);
      members.emplace_back();
    }
    members[it->second].push_back(j);
  }
  size_t pos = 0, ng = 0;
  for (size_t k = 0; k < keys.size(); ++k) {
    if (k > 0 && members[k].empty()) continue;
    if (ng < group_cap) {
      groups[ng].kind = k ? 1 : 0;
      groups[ng].partner = (int32_t)((uint64_t)rank ^ keys[k]);
      groups[ng].first = (int64_t)pos;
      groups[ng].count = (int64_t)members[k].size();
    }
    ++ng;
    for (size_t j : members[k]) {
      const Split s = split(x[j], z[j], L);
      if (k == 0) {
        out_x[pos] = s.xl;
        out_z[pos] = s.zl;
        out_coeff[pos] = (popc64((uint64_t)rank & s.zg) & 1) ? -coeff[j] : coeff[j];
      } else {
        const int sg = pair_map(s, keys[k], L, (uint64_t)rank, &out_x[pos], &out_z[pos]);
        out_coeff[pos] = 0.5 * sg * coeff[j];
      }
      ++pos;
    }
  }
  if (out_groups) *out_groups = ng;
  if (ng > group_cap) return fail(SV_EINVAL, "group capacity %zu is below the %zu groups needed", group_cap, ng);
  return SV_OK;
}
