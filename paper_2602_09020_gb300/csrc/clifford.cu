// Clifford-fullstate hybrid layer (Sec. "Clifford-Fullstate Hybrid Simulator").
//
// A state is the pair (F, Phi): psi = U Phi (Eq. cfhsstate), where U is a
// Clifford unitary kept as its Pauli frame in the backward interpretation,
// F = U^dag F_origin U (Eq. framemat): ez[j] = U^dag Z_j U, ex[j] = U^dag X_j U,
// each an exact Pauli i^q X^x Z^z.  Clifford gates only update the frame (host,
// O(1) Pauli products per gate); a rotation about P becomes the rotation about
// F(P) = U^dag P U on Phi (Eq. single_to_multirot, Eq. Fmap); expectation
// values are <F(P)> on Phi (Eq. chfsexp); reading amplitudes first applies U to
// Phi as at most 4n rotations by pi/2 (App. "Efficiently implementing Clifford
// unitaries with multi-qubit rotations"), after which F is the origin frame.
//
// All of it is host code; the rotations it produces run through the same
// planner and kernels as apply_pauli_rotations.
#include <cmath>
#include <new>
#include <vector>

#include "internal.h"

struct sv_cliff {
  int n = 0;
  std::vector<pr::Pauli> ez, ex;
};

namespace pr {
namespace {

Pauli single(int kind, int q) {  // kind 1 = X, 2 = Y, 3 = Z, as Hermitian strings
  const uint64_t b = 1ULL << q;
  if (kind == 1) return pauli_string(b, 0);
  if (kind == 2) return pauli_string(b, b);
  return pauli_string(0, b);
}

Pauli phase(Pauli p, int k) {  // i^k p
  p.q = (p.q + k) & 3;
  return p;
}

bool same(const Pauli &a, const Pauli &b) { return a.x == b.x && a.z == b.z && ((a.q - b.q) & 3) == 0; }

void set_origin(sv_cliff *f) {
  f->ez.assign(f->n, Pauli());
  f->ex.assign(f->n, Pauli());
  for (int j = 0; j < f->n; ++j) {
    f->ez[j] = single(3, j);
    f->ex[j] = single(1, j);
  }
}

// F(P) for P = i^q X^x Z^z: conjugation is a homomorphism, so
// F(P) = i^q prod_{j in x} F(X_j) prod_{j in z} F(Z_j)   (Eq. Fmap)
Pauli frame_map(const sv_cliff *f, const Pauli &p) {
  Pauli r;
  r.q = p.q;
  for (uint64_t m = p.x; m; m &= m - 1) r = pauli_mul(r, f->ex[__builtin_ctzll(m)]);
  for (uint64_t m = p.z; m; m &= m - 1) r = pauli_mul(r, f->ez[__builtin_ctzll(m)]);
  return r;
}

// A Hermitian Pauli i^q X^x Z^z as s * (the Hermitian string with masks x, z):
// s = i^{q - popc(x&z)} is +1 or -1
int hermitian_sign(const Pauli &p) { return (((p.q - popc64(p.x & p.z)) & 3) == 0) ? 1 : -1; }

bool valid_qubit(const sv_cliff *f, int q) { return q >= 0 && q < f->n; }

bool two_qubit(int g) { return g == SV_CG_CNOT || g == SV_CG_CZ || g == SV_CG_SWAP; }
bool rotation_gate(int g) { return g == SV_CG_RX || g == SV_CG_RY || g == SV_CG_RZ; }

// Gate g applied to psi = U Phi: U' = g U, so F'(P) = F(g^dag P g).  Only the
// entries of the qubits g acts on change; every new entry is a product of old
// entries.  Rotation gates do not change F: they are returned as the rotation
// Phi must undergo (axis, signed angle).  Arguments are checked by the caller.
void frame_gate(sv_cliff *f, int g, int a, int b, double theta, bool *is_rot, Pauli *axis, double *angle) {
  *is_rot = false;
  std::vector<Pauli> &ez = f->ez, &ex = f->ex;
  switch (g) {
    case SV_CG_H:  // H Z H = X, H X H = Z
      std::swap(ez[a], ex[a]);
      break;
    case SV_CG_S:  // S^dag Z S = Z, S^dag X S = -Y = i^3 X Z
      ex[a] = phase(pauli_mul(ex[a], ez[a]), 3);
      break;
    case SV_CG_SDG:  // S X S^dag = Y = i X Z
      ex[a] = phase(pauli_mul(ex[a], ez[a]), 1);
      break;
    case SV_CG_X:  // X Z X = -Z
      ez[a] = phase(ez[a], 2);
      break;
    case SV_CG_Y:  // Y Z Y = -Z, Y X Y = -X
      ez[a] = phase(ez[a], 2);
      ex[a] = phase(ex[a], 2);
      break;
    case SV_CG_Z:  // Z X Z = -X
      ex[a] = phase(ex[a], 2);
      break;
    case SV_CG_CNOT: {  // control a, target b: X_a -> X_a X_b, Z_b -> Z_a Z_b
      const Pauli xa = pauli_mul(ex[a], ex[b]), zb = pauli_mul(ez[a], ez[b]);
      ex[a] = xa;
      ez[b] = zb;
      break;
    }
    case SV_CG_CZ: {  // X_a -> X_a Z_b, X_b -> Z_a X_b
      const Pauli xa = pauli_mul(ex[a], ez[b]), xb = pauli_mul(ez[a], ex[b]);
      ex[a] = xa;
      ex[b] = xb;
      break;
    }
    case SV_CG_SWAP:
      std::swap(ez[a], ez[b]);
      std::swap(ex[a], ex[b]);
      break;
    default: {  // RX, RY, RZ
      const Pauli m = frame_map(f, single(g == SV_CG_RX ? 1 : g == SV_CG_RY ? 2 : 3, a));
      *is_rot = true;
      *axis = pauli_string(m.x, m.z);
      *angle = hermitian_sign(m) * theta;
      break;
    }
  }
}

// conjugation of every frame entry by e^{-i pi/4 Q}: entries that commute with
// Q stay, the others become -i Q E (App. A, "Clifford Pauli rotation")
void conjugate(sv_cliff *f, const Pauli &Q) {
  for (int j = 0; j < f->n; ++j) {
    if (anticommute(f->ez[j].x, f->ez[j].z, Q.x, Q.z)) f->ez[j] = phase(pauli_mul(Q, f->ez[j]), 3);
    if (anticommute(f->ex[j].x, f->ex[j].z, Q.x, Q.z)) f->ex[j] = phase(pauli_mul(Q, f->ex[j]), 3);
  }
}

// Rotations R_1..R_m (R_k = e^{-i pi/4 Q_k}) whose successive conjugations take
// F to the origin frame, so U = R_m ... R_1 up to a global phase.  Position j
// is brought to (Z_j, X_j) with at most two rotations per entry, each of which
// has no support on the qubits below j and commutes with the entries already
// fixed: an entry P that anticommutes with its target T goes there in one step
// (Q = i T P); otherwise through a W that anticommutes with both
// (Q = i W P, then Q = i T W).  The frame relations then leave the later
// entries without support on qubit j.  m <= 4n.
std::vector<Pauli> inverse_rotations(const sv_cliff *f0) {
  sv_cliff f = *f0;
  std::vector<Pauli> out;
  auto rot = [&](const Pauli &Q) {
    conjugate(&f, Q);
    out.push_back(Q);
  };
  auto move = [&](Pauli P, Pauli T, Pauli W) {
    if (anticommute(P.x, P.z, T.x, T.z)) {
      rot(phase(pauli_mul(T, P), 1));
    } else {
      rot(phase(pauli_mul(W, P), 1));
      rot(phase(pauli_mul(T, W), 1));
    }
  };
  for (int j = 0; j < f.n; ++j) {
    const uint64_t bj = 1ULL << j;
    const Pauli Tz = single(3, j), Tx = single(1, j);
    if (!same(f.ez[j], Tz)) {
      const Pauli P = f.ez[j];
      Pauli W = single(1, j);  // anticommutes with Z_j; with P when P has Z on qubit j
      if (!anticommute(P.x, P.z, W.x, W.z)) {
        // P is the identity on qubit j: take W = X_j A_m on a qubit m > j where P acts
        const uint64_t rest = (P.x | P.z) & ~((bj << 1) - 1);
        const int m = __builtin_ctzll(rest);
        W = pauli_mul(W, single(((P.x >> m) & 1ULL) ? 3 : 1, m));
      }
      move(P, Tz, W);
    }
    if (!same(f.ex[j], Tx)) move(f.ex[j], Tx, single(2, j));
  }
  return out;
}

bool is_origin(const sv_cliff *f) {
  for (int j = 0; j < f->n; ++j)
    if (!same(f->ez[j], single(3, j)) || !same(f->ex[j], single(1, j))) return false;
  return true;
}

// Process a gate stream: Clifford gates update F, rotation gates are appended
// (axis masks, signed angle) to the lists Phi must undergo, in order.  The
// whole stream is checked before F changes, so a rejected stream leaves F as
// it was.
int frame_stream(sv_cliff *f, const int *gate, const int *q0, const int *q1, const double *theta, size_t count,
                 std::vector<uint64_t> &rx, std::vector<uint64_t> &rz, std::vector<double> &rt) {
  if (count && (!gate || !q0)) return fail(SV_EINVAL, "NULL gate arrays");
  for (size_t k = 0; k < count; ++k) {
    const int g = gate[k];
    if (g < SV_CG_H || g > SV_CG_RZ) return fail(SV_EINVAL, "gate %zu: unknown gate code %d", k, g);
    if (!valid_qubit(f, q0[k])) return fail(SV_EINVAL, "gate %zu: qubit %d out of range", k, q0[k]);
    if (two_qubit(g) && !q1) return fail(SV_EINVAL, "gate %zu needs a second qubit (q1 is NULL)", k);
    if (two_qubit(g) && (!valid_qubit(f, q1[k]) || q1[k] == q0[k]))
      return fail(SV_EINVAL, "gate %zu: second qubit %d invalid", k, q1[k]);
    if (rotation_gate(g) && !theta) return fail(SV_EINVAL, "gate %zu needs an angle (theta is NULL)", k);
    if (rotation_gate(g) && !std::isfinite(theta[k])) return fail(SV_EINVAL, "gate %zu: angle is not finite", k);
  }
  for (size_t k = 0; k < count; ++k) {
    const int g = gate[k];
    bool is_rot = false;
    Pauli axis;
    double ang = 0.0;
    frame_gate(f, g, q0[k], two_qubit(g) ? q1[k] : -1, rotation_gate(g) ? theta[k] : 0.0, &is_rot, &axis, &ang);
    if (is_rot) {
      rx.push_back(axis.x);
      rz.push_back(axis.z);
      rt.push_back(ang);
    }
  }
  return SV_OK;
}

int copy_out(const std::vector<uint64_t> &rx, const std::vector<uint64_t> &rz, const std::vector<double> &rt,
             uint64_t *out_x, uint64_t *out_z, double *out_theta, size_t cap, size_t *out_count) {
  if (out_count) *out_count = rt.size();
  if (rt.empty()) return SV_OK;
  if (!out_x || !out_z || !out_theta) return fail(SV_EINVAL, "NULL output arrays for %zu rotations", rt.size());
  if (rt.size() > cap) return fail(SV_EINVAL, "%zu rotations do not fit the output capacity %zu", rt.size(), cap);
  for (size_t k = 0; k < rt.size(); ++k) {
    out_x[k] = rx[k];
    out_z[k] = rz[k];
    out_theta[k] = rt[k];
  }
  return SV_OK;
}

void frame_rotations(const sv_cliff *f, std::vector<uint64_t> &rx, std::vector<uint64_t> &rz,
                     std::vector<double> &rt) {
  const double half_pi = 1.57079632679489661923;
  for (const Pauli &Q : inverse_rotations(f)) {
    rx.push_back(Q.x);
    rz.push_back(Q.z);
    rt.push_back(hermitian_sign(Q) * half_pi);  // e^{-i pi/4 Q} = R_P(+-pi/2)
  }
}

int check_pair(const sv_state *sv, const sv_cliff *f) {
  if (!sv || !f) return fail(SV_EINVAL, "NULL state or frame");
  if (f->n != sv->n) return fail(SV_EINVAL, "frame has %d qubits, state %d", f->n, sv->n);
  return SV_OK;
}

}  // namespace
}  // namespace pr

using namespace pr;

extern "C" {

int cliff_create(sv_cliff **out, int n_qubits) {
  if (!out) return fail(SV_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_qubits < 1 || n_qubits > 63) return fail(SV_EINVAL, "n_qubits %d out of range 1..63", n_qubits);
  sv_cliff *f = new (std::nothrow) sv_cliff;
  if (!f) return fail(SV_ENOMEM, "frame allocation failed");
  f->n = n_qubits;
  set_origin(f);
  *out = f;
  return SV_OK;
}

int cliff_free(sv_cliff *f) {
  delete f;
  return SV_OK;
}

int cliff_reset(sv_cliff *f) {
  if (!f) return fail(SV_EINVAL, "frame is NULL");
  set_origin(f);
  return SV_OK;
}

int cliff_num_qubits(const sv_cliff *f, int *out) {
  if (!f || !out) return fail(SV_EINVAL, "NULL argument");
  *out = f->n;
  return SV_OK;
}

int cliff_apply_gates(sv_cliff *f, const int *gate, const int *q0, const int *q1, const double *theta, size_t count,
                      uint64_t *out_x, uint64_t *out_z, double *out_theta, size_t cap, size_t *out_count) {
  if (!f) return fail(SV_EINVAL, "frame is NULL");
  if (out_count) *out_count = 0;
  // a stream whose rotations do not fit is rejected before the frame changes
  size_t nrot = 0;
  for (size_t k = 0; gate && k < count; ++k) nrot += rotation_gate(gate[k]);
  if (nrot > cap) return fail(SV_EINVAL, "%zu rotation gates do not fit the output capacity %zu", nrot, cap);
  if (nrot && (!out_x || !out_z || !out_theta)) return fail(SV_EINVAL, "NULL output arrays for %zu rotations", nrot);
  std::vector<uint64_t> rx, rz;
  std::vector<double> rt;
  const int rc = frame_stream(f, gate, q0, q1, theta, count, rx, rz, rt);
  if (rc) return rc;
  return copy_out(rx, rz, rt, out_x, out_z, out_theta, cap, out_count);
}

int cliff_map_paulis(const sv_cliff *f, const uint64_t *x, const uint64_t *z, size_t count, uint64_t *out_x,
                     uint64_t *out_z, int *out_sign) {
  if (!f) return fail(SV_EINVAL, "frame is NULL");
  if (count && (!x || !z || !out_x || !out_z || !out_sign)) return fail(SV_EINVAL, "NULL term arrays");
  const uint64_t lim = (1ULL << f->n) - 1;
  for (size_t k = 0; k < count; ++k)
    if ((x[k] | z[k]) & ~lim) return fail(SV_EINVAL, "term %zu has bits at or above n = %d", k, f->n);
  for (size_t k = 0; k < count; ++k) {
    const Pauli m = frame_map(f, pauli_string(x[k], z[k]));
    out_x[k] = m.x;
    out_z[k] = m.z;
    out_sign[k] = hermitian_sign(m);
  }
  return SV_OK;
}

int cliff_entry(const sv_cliff *f, int qubit, uint64_t *ez_x, uint64_t *ez_z, int *ez_sign, uint64_t *ex_x,
                uint64_t *ex_z, int *ex_sign) {
  if (!f || !ez_x || !ez_z || !ez_sign || !ex_x || !ex_z || !ex_sign) return fail(SV_EINVAL, "NULL argument");
  if (!valid_qubit(f, qubit)) return fail(SV_EINVAL, "qubit %d out of range", qubit);
  const Pauli &a = f->ez[qubit], &b = f->ex[qubit];
  *ez_x = a.x;
  *ez_z = a.z;
  *ez_sign = hermitian_sign(a);
  *ex_x = b.x;
  *ex_z = b.z;
  *ex_sign = hermitian_sign(b);
  return SV_OK;
}

int cliff_is_origin(const sv_cliff *f, int *out) {
  if (!f || !out) return fail(SV_EINVAL, "NULL argument");
  *out = is_origin(f) ? 1 : 0;
  return SV_OK;
}

int cliff_inverse_rotations(const sv_cliff *f, uint64_t *out_x, uint64_t *out_z, double *out_theta, size_t cap,
                            size_t *out_count) {
  if (!f) return fail(SV_EINVAL, "frame is NULL");
  std::vector<uint64_t> rx, rz;
  std::vector<double> rt;
  frame_rotations(f, rx, rz, rt);
  return copy_out(rx, rz, rt, out_x, out_z, out_theta, cap, out_count);
}

int cfhs_apply_gates(sv_state *sv, sv_cliff *f, const int *gate, const int *q0, const int *q1, const double *theta,
                     size_t count) {
  int rc = check_pair(sv, f);
  if (rc) return rc;
  std::vector<uint64_t> rx, rz;
  std::vector<double> rt;
  rc = frame_stream(f, gate, q0, q1, theta, count, rx, rz, rt);
  if (rc) return rc;
  // Clifford gates touch only F, so Phi's rotations can be applied together
  return rt.empty() ? SV_OK : apply_pauli_rotations(sv, rx.data(), rz.data(), rt.data(), rt.size());
}

int cfhs_apply_rotations(sv_state *sv, const sv_cliff *f, const uint64_t *x, const uint64_t *z, const double *theta,
                         size_t count) {
  int rc = check_pair(sv, f);
  if (rc) return rc;
  if (count && !theta) return fail(SV_EINVAL, "NULL angles");
  std::vector<uint64_t> mx(count), mz(count);
  std::vector<int> sg(count);
  rc = cliff_map_paulis(f, x, z, count, mx.data(), mz.data(), sg.data());
  if (rc) return rc;
  std::vector<double> mt(count);
  for (size_t k = 0; k < count; ++k) mt[k] = sg[k] * theta[k];
  return count ? apply_pauli_rotations(sv, mx.data(), mz.data(), mt.data(), count) : SV_OK;
}

int cfhs_expval(sv_state *sv, const sv_cliff *f, const uint64_t *x, const uint64_t *z, const double *coeff,
                size_t count, double *out_energy, double *out_norm2) {
  int rc = check_pair(sv, f);
  if (rc) return rc;
  if (count && !coeff) return fail(SV_EINVAL, "NULL coefficients");
  std::vector<uint64_t> mx(count), mz(count);
  std::vector<int> sg(count);
  rc = cliff_map_paulis(f, x, z, count, mx.data(), mz.data(), sg.data());
  if (rc) return rc;
  std::vector<double> mc(count);
  for (size_t k = 0; k < count; ++k) mc[k] = sg[k] * coeff[k];
  return expval_pauli_sum(sv, mx.data(), mz.data(), mc.data(), count, out_energy, out_norm2);
}

int cfhs_materialize(sv_state *sv, sv_cliff *f) {
  int rc = check_pair(sv, f);
  if (rc) return rc;
  std::vector<uint64_t> rx, rz;
  std::vector<double> rt;
  frame_rotations(f, rx, rz, rt);
  if (!rt.empty()) {
    rc = apply_pauli_rotations(sv, rx.data(), rz.data(), rt.data(), rt.size());
    if (rc) return rc;
  }
  set_origin(f);
  return SV_OK;
}

}  // extern "C"
