// Host side of the rotation path: Trotter expansion, Pauli-frame rewrite,
// angle reduction into the frame, and the planner that packs a rotation list
// into fused runs (one HBM pass each).
//
// Tan form.  R_P(a) = cos(a/2) [I - i tan(a/2) P], so a pass can apply
// a_k <- a_k - i t (P a)_k with one multiply-add per real component and leave
// the positive factor cos(a/2) to a running scale that a later pass folds in.
// With |a| <= pi/2 the factor is >= 1/sqrt2 and |t| <= 1.  Larger angles are
// brought into range with R_P(a) = (-i P) R_P(a - pi) = (i P) R_P(a + pi): the
// Pauli factor goes into the frame (paper: Pauli operations are absorbed by the
// frame), so the device never sees it.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "internal.h"

namespace pr {

namespace {

constexpr double kPi = 3.14159265358979323846;

struct Item {
  uint64_t x, z;
  double theta;   // as given
  int64_t idx;    // position in the caller's list
};

// fold thresholds on log2 of the amplitude growth bound since the last fold
double fold_half(int dtype) { return dtype == SV_C128 ? 400.0 : 30.0; }

uint64_t fixed_half_angle(double theta) {
  // theta/2 as a fraction of a full turn in units of 2^-64 (wraps mod 2 pi)
  double q = theta / (4.0 * kPi);
  q -= std::nearbyint(q);  // [-0.5, 0.5]
  double s = std::ldexp(q, 64);
  if (s >= 9223372036854775807.0) return 0x8000000000000000ULL;
  if (s <= -9223372036854775808.0) return 0x8000000000000000ULL;
  return (uint64_t)(int64_t)std::llround(s);
}

struct RunBuilder {
  uint64_t basis[kDMax];
  int piv[kDMax];
  int d = 0;
  std::vector<size_t> members;  // indices into the effective list
  double growth = 0.0;

  void reset() {
    d = 0;
    members.clear();
    growth = 0.0;
  }
  uint64_t reduce(uint64_t x) const {
    for (int b = 0; b < d; ++b)
      if ((x >> piv[b]) & 1ULL) x ^= basis[b];
    return x;
  }
  void add_vector(uint64_t r) {
    int p = 63 - __builtin_clzll(r);
    for (int b = 0; b < d; ++b)
      if ((basis[b] >> p) & 1ULL) basis[b] ^= r;
    // insert keeping pivots ascending
    int pos = d;
    while (pos > 0 && piv[pos - 1] > p) {
      basis[pos] = basis[pos - 1];
      piv[pos] = piv[pos - 1];
      --pos;
    }
    basis[pos] = r;
    piv[pos] = p;
    ++d;
  }
};

struct Eff {
  uint64_t x, z;
  double t;      // tan of the reduced angle (plan-frame sign included)
  double c;      // cos of the reduced angle
};

}  // namespace

int build_plan(sv_plan *p, int n, int dtype, const uint64_t *x, const uint64_t *z,
               const double *theta, size_t count, int fusion_depth, cudaStream_t stream, bool upload,
               PlanSink *sink) {
  (void)stream;
  if (n < 1 || n > max_qubits(dtype)) return fail(SV_EINVAL, "bad n_qubits %d", n);
  if (count && (!x || !z || !theta)) return fail(SV_EINVAL, "NULL rotation arrays");
  int rc = validate_masks(n, x, z, count);
  if (rc) return rc;
  for (size_t j = 0; j < count; ++j)
    if (!std::isfinite(theta[j])) return fail(SV_EINVAL, "angle %zu is not finite", j);
  int dmax = fusion_depth;
  if (dmax < 0) {
    const int t = tuned_depth(n, dtype);
    dmax = t > 0 ? t : default_depth(dtype);
  }
  if (dmax > kDMax) return fail(SV_EINVAL, "fusion_depth must be <= %d", kDMax);
  if (dmax > n) dmax = n;

  p->n = n;
  p->dtype = dtype;
  p->dmax = dmax;
  p->runs.clear();
  p->n_input = count;
  p->frame = Pauli();
  p->order.clear();
  p->beta.clear();
  p->sigma.clear();
  p->ox.clear();
  p->oz.clear();

  std::vector<RotDev> rots;
  std::vector<DiagDev> diags;
  rots.reserve(count);
  p->order.reserve(count);
  p->beta.reserve(count);
  p->sigma.reserve(count);
  p->ox.reserve(count);
  p->oz.reserve(count);
  std::complex<double> scale(1.0, 0.0);
  double growth_since_fold = 0.0;

  // identity strings: a global phase, kept in the scale
  std::vector<Item> items;
  items.reserve(count);
  for (size_t j = 0; j < count; ++j) {
    if (x[j] == 0 && z[j] == 0) {
      scale *= std::exp(std::complex<double>(0.0, -0.5 * theta[j]));
      p->order.push_back((int64_t)j);
      p->beta.push_back(0.0);
      p->sigma.push_back(0);  // marks an identity (zero gradient)
      p->ox.push_back(0);
      p->oz.push_back(0);
      continue;
    }
    items.push_back({x[j], z[j], theta[j], (int64_t)j});
  }

  // diagonal stretches long enough for the phase-sum pass
  const size_t diag_min = 8;
  std::vector<int> in_diag(items.size(), 0);
  if (n >= kDiagMinQubits) {
    size_t a = 0;
    while (a < items.size()) {
      if (items[a].x != 0) {
        ++a;
        continue;
      }
      size_t b = a;
      while (b < items.size() && items[b].x == 0) ++b;
      if (b - a >= diag_min)
        for (size_t k = a; k < b; ++k) in_diag[k] = 1;
      a = b;
    }
  }

  RunBuilder rb;
  std::vector<Eff> eff;
  eff.reserve(items.size());
  Pauli qp;  // frame factors taken out so far (plan frame)
  const double gcap = fold_half(dtype);

  auto finish_coset_run = [&](bool force_fold) -> int {
    if (rb.members.empty() && !force_fold) return SV_OK;
    RunDev r;
    std::memset(&r, 0, sizeof(r));
    r.kind = 0;
    r.d = rb.d;
    for (int b = 0; b < rb.d; ++b) {
      r.basis[b] = rb.basis[b];
      r.piv[b] = rb.piv[b];
    }
    r.first = (int32_t)rots.size();
    r.count = (int32_t)rb.members.size();
    for (size_t m : rb.members) {
      const Eff &e = eff[m];
      uint32_t u = 0;
      for (int b = 0; b < rb.d; ++b)
        if ((e.x >> rb.piv[b]) & 1ULL) u |= 1u << b;
      // bit l of zt = parity(z & offset_l), offset_l = xor of the basis vectors
      // selected by l: the xor of the index masks {l : bit b of l} over the
      // basis vectors b with odd parity(z & basis_b)
      static const uint32_t kSel[kDMax] = {0xAAAAAAAAu, 0xCCCCCCCCu, 0xF0F0F0F0u, 0xFF00FF00u, 0xFFFF0000u};
      uint32_t zt = 0;
      for (int b = 0; b < rb.d; ++b)
        if (popc64(rb.basis[b] & e.z) & 1) zt ^= kSel[b];
      zt &= (rb.d >= 5) ? 0xFFFFFFFFu : ((1u << (1 << rb.d)) - 1u);
      int ny = popc64(e.x & e.z) & 3;
      int imag = (ny & 1) == 0;
      double ks = (ny == 0 || ny == 1) ? -1.0 : 1.0;  // kappa = (-i)^{nY+1}
      RotDev d;
      d.x = e.x;
      d.z = e.z;
      d.t = ks * e.t;
      d.zt = zt;
      d.code = (u << 1) | (uint32_t)imag;
      rots.push_back(d);
    }
    // segments: stretches of consecutive rotations with the same code
    for (size_t i = (size_t)r.first; i < rots.size();) {
      size_t e = i + 1;
      while (e < rots.size() && rots[e].code == rots[i].code) ++e;
      rots[i].code |= (uint32_t)(e - i) << kSegShift;
      i = e;
    }
    growth_since_fold += rb.growth;
    if (force_fold || growth_since_fold > gcap) {
      r.fold = 1;
      r.fold_re = scale.real();
      r.fold_im = scale.imag();
      scale = std::complex<double>(1.0, 0.0);
      growth_since_fold = 0.0;
    }
    p->runs.push_back(r);
    rb.reset();
    return sink ? sink->run(p, rots, diags) : SV_OK;
  };

  size_t k = 0;
  while (k < items.size()) {
    if (in_diag[k]) {
      rc = finish_coset_run(false);
      if (rc) return rc;
      // one phase-sum run over items[k, b) (all diagonal, so any order is
      // exact), cut at kMaxDiagRots rotations or kDiagSlots distinct patterns
      // of index bits 0..8 in the z-masks
      size_t b = k;
      {
        bool seen[1 << kDiagSlotBits] = {};
        int distinct = 0;
        while (b < items.size() && in_diag[b] && b - k < (size_t)kMaxDiagRots) {
          const int m = (int)(items[b].z & ((1u << kDiagSlotBits) - 1));
          if (!seen[m]) {
            if (distinct == kDiagSlots) break;
            seen[m] = true;
            ++distinct;
          }
          ++b;
        }
      }
      std::vector<DiagDev> chunk;
      std::vector<int> cls;
      for (size_t m = k; m < b; ++m) {
        const Item &it = items[m];
        int sp = anticommute(it.x, it.z, qp.x, qp.z) ? -1 : 1;
        DiagDev dd;
        dd.z = it.z;
        dd.a = fixed_half_angle(sp * it.theta);
        dd.slot = 0;
        dd.pad = 0;
        chunk.push_back(dd);
        // sort key: the z pattern on index bits 0..8, class bits 5..8 first
        cls.push_back((int)(it.z & ((1u << kDiagSlotBits) - 1)));
        p->order.push_back(it.idx);
        p->beta.push_back(sp * it.theta);
        p->sigma.push_back((int8_t)sp);
        p->ox.push_back(it.x);
        p->oz.push_back(it.z);
      }
      // stable sort by pattern; the adjoint order follows the device order
      std::vector<size_t> perm(chunk.size());
      for (size_t m = 0; m < perm.size(); ++m) perm[m] = m;
      std::stable_sort(perm.begin(), perm.end(), [&](size_t a1, size_t b1) { return cls[a1] < cls[b1]; });
      size_t base_order = p->order.size() - chunk.size();
      std::vector<int64_t> o2(chunk.size());
      std::vector<double> b2(chunk.size());
      std::vector<int8_t> s2(chunk.size());
      std::vector<uint64_t> x2(chunk.size()), z2(chunk.size());
      RunDev r;
      std::memset(&r, 0, sizeof(r));
      r.kind = 1;
      r.first = (int32_t)diags.size();
      r.count = (int32_t)chunk.size();
      // slots: the distinct patterns in sorted order; seg[c] = first slot of
      // class c (pattern bits 5..8), seg[16] = number of slots
      int cur = 0, slot = -1, last = -1;
      r.seg[0] = 0;
      for (size_t m = 0; m < perm.size(); ++m) {
        size_t src = perm[m];
        if (cls[src] != last) {
          ++slot;
          last = cls[src];
          while (cur < (cls[src] >> kDiagClassLo)) r.seg[++cur] = (int32_t)slot;
        }
        chunk[src].slot = (uint32_t)slot;
        diags.push_back(chunk[src]);
        o2[m] = p->order[base_order + src];
        b2[m] = p->beta[base_order + src];
        s2[m] = p->sigma[base_order + src];
        x2[m] = p->ox[base_order + src];
        z2[m] = p->oz[base_order + src];
      }
      while (cur < (1 << kDiagClassBits)) r.seg[++cur] = (int32_t)(slot + 1);
      for (size_t m = 0; m < perm.size(); ++m) {
        p->order[base_order + m] = o2[m];
        p->beta[base_order + m] = b2[m];
        p->sigma[base_order + m] = s2[m];
        p->ox[base_order + m] = x2[m];
        p->oz[base_order + m] = z2[m];
      }
      p->runs.push_back(r);
      p->n_diag_runs++;
      if (sink) {
        rc = sink->run(p, rots, diags);
        if (rc) return rc;
      }
      k = b;
      continue;
    }

    const Item &it = items[k];
    int sp = anticommute(it.x, it.z, qp.x, qp.z) ? -1 : 1;
    double a = sp * it.theta;
    // exp(-i a/2 P) is periodic up to sign: a -> a - 2 pi m gives a factor (-1)^m
    double m2 = std::nearbyint(a / (2.0 * kPi));
    if (m2 != 0.0) {
      a -= 2.0 * kPi * m2;
      if (std::fmod(std::fabs(m2), 2.0) == 1.0) scale = -scale;
    }
    if (a > 0.5 * kPi) {
      // R_P(a) = (-i P) R_P(a - pi)
      a -= kPi;
      Pauli f = pauli_string(it.x, it.z);
      f.q = (f.q + 3) & 3;
      qp = pauli_mul(qp, f);
    } else if (a < -0.5 * kPi) {
      // R_P(a) = (i P) R_P(a + pi)
      a += kPi;
      Pauli f = pauli_string(it.x, it.z);
      f.q = (f.q + 1) & 3;
      qp = pauli_mul(qp, f);
    }
    Eff e;
    e.x = it.x;
    e.z = it.z;
    e.t = std::tan(0.5 * a);
    // cos(a/2) = 1/sqrt(1 + tan^2) for |a/2| <= pi/4: the scale of exactly the
    // rotation the tan form applies; growth bound -log2 cos = log2(1 + t^2) / 2
    const double q = 1.0 + e.t * e.t;
    e.c = 1.0 / std::sqrt(q);
    double g = 0.5 * std::log2(q);
    p->order.push_back(it.idx);
    p->beta.push_back(a);
    p->sigma.push_back((int8_t)sp);
    p->ox.push_back(it.x);
    p->oz.push_back(it.z);

    // does it fit the open run?
    bool fits = rb.members.size() < (size_t)kMaxRunRots && rb.growth + g <= gcap;
    uint64_t r = 0;
    if (fits && it.x != 0) {
      r = rb.reduce(it.x);
      if (r != 0 && rb.d >= dmax) fits = false;
    }
    if (!fits) {
      rc = finish_coset_run(false);
      if (rc) return rc;
      r = it.x ? rb.reduce(it.x) : 0;
    }
    if (r != 0) rb.add_vector(r);
    eff.push_back(e);
    rb.members.push_back(eff.size() - 1);
    rb.growth += g;
    scale *= e.c;
    ++k;
  }
  bool need_fold = std::abs(scale - std::complex<double>(1.0, 0.0)) != 0.0;
  if (!rb.members.empty()) {
    rc = finish_coset_run(need_fold);
    if (rc) return rc;
  } else if (need_fold) {
    if (!p->runs.empty()) {
      RunDev &last = p->runs.back();
      // multiply onto an existing fold or add one
      std::complex<double> f = last.fold ? std::complex<double>(last.fold_re, last.fold_im) : 1.0;
      f *= scale;
      last.fold = 1;
      last.fold_re = f.real();
      last.fold_im = f.imag();
    } else {
      rc = finish_coset_run(true);  // an empty d = 0 run that only scales
      if (rc) return rc;
    }
  }
  p->frame = qp;
  p->n_effective = items.size();
  p->n_rots = rots.size();
  p->n_diag = diags.size();
  if (sink) return sink->finish(p, rots, diags);
  build_chains(p);
  if (!upload) return SV_OK;

  if (!diags.empty()) {
    rc = prepare_tables(dtype);
    if (rc) return rc;
  }
  // upload
  if (p->d_rots) cudaFree(p->d_rots);
  if (p->d_diag) cudaFree(p->d_diag);
  p->d_rots = nullptr;
  p->d_diag = nullptr;
  if (!rots.empty()) {
    if (cudaMalloc(&p->d_rots, rots.size() * sizeof(RotDev)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "plan upload allocation failed");
    }
    PR_CUDA(cudaMemcpy(p->d_rots, rots.data(), rots.size() * sizeof(RotDev), cudaMemcpyHostToDevice));
  }
  if (!diags.empty()) {
    if (cudaMalloc(&p->d_diag, diags.size() * sizeof(DiagDev)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "plan upload allocation failed");
    }
    PR_CUDA(cudaMemcpy(p->d_diag, diags.data(), diags.size() * sizeof(DiagDev), cudaMemcpyHostToDevice));
  }
  return SV_OK;
}

int apply_plan(sv_state *sv, sv_plan *plan) {
  if (!sv || !plan) return fail(SV_EINVAL, "NULL argument");
  if (sv->n != plan->n || sv->dtype != plan->dtype)
    return fail(SV_EINVAL, "plan built for n=%d dtype=%d, state has n=%d dtype=%d", plan->n, plan->dtype,
                sv->n, sv->dtype);
  const Pauli q0 = sv->frame;
  if (plan->steps.empty()) {
    for (const RunDev &r : plan->runs) {
      int rc = launch_run(sv, plan, r, q0.x, q0.z);
      if (rc) return rc;
    }
  } else {
    for (const PlanStep &st : plan->steps) {
      int rc = st.chain >= 0 ? launch_chain(sv, plan, plan->chains[st.chain], q0.x, q0.z)
                             : launch_run(sv, plan, plan->runs[st.run], q0.x, q0.z);
      if (rc) return rc;
    }
  }
  // Q <- Q0 Qp (-1)^{<Qp, Q0>}: the frame factors picked up the runtime signs
  Pauli f = pauli_mul(q0, plan->frame);
  if (anticommute(plan->frame.x, plan->frame.z, q0.x, q0.z)) f.q = (f.q + 2) & 3;
  sv->frame = f;
  return SV_OK;
}

namespace {

// apply_pauli_rotations without a stored plan: the planner hands over each run
// as it is made, and runs are launched in batches while it works on the rest
// of the list.  The launches (kernels, parameters, order, pairing into chained
// passes) are the ones plan_create + plan_apply make for the same list, so the
// result is the same bit for bit; the planning time overlaps the device work
// instead of preceding it.  Records reach the device by asynchronous copies from
// the handle's pinned staging buffer, on the handle's stream, before the runs
// that read them.
struct StreamLauncher final : PlanSink {
  static constexpr size_t kBatch = 16;  // runs per copy-and-launch batch
  sv_state *sv;
  Pauli q0;
  size_t rot_slots;
  bool init = false, chain = false;
  size_t next = 0;    // runs [0, next) are launched or pending
  long pending = -1;  // a run waiting to be paired with its successor
  size_t up_rots = 0, up_diags = 0;

  StreamLauncher(sv_state *s, size_t slots) : sv(s), q0(s->frame), rot_slots(slots) {}

  int upload(const std::vector<RotDev> &rots, const std::vector<DiagDev> &diags) {
    char *h = (char *)sv->h_rec, *d = (char *)sv->d_rec;
    if (rots.size() > up_rots) {
      const size_t off = up_rots * sizeof(RotDev), nb = (rots.size() - up_rots) * sizeof(RotDev);
      std::memcpy(h + off, rots.data() + up_rots, nb);
      PR_CUDA(cudaMemcpyAsync(d + off, h + off, nb, cudaMemcpyHostToDevice, sv->stream));
      up_rots = rots.size();
    }
    if (diags.size() > up_diags) {
      const size_t off = rot_slots * sizeof(RotDev) + up_diags * sizeof(DiagDev);
      const size_t nb = (diags.size() - up_diags) * sizeof(DiagDev);
      std::memcpy(h + off, diags.data() + up_diags, nb);
      PR_CUDA(cudaMemcpyAsync(d + off, h + off, nb, cudaMemcpyHostToDevice, sv->stream));
      up_diags = diags.size();
    }
    PR_CUDA(cudaEventRecord(sv->rec_copied, sv->stream));
    return SV_OK;
  }

  // launch runs [next, upto), pairing them as build_chains does
  int launch_upto(sv_plan *p, size_t upto) {
    for (; next < upto; ++next) {
      int rc;
      if (pending >= 0) {
        ChainDev ch;
        const bool paired = chain_pair(p, (size_t)pending, &ch);
        rc = paired ? launch_chain(sv, p, ch, q0.x, q0.z) : launch_run(sv, p, p->runs[pending], q0.x, q0.z);
        pending = -1;
        if (rc) return rc;
        if (paired) continue;
      }
      if (chain) {
        pending = (long)next;
        continue;
      }
      rc = launch_run(sv, p, p->runs[next], q0.x, q0.z);
      if (rc) return rc;
    }
    return SV_OK;
  }

  int run(sv_plan *p, const std::vector<RotDev> &rots, const std::vector<DiagDev> &diags) override {
    if (!init) {
      chain = chains_enabled(p);
      init = true;
    }
    // the newest run may still take the closing fold: keep it back
    const size_t ready = p->runs.size() - 1;
    if (ready < next + kBatch) return SV_OK;
    int rc = upload(rots, diags);
    return rc ? rc : launch_upto(p, ready);
  }

  int finish(sv_plan *p, const std::vector<RotDev> &rots, const std::vector<DiagDev> &diags) override {
    if (!init) {
      chain = chains_enabled(p);
      init = true;
    }
    int rc = upload(rots, diags);
    if (!rc) rc = launch_upto(p, p->runs.size());
    if (!rc && pending >= 0) {
      rc = launch_run(sv, p, p->runs[pending], q0.x, q0.z);
      pending = -1;
    }
    if (rc) return rc;
    // Q <- Q0 Qp (-1)^{<Qp, Q0>}, as apply_plan does
    Pauli f = pauli_mul(q0, p->frame);
    if (anticommute(p->frame.x, p->frame.z, q0.x, q0.z)) f.q = (f.q + 2) & 3;
    sv->frame = f;
    return SV_OK;
  }
};

}  // namespace

}  // namespace pr

using namespace pr;

extern "C" {

int plan_create(sv_plan **out, int n_qubits, int dtype, const uint64_t *x, const uint64_t *z,
                const double *angles, size_t count, int fusion_depth, void *cuda_stream) {
  if (!out) return fail(SV_EINVAL, "out is NULL");
  *out = nullptr;
  if (dtype != SV_C128 && dtype != SV_C64) return fail(SV_EINVAL, "bad dtype");
  sv_plan *p = new (std::nothrow) sv_plan();
  if (!p) return fail(SV_ENOMEM, "host allocation failed");
  int rc = build_plan(p, n_qubits, dtype, x, z, angles, count, fusion_depth, (cudaStream_t)cuda_stream);
  if (rc) {
    plan_free(p);
    return rc;
  }
  *out = p;
  return SV_OK;
}

int plan_apply(sv_state *sv, sv_plan *plan) { return apply_plan(sv, plan); }

int plan_free(sv_plan *plan) {
  if (!plan) return SV_OK;
  batch_forget(nullptr, plan);
  cudaDeviceSynchronize();
  if (plan->d_rots) cudaFree(plan->d_rots);
  if (plan->d_diag) cudaFree(plan->d_diag);
  delete plan;
  return SV_OK;
}

int plan_inspect(int n_qubits, int dtype, const uint64_t *x, const uint64_t *z, const double *angles,
                 size_t count, int fusion_depth, sv_run_info *runs, size_t cap, size_t *out_runs,
                 size_t *out_rotations) {
  if (dtype != SV_C128 && dtype != SV_C64) return fail(SV_EINVAL, "bad dtype");
  if (cap && !runs) return fail(SV_EINVAL, "runs is NULL");
  sv_plan p;
  int rc = build_plan(&p, n_qubits, dtype, x, z, angles, count, fusion_depth, nullptr, false);
  if (rc) return rc;
  for (size_t i = 0; i < p.runs.size() && i < cap; ++i) {
    const RunDev &r = p.runs[i];
    sv_run_info &o = runs[i];
    std::memset(&o, 0, sizeof(o));
    o.kind = r.kind;
    o.d = r.kind == 0 ? r.d : 0;
    o.count = r.count;
    if (r.kind == 0)
      for (int b = 0; b < r.d && b < kDMax; ++b) o.basis[b] = r.basis[b];
  }
  if (out_runs) *out_runs = p.runs.size();
  if (out_rotations) *out_rotations = p.n_effective;
  return SV_OK;
}

int plan_stats(const sv_plan *plan, size_t *n_rotations, size_t *n_runs, size_t *n_diag_runs) {
  if (!plan) return fail(SV_EINVAL, "plan is NULL");
  if (n_rotations) *n_rotations = plan->n_effective;
  if (n_runs) *n_runs = plan->runs.size();
  if (n_diag_runs) *n_diag_runs = plan->n_diag_runs;
  return SV_OK;
}

int plan_sweeps(const sv_plan *plan, size_t *n_sweeps) {
  if (!plan || !n_sweeps) return fail(SV_EINVAL, "NULL argument");
  *n_sweeps = plan->steps.empty() ? plan->runs.size() : plan->steps.size();
  return SV_OK;
}

int apply_pauli_rotations(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *angles,
                          size_t count) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  // the previous call's records must have left the staging buffer
  if (sv->rec_copied) PR_CUDA(cudaEventSynchronize(sv->rec_copied));
  const size_t slots = count > 0 ? count : 1;
  const size_t need = slots * (sizeof(RotDev) + sizeof(DiagDev));
  if (sv->d_rec_cap < need) {
    if (sv->d_rec) PR_CUDA(cudaFree(sv->d_rec));  // synchronises with earlier launches
    sv->d_rec = nullptr;
    sv->d_rec_cap = 0;
    if (cudaMalloc(&sv->d_rec, need) != cudaSuccess) {
      cudaGetLastError();
      sv->d_rec = nullptr;
      return fail(SV_ENOMEM, "rotation record buffer allocation failed");
    }
    sv->d_rec_cap = need;
  }
  if (sv->h_rec_cap < need) {
    if (sv->h_rec) PR_CUDA(cudaFreeHost(sv->h_rec));
    sv->h_rec = nullptr;
    sv->h_rec_cap = 0;
    if (cudaHostAlloc(&sv->h_rec, need, cudaHostAllocDefault) != cudaSuccess) {
      cudaGetLastError();
      sv->h_rec = nullptr;
      return fail(SV_ENOMEM, "rotation record staging allocation failed");
    }
    sv->h_rec_cap = need;
  }
  if (!sv->rec_copied) PR_CUDA(cudaEventCreateWithFlags(&sv->rec_copied, cudaEventDisableTiming));
  if (!sv->rec_done) {
    PR_CUDA(cudaEventCreateWithFlags(&sv->rec_done, cudaEventDisableTiming));
  } else {
    // the previous call's passes read the device buffer, maybe on another
    // stream: this call's copies into it wait for them
    PR_CUDA(cudaStreamWaitEvent(sv->stream, sv->rec_done, 0));
  }
  sv_plan p;
  p.owns_device = false;
  p.d_rots = (RotDev *)sv->d_rec;
  p.d_diag = (DiagDev *)((char *)sv->d_rec + slots * sizeof(RotDev));
  StreamLauncher L(sv, slots);
  int rc = build_plan(&p, sv->n, sv->dtype, x, z, angles, count, -1, sv->stream, false, &L);
  p.d_rots = nullptr;
  p.d_diag = nullptr;
  // after the last launch of this call, also when it stopped early
  const cudaError_t er = cudaEventRecord(sv->rec_done, sv->stream);
  if (!rc && er != cudaSuccess) return fail(SV_ECUDA, "cudaEventRecord: %s", cudaGetErrorString(er));
  return rc;
}

int trotter_expand(const uint64_t *x, const uint64_t *z, const double *c, size_t n_terms, double dt,
                   int steps, int order, int merge, uint64_t *out_x, uint64_t *out_z, double *out_theta,
                   size_t cap, size_t *out_count) {
  if (!out_count) return fail(SV_EINVAL, "out_count is NULL");
  if (n_terms && (!x || !z || !c)) return fail(SV_EINVAL, "NULL term arrays");
  if (order != 1 && order != 2) return fail(SV_EINVAL, "order must be 1 or 2");
  if (steps < 0) return fail(SV_EINVAL, "steps must be >= 0");
  if (cap && (!out_x || !out_z || !out_theta)) return fail(SV_EINVAL, "NULL output arrays");
  if (!std::isfinite(dt)) return fail(SV_EINVAL, "dt is not finite");
  size_t w = 0;
  // merging needs the previous entry; when cap is too small count exactly
  // with a shadow of the last emitted string
  uint64_t last_x = ~0ULL, last_z = ~0ULL;
  bool have_last = false;
  auto emit2 = [&](uint64_t xx, uint64_t zz, double th) {
    if (merge && have_last && last_x == xx && last_z == zz) {
      if (w - 1 < cap) out_theta[w - 1] += th;
      return;
    }
    if (w < cap) {
      out_x[w] = xx;
      out_z[w] = zz;
      out_theta[w] = th;
    }
    ++w;
    last_x = xx;
    last_z = zz;
    have_last = true;
  };
  for (int s = 0; s < steps; ++s) {
    if (order == 1) {
      for (size_t j = 0; j < n_terms; ++j) emit2(x[j], z[j], 2.0 * c[j] * dt);
    } else {
      for (size_t j = 0; j < n_terms; ++j) emit2(x[j], z[j], c[j] * dt);
      for (size_t j = n_terms; j-- > 0;) emit2(x[j], z[j], c[j] * dt);
    }
  }
  *out_count = w;
  return SV_OK;
}

}  // extern "C"
