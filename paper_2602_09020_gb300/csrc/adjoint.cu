// Adjoint gradient of E = <psi|H|psi>, psi = R_M ... R_1 psi0 (not in the
// paper).  From d/dtheta R_P(theta) = -(i/2) P R_P(theta):
//     dE/dtheta_j = Im <lambda_j| P_j |phi_j>,
// with phi_j the state right after R_j and lambda_j = R_{j+1}^dag ... R_M^dag H psi.
// One backward pass per rotation reads phi and lambda once, accumulates the
// FP64 partial of Im<lambda|P|phi> and applies R_j^dag = R_P(-beta) to both.
// In the frame representation |psi> = Q|phi>, rotation j acted on |phi> about
// +-P_j with the applied (reduced) angle beta_j; the gradient picks up the
// same frame sign (see plan.cu for the reduction).
#include <cmath>
#include <vector>

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

__device__ __forceinline__ void block_sum1(double &a) {
  __shared__ double sa[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) sa[w] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sa[i];
    a = r;
  }
}

// i^{ny} * s as (re, im)
__device__ __forceinline__ double2 unit(int ny, int neg) {
  double re = 0.0, im = 0.0;
  switch (ny & 3) {
    case 0: re = 1.0; break;
    case 1: im = 1.0; break;
    case 2: re = -1.0; break;
    default: im = -1.0; break;
  }
  if (neg) {
    re = -re;
    im = -im;
  }
  return make_double2(re, im);
}

__device__ __forceinline__ double2 mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_adjoint_step(typename Cx<R>::T *__restrict__ phi, typename Cx<R>::T *__restrict__ lam, uint64_t n_amps,
                   uint64_t x, uint64_t z, double c, double s, double *__restrict__ partials) {
  using C = typename Cx<R>::T;
  const int ny = __popcll(x & z);
  const int h = x ? 63 - __clzll((long long)x) : -1;
  const uint64_t work = x ? n_amps >> 1 : n_amps;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  double g = 0.0;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < work; t += stride) {
    if (x == 0) {
      const C pv = phi[t], lv = lam[t];
      const double2 p = make_double2(pv.x, pv.y), l = make_double2(lv.x, lv.y);
      const double sg = (__popcll(t & z) & 1) ? -1.0 : 1.0;
      // Im(conj(l) * sg * p)
      g += sg * (l.x * p.y - l.y * p.x);
      // R(-beta) = c + i s P: a <- c a + i s sg a
      const double2 pn = make_double2(c * p.x - s * sg * p.y, c * p.y + s * sg * p.x);
      const double2 ln = make_double2(c * l.x - s * sg * l.y, c * l.y + s * sg * l.x);
      C po, lo;
      po.x = (R)pn.x; po.y = (R)pn.y;
      lo.x = (R)ln.x; lo.y = (R)ln.y;
      phi[t] = po;
      lam[t] = lo;
    } else {
      const uint64_t k = ((t >> h) << (h + 1)) | (t & ((1ULL << h) - 1));
      const uint64_t m = k ^ x;
      const C pk = phi[k], pm = phi[m], lk = lam[k], lm = lam[m];
      const double2 p0 = make_double2(pk.x, pk.y), p1 = make_double2(pm.x, pm.y);
      const double2 l0 = make_double2(lk.x, lk.y), l1 = make_double2(lm.x, lm.y);
      // (P v)_k = i^{nY} s(m) v_m ; (P v)_m = i^{nY} s(k) v_k
      const double2 uk = unit(ny, __popcll(m & z) & 1), um = unit(ny, __popcll(k & z) & 1);
      const double2 Pp0 = mul(uk, p1), Pp1 = mul(um, p0);
      const double2 Pl0 = mul(uk, l1), Pl1 = mul(um, l0);
      g += (l0.x * Pp0.y - l0.y * Pp0.x) + (l1.x * Pp1.y - l1.y * Pp1.x);
      // v <- c v + i s P v
      C o;
      o.x = (R)(c * p0.x - s * Pp0.y); o.y = (R)(c * p0.y + s * Pp0.x); phi[k] = o;
      o.x = (R)(c * p1.x - s * Pp1.y); o.y = (R)(c * p1.y + s * Pp1.x); phi[m] = o;
      o.x = (R)(c * l0.x - s * Pl0.y); o.y = (R)(c * l0.y + s * Pl0.x); lam[k] = o;
      o.x = (R)(c * l1.x - s * Pl1.y); o.y = (R)(c * l1.y + s * Pl1.x); lam[m] = o;
    }
  }
  block_sum1(g);
  if (threadIdx.x == 0) partials[blockIdx.x] = g;
}

__global__ void k_sum_rows(const double *__restrict__ partials, int n_blocks, double *__restrict__ out) {
  const double *p = partials + (size_t)blockIdx.x * n_blocks;
  double a = 0.0;
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) a += p[i];
  block_sum1(a);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

int step_blocks(int n) {
  uint64_t work = (1ULL << n) >> 1;
  uint64_t need = (work + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)device_sm_count() * 4;
  uint64_t b = need < cap ? need : cap;
  return b ? (int)b : 1;
}

}  // namespace

int adjoint_step(sv_state *phi, sv_state *lam, uint64_t x, uint64_t z, double beta, double *d_out) {
  const int blocks = step_blocks(phi->n);
  const double c = std::cos(0.5 * beta), s = std::sin(0.5 * beta);
  const uint64_t n_amps = 1ULL << phi->n;
  const int tr = trace_begin(phi);
  if (phi->dtype == SV_C128)
    k_adjoint_step<double><<<blocks, kThreads, 0, phi->stream>>>((double2 *)phi->amps, (double2 *)lam->amps,
                                                                 n_amps, x, z, c, s, d_out);
  else
    k_adjoint_step<float><<<blocks, kThreads, 0, phi->stream>>>((float2 *)phi->amps, (float2 *)lam->amps,
                                                                n_amps, x, z, c, s, d_out);
  PR_CHECK_LAUNCH();
  trace_end(phi, tr, KN_ADJOINT, 4.0 * (double)amp_bytes(phi->dtype) * (double)n_amps);
  return SV_OK;
}

}  // namespace pr

using namespace pr;

extern "C" {

int rotation_grads(sv_state *psi0, const uint64_t *x, const uint64_t *z, const double *angles, size_t n_rot,
                   const uint64_t *hx, const uint64_t *hz, const double *hc, size_t n_terms, double *out_energy,
                   double *out_grads) {
  if (!psi0) return fail(SV_EINVAL, "psi0 is NULL");
  if (n_rot && !out_grads) return fail(SV_EINVAL, "out_grads is NULL");
  sv_plan *plan = nullptr;
  int rc = plan_create(&plan, psi0->n, psi0->dtype, x, z, angles, n_rot, -1, psi0->stream);
  if (rc) return rc;
  sv_state *phi = nullptr, *lam = nullptr;
  rc = sv_alloc(&phi, psi0->n, psi0->dtype, psi0->stream);
  if (!rc) rc = sv_alloc(&lam, psi0->n, psi0->dtype, psi0->stream);
  const Pauli q0 = psi0->frame;
  if (!rc) rc = sv_copy(phi, psi0);
  if (!rc) rc = apply_plan(phi, plan);
  double energy = 0.0;
  if (!rc) rc = expval_impl(phi, hx, hz, hc, n_terms, &energy, nullptr);
  if (!rc) rc = pauli_sum_impl(lam, phi, hx, hz, hc, n_terms);
  const size_t L = plan ? plan->order.size() : 0;
  const int blocks = step_blocks(psi0->n);
  if (!rc) rc = ensure_scratch(phi, (size_t)blocks * (L ? L : 1), L ? L : 1);
  if (!rc) {
    for (size_t i = L; i-- > 0;) {
      if (plan->sigma[i] == 0) {
        // identity string: only a global phase, zero gradient; keep a zero row
        cudaError_t e = cudaMemsetAsync(phi->d_partials + (size_t)blocks * i, 0, sizeof(double) * blocks,
                                        phi->stream);
        if (e != cudaSuccess) {
          rc = fail(SV_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
          break;
        }
        continue;
      }
      const int s0 = anticommute(plan->ox[i], plan->oz[i], q0.x, q0.z) ? -1 : 1;
      rc = adjoint_step(phi, lam, plan->ox[i], plan->oz[i], s0 * plan->beta[i],
                        phi->d_partials + (size_t)blocks * i);
      if (rc) break;
    }
  }
  if (!rc && L) {
    k_sum_rows<<<(unsigned)L, kThreads, 0, phi->stream>>>(phi->d_partials, blocks, phi->d_results);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) rc = fail(SV_ECUDA, "k_sum_rows: %s", cudaGetErrorString(e));
  }
  if (!rc && L) {
    cudaError_t e = cudaMemcpyAsync(phi->h_results, phi->d_results, L * sizeof(double), cudaMemcpyDeviceToHost,
                                    phi->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(phi->stream);
    if (e != cudaSuccess) rc = fail(SV_ECUDA, "gradient copy: %s", cudaGetErrorString(e));
  }
  if (!rc) {
    for (size_t j = 0; j < n_rot; ++j) out_grads[j] = 0.0;
    for (size_t i = 0; i < L; ++i) {
      if (plan->sigma[i] == 0) continue;
      const int s0 = anticommute(plan->ox[i], plan->oz[i], q0.x, q0.z) ? -1 : 1;
      out_grads[plan->order[i]] = (double)(s0 * plan->sigma[i]) * phi->h_results[i];
    }
    if (out_energy) *out_energy = energy;
  }
  sv_free(lam);
  sv_free(phi);
  plan_free(plan);
  return rc;
}

}  // extern "C"
