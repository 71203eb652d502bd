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
#include <cstring>
#include <vector>

#include "fixed64.cuh"
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

// ---- fused backward runs ------------------------------------------------------
//
// Im<lambda|P|phi> is a sum over amplitudes, and P pairs k with k^x inside any
// coset of a subspace that contains x.  So a run of consecutive rotations whose
// x-masks span <= kAdjD dimensions is walked backwards coset by coset: a thread
// keeps one coset of phi and of lambda in registers (FP64 for complex128 states,
// FP32 for complex64, gradient terms always summed in FP64) and, for each rotation
// of the run (latest first), adds the coset's share of Im<lambda|P_j|phi> to a
// per-rotation accumulator, then applies R_j^dag (tan form, below) to both.
// One read and one write of phi and lambda per run instead of per rotation.

constexpr int kAdjD = 3;     // run span dimension: 8 elements per coset
constexpr double kHalfPi = 1.5707963267948966;
constexpr int kAdjRun = 20;  // rotations per run (shared-memory accumulators)

struct AdjRotDev {
  uint64_t z;
  double t;      // R(-beta) = cos(beta/2) (1 + i t P), t = tan(beta/2)
  double unused;
  int32_t u;     // coordinates of x in the run basis
  int32_t ny;    // popc(x & z) mod 4
  uint32_t zt;   // bit e = parity(soff[e] & z)
  int32_t row;   // gradient row (plan order)
};
struct AdjRunDev {
  uint64_t soff[1 << kAdjD];
  int32_t piv[kAdjD];  // ascending
  int32_t count;
  double scale;  // product of cos(beta/2) over the run: restores the stored states
  AdjRotDev rot[kAdjRun];  // backward order
};

__host__ __device__ constexpr int adj_high_bit(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return h;
}

// Complex registers of the run: double2 for complex128 states; float2 for
// complex64, whose rotations are applied in FP32 (the precision the state is
// stored in) while every gradient term is accumulated in FP64.
template <typename V>
struct AdjScalar;
template <>
struct AdjScalar<double2> {
  using T = double;
};
template <>
struct AdjScalar<float2> {
  using T = float;
};
template <typename V>
__device__ __forceinline__ V adj_vec(typename AdjScalar<V>::T x, typename AdjScalar<V>::T y) {
  V v;
  v.x = x;
  v.y = y;
  return v;
}

// sum of N values as a tree (depth log2 N): the FP64 adds of one rotation's
// gradient do not wait on each other in one chain
template <int N>
__device__ __forceinline__ double tree_sum(double (&v)[N]) {
#pragma unroll
  for (int h = N / 2; h >= 1; h /= 2)
#pragma unroll
    for (int i = 0; i < h; ++i) v[i] += v[i + h];
  return v[0];
}

// Compensated FP32 sum (Neumaier): s + c equals the sum of the added values up
// to O(n u^2) of their magnitudes (u = 2^-24), so a coset's complex64 gradient
// terms reach the FP64 accumulator as two exactly widened floats and one FP64
// add instead of one FP64 add per term (GB300's FP64 pipe is narrow)
struct CompSum32 {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return widen_f64(s) + widen_f64(c); }
};

// Im(conj(a) b)
template <typename V>
__device__ __forceinline__ typename AdjScalar<V>::T im_conj_mul(V a, V b) {
  return a.x * b.y - a.y * b.x;
}

// i^K v, by swaps and negations
template <int K, typename V>
__device__ __forceinline__ V ipow(V v) {
  if constexpr ((K & 3) == 0) return v;
  if constexpr ((K & 3) == 1) return adj_vec<V>(-v.y, v.x);
  if constexpr ((K & 3) == 2) return adj_vec<V>(-v.x, -v.y);
  return adj_vec<V>(v.y, -v.x);
}

// Im(conj(a) i^K b)
template <int K, typename V>
__device__ __forceinline__ typename AdjScalar<V>::T im_conj_ipow(V a, V b) {
  if constexpr ((K & 3) == 0) return a.x * b.y - a.y * b.x;
  if constexpr ((K & 3) == 1) return a.x * b.x + a.y * b.y;
  if constexpr ((K & 3) == 2) return a.y * b.x - a.x * b.y;
  return -(a.x * b.x + a.y * b.y);
}

// One rotation on a coset, U = pairing pattern, K = nY mod 4.  With
// (P v)_e = i^K (-1)^{sigma_m} v_m for the partner m = e ^ U:
//   g   += (-1)^{sigma_m} Im(conj(lambda_e) i^K phi_m) + (e <-> m),
//   v_e <- v_e + t (-1)^{sigma_m} i^{K+1} v_m     (R^dag = cos (1 + i t P)),
// so the phase costs swaps and negations only.  The factor cos(beta/2) is left
// out: inside a run both vectors carry the same known scale, which the host
// folds into each gradient and the kernel into the stored states.  Each
// element's gradient term is formed in the state's precision; complex128 terms
// are summed in FP64, complex64 terms in a compensated FP32 sum per coset that
// reaches FP64 once per coset and rotation.
template <int U, int K, typename V>
__device__ __forceinline__ void adj_rot(V (&p)[1 << kAdjD], V (&l)[1 << kAdjD], const AdjRotDev &r, int sig,
                                        double &g) {
  using S = typename AdjScalar<V>::T;
  constexpr int E = 1 << kAdjD;
  const S t = (S)r.t;
  constexpr bool F32 = sizeof(S) == 4;
  CompSum32 acc;
  if constexpr (U == 0) {
    double part[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const bool neg = (sig ^ (int)(r.zt >> e)) & 1;
      const S ts = neg ? -t : t;
      const V pe = p[e], le = l[e];
      const S ge = im_conj_mul(le, pe);
      if constexpr (F32)
        acc.add(neg ? -ge : ge);
      else
        part[e] = widen_f64(neg ? -ge : ge);
      p[e] = adj_vec<V>(pe.x - ts * pe.y, pe.y + ts * pe.x);
      l[e] = adj_vec<V>(le.x - ts * le.y, le.y + ts * le.x);
    }
    if constexpr (F32)
      g = acc.value();
    else
      g = tree_sum(part);  // g enters as 0: no add of zero
  } else {
    constexpr int H = adj_high_bit(U);
    double part[E / 2];
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
      const int e = ((q >> H) << (H + 1)) | (q & ((1 << H) - 1));
      const int m = e ^ U;
      const bool ne = (sig ^ (int)(r.zt >> e)) & 1, nm = (sig ^ (int)(r.zt >> m)) & 1;
      const V pe = p[e], pm = p[m], le = l[e], lm = l[m];
      const S ge = im_conj_ipow<K>(le, pm), gm = im_conj_ipow<K>(lm, pe);
      if constexpr (F32) {
        acc.add(nm ? -ge : ge);
        acc.add(ne ? -gm : gm);
      } else {
        part[q] = widen_f64(nm ? -ge : ge) + widen_f64(ne ? -gm : gm);
      }
      const S te = ne ? -t : t, tm = nm ? -t : t;
      const V wpm = ipow<K + 1>(pm), wpe = ipow<K + 1>(pe), wlm = ipow<K + 1>(lm), wle = ipow<K + 1>(le);
      p[e] = adj_vec<V>(pe.x + tm * wpm.x, pe.y + tm * wpm.y);
      p[m] = adj_vec<V>(pm.x + te * wpe.x, pm.y + te * wpe.y);
      l[e] = adj_vec<V>(le.x + tm * wlm.x, le.y + tm * wlm.y);
      l[m] = adj_vec<V>(lm.x + te * wle.x, lm.y + te * wle.y);
    }
    if constexpr (F32)
      g = acc.value();
    else
      g = tree_sum(part);  // g enters as 0: no add of zero
  }
}

#define PR_ADJ_CASE(UK) \
  case UK: adj_rot<((UK) >> 2), ((UK)&3), V>(p, l, r, sig, g); break;

template <typename V>
__device__ __forceinline__ void adj_dispatch(int uk, V (&p)[1 << kAdjD], V (&l)[1 << kAdjD], const AdjRotDev &r,
                                             int sig, double &g) {
  switch (uk) {
    PR_ADJ_CASE(0)
    PR_ADJ_CASE(4) PR_ADJ_CASE(5) PR_ADJ_CASE(6) PR_ADJ_CASE(7)
    PR_ADJ_CASE(8) PR_ADJ_CASE(9) PR_ADJ_CASE(10) PR_ADJ_CASE(11)
    PR_ADJ_CASE(12) PR_ADJ_CASE(13) PR_ADJ_CASE(14) PR_ADJ_CASE(15)
    PR_ADJ_CASE(16) PR_ADJ_CASE(17) PR_ADJ_CASE(18) PR_ADJ_CASE(19)
    PR_ADJ_CASE(20) PR_ADJ_CASE(21) PR_ADJ_CASE(22) PR_ADJ_CASE(23)
    PR_ADJ_CASE(24) PR_ADJ_CASE(25) PR_ADJ_CASE(26) PR_ADJ_CASE(27)
    PR_ADJ_CASE(28) PR_ADJ_CASE(29) PR_ADJ_CASE(30) PR_ADJ_CASE(31)
    default: break;
  }
}

template <typename R>
__global__ void __launch_bounds__(kThreads)
    k_adjoint_run(typename Cx<R>::T *__restrict__ phi, typename Cx<R>::T *__restrict__ lam, uint64_t n_cosets,
                  const __grid_constant__ AdjRunDev run, int row_stride, double *__restrict__ partials) {
  using C = typename Cx<R>::T;
  constexpr int E = 1 << kAdjD;
  __shared__ double sacc[kAdjRun][kThreads];  // one column per thread
  // the run's rotation records in shared memory: read with the loop index
  // from the kernel parameter they would be indexed constant loads
  __shared__ AdjRotDev srot[kAdjRun];
  for (int j = 0; j < kAdjRun; ++j) sacc[j][threadIdx.x] = 0.0;
  const int count = run.count;
  if (threadIdx.x < count) srot[threadIdx.x] = run.rot[threadIdx.x];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t cs = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; cs < n_cosets; cs += stride) {
    uint64_t rep = cs;
#pragma unroll
    for (int b = 0; b < kAdjD; ++b) {
      const int pv = run.piv[b];
      rep = ((rep >> pv) << (pv + 1)) | (rep & ((1ULL << pv) - 1));
    }
    C p[E], l[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      p[e] = phi[rep ^ run.soff[e]];
      l[e] = lam[rep ^ run.soff[e]];
    }
    for (int j = 0; j < count; ++j) {
      const AdjRotDev &r = srot[j];
      // complex64: the accumulator is read before the rotation's work, so the
      // load's latency overlaps it instead of stalling the add (complex128
      // has no register to spare for it)
      double before = 0.0;
      if constexpr (sizeof(R) == 4) before = sacc[j][threadIdx.x];
      const int sig = __popcll(rep & r.z) & 1;
      double g = 0.0;
      adj_dispatch(r.u * 4 + r.ny, p, l, r, sig, g);  // x = 0 has nY = 0
      if constexpr (sizeof(R) == 4)
        sacc[j][threadIdx.x] = before + g;
      else
        sacc[j][threadIdx.x] += g;
    }
    const R sc = (R)run.scale;
#pragma unroll
    for (int e = 0; e < E; ++e) {
      phi[rep ^ run.soff[e]] = adj_vec<C>(sc * p[e].x, sc * p[e].y);
      lam[rep ^ run.soff[e]] = adj_vec<C>(sc * l[e].x, sc * l[e].y);
    }
  }
  __syncthreads();
  // block sums in a fixed order: warp w reduces rows w, w + 8, ...
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < count; j += (int)(blockDim.x >> 5)) {
    double v = 0.0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += sacc[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partials[(size_t)run.rot[j].row * row_stride + blockIdx.x] = v;
  }
}

// ---- complex128 backward runs in 64-bit fixed point ---------------------------
//
// The same run as k_adjoint_run<double> on the integer pipes (the FP64 version
// is bound by GB300's narrow FP64 pipe).  A thread converts its coset of phi
// and of lambda with one exponent each (fixed64.cuh: block floating point, the
// coset's 2-norm below 2^61); R_j^dag = cos(beta/2) (1 + i t P) is applied in tan
// form with truncated products, one per component and rotation, whose mean the
// run adds back at the end; both vectors are halved whenever the known growth
// sqrt(1 + t^2) per rotation passes a whole bit.  A rotation's share of
// Im<lambda|P|phi> over the coset is a sum of products of a lambda and a phi
// component (truncated, at the scale 2^(62 - S_phi - S_lambda)), summed exactly
// in 64 bits -- by Cauchy-Schwarz the sum stays below 2^61 -- then converted to
// FP64 once per coset and rotation and added to the FP64 accumulator.

struct AdjRotFx {
  uint64_t z;
  uint32_t zt;
  int32_t uk;     // u * 4 + nY mod 4
  int32_t th[2];  // limbs of +T and -T, T = round(t 2^62)
  int32_t tl[2];
  int32_t halve;  // 1: halve both vectors after this rotation
  int32_t pad;
};

// Im(conj(a) i^K b) from truncated products a_c b_c' / 2^62; b by its limbs
template <int K>
__device__ __forceinline__ int64_t fx_im_conj_ipow(int64_t ax, int64_t ay, int32_t bxh, int32_t bxl, int32_t byh,
                                                   int32_t byl) {
  if constexpr ((K & 3) == 0) return fx_prod(ax, byh, byl) - fx_prod(ay, bxh, bxl);
  if constexpr ((K & 3) == 1) return fx_prod(ax, bxh, bxl) + fx_prod(ay, byh, byl);
  if constexpr ((K & 3) == 2) return fx_prod(ay, bxh, bxl) - fx_prod(ax, byh, byl);
  return -(fx_prod(ax, bxh, bxl) + fx_prod(ay, byh, byl));
}

// v_e += t_m i^{K+1} v_m and v_m += t_e i^{K+1} v_e from the old values; the
// limbs (p: +t, n: -t) of t_e and t_m carry each element's sign
template <int K>
__device__ __forceinline__ void fx_adj_pair(int64_t (&ve)[2], int64_t (&vm)[2], int32_t tpe, int32_t lpe,
                                            int32_t tne, int32_t lne, int32_t tpm, int32_t lpm, int32_t tnm,
                                            int32_t lnm) {
  constexpr int k1 = (K + 1) & 3;
  const int64_t ex = ve[0], ey = ve[1], mx = vm[0], my = vm[1];
  if constexpr (k1 == 0) {
    ve[0] = ex + fx_prod(mx, tpm, lpm);
    ve[1] = ey + fx_prod(my, tpm, lpm);
    vm[0] = mx + fx_prod(ex, tpe, lpe);
    vm[1] = my + fx_prod(ey, tpe, lpe);
  } else if constexpr (k1 == 1) {  // i v = (-v.y, v.x)
    ve[0] = ex + fx_prod(my, tnm, lnm);
    ve[1] = ey + fx_prod(mx, tpm, lpm);
    vm[0] = mx + fx_prod(ey, tne, lne);
    vm[1] = my + fx_prod(ex, tpe, lpe);
  } else if constexpr (k1 == 2) {  // -v
    ve[0] = ex + fx_prod(mx, tnm, lnm);
    ve[1] = ey + fx_prod(my, tnm, lnm);
    vm[0] = mx + fx_prod(ex, tne, lne);
    vm[1] = my + fx_prod(ey, tne, lne);
  } else {  // -i v = (v.y, -v.x)
    ve[0] = ex + fx_prod(my, tpm, lpm);
    ve[1] = ey + fx_prod(mx, tnm, lnm);
    vm[0] = mx + fx_prod(ey, tpe, lpe);
    vm[1] = my + fx_prod(ex, tne, lne);
  }
}

// One rotation of the run on a coset of phi (P) and lambda (L); returns the
// coset's share of Im<lambda|P_j|phi> in units of 2^(62 - S_phi - S_lambda).
template <int U, int K>
__device__ __forceinline__ int64_t adj_rot_fx(int64_t (&P)[1 << kAdjD][2], int64_t (&L)[1 << kAdjD][2],
                                              const AdjRotFx &r, int sig) {
  constexpr int E = 1 << kAdjD;
  const int32_t th0 = r.th[0], tl0 = r.tl[0], th1 = r.th[1], tl1 = r.tl[1];
  int64_t g = 0;
  if constexpr (U == 0) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      const int neg = (sig ^ (int)(r.zt >> e)) & 1;
      const int32_t tp = neg ? th1 : th0, lp = neg ? tl1 : tl0;  // limbs of t_s
      const int32_t tn = neg ? th0 : th1, ln = neg ? tl0 : tl1;  // limbs of -t_s
      int32_t pxh, pxl, pyh, pyl;
      fx_limbs(P[e][0], pxh, pxl);
      fx_limbs(P[e][1], pyh, pyl);
      const int64_t v = fx_im_conj_ipow<0>(L[e][0], L[e][1], pxh, pxl, pyh, pyl);
      g += neg ? -v : v;
      const int64_t px = P[e][0], py = P[e][1], lx = L[e][0], ly = L[e][1];
      P[e][0] = px + fx_prod(py, tn, ln);
      P[e][1] = py + fx_prod(px, tp, lp);
      L[e][0] = lx + fx_prod(ly, tn, ln);
      L[e][1] = ly + fx_prod(lx, tp, lp);
    }
  } else {
    constexpr int H = adj_high_bit(U);
#pragma unroll
    for (int q = 0; q < E / 2; ++q) {
      const int e = ((q >> H) << (H + 1)) | (q & ((1 << H) - 1));
      const int m = e ^ U;
      const int ne = (sig ^ (int)(r.zt >> e)) & 1, nm = (sig ^ (int)(r.zt >> m)) & 1;
      int32_t exh, exl, eyh, eyl, mxh, mxl, myh, myl;
      fx_limbs(P[e][0], exh, exl);
      fx_limbs(P[e][1], eyh, eyl);
      fx_limbs(P[m][0], mxh, mxl);
      fx_limbs(P[m][1], myh, myl);
      const int64_t ge = fx_im_conj_ipow<K>(L[e][0], L[e][1], mxh, mxl, myh, myl);
      const int64_t gm = fx_im_conj_ipow<K>(L[m][0], L[m][1], exh, exl, eyh, eyl);
      g += (nm ? -ge : ge) + (ne ? -gm : gm);
      const int32_t tpe = ne ? th1 : th0, lpe = ne ? tl1 : tl0, tne = ne ? th0 : th1, lne = ne ? tl0 : tl1;
      const int32_t tpm = nm ? th1 : th0, lpm = nm ? tl1 : tl0, tnm = nm ? th0 : th1, lnm = nm ? tl0 : tl1;
      fx_adj_pair<K>(P[e], P[m], tpe, lpe, tne, lne, tpm, lpm, tnm, lnm);
      fx_adj_pair<K>(L[e], L[m], tpe, lpe, tne, lne, tpm, lpm, tnm, lnm);
    }
  }
  return g;
}

#define PR_ADJ_FX_CASE(UK) \
  case UK: return adj_rot_fx<((UK) >> 2), ((UK)&3)>(P, L, r, sig);

__device__ __forceinline__ int64_t adj_dispatch_fx(int uk, int64_t (&P)[1 << kAdjD][2], int64_t (&L)[1 << kAdjD][2],
                                                   const AdjRotFx &r, int sig) {
  switch (uk) {
    PR_ADJ_FX_CASE(0)
    PR_ADJ_FX_CASE(4) PR_ADJ_FX_CASE(5) PR_ADJ_FX_CASE(6) PR_ADJ_FX_CASE(7)
    PR_ADJ_FX_CASE(8) PR_ADJ_FX_CASE(9) PR_ADJ_FX_CASE(10) PR_ADJ_FX_CASE(11)
    PR_ADJ_FX_CASE(12) PR_ADJ_FX_CASE(13) PR_ADJ_FX_CASE(14) PR_ADJ_FX_CASE(15)
    PR_ADJ_FX_CASE(16) PR_ADJ_FX_CASE(17) PR_ADJ_FX_CASE(18) PR_ADJ_FX_CASE(19)
    PR_ADJ_FX_CASE(20) PR_ADJ_FX_CASE(21) PR_ADJ_FX_CASE(22) PR_ADJ_FX_CASE(23)
    PR_ADJ_FX_CASE(24) PR_ADJ_FX_CASE(25) PR_ADJ_FX_CASE(26) PR_ADJ_FX_CASE(27)
    PR_ADJ_FX_CASE(28) PR_ADJ_FX_CASE(29) PR_ADJ_FX_CASE(30) PR_ADJ_FX_CASE(31)
    default: return 0;
  }
}

// two CTAs per SM (128 registers, a few spilled) measured faster than one
// with 254 registers: 6.86 against 7.04 ms for the n = 20 gradient workload
__global__ void __launch_bounds__(kThreads, 2)
    k_adjoint_run_fx(double2 *__restrict__ phi, double2 *__restrict__ lam, uint64_t n_cosets,
                     const __grid_constant__ AdjRunDev run, int row_stride, double *__restrict__ partials) {
  static_assert(kAdjRun <= 32, "the run's records are set up by one warp");
  constexpr int E = 1 << kAdjD;
  constexpr int kHead = (kAdjD + 2) / 2 + 1;  // as in the rotation pass (coset_fx.cuh)
  __shared__ double sacc[kAdjRun][kThreads];  // one column per thread
  __shared__ AdjRotFx srot[kAdjRun];
  __shared__ int64_t s_bias;
  for (int j = 0; j < kAdjRun; ++j) sacc[j][threadIdx.x] = 0.0;
  const int count = run.count;
  if (threadIdx.x < 32) {
    // limbs of +-T, growth bound ceil(log2(1 + t^2) / 2 * 2^20) + 1, halvings,
    // and the mean correction of the truncated products (3/4 unit per product,
    // halved at later halvings; units of 2^-20 unit)
    const int j = threadIdx.x;
    uint32_t g = 0;
    AdjRotFx rec = {};
    if (j < count) {
      const AdjRotDev r = run.rot[j];
      long long T = __double2ll_rn(r.t * kTwo62);
      T = T > kTMax ? kTMax : (T < -kTMax ? -kTMax : T);
      fx_limbs(T, rec.th[0], rec.tl[0]);
      fx_limbs(-T, rec.th[1], rec.tl[1]);
      rec.z = r.z;
      rec.zt = r.zt;
      rec.uk = r.u * 4 + r.ny;
      const float tf = (float)r.t;
      g = (uint32_t)ceilf(0.5f * __log2f(1.0f + tf * tf) * (float)(1 << kGrowthFrac)) + 1u;
    }
    uint32_t c = g;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
      if (j >= o) c += y;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, c, 31);
    uint32_t corr = 0;
    if (j < count) {
      rec.halve = (int32_t)((c >> kGrowthFrac) - ((c - g) >> kGrowthFrac));
      srot[j] = rec;
      const uint32_t later = (total >> kGrowthFrac) - ((c - g) >> kGrowthFrac);
      corr = later < 31 ? (3u << 18) >> later : 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) corr += __shfl_down_sync(0xffffffffu, corr, o);
    if (j == 0) s_bias = (int64_t)((corr + (1u << 19)) >> 20);
  }
  __syncthreads();
  const int64_t bias = s_bias;
  const double sc = run.scale;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t cs = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; cs < n_cosets; cs += stride) {
    uint64_t rep = cs;
#pragma unroll
    for (int b = 0; b < kAdjD; ++b) {
      const int pv = run.piv[b];
      rep = ((rep >> pv) << (pv + 1)) | (rep & ((1ULL << pv) - 1));
    }
    int64_t P[E][2], L[E][2];
    int Sp, Sl;
    {
      double2 a[E], b[E];
      int ep = 0, el = 0;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        a[e] = phi[rep ^ run.soff[e]];
        b[e] = lam[rep ^ run.soff[e]];
        ep = max(ep, max((int)((__double_as_longlong(a[e].x) >> 52) & 0x7ff),
                         (int)((__double_as_longlong(a[e].y) >> 52) & 0x7ff)));
        el = max(el, max((int)((__double_as_longlong(b[e].x) >> 52) & 0x7ff),
                         (int)((__double_as_longlong(b[e].y) >> 52) & 0x7ff)));
      }
      Sp = 1083 - ep - kHead;
      Sl = 1083 - el - kHead;
#pragma unroll
      for (int e = 0; e < E; ++e) {
        P[e][0] = fx_in(a[e].x, 1085 - Sp);
        P[e][1] = fx_in(a[e].y, 1085 - Sp);
        L[e][0] = fx_in(b[e].x, 1085 - Sl);
        L[e][1] = fx_in(b[e].y, 1085 - Sl);
      }
    }
    int halved = 0;
    for (int j = 0; j < count; ++j) {
      const AdjRotFx &r = srot[j];
      const int sig = __popcll(rep & r.z) & 1;
      const int64_t gi = adj_dispatch_fx(r.uk, P, L, r, sig);
      // gi is in units of 2^-(Sp + Sl - 2 halved - 62)
      sacc[j][threadIdx.x] += fx_out(gi, 1086 - (Sp + Sl - 2 * halved - 62));
      for (int h = r.halve; h > 0; --h) {
        ++halved;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          P[e][0] >>= 1;
          P[e][1] >>= 1;
          L[e][0] >>= 1;
          L[e][1] >>= 1;
        }
      }
    }
    const int ebp = 1086 - (Sp - halved), ebl = 1086 - (Sl - halved);
#pragma unroll
    for (int e = 0; e < E; ++e) {
      phi[rep ^ run.soff[e]] = make_double2(sc * fx_out(P[e][0] + bias, ebp), sc * fx_out(P[e][1] + bias, ebp));
      lam[rep ^ run.soff[e]] = make_double2(sc * fx_out(L[e][0] + bias, ebl), sc * fx_out(L[e][1] + bias, ebl));
    }
  }
  __syncthreads();
  // block sums in a fixed order: warp w reduces rows w, w + 8, ...
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < count; j += (int)(blockDim.x >> 5)) {
    double v = 0.0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += sacc[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partials[(size_t)run.rot[j].row * row_stride + blockIdx.x] = v;
  }
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

template <typename R>
int run_blocks_t(int n) {
  // computed once, on first use (thread-safe static initialisation)
  static const int cap = [] {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_run<R>, kThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    return (per_sm > 0 ? per_sm : 1) * device_sm_count();
  }();
  const uint64_t need = (((1ULL << n) >> kAdjD) + kThreads - 1) / kThreads;
  return (int)(need < (uint64_t)cap ? (need ? need : 1) : cap);
}

int run_blocks_fx(int n) {
  // computed once, on first use (thread-safe static initialisation)
  static const int cap = [] {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_adjoint_run_fx, kThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    return (per_sm > 0 ? per_sm : 1) * device_sm_count();
  }();
  const uint64_t need = (((1ULL << n) >> kAdjD) + kThreads - 1) / kThreads;
  return (int)(need < (uint64_t)cap ? (need ? need : 1) : cap);
}

int run_blocks(const sv_state *sv) { return sv->dtype == SV_C128 ? run_blocks_fx(sv->n) : run_blocks_t<float>(sv->n); }

// The backward sweep as fused runs: rotations in applied order L-1 .. 0, grouped
// greedily into runs of <= kAdjRun whose x-masks span <= kAdjD dimensions.
// Identity strings change only a global phase of both vectors (skipped); their
// gradient rows stay zero.
int adjoint_runs(sv_state *phi, sv_state *lam, const sv_plan *plan, const Pauli &q0, int blocks,
                 std::vector<double> &gscale) {
  const size_t L = plan->order.size();
  PR_CUDA(cudaMemsetAsync(phi->d_partials, 0, sizeof(double) * (size_t)blocks * L, phi->stream));
  const uint64_t n_cosets = (1ULL << phi->n) >> kAdjD;
  size_t i = L;
  while (i > 0) {
    uint64_t basis[kAdjD];
    int piv[kAdjD];
    int d = 0;
    auto reduce = [&](uint64_t v) {
      for (int b = 0; b < d; ++b)
        if ((v >> piv[b]) & 1ULL) v ^= basis[b];
      return v;
    };
    auto add_vec = [&](uint64_t rr) {
      const int pv = 63 - __builtin_clzll(rr);
      for (int b = 0; b < d; ++b)
        if ((basis[b] >> pv) & 1ULL) basis[b] ^= rr;
      int pos = d;
      while (pos > 0 && piv[pos - 1] > pv) {
        basis[pos] = basis[pos - 1];
        piv[pos] = piv[pos - 1];
        --pos;
      }
      basis[pos] = rr;
      piv[pos] = pv;
      ++d;
    };
    // complex128 runs hold rotations with |beta| <= pi/2 only (tan(beta/2) <= 1,
    // which the fixed-point run needs; only rotations of diagonal phase-sum
    // stretches keep larger angles in the plan): a larger one takes a pass of
    // its own in FP64 between runs, with the states at their plain scale
    auto wide = [&](size_t k) {
      return phi->dtype == SV_C128 && plan->sigma[k] != 0 && std::fabs(plan->beta[k]) > kHalfPi;
    };
    if (wide(i - 1)) {
      const size_t k = i - 1;
      const int s0 = anticommute(plan->ox[k], plan->oz[k], q0.x, q0.z) ? -1 : 1;
      const int rc = adjoint_step(phi, lam, plan->ox[k], plan->oz[k], s0 * plan->beta[k],
                                  phi->d_partials + (size_t)blocks * k, blocks);
      if (rc) return rc;
      gscale[k] = 1.0;
      --i;
      continue;
    }
    std::vector<size_t> members;
    while (i > 0 && members.size() < (size_t)kAdjRun) {
      const size_t k = i - 1;
      if (plan->sigma[k] == 0) {
        --i;
        continue;
      }
      if (wide(k)) break;
      const uint64_t rr = reduce(plan->ox[k]);
      if (rr != 0) {
        if (d >= kAdjD) break;
        add_vec(rr);
      }
      members.push_back(k);
      --i;
    }
    if (members.empty()) continue;
    uint64_t usedbits = 0;
    for (int b = 0; b < d; ++b) usedbits |= 1ULL << piv[b];
    for (int bit = phi->n - 1; bit >= 0 && d < kAdjD; --bit)
      if (!((usedbits >> bit) & 1ULL)) {
        add_vec(1ULL << bit);
        usedbits |= 1ULL << bit;
      }
    AdjRunDev run;
    std::memset(&run, 0, sizeof(run));
    for (int e = 0; e < (1 << kAdjD); ++e) {
      uint64_t so = 0;
      for (int b = 0; b < kAdjD; ++b)
        if ((e >> b) & 1) so ^= basis[b];
      run.soff[e] = so;
    }
    for (int b = 0; b < kAdjD; ++b) run.piv[b] = piv[b];
    run.count = (int32_t)members.size();
    double cprod = 1.0;  // cos(beta/2) of the rotations of this run already undone
    for (size_t j = 0; j < members.size(); ++j) {
      const size_t k = members[j];
      const uint64_t x = plan->ox[k], z = plan->oz[k];
      const int s0 = anticommute(x, z, q0.x, q0.z) ? -1 : 1;
      const double beta = s0 * plan->beta[k];
      AdjRotDev &r = run.rot[j];
      r.z = z;
      r.t = std::tan(0.5 * beta);
      gscale[k] = cprod * cprod;  // both vectors carry 1/cprod at this rotation
      cprod *= std::cos(0.5 * beta);
      r.u = 0;
      for (int b = 0; b < kAdjD; ++b)
        if ((x >> piv[b]) & 1ULL) r.u |= 1 << b;
      r.ny = popc64(x & z) & 3;
      r.zt = 0;
      for (int e = 0; e < (1 << kAdjD); ++e) r.zt |= (uint32_t)(popc64(run.soff[e] & z) & 1) << e;
      r.row = (int32_t)k;
    }
    run.scale = cprod;
    const int tr = trace_begin(phi, KN_ADJOINT_RUN);
    if (phi->dtype == SV_C128)
      k_adjoint_run_fx<<<blocks, kThreads, 0, phi->stream>>>((double2 *)phi->amps, (double2 *)lam->amps, n_cosets,
                                                             run, blocks, phi->d_partials);
    else
      k_adjoint_run<float><<<blocks, kThreads, 0, phi->stream>>>((float2 *)phi->amps, (float2 *)lam->amps,
                                                                 n_cosets, run, blocks, phi->d_partials);
    PR_CHECK_LAUNCH();
    trace_end(phi, tr, KN_ADJOINT_RUN, 4.0 * (double)amp_bytes(phi->dtype) * (double)(1ULL << phi->n));
  }
  return SV_OK;
}

}  // namespace

int adjoint_step(sv_state *phi, sv_state *lam, uint64_t x, uint64_t z, double beta, double *d_out,
                 int max_blocks) {
  int blocks = step_blocks(phi->n);
  if (max_blocks > 0 && blocks > max_blocks) blocks = max_blocks;
  const double c = std::cos(0.5 * beta), s = std::sin(0.5 * beta);
  const uint64_t n_amps = 1ULL << phi->n;
  const int tr = trace_begin(phi, KN_ADJOINT);
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
  // phi and lambda live on psi0 between calls (allocated once per size and type)
  for (sv_state *&w : psi0->work)
    if (!rc && (!w || w->n != psi0->n || w->dtype != psi0->dtype)) {
      sv_free(w);
      w = nullptr;
      rc = sv_alloc(&w, psi0->n, psi0->dtype, psi0->stream);
    }
  sv_state *phi = psi0->work[0], *lam = psi0->work[1];
  if (!rc) {
    phi->stream = lam->stream = psi0->stream;
    phi->trace_owner = lam->trace_owner = psi0;  // a trace of psi0 shows the sweep's kernels
  }
  const Pauli q0 = psi0->frame;
  if (!rc) rc = sv_copy(phi, psi0);
  if (!rc) rc = apply_plan(phi, plan);
  double energy = 0.0;
  if (!rc) rc = expval_impl(phi, hx, hz, hc, n_terms, &energy, nullptr);
  if (!rc) rc = pauli_sum_impl(lam, phi, hx, hz, hc, n_terms);
  const size_t L = plan ? plan->order.size() : 0;
  // fused backward runs (a coset of kAdjD dimensions per thread); states with
  // fewer qubits take one pass per rotation
  const bool fused = psi0->n >= kAdjD;
  const int blocks = fused ? run_blocks(psi0) : step_blocks(psi0->n);
  if (!rc) rc = ensure_scratch(phi, (size_t)blocks * (L ? L : 1), L ? L : 1);
  std::vector<double> gscale(L, 1.0);
  if (!rc && fused && L) rc = adjoint_runs(phi, lam, plan, q0, blocks, gscale);
  if (!rc && !fused) {
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
      out_grads[plan->order[i]] = (double)(s0 * plan->sigma[i]) * gscale[i] * phi->h_results[i];
    }
    if (out_energy) *out_energy = energy;
  }
  plan_free(plan);
  return rc;
}

}  // extern "C"
