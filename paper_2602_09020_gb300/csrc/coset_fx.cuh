// Complex128 fused coset pass in 64-bit fixed point on the integer pipes.
//
// The pass applies the same tan-form pair update as body_coset (paper, App.
// "Amplitude update rule for multi-qubit rotations": the 2x2 update of a pair
// (k, k ^ x); here a_k += t * kappa * (-1)^{popc(k&z)} * a_{k^x} with the
// positive factor cos(theta/2) left to the plan's running scale), but it does
// the arithmetic on the integer pipes instead of GB300's narrow FP64 pipe.
//
// Representation.  A thread owns one coset of the run's x-span (2^D complex
// elements, closed under every pairing of the run).  On load every component
// becomes a signed integer A = round(a * 2^S) with one exponent S per coset:
// block floating point, S chosen from the largest exponent in the coset so
// that every component stays below 2^61 for the whole run.  That bound holds
// because the tan-form step I - i t P multiplies the coset's 2-norm by exactly
// sqrt(1 + t^2) (P restricted to the coset is a Hermitian involution), and a
// component never exceeds the coset's 2-norm: the norm grows by a known
// amount, and whenever the running growth passes a whole bit every component
// is halved (S decreases by one), so between halvings the growth stays below
// one bit of headroom.
//
// Products.  t is held as T = round(t * 2^62) (|t| < 1 after the planner's
// angle reduction, T clamped to |T| < 2^62) split as T = th * 2^31 + tl with
// 0 <= tl < 2^31, and likewise A = ah * 2^31 + al; then
//   A T / 2^62 = ah th + (ah tl + al th) / 2^31 + al tl / 2^62,
// three 32 x 32 -> 64-bit integer multiplies (fx_prod).  The last term (in
// [0, 1)) is dropped and the shift floors, so a product is low by less than 2
// units of 2^-S, by 3/4 of a unit on average; every update adds a product (a
// subtraction adds the product with -T), so the run adds that mean back to every
// component once, at the end.  Per coset the resolution is 2^-58 of the largest
// component or finer, which is finer than the 2^-53 relative rounding of the
// FP64 value the pass stores.
//
// Conversions use the IEEE-754 binary64 layout directly (sign, 11-bit biased
// exponent, 52-bit fraction with an implicit leading one), so no conversion
// instruction runs on the FP64 pipe: values below 2^-1022 in magnitude
// (subnormals) are read as zero and results below it are written as zero.
#pragma once

#include "fixed64.cuh"
#include "kernels.cuh"

namespace pr {

namespace {

template <typename Idx>
struct RotFx {
  Idx z;
  uint32_t zt;
  uint32_t code;
  int32_t th[2];  // high limbs of +T and -T
  int32_t tl[2];  // low limbs of +T and -T, in [0, 2^31)
  int32_t halve;  // 1: halve every component after this rotation
};

// Apply one rotation with coset coordinates U (compile-time) to V cosets;
// sg[v] is the sign bit (-1)^{popc(rep_v & z)}, bit l of zt the element's.
// (th0, tl0) are the limbs of +T, (th1, tl1) those of -T.  Every update is an
// addition of a truncated product (a subtraction adds the product with -T), so
// every product is low by the same 3/4 unit on average (see fx_prod).
template <int D, int V, int U, int IMAG>
__device__ __forceinline__ void apply_fx(int64_t (&re)[V][1 << D], int64_t (&im)[V][1 << D], const int (&sg)[V],
                                         uint32_t zt, int32_t th0, int32_t tl0, int32_t th1, int32_t tl1) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
#pragma unroll
    for (int l = 0; l < (1 << D); ++l) {
      const int s = sg[v] ^ (int)((zt >> l) & 1u);
      // limbs of +-T for the element's sign s, and of the opposite sign
      const int32_t tp = s ? th1 : th0, lp = s ? tl1 : tl0;
      const int32_t tn = s ? th0 : th1, ln = s ? tl0 : tl1;
      if (U == 0) {
        const int64_t r = re[v][l], i = im[v][l];
        re[v][l] = r + fx_prod(i, tn, ln);
        im[v][l] = i + fx_prod(r, tp, lp);
      } else if ((l ^ U) > l) {
        const int m = l ^ U;
        const int64_t rl = re[v][l], il = im[v][l], rm = re[v][m], iv = im[v][m];
        if (IMAG) {
          re[v][l] = rl + fx_prod(iv, tn, ln);
          im[v][l] = il + fx_prod(rm, tp, lp);
          re[v][m] = rm + fx_prod(il, tn, ln);
          im[v][m] = iv + fx_prod(rl, tp, lp);
        } else {
          re[v][l] = rl + fx_prod(rm, tp, lp);
          im[v][l] = il + fx_prod(iv, tp, lp);
          re[v][m] = rm + fx_prod(rl, tn, ln);
          im[v][m] = iv + fx_prod(il, tn, ln);
        }
      }
    }
  }
}

#define PR_CASE_FX(K)                                                                      \
  case K:                                                                                  \
    if constexpr ((((K) >> 1) < (1 << D)) && ((((K) >> 1) != 0) || ((K)&1)))               \
      apply_fx<D, V, ((K) >> 1), ((K)&1)>(re, im, sg, zt, th0, tl0, th1, tl1);             \
    break;
#define PR_CASE_FX8(B)                                                                                       \
  PR_CASE_FX(B + 0) PR_CASE_FX(B + 1) PR_CASE_FX(B + 2) PR_CASE_FX(B + 3) PR_CASE_FX(B + 4) PR_CASE_FX(B + 5) \
  PR_CASE_FX(B + 6) PR_CASE_FX(B + 7)

template <int D, int V>
__device__ __forceinline__ void dispatch_fx(uint32_t code, int64_t (&re)[V][1 << D], int64_t (&im)[V][1 << D],
                                            const int (&sg)[V], uint32_t zt, int32_t th0, int32_t tl0, int32_t th1,
                                            int32_t tl1) {
  switch (code) {
    PR_CASE_FX8(0)
    PR_CASE_FX8(8)
    PR_CASE_FX8(16)
    PR_CASE_FX8(24)
    PR_CASE_FX8(32)
    PR_CASE_FX8(40)
    PR_CASE_FX8(48)
    PR_CASE_FX8(56)
    default:
      break;
  }
}

template <typename Idx, int D>
__host__ __device__ constexpr size_t ws_coset_fx() {
  return ((sizeof(RotFx<Idx>) * kMaxRunRots + sizeof(Idx) * (1u << D) + 15) & ~size_t(15)) +
         2 * sizeof(uint32_t) * (kThreads / 32);
}

// One CTA's share of a fused complex128 run in fixed point.  The run must hold
// at most kThreads rotations (kMaxRunRots == kThreads).  ws: ws_coset_fx bytes.
template <typename Idx, int D, int V>
__device__ __forceinline__ void body_coset_fx(double2 *__restrict__ amp, Idx n_cosets, const RunDev &run,
                                              const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz,
                                              Idx cta_rank, Idx cta_count, char *ws) {
  static_assert(kMaxRunRots <= kThreads, "one rotation record per thread");
  constexpr int E = 1 << D;
  RotFx<Idx> *srot = (RotFx<Idx> *)ws;
  Idx *soff = (Idx *)(ws + sizeof(RotFx<Idx>) * kMaxRunRots);
  uint32_t *swarp = (uint32_t *)(ws + ((sizeof(RotFx<Idx>) * kMaxRunRots + sizeof(Idx) * E + 15) & ~size_t(15)));
  const int count = run.count;
  const int j = threadIdx.x;
  const int lane = j & 31, warp = j >> 5;

  // records: limbs of +-T and the growth bound of each rotation,
  // ceil(log2(1 + t^2) / 2 * 2^20) + 1 (a slight over-estimate)
  uint32_t g = 0;
  RotFx<Idx> rec;
  if (j < count) {
    const RotDev r = rots[run.first + j];
    double t = r.t;
    if (__popcll((r.x & fz) ^ (r.z & fx)) & 1) t = -t;  // runtime frame sign
    long long T = __double2ll_rn(t * kTwo62);
    T = T > kTMax ? kTMax : (T < -kTMax ? -kTMax : T);
    fx_limbs(T, rec.th[0], rec.tl[0]);
    fx_limbs(-T, rec.th[1], rec.tl[1]);
    rec.z = (Idx)r.z;
    rec.zt = r.zt;
    rec.code = r.code & kCodeMask;
    const float tf = (float)t;
    g = (uint32_t)ceilf(0.5f * __log2f(1.0f + tf * tf) * (float)(1 << kGrowthFrac)) + 1u;
  }
  // inclusive prefix sum of g over the run (block scan)
  uint32_t c = g;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, c, o);
    if (lane >= o) c += y;
  }
  if (lane == 31) swarp[warp] = c;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < warp; ++w) base += swarp[w];
  c += base;
  uint32_t total = 0;  // growth over the whole run
  for (int w = 0; w < kThreads / 32; ++w) total += swarp[w];
  // mean correction of the truncated products (fx_prod): 3/4 of a unit per
  // product, one product per component and rotation; what a rotation adds is
  // halved with the components at every later halving.  Units of 2^-20 unit.
  uint32_t corr = 0;
  if (j < count) {
    rec.halve = (int32_t)((c >> kGrowthFrac) - ((c - g) >> kGrowthFrac));
    srot[j] = rec;
    // halvings at this rotation (after its products) and at later ones
    const uint32_t later = (total >> kGrowthFrac) - ((c - g) >> kGrowthFrac);
    corr = later < 31 ? (3u << 18) >> later : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) corr += __shfl_down_sync(0xffffffffu, corr, o);
  if (lane == 0) swarp[kThreads / 32 + warp] = corr;
  if (threadIdx.x < E) {
    uint64_t s = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) s ^= run.basis[b];
    soff[threadIdx.x] = (Idx)s;
  }
  __syncthreads();
  uint32_t corr_sum = 0;
  for (int w = 0; w < kThreads / 32; ++w) corr_sum += swarp[kThreads / 32 + w];
  const int64_t bias = (int64_t)((corr_sum + (1u << 19)) >> 20);  // units added to every component

  // headroom: the coset's 2-norm is at most 2^((D+1)/2) times its largest
  // component, and the growth between halvings stays below one bit
  constexpr int kHead = (D + 2) / 2 + 1;
  const Idx chunk = (Idx)blockDim.x * V;
  const Idx stride = cta_count * chunk;
  for (Idx c0 = cta_rank * chunk + threadIdx.x; c0 < n_cosets; c0 += stride) {
    int64_t re[V][E], im[V][E];
    Idx rep[V];
    bool ok[V];
    int S[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const Idx cc = c0 + (Idx)(v * blockDim.x);
      Idx r = cc;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int p = run.piv[b];
        r = ((r >> p) << (p + 1)) | (r & ((Idx(1) << p) - 1));
      }
      rep[v] = r;
      ok[v] = cc < n_cosets;
      double2 a[E];
      int emax = 0;
#pragma unroll
      for (int l = 0; l < E; ++l) {
        a[l] = ok[v] ? amp[r ^ soff[l]] : make_double2(0.0, 0.0);
        const int ex = (int)((__double_as_longlong(a[l].x) >> 52) & 0x7ff);
        const int ey = (int)((__double_as_longlong(a[l].y) >> 52) & 0x7ff);
        emax = max(emax, max(ex, ey));
      }
      // |a| < 2^(emax - 1022); S = 61 - (emax - 1022) - kHead keeps |A| < 2^61
      S[v] = 1083 - emax - kHead;
      const int kbase = 1085 - S[v];
#pragma unroll
      for (int l = 0; l < E; ++l) {
        re[v][l] = fx_in(a[l].x, kbase);
        im[v][l] = fx_in(a[l].y, kbase);
      }
    }
    int halved = 0;
    for (int jj = 0; jj < count; ++jj) {
      const RotFx<Idx> s = srot[jj];
      int sg[V];
#pragma unroll
      for (int v = 0; v < V; ++v) sg[v] = parity(rep[v] & s.z);
      dispatch_fx<D, V>(s.code, re, im, sg, s.zt, s.th[0], s.tl[0], s.th[1], s.tl[1]);
      // written as a loop (trip count 0 or 1) so that the rare halving stays a
      // branch instead of being computed and selected after every rotation
      for (int h = s.halve; h > 0; --h) {
        ++halved;
#pragma unroll
        for (int v = 0; v < V; ++v)
#pragma unroll
          for (int l = 0; l < E; ++l) {
            re[v][l] >>= 1;
            im[v][l] >>= 1;
          }
      }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
#pragma unroll
      for (int l = 0; l < E; ++l) {
        re[v][l] += bias;
        im[v][l] += bias;
      }
    // the fold (a complex factor, last pass of a plan) in FP64 after the
    // conversion; two separate store loops keep the FP64 multiplies out of the
    // passes without a fold
    if (run.fold) {
      const double fr = run.fold_re, fi = run.fold_im;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ebase = 1086 - (S[v] - halved);
#pragma unroll
        for (int l = 0; l < E; ++l) {
          const double x = fx_out(re[v][l], ebase), y = fx_out(im[v][l], ebase);
          if (ok[v]) amp[rep[v] ^ soff[l]] = make_double2(fr * x - fi * y, fr * y + fi * x);
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int ebase = 1086 - (S[v] - halved);
#pragma unroll
        for (int l = 0; l < E; ++l)
          if (ok[v]) amp[rep[v] ^ soff[l]] = make_double2(fx_out(re[v][l], ebase), fx_out(im[v][l], ebase));
      }
    }
  }
  __syncthreads();  // the workspace may be reused by the caller's next pass
}

}  // namespace

}  // namespace pr
