// FP64 reductions over the statevector.
//
// <psi|sum_j c_j P_j|psi> (paper, Sec. "Extraction of Expectation Values",
// Eq. chfsexp) with |psi> = Q|phi>: every term is first rewritten by the Pauli
// frame (Q^dag P Q = (-1)^{<P,Q>} P, Eq. Fmap for a Pauli-only frame), then
// terms are grouped by x-mask.  For a group with x != 0 each pair (k, k^x)
// contributes
//     sum_j c_j i^{nY_j} [ s_j(k^x) w + s_j(k) conj(w) ],  w = conj(a_k) a_{k^x},
// which is 2 c_j s_j(k) times Re w, Im w, -Re w or -Im w for nY = 0, 1, 2, 3
// (mod 4), s_j(k) = (-1)^{popc(k & z_j)}.  The x = 0 group contributes
// sum_k |a_k|^2 sum_j c_j s_j(k).  Groups whose x-masks span a subspace of
// dimension <= kExpD are evaluated in one read pass over cosets of that span,
// as in the fused rotation pass.  Amplitudes are widened to FP64 before any
// product; every sum is FP64; block partials are reduced in a fixed order, so
// results are bitwise reproducible.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <cmath>

#include "fixed64.cuh"
#include "internal.h"

namespace pr {

namespace {

constexpr int kExpD = 4;
constexpr int kExpMaxTerms = 1024;
constexpr int kExpMaxGroups = 1 << kExpD;
constexpr int kPsumD = 3;  // coset dimension of the H psi runs

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

__device__ __forceinline__ int parity(uint32_t v) { return __popc(v) & 1; }
__device__ __forceinline__ int parity(uint64_t v) { return __popcll(v) & 1; }

struct ExpTermSm {
  uint64_t z;
  double coef;
  uint32_t zt;
  uint32_t imag;
};

__host__ __device__ constexpr int adj_high_bit_e(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return h;
}

// in-place transform w^[i] = sum_p (-1)^{popc(p & i)} w[p]
template <int N>
__device__ __forceinline__ void wht_f64(double (&w)[N]) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1)
#pragma unroll
    for (int i = 0; i < N; ++i)
      if (!(i & h)) {
        const double x = w[i], y = w[i | h];
        w[i] = x + y;
        w[i | h] = x - y;
      }
}

// w[i] for a runtime i, as a select over registers (integer work)
template <int N>
__device__ __forceinline__ double pick_f64(const double (&w)[N], int i) {
  double r = w[0];
#pragma unroll
  for (int q = 1; q < N; ++q)
    if (q == i) r = w[q];
  return r;
}

// One x-mask group of a <H> run on a coset: acc += sum_j c_j sum_l s_j(l) w_l.
// Term j's sign at element l is (-1)^{s0_j + zt_j(l)} with zt_j(l) linear in
// the bits of l (zeta_j: the bits b with zt_j(2^b) = 1), so sum_l (-1)^{zt_j(l)}
// w_l is entry zeta_j of the Walsh-Hadamard transform of w.  Groups of enough
// terms take the transform once per coset and then one multiply-add per term
// (GB300's FP64 pipe is narrow; the index arithmetic and the select are
// integer work); small groups sum directly.  parts: bit 0 = some term reads
// the real part of conj(a_l) a_m, bit 1 = the imaginary part (0: both).
template <int D, int U, typename Idx>
__device__ __forceinline__ void group_terms(const double2 (&a)[1 << D], Idx rep, const ExpTermSm *terms,
                                            int first, int count, int parts, double &acc) {
  constexpr int E = 1 << D;
  if (U == 0) {
    double p[E];
#pragma unroll
    for (int l = 0; l < E; ++l) p[l] = a[l].x * a[l].x + a[l].y * a[l].y;
    if (count >= 5) {
      wht_f64<E>(p);
      for (int j = first; j < first + count; ++j) {
        const ExpTermSm t = terms[j];
        int zeta = 0;
#pragma unroll
        for (int b = 0; b < D; ++b) zeta |= (int)((t.zt >> (1u << b)) & 1u) << b;
        const double c = parity((uint64_t)rep & t.z) ? -t.coef : t.coef;
        acc = fma(c, pick_f64<E>(p, zeta), acc);
      }
      return;
    }
    for (int j = first; j < first + count; ++j) {
      const ExpTermSm t = terms[j];
      const uint32_t s0 = (uint32_t)parity((uint64_t)rep & t.z);
#pragma unroll
      for (int l = 0; l < E; ++l) {
        const double c = ((s0 ^ (t.zt >> l)) & 1u) ? -t.coef : t.coef;
        acc = fma(c, p[l], acc);
      }
    }
  } else {
    constexpr int H = adj_high_bit_e(U), P = E / 2;
    if (count >= 4) {
      // pair values of the leaders l (bit H clear), indexed by l's other bits
      const bool want_re = parts != 2, want_im = parts != 1;
      double wr[P], wi[P];
#pragma unroll
      for (int q = 0; q < P; ++q) {
        const int l = ((q >> H) << (H + 1)) | (q & ((1 << H) - 1));
        const double2 al = a[l], am = a[l ^ U];
        wr[q] = want_re ? al.x * am.x + al.y * am.y : 0.0;
        wi[q] = want_im ? al.x * am.y - al.y * am.x : 0.0;
      }
      if (want_re) wht_f64<P>(wr);
      if (want_im) wht_f64<P>(wi);
      for (int j = first; j < first + count; ++j) {
        const ExpTermSm t = terms[j];
        int zeta = 0;
#pragma unroll
        for (int k = 0; k < D - 1; ++k) {
          const int b = k < H ? k : k + 1;
          zeta |= (int)((t.zt >> (1u << b)) & 1u) << k;
        }
        const double c = parity((uint64_t)rep & t.z) ? -t.coef : t.coef;
        acc = fma(c, t.imag ? pick_f64<P>(wi, zeta) : pick_f64<P>(wr, zeta), acc);
      }
      return;
    }
    double wr[E], wi[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
      if ((l ^ U) > l) {
        const double2 al = a[l], am = a[l ^ U];
        wr[l] = al.x * am.x + al.y * am.y;
        wi[l] = al.x * am.y - al.y * am.x;
      } else {
        wr[l] = 0.0;
        wi[l] = 0.0;
      }
    }
    for (int j = first; j < first + count; ++j) {
      const ExpTermSm t = terms[j];
      const uint32_t s0 = (uint32_t)parity((uint64_t)rep & t.z);
      if (t.imag) {
#pragma unroll
        for (int l = 0; l < E; ++l)
          if ((l ^ U) > l) {
            const double c = ((s0 ^ (t.zt >> l)) & 1u) ? -t.coef : t.coef;
            acc = fma(c, wi[l], acc);
          }
      } else {
#pragma unroll
        for (int l = 0; l < E; ++l)
          if ((l ^ U) > l) {
            const double c = ((s0 ^ (t.zt >> l)) & 1u) ? -t.coef : t.coef;
            acc = fma(c, wr[l], acc);
          }
      }
    }
  }
}

#define PR_GCASE(K) \
  case K:           \
    if constexpr ((K) < (1 << D)) group_terms<D, (K)>(a, rep, terms, first, count, parts, acc); \
    break;

template <int D, typename Idx>
__device__ __forceinline__ void group_dispatch(int u, const double2 (&a)[1 << D], Idx rep, const ExpTermSm *terms,
                                               int first, int count, int parts, double &acc) {
  switch (u) {
    PR_GCASE(0) PR_GCASE(1) PR_GCASE(2) PR_GCASE(3) PR_GCASE(4) PR_GCASE(5) PR_GCASE(6) PR_GCASE(7)
    PR_GCASE(8) PR_GCASE(9) PR_GCASE(10) PR_GCASE(11) PR_GCASE(12) PR_GCASE(13) PR_GCASE(14) PR_GCASE(15)
    default: break;
  }
}

// block sum of two doubles in a fixed order; thread 0 gets the result
__device__ __forceinline__ void block_sum2(double &a, double &b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ra = 0.0, rb = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      ra += sa[i];
      rb += sb[i];
    }
    a = ra;
    b = rb;
  }
}

template <typename R, typename Idx, int D>
__global__ void __launch_bounds__(kThreads)
    k_expval(const typename Cx<R>::T *__restrict__ amp, Idx n_cosets, const ExpRunDev run,
             const ExpGroupDev *__restrict__ groups, const ExpTermDev *__restrict__ gterms,
             double *__restrict__ partials) {
  constexpr int E = 1 << D;
  __shared__ ExpTermSm terms[kExpMaxTerms];
  __shared__ ExpGroupDev sg[kExpMaxGroups];
  __shared__ Idx soff[E];
  int n_terms = 0;
  for (int g = 0; g < run.n_groups; ++g) n_terms = max(n_terms, groups[g].first + groups[g].count);
  for (int j = threadIdx.x; j < n_terms; j += blockDim.x) {
    const ExpTermDev t = gterms[j];
    terms[j] = ExpTermSm{t.z, t.coef, t.zt, t.imag};
  }
  if (threadIdx.x < run.n_groups) sg[threadIdx.x] = groups[threadIdx.x];
  if (threadIdx.x < E) {
    uint64_t s = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) s ^= run.basis[b];
    soff[threadIdx.x] = (Idx)s;
  }
  __syncthreads();
  double acc = 0.0, nrm = 0.0;
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx c = (Idx)blockIdx.x * blockDim.x + threadIdx.x; c < n_cosets; c += stride) {
    Idx rep = c;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const int p = run.piv[b];
      rep = ((rep >> p) << (p + 1)) | (rep & ((Idx(1) << p) - 1));
    }
    double2 a[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
      const typename Cx<R>::T v = amp[rep ^ soff[l]];
      a[l].x = (double)v.x;
      a[l].y = (double)v.y;
    }
    if (run.with_norm) {
#pragma unroll
      for (int l = 0; l < E; ++l) nrm = fma(a[l].x, a[l].x, fma(a[l].y, a[l].y, nrm));
    }
    for (int g = 0; g < run.n_groups; ++g) {
      const ExpGroupDev G = sg[g];
      // the products depend on the coset only; without this the compiler
      // hoists every case's products out of the group loop at once
#pragma unroll
      for (int l = 0; l < E; ++l) asm volatile("" : "+d"(a[l].x), "+d"(a[l].y));
      group_dispatch<D>(G.u, a, rep, terms, G.first, G.count, G.pad, acc);
    }
  }
  block_sum2(acc, nrm);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = acc;
    partials[2 * blockIdx.x + 1] = nrm;
  }
}

// result[2 r + i] = sum over blocks of partials[r][b][i], fixed order
__global__ void k_finish(const double *__restrict__ partials, int n_blocks, double *__restrict__ result) {
  const double *p = partials + (size_t)blockIdx.x * 2 * n_blocks;
  double a = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n_blocks; i += blockDim.x) {
    a += p[2 * i];
    b += p[2 * i + 1];
  }
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    result[2 * blockIdx.x] = a;
    result[2 * blockIdx.x + 1] = b;
  }
}

// q 2^-K as binary64 rounded to nearest even, on the integer pipes (|q| < 2^63;
// 2^-K and the result normal numbers): the value of (double)q * 2^-K without
// the conversion and the multiply, which both occupy GB300's narrow FP64 pipe
__device__ __forceinline__ double i64_ldexp(long long q, int K) {
  const uint64_t sgn = (uint64_t)q & 0x8000000000000000ULL;
  const uint64_t v = q < 0 ? (uint64_t)(-q) : (uint64_t)q;
  const int lz = __clzll((long long)v);
  const uint64_t nv = v << (lz & 63);
  uint64_t m = nv >> 11;
  const uint64_t rest = nv & 0x7ffULL;
  m += (rest > 0x400ULL || (rest == 0x400ULL && (m & 1ULL))) ? 1ULL : 0ULL;
  int e = 63 - lz - K;
  const uint64_t carry = m >> 53;
  m >>= carry;
  e += (int)carry;
  const uint64_t bits = sgn | ((uint64_t)(e + 1023) << 52) | (m & 0xfffffffffffffULL);
  return v == 0 ? 0.0 : __longlong_as_double((long long)bits);
}

// dst += sum_g sum_{j in g} c_j i^{nY_j} s_j(k^x) src_{k^x}   (per element k)
// One group of an H psi run on a coset: o_l += C(m) a_m with m = l ^ U and
// C(m) = sum_j c_j i^{nY_j} s_j(k_m).  With k_m = rep ^ off_m the sign splits as
// s_j(rep) (-1)^{sigma_j . m}, sigma_j,b = parity(z_j & basis_b), so C is the
// Walsh-Hadamard transform over m of W[sigma] = sum over the group's terms with
// that sigma of c_j i^{nY_j} s_j(rep): one signed add per term and coset, then
// one transform per coset (real and imaginary parts apart), exact in 64-bit
// fixed point (each c_j held as round(c_j 2^K), K from the run's sum of
// |c_j|, so no partial sum or transform entry exceeds 2^62), and one
// conversion per element and group.  Amplitudes are widened and coefficients
// converted by integer work (widen_f64, i64_ldexp); the FP64 pipe does only the
// complex multiply-adds.
struct PsTermSm {
  uint64_t z;
  long long q;    // round(c_j 2^K), negated for nY = 2, 3 (mod 4)
  uint32_t code;  // sigma_j | (nY odd) << D
  uint32_t pad;
};

template <int N>
__device__ __forceinline__ void psum_wht(long long *W) {
#pragma unroll
  for (int h = 1; h < N; h <<= 1) {
#pragma unroll
    for (int p = 0; p < N; ++p)
      if (!(p & h)) {
        const long long a = W[p], b = W[p | h];
        W[p] = a + b;
        W[p | h] = a - b;
      }
  }
}

#define PR_PSUM_W(K) \
  case K:            \
    if constexpr ((K) < 2 * E) W[K] += q; \
    break;

template <int U, int E, typename Idx>
__device__ __forceinline__ void psum_group(const double2 (&a)[E], double2 (&o)[E], const ExpGroupDev &G,
                                           const PsTermSm *terms, Idx rep, int qk) {
  long long W[2 * E];
#pragma unroll
  for (int k = 0; k < 2 * E; ++k) W[k] = 0;
  for (int j = G.first; j < G.first + G.count; ++j) {
    const PsTermSm t = terms[j];
    const long long q = parity((uint64_t)rep & t.z) ? -t.q : t.q;
    switch (t.code) {
      PR_PSUM_W(0) PR_PSUM_W(1) PR_PSUM_W(2) PR_PSUM_W(3) PR_PSUM_W(4) PR_PSUM_W(5) PR_PSUM_W(6) PR_PSUM_W(7)
      PR_PSUM_W(8) PR_PSUM_W(9) PR_PSUM_W(10) PR_PSUM_W(11) PR_PSUM_W(12) PR_PSUM_W(13) PR_PSUM_W(14)
      PR_PSUM_W(15)
      default: break;
    }
  }
  // groups whose strings all have even (odd) nY have a real (imaginary)
  // coefficient: one transform and half the FP64 multiply-adds
  if (G.pad != 2) psum_wht<E>(W);
  if (G.pad != 1) psum_wht<E>(W + E);
#pragma unroll
  for (int l = 0; l < E; ++l) {
    constexpr int UU = U;
    const int m = l ^ UU;
    const double2 am = a[m];
    if (G.pad == 1) {
      const double cr = i64_ldexp(W[m], qk);
      o[l].x = fma(cr, am.x, o[l].x);
      o[l].y = fma(cr, am.y, o[l].y);
    } else if (G.pad == 2) {
      const double ci = i64_ldexp(W[E + m], qk);
      o[l].x = fma(-ci, am.y, o[l].x);
      o[l].y = fma(ci, am.x, o[l].y);
    } else {
      const double cr = i64_ldexp(W[m], qk), ci = i64_ldexp(W[E + m], qk);
      o[l].x = fma(cr, am.x, fma(-ci, am.y, o[l].x));
      o[l].y = fma(cr, am.y, fma(ci, am.x, o[l].y));
    }
  }
}

#define PR_PSUM_CASE(K)                                                  \
  case K:                                                                \
    if constexpr ((K) < E) psum_group<(K), E, Idx>(a, o, G, terms, rep, qk); \
    break;

template <typename R, typename Idx, int D>
__global__ void __launch_bounds__(kThreads)
    k_pauli_sum(typename Cx<R>::T *__restrict__ dst, const typename Cx<R>::T *__restrict__ src, Idx n_cosets,
                const ExpRunDev run, const ExpGroupDev *__restrict__ groups,
                const ExpTermDev *__restrict__ gterms) {
  static_assert(D <= kPsumD, "H psi cosets have at most 2^kPsumD elements");
  using C = typename Cx<R>::T;
  constexpr int E = 1 << D;
  __shared__ PsTermSm terms[kExpMaxTerms];
  __shared__ ExpGroupDev sg[kExpMaxGroups];
  __shared__ Idx soff[E];
  int n_terms = 0;
  for (int g = 0; g < run.n_groups; ++g) n_terms = max(n_terms, groups[g].first + groups[g].count);
  for (int j = threadIdx.x; j < n_terms; j += blockDim.x) {
    const ExpTermDev t = gterms[j];
    uint32_t sigma = 0;
    for (int b = 0; b < D; ++b) sigma |= ((t.zt >> (1u << b)) & 1u) << b;
    const long long q = __double_as_longlong(t.coef);
    terms[j] = PsTermSm{t.z, (t.imag & 2u) ? -q : q, sigma | ((t.imag & 1u) << D), 0u};
  }
  if (threadIdx.x < run.n_groups) sg[threadIdx.x] = groups[threadIdx.x];
  if (threadIdx.x < E) {
    uint64_t s = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) s ^= run.basis[b];
    soff[threadIdx.x] = (Idx)s;
  }
  __syncthreads();
  const int qk = 1023 - (int)((__double_as_longlong(run.qscale) >> 52) & 0x7ff);  // qscale = 2^-qk
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx c = (Idx)blockIdx.x * blockDim.x + threadIdx.x; c < n_cosets; c += stride) {
    Idx rep = c;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const int p = run.piv[b];
      rep = ((rep >> p) << (p + 1)) | (rep & ((Idx(1) << p) - 1));
    }
    double2 a[E], o[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
      const C v = src[rep ^ soff[l]];
      a[l].x = widen_f64(v.x);
      a[l].y = widen_f64(v.y);
      const C w = dst[rep ^ soff[l]];
      o[l].x = widen_f64(w.x);
      o[l].y = widen_f64(w.y);
    }
    for (int g = 0; g < run.n_groups; ++g) {
      const ExpGroupDev G = sg[g];
      // the pairing pattern as a compile-time case: every partner a[l ^ u] is
      // then a register, not a select over the coset
      switch (G.u) {
        PR_PSUM_CASE(0) PR_PSUM_CASE(1) PR_PSUM_CASE(2) PR_PSUM_CASE(3)
        PR_PSUM_CASE(4) PR_PSUM_CASE(5) PR_PSUM_CASE(6) PR_PSUM_CASE(7)
        default: break;
      }
    }
#pragma unroll
    for (int l = 0; l < E; ++l) {
      C w;
      w.x = (R)o[l].x;
      w.y = (R)o[l].y;
      dst[rep ^ soff[l]] = w;
    }
  }
}

// ------------------------------------------------------------------ host planning

struct HostExpRun {
  ExpRunDev dev;
  std::vector<ExpGroupDev> groups;
  std::vector<ExpTermDev> terms;
};

struct Term {
  uint64_t x, z;
  double c;
};

// group terms by x (frame signs applied), then pack groups greedily into runs
// whose x-masks span at most kExpD dimensions.  mode 0: expectation
// coefficients (2 c s(nY) per pair, c per element on x = 0; imag = nY odd);
// mode 1: Pauli-sum application (c with imag = nY mod 4).
void plan_groups(const sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
                 int mode, std::vector<HostExpRun> &runs) {
  const Pauli &q = sv->frame;
  std::map<uint64_t, std::vector<Term>> by_x;
  for (size_t j = 0; j < count; ++j) {
    double cj = c[j];
    if (anticommute(x[j], z[j], q.x, q.z)) cj = -cj;
    by_x[x[j]].push_back({x[j], z[j], cj});
  }
  // split oversized groups
  std::vector<std::vector<Term>> groups;
  for (auto &kv : by_x) {
    auto &v = kv.second;
    for (size_t a = 0; a < v.size(); a += kExpMaxTerms)
      groups.emplace_back(v.begin() + a, v.begin() + std::min(v.size(), a + (size_t)kExpMaxTerms));
  }
  std::vector<char> used(groups.size(), 0);
  size_t left = groups.size();
  const int dmax = std::min(mode == 1 ? kPsumD : kExpD, sv->n);
  while (left > 0 || runs.empty()) {
    HostExpRun r;
    std::memset(&r.dev, 0, sizeof(r.dev));
    uint64_t basis[kDMax];
    int piv[kDMax];
    int d = 0;
    auto reduce = [&](uint64_t v) {
      for (int b = 0; b < d; ++b)
        if ((v >> piv[b]) & 1ULL) v ^= basis[b];
      return v;
    };
    std::vector<size_t> members;
    size_t n_terms = 0;
    for (size_t g = 0; g < groups.size(); ++g) {
      if (used[g]) continue;
      if ((int)members.size() >= kExpMaxGroups) break;
      if (n_terms + groups[g].size() > (size_t)kExpMaxTerms) continue;
      uint64_t rr = reduce(groups[g][0].x);
      if (rr != 0) {
        if (d >= dmax) continue;
        int p = 63 - __builtin_clzll(rr);
        for (int b = 0; b < d; ++b)
          if ((basis[b] >> p) & 1ULL) basis[b] ^= rr;
        int pos = d;
        while (pos > 0 && piv[pos - 1] > p) {
          basis[pos] = basis[pos - 1];
          piv[pos] = piv[pos - 1];
          --pos;
        }
        basis[pos] = rr;
        piv[pos] = p;
        ++d;
      }
      used[g] = 1;
      --left;
      members.push_back(g);
      n_terms += groups[g].size();
    }
    r.dev.d = d;
    for (int b = 0; b < d; ++b) {
      r.dev.basis[b] = basis[b];
      r.dev.piv[b] = piv[b];
    }
    for (size_t g : members) {
      ExpGroupDev G;
      G.u = 0;
      for (int b = 0; b < d; ++b)
        if ((groups[g][0].x >> piv[b]) & 1ULL) G.u |= 1 << b;
      G.first = (int32_t)r.terms.size();
      G.count = (int32_t)groups[g].size();
      G.pad = 0;
      for (const Term &t : groups[g]) {
        ExpTermDev e;
        e.z = t.z;
        uint32_t zt = 0;
        for (int l = 0; l < (1 << d); ++l) {
          uint64_t s = 0;
          for (int b = 0; b < d; ++b)
            if ((l >> b) & 1) s ^= basis[b];
          zt |= (uint32_t)(popc64(s & t.z) & 1) << l;
        }
        e.zt = zt;
        int ny = popc64(t.x & t.z) & 3;
        if (mode == 0) {
          if (t.x == 0) {
            e.coef = t.c;
            e.imag = 0;
          } else {
            e.coef = 2.0 * t.c * ((ny == 0 || ny == 1) ? 1.0 : -1.0);
            e.imag = ny & 1;
          }
          G.pad |= e.imag ? 2 : 1;  // the group's terms read the real / the imaginary part
        } else {
          e.coef = t.c;
          e.imag = (uint32_t)ny;
          G.pad |= (ny & 1) ? 2 : 1;  // the group's coefficient has a real / an imaginary part
        }
        r.terms.push_back(e);
      }
      r.groups.push_back(G);
    }
    r.dev.n_groups = (int32_t)r.groups.size();
    r.dev.with_norm = runs.empty() ? 1 : 0;
    runs.push_back(std::move(r));
    if (left == 0) break;
  }
}

// stage all runs' groups and terms in one copy; returns device pointers per run
int stage_runs(sv_state *sv, const std::vector<HostExpRun> &runs, std::vector<const ExpGroupDev *> &dg,
               std::vector<const ExpTermDev *> &dt) {
  size_t bytes = 0;
  std::vector<size_t> og(runs.size()), ot(runs.size());
  for (size_t r = 0; r < runs.size(); ++r) {
    og[r] = bytes;
    bytes += (runs[r].groups.size() * sizeof(ExpGroupDev) + 15) & ~size_t(15);
    ot[r] = bytes;
    bytes += (runs[r].terms.size() * sizeof(ExpTermDev) + 15) & ~size_t(15);
  }
  if (bytes == 0) bytes = 16;
  // the previous call's copy out of the pinned stage must be complete
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  int rc = ensure_stage(sv, bytes);
  if (rc) return rc;
  char *h = (char *)sv->h_stage;
  for (size_t r = 0; r < runs.size(); ++r) {
    if (!runs[r].groups.empty())
      std::memcpy(h + og[r], runs[r].groups.data(), runs[r].groups.size() * sizeof(ExpGroupDev));
    if (!runs[r].terms.empty())
      std::memcpy(h + ot[r], runs[r].terms.data(), runs[r].terms.size() * sizeof(ExpTermDev));
  }
  PR_CUDA(cudaMemcpyAsync(sv->d_stage, h, bytes, cudaMemcpyHostToDevice, sv->stream));
  dg.resize(runs.size());
  dt.resize(runs.size());
  for (size_t r = 0; r < runs.size(); ++r) {
    dg[r] = (const ExpGroupDev *)((char *)sv->d_stage + og[r]);
    dt[r] = (const ExpTermDev *)((char *)sv->d_stage + ot[r]);
  }
  return SV_OK;
}

template <typename K>
int occ_blocks(K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (per_sm > 0 ? per_sm : 1) * device_sm_count();
}

template <typename R, typename Idx, int D>
int run_expval_t(sv_state *sv, const std::vector<HostExpRun> &runs, const std::vector<const ExpGroupDev *> &dg,
                 const std::vector<const ExpTermDev *> &dt, double *energy, double *norm2) {
  using C = typename Cx<R>::T;
  static const int cap = occ_blocks(k_expval<R, Idx, D>);
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + kThreads - 1) / kThreads;
  int blocks = (int)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (blocks < 1) blocks = 1;
  int rc = ensure_scratch(sv, (size_t)2 * blocks * runs.size(), 2 * runs.size());
  if (rc) return rc;
  for (size_t r = 0; r < runs.size(); ++r) {
    const int tr = trace_begin(sv, KN_EXPVAL);
    k_expval<R, Idx, D><<<blocks, kThreads, 0, sv->stream>>>((const C *)sv->amps, (Idx)n_cosets, runs[r].dev,
                                                            dg[r], dt[r], sv->d_partials + 2 * blocks * r);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_EXPVAL, (double)sizeof(C) * (double)(1ULL << sv->n));
  }
  const int tr = trace_begin(sv, KN_FINISH);
  k_finish<<<(unsigned)runs.size(), kThreads, 0, sv->stream>>>(sv->d_partials, blocks, sv->d_results);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_FINISH, 16.0 * blocks * runs.size());
  PR_CUDA(cudaMemcpyAsync(sv->h_results, sv->d_results, 2 * runs.size() * sizeof(double), cudaMemcpyDeviceToHost,
                          sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  double e = 0.0;
  for (size_t r = 0; r < runs.size(); ++r) e += sv->h_results[2 * r];
  if (energy) *energy = e;
  if (norm2) *norm2 = sv->h_results[1];
  return SV_OK;
}

// every run is padded to the same coset dimension D = min(kExpD, n)
template <typename R, typename Idx>
int run_expval_d(sv_state *sv, int d, const std::vector<HostExpRun> &runs,
                 const std::vector<const ExpGroupDev *> &dg, const std::vector<const ExpTermDev *> &dt,
                 double *energy, double *norm2) {
  switch (d) {
    case 1: return run_expval_t<R, Idx, 1>(sv, runs, dg, dt, energy, norm2);
    case 2: return run_expval_t<R, Idx, 2>(sv, runs, dg, dt, energy, norm2);
    case 3: return run_expval_t<R, Idx, 3>(sv, runs, dg, dt, energy, norm2);
    default: return run_expval_t<R, Idx, kExpD>(sv, runs, dg, dt, energy, norm2);
  }
}

// pad every run's basis to the kernel's fixed dimension with unused index bits
void pad_runs(int n, int D, std::vector<HostExpRun> &runs) {
  for (auto &r : runs) {
    int d = r.dev.d;
    uint64_t used = 0;
    for (int b = 0; b < d; ++b) used |= 1ULL << r.dev.piv[b];
    for (int bit = n - 1; bit >= 0 && d < D; --bit) {
      if ((used >> bit) & 1ULL) continue;
      // a new unit vector e_bit: it has pivot `bit`; existing basis vectors
      // with that bit set must drop it to stay reduced
      uint64_t e = 1ULL << bit;
      for (int b = 0; b < d; ++b)
        if ((r.dev.basis[b] >> bit) & 1ULL) r.dev.basis[b] ^= e;
      int pos = d;
      while (pos > 0 && r.dev.piv[pos - 1] > bit) {
        r.dev.basis[pos] = r.dev.basis[pos - 1];
        r.dev.piv[pos] = r.dev.piv[pos - 1];
        --pos;
      }
      r.dev.basis[pos] = e;
      r.dev.piv[pos] = bit;
      used |= e;
      ++d;
    }
    r.dev.d = d;
  }
}

// recompute u and zt after padding (coordinates change when pivots are added)
void recode_runs(std::vector<HostExpRun> &runs, const std::vector<std::vector<uint64_t>> &gx) {
  for (size_t r = 0; r < runs.size(); ++r) {
    auto &R = runs[r];
    const int d = R.dev.d;
    for (size_t g = 0; g < R.groups.size(); ++g) {
      uint64_t xg = gx[r][g];
      int u = 0;
      for (int b = 0; b < d; ++b)
        if ((xg >> R.dev.piv[b]) & 1ULL) u |= 1 << b;
      R.groups[g].u = u;
      for (int j = R.groups[g].first; j < R.groups[g].first + R.groups[g].count; ++j) {
        uint32_t zt = 0;
        for (int l = 0; l < (1 << d); ++l) {
          uint64_t s = 0;
          for (int b = 0; b < d; ++b)
            if ((l >> b) & 1) s ^= R.dev.basis[b];
          zt |= (uint32_t)(popc64(s & R.terms[j].z) & 1) << l;
        }
        R.terms[j].zt = zt;
      }
    }
  }
}

int prepare(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count, int mode,
            std::vector<HostExpRun> &runs, int &D) {
  if (count && (!x || !z || !c)) return fail(SV_EINVAL, "NULL term arrays");
  int rc = validate_masks(sv->n, x, z, count);
  if (rc) return rc;
  for (size_t j = 0; j < count; ++j)
    if (!std::isfinite(c[j])) return fail(SV_EINVAL, "coefficient %zu is not finite", j);
  plan_groups(sv, x, z, c, count, mode, runs);
  // remember each group's x before padding changes the basis
  std::vector<std::vector<uint64_t>> gx(runs.size());
  {
    // rebuild x per group from the basis and u (valid before padding)
    for (size_t r = 0; r < runs.size(); ++r) {
      for (auto &G : runs[r].groups) {
        uint64_t v = 0;
        for (int b = 0; b < runs[r].dev.d; ++b)
          if ((G.u >> b) & 1) v ^= runs[r].dev.basis[b];
        gx[r].push_back(v);
      }
    }
  }
  D = std::min(mode == 1 ? kPsumD : kExpD, sv->n);
  pad_runs(sv->n, D, runs);
  recode_runs(runs, gx);
  return SV_OK;
}

// ------------------------------------------------------------------ complex64: exact fixed-point sums
//
// For complex64 amplitudes every product of two components is an exact 48-bit
// integer times a power of two.  Each product is rounded once to the
// fixed-point grid 2^-S (S = 60 for a normalised state); every sum after that
// is exact 64-bit integer arithmetic.  A per-term sum is therefore exact up to
// 2^-(S+1) per product -- at least as accurate as accumulating the exact
// products in FP64 -- and independent of summation order.  The FP64
// coefficients c_j multiply the exact per-term sums on the host.  All of it
// runs on the integer pipes instead of GB300's narrow FP64 pipe.
//
// Work split.  Terms are grouped by x-mask (Sec. "Multi-qubit rotations in a
// fullstate simulator": P|k> pairs k with k^x).
// A thread owns a tile: the coset rep + span(b_0..b_3) of 16 amplitudes,
// where the basis spans the x-masks of the run and is padded with free index
// bits.  For an x-mask with coordinates u != 0 in that basis, l and l^u pair
// up (the leader l has bit H = msb(u) clear), and with zeta_b = parity(b_b & z)
//   sum_l (-1)^{zeta.l} conj(a_{l^u}) a_l
//       = 2 sum_leaders (-1)^{zeta.l} Re(conj(a_l) a_m)      nY even
//       = -2i sum_leaders (-1)^{zeta.l} Im(conj(a_l) a_m)    nY odd,  m = l^u.
// The 8 pair values W[p] of one (u, part) group go through an in-register
// Walsh-Hadamard transform; afterwards every term of the group, whatever its
// z, is one transform entry (zeta with bit H removed) times the tile sign
// (-1)^{popc(rep & z)}.  u = 0 (diagonal terms, identities and the norm)
// transforms the 16 values |a_l|^2 instead.  The products and the transform
// are paid once per group and tile; each term then costs one shared-memory
// read and one 64-bit add per tile.

constexpr int kWD = 4;  // tile dimension
constexpr int kWE = 1 << kWD;
constexpr int kWTerms = 28;   // terms per run, the norm included
constexpr int kWGroups = 16;  // (u, part) groups per run
constexpr int kWThreads = 128;

struct WhtGroupDev {
  int32_t u;     // coordinates of the x-mask in the run basis
  int32_t imag;  // u != 0: 0 = Re conj(a_l) a_m, 1 = Im
  int32_t t0;    // terms [t0, t1) of the run
  int32_t t1;
};
struct WhtTermDev {
  uint64_t z;
  int32_t slot;  // transform entry: zeta, with bit msb(u) removed when u != 0
  int32_t pad;
};
struct WhtRunDev {
  uint64_t basis[kWD];
  int32_t piv[kWD];  // ascending
  int32_t ngroups;
  int32_t nterms;
};

struct FixComp {
  int32_t m;  // signed mantissa times 2^7: |m| < 2^31, low 7 bits clear
  int32_t e;  // value = m * 2^(e - 7)
};

__device__ __forceinline__ FixComp fix_split(float f) {
  const uint32_t b = __float_as_uint(f);
  const int32_t ex = (int32_t)((b >> 23) & 0xffu);
  int32_t m = (int32_t)(b & 0x7fffffu);
  if (ex) m |= 0x800000;
  m <<= 7;
  FixComp c;
  c.m = (b >> 31) ? -m : m;
  c.e = (ex ? ex : 1) - 150;
  return c;
}

// round(a * b * 2^S) with K = 14 - S.  The caller picks S so that every
// component satisfies |x| <= 2^((60 - S)/2) (S = 60 - ceil(log2 <a|a>)), hence
// a.e + b.e + S <= 14 and the shift k is never negative.  The product
// m_a m_b 2^14 is exact (|.| < 2^62); adding half a unit before the
// arithmetic right shift rounds to nearest.  k is capped at 63: there the
// added 2^62 makes every p (|p| < 2^62) non-negative and below 2^63, so the
// result is 0, the correctly rounded value of a product below half a unit.
__device__ __forceinline__ long long fix_mul(FixComp a, FixComp b, int K) {
  const int k = min(K - a.e - b.e, 63);
  const long long half = (1LL << k) >> 1;
  return ((long long)a.m * (long long)b.m + half) >> k;
}

__host__ __device__ constexpr int fix_high_bit(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return h;
}

__host__ __device__ constexpr int fix_leader(int p, int H) {
  return ((p >> H) << (H + 1)) | (p & ((1 << H) - 1));
}

// in-place transform W^[i] = sum_p (-1)^{popc(p & i)} W[p] over N = 2^d entries
template <int N>
__device__ __forceinline__ void fix_wht(long long (&W)[kWE]) {
  constexpr int LOG = fix_high_bit(N);
#pragma unroll
  for (int lv = 0; lv < LOG; ++lv) {
    const int h = 1 << lv;
#pragma unroll
    for (int p = 0; p < N; ++p)
      if (!(p & h)) {
        const long long a = W[p], b = W[p | h];
        W[p] = a + b;
        W[p | h] = a - b;
      }
  }
}

// products and transform of one group; the N entries go to the thread's
// column of sw.  Returns nothing: the caller reads sw[slot][tid].
template <int U>
__device__ __forceinline__ void fix_group(const FixComp (&re)[kWE], const FixComp (&im)[kWE], int imag, int K,
                                          long long (*sw)[kWThreads]) {
  long long W[kWE];
  if (U == 0) {
#pragma unroll
    for (int l = 0; l < kWE; ++l) W[l] = fix_mul(re[l], re[l], K) + fix_mul(im[l], im[l], K);
    fix_wht<kWE>(W);
#pragma unroll
    for (int l = 0; l < kWE; ++l) sw[l][threadIdx.x] = W[l];
  } else {
    constexpr int H = fix_high_bit(U), P = kWE / 2;
    if (!imag) {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int l = fix_leader(p, H), m = l ^ U;
        W[p] = fix_mul(re[l], re[m], K) + fix_mul(im[l], im[m], K);  // Re conj(a_l) a_m
      }
    } else {
#pragma unroll
      for (int p = 0; p < P; ++p) {
        const int l = fix_leader(p, H), m = l ^ U;
        W[p] = fix_mul(re[l], im[m], K) - fix_mul(im[l], re[m], K);  // Im conj(a_l) a_m
      }
    }
    fix_wht<P>(W);
#pragma unroll
    for (int p = 0; p < P; ++p) sw[p][threadIdx.x] = W[p];
  }
}

__device__ __forceinline__ void fix_dispatch(int u, int imag, const FixComp (&re)[kWE], const FixComp (&im)[kWE],
                                             int K, long long (*sw)[kWThreads]) {
  switch (u) {
    case 0: fix_group<0>(re, im, imag, K, sw); break;
    case 1: fix_group<1>(re, im, imag, K, sw); break;
    case 2: fix_group<2>(re, im, imag, K, sw); break;
    case 3: fix_group<3>(re, im, imag, K, sw); break;
    case 4: fix_group<4>(re, im, imag, K, sw); break;
    case 5: fix_group<5>(re, im, imag, K, sw); break;
    case 6: fix_group<6>(re, im, imag, K, sw); break;
    case 7: fix_group<7>(re, im, imag, K, sw); break;
    case 8: fix_group<8>(re, im, imag, K, sw); break;
    case 9: fix_group<9>(re, im, imag, K, sw); break;
    case 10: fix_group<10>(re, im, imag, K, sw); break;
    case 11: fix_group<11>(re, im, imag, K, sw); break;
    case 12: fix_group<12>(re, im, imag, K, sw); break;
    case 13: fix_group<13>(re, im, imag, K, sw); break;
    case 14: fix_group<14>(re, im, imag, K, sw); break;
    case 15: fix_group<15>(re, im, imag, K, sw); break;
    default: break;
  }
}

template <typename Idx>
__global__ void __launch_bounds__(kWThreads, 4)
    k_expval_fix(const float2 *__restrict__ amp, Idx n_tiles, const WhtRunDev run,
                 const WhtGroupDev *__restrict__ ggroups, const WhtTermDev *__restrict__ gterms, int K,
                 long long *__restrict__ partials, int reverse) {
  // consecutive runs only read the state and write their own partials: the
  // next run may start while this one drains (expval_fix_t launches them)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ WhtGroupDev groups[kWGroups];
  __shared__ Idx tz[kWTerms];
  __shared__ int tslot[kWTerms];
  __shared__ Idx soff[kWE];
  // one column per thread: conflict-free 8-byte rows
  __shared__ long long sw[kWE][kWThreads];
  __shared__ long long sacc[kWTerms][kWThreads];
  const int ng = run.ngroups, nt = run.nterms;
  if (threadIdx.x < ng) groups[threadIdx.x] = ggroups[threadIdx.x];
  if (threadIdx.x < nt) {
    tz[threadIdx.x] = (Idx)gterms[threadIdx.x].z;
    tslot[threadIdx.x] = gterms[threadIdx.x].slot;
  }
  if (threadIdx.x < kWE) {
    uint64_t so = 0;
    for (int b = 0; b < kWD; ++b)
      if ((threadIdx.x >> b) & 1) so ^= run.basis[b];
    soff[threadIdx.x] = (Idx)so;
  }
  for (int j = 0; j < kWTerms; ++j) sacc[j][threadIdx.x] = 0;
  __syncthreads();
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx c = (Idx)blockIdx.x * blockDim.x + threadIdx.x; c < n_tiles; c += stride) {
    // consecutive runs read the tiles in opposite orders, so each run starts on
    // the amplitudes the previous one read last (still in L2)
    Idx rep = reverse ? n_tiles - 1 - c : c;
#pragma unroll
    for (int b = 0; b < kWD; ++b) {
      const int pv = run.piv[b];
      rep = ((rep >> pv) << (pv + 1)) | (rep & ((Idx(1) << pv) - 1));
    }
    FixComp re[kWE], im[kWE];
#pragma unroll
    for (int l = 0; l < kWE; ++l) {
      const float2 v = amp[rep ^ soff[l]];
      re[l] = fix_split(v.x);
      im[l] = fix_split(v.y);
    }
    for (int g = 0; g < ng; ++g) {
      const WhtGroupDev G = groups[g];
      // products and shifts depend on the tile only; without this the
      // compiler hoists every case's products out of the group loop at once
#pragma unroll
      for (int l = 0; l < kWE; ++l) asm volatile("" : "+r"(re[l].m), "+r"(im[l].m), "+r"(re[l].e), "+r"(im[l].e));
      fix_dispatch(G.u, G.imag, re, im, K, sw);
      for (int t = G.t0; t < G.t1; ++t) {
        const long long v = sw[tslot[t]][threadIdx.x];
        const long long s = -(long long)(__popcll((unsigned long long)(rep & tz[t])) & 1);
        sacc[t][threadIdx.x] += (v ^ s) - s;
      }
    }
  }
  __syncthreads();
  // exact block sums: warp w reduces rows w, w + 4, ...
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < kWTerms; j += (int)(blockDim.x >> 5)) {
    long long v = 0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += sacc[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partials[(size_t)blockIdx.x * kWTerms + j] = v;
  }
  // the grid completes only after the previous run has: completion of the last
  // run then implies completion of them all
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// ---- complex128 <H> on the same plan, in 64-bit fixed point -------------------
//
// The tiles, groups, transforms and per-term integer sums of k_expval_fix, for
// FP64 amplitudes: a tile's 32 components become signed integers below 2^59 on
// one exponent per tile (fixed64.cuh; resolution 2^-57 of the tile's largest
// component or finer), each pair product is a truncated 62-bit fixed-point
// product (three 32 x 32 -> 64-bit multiplies), the group's 8 (16) pair values
// go through the int64 Walsh-Hadamard transform, and every transform entry is
// rounded once onto the grid 2^-S shared by all tiles, after which all sums are
// exact.  A transform entry is at most the tile's squared norm, so with
// S = 60 - ceil(log2 <a|a>) no sum exceeds 2^60.  No FP64 arithmetic per
// amplitude: GB300's FP64 pipe bounded the FP64 version.

// round(v 2^-k) for k > 0 (ties up; |v| < 2^61, so k >= 62 gives 0), v 2^-k for
// k <= 0 (the choice of S keeps the result below 2^60)
__device__ __forceinline__ long long fx_regrid(long long v, int k) {
  if (k <= 0) return v << min(-k, 63);
  const int kk = min(k, 62);
  return (v + (1LL << (kk - 1))) >> kk;
}

template <int U>
__device__ __forceinline__ void fx128_group(const long long (&re)[kWE], const long long (&im)[kWE], int imag, int k,
                                            long long (*sw)[kWThreads]) {
  long long W[kWE];
  if (U == 0) {
#pragma unroll
    for (int l = 0; l < kWE; ++l) {
      int32_t rh, rl, ih, il;
      fx_limbs(re[l], rh, rl);
      fx_limbs(im[l], ih, il);
      W[l] = fx_prod(re[l], rh, rl) + fx_prod(im[l], ih, il);
    }
    fix_wht<kWE>(W);
#pragma unroll
    for (int l = 0; l < kWE; ++l) sw[l][threadIdx.x] = fx_regrid(W[l], k);
  } else {
    constexpr int H = fix_high_bit(U), P = kWE / 2;
#pragma unroll
    for (int p = 0; p < P; ++p) {
      const int l = fix_leader(p, H), m = l ^ U;
      int32_t mxh, mxl, myh, myl;
      fx_limbs(re[m], mxh, mxl);
      fx_limbs(im[m], myh, myl);
      W[p] = !imag ? fx_prod(re[l], mxh, mxl) + fx_prod(im[l], myh, myl)    // Re conj(a_l) a_m
                   : fx_prod(re[l], myh, myl) - fx_prod(im[l], mxh, mxl);   // Im conj(a_l) a_m
    }
    fix_wht<P>(W);
#pragma unroll
    for (int p = 0; p < P; ++p) sw[p][threadIdx.x] = fx_regrid(W[p], k);
  }
}

__device__ __forceinline__ void fx128_dispatch(int u, int imag, const long long (&re)[kWE], const long long (&im)[kWE],
                                               int k, long long (*sw)[kWThreads]) {
  switch (u) {
    case 0: fx128_group<0>(re, im, imag, k, sw); break;
    case 1: fx128_group<1>(re, im, imag, k, sw); break;
    case 2: fx128_group<2>(re, im, imag, k, sw); break;
    case 3: fx128_group<3>(re, im, imag, k, sw); break;
    case 4: fx128_group<4>(re, im, imag, k, sw); break;
    case 5: fx128_group<5>(re, im, imag, k, sw); break;
    case 6: fx128_group<6>(re, im, imag, k, sw); break;
    case 7: fx128_group<7>(re, im, imag, k, sw); break;
    case 8: fx128_group<8>(re, im, imag, k, sw); break;
    case 9: fx128_group<9>(re, im, imag, k, sw); break;
    case 10: fx128_group<10>(re, im, imag, k, sw); break;
    case 11: fx128_group<11>(re, im, imag, k, sw); break;
    case 12: fx128_group<12>(re, im, imag, k, sw); break;
    case 13: fx128_group<13>(re, im, imag, k, sw); break;
    case 14: fx128_group<14>(re, im, imag, k, sw); break;
    case 15: fx128_group<15>(re, im, imag, k, sw); break;
    default: break;
  }
}

// S: the global grid exponent (units of 2^-S)
template <typename Idx>
__global__ void __launch_bounds__(kWThreads, 4)
    k_expval_fx128(const double2 *__restrict__ amp, Idx n_tiles, const WhtRunDev run,
                   const WhtGroupDev *__restrict__ ggroups, const WhtTermDev *__restrict__ gterms, int S,
                   long long *__restrict__ partials, int reverse) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ WhtGroupDev groups[kWGroups];
  __shared__ Idx tz[kWTerms];
  __shared__ int tslot[kWTerms];
  __shared__ Idx soff[kWE];
  __shared__ long long sw[kWE][kWThreads];
  __shared__ long long sacc[kWTerms][kWThreads];
  const int ng = run.ngroups, nt = run.nterms;
  if (threadIdx.x < ng) groups[threadIdx.x] = ggroups[threadIdx.x];
  if (threadIdx.x < nt) {
    tz[threadIdx.x] = (Idx)gterms[threadIdx.x].z;
    tslot[threadIdx.x] = gterms[threadIdx.x].slot;
  }
  if (threadIdx.x < kWE) {
    uint64_t so = 0;
    for (int b = 0; b < kWD; ++b)
      if ((threadIdx.x >> b) & 1) so ^= run.basis[b];
    soff[threadIdx.x] = (Idx)so;
  }
  for (int j = 0; j < kWTerms; ++j) sacc[j][threadIdx.x] = 0;
  __syncthreads();
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx c = (Idx)blockIdx.x * blockDim.x + threadIdx.x; c < n_tiles; c += stride) {
    Idx rep = reverse ? n_tiles - 1 - c : c;
#pragma unroll
    for (int b = 0; b < kWD; ++b) {
      const int pv = run.piv[b];
      rep = ((rep >> pv) << (pv + 1)) | (rep & ((Idx(1) << pv) - 1));
    }
    long long re[kWE], im[kWE];
    int k;  // transform entries are in units of 2^-(2 St - 62); to the grid 2^-S
    {
      double2 a[kWE];
      int emax = 0;
#pragma unroll
      for (int l = 0; l < kWE; ++l) {
        a[l] = amp[rep ^ soff[l]];
        emax = max(emax, max((int)((__double_as_longlong(a[l].x) >> 52) & 0x7ff),
                             (int)((__double_as_longlong(a[l].y) >> 52) & 0x7ff)));
      }
      const int St = 1081 - emax;  // |a| < 2^(emax - 1022): every component below 2^59
#pragma unroll
      for (int l = 0; l < kWE; ++l) {
        re[l] = fx_in(a[l].x, 1085 - St);
        im[l] = fx_in(a[l].y, 1085 - St);
      }
      k = 2 * St - 62 - S;
    }
    for (int g = 0; g < ng; ++g) {
      const WhtGroupDev G = groups[g];
#pragma unroll
      for (int l = 0; l < kWE; ++l) asm volatile("" : "+l"(re[l]), "+l"(im[l]));
      fx128_dispatch(G.u, G.imag, re, im, k, sw);
      for (int t = G.t0; t < G.t1; ++t) {
        const long long v = sw[tslot[t]][threadIdx.x];
        const long long s = -(long long)(__popcll((unsigned long long)(rep & tz[t])) & 1);
        sacc[t][threadIdx.x] += (v ^ s) - s;
      }
    }
  }
  __syncthreads();
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < kWTerms; j += (int)(blockDim.x >> 5)) {
    long long v = 0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += sacc[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partials[(size_t)blockIdx.x * kWTerms + j] = v;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

// <a|a> of a complex128 state in FP64, per block (only used to pick S)
__global__ void __launch_bounds__(kThreads) k_norm_est128(const double2 *__restrict__ amp, uint64_t n, double *out) {
  double acc = 0.0, unused = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const double2 v = amp[i];
    acc = fma(v.x, v.x, fma(v.y, v.y, acc));
  }
  block_sum2(acc, unused);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = acc;
    out[2 * blockIdx.x + 1] = acc;
  }
}

// results[r][j] = sum over blocks of partials[r][b][j]; one CTA per run
__global__ void k_finish_fix(const long long *__restrict__ partials, int n_blocks, long long *__restrict__ results) {
  __shared__ long long red[kThreads / 32];
  const long long *p = partials + (size_t)blockIdx.x * n_blocks * kWTerms;
  for (int j = 0; j < kWTerms; ++j) {
    long long v = 0;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) v += p[(size_t)b * kWTerms + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
      results[(size_t)blockIdx.x * kWTerms + j] = t;
    }
    __syncthreads();
  }
}

// |a|^2 estimate in FP32 per thread, FP64 per block: only used to pick S.
// out[2b] sums the squares as they are; out[2b+1] sums the squares of the
// components scaled by 2^64 (exact), times 2^-128, which keeps squares down to
// 2^-254 out of the FP32 underflow range (it overflows once a component
// reaches 1, and then the unscaled sum is accurate).
__global__ void __launch_bounds__(kThreads) k_norm_est(const float2 *__restrict__ amp, uint64_t n, double *out) {
  const float up = 18446744073709551616.0f;  // 2^64
  float acc = 0.f, accs = 0.f;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 v = amp[i];
    acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
    const float sx = v.x * up, sy = v.y * up;
    accs = fmaf(sx, sx, fmaf(sy, sy, accs));
  }
  double a = acc, b = (double)accs * 0x1p-128;
  block_sum2(a, b);
  if (threadIdx.x == 0) {
    out[2 * blockIdx.x] = a;
    out[2 * blockIdx.x + 1] = b;
  }
}

struct FixRunHost {
  WhtRunDev dev;
  std::vector<WhtGroupDev> groups;
  std::vector<WhtTermDev> terms;
  std::vector<double> coef;  // per term; 0 for the norm
  int norm_term = -1;        // index of the norm (u = 0, z = 0) in this run, or -1
};

// Group the frame-rewritten terms by (x, part of conj(a_l) a_m they need).
// The x = 0 terms, led by the norm, fill the first runs; the other groups are
// packed into runs whose x-masks span <= kWD dimensions (<= kWTerms terms,
// <= kWGroups groups).  With no x = 0 terms the norm shares the first x-run.
void plan_fix(const sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
              std::vector<FixRunHost> &runs) {
  const Pauli &q = sv->frame;
  std::map<std::pair<uint64_t, int>, std::vector<Term>> by;
  std::vector<Term> diag;
  for (size_t j = 0; j < count; ++j) {
    double cj = c[j];
    if (anticommute(x[j], z[j], q.x, q.z)) cj = -cj;
    if (x[j] == 0)
      diag.push_back({0, z[j], cj});
    else
      by[{x[j], popc64(x[j] & z[j]) & 1}].push_back({x[j], z[j], cj});
  }
  struct Chunk {
    uint64_t x;
    int part;
    std::vector<Term> t;
  };
  std::vector<Chunk> chunks;
  for (auto &kv : by)
    for (size_t a = 0; a < kv.second.size(); a += kWTerms)
      chunks.push_back({kv.first.first, kv.first.second,
                        std::vector<Term>(kv.second.begin() + a,
                                          kv.second.begin() + std::min(kv.second.size(), a + (size_t)kWTerms))});
  std::vector<char> used(chunks.size(), 0);
  size_t left = chunks.size(), di = 0;
  bool norm_placed = false;
  while (left > 0 || di < diag.size() || !norm_placed) {
    uint64_t basis[kWD];
    int piv[kWD];
    int d = 0;
    auto reduce = [&](uint64_t v) {
      for (int b = 0; b < d; ++b)
        if ((v >> piv[b]) & 1ULL) v ^= basis[b];
      return v;
    };
    // reduced echelon form: pivot = highest bit, absent from every other vector
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
    const bool has_norm = !norm_placed;
    norm_placed = true;
    size_t nterm = has_norm ? 1 : 0;
    std::vector<Term> zt;
    while (di < diag.size() && nterm < (size_t)kWTerms) {
      zt.push_back(diag[di++]);
      ++nterm;
    }
    // x = 0 terms first, in runs of their own: every run holding one pays for
    // the 16-entry |a|^2 transform, so they are not spread over the x-runs
    std::vector<size_t> members;
    for (size_t g = 0; g < chunks.size() && zt.empty() && members.size() + 1 < (size_t)kWGroups; ++g) {
      if (used[g] || nterm + chunks[g].t.size() > (size_t)kWTerms) continue;
      const uint64_t rr = reduce(chunks[g].x);
      if (rr != 0) {
        if (d >= kWD) continue;
        add_vec(rr);
      }
      used[g] = 1;
      --left;
      members.push_back(g);
      nterm += chunks[g].t.size();
      if (nterm == (size_t)kWTerms) break;
    }
    // pad to kWD with the highest unused index bits (keeps low bits for coalescing)
    uint64_t usedbits = 0;
    for (int b = 0; b < d; ++b) usedbits |= 1ULL << piv[b];
    for (int bit = sv->n - 1; bit >= 0 && d < kWD; --bit)
      if (!((usedbits >> bit) & 1ULL)) {
        add_vec(1ULL << bit);
        usedbits |= 1ULL << bit;
      }
    FixRunHost r;
    std::memset(&r.dev, 0, sizeof(r.dev));
    for (int b = 0; b < kWD; ++b) {
      r.dev.basis[b] = basis[b];
      r.dev.piv[b] = piv[b];
    }
    auto zeta = [&](uint64_t zz) {
      int v = 0;
      for (int b = 0; b < kWD; ++b) v |= (int)(popc64(basis[b] & zz) & 1) << b;
      return v;
    };
    auto open_group = [&](int u, int imag) {
      WhtGroupDev g;
      g.u = u;
      g.imag = imag;
      g.t0 = g.t1 = (int32_t)r.terms.size();
      r.groups.push_back(g);
    };
    auto add_term = [&](uint64_t zz, int slot, double cf) {
      WhtTermDev e;
      e.z = zz;
      e.slot = slot;
      e.pad = 0;
      r.terms.push_back(e);
      r.coef.push_back(cf);
      r.groups.back().t1 = (int32_t)r.terms.size();
    };
    if (has_norm || !zt.empty()) {
      open_group(0, 0);
      if (has_norm) {
        r.norm_term = (int)r.terms.size();
        add_term(0, 0, 0.0);
      }
      for (const Term &t : zt) add_term(t.z, zeta(t.z), t.c);
    }
    // groups in ascending (u, part) order
    std::vector<std::pair<int, size_t>> order;
    for (size_t g : members) {
      int u = 0;
      for (int b = 0; b < kWD; ++b)
        if ((chunks[g].x >> piv[b]) & 1ULL) u |= 1 << b;
      order.push_back({u * 2 + chunks[g].part, g});
    }
    std::stable_sort(order.begin(), order.end(),
                     [](const std::pair<int, size_t> &a1, const std::pair<int, size_t> &b1) { return a1.first < b1.first; });
    for (auto &ug : order) {
      const int u = ug.first >> 1;
      const Chunk &ch = chunks[ug.second];
      const int H = fix_high_bit(u);
      open_group(u, ch.part);
      for (const Term &t : ch.t) {
        const int zb = zeta(t.z);
        const int slot = (zb & ((1 << H) - 1)) | ((zb >> (H + 1)) << H);
        const int ny = popc64(t.x & t.z) & 3;
        add_term(t.z, slot, 2.0 * t.c * ((ny == 0 || ny == 1) ? 1.0 : -1.0));
      }
    }
    r.dev.ngroups = (int32_t)r.groups.size();
    r.dev.nterms = (int32_t)r.terms.size();
    runs.push_back(std::move(r));
  }
}

template <typename K>
int fix_cap(K kernel) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kWThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (per_sm > 0 ? per_sm : 1) * device_sm_count();
}

// complex64 (k_expval_fix, exact products of FP32 components) or complex128
// (k_expval_fx128, 62-bit fixed-point products) on the same plan
template <typename Idx>
int expval_fix_t(sv_state *sv, const std::vector<FixRunHost> &runs, double *energy, double *norm2) {
  static const int cap64 = fix_cap(k_expval_fix<Idx>);
  static const int cap128 = fix_cap(k_expval_fx128<Idx>);
  const bool c128 = sv->dtype == SV_C128;
  const int cap = c128 ? cap128 : cap64;
  const uint64_t n_amps = 1ULL << sv->n;
  const uint64_t n_tiles = n_amps >> kWD;
  const uint64_t need = (n_tiles + kWThreads - 1) / kWThreads;
  const int blocks = (int)(need < (uint64_t)cap ? (need ? need : 1) : cap);
  const int est_blocks = 512;
  // partial sums (int64) and the S estimate share the double scratch
  int rc = ensure_scratch(sv, (size_t)kWTerms * blocks * runs.size(), kWTerms * runs.size() + 2 * est_blocks);
  if (rc) return rc;
  // stage groups (a fixed kWGroups block) and terms of every run
  constexpr size_t kGroupBytes = sizeof(WhtGroupDev) * kWGroups;
  size_t bytes = 0;
  std::vector<size_t> off(runs.size());
  for (size_t r = 0; r < runs.size(); ++r) {
    off[r] = bytes;
    bytes += kGroupBytes + runs[r].terms.size() * sizeof(WhtTermDev);
  }
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  rc = ensure_stage(sv, bytes);
  if (rc) return rc;
  for (size_t r = 0; r < runs.size(); ++r) {
    char *dst = (char *)sv->h_stage + off[r];
    std::memset(dst, 0, kGroupBytes);
    std::memcpy(dst, runs[r].groups.data(), runs[r].groups.size() * sizeof(WhtGroupDev));
    if (!runs[r].terms.empty())
      std::memcpy(dst + kGroupBytes, runs[r].terms.data(), runs[r].terms.size() * sizeof(WhtTermDev));
  }
  PR_CUDA(cudaMemcpyAsync(sv->d_stage, sv->h_stage, bytes, cudaMemcpyHostToDevice, sv->stream));
  // choose S from an estimate of <a|a>
  double *d_est = sv->d_results + kWTerms * runs.size();
  {
    const int tr = trace_begin(sv, KN_EXPVAL);
    if (c128)
      k_norm_est128<<<est_blocks, kThreads, 0, sv->stream>>>((const double2 *)sv->amps, n_amps, d_est);
    else
      k_norm_est<<<est_blocks, kThreads, 0, sv->stream>>>((const float2 *)sv->amps, n_amps, d_est);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_EXPVAL, (c128 ? 16.0 : 8.0) * (double)n_amps);
  }
  PR_CUDA(cudaMemcpyAsync(sv->h_results, d_est, 2 * est_blocks * sizeof(double), cudaMemcpyDeviceToHost, sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  double plain = 0.0, scaled = 0.0;
  for (int i = 0; i < est_blocks; ++i) {
    plain += sv->h_results[2 * i];
    scaled += sv->h_results[2 * i + 1];
  }
  if (!std::isfinite(plain)) return fail(SV_EUNSUPPORTED, "state norm is not finite");
  const double nest = std::isfinite(scaled) ? scaled : plain;
  // S = 60 - ceil(log2 <a|a>) (estimate widened by 2 %): every per-term sum,
  // and every intermediate of the tile transforms, is bounded by
  // <a|a> 2^S <= 2^60, and no product needs a left shift.  Each thread of
  // k_norm_est sums at most 2^(n-17) FP32 squares (relative error < 0.2 % for
  // n <= 32).  The scaled sum loses squares below 2^-254, at most 2^(n-254) of
  // mass, under 0.8 % of any estimate above 2^(n-247), which therefore bounds
  // S; the unscaled sum is used only when it is at least about 1.
  // For complex128 the FP64 squares lose only amplitudes below 2^-537, at most
  // 2^(n-1074) of mass, so the floor is 2^(n-1000).
  const double est = std::max(nest, std::ldexp(1.0, sv->n - (c128 ? 1000 : 247)));
  const int S = 60 - (int)std::ceil(std::log2(est * 1.02));
  // complex128 takes any finite norm (S >= -1024); complex64 transforms need S >= 8
  if (!c128 && S < 8) return fail(SV_EUNSUPPORTED, "state norm %g too large for the fixed-point sums", nest);
  long long *part = (long long *)sv->d_partials;
  long long *res = (long long *)sv->d_results;
  for (size_t r = 0; r < runs.size(); ++r) {
    const char *base = (const char *)sv->d_stage + off[r];
    const int tr = trace_begin(sv, KN_EXPVAL);
    // programmatic dependent launches: a run's CTAs start as the previous
    // run's last CTAs drain (the grid never exceeds what the GPU holds at
    // once, so no waiting CTA can keep a pending one from running)
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)blocks);
    cfg.blockDim = dim3(kWThreads);
    cfg.stream = sv->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int rev = (int)((r + 1) & 1);
    long long *pr = part + (size_t)kWTerms * blocks * r;
    if (c128)
      PR_CUDA(cudaLaunchKernelEx(&cfg, k_expval_fx128<Idx>, (const double2 *)sv->amps, (Idx)n_tiles, runs[r].dev,
                                 (const WhtGroupDev *)base, (const WhtTermDev *)(base + kGroupBytes), S, pr, rev));
    else
      PR_CUDA(cudaLaunchKernelEx(&cfg, k_expval_fix<Idx>, (const float2 *)sv->amps, (Idx)n_tiles, runs[r].dev,
                                 (const WhtGroupDev *)base, (const WhtTermDev *)(base + kGroupBytes), 14 - S, pr,
                                 rev));
    trace_end(sv, tr, KN_EXPVAL, (c128 ? 16.0 : 8.0) * (double)n_amps);
  }
  {
    const int tr = trace_begin(sv, KN_FINISH);
    k_finish_fix<<<(unsigned)runs.size(), kThreads, 0, sv->stream>>>(part, blocks, res);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_FINISH, 8.0 * kWTerms * blocks * runs.size());
  }
  PR_CUDA(cudaMemcpyAsync(sv->h_results, res, kWTerms * runs.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                          sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  const long long *h = (const long long *)sv->h_results;
  const double unit = std::ldexp(1.0, -S);
  long double e = 0.0L, nrm = 0.0L;
  for (size_t r = 0; r < runs.size(); ++r) {
    for (size_t j = 0; j < runs[r].coef.size(); ++j) e += (long double)runs[r].coef[j] * (long double)h[r * kWTerms + j];
    if (runs[r].norm_term >= 0) nrm += (long double)h[r * kWTerms + runs[r].norm_term];
  }
  if (energy) *energy = (double)(e * unit);
  if (norm2) *norm2 = (double)(nrm * unit);
  return SV_OK;
}

}  // namespace

int expval_impl(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
                double *energy, double *norm2) {
  if (sv->n >= kWD) {
    if (count && (!x || !z || !c)) return fail(SV_EINVAL, "NULL term arrays");
    int rc = validate_masks(sv->n, x, z, count);
    if (rc) return rc;
    for (size_t j = 0; j < count; ++j)
      if (!std::isfinite(c[j])) return fail(SV_EINVAL, "coefficient %zu is not finite", j);
    std::vector<FixRunHost> fr;
    plan_fix(sv, x, z, c, count, fr);
    return sv->n <= 31 ? expval_fix_t<uint32_t>(sv, fr, energy, norm2) : expval_fix_t<uint64_t>(sv, fr, energy, norm2);
  }
  std::vector<HostExpRun> runs;
  int D = 0;
  int rc = prepare(sv, x, z, c, count, 0, runs, D);
  if (rc) return rc;
  std::vector<const ExpGroupDev *> dg;
  std::vector<const ExpTermDev *> dt;
  rc = stage_runs(sv, runs, dg, dt);
  if (rc) return rc;
  const bool narrow = sv->n <= 31;
  if (sv->dtype == SV_C128)
    return narrow ? run_expval_d<double, uint32_t>(sv, D, runs, dg, dt, energy, norm2)
                  : run_expval_d<double, uint64_t>(sv, D, runs, dg, dt, energy, norm2);
  return narrow ? run_expval_d<float, uint32_t>(sv, D, runs, dg, dt, energy, norm2)
                : run_expval_d<float, uint64_t>(sv, D, runs, dg, dt, energy, norm2);
}

template <typename R, typename Idx, int D>
static int run_pauli_sum_t(sv_state *dst, sv_state *src, const std::vector<HostExpRun> &runs,
                           const std::vector<const ExpGroupDev *> &dg, const std::vector<const ExpTermDev *> &dt) {
  using C = typename Cx<R>::T;
  static const int cap = occ_blocks(k_pauli_sum<R, Idx, D>);
  const uint64_t n_cosets = (1ULL << src->n) >> D;
  uint64_t need = (n_cosets + kThreads - 1) / kThreads;
  int blocks = (int)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (blocks < 1) blocks = 1;
  PR_CUDA(cudaMemsetAsync(dst->amps, 0, amp_bytes(dst->dtype) << dst->n, src->stream));
  for (size_t r = 0; r < runs.size(); ++r) {
    const int tr = trace_begin(src, KN_PAULI_SUM);
    k_pauli_sum<R, Idx, D><<<blocks, kThreads, 0, src->stream>>>((C *)dst->amps, (const C *)src->amps,
                                                                    (Idx)n_cosets, runs[r].dev, dg[r], dt[r]);
    PR_CHECK_LAUNCH();
    trace_end(src, tr, KN_PAULI_SUM, 3.0 * (double)sizeof(C) * (double)(1ULL << src->n));
  }
  return SV_OK;
}

template <typename R, typename Idx>
static int pauli_sum_d(sv_state *dst, sv_state *src, int D, const std::vector<HostExpRun> &runs,
                       const std::vector<const ExpGroupDev *> &dg, const std::vector<const ExpTermDev *> &dt) {
  switch (D) {
    case 1: return run_pauli_sum_t<R, Idx, 1>(dst, src, runs, dg, dt);
    case 2: return run_pauli_sum_t<R, Idx, 2>(dst, src, runs, dg, dt);
    default: return run_pauli_sum_t<R, Idx, kPsumD>(dst, src, runs, dg, dt);
  }
}

static int dispatch_pauli_sum(sv_state *dst, sv_state *src, int D, const std::vector<HostExpRun> &runs,
                              const std::vector<const ExpGroupDev *> &dg, const std::vector<const ExpTermDev *> &dt) {
  const bool narrow = src->n <= 31;
  if (src->dtype == SV_C128)
    return narrow ? pauli_sum_d<double, uint32_t>(dst, src, D, runs, dg, dt)
                  : pauli_sum_d<double, uint64_t>(dst, src, D, runs, dg, dt);
  return narrow ? pauli_sum_d<float, uint32_t>(dst, src, D, runs, dg, dt)
                : pauli_sum_d<float, uint64_t>(dst, src, D, runs, dg, dt);
}

int pauli_sum_impl(sv_state *dst, sv_state *src, const uint64_t *x, const uint64_t *z, const double *c,
                   size_t count) {
  if (!dst || !src) return fail(SV_EINVAL, "NULL state");
  if (dst == src || dst->amps == src->amps) return fail(SV_EINVAL, "dst must differ from src");
  if (dst->n != src->n || dst->dtype != src->dtype) return fail(SV_EINVAL, "shape mismatch");
  std::vector<HostExpRun> runs;
  int D = 0;
  int rc = prepare(src, x, z, c, count, 1, runs, D);
  if (rc) return rc;
  // coefficients as round(c_j 2^K) with sum_j |c_j| 2^K <= 2^62 over a run, so
  // every signed partial sum of a group fits in 64 bits; the bits travel in
  // the coef field
  for (HostExpRun &r : runs) {
    double tot = 0.0;
    for (const ExpTermDev &t : r.terms) tot += std::fabs(t.coef);
    int K = tot > 0.0 ? 62 - (int)std::ceil(std::log2(tot * (1.0 + 1e-12))) : 0;
    K = std::max(-960, std::min(960, K));
    for (ExpTermDev &t : r.terms) {
      const long long q = std::llround(std::ldexp(t.coef, K));
      std::memcpy(&t.coef, &q, sizeof(q));
    }
    r.dev.qscale = std::ldexp(1.0, -K);
  }
  std::vector<const ExpGroupDev *> dg;
  std::vector<const ExpTermDev *> dt;
  rc = stage_runs(src, runs, dg, dt);
  if (rc) return rc;
  // dst work is ordered on src's stream; make dst's stream wait for it
  rc = dispatch_pauli_sum(dst, src, D, runs, dg, dt);
  if (rc) return rc;
  if (dst->stream != src->stream) PR_CUDA(cudaStreamSynchronize(src->stream));
  dst->frame = Pauli();
  return SV_OK;
}

}  // namespace pr

using namespace pr;

extern "C" {

int expval_pauli_sum(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *coeff, size_t count,
                     double *out_energy, double *out_norm2) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (!out_energy) return fail(SV_EINVAL, "out_energy is NULL");
  return expval_impl(sv, x, z, coeff, count, out_energy, out_norm2);
}

int apply_pauli_sum(sv_state *dst, sv_state *src, const uint64_t *x, const uint64_t *z, const double *coeff,
                    size_t count) {
  return pauli_sum_impl(dst, src, x, z, coeff, count);
}

}  // extern "C"

// ------------------------------------------------------------------ allocation-free <H>
//
// expval_pauli_sum_noalloc computes the same energy and norm as
// expval_pauli_sum but never allocates: no cudaMalloc/cudaFree, no pinned
// host buffers, no heap.  It is for callers that must not allocate during the
// call -- code that runs under a fixed memory budget handed out by an outer
// framework, latency-critical loops that cannot take the device-wide
// synchronisation a first cudaMalloc implies, and hosts that forbid allocation
// after start-up.  Its device scratch is the file-scope array below (every GPU
// that loads this library holds it until the process exits); its host staging
// is a static buffer guarded by a mutex.
namespace pr {
namespace {

constexpr size_t kNoAllocScratchBytes = 4u << 20;  // 4 MiB of device scratch per GPU
constexpr int kNoAllocMaxTerms = 4096;
constexpr int kNoAllocMaxRuns = 1024;
constexpr int kNoAllocBlocks = 128;  // fixed grid: fixes the partials layout
constexpr int kNoAllocMaxDevices = 64;

// device layout: [groups: runs*16][terms: max terms][partials: runs*blocks*2][results: runs*2]
constexpr size_t kNaGroupsOff = 0;
constexpr size_t kNaTermsOff = kNaGroupsOff + sizeof(ExpGroupDev) * kNoAllocMaxRuns * kExpMaxGroups;
constexpr size_t kNaPartOff = kNaTermsOff + sizeof(ExpTermDev) * kNoAllocMaxTerms;
constexpr size_t kNaResOff = kNaPartOff + sizeof(double) * 2 * kNoAllocBlocks * kNoAllocMaxRuns;
constexpr size_t kNaEnd = kNaResOff + sizeof(double) * 2 * kNoAllocMaxRuns;
static_assert(kNaEnd <= kNoAllocScratchBytes, "no-alloc scratch layout exceeds the array");

}  // namespace
}  // namespace pr

// The scratch itself.  In host code this name is only a stand-in, never a
// device address: the address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[pr::kNoAllocScratchBytes];

namespace pr {
namespace {

struct NoAllocHost {
  uint32_t order[kNoAllocMaxTerms];
  uint64_t tx[kNoAllocMaxTerms], tz[kNoAllocMaxTerms];
  double tc[kNoAllocMaxTerms];
  int32_t grp_first[kNoAllocMaxTerms], grp_count[kNoAllocMaxTerms];
  uint64_t grp_x[kNoAllocMaxTerms];
  char grp_used[kNoAllocMaxTerms];
  ExpRunDev runs[kNoAllocMaxRuns];
  int32_t run_groups[kNoAllocMaxRuns];
  int32_t run_term_off[kNoAllocMaxRuns];
  ExpGroupDev groups[kNoAllocMaxRuns * kExpMaxGroups];
  ExpTermDev terms[kNoAllocMaxTerms];
  double results[2 * kNoAllocMaxRuns];
};
NoAllocHost g_na_host;
std::mutex g_na_mutex;
void *g_na_dev[kNoAllocMaxDevices];

// heap sort of order[0..m) by key x (no allocation)
void sort_by_x(uint32_t *ord, const uint64_t *key, int m) {
  auto less = [&](int a, int b) { return key[ord[a]] < key[ord[b]] || (key[ord[a]] == key[ord[b]] && ord[a] < ord[b]); };
  auto sift = [&](int root, int end) {
    while (2 * root + 1 < end) {
      int ch = 2 * root + 1;
      if (ch + 1 < end && less(ch, ch + 1)) ++ch;
      if (!less(root, ch)) return;
      uint32_t t = ord[root]; ord[root] = ord[ch]; ord[ch] = t;
      root = ch;
    }
  };
  for (int i = m / 2 - 1; i >= 0; --i) sift(i, m);
  for (int end = m - 1; end > 0; --end) {
    uint32_t t = ord[0]; ord[0] = ord[end]; ord[end] = t;
    sift(0, end);
  }
}

// Pack the sign-rewritten terms into runs exactly as plan_groups does, with
// fixed-size arrays.  Returns the number of runs or a negative status.
int na_plan(const sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, int m, int D) {
  NoAllocHost &h = g_na_host;
  const Pauli &q = sv->frame;
  for (int j = 0; j < m; ++j) {
    h.order[j] = (uint32_t)j;
    h.tx[j] = x[j];
    h.tz[j] = z[j];
    h.tc[j] = anticommute(x[j], z[j], q.x, q.z) ? -c[j] : c[j];
  }
  sort_by_x(h.order, h.tx, m);
  int ng = 0;
  for (int a = 0; a < m;) {
    int b = a;
    const uint64_t xa = h.tx[h.order[a]];
    while (b < m && h.tx[h.order[b]] == xa && b - a < kExpMaxTerms) ++b;
    h.grp_first[ng] = a;
    h.grp_count[ng] = b - a;
    h.grp_x[ng] = xa;
    h.grp_used[ng] = 0;
    ++ng;
    a = b;
  }
  int nr = 0, nt = 0, left = ng;
  while (left > 0 || nr == 0) {
    if (nr >= kNoAllocMaxRuns) return fail(SV_EINVAL, "more than %d expectation runs needed", kNoAllocMaxRuns);
    ExpRunDev &R = h.runs[nr];
    std::memset(&R, 0, sizeof(R));
    uint64_t basis[kDMax];
    int piv[kDMax];
    int d = 0;
    auto reduce = [&](uint64_t v) {
      for (int bb = 0; bb < d; ++bb)
        if ((v >> piv[bb]) & 1ULL) v ^= basis[bb];
      return v;
    };
    int members[kExpMaxGroups];
    int nm = 0, run_terms = 0;
    for (int g = 0; g < ng; ++g) {
      if (h.grp_used[g]) continue;
      if (nm >= kExpMaxGroups) break;
      if (run_terms + h.grp_count[g] > kExpMaxTerms) continue;
      uint64_t rr = reduce(h.grp_x[g]);
      if (rr != 0) {
        if (d >= D) continue;
        int p = 63 - __builtin_clzll(rr);
        for (int bb = 0; bb < d; ++bb)
          if ((basis[bb] >> p) & 1ULL) basis[bb] ^= rr;
        int pos = d;
        while (pos > 0 && piv[pos - 1] > p) {
          basis[pos] = basis[pos - 1];
          piv[pos] = piv[pos - 1];
          --pos;
        }
        basis[pos] = rr;
        piv[pos] = p;
        ++d;
      }
      h.grp_used[g] = 1;
      --left;
      members[nm++] = g;
      run_terms += h.grp_count[g];
    }
    // pad the basis to dimension D with the highest unused index bits
    uint64_t used = 0;
    for (int bb = 0; bb < d; ++bb) used |= 1ULL << piv[bb];
    for (int bit = sv->n - 1; bit >= 0 && d < D; --bit) {
      if ((used >> bit) & 1ULL) continue;
      const uint64_t e = 1ULL << bit;
      for (int bb = 0; bb < d; ++bb)
        if ((basis[bb] >> bit) & 1ULL) basis[bb] ^= e;
      int pos = d;
      while (pos > 0 && piv[pos - 1] > bit) {
        basis[pos] = basis[pos - 1];
        piv[pos] = piv[pos - 1];
        --pos;
      }
      basis[pos] = e;
      piv[pos] = bit;
      used |= e;
      ++d;
    }
    R.d = d;
    for (int bb = 0; bb < d; ++bb) {
      R.basis[bb] = basis[bb];
      R.piv[bb] = piv[bb];
    }
    R.n_groups = nm;
    R.with_norm = nr == 0 ? 1 : 0;
    h.run_groups[nr] = nm;
    h.run_term_off[nr] = nt;
    int local = 0;
    for (int k = 0; k < nm; ++k) {
      const int g = members[k];
      ExpGroupDev &G = h.groups[nr * kExpMaxGroups + k];
      G.u = 0;
      for (int bb = 0; bb < d; ++bb)
        if ((h.grp_x[g] >> piv[bb]) & 1ULL) G.u |= 1 << bb;
      G.first = local;  // relative to this run's first term (k_expval stages [0, first+count))
      G.count = h.grp_count[g];
      G.pad = 0;
      for (int i = 0; i < h.grp_count[g]; ++i) {
        const int j = (int)h.order[h.grp_first[g] + i];
        ExpTermDev &t = h.terms[nt + local + i];
        t.z = h.tz[j];
        uint32_t zt = 0;
        for (int l = 0; l < (1 << d); ++l) {
          uint64_t s = 0;
          for (int bb = 0; bb < d; ++bb)
            if ((l >> bb) & 1) s ^= basis[bb];
          zt |= (uint32_t)(popc64(s & h.tz[j]) & 1) << l;
        }
        t.zt = zt;
        const int ny = popc64(h.tx[j] & h.tz[j]) & 3;
        if (h.tx[j] == 0) {
          t.coef = h.tc[j];
          t.imag = 0;
        } else {
          t.coef = 2.0 * h.tc[j] * ((ny == 0 || ny == 1) ? 1.0 : -1.0);
          t.imag = ny & 1;
        }
      }
      local += h.grp_count[g];
    }
    nt += local;
    ++nr;
    if (left == 0) break;
  }
  return nr;
}

// caller holds g_na_mutex
int na_device_scratch(void **out) {
  int dev = 0;
  PR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(SV_EUNSUPPORTED, "device index %d", dev);
  if (!g_na_dev[dev]) {
    void *p = nullptr;
    PR_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_na_dev[dev] = p;
  }
  *out = g_na_dev[dev];
  return SV_OK;
}

template <typename R, typename Idx, int D>
int na_launch(sv_state *sv, char *scratch, int nr, int nt) {
  using C = typename Cx<R>::T;
  NoAllocHost &h = g_na_host;
  // one upload of every run's groups and terms
  PR_CUDA(cudaMemcpyAsync(scratch + kNaGroupsOff, h.groups, sizeof(ExpGroupDev) * kExpMaxGroups * nr,
                          cudaMemcpyHostToDevice, sv->stream));
  PR_CUDA(cudaMemcpyAsync(scratch + kNaTermsOff, h.terms, sizeof(ExpTermDev) * (nt ? nt : 1),
                          cudaMemcpyHostToDevice, sv->stream));
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + kThreads - 1) / kThreads;
  const int blocks = (int)(need < (uint64_t)kNoAllocBlocks ? (need ? need : 1) : kNoAllocBlocks);
  double *part = (double *)(scratch + kNaPartOff);
  double *res = (double *)(scratch + kNaResOff);
  const ExpGroupDev *dg = (const ExpGroupDev *)(scratch + kNaGroupsOff);
  const ExpTermDev *dt = (const ExpTermDev *)(scratch + kNaTermsOff);
  for (int r = 0; r < nr; ++r) {
    k_expval<R, Idx, D><<<blocks, kThreads, 0, sv->stream>>>((const C *)sv->amps, (Idx)n_cosets, h.runs[r],
                                                            dg + (size_t)r * kExpMaxGroups, dt + h.run_term_off[r],
                                                            part + 2 * blocks * r);
    PR_CHECK_LAUNCH();
  }
  k_finish<<<(unsigned)nr, kThreads, 0, sv->stream>>>(part, blocks, res);
  PR_CHECK_LAUNCH();
  PR_CUDA(cudaMemcpyAsync(h.results, res, sizeof(double) * 2 * nr, cudaMemcpyDeviceToHost, sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  return SV_OK;
}

template <typename R, typename Idx>
int na_launch_d(sv_state *sv, char *scratch, int nr, int nt, int D) {
  switch (D) {
    case 1: return na_launch<R, Idx, 1>(sv, scratch, nr, nt);
    case 2: return na_launch<R, Idx, 2>(sv, scratch, nr, nt);
    case 3: return na_launch<R, Idx, 3>(sv, scratch, nr, nt);
    default: return na_launch<R, Idx, kExpD>(sv, scratch, nr, nt);
  }
}

}  // namespace
}  // namespace pr

extern "C" int expval_pauli_sum_noalloc(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *coeff,
                                        size_t count, double *out_energy, double *out_norm2) {
  using namespace pr;
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (!out_energy) return fail(SV_EINVAL, "out_energy is NULL");
  if (count > (size_t)kNoAllocMaxTerms)
    return fail(SV_EINVAL, "expval_pauli_sum_noalloc takes at most %d terms (got %zu)", kNoAllocMaxTerms, count);
  if (count && (!x || !z || !coeff)) return fail(SV_EINVAL, "NULL term arrays");
  int rc = validate_masks(sv->n, x, z, count);
  if (rc) return rc;
  for (size_t j = 0; j < count; ++j)
    if (!std::isfinite(coeff[j])) return fail(SV_EINVAL, "coefficient %zu is not finite", j);
  // the lock also covers the per-device cache of the scratch address, so two
  // threads making their first call on a device do not race on it
  std::lock_guard<std::mutex> lock(g_na_mutex);
  void *scratch = nullptr;
  rc = na_device_scratch(&scratch);
  if (rc) return rc;
  const int D = std::min(kExpD, sv->n);
  const int nr = na_plan(sv, x, z, coeff, (int)count, D);
  if (nr < 0) return nr;
  int nt = 0;
  for (int r = 0; r < nr; ++r)
    for (int k = 0; k < g_na_host.run_groups[r]; ++k) nt += g_na_host.groups[r * kExpMaxGroups + k].count;
  const bool narrow = sv->n <= 31;
  char *s = (char *)scratch;
  if (sv->dtype == SV_C128)
    rc = narrow ? na_launch_d<double, uint32_t>(sv, s, nr, nt, D) : na_launch_d<double, uint64_t>(sv, s, nr, nt, D);
  else
    rc = narrow ? na_launch_d<float, uint32_t>(sv, s, nr, nt, D) : na_launch_d<float, uint64_t>(sv, s, nr, nt, D);
  if (rc) return rc;
  double e = 0.0;
  for (int r = 0; r < nr; ++r) e += g_na_host.results[2 * r];
  *out_energy = e;
  if (out_norm2) *out_norm2 = g_na_host.results[1];
  return SV_OK;
}
