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

#include "internal.h"

namespace pr {

namespace {

constexpr int kExpD = 4;
constexpr int kExpMaxTerms = 1024;
constexpr int kExpMaxGroups = 1 << kExpD;

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

template <int D, int U, typename Idx>
__device__ __forceinline__ void group_terms(const double2 (&a)[1 << D], Idx rep, const ExpTermSm *terms,
                                            int first, int count, double &acc) {
  constexpr int E = 1 << D;
  if (U == 0) {
    double p[E];
#pragma unroll
    for (int l = 0; l < E; ++l) p[l] = a[l].x * a[l].x + a[l].y * a[l].y;
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
    if constexpr ((K) < (1 << D)) group_terms<D, (K)>(a, rep, terms, first, count, acc); \
    break;

template <int D, typename Idx>
__device__ __forceinline__ void group_dispatch(int u, const double2 (&a)[1 << D], Idx rep, const ExpTermSm *terms,
                                               int first, int count, double &acc) {
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
      group_dispatch<D>(G.u, a, rep, terms, G.first, G.count, acc);
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

// dst += sum_g sum_{j in g} c_j i^{nY_j} s_j(k^x) src_{k^x}   (per element k)
template <typename R, typename Idx, int D>
__global__ void __launch_bounds__(kThreads)
    k_pauli_sum(typename Cx<R>::T *__restrict__ dst, const typename Cx<R>::T *__restrict__ src, Idx n_cosets,
                const ExpRunDev run, const ExpGroupDev *__restrict__ groups,
                const ExpTermDev *__restrict__ gterms) {
  using C = typename Cx<R>::T;
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
      a[l].x = (double)v.x;
      a[l].y = (double)v.y;
      const C w = dst[rep ^ soff[l]];
      o[l].x = (double)w.x;
      o[l].y = (double)w.y;
    }
    for (int g = 0; g < run.n_groups; ++g) {
      const ExpGroupDev G = sg[g];
      const int u = G.u;
#pragma unroll
      for (int l = 0; l < E; ++l) {
        const int m = l ^ u;
        double cr = 0.0, ci = 0.0;  // sum_j c_j i^{nY} s_j(k_m)
        for (int j = G.first; j < G.first + G.count; ++j) {
          const ExpTermSm t = terms[j];
          const uint32_t s = (uint32_t)parity((uint64_t)rep & t.z) ^ ((t.zt >> m) & 1u);
          const double cc = (s & 1u) ? -t.coef : t.coef;
          switch (t.imag & 3u) {
            case 0: cr += cc; break;
            case 1: ci += cc; break;
            case 2: cr -= cc; break;
            default: ci -= cc; break;
          }
        }
        // a[m] read with a runtime index: keep the select explicit
        double2 am = a[0];
#pragma unroll
        for (int q = 1; q < E; ++q)
          if (q == m) am = a[q];
        o[l].x = fma(cr, am.x, fma(-ci, am.y, o[l].x));
        o[l].y = fma(cr, am.y, fma(ci, am.x, o[l].y));
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
  const int dmax = std::min(kExpD, sv->n);
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
        } else {
          e.coef = t.c;
          e.imag = (uint32_t)ny;
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
  static int cap = 0;
  if (!cap) cap = occ_blocks(k_expval<R, Idx, D>);
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + kThreads - 1) / kThreads;
  int blocks = (int)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (blocks < 1) blocks = 1;
  int rc = ensure_scratch(sv, (size_t)2 * blocks * runs.size(), 2 * runs.size());
  if (rc) return rc;
  for (size_t r = 0; r < runs.size(); ++r) {
    const int tr = trace_begin(sv);
    k_expval<R, Idx, D><<<blocks, kThreads, 0, sv->stream>>>((const C *)sv->amps, (Idx)n_cosets, runs[r].dev,
                                                            dg[r], dt[r], sv->d_partials + 2 * blocks * r);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_EXPVAL, (double)sizeof(C) * (double)(1ULL << sv->n));
  }
  const int tr = trace_begin(sv);
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
  D = std::min(kExpD, sv->n);
  pad_runs(sv->n, D, runs);
  recode_runs(runs, gx);
  return SV_OK;
}

// ------------------------------------------------------------------ complex64: exact fixed-point sums
//
// For complex64 amplitudes every product of two components is an exact 48-bit
// integer times a power of two.  k_expval_fix rounds each product once to the
// fixed-point grid 2^-S (S = 60 for a normalised state) and sums the integers
// exactly, per Pauli term, in 64-bit registers; the FP64 coefficients c_j are
// applied to the exact per-term sums on the host.  Each sum is therefore exact
// up to 2^-(S+1) per product -- at least as accurate as accumulating the exact
// products in FP64 -- and independent of summation order.  It runs on the
// integer pipes instead of GB300's narrow FP64 pipe.  Cosets of a 3-dimensional
// x-span hold 8 amplitudes per thread; a run carries at most 16 terms.

constexpr int kFixD = 3;
constexpr int kFixTerms = 32;
constexpr int kFixThreads = 128;

struct FixTermDev {
  uint64_t z;
  uint32_t psm;  // sign bit per pair slot (or per element for u = 0)
  int32_t u;
  int32_t imag;
  int32_t need;  // parts of conj(a_l) a_m any term of this u needs: 1 = Re, 2 = Im
};
struct FixRunDev {
  uint64_t basis[kFixD];
  int32_t piv[kFixD];
  int32_t d;
  int32_t nterms;
  int32_t with_norm;
};

struct FixComp {
  int32_t m;  // signed integer mantissa, |m| < 2^24
  int32_t e;  // value = m * 2^e
};

__device__ __forceinline__ FixComp fix_split(float f) {
  const uint32_t b = __float_as_uint(f);
  const int32_t ex = (int32_t)((b >> 23) & 0xffu);
  int32_t m = (int32_t)(b & 0x7fffffu);
  if (ex) m |= 0x800000;
  FixComp c;
  c.m = (b >> 31) ? -m : m;
  c.e = (ex ? ex : 1) - 150;
  return c;
}

// round(a * b * 2^S).  The caller picks S so that every component satisfies
// |x| <= 2^((60 - S)/2) (S = 60 - ceil(log2 <a|a>)), hence a.e + b.e + S <= 14
// and the shift k below is never negative: one rounding right shift of the
// exact 48-bit product pre-shifted by 14 (|p| < 2^48, so p << 14 < 2^62).
__device__ __forceinline__ long long fix_mul(FixComp a, FixComp b, int S) {
  const long long p = (long long)a.m * (long long)b.m;
  const int k = min(max(14 - (a.e + b.e + S), 0), 63);
  return ((p << 14) + ((1LL << k) >> 1)) >> k;
}

__host__ __device__ constexpr int fix_high_bit(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return h;
}

__host__ __device__ constexpr int fix_leader(int p, int H) {
  return ((p >> H) << (H + 1)) | (p & ((1 << H) - 1));
}

template <int U>
__device__ __forceinline__ void fix_products(const FixComp (&re)[1 << kFixD], const FixComp (&im)[1 << kFixD],
                                             long long (&W)[1 << kFixD], int S, int need) {
  constexpr int E = 1 << kFixD, PAIRS = E / 2;
  if (U == 0) {
#pragma unroll
    for (int l = 0; l < E; ++l) W[l] = fix_mul(re[l], re[l], S) + fix_mul(im[l], im[l], S);
  } else {
    constexpr int H = fix_high_bit(U);
    if (need & 1) {
#pragma unroll
      for (int p = 0; p < PAIRS; ++p) {
        const int l = fix_leader(p, H), m = l ^ U;
        W[p] = fix_mul(re[l], re[m], S) + fix_mul(im[l], im[m], S);  // Re conj(a_l) a_m
      }
    }
    if (need & 2) {
#pragma unroll
      for (int p = 0; p < PAIRS; ++p) {
        const int l = fix_leader(p, H), m = l ^ U;
        W[PAIRS + p] = fix_mul(re[l], im[m], S) - fix_mul(im[l], re[m], S);  // Im conj(a_l) a_m
      }
    }
  }
}

__device__ __forceinline__ void fix_dispatch(int u, int need, const FixComp (&re)[1 << kFixD],
                                             const FixComp (&im)[1 << kFixD], long long (&W)[1 << kFixD], int S) {
  switch (u) {
    case 0: fix_products<0>(re, im, W, S, need); break;
    case 1: fix_products<1>(re, im, W, S, need); break;
    case 2: fix_products<2>(re, im, W, S, need); break;
    case 3: fix_products<3>(re, im, W, S, need); break;
    case 4: fix_products<4>(re, im, W, S, need); break;
    case 5: fix_products<5>(re, im, W, S, need); break;
    case 6: fix_products<6>(re, im, W, S, need); break;
    case 7: fix_products<7>(re, im, W, S, need); break;
    default: break;
  }
}

template <typename Idx>
__global__ void __launch_bounds__(kFixThreads)
    k_expval_fix(const float2 *__restrict__ amp, Idx n_cosets, const FixRunDev run,
                 const FixTermDev *__restrict__ gterms, int S, long long *__restrict__ partials) {
  constexpr int D = kFixD, E = 1 << D, PAIRS = E / 2, NV = kFixTerms + 1;
  __shared__ FixTermDev terms[kFixTerms];
  __shared__ Idx soff[E];
  // per-term accumulators, one column per thread (conflict-free 8-byte rows)
  __shared__ long long sacc[NV][kFixThreads];
  const int nt = run.nterms;
  if (threadIdx.x < nt) terms[threadIdx.x] = gterms[threadIdx.x];
  if (threadIdx.x < E) {
    uint64_t so = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) so ^= run.basis[b];
    soff[threadIdx.x] = (Idx)so;
  }
  for (int j = 0; j < NV; ++j) sacc[j][threadIdx.x] = 0;
  __syncthreads();
  long long nrm = 0;
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx c = (Idx)blockIdx.x * blockDim.x + threadIdx.x; c < n_cosets; c += stride) {
    Idx rep = c;
#pragma unroll
    for (int b = 0; b < D; ++b) {
      const int pv = run.piv[b];
      rep = ((rep >> pv) << (pv + 1)) | (rep & ((Idx(1) << pv) - 1));
    }
    FixComp re[E], im[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
      const float2 v = amp[rep ^ soff[l]];
      re[l] = fix_split(v.x);
      im[l] = fix_split(v.y);
    }
    if (run.with_norm) {
#pragma unroll
      for (int l = 0; l < E; ++l) nrm += fix_mul(re[l], re[l], S) + fix_mul(im[l], im[l], S);
    }
    long long W[E];
    int cur = -1;
    for (int j = 0; j < nt; ++j) {
      const FixTermDev t = terms[j];
      if (t.u != cur) {
        cur = t.u;
        fix_dispatch(t.u, t.need, re, im, W, S);
      }
      long long sum = 0;
      if (t.u == 0) {
#pragma unroll
        for (int l = 0; l < E; ++l) sum += ((t.psm >> l) & 1u) ? -W[l] : W[l];
      } else if (t.imag) {
#pragma unroll
        for (int q = 0; q < PAIRS; ++q) sum += ((t.psm >> q) & 1u) ? -W[PAIRS + q] : W[PAIRS + q];
      } else {
#pragma unroll
        for (int q = 0; q < PAIRS; ++q) sum += ((t.psm >> q) & 1u) ? -W[q] : W[q];
      }
      sacc[j][threadIdx.x] += parity((uint64_t)rep & t.z) ? -sum : sum;
    }
  }
  sacc[kFixTerms][threadIdx.x] = nrm;
  __syncthreads();
  // exact block sums: warp w reduces rows w, w + 8, ...
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int j = w; j < NV; j += (int)(blockDim.x >> 5)) {
    long long v = 0;
    for (int i = lane; i < (int)blockDim.x; i += 32) v += sacc[j][i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) partials[(size_t)blockIdx.x * NV + j] = v;
  }
}

// results[r][j] = sum over blocks of partials[r][b][j]; one CTA per run
__global__ void k_finish_fix(const long long *__restrict__ partials, int n_blocks, long long *__restrict__ results) {
  constexpr int NV = kFixTerms + 1;
  __shared__ long long red[kThreads / 32];
  const long long *p = partials + (size_t)blockIdx.x * n_blocks * NV;
  for (int j = 0; j < NV; ++j) {
    long long v = 0;
    for (int b = threadIdx.x; b < n_blocks; b += blockDim.x) v += p[(size_t)b * NV + j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
      long long t = 0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
      results[(size_t)blockIdx.x * NV + j] = t;
    }
    __syncthreads();
  }
}

// |a|^2 estimate in FP32 per thread, FP64 per block: only used to pick S
__global__ void __launch_bounds__(kThreads) k_norm_est(const float2 *__restrict__ amp, uint64_t n, double *out) {
  float acc = 0.f;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float2 v = amp[i];
    acc = fmaf(v.x, v.x, fmaf(v.y, v.y, acc));
  }
  double a = acc, b = 0.0;
  block_sum2(a, b);
  if (threadIdx.x == 0) out[blockIdx.x] = a;
}

struct FixRunHost {
  FixRunDev dev;
  std::vector<FixTermDev> terms;
  std::vector<double> coef;
};

// group by x (frame signs applied), chunk groups to <= kFixTerms, pack chunks
// into runs of <= kFixTerms terms whose x-masks span <= kFixD dimensions
void plan_fix(const sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
              std::vector<FixRunHost> &runs) {
  const Pauli &q = sv->frame;
  std::map<uint64_t, std::vector<Term>> by_x;
  for (size_t j = 0; j < count; ++j) {
    double cj = c[j];
    if (anticommute(x[j], z[j], q.x, q.z)) cj = -cj;
    by_x[x[j]].push_back({x[j], z[j], cj});
  }
  std::vector<std::vector<Term>> chunks;
  for (auto &kv : by_x)
    for (size_t a = 0; a < kv.second.size(); a += kFixTerms)
      chunks.emplace_back(kv.second.begin() + a,
                          kv.second.begin() + std::min(kv.second.size(), a + (size_t)kFixTerms));
  std::vector<char> used(chunks.size(), 0);
  size_t left = chunks.size();
  while (left > 0 || runs.empty()) {
    FixRunHost r;
    std::memset(&r.dev, 0, sizeof(r.dev));
    uint64_t basis[kFixD];
    int piv[kFixD];
    int d = 0;
    auto reduce = [&](uint64_t v) {
      for (int b = 0; b < d; ++b)
        if ((v >> piv[b]) & 1ULL) v ^= basis[b];
      return v;
    };
    auto add_vec = [&](uint64_t rr, uint64_t) {
      int pv = 63 - __builtin_clzll(rr);
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
    std::vector<size_t> members;
    size_t nterm = 0;
    for (size_t g = 0; g < chunks.size(); ++g) {
      if (used[g]) continue;
      if (nterm + chunks[g].size() > (size_t)kFixTerms) continue;
      uint64_t rr = reduce(chunks[g][0].x);
      if (rr != 0) {
        if (d >= kFixD) continue;
        add_vec(rr, 0);
      }
      used[g] = 1;
      --left;
      members.push_back(g);
      nterm += chunks[g].size();
      if (nterm == (size_t)kFixTerms) break;
    }
    // pad to kFixD with the highest unused bits
    uint64_t usedbits = 0;
    for (int b = 0; b < d; ++b) usedbits |= 1ULL << piv[b];
    for (int bit = sv->n - 1; bit >= 0 && d < kFixD; --bit)
      if (!((usedbits >> bit) & 1ULL)) {
        add_vec(1ULL << bit, 0);
        usedbits |= 1ULL << bit;
      }
    r.dev.d = d;
    for (int b = 0; b < d; ++b) {
      r.dev.basis[b] = basis[b];
      r.dev.piv[b] = piv[b];
    }
    // terms sorted by u so a run recomputes products only when u changes
    std::vector<std::pair<int, const Term *>> ts;
    for (size_t g : members)
      for (const Term &t : chunks[g]) {
        int u = 0;
        for (int b = 0; b < d; ++b)
          if ((t.x >> piv[b]) & 1ULL) u |= 1 << b;
        ts.push_back({u, &t});
      }
    std::stable_sort(ts.begin(), ts.end(), [](const auto &a1, const auto &b1) { return a1.first < b1.first; });
    std::map<int, int> need;
    for (auto &ut : ts) {
      const int ny = popc64(ut.second->x & ut.second->z) & 3;
      need[ut.first] |= ut.first == 0 ? 1 : ((ny & 1) ? 2 : 1);
    }
    for (auto &ut : ts) {
      const Term &t = *ut.second;
      const int u = ut.first;
      FixTermDev e;
      e.z = t.z;
      e.u = u;
      e.need = need[u];
      uint32_t psm = 0;
      auto sgn = [&](int l) {
        uint64_t so = 0;
        for (int b = 0; b < d; ++b)
          if ((l >> b) & 1) so ^= basis[b];
        return (uint32_t)(popc64(so & t.z) & 1);
      };
      const int ny = popc64(t.x & t.z) & 3;
      if (u == 0) {
        for (int l = 0; l < (1 << kFixD); ++l) psm |= sgn(l) << l;
        e.imag = 0;
        r.coef.push_back(t.c);
      } else {
        int H = 0;
        while (u >> (H + 1)) ++H;
        for (int p = 0; p < (1 << kFixD) / 2; ++p) psm |= sgn(fix_leader(p, H)) << p;
        e.imag = ny & 1;
        r.coef.push_back(2.0 * t.c * ((ny == 0 || ny == 1) ? 1.0 : -1.0));
      }
      e.psm = psm;
      r.terms.push_back(e);
    }
    r.dev.nterms = (int32_t)r.terms.size();
    r.dev.with_norm = runs.empty() ? 1 : 0;
    runs.push_back(std::move(r));
    if (left == 0) break;
  }
}

template <typename Idx>
int expval_fix_t(sv_state *sv, const std::vector<FixRunHost> &runs, double *energy, double *norm2) {
  constexpr int NV = kFixTerms + 1;
  static int cap = 0;
  if (!cap) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_expval_fix<Idx>, kFixThreads, 0) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    cap = (per_sm > 0 ? per_sm : 1) * device_sm_count();
  }
  const uint64_t n_amps = 1ULL << sv->n;
  const uint64_t n_cosets = n_amps >> kFixD;
  uint64_t need = (n_cosets + kFixThreads - 1) / kFixThreads;
  const int blocks = (int)(need < (uint64_t)cap ? (need ? need : 1) : cap);
  const int est_blocks = 64;
  // partial sums (int64) and the S estimate share the double scratch
  int rc = ensure_scratch(sv, (size_t)NV * blocks * runs.size() + est_blocks, NV * runs.size() + est_blocks);
  if (rc) return rc;
  // stage terms
  size_t bytes = 0;
  std::vector<size_t> off(runs.size());
  for (size_t r = 0; r < runs.size(); ++r) {
    off[r] = bytes;
    bytes += ((runs[r].terms.size() * sizeof(FixTermDev)) + 15) & ~size_t(15);
  }
  if (!bytes) bytes = 16;
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  rc = ensure_stage(sv, bytes);
  if (rc) return rc;
  for (size_t r = 0; r < runs.size(); ++r)
    if (!runs[r].terms.empty())
      std::memcpy((char *)sv->h_stage + off[r], runs[r].terms.data(), runs[r].terms.size() * sizeof(FixTermDev));
  PR_CUDA(cudaMemcpyAsync(sv->d_stage, sv->h_stage, bytes, cudaMemcpyHostToDevice, sv->stream));
  // choose S from an estimate of <a|a>
  double *est = sv->d_results + NV * runs.size();
  {
    const int tr = trace_begin(sv);
    k_norm_est<<<est_blocks, kThreads, 0, sv->stream>>>((const float2 *)sv->amps, n_amps, est);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_EXPVAL, 8.0 * (double)n_amps);
  }
  PR_CUDA(cudaMemcpyAsync(sv->h_results, est, est_blocks * sizeof(double), cudaMemcpyDeviceToHost, sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  double nest = 0.0;
  for (int i = 0; i < est_blocks; ++i) nest += sv->h_results[i];
  // S = 60 - ceil(log2 <a|a>) (estimate widened by 1 %): every per-term sum is
  // bounded by <a|a> 2^S <= 2^60 and no product needs a left shift
  int S = 60;
  if (nest * 1.01 > 1.0) S = 60 - (int)std::ceil(std::log2(nest * 1.01));
  if (S < 8) return fail(SV_EUNSUPPORTED, "state norm %g too large for the fixed-point sums", nest);
  long long *part = (long long *)sv->d_partials;
  long long *res = (long long *)sv->d_results;
  for (size_t r = 0; r < runs.size(); ++r) {
    const int tr = trace_begin(sv);
    k_expval_fix<Idx><<<blocks, kFixThreads, 0, sv->stream>>>(
        (const float2 *)sv->amps, (Idx)n_cosets, runs[r].dev, (const FixTermDev *)((char *)sv->d_stage + off[r]), S,
        part + (size_t)NV * blocks * r);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_EXPVAL, 8.0 * (double)n_amps);
  }
  {
    const int tr = trace_begin(sv);
    k_finish_fix<<<(unsigned)runs.size(), kThreads, 0, sv->stream>>>(part, blocks, res);
    PR_CHECK_LAUNCH();
    trace_end(sv, tr, KN_FINISH, 8.0 * NV * blocks * runs.size());
  }
  PR_CUDA(cudaMemcpyAsync(sv->h_results, res, NV * runs.size() * sizeof(long long), cudaMemcpyDeviceToHost,
                          sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  const long long *h = (const long long *)sv->h_results;
  const double unit = std::ldexp(1.0, -S);
  long double e = 0.0L;
  for (size_t r = 0; r < runs.size(); ++r)
    for (size_t j = 0; j < runs[r].coef.size(); ++j) e += (long double)runs[r].coef[j] * (long double)h[r * NV + j];
  if (energy) *energy = (double)(e * unit);
  if (norm2) *norm2 = (double)h[kFixTerms] * unit;
  return SV_OK;
}

}  // namespace

int expval_impl(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *c, size_t count,
                double *energy, double *norm2) {
  if (sv->dtype == SV_C64 && sv->n >= kFixD) {
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
  static int cap = 0;
  if (!cap) cap = occ_blocks(k_pauli_sum<R, Idx, D>);
  const uint64_t n_cosets = (1ULL << src->n) >> D;
  uint64_t need = (n_cosets + kThreads - 1) / kThreads;
  int blocks = (int)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (blocks < 1) blocks = 1;
  PR_CUDA(cudaMemsetAsync(dst->amps, 0, amp_bytes(dst->dtype) << dst->n, src->stream));
  for (size_t r = 0; r < runs.size(); ++r) {
    const int tr = trace_begin(src);
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
    case 3: return run_pauli_sum_t<R, Idx, 3>(dst, src, runs, dg, dt);
    default: return run_pauli_sum_t<R, Idx, kExpD>(dst, src, runs, dg, dt);
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
  void *scratch = nullptr;
  rc = na_device_scratch(&scratch);
  if (rc) return rc;
  std::lock_guard<std::mutex> lock(g_na_mutex);
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
