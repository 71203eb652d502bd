// Rotation kernels.
//
// k_coset: one HBM pass applies a run of consecutive rotations whose x-masks
// span a subspace S of dimension d <= 5.  The index space splits into cosets
// {rep ^ s : s in S}; each thread loads whole cosets into registers, applies
// every rotation of the run to them in list order and writes them back.  A
// rotation about P pairs amplitude k with f_P(k) = k ^ x (paper, Sec.
// "Multi-qubit rotations in a fullstate simulator": f_P is an involution) and
// both elements of a pair lie in one coset, so no data leaves the thread.
// The 2x2 pair update of the paper's appendix ("Amplitude update rule") is
// applied in tan form (see plan.cu): a_k += t * kappa * (-1)^{popc(k&z)} *
// a_{k^x} with kappa = (-i)^{nY+1}, two fused multiply-adds per real amplitude.
// d = 0 is the per-element diagonal case (f_P(k) = k); d = 1 with one rotation
// is the plain single-rotation pair pass.
//
// k_diag_sum: a run of r diagonal (I/Z-only) rotations multiplies amplitude k
// by exp(-i sum_j (theta_j/2) (-1)^{popc(k & z_j)}) (appendix, diagonal case,
// with even parity taking e^{-i theta/2} as R_P = cos - i sin P requires).  The
// angle sum is exact in 64-bit fixed point (turns / 2^64); a thread owns 16
// amplitudes that differ in index bits 5..8 and resolves their 16 sign
// patterns with one 16-point Walsh-Hadamard transform of per-class partial
// sums, so the per-rotation work is per thread, not per amplitude.  The phase
// e^{i Phi} comes from two 256-entry tables (top 16 bits of Phi) and a short
// Taylor step for the remaining angle below 2 pi / 2^16.
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

__device__ __forceinline__ int parity(uint32_t v) { return __popc(v) & 1; }
__device__ __forceinline__ int parity(uint64_t v) { return __popcll(v) & 1; }

template <typename R, typename Idx>
struct RotSm {
  Idx z;
  uint32_t zt;
  uint32_t code;
  R t;
};

// Apply one rotation with coset coordinates U (compile-time) to V cosets of
// 2^D elements.  tp[v] is t times the sign (-1)^{popc(rep_v & z)}; bit l of zt
// adds the sign of coset element l.
template <int D, int V, int U, int IMAG, typename R, typename C>
__device__ __forceinline__ void apply_u(C (&a)[V][1 << D], const R (&tp)[V], uint32_t zt) {
#pragma unroll
  for (int v = 0; v < V; ++v) {
#pragma unroll
    for (int l = 0; l < (1 << D); ++l) {
      if (U == 0) {
        const R t = ((zt >> l) & 1u) ? -tp[v] : tp[v];
        const C x = a[v][l];
        a[v][l].x = x.x - t * x.y;
        a[v][l].y = x.y + t * x.x;
      } else if ((l ^ U) > l) {
        const int m = l ^ U;
        const R tl = ((zt >> l) & 1u) ? -tp[v] : tp[v];
        const R tm = IMAG ? tl : -tl;
        const C al = a[v][l], am = a[v][m];
        if (IMAG) {
          a[v][l].x = al.x - tl * am.y;
          a[v][l].y = al.y + tl * am.x;
          a[v][m].x = am.x - tm * al.y;
          a[v][m].y = am.y + tm * al.x;
        } else {
          a[v][l].x = al.x + tl * am.x;
          a[v][l].y = al.y + tl * am.y;
          a[v][m].x = am.x + tm * al.x;
          a[v][m].y = am.y + tm * al.y;
        }
      }
    }
  }
}

#define PR_CASE(K)                                                                 \
  case K:                                                                          \
    if constexpr ((((K) >> 1) < (1 << D)) && ((((K) >> 1) != 0) || ((K)&1)))       \
      apply_u<D, V, ((K) >> 1), ((K)&1)>(a, tp, zt);                               \
    break;
#define PR_CASE8(B) \
  PR_CASE(B + 0) PR_CASE(B + 1) PR_CASE(B + 2) PR_CASE(B + 3) PR_CASE(B + 4) PR_CASE(B + 5) PR_CASE(B + 6) PR_CASE(B + 7)

template <int D, int V, typename R, typename C>
__device__ __forceinline__ void dispatch(uint32_t code, C (&a)[V][1 << D], const R (&tp)[V], uint32_t zt) {
  switch (code) {
    PR_CASE8(0)
    PR_CASE8(8)
    PR_CASE8(16)
    PR_CASE8(24)
    PR_CASE8(32)
    PR_CASE8(40)
    PR_CASE8(48)
    PR_CASE8(56)
    default:
      break;
  }
}

template <typename R, typename Idx, int D, int V>
__global__ void __launch_bounds__(kThreads)
    k_coset(typename Cx<R>::T *__restrict__ amp, Idx n_cosets, const RunDev run,
            const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz) {
  using C = typename Cx<R>::T;
  constexpr int E = 1 << D;
  __shared__ RotSm<R, Idx> srot[kMaxRunRots];
  __shared__ Idx soff[E];
  const int count = run.count;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const RotDev r = rots[run.first + j];
    double t = r.t;
    if (__popcll((r.x & fz) ^ (r.z & fx)) & 1) t = -t;  // runtime frame sign
    RotSm<R, Idx> s;
    s.z = (Idx)r.z;
    s.zt = r.zt;
    s.code = r.code;
    s.t = (R)t;
    srot[j] = s;
  }
  if (threadIdx.x < E) {
    uint64_t s = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) s ^= run.basis[b];
    soff[threadIdx.x] = (Idx)s;
  }
  __syncthreads();

  const Idx chunk = (Idx)blockDim.x * V;
  const Idx stride = (Idx)gridDim.x * chunk;
  for (Idx c0 = (Idx)blockIdx.x * chunk + threadIdx.x; c0 < n_cosets; c0 += stride) {
    C a[V][E];
    Idx rep[V];
    bool ok[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const Idx c = c0 + (Idx)(v * blockDim.x);
      Idx r = c;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        const int p = run.piv[b];
        r = ((r >> p) << (p + 1)) | (r & ((Idx(1) << p) - 1));
      }
      rep[v] = r;
      ok[v] = c < n_cosets;
#pragma unroll
      for (int l = 0; l < E; ++l) {
        if (ok[v]) {
          a[v][l] = amp[r ^ soff[l]];
        } else {
          a[v][l].x = 0;
          a[v][l].y = 0;
        }
      }
    }
    for (int j = 0; j < count; ++j) {
      const RotSm<R, Idx> s = srot[j];
      R tp[V];
#pragma unroll
      for (int v = 0; v < V; ++v) tp[v] = parity(rep[v] & s.z) ? -s.t : s.t;
      dispatch<D, V>(s.code, a, tp, s.zt);
    }
    if (run.fold) {
      const R fr = (R)run.fold_re, fi = (R)run.fold_im;
#pragma unroll
      for (int v = 0; v < V; ++v)
#pragma unroll
        for (int l = 0; l < E; ++l) {
          const C x = a[v][l];
          a[v][l].x = fr * x.x - fi * x.y;
          a[v][l].y = fr * x.y + fi * x.x;
        }
    }
#pragma unroll
    for (int v = 0; v < V; ++v)
      if (ok[v]) {
#pragma unroll
        for (int l = 0; l < E; ++l) amp[rep[v] ^ soff[l]] = a[v][l];
      }
  }
}

// ------------------------------------------------------------------ diagonal phase sums

constexpr int kCls = 1 << kDiagClassBits;  // 16 amplitudes per thread

template <typename R>
__device__ __forceinline__ typename Cx<R>::T cmul(typename Cx<R>::T a, typename Cx<R>::T b) {
  typename Cx<R>::T o;
  o.x = a.x * b.x - a.y * b.y;
  o.y = a.x * b.y + a.y * b.x;
  return o;
}

// e^{i 2 pi phi / 2^64}
template <typename R>
__device__ __forceinline__ typename Cx<R>::T turn_phase(uint64_t phi, const typename Cx<R>::T *tab) {
  using C = typename Cx<R>::T;
  const C t0 = tab[phi >> 56];
  const C t1 = tab[256 + ((phi >> 48) & 255u)];
  const uint64_t rem = phi & ((1ULL << 48) - 1ULL);
  C s;
  if (sizeof(R) == 8) {
    const double x = (double)rem * 3.4061215800865545e-19;  // 2 pi / 2^64
    const double x2 = x * x;
    s.x = (R)fma(-0.5, x2, 1.0);
    s.y = (R)fma(x2 * (-1.0 / 6.0), x, x);
  } else {
    const float x = (float)rem * 3.40612158e-19f;
    s.x = fmaf(-0.5f * x, x, 1.0f);
    s.y = x;
  }
  return cmul<R>(cmul<R>(t0, t1), s);
}

template <typename R, typename Idx>
__global__ void __launch_bounds__(kThreads)
    k_diag_sum(typename Cx<R>::T *__restrict__ amp, Idx n_groups, const RunDev run,
               const DiagDev *__restrict__ rots, uint64_t fx, const typename Cx<R>::T *__restrict__ tab) {
  using C = typename Cx<R>::T;
  __shared__ Idx sz[kMaxDiagRots];
  __shared__ uint64_t sa[kMaxDiagRots];
  __shared__ C stab[512];
  const int count = run.count;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const DiagDev r = rots[run.first + j];
    sz[j] = (Idx)r.z;
    sa[j] = (__popcll(r.z & fx) & 1) ? (0ULL - r.a) : r.a;  // runtime frame sign
  }
  for (int j = threadIdx.x; j < 512; j += blockDim.x) stab[j] = tab[j];
  __syncthreads();
  const Idx stride = (Idx)gridDim.x * blockDim.x;
  for (Idx g = (Idx)blockIdx.x * blockDim.x + threadIdx.x; g < n_groups; g += stride) {
    const Idx base = (g & (Idx)((1u << kDiagClassLo) - 1u)) |
                     ((g >> kDiagClassLo) << (kDiagClassLo + kDiagClassBits));
    uint64_t acc[kCls];
#pragma unroll
    for (int c = 0; c < kCls; ++c) {
      uint64_t s = 0;
      const int j1 = run.seg[c + 1];
      for (int j = run.seg[c]; j < j1; ++j) {
        const uint64_t a = sa[j];
        s += parity(base & sz[j]) ? (0ULL - a) : a;
      }
      acc[c] = s;
    }
    // acc[e] <- sum_c (-1)^{popc(e & c)} acc[c]
#pragma unroll
    for (int h = 1; h < kCls; h <<= 1)
#pragma unroll
      for (int i = 0; i < kCls; ++i)
        if (!(i & h)) {
          const uint64_t u = acc[i], w = acc[i + h];
          acc[i] = u + w;
          acc[i + h] = u - w;
        }
#pragma unroll
    for (int e = 0; e < kCls; ++e) {
      const Idx k = base | ((Idx)e << kDiagClassLo);
      C ph = turn_phase<R>(0ULL - acc[e], stab);  // exp(-i sum_j s_j theta_j / 2)
      if (run.fold) {
        C f;
        f.x = (R)run.fold_re;
        f.y = (R)run.fold_im;
        ph = cmul<R>(ph, f);
      }
      amp[k] = cmul<R>(amp[k], ph);
    }
  }
}

// ------------------------------------------------------------------ launch helpers

template <typename K>
int occupancy_blocks(K kernel, int threads) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return (per_sm > 0 ? per_sm : 1) * device_sm_count();
}

template <typename R, typename Idx, int D, int V>
int launch_coset_t(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  using C = typename Cx<R>::T;
  static int cap = 0;
  if (!cap) cap = occupancy_blocks(k_coset<R, Idx, D, V>, kThreads);
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + (uint64_t)kThreads * V - 1) / ((uint64_t)kThreads * V);
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv);
  k_coset<R, Idx, D, V><<<blocks, kThreads, 0, sv->stream>>>((C *)sv->amps, (Idx)n_cosets, run,
                                                             plan->d_rots, fx, fz);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_COSET0 + D, 2.0 * (double)sizeof(C) * (double)(1ULL << sv->n));
  return SV_OK;
}

template <typename R, typename Idx>
int launch_coset_d(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  constexpr bool dbl = sizeof(R) == 8;
  switch (run.d) {
    case 0: return launch_coset_t<R, Idx, 0, dbl ? 2 : 4>(sv, plan, run, fx, fz);
    case 1: return launch_coset_t<R, Idx, 1, dbl ? 1 : 2>(sv, plan, run, fx, fz);
    case 2: return launch_coset_t<R, Idx, 2, 1>(sv, plan, run, fx, fz);
    case 3: return launch_coset_t<R, Idx, 3, 1>(sv, plan, run, fx, fz);
    case 4: return launch_coset_t<R, Idx, 4, 1>(sv, plan, run, fx, fz);
    case 5: return launch_coset_t<R, Idx, 5, 1>(sv, plan, run, fx, fz);
    default: return fail(SV_EINVAL, "run dimension %d out of range", run.d);
  }
}

// phase tables: e^{2 pi i k/256} and e^{2 pi i k/65536}, per device and precision
constexpr int kMaxDevices = 64;
void *g_tab[kMaxDevices][2];

int ensure_tables(int dev, int dtype, const void **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SV_EUNSUPPORTED, "device index %d", dev);
  const int slot = dtype == SV_C128 ? 0 : 1;
  if (!g_tab[dev][slot]) {
    const double two_pi = 6.283185307179586476925286766559;
    if (dtype == SV_C128) {
      double2 h[512];
      for (int k = 0; k < 256; ++k) {
        long double a0 = (long double)two_pi * k / 256.0L, a1 = (long double)two_pi * k / 65536.0L;
        h[k] = make_double2((double)cosl(a0), (double)sinl(a0));
        h[256 + k] = make_double2((double)cosl(a1), (double)sinl(a1));
      }
      void *d = nullptr;
      PR_CUDA(cudaMalloc(&d, sizeof(h)));
      PR_CUDA(cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice));
      g_tab[dev][slot] = d;
    } else {
      float2 h[512];
      for (int k = 0; k < 256; ++k) {
        long double a0 = (long double)two_pi * k / 256.0L, a1 = (long double)two_pi * k / 65536.0L;
        h[k] = make_float2((float)cosl(a0), (float)sinl(a0));
        h[256 + k] = make_float2((float)cosl(a1), (float)sinl(a1));
      }
      void *d = nullptr;
      PR_CUDA(cudaMalloc(&d, sizeof(h)));
      PR_CUDA(cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice));
      g_tab[dev][slot] = d;
    }
  }
  *out = g_tab[dev][slot];
  return SV_OK;
}

template <typename R, typename Idx>
int launch_diag_t(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx) {
  using C = typename Cx<R>::T;
  const void *tab = nullptr;
  int rc = ensure_tables(sv->device, sv->dtype, &tab);
  if (rc) return rc;
  static int cap = 0;
  if (!cap) cap = occupancy_blocks(k_diag_sum<R, Idx>, kThreads);
  const uint64_t n_groups = (1ULL << sv->n) >> kDiagClassBits;
  uint64_t need = (n_groups + kThreads - 1) / kThreads;
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv);
  k_diag_sum<R, Idx><<<blocks, kThreads, 0, sv->stream>>>((C *)sv->amps, (Idx)n_groups, run, plan->d_diag,
                                                          fx, (const C *)tab);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_DIAG_SUM, 2.0 * (double)sizeof(C) * (double)(1ULL << sv->n));
  return SV_OK;
}

}  // namespace

int prepare_tables(int dtype) {
  int dev = 0;
  PR_CUDA(cudaGetDevice(&dev));
  const void *t = nullptr;
  return ensure_tables(dev, dtype, &t);
}

int launch_run(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  const bool narrow = sv->n <= 31;
  if (run.kind == 1) {
    if (sv->n < kDiagMinQubits) return fail(SV_EINVAL, "diagonal run needs n >= %d", kDiagMinQubits);
    if (sv->dtype == SV_C128)
      return narrow ? launch_diag_t<double, uint32_t>(sv, plan, run, fx)
                    : launch_diag_t<double, uint64_t>(sv, plan, run, fx);
    return narrow ? launch_diag_t<float, uint32_t>(sv, plan, run, fx)
                  : launch_diag_t<float, uint64_t>(sv, plan, run, fx);
  }
  if (run.d > sv->n) return fail(SV_EINVAL, "run dimension exceeds n");
  if (sv->dtype == SV_C128)
    return narrow ? launch_coset_d<double, uint32_t>(sv, plan, run, fx, fz)
                  : launch_coset_d<double, uint64_t>(sv, plan, run, fx, fz);
  return narrow ? launch_coset_d<float, uint32_t>(sv, plan, run, fx, fz)
                : launch_coset_d<float, uint64_t>(sv, plan, run, fx, fz);
}

}  // namespace pr
