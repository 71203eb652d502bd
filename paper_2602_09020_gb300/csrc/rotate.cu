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

#include <mutex>

#include "coset_fx.cuh"
#include "kernels.cuh"

namespace pr {

namespace {

template <typename R, typename Idx, int D, int V>
__global__ void __launch_bounds__(kThreads)
    k_coset(typename Cx<R>::T *__restrict__ amp, Idx n_cosets, const __grid_constant__ RunDev run,
            const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz) {
  __shared__ __align__(16) char ws[ws_coset<R, Idx, D>()];
  body_coset<R, Idx, D, V>(amp, n_cosets, run, rots, fx, fz, (Idx)blockIdx.x, (Idx)gridDim.x, ws);
}

// complex128 runs in 64-bit fixed point on the integer pipes (coset_fx.cuh)
template <typename Idx, int D, int V>
__global__ void __launch_bounds__(kThreads)
    k_coset_fx(double2 *__restrict__ amp, Idx n_cosets, const __grid_constant__ RunDev run,
               const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz) {
  __shared__ __align__(16) char ws[ws_coset_fx<Idx, D>()];
  body_coset_fx<Idx, D, V>(amp, n_cosets, run, rots, fx, fz, (Idx)blockIdx.x, (Idx)gridDim.x, ws);
}

template <typename Idx, int D>
__global__ void __launch_bounds__(kThreads)
    k_coset_c64x2(float4 *__restrict__ amp4, Idx n_pairs, const __grid_constant__ RunDev run, const RotDev *__restrict__ rots,
                  uint64_t fx, uint64_t fz, int reverse) {
  extern __shared__ __align__(16) char dyn_ws[];
  body_c64x2<Idx, D>(amp4, n_pairs, run, rots, fx, fz, (Idx)blockIdx.x, (Idx)gridDim.x, dyn_ws, true, reverse != 0);
}

template <typename R, typename Idx>
__global__ void __launch_bounds__(kThreads, 3)
    k_diag_sum(typename Cx<R>::T *__restrict__ amp, Idx n_groups, const __grid_constant__ RunDev run,
               const DiagDev *__restrict__ rots, uint64_t fx, const typename Cx<R>::T *__restrict__ tab) {
  __shared__ __align__(16) char ws[ws_diag<R, Idx>()];
  body_diag<R, Idx>(amp, n_groups, run, rots, fx, tab, (Idx)blockIdx.x, (Idx)gridDim.x, ws);
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
  static const int cap = occupancy_blocks(k_coset<R, Idx, D, V>, kThreads);
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + (uint64_t)kThreads * V - 1) / ((uint64_t)kThreads * V);
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv, KN_COSET0 + D);
  k_coset<R, Idx, D, V><<<blocks, kThreads, 0, sv->stream>>>((C *)sv->amps, (Idx)n_cosets, run,
                                                             plan->d_rots, fx, fz);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_COSET0 + D, 2.0 * (double)sizeof(C) * (double)(1ULL << sv->n),
            4.0 * (double)run.count * (double)(1ULL << sv->n));
  return SV_OK;
}

template <typename Idx, int D, int V>
int launch_coset_fx_t(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  static const int cap = occupancy_blocks(k_coset_fx<Idx, D, V>, kThreads);
  const uint64_t n_cosets = (1ULL << sv->n) >> D;
  uint64_t need = (n_cosets + (uint64_t)kThreads * V - 1) / ((uint64_t)kThreads * V);
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv, KN_COSET0 + D);
  k_coset_fx<Idx, D, V><<<blocks, kThreads, 0, sv->stream>>>((double2 *)sv->amps, (Idx)n_cosets, run,
                                                             plan->d_rots, fx, fz);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_COSET0 + D, 2.0 * 16.0 * (double)(1ULL << sv->n),
            4.0 * (double)run.count * (double)(1ULL << sv->n));
  return SV_OK;
}

template <typename Idx>
int launch_coset_fx_d(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  switch (run.d) {
    case 0: return launch_coset_fx_t<Idx, 0, 2>(sv, plan, run, fx, fz);
    case 1: return launch_coset_fx_t<Idx, 1, 1>(sv, plan, run, fx, fz);
    case 2: return launch_coset_fx_t<Idx, 2, 1>(sv, plan, run, fx, fz);
    case 3: return launch_coset_fx_t<Idx, 3, 1>(sv, plan, run, fx, fz);
    case 4: return launch_coset_fx_t<Idx, 4, 1>(sv, plan, run, fx, fz);
    case 5: return launch_coset_fx_t<Idx, 5, 1>(sv, plan, run, fx, fz);
    default: return fail(SV_EINVAL, "run dimension %d out of range", run.d);
  }
}

template <typename Idx, int D>
int launch_c64x2_t(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  const size_t dyn = ws_c64x2<Idx, D>();
  // computed once, on first use (thread-safe static initialisation); -1 if the
  // kernel's shared-memory size cannot be set
  static const int cap = [] {
    const size_t bytes = ws_c64x2<Idx, D>();
    if (cudaFuncSetAttribute(k_coset_c64x2<Idx, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_coset_c64x2<Idx, D>, kThreads, bytes) != cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    return (per_sm > 0 ? per_sm : 1) * device_sm_count();
  }();
  if (cap < 0) return fail(SV_ECUDA, "cannot set the shared-memory size of the packed pass");
  const uint64_t n_pairs = ((1ULL << sv->n) >> D) >> 1;
  uint64_t need = (n_pairs + kThreads - 1) / kThreads;
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv, KN_COSET0 + D);
  // programmatic dependent launch: the grid never exceeds what the GPU holds at
  // once, so the early-scheduled CTAs of this pass cannot keep the previous
  // pass's CTAs from running, and each waits for that pass before touching
  // amplitudes (griddepcontrol.wait in body_c64x2)
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = sv->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  // consecutive packed passes on a state walk the cosets in opposite
  // directions: the next pass starts where the previous one ended (in L2)
  const int reverse = (int)(sv->packed_passes++ & 1u);
  PR_CUDA(cudaLaunchKernelEx(&cfg, k_coset_c64x2<Idx, D>, (float4 *)sv->amps, (Idx)n_pairs, run,
                             (const RotDev *)plan->d_rots, fx, fz, reverse));
  trace_end(sv, tr, KN_COSET0 + D, 2.0 * 8.0 * (double)(1ULL << sv->n),
            4.0 * (double)run.count * (double)(1ULL << sv->n));
  return SV_OK;
}

// the packed complex64 pass applies when bit 0 is not a pivot and there are
// at least two cosets; d = 5 keeps the one-coset kernel (register budget)
template <typename Idx>
int launch_c64x2_d(sv_state *sv, const sv_plan *plan, const RunDev &run, uint64_t fx, uint64_t fz) {
  switch (run.d) {
    case 0: return launch_c64x2_t<Idx, 0>(sv, plan, run, fx, fz);
    case 1: return launch_c64x2_t<Idx, 1>(sv, plan, run, fx, fz);
    case 2: return launch_c64x2_t<Idx, 2>(sv, plan, run, fx, fz);
    case 3: return launch_c64x2_t<Idx, 3>(sv, plan, run, fx, fz);
    case 4: return launch_c64x2_t<Idx, 4>(sv, plan, run, fx, fz);
    default: return fail(SV_EINVAL, "packed pass: dimension %d", run.d);
  }
}

bool use_c64x2(const sv_state *sv, const RunDev &run) {
  if (sv->dtype != SV_C64 || run.d > 4 || sv->n - run.d < 1) return false;
  return run.d == 0 || run.piv[0] >= 1;
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

std::mutex g_tab_mu;

int ensure_tables(int dev, int dtype, const void **out) {
  if (dev < 0 || dev >= kMaxDevices) return fail(SV_EUNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lk(g_tab_mu);
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
  static const int cap = occupancy_blocks(k_diag_sum<R, Idx>, kThreads);
  const uint64_t n_groups = (1ULL << sv->n) >> kDiagClassBits;
  uint64_t need = (n_groups + kThreads - 1) / kThreads;
  unsigned blocks = (unsigned)(need < (uint64_t)cap ? need : (uint64_t)cap);
  if (!blocks) blocks = 1;
  const int tr = trace_begin(sv, KN_DIAG_SUM);
  k_diag_sum<R, Idx><<<blocks, kThreads, 0, sv->stream>>>((C *)sv->amps, (Idx)n_groups, run, plan->d_diag,
                                                          fx, (const C *)tab);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_DIAG_SUM, 2.0 * (double)sizeof(C) * (double)(1ULL << sv->n));
  return SV_OK;
}

}  // namespace

int table_pointer(int dtype, const void **out) {
  int dev = 0;
  PR_CUDA(cudaGetDevice(&dev));
  return ensure_tables(dev, dtype, out);
}

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
    if (run.count > kMaxDiagRots || run.seg[1 << kDiagClassBits] > kDiagSlots)
      return fail(SV_EINVAL, "diagonal run exceeds %d rotations or %d z patterns", kMaxDiagRots, kDiagSlots);
    if (sv->dtype == SV_C128)
      return narrow ? launch_diag_t<double, uint32_t>(sv, plan, run, fx)
                    : launch_diag_t<double, uint64_t>(sv, plan, run, fx);
    return narrow ? launch_diag_t<float, uint32_t>(sv, plan, run, fx)
                  : launch_diag_t<float, uint64_t>(sv, plan, run, fx);
  }
  if (run.d > sv->n) return fail(SV_EINVAL, "run dimension exceeds n");
  if (use_c64x2(sv, run))
    return narrow ? launch_c64x2_d<uint32_t>(sv, plan, run, fx, fz) : launch_c64x2_d<uint64_t>(sv, plan, run, fx, fz);
  if (sv->dtype == SV_C128)
    return narrow ? launch_coset_fx_d<uint32_t>(sv, plan, run, fx, fz)
                  : launch_coset_fx_d<uint64_t>(sv, plan, run, fx, fz);
  return narrow ? launch_coset_d<float, uint32_t>(sv, plan, run, fx, fz)
                : launch_coset_d<float, uint64_t>(sv, plan, run, fx, fz);
}

}  // namespace pr
