// Arithmetic-rate probes: the measured peaks of the pipes that bound the
// complex128 work (not in the paper; they give the rooflines of the passes a
// measured denominator instead of a nominal one).
//
// Each thread runs eight independent dependency chains of one operation for
// `iters` steps, so a grid that fills every SM keeps the pipe busy and the
// rate is operations / device time.  The chains' final values are written to
// `out` (one value per thread) so the work cannot be removed.
//   kind 0: FP64 fused multiply-add (the FP64 pipe)
//   kind 1: 32 x 32 -> 64-bit signed integer multiply-add (the wide integer
//           multiply the fixed-point passes are built from)
//   kind 2: packed FP32x2 fused multiply-add (the complex64 pair update)
#include "internal.h"

namespace pr {
namespace {

constexpr int kProbeChains = 8;

__global__ void __launch_bounds__(kThreads) k_probe_dfma(double *__restrict__ out, int iters, double a, double b) {
  double x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_imad(long long *__restrict__ out, int iters, int a) {
  long long x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = (long long)(threadIdx.x * 977 + c * 131);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (long long)(int)x[c] * a + x[c];
  }
  long long s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s ^= x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kThreads) k_probe_ffma2(float2 *__restrict__ out, int iters, float a, float b) {
  float2 x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = make_float2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
  const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
  }
  float2 s = make_float2(0.0f, 0.0f);
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s = make_float2(s.x + x[c].x, s.y + x[c].y);
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace pr

extern "C" int sv_probe_rate(int kind, int blocks, int iters, void *dev_out, void *cuda_stream, double *out_ops) {
  using namespace pr;
  clear_error();
  if (kind < 0 || kind > 2)
    return fail(SV_EINVAL, "probe kind must be 0 (FP64 FMA), 1 (wide integer multiply-add) or 2 (FP32x2 FMA)");
  if (blocks < 1 || iters < 1 || !dev_out) return fail(SV_EINVAL, "probe needs blocks >= 1, iters >= 1 and a buffer");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (kind == 0)
    k_probe_dfma<<<blocks, kThreads, 0, st>>>((double *)dev_out, iters, 0.9999999, 1e-7);
  else if (kind == 1)
    k_probe_imad<<<blocks, kThreads, 0, st>>>((long long *)dev_out, iters, 3);
  else
    k_probe_ffma2<<<blocks, kThreads, 0, st>>>((float2 *)dev_out, iters, 0.9999999f, 1e-7f);
  PR_CHECK_LAUNCH();
  if (out_ops) *out_ops = (double)blocks * kThreads * (double)iters * kProbeChains;
  return SV_OK;
}
