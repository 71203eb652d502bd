// Statevector handles, the Pauli frame, host<->device copies and the small
// single-pass kernels (basis state, frame materialisation).
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace pr {

static thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_err[0] = 0; }

int device_sm_count() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
  return sms > 0 ? sms : 1;
}

int ensure_scratch(sv_state *sv, size_t partial_doubles, size_t result_doubles) {
  if (partial_doubles > sv->partials_cap) {
    if (sv->d_partials) cudaFree(sv->d_partials);
    sv->d_partials = nullptr;
    sv->partials_cap = 0;
    size_t want = partial_doubles < 4096 ? 4096 : partial_doubles;
    if (cudaMalloc(&sv->d_partials, want * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "scratch allocation of %zu bytes failed", want * sizeof(double));
    }
    sv->partials_cap = want;
  }
  if (result_doubles > sv->results_cap) {
    if (sv->d_results) cudaFree(sv->d_results);
    sv->d_results = nullptr;
    sv->results_cap = 0;
    size_t want = result_doubles < 1024 ? 1024 : result_doubles;
    if (cudaMalloc(&sv->d_results, want * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "result allocation failed");
    }
    sv->results_cap = want;
  }
  if (result_doubles > sv->h_results_cap) {
    if (sv->h_results) cudaFreeHost(sv->h_results);
    sv->h_results = nullptr;
    sv->h_results_cap = 0;
    size_t want = result_doubles < 1024 ? 1024 : result_doubles;
    if (cudaMallocHost(&sv->h_results, want * sizeof(double)) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "pinned result allocation failed");
    }
    sv->h_results_cap = want;
  }
  return SV_OK;
}

int ensure_stage(sv_state *sv, size_t bytes) {
  if (bytes > sv->stage_cap) {
    if (sv->d_stage) cudaFree(sv->d_stage);
    sv->d_stage = nullptr;
    sv->stage_cap = 0;
    size_t want = bytes < (1 << 16) ? (1 << 16) : bytes;
    if (cudaMalloc(&sv->d_stage, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "staging allocation failed");
    }
    sv->stage_cap = want;
  }
  if (bytes > sv->h_stage_cap) {
    if (sv->h_stage) cudaFreeHost(sv->h_stage);
    sv->h_stage = nullptr;
    sv->h_stage_cap = 0;
    size_t want = bytes < (1 << 16) ? (1 << 16) : bytes;
    if (cudaMallocHost(&sv->h_stage, want) != cudaSuccess) {
      cudaGetLastError();
      return fail(SV_ENOMEM, "pinned staging allocation failed");
    }
    sv->h_stage_cap = want;
  }
  return SV_OK;
}

// ---------------------------------------------------------------- small kernels

template <typename C>
__global__ void k_set_one(C *amp, uint64_t k) {
  C one;
  one.x = 1;
  one.y = 0;
  amp[k] = one;
}

// |phi> <- i^q X^x Z^z |phi>: out_k = i^q (-1)^{popc(z & (k^x))} phi_{k^x}, done
// pairwise in place over k < k^x (or per element when x = 0).
// flip the sign bit of v when neg (an integer operation: no FP pipe, exact)
__device__ __forceinline__ float sign_flip(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ (neg ? (int)0x80000000 : 0));
}
__device__ __forceinline__ double sign_flip(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}

// out = i^q (-1)^{popc(k & z)} a: a swap and sign flips, exact
template <typename R, typename C>
__device__ __forceinline__ C phase_apply(C a, bool swap, bool negx, bool negy, bool s) {
  C o;
  o.x = sign_flip(swap ? a.y : a.x, negx != s);
  o.y = sign_flip(swap ? a.x : a.y, negy != s);
  return o;
}

template <typename R, typename C>
__global__ void k_materialize(C *amp, uint64_t n_amps, uint64_t x, uint64_t z, int q) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  // i^q: q = 1 maps (re, im) to (-im, re), q = 2 to (-re, -im), q = 3 to (im, -re)
  const bool swap = q & 1, negx = q == 1 || q == 2, negy = q == 2 || q == 3;
  const int h = x ? 63 - __clzll((long long)x) : -1;
  const uint64_t work = x ? n_amps >> 1 : n_amps;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < work; t += stride) {
    if (x == 0) {
      amp[t] = phase_apply<R>(amp[t], swap, negx, negy, __popcll(t & z) & 1);
    } else {
      uint64_t k = ((t >> h) << (h + 1)) | (t & ((1ULL << h) - 1));
      uint64_t m = k ^ x;
      const C a = amp[k], b = amp[m];
      amp[k] = phase_apply<R>(b, swap, negx, negy, __popcll(z & m) & 1);  // out_k from phi_m
      amp[m] = phase_apply<R>(a, swap, negx, negy, __popcll(z & k) & 1);  // out_m from phi_k
    }
  }
}

static unsigned grid_for(uint64_t work) {
  uint64_t blocks = (work + kThreads - 1) / kThreads;
  uint64_t cap = (uint64_t)device_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  return blocks ? (unsigned)blocks : 1u;
}

int launch_set_basis(sv_state *sv, uint64_t k) {
  size_t bytes = amp_bytes(sv->dtype) << sv->n;
  PR_CUDA(cudaMemsetAsync(sv->amps, 0, bytes, sv->stream));
  const int tr = trace_begin(sv, KN_SET_BASIS);
  if (sv->dtype == SV_C128)
    k_set_one<double2><<<1, 1, 0, sv->stream>>>((double2 *)sv->amps, k);
  else
    k_set_one<float2><<<1, 1, 0, sv->stream>>>((float2 *)sv->amps, k);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_SET_BASIS, 0.0);
  return SV_OK;
}

int launch_materialize(sv_state *sv, uint64_t x, uint64_t z, int q) {
  uint64_t n_amps = 1ULL << sv->n;
  unsigned g = grid_for(x ? n_amps / 2 : n_amps);
  const int tr = trace_begin(sv, KN_MATERIALIZE);
  if (sv->dtype == SV_C128)
    k_materialize<double, double2><<<g, kThreads, 0, sv->stream>>>((double2 *)sv->amps, n_amps, x, z, q);
  else
    k_materialize<float, float2><<<g, kThreads, 0, sv->stream>>>((float2 *)sv->amps, n_amps, x, z, q);
  PR_CHECK_LAUNCH();
  trace_end(sv, tr, KN_MATERIALIZE, 2.0 * (double)amp_bytes(sv->dtype) * (double)n_amps);
  return SV_OK;
}

int validate_masks(int n, const uint64_t *x, const uint64_t *z, size_t count) {
  const uint64_t bad = n >= 64 ? 0 : ~((1ULL << n) - 1ULL);
  for (size_t j = 0; j < count; ++j)
    if ((x[j] | z[j]) & bad)
      return fail(SV_EINVAL, "Pauli string %zu has a mask bit >= n = %d", j, n);
  return SV_OK;
}

}  // namespace pr

using namespace pr;

// ---------------------------------------------------------------- C ABI

extern "C" {

const char *sv_last_error(void) { return g_err; }

int sv_version(void) { return (1 << 16) | 0; }

static int make_state(sv_state **out, void *dev, int n, int dtype, void *stream, bool alloc) {
  if (!out) return fail(SV_EINVAL, "out is NULL");
  *out = nullptr;
  if (dtype != SV_C128 && dtype != SV_C64) return fail(SV_EINVAL, "dtype must be SV_C128 or SV_C64");
  if (n < 1) return fail(SV_EINVAL, "n_qubits must be >= 1");
  if (n > max_qubits(dtype))
    return fail(SV_ENOMEM, "n_qubits = %d exceeds the limit %d for this dtype", n, max_qubits(dtype));
  sv_state *sv = new (std::nothrow) sv_state();
  if (!sv) return fail(SV_ENOMEM, "host allocation failed");
  sv->n = n;
  sv->dtype = dtype;
  sv->stream = (cudaStream_t)stream;
  if (cudaGetDevice(&sv->device) != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return fail(SV_ECUDA, "no CUDA device");
  }
  size_t bytes = amp_bytes(dtype) << n;
  if (alloc) {
    if (cudaMalloc(&sv->amps, bytes) != cudaSuccess) {
      cudaGetLastError();
      delete sv;
      return fail(SV_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    sv->owns = true;
    int rc = launch_set_basis(sv, 0);
    if (rc) {
      cudaFree(sv->amps);
      delete sv;
      return rc;
    }
  } else {
    if (!dev) {
      delete sv;
      return fail(SV_EINVAL, "dev_amps is NULL");
    }
    if (((uintptr_t)dev) & 15) {
      delete sv;
      return fail(SV_EINVAL, "dev_amps must be 16-byte aligned");
    }
    sv->amps = dev;
  }
  *out = sv;
  return SV_OK;
}

int sv_alloc(sv_state **out, int n_qubits, int dtype, void *cuda_stream) {
  return make_state(out, nullptr, n_qubits, dtype, cuda_stream, true);
}

int sv_wrap(sv_state **out, void *dev_amps, int n_qubits, int dtype, void *cuda_stream) {
  return make_state(out, dev_amps, n_qubits, dtype, cuda_stream, false);
}

int sv_free(sv_state *sv) {
  if (!sv) return SV_OK;
  batch_forget(sv, nullptr);
  if (sv->stream) cudaStreamSynchronize(sv->stream);
  else cudaDeviceSynchronize();
  for (sv_state *&w : sv->work) {
    sv_free(w);
    w = nullptr;
  }
  if (sv->owns && sv->amps) cudaFree(sv->amps);
  if (sv->d_partials) cudaFree(sv->d_partials);
  if (sv->d_results) cudaFree(sv->d_results);
  if (sv->h_results) cudaFreeHost(sv->h_results);
  if (sv->d_stage) cudaFree(sv->d_stage);
  if (sv->h_stage) cudaFreeHost(sv->h_stage);
  if (sv->d_rec) cudaFree(sv->d_rec);
  if (sv->h_rec) cudaFreeHost(sv->h_rec);
  if (sv->rec_copied) cudaEventDestroy(sv->rec_copied);
  if (sv->rec_done) cudaEventDestroy(sv->rec_done);
  trace_release(sv);
  delete sv;
  return SV_OK;
}

int sv_set_stream(sv_state *sv, void *cuda_stream) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  sv->stream = (cudaStream_t)cuda_stream;
  return SV_OK;
}

int sv_device_ptr(sv_state *sv, void **out) {
  if (!sv || !out) return fail(SV_EINVAL, "NULL argument");
  *out = sv->amps;
  return SV_OK;
}

int sv_info(sv_state *sv, int *n_qubits, int *dtype) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (n_qubits) *n_qubits = sv->n;
  if (dtype) *dtype = sv->dtype;
  return SV_OK;
}

int sv_set_basis_state(sv_state *sv, uint64_t k) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (sv->n < 64 && (k >> sv->n)) return fail(SV_EINVAL, "basis index out of range");
  sv->frame = Pauli();
  return launch_set_basis(sv, k);
}

int sv_from_host(sv_state *sv, const void *host_amps) {
  if (!sv || !host_amps) return fail(SV_EINVAL, "NULL argument");
  size_t bytes = amp_bytes(sv->dtype) << sv->n;
  PR_CUDA(cudaMemcpyAsync(sv->amps, host_amps, bytes, cudaMemcpyHostToDevice, sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  sv->frame = Pauli();
  return SV_OK;
}

int sv_materialize(sv_state *sv) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  const Pauli &f = sv->frame;
  if (f.x == 0 && f.z == 0 && f.q == 0) return SV_OK;
  int rc = launch_materialize(sv, f.x, f.z, f.q);
  if (rc) return rc;
  sv->frame = Pauli();
  return SV_OK;
}

int sv_to_host(sv_state *sv, void *host_amps, int materialize_frame) {
  if (!sv || !host_amps) return fail(SV_EINVAL, "NULL argument");
  if (materialize_frame) {
    int rc = sv_materialize(sv);
    if (rc) return rc;
  }
  size_t bytes = amp_bytes(sv->dtype) << sv->n;
  PR_CUDA(cudaMemcpyAsync(host_amps, sv->amps, bytes, cudaMemcpyDeviceToHost, sv->stream));
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  return SV_OK;
}

int sv_copy(sv_state *dst, const sv_state *src) {
  if (!dst || !src) return fail(SV_EINVAL, "NULL argument");
  if (dst->n != src->n || dst->dtype != src->dtype) return fail(SV_EINVAL, "shape mismatch");
  if (dst == src) return SV_OK;
  size_t bytes = amp_bytes(src->dtype) << src->n;
  PR_CUDA(cudaMemcpyAsync(dst->amps, src->amps, bytes, cudaMemcpyDeviceToDevice, dst->stream));
  dst->frame = src->frame;
  return SV_OK;
}

int frame_reset(sv_state *sv) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  sv->frame = Pauli();
  return SV_OK;
}

int frame_apply_pauli(sv_state *sv, char pauli, int qubit) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (qubit < 0 || qubit >= sv->n) return fail(SV_EINVAL, "qubit %d out of range", qubit);
  uint64_t b = 1ULL << qubit;
  Pauli g;
  switch (pauli) {
    case 'X': case 'x': g = pauli_string(b, 0); break;
    case 'Y': case 'y': g = pauli_string(b, b); break;
    case 'Z': case 'z': g = pauli_string(0, b); break;
    default: return fail(SV_EINVAL, "pauli must be 'X', 'Y' or 'Z'");
  }
  // the gate acts after the frame: |psi'> = G Q |phi>
  sv->frame = pauli_mul(g, sv->frame);
  return SV_OK;
}

int frame_get(sv_state *sv, uint64_t *xq, uint64_t *zq, int *phase) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (xq) *xq = sv->frame.x;
  if (zq) *zq = sv->frame.z;
  if (phase) *phase = sv->frame.q;
  return SV_OK;
}

}  // extern "C"
