// Chained complex64 passes: two consecutive fused coset runs in one HBM pass.
//
// A fused run (kernels.cuh, k_coset_c64x2) reads the whole state, applies its
// rotations and writes it back.  On GB300 a depth-4 run of the n = 24
// Jordan-Wigner workload costs about as much FMA-pipe time as its sweep takes
// at HBM speed, so half of every pass is spent moving data.  Here a CTA owns a
// block of 2^12 amplitudes, a coset of a subspace W that contains the spans of
// two consecutive runs (and index bits 0..3, so that the block's amplitudes
// come in 128-byte segments).  The block sits in shared memory; each thread
// takes its two adjacent cosets of the first run's span from it, applies that
// run, puts them back, takes its cosets of the second run's span, applies the
// second run and writes them to HBM.  Every rotation pairs k with k ^ x inside
// one coset of its run's span (paper, Sec. "Multi-qubit rotations in a
// fullstate simulator": f_P(k) = k ^ x), and both spans lie in W, so the block
// is closed under both runs and the state crosses HBM once for both.
//
// Per element the arithmetic is that of k_coset_c64x2 in the same order (the
// tan-form pair updates of the appendix "Amplitude update rule", the Gray-code
// sign walk, the run's closing scale), so a chained pass gives bitwise the
// same state as the two passes it replaces.  A run of dimension d < 4 is
// padded to 4 basis vectors with block coordinates outside its span: its
// rotations then act on 16-element cosets that are unions of its own.
#include <cstdlib>
#include <cstring>

#include "kernels.cuh"

namespace pr {

namespace {

// a thread holds 32 amplitudes (two 16-element cosets); 16 warps per SM
constexpr int kChainThreads = 1 << (kChainDim - 5);
constexpr int kChainMinBlocks = 512 / kChainThreads;

// GF(2) echelon rows, each with the combination of inserted vectors it is
// (bit k = the k-th labelled input)
struct Echelon {
  uint64_t v[64];
  uint32_t comb[64];
  bool has[64] = {};
  bool add(uint64_t x, uint32_t c) {
    while (x) {
      const int h = 63 - __builtin_clzll(x);
      if (!has[h]) {
        has[h] = true;
        v[h] = x;
        comb[h] = c;
        return true;
      }
      x ^= v[h];
      c ^= comb[h];
    }
    return false;
  }
  bool solve(uint64_t x, uint32_t &c) const {
    c = 0;
    while (x) {
      const int h = 63 - __builtin_clzll(x);
      if (!has[h]) return false;
      x ^= v[h];
      c ^= comb[h];
    }
    return true;
  }
};

bool packable(const RunDev &r) { return r.kind == 0 && r.d <= 4 && (r.d == 0 || r.piv[0] >= 1); }

bool make_chain(int n, const RunDev &r0, const RunDev &r1, ChainDev &ch) {
  std::memset(&ch, 0, sizeof(ch));
  // W: index bits 0..3, then both spans with bits 0..3 cleared, then unit
  // vectors of the lowest free bits
  Echelon W;
  int k = 0;
  for (; k < 4; ++k) {
    W.add(1ULL << k, 1u << k);
    ch.w[k] = 1ULL << k;
  }
  uint32_t c = 0;
  for (const RunDev *r : {&r0, &r1})
    for (int b = 0; b < r->d; ++b) {
      const uint64_t v = r->basis[b] & ~15ULL;
      if (W.solve(v, c)) continue;
      if (k == kChainDim) return false;
      W.add(v, 1u << k);
      ch.w[k++] = v;
    }
  for (int q = 4; k < kChainDim && q < n; ++q) {
    if (W.solve(1ULL << q, c)) continue;
    W.add(1ULL << q, 1u << k);
    ch.w[k++] = 1ULL << q;
  }
  if (k < kChainDim) return false;
  for (int h = 0, i = 0; h < 64; ++h)
    if (W.has[h]) ch.wpiv[i++] = h;

  for (int s = 0; s < 2; ++s) {
    const RunDev &r = s ? r1 : r0;
    ChainSubDev &sd = ch.sub[s];
    sd.d = r.d;
    sd.first = r.first;
    sd.count = r.count;
    sd.fold = r.fold;
    sd.fold_re = r.fold_re;
    sd.fold_im = r.fold_im;
    uint32_t bc[4];
    uint64_t bv[4];
    // span in block coordinates; C0 also holds coordinate 0 (index bit 0),
    // which must stay outside the padded span (it pairs the thread's cosets)
    Echelon C, C0;
    C0.add(1u, 0);
    for (int b = 0; b < r.d; ++b) {
      if (!W.solve(r.basis[b], bc[b])) return false;
      bv[b] = r.basis[b];
      C.add(bc[b], 0);
      if (!C0.add(bc[b], 0)) return false;
    }
    int d = r.d;
    for (int cp = kChainDim - 1; d < 4 && cp >= 1; --cp) {
      if (!C0.add(1ULL << cp, 0)) continue;
      C.add(1ULL << cp, 0);
      bc[d] = 1u << cp;
      bv[d] = ch.w[cp];
      sd.padv[d] = ch.w[cp];
      ++d;
    }
    if (d < 4) return false;
    for (int h = 0, i = 0; h < kChainDim; ++h)
      if (C.has[h]) sd.pivc[i++] = h;
    for (int l = 0; l < 16; ++l) {
      uint64_t o = 0;
      uint32_t oc = 0;
      for (int b = 0; b < 4; ++b)
        if ((l >> b) & 1) {
          o ^= bv[b];
          oc ^= bc[b];
        }
      sd.off[l] = o;
      sd.offc[l] = (uint16_t)oc;
    }
  }
  return true;
}

// ------------------------------------------------------------------ device

constexpr int kBlockF4 = 1 << (kChainDim - 1);  // float4 slots of a block

template <typename Idx>
__host__ __device__ constexpr size_t ws_chain_head() {
  return (sizeof(RotSm2<Idx>) * kMaxRunRots + 15) & ~size_t(15);
}
template <typename Idx>
__host__ __device__ constexpr size_t ws_chain() {
  return ws_chain_head<Idx>() + sizeof(float4) * kBlockF4;
}

// insert a zero bit at each of the ascending positions p[0..N-1]
template <int N, typename Idx>
__device__ __forceinline__ Idx spread(Idx v, const int32_t *p) {
#pragma unroll
  for (int b = 0; b < N; ++b) v = ((v >> p[b]) << (p[b] + 1)) | (v & ((Idx(1) << p[b]) - 1));
  return v;
}

// the thread's two adjacent cosets of a run's padded span, taken from the block
// (element l of both in one float4, halves swapped when bit 0 of its offset is set)
__device__ __forceinline__ void take(const float4 *buf, int repc, const ChainSubDev &sd, float2 (&RE)[16],
                                     float2 (&IM)[16]) {
#pragma unroll
  for (int l = 0; l < 16; ++l) {
    const int oc = sd.offc[l];
    const float4 v = buf[(repc ^ oc) >> 1];
    if (oc & 1) {
      RE[l] = make_float2(v.z, v.x);
      IM[l] = make_float2(v.w, v.y);
    } else {
      RE[l] = make_float2(v.x, v.z);
      IM[l] = make_float2(v.y, v.w);
    }
  }
}

__device__ __forceinline__ float4 pack(const float2 &re, const float2 &im, bool swap) {
  return swap ? make_float4(re.y, im.y, re.x, im.x) : make_float4(re.x, im.x, re.y, im.y);
}

template <typename Idx>
__device__ __forceinline__ void run_rotations(float2 (&RE)[16], float2 (&IM)[16], const RotSm2<Idx> *srot, int count,
                                              Idx rep, const ChainSubDev &sd) {
  for (int j = 0; j < count;) {
    const uint32_t word = srot[j].code;
    const int len = (int)(word >> kSegShift);
    dispatch_seg<Idx, 4>(word & kCodeMask, RE, IM, srot + j, len, rep);
    j += len > 0 ? len : 1;
  }
  if (sd.fold) {
    const float fr = (float)sd.fold_re, fi = (float)sd.fold_im;
    const float2 FR = make_float2(fr, fr), FI = make_float2(fi, fi), NFI = make_float2(-fi, -fi);
#pragma unroll
    for (int l = 0; l < 16; ++l) {
      const float2 re = RE[l], im = IM[l];
      RE[l] = __ffma2_rn(NFI, im, __fmul2_rn(FR, re));
      IM[l] = __ffma2_rn(FI, re, __fmul2_rn(FR, im));
    }
  }
}

// Launched as a programmatic dependent of the previous pass: the rotation
// table is built before waiting for that pass; no amplitude is touched before.
// reverse: blocks are taken from the top, so a pass that follows one walking
// upwards starts on the amplitudes its predecessor wrote last (still in L2).
template <typename Idx>
__global__ void __launch_bounds__(kChainThreads, kChainMinBlocks)
    k_chain_c64x2(float4 *__restrict__ amp4, Idx n_blocks, const __grid_constant__ ChainDev ch,
                  const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz, int reverse) {
  extern __shared__ __align__(16) char dyn_ws[];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  RotSm2<Idx> *srot = (RotSm2<Idx> *)dyn_ws;
  float4 *buf = (float4 *)(dyn_ws + ws_chain_head<Idx>());
  const int c0 = ch.sub[0].count, c1 = ch.sub[1].count;
  for (int j = threadIdx.x; j < c0 + c1; j += blockDim.x) {
    const int s = j < c0 ? 0 : 1;
    const ChainSubDev &sd = ch.sub[s];
    const RotDev r = rots[sd.first + (j - (s ? c0 : 0))];
    double t = r.t;
    if (__popcll((r.x & fz) ^ (r.z & fx)) & 1) t = -t;  // runtime frame sign
    const float tf = (float)t;
    RotSm2<Idx> q;
    q.t2 = make_float2(tf, (r.z & 1) ? -tf : tf);
    q.z = (Idx)r.z;
    q.code = r.code;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int neg = b < sd.d ? (int)((r.zt >> (1 << b)) & 1u) : (__popcll(r.z & sd.padv[b]) & 1);
      const float sb = neg ? -1.0f : 1.0f;
      q.S[b] = make_float2(sb, sb);
    }
    srot[j] = q;
  }
  // the thread's representatives: block coordinates (bit 0 clear, zeros at
  // the padded span's pivots) and their index-space vectors
  int repc[2];
  Idx repa[2];
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    repc[s] = spread<4, int>((int)threadIdx.x << 1, ch.sub[s].pivc);
    Idx a = 0;
#pragma unroll
    for (int i = 1; i < kChainDim; ++i)
      if ((repc[s] >> i) & 1) a ^= (Idx)ch.w[i];
    repa[s] = a;
  }
  __syncthreads();
  asm volatile("griddepcontrol.wait;" ::: "memory");

  const ChainSubDev &s0 = ch.sub[0], &s1 = ch.sub[1];
  auto base = [&](Idx b) { return spread<kChainDim, Idx>(reverse ? n_blocks - 1 - b : b, ch.wpiv); };
  // the first run's cosets of block b, straight into their block slots
  auto prefetch = [&](Idx b) {
    const Idx a0 = base(b) ^ repa[0];
#pragma unroll
    for (int l = 0; l < 16; ++l)
      cp_async16(buf + ((repc[0] ^ s0.offc[l]) >> 1), amp4 + ((a0 ^ (Idx)s0.off[l]) >> 1));
    cp_async_commit();
  };
  Idx b = blockIdx.x;
  if (b < n_blocks) prefetch(b);
  for (; b < n_blocks; b += gridDim.x) {
    const Idx B = base(b);
    float2 RE[16], IM[16];
    // first run: only the slots this thread copied itself
    cp_async_wait_all();
    take(buf, repc[0], s0, RE, IM);
    run_rotations<Idx>(RE, IM, srot, c0, B ^ repa[0], s0);
#pragma unroll
    for (int l = 0; l < 16; ++l) buf[(repc[0] ^ s0.offc[l]) >> 1] = pack(RE[l], IM[l], s0.offc[l] & 1);
    __syncthreads();
    // second run: its cosets cut across the first run's
    take(buf, repc[1], s1, RE, IM);
    __syncthreads();
    if (b + gridDim.x < n_blocks) prefetch(b + gridDim.x);
    run_rotations<Idx>(RE, IM, srot + c0, c1, B ^ repa[1], s1);
    const Idx a1 = B ^ repa[1];
#pragma unroll
    for (int l = 0; l < 16; ++l) amp4[(a1 ^ (Idx)s1.off[l]) >> 1] = pack(RE[l], IM[l], s1.off[l] & 1);
  }
}

template <typename Idx>
int launch_chain_t(sv_state *sv, const sv_plan *plan, const ChainDev &ch, uint64_t fx, uint64_t fz) {
  static const int cap = [] {
    const size_t bytes = ws_chain<Idx>();
    if (cudaFuncSetAttribute(k_chain_c64x2<Idx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) !=
        cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_chain_c64x2<Idx>, kChainThreads, bytes) !=
        cudaSuccess) {
      cudaGetLastError();
      per_sm = 1;
    }
    return (per_sm > 0 ? per_sm : 1) * device_sm_count();
  }();
  if (cap < 0) return fail(SV_ECUDA, "cannot set the shared-memory size of the chained pass");
  const uint64_t n_blocks = (1ULL << sv->n) >> kChainDim;
  const unsigned blocks = (unsigned)(n_blocks < (uint64_t)cap ? n_blocks : (uint64_t)cap);
  const int tr = trace_begin(sv, KN_CHAIN);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(blocks);
  cfg.blockDim = dim3(kChainThreads);
  cfg.dynamicSmemBytes = ws_chain<Idx>();
  cfg.stream = sv->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const int reverse = (int)(sv->packed_passes++ & 1u);
  PR_CUDA(cudaLaunchKernelEx(&cfg, k_chain_c64x2<Idx>, (float4 *)sv->amps, (Idx)n_blocks, ch,
                             (const RotDev *)plan->d_rots, fx, fz, reverse));
  trace_end(sv, tr, KN_CHAIN, 2.0 * 8.0 * (double)(1ULL << sv->n),
            4.0 * (double)(ch.sub[0].count + ch.sub[1].count) * (double)(1ULL << sv->n));
  return SV_OK;
}

}  // namespace

bool chains_enabled(const sv_plan *p) {
  if (p->dtype != SV_C64 || p->n <= kChainDim) return false;
  const char *env = std::getenv("PAULIROT_CHAIN");
  return !(env && env[0] == '0');
}

bool chain_pair(const sv_plan *p, size_t i, ChainDev *out) {
  const std::vector<RunDev> &runs = p->runs;
  if (i + 1 >= runs.size() || !packable(runs[i]) || !packable(runs[i + 1]) ||
      runs[i].count + runs[i + 1].count > kMaxRunRots)
    return false;
  return make_chain(p->n, runs[i], runs[i + 1], *out);
}

void build_chains(sv_plan *p) {
  p->steps.clear();
  p->chains.clear();
  if (!chains_enabled(p)) return;
  // greedy from the front: a run pairs with its successor when both fit
  for (size_t i = 0; i < p->runs.size();) {
    ChainDev ch;
    if (chain_pair(p, i, &ch)) {
      p->steps.push_back({(int32_t)i, (int32_t)p->chains.size()});
      p->chains.push_back(ch);
      i += 2;
      continue;
    }
    p->steps.push_back({(int32_t)i, -1});
    ++i;
  }
}

int launch_chain(sv_state *sv, const sv_plan *plan, const ChainDev &chain, uint64_t fx, uint64_t fz) {
  if (sv->dtype != SV_C64 || sv->n <= kChainDim) return fail(SV_EINVAL, "chained pass: complex64 and n > %d only", kChainDim);
  return sv->n <= 31 ? launch_chain_t<uint32_t>(sv, plan, chain, fx, fz)
                     : launch_chain_t<uint64_t>(sv, plan, chain, fx, fz);
}

}  // namespace pr
