// Device code of the rotation passes, shared by the one-pass-per-launch
// kernels (rotate.cu) and the persistent batched kernel (batch.cu).
//
// Every pass is a __device__ body over one CTA's share of the index space
// (cta_rank of cta_count CTAs) with an explicit shared-memory workspace, so a
// caller can run passes back to back in one launch.
#pragma once

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

template <typename R, typename Idx, int D>
__host__ __device__ constexpr size_t ws_coset() {
  return ((sizeof(RotSm<R, Idx>) * kMaxRunRots + 15) & ~size_t(15)) + sizeof(Idx) * (1u << D);
}

// One CTA's share of a fused coset run: cosets cta_rank*chunk + t, stepping by
// cta_count*chunk.  ws: ws_coset<R, Idx, D>() bytes of shared memory.
template <typename R, typename Idx, int D, int V>
__device__ __forceinline__ void body_coset(typename Cx<R>::T *__restrict__ amp, Idx n_cosets, const RunDev &run,
                                           const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz,
                                           Idx cta_rank, Idx cta_count, char *ws) {
  using C = typename Cx<R>::T;
  constexpr int E = 1 << D;
  RotSm<R, Idx> *srot = (RotSm<R, Idx> *)ws;
  Idx *soff = (Idx *)(ws + ((sizeof(RotSm<R, Idx>) * kMaxRunRots + 15) & ~size_t(15)));
  const int count = run.count;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const RotDev r = rots[run.first + j];
    double t = r.t;
    if (__popcll((r.x & fz) ^ (r.z & fx)) & 1) t = -t;  // runtime frame sign
    RotSm<R, Idx> s;
    s.z = (Idx)r.z;
    s.zt = r.zt;
    s.code = r.code & kCodeMask;
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
  const Idx stride = cta_count * chunk;
  for (Idx c0 = cta_rank * chunk + threadIdx.x; c0 < n_cosets; c0 += stride) {
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
  __syncthreads();  // the workspace may be reused by the caller's next pass
}

// ------------------------------------------------------------------ complex64, packed pairs
//
// k_coset_c64x2: the same fused pass for complex64 with two adjacent cosets
// per thread (representatives rep and rep|1, bit 0 not a pivot).  Element l of
// both cosets lies in one aligned 16-byte float4 (its halves swapped when
// bit 0 of the element offset is set), so each element is one 16-byte load.
// Registers hold RE[l] = (re of coset 0, re of coset 1) and IM[l] likewise, and
// every update is a packed FP32x2 fused multiply-add.  The sign of element l
// for a rotation is (-1)^{popc(rep & z)} * chi(l) with chi a character of l
// (chi(l) = prod of S_b over the set bits b of l, S_b = (-1)^{popc(basis_b & z)}),
// so walking the pair leaders in Gray-code order updates the coefficient with one
// packed multiply by +-1 per pair instead of a per-element select.

// per-rotation values shared by the CTA: t2 = (t, t (-1)^{z_0}) (a thread's
// two cosets differ in index bit 0), S[b] = (s_b, s_b) with
// s_b = (-1)^{popc(basis_b & z)}; three 16-byte loads for 32-bit indices
template <typename Idx>
struct alignas(16) RotSm2 {
  float2 t2;
  Idx z;
  uint32_t code;
  float2 S[4];
};

// the thread's coefficient: t2 with both signs flipped when popc(rep & z) is odd
template <typename Idx>
__device__ __forceinline__ float2 rot_t(const RotSm2<Idx> &s, Idx rep) {
  const uint32_t sg = (uint32_t)parity(rep & s.z) << 31;
  return make_float2(__uint_as_float(__float_as_uint(s.t2.x) ^ sg), __uint_as_float(__float_as_uint(s.t2.y) ^ sg));
}

// free-bit index k (0-based among bits != H) -> bit position
template <int H>
__device__ __host__ constexpr int free_bit(int k) {
  return k < H ? k : k + 1;
}
// Gray code over the D-1 free bits, mapped to element index bits
template <int D, int H>
__device__ __host__ constexpr int gray_leader(int i) {
  int g = i ^ (i >> 1), l = 0;
  for (int k = 0; k < D - 1; ++k)
    if ((g >> k) & 1) l |= 1 << free_bit<H>(k);
  return l;
}
__device__ __host__ constexpr int ctz_c(int v) {
  int c = 0;
  while (!(v & 1)) {
    v >>= 1;
    ++c;
  }
  return c;
}
__device__ __host__ constexpr int high_bit(int v) {
  int h = 0;
  while (v >> (h + 1)) ++h;
  return h;
}

// negated coefficient written inline, so the compiler can fold the sign into
// the packed FMA instead of carrying a second chain
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }

// Pair update from the old values of both elements (exact tan form; the
// compiler keeps copies of the old values where a 2-cycle needs them).
template <int D, int U, int IMAG>
__device__ __forceinline__ void apply_x2(float2 (&RE)[1 << D], float2 (&IM)[1 << D], float2 T,
                                         const float2 (&S)[D > 0 ? D : 1]) {
  if constexpr (U == 0) {
    // diagonal: every element, Gray order over all D bits
#pragma unroll
    for (int i = 0; i < (1 << D); ++i) {
      if (i > 0) T = __fmul2_rn(T, S[ctz_c(i)]);
      const int l = i ^ (i >> 1);
      const float2 re = RE[l], im = IM[l];
      RE[l] = __ffma2_rn(neg2(T), im, re);
      IM[l] = __ffma2_rn(T, re, im);
    }
  } else {
    constexpr int H = high_bit(U);
#pragma unroll
    for (int i = 0; i < (1 << (D - 1)); ++i) {
      if (i > 0) T = __fmul2_rn(T, S[free_bit<H>(ctz_c(i))]);
      const float2 N = neg2(T);
      const int l = gray_leader<D, H>(i);
      const int m = l ^ U;
      const float2 rl = RE[l], il = IM[l], rm = RE[m], im = IM[m];
      if (IMAG) {
        RE[l] = __ffma2_rn(N, im, rl);
        IM[l] = __ffma2_rn(T, rm, il);
        RE[m] = __ffma2_rn(N, il, rm);
        IM[m] = __ffma2_rn(T, rl, im);
      } else {
        RE[l] = __ffma2_rn(T, rm, rl);
        IM[l] = __ffma2_rn(T, im, il);
        RE[m] = __ffma2_rn(N, rl, rm);
        IM[m] = __ffma2_rn(N, il, im);
      }
    }
  }
}

// Two consecutive rotations with the same code, T for the first and V for the
// second, applied pair by pair (pairs are disjoint, so the order of the two
// sweeps does not matter).  The first writes each leader's new value to a
// temporary and the second writes it back to the leader's register: unlike
// one rotation at a time, the update needs no register copies.
template <int D, int U, int IMAG>
__device__ __forceinline__ void apply_x2_pair(float2 (&RE)[1 << D], float2 (&IM)[1 << D], float2 T,
                                              const float2 (&S)[D > 0 ? D : 1], float2 V,
                                              const float2 (&SV)[D > 0 ? D : 1]) {
  if constexpr (U == 0) {
#pragma unroll
    for (int i = 0; i < (1 << D); ++i) {
      if (i > 0) {
        T = __fmul2_rn(T, S[ctz_c(i)]);
        V = __fmul2_rn(V, SV[ctz_c(i)]);
      }
      const int l = i ^ (i >> 1);
      const float2 re = RE[l], im = IM[l];
      const float2 re1 = __ffma2_rn(neg2(T), im, re), im1 = __ffma2_rn(T, re, im);
      RE[l] = __ffma2_rn(neg2(V), im1, re1);
      IM[l] = __ffma2_rn(V, re1, im1);
    }
  } else {
    constexpr int H = high_bit(U);
#pragma unroll
    for (int i = 0; i < (1 << (D - 1)); ++i) {
      if (i > 0) {
        T = __fmul2_rn(T, S[free_bit<H>(ctz_c(i))]);
        V = __fmul2_rn(V, SV[free_bit<H>(ctz_c(i))]);
      }
      const float2 N = neg2(T), NV = neg2(V);
      const int l = gray_leader<D, H>(i);
      const int m = l ^ U;
      const float2 rl = RE[l], il = IM[l], rm = RE[m], im = IM[m];
      if (IMAG) {
        const float2 rl1 = __ffma2_rn(N, im, rl), il1 = __ffma2_rn(T, rm, il);
        const float2 rm1 = __ffma2_rn(N, il, rm), im1 = __ffma2_rn(T, rl, im);
        RE[l] = __ffma2_rn(NV, im1, rl1);
        IM[l] = __ffma2_rn(V, rm1, il1);
        RE[m] = __ffma2_rn(NV, il1, rm1);
        IM[m] = __ffma2_rn(V, rl1, im1);
      } else {
        const float2 rl1 = __ffma2_rn(T, rm, rl), il1 = __ffma2_rn(T, im, il);
        const float2 rm1 = __ffma2_rn(N, rl, rm), im1 = __ffma2_rn(N, il, im);
        RE[l] = __ffma2_rn(V, rm1, rl1);
        IM[l] = __ffma2_rn(V, im1, il1);
        RE[m] = __ffma2_rn(NV, rl1, rm1);
        IM[m] = __ffma2_rn(NV, il1, im1);
      }
    }
  }
}

// One segment (len consecutive rotations with code (U << 1) | IMAG): two
// rotations per sweep of the pairs, the odd one out alone.
template <typename Idx, int D, int U, int IMAG>
__device__ __forceinline__ void seg_x2(float2 (&RE)[1 << D], float2 (&IM)[1 << D], const RotSm2<Idx> *r, int len,
                                       Idx rep) {
  constexpr int NS = D > 0 ? D : 1;
  int k = 0;
  for (; k + 1 < len; k += 2) {
    const RotSm2<Idx> &a = r[k], &b = r[k + 1];
    float2 S[NS], SV[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) {
      S[q] = a.S[q];
      SV[q] = b.S[q];
    }
    apply_x2_pair<D, U, IMAG>(RE, IM, rot_t(a, rep), S, rot_t(b, rep), SV);
  }
  if (k < len) {
    const RotSm2<Idx> &a = r[k];
    float2 S[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) S[q] = a.S[q];
    apply_x2<D, U, IMAG>(RE, IM, rot_t(a, rep), S);
  }
}

#define PR_CASE2S(K)                                                               \
  case K:                                                                          \
    if constexpr ((((K) >> 1) < (1 << D)) && ((((K) >> 1) != 0) || ((K)&1)))       \
      seg_x2<Idx, D, ((K) >> 1), ((K)&1)>(RE, IM, r, len, rep);                   \
    break;
#define PR_CASE2S_8(B) \
  PR_CASE2S(B + 0) PR_CASE2S(B + 1) PR_CASE2S(B + 2) PR_CASE2S(B + 3) PR_CASE2S(B + 4) PR_CASE2S(B + 5) PR_CASE2S(B + 6) PR_CASE2S(B + 7)

template <typename Idx, int D>
__device__ __forceinline__ void dispatch_seg(uint32_t code, float2 (&RE)[1 << D], float2 (&IM)[1 << D],
                                             const RotSm2<Idx> *r, int len, Idx rep) {
  switch (code) {
    PR_CASE2S_8(0)
    PR_CASE2S_8(8)
    PR_CASE2S_8(16)
    PR_CASE2S_8(24)
    default:
      break;
  }
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <typename Idx, int D>
__device__ __forceinline__ Idx pair_rep(Idx c, const RunDev &run) {
  Idx rep = c << 1;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    const int p = run.piv[b];
    rep = ((rep >> p) << (p + 1)) | (rep & ((Idx(1) << p) - 1));
  }
  return rep;
}

template <typename Idx, int D>
__host__ __device__ constexpr size_t ws_c64x2_head() {
  return ((sizeof(RotSm2<Idx>) * kMaxRunRots + sizeof(Idx) * (1u << D)) + 15) & ~size_t(15);
}
// workspace: rotation table, element offsets, then one 16-byte slot per element
// per thread laid out [element][thread] so a warp's accesses to one element
// are contiguous
template <typename Idx, int D>
__host__ __device__ constexpr size_t ws_c64x2() {
  return ws_c64x2_head<Idx, D>() + sizeof(float4) * kThreads * (1u << D);
}

template <typename Idx, int D>
__device__ __forceinline__ void body_c64x2(float4 *__restrict__ amp4, Idx n_pairs, const RunDev &run,
                                           const RotDev *__restrict__ rots, uint64_t fx, uint64_t fz,
                                           Idx cta_rank, Idx cta_count, char *ws, bool chained = false,
                                           bool reverse = false) {
  constexpr int E = 1 << D;
  // reverse: coset pairs are taken from the top (the grid walks them in
  // descending order), so a pass that follows one in ascending order starts
  // on the amplitudes its predecessor wrote last, while they are still in L2.
  // chained: launched as a programmatic dependent of the previous pass.  The
  // next pass may be scheduled as this one's CTAs retire; this pass reads its
  // rotation table before waiting for the previous pass, and touches no
  // amplitude until that pass has completed and its writes are visible.
  if (chained) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  RotSm2<Idx> *srot = (RotSm2<Idx> *)ws;
  Idx *soff = (Idx *)(ws + sizeof(RotSm2<Idx>) * kMaxRunRots);
  float4 *stage = (float4 *)(ws + ws_c64x2_head<Idx, D>());
  const int count = run.count;
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const RotDev r = rots[run.first + j];
    double t = r.t;
    if (__popcll((r.x & fz) ^ (r.z & fx)) & 1) t = -t;  // runtime frame sign
    const float tf = (float)t;
    RotSm2<Idx> s;
    s.t2 = make_float2(tf, (r.z & 1) ? -tf : tf);
    s.z = (Idx)r.z;
    s.code = r.code;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const float sb = (b < D && ((r.zt >> (1 << b)) & 1u)) ? -1.0f : 1.0f;
      s.S[b] = make_float2(sb, sb);
    }
    srot[j] = s;
  }
  if (threadIdx.x < E) {
    uint64_t s = 0;
    for (int b = 0; b < D; ++b)
      if ((threadIdx.x >> b) & 1) s ^= run.basis[b];
    soff[threadIdx.x] = (Idx)s;
  }
  __syncthreads();
  if (chained) asm volatile("griddepcontrol.wait;" ::: "memory");

  const Idx stride = cta_count * blockDim.x;
  float4 *slot = stage + threadIdx.x;
  Idx c = cta_rank * blockDim.x + threadIdx.x;
  // prefetch the first coset pair
  if (c < n_pairs) {
    const Idx rep0 = pair_rep<Idx, D>(reverse ? n_pairs - 1 - c : c, run);
#pragma unroll
    for (int l = 0; l < E; ++l) cp_async16(slot + l * blockDim.x, amp4 + ((rep0 ^ soff[l]) >> 1));
    cp_async_commit();
  }
  for (; c < n_pairs; c += stride) {
    const Idx rep = pair_rep<Idx, D>(reverse ? n_pairs - 1 - c : c, run);
    cp_async_wait_all();
    float2 RE[E], IM[E];
#pragma unroll
    for (int l = 0; l < E; ++l) {
      const Idx e = rep ^ soff[l];
      const float4 v = slot[l * blockDim.x];
      if (e & 1) {
        RE[l] = make_float2(v.z, v.x);
        IM[l] = make_float2(v.w, v.y);
      } else {
        RE[l] = make_float2(v.x, v.z);
        IM[l] = make_float2(v.y, v.w);
      }
    }
    // the slot is free again: prefetch the next coset pair while this one computes
    const Idx cn = c + stride;
    if (cn < n_pairs) {
      const Idx repn = pair_rep<Idx, D>(reverse ? n_pairs - 1 - cn : cn, run);
#pragma unroll
      for (int l = 0; l < E; ++l) cp_async16(slot + l * blockDim.x, amp4 + ((repn ^ soff[l]) >> 1));
      cp_async_commit();
    }
    for (int j = 0; j < count;) {
      const uint32_t word = srot[j].code;
      const int len = (int)(word >> kSegShift);
      dispatch_seg<Idx, D>(word & kCodeMask, RE, IM, srot + j, len, rep);
      j += len > 0 ? len : 1;
    }
    if (run.fold) {
      const float fr = (float)run.fold_re, fi = (float)run.fold_im;
      const float2 FR = make_float2(fr, fr), FI = make_float2(fi, fi), NFI = make_float2(-fi, -fi);
#pragma unroll
      for (int l = 0; l < E; ++l) {
        const float2 re = RE[l], im = IM[l];
        RE[l] = __ffma2_rn(NFI, im, __fmul2_rn(FR, re));
        IM[l] = __ffma2_rn(FI, re, __fmul2_rn(FR, im));
      }
    }
    // recompute the element addresses instead of keeping 2^D of them live
    // across the rotation loop
    asm volatile("" ::: "memory");
#pragma unroll
    for (int l = 0; l < E; ++l) {
      const Idx e = rep ^ soff[l];
      float4 v;
      if (e & 1)
        v = make_float4(RE[l].y, IM[l].y, RE[l].x, IM[l].x);
      else
        v = make_float4(RE[l].x, IM[l].x, RE[l].y, IM[l].y);
      amp4[e >> 1] = v;
    }
  }
  __syncthreads();  // the workspace may be reused by the caller's next pass
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
    // top 32 of the 48 residual bits: a 32-bit conversion (the 64-bit one runs
    // on the FP64 pipe) is exact enough for float
    const float x = (float)(uint32_t)(rem >> 16) * 2.23223584e-14f;  // 2 pi / 2^48
    s.x = fmaf(-0.5f * x, x, 1.0f);
    s.y = x;
  }
  return cmul<R>(cmul<R>(t0, t1), s);
}

// Workspace of body_diag, in this order: phase tables (512 entries, 16-byte
// aligned for double2), per-rotation angles, per-warp slot sums, per-rotation
// z-masks, per-slot lane sign masks, per-rotation slots.
template <typename R, typename Idx>
__host__ __device__ constexpr size_t ws_diag_off(int part) {
  size_t off = 0;
  const size_t sizes[6] = {sizeof(typename Cx<R>::T) * 512, sizeof(uint64_t) * kMaxDiagRots,
                           sizeof(uint64_t) * kDiagSlots * (kThreads / 32), sizeof(Idx) * kMaxDiagRots,
                           sizeof(uint32_t) * kDiagSlots, sizeof(uint16_t) * kMaxDiagRots};
  for (int k = 0; k < part; ++k) off += sizes[k];
  return off;
}

template <typename R, typename Idx>
__host__ __device__ constexpr size_t ws_diag() {
  return ws_diag_off<R, Idx>(6);
}

// bit l = parity(l & m) for the 5 lane bits of m
__device__ __forceinline__ uint32_t lane_signs(uint32_t m) {
  uint32_t s = 0;
  if (m & 1u) s ^= 0xAAAAAAAAu;
  if (m & 2u) s ^= 0xCCCCCCCCu;
  if (m & 4u) s ^= 0xF0F0F0F0u;
  if (m & 8u) s ^= 0xFF00FF00u;
  if (m & 16u) s ^= 0xFFFF0000u;
  return s;
}

// A diagonal phase-sum run: amplitude k is multiplied by exp(-i A(k)) with
// A(k) = sum_j a_j (-1)^{popc(k & z_j)} (a_j = theta_j / 2 in units of 2 pi / 2^64,
// summed exactly modulo 2^64, so any order gives the same bits).
//
// A thread owns a group of 16 amplitudes k = base | (e << 5), e = 0..15 (class
// bits 5..8), and lane l of a warp has base bits 0..4 = l, so a warp covers
// index bits 0..8 and shares rest = base bits 9 and up.  With the run's
// rotations grouped into slots s by their z pattern m_s on bits 0..8 (lane part
// m_s & 31, class part m_s >> 5),
//   A(k) = sum_e' (-1)^{popc(e & e')} acc[e'],
//   acc[e'] = sum_{s : class part e'} (-1)^{popc(l & m_s & 31)} D[s],
//   D[s] = sum_{j in s} a_j (-1)^{popc(rest & z_j)}.
// D is warp-uniform: the warp's lanes split the rotations between them (a
// segmented scan over the slot-sorted rotations, into a warp-private shared
// array), so a rotation costs each lane a share of a scan step per group
// instead of a term; a lane then pays one term per slot (a run has at most
// kDiagSlots of them) and the 16-point transform over the class bits.
// complex128 instead sums each class's rotations per thread (acc[c] = sum over
// the rotations of class c of a_j (-1)^{popc(base & z_j)}): there the FP64
// phase products bound the pass, and they overlap that longer integer work
// better than the slot sums (measured: 582 against 701 us per pass at n = 24).
// Needs blockDim.x <= kThreads, a multiple of 32, and n_groups a multiple of 32
// (n >= 9): every warp then runs whole groups together.
template <typename R, typename Idx>
__device__ __forceinline__ void body_diag(typename Cx<R>::T *__restrict__ amp, Idx n_groups, const RunDev &run,
                                          const DiagDev *__restrict__ rots, uint64_t fx,
                                          const typename Cx<R>::T *__restrict__ tab, Idx cta_rank, Idx cta_count,
                                          char *ws) {
  static_assert(kDiagClassLo == 5, "lane bits 0..4 below the class bits");
  using C = typename Cx<R>::T;
  C *stab = (C *)(ws + ws_diag_off<R, Idx>(0));
  uint64_t *sa = (uint64_t *)(ws + ws_diag_off<R, Idx>(1));
  uint64_t *sD = (uint64_t *)(ws + ws_diag_off<R, Idx>(2));
  Idx *sz = (Idx *)(ws + ws_diag_off<R, Idx>(3));
  uint32_t *smask = (uint32_t *)(ws + ws_diag_off<R, Idx>(4));
  uint16_t *sslot = (uint16_t *)(ws + ws_diag_off<R, Idx>(5));
  const int count = run.count;
  const int nslots = run.seg[kCls];
  for (int j = threadIdx.x; j < count; j += blockDim.x) {
    const DiagDev r = rots[run.first + j];
    sz[j] = (Idx)r.z;
    sa[j] = (__popcll(r.z & fx) & 1) ? (0ULL - r.a) : r.a;  // runtime frame sign
    sslot[j] = (uint16_t)r.slot;
    smask[r.slot] = lane_signs((uint32_t)r.z & 31u);  // the same for every rotation of the slot
  }
  for (int j = threadIdx.x; j < 512; j += blockDim.x) stab[j] = tab[j];
  __syncthreads();
  // complex128: class c (z bits 5..8) holds rotations [rseg[c], rseg[c + 1])
  // (the slots, and so the rotations, are sorted by class)
  __shared__ int rseg[kCls + 1];
  if constexpr (sizeof(R) == 8) {
    if (threadIdx.x <= kCls) {
      const int c = (int)threadIdx.x;
      int lo = 0, hi = count;  // first rotation of class >= c
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if ((int)((sz[mid] >> kDiagClassLo) & (Idx)(kCls - 1)) < c)
          lo = mid + 1;
        else
          hi = mid;
      }
      rseg[c] = lo;
    }
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  unsigned long long *D = (unsigned long long *)sD + (threadIdx.x >> 5) * kDiagSlots;
  const Idx stride = cta_count * blockDim.x;
  for (Idx g = cta_rank * blockDim.x + threadIdx.x; g < n_groups; g += stride) {
    const Idx base = (g & (Idx)31) | ((g >> 5) << (kDiagClassLo + kDiagClassBits));
    const Idx rest = base & ~(Idx)((1u << (kDiagClassLo + kDiagClassBits)) - 1u);
    // complex64: the group's amplitudes first, so that their latency overlaps
    // the sums (16 double2 would cost complex128 its occupancy)
    constexpr bool kEarly = sizeof(R) == 4;
    C av[kCls];
    if (kEarly) {
#pragma unroll
      for (int e = 0; e < kCls; ++e) av[e] = amp[base | ((Idx)e << kDiagClassLo)];
    }
    // D: the warp takes the rotations 32 at a time; they are sorted by slot, so
    // a segmented scan across the lanes leaves each slot's sum over the batch on
    // the slot's last lane in it, the one writer of D[s] for that batch
    uint64_t acc[kCls];
    if constexpr (sizeof(R) == 8) {
#pragma unroll
      for (int c = 0; c < kCls; ++c) {
        uint64_t t = 0;
        const int j1 = rseg[c + 1];
        for (int j = rseg[c]; j < j1; ++j) {
          const uint64_t a = sa[j];
          t += parity(base & sz[j]) ? (0ULL - a) : a;
        }
        acc[c] = t;
      }
    } else {
      for (int s = lane; s < nslots; s += 32) D[s] = 0ULL;
      __syncwarp();
      for (int j0 = 0; j0 < count; j0 += 32) {
        const int j = j0 + lane;
        uint64_t v = 0;
        int s = -1;
        if (j < count) {
          const uint64_t a = sa[j];
          v = parity(rest & sz[j]) ? (0ULL - a) : a;
          s = sslot[j];
        }
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
          const unsigned long long vu = __shfl_up_sync(0xffffffffu, (unsigned long long)v, off);
          const int su = __shfl_up_sync(0xffffffffu, s, off);
          if (lane >= off && su == s) v += vu;
        }
        const int sn = __shfl_down_sync(0xffffffffu, s, 1);
        if (s >= 0 && (lane == 31 || sn != s)) D[s] += v;
        __syncwarp();
      }
#pragma unroll
      for (int c = 0; c < kCls; ++c) {
        uint64_t t = 0;
        const int s1 = run.seg[c + 1];
        for (int s = run.seg[c]; s < s1; ++s) {
          const uint64_t d = D[s];
          t += ((smask[s] >> lane) & 1u) ? (0ULL - d) : d;
        }
        acc[c] = t;
      }
      __syncwarp();  // D is cleared for the next group
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
      amp[k] = cmul<R>(kEarly ? av[e] : amp[k], ph);
    }
  }
  __syncthreads();  // the workspace may be reused by the caller's next pass
}

}  // namespace
}  // namespace pr
