// Checkpoint and resume of a state handle: the amplitudes phi, the Pauli frame
// Q (so the represented state Q phi is restored exactly, without materialising
// the frame) and a caller tag, e.g. the index of the next segment of a Trotter
// sequence that was compiled as several plans.
//
// File layout (little-endian):
//   0  char[8]  magic "PRCKPT01"
//   8  u32      version (1)
//  12  i32      n
//  16  i32      dtype (SV_C128 / SV_C64)
//  20  i32      frame phase q (Q = i^q X^x Z^z)
//  24  u64      frame x
//  32  u64      frame z
//  40  u64      tag
//  48  u64      amplitude bytes (= bytes per amplitude << n)
//  56  u64      checksum of the amplitude bytes
//  64  u64      checksum of bytes 0..63
//  72  amplitudes, as they lie in device memory
// Checksums are FNV-1a (offset basis 0xcbf29ce484222325, prime 0x100000001b3)
// taken over 64-bit little-endian words instead of bytes.
//
// The amplitudes move through two pinned host buffers: while one chunk is
// copied between device and host, the other is hashed and read or written.
#include <cerrno>
#include <cstdio>
#include <cstring>
#include <string>

#include <unistd.h>

#include "internal.h"

namespace pr {
namespace {

constexpr char kMagic[8] = {'P', 'R', 'C', 'K', 'P', 'T', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kHeader = 72;
constexpr size_t kChunk = size_t(64) << 20;
constexpr uint64_t kFnvBasis = 0xcbf29ce484222325ULL;
constexpr uint64_t kFnvPrime = 0x100000001b3ULL;

uint64_t fnv_words(uint64_t h, const unsigned char *p, size_t bytes) {
  for (size_t i = 0; i + 8 <= bytes; i += 8) {
    uint64_t w = 0;
    for (int b = 7; b >= 0; --b) w = (w << 8) | p[i + b];
    h = (h ^ w) * kFnvPrime;
  }
  return h;
}

void put_u32(unsigned char *p, uint32_t v) {
  for (int b = 0; b < 4; ++b) p[b] = (unsigned char)(v >> (8 * b));
}
void put_u64(unsigned char *p, uint64_t v) {
  for (int b = 0; b < 8; ++b) p[b] = (unsigned char)(v >> (8 * b));
}
uint32_t get_u32(const unsigned char *p) {
  uint32_t v = 0;
  for (int b = 3; b >= 0; --b) v = (v << 8) | p[b];
  return v;
}
uint64_t get_u64(const unsigned char *p) {
  uint64_t v = 0;
  for (int b = 7; b >= 0; --b) v = (v << 8) | p[b];
  return v;
}

struct Pinned {
  void *p[2] = {nullptr, nullptr};
  cudaEvent_t ev[2] = {nullptr, nullptr};
  ~Pinned() {
    for (int i = 0; i < 2; ++i) {
      if (ev[i]) cudaEventDestroy(ev[i]);
      if (p[i]) cudaFreeHost(p[i]);
    }
  }
  int init(size_t bytes) {
    for (int i = 0; i < 2; ++i) {
      if (cudaMallocHost(&p[i], bytes) != cudaSuccess) {
        cudaGetLastError();
        p[i] = nullptr;
        return fail(SV_ENOMEM, "pinned staging allocation of %zu bytes failed", bytes);
      }
      if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        ev[i] = nullptr;
        return fail(SV_ECUDA, "event creation failed");
      }
    }
    return SV_OK;
  }
};

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) std::fclose(f);
  }
};

}  // namespace
}  // namespace pr

using namespace pr;

extern "C" {

int sv_save(sv_state *sv, const char *path, uint64_t tag) {
  if (!sv || !path) return fail(SV_EINVAL, "NULL argument");
  const size_t total = amp_bytes(sv->dtype) << sv->n;
  const size_t chunk = total < kChunk ? total : kChunk;
  Pinned buf;
  int rc = buf.init(chunk);
  if (rc) return rc;
  const std::string tmp = std::string(path) + ".tmp";
  File out;
  out.f = std::fopen(tmp.c_str(), "wb");
  if (!out.f) return fail(SV_EIO, "cannot create %s: %s", tmp.c_str(), std::strerror(errno));
  unsigned char hdr[kHeader] = {0};
  if (std::fwrite(hdr, 1, kHeader, out.f) != kHeader) return fail(SV_EIO, "write to %s failed", tmp.c_str());

  // pipeline: copy chunk k to buffer k&1 while chunk k-1 is hashed and written
  const unsigned char *src = (const unsigned char *)sv->amps;
  const size_t n_chunks = (total + chunk - 1) / chunk;
  uint64_t h = kFnvBasis;
  auto issue = [&](size_t k) -> int {
    const size_t off = k * chunk, len = total - off < chunk ? total - off : chunk;
    PR_CUDA(cudaMemcpyAsync(buf.p[k & 1], src + off, len, cudaMemcpyDeviceToHost, sv->stream));
    PR_CUDA(cudaEventRecord(buf.ev[k & 1], sv->stream));
    return SV_OK;
  };
  rc = issue(0);
  for (size_t k = 0; k < n_chunks && rc == SV_OK; ++k) {
    PR_CUDA(cudaEventSynchronize(buf.ev[k & 1]));
    if (k + 1 < n_chunks) rc = issue(k + 1);
    if (rc) break;
    const size_t off = k * chunk, len = total - off < chunk ? total - off : chunk;
    h = fnv_words(h, (const unsigned char *)buf.p[k & 1], len);
    if (std::fwrite(buf.p[k & 1], 1, len, out.f) != len) rc = fail(SV_EIO, "write to %s failed", tmp.c_str());
  }
  if (rc) {
    cudaStreamSynchronize(sv->stream);
    std::fclose(out.f);
    out.f = nullptr;
    std::remove(tmp.c_str());
    return rc;
  }
  std::memcpy(hdr, kMagic, 8);
  put_u32(hdr + 8, kVersion);
  put_u32(hdr + 12, (uint32_t)sv->n);
  put_u32(hdr + 16, (uint32_t)sv->dtype);
  put_u32(hdr + 20, (uint32_t)(sv->frame.q & 3));
  put_u64(hdr + 24, sv->frame.x);
  put_u64(hdr + 32, sv->frame.z);
  put_u64(hdr + 40, tag);
  put_u64(hdr + 48, (uint64_t)total);
  put_u64(hdr + 56, h);
  put_u64(hdr + 64, fnv_words(kFnvBasis, hdr, 64));
  // on disk before the rename makes it the checkpoint
  const bool ok = std::fseek(out.f, 0, SEEK_SET) == 0 && std::fwrite(hdr, 1, kHeader, out.f) == kHeader &&
                  std::fflush(out.f) == 0 && fsync(fileno(out.f)) == 0;
  std::fclose(out.f);
  out.f = nullptr;
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(SV_EIO, "cannot write %s", path);
  }
  return SV_OK;
}

int sv_load(sv_state *sv, const char *path, uint64_t *out_tag) {
  if (!sv || !path) return fail(SV_EINVAL, "NULL argument");
  File in;
  in.f = std::fopen(path, "rb");
  if (!in.f) return fail(SV_EIO, "cannot open %s: %s", path, std::strerror(errno));
  unsigned char hdr[kHeader];
  if (std::fread(hdr, 1, kHeader, in.f) != kHeader) return fail(SV_EIO, "%s: truncated header", path);
  if (std::memcmp(hdr, kMagic, 8) != 0) return fail(SV_EINVAL, "%s is not a state checkpoint", path);
  if (get_u64(hdr + 64) != fnv_words(kFnvBasis, hdr, 64)) return fail(SV_EIO, "%s: header checksum mismatch", path);
  if (get_u32(hdr + 8) != kVersion) return fail(SV_EUNSUPPORTED, "%s: checkpoint version %u", path, get_u32(hdr + 8));
  const int n = (int)get_u32(hdr + 12), dtype = (int)get_u32(hdr + 16);
  if (n != sv->n || dtype != sv->dtype)
    return fail(SV_EINVAL, "%s holds n = %d dtype %d, the handle has n = %d dtype %d", path, n, dtype, sv->n,
                sv->dtype);
  const size_t total = amp_bytes(sv->dtype) << sv->n;
  if (get_u64(hdr + 48) != (uint64_t)total) return fail(SV_EIO, "%s: amplitude size mismatch", path);
  if (std::fseek(in.f, 0, SEEK_END) != 0) return fail(SV_EIO, "%s: cannot seek", path);
  const long end = std::ftell(in.f);
  if (end < 0 || (uint64_t)end != kHeader + (uint64_t)total)
    return fail(SV_EIO, "%s: file size %ld, expected %zu", path, end, kHeader + total);
  if (std::fseek(in.f, (long)kHeader, SEEK_SET) != 0) return fail(SV_EIO, "%s: cannot seek", path);
  Pauli f;
  f.x = get_u64(hdr + 24);
  f.z = get_u64(hdr + 32);
  f.q = (int)(get_u32(hdr + 20) & 3);
  const uint64_t lim = sv->n >= 64 ? ~0ULL : ((1ULL << sv->n) - 1);
  if ((f.x | f.z) & ~lim) return fail(SV_EIO, "%s: frame has bits at or above n", path);

  const size_t chunk = total < kChunk ? total : kChunk;
  Pinned buf;
  int rc = buf.init(chunk);
  if (rc) return rc;
  unsigned char *dst = (unsigned char *)sv->amps;
  const size_t n_chunks = (total + chunk - 1) / chunk;
  uint64_t h = kFnvBasis;
  for (size_t k = 0; k < n_chunks; ++k) {
    const size_t off = k * chunk, len = total - off < chunk ? total - off : chunk;
    if (k >= 2) PR_CUDA(cudaEventSynchronize(buf.ev[k & 1]));  // the buffer's previous copy is done
    if (std::fread(buf.p[k & 1], 1, len, in.f) != len) {
      cudaStreamSynchronize(sv->stream);
      return fail(SV_EIO, "%s: read failed", path);
    }
    h = fnv_words(h, (const unsigned char *)buf.p[k & 1], len);
    PR_CUDA(cudaMemcpyAsync(dst + off, buf.p[k & 1], len, cudaMemcpyHostToDevice, sv->stream));
    PR_CUDA(cudaEventRecord(buf.ev[k & 1], sv->stream));
  }
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  if (h != get_u64(hdr + 56)) return fail(SV_EIO, "%s: amplitude checksum mismatch", path);
  sv->frame = f;
  if (out_tag) *out_tag = get_u64(hdr + 40);
  return SV_OK;
}

}  // extern "C"
