// Fusion-depth autotuner.
//
// The planner's d_max bounds the dimension of the x-span fused into one pass
// (the coset runs of the fused pass).  A deeper span puts more rotations into
// each HBM sweep but gives every thread 2^d amplitudes and 2^d-way sign work,
// so the best d_max depends on the kernel variant (complex64 packs two cosets
// per thread up to d = 4), the state size and the rotation list.  The tuner
// times one rotation list compiled at every depth on the caller's state and
// records the fastest per (n, dtype); plan_create with fusion_depth = -1 then
// uses it.  A process-wide table holds the results; when PAULIROT_TUNE_CACHE
// names a file, the table is read from it before the first lookup and written
// back after every tuning call.  File format: one "<c64|c128> <n> <depth>" line
// per entry, '#' starts a comment line.
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.h"

namespace pr {
namespace {

using Key = std::pair<int, int>;  // (dtype, n)

std::mutex g_mu;
std::map<Key, int> g_table;
bool g_env_loaded = false;

const char *env_path() {
  const char *p = std::getenv("PAULIROT_TUNE_CACHE");
  return (p && *p) ? p : nullptr;
}

bool valid_entry(int dtype, int n, int depth) {
  return (dtype == SV_C128 || dtype == SV_C64) && n >= 1 && n <= max_qubits(dtype) && depth >= 1 &&
         depth <= kDMax;
}

// Parse a cache file into out (replacing nothing on error).  A missing file is
// an empty table.
int read_file(const char *path, std::map<Key, int> *out) {
  FILE *f = std::fopen(path, "r");
  if (!f) {
    if (errno == ENOENT) return SV_OK;
    return fail(SV_EINVAL, "cannot open tune cache %s: %s", path, std::strerror(errno));
  }
  std::map<Key, int> t;
  char line[256];
  int lineno = 0;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    const char *s = line;
    while (*s == ' ' || *s == '\t') ++s;
    if (*s == '#' || *s == '\n' || *s == '\r' || *s == 0) continue;
    char name[8] = {0};
    int n = 0, depth = 0;
    char extra = 0;
    if (std::sscanf(s, "%7s %d %d %c", name, &n, &depth, &extra) != 3) {
      std::fclose(f);
      return fail(SV_EINVAL, "tune cache %s line %d is malformed", path, lineno);
    }
    int dtype = std::strcmp(name, "c64") == 0 ? SV_C64 : std::strcmp(name, "c128") == 0 ? SV_C128 : -1;
    if (!valid_entry(dtype, n, depth)) {
      std::fclose(f);
      return fail(SV_EINVAL, "tune cache %s line %d has an invalid entry", path, lineno);
    }
    t[Key(dtype, n)] = depth;
  }
  std::fclose(f);
  for (const auto &kv : t) (*out)[kv.first] = kv.second;
  return SV_OK;
}

// Write the table to path (through a temporary file of this process renamed
// over it, so processes that tune at the same time never mix their writes).
int write_file(const char *path, const std::map<Key, int> &t) {
  std::string tmp = std::string(path) + ".tmp." + std::to_string((long)getpid());
  FILE *f = std::fopen(tmp.c_str(), "w");
  if (!f) return fail(SV_EINVAL, "cannot write tune cache %s: %s", tmp.c_str(), std::strerror(errno));
  std::fprintf(f, "# fusion depth per (dtype, n): <dtype> <n> <depth>\n");
  for (const auto &kv : t)
    std::fprintf(f, "%s %d %d\n", kv.first.first == SV_C64 ? "c64" : "c128", kv.first.second, kv.second);
  const bool ok = std::fflush(f) == 0;
  std::fclose(f);
  if (!ok || std::rename(tmp.c_str(), path) != 0) {
    std::remove(tmp.c_str());
    return fail(SV_EINVAL, "cannot write tune cache %s", path);
  }
  return SV_OK;
}

void load_env_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  if (const char *p = env_path()) read_file(p, &g_table);  // an unreadable cache is an empty one
}

}  // namespace

int tuned_depth(int n, int dtype) {
  std::lock_guard<std::mutex> lk(g_mu);
  load_env_locked();
  auto it = g_table.find(Key(dtype, n));
  return it == g_table.end() ? -1 : it->second;
}

}  // namespace pr

using namespace pr;

extern "C" {

int plan_tuned_depth(int n_qubits, int dtype, int *out_depth, int *out_tuned) {
  if (!out_depth) return fail(SV_EINVAL, "out_depth is NULL");
  if (dtype != SV_C128 && dtype != SV_C64) return fail(SV_EINVAL, "bad dtype");
  if (n_qubits < 1 || n_qubits > max_qubits(dtype)) return fail(SV_EINVAL, "bad n_qubits %d", n_qubits);
  const int t = tuned_depth(n_qubits, dtype);
  int d = t > 0 ? t : default_depth(dtype);
  if (d > n_qubits) d = n_qubits;
  *out_depth = d;
  if (out_tuned) *out_tuned = t > 0;
  return SV_OK;
}

int plan_set_tuned_depth(int n_qubits, int dtype, int depth) {
  if (dtype != SV_C128 && dtype != SV_C64) return fail(SV_EINVAL, "bad dtype");
  if (n_qubits < 1 || n_qubits > max_qubits(dtype)) return fail(SV_EINVAL, "bad n_qubits %d", n_qubits);
  if (depth != -1 && (depth < 1 || depth > kDMax)) return fail(SV_EINVAL, "depth must be -1 or 1..%d", kDMax);
  std::lock_guard<std::mutex> lk(g_mu);
  load_env_locked();
  if (depth < 0)
    g_table.erase(Key(dtype, n_qubits));
  else
    g_table[Key(dtype, n_qubits)] = depth;
  return SV_OK;
}

int plan_tune_cache_load(const char *path) {
  if (!path) return fail(SV_EINVAL, "path is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  g_env_loaded = true;  // an explicit load takes the place of the environment's
  return read_file(path, &g_table);
}

int plan_tune_cache_save(const char *path) {
  if (!path) return fail(SV_EINVAL, "path is NULL");
  std::lock_guard<std::mutex> lk(g_mu);
  load_env_locked();
  return write_file(path, g_table);
}

int plan_autotune(sv_state *sv, const uint64_t *x, const uint64_t *z, const double *angles, size_t count,
                  int max_depth, int reps, int *out_depth, double *out_ms) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (!out_depth) return fail(SV_EINVAL, "out_depth is NULL");
  if (count == 0) return fail(SV_EINVAL, "an empty rotation list cannot be timed");
  if (max_depth <= 0 || max_depth > kDMax) max_depth = kDMax;
  if (max_depth > sv->n) max_depth = sv->n;
  if (reps <= 0) reps = 3;
  if (out_ms)
    for (int d = 0; d < kDMax; ++d) out_ms[d] = -1.0;

  // compile every depth first: a bad list fails before any device work
  sv_plan *plans[kDMax] = {nullptr};
  auto release = [&]() {
    for (int d = 0; d < kDMax; ++d)
      if (plans[d]) plan_free(plans[d]);
  };
  for (int d = 1; d <= max_depth; ++d) {
    int rc = plan_create(&plans[d - 1], sv->n, sv->dtype, x, z, angles, count, d, sv->stream);
    if (rc) {
      release();
      return rc;
    }
  }
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaGetLastError();
    if (ev[0]) cudaEventDestroy(ev[0]);
    release();
    return fail(SV_ECUDA, "event creation failed");
  }
  double best_ms[kDMax];
  for (int d = 0; d < kDMax; ++d) best_ms[d] = -1.0;
  int rc = SV_OK;
  // one warm-up application per depth, then two timed rounds over all depths
  // (interleaved, so a clock change mid-way hits every depth), minimum per depth
  for (int round = 0; round < 3 && rc == SV_OK; ++round) {
    for (int d = 1; d <= max_depth && rc == SV_OK; ++d) {
      const int k = round == 0 ? 1 : reps;
      if (round > 0 && cudaEventRecord(ev[0], sv->stream) != cudaSuccess) rc = fail(SV_ECUDA, "event record");
      for (int r = 0; r < k && rc == SV_OK; ++r) rc = apply_plan(sv, plans[d - 1]);
      if (rc || round == 0) continue;
      if (cudaEventRecord(ev[1], sv->stream) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess) {
        rc = fail(SV_ECUDA, "event wait: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      const double per = (double)ms / k;
      if (best_ms[d - 1] < 0.0 || per < best_ms[d - 1]) best_ms[d - 1] = per;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  release();
  if (rc) return rc;

  int best = 1;
  for (int d = 2; d <= max_depth; ++d)
    if (best_ms[d - 1] < best_ms[best - 1]) best = d;
  if (out_ms)
    for (int d = 0; d < kDMax; ++d) out_ms[d] = best_ms[d];
  *out_depth = best;
  std::lock_guard<std::mutex> lk(g_mu);
  load_env_locked();
  g_table[Key(sv->dtype, sv->n)] = best;
  if (const char *p = env_path()) return write_file(p, g_table);
  return SV_OK;
}

int batch_autotune(sv_state **states, const uint64_t *const *x, const uint64_t *const *z,
                   const double *const *angles, const size_t *counts, size_t count, int max_depth, int reps,
                   int use_graph, int *out_depth, double *out_ms) {
  constexpr int kBatchDMax = 4;
  if (!states || !x || !z || !angles || !counts || !out_depth) return fail(SV_EINVAL, "NULL argument");
  if (count == 0) return fail(SV_EINVAL, "empty batch");
  for (size_t i = 0; i < count; ++i)
    if (!states[i]) return fail(SV_EINVAL, "state %zu is NULL", i);
  if (max_depth <= 0 || max_depth > kBatchDMax) max_depth = kBatchDMax;
  if (reps <= 0) reps = 3;
  if (out_ms)
    for (int d = 0; d < kBatchDMax; ++d) out_ms[d] = -1.0;
  std::vector<sv_plan *> plans(count * (size_t)max_depth, nullptr);
  auto release = [&]() {
    for (sv_plan *p : plans)
      if (p) plan_free(p);
  };
  // compile everything first: a bad list fails before any device work
  for (int d = 1; d <= max_depth; ++d)
    for (size_t i = 0; i < count; ++i) {
      const int dd = d < states[i]->n ? d : states[i]->n;
      int rc = plan_create(&plans[(size_t)(d - 1) * count + i], states[i]->n, states[i]->dtype, x[i], z[i],
                           angles[i], counts[i], dd, states[i]->stream);
      if (rc) {
        release();
        return rc;
      }
    }
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (cudaEventCreate(&ev[0]) != cudaSuccess || cudaEventCreate(&ev[1]) != cudaSuccess) {
    cudaGetLastError();
    if (ev[0]) cudaEventDestroy(ev[0]);
    release();
    return fail(SV_ECUDA, "event creation failed");
  }
  cudaStream_t s = states[0]->stream;
  double best_ms[kBatchDMax];
  for (int d = 0; d < kBatchDMax; ++d) best_ms[d] = -1.0;
  int rc = SV_OK;
  for (int d = 1; d <= max_depth && rc == SV_OK; ++d) {
    sv_plan **pl = plans.data() + (size_t)(d - 1) * count;
    rc = batch_run(states, pl, count, use_graph);  // builds (and captures) this set, warms
    for (int r = 0; r < reps && rc == SV_OK; ++r) {
      if (cudaEventRecord(ev[0], s) != cudaSuccess) {
        rc = fail(SV_ECUDA, "event record");
        break;
      }
      rc = batch_run(states, pl, count, use_graph);  // synchronises the stream
      if (rc) break;
      if (cudaEventRecord(ev[1], s) != cudaSuccess || cudaEventSynchronize(ev[1]) != cudaSuccess) {
        rc = fail(SV_ECUDA, "event wait: %s", cudaGetErrorString(cudaGetLastError()));
        break;
      }
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
      if (best_ms[d - 1] < 0.0 || ms < best_ms[d - 1]) best_ms[d - 1] = ms;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  release();
  if (rc) return rc;
  int best = 1;
  for (int d = 2; d <= max_depth; ++d)
    if (best_ms[d - 1] < best_ms[best - 1]) best = d;
  if (out_ms)
    for (int d = 0; d < kBatchDMax; ++d) out_ms[d] = best_ms[d];
  *out_depth = best;
  std::lock_guard<std::mutex> lk(g_mu);
  load_env_locked();
  for (size_t i = 0; i < count; ++i) g_table[Key(states[i]->dtype, states[i]->n)] = best;
  if (const char *p = env_path()) return write_file(p, g_table);
  return SV_OK;
}

}  // extern "C"
