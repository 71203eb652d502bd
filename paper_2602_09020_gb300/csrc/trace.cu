// CUDA-event tracing for a state handle: an event pair around every launch, or
// (block mode) one event wherever the kernel changes, so consecutive launches of
// one kernel keep running back to back (chained passes overlap) and their
// average time is the block's time over its launches.
#include <cstring>

#include "internal.h"

namespace pr {

static const char *kNames[KN_COUNT] = {
    "k_coset_d0", "k_coset_d1", "k_coset_d2", "k_coset_d3", "k_coset_d4", "k_coset_d5",
    "k_diag_sum", "k_expval", "k_finish", "k_pauli_sum", "k_materialize", "k_set_one",
    "k_adjoint_step", "k_sum_rows", "k_hadamard", "k_diag1", "k_cnot", "k_project", "k_adjoint_run", "k_chain2"};

static int next_event(sv_state *sv) {
  if (sv->events_used == (int)sv->events.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    sv->events.push_back(e);
  }
  return sv->events_used++;
}

int trace_begin(sv_state *sv, int name) {
  if (sv && sv->trace_owner) sv = sv->trace_owner;
  if (!sv || !sv->tracing) return -1;
  if (sv->trace_blocks) {
    // one event where the kernel changes: it ends the open block and opens the next
    if (!sv->trace.empty() && sv->trace.back().name == name) return (int)sv->trace.size() - 1;
    int e = next_event(sv);
    if (e < 0) return -1;
    cudaEventRecord(sv->events[e], sv->stream);
    if (!sv->trace.empty()) sv->trace.back().ev1 = e;
    sv->trace.push_back(TraceRec{name, 0.0, 0.0, e, -1, 0});
    return (int)sv->trace.size() - 1;
  }
  int s = next_event(sv);
  if (s < 0) return -1;
  cudaEventRecord(sv->events[s], sv->stream);
  return s;
}

void trace_end(sv_state *sv, int slot, int name, double bytes, double flops) {
  if (sv && sv->trace_owner) sv = sv->trace_owner;
  if (!sv || !sv->tracing || slot < 0) return;
  if (sv->trace_blocks) {
    TraceRec &r = sv->trace[slot];
    r.bytes += bytes;
    r.flops += flops;
    r.launches += 1;
    return;
  }
  int e = next_event(sv);
  if (e < 0) return;
  cudaEventRecord(sv->events[e], sv->stream);
  sv->trace.push_back(TraceRec{name, bytes, flops, slot, e, 1});
}

void trace_release(sv_state *sv) {
  for (cudaEvent_t e : sv->events) cudaEventDestroy(e);
  sv->events.clear();
  sv->events_used = 0;
  sv->trace.clear();
}

}  // namespace pr

using namespace pr;

extern "C" {

int sv_trace_start_ex(sv_state *sv, int mode) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  if (mode != SV_TRACE_LAUNCHES && mode != SV_TRACE_BLOCKS) return fail(SV_EINVAL, "bad trace mode %d", mode);
  sv->tracing = true;
  sv->trace_blocks = mode == SV_TRACE_BLOCKS;
  sv->events_used = 0;
  sv->trace.clear();
  return SV_OK;
}

int sv_trace_start(sv_state *sv) { return sv_trace_start_ex(sv, SV_TRACE_LAUNCHES); }

int sv_trace_stop(sv_state *sv, sv_trace_row *rows, int cap, int *n_rows) {
  if (!sv) return fail(SV_EINVAL, "sv is NULL");
  sv->tracing = false;
  if (sv->trace_blocks && !sv->trace.empty()) {
    // close the last block
    const int e = next_event(sv);
    if (e < 0) {
      sv->trace.clear();
      sv->events_used = 0;
      return fail(SV_ECUDA, "event creation failed");
    }
    PR_CUDA(cudaEventRecord(sv->events[e], sv->stream));
    sv->trace.back().ev1 = e;
  }
  PR_CUDA(cudaStreamSynchronize(sv->stream));
  double ms[KN_COUNT] = {0};
  double by[KN_COUNT] = {0};
  double fl[KN_COUNT] = {0};
  int64_t cnt[KN_COUNT] = {0};
  for (const TraceRec &r : sv->trace) {
    float t = 0.f;
    PR_CUDA(cudaEventElapsedTime(&t, sv->events[r.ev0], sv->events[r.ev1]));
    ms[r.name] += t;
    by[r.name] += r.bytes;
    fl[r.name] += r.flops;
    cnt[r.name] += r.launches;
  }
  int w = 0;
  for (int k = 0; k < KN_COUNT; ++k) {
    if (!cnt[k]) continue;
    if (rows && w < cap) {
      std::memset(&rows[w], 0, sizeof(sv_trace_row));
      std::strncpy(rows[w].name, kNames[k], sizeof(rows[w].name) - 1);
      rows[w].launches = cnt[k];
      rows[w].total_ms = ms[k];
      rows[w].bytes = by[k];
      rows[w].flops = fl[k];
    }
    ++w;
  }
  if (n_rows) *n_rows = w < cap ? w : cap;
  sv->trace.clear();
  sv->events_used = 0;
  return SV_OK;
}

}  // extern "C"
