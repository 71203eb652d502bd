// Batched independent states in one persistent launch (not in the paper).
//
// Each CTA of a cooperative grid gets a list of work items (state, rank, group):
// it runs every pass of that state's plan on its share (rank of group CTAs) of
// the index space.  States small enough for one CTA are packed onto CTAs by
// longest-processing-time first; larger states get a contiguous range of CTAs
// and those CTAs meet at a per-state barrier between passes.  A CTA's
// multi-CTA item always comes first in its list, so every CTA reaches its
// state's barriers without waiting behind unrelated work.  Every barrier wait
// is bounded (wall clock from %globaltimer): a CTA that gives up sets the error
// word and leaves; its peers see the word or run out of time too, and the host
// reports SV_ETIMEOUT.  No wait is unbounded.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <queue>
#include <vector>

#include "coset_fx.cuh"
#include "kernels.cuh"

namespace pr {

namespace {

struct BatchStateDev {
  void *amps;
  uint64_t fx, fz;
  const RunDev *runs;
  const RotDev *rots;
  const DiagDev *diag;
  const void *tab;
  int n;
  int n_runs;
};

struct BatchItemDev {
  int state;
  int rank;
  int group;
  int pad;
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Arrive at the state's barrier and wait (bounded) until target arrivals.
// Returns false if this CTA must stop (timeout here or an error elsewhere).
__device__ bool state_barrier(unsigned *ctr, unsigned target, unsigned long long timeout_ns, int *err,
                              bool skip_arrival) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (!skip_arrival) atomicAdd(ctr, 1u);
    const unsigned long long t0 = global_ns();
    int ok = 1;
    for (;;) {
      if (atomicAdd(ctr, 0u) >= target) break;
      if (atomicAdd(err, 0) != 0) {
        ok = 0;
        break;
      }
      if (global_ns() - t0 > timeout_ns) {
        atomicCAS(err, 0, 1);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

template <typename Idx>
__device__ __forceinline__ bool c64x2_ok(int n, const RunDev &run) {
  return run.d <= 4 && n - run.d >= 1 && (run.d == 0 || run.piv[0] >= 1);
}

template <typename R, typename Idx>
__device__ void run_pass(const BatchStateDev &st, const RunDev &run, Idx rank, Idx group, char *ws) {
  using C = typename Cx<R>::T;
  const uint64_t n_amps = 1ULL << st.n;
  if (run.kind == 1) {
    body_diag<R, Idx>((C *)st.amps, (Idx)(n_amps >> kDiagClassBits), run, st.diag, st.fx, (const C *)st.tab, rank,
                      group, ws);
    return;
  }
  if constexpr (sizeof(R) == 4) {
    if (c64x2_ok<Idx>(st.n, run)) {
      float4 *a4 = (float4 *)st.amps;
      const Idx np = (Idx)(((n_amps) >> run.d) >> 1);
      switch (run.d) {
        case 0: body_c64x2<Idx, 0>(a4, np, run, st.rots, st.fx, st.fz, rank, group, ws); return;
        case 1: body_c64x2<Idx, 1>(a4, np, run, st.rots, st.fx, st.fz, rank, group, ws); return;
        case 2: body_c64x2<Idx, 2>(a4, np, run, st.rots, st.fx, st.fz, rank, group, ws); return;
        case 3: body_c64x2<Idx, 3>(a4, np, run, st.rots, st.fx, st.fz, rank, group, ws); return;
        default: body_c64x2<Idx, 4>(a4, np, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      }
    }
  }
  const Idx nc = (Idx)(n_amps >> run.d);
  if constexpr (sizeof(R) == 8) {
    // complex128: the fixed-point body of the single-state passes (same results bit for bit)
    double2 *a = (double2 *)st.amps;
    switch (run.d) {
      case 0: body_coset_fx<Idx, 0, 2>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 1: body_coset_fx<Idx, 1, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 2: body_coset_fx<Idx, 2, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 3: body_coset_fx<Idx, 3, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      default: body_coset_fx<Idx, 4, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
    }
  } else {
    C *a = (C *)st.amps;
    switch (run.d) {
      case 0: body_coset<R, Idx, 0, 4>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 1: body_coset<R, Idx, 1, 2>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 2: body_coset<R, Idx, 2, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      case 3: body_coset<R, Idx, 3, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
      default: body_coset<R, Idx, 4, 1>(a, nc, run, st.rots, st.fx, st.fz, rank, group, ws); return;
    }
  }
}

template <typename R, typename Idx>
__global__ void __launch_bounds__(kThreads)
    k_batch(const BatchStateDev *__restrict__ states, const BatchItemDev *__restrict__ items,
            const int *__restrict__ cta_first, unsigned *__restrict__ bars, int *__restrict__ err,
            unsigned long long timeout_ns, int skip_state) {
  extern __shared__ __align__(16) char ws[];
  __shared__ RunDev s_run;
  __shared__ BatchStateDev s_st;
  for (int it = cta_first[blockIdx.x]; it < cta_first[blockIdx.x + 1]; ++it) {
    const BatchItemDev item = items[it];
    if (threadIdx.x == 0) s_st = states[item.state];
    __syncthreads();
    const int n_runs = s_st.n_runs;
    for (int r = 0; r < n_runs; ++r) {
      if (threadIdx.x == 0) s_run = s_st.runs[r];
      __syncthreads();
      run_pass<R, Idx>(s_st, s_run, (Idx)item.rank, (Idx)item.group, ws);
      if (item.group > 1 && r + 1 < n_runs) {
        const bool skip = item.state == skip_state && item.rank == 0 && r == 0;
        if (!state_barrier(&bars[item.state], (unsigned)((r + 1) * item.group), timeout_ns, err, skip)) {
          // nothing of ours is in flight: every pass body drains its copies
          return;
        }
      }
    }
    __syncthreads();
  }
}

template <typename R, typename Idx>
constexpr size_t batch_ws() {
  if constexpr (sizeof(R) == 4) {
    size_t a = ws_c64x2<Idx, 4>(), b = ws_coset<R, Idx, 4>(), c = ws_diag<R, Idx>();
    return std::max(a, std::max(b, c));
  } else {
    return std::max(ws_coset_fx<Idx, 4>(), ws_diag<R, Idx>());
  }
}

// ------------------------------------------------------------------ host side

struct BatchCache {
  std::vector<sv_state *> states;
  std::vector<sv_plan *> plans;
  int dtype = -1;
  bool narrow = true;
  int grid = 0;
  size_t ws = 0;
  BatchStateDev *h_states = nullptr;  // pinned: frames refreshed every call
  BatchStateDev *d_states = nullptr;
  BatchItemDev *d_items = nullptr;
  int *d_cta_first = nullptr;
  RunDev *d_runs = nullptr;
  unsigned *d_bars = nullptr;
  int *d_err = nullptr;
  int *h_err = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaStream_t stream = nullptr;
  unsigned long long timeout_ns = 0;
  int skip_state = -1;
  int multi_cta_states = 0;
  bool graph_ok = true;
  int capture_error = 0;     // cudaError_t of the first failed capture step (0 = none)

  void release() {
    if (graph) cudaGraphExecDestroy(graph);
    if (h_states) cudaFreeHost(h_states);
    if (h_err) cudaFreeHost(h_err);
    if (d_states) cudaFree(d_states);
    if (d_items) cudaFree(d_items);
    if (d_cta_first) cudaFree(d_cta_first);
    if (d_runs) cudaFree(d_runs);
    if (d_bars) cudaFree(d_bars);
    if (d_err) cudaFree(d_err);
    graph = nullptr;
    h_states = nullptr;
    h_err = nullptr;
    d_states = nullptr;
    d_items = nullptr;
    d_cta_first = nullptr;
    d_runs = nullptr;
    d_bars = nullptr;
    d_err = nullptr;
  }
};

BatchCache g_batch;
std::mutex g_batch_mu;  // guards g_batch: one batched launch at a time

template <typename R, typename Idx>
int batch_grid(size_t *ws_out) {
  const size_t ws = batch_ws<R, Idx>();
  PR_CUDA(cudaFuncSetAttribute(k_batch<R, Idx>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ws));
  int per_sm = 0;
  PR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch<R, Idx>, kThreads, ws));
  if (per_sm < 1) return fail(SV_EUNSUPPORTED, "batched kernel does not fit on an SM");
  *ws_out = ws;
  return per_sm * device_sm_count();
}

template <typename R, typename Idx>
int batch_launch(BatchCache &b, cudaStream_t s) {
  void *args[] = {(void *)&b.d_states, (void *)&b.d_items, (void *)&b.d_cta_first, (void *)&b.d_bars,
                  (void *)&b.d_err, (void *)&b.timeout_ns, (void *)&b.skip_state};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)b.grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = b.ws;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  PR_CUDA(cudaLaunchKernelExC(&cfg, (const void *)k_batch<R, Idx>, args));
  return SV_OK;
}

int launch_by_type(BatchCache &b, cudaStream_t s) {
  if (b.dtype == SV_C64) return b.narrow ? batch_launch<float, uint32_t>(b, s) : batch_launch<float, uint64_t>(b, s);
  return b.narrow ? batch_launch<double, uint32_t>(b, s) : batch_launch<double, uint64_t>(b, s);
}

int enqueue(BatchCache &b, cudaStream_t s) {
  const size_t n = b.states.size();
  PR_CUDA(cudaMemcpyAsync(b.d_states, b.h_states, sizeof(BatchStateDev) * n, cudaMemcpyHostToDevice, s));
  PR_CUDA(cudaMemsetAsync(b.d_bars, 0, sizeof(unsigned) * n, s));
  PR_CUDA(cudaMemsetAsync(b.d_err, 0, sizeof(int), s));
  return launch_by_type(b, s);
}

double batch_cost(int n, size_t rotations, size_t passes) {
  return (double)(1ULL << n) * ((double)rotations + 4.0 * (double)passes);
}

// Assign work items to CTAs.  cost ~ amplitudes x (rotations + 4 passes): a
// pass costs about as much as four of its rotations beyond the rotations
// themselves.  States of n >= 16 whose cost exceeds one CTA's share are split
// over several CTAs; how many is decided greedily against the largest load
// per CTA: start from floor(cost / share), then hand out the CTAs left after
// the single-CTA states' needs one at a time to the state with the largest
// load per CTA (or take them back from the state whose load per CTA grows
// least), so no split state ends up far above the average.
void assign(const std::vector<double> &cost, const std::vector<int> &n, int grid, std::vector<BatchItemDev> &items,
            std::vector<int> &cta_first, int &multi) {
  const size_t S = cost.size();
  double total = 0.0;
  for (double c : cost) total += c;
  const double share = total / grid;
  std::vector<int> g(S, 1);
  std::vector<size_t> big;
  double small_total = 0.0;
  for (size_t i = 0; i < S; ++i) {
    if (cost[i] > share && n[i] >= 16) {
      g[i] = std::max(1, (int)(cost[i] / share));
      big.push_back(i);
    } else {
      small_total += cost[i];
    }
  }
  int limit = grid - (small_total > 0.0 ? (int)std::ceil(small_total / share) : 0);
  limit = std::max(limit, (int)big.size());
  int used = 0;
  for (size_t i : big) used += g[i];
  while (!big.empty() && used < limit) {
    size_t best = big[0];
    for (size_t i : big)
      if (cost[i] / g[i] > cost[best] / g[best]) best = i;
    ++g[best];
    ++used;
  }
  while (used > limit) {
    size_t best = S;
    for (size_t i : big)
      if (g[i] > 1 && (best == S || cost[i] / (g[i] - 1) < cost[best] / (g[best] - 1))) best = i;
    if (best == S) break;
    --g[best];
    --used;
  }
  std::vector<std::vector<BatchItemDev>> per_cta(grid);
  std::vector<double> load(grid, 0.0);
  int next = 0;
  multi = 0;
  for (size_t i : big) {
    if (g[i] > 1) ++multi;
    for (int k = 0; k < g[i]; ++k) {
      per_cta[next].push_back({(int)i, k, g[i], 0});
      load[next] += cost[i] / g[i];
      ++next;
    }
  }
  std::vector<size_t> small;
  for (size_t i = 0; i < S; ++i)
    if (std::find(big.begin(), big.end(), i) == big.end()) small.push_back(i);
  std::sort(small.begin(), small.end(), [&](size_t a, size_t b2) { return cost[a] > cost[b2]; });
  using Slot = std::pair<double, int>;
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> pq;
  for (int c = 0; c < grid; ++c) pq.push({load[c], c});
  for (size_t i : small) {
    Slot sl = pq.top();
    pq.pop();
    per_cta[sl.second].push_back({(int)i, 0, 1, 0});
    sl.first += cost[i];
    pq.push(sl);
  }
  items.clear();
  cta_first.assign(grid + 1, 0);
  for (int c = 0; c < grid; ++c) {
    cta_first[c] = (int)items.size();
    for (const auto &it : per_cta[c]) items.push_back(it);
  }
  cta_first[grid] = (int)items.size();
}

int build_cache(BatchCache &b, sv_state **states, sv_plan **plans, size_t count, const sv_batch_opts *opts) {
  b.release();
  b.states.assign(states, states + count);
  b.plans.assign(plans, plans + count);
  b.dtype = states[0]->dtype;
  b.narrow = true;
  for (size_t i = 0; i < count; ++i) b.narrow = b.narrow && states[i]->n <= 31;
  int grid = 0;
  size_t ws = 0;
  if (b.dtype == SV_C64)
    grid = b.narrow ? batch_grid<float, uint32_t>(&ws) : batch_grid<float, uint64_t>(&ws);
  else
    grid = b.narrow ? batch_grid<double, uint32_t>(&ws) : batch_grid<double, uint64_t>(&ws);
  if (grid < 0) return grid;
  b.grid = grid;
  b.ws = ws;
  // runs of every plan in one device array
  std::vector<RunDev> runs;
  std::vector<size_t> off(count);
  for (size_t i = 0; i < count; ++i) {
    off[i] = runs.size();
    runs.insert(runs.end(), plans[i]->runs.begin(), plans[i]->runs.end());
  }
  if (runs.empty()) runs.push_back(RunDev());
  PR_CUDA(cudaMalloc(&b.d_runs, sizeof(RunDev) * runs.size()));
  PR_CUDA(cudaMemcpy(b.d_runs, runs.data(), sizeof(RunDev) * runs.size(), cudaMemcpyHostToDevice));
  PR_CUDA(cudaMallocHost(&b.h_states, sizeof(BatchStateDev) * count));
  PR_CUDA(cudaMalloc(&b.d_states, sizeof(BatchStateDev) * count));
  std::vector<double> cost(count);
  std::vector<int> nq(count);
  for (size_t i = 0; i < count; ++i) {
    const void *tab = nullptr;
    int rc = prepare_tables(b.dtype);
    if (rc) return rc;
    rc = table_pointer(b.dtype, &tab);
    if (rc) return rc;
    BatchStateDev &d = b.h_states[i];
    d.amps = states[i]->amps;
    d.fx = states[i]->frame.x;
    d.fz = states[i]->frame.z;
    d.runs = b.d_runs + off[i];
    d.rots = plans[i]->d_rots;
    d.diag = plans[i]->d_diag;
    d.tab = tab;
    d.n = states[i]->n;
    d.n_runs = (int)plans[i]->runs.size();
    cost[i] = batch_cost(states[i]->n, plans[i]->n_effective, (size_t)d.n_runs + 1);
    nq[i] = states[i]->n;
  }
  std::vector<BatchItemDev> items;
  std::vector<int> cta_first;
  assign(cost, nq, grid, items, cta_first, b.multi_cta_states);
  if (items.empty()) items.push_back(BatchItemDev());
  PR_CUDA(cudaMalloc(&b.d_items, sizeof(BatchItemDev) * items.size()));
  PR_CUDA(cudaMemcpy(b.d_items, items.data(), sizeof(BatchItemDev) * items.size(), cudaMemcpyHostToDevice));
  PR_CUDA(cudaMalloc(&b.d_cta_first, sizeof(int) * cta_first.size()));
  PR_CUDA(cudaMemcpy(b.d_cta_first, cta_first.data(), sizeof(int) * cta_first.size(), cudaMemcpyHostToDevice));
  PR_CUDA(cudaMalloc(&b.d_bars, sizeof(unsigned) * count));
  PR_CUDA(cudaMalloc(&b.d_err, sizeof(int)));
  PR_CUDA(cudaMallocHost(&b.h_err, sizeof(int)));
  const double t = (opts && opts->wait_timeout_s > 0) ? opts->wait_timeout_s : 1.0;
  b.timeout_ns = (unsigned long long)(t * 1e9);
  b.skip_state = -1;
  if (opts && opts->test_skip_arrival) {
    // the first state that spans several CTAs
    for (size_t i = 0; i < items.size(); ++i)
      if (items[i].group > 1) {
        b.skip_state = items[i].state;
        break;
      }
  }
  b.graph_ok = true;
  return SV_OK;
}

bool same_set(const BatchCache &b, sv_state **states, sv_plan **plans, size_t count, const sv_batch_opts *opts) {
  if (b.states.size() != count || !b.h_states) return false;
  for (size_t i = 0; i < count; ++i)
    if (b.states[i] != states[i] || b.plans[i] != plans[i] || b.h_states[i].amps != states[i]->amps) return false;
  const double t = (opts && opts->wait_timeout_s > 0) ? opts->wait_timeout_s : 1.0;
  if (b.timeout_ns != (unsigned long long)(t * 1e9)) return false;
  if ((opts && opts->test_skip_arrival) != (b.skip_state >= 0)) return false;
  return true;
}

}  // namespace

// drop the cached batch if it refers to a handle that is being freed
void batch_forget(const sv_state *sv, const sv_plan *plan) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchCache &b = g_batch;
  bool hit = false;
  for (auto *s : b.states) hit = hit || (sv && s == sv);
  for (auto *p : b.plans) hit = hit || (plan && p == plan);
  if (hit) {
    b.release();
    b.states.clear();
    b.plans.clear();
  }
}

}  // namespace pr

using namespace pr;

extern "C" {

int batch_run_ex(sv_state **states, sv_plan **plans, size_t count, int use_graph, const sv_batch_opts *opts) {
  if (count == 0) return SV_OK;
  if (!states || !plans) return fail(SV_EINVAL, "NULL arrays");
  for (size_t i = 0; i < count; ++i) {
    if (!states[i] || !plans[i]) return fail(SV_EINVAL, "NULL entry %zu", i);
    if (states[i]->n != plans[i]->n || states[i]->dtype != plans[i]->dtype)
      return fail(SV_EINVAL, "plan %zu does not match its state", i);
    if (states[i]->dtype != states[0]->dtype) return fail(SV_EINVAL, "all states must have one dtype");
    for (const RunDev &r : plans[i]->runs)
      if (r.kind == 0 && r.d > 4) return fail(SV_EUNSUPPORTED, "batched plans need fusion_depth <= 4 (plan %zu)", i);
    for (size_t j = 0; j < i; ++j)
      if (states[j]->amps == states[i]->amps) return fail(SV_EINVAL, "state %zu appears twice", i);
  }
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchCache &b = g_batch;
  int rc = SV_OK;
  if (!same_set(b, states, plans, count, opts)) {
    rc = build_cache(b, states, plans, count, opts);
    if (rc) {
      b.release();
      b.states.clear();
      return rc;
    }
  }
  for (size_t i = 0; i < count; ++i) {
    b.h_states[i].fx = states[i]->frame.x;
    b.h_states[i].fz = states[i]->frame.z;
  }
  cudaStream_t s = states[0]->stream;
  if (use_graph && s != nullptr && b.graph_ok) {
    // capture the cooperative launch once.  A plain launch of the same grid is
    // never captured instead: its per-state barriers would rely on every CTA
    // being resident together, which only the cooperative launch guarantees;
    // when the capture fails the cooperative launch runs without a graph.
    if (!b.graph) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
      if (e == cudaSuccess) {
        const int erc = enqueue(b, s);
        cudaError_t e2 = cudaStreamEndCapture(s, &g);
        if (erc || e2 != cudaSuccess || !g) {
          cudaError_t le = cudaGetLastError();
          if (!b.capture_error) b.capture_error = (int)(e2 != cudaSuccess ? e2 : (le != cudaSuccess ? le : cudaErrorUnknown));
          if (g) cudaGraphDestroy(g);
          g = nullptr;
        } else {
          e = cudaGraphInstantiate(&b.graph, g, 0);
          cudaGraphDestroy(g);
          if (e != cudaSuccess) {
            if (!b.capture_error) b.capture_error = (int)e;
            cudaGetLastError();
            b.graph = nullptr;
          }
        }
      } else {
        if (!b.capture_error) b.capture_error = (int)e;
        cudaGetLastError();
      }
      if (!b.graph) b.graph_ok = false;
    }
    if (b.graph) {
      PR_CUDA(cudaGraphLaunch(b.graph, s));
    } else {
      rc = enqueue(b, s);
      if (rc) return rc;
    }
  } else {
    rc = enqueue(b, s);
    if (rc) return rc;
  }
  PR_CUDA(cudaMemcpyAsync(b.h_err, b.d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PR_CUDA(cudaStreamSynchronize(s));
  if (*b.h_err) return fail(SV_ETIMEOUT, "a batched barrier wait ran out of time (%.3f s)", b.timeout_ns * 1e-9);
  for (size_t i = 0; i < count; ++i) {
    const Pauli q0 = states[i]->frame;
    Pauli f = pauli_mul(q0, plans[i]->frame);
    if (anticommute(plans[i]->frame.x, plans[i]->frame.z, q0.x, q0.z)) f.q = (f.q + 2) & 3;
    states[i]->frame = f;
  }
  return SV_OK;
}

int batch_run(sv_state **states, sv_plan **plans, size_t count, int use_graph) {
  return batch_run_ex(states, plans, count, use_graph, nullptr);
}

int batch_inspect(const int *n_qubits, const size_t *rotations, const size_t *passes, size_t count, int grid_ctas,
                  int *out_ctas, double *out_max_over_mean) {
  if (count && (!n_qubits || !rotations || !passes)) return fail(SV_EINVAL, "NULL arrays");
  if (grid_ctas < 1) return fail(SV_EINVAL, "grid_ctas must be >= 1");
  std::vector<double> cost(count);
  std::vector<int> nq(count);
  for (size_t i = 0; i < count; ++i) {
    if (n_qubits[i] < 1 || n_qubits[i] > 34) return fail(SV_EINVAL, "bad n_qubits %d (state %zu)", n_qubits[i], i);
    cost[i] = batch_cost(n_qubits[i], rotations[i], passes[i] + 1);
    nq[i] = n_qubits[i];
  }
  std::vector<BatchItemDev> items;
  std::vector<int> cta_first;
  int multi = 0;
  if (count) assign(cost, nq, grid_ctas, items, cta_first, multi);
  if (out_ctas) {
    for (size_t i = 0; i < count; ++i) out_ctas[i] = 1;
    for (const BatchItemDev &it : items) out_ctas[it.state] = it.group;
  }
  if (out_max_over_mean) {
    double total = 0.0, worst = 0.0;
    for (double c : cost) total += c;
    for (int c = 0; c < grid_ctas && count; ++c) {
      double load = 0.0;
      for (int k = cta_first[c]; k < cta_first[c + 1]; ++k) load += cost[items[k].state] / items[k].group;
      worst = std::max(worst, load);
    }
    *out_max_over_mean = total > 0.0 ? worst / (total / grid_ctas) : 0.0;
  }
  return SV_OK;
}

int batch_info(int *grid_ctas, int *multi_cta_states, int *graph_used) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (grid_ctas) *grid_ctas = g_batch.grid;
  if (multi_cta_states) *multi_cta_states = g_batch.multi_cta_states;
  // 1 = cooperative launch in a graph, 0 = no graph; -e = capture failed with
  // cudaError_t e (the cooperative launch then runs without a graph)
  if (graph_used) *graph_used = g_batch.graph ? 1 : (g_batch.capture_error ? -g_batch.capture_error : 0);
  return SV_OK;
}

}  // extern "C"
