// Batched independent shells (declared in include/chorus.h): the shells of one order form one
// mesh (their disjoint union: the face pairing joins only faces that share nodes, and the shells
// share none).  Three schedules of an RK step: the orders concurrently on streams forked from the
// caller's stream or one after another on it (both captured as a CUDA graph and replayed), or every
// order in one persistent cooperative launch per RK stage (batch_persist.cu).  A small autotuner
// picks the FP32 tile shape per order on the batch's own meshes and then the fastest schedule.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "chorus.h"
#include "mesh_state.h"

using namespace chorus;

struct chorus_batch_s {
  struct Group {
    int p = 0;
    chorus_mesh mesh = nullptr;
    std::vector<int> shells;      // shell ids of this order, in input order
    std::vector<int64_t> e0, ne;  // their element ranges in the union mesh
    int64_t state_off = 0;        // float offset of the group's state in the batch array
    size_t ws_off = 0;            // byte offset of the group's workspace
    size_t ws_bytes = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t join = nullptr;
  };
  std::vector<Group> groups;
  int n_shells = 0;
  std::vector<int> shell_group, shell_slot;
  std::vector<uint64_t> seed;
  std::vector<double> amp;
  chorus_params params{};
  int64_t n_state = 0;
  size_t ws_bytes = 0;
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (the caller's may be the legacy stream, which cannot be captured)
  bool concurrent = true;  // orders on forked streams (true) or one after another (false)
  bool persistent = false;  // one persistent launch per RK stage for all orders (overrides concurrent)
  unsigned* d_sync = nullptr;  // the persistent launch's grid-barrier and work counters
  // chorus_batch_rk_step_host: the copy-in and copy-out streams and their events
  cudaStream_t in_stream = nullptr, out_stream = nullptr;
  std::vector<cudaEvent_t> host_ev;
  cudaGraphExec_t exec = nullptr;
  const float* g_Q = nullptr;
  const void* g_ws = nullptr;
  double g_dt = 0.0;
};

namespace {

constexpr int64_t kStateAlign = 64;  // floats (256 bytes) between group state blocks
constexpr size_t kWsAlign = 256;

void drop_graph(chorus_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  b->g_Q = nullptr;
  b->g_ws = nullptr;
}

void free_batch(chorus_batch_s* b) {
  drop_graph(b);
  for (auto& g : b->groups) {
    if (g.mesh) chorus_mesh_destroy(g.mesh);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.join) cudaEventDestroy(g.join);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->d_sync) cudaFree(b->d_sync);
  for (cudaEvent_t e : b->host_ev) cudaEventDestroy(e);
  if (b->in_stream) cudaStreamDestroy(b->in_stream);
  if (b->out_stream) cudaStreamDestroy(b->out_stream);
  delete b;
}

// One RK step of every group: forked from and joined back into `st`, or one group after another on it.
chorus_status step_all(chorus_batch_s* b, float* Q, void* ws, double dt, cudaStream_t st) {
  if (!b->concurrent) {
    for (auto& g : b->groups) {
      const chorus_status s = chorus_rk_step_scheme(g.mesh, &b->params, CHORUS_FP32_PERT, 0, Q + g.state_off,
                                                    (char*)ws + g.ws_off, dt, 1, st);
      if (s != CHORUS_OK) return s;
    }
    return CHORUS_OK;
  }
  if (cudaEventRecord(b->fork, st) != cudaSuccess) return CHORUS_ECUDA;
  for (auto& g : b->groups) {
    if (cudaStreamWaitEvent(g.stream, b->fork, 0) != cudaSuccess) return CHORUS_ECUDA;
    const chorus_status s = chorus_rk_step_scheme(g.mesh, &b->params, CHORUS_FP32_PERT, 0, Q + g.state_off,
                                                  (char*)ws + g.ws_off, dt, 1, g.stream);
    if (s != CHORUS_OK) return s;
    if (cudaEventRecord(g.join, g.stream) != cudaSuccess) return CHORUS_ECUDA;
    if (cudaStreamWaitEvent(st, g.join, 0) != cudaSuccess) return CHORUS_ECUDA;
  }
  return CHORUS_OK;
}

// Whether the persistent schedule can run this batch: a device with cooperative launch, and no
// radial radiative diffusivity (its kernel is built for a constant kappa_r).
bool persistent_ok(const chorus_batch_s* b) {
  return b->params.kappa_r1 == 0.0 && b->params.kappa_r2 == 0.0 && persist_grid() > 0;
}

// One RK step of every group as three persistent launches (one per SSP-RK3 stage).
chorus_status step_persistent(chorus_batch_s* b, float* Q, void* ws, double dt, cudaStream_t st) {
  if (!persistent_ok(b)) return CHORUS_EUNSUPPORTED;
  if (!b->d_sync && cudaMalloc(&b->d_sync, 8 * sizeof(unsigned)) != cudaSuccess) {
    b->d_sync = nullptr;
    return CHORUS_ENOMEM;
  }
  StagePtrs sp[4];
  StagePtrs* gp[4] = {nullptr, nullptr, nullptr, nullptr};
  for (auto& g : b->groups) {
    const int s = g.p - 2;
    const chorus_status r = mesh_stage_ptrs(g.mesh, b->params, Q + g.state_off, (char*)ws + g.ws_off, &sp[s]);
    if (r != CHORUS_OK) return r;
    gp[s] = &sp[s];
  }
  return persist_rk3_step(gp, dt, b->d_sync, st);
}

chorus_status capture(chorus_batch_s* b, float* Q, void* ws, double dt) {
  drop_graph(b);
  // relaxed mode: the launch helpers set kernel attributes, which is not a stream operation
  if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
    cudaGetLastError();
    return CHORUS_ECUDA;
  }
  const chorus_status s = step_all(b, Q, ws, dt, b->cap);
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
  if (s != CHORUS_OK || ce != cudaSuccess || graph == nullptr) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return s != CHORUS_OK ? s : CHORUS_ECUDA;
  }
  const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    b->exec = nullptr;
    return CHORUS_ECUDA;
  }
  b->g_Q = Q;
  b->g_ws = ws;
  b->g_dt = dt;
  return CHORUS_OK;
}

bool shell_ok(const chorus_shell_desc& d) {
  return d.n_nodes > 0 && d.node_xyz && d.n_elem > 0 && d.hex20 && d.p >= 2 && d.p <= 5 &&
         d.entropy_amp >= 0.0 && d.entropy_amp < 1.0;
}

}  // namespace

extern "C" {

chorus_status chorus_batch_create(int n_shells, const chorus_shell_desc* shells, double r_inner, double r_outer,
                                  const chorus_params* params, void* stream, chorus_batch* out) {
  if (!out) return CHORUS_EINVAL;
  *out = nullptr;
  if (n_shells <= 0 || !shells || !params || !(r_inner > 0.0) || !(r_outer > r_inner)) return CHORUS_EINVAL;
  for (int s = 0; s < n_shells; ++s)
    if (!shell_ok(shells[s])) return CHORUS_EINVAL;
  chorus_batch_s* b = new (std::nothrow) chorus_batch_s();
  if (!b) return CHORUS_ENOMEM;
  b->n_shells = n_shells;
  b->params = *params;
  b->shell_group.assign(n_shells, -1);
  b->shell_slot.assign(n_shells, -1);
  for (int s = 0; s < n_shells; ++s) {
    b->seed.push_back(shells[s].seed);
    b->amp.push_back(shells[s].entropy_amp);
  }
  cudaStream_t st = (cudaStream_t)stream;
  chorus_status status = CHORUS_OK;
  if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
    status = CHORUS_ECUDA;
  for (int p = 2; p <= 5 && status == CHORUS_OK; ++p) {
    chorus_batch_s::Group g;
    g.p = p;
    std::vector<double> xyz;
    std::vector<int64_t> hex;
    int64_t nodes = 0, elems = 0;
    for (int s = 0; s < n_shells; ++s) {
      const chorus_shell_desc& d = shells[s];
      if (d.p != p) continue;
      for (int64_t i = 0; i < d.n_elem * 20; ++i) {
        const int64_t v = d.hex20[i];
        if (v < 0 || v >= d.n_nodes) {
          status = CHORUS_EMESH;
          break;
        }
        hex.push_back(v + nodes);
      }
      if (status != CHORUS_OK) break;
      xyz.insert(xyz.end(), d.node_xyz, d.node_xyz + 3 * d.n_nodes);
      b->shell_group[s] = (int)b->groups.size();
      b->shell_slot[s] = (int)g.shells.size();
      g.shells.push_back(s);
      g.e0.push_back(elems);
      g.ne.push_back(d.n_elem);
      nodes += d.n_nodes;
      elems += d.n_elem;
    }
    if (status != CHORUS_OK || g.shells.empty()) continue;
    status = chorus_mesh_create(nodes, xyz.data(), elems, hex.data(), p, r_inner, r_outer, 0, stream, &g.mesh);
    if (status == CHORUS_OK) status = chorus_prepare(g.mesh, params, stream);
    if (status == CHORUS_OK && (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
                                cudaEventCreateWithFlags(&g.join, cudaEventDisableTiming) != cudaSuccess))
      status = CHORUS_ECUDA;
    b->groups.push_back(g);  // owned by the batch from here on (freed on failure)
  }
  if (status == CHORUS_OK) {
    int64_t off = 0;
    size_t ws = 0;
    for (auto& g : b->groups) {
      const int N = g.p + 1;
      g.state_off = off;
      off += (g.mesh->E * 5 * N * N * N + kStateAlign - 1) / kStateAlign * kStateAlign;
      g.ws_off = ws;
      g.ws_bytes = chorus_rk_workspace_bytes(g.mesh, CHORUS_FP32_PERT);
      ws += (g.ws_bytes + kWsAlign - 1) / kWsAlign * kWsAlign;
    }
    b->n_state = off;
    b->ws_bytes = ws;
    if (cudaStreamSynchronize(st) != cudaSuccess) status = CHORUS_ECUDA;
  }
  if (status != CHORUS_OK) {
    free_batch(b);
    return status;
  }
  *out = b;
  return CHORUS_OK;
}

chorus_status chorus_batch_destroy(chorus_batch b) {
  if (!b) return CHORUS_EINVAL;
  cudaDeviceSynchronize();
  free_batch(b);
  return CHORUS_OK;
}

chorus_status chorus_batch_layout(chorus_batch b, int64_t* state_offset, int64_t* n_state, size_t* workspace_bytes,
                                  int* n_groups, int* group_p, double* group_h_min) {
  if (!b) return CHORUS_EINVAL;
  if (state_offset) {
    for (int s = 0; s < b->n_shells; ++s) {
      const auto& g = b->groups[b->shell_group[s]];
      const int N = g.p + 1;
      state_offset[s] = g.state_off + g.e0[b->shell_slot[s]] * 5 * N * N * N;
    }
  }
  if (n_state) *n_state = b->n_state;
  if (workspace_bytes) *workspace_bytes = b->ws_bytes;
  if (n_groups) *n_groups = (int)b->groups.size();
  for (size_t g = 0; g < b->groups.size(); ++g) {
    if (group_p) group_p[g] = b->groups[g].p;
    if (group_h_min) chorus_mesh_info(b->groups[g].mesh, nullptr, nullptr, &group_h_min[g], nullptr);
  }
  return CHORUS_OK;
}

chorus_status chorus_batch_init(chorus_batch b, float* Q, void* stream) {
  if (!b || !Q) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  for (auto& g : b->groups)
    for (size_t i = 0; i < g.shells.size(); ++i) {
      const int s = g.shells[i];
      const chorus_status r = mesh_init_range(g.mesh, b->seed[s], b->amp[s], Q + g.state_off, g.e0[i], g.ne[i], st);
      if (r != CHORUS_OK) return r;
    }
  return CHORUS_OK;
}

chorus_status chorus_batch_rk_step(chorus_batch b, float* Q, void* workspace, double dt, int64_t n_steps,
                                   void* stream, int64_t* launches) {
  if (!b || !Q || !workspace || !(dt > 0.0) || !std::isfinite(dt) || n_steps < 0) return CHORUS_EINVAL;
  // per order: trace + 3 x (gradient, face, residual); persistent: one launch per stage
  if (launches) *launches = b->persistent ? 3 : 10 * (int64_t)b->groups.size();
  if (n_steps == 0) return CHORUS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (b->persistent) {
    for (int64_t n = 0; n < n_steps; ++n) {
      const chorus_status s = step_persistent(b, Q, workspace, dt, st);
      if (s != CHORUS_OK) return s;
    }
    return CHORUS_OK;
  }
  if (!b->exec || b->g_Q != Q || b->g_ws != workspace || b->g_dt != dt) {
    // capturing runs nothing; the graph is launched on the caller's stream, which orders it
    const chorus_status s = capture(b, Q, workspace, dt);
    if (s != CHORUS_OK) return s;
  }
  for (int64_t n = 0; n < n_steps; ++n)
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return CHORUS_ECUDA;
  return CHORUS_OK;
}

chorus_status chorus_batch_rk_step_host(chorus_batch b, float* Q_host, float* Q_dev, void* workspace, double dt,
                                        int64_t n_steps, void* stream) {
  if (!b || !Q_host || !Q_dev || !workspace || !(dt > 0.0) || !std::isfinite(dt) || n_steps < 0) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t ng = b->groups.size();
  if (!b->in_stream) {
    if (cudaStreamCreateWithFlags(&b->in_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->out_stream, cudaStreamNonBlocking) != cudaSuccess)
      return CHORUS_ECUDA;
    b->host_ev.assign(2 * ng + 2, nullptr);
    for (cudaEvent_t& e : b->host_ev)
      if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return CHORUS_ECUDA;
  }
  auto bytes_of = [&](size_t g) {
    const int N = b->groups[g].p + 1;
    return (size_t)b->groups[g].mesh->E * 5 * N * N * N * sizeof(float);
  };
  // the order of the groups: the smallest state first (its copy in is not overlapped), then from the
  // largest down, the second smallest last (its copy out is not overlapped)
  std::vector<size_t> ord(ng);
  for (size_t g = 0; g < ng; ++g) ord[g] = g;
  std::sort(ord.begin(), ord.end(), [&](size_t x, size_t y) { return bytes_of(x) < bytes_of(y); });
  if (ng > 2) std::reverse(ord.begin() + 1, ord.end());
  cudaEvent_t* ev_in = b->host_ev.data();
  cudaEvent_t* ev_done = ev_in + ng;
  cudaEvent_t start = ev_in[2 * ng], end = ev_in[2 * ng + 1];
  auto cu = [](cudaError_t e) { return e == cudaSuccess ? CHORUS_OK : CHORUS_ECUDA; };
  chorus_status s = cu(cudaEventRecord(start, st));  // after the caller's earlier work on st
  if (s == CHORUS_OK) s = cu(cudaStreamWaitEvent(b->in_stream, start, 0));
  for (size_t i = 0; i < ng && s == CHORUS_OK; ++i) {  // every copy in, one after another
    const auto& g = b->groups[ord[i]];
    s = cu(cudaMemcpyAsync(Q_dev + g.state_off, Q_host + g.state_off, bytes_of(ord[i]), cudaMemcpyHostToDevice,
                           b->in_stream));
    if (s == CHORUS_OK) s = cu(cudaEventRecord(ev_in[i], b->in_stream));
  }
  for (size_t i = 0; i < ng && s == CHORUS_OK; ++i) {  // each group's steps once its state is in
    const auto& g = b->groups[ord[i]];
    s = cu(cudaStreamWaitEvent(st, ev_in[i], 0));
    if (s == CHORUS_OK)
      s = chorus_rk_step_scheme(g.mesh, &b->params, CHORUS_FP32_PERT, 0, Q_dev + g.state_off, (char*)workspace + g.ws_off,
                                dt, n_steps, st);
    if (s == CHORUS_OK) s = cu(cudaEventRecord(ev_done[i], st));
    if (s == CHORUS_OK) s = cu(cudaStreamWaitEvent(b->out_stream, ev_done[i], 0));
    if (s == CHORUS_OK)
      s = cu(cudaMemcpyAsync(Q_host + g.state_off, Q_dev + g.state_off, bytes_of(ord[i]), cudaMemcpyDeviceToHost,
                             b->out_stream));
  }
  if (s == CHORUS_OK) s = cu(cudaEventRecord(end, b->out_stream));
  if (s == CHORUS_OK) s = cu(cudaStreamWaitEvent(st, end, 0));
  if (s == CHORUS_OK) s = cu(cudaStreamSynchronize(st));
  return s;
}

chorus_status chorus_batch_reduce(chorus_batch b, const float* Q, double* out, void* stream) {
  if (!b || !Q || !out) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  for (auto& g : b->groups)
    for (size_t i = 0; i < g.shells.size(); ++i) {
      const chorus_status r = mesh_reduce_range(g.mesh, Q + g.state_off, g.e0[i], g.ne[i], out + 4 * g.shells[i], st);
      if (r != CHORUS_OK) return r;
    }
  for (auto& g : b->groups) {
    const chorus_status r = chorus_check(g.mesh, st);
    if (r != CHORUS_OK) return r;
  }
  return CHORUS_OK;
}

chorus_status chorus_batch_autotune(chorus_batch b, float* Q, void* workspace, double dt, int n_trials, void* stream,
                                    int* choice) {
  if (!b || !Q || !workspace || !(dt > 0.0) || !std::isfinite(dt) || n_trials < 1) return CHORUS_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  drop_graph(b);
  if (choice)
    for (int i = 0; i < 4; ++i) choice[i] = 0;
  cudaEvent_t t0, t1;
  if (cudaEventCreate(&t0) != cudaSuccess) return CHORUS_ECUDA;
  if (cudaEventCreate(&t1) != cudaSuccess) {
    cudaEventDestroy(t0);
    return CHORUS_ECUDA;
  }
  chorus_status status = CHORUS_OK;
  for (auto& g : b->groups) {
    float best_ms = 0.0f;
    int best = 0;
    for (int t = 0; t < kTiles && status == CHORUS_OK; ++t) {
      if (mesh_set_tile(g.mesh, t) < 0) {
        status = CHORUS_EINVAL;
        break;
      }
      float* Qg = Q + g.state_off;
      void* wg = (char*)workspace + g.ws_off;
      for (size_t i = 0; i < g.shells.size() && status == CHORUS_OK; ++i)
        status = mesh_init_range(g.mesh, b->seed[g.shells[i]], b->amp[g.shells[i]], Qg, g.e0[i], g.ne[i], st);
      if (status == CHORUS_OK)  // warm-up step
        status = chorus_rk_step_scheme(g.mesh, &b->params, CHORUS_FP32_PERT, 0, Qg, wg, dt, 1, st);
      if (status != CHORUS_OK) break;
      if (cudaEventRecord(t0, st) != cudaSuccess) status = CHORUS_ECUDA;
      if (status == CHORUS_OK)
        status = chorus_rk_step_scheme(g.mesh, &b->params, CHORUS_FP32_PERT, 0, Qg, wg, dt, n_trials, st);
      float ms = 0.0f;
      if (status == CHORUS_OK && (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
                                  cudaEventElapsedTime(&ms, t0, t1) != cudaSuccess))
        status = CHORUS_ECUDA;
      if (status == CHORUS_OK && (t == 0 || ms < best_ms)) {
        best_ms = ms;
        best = t;
      }
    }
    if (status != CHORUS_OK) break;
    const int epb = mesh_set_tile(g.mesh, best);
    if (choice) choice[g.p - 2] = epb;
  }
  // then the schedule: the captured step with the orders concurrent and one after another, and the
  // persistent launches
  float sched_ms[3] = {0.0f, 0.0f, 0.0f};
  b->persistent = false;
  for (int c = 0; c < 2 && status == CHORUS_OK; ++c) {
    b->concurrent = c == 0;
    status = capture(b, Q, workspace, dt);
    if (status == CHORUS_OK && cudaGraphLaunch(b->exec, st) != cudaSuccess) status = CHORUS_ECUDA;  // warm-up
    if (status == CHORUS_OK && cudaEventRecord(t0, st) != cudaSuccess) status = CHORUS_ECUDA;
    for (int n = 0; n < n_trials && status == CHORUS_OK; ++n)
      if (cudaGraphLaunch(b->exec, st) != cudaSuccess) status = CHORUS_ECUDA;
    if (status == CHORUS_OK && (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
                                cudaEventElapsedTime(&sched_ms[c], t0, t1) != cudaSuccess))
      status = CHORUS_ECUDA;
  }
  b->concurrent = sched_ms[0] <= sched_ms[1];
  drop_graph(b);
  if (status == CHORUS_OK && persistent_ok(b)) {
    status = step_persistent(b, Q, workspace, dt, st);  // warm-up
    if (status == CHORUS_OK && cudaEventRecord(t0, st) != cudaSuccess) status = CHORUS_ECUDA;
    for (int n = 0; n < n_trials && status == CHORUS_OK; ++n) status = step_persistent(b, Q, workspace, dt, st);
    if (status == CHORUS_OK && (cudaEventRecord(t1, st) != cudaSuccess || cudaEventSynchronize(t1) != cudaSuccess ||
                                cudaEventElapsedTime(&sched_ms[2], t0, t1) != cudaSuccess))
      status = CHORUS_ECUDA;
    if (status == CHORUS_OK) b->persistent = sched_ms[2] < std::min(sched_ms[0], sched_ms[1]);
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  return status;
}

chorus_status chorus_batch_set_wait_limit(chorus_batch b, int64_t polls) {
  if (!b) return CHORUS_EINVAL;
  for (auto& g : b->groups) {
    const chorus_status s = chorus_set_wait_limit(g.mesh, polls);
    if (s != CHORUS_OK) return s;
  }
  return CHORUS_OK;
}

chorus_status chorus_batch_schedule(chorus_batch b, int set, int* concurrent) {
  if (!b) return CHORUS_EINVAL;
  if (set == 2 && !persistent_ok(b)) return CHORUS_EUNSUPPORTED;
  if (set == 0 || set == 1) {
    if (b->concurrent != (set == 1)) drop_graph(b);
    b->concurrent = set == 1;
    b->persistent = false;
  } else if (set == 2) {
    drop_graph(b);
    b->persistent = true;
  }
  if (concurrent) *concurrent = b->persistent ? 2 : b->concurrent ? 1 : 0;
  return CHORUS_OK;
}

}  // extern "C"
