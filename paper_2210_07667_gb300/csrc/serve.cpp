// Served form: a trace of phi-action requests arriving over time, dispatched
// with continuous batching onto a fixed set of slots (one CUDA stream each),
// admitted by the device memory their workspaces take, with per-request
// latency measured from arrival to completion.
//
// One dispatcher loop on the calling thread: it moves requests whose arrival
// time has passed into a FIFO queue, hands the queue head to a free slot when
// the workspace bytes in flight stay within the budget (a request that alone
// exceeds the budget runs when nothing else is in flight), and retires slots
// whose work has finished.  Completion times are stamped by a host function
// enqueued behind the request's kernels.
//
// Submission (cfg->graphs): the dispatcher is one host thread, and a request
// is hundreds of short kernels, so issuing them one by one would make the
// host the bound.  Each slot therefore owns a workspace, input staging
// vectors and an output staging buffer (from a memory pool of this call,
// allocated once); a request's inputs are copied into the slot's staging
// vectors, its applies replay CUDA graphs captured once per (plan, tau, p,
// slot) (phiks_options.graph: the graph key holds only slot-owned pointers),
// and the outputs are copied to the request's buffers.  Without graphs each
// request takes a workspace from the pool and launches its kernels directly.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "../../include/phiks.h"
#include "kernels.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Done {
  std::atomic<int> flag{0};
  std::atomic<int64_t> ns{0};
  Clock::time_point t0;
};

void CUDART_CB stamp(void* p) {
  Done* d = static_cast<Done*>(p);
  d->ns.store(std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now() - d->t0).count());
  d->flag.store(1, std::memory_order_release);
}

struct Slot {
  cudaStream_t st = nullptr;
  int req = -1;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // graph submission: slot-owned buffers
  void* ws_fixed = nullptr;
  void* stage_v[PHIKS_MAX_P + 1] = {nullptr};
  void* stage_out = nullptr;
};

// Bytes of one vector and of the output of one apply.
void apply_bytes(const phiks_apply_args& x, size_t* vec, size_t* out) {
  int d = 0;
  int64_t n[PHIKS_MAX_D];
  phiks_plan_shape(x.plan, &d, n);
  int64_t N = 1;
  for (int mu = 0; mu < d; ++mu) N *= n[mu];
  const int dt = phiks::plan_dtype(x.plan);
  const size_t elt = dt == PHIKS_C128 ? 16 : (dt == PHIKS_FP64 || dt == PHIKS_FP64_EMU) ? 8 : 4;
  *vec = (size_t)N * elt;
  const int per = x.nv == 1 ? x.p + 1 - (x.skip_phi0 ? 1 : 0) : 1;
  *out = (size_t)std::max(1, x.nscales) * per * N * elt;
}

phiks_status sfail(phiks_status st, const std::string& m) {
  phiks::set_error_message(("phiks_serve_trace: " + m).c_str());
  return st;
}

}  // namespace

extern "C" phiks_status phiks_serve_trace(const phiks_serve_config* cfg, int count,
                                          const phiks_request* reqs, const double* arrival_s,
                                          double* latency_ms, double* queue_ms,
                                          double* makespan_s) {
  phiks::set_error_message("");
  if (!cfg || count < 0 || (count > 0 && (!reqs || !arrival_s || !latency_ms)))
    return sfail(PHIKS_ERR_INVALID, "bad arguments");
  if (cfg->slots < 1 || cfg->slots > 256) return sfail(PHIKS_ERR_INVALID, "slots out of [1, 256]");
  for (int k = 0; k < count; ++k) {
    if (k && arrival_s[k] < arrival_s[k - 1]) return sfail(PHIKS_ERR_INVALID, "arrivals not sorted");
    const phiks_request& r = reqs[k];
    if (r.napply < 1 || r.napply > PHIKS_SERVE_MAX_APPLY)
      return sfail(PHIKS_ERR_INVALID, "napply out of range in request " + std::to_string(k));
    for (int a = 0; a < r.napply; ++a)
      if (!r.apply[a].plan || !r.apply[a].vnorms)
        return sfail(PHIKS_ERR_INVALID, "request " + std::to_string(k) + " lacks a plan or norms");
  }
  if (count == 0) {
    if (makespan_s) *makespan_s = 0;
    return PHIKS_OK;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return sfail(PHIKS_ERR_CUDA, "no device");

  // per-request workspace: the largest of its applies (they run in order on one slot)
  std::vector<size_t> need(count, 0);
  for (int k = 0; k < count; ++k)
    for (int a = 0; a < reqs[k].napply; ++a) {
      const phiks_apply_args& x = reqs[k].apply[a];
      size_t b = 0;
      phiks_status s = phiks_workspace_size(x.plan, x.p, x.nv, std::max(1, x.nscales), &b);
      if (s != PHIKS_OK) return s;
      need[k] = std::max(need[k], b);
    }

  cudaMemPool_t pool = nullptr;
  cudaMemPoolProps props;
  std::memset(&props, 0, sizeof props);
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = dev;
  if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return sfail(PHIKS_ERR_CUDA, "memory pool");
  uint64_t keep = UINT64_MAX;
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);

  std::vector<Slot> slots(cfg->slots);
  phiks_status result = PHIKS_OK;
  std::string msg;
  for (auto& s : slots)
    if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess) {
      result = PHIKS_ERR_CUDA;
      msg = "stream creation";
    }
  const bool graphs = cfg->graphs != 0;
  if (graphs && result == PHIKS_OK) {
    // every slot's buffers, sized for the largest request
    size_t ws_max = 0, vec_max = 0, out_max = 0;
    int nv_max = 1;
    for (int k = 0; k < count; ++k) {
      ws_max = std::max(ws_max, need[k]);
      for (int a = 0; a < reqs[k].napply; ++a) {
        size_t vb = 0, ob = 0;
        apply_bytes(reqs[k].apply[a], &vb, &ob);
        vec_max = std::max(vec_max, vb);
        out_max = std::max(out_max, ob);
        nv_max = std::max(nv_max, reqs[k].apply[a].nv);
      }
    }
    for (auto& s : slots) {
      bool ok = cudaMallocFromPoolAsync(&s.ws_fixed, ws_max, pool, s.st) == cudaSuccess &&
                cudaMallocFromPoolAsync(&s.stage_out, out_max, pool, s.st) == cudaSuccess;
      for (int l = 0; l < nv_max && ok; ++l)
        ok = cudaMallocFromPoolAsync(&s.stage_v[l], vec_max, pool, s.st) == cudaSuccess;
      if (!ok) {
        result = PHIKS_ERR_OOM;
        msg = "slot buffers";
        break;
      }
      s.ws_bytes = 0;
    }
    for (auto& s : slots) cudaStreamSynchronize(s.st);  // (before the clock starts)
  }

  std::vector<Done> done(count);
  std::vector<double> t_dispatch(count, 0.0);
  const Clock::time_point t0 = Clock::now();
  for (auto& d : done) d.t0 = t0;
  auto now_s = [&]() { return std::chrono::duration<double>(Clock::now() - t0).count(); };

  std::deque<int> queue;
  int next = 0, completed = 0, inflight = 0;
  size_t inflight_bytes = 0;
  const size_t budget = cfg->hbm_budget;

  while (result == PHIKS_OK && completed < count) {
    bool progressed = false;
    const double t = now_s();
    while (next < count && arrival_s[next] <= t) queue.push_back(next++);
    for (auto& s : slots) {
      if (s.req < 0 || !done[s.req].flag.load(std::memory_order_acquire)) continue;
      if (s.ws) cudaFreeAsync(s.ws, s.st);
      inflight_bytes -= s.ws_bytes;
      s.ws = nullptr;
      s.ws_bytes = 0;
      s.req = -1;
      --inflight;
      ++completed;
      progressed = true;
    }
    while (!queue.empty()) {
      auto free_slot = std::find_if(slots.begin(), slots.end(), [](const Slot& s) { return s.req < 0; });
      if (free_slot == slots.end()) break;
      const int k = queue.front();
      if (budget && inflight > 0 && inflight_bytes + need[k] > budget) break;
      queue.pop_front();
      Slot& s = *free_slot;
      if (!graphs && cudaMallocFromPoolAsync(&s.ws, need[k], pool, s.st) != cudaSuccess) {
        result = PHIKS_ERR_OOM;
        msg = "workspace allocation for request " + std::to_string(k);
        break;
      }
      s.ws_bytes = need[k];
      s.req = k;
      inflight_bytes += need[k];
      ++inflight;
      t_dispatch[k] = now_s();
      for (int a = 0; a < reqs[k].napply && result == PHIKS_OK; ++a) {
        const phiks_apply_args& x = reqs[k].apply[a];
        phiks_options o;
        phiks_options_init(&o);
        o.nscales = std::max(1, x.nscales);
        o.skip_phi0 = x.skip_phi0;
        if (x.tol > 0) o.tol = x.tol;
        o.vnorms = x.vnorms;
        phiks_status r;
        if (graphs) {
          size_t vb = 0, ob = 0;
          apply_bytes(x, &vb, &ob);
          const void* sv[PHIKS_MAX_P + 1];
          for (int l = 0; l < x.nv; ++l) {
            sv[l] = x.v[l] ? s.stage_v[l] : nullptr;
            if (x.v[l] && cudaMemcpyAsync(s.stage_v[l], x.v[l], vb, cudaMemcpyDeviceToDevice, s.st) != cudaSuccess)
              result = PHIKS_ERR_CUDA;
          }
          o.workspace = s.ws_fixed;
          o.workspace_bytes = need[k];
          o.graph = 1;
          r = phiks_apply_ex(x.plan, x.tau, x.p, sv, x.nv, &o, s.stage_out, s.st);
          if (r == PHIKS_OK && cudaMemcpyAsync(x.out, s.stage_out, ob, cudaMemcpyDeviceToDevice, s.st) != cudaSuccess)
            r = PHIKS_ERR_CUDA;
        } else {
          o.workspace = s.ws;
          o.workspace_bytes = need[k];
          r = phiks_apply_ex(x.plan, x.tau, x.p, x.v, x.nv, &o, x.out, s.st);
        }
        if (r != PHIKS_OK && result == PHIKS_OK) {
          result = r;
          msg = "request " + std::to_string(k) + ": " + phiks_last_error();
        } else if (result != PHIKS_OK && msg.empty()) {
          msg = "request " + std::to_string(k) + ": staging copy";
        }
      }
      if (result != PHIKS_OK) break;
      if (cudaLaunchHostFunc(s.st, stamp, &done[k]) != cudaSuccess) {
        result = PHIKS_ERR_CUDA;
        msg = "host function";
        break;
      }
      progressed = true;
    }
    if (!progressed) {
      if (cfg->poll_us > 0) std::this_thread::sleep_for(std::chrono::microseconds(cfg->poll_us));
      else std::this_thread::yield();
    }
  }
  // drain and release everything, whatever happened
  for (auto& s : slots) {
    if (!s.st) continue;
    cudaStreamSynchronize(s.st);
    if (s.ws) cudaFreeAsync(s.ws, s.st);
    if (s.ws_fixed) cudaFreeAsync(s.ws_fixed, s.st);
    if (s.stage_out) cudaFreeAsync(s.stage_out, s.st);
    for (void* v : s.stage_v)
      if (v) cudaFreeAsync(v, s.st);
    cudaStreamSynchronize(s.st);
    cudaStreamDestroy(s.st);
  }
  cudaMemPoolDestroy(pool);
  if (result != PHIKS_OK) return sfail(result, msg);
  double last = 0;
  for (int k = 0; k < count; ++k) {
    const double tdone = done[k].ns.load() * 1e-9;
    latency_ms[k] = 1e3 * (tdone - arrival_s[k]);
    if (queue_ms) queue_ms[k] = 1e3 * (t_dispatch[k] - arrival_s[k]);
    last = std::max(last, tdone);
  }
  if (makespan_s) *makespan_s = last;
  return PHIKS_OK;
}
