// Serving runtime of libsrp: many concurrent sessions (each a microphone array with its
// own grid, method, rank / taps and precision) share one GPU.
//
//   * Admission by HBM footprint: a session opened with srp_server_open is queued; a
//     builder thread creates its plan (tables, factors, tap lists, scratch) once the
//     estimated footprint fits the server's budget and a slot is free, so plan fitting
//     never stalls the sessions already being served.
//   * Framing with overlap state: pushed samples are cut into frames of N samples with
//     hop `hop` on the host; the last N - hop samples of every channel carry over.
//   * Continuous batching: a scheduler thread takes each session's pending frames (up to
//     max_batch, as a power of two) into one of its launch slots as soon as the session's
//     previous launch has finished, so frames arriving while a batch runs join the next
//     launch.  Sessions are spread over several CUDA streams, so their work overlaps on
//     the device.
//   * CUDA graphs: the launch sequence of a slot and batch size (H2D frames, the whole
//     SRP path, D2H maps and argmax, completion callback) is captured by the builder at
//     admission, for every power-of-two batch size, and replayed by the scheduler.
//   * Latency: each frame carries its arrival time (when its last sample was pushed);
//     the completion callback stamps the time its map is in host memory.
#include "srp_internal.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

namespace srp {
namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int floor_log2(int v) {
  int l = 0;
  while ((2 << l) <= v) ++l;
  return l;
}

struct Server;
struct Session;

// One launch slot: pinned host and device buffers for up to max_batch frames.
struct Slot {
  Server* server = nullptr;
  Session* owner = nullptr;
  float* h_frames = nullptr;  // pinned [max_batch][M][N]
  float* h_maps = nullptr;    // pinned [max_batch][J]
  int* h_arg = nullptr;       // pinned [max_batch]
  float* d_frames = nullptr;
  float* d_maps = nullptr;
  int* d_arg = nullptr;
  int b = 0;
  std::atomic<int> state{0};  // 0 free, 1 in flight, 2 done (results wait for poll)
  double done_t = 0;
  long long seq = 0;  // launch order within the session
  std::vector<long long> idx;
  std::vector<double> t_arr;
  std::vector<cudaGraphExec_t> graphs;  // per log2(batch)
};

enum {
  ST_QUEUED = SRP_SESSION_QUEUED, ST_ACTIVE = SRP_SESSION_ACTIVE, ST_CLOSING = SRP_SESSION_CLOSING,
  ST_CLOSED = SRP_SESSION_CLOSED, ST_FAILED = SRP_SESSION_FAILED, ST_BUILDING = 5
};

struct Session {
  int id = 0;
  int state = ST_QUEUED;
  srp_plan_desc desc{};
  std::vector<double> mic, grid;
  int hop = 0, M = 0, N = 0, J = 0;
  size_t est_bytes = 0, bytes = 0;
  srp_plan_t plan = nullptr;
  cudaStream_t stream = nullptr;  // shared server stream
  std::string error;
  // framing
  std::vector<std::vector<float>> hist;  // per channel: samples from the next frame's start
  long long next_frame = 0;
  // pending frames (ring)
  std::vector<float> pend;  // [pend_cap][M][N]
  std::vector<long long> pend_idx;
  std::vector<double> pend_t;
  int pend_head = 0, pend_count = 0, pend_cap = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  long long launch_seq = 0;
  long long frames_done = 0;
};

struct Server {
  srp_server_desc desc{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  cudaStream_t build_stream = nullptr;
  std::mutex mu;
  std::condition_variable cv, build_cv;
  std::map<int, std::unique_ptr<Session>> sessions;
  std::deque<int> queue;  // admission order
  int next_id = 1;
  size_t used_bytes = 0;
  int active = 0;
  bool stop = false;
  bool building = false;
  std::thread sched, builder;
  // stats
  long long frames_done = 0, launches = 0, graph_launches = 0, frames_launched = 0;
  std::vector<float> latencies;
  std::atomic<int> completions{0};
};

size_t slot_bytes(const Server& sv, const Session& ss) {
  return static_cast<size_t>(sv.desc.max_batch) * (static_cast<size_t>(ss.M) * ss.N + ss.J + 1) * 4;
}

void CUDART_CB done_cb(void* u) {
  Slot* sl = static_cast<Slot*>(u);
  sl->done_t = now_s();
  sl->state.store(2);
  sl->server->completions.fetch_add(1);
  sl->server->cv.notify_all();
}

void free_slot(Slot* sl) {
  for (cudaGraphExec_t g : sl->graphs)
    if (g) cudaGraphExecDestroy(g);
  sl->graphs.clear();
  if (sl->h_frames) cudaFreeHost(sl->h_frames);
  if (sl->h_maps) cudaFreeHost(sl->h_maps);
  if (sl->h_arg) cudaFreeHost(sl->h_arg);
  if (sl->d_frames) cudaFree(sl->d_frames);
  if (sl->d_maps) cudaFree(sl->d_maps);
  if (sl->d_arg) cudaFree(sl->d_arg);
  sl->h_frames = sl->h_maps = sl->d_frames = sl->d_maps = nullptr;
  sl->h_arg = sl->d_arg = nullptr;
}

void release_session(Server& sv, Session& ss) {
  if (ss.stream) cudaStreamSynchronize(ss.stream);
  for (auto& sl : ss.slots) free_slot(sl.get());
  ss.slots.clear();
  if (ss.plan) srp_destroy(ss.plan);
  ss.plan = nullptr;
  if (ss.state == ST_ACTIVE || ss.state == ST_CLOSING) {
    sv.used_bytes -= std::min(sv.used_bytes, ss.bytes);
    --sv.active;
  }
}

// The per-batch launch sequence of one slot (captured into a graph or issued directly).
cudaError_t enqueue(Session& ss, Slot& sl, int b, cudaStream_t s) {
  const size_t fbytes = static_cast<size_t>(b) * ss.M * ss.N * 4;
  cudaError_t e = cudaMemcpyAsync(sl.d_frames, sl.h_frames, fbytes, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  if (srp_map(ss.plan, sl.d_frames, b, sl.d_maps, sl.d_arg, s) != SRP_OK) return cudaErrorLaunchFailure;
  e = cudaMemcpyAsync(sl.h_maps, sl.d_maps, static_cast<size_t>(b) * ss.J * 4, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(sl.h_arg, sl.d_arg, static_cast<size_t>(b) * 4, cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaLaunchHostFunc(s, done_cb, &sl);
}

cudaError_t launch_slot(Server& sv, Session& ss, Slot& sl, int b) {
  const int k = floor_log2(b);
  if (sv.desc.use_graphs && (1 << k) == b) {
    if (!sl.graphs[k]) {
      cudaGraph_t g = nullptr;
      cudaError_t e = cudaStreamBeginCapture(ss.stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return e;
      cudaError_t e2 = enqueue(ss, sl, b, ss.stream);
      e = cudaStreamEndCapture(ss.stream, &g);
      if (e2 != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return e2;
      }
      if (e != cudaSuccess) return e;
      e = cudaGraphInstantiate(&sl.graphs[k], g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) return e;
    }
    ++sv.graph_launches;
    return cudaGraphLaunch(sl.graphs[k], ss.stream);
  }
  return enqueue(ss, sl, b, ss.stream);
}

// Moves up to max_batch pending frames (a power of two) of a session into a free slot
// and launches them.  Called with the server lock held.
void schedule_session(Server& sv, Session& ss) {
  while (ss.pend_count > 0) {
    Slot* free_sl = nullptr;
    bool in_flight = false;
    for (auto& sl : ss.slots) {
      const int st = sl->state.load();
      in_flight = in_flight || st == 1;
      if (st == 0 && !free_sl) free_sl = sl.get();
    }
    // One launch in flight per session: frames that arrive meanwhile wait and leave together
    // in the next launch, which costs about as much as a single frame (a 128-frame tile).
    if (!free_sl || in_flight) return;
    const int want = std::min(ss.pend_count, sv.desc.max_batch);
    const int b = 1 << floor_log2(want);
    const size_t fsz = static_cast<size_t>(ss.M) * ss.N;
    free_sl->idx.resize(b);
    free_sl->t_arr.resize(b);
    for (int j = 0; j < b; ++j) {
      const int slot_i = (ss.pend_head + j) % ss.pend_cap;
      std::memcpy(free_sl->h_frames + j * fsz, ss.pend.data() + slot_i * fsz, fsz * 4);
      free_sl->idx[j] = ss.pend_idx[slot_i];
      free_sl->t_arr[j] = ss.pend_t[slot_i];
    }
    ss.pend_head = (ss.pend_head + b) % ss.pend_cap;
    ss.pend_count -= b;
    free_sl->b = b;
    free_sl->seq = ss.launch_seq++;
    free_sl->state.store(1);
    const cudaError_t e = launch_slot(sv, ss, *free_sl, b);
    if (e != cudaSuccess) {
      ss.error = std::string("launch failed: ") + cudaGetErrorString(e) + " / " + srp_last_error();
      ss.state = ST_FAILED;
      free_sl->state.store(0);
      return;
    }
    ++sv.launches;
    sv.frames_launched += b;
  }
}

void scheduler_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    for (auto& kv : sv->sessions) {
      Session& ss = *kv.second;
      if (ss.state == ST_ACTIVE) schedule_session(*sv, ss);
      if (ss.state == ST_CLOSING || ss.state == ST_FAILED) {
        bool busy = false;
        for (auto& sl : ss.slots) busy = busy || sl->state.load() == 1;
        if (!busy && ss.state == ST_CLOSING) {
          release_session(*sv, ss);
          ss.state = ST_CLOSED;
          sv->build_cv.notify_all();
        }
      }
    }
    sv->cv.wait_for(lk, std::chrono::microseconds(200));
  }
}

void builder_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    Session* pick = nullptr;
    for (int id : sv->queue) {
      Session& ss = *sv->sessions[id];
      if (ss.state != ST_QUEUED) continue;
      if (sv->active < sv->desc.max_sessions &&
          sv->used_bytes + ss.est_bytes <= sv->desc.hbm_budget) {
        pick = &ss;
      }
      break;  // strict arrival order: a large session is not overtaken
    }
    if (!pick) {
      sv->build_cv.wait_for(lk, std::chrono::milliseconds(20));
      continue;
    }
    pick->state = ST_BUILDING;
    sv->used_bytes += pick->est_bytes;  // reserved until the actual size is known
    ++sv->active;
    sv->queue.erase(std::find(sv->queue.begin(), sv->queue.end(), pick->id));
    lk.unlock();
    // --- build outside the lock: plan, slots
    srp_plan_t plan = nullptr;
    std::string err;
    srp_status st = srp_plan_create(&pick->desc, sv->build_stream, &plan);
    // tile shape for this session's batch size (the autotuner times the variants)
    if (st == SRP_OK) st = srp_plan_autotune(plan, sv->desc.max_batch, sv->build_stream, nullptr);
    std::vector<std::unique_ptr<Slot>> slots;
    size_t bytes = 0;
    if (st != SRP_OK) {
      err = srp_last_error();
    } else {
      srp_plan_info_t info;
      srp_plan_info(plan, &info);
      bytes = info.device_bytes;
      const int mb = sv->desc.max_batch;
      for (int i = 0; i < sv->desc.slots_per_session && err.empty(); ++i) {
        auto sl = std::make_unique<Slot>();
        sl->server = sv;
        sl->owner = pick;
        sl->graphs.assign(floor_log2(mb) + 1, nullptr);
        const size_t fb = static_cast<size_t>(mb) * pick->M * pick->N * 4;
        const size_t mbytes = static_cast<size_t>(mb) * pick->J * 4;
        if (cudaMallocHost(&sl->h_frames, fb) != cudaSuccess ||
            cudaMallocHost(&sl->h_maps, mbytes) != cudaSuccess ||
            cudaMallocHost(&sl->h_arg, mb * 4) != cudaSuccess ||
            device_alloc(reinterpret_cast<void**>(&sl->d_frames), fb) != cudaSuccess ||
            device_alloc(reinterpret_cast<void**>(&sl->d_maps), mbytes) != cudaSuccess ||
            device_alloc(reinterpret_cast<void**>(&sl->d_arg), mb * 4) != cudaSuccess) {
          cudaGetLastError();
          err = "slot allocation failed";
        }
        bytes += fb + mbytes + mb * 4;
        slots.push_back(std::move(sl));
      }
      // capture every (slot, power-of-two batch) launch sequence now, on the builder's own
      // stream (a graph can be launched into any stream), so that no capture or
      // instantiation happens on the scheduler thread while sessions are served
      if (err.empty() && sv->desc.use_graphs) {
        Session tmp_view;  // enqueue() reads the plan and the sizes only
        tmp_view.plan = plan;
        tmp_view.M = pick->M;
        tmp_view.N = pick->N;
        tmp_view.J = pick->J;
        for (auto& sl : slots) {
          for (int k = 0; (1 << k) <= sv->desc.max_batch && err.empty(); ++k) {
            cudaGraph_t gr = nullptr;
            cudaError_t e = cudaStreamBeginCapture(sv->build_stream, cudaStreamCaptureModeThreadLocal);
            cudaError_t e2 = e == cudaSuccess ? enqueue(tmp_view, *sl, 1 << k, sv->build_stream) : e;
            if (e == cudaSuccess) e = cudaStreamEndCapture(sv->build_stream, &gr);
            if (e == cudaSuccess && e2 == cudaSuccess) e = cudaGraphInstantiate(&sl->graphs[k], gr, 0);
            if (gr) cudaGraphDestroy(gr);
            if (e != cudaSuccess || e2 != cudaSuccess) {
              cudaGetLastError();
              err = std::string("graph capture failed: ") + cudaGetErrorString(e2 != cudaSuccess ? e2 : e);
            }
          }
        }
      }
    }
    lk.lock();
    sv->used_bytes -= std::min(sv->used_bytes, pick->est_bytes);
    if (!err.empty()) {
      for (auto& sl : slots) free_slot(sl.get());
      if (plan) srp_destroy(plan);
      pick->error = err;
      pick->state = ST_FAILED;
      --sv->active;
    } else {
      pick->plan = plan;
      pick->slots = std::move(slots);
      pick->bytes = bytes;
      sv->used_bytes += bytes;
      pick->state = pick->state == ST_BUILDING ? ST_ACTIVE : pick->state;
      if (pick->state == ST_CLOSING) {  // closed while building: release now
        release_session(*sv, *pick);
        pick->state = ST_CLOSED;
      }
    }
    sv->cv.notify_all();
  }
}

Server* as_server(srp_server_t s) { return reinterpret_cast<Server*>(s); }

srp_status fail(srp_status st, const std::string& msg) {
  set_error(msg);
  return st;
}

}  // namespace
}  // namespace srp

using namespace srp;

extern "C" srp_status srp_server_create(const srp_server_desc* desc, srp_server_t* out) {
  clear_error();
  if (!desc || !out) return fail(SRP_EINVAL, "desc or out is NULL");
  *out = nullptr;
  if (desc->max_sessions < 1 || desc->max_sessions > 4096) return fail(SRP_EINVAL, "max_sessions must be in 1..4096");
  if (desc->max_batch < 1 || desc->max_batch > 4096 || (desc->max_batch & (desc->max_batch - 1)))
    return fail(SRP_EINVAL, "max_batch must be a power of two in 1..4096");
  if (desc->streams < 1 || desc->streams > 64) return fail(SRP_EINVAL, "streams must be in 1..64");
  if (desc->slots_per_session < 1 || desc->slots_per_session > 16)
    return fail(SRP_EINVAL, "slots_per_session must be in 1..16");
  if (desc->pending_frames < desc->max_batch)
    return fail(SRP_EINVAL, "pending_frames must be >= max_batch");
  auto sv = std::make_unique<Server>();
  sv->desc = *desc;
  SRP_CUDA_TRY(cudaGetDevice(&sv->device));
  for (int i = 0; i < desc->streams; ++i) {
    cudaStream_t s;
    SRP_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    sv->streams.push_back(s);
  }
  SRP_CUDA_TRY(cudaStreamCreateWithFlags(&sv->build_stream, cudaStreamNonBlocking));
  Server* raw = sv.get();
  sv->sched = std::thread(scheduler_loop, raw);
  sv->builder = std::thread(builder_loop, raw);
  *out = reinterpret_cast<srp_server_t>(sv.release());
  return SRP_OK;
}

extern "C" srp_status srp_server_open(srp_server_t server, const srp_plan_desc* desc, int hop,
                                      int* session) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv || !desc || !session) return fail(SRP_EINVAL, "server, desc or session is NULL");
  if (hop < 1 || hop > desc->N) return fail(SRP_EINVAL, "hop must be in 1..N");
  if (desc->max_frames < sv->desc.max_batch)
    return fail(SRP_EINVAL, "desc->max_frames must be >= the server's max_batch");
  size_t est = 0;
  srp_status st = srp_plan_estimate_bytes(desc, &est);
  if (st != SRP_OK) return st;
  auto ss = std::make_unique<Session>();
  ss->desc = *desc;
  ss->mic.assign(desc->mic_xyz, desc->mic_xyz + 3 * desc->M);
  ss->grid.assign(desc->grid_xyz, desc->grid_xyz + 3 * static_cast<size_t>(desc->J));
  ss->desc.mic_xyz = ss->mic.data();
  ss->desc.grid_xyz = ss->grid.data();
  ss->hop = hop;
  ss->M = desc->M;
  ss->N = desc->N;
  ss->J = desc->J;
  ss->hist.assign(desc->M, {});
  ss->pend_cap = sv->desc.pending_frames;
  ss->pend.assign(static_cast<size_t>(ss->pend_cap) * ss->M * ss->N, 0.f);
  ss->pend_idx.assign(ss->pend_cap, 0);
  ss->pend_t.assign(ss->pend_cap, 0.0);
  ss->est_bytes = est + slot_bytes(*sv, *ss) * sv->desc.slots_per_session;
  if (ss->est_bytes > sv->desc.hbm_budget)
    return fail(SRP_ENOMEM, "the session's footprint (" + std::to_string(ss->est_bytes) +
                                " bytes) exceeds the server's HBM budget");
  std::lock_guard<std::mutex> lk(sv->mu);
  ss->id = sv->next_id++;
  ss->stream = sv->streams[(ss->id - 1) % sv->streams.size()];
  *session = ss->id;
  sv->queue.push_back(ss->id);
  sv->sessions[ss->id] = std::move(ss);
  sv->build_cv.notify_all();
  return SRP_OK;
}

extern "C" srp_status srp_server_push(srp_server_t server, int session, const float* samples,
                                      int n, double t_arrival) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv) return fail(SRP_EINVAL, "server is NULL");
  if (n < 0 || (n > 0 && !samples)) return fail(SRP_EINVAL, "bad samples");
  const double t = t_arrival >= 0 ? t_arrival : now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return fail(SRP_EINVAL, "unknown session");
  Session& ss = *it->second;
  if (ss.state == ST_FAILED) return fail(SRP_ECUDA, ss.error);
  if (ss.state == ST_CLOSING || ss.state == ST_CLOSED) return fail(SRP_EINVAL, "session is closed");
  // frames that this push completes
  const size_t have = ss.hist[0].size();
  long long nf = 0;
  if (have + n >= static_cast<size_t>(ss.N)) nf = (have + n - ss.N) / ss.hop + 1;
  if (ss.pend_count + nf > ss.pend_cap)
    return fail(SRP_EAGAIN, "pending-frame queue full (poll results or push later)");
  for (int m = 0; m < ss.M; ++m) ss.hist[m].insert(ss.hist[m].end(), samples + static_cast<size_t>(m) * n,
                                                   samples + static_cast<size_t>(m) * n + n);
  const size_t fsz = static_cast<size_t>(ss.M) * ss.N;
  size_t start = 0;
  while (ss.hist[0].size() - start >= static_cast<size_t>(ss.N)) {
    const int slot_i = (ss.pend_head + ss.pend_count) % ss.pend_cap;
    float* dst = ss.pend.data() + slot_i * fsz;
    for (int m = 0; m < ss.M; ++m) std::memcpy(dst + static_cast<size_t>(m) * ss.N, ss.hist[m].data() + start, ss.N * 4);
    ss.pend_idx[slot_i] = ss.next_frame++;
    ss.pend_t[slot_i] = t;
    ++ss.pend_count;
    start += ss.hop;
  }
  if (start > 0)
    for (int m = 0; m < ss.M; ++m) ss.hist[m].erase(ss.hist[m].begin(), ss.hist[m].begin() + start);
  sv->cv.notify_all();
  return SRP_OK;
}

extern "C" srp_status srp_server_poll(srp_server_t server, int session, int max_frames,
                                      float* maps, int* argmax, long long* frame_index,
                                      double* latency_s, int* n_out) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv || !n_out) return fail(SRP_EINVAL, "server or n_out is NULL");
  *n_out = 0;
  if (max_frames < sv->desc.max_batch) return fail(SRP_EINVAL, "max_frames must be >= max_batch");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return fail(SRP_EINVAL, "unknown session");
  Session& ss = *it->second;
  int n = 0;
  for (;;) {  // completed slots in launch order
    Slot* next = nullptr;
    for (auto& sl : ss.slots) {
      const int st = sl->state.load();
      if (st != 0 && (!next || sl->seq < next->seq)) next = sl.get();
    }
    if (!next || next->state.load() != 2 || n + next->b > max_frames) break;
    for (int j = 0; j < next->b; ++j) {
      if (maps) std::memcpy(maps + static_cast<size_t>(n + j) * ss.J, next->h_maps + static_cast<size_t>(j) * ss.J, ss.J * 4);
      if (argmax) argmax[n + j] = next->h_arg[j];
      if (frame_index) frame_index[n + j] = next->idx[j];
      const double lat = next->done_t - next->t_arr[j];
      if (latency_s) latency_s[n + j] = lat;
      if (sv->latencies.size() < (1u << 22)) sv->latencies.push_back(static_cast<float>(lat));
    }
    n += next->b;
    ss.frames_done += next->b;
    sv->frames_done += next->b;
    next->state.store(0);
  }
  *n_out = n;
  sv->cv.notify_all();
  if (ss.state == ST_FAILED) return fail(SRP_ECUDA, ss.error);
  return SRP_OK;
}

extern "C" srp_status srp_server_session_info(srp_server_t server, int session, int* state,
                                              size_t* device_bytes, int* pending) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv) return fail(SRP_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return fail(SRP_EINVAL, "unknown session");
  Session& ss = *it->second;
  int st = ss.state == ST_BUILDING ? ST_QUEUED : ss.state;
  if (state) *state = st;
  if (device_bytes) *device_bytes = ss.bytes;
  if (pending) {
    int inflight = 0;
    for (auto& sl : ss.slots) inflight += sl->state.load() != 0 ? sl->b : 0;
    *pending = ss.pend_count + inflight;
  }
  if (ss.state == ST_FAILED) return fail(SRP_ECUDA, ss.error);
  return SRP_OK;
}

extern "C" srp_status srp_server_close(srp_server_t server, int session) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv) return fail(SRP_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->sessions.find(session);
  if (it == sv->sessions.end()) return fail(SRP_EINVAL, "unknown session");
  Session& ss = *it->second;
  if (ss.state == ST_QUEUED) {
    sv->queue.erase(std::remove(sv->queue.begin(), sv->queue.end(), session), sv->queue.end());
    ss.state = ST_CLOSED;
  } else if (ss.state == ST_ACTIVE || ss.state == ST_BUILDING) {
    ss.state = ST_CLOSING;
    ss.pend_count = 0;
  } else if (ss.state == ST_FAILED) {
    if (ss.plan) {
      ss.state = ST_CLOSING;  // failed while serving: the scheduler releases its resources
      ss.pend_count = 0;
    } else {
      ss.state = ST_CLOSED;  // failed while building: nothing is held
    }
  }
  sv->cv.notify_all();
  return SRP_OK;
}

extern "C" srp_status srp_server_stats(srp_server_t server, srp_server_stats_t* st) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv || !st) return fail(SRP_EINVAL, "server or stats is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(st, 0, sizeof(*st));
  st->frames_done = sv->frames_done;
  st->frames_launched = sv->frames_launched;
  st->launches = sv->launches;
  st->graph_launches = sv->graph_launches;
  st->device_bytes = sv->used_bytes;
  for (auto& kv : sv->sessions) {
    const int s = kv.second->state;
    if (s == ST_ACTIVE) ++st->sessions_active;
    if (s == ST_QUEUED || s == ST_BUILDING) ++st->sessions_queued;
  }
  if (!sv->latencies.empty()) {
    std::vector<float> v(sv->latencies);
    auto pct = [&](double q) {
      const size_t k = static_cast<size_t>(std::min<double>(v.size() - 1, std::floor(q * (v.size() - 1) + 0.5)));
      std::nth_element(v.begin(), v.begin() + k, v.end());
      return static_cast<double>(v[k]);
    };
    st->latency_p50_s = pct(0.50);
    st->latency_p99_s = pct(0.99);
    st->latency_max_s = static_cast<double>(*std::max_element(v.begin(), v.end()));
  }
  return SRP_OK;
}

extern "C" srp_status srp_server_reset_stats(srp_server_t server) {
  clear_error();
  Server* sv = as_server(server);
  if (!sv) return fail(SRP_EINVAL, "server is NULL");
  std::lock_guard<std::mutex> lk(sv->mu);
  sv->latencies.clear();
  sv->frames_done = sv->frames_launched = sv->launches = sv->graph_launches = 0;
  return SRP_OK;
}

extern "C" double srp_server_now(void) { return now_s(); }

extern "C" void srp_server_destroy(srp_server_t server) {
  Server* sv = as_server(server);
  if (!sv) return;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv.notify_all();
  sv->build_cv.notify_all();
  if (sv->sched.joinable()) sv->sched.join();
  if (sv->builder.joinable()) sv->builder.join();
  for (cudaStream_t s : sv->streams) cudaStreamSynchronize(s);
  for (auto& kv : sv->sessions) {
    Session& ss = *kv.second;
    release_session(*sv, ss);
  }
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  if (sv->build_stream) cudaStreamDestroy(sv->build_stream);
  delete sv;
}
