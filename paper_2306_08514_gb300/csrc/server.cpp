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
//   * Grouped launches: sessions with FP32 plans on the fused front end (SLRI, or SSPI with
//     the whole-vector gather) are bucketed by (method, N, sampling tiles, padded rank or
//     gather width); the pending frames of every such session of a bucket that has no
//     launch in flight leave together: one copy of all their frames and of a work list in,
//     one front-end kernel over (session, frame) items, one interpolation kernel over
//     (session, cell block, frame block) items, one argmax pass, one copy of all maps out.
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
struct GroupSlot;

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
  GroupSlot* group = nullptr;  // grouped launch carrying this batch (h_maps / h_arg point into it)
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
  // grouped launches (FP32 plans on the fused front end, SLRI or whole-vector SSPI)
  bool grouped = false;
  long long gkey = 0;        // bucket
  FrontParams fp{};          // front-end arguments (frames and out filled per launch)
  int cols = 0;              // front-end output row: Rp (SLRI) or L (SSPI)
  size_t front_smem = 0;
  int Rp = 0, L = 0, nrb = 0;
};

// One grouped launch in flight or awaiting polls: pinned host and device buffers shared by
// the sessions it carries.
struct GroupSlot {
  cudaStream_t stream = nullptr;
  int cap_frames = 0, cap_items = 0;
  size_t cap_in = 0, cap_out = 0, cap_scr = 0, cap_desc = 0;  // floats / bytes
  float* h_in = nullptr;   // pinned frames
  float* d_in = nullptr;
  float* h_out = nullptr;  // pinned maps
  float* d_out = nullptr;
  int* h_arg = nullptr;
  int* d_arg = nullptr;
  float* d_scr = nullptr;  // front-end outputs (u or xi)
  unsigned long long* d_keys = nullptr;
  char* h_desc = nullptr;  // work list: counts, front arguments, interpolation arguments, items
  char* d_desc = nullptr;
  size_t o_fp = 0, o_gi = 0, o_fi = 0, o_ci = 0;  // fixed work-list layout in h_desc / d_desc
  std::atomic<int> state{0};  // 0 free, 1 in flight, 2 done (members await polls)
  int refs = 0;               // member batches not yet polled
  std::vector<Slot*> members;
  Server* server = nullptr;
  // one captured graph per bucket; its copies are resized before each replay
  struct Graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphNode_t copy[7] = {};  // counts + front args, interp args, front items, interp
                                   // items, frames (in); maps, argmax (out)
    size_t front_smem = 0;
    int Lmax = 0;
  };
  std::map<long long, Graph> graphs;
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
  std::vector<std::unique_ptr<GroupSlot>> gslots;  // grouped launches (made on first use)
  int num_sms = 0;
  // stats
  long long frames_done = 0, launches = 0, graph_launches = 0, frames_launched = 0;
  long long group_launches = 0, group_frames = 0, group_sessions = 0;
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
  if (sl->group) {  // maps and argmax lived in the grouped launch's buffers
    sl->h_maps = nullptr;
    sl->h_arg = nullptr;
    sl->group = nullptr;
  }
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

// A batch of a grouped launch is consumed (polled, or dropped with its session).  The
// launch's buffers are free again once it is done and every batch it carried is consumed
// (the scheduler checks; the completion callback may still be running until it marks the
// launch done, so nothing else touches the member list).  Called with the server lock held.
void group_batch_done(Slot* sl) {
  GroupSlot* g = sl->group;
  sl->h_maps = nullptr;
  sl->h_arg = nullptr;
  sl->group = nullptr;
  if (g) --g->refs;
}

void release_session(Server& sv, Session& ss) {
  if (ss.stream) cudaStreamSynchronize(ss.stream);
  for (auto& sl : ss.slots)
    if (sl->group && sl->state.load() == 2) group_batch_done(sl.get());
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

// ------------------------------------------------------------------ grouped launches
constexpr int kGroupSlots = 4;
constexpr size_t kGroupInFloats = size_t(8) << 20;    // 32 MB of frames per launch
constexpr size_t kGroupOutFloats = size_t(16) << 20;  // 64 MB of maps per launch
constexpr int kGroupMaxCols = 1664;                   // front-end output row (Rp or L <= 1643)
constexpr int kGroupItems = 1 << 16;                  // interpolation work items per launch
constexpr int kSspiRowChunk = 8;                      // row blocks of 64 cells per SSPI item

size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

// A grouped session runs the front end's own sampling instantiation (its n-tile count:
// the wider ones accumulate in another order), so that its maps equal srp_map's bit for bit.
long long group_key(const srp_plan_s* P) {
  const int method = P->desc.method == SRP_SLRI ? 1 : 2;
  const int w = P->desc.method == SRP_SLRI ? (P->R + 7) / 8 * 8 : sspi_group_frames(P->g.L);
  return (static_cast<long long>(method) << 40) | (static_cast<long long>(P->g.N) << 24) |
         (static_cast<long long>(front_ntm(P->max_Np)) << 16) | w;
}

bool group_eligible(const srp_plan_s* P) {
  return P->op == OpType::F32 && P->use_front &&
         front_smem_bytes(P->g.M, P->g.N, P->g.L, P->max_Np) <= 200 * 1024 &&
         (P->desc.method == SRP_SLRI || (P->desc.method == SRP_SSPI && P->sspi_umax == 0)) &&
         ((P->R + 7) / 8 * 8 <= kGroupMaxCols) && P->g.L <= kGroupMaxCols;
}

void free_group(GroupSlot* g) {
  if (g->stream) cudaStreamSynchronize(g->stream);
  for (auto& kv : g->graphs) {
    if (kv.second.exec) cudaGraphExecDestroy(kv.second.exec);
    if (kv.second.graph) cudaGraphDestroy(kv.second.graph);
  }
  g->graphs.clear();
  if (g->h_in) cudaFreeHost(g->h_in);
  if (g->h_out) cudaFreeHost(g->h_out);
  if (g->h_arg) cudaFreeHost(g->h_arg);
  if (g->h_desc) cudaFreeHost(g->h_desc);
  void* d[] = {g->d_in, g->d_out, g->d_arg, g->d_scr, g->d_keys, g->d_desc};
  for (void* q : d)
    if (q) cudaFree(q);
  if (g->stream) cudaStreamDestroy(g->stream);
}

// The grouped launches' buffers, made once by the builder thread (outside the server lock)
// when the first session that qualifies is admitted.  Returns false if they cannot be
// allocated (the session then launches on its own).
bool make_groups(const Server& sv, std::vector<std::unique_ptr<GroupSlot>>& out) {
  const int cap_frames = std::min(4096, sv.desc.max_batch * sv.desc.max_sessions);
  std::vector<std::unique_ptr<GroupSlot>> gs;
  bool ok = true;
  for (int i = 0; i < kGroupSlots && ok; ++i) {
    auto g = std::make_unique<GroupSlot>();
    g->server = const_cast<Server*>(&sv);
    g->cap_frames = cap_frames;
    g->cap_items = kGroupItems;
    g->cap_in = kGroupInFloats;
    g->cap_out = kGroupOutFloats;
    g->cap_scr = static_cast<size_t>(cap_frames) * kGroupMaxCols;
    g->o_fp = 16;
    g->o_gi = g->o_fp + align16(sizeof(FrontParams) * cap_frames);
    g->o_fi = g->o_gi + align16(sizeof(GroupInterp) * cap_frames);
    g->o_ci = g->o_fi + align16(sizeof(int2) * cap_frames);
    g->cap_desc = g->o_ci + align16(sizeof(int4) * g->cap_items);
    ok = cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) == cudaSuccess &&
         cudaMallocHost(&g->h_in, 4 * g->cap_in) == cudaSuccess &&
         cudaMallocHost(&g->h_out, 4 * g->cap_out) == cudaSuccess &&
         cudaMallocHost(&g->h_arg, 4 * static_cast<size_t>(cap_frames)) == cudaSuccess &&
         cudaMallocHost(&g->h_desc, g->cap_desc) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_in), 4 * g->cap_in) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_out), 4 * g->cap_out) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_arg), 4 * static_cast<size_t>(cap_frames)) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_scr), 4 * g->cap_scr) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_keys), 8 * static_cast<size_t>(cap_frames)) == cudaSuccess &&
         device_alloc(reinterpret_cast<void**>(&g->d_desc), g->cap_desc) == cudaSuccess;
    gs.push_back(std::move(g));
  }
  if (!ok) {
    cudaGetLastError();
    for (auto& g : gs) free_group(g.get());
    return false;
  }
  out = std::move(gs);
  return true;
}

void CUDART_CB group_done_cb(void* u);

// The launch sequence of a grouped launch on stream s (issued directly or captured): the
// work list and the frames in, the keys cleared, the front end over the front items, the
// interpolation over its items, the argmax, the maps and argmax out, the completion
// callback.  sizes: the bytes of the seven copies (see GroupSlot::Graph).  Grids are
// fixed (the kernels walk the item counts the work list carries), so a captured sequence
// stays valid for any work list once its copies are resized.
cudaError_t enqueue_group(Server& sv, GroupSlot& g, long long key, size_t front_smem, int Lmax,
                          const size_t* sizes, cudaStream_t s) {
  const bool slri = (key >> 40) == 1;
  const int N = static_cast<int>((key >> 24) & 0xFFFF);
  const int NTM = static_cast<int>((key >> 16) & 0xFF);
  const int width = static_cast<int>(key & 0xFFFF);
  const int grid = 4 * std::max(1, sv.num_sms);
  const int* d_counts = reinterpret_cast<const int*>(g.d_desc);
  cudaError_t e = cudaMemcpyAsync(g.d_desc, g.h_desc, sizes[0], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_desc + g.o_gi, g.h_desc + g.o_gi, sizes[1], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_desc + g.o_fi, g.h_desc + g.o_fi, sizes[2], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(g.d_desc + g.o_ci, g.h_desc + g.o_ci, sizes[3], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g.d_in, g.h_in, sizes[4], cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(g.d_keys, 0, 8 * static_cast<size_t>(g.cap_frames), s);
  if (e == cudaSuccess)
    e = launch_front_group(reinterpret_cast<const FrontParams*>(g.d_desc + g.o_fp),
                           reinterpret_cast<const int2*>(g.d_desc + g.o_fi), d_counts, grid, N, NTM,
                           front_smem, s);
  const GroupInterp* d_gi = reinterpret_cast<const GroupInterp*>(g.d_desc + g.o_gi);
  const int4* d_ci = reinterpret_cast<const int4*>(g.d_desc + g.o_ci);
  if (e == cudaSuccess)
    e = slri ? launch_slri_tall_group(d_gi, d_ci, d_counts + 1, grid, width, s)
             : launch_sspi_group(d_gi, d_ci, d_counts + 1, grid, Lmax, s);
  if (e == cudaSuccess) e = launch_argmax_finalize(g.d_keys, g.d_arg, g.cap_frames, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_out, g.d_out, sizes[5], cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(g.h_arg, g.d_arg, sizes[6], cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s, group_done_cb, &g);
  return e;
}

// Captures the sequence into gg (on success gg.exec is set and its seven copy nodes found).
void capture_group(Server& sv, GroupSlot& g, long long key, size_t front_smem, int Lmax,
                   const size_t* sizes, GroupSlot::Graph& gg) {
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(g.stream, cudaStreamCaptureModeThreadLocal);
  const cudaError_t e2 = e == cudaSuccess ? enqueue_group(sv, g, key, front_smem, Lmax, sizes, g.stream) : e;
  if (e == cudaSuccess) e = cudaStreamEndCapture(g.stream, &graph);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    cudaGetLastError();
    if (graph) cudaGraphDestroy(graph);
    return;
  }
  // the copy nodes, told apart by their endpoints
  const void* src[7] = {g.h_desc, g.h_desc + g.o_gi, g.h_desc + g.o_fi, g.h_desc + g.o_ci,
                        g.h_in, g.d_out, g.d_arg};
  size_t n = 0;
  cudaGraphGetNodes(graph, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(graph, nodes.data(), &n);
  int found = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType ty;
    if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeMemcpy) continue;
    cudaMemcpy3DParms mp{};
    if (cudaGraphMemcpyNodeGetParams(nd, &mp) != cudaSuccess) continue;
    for (int i = 0; i < 7; ++i)
      if (mp.srcPtr.ptr == src[i] && !gg.copy[i]) {
        gg.copy[i] = nd;
        ++found;
      }
  }
  cudaGraphExec_t exec = nullptr;
  if (found == 7 && cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess) {
    gg.graph = graph;
    gg.exec = exec;
    gg.front_smem = front_smem;
    gg.Lmax = Lmax;
  } else {
    cudaGetLastError();
    cudaGraphDestroy(graph);
    gg = GroupSlot::Graph();
  }
}

// Resizes the seven copies of a captured grouped launch.
cudaError_t update_group_graph(GroupSlot& g, GroupSlot::Graph& gg, const size_t* sizes) {
  void* dst[7] = {g.d_desc, g.d_desc + g.o_gi, g.d_desc + g.o_fi, g.d_desc + g.o_ci, g.d_in,
                  g.h_out, g.h_arg};
  const void* src[7] = {g.h_desc, g.h_desc + g.o_gi, g.h_desc + g.o_fi, g.h_desc + g.o_ci,
                        g.h_in, g.d_out, g.d_arg};
  for (int i = 0; i < 7; ++i) {
    const cudaMemcpyKind kind = i < 5 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
    const cudaError_t e = cudaGraphExecMemcpyNodeSetParams1D(gg.exec, gg.copy[i], dst[i], src[i],
                                                             std::max<size_t>(sizes[i], 16), kind);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// One grouped launch of bucket `key` carrying the pending frames of `list` (sessions with no
// launch in flight and a free slot), as many as the launch's buffers hold.  Called with the
// server lock held.
void issue_group(Server& sv, GroupSlot& g, long long key, const std::vector<Session*>& list) {
  const bool slri = (key >> 40) == 1;
  const int N = static_cast<int>((key >> 24) & 0xFFFF);
  const int NTM = static_cast<int>((key >> 16) & 0xFF);
  const int width = static_cast<int>(key & 0xFFFF);  // SLRI: Rp; SSPI: frames per item
  struct Entry {
    Session* ss;
    Slot* sl;
    int b, f_off, n_items;
    size_t in_off, out_off, scr_off;
  };
  std::vector<Entry> es;
  size_t in = 0, out = 0, scr = 0;
  int frames = 0, items = 0, Lmax = 0;
  size_t smem = 0;
  for (Session* ss : list) {
    Slot* sl = nullptr;
    for (auto& x : ss->slots)
      if (x->state.load() == 0) {
        sl = x.get();
        break;
      }
    if (!sl) continue;
    const size_t fsz = static_cast<size_t>(ss->M) * ss->N;
    const int cpb = slri ? slri_tall_cells_per_block(ss->Rp) : 0;
    auto n_items = [&](int b) {
      return slri ? ((ss->J + cpb - 1) / cpb) * ((b + 63) / 64)
                  : ((b + width - 1) / width) * ((ss->nrb + kSspiRowChunk - 1) / kSspiRowChunk);
    };
    int b = std::min(ss->pend_count, sv.desc.max_batch);
    while (b > 0 && (frames + b > g.cap_frames || in + b * fsz > g.cap_in ||
                     out + static_cast<size_t>(b) * ss->J > g.cap_out ||
                     scr + static_cast<size_t>(b) * ss->cols > g.cap_scr ||
                     items + n_items(b) > g.cap_items))
      --b;
    if (b == 0) break;  // the launch is full; the rest leave with the next one
    es.push_back({ss, sl, b, frames, n_items(b), in, out, scr});
    in += (b * fsz + 3) & ~size_t(3);
    out += (static_cast<size_t>(b) * ss->J + 3) & ~size_t(3);
    scr += (static_cast<size_t>(b) * ss->cols + 3) & ~size_t(3);
    frames += b;
    items += n_items(b);
    Lmax = std::max(Lmax, ss->L);
    smem = std::max(smem, ss->front_smem);
  }
  if (es.empty()) return;
  const int E = static_cast<int>(es.size());
  // work list in pinned memory (fixed layout): counts | front arguments | interpolation
  // arguments | front items | interpolation items
  char* h = g.h_desc;
  const size_t o_fp = g.o_fp, o_gi = g.o_gi, o_fi = g.o_fi, o_ci = g.o_ci;
  int* counts = reinterpret_cast<int*>(h);
  FrontParams* fp = reinterpret_cast<FrontParams*>(h + o_fp);
  GroupInterp* gi = reinterpret_cast<GroupInterp*>(h + o_gi);
  int2* fi = reinterpret_cast<int2*>(h + o_fi);
  int4* ci = reinterpret_cast<int4*>(h + o_ci);
  int nfi = 0, nci = 0;
  g.members.clear();
  for (int e = 0; e < E; ++e) {
    Entry& x = es[e];
    Session& ss = *x.ss;
    Slot& sl = *x.sl;
    const size_t fsz = static_cast<size_t>(ss.M) * ss.N;
    sl.idx.resize(x.b);
    sl.t_arr.resize(x.b);
    for (int j = 0; j < x.b; ++j) {
      const int slot_i = (ss.pend_head + j) % ss.pend_cap;
      std::memcpy(g.h_in + x.in_off + j * fsz, ss.pend.data() + slot_i * fsz, fsz * 4);
      sl.idx[j] = ss.pend_idx[slot_i];
      sl.t_arr[j] = ss.pend_t[slot_i];
    }
    ss.pend_head = (ss.pend_head + x.b) % ss.pend_cap;
    ss.pend_count -= x.b;
    sl.b = x.b;
    sl.seq = ss.launch_seq++;
    sl.group = &g;
    sl.h_maps = g.h_out + x.out_off;
    sl.h_arg = g.h_arg + x.f_off;
    sl.state.store(1);
    g.members.push_back(&sl);
    const srp_plan_s* P = ss.plan;
    FrontParams a = ss.fp;
    a.frames = g.d_in + x.in_off;
    a.out = g.d_scr + x.scr_off;
    a.out_lo = nullptr;
    fp[e] = a;
    gi[e] = GroupInterp{g.d_scr + x.scr_off, P->d_tall, P->d_row_ptr, P->d_taps, g.d_out + x.out_off,
                        g.d_keys + x.f_off, x.b, ss.J, ss.L};
    for (int j = 0; j < x.b; ++j) fi[nfi++] = make_int2(e, j);
    if (slri) {
      const int cpb = slri_tall_cells_per_block(ss.Rp);
      for (int by = 0; by < (x.b + 63) / 64; ++by)
        for (int bx = 0; bx < (ss.J + cpb - 1) / cpb; ++bx) ci[nci++] = make_int4(e, bx, by, 0);
    } else {
      for (int fx = 0; fx < (x.b + width - 1) / width; ++fx)
        for (int rb = 0; rb < ss.nrb; rb += kSspiRowChunk)
          ci[nci++] = make_int4(e, fx, rb, std::min(rb + kSspiRowChunk, ss.nrb));
    }
  }
  counts[0] = nfi;
  counts[1] = nci;
  g.refs = E;
  g.state.store(1);
  cudaStream_t s = g.stream;
  const size_t sizes[7] = {o_fp + sizeof(FrontParams) * E, sizeof(GroupInterp) * E,
                           sizeof(int2) * nfi, sizeof(int4) * nci, 4 * in, 4 * out,
                           4 * static_cast<size_t>(frames)};
  cudaError_t e = cudaErrorUnknown;
  bool replayed = false;
  if (sv.desc.use_graphs) {
    GroupSlot::Graph& gg = g.graphs[key];
    if (gg.exec && (gg.front_smem < smem || gg.Lmax < Lmax)) {  // recapture with more smem
      cudaGraphExecDestroy(gg.exec);
      cudaGraphDestroy(gg.graph);
      gg = GroupSlot::Graph();
    }
    if (!gg.exec) capture_group(sv, g, key, std::max(smem, gg.front_smem), std::max(Lmax, gg.Lmax), sizes, gg);
    if (gg.exec) {
      e = update_group_graph(g, gg, sizes);
      if (e == cudaSuccess) e = cudaGraphLaunch(gg.exec, s);
      replayed = e == cudaSuccess;
      if (!replayed) cudaGetLastError();
    }
  }
  if (!replayed) e = enqueue_group(sv, g, key, smem, Lmax, sizes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaStreamSynchronize(s);
    for (Entry& x : es) {
      x.ss->error = std::string("grouped launch failed: ") + cudaGetErrorString(e);
      x.ss->state = ST_FAILED;
      x.sl->group = nullptr;
      x.sl->h_maps = nullptr;
      x.sl->h_arg = nullptr;
      x.sl->state.store(0);
    }
    g.members.clear();
    g.refs = 0;
    g.state.store(0);
    return;
  }
  if (replayed) ++sv.graph_launches;
  ++sv.launches;
  ++sv.group_launches;
  sv.frames_launched += frames;
  sv.group_frames += frames;
  sv.group_sessions += E;
}

// Grouped launches for every bucket with work, one per free launch buffer set.  Called with
// the server lock held.
void schedule_groups(Server& sv) {
  if (sv.gslots.empty()) return;
  std::map<long long, std::vector<Session*>> buckets;
  for (auto& kv : sv.sessions) {
    Session& ss = *kv.second;
    if (ss.state != ST_ACTIVE || !ss.grouped || ss.pend_count == 0) continue;
    bool in_flight = false, has_free = false;
    for (auto& sl : ss.slots) {
      const int st = sl->state.load();
      in_flight = in_flight || st == 1;
      has_free = has_free || st == 0;
    }
    if (has_free && !in_flight) buckets[ss.gkey].push_back(&ss);
  }
  for (auto& kb : buckets) {
    GroupSlot* g = nullptr;
    for (auto& gs : sv.gslots) {
      const int st = gs->state.load();
      if (st == 0 || (st == 2 && gs->refs == 0)) {
        g = gs.get();
        break;
      }
    }
    if (!g) return;
    g->members.clear();
    g->state.store(0);
    issue_group(sv, *g, kb.first, kb.second);
  }
}

void CUDART_CB group_done_cb(void* u) {
  GroupSlot* g = static_cast<GroupSlot*>(u);
  const double t = now_s();
  for (Slot* sl : g->members) {
    sl->done_t = t;
    sl->state.store(2);
  }
  g->state.store(2);  // last: after this the callback no longer reads the member list
  g->server->completions.fetch_add(1);
  g->server->cv.notify_all();
}

void scheduler_loop(Server* sv) {
  cudaSetDevice(sv->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (!sv->stop) {
    schedule_groups(*sv);
    for (auto& kv : sv->sessions) {
      Session& ss = *kv.second;
      if (ss.state == ST_ACTIVE && !ss.grouped) schedule_session(*sv, ss);
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
  bool groups_made = false;  // the grouped launches' buffers (made by this thread only)
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
    // grouped launches: the session's batches travel in shared launch buffers, so its
    // slots are bookkeeping only (no buffers, no graphs of their own)
    bool grouped = false;
    std::vector<std::unique_ptr<GroupSlot>> new_groups;
    if (st == SRP_OK && sv->desc.group_launches && group_eligible(plan)) {
      grouped = groups_made || make_groups(*sv, new_groups);
      groups_made = groups_made || grouped;
    }
    if (st != SRP_OK) {
      err = srp_last_error();
    } else if (grouped) {
      srp_plan_info_t info;
      srp_plan_info(plan, &info);
      bytes = info.device_bytes;
      for (int i = 0; i < sv->desc.slots_per_session; ++i) {
        auto sl = std::make_unique<Slot>();
        sl->server = sv;
        sl->owner = pick;
        slots.push_back(std::move(sl));
      }
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
    if (!new_groups.empty()) sv->gslots = std::move(new_groups);
    sv->used_bytes -= std::min(sv->used_bytes, pick->est_bytes);
    if (!err.empty()) {
      for (auto& sl : slots) free_slot(sl.get());
      if (plan) srp_destroy(plan);
      pick->error = err;
      pick->state = ST_FAILED;
      --sv->active;
    } else {
      pick->plan = plan;
      if (grouped) {
        const srp_plan_s* P = plan;
        const Geometry& g = P->g;
        const bool slri = P->desc.method == SRP_SLRI;
        pick->grouped = true;
        pick->gkey = group_key(P);
        pick->Rp = (P->R + 7) / 8 * 8;
        pick->L = g.L;
        pick->nrb = (g.J + 63) / 64;
        pick->cols = slri ? pick->Rp : g.L;
        pick->front_smem = front_smem_bytes(g.M, g.N, g.L, P->max_Np);
        pick->fp = front_params(g.M, g.N, P->d_window, P->d_twiddle, g.P, P->d_pairs, P->d_Np,
                                P->d_off, P->d_stab, g.L, P->max_Np, slri ? P->d_ftab : nullptr,
                                pick->Rp, pick->cols, 1.f, OpType::F32, 0);
      }
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
  SRP_CUDA_TRY(cudaDeviceGetAttribute(&sv->num_sms, cudaDevAttrMultiProcessorCount, sv->device));
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
    if (next->group) group_batch_done(next);
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
  st->group_launches = sv->group_launches;
  st->group_frames = sv->group_frames;
  st->group_sessions = sv->group_sessions;
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
  sv->group_launches = sv->group_frames = sv->group_sessions = 0;
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
  for (auto& g : sv->gslots)
    if (g->stream) cudaStreamSynchronize(g->stream);
  for (auto& kv : sv->sessions) {
    Session& ss = *kv.second;
    release_session(*sv, ss);
  }
  for (auto& g : sv->gslots) free_group(g.get());
  sv->gslots.clear();
  for (cudaStream_t s : sv->streams) cudaStreamDestroy(s);
  if (sv->build_stream) cudaStreamDestroy(sv->build_stream);
  delete sv;
}
