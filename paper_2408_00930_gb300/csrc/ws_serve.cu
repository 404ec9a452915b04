// ws_serve.cu -- roll-out serving: a request loop with continuous batching.
//
// Trainer clients submit roll-out requests of any env type and size; each is
// admitted as soon as its device bytes (env state + a two-chunk trajectory
// ring) fit in the server's HBM budget, gets its own context, stream and
// resident state, and is advanced one chunk of steps at a time.  Chunks of
// different requests run concurrently on their own streams; a finished or
// released request frees its bytes and pending requests are admitted in its
// place.  Per chunk the loop records its completion time, so that latency
// (chunk k ready minus chunk k-1 ready; chunk 0 from arrival) and aggregate
// agent-steps/s can be reported.  (The paper describes no serving layer; this
// is the multi-client front end of the roll-out loop of Sec. 2 / App. B.)
#include <sys/socket.h>
#include <sys/un.h>
#include <unistd.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "ws_kernels.cuh"

// Internal helpers of ws_runtime.cu.
ws_status ws_fetch_async(ws_ctx *ctx, ws_field field, uint64_t t0, uint32_t n_steps, void *dst,
                         size_t dst_bytes, int dst_on_device, cudaStream_t stream);
size_t ws_field_step_bytes(const ws_ctx *ctx, ws_field field);

namespace {
struct Ipc;
}

namespace {

using Clock = std::chrono::steady_clock;
double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

constexpr size_t kAlign = 256;
inline size_t up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

struct Req {
  uint64_t id = 0;
  ws_request q{};
  ws_config cfg{};
  std::vector<int32_t> agents;
  enum { PENDING, ACTIVE, DONE, FAILED } st = PENDING;
  ws_ctx *ctx = nullptr;
  size_t off = 0, bytes = 0, state_bytes = 0, ring_bytes = 0;
  uint32_t n_slots = 0;
  cudaStream_t stream = nullptr;
  cudaEvent_t ev = nullptr;
  uint32_t n_chunks = 0, launched = 0, ready = 0, acked = 0;
  bool inflight = false;
  double t_arrival = 0, t_last = 0;
  ws_status err = WS_OK;
};

}  // namespace

struct ws_server {
  std::mutex mu;
  std::condition_variable cv;
  std::thread sched;
  bool stop = false;
  int device = 0;
  char *arena = nullptr;
  size_t budget = 0, used = 0, peak = 0;
  std::map<size_t, size_t> free_blocks;  // offset -> size
  std::map<uint64_t, Req *> reqs;
  std::deque<uint64_t> pending;
  uint64_t next_id = 1;
  cudaStream_t copy_stream = nullptr;
  // statistics
  uint64_t submitted = 0, admitted = 0, completed = 0, rejected = 0, failed = 0, chunks = 0;
  double agent_steps = 0, t_first = 0, t_last = 0;
  std::vector<float> lat_ms;
  Ipc *ipc = nullptr;  // clients in other processes (ws_server_listen)
};

namespace {

bool arena_alloc(ws_server *s, size_t bytes, size_t *off) {
  for (auto it = s->free_blocks.begin(); it != s->free_blocks.end(); ++it) {
    if (it->second >= bytes) {
      *off = it->first;
      const size_t rest = it->second - bytes;
      const size_t roff = it->first + bytes;
      s->free_blocks.erase(it);
      if (rest) s->free_blocks[roff] = rest;
      s->used += bytes;
      s->peak = std::max(s->peak, s->used);
      return true;
    }
  }
  return false;
}

void arena_free(ws_server *s, size_t off, size_t bytes) {
  s->used -= bytes;
  auto it = s->free_blocks.emplace(off, bytes).first;
  auto nx = std::next(it);
  if (nx != s->free_blocks.end() && it->first + it->second == nx->first) {
    it->second += nx->second;
    s->free_blocks.erase(nx);
  }
  if (it != s->free_blocks.begin()) {
    auto pv = std::prev(it);
    if (pv->first + pv->second == it->first) {
      pv->second += it->second;
      s->free_blocks.erase(it);
    }
  }
}

ws_config make_cfg(const ws_request &q, const std::vector<int32_t> &agents) {
  ws_config c{};
  c.struct_size = sizeof(ws_config);
  c.env = q.env;
  c.path = q.path;
  c.n_envs = q.n_envs;
  c.ring_steps = 2 * q.chunk_steps;  // double-buffered chunks
  c.episode_limit = q.episode_limit;
  c.chunk_steps = q.chunk_steps;
  c.hidden0 = q.hidden0;
  c.hidden1 = q.hidden1;
  c.dim = q.dim;
  c.n_gauss = q.n_gauss;
  c.noise_sigma = 0.05f;
  c.step_clip = 0.1f;
  c.gamma = 0.99f;
  c.flags = 0;
  c.param_seed = q.seed;
  c.agents_per_env = agents.empty() ? nullptr : agents.data();
  return c;
}

void release_locked(ws_server *s, Req *r) {
  if (r->stream) cudaStreamSynchronize(r->stream);
  if (r->ctx) ws_destroy(r->ctx);
  r->ctx = nullptr;
  if (r->ev) cudaEventDestroy(r->ev);
  r->ev = nullptr;
  if (r->stream) cudaStreamDestroy(r->stream);
  r->stream = nullptr;
  if (r->bytes) arena_free(s, r->off, r->bytes);
  r->bytes = 0;
}

bool admit_locked(ws_server *s, Req *r) {
  size_t off;
  if (!arena_alloc(s, r->bytes, &off)) return false;
  r->off = off;
  cudaError_t e = cudaStreamCreateWithFlags(&r->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
  ws_status st = e == cudaSuccess ? WS_OK : WS_ERR_CUDA;
  if (st == WS_OK) {
    r->cfg.agents_per_env = r->agents.empty() ? nullptr : r->agents.data();
    st = ws_create(&r->cfg, s->arena + off, r->state_bytes, s->arena + off + up(r->state_bytes),
                   r->ring_bytes, r->stream, &r->ctx);
  }
  if (st != WS_OK) {
    r->err = st;
    r->st = Req::FAILED;
    ++s->failed;
    release_locked(s, r);
    return true;  // consumed (failed) either way
  }
  r->st = Req::ACTIVE;
  ++s->admitted;
  return true;
}

void scheduler(ws_server *s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  while (!s->stop) {
    bool progress = false;
    // admission: arrival order, later requests may pass a head that does not fit
    // yet, unless the head has waited over 2 s (then it goes first)
    const double tnow = now_s();
    for (auto it = s->pending.begin(); it != s->pending.end();) {
      Req *r = s->reqs[*it];
      if (admit_locked(s, r)) {
        it = s->pending.erase(it);
        progress = true;
        s->cv.notify_all();
      } else {
        if (tnow - r->t_arrival > 2.0) break;
        ++it;
      }
    }
    // completions and launches
    for (auto &kv : s->reqs) {
      Req *r = kv.second;
      if (r->st != Req::ACTIVE) continue;
      if (r->inflight) {
        cudaError_t e = cudaEventQuery(r->ev);
        if (e == cudaErrorNotReady) continue;
        r->inflight = false;
        progress = true;
        const double t = now_s();
        if (e != cudaSuccess) {
          r->err = WS_ERR_CUDA;
          r->st = Req::FAILED;
          ++s->failed;
        } else {
          const uint32_t c = r->ready;
          const uint32_t steps = std::min(r->q.chunk_steps, r->q.horizon - c * r->q.chunk_steps);
          s->lat_ms.push_back((float)((t - (c == 0 ? r->t_arrival : r->t_last)) * 1e3));
          r->t_last = t;
          r->ready = c + 1;
          ++s->chunks;
          s->agent_steps += (double)r->n_slots * steps;
          s->t_last = t;
          if (r->ready == r->n_chunks) {
            r->st = Req::DONE;
            ++s->completed;
            if (r->q.flags & WS_REQ_CONSUME_ON_READY) release_locked(s, r);
          }
        }
        s->cv.notify_all();
      }
      if (r->st == Req::ACTIVE && !r->inflight && r->launched < r->n_chunks) {
        const bool room = (r->q.flags & WS_REQ_CONSUME_ON_READY) || r->launched < r->acked + 2;
        if (!room) continue;
        const uint32_t c = r->launched;
        const uint32_t steps = std::min(r->q.chunk_steps, r->q.horizon - c * r->q.chunk_steps);
        ws_status st = ws_rollout(r->ctx, steps);
        if (st == WS_OK && cudaEventRecord(r->ev, r->stream) != cudaSuccess) st = WS_ERR_CUDA;
        if (st != WS_OK) {
          r->err = st;
          r->st = Req::FAILED;
          ++s->failed;
          s->cv.notify_all();
          continue;
        }
        r->launched = c + 1;
        r->inflight = true;
        progress = true;
      }
    }
    if (!progress) s->cv.wait_for(lk, std::chrono::microseconds(20));
  }
}

// ---------------------------------------------------------------------------
// Clients in other processes: a Unix-domain stream socket, one thread per
// connection.  Messages are [u32 op][u32 payload bytes][payload] (host byte
// order: both ends run on the same machine); every reply starts with an i32
// status.  A connection that closes (the client exited, or was killed) has the
// requests it submitted and did not release released, freeing their bytes.
enum IpcOp : uint32_t {
  kOpSubmit = 1,   // ws_request [+ i32 agents_per_env[n_envs]] -> status, u64 id
  kOpWait = 2,     // u64 id, u32 chunk, u32 timeout_ms -> status
  kOpFetch = 3,    // u64 id, i32 field, u32 chunk -> status, u64 bytes, bytes
  kOpAck = 4,      // u64 id, u32 chunk -> status
  kOpRelease = 5,  // u64 id -> status
  kOpStats = 6     // -> status, ws_server_stats
};

struct Ipc {
  int listen_fd = -1;
  std::string path;
  std::atomic<bool> stop{false};
  std::thread acceptor;
  std::mutex mu;
  std::vector<std::thread> conns;
  std::set<int> fds;
};

bool read_all(int fd, void *buf, size_t n) {
  char *p = (char *)buf;
  while (n) {
    const ssize_t k = ::recv(fd, p, n, 0);
    if (k <= 0) return false;
    p += k;
    n -= (size_t)k;
  }
  return true;
}

bool write_all(int fd, const void *buf, size_t n) {
  const char *p = (const char *)buf;
  while (n) {
    const ssize_t k = ::send(fd, p, n, MSG_NOSIGNAL);
    if (k <= 0) return false;
    p += k;
    n -= (size_t)k;
  }
  return true;
}

bool reply_status(int fd, ws_status st) {
  const int32_t v = (int32_t)st;
  return write_all(fd, &v, 4);
}

void serve_connection(ws_server *s, int fd) {
  std::set<uint64_t> owned;
  std::vector<char> payload;
  for (;;) {
    uint32_t hdr[2];
    if (!read_all(fd, hdr, 8)) break;
    if (hdr[1] > (64u << 20)) break;  // malformed
    payload.resize(hdr[1]);
    if (hdr[1] && !read_all(fd, payload.data(), hdr[1])) break;
    const char *p = payload.data();
    bool ok = true;
    switch (hdr[0]) {
      case kOpSubmit: {
        ws_request q{};
        if (hdr[1] < sizeof(ws_request)) {
          ok = reply_status(fd, WS_ERR_INVALID) && write_all(fd, "\0\0\0\0\0\0\0\0", 8);
          break;
        }
        std::memcpy(&q, p, sizeof(ws_request));
        q.agents_per_env = nullptr;
        std::vector<int32_t> agents;
        if (hdr[1] > sizeof(ws_request)) {
          const size_t n = (hdr[1] - sizeof(ws_request)) / 4;
          agents.resize(n);
          std::memcpy(agents.data(), p + sizeof(ws_request), n * 4);
          if (n == q.n_envs) q.agents_per_env = agents.data();
        }
        uint64_t id = 0;
        const ws_status st = ws_server_submit(s, &q, &id);
        if (st == WS_OK) owned.insert(id);
        ok = reply_status(fd, st) && write_all(fd, &id, 8);
        break;
      }
      case kOpWait: {
        if (hdr[1] < 16) { ok = reply_status(fd, WS_ERR_INVALID); break; }
        uint64_t id;
        uint32_t chunk, timeout_ms;
        std::memcpy(&id, p, 8);
        std::memcpy(&chunk, p + 8, 4);
        std::memcpy(&timeout_ms, p + 12, 4);
        // bounded slices, so that a closing server is never held up by a waiter
        ws_status st = WS_ERR_TIMEOUT;
        const auto t_end = Clock::now() + std::chrono::milliseconds(timeout_ms);
        while (!s->ipc->stop.load()) {
          st = ws_server_wait_chunk(s, id, chunk, 200);
          if (st != WS_ERR_TIMEOUT) break;
          if (timeout_ms && Clock::now() >= t_end) break;
        }
        ok = reply_status(fd, st);
        break;
      }
      case kOpFetch: {
        if (hdr[1] < 16) { ok = reply_status(fd, WS_ERR_INVALID) && write_all(fd, "\0\0\0\0\0\0\0\0", 8); break; }
        uint64_t id;
        int32_t field;
        uint32_t chunk;
        std::memcpy(&id, p, 8);
        std::memcpy(&field, p + 8, 4);
        std::memcpy(&chunk, p + 12, 4);
        size_t bytes = 0;
        ws_status st = WS_ERR_INVALID;
        {
          std::lock_guard<std::mutex> lk(s->mu);
          auto it = s->reqs.find(id);
          if (it != s->reqs.end() && it->second->ctx) {
            const Req *r = it->second;
            const uint32_t steps =
                chunk < r->n_chunks ? std::min(r->q.chunk_steps, r->q.horizon - chunk * r->q.chunk_steps)
                                    : 0u;
            bytes = ws_field_step_bytes(r->ctx, (ws_field)field) * steps;
            st = bytes ? WS_OK : WS_ERR_INVALID;
          }
        }
        std::vector<char> buf(bytes);
        if (st == WS_OK) st = ws_server_fetch(s, id, (ws_field)field, chunk, buf.data(), bytes, 0);
        const uint64_t nb = st == WS_OK ? (uint64_t)bytes : 0u;
        ok = reply_status(fd, st) && write_all(fd, &nb, 8) && (nb == 0 || write_all(fd, buf.data(), nb));
        break;
      }
      case kOpAck: {
        if (hdr[1] < 12) { ok = reply_status(fd, WS_ERR_INVALID); break; }
        uint64_t id;
        uint32_t chunk;
        std::memcpy(&id, p, 8);
        std::memcpy(&chunk, p + 8, 4);
        ok = reply_status(fd, ws_server_ack(s, id, chunk));
        break;
      }
      case kOpRelease: {
        if (hdr[1] < 8) { ok = reply_status(fd, WS_ERR_INVALID); break; }
        uint64_t id;
        std::memcpy(&id, p, 8);
        const ws_status st = owned.count(id) ? ws_server_release(s, id) : WS_ERR_INVALID;
        owned.erase(id);
        ok = reply_status(fd, st);
        break;
      }
      case kOpStats: {
        ws_server_stats st{};
        st.struct_size = sizeof(st);
        const ws_status rc = ws_server_get_stats(s, &st);
        ok = reply_status(fd, rc) && write_all(fd, &st, sizeof(st));
        break;
      }
      default:
        ok = false;
    }
    if (!ok) break;
  }
  // the client is gone: its requests free their bytes
  for (uint64_t id : owned) ws_server_release(s, id);
  {
    std::lock_guard<std::mutex> lk(s->ipc->mu);
    s->ipc->fds.erase(fd);
  }
  ::close(fd);
}

void accept_loop(ws_server *s) {
  Ipc *ipc = s->ipc;
  cudaSetDevice(s->device);
  while (!ipc->stop.load()) {
    const int fd = ::accept(ipc->listen_fd, nullptr, nullptr);
    if (fd < 0) {
      if (ipc->stop.load()) break;
      std::this_thread::sleep_for(std::chrono::milliseconds(1));
      continue;
    }
    std::lock_guard<std::mutex> lk(ipc->mu);
    if (ipc->stop.load()) {
      ::close(fd);
      break;
    }
    ipc->fds.insert(fd);
    ipc->conns.emplace_back([s, fd] {
      cudaSetDevice(s->device);
      serve_connection(s, fd);
    });
  }
}

void ipc_stop(ws_server *s) {
  Ipc *ipc = s->ipc;
  if (!ipc) return;
  ipc->stop.store(true);
  if (ipc->listen_fd >= 0) ::shutdown(ipc->listen_fd, SHUT_RDWR);
  if (ipc->acceptor.joinable()) ipc->acceptor.join();
  if (ipc->listen_fd >= 0) ::close(ipc->listen_fd);
  std::vector<std::thread> conns;
  {
    std::lock_guard<std::mutex> lk(ipc->mu);
    for (int fd : ipc->fds) ::shutdown(fd, SHUT_RDWR);
    conns.swap(ipc->conns);
  }
  for (auto &t : conns)
    if (t.joinable()) t.join();
  ::unlink(ipc->path.c_str());
  delete ipc;
  s->ipc = nullptr;
}

}  // namespace

extern "C" {

ws_status ws_server_listen(ws_server *s, const char *path) {
  if (!s || !path || s->ipc) return WS_ERR_INVALID;
  sockaddr_un addr{};
  if (std::strlen(path) >= sizeof(addr.sun_path)) return WS_ERR_INVALID;
  addr.sun_family = AF_UNIX;
  std::strncpy(addr.sun_path, path, sizeof(addr.sun_path) - 1);
  const int fd = ::socket(AF_UNIX, SOCK_STREAM, 0);
  if (fd < 0) return WS_ERR_STATE;
  ::unlink(path);
  if (::bind(fd, (const sockaddr *)&addr, sizeof(addr)) != 0 || ::listen(fd, 64) != 0) {
    ::close(fd);
    return WS_ERR_STATE;
  }
  Ipc *ipc = new Ipc();
  ipc->listen_fd = fd;
  ipc->path = path;
  s->ipc = ipc;
  ipc->acceptor = std::thread(accept_loop, s);
  return WS_OK;
}

ws_status ws_server_create(size_t budget_bytes, ws_server **out) {
  if (!out || budget_bytes < 4096) return WS_ERR_INVALID;
  *out = nullptr;
  ws_server *s = new ws_server();
  cudaGetDevice(&s->device);
  if (cudaMalloc(&s->arena, budget_bytes) != cudaSuccess) {
    delete s;
    cudaGetLastError();
    return WS_ERR_NOMEM;
  }
  if (cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaFree(s->arena);
    delete s;
    return WS_ERR_CUDA;
  }
  s->budget = budget_bytes;
  s->free_blocks[0] = budget_bytes;
  s->sched = std::thread(scheduler, s);
  *out = s;
  return WS_OK;
}

ws_status ws_server_submit(ws_server *s, const ws_request *q, uint64_t *id) {
  if (!s || !q || !id || q->struct_size != sizeof(ws_request)) return WS_ERR_INVALID;
  if (q->chunk_steps < 1 || q->horizon < 1) return WS_ERR_INVALID;
  Req *r = new Req();
  r->q = *q;
  if (q->agents_per_env) r->agents.assign(q->agents_per_env, q->agents_per_env + q->n_envs);
  r->q.agents_per_env = nullptr;
  r->cfg = make_cfg(r->q, r->agents);
  ws_status st = ws_query_bytes(&r->cfg, &r->state_bytes, &r->ring_bytes, &r->n_slots);
  std::lock_guard<std::mutex> lk(s->mu);
  ++s->submitted;
  if (st != WS_OK) {
    ++s->rejected;
    delete r;
    return st;
  }
  r->bytes = up(r->state_bytes) + up(r->ring_bytes);
  if (r->bytes > s->budget) {
    ++s->rejected;
    delete r;
    return WS_ERR_NOMEM;
  }
  r->n_chunks = (q->horizon + q->chunk_steps - 1) / q->chunk_steps;
  r->id = s->next_id++;
  r->t_arrival = now_s();
  if (s->t_first == 0) s->t_first = r->t_arrival;
  s->reqs[r->id] = r;
  s->pending.push_back(r->id);
  *id = r->id;
  s->cv.notify_all();
  return WS_OK;
}

ws_status ws_server_wait_chunk(ws_server *s, uint64_t id, uint32_t chunk, uint32_t timeout_ms) {
  if (!s) return WS_ERR_INVALID;
  std::unique_lock<std::mutex> lk(s->mu);
  auto pred = [&] {
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return true;
    Req *r = it->second;
    return r->st == Req::FAILED || r->ready > chunk;
  };
  if (timeout_ms == 0) {
    s->cv.wait(lk, pred);
  } else if (!s->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
    return WS_ERR_TIMEOUT;
  }
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return WS_ERR_INVALID;
  if (it->second->st == Req::FAILED) return it->second->err;
  if (chunk >= it->second->n_chunks) return WS_ERR_RANGE;
  return WS_OK;
}

ws_status ws_server_fetch(ws_server *s, uint64_t id, ws_field field, uint32_t chunk, void *dst,
                          size_t dst_bytes, int dst_on_device) {
  if (!s) return WS_ERR_INVALID;
  cudaStream_t cs;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(id);
    if (it == s->reqs.end()) return WS_ERR_INVALID;
    Req *r = it->second;
    if (!r->ctx) return WS_ERR_STATE;
    if (chunk >= r->ready || chunk < r->acked) return WS_ERR_RANGE;
    const uint32_t steps = std::min(r->q.chunk_steps, r->q.horizon - chunk * r->q.chunk_steps);
    cs = s->copy_stream;
    ws_status st = ws_fetch_async(r->ctx, field, (uint64_t)chunk * r->q.chunk_steps, steps, dst,
                                  dst_bytes, dst_on_device, cs);
    if (st != WS_OK) return st;
  }
  if (cudaStreamSynchronize(cs) != cudaSuccess) return WS_ERR_CUDA;
  return WS_OK;
}

ws_status ws_server_ack(ws_server *s, uint64_t id, uint32_t chunk) {
  if (!s) return WS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return WS_ERR_INVALID;
  Req *r = it->second;
  if (chunk >= r->ready) return WS_ERR_RANGE;
  r->acked = std::max(r->acked, chunk + 1);
  s->cv.notify_all();
  return WS_OK;
}

ws_status ws_server_release(ws_server *s, uint64_t id) {
  if (!s) return WS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return WS_ERR_INVALID;
  Req *r = it->second;
  s->pending.erase(std::remove(s->pending.begin(), s->pending.end(), id), s->pending.end());
  release_locked(s, r);
  s->reqs.erase(it);
  delete r;
  s->cv.notify_all();
  return WS_OK;
}

ws_status ws_server_get_stats(ws_server *s, ws_server_stats *out) {
  if (!s || !out || out->struct_size != sizeof(ws_server_stats)) return WS_ERR_INVALID;
  std::lock_guard<std::mutex> lk(s->mu);
  out->submitted = s->submitted;
  out->admitted = s->admitted;
  out->completed = s->completed;
  out->rejected = s->rejected;
  out->failed = s->failed;
  out->chunks = s->chunks;
  out->agent_steps = s->agent_steps;
  out->elapsed_s = s->t_last > s->t_first ? s->t_last - s->t_first : 0.0;
  out->used_bytes = s->used;
  out->peak_bytes = s->peak;
  out->budget_bytes = s->budget;
  uint32_t act = 0;
  for (auto &kv : s->reqs) act += kv.second->st == Req::ACTIVE;
  out->active = act;
  out->pending = (uint32_t)s->pending.size();
  std::vector<float> l = s->lat_ms;
  out->p50_ms = out->p99_ms = 0;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    out->p50_ms = l[(size_t)(0.50 * (l.size() - 1))];
    out->p99_ms = l[(size_t)(0.99 * (l.size() - 1))];
  }
  return WS_OK;
}

void ws_server_destroy(ws_server *s) {
  if (!s) return;
  ipc_stop(s);  // no client thread touches the server after this
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
  }
  if (s->sched.joinable()) s->sched.join();
  for (auto &kv : s->reqs) {
    release_locked(s, kv.second);
    delete kv.second;
  }
  s->reqs.clear();
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  cudaFree(s->arena);
  delete s;
}

}  // extern "C"
