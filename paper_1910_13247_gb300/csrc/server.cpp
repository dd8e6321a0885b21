// Native solve server: admission by device-memory budget, operator set-up on host threads, and one
// scheduler thread that advances every running solve through the batch engine (mfx_batch_advance).
//
// Life of a request: QUEUED (submitted) -> SETUP (admitted: a set-up thread builds the mesh, the
// operator, the solver workspace, b and x on its own stream) -> RUNNING (in a batch slot; each
// solve takes its next step as soon as its previous one has finished) -> DONE (slot released; the
// operator and the solution stay on the device until the caller retires the request).  Nothing on
// the scheduler thread waits for the GPU except the release of a finished or cancelled slot, which
// waits for that slot's own stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "mfx_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
  int64_t ticket = 0;
  mfx_request r{};
  std::vector<int32_t> leaves;  // octree description (copied at submission)
  std::vector<double> verts;
  int state = MFX_REQ_QUEUED;
  int error = 0;
  bool cancel = false;
  int pinned = 0;  // result copies in progress
  int64_t est = 0, bytes = 0, n_dofs = 0;
  double t_submit = -1, t_admit = -1, t_ready = -1, t_done = -1, setup_s = 0;
  mfx_solve_stats stats{};
  mfx_op* op = nullptr;
  double* b = nullptr;
  double* x = nullptr;
  int32_t slot = -1;
};
using ReqPtr = std::shared_ptr<Req>;

// Device bytes of a request before its operator exists: FP64 + FP32 metric, JxW and index table per
// quadrature point, and per DoF the solver workspace, diagonals and the two vectors, with the DoF
// count taken as 2 k^3 per cell (an over-estimate for meshes of more than a few cells).
int64_t estimate_bytes(int64_t n_cells, int k) {
  const int64_t n3 = (int64_t)(k + 1) * (k + 1) * (k + 1);
  const int64_t nq = n_cells * n3;
  const int64_t nd = std::max<int64_t>(8, 2 * n_cells * (int64_t)k * k * k);
  return nq * (6 * 8 + 6 * 4 + 8 + 4) + nd * (9 * 8 + 9 * 4 + 2 * 8 + 8 + 4 + 1 + 2 * 8);
}

}  // namespace

struct mfx_server {
  mfx_server_config cfg{};
  Clock::time_point t0;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_setup, cv_sched;
  std::map<int64_t, ReqPtr> reqs;
  std::deque<ReqPtr> queue, setup_jobs, ready;
  std::vector<ReqPtr> running;
  int in_setup = 0;  // admitted, not yet running (waiting for, in, or just out of set-up)
  int64_t bytes_in_use = 0;
  int64_t next_ticket = 1;
  mfx_server_stats counts{};
  bool stop = false;
  mfx_batch* batch = nullptr;
  cudaStream_t release_stream = nullptr;
  std::vector<std::thread> workers;
  std::thread scheduler;

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

// Frees a request's device data in stream order (every use of it has finished).
void free_request(mfx_server* s, Req& q) {
  if (q.b) cudaFreeAsync(q.b, s->release_stream);
  if (q.x) cudaFreeAsync(q.x, s->release_stream);
  if (q.op) mfx_operator_release(q.op, s->release_stream);
  q.b = q.x = nullptr;
  q.op = nullptr;
}

// Runs on a set-up thread: mesh (octree description), operator, workspace, b, x.
// Every resource a set-up makes is owned by q (operator, vectors; freed by free_request when the
// set-up fails, whether by a status or a host exception) or by a local RAII owner (the mesh).
mfx_status setup_request(Req& q, cudaStream_t st, std::vector<double>& hb) {
  std::unique_ptr<mfx_mesh, void (*)(mfx_mesh*)> own(nullptr, mfx_mesh_destroy);
  const mfx_mesh* mesh = q.r.mesh;
  if (!mesh) {
    mfx_mesh* m = nullptr;
    mfx_status rc = mfx_mesh_create_octree(&m, q.r.nx, q.r.ny, q.r.nz, q.verts.empty() ? nullptr : q.verts.data(),
                                           q.leaves.data(), (int64_t)q.leaves.size() / 4);
    if (rc != MFX_OK) return rc;
    own.reset(m);
    mesh = m;
  }
  mfx_op* op = nullptr;
  mfx_status rc = mfx_operator_create(&op, mesh, &q.r.desc, (mfx_stream)st);
  own.reset();
  if (rc != MFX_OK) return rc;
  q.op = op;
  rc = mfx_solver_prepare(op);
  if (rc != MFX_OK) return rc;
  mfx_op_info info;
  mfx_operator_info(op, &info);
  const int64_t n = info.n_dofs;
  q.n_dofs = n;
  if (cudaMallocAsync((void**)&q.b, sizeof(double) * n, st) != cudaSuccess ||
      cudaMallocAsync((void**)&q.x, sizeof(double) * n, st) != cudaSuccess)
    return mfx::set_error(MFX_ENOMEM, "server: vector allocation failed");
  hb.assign((size_t)n, 1.0);
  if (q.r.rhs) q.r.rhs(op, hb.data(), n, q.r.user);
  // pageable source: the call returns once the data is staged, so hb may be reused at once
  if (cudaMemcpyAsync(q.b, hb.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st) != cudaSuccess)
    return mfx::set_error(MFX_ECUDA, "server: right-hand side upload failed");
  rc = mfx_distribute(op, q.b, (mfx_stream)st);
  if (rc != MFX_OK) return rc;
  if (cudaMemsetAsync(q.x, 0, sizeof(double) * n, st) != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess)
    return mfx::set_error(MFX_ECUDA, "server: set-up stream failed");
  q.bytes = info.bytes_device + 2 * (int64_t)sizeof(double) * n;
  return MFX_OK;
}

void worker_main(mfx_server* s) {
  cudaSetDevice(s->device);
  cudaStream_t st = nullptr;
  cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  std::vector<double> hb;
  for (;;) {
    ReqPtr q;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_setup.wait(lk, [&] { return s->stop || !s->setup_jobs.empty(); });
      if (s->stop) break;
      q = s->setup_jobs.front();
      s->setup_jobs.pop_front();
    }
    const double t = s->now();
    mfx_status rc;
    {
      MFX_TRACE("mfx_server_setup");
      try {
        rc = setup_request(*q, st, hb);
      } catch (...) {  // a host failure fails the request, not the process
        rc = mfx::host_exception();
      }
    }
    {
      std::lock_guard<std::mutex> g(s->mu);
      q->setup_s = s->now() - t;
      if (rc != MFX_OK) {
        free_request(s, *q);
        q->state = MFX_REQ_FAILED;
        q->error = rc;
        q->t_done = s->now();
        s->bytes_in_use -= q->bytes;
        --s->in_setup;
      } else {
        s->bytes_in_use += q->bytes - q->est;
        s->ready.push_back(q);
      }
    }
    s->cv_sched.notify_one();
  }
  if (st) cudaStreamDestroy(st);
}

// Admission under the lock: policy order, slots and memory budget (one request always fits when
// nothing else is admitted).
void admit_locked(mfx_server* s) {
  while (!s->queue.empty() && (int)s->running.size() + s->in_setup < s->cfg.max_slots) {
    size_t pick = 0;
    if (s->cfg.policy == MFX_ADMIT_SMALLEST_FIRST)
      for (size_t i = 1; i < s->queue.size(); ++i)
        if (s->queue[i]->est < s->queue[pick]->est) pick = i;
    ReqPtr q = s->queue[pick];
    const bool busy = !s->running.empty() || s->in_setup > 0;
    if (busy && s->bytes_in_use + q->est > s->cfg.budget_bytes) break;
    s->queue.erase(s->queue.begin() + (std::ptrdiff_t)pick);
    q->state = MFX_REQ_SETUP;
    q->t_admit = s->now();
    q->bytes = q->est;
    s->bytes_in_use += q->est;
    ++s->in_setup;
    s->setup_jobs.push_back(q);
    s->cv_setup.notify_one();
  }
}

void finish_locked(mfx_server* s, Req& q, int state) {
  q.state = state;
  q.t_done = s->now();
}

void scheduler_main(mfx_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    std::deque<ReqPtr> to_add;
    bool stopping;
    {
      std::lock_guard<std::mutex> g(s->mu);
      stopping = s->stop;
      if (s->stop && s->in_setup == (int)s->setup_jobs.size() + (int)s->ready.size() && s->running.empty()) {
        // stopping: whatever is still waiting for a worker or a slot is cancelled
        for (auto* dq : {&s->setup_jobs, &s->ready})
          for (auto& q : *dq) {
            free_request(s, *q);
            finish_locked(s, *q, MFX_REQ_CANCELLED);
            --s->in_setup;
          }
        s->setup_jobs.clear();
        s->ready.clear();
        break;
      }
      if (!s->stop) admit_locked(s);
      to_add.swap(s->ready);
    }
    for (auto& q : to_add) {
      bool cancel;
      {
        std::lock_guard<std::mutex> g(s->mu);
        cancel = q->cancel || stopping;
      }
      if (cancel) {
        std::lock_guard<std::mutex> g(s->mu);
        free_request(s, *q);
        s->bytes_in_use -= q->bytes;
        q->bytes = 0;
        finish_locked(s, *q, MFX_REQ_CANCELLED);
        --s->in_setup;
        continue;
      }
      int32_t slot = -1;
      const mfx_status rc = mfx_batch_add(s->batch, q->op, q->b, q->x, &q->r.params, &slot);
      std::lock_guard<std::mutex> g(s->mu);
      --s->in_setup;
      if (rc != MFX_OK) {
        free_request(s, *q);
        s->bytes_in_use -= q->bytes;
        q->bytes = 0;
        q->error = rc;
        finish_locked(s, *q, MFX_REQ_FAILED);
        continue;
      }
      q->slot = slot;
      q->state = MFX_REQ_RUNNING;
      q->t_ready = s->now();
      s->running.push_back(q);
      s->counts.max_concurrent = std::max<int32_t>(s->counts.max_concurrent, (int32_t)s->running.size());
    }
    if (!s->running.empty()) {
      int32_t n_active = 0;
      const mfx_status rc = mfx_batch_advance(s->batch, &n_active);
      std::vector<ReqPtr> still;
      for (auto& q : s->running) {
        int32_t done = 0;
        mfx_solve_stats st{};
        bool cancel;
        {
          std::lock_guard<std::mutex> g(s->mu);
          cancel = q->cancel || s->stop;
        }
        if (rc == MFX_OK && !cancel) mfx_batch_poll(s->batch, q->slot, &done, &st);
        if (rc == MFX_OK && !cancel && !done) {
          still.push_back(q);
          continue;
        }
        mfx_batch_release(s->batch, q->slot);  // waits for the slot's own stream only
        std::lock_guard<std::mutex> g(s->mu);
        q->slot = -1;
        if (rc != MFX_OK) {
          q->error = rc;
          finish_locked(s, *q, MFX_REQ_FAILED);
        } else if (cancel) {
          finish_locked(s, *q, MFX_REQ_CANCELLED);
        } else {
          q->stats = st;
          finish_locked(s, *q, MFX_REQ_DONE);
        }
      }
      std::lock_guard<std::mutex> g(s->mu);
      s->running.swap(still);
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->running.empty()) {
      s->cv_sched.wait_for(lk, std::chrono::milliseconds(2), [&] {
        return s->stop || !s->ready.empty() ||
               (!s->queue.empty() && (int)s->running.size() + s->in_setup < s->cfg.max_slots);
      });
    } else {
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
  }
}

}  // namespace

using mfx::host_exception;
using mfx::set_error;

extern "C" {

mfx_status mfx_server_create(mfx_server** out, const mfx_server_config* config) try {
  if (!out || !config) return set_error(MFX_EINVAL, "null argument");
  *out = nullptr;
  mfx_server_config c = *config;
  if (c.max_slots < 1 || c.max_slots > 4096 || c.budget_bytes < 0 || c.setup_threads < 0 || c.setup_threads > 64 ||
      (c.policy != MFX_ADMIT_FIFO && c.policy != MFX_ADMIT_SMALLEST_FIRST))
    return set_error(MFX_EINVAL, "mfx_server_create: bad configuration");
  if (c.chunk <= 0) c.chunk = 16;
  if (c.setup_threads == 0) c.setup_threads = 4;
  auto* s = new (std::nothrow) mfx_server();
  if (!s) return set_error(MFX_ENOMEM, "host allocation failed");
  s->cfg = c;
  s->t0 = Clock::now();
  cudaGetDevice(&s->device);
  if (cudaStreamCreateWithFlags(&s->release_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete s;
    return set_error(MFX_ECUDA, "mfx_server_create: stream");
  }
  mfx_status rc = mfx_batch_create(&s->batch, c.max_slots, c.chunk);
  if (rc != MFX_OK) {
    cudaStreamDestroy(s->release_stream);
    delete s;
    return rc;
  }
  for (int i = 0; i < c.setup_threads; ++i) s->workers.emplace_back(worker_main, s);
  s->scheduler = std::thread(scheduler_main, s);
  *out = s;
  return MFX_OK;
} catch (...) {
  return host_exception();
}

void mfx_server_destroy(mfx_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stop = true;
    for (auto& q : s->queue) finish_locked(s, *q, MFX_REQ_CANCELLED);
    s->queue.clear();
  }
  s->cv_setup.notify_all();
  s->cv_sched.notify_all();
  for (auto& w : s->workers) w.join();  // each finishes the set-up it is in
  s->cv_sched.notify_all();
  s->scheduler.join();                  // cancels the rest, releases running slots
  mfx_batch_destroy(s->batch);
  for (auto& kv : s->reqs) free_request(s, *kv.second);
  cudaStreamSynchronize(s->release_stream);
  cudaStreamDestroy(s->release_stream);
  delete s;
}

mfx_status mfx_server_submit(mfx_server* s, const mfx_request* request, int64_t* ticket) try {
  if (!s || !request || !ticket) return set_error(MFX_EINVAL, "null argument");
  auto q = std::make_shared<Req>();
  q->r = *request;
  int64_t n_cells = 0;
  if (request->mesh) {
    const mfx::Mesh& m = request->mesh->m;
    n_cells = m.structured ? (int64_t)m.nx * m.ny * m.nz : (int64_t)m.leaves.size() / 4;
  } else {
    if (!request->leaves || request->n_leaves < 1 || request->nx < 1 || request->ny < 1 || request->nz < 1)
      return set_error(MFX_EINVAL, "mfx_server_submit: no mesh and no octree description");
    q->leaves.assign(request->leaves, request->leaves + 4 * request->n_leaves);
    if (request->coarse_vertices)
      q->verts.assign(request->coarse_vertices,
                      request->coarse_vertices + 3 * (int64_t)(request->nx + 1) * (request->ny + 1) * (request->nz + 1));
    n_cells = request->n_leaves;
  }
  if (request->desc.degree < 1 || request->desc.degree > mfx::kMaxDegree)
    return set_error(MFX_EUNSUPPORTED, "degree must be in 1..8");
  q->r.leaves = nullptr;
  q->r.coarse_vertices = nullptr;
  q->est = request->est_bytes > 0 ? request->est_bytes : estimate_bytes(n_cells, request->desc.degree);
  {
    std::lock_guard<std::mutex> g(s->mu);
    if (s->stop) return set_error(MFX_EINVAL, "server is stopping");
    q->ticket = s->next_ticket++;
    q->t_submit = s->now();
    s->reqs[q->ticket] = q;
    s->queue.push_back(q);
    ++s->counts.submitted;
    *ticket = q->ticket;
  }
  s->cv_sched.notify_one();
  return MFX_OK;
} catch (...) {
  return host_exception();
}

mfx_status mfx_server_poll(mfx_server* s, int64_t ticket, mfx_request_info* info) {
  if (!s || !info) return set_error(MFX_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(MFX_EINVAL, "unknown ticket");
  const Req& q = *it->second;
  *info = mfx_request_info{};
  info->state = q.state;
  info->error = q.error;
  info->n_dofs = q.n_dofs;
  info->bytes = q.bytes;
  info->t_submit = q.t_submit;
  info->t_admit = q.t_admit;
  info->t_ready = q.t_ready;
  info->t_done = q.t_done;
  info->setup_seconds = q.setup_s;
  info->stats = q.stats;
  return MFX_OK;
}

mfx_status mfx_server_cancel(mfx_server* s, int64_t ticket) {
  if (!s) return set_error(MFX_EINVAL, "null server");
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(MFX_EINVAL, "unknown ticket");
    Req& q = *it->second;
    if (q.state == MFX_REQ_QUEUED) {
      auto pos = std::find(s->queue.begin(), s->queue.end(), it->second);
      if (pos != s->queue.end()) s->queue.erase(pos);
      finish_locked(s, q, MFX_REQ_CANCELLED);
    } else if (q.state == MFX_REQ_SETUP || q.state == MFX_REQ_RUNNING) {
      q.cancel = true;
    }
  }
  s->cv_sched.notify_one();
  return MFX_OK;
}

mfx_status mfx_server_result_copy(mfx_server* s, int64_t ticket, double* x_host, int64_t n) {
  if (!s || !x_host) return set_error(MFX_EINVAL, "null argument");
  ReqPtr q;
  {
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return set_error(MFX_EINVAL, "unknown ticket");
    q = it->second;
    if (q->state != MFX_REQ_DONE) return set_error(MFX_EBUSY, "request is not done");
    if (n != q->n_dofs) return set_error(MFX_EINVAL, "size differs from the request's n_dofs");
    ++q->pinned;
  }
  const cudaError_t e = cudaMemcpy(x_host, q->x, sizeof(double) * n, cudaMemcpyDeviceToHost);
  {
    std::lock_guard<std::mutex> g(s->mu);
    --q->pinned;
  }
  if (e != cudaSuccess) return set_error(MFX_ECUDA, std::string("result copy: ") + cudaGetErrorString(e));
  return MFX_OK;
}

mfx_status mfx_server_operator(mfx_server* s, int64_t ticket, const mfx_op** op) {
  if (!s || !op) return set_error(MFX_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(MFX_EINVAL, "unknown ticket");
  if (it->second->state != MFX_REQ_DONE) return set_error(MFX_EBUSY, "request is not done");
  *op = it->second->op;
  return MFX_OK;
}

mfx_status mfx_server_retire(mfx_server* s, int64_t ticket) {
  if (!s) return set_error(MFX_EINVAL, "null server");
  std::lock_guard<std::mutex> g(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return set_error(MFX_EINVAL, "unknown ticket");
  Req& q = *it->second;
  if (q.state == MFX_REQ_QUEUED || q.state == MFX_REQ_SETUP || q.state == MFX_REQ_RUNNING || q.pinned > 0)
    return set_error(MFX_EBUSY, "request still in flight");
  free_request(s, q);
  s->bytes_in_use -= q.bytes;
  ++s->counts.retired;
  s->reqs.erase(it);
  s->cv_sched.notify_one();
  return MFX_OK;
}

mfx_status mfx_server_stats_get(mfx_server* s, mfx_server_stats* st) {
  if (!s || !st) return set_error(MFX_EINVAL, "null argument");
  std::lock_guard<std::mutex> g(s->mu);
  mfx_server_stats c = s->counts;
  c.queued = c.in_setup = c.running = c.done = c.cancelled = c.failed = 0;
  for (auto& kv : s->reqs) {
    switch (kv.second->state) {
      case MFX_REQ_QUEUED: ++c.queued; break;
      case MFX_REQ_SETUP: ++c.in_setup; break;
      case MFX_REQ_RUNNING: ++c.running; break;
      case MFX_REQ_DONE: ++c.done; break;
      case MFX_REQ_CANCELLED: ++c.cancelled; break;
      default: ++c.failed; break;
    }
  }
  c.bytes_in_use = s->bytes_in_use;
  c.now = s->now();
  *st = c;
  return MFX_OK;
}

}  // extern "C"
