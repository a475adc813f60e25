// Request server: many independent contact solves in flight on one GPU.
//
// Worker threads (one CUDA stream each, through their handles) take jobs from
// a queue.  A job is admitted when its device-memory footprint fits the HBM
// budget next to the jobs already running and the cached handles; a job that
// does not fit lets later, smaller jobs go first (continuous batching rather
// than a plain FIFO), and idle cached handles are evicted least recently used
// first to make room.  Handles are cached by (Nx, Ny, dx, dy, k): the influence
// spectrum depends only on these, and nu, E0, c0 enter through the scalar A,
// which bem_set_material updates.  Each solve is deterministic and touches only
// its own handle, so its result is the same alone and in any mix.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "bem.h"
#include "bem_impl.h"

namespace {

int pow2_at_least(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Device bytes a handle of this grid holds after FP32 and FP64 solves, plus the
// set-up workspace of bem_create (the largest transient).
size_t footprint(int nx, int ny) {
  const size_t px = pow2_at_least(2 * nx < 32 ? 32 : 2 * nx), py = pow2_at_least(2 * ny < 32 ? 32 : 2 * ny);
  const size_t M = px / 2, hyq = py / 2 + 1, n = (size_t)nx * ny;
  size_t b = 0;
  b += hyq * (M + 1) * 8;               // influence quarter
  b += hyq * (M + 1) * 12;              // spectrum FP64 + FP32
  b += (2 * M + py + 1) * 24;           // twiddles
  b += 2 * (224 + M + py) * 4;          // index tables
  b += 16 * (M + 1) * ny;               // W (FP64 size)
  b += 3 * 8 * n + n;                   // profile, two FP64 staging fields, contact set
  b += 5 * 4 * n + 5 * 8 * n;           // FP32 and FP64 CG fields
  b += 16 * (M + 1) * py;               // spectrum set-up workspace
  b += 1 << 20;                         // partial sums, statistics, scalars
  b += b / 3;                           // contact-box sub-contexts (tori of 1/4, 1/16, ... the area)
  return b;
}

double now_s(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

struct Key {
  int nx, ny;
  double dx, dy, k;
  bool operator==(const Key& o) const {
    return nx == o.nx && ny == o.ny && dx == o.dx && dy == o.dy && k == o.k;
  }
};

struct Cached {
  Key key;
  bem_handle h;
  size_t bytes;
  bool busy;
};

struct Pending {
  bem_job job;
  double t_submit;
  size_t need;
};

}  // namespace

struct bem_server {
  int device = 0;
  size_t budget = 0;
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::list<Cached> cache;  // front = most recently used
  size_t used = 0;          // bytes of cached handles (busy or idle) + reservations
  int running = 0;
  bool stop = false;
  std::deque<bem_completion> done;
  std::vector<std::thread> workers;
};

namespace {

// Find a cached idle handle for key (moved to the front) or nullptr.
Cached* take_cached(bem_server* s, const Key& k) {
  for (auto it = s->cache.begin(); it != s->cache.end(); ++it) {
    if (!it->busy && it->key == k) {
      s->cache.splice(s->cache.begin(), s->cache, it);
      s->cache.front().busy = true;
      return &s->cache.front();
    }
  }
  return nullptr;
}

// Evict idle cached handles (least recently used first) until `need` bytes fit.
bool make_room(bem_server* s, size_t need) {
  while (s->used + need > s->budget) {
    auto it = s->cache.end();
    bool found = false;
    while (it != s->cache.begin()) {
      --it;
      if (!it->busy) { found = true; break; }
    }
    if (!found) return false;
    s->used -= it->bytes;
    bem_destroy(it->h);
    s->cache.erase(it);
  }
  return true;
}

void worker_main(bem_server* s) {
  cudaSetDevice(s->device);
  for (;;) {
    Pending p;
    Cached* slot = nullptr;
    size_t reserved = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      for (;;) {
        if (s->stop && s->queue.empty()) return;
        // first queued job that is cached or fits the budget (after evictions)
        bool picked = false;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          const Key k{it->job.Nx, it->job.Ny, it->job.dx, it->job.dy, it->job.k};
          if ((slot = take_cached(s, k)) != nullptr) {
            // room for the fields of a precision the cached handle has not used yet
            const size_t grow = it->need > slot->bytes ? it->need - slot->bytes : 0;
            if (make_room(s, grow)) {
              p = *it;
              reserved = grow;
              s->used += reserved;
              s->queue.erase(it);
              picked = true;
              break;
            }
            slot->busy = false;
            slot = nullptr;
          }
          if (make_room(s, it->need)) {
            p = *it;
            reserved = it->need;
            s->used += reserved;
            s->queue.erase(it);
            picked = true;
            break;
          }
        }
        if (picked) break;
        s->cv_work.wait(lk);
      }
      s->running++;
    }
    bem_completion c{};
    c.tag = p.job.tag;
    c.t_submit = p.t_submit;
    c.t_start = now_s(s->t0);
    int rc = BEM_OK;
    p.job.opts.stream = nullptr;
    bem_handle h = slot ? slot->h : nullptr;
    if (!h) {
      rc = bem_create(p.job.Nx, p.job.Ny, p.job.dx, p.job.dy, p.job.k, p.job.nu, p.job.E0, p.job.c0, &h);
    } else {
      rc = bem_set_material(h, p.job.nu, p.job.E0, p.job.c0);
    }
    if (rc == BEM_OK)
      rc = bem_sweep(h, p.job.profile, p.job.d_steps, p.job.nsteps, p.job.dgamma, &p.job.opts,
                     p.job.per_step, p.job.final_pressure);
    c.t_end = now_s(s->t0);
    c.status = rc;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->used -= reserved;
      if (slot) {
        // the job may have allocated the other precision's fields
        bem_info inf;
        if (bem_get_info(h, &inf) == BEM_OK && inf.device_bytes != slot->bytes) {
          s->used = s->used - slot->bytes + inf.device_bytes;
          slot->bytes = inf.device_bytes;
        }
        slot->busy = false;
      } else {
        if (h) {
          bem_info inf;
          size_t bytes = reserved;
          if (bem_get_info(h, &inf) == BEM_OK) bytes = inf.device_bytes;
          if (rc == BEM_OK || rc == BEM_ENOCONV) {
            s->cache.push_front(Cached{Key{p.job.Nx, p.job.Ny, p.job.dx, p.job.dy, p.job.k}, h, bytes, false});
            s->used += bytes;
          } else {
            bem_destroy(h);
          }
        }
      }
      // keep the cache within the budget
      make_room(s, 0);
      s->running--;
      s->done.push_back(c);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" size_t bem_server_footprint(int Nx, int Ny) {
  if (Nx < 2 || Ny < 2 || Nx > 4096 || Ny > 4096) return 0;
  return footprint(Nx, Ny);
}

extern "C" int bem_server_create(int nworkers, size_t hbm_budget_bytes, bem_server_handle* out) {
  if (!out || nworkers < 1 || nworkers > 64 || hbm_budget_bytes < ((size_t)64 << 20))
    return bem::set_error(BEM_EINVAL, "bem_server_create: nworkers must be 1..64 and the budget at least 64 MiB");
  int dev = 0, ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return bem::set_error(BEM_ECUDA, "bem_server_create: no CUDA device");
  }
  bem_server* s = new bem_server();
  s->device = dev;
  s->budget = hbm_budget_bytes;
  s->t0 = std::chrono::steady_clock::now();
  for (int i = 0; i < nworkers; ++i) s->workers.emplace_back(worker_main, s);
  *out = s;
  return BEM_OK;
}

extern "C" int bem_server_submit(bem_server_handle s, const bem_job* job) {
  if (!s || !job || !job->profile || !job->d_steps || !job->per_step || job->nsteps < 1)
    return bem::set_error(BEM_EINVAL, "bem_server_submit: NULL array or nsteps < 1");
  if (job->Nx < 2 || job->Ny < 2 || job->Nx > 4096 || job->Ny > 4096)
    return bem::set_error(BEM_EINVAL, "bem_server_submit: Nx and Ny must be in 2..4096");
  const size_t need = footprint(job->Nx, job->Ny);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return bem::set_error(BEM_EINVAL, "bem_server_submit: server is shutting down");
  if (need > s->budget) return bem::set_error(BEM_ENOMEM, "bem_server_submit: job footprint exceeds the budget");
  s->queue.push_back(Pending{*job, now_s(s->t0), need});
  s->cv_work.notify_one();
  return BEM_OK;
}

extern "C" int bem_server_poll(bem_server_handle s, bem_completion* out, int max, int wait_ms) {
  if (!s || !out || max < 1) return BEM_EINVAL;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int n = 0;
  while (n < max && !s->done.empty()) {
    out[n++] = s->done.front();
    s->done.pop_front();
  }
  return n;
}

extern "C" int bem_server_cancel(bem_server_handle s, long long tag) {
  if (!s) return bem::set_error(BEM_EINVAL, "bem_server_cancel: NULL server");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
      if (it->job.tag != tag) continue;
      bem_completion c{};
      c.tag = tag;
      c.status = BEM_ECANCELED;
      c.t_submit = it->t_submit;
      c.t_start = c.t_end = now_s(s->t0);
      s->queue.erase(it);
      s->done.push_back(c);
      s->cv_done.notify_all();
      return BEM_OK;
    }
  }
  return bem::set_error(BEM_EINVAL, "bem_server_cancel: no queued job with this tag");
}

extern "C" int bem_server_pending(bem_server_handle s) {
  if (!s) return BEM_EINVAL;
  std::lock_guard<std::mutex> lk(s->mu);
  return (int)s->queue.size() + s->running;
}

extern "C" size_t bem_server_bytes(bem_server_handle s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  return s->used;
}

extern "C" void bem_server_destroy(bem_server_handle s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  for (auto& c : s->cache) bem_destroy(c.h);
  delete s;
}
