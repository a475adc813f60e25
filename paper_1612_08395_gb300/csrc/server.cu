// Request server: many independent contact solves in flight on one or more GPUs.
//
// Worker threads (one CUDA stream each, through their handles) take jobs from
// a shared queue; each worker belongs to one device.  A job is admitted on a
// device when its device-memory footprint fits that device's HBM budget next
// to the jobs already running there and the handles cached there; a job that
// does not fit yet lets later, smaller jobs go first (continuous batching
// rather than a plain FIFO), and idle cached handles are evicted least
// recently used first to make room.  With several devices, the placement
// policy (place_job) sends a job to a device with an idle worker where it
// fits, preferring one that holds an idle cached handle for its spectrum,
// then the one with the most budget left after it.  Devices never share
// work: a solve runs wholly on its device (no collective, no peer memory).
// Handles are cached per device by (Nx, Ny, dx, dy, k): the influence
// spectrum depends only on these, and nu, E0, c0 enter through the scalar A,
// which bem_set_material updates.  Each solve is deterministic and touches
// only its own handle, so its result is the same alone and in any mix.
#include <math.h>
#include <stdlib.h>

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

// One device's share of the server: its budget, cached handles and workers.
struct DevPool {
  int device = 0;
  size_t budget = 0;
  size_t used = 0;          // bytes of cached handles (busy or idle) + reservations
  std::list<Cached> cache;  // front = most recently used
  int workers = 0, busy = 0;
  // CG loops of the jobs running here join this batcher (null: each job
  // launches its own loops; BEM_BATCH_LOOPS=0 switches batching off)
  bem::LoopBatcher* batcher = nullptr;
  bool batcher_tried = false;
};

}  // namespace

struct bem_server {
  std::chrono::steady_clock::time_point t0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;
  std::vector<DevPool> devs;
  int running = 0;
  bool stop = false;
  std::deque<bem_completion> done;
  std::vector<std::thread> workers;
};

namespace {

// Find a cached idle handle for key (moved to the front) or nullptr.
Cached* take_cached(DevPool& d, const Key& k) {
  for (auto it = d.cache.begin(); it != d.cache.end(); ++it) {
    if (!it->busy && it->key == k) {
      d.cache.splice(d.cache.begin(), d.cache, it);
      d.cache.front().busy = true;
      return &d.cache.front();
    }
  }
  return nullptr;
}

// Evict idle cached handles (least recently used first) until `need` bytes fit.
bool make_room(DevPool& d, size_t need) {
  while (d.used + need > d.budget) {
    auto it = d.cache.end();
    bool found = false;
    while (it != d.cache.begin()) {
      --it;
      if (!it->busy) { found = true; break; }
    }
    if (!found) return false;
    d.used -= it->bytes;
    bem_destroy(it->h);
    d.cache.erase(it);
  }
  return true;
}

// The placement view of every device for one job (see bem_device_view).
void device_views(const bem_server* s, const Key& k, std::vector<bem_device_view>& v) {
  v.resize(s->devs.size());
  for (size_t i = 0; i < s->devs.size(); ++i) {
    const DevPool& d = s->devs[i];
    bem_device_view& w = v[i];
    w.budget = d.budget;
    w.used = d.used;
    w.evictable = 0;
    w.cached_bytes = 0;
    w.has_cached = 0;
    for (const Cached& c : d.cache) {
      if (c.busy) continue;
      if (!w.has_cached && c.key == k) { w.has_cached = 1; w.cached_bytes = c.bytes; }
      else w.evictable += c.bytes;
    }
    w.idle_workers = d.workers - d.busy;
  }
}

void worker_main(bem_server* s, int di) {
  cudaSetDevice(s->devs[di].device);
  {
    std::lock_guard<std::mutex> lk(s->mu);
    DevPool& dev = s->devs[di];
    if (!dev.batcher_tried) {
      dev.batcher_tried = true;
      const char* env = getenv("BEM_BATCH_LOOPS");
      if (!(env && env[0] == '0')) dev.batcher = bem::batcher_create();
    }
  }
  bem::LoopBatcher* batcher = s->devs[di].batcher;
  std::vector<bem_device_view> views;
  for (;;) {
    Pending p;
    Cached* slot = nullptr;
    size_t reserved = 0;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      DevPool& dev = s->devs[di];
      for (;;) {
        if (s->stop && s->queue.empty()) return;
        // the first queued job whose placement is this worker's device
        bool picked = false;
        for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
          const Key k{it->job.Nx, it->job.Ny, it->job.dx, it->job.dy, it->job.k};
          device_views(s, k, views);
          if (bem_server_place((int)views.size(), views.data(), it->need) != di) continue;
          if ((slot = take_cached(dev, k)) != nullptr) {
            // room for the fields of a precision the cached handle has not used yet
            const size_t grow = it->need > slot->bytes ? it->need - slot->bytes : 0;
            if (make_room(dev, grow)) {
              p = *it;
              reserved = grow;
              dev.used += reserved;
              s->queue.erase(it);
              picked = true;
              break;
            }
            slot->busy = false;
            slot = nullptr;
          }
          if (make_room(dev, it->need)) {
            p = *it;
            reserved = it->need;
            dev.used += reserved;
            s->queue.erase(it);
            picked = true;
            break;
          }
        }
        if (picked) break;
        s->cv_work.wait(lk);
      }
      dev.busy++;
      s->running++;
    }
    // another device's worker may be the placement of the next queued job
    s->cv_work.notify_all();
    bem_completion c{};
    c.tag = p.job.tag;
    c.device = s->devs[di].device;
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
    if (rc == BEM_OK) {
      if (batcher) {
        bem::attach_batcher(h, batcher);
        bem::batcher_enter(batcher);
      }
      rc = bem_sweep(h, p.job.profile, p.job.d_steps, p.job.nsteps, p.job.dgamma, &p.job.opts,
                     p.job.per_step, p.job.final_pressure);
      if (batcher) bem::batcher_leave(batcher);
    }
    c.t_end = now_s(s->t0);
    c.status = rc;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      DevPool& dev = s->devs[di];
      dev.used -= reserved;
      if (slot) {
        // the job may have allocated the other precision's fields
        bem_info inf;
        if (bem_get_info(h, &inf) == BEM_OK && inf.device_bytes != slot->bytes) {
          dev.used = dev.used - slot->bytes + inf.device_bytes;
          slot->bytes = inf.device_bytes;
        }
        slot->busy = false;
      } else {
        if (h) {
          bem_info inf;
          size_t bytes = reserved;
          if (bem_get_info(h, &inf) == BEM_OK) bytes = inf.device_bytes;
          if (rc == BEM_OK || rc == BEM_ENOCONV) {
            dev.cache.push_front(Cached{Key{p.job.Nx, p.job.Ny, p.job.dx, p.job.dy, p.job.k}, h, bytes, false});
            dev.used += bytes;
          } else {
            bem_destroy(h);
          }
        }
      }
      // keep the cache within the budget
      make_room(dev, 0);
      dev.busy--;
      s->running--;
      s->done.push_back(c);
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int bem_server_place(int ndev, const bem_device_view* v, size_t need) {
  if (ndev < 1 || !v) return -1;
  int best = -1;
  bool best_cached = false;
  size_t best_left = 0;
  for (int i = 0; i < ndev; ++i) {
    if (v[i].idle_workers < 1) continue;
    const bool cached = v[i].has_cached != 0;
    const size_t here = cached ? (need > v[i].cached_bytes ? need - v[i].cached_bytes : 0) : need;
    // bytes that stay held: running jobs' reservations and busy handles (idle
    // cached handles other than the job's own can be evicted)
    const size_t idle = v[i].evictable + (cached ? v[i].cached_bytes : 0);
    const size_t pinned = v[i].used > idle ? v[i].used - idle : 0;
    const size_t keep = pinned + (cached ? v[i].cached_bytes : 0);
    if (keep + here > v[i].budget) continue;
    const size_t left = v[i].budget - (keep + here);
    if (best < 0 || (cached && !best_cached) || (cached == best_cached && left > best_left)) {
      best = i;
      best_cached = cached;
      best_left = left;
    }
  }
  return best;
}

extern "C" size_t bem_server_footprint(int Nx, int Ny) {
  if (Nx < 2 || Ny < 2 || Nx > 4096 || Ny > 4096) return 0;
  return footprint(Nx, Ny);
}

extern "C" int bem_server_create_on(int ndev, const int* devices, int workers_per_device,
                                    size_t hbm_budget_per_device, bem_server_handle* out) {
  if (!out || ndev < 1 || ndev > 64 || !devices || workers_per_device < 1 || workers_per_device > 64 ||
      hbm_budget_per_device < ((size_t)64 << 20))
    return bem::set_error(BEM_EINVAL, "bem_server_create_on: 1..64 devices, 1..64 workers each and a budget "
                                      "of at least 64 MiB per device");
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count < 1) {
    cudaGetLastError();
    return bem::set_error(BEM_ECUDA, "bem_server_create_on: no CUDA device");
  }
  for (int i = 0; i < ndev; ++i) {
    if (devices[i] < 0 || devices[i] >= count)
      return bem::set_error(BEM_EINVAL, "bem_server_create_on: device index out of range");
    for (int j = 0; j < i; ++j)
      if (devices[j] == devices[i]) return bem::set_error(BEM_EINVAL, "bem_server_create_on: repeated device");
  }
  bem_server* s = new bem_server();
  s->t0 = std::chrono::steady_clock::now();
  s->devs.resize(ndev);
  for (int i = 0; i < ndev; ++i) {
    s->devs[i].device = devices[i];
    s->devs[i].budget = hbm_budget_per_device;
    s->devs[i].workers = workers_per_device;
  }
  for (int i = 0; i < ndev; ++i)
    for (int w = 0; w < workers_per_device; ++w) s->workers.emplace_back(worker_main, s, i);
  *out = s;
  return BEM_OK;
}

extern "C" int bem_server_create(int nworkers, size_t hbm_budget_bytes, bem_server_handle* out) {
  if (!out || nworkers < 1 || nworkers > 64 || hbm_budget_bytes < ((size_t)64 << 20))
    return bem::set_error(BEM_EINVAL, "bem_server_create: nworkers must be 1..64 and the budget at least 64 MiB");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return bem::set_error(BEM_ECUDA, "bem_server_create: no CUDA device");
  }
  return bem_server_create_on(1, &dev, nworkers, hbm_budget_bytes, out);
}

extern "C" int bem_server_submit(bem_server_handle s, const bem_job* job) {
  if (!s || !job || !job->profile || !job->d_steps || !job->per_step || job->nsteps < 1)
    return bem::set_error(BEM_EINVAL, "bem_server_submit: NULL array or nsteps < 1");
  if (job->Nx < 2 || job->Ny < 2 || job->Nx > 4096 || job->Ny > 4096)
    return bem::set_error(BEM_EINVAL, "bem_server_submit: Nx and Ny must be in 2..4096");
  const size_t need = footprint(job->Nx, job->Ny);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return bem::set_error(BEM_EINVAL, "bem_server_submit: server is shutting down");
  size_t largest = 0;
  for (const DevPool& d : s->devs) largest = d.budget > largest ? d.budget : largest;
  if (need > largest) return bem::set_error(BEM_ENOMEM, "bem_server_submit: job footprint exceeds the budget");
  s->queue.push_back(Pending{*job, now_s(s->t0), need});
  s->cv_work.notify_all();
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
      c.device = -1;
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

extern "C" int bem_server_loop_stats(bem_server_handle s, long long* launches, long long* loops) {
  if (!s || !launches || !loops) return bem::set_error(BEM_EINVAL, "bem_server_loop_stats: NULL argument");
  *launches = 0;
  *loops = 0;
  std::lock_guard<std::mutex> lk(s->mu);
  for (DevPool& d : s->devs)
    if (d.batcher) bem::batcher_stats(d.batcher, launches, loops);
  return BEM_OK;
}

extern "C" size_t bem_server_bytes(bem_server_handle s) {
  if (!s) return 0;
  std::lock_guard<std::mutex> lk(s->mu);
  size_t b = 0;
  for (const DevPool& d : s->devs) b += d.used;
  return b;
}

extern "C" void bem_server_destroy(bem_server_handle s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  int prev = 0;
  const bool have_prev = cudaGetDevice(&prev) == cudaSuccess;
  for (DevPool& d : s->devs) {
    cudaSetDevice(d.device);
    for (auto& c : d.cache) bem_destroy(c.h);
    bem::batcher_destroy(d.batcher);
  }
  if (have_prev) cudaSetDevice(prev);
  delete s;
}
