// Serving loop of many concurrent episodes (include/nf.h, "serving").
//
// Design: `slots` worker threads, each owning an nf_ctx (its own CUDA stream,
// reduction scratch and captured solver graphs). An episode is bound to the
// slot that admits it; its requests run there in submission order, while the
// other slots run other episodes' requests at the same time on their own
// streams, so the device overlaps their kernels. Admission: an OPEN reserves
// an estimate of the episode's device bytes against the budget; OPENs that
// do not fit wait in FIFO order (and so do the requests queued behind them)
// until a CLOSE returns memory.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "ctx.h"

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
  int64_t ticket = 0;
  nf_request req{};
  std::vector<double> spheres;  // owned copy of an OPEN's sphere list
  std::vector<double> shapes;   // owned copy of an OPEN's shape table
  double submit_ms = 0.0;
};

struct EpisodeRec {
  int slot = -1;           // -1 until admitted
  int nx = 0, ny = 0, nz = 0;  // cell counts (batching: same-size members)
  int64_t id = 0;          // episode id inside the slot's nf_ctx
  bool created = false;
  bool failed = false;
  size_t estimate = 0;     // reservation made at admission
  size_t reserved = 0;     // bytes currently held against the budget
  std::deque<Job> waiting; // the OPEN and later requests, until admitted
};

struct Slot {
  nf_ctx *ctx = nullptr;
  std::deque<Job> queue;
  std::condition_variable cv;
  std::thread worker;
  int pending = 0;         // queued + running requests
};

}  // namespace

struct nf_server {
  nf_config cfg{};
  int device = 0;
  size_t budget = 0, reserved = 0, peak = 0;
  std::vector<std::unique_ptr<Slot>> slots;
  std::map<int64_t, EpisodeRec> eps;
  std::deque<int64_t> open_wait;
  std::map<int64_t, nf_result> done;
  std::set<int64_t> in_flight;
  std::mutex mu;
  std::condition_variable done_cv;
  int64_t next_ticket = 1, submitted = 0, completed = 0;
  int64_t batches = 0, batched_requests = 0;
  int batch_max = 1;       // most episodes stepped as one batch (1: none)
  int64_t batch_cells = 64 * 64 * 64;  // only episodes of at most this many cells batch
  bool batchable(const EpisodeRec &r) const {
    return batch_max > 1 && (int64_t)r.nx * r.ny * r.nz <= batch_cells;
  }
  bool stop = false;
  Clock::time_point t0 = Clock::now();

  double now_ms() const {
    return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
  }

  size_t estimate(const nf_grid &g) const {
    const size_t nf = (size_t)(g.nx + 1) * g.ny * g.nz + (size_t)g.nx * (g.ny + 1) * g.nz +
                      (size_t)g.nx * g.ny * (g.nz + 1);
    const size_t nc = (size_t)g.nx * g.ny * g.nz;
    const size_t t = cfg.precision == NF_PREC_FP64 ? 8 : 4;
    const size_t s = cfg.precision == NF_PREC_FP32 ? 4 : 8;
    const size_t C = (size_t)std::max(1, cfg.checkpoint_every);
    // base state + a segment's tape (U, U^, alpha, P per step) + checkpoints
    return nf::episode_base_bytes(cfg, g) + (C + 2) * (3 * nf * t + nc * s);
  }

  // The slot with the fewest queued or running requests; with batching, a
  // slot that already holds episodes of the same cell counts when it is
  // within two requests of the least loaded (their steps can then share
  // launches).
  int pick_slot(const EpisodeRec &rec) const {
    int best = 0;
    for (int s = 1; s < (int)slots.size(); ++s)
      if (slots[s]->pending < slots[best]->pending) best = s;
    if (!batchable(rec)) return best;
    std::vector<int> same(slots.size(), 0);
    for (const auto &kv : eps) {
      const EpisodeRec &o = kv.second;
      if (&o != &rec && o.slot >= 0 && o.nx == rec.nx && o.ny == rec.ny && o.nz == rec.nz)
        same[o.slot] += 1;
    }
    int pick = -1;
    for (int s = 0; s < (int)slots.size(); ++s)
      if (same[s] > 0 && slots[s]->pending <= slots[best]->pending + 2 &&
          (pick < 0 || slots[s]->pending < slots[pick]->pending))
        pick = s;
    return pick >= 0 ? pick : best;
  }

  void enqueue(int s, Job &&job) {
    slots[s]->queue.push_back(std::move(job));
    slots[s]->pending += 1;
    slots[s]->cv.notify_one();
  }

  bool fits(size_t bytes) const { return budget == 0 || reserved + bytes <= budget; }

  void admit(int64_t key, EpisodeRec &rec) {
    rec.slot = pick_slot(rec);
    rec.reserved = rec.estimate;
    reserved += rec.reserved;
    peak = std::max(peak, reserved);
    while (!rec.waiting.empty()) {
      enqueue(rec.slot, std::move(rec.waiting.front()));
      rec.waiting.pop_front();
    }
    (void)key;
  }

  // Admit waiting OPENs in arrival order while the budget allows.
  void admit_waiting() {
    while (!open_wait.empty()) {
      auto it = eps.find(open_wait.front());
      if (it == eps.end()) {
        open_wait.pop_front();
        continue;
      }
      if (!fits(it->second.estimate)) break;
      admit(it->first, it->second);
      open_wait.pop_front();
    }
  }

  void finish(int64_t ticket, const nf_result &res) {
    done[ticket] = res;
    in_flight.erase(ticket);
    completed += 1;
    done_cv.notify_all();
  }

  nf_result immediate(const Job &job, int status) const {
    nf_result r{};
    r.status = status;
    r.kind = job.req.kind;
    r.episode = job.req.episode;
    r.submit_ms = r.start_ms = r.end_ms = job.submit_ms;
    return r;
  }

  void work(int s);
  // Under the lock: queued step requests of the same slot that can run as
  // one batch with `first` (same cell counts and frames, distinct episodes,
  // each the oldest queued request of its episode, or the first after the
  // episode's own queued OPEN, which then runs first: `opens`).
  void gather_batch(Slot &slot, const Job &first, std::vector<Job> &group,
                    std::vector<Job> &opens);
  // Under the lock: bookkeeping of a finished request.
  void complete(Slot &slot, const Job &job, nf_result &res, int64_t id, bool created,
                size_t bytes);
};

void nf_server::gather_batch(Slot &slot, const Job &first_job, std::vector<Job> &group,
                             std::vector<Job> &opens) {
  // (group grows below: keep copies, not a reference into it)
  const int64_t first = first_job.req.episode;
  const int frames = first_job.req.frames;
  auto f = eps.find(first);
  if (f == eps.end() || !batchable(f->second) || !f->second.created || f->second.failed) return;
  const int nx = f->second.nx, ny = f->second.ny, nz = f->second.nz;
  std::set<int64_t> seen = {first};
  std::map<int64_t, size_t> open_at;  // episodes whose only queued job so far is their OPEN
  std::vector<size_t> take_open, take_step;
  for (size_t i = 0; i < slot.queue.size() && (int)(group.size() + take_step.size()) < batch_max;
       ++i) {
    const Job &q = slot.queue[i];
    const int64_t key = q.req.episode;
    if (seen.count(key)) continue;
    auto e = eps.find(key);
    const bool same = e != eps.end() && !e->second.failed && e->second.nx == nx &&
                      e->second.ny == ny && e->second.nz == nz;
    const auto o = open_at.find(key);
    if (q.req.kind == NF_REQ_OPEN && same && !e->second.created && o == open_at.end()) {
      open_at[key] = i;  // its first step may join, the OPEN run just before the batch
      continue;
    }
    const bool step = (q.req.kind == NF_REQ_STEP || q.req.kind == NF_REQ_STEP_ADJOINT) &&
                      q.req.frames == frames;
    if (step && same && (e->second.created || o != open_at.end())) {
      if (o != open_at.end()) take_open.push_back(o->second);
      take_step.push_back(i);
    }
    seen.insert(key);  // later requests of this episode wait for this one
  }
  std::vector<size_t> all(take_open);
  all.insert(all.end(), take_step.begin(), take_step.end());
  for (size_t i : take_open) opens.push_back(std::move(slot.queue[i]));
  for (size_t i : take_step) group.push_back(std::move(slot.queue[i]));
  std::sort(all.begin(), all.end());
  for (auto it = all.rbegin(); it != all.rend(); ++it)
    slot.queue.erase(slot.queue.begin() + (std::ptrdiff_t)*it);
}

void nf_server::complete(Slot &slot, const Job &job, nf_result &res, int64_t id, bool created,
                         size_t bytes) {
  slot.pending -= 1;
  auto it = eps.find(job.req.episode);
  if (it != eps.end()) {
    EpisodeRec &rec = it->second;
    if (job.req.kind == NF_REQ_OPEN) {
      rec.id = id;
      rec.created = created;
      rec.failed = !created;
      if (rec.failed) {  // nothing stays resident: release the reservation
        reserved -= std::min(reserved, rec.reserved);
        rec.reserved = 0;
      }
    }
    if (job.req.kind == NF_REQ_CLOSE) {
      // memory returns to the budget
      reserved -= std::min(reserved, rec.reserved);
      eps.erase(it);
    } else if (bytes > rec.reserved) {
      reserved += bytes - rec.reserved;
      rec.reserved = bytes;
      peak = std::max(peak, reserved);
    }
    admit_waiting();
  }
  finish(job.ticket, res);
}

void nf_server::work(int s) {
  cudaSetDevice(device);
  Slot &slot = *slots[s];
  for (;;) {
    std::vector<Job> group, opens;
    std::vector<int64_t> ids;
    std::vector<char> created, failed;
    {
      std::unique_lock<std::mutex> lk(mu);
      slot.cv.wait(lk, [&] { return stop || !slot.queue.empty(); });
      if (slot.queue.empty()) return;  // stop requested and nothing left
      group.push_back(std::move(slot.queue.front()));
      slot.queue.pop_front();
      if (group[0].req.kind == NF_REQ_STEP || group[0].req.kind == NF_REQ_STEP_ADJOINT)
        gather_batch(slot, group[0], group, opens);
    }
    // the OPENs of batch members whose episode was not created yet run first
    // (each request of an episode still runs in its submission order)
    for (Job &job : opens) {
      nf_result r{};
      r.kind = job.req.kind;
      r.episode = job.req.episode;
      r.submit_ms = job.submit_ms;
      r.start_ms = now_ms();
      nf_scene sc = job.req.scene;
      sc.spheres = job.spheres.empty() ? nullptr : job.spheres.data();
      sc.shapes = job.shapes.empty() ? nullptr : job.shapes.data();
      int64_t id = 0;
      r.status = nf_episode_create(slot.ctx, &job.req.grid, &sc, &id);
      size_t bytes = 0;
      if (r.status == NF_OK) nf_episode_bytes(slot.ctx, id, &bytes);
      nf_synchronize(slot.ctx);
      r.end_ms = now_ms();
      r.episode_bytes = bytes;
      std::lock_guard<std::mutex> lk(mu);
      complete(slot, job, r, id, r.status == NF_OK, bytes);
    }
    {
      std::lock_guard<std::mutex> lk(mu);
      for (const Job &job : group) {
        auto it = eps.find(job.req.episode);
        ids.push_back(it != eps.end() ? it->second.id : 0);
        created.push_back(it != eps.end() && it->second.created);
        failed.push_back(it != eps.end() && it->second.failed);
      }
    }
    const int n = (int)group.size();
    std::vector<nf_result> res(n);
    for (int i = 0; i < n; ++i) {
      res[i].kind = group[i].req.kind;
      res[i].episode = group[i].req.episode;
      res[i].submit_ms = group[i].submit_ms;
      res[i].start_ms = now_ms();
    }
    if (n > 1) {
      // one batch: the members' forward frames with every projection solved
      // for all of them at once, then each STEP_ADJOINT member's backward.
      // Members whose episode failed to open are left out.
      std::vector<int> run;
      std::vector<int64_t> rid;
      for (int i = 0; i < n; ++i)
        if (created[i] && !failed[i]) {
          run.push_back(i);
          rid.push_back(ids[i]);
        }
      const int m = (int)run.size();
      std::vector<nf_step_stats> st(n), mst(std::max(m, 1));
      std::vector<int> stat(n, NF_E_STATE), mstat(std::max(m, 1), NF_E_STATE);
      int rc = m > 0 ? nf_step_batch(slot.ctx, rid.data(), m, group[0].req.frames, mst.data(),
                                     mstat.data())
                     : NF_OK;
      if (rc == NF_E_INVALID)  // not batchable after all: one at a time
        for (int k = 0; k < m; ++k) {
          mstat[k] = nf_step(slot.ctx, rid[k], group[run[k]].req.frames, &mst[k]);
          rc = NF_OK;
        }
      for (int k = 0; k < m; ++k) {
        stat[run[k]] = rc == NF_E_CUDA || rc == NF_E_OOM ? rc : mstat[k];
        st[run[k]] = mst[k];
      }
      for (int i = 0; i < n; ++i) {
        res[i].status = stat[i];
        res[i].fwd = st[i];
        if (group[i].req.kind == NF_REQ_STEP_ADJOINT &&
            (res[i].status == NF_OK || res[i].status == NF_E_NOT_CONVERGED)) {
          auto e = slot.ctx->eps.find(ids[i]);
          const int rb = e == slot.ctx->eps.end()
                             ? NF_E_STATE
                             : e->second->loss_backward(group[i].req.loss_kind, &res[i].loss,
                                                        res[i].g_theta, &res[i].bwd);
          if (rb != NF_OK && res[i].status == NF_OK) res[i].status = rb;
        }
      }
    } else {
      Job &job = group[0];
      int64_t &id = ids[0];
      nf_result &r = res[0];
      if (job.req.kind == NF_REQ_OPEN) {
        nf_scene sc = job.req.scene;
        sc.spheres = job.spheres.empty() ? nullptr : job.spheres.data();
        sc.shapes = job.shapes.empty() ? nullptr : job.shapes.data();
        r.status = nf_episode_create(slot.ctx, &job.req.grid, &sc, &id);
        created[0] = r.status == NF_OK;
      } else if (failed[0] || !created[0]) {
        r.status = NF_E_STATE;
      } else if (job.req.kind == NF_REQ_STEP || job.req.kind == NF_REQ_STEP_ADJOINT) {
        r.status = nf_step(slot.ctx, id, job.req.frames, &r.fwd);
        if (job.req.kind == NF_REQ_STEP_ADJOINT &&
            (r.status == NF_OK || r.status == NF_E_NOT_CONVERGED)) {
          auto e = slot.ctx->eps.find(id);
          const int rc = e == slot.ctx->eps.end()
                             ? NF_E_STATE
                             : e->second->loss_backward(job.req.loss_kind, &r.loss, r.g_theta,
                                                        &r.bwd);
          if (rc != NF_OK && r.status == NF_OK) r.status = rc;
        }
      } else if (job.req.kind == NF_REQ_CLOSE) {
        r.status = nf_episode_destroy(slot.ctx, id);
      } else {
        r.status = NF_E_INVALID;
      }
    }
    std::vector<size_t> bytes(n, 0);
    for (int i = 0; i < n; ++i)
      if (group[i].req.kind != NF_REQ_CLOSE && created[i])
        nf_episode_bytes(slot.ctx, ids[i], &bytes[i]);
    nf_synchronize(slot.ctx);
    const double end = now_ms();
    {
      std::lock_guard<std::mutex> lk(mu);
      if (n > 1) {
        batches += 1;
        batched_requests += n;
      }
      for (int i = 0; i < n; ++i) {
        res[i].end_ms = end;
        res[i].episode_bytes = bytes[i];
        complete(slot, group[i], res[i], ids[i], created[i] != 0, bytes[i]);
      }
    }
  }
}

extern "C" int nf_server_create(const nf_config *cfg, int slots, size_t hbm_budget,
                                nf_server **out) {
  if (!cfg || !out || slots < 1 || slots > 64) {
    nf::set_error("nf_server_create: need a config, an output and 1..64 slots");
    return NF_E_INVALID;
  }
  *out = nullptr;
  auto srv = std::make_unique<nf_server>();
  srv->cfg = *cfg;
  srv->device = cfg->device;
  srv->budget = hbm_budget;
  for (int s = 0; s < slots; ++s) {
    nf_config c = *cfg;
    c.stream = nullptr;  // every slot runs on a stream of its own
    auto slot = std::make_unique<Slot>();
    const int rc = nf_create(&slot->ctx, &c);
    if (rc != NF_OK) {
      for (auto &p : srv->slots) nf_destroy(p->ctx);
      return rc;
    }
    srv->slots.push_back(std::move(slot));
  }
  for (int s = 0; s < slots; ++s)
    srv->slots[s]->worker = std::thread(&nf_server::work, srv.get(), s);
  *out = srv.release();
  return NF_OK;
}

extern "C" int nf_server_submit(nf_server *srv, const nf_request *req, int64_t *ticket) {
  if (!srv || !req || !ticket) {
    nf::set_error("nf_server_submit: null argument");
    return NF_E_INVALID;
  }
  Job job;
  job.req = *req;
  if (req->kind == NF_REQ_OPEN && req->scene.kind == NF_SCENE_SPHERES &&
      req->scene.nspheres > 0) {
    if (!req->scene.spheres) {
      nf::set_error("nf_server_submit: spheres scene without a sphere list");
      return NF_E_INVALID;
    }
    job.spheres.assign(req->scene.spheres, req->scene.spheres + 4 * req->scene.nspheres);
  }
  job.req.scene.spheres = nullptr;
  if (req->kind == NF_REQ_OPEN && req->scene.kind == NF_SCENE_EXTRUDED &&
      req->scene.nshape_values > 0) {
    if (!req->scene.shapes) {
      nf::set_error("nf_server_submit: extruded scene without a shape table");
      return NF_E_INVALID;
    }
    job.shapes.assign(req->scene.shapes, req->scene.shapes + req->scene.nshape_values);
  }
  job.req.scene.shapes = nullptr;
  std::lock_guard<std::mutex> lk(srv->mu);
  if (srv->stop) return NF_E_STATE;
  job.ticket = srv->next_ticket++;
  job.submit_ms = srv->now_ms();
  *ticket = job.ticket;
  srv->submitted += 1;
  srv->in_flight.insert(job.ticket);
  const int64_t key = req->episode;
  auto it = srv->eps.find(key);
  if (req->kind == NF_REQ_OPEN) {
    if (it != srv->eps.end()) {
      srv->finish(job.ticket, srv->immediate(job, NF_E_INVALID));
      return NF_OK;
    }
    EpisodeRec rec;
    rec.estimate = srv->estimate(req->grid);
    rec.nx = req->grid.nx;
    rec.ny = req->grid.ny;
    rec.nz = req->grid.nz;
    if (srv->budget && rec.estimate > srv->budget) {
      srv->finish(job.ticket, srv->immediate(job, NF_E_OOM));
      return NF_OK;
    }
    EpisodeRec &r = srv->eps.emplace(key, std::move(rec)).first->second;
    r.waiting.push_back(std::move(job));
    if (srv->open_wait.empty() && srv->fits(r.estimate))
      srv->admit(key, r);
    else
      srv->open_wait.push_back(key);
    return NF_OK;
  }
  if (req->kind == NF_REQ_CANCEL) {
    if (it == srv->eps.end()) {
      srv->finish(job.ticket, srv->immediate(job, NF_E_INVALID));
      return NF_OK;
    }
    EpisodeRec &rec = it->second;
    // the episode's requests that have not started complete as cancelled
    bool open_dropped = false;
    auto drop = [&](std::deque<Job> &q, Slot *slot) {
      for (auto j = q.begin(); j != q.end();) {
        if (j->req.episode != key) {
          ++j;
          continue;
        }
        if (j->req.kind == NF_REQ_OPEN) open_dropped = true;
        srv->finish(j->ticket, srv->immediate(*j, NF_E_CANCELED));
        if (slot) slot->pending -= 1;
        j = q.erase(j);
      }
    };
    if (rec.slot < 0) {  // not admitted: nothing reserved, nothing on a slot
      drop(rec.waiting, nullptr);
      srv->eps.erase(it);  // (its key leaves the admission queue)
      srv->admit_waiting();
      srv->finish(job.ticket, srv->immediate(job, NF_OK));
      return NF_OK;
    }
    Slot *sl = srv->slots[rec.slot].get();
    drop(sl->queue, sl);
    if (open_dropped) {  // never created: its reservation returns
      srv->reserved -= std::min(srv->reserved, rec.reserved);
      srv->eps.erase(it);
      srv->admit_waiting();
      srv->finish(job.ticket, srv->immediate(job, NF_OK));
      return NF_OK;
    }
    // created (or being created): it closes after its running request
    job.req.kind = NF_REQ_CLOSE;
    srv->enqueue(rec.slot, std::move(job));
    return NF_OK;
  }
  if (req->kind != NF_REQ_STEP && req->kind != NF_REQ_STEP_ADJOINT &&
      req->kind != NF_REQ_CLOSE) {
    srv->finish(job.ticket, srv->immediate(job, NF_E_INVALID));
    return NF_OK;
  }
  if (it == srv->eps.end()) {
    srv->finish(job.ticket, srv->immediate(job, NF_E_INVALID));
    return NF_OK;
  }
  if (it->second.slot < 0)
    it->second.waiting.push_back(std::move(job));
  else
    srv->enqueue(it->second.slot, std::move(job));
  return NF_OK;
}

static bool wait_for(nf_server *srv, std::unique_lock<std::mutex> &lk, int wait_ms,
                     const std::function<bool()> &ready) {
  if (wait_ms < 0) {
    srv->done_cv.wait(lk, ready);
    return true;
  }
  return srv->done_cv.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
}

extern "C" int nf_server_poll(nf_server *srv, int64_t ticket, int wait_ms, nf_result *out) {
  if (!srv || !out) {
    nf::set_error("nf_server_poll: null argument");
    return NF_E_INVALID;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  if (!srv->done.count(ticket) && !srv->in_flight.count(ticket)) {
    nf::set_error("nf_server_poll: unknown or already collected ticket");
    return NF_E_INVALID;
  }
  if (!wait_for(srv, lk, wait_ms, [&] { return srv->done.count(ticket) > 0; }))
    return NF_E_TIMEOUT;
  *out = srv->done[ticket];
  srv->done.erase(ticket);
  return NF_OK;
}

extern "C" int nf_server_drain(nf_server *srv, int wait_ms) {
  if (!srv) return NF_E_INVALID;
  std::unique_lock<std::mutex> lk(srv->mu);
  return wait_for(srv, lk, wait_ms, [&] { return srv->completed == srv->submitted; })
             ? NF_OK
             : NF_E_TIMEOUT;
}

extern "C" int nf_server_set_batching(nf_server *srv, int max_members, int64_t max_cells) {
  if (!srv || max_members < 1 || max_members > 64 || max_cells < 0) return NF_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  srv->batch_max = max_members;
  srv->batch_cells = max_cells;
  return NF_OK;
}

extern "C" int nf_server_stats_get(nf_server *srv, nf_server_stats *out) {
  if (!srv || !out) return NF_E_INVALID;
  std::lock_guard<std::mutex> lk(srv->mu);
  out->batches = srv->batches;
  out->batched_requests = srv->batched_requests;
  out->submitted = srv->submitted;
  out->completed = srv->completed;
  out->open_waiting = (int64_t)srv->open_wait.size();
  out->episodes = (int64_t)srv->eps.size();
  out->bytes_reserved = srv->reserved;
  out->bytes_peak = srv->peak;
  out->budget = srv->budget;
  out->slots = (int)srv->slots.size();
  return NF_OK;
}

extern "C" int nf_server_destroy(nf_server *srv) {
  if (!srv) return NF_E_INVALID;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
    for (auto &s : srv->slots) s->cv.notify_all();
  }
  for (auto &s : srv->slots)
    if (s->worker.joinable()) s->worker.join();
  for (auto &s : srv->slots) nf_destroy(s->ctx);
  delete srv;
  return NF_OK;
}
