// serve.cu -- serving loop (include/graphic_serve.h): admission by device
// memory, resident cubes, continuous cross-request batching of the reduction
// stages (Sect. 3), per-request latency.
//
// Threads.  Clients call submit / wait; one scheduler thread makes every
// CUDA call.  Host callbacks enqueued with cudaLaunchHostFunc mark
// iterations and requests finished on the device; they touch only atomics
// and the condition variable.  The mutex is never held across a CUDA call.
//
// Streams.  s_in carries the copies in (plan, cube) and each request's
// shift, enqueued piece by piece right behind the piece's copy (so a request
// is shifted while the rest of its cube is still landing, as in a lone
// reduction of host buffers); s_out the copies out (result, status); s_comp
// the other kernels: a copy-out that waits for a collapse never holds up a
// later request's copy-in.  A request joins an iteration's median stage once
// its copy-in and shift have completed (so the kernels never wait on a copy
// while other work is ready), and its copy-out waits on the event recorded
// after its collapse.
//
// Iterations.  Each issued iteration takes every resident request one stage
// on: ADMITTED (copied in and shifted) -> median PSF subtraction,
// SUBTRACTED -> derotation, ROTATED -> collapse + copy-out.  The derotation
// items of one iteration form one uneven batch on one of two library
// contexts (alternating, so that a context's host plan buffer is not
// rewritten while the other iteration's copy of it may still be pending: at
// most two iterations are in flight).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/graphic.h"
#include "../../include/graphic_serve.h"
#include "graphic_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// First-fit sub-allocator over one block; offsets and sizes in 256-byte units.
class Arena {
 public:
  static constexpr size_t kAlign = 256;
  static constexpr size_t kNone = ~size_t(0);
  void reset(size_t cap) {
    free_.clear();
    cap_ = cap & ~(kAlign - 1);
    if (cap_) free_[0] = cap_;
    used_ = peak_ = 0;
  }
  static size_t round(size_t b) { return std::max(kAlign, (b + kAlign - 1) & ~(kAlign - 1)); }
  size_t alloc(size_t bytes) {
    bytes = round(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < bytes) continue;
      const size_t off = it->first, rest = it->second - bytes;
      free_.erase(it);
      if (rest) free_[off + bytes] = rest;
      used_ += bytes;
      peak_ = std::max(peak_, used_);
      return off;
    }
    return kNone;
  }
  void release(size_t off, size_t bytes) {
    bytes = round(bytes);
    used_ -= bytes;
    auto it = free_.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t cap() const { return cap_; }
  size_t peak() const { return peak_; }

 private:
  std::map<size_t, size_t> free_;
  size_t cap_ = 0, used_ = 0, peak_ = 0;
};

enum Stage { QUEUED, ADMITTED, SHIFTED, SUBTRACTED, ROTATED, FINISHING, DONE };

struct Req {
  struct graphic_server *srv = nullptr;
  int64_t id = 0;
  const float *host_in = nullptr;
  float *host_out = nullptr;
  int64_t T = 0;
  int32_t n = 0;
  std::vector<double> dx, dy, theta;   // theta = -parang (derotation)
  graphic::AdiPlanHost ap;
  int n_ann = 0;
  // device arena: cube, result, plan
  // (plan_dev_bytes: the plan's device region, the staged tables)
  size_t cube_bytes = 0, out_bytes = 0, plan_bytes = 0, plan_dev_bytes = 0;
  size_t off_cube = Arena::kNone, off_out = Arena::kNone, off_plan = Arena::kNone;
  size_t o_perm = 0, o_lr = 0, o_e2 = 0, o_band = 0, o_evq = 0, o_groups = 0;   // within the plan
  size_t o_dx = 0, o_dy = 0;   // staged shifts
  size_t o_ptab = 0;           // device only (after the staged part): the shift passes' parameter tables
  // pinned staging: plan copy-in, result copy-out
  size_t stage_bytes = 0, off_stage = Arena::kNone;
  int slot = -1;   // per-request device status word
  Stage stage = QUEUED;            // scheduler
  bool published = false;          // under the server mutex: result final
  std::atomic<bool> gpu_done{false};
  int status = GRAPHIC_OK;
  std::string err;
  double t_submit = 0, t_admit = -1, t_done = -1;
  cudaEvent_t ev_in = nullptr, ev_col = nullptr;
};

struct Iter {
  std::vector<Req *> batch;   // requests in this iteration's batch
  const int *h_status = nullptr;
};

}  // namespace

struct graphic_server {
  int device = 0;
  int max_active = 16;
  int mode = GRAPHIC_BATCH_GROUPED;
  Clock::time_point t0;
  char *d_arena = nullptr;
  Arena arena;
  char *d_band = nullptr;   // median PSF band path tables (kBandScratchMax), shared by the requests
  char *h_stage = nullptr;
  Arena stage;
  int *d_status = nullptr;     // [max_active]
  int *h_status = nullptr;     // [max_active] pinned
  std::vector<int> free_slots;
  graphic_ctx *ctx[2] = {nullptr, nullptr};
  cudaStream_t s_comp = nullptr, s_in = nullptr, s_out = nullptr;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_sched, cv_done;
  std::deque<Req *> queue;                     // under mu
  std::unordered_map<int64_t, Req *> reqs;     // under mu
  int64_t next_id = 1;                         // under mu
  bool stop = false;                           // under mu
  std::atomic<int64_t> iters_done{0};
  int64_t iters_issued = 0;                    // scheduler
  std::deque<Iter> inflight;                   // scheduler
  std::vector<Req *> active;                   // scheduler
  graphic_server_stats st{};                   // under mu
  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

void CUDART_CB on_iter_done(void *p) {
  graphic_server *s = static_cast<graphic_server *>(p);
  s->iters_done.fetch_add(1);
  std::lock_guard<std::mutex> lk(s->mu);
  s->cv_sched.notify_all();
}

void CUDART_CB on_wake(void *p) {
  graphic_server *s = static_cast<graphic_server *>(p);
  std::lock_guard<std::mutex> lk(s->mu);
  s->cv_sched.notify_all();
}

void CUDART_CB on_req_done(void *p) {
  Req *r = static_cast<Req *>(p);
  // once gpu_done is set the scheduler may retire r and a waiter free it:
  // read the server first and set the flag under the server mutex, which
  // retiring needs, so that r is not touched after it may be gone
  graphic_server *srv = r->srv;
  std::lock_guard<std::mutex> lk(srv->mu);
  r->gpu_done.store(true);
  srv->cv_sched.notify_all();
}

int status_code(int bits) {
  if (bits & graphic::STATUS_NONFINITE) return GRAPHIC_ERR_NONFINITE;
  if (bits & graphic::STATUS_TIMEOUT) return GRAPHIC_ERR_TIMEOUT;
  if (bits & graphic::STATUS_INTERNAL) return GRAPHIC_ERR_INTERNAL;
  return GRAPHIC_OK;
}

void fail_req(Req *r, int code, const std::string &msg) {
  if (r->status == GRAPHIC_OK) {
    r->status = code;
    r->err = msg;
  }
}

// Free a finished request's resources and publish it (a waiter may free r
// right after; iterations still in flight stop referring to it first).
void retire(graphic_server *s, Req *r) {
  for (Iter &it : s->inflight) it.batch.erase(std::remove(it.batch.begin(), it.batch.end(), r), it.batch.end());
  if (r->off_cube != Arena::kNone) s->arena.release(r->off_cube, r->cube_bytes);
  if (r->off_out != Arena::kNone) s->arena.release(r->off_out, r->out_bytes);
  if (r->off_plan != Arena::kNone) s->arena.release(r->off_plan, r->plan_dev_bytes);
  if (r->off_stage != Arena::kNone) s->stage.release(r->off_stage, r->stage_bytes);
  r->off_cube = r->off_out = r->off_plan = r->off_stage = Arena::kNone;
  if (r->slot >= 0) s->free_slots.push_back(r->slot);
  r->slot = -1;
  if (r->ev_in) cudaEventDestroy(r->ev_in);
  if (r->ev_col) cudaEventDestroy(r->ev_col);
  r->ev_in = r->ev_col = nullptr;
  r->t_done = s->now();
  std::lock_guard<std::mutex> lk(s->mu);
  r->stage = DONE;
  r->published = true;
  s->st.completed++;
  if (r->status != GRAPHIC_OK) s->st.failed++;
  s->st.device_bytes_peak = (int64_t)s->arena.peak();
  s->cv_done.notify_all();
}

// Requests whose copy-out finished: result to host_out, resources back.
void collect(graphic_server *s) {
  for (size_t i = 0; i < s->active.size();) {
    Req *r = s->active[i];
    if (r->stage == FINISHING && r->gpu_done.load()) {
      if (r->status == GRAPHIC_OK) {
        const int bits = s->h_status[r->slot];
        if (bits) fail_req(r, status_code(bits), "device status of this request");
      }
      if (r->status == GRAPHIC_OK)
        memcpy(r->host_out, s->h_stage + r->off_stage + r->plan_bytes, r->out_bytes);
      s->active.erase(s->active.begin() + i);
      retire(s, r);
    } else {
      i++;
    }
  }
}

// Iterations the device finished, oldest first: the batch's own status word.
// Its non-finite bit is not attributed to the batch's requests: a non-finite
// input reaches the median stage, which flags it in that request's own word.
void reap_iterations(graphic_server *s) {
  const int64_t done = s->iters_done.load();
  while (!s->inflight.empty() && s->iters_issued - (int64_t)s->inflight.size() < done) {
    Iter &it = s->inflight.front();
    const int bits = (it.h_status ? *it.h_status : graphic::STATUS_INTERNAL) & ~graphic::STATUS_NONFINITE;
    if (bits)
      for (Req *r : it.batch) fail_req(r, status_code(bits), "device status of a batch this request was in");
    s->inflight.pop_front();
  }
}

// Copy-in of an admitted request: plan (via pinned staging), then the cube.
int start_copy_in(graphic_server *s, Req *r) {
  char *hp = s->h_stage + r->off_stage;
  const int64_t T = r->T;
  memcpy(hp + r->o_perm, r->ap.perm.data(), T * sizeof(int));
  memcpy(hp + r->o_lr, r->ap.lr.data(), r->ap.lr.size() * sizeof(int));
  memcpy(hp + r->o_e2, r->ap.edge2.data(), r->ap.edge2.size() * sizeof(double));
  memcpy(hp + r->o_band, r->ap.band.data(), r->ap.band.size() * sizeof(int));
  memcpy(hp + r->o_evq, r->ap.evq.data(), r->ap.evq.size() * sizeof(uint32_t));
  memcpy(hp + r->o_groups, r->ap.groups.data(), r->ap.groups.size() * sizeof(int));
  memcpy(hp + r->o_dx, r->dx.data(), T * sizeof(double));
  memcpy(hp + r->o_dy, r->dy.data(), T * sizeof(double));
  char *plan = s->d_arena + r->off_plan;
  float *cube = reinterpret_cast<float *>(s->d_arena + r->off_cube);
  cudaError_t e = cudaMemcpyAsync(plan, hp, r->plan_bytes, cudaMemcpyHostToDevice, s->s_in);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_status + r->slot, 0, sizeof(int), s->s_in);
  // the shift (Sect. 3.3.1) is done on the copy stream, piece by piece as the
  // cube lands, so that it overlaps the copy as in a lone reduction
  graphic::LineArgs a{};
  a.p0 = reinterpret_cast<const double *>(plan + r->o_dx);
  a.p1 = reinterpret_cast<const double *>(plan + r->o_dy);
  a.n = r->n;
  a.status = s->d_status + r->slot;
  const size_t pb = graphic::line_params_bytes(graphic::SHIFT_X, r->n, T);
  if (e == cudaSuccess) e = graphic::launch_line_params(graphic::SHIFT_X, a, T, plan + r->o_ptab, s->s_in);
  if (e == cudaSuccess) e = graphic::launch_line_params(graphic::SHIFT_Y, a, T, plan + r->o_ptab + pb, s->s_in);
  const int64_t NN = (int64_t)r->n * r->n;
  const int64_t ch = std::max<int64_t>(1, std::min<int64_t>(T, ((int64_t)256 << 20) / (NN * (int64_t)sizeof(float))));
  for (int64_t f0 = 0; f0 < T && e == cudaSuccess; f0 += ch) {
    const int64_t nf = std::min<int64_t>(ch, T - f0);
    e = cudaMemcpyAsync(cube + f0 * NN, r->host_in + f0 * NN, nf * NN * sizeof(float), cudaMemcpyHostToDevice, s->s_in);
    graphic::LineArgs b = a;
    b.in = cube + f0 * NN;
    b.out = cube + f0 * NN;
    b.in_fstride = b.out_fstride = NN;
    b.p0 = a.p0 + f0;
    b.p1 = a.p1 + f0;
    b.lp_lines = 1;
    b.lp_tab = plan + r->o_ptab + (size_t)f0 * (pb / T);
    if (e == cudaSuccess) e = graphic::launch_line_pass(graphic::SHIFT_X, b, nf, s->s_in);
    b.lp_tab = plan + r->o_ptab + pb + (size_t)f0 * (pb / T);
    if (e == cudaSuccess) e = graphic::launch_line_pass(graphic::SHIFT_Y, b, nf, s->s_in);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&r->ev_col, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(r->ev_in, s->s_in);
  if (e == cudaSuccess) e = cudaLaunchHostFunc(s->s_in, on_wake, s);   // its median may start
  return e == cudaSuccess ? GRAPHIC_OK : GRAPHIC_ERR_CUDA;
}

// Admit queued requests first come first served while they fit.
void admit(graphic_server *s) {
  for (;;) {
    Req *r;
    {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->queue.empty()) return;
      r = s->queue.front();
    }
    const size_t need = Arena::round(r->cube_bytes) + Arena::round(r->out_bytes) + Arena::round(r->plan_dev_bytes);
    if (need > s->arena.cap() || Arena::round(r->stage_bytes) > s->stage.cap()) {
      {
        std::lock_guard<std::mutex> lk(s->mu);
        s->queue.pop_front();
      }
      fail_req(r, GRAPHIC_ERR_OOM, "request larger than the server's device budget or staging");
      retire(s, r);
      continue;
    }
    if (s->free_slots.empty()) return;
    r->off_cube = s->arena.alloc(r->cube_bytes);
    if (r->off_cube != Arena::kNone) r->off_out = s->arena.alloc(r->out_bytes);
    if (r->off_out != Arena::kNone) r->off_plan = s->arena.alloc(r->plan_dev_bytes);
    if (r->off_plan != Arena::kNone) r->off_stage = s->stage.alloc(r->stage_bytes);
    if (r->off_stage == Arena::kNone) {
      // does not fit yet: give back what was taken, wait for completions
      if (r->off_cube != Arena::kNone) s->arena.release(r->off_cube, r->cube_bytes);
      if (r->off_out != Arena::kNone) s->arena.release(r->off_out, r->out_bytes);
      if (r->off_plan != Arena::kNone) s->arena.release(r->off_plan, r->plan_dev_bytes);
      r->off_cube = r->off_out = r->off_plan = Arena::kNone;
      return;
    }
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->queue.pop_front();
      s->st.admitted++;
    }
    r->t_admit = s->now();
    if (start_copy_in(s, r) != GRAPHIC_OK) {
      fail_req(r, GRAPHIC_ERR_CUDA, "copy-in");
      r->stage = FINISHING;
      s->active.push_back(r);
      cudaLaunchHostFunc(s->s_in, on_req_done, r);
      continue;
    }
    r->stage = ADMITTED;
    s->active.push_back(r);
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.max_resident = std::max<int64_t>(s->st.max_resident, (int64_t)s->active.size());
  }
}

bool copied_in(const Req *r) { return cudaEventQuery(r->ev_in) == cudaSuccess; }

// Work an iteration could do now: a request past its shift, or one whose
// copy-in and shift have completed; with nothing else pending, one still
// copying in (the iteration then waits for it on the device).
bool has_stage_work(const graphic_server *s) {
  bool admitted = false;
  for (const Req *r : s->active) {
    if (r->stage > ADMITTED && r->stage <= ROTATED) return true;
    if (r->stage == ADMITTED) {
      if (copied_in(r)) return true;
      admitted = true;
    }
  }
  return admitted && s->inflight.empty();
}

// Enqueue one iteration: every resident request one stage on.
void issue_iteration(graphic_server *s) {
  graphic_ctx *ctx = s->ctx[s->iters_issued & 1];
  Iter it;
  std::vector<graphic_batch_item> items;
  std::vector<Req *> adi, rot, col;
  bool others = false;
  for (Req *r : s->active) others |= (r->stage > ADMITTED && r->stage <= ROTATED) || (r->stage == ADMITTED && copied_in(r));
  for (Req *r : s->active) {
    switch (r->stage) {
      case ADMITTED:   // copied in and shifted on the copy stream (or, with nothing else to do, soon)
        if (!others || copied_in(r)) {
          cudaStreamWaitEvent(s->s_comp, r->ev_in, 0);
          adi.push_back(r);
        }
        break;
      case SHIFTED: adi.push_back(r); break;
      case SUBTRACTED: rot.push_back(r); break;
      case ROTATED: col.push_back(r); break;
      default: break;
    }
  }
  for (Req *r : rot) {
    float *cube = reinterpret_cast<float *>(s->d_arena + r->off_cube);
    graphic_batch_item b{};
    b.in = cube;
    b.out = cube;
    b.n_frames = r->T;
    b.n = r->n;
    b.passes = GRAPHIC_PASS_ROTATE;
    b.theta_deg = r->theta.data();
    items.push_back(b);
  }
  if (!items.empty()) {
    int rc = graphic::ctx_batch_async(ctx, items.data(), (int32_t)items.size(), s->mode);
    it.h_status = graphic::ctx_status_async(ctx);
    if (rc != GRAPHIC_OK)
      for (Req *r : rot) fail_req(r, rc, graphic_last_error());
    it.batch = rot;
    std::lock_guard<std::mutex> lk(s->mu);
    s->st.batch_launches++;
    s->st.batch_items += (int64_t)items.size();
    s->st.max_batch_items = std::max<int64_t>(s->st.max_batch_items, (int64_t)items.size());
  } else {
    static const int zero = 0;
    it.h_status = &zero;
  }
  for (Req *r : adi) {
    float *cube = reinterpret_cast<float *>(s->d_arena + r->off_cube);
    const char *plan = s->d_arena + r->off_plan;
    graphic::AdiArgs a{};
    a.in = cube;
    a.out = cube;
    a.perm = reinterpret_cast<const int *>(plan + r->o_perm);
    a.lr = reinterpret_cast<const int *>(plan + r->o_lr);
    a.edge2 = reinterpret_cast<const double *>(plan + r->o_e2);
    a.band = reinterpret_cast<const int *>(plan + r->o_band);
    a.wmax = r->ap.wmax;
    a.evq = reinterpret_cast<const uint32_t *>(plan + r->o_evq);
    a.groups = reinterpret_cast<const int *>(plan + r->o_groups);
    for (int k = 0; k < 8; k++) a.class_off[k] = k < (int)r->ap.class_off.size() ? r->ap.class_off[k] : 0;
    a.gen_list = r->ap.gen_off >= 0 ? 1 : 0;
    a.gen_off = r->ap.gen_off;
    a.gen_n = r->ap.gen_n;
    a.band_scratch = s->d_band;   // shared: the median launches run one after the other on s_comp
    a.band_scratch_cap = graphic::kBandScratchMax;
    a.status = s->d_status + r->slot;
    a.T = (int)r->T;
    a.n = r->n;
    a.in_fs = a.out_fs = (long long)r->n * r->n;
    a.perm_id = 1;
    for (int64_t t = 0; t < r->T && a.perm_id; t++) a.perm_id = r->ap.perm[t] == (int)t;
    a.n_ann = r->n_ann;
    if (graphic::launch_adi_median(a, s->s_comp) != cudaSuccess) fail_req(r, GRAPHIC_ERR_CUDA, "median PSF kernel");
  }
  for (Req *r : col) {
    graphic::CollapseArgs a{};
    a.in = reinterpret_cast<const float *>(s->d_arena + r->off_cube);
    a.out = reinterpret_cast<float *>(s->d_arena + r->off_out);
    a.status = s->d_status + r->slot;
    a.T = r->T;
    a.n = r->n;
    if (graphic::launch_collapse(a, s->s_comp) != cudaSuccess) fail_req(r, GRAPHIC_ERR_CUDA, "collapse kernel");
    cudaEventRecord(r->ev_col, s->s_comp);
    cudaStreamWaitEvent(s->s_out, r->ev_col, 0);
    cudaMemcpyAsync(s->h_stage + r->off_stage + r->plan_bytes, s->d_arena + r->off_out, r->out_bytes,
                    cudaMemcpyDeviceToHost, s->s_out);
    cudaMemcpyAsync(s->h_status + r->slot, s->d_status + r->slot, sizeof(int), cudaMemcpyDeviceToHost, s->s_out);
    if (cudaLaunchHostFunc(s->s_out, on_req_done, r) != cudaSuccess) {
      fail_req(r, GRAPHIC_ERR_CUDA, "completion callback");
      r->gpu_done.store(true);
    }
  }
  for (Req *r : adi) r->stage = SUBTRACTED;
  for (Req *r : rot) r->stage = ROTATED;
  for (Req *r : col) r->stage = FINISHING;
  s->inflight.push_back(std::move(it));
  s->iters_issued++;
  if (cudaLaunchHostFunc(s->s_comp, on_iter_done, s) != cudaSuccess) s->iters_done.fetch_add(1);
  std::lock_guard<std::mutex> lk(s->mu);
  s->st.iterations = s->iters_issued;
}

void scheduler(graphic_server *s) {
  cudaSetDevice(s->device);
  for (;;) {
    reap_iterations(s);
    collect(s);
    admit(s);
    // at most two iterations unreaped: a context's status copy is read
    // before the context is used again
    const bool can_issue = s->inflight.size() < 2 && has_stage_work(s);
    if (can_issue) {
      issue_iteration(s);
      continue;
    }
    std::unique_lock<std::mutex> lk(s->mu);
    if (s->stop && s->queue.empty() && s->active.empty() && s->inflight.empty()) break;
    // woken by a submission or a device callback; the timeout is a safety net
    s->cv_sched.wait_for(lk, std::chrono::milliseconds(2));
  }
}

int check_request(const graphic_request *r) {
  if (!r) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null request");
  if (!r->host_in || !r->host_out) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null host buffer");
  if (r->n_frames < 1) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "n_frames < 1");
  const int n = r->n;
  if (!(n == 64 || n == 128 || n == 256 || n == 512 || n == 1024))
    return graphic::set_last_error(GRAPHIC_ERR_UNSUPPORTED, "n must be one of 64, 128, 256, 512, 1024");
  int rc = graphic::validate_shift(r->dx, r->dy, r->n_frames, n);
  if (rc) return rc;
  rc = graphic::validate_adi(r->parang, r->n_frames, r->fwhm, r->n_fwhm, r->edges, r->n_edges);
  if (rc) return rc;
  for (int64_t t = 0; t < r->n_frames; t++)
    if (fabs(r->parang[t]) > 1e6) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "|angle| > 1e6 deg");
  return GRAPHIC_OK;
}

size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

}  // namespace

extern "C" {

int graphic_server_create(graphic_server **out, const graphic_server_config *cfg) {
  if (!out) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null out");
  *out = nullptr;
  graphic_server_config c{};
  if (cfg) c = *cfg;
  if (c.max_active < 0 || c.max_device_bytes < 0 || c.staging_bytes < 0)
    return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "negative server limit");
  const int mode = c.batch_mode;
  if (mode < GRAPHIC_BATCH_PER_CUBE || mode > GRAPHIC_BATCH_AUTO)
    return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "unknown batch mode");
  graphic_server *s = new graphic_server();
  s->device = c.device;
  s->max_active = c.max_active ? c.max_active : 16;
  s->mode = mode;
  s->t0 = Clock::now();
  int rc = GRAPHIC_OK;
  for (int k = 0; k < 2 && rc == GRAPHIC_OK; k++) rc = graphic_create(&s->ctx[k], c.device);
  if (rc != GRAPHIC_OK) {
    graphic_server_destroy(s);
    return rc;
  }
  cudaSetDevice(c.device);
  cudaError_t e = cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->s_out, cudaStreamNonBlocking);
  for (int k = 0; k < 2 && e == cudaSuccess; k++) {
    if (graphic_set_stream(s->ctx[k], s->s_comp) != GRAPHIC_OK) e = cudaErrorInvalidValue;
    graphic::ctx_set_graph_batches(s->ctx[k], false);   // every iteration has its own layout
  }
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    graphic_server_destroy(s);
    return graphic::set_last_error(GRAPHIC_ERR_CUDA, cudaGetErrorString(e));
  }
  // budget: the asked bytes, at most free HBM minus both contexts' workspaces and a margin
  const size_t ws = 2 * graphic::ctx_workspace_bound(s->ctx[0], mode) + ((size_t)1 << 30) + graphic::kBandScratchMax;
  size_t budget = c.max_device_bytes ? (size_t)c.max_device_bytes : ((size_t)150 << 30);
  budget = std::min(budget, free_b > ws ? free_b - ws : 0);
  budget &= ~(Arena::kAlign - 1);
  if (budget < ((size_t)1 << 20)) {
    graphic_server_destroy(s);
    return graphic::set_last_error(GRAPHIC_ERR_OOM, "no device memory left for the server's arena");
  }
  const size_t staging = c.staging_bytes ? (size_t)c.staging_bytes : ((size_t)256 << 20);
  e = cudaMalloc(&s->d_arena, budget);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_band, graphic::kBandScratchMax);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_stage, staging);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_status, sizeof(int) * s->max_active);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_status, sizeof(int) * s->max_active);
  if (e != cudaSuccess) {
    graphic_server_destroy(s);
    return graphic::set_last_error(e == cudaErrorMemoryAllocation ? GRAPHIC_ERR_OOM : GRAPHIC_ERR_CUDA,
                                   cudaGetErrorString(e));
  }
  s->arena.reset(budget);
  s->stage.reset(staging);
  for (int k = s->max_active - 1; k >= 0; k--) s->free_slots.push_back(k);
  s->st.device_bytes_cap = (int64_t)budget;
  s->th = std::thread(scheduler, s);
  *out = s;
  return GRAPHIC_OK;
}

int graphic_server_submit(graphic_server *s, const graphic_request *rq, int64_t *id) {
  if (!s || !id) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null server or id");
  int rc = check_request(rq);
  if (rc) return rc;
  Req *r = new Req();
  r->srv = s;
  r->host_in = rq->host_in;
  r->host_out = rq->host_out;
  r->T = rq->n_frames;
  r->n = rq->n;
  const int64_t T = r->T;
  r->dx.assign(rq->dx, rq->dx + T);
  r->dy.assign(rq->dy, rq->dy + T);
  r->theta.resize(T);
  for (int64_t t = 0; t < T; t++) r->theta[t] = -rq->parang[t];
  if ((rc = graphic::plan_adi(rq->parang, T, rq->fwhm, rq->n_fwhm, rq->edges, rq->n_edges, r->ap)) ||
      (rc = graphic::plan_band_path(r->ap, T, rq->n))) {
    delete r;
    return rc;
  }
  r->n_ann = rq->n_edges - 1;
  const size_t NN = (size_t)r->n * r->n;
  r->cube_bytes = (size_t)T * NN * sizeof(float);
  r->out_bytes = NN * sizeof(float);
  size_t o = 0;
  r->o_perm = o;
  o = align16(o + T * sizeof(int));
  r->o_lr = o;
  o = align16(o + r->ap.lr.size() * sizeof(int));
  r->o_e2 = o;
  o = align16(o + r->ap.edge2.size() * sizeof(double));
  r->o_band = o;
  o = align16(o + r->ap.band.size() * sizeof(int));
  r->o_evq = o;
  o = align16(o + r->ap.evq.size() * sizeof(uint32_t));
  r->o_groups = o;
  o = align16(o + r->ap.groups.size() * sizeof(int));
  r->o_dx = o;
  o = align16(o + T * sizeof(double));
  r->o_dy = o;
  o = align16(o + T * sizeof(double));
  r->plan_bytes = o;
  r->o_ptab = o;
  o = align16(o + 2 * graphic::line_params_bytes(graphic::SHIFT_X, r->n, T));
  r->plan_dev_bytes = o;
  r->stage_bytes = r->plan_bytes + r->out_bytes;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) {
    delete r;
    return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "server is stopping");
  }
  r->id = s->next_id++;
  r->t_submit = s->now();
  s->reqs[r->id] = r;
  s->queue.push_back(r);
  s->st.submitted++;
  s->cv_sched.notify_all();
  *id = r->id;
  return GRAPHIC_OK;
}

int graphic_server_wait(graphic_server *s, int64_t id, double timeout_s, graphic_request_info *info) {
  if (!s) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->reqs.find(id);
  if (it == s->reqs.end()) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "unknown request id");
  Req *r = it->second;
  auto done = [&] { return r->published; };
  if (timeout_s < 0) {
    s->cv_done.wait(lk, done);
  } else if (!s->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), done)) {
    return graphic::set_last_error(GRAPHIC_ERR_TIMEOUT, "request still running");
  }
  if (info) {
    info->status = r->status;
    info->reserved = 0;
    info->t_submit = r->t_submit;
    info->t_admit = r->t_admit;
    info->t_done = r->t_done;
  }
  const int st = r->status;
  const std::string msg = r->err;
  s->reqs.erase(it);
  lk.unlock();
  delete r;
  if (st != GRAPHIC_OK) graphic::set_last_error(st, msg.c_str());
  return GRAPHIC_OK;
}

double graphic_server_clock(graphic_server *s) { return s ? s->now() : 0.0; }

int graphic_server_stats_read(graphic_server *s, graphic_server_stats *st) {
  if (!s || !st) return graphic::set_last_error(GRAPHIC_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> lk(s->mu);
  *st = s->st;
  return GRAPHIC_OK;
}

int graphic_server_destroy(graphic_server *s) {
  if (!s) return GRAPHIC_OK;
  if (s->th.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
      s->cv_sched.notify_all();
    }
    s->th.join();
  }
  cudaSetDevice(s->device);
  if (s->s_comp) cudaStreamSynchronize(s->s_comp);
  if (s->s_in) cudaStreamSynchronize(s->s_in);
  if (s->s_out) cudaStreamSynchronize(s->s_out);
  for (auto &kv : s->reqs) delete kv.second;
  s->reqs.clear();
  for (int k = 0; k < 2; k++)
    if (s->ctx[k]) graphic_destroy(s->ctx[k]);
  cudaFree(s->d_arena);
  cudaFree(s->d_band);
  cudaFreeHost(s->h_stage);
  cudaFree(s->d_status);
  cudaFreeHost(s->h_status);
  if (s->s_comp) cudaStreamDestroy(s->s_comp);
  if (s->s_in) cudaStreamDestroy(s->s_in);
  if (s->s_out) cudaStreamDestroy(s->s_out);
  delete s;
  return GRAPHIC_OK;
}

}  // extern "C"
