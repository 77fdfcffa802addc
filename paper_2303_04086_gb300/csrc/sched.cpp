// Multi-user scheduling policy of the paper's task assigner (Sec. 6.2,
// Algorithm 1 and Eq. 13), for one GPU's request loop.
//
// Users are viewers with a target frame rate FPS_i.  Each keeps a moving
// average t_i of its frames' completion times (dispatch -> completion) and
// the time of its last completed frame; its wait time is
//   w_i = 1 / FPS_i - t_i                                       (Eq. 13)
// and its target time is last_frame_i + w_i.  A pending frame whose viewer's
// target time has passed is starved.  While any frame is starved the
// scheduler is in the starvation state: starved frames are dispatched first,
// regardless of the ray budget, and admissions from new clients (viewers not
// seen before) are denied.  Otherwise frames are dispatched in the order of
// their viewers' (frames in flight, target time), while the rays in flight
// stay within the budget -- the first frame that does not fit stops the
// dispatch round (Algorithm 1's "break").  Sharing of rays between adjacent
// views is not modelled.
//
// The scheduler is host-only and deterministic: every call takes the current
// time in nanoseconds from the caller.
#include <algorithm>
#include <cstdint>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "inolf_internal.h"

using namespace inolf;

namespace {

struct Viewer {
  double fps = 50.0;  // the paper's clients send a camera every 20 ms
  double ema_s = 0.0;
  bool have_ema = false;
  int64_t last_frame_ns = 0;
  int32_t loaded = 0;  // frames in flight
};

struct Pending {
  uint64_t id;
  uint32_t viewer;
  int64_t rays;
  int64_t admit_ns;
};

struct InFlight {
  uint32_t viewer;
  int64_t rays;
  int64_t start_ns;
};

}  // namespace

struct inolf_sched {
  std::mutex mu;
  int64_t max_rays = 0;  // 0: no budget
  double ema_alpha = 0.25;
  std::map<uint32_t, Viewer> viewers;
  std::vector<Pending> pending;
  std::map<uint64_t, InFlight> inflight;
  int64_t rays_in_flight = 0;
  bool starving = false;
  int64_t denied = 0;

  int64_t target_ns(const Viewer& v) const {
    const double w = std::max(0.0, 1.0 / v.fps - (v.have_ema ? v.ema_s : 0.0));
    return v.last_frame_ns + (int64_t)(w * 1e9);
  }

  bool any_starved(int64_t now) const {
    for (const Pending& p : pending)
      if (target_ns(viewers.at(p.viewer)) <= now) return true;
    return false;
  }
};

extern "C" inolf_status inolf_sched_create(int64_t max_rays_in_flight, inolf_sched** out) {
  clear_error();
  if (!out || max_rays_in_flight < 0) return fail(INOLF_E_INVALID, "inolf_sched_create: bad argument");
  inolf_sched* s = new (std::nothrow) inolf_sched();
  if (!s) return fail(INOLF_E_OOM, "inolf_sched_create: oom");
  s->max_rays = max_rays_in_flight;
  *out = s;
  return INOLF_OK;
}

extern "C" void inolf_sched_destroy(inolf_sched* s) { delete s; }

extern "C" inolf_status inolf_sched_set_viewer(inolf_sched* s, uint32_t viewer, double target_fps, int64_t now_ns) {
  clear_error();
  if (!s || !(target_fps > 0)) return fail(INOLF_E_INVALID, "inolf_sched_set_viewer: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->viewers.find(viewer);
  if (it == s->viewers.end()) {
    Viewer v;
    v.last_frame_ns = now_ns;
    it = s->viewers.emplace(viewer, v).first;
  }
  it->second.fps = target_fps;
  return INOLF_OK;
}

extern "C" inolf_status inolf_sched_admit(inolf_sched* s, uint32_t viewer, uint64_t id, int64_t rays, int64_t now_ns) {
  clear_error();
  if (!s || rays < 0) return fail(INOLF_E_INVALID, "inolf_sched_admit: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  s->starving = s->any_starved(now_ns);
  auto it = s->viewers.find(viewer);
  if (it == s->viewers.end()) {
    if (s->starving) {
      ++s->denied;
      return fail(INOLF_E_BUDGET, "inolf_sched_admit: starvation state, new clients are denied");
    }
    Viewer v;
    v.last_frame_ns = now_ns;
    s->viewers.emplace(viewer, v);
  }
  s->pending.push_back({id, viewer, rays, now_ns});
  return INOLF_OK;
}

extern "C" inolf_status inolf_sched_next(inolf_sched* s, int64_t now_ns, uint64_t* id) {
  clear_error();
  if (!s || !id) return fail(INOLF_E_INVALID, "inolf_sched_next: bad argument");
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->pending.empty()) {
    s->starving = false;
    return INOLF_PENDING;
  }
  // 1) starved frames first (earliest target time, then admission order)
  int best = -1;
  int64_t best_t = 0;
  for (int k = 0; k < (int)s->pending.size(); ++k) {
    const int64_t t = s->target_ns(s->viewers.at(s->pending[k].viewer));
    if (t > now_ns) continue;
    if (best < 0 || t < best_t || (t == best_t && s->pending[k].admit_ns < s->pending[best].admit_ns)) {
      best = k;
      best_t = t;
    }
  }
  s->starving = best >= 0;
  if (best < 0) {
    // 2) otherwise by (frames in flight, target time, admission order) within the ray budget
    auto key = [&](const Pending& p) {
      const Viewer& v = s->viewers.at(p.viewer);
      return std::make_tuple(v.loaded, s->target_ns(v), p.admit_ns, p.id);
    };
    best = 0;
    for (int k = 1; k < (int)s->pending.size(); ++k)
      if (key(s->pending[k]) < key(s->pending[best])) best = k;
    if (s->max_rays > 0 && s->rays_in_flight > 0 && s->rays_in_flight + s->pending[best].rays > s->max_rays)
      return INOLF_PENDING;  // the farm is full
  }
  const Pending p = s->pending[best];
  s->pending.erase(s->pending.begin() + best);
  s->inflight[p.id] = {p.viewer, p.rays, now_ns};
  s->rays_in_flight += p.rays;
  s->viewers[p.viewer].loaded += 1;
  *id = p.id;
  return INOLF_OK;
}

extern "C" inolf_status inolf_sched_complete(inolf_sched* s, uint64_t id, int64_t now_ns) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_sched_complete: NULL scheduler");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->inflight.find(id);
  if (it == s->inflight.end()) return fail(INOLF_E_UNKNOWN_TICKET, "inolf_sched_complete: not in flight");
  Viewer& v = s->viewers[it->second.viewer];
  const double dt = (double)(now_ns - it->second.start_ns) * 1e-9;
  v.ema_s = v.have_ema ? (1.0 - s->ema_alpha) * v.ema_s + s->ema_alpha * dt : dt;
  v.have_ema = true;
  v.last_frame_ns = now_ns;
  v.loaded -= 1;
  s->rays_in_flight -= it->second.rays;
  s->inflight.erase(it);
  return INOLF_OK;
}

extern "C" inolf_status inolf_sched_cancel(inolf_sched* s, uint64_t id) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_sched_cancel: NULL scheduler");
  std::lock_guard<std::mutex> lk(s->mu);
  for (size_t k = 0; k < s->pending.size(); ++k)
    if (s->pending[k].id == id) {
      s->pending.erase(s->pending.begin() + k);
      return INOLF_OK;
    }
  return fail(INOLF_E_UNKNOWN_TICKET, "inolf_sched_cancel: not pending");
}

extern "C" inolf_status inolf_sched_state(inolf_sched* s, int64_t now_ns, int32_t* starving, int64_t* rays_in_flight,
                                          int64_t* pending, int64_t* denied) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_sched_state: NULL scheduler");
  std::lock_guard<std::mutex> lk(s->mu);
  if (starving) *starving = s->any_starved(now_ns) ? 1 : 0;
  if (rays_in_flight) *rays_in_flight = s->rays_in_flight;
  if (pending) *pending = (int64_t)s->pending.size();
  if (denied) *denied = s->denied;
  return INOLF_OK;
}

extern "C" inolf_status inolf_sched_wait_ns(inolf_sched* s, uint32_t viewer, int64_t* w_ns, int64_t* target_ns) {
  clear_error();
  if (!s) return fail(INOLF_E_INVALID, "inolf_sched_wait_ns: NULL scheduler");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->viewers.find(viewer);
  if (it == s->viewers.end()) return fail(INOLF_E_UNKNOWN_TICKET, "inolf_sched_wait_ns: unknown viewer");
  const Viewer& v = it->second;
  if (w_ns) *w_ns = (int64_t)(std::max(0.0, 1.0 / v.fps - (v.have_ema ? v.ema_s : 0.0)) * 1e9);
  if (target_ns) *target_ns = s->target_ns(v);
  return INOLF_OK;
}
