// pa_server.cu -- serving: annealing runs submitted as requests and
// advanced with continuous batching.
#include "pa_engine.h"


// ---------------------------------------------------------------------------
// Serving: continuous batching of annealing requests.  A fixed table of run
// slots lives on the device; every tick admits queued requests whose memory
// fits the budget (FIFO), advances all admitted runs together -- one launch
// of each step kernel covers every active run, whatever its lattice, step
// or temperature -- and retires finished runs, returning their memory.
// ---------------------------------------------------------------------------
#include <chrono>
#include <deque>
#include <map>

struct ServerReq {
  int64_t id = 0;
  pa_run_spec spec{};
  std::vector<int8_t> J;
  std::vector<double> betas;
  int theta = 10;
  int n_steps = 0;
  Geometry geo{};
  int64_t cap = 0;
  size_t bytes = 0;
  int status = 0;  // 0 queued, 1 running, 2 done, 3 failed
  int error = 0;
  int slot = -1;
  int steps_done = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  RunDev last{};
  std::vector<double> traj;
  int64_t flips = 0;
};

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

struct pa_server {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  pa_alloc_fn fa = nullptr;
  pa_free_fn ff = nullptr;
  void* actx = nullptr;
  int max_runs = 0, max_steps = 0, tpb_opt = 0, split_opt = 0;
  size_t budget = 0, used = 0;
  RunDev* d_runs = nullptr;
  std::vector<RunDev> h;
  std::vector<int64_t> slot_req;
  std::vector<DevBuf> slot_mem;
  std::map<int64_t, ServerReq> reqs;
  std::deque<int64_t> queue;
  int64_t next_id = 1;
  bool dirty = true;
  std::vector<int32_t> active;
  DevBuf ids_buf, copy_buf, init_ids_buf;
  int n_copy = 0;
  std::vector<LatticeClass> cls;
  std::vector<DevBuf> cls_buf, init_buf;
  std::chrono::steady_clock::time_point t0;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  void* dalloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    void* p = nullptr;
    if (fa) p = fa(bytes, (void*)st, actx);
    else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    return p;
  }
  void dfree(void* p, size_t bytes) {
    if (!p) return;
    if (ff) ff(p, (bytes + 255) / 256 * 256, (void*)st, actx);
    else cudaFreeAsync(p, st);
  }
  // grow-only device buffer
  bool ensure(DevBuf& b, size_t bytes) {
    if (b.n >= bytes && b.p) return true;
    dfree(b.p, b.n);
    b.p = dalloc(std::max<size_t>(bytes, 256));
    b.n = b.p ? std::max<size_t>(bytes, 256) : 0;
    return b.p != nullptr;
  }
};

static int server_rebuild_tables(pa_server* S) {
  S->active.clear();
  for (int sl = 0; sl < S->max_runs; ++sl)
    if (S->slot_req[sl] >= 0 && S->reqs[S->slot_req[sl]].status == 1) S->active.push_back(sl);
  std::vector<Work> ct;
  for (int32_t sl : S->active)
    for (int64_t f = 0; f < S->h[sl].R_cap; f += CHUNK) ct.push_back({sl, (int32_t)f});
  S->n_copy = (int)ct.size();
  if (!S->ensure(S->ids_buf, 4 * std::max<size_t>(S->active.size(), 1)) ||
      !S->ensure(S->copy_buf, sizeof(Work) * std::max<size_t>(ct.size(), 1)))
    return fail(PA_ERR_OOM, "server tables");
  if (!S->active.empty())
    PA_CUDA(cudaMemcpyAsync(S->ids_buf.p, S->active.data(), 4 * S->active.size(), cudaMemcpyHostToDevice, S->st));
  if (!ct.empty())
    PA_CUDA(cudaMemcpyAsync(S->copy_buf.p, ct.data(), sizeof(Work) * ct.size(), cudaMemcpyHostToDevice, S->st));
  for (auto& c : S->cls) {
    c.runs.clear();
    c.nwork = 0;
  }
  for (int32_t sl : S->active) {
    const RunDev& d = S->h[sl];
    size_t k = 0;
    while (k < S->cls.size() && !(S->cls[k].dim == d.dim && S->cls[k].L == d.L)) ++k;
    if (k == S->cls.size()) {
      LatticeClass c;
      c.dim = d.dim;
      c.L = d.L;
      c.W = d.W;
      c.Wr = d.Wr;
      set_default_launch(c, S->tpb_opt, S->split_opt);
      S->cls.push_back(c);
      S->cls_buf.push_back(DevBuf());
      S->init_buf.push_back(DevBuf());
      int st = prepare_class_launches(S->d_runs, S->st, c);  // shared-memory limits, outside any capture
      if (st != PA_OK) return st;
    }
    S->cls[k].runs.push_back(sl);
  }
  for (size_t k = 0; k < S->cls.size(); ++k) {
    LatticeClass& c = S->cls[k];
    std::vector<Work> t;
    for (int32_t sl : c.runs)
      for (int64_t f = 0; f < S->h[sl].R_cap; f += c.tpb) t.push_back({sl, (int32_t)f});
    c.nwork = (int)t.size();
    if (!S->ensure(S->cls_buf[k], sizeof(Work) * std::max<size_t>(t.size(), 1))) return fail(PA_ERR_OOM, "server tables");
    c.d_table = (Work*)S->cls_buf[k].p;
    if (!t.empty())
      PA_CUDA(cudaMemcpyAsync(c.d_table, t.data(), sizeof(Work) * t.size(), cudaMemcpyHostToDevice, S->st));
  }
  // pageable uploads above: let them land before the host vectors go away
  PA_CUDA(cudaStreamSynchronize(S->st));
  S->dirty = false;
  return PA_OK;
}

static int server_init_runs(pa_server* S, const std::vector<int32_t>& fresh) {
  if (fresh.empty()) return PA_OK;
  if (!S->ensure(S->init_ids_buf, 4 * fresh.size())) return fail(PA_ERR_OOM, "server tables");
  PA_CUDA(cudaMemcpyAsync(S->init_ids_buf.p, fresh.data(), 4 * fresh.size(), cudaMemcpyHostToDevice, S->st));
  int max_bins = 0;
  for (int32_t sl : fresh) max_bins = std::max(max_bins, S->h[sl].nbins);
  PA_CUDA(launch_init_state(S->d_runs, (const int32_t*)S->init_ids_buf.p, (int)fresh.size(), max_bins, S->st));
  for (size_t k = 0; k < S->cls.size(); ++k) {
    const LatticeClass& c = S->cls[k];
    std::vector<Work> t;
    for (int32_t sl : fresh)
      if (S->h[sl].dim == c.dim && S->h[sl].L == c.L)
        for (int64_t f = 0; f < S->h[sl].R_cap; f += c.tpb) t.push_back({sl, (int32_t)f});
    if (t.empty()) continue;
    if (!S->ensure(S->init_buf[k], sizeof(Work) * t.size())) return fail(PA_ERR_OOM, "server tables");
    PA_CUDA(cudaMemcpyAsync(S->init_buf[k].p, t.data(), sizeof(Work) * t.size(), cudaMemcpyHostToDevice, S->st));
    int st = launch_class_on(S->d_runs, S->st, c, (const Work*)S->init_buf[k].p, (int)t.size(), true, c.tpb);
    if (st != PA_OK) return st;
  }
  PA_CUDA(launch_init_finish(S->d_runs, (const int32_t*)S->init_ids_buf.p, (int)fresh.size(), S->st));
  PA_CUDA(cudaStreamSynchronize(S->st));
  return PA_OK;
}

extern "C" {

int pa_server_create(const pa_opts* opts, double hbm_budget_bytes, int max_runs, pa_server** out) {
  if (!out || max_runs < 1) return fail(PA_ERR_INVALID, "bad server arguments");
  *out = nullptr;
  pa_server* S = new (std::nothrow) pa_server();
  if (!S) return fail(PA_ERR_OOM, "host allocation");
  S->t0 = std::chrono::steady_clock::now();
  cudaGetDevice(&S->device);
  int st = ensure_device_constants(S->device);
  if (st != PA_OK) {
    delete S;
    return st;
  }
  S->st = opts ? (cudaStream_t)opts->stream : nullptr;
  S->fa = opts ? opts->alloc : nullptr;
  S->ff = opts ? opts->free : nullptr;
  S->actx = opts ? opts->alloc_ctx : nullptr;
  S->max_steps = (opts && opts->max_steps > 0) ? opts->max_steps : 1024;
  S->tpb_opt = opts ? opts->threads_per_block : 0;
  S->split_opt = opts ? opts->threads_per_replica : 0;
  S->max_runs = max_runs;
  if (!S->st) {
    if (cudaStreamCreateWithFlags(&S->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete S;
      return fail(PA_ERR_CUDA, "stream creation");
    }
    S->own_stream = true;
  }
  if (hbm_budget_bytes > 0) {
    S->budget = (size_t)hbm_budget_bytes;
  } else {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    S->budget = (size_t)(0.8 * (double)fr);
  }
  S->h.assign(max_runs, RunDev());
  S->slot_req.assign(max_runs, -1);
  S->slot_mem.assign(max_runs, DevBuf());
  S->d_runs = (RunDev*)S->dalloc(sizeof(RunDev) * max_runs);
  if (!S->d_runs) {
    if (S->own_stream) cudaStreamDestroy(S->st);
    delete S;
    return fail(PA_ERR_OOM, "server run table");
  }
  *out = S;
  return PA_OK;
}

void pa_server_destroy(pa_server* S) {
  if (!S) return;
  cudaSetDevice(S->device);
  cudaStreamSynchronize(S->st);
  for (int sl = 0; sl < S->max_runs; ++sl) S->dfree(S->slot_mem[sl].p, S->slot_mem[sl].n);
  S->dfree(S->ids_buf.p, S->ids_buf.n);
  S->dfree(S->copy_buf.p, S->copy_buf.n);
  S->dfree(S->init_ids_buf.p, S->init_ids_buf.n);
  for (auto& b : S->cls_buf) S->dfree(b.p, b.n);
  for (auto& b : S->init_buf) S->dfree(b.p, b.n);
  S->dfree(S->d_runs, sizeof(RunDev) * S->max_runs);
  cudaStreamSynchronize(S->st);
  if (S->own_stream) cudaStreamDestroy(S->st);
  delete S;
}

double pa_server_clock(pa_server* S) { return S ? S->now() : 0.0; }

int pa_server_submit(pa_server* S, const pa_request* q, int64_t* id) {
  if (!S || !q || !q->betas) return fail(PA_ERR_INVALID, "bad request");
  if (q->n_steps < 1 || q->n_steps > S->max_steps || q->theta < 0 || q->R0 < 1)
    return fail(PA_ERR_INVALID, "request: n_steps in 1..%d, theta >= 0, R0 >= 1", S->max_steps);
  ServerReq r;
  r.spec.dim = q->dim;
  r.spec.L = q->L;
  r.spec.R0 = q->R0;
  r.spec.seed = q->seed;
  r.spec.R_cap = 0;
  int st = make_geometry(q->couplings, q->L, q->dim, &r.geo);
  if (st != PA_OK) return st;
  const size_t jn = (size_t)(q->dim == 3 ? 3 * r.geo.N : r.geo.N);
  r.J.assign(q->couplings, q->couplings + jn);
  r.spec.couplings = r.J.data();
  double prev = 0.0;
  for (int k = 0; k < q->n_steps; ++k) {
    if (!(q->betas[k] >= prev) || !std::isfinite(q->betas[k])) return fail(PA_ERR_INVALID, "betas must not decrease");
    prev = q->betas[k];
  }
  r.betas.assign(q->betas, q->betas + q->n_steps);
  r.theta = q->theta;
  r.n_steps = q->n_steps;
  r.cap = default_capacity(q->R0);
  r.bytes = run_slab_bytes(r.geo, r.cap, S->max_steps);
  if (r.bytes > S->budget) return fail(PA_ERR_OOM, "request needs %zu bytes, budget %zu", r.bytes, S->budget);
  r.id = S->next_id++;
  r.t_submit = S->now();
  const int64_t rid = r.id;
  S->reqs[rid] = std::move(r);
  S->reqs[rid].spec.couplings = S->reqs[rid].J.data();
  S->queue.push_back(rid);
  if (id) *id = rid;
  return PA_OK;
}

int pa_server_tick(pa_server* S, int steps, int32_t* n_active, int32_t* n_queued, int32_t* n_finished) {
  if (!S || steps < 0) return fail(PA_ERR_INVALID, "bad tick arguments");
  PA_CUDA(cudaSetDevice(S->device));
  NvtxRange tick_range("pa_server_tick");
  int st;
  // 1. admission by device-memory budget, in arrival order
  std::vector<int32_t> fresh;
  while (!S->queue.empty()) {
    ServerReq& q = S->reqs[S->queue.front()];
    if (S->used + q.bytes > S->budget) break;
    int slot = -1;
    for (int sl = 0; sl < S->max_runs; ++sl)
      if (S->slot_req[sl] < 0) {
        slot = sl;
        break;
      }
    if (slot < 0) break;
    void* mem = S->dalloc(q.bytes);
    if (!mem) break;  // refused: the request stays first in the queue, retried on a later tick
    RunDev d;
    st = setup_run((char*)mem, q.geo, q.spec, q.cap, S->max_steps, S->st, &d);
    if (st != PA_OK) {
      // the request fails alone; its memory goes back and the server carries on
      cudaStreamSynchronize(S->st);
      S->dfree(mem, q.bytes);
      q.status = 3;
      q.error = st;
      q.t_done = S->now();
      S->queue.pop_front();
      continue;
    }
    std::vector<int32_t> th(q.n_steps, q.theta);
    std::vector<int64_t> rt(q.n_steps, q.spec.R0);
    PA_CUDA(cudaMemcpyAsync(d.sched_beta, q.betas.data(), 8 * (size_t)q.n_steps, cudaMemcpyHostToDevice, S->st));
    PA_CUDA(cudaMemcpyAsync(d.sched_theta, th.data(), 4 * (size_t)q.n_steps, cudaMemcpyHostToDevice, S->st));
    PA_CUDA(cudaMemcpyAsync(d.sched_R, rt.data(), 8 * (size_t)q.n_steps, cudaMemcpyHostToDevice, S->st));
    d.n_sched = q.n_steps;
    S->h[slot] = d;
    PA_CUDA(cudaMemcpyAsync(&S->d_runs[slot], &S->h[slot], sizeof(RunDev), cudaMemcpyHostToDevice, S->st));
    PA_CUDA(cudaStreamSynchronize(S->st));
    S->slot_mem[slot] = {mem, (q.bytes + 255) / 256 * 256};
    S->slot_req[slot] = q.id;
    S->used += q.bytes;
    q.slot = slot;
    q.status = 1;
    q.t_admit = S->now();
    fresh.push_back(slot);
    S->queue.pop_front();
    S->dirty = true;
  }
  if (S->dirty) {
    st = server_rebuild_tables(S);
    if (st != PA_OK) return st;
  }
  st = server_init_runs(S, fresh);
  if (st != PA_OK) return st;
  // 2. advance every active run by up to `steps` annealing steps
  const int na = (int)S->active.size();
  const int32_t* ids = (const int32_t*)S->ids_buf.p;
  for (int k = 0; k < steps && na > 0; ++k) {
    PA_CUDA(launch_prepare(S->d_runs, ids, na, false, 0.0, 0, 0, S->st));
    PA_CUDA(launch_copies(S->d_runs, (const Work*)S->copy_buf.p, S->n_copy, S->st));
    PA_CUDA(launch_scan(S->d_runs, ids, na, S->st));
    PA_CUDA(launch_scatter(S->d_runs, (const Work*)S->copy_buf.p, S->n_copy, S->st));
    for (auto& c : S->cls) {
      if (c.nwork == 0) continue;
      st = launch_class_on(S->d_runs, S->st, c, c.d_table, c.nwork, false, c.tpb);
      if (st != PA_OK) return st;
    }
    PA_CUDA(launch_commit(S->d_runs, ids, na, S->st));
  }
  // 3. retire finished (or failed) runs
  PA_CUDA(cudaStreamSynchronize(S->st));
  int finished = 0;
  if (na > 0) {
    std::vector<RunDev> cur(S->max_runs);
    PA_CUDA(cudaMemcpy(cur.data(), S->d_runs, sizeof(RunDev) * S->max_runs, cudaMemcpyDeviceToHost));
    for (int32_t sl : S->active) {
      ServerReq& q = S->reqs[S->slot_req[sl]];
      const RunDev& D = cur[sl];
      q.steps_done = (int)D.step;
      if (D.error == 0 && D.step < q.n_steps) continue;
      q.last = D;
      q.error = D.error;
      q.status = D.error ? 3 : 2;
      q.t_done = S->now();
      const int64_t cnt = std::min<int64_t>(D.step, D.max_steps) + 1;
      q.traj.resize(cnt);
      PA_CUDA(cudaMemcpy(q.traj.data(), D.rec_mbF, 8 * cnt, cudaMemcpyDeviceToHost));
      std::vector<int64_t> rr(cnt);
      PA_CUDA(cudaMemcpy(rr.data(), D.rec_R, 8 * cnt, cudaMemcpyDeviceToHost));
      q.flips = 0;
      for (int64_t k = 1; k < cnt; ++k) q.flips += rr[k] * (int64_t)D.N * (int64_t)q.theta;
      S->dfree(S->slot_mem[sl].p, S->slot_mem[sl].n);
      S->slot_mem[sl] = DevBuf();
      S->slot_req[sl] = -1;
      S->used -= q.bytes;
      S->dirty = true;
      ++finished;
    }
  }
  if (n_active) *n_active = (int32_t)(na - finished);
  if (n_queued) *n_queued = (int32_t)S->queue.size();
  if (n_finished) *n_finished = finished;
  return PA_OK;
}

int pa_server_cancel(pa_server* S, int64_t id) {
  if (!S) return fail(PA_ERR_INVALID, "server is NULL");
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(PA_ERR_INVALID, "unknown request %lld", (long long)id);
  ServerReq& q = it->second;
  if (q.status == 0) {
    for (auto qi = S->queue.begin(); qi != S->queue.end(); ++qi)
      if (*qi == id) {
        S->queue.erase(qi);
        break;
      }
  } else if (q.status == 1) {
    // between ticks nothing of the server is in flight: its slot and memory
    // are released at once (stream-ordered), and the next tick's tables leave
    // the slot out
    PA_CUDA(cudaSetDevice(S->device));
    PA_CUDA(cudaStreamSynchronize(S->st));
    const int sl = q.slot;
    S->dfree(S->slot_mem[sl].p, S->slot_mem[sl].n);
    S->slot_mem[sl] = DevBuf();
    S->slot_req[sl] = -1;
    S->used -= q.bytes;
    S->dirty = true;
    q.slot = -1;
  } else {
    return PA_OK;  // finished, failed or cancelled already: nothing to do
  }
  q.status = 4;
  q.t_done = S->now();
  return PA_OK;
}

int pa_server_memory(pa_server* S, int64_t* used_bytes, int64_t* budget_bytes, int32_t* runs_resident) {
  if (!S) return fail(PA_ERR_INVALID, "server is NULL");
  if (used_bytes) *used_bytes = (int64_t)S->used;
  if (budget_bytes) *budget_bytes = (int64_t)S->budget;
  if (runs_resident) {
    int32_t n = 0;
    for (int sl = 0; sl < S->max_runs; ++sl) n += S->slot_req[sl] >= 0;
    *runs_resident = n;
  }
  return PA_OK;
}

int pa_server_result(pa_server* S, int64_t id, pa_result* out, double* traj, int64_t count) {
  if (!S || !out) return fail(PA_ERR_INVALID, "bad arguments");
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(PA_ERR_INVALID, "unknown request %lld", (long long)id);
  const ServerReq& q = it->second;
  memset(out, 0, sizeof *out);
  out->status = q.status;
  out->error = q.error;
  const bool ended = q.status == 2 || q.status == 3;
  out->steps = ended ? q.last.step : q.steps_done;
  out->submit_s = q.t_submit;
  out->admit_s = q.t_admit;
  out->done_s = q.t_done;
  out->device_bytes = (int64_t)q.bytes;
  out->flips = q.flips;
  if (ended) {
    out->R = q.last.R;
    out->beta = q.last.beta;
    out->minus_beta_F = q.last.mbF;
    out->E_mean = (double)q.last.sumE / (double)q.last.R;
    out->sumE = q.last.sumE;
    out->sumE2 = q.last.sumE2;
    if (traj)
      for (int64_t k = 0; k < count && k < (int64_t)q.traj.size(); ++k) traj[k] = q.traj[k];
  }
  return PA_OK;
}

}  // extern "C"
