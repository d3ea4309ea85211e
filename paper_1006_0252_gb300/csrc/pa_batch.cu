// pa_batch.cu -- the C ABI of batches: many independent runs (Sec. 3)
// advanced together by one Engine, their schedules captured as CUDA graphs,
// and the Sec. 3 estimators over groups of runs computed on the device.
#include <algorithm>
#include "pa_engine.h"

extern "C" {

// ---------------------------------------------------------------------------
// C ABI: batches
// ---------------------------------------------------------------------------
int pa_batch_create(int n_runs, const pa_run_spec* specs, const pa_opts* opts, pa_batch** out) {
  if (!out) return fail(PA_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  pa_batch* b = new (std::nothrow) pa_batch();
  if (!b) return fail(PA_ERR_OOM, "host allocation");
  int st = engine_create(b->e, n_runs, specs, opts);
  if (st != PA_OK) {
    const std::string msg = last_error_message();  // release() may overwrite it
    b->e.release();
    delete b;
    return fail(st, "%s", msg.c_str());
  }
  *out = b;
  clear_last_error();
  return PA_OK;
}

int pa_batch_reset(pa_batch* b, const uint64_t* seeds) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  // the seeds and population sizes live in the device run table; patch them
  // there in stream order (the host copies outlive the copies)
  for (int r = 0; r < E.n; ++r) {
    if (seeds) E.h[r].seed = seeds[r];
    PA_CUDA(cudaMemcpyAsync(&E.d_runs[r].seed, &E.h[r].seed, sizeof(uint64_t), cudaMemcpyHostToDevice, E.st));
    PA_CUDA(cudaMemcpyAsync(&E.d_runs[r].R, &E.R0[r], sizeof(int64_t), cudaMemcpyHostToDevice, E.st));
  }
  int st = engine_init_population(E);
  if (st != PA_OK) return st;
  for (int r = 0; r < E.n; ++r) E.host_beta[r] = 0.0;
  E.host_steps = 0;
  return PA_OK;
}

void pa_batch_destroy(pa_batch* b) {
  if (!b) return;
  cudaSetDevice(b->e.device);
  b->e.release();
  delete b;
}

int pa_batch_run(pa_batch* b, int n_steps, const double* betas, int per_run, const int32_t* thetas,
                 const int64_t* R_targets, int use_graph) {
  if (!b || !betas || n_steps < 0) return fail(PA_ERR_INVALID, "bad batch-run arguments");
  return engine_run_schedule(b->e, n_steps, betas, per_run, thetas, R_targets, use_graph);
}

int pa_batch_sync(pa_batch* b, int32_t* errors) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  return engine_sync(b->e, errors);
}

int pa_batch_results(pa_batch* b, double* beta, double* mbF, int64_t* R, int64_t* sumE, int64_t* sumE2,
                     int64_t* step) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  std::vector<RunDev> d;
  int st = engine_fetch(b->e, d);
  if (st != PA_OK) return st;
  for (int r = 0; r < b->e.n; ++r) {
    if (beta) beta[r] = d[r].beta;
    if (mbF) mbF[r] = d[r].mbF;
    if (R) R[r] = d[r].R;
    if (sumE) sumE[r] = d[r].sumE;
    if (sumE2) sumE2[r] = d[r].model == 1 ? 0 : d[r].sumE2;
    if (step) step[r] = d[r].step;
  }
  return PA_OK;
}

int pa_batch_trajectory(pa_batch* b, int64_t count, double* mbF, int64_t* R, int64_t* sumE, int64_t* sumE2) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  const int64_t c = std::min<int64_t>(count, E.max_steps + 1);
  for (int r = 0; r < E.n; ++r) {
    const RunDev& D = E.h[r];
    if (mbF) PA_CUDA(cudaMemcpy(mbF + r * count, D.rec_mbF, 8 * c, cudaMemcpyDeviceToHost));
    if (R) PA_CUDA(cudaMemcpy(R + r * count, D.rec_R, 8 * c, cudaMemcpyDeviceToHost));
    if (sumE) PA_CUDA(cudaMemcpy(sumE + r * count, D.rec_sumE, 8 * c, cudaMemcpyDeviceToHost));
    if (sumE2) {
      if (D.model == 1) memset(sumE2 + r * count, 0, 8 * c);
      else PA_CUDA(cudaMemcpy(sumE2 + r * count, D.rec_sumE2, 8 * c, cudaMemcpyDeviceToHost));
    }
  }
  return PA_OK;
}

int pa_batch_energy(pa_batch* b, int64_t count, double* E_mean, double* E2_mean) {
  if (!b || count < 0) return fail(PA_ERR_INVALID, "bad arguments");
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  const int64_t c = std::min<int64_t>(count, E.max_steps + 1);
  std::vector<int64_t> R(c), s1(c), s2(c);
  for (int r = 0; r < E.n; ++r) {
    const RunDev& D = E.h[r];
    if (c == 0) break;
    PA_CUDA(cudaMemcpy(R.data(), D.rec_R, 8 * c, cudaMemcpyDeviceToHost));
    PA_CUDA(cudaMemcpy(s1.data(), D.rec_sumE, 8 * c, cudaMemcpyDeviceToHost));
    PA_CUDA(cudaMemcpy(s2.data(), D.rec_sumE2, 8 * c, cudaMemcpyDeviceToHost));
    const double unit = D.model == 1 ? 0x1.0p-15 : 1.0;
    for (int64_t k = 0; k < c; ++k) {
      double e2;
      if (D.model == 1) memcpy(&e2, &s2[k], 8);
      else e2 = (double)s2[k];
      const double Rk = R[k] > 0 ? (double)R[k] : 1.0;
      if (E_mean) E_mean[r * count + k] = (double)s1[k] * unit / Rk;
      if (E2_mean) E2_mean[r * count + k] = e2 / Rk;
    }
  }
  return PA_OK;
}

int pa_batch_diagnostics(pa_batch* b, int M, int64_t count, double* E_bar, double* minus_beta_Fbar,
                         double* var_minus_beta_F) {
  if (!b || M < 1 || count < 1) return fail(PA_ERR_INVALID, "bad arguments");
  Engine& E = b->e;
  if (E.n % M != 0) return fail(PA_ERR_INVALID, "%d runs do not split into groups of %d", E.n, M);
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  for (int r = 0; r < E.n; ++r) {
    if (d[r].error) return fail(d[r].error, "run %d: device: %s", r, err_name(d[r].error));
    if (count > std::min<int64_t>(d[r].step, d[r].max_steps) + 1)
      return fail(PA_ERR_INVALID, "run %d has only %lld records", r, (long long)(std::min<int64_t>(d[r].step, d[r].max_steps) + 1));
  }
  const int G = E.n / M;
  const int64_t GK = (int64_t)G * count;
  if (GK > INT32_MAX) return fail(PA_ERR_INVALID, "too many groups and records");
  const size_t nval = (size_t)GK * M;
  const size_t bytes = sizeof(double) * (3 * nval + 3 * (size_t)GK);
  double* buf = (double*)E.dalloc(bytes);
  if (!buf) return fail(PA_ERR_OOM, "diagnostics scratch of %zu bytes refused", bytes);
  double *x = buf, *A = x + nval, *Rw = A + nval, *mean = Rw + nval, *fbar = mean + GK, *var = fbar + GK;
  cudaError_t e = launch_gather_records(E.d_runs, M, (int)count, G, x, A, Rw, E.st);
  if (e == cudaSuccess) e = launch_weighted((int)GK, M, x, A, Rw, mean, fbar, E.st);
  if (e == cudaSuccess) e = launch_variance((int)GK, M, x, var, E.st);
  if (e == cudaSuccess && E_bar) e = cudaMemcpyAsync(E_bar, mean, 8 * GK, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess && minus_beta_Fbar) e = cudaMemcpyAsync(minus_beta_Fbar, fbar, 8 * GK, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess && var_minus_beta_F) e = cudaMemcpyAsync(var_minus_beta_F, var, 8 * GK, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.st);
  E.dfree(buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "batch diagnostics");
  return PA_OK;
}

int pa_batch_bootstrap(pa_batch* b, int M, int64_t count, int B, uint64_t seed, double* sd_E_bar,
                       double* sd_minus_beta_Fbar) {
  if (!b || M < 1 || count < 1 || B < 2 || B > (1 << 20)) return fail(PA_ERR_INVALID, "bad arguments");
  Engine& E = b->e;
  if (E.n % M != 0) return fail(PA_ERR_INVALID, "%d runs do not split into groups of %d", E.n, M);
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  for (int r = 0; r < E.n; ++r) {
    if (d[r].error) return fail(d[r].error, "run %d: device: %s", r, err_name(d[r].error));
    if (count > std::min<int64_t>(d[r].step, d[r].max_steps) + 1)
      return fail(PA_ERR_INVALID, "run %d has only %lld records", r, (long long)(std::min<int64_t>(d[r].step, d[r].max_steps) + 1));
  }
  const int G = E.n / M;
  const int64_t GK = (int64_t)G * count;
  if (GK > INT32_MAX) return fail(PA_ERR_INVALID, "too many groups and records");
  const size_t nval = (size_t)GK * M, nres = (size_t)GK * B;
  const size_t bytes = sizeof(double) * (3 * nval + 2 * nres + 2 * (size_t)GK);
  double* buf = (double*)E.dalloc(bytes);
  if (!buf) return fail(PA_ERR_OOM, "bootstrap scratch of %zu bytes refused", bytes);
  double *x = buf, *A = x + nval, *Rw = A + nval, *bm = Rw + nval, *bf = bm + nres, *sm = bf + nres, *sf = sm + GK;
  cudaError_t e = launch_gather_records(E.d_runs, M, (int)count, G, x, A, Rw, E.st);
  if (e == cudaSuccess) e = launch_bootstrap(M, x, A, Rw, B, seed, bm, bf, E.st, (int)GK);
  if (e == cudaSuccess) e = launch_variance((int)GK, B, bm, sm, E.st, true);
  if (e == cudaSuccess) e = launch_variance((int)GK, B, bf, sf, E.st, true);
  if (e == cudaSuccess && sd_E_bar) e = cudaMemcpyAsync(sd_E_bar, sm, 8 * GK, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess && sd_minus_beta_Fbar)
    e = cudaMemcpyAsync(sd_minus_beta_Fbar, sf, 8 * GK, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.st);
  E.dfree(buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "batch bootstrap");
  return PA_OK;
}

int pa_batch_overlap(pa_batch* b, int n_pairs, const int32_t* run_a, const int32_t* run_b, double qcut,
                     double* gamma, int64_t* npairs) {
  if (!b || n_pairs < 1 || !run_a || !run_b || !gamma) return fail(PA_ERR_INVALID, "bad arguments");
  if (n_pairs > 65535) return fail(PA_ERR_INVALID, "at most 65535 pairs per call");
  Engine& E = b->e;
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  for (int p = 0; p < n_pairs; ++p) {
    const int a = run_a[p], c = run_b[p];
    if (a < 0 || a >= E.n || c < 0 || c >= E.n) return fail(PA_ERR_INVALID, "pair %d: run index out of range", p);
    if (d[a].N != d[c].N || d[a].W != d[c].W || d[a].dim != d[c].dim)
      return fail(PA_ERR_INVALID, "pair %d: runs differ in lattice", p);
    if (d[a].error || d[c].error) return fail(PA_ERR_INVALID, "pair %d: a run has a sticky error", p);
  }
  const size_t bytes = 8 * (size_t)n_pairs + 2 * 4 * (size_t)n_pairs;
  char* buf = (char*)E.dalloc(bytes);
  if (!buf) return fail(PA_ERR_OOM, "overlap scratch refused");
  unsigned long long* cnt = (unsigned long long*)buf;
  int32_t* ia = (int32_t*)(buf + 8 * (size_t)n_pairs);
  int32_t* ib = ia + n_pairs;
  std::vector<unsigned long long> hc(n_pairs);
  cudaError_t e = cudaMemsetAsync(cnt, 0, 8 * (size_t)n_pairs, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ia, run_a, 4 * (size_t)n_pairs, cudaMemcpyHostToDevice, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ib, run_b, 4 * (size_t)n_pairs, cudaMemcpyHostToDevice, E.st);
  if (e == cudaSuccess) e = launch_overlap_pairs(E.d_runs, ia, ib, n_pairs, qcut, cnt, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hc.data(), cnt, 8 * (size_t)n_pairs, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.st);
  E.dfree(buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "batch overlap");
  for (int p = 0; p < n_pairs; ++p) {
    const int64_t np = std::min(d[run_a[p]].R, d[run_b[p]].R);
    gamma[p] = np > 0 ? (double)hc[p] / (double)np : 0.0;
    if (npairs) npairs[p] = np;
  }
  return PA_OK;
}

int pa_batch_overlap_hist(pa_batch* b, int n_pairs, const int32_t* run_a, const int32_t* run_b, int64_t* hist) {
  if (!b || n_pairs < 1 || !run_a || !run_b || !hist) return fail(PA_ERR_INVALID, "bad arguments");
  if (n_pairs > 65535) return fail(PA_ERR_INVALID, "at most 65535 pairs per call");
  Engine& E = b->e;
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  if (run_a[0] < 0 || run_a[0] >= E.n) return fail(PA_ERR_INVALID, "pair 0: run index out of range");
  const RunDev& D0 = d[run_a[0]];
  for (int p = 0; p < n_pairs; ++p) {
    const int a = run_a[p], c = run_b[p];
    if (a < 0 || a >= E.n || c < 0 || c >= E.n) return fail(PA_ERR_INVALID, "pair %d: run index out of range", p);
    if (d[a].N != D0.N || d[c].N != D0.N || d[a].W != D0.W || d[c].W != D0.W || d[a].dim != D0.dim ||
        d[c].dim != D0.dim)
      return fail(PA_ERR_INVALID, "pair %d: runs differ in lattice from the first pair", p);
    if (d[a].error || d[c].error) return fail(PA_ERR_INVALID, "pair %d: a run has a sticky error", p);
  }
  const int nbins = D0.N + 1;
  const size_t hbytes = 8 * (size_t)n_pairs * nbins;
  const size_t bytes = hbytes + 2 * 4 * (size_t)n_pairs;
  char* buf = (char*)E.dalloc(bytes);
  if (!buf) return fail(PA_ERR_OOM, "overlap histogram scratch refused");
  unsigned long long* hd = (unsigned long long*)buf;
  int32_t* ia = (int32_t*)(buf + hbytes);
  int32_t* ib = ia + n_pairs;
  cudaError_t e = cudaMemsetAsync(hd, 0, hbytes, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ia, run_a, 4 * (size_t)n_pairs, cudaMemcpyHostToDevice, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ib, run_b, 4 * (size_t)n_pairs, cudaMemcpyHostToDevice, E.st);
  if (e == cudaSuccess) e = launch_overlap_hist(E.d_runs, ia, ib, n_pairs, nbins, hd, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hist, hd, hbytes, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.st);
  E.dfree(buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "batch overlap histogram");
  return PA_OK;
}

int pa_batch_copy_spins(pa_batch* b, int r, int8_t* host_dst, int64_t max_replicas, int64_t* n) {
  if (!b || !host_dst || r < 0 || r >= b->e.n) return fail(PA_ERR_INVALID, "bad arguments");
  return engine_copy_spins(b->e, r, host_dst, max_replicas, n);
}

int pa_batch_autotune(pa_batch* b, int32_t sweeps, int32_t* host_L, int32_t* host_tpb, int32_t* host_split,
                      int* n_out) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  const int dry_sweeps = sweeps <= 0 ? 10 : std::min(sweeps, 20);
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  // Dry step at the current temperature, with the schedule's sweeps per step
  // (up to 20: a block's fixed cost, the uniform tables it builds, weighs
  // less the more sweeps it runs, so too few sweeps favour fewer, larger
  // shares per block): prepare/copies/scan/scatter fill the
  // staged population; each candidate sweep launch reads the unchanged
  // population and writes only the spare buffer; nothing is committed.
  int pst = engine_prep(E, true, -1.0, dry_sweeps, -1);
  if (pst != PA_OK) return pst;
  PA_CUDA(launch_copies(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  PA_CUDA(launch_scan(E.d_runs, nullptr, E.n, E.st));
  PA_CUDA(launch_scatter(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  cudaEvent_t t0, t1;
  PA_CUDA(cudaEventCreate(&t0));
  PA_CUDA(cudaEventCreate(&t1));
  int count = 0;
  for (auto& c : E.cls) {
    // candidates: (block size, threads per replica); several threads per
    // replica only for +-1 cubic lattices whose rows split evenly
    std::vector<std::pair<int, int>> cands;
    for (int split : {1, 2, 4, 8}) {
      if (!split_supported(c, split)) continue;
      for (int tpb : {32, 64, 128, 256, 512, 1024}) {
        if (!tpb_supported(c, tpb)) continue;
        if (split == 1 && tpb == 256) continue;
        if (split > 1 && (tpb < 64 || tpb / split < 4)) continue;
        cands.push_back({tpb, split});
      }
    }
    float best = 1e30f;
    std::pair<int, int> pick = {c.tpb, c.split};
    LatticeClass trial = c;
    for (const auto& cand : cands) {
      trial.tpb = cand.first;
      trial.split = cand.second;
      trial.d_table = nullptr;
      int st = build_class_table(E, trial);
      if (st != PA_OK) return st;
      st = launch_class(E, trial, trial.d_table, trial.nwork, false, trial.tpb);  // warm-up
      if (st != PA_OK) return st;
      PA_CUDA(cudaEventRecord(t0, E.st));
      for (int rep = 0; rep < 2; ++rep) {
        st = launch_class(E, trial, trial.d_table, trial.nwork, false, trial.tpb);
        if (st != PA_OK) return st;
      }
      PA_CUDA(cudaEventRecord(t1, E.st));
      PA_CUDA(cudaEventSynchronize(t1));
      float ms = 0.f;
      PA_CUDA(cudaEventElapsedTime(&ms, t0, t1));
      E.dfree(trial.d_table, sizeof(Work) * std::max(trial.nwork, 1));
      if (ms < best) {
        best = ms;
        pick = cand;
      }
    }
    if (pick.first != c.tpb || pick.second != c.split) {
      E.dfree(c.d_table, sizeof(Work) * std::max(c.nwork, 1));
      c.tpb = pick.first;
      c.split = pick.second;
      int st = build_class_table(E, c);
      if (st != PA_OK) return st;
    }
    if (count < 8) {
      if (host_L) host_L[count] = c.dim == 1 ? -c.L : c.L;
      if (host_tpb) host_tpb[count] = c.tpb;
      if (host_split) host_split[count] = c.split;
      ++count;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  E.drop_graph();  // the launch shapes changed
  if (n_out) *n_out = count;
  return PA_OK;
}

}  // extern "C"
