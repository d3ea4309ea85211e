// pa_checkpoint.cu -- checkpoint and resume of runs and batches (no
// counterpart in the paper): a run's state is its population, energies,
// histogram, counters and per-step record, the random streams being
// counter-based.
#include "pa_engine.h"

extern "C" {

// ---- checkpoint / resume ---------------------------------------------------
// Layout: CkHeader, then spins [R][W] u32, energies [R] i32, histogram
// [nbins] u32, per-step record 6 x [n_rec] (beta, lnQ, -beta F, R, sumE, sumE2).
struct CkHeader {
  uint64_t magic;
  uint32_t version, dim;
  int32_t L, N, W, nbins;
  int64_t R_cap, R, step, sweeps;
  uint64_t seed, bonds_hash;
  double beta, mbF, lnQ_last, Qp_last;
  int64_t sumE, sumE2, n_rec;
  int64_t model, emin;  // coupling model; lowest energy (Gaussian model)
  double sumE2d;        // physical sum of E^2 (Gaussian model)
};
constexpr uint64_t CK_MAGIC = 0x504147423330304bULL;

static int fetch_hash(const RunDev& D, cudaStream_t st, uint64_t* out) {
  // +-1: the coupling masks; Gaussian: the per-site coupling table; general
  // boxes: the coupling table and the neighbour table (extents, open axes)
  size_t nw;
  const void* src;
  if (D.bx > 0) {
    nw = (size_t)12 * D.Wr * D.bsites;
    src = D.gJ;
  } else if (D.model == 1) {
    nw = D.dim == 1 ? (size_t)D.N : (size_t)12 * D.Wr * (((lanes_for(D.L) * D.L / 2) + 3) & ~3);
    src = D.gJ;
  } else {
    nw = (size_t)(D.dim == 3 ? 6 : 4) * D.W;
    src = D.bonds;
  }
  const size_t nc = D.bx > 0 ? (size_t)14 * D.Wr * D.bsites : 0;
  std::vector<uint32_t> b(nw + nc);
  PA_CUDA(cudaMemcpyAsync(b.data(), src, 4 * nw, cudaMemcpyDeviceToHost, st));
  if (nc) PA_CUDA(cudaMemcpyAsync(b.data() + nw, D.box_code, 4 * nc, cudaMemcpyDeviceToHost, st));
  PA_CUDA(cudaStreamSynchronize(st));
  uint64_t h = 1469598103934665603ULL;  // FNV-1a over the coupling masks
  for (uint32_t w : b)
    for (int k = 0; k < 4; ++k) {
      h ^= (w >> (8 * k)) & 0xFF;
      h *= 1099511628211ULL;
    }
  *out = h;
  return PA_OK;
}

static int64_t ck_records(const RunDev& D) { return std::min<int64_t>(D.step, D.max_steps) + 1; }

static size_t ck_payload(int64_t R, int W, int nbins, int64_t n_rec) {
  return (size_t)R * W * 4 + (size_t)R * 4 + (size_t)nbins * 4 + (size_t)n_rec * 48;
}

static size_t ck_bytes(const RunDev& D) {
  return sizeof(CkHeader) + ck_payload(D.R, D.W, D.nbins, ck_records(D));
}

// One run's state into a host buffer of ck_bytes(D) bytes: header, spins,
// energies, histogram and the per-step records.
static int ck_write_run(const RunDev& D, cudaStream_t st, char* p) {
  if (D.error) return fail(D.error, "device: %s (no checkpoint of a failed run)", err_name(D.error));
  CkHeader h;
  memset(&h, 0, sizeof h);
  h.magic = CK_MAGIC;
  h.version = 2;
  h.dim = (uint32_t)D.dim;
  h.L = D.L;
  h.N = D.N;
  h.W = D.W;
  h.nbins = D.nbins;
  h.R_cap = D.R_cap;
  h.R = D.R;
  h.step = D.step;
  h.sweeps = D.sweeps;
  h.seed = D.seed;
  h.beta = D.beta;
  h.mbF = D.mbF;
  h.lnQ_last = D.lnQ_last;
  h.Qp_last = D.Qp_last;
  h.sumE = D.sumE;
  h.sumE2 = D.sumE2;
  h.n_rec = ck_records(D);
  h.model = D.model;
  h.emin = D.emin;
  h.sumE2d = D.sumE2d;
  int s = fetch_hash(D, st, &h.bonds_hash);
  if (s != PA_OK) return s;
  memcpy(p, &h, sizeof h);
  p += sizeof h;
  PA_CUDA(cudaMemcpy(p, D.spins[D.cur], (size_t)D.R * D.W * 4, cudaMemcpyDeviceToHost));
  p += (size_t)D.R * D.W * 4;
  PA_CUDA(cudaMemcpy(p, D.E[D.cur], (size_t)D.R * 4, cudaMemcpyDeviceToHost));
  p += (size_t)D.R * 4;
  PA_CUDA(cudaMemcpy(p, D.hist[D.cur], (size_t)D.nbins * 4, cudaMemcpyDeviceToHost));
  p += (size_t)D.nbins * 4;
  const void* recs[6] = {D.rec_beta, D.rec_lnQ, D.rec_mbF, D.rec_R, D.rec_sumE, D.rec_sumE2};
  for (int k = 0; k < 6; ++k) {
    PA_CUDA(cudaMemcpy(p, recs[k], 8 * (size_t)h.n_rec, cudaMemcpyDeviceToHost));
    p += 8 * (size_t)h.n_rec;
  }
  return PA_OK;
}

// Check that the run state at p (avail bytes) fits the run D (lattice,
// model, capacity, record length, couplings) and give its total size.
static int ck_check_run(const RunDev& D, cudaStream_t st, const char* p, size_t avail, CkHeader* hout,
                        size_t* used) {
  if (avail < sizeof(CkHeader)) return fail(PA_ERR_INVALID, "checkpoint truncated");
  CkHeader h;
  memcpy(&h, p, sizeof h);
  if (h.magic != CK_MAGIC || h.version != 2) return fail(PA_ERR_INVALID, "not a checkpoint of this library");
  if ((int)h.dim != D.dim || h.L != D.L || h.W != D.W || h.nbins != D.nbins || h.model != D.model)
    return fail(PA_ERR_INVALID, "checkpoint lattice differs from the run's");
  if (h.R < 1 || h.R > D.R_cap) return fail(PA_ERR_INVALID, "checkpoint population exceeds the run's capacity");
  if (h.n_rec > (int64_t)D.max_steps + 1 || h.n_rec < 1 || h.step < 0)
    return fail(PA_ERR_INVALID, "checkpoint record too long");
  const size_t need = sizeof(CkHeader) + ck_payload(h.R, h.W, h.nbins, h.n_rec);
  if (avail < need) return fail(PA_ERR_INVALID, "checkpoint truncated");
  uint64_t hash;
  int s = fetch_hash(D, st, &hash);
  if (s != PA_OK) return s;
  if (hash != h.bonds_hash) return fail(PA_ERR_INVALID, "checkpoint couplings differ from the run's");
  *hout = h;
  *used = need;
  return PA_OK;
}

// Load a checked run state into D's device buffers (the population goes to
// buffer 0, which becomes current) and set D's counters from its header.
static int ck_read_run(RunDev& D, const CkHeader& h, const char* p) {
  p += sizeof h;
  PA_CUDA(cudaMemcpy(D.spins[0], p, (size_t)h.R * h.W * 4, cudaMemcpyHostToDevice));
  p += (size_t)h.R * h.W * 4;
  PA_CUDA(cudaMemcpy(D.E[0], p, (size_t)h.R * 4, cudaMemcpyHostToDevice));
  p += (size_t)h.R * 4;
  PA_CUDA(cudaMemcpy(D.hist[0], p, (size_t)h.nbins * 4, cudaMemcpyHostToDevice));
  p += (size_t)h.nbins * 4;
  void* recs[6] = {D.rec_beta, D.rec_lnQ, D.rec_mbF, D.rec_R, D.rec_sumE, D.rec_sumE2};
  for (int k = 0; k < 6; ++k) {
    PA_CUDA(cudaMemcpy(recs[k], p, 8 * (size_t)h.n_rec, cudaMemcpyHostToDevice));
    p += 8 * (size_t)h.n_rec;
  }
  D.seed = h.seed;
  D.cur = 0;
  D.error = 0;
  D.skip = 0;
  D.R = h.R;
  D.R_next = h.R;
  D.step = h.step;
  D.sweeps = h.sweeps;
  D.beta = h.beta;
  D.mbF = h.mbF;
  D.lnQ_last = h.lnQ_last;
  D.Qp_last = h.Qp_last;
  D.sumE = h.sumE;
  D.sumE2 = h.sumE2;
  D.emin = h.emin;
  D.sumE2d = h.sumE2d;
  return PA_OK;
}

int pa_checkpoint_bytes(pa_run* run, size_t* bytes) {
  if (!run || !bytes) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  *bytes = ck_bytes(d[0]);
  return PA_OK;
}

int pa_checkpoint(pa_run* run, void* host_buf, size_t bytes) {
  if (!run || !host_buf) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  if (d[0].error) return fail(d[0].error, "device: %s (no checkpoint of a failed run)", err_name(d[0].error));
  if (bytes < ck_bytes(d[0])) return fail(PA_ERR_INVALID, "checkpoint buffer too small");
  return ck_write_run(d[0], run->e.st, (char*)host_buf);
}

int pa_restore(pa_run* run, const void* host_buf, size_t bytes) {
  if (!run || !host_buf) return fail(PA_ERR_INVALID, "bad checkpoint arguments");
  Engine& E = run->e;
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  CkHeader h;
  size_t used;
  RunDev D = E.h[0];
  int st = ck_check_run(D, E.st, (const char*)host_buf, bytes, &h, &used);
  if (st != PA_OK) return st;
  st = ck_read_run(D, h, (const char*)host_buf);
  if (st != PA_OK) return st;
  E.h[0] = D;
  PA_CUDA(cudaMemcpy(E.d_runs, &E.h[0], sizeof(RunDev), cudaMemcpyHostToDevice));
  E.host_beta[0] = h.beta;
  E.host_steps = h.step;
  return PA_OK;
}

// A batch checkpoint: this header, then the state of every run in order,
// each in the single-run format above.
struct CkBatchHeader {
  uint64_t magic;
  uint32_t version, n_runs;
  int64_t step;
};
constexpr uint64_t CK_BATCH_MAGIC = 0x5041474233304254ULL;

int pa_batch_checkpoint_bytes(pa_batch* b, size_t* bytes) {
  if (!b || !bytes) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(b->e, d);
  if (st != PA_OK) return st;
  size_t n = sizeof(CkBatchHeader);
  for (const RunDev& D : d) n += ck_bytes(D);
  *bytes = n;
  return PA_OK;
}

int pa_batch_checkpoint(pa_batch* b, void* host_buf, size_t bytes) {
  if (!b || !host_buf) return fail(PA_ERR_INVALID, "NULL argument");
  Engine& E = b->e;
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  size_t n = sizeof(CkBatchHeader);
  for (int r = 0; r < E.n; ++r) {
    if (d[r].error) return fail(d[r].error, "run %d: device: %s (no checkpoint of a failed run)", r,
                                err_name(d[r].error));
    n += ck_bytes(d[r]);
  }
  if (bytes < n) return fail(PA_ERR_INVALID, "checkpoint buffer too small");
  CkBatchHeader bh;
  memset(&bh, 0, sizeof bh);
  bh.magic = CK_BATCH_MAGIC;
  bh.version = 1;
  bh.n_runs = (uint32_t)E.n;
  bh.step = E.host_steps;
  char* p = (char*)host_buf;
  memcpy(p, &bh, sizeof bh);
  p += sizeof bh;
  for (int r = 0; r < E.n; ++r) {
    st = ck_write_run(d[r], E.st, p);
    if (st != PA_OK) return st;
    p += ck_bytes(d[r]);
  }
  return PA_OK;
}

int pa_batch_restore(pa_batch* b, const void* host_buf, size_t bytes) {
  if (!b || !host_buf || bytes < sizeof(CkBatchHeader)) return fail(PA_ERR_INVALID, "bad checkpoint arguments");
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  CkBatchHeader bh;
  memcpy(&bh, host_buf, sizeof bh);
  if (bh.magic != CK_BATCH_MAGIC || bh.version != 1) return fail(PA_ERR_INVALID, "not a batch checkpoint of this library");
  if ((int)bh.n_runs != E.n) return fail(PA_ERR_INVALID, "checkpoint holds %u runs, the batch %d", bh.n_runs, E.n);
  if (bh.step < 0 || bh.step > E.max_steps) return fail(PA_ERR_INVALID, "checkpoint step out of range");
  // check every run before touching any, so that a refused restore leaves the
  // batch as it was
  std::vector<CkHeader> hs(E.n);
  std::vector<size_t> at(E.n);
  size_t off = sizeof bh;
  for (int r = 0; r < E.n; ++r) {
    size_t used;
    int st = ck_check_run(E.h[r], E.st, (const char*)host_buf + off, bytes - off, &hs[r], &used);
    if (st != PA_OK) return fail(st, "run %d: %s", r, last_error_message());
    if (hs[r].step != bh.step) return fail(PA_ERR_INVALID, "run %d: step differs from the batch's", r);
    at[r] = off;
    off += used;
  }
  for (int r = 0; r < E.n; ++r) {
    RunDev D = E.h[r];
    int st = ck_read_run(D, hs[r], (const char*)host_buf + at[r]);
    if (st != PA_OK) return st;
    E.h[r] = D;
    E.host_beta[r] = hs[r].beta;
  }
  PA_CUDA(cudaMemcpy(E.d_runs, E.h.data(), sizeof(RunDev) * E.n, cudaMemcpyHostToDevice));
  E.host_steps = bh.step;
  return PA_OK;
}

}  // extern "C"
