// pa_engine.h -- declarations shared by the host runtime's translation units
// (pa_engine.cu: engine and single runs; pa_checkpoint.cu; pa_batch.cu;
// pa_server.cu): kernel launchers, error helpers, the run geometry, the
// Engine and the entry points of the engine used across them.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "pa.h"
#include "pa_device.cuh"
#include "pa_internal.h"

namespace pa {
cudaError_t set_exp_coefficients();
cudaError_t launch_setup_bonds3d(const int8_t* J, int L, uint32_t* bonds, int W, cudaStream_t st);
cudaError_t launch_setup_bonds1d(const int8_t* J, int N, uint32_t* bonds, int W, cudaStream_t st);
cudaError_t launch_init_state(RunDev* runs, const int32_t* ids, int n, int max_bins, cudaStream_t st);
cudaError_t launch_init_finish(RunDev* runs, const int32_t* ids, int n, cudaStream_t st);
cudaError_t launch_prepare(RunDev* runs, const int32_t* ids, int n, bool ovr, double beta, int theta,
                           int64_t Rt, cudaStream_t st);
cudaError_t launch_copies(RunDev* runs, const Work* table, int nwork, cudaStream_t st);
cudaError_t launch_scan(RunDev* runs, const int32_t* ids, int n, cudaStream_t st);
cudaError_t launch_scatter(RunDev* runs, const Work* table, int nwork, cudaStream_t st);
cudaError_t launch_commit(RunDev* runs, const int32_t* ids, int n, cudaStream_t st);
cudaError_t launch_unpack(const RunDev* runs, int r, int64_t n, int8_t* out, cudaStream_t st);
cudaError_t launch_overlap(const RunDev* a, const RunDev* b, double qcut, unsigned long long* count,
                           unsigned long long* hist, cudaStream_t st);
cudaError_t launch_weighted(int G, int M, const double* x, const double* A, const double* Rw, double* mean,
                            double* fbar, cudaStream_t st);
cudaError_t launch_weighted_pairs(int G, int M, const double* x1, const double* x2, const double* A,
                                  const double* R1, const double* R2, double* mean, double* fbar, cudaStream_t st);
cudaError_t launch_bootstrap(int M, const double* x, const double* A, const double* Rw, int B, uint64_t seed,
                             double* bmean, double* bfbar, cudaStream_t st, int GK = 1);
bool sweep1d_split_ok(int split);
cudaError_t launch_sweep1d(int tpb, int split, RunDev* runs, const Work* table, int nwork, int W, int WR,
                           cudaStream_t st, bool init);
cudaError_t launch_setup_gauss3d(const int32_t* J, int L, int32_t* gJ, int32_t* gS, cudaStream_t st);
cudaError_t launch_gprep_head(RunDev* runs, const int32_t* ids, int n, bool ovr, double beta, int theta, int64_t Rt,
                              cudaStream_t st);
cudaError_t launch_gweights(RunDev* runs, const Work* table, int nwork, cudaStream_t st);
cudaError_t launch_gprep_tail(RunDev* runs, const int32_t* ids, int n, cudaStream_t st);
cudaError_t launch_gather_records(const RunDev* runs, int M, int count, int G, double* x, double* A, double* Rw,
                                  cudaStream_t st);
cudaError_t launch_variance(int G, int M, const double* x, double* var, cudaStream_t st, bool root = false);
cudaError_t launch_check_division(int64_t n, uint64_t seed, unsigned long long* mismatches, cudaStream_t st);
cudaError_t launch_check_exp(int64_t n, uint64_t seed, unsigned long long* out, cudaStream_t st);
cudaError_t launch_check_philox(int64_t n, uint64_t seed, unsigned long long* mismatches);
cudaError_t launch_overlap_hist(const RunDev* runs, const int32_t* ra, const int32_t* rb, int n_pairs, int nbins,
                                unsigned long long* hist, cudaStream_t st);
cudaError_t launch_overlap_pairs(const RunDev* runs, const int32_t* ra, const int32_t* rb, int n_pairs, double qcut,
                                 unsigned long long* count, cudaStream_t st);
cudaError_t launch_box(int tpb, RunDev* runs, const Work* table, int nwork, int WR, int S, cudaStream_t st,
                       bool init);
size_t box_smem_bytes(int WR, int S, int tpb);
cudaError_t launch_gauss_thresholds(int64_t n, double beta, const int32_t* dE, uint32_t* thr);
cudaError_t launch_gauss1d(int tpb, RunDev* runs, const Work* table, int nwork, int WR, cudaStream_t st, bool init);
// Shared memory of the Gaussian chain kernel (thresholds, uniform tables, couplings, columns).
size_t gauss1d_smem_bytes(int tpb, int WR);
#define PA_DECLG(LL)                                                                                \
  cudaError_t launch_gauss3d_L##LL(int tpb, int split, RunDev* runs, const Work* table, int nwork, \
                                   cudaStream_t st, bool init);                                    \
  bool gauss3d_split_ok_L##LL(int split);
PA_DECLG(4)
PA_DECLG(6)
PA_DECLG(8)
PA_DECLG(10)
PA_DECLG(12)
#undef PA_DECLG
#define PA_DECL3(LL)                                                                                \
  cudaError_t launch_sweep3d_L##LL(int tpb, int split, RunDev* runs, const Work* table, int nwork, \
                                   cudaStream_t st, bool init);                                    \
  bool sweep3d_split_ok_L##LL(int split);
PA_DECL3(2)
PA_DECL3(4)
PA_DECL3(6)
PA_DECL3(8)
PA_DECL3(10)
PA_DECL3(12)
PA_DECL3(14)
PA_DECL3(16)
#undef PA_DECL3
}  // namespace pa

using namespace pa;

// errors: the message of the last failing call on this host thread
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);
const char* err_name(int code);
const char* last_error_message();
void clear_last_error();

// Host-side NVTX range (profilers show the annealing steps and each kernel's
// enqueue under these names; without a profiler attached it costs a check).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

#define PA_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

// ---------------------------------------------------------------------------
// geometry and validation
// ---------------------------------------------------------------------------
struct Geometry {
  int dim, L, N, Nb, W, Wr;
  size_t bond_words;
  int model = 0;          // 1: Gaussian couplings (fixed point)
  size_t gj_words = 0;    // Gaussian coupling table: 3D [2][6][WR][SITES]; 1D J[N]
  size_t gs_words = 0;    // 3D per-site coupling sums [2][WR][SITES]; 1D none
  int64_t gC0 = 0;        // sum of all couplings (Gaussian, general boxes)
  // general boxes: extents, periodic axes, lanes per word, colour-c sites per
  // word, used bits of a word, and the per-site tables built on the host
  int bx = 0, by = 0, bz = 0, bk = 0, bsites = 0;
  unsigned bper = 0;
  uint32_t bvalid = 0;
  std::vector<int32_t> box_code, box_J, box_S;
};


// ---------------------------------------------------------------------------
// Engine
// ---------------------------------------------------------------------------
struct Slab {
  void* p = nullptr;
  size_t n = 0;
};

struct LatticeClass {
  int dim, L, W, Wr;
  int model = 0;
  int bx = 0, by = 0, bz = 0, bsites = 0;  // general box (bx > 0)
  unsigned bper = 0;
  int max_tpb = 256;                        // largest block whose shared memory fits
  int tpb;
  int split = 1;     // cubic lattices: threads per replica in the sweep kernel (1, 2, 4, 8)
  std::vector<int32_t> runs;
  Work* d_table = nullptr;
  int nwork = 0;
};

struct Engine {
  int device = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  pa_alloc_fn fa = nullptr;
  pa_free_fn ff = nullptr;
  void* actx = nullptr;
  std::vector<Slab> slabs;
  int n = 0;
  std::vector<RunDev> h;           // host copies of the static part
  std::vector<int64_t> R0;
  RunDev* d_runs = nullptr;
  std::vector<LatticeClass> cls;
  Work* d_copy_table = nullptr;
  int n_copy_work = 0;
  int max_bins = 0;
  int max_steps = 0;
  int64_t host_steps = 0;          // steps queued so far (host view)
  std::vector<double> host_beta;   // last requested beta per run (host view)
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  int64_t graph_kernels = 0;   // kernels one replay of the graph launches
  int graph_prof_stride = 0;   // sweep-timing stride the graph was captured with (0: untimed)
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> graph_ev;  // timing events recorded by the graph
  bool graph_pending = false;  // a timed replay whose events have not been read yet
  bool capturing = false;
  int model = 0;  // all runs of an engine share one coupling model
  // measurement hooks
  bool prof = false;
  int prof_stride = 1;       // time every prof_stride-th sweep launch
  int64_t prof_seen = 0;     // sweep launches since timing was enabled
  double prof_ms_acc = 0.0;  // timed milliseconds and launches read from graph replays
  int64_t prof_n_acc = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  int64_t launches = 0;

  void* dalloc(size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    void* p = nullptr;
    if (fa) {
      p = fa(bytes, (void*)st, actx);
    } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    if (p) slabs.push_back({p, bytes});
    return p;
  }
  // Return scratch from dalloc before the engine is released.
  void dfree(void* p, size_t bytes) {
    bytes = (bytes + 255) / 256 * 256;
    for (size_t i = 0; i < slabs.size(); ++i)
      if (slabs[i].p == p) {
        slabs.erase(slabs.begin() + i);
        break;
      }
    if (ff) ff(p, bytes, (void*)st, actx);
    else cudaFreeAsync(p, st);
  }
  // The schedule graph and the timing events it records (they live as long
  // as the graph).
  void drop_graph() {
    if (graph) {
      cudaGraphExecDestroy(graph);
      graph = nullptr;
    }
    for (auto& p : graph_ev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    graph_ev.clear();
    graph_steps = -1;
    graph_kernels = 0;
    graph_prof_stride = 0;
    graph_pending = false;
  }
  // After a synchronisation: add the sweep times of the last timed replay.
  void harvest_graph_timing() {
    if (!graph_pending) return;
    for (auto& p : graph_ev) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, p.first, p.second) == cudaSuccess) prof_ms_acc += ms;
      else cudaGetLastError();  // a timing that cannot be read must not fail a later launch check
    }
    prof_n_acc += (int64_t)graph_ev.size();
    graph_pending = false;
  }
  void release() {
    for (auto& p : prof_ev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    prof_ev.clear();
    drop_graph();
    for (auto& s : slabs) {
      if (ff) ff(s.p, s.n, (void*)st, actx);
      else cudaFreeAsync(s.p, st);
    }
    slabs.clear();
    if (!ff) cudaStreamSynchronize(st);
    if (own_stream && st) cudaStreamDestroy(st);
    st = nullptr;
  }
};

struct pa_run {
  Engine e;
};
struct pa_batch {
  Engine e;
};

// shared engine functions (pa_engine.cu)
int ensure_device_constants(int dev);
int make_geometry(const int8_t* J, int L, int dim, Geometry* g);
int64_t default_capacity(int64_t R0);
size_t run_slab_bytes(const Geometry& g, int64_t cap, int max_steps);
int setup_run(char* base, const Geometry& g, const pa_run_spec& s, int64_t cap, int max_steps,
              cudaStream_t st, RunDev* out);
int default_tpb(int dim, int L);
void set_default_launch(LatticeClass& c, int tpb_opt, int split_opt);
bool split_supported(const LatticeClass& c, int split);
bool tpb_supported(const LatticeClass& c, int tpb);
int launch_class_on(RunDev* runs, cudaStream_t st, const LatticeClass& c, const Work* table, int nwork,
                    bool init, int tpb);
int launch_class(Engine& E, const LatticeClass& c, const Work* table, int nwork, bool init, int tpb);
int prepare_class_launches(RunDev* runs, cudaStream_t st, const LatticeClass& c);
int build_class_table(Engine& E, LatticeClass& c);
int engine_create(Engine& E, int n_runs, const pa_run_spec* specs, const pa_opts* opts);
int engine_prep(Engine& E, bool ovr, double beta, int theta, int64_t Rt);
int engine_init_population(Engine& E);
int engine_fetch(Engine& E, std::vector<RunDev>& out);
int engine_sync(Engine& E, int32_t* errors);
int engine_copy_spins(Engine& E, int r, int8_t* host_dst, int64_t max_replicas, int64_t* n);
int engine_run_schedule(Engine& E, int n_steps, const double* betas, int per_run, const int32_t* thetas,
                        const int64_t* R_targets, int use_graph);
