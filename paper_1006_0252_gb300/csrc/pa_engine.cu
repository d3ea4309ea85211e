// pa_engine.cu -- host runtime behind the C ABI of include/pa.h.
//
// An Engine owns a set of annealing runs on one GPU: one device-memory slab
// per run, the RunDev array, and the work tables that map kernel blocks to
// (run, slot range).  Single runs (pa_run) and batches (pa_batch) are both
// Engines; every step enqueues the same seven launches (prepare, copies,
// scan, scatter, one sweep launch per lattice class, commit) with no host
// synchronisation, so a batch schedule can be captured as one CUDA graph.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

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
cudaError_t launch_bootstrap(int M, const double* x, const double* A, const double* Rw, int B, uint64_t seed,
                             double* bmean, double* bfbar, cudaStream_t st, int GK = 1);
cudaError_t launch_sweep1d(int tpb, RunDev* runs, const Work* table, int nwork, int W, int WR,
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
cudaError_t launch_overlap_pairs(const RunDev* runs, const int32_t* ra, const int32_t* rb, int n_pairs, double qcut,
                                 unsigned long long* count, cudaStream_t st);
cudaError_t launch_box(int tpb, RunDev* runs, const Work* table, int nwork, int WR, int S, cudaStream_t st,
                       bool init);
size_t box_smem_bytes(int WR, int S, int tpb);
cudaError_t launch_gauss1d(int tpb, RunDev* runs, const Work* table, int nwork, int WR, cudaStream_t st, bool init);
#define PA_DECLG(LL)                                                                      \
  cudaError_t launch_gauss3d_L##LL(int tpb, RunDev* runs, const Work* table, int nwork, \
                                   cudaStream_t st, bool init, int64_t wave);           \
  int64_t gauss3d_wave_L##LL(int tpb);
PA_DECLG(4)
PA_DECLG(6)
PA_DECLG(8)
PA_DECLG(10)
PA_DECLG(12)
#undef PA_DECLG
#define PA_DECL3(LL)                                                                      \
  cudaError_t launch_sweep3d_L##LL(int tpb, RunDev* runs, const Work* table, int nwork, \
                                   cudaStream_t st, bool init, int64_t wave);           \
  int64_t sweep3d_wave_L##LL(int tpb);
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

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

static int cuda_fail(cudaError_t e, const char* where) {
  return fail(PA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define PA_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

static const char* err_name(int code) {
  switch (code) {
    case PA_OK: return "ok";
    case PA_ERR_INVALID: return "invalid argument or schedule";
    case PA_ERR_OOM: return "device allocation refused";
    case PA_ERR_CAPACITY: return "population would exceed its capacity R_cap";
    case PA_ERR_EXTINCT: return "population died out (no replica resampled)";
    case PA_ERR_TIMEOUT: return "bounded wait ran out";
    case PA_ERR_CUDA: return "CUDA error";
    case PA_ERR_UNSUPPORTED: return "lattice shape without a compiled kernel";
    default: return "unknown error";
  }
}

static std::mutex g_coef_mu;
static bool g_coef_ready[64];

static int ensure_device_constants(int dev) {
  std::lock_guard<std::mutex> lk(g_coef_mu);
  if (dev < 0 || dev >= 64) return fail(PA_ERR_CUDA, "device index %d out of range", dev);
  if (!g_coef_ready[dev]) {
    PA_CUDA(set_exp_coefficients());
    g_coef_ready[dev] = true;
  }
  return PA_OK;
}

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

// Largest general box: its per-site tables (28 words per site pair) stay in
// shared memory next to the spin columns.
constexpr int MAX_BOX_SITES = 2048;
constexpr size_t SMEM_LIMIT = 227 * 1024 - 256;

// General Lx x Ly x Lz box (periodic axis d where bit d of mask is set),
// either coupling model; J is int8 (model 0) or int32 fixed point (model 1)
// in the [3][N] layout.  The bond set, colouring and validation follow the
// nearest-neighbour lattice of Sec. 4: a bond (i, i + e_d) exists unless the
// axis is open and i is on its last plane, or its coupling is 0; bonds must
// join sites of different colours (bipartite, no self-loops).
static int make_geometry_box(const void* Jv, int model, const int Ls[3], unsigned mask, Geometry* g) {
  if (!Jv || !Ls) return fail(PA_ERR_INVALID, "couplings and extents must not be NULL");
  const int Lx = Ls[0], Ly = Ls[1], Lz = Ls[2];
  if (Lx < 2 || Lx > 32 || (Lx & 1) || Ly < 1 || Lz < 1)
    return fail(PA_ERR_INVALID, "box extents: Lx even in 2..32, Ly, Lz >= 1 (got %d x %d x %d)", Lx, Ly, Lz);
  const int64_t N64 = (int64_t)Lx * Ly * Lz;
  if (N64 > MAX_BOX_SITES) return fail(PA_ERR_UNSUPPORTED, "general boxes up to %d sites", MAX_BOX_SITES);
  const int N = (int)N64;
  int k = 1;
  for (int d = Lz; d >= 1; --d)
    if (Lz % d == 0 && d * Lx <= 32) {
      k = d;
      break;
    }
  const int G = Lz / k, WR = Ly * G, S = k * Lx / 2;
  g->dim = 3;
  g->L = Lx;
  g->N = N;
  g->Wr = WR;
  g->W = (WR + 3) / 4 * 4;
  g->model = model;
  g->bond_words = 0;
  g->bx = Lx;
  g->by = Ly;
  g->bz = Lz;
  g->bk = k;
  g->bsites = S;
  g->bper = mask & 7u;
  g->bvalid = k * Lx == 32 ? 0xFFFFFFFFu : ((1u << (k * Lx)) - 1u);
  const int plane = WR * S;
  g->gj_words = (size_t)12 * plane;
  g->gs_words = (size_t)2 * plane;
  g->box_code.assign((size_t)14 * plane, 0);
  g->box_J.assign((size_t)12 * plane, 0);
  g->box_S.assign((size_t)2 * plane, 0);
  auto coupling = [&](int d, int64_t i) -> int64_t {
    return model == 1 ? (int64_t)((const int32_t*)Jv)[d * N64 + i] : (int64_t)((const int8_t*)Jv)[d * N64 + i];
  };
  const int ext[3] = {Lx, Ly, Lz};
  auto code_of = [&](int x, int y, int z) { return 32 * (y * G + z % G) + (z / G) * Lx + x; };
  int64_t nb = 0, c0 = 0, sabs = 0;
  // validate every stored bond once (from its "+" end)
  for (int d = 0; d < 3; ++d)
    for (int z = 0; z < Lz; ++z)
      for (int y = 0; y < Ly; ++y)
        for (int x = 0; x < Lx; ++x) {
          const int c[3] = {x, y, z};
          if (c[d] == ext[d] - 1 && !((mask >> d) & 1u)) continue;
          const int64_t i = x + (int64_t)Lx * (y + (int64_t)Ly * z);
          const int64_t J = coupling(d, i);
          if (J == 0) continue;
          if (model == 0 && J != 1 && J != -1) return fail(PA_ERR_INVALID, "+-1 couplings must be -1, 0 or 1");
          if (model == 1 && (J > (1 << 18) || J < -(1 << 18)))
            return fail(PA_ERR_INVALID, "Gaussian coupling outside +-2^18 (fixed point 2^-15)");
          if (c[d] == ext[d] - 1 && (ext[d] == 1 || (ext[d] & 1)))
            return fail(PA_ERR_INVALID, "bond across a periodic axis of odd length %d (not bipartite)", ext[d]);
          ++nb;
          c0 += J;
          sabs += J < 0 ? -J : J;
        }
  if (sabs >= (1LL << 31)) return fail(PA_ERR_INVALID, "sum of |J| exceeds the 32-bit energy range");
  for (int c = 0; c < 2; ++c)
    for (int w = 0; w < WR; ++w)
      for (int m = 0; m < S; ++m) {
        const int y = w / G, gg = w % G, j = m / (Lx / 2), xh = m % (Lx / 2);
        const int z = gg + j * G;
        const int x = 2 * xh + ((c + y + z) & 1);
        const int own = code_of(x, y, z);
        const int base = w * S + m;
        g->box_code[(size_t)(c * 7) * plane + base] = own;
        int32_t sum = 0;
        for (int d = 0; d < 3; ++d) {
          for (int sgn = 0; sgn < 2; ++sgn) {  // 0: + neighbour, 1: - neighbour
            int n[3] = {x, y, z};
            const bool edge = sgn == 0 ? n[d] == ext[d] - 1 : n[d] == 0;
            n[d] = sgn == 0 ? (n[d] + 1) % ext[d] : (n[d] + ext[d] - 1) % ext[d];
            int64_t J = 0;
            if (!edge || ((mask >> d) & 1u)) {
              // the bond is stored at its "+" end: this site (sgn 0) or the neighbour (sgn 1)
              const int sx = sgn == 0 ? x : n[0], sy = sgn == 0 ? y : n[1], sz = sgn == 0 ? z : n[2];
              J = coupling(d, sx + (int64_t)Lx * (sy + (int64_t)Ly * sz));
            }
            const int slot = 2 * d + sgn;
            g->box_code[(size_t)(c * 7 + 1 + slot) * plane + base] = J != 0 ? code_of(n[0], n[1], n[2]) : own;
            g->box_J[(size_t)(c * 6 + slot) * plane + base] = (int32_t)J;
            sum += (int32_t)J;
          }
        }
        g->box_S[(size_t)c * plane + base] = sum;
      }
  g->gC0 = c0;
  g->Nb = model == 1 ? 0 : (int)nb;
  if (box_smem_bytes(WR, S, 32) > SMEM_LIMIT)
    return fail(PA_ERR_UNSUPPORTED, "box %d x %d x %d does not fit one block's shared memory", Lx, Ly, Lz);
  return PA_OK;
}

// Longest chain: a block of 256 replicas keeps its spins and the chain's
// couplings in shared memory.
constexpr int MAX_CHAIN = 4096;

static bool have_gauss_kernel(int L) { return L == 4 || L == 6 || L == 8 || L == 10 || L == 12; }

static int make_geometry_gauss(const int32_t* J, int L, int dim, Geometry* g) {
  if (!J) return fail(PA_ERR_INVALID, "couplings must not be NULL");
  const int64_t nJ = dim == 3 ? 3LL * L * L * L : (int64_t)L;
  if (dim == 3) {
    if (L < 2 || (L & 1)) return fail(PA_ERR_INVALID, "3D edge L=%d must be even", L);
    if (!have_gauss_kernel(L)) return fail(PA_ERR_UNSUPPORTED, "no Gaussian 3D kernel for L=%d (4..12 even)", L);
    const int K = lanes_for(L), G = L / K;
    g->dim = 3;
    g->L = L;
    g->N = L * L * L;
    g->Wr = L * G;
    g->W = (g->Wr + 3) / 4 * 4;
    const size_t sp = (size_t)(((K * L / 2) + 3) & ~3);  // ranks per word, padded to 16-byte rows
    g->gj_words = 12 * g->Wr * sp;
    g->gs_words = 2 * g->Wr * sp;
  } else if (dim == 1) {
    if (L < 2) return fail(PA_ERR_INVALID, "chain length %d must be >= 2", L);
    if (L > MAX_CHAIN) return fail(PA_ERR_UNSUPPORTED, "chain length %d above %d", L, MAX_CHAIN);
    if ((L & 1) && J[L - 1] != 0) return fail(PA_ERR_INVALID, "odd periodic chain is not bipartite");
    g->dim = 1;
    g->L = L;
    g->N = L;
    g->Wr = (L + 31) / 32;
    g->W = (g->Wr + 3) / 4 * 4;
    g->gj_words = (size_t)L;
    g->gs_words = 0;
  } else {
    return fail(PA_ERR_UNSUPPORTED, "Gaussian couplings: dim must be 1 or 3");
  }
  g->Nb = 0;  // no energy histogram for continuous couplings
  g->bond_words = 0;
  g->model = 1;
  int64_t sabs = 0, c0 = 0;
  for (int64_t i = 0; i < nJ; ++i) {
    if (J[i] > (1 << 18) || J[i] < -(1 << 18))
      return fail(PA_ERR_INVALID, "Gaussian coupling %lld outside +-2^18 (fixed point 2^-15)", (long long)i);
    sabs += J[i] < 0 ? -(int64_t)J[i] : J[i];
    c0 += J[i];
  }
  if (sabs >= (1LL << 31)) return fail(PA_ERR_INVALID, "sum of |J| exceeds the 32-bit energy range");
  g->gC0 = c0;
  return PA_OK;
}

static bool have_3d_kernel(int L) {
  return L == 2 || L == 4 || L == 6 || L == 8 || L == 10 || L == 12 || L == 14 || L == 16;
}

static int make_geometry(const int8_t* J, int L, int dim, Geometry* g) {
  if (!J) return fail(PA_ERR_INVALID, "couplings must not be NULL");
  g->dim = dim;
  g->L = L;
  if (dim == 3) {
    if (L < 2 || (L & 1)) return fail(PA_ERR_INVALID, "3D edge L=%d must be even and >= 2 (checkerboard)", L);
    if (!have_3d_kernel(L)) return fail(PA_ERR_UNSUPPORTED, "no 3D kernel for L=%d (even L in 2..16)", L);
    const int K = lanes_for(L), G = L / K;
    g->N = L * L * L;
    g->Wr = L * G;
    g->W = (g->Wr + 3) / 4 * 4;
    for (int64_t i = 0; i < 3LL * g->N; ++i)
      if (J[i] != 1 && J[i] != -1) return fail(PA_ERR_INVALID, "3D couplings must be +-1 (entry %lld)", (long long)i);
    g->Nb = 3 * g->N;
    g->bond_words = 6 * (size_t)g->W;
  } else if (dim == 1) {
    if (L < 2) return fail(PA_ERR_INVALID, "chain length %d must be >= 2", L);
    if (L > MAX_CHAIN) return fail(PA_ERR_UNSUPPORTED, "chain length %d above %d", L, MAX_CHAIN);
    g->N = L;
    g->Wr = (L + 31) / 32;
    g->W = (g->Wr + 3) / 4 * 4;
    int nb = 0;
    for (int i = 0; i < L; ++i) {
      if (J[i] < -1 || J[i] > 1) return fail(PA_ERR_INVALID, "chain couplings must be in {-1,0,1}");
      nb += J[i] != 0;
    }
    if ((L & 1) && J[L - 1] != 0) return fail(PA_ERR_INVALID, "odd periodic chain is not bipartite");
    g->Nb = nb;
    g->bond_words = 4 * (size_t)g->W;
  } else {
    return fail(PA_ERR_INVALID, "dim must be 1 or 3 (got %d)", dim);
  }
  return PA_OK;
}

static int64_t default_capacity(int64_t R0) {
  int64_t r = (int64_t)std::floor(std::sqrt((double)R0));
  while (r * r > R0) --r;
  while ((r + 1) * (r + 1) <= R0) ++r;
  if (r * r < R0) ++r;
  return R0 + 10 * r + 64;
}


// Device bytes of one run: both populations, energies, histograms, coupling
// masks, resampling scratch, per-bin tables, schedule and record.
struct SlabPart {
  void** dst;
  size_t bytes;
};
static const int N_SLAB_PARTS = 33;

static size_t slab_parts(RunDev& d, const Geometry& g, int64_t cap_, int max_steps, SlabPart* parts) {
  const size_t cap = (size_t)cap_, nb = (size_t)(g.Nb + 1), ms = (size_t)max_steps;
  const size_t nch = (size_t)((cap_ + CHUNK - 1) / CHUNK);
  SlabPart p[] = {
      {(void**)&d.spins[0], cap * g.W * 4}, {(void**)&d.spins[1], cap * g.W * 4},
      {(void**)&d.E[0], cap * 4},           {(void**)&d.E[1], cap * 4},
      {(void**)&d.hist[0], nb * 4},         {(void**)&d.hist[1], nb * 4},
      {(void**)&d.bonds, g.bond_words * 4}, {(void**)&d.copies, cap * 4},
      {(void**)&d.src, cap * 4},            {(void**)&d.chunk_sum, nch * 8},
      {(void**)&d.chunk_off, nch * 8},      {(void**)&d.occ, nb * 4},
      {(void**)&d.bin_w, nb * 8},
      {(void**)&d.bin_am, nb * 8},          {(void**)&d.bin_p0, nb * 8},
      {(void**)&d.bin_m, nb * 8},           {(void**)&d.sched_beta, ms * 8},
      {(void**)&d.bin_thr, g.model ? 0 : nb * POISSON_TAB * 8}, {(void**)&d.bin_end, g.model ? 0 : nb * 16},
      {(void**)&d.sched_theta, ms * 4},     {(void**)&d.sched_R, ms * 8},
      {(void**)&d.rec_beta, (ms + 1) * 8},  {(void**)&d.rec_lnQ, (ms + 1) * 8},
      {(void**)&d.rec_mbF, (ms + 1) * 8},   {(void**)&d.rec_R, (ms + 1) * 8},
      {(void**)&d.rec_sumE, (ms + 1) * 8},  {(void**)&d.rec_sumE2, (ms + 1) * 8},
      {(void**)&d.gJ, g.gj_words * 4}, {(void**)&d.gS, g.gs_words * 4},
      {(void**)&d.box_code, g.box_code.size() * 4},
      {(void**)&d.w_rep, g.model ? cap * 8 : 0}, {(void**)&d.chunk_q, g.model ? nch * 8 : 0},
      {nullptr, (size_t)(g.dim == 3 ? 3 * g.N : g.N) * (g.model ? 4 : 1)},  // couplings
  };
  const size_t n = sizeof(p) / sizeof(p[0]);
  static_assert(sizeof(p) / sizeof(p[0]) == N_SLAB_PARTS, "slab part count");
  if (parts)
    for (size_t i = 0; i < n; ++i) parts[i] = p[i];
  size_t total = 0;
  for (size_t i = 0; i < n; ++i) total += (p[i].bytes + 255) / 256 * 256;
  return total;
}

static size_t run_slab_bytes(const Geometry& g, int64_t cap, int max_steps) {
  RunDev d;
  return slab_parts(d, g, cap, max_steps, nullptr);
}

// Carve the slab, upload the couplings, build the coupling masks and fill the
// static part of the run record (population not yet initialised).
static int setup_run(char* base, const Geometry& g, const pa_run_spec& s, int64_t cap, int max_steps,
                     cudaStream_t st, RunDev* out) {
  RunDev d;
  memset(&d, 0, sizeof d);
  SlabPart parts[N_SLAB_PARTS];
  slab_parts(d, g, cap, max_steps, parts);
  size_t off = 0;
  int8_t* dJ = nullptr;
  for (int i = 0; i < N_SLAB_PARTS; ++i) {
    if (parts[i].dst) *parts[i].dst = base + off;
    else dJ = (int8_t*)(base + off);
    off += (parts[i].bytes + 255) / 256 * 256;
  }
  d.seed = s.seed;
  d.dim = g.dim;
  d.L = g.L;
  d.N = g.N;
  d.Nb = g.Nb;
  d.nbins = g.Nb + 1;
  d.W = g.W;
  d.Wr = g.Wr;
  d.R_cap = cap;
  d.max_steps = max_steps;
  d.n_chunks = (int32_t)((cap + CHUNK - 1) / CHUNK);
  d.one = 1;
  d.n_sched = 0;
  d.R = s.R0;
  d.model = g.model;
  d.gC0 = (int32_t)g.gC0;
  d.bx = g.bx;
  d.by = g.by;
  d.bz = g.bz;
  d.bk = g.bk;
  d.bsites = g.bsites;
  d.bvalid = g.bvalid;
  const size_t jbytes = (size_t)(g.dim == 3 ? 3 * g.N : g.N) * (g.model ? 4 : 1);
  const void* hJ = g.model ? (const void*)s.gauss_couplings : (const void*)s.couplings;
  PA_CUDA(cudaMemcpyAsync(dJ, hJ, jbytes, cudaMemcpyHostToDevice, st));
  PA_CUDA(cudaMemsetAsync(d.spins[0], 0, (size_t)cap * g.W * 4, st));
  if (g.bx > 0) {
    PA_CUDA(cudaMemcpyAsync(d.box_code, g.box_code.data(), 4 * g.box_code.size(), cudaMemcpyHostToDevice, st));
    PA_CUDA(cudaMemcpyAsync(d.gJ, g.box_J.data(), 4 * g.box_J.size(), cudaMemcpyHostToDevice, st));
    PA_CUDA(cudaMemcpyAsync(d.gS, g.box_S.data(), 4 * g.box_S.size(), cudaMemcpyHostToDevice, st));
  } else if (g.model == 1 && g.dim == 1) {
    PA_CUDA(cudaMemcpyAsync(d.gJ, hJ, jbytes, cudaMemcpyHostToDevice, st));
  } else if (g.model == 1) {
    PA_CUDA(launch_setup_gauss3d((const int32_t*)dJ, g.L, d.gJ, d.gS, st));
  } else if (g.dim == 3) {
    PA_CUDA(launch_setup_bonds3d(dJ, g.L, d.bonds, g.W, st));
  } else {
    PA_CUDA(launch_setup_bonds1d(dJ, g.N, d.bonds, g.W, st));
  }
  *out = d;
  return PA_OK;
}

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
  int64_t wave = 0;  // one-run +-1 cubic class: replicas the sweep kernel holds resident (wave tail split)
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

static int default_tpb(int dim, int L) {
  if (dim == 1) return 64;
  return L >= 12 ? 64 : 128;
}

static int launch_class_on(RunDev* runs, cudaStream_t st, const LatticeClass& c, const Work* table, int nwork,
                           bool init, int tpb) {
  cudaError_t err;
  if (c.bx > 0) {
    if (tpb > c.max_tpb) {
      if (nwork <= 0) return PA_OK;  // nothing to set up for a block size that cannot run
      return fail(PA_ERR_UNSUPPORTED, "block of %d threads exceeds shared memory for this box", tpb);
    }
    err = launch_box(tpb, runs, table, nwork, c.Wr, c.bsites, st, init);
  } else if (c.model == 1 && c.dim == 1) {
    err = launch_gauss1d(tpb, runs, table, nwork, c.Wr, st, init);
  } else if (c.model == 1) {
    switch (c.L) {
      case 4: err = launch_gauss3d_L4(tpb, runs, table, nwork, st, init, c.wave); break;
      case 6: err = launch_gauss3d_L6(tpb, runs, table, nwork, st, init, c.wave); break;
      case 8: err = launch_gauss3d_L8(tpb, runs, table, nwork, st, init, c.wave); break;
      case 10: err = launch_gauss3d_L10(tpb, runs, table, nwork, st, init, c.wave); break;
      case 12: err = launch_gauss3d_L12(tpb, runs, table, nwork, st, init, c.wave); break;
      default: return fail(PA_ERR_UNSUPPORTED, "no Gaussian kernel for L=%d", c.L);
    }
  } else if (c.dim == 1) {
    err = launch_sweep1d(tpb, runs, table, nwork, c.W, c.Wr, st, init);
  } else {
    switch (c.L) {
      case 2: err = launch_sweep3d_L2(tpb, runs, table, nwork, st, init, c.wave); break;
      case 4: err = launch_sweep3d_L4(tpb, runs, table, nwork, st, init, c.wave); break;
      case 6: err = launch_sweep3d_L6(tpb, runs, table, nwork, st, init, c.wave); break;
      case 8: err = launch_sweep3d_L8(tpb, runs, table, nwork, st, init, c.wave); break;
      case 10: err = launch_sweep3d_L10(tpb, runs, table, nwork, st, init, c.wave); break;
      case 12: err = launch_sweep3d_L12(tpb, runs, table, nwork, st, init, c.wave); break;
      case 14: err = launch_sweep3d_L14(tpb, runs, table, nwork, st, init, c.wave); break;
      case 16: err = launch_sweep3d_L16(tpb, runs, table, nwork, st, init, c.wave); break;
      default: return fail(PA_ERR_UNSUPPORTED, "no kernel for L=%d", c.L);
    }
  }
  if (err != cudaSuccess) return cuda_fail(err, "sweep kernel launch");
  return PA_OK;
}

static int launch_class(Engine& E, const LatticeClass& c, const Work* table, int nwork, bool init, int tpb) {
  return launch_class_on(E.d_runs, E.st, c, table, nwork, init, tpb);
}

static int64_t sweep3d_wave(int L, int tpb) {
  switch (L) {
    case 2: return sweep3d_wave_L2(tpb);
    case 4: return sweep3d_wave_L4(tpb);
    case 6: return sweep3d_wave_L6(tpb);
    case 8: return sweep3d_wave_L8(tpb);
    case 10: return sweep3d_wave_L10(tpb);
    case 12: return sweep3d_wave_L12(tpb);
    case 14: return sweep3d_wave_L14(tpb);
    case 16: return sweep3d_wave_L16(tpb);
    default: return 0;
  }
}

static int64_t gauss3d_wave(int L, int tpb) {
  switch (L) {
    case 4: return gauss3d_wave_L4(tpb);
    case 6: return gauss3d_wave_L6(tpb);
    case 8: return gauss3d_wave_L8(tpb);
    case 10: return gauss3d_wave_L10(tpb);
    case 12: return gauss3d_wave_L12(tpb);
    default: return 0;
  }
}

static int build_class_table(Engine& E, LatticeClass& c) {
  // a class of one cubic run may split its wave tail (k_sweep3d, k_sweep_gauss3d)
  c.wave = 0;
  if (c.runs.size() == 1 && c.dim == 3 && c.bx == 0)
    c.wave = c.model == 0 ? sweep3d_wave(c.L, c.tpb) : gauss3d_wave(c.L, c.tpb);
  std::vector<Work> t;
  for (int32_t r : c.runs)
    for (int64_t f = 0; f < E.h[r].R_cap; f += c.tpb) t.push_back({r, (int32_t)f});
  c.nwork = (int)t.size();
  c.d_table = (Work*)E.dalloc(sizeof(Work) * std::max<size_t>(t.size(), 1));
  if (!c.d_table) return fail(PA_ERR_OOM, "work table allocation refused");
  if (!t.empty()) PA_CUDA(cudaMemcpyAsync(c.d_table, t.data(), sizeof(Work) * t.size(), cudaMemcpyHostToDevice, E.st));
  PA_CUDA(cudaStreamSynchronize(E.st));
  return PA_OK;
}

static int engine_init_population(Engine& E);

// model 0: specs[r].couplings are int8 (+-1 / 0); model 1: they point to
// int32 fixed-point Gaussian couplings (J = J_q 2^-15).
static int engine_create(Engine& E, int n_runs, const pa_run_spec* specs, const pa_opts* opts) {
  if (n_runs < 1 || !specs) return fail(PA_ERR_INVALID, "need at least one run");
  const int model = specs[0].gauss_couplings ? 1 : 0;
  for (int r = 1; r < n_runs; ++r)
    if ((specs[r].gauss_couplings ? 1 : 0) != model)
      return fail(PA_ERR_INVALID, "runs of one batch must share the coupling model");
  E.model = model;
  PA_CUDA(cudaGetDevice(&E.device));
  int st = ensure_device_constants(E.device);
  if (st != PA_OK) return st;
  E.st = opts ? (cudaStream_t)opts->stream : nullptr;
  E.fa = opts ? opts->alloc : nullptr;
  E.ff = opts ? opts->free : nullptr;
  E.actx = opts ? opts->alloc_ctx : nullptr;
  if ((E.fa == nullptr) != (E.ff == nullptr)) return fail(PA_ERR_INVALID, "alloc and free hooks come together");
  E.max_steps = (opts && opts->max_steps > 0) ? opts->max_steps : 4096;
  const int tpb_opt = opts ? opts->threads_per_block : 0;
  if (tpb_opt != 0 && tpb_opt != 32 && tpb_opt != 64 && tpb_opt != 128 && tpb_opt != 256)
    return fail(PA_ERR_INVALID, "threads_per_block must be 0, 32, 64, 128 or 256");
  E.n = n_runs;
  E.h.resize(n_runs);
  E.R0.resize(n_runs);
  E.host_beta.assign(n_runs, 0.0);
  std::vector<Geometry> geo(n_runs);
  for (int r = 0; r < n_runs; ++r) {
    const pa_run_spec& s = specs[r];
    if (s.dim == 3 && s.Ls[0] > 0)
      st = make_geometry_box(model == 1 ? (const void*)s.gauss_couplings : (const void*)s.couplings, model, s.Ls,
                             s.periodic_mask, &geo[r]);
    else
      st = model == 1 ? make_geometry_gauss(s.gauss_couplings, s.L, s.dim, &geo[r])
                      : make_geometry(s.couplings, s.L, s.dim, &geo[r]);
    if (st != PA_OK) return st;
    if (s.R0 < 1) return fail(PA_ERR_INVALID, "R0 must be >= 1");
    int64_t cap = s.R_cap > 0 ? s.R_cap : ((opts && opts->R_cap > 0 && n_runs == 1) ? opts->R_cap : default_capacity(s.R0));
    if (cap < s.R0) return fail(PA_ERR_INVALID, "R_cap %lld below R0 %lld", (long long)cap, (long long)s.R0);
    if (cap > 0x7FFFFF00LL) return fail(PA_ERR_INVALID, "R_cap too large");
    E.R0[r] = s.R0;
  }
  if (E.st == nullptr) {
    // a private stream: graph capture needs a non-default stream
    PA_CUDA(cudaStreamCreateWithFlags(&E.st, cudaStreamNonBlocking));
    E.own_stream = true;
  }
  // per-run slabs
  for (int r = 0; r < n_runs; ++r) {
    const pa_run_spec& s = specs[r];
    const int64_t cap = s.R_cap > 0 ? s.R_cap
                                     : ((opts && opts->R_cap > 0 && n_runs == 1) ? opts->R_cap : default_capacity(s.R0));
    RunDev d;
    const size_t total = run_slab_bytes(geo[r], cap, E.max_steps);
    char* base = (char*)E.dalloc(total);
    if (!base) return fail(PA_ERR_OOM, "device allocation of %zu bytes refused (run %d)", total, r);
    st = setup_run(base, geo[r], s, cap, E.max_steps, E.st, &d);
    if (st != PA_OK) return st;
    E.max_bins = std::max(E.max_bins, d.nbins);
    E.h[r] = d;
  }
  E.d_runs = (RunDev*)E.dalloc(sizeof(RunDev) * n_runs);
  if (!E.d_runs) return fail(PA_ERR_OOM, "run table allocation refused");
  PA_CUDA(cudaMemcpyAsync(E.d_runs, E.h.data(), sizeof(RunDev) * n_runs, cudaMemcpyHostToDevice, E.st));
  // work tables
  std::vector<Work> ct;
  for (int r = 0; r < n_runs; ++r)
    for (int64_t f = 0; f < E.h[r].R_cap; f += CHUNK) ct.push_back({r, (int32_t)f});
  E.n_copy_work = (int)ct.size();
  E.d_copy_table = (Work*)E.dalloc(sizeof(Work) * ct.size());
  if (!E.d_copy_table) return fail(PA_ERR_OOM, "work table allocation refused");
  PA_CUDA(cudaMemcpyAsync(E.d_copy_table, ct.data(), sizeof(Work) * ct.size(), cudaMemcpyHostToDevice, E.st));
  for (int r = 0; r < n_runs; ++r) {
    const RunDev& d = E.h[r];
    const Geometry& gr = geo[r];
    auto it = std::find_if(E.cls.begin(), E.cls.end(), [&](const LatticeClass& c) {
      return c.dim == d.dim && c.L == d.L && c.model == d.model && c.bx == gr.bx && c.by == gr.by &&
             c.bz == gr.bz && c.bper == gr.bper;
    });
    if (it == E.cls.end()) {
      LatticeClass c;
      c.dim = d.dim;
      c.L = d.L;
      c.model = d.model;
      c.bx = gr.bx;
      c.by = gr.by;
      c.bz = gr.bz;
      c.bper = gr.bper;
      c.bsites = gr.bsites;
      if (gr.bx > 0) {
        c.max_tpb = 32;
        for (int t = 256; t >= 32; t >>= 1)
          if (box_smem_bytes(d.Wr, gr.bsites, t) <= SMEM_LIMIT) {
            c.max_tpb = t;
            break;
          }
      }
      c.W = d.W;
      c.Wr = d.Wr;
      c.tpb = tpb_opt ? tpb_opt : (gr.bx > 0 ? std::min(64, c.max_tpb) : default_tpb(d.dim, d.L));
      E.cls.push_back(c);
      it = E.cls.end() - 1;
    }
    it->runs.push_back(r);
  }
  for (auto& c : E.cls) {
    st = build_class_table(E, c);
    if (st != PA_OK) return st;
    // set the dynamic shared-memory limits of every block size now, outside
    // any stream capture
    const int cands[] = {32, 64, 128, 256};
    for (int t : cands) {
      st = launch_class(E, c, nullptr, 0, false, t);
      if (st != PA_OK) return st;
      st = launch_class(E, c, nullptr, 0, true, t);
      if (st != PA_OK) return st;
    }
  }
  // beta = 0 population (Sec. 2)
  st = engine_init_population(E);
  if (st != PA_OK) return st;
  PA_CUDA(cudaStreamSynchronize(E.st));
  return PA_OK;
}

// Enqueue one annealing step for all runs of the engine.
// Reweighting factors, Q', ln Q and the Poisson means of the coming step
// (staged, not committed).
static int engine_prep(Engine& E, bool ovr, double beta, int theta, int64_t Rt) {
  if (E.model == 1) {
    // Q' over replicas: set-up, per-chunk weights, chunk-ordered sum
    PA_CUDA(launch_gprep_head(E.d_runs, nullptr, E.n, ovr, beta, theta, Rt, E.st));
    PA_CUDA(launch_gweights(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
    PA_CUDA(launch_gprep_tail(E.d_runs, nullptr, E.n, E.st));
    E.launches += 2;
  } else {
    PA_CUDA(launch_prepare(E.d_runs, nullptr, E.n, ovr, beta, theta, Rt, E.st));
  }
  return PA_OK;
}

static int engine_step(Engine& E, bool ovr, double beta, int theta, int64_t Rt) {
  int pst = engine_prep(E, ovr, beta, theta, Rt);
  if (pst != PA_OK) return pst;
  PA_CUDA(launch_copies(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  PA_CUDA(launch_scan(E.d_runs, nullptr, E.n, E.st));
  PA_CUDA(launch_scatter(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  for (auto& c : E.cls) {
    cudaEvent_t a = nullptr, b = nullptr;
    const bool timed = E.prof && (E.prof_seen++ % E.prof_stride) == 0;
    // in a stream capture an event record becomes a node of the graph only
    // with the external flag (without it, it only orders captured work)
    const unsigned rec_flags = E.capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) {
      PA_CUDA(cudaEventCreate(&a));
      PA_CUDA(cudaEventCreate(&b));
      PA_CUDA(cudaEventRecordWithFlags(a, E.st, rec_flags));
    }
    int st = launch_class(E, c, c.d_table, c.nwork, false, c.tpb);
    if (st != PA_OK) return st;
    if (timed) {
      PA_CUDA(cudaEventRecordWithFlags(b, E.st, rec_flags));
      (E.capturing ? E.graph_ev : E.prof_ev).push_back({a, b});
    }
  }
  PA_CUDA(launch_commit(E.d_runs, nullptr, E.n, E.st));
  E.launches += 5 + (int64_t)E.cls.size();
  E.host_steps += 1;
  return PA_OK;
}

// Fresh beta = 0 population for every run (Sec. 2), on existing buffers.
static int engine_init_population(Engine& E) {
  PA_CUDA(launch_init_state(E.d_runs, nullptr, E.n, E.max_bins, E.st));
  for (auto& c : E.cls) {
    int st = launch_class(E, c, c.d_table, c.nwork, true, c.tpb);
    if (st != PA_OK) return st;
  }
  PA_CUDA(launch_init_finish(E.d_runs, nullptr, E.n, E.st));
  E.launches += 3 + (int64_t)E.cls.size();
  return PA_OK;
}

static int engine_fetch(Engine& E, std::vector<RunDev>& out) {
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  E.harvest_graph_timing();
  out.resize(E.n);
  PA_CUDA(cudaMemcpy(out.data(), E.d_runs, sizeof(RunDev) * E.n, cudaMemcpyDeviceToHost));
  return PA_OK;
}

static int engine_sync(Engine& E, int32_t* errors) {
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  int first = PA_OK;
  for (int r = 0; r < E.n; ++r) {
    if (errors) errors[r] = d[r].error;
    if (first == PA_OK && d[r].error != 0) first = d[r].error;
  }
  if (first != PA_OK) return fail(first, "device: %s", err_name(first));
  return PA_OK;
}

static int engine_copy_spins(Engine& E, int r, int8_t* host_dst, int64_t max_replicas, int64_t* n) {
  std::vector<RunDev> d;
  int st = engine_fetch(E, d);
  if (st != PA_OK) return st;
  const int64_t cnt = std::min<int64_t>(d[r].R, max_replicas);
  if (n) *n = cnt;
  if (cnt <= 0) return PA_OK;
  const size_t bytes = (size_t)cnt * d[r].N;
  int8_t* tmp = (int8_t*)E.dalloc(bytes);
  if (!tmp) return fail(PA_ERR_OOM, "scratch for spin copy refused");
  cudaError_t e = launch_unpack(E.d_runs, r, cnt, tmp, E.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_dst, tmp, bytes, cudaMemcpyDeviceToHost, E.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(E.st);
  E.dfree(tmp, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "spin copy");
  return PA_OK;
}

// The next n_steps annealing steps of every run of an engine, the schedule
// uploaded to the device; with use_graph the steps are captured once as one
// CUDA graph (kept while the step count and the timing stride stay the
// same) and replayed.
static int engine_run_schedule(Engine& E, int n_steps, const double* betas, int per_run, const int32_t* thetas,
                               const int64_t* R_targets, int use_graph) {
  if (E.host_steps + n_steps > E.max_steps)
    return fail(PA_ERR_INVALID, "schedule exceeds max_steps (%d)", E.max_steps);
  PA_CUDA(cudaSetDevice(E.device));
  // validate and upload the schedule segment of every run
  std::vector<double> bb(n_steps), last(E.n);
  std::vector<int32_t> tt(n_steps);
  std::vector<int64_t> rr(n_steps);
  for (int r = 0; r < E.n; ++r) {  // every run is checked before anything is uploaded
    double prev = E.host_beta[r];
    for (int k = 0; k < n_steps; ++k) {
      const size_t idx = per_run ? (size_t)r * n_steps + k : (size_t)k;
      const double bk = betas[idx];
      const int32_t tk = thetas ? thetas[idx] : 10;
      const int64_t rk = R_targets ? R_targets[idx] : E.R0[r];
      if (!(bk >= prev) || !std::isfinite(bk) || tk < 0 || rk < 1)
        return fail(PA_ERR_INVALID, "run %d step %d: bad schedule entry", r, k);
      prev = bk;
    }
    last[r] = prev;
  }
  for (int r = 0; r < E.n; ++r) {
    for (int k = 0; k < n_steps; ++k) {
      const size_t idx = per_run ? (size_t)r * n_steps + k : (size_t)k;
      bb[k] = betas[idx];
      tt[k] = thetas ? thetas[idx] : 10;
      rr[k] = R_targets ? R_targets[idx] : E.R0[r];
    }
    const RunDev& D = E.h[r];
    const int64_t o = E.host_steps;
    PA_CUDA(cudaMemcpyAsync(D.sched_beta + o, bb.data(), 8 * (size_t)n_steps, cudaMemcpyHostToDevice, E.st));
    PA_CUDA(cudaMemcpyAsync(D.sched_theta + o, tt.data(), 4 * (size_t)n_steps, cudaMemcpyHostToDevice, E.st));
    PA_CUDA(cudaMemcpyAsync(D.sched_R + o, rr.data(), 8 * (size_t)n_steps, cudaMemcpyHostToDevice, E.st));
    E.host_beta[r] = last[r];
  }
  std::vector<int32_t> ns(1, (int32_t)(E.host_steps + n_steps));
  for (int r = 0; r < E.n; ++r)
    PA_CUDA(cudaMemcpyAsync(&E.d_runs[r].n_sched, ns.data(), sizeof(int32_t), cudaMemcpyHostToDevice, E.st));
  // the uploads above are from pageable memory; make sure they landed (and
  // read the timing of a replay still pending)
  PA_CUDA(cudaStreamSynchronize(E.st));
  E.harvest_graph_timing();
  if (!use_graph) {
    for (int k = 0; k < n_steps; ++k) {
      int st = engine_step(E, false, 0.0, 0, 0);
      if (st != PA_OK) return st;
    }
    return PA_OK;
  }
  const int stride = E.prof ? E.prof_stride : 0;
  if (E.graph && (E.graph_steps != n_steps || E.graph_prof_stride != stride)) E.drop_graph();
  if (!E.graph) {
    cudaGraph_t g;
    PA_CUDA(cudaStreamBeginCapture(E.st, cudaStreamCaptureModeThreadLocal));
    int st = PA_OK;
    const int64_t saved = E.host_steps, saved_launches = E.launches, saved_seen = E.prof_seen;
    E.capturing = true;
    E.prof_seen = 0;
    for (int k = 0; k < n_steps && st == PA_OK; ++k) st = engine_step(E, false, 0.0, 0, 0);
    E.capturing = false;
    E.graph_kernels = E.launches - saved_launches;
    E.host_steps = saved;
    E.launches = saved_launches;
    E.prof_seen = saved_seen;
    cudaError_t e = cudaStreamEndCapture(E.st, &g);
    if (st != PA_OK || e != cudaSuccess) {
      if (e == cudaSuccess) cudaGraphDestroy(g);
      E.drop_graph();
      if (st != PA_OK) return st;
      return cuda_fail(e, "graph capture");
    }
    e = cudaGraphInstantiate(&E.graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      E.graph = nullptr;
      E.drop_graph();
      return cuda_fail(e, "graph instantiate");
    }
    E.graph_steps = n_steps;
    E.graph_prof_stride = stride;
  }
  PA_CUDA(cudaGraphLaunch(E.graph, E.st));
  E.launches += E.graph_kernels;
  if (E.prof && !E.graph_ev.empty()) E.graph_pending = true;
  E.host_steps += n_steps;
  return PA_OK;
}

// ---------------------------------------------------------------------------
// C ABI: single runs
// ---------------------------------------------------------------------------
extern "C" {

int pa_version(void) { return 10000; }

int pa_check_exp(int64_t n, uint64_t seed, int64_t* max_ulp_double, int64_t* max_ulp_float) {
  if (n < 0 || !max_ulp_double || !max_ulp_float) return fail(PA_ERR_INVALID, "bad arguments");
  int dev = 0;
  PA_CUDA(cudaGetDevice(&dev));
  int st = ensure_device_constants(dev);
  if (st != PA_OK) return st;
  unsigned long long* d = nullptr;
  PA_CUDA(cudaMalloc(&d, 2 * sizeof *d));
  unsigned long long h[2] = {0ull, 0ull};
  cudaError_t e = cudaMemset(d, 0, 2 * sizeof *d);
  if (e == cudaSuccess) e = launch_check_exp(n, seed, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "exp self-check");
  *max_ulp_double = (int64_t)h[0];
  *max_ulp_float = (int64_t)h[1];
  return PA_OK;
}

int pa_check_philox(int64_t n, uint64_t seed, int64_t* mismatches) {
  if (n < 0 || !mismatches) return fail(PA_ERR_INVALID, "bad arguments");
  unsigned long long* d = nullptr;
  PA_CUDA(cudaMalloc(&d, sizeof *d));
  unsigned long long h = 0ull;
  cudaError_t e = cudaMemset(d, 0, sizeof *d);
  if (e == cudaSuccess) e = launch_check_philox(n, seed, d);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "Philox self-check");
  *mismatches = (int64_t)h;
  return PA_OK;
}

int pa_check_division(int64_t n, uint64_t seed, int64_t* mismatches) {
  if (n < 0 || !mismatches) return fail(PA_ERR_INVALID, "bad arguments");
  int dev = 0;
  PA_CUDA(cudaGetDevice(&dev));
  int st = ensure_device_constants(dev);
  if (st != PA_OK) return st;
  unsigned long long* d = nullptr;
  PA_CUDA(cudaMalloc(&d, sizeof *d));
  unsigned long long hcount = 0ull;
  cudaError_t e = cudaMemset(d, 0, sizeof *d);
  if (e == cudaSuccess) e = launch_check_division(n, seed, d, nullptr);
  if (e == cudaSuccess) e = cudaMemcpy(&hcount, d, sizeof hcount, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "division self-check");
  *mismatches = (int64_t)hcount;
  return PA_OK;
}

const char* pa_last_error(void) { return g_err.c_str(); }

static int create_single(const void* couplings, int L, int dim, int64_t R0, uint64_t seed, const pa_opts* opts,
                         int model, pa_run** out) {
  if (!out) return fail(PA_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  pa_run_spec s;
  memset(&s, 0, sizeof s);
  s.dim = dim;
  s.L = L;
  s.couplings = model ? nullptr : (const int8_t*)couplings;
  s.gauss_couplings = model ? (const int32_t*)couplings : nullptr;
  s.R0 = R0;
  s.seed = seed;
  s.R_cap = opts ? opts->R_cap : 0;
  pa_run* run = new (std::nothrow) pa_run();
  if (!run) return fail(PA_ERR_OOM, "host allocation");
  int st = engine_create(run->e, 1, &s, opts);
  if (st != PA_OK) {
    std::string msg = g_err;
    run->e.release();
    delete run;
    g_err = msg;
    return st;
  }
  *out = run;
  g_err.clear();
  return PA_OK;
}

int pa_create_ex(const int8_t* couplings, int L, int dim, int64_t R0, uint64_t seed, const pa_opts* opts,
                 pa_run** out) {
  return create_single(couplings, L, dim, R0, seed, opts, 0, out);
}

static bool cubic_kernel_for(int model, int L) {
  return model == 1 ? have_gauss_kernel(L) : have_3d_kernel(L);
}

static int create_lattice(const void* couplings, int model, const int Ls[3], int dim, unsigned mask, int64_t R0,
                          uint64_t seed, const pa_opts* opts, pa_run** out) {
  if (!out) return fail(PA_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  if (!couplings || !Ls) return fail(PA_ERR_INVALID, "couplings and extents must not be NULL");
  if (dim == 1) {
    // a chain: the wrap coupling J[N-1] of an open chain becomes 0
    const int N = Ls[0];
    if (N < 2) return fail(PA_ERR_INVALID, "chain length %d must be >= 2", N);
    if (mask & 1u) return create_single(couplings, N, 1, R0, seed, opts, model, out);
    if (model == 1) {
      std::vector<int32_t> J((const int32_t*)couplings, (const int32_t*)couplings + N);
      J[N - 1] = 0;
      return create_single(J.data(), N, 1, R0, seed, opts, 1, out);
    }
    std::vector<int8_t> J((const int8_t*)couplings, (const int8_t*)couplings + N);
    J[N - 1] = 0;
    return create_single(J.data(), N, 1, R0, seed, opts, 0, out);
  }
  if (dim != 3) return fail(PA_ERR_INVALID, "dim must be 1 or 3 (got %d)", dim);
  if (Ls[0] == Ls[1] && Ls[1] == Ls[2] && (mask & 7u) == 7u && cubic_kernel_for(model, Ls[0]))
    return create_single(couplings, Ls[0], 3, R0, seed, opts, model, out);
  pa_run_spec s;
  memset(&s, 0, sizeof s);
  s.dim = 3;
  s.L = Ls[0];
  s.couplings = model ? nullptr : (const int8_t*)couplings;
  s.gauss_couplings = model ? (const int32_t*)couplings : nullptr;
  s.R0 = R0;
  s.seed = seed;
  s.R_cap = opts ? opts->R_cap : 0;
  s.Ls[0] = Ls[0];
  s.Ls[1] = Ls[1];
  s.Ls[2] = Ls[2];
  s.periodic_mask = mask;
  pa_run* run = new (std::nothrow) pa_run();
  if (!run) return fail(PA_ERR_OOM, "host allocation");
  int st = engine_create(run->e, 1, &s, opts);
  if (st != PA_OK) {
    std::string msg = g_err;
    run->e.release();
    delete run;
    g_err = msg;
    return st;
  }
  *out = run;
  g_err.clear();
  return PA_OK;
}

int pa_create_lattice(const int8_t* couplings, const int Ls[3], int dim, unsigned periodic_mask, int64_t R0,
                      uint64_t seed, const pa_opts* opts, pa_run** out) {
  return create_lattice(couplings, 0, Ls, dim, periodic_mask, R0, seed, opts, out);
}

int pa_create_lattice_gauss(const int32_t* couplings, const int Ls[3], int dim, unsigned periodic_mask, int64_t R0,
                            uint64_t seed, const pa_opts* opts, pa_run** out) {
  return create_lattice(couplings, 1, Ls, dim, periodic_mask, R0, seed, opts, out);
}

int pa_create_gauss(const int32_t* couplings, int L, int dim, int64_t R0, uint64_t seed, const pa_opts* opts,
                    pa_run** out) {
  return create_single(couplings, L, dim, R0, seed, opts, 1, out);
}

int pa_create(const int8_t* couplings, int L, int dim, int64_t R0, uint64_t seed, pa_run** out) {
  return pa_create_ex(couplings, L, dim, R0, seed, nullptr, out);
}

void pa_destroy(pa_run* run) {
  if (!run) return;
  cudaSetDevice(run->e.device);
  run->e.release();
  delete run;
}

int pa_reset(pa_run* run, uint64_t seed) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  Engine& E = run->e;
  PA_CUDA(cudaSetDevice(E.device));
  // the seed lives in the device run table; patch it there in stream order
  E.h[0].seed = seed;
  PA_CUDA(cudaMemcpyAsync(&E.d_runs[0].seed, &E.h[0].seed, sizeof(uint64_t), cudaMemcpyHostToDevice, E.st));
  PA_CUDA(cudaMemcpyAsync(&E.d_runs[0].R, &E.R0[0], sizeof(int64_t), cudaMemcpyHostToDevice, E.st));
  int st = engine_init_population(E);
  if (st != PA_OK) return st;
  E.host_beta[0] = 0.0;
  E.host_steps = 0;
  return PA_OK;
}

int pa_kernel_time(pa_run* run, int enable, double* sweep_ms, int64_t* sweep_launches,
                   int64_t* kernel_launches) {
  if (!run || enable < 0) return fail(PA_ERR_INVALID, "bad kernel-timing arguments");
  Engine& E = run->e;
  PA_CUDA(cudaSetDevice(E.device));
  if (enable) {
    PA_CUDA(cudaStreamSynchronize(E.st));
    for (auto& p : E.prof_ev) {
      cudaEventDestroy(p.first);
      cudaEventDestroy(p.second);
    }
    E.prof_ev.clear();
    E.launches = 0;
    E.prof = true;
    E.prof_stride = enable;
    E.prof_seen = 0;
    E.prof_ms_acc = 0.0;
    E.prof_n_acc = 0;
    E.graph_pending = false;
    return PA_OK;
  }
  PA_CUDA(cudaStreamSynchronize(E.st));
  E.harvest_graph_timing();
  double total = E.prof_ms_acc;
  for (auto& p : E.prof_ev) {
    float ms = 0.f;
    PA_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
    total += ms;
  }
  if (sweep_ms) *sweep_ms = total;
  if (sweep_launches) *sweep_launches = (int64_t)E.prof_ev.size() + E.prof_n_acc;
  if (kernel_launches) *kernel_launches = E.launches;
  E.prof_seen = 0;
  E.prof_ms_acc = 0.0;
  E.prof_n_acc = 0;
  for (auto& p : E.prof_ev) {
    cudaEventDestroy(p.first);
    cudaEventDestroy(p.second);
  }
  E.prof_ev.clear();
  E.prof = false;
  return PA_OK;
}

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
    if (st != PA_OK) return fail(st, "run %d: %s", r, g_err.c_str());
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

int pa_step_target(pa_run* run, double beta_next, int sweeps, int64_t R_target) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  if (sweeps < 0) return fail(PA_ERR_INVALID, "sweeps must be >= 0");
  if (R_target < 1) return fail(PA_ERR_INVALID, "R_target must be >= 1");
  if (!(beta_next >= run->e.host_beta[0]) || !std::isfinite(beta_next))
    return fail(PA_ERR_INVALID, "beta must not decrease (%g after %g)", beta_next, run->e.host_beta[0]);
  PA_CUDA(cudaSetDevice(run->e.device));
  int st = engine_step(run->e, true, beta_next, sweeps, R_target);
  if (st != PA_OK) return st;
  run->e.host_beta[0] = beta_next;
  return PA_OK;
}

int pa_run_schedule(pa_run* run, int n_steps, const double* betas, const int32_t* thetas, const int64_t* R_targets,
                    int use_graph) {
  if (!run || !betas || n_steps < 0) return fail(PA_ERR_INVALID, "bad schedule arguments");
  return engine_run_schedule(run->e, n_steps, betas, 0, thetas, R_targets, use_graph);
}

int pa_step(pa_run* run, double beta_next, int sweeps) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  return pa_step_target(run, beta_next, sweeps, run->e.R0[0]);
}

int pa_sync(pa_run* run) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  return engine_sync(run->e, nullptr);
}

int pa_observables(pa_run* run, pa_obs* o) {
  if (!run || !o) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  const RunDev& R = d[0];
  o->beta = R.beta;
  o->R = R.R;
  if (R.model == 1) {
    o->E_mean = (double)R.sumE * 0x1.0p-15 / (double)R.R;
    o->E2_mean = R.sumE2d / (double)R.R;
  } else {
    o->E_mean = (double)R.sumE / (double)R.R;
    o->E2_mean = (double)R.sumE2 / (double)R.R;
  }
  o->lnQ_last = R.lnQ_last;
  o->minus_beta_F = R.mbF;
  o->step = R.step;
  o->sweeps = R.sweeps;
  o->sumE = R.sumE;
  o->sumE2 = R.model == 1 ? 0 : R.sumE2;
  if (R.error) return fail(R.error, "device: %s", err_name(R.error));
  return PA_OK;
}

int pa_free_energy(pa_run* run, double* minus_beta_F) {
  pa_obs o;
  int st = pa_observables(run, &o);
  if (minus_beta_F) *minus_beta_F = o.minus_beta_F;
  return st;
}

int pa_trajectory(pa_run* run, int64_t count, double* beta, double* lnQ, double* mbF, int64_t* R,
                  int64_t* sumE, int64_t* sumE2, int64_t* n) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  const RunDev& D = d[0];
  const int64_t avail = std::min<int64_t>(D.step, D.max_steps) + 1;
  const int64_t c = std::min<int64_t>(count, avail);
  if (n) *n = c;
  if (c > 0) {
    if (beta) PA_CUDA(cudaMemcpy(beta, D.rec_beta, 8 * c, cudaMemcpyDeviceToHost));
    if (lnQ) PA_CUDA(cudaMemcpy(lnQ, D.rec_lnQ, 8 * c, cudaMemcpyDeviceToHost));
    if (mbF) PA_CUDA(cudaMemcpy(mbF, D.rec_mbF, 8 * c, cudaMemcpyDeviceToHost));
    if (R) PA_CUDA(cudaMemcpy(R, D.rec_R, 8 * c, cudaMemcpyDeviceToHost));
    if (sumE) PA_CUDA(cudaMemcpy(sumE, D.rec_sumE, 8 * c, cudaMemcpyDeviceToHost));
    if (sumE2) {
      if (D.model == 1) memset(sumE2, 0, 8 * c);
      else PA_CUDA(cudaMemcpy(sumE2, D.rec_sumE2, 8 * c, cudaMemcpyDeviceToHost));
    }
  }
  if (D.error) return fail(D.error, "device: %s", err_name(D.error));
  return PA_OK;
}

int pa_trajectory_energy(pa_run* run, int64_t count, double* E_mean, double* E2_mean, int64_t* n) {
  if (!run) return fail(PA_ERR_INVALID, "run is NULL");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  const RunDev& D = d[0];
  const int64_t avail = std::min<int64_t>(D.step, D.max_steps) + 1;
  const int64_t c = std::max<int64_t>(0, std::min<int64_t>(count, avail));
  if (n) *n = c;
  std::vector<int64_t> R(c), s1(c), s2(c);
  if (c > 0) {
    PA_CUDA(cudaMemcpy(R.data(), D.rec_R, 8 * c, cudaMemcpyDeviceToHost));
    PA_CUDA(cudaMemcpy(s1.data(), D.rec_sumE, 8 * c, cudaMemcpyDeviceToHost));
    PA_CUDA(cudaMemcpy(s2.data(), D.rec_sumE2, 8 * c, cudaMemcpyDeviceToHost));
  }
  for (int64_t k = 0; k < c; ++k) {
    double e2;
    if (D.model == 1) memcpy(&e2, &s2[k], 8);  // the record holds the physical sum's bits
    else e2 = (double)s2[k];
    const double unit = D.model == 1 ? 0x1.0p-15 : 1.0;
    if (E_mean) E_mean[k] = (double)s1[k] * unit / (double)R[k];
    if (E2_mean) E2_mean[k] = e2 / (double)R[k];
  }
  if (D.error) return fail(D.error, "device: %s", err_name(D.error));
  return PA_OK;
}

int pa_copy_spins(pa_run* run, int8_t* host_dst, int64_t max_replicas, int64_t* n) {
  if (!run || !host_dst) return fail(PA_ERR_INVALID, "NULL argument");
  return engine_copy_spins(run->e, 0, host_dst, max_replicas, n);
}

int pa_copy_energies(pa_run* run, int32_t* host_dst, int64_t max_replicas, int64_t* n) {
  if (!run || !host_dst) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  const int64_t c = std::min<int64_t>(d[0].R, max_replicas);
  if (n) *n = c;
  if (c > 0) PA_CUDA(cudaMemcpy(host_dst, d[0].E[d[0].cur], 4 * c, cudaMemcpyDeviceToHost));
  return PA_OK;
}

int pa_copy_copies(pa_run* run, int32_t* host_dst, int64_t max_replicas, int64_t* n) {
  if (!run || !host_dst) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> d;
  int st = engine_fetch(run->e, d);
  if (st != PA_OK) return st;
  const RunDev& D = d[0];
  int64_t prev = 0;
  if (D.step >= 1 && D.step - 1 <= D.max_steps) PA_CUDA(cudaMemcpy(&prev, D.rec_R + (D.step - 1), 8, cudaMemcpyDeviceToHost));
  const int64_t c = std::min<int64_t>(prev, max_replicas);
  if (n) *n = c;
  if (c > 0) PA_CUDA(cudaMemcpy(host_dst, D.copies, 4 * c, cudaMemcpyDeviceToHost));
  return PA_OK;
}

int pa_overlap(pa_run* a, pa_run* b, double qcut, double* gamma, int64_t* npairs, int64_t* hist) {
  if (!a || !b || !gamma) return fail(PA_ERR_INVALID, "NULL argument");
  std::vector<RunDev> da, db;
  int st = engine_fetch(a->e, da);
  if (st != PA_OK) return st;
  st = engine_fetch(b->e, db);
  if (st != PA_OK) return st;
  if (a->e.device != b->e.device) return fail(PA_ERR_INVALID, "runs live on different GPUs");
  if (da[0].dim != db[0].dim || da[0].L != db[0].L) return fail(PA_ERR_INVALID, "runs differ in lattice");
  const int N = da[0].N;
  const size_t bytes = 8 * (size_t)(N + 2);
  unsigned long long* buf = (unsigned long long*)a->e.dalloc(bytes);  // run a's allocator
  if (!buf) return fail(PA_ERR_OOM, "overlap scratch refused");
  cudaError_t e = cudaMemsetAsync(buf, 0, bytes, a->e.st);
  if (e == cudaSuccess) e = launch_overlap(a->e.d_runs, b->e.d_runs, qcut, buf, buf + 1, a->e.st);
  std::vector<unsigned long long> hb(N + 2);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hb.data(), buf, bytes, cudaMemcpyDeviceToHost, a->e.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(a->e.st);
  a->e.dfree(buf, bytes);
  if (e != cudaSuccess) return cuda_fail(e, "overlap");
  const int64_t np = std::min(da[0].R, db[0].R);
  if (npairs) *npairs = np;
  *gamma = np > 0 ? (double)hb[0] / (double)np : 0.0;
  if (hist)
    for (int k = 0; k <= N; ++k) hist[k] = (int64_t)hb[1 + k];
  return PA_OK;
}

// ---------------------------------------------------------------------------
// Sec. 3 weighted averages and bootstrap
// ---------------------------------------------------------------------------
int pa_weighted_average_dev(int G, int M, const double* x_dev, const double* A_dev, const double* R_dev,
                            double* mean_dev, double* fbar_dev, void* stream) {
  if (G < 1 || M < 1 || !x_dev || !mean_dev || !fbar_dev) return fail(PA_ERR_INVALID, "bad weighted-average arguments");
  int dev;
  PA_CUDA(cudaGetDevice(&dev));
  PA_CUDA(launch_weighted(G, M, x_dev, A_dev, R_dev, mean_dev, fbar_dev, (cudaStream_t)stream));
  return PA_OK;
}

static int stage_inputs(int M, const double* x, const double* A, const double* R, double** buf, cudaStream_t st,
                        size_t extra) {
  const size_t bytes = 8 * (3 * (size_t)M + extra);
  PA_CUDA(cudaMallocAsync((void**)buf, bytes, st));
  PA_CUDA(cudaMemcpyAsync(*buf, x, 8 * M, cudaMemcpyHostToDevice, st));
  if (A) PA_CUDA(cudaMemcpyAsync(*buf + M, A, 8 * M, cudaMemcpyHostToDevice, st));
  if (R) PA_CUDA(cudaMemcpyAsync(*buf + 2 * M, R, 8 * M, cudaMemcpyHostToDevice, st));
  return PA_OK;
}

int pa_weighted_average(int M, const double* x, const double* A, const double* R, double* mean, double* fbar) {
  if (M < 1 || !x) return fail(PA_ERR_INVALID, "bad weighted-average arguments");
  if (R)
    for (int r = 0; r < M; ++r)
      if (!(R[r] > 0.0)) return fail(PA_ERR_INVALID, "R weights must be positive");
  cudaStream_t st = nullptr;
  double* buf = nullptr;
  int s = stage_inputs(M, x, A, R, &buf, st, 2);
  if (s != PA_OK) return s;
  cudaError_t e = launch_weighted(1, M, buf, A ? buf + M : nullptr, R ? buf + 2 * M : nullptr, buf + 3 * M,
                                  buf + 3 * M + 1, st);
  double out[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf + 3 * M, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "weighted average");
  if (mean) *mean = out[0];
  if (fbar) *fbar = out[1];
  return PA_OK;
}

static double sample_std(const std::vector<double>& v) {
  const size_t n = v.size();
  if (n < 2) return 0.0;
  double m = 0.0;
  for (double x : v) m += x;
  m /= (double)n;
  double s = 0.0;
  for (double x : v) s += (x - m) * (x - m);
  return std::sqrt(s / (double)(n - 1));
}

int pa_bootstrap(int M, const double* x, const double* A, const double* R, int B, uint64_t seed, double* std_mean,
                 double* std_fbar) {
  if (M < 1 || B < 2 || !x) return fail(PA_ERR_INVALID, "bad bootstrap arguments");
  cudaStream_t st = nullptr;
  double* buf = nullptr;
  int s = stage_inputs(M, x, A, R, &buf, st, 2 * (size_t)B);
  if (s != PA_OK) return s;
  cudaError_t e = launch_bootstrap(M, buf, A ? buf + M : nullptr, R ? buf + 2 * M : nullptr, B, seed, buf + 3 * M,
                                   buf + 3 * M + B, st);
  std::vector<double> bm(B), bf(B);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bm.data(), buf + 3 * M, 8 * B, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(bf.data(), buf + 3 * M + B, 8 * B, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "bootstrap");
  if (std_mean) *std_mean = sample_std(bm);
  if (std_fbar) *std_fbar = sample_std(bf);
  return PA_OK;
}

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
    std::string msg = g_err;
    b->e.release();
    delete b;
    g_err = msg;
    return st;
  }
  *out = b;
  g_err.clear();
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

int pa_batch_copy_spins(pa_batch* b, int r, int8_t* host_dst, int64_t max_replicas, int64_t* n) {
  if (!b || !host_dst || r < 0 || r >= b->e.n) return fail(PA_ERR_INVALID, "bad arguments");
  return engine_copy_spins(b->e, r, host_dst, max_replicas, n);
}

int pa_batch_autotune(pa_batch* b, int32_t* host_L, int32_t* host_tpb, int* n_out) {
  if (!b) return fail(PA_ERR_INVALID, "batch is NULL");
  Engine& E = b->e;
  PA_CUDA(cudaSetDevice(E.device));
  // Dry step at the current temperature: prepare/copies/scan/scatter fill the
  // staged population; each candidate sweep launch reads the unchanged
  // population and writes only the spare buffer; nothing is committed.
  int pst = engine_prep(E, true, -1.0, 2, -1);
  if (pst != PA_OK) return pst;
  PA_CUDA(launch_copies(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  PA_CUDA(launch_scan(E.d_runs, nullptr, E.n, E.st));
  PA_CUDA(launch_scatter(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  cudaEvent_t t0, t1;
  PA_CUDA(cudaEventCreate(&t0));
  PA_CUDA(cudaEventCreate(&t1));
  int count = 0;
  for (auto& c : E.cls) {
    const int cands3[] = {32, 64, 128};
    const int cands1[] = {32, 64, 128};
    const int* cands = c.dim == 1 ? cands1 : cands3;
    float best = 1e30f;
    int best_tpb = c.tpb;
    LatticeClass trial = c;
    for (int i = 0; i < 3; ++i) {
      if (cands[i] > c.max_tpb) continue;
      trial.tpb = cands[i];
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
      if (ms < best) {
        best = ms;
        best_tpb = cands[i];
      }
    }
    if (best_tpb != c.tpb) {
      c.tpb = best_tpb;
      int st = build_class_table(E, c);
      if (st != PA_OK) return st;
    }
    if (count < 8) {
      if (host_L) host_L[count] = c.dim == 1 ? -c.L : c.L;
      if (host_tpb) host_tpb[count] = c.tpb;
      ++count;
    }
  }
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  E.drop_graph();  // the block sizes changed
  if (n_out) *n_out = count;
  return PA_OK;
}

}  // extern "C"

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
  int max_runs = 0, max_steps = 0, tpb_opt = 0;
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
      c.tpb = S->tpb_opt ? S->tpb_opt : default_tpb(d.dim, d.L);
      S->cls.push_back(c);
      S->cls_buf.push_back(DevBuf());
      S->init_buf.push_back(DevBuf());
      for (int t : {32, 64, 128, 256}) {  // shared-memory limits, outside any capture
        int st = launch_class_on(S->d_runs, S->st, c, nullptr, 0, false, t);
        if (st != PA_OK) return st;
        st = launch_class_on(S->d_runs, S->st, c, nullptr, 0, true, t);
        if (st != PA_OK) return st;
      }
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
    if (!mem) break;  // retry on a later tick
    RunDev d;
    st = setup_run((char*)mem, q.geo, q.spec, q.cap, S->max_steps, S->st, &d);
    if (st != PA_OK) return st;
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

int pa_server_result(pa_server* S, int64_t id, pa_result* out, double* traj, int64_t count) {
  if (!S || !out) return fail(PA_ERR_INVALID, "bad arguments");
  auto it = S->reqs.find(id);
  if (it == S->reqs.end()) return fail(PA_ERR_INVALID, "unknown request %lld", (long long)id);
  const ServerReq& q = it->second;
  memset(out, 0, sizeof *out);
  out->status = q.status;
  out->error = q.error;
  out->steps = q.status >= 2 ? q.last.step : q.steps_done;
  out->submit_s = q.t_submit;
  out->admit_s = q.t_admit;
  out->done_s = q.t_done;
  out->device_bytes = (int64_t)q.bytes;
  out->flips = q.flips;
  if (q.status >= 2) {
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
