// pa_engine.cu -- host runtime behind the C ABI of include/pa.h: errors,
// geometry, the Engine, single runs and the Sec. 3 averages (checkpoints in
// pa_checkpoint.cu, batches in pa_batch.cu, serving in pa_server.cu; the
// declarations they share in pa_engine.h).
//
// An Engine owns a set of annealing runs on one GPU: one device-memory slab
// per run, the RunDev array, and the work tables that map kernel blocks to
// (run, slot range).  Single runs (pa_run) and batches (pa_batch) are both
// Engines; every step enqueues the same seven launches (prepare, copies,
// scan, scatter, one sweep launch per lattice class, commit) with no host
// synchronisation, so a batch schedule can be captured as one CUDA graph.
#include "pa_engine.h"


// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(PA_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}



const char* err_name(int code) {
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

int ensure_device_constants(int dev) {
  std::lock_guard<std::mutex> lk(g_coef_mu);
  if (dev < 0 || dev >= 64) return fail(PA_ERR_CUDA, "device index %d out of range", dev);
  if (!g_coef_ready[dev]) {
    PA_CUDA(set_exp_coefficients());
    g_coef_ready[dev] = true;
  }
  return PA_OK;
}
const char* last_error_message() { return g_err.c_str(); }
void clear_last_error() { g_err.clear(); }


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

int make_geometry(const int8_t* J, int L, int dim, Geometry* g) {
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

int64_t default_capacity(int64_t R0) {
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

size_t run_slab_bytes(const Geometry& g, int64_t cap, int max_steps) {
  RunDev d;
  return slab_parts(d, g, cap, max_steps, nullptr);
}

// Carve the slab, upload the couplings, build the coupling masks and fill the
// static part of the run record (population not yet initialised).
int setup_run(char* base, const Geometry& g, const pa_run_spec& s, int64_t cap, int max_steps,
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

int default_tpb(int dim, int L) {
  if (dim == 1) return 64;
  return L >= 12 ? 64 : 128;
}

// Block sizes the sweep kernels of a class support: 32 .. 256 threads for
// every class (general boxes and Gaussian chains up to what their
// shared-memory tables allow);
// 512 and 1024 too for Gaussian cubic lattices of L <= 8, whose kernel at
// those sizes tabulates the acceptance thresholds of every site and pattern
// in shared memory (the table is shared by all the block's replicas).
bool tpb_supported(const LatticeClass& c, int tpb) {
  if (tpb == 32 || tpb == 64 || tpb == 128 || tpb == 256) {
    if (c.bx > 0) return tpb <= c.max_tpb;
    if (c.dim == 1 && c.model == 1) return gauss1d_smem_bytes(tpb, c.Wr) <= SMEM_LIMIT;
    return true;
  }
  if (tpb == 512 || tpb == 1024) return c.bx == 0 && c.dim == 3 && c.model == 1 && c.L <= 8;
  return false;
}

// Block size and threads per replica of a class before any autotuning: the
// cubic sweeps run 4 threads per replica where the rows split so, which keeps
// enough warps resident to hide the latency of the generator's dependent
// multiplies; +-1 chains 4 or 8 on ranges of words; other classes 1.
void set_default_launch(LatticeClass& c, int tpb_opt, int split_opt) {
  c.split = 1;
  if (split_opt > 0) {
    c.split = split_supported(c, split_opt) ? split_opt : 1;
  } else if (c.dim == 3 && c.bx == 0 && c.model == 1 && c.L <= 8) {
    // the threshold-table kernel: 512 threads, two per replica (one block per
    // SM; measured the fastest shape for a single run of 1e5 replicas)
    if (split_supported(c, 2)) c.split = 2;
  } else if (c.dim == 3 && c.bx == 0) {
    if (split_supported(c, 4)) c.split = 4;
  } else if (c.dim == 1 && c.model == 0) {
    // +-1 chains: the word ranges keep the uniform tables and the columns of
    // a block within shared memory at long chains
    c.split = c.Wr >= 16 ? 8 : (c.Wr >= 4 ? 4 : 1);
  }
  if (tpb_opt && tpb_supported(c, tpb_opt)) c.tpb = tpb_opt;
  else if (c.bx > 0) c.tpb = std::min(64, c.max_tpb);
  else if (c.dim == 3 && c.model == 1 && c.L <= 8) c.tpb = 512;
  else if (c.split > 1) c.tpb = (c.dim == 3 && c.L == 16) ? 64 : 128;
  else c.tpb = default_tpb(c.dim, c.L);
  if (c.tpb / c.split < 4 || (c.split > 1 && c.tpb < 64)) c.split = 1;
}

bool split_supported(const LatticeClass& c, int split) {
  if (c.bx != 0) return split == 1;
  if (c.dim == 1) return c.model == 0 ? sweep1d_split_ok(split) : split == 1;
  if (c.model == 1) {
    switch (c.L) {
      case 4: return gauss3d_split_ok_L4(split);
      case 6: return gauss3d_split_ok_L6(split);
      case 8: return gauss3d_split_ok_L8(split);
      case 10: return gauss3d_split_ok_L10(split);
      case 12: return gauss3d_split_ok_L12(split);
      default: return split == 1;
    }
  }
  switch (c.L) {
    case 2: return sweep3d_split_ok_L2(split);
    case 4: return sweep3d_split_ok_L4(split);
    case 6: return sweep3d_split_ok_L6(split);
    case 8: return sweep3d_split_ok_L8(split);
    case 10: return sweep3d_split_ok_L10(split);
    case 12: return sweep3d_split_ok_L12(split);
    case 14: return sweep3d_split_ok_L14(split);
    case 16: return sweep3d_split_ok_L16(split);
    default: return split == 1;
  }
}

int launch_class_on(RunDev* runs, cudaStream_t st, const LatticeClass& c, const Work* table, int nwork,
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
      case 4: err = launch_gauss3d_L4(tpb, c.split, runs, table, nwork, st, init); break;
      case 6: err = launch_gauss3d_L6(tpb, c.split, runs, table, nwork, st, init); break;
      case 8: err = launch_gauss3d_L8(tpb, c.split, runs, table, nwork, st, init); break;
      case 10: err = launch_gauss3d_L10(tpb, c.split, runs, table, nwork, st, init); break;
      case 12: err = launch_gauss3d_L12(tpb, c.split, runs, table, nwork, st, init); break;
      default: return fail(PA_ERR_UNSUPPORTED, "no Gaussian kernel for L=%d", c.L);
    }
  } else if (c.dim == 1) {
    err = launch_sweep1d(tpb, c.split, runs, table, nwork, c.W, c.Wr, st, init);
  } else {
    switch (c.L) {
      case 2: err = launch_sweep3d_L2(tpb, c.split, runs, table, nwork, st, init); break;
      case 4: err = launch_sweep3d_L4(tpb, c.split, runs, table, nwork, st, init); break;
      case 6: err = launch_sweep3d_L6(tpb, c.split, runs, table, nwork, st, init); break;
      case 8: err = launch_sweep3d_L8(tpb, c.split, runs, table, nwork, st, init); break;
      case 10: err = launch_sweep3d_L10(tpb, c.split, runs, table, nwork, st, init); break;
      case 12: err = launch_sweep3d_L12(tpb, c.split, runs, table, nwork, st, init); break;
      case 14: err = launch_sweep3d_L14(tpb, c.split, runs, table, nwork, st, init); break;
      case 16: err = launch_sweep3d_L16(tpb, c.split, runs, table, nwork, st, init); break;
      default: return fail(PA_ERR_UNSUPPORTED, "no kernel for L=%d", c.L);
    }
  }
  if (err != cudaSuccess) return cuda_fail(err, "sweep kernel launch");
  return PA_OK;
}

int launch_class(Engine& E, const LatticeClass& c, const Work* table, int nwork, bool init, int tpb) {
  return launch_class_on(E.d_runs, E.st, c, table, nwork, init, tpb);
}

// Set the dynamic shared-memory limits of every block size and every
// supported number of threads per replica of the class now, outside any
// stream capture (the autotuner may pick any of them later).
int prepare_class_launches(RunDev* runs, cudaStream_t st, const LatticeClass& c) {
  LatticeClass t = c;
  for (int split : {1, 2, 4, 8}) {
    if (!split_supported(c, split)) continue;
    t.split = split;
    for (int tpb : {32, 64, 128, 256, 512, 1024}) {
      if (!tpb_supported(c, tpb) || (split > 1 && (tpb < 64 || tpb / split < 4))) continue;
      int s = launch_class_on(runs, st, t, nullptr, 0, false, tpb);
      if (s != PA_OK) return s;
      s = launch_class_on(runs, st, t, nullptr, 0, true, tpb);
      if (s != PA_OK) return s;
    }
  }
  return PA_OK;
}

int build_class_table(Engine& E, LatticeClass& c) {
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

int engine_init_population(Engine& E);

// model 0: specs[r].couplings are int8 (+-1 / 0); model 1: they point to
// int32 fixed-point Gaussian couplings (J = J_q 2^-15).
int engine_create(Engine& E, int n_runs, const pa_run_spec* specs, const pa_opts* opts) {
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
  if (tpb_opt != 0 && tpb_opt != 32 && tpb_opt != 64 && tpb_opt != 128 && tpb_opt != 256 && tpb_opt != 512 &&
      tpb_opt != 1024)
    return fail(PA_ERR_INVALID, "threads_per_block must be 0, 32, 64, 128, 256, 512 or 1024");
  const int split_opt = opts ? opts->threads_per_replica : 0;
  if (split_opt != 0 && split_opt != 1 && split_opt != 2 && split_opt != 4 && split_opt != 8)
    return fail(PA_ERR_INVALID, "threads_per_replica must be 0, 1, 2, 4 or 8");
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
      set_default_launch(c, tpb_opt, split_opt);
      if (split_opt > 1 && c.split != split_opt)
        return fail(PA_ERR_INVALID, "%d threads per replica do not split the rows of this lattice or block",
                    split_opt);
      E.cls.push_back(c);
      it = E.cls.end() - 1;
    }
    it->runs.push_back(r);
  }
  for (auto& c : E.cls) {
    st = build_class_table(E, c);
    if (st != PA_OK) return st;
    st = prepare_class_launches(E.d_runs, E.st, c);
    if (st != PA_OK) return st;
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
int engine_prep(Engine& E, bool ovr, double beta, int theta, int64_t Rt) {
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
  NvtxRange step_range("pa_step");
  int pst;
  {
    NvtxRange r("reweight+Q (k_prepare)");
    pst = engine_prep(E, ovr, beta, theta, Rt);
  }
  if (pst != PA_OK) return pst;
  {
    NvtxRange r("copy counts (k_copies)");
    PA_CUDA(launch_copies(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  }
  {
    NvtxRange r("scan (k_scan)");
    PA_CUDA(launch_scan(E.d_runs, nullptr, E.n, E.st));
  }
  {
    NvtxRange r("replica sources (k_scatter)");
    PA_CUDA(launch_scatter(E.d_runs, E.d_copy_table, E.n_copy_work, E.st));
  }
  NvtxRange sweep_range("gather+sweeps+measure (k_sweep*)");
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
  {
    NvtxRange r("commit (k_commit)");
    PA_CUDA(launch_commit(E.d_runs, nullptr, E.n, E.st));
  }
  E.launches += 5 + (int64_t)E.cls.size();
  E.host_steps += 1;
  return PA_OK;
}

// Fresh beta = 0 population for every run (Sec. 2), on existing buffers.
int engine_init_population(Engine& E) {
  NvtxRange init_range("pa_init");
  PA_CUDA(launch_init_state(E.d_runs, nullptr, E.n, E.max_bins, E.st));
  for (auto& c : E.cls) {
    int st = launch_class(E, c, c.d_table, c.nwork, true, c.tpb);
    if (st != PA_OK) return st;
  }
  PA_CUDA(launch_init_finish(E.d_runs, nullptr, E.n, E.st));
  E.launches += 3 + (int64_t)E.cls.size();
  return PA_OK;
}

int engine_fetch(Engine& E, std::vector<RunDev>& out) {
  PA_CUDA(cudaSetDevice(E.device));
  PA_CUDA(cudaStreamSynchronize(E.st));
  E.harvest_graph_timing();
  out.resize(E.n);
  PA_CUDA(cudaMemcpy(out.data(), E.d_runs, sizeof(RunDev) * E.n, cudaMemcpyDeviceToHost));
  return PA_OK;
}

int engine_sync(Engine& E, int32_t* errors) {
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

int engine_copy_spins(Engine& E, int r, int8_t* host_dst, int64_t max_replicas, int64_t* n) {
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
int engine_run_schedule(Engine& E, int n_steps, const double* betas, int per_run, const int32_t* thetas,
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

int pa_gauss_thresholds(double beta, int64_t n, const int32_t* dE, uint32_t* thr) {
  if (n < 0 || (n > 0 && (!dE || !thr)) || !(beta >= 0.0)) return fail(PA_ERR_INVALID, "bad arguments");
  if (n == 0) return PA_OK;
  int32_t* d_dE = nullptr;
  uint32_t* d_thr = nullptr;
  cudaError_t e = cudaMalloc(&d_dE, sizeof(int32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMalloc(&d_thr, sizeof(uint32_t) * (size_t)n);
  if (e == cudaSuccess) e = cudaMemcpy(d_dE, dE, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_gauss_thresholds(n, beta, d_dE, d_thr);
  if (e == cudaSuccess) e = cudaMemcpy(thr, d_thr, sizeof(uint32_t) * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d_dE);
  cudaFree(d_thr);
  if (e != cudaSuccess) return cuda_fail(e, "Gaussian thresholds");
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

int pa_sweep_shape(pa_run* run, int32_t* threads_per_block, int32_t* threads_per_replica) {
  if (!run || run->e.cls.empty()) return fail(PA_ERR_INVALID, "run is NULL");
  if (threads_per_block) *threads_per_block = run->e.cls[0].tpb;
  if (threads_per_replica) *threads_per_replica = run->e.cls[0].split;
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

// Copies M-element host arrays (NULL ones skipped) into consecutive M-element
// slots of one device buffer of (n_arrays * M + extra) doubles; on failure
// the buffer is released and *buf is NULL.
static int stage_arrays(int M, const double* const* arrays, int n_arrays, double** buf, cudaStream_t st,
                        size_t extra) {
  const size_t bytes = 8 * ((size_t)n_arrays * M + extra);
  *buf = nullptr;
  PA_CUDA(cudaMallocAsync((void**)buf, bytes, st));
  for (int i = 0; i < n_arrays; ++i) {
    if (!arrays[i]) continue;
    const cudaError_t e = cudaMemcpyAsync(*buf + (size_t)i * M, arrays[i], 8 * (size_t)M, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFreeAsync(*buf, st);
      *buf = nullptr;
      return cuda_fail(e, "staging inputs");
    }
  }
  return PA_OK;
}

static int stage_inputs(int M, const double* x, const double* A, const double* R, double** buf, cudaStream_t st,
                        size_t extra) {
  const double* arrays[3] = {x, A, R};
  return stage_arrays(M, arrays, 3, buf, st, extra);
}

static bool all_positive(int M, const double* R) {
  for (int r = 0; r < M; ++r)
    if (!(R[r] > 0.0)) return false;
  return true;
}

int pa_weighted_average(int M, const double* x, const double* A, const double* R, double* mean, double* fbar) {
  if (M < 1 || !x) return fail(PA_ERR_INVALID, "bad weighted-average arguments");
  if (R && !all_positive(M, R)) return fail(PA_ERR_INVALID, "R weights must be positive");
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

int pa_weighted_average_pairs(int M, const double* x1, const double* x2, const double* A, const double* R1,
                              const double* R2, double* mean, double* fbar2) {
  if (M < 1 || !x1 || !x2 || (R1 == nullptr) != (R2 == nullptr))
    return fail(PA_ERR_INVALID, "bad pair weighted-average arguments");
  if (R1 && (!all_positive(M, R1) || !all_positive(M, R2)))
    return fail(PA_ERR_INVALID, "R weights must be positive");
  cudaStream_t st = nullptr;
  double* buf = nullptr;
  const double* arrays[5] = {x1, x2, A, R1, R2};
  int s = stage_arrays(M, arrays, 5, &buf, st, 2);
  if (s != PA_OK) return s;
  cudaError_t e = launch_weighted_pairs(1, M, buf, buf + M, A ? buf + 2 * M : nullptr, R1 ? buf + 3 * M : nullptr,
                                        R1 ? buf + 4 * M : nullptr, buf + 5 * M, buf + 5 * M + 1, st);
  double out[2] = {0, 0};
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, buf + 5 * M, 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(buf, st);
  if (e != cudaSuccess) return cuda_fail(e, "pair weighted average");
  if (mean) *mean = out[0];
  if (fbar2) *fbar2 = out[1];
  return PA_OK;
}

int pa_weighted_average_pairs_dev(int G, int M, const double* x1_dev, const double* x2_dev, const double* A_dev,
                                  const double* R1_dev, const double* R2_dev, double* mean_dev, double* fbar2_dev,
                                  void* stream) {
  if (G < 1 || M < 1 || !x1_dev || !x2_dev || !mean_dev || !fbar2_dev || (R1_dev == nullptr) != (R2_dev == nullptr))
    return fail(PA_ERR_INVALID, "bad pair weighted-average arguments");
  PA_CUDA(launch_weighted_pairs(G, M, x1_dev, x2_dev, A_dev, R1_dev, R2_dev, mean_dev, fbar2_dev,
                                (cudaStream_t)stream));
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
  if (R && !all_positive(M, R)) return fail(PA_ERR_INVALID, "R weights must be positive");
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


}  // extern "C"
